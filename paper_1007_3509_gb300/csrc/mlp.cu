// Learned field surrogate: 11 -> 64 -> 64 -> 64 -> 2 perceptron with GELU,
// BF16 operands and FP32 accumulation on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory).  It stands in for the
// per-material-point crystal plasticity of Sec. 2 (elastic energy density and
// dislocation energy, Eq. (4)) when the driving field is refreshed.
//
// Parameters (FP32 master copy, one buffer, this order):
//   W1 [64][11], b1[64], W2 [64][64], b2[64], W3 [64][64], b3[64], W4 [2][64], b4[2]
// Forward:  h_l = bf16(GELU(h_{l-1} W_l^T + b_l)), y = h_3 W4^T + b4, with x,
// W and h rounded to BF16 and every sum accumulated in FP32.
// Training: L = 1/(2B) sum (y - t)^2; dz_l = (dh_l) * GELU'(z_l); dW_l = dz_l^T h_{l-1};
// dh_{l-1} = dz_l W_l; then Adam on the FP32 master weights.
//
// Tensor-core layout: operands in shared memory use the canonical K-major
// layout without swizzle -- 8x8 BF16 core matrices of 128 contiguous bytes,
// consecutive along K (leading byte offset 128), row groups of 8 rows
// 16*K bytes apart (stride byte offset).  One CTA = one 128-row tile at a time:
// inference with 4 warps (row r = thread r = TMEM lane r), training with 16
// warps (four threads per row, 16 features each).  A single thread issues the
// MMAs and commits them to an mbarrier; all waits are bounded by a clock
// budget after which the kernel raises an error flag and leaves cleanly.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"

namespace hp {
namespace {

constexpr int IN = 11, INP = 16, HID = 64, OUT = 2;
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + HID * HID, OW4 = OB3 + HID, OB4 = OW4 + OUT * HID, NPARAM = OB4 + OUT;
constexpr int TILE = 128, NT = 128;
constexpr long long kWaitCycles = 1ll << 32;  // about two seconds at the boost clock

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait on an mbarrier phase; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// After a timed-out wait (every thread of the block calls this): wait up to
// four more limits for the MMA commit that did not arrive (parity phase ^ 1,
// the phase the block gave up on), so that no tensor-core operation is still
// writing the accumulators when they are freed.  *err = 1, or 2 if the drain
// ran out as well (the context must then not be trusted).
__device__ __forceinline__ void drain_after_timeout(uint32_t mbar, uint32_t phase, int* err) {
    bool done = false;
    for (int i = 0; i < 4 && !done; ++i) done = mbar_wait(mbar, phase ^ 1u);
    const bool all = !__syncthreads_or(!done);
    if (threadIdx.x == 0) atomicMax(err, all ? 1 : 2);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
    tmem_ld32(taddr, v);
    tmem_ld32(taddr + 32, v + 32);
}

// ---------------------------------------------------------------------------
// Operand layout helpers
// ---------------------------------------------------------------------------
// byte offset of element (r, k) of an R x K BF16 operand, K-major, no swizzle
__device__ __forceinline__ int canon(int r, int k, int K) {
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Standard normal distribution Phi(z) and density phi(z).  erf(x) for x >= 0
// by the rational approximation of Abramowitz and Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (Hastings): erf(x) = 1 - t (a1 + t (a2 +
// t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1/(1 + p x), |error| <= 1.5e-7; odd
// in x.  Its exp(-x^2) with x = |z|/sqrt2 is exp(-z^2/2), which phi reuses.
__device__ __forceinline__ void ncdf_pdf(float z, float& cdf, float& pdf) {
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    const float e = __expf(-x * x);
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    const float er = fmaf(-poly, e, 1.0f);  // erf(|z| / sqrt2)
    cdf = fmaf(0.5f, copysignf(er, z), 0.5f);
    pdf = 0.39894228040143268f * e;
}
// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z)
__device__ __forceinline__ float gelu(float z) {
    float c, d;
    ncdf_pdf(z, c, d);
    return z * c;
}
__device__ __forceinline__ float gelu_grad(float z) {
    float c, d;
    ncdf_pdf(z, c, d);
    return fmaf(z, d, c);
}

// write a full row of K values (K multiple of 8) into a K-major operand
template <int K>
__device__ __forceinline__ void put_row(unsigned char* base, int r, const float* v) {
#pragma unroll
    for (int c = 0; c < K / 8; ++c) {
        __align__(16) __nv_bfloat16 t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = __float2bfloat16_rn(v[8 * c + j]);
        *reinterpret_cast<int4*>(base + canon(r, 8 * c, K)) = *reinterpret_cast<const int4*>(t);
    }
}

// write value v[i] at (i, col) for i < ROWS of a ROWS x K operand (a column)
template <int ROWS, int K>
__device__ __forceinline__ void put_col(unsigned char* base, int col, const float* v) {
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
        *reinterpret_cast<__nv_bfloat16*>(base + canon(i, col, K)) = __float2bfloat16_rn(v[i]);
}

// stage W [N][Kreal] (FP32, row-major) as an N x KP BF16 K-major operand; zero pad
__device__ void stage_weight(unsigned char* dst, const float* W, int N, int Kreal, int KP) {
    for (int idx = threadIdx.x; idx < N * KP; idx += NT) {
        const int n = idx / KP, k = idx - n * KP;
        const float v = k < Kreal ? W[n * Kreal + k] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(dst + canon(n, k, KP)) = __float2bfloat16_rn(v);
    }
}

__device__ __forceinline__ void sync_for_mma() {
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

// ---------------------------------------------------------------------------
// Forward (inference)
// ---------------------------------------------------------------------------
struct FwdSmem {
    alignas(1024) unsigned char w1[HID * INP * 2];
    alignas(1024) unsigned char w2[HID * HID * 2];
    alignas(1024) unsigned char w3[HID * HID * 2];
    alignas(1024) unsigned char x[TILE * INP * 2];
    alignas(1024) unsigned char h[TILE * HID * 2];
    float b1[HID], b2[HID], b3[HID], w4[OUT * HID], b4[OUT];
    alignas(8) unsigned long long mbar;
    uint32_t tmem;
    int bad;
};

__global__ void __launch_bounds__(NT) k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ X, int64_t M,
                                                float* __restrict__ Y, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(saddr(&S.tmem), 64);
    if (tid == 0) {
        mbar_init(saddr(&S.mbar));
        S.bad = 0;
    }
    stage_weight(S.w1, P + OW1, HID, IN, INP);
    stage_weight(S.w2, P + OW2, HID, HID, HID);
    stage_weight(S.w3, P + OW3, HID, HID, HID);
    for (int i = tid; i < HID; i += NT) {
        S.b1[i] = P[OB1 + i];
        S.b2[i] = P[OB2 + i];
        S.b3[i] = P[OB3 + i];
    }
    for (int i = tid; i < OUT * HID; i += NT) S.w4[i] = bf16r(P[OW4 + i]);
    if (tid < OUT) S.b4[tid] = P[OB4 + tid];
    sync_for_mma();
    const uint32_t tm = S.tmem;
    const uint32_t mbar = saddr(&S.mbar);
    const uint32_t lane_base = tm + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    const int64_t ntiles = (M + TILE - 1) / TILE;
    bool ok = true;
    float v[HID];
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int64_t row = t * TILE + tid;
        float xr[INP];
#pragma unroll
        for (int k = 0; k < INP; ++k) xr[k] = (k < IN && row < M) ? X[row * IN + k] : 0.0f;
        put_row<INP>(S.x, tid, xr);
        sync_for_mma();
        // layer 1
        if (tid == 0) {
            mma(tm, sdesc(saddr(S.x), 128, INP * 16), sdesc(saddr(S.w1), 128, INP * 16), idesc_bf16(TILE, HID), 0);
            mma_commit(mbar);
        }
        ok = mbar_wait(mbar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        fence_after();
        tmem_ld64(lane_base, v);
#pragma unroll
        for (int k = 0; k < HID; ++k) v[k] = gelu(v[k] + S.b1[k]);
        put_row<HID>(S.h, tid, v);
        sync_for_mma();
        // layers 2 and 3
        for (int l = 0; l < 2 && ok; ++l) {
            if (tid == 0) {
                const unsigned char* w = l == 0 ? S.w2 : S.w3;
#pragma unroll
                for (int kk = 0; kk < HID / 16; ++kk)
                    mma(tm, sdesc(saddr(S.h) + 256 * kk, 128, HID * 16), sdesc(saddr(w) + 256 * kk, 128, HID * 16),
                        idesc_bf16(TILE, HID), kk > 0);
                mma_commit(mbar);
            }
            ok = mbar_wait(mbar, phase);
            phase ^= 1;
            if (__syncthreads_or(!ok)) { ok = false; break; }
            fence_after();
            tmem_ld64(lane_base, v);
            const float* b = l == 0 ? S.b2 : S.b3;
#pragma unroll
            for (int k = 0; k < HID; ++k) v[k] = gelu(v[k] + b[k]);
            if (l == 0) {
                put_row<HID>(S.h, tid, v);
                sync_for_mma();
            }
        }
        if (!ok) break;
        // output layer on CUDA cores with BF16-rounded activations and weights
        float y0 = S.b4[0], y1 = S.b4[1];
#pragma unroll
        for (int k = 0; k < HID; ++k) {
            const float h = bf16r(v[k]);
            y0 = fmaf(h, S.w4[k], y0);
            y1 = fmaf(h, S.w4[HID + k], y1);
        }
        if (row < M) {
            Y[row * OUT + 0] = y0;
            Y[row * OUT + 1] = y1;
        }
        fence_before();
        __syncthreads();
    }
    if (!ok) drain_after_timeout(mbar, phase, err);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tm, 64);
}

// ---------------------------------------------------------------------------
// Training: gradients of L over a batch (accumulated into grads and loss)
// ---------------------------------------------------------------------------
struct TrainSmem {
    alignas(1024) unsigned char w1[HID * INP * 2];   // B, layer 1 (N=64, K=16)
    alignas(1024) unsigned char w2[HID * HID * 2];   // B, layer 2
    alignas(1024) unsigned char w3[HID * HID * 2];   // B, layer 3
    alignas(1024) unsigned char w2t[HID * HID * 2];  // B of dh1 = dz2 W2 (N = in, K = out)
    alignas(1024) unsigned char w3t[HID * HID * 2];  // B of dh2 = dz3 W3
    alignas(1024) unsigned char x[TILE * INP * 2];   // A, layer 1
    alignas(1024) unsigned char xt[INP * TILE * 2];  // B of dW1 (N = 16 inputs, K = 128 rows)
    alignas(1024) unsigned char h1[TILE * HID * 2];  // A, layer 2
    alignas(1024) unsigned char h2[TILE * HID * 2];  // A, layer 3
    alignas(1024) unsigned char h1t[HID * TILE * 2]; // B of dW2 (N = 64, K = 128 rows)
    alignas(1024) unsigned char h2t[HID * TILE * 2]; // B of dW3
    alignas(1024) unsigned char dz[TILE * HID * 2];  // A of dh = dz W (K = out features)
    alignas(1024) unsigned char dzt[TILE * TILE * 2];// A of dW (M = 128: 64 features + 64 zero rows, K = rows)
    float b1[HID], b2[HID], b3[HID], w4[OUT * HID], b4[OUT];
    float gb1[HID], gb2[HID], gb3[HID], gw4[OUT * HID], gb4[OUT], loss;
    float2 yp[4][TILE];  // each feature group's share of the output layer, per row
    alignas(8) unsigned long long mbar;
    uint32_t tmem;
};

// TMEM columns
constexpr uint32_t CZ1 = 0, CZ2 = 64, CZ3 = 128, CDH = 192, CDW3 = 256, CDW2 = 320, CDW1 = 384;

// Training runs NH threads per row: warp w serves TMEM lane quadrant w % 4
// (rows 32 (w % 4) .. + 31) and features FW (w / 4) .. + FW - 1 of every
// layer, so that each thread's element-wise work, and its unrolled code, is
// 1/NH of a row.
constexpr int NH = 4, FW = HID / NH, NTT = NH * TILE;

// chunks c0 .. c0 + NCH - 1 (8 values each, v[0 .. 8 NCH)) of row r of a K-major operand
template <int K, int NCH>
__device__ __forceinline__ void put_row_part(unsigned char* base, int r, int c0, const float* v) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        __align__(16) __nv_bfloat16 t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = __float2bfloat16_rn(v[8 * c + j]);
        *reinterpret_cast<int4*>(base + canon(r, 8 * (c0 + c), K)) = *reinterpret_cast<const int4*>(t);
    }
}

// v[i] at (f0 + i, col) for i < N of a ROWS x K operand
template <int N, int K>
__device__ __forceinline__ void put_col_off(unsigned char* base, int col, int f0, const float* v) {
#pragma unroll
    for (int i = 0; i < N; ++i)
        *reinterpret_cast<__nv_bfloat16*>(base + canon(f0 + i, col, K)) = __float2bfloat16_rn(v[i]);
}

// Sum N (16 or 32) per-lane values over the 32 lanes of a warp (a butterfly
// reduce-scatter): lane l ends with the sum of value l / (32 / N) in v[0].
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(float* v) {
    const int lane = threadIdx.x & 31;
    int m = 16;
#pragma unroll
    for (int half = N / 2; half >= 1; half >>= 1, m >>= 1) {
        const bool up = lane & m;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float a = v[i], b = v[i + half];
            const float send = up ? a : b, keep = up ? b : a;
            v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, m);
        }
    }
#pragma unroll
    for (; m >= 1; m >>= 1) v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], m);
}

// FW consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, float* v) {
    if (FW == 32) {
        tmem_ld32(taddr, v);
    } else {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
    }
}

// The packed weight image: the BF16 operands of TrainSmem (w1 .. w3t, in that
// order and layout) followed by the FP32 biases and output layer
// (b1, b2, b3, bf16-rounded W4, b4).  Built from the FP32 parameters by
// k_mlp_pack and rewritten by the fused reduce + Adam kernel after every step.
constexpr int IMG_BF = 2 * (HID * INP + 4 * HID * HID);  // bytes of BF16 operands
constexpr int IMG_F = 3 * HID + OUT * HID + OUT;         // floats after them
constexpr size_t IMG_BYTES = ((size_t)IMG_BF + 4 * IMG_F + 15) / 16 * 16;
// per-CTA gradient slot: NPARAM gradients then the CTA's share of the loss
constexpr int PSTR = (NPARAM + 1 + 3) / 4 * 4;
// at most this many gradient slots (CTAs of the gradient kernel, at most one per SM)
constexpr int kMaxSlots = 160;
static_assert(offsetof(TrainSmem, w1) == 0 && offsetof(TrainSmem, w2) == 2 * HID * INP &&
                  offsetof(TrainSmem, w3t) + 2 * HID * HID == IMG_BF,
              "the BF16 operands are one block at the start of TrainSmem");

// write parameter i (value p) into the packed image
__device__ __forceinline__ void pack_param(unsigned char* img, int i, float p) {
    float* f = reinterpret_cast<float*>(img + IMG_BF);
    const __nv_bfloat16 h = __float2bfloat16_rn(p);
    unsigned char* w2 = img + 2 * HID * INP;
    unsigned char* w3 = w2 + 2 * HID * HID;
    unsigned char* w2t = w3 + 2 * HID * HID;
    unsigned char* w3t = w2t + 2 * HID * HID;
    if (i < OB1) {
        *reinterpret_cast<__nv_bfloat16*>(img + canon(i / IN, i % IN, INP)) = h;
    } else if (i < OW2) {
        f[i - OB1] = p;
    } else if (i < OB2) {
        const int t = i - OW2, n = t / HID, k = t - n * HID;
        *reinterpret_cast<__nv_bfloat16*>(w2 + canon(n, k, HID)) = h;
        *reinterpret_cast<__nv_bfloat16*>(w2t + canon(k, n, HID)) = h;
    } else if (i < OW3) {
        f[HID + i - OB2] = p;
    } else if (i < OB3) {
        const int t = i - OW3, n = t / HID, k = t - n * HID;
        *reinterpret_cast<__nv_bfloat16*>(w3 + canon(n, k, HID)) = h;
        *reinterpret_cast<__nv_bfloat16*>(w3t + canon(k, n, HID)) = h;
    } else if (i < OW4) {
        f[2 * HID + i - OB3] = p;
    } else if (i < OB4) {
        f[3 * HID + i - OW4] = bf16r(p);
    } else {
        f[3 * HID + OUT * HID + i - OB4] = p;
    }
}

__global__ void k_mlp_pack(const float* __restrict__ P, unsigned char* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) pack_param(img, i, P[i]);
    if (i < HID * (INP - IN)) {  // zero padding of the first layer's K
        const int n = i / (INP - IN), k = IN + i % (INP - IN);
        *reinterpret_cast<__nv_bfloat16*>(img + canon(n, k, INP)) = __float2bfloat16_rn(0.0f);
    }
}

// Arguments of the gradient kernels.  One step (k_mlp_train): the minibatch is
// X, T (M rows), the packed weights img_in, gradients to the CTA's slot.  A whole
// training run (k_mlp_train_loop, a cooperative launch with every CTA resident):
// step s = 1..steps takes minibatch (s - 1) mod n_batches (rows (s - 1 mod
// n_batches) M .. + M of X, T), reads the packed weights from img, writes its
// slot; after a grid barrier each CTA reduces its share of the entries over all
// slots, applies Adam (sched[3(s-1) ..] = lr, 1 - beta1^t, 1 - beta2^t) to P,
// m, v and rewrites those entries of img; a second grid barrier ends the step.
struct TrainArgs {
    const unsigned char* img_in;
    unsigned char* img;
    const float* X;
    const float* T;
    int64_t M;
    float inv_batch;
    float* part;
    int* err;
    int64_t n_batches;
    int32_t steps;
    const float* sched;
    float b1, b2, eps;
    float* P;
    float* m;
    float* v;
    float* loss_log;    // [steps] or null
    float* loss_last;   // or null
    unsigned int* bar;  // grid barrier: arrivals, generation (zeroed before launch)
};

// Grid-wide barrier of a cooperative launch (every CTA resident): thread 0 of
// each CTA arrives on a counter; the last to arrive resets it and advances the
// generation the others poll.  Bounded: after `limit` cycles a waiting CTA
// gives up (false).  Global writes before the barrier are visible after it to
// loads that go through L2.
__device__ bool grid_barrier(unsigned int* bar, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        bool ok = true;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > limit) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum of entry i over the slots written earlier in the same launch (loads
// through L2), by the 8 consecutive lanes of a group in a fixed order; i < 0
// adds nothing but takes part in the shuffles.
__device__ __forceinline__ float slot_sum_cg(const float* part, int nslots, int i) {
    const int j = threadIdx.x & 7;
    float acc = 0.0f;
    if (i >= 0 && i <= NPARAM) {
        // every load of the group issued before the sum (at most kMaxSlots slots)
        float g[kMaxSlots / 8];
#pragma unroll
        for (int k = 0; k < kMaxSlots / 8; ++k) {
            const int c = j + 8 * k;
            g[k] = c < nslots ? __ldcg(part + (size_t)c * PSTR + i) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kMaxSlots / 8; ++k) acc += g[k];
    }
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
    return acc;
}

template <bool LOOP>
__device__ __forceinline__ void train_body(const TrainArgs& a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, hf = warp >> 2;
    const int r = quad * 32 + lane;  // row of the tile = TMEM lane
    const int f0 = FW * hf;          // first feature of this thread
    constexpr int RL = 32 / FW;      // lanes holding each feature after a reduce-scatter
    const int64_t M = a.M;
    const float inv_batch = a.inv_batch;
    float* __restrict__ part = a.part;
    int* err = a.err;
    if (warp == 0) tmem_alloc(saddr(&S.tmem), 512);
    if (tid == 0) mbar_init(saddr(&S.mbar));
    for (int i = tid; i < TILE * TILE * 2 / 16; i += NTT) reinterpret_cast<int4*>(S.dzt)[i] = make_int4(0, 0, 0, 0);
    sync_for_mma();
    const uint32_t tm = S.tmem;
    const uint32_t mbar = saddr(&S.mbar);
    const uint32_t lb = tm + ((uint32_t)(quad * 32) << 16) + (uint32_t)f0;
    uint32_t phase = 0;
    const int64_t ntiles = (M + TILE - 1) / TILE;
    bool ok = true, mma_ok = true;
    float v[FW], z[FW];

    auto wait_mma = [&]() -> bool {
        const bool w = mbar_wait(mbar, phase);
        phase ^= 1;
        const bool any_bad = __syncthreads_or(!w);
        fence_after();
        return !any_bad;
    };
    // bias gradient of this thread's FW features summed over the warp's 32 rows
    auto bias_grad = [&](float* g) {
        warp_reduce_scatter<FW>(v);
        if (lane % RL == 0) atomicAdd(&g[f0 + lane / RL], v[0]);
    };

    const int32_t nsteps = LOOP ? a.steps : 1;
    for (int32_t step = 1; step <= nsteps && ok; ++step) {
        const int64_t r0 = LOOP ? ((int64_t)(step - 1) % a.n_batches) * M : 0;
        const float* __restrict__ X = a.X + r0 * IN;
        const float* __restrict__ T = a.T + r0 * OUT;
        {   // the packed weights: the BF16 operands are one contiguous block at
            // the start of TrainSmem (the image of a running loop is read
            // through L2: it was rewritten in this launch)
            const unsigned char* img = LOOP ? a.img : a.img_in;
            const int4* src = reinterpret_cast<const int4*>(img);
            int4* dst = reinterpret_cast<int4*>(S.w1);
            for (int i = tid; i < IMG_BF / 16; i += NTT) dst[i] = LOOP ? __ldcg(src + i) : __ldg(src + i);
            const float* f = reinterpret_cast<const float*>(img + IMG_BF);
            for (int i = tid; i < HID; i += NTT) {
                S.b1[i] = __ldcg(f + i);
                S.b2[i] = __ldcg(f + HID + i);
                S.b3[i] = __ldcg(f + 2 * HID + i);
                S.gb1[i] = S.gb2[i] = S.gb3[i] = 0.0f;
            }
            for (int i = tid; i < OUT * HID; i += NTT) {
                S.w4[i] = __ldcg(f + 3 * HID + i);
                S.gw4[i] = 0.0f;
            }
            if (tid < OUT) {
                S.b4[tid] = __ldcg(f + 3 * HID + OUT * HID + tid);
                S.gb4[tid] = 0.0f;
            }
            if (tid == 0) S.loss = 0.0f;
        }
        sync_for_mma();
        uint32_t first = 1;  // first tile of this CTA in the step: weight-gradient accumulators start from zero
        float my_loss = 0.0f, gb4_0 = 0.0f, gb4_1 = 0.0f;

        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int64_t row = t * TILE + r;
            const bool valid = row < M;
            if (hf < 2) {   // inputs 8 hf .. 8 hf + 7 of this row
                float xr[8];
    #pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int f = 8 * hf + k;
                    xr[k] = (f < IN && valid) ? X[row * IN + f] : 0.0f;
                }
                put_row_part<INP, 1>(S.x, r, hf, xr);
                put_col_off<8, TILE>(S.xt, r, 8 * hf, xr);
            }
            sync_for_mma();
            // ---- forward ------------------------------------------------------
            if (tid == 0) {
                mma(tm + CZ1, sdesc(saddr(S.x), 128, INP * 16), sdesc(saddr(S.w1), 128, INP * 16), idesc_bf16(TILE, HID), 0);
                mma_commit(mbar);
            }
            if (!(ok = wait_mma())) break;
            tmem_ldw(lb + CZ1, v);
    #pragma unroll
            for (int k = 0; k < FW; ++k) v[k] = gelu(v[k] + S.b1[f0 + k]);
            put_row_part<HID, FW / 8>(S.h1, r, (FW / 8) * hf, v);
            put_col_off<FW, TILE>(S.h1t, r, f0, v);
            sync_for_mma();
            if (tid == 0) {
    #pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma(tm + CZ2, sdesc(saddr(S.h1) + 256 * kk, 128, HID * 16), sdesc(saddr(S.w2) + 256 * kk, 128, HID * 16),
                        idesc_bf16(TILE, HID), kk > 0);
                mma_commit(mbar);
            }
            if (!(ok = wait_mma())) break;
            tmem_ldw(lb + CZ2, v);
    #pragma unroll
            for (int k = 0; k < FW; ++k) v[k] = gelu(v[k] + S.b2[f0 + k]);
            put_row_part<HID, FW / 8>(S.h2, r, (FW / 8) * hf, v);
            put_col_off<FW, TILE>(S.h2t, r, f0, v);
            sync_for_mma();
            if (tid == 0) {
    #pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma(tm + CZ3, sdesc(saddr(S.h2) + 256 * kk, 128, HID * 16), sdesc(saddr(S.w3) + 256 * kk, 128, HID * 16),
                        idesc_bf16(TILE, HID), kk > 0);
                mma_commit(mbar);
            }
            if (!(ok = wait_mma())) break;
            tmem_ldw(lb + CZ3, z);
            // ---- output layer, loss, dz3 ---------------------------------------
            float p0 = 0.0f, p1 = 0.0f;  // this half's share of y
    #pragma unroll
            for (int k = 0; k < FW; ++k) {
                z[k] += S.b3[f0 + k];
                v[k] = bf16r(gelu(z[k]));  // h3
                p0 = fmaf(v[k], S.w4[f0 + k], p0);
                p1 = fmaf(v[k], S.w4[HID + f0 + k], p1);
            }
            S.yp[hf][r] = make_float2(p0, p1);
            __syncthreads();
            float y0 = S.b4[0], y1 = S.b4[1];
    #pragma unroll
            for (int h = 0; h < NH; ++h) {
                const float2 yh = S.yp[h][r];
                y0 += yh.x;
                y1 += yh.y;
            }
            float d0 = 0.0f, d1 = 0.0f;
            if (valid) {
                const float e0 = y0 - T[row * OUT + 0], e1 = y1 - T[row * OUT + 1];
                if (hf == 0) my_loss += e0 * e0 + e1 * e1;
                d0 = e0 * inv_batch;
                d1 = e1 * inv_batch;
            }
            if (hf == 0) {
                gb4_0 += d0;
                gb4_1 += d1;
            }
            {   // dW4[o][k] = sum_rows d_o h3_k
                float g[FW];
    #pragma unroll
                for (int k = 0; k < FW; ++k) g[k] = d0 * v[k];
                warp_reduce_scatter<FW>(g);
                if (lane % RL == 0) atomicAdd(&S.gw4[f0 + lane / RL], g[0]);
    #pragma unroll
                for (int k = 0; k < FW; ++k) g[k] = d1 * v[k];
                warp_reduce_scatter<FW>(g);
                if (lane % RL == 0) atomicAdd(&S.gw4[HID + f0 + lane / RL], g[0]);
            }
    #pragma unroll
            for (int k = 0; k < FW; ++k)
                v[k] = (d0 * S.w4[f0 + k] + d1 * S.w4[HID + f0 + k]) * gelu_grad(z[k]);  // dz3
            put_row_part<HID, FW / 8>(S.dz, r, (FW / 8) * hf, v);
            put_col_off<FW, TILE>(S.dzt, r, f0, v);
            bias_grad(S.gb3);
            sync_for_mma();
            // ---- dh2 = dz3 W3, dW3 += dz3^T h2 ---------------------------------
            if (tid == 0) {
    #pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma(tm + CDH, sdesc(saddr(S.dz) + 256 * kk, 128, HID * 16), sdesc(saddr(S.w3t) + 256 * kk, 128, HID * 16),
                        idesc_bf16(TILE, HID), kk > 0);
    #pragma unroll
                for (int kk = 0; kk < 8; ++kk)
                    mma(tm + CDW3, sdesc(saddr(S.dzt) + 256 * kk, 128, TILE * 16), sdesc(saddr(S.h2t) + 256 * kk, 128, TILE * 16),
                        idesc_bf16(TILE, HID), (kk > 0) | (first ^ 1));
                mma_commit(mbar);
            }
            if (!(ok = wait_mma())) break;
            tmem_ldw(lb + CDH, v);
            tmem_ldw(lb + CZ2, z);
    #pragma unroll
            for (int k = 0; k < FW; ++k) v[k] *= gelu_grad(z[k] + S.b2[f0 + k]);  // dz2
            put_row_part<HID, FW / 8>(S.dz, r, (FW / 8) * hf, v);
            put_col_off<FW, TILE>(S.dzt, r, f0, v);
            bias_grad(S.gb2);
            sync_for_mma();
            // ---- dh1 = dz2 W2, dW2 += dz2^T h1 ---------------------------------
            if (tid == 0) {
    #pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma(tm + CDH, sdesc(saddr(S.dz) + 256 * kk, 128, HID * 16), sdesc(saddr(S.w2t) + 256 * kk, 128, HID * 16),
                        idesc_bf16(TILE, HID), kk > 0);
    #pragma unroll
                for (int kk = 0; kk < 8; ++kk)
                    mma(tm + CDW2, sdesc(saddr(S.dzt) + 256 * kk, 128, TILE * 16), sdesc(saddr(S.h1t) + 256 * kk, 128, TILE * 16),
                        idesc_bf16(TILE, HID), (kk > 0) | (first ^ 1));
                mma_commit(mbar);
            }
            if (!(ok = wait_mma())) break;
            tmem_ldw(lb + CDH, v);
            tmem_ldw(lb + CZ1, z);
    #pragma unroll
            for (int k = 0; k < FW; ++k) v[k] *= gelu_grad(z[k] + S.b1[f0 + k]);  // dz1
            put_col_off<FW, TILE>(S.dzt, r, f0, v);
            bias_grad(S.gb1);
            sync_for_mma();
            // ---- dW1 += dz1^T x -------------------------------------------------
            if (tid == 0) {
    #pragma unroll
                for (int kk = 0; kk < 8; ++kk)
                    mma(tm + CDW1, sdesc(saddr(S.dzt) + 256 * kk, 128, TILE * 16), sdesc(saddr(S.xt) + 256 * kk, 128, TILE * 16),
                        idesc_bf16(TILE, INP), (kk > 0) | (first ^ 1));
                mma_commit(mbar);
            }
            if (!(ok = wait_mma())) break;
            first = 0;
        }
        // ---- this CTA's gradients to its slot (plain stores; every entry written) --
        if (ok && !first) {
            float* slot = part + (size_t)blockIdx.x * PSTR;
            // weight gradients: TMEM lanes 0..63 (quadrants 0 and 1) hold dW rows
            // (out features); each group of four warps takes FW of the columns
            if (quad < 2) {
                const int o = r;  // out feature
                tmem_ldw(lb + CDW3, v);
    #pragma unroll
                for (int k = 0; k < FW; k += 4)
                    *reinterpret_cast<float4*>(slot + OW3 + o * HID + f0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                tmem_ldw(lb + CDW2, v);
    #pragma unroll
                for (int k = 0; k < FW; k += 4)
                    *reinterpret_cast<float4*>(slot + OW2 + o * HID + f0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                if (hf == 0) {
                    tmem_ldw(lb + CDW1, v);  // the first 16 columns hold dW1
    #pragma unroll
                    for (int k = 0; k < IN; ++k) slot[OW1 + o * IN + k] = v[k];
                }
            }
            // per-row reductions of the loss and b4 gradient (the other groups add zeros)
            for (int m = 16; m >= 1; m >>= 1) {
                my_loss += __shfl_xor_sync(0xFFFFFFFFu, my_loss, m);
                gb4_0 += __shfl_xor_sync(0xFFFFFFFFu, gb4_0, m);
                gb4_1 += __shfl_xor_sync(0xFFFFFFFFu, gb4_1, m);
            }
            if (lane == 0) {
                atomicAdd(&S.loss, my_loss);
                atomicAdd(&S.gb4[0], gb4_0);
                atomicAdd(&S.gb4[1], gb4_1);
            }
            __syncthreads();
            for (int i = tid; i < HID; i += NTT) {
                slot[OB1 + i] = S.gb1[i];
                slot[OB2 + i] = S.gb2[i];
                slot[OB3 + i] = S.gb3[i];
            }
            for (int i = tid; i < OUT * HID; i += NTT) slot[OW4 + i] = S.gw4[i];
            if (tid < OUT) slot[OB4 + tid] = S.gb4[tid];
            if (tid == 0) slot[NPARAM] = S.loss * 0.5f * inv_batch;
        }
        mma_ok = ok;
        if (LOOP && ok) {
            ok = grid_barrier(a.bar, kWaitCycles);
            if (ok) {
                // this CTA's share of the entries: reduce over every slot, Adam, repack
                const int nslots = (int)gridDim.x;
                const int chunk = (NPARAM + 1 + nslots - 1) / nslots;
                const int lo = (int)blockIdx.x * chunk, hi = min(lo + chunk, NPARAM + 1);
                const float lr = a.sched[3 * (step - 1)], c1 = a.sched[3 * (step - 1) + 1],
                            c2 = a.sched[3 * (step - 1) + 2];
                for (int base = lo; base < hi; base += NTT / 8) {
                    const int i = base + (tid >> 3);
                    const float gi = slot_sum_cg(part, nslots, i < hi ? i : -1);
                    if ((tid & 7) == 0 && i < hi) {
                        if (i == NPARAM) {
                            if (a.loss_log) a.loss_log[step - 1] = gi;
                            if (a.loss_last) *a.loss_last = gi;
                        } else {
                            const float mi = a.b1 * a.m[i] + (1.0f - a.b1) * gi;
                            const float vi = a.b2 * a.v[i] + (1.0f - a.b2) * gi * gi;
                            a.m[i] = mi;
                            a.v[i] = vi;
                            const float pv = a.P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + a.eps);
                            a.P[i] = pv;
                            pack_param(a.img, i, pv);
                        }
                    }
                }
                ok = grid_barrier(a.bar, kWaitCycles);
            }
            if (!ok && tid == 0) atomicMax(err, 1);  // a barrier ran out; nothing is in flight
        }
    }
    if (!mma_ok) drain_after_timeout(mbar, phase, err);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tm, 512);
}

__global__ void __launch_bounds__(NTT, 1) k_mlp_train(const __grid_constant__ TrainArgs a) { train_body<false>(a); }
__global__ void __launch_bounds__(NTT, 1) k_mlp_train_loop(const __grid_constant__ TrainArgs a) { train_body<true>(a); }

// Adam on the FP32 master weights (bias-corrected; t counts from 1)
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Sum of entry i over the nslots gradient slots, by the 8 consecutive lanes
// of a group (lane j of the group takes slots j, j + 8, ...; a fixed shuffle
// tree then adds the eight partial sums, so the order never varies).
__device__ __forceinline__ float slot_sum(const float* __restrict__ part, int nslots, int i) {
    const int j = threadIdx.x & 7;
    float acc = 0.0f;
    if (i <= NPARAM) {
        float g[kMaxSlots / 8];
#pragma unroll
        for (int k = 0; k < kMaxSlots / 8; ++k) {
            const int c = j + 8 * k;
            g[k] = c < nslots ? part[(size_t)c * PSTR + i] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kMaxSlots / 8; ++k) acc += g[k];
    }
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
    return acc;
}

constexpr int kRedT = 256, kRedPer = kRedT / 8;  // entries per block
constexpr int kRedBlocks = (NPARAM + 1 + kRedPer - 1) / kRedPer;

// gradients (and the loss, entry NPARAM) of a batch from its slots
__global__ void __launch_bounds__(kRedT) k_mlp_reduce(const float* __restrict__ part, int nslots,
                                                      float* __restrict__ grads, float* __restrict__ loss) {
    const int i = blockIdx.x * kRedPer + (threadIdx.x >> 3);
    const float g = slot_sum(part, nslots, i);
    if ((threadIdx.x & 7) == 0) {
        if (i < NPARAM) grads[i] = g;
        if (i == NPARAM && loss) *loss = g;
    }
}

// One training step's update: the slots summed (as k_mlp_reduce), Adam (as
// k_adam) and the new parameter written into the packed image for the next step.
__global__ void __launch_bounds__(kRedT) k_mlp_reduce_adam(const float* __restrict__ part, int nslots,
                                                           float* __restrict__ P, float* __restrict__ m,
                                                           float* __restrict__ v, unsigned char* __restrict__ img,
                                                           float* __restrict__ loss, float lr, float b1, float b2,
                                                           float eps, float c1, float c2) {
    const int i = blockIdx.x * kRedPer + (threadIdx.x >> 3);
    const float gi = slot_sum(part, nslots, i);
    if ((threadIdx.x & 7) != 0) return;
    if (i == NPARAM && loss) *loss = gi;
    if (i >= NPARAM) return;
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    P[i] = p;
    pack_param(img, i, p);
}

__global__ void k_gelu_eval(const float* __restrict__ z, int64_t n, float* __restrict__ g, float* __restrict__ dg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    g[i] = gelu(z[i]);
    dg[i] = gelu_grad(z[i]);
}

int g_err_dev = -1;
int* g_err = nullptr;

// One block, nothing in flight: an mbarrier that expects one arrival, waited
// on with a short limit; the arrival comes from thread 32 after two limits
// (`late`: the drain sees it, flag 1) or never (flag 2).
__global__ void k_mlp_wait_probe(long long limit, int late, int* err) {
    __shared__ unsigned long long bar;
    const uint32_t mb = saddr(&bar);
    if (threadIdx.x == 0) mbar_init(mb);
    __syncthreads();
    if (late && threadIdx.x == 32) {
        const long long t0 = clock64();
        while (clock64() - t0 < 2 * limit) {
        }
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
    }
    bool ok = mbar_wait(mb, 0u, limit);
    if (__syncthreads_or(!ok)) {
        bool done = false;
        for (int i = 0; i < 4 && !done; ++i) done = mbar_wait(mb, 0u, limit);
        const bool all = !__syncthreads_or(!done);
        if (threadIdx.x == 0) atomicMax(err, all ? 1 : 2);
    }
}

int error_flag(int** out) {
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    if (!g_err || g_err_dev != dev) {
        HP_CUDA(cudaMalloc((void**)&g_err, sizeof(int)));
        HP_CUDA(cudaMemset(g_err, 0, sizeof(int)));
        g_err_dev = dev;
    }
    *out = g_err;
    return HP_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_mlp_param_count(int64_t* n) {
    if (!n) return set_error(HP_ERR_ARG, "hp_mlp_param_count: null argument");
    *n = NPARAM;
    return HP_OK;
}

extern "C" int hp_mlp_forward(const float* params, const float* X, int64_t M, float* Y, void* stream) {
    if (!params || !X || !Y || M < 0) return set_error(HP_ERR_ARG, "hp_mlp_forward: bad arguments");
    if (M == 0) return HP_OK;
    int* err = nullptr;
    int rc = error_flag(&err);
    if (rc) return rc;
    const size_t smem = sizeof(FwdSmem) + 1024;
    static bool configured = false;
    if (!configured) {
        HP_CUDA(cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    const int64_t tiles = (M + TILE - 1) / TILE;
    const int64_t grid = tiles < 4LL * sm_count() ? tiles : 4LL * sm_count();
    cudaStream_t s = as_stream(stream);
    ::hp::count_launch();
    k_mlp_fwd<<<(unsigned)grid, NT, smem, s>>>(params, X, M, Y, err);
    HP_LAUNCH_CHECK("k_mlp_fwd");
    return HP_OK;
}

namespace hp {
namespace {
int train_configure() {
    static bool configured = false;
    if (!configured) {
        HP_CUDA(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(TrainSmem) + 1024)));
        HP_CUDA(cudaFuncSetAttribute(k_mlp_train_loop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(TrainSmem) + 1024)));
        configured = true;
    }
    return HP_OK;
}

int64_t train_grid(int64_t M) {
    const int64_t tiles = (M + TILE - 1) / TILE;
    int64_t g = tiles < sm_count() ? tiles : sm_count();
    return g < kMaxSlots ? g : kMaxSlots;
}

int launch_train(const unsigned char* img, const float* X, const float* T, int64_t M, float* part, int* err,
                 cudaStream_t s) {
    TrainArgs a;
    memset(&a, 0, sizeof(a));
    a.img_in = img;
    a.X = X;
    a.T = T;
    a.M = M;
    a.inv_batch = 1.0f / (float)M;
    a.part = part;
    a.err = err;
    a.n_batches = 1;
    a.steps = 1;
    ::hp::count_launch();
    k_mlp_train<<<(unsigned)train_grid(M), NTT, sizeof(TrainSmem) + 1024, s>>>(a);
    HP_LAUNCH_CHECK("k_mlp_train");
    return HP_OK;
}

int launch_pack(const float* params, unsigned char* img, cudaStream_t s) {
    ::hp::count_launch();
    k_mlp_pack<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, img);
    HP_LAUNCH_CHECK("k_mlp_pack");
    return HP_OK;
}
}  // namespace

int mlp_train_begin(const float* params, int64_t rows, MlpTrain* t, cudaStream_t s) {
    if (!params || rows < 1 || !t) return set_error(HP_ERR_ARG, "mlp_train_begin: bad arguments");
    int rc = train_configure();
    if (rc) return rc;
    t->rows = rows;
    t->grid = train_grid(rows);
    if (cudaMallocAsync((void**)&t->img, IMG_BYTES, s) != cudaSuccess ||
        cudaMallocAsync((void**)&t->part, sizeof(float) * (size_t)PSTR * (size_t)t->grid, s) != cudaSuccess) {
        mlp_train_end(t, s);
        return set_error(HP_ERR_OOM, "mlp_train_begin: allocation failed");
    }
    return launch_pack(params, t->img, s);
}

int mlp_train_step(MlpTrain* t, float* params, float* m, float* v, const float* X, const float* Y, int32_t step,
                   float lr, float beta1, float beta2, float eps, float* loss, cudaStream_t s) {
    if (!t || !t->img || !t->part || step < 1) return set_error(HP_ERR_ARG, "mlp_train_step: bad arguments");
    int* err = nullptr;
    int rc = error_flag(&err);
    if (rc) return rc;
    rc = launch_train(t->img, X, Y, t->rows, t->part, err, s);
    if (rc) return rc;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    ::hp::count_launch();
    k_mlp_reduce_adam<<<kRedBlocks, kRedT, 0, s>>>(t->part, (int)t->grid, params, m, v, t->img, loss, lr, beta1, beta2,
                                                   eps, c1, c2);
    HP_LAUNCH_CHECK("k_mlp_reduce_adam");
    return HP_OK;
}

int mlp_train_loop(MlpTrain* t, float* params, float* m, float* v, const float* X, const float* Y, int64_t n_batches,
                   int32_t steps, const float* sched, float beta1, float beta2, float eps, float* loss_log,
                   float* loss_last, cudaStream_t s, bool* ran) {
    *ran = false;
    if (!t || !t->img || !t->part || steps < 1 || n_batches < 1)
        return set_error(HP_ERR_ARG, "mlp_train_loop: bad arguments");
    int dev = 0, coop = 0, per_sm = 0;
    HP_CUDA(cudaGetDevice(&dev));
    HP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    HP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_train_loop, NTT, sizeof(TrainSmem) + 1024));
    if (!coop || (int64_t)per_sm * sm_count() < t->grid) return HP_OK;  // every CTA must be resident
    int* err = nullptr;
    int rc = error_flag(&err);
    if (rc) return rc;
    unsigned int* bar = nullptr;
    if (cudaMallocAsync((void**)&bar, 2 * sizeof(unsigned int), s) != cudaSuccess)
        return set_error(HP_ERR_OOM, "mlp_train_loop: allocation failed");
    HP_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s));
    TrainArgs a;
    memset(&a, 0, sizeof(a));
    a.img = t->img;
    a.X = X;
    a.T = Y;
    a.M = t->rows;
    a.inv_batch = 1.0f / (float)t->rows;
    a.part = t->part;
    a.err = err;
    a.n_batches = n_batches;
    a.steps = steps;
    a.sched = sched;
    a.b1 = beta1;
    a.b2 = beta2;
    a.eps = eps;
    a.P = params;
    a.m = m;
    a.v = v;
    a.loss_log = loss_log;
    a.loss_last = loss_last;
    a.bar = bar;
    void* args[] = {&a};
    ::hp::count_launch();
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_mlp_train_loop, dim3((unsigned)t->grid), dim3(NTT),
                                                      args, sizeof(TrainSmem) + 1024, s);
    cudaFreeAsync(bar, s);
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
        cudaGetLastError();  // refused before any work: the caller steps instead
        return HP_OK;
    }
    if (e != cudaSuccess) return cuda_error(e, "k_mlp_train_loop");
    *ran = true;
    return HP_OK;
}

void mlp_train_end(MlpTrain* t, cudaStream_t s) {
    if (!t) return;
    if (t->img) cudaFreeAsync(t->img, s);
    if (t->part) cudaFreeAsync(t->part, s);
    t->img = nullptr;
    t->part = nullptr;
}
}  // namespace hp

extern "C" int hp_mlp_gradients(const float* params, const float* X, const float* T, int64_t M, float* grads,
                                float* loss, void* stream) {
    if (!params || !X || !T || !grads || M < 1) return set_error(HP_ERR_ARG, "hp_mlp_gradients: bad arguments");
    int* err = nullptr;
    int rc = error_flag(&err);
    if (rc) return rc;
    cudaStream_t s = as_stream(stream);
    MlpTrain t;
    rc = mlp_train_begin(params, M, &t, s);
    if (rc == HP_OK) rc = launch_train(t.img, X, T, M, t.part, err, s);
    if (rc == HP_OK) {
        ::hp::count_launch();
        k_mlp_reduce<<<kRedBlocks, kRedT, 0, s>>>(t.part, (int)t.grid, grads, loss);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error(e, "k_mlp_reduce");
    }
    mlp_train_end(&t, s);
    return rc;
}

extern "C" int hp_debug_gelu(const float* z, int64_t n, float* g, float* dg, void* stream) {
    if (!z || !g || !dg || n < 0) return set_error(HP_ERR_ARG, "hp_debug_gelu: bad arguments");
    if (n == 0) return HP_OK;
    ::hp::count_launch();
    k_gelu_eval<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(z, n, g, dg);
    HP_LAUNCH_CHECK("k_gelu_eval");
    return HP_OK;
}

extern "C" int hp_mlp_adam(float* params, const float* grads, float* m, float* v, int32_t step, float lr, float beta1,
                           float beta2, float eps, void* stream) {
    if (!params || !grads || !m || !v || step < 1) return set_error(HP_ERR_ARG, "hp_mlp_adam: bad arguments");
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    ::hp::count_launch();
    k_adam<<<(NPARAM + 255) / 256, 256, 0, as_stream(stream)>>>(params, grads, m, v, NPARAM, lr, beta1, beta2, eps, c1, c2);
    HP_LAUNCH_CHECK("k_adam");
    return HP_OK;
}

namespace hp {
int mlp_wait_probe(long long limit, int late, cudaStream_t s) {
    if (limit < 1 || limit > kWaitCycles) return set_error(HP_ERR_ARG, "wait probe: limit out of range");
    int* err = nullptr;
    int rc = error_flag(&err);
    if (rc) return rc;
    count_launch();
    k_mlp_wait_probe<<<1, 64, 0, s>>>(limit, late, err);
    HP_LAUNCH_CHECK("k_mlp_wait_probe");
    return HP_OK;
}
}  // namespace hp

extern "C" int hp_mlp_status(int32_t* timed_out) {
    if (!timed_out) return set_error(HP_ERR_ARG, "hp_mlp_status: null argument");
    int* err = nullptr;
    int rc = error_flag(&err);
    if (rc) return rc;
    int v = 0;
    HP_CUDA(cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost));
    *timed_out = v;
    if (v) HP_CUDA(cudaMemset(err, 0, sizeof(int)));
    return v ? set_error(HP_ERR_TIMEOUT, "surrogate kernel gave up waiting for the tensor cores") : HP_OK;
}
