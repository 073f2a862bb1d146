// Internal definitions shared by the library's translation units.
// (Device side: Philox, lattice geometry; host side: error plumbing and the
// handle layout.)  Nothing here is part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "../../include/hmcpotts.h"

namespace hp {

// ---------------------------------------------------------------------------
// Errors: thread-local last message, HP_* codes.
// ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);

#define HP_CUDA(call)                                  \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return ::hp::cuda_error(_e, #call); \
    } while (0)

#define HP_LAUNCH_CHECK(what)                                     \
    do {                                                          \
        cudaError_t _e = cudaGetLastError();                      \
        if (_e != cudaSuccess) return ::hp::cuda_error(_e, what); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// NVTX range over a scope (host side: the calls that launch work, each MCS of
// a sweep); free when no profiler is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Process-wide count of kernel launches issued by this library (graph
// replays add their kernel nodes).
void count_launch();
void count_launch_n(unsigned long long n);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Counter words: unit lo, unit hi,
// step, tag << 24 | sub.  Key: seed lo, seed hi.
// ---------------------------------------------------------------------------
enum : uint32_t { kTagSweep = 0, kTagMcp = 1, kTagVoronoi = 2, kTagSurrogate = 3 };

__device__ __forceinline__ uint4 philox10(uint32_t k0, uint32_t k1, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same rounds with the ten round keys given (rk[2r], rk[2r+1] for round r,
// as philox_round_keys makes them), so that a kernel can take them from its
// launch parameters instead of stepping the key in every thread.
__device__ __forceinline__ uint4 philox10_keyed(const uint32_t* rk, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

__host__ __device__ inline void philox_round_keys(uint64_t seed, uint32_t rk[20]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t unit, uint32_t step, uint32_t tag, uint32_t sub) {
    return philox10((uint32_t)seed, (uint32_t)(seed >> 32),
                     make_uint4((uint32_t)unit, (uint32_t)(unit >> 32), step, (tag << 24) | sub));
}

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct Lattice {
    int dim;
    int64_t L[3];  // L[2] = 1 in 2D
    int nbr;
    int colours;
    int64_t N;
};

}  // namespace hp

struct hp_handle {
    hp_desc desc;
    hp::Lattice lat;
    int32_t* q = nullptr;       // borrowed
    int32_t* mp = nullptr;      // borrowed (may be null)
    int32_t* q_alt = nullptr;   // owned double buffers
    int32_t* mp_alt = nullptr;
    const int32_t* table = nullptr;  // borrowed field table
    int64_t table_n = 0;
    uint32_t* thr = nullptr;    // owned device threshold table
    int32_t D = -1;
    int32_t thr_cap = 0;
    uint64_t sweep = 0;
    int sweep_kernel = HP_SWEEP_AUTO;
    int sweep_variant = -1;     // tile variant of the fused kernel (-1: the lattice's default)
    // misorientation-dependent pair energy and mobility (hp_set_anisotropy)
    const int32_t* an_ang = nullptr;  // borrowed grain angles
    int32_t* an_J = nullptr;          // owned device tables
    uint32_t* an_mob = nullptr;
    int32_t an_period = 0, an_bin = 0, an_nbins = 0;
    // owned scratch of hp_measure (allocated on its first call)
    unsigned long long* m_counts = nullptr;  // int64[G]
    int32_t* m_bins = nullptr;               // int32[2G]
    unsigned long long* m_small = nullptr;   // hist[90] | field sum | alive | bad ids
};

namespace hp {
// launchers (sweep.cu)
int sweep_run(hp_handle* h, int32_t n_mcs, cudaStream_t s);
// launchers (voronoi.cu)
int voronoi_run(hp_handle* h, int32_t orient_kind, float* orient, int64_t* seed_pos, cudaStream_t s);
int orientations_run(int32_t G, uint64_t seed, int32_t kind, float* orient, cudaStream_t s);
// Bounded-wait probes for tests of the timeout paths (lean.cu, mlp.cu): one
// block waits on an mbarrier with nothing in flight, the arrival coming after
// two limits (late != 0) or never; the sweep or surrogate timeout flag is
// raised exactly as by a kernel that timed out.
int lean_wait_probe(long long limit, int late, cudaStream_t s);
int mlp_wait_probe(long long limit, int late, cudaStream_t s);

// Training state of one hp_sur_train call: the packed weight image and the
// per-CTA gradient slots, owned by the call.
struct MlpTrain {
    unsigned char* img = nullptr;
    float* part = nullptr;
    int64_t grid = 0;  // CTAs of the gradient kernel for a batch of `rows`
    int64_t rows = 0;
};
// allocates the buffers for batches of `rows` rows and packs params
int mlp_train_begin(const float* params, int64_t rows, MlpTrain* t, cudaStream_t s);
// gradients of the batch (X, Y: t->rows rows) and the Adam step `step`;
// *loss (device, may be null) receives the batch loss
int mlp_train_step(MlpTrain* t, float* params, float* m, float* v, const float* X, const float* Y, int32_t step,
                   float lr, float beta1, float beta2, float eps, float* loss, cudaStream_t s);
// The whole run in one cooperative launch (every CTA resident, grid barriers
// between a step's gradients and its update): step s takes minibatch (s - 1) mod
// n_batches of X, Y (t->rows rows each) and sched[3 (s - 1) ..] = (lr, 1 - beta1^t,
// 1 - beta2^t) (device); loss_log (device float[steps], may be null) and
// *loss_last (device, may be null) receive the batch losses.  *ran = false (and
// nothing done) when the device cannot keep every CTA resident.
int mlp_train_loop(MlpTrain* t, float* params, float* m, float* v, const float* X, const float* Y, int64_t n_batches,
                   int32_t steps, const float* sched, float beta1, float beta2, float eps, float* loss_log,
                   float* loss_last, cudaStream_t s, bool* ran);
void mlp_train_end(MlpTrain* t, cudaStream_t s);
}  // namespace hp
