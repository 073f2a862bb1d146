// Lean 3D kernel of the fused checkerboard sweep (Eq. (7), Sec. 4) for the
// 26-neighbour simple cubic lattice, built to spend few instructions per
// site-update.
//
// Colours c = (x&1) + 2(y&1) + 4(z&1): one MCS is two launches, the even planes
// (colours 0-3, their z-neighbours the odd planes as they were) and then the odd
// planes (colours 4-7, their z-neighbours the even planes as just updated).  One
// CTA = one 64 x WY window of one plane with its two z-neighbour windows: q (and,
// with material points, mp) of the three planes, filled by 16-byte asynchronous
// copies that every thread issues (a few hundred small bulk copies from one warp
// queue up behind each other in the copy engine; spread over all threads they
// overlap the draws).  The window keeps a halo of four columns and two
// rows on each side (the exact region of the four in-plane phases, as in the 2D
// Moore tiles), so the core is (64 - 8) x (WY - 4).
//
// Three ideas keep the instruction count down:
//  * every random number of the launch is drawn while the window is in flight:
//    each thread owns a fixed set of sites of each phase (lane = column of the
//    colour sub-grid, warp = rows) and keeps their neighbour choice k and
//    acceptance draw u1 in registers, so Philox overlaps the memory latency;
//  * there is no interior test: a site proposes its k-th neighbour's grain and
//    only proposals of another grain (about a fifth of the sites in a
//    polycrystal) go on to a block-wide queue;
//  * the queue is worked by consecutive threads (whole warps busy), which count
//    both grains among the 26 neighbours with two shared loads per row and run
//    the integer Metropolis test of Sec. 4.
// Each phase is then: propose + enqueue, barrier, test + flip, barrier.
#include <string.h>

#include <cudaTypedefs.h>

#include "sweep.cuh"

namespace hp {
namespace {

__device__ int g_lean_err;

// Tiled TMA descriptors of the launch's source arrays (3D, Lx x Ly x Lz int32,
// box 64 x WY x 1); zeroed when a window is never copied by TMA.  `tab` maps a
// per-material-point field table laid out like the lattice (entry p belongs to
// the point that started at site p).
struct alignas(64) LeanMaps {
    CUtensorMap q_in, q_nb, mp_in, mp_nb, tab;
    int ok;   // 1: the q (and mp) descriptors are valid
    int pf;   // 1: `tab` is valid (the field table is prefetched into L2)
};

__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar) : "memory");
}

// Bring one box of a mapped array into L2 (a hint: nothing lands in shared
// memory and nothing is waited for).
__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap* map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z) : "memory");
}


template <int WY, bool HASMP>
struct LeanCfg {
    static constexpr int kLT = 256, NW = kLT / 32;
    static constexpr int WX = 64, HX = 4, HY = 2, TX = WX - 2 * HX, TY = WY - 2 * HY;
    static constexpr int PS = WX * WY;             // one plane window, ints
    static constexpr int NA = HASMP ? 6 : 3;       // q(z-1) q(z) q(z+1) [mp(z-1) mp(z) mp(z+1)]
    static constexpr int SX = WX / 2, SY = WY / 2, NSUB = SX * SY;  // sites of one colour in the window
    static constexpr int PER = (NSUB + kLT - 1) / kLT;               // of them per thread
    static_assert(SX == 32 && WY % 2 == 0 && TY % 2 == 0 && PER <= 4, "lean window shape");
    // blocks per SM: shared memory allows 4 with the material-point planes when
    // WY <= 32 (3 above), 5 without them
    static constexpr int MINB = HASMP ? (WY <= 32 ? 4 : 3) : 5;
    static constexpr size_t smem() { return 128 + 4 * (size_t)NA * PS + 8 * (size_t)NSUB + 4 * 32 + 4 * 4 + 8; }
    __host__ __device__ static constexpr int ylo(int p) { return 1 + (p >> 1); }
};

// One block, nothing in flight: an mbarrier that expects one arrival, waited
// on by the whole block with a short limit.  With `late` the arrival comes from
// thread 32 after two limits (the first wait gives up, the drain sees it: flag
// 1); otherwise it never comes (the drain runs out as well: flag 2).
__global__ void k_wait_probe(long long limit, int late) {
    __shared__ unsigned long long bar;
    const uint32_t mb = s_addr(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (late && threadIdx.x == 32) {
        const long long t0 = clock64();
        while (clock64() - t0 < 2 * limit) {
        }
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
    }
    wait_or_drain(mb, &g_lean_err, limit);
}

// One window (tile `tile` of plane 2 zidx + a.zpar) of one lattice; maps NULL
// when no window of this launch is copied by TMA boxes.
// KEYED: the Philox round keys come from a.rk (launch parameters); otherwise
// every thread steps the key from a.seed.
template <int WY, int FIELD, bool HASMP, bool KEYED>
__device__ __forceinline__ void lean_body(const PlaneArgs& a, const LeanMaps* maps, const int tile, const int zidx,
                                          unsigned char* raw) {
    using Cfg = LeanCfg<WY, HASMP>;
    constexpr int WX = Cfg::WX, PS = Cfg::PS, NA = Cfg::NA, NSUB = Cfg::NSUB, PER = Cfg::PER, kLT = Cfg::kLT;
    constexpr int NW = Cfg::NW;
    int32_t* base = reinterpret_cast<int32_t*>(raw + ((128u - (s_addr(raw) & 127u)) & 127u));
    int32_t* Q = base + PS;                                       // q of plane z (z-1 at -PS, z+1 at +PS)
    int32_t* MP = base + 4 * PS;                                  // mp of plane z, same layout
    uint2* queue = reinterpret_cast<uint2*>(base + NA * PS);      // NSUB entries
    int* off = reinterpret_cast<int*>(queue + NSUB);              // 26 neighbour offsets (+ pad)
    int* qn = off + 32;                                           // 4 phase counters
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(qn + 4);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
    const int x0 = tx * Cfg::TX, y0 = ty * Cfg::TY;
    const int z = 2 * zidx + a.zpar;
    const int zlo = wrapi(z - 1, a.Lz), zhi = wrapi(z + 1, a.Lz);
    const int64_t sxy = (int64_t)a.Lx * a.Ly;
    const bool fast = a.fast != 0;
    auto gx_of = [&](int col) { return fast ? wrap1(x0 - 4 + col, a.Lx) : wrapi(x0 - 4 + col, a.Lx); };
    auto gy_of = [&](int r) { return fast ? wrap1(y0 - 2 + r, a.Ly) : wrapi(y0 - 2 + r, a.Ly); };
    auto src = [&](int arr) -> const int32_t* {
        const int pl = arr % 3;
        const int zz = pl == 0 ? zlo : (pl == 1 ? z : zhi);
        if (arr < 3) return (pl == 1 ? a.q_in : a.q_nb) + sxy * zz;
        return (pl == 1 ? a.mp_in : a.mp_nb) + sxy * zz;
    };

    // ---- window in flight ----------------------------------------------------
    // A window inside the lattice arrives as one tiled TMA box per array (64 x WY
    // of plane z, one request each, completing on an mbarrier that warp 0 polls).
    // A window that crosses the periodic edge is filled with 16-byte asynchronous
    // copies issued by every thread (4 ints of one window row each: x0 - 4 and Lx
    // are multiples of 4, so a chunk never straddles the edge).  Either way the
    // copies land while the draws below run.
    const bool vec = a.Lx % 4 == 0 && ((uintptr_t)a.q_in & 15u) == 0 && ((uintptr_t)a.q_nb & 15u) == 0 &&
                     (!HASMP || (((uintptr_t)a.mp_in & 15u) == 0 && ((uintptr_t)a.mp_nb & 15u) == 0));
    const bool boxed = vec && maps && maps->ok && x0 >= 4 && x0 - 4 + WX <= a.Lx && y0 >= 2 && y0 - 2 + WY <= a.Ly;
    if (tid < 26) {
        const int kk = tid + (tid >= 13);
        off[tid] = (kk / 9 - 1) * PS + ((kk / 3) % 3 - 1) * WX + (kk % 3 - 1);
    }
    if (tid < 4) qn[tid] = 0;
    const uint32_t mb = s_addr(mbar);
    if (boxed) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                         "r"((uint32_t)(NA * PS * 4)) : "memory");
            const int xs = x0 - 4, ys = y0 - 2;
            tma_box(s_addr(base), &maps->q_nb, xs, ys, zlo, mb);
            tma_box(s_addr(base + PS), &maps->q_in, xs, ys, z, mb);
            tma_box(s_addr(base + 2 * PS), &maps->q_nb, xs, ys, zhi, mb);
            if (HASMP) {
                tma_box(s_addr(base + 3 * PS), &maps->mp_nb, xs, ys, zlo, mb);
                tma_box(s_addr(base + 4 * PS), &maps->mp_in, xs, ys, z, mb);
                tma_box(s_addr(base + 5 * PS), &maps->mp_nb, xs, ys, zhi, mb);
            }
            // The test stages look up the field of the window's material points.
            // A point moves only a few sites under grain growth, so most of them
            // lie in the table's boxes at the window's own coordinates: start
            // those towards L2 now, a few thousand cycles before the lookups.
            if (FIELD == 2 && maps->pf) {
                tma_prefetch_l2(&maps->tab, xs, ys, zlo);
                tma_prefetch_l2(&maps->tab, xs, ys, z);
                tma_prefetch_l2(&maps->tab, xs, ys, zhi);
            }
        }
    } else if (vec) {
        constexpr int CH = WX / 4;  // chunks per window row
        for (int i = tid; i < NA * WY * CH; i += kLT) {
            const int arr = i / (WY * CH), rem = i - arr * (WY * CH), r = rem / CH, c = rem - r * CH;
            const int gx = fast ? wrap1(x0 - 4 + 4 * c, a.Lx) : wrapi(x0 - 4 + 4 * c, a.Lx);
            const int32_t* g = src(arr) + (int64_t)a.Lx * gy_of(r) + gx;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s_addr(base + arr * PS + r * WX + 4 * c)),
                         "l"(g) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // every thread sees the barrier initialised (and the offsets) before it waits
    __syncthreads();

    // ---- every draw of the launch, while the copies land -------------------
    // site m of phase p for this thread: colour sub-grid column = lane, row
    // j = warp + NW m; window column 2 lane + (p & 1), row 2 j + (p >> 1).  Its
    // Philox unit gx + Lx (gy + Ly z) is a row base plus a column, each wrapped
    // once per thread.  Whether the row lies in the phase's region is the same
    // for the whole warp (a branch); whether the column does is a select, so a
    // warp never diverges here (the few edge lanes draw and drop the result).
    const uint32_t cz = 4u * (uint32_t)a.zpar;
    const uint64_t gxc[2] = {(uint64_t)gx_of(2 * lane), (uint64_t)gx_of(2 * lane + 1)};
    uint64_t rowb[PER][2];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int j = warp + NW * m;
#pragma unroll
        for (int r = 0; r < 2; ++r)
            rowb[m][r] = j < Cfg::SY ? (uint64_t)a.Lx * ((uint64_t)gy_of(2 * j + r) + (uint64_t)a.Ly * (uint64_t)z) : 0;
    }
    uint32_t u1[4][PER];
    uint32_t kk[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        kk[p] = 0;
        const int x = 2 * lane + (p & 1), loy = Cfg::ylo(p);
        const bool colok = x >= p + 1 && x < WX - p - 1;
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int j = warp + NW * m, y = 2 * j + (p >> 1);
            u1[p][m] = 0;
            if (j < Cfg::SY && y >= loy && y < WY - loy) {
                const uint64_t unit = rowb[m][p >> 1] + gxc[p & 1];
                const uint4 u =
                    KEYED ? philox10_keyed(a.rk, make_uint4((uint32_t)unit, (uint32_t)(unit >> 32), a.sweep,
                                                            (kTagSweep << 24) | (cz + (uint32_t)p)))
                          : draw(a.seed, unit, a.sweep, kTagSweep, cz + (uint32_t)p);
                u1[p][m] = u.y;
                kk[p] |= (colok ? __umulhi(u.x, 26u) + 1u : 0u) << (8 * m);  // 0 marks "no site"
            }
        }
    }

    if (boxed) {
        if (!wait_or_drain(mb, &g_lean_err)) return;
    } else if (vec) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    } else {
        for (int i = tid; i < NA * PS; i += kLT) {
            const int arr = i / PS, rem = i - arr * PS, r = rem / WX, c = rem - r * WX;
            base[arr * PS + rem] = src(arr)[(int64_t)a.Lx * wrapi(y0 - 2 + r, a.Ly) + wrapi(x0 - 4 + c, a.Lx)];
        }
        __syncthreads();
    }

    const unsigned lt = (1u << lane) - 1u;
    // kernel parameters of the test stage, once
    const int32_t* __restrict__ ftab = a.table;
    const uint32_t ftab_n = a.table_n;
    const uint32_t* __restrict__ thr = a.thr;
    const int32_t Jc = a.J, Dmax = a.D;
    constexpr int SAFE = (WY / 2) * WX + WX / 2;  // a window position whose 26 neighbours all lie in the window
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        // ---- propose: the k-th neighbour's grain; queue those of another grain.
        // An empty slot (kc = 0) reads at SAFE instead, so every lane loads and
        // no branch is taken.
        uint32_t e[PER];
        unsigned bal[PER];
        int tot = 0;
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const uint32_t kc = (kk[p] >> (8 * m)) & 255u;
            const int pos = (2 * (warp + NW * m) + (p >> 1)) * WX + 2 * lane + (p & 1);
            const int k = kc ? (int)kc - 1 : 0;
            const int pq = kc ? pos : SAFE;
            const int32_t qa = Q[pq + off[k]], qb = Q[pq];
            const bool pr = (kc != 0u) & (qa != qb);
            e[m] = (uint32_t)pos | ((uint32_t)k << 16);
            bal[m] = __ballot_sync(0xFFFFFFFFu, pr);
            tot += __popc(bal[m]);
        }
        if (tot) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(qn + p, tot);
            b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                if (bal[m] & (1u << lane)) queue[b0 + __popc(bal[m] & lt)] = make_uint2(e[m], u1[p][m]);
                b0 += __popc(bal[m]);
            }
        }
        __syncthreads();
        // ---- test: count both grains among the 26 neighbours, Metropolis ------
        const int n = qn[p];
        for (int i = tid; i < n; i += kLT) {
            const uint2 w = queue[i];
            const int pos = (int)(w.x & 0xFFFFu), o = off[w.x >> 16];
            const int32_t* c = Q + pos;
            const int32_t qi = c[0], qj = c[o];
            int32_t mpj = 0, bi = 0, bj = 0;
            if (HASMP) mpj = MP[pos + o];
            if (FIELD == 1) { bi = tab(ftab, ftab_n, qi); bj = tab(ftab, ftab_n, qj); }
            if (FIELD == 2) { bi = tab(ftab, ftab_n, MP[pos]); bj = tab(ftab, ftab_n, mpj); }
            int so = 0, sn = 0;
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    const int32_t* r = c + dz * PS + dy * WX;
                    int32_t v0, v1, v2;
                    if (p & 1) {  // column odd: (x-1, x) is an aligned pair
                        const int2 l = *reinterpret_cast<const int2*>(r - 1);
                        v0 = l.x; v1 = l.y; v2 = r[1];
                    } else {      // column even: (x, x+1) is an aligned pair
                        const int2 h = *reinterpret_cast<const int2*>(r);
                        v0 = r[-1]; v1 = h.x; v2 = h.y;
                    }
                    so += (v0 == qi) + (v2 == qi);
                    sn += (v0 == qj) + (v2 == qj);
                    if (dz != 0 || dy != 0) { so += v1 == qi; sn += v1 == qj; }
                }
            const int32_t d = Jc * (so - sn) + (bj - bi);
            if (metropolis(d, Dmax, thr, w.y)) {
                Q[pos] = qj;
                if (HASMP) MP[pos] = mpj;
            }
        }
        __syncthreads();
    }

    // ---- write the core: rows [2, WY - 2), columns [4, WX - 4) ---------------
    int32_t* qo = a.q_out + sxy * z;
    int32_t* mpo = HASMP ? a.mp_out + sxy * z : nullptr;
    constexpr int CQ = WX / 4 - 2;
    for (int i = tid; i < Cfg::TY * CQ; i += kLT) {
        const int cy = i / CQ, qq = 1 + (i - cy * CQ);
        const int gx = x0 + 4 * (qq - 1), gy = y0 + cy;
        if (gx >= a.Lx || gy >= a.Ly) continue;
        const int li = (cy + 2) * WX + 4 * qq;
        const int64_t o = gx + (int64_t)a.Lx * gy;
        if (a.vec) {
            *reinterpret_cast<int4*>(qo + o) = *reinterpret_cast<const int4*>(Q + li);
            if (HASMP) *reinterpret_cast<int4*>(mpo + o) = *reinterpret_cast<const int4*>(MP + li);
        } else {
#pragma unroll
            for (int jx = 0; jx < 4; ++jx) {
                if (gx + jx >= a.Lx) break;
                qo[o + jx] = Q[li + jx];
                if (HASMP) mpo[o + jx] = MP[li + jx];
            }
        }
    }
}

template <int WY, int FIELD, bool HASMP>
__global__ void __launch_bounds__(LeanCfg<WY, HASMP>::kLT, LeanCfg<WY, HASMP>::MINB)
    k_lean26(const __grid_constant__ PlaneArgs a, const __grid_constant__ LeanMaps maps) {
    extern __shared__ __align__(16) unsigned char raw[];
    lean_body<WY, FIELD, HASMP, true>(a, &maps, (int)blockIdx.x, (int)blockIdx.y, raw);
}

// Many independent lattices in one launch: block b belongs to the replica r
// with start[r] <= b < start[r+1]; within it b - start[r] = zidx * tiles + tile.
// Windows are filled by the asynchronous 16-byte copies.
template <int WY, int FIELD, bool HASMP>
__global__ void __launch_bounds__(LeanCfg<WY, HASMP>::kLT, HASMP ? 3 : 4)
    k_lean26_batch(const PlaneArgs* __restrict__ args, const int64_t* __restrict__ start, int R, uint32_t sweep_add) {
    extern __shared__ __align__(16) unsigned char raw[];
    __shared__ PlaneArgs sa;
    __shared__ int s_tile, s_zidx;
    if (threadIdx.x == 0) {
        const int64_t blk = blockIdx.x;
        int lo = 0, hi = R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= blk) lo = mid; else hi = mid - 1;
        }
        sa = args[lo];
        sa.sweep += sweep_add;
        const int64_t local = blk - start[lo];
        s_zidx = (int)(local / sa.tiles);
        s_tile = (int)(local - (int64_t)s_zidx * sa.tiles);
    }
    __syncthreads();
    lean_body<WY, FIELD, HASMP, false>(sa, nullptr, s_tile, s_zidx, raw);
}

PFN_cuTensorMapEncodeTiled_v12000 map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Descriptor of one int32 lattice array (Lx x Ly x Lz) with a 64 x WY x 1 box;
// false when it cannot be encoded (the kernel then copies every window with
// asynchronous 16-byte copies instead).
bool encode_box(CUtensorMap* m, const void* base, const PlaneArgs& a, int WY) {
    memset(m, 0, sizeof(*m));
    PFN_cuTensorMapEncodeTiled_v12000 enc = map_encoder();
    if (!enc || !base || a.Lx % 4 != 0 || ((uintptr_t)base & 15u) != 0) return false;
    cuuint64_t dims[3] = {(cuuint64_t)a.Lx, (cuuint64_t)a.Ly, (cuuint64_t)a.Lz};
    cuuint64_t strides[2] = {(cuuint64_t)a.Lx * 4, (cuuint64_t)a.Lx * (cuuint64_t)a.Ly * 4};
    cuuint32_t box[3] = {64u, (cuuint32_t)WY, 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_INT32, 3u, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Opt both kernels of an instantiation into their dynamic shared memory, once.
template <int WY, int FIELD, bool HASMP>
int lean_configure(size_t smem) {
    static bool configured = false;
    if (!configured) {
        HP_CUDA(cudaFuncSetAttribute(k_lean26<WY, FIELD, HASMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        HP_CUDA(cudaFuncSetAttribute(k_lean26_batch<WY, FIELD, HASMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        configured = true;
    }
    return HP_OK;
}
#define HP_CUDA_ONCE_ATTR(WY_, F_, M_, SM_)                   \
    do {                                                      \
        const int rc_ = lean_configure<WY_, F_, M_>(SM_);     \
        if (rc_) return rc_;                                  \
    } while (0)

template <int WY, int FIELD, bool HASMP>
int launch_lean(const PlaneArgs& a, int planes, cudaStream_t s) {
    using Cfg = LeanCfg<WY, HASMP>;
    constexpr size_t smem = Cfg::smem();
    HP_CUDA_ONCE_ATTR(WY, FIELD, HASMP, smem);
    if (a.tiles == 0 || planes == 0) return HP_OK;
    LeanMaps maps;
    memset(&maps, 0, sizeof(maps));
    bool ok = a.Lx >= 64 && encode_box(&maps.q_in, a.q_in, a, WY) && encode_box(&maps.q_nb, a.q_nb, a, WY);
    if (ok && HASMP) ok = encode_box(&maps.mp_in, a.mp_in, a, WY) && encode_box(&maps.mp_nb, a.mp_nb, a, WY);
    maps.ok = ok ? 1 : 0;
    // a per-point field table of one entry per site shares the lattice's layout
    if (ok && FIELD == 2 && a.table_n == (uint32_t)((uint64_t)a.Lx * a.Ly * a.Lz) &&
        (uint64_t)a.Lx * a.Ly * a.Lz <= 0xFFFFFFFFull)
        maps.pf = encode_box(&maps.tab, a.table, a, WY) ? 1 : 0;
    count_launch();
    k_lean26<WY, FIELD, HASMP><<<dim3((unsigned)a.tiles, (unsigned)planes), Cfg::kLT, smem, s>>>(a, maps);
    HP_LAUNCH_CHECK("k_lean26");
    return HP_OK;
}

template <int WY, int FIELD, bool HASMP>
int launch_lean_batch(const PlaneArgs* d_args, const int64_t* d_start, int R, int64_t blocks, uint32_t sweep_add,
                      cudaStream_t s) {
    using Cfg = LeanCfg<WY, HASMP>;
    constexpr size_t smem = Cfg::smem();
    HP_CUDA_ONCE_ATTR(WY, FIELD, HASMP, smem);
    if (blocks == 0) return HP_OK;  // configure only (outside a graph capture)
    count_launch();
    k_lean26_batch<WY, FIELD, HASMP><<<(unsigned)blocks, Cfg::kLT, smem, s>>>(d_args, d_start, R, sweep_add);
    HP_LAUNCH_CHECK("k_lean26_batch");
    return HP_OK;
}

template <int WY>
int lean_fm_batch(const PlaneArgs* d_args, const int64_t* d_start, int R, int64_t blocks, uint32_t sweep_add, int field,
                  bool m, cudaStream_t s) {
    if (field == HP_FIELD_POINT) return launch_lean_batch<WY, 2, true>(d_args, d_start, R, blocks, sweep_add, s);
    if (field == HP_FIELD_GRAIN)
        return m ? launch_lean_batch<WY, 1, true>(d_args, d_start, R, blocks, sweep_add, s)
                 : launch_lean_batch<WY, 1, false>(d_args, d_start, R, blocks, sweep_add, s);
    return m ? launch_lean_batch<WY, 0, true>(d_args, d_start, R, blocks, sweep_add, s)
             : launch_lean_batch<WY, 0, false>(d_args, d_start, R, blocks, sweep_add, s);
}

template <int WY>
int lean_fm(const PlaneArgs& a, int field, bool m, int planes, cudaStream_t s) {
    if (field == HP_FIELD_POINT) return launch_lean<WY, 2, true>(a, planes, s);
    if (field == HP_FIELD_GRAIN) return m ? launch_lean<WY, 1, true>(a, planes, s) : launch_lean<WY, 1, false>(a, planes, s);
    return m ? launch_lean<WY, 0, true>(a, planes, s) : launch_lean<WY, 0, false>(a, planes, s);
}

}  // namespace

int lean_launch(const PlaneArgs& a, int field, bool hasmp, int planes, int WY, cudaStream_t s) {
    if (WY == 44) return lean_fm<44>(a, field, hasmp, planes, s);
    if (WY == 40) return lean_fm<40>(a, field, hasmp, planes, s);
    if (WY == 36) return lean_fm<36>(a, field, hasmp, planes, s);
    if (WY == 32) return lean_fm<32>(a, field, hasmp, planes, s);
    return set_error(HP_ERR_ARG, "sweep: no lean kernel of this shape");
}

int lean_launch_batch(const PlaneArgs* d_args, const int64_t* d_start, int R, int64_t blocks, uint32_t sweep_add,
                      int field, bool hasmp, int WY, cudaStream_t s) {
    if (WY == 44) return lean_fm_batch<44>(d_args, d_start, R, blocks, sweep_add, field, hasmp, s);
    if (WY == 40) return lean_fm_batch<40>(d_args, d_start, R, blocks, sweep_add, field, hasmp, s);
    if (WY == 36) return lean_fm_batch<36>(d_args, d_start, R, blocks, sweep_add, field, hasmp, s);
    if (WY == 32) return lean_fm_batch<32>(d_args, d_start, R, blocks, sweep_add, field, hasmp, s);
    return set_error(HP_ERR_ARG, "sweep: no lean kernel of this shape");
}

int lean_wait_probe(long long limit, int late, cudaStream_t s) {
    if (limit < 1 || limit > kWaitCycles) return set_error(HP_ERR_ARG, "wait probe: limit out of range");
    count_launch();
    k_wait_probe<<<1, 64, 0, s>>>(limit, late);
    HP_LAUNCH_CHECK("k_wait_probe");
    return HP_OK;
}

int lean_status(int* timed_out) {
    int v = 0, zero = 0;
    HP_CUDA(cudaMemcpyFromSymbol(&v, g_lean_err, sizeof(int)));
    if (v) HP_CUDA(cudaMemcpyToSymbol(g_lean_err, &zero, sizeof(int)));
    *timed_out = v;
    return HP_OK;
}

}  // namespace hp
