// Strip kernel: the fused checkerboard sweep (Eq. (7), Sec. 4) with one warp
// per strip and no block-wide barrier.
//
// A strip is a window of W = core + 8 columns of one lattice plane (a halo of
// four columns on each side) and the core rows [y0, y0 + ty).  Lane l holds
// columns CPL*l .. CPL*l + CPL - 1 of the window.  The warp walks down the
// strip two rows per step with the colour phases skewed so that every phase
// sees its neighbours in the state the synchronous half-steps of Sec. 4 give
// them (rows relative to y0):
//   Moore planes (colour = (x&1) + 2(y&1) [+ 4(z&1)]):
//     step k: phases 0, 1 on even row 2k (odd rows 2k +- 1 still old), then
//             phases 2, 3 on odd row 2k-1 (even rows 2k-2, 2k already new);
//   4-neighbour planes (colour = (x+y)&1):
//     step k: phase 0 on rows 2k-1, 2k, then phase 1 on rows 2k-2, 2k-1.
// After step k rows 2k-2 and 2k-1 are final and are written to the output
// buffer.  In 3D one launch handles the planes of one parity; the planes of
// the other parity are read-only neighbours (old ones for even planes, the new
// ones for odd planes), exactly as in the plane kernel.  Columns and rows
// outside the core are computed from an incomplete neighbourhood and never
// written: each phase narrows the columns it updates by one on each side, and
// the halo of four columns covers the four in-plane phases.
//
// Rows stream through an eight-row ring in shared memory (own q, own mp, and
// in 3D the q rows of planes z-1 and z+1), two rows per mbarrier, filled by
// bulk TMA copies (cp.async.bulk) that lane 0 issues two row pairs ahead; a
// row crossing the periodic x boundary is two copies.  Lattices whose rows are
// narrower than a window, or not 16-byte aligned, load with per-lane reads.
//
// In each phase row a lane tests its sites of the colour for an all-equal
// neighbourhood (OR of XORs); the remaining sites are compacted through a
// per-warp queue so that each lane of a pass draws Philox for a different
// site and runs its Metropolis update.  Waits on the mbarriers give up after
// about two seconds, set g_strip_err and return once the copies in flight
// have landed (bounded as well).
#include "sweep.cuh"

namespace hp {
namespace {

constexpr int kStripWarps = 4;
__device__ int g_strip_err;

struct StripGeo {
    int core;   // core columns per strip (multiple of 4)
    int W;      // window columns = core + 8
    int nsx;    // strips across x
    int ty;     // core rows per strip (even)
    int nsy;    // strips down y
    int items;  // nsx * nsy * planes
    int tma;    // 1: rows arrive by bulk TMA copies
};

template <int NBR, int CPL, bool HASMP>
struct StripCfg {
    static constexpr bool Z = NBR == 26;
    static constexpr int ARR = 1 + (HASMP ? 1 : 0) + (Z ? 2 : 0);  // q, mp, q(z-1), q(z+1)
    static constexpr int A_MP = 1, A_LO = HASMP ? 2 : 1, A_HI = A_LO + 1;
    static constexpr int WP = 32 * CPL;       // widest window
    static constexpr int RS = WP + 8;         // row stride in ints: 4 padding ints on each side
    // rows in the ring: a step reads rows 2k-2 .. 2k+1 (Moore) or 2k-3 .. 2k+1
    // (4-neighbour), plus the row pair in flight
    static constexpr int RING = NBR == 4 ? 8 : 6;
    static constexpr int QCAP = 16 * CPL;     // sites of one colour in a window row
    static constexpr int HDR = 8 + QCAP;      // 4 mbarriers (8 ints) + queue
    static constexpr int WARP_INTS = HDR + RING * ARR * RS;
    static_assert((HDR * 4) % 16 == 0 && (RS * 4) % 16 == 0, "16-byte aligned rows");
    static size_t smem() { return sizeof(int32_t) * (size_t)WARP_INTS * kStripWarps; }
};

template <int NBR, int CPL, int FIELD, bool HASMP>
struct Strip {
    using Cfg = StripCfg<NBR, CPL, HASMP>;
    static constexpr bool Z = Cfg::Z;
    static constexpr int ARR = Cfg::ARR, RS = Cfg::RS, SPL = CPL / 2;
    static constexpr int M = NBR;

    const PlaneArgs& a;
    const StripGeo& g;
    int32_t* ring;
    int32_t* queue;
    int lane, x0, y0, z, zlo, zhi;
    int64_t sxy;
    uint32_t sweep;

    __device__ Strip(const PlaneArgs& a_, const StripGeo& g_) : a(a_), g(g_) {}

    __device__ __forceinline__ int32_t* row(int r, int arr) const {
        return ring + (((r + 2 * Cfg::RING) % Cfg::RING) * ARR + arr) * RS + 4;
    }
    // periodic column of window column c (one add on the TMA path, W <= Lx)
    __device__ __forceinline__ int gcol(int c) const {
        return g.tma ? wrap1(x0 - 4 + c, a.Lx) : wrapi(x0 - 4 + c, a.Lx);
    }
    __device__ __forceinline__ const int32_t* src(int arr) const {
        if (arr == 0) return a.q_in + sxy * z;
        if (HASMP && arr == Cfg::A_MP) return a.mp_in + sxy * z;
        return a.q_nb + sxy * (arr == Cfg::A_LO ? zlo : zhi);
    }

    // rows r0, r0 + 1 of every array; TMA: lane 0 issues, completion on mb
    __device__ __forceinline__ void issue(int r0, uint32_t mb) const {
        if (g.tma) {
            if (lane == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                             "r"((uint32_t)(2 * ARR * g.W * 4)) : "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int gy = wrapi(y0 + r0 + h, a.Ly);
#pragma unroll
                    for (int arr = 0; arr < ARR; ++arr)
                        copy_row(row(r0 + h, arr), src(arr) + (int64_t)a.Lx * gy, x0 - 4, g.W, a.Lx, mb);
                }
            }
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gy = wrapi(y0 + r0 + h, a.Ly);
#pragma unroll
                for (int arr = 0; arr < ARR; ++arr) {
                    const int32_t* s = src(arr) + (int64_t)a.Lx * gy;
                    int32_t* d = row(r0 + h, arr);
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int c = CPL * lane + i;
                        if (c < g.W) d[c] = s[gcol(c)];
                    }
                }
            }
        }
    }

    // a window row as CPL values plus the one edge column this parity needs
    template <int PX>
    __device__ __forceinline__ void load(const int32_t* R, int32_t (&v)[CPL + 2]) const {
        const int c0 = CPL * lane;
        if (CPL == 8) {
            const int4 t = *reinterpret_cast<const int4*>(R + c0), w = *reinterpret_cast<const int4*>(R + c0 + 4);
            v[1] = t.x; v[2] = t.y; v[3] = t.z; v[4] = t.w;
            v[5] = w.x; v[6] = w.y; v[7] = w.z; v[8] = w.w;
        } else if (CPL == 4) {
            const int4 t = *reinterpret_cast<const int4*>(R + c0);
            v[1] = t.x; v[2] = t.y; v[3] = t.z; v[4] = t.w;
        } else {
            const int2 t = *reinterpret_cast<const int2*>(R + c0);
            v[1] = t.x; v[2] = t.y;
        }
        if (PX == 0) { v[0] = R[c0 - 1]; v[CPL + 1] = 0; }
        else { v[0] = 0; v[CPL + 1] = R[c0 + CPL]; }
    }

    // Metropolis update of the site at window column col of row r (gy its
    // periodic row, rb = sxy * z + Lx * gy).
    __device__ __forceinline__ void update(int r, int col, uint32_t colour, int gy, int64_t rb) const {
        const int gx = gcol(col);
        const int64_t gi = rb + gx;
        const uint4 u = draw(a.seed, (uint64_t)gi, sweep, kTagSweep, colour);
        const int kp = (int)__umulhi(u.x, (uint32_t)M);
        int dx, dy, dz;
        if (NBR == 4) Geo<2, 4>::off(kp, dx, dy, dz);
        else if (NBR == 8) Geo<2, 8>::off(kp, dx, dy, dz);
        else Geo<3, 26>::off(kp, dx, dy, dz);
        int32_t* own = row(r, 0);
        const int32_t qi = own[col];
        const int32_t qj = row(r + dy, dz == 0 ? 0 : (dz < 0 ? Cfg::A_LO : Cfg::A_HI))[col + dx];
        if (qj == qi) return;
        int32_t mpj = 0;
        if (HASMP) {
            if (dz == 0) mpj = row(r + dy, Cfg::A_MP)[col + dx];
            else
                mpj = __ldg(a.mp_nb + wrap1(gx + dx, a.Lx) + (int64_t)a.Lx * wrap1(gy + dy, a.Ly) +
                            sxy * (dz < 0 ? zlo : zhi));
        }
        int32_t bi = 0, bj = 0;
        if (FIELD == 1) { bi = tab(a.table, a.table_n, qi); bj = tab(a.table, a.table_n, qj); }
        if (FIELD == 2) { bi = tab(a.table, a.table_n, row(r, Cfg::A_MP)[col]); bj = tab(a.table, a.table_n, mpj); }
        int so = 0, sn = 0;
        if (NBR == 4) {
            const int32_t n0 = own[col - 1], n1 = own[col + 1], n2 = row(r - 1, 0)[col], n3 = row(r + 1, 0)[col];
            so = (n0 == qi) + (n1 == qi) + (n2 == qi) + (n3 == qi);
            sn = (n0 == qj) + (n1 == qj) + (n2 == qj) + (n3 == qj);
        } else {
#pragma unroll
            for (int ddy = -1; ddy <= 1; ++ddy) {
#pragma unroll
                for (int ddx = -1; ddx <= 1; ++ddx) {
                    if (ddx || ddy) {
                        const int32_t n = row(r + ddy, 0)[col + ddx];
                        so += n == qi; sn += n == qj;
                    }
                    if (Z) {
                        const int32_t l = row(r + ddy, Cfg::A_LO)[col + ddx], h = row(r + ddy, Cfg::A_HI)[col + ddx];
                        so += (l == qi) + (h == qi);
                        sn += (l == qj) + (h == qj);
                    }
                }
            }
        }
        const int32_t d = a.J * (so - sn) + (bj - bi);
        if (metropolis(d, a.D, a.thr, u.y)) {
            own[col] = qj;
            if (HASMP) row(r, Cfg::A_MP)[col] = mpj;
        }
    }

    // One colour phase on row r: sites at window columns of parity PX in
    // [p + 1, W - p - 1).
    template <int PX>
    __device__ __forceinline__ void phase_row(int r, int p, uint32_t colour) const {
        const int c0 = CPL * lane;
        int32_t v[CPL + 2];
        int32_t qs[SPL];
        uint32_t acc[SPL];
        load<PX>(row(r, 0), v);
#pragma unroll
        for (int s = 0; s < SPL; ++s) {
            qs[s] = v[1 + PX + 2 * s];
            acc[s] = (v[PX + 2 * s] ^ qs[s]) | (v[2 + PX + 2 * s] ^ qs[s]);
        }
        auto rowacc = [&](const int32_t* R, bool centre) {
            load<PX>(R, v);
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                acc[s] |= v[1 + PX + 2 * s] ^ qs[s];
                if (!centre) acc[s] |= (v[PX + 2 * s] ^ qs[s]) | (v[2 + PX + 2 * s] ^ qs[s]);
            }
        };
        rowacc(row(r - 1, 0), NBR == 4);
        rowacc(row(r + 1, 0), NBR == 4);
        if (Z) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                rowacc(row(r + dy, Cfg::A_LO), false);
                rowacc(row(r + dy, Cfg::A_HI), false);
            }
        }
        const int lo = p + 1, hi = g.W - p - 1;
        const unsigned lt = (1u << lane) - 1u;
        int n = 0;
#pragma unroll
        for (int s = 0; s < SPL; ++s) {
            const int col = c0 + PX + 2 * s;
            const bool b = acc[s] != 0u && col >= lo && col < hi;
            const unsigned m = __ballot_sync(0xFFFFFFFFu, b);
            if (b) queue[n + __popc(m & lt)] = col;
            n += __popc(m);
        }
        if (n == 0) return;
        __syncwarp();
        const int gy = wrapi(y0 + r, a.Ly);
        const int64_t rb = sxy * z + (int64_t)a.Lx * gy;
        for (int k = lane; k < n; k += 32) update(r, queue[k], colour, gy, rb);
        __syncwarp();
    }

    // write row r (0 <= r < ty) of the window core [4, W - 4)
    __device__ __forceinline__ void store(int r) const {
        if (y0 + r >= a.Ly) return;
        const int c0 = CPL * lane;
        const int cb = c0 > 4 ? c0 : 4, ce = c0 + CPL < g.W - 4 ? c0 + CPL : g.W - 4;
        if (cb >= ce) return;
        const int64_t ob = sxy * z + (int64_t)a.Lx * (y0 + r) + (x0 - 4);  // + window column
        const int32_t* R = row(r, 0);
        const int32_t* P = HASMP ? row(r, Cfg::A_MP) : nullptr;
        if (g.tma && cb == c0 && ce == c0 + CPL && x0 - 4 + c0 + CPL <= a.Lx) {
            if (CPL >= 4) {
#pragma unroll
                for (int i = 0; i < CPL; i += 4) {
                    *reinterpret_cast<int4*>(a.q_out + ob + c0 + i) = *reinterpret_cast<const int4*>(R + c0 + i);
                    if (HASMP)
                        *reinterpret_cast<int4*>(a.mp_out + ob + c0 + i) = *reinterpret_cast<const int4*>(P + c0 + i);
                }
            } else {
                *reinterpret_cast<int2*>(a.q_out + ob + c0) = *reinterpret_cast<const int2*>(R + c0);
                if (HASMP) *reinterpret_cast<int2*>(a.mp_out + ob + c0) = *reinterpret_cast<const int2*>(P + c0);
            }
        } else {
            for (int c = cb; c < ce; ++c) {
                if (x0 - 4 + c >= a.Lx) break;
                a.q_out[ob + c] = R[c];
                if (HASMP) a.mp_out[ob + c] = P[c];
            }
        }
    }
};

template <int NBR, int CPL, int FIELD, bool HASMP>
__global__ void __launch_bounds__(32 * kStripWarps)
    k_strip(const __grid_constant__ PlaneArgs a, const __grid_constant__ StripGeo g) {
    using S = Strip<NBR, CPL, FIELD, HASMP>;
    using Cfg = typename S::Cfg;
    extern __shared__ __align__(16) int32_t smem[];
    const int warp = threadIdx.x >> 5;
    const int item = blockIdx.x * kStripWarps + warp;
    if (item >= g.items) return;
    S st(a, g);
    int32_t* ws = smem + warp * Cfg::WARP_INTS;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(ws);
    st.queue = ws + 8;
    st.ring = ws + Cfg::HDR;
    st.lane = threadIdx.x & 31;
    const int sx = item % g.nsx, rest = item / g.nsx;
    const int sy = rest % g.nsy, zi = rest / g.nsy;
    st.x0 = sx * g.core;
    st.y0 = sy * g.ty;
    st.z = Cfg::Z ? 2 * zi + a.zpar : 0;
    st.zlo = Cfg::Z ? wrapi(st.z - 1, a.Lz) : 0;
    st.zhi = Cfg::Z ? wrapi(st.z + 1, a.Lz) : 0;
    st.sxy = (int64_t)a.Lx * a.Ly;
    st.sweep = a.sweep;
    if (g.tma && st.lane == 0) {
        for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(mbar + i)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // pair j = rows 2j - 2, 2j - 1; step k reads pairs k-1 .. k+1 (4-neighbour)
    // or k, k+1 (Moore), and pair k+2 is in flight, filling the ring slots of
    // the pair no longer read
    constexpr int OFF = -2;
    const int K = g.ty / 2, last = K + 1;
    constexpr int NB = Cfg::RING / 2;  // mbarriers in use, one per ring pair
    auto mb = [&](int j) { return s_addr(mbar + (j % NB)); };
    auto par = [&](int j) { return (uint32_t)((j / NB) & 1); };
    auto wait = [&](int j) -> bool {
        if (!g.tma) { __syncwarp(); return true; }
        return __all_sync(0xFFFFFFFFu, wait_parity(mb(j), par(j)));
    };
    st.issue(2 * 0 + OFF, mb(0));
    st.issue(2 * 1 + OFF, mb(1));
    int issued = 1, done = -1;  // pairs 0 .. issued started, 0 .. done landed
    bool ok = wait(0);
    if (ok) done = 0;
    const uint32_t cz = Cfg::Z ? 4u * (uint32_t)a.zpar : 0u;
    for (int k = 0; ok && k <= K; ++k) {
        if (k + 2 <= last) {
            st.issue(2 * (k + 2) + OFF, mb(k + 2));
            issued = k + 2;
        }
        ok = wait(k + 1);
        if (!ok) break;
        done = k + 1;
        if (NBR == 4) {
            st.template phase_row<1>(2 * k - 1, 0, 0u);
            st.template phase_row<0>(2 * k, 0, 0u);
            if (k > 0) {
                st.template phase_row<1>(2 * k - 2, 1, 1u);
                st.template phase_row<0>(2 * k - 1, 1, 1u);
            }
        } else {
            st.template phase_row<0>(2 * k, 0, cz + 0u);
            st.template phase_row<1>(2 * k, 1, cz + 1u);
            if (k > 0) {
                st.template phase_row<0>(2 * k - 1, 2, cz + 2u);
                st.template phase_row<1>(2 * k - 1, 3, cz + 3u);
            }
        }
        if (k > 0) {
            st.store(2 * k - 2);
            st.store(2 * k - 1);
        }
        // the ring slots of pair k - 1 are refilled by TMA in the next step
        if (g.tma) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
    }
    if (!ok) {
        if (st.lane == 0) atomicExch(&g_strip_err, 1);
        // let the copies still in flight land before the warp leaves (bounded)
        for (int j = done + 1; j <= issued; ++j) wait_parity(mb(j), par(j));
    }
}

template <int NBR, int CPL, int FIELD, bool HASMP>
int launch_strip(const PlaneArgs& a, const StripGeo& g, cudaStream_t s) {
    using Cfg = StripCfg<NBR, CPL, HASMP>;
    auto fn = k_strip<NBR, CPL, FIELD, HASMP>;
    const size_t smem = Cfg::smem();
    static bool configured = false;
    if (!configured) {
        HP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    if (g.items == 0) return HP_OK;
    const int blocks = (g.items + kStripWarps - 1) / kStripWarps;
    count_launch();
    fn<<<blocks, 32 * kStripWarps, smem, s>>>(a, g);
    HP_LAUNCH_CHECK("k_strip");
    return HP_OK;
}

template <int NBR, int CPL>
int strip_fm(const PlaneArgs& a, const StripGeo& g, int field, bool m, cudaStream_t s) {
    if (field == HP_FIELD_GRAIN && !m) return launch_strip<NBR, CPL, 1, false>(a, g, s);
    if (field == HP_FIELD_POINT) return launch_strip<NBR, CPL, 2, true>(a, g, s);
    return set_error(HP_ERR_ARG, "sweep: strip variant not built for this field mode");
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

int strip_launch(const PlaneArgs& a, int field, bool hasmp, int nbr, int planes, int cpl, int ty_max,
                 cudaStream_t s) {
    StripGeo g;
    const int maxcore = 32 * cpl - 8;
    g.nsx = (a.Lx + maxcore - 1) / maxcore;
    const int per = (a.Lx + g.nsx - 1) / g.nsx;
    g.core = (per + 3) & ~3;
    g.nsx = (a.Lx + g.core - 1) / g.core;  // every strip starts inside the lattice
    g.W = g.core + 8;
    g.nsy = (a.Ly + ty_max - 1) / ty_max;
    const int pery = (a.Ly + g.nsy - 1) / g.nsy;
    g.ty = (pery + 1) & ~1;
    g.nsy = (a.Ly + g.ty - 1) / g.ty;
    const int64_t items = (int64_t)g.nsx * g.nsy * planes;
    if (items > (int64_t)1 << 30) return set_error(HP_ERR_ARG, "sweep: lattice too large for the strip kernel");
    g.items = (int)items;
    const bool ptr_ok = aligned16(a.q_in) && aligned16(a.q_out) && (!hasmp || (aligned16(a.mp_in) && aligned16(a.mp_out))) &&
                        (nbr != 26 || aligned16(a.q_nb));
    g.tma = (a.Lx % 4 == 0 && g.W <= a.Lx && ptr_ok) ? 1 : 0;
    if (nbr == 4) return cpl == 8 ? strip_fm<4, 8>(a, g, field, hasmp, s)
                                  : (cpl == 4 ? strip_fm<4, 4>(a, g, field, hasmp, s) : strip_fm<4, 2>(a, g, field, hasmp, s));
    if (nbr == 8) return cpl == 8 ? strip_fm<8, 8>(a, g, field, hasmp, s)
                                  : (cpl == 4 ? strip_fm<8, 4>(a, g, field, hasmp, s) : strip_fm<8, 2>(a, g, field, hasmp, s));
    if (nbr == 26) return cpl == 4 ? strip_fm<26, 4>(a, g, field, hasmp, s) : strip_fm<26, 2>(a, g, field, hasmp, s);
    return set_error(HP_ERR_ARG, "sweep: no strip kernel for this neighbourhood");
}

int strip_status(int* timed_out) {
    int v = 0, zero = 0;
    HP_CUDA(cudaMemcpyFromSymbol(&v, g_strip_err, sizeof(int)));
    if (v) HP_CUDA(cudaMemcpyToSymbol(g_strip_err, &zero, sizeof(int)));
    *timed_out = v;
    return HP_OK;
}

}  // namespace hp
