// Tile kernel: the fused checkerboard sweep (Eq. (7), Sec. 4) on a row-major
// window in shared memory, built to spend few instructions per site.
//
// One CTA = one WX x WY window of one plane: a (WX-8) x (WY-4) core with a
// halo of four columns and two rows.  The window's rows arrive by bulk TMA copies
// (cp.async.bulk, one per row and array, a second one where a row crosses the
// periodic x boundary; completion on one mbarrier with a clock-limited wait).
// All colour phases that live in the plane then run in shared memory; in 3D
// the planes z-1 and z+1 are read-only neighbours (old for even planes, new for
// odd planes), exactly as in the plane kernel, and each MCS is two launches.
//
// Per phase:
//   A. the phase's (row, quad) items go out in chunks of 64 per warp trip, two
//      per lane; a lane keeps one aligned quad of four columns.  One 128-bit
//      shared load per neighbour row, with the edge columns taken from the
//      neighbouring lanes by shuffle, gives the two sites of the colour in the
//      quad and all their neighbours; a site is interior when the OR of
//      (neighbour XOR site) over its neighbourhood is zero.  The other sites go
//      to a block-wide queue, one atomic per warp.
//   B. every queued site draws Philox and picks its neighbour (each thread
//      takes two queue entries at once, so their Philox rounds overlap); the
//      proposals of another grain are compacted into a per-warp queue, and the
//      warp then counts both grains among each one's neighbours and runs the
//      Metropolis test with all lanes busy.
// Phase p updates the columns [p+1, WX-p-1) and the rows [y_p, WY-y_p); after
// the last phase the core is exact and is written to the output buffer.  The
// halo follows from which earlier phases a phase reads.  Red/black: phase 1
// reads phase 0 along x and y, so y_p = p + 1.  Four colours (x&1) + 2(y&1):
// phase 1 reads phase 0 only along x; phase 2 reads phase 0 along y and phase
// 1 diagonally; phase 3 reads phase 0 diagonally, phase 1 along y and phase 2
// along x.  The exact region thus loses a column at every phase but a row only
// at phases 0 and 2: y_p = 1 + p/2, two rows of halo (the four columns are
// also what keeps every window row on a 16-byte boundary).
#include "sweep.cuh"

namespace hp {
namespace {

constexpr int kTileThreads = 256;
__device__ int g_tile_err;

template <int NBR, int WX, int WY, bool HASMP>
struct TileCfg {
    static constexpr bool Z = NBR == 26;
    static constexpr int HX = 4, HY = 2, TX = WX - 2 * HX, TY = WY - 2 * HY;
    static constexpr int ARR = 1 + (HASMP ? 1 : 0) + (Z ? 2 : 0);  // q, mp, q(z-1), q(z+1)
    static constexpr int A_MP = 1, A_LO = HASMP ? 2 : 1, A_HI = A_LO + 1;
    static constexpr int NP = NBR == 4 ? 2 : 4;
    static constexpr int PAD = 8;                  // ints of padding before and after each array
    static constexpr int AS = WX * WY + 2 * PAD;   // array stride in ints
    static constexpr int QPR = WX / 4;             // quads per row (a lane keeps its quad)
    static constexpr int QCAP = NBR == 4 ? (WX / 2) * WY : (WX / 2) * ((WY + 1) / 2);
    static_assert(WX % 4 == 0 && (AS * 4) % 16 == 0 && 32 % QPR == 0 && TY % 2 == 0, "tile shape");
    __host__ __device__ static constexpr int ylo(int p) { return NBR == 4 ? p + 1 : 1 + (p >> 1); }
    static size_t smem() { return 128 + sizeof(int32_t) * ((size_t)ARR * AS + QCAP + 8) + sizeof(uint2) * 64 * (kTileThreads / 32); }
};

template <int NBR, int WX, int WY, int FIELD, bool HASMP>
struct Tile {
    using Cfg = TileCfg<NBR, WX, WY, HASMP>;
    static constexpr int M = NBR;
    const PlaneArgs& a;
    int32_t* S;      // q of the plane
    int32_t* SMP;    // mp of the plane
    int32_t* SLO;    // q of plane z-1
    int32_t* SHI;    // q of plane z+1
    int x0, y0, z, zlo, zhi;
    int64_t sxy;
    bool fast;

    __device__ Tile(const PlaneArgs& a_) : a(a_) {}

    __device__ __forceinline__ int gx_of(int col) const {
        return fast ? wrap1(x0 - 4 + col, a.Lx) : wrapi(x0 - 4 + col, a.Lx);
    }
    __device__ __forceinline__ int gy_of(int r) const {
        return fast ? wrap1(y0 - Cfg::HY + r, a.Ly) : wrapi(y0 - Cfg::HY + r, a.Ly);
    }
    __device__ __forceinline__ static void offs(int kp, int& dx, int& dy, int& dz) {
        if (NBR == 4) Geo<2, 4>::off(kp, dx, dy, dz);
        else if (NBR == 8) Geo<2, 8>::off(kp, dx, dy, dz);
        else Geo<3, 26>::off(kp, dx, dy, dz);
    }

    // Draw for the queued site e = (row << 8) | col; true when the proposed
    // neighbour carries another grain (then w = (pos | k << 16, u1) goes on).
    __device__ __forceinline__ bool draw_site(uint32_t e, uint32_t colour, uint2& w) const {
        const int r = (int)(e >> 8), col = (int)(e & 255u);
        const int pos = r * WX + col;
        const uint4 u = draw(a.seed, (uint64_t)(gx_of(col) + (int64_t)a.Lx * gy_of(r) + sxy * z), a.sweep, kTagSweep,
                             colour);
        const int kp = (int)__umulhi(u.x, (uint32_t)M);
        int dx, dy, dz;
        offs(kp, dx, dy, dz);
        const int32_t qj = (dz == 0 ? S : (dz < 0 ? SLO : SHI))[pos + dy * WX + dx];
        w = make_uint2((uint32_t)pos | ((uint32_t)kp << 16), u.y);
        return qj != S[pos];
    }

    // Metropolis test of a proposal that changes the site's grain.
    __device__ __forceinline__ void test(uint2 w) const {
        const int pos = (int)(w.x & 0xFFFFu), kp = (int)(w.x >> 16);
        int dx, dy, dz;
        offs(kp, dx, dy, dz);
        const int off = dy * WX + dx;
        const int32_t qi = S[pos];
        const int32_t qj = (dz == 0 ? S : (dz < 0 ? SLO : SHI))[pos + off];
        int32_t mpj = 0, bi = 0, bj = 0;
        if (HASMP) {
            if (dz == 0) {
                mpj = SMP[pos + off];
            } else {
                const int r = pos / WX, col = pos - r * WX;
                mpj = __ldg(a.mp_nb + wrap1(gx_of(col) + dx, a.Lx) + (int64_t)a.Lx * wrap1(gy_of(r) + dy, a.Ly) +
                            sxy * (dz < 0 ? zlo : zhi));
            }
        }
        if (FIELD == 1) { bi = tab(a.table, a.table_n, qi); bj = tab(a.table, a.table_n, qj); }
        if (FIELD == 2) { bi = tab(a.table, a.table_n, SMP[pos]); bj = tab(a.table, a.table_n, mpj); }
        int so = 0, sn = 0;
        auto cnt = [&](int32_t v) { so += v == qi; sn += v == qj; };
        const int32_t* c = S + pos;
        if (NBR == 4) {
            cnt(c[-1]); cnt(c[1]); cnt(c[-WX]); cnt(c[WX]);
        } else {
#pragma unroll
            for (int ddy = -1; ddy <= 1; ++ddy)
#pragma unroll
                for (int ddx = -1; ddx <= 1; ++ddx)
                    if (ddx || ddy) cnt(c[ddy * WX + ddx]);
            if (Cfg::Z) {
                const int32_t* l = SLO + pos;
                const int32_t* h = SHI + pos;
#pragma unroll
                for (int ddy = -1; ddy <= 1; ++ddy)
#pragma unroll
                    for (int ddx = -1; ddx <= 1; ++ddx) {
                        cnt(l[ddy * WX + ddx]);
                        cnt(h[ddy * WX + ddx]);
                    }
            }
        }
        const int32_t d = a.J * (so - sn) + (bj - bi);
        if (metropolis(d, a.D, a.thr, w.y)) {
            S[pos] = qj;
            if (HASMP) SMP[pos] = mpj;
        }
    }
};

__device__ __forceinline__ bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <int NBR, int WX, int WY, int FIELD, bool HASMP>
__device__ __forceinline__ void tile_body(const PlaneArgs& a, const int tile, const int zidx, unsigned char* raw) {
    using T = Tile<NBR, WX, WY, FIELD, HASMP>;
    using Cfg = typename T::Cfg;
    constexpr int ARR = Cfg::ARR, AS = Cfg::AS, PAD = Cfg::PAD, NP = Cfg::NP, QPR = Cfg::QPR;
    constexpr int M = NBR;
    constexpr bool Z = Cfg::Z;
    // rows by bulk TMA copies when a row of the window wraps at most once and
    // every source row starts on a 16-byte boundary
    const bool tma = a.Lx % 4 == 0 && WX <= a.Lx && al16(a.q_in) && (!HASMP || al16(a.mp_in)) && (!Z || al16(a.q_nb));
    int32_t* base = reinterpret_cast<int32_t*>(raw + ((128u - (s_addr(raw) & 127u)) & 127u));
    uint32_t* queue = reinterpret_cast<uint32_t*>(base + ARR * AS);
    int* qn = reinterpret_cast<int*>(queue + Cfg::QCAP);                       // 4 counters
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(qn + 4);  // 8-byte aligned
    uint2* wqueue = reinterpret_cast<uint2*>(qn + 8);                          // 64 per warp

    T t(a);
    t.S = base + PAD;
    t.SMP = base + (HASMP ? AS + PAD : PAD);
    t.SLO = base + Cfg::A_LO * AS + PAD;
    t.SHI = base + Cfg::A_HI * AS + PAD;
    const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
    t.x0 = tx * Cfg::TX;
    t.y0 = ty * Cfg::TY;
    t.z = Z ? 2 * zidx + a.zpar : 0;
    t.zlo = Z ? wrapi(t.z - 1, a.Lz) : 0;
    t.zhi = Z ? wrapi(t.z + 1, a.Lz) : 0;
    t.sxy = (int64_t)a.Lx * a.Ly;
    t.fast = a.fast != 0;
    const int64_t sxy = t.sxy;

    auto src = [&](int arr) -> const int32_t* {
        if (arr == 0) return a.q_in + sxy * t.z;
        if (HASMP && arr == Cfg::A_MP) return a.mp_in + sxy * t.z;
        return a.q_nb + sxy * (arr == Cfg::A_LO ? t.zlo : t.zhi);
    };
    if (threadIdx.x < 4) qn[threadIdx.x] = 0;
    if (tma) {
        const uint32_t mb = s_addr(mbar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                             "r"((uint32_t)(ARR * WY * WX * 4)) : "memory");
            __syncwarp();
            for (int i = threadIdx.x; i < ARR * WY; i += 32) {
                const int arr = i / WY, r = i - arr * WY;
                copy_row(base + arr * AS + PAD + r * WX, src(arr) + (int64_t)a.Lx * t.gy_of(r), t.x0 - 4, WX, a.Lx, mb);
            }
        }
        if (!wait_or_drain(mb, &g_tile_err)) return;
    } else {
        for (int i = threadIdx.x; i < ARR * WY * WX; i += kTileThreads) {
            const int arr = i / (WY * WX), rem = i - arr * (WY * WX), r = rem / WX, c = rem - r * WX;
            base[arr * AS + PAD + rem] = src(arr)[(int64_t)a.Lx * wrapi(t.y0 - Cfg::HY + r, a.Ly) + wrapi(t.x0 - 4 + c, a.Lx)];
        }
        __syncthreads();
    }

    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int warp = (int)(threadIdx.x >> 5);
    const int c0 = 4 * (lane % QPR);
    const uint32_t cz = Z ? 4u * (uint32_t)a.zpar : 0u;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int lo = p + 1, hi = WX - p - 1, loy = Cfg::ylo(p), hiy = WY - loy;
        // ---- A: interior test, queue the rest ---------------------------------
        constexpr int RSTEP = NBR == 4 ? 1 : 2;
        const int rstart = NBR == 4 ? loy : loy + ((loy ^ (p >> 1)) & 1);
        // one quad of row r: sites ca = c0 + px and cb = ca + 2; bits 0/1 of
        // the result say which of them need the Metropolis stage
        auto item = [&](const int r, int& ca, int& cb) -> uint32_t {
            const int px = NBR == 4 ? ((r + p) & 1) : (p & 1);
            const int ca_ = c0 + px, cb_ = ca_ + 2;
            const bool rowok = r < hiy;
            const bool va = rowok && ca_ >= lo && ca_ < hi;
            const bool vb = rowok && cb_ >= lo && cb_ < hi;
            // every lane loads (lanes past the last row read row hiy - 1 and
            // discard it) so that the edge columns can come from the
            // neighbouring lanes: the left lane's last column and the right
            // lane's first.  A lane at the end of a warp row only ever holds a
            // site outside [lo, hi) on that side.
            const int rowq = (rowok ? r : hiy - 1) * WX + c0;
            const int32_t* own = t.S + rowq;
            const int4 cv = *reinterpret_cast<const int4*>(own);
            const int32_t q0 = px ? cv.y : cv.x, q1 = px ? cv.w : cv.z;
            uint32_t acc0 = 0, acc1 = 0;
            // the three columns around each site in one row (values v)
            auto cols = [&](const int4 v, bool centre) {
                const int32_t el = __shfl_up_sync(0xFFFFFFFFu, v.w, 1);
                const int32_t er = __shfl_down_sync(0xFFFFFFFFu, v.x, 1);
                const int32_t l0 = px ? v.x : el, m0 = px ? v.y : v.x, r0_ = px ? v.z : v.y;
                const int32_t l1 = px ? v.z : v.y, m1 = px ? v.w : v.z, r1 = px ? er : v.w;
                acc0 |= (l0 ^ q0) | (r0_ ^ q0);
                acc1 |= (l1 ^ q1) | (r1 ^ q1);
                if (!centre) { acc0 |= m0 ^ q0; acc1 |= m1 ^ q1; }
            };
            auto ld = [&](const int32_t* P) { return *reinterpret_cast<const int4*>(P); };
            if (NBR == 4) {
                cols(cv, true);
                const int4 u = ld(own - WX), d = ld(own + WX);
                acc0 |= ((px ? u.y : u.x) ^ q0) | ((px ? d.y : d.x) ^ q0);
                acc1 |= ((px ? u.w : u.z) ^ q1) | ((px ? d.w : d.z) ^ q1);
            } else {
                cols(ld(own - WX), false);
                cols(cv, true);
                cols(ld(own + WX), false);
                if (Z) {
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy) {
                        cols(ld(t.SLO + rowq + dy * WX), false);
                        cols(ld(t.SHI + rowq + dy * WX), false);
                    }
                }
            }
            ca = ca_;
            cb = cb_;
            return (va && acc0 != 0u ? 1u : 0u) | (vb && acc1 != 0u ? 2u : 0u);
        };
        // the phase's (row, quad) items in chunks of 64, one chunk per warp
        // trip, two items per lane whose loads and shuffles overlap; a lane
        // keeps its quad, so both items and all chunks share its columns
        const int nitems = (hiy - rstart + RSTEP - 1) / RSTEP * QPR;
        for (int ch = warp; 64 * ch < nitems; ch += kTileThreads / 32) {
            const int r1 = rstart + RSTEP * ((64 * ch + lane) / QPR), r2 = r1 + RSTEP * (32 / QPR);
            int ca1, cb1, ca2, cb2;
            const uint32_t f1 = item(r1, ca1, cb1);
            const uint32_t f2 = item(r2, ca2, cb2);
            const unsigned m0 = __ballot_sync(0xFFFFFFFFu, f1 & 1u), m1 = __ballot_sync(0xFFFFFFFFu, f1 & 2u);
            const unsigned m2 = __ballot_sync(0xFFFFFFFFu, f2 & 1u), m3 = __ballot_sync(0xFFFFFFFFu, f2 & 2u);
            if (m0 | m1 | m2 | m3) {
                const int n0 = __popc(m0), n1 = __popc(m1), n2 = __popc(m2);
                int k = 0;
                if (lane == 0) k = atomicAdd(qn + p, n0 + n1 + n2 + __popc(m3));
                k = __shfl_sync(0xFFFFFFFFu, k, 0);
                if (f1 & 1u) queue[k + __popc(m0 & lt)] = ((uint32_t)r1 << 8) | (uint32_t)ca1;
                if (f1 & 2u) queue[k + n0 + __popc(m1 & lt)] = ((uint32_t)r1 << 8) | (uint32_t)cb1;
                if (f2 & 1u) queue[k + n0 + n1 + __popc(m2 & lt)] = ((uint32_t)r2 << 8) | (uint32_t)ca2;
                if (f2 & 2u) queue[k + n0 + n1 + n2 + __popc(m3 & lt)] = ((uint32_t)r2 << 8) | (uint32_t)cb2;
            }
        }
        __syncthreads();
        // ---- B: Metropolis update of the queued sites, two per thread --------
        const uint32_t colour = NBR == 4 ? (uint32_t)p : cz + (uint32_t)p;
        // B1: each warp takes the next 64 queued sites (two per lane), so that
        // when the queue is short a few warps are busy and the rest skip; the
        // proposals of another grain go to the warp's queue.  B2: the warp
        // tests them, all lanes busy.
        const int n = qn[p];
        uint2* wq = wqueue + 64 * warp;
        for (int k0 = 0; k0 < n; k0 += 2 * kTileThreads) {
            const int k1 = k0 + 64 * warp + lane, k2 = k1 + 32;
            uint2 w1 = make_uint2(0u, 0u), w2 = make_uint2(0u, 0u);
            const bool a1 = k1 < n && t.draw_site(queue[k1], colour, w1);
            const bool a2 = k2 < n && t.draw_site(queue[k2], colour, w2);
            const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1), m2 = __ballot_sync(0xFFFFFFFFu, a2);
            if (a1) wq[__popc(m1 & lt)] = w1;
            if (a2) wq[__popc(m1) + __popc(m2 & lt)] = w2;
            __syncwarp();
            const int na = __popc(m1) + __popc(m2);
            for (int j = lane; j < na; j += 32) t.test(wq[j]);
            __syncwarp();
        }
        __syncthreads();
    }
    (void)M;

    // ---- write the core: rows [HY, WY - HY), quads 1 .. QPR - 2 --------------
    int32_t* qo = a.q_out + sxy * t.z;
    int32_t* mpo = HASMP ? a.mp_out + sxy * t.z : nullptr;
    constexpr int CQ = QPR - 2;
    for (int i = threadIdx.x; i < Cfg::TY * CQ; i += kTileThreads) {
        const int cy = i / CQ, qq = 1 + (i - cy * CQ);
        const int gx = t.x0 + 4 * (qq - 1), gy = t.y0 + cy;
        if (gx >= a.Lx || gy >= a.Ly) continue;
        const int li = (cy + Cfg::HY) * WX + 4 * qq;
        const int64_t o = gx + (int64_t)a.Lx * gy;
        if (a.vec) {
            *reinterpret_cast<int4*>(qo + o) = *reinterpret_cast<const int4*>(t.S + li);
            if (HASMP) *reinterpret_cast<int4*>(mpo + o) = *reinterpret_cast<const int4*>(t.SMP + li);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (gx + j >= a.Lx) break;
                qo[o + j] = t.S[li + j];
                if (HASMP) mpo[o + j] = t.SMP[li + j];
            }
        }
    }
}

template <int NBR, int WX, int WY, int FIELD, bool HASMP>
__global__ void __launch_bounds__(kTileThreads, NBR == 26 ? 4 : 5) k_tile(const __grid_constant__ PlaneArgs a) {
    extern __shared__ __align__(16) unsigned char raw[];
    tile_body<NBR, WX, WY, FIELD, HASMP>(a, (int)blockIdx.x, (int)blockIdx.y, raw);
}

// Many independent lattices in one launch: block b belongs to the replica r
// with start[r] <= b < start[r+1]; within it b - start[r] = zidx * tiles + tile.
template <int NBR, int WX, int WY, int FIELD, bool HASMP>
__global__ void __launch_bounds__(kTileThreads, NBR == 26 ? 4 : 5)
    k_tile_batch(const PlaneArgs* __restrict__ args, const int64_t* __restrict__ start, int R, uint32_t sweep_add) {
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
    tile_body<NBR, WX, WY, FIELD, HASMP>(sa, s_tile, s_zidx, raw);
}

struct TileBatch {
    const PlaneArgs* args;
    const int64_t* start;
    int R;
    int64_t blocks;
    uint32_t sweep_add;
};

template <int NBR, int WX, int WY, int FIELD, bool HASMP>
int launch_tile(const PlaneArgs* a, const TileBatch* b, int planes, cudaStream_t s) {
    using Cfg = TileCfg<NBR, WX, WY, HASMP>;
    const size_t smem = Cfg::smem();
    static bool configured = false;
    if (!configured) {
        HP_CUDA(cudaFuncSetAttribute(k_tile<NBR, WX, WY, FIELD, HASMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        HP_CUDA(cudaFuncSetAttribute(k_tile_batch<NBR, WX, WY, FIELD, HASMP>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    if (a) {
        if (a->tiles == 0) return HP_OK;
        count_launch();
        k_tile<NBR, WX, WY, FIELD, HASMP><<<dim3((unsigned)a->tiles, (unsigned)planes), kTileThreads, smem, s>>>(*a);
    } else {
        if (b->blocks == 0) return HP_OK;  // configure only
        count_launch();
        k_tile_batch<NBR, WX, WY, FIELD, HASMP><<<(unsigned)b->blocks, kTileThreads, smem, s>>>(b->args, b->start, b->R,
                                                                                                 b->sweep_add);
    }
    HP_LAUNCH_CHECK("k_tile");
    return HP_OK;
}

template <int NBR, int WX, int WY>
int tile_fm(const PlaneArgs* a, const TileBatch* b, int field, bool m, int planes, cudaStream_t s) {
    if (field == HP_FIELD_GRAIN && !m) return launch_tile<NBR, WX, WY, 1, false>(a, b, planes, s);
    if (field == HP_FIELD_POINT) return launch_tile<NBR, WX, WY, 2, true>(a, b, planes, s);
    return set_error(HP_ERR_ARG, "sweep: tile variant not built for this field mode");
}

int tile_dispatch(const PlaneArgs* a, const TileBatch* b, int field, bool hasmp, int nbr, int planes, int WX, int WY,
                  cudaStream_t s) {
    if (nbr == 8) {
        if (WX == 128 && WY == 32) return tile_fm<8, 128, 32>(a, b, field, hasmp, planes, s);
        if (WX == 128 && WY == 64) return tile_fm<8, 128, 64>(a, b, field, hasmp, planes, s);
        if (WX == 64 && WY == 64) return tile_fm<8, 64, 64>(a, b, field, hasmp, planes, s);
    } else if (nbr == 4) {
        if (WX == 128 && WY == 32) return tile_fm<4, 128, 32>(a, b, field, hasmp, planes, s);
        if (WX == 128 && WY == 64) return tile_fm<4, 128, 64>(a, b, field, hasmp, planes, s);
        if (WX == 64 && WY == 64) return tile_fm<4, 64, 64>(a, b, field, hasmp, planes, s);
    } else if (nbr == 26) {
        if (WX == 64 && WY == 64) return tile_fm<26, 64, 64>(a, b, field, hasmp, planes, s);
        if (WX == 64 && WY == 32) return tile_fm<26, 64, 32>(a, b, field, hasmp, planes, s);
        if (WX == 128 && WY == 32) return tile_fm<26, 128, 32>(a, b, field, hasmp, planes, s);
        if (WX == 64 && WY == 40) return tile_fm<26, 64, 40>(a, b, field, hasmp, planes, s);
    }
    return set_error(HP_ERR_ARG, "sweep: no tile kernel of this shape");
}

}  // namespace

int tile_launch(const PlaneArgs& a, int field, bool hasmp, int nbr, int planes, int WX, int WY, cudaStream_t s) {
    return tile_dispatch(&a, nullptr, field, hasmp, nbr, planes, WX, WY, s);
}

int tile_launch_batch(const PlaneArgs* d_args, const int64_t* d_start, int R, int64_t blocks, uint32_t sweep_add,
                      int field, bool hasmp, int nbr, int WX, int WY, cudaStream_t s) {
    TileBatch b{d_args, d_start, R, blocks, sweep_add};
    return tile_dispatch(nullptr, &b, field, hasmp, nbr, 1, WX, WY, s);
}

int tile_status(int* timed_out) {
    int v = 0, zero = 0;
    HP_CUDA(cudaMemcpyFromSymbol(&v, g_tile_err, sizeof(int)));
    if (v) HP_CUDA(cudaMemcpyToSymbol(g_tile_err, &zero, sizeof(int)));
    *timed_out = v;
    return HP_OK;
}

}  // namespace hp
