// Checkerboard Potts sweep (Eq. (7), Sec. 4; bulk-energy carry, Sec. 6).
//
// Two kernels give bit-identical lattices:
//  * k_phase  -- one launch per colour phase, one thread per site of that
//    colour, neighbours read from global memory, state updated in place
//    (no two sites of a colour are neighbours, so this equals the synchronous
//    half-step of Sec. 4).
//  * k_plane  -- all colour phases that live in one lattice plane are run on a
//    shared-memory window of the plane (tile + halo of one site per phase),
//    reading the previous state and writing the tile's new state to a second
//    buffer.  2D lattices: one launch per MCS.  3D 26-neighbour lattices
//    (colours 0-3 on even z planes, 4-7 on odd z planes): two launches per
//    MCS, even planes first (their z neighbours are the old odd planes), then
//    odd planes (z neighbours are the new even planes).
//
// Per site of colour c (sweep = MCS index):
//   u = Philox(seed; site, sweep, tag 0 | c); k = (u.x * M) >> 32; j = nbr_k(i)
//   if q_j == q_i: no change
//   d = J*(#nbrs == q_i - #nbrs == q_j) + (b_j - b_i)
//   accept: d < 0, or d <= D and (thr[d] == ~0 or u.y < thr[d])
//   on accept q_i <- q_j, mp_i <- mp_j.
// A site whose M neighbours all carry q_i cannot change; it skips the draw.
#include <string.h>

#include "sweep.cuh"

namespace hp {
namespace {

constexpr int kThreads = 256;

struct PhaseArgs {
    int32_t* q;
    int32_t* mp;
    const int32_t* table;
    uint32_t table_n;
    const uint32_t* thr;
    int32_t D, J;
    uint64_t seed;
    uint32_t sweep;
    int colour;
    int Lx, Ly, Lz;
    int64_t n_colour_sites;
    // misorientation-dependent pair energy and mobility (ANI kernels only)
    const int32_t* ang;   // grain angles (borrowed, G entries)
    const int32_t* jtab;  // energy per misorientation bin (256 = 1 J)
    const uint32_t* mob;  // relative mobility per bin (all ones = 1), or null
    int32_t period, bin_w, nbins, G;
};

// Misorientation bin of grains a and b: |ang_a - ang_b| folded by the angle's
// symmetry period, divided by the bin width, clamped to the last bin (grain ids
// clamped into the table: they come from caller buffers).
__device__ __forceinline__ int mis_bin(const PhaseArgs& a, int32_t qa, int32_t qb) {
    const uint32_t ua = (uint32_t)qa < (uint32_t)a.G ? (uint32_t)qa : (uint32_t)(a.G - 1);
    const uint32_t ub = (uint32_t)qb < (uint32_t)a.G ? (uint32_t)qb : (uint32_t)(a.G - 1);
    int64_t d = (int64_t)__ldg(a.ang + ua) - (int64_t)__ldg(a.ang + ub);
    d = (d < 0 ? -d : d) % a.period;
    if (a.period - d < d) d = a.period - d;
    const int64_t k = d / a.bin_w;
    return (int)(k < a.nbins ? k : a.nbins - 1);
}

// ---------------------------------------------------------------------------
// One colour phase, one thread per site of that colour, in place.
// FIELD: 0 none, 1 grain (table[q]), 2 point (table[mp]).
// ---------------------------------------------------------------------------
// ANI: the energy of a site in state s is the sum over neighbours n with
// q_n != s of jtab[bin(s, q_n)], and the Metropolis threshold is scaled by the
// mobility of the (q_i, q_j) boundary: eff = thr[d] (all ones for d < 0) when
// the mobility m is all ones, m when thr is all ones, else floor(thr m / 2^32);
// accept iff d <= D and (eff is all ones or u1 < eff).
template <int DIM, int NBR, int FIELD, bool HASMP, bool ANI>
__global__ void __launch_bounds__(kThreads) k_phase(PhaseArgs a) {
    using G = Geo<DIM, NBR>;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_colour_sites) return;
    const int c = a.colour;
    const int hx = a.Lx >> 1;
    int x, y, z;
    if (G::C == 2) {
        const int64_t r = t / hx;
        const int k = (int)(t - r * hx);
        y = (int)(r % a.Ly);
        z = (int)(r / a.Ly);
        x = 2 * k + ((y + z + c) & 1);
    } else if (G::C == 4) {
        const int64_t r = t / hx;
        x = 2 * (int)(t - r * hx) + (c & 1);
        y = 2 * (int)r + (c >> 1);
        z = 0;
    } else {
        const int hy = a.Ly >> 1;
        const int64_t r = t / hx;
        x = 2 * (int)(t - r * hx) + (c & 1);
        y = 2 * (int)(r % hy) + ((c >> 1) & 1);
        z = 2 * (int)(r / hy) + (c >> 2);
    }
    const int64_t sxy = (int64_t)a.Lx * a.Ly;
    const int64_t i = x + (int64_t)a.Lx * y + sxy * z;
    const int32_t qi = a.q[i];
    int32_t nv[G::M];
    int64_t ni[G::M];
    int same_old = 0;
#pragma unroll
    for (int k = 0; k < G::M; ++k) {
        int dx, dy, dz;
        G::off(k, dx, dy, dz);
        const int xx = wrapi(x + dx, a.Lx), yy = wrapi(y + dy, a.Ly), zz = DIM == 3 ? wrapi(z + dz, a.Lz) : 0;
        ni[k] = xx + (int64_t)a.Lx * yy + sxy * zz;
        nv[k] = a.q[ni[k]];
        same_old += nv[k] == qi;
    }
    if (same_old == G::M) return;
    const uint4 u = draw(a.seed, (uint64_t)i, a.sweep, kTagSweep, (uint32_t)c);
    const int kp = (int)__umulhi(u.x, (uint32_t)G::M);
    int32_t qj = 0;
    int64_t j = 0;
#pragma unroll
    for (int k = 0; k < G::M; ++k)
        if (k == kp) { qj = nv[k]; j = ni[k]; }
    if (qj == qi) return;
    int same_new = 0;
#pragma unroll
    for (int k = 0; k < G::M; ++k) same_new += nv[k] == qj;
    int32_t db = 0;
    int32_t mpj = 0;
    if (HASMP) mpj = a.mp[j];
    if (FIELD == 1) db = tab(a.table, a.table_n, qj) - tab(a.table, a.table_n, qi);
    if (FIELD == 2) db = tab(a.table, a.table_n, mpj) - tab(a.table, a.table_n, a.mp[i]);
    if (!ANI) {
        const int32_t d = a.J * (same_old - same_new) + db;
        if (metropolis(d, a.D, a.thr, u.y)) {
            a.q[i] = qj;
            if (HASMP) a.mp[i] = mpj;
        }
        return;
    }
    int32_t e_old = 0, e_new = 0;
#pragma unroll
    for (int k = 0; k < G::M; ++k) {
        if (nv[k] != qi) e_old += __ldg(a.jtab + mis_bin(a, qi, nv[k]));
        if (nv[k] != qj) e_new += __ldg(a.jtab + mis_bin(a, qj, nv[k]));
    }
    const int32_t d = e_new - e_old + db;
    if (d > a.D) return;
    const uint32_t th = d < 0 ? 0xFFFFFFFFu : __ldg(a.thr + d);
    const uint32_t m = a.mob ? __ldg(a.mob + mis_bin(a, qi, qj)) : 0xFFFFFFFFu;
    const uint32_t eff = m == 0xFFFFFFFFu ? th : (th == 0xFFFFFFFFu ? m : __umulhi(th, m));
    if (eff == 0xFFFFFFFFu || u.y < eff) {
        a.q[i] = qj;
        if (HASMP) a.mp[i] = mpj;
    }
}

// ---------------------------------------------------------------------------
// Fused plane kernel.  One CTA = one TX x TY tile of one plane.  The window
// holds the tile plus a halo of H = 4 sites (at least one site per colour
// phase run here: 2 for the 4-neighbour lattice, 4 for Moore planes).
//
// Shared layout: each window row is split by x parity, element (lx, ly) at
// [lx & 1][ly][lx >> 1].  Sites of one colour then sit at unit stride, and so
// do their x neighbours, so warps read shared memory without bank conflicts.
//
// Each phase has two stages.  A: every site of the colour in the still-valid
// region counts its neighbours equal to itself; a site whose neighbours all
// match cannot change, the others are appended to a shared queue.  B: the
// queued sites draw their random numbers and run the Metropolis update, with
// every lane of every warp busy.  The order inside a phase is irrelevant: no
// two sites of one colour are neighbours.
// ---------------------------------------------------------------------------
template <int NBR, int WX_, int TY>
struct PlaneCfg {
    static constexpr int H = 4;
    static constexpr int WX = WX_, WXH = WX_ / 2, TX = WX - 2 * H;
    static_assert(WX == 64 || WX == 128, "window width");
    static constexpr int WY = TY + 2 * H;
    static constexpr int PL = WY * WXH;                  // one parity half of a window plane
    static constexpr int NP = NBR == 4 ? 2 : 4;          // colour phases in a plane
    static constexpr bool Z = NBR == 26;
    // queue capacity: at most the sites of one colour in the window -- every row
    // (2 colours) or every other row (Moore planes), WXH per row
    static constexpr int QCAP = NBR == 4 ? WXH * WY : WXH * ((WY + 1) / 2);
    static constexpr int planes = Z ? 3 : 1;
    static size_t smem(bool hasmp) {
        return sizeof(int32_t) * (size_t)(2 * PL) * (planes + (hasmp ? 1 : 0)) + sizeof(uint32_t) * QCAP +
               sizeof(int) * 8;
    }
};

// Load a window plane (q, and optionally mp) into the parity-split layout.
template <class Cfg>
__device__ __forceinline__ void load_window(const PlaneArgs& a, const int32_t* __restrict__ src,
                                            int32_t* __restrict__ dst, int x0, int y0) {
    constexpr int WX = Cfg::WX, WXH = Cfg::WXH, WY = Cfg::WY, PL = Cfg::PL, H = Cfg::H;
    if (a.vec) {
        constexpr int CH = WX / 4;  // 16-byte chunks per row
        for (int idx = threadIdx.x; idx < CH * WY; idx += kThreads) {
            const int ly = idx / CH, c = idx - ly * CH;
            const int gy = wrap1(y0 - H + ly, a.Ly);
            const int gx = wrap1(x0 - H + 4 * c, a.Lx);
            const int4 v = __ldg(reinterpret_cast<const int4*>(src + gx + (int64_t)a.Lx * gy));
            int32_t* row = dst + ly * WXH + 2 * c;
            *reinterpret_cast<int2*>(row) = make_int2(v.x, v.z);
            *reinterpret_cast<int2*>(row + PL) = make_int2(v.y, v.w);
        }
    } else {
        for (int idx = threadIdx.x; idx < WX * WY; idx += kThreads) {
            const int ly = idx / WX, lx = idx - ly * WX;
            const int gx = a.fast ? wrap1(x0 - H + lx, a.Lx) : wrapi(x0 - H + lx, a.Lx);
            const int gy = a.fast ? wrap1(y0 - H + ly, a.Ly) : wrapi(y0 - H + ly, a.Ly);
            dst[(lx & 1) * PL + ly * WXH + (lx >> 1)] = src[gx + (int64_t)a.Lx * gy];
        }
    }
}

template <int NBR, int WX_, int TY, int FIELD, bool HASMP>
__device__ __forceinline__ void plane_body(const PlaneArgs& a, const int tile, const int zidx, int32_t* smem) {
    using Cfg = PlaneCfg<NBR, WX_, TY>;
    constexpr int H = Cfg::H, WX = Cfg::WX, WXH = Cfg::WXH, WY = Cfg::WY, PL = Cfg::PL, TX = Cfg::TX;
    constexpr int NP = Cfg::NP;
    constexpr bool Z = Cfg::Z;
    constexpr int M = NBR;
    int32_t* s_q = smem;
    int32_t* s_mp = smem + 2 * PL;                              // when HASMP
    int32_t* s_lo = smem + (HASMP ? 2 : 1) * 2 * PL;            // plane z-1 (3D)
    int32_t* s_hi = s_lo + 2 * PL;                              // plane z+1 (3D)
    uint32_t* queue = reinterpret_cast<uint32_t*>(smem + 2 * PL * Cfg::planes + (HASMP ? 2 * PL : 0));
    int* qn = reinterpret_cast<int*>(queue + Cfg::QCAP);

    const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
    const int x0 = tx * TX, y0 = ty * TY;
    const int z = Z ? 2 * zidx + a.zpar : 0;
    const int zlo = Z ? wrapi(z - 1, a.Lz) : 0, zhi = Z ? wrapi(z + 1, a.Lz) : 0;
    const int64_t sxy = (int64_t)a.Lx * a.Ly;

    if (threadIdx.x < 8) qn[threadIdx.x] = 0;
    load_window<Cfg>(a, a.q_in + sxy * z, s_q, x0, y0);
    if (HASMP) load_window<Cfg>(a, a.mp_in + sxy * z, s_mp, x0, y0);
    if (Z) {
        load_window<Cfg>(a, a.q_nb + sxy * zlo, s_lo, x0, y0);
        load_window<Cfg>(a, a.q_nb + sxy * zhi, s_hi, x0, y0);
    }
    __syncthreads();

    // stage A works on pairs of same-colour sites (half-indices xh, xh+1 of one
    // parity in one row): their own values and same-parity neighbours are one
    // aligned 64-bit load per row, their other-parity neighbours a 64-bit and a
    // 32-bit load per row.
    constexpr int PAIRS = WXH / 2;
    const int lane_p = threadIdx.x % PAIRS;
    const int row_slot = threadIdx.x / PAIRS;
    constexpr int ROWS_PER_PASS = kThreads / PAIRS;
    const int cz = Z ? 4 * a.zpar : 0;

#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int lo = p + 1, hix = WX - p - 1, hiy = WY - p - 1;
        // ---- stage A: interior test, queue the rest --------------------------
        // rows holding sites of this colour: every row (4-neighbour) or every
        // other row (Moore, y parity = p >> 1)
        constexpr int RSTEP = NBR == 4 ? 1 : 2;
        const int ys = NBR == 4 ? lo : lo + ((lo ^ (p >> 1)) & 1);
        for (int ly0 = ys; ly0 < hiy; ly0 += RSTEP * ROWS_PER_PASS) {
            const int ly = ly0 + RSTEP * row_slot;
            const int px = NBR == 4 ? ((ly + p) & 1) : (p & 1);  // x parity of this colour in row ly
            const bool rowok = ly < hiy;
            const int xh = 2 * lane_p;
            const int lxa = 2 * xh + px, lxb = lxa + 2;
            const bool va = rowok && lxa >= lo && lxa < hix;
            const bool vb = rowok && lxb >= lo && lxb < hix;
            int same_a = 0, same_b = 0;
            if (va || vb) {
                const int base = ly * WXH;
                const int own = px * PL + base + xh;
                const int oth = (px ^ 1) * PL + base + xh;
                const int oth3 = (px ^ 1) * PL + base + (px ? min(xh + 2, WXH - 1) : max(xh - 1, 0));
                const int2 qq = *reinterpret_cast<const int2*>(s_q + own);
                // one row of plane P at row offset o; `centre` excludes the site itself
                auto row = [&](const int32_t* P, int o, bool centre, bool sides, bool middle) {
                    if (sides) {
                        const int2 op = *reinterpret_cast<const int2*>(P + oth + o);
                        const int32_t o3 = P[oth3 + o];
                        const int32_t al = px ? op.x : o3, ar = px ? op.y : op.x;
                        const int32_t bl = px ? op.y : op.x, br = px ? o3 : op.y;
                        same_a += (al == qq.x) + (ar == qq.x);
                        same_b += (bl == qq.y) + (br == qq.y);
                    }
                    if (middle && !centre) {
                        const int2 sp = *reinterpret_cast<const int2*>(P + own + o);
                        same_a += sp.x == qq.x;
                        same_b += sp.y == qq.y;
                    }
                };
                if (NBR == 4) {
                    row(s_q, 0, true, true, false);
                    row(s_q, -WXH, false, false, true);
                    row(s_q, WXH, false, false, true);
                } else {
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy) {
                        row(s_q, dy * WXH, dy == 0, true, true);
                        if (Z) {
                            row(s_lo, dy * WXH, false, true, true);
                            row(s_hi, dy * WXH, false, true, true);
                        }
                    }
                }
            }
            const int lane = threadIdx.x & 31;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool cand = h == 0 ? (va && same_a != M) : (vb && same_b != M);
                const unsigned ball = __ballot_sync(0xFFFFFFFFu, cand);
                if (ball) {
                    int slot = 0;
                    if (lane == __ffs(ball) - 1) slot = atomicAdd(qn + p, __popc(ball));
                    slot = __shfl_sync(0xFFFFFFFFu, slot, __ffs(ball) - 1);
                    if (cand) {
                        const int k = slot + __popc(ball & ((1u << lane) - 1));
                        const int lx = h == 0 ? lxa : lxb, same = h == 0 ? same_a : same_b;
                        queue[k] = ((uint32_t)ly << 13) | ((uint32_t)lx << 5) | (uint32_t)same;
                    }
                }
            }
        }
        __syncthreads();
        // ---- stage B: Metropolis update of the queued sites ----------------
        const int n = qn[p];
        for (int k = threadIdx.x; k < n; k += kThreads) {
            const uint32_t e = queue[k];
            const int same_old = (int)(e & 31u), lx = (int)((e >> 5) & 255u), ly = (int)(e >> 13);
            const int px = lx & 1, xs = lx >> 1, base = ly * WXH;
            const int c0 = px * PL + base + xs;
            const int cl = (px ? 0 : PL) + base + xs - (px ? 0 : 1);
            const int cr = (px ? 0 : PL) + base + xs + (px ? 1 : 0);
            const int32_t qi = s_q[c0];
            const int gx = a.fast ? wrap1(x0 - H + lx, a.Lx) : wrapi(x0 - H + lx, a.Lx);
            const int gy = a.fast ? wrap1(y0 - H + ly, a.Ly) : wrapi(y0 - H + ly, a.Ly);
            const int64_t gi = gx + (int64_t)a.Lx * gy + sxy * z;
            const int colour = NBR == 4 ? p : cz + p;
            const uint4 u = draw(a.seed, (uint64_t)gi, a.sweep, kTagSweep, (uint32_t)colour);
            const int kp = (int)__umulhi(u.x, (uint32_t)M);
            int dx, dy, dz;
            if (NBR == 4) Geo<2, 4>::off(kp, dx, dy, dz);
            else if (NBR == 8) Geo<2, 8>::off(kp, dx, dy, dz);
            else Geo<3, 26>::off(kp, dx, dy, dz);
            const int cj = (dx == 0 ? c0 : (dx < 0 ? cl : cr)) + dy * WXH;
            const int32_t* pj = dz == 0 ? s_q : (dz < 0 ? s_lo : s_hi);
            const int32_t qj = pj[cj];
            if (qj == qi) continue;
            // the material point and field loads go out first; their latency
            // overlaps the neighbour count
            int32_t mpj = 0;
            if (HASMP) {
                if (dz == 0) {
                    mpj = s_mp[cj];
                } else {
                    const int jx = wrap1(gx + dx, a.Lx), jy = wrap1(gy + dy, a.Ly);
                    mpj = __ldg(a.mp_nb + jx + (int64_t)a.Lx * jy + sxy * (dz < 0 ? zlo : zhi));
                }
            }
            int32_t bi = 0, bj = 0;
            if (FIELD == 1) { bi = tab(a.table, a.table_n, qi); bj = tab(a.table, a.table_n, qj); }
            if (FIELD == 2) { bi = tab(a.table, a.table_n, s_mp[c0]); bj = tab(a.table, a.table_n, mpj); }
            int same_new;
            if (NBR == 4) {
                same_new = (s_q[cl] == qj) + (s_q[cr] == qj) + (s_q[c0 - WXH] == qj) + (s_q[c0 + WXH] == qj);
            } else {
                same_new = 0;
#pragma unroll
                for (int ddy = -1; ddy <= 1; ++ddy) {
                    const int o = ddy * WXH;
                    same_new += (s_q[cl + o] == qj) + (s_q[cr + o] == qj) + (ddy ? (s_q[c0 + o] == qj) : 0);
                    if (Z) {
                        same_new += (s_lo[cl + o] == qj) + (s_lo[cr + o] == qj) + (s_lo[c0 + o] == qj);
                        same_new += (s_hi[cl + o] == qj) + (s_hi[cr + o] == qj) + (s_hi[c0 + o] == qj);
                    }
                }
            }
            const int32_t d = a.J * (same_old - same_new) + (bj - bi);
            if (metropolis(d, a.D, a.thr, u.y)) {
                s_q[c0] = qj;
                if (HASMP) s_mp[c0] = mpj;
            }
        }
        __syncthreads();
    }

    // ---- write the tile's core (skip columns/rows beyond a ragged edge) -----
    int32_t* qo = a.q_out + sxy * z;
    int32_t* mpo = HASMP ? a.mp_out + sxy * z : nullptr;
    if (a.vec) {
        constexpr int CH = TX / 4;
        for (int idx = threadIdx.x; idx < CH * TY; idx += kThreads) {
            const int cy = idx / CH, c = idx - cy * CH;
            const int gx = x0 + 4 * c, gy = y0 + cy;
            if (gx >= a.Lx || gy >= a.Ly) continue;
            const int r = (cy + H) * WXH + ((H + 4 * c) >> 1);
            const int2 ev = *reinterpret_cast<const int2*>(s_q + r), od = *reinterpret_cast<const int2*>(s_q + PL + r);
            *reinterpret_cast<int4*>(qo + gx + (int64_t)a.Lx * gy) = make_int4(ev.x, od.x, ev.y, od.y);
            if (HASMP) {
                const int2 me = *reinterpret_cast<const int2*>(s_mp + r), mo = *reinterpret_cast<const int2*>(s_mp + PL + r);
                *reinterpret_cast<int4*>(mpo + gx + (int64_t)a.Lx * gy) = make_int4(me.x, mo.x, me.y, mo.y);
            }
        }
    } else {
        for (int idx = threadIdx.x; idx < TX * TY; idx += kThreads) {
            const int cy = idx / TX, cx = idx - cy * TX;
            const int gx = x0 + cx, gy = y0 + cy;
            if (gx >= a.Lx || gy >= a.Ly) continue;
            const int lx = cx + H, ly = cy + H;
            const int li = (lx & 1) * PL + ly * WXH + (lx >> 1);
            const int64_t o = gx + (int64_t)a.Lx * gy;
            qo[o] = s_q[li];
            if (HASMP) mpo[o] = s_mp[li];
        }
    }
}

// at most 51 registers so that five 256-thread CTAs fit on an SM
constexpr int kPlaneMinBlocks = 5;

template <int NBR, int WX, int TY, int FIELD, bool HASMP>
__global__ void __launch_bounds__(kThreads, kPlaneMinBlocks) k_plane(PlaneArgs a) {
    extern __shared__ __align__(16) int32_t smem[];
    plane_body<NBR, WX, TY, FIELD, HASMP>(a, (int)blockIdx.x, (int)blockIdx.y, smem);
}

// Many independent lattices (replicas) in one launch: block b belongs to the
// replica r with start[r] <= b < start[r+1]; within it, b - start[r] =
// zidx * tiles + tile.  Each replica carries its own geometry, seed, sweep
// counter, field table and threshold table in its PlaneArgs.
struct BatchArgs {
    const PlaneArgs* args;
    const int64_t* start;  // R + 1 block offsets
    int R;
    uint32_t sweep_add;    // added to every replica's sweep counter
};

template <int NBR, int WX, int TY, int FIELD, bool HASMP>
__global__ void __launch_bounds__(kThreads, kPlaneMinBlocks) k_plane_batch(BatchArgs b) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ PlaneArgs sa;
    __shared__ int s_tile, s_zidx;
    if (threadIdx.x == 0) {
        const int64_t blk = blockIdx.x;
        int lo = 0, hi = b.R - 1;
        while (lo < hi) {  // largest r with start[r] <= blk
            const int mid = (lo + hi + 1) >> 1;
            if (b.start[mid] <= blk) lo = mid; else hi = mid - 1;
        }
        sa = b.args[lo];
        sa.sweep += b.sweep_add;
        const int64_t local = blk - b.start[lo];
        s_zidx = (int)(local / sa.tiles);
        s_tile = (int)(local - (int64_t)s_zidx * sa.tiles);
    }
    __syncthreads();
    plane_body<NBR, WX, TY, FIELD, HASMP>(sa, s_tile, s_zidx, smem);
}

template <int DIM, int NBR, int FIELD, bool HASMP, bool ANI>
int launch_phase(hp_handle* h, uint32_t sweep, int colour, cudaStream_t s) {
    PhaseArgs a;
    a.q = h->q;
    a.mp = h->mp;
    a.table = h->table;
    a.table_n = (uint32_t)h->table_n;
    a.thr = h->thr;
    a.D = h->D;
    a.J = h->desc.J_fix;
    a.seed = h->desc.seed;
    a.sweep = sweep;
    a.colour = colour;
    a.Lx = (int)h->lat.L[0];
    a.Ly = (int)h->lat.L[1];
    a.Lz = (int)h->lat.L[2];
    a.n_colour_sites = h->lat.N / Geo<DIM, NBR>::C;
    a.ang = h->an_ang;
    a.jtab = h->an_J;
    a.mob = h->an_mob;
    a.period = h->an_period;
    a.bin_w = h->an_bin;
    a.nbins = h->an_nbins;
    a.G = h->desc.n_grains;
    const int64_t blocks = (a.n_colour_sites + kThreads - 1) / kThreads;
    ::hp::count_launch();
    k_phase<DIM, NBR, FIELD, HASMP, ANI><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    HP_LAUNCH_CHECK("k_phase");
    return HP_OK;
}

template <int DIM, int NBR, bool ANI>
int phase_dispatch_a(hp_handle* h, uint32_t sweep, int colour, cudaStream_t s) {
    const bool m = h->mp != nullptr;
    switch (h->desc.field_mode) {
        case HP_FIELD_NONE:
            return m ? launch_phase<DIM, NBR, 0, true, ANI>(h, sweep, colour, s)
                     : launch_phase<DIM, NBR, 0, false, ANI>(h, sweep, colour, s);
        case HP_FIELD_GRAIN:
            return m ? launch_phase<DIM, NBR, 1, true, ANI>(h, sweep, colour, s)
                     : launch_phase<DIM, NBR, 1, false, ANI>(h, sweep, colour, s);
        default:
            return launch_phase<DIM, NBR, 2, true, ANI>(h, sweep, colour, s);
    }
}

template <int DIM, int NBR>
int phase_dispatch(hp_handle* h, uint32_t sweep, int colour, cudaStream_t s) {
    return h->an_J ? phase_dispatch_a<DIM, NBR, true>(h, sweep, colour, s)
                   : phase_dispatch_a<DIM, NBR, false>(h, sweep, colour, s);
}

int run_phase_kernel(hp_handle* h, uint32_t sweep, int colour, cudaStream_t s) {
    const int dim = h->lat.dim, nbr = h->lat.nbr;
    if (dim == 2 && nbr == 4) return phase_dispatch<2, 4>(h, sweep, colour, s);
    if (dim == 2 && nbr == 8) return phase_dispatch<2, 8>(h, sweep, colour, s);
    if (dim == 3 && nbr == 6) return phase_dispatch<3, 6>(h, sweep, colour, s);
    return phase_dispatch<3, 26>(h, sweep, colour, s);
}

// Tile variants of the fused kernel.  Plane tiles (this file): window width WX
// (core TX = WX - 8) and core height TY, parity-split window, one CTA per item.
// Lean tiles (tile.cu): WX x (TY + 4) row-major windows fed by bulk TMA copies.
// Lean 3D windows (lean.cu, 26 neighbours): 64 x (TY + 4), every draw made
// while the window is in flight.  All give identical lattices; the autotuner
// picks one.  Ensembles take every variant.
struct Variant {
    int WX, TY;
    bool tile;
    bool lean;
};
constexpr int kVariants2D = 6, kVariants3D = 12;
constexpr Variant kV2D[kVariants2D] = {
    {128, 64, false, false}, {128, 32, false, false}, {64, 64, false, false},
    {128, 28, true, false},  {128, 60, true, false},  {64, 60, true, false}};
constexpr Variant kV3D[kVariants3D] = {
    {128, 32, false, false}, {128, 16, false, false}, {64, 32, false, false}, {64, 16, false, false},
    {64, 60, true, false},   {64, 28, true, false},   {128, 28, true, false}, {64, 36, true, false},
    {64, 40, false, true},   {64, 36, false, true},   {64, 32, false, true}, {64, 28, false, true}};

int n_variants(int nbr) { return nbr == 26 ? kVariants3D : (nbr == 6 ? 1 : kVariants2D); }
Variant variant_of(int nbr, int v) { return nbr == 26 ? kV3D[v] : kV2D[v]; }
// Window rows: tile windows carry two halo rows above and below the core, the
// plane kernels four.
int window_rows(const Variant& v) { return v.TY + (v.tile || v.lean ? 4 : 8); }

template <int NBR, int WX, int TY, int FIELD, bool HASMP>
int launch_one(const PlaneArgs* a, const BatchArgs* b, int64_t blocks, int planes, cudaStream_t s) {
    using Cfg = PlaneCfg<NBR, WX, TY>;
    const size_t smem = Cfg::smem(HASMP);
    static bool configured = false;  // per template instance
    if (!configured) {
        HP_CUDA(cudaFuncSetAttribute(k_plane<NBR, WX, TY, FIELD, HASMP>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HP_CUDA(cudaFuncSetAttribute(k_plane_batch<NBR, WX, TY, FIELD, HASMP>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    if (blocks == 0) return HP_OK;  // configure only
    ::hp::count_launch();
    if (a) k_plane<NBR, WX, TY, FIELD, HASMP><<<dim3((unsigned)blocks, (unsigned)planes), kThreads, smem, s>>>(*a);
    else k_plane_batch<NBR, WX, TY, FIELD, HASMP><<<(unsigned)blocks, kThreads, smem, s>>>(*b);
    HP_LAUNCH_CHECK("k_plane");
    return HP_OK;
}

// field / material-point combinations; variants other than 0 are compiled for
// the two production combinations only (grain field without mp, point field)
template <int NBR, int WX, int TY, bool ALL>
int launch_fm(int field, bool m, const PlaneArgs* a, const BatchArgs* b, int64_t blocks, int planes,
              cudaStream_t s) {
    if (field == HP_FIELD_GRAIN && !m) return launch_one<NBR, WX, TY, 1, false>(a, b, blocks, planes, s);
    if (field == HP_FIELD_POINT) return launch_one<NBR, WX, TY, 2, true>(a, b, blocks, planes, s);
    if constexpr (ALL) {
        if (field == HP_FIELD_NONE) return m ? launch_one<NBR, WX, TY, 0, true>(a, b, blocks, planes, s)
                                             : launch_one<NBR, WX, TY, 0, false>(a, b, blocks, planes, s);
        return launch_one<NBR, WX, TY, 1, true>(a, b, blocks, planes, s);
    }
    return set_error(HP_ERR_ARG, "sweep: tile variant not built for this field mode");
}

int launch_variant(int nbr, int v, int field, bool m, const PlaneArgs* a, const BatchArgs* b, int64_t blocks,
                   int planes, cudaStream_t s) {
    const Variant var = variant_of(nbr, v);
    if (var.lean) {
        if (a) return blocks == 0 ? HP_OK : lean_launch(*a, field, m, planes, window_rows(var), s);
        return lean_launch_batch(b->args, b->start, b->R, blocks, b->sweep_add, field, m, window_rows(var), s);
    }
    if (var.tile) {
        if (a) return blocks == 0 ? HP_OK : tile_launch(*a, field, m, nbr, planes, var.WX, window_rows(var), s);
        return tile_launch_batch(b->args, b->start, b->R, blocks, b->sweep_add, field, m, nbr, var.WX,
                                 window_rows(var), s);
    }
    if (nbr == 4) {
        switch (v) {
            case 0: return launch_fm<4, 128, 64, true>(field, m, a, b, blocks, planes, s);
            case 1: return launch_fm<4, 128, 32, false>(field, m, a, b, blocks, planes, s);
            default: return launch_fm<4, 64, 64, false>(field, m, a, b, blocks, planes, s);
        }
    }
    if (nbr == 8) {
        switch (v) {
            case 0: return launch_fm<8, 128, 64, true>(field, m, a, b, blocks, planes, s);
            case 1: return launch_fm<8, 128, 32, false>(field, m, a, b, blocks, planes, s);
            default: return launch_fm<8, 64, 64, false>(field, m, a, b, blocks, planes, s);
        }
    }
    switch (v) {
        case 0: return launch_fm<26, 128, 32, true>(field, m, a, b, blocks, planes, s);
        case 1: return launch_fm<26, 128, 16, false>(field, m, a, b, blocks, planes, s);
        case 2: return launch_fm<26, 64, 32, false>(field, m, a, b, blocks, planes, s);
        default: return launch_fm<26, 64, 16, false>(field, m, a, b, blocks, planes, s);
    }
}

bool variant_ok(int nbr, int v, int field, bool m) {
    if (v < 0 || v >= n_variants(nbr)) return false;
    if (variant_of(nbr, v).lean) return true;  // built for every field mode
    return v == 0 || (field == HP_FIELD_GRAIN && !m) || field == HP_FIELD_POINT;
}

bool variant_batch_ok(int nbr, int v, int field, bool m) {
    const Variant var = variant_of(nbr, v);
    return variant_ok(nbr, v, field, m);
}

// Arguments of the fused kernel for one lattice and one launch.
PlaneArgs plane_args(const hp_handle* h, int variant, const int32_t* q_in, const int32_t* mp_in,
                     const int32_t* q_nb, const int32_t* mp_nb, int32_t* q_out, int32_t* mp_out, uint32_t sweep,
                     int zpar, int* planes) {
    PlaneArgs a;
    a.q_in = q_in;
    a.mp_in = mp_in;
    a.q_nb = q_nb;
    a.mp_nb = mp_nb;
    a.q_out = q_out;
    a.mp_out = mp_out;
    a.table = h->table;
    a.table_n = (uint32_t)h->table_n;
    a.thr = h->thr;
    a.D = h->D;
    a.J = h->desc.J_fix;
    a.seed = h->desc.seed;
    philox_round_keys(a.seed, a.rk);
    a.sweep = sweep;
    a.Lx = (int)h->lat.L[0];
    a.Ly = (int)h->lat.L[1];
    a.Lz = (int)h->lat.L[2];
    a.zpar = zpar;
    const Variant v = variant_of(h->lat.nbr, variant);
    const int TX = v.WX - 8, WY = window_rows(v);
    a.tiles_x = (a.Lx + TX - 1) / TX;
    a.tiles = a.tiles_x * ((a.Ly + v.TY - 1) / v.TY);
    a.fast = (a.Lx >= v.WX && a.Ly >= WY) ? 1 : 0;
    a.vec = (a.fast && (a.Lx % 4) == 0) ? 1 : 0;
    *planes = h->lat.nbr == 26 ? a.Lz / 2 : 1;
    return a;
}

int plane_launch(const hp_handle* h, int variant, const PlaneArgs& a, int planes, cudaStream_t s) {
    return launch_variant(h->lat.nbr, variant, h->desc.field_mode, h->mp != nullptr, &a, nullptr, a.tiles, planes, s);
}

int plane_launch_batch(int nbr, int variant, int field, bool m, const PlaneArgs* d_args, const int64_t* d_start,
                       int R, int64_t blocks, uint32_t sweep_add, cudaStream_t s) {
    BatchArgs b;
    b.args = d_args;
    b.start = d_start;
    b.R = R;
    b.sweep_add = sweep_add;
    return launch_variant(nbr, variant, field, m, nullptr, &b, blocks, 1, s);
}

// Variant a handle sweeps with until one is chosen (hp_set_sweep_variant or the
// autotuner): the fastest measured on the benchmark lattices -- in 3D the lean
// 64 x 32 window with material points (four blocks per SM) and the 64 x 44 one
// without; in 2D the 128 x 60 lean tile.
int default_variant(const hp_handle* h) {
    int v = 0;
    if (h->lat.nbr == 26) v = h->mp ? 11 : 8;
    else if (h->lat.nbr == 8 || h->lat.nbr == 4) v = 4;
    // variant 0 is built for every field mode; the others for the production ones
    return variant_ok(h->lat.nbr, v, h->desc.field_mode, h->mp != nullptr) ? v : 0;
}

int sweep_variants(int nbr) { return n_variants(nbr); }
bool sweep_variant_ok(int nbr, int v, int field, bool m) { return variant_ok(nbr, v, field, m); }
bool sweep_variant_batch_ok(int nbr, int v, int field, bool m) { return variant_batch_ok(nbr, v, field, m); }

}  // namespace

int sweep_run(hp_handle* h, int32_t n_mcs, cudaStream_t s) {
    const int nbr = h->lat.nbr;
    const bool fused_ok = nbr != 6 && !h->an_J;  // the pair-energy tables run on the per-colour kernel
    const bool fused = fused_ok && h->sweep_kernel != HP_SWEEP_PHASE;
    if (!fused) {
        for (int32_t t = 0; t < n_mcs; ++t)
            for (int c = 0; c < h->lat.colours; ++c) {
                const int rc = run_phase_kernel(h, (uint32_t)(h->sweep + t), c, s);
                if (rc) return rc;
            }
        h->sweep += (uint64_t)n_mcs;
        return HP_OK;
    }
    const bool m = h->mp != nullptr;
    const int v = h->sweep_variant >= 0 ? h->sweep_variant : default_variant(h);
    int32_t *qc = h->q, *mc = h->mp, *qa = h->q_alt, *ma = m ? h->mp_alt : nullptr;
    for (int32_t t = 0; t < n_mcs; ++t) {
        Range r_("mcs");
        const uint32_t sw = (uint32_t)(h->sweep + t);
        int planes = 1, rc;
        if (nbr == 26) {
            const PlaneArgs a0 = plane_args(h, v, qc, mc, qc, mc, qa, ma, sw, 0, &planes);
            rc = plane_launch(h, v, a0, planes, s);
            if (rc) return rc;
            const PlaneArgs a1 = plane_args(h, v, qc, mc, qa, ma, qa, ma, sw, 1, &planes);
            rc = plane_launch(h, v, a1, planes, s);
        } else {
            const PlaneArgs a0 = plane_args(h, v, qc, mc, nullptr, nullptr, qa, ma, sw, 0, &planes);
            rc = plane_launch(h, v, a0, planes, s);
        }
        if (rc) return rc;
        int32_t* tq = qc; qc = qa; qa = tq;
        int32_t* tm = mc; mc = ma; ma = tm;
    }
    if (qc != h->q) {
        const size_t bytes = sizeof(int32_t) * (size_t)h->lat.N;
        HP_CUDA(cudaMemcpyAsync(h->q, qc, bytes, cudaMemcpyDeviceToDevice, s));
        if (m) HP_CUDA(cudaMemcpyAsync(h->mp, mc, bytes, cudaMemcpyDeviceToDevice, s));
    }
    h->sweep += (uint64_t)n_mcs;
    return HP_OK;
}

}  // namespace hp

// ---------------------------------------------------------------------------
// Autotuner and batched ensembles (C ABI)
// ---------------------------------------------------------------------------
#include <vector>

using namespace hp;

extern "C" int hp_sweep_autotune(hp_handle* h, int32_t n_mcs, float* ms_out, int32_t* chosen, void* stream) {
    hp::Range r_("hp_sweep_autotune");
    if (!h || n_mcs < 1) return set_error(HP_ERR_ARG, "hp_sweep_autotune: bad arguments");
    if (!h->q || !h->thr) return set_error(HP_ERR_STATE, "hp_sweep_autotune: bind buffers and thresholds first");
    cudaStream_t s = as_stream(stream);
    const int nbr = h->lat.nbr;
    const int nv = sweep_variants(nbr);
    const bool m = h->mp != nullptr;
    const size_t bytes = sizeof(int32_t) * (size_t)h->lat.N;
    int32_t *bq = nullptr, *bm = nullptr;
    HP_CUDA(cudaMallocAsync((void**)&bq, bytes, s));
    if (m && cudaMallocAsync((void**)&bm, bytes, s) != cudaSuccess) {
        cudaFreeAsync(bq, s);
        return set_error(HP_ERR_OOM, "hp_sweep_autotune: backup allocation failed");
    }
    cudaMemcpyAsync(bq, h->q, bytes, cudaMemcpyDeviceToDevice, s);
    if (m) cudaMemcpyAsync(bm, h->mp, bytes, cudaMemcpyDeviceToDevice, s);
    const uint64_t sweep0 = h->sweep;
    const int kernel0 = h->sweep_kernel;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0, rc = HP_OK;
    float best_ms = 3.4e38f;
    h->sweep_kernel = HP_SWEEP_FUSED;
    for (int v = 0; v < nv && rc == HP_OK; ++v) {
        if (ms_out) ms_out[v] = -1.0f;
        if (!sweep_variant_ok(nbr, v, h->desc.field_mode, m)) continue;
        h->sweep_variant = v;
        h->sweep = sweep0;
        rc = sweep_run(h, 1, s);  // warm-up (also configures the kernel)
        if (rc) break;
        cudaMemcpyAsync(h->q, bq, bytes, cudaMemcpyDeviceToDevice, s);
        if (m) cudaMemcpyAsync(h->mp, bm, bytes, cudaMemcpyDeviceToDevice, s);
        h->sweep = sweep0;
        cudaEventRecord(e0, s);
        rc = sweep_run(h, n_mcs, s);
        cudaEventRecord(e1, s);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = cuda_error(cudaGetLastError(), "hp_sweep_autotune"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) ms_out[v] = ms;
        if (ms < best_ms) { best_ms = ms; best = v; }
        cudaMemcpyAsync(h->q, bq, bytes, cudaMemcpyDeviceToDevice, s);
        if (m) cudaMemcpyAsync(h->mp, bm, bytes, cudaMemcpyDeviceToDevice, s);
    }
    h->sweep = sweep0;
    h->sweep_kernel = kernel0;
    h->sweep_variant = best;
    cudaFreeAsync(bq, s);
    if (bm) cudaFreeAsync(bm, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == HP_OK) rc = cuda_error(cudaGetLastError(), "hp_sweep_autotune");
    if (chosen) *chosen = best;
    return rc;
}

struct hp_ensemble {
    std::vector<hp_handle*> m;
    int nbr = 0, field = 0;
    bool hasmp = false;
    int variant = 0;
    std::vector<PlaneArgs> args;   // [mcs parity][zpar][R]
    std::vector<int64_t> start;    // R + 1
    PlaneArgs* d_args = nullptr;
    int64_t* d_start = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_n = -1, exec_variant = -1;
    unsigned long long exec_kernels = 0;
};

namespace {

int ensemble_build(hp_ensemble* e, cudaStream_t s) {
    const int R = (int)e->m.size();
    e->args.assign((size_t)4 * R, PlaneArgs{});
    e->start.assign((size_t)R + 1, 0);
    for (int r = 0; r < R; ++r) {
        hp_handle* h = e->m[r];
        int planes = 1;
        for (int k = 0; k < 2; ++k) {
            int32_t* in_q = k == 0 ? h->q : h->q_alt;
            int32_t* out_q = k == 0 ? h->q_alt : h->q;
            int32_t* in_m = e->hasmp ? (k == 0 ? h->mp : h->mp_alt) : nullptr;
            int32_t* out_m = e->hasmp ? (k == 0 ? h->mp_alt : h->mp) : nullptr;
            e->args[(size_t)(2 * k + 0) * R + r] =
                plane_args(h, e->variant, in_q, in_m, in_q, in_m, out_q, out_m, (uint32_t)h->sweep, 0, &planes);
            e->args[(size_t)(2 * k + 1) * R + r] =
                plane_args(h, e->variant, in_q, in_m, out_q, out_m, out_q, out_m, (uint32_t)h->sweep, 1, &planes);
        }
        e->start[r + 1] = e->start[r] + (int64_t)e->args[r].tiles * planes;
    }
    HP_CUDA(cudaMemcpyAsync(e->d_args, e->args.data(), sizeof(PlaneArgs) * e->args.size(), cudaMemcpyHostToDevice, s));
    HP_CUDA(cudaMemcpyAsync(e->d_start, e->start.data(), sizeof(int64_t) * e->start.size(), cudaMemcpyHostToDevice, s));
    return HP_OK;
}

int ensemble_launches(hp_ensemble* e, int32_t n, cudaStream_t s, unsigned long long* kernels) {
    const int R = (int)e->m.size();
    const int64_t blocks = e->start[R];
    unsigned long long nk = 0;
    for (int32_t t = 0; t < n; ++t) {
        const int k = t & 1;
        for (int zp = 0; zp < (e->nbr == 26 ? 2 : 1); ++zp) {
            const int rc = plane_launch_batch(e->nbr, e->variant, e->field, e->hasmp, e->d_args + (size_t)(2 * k + zp) * R,
                                              e->d_start, R, blocks, (uint32_t)t, s);
            if (rc) return rc;
            ++nk;
        }
    }
    if (n & 1)
        for (hp_handle* h : e->m) {
            const size_t bytes = sizeof(int32_t) * (size_t)h->lat.N;
            HP_CUDA(cudaMemcpyAsync(h->q, h->q_alt, bytes, cudaMemcpyDeviceToDevice, s));
            if (e->hasmp) HP_CUDA(cudaMemcpyAsync(h->mp, h->mp_alt, bytes, cudaMemcpyDeviceToDevice, s));
        }
    if (kernels) *kernels = nk;
    return HP_OK;
}

}  // namespace

extern "C" int hp_ensemble_create(hp_handle* const* members, int32_t R, hp_ensemble** out) {
    if (!members || R < 1 || !out) return set_error(HP_ERR_ARG, "hp_ensemble_create: bad arguments");
    *out = nullptr;
    const hp_handle* h0 = members[0];
    if (!h0) return set_error(HP_ERR_ARG, "hp_ensemble_create: null member");
    for (int r = 0; r < R; ++r) {
        const hp_handle* h = members[r];
        if (!h) return set_error(HP_ERR_ARG, "hp_ensemble_create: null member");
        if (h->lat.nbr != h0->lat.nbr || h->lat.dim != h0->lat.dim || h->desc.field_mode != h0->desc.field_mode ||
            (h->mp != nullptr) != (h0->mp != nullptr))
            return set_error(HP_ERR_ARG, "hp_ensemble_create: members must share dim, nbr, field mode and mp binding");
        if (!h->q || !h->thr || (h->desc.field_mode != HP_FIELD_NONE && !h->table))
            return set_error(HP_ERR_STATE, "hp_ensemble_create: every member needs buffers, thresholds and field");
    }
    if (h0->lat.nbr == 6) return set_error(HP_ERR_ARG, "hp_ensemble_create: no fused kernel for 3D 6-neighbour lattices");
    hp_ensemble* e = new (std::nothrow) hp_ensemble();
    if (!e) return set_error(HP_ERR_OOM, "hp_ensemble_create: out of host memory");
    e->m.assign(members, members + R);
    e->nbr = h0->lat.nbr;
    e->field = h0->desc.field_mode;
    e->hasmp = h0->mp != nullptr;
    if (cudaMalloc((void**)&e->d_args, sizeof(PlaneArgs) * 4 * (size_t)R) != cudaSuccess ||
        cudaMalloc((void**)&e->d_start, sizeof(int64_t) * ((size_t)R + 1)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(e->d_args);
        cudaFree(e->d_start);
        delete e;
        return set_error(HP_ERR_OOM, "hp_ensemble_create: device allocation failed");
    }
    *out = e;
    return HP_OK;
}

extern "C" int hp_ensemble_destroy(hp_ensemble* e) {
    if (!e) return HP_OK;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->cap) cudaStreamDestroy(e->cap);
    cudaFree(e->d_args);
    cudaFree(e->d_start);
    delete e;
    return HP_OK;
}

extern "C" int hp_set_sweep_variant(hp_handle* h, int32_t v) {
    if (!h || !sweep_variant_ok(h->lat.nbr, v, h->desc.field_mode, h->mp != nullptr))
        return set_error(HP_ERR_ARG, "hp_set_sweep_variant: variant not available for this lattice");
    h->sweep_variant = v;
    return HP_OK;
}

extern "C" int hp_sweep_status(int32_t* timed_out) {
    if (!timed_out) return set_error(HP_ERR_ARG, "hp_sweep_status: null argument");
    int vt = 0, vl = 0;
    int rc = tile_status(&vt);
    if (!rc) rc = lean_status(&vl);
    if (rc) return rc;
    *timed_out = vt > vl ? vt : vl;
    if (*timed_out) return set_error(HP_ERR_TIMEOUT, "sweep: a TMA copy did not complete in time");
    return HP_OK;
}

extern "C" int hp_sweep_variants(int32_t nbr, int32_t* n) {
    if (!n) return set_error(HP_ERR_ARG, "hp_sweep_variants: null argument");
    *n = sweep_variants(nbr);
    return HP_OK;
}

extern "C" int hp_ensemble_set_variant(hp_ensemble* e, int32_t v) {
    if (!e || !sweep_variant_batch_ok(e->nbr, v, e->field, e->hasmp))
        return set_error(HP_ERR_ARG, "hp_ensemble_set_variant: variant not available");
    e->variant = v;
    return HP_OK;
}

extern "C" int hp_ensemble_sweep(hp_ensemble* e, int32_t n_mcs, void* stream) {
    hp::Range r_("hp_ensemble_sweep");
    if (!e || n_mcs < 0) return set_error(HP_ERR_ARG, "hp_ensemble_sweep: bad arguments");
    if (n_mcs == 0) return HP_OK;
    cudaStream_t s = as_stream(stream);
    int rc = ensemble_build(e, s);  // refresh per-member sweep counters
    if (rc) return rc;
    if (!e->exec || e->exec_n != n_mcs || e->exec_variant != e->variant) {
        if (e->exec) { cudaGraphExecDestroy(e->exec); e->exec = nullptr; }
        // kernel attributes are set outside the capture
        rc = plane_launch_batch(e->nbr, e->variant, e->field, e->hasmp, e->d_args, e->d_start, 1, 0, 0, s);
        if (rc) return rc;
        cudaGraph_t g = nullptr;
        HP_CUDA(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
        unsigned long long nk = 0;
        rc = ensemble_launches(e, n_mcs, e->cap, &nk);
        const cudaError_t ce = cudaStreamEndCapture(e->cap, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (ce != cudaSuccess) return cuda_error(ce, "hp_ensemble_sweep: capture");
        const cudaError_t ie = cudaGraphInstantiate(&e->exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { e->exec = nullptr; return cuda_error(ie, "hp_ensemble_sweep: instantiate"); }
        e->exec_n = n_mcs;
        e->exec_variant = e->variant;
        e->exec_kernels = nk;
    } else {
        count_launch_n(e->exec_kernels);
    }
    HP_CUDA(cudaGraphLaunch(e->exec, s));
    for (hp_handle* h : e->m) h->sweep += (uint64_t)n_mcs;
    return HP_OK;
}

extern "C" int hp_ensemble_autotune(hp_ensemble* e, int32_t n_mcs, float* ms_out, int32_t* chosen, void* stream) {
    if (!e || n_mcs < 1) return set_error(HP_ERR_ARG, "hp_ensemble_autotune: bad arguments");
    cudaStream_t s = as_stream(stream);
    // back up every member's state, time each variant with direct launches, restore
    std::vector<int32_t*> bq(e->m.size(), nullptr), bm(e->m.size(), nullptr);
    int rc = HP_OK;
    for (size_t r = 0; r < e->m.size() && rc == HP_OK; ++r) {
        const size_t bytes = sizeof(int32_t) * (size_t)e->m[r]->lat.N;
        if (cudaMallocAsync((void**)&bq[r], bytes, s) != cudaSuccess ||
            (e->hasmp && cudaMallocAsync((void**)&bm[r], bytes, s) != cudaSuccess))
            rc = set_error(HP_ERR_OOM, "hp_ensemble_autotune: backup allocation failed");
        else {
            cudaMemcpyAsync(bq[r], e->m[r]->q, bytes, cudaMemcpyDeviceToDevice, s);
            if (e->hasmp) cudaMemcpyAsync(bm[r], e->m[r]->mp, bytes, cudaMemcpyDeviceToDevice, s);
        }
    }
    auto restore = [&]() {
        for (size_t r = 0; r < e->m.size(); ++r) {
            const size_t bytes = sizeof(int32_t) * (size_t)e->m[r]->lat.N;
            cudaMemcpyAsync(e->m[r]->q, bq[r], bytes, cudaMemcpyDeviceToDevice, s);
            if (e->hasmp) cudaMemcpyAsync(e->m[r]->mp, bm[r], bytes, cudaMemcpyDeviceToDevice, s);
        }
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 3.4e38f;
    const int v0 = e->variant;
    for (int v = 0; v < sweep_variants(e->nbr) && rc == HP_OK; ++v) {
        if (ms_out) ms_out[v] = -1.0f;
        if (!sweep_variant_batch_ok(e->nbr, v, e->field, e->hasmp)) continue;
        e->variant = v;
        if ((rc = ensemble_build(e, s))) break;
        if ((rc = ensemble_launches(e, 1, s, nullptr))) break;  // warm-up
        restore();
        cudaEventRecord(e0, s);
        if ((rc = ensemble_launches(e, n_mcs, s, nullptr))) break;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = cuda_error(cudaGetLastError(), "hp_ensemble_autotune"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) ms_out[v] = ms;
        if (ms < best_ms) { best_ms = ms; best = v; }
        restore();
    }
    e->variant = rc == HP_OK ? best : v0;
    for (size_t r = 0; r < e->m.size(); ++r) {
        if (bq[r]) cudaFreeAsync(bq[r], s);
        if (bm[r]) cudaFreeAsync(bm[r], s);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == HP_OK) rc = cuda_error(cudaGetLastError(), "hp_ensemble_autotune");
    if (chosen) *chosen = e->variant;
    return rc;
}

extern "C" int hp_set_anisotropy(hp_handle* h, const int32_t* angle, int32_t period, int32_t bin, int32_t nbins,
                                 const int32_t* J, const uint32_t* mobility, void* stream) {
    if (!h) return set_error(HP_ERR_ARG, "hp_set_anisotropy: null handle");
    cudaFree(h->an_J);
    cudaFree(h->an_mob);
    h->an_J = nullptr;
    h->an_mob = nullptr;
    h->an_ang = nullptr;
    if (!angle && !J) return HP_OK;  // back to the isotropic J_fix
    if (!angle || !J || period < 2 || bin < 1 || nbins < 1 || (int64_t)nbins * bin < period / 2)
        return set_error(HP_ERR_ARG, "hp_set_anisotropy: bad arguments (the bins must cover [0, period/2])");
    for (int32_t k = 0; k < nbins; ++k)
        if (J[k] < 0 || J[k] > (1 << 20)) return set_error(HP_ERR_ARG, "hp_set_anisotropy: J out of [0, 2^20]");
    cudaStream_t s = as_stream(stream);
    HP_CUDA(cudaMalloc((void**)&h->an_J, sizeof(int32_t) * (size_t)nbins));
    HP_CUDA(cudaMemcpyAsync(h->an_J, J, sizeof(int32_t) * (size_t)nbins, cudaMemcpyHostToDevice, s));
    if (mobility) {
        HP_CUDA(cudaMalloc((void**)&h->an_mob, sizeof(uint32_t) * (size_t)nbins));
        HP_CUDA(cudaMemcpyAsync(h->an_mob, mobility, sizeof(uint32_t) * (size_t)nbins, cudaMemcpyHostToDevice, s));
    }
    HP_CUDA(cudaStreamSynchronize(s));  // the host tables may be released after return
    h->an_ang = angle;
    h->an_period = period;
    h->an_bin = bin;
    h->an_nbins = nbins;
    return HP_OK;
}
