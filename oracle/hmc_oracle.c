/*
 * hmc_oracle.c -- plain, slow, single-threaded CPU oracle for the hybrid
 * Monte Carlo method of Zhang, Dingreville, Bartel and Lusk (arXiv 1007.3509).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this file; only the tests, __graft_entry__.smoke() and the CPU baseline leg
 * of bench.py load it.  It shares no code, header, table or constant generator
 * with the CUDA path: every table below (neighbour offsets, colourings, slip
 * systems) is written out here on its own from the paper and the readings
 * listed in the design notes.
 *
 * Integer work (the Potts sweep, Voronoi, statistics) is exact; floating point
 * (crystal plasticity, closed-form energies) is FP64.  No blocking, fusion or
 * reordering beyond what each definition states.
 *
 * Contents (paper passage each part follows):
 *   philox4x32_10        counter-based RNG (Salmon et al., SC'11), the random
 *                        numbers R of Eq. (2) and the trial/accept draws of Sec. 4
 *   threshold_table      Metropolis acceptance exp(-dE/kT) (Sec. 4, Metropolis)
 *   sweep                Q-state Potts Hamiltonian, Eq. (7), red/black update Sec. 4,
 *                        bulk-energy carry with the moving boundary, Sec. 6
 *   voronoi / orient.    initial polycrystal (Sec. 4-5 set-up)
 *   grain statistics     average grain size and texture histograms (Sec. 4, 5)
 *   closed-form energies Schmid factor (Sec. 5, Fig. 4), directional Young's
 *                        modulus (Sec. 5, Fig. 6 discussion), elastic energy
 *   MCP                  Monte Carlo crystal plasticity, Eqs. (1)-(3), Table 1,
 *                        dislocation energy Eq. (4)
 *
 * Parity status: every function here is pinned by a -m "not gpu" test against
 * a library routine, a closed form, brute force or an invariant, except the
 * ones whose header says "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Round: two 32x32->64 products of counter words */
/* 0 and 2 with the round multipliers, output words permuted and xor-ed with */
/* the other counter words and the key; key bumped by the Weyl constants     */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    const uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void oracle_philox4x32_10(uint64_t seed, const uint32_t ctr[4], uint32_t out[4]) {
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Batch form for the tests: n counters laid out as ctr[4*i + w]. */
void oracle_philox_batch(uint64_t seed, const uint32_t* ctr, int64_t n, uint32_t* out) {
    for (int64_t i = 0; i < n; ++i) oracle_philox4x32_10(seed, ctr + 4 * i, out + 4 * i);
}

/* Counter layout shared by definition (not by code) with the device side:
 *   word0/word1 = low/high half of the unit index (site, material point, grain)
 *   word2       = step (MCS index, load increment, attempt)
 *   word3       = tag << 24 | sub   (tag: 0 sweep, 1 MCP, 2 Voronoi, 3 surrogate) */
enum { TAG_SWEEP = 0, TAG_MCP = 1, TAG_VORONOI = 2, TAG_SURROGATE = 3 };

static void draw(uint64_t seed, uint64_t unit, uint32_t step, uint32_t tag, uint32_t sub, uint32_t out[4]) {
    uint32_t c[4] = {(uint32_t)unit, (uint32_t)(unit >> 32), step, (tag << 24) | sub};
    oracle_philox4x32_10(seed, c, out);
}

/* ------------------------------------------------------------------------ */
/* Metropolis threshold table (Sec. 4; acceptance min(1, exp(-dE/kT))).      */
/* Energies are fixed point, 256 units = 1 J (the interaction energy unit).  */
/* thr[0] = 0xFFFFFFFF (dE = 0 accepted, Metropolis) or 0 (strict rule).     */
/* thr[d>=1] = min(floor(2^32 exp(-d / (256 kT))), 0xFFFFFFFE).              */
/* D = largest d with thr[d] > 0 (0 when kT = 0).  An accepted trial with    */
/* 0 <= d <= D needs u < thr[d] (or thr[d] == 0xFFFFFFFF).                   */
/* ------------------------------------------------------------------------ */
int oracle_threshold_table(double kT, int zero_rule, uint32_t* thr, int32_t cap, int32_t* D_out) {
    if (kT < 0.0 || cap < 1 || !thr || !D_out) return OR_ERR_ARG;
    thr[0] = zero_rule ? 0u : 0xFFFFFFFFu;
    int32_t D = 0;
    if (kT > 0.0) {
        for (int32_t d = 1;; ++d) {
            const double v = ldexp(exp(-(double)d / (256.0 * kT)), 32);
            const double f = floor(v);
            if (f < 1.0) break;
            if (d >= cap) return OR_ERR_ARG;
            thr[d] = f > 4294967294.0 ? 0xFFFFFFFEu : (uint32_t)f;
            D = d;
        }
    }
    *D_out = D;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry: periodic box, linear index x + Lx*(y + Ly*z).           */
/* Neighbourhoods and their fixed order (the proposal picks index k):        */
/*   2D-4 : +x, -x, +y, -y                                                   */
/*   2D-8 : (dy,dx) row-major over {-1,0,1}^2 without (0,0)                  */
/*   3D-6 : +x, -x, +y, -y, +z, -z                                           */
/*   3D-26: (dz,dy,dx) lexicographic over {-1,0,1}^3 without (0,0,0)         */
/* Colourings (no two neighbours share a colour; every L is even):           */
/*   2D-4, 3D-6 : c = (x+y+z) & 1                (2 colours, red/black)      */
/*   2D-8       : c = (x&1) + 2(y&1)             (4 colours)                 */
/*   3D-26      : c = (x&1) + 2(y&1) + 4(z&1)    (8 colours)                 */
/* ------------------------------------------------------------------------ */
typedef struct { int dx, dy, dz; } off3;

static int neighbourhood(int dim, int nbr, off3* o) {
    int m = 0;
    if (dim == 2 && nbr == 4) {
        o[0] = (off3){1, 0, 0}; o[1] = (off3){-1, 0, 0}; o[2] = (off3){0, 1, 0}; o[3] = (off3){0, -1, 0};
        return 4;
    }
    if (dim == 2 && nbr == 8) {
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if (dx || dy) o[m++] = (off3){dx, dy, 0};
        return m;
    }
    if (dim == 3 && nbr == 6) {
        o[0] = (off3){1, 0, 0}; o[1] = (off3){-1, 0, 0}; o[2] = (off3){0, 1, 0};
        o[3] = (off3){0, -1, 0}; o[4] = (off3){0, 0, 1}; o[5] = (off3){0, 0, -1};
        return 6;
    }
    if (dim == 3 && nbr == 26) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    if (dx || dy || dz) o[m++] = (off3){dx, dy, dz};
        return m;
    }
    return 0;
}

static int n_colours(int dim, int nbr) {
    if (nbr == 4 || nbr == 6) return 2;
    if (dim == 2 && nbr == 8) return 4;
    if (dim == 3 && nbr == 26) return 8;
    return 0;
}

static int colour_of(int dim, int nbr, int64_t x, int64_t y, int64_t z) {
    if (nbr == 4 || nbr == 6) return (int)((x + y + z) & 1);
    if (dim == 2) return (int)((x & 1) + 2 * (y & 1));
    return (int)((x & 1) + 2 * (y & 1) + 4 * (z & 1));
}

static int64_t wrap(int64_t a, int64_t L) { a %= L; return a < 0 ? a + L : a; }

/* ------------------------------------------------------------------------ */
/* Checkerboard Potts sweep, Eq. (7) and Sec. 4.                             */
/* Hamiltonian read as J * (1 - delta) per unlike neighbour bond, each bond  */
/* counted once from the site being updated, plus the bulk energy b_i.       */
/* One MCS = colours 0..C-1 in order.  Within a colour phase no two updated  */
/* sites are neighbours, so the in-place scan below equals the synchronous   */
/* half-step of Sec. 4.                                                       */
/* For each site i of colour c:                                              */
/*   (u0,u1,..) = Philox(seed; i, sweep, TAG_SWEEP<<24 | c)                  */
/*   j = neighbour number (u0 * M) >> 32 of i                                */
/*   if q_j == q_i: nothing happens                                          */
/*   d = J_fix*(#nbrs with q_i - #nbrs with q_j) + (b_j - b_i)               */
/*   accept if d < 0, reject if d > D, else accept iff thr[d] == ~0 or       */
/*   u1 < thr[d]                                                              */
/*   on accept: q_i <- q_j, b_i <- b_j, mp_i <- mp_j (the swept site takes   */
/*   the dislocation content of the overtaking grain, Sec. 6)                */
/* b and mp may be NULL (zero field / no material-point index).              */
/* Returns the number of accepted flips in *n_flips.                         */
/* ------------------------------------------------------------------------ */
int oracle_sweep(int dim, const int64_t* L, int nbr, int32_t J_fix, uint64_t seed,
                 uint32_t sweep0, int32_t n_mcs, const uint32_t* thr, int32_t D,
                 int32_t* q, int32_t* b, int32_t* mp, int64_t* n_flips) {
    off3 o[26];
    const int M = neighbourhood(dim, nbr, o);
    const int C = n_colours(dim, nbr);
    if (!M || !C || !q || !thr || D < 0 || n_mcs < 0) return OR_ERR_ARG;
    const int64_t Lx = L[0], Ly = L[1], Lz = dim == 3 ? L[2] : 1;
    if (Lx < 2 || Ly < 2 || Lz < 1 || (Lx & 1) || (Ly & 1) || (dim == 3 && (Lz & 1) )) return OR_ERR_ARG;
    int64_t flips = 0;
    for (int32_t t = 0; t < n_mcs; ++t) {
        const uint32_t sweep = sweep0 + (uint32_t)t;
        for (int c = 0; c < C; ++c) {
            for (int64_t z = 0; z < Lz; ++z)
                for (int64_t y = 0; y < Ly; ++y)
                    for (int64_t x = 0; x < Lx; ++x) {
                        if (colour_of(dim, nbr, x, y, z) != c) continue;
                        const int64_t i = x + Lx * (y + Ly * z);
                        int64_t nb[26];
                        for (int k = 0; k < M; ++k)
                            nb[k] = wrap(x + o[k].dx, Lx) + Lx * (wrap(y + o[k].dy, Ly) + Ly * wrap(z + o[k].dz, Lz));
                        uint32_t u[4];
                        draw(seed, (uint64_t)i, sweep, TAG_SWEEP, (uint32_t)c, u);
                        const int k = (int)(((uint64_t)u[0] * (uint64_t)M) >> 32);
                        const int64_t j = nb[k];
                        const int32_t qi = q[i], qj = q[j];
                        if (qj == qi) continue;
                        int same_old = 0, same_new = 0;
                        for (int n = 0; n < M; ++n) {
                            same_old += q[nb[n]] == qi;
                            same_new += q[nb[n]] == qj;
                        }
                        const int32_t db = b ? (b[j] - b[i]) : 0;
                        const int32_t d = J_fix * (same_old - same_new) + db;
                        int accept;
                        if (d < 0) accept = 1;
                        else if (d > D) accept = 0;
                        else accept = thr[d] == 0xFFFFFFFFu || u[1] < thr[d];
                        if (accept) {
                            q[i] = qj;
                            if (b) b[i] = b[j];
                            if (mp) mp[i] = mp[j];
                            ++flips;
                        }
                    }
        }
    }
    if (n_flips) *n_flips = flips;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Misorientation-dependent interaction energy and mobility (the pair energy  */
/* J_{q_i,q_n} of Eq. (7); the arbitrary-misorientation extension of Sec. 6). */
/* Grain g has an integer orientation angle ang[g] in [0, period) (e.g.       */
/* millidegrees of a rotation about z, period 90000 for a cubic crystal).     */
/* The misorientation of grains a, b is min(d, period - d) with               */
/* d = |ang[a] - ang[b]|; its bin is mis / bin_w (clamped to nbins - 1).      */
/* J(a, b) = Jtab[bin] (256 = 1 J), mob(a, b) = mtab[bin] (uint32, all ones   */
/* = 1; NULL = every boundary equally mobile).                                */
/* Site energy in state s: sum over neighbours n with q_n != s of J(s, q_n).  */
/* Trial as in oracle_sweep; d = E(q_j) - E(q_i) + (b_j - b_i); with          */
/* m = mob(q_i, q_j) and t = thr[d] (all ones for d < 0):                     */
/*   eff = t when m is all ones, m when t is all ones, else floor(t m / 2^32) */
/*   accept iff d <= D and (eff is all ones or u1 < eff).                    */
/* A constant Jtab = J_fix without mobility gives oracle_sweep exactly.      */
/* ------------------------------------------------------------------------ */
static int32_t mis_bin(const int32_t* ang, int32_t a, int32_t b, int32_t period, int32_t bin_w, int32_t nbins) {
    int64_t d = (int64_t)ang[a] - (int64_t)ang[b];
    if (d < 0) d = -d;
    d %= period;
    if (period - d < d) d = period - d;
    int64_t k = d / bin_w;
    return (int32_t)(k < nbins ? k : nbins - 1);
}

int oracle_sweep_aniso(int dim, const int64_t* L, int nbr, uint64_t seed, uint32_t sweep0, int32_t n_mcs,
                       const uint32_t* thr, int32_t D, const int32_t* ang, int32_t period, int32_t bin_w,
                       int32_t nbins, const int32_t* Jtab, const uint32_t* mtab, int32_t* q, int32_t* b,
                       int32_t* mp, int64_t* n_flips) {
    off3 o[26];
    const int M = neighbourhood(dim, nbr, o);
    const int C = n_colours(dim, nbr);
    if (!M || !C || !q || !thr || D < 0 || n_mcs < 0 || !ang || !Jtab || period < 1 || bin_w < 1 || nbins < 1)
        return OR_ERR_ARG;
    const int64_t Lx = L[0], Ly = L[1], Lz = dim == 3 ? L[2] : 1;
    if (Lx < 2 || Ly < 2 || Lz < 1 || (Lx & 1) || (Ly & 1) || (dim == 3 && (Lz & 1))) return OR_ERR_ARG;
    int64_t flips = 0;
    for (int32_t t = 0; t < n_mcs; ++t) {
        const uint32_t sweep = sweep0 + (uint32_t)t;
        for (int c = 0; c < C; ++c)
            for (int64_t z = 0; z < Lz; ++z)
                for (int64_t y = 0; y < Ly; ++y)
                    for (int64_t x = 0; x < Lx; ++x) {
                        if (colour_of(dim, nbr, x, y, z) != c) continue;
                        const int64_t i = x + Lx * (y + Ly * z);
                        int64_t nb[26];
                        for (int k = 0; k < M; ++k)
                            nb[k] = wrap(x + o[k].dx, Lx) + Lx * (wrap(y + o[k].dy, Ly) + Ly * wrap(z + o[k].dz, Lz));
                        uint32_t u[4];
                        draw(seed, (uint64_t)i, sweep, TAG_SWEEP, (uint32_t)c, u);
                        const int k = (int)(((uint64_t)u[0] * (uint64_t)M) >> 32);
                        const int64_t j = nb[k];
                        const int32_t qi = q[i], qj = q[j];
                        if (qj == qi) continue;
                        int32_t e_old = 0, e_new = 0;
                        for (int n = 0; n < M; ++n) {
                            const int32_t qn = q[nb[n]];
                            if (qn != qi) e_old += Jtab[mis_bin(ang, qi, qn, period, bin_w, nbins)];
                            if (qn != qj) e_new += Jtab[mis_bin(ang, qj, qn, period, bin_w, nbins)];
                        }
                        const int32_t d = e_new - e_old + (b ? (b[j] - b[i]) : 0);
                        int accept = 0;
                        if (d <= D) {
                            const uint32_t tt = d < 0 ? 0xFFFFFFFFu : thr[d];
                            const uint32_t m = mtab ? mtab[mis_bin(ang, qi, qj, period, bin_w, nbins)] : 0xFFFFFFFFu;
                            uint32_t eff;
                            if (m == 0xFFFFFFFFu) eff = tt;
                            else if (tt == 0xFFFFFFFFu) eff = m;
                            else eff = (uint32_t)(((uint64_t)tt * (uint64_t)m) >> 32);
                            accept = eff == 0xFFFFFFFFu || u[1] < eff;
                        }
                        if (accept) {
                            q[i] = qj;
                            if (b) b[i] = b[j];
                            if (mp) mp[i] = mp[j];
                            ++flips;
                        }
                    }
    }
    if (n_flips) *n_flips = flips;
    return OR_OK;
}

/* Read-Shockley boundary energy per misorientation bin (bin centres, in     */
/* degrees: (k + 1/2) bin_w / unit_per_degree): J(th) = J_max (th/th_m)      */
/* (1 - ln(th/th_m)) below th_m, J_max above, rounded half-even to 256 = 1 J  */
/* units; optional mobility m(th) = 1 - exp(-5 (th/th_m)^4) as a uint32       */
/* fraction (all ones = 1).                                                    */
int oracle_read_shockley(double J_max, double th_m, int32_t bin_w, int32_t nbins, int32_t unit_per_degree,
                         int32_t* Jtab, uint32_t* mtab) {
    if (!(J_max >= 0.0) || !(th_m > 0.0) || bin_w < 1 || nbins < 1 || unit_per_degree < 1 || !Jtab) return OR_ERR_ARG;
    for (int32_t k = 0; k < nbins; ++k) {
        const double th = ((double)k + 0.5) * (double)bin_w / (double)unit_per_degree;
        const double r = th / th_m;
        const double e = r < 1.0 ? J_max * r * (1.0 - log(r)) : J_max;
        Jtab[k] = (int32_t)nearbyint(256.0 * e);
        if (mtab) {
            const double m = 1.0 - exp(-5.0 * r * r * r * r);
            const double f = floor(ldexp(m, 32));
            mtab[k] = f >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)f;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Initial polycrystal: Voronoi tessellation of G seeds.                     */
/* Seed placement in rounds: in round a every still-unplaced seed g draws    */
/* site floor(u0 * N / 2^32) from Philox(seed; g, a, TAG_VORONOI<<24 | 0)    */
/* (word0 = g, word2 = a; N < 2^32).  A drawn site already owned by a seed   */
/* placed in an earlier round is lost; a site drawn by several seeds in the  */
/* same round goes to the lowest g.  Losers draw again in round a+1.         */
/* ------------------------------------------------------------------------ */
int oracle_voronoi_seeds(int dim, const int64_t* L, int32_t G, uint64_t seed, int64_t* pos) {
    const int64_t N = L[0] * L[1] * (dim == 3 ? L[2] : 1);
    if (G < 1 || (int64_t)G > N || N >= ((int64_t)1 << 32)) return OR_ERR_ARG;
    int32_t* owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    char* placed = (char*)calloc((size_t)G, 1);
    int64_t* want = (int64_t*)malloc(sizeof(int64_t) * (size_t)G);
    if (!owner || !placed || !want) { free(owner); free(placed); free(want); return OR_ERR_ARG; }
    for (int64_t s = 0; s < N; ++s) owner[s] = -1;
    int32_t left = G;
    for (uint32_t a = 0; left > 0; ++a) {
        for (int32_t g = 0; g < G; ++g) {
            if (placed[g]) continue;
            uint32_t u[4];
            draw(seed, (uint64_t)g, a, TAG_VORONOI, 0, u);
            want[g] = (int64_t)(((uint64_t)u[0] * (uint64_t)N) >> 32);
        }
        /* lowest unplaced g wins each free site (scan g ascending) */
        for (int32_t g = 0; g < G; ++g) {
            if (placed[g]) continue;
            if (owner[want[g]] == -1) { owner[want[g]] = g; placed[g] = 2; pos[g] = want[g]; }
        }
        for (int32_t g = 0; g < G; ++g)
            if (placed[g] == 2) { placed[g] = 1; --left; }
    }
    free(owner); free(placed); free(want);
    return OR_OK;
}

static int64_t min_image(int64_t d, int64_t L) { if (d < 0) d = -d; return d < L - d ? d : L - d; }

/* Nearest seed under the periodic minimum-image squared integer distance;  */
/* ties go to the lowest seed index.  Brute force over all seeds.            */
int32_t oracle_voronoi_site(int dim, const int64_t* L, int32_t G, const int64_t* pos, int64_t site) {
    const int64_t Lx = L[0], Ly = L[1], Lz = dim == 3 ? L[2] : 1;
    const int64_t x = site % Lx, y = (site / Lx) % Ly, z = site / (Lx * Ly);
    int64_t best = -1; int32_t arg = -1;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t sx = pos[g] % Lx, sy = (pos[g] / Lx) % Ly, sz = pos[g] / (Lx * Ly);
        const int64_t dx = min_image(x - sx, Lx), dy = min_image(y - sy, Ly), dz = min_image(z - sz, Lz);
        const int64_t d2 = dx * dx + dy * dy + dz * dz;
        if (best < 0 || d2 < best) { best = d2; arg = g; }
    }
    return arg;
}

int oracle_voronoi(int dim, const int64_t* L, int32_t G, uint64_t seed, int32_t* q, int64_t* pos_out) {
    const int64_t N = L[0] * L[1] * (dim == 3 ? L[2] : 1);
    int64_t* pos = pos_out ? pos_out : (int64_t*)malloc(sizeof(int64_t) * (size_t)G);
    if (!pos) return OR_ERR_ARG;
    int rc = oracle_voronoi_seeds(dim, L, G, seed, pos);
    if (rc == OR_OK)
        for (int64_t s = 0; s < N; ++s) q[s] = oracle_voronoi_site(dim, L, G, pos, s);
    if (!pos_out) free(pos);
    return rc;
}

/* Grain orientations from Philox(seed; g, 0, TAG_VORONOI<<24 | 1).
 * kind 0: single rotation angle about z, angle = (u0 / 2^32) * pi/2 (the
 *         paper's one-angle grains, Sec. 5), rounded to FP32.
 * kind 2: the kind-0 angle t as the quaternion (cos t/2, 0, 0, sin t/2) of a
 *         rotation about z, rounded to FP32.
 * kind 1: unit quaternion (w,x,y,z) uniform on SO(3) by Shoemake's method
 *         ("Uniform random rotations", Graphics Gems III, 1992) from
 *         u1,u2,u3 = u0,u1,u2 / 2^32, computed in FP64, rounded to FP32:
 *         w = sqrt(1-u1) sin(2 pi u2), x = sqrt(1-u1) cos(2 pi u2),
 *         y = sqrt(u1) sin(2 pi u3),   z = sqrt(u1) cos(2 pi u3).      */
int oracle_orientations(int32_t G, uint64_t seed, int kind, float* out) {
    const double two32 = 4294967296.0, pi = 3.14159265358979323846;
    for (int32_t g = 0; g < G; ++g) {
        uint32_t u[4];
        draw(seed, (uint64_t)g, 0, TAG_VORONOI, 1, u);
        if (kind == 0) {
            out[g] = (float)(((double)u[0] / two32) * (pi / 2.0));
        } else if (kind == 2) {
            /* the same angle as kind 0, as the quaternion of a rotation about z */
            const double t = ((double)u[0] / two32) * (pi / 2.0);
            out[4 * g + 0] = (float)cos(0.5 * t);
            out[4 * g + 1] = 0.0f;
            out[4 * g + 2] = 0.0f;
            out[4 * g + 3] = (float)sin(0.5 * t);
        } else if (kind == 1) {
            const double u1 = (double)u[0] / two32, u2 = (double)u[1] / two32, u3 = (double)u[2] / two32;
            const double a = sqrt(1.0 - u1), c = sqrt(u1);
            out[4 * g + 0] = (float)(a * sin(2.0 * pi * u2));
            out[4 * g + 1] = (float)(a * cos(2.0 * pi * u2));
            out[4 * g + 2] = (float)(c * sin(2.0 * pi * u3));
            out[4 * g + 3] = (float)(c * cos(2.0 * pi * u3));
        } else {
            return OR_ERR_ARG;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Grain statistics (Sec. 4, average grain size; Sec. 5, texture).           */
/* counts[g] = number of sites with q == g; alive = #{g : counts[g] > 0}.    */
/* ------------------------------------------------------------------------ */
int oracle_grain_counts(int64_t N, const int32_t* q, int32_t G, int64_t* counts, int32_t* alive) {
    for (int32_t g = 0; g < G; ++g) counts[g] = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (q[i] < 0 || q[i] >= G) return OR_ERR_ARG;
        counts[q[i]]++;
    }
    int32_t a = 0;
    for (int32_t g = 0; g < G; ++g) a += counts[g] > 0;
    *alive = a;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Rotation and cubic elasticity (FP64, full tensors, plain definitions).    */
/* R(q) maps crystal to sample axes: v_sample = R v_crystal, q = (w,x,y,z).  */
/* ------------------------------------------------------------------------ */
static void quat_to_R(const double qin[4], double R[3][3]) {
    const double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    const double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Cubic stiffness C_ijkl = C12 d_ij d_kl + C44 (d_ik d_jl + d_il d_jk)
 *                         + (C11 - C12 - 2 C44) sum_a d_ia d_ja d_ka d_la    */
static double cubic_C(const double Cc[3], int i, int j, int k, int l) {
    const double C11 = Cc[0], C12 = Cc[1], C44 = Cc[2];
    double v = C12 * (i == j) * (k == l) + C44 * ((i == k) * (j == l) + (i == l) * (j == k));
    if (i == j && j == k && k == l) v += C11 - C12 - 2.0 * C44;
    return v;
}

static void C_apply(const double Cc[3], const double e[3][3], double s[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) a += cubic_C(Cc, i, j, k, l) * e[k][l];
            s[i][j] = a;
        }
}

static double ddot(const double a[3][3], const double b[3][3]) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += a[i][j] * b[i][j];
    return s;
}

/* FCC {111}<110> slip systems: plane normals n and slip directions m
 * (unnormalised integer vectors, normalised on use).  The order fixes the
 * index alpha of Eq. (1)-(2).                                               */
static const int FCC_N[12][3] = {
    {1, 1, 1}, {1, 1, 1}, {1, 1, 1},
    {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
    {1, -1, 1}, {1, -1, 1}, {1, -1, 1},
    {1, 1, -1}, {1, 1, -1}, {1, 1, -1}};
static const int FCC_M[12][3] = {
    {0, 1, -1}, {-1, 0, 1}, {1, -1, 0},
    {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
    {0, 1, 1}, {1, 0, -1}, {1, 1, 0},
    {0, 1, 1}, {1, 0, 1}, {1, -1, 0}};

/* Schmid tensor P = sym(m (x) n) with unit m, n (crystal frame). */
static void schmid_tensor(int a, double P[3][3]) {
    double n[3], m[3];
    const double sn = 1.0 / sqrt(3.0), sm = 1.0 / sqrt(2.0);
    for (int i = 0; i < 3; ++i) { n[i] = FCC_N[a][i] * sn; m[i] = FCC_M[a][i] * sm; }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i][j] = 0.5 * (m[i] * n[j] + n[i] * m[j]);
}

void oracle_slip_systems(double* n_out, double* m_out) {
    const double sn = 1.0 / sqrt(3.0), sm = 1.0 / sqrt(2.0);
    for (int a = 0; a < 12; ++a)
        for (int i = 0; i < 3; ++i) { n_out[3 * a + i] = FCC_N[a][i] * sn; m_out[3 * a + i] = FCC_M[a][i] * sm; }
}

/* ------------------------------------------------------------------------ */
/* Closed-form per-grain energies under uniaxial stress sigma along sample x */
/* (Sec. 5: "uniaxial loading ... in the x-direction").                      */
/*   d      = loading axis in the crystal frame = R^T e_x                    */
/*   m_max  = max_alpha |(d.n_alpha)(d.m_alpha)| (Schmid factor, Fig. 4)     */
/*   E(d)   = 1 / (d (x) d : S : d (x) d), S = C^-1 (directional modulus)    */
/*   w      = sigma^2 / (2 E(d))  (elastic energy density, uniaxial stress)  */
/* S is obtained by inverting the 6x6 Voigt matrix of C numerically (no      */
/* closed-form compliance formula is used), so the directional modulus is    */
/* the definition itself.                                                    */
/* ------------------------------------------------------------------------ */
static int invert6(double A[6][6], double Ainv[6][6]) {
    double M[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) M[i][j] = j < 6 ? A[i][j] : (j - 6 == i ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int p = c;
        for (int r = c + 1; r < 6; ++r) if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (fabs(M[p][c]) < 1e-300) return OR_ERR_ARG;
        if (p != c) for (int j = 0; j < 12; ++j) { double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
        const double piv = M[c][c];
        for (int j = 0; j < 12; ++j) M[c][j] /= piv;
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            const double f = M[r][c];
            for (int j = 0; j < 12; ++j) M[r][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) Ainv[i][j] = M[i][j + 6];
    return OR_OK;
}

/* Voigt index pairs: 0:xx 1:yy 2:zz 3:yz 4:xz 5:xy */
static const int VI[6] = {0, 1, 2, 1, 0, 0}, VJ[6] = {0, 1, 2, 2, 2, 1};

double oracle_directional_modulus(const double Cc[3], const double d_in[3]) {
    double A[6][6], S[6][6];
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) A[I][J] = cubic_C(Cc, VI[I], VJ[I], VI[J], VJ[J]);
    /* engineering shear strain: sigma_I = A_IJ eps_J with eps_J = 2 e_ij for J>=3 */
    if (invert6(A, S) != OR_OK) return NAN;
    const double nn = sqrt(d_in[0] * d_in[0] + d_in[1] * d_in[1] + d_in[2] * d_in[2]);
    const double d[3] = {d_in[0] / nn, d_in[1] / nn, d_in[2] / nn};
    /* uniaxial stress sigma = d (x) d (unit); strain = S sigma; normal strain along d */
    double sv[6], ev[6];
    for (int I = 0; I < 6; ++I) sv[I] = d[VI[I]] * d[VJ[I]];
    for (int I = 0; I < 6; ++I) { ev[I] = 0.0; for (int J = 0; J < 6; ++J) ev[I] += S[I][J] * sv[J]; }
    /* eps_dd = sum_ij d_i e_ij d_j ; e_ij = ev/2 for shear */
    double e[3][3];
    for (int I = 0; I < 6; ++I) {
        const double v = I < 3 ? ev[I] : 0.5 * ev[I];
        e[VI[I]][VJ[I]] = v; e[VJ[I]][VI[I]] = v;
    }
    double edd = 0.0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) edd += d[i] * e[i][j] * d[j];
    return 1.0 / edd;
}

double oracle_max_schmid(const double d_in[3]) {
    const double nn = sqrt(d_in[0] * d_in[0] + d_in[1] * d_in[1] + d_in[2] * d_in[2]);
    const double d[3] = {d_in[0] / nn, d_in[1] / nn, d_in[2] / nn};
    const double sn = 1.0 / sqrt(3.0), sm = 1.0 / sqrt(2.0);
    double best = 0.0;
    for (int a = 0; a < 12; ++a) {
        double dn = 0.0, dm = 0.0;
        for (int i = 0; i < 3; ++i) { dn += d[i] * FCC_N[a][i] * sn; dm += d[i] * FCC_M[a][i] * sm; }
        const double m = fabs(dn * dm);
        if (m > best) best = m;
    }
    return best;
}

/* Per-grain loading axis in the crystal frame from an FP32 quaternion. */
void oracle_loading_axis(const float* quat, double d[3]) {
    double q[4] = {quat[0], quat[1], quat[2], quat[3]}, R[3][3];
    quat_to_R(q, R);
    d[0] = R[0][0]; d[1] = R[0][1]; d[2] = R[0][2];   /* R^T e_x = first row of R */
}

/* Per-grain closed-form field (uniaxial sigma [MPa] along x):
 *   w[g]    = sigma^2 / (2 E(d_g))         [MJ/m^3]
 *   mmax[g] = max Schmid factor of d_g
 *   e[g]    = energy_scale * (w[g] + k_disl * mmax[g])   [J, MC units]
 *   bfix[g] = round-half-even(256 e[g]) clamped to [-2^20, 2^20]            */
int oracle_grain_field(int32_t G, const float* quat, const double Cc[3], double sigma, double k_disl,
                       double energy_scale, double* w, double* mmax, double* e, int32_t* bfix) {
    for (int32_t g = 0; g < G; ++g) {
        double d[3];
        oracle_loading_axis(quat + 4 * g, d);
        const double E = oracle_directional_modulus(Cc, d);
        w[g] = sigma * sigma / (2.0 * E);
        mmax[g] = oracle_max_schmid(d);
        e[g] = energy_scale * (w[g] + k_disl * mmax[g]);
        double v = nearbyint(256.0 * e[g]);
        if (v > 1048576.0) v = 1048576.0;
        if (v < -1048576.0) v = -1048576.0;
        bfix[g] = (int32_t)v;
    }
    return OR_OK;
}

/* Fixed-point quantisation of energies in J (MC units), round half to even,
 * clamped to +-2^20: b = rint(256 * e).                                     */
void oracle_quantise(int64_t n, const double* e, int32_t* b) {
    for (int64_t i = 0; i < n; ++i) {
        double v = nearbyint(256.0 * e[i]);
        if (v > 1048576.0) v = 1048576.0;
        if (v < -1048576.0) v = -1048576.0;
        b[i] = (int32_t)v;
    }
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo crystal plasticity (Sec. 2, Eqs. (1)-(3), Table 1).           */
/* Per material point p with crystal orientation q_p, one load increment t:  */
/*  1. total sample strain eps_s = t * e * diag(1, -1/2, -1/2)  (Eq. (3),    */
/*     Taylor: every point sees the prescribed increment)                    */
/*  2. crystal frame eps_c = R^T eps_s R; trial elastic strain               */
/*     ee_tr = eps_c - eps_p; trial stress s_tr = C : ee_tr                  */
/*  3. slip resistance g(gamma) (Voce: tau_s - (tau_s - tau_0)               */
/*     exp(-h0 gamma/(tau_s - tau_0)), isotropic: one g for all systems)     */
/*  4. candidate set zeta = {alpha : |s_tr : P_alpha| > g}                   */
/*  5. for each candidate alone: single-slip return map, the one equation    */
/*     |tau_tr| - dg (P:C:P) = g(gamma + dg), solved by Newton in FP64;      */
/*     trial state ee = ee_tr - dg sign(tau) P; energy E = 1/2 ee : C : ee   */
/*  6. p_alpha = exp(-beta E_alpha) / Z  (Eq. (1); shifted by min E)         */
/*  7. R = u0 / 2^32 from Philox(seed; p, t, TAG_MCP<<24); pick the first    */
/*     i in zeta order with R < sum_{alpha<=i} p_alpha  (Eq. (2))            */
/*  8. commit eps_p += dg_i sign_i P_i; gamma += dg_i                        */
/* Units: MPa for stresses and moduli, MJ/m^3 for energies.                  */
/* state layout per point (FP64): eps_p[6] (Voigt tensor components xx yy zz */
/* yz xz xy, not engineering), gamma.  sigma_out[6] = C : (eps_c - eps_p).   */
/* near[p] returns the smallest distance |R - boundary| and |(|tau|-g)|/g   */
/* seen (for near-tie bookkeeping in the parity tests).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double C11, C12, C44, tau0, taus, h0, beta, G, e_incr;
} oracle_cp_params;

static double voce(const oracle_cp_params* P, double gamma) {
    const double dt = P->taus - P->tau0;
    if (dt <= 0.0 || P->h0 <= 0.0) return P->tau0;   /* no hardening: g = tau_0 */
    return P->taus - dt * exp(-P->h0 * gamma / dt);
}

/* dg/dgamma of the Voce law (h0 at gamma = 0). */
static double voce_slope(const oracle_cp_params* P, double gamma) {
    const double dt = P->taus - P->tau0;
    if (dt <= 0.0 || P->h0 <= 0.0) return 0.0;
    return P->h0 * exp(-P->h0 * gamma / dt);
}

static void sym_from_voigt(const double* v, double t[3][3]) {
    t[0][0] = v[0]; t[1][1] = v[1]; t[2][2] = v[2];
    t[1][2] = t[2][1] = v[3]; t[0][2] = t[2][0] = v[4]; t[0][1] = t[1][0] = v[5];
}
static void voigt_from_sym(const double t[3][3], double* v) {
    v[0] = t[0][0]; v[1] = t[1][1]; v[2] = t[2][2]; v[3] = t[1][2]; v[4] = t[0][2]; v[5] = t[0][1];
}

/* One increment t of one material point whose total strain in the sample
 * frame is es_v (Voigt xx yy zz yz xz xy, tensor components): the Taylor form
 * of Eq. (3) below passes t e diag(1, -1/2, -1/2); the elastic-equilibrium
 * coupling passes the point's own strain from the periodic elastic solve.      */
int oracle_mcp_increment_strain(const oracle_cp_params* P, uint64_t seed, int64_t p_index, uint32_t t,
                                const float* quat, const double* es_v, double* eps_p_v, double* gamma,
                                double* sigma_v, double* near_R, double* near_tau, int32_t* chosen,
                                int32_t* n_cand);

int oracle_mcp_increment(const oracle_cp_params* P, uint64_t seed, int64_t p_index, uint32_t t,
                         const float* quat, double* eps_p_v, double* gamma, double* sigma_v,
                         double* near_R, double* near_tau, int32_t* chosen, int32_t* n_cand) {
    const double es_v[6] = {(double)t * P->e_incr, -0.5 * (double)t * P->e_incr, -0.5 * (double)t * P->e_incr,
                            0.0, 0.0, 0.0};
    return oracle_mcp_increment_strain(P, seed, p_index, t, quat, es_v, eps_p_v, gamma, sigma_v, near_R, near_tau,
                                       chosen, n_cand);
}

int oracle_mcp_increment_strain(const oracle_cp_params* P, uint64_t seed, int64_t p_index, uint32_t t,
                                const float* quat, const double* es_v, double* eps_p_v, double* gamma,
                                double* sigma_v, double* near_R, double* near_tau, int32_t* chosen,
                                int32_t* n_cand) {
    const double Cc[3] = {P->C11, P->C12, P->C44};
    double q[4] = {quat[0], quat[1], quat[2], quat[3]}, R[3][3];
    quat_to_R(q, R);
    double es[3][3];
    sym_from_voigt(es_v, es);
    double ec[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) a += R[k][i] * es[k][l] * R[l][j];
            ec[i][j] = a;
        }
    double ep[3][3], ee[3][3], s[3][3];
    sym_from_voigt(eps_p_v, ep);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) ee[i][j] = ec[i][j] - ep[i][j];
    C_apply(Cc, ee, s);
    const double g = voce(P, *gamma);
    double tau[12], dg[12], E[12], sgn[12];
    int cand[12], nc = 0;
    double ntau = INFINITY;
    for (int a = 0; a < 12; ++a) {
        double Pa[3][3];
        schmid_tensor(a, Pa);
        tau[a] = ddot(s, Pa);
        const double m = fabs(fabs(tau[a]) - g) / g;
        if (m < ntau) ntau = m;
        if (fabs(tau[a]) > g) cand[nc++] = a;
    }
    if (near_tau) *near_tau = ntau;
    if (near_R) *near_R = INFINITY;
    if (n_cand) *n_cand = nc;
    if (chosen) *chosen = -1;
    if (nc > 0) {
        double Emin = INFINITY;
        for (int c = 0; c < nc; ++c) {
            const int a = cand[c];
            double Pa[3][3], CP[3][3];
            schmid_tensor(a, Pa);
            C_apply(Cc, Pa, CP);
            const double k = ddot(Pa, CP);
            const double at = fabs(tau[a]);
            sgn[a] = tau[a] > 0 ? 1.0 : -1.0;
            /* Newton on f(x) = |tau| - x k - g(gamma + x), f(0) > 0, f decreasing */
            double x = 0.0;
            for (int it = 0; it < 100; ++it) {
                const double gx = voce(P, *gamma + x);
                const double hx = voce_slope(P, *gamma + x);
                const double f = at - x * k - gx;
                if (fabs(f) < 1e-13 * P->tau0 && it > 0) break;
                x -= f / (-k - hx);
            }
            dg[a] = x;
            double e2[3][3], s2[3][3];
            for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) e2[i][j] = ee[i][j] - x * sgn[a] * Pa[i][j];
            C_apply(Cc, e2, s2);
            E[a] = 0.5 * ddot(e2, s2);
            if (E[a] < Emin) Emin = E[a];
        }
        double w[12], Z = 0.0;
        for (int c = 0; c < nc; ++c) { w[c] = exp(-P->beta * (E[cand[c]] - Emin)); Z += w[c]; }
        uint32_t u[4];
        draw(seed, (uint64_t)p_index, t, TAG_MCP, 0, u);
        const double Rn = (double)u[0] / 4294967296.0;
        double cum = 0.0, nr = INFINITY;
        int pick = nc - 1;
        int found = 0;
        for (int c = 0; c < nc; ++c) {
            cum += w[c] / Z;
            if (c < nc - 1 && fabs(Rn - cum) < nr) nr = fabs(Rn - cum);
            if (!found && Rn < cum) { pick = c; found = 1; }
        }
        if (near_R) *near_R = nr;
        const int a = cand[pick];
        if (chosen) *chosen = a;
        double Pa[3][3];
        schmid_tensor(a, Pa);
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) ep[i][j] += dg[a] * sgn[a] * Pa[i][j];
        *gamma += dg[a];
        voigt_from_sym(ep, eps_p_v);
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) ee[i][j] = ec[i][j] - ep[i][j];
        C_apply(Cc, ee, s);
    }
    voigt_from_sym(s, sigma_v);
    return OR_OK;
}

/* Candidate set and probabilities of Eq. (1) for one state (no commit), for
 * the statistical selection test: returns n = |zeta|, cand[] and prob[].     */
int oracle_mcp_probabilities(const oracle_cp_params* P, uint32_t t, const float* quat,
                             const double* eps_p_v, double gamma, int32_t* cand_out, double* prob_out) {
    const double Cc[3] = {P->C11, P->C12, P->C44};
    double q[4] = {quat[0], quat[1], quat[2], quat[3]}, R[3][3];
    quat_to_R(q, R);
    double es[3][3] = {{0}}, ec[3][3], epm[3][3], ee[3][3], s[3][3];
    es[0][0] = (double)t * P->e_incr; es[1][1] = es[2][2] = -0.5 * (double)t * P->e_incr;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) a += R[k][i] * es[k][l] * R[l][j];
            ec[i][j] = a;
        }
    sym_from_voigt(eps_p_v, epm);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) ee[i][j] = ec[i][j] - epm[i][j];
    C_apply(Cc, ee, s);
    const double g = voce(P, gamma);
    double E[12], Emin = INFINITY;
    int n = 0;
    for (int a = 0; a < 12; ++a) {
        double Pa[3][3], CP[3][3];
        schmid_tensor(a, Pa);
        const double tau = ddot(s, Pa);
        if (!(fabs(tau) > g)) continue;
        C_apply(Cc, Pa, CP);
        const double k = ddot(Pa, CP), at = fabs(tau), sg2 = tau > 0 ? 1.0 : -1.0;
        double x = 0.0;
        for (int it = 0; it < 100; ++it) {
            const double f = at - x * k - voce(P, gamma + x);
            if (fabs(f) < 1e-13 * P->tau0 && it > 0) break;
            x -= f / (-k - voce_slope(P, gamma + x));
        }
        double e2[3][3], s2[3][3];
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) e2[i][j] = ee[i][j] - x * sg2 * Pa[i][j];
        C_apply(Cc, e2, s2);
        E[n] = 0.5 * ddot(e2, s2);
        if (E[n] < Emin) Emin = E[n];
        cand_out[n++] = a;
    }
    double Z = 0.0;
    for (int c = 0; c < n; ++c) { prob_out[c] = exp(-P->beta * (E[c] - Emin)); Z += prob_out[c]; }
    for (int c = 0; c < n; ++c) prob_out[c] /= Z;
    return n;
}

/* Run n_incr increments t = t0+1 .. t0+n_incr over P points; state arrays are
 * FP64 SoA: eps_p[6*P] (point-major), gamma[P].  Orientation of point p is
 * quat[4*grain[p]].  Returns sigma[6*P] after the last increment, and per
 * point the smallest near-tie distances over all increments.                 */
int oracle_mcp_run(const oracle_cp_params* P, uint64_t seed, int64_t npts, const int32_t* grain,
                   const float* quat, uint32_t t0, int32_t n_incr, double* eps_p, double* gamma,
                   double* sigma, double* near_R, double* near_tau) {
    for (int64_t p = 0; p < npts; ++p) {
        double nr_min = INFINITY, nt_min = INFINITY;
        for (int32_t s = 1; s <= n_incr; ++s) {
            double nr, nt;
            int32_t ch, nc;
            oracle_mcp_increment(P, seed, p, t0 + (uint32_t)s, quat + 4 * grain[p], eps_p + 6 * p, gamma + p,
                                 sigma + 6 * p, &nr, &nt, &ch, &nc);
            if (nr < nr_min) nr_min = nr;
            if (nt < nt_min) nt_min = nt;
        }
        if (near_R) near_R[p] = nr_min;
        if (near_tau) near_tau[p] = nt_min;
    }
    return OR_OK;
}

/* One increment t over P points, point p with its own sample-frame total
 * strain eps_total[6*p..] (the elastic-equilibrium coupling).                  */
int oracle_mcp_run_strain(const oracle_cp_params* P, uint64_t seed, int64_t npts, const int32_t* grain,
                          const float* quat, uint32_t t, const double* eps_total, double* eps_p, double* gamma,
                          double* sigma, double* near_R, double* near_tau) {
    for (int64_t p = 0; p < npts; ++p) {
        double nr, nt;
        int32_t ch, nc;
        oracle_mcp_increment_strain(P, seed, p, t, quat + 4 * grain[p], eps_total + 6 * p, eps_p + 6 * p,
                                    gamma + p, sigma + 6 * p, &nr, &nt, &ch, &nc);
        if (near_R) near_R[p] = nr;
        if (near_tau) near_tau[p] = nt;
    }
    return OR_OK;
}

/* Energies of a material point after an increment (Sec. 3, Eq. (4)):
 *   sigma_f = g(gamma) (the current slip resistance),
 *   E_rho = 1/2 rho G b^2 with rho = (2 sigma_f / (G b))^2, i.e. 2 sigma_f^2 / G
 *   w     = 1/2 sigma : C^-1 : sigma (elastic energy density)
 * G is the Voigt average shear modulus (C11 - C12 + 3 C44) / 5.              */
int oracle_mcp_energies(const oracle_cp_params* P, int64_t npts, const double* sigma, const double* gamma,
                        double* w, double* Erho) {
    const double Cc[3] = {P->C11, P->C12, P->C44};
    double A[6][6], S[6][6];
    for (int I = 0; I < 6; ++I) for (int J = 0; J < 6; ++J) A[I][J] = cubic_C(Cc, VI[I], VJ[I], VI[J], VJ[J]);
    if (invert6(A, S) != OR_OK) return OR_ERR_ARG;
    for (int64_t p = 0; p < npts; ++p) {
        const double* s = sigma + 6 * p;
        /* Voigt: stress vector (s_xx, s_yy, s_zz, s_yz, s_xz, s_xy); strain = S sigma
         * (engineering shears), energy = 1/2 sum_I sigma_I strain_I */
        double e = 0.0;
        for (int I = 0; I < 6; ++I) { double a = 0.0; for (int J = 0; J < 6; ++J) a += S[I][J] * s[J]; e += s[I] * a; }
        w[p] = 0.5 * e;
        const double sf = voce(P, gamma[p]);
        /* dislocation density and energy with a unit Burgers vector; b cancels */
        const double bg = 1.0, rho = (2.0 * sf / (P->G * bg)) * (2.0 * sf / (P->G * bg));
        Erho[p] = 0.5 * rho * P->G * bg * bg;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Texture bins per grain (Sec. 5 orientation distributions).                */
/* kind 0 (one rotation angle about z) and kind 2 (its quaternion, angle      */
/*        2 atan2(z, w)): bin = floor(angle * 180/pi), clamped               */
/*        to 0..89 (1 degree bins over [0, 90)).                             */
/* kind 1 (SO(3) quaternion): bins[2g] = floor(m_max / 0.5 * 20) clamped to  */
/*        0..19; bins[2g+1] = 20 + family, family 1/2/3 when the loading     */
/*        axis lies within 15 degrees of a <100>/<110>/<111> direction, else */
/*        0.  hist layout for kind 1: 20 m_max bins, then 4 family bins.     */
/* near[g] = distance of the deciding value to its nearest bin edge.         */
/* ------------------------------------------------------------------------ */
int oracle_grain_bins(int32_t G, int kind, const float* orient, int32_t* bins, double* near) {
    const double pi = 3.14159265358979323846;
    const double c15 = cos(15.0 * pi / 180.0);
    for (int32_t g = 0; g < G; ++g) {
        if (kind == 0 || kind == 2) {
            const double t = kind == 0 ? (double)orient[g]
                                       : 2.0 * atan2((double)orient[4 * g + 3], (double)orient[4 * g]);
            const double deg = t * (180.0 / pi);
            double f = floor(deg);
            int b = (int)f;
            if (b < 0) b = 0;
            if (b > 89) b = 89;
            bins[g] = b;
            if (near) near[g] = fmin(deg - f, f + 1.0 - deg);
        } else if (kind == 1) {
            double d[3];
            oracle_loading_axis(orient + 4 * g, d);
            const double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int i = 0; i < 3; ++i) d[i] = fabs(d[i] / nn);
            const double mm = oracle_max_schmid(d);
            const double v = mm / 0.5 * 20.0;
            double f = floor(v);
            int b = (int)f;
            if (b < 0) b = 0;
            if (b > 19) b = 19;
            bins[2 * g] = b;
            /* cosines to the nearest member of each family */
            const double c100 = fmax(d[0], fmax(d[1], d[2]));
            const double c110 = fmax(d[0] + d[1], fmax(d[1] + d[2], d[0] + d[2])) / sqrt(2.0);
            const double c111 = (d[0] + d[1] + d[2]) / sqrt(3.0);
            int fam = 0;
            if (c100 > c15) fam = 1;
            else if (c110 > c15) fam = 2;
            else if (c111 > c15) fam = 3;
            bins[2 * g + 1] = 20 + fam;
            if (near) {
                double nr = fmin(v - f, f + 1.0 - v);
                nr = fmin(nr, fabs(c100 - c15));
                nr = fmin(nr, fabs(c110 - c15));
                nr = fmin(nr, fabs(c111 - c15));
                near[g] = nr;
            }
        } else {
            return OR_ERR_ARG;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* One colour phase on a slab with ghost layers (the domain decomposition of */
/* Sec. 4: the lattice is divided among processors, which exchange boundary  */
/* layers at every half step).  The slab holds global layers                 */
/* [s0 - 1, s0 + ns + 1) of the slowest axis (y in 2D, z in 3D), periodic;   */
/* only colour-c sites of the owned layers [s0, s0 + ns) are updated, with   */
/* the same keyed draws (global site index) as oracle_sweep, so a run over   */
/* slabs with exchanged ghost layers equals the undecomposed run.            */
/* q, b, mp: (ns + 2) layers of the slab (b, mp may be NULL).                */
/* ------------------------------------------------------------------------ */
int oracle_sweep_phase_slab(int dim, const int64_t* L, int nbr, int32_t J_fix, uint64_t seed, uint32_t sweep,
                            int colour, const uint32_t* thr, int32_t D, int64_t s0, int64_t ns,
                            int32_t* q, int32_t* b, int32_t* mp, int64_t* n_flips) {
    off3 o[26];
    const int M = neighbourhood(dim, nbr, o);
    if (!M || !q || !thr || ns < 1) return OR_ERR_ARG;
    const int64_t Lx = L[0], Ly = L[1], Lz = dim == 3 ? L[2] : 1;
    const int64_t Ls = dim == 3 ? Lz : Ly;      /* slowest axis */
    const int64_t layer = dim == 3 ? Lx * Ly : Lx;
    int64_t flips = 0;
    for (int64_t t = 0; t < ns; ++t) {
        const int64_t gs = s0 + t;              /* global layer */
        for (int64_t r = 0; r < layer; ++r) {
            const int64_t x = r % Lx, y = dim == 3 ? r / Lx : gs, z = dim == 3 ? gs : 0;
            if (colour_of(dim, nbr, x, y, z) != colour) continue;
            const int64_t li = (t + 1) * layer + r;
            int64_t nb[26];
            for (int k = 0; k < M; ++k) {
                const int64_t xx = wrap(x + o[k].dx, Lx);
                int64_t ll;
                if (dim == 3) {
                    const int64_t yy = wrap(y + o[k].dy, Ly);
                    ll = (t + 1 + o[k].dz) * layer + xx + Lx * yy;
                } else {
                    ll = (t + 1 + o[k].dy) * layer + xx;
                }
                nb[k] = ll;
            }
            const int64_t gi = x + Lx * (y + Ly * z);
            uint32_t u[4];
            draw(seed, (uint64_t)gi, sweep, TAG_SWEEP, (uint32_t)colour, u);
            const int k = (int)(((uint64_t)u[0] * (uint64_t)M) >> 32);
            const int64_t j = nb[k];
            const int32_t qi = q[li], qj = q[j];
            if (qj == qi) continue;
            int same_old = 0, same_new = 0;
            for (int n = 0; n < M; ++n) {
                same_old += q[nb[n]] == qi;
                same_new += q[nb[n]] == qj;
            }
            const int32_t db = b ? (b[j] - b[li]) : 0;
            const int32_t d = J_fix * (same_old - same_new) + db;
            int accept;
            if (d < 0) accept = 1;
            else if (d > D) accept = 0;
            else accept = thr[d] == 0xFFFFFFFFu || u[1] < thr[d];
            if (accept) {
                q[li] = qj;
                if (b) b[li] = b[j];
                if (mp) mp[li] = mp[j];
                ++flips;
            }
        }
    }
    (void)Ls;
    if (n_flips) *n_flips = flips;
    return OR_OK;
}

/* Orientation-dependent Gaussian bulk energy, Eq. (9): orientation
 * n = floor(angle in degrees) + 1 and e = (32 pi)^(-1/2) exp(-(n-46)^2/(2 46^2)). */
void oracle_gaussian_field(int32_t G, const float* angle, double scale, double* e, int32_t* b) {
    const double pi = 3.14159265358979323846;
    for (int32_t g = 0; g < G; ++g) {
        int bin = (int)floor((double)angle[g] * (180.0 / pi));
        bin = bin < 0 ? 0 : (bin > 89 ? 89 : bin);
        const double n = bin + 1.0;
        e[g] = scale * exp(-(n - 46.0) * (n - 46.0) / (2.0 * 46.0 * 46.0)) / sqrt(32.0 * pi);
        b[g] = (int32_t)nearbyint(256.0 * e[g]);
    }
}
