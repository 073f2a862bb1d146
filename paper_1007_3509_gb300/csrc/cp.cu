// Monte Carlo crystal plasticity (Sec. 2, Eqs. (1)-(3), Table 1) and the
// per-point driving field (Sec. 3, Eq. (4)).  One thread per material point.
//
// Per increment t (Eq. (3), Taylor: every point takes the prescribed strain):
//   eps_c = R^T (t e diag(1,-1/2,-1/2)) R          crystal-frame total strain
//   ee = eps_c - eps_p; s = C : ee                   trial stress (FP32)
//   tau_a = m_a . s . n_a; zeta = {a : |tau_a| > g}  candidates (FP32)
//   per candidate, the single-slip return map |tau_a| - x k = g(gamma + x),
//   k = P:C:P, Voce g(gamma + x) = taus - (taus - g) exp(-h0 x/(taus - tau0));
//   energy change of the candidate state  dE_a = -x |tau_a| + x^2 k / 2
//   (E_a = 1/2 ee_a : C : ee_a with ee_a = ee - x sign(tau_a) P_a).  For the
//   selection the candidates use the first Newton iterate from x = 0 in FP32
//   (relative error ~1e-6 for load steps of 1e-4); the chosen system's map is
//   then solved in FP64 (for hr x <= 1e-2 three fixed-point steps on the cubic
//   Taylor form of the Voce term, relative error ~1e-10; Newton otherwise) and
//   committed, the new resistance from consistency, g = |tau| - k x;
//   p_a = exp(-beta (dE_a - min dE)) / Z (Eq. (1)); R = u0 / 2^32 from
//   Philox(seed; p, t, tag 1); first a with R < sum_{b<=a} p_b (Eq. (2)),
//   all in FP32 (FP64 is kept for the return map alone);
//   commit eps_p += x sign P, gamma += x, g = g(gamma + x).
// After the last increment: sigma = C : (eps_c - eps_p); E_rho = 2 g^2 / G
// (Eq. (4) with sigma_f = g; the Burgers vector cancels); w = 1/2 sigma : ee;
// b = round-half-even(256 scale (w_weight w + E_rho)) clamped to +-2^20.
#include <math.h>

#include "common.cuh"

namespace hp {
namespace {

constexpr int kT = 128;

__constant__ float c_m[12][3];
__constant__ float c_n[12][3];
__constant__ double c_k[12];  // P:C:P per system
__constant__ float c_kf[12];

// Constants of the single-slip return map for Voce hardening (taus, tau0, h0).
struct RMConsts {
    double taus, tau0, hr;  // hr = h0 / (taus - tau0); 0 without hardening
    float taus32, hr32, hr2h, hr3s;
    bool hard;
};

__host__ __device__ inline RMConsts rm_consts(double tau0, double taus, double h0) {
    RMConsts c;
    c.hard = taus - tau0 > 0.0 && h0 > 0.0;
    c.taus = taus;
    c.tau0 = tau0;
    c.hr = c.hard ? h0 / (taus - tau0) : 0.0;
    c.taus32 = (float)taus;
    c.hr32 = (float)c.hr;
    // series coefficients of 1 - exp(-hr x) = hr x - (hr x)^2 / 2 + (hr x)^3 / 6 - ...
    c.hr2h = (float)(0.5 * c.hr * c.hr);
    c.hr3s = (float)(c.hr * c.hr * c.hr / 6.0);
    return c;
}

struct CPArgs {
    float C11, C12, C44;
    double tau0, taus, h0;
    RMConsts rm;  // rm_consts(tau0, taus, h0), once per launch on the host
    float beta;
    float G;
    float e;
    float scale;
    float w_weight;
    uint64_t seed;
    const int32_t* grain;
    const float* quat;
    uint32_t t0;
    int32_t n_incr;
    int64_t P;
    const float* eps_total;  // sample-frame total strain [6][P] per point, or null (Taylor)
    float* eps_p;
    float* gamma;
    float* g;
    float* sigma;
    float* w;
    float* erho;
    int32_t* b;
};

__device__ __forceinline__ void stress(const CPArgs& a, const float ee[6], float s[6]) {
    const float tr = ee[0] + ee[1] + ee[2];
    const float d = a.C11 - a.C12;
    s[0] = d * ee[0] + a.C12 * tr;
    s[1] = d * ee[1] + a.C12 * tr;
    s[2] = d * ee[2] + a.C12 * tr;
    s[3] = 2.0f * a.C44 * ee[3];
    s[4] = 2.0f * a.C44 * ee[4];
    s[5] = 2.0f * a.C44 * ee[5];
}

// exp(-y) for y >= 0: Taylor series for small y, libm otherwise.
__device__ __forceinline__ double exp_neg(double y) {
    if (y < 0.02) {
        // truncation after y^6/720: below 1e-16 relative for y < 0.02
        return 1.0 - y * (1.0 - y * (0.5 - y * (1.0 / 6.0 - y * (1.0 / 24.0 - y * (1.0 / 120.0 - y * (1.0 / 720.0))))));
    }
    return exp(-y);
}

// Newton on the exact FP64 Voce residual at - x k - (taus - sat exp(-hr x)) from
// x; the step uses an FP32 reciprocal of the slope (a relative step error near
// 1e-7 leaves the iteration converging to the same FP64 root, tested on the
// exact residual).  Not inlined: the compiler would otherwise evaluate its
// first residual speculatively on every lane of the common (series) path.
__device__ __noinline__ double newton_slip(double at, double k, double taus, double tau0, double hr, double sat,
                                           double xs) {
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        const double ey = exp_neg(hr * xs);
        const double f = at - xs * k - (taus - sat * ey);
        if (fabs(f) < 1e-13 * tau0) break;
        const double fp = -k - sat * hr * ey;
        xs -= f * (double)(1.0f / (float)fp);
    }
    return xs;
}

// Slip x >= 0 of one system with resolved shear |tau| = at > g (slip resistance
// g, P:C:P = k): the root of f(x) = (at - g) - k x - sat (1 - exp(-hr x)),
// sat = taus - g, i.e. |tau| - x k = g(gamma + x) for the Voce law; x = (at - g) / k
// without hardening.  *g_new = g(gamma + x), from consistency at - k x.
//
// With y = hr x and q = sat hr / K (K = k + sat hr, q < 1), the exponential's
// cubic Taylor polynomial changes x by at most q y^3 / 24 relative; where that
// is below 4e-10 (q y^3 <= 1e-8, y <= 1e-2) x solves
// x = (a0 + c2 x^2 - c3 x^3) / K with a0 = at - g, c2 = sat hr^2 / 2,
// c3 = sat hr^3 / 6.  The leading term a0 / K is formed in FP64 (1 / K: an FP32
// reciprocal with one FP64 Newton correction, relative error near 1e-14); the
// correction x^2 (c2 - c3 x) / K is at most q y / 2 of x and each fixed-point
// step shrinks its error by a factor q y, so three steps in FP32 leave it below
// 1e-10.  Other slips take Newton on the exact FP64 residual.  The
// constants come as scalars so that the inlined code keeps the kernel's own
// registers and launch parameters.
__device__ __forceinline__ double return_map(float at_f, float g, double k, bool hard, double taus, double tau0,
                                             double hr, float taus32, float hr32, float hr2h, float hr3s,
                                             float* g_new) {
    const double g0 = g;
    const double at = at_f;
    double xs;
    if (!hard) {
        xs = (at - g0) / k;
    } else {
        const double sat = taus - g0;
        const double K = k + sat * hr;
        const float rKf = 1.0f / (float)K;
        double rK = (double)rKf;
        rK = rK * (2.0 - K * rK);
        xs = (at - g0) * rK;
        const float x1f = (float)xs;
        const float sr = (taus32 - g) * rKf;  // sat / K
        const float y = hr32 * x1f, q = hr32 * sr;
        if (y <= 1e-2f && y * y * y * q <= 1e-8f) {
            const float c2 = hr2h * sr, c3 = hr3s * sr;
            float d = 0.0f;
#pragma unroll
            for (int it = 0; it < 3; ++it) {
                const float xf = x1f + d;
                d = xf * xf * (c2 - c3 * xf);
            }
            xs += (double)d;
        } else {
            xs = newton_slip(at, k, taus, tau0, hr, sat, xs);
        }
    }
    *g_new = hard ? (float)(at - k * xs) : g;
    return xs;
}

// The return map as the plasticity kernel evaluates it, for testing.
__global__ void k_rm_eval(const float* __restrict__ at, const float* __restrict__ g, const double* __restrict__ k,
                          int64_t n, RMConsts c, double* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float gn;
    if (i < n)
        x[i] = return_map(at[i], g[i], k[i], c.hard, c.taus, c.tau0, c.hr, c.taus32, c.hr32, c.hr2h, c.hr3s, &gn);
}

template <bool STRAIN>
__global__ void __launch_bounds__(kT) k_cp(CPArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const float* qq = a.quat + 4 * (int64_t)a.grain[p];
    float qw = qq[0], qx = qq[1], qy = qq[2], qz = qq[3];
    const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    float R[3][3];
    R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); R[0][1] = 2.f * (qx * qy - qw * qz); R[0][2] = 2.f * (qx * qz + qw * qy);
    R[1][0] = 2.f * (qx * qy + qw * qz); R[1][1] = 1.f - 2.f * (qx * qx + qz * qz); R[1][2] = 2.f * (qy * qz - qw * qx);
    R[2][0] = 2.f * (qx * qz - qw * qy); R[2][1] = 2.f * (qy * qz + qw * qx); R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
    // unit-strain crystal-frame tensor U = R^T diag(1,-1/2,-1/2) R (Voigt order xx yy zz yz xz xy)
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
    float U[6];
#pragma unroll
    for (int v = 0; v < 6; ++v)
        U[v] = R[0][I[v]] * R[0][J[v]] - 0.5f * (R[1][I[v]] * R[1][J[v]] + R[2][I[v]] * R[2][J[v]]);
    // a point with its own total strain (elastic-equilibrium coupling): the
    // crystal-frame strain R^T eps R takes the place of t e U
    float Ut[6];
    if (STRAIN) {
        float es[3][3];
        const float e0 = a.eps_total[p], e1 = a.eps_total[a.P + p], e2 = a.eps_total[2 * a.P + p];
        const float e3 = a.eps_total[3 * a.P + p], e4 = a.eps_total[4 * a.P + p], e5 = a.eps_total[5 * a.P + p];
        es[0][0] = e0; es[1][1] = e1; es[2][2] = e2;
        es[1][2] = es[2][1] = e3; es[0][2] = es[2][0] = e4; es[0][1] = es[1][0] = e5;
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int l = 0; l < 3; ++l) acc += R[k][I[v]] * es[k][l] * R[l][J[v]];
            Ut[v] = acc;
        }
    }
    float ep[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) ep[v] = a.eps_p[(int64_t)v * a.P + p];
    float gam = a.gamma[p];
    float gres = a.g[p];
    // the return map's constants (two FP64 divisions among them) come from the
    // host: per thread they cost about as much FP64 work as the two increments
    const bool hard = a.rm.hard;
    const double hr = a.rm.hr;
    const float hr32 = a.rm.hr32, taus32 = a.rm.taus32;
    const float hr2h = a.rm.hr2h, hr3s = a.rm.hr3s;
    float ee[6], s[6];
    for (int32_t inc = 1; inc <= a.n_incr; ++inc) {
        const uint32_t t = a.t0 + (uint32_t)inc;
        const float et = (float)t * a.e;
#pragma unroll
        for (int v = 0; v < 6; ++v) ee[v] = (STRAIN ? Ut[v] : et * U[v]) - ep[v];
        stress(a, ee, s);
        float tau[12];
        int mask = 0;
#pragma unroll
        for (int al = 0; al < 12; ++al) {
            const float m0 = c_m[al][0], m1 = c_m[al][1], m2 = c_m[al][2];
            const float n0 = c_n[al][0], n1 = c_n[al][1], n2 = c_n[al][2];
            // m . s . n with s symmetric: s = [[s0,s5,s4],[s5,s1,s3],[s4,s3,s2]]
            tau[al] = m0 * (s[0] * n0 + s[5] * n1 + s[4] * n2) + m1 * (s[5] * n0 + s[1] * n1 + s[3] * n2) +
                      m2 * (s[4] * n0 + s[3] * n1 + s[2] * n2);
            if (fabsf(tau[al]) > gres) mask |= 1 << al;
        }
        if (!mask) continue;
        // candidate energies for the selection (Eq. (1)): the linearised
        // return map x_a = (|tau_a| - g)/(k_a + dg/dgamma), relative error
        // about 1e-6 against the converged one, in FP32
        const float hg = hard ? (taus32 - gres) * hr32 : 0.0f;
        float dE[12];
        float dEmin = 3.4e38f;
#pragma unroll
        for (int al = 0; al < 12; ++al) {
            dE[al] = 0.0f;
            if (!(mask >> al & 1)) continue;
            const float at = fabsf(tau[al]);
            const float k = c_kf[al];
            const float xx = (at - gres) / (k + hg);
            dE[al] = -xx * at + 0.5f * xx * xx * k;
            dEmin = fminf(dEmin, dE[al]);
        }
        float Z = 0.0f;
        float wgt[12];
#pragma unroll
        for (int al = 0; al < 12; ++al) {
            wgt[al] = (mask >> al & 1) ? expf(-a.beta * (dE[al] - dEmin)) : 0.0f;
            Z += wgt[al];
        }
        const uint4 u = draw(a.seed, (uint64_t)p, t, kTagMcp, 0);
        // first a with R < sum_{b <= a} w_b / Z, tested as R Z < sum_{b <= a} w_b
        // (no division per candidate; FP32 sums of at most 12 positive terms,
        // relative error near 1e-7, far inside the 1e-5 band around a decision
        // where the FP64 oracle and this kernel may legitimately differ)
        const float RZ = (float)u.x * (1.0f / 4294967296.0f) * Z;
        float cum = 0.0f;
        int pick = -1, last = -1;
        float tau_pick = 0.0f;
#pragma unroll
        for (int al = 0; al < 12; ++al) {
            if (!(mask >> al & 1)) continue;
            last = al;
            cum += wgt[al];
            if (pick < 0 && RZ < cum) { pick = al; tau_pick = tau[al]; }
        }
        if (pick < 0) {
            pick = last;
#pragma unroll
            for (int al = 0; al < 12; ++al)
                if (al == last) tau_pick = tau[al];
        }
        // the single-slip return map of the chosen system (FP64 where it matters)
        float g_next;
        const double xs = return_map(fabsf(tau_pick), gres, c_k[pick], hard, a.taus, a.tau0, hr, taus32, hr32, hr2h,
                                     hr3s, &g_next);
        const float sg = tau_pick > 0.f ? 1.f : -1.f;
        const float m0 = c_m[pick][0], m1 = c_m[pick][1], m2 = c_m[pick][2];
        const float n0 = c_n[pick][0], n1 = c_n[pick][1], n2 = c_n[pick][2];
        const float xf = (float)xs * sg;
        ep[0] += xf * m0 * n0;
        ep[1] += xf * m1 * n1;
        ep[2] += xf * m2 * n2;
        ep[3] += xf * 0.5f * (m1 * n2 + m2 * n1);
        ep[4] += xf * 0.5f * (m0 * n2 + m2 * n0);
        ep[5] += xf * 0.5f * (m0 * n1 + m1 * n0);
        gam += (float)xs;
        gres = g_next;  // g(gamma + x) = |tau| - k x at the solved slip
    }
#pragma unroll
    for (int v = 0; v < 6; ++v) a.eps_p[(int64_t)v * a.P + p] = ep[v];
    a.gamma[p] = gam;
    a.g[p] = gres;
    if (a.sigma || a.w || a.erho || a.b) {
        const uint32_t t = a.t0 + (uint32_t)a.n_incr;
        const float et = (float)t * a.e;
#pragma unroll
        for (int v = 0; v < 6; ++v) ee[v] = (STRAIN ? Ut[v] : et * U[v]) - ep[v];
        stress(a, ee, s);
        if (a.sigma)
#pragma unroll
            for (int v = 0; v < 6; ++v) a.sigma[(int64_t)v * a.P + p] = s[v];
        const float w = 0.5f * (s[0] * ee[0] + s[1] * ee[1] + s[2] * ee[2]) + (s[3] * ee[3] + s[4] * ee[4] + s[5] * ee[5]);
        const float er = 2.0f * gres * gres / a.G;
        if (a.w) a.w[p] = w;
        if (a.erho) a.erho[p] = er;
        if (a.b) {
            float v = rintf(256.0f * a.scale * (a.w_weight * w + er));
            v = fminf(fmaxf(v, -1048576.0f), 1048576.0f);
            a.b[p] = (int32_t)v;
        }
    }
}

__global__ void k_cp_reset(int64_t P, float* eps_p, float* gamma, float* g, float tau0) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
#pragma unroll
    for (int v = 0; v < 6; ++v) eps_p[(int64_t)v * P + p] = 0.0f;
    gamma[p] = 0.0f;
    g[p] = tau0;
}

// Constant tables depend on the moduli only; re-upload when they change.
double g_loaded[3] = {0.0, 0.0, 0.0};
int g_loaded_dev = -1;

int upload_tables(const hp_cp_params* prm) {
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    if (dev == g_loaded_dev && g_loaded[0] == prm->C11 && g_loaded[1] == prm->C12 && g_loaded[2] == prm->C44)
        return HP_OK;
    static const int N[12][3] = {{1, 1, 1},  {1, 1, 1},  {1, 1, 1},  {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
                                 {1, -1, 1}, {1, -1, 1}, {1, -1, 1}, {1, 1, -1}, {1, 1, -1}, {1, 1, -1}};
    static const int Mv[12][3] = {{0, 1, -1}, {-1, 0, 1}, {1, -1, 0}, {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
                                  {0, 1, 1},  {1, 0, -1}, {1, 1, 0},  {0, 1, 1},  {1, 0, 1}, {1, -1, 0}};
    float m[12][3], n[12][3];
    double k[12];
    const double sn = 1.0 / sqrt(3.0), sm = 1.0 / sqrt(2.0);
    for (int a = 0; a < 12; ++a) {
        double md[3], nd[3], P[3][3];
        for (int i = 0; i < 3; ++i) {
            md[i] = Mv[a][i] * sm;
            nd[i] = N[a][i] * sn;
            m[a][i] = (float)md[i];
            n[a][i] = (float)nd[i];
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) P[i][j] = 0.5 * (md[i] * nd[j] + nd[i] * md[j]);
        // P : C : P for cubic C
        const double tr = P[0][0] + P[1][1] + P[2][2];
        double v = 0.0;
        for (int i = 0; i < 3; ++i) v += P[i][i] * ((prm->C11 - prm->C12) * P[i][i] + prm->C12 * tr);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (i != j) v += P[i][j] * 2.0 * prm->C44 * P[i][j];
        k[a] = v;
    }
    HP_CUDA(cudaMemcpyToSymbol(c_m, m, sizeof m));
    HP_CUDA(cudaMemcpyToSymbol(c_n, n, sizeof n));
    HP_CUDA(cudaMemcpyToSymbol(c_k, k, sizeof k));
    float kf[12];
    for (int i = 0; i < 12; ++i) kf[i] = (float)k[i];
    HP_CUDA(cudaMemcpyToSymbol(c_kf, kf, sizeof kf));
    g_loaded[0] = prm->C11; g_loaded[1] = prm->C12; g_loaded[2] = prm->C44;
    g_loaded_dev = dev;
    return HP_OK;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_debug_return_map(const hp_cp_params* prm, const float* at, const float* g, const double* k,
                                   int64_t n, double* x, void* stream) {
    if (!prm || !at || !g || !k || !x || n < 0) return set_error(HP_ERR_ARG, "hp_debug_return_map: bad arguments");
    if (n == 0) return HP_OK;
    ::hp::count_launch();
    k_rm_eval<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(at, g, k, n, rm_consts(prm->tau0, prm->taus, prm->h0),
                                                                           x);
    HP_LAUNCH_CHECK("k_rm_eval");
    return HP_OK;
}

extern "C" int hp_cp_reset(const hp_cp_params* prm, hp_cp_state* st, void* stream) {
    if (!prm || !st || st->P < 1 || !st->eps_p || !st->gamma || !st->g)
        return set_error(HP_ERR_ARG, "hp_cp_reset: bad arguments");
    ::hp::count_launch();
    k_cp_reset<<<(unsigned)((st->P + 255) / 256), 256, 0, as_stream(stream)>>>(st->P, st->eps_p, st->gamma, st->g,
                                                                               (float)prm->tau0);
    HP_LAUNCH_CHECK("k_cp_reset");
    return HP_OK;
}

extern "C" int hp_cp_step(const hp_cp_params* prm, uint64_t seed, const int32_t* grain, const float* quat,
                          uint32_t t0, int32_t n_incr, hp_cp_state* st, float* sigma, float* w, float* erho,
                          int32_t* b, void* stream) {
    hp::Range r_("hp_cp_step");
    if (!prm || !st || !grain || !quat || n_incr < 0 || st->P < 1 || !st->eps_p || !st->gamma || !st->g)
        return set_error(HP_ERR_ARG, "hp_cp_step: bad arguments");
    if (!(prm->C11 > prm->C12) || !(prm->C44 > 0) || !(prm->tau0 > 0) || !(prm->G > 0))
        return set_error(HP_ERR_ARG, "hp_cp_step: bad material constants");
    int rc = upload_tables(prm);
    if (rc) return rc;
    CPArgs a;
    a.C11 = (float)prm->C11; a.C12 = (float)prm->C12; a.C44 = (float)prm->C44;
    a.tau0 = prm->tau0; a.taus = prm->taus; a.h0 = prm->h0;
    a.rm = rm_consts(prm->tau0, prm->taus, prm->h0);
    a.beta = (float)prm->beta; a.G = (float)prm->G; a.e = (float)prm->e_incr; a.scale = (float)prm->energy_scale;
    a.w_weight = (float)prm->w_weight;
    a.seed = seed; a.grain = grain; a.quat = quat; a.t0 = t0; a.n_incr = n_incr; a.P = st->P;
    a.eps_total = nullptr;
    a.eps_p = st->eps_p; a.gamma = st->gamma; a.g = st->g;
    a.sigma = sigma; a.w = w; a.erho = erho; a.b = b;
    ::hp::count_launch();
    k_cp<false><<<(unsigned)((st->P + kT - 1) / kT), kT, 0, as_stream(stream)>>>(a);
    HP_LAUNCH_CHECK("k_cp");
    return HP_OK;
}

extern "C" int hp_cp_step_strain(const hp_cp_params* prm, uint64_t seed, const int32_t* grain, const float* quat,
                                 uint32_t t, const float* eps_total, hp_cp_state* st, float* sigma, float* w,
                                 float* erho, int32_t* b, void* stream) {
    hp::Range r_("hp_cp_step_strain");
    if (!prm || !st || !grain || !quat || !eps_total || t < 1 || st->P < 1 || !st->eps_p || !st->gamma || !st->g)
        return set_error(HP_ERR_ARG, "hp_cp_step_strain: bad arguments");
    if (!(prm->C11 > prm->C12) || !(prm->C44 > 0) || !(prm->tau0 > 0) || !(prm->G > 0))
        return set_error(HP_ERR_ARG, "hp_cp_step_strain: bad material constants");
    int rc = upload_tables(prm);
    if (rc) return rc;
    CPArgs a;
    a.C11 = (float)prm->C11; a.C12 = (float)prm->C12; a.C44 = (float)prm->C44;
    a.tau0 = prm->tau0; a.taus = prm->taus; a.h0 = prm->h0;
    a.rm = rm_consts(prm->tau0, prm->taus, prm->h0);
    a.beta = (float)prm->beta; a.G = (float)prm->G; a.e = (float)prm->e_incr; a.scale = (float)prm->energy_scale;
    a.w_weight = (float)prm->w_weight;
    a.seed = seed; a.grain = grain; a.quat = quat; a.t0 = t - 1; a.n_incr = 1; a.P = st->P;
    a.eps_total = eps_total;
    a.eps_p = st->eps_p; a.gamma = st->gamma; a.g = st->g;
    a.sigma = sigma; a.w = w; a.erho = erho; a.b = b;
    ::hp::count_launch();
    k_cp<true><<<(unsigned)((st->P + kT - 1) / kT), kT, 0, as_stream(stream)>>>(a);
    HP_LAUNCH_CHECK("k_cp");
    return HP_OK;
}
