// Deterministic rate-independent multi-slip crystal plasticity: the comparator
// the Monte Carlo plasticity is checked against on a single nickel crystal
// (Sec. 2, Fig. 1: the constraint equations of the active slip systems are
// ill-conditioned and are solved with a singular value decomposition).  One
// thread per material point, FP64 throughout.
//
// Per load increment, crystal frame, 12 FCC {111}<110> systems with Schmid
// tensors P_a, cubic stiffness C, Voce hardening g(gamma) shared by all systems:
//   ee = eps - eps_p; trial stress C : ee; tau_a = P_a : C : ee; s_a = sign(tau_a);
//   active set {a : |tau_a| - g(gamma) > tol}, tol = 1e-12 tau0;
//   on the active set solve s_a tau_a - sum_b s_a s_b (P_a:C:P_b) x_b = g(gamma + sum x)
//   by Newton steps x += M^+ r, M = A + g'(gamma + sum x) 1 1^T, r the residual;
//   while a slip falls below -1e-6 tol drop the system of the most negative one
//   and solve again; then, while an inactive system's resolved shear exceeds g
//   by more than 10 tol, add the most over-stressed one with s_a the sign of its
//   current resolved shear and solve again (one change per pass: changing every
//   offending system at once cycles on increments far beyond yield); at most
//   50 passes, ties to the lowest system index; commit eps_p += sum x_a s_a P_a,
//   gamma += sum x_a.
//
// The pseudo-inverse.  Cubic C maps the deviatoric subspace to itself with
// eigenvalues D = (C11-C12, C11-C12, 2C44, 2C44, 2C44) on the orthonormal basis
// E1 = diag(1,-1,0)/sqrt2, E2 = diag(1,1,-2)/sqrt6, E3..E5 the sqrt2-normalised
// yz, xz, xy shears, and every P_a is deviatoric.  With c_a the coordinates of
// P_a on that basis, b_a = (s_a sqrt(D) c_a, sqrt(g')) is a 6-vector and
// M = B^T B for B = [b_a] (6 x n).  Hence M^+ r = B^T (B B^T)^+2 B r: the
// eigen-decomposition of the 6 x 6 matrix B B^T (cyclic Jacobi, in registers)
// gives the Moore-Penrose inverse of the n x n constraint matrix for any n <= 12,
// with the same spectrum and so the same relative cut-off (eigenvalues at or
// below 1e-10 of the largest are discarded).
#include <math.h>

#include "common.cuh"

namespace hp {
namespace {

constexpr int kDT = 64;

// Schmid tensors (Voigt xx yy zz yz xz xy, tensor components) and their
// deviatoric coordinates, filled once per device.
__constant__ double c_dP[12][6];
__constant__ double c_dc[12][5];

struct DetArgs {
    double C11, C12, C44;
    double tau0, taus, h0;
    double e;
    const int32_t* grain;
    const float* quat;
    uint32_t t0;
    int32_t n_incr;
    int64_t P;
    const float* eps_total;  // sample-frame total strain [6][P], or null (Taylor)
    double* eps_p;
    double* gamma;
    double* sigma;
    int32_t* n_active;
};

// upper-triangle storage of the symmetric 6 x 6 matrix
__host__ __device__ constexpr int tri(int i, int j) {
    return i <= j ? i * 6 - i * (i - 1) / 2 + (j - i) : j * 6 - j * (j - 1) / 2 + (i - j);
}

// Cyclic Jacobi eigen-decomposition of a symmetric 6 x 6 matrix: on return A
// holds the eigenvalues on its diagonal and V (row-major) the eigenvectors as
// columns.  Each rotation zeroes one off-diagonal pair (Golub and Van Loan,
// the symmetric Schur step); sweeps stop once the off-diagonal mass is below
// 1e-32 of the diagonal's.
__device__ __forceinline__ void jacobi6(double A[21], double V[36]) {
#pragma unroll
    for (int i = 0; i < 36; ++i) V[i] = (i % 7 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = 0.0, dg = 0.0;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            dg += A[tri(p, p)] * A[tri(p, p)];
#pragma unroll
            for (int q = p + 1; q < 6; ++q) off += A[tri(p, q)] * A[tri(p, q)];
        }
        if (off <= 1e-32 * dg) break;
#pragma unroll
        for (int p = 0; p < 5; ++p) {
#pragma unroll
            for (int q = p + 1; q < 6; ++q) {
                const double apq = A[tri(p, q)];
                if (apq != 0.0) {
                    const double th = (A[tri(q, q)] - A[tri(p, p)]) / (2.0 * apq);
                    double t;
                    if (fabs(th) > 1e150) {
                        t = 0.5 / th;
                    } else {
                        t = 1.0 / (fabs(th) + sqrt(1.0 + th * th));
                        if (th < 0.0) t = -t;
                    }
                    const double c = 1.0 / sqrt(1.0 + t * t);
                    const double s = t * c;
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        if (k == p || k == q) continue;
                        const double akp = A[tri(k, p)], akq = A[tri(k, q)];
                        A[tri(k, p)] = c * akp - s * akq;
                        A[tri(k, q)] = s * akp + c * akq;
                    }
                    A[tri(p, p)] -= t * apq;
                    A[tri(q, q)] += t * apq;
                    A[tri(p, q)] = 0.0;
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const double vkp = V[k * 6 + p], vkq = V[k * 6 + q];
                        V[k * 6 + p] = c * vkp - s * vkq;
                        V[k * 6 + q] = s * vkp + c * vkq;
                    }
                }
            }
        }
    }
}

struct Voce {
    double tau0, taus, h0;
    bool hard;
    __device__ double g(double gm) const {
        return hard ? taus - (taus - tau0) * exp(-h0 * gm / (taus - tau0)) : tau0;
    }
    __device__ double slope(double gm) const { return hard ? h0 * exp(-h0 * gm / (taus - tau0)) : 0.0; }
};

__device__ __forceinline__ void cubic_stress(const DetArgs& a, const double ee[6], double s[6]) {
    const double tr = ee[0] + ee[1] + ee[2];
    const double d = a.C11 - a.C12;
    s[0] = d * ee[0] + a.C12 * tr;
    s[1] = d * ee[1] + a.C12 * tr;
    s[2] = d * ee[2] + a.C12 * tr;
    s[3] = 2.0 * a.C44 * ee[3];
    s[4] = 2.0 * a.C44 * ee[4];
    s[5] = 2.0 * a.C44 * ee[5];
}

__device__ __forceinline__ double resolve(int a, const double s[6]) {
    return c_dP[a][0] * s[0] + c_dP[a][1] * s[1] + c_dP[a][2] * s[2] +
           2.0 * (c_dP[a][3] * s[3] + c_dP[a][4] * s[4] + c_dP[a][5] * s[5]);
}

// Newton on the active set `act` (bit a set = system a active; bit a of `neg`
// set = tau_a < 0).  x is zero outside the set on return.
__device__ void solve_active(uint32_t act, uint32_t neg, const double tau[12], double gam0, const double sD[5],
                             const Voce& vo, double tol, double x[12]) {
#pragma unroll
    for (int a = 0; a < 12; ++a) x[a] = 0.0;
    const double n = (double)__popc(act);
    for (int it = 0; it < 100; ++it) {
        double sx = 0.0;
#pragma unroll
        for (int a = 0; a < 12; ++a) sx += x[a];
        const double gg = vo.g(gam0 + sx);
        // w = sum_b s_b x_b sqrt(D) c_b: then (A x)_a = s_a sqrt(D) c_a . w
        double w[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            const double sb = ((neg >> b) & 1u) ? -x[b] : x[b];
#pragma unroll
            for (int k = 0; k < 5; ++k) w[k] += sb * sD[k] * c_dc[b][k];
        }
        double r[12], rmax = 0.0;
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            double ax = 0.0;
#pragma unroll
            for (int k = 0; k < 5; ++k) ax += sD[k] * c_dc[a][k] * w[k];
            if ((neg >> a) & 1u) ax = -ax;
            const double st = ((neg >> a) & 1u) ? -tau[a] : tau[a];
            r[a] = ((act >> a) & 1u) ? st - ax - gg : 0.0;
            rmax = fmax(rmax, fabs(r[a]));
        }
        if (rmax < tol) break;
        const double hs = vo.slope(gam0 + sx);
        const double rh = sqrt(hs);
        // G = B B^T and y = B r
        double G[21], y[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < 21; ++i) G[i] = 0.0;
        double rs = 0.0;
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            if (!((act >> a) & 1u)) continue;
            const double sa = ((neg >> a) & 1u) ? -1.0 : 1.0;
            double bv[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) bv[k] = sD[k] * c_dc[a][k];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
#pragma unroll
                for (int l = k; l < 5; ++l) G[tri(k, l)] += bv[k] * bv[l];
                G[tri(k, 5)] += sa * bv[k] * rh;
                y[k] += r[a] * sa * bv[k];
            }
            rs += r[a];
        }
        G[tri(5, 5)] = n * hs;
        y[5] = rh * rs;
        double V[36];
        jacobi6(G, V);
        double lmax = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) lmax = fmax(lmax, G[tri(k, k)]);
        const double cut = 1e-10 * lmax;
        double z[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < 6; ++i) v += V[i * 6 + k] * y[i];
            const double lam = G[tri(k, k)];
            z[k] = lam > cut ? v / (lam * lam) : 0.0;
        }
        double w6[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) v += V[i * 6 + k] * z[k];
            w6[i] = v;
        }
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            if (!((act >> a) & 1u)) continue;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 5; ++k) v += sD[k] * c_dc[a][k] * w6[k];
            if ((neg >> a) & 1u) v = -v;
            x[a] += v + rh * w6[5];
        }
    }
}

template <bool STRAIN>
__global__ void __launch_bounds__(kDT) k_det(DetArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const float* qq = a.quat + 4 * (int64_t)a.grain[p];
    double qw = qq[0], qx = qq[1], qy = qq[2], qz = qq[3];
    const double inv = 1.0 / sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    double R[3][3];
    R[0][0] = 1.0 - 2.0 * (qy * qy + qz * qz); R[0][1] = 2.0 * (qx * qy - qw * qz); R[0][2] = 2.0 * (qx * qz + qw * qy);
    R[1][0] = 2.0 * (qx * qy + qw * qz); R[1][1] = 1.0 - 2.0 * (qx * qx + qz * qz); R[1][2] = 2.0 * (qy * qz - qw * qx);
    R[2][0] = 2.0 * (qx * qz - qw * qy); R[2][1] = 2.0 * (qy * qz + qw * qx); R[2][2] = 1.0 - 2.0 * (qx * qx + qy * qy);
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
    // crystal-frame strain per unit load R^T diag(1,-1/2,-1/2) R, or R^T eps R
    double U[6];
    if (STRAIN) {
        double es[3][3];
        es[0][0] = a.eps_total[p]; es[1][1] = a.eps_total[a.P + p]; es[2][2] = a.eps_total[2 * a.P + p];
        es[1][2] = es[2][1] = a.eps_total[3 * a.P + p];
        es[0][2] = es[2][0] = a.eps_total[4 * a.P + p];
        es[0][1] = es[1][0] = a.eps_total[5 * a.P + p];
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int l = 0; l < 3; ++l) acc += R[k][I[v]] * es[k][l] * R[l][J[v]];
            U[v] = acc;
        }
    } else {
#pragma unroll
        for (int v = 0; v < 6; ++v)
            U[v] = R[0][I[v]] * R[0][J[v]] - 0.5 * (R[1][I[v]] * R[1][J[v]] + R[2][I[v]] * R[2][J[v]]);
    }
    double ep[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) ep[v] = a.eps_p[(int64_t)v * a.P + p];
    double gam = a.gamma[p];
    Voce vo;
    vo.tau0 = a.tau0; vo.taus = a.taus; vo.h0 = a.h0;
    vo.hard = a.taus - a.tau0 > 0.0 && a.h0 > 0.0;
    const double sD[5] = {sqrt(a.C11 - a.C12), sqrt(a.C11 - a.C12), sqrt(2.0 * a.C44), sqrt(2.0 * a.C44),
                          sqrt(2.0 * a.C44)};
    const double tol = 1e-12 * a.tau0;
    int32_t nact = 0;
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int32_t inc = 1; inc <= a.n_incr; ++inc) {
        const double et = STRAIN ? 1.0 : (double)(a.t0 + (uint32_t)inc) * a.e;
        double ee[6], str[6], tau[12];
#pragma unroll
        for (int v = 0; v < 6; ++v) ee[v] = et * U[v] - ep[v];
        cubic_stress(a, ee, str);
        const double g0 = vo.g(gam);
        uint32_t act = 0, neg = 0;
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            tau[b] = resolve(b, str);
            if (tau[b] < 0.0) neg |= 1u << b;
            if (fabs(tau[b]) - g0 > tol) act |= 1u << b;
        }
#pragma unroll
        for (int v = 0; v < 6; ++v) s[v] = str[v];
        nact = 0;
        if (!act) continue;
        bool settled = false;
        for (int pass = 0; pass < 50 && !settled; ++pass) {
            double x[12];
            solve_active(act, neg, tau, gam, sD, vo, tol, x);
            bool below = false;
            int worst = -1;
            double xmin = 0.0;
#pragma unroll
            for (int b = 0; b < 12; ++b) {
                if (!((act >> b) & 1u)) continue;
                if (x[b] < -tol * 1e-6) below = true;
                if (x[b] < xmin) {
                    xmin = x[b];
                    worst = b;
                }
            }
            if (below) {
                act &= ~(1u << worst);
                if (!act) settled = true;  // back to the elastic trial state
                continue;
            }
            double dep[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, sx = 0.0;
#pragma unroll
            for (int b = 0; b < 12; ++b) {
                const double xs = ((neg >> b) & 1u) ? -x[b] : x[b];
                sx += x[b];
#pragma unroll
                for (int v = 0; v < 6; ++v) dep[v] += xs * c_dP[b][v];
            }
            double ee2[6], s2[6];
#pragma unroll
            for (int v = 0; v < 6; ++v) ee2[v] = ee[v] - dep[v];
            cubic_stress(a, ee2, s2);
            const double g1 = vo.g(gam + sx);
            int add = -1;
            double over = 10.0 * tol, tadd = 0.0;
#pragma unroll
            for (int b = 0; b < 12; ++b) {
                if ((act >> b) & 1u) continue;
                const double tb = resolve(b, s2);
                if (fabs(tb) - g1 > over) {
                    over = fabs(tb) - g1;
                    add = b;
                    tadd = tb;
                }
            }
            if (add >= 0) {
                act |= 1u << add;
                if (tadd < 0.0)
                    neg |= 1u << add;
                else
                    neg &= ~(1u << add);
                continue;
            }
#pragma unroll
            for (int v = 0; v < 6; ++v) {
                ep[v] += dep[v];
                s[v] = s2[v];
            }
            gam += sx;
            nact = __popc(act);
            settled = true;
        }
        if (!settled) {
            nact = -1;
            break;
        }
    }
#pragma unroll
    for (int v = 0; v < 6; ++v) a.eps_p[(int64_t)v * a.P + p] = ep[v];
    a.gamma[p] = gam;
    if (a.sigma)
#pragma unroll
        for (int v = 0; v < 6; ++v) a.sigma[(int64_t)v * a.P + p] = s[v];
    if (a.n_active) a.n_active[p] = nact;
}

int g_det_dev = -1;

int upload_det_tables() {
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    if (dev == g_det_dev) return HP_OK;
    // the 12 FCC {111}<110> systems: plane normal and slip direction, three
    // directions per plane, planes (111), (-111), (1-11), (11-1)
    static const int Nn[12][3] = {{1, 1, 1},  {1, 1, 1},  {1, 1, 1},  {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
                                  {1, -1, 1}, {1, -1, 1}, {1, -1, 1}, {1, 1, -1}, {1, 1, -1}, {1, 1, -1}};
    static const int Md[12][3] = {{0, 1, -1}, {-1, 0, 1}, {1, -1, 0}, {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
                                  {0, 1, 1},  {1, 0, -1}, {1, 1, 0},  {0, 1, 1},  {1, 0, 1}, {1, -1, 0}};
    double P[12][6], c[12][5];
    int a = 0;
    for (int k = 0; k < 12; ++k) {
        if (Nn[k][0] * Md[k][0] + Nn[k][1] * Md[k][1] + Nn[k][2] * Md[k][2] != 0) continue;
        double n[3], m[3];
        for (int i = 0; i < 3; ++i) {
            n[i] = Nn[k][i] / sqrt(3.0);
            m[i] = Md[k][i] / sqrt(2.0);
        }
        double T[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) T[i][j] = 0.5 * (m[i] * n[j] + n[i] * m[j]);
        P[a][0] = T[0][0]; P[a][1] = T[1][1]; P[a][2] = T[2][2];
        P[a][3] = T[1][2]; P[a][4] = T[0][2]; P[a][5] = T[0][1];
        c[a][0] = (T[0][0] - T[1][1]) / sqrt(2.0);
        c[a][1] = (T[0][0] + T[1][1] - 2.0 * T[2][2]) / sqrt(6.0);
        c[a][2] = sqrt(2.0) * T[1][2];
        c[a][3] = sqrt(2.0) * T[0][2];
        c[a][4] = sqrt(2.0) * T[0][1];
        ++a;
    }
    if (a != 12) return set_error(HP_ERR_STATE, "upload_det_tables: slip-system table");
    HP_CUDA(cudaMemcpyToSymbol(c_dP, P, sizeof P));
    HP_CUDA(cudaMemcpyToSymbol(c_dc, c, sizeof c));
    g_det_dev = dev;
    return HP_OK;
}

int det_launch(const hp_cp_params* prm, const int32_t* grain, const float* quat, uint32_t t0, int32_t n_incr,
               const float* eps_total, hp_det_state* st, double* sigma, int32_t* n_active, void* stream,
               const char* who) {
    if (!prm || !st || !grain || !quat || n_incr < 0 || st->P < 1 || !st->eps_p || !st->gamma)
        return set_error(HP_ERR_ARG, std::string(who) + ": bad arguments");
    if (!(prm->C11 > prm->C12) || !(prm->C44 > 0) || !(prm->tau0 > 0))
        return set_error(HP_ERR_ARG, std::string(who) + ": bad material constants");
    int rc = upload_det_tables();
    if (rc) return rc;
    DetArgs a;
    a.C11 = prm->C11; a.C12 = prm->C12; a.C44 = prm->C44;
    a.tau0 = prm->tau0; a.taus = prm->taus; a.h0 = prm->h0; a.e = prm->e_incr;
    a.grain = grain; a.quat = quat; a.t0 = t0; a.n_incr = n_incr; a.P = st->P;
    a.eps_total = eps_total;
    a.eps_p = st->eps_p; a.gamma = st->gamma; a.sigma = sigma; a.n_active = n_active;
    ::hp::count_launch();
    const unsigned grid = (unsigned)((st->P + kDT - 1) / kDT);
    if (eps_total)
        k_det<true><<<grid, kDT, 0, as_stream(stream)>>>(a);
    else
        k_det<false><<<grid, kDT, 0, as_stream(stream)>>>(a);
    HP_LAUNCH_CHECK("k_det");
    return HP_OK;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_det_reset(hp_det_state* st, void* stream) {
    if (!st || st->P < 1 || !st->eps_p || !st->gamma) return set_error(HP_ERR_ARG, "hp_det_reset: bad arguments");
    HP_CUDA(cudaMemsetAsync(st->eps_p, 0, sizeof(double) * 6 * (size_t)st->P, as_stream(stream)));
    HP_CUDA(cudaMemsetAsync(st->gamma, 0, sizeof(double) * (size_t)st->P, as_stream(stream)));
    return HP_OK;
}

extern "C" int hp_det_step(const hp_cp_params* prm, const int32_t* grain, const float* quat, uint32_t t0,
                           int32_t n_incr, hp_det_state* st, double* sigma, int32_t* n_active, void* stream) {
    hp::Range r_("hp_det_step");
    return det_launch(prm, grain, quat, t0, n_incr, nullptr, st, sigma, n_active, stream, "hp_det_step");
}

extern "C" int hp_det_step_strain(const hp_cp_params* prm, const int32_t* grain, const float* quat,
                                  const float* eps_total, hp_det_state* st, double* sigma, int32_t* n_active,
                                  void* stream) {
    hp::Range r_("hp_det_step_strain");
    if (!eps_total) return set_error(HP_ERR_ARG, "hp_det_step_strain: bad arguments");
    return det_launch(prm, grain, quat, 0, 1, eps_total, st, sigma, n_active, stream, "hp_det_step_strain");
}
