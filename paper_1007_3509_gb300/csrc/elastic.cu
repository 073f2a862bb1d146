// Periodic elastic equilibrium of the cubic polycrystal on the lattice grid
// (Sec. 5: the plasticity is coupled to a deformation solver and each load
// increment is iterated to quasi-static equilibrium; here the solver is the
// Lippmann-Schwinger fixed point of Moulinec and Suquet on the voxel grid, one
// material point per voxel).  FP32 throughout.
//
//   sigma(x) = C(x) : (eps(x) - eps_p(x))        evaluated in the crystal frame
//   tau      = sigma - C0 : eps                   C0 isotropic (lambda0, mu0)
//   eps^hat  = -Gamma0 : tau^hat,  xi != 0        Green operator of C0
//   eps^hat(0) = E; zero on the Nyquist planes of even axes
//   Gamma0 : tau = (n (x) a + a (x) n)/(2 mu0) - kappa (n . a) n (x) n,
//   n = xi/|xi|, a = tau n, kappa = (lambda0 + mu0)/(mu0 (lambda0 + 2 mu0))
//
// The six strain components live in six complex fields [6][N] (float2) for the
// transforms.  The 3D transforms are three passes of a radix-2 FFT over lines of
// one axis: a block takes W lines of length n into shared memory (adjacent lines
// side by side, so the global accesses are coalesced along x for every axis),
// stores them bit-reversed, runs the log2 n butterfly stages in place and writes
// them back in natural order.  The twiddles exp(-+2 pi i k / n), k < n/2, are
// computed once per block (sincospif) into a shared table.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace hp {
namespace {

constexpr int kET = 256;
constexpr int kTile = 4096;  // complex elements per FFT block (32 KB)

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// lines of axis `axis` of field-major data [6][nz][ny][nx]: line L, element i
struct Lines {
    int nx, ny, nz, axis, n, logn, W;
    int64_t N;
    __device__ __forceinline__ int64_t base(int64_t L) const {
        if (axis == 0) return L * nx;
        const int64_t x = L % nx, r = L / nx;
        if (axis == 1) {  // r = z + nz f
            const int64_t z = r % nz, f = r / nz;
            return f * N + z * (int64_t)nx * ny + x;
        }
        const int64_t y = r % ny, f = r / ny;  // r = y + ny f
        return f * N + y * (int64_t)nx + x;
    }
    __device__ __forceinline__ int64_t stride() const {
        return axis == 0 ? 1 : (axis == 1 ? (int64_t)nx : (int64_t)nx * ny);
    }
};

__global__ void __launch_bounds__(kET) k_fft(float2* __restrict__ data, Lines g, float sign) {
    __shared__ float2 sm[kTile];
    __shared__ float2 tw[512];  // exp(sign 2 pi i k / n), k < n/2
    const int n = g.n, W = g.W;
    for (int k = threadIdx.x; k < (n >> 1); k += kET) {
        float s, c;
        sincospif(2.0f * (float)k / (float)n, &s, &c);
        tw[k] = make_float2(c, sign * s);
    }
    const int64_t L0 = (int64_t)blockIdx.x * W;
    const int64_t st = g.stride();
    // load: for axis 0 consecutive threads walk a line, otherwise across lines
    for (int t = threadIdx.x; t < W * n; t += kET) {
        int w, i;
        if (g.axis == 0) { w = t / n; i = t - w * n; } else { i = t / W; w = t - i * W; }
        const int64_t a = (g.axis == 0 ? g.base(L0 + w) : g.base(L0) + w) + (int64_t)i * st;
        sm[w * n + bitrev((unsigned)i, g.logn)] = data[a];
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        for (int b = threadIdx.x; b < W * (n >> 1); b += kET) {
            const int w = b / (n >> 1), bb = b - w * (n >> 1);
            const int grp = bb / half, j = bb - grp * half;
            const int i0 = w * n + grp * len + j, i1 = i0 + half;
            const float2 tj = tw[j * (n / len)];  // exp(sign 2 pi i j / len)
            const float wr = tj.x, wi = tj.y;
            const float2 u = sm[i0], v = sm[i1];
            const float vr = v.x * wr - v.y * wi, vi = v.x * wi + v.y * wr;
            sm[i0] = make_float2(u.x + vr, u.y + vi);
            sm[i1] = make_float2(u.x - vr, u.y - vi);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < W * n; t += kET) {
        int w, i;
        if (g.axis == 0) { w = t / n; i = t - w * n; } else { i = t / W; w = t - i * W; }
        const int64_t a = (g.axis == 0 ? g.base(L0 + w) : g.base(L0) + w) + (int64_t)i * st;
        data[a] = sm[w * n + i];
    }
}

struct ElArgs {
    int nx, ny, nz;
    int64_t N;
    float C11, C12, C44, lam0, mu0;
    const int32_t* grain;
    const float* quat;
    const float* eps_p;  // crystal frame, [6][N], or null
    float E[6];
};

__device__ __forceinline__ void rot_of(const float* qq, float R[3][3]) {
    float w = qq[0], x = qq[1], y = qq[2], z = qq[3];
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void sym(const float v[6], float t[3][3]) {
    t[0][0] = v[0]; t[1][1] = v[1]; t[2][2] = v[2];
    t[1][2] = t[2][1] = v[3]; t[0][2] = t[2][0] = v[4]; t[0][1] = t[1][0] = v[5];
}

// sample-frame stress of voxel i at sample-frame strain e (Voigt)
__device__ __forceinline__ void voxel_stress(const ElArgs& a, int64_t i, const float e[6], float s_out[6]) {
    float R[3][3], es[3][3], ec[3][3], sc[3][3], tmp[3][3];
    rot_of(a.quat + 4 * (int64_t)a.grain[i], R);
    sym(e, es);
    // ec = R^T es R
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) tmp[p][q] = es[p][0] * R[0][q] + es[p][1] * R[1][q] + es[p][2] * R[2][q];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) ec[p][q] = R[0][p] * tmp[0][q] + R[1][p] * tmp[1][q] + R[2][p] * tmp[2][q];
    if (a.eps_p) {
        float ep[6], et[3][3];
#pragma unroll
        for (int c = 0; c < 6; ++c) ep[c] = a.eps_p[(int64_t)c * a.N + i];
        sym(ep, et);
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) ec[p][q] -= et[p][q];
    }
    const float tr = ec[0][0] + ec[1][1] + ec[2][2];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) sc[p][q] = 2.f * a.C44 * ec[p][q];
#pragma unroll
    for (int p = 0; p < 3; ++p) sc[p][p] = (a.C11 - a.C12) * ec[p][p] + a.C12 * tr;
    // s = R sc R^T
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) tmp[p][q] = sc[p][0] * R[q][0] + sc[p][1] * R[q][1] + sc[p][2] * R[q][2];
    float s[3][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) s[p][q] = R[p][0] * tmp[0][q] + R[p][1] * tmp[1][q] + R[p][2] * tmp[2][q];
    s_out[0] = s[0][0]; s_out[1] = s[1][1]; s_out[2] = s[2][2];
    s_out[3] = s[1][2]; s_out[4] = s[0][2]; s_out[5] = s[0][1];
}

// tau = sigma - C0 : eps into the complex fields (imaginary part 0)
__global__ void k_el_polar(ElArgs a, const float* __restrict__ eps, float2* __restrict__ W) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    float e[6], s[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps[(int64_t)c * a.N + i];
    voxel_stress(a, i, e, s);
    const float tr = e[0] + e[1] + e[2];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float t = s[c] - 2.f * a.mu0 * e[c] - (c < 3 ? a.lam0 * tr : 0.f);
        W[(int64_t)c * a.N + i] = make_float2(t, 0.f);
    }
}

// eps^hat = -Gamma0 : tau^hat per frequency (E N at xi = 0, zero on Nyquist planes)
__global__ void k_el_green(ElArgs a, float2* __restrict__ W) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.N) return;
    const int x = (int)(k % a.nx);
    const int64_t r = k / a.nx;
    const int y = (int)(r % a.ny), z = (int)(r / a.ny);
    const int kx = x < a.nx / 2 ? x : x - a.nx, ky = y < a.ny / 2 ? y : y - a.ny, kz = z < a.nz / 2 ? z : z - a.nz;
    const bool nyq = (a.nx % 2 == 0 && kx == -a.nx / 2) || (a.ny % 2 == 0 && ky == -a.ny / 2) ||
                     (a.nz % 2 == 0 && kz == -a.nz / 2);
    float2 out[6];
    if (k == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) out[c] = make_float2(a.E[c] * (float)a.N, 0.f);
    } else if (nyq) {
#pragma unroll
        for (int c = 0; c < 6; ++c) out[c] = make_float2(0.f, 0.f);
    } else {
        const float inv = rsqrtf((float)kx * kx + (float)ky * ky + (float)kz * kz);
        const float n[3] = {kx * inv, ky * inv, kz * inv};
        float2 t[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = W[(int64_t)c * a.N + k];
        // a = tau n (complex), tau symmetric: rows (xx xy xz), (xy yy yz), (xz yz zz)
        const float2 a0 = make_float2(t[0].x * n[0] + t[5].x * n[1] + t[4].x * n[2], t[0].y * n[0] + t[5].y * n[1] + t[4].y * n[2]);
        const float2 a1 = make_float2(t[5].x * n[0] + t[1].x * n[1] + t[3].x * n[2], t[5].y * n[0] + t[1].y * n[1] + t[3].y * n[2]);
        const float2 a2 = make_float2(t[4].x * n[0] + t[3].x * n[1] + t[2].x * n[2], t[4].y * n[0] + t[3].y * n[1] + t[2].y * n[2]);
        const float2 cc = make_float2(n[0] * a0.x + n[1] * a1.x + n[2] * a2.x, n[0] * a0.y + n[1] * a1.y + n[2] * a2.y);
        const float h = 0.5f / a.mu0, kap = (a.lam0 + a.mu0) / (a.mu0 * (a.lam0 + 2.f * a.mu0));
        const float2 av[3] = {a0, a1, a2};
        const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int p = I[c], q = J[c];
            out[c].x = -(h * (n[p] * av[q].x + av[p].x * n[q]) - kap * cc.x * n[p] * n[q]);
            out[c].y = -(h * (n[p] * av[q].y + av[p].y * n[q]) - kap * cc.y * n[p] * n[q]);
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) W[(int64_t)c * a.N + k] = out[c];
}

// eps <- Re(W) / N; the largest change over all components into *change (as
// the bits of a non-negative float, atomicMax on the integer view)
__global__ void k_el_update(ElArgs a, const float2* __restrict__ W, float* __restrict__ eps, unsigned* change) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < a.N) {
        const float invN = 1.0f / (float)a.N;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float v = W[(int64_t)c * a.N + i].x * invN;
            m = fmaxf(m, fabsf(v - eps[(int64_t)c * a.N + i]));
            eps[(int64_t)c * a.N + i] = v;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(change, __float_as_uint(m));
}

__global__ void k_el_fill(ElArgs a, float* __restrict__ eps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
#pragma unroll
    for (int c = 0; c < 6; ++c) eps[(int64_t)c * a.N + i] = a.E[c];
}

__global__ void k_el_stress(ElArgs a, const float* __restrict__ eps, float* __restrict__ sig) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    float e[6], s[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps[(int64_t)c * a.N + i];
    voxel_stress(a, i, e, s);
#pragma unroll
    for (int c = 0; c < 6; ++c) sig[(int64_t)c * a.N + i] = s[c];
}

int log2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

int fft3(float2* W, int nx, int ny, int nz, int64_t N, float sign, cudaStream_t s) {
    const int dims[3] = {nx, ny, nz};
    for (int axis = 0; axis < 3; ++axis) {
        const int n = dims[axis];
        if (n == 1) continue;
        Lines g;
        g.nx = nx; g.ny = ny; g.nz = nz; g.axis = axis; g.n = n; g.logn = log2_exact(n); g.N = N;
        // lines per block: a power of two that divides the line count (6 ny nz
        // lines along x; along y and z adjacent lines share (field, z or y) only
        // within one row of x)
        int W_ = kTile / n;
        if (W_ < 1) W_ = 1;
        if (axis == 0 && (int64_t)W_ > 2 * (int64_t)ny * nz) W_ = 2 * ny * nz;
        if (axis != 0 && W_ > nx) W_ = nx;
        if (axis != 0 && W_ > 32) W_ = 32;
        g.W = W_;
        const int64_t lines = 6 * N / n;
        count_launch();
        k_fft<<<(unsigned)(lines / W_), kET, 0, s>>>(W, g, sign);
    }
    HP_LAUNCH_CHECK("k_fft");
    return HP_OK;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_elastic_solve(const hp_cp_params* prm, const hp_elastic_params* ep, const int32_t* grain,
                                const float* quat, const float* eps_p, const double E[6], float* eps, float* sigma,
                                int32_t* iters, double* change_out, void* stream) {
    hp::Range r_("hp_elastic_solve");
    if (!prm || !ep || !grain || !quat || !E || !eps) return set_error(HP_ERR_ARG, "hp_elastic_solve: bad arguments");
    for (int d = 0; d < 3; ++d)
        if (ep->n[d] < 1 || ep->n[d] > 1024 || log2_exact(ep->n[d]) < 0)
            return set_error(HP_ERR_ARG, "hp_elastic_solve: grid edges must be powers of two up to 1024");
    if (!(ep->tol > 0.0) || ep->max_iter < 1) return set_error(HP_ERR_ARG, "hp_elastic_solve: bad tolerance");
    cudaStream_t s = as_stream(stream);
    ElArgs a;
    a.nx = ep->n[0]; a.ny = ep->n[1]; a.nz = ep->n[2];
    a.N = (int64_t)a.nx * a.ny * a.nz;
    a.C11 = (float)prm->C11; a.C12 = (float)prm->C12; a.C44 = (float)prm->C44;
    // isotropic reference: the mean of the two shear moduli, the crystal's bulk modulus
    const double mu0 = 0.5 * (prm->C44 + 0.5 * (prm->C11 - prm->C12));
    const double K = (prm->C11 + 2.0 * prm->C12) / 3.0;
    a.mu0 = (float)mu0;
    a.lam0 = (float)(K - 2.0 * mu0 / 3.0);
    a.grain = grain; a.quat = quat; a.eps_p = eps_p;
    double emax = 0.0;
    for (int c = 0; c < 6; ++c) {
        a.E[c] = (float)E[c];
        emax = fabs(E[c]) > emax ? fabs(E[c]) : emax;
    }
    if (!(emax > 0.0)) return set_error(HP_ERR_ARG, "hp_elastic_solve: zero mean strain");
    float2* W = nullptr;
    unsigned* d_change = nullptr;
    if (cudaMallocAsync((void**)&W, sizeof(float2) * 6 * (size_t)a.N, s) != cudaSuccess ||
        cudaMallocAsync((void**)&d_change, sizeof(unsigned), s) != cudaSuccess) {
        cudaFreeAsync(W, s);
        cudaFreeAsync(d_change, s);
        return set_error(HP_ERR_OOM, "hp_elastic_solve: work buffer allocation failed");
    }
    const unsigned nb = (unsigned)((a.N + kET - 1) / kET);
    int rc = HP_OK;
    if (ep->start_from_mean) {
        count_launch();
        k_el_fill<<<nb, kET, 0, s>>>(a, eps);
    }
    int it = 0;
    double ch = INFINITY;
    for (it = 1; it <= ep->max_iter && rc == HP_OK; ++it) {
        count_launch();
        k_el_polar<<<nb, kET, 0, s>>>(a, eps, W);
        if ((rc = fft3(W, a.nx, a.ny, a.nz, a.N, -1.0f, s))) break;
        count_launch();
        k_el_green<<<nb, kET, 0, s>>>(a, W);
        if ((rc = fft3(W, a.nx, a.ny, a.nz, a.N, 1.0f, s))) break;
        cudaMemsetAsync(d_change, 0, sizeof(unsigned), s);
        count_launch();
        k_el_update<<<nb, kET, 0, s>>>(a, W, eps, d_change);
        unsigned hc = 0;
        cudaError_t e = cudaMemcpyAsync(&hc, d_change, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_error(e, "hp_elastic_solve"); break; }
        float hf;
        memcpy(&hf, &hc, sizeof hf);
        ch = (double)hf / emax;
        if (ch < ep->tol) break;
    }
    if (it > ep->max_iter) it = ep->max_iter;
    if (rc == HP_OK && sigma) {
        count_launch();
        k_el_stress<<<nb, kET, 0, s>>>(a, eps, sigma);
    }
    if (rc == HP_OK) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error(e, "hp_elastic_solve");
    }
    cudaFreeAsync(W, s);
    cudaFreeAsync(d_change, s);
    if (iters) *iters = it;
    if (change_out) *change_out = ch;
    return rc;
}
