// Per-grain driving field in closed form, grain statistics and texture.
//
// Field (Sec. 5, uniaxial load along sample x): loading axis in the crystal
// frame d = R(q)^T e_x; directional modulus of a cubic crystal
//   1/E(d) = S11 - 2 (S11 - S12 - S44/2)(d1^2 d2^2 + d2^2 d3^2 + d3^2 d1^2),
//   S11 = (C11+C12)/((C11-C12)(C11+2C12)), S12 = -C12/((C11-C12)(C11+2C12)),
//   S44 = 1/C44;
// elastic energy density w = sigma^2/(2E); max FCC {111}<110> Schmid factor
// m_max = max_a |(d.n_a)(d.m_a)|; e = scale (w + k m_max) [J];
// b = round-half-even(256 e), clamped to +-2^20.  One thread per grain, FP64.
//
// Statistics (Sec. 4 average grain size, Sec. 5 texture): per-grain site
// counts, number of grains alive, per-grain texture bins and the
// area-weighted histogram.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace hp {
namespace {

constexpr int kT = 256;

// FCC slip systems: plane normals and slip directions (unnormalised).
__constant__ int8_t c_fcc_n[12][3] = {{1, 1, 1},  {1, 1, 1},  {1, 1, 1},  {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
                                      {1, -1, 1}, {1, -1, 1}, {1, -1, 1}, {1, 1, -1}, {1, 1, -1}, {1, 1, -1}};
__constant__ int8_t c_fcc_m[12][3] = {{0, 1, -1}, {-1, 0, 1}, {1, -1, 0}, {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
                                      {0, 1, 1},  {1, 0, -1}, {1, 1, 0},  {0, 1, 1},  {1, 0, 1}, {1, -1, 0}};

__device__ void axis_from_quat(const float* qf, double d[3]) {
    const double w0 = qf[0], x0 = qf[1], y0 = qf[2], z0 = qf[3];
    const double n = sqrt(w0 * w0 + x0 * x0 + y0 * y0 + z0 * z0);
    const double w = w0 / n, x = x0 / n, y = y0 / n, z = z0 / n;
    // first row of the crystal-to-sample rotation matrix
    d[0] = 1.0 - 2.0 * (y * y + z * z);
    d[1] = 2.0 * (x * y - w * z);
    d[2] = 2.0 * (x * z + w * y);
}

__device__ double max_schmid(const double d_in[3]) {
    const double nn = sqrt(d_in[0] * d_in[0] + d_in[1] * d_in[1] + d_in[2] * d_in[2]);
    const double d0 = d_in[0] / nn, d1 = d_in[1] / nn, d2 = d_in[2] / nn;
    const double sn = 1.0 / sqrt(3.0), sm = 1.0 / sqrt(2.0);
    double best = 0.0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        const double dn = (d0 * c_fcc_n[a][0] + d1 * c_fcc_n[a][1] + d2 * c_fcc_n[a][2]) * sn;
        const double dm = (d0 * c_fcc_m[a][0] + d1 * c_fcc_m[a][1] + d2 * c_fcc_m[a][2]) * sm;
        best = fmax(best, fabs(dn * dm));
    }
    return best;
}

struct FieldArgs {
    const float* quat;
    int32_t G;
    double S11, S12, S44, sigma, k, scale;
    int32_t* b;
    float* w;
    float* mmax;
};

__global__ void k_grain_field(FieldArgs a) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.G) return;
    double d[3];
    axis_from_quat(a.quat + 4 * g, d);
    const double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double l = d[0] / nn, m = d[1] / nn, n = d[2] / nn;
    const double inv_e = a.S11 - 2.0 * (a.S11 - a.S12 - 0.5 * a.S44) * (l * l * m * m + m * m * n * n + n * n * l * l);
    const double w = 0.5 * a.sigma * a.sigma * inv_e;
    const double mm = max_schmid(d);
    const double e = a.scale * (w + a.k * mm);
    double v = rint(256.0 * e);
    v = fmin(fmax(v, -1048576.0), 1048576.0);
    a.b[g] = (int32_t)v;
    if (a.w) a.w[g] = (float)w;
    if (a.mmax) a.mmax[g] = (float)mm;
}

// Per-grain counts: each thread scans a run of consecutive sites and adds the
// length of each run of equal ids with one atomic.
constexpr int kSeg = 32;

__global__ void __launch_bounds__(kT) k_counts(const int32_t* __restrict__ q, int64_t N, int32_t G,
                                               unsigned long long* counts, int32_t* bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = t * kSeg;
    if (b >= N) return;
    const int64_t e = b + kSeg < N ? b + kSeg : N;
    int32_t cur = q[b];
    unsigned long long run = 0;
    for (int64_t i = b; i < e; ++i) {
        const int32_t v = q[i];
        if (v != cur) {
            if ((uint32_t)cur < (uint32_t)G) atomicAdd(counts + cur, run); else atomicAdd(bad, 1);
            cur = v;
            run = 0;
        }
        ++run;
    }
    if ((uint32_t)cur < (uint32_t)G) atomicAdd(counts + cur, run); else atomicAdd(bad, 1);
}

__global__ void k_alive(const unsigned long long* counts, int32_t G, int32_t* alive) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = g < G && counts[g] > 0;
    const int s = __syncthreads_count(v);
    if (threadIdx.x == 0 && s) atomicAdd(alive, s);
}

__global__ void k_bins(int32_t G, int32_t kind, const float* orient, int32_t* bins) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const double pi = 3.14159265358979323846;
    if (kind == HP_ORIENT_ANGLE || kind == HP_ORIENT_ZROT) {
        const double t = kind == HP_ORIENT_ANGLE ? (double)orient[g]
                                                 : 2.0 * atan2((double)orient[4 * g + 3], (double)orient[4 * g]);
        const double deg = t * (180.0 / pi);
        int b = (int)floor(deg);
        bins[g] = b < 0 ? 0 : (b > 89 ? 89 : b);
        return;
    }
    double d[3];
    axis_from_quat(orient + 4 * g, d);
    const double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double a0 = fabs(d[0] / nn), a1 = fabs(d[1] / nn), a2 = fabs(d[2] / nn);
    const double ad[3] = {a0, a1, a2};
    const double v = max_schmid(ad) / 0.5 * 20.0;
    int b = (int)floor(v);
    bins[2 * g] = b < 0 ? 0 : (b > 19 ? 19 : b);
    const double c15 = cos(15.0 * pi / 180.0);
    const double c100 = fmax(a0, fmax(a1, a2));
    const double c110 = fmax(a0 + a1, fmax(a1 + a2, a0 + a2)) / sqrt(2.0);
    const double c111 = (a0 + a1 + a2) / sqrt(3.0);
    int fam = 0;
    if (c100 > c15) fam = 1;
    else if (c110 > c15) fam = 2;
    else if (c111 > c15) fam = 3;
    bins[2 * g + 1] = 20 + fam;
}

__global__ void k_hist(int32_t G, int32_t kind, const int32_t* bins, const unsigned long long* counts,
                       unsigned long long* hist) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const unsigned long long c = counts[g];
    if (!c) return;
    if (kind != HP_ORIENT_SO3) {
        atomicAdd(hist + bins[g], c);
    } else {
        atomicAdd(hist + bins[2 * g], c);
        atomicAdd(hist + bins[2 * g + 1], c);
    }
}

// Orientation-dependent Gaussian bulk energy of Eq. (9): the grain's angle
// selects orientation n = floor(angle in degrees) + 1 (1..90) and
// b(n) = (32 pi)^(-1/2) exp(-(n - 46)^2 / (2 * 46^2)) [J], quantised.
__global__ void k_gaussian_field(int32_t G, const float* angle, double scale, int32_t* b) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const double pi = 3.14159265358979323846;
    int bin = (int)floor((double)angle[g] * (180.0 / pi));
    bin = bin < 0 ? 0 : (bin > 89 ? 89 : bin);
    const double n = bin + 1.0;
    const double e = scale * exp(-(n - 46.0) * (n - 46.0) / (2.0 * 46.0 * 46.0)) / sqrt(32.0 * pi);
    b[g] = (int32_t)rint(256.0 * e);
}

// Sum over a block of a signed 64-bit value, added to *sum with one atomic
// (two's complement: the unsigned atomic adds signed values exactly).
__device__ __forceinline__ void block_add(long long v, unsigned long long* sum) {
    __shared__ long long part[kT / 32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < kT / 32; ++w) t += part[w];
        if (t) atomicAdd(sum, (unsigned long long)t);
    }
}

// Volume-weighted field sum, per-grain table: sum_g counts[g] table[g].
__global__ void __launch_bounds__(kT) k_field_sum_grain(const unsigned long long* counts, const int32_t* table,
                                                        int32_t G, unsigned long long* sum) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    block_add(g < G ? (long long)counts[g] * (long long)table[g] : 0ll, sum);
}

// Per-point table: sum_i table[mp_i] (index clamped into the table).
__global__ void __launch_bounds__(kT) k_field_sum_point(const int32_t* __restrict__ mp, const int32_t* __restrict__ table,
                                                        uint32_t n_table, int64_t N, unsigned long long* sum) {
    long long v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)mp[i];
        v += table[u < n_table ? u : n_table - 1];
    }
    block_add(v, sum);
}

// angle [rad] of HP_ORIENT_ANGLE (or the rotation angle of HP_ORIENT_ZROT) to
// integer units: floor(degrees * unit_per_degree) mod period
__global__ void k_angle_units(int32_t G, int32_t kind, const float* orient, int32_t unit, int32_t period, int32_t* out) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const double pi = 3.14159265358979323846;
    const double t = kind == HP_ORIENT_ANGLE ? (double)orient[g]
                                             : 2.0 * atan2((double)orient[4 * g + 3], (double)orient[4 * g]);
    int64_t v = (int64_t)floor(t * (180.0 / pi) * (double)unit) % period;
    out[g] = (int32_t)(v < 0 ? v + period : v);
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_gaussian_field(int32_t G, const float* angle, double scale, int32_t* b_out, void* stream) {
    if (G < 1 || !angle || !b_out || !(fabs(scale) < 1e3)) return set_error(HP_ERR_ARG, "hp_gaussian_field: bad arguments");
    ::hp::count_launch();
    k_gaussian_field<<<(G + kT - 1) / kT, kT, 0, as_stream(stream)>>>(G, angle, scale, b_out);
    HP_LAUNCH_CHECK("k_gaussian_field");
    return HP_OK;
}

extern "C" int hp_grain_field(int32_t G, const float* quat, double C11, double C12, double C44, double sigma,
                              double k_disl, double energy_scale, int32_t* b_out, float* w_out, float* mmax_out,
                              void* stream) {
    if (G < 1 || !quat || !b_out) return set_error(HP_ERR_ARG, "hp_grain_field: bad arguments");
    const double den = (C11 - C12) * (C11 + 2.0 * C12);
    if (!(den != 0.0) || !(C44 != 0.0)) return set_error(HP_ERR_ARG, "hp_grain_field: singular moduli");
    FieldArgs a;
    a.quat = quat;
    a.G = G;
    a.S11 = (C11 + C12) / den;
    a.S12 = -C12 / den;
    a.S44 = 1.0 / C44;
    a.sigma = sigma;
    a.k = k_disl;
    a.scale = energy_scale;
    a.b = b_out;
    a.w = w_out;
    a.mmax = mmax_out;
    ::hp::count_launch();
    k_grain_field<<<(G + kT - 1) / kT, kT, 0, as_stream(stream)>>>(a);
    HP_LAUNCH_CHECK("k_grain_field");
    return HP_OK;
}

extern "C" int hp_grain_counts(hp_handle* h, int64_t* counts, int32_t* alive, void* stream) {
    hp::Range r_("hp_grain_counts");
    if (!h || !counts) return set_error(HP_ERR_ARG, "hp_grain_counts: bad arguments");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_grain_counts: no lattice bound");
    cudaStream_t s = as_stream(stream);
    const int32_t G = h->desc.n_grains;
    HP_CUDA(cudaMemsetAsync(counts, 0, sizeof(int64_t) * G, s));
    int32_t* bad = nullptr;
    HP_CUDA(cudaMallocAsync((void**)&bad, sizeof(int32_t), s));
    cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
    const int64_t threads = (h->lat.N + kSeg - 1) / kSeg;
    ::hp::count_launch();
    k_counts<<<(unsigned)((threads + kT - 1) / kT), kT, 0, s>>>(h->q, h->lat.N, G,
                                                                reinterpret_cast<unsigned long long*>(counts), bad);
    if (alive) {
        cudaMemsetAsync(alive, 0, sizeof(int32_t), s);
        ::hp::count_launch();
        k_alive<<<(G + kT - 1) / kT, kT, 0, s>>>(reinterpret_cast<const unsigned long long*>(counts), G, alive);
    }
    int32_t nbad = 0;
    cudaMemcpyAsync(&nbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(bad, s);
    HP_CUDA(cudaStreamSynchronize(s));
    HP_LAUNCH_CHECK("k_counts");
    if (nbad) return set_error(HP_ERR_STATE, "hp_grain_counts: lattice holds ids outside 0..G-1");
    return HP_OK;
}

extern "C" int hp_texture(int32_t G, int32_t orient_kind, const float* orient, const int64_t* counts, int32_t* bins,
                          int64_t* hist, void* stream) {
    if (G < 1 || !orient || !bins || orient_kind < HP_ORIENT_ANGLE || orient_kind > HP_ORIENT_ZROT)
        return set_error(HP_ERR_ARG, "hp_texture: bad arguments");
    cudaStream_t s = as_stream(stream);
    ::hp::count_launch();
    k_bins<<<(G + kT - 1) / kT, kT, 0, s>>>(G, orient_kind, orient, bins);
    if (hist && counts) {
        const int nb = orient_kind == HP_ORIENT_SO3 ? 24 : 90;
        HP_CUDA(cudaMemsetAsync(hist, 0, sizeof(int64_t) * nb, s));
        ::hp::count_launch();
        k_hist<<<(G + kT - 1) / kT, kT, 0, s>>>(G, orient_kind, bins,
                                                 reinterpret_cast<const unsigned long long*>(counts),
                                                 reinterpret_cast<unsigned long long*>(hist));
    }
    HP_LAUNCH_CHECK("k_bins/k_hist");
    return HP_OK;
}

// Slots of the handle's small measurement buffer (unsigned long long each).
enum { kSlotHist = 0, kSlotField = 90, kSlotAlive = 91, kSlotBad = 92, kSlots = 93 };

extern "C" int hp_measure(hp_handle* h, int32_t orient_kind, const float* orient, int32_t accumulate,
                          hp_stats* st, int64_t* hist, int32_t n_bins, void* stream) {
    hp::Range r_("hp_measure");
    if (!h || !st) return set_error(HP_ERR_ARG, "hp_measure: null handle or stats");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_measure: no lattice bound");
    if (orient && (orient_kind < HP_ORIENT_ANGLE || orient_kind > HP_ORIENT_ZROT))
        return set_error(HP_ERR_ARG, "hp_measure: bad orient_kind");
    const int nb = orient ? (orient_kind == HP_ORIENT_SO3 ? 24 : 90) : 0;
    if (hist && n_bins < nb) return set_error(HP_ERR_ARG, "hp_measure: histogram capacity too small");
    if (h->desc.field_mode != HP_FIELD_NONE && !h->table)
        return set_error(HP_ERR_STATE, "hp_measure: no field table set");
    const int32_t G = h->desc.n_grains;
    cudaStream_t s = as_stream(stream);
    if (!h->m_counts) HP_CUDA(cudaMalloc((void**)&h->m_counts, sizeof(unsigned long long) * (size_t)G));
    if (!h->m_bins) HP_CUDA(cudaMalloc((void**)&h->m_bins, sizeof(int32_t) * 2 * (size_t)G));
    if (!h->m_small) HP_CUDA(cudaMalloc((void**)&h->m_small, sizeof(unsigned long long) * kSlots));
    unsigned long long* sm = h->m_small;
    HP_CUDA(cudaMemsetAsync(h->m_counts, 0, sizeof(unsigned long long) * (size_t)G, s));
    HP_CUDA(cudaMemsetAsync(sm, 0, sizeof(unsigned long long) * kSlots, s));
    int32_t* alive = reinterpret_cast<int32_t*>(sm + kSlotAlive);
    int32_t* bad = reinterpret_cast<int32_t*>(sm + kSlotBad);
    const int64_t N = h->lat.N;
    const int64_t threads = (N + kSeg - 1) / kSeg;
    ::hp::count_launch();
    k_counts<<<(unsigned)((threads + kT - 1) / kT), kT, 0, s>>>(h->q, N, G, h->m_counts, bad);
    ::hp::count_launch();
    k_alive<<<(G + kT - 1) / kT, kT, 0, s>>>(h->m_counts, G, alive);
    if (orient) {
        ::hp::count_launch();
        k_bins<<<(G + kT - 1) / kT, kT, 0, s>>>(G, orient_kind, orient, h->m_bins);
        ::hp::count_launch();
        k_hist<<<(G + kT - 1) / kT, kT, 0, s>>>(G, orient_kind, h->m_bins, h->m_counts, sm + kSlotHist);
    }
    if (h->desc.field_mode == HP_FIELD_GRAIN) {
        ::hp::count_launch();
        k_field_sum_grain<<<(G + kT - 1) / kT, kT, 0, s>>>(h->m_counts, h->table, G, sm + kSlotField);
    } else if (h->desc.field_mode == HP_FIELD_POINT) {
        ::hp::count_launch();
        k_field_sum_point<<<4 * 152, kT, 0, s>>>(h->mp, h->table, (uint32_t)h->table_n, N, sm + kSlotField);
    }
    HP_LAUNCH_CHECK("hp_measure");
    unsigned long long host[kSlots];
    HP_CUDA(cudaMemcpyAsync(host, sm, sizeof(host), cudaMemcpyDeviceToHost, s));
    HP_CUDA(cudaStreamSynchronize(s));
    int32_t nbad = 0, nalive = 0;
    memcpy(&nbad, &host[kSlotBad], sizeof(int32_t));
    memcpy(&nalive, &host[kSlotAlive], sizeof(int32_t));
    if (nbad) return set_error(HP_ERR_STATE, "hp_measure: lattice holds ids outside 0..G-1");
    if (!accumulate) {
        memset(st, 0, sizeof(*st));
        if (hist) memset(hist, 0, sizeof(int64_t) * (size_t)nb);
    }
    st->sites += N;
    st->alive += nalive;
    st->field_sum += (int64_t)host[kSlotField];
    if (hist)
        for (int b = 0; b < nb; ++b) hist[b] += (int64_t)host[kSlotHist + b];
    // derived figures over everything accumulated so far
    st->mean_area = st->alive ? (double)st->sites / (double)st->alive : 0.0;
    st->mean_field = st->sites ? (double)st->field_sum / 256.0 / (double)st->sites : 0.0;
    if (hist && orient_kind == HP_ORIENT_SO3 && orient) {
        int64_t tot = 0;
        double m = 0.0;
        for (int b = 0; b < 20; ++b) {
            tot += hist[b];
            m += (double)hist[b] * (b + 0.5) * (0.5 / 20.0);
        }
        st->hist_total = tot;
        st->mean_mmax = tot ? m / (double)tot : 0.0;
        for (int f = 0; f < 4; ++f) st->families[f] = tot ? (double)hist[20 + f] / (double)tot : 0.0;
    } else if (hist && orient) {
        int64_t tot = 0;
        for (int b = 0; b < nb; ++b) tot += hist[b];
        st->hist_total = tot;
    }
    return HP_OK;
}

extern "C" int hp_angle_units(int32_t G, int32_t orient_kind, const float* orient, int32_t unit_per_degree,
                              int32_t period, int32_t* out, void* stream) {
    if (G < 1 || !orient || !out || unit_per_degree < 1 || period < 2 ||
        (orient_kind != HP_ORIENT_ANGLE && orient_kind != HP_ORIENT_ZROT))
        return set_error(HP_ERR_ARG, "hp_angle_units: bad arguments");
    ::hp::count_launch();
    k_angle_units<<<(G + kT - 1) / kT, kT, 0, as_stream(stream)>>>(G, orient_kind, orient, unit_per_degree, period, out);
    HP_LAUNCH_CHECK("k_angle_units");
    return HP_OK;
}
