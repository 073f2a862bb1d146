// C ABI entry points: handle lifecycle, buffers, threshold table, dispatch.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>

#include "common.cuh"

namespace hp {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launch_n(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return set_error(e == cudaErrorMemoryAllocation ? HP_ERR_OOM : HP_ERR_CUDA, m);
}

namespace {

__global__ void k_philox(uint64_t seed, const uint4* ctr, int64_t n, uint4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox10((uint32_t)seed, (uint32_t)(seed >> 32), ctr[i]);
}

int colours_of(int dim, int nbr) {
    if (dim == 2 && nbr == 4) return 2;
    if (dim == 2 && nbr == 8) return 4;
    if (dim == 3 && nbr == 6) return 2;
    if (dim == 3 && nbr == 26) return 8;
    return 0;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" const char* hp_last_error_message(void) { return g_last_error.c_str(); }

extern "C" int hp_last_error(const hp_handle* h, char* buf, size_t n) {
    (void)h;  // messages are kept per host thread, not per handle
    if (!buf || n == 0) return HP_ERR_ARG;
    const size_t k = g_last_error.size() < n - 1 ? g_last_error.size() : n - 1;
    memcpy(buf, g_last_error.data(), k);
    buf[k] = '\0';
    return HP_OK;
}

extern "C" const char* hp_version(void) { return "hmcpotts 0.1 sm_103a"; }

extern "C" int hp_kernel_launches(uint64_t* out) {
    if (!out) return set_error(HP_ERR_ARG, "hp_kernel_launches: null argument");
    *out = g_launches.load(std::memory_order_relaxed);
    return HP_OK;
}

extern "C" int hp_create(const hp_desc* d, hp_handle** out) {
    if (!d || !out) return set_error(HP_ERR_ARG, "hp_create: null argument");
    *out = nullptr;
    const int C = colours_of(d->dim, d->nbr);
    if (!C) return set_error(HP_ERR_ARG, "hp_create: unsupported (dim, nbr); use 2D 4/8 or 3D 6/26");
    const int64_t Lz = d->dim == 3 ? d->L[2] : 1;
    for (int k = 0; k < d->dim; ++k)
        if (d->L[k] < 2 || (d->L[k] & 1) || d->L[k] > (1 << 30))
            return set_error(HP_ERR_ARG, "hp_create: every edge must be even and >= 2");
    const int64_t N = d->L[0] * d->L[1] * Lz;
    if (N > ((int64_t)1 << 31) - 1) return set_error(HP_ERR_ARG, "hp_create: more than 2^31-1 sites");
    if (d->n_grains < 1) return set_error(HP_ERR_ARG, "hp_create: n_grains must be >= 1");
    if (d->field_mode < HP_FIELD_NONE || d->field_mode > HP_FIELD_POINT)
        return set_error(HP_ERR_ARG, "hp_create: bad field_mode");
    if (d->J_fix < 0 || d->J_fix > (1 << 20)) return set_error(HP_ERR_ARG, "hp_create: J_fix out of range");
    hp_handle* h = new (std::nothrow) hp_handle();
    if (!h) return set_error(HP_ERR_OOM, "hp_create: out of host memory");
    h->desc = *d;
    h->lat.dim = d->dim;
    h->lat.L[0] = d->L[0];
    h->lat.L[1] = d->L[1];
    h->lat.L[2] = Lz;
    h->lat.nbr = d->nbr;
    h->lat.colours = C;
    h->lat.N = N;
    *out = h;
    return HP_OK;
}

extern "C" int hp_destroy(hp_handle* h) {
    if (!h) return HP_OK;
    cudaFree(h->q_alt);
    cudaFree(h->mp_alt);
    cudaFree(h->thr);
    cudaFree(h->an_J);
    cudaFree(h->an_mob);
    cudaFree(h->m_counts);
    cudaFree(h->m_bins);
    cudaFree(h->m_small);
    delete h;
    return HP_OK;
}

extern "C" int hp_bind(hp_handle* h, int32_t* q, int32_t* mp) {
    if (!h || !q) return set_error(HP_ERR_ARG, "hp_bind: null handle or q");
    if (h->desc.field_mode == HP_FIELD_POINT && !mp)
        return set_error(HP_ERR_ARG, "hp_bind: HP_FIELD_POINT needs the material-point index buffer mp");
    const size_t bytes = sizeof(int32_t) * (size_t)h->lat.N;
    if (!h->q_alt) HP_CUDA(cudaMalloc((void**)&h->q_alt, bytes));
    if (mp && !h->mp_alt) HP_CUDA(cudaMalloc((void**)&h->mp_alt, bytes));
    h->q = q;
    h->mp = mp;
    return HP_OK;
}

// Upload (is_host != 0: from pageable or pinned host memory) or take from
// device memory the lattice state q (and mp) of a bound handle.
extern "C" int hp_set_spins(hp_handle* h, const int32_t* q, const int32_t* mp, int32_t is_host, void* stream) {
    hp::Range r_("hp_set_spins");
    if (!h || !q) return set_error(HP_ERR_ARG, "hp_set_spins: null handle or q");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_set_spins: no lattice bound");
    if (mp && !h->mp) return set_error(HP_ERR_STATE, "hp_set_spins: no material-point buffer bound");
    const size_t bytes = sizeof(int32_t) * (size_t)h->lat.N;
    const cudaMemcpyKind k = is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaStream_t s = as_stream(stream);
    HP_CUDA(cudaMemcpyAsync(h->q, q, bytes, k, s));
    if (mp) HP_CUDA(cudaMemcpyAsync(h->mp, mp, bytes, k, s));
    return HP_OK;
}

extern "C" int hp_get_spins(const hp_handle* h, int32_t* q, int32_t* mp, int32_t is_host, void* stream) {
    hp::Range r_("hp_get_spins");
    if (!h || !q) return set_error(HP_ERR_ARG, "hp_get_spins: null handle or q");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_get_spins: no lattice bound");
    if (mp && !h->mp) return set_error(HP_ERR_STATE, "hp_get_spins: no material-point buffer bound");
    const size_t bytes = sizeof(int32_t) * (size_t)h->lat.N;
    const cudaMemcpyKind k = is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaStream_t s = as_stream(stream);
    HP_CUDA(cudaMemcpyAsync(q, h->q, bytes, k, s));
    if (mp) HP_CUDA(cudaMemcpyAsync(mp, h->mp, bytes, k, s));
    return HP_OK;
}

extern "C" int hp_init_voronoi(hp_handle* h, int32_t orient_kind, float* orient, int64_t* seed_pos, void* stream) {
    hp::Range r_("hp_init_voronoi");
    if (!h) return set_error(HP_ERR_ARG, "hp_init_voronoi: null handle");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_init_voronoi: no lattice bound");
    if (orient && (orient_kind < HP_ORIENT_ANGLE || orient_kind > HP_ORIENT_ZROT))
        return set_error(HP_ERR_ARG, "hp_init_voronoi: bad orient_kind");
    return voronoi_run(h, orient_kind, orient, seed_pos, as_stream(stream));
}

extern "C" int hp_orientations(int32_t G, uint64_t seed, int32_t orient_kind, float* orient, void* stream) {
    return orientations_run(G, seed, orient_kind, orient, as_stream(stream));
}

extern "C" int hp_set_field(hp_handle* h, const int32_t* table, int64_t n) {
    if (!h) return set_error(HP_ERR_ARG, "hp_set_field: null handle");
    const int64_t want = h->desc.field_mode == HP_FIELD_GRAIN ? h->desc.n_grains
                         : h->desc.field_mode == HP_FIELD_POINT ? h->lat.N : 0;
    if (h->desc.field_mode == HP_FIELD_NONE) return set_error(HP_ERR_STATE, "hp_set_field: handle has HP_FIELD_NONE");
    if (!table || n != want) return set_error(HP_ERR_ARG, "hp_set_field: table size must be G (grain) or N (point)");
    h->table = table;
    h->table_n = n;
    return HP_OK;
}

extern "C" int hp_build_threshold_table(double kT, int32_t zero_rule, uint32_t* out, int32_t cap, int32_t* D) {
    if (!(kT >= 0.0) || !out || !D || cap < 1) return set_error(HP_ERR_ARG, "hp_build_threshold_table: bad arguments");
    out[0] = zero_rule ? 0u : 0xFFFFFFFFu;
    int32_t last = 0;
    if (kT > 0.0) {
        const double scale = 256.0 * kT;
        for (int32_t d = 1;; ++d) {
            const double f = floor(ldexp(exp(-(double)d / scale), 32));
            if (f < 1.0) break;
            if (d >= cap) return set_error(HP_ERR_ARG, "hp_build_threshold_table: capacity too small");
            out[d] = f > 4294967294.0 ? 0xFFFFFFFEu : (uint32_t)f;
            last = d;
        }
    }
    *D = last;
    return HP_OK;
}

extern "C" int hp_set_threshold_table(hp_handle* h, const uint32_t* thr, int32_t D, void* stream) {
    if (!h || !thr || D < 0) return set_error(HP_ERR_ARG, "hp_set_threshold_table: bad arguments");
    cudaStream_t s = as_stream(stream);
    if (D + 1 > h->thr_cap) {
        cudaFree(h->thr);
        h->thr = nullptr;
        HP_CUDA(cudaMalloc((void**)&h->thr, sizeof(uint32_t) * (size_t)(D + 1)));
        h->thr_cap = D + 1;
    }
    HP_CUDA(cudaMemcpyAsync(h->thr, thr, sizeof(uint32_t) * (size_t)(D + 1), cudaMemcpyHostToDevice, s));
    HP_CUDA(cudaStreamSynchronize(s));  // the host table may be freed after return
    h->D = D;
    return HP_OK;
}

extern "C" int hp_set_sweep_kernel(hp_handle* h, int32_t kind) {
    if (!h || kind < HP_SWEEP_AUTO || kind > HP_SWEEP_FUSED) return set_error(HP_ERR_ARG, "hp_set_sweep_kernel: bad kind");
    if (kind == HP_SWEEP_FUSED && h->lat.nbr == 6)
        return set_error(HP_ERR_ARG, "hp_set_sweep_kernel: no fused kernel for the 3D 6-neighbour lattice");
    h->sweep_kernel = kind;
    return HP_OK;
}

extern "C" int hp_sweep(hp_handle* h, int32_t n_mcs, void* stream) {
    hp::Range r_("hp_sweep");
    if (!h || n_mcs < 0) return set_error(HP_ERR_ARG, "hp_sweep: bad arguments");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_sweep: no lattice bound");
    if (!h->thr) return set_error(HP_ERR_STATE, "hp_sweep: no threshold table");
    if (h->desc.field_mode != HP_FIELD_NONE && !h->table) return set_error(HP_ERR_STATE, "hp_sweep: no field table");
    if (n_mcs == 0) return HP_OK;
    return sweep_run(h, n_mcs, as_stream(stream));
}

extern "C" int hp_get_sweep_counter(const hp_handle* h, uint64_t* out) {
    if (!h || !out) return set_error(HP_ERR_ARG, "hp_get_sweep_counter: null argument");
    *out = h->sweep;
    return HP_OK;
}

extern "C" int hp_set_sweep_counter(hp_handle* h, uint64_t v) {
    if (!h) return set_error(HP_ERR_ARG, "hp_set_sweep_counter: null handle");
    h->sweep = v;
    return HP_OK;
}

extern "C" int hp_philox(uint64_t seed, const uint32_t* ctr, int64_t n, uint32_t* out, void* stream) {
    if (!ctr || !out || n < 0) return set_error(HP_ERR_ARG, "hp_philox: bad arguments");
    if (n == 0) return HP_OK;
    ::hp::count_launch();
    k_philox<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(seed, reinterpret_cast<const uint4*>(ctr), n,
                                                                         reinterpret_cast<uint4*>(out));
    HP_LAUNCH_CHECK("k_philox");
    return HP_OK;
}

extern "C" int hp_debug_wait_timeout(int32_t unit, int64_t limit_cycles, int32_t late, void* stream) {
    if (unit == 0) return lean_wait_probe((long long)limit_cycles, late, as_stream(stream));
    if (unit == 1) return mlp_wait_probe((long long)limit_cycles, late, as_stream(stream));
    return set_error(HP_ERR_ARG, "hp_debug_wait_timeout: unit must be 0 (sweep) or 1 (surrogate)");
}

extern "C" int hp_build_read_shockley(double J_max, double theta_max, int32_t bin, int32_t nbins,
                                      int32_t unit_per_degree, int32_t* J_out, uint32_t* mob_out) {
    if (!(J_max >= 0.0) || J_max > 4096.0 || !(theta_max > 0.0) || bin < 1 || nbins < 1 || unit_per_degree < 1 ||
        !J_out)
        return set_error(HP_ERR_ARG, "hp_build_read_shockley: bad arguments");
    for (int32_t k = 0; k < nbins; ++k) {
        const double x = ((double)k + 0.5) * (double)bin / (double)unit_per_degree / theta_max;
        const double e = x < 1.0 ? J_max * x * (1.0 - log(x)) : J_max;
        J_out[k] = (int32_t)nearbyint(256.0 * e);
        if (mob_out) {
            const double f = floor(ldexp(1.0 - exp(-5.0 * x * x * x * x), 32));
            mob_out[k] = f >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)f;
        }
    }
    return HP_OK;
}

extern "C" int hp_si_links(const hp_si_in* in, hp_si_out* out) {
    if (!in || !out || !(in->gamma_s > 0) || !(in->m_s > 0) || !(in->l0 > 0) || !(in->gamma_mc > 0) ||
        !(in->m_mc > 0) || !(in->Delta > 0) || !(in->J > 0) || !(in->tau_mc > 0))
        return set_error(HP_ERR_ARG, "hp_si_links: every quantity must be positive");
    // Eq. (8): gamma_s = gamma E0 / (Delta^2 J l0^2)  ->  E0
    //          m_s = Delta^4 m l0^4 / (J tau E0 t0)    ->  t0
    //          b_s = 2 b E0 / (Delta^3 l0^3)           ->  b per unit b_s
    const double D = in->Delta, l0 = in->l0;
    out->E0 = in->gamma_s * D * D * in->J * l0 * l0 / in->gamma_mc;
    out->t0 = D * D * D * D * in->m_mc * l0 * l0 * l0 * l0 / (in->J * in->tau_mc * out->E0 * in->m_s);
    out->seconds_per_mcs = in->tau_mc * out->t0;
    out->b_per_bs = D * D * D * l0 * l0 * l0 / (2.0 * out->E0);
    return HP_OK;
}
