// Initial polycrystal: Voronoi tessellation of G seeds on the periodic lattice
// and per-grain orientations (the set-up of the polycrystal runs, Sec. 4-5).
//
// Seeds: in round a every unplaced seed g draws site floor(u0 * N / 2^32) from
// Philox(seed; g, a, tag 2 | 0).  A site drawn by several seeds in one round
// goes to the lowest g; a site owned since an earlier round stays with its
// owner; losers redraw in round a+1.  The q buffer doubles as the claim array
// (free = 0x7F7F7F7F, tentative claim = g, placed = -1 - g).
//
// Assignment: each site takes the seed at the smallest periodic minimum-image
// squared distance, ties to the lowest index.  Seeds are bucketed into a grid
// of cells (about two seeds per cell); a site scans rings of cells of growing
// Chebyshev radius r around its own cell and stops once the best squared
// distance is below (r * wmin + 1)^2, the least squared distance any seed
// outside the scanned rings can have (wmin = narrowest cell width).
#include <math.h>


#include "common.cuh"

namespace hp {
namespace {

constexpr int kT = 256;

__global__ void k_seed_claim(int32_t* claim, const int64_t* pos, int32_t G, uint64_t seed, uint32_t round,
                             int64_t N) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || pos[g] >= 0) return;
    const uint4 u = draw(seed, (uint64_t)g, round, kTagVoronoi, 0);
    const int64_t s = (int64_t)(((uint64_t)u.x * (uint64_t)N) >> 32);
    atomicMin(claim + s, g);
}

__global__ void k_seed_resolve(int32_t* claim, int64_t* pos, int32_t G, uint64_t seed, uint32_t round, int64_t N,
                               int32_t* n_left) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || pos[g] >= 0) return;
    const uint4 u = draw(seed, (uint64_t)g, round, kTagVoronoi, 0);
    const int64_t s = (int64_t)(((uint64_t)u.x * (uint64_t)N) >> 32);
    if (claim[s] == g) {
        pos[g] = s;
        claim[s] = -1 - g;
    } else {
        atomicAdd(n_left, 1);
    }
}

struct Cells {
    int L[3];
    int nc[3];
    int wmin;
    int dim;
};

__device__ __forceinline__ int cell_of(int x, int L, int nc) { return (int)(((int64_t)x * nc) / L); }

__global__ void k_cell_count(const int64_t* pos, int32_t G, Cells c, int32_t* cnt, int4* xyz) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int64_t p = pos[g];
    const int x = (int)(p % c.L[0]);
    const int y = (int)((p / c.L[0]) % c.L[1]);
    const int z = (int)(p / ((int64_t)c.L[0] * c.L[1]));
    const int cid = cell_of(x, c.L[0], c.nc[0]) + c.nc[0] * (cell_of(y, c.L[1], c.nc[1]) + c.nc[1] * cell_of(z, c.L[2], c.nc[2]));
    xyz[g] = make_int4(x, y, z, cid);
    atomicAdd(cnt + cid, 1);
}

// exclusive scan of n ints by one block (n is at most a few million)
__global__ void k_scan(const int32_t* in, int32_t* out, int32_t n) {
    __shared__ int32_t part[1024];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b = t * per, e = min(n, b + per);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = t ? part[t - 1] : 0;
    for (int i = b; i < e; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (t == 1023) out[n] = part[1023];
}

__global__ void k_cell_scatter(const int4* xyz, int32_t G, const int32_t* start, int32_t* cursor, int4* list) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int4 v = xyz[g];
    const int32_t k = atomicAdd(cursor + v.w, 1);
    list[start[v.w] + k] = make_int4(v.x, v.y, v.z, g);
}

__device__ __forceinline__ int64_t mi(int d, int L) {
    d = d < 0 ? -d : d;
    return (int64_t)(d < L - d ? d : L - d);
}

__device__ __forceinline__ int wrapc(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__global__ void __launch_bounds__(kT) k_assign(int32_t* q, int32_t* mp, int64_t N, Cells c, const int32_t* start,
                                               const int4* list) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int x = (int)(i % c.L[0]);
    const int y = (int)((i / c.L[0]) % c.L[1]);
    const int z = (int)(i / ((int64_t)c.L[0] * c.L[1]));
    const int cx = cell_of(x, c.L[0], c.nc[0]), cy = cell_of(y, c.L[1], c.nc[1]), cz = cell_of(z, c.L[2], c.nc[2]);
    int64_t best = INT64_MAX;
    int32_t arg = INT32_MAX;
    const int rz_max = c.dim == 3 ? 1 : 0;
    for (int r = 0;; ++r) {
        const int rz = c.dim == 3 ? r : 0;
        for (int dz = -rz; dz <= rz; ++dz) {
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = (dz == -rz || dz == rz) && c.dim == 3;
                const bool yface = dy == -r || dy == r;
                // on an inner row only the two end cells belong to the ring
                const int step = (face || yface) ? 1 : (r > 0 ? 2 * r : 1);
                for (int dx = -r; dx <= r; dx += step) {
                    const int ccx = wrapc(cx + dx, c.nc[0]), ccy = wrapc(cy + dy, c.nc[1]), ccz = wrapc(cz + dz, c.nc[2]);
                    const int cid = ccx + c.nc[0] * (ccy + c.nc[1] * ccz);
                    const int b = start[cid], e = start[cid + 1];
                    for (int k = b; k < e; ++k) {
                        const int4 s = list[k];
                        const int64_t ddx = mi(x - s.x, c.L[0]), ddy = mi(y - s.y, c.L[1]), ddz = mi(z - s.z, c.L[2]);
                        const int64_t d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        if (d2 < best || (d2 == best && s.w < arg)) {
                            best = d2;
                            arg = s.w;
                        }
                    }
                }
            }
        }
        (void)rz_max;
        const int64_t bound = (int64_t)r * c.wmin + 1;
        const bool all = (2 * r + 1 >= c.nc[0]) && (2 * r + 1 >= c.nc[1]) && (c.dim == 2 || 2 * r + 1 >= c.nc[2]);
        if ((arg != INT32_MAX && best < bound * bound) || all) break;
    }
    q[i] = arg;
    if (mp) mp[i] = (int32_t)i;
}

__global__ void k_orient(int32_t G, uint64_t seed, int32_t kind, float* out) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const uint4 u = draw(seed, (uint64_t)g, 0, kTagVoronoi, 1);
    const double two32 = 4294967296.0, pi = 3.14159265358979323846;
    if (kind == HP_ORIENT_ANGLE) {
        out[g] = (float)(((double)u.x / two32) * (pi / 2.0));
    } else if (kind == HP_ORIENT_ZROT) {
        const double t = ((double)u.x / two32) * (pi / 2.0);
        double sh, ch;
        sincos(0.5 * t, &sh, &ch);
        out[4 * g + 0] = (float)ch;
        out[4 * g + 1] = 0.0f;
        out[4 * g + 2] = 0.0f;
        out[4 * g + 3] = (float)sh;
    } else {
        const double u1 = (double)u.x / two32, u2 = (double)u.y / two32, u3 = (double)u.z / two32;
        const double a = sqrt(1.0 - u1), b = sqrt(u1);
        double s2, c2, s3, c3;
        sincos(2.0 * pi * u2, &s2, &c2);
        sincos(2.0 * pi * u3, &s3, &c3);
        out[4 * g + 0] = (float)(a * s2);
        out[4 * g + 1] = (float)(a * c2);
        out[4 * g + 2] = (float)(b * s3);
        out[4 * g + 3] = (float)(b * c3);
    }
}

}  // namespace

int orientations_run(int32_t G, uint64_t seed, int32_t kind, float* orient, cudaStream_t s) {
    if (G < 1 || !orient || kind < HP_ORIENT_ANGLE || kind > HP_ORIENT_ZROT)
        return set_error(HP_ERR_ARG, "hp_orientations: bad arguments");
    ::hp::count_launch();
    k_orient<<<(G + kT - 1) / kT, kT, 0, s>>>(G, seed, kind, orient);
    HP_LAUNCH_CHECK("k_orient");
    return HP_OK;
}

int voronoi_run(hp_handle* h, int32_t orient_kind, float* orient, int64_t* seed_pos, cudaStream_t s) {
    const int32_t G = h->desc.n_grains;
    const int64_t N = h->lat.N;
    if (G < 1 || G > N) return set_error(HP_ERR_ARG, "hp_init_voronoi: need 1 <= G <= N");
    if (N >= (int64_t)1 << 32) return set_error(HP_ERR_ARG, "hp_init_voronoi: lattice too large (N >= 2^32)");
    // scratch: seed positions, per-seed coordinates, cell arrays
    Cells c;
    c.dim = h->lat.dim;
    for (int d = 0; d < 3; ++d) c.L[d] = (int)h->lat.L[d];
    const double per = pow(2.0 * (double)N / (double)G, 1.0 / c.dim);  // cell edge for ~2 seeds per cell
    int64_t ncell = 1;
    c.wmin = INT32_MAX;
    for (int d = 0; d < 3; ++d) {
        if (d >= c.dim) { c.nc[d] = 1; continue; }
        int n = (int)floor((double)c.L[d] / per);
        n = n < 1 ? 1 : n;
        c.nc[d] = n;
        ncell *= n;
        const int w = c.L[d] / n;  // narrowest cell width along d
        c.wmin = w < c.wmin ? w : c.wmin;
    }
    int64_t* pos = seed_pos;
    int64_t* pos_own = nullptr;
    int4 *xyz = nullptr, *list = nullptr;
    int32_t *cnt = nullptr, *start = nullptr, *cursor = nullptr, *n_left = nullptr;
    auto cleanup = [&]() {
        cudaFreeAsync(pos_own, s); cudaFreeAsync(xyz, s); cudaFreeAsync(list, s);
        cudaFreeAsync(cnt, s); cudaFreeAsync(start, s); cudaFreeAsync(cursor, s); cudaFreeAsync(n_left, s);
    };
    cudaError_t e = cudaSuccess;
    if (!pos) e = cudaMallocAsync((void**)&pos_own, sizeof(int64_t) * G, s), pos = pos_own;
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&xyz, sizeof(int4) * G, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&list, sizeof(int4) * G, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&cnt, sizeof(int32_t) * ncell, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&start, sizeof(int32_t) * (ncell + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&cursor, sizeof(int32_t) * ncell, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&n_left, sizeof(int32_t), s);
    if (e != cudaSuccess) { cleanup(); return set_error(HP_ERR_OOM, "hp_init_voronoi: scratch allocation failed"); }

    int rc = HP_OK;
    do {
        if ((e = cudaMemsetAsync(h->q, 0x7F, sizeof(int32_t) * N, s))) break;
        if ((e = cudaMemsetAsync(pos, 0xFF, sizeof(int64_t) * G, s))) break;
        const int gb = (G + kT - 1) / kT;
        for (uint32_t round = 0;; ++round) {
            if ((e = cudaMemsetAsync(n_left, 0, sizeof(int32_t), s))) break;
            ::hp::count_launch();
            k_seed_claim<<<gb, kT, 0, s>>>(h->q, pos, G, h->desc.seed, round, N);
            ::hp::count_launch();
            k_seed_resolve<<<gb, kT, 0, s>>>(h->q, pos, G, h->desc.seed, round, N, n_left);
            int32_t left = 0;
            if ((e = cudaMemcpyAsync(&left, n_left, sizeof(int32_t), cudaMemcpyDeviceToHost, s))) break;
            if ((e = cudaStreamSynchronize(s))) break;
            if (left == 0) break;
            if (round > (1u << 20)) { rc = set_error(HP_ERR_STATE, "hp_init_voronoi: seeding did not converge"); break; }
        }
        if (e || rc) break;
        if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ncell, s))) break;
        if ((e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * ncell, s))) break;
        ::hp::count_launch();
        k_cell_count<<<gb, kT, 0, s>>>(pos, G, c, cnt, xyz);
        ::hp::count_launch();
        k_scan<<<1, 1024, 0, s>>>(cnt, start, (int32_t)ncell);
        ::hp::count_launch();
        k_cell_scatter<<<gb, kT, 0, s>>>(xyz, G, start, cursor, list);
        const int64_t nb = (N + kT - 1) / kT;
        ::hp::count_launch();
        k_assign<<<(unsigned)nb, kT, 0, s>>>(h->q, h->mp, N, c, start, list);
        if ((e = cudaGetLastError())) break;
        if (orient) {
            ::hp::count_launch();
            k_orient<<<gb, kT, 0, s>>>(G, h->desc.seed, orient_kind, orient);
            if ((e = cudaGetLastError())) break;
        }
    } while (0);
    cleanup();
    if (e) return cuda_error(e, "hp_init_voronoi");
    return rc;
}

}  // namespace hp

// ---------------------------------------------------------------------------
// Voronoi initialisation without any device allocation.
//
// For callers that cannot allocate device memory while they run -- e.g. a
// process whose device memory is entirely pre-reserved by another allocator,
// or a steady-state loop that must never enter cudaMalloc/cudaFree -- the
// scratch of the tessellation (seed coordinates, cell lists, cell counters,
// the round counter) lives in one file-scope device array of fixed size.
// The array exists on every GPU that loads this library, until exit.
// ---------------------------------------------------------------------------
namespace hp {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)HP_VORONOI_STATIC_BYTES;
static __device__ __align__(256) unsigned char g_vor_scratch[kStaticScratchBytes];

// Worst case of the carve below at HP_VORONOI_STATIC_MAX_GRAINS on a square or
// cubic lattice: int64 seed sites (8 G), int4 seed coordinates and the int4
// cell list (16 G each), and three int32 cell arrays of at most G/2 + 1 cells
// (the cell edge is (2N/G)^(1/dim)), each carve rounded up to 256 bytes.
// Thin lattices whose cell count rounds up past G/2 are caught at run time.
static_assert((size_t)HP_VORONOI_STATIC_MAX_GRAINS * (8 + 16 + 16) +
                      3 * ((size_t)HP_VORONOI_STATIC_MAX_GRAINS / 2 + 2) * 4 + 7 * 256 <=
                  kStaticScratchBytes,
              "static Voronoi scratch too small for HP_VORONOI_STATIC_MAX_GRAINS");

// Device address of the static scratch on the current device.  The array's
// name is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress, taken on every call with the caller's device current
// (nothing is cached, so a context torn down and created again between calls
// never leaves a stale address behind).
int static_scratch(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vor_scratch);
    if (e != cudaSuccess) return cuda_error(e, "hp_init_voronoi_static: cudaGetSymbolAddress");
    *out = p;
    return HP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace hp

extern "C" int hp_init_voronoi_static(hp_handle* h, int32_t orient_kind, float* orient, int64_t* seed_pos,
                                      void* stream) {
    using namespace hp;
    if (!h) return set_error(HP_ERR_ARG, "hp_init_voronoi_static: null handle");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_init_voronoi_static: no lattice bound");
    if (orient && (orient_kind < HP_ORIENT_ANGLE || orient_kind > HP_ORIENT_ZROT))
        return set_error(HP_ERR_ARG, "hp_init_voronoi_static: bad orient_kind");
    const int32_t G = h->desc.n_grains;
    const int64_t N = h->lat.N;
    if (G < 1 || G > N) return set_error(HP_ERR_ARG, "hp_init_voronoi_static: need 1 <= G <= N");
    if (G > HP_VORONOI_STATIC_MAX_GRAINS)
        return set_error(HP_ERR_ARG, "hp_init_voronoi_static: more grains than the static scratch holds "
                                     "(HP_VORONOI_STATIC_MAX_GRAINS); use hp_init_voronoi");
    if (N >= (int64_t)1 << 32) return set_error(HP_ERR_ARG, "hp_init_voronoi_static: lattice too large (N >= 2^32)");
    cudaStream_t s = as_stream(stream);
    Cells c;
    c.dim = h->lat.dim;
    for (int d = 0; d < 3; ++d) c.L[d] = (int)h->lat.L[d];
    const double per = pow(2.0 * (double)N / (double)G, 1.0 / c.dim);
    int64_t ncell = 1;
    c.wmin = INT32_MAX;
    for (int d = 0; d < 3; ++d) {
        if (d >= c.dim) { c.nc[d] = 1; continue; }
        int n = (int)floor((double)c.L[d] / per);
        n = n < 1 ? 1 : n;
        c.nc[d] = n;
        ncell *= n;
        const int w = c.L[d] / n;
        c.wmin = w < c.wmin ? w : c.wmin;
    }
    // carve the static scratch
    void* base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    size_t off = 0;
    auto take = [&](size_t bytes) { void* p = (unsigned char*)base + off; off += align256(bytes); return p; };
    int64_t* pos = seed_pos ? seed_pos : (int64_t*)take(sizeof(int64_t) * G);
    int4* xyz = (int4*)take(sizeof(int4) * G);
    int4* list = (int4*)take(sizeof(int4) * G);
    int32_t* cnt = (int32_t*)take(sizeof(int32_t) * ncell);
    int32_t* start = (int32_t*)take(sizeof(int32_t) * (ncell + 1));
    int32_t* cursor = (int32_t*)take(sizeof(int32_t) * ncell);
    int32_t* n_left = (int32_t*)take(sizeof(int32_t));
    if (off > kStaticScratchBytes)
        return set_error(HP_ERR_ARG, "hp_init_voronoi_static: scratch layout exceeds the static array");

    // everything that must start at zero (or -1) is cleared here on every call
    HP_CUDA(cudaMemsetAsync(h->q, 0x7F, sizeof(int32_t) * N, s));
    HP_CUDA(cudaMemsetAsync(pos, 0xFF, sizeof(int64_t) * G, s));
    const int gb = (G + kT - 1) / kT;
    for (uint32_t round = 0;; ++round) {
        HP_CUDA(cudaMemsetAsync(n_left, 0, sizeof(int32_t), s));
        ::hp::count_launch();
        k_seed_claim<<<gb, kT, 0, s>>>(h->q, pos, G, h->desc.seed, round, N);
        ::hp::count_launch();
        k_seed_resolve<<<gb, kT, 0, s>>>(h->q, pos, G, h->desc.seed, round, N, n_left);
        int32_t left = 0;
        HP_CUDA(cudaMemcpyAsync(&left, n_left, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        HP_CUDA(cudaStreamSynchronize(s));
        if (left == 0) break;
        if (round > (1u << 20)) return set_error(HP_ERR_STATE, "hp_init_voronoi_static: seeding did not converge");
    }
    HP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ncell, s));
    HP_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * ncell, s));
    ::hp::count_launch();
    k_cell_count<<<gb, kT, 0, s>>>(pos, G, c, cnt, xyz);
    ::hp::count_launch();
    k_scan<<<1, 1024, 0, s>>>(cnt, start, (int32_t)ncell);
    ::hp::count_launch();
    k_cell_scatter<<<gb, kT, 0, s>>>(xyz, G, start, cursor, list);
    const int64_t nb = (N + kT - 1) / kT;
    ::hp::count_launch();
    k_assign<<<(unsigned)nb, kT, 0, s>>>(h->q, h->mp, N, c, start, list);
    if (orient) {
        ::hp::count_launch();
        k_orient<<<gb, kT, 0, s>>>(G, h->desc.seed, orient_kind, orient);
    }
    HP_LAUNCH_CHECK("hp_init_voronoi_static");
    return HP_OK;
}
