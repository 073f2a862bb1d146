// Device helpers shared by the sweep kernels (sweep.cu, tile.cu, lean.cu): lattice
// neighbourhoods and colourings (Sec. 4), the integer Metropolis test (Eq. (7)
// with the acceptance table of Sec. 4), periodic wrapping, the launch
// arguments of one fused sweep launch, and the mbarrier wait used by the
// TMA-fed kernels.  Internal; not part of the public ABI.
#pragma once

#include "common.cuh"

namespace hp {

// Arguments of one fused sweep launch over the planes of one parity.
struct PlaneArgs {
    const int32_t* q_in;    // own plane, previous state
    const int32_t* mp_in;
    const int32_t* q_nb;    // z-neighbour planes (3D)
    const int32_t* mp_nb;
    int32_t* q_out;
    int32_t* mp_out;
    const int32_t* table;
    uint32_t table_n;
    const uint32_t* thr;
    int32_t D, J;
    uint64_t seed;
    uint32_t sweep;
    int Lx, Ly, Lz;
    int zpar;               // 3D: parity of the planes handled by this launch
    int tiles_x;
    int tiles;              // tiles per plane
    int fast;               // 1: window narrower than the lattice (wrap by one add)
    int vec;                // 1: fast and Lx % 4 == 0 (16-byte row chunks)
    uint32_t rk[20];        // Philox round keys of seed (philox_round_keys)
};

namespace {

template <int DIM, int NBR>
struct Geo;

// 2D-4: +x, -x, +y, -y ; colours (x+y)&1
template <>
struct Geo<2, 4> {
    static constexpr int M = 4, C = 2;
    __device__ static void off(int k, int& dx, int& dy, int& dz) {
        dx = k == 0 ? 1 : (k == 1 ? -1 : 0);
        dy = k == 2 ? 1 : (k == 3 ? -1 : 0);
        dz = 0;
    }
};
// 2D-8: (dy,dx) row-major without (0,0) ; colours (x&1) + 2(y&1)
template <>
struct Geo<2, 8> {
    static constexpr int M = 8, C = 4;
    __device__ static void off(int k, int& dx, int& dy, int& dz) {
        const int kk = k + (k >= 4);
        dy = kk / 3 - 1;
        dx = kk % 3 - 1;
        dz = 0;
    }
};
// 3D-6: +x, -x, +y, -y, +z, -z ; colours (x+y+z)&1
template <>
struct Geo<3, 6> {
    static constexpr int M = 6, C = 2;
    __device__ static void off(int k, int& dx, int& dy, int& dz) {
        dx = k == 0 ? 1 : (k == 1 ? -1 : 0);
        dy = k == 2 ? 1 : (k == 3 ? -1 : 0);
        dz = k == 4 ? 1 : (k == 5 ? -1 : 0);
    }
};
// 3D-26: (dz,dy,dx) lexicographic without (0,0,0) ; colours (x&1)+2(y&1)+4(z&1)
template <>
struct Geo<3, 26> {
    static constexpr int M = 26, C = 8;
    __device__ static void off(int k, int& dx, int& dy, int& dz) {
        const int kk = k + (k >= 13);
        dz = kk / 9 - 1;
        dy = (kk / 3) % 3 - 1;
        dx = kk % 3 - 1;
    }
};

__device__ __forceinline__ int wrapi(int a, int L) {
    a %= L;
    return a < 0 ? a + L : a;
}

// a in [-L, 2L)
__device__ __forceinline__ int wrap1(int a, int L) {
    a += a < 0 ? L : 0;
    return a - (a >= L ? L : 0);
}

__device__ __forceinline__ bool metropolis(int32_t d, int32_t D, const uint32_t* __restrict__ thr, uint32_t u) {
    if (d < 0) return true;
    if (d > D) return false;
    const uint32_t t = __ldg(thr + d);
    return t == 0xFFFFFFFFu || u < t;
}

// Field-table lookup with the index clamped into the table (ids come from
// caller buffers; an out-of-range id must not read outside the table).
__device__ __forceinline__ int32_t tab(const int32_t* __restrict__ t, uint32_t n, int32_t i) {
    const uint32_t u = (uint32_t)i;
    return __ldg(t + (u < n ? u : n - 1));
}

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Wait for an mbarrier phase with a clock limit (default about two seconds at
// the boost clock); false on timeout.  Each try_wait may suspend the thread for
// up to 20 us (it wakes as soon as the phase completes), so a waiting warp
// issues few instructions.
constexpr long long kWaitCycles = 1ll << 32;
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(mbar), "r"(parity), "r"(20000u) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Block-wide wait for a window's bulk copies (every thread calls it).  Warp 0
// polls the barrier while the other warps wait at the block barrier (issuing
// nothing); once the copies have landed every thread observes the completed
// phase itself (a try_wait that succeeds at once), which orders its reads
// after the copies.  On a timeout every thread of the block keeps waiting, up
// to four more limits, so that no copy is still landing in this block's shared
// memory when it leaves; *flag becomes 1, or 2 if even that drain ran out
// (copies may still have been in flight at exit: the context must not be
// trusted).  False after a timeout.
__device__ __forceinline__ bool wait_or_drain(uint32_t mbar, int* flag, long long limit = kWaitCycles) {
    bool ok = true;
    if (threadIdx.x < 32) ok = wait_parity(mbar, 0u, limit);
    if (!__syncthreads_or(!ok)) {
        if (threadIdx.x >= 32) wait_parity(mbar, 0u, limit);
        return true;
    }
    bool drained = false;
    for (int i = 0; i < 5 && !drained; ++i) drained = wait_parity(mbar, 0u, limit);
    const bool all = !__syncthreads_or(!drained);
    if (threadIdx.x == 0) atomicMax(flag, all ? 1 : 2);
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const int32_t* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// Copy window columns [xs, xs + W) of one lattice row (xs >= -4, W <= Lx,
// all multiples of 4 ints) into dst, wrapping periodically.
__device__ __forceinline__ void copy_row(int32_t* dst, const int32_t* row, int xs, int W, int Lx, uint32_t mb) {
    if (xs < 0) {
        bulk_g2s(s_addr(dst), row + Lx + xs, (uint32_t)(-xs) * 4u, mb);
        bulk_g2s(s_addr(dst - xs), row, (uint32_t)(W + xs) * 4u, mb);
    } else if (xs + W > Lx) {
        bulk_g2s(s_addr(dst), row + xs, (uint32_t)(Lx - xs) * 4u, mb);
        bulk_g2s(s_addr(dst + (Lx - xs)), row, (uint32_t)(xs + W - Lx) * 4u, mb);
    } else {
        bulk_g2s(s_addr(dst), row + xs, (uint32_t)W * 4u, mb);
    }
}

}  // namespace

// Tile kernel (tile.cu): one launch over the planes of one parity; WX x WY
// window (core (WX - 8) x (WY - 8)), a.tiles_x / a.tiles set for that core.
int tile_launch(const PlaneArgs& a, int field, bool hasmp, int nbr, int planes, int WX, int WY, cudaStream_t s);
// The same over many lattices: d_args[R] (device), block offsets d_start[R+1];
// blocks == 0 only configures the kernel (outside a graph capture).
int tile_launch_batch(const PlaneArgs* d_args, const int64_t* d_start, int R, int64_t blocks, uint32_t sweep_add,
                      int field, bool hasmp, int nbr, int WX, int WY, cudaStream_t s);
// Reads and clears the tile kernel's timeout flag.
int tile_status(int* timed_out);

// Lean 3D kernel (lean.cu): one launch over the planes of one parity; 64 x WY
// windows (WY 40 or 44), draws made while the window is in flight.
int lean_launch(const PlaneArgs& a, int field, bool hasmp, int planes, int WY, cudaStream_t s);
// The same over many lattices (see tile_launch_batch).
int lean_launch_batch(const PlaneArgs* d_args, const int64_t* d_start, int R, int64_t blocks, uint32_t sweep_add,
                      int field, bool hasmp, int WY, cudaStream_t s);
// Reads and clears the lean kernel's timeout flag (2: a drain ran out too).
int lean_status(int* timed_out);


}  // namespace hp
