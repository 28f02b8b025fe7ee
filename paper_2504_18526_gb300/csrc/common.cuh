// Internal device helpers shared by the SI-MLSDC kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace sisdc {

constexpr int NQMAX = 16;     // nodes per direction: P <= 8 in 2D, P <= 15 in 1D
constexpr int MMAX = 8;       // collocation nodes per level
constexpr int MAXTERMS = 8;   // terms of a fused linear combination

// Device error codes (mirrors sisdc_status, stored as a positive flag bitmask).
enum DevErr : int { DEV_NOCONV = 1, DEV_TIMEOUT = 2, DEV_NONFINITE = 4 };

// Stats slots (long long).
enum StatSlot : int { ST_SOLVES = 0, ST_ITERS = 1, ST_MAXIT = 2, ST_NOCONV = 3, ST_IR = 4, ST_N = 8 };

// A coefficient a = a0 + a2 * lam^2, lam read from device memory when given.
// Used for the nu_tilde-dependent factors dt_m nu_tilde(u) with
// nu_tilde = nu_d + dt_m/2 * lam_max(u)^2.
struct Coef {
    double a0;
    double a2;
    const double* lam;
};

__device__ __forceinline__ double coef_value(const Coef& c) {
    double v = c.a0;
    if (c.lam) { double l = *c.lam; v += c.a2 * l * l; }
    return v;
}

// Block size for `n` working threads, rounded up to whole warps: the block
// reductions shuffle with full warp masks, so no warp may be partial.  The
// extra threads are idle (their element index is past the tile).
inline int warp_round(int n) { return (n + 31) & ~31; }

// Geometry and tables of one level, passed by value.
struct Geo {
    int dim, nq, nqy, q;          // nodes per direction / per element
    int nex, ney, nel, ncomp;
    long long N;                  // nodes per component = nel * q
    double hx, hy;                // element sizes
    double taux, tauy;            // SIPG penalties 2 (P+1)^2 / h
    const double* D;              // [nq*nq] d l_j/dxi at xi_i (device)
    const double* K;              // [nq*nq] D^T W D (device)
    const double* w;              // [nq] GLL weights (device)
    const double* dline_x;        // [nq] diagonal of the 1D SIPG line operator (x)
    const double* dline_y;        // [nq] (y)
    const double* fds;            // element-wise fast diagonalisation: S_x [nq*nq], lam_x [nq],
                                  // S_y, lam_y (nullable: Jacobi only)
    // host-computed factors (no divisions in the kernels' inner loops)
    double sx, sy;                // 2/h_x, 2/h_y
    double ihx, ihy;              // 1/h_x, 1/h_y
    double liftLx, liftRx;        // (2/h_x)/w_0, (2/h_x)/w_P: Rusanov flux lifting
    double liftLy, liftRy;
};

// Deterministic block reduction (fixed shuffle tree, fixed warp order).
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the block; result valid in thread 0. `scratch` >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

__device__ __forceinline__ double block_max(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? scratch[lane] : 0.0;
        r = warp_max(r);
    }
    return r;
}

// Max of non-negative doubles through their bit patterns (monotone for x >= 0).
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff8000000000000LL);   // NaN marks trouble
    atomicMax(reinterpret_cast<unsigned long long*>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for cooperative launches with a bounded wait, over a
// monotonically increasing arrival counter: `count` is 0 when a launch starts
// (grid_exit resets it), every barrier adds exactly gridDim.x arrivals, so the
// k-th barrier's arrivals see old values in [(k-1) G, k G) and wait until the
// counter reaches k G.  One release-add per block and acquire-load polling;
// thread 0 waits for the block (bar.sync before and after, so the block's
// writes are ordered before the release and the acquire before its reads).
// On timeout the block records DEV_TIMEOUT in *err and returns false; callers
// then leave the kernel, so that every wait in the grid ends.
constexpr unsigned long long BARRIER_TIMEOUT_NS = 2000000000ull;   // 2 s
// second bound on the polls, in case the global timer does not advance
// (about 10-15 s of L2 round trips)
constexpr unsigned BARRIER_MAX_SPINS = 1u << 24;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* /*exits*/, int* err,
                                             unsigned long long timeout_ns = BARRIER_TIMEOUT_NS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        const unsigned old = atom_add_release_gpu(count, 1u);
        const unsigned target = (old / nb + 1u) * nb;
        if (ld_acquire_gpu(count) < target) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire_gpu(count) < target) {
                if ((++spins & 255u) == 0u && (globaltimer_ns() - t0 > timeout_ns || spins >= BARRIER_MAX_SPINS)) {
                    atomicOr(err, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok && ((*(volatile int*)err & DEV_TIMEOUT) == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// Every block of a launch that uses grid_barrier calls this once, at its end
// (on every path): the last block out resets the arrival counter for the next
// launch on the stream (all blocks have left every barrier by then).
__device__ __forceinline__ void grid_exit(unsigned* count, unsigned* exits) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(exits, 1u) == nb - 1u) {
            atomicExch(count, 0u);
            atomicExch(exits, 0u);
        }
    }
}

// Sum of gridDim.x partials in a fixed order; every block gets the same bits.
__device__ __forceinline__ double grid_total(const double* partials, double* scratch) {
    __shared__ double s_tot;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
            v += *((volatile const double*)(partials + b));
        v = warp_sum(v);
        if (threadIdx.x == 0) s_tot = v;
    }
    __syncthreads();
    const double r = s_tot;
    __syncthreads();
    return r;
}

}  // namespace sisdc
