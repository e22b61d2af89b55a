// Bounded software grid barrier and block helpers for the standalone
// persistent solvers (cooperative launches, one block per SM).
//
// A scalars struct S provides `unsigned long long bar` (monotonic arrival
// count, zeroed before the launch), `int err` and `int err_where`.  Every
// wait is bounded: after `limit` clock cycles the waiting block records
// QS_ERR_TIMEOUT (and where it waited) and returns false, and every other
// block returns false at its next barrier, so the kernel ends and the host
// reads the status.
#pragma once

#include <cuda_runtime.h>

#include "qs.h"

namespace qsync {

__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ double vload(const double *p) { return *(const volatile double *)p; }

__device__ __forceinline__ unsigned long long acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename S>
struct GridBarrier {
    S *sc;
    unsigned long long *epoch;  // shared-memory count of this block's barriers
    long long limit;            // clock cycles a block may wait
    __device__ bool operator()(int where) const {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = vload(&sc->err) == 0;
            if (ok) {
                const unsigned long long target = (*epoch + 1) * gridDim.x;
                *epoch += 1;
                release_add_u64(&sc->bar, 1ull);
                const long long t0 = clock64();
                while (acquire_u64(&sc->bar) < target) {
                    if (vload(&sc->err) != 0) {
                        ok = 0;
                        break;
                    }
                    if (clock64() - t0 > limit) {
                        if (atomicCAS(&sc->err, 0, QS_ERR_TIMEOUT) == 0) sc->err_where = where;
                        ok = 0;
                        break;
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

struct BlockSync {
    __device__ bool operator()(int) const {
        __syncthreads();
        return true;
    }
};

// Threads taking part in a phase: the whole grid, or one block.
struct Team {
    int t, nt;
};

// The grid-wide team of a persistent launch with runs of 32 consecutive
// indices handed to the blocks in turn (run w * gridDim.x + b to warp w of
// block b): a loop shorter than the launch (a coarse level) still spreads
// over every SM, which float64 work needs on GB300 (about two FMA per clock
// per SM), while each warp's accesses stay contiguous.  t ranges over a
// permutation of [0, nt) (blockDim.x a multiple of 32).
__device__ __forceinline__ Team spread_team() {
    const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    return Team{((w * (int)gridDim.x + (int)blockIdx.x) << 5) + lane,
                (int)(gridDim.x * blockDim.x)};
}

// Adds the block's sums of vals[0 .. k) into dst[0 .. k) (one atomic each).
template <int kThreadsMax>
__device__ void block_sum_add(const double *vals, int k, double *dst) {
    __shared__ double red[kThreadsMax / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = 0; c < k; ++c) {
        double v = vals[c];
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w][c];
            atomicAdd(&dst[c], s);
        }
    __syncthreads();
}

}  // namespace qsync
