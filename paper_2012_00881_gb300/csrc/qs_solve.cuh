// Device machinery shared by the slice engine and the adjoint engine: the
// bounded grid barrier, block reductions, and the multigrid solves (float64
// V-cycles; refined form: float64 residual, float32 staged V-cycles, float64
// correction).  Everything is in an unnamed namespace: each translation unit
// that includes this header gets its own copy.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "qs_cluster.cuh"
#include "qs_tile.cuh"

namespace {

#define SYNC(where)                 \
    do {                            \
        if (!S(where)) return false; \
    } while (0)

__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ double vload(const double *p) { return *(const volatile double *)p; }
__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

__device__ __forceinline__ int64_t global_ns() {
    int64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  Each
// block counts the barriers it has passed (its epoch); on arrival its thread
// 0 adds 1 to a monotonic counter with a release reduction (no round trip)
// and polls with acquire loads until the counter reaches epoch * nblk.
struct Sync {
    DevScalars *sc;             // the instance's scalars (error word, trace count)
    unsigned long long *bar;    // monotonic arrival counter of the blocks in the team
    unsigned nblk;              // blocks in the team
    long long limit;
    int64_t *trace;
    int trace_cap;
    unsigned long long *epoch;  // this block's barrier count (shared memory)
    bool tracer;                // this block records the phase trace
    int cl = 1;                 // cluster size of the launch (> 1: clusters run
                                // the multigrid cycles, see qs_cluster.cuh)
    __device__ bool operator()(int where) const {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            if (vload(&sc->err) != 0) {
                ok = 0;
            } else {
                const unsigned long long target = (*epoch + 1) * nblk;
                *epoch += 1;
                red_release_add_u64(bar, 1ull);
                if (ld_acquire_u64(bar) < target) {
                    const long long t0 = clock64();
                    while (ld_acquire_u64(bar) < target) {
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
            }
            s_ok = ok;
            if (trace && tracer) {
                const unsigned long long k = sc->trace_n;
                if (k < (unsigned long long)trace_cap) {
                    trace[2 * k] = where;
                    trace[2 * k + 1] = global_ns();
                    sc->trace_n = k + 1;
                }
            }
        }
        __syncthreads();
        if (cl > 1) {
            // The blocks of a cluster take one decision: after a timed-out
            // wait some blocks may see the barrier complete and others the
            // error word, and a block that went on into a cluster solve
            // would wait at a cluster barrier for one that has left.
            namespace cg = cooperative_groups;
            cg::cluster_group clu = cg::this_cluster();
            __shared__ int s_oks[16];
            if (threadIdx.x == 0)
                clu.map_shared_rank(s_oks, 0)[clu.block_rank()] = s_ok;
            clu.sync();
            if (threadIdx.x == 0) {
                const int *all = clu.map_shared_rank(s_oks, 0);
                int ok = 1;
                for (int b = 0; b < cl; ++b) ok &= all[b] != 0;
                s_ok = ok;
            }
            clu.sync();  // s_oks is rewritten at the next barrier
        }
        return s_ok != 0;
    }
};

using qsmg::Thr;
// The first index of this thread in the grid-wide loops
// `for (i = t0; i < count; i += nt)`.  Runs of 32 consecutive indices go to
// the blocks in turn (run w * nblk + b to warp w of block b), so that a loop
// shorter than the launch (a coarse level, a 64^2 grid, the cells of a small
// grid) still spreads over every SM, while each warp's accesses stay
// contiguous.  float64 work is throughput-bound on GB300 (about two FMA per
// clock per SM): the same loop on the first few blocks alone took several
// times longer.  t0 ranges over a permutation of [0, nt) (blockDim.x is a
// multiple of 32), so every index is visited exactly once.
__device__ __forceinline__ Thr grid_thr(int bid, int nblk) {
    const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    return Thr{((w * nblk + bid) << 5) + lane, nblk * (int)blockDim.x};
}

// sum over the block; valid in thread 0
__device__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}
// four float32 sums over the block in one pass (one block barrier); valid in
// thread 0
__device__ void block_sum4f(float v[4]) {
    __shared__ float red4[32][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) red4[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float t = lane < nw ? red4[lane][k] : 0.f;
            for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            v[k] = t;
        }
    }
    __syncthreads();  // red4 is reused by the next call
}

__device__ double block_max(double v) {
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
    }
    return t;
}

// ---------------------------------------------------------------------------
// multigrid solves (1 or 2 components sharing the operator)
// ---------------------------------------------------------------------------
using qsmg::Hier;
using qsmg::Lvl;

struct SolveSpec {
    int nc;
    int kind;  // 0 psi, 1 (Ez,Bz), 2 (Bx,By): index into fnorm / vcycles
    double *u[2];
    double *f[2];
    bool screened;
    float *u32[2] = {nullptr, nullptr};  // refined form: float32 copy of the solution
};

// The hierarchy descriptors live in shared memory, one copy per block:
// thread l fills level l (a per-thread copy indexed by level would sit in
// local memory and be re-read from L1/L2 on every access).
__device__ void hier64(const EngineArgs &A, const SolveSpec &V, Hier<double> &H) {
    H.L = A.nlev;
    for (int l = threadIdx.x; l < A.nlev; l += blockDim.x) {
        Lvl<double> &v = H.lv[l];
        v.n = A.lev_n[l];
        v.h2 = A.lev_h2[l];
        v.inv_h2 = A.lev_inv_h2[l];
        v.h2t = A.lev_h2[l];
        v.inv_h2t = A.lev_inv_h2[l];
        v.omega = A.omega;
        for (int c = 0; c < 2; ++c) {
            v.u[c] = l == 0 ? V.u[c] : A.lev[l].u[c];
            v.f[c] = l == 0 ? V.f[c] : A.lev[l].f[c];
        }
        v.k = V.screened ? (l == 0 ? A.kap : A.lev[l].kap) : nullptr;
        v.d = V.screened ? (l == 0 ? A.invd0 : A.lev[l].d) : nullptr;
    }
}

__device__ void hier32(const EngineArgs &A, const SolveSpec &V, Hier<float> &H) {
    H.L = A.nlev;
    for (int l = threadIdx.x; l < A.nlev; l += blockDim.x) {
        Lvl<float> &v = H.lv[l];
        v.n = A.lev_n[l];
        v.h2 = A.lev_h2[l];
        v.inv_h2 = A.lev_inv_h2[l];
        v.h2t = A.lev_h2f[l];
        v.inv_h2t = A.lev_inv_h2f[l];
        v.omega = (float)A.omega;
        for (int c = 0; c < 2; ++c) {
            v.u[c] = l == 0 ? A.e32[c] : A.lev32[l].u[c];
            v.f[c] = l == 0 ? A.r32[0][c] : A.lev32[l].f[c];
        }
        v.k = V.screened ? (l == 0 ? A.k32 : A.lev32[l].k) : nullptr;
        v.d = V.screened ? (l == 0 ? A.d32 : A.lev32[l].d) : nullptr;
    }
}

// Level-0 red-black half sweep of the float32 correction that also adds the
// final correction into the float64 iterate: u64 += e at the points this
// thread updates and at the points of the other colour (not written here).
template <int NC>
__device__ void relax_half_finalize(const Lvl<float> L, int color, Thr R, double *fin0,
                                    double *fin1) {
    const int n = L.n;
    const float h2 = L.h2t;
    float *const u0 = L.u[0];
    float *const u1 = L.u[NC - 1];
    const float *const f0 = L.f[0];
    const float *const f1 = L.f[NC - 1];
    const int npts = n * n;
    for (qsmg::Walk w(R.t0, R.nt, n); w.q < npts; w.next()) {
        const int ix = w.col, iy = w.row;
        const int i = w.q;
        if (((ix + iy) & 1) == color) {
            const float di = L.d ? L.d[i] : qsmg::const_inv_diag<float>(qsmg::walls(ix, iy, n));
            qsmg::gs_point<float, NC>(u0, u1, f0, f1, h2, di, L.omega, n, ix, iy);
        }
        fin0[i] += (double)u0[i];
        if (NC > 1) fin1[i] += (double)u1[i];
    }
}

// One V-cycle on hierarchy H.  Levels of side > block_level_n are relaxed by
// the whole grid, the rest by block 0 in shared memory.  With `fin0` set (the
// refined form) the float32 correction is added into the float64 iterate
// during the last level-0 phase.
template <typename T, int NC>
__device__ bool vcycle(const EngineArgs &A, const Sync &S, const Hier<T> &H, int bid, int nblk,
                       void *smem, qsmg::CoarseInv ci, double *fin0, double *fin1) {
    const int L = H.L;
    int lg = 0;
    while (lg < L - 1 && H.lv[lg].n > A.block_level_n) ++lg;
    const Thr T0 = grid_thr(bid, nblk);
    for (int l = 0; l < lg; ++l) {
        const Lvl<T> F = H.lv[l], C = H.lv[l + 1];
        for (int s = 0; s < A.nu1; ++s) {
            qsmg::relax_half<T, NC>(F, 0, T0);
            SYNC(10);
            qsmg::relax_half<T, NC>(F, 1, T0);
            SYNC(11);
        }
        qsmg::restrict_res<T, NC>(F, C, T0);
        SYNC(12);
    }
    if (bid == 0) qsmg::block_vcycle<T, NC>(H, lg, A.nu1c, A.nu2, smem, ci);
    SYNC(13);
    if constexpr (sizeof(T) == 4) {
        if (fin0 && (lg == 0 || A.nu2 == 0)) {
            // no fused level-0 sweep: add the correction in a phase of its own
            for (int l = lg - 1; l >= 0; --l) {
                qsmg::prolong_add<T, NC>(H.lv[l], H.lv[l + 1], T0);
                SYNC(14);
            }
            const int nn = H.lv[0].n * H.lv[0].n;
            const float *e0 = H.lv[0].u[0];
            const float *e1 = H.lv[0].u[NC - 1];
            for (int q = T0.t0; q < nn; q += T0.nt) {
                fin0[q] += (double)e0[q];
                if (NC > 1) fin1[q] += (double)e1[q];
            }
            SYNC(17);
            return true;
        }
    }
    for (int l = lg - 1; l >= 0; --l) {
        const Lvl<T> F = H.lv[l], C = H.lv[l + 1];
        qsmg::prolong_add<T, NC>(F, C, T0);
        SYNC(14);
        for (int s = 0; s < A.nu2; ++s) {
            qsmg::relax_half<T, NC>(F, 0, T0);
            SYNC(15);
            if constexpr (sizeof(T) == 4) {
                if (fin0 && l == 0 && s == A.nu2 - 1) {
                    relax_half_finalize<NC>(F, 1, T0, fin0, fin1);
                    SYNC(16);
                    continue;
                }
            }
            qsmg::relax_half<T, NC>(F, 1, T0);
            SYNC(16);
        }
    }
    return true;
}

// Output tile of a staged level of side n: the configured tile, halved
// (the longer side first, down to 8) while the level has fewer than nblk/2
// tiles, so that coarser grid-wide levels still spread over the blocks and
// each block's region stays small.
__device__ __forceinline__ void level_tile(const EngineArgs &A, int n, int nblk, int &TX,
                                           int &TY) {
    TX = A.tile_x;
    TY = A.tile_y;
    for (;;) {
        const int tiles = ((n + TX - 1) / TX) * ((n + TY - 1) / TY);
        if (2 * tiles >= nblk) break;
        if (TX >= TY && TX > 8) TX >>= 1;
        else if (TY > 8) TY >>= 1;
        else break;
    }
}

// Refined form: one float32 V-cycle on the correction.  The grid-wide levels
// are staged tile by tile on the way down (one grid barrier per level);
// every block then solves the coarse levels itself in shared memory (no
// barrier); one phase runs every up leg and the level-0 update of the
// float64 iterate u and residual r (r <- r - A e) and accumulates ||r||^2,
// ||u||^2 into norms_out (the slot of the convergence test).
// *fused_done reports whether that happened: grids too small to stage fall
// back to the plain cycle, which leaves the residual to a separate pass.
template <int NC>
__device__ bool vcycle_staged(const EngineArgs &A, const Sync &S, const Hier<float> &H, int bid,
                              int nblk, void *smem, qsmg::CoarseInv ci, double *fin0,
                              double *fin1, const qstile::Fused *fused, double *norms_out,
                              double *norms_clear, bool *fused_done) {
    const int L = H.L;
    int lg = 0;
    while (lg < L - 1 && H.lv[lg].n > A.block_level_n) ++lg;
    *fused_done = false;
    if (lg == 0) return vcycle<float, NC>(A, S, H, bid, nblk, smem, ci, fin0, fin1);
    // shared memory: the coarse part's levels first, the staged tile after them
    float *sm = (float *)((char *)smem + A.tile_smem_offset);
    const qsmg::Marks mk{bid == 0 ? A.trace : nullptr, &A.sc->trace_n, A.trace_cap};
    for (int l = 0; l < lg; ++l) {
        int TX, TY;
        level_tile(A, H.lv[l].n, nblk, TX, TY);
        // the correction starts from zero; its pre-smoothed tile goes to
        // the level's own array (the up cascade reads it there)
        qstile::down_level<float, NC>(H.lv[l], H.lv[l + 1], A.nu1, TX, TY, sm, bid, nblk,
                                      H.lv[l].u, nullptr, mk);
        mk(62);
        SYNC(30);
    }
    qsmg::block_vcycle<float, NC>(H, lg, A.nu1c, A.nu2, smem, ci, false, mk);
    const int mg2 = H.lv[lg].n * H.lv[lg].n;
    // every up leg and the level-0 update in one phase
    int TX, TY;
    level_tile(A, H.lv[0].n, nblk, TX, TY);
    // ||r||^2, ||u||^2 of the tile in float32: the stopping test needs a
    // few digits of them
    float nrm[4] = {0.f, 0.f, 0.f, 0.f};
    qstile::up_cascade_fused<NC>(H, lg, (const float *)smem, (const float *)smem + 2 * mg2,
                                 A.nu2, TX, TY, sm, bid, nblk, *fused, nrm, mk);
    block_sum4f(nrm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            atomicAdd(norms_out + c, (double)nrm[c]);
            atomicAdd(norms_out + 2 + c, (double)nrm[2 + c]);
        }
    if (bid == 0 && threadIdx.x == 0)
        for (int e = 0; e < 4; ++e) norms_clear[e] = 0.0;
    mk(67);
    *fused_done = true;
    SYNC(32);
    return true;
}

// Float64 form: one V-cycle with the grid-wide levels staged tile by tile
// (qs_tile.cuh): a down leg per level (pre-sweeps from the iterate at level
// 0, from zero below, residual, restriction; the pre-smoothed tile to the
// level's scratch pair), the coarse levels by block 0, an up leg per level
// (prolongation, post-sweeps) reading the scratch pair; the level-0 up leg
// also sums ||f - A u||^2 and ||u||^2 of its tile into norms_out for the
// stopping test.  One grid barrier per level and leg instead of one per
// colour sweep, restriction and prolongation.
template <int NC>
__device__ bool vcycle_staged64(const EngineArgs &A, const Sync &S, const Hier<double> &H,
                                int bid, int nblk, void *smem, qsmg::CoarseInv ci,
                                double *norms_out, double *norms_clear) {
    const int L = H.L;
    int lg = 0;
    while (lg < L - 1 && H.lv[lg].n > A.block_level_n) ++lg;
    double *sm = (double *)((char *)smem + A.tile_smem_offset);
    for (int l = 0; l < lg; ++l) {
        int TX, TY;
        level_tile(A, H.lv[l].n, nblk, TX, TY);
        qstile::down_level<double, NC>(H.lv[l], H.lv[l + 1], A.nu1, TX, TY, sm, bid, nblk,
                                       A.lev[l].s, l == 0 ? H.lv[0].u : nullptr);
        SYNC(40);
    }
    if (bid == 0) qsmg::block_vcycle<double, NC>(H, lg, A.nu1c, A.nu2, smem, ci);
    SYNC(41);
    double nrm[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = lg - 1; l >= 0; --l) {
        int TX, TY;
        level_tile(A, H.lv[l].n, nblk, TX, TY);
        qstile::up_level<double, NC>(H.lv[l], H.lv[l + 1], A.lev[l].s, A.nu2, TX, TY, sm, bid,
                                     nblk, l == 0, nrm);
        if (l > 0) SYNC(42);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double t = block_sum(nrm[k]);
        if (threadIdx.x == 0 && (k & 1) < NC) atomicAdd(norms_out + k, t);
    }
    if (bid == 0 && threadIdx.x == 0)
        for (int e = 0; e < 4; ++e) norms_clear[e] = 0.0;
    SYNC(43);
    return true;
}

// ||f - A u||^2 and ||u||^2 per component at level 0 in float64, accumulated
// into out[c] and out[2 + c].  For the refined form the residual also becomes
// the float32 right-hand side of the next inner cycle, whose correction
// starts at zero.
template <int NC>
__device__ void residual_norm(const EngineArgs &A, const SolveSpec &V, double *out, Thr T,
                              bool to32, float *const *r32) {
    const int n = A.N;
    const double inv_h2 = A.lev_inv_h2[0];
    const double *const kap = V.screened ? A.kap : nullptr;
    const double *const u0 = V.u[0];
    const double *const u1 = V.u[NC - 1];
    const double *const f0 = V.f[0];
    const double *const f1 = V.f[NC - 1];
    float *const r0 = r32[0];
    float *const r1 = r32[NC - 1];
    float *const e0 = A.e32[0];
    float *const e1 = A.e32[NC - 1];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (qsmg::Walk w(T.t0, T.nt, n); w.q < n * n; w.next()) {
        const int k = w.q;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double *u = c ? u1 : u0;
            const double r = (c ? f1 : f0)[k] - qsmg::apply_op<double>(u, kap, n, inv_h2, w.col, w.row);
            s[c] += r * r;
            s[2 + c] += u[k] * u[k];
            if (to32) {
                (c ? r1 : r0)[k] = (float)r;
                (c ? e1 : e0)[k] = 0.f;
                A.r64[c][k] = r;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double t = block_sum(s[c]);
        if (threadIdx.x == 0) atomicAdd(out + c, t);
        t = block_sum(s[2 + c]);
        if (threadIdx.x == 0) atomicAdd(out + 2 + c, t);
    }
}

// ---------------------------------------------------------------------------
// V-cycles inside thread-block clusters (qs_cluster.cuh): one cluster per
// component, cluster k = blocks [k C, (k + 1) C) of the launch.
// ---------------------------------------------------------------------------

// The cluster's view of its hierarchy: distributed level l (l < Y.ld) and
// the local levels of block 0.
template <typename T>
struct ClusterView {
    void *cb;  // the cluster region of this block's shared memory
    const qsclu::Layout *Y;
    int rank, C;
    bool scr;
    __device__ qsclu::DLvl<T> dl(const EngineArgs &A, cooperative_groups::cluster_group &cl,
                                 int l) const {
        qsclu::DLvl<T> D;
        D.n = Y->n[l];
        D.R = Y->R[l];
        D.row0 = rank * D.R;
        D.u = qsclu::arr<T>(cb, *Y, l, 0);
        D.f = qsclu::arr<T>(cb, *Y, l, 1);
        D.k = scr ? qsclu::arr<T>(cb, *Y, l, 2) : nullptr;
        D.d = scr ? qsclu::arr<T>(cb, *Y, l, 3) : nullptr;
        D.up_u = rank > 0 ? cl.map_shared_rank(D.u, rank - 1) : nullptr;
        D.dn_u = rank < C - 1 ? cl.map_shared_rank(D.u, rank + 1) : nullptr;
        D.h2 = (T)A.lev_h2[l];
        D.inv_h2 = (T)A.lev_inv_h2[l];
        D.omega = (T)A.omega;
        return D;
    }
    __device__ Lvl<T> lv(const EngineArgs &A, int l) const {
        Lvl<T> v;
        v.u[0] = v.u[1] = qsclu::arr<T>(cb, *Y, l, 0);
        v.f[0] = v.f[1] = qsclu::arr<T>(cb, *Y, l, 1);
        v.k = scr ? qsclu::arr<T>(cb, *Y, l, 2) : nullptr;
        v.d = scr ? qsclu::arr<T>(cb, *Y, l, 3) : nullptr;
        v.n = Y->n[l];
        v.h2 = A.lev_h2[l];
        v.inv_h2 = A.lev_inv_h2[l];
        v.h2t = (T)A.lev_h2[l];
        v.inv_h2t = (T)A.lev_inv_h2[l];
        v.omega = (T)A.omega;
        return v;
    }
};

// One V(nu1, nu2) cycle of the cluster's component on the hierarchy held in
// its shared memory (level 0's u and f already there).  with_k: restrict
// kappa too (the first cycle of a solve).
template <typename T>
__device__ void cluster_vcycle(const EngineArgs &A, cooperative_groups::cluster_group &cl,
                               const ClusterView<T> &V, qsmg::CoarseInv ci, bool with_k,
                               const qsmg::Marks &mk) {
    const qsclu::Layout &Y = *V.Y;
    const int ld = Y.ld, L = Y.L;
    for (int l = 0; l < ld; ++l) {
        const qsclu::DLvl<T> D = V.dl(A, cl, l);
        const int nu = D.n > A.block_level_n ? A.nu1 : A.nu1c;
        for (int s = 0; s < nu; ++s) {
            qsclu::d_relax<T>(D, 0);
            cl.sync();
            qsclu::d_relax<T>(D, 1);
            cl.sync();
        }
        const int m = Y.n[l + 1];
        T *cu, *cf, *ck = nullptr, *cd = nullptr;
        int crow0;
        if (l + 1 < ld) {  // into this block's strip of the next level
            cu = qsclu::arr<T>(V.cb, Y, l + 1, 0);
            cf = qsclu::arr<T>(V.cb, Y, l + 1, 1);
            if (V.scr) {
                ck = qsclu::arr<T>(V.cb, Y, l + 1, 2);
                cd = qsclu::arr<T>(V.cb, Y, l + 1, 3);
            }
            crow0 = D.row0 >> 1;
        } else {  // into block 0's whole first local level
            cu = cl.map_shared_rank(qsclu::arr<T>(V.cb, Y, ld, 0), 0);
            cf = cl.map_shared_rank(qsclu::arr<T>(V.cb, Y, ld, 1), 0);
            if (V.scr) {
                ck = cl.map_shared_rank(qsclu::arr<T>(V.cb, Y, ld, 2), 0);
                cd = cl.map_shared_rank(qsclu::arr<T>(V.cb, Y, ld, 3), 0);
            }
            crow0 = 0;
        }
        qsclu::d_restrict<T>(D, m, crow0, cu, cf, ck, cd, (T)A.lev_h2[l + 1], with_k);
        cl.sync();
        mk(71 + l);
    }
    if (V.rank == 0) {  // the local levels, all of block 0's warps
        const Thr B{(int)threadIdx.x, (int)blockDim.x};
        for (int l = ld; l < L - 1; ++l) {
            const Lvl<T> F = V.lv(A, l), Cc = V.lv(A, l + 1);
            const int nu = F.n > A.block_level_n ? A.nu1 : A.nu1c;
            for (int s = 0; s < nu; ++s) {
                qsmg::relax_half<T, 1>(F, 0, B);
                __syncthreads();
                qsmg::relax_half<T, 1>(F, 1, B);
                __syncthreads();
            }
            qsmg::restrict_res<T, 1>(F, Cc, B, with_k);
            __syncthreads();
        }
        qsmg::coarse_solve<T, 1>(V.lv(A, L - 1), (double *)((char *)V.cb + Y.work), ci);
        for (int l = L - 2; l >= ld; --l) {
            const Lvl<T> F = V.lv(A, l), Cc = V.lv(A, l + 1);
            qsmg::prolong_add<T, 1>(F, Cc, B);
            __syncthreads();
            for (int s = 0; s < A.nu2; ++s) {
                qsmg::relax_half<T, 1>(F, 0, B);
                __syncthreads();
                qsmg::relax_half<T, 1>(F, 1, B);
                __syncthreads();
            }
        }
    }
    cl.sync();
    mk(78);
    for (int l = ld - 1; l >= 0; --l) {
        const qsclu::DLvl<T> D = V.dl(A, cl, l);
        if (l + 1 == ld)
            qsclu::d_prolong_w<T>(D, cl.map_shared_rank(qsclu::arr<T>(V.cb, Y, ld, 0), 0),
                                  Y.n[ld]);
        else
            qsclu::d_prolong_d<T>(D, V.dl(A, cl, l + 1));
        cl.sync();
        for (int s = 0; s < A.nu2; ++s) {
            qsclu::d_relax<T>(D, 0);
            cl.sync();
            qsclu::d_relax<T>(D, 1);
            cl.sync();
        }
        mk(81 + l);
    }
}

// Float64 form: the solve of component bid / C by its cluster, to the grid
// path's stopping test; fn: ||f||^2 per component (thread 0).  Blocks of
// other clusters return at once; the caller's grid barrier follows.
__device__ __noinline__ void mg_solve_cluster64(const EngineArgs &A, const SolveSpec &V, int bid,
                                   void *smem_base, qsmg::CoarseInv ci, const double *fn) {
    namespace cg = cooperative_groups;
    const int C = A.cl_size, comp = bid / C;
    if (comp >= V.nc) return;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ qsclu::Layout Y;
    __shared__ int s_conv;
    __shared__ double s_rel;
    if (threadIdx.x == 0) Y = qsclu::cluster_layout(A.lev_n, A.nlev, C, sizeof(double));
    __syncthreads();
    const ClusterView<double> cv{(char *)smem_base + A.cl_smem_offset, &Y,
                                 (int)cl.block_rank(), C, V.screened};
    const double *const gu = V.u[comp];
    const double *const gf = V.f[comp];
    {  // level 0: this block's rows of the warm start, the source and kappa
        const qsclu::DLvl<double> D = cv.dl(A, cl, 0);
        const size_t g0 = (size_t)D.row0 * D.n;
        for (int q = threadIdx.x; q < D.R * D.n; q += blockDim.x) {
            D.u[q] = gu[g0 + q];
            D.f[q] = gf[g0 + q];
            if (cv.scr) {
                D.k[q] = A.kap[g0 + q];
                D.d[q] = A.invd0[g0 + q];
            }
        }
    }
    cl.sync();
    double *const slots0 = cl.map_shared_rank((double *)((char *)cv.cb + Y.slots), 0);
    const double fl = 1e-13 * A.lev_inv_h2[0];
    const qsmg::Marks mk{A.trace, &A.sc->trace_n, A.trace_cap};  // block 0, thread 0
    int it = 0;
    bool conv = false;
    for (;;) {
        if (it > 0) {  // ||f - A u||^2 and ||u||^2 of the component
            const qsclu::DLvl<double> D = cv.dl(A, cl, 0);
            double s[2] = {0.0, 0.0};
            for (int q = threadIdx.x; q < D.R * D.n; q += blockDim.x) {
                const int ly = q / D.n, x = q - ly * D.n;
                const double r = qsclu::d_res(D, x, D.row0 + ly, q);
                s[0] += r * r;
                s[1] += D.u[q] * D.u[q];
            }
            for (int e = 0; e < 2; ++e) {
                const double t = block_sum(s[e]);
                if (threadIdx.x == 0) slots0[cv.rank * 2 + e] = t;
            }
            cl.sync();
            __shared__ double s_tot[2];
            if (threadIdx.x < 32) {  // warp 0: one remote load per lane, then a warp sum
                for (int e = 0; e < 2; ++e) {
                    double v = 0.0;
                    for (int b = threadIdx.x; b < C; b += 32) v += slots0[b * 2 + e];
                    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if (threadIdx.x == 0) s_tot[e] = v;
                }
            }
            if (threadIdx.x == 0) {
                const double f2 = fn[comp];
                double thr = fmax(A.mg_tol * A.mg_tol * f2, A.mg_atol * A.mg_atol);
                thr = fmax(thr, fl * fl * s_tot[1]);
                s_conv = f2 == 0.0 || s_tot[0] <= thr;
                s_rel = f2 > 0.0 ? sqrt(s_tot[0] / f2) : 0.0;
            }
            __syncthreads();
            conv = s_conv != 0;
            mk(70);
            if (conv || it >= A.mg_max_vcycles) break;
        }
        cluster_vcycle<double>(A, cl, cv, ci, it == 0, mk);
        ++it;
    }
    {  // this block's rows of the solution
        const qsclu::DLvl<double> D = cv.dl(A, cl, 0);
        const size_t g0 = (size_t)D.row0 * D.n;
        double *const u = V.u[comp];
        for (int q = threadIdx.x; q < D.R * D.n; q += blockDim.x) u[g0 + q] = D.u[q];
    }
    if (cv.rank == 0 && threadIdx.x == 0) {
        DevScalars *sc = A.sc;
        atomicMax(&sc->cl_cycles, it);
        atomicMax((unsigned long long *)&sc->max_relres,
                  (unsigned long long)__double_as_longlong(s_rel));
        if (!conv) sc->not_converged = 1;
    }
    cl.sync();  // no block leaves while another may still read its shared memory
}

// Refined form, the cluster part of an outer iteration: the float32 V-cycle
// of the correction e (from zero) with the float32 residual as right-hand
// side, by the cluster of component bid / C; e is written to A.e32[comp].
__device__ __noinline__ void cluster_inner_cycle(const EngineArgs &A, const SolveSpec &V, int bid,
                                    void *smem_base, qsmg::CoarseInv ci, bool first) {
    namespace cg = cooperative_groups;
    const int C = A.cl_size, comp = bid / C;
    if (comp >= V.nc) return;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ qsclu::Layout Y;
    if (threadIdx.x == 0) Y = qsclu::cluster_layout(A.lev_n, A.nlev, C, sizeof(float));
    __syncthreads();
    const ClusterView<float> cv{(char *)smem_base + A.cl_smem_offset, &Y,
                                (int)cl.block_rank(), C, V.screened};
    const qsmg::Marks mk{A.trace, &A.sc->trace_n, A.trace_cap};
    {
        const qsclu::DLvl<float> D = cv.dl(A, cl, 0);
        const size_t g0 = (size_t)D.row0 * D.n;
        const float *const r = A.r32[0][comp];
        for (int q = threadIdx.x; q < D.R * D.n; q += blockDim.x) {
            D.u[q] = 0.f;
            D.f[q] = r[g0 + q];
            if (first && cv.scr) {  // kappa is fixed during a solve
                D.k[q] = A.k32[g0 + q];
                D.d[q] = A.d32[g0 + q];
            }
        }
    }
    cl.sync();
    cluster_vcycle<float>(A, cl, cv, ci, first, mk);
    {
        const qsclu::DLvl<float> D = cv.dl(A, cl, 0);
        const size_t g0 = (size_t)D.row0 * D.n;
        float *const e = A.e32[comp];
        for (int q = threadIdx.x; q < D.R * D.n; q += blockDim.x) e[g0 + q] = D.u[q];
    }
    cl.sync();
}

// Refined form, the grid-wide part of an outer iteration: in float64,
// u += e and r <- r - (lap_h - kappa) e (= f - A(u + e)), with the 5-point
// sum of the float32 e formed exactly as a float32 pair (error-free sums and
// an FMA product) before it is widened; r32 = (float) r for the next cycle;
// the float32 copy of u where asked; ||r||^2, ||u||^2 into norms_out.
template <int NC>
__device__ __noinline__ void update_from_e(const EngineArgs &A, const SolveSpec &V, Thr T,
                              double *norms_out) {
    const int n = A.N;
    const double inv_h2 = A.lev_inv_h2[0];
    const double *const kap = V.screened ? A.kap : nullptr;
    float nrm[4] = {0.f, 0.f, 0.f, 0.f};
    for (qsmg::Walk w(T.t0, T.nt, n); w.q < n * n; w.next()) {
        const int x = w.col, y = w.row, i = w.q;
        const float cw = (float)(4 + qsmg::walls(x, y, n));
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float *e = A.e32[c];
            const float ef = e[i];
            float hi = 0.f, lo = 0.f;
            if (x > 0) qstile::two_sum_acc(hi, lo, e[i - 1]);
            if (x < n - 1) qstile::two_sum_acc(hi, lo, e[i + 1]);
            if (y > 0) qstile::two_sum_acc(hi, lo, e[i - n]);
            if (y < n - 1) qstile::two_sum_acc(hi, lo, e[i + n]);
            const float pc = __fmul_rn(cw, ef);
            const float pe = __fmaf_rn(cw, ef, -pc);  // cw ef = pc + pe exactly
            qstile::two_sum_acc(hi, lo, -pc);
            lo = __fsub_rn(lo, pe);
            const double ec = (double)ef;
            double ae = ((double)hi + (double)lo) * inv_h2;
            if (kap) ae -= kap[i] * ec;
            const double u = V.u[c][i] + ec;
            const double r = A.r64[c][i] - ae;
            const float rf = (float)r, uf = (float)u;
            V.u[c][i] = u;
            A.r64[c][i] = r;
            A.r32[0][c][i] = rf;
            if (V.u32[c]) V.u32[c][i] = uf;
            nrm[c] = __fmaf_rn(rf, rf, nrm[c]);
            nrm[2 + c] = __fmaf_rn(uf, uf, nrm[2 + c]);
        }
    }
    block_sum4f(nrm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            atomicAdd(norms_out + c, (double)nrm[c]);
            atomicAdd(norms_out + 2 + c, (double)nrm[2 + c]);
        }
}

// Refined form in clusters: each outer iteration is one float32 V-cycle of
// the correction per component, by that component's cluster, then the
// float64 update of u and r by the whole grid (two grid barriers).  A
// separate function: inlined, its registers made the slice engine spill.
__device__ __noinline__ bool mg_solve_ref_cluster(const EngineArgs &A, const Sync &S,
                                                  const SolveSpec &V, int &slot, int bid,
                                                  int nblk, void *smem_base, qsmg::CoarseInv ci,
                                                  const double *s_fn) {
    DevScalars *sc = A.sc;
    const Thr T = grid_thr(bid, nblk);
    __shared__ int s_conv;
    // Refined form in clusters: each outer iteration is one float32
    // V-cycle of the correction per component, by that component's
    // cluster, then the float64 update of u and r by the whole grid.
    if (V.nc == 1) residual_norm<1>(A, V, sc->rnorm[slot & 3], T, true, A.r32[0]);
    else residual_norm<2>(A, V, sc->rnorm[slot & 3], T, true, A.r32[0]);
    if (bid == 0 && threadIdx.x == 0)
        for (int e = 0; e < 4; ++e) sc->rnorm[(slot + 2) & 3][e] = 0.0;
    SYNC(21);
    double rel = 0.0;
    int it = 0;
    bool conv = false;
    for (;;) {
        if (threadIdx.x == 0) {
            const double fl = 1e-13 * A.lev_inv_h2[0];
            int cv = 1;
            rel = 0.0;
            for (int c = 0; c < V.nc; ++c) {
                const double fn = s_fn[c];
                if (fn == 0.0) continue;
                const double rn = vload(&sc->rnorm[slot & 3][c]);
                const double un = vload(&sc->rnorm[slot & 3][2 + c]);
                double thr = fmax(A.mg_tol * A.mg_tol * fn, A.mg_atol * A.mg_atol);
                thr = fmax(thr, fl * fl * un);
                if (rn > thr) cv = 0;
                rel = fmax(rel, sqrt(rn / fn));
            }
            s_conv = cv;
        }
        __syncthreads();
        conv = s_conv != 0;
        __syncthreads();
        ++slot;
        if (conv || it >= A.mg_max_vcycles) break;
        cluster_inner_cycle(A, V, bid, smem_base, ci, it == 0);
        SYNC(24);
        if (V.nc == 1) update_from_e<1>(A, V, T, sc->rnorm[slot & 3]);
        else update_from_e<2>(A, V, T, sc->rnorm[slot & 3]);
        if (bid == 0 && threadIdx.x == 0)
            for (int e = 0; e < 4; ++e) sc->rnorm[(slot + 2) & 3][e] = 0.0;
        SYNC(25);
        ++it;
    }
    if (bid == 0 && threadIdx.x == 0) {
        sc->vcycles[V.kind] += it;
        if (rel > sc->max_relres) sc->max_relres = rel;
        if (!conv) sc->not_converged = 1;
    }
    if (V.u32[0] && it == 0) {  // converged at once: the float32 copy of u
        const int nn = A.N * A.N;
        for (int c = 0; c < V.nc; ++c)
            for (int k = T.t0; k < nn; k += T.nt) V.u32[c][k] = (float)V.u[c][k];
        SYNC(23);
    }
    return true;
}

// Iterate until, for every component,
//   ||f - A u|| <= max(tol ||f||, 1e-13 ||u|| / h^2, atol)
// (the second bound is a small multiple of the rounding level of the
// float64 residual; atol stops solves whose source is rounding noise).
// Float64 form: V-cycles on u.  Refined form: float64 residual, float32
// V-cycle on the correction, float64 update (iterative refinement).
template <bool REF>
__device__ bool mg_solve(const EngineArgs &A, const Sync &S, const SolveSpec &V, int &slot,
                         int bid, int nblk, void *smem_base, int *inv_ready) {
    DevScalars *sc = A.sc;
    // shared memory: [coarsest inverses][coarse levels + work][staged tile]
    void *smem = (char *)smem_base + A.block_smem_offset;
    const int mc = A.lev_n[A.nlev - 1] * A.lev_n[A.nlev - 1];
    const qsmg::CoarseInv ci{(double *)smem_base + (V.screened ? mc * mc : 0),
                             inv_ready + (V.screened ? 1 : 0)};
    if (V.screened) {  // kappa changed: the screened inverse must be rebuilt
        __syncthreads();
        if (threadIdx.x == 0) inv_ready[1] = 0;
        __syncthreads();
    }
    // The scalar bookkeeping of the solve (source norms, the convergence
    // test) is done by thread 0 alone and broadcast through shared memory:
    // float64 divides and square roots repeated by every thread would cost
    // microseconds on GB300's float64 pipe.
    __shared__ double s_fn[2];
    __shared__ int s_zero_mask, s_conv;
    __syncthreads();
    if (threadIdx.x == 0) {
        int mask = 0;
        for (int c = 0; c < V.nc; ++c) {
            s_fn[c] = vload(&sc->fnorm[V.kind][c]);
            if (s_fn[c] == 0.0) mask |= 1 << c;
        }
        s_zero_mask = mask;
    }
    __syncthreads();
    const int zero_mask = s_zero_mask;
    const Thr T = grid_thr(bid, nblk);
    if (zero_mask) {
        const int nn = A.N * A.N;
        for (int c = 0; c < V.nc; ++c)
            if (zero_mask & (1 << c))
                for (int k = T.t0; k < nn; k += T.nt) {
                    V.u[c][k] = 0.0;
                    if (V.u32[c]) V.u32[c][k] = 0.f;
                }
        SYNC(20);
    }
    if (zero_mask == (1 << V.nc) - 1) return true;
#ifndef QS_NO_CLUSTER_SOLVES
    if (!REF && A.cl_size > 1) {  // one cluster per component solves alone
        mg_solve_cluster64(A, V, bid, smem_base, ci, s_fn);
        SYNC(22);
        if (bid == 0 && threadIdx.x == 0) {
            A.sc->vcycles[V.kind] += A.sc->cl_cycles;
            A.sc->cl_cycles = 0;
        }
        return true;
    }
#endif
#ifndef QS_NO_CLUSTER_SOLVES
    if (REF && A.cl_size > 1)
        return mg_solve_ref_cluster(A, S, V, slot, bid, nblk, smem_base, ci, s_fn);
#endif
    __shared__ Hier<double> H64;
    __shared__ Hier<float> H32;
    __syncthreads();
    if (REF) hier32(A, V, H32);
    else hier64(A, V, H64);
    __syncthreads();
    bool conv = false;
    double rel = 0.0;  // thread 0 only
    int it = 0;
    bool norms_ready = false;  // the last cycle already produced this slot's norms
    // The fused residual update writes the next float32 right-hand side into
    // the other buffer of a pair: the current one is still read as halo by
    // other blocks while it is written.
    int rbuf = 0;
    bool u32_fresh = false;  // the last cycle wrote the float32 copy of u
    for (;;) {
        if (REF || it > 0) {
            if (!norms_ready) {
                if (V.nc == 1) residual_norm<1>(A, V, sc->rnorm[slot & 3], T, REF, H32.lv[0].f);
                else residual_norm<2>(A, V, sc->rnorm[slot & 3], T, REF, H32.lv[0].f);
                if (bid == 0 && threadIdx.x == 0)
                    for (int e = 0; e < 4; ++e) sc->rnorm[(slot + 2) & 3][e] = 0.0;
                SYNC(21);
            }
            if (threadIdx.x == 0) {
                const double fl = 1e-13 * A.lev_inv_h2[0];
                int cv = 1;
                rel = 0.0;
                for (int c = 0; c < V.nc; ++c) {
                    const double fn = s_fn[c];
                    if (fn == 0.0) continue;
                    const double rn = vload(&sc->rnorm[slot & 3][c]);
                    const double un = vload(&sc->rnorm[slot & 3][2 + c]);
                    double thr = fmax(A.mg_tol * A.mg_tol * fn, A.mg_atol * A.mg_atol);
                    thr = fmax(thr, fl * fl * un);
                    if (rn > thr) cv = 0;
                    rel = fmax(rel, sqrt(rn / fn));
                }
                s_conv = cv;
            }
            __syncthreads();
            conv = s_conv != 0;
            __syncthreads();  // s_conv is rewritten by the next test
            ++slot;
            if (conv || it >= A.mg_max_vcycles) break;
        }
        bool ok;
        norms_ready = false;
        if (REF) {
            const qstile::Fused fz{{V.u[0], V.u[V.nc - 1]},
                                   {A.r64[0], A.r64[V.nc - 1]},
                                   {A.r32[1 - rbuf][0], A.r32[1 - rbuf][V.nc - 1]},
                                   {V.u32[0], V.u32[V.nc - 1]},
                                   V.screened ? A.kap : nullptr,
                                   A.lev_inv_h2[0]};
            double *nout = sc->rnorm[slot & 3], *nclr = sc->rnorm[(slot + 2) & 3];
            if (V.nc == 1)
                ok = A.tile_x > 0
                         ? vcycle_staged<1>(A, S, H32, bid, nblk, smem, ci, V.u[0], V.u[0], &fz,
                                            nout, nclr, &norms_ready)
                         : vcycle<float, 1>(A, S, H32, bid, nblk, smem, ci, V.u[0], V.u[0]);
            else
                ok = A.tile_x > 0
                         ? vcycle_staged<2>(A, S, H32, bid, nblk, smem, ci, V.u[0], V.u[1], &fz,
                                            nout, nclr, &norms_ready)
                         : vcycle<float, 2>(A, S, H32, bid, nblk, smem, ci, V.u[0], V.u[1]);
        } else if (A.tile_x > 0 && H64.lv[0].n > A.block_level_n) {
            double *nout = sc->rnorm[slot & 3], *nclr = sc->rnorm[(slot + 2) & 3];
            ok = V.nc == 1 ? vcycle_staged64<1>(A, S, H64, bid, nblk, smem, ci, nout, nclr)
                           : vcycle_staged64<2>(A, S, H64, bid, nblk, smem, ci, nout, nclr);
            norms_ready = true;  // the level-0 up leg summed the stopping test's norms
        } else {
            ok = V.nc == 1 ? vcycle<double, 1>(A, S, H64, bid, nblk, smem, ci, nullptr, nullptr)
                           : vcycle<double, 2>(A, S, H64, bid, nblk, smem, ci, nullptr, nullptr);
        }
        if (!ok) return false;
        u32_fresh = REF && norms_ready;
        if (REF && norms_ready) {  // all blocks are past the cycle's last barrier
            rbuf ^= 1;
            if (threadIdx.x == 0)
                for (int c = 0; c < 2; ++c) H32.lv[0].f[c] = A.r32[rbuf][c];
            __syncthreads();
        }
        ++it;
    }
    if (bid == 0 && threadIdx.x == 0) {
        sc->vcycles[V.kind] += it;
        if (rel > sc->max_relres) sc->max_relres = rel;
        if (!conv) sc->not_converged = 1;
    }
    if (V.u32[0] && !u32_fresh) {  // no cycle, or a cycle without the fused update
        const int nn = A.N * A.N;
        for (int c = 0; c < V.nc; ++c)
            for (int k = T.t0; k < nn; k += T.nt) V.u32[c][k] = (float)V.u[c][k];
        SYNC(23);
    }
    return true;
}

__device__ __forceinline__ double guard(double a, double floor_, unsigned &hits) {
    if (a < floor_) {
        ++hits;
        return floor_;
    }
    return a;
}

__device__ void add_hits(DevScalars *sc, unsigned hits) {
    double t = block_sum((double)hits);
    if (threadIdx.x == 0 && t > 0.0) atomicAdd(&sc->guard_hits, (unsigned long long)t);
}

}  // namespace
