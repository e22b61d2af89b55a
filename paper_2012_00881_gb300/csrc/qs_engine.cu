// The slice engine: one persistent cooperative kernel runs the whole xi loop
// of Algorithm 1 (Collect_Source, Solve_Wakefield, Push_Trajectory,
// Step_Size_Refinement) for one 3D step.  Phases are separated by a grid
// barrier whose waits are bounded in time; a timed-out wait records
// QS_ERR_TIMEOUT and every block leaves the kernel at its next barrier.
//
// Float64 form.  Multigrid: red-black Gauss-Seidel V(nu1, nu2) cycles,
// full-weighting (4-cell average) restriction of the residual, bilinear
// prolongation, rediscretised coarse operators (kappa averaged), dense
// Gaussian elimination on the coarsest grid (side <= 8).  Levels whose side
// is at most block_level_n are relaxed by block 0 alone.
#include <cuda_runtime.h>

#include "qs_internal.cuh"

namespace {

#define SYNC(where)                 \
    do {                            \
        if (!S(where)) return false; \
    } while (0)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ double vload(const double *p) { return *(const volatile double *)p; }
__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
struct Sync {
    DevScalars *sc;
    unsigned nblk;
    long long limit;
    __device__ bool operator()(int where) const {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            if (vload(&sc->err) != 0) {
                ok = 0;
            } else {
                unsigned gen = ld_acquire_u32(&sc->bar_gen);
                __threadfence();
                unsigned arrived = atomicAdd(&sc->bar_count, 1u);
                if (arrived == nblk - 1) {
                    atomicExch(&sc->bar_count, 0u);
                    __threadfence();
                    atomicAdd(&sc->bar_gen, 1u);
                } else {
                    long long t0 = clock64();
                    while (ld_acquire_u32(&sc->bar_gen) == gen) {
                        if (vload(&sc->err) != 0) {
                            ok = 0;
                            break;
                        }
                        if (clock64() - t0 > limit) {
                            if (atomicCAS(&sc->err, 0, QS_ERR_TIMEOUT) == 0) sc->err_where = where;
                            ok = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                __threadfence();
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

struct Thr {
    int t0, nt;
};
__device__ __forceinline__ Thr grid_thr(int bid, int nblk) {
    return Thr{bid * (int)blockDim.x + (int)threadIdx.x, nblk * (int)blockDim.x};
}
__device__ __forceinline__ Thr block_thr() { return Thr{(int)threadIdx.x, (int)blockDim.x}; }

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
// multigrid on one solve (1 or 2 components sharing the operator)
// ---------------------------------------------------------------------------
struct SolveView {
    int ncomp;
    int kind;  // 0 psi, 1 (Ez,Bz), 2 (Bx,By): index into fnorm / vcycles
    double *u0[2];
    double *f0[2];
    double *k0;  // kappa at level 0, nullptr for the Poisson operator
};

__device__ __forceinline__ double *Ul(const EngineArgs &A, const SolveView &V, int l, int c) {
    return l == 0 ? V.u0[c] : A.lev[l].u[c];
}
__device__ __forceinline__ double *Fl(const EngineArgs &A, const SolveView &V, int l, int c) {
    return l == 0 ? V.f0[c] : A.lev[l].f[c];
}
__device__ __forceinline__ const double *Kl(const EngineArgs &A, const SolveView &V, int l) {
    if (!V.k0) return nullptr;
    return l == 0 ? V.k0 : A.lev[l].kap;
}

// (lap_h - kappa) u at (ix, iy) with odd (zero-wall) ghosts
__device__ __forceinline__ double apply_op(const double *u, const double *kap, int n,
                                           double inv_h2, int ix, int iy) {
    int i = iy * n + ix;
    double uc = u[i];
    double nb = 0.0;
    int nw = 0;
    if (ix > 0) nb += u[i - 1]; else ++nw;
    if (ix < n - 1) nb += u[i + 1]; else ++nw;
    if (iy > 0) nb += u[i - n]; else ++nw;
    if (iy < n - 1) nb += u[i + n]; else ++nw;
    double r = (nb - (4.0 + nw) * uc) * inv_h2;
    if (kap) r -= kap[i] * uc;
    return r;
}

__device__ void relax_half(const EngineArgs &A, const SolveView &V, int l, int color, Thr T) {
    const int n = A.lev_n[l];
    const double h2 = A.lev_h2[l];
    const double *kap = Kl(A, V, l);
    const int npts = (n & 1) ? n * n : (n * n) / 2;
    const int hn = n >> 1;
    for (int k = T.t0; k < npts; k += T.nt) {
        int ix, iy;
        if (n & 1) {
            iy = k / n;
            ix = k - iy * n;
            if (((ix + iy) & 1) != color) continue;
        } else {
            iy = k / hn;
            ix = 2 * (k - iy * hn) + ((iy + color) & 1);
        }
        const int i = iy * n + ix;
        int nw = (ix == 0) + (ix == n - 1) + (iy == 0) + (iy == n - 1);
        double d = 4.0 + nw + (kap ? h2 * kap[i] : 0.0);
        double inv_d = 1.0 / d;
        for (int c = 0; c < V.ncomp; ++c) {
            double *u = Ul(A, V, l, c);
            const double *f = Fl(A, V, l, c);
            double nb = 0.0;
            if (ix > 0) nb += u[i - 1];
            if (ix < n - 1) nb += u[i + 1];
            if (iy > 0) nb += u[i - n];
            if (iy < n - 1) nb += u[i + n];
            u[i] = (nb - h2 * f[i]) * inv_d;
        }
    }
}

// f_{l+1} = 4-cell average of (f - A u) at level l; u_{l+1} = 0; for the
// screened operator also kappa_{l+1} = 4-cell average of kappa_l
__device__ void restrict_residual(const EngineArgs &A, const SolveView &V, int l, Thr T) {
    const int n = A.lev_n[l], nc = A.lev_n[l + 1];
    const double inv_h2 = 1.0 / A.lev_h2[l];
    const double *kap = Kl(A, V, l);
    for (int k = T.t0; k < nc * nc; k += T.nt) {
        const int J = k / nc, I = k - J * nc;
        for (int c = 0; c < V.ncomp; ++c) {
            const double *u = Ul(A, V, l, c);
            const double *f = Fl(A, V, l, c);
            double s = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int ix = 2 * I + a, iy = 2 * J + b;
                    s += f[iy * n + ix] - apply_op(u, kap, n, inv_h2, ix, iy);
                }
            Fl(A, V, l + 1, c)[k] = 0.25 * s;
            Ul(A, V, l + 1, c)[k] = 0.0;
        }
        if (kap) {  // coarse kappa: average of the four children
            const int i0 = (2 * J) * n + 2 * I;
            A.lev[l + 1].kap[k] = 0.25 * (kap[i0] + kap[i0 + 1] + kap[i0 + n] + kap[i0 + n + 1]);
        }
    }
}

// u_l += bilinear interpolation of u_{l+1} (cell-centred, odd ghosts)
__device__ void prolong_correct(const EngineArgs &A, const SolveView &V, int l, Thr T) {
    const int n = A.lev_n[l], nc = A.lev_n[l + 1];
    for (int k = T.t0; k < n * n; k += T.nt) {
        const int iy = k / n, ix = k - iy * n;
        const int I = ix >> 1, J = iy >> 1;
        const int I2 = I + ((ix & 1) ? 1 : -1);
        const int J2 = J + ((iy & 1) ? 1 : -1);
        const bool xin = (I2 >= 0 && I2 < nc), yin = (J2 >= 0 && J2 < nc);
        for (int c = 0; c < V.ncomp; ++c) {
            const double *uc = Ul(A, V, l + 1, c);
            double v00 = uc[J * nc + I];
            double v10 = xin ? uc[J * nc + I2] : -v00;
            double v01 = yin ? uc[J2 * nc + I] : -v00;
            double v11;
            if (xin && yin) v11 = uc[J2 * nc + I2];
            else if (xin) v11 = -uc[J * nc + I2];
            else if (yin) v11 = -uc[J2 * nc + I];
            else v11 = v00;
            Ul(A, V, l, c)[k] += (9.0 * v00 + 3.0 * v10 + 3.0 * v01 + v11) * 0.0625;
        }
    }
}

// Dense solve on the coarsest level by block 0: Gaussian elimination of the
// symmetric positive definite matrix -(lap_h - kappa), no pivoting needed.
__device__ void coarse_solve(const EngineArgs &A, const SolveView &V, double *sm) {
    const int l = A.nlev - 1;
    const int n = A.lev_n[l], m = n * n, nc = V.ncomp;
    const int ld = m + 2;
    const double inv_h2 = 1.0 / A.lev_h2[l];
    const double *kap = Kl(A, V, l);
    double *fac = sm + m * ld;  // m factors
    for (int idx = threadIdx.x; idx < m * ld; idx += blockDim.x) sm[idx] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int iy = i / n, ix = i - iy * n;
        int nw = (ix == 0) + (ix == n - 1) + (iy == 0) + (iy == n - 1);
        sm[i * ld + i] = (4.0 + nw) * inv_h2 + (kap ? kap[i] : 0.0);
        if (ix > 0) sm[i * ld + i - 1] = -inv_h2;
        if (ix < n - 1) sm[i * ld + i + 1] = -inv_h2;
        if (iy > 0) sm[i * ld + i - n] = -inv_h2;
        if (iy < n - 1) sm[i * ld + i + n] = -inv_h2;
        for (int c = 0; c < nc; ++c) sm[i * ld + m + c] = -Fl(A, V, l, c)[i];
    }
    __syncthreads();
    const int ncol = m + nc;
    for (int k = 0; k < m - 1; ++k) {
        const double piv = sm[k * ld + k];
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) fac[i] = sm[i * ld + k] / piv;
        __syncthreads();
        const int rows = m - k - 1, cols = ncol - k;
        for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
            const int i = k + 1 + e / cols, j = k + e % cols;
            sm[i * ld + j] -= fac[i] * sm[k * ld + j];
        }
        __syncthreads();
    }
    if ((int)threadIdx.x < nc) {
        const int c = threadIdx.x;
        double *u = Ul(A, V, l, c);
        for (int i = m - 1; i >= 0; --i) {
            double s = sm[i * ld + m + c];
            for (int j = i + 1; j < m; ++j) s -= sm[i * ld + j] * u[j];
            u[i] = s / sm[i * ld + i];
        }
    }
    __syncthreads();
}

__device__ bool vcycle(const EngineArgs &A, const Sync &S, const SolveView &V, int bid, int nblk,
                       double *sm) {
    const int L = A.nlev;
    int lg = 0;
    while (lg < L - 1 && A.lev_n[lg] > A.block_level_n) ++lg;
    const Thr T = grid_thr(bid, nblk);
    for (int l = 0; l < lg; ++l) {
        for (int s = 0; s < A.nu1; ++s) {
            relax_half(A, V, l, 0, T);
            SYNC(10);
            relax_half(A, V, l, 1, T);
            SYNC(11);
        }
        restrict_residual(A, V, l, T);
        SYNC(12);
    }
    if (bid == 0) {
        const Thr B = block_thr();
        for (int l = lg; l < L - 1; ++l) {
            for (int s = 0; s < A.nu1; ++s) {
                relax_half(A, V, l, 0, B);
                __syncthreads();
                relax_half(A, V, l, 1, B);
                __syncthreads();
            }
            restrict_residual(A, V, l, B);
            __syncthreads();
        }
        coarse_solve(A, V, sm);
        for (int l = L - 2; l >= lg; --l) {
            prolong_correct(A, V, l, B);
            __syncthreads();
            for (int s = 0; s < A.nu2; ++s) {
                relax_half(A, V, l, 0, B);
                __syncthreads();
                relax_half(A, V, l, 1, B);
                __syncthreads();
            }
        }
    }
    SYNC(13);
    for (int l = lg - 1; l >= 0; --l) {
        prolong_correct(A, V, l, T);
        SYNC(14);
        for (int s = 0; s < A.nu2; ++s) {
            relax_half(A, V, l, 0, T);
            SYNC(15);
            relax_half(A, V, l, 1, T);
            SYNC(16);
        }
    }
    return true;
}

// ||f - A u||^2 and ||u||^2 per component at level 0, accumulated into
// out[c] and out[2 + c]
__device__ void residual_norm(const EngineArgs &A, const SolveView &V, double *out, Thr T) {
    const int n = A.lev_n[0];
    const double inv_h2 = 1.0 / A.lev_h2[0];
    const double *kap = Kl(A, V, 0);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = T.t0; k < n * n; k += T.nt) {
        const int iy = k / n, ix = k - iy * n;
        for (int c = 0; c < V.ncomp; ++c) {
            const double r = V.f0[c][k] - apply_op(V.u0[c], kap, n, inv_h2, ix, iy);
            const double u = V.u0[c][k];
            s[c] += r * r;
            s[2 + c] += u * u;
        }
    }
    for (int c = 0; c < V.ncomp; ++c) {
        double t = block_sum(s[c]);
        if (threadIdx.x == 0) atomicAdd(out + c, t);
        t = block_sum(s[2 + c]);
        if (threadIdx.x == 0) atomicAdd(out + 2 + c, t);
    }
}

// V-cycles until, for every component,
//   ||f - A u|| <= max(tol ||f||, 1e-13 ||u|| / h^2, atol)
// (the second bound is a small multiple of the rounding level of the
// residual itself; atol stops solves whose source is rounding noise).
__device__ bool mg_solve(const EngineArgs &A, const Sync &S, const SolveView &V, int &slot,
                         int bid, int nblk, double *sm) {
    DevScalars *sc = A.sc;
    double fn[2] = {0.0, 0.0};
    bool any_zero = false, all_zero = true;
    for (int c = 0; c < V.ncomp; ++c) {
        fn[c] = vload(&sc->fnorm[V.kind][c]);
        if (fn[c] == 0.0) any_zero = true;
        else all_zero = false;
    }
    const Thr T = grid_thr(bid, nblk);
    if (any_zero) {
        const int nn = A.N * A.N;
        for (int c = 0; c < V.ncomp; ++c)
            if (fn[c] == 0.0)
                for (int k = T.t0; k < nn; k += T.nt) V.u0[c][k] = 0.0;
        SYNC(20);
    }
    if (all_zero) return true;
    bool conv = false;
    double rel = 0.0;
    int it = 0;
    for (; it < A.mg_max_vcycles; ++it) {
        if (!vcycle(A, S, V, bid, nblk, sm)) return false;
        residual_norm(A, V, sc->rnorm[slot & 3], T);
        if (bid == 0 && threadIdx.x == 0)
            for (int e = 0; e < 4; ++e) sc->rnorm[(slot + 2) & 3][e] = 0.0;
        SYNC(21);
        conv = true;
        rel = 0.0;
        for (int c = 0; c < V.ncomp; ++c) {
            if (fn[c] == 0.0) continue;
            const double rn = vload(&sc->rnorm[slot & 3][c]);
            const double un = vload(&sc->rnorm[slot & 3][2 + c]);
            const double fl = 1e-13 / A.lev_h2[0];
            double thr = fmax(A.mg_tol * A.mg_tol * fn[c], A.mg_atol * A.mg_atol);
            thr = fmax(thr, fl * fl * un);
            if (rn > thr) conv = false;
            rel = fmax(rel, sqrt(rn / fn[c]));
        }
        ++slot;
        if (conv) break;
    }
    if (bid == 0 && threadIdx.x == 0) {
        sc->vcycles[V.kind] += (it < A.mg_max_vcycles) ? it + 1 : it;
        if (rel > sc->max_relres) sc->max_relres = rel;
        if (!conv) sc->not_converged = 1;
    }
    return true;
}

// ---------------------------------------------------------------------------
// particle and grid phases
// ---------------------------------------------------------------------------
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

// n_* of the initial particles
__device__ void phase_deposit_n(const EngineArgs &A, double *ng, Thr T) {
    const double s = A.inv_h * A.inv_h;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        Cic c = cic_stencil(A.x[p], A.y[p], A.x_min, A.y_min, A.h, A.N);
        cic_deposit(ng, c, A.w[p] * s);
    }
}

// f_psi = n_* - n_ion (Eq. EqM_N8_AA) and its norm; charge sum; clear the
// moment accumulators and the next-slice density buffer
__device__ void phase_psi_rhs(const EngineArgs &A, const double *ncur, double *nnext, bool base,
                              int j, Thr T) {
    const int nn = A.N * A.N;
    double s = 0.0, cs = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        double nv = ncur[i];
        double f = nv - A.n_ion[i];
        A.f_psi[i] = f;
        s += f * f;
        cs += nv;
        A.jx[i] = 0.0;
        A.jy[i] = 0.0;
        A.txx[i] = 0.0;
        A.txy[i] = 0.0;
        A.tyy[i] = 0.0;
        A.G[i] = 0.0;
        nnext[i] = 0.0;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[0][0], s);
    if (base) {
        cs = block_sum(cs);
        if (threadIdx.x == 0) atomicAdd(&A.diag_charge[j], cs * A.h * A.h);
    }
}

// gather psi at every particle; deposit j_perp, T, G (Eqs. Jr, FluxPres)
__device__ void phase_moments(const EngineArgs &A, Thr T) {
    const double s = A.inv_h * A.inv_h;
    unsigned hits = 0;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        Cic c = cic_stencil(A.x[p], A.y[p], A.x_min, A.y_min, A.h, A.N);
        double a = guard(1.0 + cic_gather(A.psi, c), A.psi_floor, hits);
        double px = A.px[p], py = A.py[p];
        double gam = (1.0 + px * px + py * py + a * a) / (2.0 * a);
        double vx = px / a, vy = py / a;
        double wq = A.w[p] * s;
        cic_deposit(A.jx, c, wq * vx);
        cic_deposit(A.jy, c, wq * vy);
        cic_deposit(A.txx, c, wq * vx * vx);
        cic_deposit(A.txy, c, wq * vx * vy);
        cic_deposit(A.tyy, c, wq * vy * vy);
        cic_deposit(A.G, c, wq * gam);
    }
    add_hits(A.sc, hits);
}

// central differences: zero ghosts (moments) and odd ghosts (fields)
__device__ __forceinline__ double dx0(const double *u, int n, int ix, int i, double inv2h) {
    double e = ix < n - 1 ? u[i + 1] : 0.0;
    double w = ix > 0 ? u[i - 1] : 0.0;
    return (e - w) * inv2h;
}
__device__ __forceinline__ double dy0(const double *u, int n, int iy, int i, double inv2h) {
    double s = iy < n - 1 ? u[i + n] : 0.0;
    double q = iy > 0 ? u[i - n] : 0.0;
    return (s - q) * inv2h;
}
__device__ __forceinline__ double dxo(const double *u, int n, int ix, int i, double inv2h) {
    double e = ix < n - 1 ? u[i + 1] : -u[i];
    double w = ix > 0 ? u[i - 1] : -u[i];
    return (e - w) * inv2h;
}
__device__ __forceinline__ double dyo(const double *u, int n, int iy, int i, double inv2h) {
    double s = iy < n - 1 ? u[i + n] : -u[i];
    double q = iy > 0 ? u[i - n] : -u[i];
    return (s - q) * inv2h;
}

// sources of E_z, B_z (Eqs. EqM_N8_A, Mag_z_A); j_z (Eq. Jr plus the
// driver), kappa = n_* / (1+psi), grad psi
__device__ void phase_assemble1(const EngineArgs &A, const double *ncur, int j, int q, int m,
                                Thr T) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    const double frac = (double)q / (double)m;
    const double *J0 = A.jzb + (size_t)j * nn;
    const double *J1 = (j + 1 < A.n_xi) ? A.jzb + (size_t)(j + 1) * nn : nullptr;
    unsigned hits = 0;
    double sez = 0.0, sbz = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        double fez = -(dx0(A.jx, n, ix, i, inv2h) + dy0(A.jy, n, iy, i, inv2h));
        double fbz = dx0(A.jy, n, ix, i, inv2h) - dy0(A.jx, n, iy, i, inv2h);
        A.f_ez[i] = fez;
        A.f_bz[i] = fbz;
        sez += fez * fez;
        sbz += fbz * fbz;
        double a = guard(1.0 + A.psi[i], A.psi_floor, hits);
        double jzb = q == 0 ? J0[i] : (1.0 - frac) * J0[i] + frac * (J1 ? J1[i] : 0.0);
        double nv = ncur[i];
        A.jz[i] = A.G[i] / a - nv + jzb;
        A.kap[i] = nv / a;
        A.dpx[i] = dxo(A.psi, n, ix, i, inv2h);
        A.dpy[i] = dyo(A.psi, n, iy, i, inv2h);
    }
    sez = block_sum(sez);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[1][0], sez);
    sbz = block_sum(sbz);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[1][1], sbz);
    add_hits(A.sc, hits);
}

// explicit source S of Eq. FluxCurr1_A; rhs of Eq. Main_Eq_A is -e_z x S =
// (S_y, -S_x)
__device__ void phase_assemble2(const EngineArgs &A, Thr T) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    double sbx = 0.0, sby = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        double a = 1.0 + A.psi[i];
        if (a < A.psi_floor) a = A.psi_floor;
        const double jx = A.jx[i], jy = A.jy[i], txx = A.txx[i], txy = A.txy[i],
                     tyy = A.tyy[i], G = A.G[i], ez = A.ez[i], bz = A.bz[i];
        const double gx = A.dpx[i], gy = A.dpy[i];
        double sx = dx0(A.jz, n, ix, i, inv2h) - dx0(A.txx, n, ix, i, inv2h) -
                    dy0(A.txy, n, iy, i, inv2h) - jy * bz / a + G * gx / (a * a) - jx * ez / a -
                    (txx * gx + txy * gy) / a;
        double sy = dy0(A.jz, n, iy, i, inv2h) - dx0(A.txy, n, ix, i, inv2h) -
                    dy0(A.tyy, n, iy, i, inv2h) + jx * bz / a + G * gy / (a * a) - jy * ez / a -
                    (txy * gx + tyy * gy) / a;
        A.f_bx[i] = sy;
        A.f_by[i] = -sx;
        sbx += sy * sy;
        sby += sx * sx;
    }
    sbx = block_sum(sbx);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[2][0], sbx);
    sby = block_sum(sby);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[2][1], sby);
}

// store the base slice; push every trajectory (Eqs. EoM_112_A, EoM_111);
// deposit n_* of the next slice; V_max
__device__ void phase_push(const EngineArgs &A, double *nnext, bool base, bool last, int j,
                           double dxi, int pk, Thr T) {
    const int nn = A.N * A.N;
    if (base) {
        double *h0 = A.hist + (size_t)j * nn;
        const size_t fs = (size_t)A.n_xi * nn;
        for (int i = T.t0; i < nn; i += T.nt) {
            h0[i] = A.psi[i];
            h0[fs + i] = A.ez[i];
            h0[2 * fs + i] = A.bz[i];
            h0[3 * fs + i] = A.bx[i];
            h0[4 * fs + i] = A.by[i];
        }
    }
    if (last) return;
    const double s = A.inv_h * A.inv_h;
    const double half = 0.5 * dxi;
    unsigned hits = 0;
    double vmax = 0.0;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        const double x = A.x[p], y = A.y[p];
        Cic c = cic_stencil(x, y, A.x_min, A.y_min, A.h, A.N);
        double a = guard(1.0 + cic_gather(A.psi, c), A.psi_floor, hits);
        const double gx = cic_gather(A.dpx, c), gy = cic_gather(A.dpy, c);
        const double bx = cic_gather(A.bx, c), by = cic_gather(A.by, c),
                     bz = cic_gather(A.bz, c);
        double px = A.px[p], py = A.py[p];
        // half kick: gamma grad psi / (1+psi) + e_z x B_perp
        double gam = (1.0 + px * px + py * py + a * a) / (2.0 * a);
        double pxm = px + half * (gam * gx / a - by);
        double pym = py + half * (gam * gy / a + bx);
        // rotation by the B_z term (e_z x p) B_z / (1+psi)
        double tau = half * bz / a;
        double pxp = pxm - tau * pym;
        double pyp = pym + tau * pxm;
        double sr = 2.0 * tau / (1.0 + tau * tau);
        double pxr = pxm - sr * pyp;
        double pyr = pym + sr * pxp;
        double gam2 = (1.0 + pxr * pxr + pyr * pyr + a * a) / (2.0 * a);
        px = pxr + half * (gam2 * gx / a - by);
        py = pyr + half * (gam2 * gy / a + bx);
        double nx = x + dxi * px / a;
        double ny = y + dxi * py / a;
        if (nx > A.x_max) { nx = 2.0 * A.x_max - nx; px = -px; }
        if (nx < A.x_min) { nx = 2.0 * A.x_min - nx; px = -px; }
        if (ny > A.y_max) { ny = 2.0 * A.y_max - ny; py = -py; }
        if (ny < A.y_min) { ny = 2.0 * A.y_min - ny; py = -py; }
        A.x[p] = nx;
        A.y[p] = ny;
        A.px[p] = px;
        A.py[p] = py;
        vmax = fmax(vmax, sqrt(px * px + py * py) / a);
        Cic c2 = cic_stencil(nx, ny, A.x_min, A.y_min, A.h, A.N);
        cic_deposit(nnext, c2, A.w[p] * s);
    }
    add_hits(A.sc, hits);
    vmax = block_max(vmax);
    if (threadIdx.x == 0) {
        atomicMax(&A.sc->vmax_bits[pk & 1], (unsigned long long)__double_as_longlong(vmax));
        atomicMax(&A.sc->vmax_all_bits, (unsigned long long)__double_as_longlong(vmax));
    }
}

__global__ void __launch_bounds__(QS_ENGINE_THREADS, 1) slice_engine(EngineArgs A) {
    extern __shared__ double smem[];
    const int bid = blockIdx.x, nblk = gridDim.x;
    const Sync S{A.sc, (unsigned)nblk, A.spin_cycles};
    DevScalars *sc = A.sc;
    const Thr T = grid_thr(bid, nblk);
    const bool lead = (bid == 0 && threadIdx.x == 0);

    double *ncur = A.n_a, *nnext = A.n_b;
    phase_deposit_n(A, ncur, T);
    if (!S(1)) return;

    SolveView Vpsi{1, 0, {A.psi, nullptr}, {A.f_psi, nullptr}, nullptr};
    SolveView Veb{2, 1, {A.ez, A.bz}, {A.f_ez, A.f_bz}, nullptr};
    SolveView Vbp{2, 2, {A.bx, A.by}, {A.f_bx, A.f_by}, A.kap};

    int m = A.m_sched ? A.m_sched[0] : 1;
    int slot = 0, pk = 0;
    for (int j = 0; j < A.n_xi; ++j) {
        if (lead) {
            A.diag_m[j] = m;
            if (m > sc->max_m) sc->max_m = m;
        }
        const bool last = (j == A.n_xi - 1);
        const double dxi = A.dxi0 / m;
        for (int q = 0; q < m; ++q) {
            const bool base = (q == 0);
            phase_psi_rhs(A, ncur, nnext, base, j, T);
            if (!S(2)) return;
            if (!mg_solve(A, S, Vpsi, slot, bid, nblk, smem)) return;
            phase_moments(A, T);
            if (!S(3)) return;
            phase_assemble1(A, ncur, j, q, m, T);
            if (!S(4)) return;
            if (!mg_solve(A, S, Veb, slot, bid, nblk, smem)) return;
            phase_assemble2(A, T);
            if (!S(5)) return;
            if (!mg_solve(A, S, Vbp, slot, bid, nblk, smem)) return;
            phase_push(A, nnext, base, last, j, dxi, pk, T);
            if (lead) {
                sc->slices += 1;
                if (!last) {
                    sc->pushes += A.np;
                    sc->vmax_bits[(pk + 1) & 1] = 0ull;
                }
                sc->fnorm[0][0] = sc->fnorm[0][1] = 0.0;
                sc->fnorm[1][0] = sc->fnorm[1][1] = 0.0;
                sc->fnorm[2][0] = sc->fnorm[2][1] = 0.0;
            }
            if (!S(6)) return;
            if (last) break;
            double *t = ncur;
            ncur = nnext;
            nnext = t;
            ++pk;
        }
        if (last) break;
        const double vm = __longlong_as_double((long long)vload(&sc->vmax_bits[(pk - 1) & 1]));
        if (lead) A.diag_vmax[j] = vm;
        if (A.m_sched) {
            m = A.m_sched[j + 1];
        } else if (vm <= A.V0) {
            m = 1;
        } else {
            double r = ceil(vm / A.V0);
            m = r > (double)A.refine_k ? A.refine_k : (int)r;
            if (m < 1) m = 1;
        }
    }
}

}  // namespace

int qs_engine_max_blocks(int device, size_t smem_bytes, int *blocks) {
    int per_sm = 0, sms = 0;
    if (cudaFuncSetAttribute(slice_engine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slice_engine, QS_ENGINE_THREADS,
                                                      smem_bytes) != cudaSuccess)
        return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return -1;
    *blocks = per_sm * sms;
    return 0;
}

cudaError_t qs_launch_engine(cudaStream_t st, const EngineArgs &a, int grid_blocks,
                             size_t smem_bytes) {
    EngineArgs copy = a;
    void *args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void *)slice_engine, dim3(grid_blocks),
                                       dim3(QS_ENGINE_THREADS), args, smem_bytes, st);
}
