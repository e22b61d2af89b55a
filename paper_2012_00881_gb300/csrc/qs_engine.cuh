// The slice engine: one persistent cooperative kernel runs the whole xi loop
// of Algorithm 1 (Collect_Source, Solve_Wakefield, Push_Trajectory,
// Step_Size_Refinement) for one 3D step.  Phases are separated by a grid
// barrier whose waits are bounded in time; a timed-out wait records
// QS_ERR_TIMEOUT and every block leaves the kernel at its next barrier.
//
// The solves (qs_solve.cuh) are red-black Gauss-Seidel V(nu1, nu2) cycles
// with 4-cell-average restriction, bilinear prolongation and rediscretised
// coarse operators (kappa averaged).  Levels of side <= block_level_n are
// solved redundantly by every block in its shared memory, down to a coarsest
// grid of side <= 4 whose dense inverse is cached.  Refined form: float64
// residual, float32 inner cycles whose grid-wide levels are staged tile by
// tile in shared memory, float64 correction.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "qs_solve.cuh"

namespace {

// ---------------------------------------------------------------------------
// particle and grid phases
// ---------------------------------------------------------------------------

// Plasma macroparticles and the grids they deposit into.  Positions and
// n_* are float64 in both forms (the density source n_* - n_ion and the
// sources built on it are small differences of O(1) numbers); momenta,
// weights and the other six moments are in the particle precision P (float64
// form: double; refined form: float).  In the refined form the gamma moment
// holds n_* <gamma - 1>, which has no cancellation.
template <typename P>
struct PS {
    double *x, *y;
    P *px, *py, *w;
    double *wd;  // float64 weights: n_* must cancel n_ion to rounding
    double *na, *nb;   // n_* of this slice and of the next one
    P *jx, *jy, *txx, *txy, *tyy, *G;
};

// n_* <gamma> from the gamma moment of either form
template <typename P>
__device__ __forceinline__ double g_total(const P *G, const double *n, int i) {
    if constexpr (sizeof(P) == 8) return G[i];
    else return n[i] + (double)G[i];
}

template <typename P>
struct CicP {
    int i00, i01, i10, i11;
    P w00, w01, w10, w11;
};

// CIC weights of a float64 stencil in the particle precision
template <typename P>
__device__ __forceinline__ CicP<P> cic_p(const Cic &c) {
    CicP<P> r;
    r.i00 = c.i00; r.i01 = c.i01; r.i10 = c.i10; r.i11 = c.i11;
    r.w00 = (P)c.w00; r.w01 = (P)c.w01; r.w10 = (P)c.w10; r.w11 = (P)c.w11;
    return r;
}

template <typename P, typename G>
__device__ __forceinline__ P gat(const G *u, const CicP<P> &c) {
    return (P)u[c.i00] * c.w00 + (P)u[c.i01] * c.w01 + (P)u[c.i10] * c.w10 + (P)u[c.i11] * c.w11;
}

template <typename P>
__device__ __forceinline__ void dep(P *g, const CicP<P> &c, P q) {
    atomicAdd(g + c.i00, q * c.w00);
    atomicAdd(g + c.i01, q * c.w01);
    atomicAdd(g + c.i10, q * c.w10);
    atomicAdd(g + c.i11, q * c.w11);
}

// 1 / a in float64 for a >= psi_floor > 0 by Newton's iteration for the
// reciprocal, r <- r (2 - a r), from the float32 reciprocal: each step doubles
// the correct bits (24, 48, then float64 rounding).  Four float64 operations
// and two conversions instead of a float64 divide, a long instruction
// sequence on GB300's 1/64-rate float64 pipe.
__device__ __forceinline__ double rcp_newton(double a) {
    double r = (double)__frcp_rn((float)a);
    r = r * fma(-a, r, 2.0);
    r = r * fma(-a, r, 2.0);
    return r;
}

// ---------------------------------------------------------------------------
// Privatised deposits.  With the plasma sorted by cell, a block that takes a
// contiguous chunk of the particle array finds its CIC stencils in a narrow
// band of grid rows (a 262,144-particle chunk of 1/152 covers about two rows
// of a 256^2 grid).  The block accumulates the band in shared memory and
// adds it to the grid once per cell: one global atomic per cell and moment
// instead of four per particle and moment.  A stencil outside the band (a
// particle that moved far since the last sort) is added to the grid directly.
// ---------------------------------------------------------------------------

// the block's contiguous chunk [p0, p1) of np particles
__device__ __forceinline__ void chunk_of(int64_t np, int bid, int nblk, int64_t &p0,
                                         int64_t &p1) {
    const int64_t cs = (np + nblk - 1) / nblk;
    p0 = min(np, (int64_t)bid * cs);
    p1 = min(np, p0 + cs);
}

// Rows [r0, r0 + rows) holding the CIC stencils (rows of y - h/2 and the
// next) of the chunk's particles, widened by `margin` rows on each side and
// clipped to the grid and to max_rows; rows = 0 for an empty chunk.
struct Band {
    int r0, rows;
};

__device__ Band band_of(const EngineArgs &A, const double *y, int64_t p0, int64_t p1, int margin,
                        int max_rows) {
    __shared__ int s_lo, s_hi;
    if (threadIdx.x == 0) {
        s_lo = A.N;
        s_hi = -1;
    }
    __syncthreads();
    int lo = A.N, hi = -1;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const int a = (int)floor((y[p] - A.y_min) * A.inv_h - 0.5);
        lo = min(lo, a);
        hi = max(hi, a + 1);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    __syncthreads();
    Band b{0, 0};
    if (s_hi >= 0) {
        const int r0 = max(0, s_lo - margin);
        const int r1 = min(A.N - 1, s_hi + margin);
        b.r0 = r0;
        b.rows = min(r1 - r0 + 1, max_rows);
    }
    __syncthreads();  // s_lo, s_hi are rewritten by the next call
    return b;
}

// deposit q into the band s (cells lo .. hi - 1 of the grid) when the whole
// stencil is inside, else into the grid g
template <typename P, typename W>
__device__ __forceinline__ void dep_band(P *g, P *s, int lo, int hi, const W &c, P q) {
    const int a = min(min(c.i00, c.i01), min(c.i10, c.i11));
    const int b = max(max(c.i00, c.i01), max(c.i10, c.i11));
    if (a >= lo && b < hi) {
        atomicAdd(s + (c.i00 - lo), q * (P)c.w00);
        atomicAdd(s + (c.i01 - lo), q * (P)c.w01);
        atomicAdd(s + (c.i10 - lo), q * (P)c.w10);
        atomicAdd(s + (c.i11 - lo), q * (P)c.w11);
    } else {
        atomicAdd(g + c.i00, q * (P)c.w00);
        atomicAdd(g + c.i01, q * (P)c.w01);
        atomicAdd(g + c.i10, q * (P)c.w10);
        atomicAdd(g + c.i11, q * (P)c.w11);
    }
}

// the band's nonzero cells added to the grid, one atomic per cell
template <typename P>
__device__ __forceinline__ void flush_band(P *g, const P *s, int lo, int cells) {
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        const P v = s[k];
        if (v != P(0)) atomicAdd(g + lo + k, v);
    }
}

template <typename P>
__device__ __forceinline__ void zero_band(P *s, int cells) {
    for (int k = threadIdx.x; k < cells; k += blockDim.x) s[k] = P(0);
}

// n_* of the initial particles
template <typename P>
__device__ void phase_deposit_n(const EngineArgs &A, const PS<P> &Q, double *ng, Thr T) {
    const double s = A.inv_h * A.inv_h;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        const Cic c = cic_stencil_inv(Q.x[p], Q.y[p], A.x_min, A.y_min, A.inv_h, A.N);
        cic_deposit(ng, c, Q.wd[p] * s);
    }
}

// Initial guess of a solve: the solutions of the last (up to three) slices
// extrapolated in xi to the new slice (order 0 is the plain warm start from
// the previous slice, Sec. 7.1).  w[k] multiplies the solution k slices back;
// the history of each field shifts by one as the guess replaces it.
struct Guess {
    double w0, w1, w2;
    bool active;
};

__device__ __forceinline__ Guess make_guess(int order, int have, double xt, double x0, double x1,
                                            double x2) {
    Guess g{1.0, 0.0, 0.0, order > 0 || have > 0};
    const int o = min(order, have - 1);
    if (o == 1) {
        g.w0 = (xt - x1) / (x0 - x1);
        g.w1 = (xt - x0) / (x1 - x0);
    } else if (o >= 2) {
        g.w0 = (xt - x1) * (xt - x2) / ((x0 - x1) * (x0 - x2));
        g.w1 = (xt - x0) * (xt - x2) / ((x1 - x0) * (x1 - x2));
        g.w2 = (xt - x0) * (xt - x1) / ((x2 - x0) * (x2 - x1));
    }
    return g;
}

__device__ __forceinline__ void apply_guess(double *u, double *h1, double *h2, int i,
                                            const Guess &g) {
    const double u0 = u[i], p1 = h1[i], p2 = h2[i];
    h2[i] = p1;
    h1[i] = u0;
    u[i] = g.w0 * u0 + g.w1 * p1 + g.w2 * p2;
}

// f_psi = n_* - n_ion (Eq. EqM_N8_AA) and its norm; charge sum; clear the
// moment accumulators and the next-slice density buffer
template <typename P>
__device__ void phase_psi_rhs(const EngineArgs &A, const PS<P> &Q, const double *ncur,
                              double *nnext, bool base, int j, int q, double frac, Thr T,
                              const Guess &g) {
    const int nn = A.N * A.N;
    double s = 0.0, cs = 0.0;
    if (A.a2_base) {  // |A|^2 of this slice, linear in xi between base slices
        const double *a0 = A.a2_base + (size_t)j * nn;
        const double *a1 = (j + 1 < A.n_xi) ? a0 + nn : nullptr;
        for (int i = T.t0; i < nn; i += T.nt)
            A.a2[i] = q == 0 ? a0[i] : (1.0 - frac) * a0[i] + frac * (a1 ? a1[i] : 0.0);
    }
    for (int i = T.t0; i < nn; i += T.nt) {
        if (g.active) apply_guess(A.psi, A.hist1[0], A.hist2[0], i, g);
        const double nv = (double)ncur[i];
        const double f = nv - A.n_ion[i];
        A.f_psi[i] = f;
        s += f * f;
        cs += nv;
        Q.jx[i] = P(0);
        Q.jy[i] = P(0);
        Q.txx[i] = P(0);
        Q.txy[i] = P(0);
        Q.tyy[i] = P(0);
        Q.G[i] = P(0);
        nnext[i] = 0.0;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[0][0], s);
    if (base && A.diag_charge) {
        cs = block_sum(cs);
        if (threadIdx.x == 0) atomicAdd(&A.diag_charge[j], cs * A.h * A.h);
    }
}

// gather psi at every particle; deposit j_perp, T, G (Eqs. Jr, FluxPres);
// gamma from the constant of motion is always evaluated in float64
template <typename P>
__device__ void phase_moments(const EngineArgs &A, const PS<P> &Q, Thr T, int bid, int nblk,
                              void *smem) {
    const P s = (P)(A.inv_h * A.inv_h);
    unsigned hits = 0;
    // privatised: this block's chunk into the six bands of sb
    const bool banded = A.band_rows > 0;
    int64_t p0 = T.t0, p1 = A.np, pst = T.nt;
    P *sb = nullptr;
    int lo = 0, hi = 0, cells = 0;
    if (banded) {
        int64_t c0, c1;
        chunk_of(A.np, bid, nblk, c0, c1);
        const Band b = band_of(A, Q.y, c0, c1, 0, A.band_rows);
        cells = b.rows * A.N;
        lo = b.r0 * A.N;
        hi = lo + cells;
        sb = (P *)((char *)smem + A.band_off);
        zero_band(sb, 6 * cells);
        __syncthreads();
        p0 = c0 + threadIdx.x;
        p1 = c1;
        pst = blockDim.x;
    }
    auto put = [&](P *g, int k, const CicP<P> &c, P q) {
        if (banded) dep_band(g, sb + k * cells, lo, hi, c, q);
        else dep(g, c, q);
    };
    for (int64_t p = p0; p < p1; p += pst) {
        const Cic cd = cic_stencil_inv(Q.x[p], Q.y[p], A.x_min, A.y_min, A.inv_h, A.N);
        const CicP<P> c = cic_p<P>(cd);
        const double a = guard(1.0 + cic_gather(A.psi, cd), A.psi_floor, hits);
        const P px = Q.px[p], py = Q.py[p];
        const double p2 = (double)px * px + (double)py * py;
        // one reciprocal per particle (float64 divides are slow)
        const double ia = sizeof(P) == 8 ? 1.0 / a : rcp_newton(a);
        const P iap = (P)ia;
        const P vx = px * iap, vy = py * iap;
        const P wq = Q.w[p] * s;
        // the laser's |A|^2 / 2 in the numerator of gamma (line after Eq. EoM_111)
        const double ha2 = A.a2_base ? 0.5 * cic_gather(A.a2, cd) : 0.0;
        put(Q.jx, 0, c, wq * vx);
        put(Q.jy, 1, c, wq * vy);
        put(Q.txx, 2, c, wq * vx * vx);
        put(Q.txy, 3, c, wq * vx * vy);
        put(Q.tyy, 4, c, wq * vy * vy);
        if constexpr (sizeof(P) == 8) {
            put(Q.G, 5, c, wq * ((1.0 + p2 + a * a + ha2) * (0.5 * ia)));  // gamma
        } else {
            const double am1 = a - 1.0;  // gamma - 1 = (p^2 + psi^2) / (2 (1 + psi))
            put(Q.G, 5, c, wq * (P)((p2 + am1 * am1 + ha2) * (0.5 * ia)));
        }
    }
    add_hits(A.sc, hits);
    if (banded) {
        __syncthreads();
        P *const g[6] = {Q.jx, Q.jy, Q.txx, Q.txy, Q.tyy, Q.G};
#pragma unroll
        for (int k = 0; k < 6; ++k) flush_band(g[k], sb + k * cells, lo, cells);
    }
}

// central differences: zero ghosts (moments) and odd ghosts (fields)
template <typename G>
__device__ __forceinline__ double dx0(const G *u, int n, int ix, int i, double inv2h) {
    const double e = ix < n - 1 ? (double)u[i + 1] : 0.0;
    const double w = ix > 0 ? (double)u[i - 1] : 0.0;
    return (e - w) * inv2h;
}
template <typename G>
__device__ __forceinline__ double dy0(const G *u, int n, int iy, int i, double inv2h) {
    const double s = iy < n - 1 ? (double)u[i + n] : 0.0;
    const double q = iy > 0 ? (double)u[i - n] : 0.0;
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
// driver), kappa = n_* / (1+psi) with the smoother's inverse diagonal, grad psi
template <typename P>
__device__ void phase_assemble1(const EngineArgs &A, const PS<P> &Q, const double *ncur, int j,
                                int q, double frac, Thr T, const Guess &g) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    const double *J0 = A.jzb + (size_t)j * nn;
    const double *J1 = (j + 1 < A.n_xi) ? A.jzb + (size_t)(j + 1) * nn : nullptr;
    unsigned hits = 0;
    double sez = 0.0, sbz = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        if (g.active) {
            apply_guess(A.ez, A.hist1[1], A.hist2[1], i, g);
            apply_guess(A.bz, A.hist1[2], A.hist2[2], i, g);
        }
        double fez = -(dx0(Q.jx, n, ix, i, inv2h) + dy0(Q.jy, n, iy, i, inv2h));
        double fbz = dx0(Q.jy, n, ix, i, inv2h) - dy0(Q.jx, n, iy, i, inv2h);
        A.f_ez[i] = fez;
        A.f_bz[i] = fbz;
        sez += fez * fez;
        sbz += fbz * fbz;
        double a = guard(1.0 + A.psi[i], A.psi_floor, hits);
        double jzb = q == 0 ? J0[i] : (1.0 - frac) * J0[i] + frac * (J1 ? J1[i] : 0.0);
        const double nv = ncur[i];
        const double ia = 1.0 / a;
        A.jz[i] = g_total(Q.G, ncur, i) * ia - nv + jzb;
        const double kap = nv * ia;
        A.kap[i] = kap;
        const int nw = qsmg::walls(ix, iy, n);
        if (A.precision == QS_FP32_REFINED) {
            const float k32 = (float)kap;
            A.k32[i] = k32;
            A.d32[i] = 1.f / ((float)(4 + nw) + A.lev_h2f[0] * k32);
        } else {
            A.invd0[i] = 1.0 / ((double)(4 + nw) + A.lev_h2[0] * kap);
        }
        A.dpx[i] = dxo(A.psi, n, ix, i, inv2h);
        A.dpy[i] = dyo(A.psi, n, iy, i, inv2h);
        if (A.dpx32) {
            A.dpx32[i] = (float)A.dpx[i];
            A.dpy32[i] = (float)A.dpy[i];
        }
        if (A.a2_base) {
            // grad(|A|^2 / 4), even ghosts (the ghost repeats the edge cell)
            const double *a2 = A.a2;
            const double e = ix < n - 1 ? a2[i + 1] : a2[i];
            const double w = ix > 0 ? a2[i - 1] : a2[i];
            const double so = iy < n - 1 ? a2[i + n] : a2[i];
            const double no = iy > 0 ? a2[i - n] : a2[i];
            A.pondx[i] = 0.25 * (e - w) * inv2h;
            A.pondy[i] = 0.25 * (so - no) * inv2h;
            if (A.chi && q == 0) A.chi[(size_t)j * nn + i] = kap;  // Eq. laser_Enve
        }
    }
    sez = block_sum(sez);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[1][0], sez);
    sbz = block_sum(sbz);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[1][1], sbz);
    add_hits(A.sc, hits);
}

// explicit source S of Eq. FluxCurr1_A; rhs of Eq. Main_Eq_A is -e_z x S =
// (S_y, -S_x)
template <typename P>
__device__ void phase_assemble2(const EngineArgs &A, const PS<P> &Q, const double *ncur, Thr T,
                                const Guess &g) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    double sbx = 0.0, sby = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        if (g.active) {
            apply_guess(A.bx, A.hist1[3], A.hist2[3], i, g);
            apply_guess(A.by, A.hist1[4], A.hist2[4], i, g);
        }
        double a = 1.0 + A.psi[i];
        if (a < A.psi_floor) a = A.psi_floor;
        const double jx = Q.jx[i], jy = Q.jy[i], txx = Q.txx[i], txy = Q.txy[i],
                     tyy = Q.tyy[i], G = g_total(Q.G, ncur, i), ez = A.ez[i], bz = A.bz[i];
        if (A.bz32) A.bz32[i] = (float)bz;  // B_z is final here
        const double gx = A.dpx[i], gy = A.dpy[i];
        const double ia = 1.0 / a, Gia2 = G * ia * ia;
        double sx = dx0(A.jz, n, ix, i, inv2h) - dx0(Q.txx, n, ix, i, inv2h) -
                    dy0(Q.txy, n, iy, i, inv2h) + Gia2 * gx -
                    (jy * bz + jx * ez + txx * gx + txy * gy) * ia;
        double sy = dy0(A.jz, n, iy, i, inv2h) - dx0(Q.txy, n, ix, i, inv2h) -
                    dy0(Q.tyy, n, iy, i, inv2h) + Gia2 * gy +
                    (jx * bz - jy * ez - txy * gx - tyy * gy) * ia;
        if (A.a2_base) {  // -n_* grad(|A|^2/4) / (1+psi)^2 of Eq. FluxCurr1_A
            const double nia2 = ncur[i] * ia * ia;
            sx -= nia2 * A.pondx[i];
            sy -= nia2 * A.pondy[i];
        }
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
// deposit n_* of the next slice; V_max.  gamma is evaluated in float64.
template <typename P>
__device__ void phase_push(const EngineArgs &A, const PS<P> &Q, double *nnext, bool base,
                           bool last, int j, double dxi, int pk, int sub, Thr T, int bid,
                           int nblk, void *smem) {
    const int nn = A.N * A.N;
    if (A.seg_g && sub < A.seg_cap) {  // segment store for the adjoint (float64)
        double *g = A.seg_g + (size_t)sub * SG_COUNT * nn;
        const double *ncur = Q.na == nnext ? Q.nb : Q.na;
        for (int i = T.t0; i < nn; i += T.nt) {
            g[SG_PSI * nn + i] = A.psi[i];
            g[SG_EZ * nn + i] = A.ez[i];
            g[SG_BZ * nn + i] = A.bz[i];
            g[SG_BX * nn + i] = A.bx[i];
            g[SG_BY * nn + i] = A.by[i];
            g[SG_N * nn + i] = ncur[i];
            g[SG_JX * nn + i] = (double)Q.jx[i];
            g[SG_JY * nn + i] = (double)Q.jy[i];
            g[SG_TXX * nn + i] = (double)Q.txx[i];
            g[SG_TXY * nn + i] = (double)Q.txy[i];
            g[SG_TYY * nn + i] = (double)Q.tyy[i];
            g[SG_G * nn + i] = g_total(Q.G, ncur, i);
        }
        double *sp = A.seg_p + (size_t)sub * 4 * A.np;
        for (int64_t p = T.t0; p < A.np; p += T.nt) {
            sp[p] = Q.x[p];
            sp[A.np + p] = Q.y[p];
            sp[2 * A.np + p] = (double)Q.px[p];
            sp[3 * A.np + p] = (double)Q.py[p];
        }
    }
    if (base && A.hist) {
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
    const P half = (P)(0.5 * dxi), dxp = (P)dxi;
    unsigned hits = 0;
    P vm = P(0);  // V_max (refined form: its square, in float32)
    // privatised n_* of the next slice: the band of the chunk's present rows
    // widened by two rows for the particles' motion
    const bool banded = A.band_rows_n > 0;
    int64_t p0 = T.t0, p1 = A.np, pst = T.nt;
    double *sb = nullptr;
    int lo = 0, hi = 0, cells = 0;
    if (banded) {
        int64_t c0, c1;
        chunk_of(A.np, bid, nblk, c0, c1);
        const Band b = band_of(A, Q.y, c0, c1, 2, A.band_rows_n);
        cells = b.rows * A.N;
        lo = b.r0 * A.N;
        hi = lo + cells;
        sb = (double *)((char *)smem + A.band_off);
        zero_band(sb, cells);
        __syncthreads();
        p0 = c0 + threadIdx.x;
        p1 = c1;
        pst = blockDim.x;
    }
    for (int64_t p = p0; p < p1; p += pst) {
        const double x = Q.x[p], y = Q.y[p];
        const Cic cd = cic_stencil_inv(x, y, A.x_min, A.y_min, A.inv_h, A.N);
        const CicP<P> c = cic_p<P>(cd);
        const double a = guard(1.0 + cic_gather(A.psi, cd), A.psi_floor, hits);
        const double ia = sizeof(P) == 8 ? 1.0 / a : rcp_newton(a);
        const P iap = (P)ia;
        P gx, gy, bx, by, bz;
        if constexpr (sizeof(P) == 8) {
            gx = gat<P>(A.dpx, c);
            gy = gat<P>(A.dpy, c);
            bx = gat<P>(A.bx, c);
            by = gat<P>(A.by, c);
            bz = gat<P>(A.bz, c);
        } else {  // the float32 copies: no conversions
            gx = gat<P>(A.dpx32, c);
            gy = gat<P>(A.dpy32, c);
            bx = gat<P>(A.bx32, c);
            by = gat<P>(A.by32, c);
            bz = gat<P>(A.bz32, c);
        }
        P px = Q.px[p], py = Q.py[p];
        // laser (Eq. EoM_111): |A|^2 / 2 in gamma and the ponderomotive force
        // -grad(|A|^2/4) / (1+psi); zero without a laser
        double ha2 = 0.0;
        P fx = P(0), fy = P(0);
        if (A.a2_base) {
            ha2 = 0.5 * cic_gather(A.a2, cd);
            fx = gat<P>(A.pondx, c);
            fy = gat<P>(A.pondy, c);
        }
        // half kick: (gamma grad psi - grad(|A|^2/4)) / (1+psi) + e_z x B_perp
        const double gam = (1.0 + (double)px * px + (double)py * py + a * a + ha2) * (0.5 * ia);
        const P pxm = px + half * (((P)gam * gx - fx) * iap - by);
        const P pym = py + half * (((P)gam * gy - fy) * iap + bx);
        // rotation by the B_z term (e_z x p) B_z / (1+psi)
        const P tau = half * bz * iap;
        const P pxp = pxm - tau * pym;
        const P pyp = pym + tau * pxm;
        const P sr = P(2) * tau / (P(1) + tau * tau);
        const P pxr = pxm - sr * pyp;
        const P pyr = pym + sr * pxp;
        const double gam2 =
            (1.0 + (double)pxr * pxr + (double)pyr * pyr + a * a + ha2) * (0.5 * ia);
        px = pxr + half * (((P)gam2 * gx - fx) * iap - by);
        py = pyr + half * (((P)gam2 * gy - fy) * iap + bx);
        double nx = x + (double)(dxp * px * iap);
        double ny = y + (double)(dxp * py * iap);
        if (nx > A.x_max) { nx = 2.0 * A.x_max - nx; px = -px; }
        if (nx < A.x_min) { nx = 2.0 * A.x_min - nx; px = -px; }
        if (ny > A.y_max) { ny = 2.0 * A.y_max - ny; py = -py; }
        if (ny < A.y_min) { ny = 2.0 * A.y_min - ny; py = -py; }
        Q.x[p] = nx;
        Q.y[p] = ny;
        Q.px[p] = px;
        Q.py[p] = py;
        if constexpr (sizeof(P) == 8) {
            vm = fmax(vm, sqrt((double)px * px + (double)py * py) * ia);
        } else {  // float32 (the step rule needs a few digits); squared, root below
            vm = fmaxf(vm, (px * px + py * py) * (iap * iap));
        }
        const Cic c2 = cic_stencil_inv(nx, ny, A.x_min, A.y_min, A.inv_h, A.N);
        if (banded) dep_band(nnext, sb, lo, hi, c2, Q.wd[p] * s);
        else cic_deposit(nnext, c2, Q.wd[p] * s);
    }
    add_hits(A.sc, hits);
    if (banded) {
        __syncthreads();
        flush_band(nnext, sb, lo, cells);
    }
    double vmax = block_max((double)vm);
    if (sizeof(P) == 4) vmax = sqrt(vmax);
    if (threadIdx.x == 0) {
        atomicMax(&A.sc->vmax_bits[pk & 1], (unsigned long long)__double_as_longlong(vmax));
        atomicMax(&A.sc->vmax_all_bits, (unsigned long long)__double_as_longlong(vmax));
    }
}

// ---------------------------------------------------------------------------
// cell sort inside the slice loop
// ---------------------------------------------------------------------------

// exclusive scan of v over the block (any blockDim.x <= 1024); returns the
// prefix of this thread and the block total in *total
__device__ int block_exscan(int v, int *total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        int t = lane < nw ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;  // inclusive prefix of the warp sums
    }
    __syncthreads();
    *total = ws[((blockDim.x + 31) >> 5) - 1];
    return x - v + (wid > 0 ? ws[wid - 1] : 0);
}

// Stable counting sort of the plasma by (cell, id), cell = iy N + ix of the
// position's cell (floor, clamped), the order of the standalone cell sort;
// the arrays are gathered into the spare set and copied back (the slice
// loop's particle pointers stay fixed: swapping them would keep two sets of
// pointers live in registers through the whole loop).
template <typename P>
__device__ __noinline__ bool sort_plasma(const EngineArgs &A, const PS<P> &Q, const Sync &S,
                                         int bid, int nblk) {
    int32_t *const id = A.id, *const id2 = A.id2;
    P *const px2 = (P *)A.px2, *const py2 = (P *)A.py2, *const w2 = (P *)A.w2;
    const int nn = A.N * A.N;
    const Thr T = grid_thr(bid, nblk);
    for (int i = T.t0; i < nn; i += T.nt) A.s_count[i] = 0;
    SYNC(90);
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        int ix = (int)floor((Q.x[p] - A.x_min) * A.inv_h);
        int iy = (int)floor((Q.y[p] - A.y_min) * A.inv_h);
        ix = min(max(ix, 0), A.N - 1);
        iy = min(max(iy, 0), A.N - 1);
        const int c = iy * A.N + ix;
        A.s_cell[p] = c;
        atomicAdd(A.s_count + c, 1);
    }
    SYNC(91);
    // exclusive scan: each block its chunk of cells, then the chunk offsets
    const int ch = (nn + nblk - 1) / nblk;
    const int c0 = min(bid * ch, nn), c1 = min(c0 + ch, nn);
    int run = 0;
    for (int b = c0; b < c1; b += blockDim.x) {
        const int i = b + (int)threadIdx.x;
        int tot;
        const int pre = block_exscan(i < c1 ? A.s_count[i] : 0, &tot);
        if (i < c1) A.s_offset[i] = run + pre;
        run += tot;
    }
    if (threadIdx.x == 0) A.s_bsum[bid] = run;
    SYNC(92);
    __shared__ int s_base;
    if (threadIdx.x == 0) {
        int base = 0;
        for (int b = 0; b < bid; ++b) base += A.s_bsum[b];
        s_base = base;
        if (bid == nblk - 1) A.s_offset[nn] = base + run;
    }
    __syncthreads();
    for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x) {
        A.s_offset[i] += s_base;
        A.s_cursor[i] = A.s_offset[i];
    }
    SYNC(93);
    for (int64_t p = T.t0; p < A.np; p += T.nt)
        A.s_order[atomicAdd(A.s_cursor + A.s_cell[p], 1)] = (int32_t)p;
    SYNC(94);
    // within a cell, ascending id (segments hold a few particles)
    for (int i = T.t0; i < nn; i += T.nt) {
        const int b = A.s_offset[i], e = A.s_offset[i + 1];
        for (int k = b + 1; k < e; ++k) {
            const int32_t v = A.s_order[k], key = id[v];
            int m = k - 1;
            while (m >= b && id[A.s_order[m]] > key) {
                A.s_order[m + 1] = A.s_order[m];
                --m;
            }
            A.s_order[m + 1] = v;
        }
    }
    SYNC(95);
    const bool sep_wd = (const void *)Q.wd != (const void *)Q.w;
    for (int64_t s = T.t0; s < A.np; s += T.nt) {
        const int32_t p = A.s_order[s];
        A.x2[s] = Q.x[p];
        A.y2[s] = Q.y[p];
        px2[s] = Q.px[p];
        py2[s] = Q.py[p];
        w2[s] = Q.w[p];
        if (sep_wd) A.wd2[s] = Q.wd[p];
        id2[s] = id[p];
    }
    SYNC(96);
    for (int64_t s = T.t0; s < A.np; s += T.nt) {
        Q.x[s] = A.x2[s];
        Q.y[s] = A.y2[s];
        Q.px[s] = px2[s];
        Q.py[s] = py2[s];
        Q.w[s] = w2[s];
        if (sep_wd) Q.wd[s] = A.wd2[s];
        id[s] = id2[s];
    }
    SYNC(97);
    return true;
}

// One 3D step of one instance on `nblk` blocks (this one is `bid`): the xi
// loop of Algorithm 1.  Returns false if a barrier failed (the error word of
// the instance says why).
template <bool REF>
__device__ bool run_step(const EngineArgs &A, int bid, int nblk, const Sync &S, void *smem,
                         int *s_inv_ready) {
    if (A.trace && bid == 0 && threadIdx.x == 0) {
        A.trace[0] = 0;
        A.trace[1] = global_ns();
        A.sc->trace_n = 1;
    }
    DevScalars *sc = A.sc;
    const Thr T = grid_thr(bid, nblk);
    const bool lead = (bid == 0 && threadIdx.x == 0);

    using P = typename std::conditional<REF, float, double>::type;
    PS<P> Q;
    if constexpr (REF) {
        Q = PS<P>{A.x, A.y, A.px32, A.py32, A.w32, A.w, A.n_a, A.n_b,
                  A.jx32, A.jy32, A.txx32, A.txy32, A.tyy32, A.G32};
    } else {
        Q = PS<P>{A.x, A.y, A.px, A.py, A.w, A.w, A.n_a, A.n_b,
                  A.jx, A.jy, A.txx, A.txy, A.tyy, A.G};
    }
    // the spare particle set of the in-loop sort (not with the adjoint's
    // checkpoints or slice store: those keep the lattice's order)
    const bool sorting = A.sort_every > 0 && A.x2 && !A.ckpt && !A.seg_p;
    int n_sorts = 0;
    double *ncur = Q.na, *nnext = Q.nb;
    phase_deposit_n<P>(A, Q, ncur, T);
    if (!S(1)) return false;

    const SolveSpec Vpsi{1, 0, {A.psi, nullptr}, {A.f_psi, nullptr}, false};
    const SolveSpec Veb{2, 1, {A.ez, A.bz}, {A.f_ez, A.f_bz}, false};
    const SolveSpec Vbp{2, 2, {A.bx, A.by}, {A.f_bx, A.f_by}, true,
                        {REF ? A.bx32 : nullptr, REF ? A.by32 : nullptr}};

    int m = A.m_sched ? A.m_sched[A.j_begin] : 1;
    // per-slice scalars computed by thread 0 and read by every thread
    __shared__ struct {
        Guess g;
        double frac, dxi;
        int m;
    } s_ctl;
    __syncthreads();
    if (threadIdx.x == 0) s_ctl.dxi = A.dxi0 / m;
    __syncthreads();
    int slot = 0, pk = 0, sub = 0;
    int have = 0;                        // previous solutions available for the guess
    double gx0 = 0.0, gx1 = 0.0, gx2 = 0.0;  // their xi
    for (int j = A.j_begin; j < A.j_end; ++j) {
        if (sorting && j > A.j_begin && j % A.sort_every == 0) {
            if (!sort_plasma<P>(A, Q, S, bid, nblk)) return false;
            ++n_sorts;
            if (lead) sc->sorts = n_sorts;
        }
        if (lead && A.diag_m) {
            A.diag_m[j] = m;
            if (m > sc->max_m) sc->max_m = m;
        }
        const bool last = (j == A.n_xi - 1);
        const double dxi = s_ctl.dxi;
        if (A.ckpt && j % A.ckpt_every == 0) {  // plasma state before slice j
            double *cp = A.ckpt + (size_t)(j / A.ckpt_every) * 4 * A.np;
            for (int64_t p = T.t0; p < A.np; p += T.nt) {
                cp[p] = Q.x[p];
                cp[A.np + p] = Q.y[p];
                cp[2 * A.np + p] = (double)Q.px[p];
                cp[3 * A.np + p] = (double)Q.py[p];
            }
        }
        for (int q = 0; q < m; ++q) {
            const bool base = (q == 0);
            const double xs = j * A.dxi0 + q * dxi;  // xi of this slice (from xi_min)
            // the guess weights and the sub-step fraction by one thread
            // (float64 divides repeated by every thread cost microseconds)
            __syncthreads();
            if (threadIdx.x == 0) {
                s_ctl.g = make_guess(A.ws_order, have, xs, gx0, gx1, gx2);
                s_ctl.frac = (double)q / (double)m;
            }
            __syncthreads();
            const Guess g = s_ctl.g;
            const double frac = s_ctl.frac;
            phase_psi_rhs<P>(A, Q, ncur, nnext, base, j, q, frac, T, g);
            if (!S(2)) return false;
            if (!mg_solve<REF>(A, S, Vpsi, slot, bid, nblk, smem, s_inv_ready)) return false;
            phase_moments<P>(A, Q, T, bid, nblk, smem);
            if (!S(3)) return false;
            phase_assemble1<P>(A, Q, ncur, j, q, frac, T, g);
            if (!S(4)) return false;
            if (!mg_solve<REF>(A, S, Veb, slot, bid, nblk, smem, s_inv_ready)) return false;
            phase_assemble2<P>(A, Q, ncur, T, g);
            if (!S(5)) return false;
            if (!mg_solve<REF>(A, S, Vbp, slot, bid, nblk, smem, s_inv_ready)) return false;
            phase_push<P>(A, Q, nnext, base, last, j, dxi, pk, sub, T, bid, nblk, smem);
            ++sub;
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
            if (!S(6)) return false;
            gx2 = gx1;
            gx1 = gx0;
            gx0 = xs;
            have = min(have + 1, 3);
            if (last) break;
            double *t = ncur;
            ncur = nnext;
            nnext = t;
            ++pk;
        }
        if (last) break;
        // the next base slice's sub-steps (Sec. 5.1), by one thread
        __syncthreads();
        if (threadIdx.x == 0) {
            const double vm =
                __longlong_as_double((long long)vload(&sc->vmax_bits[(pk - 1) & 1]));
            if (lead && A.diag_vmax) A.diag_vmax[j] = vm;
            int mn;
            if (A.m_sched) {
                mn = A.m_sched[j + 1];
            } else if (vm <= A.V0) {
                mn = 1;
            } else {
                double r = ceil(vm / A.V0);
                mn = r > (double)A.refine_k ? A.refine_k : (int)r;
                if (mn < 1) mn = 1;
            }
            s_ctl.m = mn;
            s_ctl.dxi = A.dxi0 / mn;
        }
        __syncthreads();
        m = s_ctl.m;
    }
    return true;
}

// The arguments are copied into shared memory once: the phases take them by
// reference, and a reference to a by-value kernel parameter would make a
// per-thread copy in local memory.
template <bool REF>
__global__ void __launch_bounds__(QS_ENGINE_THREADS, 1) slice_engine(const __grid_constant__ EngineArgs A0) {
    extern __shared__ double smem[];
    __shared__ unsigned long long s_epoch;
    __shared__ int s_inv_ready[2];
    __shared__ EngineArgs A;
    for (int k = threadIdx.x; k < (int)(sizeof(EngineArgs) / 4); k += blockDim.x)
        ((int *)&A)[k] = ((const int *)&A0)[k];
    if (threadIdx.x == 0) {
        s_epoch = 0ull;
        s_inv_ready[0] = s_inv_ready[1] = 0;
    }
    __syncthreads();
    // A launch without the configured thread-block clusters (a profiler's
    // kernel replay can drop the attribute) would reach distributed shared
    // memory of blocks that are not there: every block returns at once with
    // an error instead, before the first grid barrier.
    if (A.cl_size > 1 && (int)cooperative_groups::this_cluster().num_blocks() != A.cl_size) {
        if (threadIdx.x == 0 && atomicCAS(&A.sc->err, 0, QS_ERR_CUDA) == 0)
            A.sc->err_where = -1;
        return;
    }
    const Sync S{A.sc, &A.sc->bar_arrive, gridDim.x, A.spin_cycles, A.trace, A.trace_cap,
                 &s_epoch, blockIdx.x == 0, A.cl_size};
    run_step<REF>(A, blockIdx.x, gridDim.x, S, smem, s_inv_ready);
}

// Batched form: the launch is split into teams of `team` consecutive blocks;
// each team takes the next instance from a device-side queue, runs its whole
// 3D step behind the team's own barrier, and repeats until the queue is
// empty.  Instances may differ in size, tiles and sweeps.
template <bool REF>
__global__ void __launch_bounds__(QS_ENGINE_THREADS, 1)
    slice_engine_batched(const EngineArgs *list, int n_inst, int team, BatchState *bs) {
    extern __shared__ double smem[];
    __shared__ unsigned long long s_epoch;
    __shared__ int s_inv_ready[2];
    __shared__ EngineArgs sA;
    const int tid = blockIdx.x / team, bid = blockIdx.x % team;
    if (threadIdx.x == 0) s_epoch = 0ull;
    __syncthreads();
    for (;;) {
        if (bid == 0 && threadIdx.x == 0) {
            bs->team_inst[tid] = atomicAdd(&bs->next, 1);
            __threadfence();
        }
        // team barrier on the team's counter (errors of a finished instance do
        // not concern the next one, so this one checks the batch error word)
        const Sync T0{&bs->sc, &bs->team_bar[tid], (unsigned)team, list[0].spin_cycles, nullptr,
                      0, &s_epoch, false};
        if (!T0(60)) return;
        const int idx = vload(&bs->team_inst[tid]);
        if (idx >= n_inst) return;
        for (int k = threadIdx.x; k < (int)(sizeof(EngineArgs) / 4); k += blockDim.x)
            ((int *)&sA)[k] = ((const int *)(list + idx))[k];
        if (threadIdx.x == 0) s_inv_ready[0] = s_inv_ready[1] = 0;
        __syncthreads();
        const Sync S{sA.sc, &bs->team_bar[tid], (unsigned)team, sA.spin_cycles, nullptr, 0,
                     &s_epoch, false};
        if (!run_step<REF>(sA, bid, team, S, smem, s_inv_ready)) {
            // the instance failed: its blocks stop; record it for the batch
            if (bid == 0 && threadIdx.x == 0) atomicCAS(&bs->sc.err, 0, vload(&sA.sc->err));
            return;
        }
    }
}

}  // namespace
