// The adjoint engine: reverse-mode differentiation of the slice loop over one
// segment of stored slices, as one persistent cooperative kernel.
//
// The forward slice (Algorithm 1, Collect_Source / Solve_Wakefield /
// Push_Trajectory) maps the plasma state P_s = (x, y, px, py) to the fields
// of the slice and to P_{s+1}.  Walking the segment's slices backwards, this
// kernel carries the cotangent of P and accumulates the cotangents of the
// weights, of n_ion and of the bunches' j_z.  Per slice, in reverse order of
// the forward computation:
//
//   push      reverse Boris step; gather cotangents are scattered (the
//             adjoint of a gather is a deposit), the gather weights' slope
//             adds to the position cotangent
//   B_perp    (lap - kappa) mu = dL/dB (the operator is symmetric, so the
//             transposed solve is the same multigrid solve); then the source
//             S of Eq. FluxCurr1_A backwards, kappa = n_*/(1+psi), j_z
//   E_z, B_z  lap nu = dL/dE_z, dL/dB_z; then j_perp backwards through the
//             central differences of Eqs. EqM_N8_A and Mag_z_A
//   moments   reverse of the moment deposit of Eq. Jr / FluxPres (the
//             adjoint of a deposit is a gather) through V = p/(1+psi) and the
//             constant of motion gamma = (1 + p^2 + (1+psi)^2) / (2 (1+psi))
//   psi       lap nu = dL/dpsi (Eq. EqM_N8_AA); then n_* and n_ion
//   n_*       reverse of the density deposit
//
// The sub-step schedule is that of the forward run and the 1+psi guard is
// treated as inactive where it did not clamp (a clamped value has no
// derivative).  All arithmetic is float64; the transposed solves use the
// context's multigrid (refined form: float32 inner cycles, float64 residual).
#pragma once

#include <cuda_runtime.h>

#include "qs_solve.cuh"

namespace {

// CIC with the per-axis weights kept, so that the slope of an interpolation
// in x and y is available: for a gather v = sum_c w_c u_c,
//   dv/dx = (1/h) (wy0 (u01 - u00) + wy1 (u11 - u10)),
//   dv/dy = (1/h) (wx0 (u10 - u00) + wx1 (u11 - u01)).
struct CicD {
    int i00, i01, i10, i11;
    double wx0, wx1, wy0, wy1;
};

__device__ __forceinline__ CicD cic_d(double x, double y, const EngineArgs &A) {
    int ix0, ix1, iy0, iy1;
    CicD c;
    cic_axis((x - A.x_min) * A.inv_h, A.N, ix0, ix1, c.wx0, c.wx1);
    cic_axis((y - A.y_min) * A.inv_h, A.N, iy0, iy1, c.wy0, c.wy1);
    const int n = A.N;
    c.i00 = iy0 * n + ix0;
    c.i01 = iy0 * n + ix1;
    c.i10 = iy1 * n + ix0;
    c.i11 = iy1 * n + ix1;
    return c;
}

struct GatherD {
    double v, dx, dy;  // value and slopes (slopes without the 1/h)
};

__device__ __forceinline__ GatherD gather_d(const double *u, const CicD &c) {
    const double u00 = u[c.i00], u01 = u[c.i01], u10 = u[c.i10], u11 = u[c.i11];
    GatherD g;
    g.v = c.wy0 * (c.wx0 * u00 + c.wx1 * u01) + c.wy1 * (c.wx0 * u10 + c.wx1 * u11);
    g.dx = c.wy0 * (u01 - u00) + c.wy1 * (u11 - u10);
    g.dy = c.wx0 * (u10 - u00) + c.wx1 * (u11 - u01);
    return g;
}

// deposit with the same weights (no 1/h^2): the adjoint of gather_d's value
__device__ __forceinline__ void scatter(double *g, const CicD &c, double q) {
    if (q == 0.0) return;
    atomicAdd(g + c.i00, q * c.wy0 * c.wx0);
    atomicAdd(g + c.i01, q * c.wy0 * c.wx1);
    atomicAdd(g + c.i10, q * c.wy1 * c.wx0);
    atomicAdd(g + c.i11, q * c.wy1 * c.wx1);
}

// central differences: zero ghosts (moment grids) and the transpose of the
// odd-ghost difference of psi, which is minus the difference with even
// (mirror) ghosts
__device__ __forceinline__ double cdx0(const double *u, int n, int ix, int i) {
    return (ix < n - 1 ? u[i + 1] : 0.0) - (ix > 0 ? u[i - 1] : 0.0);
}
__device__ __forceinline__ double cdy0(const double *u, int n, int iy, int i) {
    return (iy < n - 1 ? u[i + n] : 0.0) - (iy > 0 ? u[i - n] : 0.0);
}
__device__ __forceinline__ double cdxo(const double *u, int n, int ix, int i) {
    return (ix < n - 1 ? u[i + 1] : -u[i]) - (ix > 0 ? u[i - 1] : -u[i]);
}
__device__ __forceinline__ double cdyo(const double *u, int n, int iy, int i) {
    return (iy < n - 1 ? u[i + n] : -u[i]) - (iy > 0 ? u[i - n] : -u[i]);
}
__device__ __forceinline__ double cdxo_t(const double *v, int n, int ix, int i) {
    return (ix > 0 ? v[i - 1] : v[i]) - (ix < n - 1 ? v[i + 1] : v[i]);
}
__device__ __forceinline__ double cdyo_t(const double *v, int n, int iy, int i) {
    return (iy > 0 ? v[i - n] : v[i]) - (iy < n - 1 ? v[i + n] : v[i]);
}

// One stored slice of the segment.
struct Slice {
    const double *x, *y, *px, *py;  // plasma state before the push
    const double *psi, *ez, *bz, *bx, *by, *n, *jx, *jy, *txx, *txy, *tyy, *G;
    int j, q, m;                    // base slice, sub-step, sub-steps of the slice
    bool last;                      // the last base slice of the window (no push)
};

__device__ __forceinline__ Slice slice_at(const EngineArgs &A, int s, int j, int q, int m) {
    const size_t nn = (size_t)A.N * A.N;
    const double *g = A.seg_g + (size_t)s * SG_COUNT * nn;
    const double *p = A.seg_p + (size_t)s * 4 * A.np;
    Slice S;
    S.x = p;
    S.y = p + A.np;
    S.px = p + 2 * A.np;
    S.py = p + 3 * A.np;
    S.psi = g + SG_PSI * nn;
    S.ez = g + SG_EZ * nn;
    S.bz = g + SG_BZ * nn;
    S.bx = g + SG_BX * nn;
    S.by = g + SG_BY * nn;
    S.n = g + SG_N * nn;
    S.jx = g + SG_JX * nn;
    S.jy = g + SG_JY * nn;
    S.txx = g + SG_TXX * nn;
    S.txy = g + SG_TXY * nn;
    S.tyy = g + SG_TYY * nn;
    S.G = g + SG_G * nn;
    S.j = j;
    S.q = q;
    S.m = m;
    S.last = (j == A.n_xi - 1);
    return S;
}

// P0: per-slice grids (1+psi, kappa and the screened smoother's diagonal,
// grad psi), cleared accumulators, and the loss cotangent of the stored
// fields of a base slice.
__device__ void adj_prepare(const EngineArgs &A, const AdjArgs &D, const Slice &S, Thr T) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    const bool base = (S.q == 0);
    const size_t fs = (size_t)A.n_xi * nn;
    const double *dh = (base && D.d_hist) ? D.d_hist + (size_t)S.j * nn : nullptr;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        double a = 1.0 + S.psi[i];
        if (a < A.psi_floor) a = A.psi_floor;
        const double kap = S.n[i] * (1.0 / a);
        A.kap[i] = kap;
        const int nw = qsmg::walls(ix, iy, n);
        if (A.precision == QS_FP32_REFINED) {
            const float k32 = (float)kap;
            A.k32[i] = k32;
            A.d32[i] = 1.f / ((float)(4 + nw) + A.lev_h2f[0] * k32);
        } else {
            A.invd0[i] = 1.0 / ((double)(4 + nw) + A.lev_h2[0] * kap);
        }
        A.dpx[i] = cdxo(S.psi, n, ix, i) * inv2h;
        A.dpy[i] = cdyo(S.psi, n, iy, i) * inv2h;
        D.g_psi[i] = dh ? dh[i] : 0.0;
        D.g_ez[i] = dh ? dh[fs + i] : 0.0;
        D.g_bz[i] = dh ? dh[2 * fs + i] : 0.0;
        D.g_bx[i] = dh ? dh[3 * fs + i] : 0.0;
        D.g_by[i] = dh ? dh[4 * fs + i] : 0.0;
        D.g_dpx[i] = 0.0;
        D.g_dpy[i] = 0.0;
    }
}

// P1: reverse of the plasma push of this slice (Eqs. EoM_112_A, EoM_111 with
// the Boris-like half kick / rotation / half kick and the drift; specular
// walls).  On entry l* hold dL/dP_{s+1}; on exit the part of dL/dP_s that
// flows through the push.  Field cotangents are scattered.
__device__ void adj_push(const EngineArgs &A, const AdjArgs &D, const Slice &S, Thr T) {
    const double dxi = A.dxi0 / S.m, half = 0.5 * dxi;
    const double ih = A.inv_h;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        const double x = S.x[p], y = S.y[p], px = S.px[p], py = S.py[p];
        const CicD c = cic_d(x, y, A);
        const GatherD Gp = gather_d(S.psi, c), Ggx = gather_d(A.dpx, c),
                      Ggy = gather_d(A.dpy, c), Gbx = gather_d(S.bx, c),
                      Gby = gather_d(S.by, c), Gbz = gather_d(S.bz, c);
        double a = 1.0 + Gp.v;
        const bool act = a >= A.psi_floor;
        if (!act) a = A.psi_floor;
        const double ia = 1.0 / a, ia2 = ia * ia;  // one divide per particle
        const double gx = Ggx.v, gy = Ggy.v, bx = Gbx.v, by = Gby.v, bz = Gbz.v;
        // forward
        const double gam = (1.0 + px * px + py * py + a * a) * (0.5 * ia);
        const double pxm = px + half * (gam * gx * ia - by);
        const double pym = py + half * (gam * gy * ia + bx);
        const double tau = half * bz * ia;
        const double pxp = pxm - tau * pym;
        const double pyp = pym + tau * pxm;
        const double t2 = 1.0 + tau * tau;
        const double sr = 2.0 * tau / t2;
        const double pxr = pxm - sr * pyp;
        const double pyr = pym + sr * pxp;
        const double gam2 = (1.0 + pxr * pxr + pyr * pyr + a * a) * (0.5 * ia);
        const double px2 = pxr + half * (gam2 * gx * ia - by);
        const double py2 = pyr + half * (gam2 * gy * ia + bx);
        const double nx0 = x + dxi * px2 * ia;
        const double ny0 = y + dxi * py2 * ia;
        int fx = 0, fy = 0;  // reflections at the walls (each flips position and momentum)
        {
            double v = nx0;
            if (v > A.x_max) { v = 2.0 * A.x_max - v; ++fx; }
            if (v < A.x_min) { ++fx; }
            v = ny0;
            if (v > A.y_max) { v = 2.0 * A.y_max - v; ++fy; }
            if (v < A.y_min) { ++fy; }
        }
        // reverse
        const double sx = (fx & 1) ? -1.0 : 1.0, sy = (fy & 1) ? -1.0 : 1.0;
        const double l_nx = sx * D.lx[p], l_ny = sy * D.ly[p];
        double l_px2 = sx * D.lpx[p], l_py2 = sy * D.lpy[p];
        double l_x = l_nx, l_y = l_ny;
        double ab = 0.0, gxb = 0.0, gyb = 0.0, bxb = 0.0, byb = 0.0, bzb = 0.0;
        l_px2 += l_nx * dxi * ia;
        l_py2 += l_ny * dxi * ia;
        ab -= (l_nx * px2 + l_ny * py2) * dxi * ia2;
        // second half kick
        double l_pxr = l_px2, l_pyr = l_py2;
        double g2b = half * (l_px2 * gx + l_py2 * gy) * ia;
        gxb += l_px2 * half * gam2 * ia;
        gyb += l_py2 * half * gam2 * ia;
        ab -= half * gam2 * (l_px2 * gx + l_py2 * gy) * ia2;
        byb -= l_px2 * half;
        bxb += l_py2 * half;
        // gamma2
        l_pxr += g2b * pxr * ia;
        l_pyr += g2b * pyr * ia;
        ab += g2b * (0.5 - (1.0 + pxr * pxr + pyr * pyr) * (0.5 * ia2));
        // rotation
        double l_pxm = l_pxr, l_pym = l_pyr;
        double srb = -l_pxr * pyp + l_pyr * pxp;
        const double l_pyp = -l_pxr * sr;
        const double l_pxp = l_pyr * sr;
        l_pxm += l_pxp;
        double taub = -l_pxp * pym;
        l_pym -= l_pxp * tau;
        l_pym += l_pyp;
        taub += l_pyp * pxm;
        l_pxm += l_pyp * tau;
        taub += srb * 2.0 * (1.0 - tau * tau) / (t2 * t2);
        bzb += taub * half * ia;
        ab -= taub * tau * ia;
        // first half kick
        double l_px = l_pxm, l_py = l_pym;
        const double g1b = half * (l_pxm * gx + l_pym * gy) * ia;
        gxb += l_pxm * half * gam * ia;
        gyb += l_pym * half * gam * ia;
        ab -= half * gam * (l_pxm * gx + l_pym * gy) * ia2;
        byb -= l_pxm * half;
        bxb += l_pym * half;
        l_px += g1b * px * ia;
        l_py += g1b * py * ia;
        ab += g1b * (0.5 - (1.0 + px * px + py * py) * (0.5 * ia2));
        if (!act) ab = 0.0;
        // gathers: slopes into the position cotangent, values scattered
        l_x += (ab * Gp.dx + gxb * Ggx.dx + gyb * Ggy.dx + bxb * Gbx.dx + byb * Gby.dx +
                bzb * Gbz.dx) * ih;
        l_y += (ab * Gp.dy + gxb * Ggx.dy + gyb * Ggy.dy + bxb * Gbx.dy + byb * Gby.dy +
                bzb * Gbz.dy) * ih;
        scatter(D.g_psi, c, ab);
        scatter(D.g_dpx, c, gxb);
        scatter(D.g_dpy, c, gyb);
        scatter(D.g_bx, c, bxb);
        scatter(D.g_by, c, byb);
        scatter(D.g_bz, c, bzb);
        D.lx[p] = l_x;
        D.ly[p] = l_y;
        D.lpx[p] = l_px;
        D.lpy[p] = l_py;
    }
}

// squared norms of a 1- or 2-component right-hand side into fnorm[kind]
__device__ void rhs_norms(const EngineArgs &A, int kind, const double *f0, const double *f1,
                          Thr T) {
    const int nn = A.N * A.N;
    double s0 = 0.0, s1 = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        s0 += f0[i] * f0[i];
        if (f1) s1 += f1[i] * f1[i];
    }
    s0 = block_sum(s0);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[kind][0], s0);
    if (f1) {
        s1 = block_sum(s1);
        if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[kind][1], s1);
    }
}

// P3: reverse of Eq. FluxCurr1_A (source S from the moments and psi, E_z,
// B_z), of Eq. Main_Eq_A's right-hand side (S_y, -S_x) and kappa, and of
// j_z = n_* <gamma> / (1+psi) - n_* + j_z,b.  mu = (mu_x, mu_y) is the
// solution of the transposed B_perp solve: dL/dS_x = -mu_y, dL/dS_y = mu_x,
// dL/dkappa = mu . B_perp.  Also the norms of the E_z, B_z adjoint sources.
__device__ void adj_source(const EngineArgs &A, const AdjArgs &D, const Slice &S, Thr T) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    const double frac = (double)S.q / (double)S.m;
    double *J0 = D.d_jzb + (size_t)S.j * nn;
    double *J1 = (S.j + 1 < A.n_xi) ? D.d_jzb + (size_t)(S.j + 1) * nn : nullptr;
    double sez = 0.0, sbz = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        double a = 1.0 + S.psi[i];
        const bool act = a >= A.psi_floor;
        if (!act) a = A.psi_floor;
        const double ia = 1.0 / a, ia2 = ia * ia, ia3 = ia2 * ia;
        const double sxb = -D.mu_y[i], syb = D.mu_x[i];
        const double jx = S.jx[i], jy = S.jy[i], txx = S.txx[i], txy = S.txy[i],
                     tyy = S.tyy[i], G = S.G[i], nv = S.n[i], ez = S.ez[i], bz = S.bz[i];
        const double gx = A.dpx[i], gy = A.dpy[i];
        const double kapb = D.mu_x[i] * S.bx[i] + D.mu_y[i] * S.by[i];
        // differences of dL/dS (zero ghosts; the difference is antisymmetric)
        const double dsx_x = -(ix < n - 1 ? D.mu_y[i + 1] : 0.0) + (ix > 0 ? D.mu_y[i - 1] : 0.0);
        const double dsx_y = -(iy < n - 1 ? D.mu_y[i + n] : 0.0) + (iy > 0 ? D.mu_y[i - n] : 0.0);
        const double dsy_x = cdx0(D.mu_x, n, ix, i);
        const double dsy_y = cdy0(D.mu_x, n, iy, i);
        const double jzb_ = -(dsx_x + dsy_y) * inv2h;  // dL/dj_z
        // pointwise terms of S
        const double jyb = -sxb * bz * ia - syb * ez * ia;
        const double jxb = -sxb * ez * ia + syb * bz * ia;
        const double bzb = (-sxb * jy + syb * jx) * ia;
        const double ezb = -(sxb * jx + syb * jy) * ia;
        double Gb = (sxb * gx + syb * gy) * ia2;
        const double gxb = sxb * (G * ia2 - txx * ia) - syb * txy * ia;
        const double gyb = syb * (G * ia2 - tyy * ia) - sxb * txy * ia;
        const double txxb = -sxb * gx * ia + dsx_x * inv2h;
        const double txyb = -(sxb * gy + syb * gx) * ia + (dsx_y + dsy_x) * inv2h;
        const double tyyb = -syb * gy * ia + dsy_y * inv2h;
        double ab = sxb * (jy * bz * ia2 - 2.0 * G * gx * ia3 + jx * ez * ia2 +
                           (txx * gx + txy * gy) * ia2) +
                    syb * (-jx * bz * ia2 - 2.0 * G * gy * ia3 + jy * ez * ia2 +
                           (txy * gx + tyy * gy) * ia2);
        // j_z and kappa
        Gb += jzb_ * ia;
        const double nb = -jzb_ + kapb * ia;
        ab += -jzb_ * G * ia2 - kapb * nv * ia2;
        if (!act) ab = 0.0;
        J0[i] += (S.q == 0 ? 1.0 : 1.0 - frac) * jzb_;
        if (S.q != 0 && J1) J1[i] += frac * jzb_;
        D.g_psi[i] += ab;
        const double fez = D.g_ez[i] + ezb, fbz = D.g_bz[i] + bzb;
        D.g_ez[i] = fez;
        D.g_bz[i] = fbz;
        sez += fez * fez;
        sbz += fbz * fbz;
        D.g_dpx[i] += gxb;
        D.g_dpy[i] += gyb;
        D.g_jx[i] = jxb;
        D.g_jy[i] = jyb;
        D.g_txx[i] = txxb;
        D.g_txy[i] = txyb;
        D.g_tyy[i] = tyyb;
        D.g_G[i] = Gb;
        D.g_n[i] = nb;
    }
    sez = block_sum(sez);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[1][0], sez);
    sbz = block_sum(sbz);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[1][1], sbz);
}

// P4: j_perp backwards through the sources of E_z = lap^-1 (-(D_x j_x + D_y
// j_y)) and B_z = lap^-1 (D_x j_y - D_y j_x) (zero-ghost differences, whose
// transpose is their negative).
__device__ void adj_jperp(const EngineArgs &A, const AdjArgs &D, Thr T) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        D.g_jx[i] += (cdx0(D.nu_ez, n, ix, i) + cdy0(D.nu_bz, n, iy, i)) * inv2h;
        D.g_jy[i] += (cdy0(D.nu_ez, n, iy, i) - cdx0(D.nu_bz, n, ix, i)) * inv2h;
    }
}

// P5: reverse of the moment deposits (j = n_* <V>, T = n_* <V V>, G = n_*
// <gamma>; deposits carry 1/h^2) through V = p/(1+psi_p) and gamma from the
// constant of motion; 1 + psi_p is a gather of psi.
__device__ void adj_moments(const EngineArgs &A, const AdjArgs &D, const Slice &S, Thr T) {
    const double ih = A.inv_h, s2 = A.inv_h * A.inv_h;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        const double px = S.px[p], py = S.py[p], w = A.w[p];
        const CicD c = cic_d(S.x[p], S.y[p], A);
        const GatherD Gp = gather_d(S.psi, c);
        double a = 1.0 + Gp.v;
        const bool act = a >= A.psi_floor;
        if (!act) a = A.psi_floor;
        const double ia = 1.0 / a, ia2 = ia * ia;
        const double vx = px * ia, vy = py * ia;
        const double gam = (1.0 + px * px + py * py + a * a) * (0.5 * ia);
        const GatherD Gjx = gather_d(D.g_jx, c), Gjy = gather_d(D.g_jy, c),
                      Gxx = gather_d(D.g_txx, c), Gxy = gather_d(D.g_txy, c),
                      Gyy = gather_d(D.g_tyy, c), GG = gather_d(D.g_G, c);
        // deposited values per unit weight
        const double qjx = vx, qjy = vy, qxx = vx * vx, qxy = vx * vy, qyy = vy * vy, qG = gam;
        D.lw[p] += (qjx * Gjx.v + qjy * Gjy.v + qxx * Gxx.v + qxy * Gxy.v + qyy * Gyy.v +
                    qG * GG.v) * s2;
        const double vxb = w * s2 * (Gjx.v + 2.0 * vx * Gxx.v + vy * Gxy.v);
        const double vyb = w * s2 * (Gjy.v + vx * Gxy.v + 2.0 * vy * Gyy.v);
        const double gb = w * s2 * GG.v;
        double ab = -(vxb * px + vyb * py) * ia2 +
                    gb * (0.5 - (1.0 + px * px + py * py) * (0.5 * ia2));
        if (!act) ab = 0.0;
        D.lpx[p] += vxb * ia + gb * px * ia;
        D.lpy[p] += vyb * ia + gb * py * ia;
        const double wq = w * s2 * ih;
        D.lx[p] += wq * (qjx * Gjx.dx + qjy * Gjy.dx + qxx * Gxx.dx + qxy * Gxy.dx +
                         qyy * Gyy.dx + qG * GG.dx) + ab * Gp.dx * ih;
        D.ly[p] += wq * (qjx * Gjx.dy + qjy * Gjy.dy + qxx * Gxx.dy + qxy * Gxy.dy +
                         qyy * Gyy.dy + qG * GG.dy) + ab * Gp.dy * ih;
        scatter(D.g_psi, c, ab);
    }
}

// P6: the right-hand side of the psi adjoint: dL/dpsi plus grad psi's
// cotangents through the transposed odd-ghost differences.
__device__ void adj_psi_rhs(const EngineArgs &A, const AdjArgs &D, Thr T) {
    const int n = A.N, nn = n * n;
    const double inv2h = 0.5 * A.inv_h;
    double s = 0.0;
    for (int i = T.t0; i < nn; i += T.nt) {
        const int iy = i / n, ix = i - iy * n;
        const double f = D.g_psi[i] + (cdxo_t(D.g_dpx, n, ix, i) + cdyo_t(D.g_dpy, n, iy, i)) * inv2h;
        D.f_nu_psi[i] = f;
        s += f * f;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(&A.sc->fnorm[0][0], s);
}

// P7: reverse of the n_* deposit (Eq. continuity; 1/h^2) with dL/dn_* =
// g_n + nu_psi; n_ion's cotangent is -nu_psi.
__device__ void adj_density(const EngineArgs &A, const AdjArgs &D, const Slice &S, Thr T) {
    const int nn = A.N * A.N;
    const double ih = A.inv_h, s2 = A.inv_h * A.inv_h;
    for (int64_t p = T.t0; p < A.np; p += T.nt) {
        const CicD c = cic_d(S.x[p], S.y[p], A);
        const GatherD g1 = gather_d(D.g_n, c), g2 = gather_d(D.nu_psi, c);
        const double w = A.w[p];
        D.lw[p] += (g1.v + g2.v) * s2;
        D.lx[p] += w * s2 * ih * (g1.dx + g2.dx);
        D.ly[p] += w * s2 * ih * (g1.dy + g2.dy);
    }
    for (int i = T.t0; i < nn; i += T.nt) D.d_nion[i] -= D.nu_psi[i];
}

template <bool REF>
__device__ bool run_adjoint(const EngineArgs &A, const AdjArgs &D, int bid, int nblk,
                            const Sync &S, void *smem, int *s_inv_ready) {
    DevScalars *sc = A.sc;
    const Thr T = grid_thr(bid, nblk);
    const bool lead = (bid == 0 && threadIdx.x == 0);
    const SolveSpec Vbp{2, 2, {D.mu_x, D.mu_y}, {D.g_bx, D.g_by}, true};
    const SolveSpec Veb{2, 1, {D.nu_ez, D.nu_bz}, {D.g_ez, D.g_bz}, false};
    const SolveSpec Vpsi{1, 0, {D.nu_psi, nullptr}, {D.f_nu_psi, nullptr}, false};
    int slot = 0;
    // the last stored slice of the segment
    int j = D.j1 - 1;
    int m = A.m_sched[j];
    int q = (j == A.n_xi - 1) ? 0 : m - 1;
    for (int s = D.n_sub - 1; s >= 0; --s) {
        const Slice Sl = slice_at(A, s, j, q, m);
        adj_prepare(A, D, Sl, T);
        SYNC(101);
        if (!Sl.last) {
            adj_push(A, D, Sl, T);
            SYNC(102);
        }
        rhs_norms(A, 2, D.g_bx, D.g_by, T);
        SYNC(103);
        if (!mg_solve<REF>(A, S, Vbp, slot, bid, nblk, smem, s_inv_ready)) return false;
        adj_source(A, D, Sl, T);
        SYNC(104);
        if (!mg_solve<REF>(A, S, Veb, slot, bid, nblk, smem, s_inv_ready)) return false;
        adj_jperp(A, D, T);
        SYNC(105);
        adj_moments(A, D, Sl, T);
        SYNC(106);
        adj_psi_rhs(A, D, T);
        SYNC(107);
        if (!mg_solve<REF>(A, S, Vpsi, slot, bid, nblk, smem, s_inv_ready)) return false;
        adj_density(A, D, Sl, T);
        if (lead) {
            sc->slices += 1;
            sc->fnorm[0][0] = sc->fnorm[0][1] = 0.0;
            sc->fnorm[1][0] = sc->fnorm[1][1] = 0.0;
            sc->fnorm[2][0] = sc->fnorm[2][1] = 0.0;
        }
        SYNC(108);
        // previous slice in forward order
        if (q > 0) {
            --q;
        } else {
            --j;
            if (j >= 0) {
                m = A.m_sched[j];
                q = m - 1;
            }
        }
    }
    return true;
}

template <bool REF>
__global__ void __launch_bounds__(QS_ENGINE_THREADS, 1)
    adjoint_engine(const __grid_constant__ EngineArgs A0, const __grid_constant__ AdjArgs D0) {
    extern __shared__ double smem[];
    __shared__ unsigned long long s_epoch;
    __shared__ int s_inv_ready[2];
    __shared__ EngineArgs A;
    __shared__ AdjArgs D;
    for (int k = threadIdx.x; k < (int)(sizeof(EngineArgs) / 4); k += blockDim.x)
        ((int *)&A)[k] = ((const int *)&A0)[k];
    for (int k = threadIdx.x; k < (int)(sizeof(AdjArgs) / 4); k += blockDim.x)
        ((int *)&D)[k] = ((const int *)&D0)[k];
    if (threadIdx.x == 0) {
        s_epoch = 0ull;
        s_inv_ready[0] = s_inv_ready[1] = 0;
    }
    __syncthreads();
    const Sync S{A.sc, &A.sc->bar_arrive, gridDim.x, A.spin_cycles, nullptr, 0, &s_epoch, false};
    run_adjoint<REF>(A, D, blockIdx.x, gridDim.x, S, smem, s_inv_ready);
}

}  // namespace
