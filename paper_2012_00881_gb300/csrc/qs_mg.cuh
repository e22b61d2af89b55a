// Geometric multigrid pieces for the slice engine (device code only).
//
// The operator on every level is A u = lap_h u - kappa u with the 5-point
// Laplacian of Eq. 2D_Laplac_Uni and odd (zero-wall) ghosts; kappa = 0 for
// psi, E_z, B_z (Eqs. EqM_N8_AA, EqM_N8_A, Mag_z_A) and kappa = n_* / (1+psi)
// for B_perp (Eq. Main_Eq_A).  Red-black Gauss-Seidel smoothing, 4-cell
// average restriction of the residual (and of kappa), bilinear cell-centred
// prolongation, rediscretised coarse operators, dense elimination on the
// coarsest level.  Templated on the storage type (double, or float for the
// inner cycles of the refined form); the coarsest solve is always float64.
#pragma once

#include "qs_internal.cuh"

namespace qsmg {

struct Thr {
    int t0, nt;
};

template <typename T>
struct Lvl {
    T *u[2];
    T *f[2];
    T *k;  // kappa (screened levels) or nullptr
    T *d;  // inverse diagonal 1/(4 + walls + h^2 kappa) (screened) or nullptr
    int n;
    double h2;
};

template <typename T>
struct Hier {
    Lvl<T> lv[QS_MAX_LEV];
    int L;
};

__device__ __forceinline__ int walls(int ix, int iy, int n) {
    return (ix == 0) + (ix == n - 1) + (iy == 0) + (iy == n - 1);
}

template <typename T>
__device__ __forceinline__ T inv_diag(const Lvl<T> &L, int i, int nw) {
    if (L.d) return L.d[i];
    return nw == 0 ? T(0.25) : (nw == 1 ? T(0.2) : (nw == 2 ? T(1.0 / 6.0) : T(1) / T(4 + nw)));
}

// (lap_h - kappa) u at (ix, iy), computed in T
template <typename T>
__device__ __forceinline__ T apply_op(const T *u, const T *k, int n, T inv_h2, int ix, int iy) {
    const int i = iy * n + ix;
    const T uc = u[i];
    T nb = T(0);
    if (ix > 0) nb += u[i - 1];
    if (ix < n - 1) nb += u[i + 1];
    if (iy > 0) nb += u[i - n];
    if (iy < n - 1) nb += u[i + n];
    T r = (nb - T(4 + walls(ix, iy, n)) * uc) * inv_h2;
    if (k) r -= k[i] * uc;
    return r;
}

// one red-black half sweep of `color` on every component
template <typename T>
__device__ void relax_half(const Lvl<T> &L, int nc, int color, Thr R) {
    const int n = L.n;
    const T h2 = T(L.h2);
    const int npts = (n & 1) ? n * n : (n * n) / 2;
    const int hn = n >> 1;
    for (int q = R.t0; q < npts; q += R.nt) {
        int ix, iy;
        if (n & 1) {
            iy = q / n;
            ix = q - iy * n;
            if (((ix + iy) & 1) != color) continue;
        } else {
            iy = q / hn;
            ix = 2 * (q - iy * hn) + ((iy + color) & 1);
        }
        const int i = iy * n + ix;
        const T di = inv_diag(L, i, walls(ix, iy, n));
        for (int c = 0; c < nc; ++c) {
            T *u = L.u[c];
            T nb = T(0);
            if (ix > 0) nb += u[i - 1];
            if (ix < n - 1) nb += u[i + 1];
            if (iy > 0) nb += u[i - n];
            if (iy < n - 1) nb += u[i + n];
            u[i] = (nb - h2 * L.f[c][i]) * di;
        }
    }
}

// C.f = 4-cell average of the residual of F; C.u = 0; screened levels also
// get C.k (4-cell average of F.k) and C.d
template <typename T>
__device__ void restrict_res(const Lvl<T> &F, const Lvl<T> &C, int nc, Thr R) {
    const int n = F.n, m = C.n;
    const T inv_h2 = T(1.0 / F.h2);
    for (int q = R.t0; q < m * m; q += R.nt) {
        const int J = q / m, I = q - J * m;
        const int i0 = (2 * J) * n + 2 * I;
        for (int c = 0; c < nc; ++c) {
            const T *u = F.u[c];
            const T *f = F.f[c];
            T s = f[i0] - apply_op(u, (const T *)F.k, n, inv_h2, 2 * I, 2 * J);
            s += f[i0 + 1] - apply_op(u, (const T *)F.k, n, inv_h2, 2 * I + 1, 2 * J);
            s += f[i0 + n] - apply_op(u, (const T *)F.k, n, inv_h2, 2 * I, 2 * J + 1);
            s += f[i0 + n + 1] - apply_op(u, (const T *)F.k, n, inv_h2, 2 * I + 1, 2 * J + 1);
            C.f[c][q] = T(0.25) * s;
            C.u[c][q] = T(0);
        }
        if (F.k) {
            const T kk = T(0.25) * (F.k[i0] + F.k[i0 + 1] + F.k[i0 + n] + F.k[i0 + n + 1]);
            C.k[q] = kk;
            C.d[q] = T(1) / (T(4 + walls(I, J, m)) + T(C.h2) * kk);
        }
    }
}

// F.u += bilinear interpolation of C.u (odd ghosts on the coarse level)
template <typename T>
__device__ void prolong_add(const Lvl<T> &F, const Lvl<T> &C, int nc, Thr R) {
    const int n = F.n, m = C.n;
    for (int q = R.t0; q < n * n; q += R.nt) {
        const int iy = q / n, ix = q - iy * n;
        const int I = ix >> 1, J = iy >> 1;
        const int I2 = I + ((ix & 1) ? 1 : -1);
        const int J2 = J + ((iy & 1) ? 1 : -1);
        const bool xin = (I2 >= 0 && I2 < m), yin = (J2 >= 0 && J2 < m);
        for (int c = 0; c < nc; ++c) {
            const T *uc = C.u[c];
            const T v00 = uc[J * m + I];
            const T v10 = xin ? uc[J * m + I2] : -v00;
            const T v01 = yin ? uc[J2 * m + I] : -v00;
            T v11;
            if (xin && yin) v11 = uc[J2 * m + I2];
            else if (xin) v11 = -uc[J * m + I2];
            else if (yin) v11 = -uc[J2 * m + I];
            else v11 = v00;
            F.u[c][q] += (T(9) * v00 + T(3) * v10 + T(3) * v01 + v11) * T(0.0625);
        }
    }
}

// Dense float64 elimination of -(lap_h - kappa) on the coarsest level by the
// calling block (no pivoting: the matrix is symmetric positive definite).
// `mat` needs n^2 * (n^2 + 3) doubles.
template <typename T>
__device__ void coarse_solve(const Lvl<T> &L, int nc, double *mat) {
    const int n = L.n, m = n * n, ld = m + 2;
    const double inv_h2 = 1.0 / L.h2;
    double *fac = mat + m * ld;
    for (int e = threadIdx.x; e < m * ld; e += blockDim.x) mat[e] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int iy = i / n, ix = i - iy * n;
        mat[i * ld + i] = (4.0 + walls(ix, iy, n)) * inv_h2 + (L.k ? (double)L.k[i] : 0.0);
        if (ix > 0) mat[i * ld + i - 1] = -inv_h2;
        if (ix < n - 1) mat[i * ld + i + 1] = -inv_h2;
        if (iy > 0) mat[i * ld + i - n] = -inv_h2;
        if (iy < n - 1) mat[i * ld + i + n] = -inv_h2;
        for (int c = 0; c < nc; ++c) mat[i * ld + m + c] = -(double)L.f[c][i];
    }
    __syncthreads();
    const int ncol = m + nc;
    for (int k = 0; k < m - 1; ++k) {
        const double inv_piv = 1.0 / mat[k * ld + k];
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) fac[i] = mat[i * ld + k] * inv_piv;
        __syncthreads();
        const int rows = m - k - 1, cols = ncol - k;
        for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
            const int i = k + 1 + e / cols, j = k + e % cols;
            mat[i * ld + j] -= fac[i] * mat[k * ld + j];
        }
        __syncthreads();
    }
    if ((int)threadIdx.x < nc) {  // back substitution; x overwrites column m + c
        const int c = threadIdx.x;
        for (int i = m - 1; i >= 0; --i) {
            double s = mat[i * ld + m + c];
            for (int j = i + 1; j < m; ++j) s -= mat[i * ld + j] * mat[j * ld + m + c];
            mat[i * ld + m + c] = s / mat[i * ld + i];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        for (int c = 0; c < nc; ++c) L.u[c][i] = (T)mat[i * ld + m + c];
    __syncthreads();
}

// Shared-memory bytes that block_vcycle needs from level lg down.
template <typename T>
__host__ __device__ inline size_t block_smem_bytes(const int *lev_n, int L, int lg, int nc_max) {
    size_t pts = 0;
    for (int l = lg; l < L; ++l) pts += (size_t)lev_n[l] * lev_n[l];
    const int mc = lev_n[L - 1] * lev_n[L - 1];
    size_t b = pts * (2 * nc_max + 2) * sizeof(T);
    b = (b + 15) & ~(size_t)15;
    return b + (size_t)mc * (mc + 3) * sizeof(double);
}

// The rest of a V-cycle from level lg down, entirely in the calling block's
// shared memory.  Level lg's right-hand side (and kappa) come from global
// memory; its initial iterate is zero unless lg == 0 (then the global u is
// the warm start).  Level lg's result is written back to global memory.
template <typename T>
__device__ void block_vcycle(const Hier<T> &H, int lg, int nc, int nu1, int nu2, void *smem) {
    const int L = H.L;
    Lvl<T> S[QS_MAX_LEV];
    T *p = (T *)smem;
    for (int l = lg; l < L; ++l) {
        const int m = H.lv[l].n * H.lv[l].n;
        S[l].n = H.lv[l].n;
        S[l].h2 = H.lv[l].h2;
        for (int c = 0; c < 2; ++c) {
            S[l].u[c] = p;
            p += m;
            S[l].f[c] = p;
            p += m;
        }
        if (H.lv[lg].k) {
            S[l].k = p;
            p += m;
            S[l].d = p;
            p += m;
        } else {
            S[l].k = S[l].d = nullptr;
            p += 2 * m;
        }
    }
    size_t off = ((size_t)((char *)p - (char *)smem) + 15) & ~(size_t)15;
    double *mat = (double *)((char *)smem + off);
    const Lvl<T> &G = H.lv[lg];
    const int m0 = G.n * G.n;
    for (int i = threadIdx.x; i < m0; i += blockDim.x) {
        for (int c = 0; c < nc; ++c) {
            S[lg].u[c][i] = (lg == 0) ? G.u[c][i] : T(0);
            S[lg].f[c][i] = G.f[c][i];
        }
        if (G.k) {
            S[lg].k[i] = G.k[i];
            S[lg].d[i] = G.d[i];
        }
    }
    __syncthreads();
    const Thr B{(int)threadIdx.x, (int)blockDim.x};
    for (int l = lg; l < L - 1; ++l) {
        for (int s = 0; s < nu1; ++s) {
            relax_half(S[l], nc, 0, B);
            __syncthreads();
            relax_half(S[l], nc, 1, B);
            __syncthreads();
        }
        restrict_res(S[l], S[l + 1], nc, B);
        __syncthreads();
    }
    coarse_solve(S[L - 1], nc, mat);
    for (int l = L - 2; l >= lg; --l) {
        prolong_add(S[l], S[l + 1], nc, B);
        __syncthreads();
        for (int s = 0; s < nu2; ++s) {
            relax_half(S[l], nc, 0, B);
            __syncthreads();
            relax_half(S[l], nc, 1, B);
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < m0; i += blockDim.x)
        for (int c = 0; c < nc; ++c) G.u[c][i] = S[lg].u[c][i];
    __syncthreads();
}

}  // namespace qsmg
