// Geometric multigrid pieces for the slice engine (device code only).
//
// The operator on every level is A u = lap_h u - kappa u with the 5-point
// Laplacian of Eq. 2D_Laplac_Uni and odd (zero-wall) ghosts; kappa = 0 for
// psi, E_z, B_z (Eqs. EqM_N8_AA, EqM_N8_A, Mag_z_A) and kappa = n_* / (1+psi)
// for B_perp (Eq. Main_Eq_A).  Red-black Gauss-Seidel smoothing, 4-cell
// average restriction of the residual (and of kappa), bilinear cell-centred
// prolongation, rediscretised coarse operators, dense elimination on the
// coarsest level.  Templated on the storage type (double, or float for the
// inner cycles of the refined form) and on the number of components solved
// together (1 or 2, sharing the operator); the coarsest solve is float64.
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
    double inv_h2;  // 1 / h2
    T h2t;          // h2 and 1 / h2 in the storage type (no per-thread
    T inv_h2t;      // float64 divide or conversion in the sweeps)
    T omega;  // relaxation factor of the red-black sweeps (1 = Gauss-Seidel)
};

template <typename T>
struct Hier {
    Lvl<T> lv[QS_MAX_LEV];
    int L;
};

__device__ __forceinline__ int walls(int ix, int iy, int n) {
    return (ix == 0) + (ix == n - 1) + (iy == 0) + (iy == n - 1);
}

// 1 / (4 + walls) without a divide (a float64 divide is a long sequence on
// GB300's 1/64-rate float64 pipe, and a select may evaluate it regardless)
template <typename T>
__device__ __forceinline__ T const_inv_diag(int nw) {
    return nw == 0 ? T(0.25)
                   : (nw == 1 ? T(0.2)
                              : (nw == 2 ? T(1.0 / 6.0) : (nw == 3 ? T(1.0 / 7.0) : T(0.125))));
}

// Walk q = t0, t0 + nt, ... over a row-major index space with `w` columns,
// keeping (row, col) without a division per step.
// Global -> shared copies are issued asynchronously (cp.async) for a whole
// staged region and waited for once, so a load phase costs one L2 round trip
// instead of one per loop iteration.  A copy whose source is outside the
// domain reads nothing and writes zero (source size 0); its source address
// is then the array base, which is always valid.
__device__ __forceinline__ void cp_async_f32(float *dst, const float *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_f64(double *dst, const double *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void cp_async(T *dst, const T *src, bool valid) {
    if (sizeof(T) == 8) cp_async_f64((double *)dst, (const double *)src, valid);
    else cp_async_f32((float *)dst, (const float *)src, valid);
}

struct Walk {
    int q, row, col, nt, drow, dcol, w;
    __device__ __forceinline__ Walk(int t0, int nt_, int w_) : q(t0), nt(nt_), w(w_) {
        if ((w & (w - 1)) == 0) {  // power of two: shifts instead of divides
            const int sh = __ffs(w) - 1;
            row = t0 >> sh;
            col = t0 & (w - 1);
            drow = nt >> sh;
            dcol = nt & (w - 1);
        } else {
            row = t0 / w;
            col = t0 - row * w;
            drow = nt / w;
            dcol = nt - drow * w;
        }
    }
    __device__ __forceinline__ void next() {
        q += nt;
        row += drow;
        col += dcol;
        if (col >= w) {
            col -= w;
            ++row;
        }
    }
};

// (lap_h - kappa) u at (ix, iy) of an n x n array, computed in T
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

// Red-black update of one point: the Gauss-Seidel value g, over-relaxed by
// omega (u <- u + omega (g - u)).
template <typename T, int NC>
__device__ __forceinline__ void gs_point(T *const u0, T *const u1, const T *const f0,
                                         const T *const f1, T h2, T di, T omega, int n, int ix,
                                         int iy) {
    const int i = iy * n + ix;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        T *u = c ? u1 : u0;
        T nb = T(0);
        if (ix > 0) nb += u[i - 1];
        if (ix < n - 1) nb += u[i + 1];
        if (iy > 0) nb += u[i - n];
        if (iy < n - 1) nb += u[i + n];
        const T g = (nb - h2 * (c ? f1 : f0)[i]) * di;
        const T uo = u[i];
        u[i] = uo + omega * (g - uo);
    }
}

// one red-black half sweep of `color` on every component
template <typename T, int NC>
__device__ void relax_half(const Lvl<T> L, int color, Thr R) {
    const int n = L.n;
    const T h2 = L.h2t;
    T *const u0 = L.u[0];
    T *const u1 = L.u[NC - 1];
    const T *const f0 = L.f[0];
    const T *const f1 = L.f[NC - 1];
    const T *const dd = L.d;
    if (n & 1) {
        for (Walk w(R.t0, R.nt, n); w.q < n * n; w.next()) {
            const int ix = w.col, iy = w.row;
            if (((ix + iy) & 1) != color) continue;
            const T di = dd ? dd[iy * n + ix] : const_inv_diag<T>(walls(ix, iy, n));
            gs_point<T, NC>(u0, u1, f0, f1, h2, di, L.omega, n, ix, iy);
        }
        return;
    }
    const int hn = n >> 1;
    for (Walk w(R.t0, R.nt, hn); w.q < n * hn; w.next()) {
        const int iy = w.row;
        const int ix = 2 * w.col + ((iy + color) & 1);
        const T di = dd ? dd[iy * n + ix] : const_inv_diag<T>(walls(ix, iy, n));
        gs_point<T, NC>(u0, u1, f0, f1, h2, di, L.omega, n, ix, iy);
    }
}

// C.f = 4-cell average of the residual of F; C.u = 0; screened levels also
// get C.k (4-cell average of F.k) and C.d
template <typename T, int NC>
__device__ void restrict_res(const Lvl<T> F, const Lvl<T> C, Thr R, bool with_k = true) {
    const int n = F.n, m = C.n;
    const T inv_h2 = F.inv_h2t;
    const T *const k = F.k;
    const T ch2 = C.h2t;
    for (Walk w(R.t0, R.nt, m); w.q < m * m; w.next()) {
        const int I = w.col, J = w.row;
        const int i0 = (2 * J) * n + 2 * I;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const T *u = F.u[c];
            const T *f = F.f[c];
            T s = f[i0] - apply_op(u, k, n, inv_h2, 2 * I, 2 * J);
            s += f[i0 + 1] - apply_op(u, k, n, inv_h2, 2 * I + 1, 2 * J);
            s += f[i0 + n] - apply_op(u, k, n, inv_h2, 2 * I, 2 * J + 1);
            s += f[i0 + n + 1] - apply_op(u, k, n, inv_h2, 2 * I + 1, 2 * J + 1);
            C.f[c][w.q] = T(0.25) * s;
            C.u[c][w.q] = T(0);
        }
        if (k && with_k) {
            const T kk = T(0.25) * (k[i0] + k[i0 + 1] + k[i0 + n] + k[i0 + n + 1]);
            C.k[w.q] = kk;
            C.d[w.q] = T(1) / (T(4 + walls(I, J, m)) + ch2 * kk);
        }
    }
}

// bilinear cell-centred interpolation of the coarse array uc (side m, odd
// ghosts) at fine cell (ix, iy)
template <typename T>
__device__ __forceinline__ T bilinear(const T *uc, int m, int ix, int iy) {
    const int I = ix >> 1, J = iy >> 1;
    const int I2 = I + ((ix & 1) ? 1 : -1);
    const int J2 = J + ((iy & 1) ? 1 : -1);
    const bool xin = (I2 >= 0 && I2 < m), yin = (J2 >= 0 && J2 < m);
    const T v00 = uc[J * m + I];
    const T v10 = xin ? uc[J * m + I2] : -v00;
    const T v01 = yin ? uc[J2 * m + I] : -v00;
    T v11;
    if (xin && yin) v11 = uc[J2 * m + I2];
    else if (xin) v11 = -uc[J * m + I2];
    else if (yin) v11 = -uc[J2 * m + I];
    else v11 = v00;
    return (T(9) * v00 + T(3) * v10 + T(3) * v01 + v11) * T(0.0625);
}

// F.u += bilinear interpolation of C.u
template <typename T, int NC>
__device__ void prolong_add(const Lvl<T> F, const Lvl<T> C, Thr R) {
    const int n = F.n, m = C.n;
    for (Walk w(R.t0, R.nt, n); w.q < n * n; w.next()) {
#pragma unroll
        for (int c = 0; c < NC; ++c) F.u[c][w.q] += bilinear(C.u[c], m, w.col, w.row);
    }
}

// Inverse of -(lap_h - kappa) on the coarsest level (float64, row-major m x m
// with m = n^2), kept in the block's shared memory.  `ready` (shared) says
// whether `inv` holds the inverse of the current operator; the Poisson
// operator never changes, the screened one changes with kappa at each solve.
struct CoarseInv {
    double *inv;
    int *ready;
};

// Solve on the coarsest level by the calling block: x = inv * f with the
// float64 inverse, computed here by Gauss-Jordan elimination (no pivoting:
// the matrix is symmetric positive definite) when not ready.  `work` needs
// m * (2m + 1) doubles.
template <typename T, int NC>
__device__ void coarse_solve(const Lvl<T> L, double *work, CoarseInv ci) {
    const int n = L.n, m = n * n, W = 2 * m;
    if (!*ci.ready) {
        const double inv_h2 = L.inv_h2;
        double *fac = work + m * W;
        for (int e = threadIdx.x; e < m * W; e += blockDim.x) {
            const int i = e / W, j = e - i * W;
            work[e] = (j == m + i) ? 1.0 : 0.0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const int iy = i / n, ix = i - iy * n;
            work[i * W + i] = (4.0 + walls(ix, iy, n)) * inv_h2 + (L.k ? (double)L.k[i] : 0.0);
            if (ix > 0) work[i * W + i - 1] = -inv_h2;
            if (ix < n - 1) work[i * W + i + 1] = -inv_h2;
            if (iy > 0) work[i * W + i - n] = -inv_h2;
            if (iy < n - 1) work[i * W + i + n] = -inv_h2;
        }
        __syncthreads();
        __shared__ double s_inv_piv;
        for (int k = 0; k < m; ++k) {
            // one float64 divide per pivot, not one per thread
            if (threadIdx.x == 0) s_inv_piv = 1.0 / work[k * W + k];
            __syncthreads();
            const double inv_piv = s_inv_piv;
            for (int i = threadIdx.x; i < m; i += blockDim.x)
                fac[i] = (i == k) ? 0.0 : work[i * W + k] * inv_piv;
            __syncthreads();
            for (int e = threadIdx.x; e < m * (W - k); e += blockDim.x) {
                const int i = e / (W - k), j = k + (e - i * (W - k));
                if (i != k) work[i * W + j] -= fac[i] * work[k * W + j];
            }
            __syncthreads();
            for (int j = k + threadIdx.x; j < W; j += blockDim.x) work[k * W + j] *= inv_piv;
            __syncthreads();
        }
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = e / m, j = e - i * m;
            ci.inv[e] = work[i * W + m + j];
        }
        __syncthreads();
        if (threadIdx.x == 0) *ci.ready = 1;
    }
    __syncthreads();
    // -(lap - kappa) u = -f  =>  u = inv * (-f)
    for (int e = threadIdx.x; e < NC * m; e += blockDim.x) {
        const int c = e / m, i = e - c * m;
        const T *f = L.f[c];
        double s = 0.0;
        for (int j = 0; j < m; ++j) s -= ci.inv[i * m + j] * (double)f[j];
        work[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NC * m; e += blockDim.x) {
        const int c = e / m, i = e - c * m;
        L.u[c][i] = (T)work[e];
    }
    __syncthreads();
}

// Shared-memory bytes that block_vcycle needs from level lg down (levels and
// the coarse-solve work area; the CoarseInv storage is separate).
template <typename T>
__host__ __device__ inline size_t block_smem_bytes(const int *lev_n, int L, int lg, int nc_max) {
    size_t pts = 0;
    for (int l = lg; l < L; ++l) pts += (size_t)lev_n[l] * lev_n[l];
    const int mc = lev_n[L - 1] * lev_n[L - 1];
    size_t b = pts * (2 * nc_max + 2) * sizeof(T);
    b = (b + 15) & ~(size_t)15;
    return b + (size_t)mc * (2 * mc + 1) * sizeof(double);
}

// Bytes of the two coarsest-level inverses (Poisson, screened).
__host__ __device__ inline size_t coarse_inv_bytes(const int *lev_n, int L) {
    const size_t mc = (size_t)lev_n[L - 1] * lev_n[L - 1];
    return 2 * mc * mc * sizeof(double);
}

// The rest of a V-cycle from level lg down, entirely in the calling block's
// shared memory.  Level lg's right-hand side (and kappa) come from global
// memory; its initial iterate is zero unless lg == 0 (then the global u is
// the warm start).  Level lg's result is written back to global memory.
//
// With writeback == false the result stays in shared memory only: it is
// component c of level lg at ((T *)smem) + 2 * c * n_lg^2 (every block can
// then run this part redundantly and read its own copy).
// Optional sub-phase timestamps (block 0, thread 0): trace[2k] = id,
// trace[2k+1] = %globaltimer; *count is the next free entry.
struct Marks {
    int64_t *trace;
    unsigned long long *count;
    int cap;
    __device__ __forceinline__ void operator()(int id) const {
        if (!trace || blockIdx.x != 0 || threadIdx.x != 0) return;
        const unsigned long long k = *count;
        if (k < (unsigned long long)cap) {
            int64_t t;
            asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
            trace[2 * k] = id;
            trace[2 * k + 1] = t;
            *count = k + 1;
        }
    }
};

template <typename T, int NC>
__device__ void block_vcycle(const Hier<T> &H, int lg, int nu1, int nu2, void *smem,
                             CoarseInv ci, bool writeback = true,
                             Marks mark = Marks{nullptr, nullptr, 0}) {
    const int L = H.L;
    // level descriptors of the shared-memory copy, one per block (a
    // per-thread array indexed by level would live in local memory)
    __shared__ Lvl<T> S[QS_MAX_LEV];
    __shared__ double *s_mat;
    const bool scr = H.lv[lg].k != nullptr;
    if (threadIdx.x == 0) {
        T *p = (T *)smem;
        for (int l = lg; l < L; ++l) {
            const int m = H.lv[l].n * H.lv[l].n;
            S[l].n = H.lv[l].n;
            S[l].h2 = H.lv[l].h2;
            S[l].inv_h2 = H.lv[l].inv_h2;
            S[l].h2t = H.lv[l].h2t;
            S[l].inv_h2t = H.lv[l].inv_h2t;
            S[l].omega = H.lv[l].omega;
            for (int c = 0; c < 2; ++c) {
                S[l].u[c] = p;
                p += m;
                S[l].f[c] = p;
                p += m;
            }
            S[l].k = scr ? p : nullptr;
            S[l].d = scr ? p + m : nullptr;
            p += 2 * m;
        }
        const size_t off = ((size_t)((char *)p - (char *)smem) + 15) & ~(size_t)15;
        s_mat = (double *)((char *)smem + off);
    }
    __syncthreads();
    double *const mat = s_mat;
    const Lvl<T> G = H.lv[lg];
    const Lvl<T> S0 = S[lg];
    const int m0 = G.n * G.n;
    for (int i = threadIdx.x; i < m0; i += blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (lg == 0) cp_async(S0.u[c] + i, G.u[c] + i, true);
            else S0.u[c][i] = T(0);
            cp_async(S0.f[c] + i, G.f[c] + i, true);
        }
        if (scr) {
            cp_async(S0.k + i, G.k + i, true);
            cp_async(S0.d + i, G.d + i, true);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    mark(40);
    const Thr B{(int)threadIdx.x, (int)blockDim.x};
    for (int l = lg; l < L - 1; ++l) {
        const Lvl<T> Sl = S[l], Sc = S[l + 1];
        for (int s = 0; s < nu1; ++s) {
            relax_half<T, NC>(Sl, 0, B);
            __syncthreads();
            relax_half<T, NC>(Sl, 1, B);
            __syncthreads();
        }
        restrict_res<T, NC>(Sl, Sc, B);
        __syncthreads();
        mark(41 + l - lg);
    }
    coarse_solve<T, NC>(S[L - 1], mat, ci);
    mark(50);
    for (int l = L - 2; l >= lg; --l) {
        const Lvl<T> Sl = S[l], Sc = S[l + 1];
        prolong_add<T, NC>(Sl, Sc, B);
        __syncthreads();
        for (int s = 0; s < nu2; ++s) {
            relax_half<T, NC>(Sl, 0, B);
            __syncthreads();
            relax_half<T, NC>(Sl, 1, B);
            __syncthreads();
        }
        mark(51 + l - lg);
    }
    if (writeback) {
        for (int i = threadIdx.x; i < m0; i += blockDim.x) {
#pragma unroll
            for (int c = 0; c < NC; ++c) G.u[c][i] = S0.u[c][i];
        }
        __syncthreads();
    }
}

}  // namespace qsmg
