// Multigrid V-cycles inside thread-block clusters.
//
// On small grids (and for the float32 inner cycles of the refined form) a
// V-cycle spread over the whole GPU is a chain of short phases, each a grid
// barrier of one to two microseconds for a fraction of a microsecond of work.
// Here a cluster of C thread blocks (C = 8 or 16) runs the cycle of one
// component alone: the finer levels are distributed as strips of whole rows
// over the blocks' shared memory, a stencil at a strip's first or last row
// reads the neighbouring strip through distributed shared memory, and the half
// sweeps are separated by cluster barriers (a quarter of a microsecond on
// GB300).  A 2-component solve uses two clusters, one per component (the
// components share the operator but not their iterates).  Levels whose strips
// would be thinner than two rows are gathered into block 0 of the cluster and
// relaxed there by the whole block, down to the coarsest level's cached dense
// inverse.  The cycle is the grid path's V(nu1, nu2): over-relaxed red-black
// sweeps, 4-cell restriction of the residual (kappa restricted in a solve's
// first cycle only: it is fixed during a solve), bilinear prolongation with
// odd ghosts.  T is the storage type of the cycle (double, or float for the
// refined form's inner cycles); the coarsest solve is float64.
#pragma once

#include <cooperative_groups.h>

#include "qs_mg.cuh"

namespace qsclu {

namespace cg = cooperative_groups;
using qsmg::Lvl;

// One distributed level as seen by one block: the block's strip of rows
// [row0, row0 + R) of an n x n level (R * n values per array), and the u
// strips of the blocks above (rank - 1, the rows just before row0) and below
// (rank + 1) mapped into this block's address space (nullptr at a wall).
template <typename T>
struct DLvl {
    T *u, *f, *k, *d;
    const T *up_u, *dn_u;
    int n, R, row0;
    T h2, inv_h2, omega;
};

// Shared-memory layout (identical in every block of the cluster, so a
// neighbour's array is this block's offset mapped to its rank): for every
// level, u, f, kappa, inverse diagonal (R_l * n_l values each in the storage
// type; a local level has R = n); slots[C][2] for the norm reduction
// (float64); the coarsest solve's work area (float64).
struct Layout {
    int C, ld, L;
    int n[QS_MAX_LEV], R[QS_MAX_LEV];
    size_t off[QS_MAX_LEV];  // byte offset of level l's first array
    size_t slots, work, total;
};

// ld: the first level not distributed (a distributed level's strips are
// even and at least two rows, so restriction stays inside a block).
__host__ __device__ inline Layout cluster_layout(const int *lev_n, int L, int C, int tsize) {
    Layout y;
    y.C = C;
    y.L = L;
    int ld = 0;
    while (ld < L - 1 && lev_n[ld] % (2 * C) == 0 && lev_n[ld] / C >= 2) ++ld;
    y.ld = ld;
    size_t o = 0;
    for (int l = 0; l < L; ++l) {
        y.n[l] = lev_n[l];
        y.R[l] = l < ld ? lev_n[l] / C : lev_n[l];
        y.off[l] = o;
        o += (size_t)4 * y.R[l] * y.n[l] * tsize;
        o = (o + 15) & ~(size_t)15;
    }
    y.slots = o;
    o += (size_t)C * 2 * sizeof(double);
    y.work = o;
    const size_t mc = (size_t)lev_n[L - 1] * lev_n[L - 1];
    o += mc * (2 * mc + 1) * sizeof(double);
    y.total = (o + 255) & ~(size_t)255;
    return y;
}

template <typename T>
__device__ __forceinline__ T *arr(void *base, const Layout &y, int l, int a) {
    return (T *)((char *)base + y.off[l]) + (size_t)a * y.R[l] * y.n[l];
}

// u at global row gy (gy in [row0 - 1, row0 + R]) and column x: the local
// strip or a neighbour's edge row (walls are handled by the caller)
template <typename T>
__device__ __forceinline__ T row_val(const DLvl<T> &L, int gy, int x) {
    const int ly = gy - L.row0;
    if (ly >= 0 && ly < L.R) return L.u[ly * L.n + x];
    if (ly < 0) return L.up_u[(L.R - 1) * L.n + x];
    return L.dn_u[x];
}

// neighbour sum of u at (x, gy) (zero ghosts: the wall count goes into the
// diagonal, as qsmg::apply_op)
template <typename T>
__device__ __forceinline__ T nb_sum(const DLvl<T> &L, int x, int gy, int i) {
    const int n = L.n;
    T nb = T(0);
    if (x > 0) nb += L.u[i - 1];
    if (x < n - 1) nb += L.u[i + 1];
    if (gy > 0) nb += row_val(L, gy - 1, x);
    if (gy < n - 1) nb += row_val(L, gy + 1, x);
    return nb;
}

// one red-black half sweep of `color` on the block's strip
template <typename T>
__device__ void d_relax(const DLvl<T> &L, int color) {
    const int n = L.n, hn = n >> 1, cnt = L.R * hn;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int ly = q / hn, gy = L.row0 + ly;
        const int x = 2 * (q - ly * hn) + ((gy + color) & 1);
        const int i = ly * n + x;
        const T di = L.d ? L.d[i] : qsmg::const_inv_diag<T>(qsmg::walls(x, gy, n));
        const T g = (nb_sum(L, x, gy, i) - L.h2 * L.f[i]) * di;
        const T uo = L.u[i];
        L.u[i] = uo + L.omega * (g - uo);
    }
}

// residual f - (lap - kappa) u at a strip cell
template <typename T>
__device__ __forceinline__ T d_res(const DLvl<T> &L, int x, int gy, int i) {
    const T uc = L.u[i];
    T r = (nb_sum(L, x, gy, i) - T(4 + qsmg::walls(x, gy, L.n)) * uc) * L.inv_h2;
    if (L.k) r -= L.k[i] * uc;
    return L.f[i] - r;
}

// 4-cell restriction of the residual (and, with_k, of kappa) from the strip
// of F into coarse arrays cu (cleared), cf, ck, cd of a level of side m whose
// rows start at coarse row crow0 in those arrays (the coarse strip of this
// block, or the whole first local level of block 0 reached through
// distributed shared memory)
template <typename T>
__device__ void d_restrict(const DLvl<T> &F, int m, int crow0, T *cu, T *cf, T *ck, T *cd,
                           T ch2, bool with_k) {
    const int n = F.n, cnt = (F.R >> 1) * m;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int lJ = q / m, I = q - lJ * m;
        const int J = (F.row0 >> 1) + lJ;  // global coarse row
        const int ly = 2 * lJ, gy = F.row0 + ly;
        const int i0 = ly * n + 2 * I;
        const int ci = (J - crow0) * m + I;
        const T s = d_res(F, 2 * I, gy, i0) + d_res(F, 2 * I + 1, gy, i0 + 1) +
                    d_res(F, 2 * I, gy + 1, i0 + n) + d_res(F, 2 * I + 1, gy + 1, i0 + n + 1);
        cf[ci] = T(0.25) * s;
        cu[ci] = T(0);
        if (F.k && with_k) {
            const T kk = T(0.25) * (F.k[i0] + F.k[i0 + 1] + F.k[i0 + n] + F.k[i0 + n + 1]);
            ck[ci] = kk;
            cd[ci] = T(1) / (T(4 + qsmg::walls(I, J, m)) + ch2 * kk);
        }
    }
}

// F.u += bilinear prolongation of a distributed coarse level C (a coarse row
// within one row of C's strip)
template <typename T>
__device__ void d_prolong_d(const DLvl<T> &F, const DLvl<T> &C) {
    const int n = F.n, m = C.n, cnt = F.R * n;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int ly = q / n, x = q - ly * n, gy = F.row0 + ly;
        const int I = x >> 1, J = gy >> 1;
        const int I2 = I + ((x & 1) ? 1 : -1);
        const int J2 = J + ((gy & 1) ? 1 : -1);
        const bool xin = I2 >= 0 && I2 < m, yin = J2 >= 0 && J2 < m;
        const T v00 = row_val(C, J, I);
        const T v10 = xin ? row_val(C, J, I2) : -v00;
        const T v01 = yin ? row_val(C, J2, I) : -v00;
        T v11;
        if (xin && yin) v11 = row_val(C, J2, I2);
        else if (xin) v11 = -row_val(C, J, I2);
        else if (yin) v11 = -row_val(C, J2, I);
        else v11 = v00;
        F.u[q] += (T(9) * v00 + T(3) * v10 + T(3) * v01 + v11) * T(0.0625);
    }
}

// F.u += bilinear prolongation of a whole coarse level held by block 0 (uc
// mapped through distributed shared memory)
template <typename T>
__device__ void d_prolong_w(const DLvl<T> &F, const T *uc, int m) {
    const int n = F.n, cnt = F.R * n;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int ly = q / n, x = q - ly * n, gy = F.row0 + ly;
        F.u[q] += qsmg::bilinear(uc, m, x, gy);
    }
}

}  // namespace qsclu
