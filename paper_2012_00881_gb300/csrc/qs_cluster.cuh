// Multigrid solves of small grids inside one thread-block cluster (float64).
//
// On a grid of side N <= 64 a slice's solve has a few thousand cells per
// level: spread over the whole GPU each red-black half sweep is a few
// microseconds of grid barrier for a fraction of a microsecond of work.  Here
// the first cluster of the launch (C thread blocks, C = 8 or 16) solves alone:
// the finer levels are distributed as strips of whole rows over the blocks'
// shared memory, a stencil at a strip's first or last row reads the
// neighbouring strip through distributed shared memory, and the half sweeps
// are separated by cluster barriers (a quarter of a microsecond on GB300).
// Levels whose strips would be thinner than two rows are gathered into block
// 0 of the cluster and relaxed there, down to the coarsest level's cached
// dense inverse.  Float64 work is throughput-bound here (GB300 issues about
// two float64 multiply-adds per clock per SM), so every level keeps all of a
// block's warps busy and kappa is restricted only in a solve's first cycle.  The cycle is the grid path's V(nu1, nu2): the same
// over-relaxed red-black sweeps, 4-cell restriction (of the residual and of
// kappa), bilinear prolongation with odd ghosts, and the same stopping test.
// The other blocks of the launch wait at the grid barrier that follows.
#pragma once

#include <cooperative_groups.h>

#include "qs_mg.cuh"

namespace qsclu {

namespace cg = cooperative_groups;
using qsmg::Lvl;

// One distributed level as seen by one block: the block's strip of rows
// [row0, row0 + R) of an n x n level (R * n values per array), and the
// strips of the blocks above (rank - 1, rows just before row0) and below
// (rank + 1) mapped into this block's address space (nullptr at a wall).
struct DLvl {
    double *u[2], *f[2], *k, *d;
    const double *up_u[2], *dn_u[2];  // neighbour strips of u (same layout)
    const double *up_k, *dn_k;        // neighbour strips of kappa (screened)
    int n, R, row0;
    double h2, inv_h2, omega;
};

// Shared-memory layout (identical in every block of the cluster, so a
// neighbour's array is this block's offset mapped to its rank):
//   for each distributed level l < ld: u0, u1, f0, f1, k, d, R_l * n_l each;
//   the local levels ld .. L-1 (block 0 only uses them): u0, u1, f0, f1, k, d;
//   slots[C][4] for the norm reduction; work for the coarsest solve.
struct Layout {
    int C, ld, L;
    int n[QS_MAX_LEV], R[QS_MAX_LEV];
    size_t off[QS_MAX_LEV];  // byte offset of level l's first array
    size_t slots, work, total;
};

// ld: the first level not distributed (strips must be even, >= 2 rows, and
// the side even); the local levels need the coarsest inverse's work area.
__host__ __device__ inline Layout cluster_layout(const int *lev_n, int L, int C) {
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
        o += (size_t)6 * y.R[l] * y.n[l] * sizeof(double);
    }
    y.slots = o;
    o += (size_t)C * 4 * sizeof(double);
    y.work = o;
    const size_t mc = (size_t)lev_n[L - 1] * lev_n[L - 1];
    o += mc * (2 * mc + 1) * sizeof(double);
    y.total = (o + 255) & ~(size_t)255;
    return y;
}

__device__ __forceinline__ double *arr(void *base, const Layout &y, int l, int a) {
    return (double *)((char *)base + y.off[l]) + (size_t)a * y.R[l] * y.n[l];
}

// value of u at global row gy (gy in [row0 - 1, row0 + R]) and column x of a
// distributed level: the local strip, or the neighbour's edge row, or the odd
// ghost beyond a wall (handled by the caller through the wall count)
__device__ __forceinline__ double row_val(const DLvl &L, int c, int gy, int x) {
    const int ly = gy - L.row0;
    if (ly >= 0 && ly < L.R) return L.u[c][ly * L.n + x];
    if (ly < 0) return L.up_u[c][(L.R - 1) * L.n + x];
    return L.dn_u[c][x];
}

// neighbour sum of u at (x, gy) (zero ghosts: the wall count goes into the
// diagonal, as qsmg::apply_op)
__device__ __forceinline__ double nb_sum(const DLvl &L, int c, int x, int gy, int i) {
    const int n = L.n;
    double nb = 0.0;
    if (x > 0) nb += L.u[c][i - 1];
    if (x < n - 1) nb += L.u[c][i + 1];
    if (gy > 0) nb += row_val(L, c, gy - 1, x);
    if (gy < n - 1) nb += row_val(L, c, gy + 1, x);
    return nb;
}

// one red-black half sweep of `color` on the block's strip
template <int NC>
__device__ void d_relax(const DLvl &L, int color) {
    const int n = L.n, hn = n >> 1, cnt = L.R * hn;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int ly = q / hn, gy = L.row0 + ly;
        const int x = 2 * (q - ly * hn) + ((gy + color) & 1);
        const int i = ly * n + x;
        const double di = L.d ? L.d[i] : qsmg::const_inv_diag<double>(qsmg::walls(x, gy, n));
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double g = (nb_sum(L, c, x, gy, i) - L.h2 * L.f[c][i]) * di;
            const double uo = L.u[c][i];
            L.u[c][i] = uo + L.omega * (g - uo);
        }
    }
}

// residual f - (lap - kappa) u at a strip cell
__device__ __forceinline__ double d_res(const DLvl &L, int c, int x, int gy, int i) {
    const double uc = L.u[c][i];
    double r = (nb_sum(L, c, x, gy, i) - (double)(4 + qsmg::walls(x, gy, L.n)) * uc) * L.inv_h2;
    if (L.k) r -= L.k[i] * uc;
    return L.f[c][i] - r;
}

// 4-cell restriction of the residual (and of kappa) from the strip of F into
// the coarse arrays cf[c], ck, cd of a level of side m whose rows start at
// coarse row crow0 in those arrays (the coarse strip, or a whole local level
// of block 0 reached through distributed shared memory); cu is cleared
template <int NC>
__device__ void d_restrict(const DLvl &F, int m, int crow0, double *const cu[2],
                           double *const cf[2], double *ck, double *cd, double ch2,
                           bool with_k) {
    const int n = F.n, CR = F.R >> 1, cnt = CR * m;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int lJ = q / m, I = q - lJ * m;
        const int J = (F.row0 >> 1) + lJ;  // global coarse row
        const int ly = 2 * lJ, gy = F.row0 + ly;
        const int i0 = ly * n + 2 * I;
        const int ci = (J - crow0) * m + I;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double s = d_res(F, c, 2 * I, gy, i0) + d_res(F, c, 2 * I + 1, gy, i0 + 1) +
                       d_res(F, c, 2 * I, gy + 1, i0 + n) +
                       d_res(F, c, 2 * I + 1, gy + 1, i0 + n + 1);
            cf[c][ci] = 0.25 * s;
            cu[c][ci] = 0.0;
        }
        if (F.k && with_k) {  // kappa is fixed during a solve: its first cycle
            const double kk = 0.25 * (F.k[i0] + F.k[i0 + 1] + F.k[i0 + n] + F.k[i0 + n + 1]);
            ck[ci] = kk;
            cd[ci] = 1.0 / ((double)(4 + qsmg::walls(I, J, m)) + ch2 * kk);
        }
    }
}

// coarse value at global (I, J) of a distributed coarse level C (J within
// one row of C's strip) with odd ghosts outside the domain
__device__ __forceinline__ double c_at(const DLvl &C, int c, int I, int J) {
    return row_val(C, c, J, I);
}

// F.u += bilinear prolongation of a distributed coarse level C
template <int NC>
__device__ void d_prolong_d(const DLvl &F, const DLvl &C) {
    const int n = F.n, m = C.n, cnt = F.R * n;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int ly = q / n, x = q - ly * n, gy = F.row0 + ly;
        const int I = x >> 1, J = gy >> 1;
        const int I2 = I + ((x & 1) ? 1 : -1);
        const int J2 = J + ((gy & 1) ? 1 : -1);
        const bool xin = I2 >= 0 && I2 < m, yin = J2 >= 0 && J2 < m;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double v00 = c_at(C, c, I, J);
            const double v10 = xin ? c_at(C, c, I2, J) : -v00;
            const double v01 = yin ? c_at(C, c, I, J2) : -v00;
            double v11;
            if (xin && yin) v11 = c_at(C, c, I2, J2);
            else if (xin) v11 = -c_at(C, c, I2, J);
            else if (yin) v11 = -c_at(C, c, I, J2);
            else v11 = v00;
            F.u[c][q] += (9.0 * v00 + 3.0 * v10 + 3.0 * v01 + v11) * 0.0625;
        }
    }
}

// F.u += bilinear prolongation of a whole coarse level held by block 0
// (uc0, uc1 mapped through distributed shared memory)
template <int NC>
__device__ void d_prolong_w(const DLvl &F, const double *uc0, const double *uc1, int m) {
    const int n = F.n, cnt = F.R * n;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int ly = q / n, x = q - ly * n, gy = F.row0 + ly;
        F.u[0][q] += qsmg::bilinear(uc0, m, x, gy);
        if (NC > 1) F.u[1][q] += qsmg::bilinear(uc1, m, x, gy);
    }
}

}  // namespace qsclu
