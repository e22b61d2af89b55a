// Multigrid field solver on a nonuniform transverse grid (Sec. "Multigrid
// Solver with Nonuniform Grids").
//
// Operator.  On nodes x_i with spacings h^- = x_i - x_{i-1}, h^+ = x_{i+1} - x_i
// the equation (d_xx + d_yy) Psi + M Psi = J is discretised with the
// three-point second difference D2 of Eq. 2D_Laplac and its third-order term
// replaced as in Eq. 2D_Laplac_3rd (mixed third derivatives as the first
// difference D1 of the other axis' D2, d(lap) as D1 of J - M Psi):
//     A   = D2x + D2y + M + cx (D1x D2y + D1x M) + cy (D1y D2x + D1y M)
//     J'  = J + (cx D1x + cy D1y) J,           c = (h^+ - h^-) / 3.
// The third-order term enters with a minus sign (the Taylor expansion of D2 is
// d^2 + (h^b/3) d^3), and the y bracket carries h_y^b.  With correction off,
// c = 0.  Walls are nodes with Psi = 0 and J = 0.  A couples the 3x3
// neighbourhood of a node and is not symmetric.
//
// Multigrid.  n = 2^k - 1 nodes per side; a coarse level keeps every other
// node (the walls stay), so its spacings are sums of two fine ones and its
// operator is the same 9-point formula on the coarse nodes.  Prolongation is
// linear interpolation in physical coordinates (tensor product); restriction
// is its dual-volume-weighted transpose (every row sums to 1) and also carries
// M down.  The smoother is four-colour Gauss-Seidel: colour (i & 1, j & 1),
// since the corner couplings of the 9-point stencil would join points of one
// red-black colour; it is over-relaxed (omega = 1.3 by default, which halves
// the cycles on grids with 3:1 cells, where point smoothing is weakest).  The
// coarsest level (3 x 3) is solved exactly with its inverse, formed once per
// solve.
//
// Execution.  One persistent cooperative launch per solve: 152 blocks on a
// bounded software grid barrier for the levels larger than local_n (31 by
// default), block 0 on __syncthreads for the rest.  Smoothing is staged in
// shared memory: a level's down leg (pre-sweeps, residual, restriction) and up
// leg (prolongation, post-sweeps) each run on tiles with a recomputed halo of
// 4 max(nu1, nu2) + 2 nodes, one grid barrier per leg instead of one per
// colour; the block-0 levels are staged whole.  Grid-wide colour sweeps (a
// barrier per colour) remain for settings whose tiles do not fit.
//
// Forms.  FP64 cycles on a float64 hierarchy.  The refined form keeps the
// solution, J' and the residual in float64 and cycles in float32 on the
// residual equation (iterative refinement): every outer step is one float32
// V-cycle for the correction, u += e, then the float64 residual, which is
// also the stopping test, so both forms stop at the same float64 accuracy.
//
// Every wait is bounded; a timeout sets an error word that ends the kernel at
// the next barrier.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <new>
#include <vector>

#include "qs.h"
#include "qs_grid_sync.cuh"

namespace {

constexpr int kMaxLevels = 12;      // n <= 4095
constexpr int kMaxRhs = 4;
constexpr int kThreads = 512;
constexpr int kDefaultLocalN = 31;  // levels this small run in one block
constexpr int kDefaultNu1 = 2, kDefaultNu2 = 2;  // V(2,2)
constexpr double kDefaultOmega = 1.3;
constexpr size_t kStageSmemMax = 200 * 1024;  // dynamic shared memory of staged tiles
constexpr long long kBarrierLimit = 4000000000LL;  // clock cycles, ~2 s

// Per-node coefficients of one axis: D2 (at i-1, i, i+1), D1 (same), c.
template <typename T>
struct AxisCoef {
    T d2[3];
    T d1[3];
    T c;
    T pad;
};

// One level of a hierarchy in precision T.
template <typename T>
struct Level {
    int n;
    const AxisCoef<T> *ax, *ay;  // n each
    const T *pwx, *pwy;          // prolongation weights (2 per node; even nodes used)
    const T *rwx, *rwy;          // restriction weights to the next coarser level (3 per coarse node)
    T *u, *f, *r;                // kMaxRhs * n * n
    T *m, *idiag;                // n * n (m: nullptr when M = 0)
};

struct NuScalars {
    unsigned long long bar;
    int err;
    int err_where;
    int cycles;
    int converged;
    double norm[3][kMaxRhs];  // rotating residual-norm slots
    double fnorm[kMaxRhs];
    double relres[kMaxRhs];
};

struct NuArgs {
    // The float64 finest level: the caller's u and M, J' and float64
    // coefficients.  The FP64 form cycles on h64 (whose level 0 is `top`
    // with residual and diagonal arrays); the refined form keeps `top` for
    // the residual and the update and cycles on h32.
    Level<double> top;
    Level<double> h64[kMaxLevels];
    Level<float> h32[kMaxLevels];
    int levels;
    int nrhs;
    int has_m;
    int max_cycles;
    int nu1, nu2;             // pre- and post-smoothing sweeps
    double omega;             // Gauss-Seidel relaxation factor (folded into idiag)
    int local_n;              // levels of side <= local_n run in block 0 alone
    int staged;               // levels smoothed in shared-memory tiles
    int halo;                 // staged tiles' halo: 4 max(nu1, nu2) + 2
    int stage_cap;            // nodes a staged region may hold
    double tol;
    const double *j;          // caller's sources (solve) / input (apply, source)
    const double *m_in;       // caller's M or nullptr
    double *coarse_inv;       // 81 entries (double or float): inverse of the 3 x 3 level
    NuScalars *sc;
};

template <typename T> __device__ __forceinline__ const Level<T> *hier(const NuArgs &A);
template <> __device__ __forceinline__ const Level<double> *hier<double>(const NuArgs &A) {
    return A.h64;
}
template <> __device__ __forceinline__ const Level<float> *hier<float>(const NuArgs &A) {
    return A.h32;
}

using qsync::BlockSync;
using qsync::Team;
using qsync::vload;
using GridBarrier = qsync::GridBarrier<NuScalars>;

template <typename T>
__device__ __forceinline__ T at(const T *u, int n, int i, int j) {
    return (i < 0 || j < 0 || i >= n || j >= n) ? T(0) : u[j * n + i];
}

// (A u)(i, j) of one field; mrow/mcol are M at (i+a, j) and (i, j+b).
template <bool CORR, typename T>
__device__ __forceinline__ T apply_point(const AxisCoef<T> &cx, const AxisCoef<T> &cy,
                                         const T (&v)[3][3], const T (&mrow)[3],
                                         const T (&mcol)[3], T m0) {
    T lx[3], ly[3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
        lx[b] = cx.d2[0] * v[b][0] + cx.d2[1] * v[b][1] + cx.d2[2] * v[b][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        ly[a] = cy.d2[0] * v[0][a] + cy.d2[1] * v[1][a] + cy.d2[2] * v[2][a];
    T s = lx[1] + ly[1] + m0 * v[1][1];
    if (CORR) {
        T tx = T(0), ty = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) tx += cx.d1[a] * (ly[a] + mrow[a] * v[1][a]);
#pragma unroll
        for (int b = 0; b < 3; ++b) ty += cy.d1[b] * (lx[b] + mcol[b] * v[b][1]);
        s += cx.c * tx + cy.c * ty;
    }
    return s;
}

template <typename T>
__device__ __forceinline__ void load_m(const T *m, int n, int i, int j, T (&mrow)[3],
                                       T (&mcol)[3], T &m0) {
    if (m) {
        m0 = m[j * n + i];
        mrow[0] = at(m, n, i - 1, j);
        mrow[1] = m0;
        mrow[2] = at(m, n, i + 1, j);
        mcol[0] = at(m, n, i, j - 1);
        mcol[1] = m0;
        mcol[2] = at(m, n, i, j + 1);
    } else {
        m0 = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) mrow[k] = mcol[k] = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void load_v(const T *u, int n, int i, int j, T (&v)[3][3]) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) v[b][a] = at(u, n, i + a - 1, j + b - 1);
}

// Diagonal of A at (i, j): the coefficient of u(i, j) in apply_point.
template <bool CORR, typename T>
__device__ __forceinline__ T diag_point(const AxisCoef<T> &cx, const AxisCoef<T> &cy, T m0) {
    T d = cx.d2[1] + cy.d2[1] + m0;
    if (CORR) d += cx.c * cx.d1[1] * (cy.d2[1] + m0) + cy.c * cy.d1[1] * (cx.d2[1] + m0);
    return d;
}

// J' = J + (cx D1x + cy D1y) J at (i, j) of one field.
template <bool CORR>
__device__ __forceinline__ double corrected_source(const Level<double> &L, const double *jc,
                                                   int i, int j) {
    const int n = L.n;
    double fv = jc[j * n + i];
    if (CORR) {
        const AxisCoef<double> &cx = L.ax[i], &cy = L.ay[j];
        const double dx =
            cx.d1[0] * at(jc, n, i - 1, j) + cx.d1[1] * fv + cx.d1[2] * at(jc, n, i + 1, j);
        const double dy =
            cy.d1[0] * at(jc, n, i, j - 1) + cy.d1[1] * fv + cy.d1[2] * at(jc, n, i, j + 1);
        fv += cx.c * dx + cy.c * dy;
    }
    return fv;
}

// One colour of Gauss-Seidel on all fields: points with (i & 1, j & 1) = (ci, cj).
template <bool CORR, typename T>
__device__ void gs_colour(const Level<T> &L, int nrhs, int ci, int cj, Team tm) {
    const int n = L.n;
    const int ni = (n - ci + 1) / 2, nj = (n - cj + 1) / 2;
    const int cnt = ni * nj;
    for (int p = tm.t; p < cnt; p += tm.nt) {
        const int jj = p / ni;
        const int i = 2 * (p - jj * ni) + ci, j = 2 * jj + cj;
        const AxisCoef<T> &cx = L.ax[i], &cy = L.ay[j];
        T mrow[3], mcol[3], m0;
        load_m(L.m, n, i, j, mrow, mcol, m0);
        const T id = L.idiag[j * n + i];
        for (int c = 0; c < nrhs; ++c) {
            T *u = L.u + (size_t)c * n * n;
            T v[3][3];
            load_v(u, n, i, j, v);
            const T res = L.f[(size_t)c * n * n + j * n + i] -
                          apply_point<CORR>(cx, cy, v, mrow, mcol, m0);
            u[j * n + i] = v[1][1] + res * id;
        }
    }
}

template <bool CORR, typename T, typename Sync>
__device__ bool smooth(const Level<T> &L, int nrhs, int sweeps, Team tm, const Sync &sync,
                       int where) {
    for (int s = 0; s < sweeps; ++s)
        for (int col = 0; col < 4; ++col) {
            gs_colour<CORR>(L, nrhs, col & 1, col >> 1, tm);
            if (!sync(where)) return false;
        }
    return true;
}

// r = f - A u on a level.
template <bool CORR, typename T>
__device__ void residual(const Level<T> &L, int nrhs, Team tm) {
    const int n = L.n;
    for (int p = tm.t; p < n * n; p += tm.nt) {
        const int j = p / n, i = p - j * n;
        T mrow[3], mcol[3], m0;
        load_m(L.m, n, i, j, mrow, mcol, m0);
        for (int c = 0; c < nrhs; ++c) {
            T v[3][3];
            load_v(L.u + (size_t)c * n * n, n, i, j, v);
            L.r[(size_t)c * n * n + p] = L.f[(size_t)c * n * n + p] -
                                         apply_point<CORR>(L.ax[i], L.ay[j], v, mrow, mcol, m0);
        }
    }
}

// Coarse f = R r (dual-length-weighted full weighting), coarse u = 0.
template <typename T>
__device__ void restrict_residual(const Level<T> &F, const Level<T> &C, int nrhs, Team tm) {
    const int nc = C.n, nf = F.n;
    for (int p = tm.t; p < nc * nc; p += tm.nt) {
        const int J = p / nc, I = p - J * nc;
        const int i = 2 * I + 1, j = 2 * J + 1;
        const T *wx = F.rwx + 3 * I, *wy = F.rwy + 3 * J;
        for (int c = 0; c < nrhs; ++c) {
            const T *r = F.r + (size_t)c * nf * nf;
            T s = T(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const T *row = r + (size_t)(j + b - 1) * nf + i - 1;
                s += wy[b] * (wx[0] * row[0] + wx[1] * row[1] + wx[2] * row[2]);
            }
            C.f[(size_t)c * nc * nc + p] = s;
            C.u[(size_t)c * nc * nc + p] = T(0);
        }
    }
}

// Fine u += P (coarse u): bilinear interpolation in physical coordinates.
template <typename T>
__device__ void prolong_correct(const Level<T> &F, const Level<T> &C, int nrhs, Team tm) {
    const int nf = F.n, nc = C.n;
    for (int p = tm.t; p < nf * nf; p += tm.nt) {
        const int j = p / nf, i = p - j * nf;
        // odd i is coarse node (i-1)/2; even i lies between (i-2)/2 and i/2
        int ix0, ix1, iy0, iy1;
        T wx0, wx1, wy0, wy1;
        if (i & 1) {
            ix0 = ix1 = (i - 1) / 2;
            wx0 = T(1);
            wx1 = T(0);
        } else {
            ix0 = (i - 2) / 2;
            ix1 = i / 2;
            wx0 = F.pwx[2 * i];
            wx1 = F.pwx[2 * i + 1];
        }
        if (j & 1) {
            iy0 = iy1 = (j - 1) / 2;
            wy0 = T(1);
            wy1 = T(0);
        } else {
            iy0 = (j - 2) / 2;
            iy1 = j / 2;
            wy0 = F.pwy[2 * j];
            wy1 = F.pwy[2 * j + 1];
        }
        for (int c = 0; c < nrhs; ++c) {
            const T *e = C.u + (size_t)c * nc * nc;
            const T v = wy0 * (wx0 * at(e, nc, ix0, iy0) + wx1 * at(e, nc, ix1, iy0)) +
                        wy1 * (wx0 * at(e, nc, ix0, iy1) + wx1 * at(e, nc, ix1, iy1));
            F.u[(size_t)c * nf * nf + p] += v;
        }
    }
}

// M of level l from level l - 1 (same weights as the residual).
template <typename T>
__device__ void restrict_m(const Level<T> &F, const Level<T> &L, Team tm) {
    const int n = L.n, nf = F.n;
    for (int p = tm.t; p < n * n; p += tm.nt) {
        const int J = p / n, I = p - J * n;
        const int i = 2 * I + 1, j = 2 * J + 1;
        const T *wx = F.rwx + 3 * I, *wy = F.rwy + 3 * J;
        T s = T(0);
        for (int b = 0; b < 3; ++b) {
            const T *row = F.m + (size_t)(j + b - 1) * nf + i - 1;
            s += wy[b] * (wx[0] * row[0] + wx[1] * row[1] + wx[2] * row[2]);
        }
        L.m[p] = s;
    }
}

// omega / diag(A): the Gauss-Seidel update is u += omega (f - A u) / diag.
template <bool CORR, typename T>
__device__ void level_idiag(const Level<T> &L, double omega, Team tm) {
    const int n = L.n;
    for (int p = tm.t; p < n * n; p += tm.nt) {
        const int j = p / n, i = p - j * n;
        const T m0 = L.m ? L.m[p] : T(0);
        L.idiag[p] = T(omega / (double)diag_point<CORR>(L.ax[i], L.ay[j], m0));
    }
}

// Inverse of the 3 x 3 level's 9 x 9 matrix by Gauss-Jordan with partial
// pivoting, in double (one thread; the columns are A applied to unit vectors).
template <bool CORR, typename T>
__device__ void coarse_inverse(const Level<T> &L, T *inv) {
    double a[9][18];
    for (int q = 0; q < 9; ++q) {
        const int j = q / 3, i = q - 3 * j;
        T mrow[3], mcol[3], m0;
        load_m(L.m, 3, i, j, mrow, mcol, m0);
        for (int col = 0; col < 9; ++col) {
            T v[3][3];
            for (int b = 0; b < 3; ++b)
                for (int aa = 0; aa < 3; ++aa) {
                    const int ii = i + aa - 1, jj = j + b - 1;
                    v[b][aa] = (ii >= 0 && jj >= 0 && ii < 3 && jj < 3 && jj * 3 + ii == col)
                                   ? T(1)
                                   : T(0);
                }
            a[q][col] = (double)apply_point<CORR>(L.ax[i], L.ay[j], v, mrow, mcol, m0);
            a[q][9 + col] = (q == col) ? 1.0 : 0.0;
        }
    }
    for (int k = 0; k < 9; ++k) {
        int piv = k;
        for (int q = k + 1; q < 9; ++q)
            if (fabs(a[q][k]) > fabs(a[piv][k])) piv = q;
        if (piv != k)
            for (int col = 0; col < 18; ++col) {
                const double t = a[k][col];
                a[k][col] = a[piv][col];
                a[piv][col] = t;
            }
        const double ip = 1.0 / a[k][k];
        for (int col = 0; col < 18; ++col) a[k][col] *= ip;
        for (int q = 0; q < 9; ++q) {
            if (q == k) continue;
            const double f = a[q][k];
            if (f != 0.0)
                for (int col = 0; col < 18; ++col) a[q][col] -= f * a[k][col];
        }
    }
    for (int q = 0; q < 9; ++q)
        for (int col = 0; col < 9; ++col) inv[q * 9 + col] = T(a[q][9 + col]);
}

template <typename T>
__device__ void coarse_solve(const Level<T> &L, const T *inv, int nrhs, Team tm) {
    for (int p = tm.t; p < 9 * nrhs; p += tm.nt) {
        const int c = p / 9, q = p - 9 * c;
        const T *f = L.f + 9 * c;
        T s = T(0);
        for (int k = 0; k < 9; ++k) s += inv[q * 9 + k] * f[k];
        L.u[9 * c + q] = s;
    }
}

// Levels from..to-1: pre-smooth, residual, restrict (team `tm`, `sync`).
template <bool CORR, typename T, typename Sync>
__device__ bool down_legs(const Level<T> *H, int nr, int nu1, int from, int to, Team tm,
                          const Sync &sync) {
    for (int l = from; l < to; ++l) {
        if (!smooth<CORR>(H[l], nr, nu1, tm, sync, 10 + l)) return false;
        residual<CORR>(H[l], nr, tm);
        if (!sync(30 + l)) return false;
        restrict_residual(H[l], H[l + 1], nr, tm);
        if (!sync(50 + l)) return false;
    }
    return true;
}

// Levels from down to `to`: prolongate-correct, post-smooth.
template <bool CORR, typename T, typename Sync>
__device__ bool up_legs(const Level<T> *H, int nr, int nu2, int from, int to, Team tm,
                        const Sync &sync) {
    for (int l = from; l >= to; --l) {
        prolong_correct(H[l], H[l + 1], nr, tm);
        if (!sync(70 + l)) return false;
        if (!smooth<CORR>(H[l], nr, nu2, tm, sync, 90 + l)) return false;
    }
    return true;
}


// ---------------------------------------------------------------------------
// Smoothing staged in shared memory.  A block takes a tile of a level, loads
// the tile plus a halo of H = 4 max(nu1, nu2) + 2 nodes (u, f, M, omega/diag;
// zero outside the domain), and runs every colour step of the sweeps there.
// Each colour step can spoil at most one more ring from the region's stale
// edge inwards, so after 4 nu steps the tile and two rings around it hold
// exactly what the grid-wide sweeps would give; the residual on the tile and
// one ring then feeds the restriction of the coarse nodes the tile owns.  A
// level's down leg (nu1 sweeps, residual, restriction) and up leg
// (prolongation, nu2 sweeps) are then one grid barrier each.
// ---------------------------------------------------------------------------
constexpr int kTileX = 32, kTileY = 16;

struct TileGeom {
    int tx, ty;               // tile size
    int ntx, nty;             // tiles per row / column
};

// Tile size of a level: 32 x 16, halved (larger side first) while the level
// has fewer than 64 tiles and the tile more than 64 nodes.
__device__ __forceinline__ TileGeom tile_geom(int n) {
    TileGeom g{kTileX, kTileY, 0, 0};
    for (;;) {
        g.ntx = (n + g.tx - 1) / g.tx;
        g.nty = (n + g.ty - 1) / g.ty;
        if (g.ntx * g.nty >= 64 || g.tx * g.ty <= 64) break;
        if (g.tx >= g.ty) g.tx /= 2;
        else g.ty /= 2;
    }
    return g;
}

// A level staged whole by one block: one tile of side n + 1 (even), halo 1.
// Every in-domain node is in the region and the ring outside it holds the
// walls' zeros, so no colour step can read a stale value.
__device__ __forceinline__ TileGeom whole_geom(int n) { return TileGeom{n + 1, n + 1, 1, 1}; }

__device__ __forceinline__ bool whole_fits(int n, int cap) { return (n + 3) * (n + 3) <= cap; }

template <typename T>
struct Region {
    int x0, y0;     // global index of the region's first node (tile origin - H)
    int rw, rh;     // region size
    int tw, th;     // tile size, clipped at the domain's end
    T *su, *sf;     // nrhs * rw * rh
    T *sm, *sd;     // rw * rh
};

template <typename T>
__device__ __forceinline__ Region<T> make_region(unsigned char *smem, int x0t, int y0t,
                                                 const TileGeom &g, int n, int halo, int nrhs) {
    Region<T> R;
    R.x0 = x0t - halo;
    R.y0 = y0t - halo;
    R.rw = g.tx + 2 * halo;
    R.rh = g.ty + 2 * halo;
    R.tw = min(g.tx, n - x0t);
    R.th = min(g.ty, n - y0t);
    const int np = R.rw * R.rh;
    T *p = reinterpret_cast<T *>(smem);
    R.su = p;
    R.sf = p + (size_t)nrhs * np;
    R.sm = p + (size_t)2 * nrhs * np;
    R.sd = p + (size_t)(2 * nrhs + 1) * np;
    return R;
}

// Region load of u (from `usrc`, or zero), f, M and omega/diag; with a coarse
// level C, u += P (coarse u) on the way in.
template <typename T>
__device__ void stage_load(const Level<T> &L, const T *usrc, const Level<T> *C,
                           const Region<T> &R, int nrhs) {
    const int n = L.n, np = R.rw * R.rh;
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const int b = q / R.rw, a = q - b * R.rw;
        const int gi = R.x0 + a, gj = R.y0 + b;
        const bool in = gi >= 0 && gj >= 0 && gi < n && gj < n;
        const int g = gj * n + gi;
        R.sm[q] = (in && L.m) ? L.m[g] : T(0);
        R.sd[q] = in ? L.idiag[g] : T(0);
        for (int c = 0; c < nrhs; ++c) {
            T uv = (in && usrc) ? usrc[(size_t)c * n * n + g] : T(0);
            if (in && C) {
                // prolongation of the coarse correction at (gi, gj)
                const int nc = C->n;
                int ix0, ix1, iy0, iy1;
                T wx0, wx1, wy0, wy1;
                if (gi & 1) {
                    ix0 = ix1 = (gi - 1) / 2;
                    wx0 = T(1);
                    wx1 = T(0);
                } else {
                    ix0 = (gi - 2) / 2;
                    ix1 = gi / 2;
                    wx0 = L.pwx[2 * gi];
                    wx1 = L.pwx[2 * gi + 1];
                }
                if (gj & 1) {
                    iy0 = iy1 = (gj - 1) / 2;
                    wy0 = T(1);
                    wy1 = T(0);
                } else {
                    iy0 = (gj - 2) / 2;
                    iy1 = gj / 2;
                    wy0 = L.pwy[2 * gj];
                    wy1 = L.pwy[2 * gj + 1];
                }
                const T *e = C->u + (size_t)c * nc * nc;
                uv += wy0 * (wx0 * at(e, nc, ix0, iy0) + wx1 * at(e, nc, ix1, iy0)) +
                      wy1 * (wx0 * at(e, nc, ix0, iy1) + wx1 * at(e, nc, ix1, iy1));
            }
            R.su[(size_t)c * np + q] = uv;
            R.sf[(size_t)c * np + q] = in ? L.f[(size_t)c * n * n + g] : T(0);
        }
    }
}

// (A u) at region node (a, b) from the staged arrays (1 <= a <= rw-2, 1 <= b <= rh-2).
template <bool CORR, typename T>
__device__ __forceinline__ T staged_apply(const Level<T> &L, const Region<T> &R, const T *u,
                                          int a, int b, T &m0) {
    const int q = b * R.rw + a;
    const int gi = R.x0 + a, gj = R.y0 + b;
    T v[3][3], mrow[3], mcol[3];
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) v[bb][aa] = u[q + (bb - 1) * R.rw + (aa - 1)];
    m0 = R.sm[q];
    mrow[0] = R.sm[q - 1];
    mrow[1] = m0;
    mrow[2] = R.sm[q + 1];
    mcol[0] = R.sm[q - R.rw];
    mcol[1] = m0;
    mcol[2] = R.sm[q + R.rw];
    return apply_point<CORR>(L.ax[gi], L.ay[gj], v, mrow, mcol, m0);
}

// The colour steps of `sweeps` sweeps on the region (every in-domain node
// whose 3 x 3 neighbourhood is staged).
template <bool CORR, typename T>
__device__ void staged_sweeps(const Level<T> &L, const Region<T> &R, int nrhs, int sweeps) {
    const int n = L.n, np = R.rw * R.rh;
    for (int s = 0; s < sweeps; ++s)
        for (int col = 0; col < 4; ++col) {
            const int ci = col & 1, cj = col >> 1;
            const int a0 = 1 + (((R.x0 + 1) & 1) != ci), b0 = 1 + (((R.y0 + 1) & 1) != cj);
            const int na = a0 <= R.rw - 2 ? (R.rw - 2 - a0) / 2 + 1 : 0;
            const int nb = b0 <= R.rh - 2 ? (R.rh - 2 - b0) / 2 + 1 : 0;
            for (int k = threadIdx.x; k < na * nb; k += blockDim.x) {
                const int kb = k / na;
                const int a = a0 + 2 * (k - kb * na), b = b0 + 2 * kb;
                const int gi = R.x0 + a, gj = R.y0 + b;
                if (gi < 0 || gj < 0 || gi >= n || gj >= n) continue;
                const int q = b * R.rw + a;
                const T id = R.sd[q];
                for (int c = 0; c < nrhs; ++c) {
                    T *u = R.su + (size_t)c * np;
                    T m0;
                    const T au = staged_apply<CORR>(L, R, u, a, b, m0);
                    u[q] += (R.sf[(size_t)c * np + q] - au) * id;
                }
            }
            __syncthreads();
        }
}

// Down leg of level l, one barrier: nu1 sweeps, residual, restriction into
// level l + 1 (f, and u = 0).  The smoothed u goes to the level's r array,
// not to u, which other blocks are still reading as halo in this phase; the
// up leg reads it from there.  `u_zero`: u is known to be zero (every level
// below the finest, and the finest of the refined form), so it is not read.
template <bool CORR, typename T>
__device__ void staged_down(const NuArgs &A, const Level<T> *H, int l, const TileGeom &g, int h,
                            bool u_zero, unsigned char *smem) {
    const Level<T> &L = H[l], &C = H[l + 1];
    const int n = L.n, nc = C.n, nr = A.nrhs;
    for (int t = blockIdx.x; t < g.ntx * g.nty; t += gridDim.x) {
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const Region<T> R = make_region<T>(smem, tx * g.tx, ty * g.ty, g, n, h, nr);
        const int np = R.rw * R.rh;
        stage_load<T>(L, u_zero ? nullptr : L.u, nullptr, R, nr);
        __syncthreads();
        staged_sweeps<CORR>(L, R, nr, A.nu1);
        // residual on the tile and one ring, in place of f
        const int rw1 = R.tw + 2, rh1 = R.th + 2;
        for (int k = threadIdx.x; k < rw1 * rh1; k += blockDim.x) {
            const int kb = k / rw1;
            const int a = h - 1 + (k - kb * rw1), b = h - 1 + kb;
            const int gi = R.x0 + a, gj = R.y0 + b;
            if (gi < 0 || gj < 0 || gi >= n || gj >= n) continue;
            const int q = b * R.rw + a;
            for (int c = 0; c < nr; ++c) {
                T m0;
                const T au = staged_apply<CORR>(L, R, R.su + (size_t)c * np, a, b, m0);
                R.sf[(size_t)c * np + q] -= au;
            }
        }
        __syncthreads();
        // smoothed u of the tile, kept in r for the up leg
        for (int k = threadIdx.x; k < R.tw * R.th; k += blockDim.x) {
            const int kb = k / R.tw;
            const int a = h + (k - kb * R.tw), b = h + kb;
            const int g0 = (R.y0 + b) * n + (R.x0 + a), q = b * R.rw + a;
            for (int c = 0; c < nr; ++c) L.r[(size_t)c * n * n + g0] = R.su[(size_t)c * np + q];
        }
        // coarse nodes of the tile: fine odd (gi, gj) inside it
        const int x0t = R.x0 + h, y0t = R.y0 + h;
        const int I0 = x0t / 2, J0 = y0t / 2;  // first coarse node with fine index >= origin
        const int I1 = min((x0t + R.tw) / 2, nc), J1 = min((y0t + R.th) / 2, nc);
        const int ni = I1 - I0;
        for (int k = threadIdx.x; k < ni * (J1 - J0); k += blockDim.x) {
            const int kJ = k / ni;
            const int I = I0 + (k - kJ * ni), J = J0 + kJ;
            const int a = 2 * I + 1 - R.x0, b = 2 * J + 1 - R.y0;
            const T *wx = L.rwx + 3 * I, *wy = L.rwy + 3 * J;
            for (int c = 0; c < nr; ++c) {
                const T *r = R.sf + (size_t)c * np + b * R.rw + a;
                T s = T(0);
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) {
                    const T *row = r + (bb - 1) * R.rw;
                    s += wy[bb] * (wx[0] * row[-1] + wx[1] * row[0] + wx[2] * row[1]);
                }
                C.f[(size_t)c * nc * nc + J * nc + I] = s;
                C.u[(size_t)c * nc * nc + J * nc + I] = T(0);
            }
        }
        __syncthreads();
    }
}

// Up leg of level l, one barrier: the down leg's smoothed u (in r) plus
// P (coarse u), nu2 sweeps, tile back to u.
template <bool CORR, typename T>
__device__ void staged_up(const NuArgs &A, const Level<T> *H, int l, const TileGeom &g, int h,
                          unsigned char *smem) {
    const Level<T> &L = H[l];
    const int n = L.n, nr = A.nrhs;
    for (int t = blockIdx.x; t < g.ntx * g.nty; t += gridDim.x) {
        const int ty = t / g.ntx, tx = t - ty * g.ntx;
        const Region<T> R = make_region<T>(smem, tx * g.tx, ty * g.ty, g, n, h, nr);
        const int np = R.rw * R.rh;
        stage_load<T>(L, L.r, &H[l + 1], R, nr);
        __syncthreads();
        staged_sweeps<CORR>(L, R, nr, A.nu2);
        for (int k = threadIdx.x; k < R.tw * R.th; k += blockDim.x) {
            const int kb = k / R.tw;
            const int a = h + (k - kb * R.tw), b = h + kb;
            const int g0 = (R.y0 + b) * n + (R.x0 + a), q = b * R.rw + a;
            for (int c = 0; c < nr; ++c) L.u[(size_t)c * n * n + g0] = R.su[(size_t)c * np + q];
        }
        __syncthreads();
    }
}

// One V-cycle on hierarchy H: the grid-wide levels 0..loc-1, then block 0
// alone from loc to the exact coarsest solve and back.
template <bool CORR, typename T>
__device__ bool vcycle(const NuArgs &A, const Level<T> *H, int loc, Team grid, Team blk,
                       const GridBarrier &gsync) {
    const int nr = A.nrhs, Lc = A.levels - 1;
    const T *inv = reinterpret_cast<const T *>(A.coarse_inv);
    if (Lc == 0) {
        if (blockIdx.x == 0) coarse_solve(H[0], inv, nr, blk);
        return gsync(3);
    }
    extern __shared__ __align__(16) unsigned char nu_dsmem[];
    if (!A.staged) {
        if (!down_legs<CORR>(H, nr, A.nu1, 0, loc, grid, gsync)) return false;
        if (blockIdx.x == 0) {
            const BlockSync bs;
            down_legs<CORR>(H, nr, A.nu1, loc, Lc, blk, bs);
            coarse_solve(H[Lc], inv, nr, blk);
            __syncthreads();
            up_legs<CORR>(H, nr, A.nu2, Lc - 1, loc, blk, bs);
        }
        if (!gsync(3)) return false;
        return loc == 0 || up_legs<CORR>(H, nr, A.nu2, loc - 1, 0, grid, gsync);
    }
    // staged: grid-wide levels in tiles, the block-0 levels whole where they
    // fit (else with block-wide colour sweeps through global memory)
    for (int l = 0; l < loc; ++l) {
        staged_down<CORR, T>(A, H, l, tile_geom(H[l].n), A.halo, l > 0 || sizeof(T) == 4,
                             nu_dsmem);
        if (!gsync(60 + l)) return false;
    }
    if (blockIdx.x == 0) {
        const BlockSync bs;
        for (int l = loc; l < Lc; ++l) {
            if (whole_fits(H[l].n, A.stage_cap))
                staged_down<CORR, T>(A, H, l, whole_geom(H[l].n), 1, l > 0 || sizeof(T) == 4,
                                     nu_dsmem);
            else
                down_legs<CORR>(H, nr, A.nu1, l, l + 1, blk, bs);
            __syncthreads();
        }
        coarse_solve(H[Lc], inv, nr, blk);
        __syncthreads();
        for (int l = Lc - 1; l >= loc; --l) {
            if (whole_fits(H[l].n, A.stage_cap))
                staged_up<CORR, T>(A, H, l, whole_geom(H[l].n), 1, nu_dsmem);
            else
                up_legs<CORR>(H, nr, A.nu2, l, l, blk, bs);
            __syncthreads();
        }
    }
    if (!gsync(3)) return false;
    for (int l = loc - 1; l >= 0; --l) {
        staged_up<CORR, T>(A, H, l, tile_geom(H[l].n), A.halo, nu_dsmem);
        if (!gsync(80 + l)) return false;
    }
    return true;
}

// FP64 form (T = double): every cycle in float64 on h64.
// Refined form (T = float): the float64 residual of `top` drives float32
// V-cycles on h32 for the correction, added to the float64 solution
// (iterative refinement; the stopping test is on the float64 residual).
template <bool CORR, typename T>
__global__ void __launch_bounds__(kThreads, 1) nu_solve_kernel(const __grid_constant__ NuArgs P) {
    constexpr bool REF = sizeof(T) == 4;
    __shared__ NuArgs A;
    __shared__ unsigned long long epoch;
    if (threadIdx.x == 0) {
        A = P;
        epoch = 0;
    }
    __syncthreads();
    const GridBarrier gsync{A.sc, &epoch, kBarrierLimit};
    const Team grid = qsync::spread_team();
    const Team blk{(int)threadIdx.x, (int)blockDim.x};
    NuScalars *sc = A.sc;
    const Level<T> *H = hier<T>(A);
    const Level<double> &top = A.top;
    const int nr = A.nrhs, Lc = A.levels - 1, n = top.n;
    // first level handled by block 0 alone
    int loc = 0;
    while (loc < Lc && H[loc].n > A.local_n) ++loc;

    // setup: M hierarchy and inverse diagonals (each level by the team that
    // smooths it)
    if (REF && A.has_m) {
        for (int p = grid.t; p < n * n; p += grid.nt) H[0].m[p] = T(A.m_in[p]);
        if (!gsync(1)) return;
    }
    level_idiag<CORR>(H[0], A.omega, grid);
    for (int l = 1; l <= Lc; ++l) {
        if (l <= loc) {
            if (A.has_m) restrict_m(H[l - 1], H[l], grid);
            if (!gsync(1)) return;
            level_idiag<CORR>(H[l], A.omega, grid);
        } else if (blockIdx.x == 0) {
            if (A.has_m) restrict_m(H[l - 1], H[l], blk);
            __syncthreads();
            level_idiag<CORR>(H[l], A.omega, blk);
            __syncthreads();
        }
    }
    // J' and the initial float64 residual (the refined form hands it to h32
    // as the right-hand side of the first correction, from zero)
    {
        double fn[kMaxRhs] = {0, 0, 0, 0}, rn[kMaxRhs] = {0, 0, 0, 0};
        for (int p = grid.t; p < n * n; p += grid.nt) {
            const int j = p / n, i = p - j * n;
            double mrow[3], mcol[3], m0;
            load_m(A.m_in, n, i, j, mrow, mcol, m0);
            for (int c = 0; c < nr; ++c) {
                const double fv = corrected_source<CORR>(top, A.j + (size_t)c * n * n, i, j);
                top.f[(size_t)c * n * n + p] = fv;
                double v[3][3];
                load_v(top.u + (size_t)c * n * n, n, i, j, v);
                const double r = fv - apply_point<CORR>(top.ax[i], top.ay[j], v, mrow, mcol, m0);
                if (REF) {
                    H[0].f[(size_t)c * n * n + p] = T(r);
                    H[0].u[(size_t)c * n * n + p] = T(0);
                }
                fn[c] += fv * fv;
                rn[c] += r * r;
            }
        }
        qsync::block_sum_add<kThreads>(fn, nr, sc->fnorm);
        qsync::block_sum_add<kThreads>(rn, nr, sc->norm[0]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        coarse_inverse<CORR>(H[Lc], reinterpret_cast<T *>(A.coarse_inv));
    if (!gsync(2)) return;

    double fn2[kMaxRhs];
    for (int c = 0; c < nr; ++c) fn2[c] = vload(&sc->fnorm[c]);
    for (int cyc = 0;; ++cyc) {
        // convergence test on the float64 residual left by the previous
        // cycle (slot cyc % 3)
        bool conv = true;
        for (int c = 0; c < nr; ++c) {
            const double rn = vload(&sc->norm[cyc % 3][c]);
            if (fn2[c] > 0.0 && rn > A.tol * A.tol * fn2[c]) conv = false;
        }
        if (conv || cyc >= A.max_cycles) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                sc->cycles = cyc;
                sc->converged = conv ? 1 : 0;
                for (int c = 0; c < nr; ++c)
                    sc->relres[c] =
                        fn2[c] > 0.0 ? sqrt(vload(&sc->norm[cyc % 3][c]) / fn2[c]) : 0.0;
            }
            // a field whose source is zero has the solution zero
            for (int c = 0; c < nr; ++c)
                if (fn2[c] == 0.0)
                    for (int p = grid.t; p < n * n; p += grid.nt)
                        top.u[(size_t)c * n * n + p] = 0.0;
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0)
            for (int c = 0; c < kMaxRhs; ++c) sc->norm[(cyc + 1) % 3][c] = 0.0;
        if (!vcycle<CORR>(A, H, loc, grid, blk, gsync)) return;
        if (REF) {
            // u += e (float64), then the new float64 residual
            for (int p = grid.t; p < n * n; p += grid.nt)
                for (int c = 0; c < nr; ++c)
                    top.u[(size_t)c * n * n + p] += (double)H[0].u[(size_t)c * n * n + p];
            if (!gsync(5)) return;
        }
        double rn[kMaxRhs] = {0, 0, 0, 0};
        for (int p = grid.t; p < n * n; p += grid.nt) {
            const int j = p / n, i = p - j * n;
            double mrow[3], mcol[3], m0;
            load_m(A.m_in, n, i, j, mrow, mcol, m0);
            for (int c = 0; c < nr; ++c) {
                double v[3][3];
                load_v(top.u + (size_t)c * n * n, n, i, j, v);
                const double r = top.f[(size_t)c * n * n + p] -
                                 apply_point<CORR>(top.ax[i], top.ay[j], v, mrow, mcol, m0);
                if (REF) {
                    H[0].f[(size_t)c * n * n + p] = T(r);
                    H[0].u[(size_t)c * n * n + p] = T(0);
                }
                rn[c] += r * r;
            }
        }
        qsync::block_sum_add<kThreads>(rn, nr, sc->norm[(cyc + 1) % 3]);
        if (!gsync(4)) return;
    }
}

// Operator and corrected source of the finest level for one field (tests,
// diagnostics), in float64.
template <bool CORR>
__global__ void nu_apply_kernel(const __grid_constant__ NuArgs A, const double *u, double *out,
                                int source) {
    const Level<double> &L = A.top;
    const int n = L.n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n * n; p += gridDim.x * blockDim.x) {
        const int j = p / n, i = p - j * n;
        if (source) {
            out[p] = corrected_source<CORR>(L, u, i, j);
        } else {
            double mrow[3], mcol[3], m0, v[3][3];
            load_m(A.m_in, n, i, j, mrow, mcol, m0);
            load_v(u, n, i, j, v);
            out[p] = apply_point<CORR>(L.ax[i], L.ay[j], v, mrow, mcol, m0);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct qs_nu_solver {
    int n = 0, levels = 0, correction = 0, precision = QS_FP64;
    int want_staged = 1;
    cudaStream_t stream = nullptr;
    int grid_blocks = 0;
    NuArgs args{};
    void *dev = nullptr;       // one allocation: coefficients, level arrays, scalars
    void *pinned = nullptr;    // host copy of NuScalars
};

namespace {

void axis_coefficients(const std::vector<double> &x, int correction,
                       std::vector<AxisCoef<double>> &out) {
    const int n = (int)x.size() - 2;
    out.resize(n);
    for (int i = 0; i < n; ++i) {
        const double hm = x[i + 1] - x[i], hp = x[i + 2] - x[i + 1], ha = hm + hp;
        AxisCoef<double> c{};
        c.d2[0] = 2.0 / (hm * ha);
        c.d2[1] = -2.0 / (hm * hp);
        c.d2[2] = 2.0 / (hp * ha);
        const double fw = hm / (ha * hp), bw = hp / (ha * hm);
        c.d1[0] = -bw;
        c.d1[1] = bw - fw;
        c.d1[2] = fw;
        c.c = correction ? (hp - hm) / 3.0 : 0.0;
        out[i] = c;
    }
}

// Prolongation weights of the fine nodes (pairs; used at even 0-based nodes,
// which lie between the coarse nodes or a coarse node and a wall).
void prolong_weights(const std::vector<double> &x, std::vector<double> &out) {
    const int n = (int)x.size() - 2;
    out.assign(2 * n, 0.0);
    for (int i = 0; i < n; i += 2) {
        const int f = i + 1;  // index with the wall at 0
        const double span = x[f + 1] - x[f - 1];
        out[2 * i] = (x[f + 1] - x[f]) / span;       // weight of the left coarse node
        out[2 * i + 1] = (x[f] - x[f - 1]) / span;   // weight of the right coarse node
    }
}

// Restriction weights of each coarse node: the transpose of the prolongation
// scaled by fine dual lengths over the coarse dual length (rows sum to 1).
void restrict_weights(const std::vector<double> &x, const std::vector<double> &pw,
                      std::vector<double> &out) {
    const int n = (int)x.size() - 2, nc = (n - 1) / 2;
    out.assign(3 * nc, 0.0);
    auto dual = [&](int f) { return 0.5 * (x[f + 1] - x[f - 1]); };
    for (int I = 0; I < nc; ++I) {
        const int i = 2 * I + 1, f = i + 1;
        const double vc = 0.5 * (x[f + 2] - x[f - 2]);
        out[3 * I + 0] = pw[2 * (i - 1) + 1] * dual(f - 1) / vc;
        out[3 * I + 1] = dual(f) / vc;
        out[3 * I + 2] = pw[2 * (i + 1)] * dual(f + 1) / vc;
    }
}

bool valid_axis(const double *x, int n) {
    if (!x) return false;
    for (int i = 0; i < n + 1; ++i)
        if (!(x[i + 1] > x[i])) return false;  // also rejects NaN
    return true;
}

int levels_for(int n) {
    int l = 1;
    while (n > 3) {
        if ((n & 1) == 0) return 0;
        n = (n - 1) / 2;
        ++l;
    }
    return n == 3 ? l : 0;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return QS_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA;
}

struct HostLevel {
    int n;
    std::vector<AxisCoef<double>> ax, ay;
    std::vector<double> pwx, pwy, rwx, rwy;
};

// Carves one device allocation into arrays and fills a host image of it.
struct Arena {
    char *base = nullptr;
    size_t off = 0;
    std::vector<char> *image = nullptr;  // null while sizing
    static size_t align(size_t b) { return (b + 255) & ~(size_t)255; }
    template <typename T>
    T *take(size_t count) {
        T *p = reinterpret_cast<T *>(base + off);
        off += align(count * sizeof(T));
        return p;
    }
    template <typename T, typename S>
    const T *put(const std::vector<S> &src) {
        T *p = take<T>(src.size());
        if (image)
            for (size_t k = 0; k < src.size(); ++k)
                reinterpret_cast<T *>(image->data() + (reinterpret_cast<char *>(p) - base))[k] =
                    static_cast<T>(src[k]);
        return p;
    }
    template <typename T>
    const AxisCoef<T> *put_axis(const std::vector<AxisCoef<double>> &src) {
        AxisCoef<T> *p = take<AxisCoef<T>>(src.size());
        if (image)
            for (size_t k = 0; k < src.size(); ++k) {
                AxisCoef<T> c{};
                for (int q = 0; q < 3; ++q) {
                    c.d2[q] = static_cast<T>(src[k].d2[q]);
                    c.d1[q] = static_cast<T>(src[k].d1[q]);
                }
                c.c = static_cast<T>(src[k].c);
                std::memcpy(image->data() + (reinterpret_cast<char *>(p) - base) +
                                k * sizeof(AxisCoef<T>),
                            &c, sizeof(c));
            }
        return p;
    }
};

// Lays out a whole hierarchy in precision T (level 0 included).
template <typename T>
void lay_hierarchy(Arena &ar, const std::vector<HostLevel> &hl, Level<T> *H) {
    for (size_t l = 0; l < hl.size(); ++l) {
        const HostLevel &h = hl[l];
        const size_t nn = (size_t)h.n * h.n;
        Level<T> &L = H[l];
        L.n = h.n;
        L.ax = ar.put_axis<T>(h.ax);
        L.ay = ar.put_axis<T>(h.ay);
        L.pwx = ar.put<T>(h.pwx);
        L.pwy = ar.put<T>(h.pwy);
        L.rwx = ar.put<T>(h.rwx);
        L.rwy = ar.put<T>(h.rwy);
        L.u = ar.take<T>(kMaxRhs * nn);
        L.f = ar.take<T>(kMaxRhs * nn);
        L.r = ar.take<T>(kMaxRhs * nn);
        L.m = ar.take<T>(nn);
        L.idiag = ar.take<T>(nn);
    }
}

// The float64 finest level of both forms, then the cycling hierarchy.
void lay_out(Arena &ar, const std::vector<HostLevel> &hl, int precision, NuArgs &A) {
    A.sc = ar.take<NuScalars>(1);
    A.coarse_inv = ar.take<double>(81);
    const size_t nn = (size_t)hl[0].n * hl[0].n;
    A.top = Level<double>{};
    A.top.n = hl[0].n;
    if (precision == QS_FP64) {
        lay_hierarchy<double>(ar, hl, A.h64);
        A.top = A.h64[0];
    } else {
        A.top.ax = ar.put_axis<double>(hl[0].ax);
        A.top.ay = ar.put_axis<double>(hl[0].ay);
        A.top.f = ar.take<double>(kMaxRhs * nn);
        lay_hierarchy<float>(ar, hl, A.h32);
    }
}

}  // namespace

extern "C" int qs_nu_create(int n, const double *x_nodes, const double *y_nodes, int correction,
                            int precision, void *cuda_stream, qs_nu_solver **out) {
    if (!out) return QS_ERR_ARG;
    *out = nullptr;
    if (n < 3 || n > 4095 || (correction != 0 && correction != 1)) return QS_ERR_ARG;
    if (precision != QS_FP64 && precision != QS_FP32_REFINED) return QS_ERR_ARG;
    const int levels = levels_for(n);
    if (levels < 1 || levels > kMaxLevels) return QS_ERR_ARG;
    if (!valid_axis(x_nodes, n) || !valid_axis(y_nodes, n)) return QS_ERR_ARG;

    qs_nu_solver *s = new (std::nothrow) qs_nu_solver();
    if (!s) return QS_ERR_OOM;
    s->n = n;
    s->levels = levels;
    s->correction = correction;
    s->precision = precision;
    s->stream = static_cast<cudaStream_t>(cuda_stream);

    // host tables per level (coarse nodes: every other node, walls kept)
    std::vector<double> xs(x_nodes, x_nodes + n + 2), ys(y_nodes, y_nodes + n + 2);
    std::vector<HostLevel> hl(levels);
    for (int l = 0; l < levels; ++l) {
        HostLevel &h = hl[l];
        h.n = (int)xs.size() - 2;
        axis_coefficients(xs, correction, h.ax);
        axis_coefficients(ys, correction, h.ay);
        prolong_weights(xs, h.pwx);
        prolong_weights(ys, h.pwy);
        if (l + 1 < levels) {
            restrict_weights(xs, h.pwx, h.rwx);
            restrict_weights(ys, h.pwy, h.rwy);
            std::vector<double> cx, cy;
            for (size_t k = 0; k < xs.size(); k += 2) cx.push_back(xs[k]);
            for (size_t k = 0; k < ys.size(); k += 2) cy.push_back(ys[k]);
            xs.swap(cx);
            ys.swap(cy);
        }
    }
    // size the layout, allocate, lay it out again with a host image
    NuArgs &A = s->args;
    Arena sizing;
    lay_out(sizing, hl, precision, A);
    const size_t bytes = sizing.off;
    int st = cuda_status(cudaMalloc(&s->dev, bytes));
    if (st == QS_OK) st = cuda_status(cudaMallocHost(&s->pinned, sizeof(NuScalars)));
    if (st != QS_OK) {
        qs_nu_destroy(s);
        return st;
    }
    std::vector<char> image(bytes, 0);
    Arena ar;
    ar.base = static_cast<char *>(s->dev);
    ar.image = &image;
    A = NuArgs{};
    lay_out(ar, hl, precision, A);
    A.levels = levels;
    A.nu1 = kDefaultNu1;
    A.nu2 = kDefaultNu2;
    A.omega = kDefaultOmega;
    A.local_n = kDefaultLocalN;
    st = cuda_status(cudaMemcpyAsync(s->dev, image.data(), bytes, cudaMemcpyHostToDevice,
                                     s->stream));
    if (st == QS_OK) st = cuda_status(cudaStreamSynchronize(s->stream));
    if (st != QS_OK) {
        qs_nu_destroy(s);
        return st;
    }
    // one block per SM (co-resident: the cooperative launch checks it)
    int dev = 0, sms = 0, per_sm = 0;
    const void *fn = nullptr;
    if (precision == QS_FP64)
        fn = correction ? (const void *)nu_solve_kernel<true, double>
                        : (const void *)nu_solve_kernel<false, double>;
    else
        fn = correction ? (const void *)nu_solve_kernel<true, float>
                        : (const void *)nu_solve_kernel<false, float>;
    st = cuda_status(cudaGetDevice(&dev));
    if (st == QS_OK) st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (st == QS_OK)
        st = cuda_status(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kStageSmemMax));
    if (st == QS_OK)
        st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads,
                                                                       kStageSmemMax));
    if (st == QS_OK && per_sm < 1) st = QS_ERR_CUDA;
    if (st != QS_OK) {
        qs_nu_destroy(s);
        return st;
    }
    s->grid_blocks = sms;
    *out = s;
    return QS_OK;
}

extern "C" int qs_nu_solve(qs_nu_solver *s, const double *d_m, int nrhs, const double *d_j,
                           double *d_u, double tol, int max_cycles, int *cycles, double *relres) {
    if (!s || !d_j || !d_u || nrhs < 1 || nrhs > kMaxRhs || max_cycles < 1) return QS_ERR_ARG;
    if (!(tol > 0.0)) return QS_ERR_ARG;
    NuArgs A = s->args;
    A.nrhs = nrhs;
    A.has_m = d_m != nullptr;
    A.max_cycles = max_cycles;
    A.tol = tol;
    A.j = d_j;
    A.m_in = d_m;
    // the float64 finest level works in place on the caller's u and reads the
    // caller's M (never written); the cycling levels hold their own M
    A.top.u = d_u;
    A.top.m = const_cast<double *>(d_m);
    if (s->precision == QS_FP64) {
        A.h64[0].u = d_u;
        A.h64[0].m = A.top.m;
    }
    if (!d_m)
        for (int l = 0; l < A.levels; ++l) A.h64[l].m = nullptr, A.h32[l].m = nullptr;
    // staged smoothing when the largest tile's region fits in shared memory
    A.halo = 4 * (A.nu1 > A.nu2 ? A.nu1 : A.nu2) + 2;
    const size_t elem = s->precision == QS_FP64 ? sizeof(double) : sizeof(float);
    const size_t stage_bytes = (size_t)(2 * nrhs + 2) * (kTileX + 2 * A.halo) *
                               (kTileY + 2 * A.halo) * elem;
    A.staged = s->want_staged && stage_bytes <= kStageSmemMax;
    A.stage_cap = (kTileX + 2 * A.halo) * (kTileY + 2 * A.halo);
    const size_t dyn = A.staged ? stage_bytes : 0;
    int st = cuda_status(cudaMemsetAsync(A.sc, 0, sizeof(NuScalars), s->stream));
    if (st != QS_OK) return st;
    void *params[] = {&A};
    const void *fn = nullptr;
    if (s->precision == QS_FP64)
        fn = s->correction ? (const void *)nu_solve_kernel<true, double>
                           : (const void *)nu_solve_kernel<false, double>;
    else
        fn = s->correction ? (const void *)nu_solve_kernel<true, float>
                           : (const void *)nu_solve_kernel<false, float>;
    st = cuda_status(cudaLaunchCooperativeKernel(fn, dim3(s->grid_blocks), dim3(kThreads), params,
                                                 dyn, s->stream));
    if (st != QS_OK) return st;
    st = cuda_status(cudaMemcpyAsync(s->pinned, A.sc, sizeof(NuScalars), cudaMemcpyDeviceToHost,
                                     s->stream));
    if (st == QS_OK) st = cuda_status(cudaStreamSynchronize(s->stream));
    if (st != QS_OK) return st;
    const NuScalars *h = static_cast<const NuScalars *>(s->pinned);
    if (h->err) return h->err;
    if (cycles) *cycles = h->cycles;
    if (relres)
        for (int c = 0; c < nrhs; ++c) relres[c] = h->relres[c];
    return h->converged ? QS_OK : QS_ERR_NOT_CONVERGED;
}

extern "C" int qs_nu_set_cycle(qs_nu_solver *s, int pre_sweeps, int post_sweeps, double omega,
                               int coarse_block_n, int staged) {
    if (!s || pre_sweeps < 0 || post_sweeps < 0 || pre_sweeps > 8 || post_sweeps > 8 ||
        pre_sweeps + post_sweeps < 1 || !(omega > 0.0 && omega < 2.0) || coarse_block_n < 0 ||
        (staged != 0 && staged != 1))
        return QS_ERR_ARG;
    s->want_staged = staged;
    s->args.nu1 = pre_sweeps;
    s->args.nu2 = post_sweeps;
    s->args.omega = omega;
    s->args.local_n = coarse_block_n ? coarse_block_n : kDefaultLocalN;
    return QS_OK;
}

extern "C" int qs_nu_apply(qs_nu_solver *s, const double *d_m, const double *d_u, double *d_out) {
    if (!s || !d_u || !d_out) return QS_ERR_ARG;
    NuArgs A = s->args;
    A.m_in = d_m;
    const int nn = s->n * s->n;
    const int blocks = (nn + 255) / 256;
    if (s->correction)
        nu_apply_kernel<true><<<blocks, 256, 0, s->stream>>>(A, d_u, d_out, 0);
    else
        nu_apply_kernel<false><<<blocks, 256, 0, s->stream>>>(A, d_u, d_out, 0);
    return cuda_status(cudaGetLastError());
}

extern "C" int qs_nu_source(qs_nu_solver *s, const double *d_j, double *d_out) {
    if (!s || !d_j || !d_out) return QS_ERR_ARG;
    const int nn = s->n * s->n;
    const int blocks = (nn + 255) / 256;
    if (s->correction)
        nu_apply_kernel<true><<<blocks, 256, 0, s->stream>>>(s->args, d_j, d_out, 1);
    else
        nu_apply_kernel<false><<<blocks, 256, 0, s->stream>>>(s->args, d_j, d_out, 1);
    return cuda_status(cudaGetLastError());
}

extern "C" void qs_nu_destroy(qs_nu_solver *s) {
    if (!s) return;
    if (s->dev) cudaFree(s->dev);
    if (s->pinned) cudaFreeHost(s->pinned);
    delete s;
}
