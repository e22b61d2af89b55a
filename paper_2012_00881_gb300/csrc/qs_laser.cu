// Laser-envelope advance (Sec. "Description of different plasma wake
// drivers", Eq. laser_Enve): the complex envelope A of a laser with vector
// potential A exp(-i k0 xi) obeys
//     (2 i k0 d_t - 2 d_t d_xi + lap_perp) A = chi A,   chi = n_* / (1 + psi).
// Time-centred in t, the mixed derivative as the time difference of a
// backward (towards the head) difference in xi, so slices advance from the
// head j = 0 to the tail, each one a complex screened-Poisson equation
//     (lap - kappa) A^{n+1}_j = (c + chi_j - lap) A^n_j - q (A^{n+1}_{j-1} - A^n_{j-1}),
//     kappa = chi_j - c,   c = 4 (i k0 - 1/dxi) / dt,   q = 4 / (dt dxi)
// (dxi = inf: q = 0, c = 4 i k0 / dt).  chi is held at t_n; A = 0 ahead of
// the window and on the walls (odd ghosts, the slice advance's cell-centred
// 5-point Laplacian).  The paper solves it with the same multigrid as the
// wake, warm-started from the previous time step (Sec. 7.1).
//
// Solver: complex multigrid V(2,2) on the cell-centred grid, red-black
// Gauss-Seidel (the 5-point operator decouples the colours), 4-cell average
// restriction of the residual and of kappa, bilinear prolongation with odd
// ghosts, rediscretised coarse operators, 20 red-black sweeps on the
// coarsest level (side <= 4); each slice's solve stops when ||f - A u||_2 <=
// tol ||f||_2.  Initial guess: the slice's envelope at t_n.
//
// Execution: one persistent cooperative launch per call runs every time step
// and slice: a right-hand-side phase per slice (which also writes the
// previous slice's new envelope back), the kappa hierarchy, then the cycles.
// Levels of side <= 8 run in block 0 on __syncthreads; larger ones are
// staged tile by tile in shared memory (see "Staged grid levels" below), one
// bounded grid barrier (qs_grid_sync.cuh) per level and leg.  Grid-wide
// loops hand runs of 32 cells to the blocks in turn, so that float64 work
// spreads over every SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <new>

#include "qs.h"
#include "qs_grid_sync.cuh"

namespace {

using qsync::BlockSync;
using qsync::Team;

constexpr int kMaxLevels = 14;
constexpr int kThreads = 512;
constexpr int kLocalN = 8;             // levels this small run in block 0
constexpr int kNu = 2;                 // pre- and post-sweeps, V(2, 2)
constexpr int kTileX = 32, kTileY = 16;  // largest staged output tile
constexpr int kCoarseSweeps = 20;
constexpr long long kBarrierLimit = 4000000000LL;  // clock cycles, ~2 s

struct LzScalars {
    unsigned long long bar;
    int err;
    int err_where;
    int fail;                 // a slice hit max_cycles
    int pad;
    long long cycles;         // V-cycles over all slices and steps
    double max_relres;        // largest final relative residual of a slice
    double norm[3];           // rotating residual-norm slots
    double fnorm[3];          // |f|^2 of the slices (rotating by slice count)
};

struct LzLevel {
    int n;
    double ih2;               // 1 / h^2
    double2 *u, *f, *r;       // n * n each (level 0: u is a ping-pong buffer)
    double2 *kap, *idg;       // kappa and 1 / diag(A)
};

struct LzArgs {
    LzLevel lv[kMaxLevels];
    int levels;
    int n, n_xi, steps, max_cycles;
    double tol, q;
    double2 c;
    const double *chi;        // caller: [n_xi][n][n]
    double2 *a;               // caller: [n_xi][n][n], A^n in, A^{n+steps} out
    double2 *ubuf[2];         // level-0 solutions of consecutive slices
    double2 *old[2];          // A^n of consecutive slices
    LzScalars *sc;
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cinv(double2 a) {
    const double d = 1.0 / (a.x * a.x + a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// u at (i, j) with odd ghosts (zero on the walls half a cell outside).
__device__ __forceinline__ double2 ghost_at(const double2 *u, int n, int i, int j) {
    double s = 1.0;
    if (i < 0) i = 0, s = -s;
    else if (i >= n) i = n - 1, s = -s;
    if (j < 0) j = 0, s = -s;
    else if (j >= n) j = n - 1, s = -s;
    return cscale(s, u[j * n + i]);
}

__device__ __forceinline__ double2 lap_at(const double2 *u, int n, double ih2, int i, int j) {
    const double2 s = cadd(cadd(ghost_at(u, n, i - 1, j), ghost_at(u, n, i + 1, j)),
                           cadd(ghost_at(u, n, i, j - 1), ghost_at(u, n, i, j + 1)));
    return cscale(ih2, csub(s, cscale(4.0, u[j * n + i])));
}

// A u = lap u - kappa u at cell p = (i, j)
__device__ __forceinline__ double2 apply_at(const LzLevel &L, const double2 *u, int i, int j) {
    const int p = j * L.n + i;
    return csub(lap_at(u, L.n, L.ih2, i, j), cmul(L.kap[p], u[p]));
}

__device__ void set_idiag(const LzLevel &L, Team tm) {
    const int n = L.n;
    for (int p = tm.t; p < n * n; p += tm.nt) {
        const int j = p / n, i = p - j * n;
        const int w = (i == 0) + (i == n - 1) + (j == 0) + (j == n - 1);
        const double2 d = make_double2(-(4.0 + w) * L.ih2 - L.kap[p].x, -L.kap[p].y);
        L.idg[p] = cinv(d);
    }
}

// kappa of the next coarser level: average of the 4 children
__device__ void restrict_kappa(const LzLevel &F, const LzLevel &C, Team tm) {
    const int nc = C.n, nf = F.n;
    for (int p = tm.t; p < nc * nc; p += tm.nt) {
        const int J = p / nc, I = p - J * nc;
        const double2 *k = F.kap + (2 * J) * nf + 2 * I;
        C.kap[p] = cscale(0.25, cadd(cadd(k[0], k[1]), cadd(k[nf], k[nf + 1])));
    }
}

__device__ void rb_colour(const LzLevel &L, int colour, Team tm) {
    const int n = L.n, half = (n * n + 1) / 2;
    for (int k = tm.t; k < half; k += tm.nt) {
        // k-th cell of the colour: rows alternate the parity of their first cell
        const int p2 = 2 * k;
        int j = p2 / n, i = p2 - j * n;
        if (((i + j) & 1) != colour) {
            ++i;
            if (i >= n) {
                i -= n;
                ++j;
            }
        }
        if (j >= n) continue;
        const int p = j * n + i;
        const double2 res = csub(L.f[p], apply_at(L, L.u, i, j));
        L.u[p] = cadd(L.u[p], cmul(res, L.idg[p]));
    }
}

template <typename Sync>
__device__ bool smooth(const LzLevel &L, int sweeps, Team tm, const Sync &sync, int where) {
    for (int s = 0; s < sweeps; ++s)
        for (int col = 0; col < 2; ++col) {
            rb_colour(L, col, tm);
            if (!sync(where)) return false;
        }
    return true;
}

__device__ void residual(const LzLevel &L, Team tm) {
    const int n = L.n;
    for (int p = tm.t; p < n * n; p += tm.nt) {
        const int j = p / n, i = p - j * n;
        L.r[p] = csub(L.f[p], apply_at(L, L.u, i, j));
    }
}

__device__ void restrict_residual(const LzLevel &F, const LzLevel &C, Team tm) {
    const int nc = C.n, nf = F.n;
    for (int p = tm.t; p < nc * nc; p += tm.nt) {
        const int J = p / nc, I = p - J * nc;
        const double2 *r = F.r + (2 * J) * nf + 2 * I;
        C.f[p] = cscale(0.25, cadd(cadd(r[0], r[1]), cadd(r[nf], r[nf + 1])));
        C.u[p] = make_double2(0.0, 0.0);
    }
}

// fine u += bilinear interpolation of the coarse u (weights 9, 3, 3, 1 / 16)
__device__ void prolong_correct(const LzLevel &F, const LzLevel &C, Team tm) {
    const int nf = F.n, nc = C.n;
    for (int p = tm.t; p < nf * nf; p += tm.nt) {
        const int j = p / nf, i = p - j * nf;
        const int I = i >> 1, J = j >> 1;
        const int di = (i & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1;
        const double2 e = cadd(cadd(cscale(9.0 / 16.0, ghost_at(C.u, nc, I, J)),
                                    cscale(3.0 / 16.0, ghost_at(C.u, nc, I + di, J))),
                               cadd(cscale(3.0 / 16.0, ghost_at(C.u, nc, I, J + dj)),
                                    cscale(1.0 / 16.0, ghost_at(C.u, nc, I + di, J + dj))));
        F.u[p] = cadd(F.u[p], e);
    }
}

// ---------------------------------------------------------------------------
// Staged grid levels.  A grid-wide level costs a grid barrier per colour
// sweep, residual, restriction and prolongation (eleven per V-cycle).  Here
// every block takes an output tile plus a halo, stages u, f, kappa and the
// inverse diagonal in shared memory and runs all the half sweeps of a leg
// there, recomputing the halo: after half sweep s only the cells at least
// s + 1 from a cut side of the region are exact, and those are the only ones
// updated.  A down leg (pre-sweeps, residual, restriction) and an up leg
// (prolongation, post-sweeps) each cost one grid barrier; the level-0 up leg
// also sums |f - A u|^2 of its tile for the stopping test.
// ---------------------------------------------------------------------------

struct Reg {
    int ox, oy, RX, RY, R;  // staged region: origin and extent
    int ax, bx, ay, by;     // its intersection with the domain
    bool cl, cr, cb, ct;    // which sides are cut (not the domain wall)
};

__device__ __forceinline__ Reg make_reg(int tx0, int ty0, int TX, int TY, int H, int n) {
    Reg g;
    g.ox = tx0 - H;
    g.oy = ty0 - H;
    g.RX = TX + 2 * H;
    g.RY = TY + 2 * H;
    g.R = g.RX * g.RY;
    g.ax = max(g.ox, 0);
    g.bx = min(g.ox + g.RX - 1, n - 1);
    g.ay = max(g.oy, 0);
    g.by = min(g.oy + g.RY - 1, n - 1);
    g.cl = g.ax > 0;
    g.cr = g.bx < n - 1;
    g.cb = g.ay > 0;
    g.ct = g.by < n - 1;
    return g;
}

// output tile of a staged level: halved (down to 8) while the level has
// fewer tiles than half the blocks, so that its work still spreads
__device__ __forceinline__ void lz_tile(int n, int nblk, int &TX, int &TY) {
    TX = kTileX;
    TY = kTileY;
    for (;;) {
        const int tiles = ((n + TX - 1) / TX) * ((n + TY - 1) / TY);
        if (2 * tiles >= nblk) break;
        if (TX >= TY && TX > 8) TX >>= 1;
        else if (TY > 8) TY >>= 1;
        else break;
    }
}

// staged arrays of a region of R cells: u, f, kappa, inverse diagonal
struct LzSmem {
    double2 *u, *f, *k, *d;
};

__device__ __forceinline__ LzSmem lz_layout(double2 *sm, int R) {
    return LzSmem{sm, sm + R, sm + 2 * R, sm + 3 * R};
}

// shared memory of the largest staged region (tile + halo 2 kNu + 1)
__host__ __device__ constexpr size_t lz_smem_bytes() {
    return (size_t)4 * (kTileX + 2 * (2 * kNu + 1)) * (kTileY + 2 * (2 * kNu + 1)) *
           sizeof(double2);
}

// 16-byte global -> shared copy, zero-filled when !valid (source size 0)
__device__ __forceinline__ void cp16(double2 *dst, const double2 *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// (lap - kappa) u at staged cell li = (x, y) (odd ghosts: a wall adds to the
// diagonal)
__device__ __forceinline__ double2 staged_apply(const LzSmem &t, int RX, int n, double ih2, int li,
                                                int x, int y) {
    double2 nb = make_double2(0.0, 0.0);
    if (x > 0) nb = cadd(nb, t.u[li - 1]);
    if (x < n - 1) nb = cadd(nb, t.u[li + 1]);
    if (y > 0) nb = cadd(nb, t.u[li - RX]);
    if (y < n - 1) nb = cadd(nb, t.u[li + RX]);
    const int w = (x == 0) + (x == n - 1) + (y == 0) + (y == n - 1);
    const double2 lap = cscale(ih2, csub(nb, cscale(4.0 + w, t.u[li])));
    return csub(lap, cmul(t.k[li], t.u[li]));
}

// half sweeps 0 .. ns - 1 (colour s & 1) on the staged region
__device__ void staged_sweeps(const Reg &g, int n, double ih2, const LzSmem &t, int ns) {
    for (int s = 0; s < ns; ++s) {
        const int colour = s & 1;
        const int X0 = g.cl ? g.ax + s + 1 : g.ax, X1 = g.cr ? g.bx - s - 1 : g.bx;
        const int Y0 = g.cb ? g.ay + s + 1 : g.ay, Y1 = g.ct ? g.by - s - 1 : g.by;
        const int rows = Y1 - Y0 + 1, hw = (X1 - X0 + 2) >> 1;
        const int cnt = (rows > 0 && hw > 0) ? rows * hw : 0;
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
            const int r = q / hw, y = Y0 + r;
            const int x = X0 + ((X0 + y + colour) & 1) + 2 * (q - r * hw);
            if (x > X1) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            const double2 res = csub(t.f[li], staged_apply(t, g.RX, n, ih2, li, x, y));
            t.u[li] = cadd(t.u[li], cmul(res, t.d[li]));
        }
        __syncthreads();
    }
}

// stage f, kappa, 1/diag of level F and u from usrc (nullptr: zero) on g
__device__ void stage(const LzLevel &F, const Reg &g, const LzSmem &t, const double2 *usrc) {
    const int n = F.n;
    for (int q = threadIdx.x; q < g.R; q += blockDim.x) {
        const int r = q / g.RX, x = g.ox + (q - r * g.RX), y = g.oy + r;
        const bool in = x >= 0 && x < n && y >= 0 && y < n;
        const int gi = in ? y * n + x : 0;
        cp16(t.f + q, F.f + gi, in);
        cp16(t.k + q, F.kap + gi, in);
        cp16(t.d + q, F.idg + gi, in);
        if (usrc) cp16(t.u + q, usrc + gi, in);
        else t.u[q] = make_double2(0.0, 0.0);
    }
    cp_wait();
    __syncthreads();
}

// Down leg of level F -> C for this block's tiles: pre-sweeps from the
// warm start F.u (level 0) or zero, residual, restriction into C.f
// (C.u = 0).  The smoothed tile goes to F.r, not F.u: other blocks still
// stage F.u around their tiles during this leg.
__device__ void staged_down(const LzLevel &F, const LzLevel &C, bool warm, double2 *sm, int bid,
                            int nblk) {
    const int n = F.n, m = C.n;
    int TX, TY;
    lz_tile(n, nblk, TX, TY);
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const Reg g = make_reg(tx0, ty0, TX, TY, 2 * kNu + 1, n);
        const LzSmem t = lz_layout(sm, g.R);
        stage(F, g, t, warm ? F.u : nullptr);
        staged_sweeps(g, n, F.ih2, t, 2 * kNu);
        const int CX = TX / 2, CY = TY / 2;
        for (int q = threadIdx.x; q < CX * CY; q += blockDim.x) {
            const int r = q / CX;
            const int I = tx0 / 2 + (q - r * CX), J = ty0 / 2 + r;
            if (I >= m || J >= m) continue;
            double2 s = make_double2(0.0, 0.0);
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int x = 2 * I + a, y = 2 * J + b;
                    const int li = (y - g.oy) * g.RX + (x - g.ox);
                    s = cadd(s, csub(t.f[li], staged_apply(t, g.RX, n, F.ih2, li, x, y)));
                }
            C.f[J * m + I] = cscale(0.25, s);
            C.u[J * m + I] = make_double2(0.0, 0.0);
        }
        for (int q = threadIdx.x; q < TX * TY; q += blockDim.x) {
            const int r = q / TX, x = tx0 + (q - r * TX), y = ty0 + r;
            if (x < n && y < n) F.r[y * n + x] = t.u[(y - g.oy) * g.RX + (x - g.ox)];
        }
        __syncthreads();  // the next tile reuses the staged arrays
    }
}

// Up leg of level F for this block's tiles: the pre-smoothed u (F.r, from
// the down leg) plus the bilinear prolongation of C.u, post-sweeps, the tile
// to F.u.  With `norm` (level 0) the halo is one cell wider and
// |f - A u|^2 of the tile is added to *norm_sum (this thread's share).
__device__ void staged_up(const LzLevel &F, const LzLevel &C, double2 *sm, int bid, int nblk,
                          bool norm, double *norm_sum) {
    const int n = F.n, nc = C.n;
    int TX, TY;
    lz_tile(n, nblk, TX, TY);
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const Reg g = make_reg(tx0, ty0, TX, TY, 2 * kNu + (norm ? 1 : 0), n);
        const LzSmem t = lz_layout(sm, g.R);
        stage(F, g, t, F.r);
        for (int q = threadIdx.x; q < g.R; q += blockDim.x) {
            const int r = q / g.RX, i = g.ox + (q - r * g.RX), j = g.oy + r;
            if (i < 0 || i >= n || j < 0 || j >= n) continue;
            const int I = i >> 1, J = j >> 1;
            const int di = (i & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1;
            const double2 e = cadd(cadd(cscale(9.0 / 16.0, ghost_at(C.u, nc, I, J)),
                                        cscale(3.0 / 16.0, ghost_at(C.u, nc, I + di, J))),
                                   cadd(cscale(3.0 / 16.0, ghost_at(C.u, nc, I, J + dj)),
                                        cscale(1.0 / 16.0, ghost_at(C.u, nc, I + di, J + dj))));
            t.u[q] = cadd(t.u[q], e);
        }
        __syncthreads();
        staged_sweeps(g, n, F.ih2, t, 2 * kNu);
        for (int q = threadIdx.x; q < TX * TY; q += blockDim.x) {
            const int r = q / TX, x = tx0 + (q - r * TX), y = ty0 + r;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            F.u[y * n + x] = t.u[li];
            if (norm) *norm_sum += cabs2(csub(t.f[li], staged_apply(t, g.RX, n, F.ih2, li, x, y)));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The coarse part (levels of side <= kLocalN) in every block's own shared
// memory, redundantly: no block waits for block 0 at a grid barrier, and the
// up leg of the first staged level prolongs from the block's own copy.  The
// coarsest level (up to kMaxExact unknowns) is solved with its exact
// inverse, formed once per slice by complex Gauss-Jordan elimination (no
// pivoting: -A has a positive definite Hermitian part, the 5-point -lap
// plus kappa with Re kappa = chi + q >= 0); larger coarsest levels take
// kCoarseSweeps red-black sweeps.
// ---------------------------------------------------------------------------
constexpr int kMaxExact = 16;
constexpr int kCoarseCells = 128;  // room for the levels of side <= kLocalN
constexpr size_t kCoarseBytes =
    (size_t)5 * kCoarseCells * sizeof(double2) + (size_t)kMaxExact * 2 * kMaxExact * sizeof(double2);

// the shared-memory hierarchy of levels loc .. Lc (pointers into sm)
__device__ void coarse_levels(const LzArgs &A, int loc, int Lc, double2 *sm, LzLevel *S) {
    double2 *p = sm;
    for (int l = loc; l <= Lc; ++l) {
        const int m = A.lv[l].n * A.lv[l].n;
        S[l].n = A.lv[l].n;
        S[l].ih2 = A.lv[l].ih2;
        S[l].u = p;
        S[l].f = p + m;
        S[l].r = p + 2 * m;
        S[l].kap = p + 3 * m;
        S[l].idg = p + 4 * m;
        p += 5 * m;
    }
}

// [A | I] -> [I | A^{-1}] for the coarsest operator A = lap - kappa
// (m = n^2 unknowns) in work (m x 2m, row-major): the inverse is the right
// half, work[i * 2m + m + j]
__device__ void coarse_inverse(const LzLevel &C, double2 *work) {
    const int n = C.n, m = n * n, W = 2 * m;
    __shared__ double2 s_piv;
    __shared__ double2 fac[kMaxExact];
    for (int e = threadIdx.x; e < m * W; e += blockDim.x) {
        const int i = e / W, j = e - i * W;
        double2 v = make_double2(0.0, 0.0);
        if (j >= m) {
            if (j - m == i) v.x = 1.0;
        } else {
            const int ix = i % n, iy = i / n, jx = j % n, jy = j / n;
            if (i == j) {
                const int w = (ix == 0) + (ix == n - 1) + (iy == 0) + (iy == n - 1);
                v = make_double2(-(4.0 + w) * C.ih2 - C.kap[i].x, -C.kap[i].y);
            } else if (abs(ix - jx) + abs(iy - jy) == 1) {
                v.x = C.ih2;
            }
        }
        work[e] = v;
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (threadIdx.x == 0) s_piv = cinv(work[k * W + k]);
        __syncthreads();
        const double2 piv = s_piv;
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            fac[i] = i == k ? make_double2(0.0, 0.0) : cmul(work[i * W + k], piv);
        __syncthreads();
        for (int e = threadIdx.x; e < m * (W - k); e += blockDim.x) {
            const int i = e / (W - k), j = k + (e - i * (W - k));
            if (i != k) work[i * W + j] = csub(work[i * W + j], cmul(fac[i], work[k * W + j]));
        }
        __syncthreads();
        for (int j = k + threadIdx.x; j < W; j += blockDim.x) work[k * W + j] = cmul(work[k * W + j], piv);
        __syncthreads();
    }
}

template <typename Sync>
__device__ bool down(const LzLevel *H, int from, int to, Team tm, const Sync &sync) {
    for (int l = from; l < to; ++l) {
        if (!smooth(H[l], 2, tm, sync, 10 + l)) return false;
        residual(H[l], tm);
        if (!sync(30 + l)) return false;
        restrict_residual(H[l], H[l + 1], tm);
        if (!sync(50 + l)) return false;
    }
    return true;
}

template <typename Sync>
__device__ bool up(const LzLevel *H, int from, int to, Team tm, const Sync &sync) {
    for (int l = from; l >= to; --l) {
        prolong_correct(H[l], H[l + 1], tm);
        if (!sync(70 + l)) return false;
        if (!smooth(H[l], 2, tm, sync, 90 + l)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 1) laser_kernel(const __grid_constant__ LzArgs P) {
    extern __shared__ double2 lz_dyn[];  // the staged regions
    __shared__ LzArgs A;
    __shared__ unsigned long long epoch;
    if (threadIdx.x == 0) {
        A = P;
        epoch = 0;
    }
    __syncthreads();
    LzScalars *sc = A.sc;
    const qsync::GridBarrier<LzScalars> gsync{sc, &epoch, kBarrierLimit};
    const Team grid = qsync::spread_team();
    const Team blk{(int)threadIdx.x, (int)blockDim.x};
    const int n = A.n, nn = n * n, Lc = A.levels - 1;
    int loc = 0;  // first level of the coarse part
    while (loc < Lc && A.lv[loc].n > kLocalN) ++loc;
    // the coarse part's levels in shared memory, after the staged regions
    // (used when loc > 0; the host checks that they fit)
    __shared__ LzLevel S[kMaxLevels];
    double2 *const csm = lz_dyn + lz_smem_bytes() / sizeof(double2);
    const bool exact = A.lv[Lc].n * A.lv[Lc].n <= kMaxExact;
    double2 *const cwork = csm + 5 * kCoarseCells;  // [I | A^{-1}] of the coarsest level
    int coarse_cells = 0;
    for (int l = loc; l <= Lc; ++l) coarse_cells += A.lv[l].n * A.lv[l].n;
    const bool local = loc > 0 && coarse_cells <= kCoarseCells;
    if (threadIdx.x == 0 && local) coarse_levels(A, loc, Lc, csm, S);
    __syncthreads();
    long long kglob = 0;  // residual-norm computations so far (slot kglob % 3)
    long long g = 0;      // slices so far

    for (int step = 0; step < A.steps; ++step) {
        for (int j = 0; j < A.n_xi; ++j, ++g) {
            double2 *U = A.ubuf[j & 1], *O = A.old[j & 1];
            const double2 *Up = A.ubuf[(j + 1) & 1], *Op = A.old[(j + 1) & 1];
            if (threadIdx.x == 0) A.lv[0].u = U;
            __syncthreads();
            const LzLevel &L0 = A.lv[0];
            // right-hand side, warm start, kappa and 1/diag of level 0; the
            // previous slice's new envelope goes back to the caller's array
            double fn = 0.0;
            const double2 *aj = A.a + (size_t)j * nn;
            const double *chij = A.chi + (size_t)j * nn;
            // slot (g + 1) % 3 was last read two slices ago, before a barrier
            if (blockIdx.x == 0 && threadIdx.x == 0) sc->fnorm[(g + 1) % 3] = 0.0;
            for (int p = grid.t; p < nn; p += grid.nt) {
                const int jj = p / n, i = p - jj * n;
                const double2 ao = aj[p];
                const double chi = chij[p];
                double2 f = csub(cmul(make_double2(A.c.x + chi, A.c.y), ao),
                                 lap_at(aj, n, L0.ih2, i, jj));
                if (j > 0) {
                    f = csub(f, cscale(A.q, csub(Up[p], Op[p])));
                    A.a[(size_t)(j - 1) * nn + p] = Up[p];
                }
                L0.f[p] = f;
                U[p] = ao;
                O[p] = ao;
                L0.kap[p] = make_double2(chi - A.c.x, -A.c.y);
                fn += cabs2(f);
            }
            qsync::block_sum_add<kThreads>(&fn, 1, &sc->fnorm[g % 3]);
            set_idiag(L0, grid);
            if (!gsync(1)) return;
            for (int l = 1; l <= Lc; ++l) {
                if (l <= loc) {
                    restrict_kappa(A.lv[l - 1], A.lv[l], grid);
                    if (!gsync(2)) return;
                    set_idiag(A.lv[l], grid);
                } else if (blockIdx.x == 0) {
                    restrict_kappa(A.lv[l - 1], A.lv[l], blk);
                    __syncthreads();
                    set_idiag(A.lv[l], blk);
                    __syncthreads();
                }
            }
            // initial residual, then V-cycles until converged; each cycle's
            // level-0 up leg sums the residual of its result
            int cyc = 0;
            {
                double rn = 0.0;
                if (blockIdx.x == 0 && threadIdx.x == 0) sc->norm[(kglob + 1) % 3] = 0.0;
                for (int p = grid.t; p < nn; p += grid.nt) {
                    const int jj = p / n, i = p - jj * n;
                    rn += cabs2(csub(L0.f[p], apply_at(L0, U, i, jj)));
                }
                qsync::block_sum_add<kThreads>(&rn, 1, &sc->norm[kglob % 3]);
                if (!gsync(4)) return;
            }
            for (;;) {
                const double r2 = qsync::vload(&sc->norm[kglob % 3]);
                const double f2 = qsync::vload(&sc->fnorm[g % 3]);
                ++kglob;
                const bool conv = r2 <= A.tol * A.tol * f2;
                if (conv || cyc >= A.max_cycles) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) {
                        sc->cycles += cyc;
                        const double rel = f2 > 0.0 ? sqrt(r2 / f2) : 0.0;
                        if (rel > sc->max_relres) sc->max_relres = rel;
                        if (!conv) sc->fail = 1;
                    }
                    break;
                }
                ++cyc;
                if (blockIdx.x == 0 && threadIdx.x == 0) sc->norm[(kglob + 1) % 3] = 0.0;
                double rn = 0.0;
                if (loc == 0) {  // a grid this small: block 0 alone, then the residual
                    if (blockIdx.x == 0) {
                        const BlockSync bs;
                        if (Lc == 0) {
                            smooth(A.lv[0], kCoarseSweeps, blk, bs, 5);
                        } else {
                            down(A.lv, 0, Lc, blk, bs);
                            smooth(A.lv[Lc], kCoarseSweeps, blk, bs, 5);
                            up(A.lv, Lc - 1, 0, blk, bs);
                        }
                    }
                    if (!gsync(3)) return;
                    for (int p = grid.t; p < nn; p += grid.nt) {
                        const int jj = p / n, i = p - jj * n;
                        rn += cabs2(csub(L0.f[p], apply_at(L0, U, i, jj)));
                    }
                } else {
                    for (int l = 0; l < loc; ++l) {
                        staged_down(A.lv[l], A.lv[l + 1], l == 0, lz_dyn, blockIdx.x, gridDim.x);
                        if (!gsync(10 + l)) return;
                    }
                    if (!local) {  // block 0 in global memory
                        if (blockIdx.x == 0) {
                            const BlockSync bs;
                            down(A.lv, loc, Lc, blk, bs);
                            smooth(A.lv[Lc], kCoarseSweeps, blk, bs, 5);
                            up(A.lv, Lc - 1, loc, blk, bs);
                        }
                        if (!gsync(3)) return;
                    } else {  // the coarse part, redundantly in every block's shared memory
                        const BlockSync bs;
                        const LzLevel &G = A.lv[loc];
                        const int m0 = G.n * G.n;
                        for (int p = threadIdx.x; p < m0; p += blockDim.x) {
                            cp16(S[loc].f + p, G.f + p, true);
                            S[loc].u[p] = make_double2(0.0, 0.0);
                        }
                        if (cyc == 1) {  // kappa and 1/diag change once per slice
                            for (int l = loc; l <= Lc; ++l)
                                for (int p = threadIdx.x; p < S[l].n * S[l].n; p += blockDim.x) {
                                    cp16(S[l].kap + p, A.lv[l].kap + p, true);
                                    cp16(S[l].idg + p, A.lv[l].idg + p, true);
                                }
                        }
                        cp_wait();
                        __syncthreads();
                        if (cyc == 1 && exact) coarse_inverse(S[Lc], cwork);
                        down(S, loc, Lc, blk, bs);
                        if (exact) {
                            const int mc = S[Lc].n * S[Lc].n;
                            const double2 *inv = cwork + mc;  // row i at inv + 2 mc i
                            for (int i = threadIdx.x; i < mc; i += blockDim.x) {
                                double2 s = make_double2(0.0, 0.0);
                                for (int k = 0; k < mc; ++k)
                                    s = cadd(s, cmul(inv[2 * mc * i + k], S[Lc].f[k]));
                                S[Lc].u[i] = s;
                            }
                            __syncthreads();
                        } else {
                            smooth(S[Lc], kCoarseSweeps, blk, bs, 5);
                        }
                        up(S, Lc - 1, loc, blk, bs);
                    }
                    for (int l = loc - 1; l >= 0; --l) {
                        staged_up(A.lv[l], (local && l + 1 == loc) ? S[loc] : A.lv[l + 1], lz_dyn,
                                  blockIdx.x, gridDim.x, l == 0, &rn);
                        if (l > 0 && !gsync(30 + l)) return;
                    }
                }
                qsync::block_sum_add<kThreads>(&rn, 1, &sc->norm[kglob % 3]);
                if (!gsync(4)) return;
            }
        }
        // the last slice's new envelope
        const double2 *Ul = A.ubuf[(A.n_xi - 1) & 1];
        for (int p = grid.t; p < nn; p += grid.nt) A.a[(size_t)(A.n_xi - 1) * nn + p] = Ul[p];
        if (!gsync(6)) return;
    }
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return QS_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA;
}

}  // namespace

struct qs_laser {
    int n = 0, n_xi = 0;
    double width = 0.0, dxi = 0.0;
    cudaStream_t stream = nullptr;
    int grid_blocks = 0;
    LzArgs args{};
    void *dev = nullptr;
    void *pinned = nullptr;
};

extern "C" int qs_laser_create(int n, double width, int n_xi, double k0, double dt, double dxi,
                               void *cuda_stream, qs_laser **out) {
    if (!out) return QS_ERR_ARG;
    *out = nullptr;
    if (n < 2 || n > 8192 || n_xi < 1 || !(width > 0.0) || !std::isfinite(width)) return QS_ERR_ARG;
    if (!(k0 > 0.0) || !std::isfinite(k0) || !(dt > 0.0) || !std::isfinite(dt)) return QS_ERR_ARG;
    if (!(dxi > 0.0)) return QS_ERR_ARG;  // +inf allowed: no xi coupling
    qs_laser *s = new (std::nothrow) qs_laser();
    if (!s) return QS_ERR_OOM;
    s->n = n;
    s->n_xi = n_xi;
    s->width = width;
    s->dxi = dxi;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    LzArgs &A = s->args;
    A.n = n;
    A.n_xi = n_xi;
    const double q = std::isinf(dxi) ? 0.0 : 4.0 / (dt * dxi);
    A.q = q;
    A.c = make_double2(-q, 4.0 * k0 / dt);
    // levels: halve while the side is even and above 4
    int sides[kMaxLevels];
    int levels = 0;
    for (int m = n;;) {
        sides[levels++] = m;
        if (m % 2 || m <= 4 || levels == kMaxLevels) break;
        m /= 2;
    }
    A.levels = levels;
    size_t elems = 4 * (size_t)n * n;  // ubuf[2], old[2]
    for (int l = 0; l < levels; ++l) elems += 5 * (size_t)sides[l] * sides[l];
    const size_t bytes = 256 + elems * sizeof(double2);
    int st = cuda_status(cudaMalloc(&s->dev, bytes));
    if (st == QS_OK) st = cuda_status(cudaMallocHost(&s->pinned, sizeof(LzScalars)));
    if (st != QS_OK) {
        qs_laser_destroy(s);
        return st;
    }
    char *base = static_cast<char *>(s->dev);
    A.sc = reinterpret_cast<LzScalars *>(base);
    double2 *p = reinterpret_cast<double2 *>(base + 256);
    for (int k = 0; k < 2; ++k) {
        A.ubuf[k] = p;
        p += (size_t)n * n;
        A.old[k] = p;
        p += (size_t)n * n;
    }
    for (int l = 0; l < levels; ++l) {
        LzLevel &L = A.lv[l];
        const size_t m = (size_t)sides[l] * sides[l];
        const double h = width / sides[l];
        L.n = sides[l];
        L.ih2 = 1.0 / (h * h);
        L.u = p;  // level 0's u is replaced by a ping-pong buffer per slice
        p += m;
        L.f = p;
        p += m;
        L.r = p;
        p += m;
        L.kap = p;
        p += m;
        L.idg = p;
        p += m;
    }
    int dev = 0, sms = 0, per_sm = 0;
    st = cuda_status(cudaGetDevice(&dev));
    if (st == QS_OK) st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (st == QS_OK)
        st = cuda_status(cudaFuncSetAttribute((const void *)laser_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(lz_smem_bytes() + kCoarseBytes)));
    if (st == QS_OK)
        st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, laser_kernel, kThreads,
                                                                       lz_smem_bytes() + kCoarseBytes));
    if (st == QS_OK && per_sm < 1) st = QS_ERR_CUDA;
    if (st != QS_OK) {
        qs_laser_destroy(s);
        return st;
    }
    s->grid_blocks = sms;
    *out = s;
    return QS_OK;
}

extern "C" int qs_laser_advance(qs_laser *s, const double *d_chi, double *d_a, int steps,
                                double tol, int max_cycles, int64_t *cycles, double *max_relres) {
    if (!s || !d_chi || !d_a || steps < 0 || max_cycles < 1 || !(tol > 0.0)) return QS_ERR_ARG;
    if (steps == 0) {
        if (cycles) *cycles = 0;
        if (max_relres) *max_relres = 0.0;
        return QS_OK;
    }
    LzArgs A = s->args;
    A.chi = d_chi;
    A.a = reinterpret_cast<double2 *>(d_a);
    A.steps = steps;
    A.tol = tol;
    A.max_cycles = max_cycles;
    int st = cuda_status(cudaMemsetAsync(A.sc, 0, sizeof(LzScalars), s->stream));
    if (st != QS_OK) return st;
    void *params[] = {&A};
    st = cuda_status(cudaLaunchCooperativeKernel((const void *)laser_kernel, dim3(s->grid_blocks),
                                                 dim3(kThreads), params,
                                                 lz_smem_bytes() + kCoarseBytes, s->stream));
    if (st != QS_OK) return st;
    st = cuda_status(cudaMemcpyAsync(s->pinned, A.sc, sizeof(LzScalars), cudaMemcpyDeviceToHost,
                                     s->stream));
    if (st == QS_OK) st = cuda_status(cudaStreamSynchronize(s->stream));
    if (st != QS_OK) return st;
    const LzScalars *h = static_cast<const LzScalars *>(s->pinned);
    if (h->err) return h->err;
    if (cycles) *cycles = h->cycles;
    if (max_relres) *max_relres = h->max_relres;
    return h->fail ? QS_ERR_NOT_CONVERGED : QS_OK;
}

extern "C" void qs_laser_destroy(qs_laser *s) {
    if (!s) return;
    if (s->dev) cudaFree(s->dev);
    if (s->pinned) cudaFreeHost(s->pinned);
    delete s;
}

// Grid of an envelope object (for the laser-driven 3D step, which checks that
// the slice loop and the envelope share cells, box and slices).
void qs_laser_shape(const qs_laser *s, int *n, double *width, int *n_xi, double *dxi) {
    *n = s->n;
    *width = s->width;
    *n_xi = s->n_xi;
    *dxi = s->dxi;
}
