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
// Levels of side <= 32 run in block 0 on __syncthreads, larger ones on the
// bounded grid barrier of qs_grid_sync.cuh.
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
constexpr int kLocalN = 32;            // levels this small run in block 0
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
    __shared__ LzArgs A;
    __shared__ unsigned long long epoch;
    if (threadIdx.x == 0) {
        A = P;
        epoch = 0;
    }
    __syncthreads();
    LzScalars *sc = A.sc;
    const qsync::GridBarrier<LzScalars> gsync{sc, &epoch, kBarrierLimit};
    const Team grid{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x)};
    const Team blk{(int)threadIdx.x, (int)blockDim.x};
    const int n = A.n, nn = n * n, Lc = A.levels - 1;
    int loc = 0;  // first level run by block 0 alone
    while (loc < Lc && A.lv[loc].n > kLocalN) ++loc;
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
            // initial residual, then V-cycles until converged
            int cyc = 0;
            for (;;) {
                double rn = 0.0;
                if (blockIdx.x == 0 && threadIdx.x == 0) sc->norm[(kglob + 1) % 3] = 0.0;
                for (int p = grid.t; p < nn; p += grid.nt) {
                    const int jj = p / n, i = p - jj * n;
                    rn += cabs2(csub(L0.f[p], apply_at(L0, U, i, jj)));
                }
                qsync::block_sum_add<kThreads>(&rn, 1, &sc->norm[kglob % 3]);
                if (!gsync(4)) return;
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
                if (Lc == 0) {
                    if (blockIdx.x == 0) {
                        const BlockSync bs;
                        smooth(A.lv[0], kCoarseSweeps, blk, bs, 5);
                    }
                    if (!gsync(3)) return;
                    continue;
                }
                if (!down(A.lv, 0, loc, grid, gsync)) return;
                if (blockIdx.x == 0) {
                    const BlockSync bs;
                    down(A.lv, loc, Lc, blk, bs);
                    smooth(A.lv[Lc], kCoarseSweeps, blk, bs, 5);
                    up(A.lv, Lc - 1, loc, blk, bs);
                }
                if (!gsync(3)) return;
                if (loc > 0 && !up(A.lv, loc - 1, 0, grid, gsync)) return;
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
        st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, laser_kernel, kThreads, 0));
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
                                                 dim3(kThreads), params, 0, s->stream));
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
