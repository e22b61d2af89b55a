// The slice advance on a nonuniform transverse grid (Sec. "Multigrid Solver
// with Nonuniform Grids", used there for the whole quasi-static loop).
//
// The uniform-grid slice loop of Algorithm 1 with every grid operation taken
// on the tensor-product node grid of qs_nonuniform.cu:
//   deposits and gathers   CIC on the nodes: linear weights in physical
//                          coordinates between the two nodes around a
//                          particle; weight on a wall node folds into the
//                          adjacent interior node; density = deposit / the
//                          node's dual area;
//   gradients              the three-point first difference printed after
//                          Eq. 2D_Laplac_3rd, with zero beyond the walls;
//   the five field solves  the 9-point operator with the third-order
//                          correction (Eqs. 2D_Laplac, 2D_Laplac_3rd) by the
//                          nonuniform multigrid solver, warm-started from the
//                          previous slice: M = 0 for psi, E_z, B_z and
//                          M = -kappa for B_perp (Eq. Main_Eq_A);
//   the push               the Boris-like step of the uniform loop (the fields
//                          of the slice frozen at the particle), specular
//                          walls, V_max for Step_Size_Refinement with
//                          V0 = (smallest spacing) / dxi0.
// The driver enters as a given j_z on the nodes of the base slices, linear in
// xi at sub-steps.  Particles and grids are float64; the solver runs in the
// form chosen at creation (float64, or float32 cycles with float64 residual).
// The xi loop is driven from the host: each solve is one persistent launch of
// the solver, each particle or grid phase one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "qs_internal.cuh"

namespace {

constexpr int kT = 256;

int blocks_of(int64_t n) { return (int)std::min<int64_t>((n + kT - 1) / kT, 152 * 16); }

struct Axes {
    const double *xn, *yn;    // n + 2 node coordinates per axis, walls included
    const double *lx, *ly;    // dual lengths of the interior nodes
    const double *ax, *bx;    // first difference: a_i (forward) and b_i (backward) weights
    const double *ay, *by;
    int n;
};

// interval [xn[k], xn[k+1]] holding x (clamped to the box), as the left
// interior node k - 1 (-1 at the wall) and the weight f of the right node
__device__ __forceinline__ void node_interval(const double *xn, int n, double x, int &left,
                                              double &f) {
    x = fmin(fmax(x, xn[0]), xn[n + 1]);
    int lo = 0, hi = n + 1;  // xn[lo] <= x, find the last k with xn[k] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (xn[mid] <= x) lo = mid;
        else hi = mid;
    }
    const int k = min(lo, n);
    f = (x - xn[k]) / (xn[k + 1] - xn[k]);
    left = k - 1;
}

struct NStencil {
    int i[4];
    double w[4];
};

__device__ __forceinline__ NStencil node_stencil(const Axes &A, double x, double y) {
    int lx, ly;
    double fx, fy;
    node_interval(A.xn, A.n, x, lx, fx);
    node_interval(A.yn, A.n, y, ly, fy);
    NStencil s;
    const int n = A.n;
    const int x0 = min(max(lx, 0), n - 1), x1 = min(max(lx + 1, 0), n - 1);
    const int y0 = min(max(ly, 0), n - 1), y1 = min(max(ly + 1, 0), n - 1);
    s.i[0] = y0 * n + x0;
    s.i[1] = y0 * n + x1;
    s.i[2] = y1 * n + x0;
    s.i[3] = y1 * n + x1;
    s.w[0] = (1.0 - fy) * (1.0 - fx);
    s.w[1] = (1.0 - fy) * fx;
    s.w[2] = fy * (1.0 - fx);
    s.w[3] = fy * fx;
    return s;
}

__device__ __forceinline__ double n_gather(const double *u, const NStencil &s) {
    return s.w[0] * u[s.i[0]] + s.w[1] * u[s.i[1]] + s.w[2] * u[s.i[2]] + s.w[3] * u[s.i[3]];
}

// deposit q at the stencil as a density: weight / dual area of the node
__device__ __forceinline__ void n_deposit(double *g, const Axes &A, const NStencil &s, double q) {
    for (int k = 0; k < 4; ++k) {
        const int i = s.i[k], iy = i / A.n, ix = i - iy * A.n;
        atomicAdd(g + i, q * s.w[k] / (A.ly[iy] * A.lx[ix]));
    }
}

// first differences with zero beyond the walls
__device__ __forceinline__ double d1x(const Axes &A, const double *u, int ix, int i) {
    const double e = ix < A.n - 1 ? u[i + 1] : 0.0, w = ix > 0 ? u[i - 1] : 0.0;
    return -A.bx[ix] * w + (A.bx[ix] - A.ax[ix]) * u[i] + A.ax[ix] * e;
}
__device__ __forceinline__ double d1y(const Axes &A, const double *u, int iy, int i) {
    const double s = iy < A.n - 1 ? u[i + A.n] : 0.0, q = iy > 0 ? u[i - A.n] : 0.0;
    return -A.by[iy] * q + (A.by[iy] - A.ay[iy]) * u[i] + A.ay[iy] * s;
}

__device__ __forceinline__ double guard(double a, double fl, unsigned &hits) {
    if (a < fl) {
        ++hits;
        return fl;
    }
    return a;
}

__device__ void add_hits(unsigned long long *h, unsigned hits) {
    for (int o = 16; o; o >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, o);
    if ((threadIdx.x & 31) == 0 && hits) atomicAdd(h, (unsigned long long)hits);
}

// quiet start: s x s particles in every interval rectangle between
// neighbouring nodes (walls included), weight = rectangle area / s^2; the
// order is row-major over the sub-lattice coordinates (y slowest)
__global__ void k_nu_lattice(Axes A, int s, double *x, double *y, double *px, double *py,
                             double *w, int32_t *id) {
    const int nx = s * (A.n + 1);
    const int64_t np = (int64_t)nx * nx;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int jy = (int)(p / nx), jx = (int)(p - (int64_t)jy * nx);
        const int kx = jx / s, ox = jx - kx * s, ky = jy / s, oy = jy - ky * s;
        const double dx = A.xn[kx + 1] - A.xn[kx], dy = A.yn[ky + 1] - A.yn[ky];
        x[p] = A.xn[kx] + dx * ((ox + 0.5) / s);
        y[p] = A.yn[ky] + dy * ((oy + 0.5) / s);
        px[p] = 0.0;
        py[p] = 0.0;
        w[p] = (dy / s) * (dx / s);
        id[p] = (int32_t)p;
    }
}

__global__ void k_nu_deposit(Axes A, const double *x, const double *y, const double *q,
                             int64_t np, double *g) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x)
        n_deposit(g, A, node_stencil(A, x[p], y[p]), q[p]);
}

__global__ void k_nu_sub(const double *a, const double *b, double *out, int nn) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// moments of Eqs. Jr and FluxPres: j_perp = n_*<V>, T = n_*<V V>, G = n_*<gamma>
__global__ void k_nu_moments(Axes A, const double *x, const double *y, const double *px,
                             const double *py, const double *w, int64_t np, const double *psi,
                             double psi_floor, double *jx, double *jy, double *txx,
                             double *txy, double *tyy, double *G, unsigned long long *hits_out) {
    unsigned hits = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const NStencil s = node_stencil(A, x[p], y[p]);
        const double a = guard(1.0 + n_gather(psi, s), psi_floor, hits);
        const double ux = px[p], uy = py[p];
        const double gam = (1.0 + ux * ux + uy * uy + a * a) / (2.0 * a);
        const double vx = ux / a, vy = uy / a, q = w[p];
        n_deposit(jx, A, s, q * vx);
        n_deposit(jy, A, s, q * vy);
        n_deposit(txx, A, s, q * vx * vx);
        n_deposit(txy, A, s, q * vx * vy);
        n_deposit(tyy, A, s, q * vy * vy);
        n_deposit(G, A, s, q * gam);
    }
    add_hits(hits_out, hits);
}

// sources of E_z, B_z (Eqs. EqM_N8_A, Mag_z_A); j_z, kappa = n_*/(1+psi),
// M = -kappa, grad psi
__global__ void k_nu_assemble1(Axes A, const double *jx, const double *jy, const double *G,
                               const double *nstar, const double *psi, const double *jzb0,
                               const double *jzb1, double frac, double psi_floor,
                               double *f_eb, double *jz, double *kap, double *negkap,
                               double *dpx, double *dpy, unsigned long long *hits_out) {
    const int n = A.n, nn = n * n;
    unsigned hits = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const int iy = i / n, ix = i - iy * n;
        f_eb[i] = -(d1x(A, jx, ix, i) + d1y(A, jy, iy, i));
        f_eb[nn + i] = d1x(A, jy, ix, i) - d1y(A, jx, iy, i);
        const double a = guard(1.0 + psi[i], psi_floor, hits);
        const double jb = frac == 0.0 ? jzb0[i]
                                      : (1.0 - frac) * jzb0[i] + frac * (jzb1 ? jzb1[i] : 0.0);
        jz[i] = G[i] / a - nstar[i] + jb;
        kap[i] = nstar[i] / a;
        negkap[i] = -kap[i];
        dpx[i] = d1x(A, psi, ix, i);
        dpy[i] = d1y(A, psi, iy, i);
    }
    add_hits(hits_out, hits);
}

// the explicit source S of Eq. FluxCurr1_A; B_perp sources (S_y, -S_x)
__global__ void k_nu_assemble2(Axes A, const double *jx, const double *jy, const double *txx,
                               const double *txy, const double *tyy, const double *G,
                               const double *jz, const double *psi, const double *ez,
                               const double *bz, const double *dpx, const double *dpy,
                               double psi_floor, double *f_b) {
    const int n = A.n, nn = n * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const int iy = i / n, ix = i - iy * n;
        double a = 1.0 + psi[i];
        if (a < psi_floor) a = psi_floor;
        const double gx = dpx[i], gy = dpy[i];
        const double sx = d1x(A, jz, ix, i) - d1x(A, txx, ix, i) - d1y(A, txy, iy, i) -
                          jy[i] * bz[i] / a + G[i] * gx / (a * a) - jx[i] * ez[i] / a -
                          (txx[i] * gx + txy[i] * gy) / a;
        const double sy = d1y(A, jz, iy, i) - d1x(A, txy, ix, i) - d1y(A, tyy, iy, i) +
                          jx[i] * bz[i] / a + G[i] * gy / (a * a) - jy[i] * ez[i] / a -
                          (txy[i] * gx + tyy[i] * gy) / a;
        f_b[i] = sy;
        f_b[nn + i] = -sx;
    }
}

// the Boris-like push of the uniform loop with node gathers; V_max (as the
// bits of a non-negative double)
__global__ void k_nu_push(Axes A, double *x, double *y, double *px, double *py, int64_t np,
                          const double *psi, const double *dpx, const double *dpy,
                          const double *bx_, const double *by_, const double *bz_, double dxi,
                          double psi_floor, unsigned long long *vmax_bits,
                          unsigned long long *hits_out) {
    const double x_lo = A.xn[0], x_hi = A.xn[A.n + 1], y_lo = A.yn[0], y_hi = A.yn[A.n + 1];
    const double half = 0.5 * dxi;
    unsigned hits = 0;
    double vmax = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double x0 = x[p], y0 = y[p];
        const NStencil s = node_stencil(A, x0, y0);
        const double a = guard(1.0 + n_gather(psi, s), psi_floor, hits);
        const double gx = n_gather(dpx, s), gy = n_gather(dpy, s);
        const double bx = n_gather(bx_, s), by = n_gather(by_, s), bz = n_gather(bz_, s);
        double ux = px[p], uy = py[p];
        const double gam = (1.0 + ux * ux + uy * uy + a * a) / (2.0 * a);
        const double pxm = ux + half * (gam * gx / a - by);
        const double pym = uy + half * (gam * gy / a + bx);
        const double tau = half * bz / a;
        const double pxp = pxm - tau * pym, pyp = pym + tau * pxm;
        const double sr = 2.0 * tau / (1.0 + tau * tau);
        const double pxr = pxm - sr * pyp, pyr = pym + sr * pxp;
        const double gam2 = (1.0 + pxr * pxr + pyr * pyr + a * a) / (2.0 * a);
        ux = pxr + half * (gam2 * gx / a - by);
        uy = pyr + half * (gam2 * gy / a + bx);
        double nx = x0 + dxi * ux / a, ny = y0 + dxi * uy / a;
        if (nx > x_hi) { nx = 2.0 * x_hi - nx; ux = -ux; }
        if (nx < x_lo) { nx = 2.0 * x_lo - nx; ux = -ux; }
        if (ny > y_hi) { ny = 2.0 * y_hi - ny; uy = -uy; }
        if (ny < y_lo) { ny = 2.0 * y_lo - ny; uy = -uy; }
        x[p] = nx;
        y[p] = ny;
        px[p] = ux;
        py[p] = uy;
        vmax = fmax(vmax, sqrt(ux * ux + uy * uy) / a);
    }
    for (int o = 16; o; o >>= 1) vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(vmax));
    add_hits(hits_out, hits);
}

}  // namespace

struct qs_nu_pic {
    int n = 0, n_xi = 0, refine_k = 8, precision = QS_FP64;
    double dxi0 = 0.0, psi_floor = 1e-3, h_min = 0.0;
    cudaStream_t st = nullptr;
    qs_nu_solver *solver = nullptr;
    std::vector<void *> allocs, plasma_allocs;
    Axes ax{};
    int64_t np = 0;
    double *t_x = nullptr, *t_y = nullptr, *t_w = nullptr;
    double *x = nullptr, *y = nullptr, *px = nullptr, *py = nullptr, *w = nullptr;
    int32_t *id = nullptr;
    double *n_ion = nullptr, *nstar = nullptr, *f_psi = nullptr, *psi = nullptr;
    double *jx = nullptr, *jy = nullptr, *txx = nullptr, *txy = nullptr, *tyy = nullptr,
           *G = nullptr, *jz = nullptr, *kap = nullptr, *negkap = nullptr, *dpx = nullptr,
           *dpy = nullptr;
    double *f_eb = nullptr, *eb = nullptr, *f_b = nullptr, *bp = nullptr;  // [2][nn] each
    unsigned long long *scal = nullptr;  // [0] vmax bits, [1] guard hits
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int cuda_ok(cudaError_t e) {
    if (e == cudaSuccess) return QS_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA;
}

template <typename T>
int nalloc(qs_nu_pic *s, T **p, size_t count, bool plasma = false) {
    void *q = nullptr;
    const int r = cuda_ok(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    if (r != QS_OK) return r;
    (plasma ? s->plasma_allocs : s->allocs).push_back(q);
    *p = static_cast<T *>(q);
    return QS_OK;
}

#define NCK(expr)                       \
    do {                                \
        const int r_ = (expr);          \
        if (r_ != QS_OK) return r_;     \
    } while (0)

}  // namespace

extern "C" int qs_nu_pic_create(int n, const double *x_nodes, const double *y_nodes, int n_xi,
                                double xi_len, int refine_k, double psi_floor, int precision,
                                void *cuda_stream, qs_nu_pic **out) {
    if (!out) return QS_ERR_ARG;
    *out = nullptr;
    if (!x_nodes || !y_nodes || n_xi < 1 || !(xi_len > 0.0) || refine_k < 1 ||
        !(psi_floor > 0.0))
        return QS_ERR_ARG;
    for (int i = 0; i < n + 1; ++i)
        if (!(x_nodes[i + 1] > x_nodes[i]) || !(y_nodes[i + 1] > y_nodes[i])) return QS_ERR_ARG;
    qs_nu_pic *s = new (std::nothrow) qs_nu_pic();
    if (!s) return QS_ERR_OOM;
    s->n = n;
    s->n_xi = n_xi;
    s->dxi0 = xi_len / n_xi;
    s->refine_k = refine_k;
    s->psi_floor = psi_floor;
    s->precision = precision;
    s->st = static_cast<cudaStream_t>(cuda_stream);
    int r = qs_nu_create(n, x_nodes, y_nodes, 1, precision, cuda_stream, &s->solver);
    if (r != QS_OK) {
        delete s;
        return r;
    }
    // axis tables on the host: dual lengths, first-difference weights
    std::vector<double> hv[2][5];
    const double *nodes[2] = {x_nodes, y_nodes};
    double hmin = 1e300;
    for (int a = 0; a < 2; ++a) {
        const double *xn = nodes[a];
        hv[a][0].assign(xn, xn + n + 2);
        hv[a][1].resize(n);
        hv[a][2].resize(n);
        hv[a][3].resize(n);
        for (int i = 0; i < n; ++i) {
            const double hm = xn[i + 1] - xn[i], hp = xn[i + 2] - xn[i + 1], ha = hm + hp;
            double v = 0.5 * (hm + hp);
            if (i == 0) v += 0.5 * hm;
            if (i == n - 1) v += 0.5 * hp;
            hv[a][1][i] = v;
            hv[a][2][i] = hm / (ha * hp);  // forward-difference weight
            hv[a][3][i] = hp / (ha * hm);  // backward-difference weight
            hmin = std::min(hmin, std::min(hm, hp));
        }
    }
    s->h_min = hmin;
    double *d[2][4];
    for (int a = 0; a < 2 && r == QS_OK; ++a) {
        r = nalloc(s, &d[a][0], (size_t)n + 2);
        for (int k = 1; k < 4 && r == QS_OK; ++k) r = nalloc(s, &d[a][k], (size_t)n);
        for (int k = 0; k < 4 && r == QS_OK; ++k)
            r = cuda_ok(cudaMemcpy(d[a][k], hv[a][k].data(), hv[a][k].size() * sizeof(double),
                                   cudaMemcpyHostToDevice));
    }
    const size_t nn = (size_t)n * n;
    double **grids[] = {&s->n_ion, &s->nstar, &s->f_psi, &s->psi, &s->jx,  &s->jy,
                        &s->txx,   &s->txy,   &s->tyy,   &s->G,   &s->jz,  &s->kap,
                        &s->negkap, &s->dpx,  &s->dpy};
    for (double **g : grids)
        if (r == QS_OK) r = nalloc(s, g, nn);
    if (r == QS_OK) r = nalloc(s, &s->f_eb, 2 * nn);
    if (r == QS_OK) r = nalloc(s, &s->eb, 2 * nn);
    if (r == QS_OK) r = nalloc(s, &s->f_b, 2 * nn);
    if (r == QS_OK) r = nalloc(s, &s->bp, 2 * nn);
    if (r == QS_OK) r = nalloc(s, &s->scal, 2);
    if (r == QS_OK) r = cuda_ok(cudaEventCreate(&s->ev0));
    if (r == QS_OK) r = cuda_ok(cudaEventCreate(&s->ev1));
    if (r != QS_OK) {
        qs_nu_pic_destroy(s);
        return r;
    }
    s->ax = Axes{d[0][0], d[1][0], d[0][1], d[1][1], d[0][2], d[0][3], d[1][2], d[1][3], n};
    *out = s;
    return QS_OK;
}

extern "C" int qs_nu_pic_init_plasma(qs_nu_pic *s, int ppc) {
    if (!s) return QS_ERR_ARG;
    int q = 1;
    while (q * q < ppc) ++q;
    if (ppc < 1 || q * q != ppc) return QS_ERR_ARG;
    const int64_t np = (int64_t)(q * (s->n + 1)) * (q * (s->n + 1));
    if (np > 0x7fffffffLL) return QS_ERR_ARG;
    if (np != s->np) {
        NCK(cuda_ok(cudaStreamSynchronize(s->st)));
        for (void *p : s->plasma_allocs) cudaFree(p);
        s->plasma_allocs.clear();
        s->np = 0;
        double **arrs[] = {&s->t_x, &s->t_y, &s->t_w, &s->x, &s->y, &s->px, &s->py, &s->w};
        for (double **a : arrs) NCK(nalloc(s, a, (size_t)np, true));
        NCK(nalloc(s, &s->id, (size_t)np, true));
        s->np = np;
    }
    k_nu_lattice<<<blocks_of(np), kT, 0, s->st>>>(s->ax, q, s->t_x, s->t_y, s->px, s->py,
                                                   s->t_w, s->id);
    NCK(cuda_ok(cudaGetLastError()));
    const size_t nn = (size_t)s->n * s->n;
    NCK(cuda_ok(cudaMemsetAsync(s->n_ion, 0, nn * sizeof(double), s->st)));
    k_nu_deposit<<<blocks_of(np), kT, 0, s->st>>>(s->ax, s->t_x, s->t_y, s->t_w, np, s->n_ion);
    NCK(cuda_ok(cudaGetLastError()));
    return cuda_ok(cudaStreamSynchronize(s->st));
}

extern "C" int qs_nu_pic_step3d(qs_nu_pic *s, const double *d_jzb, double *d_hist, double tol,
                                int max_cycles, qs_step_stats *stats) {
    if (!s || !d_jzb || !d_hist || !(tol > 0.0) || max_cycles < 1) return QS_ERR_ARG;
    if (s->np == 0) return QS_ERR_STATE;
    const int n = s->n, nxi = s->n_xi;
    const size_t nn = (size_t)n * n, bd = s->np * sizeof(double);
    cudaStream_t st = s->st;
    // fresh plasma at the head of the window; fields start at zero
    NCK(cuda_ok(cudaMemcpyAsync(s->x, s->t_x, bd, cudaMemcpyDeviceToDevice, st)));
    NCK(cuda_ok(cudaMemcpyAsync(s->y, s->t_y, bd, cudaMemcpyDeviceToDevice, st)));
    NCK(cuda_ok(cudaMemcpyAsync(s->w, s->t_w, bd, cudaMemcpyDeviceToDevice, st)));
    NCK(cuda_ok(cudaMemsetAsync(s->px, 0, bd, st)));
    NCK(cuda_ok(cudaMemsetAsync(s->py, 0, bd, st)));
    for (double *f : {s->psi, s->eb, s->eb + nn, s->bp, s->bp + nn})
        NCK(cuda_ok(cudaMemsetAsync(f, 0, nn * sizeof(double), st)));
    NCK(cuda_ok(cudaMemsetAsync(s->scal, 0, 2 * sizeof(unsigned long long), st)));
    NCK(cuda_ok(cudaEventRecord(s->ev0, st)));
    const Axes A = s->ax;
    const int gb = blocks_of((int64_t)nn), pb = blocks_of(s->np);
    const double v0 = s->h_min / s->dxi0;
    int64_t slices = 0, pushes = 0, vc[3] = {0, 0, 0};
    int max_m = 1, m = 1, status = QS_OK;
    double max_rel = 0.0;
    for (int j = 0; j < nxi; ++j) {
        const bool last = j == nxi - 1;
        for (int q = 0; q < m; ++q) {
            const double frac = (double)q / m;
            const double *jb0 = d_jzb + (size_t)j * nn;
            const double *jb1 = last ? nullptr : jb0 + nn;
            // n_* (Eq. continuity) and psi (Eq. EqM_N8_AA)
            NCK(cuda_ok(cudaMemsetAsync(s->nstar, 0, nn * sizeof(double), st)));
            k_nu_deposit<<<pb, kT, 0, st>>>(A, s->x, s->y, s->w, s->np, s->nstar);
            k_nu_sub<<<gb, kT, 0, st>>>(s->nstar, s->n_ion, s->f_psi, (int)nn);
            NCK(cuda_ok(cudaGetLastError()));
            int cyc = 0;
            double rel[2] = {0.0, 0.0};
            int r = qs_nu_solve(s->solver, nullptr, 1, s->f_psi, s->psi, tol, max_cycles, &cyc,
                                rel);
            if (r != QS_OK && r != QS_ERR_NOT_CONVERGED) return r;
            if (r != QS_OK) status = r;
            vc[0] += cyc;
            max_rel = std::max(max_rel, rel[0]);
            // moments (Eqs. Jr, FluxPres)
            for (double *g : {s->jx, s->jy, s->txx, s->txy, s->tyy, s->G})
                NCK(cuda_ok(cudaMemsetAsync(g, 0, nn * sizeof(double), st)));
            k_nu_moments<<<pb, kT, 0, st>>>(A, s->x, s->y, s->px, s->py, s->w, s->np, s->psi,
                                             s->psi_floor, s->jx, s->jy, s->txx, s->txy,
                                             s->tyy, s->G, s->scal + 1);
            k_nu_assemble1<<<gb, kT, 0, st>>>(A, s->jx, s->jy, s->G, s->nstar, s->psi, jb0, jb1,
                                               frac, s->psi_floor, s->f_eb, s->jz, s->kap,
                                               s->negkap, s->dpx, s->dpy, s->scal + 1);
            NCK(cuda_ok(cudaGetLastError()));
            // E_z, B_z (Eqs. EqM_N8_A, Mag_z_A)
            r = qs_nu_solve(s->solver, nullptr, 2, s->f_eb, s->eb, tol, max_cycles, &cyc, rel);
            if (r != QS_OK && r != QS_ERR_NOT_CONVERGED) return r;
            if (r != QS_OK) status = r;
            vc[1] += cyc;
            max_rel = std::max(max_rel, std::max(rel[0], rel[1]));
            // B_perp (Eq. Main_Eq_A with the source of Eq. FluxCurr1_A)
            k_nu_assemble2<<<gb, kT, 0, st>>>(A, s->jx, s->jy, s->txx, s->txy, s->tyy, s->G,
                                               s->jz, s->psi, s->eb, s->eb + nn, s->dpx, s->dpy,
                                               s->psi_floor, s->f_b);
            NCK(cuda_ok(cudaGetLastError()));
            r = qs_nu_solve(s->solver, s->negkap, 2, s->f_b, s->bp, tol, max_cycles, &cyc, rel);
            if (r != QS_OK && r != QS_ERR_NOT_CONVERGED) return r;
            if (r != QS_OK) status = r;
            vc[2] += cyc;
            max_rel = std::max(max_rel, std::max(rel[0], rel[1]));
            ++slices;
            if (q == 0) {  // the base slice: psi, E_z, B_z, B_x, B_y
                const double *src[5] = {s->psi, s->eb, s->eb + nn, s->bp, s->bp + nn};
                for (int f = 0; f < 5; ++f)
                    NCK(cuda_ok(cudaMemcpyAsync(d_hist + ((size_t)f * nxi + j) * nn, src[f],
                                                nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                                st)));
            }
            if (last) break;
            // V_max of this push alone (the interval's last one decides m)
            NCK(cuda_ok(cudaMemsetAsync(s->scal, 0, sizeof(unsigned long long), st)));
            k_nu_push<<<pb, kT, 0, st>>>(A, s->x, s->y, s->px, s->py, s->np, s->psi, s->dpx,
                                          s->dpy, s->bp, s->bp + nn, s->eb + nn, s->dxi0 / m,
                                          s->psi_floor, s->scal, s->scal + 1);
            NCK(cuda_ok(cudaGetLastError()));
            pushes += s->np;
        }
        if (last) break;
        // Step_Size_Refinement: V_max of the interval's last push
        unsigned long long vb = 0;
        NCK(cuda_ok(cudaMemcpyAsync(&vb, s->scal, sizeof(vb), cudaMemcpyDeviceToHost, st)));
        NCK(cuda_ok(cudaStreamSynchronize(st)));
        double vm;
        std::memcpy(&vm, &vb, sizeof(vm));
        m = vm <= v0 ? 1 : (int)std::min<double>(s->refine_k, std::max(1.0, std::ceil(vm / v0)));
        max_m = std::max(max_m, m);
    }
    NCK(cuda_ok(cudaEventRecord(s->ev1, st)));
    unsigned long long hits = 0;
    NCK(cuda_ok(cudaMemcpyAsync(&hits, s->scal + 1, sizeof(hits), cudaMemcpyDeviceToHost, st)));
    NCK(cuda_ok(cudaStreamSynchronize(st)));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->ev0, s->ev1);
        stats->slices = slices;
        stats->substeps = slices - nxi;
        stats->pushes = pushes;
        for (int k = 0; k < 3; ++k) stats->vcycles[k] = vc[k];
        stats->psi_guard_hits = (int64_t)hits;
        stats->max_relres = max_rel;
        stats->max_m = max_m;
        stats->status = status;
        stats->gpu_ms = ms;
    }
    return status;
}

extern "C" int qs_nu_pic_get_plasma(qs_nu_pic *s, double *x, double *y, double *px, double *py,
                                    double *w) {
    if (!s) return QS_ERR_ARG;
    if (s->np == 0) return QS_ERR_STATE;
    const size_t bd = s->np * sizeof(double);
    const double *src[5] = {s->x, s->y, s->px, s->py, s->w};
    double *dst[5] = {x, y, px, py, w};
    for (int k = 0; k < 5; ++k)
        if (dst[k]) NCK(cuda_ok(cudaMemcpyAsync(dst[k], src[k], bd, cudaMemcpyDeviceToHost, s->st)));
    return cuda_ok(cudaStreamSynchronize(s->st));
}

extern "C" int64_t qs_nu_pic_count(const qs_nu_pic *s) { return s ? s->np : 0; }

extern "C" void qs_nu_pic_destroy(qs_nu_pic *s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    for (void *p : s->allocs) cudaFree(p);
    for (void *p : s->plasma_allocs) cudaFree(p);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    qs_nu_destroy(s->solver);
    delete s;
}
