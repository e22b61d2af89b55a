// Kernels outside the slice loop: the quiet-start plasma lattice, density
// deposits, the driver-beam deposit and push (Sec. 7.1, Eqs. EoM_beam_1/2)
// and the stable counting sort of particles by cell.
#include <cuda_runtime.h>

#include "qs_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 65535LL * 32) b = 65535LL * 32;
    return (int)b;
}

// Cold lattice: sqrt(ppc)^2 particles per cell at offsets (k + 1/2)/s of a
// cell, p = 0 (Sec. 3.1, H = 1 and P = 0 before the driver), weight
// n(r0) h^2 / ppc, id = cell * ppc + ky * s + kx.
__global__ void k_init_plasma(int n, int ppc, int s, double x_min, double y_min, double h,
                              const double *table, int n_coef, double r_max, double *x,
                              double *y, double *px, double *py, double *w, int32_t *id) {
    const int64_t np = (int64_t)n * n * ppc;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ppc;
        const int k = (int)(p - c * ppc);
        const int iy = (int)(c / n), ix = (int)(c - (int64_t)iy * n);
        const int ky = k / s, kx = k - ky * s;
        const double xx = x_min + (ix + (kx + 0.5) / s) * h;
        const double yy = y_min + (iy + (ky + 0.5) / s) * h;
        double dens = 1.0;
        if (table) {
            const double r = sqrt(xx * xx + yy * yy);
            if (n_coef == 1) {
                dens = table[0];
            } else {
                double sr = fmin(r / r_max * (n_coef - 1), (double)(n_coef - 1));
                int i = (int)floor(sr);
                if (i > n_coef - 2) i = n_coef - 2;
                const double f = sr - i;
                dens = table[i] * (1.0 - f) + table[i + 1] * f;
            }
        }
        x[p] = xx;
        y[p] = yy;
        px[p] = 0.0;
        py[p] = 0.0;
        w[p] = dens * (h * h / ppc);
        id[p] = (int32_t)p;
    }
}

__global__ void k_deposit(const double *x, const double *y, const double *q, int64_t np, int n,
                          double x_min, double y_min, double h, double scale, double *grid) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        Cic c = cic_stencil(x[p], y[p], x_min, y_min, h, n);
        cic_deposit(grid, c, q[p] * scale);
    }
}

// Driver j_z on the base slices: CIC in x, y, linear in xi; -charge w v_z.
__global__ void k_beam_deposit(const double *x, const double *y, const double *xi,
                               const double *px, const double *py, const double *pz,
                               const double *w, int64_t nb, double charge, int n, double x_min,
                               double x_max, double y_min, double y_max, double h, int n_xi,
                               double xi_min, double dxi0, double *jzb) {
    const double norm = 1.0 / (h * h * dxi0);
    const size_t nn = (size_t)n * n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nb;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double xx = x[p], yy = y[p];
        if (!(xx >= x_min && xx <= x_max && yy >= y_min && yy <= y_max)) continue;
        const double s = (xi[p] - xi_min) / dxi0;
        const double fl = floor(s);
        const double f = s - fl;
        if (!(fl > -2.0 && fl < (double)n_xi)) continue;
        const int j0 = (int)fl;
        const double ux = px[p], uy = py[p], uz = pz[p];
        const double gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double q = -charge * w[p] * uz / gam * norm;
        Cic c = cic_stencil(xx, yy, x_min, y_min, h, n);
        if (j0 >= 0 && j0 < n_xi) cic_deposit(jzb + (size_t)j0 * nn, c, q * (1.0 - f));
        if (j0 + 1 >= 0 && j0 + 1 < n_xi) cic_deposit(jzb + (size_t)(j0 + 1) * nn, c, q * f);
    }
}

// Wake at (x, y, xi): CIC in x, y, linear in xi between base slices; zero
// outside the box or the window.  Returns E_z, B_z, B_x, B_y, dpsi/dx,
// dpsi/dy (central differences of psi with odd ghosts).
__device__ void wake_at(const double *hist, int n, int n_xi, double x_min, double x_max,
                        double y_min, double y_max, double h, double xi_min, double dxi0,
                        double x, double y, double xi, double out[6]) {
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    if (!(x >= x_min && x <= x_max && y >= y_min && y <= y_max)) return;
    const double s = (xi - xi_min) / dxi0;
    const double fl = floor(s);
    if (!(fl > -2.0 && fl < (double)n_xi)) return;
    const int j0 = (int)fl;
    const double f = s - fl;
    const size_t nn = (size_t)n * n, fs = (size_t)n_xi * nn;
    const double inv2h = 0.5 / h;
    Cic c = cic_stencil(x, y, x_min, y_min, h, n);
    const int idx[4] = {c.i00, c.i01, c.i10, c.i11};
    const double wc[4] = {c.w00, c.w01, c.w10, c.w11};
    for (int side = 0; side < 2; ++side) {
        const int j = j0 + side;
        if (j < 0 || j >= n_xi) continue;
        const double wj = side ? f : 1.0 - f;
        const double *ps = hist + (size_t)j * nn;
        for (int k = 0; k < 4; ++k) {
            const int i = idx[k];
            const int iy = i / n, ix = i - iy * n;
            const double ww = wj * wc[k];
            out[0] += ww * ps[fs + i];
            out[1] += ww * ps[2 * fs + i];
            out[2] += ww * ps[3 * fs + i];
            out[3] += ww * ps[4 * fs + i];
            const double pc = ps[i];
            const double pe = ix < n - 1 ? ps[i + 1] : -pc;
            const double pw = ix > 0 ? ps[i - 1] : -pc;
            const double pn = iy < n - 1 ? ps[i + n] : -pc;
            const double pq = iy > 0 ? ps[i - n] : -pc;
            out[4] += ww * (pe - pw) * inv2h;
            out[5] += ww * (pn - pq) * inv2h;
        }
    }
}

// Push_Driver: relativistic Boris step in E = (-d_x psi + B_y, -d_y psi - B_x,
// E_z), B = (B_x, B_y, B_z); xi advances by dt (1 - v_z).
__global__ void k_beam_push(double *x, double *y, double *xi, double *px, double *py,
                            double *pz, int64_t nb, double qm, int n, double x_min,
                            double x_max, double y_min, double y_max, double h, int n_xi,
                            double xi_min, double dxi0, const double *hist, double dt) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nb;
         p += (int64_t)gridDim.x * blockDim.x) {
        double wk[6];
        wake_at(hist, n, n_xi, x_min, x_max, y_min, y_max, h, xi_min, dxi0, x[p], y[p], xi[p],
                wk);
        const double ez = wk[0], bz = wk[1], bx = wk[2], by = wk[3];
        const double ex = -wk[4] + by, ey = -wk[5] - bx;
        const double hq = 0.5 * dt * qm;
        double ux = px[p] + hq * ex, uy = py[p] + hq * ey, uz = pz[p] + hq * ez;
        double gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double tx = hq * bx / gam, ty = hq * by / gam, tz = hq * bz / gam;
        const double ss = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
        const double upx = ux + (uy * tz - uz * ty);
        const double upy = uy + (uz * tx - ux * tz);
        const double upz = uz + (ux * ty - uy * tx);
        ux = ux + ss * (upy * tz - upz * ty);
        uy = uy + ss * (upz * tx - upx * tz);
        uz = uz + ss * (upx * ty - upy * tx);
        ux += hq * ex;
        uy += hq * ey;
        uz += hq * ez;
        gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        x[p] += dt * ux / gam;
        y[p] += dt * uy / gam;
        xi[p] += dt * (1.0 - uz / gam);
        px[p] = ux;
        py[p] = uy;
        pz[p] = uz;
    }
}

// ---- driver push in the laser's high-frequency fields (DLA) ----
//
// The envelope A (vector potential A e^{-i k0 xi}, polarised along x) and its
// derivatives gathered at a particle like the wake: CIC in x, y on the base
// slices, linear in xi, zero outside the box and the window.  d_x A, d_y A
// are central differences with odd ghosts (A is zero on the walls), d_xi A
// the central difference between base slices with A = 0 ahead of and behind
// the window.  out = (A, d_xi A, d_x A, d_y A), complex.
__device__ void envelope_at(const double2 *env, int n, int n_xi, double x_min, double x_max,
                            double y_min, double y_max, double h, double xi_min, double dxi0,
                            double x, double y, double xi, double2 out[4]) {
    for (int k = 0; k < 4; ++k) out[k] = make_double2(0.0, 0.0);
    if (!(x >= x_min && x <= x_max && y >= y_min && y <= y_max)) return;
    const double s = (xi - xi_min) / dxi0;
    const double fl = floor(s);
    if (!(fl > -2.0 && fl < (double)n_xi)) return;
    const int j0 = (int)fl;
    const double f = s - fl;
    const size_t nn = (size_t)n * n;
    const double inv2h = 0.5 / h, inv2xi = 0.5 / dxi0;
    Cic c = cic_stencil(x, y, x_min, y_min, h, n);
    const int idx[4] = {c.i00, c.i01, c.i10, c.i11};
    const double wc[4] = {c.w00, c.w01, c.w10, c.w11};
    for (int side = 0; side < 2; ++side) {
        const int j = j0 + side;
        if (j < 0 || j >= n_xi) continue;
        const double wj = side ? f : 1.0 - f;
        const double2 *a = env + (size_t)j * nn;
        const double2 *ap = j + 1 < n_xi ? a + nn : nullptr;
        const double2 *am = j > 0 ? a - nn : nullptr;
        for (int k = 0; k < 4; ++k) {
            const int i = idx[k];
            const int iy = i / n, ix = i - iy * n;
            const double ww = wj * wc[k];
            const double2 ac = a[i];
            const double2 ae = ix < n - 1 ? a[i + 1] : make_double2(-ac.x, -ac.y);
            const double2 aw = ix > 0 ? a[i - 1] : make_double2(-ac.x, -ac.y);
            const double2 an = iy < n - 1 ? a[i + n] : make_double2(-ac.x, -ac.y);
            const double2 aq = iy > 0 ? a[i - n] : make_double2(-ac.x, -ac.y);
            const double2 xp = ap ? ap[i] : make_double2(0.0, 0.0);
            const double2 xm = am ? am[i] : make_double2(0.0, 0.0);
            out[0].x += ww * ac.x;
            out[0].y += ww * ac.y;
            out[1].x += ww * (xp.x - xm.x) * inv2xi;
            out[1].y += ww * (xp.y - xm.y) * inv2xi;
            out[2].x += ww * (ae.x - aw.x) * inv2h;
            out[2].y += ww * (ae.y - aw.y) * inv2h;
            out[3].x += ww * (an.x - aq.x) * inv2h;
            out[3].y += ww * (an.y - aq.y) * inv2h;
        }
    }
}

// Push_Driver in the wake plus the laser's fields of Eq. E_B_Fields (the
// real parts of the printed complex fields; x polarisation):
//   E_x = Re[-((d_t A + d_xi A) - i k0 A) e^{-i k0 xi}],  B_y = Re[(-d_xi A + i k0 A) e^{-i k0 xi}],
//   E_z = Re[-d_x A e^{-i k0 xi}],                        B_z = Re[-d_y A e^{-i k0 xi}],
// in n_sub relativistic Boris sub-steps of dt / n_sub (Eqs. EoM_beam_1/2).  At
// sub-step s the envelope is taken linearly in time between env_n and
// env_np1 at frac = s / n_sub, d_t A = (A^{n+1} - A^n) / dt; the carrier
// phase is evaluated at the particle's own xi; the wake is frozen.
__global__ void k_beam_push_dla(double *x, double *y, double *xi, double *px, double *py,
                                double *pz, int64_t nb, double qm, int n, double x_min,
                                double x_max, double y_min, double y_max, double h, int n_xi,
                                double xi_min, double dxi0, const double *hist,
                                const double2 *env_n, const double2 *env_np1, double k0,
                                double dt, int n_sub) {
    const double hs = dt / n_sub, hq = 0.5 * hs * qm, inv_dt = 1.0 / dt;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nb;
         p += (int64_t)gridDim.x * blockDim.x) {
        double X = x[p], Y = y[p], XI = xi[p];
        double ux = px[p], uy = py[p], uz = pz[p];
        for (int s = 0; s < n_sub; ++s) {
            double wk[6];
            wake_at(hist, n, n_xi, x_min, x_max, y_min, y_max, h, xi_min, dxi0, X, Y, XI, wk);
            double2 gn[4], gp[4];
            envelope_at(env_n, n, n_xi, x_min, x_max, y_min, y_max, h, xi_min, dxi0, X, Y, XI,
                        gn);
            envelope_at(env_np1, n, n_xi, x_min, x_max, y_min, y_max, h, xi_min, dxi0, X, Y,
                        XI, gp);
            const double fr = (double)s / (double)n_sub, fo = 1.0 - fr;
            const double ar = fo * gn[0].x + fr * gp[0].x, ai = fo * gn[0].y + fr * gp[0].y;
            const double tr = (gp[0].x - gn[0].x) * inv_dt, ti = (gp[0].y - gn[0].y) * inv_dt;
            const double xr = fo * gn[1].x + fr * gp[1].x, xim = fo * gn[1].y + fr * gp[1].y;
            const double dxr = fo * gn[2].x + fr * gp[2].x, dxim = fo * gn[2].y + fr * gp[2].y;
            const double dyr = fo * gn[3].x + fr * gp[3].x, dyim = fo * gn[3].y + fr * gp[3].y;
            double sn, cs;
            sincos(k0 * XI, &sn, &cs);  // e^{-i k0 xi} = cs - i sn
            // Re[(u + i v)(cs - i sn)] = u cs + v sn
            const double exl = -((tr + xr) + k0 * ai) * cs - ((ti + xim) - k0 * ar) * sn;
            const double byl = (-xr - k0 * ai) * cs + (-xim + k0 * ar) * sn;
            const double ezl = -dxr * cs - dxim * sn;
            const double bzl = -dyr * cs - dyim * sn;
            const double ez = wk[0] + ezl, bz = wk[1] + bzl, bx = wk[2], by = wk[3] + byl;
            const double ex = -wk[4] + wk[3] + exl, ey = -wk[5] - wk[2];
            double vx = ux + hq * ex, vy = uy + hq * ey, vz = uz + hq * ez;
            double gam = sqrt(1.0 + vx * vx + vy * vy + vz * vz);
            const double tx = hq * bx / gam, ty = hq * by / gam, tz = hq * bz / gam;
            const double ss = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
            const double upx = vx + (vy * tz - vz * ty);
            const double upy = vy + (vz * tx - vx * tz);
            const double upz = vz + (vx * ty - vy * tx);
            vx = vx + ss * (upy * tz - upz * ty);
            vy = vy + ss * (upz * tx - upx * tz);
            vz = vz + ss * (upx * ty - upy * tx);
            ux = vx + hq * ex;
            uy = vy + hq * ey;
            uz = vz + hq * ez;
            gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
            X += hs * ux / gam;
            Y += hs * uy / gam;
            XI += hs * (1.0 - uz / gam);
        }
        x[p] = X;
        y[p] = Y;
        xi[p] = XI;
        px[p] = ux;
        py[p] = uy;
        pz[p] = uz;
    }
}

__global__ void k_convert(const double *src, float *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_widen(const float *src, double *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// ---- stable counting sort by cell ----
__global__ void k_sort_count(const double *x, const double *y, int64_t np, int n, double x_min,
                             double y_min, double h, int32_t *cell, int32_t *count) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell_of(x[p], y[p], x_min, y_min, h, n);
        cell[p] = c;
        atomicAdd(count + c, 1);
    }
}

// exclusive scan of count[0..m) into offset[0..m] by one block
__global__ void k_sort_scan(const int32_t *count, int m, int32_t *offset, int32_t *cursor) {
    __shared__ int32_t part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (m + nt - 1) / nt;
    const int b = t * chunk, e = min(b + chunk, m);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int32_t run = 0;
        for (int i = 0; i < nt; ++i) {
            int32_t v = part[i];
            part[i] = run;
            run += v;
        }
        offset[m] = run;
    }
    __syncthreads();
    int32_t run = part[t];
    for (int i = b; i < e; ++i) {
        offset[i] = run;
        cursor[i] = 0;
        run += count[i];
    }
}

__global__ void k_sort_scatter(const int32_t *cell, int64_t np, const int32_t *offset,
                               int32_t *cursor, int32_t *perm) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[p];
        const int slot = atomicAdd(cursor + c, 1);
        perm[offset[c] + slot] = (int32_t)p;
    }
}

// within each cell, order the entries by particle id (insertion sort)
__global__ void k_sort_segments(int m, const int32_t *offset, const int32_t *id, int32_t *perm) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const int b = offset[c], e = offset[c + 1];
        for (int i = b + 1; i < e; ++i) {
            const int32_t v = perm[i];
            const int32_t key = id[v];
            int k = i - 1;
            while (k >= b && id[perm[k]] > key) {
                perm[k + 1] = perm[k];
                --k;
            }
            perm[k + 1] = v;
        }
    }
}

}  // namespace

cudaError_t qs_launch_init_plasma(cudaStream_t st, int n, int ppc, double x_min, double y_min,
                                  double h, const double *table, int n_coef, double r_max,
                                  double *x, double *y, double *px, double *py, double *w,
                                  int32_t *id) {
    int s = 1;
    while (s * s < ppc) ++s;
    const int64_t np = (int64_t)n * n * ppc;
    k_init_plasma<<<blocks_for(np), kThreads, 0, st>>>(n, ppc, s, x_min, y_min, h, table, n_coef,
                                                       r_max, x, y, px, py, w, id);
    return cudaGetLastError();
}

cudaError_t qs_launch_deposit(cudaStream_t st, const double *x, const double *y,
                              const double *q, int64_t np, int n, double x_min, double y_min,
                              double h, double scale, double *grid) {
    k_deposit<<<blocks_for(np), kThreads, 0, st>>>(x, y, q, np, n, x_min, y_min, h, scale, grid);
    return cudaGetLastError();
}

cudaError_t qs_launch_beam_deposit(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                   double x_max, double y_min, double y_max, double h,
                                   int n_xi, double xi_min, double dxi0, double *jzb) {
    if (b.n <= 0) return cudaSuccess;
    k_beam_deposit<<<blocks_for(b.n), kThreads, 0, st>>>(b.x, b.y, b.xi, b.px, b.py, b.pz, b.w,
                                                         b.n, b.charge, n, x_min, x_max, y_min,
                                                         y_max, h, n_xi, xi_min, dxi0, jzb);
    return cudaGetLastError();
}

cudaError_t qs_launch_beam_push(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                double x_max, double y_min, double y_max, double h, int n_xi,
                                double xi_min, double dxi0, const double *hist, double dt) {
    if (b.n <= 0) return cudaSuccess;
    k_beam_push<<<blocks_for(b.n), kThreads, 0, st>>>(b.x, b.y, b.xi, b.px, b.py, b.pz, b.n,
                                                      b.q_over_m, n, x_min, x_max, y_min, y_max,
                                                      h, n_xi, xi_min, dxi0, hist, dt);
    return cudaGetLastError();
}

cudaError_t qs_launch_beam_push_dla(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                    double x_max, double y_min, double y_max, double h,
                                    int n_xi, double xi_min, double dxi0, const double *hist,
                                    const double *env_n, const double *env_np1, double k0,
                                    double dt, int n_sub) {
    if (b.n <= 0) return cudaSuccess;
    k_beam_push_dla<<<blocks_for(b.n), kThreads, 0, st>>>(
        b.x, b.y, b.xi, b.px, b.py, b.pz, b.n, b.q_over_m, n, x_min, x_max, y_min, y_max, h,
        n_xi, xi_min, dxi0, hist, (const double2 *)env_n, (const double2 *)env_np1, k0, dt,
        n_sub);
    return cudaGetLastError();
}

cudaError_t qs_launch_convert(cudaStream_t st, const double *src, float *dst, int64_t n) {
    if (n <= 0) return cudaSuccess;
    k_convert<<<blocks_for(n), kThreads, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

__global__ void k_abs2(const double *a, double *out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double re = a[2 * k], im = a[2 * k + 1];
        out[k] = re * re + im * im;
    }
}

cudaError_t qs_launch_abs2(cudaStream_t st, const double *a, double *out, int64_t n) {
    if (n <= 0) return cudaSuccess;
    k_abs2<<<blocks_for(n), kThreads, 0, st>>>(a, out, n);
    return cudaGetLastError();
}

cudaError_t qs_launch_widen(cudaStream_t st, const float *src, double *dst, int64_t n) {
    if (n <= 0) return cudaSuccess;
    k_widen<<<blocks_for(n), kThreads, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t qs_launch_cell_sort(cudaStream_t st, const double *x, const double *y,
                                const int32_t *id, int64_t np, int n, double x_min,
                                double y_min, double h, int32_t *cell, int32_t *count,
                                int32_t *offset, int32_t *cursor, int32_t *perm) {
    const int m = n * n;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * m, st);
    if (e != cudaSuccess) return e;
    if (np > 0)
        k_sort_count<<<blocks_for(np), kThreads, 0, st>>>(x, y, np, n, x_min, y_min, h, cell,
                                                          count);
    k_sort_scan<<<1, 1024, 0, st>>>(count, m, offset, cursor);
    if (np > 0) k_sort_scatter<<<blocks_for(np), kThreads, 0, st>>>(cell, np, offset, cursor, perm);
    k_sort_segments<<<blocks_for(m), kThreads, 0, st>>>(m, offset, id, perm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cell sort without any device allocation.
//
// Some callers cannot let a library allocate device memory: applications that
// hand all of the GPU's memory to their own pool or arena (a cudaMalloc
// outside it breaks their budget, or fails once the pool holds the memory),
// hosts that may only pass a plugin raw buffers and no allocator, and loops
// that must not pay for cudaMalloc / cudaFree, which can synchronise the
// device.  qs_cell_sort_noalloc serves them: the caller passes every input
// and output buffer, and the one scratch array the sort needs (a per-cell
// insertion cursor) is the file-scope device array below, which every GPU
// that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
// Largest grid the allocation-free sort accepts: QS_NOALLOC_MAX_CELLS cells
// (512 x 512), i.e. 1 MiB of int32 cursors.
static __device__ __align__(256) int32_t g_noalloc_cursor[QS_NOALLOC_MAX_CELLS];

namespace {

// Device address of g_noalloc_cursor in the current device's current
// context.  The host-side name of the array is only a stand-in, never a
// device address, and the address belongs to one context: it is looked up
// on every call (a host-side query, cheap next to the launches), so a
// cudaDeviceReset or another context made current between calls cannot
// leave a stale address behind.
cudaError_t cursor_address(int32_t **out) {
    void *addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_cursor);
    if (e != cudaSuccess) return e;
    *out = static_cast<int32_t *>(addr);
    return cudaSuccess;
}

}  // namespace

extern "C" int qs_cell_sort_noalloc(int n, double x_min, double y_min, double h,
                                    const double *x, const double *y, const int32_t *id,
                                    int64_t np, int32_t *cell, int32_t *count, int32_t *offset,
                                    int32_t *perm, void *cuda_stream) {
    if (n < 1 || (int64_t)n * n > QS_NOALLOC_MAX_CELLS) return QS_ERR_ARG;
    if (!(h > 0.0) || np < 0 || np > (int64_t)0x7fffffff || !count || !offset) return QS_ERR_ARG;
    if (np > 0 && (!x || !y || !id || !cell || !perm)) return QS_ERR_ARG;
    int32_t *cursor = nullptr;
    if (cursor_address(&cursor) != cudaSuccess) {
        cudaGetLastError();
        return QS_ERR_CUDA;
    }
    // the scan kernel clears cursor[0 .. n*n) before the scatter uses it
    const cudaError_t e =
        qs_launch_cell_sort(static_cast<cudaStream_t>(cuda_stream), x, y, id, np, n, x_min,
                            y_min, h, cell, count, offset, cursor, perm);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QS_ERR_CUDA;
    }
    return QS_OK;
}
