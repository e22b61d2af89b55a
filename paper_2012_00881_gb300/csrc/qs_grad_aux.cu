// Kernels of the differentiable form outside the slice loop: the energy
// gain of a bunch in the stored wake and its reverse (the reverse
// relativistic Boris step of Eqs. EoM_beam_1/2 and the reverse of the
// trilinear wake gather), the reverse of the bunch j_z deposit, the chain
// rule of the radial density table, and the bi-Gaussian bunch of Sec. 5.1
// with its parameter chain rule.
#include <cuda_runtime.h>

#include <cmath>

#include "qs_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

__device__ double block_sum256(double v, double *red) {
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

struct Geo {
    int n, n_xi;
    double x_min, x_max, y_min, y_max, h, xi_min, dxi0;
};

// Trilinear stencil of a bunch particle: CIC in x, y (per-axis weights kept)
// and linear in xi between base slices j0 and j0 + 1.
struct Tri {
    bool ok;           // inside the box and near the window
    int j0;
    double f;          // xi weight of slice j0 + 1
    int ix0, ix1, iy0, iy1;
    double wx0, wx1, wy0, wy1;
};

__device__ __forceinline__ Tri tri(const Geo &g, double x, double y, double xi) {
    Tri t;
    t.ok = false;
    t.j0 = 0;
    t.f = 0.0;
    t.ix0 = t.ix1 = t.iy0 = t.iy1 = 0;
    t.wx0 = t.wx1 = t.wy0 = t.wy1 = 0.0;
    if (!(x >= g.x_min && x <= g.x_max && y >= g.y_min && y <= g.y_max)) return t;
    const double s = (xi - g.xi_min) / g.dxi0;
    const double fl = floor(s);
    if (!(fl > -2.0 && fl < (double)g.n_xi)) return t;
    t.ok = true;
    t.j0 = (int)fl;
    t.f = s - fl;
    cic_axis((x - g.x_min) / g.h, g.n, t.ix0, t.ix1, t.wx0, t.wx1);
    cic_axis((y - g.y_min) / g.h, g.n, t.iy0, t.iy1, t.wy0, t.wy1);
    return t;
}

// Energy gain of each particle after one Boris step of dt in the wake
// (summed into *gain_sum), and with d_hist != nullptr the cotangent of
// L = gain_sum * scale with respect to the stored history, added to d_hist.
__global__ void k_beam_gain(const double *x, const double *y, const double *xi,
                            const double *px, const double *py, const double *pz, int64_t nb,
                            double qm, Geo g, const double *hist, double dt, double scale,
                            double *gain_sum, double *d_hist) {
    __shared__ double red[32];
    const size_t nn = (size_t)g.n * g.n, fs = (size_t)g.n_xi * nn;
    const double inv2h = 0.5 / g.h;
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nb;
         p += (int64_t)gridDim.x * blockDim.x) {
        const Tri t = tri(g, x[p], y[p], xi[p]);
        // gather E_z, B_z, B_x, B_y, dpsi/dx, dpsi/dy (as qs_push_beam)
        double wk[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const int idx[4] = {t.iy0 * g.n + t.ix0, t.iy0 * g.n + t.ix1, t.iy1 * g.n + t.ix0,
                            t.iy1 * g.n + t.ix1};
        const double wc[4] = {t.wy0 * t.wx0, t.wy0 * t.wx1, t.wy1 * t.wx0, t.wy1 * t.wx1};
        if (t.ok) {
            for (int side = 0; side < 2; ++side) {
                const int j = t.j0 + side;
                if (j < 0 || j >= g.n_xi) continue;
                const double wj = side ? t.f : 1.0 - t.f;
                const double *ps = hist + (size_t)j * nn;
                for (int k = 0; k < 4; ++k) {
                    const int i = idx[k];
                    const int iy = i / g.n, ix = i - iy * g.n;
                    const double ww = wj * wc[k];
                    wk[0] += ww * ps[fs + i];
                    wk[1] += ww * ps[2 * fs + i];
                    wk[2] += ww * ps[3 * fs + i];
                    wk[3] += ww * ps[4 * fs + i];
                    const double pc = ps[i];
                    const double pe = ix < g.n - 1 ? ps[i + 1] : -pc;
                    const double pw = ix > 0 ? ps[i - 1] : -pc;
                    const double pn = iy < g.n - 1 ? ps[i + g.n] : -pc;
                    const double pq = iy > 0 ? ps[i - g.n] : -pc;
                    wk[4] += ww * (pe - pw) * inv2h;
                    wk[5] += ww * (pn - pq) * inv2h;
                }
            }
        }
        const double ez = wk[0], bz = wk[1], bx = wk[2], by = wk[3];
        const double ex = -wk[4] + by, ey = -wk[5] - bx;
        const double hq = 0.5 * dt * qm;
        const double p0x = px[p], p0y = py[p], p0z = pz[p];
        const double ux = p0x + hq * ex, uy = p0y + hq * ey, uz = p0z + hq * ez;
        const double g1 = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double tx = hq * bx / g1, ty = hq * by / g1, tz = hq * bz / g1;
        const double t2 = 1.0 + tx * tx + ty * ty + tz * tz;
        const double ss = 2.0 / t2;
        const double upx = ux + (uy * tz - uz * ty);
        const double upy = uy + (uz * tx - ux * tz);
        const double upz = uz + (ux * ty - uy * tx);
        const double cx = upy * tz - upz * ty, cy = upz * tx - upx * tz, cz = upx * ty - upy * tx;
        const double vx = ux + ss * cx + hq * ex;
        const double vy = uy + ss * cy + hq * ey;
        const double vz = uz + ss * cz + hq * ez;
        const double gf = sqrt(1.0 + vx * vx + vy * vy + vz * vz);
        acc += gf - sqrt(1.0 + p0x * p0x + p0y * p0y + p0z * p0z);
        if (!d_hist || !t.ok) continue;
        // reverse, with dL/dgamma_f = scale
        const double vbx = scale * vx / gf, vby = scale * vy / gf, vbz = scale * vz / gf;
        double ebx = hq * vbx, eby = hq * vby, ebz = hq * vbz;
        // u+ = u + ss (up x t): c = up x t
        double ubx = vbx, uby = vby, ubz = vbz;
        const double ssb = vbx * cx + vby * cy + vbz * cz;
        const double cbx = ss * vbx, cby = ss * vby, cbz = ss * vbz;
        // d(cb . (up x t)): up_bar = t x cb, t_bar = cb x up
        const double upbx = ty * cbz - tz * cby, upby = tz * cbx - tx * cbz,
                     upbz = tx * cby - ty * cbx;
        double tbx = cby * upz - cbz * upy, tby = cbz * upx - cbx * upz,
               tbz = cbx * upy - cby * upx;
        // up = u + u x t: u_bar += up_bar + t x up_bar, t_bar += up_bar x u
        ubx += upbx + (ty * upbz - tz * upby);
        uby += upby + (tz * upbx - tx * upbz);
        ubz += upbz + (tx * upby - ty * upbx);
        tbx += upby * uz - upbz * uy;
        tby += upbz * ux - upbx * uz;
        tbz += upbx * uy - upby * ux;
        // ss = 2 / (1 + |t|^2)
        tbx -= ssb * ss * ss * tx;
        tby -= ssb * ss * ss * ty;
        tbz -= ssb * ss * ss * tz;
        // t = hq B / g1
        const double bbx = hq * tbx / g1, bby = hq * tby / g1, bbz = hq * tbz / g1;
        const double g1b = -(tbx * tx + tby * ty + tbz * tz) / g1;
        ubx += g1b * ux / g1;
        uby += g1b * uy / g1;
        ubz += g1b * uz / g1;
        // u = p + hq E
        ebx += hq * ubx;
        eby += hq * uby;
        ebz += hq * ubz;
        // E_x = -dpsi/dx + B_y, E_y = -dpsi/dy - B_x
        const double wb[6] = {ebz, bbz, bbx - eby, bby + ebx, -ebx, -eby};
        for (int side = 0; side < 2; ++side) {
            const int j = t.j0 + side;
            if (j < 0 || j >= g.n_xi) continue;
            const double wj = side ? t.f : 1.0 - t.f;
            double *ds = d_hist + (size_t)j * nn;
            for (int k = 0; k < 4; ++k) {
                const int i = idx[k];
                const int iy = i / g.n, ix = i - iy * g.n;
                const double ww = wj * wc[k];
                atomicAdd(ds + fs + i, ww * wb[0]);
                atomicAdd(ds + 2 * fs + i, ww * wb[1]);
                atomicAdd(ds + 3 * fs + i, ww * wb[2]);
                atomicAdd(ds + 4 * fs + i, ww * wb[3]);
                // grad psi with odd ghosts, transposed
                const double kx = ww * wb[4] * inv2h, ky = ww * wb[5] * inv2h;
                if (ix < g.n - 1) atomicAdd(ds + i + 1, kx); else atomicAdd(ds + i, -kx);
                if (ix > 0) atomicAdd(ds + i - 1, -kx); else atomicAdd(ds + i, kx);
                if (iy < g.n - 1) atomicAdd(ds + i + g.n, ky); else atomicAdd(ds + i, -ky);
                if (iy > 0) atomicAdd(ds + i - g.n, -ky); else atomicAdd(ds + i, ky);
            }
        }
    }
    acc = block_sum256(acc, red);
    if (threadIdx.x == 0) atomicAdd(gain_sum, acc);
}

// Reverse of k_beam_deposit (CIC in x, y, linear in xi; -charge w v_z / (h^2
// dxi0)) for one bunch, momenta fixed.
__global__ void k_beam_deposit_adjoint(const double *x, const double *y, const double *xi,
                                       const double *px, const double *py, const double *pz,
                                       const double *w, int64_t nb, double charge, Geo g,
                                       const double *d_jzb, double *dx, double *dy,
                                       double *dxi, double *dw) {
    const double norm = 1.0 / (g.h * g.h * g.dxi0);
    const size_t nn = (size_t)g.n * g.n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nb;
         p += (int64_t)gridDim.x * blockDim.x) {
        const Tri t = tri(g, x[p], y[p], xi[p]);
        if (!t.ok) {
            dx[p] = dy[p] = dxi[p] = dw[p] = 0.0;
            continue;
        }
        const double ux = px[p], uy = py[p], uz = pz[p];
        const double gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double qw = -charge * uz / gam * norm;  // d q / d w
        const double q = qw * w[p];
        double A[2] = {0.0, 0.0}, X[2] = {0.0, 0.0}, Y[2] = {0.0, 0.0};
        for (int side = 0; side < 2; ++side) {
            const int j = t.j0 + side;
            if (j < 0 || j >= g.n_xi) continue;
            const double *d = d_jzb + (size_t)j * nn;
            const double u00 = d[t.iy0 * g.n + t.ix0], u01 = d[t.iy0 * g.n + t.ix1];
            const double u10 = d[t.iy1 * g.n + t.ix0], u11 = d[t.iy1 * g.n + t.ix1];
            A[side] = t.wy0 * (t.wx0 * u00 + t.wx1 * u01) + t.wy1 * (t.wx0 * u10 + t.wx1 * u11);
            X[side] = (t.wy0 * (u01 - u00) + t.wy1 * (u11 - u10)) / g.h;
            Y[side] = (t.wx0 * (u10 - u00) + t.wx1 * (u11 - u01)) / g.h;
        }
        const double w0 = 1.0 - t.f, w1 = t.f;
        dw[p] = qw * (w0 * A[0] + w1 * A[1]);
        dx[p] = q * (w0 * X[0] + w1 * X[1]);
        dy[p] = q * (w0 * Y[0] + w1 * Y[1]);
        dxi[p] = q * (A[1] - A[0]) / g.dxi0;
    }
}

// dL/dtable of the lattice weights w = n(r0) h^2 / ppc and of n_ion = their
// deposit; the table is piecewise linear on [0, r_max] (k_init_plasma).
__global__ void k_profile_adjoint(int n, int ppc, int s, double x_min, double y_min, double h,
                                  int n_coef, double r_max, const double *d_w,
                                  const double *d_nion, double *d_table) {
    extern __shared__ double acc[];
    for (int k = threadIdx.x; k < n_coef; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    const int64_t np = (int64_t)n * n * ppc;
    const double s2 = 1.0 / (h * h);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ppc;
        const int k = (int)(p - c * ppc);
        const int iy = (int)(c / n), ix = (int)(c - (int64_t)iy * n);
        const int ky = k / s, kx = k - ky * s;
        const double xx = x_min + (ix + (kx + 0.5) / s) * h;
        const double yy = y_min + (iy + (ky + 0.5) / s) * h;
        const Cic cc = cic_stencil(xx, yy, x_min, y_min, h, n);
        const double wb = (d_w[p] + cic_gather(d_nion, cc) * s2) * (h * h / ppc);
        if (n_coef == 1) {
            atomicAdd(acc, wb);
            continue;
        }
        const double r = sqrt(xx * xx + yy * yy);
        const double sr = fmin(r / r_max * (n_coef - 1), (double)(n_coef - 1));
        int i = (int)floor(sr);
        if (i > n_coef - 2) i = n_coef - 2;
        const double f = sr - i;
        atomicAdd(acc + i, wb * (1.0 - f));
        atomicAdd(acc + i + 1, wb * f);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_coef; k += blockDim.x)
        if (acc[k] != 0.0) atomicAdd(d_table + k, acc[k]);
}

struct Theta {
    double a, sx, sy, sz, xc, yc, xic, tilt;
};

__global__ void k_bigaussian(Theta th, const double *z, int64_t n, double pz0, double w0,
                             double *x, double *y, double *xi, double *px, double *py,
                             double *pz, double *w) {
    const double r2 = 0.70710678118654752440;  // 1/sqrt(2)
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double z0 = z[p], z1 = z[n + p], z2 = z[2 * n + p];
        const double d = th.sz * r2 * z2;
        xi[p] = th.xic + d;
        x[p] = th.xc + th.tilt * d + th.sx * r2 * z0;
        y[p] = th.yc + th.sy * r2 * z1;
        px[p] = 0.0;
        py[p] = 0.0;
        pz[p] = pz0;
        w[p] = w0;
    }
}

// partial sums of dL/dtheta over the particles (8 sums per block -> out)
__global__ void k_bigaussian_adjoint(Theta th, const double *z, int64_t n, const double *dx,
                                     const double *dy, const double *dxi, const double *dw,
                                     double *out) {
    __shared__ double red[32];
    const double r2 = 0.70710678118654752440;
    double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double sw = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double z0 = z[p], z1 = z[n + p], z2 = z[2 * n + p];
        const double bx = dx[p], by = dy[p], bxi = dxi[p];
        sw += dw[p];
        s[1] += bx * r2 * z0;
        s[2] += by * r2 * z1;
        s[3] += (bxi + th.tilt * bx) * r2 * z2;
        s[4] += bx;
        s[5] += by;
        s[6] += bxi;
        s[7] += bx * th.sz * r2 * z2;
    }
    // w = A pi^(3/2) sx sy sz / n: its partial derivatives times sum(dw)
    const double c = pow(M_PI, 1.5) / (double)n;
    s[0] = sw * c * th.sx * th.sy * th.sz;
    s[1] += sw * c * th.a * th.sy * th.sz;
    s[2] += sw * c * th.a * th.sx * th.sz;
    s[3] += sw * c * th.a * th.sx * th.sy;
    for (int k = 0; k < 8; ++k) {
        const double t = block_sum256(s[k], red);
        if (threadIdx.x == 0) atomicAdd(out + k, t);
    }
}

}  // namespace

cudaError_t qs_launch_beam_gain(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                double x_max, double y_min, double y_max, double h, int n_xi,
                                double xi_min, double dxi0, const double *hist, double dt,
                                double scale, double *gain_sum, double *d_hist) {
    if (b.n <= 0) return cudaSuccess;
    const Geo g{n, n_xi, x_min, x_max, y_min, y_max, h, xi_min, dxi0};
    k_beam_gain<<<blocks_for(b.n), kThreads, 0, st>>>(b.x, b.y, b.xi, b.px, b.py, b.pz, b.n,
                                                      b.q_over_m, g, hist, dt, scale, gain_sum,
                                                      d_hist);
    return cudaGetLastError();
}

cudaError_t qs_launch_beam_deposit_adjoint(cudaStream_t st, const qs_beam &b, int n,
                                           double x_min, double x_max, double y_min,
                                           double y_max, double h, int n_xi, double xi_min,
                                           double dxi0, const double *d_jzb, double *dx,
                                           double *dy, double *dxi, double *dw) {
    if (b.n <= 0) return cudaSuccess;
    const Geo g{n, n_xi, x_min, x_max, y_min, y_max, h, xi_min, dxi0};
    k_beam_deposit_adjoint<<<blocks_for(b.n), kThreads, 0, st>>>(
        b.x, b.y, b.xi, b.px, b.py, b.pz, b.w, b.n, b.charge, g, d_jzb, dx, dy, dxi, dw);
    return cudaGetLastError();
}

cudaError_t qs_launch_profile_adjoint(cudaStream_t st, int n, int ppc, double x_min,
                                      double y_min, double h, int n_coef, double r_max,
                                      const double *d_w, const double *d_nion,
                                      double *d_table) {
    int s = 1;
    while (s * s < ppc) ++s;
    const int64_t np = (int64_t)n * n * ppc;
    k_profile_adjoint<<<blocks_for(np), kThreads, n_coef * sizeof(double), st>>>(
        n, ppc, s, x_min, y_min, h, n_coef, r_max, d_w, d_nion, d_table);
    return cudaGetLastError();
}

extern "C" {

int qs_bigaussian_beam(const double *theta, const double *z, int64_t n, double gamma,
                       qs_beam *out, void *cuda_stream) {
    if (!theta || !out || n < 0 || (n > 0 && !z) || !(gamma >= 1.0)) return QS_ERR_ARG;
    if (n > 0 && (!out->x || !out->y || !out->xi || !out->px || !out->py || !out->pz || !out->w))
        return QS_ERR_ARG;
    out->n = n;
    if (n == 0) return QS_OK;
    const Theta th{theta[0], theta[1], theta[2], theta[3], theta[4], theta[5], theta[6], theta[7]};
    const double w0 = th.a * pow(M_PI, 1.5) * th.sx * th.sy * th.sz / (double)n;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_bigaussian<<<blocks_for(n), kThreads, 0, st>>>(th, z, n, sqrt(gamma * gamma - 1.0), w0,
                                                     out->x, out->y, out->xi, out->px, out->py,
                                                     out->pz, out->w);
    return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

int qs_bigaussian_adjoint(const double *theta, const double *z, int64_t n, const double *d_x,
                          const double *d_y, const double *d_xi, const double *d_w,
                          double *d_theta, void *cuda_stream) {
    if (!theta || !d_theta || n < 0 || (n > 0 && (!z || !d_x || !d_y || !d_xi || !d_w)))
        return QS_ERR_ARG;
    for (int k = 0; k < 8; ++k) d_theta[k] = 0.0;
    if (n == 0) return QS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const Theta th{theta[0], theta[1], theta[2], theta[3], theta[4], theta[5], theta[6], theta[7]};
    double *dev = nullptr;
    if (cudaMallocAsync(&dev, 8 * sizeof(double), st) != cudaSuccess) {
        cudaGetLastError();
        return QS_ERR_OOM;
    }
    cudaError_t e = cudaMemsetAsync(dev, 0, 8 * sizeof(double), st);
    if (e == cudaSuccess) {
        k_bigaussian_adjoint<<<blocks_for(n), kThreads, 0, st>>>(th, z, n, d_x, d_y, d_xi, d_w,
                                                                 dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_theta, dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dev, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        return QS_ERR_CUDA;
    }
    return QS_OK;
}

}  // extern "C"
