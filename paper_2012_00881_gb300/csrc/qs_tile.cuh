// Tiled (temporally blocked) grid levels for the float32 inner cycles of the
// refined form.
//
// A grid-wide level normally costs one grid barrier per red-black half sweep.
// Here every block takes an output tile plus a halo, stages the level's data
// in shared memory and performs all half sweeps of a leg there, recomputing
// the halo redundantly; only the cells far enough from a cut edge of the
// staged region are exact after each half sweep, and the halo is as wide as
// the number of half sweeps (plus one for the residual).  A level then costs
// two grid barriers per V-cycle (down: smooth + residual + restriction; up:
// prolongation + smooth).  The inner correction starts from zero on every
// level, so the down leg needs no neighbour data but the right-hand side.
#pragma once

#include "qs_mg.cuh"

namespace qstile {

using qsmg::Lvl;

struct Region {
    int ox, oy, RX, RY, R;   // staged region: origin and extent
    int ax, bx, ay, by;      // its intersection with the domain
    bool cl, cr, cb, ct;     // which sides are cut (not the domain wall)
};

__device__ __forceinline__ Region make_region(int tx0, int ty0, int TX, int TY, int H, int n) {
    Region g;
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

// distance of (x, y) from the nearest cut side of the staged region
__device__ __forceinline__ int cut_distance(const Region &g, int x, int y) {
    int d = 1 << 30;
    if (g.cl) d = min(d, x - g.ax);
    if (g.cr) d = min(d, g.bx - x);
    if (g.cb) d = min(d, y - g.ay);
    if (g.ct) d = min(d, g.by - y);
    return d;
}

// Half sweeps s = s0 .. s0 + ns - 1 on the staged region: a cell is updated
// in half sweep s only if it is at least s + 1 cells from every cut side.
__device__ void staged_sweeps(const Region &g, int n, float h2, int nc, float *su[2],
                              float *sf[2], const float *sd, int ns) {
    for (int s = 0; s < ns; ++s) {
        const int color = s & 1;
        for (int li = threadIdx.x; li < g.R; li += blockDim.x) {
            const int x = g.ox + li % g.RX, y = g.oy + li / g.RX;
            if (x < g.ax || x > g.bx || y < g.ay || y > g.by) continue;
            if (((x + y) & 1) != color) continue;
            if (cut_distance(g, x, y) < s + 1) continue;
            const int nw = qsmg::walls(x, y, n);
            const float di = sd ? sd[li]
                                : (nw == 0 ? 0.25f : (nw == 1 ? 0.2f : (nw == 2 ? (1.f / 6.f) : 1.f / (4 + nw))));
            for (int c = 0; c < nc; ++c) {
                const float *u = su[c];
                float nb = 0.f;
                if (x > 0) nb += u[li - 1];
                if (x < n - 1) nb += u[li + 1];
                if (y > 0) nb += u[li - g.RX];
                if (y < n - 1) nb += u[li + g.RX];
                su[c][li] = (nb - h2 * sf[c][li]) * di;
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float staged_op(const float *u, const float *k, const Region &g,
                                           int n, float inv_h2, int li, int x, int y) {
    float nb = 0.f;
    if (x > 0) nb += u[li - 1];
    if (x < n - 1) nb += u[li + 1];
    if (y > 0) nb += u[li - g.RX];
    if (y < n - 1) nb += u[li + g.RX];
    float r = (nb - (float)(4 + qsmg::walls(x, y, n)) * u[li]) * inv_h2;
    if (k) r -= k[li] * u[li];
    return r;
}

// Shared memory (bytes) for one staged tile.
__host__ __device__ inline size_t tile_smem_bytes(int TX, int TY, int nu) {
    const int H = 2 * nu + 1;
    return (size_t)6 * (TX + 2 * H) * (TY + 2 * H) * sizeof(float);
}

// Down leg of grid level F -> coarse C for every tile owned by this block:
// pre-smoothing from a zero iterate, residual, 4-cell restriction (and kappa,
// inverse diagonal); the pre-smoothed tile is written to F.u.
__device__ void down_level(const Lvl<float> &F, const Lvl<float> &C, int nc, int nu1, int TX,
                           int TY, float *sm, int bid, int nblk) {
    const int n = F.n, m = C.n;
    const int H = 2 * nu1 + 1;
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const float h2 = (float)F.h2, inv_h2 = (float)(1.0 / F.h2);
    const bool scr = F.k != nullptr;
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const Region g = make_region(tx0, ty0, TX, TY, H, n);
        float *su[2] = {sm, sm + g.R};
        float *sf[2] = {sm + 2 * g.R, sm + 3 * g.R};
        float *sk = scr ? sm + 4 * g.R : nullptr;
        float *sd = scr ? sm + 5 * g.R : nullptr;
        for (int li = threadIdx.x; li < g.R; li += blockDim.x) {
            const int x = g.ox + li % g.RX, y = g.oy + li / g.RX;
            const bool in = x >= 0 && x < n && y >= 0 && y < n;
            const int gi = y * n + x;
            for (int c = 0; c < nc; ++c) {
                su[c][li] = 0.f;
                sf[c][li] = in ? F.f[c][gi] : 0.f;
            }
            if (scr) {
                sk[li] = in ? F.k[gi] : 0.f;
                sd[li] = in ? F.d[gi] : 0.f;
            }
        }
        __syncthreads();
        staged_sweeps(g, n, h2, nc, su, sf, sd, 2 * nu1);
        // residual on the tile, restricted to the coarse cells it covers
        const int CTX = TX / 2, CTY = TY / 2, cx0 = tx0 / 2, cy0 = ty0 / 2;
        for (int q = threadIdx.x; q < CTX * CTY; q += blockDim.x) {
            const int I = cx0 + q % CTX, J = cy0 + q / CTX;
            if (I >= m || J >= m) continue;
            const int x0 = 2 * I, y0 = 2 * J;
            const int l0 = (y0 - g.oy) * g.RX + (x0 - g.ox);
            for (int c = 0; c < nc; ++c) {
                float s = sf[c][l0] - staged_op(su[c], sk, g, n, inv_h2, l0, x0, y0);
                s += sf[c][l0 + 1] - staged_op(su[c], sk, g, n, inv_h2, l0 + 1, x0 + 1, y0);
                s += sf[c][l0 + g.RX] - staged_op(su[c], sk, g, n, inv_h2, l0 + g.RX, x0, y0 + 1);
                s += sf[c][l0 + g.RX + 1] -
                     staged_op(su[c], sk, g, n, inv_h2, l0 + g.RX + 1, x0 + 1, y0 + 1);
                C.f[c][J * m + I] = 0.25f * s;
            }
            if (scr) {
                const float kk = 0.25f * (sk[l0] + sk[l0 + 1] + sk[l0 + g.RX] + sk[l0 + g.RX + 1]);
                C.k[J * m + I] = kk;
                C.d[J * m + I] = 1.f / ((float)(4 + qsmg::walls(I, J, m)) + (float)C.h2 * kk);
            }
        }
        for (int q = threadIdx.x; q < TX * TY; q += blockDim.x) {
            const int x = tx0 + q % TX, y = ty0 + q / TX;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            for (int c = 0; c < nc; ++c) F.u[c][y * n + x] = su[c][li];
        }
        __syncthreads();
    }
}

// Up leg of grid level F: F.u (pre-smoothed) + bilinear interpolation of the
// coarse correction `cu` (side m), then post-smoothing; the tile result goes
// to `out` (float32), or is added into the float64 iterate `fin` (level 0 of
// the refined form).
__device__ void up_level(const Lvl<float> &F, float *const cu[2], int m, int nc, int nu2, int TX,
                         int TY, float *sm, int bid, int nblk, float *const out[2],
                         double *const *fin) {
    const int n = F.n;
    const int H = 2 * nu2;
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const float h2 = (float)F.h2;
    const bool scr = F.k != nullptr;
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const Region g = make_region(tx0, ty0, TX, TY, H, n);
        float *su[2] = {sm, sm + g.R};
        float *sf[2] = {sm + 2 * g.R, sm + 3 * g.R};
        float *sd = scr ? sm + 5 * g.R : nullptr;
        for (int li = threadIdx.x; li < g.R; li += blockDim.x) {
            const int x = g.ox + li % g.RX, y = g.oy + li / g.RX;
            const bool in = x >= 0 && x < n && y >= 0 && y < n;
            const int gi = y * n + x;
            if (scr) sd[li] = in ? F.d[gi] : 0.f;
            if (!in) {
                for (int c = 0; c < nc; ++c) su[c][li] = sf[c][li] = 0.f;
                continue;
            }
            const int I = x >> 1, J = y >> 1;
            const int I2 = I + ((x & 1) ? 1 : -1), J2 = J + ((y & 1) ? 1 : -1);
            const bool xin = (I2 >= 0 && I2 < m), yin = (J2 >= 0 && J2 < m);
            for (int c = 0; c < nc; ++c) {
                const float *uc = cu[c];
                const float v00 = uc[J * m + I];
                const float v10 = xin ? uc[J * m + I2] : -v00;
                const float v01 = yin ? uc[J2 * m + I] : -v00;
                float v11;
                if (xin && yin) v11 = uc[J2 * m + I2];
                else if (xin) v11 = -uc[J * m + I2];
                else if (yin) v11 = -uc[J2 * m + I];
                else v11 = v00;
                su[c][li] = F.u[c][gi] + (9.f * v00 + 3.f * v10 + 3.f * v01 + v11) * 0.0625f;
                sf[c][li] = F.f[c][gi];
            }
        }
        __syncthreads();
        staged_sweeps(g, n, h2, nc, su, sf, sd, 2 * nu2);
        for (int q = threadIdx.x; q < TX * TY; q += blockDim.x) {
            const int x = tx0 + q % TX, y = ty0 + q / TX;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            for (int c = 0; c < nc; ++c) {
                if (fin) fin[c][y * n + x] += (double)su[c][li];
                else out[c][y * n + x] = su[c][li];
            }
        }
        __syncthreads();
    }
}

}  // namespace qstile
