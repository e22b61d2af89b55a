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
using qsmg::Walk;

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

// Half sweeps 0 .. ns-1 on the staged region: a cell is updated in half
// sweep s only if it is at least s + 1 cells from every cut side.
template <int NC>
__device__ void staged_sweeps(const Region &g, int n, float h2, float *const su0,
                              float *const su1, const float *const sf0, const float *const sf1,
                              const float *const sd, int ns) {
    // cells are visited through the in-domain part of the region only
    const int wx = g.bx - g.ax + 1, wy = g.by - g.ay + 1;
    const int RX = g.RX;
    const int lo_x = g.cl ? g.ax : -(1 << 20), hi_x = g.cr ? g.bx : (1 << 20);
    const int lo_y = g.cb ? g.ay : -(1 << 20), hi_y = g.ct ? g.by : (1 << 20);
    for (int s = 0; s < ns; ++s) {
        const int color = s & 1;
        for (Walk w(threadIdx.x, blockDim.x, wx); w.q < wx * wy; w.next()) {
            const int x = g.ax + w.col, y = g.ay + w.row;
            if (((x + y) & 1) != color) continue;
            const int d = min(min(x - lo_x, hi_x - x), min(y - lo_y, hi_y - y));
            if (d < s + 1) continue;
            const int li = (y - g.oy) * RX + (x - g.ox);
            const float di = sd ? sd[li] : qsmg::const_inv_diag<float>(qsmg::walls(x, y, n));
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float *u = c ? su1 : su0;
                float nb = 0.f;
                if (x > 0) nb += u[li - 1];
                if (x < n - 1) nb += u[li + 1];
                if (y > 0) nb += u[li - RX];
                if (y < n - 1) nb += u[li + RX];
                u[li] = (nb - h2 * (c ? sf1 : sf0)[li]) * di;
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float staged_op(const float *u, const float *k, int RX, int n,
                                           float inv_h2, int li, int x, int y) {
    float nb = 0.f;
    if (x > 0) nb += u[li - 1];
    if (x < n - 1) nb += u[li + 1];
    if (y > 0) nb += u[li - RX];
    if (y < n - 1) nb += u[li + RX];
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
template <int NC>
__device__ void down_level(const Lvl<float> F, const Lvl<float> C, int nu1, int TX, int TY,
                           float *sm, int bid, int nblk) {
    const int n = F.n, m = C.n;
    const int H = 2 * nu1 + 1;
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const float h2 = (float)F.h2, inv_h2 = (float)(1.0 / F.h2), ch2 = (float)C.h2;
    const bool scr = F.k != nullptr;
    const float *const gf0 = F.f[0];
    const float *const gf1 = F.f[NC - 1];
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const Region g = make_region(tx0, ty0, TX, TY, H, n);
        float *const su0 = sm;
        float *const su1 = sm + g.R;
        float *const sf0 = sm + 2 * g.R;
        float *const sf1 = sm + 3 * g.R;
        float *const sk = scr ? sm + 4 * g.R : nullptr;
        float *const sd = scr ? sm + 5 * g.R : nullptr;
        for (Walk w(threadIdx.x, blockDim.x, g.RX); w.q < g.R; w.next()) {
            const int x = g.ox + w.col, y = g.oy + w.row;
            const bool in = x >= 0 && x < n && y >= 0 && y < n;
            const int gi = y * n + x, li = w.q;
            su0[li] = 0.f;
            sf0[li] = in ? gf0[gi] : 0.f;
            if (NC > 1) {
                su1[li] = 0.f;
                sf1[li] = in ? gf1[gi] : 0.f;
            }
            if (scr) {
                sk[li] = in ? F.k[gi] : 0.f;
                sd[li] = in ? F.d[gi] : 0.f;
            }
        }
        __syncthreads();
        staged_sweeps<NC>(g, n, h2, su0, su1, sf0, sf1, sd, 2 * nu1);
        // residual on the tile, restricted to the coarse cells it covers
        const int CTX = TX / 2, CTY = TY / 2, cx0 = tx0 / 2, cy0 = ty0 / 2;
        for (Walk w(threadIdx.x, blockDim.x, CTX); w.q < CTX * CTY; w.next()) {
            const int I = cx0 + w.col, J = cy0 + w.row;
            if (I >= m || J >= m) continue;
            const int x0 = 2 * I, y0 = 2 * J;
            const int l0 = (y0 - g.oy) * g.RX + (x0 - g.ox);
            const int RX = g.RX;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float *su = c ? su1 : su0;
                const float *sf = c ? sf1 : sf0;
                float s = sf[l0] - staged_op(su, sk, RX, n, inv_h2, l0, x0, y0);
                s += sf[l0 + 1] - staged_op(su, sk, RX, n, inv_h2, l0 + 1, x0 + 1, y0);
                s += sf[l0 + RX] - staged_op(su, sk, RX, n, inv_h2, l0 + RX, x0, y0 + 1);
                s += sf[l0 + RX + 1] - staged_op(su, sk, RX, n, inv_h2, l0 + RX + 1, x0 + 1, y0 + 1);
                C.f[c][J * m + I] = 0.25f * s;
            }
            if (scr) {
                const float kk = 0.25f * (sk[l0] + sk[l0 + 1] + sk[l0 + RX] + sk[l0 + RX + 1]);
                C.k[J * m + I] = kk;
                C.d[J * m + I] = 1.f / ((float)(4 + qsmg::walls(I, J, m)) + ch2 * kk);
            }
        }
        for (Walk w(threadIdx.x, blockDim.x, TX); w.q < TX * TY; w.next()) {
            const int x = tx0 + w.col, y = ty0 + w.row;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            F.u[0][y * n + x] = su0[li];
            if (NC > 1) F.u[1][y * n + x] = su1[li];
        }
        __syncthreads();
    }
}

// Up leg of grid level F: F.u (pre-smoothed) + bilinear interpolation of the
// coarse correction `cu` (side m), then post-smoothing; the tile result goes
// to `out` (float32), or is added into the float64 iterate `fin` (level 0 of
// the refined form).
template <int NC>
__device__ void up_level(const Lvl<float> F, const float *cu0, const float *cu1, int m, int nu2,
                         int TX, int TY, float *sm, int bid, int nblk, float *out0, float *out1,
                         double *fin0, double *fin1) {
    const int n = F.n;
    const int H = 2 * nu2;
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const float h2 = (float)F.h2;
    const bool scr = F.k != nullptr;
    const float *const gu0 = F.u[0];
    const float *const gu1 = F.u[NC - 1];
    const float *const gf0 = F.f[0];
    const float *const gf1 = F.f[NC - 1];
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const Region g = make_region(tx0, ty0, TX, TY, H, n);
        float *const su0 = sm;
        float *const su1 = sm + g.R;
        float *const sf0 = sm + 2 * g.R;
        float *const sf1 = sm + 3 * g.R;
        float *const sd = scr ? sm + 5 * g.R : nullptr;
        for (Walk w(threadIdx.x, blockDim.x, g.RX); w.q < g.R; w.next()) {
            const int x = g.ox + w.col, y = g.oy + w.row;
            const bool in = x >= 0 && x < n && y >= 0 && y < n;
            const int gi = y * n + x, li = w.q;
            if (scr) sd[li] = in ? F.d[gi] : 0.f;
            if (!in) {
                su0[li] = sf0[li] = 0.f;
                if (NC > 1) su1[li] = sf1[li] = 0.f;
                continue;
            }
            su0[li] = gu0[gi] + qsmg::bilinear(cu0, m, x, y);
            sf0[li] = gf0[gi];
            if (NC > 1) {
                su1[li] = gu1[gi] + qsmg::bilinear(cu1, m, x, y);
                sf1[li] = gf1[gi];
            }
        }
        __syncthreads();
        staged_sweeps<NC>(g, n, h2, su0, su1, sf0, sf1, sd, 2 * nu2);
        for (Walk w(threadIdx.x, blockDim.x, TX); w.q < TX * TY; w.next()) {
            const int x = tx0 + w.col, y = ty0 + w.row;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            const int gi = y * n + x;
            if (fin0) {
                fin0[gi] += (double)su0[li];
                if (NC > 1) fin1[gi] += (double)su1[li];
            } else {
                out0[gi] = su0[li];
                if (NC > 1) out1[gi] = su1[li];
            }
        }
        __syncthreads();
    }
}

}  // namespace qstile
