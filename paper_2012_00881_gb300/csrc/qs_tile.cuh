// Tiled (temporally blocked) grid levels for the float32 inner cycles of the
// refined form.
//
// A grid-wide level normally costs one grid barrier per red-black half sweep.
// Here every block takes an output tile plus a halo, stages the level's data
// in shared memory and performs all half sweeps of a leg there, recomputing
// the halo redundantly; only the cells far enough from a cut edge of the
// staged region are exact after each half sweep, and the halo is as wide as
// the number of half sweeps (plus one for the residual).  A down leg then
// costs one grid barrier per level (smooth + residual + restriction), and
// all the up legs together one (the up cascade below).  The inner correction
// starts from zero on every level, so the down leg needs no neighbour data
// but the right-hand side.
#pragma once

#include "qs_mg.cuh"

namespace qstile {

using qsmg::Lvl;
using qsmg::Walk;
using qsmg::cp_async_f32;
using qsmg::cp_async_f64;
using qsmg::cp_async_wait_all;

struct Region {
    int ox, oy, RX, RY, R;   // staged storage: origin and extent (cell (x, y) at
                             // (y - oy) RX + (x - ox))
    int ax, bx, ay, by;      // the region's intersection with the domain
    bool cl, cr, cb, ct;     // which sides are cut (not the domain wall)
};

// Columns of padding a storage window may add to a region's width (V - 1 on
// each side for vectors of V = 4 float32 values).
constexpr int kAlignPad = 6;

// The region of the tile at (tx0, ty0) with halo H on a level of side n.
// Its storage starts at a column that is a multiple of V and has a width
// that is a multiple of V, so that rows can be staged with 16-byte copies of
// V = 16 / sizeof(element) values; the extra columns are never updated.
__device__ __forceinline__ Region make_region(int tx0, int ty0, int TX, int TY, int H, int n,
                                              int V = 1) {
    Region g;
    const int ox = tx0 - H;
    g.oy = ty0 - H;
    g.RY = TY + 2 * H;
    g.ax = max(ox, 0);
    g.bx = min(ox + TX + 2 * H - 1, n - 1);
    g.ay = max(g.oy, 0);
    g.by = min(g.oy + g.RY - 1, n - 1);
    g.cl = g.ax > 0;
    g.cr = g.bx < n - 1;
    g.cb = g.ay > 0;
    g.ct = g.by < n - 1;
    g.ox = ox >= 0 ? ox - ox % V : -((-ox + V - 1) / V) * V;
    const int end = ox + TX + 2 * H;  // one past the region's last column
    g.RX = ((end - g.ox + V - 1) / V) * V;
    g.R = g.RX * g.RY;
    return g;
}

// 16-byte global -> shared copy (zero-filled when !valid); both addresses
// 16-byte aligned
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// Visit the storage of region g on a level of side n in groups of V cells
// (V = 16 / sizeof(T)): f(li, gi, in) for the group's first cell, its
// global index and whether the group lies in the domain.  With n a multiple
// of V every group lies wholly inside or outside the domain (group origins
// are multiples of V), so one 16-byte copy stages it.
template <typename T, typename F>
__device__ __forceinline__ void for_groups(const Region &g, int n, F f) {
    constexpr int V = 16 / (int)sizeof(T);
    const int gx = g.RX / V;
    for (int q = threadIdx.x; q < g.RY * gx; q += blockDim.x) {
        const int r = q / gx, c = q - r * gx;
        const int x = g.ox + c * V, y = g.oy + r;
        const bool in = x >= 0 && x < n && y >= 0 && y < n;
        f(r * g.RX + c * V, in ? y * n + x : 0, in);
    }
}

// Half sweeps 0 .. ns-1 on the staged region: a cell is updated in half
// sweep s only if it is at least s + 1 cells from every cut side.
template <int NC, typename T>
__device__ void staged_sweeps(const Region &g, int n, T h2, T *const su0, T *const su1,
                              const T *const sf0, const T *const sf1, const T *const sd, int ns,
                              T omega) {
    // Half sweep s updates, within the in-domain part of the region, the
    // cells of its colour at least s + 1 cells from every cut side: a
    // rectangle shrinking by one cell per half sweep on the cut sides.  Only
    // those cells are visited (the colour's cells of each row, two apart).
    const int RX = g.RX;
    for (int s = 0; s < ns; ++s) {
        const int color = s & 1;
        const int X0 = g.cl ? g.ax + s + 1 : g.ax, X1 = g.cr ? g.bx - s - 1 : g.bx;
        const int Y0 = g.cb ? g.ay + s + 1 : g.ay, Y1 = g.ct ? g.by - s - 1 : g.by;
        const int rows = Y1 - Y0 + 1, hw = (X1 - X0 + 2) >> 1;
        const int cnt = (rows > 0 && X1 >= X0) ? rows * hw : 0;
        for (Walk w(threadIdx.x, blockDim.x, hw > 0 ? hw : 1); w.q < cnt; w.next()) {
            const int y = Y0 + w.row;
            const int x = X0 + ((X0 + y + color) & 1) + 2 * w.col;
            if (x > X1) continue;
            const int li = (y - g.oy) * RX + (x - g.ox);
            const T di = sd ? sd[li] : qsmg::const_inv_diag<T>(qsmg::walls(x, y, n));
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T *u = c ? su1 : su0;
                T nb = T(0);
                if (x > 0) nb += u[li - 1];
                if (x < n - 1) nb += u[li + 1];
                if (y > 0) nb += u[li - RX];
                if (y < n - 1) nb += u[li + RX];
                const T gv = (nb - h2 * (c ? sf1 : sf0)[li]) * di;
                const T uo = u[li];
                u[li] = uo + omega * (gv - uo);
            }
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ T staged_op(const T *u, const T *k, int RX, int n, T inv_h2, int li,
                                       int x, int y) {
    T nb = T(0);
    if (x > 0) nb += u[li - 1];
    if (x < n - 1) nb += u[li + 1];
    if (y > 0) nb += u[li - RX];
    if (y < n - 1) nb += u[li + RX];
    T r = (nb - (T)(4 + qsmg::walls(x, y, n)) * u[li]) * inv_h2;
    if (k) r -= k[li] * u[li];
    return r;
}

// Layout of a staged down-leg region in shared memory: six arrays (u0, u1,
// f0, f1, kappa, inverse diagonal) of R cells.
template <typename T>
struct TileSmem {
    T *su0, *su1, *sf0, *sf1, *sk, *sd;
};

template <typename T>
__device__ __forceinline__ TileSmem<T> tile_layout(T *sm, int R) {
    TileSmem<T> t;
    t.su0 = sm;
    t.su1 = sm + R;
    t.sf0 = sm + 2 * R;
    t.sf1 = sm + 3 * R;
    t.sk = sm + 4 * R;
    t.sd = sm + 5 * R;
    return t;
}

// Region and coarse-window sizes (cells) of the up cascade for a level-0
// tile TX x TY and nu2 post-sweeps: the level-0 region is the tile plus a
// halo 2 nu2 + 1; each coarser level needs the window of coarse cells that
// the finer region prolongs from (at most half its width plus 3), staged
// with a halo 2 nu2.  The widths converge to 6 + 8 nu2, so a fixed number of
// levels bounds them.
__host__ __device__ inline void cascade_bounds(int TX, int TY, int nu2, int &rbig, int &wbig) {
    int x = TX + 2 * (2 * nu2 + 1), y = TY + 2 * (2 * nu2 + 1);
    rbig = (x + kAlignPad) * y;  // storage may be kAlignPad columns wider
    wbig = 0;
    for (int l = 1; l < 16; ++l) {
        const int wx = x / 2 + 3, wy = y / 2 + 3;
        wbig = wbig > wx * wy ? wbig : wx * wy;
        x = wx + 4 * nu2;
        y = wy + 4 * nu2;
        rbig = rbig > (x + kAlignPad) * y ? rbig : (x + kAlignPad) * y;
    }
}

// Layout of the up cascade: six region arrays, two ping-pong coarse windows
// of two components, float64 copies of the level-0 tile.
struct CascadeSmem {
    float *su0, *su1, *sf0, *sf1, *sd;
    float *win;  // window buffer b, component c at win + (2 b + c) * wbig
    int wbig;
    double *du0, *du1, *dr0, *dr1, *dk;
};

__device__ __forceinline__ CascadeSmem cascade_layout(float *sm, int R, int TX, int TY,
                                                      int nu2) {
    int rbig, wbig;
    cascade_bounds(TX, TY, nu2, rbig, wbig);
    CascadeSmem t;
    t.su0 = sm;
    t.su1 = sm + R;
    t.sf0 = sm + 2 * R;
    t.sf1 = sm + 3 * R;
    t.sd = sm + 5 * R;
    t.win = sm + 6 * rbig;
    t.wbig = wbig;
    const size_t off = ((size_t)(6 * rbig + 4 * wbig) * sizeof(float) + 15) & ~(size_t)15;
    double *d = (double *)((char *)sm + off);
    const int T = TX * TY;
    t.du0 = d;
    t.du1 = d + T;
    t.dr0 = d + 2 * T;
    t.dr1 = d + 3 * T;
    t.dk = d + 4 * T;
    return t;
}

// Shared memory (bytes) for the staged legs with tile TX x TY and any tile
// obtained from it by halving sides down to 8 (nu = the larger sweep count,
// nu2 = post-sweeps): the down legs' region or the up cascade, whichever is
// larger.
__host__ __device__ inline size_t tile_smem_bytes(int TX, int TY, int nu, int nu2) {
    size_t best = 0;
    for (int tx = TX, ty = TY;;) {
        const int H = 2 * nu + 1;
        const size_t a = (size_t)6 * (tx + 2 * H + kAlignPad) * (ty + 2 * H) * sizeof(float);
        int rbig, wbig;
        cascade_bounds(tx, ty, nu2, rbig, wbig);
        size_t b = ((size_t)(6 * rbig + 4 * wbig) * sizeof(float) + 15) & ~(size_t)15;
        b += (size_t)5 * tx * ty * sizeof(double);
        best = best > a ? best : a;
        best = best > b ? best : b;
        if (tx >= ty && tx > 8) tx >>= 1;
        else if (ty > 8) ty >>= 1;
        else break;
    }
    return best;
}

// Shared memory (bytes) of the float64 form's staged legs (down_level and
// up_level with T = double) for tile TX x TY and its halvings down to 8: six
// float64 arrays over the tile plus the larger halo (2 nu1 + 1 down,
// 2 nu2 + 1 on the level-0 up leg).
__host__ __device__ inline size_t tile64_smem_bytes(int TX, int TY, int nu, int nu2) {
    size_t best = 0;
    const int H = 2 * (nu > nu2 ? nu : nu2) + 1;
    for (int tx = TX, ty = TY;;) {
        const size_t a = (size_t)6 * (tx + 2 * H + kAlignPad) * (ty + 2 * H) * sizeof(double);
        best = best > a ? best : a;
        if (tx >= ty && tx > 8) tx >>= 1;
        else if (ty > 8) ty >>= 1;
        else break;
    }
    return best;
}

// Bilinear cell-centred interpolation (odd ghosts) of a coarse array of side
// m held as a window with origin (cox, coy) and row pitch cp; the same
// weights as qsmg::bilinear.
__device__ __forceinline__ float bilinear_win(const float *cs, int cox, int coy, int cp, int m,
                                              int ix, int iy) {
    const int I = ix >> 1, J = iy >> 1;
    const int I2 = I + ((ix & 1) ? 1 : -1);
    const int J2 = J + ((iy & 1) ? 1 : -1);
    const bool xin = (I2 >= 0 && I2 < m), yin = (J2 >= 0 && J2 < m);
    const float *r0 = cs + (J - coy) * cp - cox;
    const float *r1 = cs + (J2 - coy) * cp - cox;
    const float v00 = r0[I];
    const float v10 = xin ? r0[I2] : -v00;
    const float v01 = yin ? r1[I] : -v00;
    float v11;
    if (xin && yin) v11 = r1[I2];
    else if (xin) v11 = -r0[I2];
    else if (yin) v11 = -r1[I];
    else v11 = v00;
    return (9.f * v00 + 3.f * v10 + 3.f * v01 + v11) * 0.0625f;
}

__device__ __forceinline__ void cp_async_t(float *dst, const float *src, bool valid) {
    cp_async_f32(dst, src, valid);
}
__device__ __forceinline__ void cp_async_t(double *dst, const double *src, bool valid) {
    cp_async_f64(dst, src, valid);
}

// Down leg of grid level F -> coarse C for every tile owned by this block:
// pre-smoothing from u_in (nullptr: a zero iterate), residual, 4-cell
// restriction (and kappa, inverse diagonal; the coarse level starts from
// zero where it is solved); the pre-smoothed tile is written to u_out.
// u_out must not be u_in: neighbours still stage u_in around their tiles
// during the leg.
template <typename T, int NC>
__device__ void down_level(const Lvl<T> F, const Lvl<T> C, int nu1, int TX, int TY, T *sm,
                           int bid, int nblk, T *const *u_out, const T *const *u_in = nullptr,
                           qsmg::Marks mark = qsmg::Marks{nullptr, nullptr, 0}) {
    const int n = F.n, m = C.n;
    const int H = 2 * nu1 + 1;
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const T h2 = F.h2t, inv_h2 = F.inv_h2t, ch2 = C.h2t;
    const bool scr = F.k != nullptr;
    const T *const gf0 = F.f[0];
    const T *const gf1 = F.f[NC - 1];
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        constexpr int V = 16 / (int)sizeof(T);
        const Region g = make_region(tx0, ty0, TX, TY, H, n, V);
        const TileSmem<T> t = tile_layout(sm, g.R);
        T *const su0 = t.su0;
        T *const su1 = t.su1;
        T *const sf0 = t.sf0;
        T *const sf1 = t.sf1;
        T *const sk = scr ? t.sk : nullptr;
        T *const sd = scr ? t.sd : nullptr;
        if (n % V == 0) {  // whole rows in 16-byte copies
            for_groups<T>(g, n, [&](int li, int gi, bool in) {
                if (u_in) {
                    cp_async16(su0 + li, u_in[0] + gi, in);
                    if (NC > 1) cp_async16(su1 + li, u_in[1] + gi, in);
                } else {
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        su0[li + k] = T(0);
                        if (NC > 1) su1[li + k] = T(0);
                    }
                }
                cp_async16(sf0 + li, gf0 + gi, in);
                if (NC > 1) cp_async16(sf1 + li, gf1 + gi, in);
                if (scr) {
                    cp_async16(sk + li, F.k + gi, in);
                    cp_async16(sd + li, F.d + gi, in);
                }
            });
        } else for (Walk w(threadIdx.x, blockDim.x, g.RX); w.q < g.R; w.next()) {
            const int x = g.ox + w.col, y = g.oy + w.row;
            const bool in = x >= 0 && x < n && y >= 0 && y < n;
            const int gi = in ? y * n + x : 0, li = w.q;
            if (u_in) cp_async_t(su0 + li, u_in[0] + gi, in);
            else su0[li] = T(0);
            cp_async_t(sf0 + li, gf0 + gi, in);
            if (NC > 1) {
                if (u_in) cp_async_t(su1 + li, u_in[1] + gi, in);
                else su1[li] = T(0);
                cp_async_t(sf1 + li, gf1 + gi, in);
            }
            if (scr) {
                cp_async_t(sk + li, F.k + gi, in);
                cp_async_t(sd + li, F.d + gi, in);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        mark(60);
        staged_sweeps<NC, T>(g, n, h2, su0, su1, sf0, sf1, sd, 2 * nu1, F.omega);
        mark(61);
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
                const T *su = c ? su1 : su0;
                const T *sf = c ? sf1 : sf0;
                T s = sf[l0] - staged_op<T>(su, sk, RX, n, inv_h2, l0, x0, y0);
                s += sf[l0 + 1] - staged_op<T>(su, sk, RX, n, inv_h2, l0 + 1, x0 + 1, y0);
                s += sf[l0 + RX] - staged_op<T>(su, sk, RX, n, inv_h2, l0 + RX, x0, y0 + 1);
                s += sf[l0 + RX + 1] - staged_op<T>(su, sk, RX, n, inv_h2, l0 + RX + 1, x0 + 1, y0 + 1);
                C.f[c][J * m + I] = T(0.25) * s;
            }
            if (scr) {
                const T kk = T(0.25) * (sk[l0] + sk[l0 + 1] + sk[l0 + RX] + sk[l0 + RX + 1]);
                C.k[J * m + I] = kk;
                C.d[J * m + I] = T(1) / ((T)(4 + qsmg::walls(I, J, m)) + ch2 * kk);
            }
        }
        for (Walk w(threadIdx.x, blockDim.x, TX); w.q < TX * TY; w.next()) {
            const int x = tx0 + w.col, y = ty0 + w.row;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
            u_out[0][y * n + x] = su0[li];
            if (NC > 1) u_out[1][y * n + x] = su1[li];
        }
        __syncthreads();
    }
}

// Up leg of grid level F for every tile owned by this block (the float64
// form's cycle): the pre-smoothed iterate s_in (the down leg's u_out) plus
// the bilinear prolongation of the coarse correction C.u, post-sweeps, the
// tile written to F.u.  With `norm` (level 0) the halo is one cell wider
// and the thread's sums of |f - A u|^2 and u^2 per component go to
// norms[0 .. 3].
template <typename T, int NC>
__device__ void up_level(const Lvl<T> F, const Lvl<T> C, const T *const *s_in, int nu2, int TX,
                         int TY, T *sm, int bid, int nblk, bool norm, double norms[4]) {
    const int n = F.n, m = C.n;
    const int H = 2 * nu2 + (norm ? 1 : 0);
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const bool scr = F.k != nullptr;
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        constexpr int V = 16 / (int)sizeof(T);
        const Region g = make_region(tx0, ty0, TX, TY, H, n, V);
        const TileSmem<T> t = tile_layout(sm, g.R);
        T *const sk = scr ? t.sk : nullptr;
        T *const sd = scr ? t.sd : nullptr;
        if (n % V == 0) {  // whole rows in 16-byte copies
            for_groups<T>(g, n, [&](int li, int gi, bool in) {
                cp_async16(t.su0 + li, s_in[0] + gi, in);
                cp_async16(t.sf0 + li, F.f[0] + gi, in);
                if (NC > 1) {
                    cp_async16(t.su1 + li, s_in[1] + gi, in);
                    cp_async16(t.sf1 + li, F.f[1] + gi, in);
                }
                if (scr) {
                    cp_async16(sk + li, F.k + gi, in);
                    cp_async16(sd + li, F.d + gi, in);
                }
            });
        } else for (Walk w(threadIdx.x, blockDim.x, g.RX); w.q < g.R; w.next()) {
            const int x = g.ox + w.col, y = g.oy + w.row;
            const bool in = x >= 0 && x < n && y >= 0 && y < n;
            const int gi = in ? y * n + x : 0, li = w.q;
            cp_async_t(t.su0 + li, s_in[0] + gi, in);
            cp_async_t(t.sf0 + li, F.f[0] + gi, in);
            if (NC > 1) {
                cp_async_t(t.su1 + li, s_in[1] + gi, in);
                cp_async_t(t.sf1 + li, F.f[1] + gi, in);
            }
            if (scr) {
                cp_async_t(sk + li, F.k + gi, in);
                cp_async_t(sd + li, F.d + gi, in);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (Walk w(threadIdx.x, blockDim.x, g.RX); w.q < g.R; w.next()) {
            const int x = g.ox + w.col, y = g.oy + w.row;
            if (x < 0 || x >= n || y < 0 || y >= n) continue;
            t.su0[w.q] += qsmg::bilinear(C.u[0], m, x, y);
            if (NC > 1) t.su1[w.q] += qsmg::bilinear(C.u[1], m, x, y);
        }
        __syncthreads();
        staged_sweeps<NC, T>(g, n, F.h2t, t.su0, t.su1, t.sf0, t.sf1, sd, 2 * nu2, F.omega);
        for (Walk w(threadIdx.x, blockDim.x, TX); w.q < TX * TY; w.next()) {
            const int x = tx0 + w.col, y = ty0 + w.row;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * g.RX + (x - g.ox);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T *su = c ? t.su1 : t.su0;
                F.u[c][y * n + x] = su[li];
                if (norm) {
                    const T r = (c ? t.sf1 : t.sf0)[li] -
                                staged_op<T>(su, sk, g.RX, n, F.inv_h2t, li, x, y);
                    norms[c] += (double)r * (double)r;
                    norms[2 + c] += (double)su[li] * (double)su[li];
                }
            }
        }
        __syncthreads();
    }
}

// The level-0 update of the refined form, fused into the last up phase.  The
// level-0 region's halo is one cell wider than the sweeps need, so the final
// float32 correction e is known on the tile and on the ring around it.
// Then, on the tile only, in float64:
//   u += e;   r -= (lap_h - kappa) e;   r32 = (float) r
// (the residual update r_new = f - A(u + e) = r - A e), and this thread's
// sums of r^2 and u^2 per component are added to norms[0..3].  No cell of u
// or r is read outside the block's own tile, so no other block's writes
// interfere.  The float64 tile values are staged with the region.
struct Fused {
    double *u64[2];
    double *r64[2];
    float *r32[2];
    float *u32[2];      // float32 copy of u64 (nullptr: none)
    const double *kap;  // float64 kappa (screened) or nullptr
    double inv_h2;
};

// ---------------------------------------------------------------------------
// Up cascade: the up legs of every staged level and the fused level-0 update
// in one grid phase.
//
// The separate up legs cost a grid barrier and a global round trip per
// level.  Here each block starts from the coarse correction of the first
// block-local level (held, complete, in its shared memory after the
// redundant coarse part) and walks up to level 0 for its own level-0 tile.
// At level l it needs the corrected values only on the window of level-l
// cells that the finer region prolongs from; it stages that window plus a
// halo of 2 nu2 (pre-smoothed u, f, inverse diagonal), adds the prolongated
// correction, sweeps, and keeps the window, which is exact.  The level-0
// region is the tile plus a halo 2 nu2 + 1 (see Fused above).
// ---------------------------------------------------------------------------

// hi + lo += v with hi + lo kept exact up to the rounding of lo (TwoSum of
// hi and v; the round-to-nearest intrinsics keep the compiler from fusing
// or reassociating the steps).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// coarse window of an in-domain box [ax, bx] x [ay, by] at a level of side m
__device__ __forceinline__ void coarse_window(const Region &g, int m, int &wx0, int &wy0,
                                              int &wx1, int &wy1) {
    wx0 = max((g.ax >> 1) - 1, 0);
    wy0 = max((g.ay >> 1) - 1, 0);
    wx1 = min((g.bx >> 1) + 1, m - 1);
    wy1 = min((g.by >> 1) + 1, m - 1);
}

// region of cascade level l for the level-0 tile at (tx0, ty0)
__device__ __forceinline__ Region cascade_region(const qsmg::Hier<float> &Hh, int l, int tx0,
                                                 int ty0, int TX, int TY, int nu2) {
    Region g = make_region(tx0, ty0, TX, TY, 2 * nu2 + 1, Hh.lv[0].n, 4);
    for (int k = 1; k <= l; ++k) {
        int wx0, wy0, wx1, wy1;
        coarse_window(g, Hh.lv[k].n, wx0, wy0, wx1, wy1);
        g = make_region(wx0, wy0, wx1 - wx0 + 1, wy1 - wy0 + 1, 2 * nu2, Hh.lv[k].n, 4);
    }
    return g;
}

// stage u, f (and the inverse diagonal) of level F on region g and add the
// prolongation of the coarse correction held as a window (origin sox, soy,
// pitch sp) of a level of side m; ends with a block barrier
template <int NC>
__device__ void stage_cascade(const Lvl<float> F, const Region &g, const CascadeSmem &t,
                              const float *src0, const float *src1, int sox, int soy, int sp,
                              int m) {
    const int n = F.n;
    const bool scr = F.d != nullptr;
    if (n % 4 == 0) {  // whole rows in 16-byte copies
        for_groups<float>(g, n, [&](int li, int gi, bool in) {
            if (scr) cp_async16(t.sd + li, F.d + gi, in);
            cp_async16(t.su0 + li, F.u[0] + gi, in);
            cp_async16(t.sf0 + li, F.f[0] + gi, in);
            if (NC > 1) {
                cp_async16(t.su1 + li, F.u[1] + gi, in);
                cp_async16(t.sf1 + li, F.f[1] + gi, in);
            }
        });
    } else for (Walk w(threadIdx.x, blockDim.x, g.RX); w.q < g.R; w.next()) {
        const int x = g.ox + w.col, y = g.oy + w.row;
        const bool in = x >= 0 && x < n && y >= 0 && y < n;
        const int gi = in ? y * n + x : 0, li = w.q;
        if (scr) cp_async_f32(t.sd + li, F.d + gi, in);
        cp_async_f32(t.su0 + li, F.u[0] + gi, in);
        cp_async_f32(t.sf0 + li, F.f[0] + gi, in);
        if (NC > 1) {
            cp_async_f32(t.su1 + li, F.u[1] + gi, in);
            cp_async_f32(t.sf1 + li, F.f[1] + gi, in);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int wx = g.bx - g.ax + 1, wy = g.by - g.ay + 1;
    for (Walk w(threadIdx.x, blockDim.x, wx); w.q < wx * wy; w.next()) {
        const int x = g.ax + w.col, y = g.ay + w.row;
        const int li = (y - g.oy) * g.RX + (x - g.ox);
        t.su0[li] += bilinear_win(src0, sox, soy, sp, m, x, y);
        if (NC > 1) t.su1[li] += bilinear_win(src1, sox, soy, sp, m, x, y);
    }
    __syncthreads();
}

// cs0, cs1: the correction of level lg (side H.lv[lg].n), complete, in this
// block's shared memory.
template <int NC>
__device__ void up_cascade_fused(const qsmg::Hier<float> &Hh, int lg, const float *cs0,
                                 const float *cs1, int nu2, int TX, int TY, float *sm, int bid,
                                 int nblk, const Fused &o, float norms[4],
                                 qsmg::Marks mark = qsmg::Marks{nullptr, nullptr, 0}) {
    const int n = Hh.lv[0].n;
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    double *const u64_0 = o.u64[0], *const u64_1 = o.u64[NC - 1];
    double *const r64_0 = o.r64[0], *const r64_1 = o.r64[NC - 1];
    float *const r32_0 = o.r32[0], *const r32_1 = o.r32[NC - 1];
    float *const u32_0 = o.u32[0], *const u32_1 = o.u32[NC - 1];
    const double *const kap = o.kap;
    const double inv_h2 = o.inv_h2;
    for (int tile = bid; tile < ntx * nty; tile += nblk) {
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY;
        const float *src0 = cs0, *src1 = cs1;
        int sox = 0, soy = 0, sp = Hh.lv[lg].n, cur = 0;
        for (int l = lg - 1; l >= 1; --l) {
            const Lvl<float> F = Hh.lv[l];
            const Region g = cascade_region(Hh, l, tx0, ty0, TX, TY, nu2);
            const CascadeSmem t = cascade_layout(sm, g.R, TX, TY, nu2);
            stage_cascade<NC>(F, g, t, src0, src1, sox, soy, sp, Hh.lv[l + 1].n);
            staged_sweeps<NC, float>(g, F.n, F.h2t, t.su0, t.su1, t.sf0, t.sf1,
                              F.d ? t.sd : nullptr, 2 * nu2, F.omega);
            // keep the window that the next finer region prolongs from
            const Region gf = cascade_region(Hh, l - 1, tx0, ty0, TX, TY, nu2);
            int wx0, wy0, wx1, wy1;
            coarse_window(gf, F.n, wx0, wy0, wx1, wy1);
            const int wpx = wx1 - wx0 + 1, wpy = wy1 - wy0 + 1;
            float *const w0 = t.win + (2 * cur) * t.wbig;
            float *const w1 = w0 + t.wbig;
            for (Walk w(threadIdx.x, blockDim.x, wpx); w.q < wpx * wpy; w.next()) {
                const int li = (wy0 + w.row - g.oy) * g.RX + (wx0 + w.col - g.ox);
                w0[w.q] = t.su0[li];
                if (NC > 1) w1[w.q] = t.su1[li];
            }
            __syncthreads();
            src0 = w0;
            src1 = w1;
            sox = wx0;
            soy = wy0;
            sp = wpx;
            cur ^= 1;
        }
        // level 0
        const Lvl<float> F = Hh.lv[0];
        const Region g = cascade_region(Hh, 0, tx0, ty0, TX, TY, nu2);
        const CascadeSmem t = cascade_layout(sm, g.R, TX, TY, nu2);
        for (Walk w(threadIdx.x, blockDim.x, TX); w.q < TX * TY; w.next()) {
            const int x = tx0 + w.col, y = ty0 + w.row;
            const bool in = x < n && y < n;
            const int gi = in ? y * n + x : 0;
            cp_async_f64(t.du0 + w.q, u64_0 + gi, in);
            cp_async_f64(t.dr0 + w.q, r64_0 + gi, in);
            if (NC > 1) {
                cp_async_f64(t.du1 + w.q, u64_1 + gi, in);
                cp_async_f64(t.dr1 + w.q, r64_1 + gi, in);
            }
            if (kap) cp_async_f64(t.dk + w.q, kap + gi, in);
        }
        stage_cascade<NC>(F, g, t, src0, src1, sox, soy, sp, Hh.lv[1].n);
        mark(65);
        staged_sweeps<NC, float>(g, n, F.h2t, t.su0, t.su1, t.sf0, t.sf1, F.d ? t.sd : nullptr,
                          2 * nu2, F.omega);
        mark(66);
        const int RX = g.RX;
        float nrm32[4] = {0.f, 0.f, 0.f, 0.f};
        for (Walk w(threadIdx.x, blockDim.x, TX); w.q < TX * TY; w.next()) {
            const int x = tx0 + w.col, y = ty0 + w.row;
            if (x >= n || y >= n) continue;
            const int li = (y - g.oy) * RX + (x - g.ox);
            const int gi = y * n + x;
            const float cw = (float)(4 + qsmg::walls(x, y, n));
            const double kk = kap ? t.dk[w.q] : 0.0;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float *e = c ? t.su1 : t.su0;
                const float ef = e[li];
                // the 5-point sum of the float32 e, exact as an unevaluated
                // float32 pair (hi, lo) by error-free sums (Knuth's TwoSum)
                // and product (FMA): only the pair is widened to float64
                float hi = 0.f, lo = 0.f;
                if (x > 0) two_sum_acc(hi, lo, e[li - 1]);
                if (x < n - 1) two_sum_acc(hi, lo, e[li + 1]);
                if (y > 0) two_sum_acc(hi, lo, e[li - RX]);
                if (y < n - 1) two_sum_acc(hi, lo, e[li + RX]);
                const float pc = __fmul_rn(cw, ef);
                const float pe = __fmaf_rn(cw, ef, -pc);  // cw ef = pc + pe exactly
                two_sum_acc(hi, lo, -pc);
                lo = __fsub_rn(lo, pe);
                const double ec = (double)ef;
                const double ae = ((double)hi + (double)lo) * inv_h2 - kk * ec;
                const double u = (c ? t.du1 : t.du0)[w.q] + ec;
                const double r = (c ? t.dr1 : t.dr0)[w.q] - ae;
                const float rf = (float)r, uf = (float)u;
                (c ? u64_1 : u64_0)[gi] = u;
                (c ? r64_1 : r64_0)[gi] = r;
                (c ? r32_1 : r32_0)[gi] = rf;
                if (u32_0) (c ? u32_1 : u32_0)[gi] = uf;
                // the convergence test needs the norms to a few digits only
                nrm32[c] = __fmaf_rn(rf, rf, nrm32[c]);
                nrm32[2 + c] = __fmaf_rn(uf, uf, nrm32[2 + c]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) norms[k] += nrm32[k];
        __syncthreads();
    }
}

}  // namespace qstile
