// Internal declarations shared by the libqs translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qs.h"

#define QS_MAX_LEV 12
#define QS_DEFAULT_OMEGA_PCT 120
#define QS_ENGINE_THREADS 512

// ---------------------------------------------------------------------------
// device scalars of the slice engine (one instance per context, in global
// memory; reset before every launch)
// ---------------------------------------------------------------------------
struct DevScalars {
    unsigned long long bar_arrive; // grid barrier: total arrivals (monotonic)
    int err;                       // first error status seen on the device
    int err_where;                 // phase id of a timeout; -1: no clusters
    double rnorm[4][4];            // ||r||^2 (comps 0,1) and ||u||^2 (2,3), ring of 4
    double fnorm[3][2];            // ||f||^2 of the psi / (Ez,Bz) / (Bx,By) solves
    unsigned long long vmax_bits[2];  // V_max of a push (bits of a double >= 0)
    unsigned long long guard_hits;
    long long vcycles[3];
    long long slices;
    long long pushes;
    long long sorts;  // cell sorts of the plasma inside the slice loop
    int max_m;
    int not_converged;
    int cl_cycles;  // V-cycles of the last cluster solve (the largest over its clusters)
    double max_relres;
    unsigned long long vmax_all_bits;
    unsigned long long trace_n;
};

// Device state of a batched launch: the instance queue, one barrier counter
// and current instance per team, and a batch-wide error word.
#define QS_MAX_TEAMS 1024
struct BatchState {
    int next;                       // next instance to hand out
    int team_inst[QS_MAX_TEAMS];    // instance each team is working on
    unsigned long long team_bar[QS_MAX_TEAMS];
    DevScalars sc;                  // error word of the team barriers
};

// one grid level of a multigrid hierarchy (float64 levels, and the float32
// levels of the refined form's inner cycles)
struct LevelArrays {
    double *u[2];
    double *f[2];
    double *kap;
    double *d;
    double *s[2];  // the staged down leg's pre-smoothed iterate (float64 form)
};
struct LevelArrays32 {
    float *u[2];   // pre-smoothed iterate (tiled down leg) / block-level result
    float *f[2];
    float *k;
    float *d;
};

// Everything the slice engine reads or writes (passed by value).
struct EngineArgs {
    // geometry (Sec. 3 normalised units)
    int N;
    double h, inv_h, x_min, x_max, y_min, y_max;
    int n_xi;
    double dxi0, V0;
    int refine_k;
    double psi_floor;
    double mg_tol, mg_atol;
    int mg_max_vcycles;
    int nu1, nu2;
    int nu1c;      // pre-sweeps on the levels solved in shared memory
    double omega;  // over-relaxation factor of the red-black smoother
    int64_t np;
    long long spin_cycles;
    // plasma macroparticles (working copy; the refined form keeps positions
    // in float64 and momenta and weights in float32)
    double *x, *y, *px, *py, *w;
    float *px32, *py32, *w32;
    // deposited grids
    double *n_a, *n_b, *n_ion;
    double *jx, *jy, *txx, *txy, *tyy, *G;
    float *jx32, *jy32, *txx32, *txy32, *tyy32, *G32;  // refined form (G32: n_* <gamma - 1>)
    // level-0 fields (multigrid unknowns) and right-hand sides
    double *psi, *ez, *bz, *bx, *by;
    double *f_psi, *f_ez, *f_bz, *f_bx, *f_by;
    double *dpx, *dpy, *jz, *kap, *invd0;
    // warm start: solutions one and two slices back (psi, Ez, Bz, Bx, By)
    double *hist1[5], *hist2[5];
    int ws_order;
    // coarse levels 1..nlev-1 (scratch shared by the three solves)
    int nlev;
    int lev_n[QS_MAX_LEV];
    double lev_h2[QS_MAX_LEV];
    // the same spacing as constants of each storage type, computed on the
    // host: GB300's float64 pipe runs at 1/64 of float32, so a divide or a
    // conversion that every thread repeats costs microseconds per phase
    double lev_inv_h2[QS_MAX_LEV];
    float lev_h2f[QS_MAX_LEV], lev_inv_h2f[QS_MAX_LEV];
    LevelArrays lev[QS_MAX_LEV];
    int block_level_n;  // levels with side <= this are relaxed by one block
    // multigrid cycles in thread-block clusters (qs_cluster.cuh; the float64
    // solves of small grids, the refined form's float32 inner cycles):
    // cluster size of the launch (<= 1: off) and the byte offset of the
    // cluster's arrays in dynamic shared memory
    int cl_size;
    int cl_smem_offset;
    // privatised deposits: each block deposits a contiguous chunk of the
    // particle array into a band of grid rows held in shared memory at byte
    // offset band_off, at most band_rows rows for the six moments and
    // band_rows_n for n_* (0: plain global atomics, particles grid-strided)
    int band_rows, band_rows_n, band_off;
    // refined form: float32 inner hierarchy (level 0: correction e, residual r)
    int precision;
    int tile_x, tile_y;  // output tile of the staged grid levels (refined form)
    int block_smem_offset; // byte offset of the coarse part in shared memory
    int tile_smem_offset;  // byte offset of the staged tile after the coarse part
    float *e32[2], *r32[2][2], *k32, *d32;  // r32[buffer][component]
    // refined form: float32 copies of the push's fields (grad psi, B), so
    // that its gathers need no float64 conversions
    float *dpx32, *dpy32, *bx32, *by32, *bz32;
    double *r64[2];  // float64 residual of the refined iteration
    LevelArrays32 lev32[QS_MAX_LEV];
    // cell sort of the plasma inside the slice loop: every sort_every base
    // slices (0: never) the particle arrays are reordered by (cell, id) into
    // the spare arrays x2 ... id2 (counting sort; count, offset and cursor
    // have N^2 (+1) entries, cell and order np, bsum one per block)
    int sort_every;
    int32_t *id, *id2;
    double *x2, *y2, *wd2;
    void *px2, *py2, *w2;  // in the particle precision
    int32_t *s_count, *s_offset, *s_cursor, *s_cell, *s_order, *s_bsum;
    // laser driver (Eq. EoM_111 and the line after it, Eq. FluxCurr1_A):
    // |A|^2 of the envelope on the base slices [n_xi][N*N] (nullptr: no
    // laser); the value at the current slice (linear in xi between base
    // slices, like the driver current), grad(|A|^2 / 4) by central
    // differences with even ghosts (A is odd at the walls), and
    // chi = n_* / (1+psi) stored at the base slices [n_xi][N*N] for the
    // envelope advance of Eq. laser_Enve (nullptr: not stored)
    const double *a2_base;
    double *a2, *pondx, *pondy;
    double *chi;
    // outputs
    double *hist;        // [5][n_xi][N*N]
    const double *jzb;   // [n_xi][N*N]
    const int32_t *m_sched;  // optional [n_xi]
    int32_t *diag_m;
    double *diag_vmax, *diag_charge;
    DevScalars *sc;
    // optional phase trace: block 0 records (phase id, %globaltimer) after
    // every grid barrier, up to trace_cap entries
    int64_t *trace;
    int trace_cap;
    // base slices [j_begin, j_end) of this launch (the whole window, or one
    // segment recomputed for the adjoint from a stored plasma state)
    int j_begin, j_end;
    // checkpoints: the plasma state (x, y, px, py; momenta in the particle
    // precision, widened to float64) before base slice j = k * ckpt_every is
    // stored at ckpt + k * 4 * np (nullptr: none)
    int ckpt_every;
    double *ckpt;
    // segment store for the adjoint (nullptr: none): for the s-th computed
    // slice of the launch, the plasma state before its push at
    // seg_p + s * 4 * np (x, y, px, py) and 12 grids at seg_g + s * 12 * N^2
    // (psi, Ez, Bz, Bx, By, n_*, jx, jy, Txx, Txy, Tyy, n_* <gamma>)
    double *seg_p, *seg_g;
    int seg_cap;  // slots of the segment store; slices beyond it are not stored
};

// Arguments of the adjoint engine (the reverse slice loop over one segment).
// Cotangents are written g_<name> = dL/d<name>; all float64.
struct AdjArgs {
    // the segment: base slices [j0, j1), n_sub stored slices (sub-steps
    // included) in forward order in the segment store of EngineArgs
    int j0, j1, n_sub;
    // cotangents of the plasma state (x, y, px, py) of the current slice and
    // of the lattice weights (accumulated over the whole window)
    double *lx, *ly, *lpx, *lpy, *lw;
    // grid cotangents
    double *g_psi, *g_ez, *g_bz, *g_bx, *g_by, *g_dpx, *g_dpy;
    double *g_jx, *g_jy, *g_txx, *g_txy, *g_tyy, *g_G, *g_n;
    // adjoint solutions (transposed solves; also the warm start of the next
    // reverse slice) and the right-hand side of the psi adjoint
    double *mu_x, *mu_y, *nu_ez, *nu_bz, *nu_psi, *f_nu_psi;
    // inputs / outputs
    const double *d_hist;  // [5][n_xi][N*N] dL/d(stored fields) or nullptr
    double *d_jzb;         // [n_xi][N*N] dL/d(j_z of the bunches), accumulated
    double *d_nion;        // [N*N] dL/d(n_ion), accumulated
};

// grids of one stored slice in the segment store
enum SegGrid { SG_PSI = 0, SG_EZ, SG_BZ, SG_BX, SG_BY, SG_N, SG_JX, SG_JY, SG_TXX, SG_TXY,
               SG_TYY, SG_G, SG_COUNT };

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

// Two-cell linear (CIC) weights along one axis for s = (x - x_min) / h; cell
// centres at s = i + 1/2.  Index -1 folds to 0, index n to n-1 (the ghost
// weight goes to the mirror interior cell).  Indices are clamped to [0, n-1]
// for memory safety.
__device__ __forceinline__ void cic_axis(double s, int n, int &i0, int &i1, double &w0,
                                         double &w1) {
    double t = s - 0.5;
    double fl = floor(t);
    double f = t - fl;
    int a = (int)fl;
    int b = a + 1;
    if (a < 0) a = -1 - a;
    if (b > n - 1) b = 2 * n - 1 - b;
    a = min(max(a, 0), n - 1);
    b = min(max(b, 0), n - 1);
    i0 = a;
    i1 = b;
    w0 = 1.0 - f;
    w1 = f;
}

struct Cic {
    int i00, i01, i10, i11;  // flat indices (iy0,ix0) (iy0,ix1) (iy1,ix0) (iy1,ix1)
    double w00, w01, w10, w11;
};

__device__ __forceinline__ Cic cic_stencil(double x, double y, double x_min, double y_min,
                                           double h, int n) {
    int ix0, ix1, iy0, iy1;
    double wx0, wx1, wy0, wy1;
    cic_axis((x - x_min) / h, n, ix0, ix1, wx0, wx1);
    cic_axis((y - y_min) / h, n, iy0, iy1, wy0, wy1);
    Cic c;
    c.i00 = iy0 * n + ix0;
    c.i01 = iy0 * n + ix1;
    c.i10 = iy1 * n + ix0;
    c.i11 = iy1 * n + ix1;
    c.w00 = wy0 * wx0;
    c.w01 = wy0 * wx1;
    c.w10 = wy1 * wx0;
    c.w11 = wy1 * wx1;
    return c;
}

// The same stencil from the reciprocal cell size (no float64 divide: the
// slice loop evaluates it several times per particle and slice).
__device__ __forceinline__ Cic cic_stencil_inv(double x, double y, double x_min, double y_min,
                                               double inv_h, int n) {
    int ix0, ix1, iy0, iy1;
    double wx0, wx1, wy0, wy1;
    cic_axis((x - x_min) * inv_h, n, ix0, ix1, wx0, wx1);
    cic_axis((y - y_min) * inv_h, n, iy0, iy1, wy0, wy1);
    Cic c;
    c.i00 = iy0 * n + ix0;
    c.i01 = iy0 * n + ix1;
    c.i10 = iy1 * n + ix0;
    c.i11 = iy1 * n + ix1;
    c.w00 = wy0 * wx0;
    c.w01 = wy0 * wx1;
    c.w10 = wy1 * wx0;
    c.w11 = wy1 * wx1;
    return c;
}

__device__ __forceinline__ double cic_gather(const double *u, const Cic &c) {
    return u[c.i00] * c.w00 + u[c.i01] * c.w01 + u[c.i10] * c.w10 + u[c.i11] * c.w11;
}

__device__ __forceinline__ void cic_deposit(double *g, const Cic &c, double q) {
    atomicAdd(g + c.i00, q * c.w00);
    atomicAdd(g + c.i01, q * c.w01);
    atomicAdd(g + c.i10, q * c.w10);
    atomicAdd(g + c.i11, q * c.w11);
}

// Cell index c = iy * N + ix, ix = floor((x - x_min) / h) clamped to [0, N-1].
__device__ __forceinline__ int cell_of(double x, double y, double x_min, double y_min, double h,
                                       int n) {
    int ix = (int)floor((x - x_min) / h);
    int iy = (int)floor((y - y_min) / h);
    ix = min(max(ix, 0), n - 1);
    iy = min(max(iy, 0), n - 1);
    return iy * n + ix;
}

// ---------------------------------------------------------------------------
// host-side launchers implemented in qs_aux.cu
// ---------------------------------------------------------------------------
cudaError_t qs_launch_init_plasma(cudaStream_t st, int n, int ppc, double x_min, double y_min,
                                  double h, const double *table, int n_coef, double r_max,
                                  double *x, double *y, double *px, double *py, double *w,
                                  int32_t *id);
cudaError_t qs_launch_deposit(cudaStream_t st, const double *x, const double *y,
                              const double *q, int64_t np, int n, double x_min, double y_min,
                              double h, double scale, double *grid);
cudaError_t qs_launch_beam_deposit(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                   double x_max, double y_min, double y_max, double h,
                                   int n_xi, double xi_min, double dxi0, double *jzb);
cudaError_t qs_launch_beam_push(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                double x_max, double y_min, double y_max, double h, int n_xi,
                                double xi_min, double dxi0, const double *hist, double dt);
cudaError_t qs_launch_beam_push_dla(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                    double x_max, double y_min, double y_max, double h,
                                    int n_xi, double xi_min, double dxi0, const double *hist,
                                    const double *env_n, const double *env_np1, double k0,
                                    double dt, int n_sub);
cudaError_t qs_launch_convert(cudaStream_t st, const double *src, float *dst, int64_t n);
// |a|^2 of n interleaved complex128 values
cudaError_t qs_launch_abs2(cudaStream_t st, const double *a, double *out, int64_t n);
// implemented in qs_laser.cu
void qs_laser_shape(const qs_laser *s, int *n, double *width, int *n_xi, double *dxi);
// implemented in qs_grad_aux.cu
cudaError_t qs_launch_beam_gain(cudaStream_t st, const qs_beam &b, int n, double x_min,
                                double x_max, double y_min, double y_max, double h, int n_xi,
                                double xi_min, double dxi0, const double *hist, double dt,
                                double scale, double *gain_sum, double *d_hist);
cudaError_t qs_launch_beam_deposit_adjoint(cudaStream_t st, const qs_beam &b, int n,
                                           double x_min, double x_max, double y_min,
                                           double y_max, double h, int n_xi, double xi_min,
                                           double dxi0, const double *d_jzb, double *dx,
                                           double *dy, double *dxi, double *dw);
cudaError_t qs_launch_profile_adjoint(cudaStream_t st, int n, int ppc, double x_min,
                                      double y_min, double h, int n_coef, double r_max,
                                      const double *d_w, const double *d_nion,
                                      double *d_table);
cudaError_t qs_launch_widen(cudaStream_t st, const float *src, double *dst, int64_t n);
cudaError_t qs_launch_cell_sort(cudaStream_t st, const double *x, const double *y,
                                const int32_t *id, int64_t np, int n, double x_min,
                                double y_min, double h, int32_t *cell, int32_t *count,
                                int32_t *offset, int32_t *cursor, int32_t *perm);
// launch handles of the persistent kernels, one translation unit per form
const void *qs_kernel_engine_fp64();
const void *qs_kernel_engine_fp32r();
const void *qs_kernel_engine_batched_fp64();
const void *qs_kernel_engine_batched_fp32r();
const void *qs_kernel_adjoint_fp64();
const void *qs_kernel_adjoint_fp32r();
const void *qs_kernel_engine(int precision);
const void *qs_kernel_engine_batched(int precision);
const void *qs_kernel_adjoint(int precision);
cudaError_t qs_launch_engine(cudaStream_t st, const EngineArgs &a, int grid_blocks,
                             size_t smem_bytes);
cudaError_t qs_launch_engine_batched(cudaStream_t st, const EngineArgs *list, int n_inst,
                                     int precision, int team, int teams, BatchState *bs,
                                     size_t smem_bytes);
int qs_engine_batched_max_blocks(int device, int precision, size_t smem_bytes, int *blocks);
cudaError_t qs_launch_adjoint(cudaStream_t st, const EngineArgs &a, const AdjArgs &d,
                              int grid_blocks, size_t smem_bytes);
int qs_adjoint_max_blocks(int device, int precision, size_t smem_bytes, int *blocks);
int qs_engine_max_blocks(int device, int precision, size_t smem_bytes, int *blocks,
                         int cluster = 1);
size_t qs_cluster_smem_bytes(const int *lev_n, int nlev, int cluster, int tsize);
size_t qs_engine_smem_bytes(const int *lev_n, int nlev, int block_level_n, int precision,
                            int tile_x, int tile_y, int nu, int nu2, size_t *block_offset,
                            size_t *tile_offset);
