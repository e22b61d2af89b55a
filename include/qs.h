/*
 * qs.h -- C ABI of libqs, a single-GPU (GB300, sm_103a) implementation of the
 * quasi-static xi-slice advance of Wang, Khudik, Kim and Shvets, "WAND-PIC: an
 * accelerated three-dimensional quasi-static particle-in-cell code"
 * (arXiv 2012.00881).
 *
 * Units are the paper's normalised units (Sec. 3, first paragraph): time in
 * 1/omega_p, lengths in 1/k_p, momenta in mc, fields in m c omega_p / e,
 * densities in n0, current density in -e n0 c (electron flux).  xi = t - z
 * grows from the head of the window backwards (Sec. 2, item 1).
 *
 * Conventions shared by every entry point
 *   - Grids are cell-centred, nx = ny = N cells on a square box;
 *     h = (x_max - x_min) / N.  2D arrays are row-major [iy][ix], ix fastest.
 *   - Fields are zero on the box walls (odd ghost cells).  Particles reflect
 *     specularly at the walls.  CIC weight that falls into a ghost cell is
 *     folded back into the mirror interior cell (deposits conserve charge);
 *     gathers use the same weights.
 *   - Every function returns QS_OK (0) or a negative QS_ERR_* status; nothing
 *     aborts, traps or throws across the ABI.  qs_strerror() names a status;
 *     qs_last_error() gives the context's last detailed message.
 *   - Device pointers are CUDA device addresses on the context's device.
 *     Caller-owned buffers stay owned by the caller; the library never frees
 *     them.  The library allocates its own state at qs_create /
 *     qs_init_plasma and frees it at qs_destroy.
 *   - All work is issued on the stream given to qs_create.  Calls that return
 *     results to the host (qs_step3d with stats, qs_fields to a host buffer,
 *     qs_slice_diagnostics, qs_get_plasma) synchronise that stream.
 */
#ifndef QS_H
#define QS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QS_OK 0
#define QS_ERR_ARG (-1)            /* invalid argument or configuration      */
#define QS_ERR_CUDA (-2)           /* a CUDA runtime call failed             */
#define QS_ERR_OOM (-3)            /* device allocation failed               */
#define QS_ERR_NOT_CONVERGED (-4)  /* a multigrid solve hit mg_max_vcycles;   */
                                   /* fields hold the last iterate            */
#define QS_ERR_PSI_FLOOR (-5)      /* 1+psi fell below psi_floor more often   */
                                   /* than max_psi_guard_hits allows          */
#define QS_ERR_STATE (-6)          /* calls out of order (e.g. no plasma)     */
#define QS_ERR_TIMEOUT (-7)        /* a device-side wait exceeded its limit;  */
                                   /* the kernel returned early               */

/* ---- arithmetic forms -------------------------------------------------- */
#define QS_FP64 0          /* every step in float64                          */
#define QS_FP32_REFINED 1  /* float32 particles, smoothing and grid transfers; */
                           /* float64 residuals, defect correction, coarsest */
                           /* solve and gamma reconstruction                  */

/* ---- field selection for qs_fields (order of the output blocks) -------- */
#define QS_FIELD_PSI 1  /* wake potential psi = phi - A_z (Eq. EqM_N8_AA)  */
#define QS_FIELD_EZ 2   /* E_z (Eq. EqM_N8_A)                              */
#define QS_FIELD_BZ 4   /* B_z (Eq. Mag_z_A)                               */
#define QS_FIELD_BX 8   /* B_x (Eq. Main_Eq_A)                             */
#define QS_FIELD_BY 16  /* B_y (Eq. Main_Eq_A)                             */
#define QS_FIELD_JZB 32 /* driver-beam j_z deposited on the base slices     */
#define QS_FIELD_ALL 31

typedef struct qs_ctx qs_ctx; /* opaque, library-owned */

/* Problem description (Sec. 3 normalised units).  Fill with
 * qs_config_default() and override. */
typedef struct {
    int nx, ny;                 /* transverse cells; nx == ny == N required;   */
                                /* N = c * 2^L with coarsest side c <= 8       */
    double x_min, x_max;        /* box edges; the box must be square           */
    double y_min, y_max;
    int n_xi;                   /* base xi slices                               */
    double xi_min, xi_max;      /* window; dxi0 = (xi_max - xi_min) / n_xi      */
    int refine_k;               /* smallest sub-step is dxi0 / refine_k         */
                                /* (refinement level k of Sec. 5.1), >= 1       */
    int precision;              /* QS_FP64 or QS_FP32_REFINED                   */
    double mg_tol;              /* stop when ||f - A u||_2 <= mg_tol ||f||_2    */
    int mg_max_vcycles;         /* per solve; exceeding it -> NOT_CONVERGED     */
    double psi_floor;           /* 1+psi is clamped to >= psi_floor             */
    int64_t max_psi_guard_hits; /* -1: unlimited                                */
    int sort_every;             /* > 0: every this many base slices the slice   */
                                /* loop reorders the plasma by (cell, id), the  */
                                /* order of qs_cell_sort (not in steps that     */
                                /* store checkpoints for the adjoint); 0 = the  */
                                /* lattice order throughout                     */
    int pre_sweeps, post_sweeps;/* red-black Gauss-Seidel sweeps per level      */
                                /* (0 .. 8, not both 0); pre_sweeps -1 = the    */
                                /* form's default (3 refined, 2 QS_FP64)        */
    int coarse_block_n;         /* multigrid levels of side <= this are relaxed  */
                                /* by one thread block in shared memory;         */
                                /* 0 = default (16 for QS_FP64, 32 for refined) */
    int trace_capacity;         /* > 0: record up to this many phase timestamps */
                                /* per step (see qs_phase_trace); 0 = off        */
    int warm_start_order;       /* initial guess of each solve: 0 = previous    */
                                /* slice's solution (Sec. 7.1); 1, 2 = that     */
                                /* history extrapolated in xi, linear/quadratic */
    int tile_x, tile_y;         /* output tile of the grid-wide multigrid      */
                                /* levels staged in shared memory (both forms); */
                                /* even, 0 = default 32 x 16 (QS_FP64 on grids  */
                                /* of 512^2 and more: 64 x 32)                  */
    int omega_pct;              /* red-black smoother over-relaxation, percent: */
                                /* u += omega (u_GS - u), omega = omega_pct/100 */
                                /* in [0.5, 1.95]; 0 = default (1.2)            */
    int coarse_pre_sweeps;      /* pre-sweeps on the levels solved in shared    */
                                /* memory (side <= coarse_block_n); 0 = same    */
                                /* as pre_sweeps                                */
    int checkpoint_every;       /* > 0: qs_step3d also stores the plasma state  */
                                /* every this many base slices, which           */
                                /* qs_step3d_adjoint then uses instead of a     */
                                /* replay; >= n_xi: it keeps every slice's      */
                                /* state (up to 2 n_xi slices, if that fits in  */
                                /* 40 % of free device memory), so the adjoint  */
                                /* recomputes nothing; 0 = off                  */
    int64_t barrier_wait_cycles;/* limit of every grid-barrier wait of the slice */
                                /* loop, in SM clock cycles; a wait that runs   */
                                /* out records QS_ERR_TIMEOUT and the kernel    */
                                /* returns; 0 = default 4e9 (about 2 s)         */
    int cluster_size;           /* multigrid cycles in thread-block clusters of */
                                /* this many blocks (8 or 16; N must divide by  */
                                /* 2 * size), one cluster per component, the    */
                                /* rest of the slice loop on every block:       */
                                /* QS_FP64 solves of grids N <= 128, the float32 */
                                /* inner cycles of QS_FP32_REFINED up to 256;   */
                                /* 0 = automatic (float64: 16 for N <= 64      */
                                /* dividing by 32, 8 dividing by 16; refined:   */
                                /* off, its grid-wide cycles being faster), 1 = */
                                /* off                                           */
    int deposit_band_rows;      /* privatised deposits of the moments and n_*:  */
                                /* each block adds its contiguous chunk of the  */
                                /* (cell-sorted) plasma into a band of at most  */
                                /* this many grid rows in shared memory, then   */
                                /* the band to the grid once per cell; stencils */
                                /* outside the band go to the grid directly;    */
                                /* 0 = off (every stencil to the grid: faster  */
                                /* on the cases measured), -1 = as many rows   */
                                /* as shared memory holds (>= 8 where 200 KB   */
                                /* allow), else >= 3 rows at most              */
} qs_config;

/* Driver-beam macroparticles: structure of arrays of float64, n entries each.
 * For qs_step3d / qs_push_beam the arrays are DEVICE pointers owned by the
 * caller.  x, y in 1/k_p; xi = t - z in 1/k_p; p in mc; w = number of beam
 * particles per macroparticle in units of n0 / k_p^3. */
typedef struct {
    double *x, *y, *xi, *px, *py, *pz, *w;
    int64_t n;
    double charge;   /* charge per particle in units of e (electron: -1)     */
    double q_over_m; /* charge/mass in units of e/m (electron: -1)           */
} qs_beam;

/* Counters of one qs_step3d call. */
typedef struct {
    int64_t slices;          /* computed slices including sub-steps          */
    int64_t substeps;        /* computed slices that are not base slices     */
    int64_t pushes;          /* plasma macroparticle pushes                  */
    int64_t vcycles[3];      /* V-cycles (or outer refinement iterations):   */
                             /* [0] psi, [1] (E_z, B_z), [2] (B_x, B_y)       */
    int64_t psi_guard_hits;  /* clamps of 1+psi (particles and grid points)  */
    int64_t sorts;           /* cell sorts performed                          */
    double max_relres;       /* largest final relative residual of any solve */
    double vmax;             /* largest V_max of any push                     */
    int32_t max_m;           /* largest sub-step count of any base interval   */
    int32_t status;          /* same as the return value                      */
    double gpu_ms;           /* device time of the slice loop (CUDA events)   */
} qs_step_stats;

/* Defaults: N = 64 on [-6,6]^2, 128 slices on [0,12], refine_k = 8,
 * QS_FP64, mg_tol = 1e-10, 60 V-cycles, psi_floor = 1e-3, unlimited guard
 * hits, sort_every = 16, V(2,2) red-black sweeps over-relaxed by 1.2 with
 * one pre-sweep on the shared-memory levels, warm_start_order = 2. */
void qs_config_default(qs_config *cfg);

/* Create a context on the current CUDA device; `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Allocates the grids, the
 * multigrid hierarchy and the base-slice history (6 * n_xi * N^2 float64).
 * Errors: QS_ERR_ARG (bad config), QS_ERR_OOM, QS_ERR_CUDA. */
int qs_create(const qs_config *cfg, void *cuda_stream, qs_ctx **out);

/* Free everything the context owns.  NULL is accepted. */
void qs_destroy(qs_ctx *ctx);

/* Plasma macroparticles at the head of the window (Sec. 3.1: cold plasma,
 * H = 1, P = 0 before the driver arrives).  A quiet-start lattice of
 * sqrt(ppc) x sqrt(ppc) particles per cell at offsets (k + 1/2)/sqrt(ppc) of
 * a cell, p_perp = 0, weight n(r0) h^2 / ppc and id = cell * ppc + k.  The
 * transverse density n(r) is interpolated piecewise-linearly from
 * `profile[0..n_coef-1]` at equispaced radii on [0, r_max] (held beyond
 * r_max); profile == NULL means n = 1.  `profile` is a HOST array.  The ion
 * background of Eq. EqM_N8_AA is the deposit of this lattice.
 * Errors: QS_ERR_ARG (ppc not a perfect square, n_coef < 1, r_max <= 0). */
int qs_init_plasma(qs_ctx *ctx, int ppc, const double *profile, int n_coef, double r_max);

/* One 3D step with the drivers frozen: the xi loop of Algorithm 1
 * (Collect_Source, Solve_Wakefield, Push_Trajectory, Step_Size_Refinement)
 * from the unperturbed lattice at xi_min over all n_xi base slices.
 * Per slice: n_* deposit; psi from lap psi = n_* - n_ion (Eq. EqM_N8_AA);
 * moments j_perp, T, n_*<gamma> (Eqs. Jr, FluxPres); E_z, B_z (Eqs.
 * EqM_N8_A, Mag_z_A); B_perp from lap B - n_* / (1+psi) B = -e_z x S with the
 * explicit source S of Eq. FluxCurr1_A (Eq. Main_Eq_A), no predictor-
 * corrector; Boris-like push of Eqs. EoM_112_A/EoM_111; then
 * m = min(refine_k, max(1, ceil(V_max / V0))) sub-steps of dxi0/m for the
 * next base interval, V0 = h / dxi0 (Algorithm 1, Step_Size_Refinement).
 * Multigrid solves warm-start from the previous slice (Sec. 7.1).  The
 * drivers enter through j_z only: CIC in x, y and linear in xi on the base
 * slices, -charge * w * v_z; sub-steps interpolate linearly in xi.  Fields of
 * the base slices are stored for qs_fields and qs_push_beam.
 * `beams` holds n_beams descriptors with DEVICE arrays (n_beams may be 0).
 * `stats` (may be NULL) receives the counters; the call then synchronises.
 * Errors: QS_ERR_STATE (no plasma), QS_ERR_ARG, QS_ERR_NOT_CONVERGED,
 * QS_ERR_PSI_FLOOR, QS_ERR_TIMEOUT, QS_ERR_CUDA. */
int qs_step3d(qs_ctx *ctx, const qs_beam *beams, int n_beams, qs_step_stats *stats);

/* As qs_step3d, with the sub-step count of every base interval fixed to
 * m_schedule[j] (HOST array of n_xi ints in [1, refine_k]) instead of the
 * adaptive rule; used to replay a schedule. */
int qs_step3d_schedule(qs_ctx *ctx, const qs_beam *beams, int n_beams,
                       const int32_t *m_schedule, qs_step_stats *stats);

/* As qs_step3d, with a laser driver in the slice advance (Sec. "Description
 * of different plasma wake drivers"): `a2` (DEVICE float64 [n_xi][ny][nx],
 * caller-owned, read only) is |A|^2 of the laser envelope at the base
 * slices; at sub-steps it is taken linearly in xi between base slices, like
 * the beam current.  It adds |A|^2 / 2 to the numerator of gamma (the line
 * after Eq. EoM_111), hence to n_*<gamma> and j_z; the ponderomotive force
 * -grad(|A|^2 / 4) / (1+psi) to the push (Eq. EoM_111); and
 * -n_* grad(|A|^2 / 4) / (1+psi)^2 to the source S of Eq. FluxCurr1_A.  The
 * gradient is the central difference with even ghosts (A is odd at the
 * walls, so |A|^2 is mirrored).  `chi` (DEVICE float64 [n_xi][ny][nx], may
 * be NULL) receives the susceptibility chi = n_* / (1+psi) of Eq.
 * laser_Enve at every base slice.  beams / n_beams as qs_step3d (n_beams may
 * be 0: a laser-only driver).  qs_step3d_adjoint is not available after this
 * step (QS_ERR_STATE).  Errors: as qs_step3d; QS_ERR_ARG if a2 is NULL. */
int qs_step3d_laser(qs_ctx *ctx, const qs_beam *beams, int n_beams, const double *a2,
                    double *chi, qs_step_stats *stats);

/* Batched form: one 3D step (as qs_step3d) of each of n independent
 * contexts, which may differ in size, window, drivers, tiles and sweeps, in a
 * single persistent launch.  The launch is split into teams of `team_blocks`
 * thread blocks (0 = as many blocks per team as leave every instance its own
 * team); each team takes the next context from a device-side queue (largest
 * first: cells plus particles, times slices) and runs its whole slice loop
 * behind the team's own barrier.  All contexts must use
 * one precision and one device; the launch is queued on the first context's
 * stream and the call synchronises it.  beams[i] / n_beams[i] give context
 * i's drivers (DEVICE arrays; both lists may be NULL for no drivers).
 * stats (may be NULL) receives n entries; gpu_ms is the whole launch.
 * Returns the first failing status of any context (QS_ERR_ARG for repeated
 * contexts or mixed precisions). */
int qs_step3d_batched(qs_ctx **ctxs, int n, const qs_beam *const *beams, const int *n_beams,
                      int team_blocks, qs_step_stats *stats);

/* Push_Driver of Algorithm 1: advance every beam macroparticle by one
 * relativistic Boris step of length dt (Eqs. EoM_beam_1/2) in the wake stored
 * by the last qs_step3d: E = e_z E_z + E_perp, B = e_z B_z + B_perp with
 * E_perp = -grad psi - e_z x B_perp (the sign that follows from psi = phi -
 * A_z; the paper prints "+").  Fields are gathered by CIC in x, y and
 * linearly in xi between base slices; outside the box or the window the
 * wake is zero.  xi advances by dt (1 - v_z).  Arrays are updated IN PLACE
 * (DEVICE pointers).  Errors: QS_ERR_STATE (no step yet), QS_ERR_ARG. */
int qs_push_beam(qs_ctx *ctx, qs_beam *beams, int n_beams, double dt);

/* Push_Driver with the laser's own high-frequency fields (Sec. "Description
 * of different plasma wake drivers", Eq. E_B_Fields; the sub-cycling of Sec.
 * "Modeling direct laser acceleration of electrons with WAND-PIC"): beam
 * particles are not ponderomotive, so besides the stored wake (as
 * qs_push_beam) they feel the fields rebuilt from the envelope A (vector
 * potential Re[A e^{-i k0 xi}], polarised along x):
 *   E_x = Re[-((d_t A + d_xi A) - i k0 A) e^{-i k0 xi}],  B_y = Re[(-d_xi A + i k0 A) e^{-i k0 xi}],
 *   E_z = Re[-d_x A e^{-i k0 xi}],                        B_z = Re[-d_y A e^{-i k0 xi}].
 * The step dt is split into n_sub (>= 1) relativistic Boris sub-steps
 * (Eqs. EoM_beam_1/2); at sub-step s the envelope is linear in time between
 * env_n (time t) and env_np1 (t + dt) at s / n_sub, d_t A = (env_np1 -
 * env_n) / dt.  A and its derivatives are gathered like the wake (CIC in x,
 * y, linear in xi, zero outside the box and the window); d_x A, d_y A are
 * central differences with odd ghosts, d_xi A the central difference between
 * base slices with A = 0 beyond the window; the carrier phase is taken at the
 * particle's own xi.  env_n, env_np1: DEVICE complex128 [n_xi][ny][nx]
 * (interleaved re, im), caller-owned, read only (they may be the same
 * array).  k0 = omega_0 / omega_p > 0.  Beam arrays are updated IN PLACE.
 * Errors: QS_ERR_STATE (no step yet), QS_ERR_ARG. */
int qs_push_beam_dla(qs_ctx *ctx, qs_beam *beams, int n_beams, double dt, const double *env_n,
                     const double *env_np1, double k0, int n_sub);

/* ---- differentiable form: the adjoint of one 3D step ----
 *
 * The paper has no adjoint; these entry points give reverse-mode derivatives
 * of the computation that qs_step3d performs (same schedule of sub-steps,
 * the 1+psi guard inactive), for losses of the stored wake.
 *
 * qs_step3d_adjoint: given d_hist = dL/d(history), DEVICE [5][n_xi][ny*nx]
 * in qs_fields' order (psi, E_z, B_z, B_x, B_y; NULL = zero), runs the slice
 * loop backwards over the last qs_step3d of this context and OVERWRITES the
 * DEVICE outputs
 *   d_jzb  [n_xi][ny*nx]  dL/d(j_z of the bunches on the base slices),
 *   d_w    [qs_plasma_count()]  dL/d(weight) of each lattice particle, in
 *                        the order of qs_init_plasma's lattice (id order),
 *   d_nion [ny*nx]        dL/d(n_ion), the ion background.
 * Per reverse slice: the reverse Boris push, the transposed B_perp, E_z/B_z
 * and psi multigrid solves (the 5-point operators are symmetric, so they are
 * the forward solves with the cotangents as sources), the reverse of the
 * source S of Eq. FluxCurr1_A, and the adjoint of each CIC deposit (a
 * gather) and gather (a deposit).  Memory: the plasma state is stored every
 * `checkpoint_every` base slices (0 = 32) by one forward replay (skipped when
 * the last qs_step3d already stored them: config.checkpoint_every > 0 and
 * equal to this argument, or this argument 0), and each
 * segment is recomputed from its checkpoint before its reverse pass, which
 * holds every slice of the segment (4 floats per particle and 12 grids per
 * slice, float64).  Library-owned scratch is allocated and freed inside
 * the call.  stats (may be NULL): slices of the reverse loop, V-cycles of the
 * transposed solves, gpu_ms of all passes.  Synchronises.
 * Errors: QS_ERR_STATE (no completed qs_step3d), QS_ERR_ARG (NULL output),
 * QS_ERR_OOM, QS_ERR_NOT_CONVERGED, QS_ERR_TIMEOUT, QS_ERR_CUDA. */
int qs_step3d_adjoint(qs_ctx *ctx, const double *d_hist, int checkpoint_every, double *d_jzb,
                      double *d_w, double *d_nion, qs_step_stats *stats);

/* Mean energy gain of a bunch over one qs_push_beam step of length dt in
 * the stored wake, L = mean_p (gamma_p after - gamma_p before), WITHOUT
 * moving the bunch; *gain (HOST) receives L.  If d_hist is not NULL, dL/d
 * (history) is ADDED to it (DEVICE [5][n_xi][ny*nx], as qs_step3d_adjoint
 * takes it): the reverse relativistic Boris step, then the trilinear gather
 * of E_z, B_z, B_x, B_y and grad psi backwards (a deposit).  Synchronises.
 * Errors: QS_ERR_STATE (no step), QS_ERR_ARG (empty bunch, NULL arrays). */
int qs_beam_gain(qs_ctx *ctx, const qs_beam *beam, double dt, double *gain, double *d_hist);

/* Reverse of the bunch j_z deposit of qs_step3d for one bunch: from d_jzb
 * (DEVICE [n_xi][ny*nx], as qs_step3d_adjoint returns it) the DEVICE
 * outputs d_x, d_y, d_xi, d_w (n entries each, OVERWRITTEN) are the
 * derivatives with respect to each macroparticle's position and weight
 * (momenta held fixed).  Macroparticles outside the box or the window get
 * zero.  Errors: QS_ERR_STATE (no step), QS_ERR_ARG. */
int qs_beam_deposit_adjoint(qs_ctx *ctx, const qs_beam *beam, const double *d_jzb, double *d_x,
                            double *d_y, double *d_xi, double *d_w);

/* Derivative with respect to the radial density table of qs_init_plasma
 * (`profile`, n_coef values on [0, r_max], HOST): the lattice weights are
 * n(r0) h^2 / ppc and n_ion is their deposit, so
 *   dL/dtable_k = sum_p (d_w[p] + gather(d_nion)(r0_p) / h^2) h^2/ppc
 *                 * dn(r0_p)/dtable_k.
 * d_w (qs_plasma_count() entries) and d_nion (ny*nx) are DEVICE arrays as
 * qs_step3d_adjoint returns them; d_table (HOST, n_coef) is OVERWRITTEN.
 * Synchronises.  Errors: QS_ERR_STATE (no plasma), QS_ERR_ARG. */
int qs_profile_adjoint(qs_ctx *ctx, const double *d_w, const double *d_nion, int n_coef,
                       double r_max, double *d_table);

/* A bi-Gaussian bunch from parameters theta = (A, sigma_x, sigma_y,
 * sigma_z, x_c, y_c, xi_c, tilt) (HOST, 8) acting on standard normals z
 * (DEVICE, [3][n]): xi = xi_c + sigma_z/sqrt2 z2, x = x_c + tilt (xi - xi_c)
 * + sigma_x/sqrt2 z0, y = y_c + sigma_y/sqrt2 z1, equal weights
 * A pi^(3/2) sigma_x sigma_y sigma_z / n (the density A exp(-r^2/sigma_r^2 -
 * xi^2/sigma_z^2) of Sec. 5.1), p = (0, 0, sqrt(gamma^2 - 1)).  Writes the
 * DEVICE arrays of `out` (x, y, xi, px, py, pz, w; n entries, caller-owned)
 * on `cuda_stream` without waiting.  Errors: QS_ERR_ARG. */
int qs_bigaussian_beam(const double *theta, const double *z, int64_t n, double gamma,
                       qs_beam *out, void *cuda_stream);

/* Chain rule of qs_bigaussian_beam: from the DEVICE derivatives d_x, d_y,
 * d_xi, d_w (n each) with respect to the macroparticles, dL/dtheta (HOST, 8)
 * is OVERWRITTEN.  Synchronises `cuda_stream`.  Errors: QS_ERR_ARG,
 * QS_ERR_CUDA. */
int qs_bigaussian_adjoint(const double *theta, const double *z, int64_t n, const double *d_x,
                          const double *d_y, const double *d_xi, const double *d_w,
                          double *d_theta, void *cuda_stream);

/* Copy base-slice fields [slice_begin, slice_end) into `out`, laid out
 * [field][slice][iy][ix] for the fields selected in `field_mask` in the
 * order psi, E_z, B_z, B_x, B_y, j_z(beam).  `out` is a device pointer if
 * out_on_device != 0, else a host pointer (the call then synchronises).
 * Errors: QS_ERR_ARG (empty mask, bad range), QS_ERR_STATE. */
int qs_fields(qs_ctx *ctx, int field_mask, int slice_begin, int slice_end, double *out,
              int out_on_device);

/* Per-base-slice diagnostics of the last step (HOST arrays of n_xi entries;
 * any may be NULL): m[j] sub-steps used from slice j, vmax[j] = V_max after
 * the last push of interval j, charge[j] = sum of n_* h^2 at slice j (equal
 * to the sum of plasma weights by Eq. continuity).  Synchronises. */
int qs_slice_diagnostics(qs_ctx *ctx, int32_t *m, double *vmax, double *charge);

/* Copy the current plasma macroparticles (after the last step, or the
 * initial lattice) to HOST arrays of qs_plasma_count() entries, in the
 * library's current storage order; any pointer may be NULL.  Synchronises. */
int qs_get_plasma(qs_ctx *ctx, double *x, double *y, double *px, double *py, double *w,
                  int32_t *id);
int64_t qs_plasma_count(const qs_ctx *ctx);

/* Phase trace of the last qs_step3d (config.trace_capacity > 0): for each
 * grid barrier of the slice engine, in order, the id of the phase that
 * ended there (`where`: 1 density deposit, 2 psi source, 3 moments,
 * 4 and 5 source assembly, 6 push, 10-17 and 20-21 multigrid phases, 30 and
 * 32 staged down and up legs, 40-67 sub-phase marks of block 0) and the
 * device clock in nanoseconds (`t_ns`, %globaltimer).  Entry 0 is the kernel
 * start.  HOST arrays of `cap` entries; returns the number of entries
 * written (>= 0) or a status < 0. */
int qs_phase_trace(qs_ctx *ctx, int32_t *where, int64_t *t_ns, int cap);

/* Stable counting sort of n particles by cell, c = iy * N + ix with
 * ix = floor((x - x_min) / h) clamped to [0, N-1], ties in ascending id.
 * DEVICE arrays: x, y (float64, n), id (int32, n) in; cell (int32, n),
 * count (int32, N^2), offset (int32, N^2 + 1) and perm (int32, n: input
 * positions in sorted order) out.  Synchronises. */
int qs_cell_sort(qs_ctx *ctx, const double *x, const double *y, const int32_t *id, int64_t n,
                 int32_t *cell, int32_t *count, int32_t *offset, int32_t *perm);

/* Largest grid (N * N cells) that qs_cell_sort_noalloc accepts. */
#define QS_NOALLOC_MAX_CELLS (512 * 512)

/* The cell sort of qs_cell_sort without a context and without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory, such as
 * applications that give all of the GPU's memory to their own pool or arena
 * (an outside cudaMalloc breaks their budget or fails), hosts that hand a
 * plugin raw buffers but no allocator, and loops that must not pay for
 * cudaMalloc / cudaFree, which can synchronise the device.
 *
 * Grid: n x n cells of side h with lower corner (x_min, y_min); n * n must
 * not exceed QS_NOALLOC_MAX_CELLS, else QS_ERR_ARG.  DEVICE arrays as in
 * qs_cell_sort: x, y (float64, np), id (int32, np) in; cell (int32, np),
 * count (int32, n*n), offset (int32, n*n + 1), perm (int32, np) out.  The
 * work is queued on `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without waiting; the outputs are ready once
 * the stream reaches that point.
 *
 * Scratch: a file-scope device array of QS_NOALLOC_MAX_CELLS int32 (1 MiB)
 * that every GPU loading this library holds until the process exits.  All
 * calls share it and it keeps the last call's contents; each call clears the
 * part it uses before using it.  Calls that overlap on the GPU (on different
 * streams, or from different host threads without ordering) race on it and
 * give wrong results: order them.  Every call looks up the array's device
 * address (cudaGetSymbolAddress) in the current device's current context,
 * so a device reset or a context switch between calls is harmless; the
 * first call on a device also loads the module there, so make that first
 * call before any stream capture begins.
 * Errors: QS_ERR_ARG, QS_ERR_CUDA (launch or address lookup failed). */
int qs_cell_sort_noalloc(int n, double x_min, double y_min, double h, const double *x,
                         const double *y, const int32_t *id, int64_t np, int32_t *cell,
                         int32_t *count, int32_t *offset, int32_t *perm, void *cuda_stream);

/* ---- Field solver on a nonuniform transverse grid ----------------------
 * Sec. "Multigrid Solver with Nonuniform Grids": (d_xx + d_yy) Psi + M Psi = J
 * on a tensor-product grid of nodes x_i, y_j, discretised with the
 * three-point second differences of Eq. 2D_Laplac and, with the correction
 * on, the third-order terms replaced as in Eq. 2D_Laplac_3rd (the mixed
 * third derivatives as the three-point first difference of the other axis'
 * second difference, d(lap) as that first difference of J - M Psi).  The
 * discrete system is A Psi = J' with
 *   A  = D2x + D2y + M + cx (D1x D2y + D1x M) + cy (D1y D2x + D1y M),
 *   J' = J + (cx D1x + cy D1y) J,   c = (h^+ - h^-) / 3 per node and axis,
 * a 9-point, non-symmetric operator (c = 0 with the correction off).  The
 * third-order term is subtracted (Taylor expansion of the three-point
 * difference) and the y bracket carries h_y^b.  Walls are nodes where Psi = 0
 * and J = 0.  Arrays are [iy][ix] with ix fastest, float64.
 *
 * The solver is a multigrid V(2,2) cycle: coarse levels keep every other
 * node and rediscretise A there, prolongation is linear interpolation in
 * physical coordinates, restriction its dual-length-weighted transpose (also
 * applied to M), the smoother four-colour Gauss-Seidel over-relaxed by 1.3,
 * the 3 x 3 level is solved exactly.  The paper cites the transfer weights without giving
 * them; these are the readings. */
typedef struct qs_nu_solver qs_nu_solver;

/* Build the hierarchy for n interior nodes per side, n = 2^k - 1 with
 * 2 <= k <= 12 (3 .. 4095).  x_nodes, y_nodes: HOST arrays of n + 2 strictly
 * increasing coordinates, the first and the last being the walls; copied (the
 * caller keeps them).  correction: 1 = with the third-order correction, 0 =
 * the plain three-point scheme.  precision: QS_FP64 (every cycle in float64)
 * or QS_FP32_REFINED (float32 V-cycles correct a float64 solution from its
 * float64 residual each cycle; the stopping test and the result are those of
 * float64).  cuda_stream: the cudaStream_t every call of this solver queues
 * on (NULL = legacy default stream).  The solver owns its device memory
 * (about 14 * 4/3 * n^2 elements of its precision, plus 5 n^2 float64 for
 * the refined form) until qs_nu_destroy.  Argument checks come before any
 * CUDA call.  Errors: QS_ERR_ARG (n not 2^k - 1, axes not increasing, bad
 * flag), QS_ERR_OOM, QS_ERR_CUDA. */
int qs_nu_create(int n, const double *x_nodes, const double *y_nodes, int correction,
                 int precision, void *cuda_stream, qs_nu_solver **out);

/* Solve A Psi = J' for nrhs (1 .. 4) fields that share M.
 * d_m: DEVICE n*n screening M, or NULL for M = 0 (Poisson).  M <= 0 keeps the
 *      operator elliptic (the screened equation of B_perp has M = -kappa).
 * d_j: DEVICE [nrhs][n][n] sources J (not J'); J' is formed inside.
 * d_u: DEVICE [nrhs][n][n]; in: initial guess, out: the solution (the last
 *      iterate when the cycle cap is hit).  Caller-owned, written in place.
 * Stops when every field has ||J' - A u||_2 <= tol ||J'||_2 (a field with
 * J' = 0 gets u = 0), or after max_cycles V-cycles.  cycles (HOST, may be
 * NULL) receives the V-cycles done; relres (HOST, nrhs, may be NULL) the
 * final relative residuals.  Synchronises the solver's stream.
 * Errors: QS_ERR_ARG, QS_ERR_NOT_CONVERGED (cap hit), QS_ERR_TIMEOUT (a grid
 * barrier wait ran out; the kernel returned), QS_ERR_CUDA. */
int qs_nu_solve(qs_nu_solver *s, const double *d_m, int nrhs, const double *d_j, double *d_u,
                double tol, int max_cycles, int *cycles, double *relres);

/* Cycle of the following solves: pre_sweeps and post_sweeps (0 .. 8,
 * sum >= 1) four-colour Gauss-Seidel sweeps per level, relaxed by omega
 * (0 < omega < 2; 1 = plain Gauss-Seidel); levels of side <= coarse_block_n
 * are relaxed by one thread block, the larger ones by the whole GPU
 * (0 = default).  staged: 1 = the larger levels are smoothed in
 * shared-memory tiles with recomputed halos (one grid barrier per level and
 * leg; used when a tile's region fits in 200 KB, else 0), 0 = grid-wide
 * colour sweeps (a barrier per colour).  Both give the same iterates up to
 * rounding.
 * Defaults 2, 2, 1.3, 31, 1.  Host only.  Errors: QS_ERR_ARG. */
int qs_nu_set_cycle(qs_nu_solver *s, int pre_sweeps, int post_sweeps, double omega,
                    int coarse_block_n, int staged);

/* d_out = A d_u for one field (DEVICE, n*n each; d_m as in qs_nu_solve).
 * Queued on the solver's stream without waiting.  Errors: QS_ERR_ARG,
 * QS_ERR_CUDA. */
int qs_nu_apply(qs_nu_solver *s, const double *d_m, const double *d_u, double *d_out);

/* d_out = J' = J + (cx D1x + cy D1y) J for one field (DEVICE, n*n each).
 * Queued on the solver's stream without waiting.  Errors: QS_ERR_ARG,
 * QS_ERR_CUDA. */
int qs_nu_source(qs_nu_solver *s, const double *d_j, double *d_out);

/* Free the solver and its device memory (NULL is a no-op). */
void qs_nu_destroy(qs_nu_solver *s);

/* ---- The slice advance on a nonuniform transverse grid ------------------
 * Sec. "Multigrid Solver with Nonuniform Grids" uses the node grid for the
 * whole quasi-static loop.  This is the slice loop of qs_step3d (Algorithm 1)
 * with every grid operation on the tensor-product node grid of qs_nu_create:
 * CIC deposits and gathers linear in physical coordinates between the nodes
 * around a particle (weight on a wall node folded into the adjacent interior
 * node, density = deposit / the node's dual area: half of each adjacent
 * interval, the whole interval to the wall for the first and last node);
 * gradients by the three-point first difference printed after Eq.
 * 2D_Laplac_3rd, zero beyond the walls; the five field equations by the
 * nonuniform solver with the third-order correction, warm-started from the
 * previous slice (M = 0 for psi, E_z, B_z; M = -kappa for B_perp); the
 * Boris-like push with specular walls at the outer nodes; sub-steps by
 * Step_Size_Refinement with V0 = (smallest node spacing) / dxi0.  Particles
 * and grids are float64; the solves run in `precision` (QS_FP64 or
 * QS_FP32_REFINED, see qs_nu_create).  The driver enters as a given j_z on
 * the nodes of the base slices.  Arrays are [iy][ix] over the n x n interior
 * nodes. */
typedef struct qs_nu_pic qs_nu_pic;

/* n = 2^k - 1 interior nodes per side; x_nodes, y_nodes: HOST, n + 2
 * strictly increasing coordinates, walls first and last (copied).  n_xi base
 * slices over a window of length xi_len; refine_k and psi_floor as in
 * qs_config.  The object owns its device memory until qs_nu_pic_destroy.
 * Errors: QS_ERR_ARG, QS_ERR_OOM, QS_ERR_CUDA. */
int qs_nu_pic_create(int n, const double *x_nodes, const double *y_nodes, int n_xi,
                     double xi_len, int refine_k, double psi_floor, int precision,
                     void *cuda_stream, qs_nu_pic **out);

/* Quiet-start plasma: sqrt(ppc) x sqrt(ppc) particles in every rectangle
 * between neighbouring nodes (walls included) at offsets (k + 1/2)/sqrt(ppc)
 * of it, weight = its area / ppc, p_perp = 0; the ion background is their
 * deposit.  (n + 1)^2 ppc particles.  Synchronises.  Errors: QS_ERR_ARG
 * (ppc not a perfect square), QS_ERR_OOM, QS_ERR_CUDA. */
int qs_nu_pic_init_plasma(qs_nu_pic *s, int ppc);

/* One 3D step from the lattice at the head of the window.  d_jzb: DEVICE
 * float64 [n_xi][n][n] driver j_z on the nodes of the base slices (linear in
 * xi at sub-steps).  d_hist: DEVICE float64 [5][n_xi][n][n], OVERWRITTEN with
 * psi, E_z, B_z, B_x, B_y at the base slices.  Each solve stops at relative
 * residual tol or max_cycles V-cycles.  stats (may be NULL): slices,
 * pushes, V-cycles per solve kind, max_m, gpu_ms.  Synchronises.  Errors:
 * QS_ERR_STATE (no plasma), QS_ERR_ARG, QS_ERR_NOT_CONVERGED (a solve hit
 * max_cycles; the step still completed), QS_ERR_TIMEOUT, QS_ERR_CUDA. */
int qs_nu_pic_step3d(qs_nu_pic *s, const double *d_jzb, double *d_hist, double tol,
                     int max_cycles, qs_step_stats *stats);

/* The plasma after the last step (or the lattice), HOST arrays of
 * qs_nu_pic_count() entries (any may be NULL).  Synchronises. */
int qs_nu_pic_get_plasma(qs_nu_pic *s, double *x, double *y, double *px, double *py, double *w);
int64_t qs_nu_pic_count(const qs_nu_pic *s);

/* Free the object and its device memory (NULL is a no-op). */
void qs_nu_pic_destroy(qs_nu_pic *s);

/* ---- Laser-envelope advance ---------------------------------------------
 * Sec. "Description of different plasma wake drivers", Eq. laser_Enve: the
 * complex envelope A of a laser with vector potential A exp(-i k0 xi) obeys
 *   (2 i k0 d_t - 2 d_t d_xi + lap_perp) A = chi A,   chi = n_* / (1 + psi).
 * One time step is time-centred for lap_perp and chi, with the mixed
 * derivative as the time difference of a backward (towards the head)
 * difference in xi; slices advance from the head (j = 0) to the tail, each a
 * complex screened-Poisson equation
 *   (lap - chi_j + c) A^{n+1}_j = (c + chi_j - lap) A^n_j - q (A^{n+1}_{j-1} - A^n_{j-1}),
 *   c = 4 (i k0 - 1/dxi) / dt,  q = 4 / (dt dxi)
 * solved by complex multigrid (red-black Gauss-Seidel V(2,2), warm-started
 * from A^n_j as the paper does).  chi is held at t_n; A = 0 ahead of the
 * window and on the walls.  The grid is the slice advance's: n x n cells on a
 * square box of side `width`, cell-centred, 5-point Laplacian with odd
 * ghosts; multigrid coarsens while the side is even and above 4, so n should
 * be c * 2^L with c <= 4. */
typedef struct qs_laser qs_laser;

/* n cells per side (2 .. 8192), width > 0 (k_p^-1), n_xi >= 1 slices, k0 =
 * omega_0 / omega_p > 0, dt > 0 (1/omega_p), dxi > 0 the slice spacing, or
 * +inf for no xi coupling (q = 0).  cuda_stream: the cudaStream_t of every
 * call (NULL = legacy default).  The object owns about (4 + 5 * 4/3) n^2
 * complex128 of device memory until qs_laser_destroy.  Argument checks come
 * before any CUDA call.  Errors: QS_ERR_ARG, QS_ERR_OOM, QS_ERR_CUDA. */
int qs_laser_create(int n, double width, int n_xi, double k0, double dt, double dxi,
                    void *cuda_stream, qs_laser **out);

/* Advance the envelope `steps` (>= 0) time steps with chi held fixed.
 * d_chi: DEVICE float64 [n_xi][n][n]; d_a: DEVICE complex128 [n_xi][n][n]
 * (interleaved re, im), A^n in, A^{n+steps} out, caller-owned, written in
 * place.  Each slice's solve stops at ||f - A u||_2 <= tol ||f||_2 or after
 * max_cycles V-cycles.  cycles (HOST, may be NULL): V-cycles over all slices
 * and steps; max_relres (HOST, may be NULL): the largest final relative
 * residual of a slice.  Synchronises the stream.  Errors: QS_ERR_ARG,
 * QS_ERR_NOT_CONVERGED (some slice hit max_cycles; the advance still
 * completed), QS_ERR_TIMEOUT, QS_ERR_CUDA. */
int qs_laser_advance(qs_laser *s, const double *d_chi, double *d_a, int steps, double tol,
                     int max_cycles, int64_t *cycles, double *max_relres);

/* Free the object and its device memory (NULL is a no-op). */
void qs_laser_destroy(qs_laser *s);

/* One 3D step of a laser-driven wake (Algorithm 1 with the laser driver,
 * Sec. "WAND-PIC's Global Algorithm", last paragraph): |A|^2 of `envelope`
 * (DEVICE complex128 [n_xi][ny][nx], interleaved re, im, caller-owned)
 * drives the slice loop of qs_step3d_laser, together with the beams (n_beams
 * may be 0), which yields chi = n_* / (1+psi) at the base slices; then the
 * envelope advances one time step of Eq. laser_Enve with that chi
 * (qs_laser_advance with steps = 1, tol, max_cycles), IN PLACE.  The laser
 * object must have the context's cells, box width, slice count and slice
 * spacing (QS_ERR_ARG otherwise).  The context allocates, on first use, two
 * float64 arrays of n_xi * N^2 (|A|^2 and chi), kept until qs_destroy.
 * stats: the slice loop's counters; env_cycles, env_relres (HOST, may be
 * NULL): the envelope advance's V-cycles and largest final relative
 * residual.  Synchronises.  Errors: those of qs_step3d_laser and
 * qs_laser_advance, QS_ERR_OOM. */
int qs_laser_step3d(qs_ctx *ctx, qs_laser *laser, const qs_beam *beams, int n_beams,
                    double *envelope, double tol, int max_cycles, qs_step_stats *stats,
                    int64_t *env_cycles, double *env_relres);

/* Name of a status code (static string). */
const char *qs_strerror(int status);

/* Last detailed error message of a context ("" if none). */
const char *qs_last_error(const qs_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
