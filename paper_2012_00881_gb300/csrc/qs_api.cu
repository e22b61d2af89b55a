// Host side of the libqs C ABI (declared in include/qs.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "qs_internal.cuh"

struct qs_ctx {
    qs_config cfg;
    cudaStream_t st = nullptr;
    int dev = 0;
    int N = 0;
    double h = 0.0;
    int nlev = 0;
    int lev_n[QS_MAX_LEV] = {};
    std::vector<void *> allocs;
    // grids
    double *n_a = nullptr, *n_b = nullptr, *n_ion = nullptr;
    double *jx = nullptr, *jy = nullptr, *txx = nullptr, *txy = nullptr, *tyy = nullptr,
           *G = nullptr;
    double *psi = nullptr, *ez = nullptr, *bz = nullptr, *bx = nullptr, *by = nullptr;
    double *f_psi = nullptr, *f_ez = nullptr, *f_bz = nullptr, *f_bx = nullptr, *f_by = nullptr;
    double *dpx = nullptr, *dpy = nullptr, *jz = nullptr, *kap = nullptr, *invd0 = nullptr;
    double *hist1[5] = {}, *hist2[5] = {};
    LevelArrays lev[QS_MAX_LEV] = {};
    float *e32[2] = {nullptr, nullptr}, *r32[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    double *r64[2] = {nullptr, nullptr};
    float *k32 = nullptr, *d32 = nullptr;
    LevelArrays32 lev32[QS_MAX_LEV] = {};
    int block_level_n = 16;
    int tile_x = 0, tile_y = 0;
    size_t tile_offset = 0, block_offset = 0;
    double *hist = nullptr, *jzb = nullptr;
    // laser driver: |A|^2 and grad(|A|^2/4) of the current slice; |A|^2 and
    // chi of every base slice for the laser-driven step (allocated on use)
    double *a2 = nullptr, *pondx = nullptr, *pondy = nullptr;
    float *f32[5] = {};  // refined form: float32 grad psi and B for the push
    double *a2_all = nullptr, *chi_all = nullptr;
    bool last_laser = false;
    DevScalars *sc = nullptr;
    int32_t *diag_m = nullptr, *d_sched = nullptr;
    double *diag_vmax = nullptr, *diag_charge = nullptr;
    // sort scratch
    int32_t *s_cursor = nullptr;
    // the in-loop sort (config.sort_every > 0): cell counts and offsets, the
    // per-block chunk sums, per-particle cells and order, the spare particle set
    int32_t *l_count = nullptr, *l_offset = nullptr, *l_cursor = nullptr, *l_bsum = nullptr;
    int32_t *l_cell = nullptr, *l_order = nullptr, *id2 = nullptr;
    double *x2 = nullptr, *y2 = nullptr, *wd2 = nullptr;
    void *px2 = nullptr, *py2 = nullptr, *w2 = nullptr;
    int64_t *trace = nullptr;
    // plasma
    int64_t np = 0;
    int ppc = 0;
    double *t_x = nullptr, *t_y = nullptr, *t_px = nullptr, *t_py = nullptr, *t_w = nullptr;
    int32_t *t_id = nullptr;
    double *x = nullptr, *y = nullptr, *px = nullptr, *py = nullptr, *w = nullptr;
    int32_t *id = nullptr;
    float *px32 = nullptr, *py32 = nullptr, *w32 = nullptr;
    float *g32[6] = {};  // refined form: jx, jy, txx, txy, tyy, G
    std::vector<void *> plasma_allocs;
    bool have_plasma = false, have_step = false;
    // plasma checkpoints of the last qs_step3d (config.checkpoint_every > 0)
    double *ckpt = nullptr;
    size_t ckpt_count = 0;
    int ckpt_every = 0;
    bool ckpt_valid = false;
    // every slice of the last qs_step3d (config.checkpoint_every >= n_xi and
    // room in device memory): the adjoint's segment store for the whole window
    double *store = nullptr;
    size_t store_slots = 0;
    int store_n_sub = 0;
    bool store_valid = false;
    int engine_blocks = 0;
    size_t engine_smem = 0;
    int cl_size = 1;          // thread-block cluster of the float64 small-grid solves
    size_t cl_offset = 0;     // its arrays in the engine's dynamic shared memory
    int band_rows = 0, band_rows_n = 0;  // privatised deposit bands (rows)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    char msg[512] = {0};
};

namespace {

int fail(qs_ctx *c, int status, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
        va_end(ap);
    }
    return status;
}

int cuda_fail(qs_ctx *c, cudaError_t e, const char *what) {
    cudaGetLastError();
    int st = (e == cudaErrorMemoryAllocation) ? QS_ERR_OOM : QS_ERR_CUDA;
    return fail(c, st, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename T>
int dalloc(qs_ctx *c, std::vector<void *> &list, T **p, size_t count) {
    void *q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
    list.push_back(q);
    *p = static_cast<T *>(q);
    return QS_OK;
}

#define AL(list, ptr, count)                        \
    do {                                            \
        int r_ = dalloc(c, list, &(ptr), (count));  \
        if (r_ != QS_OK) return r_;                 \
    } while (0)

int validate(const qs_config *cfg, char *why, size_t nwhy) {
    if (!cfg) {
        snprintf(why, nwhy, "config is NULL");
        return QS_ERR_ARG;
    }
    if (cfg->nx != cfg->ny || cfg->nx < 2) {
        snprintf(why, nwhy, "nx must equal ny and be >= 2 (got %d, %d)", cfg->nx, cfg->ny);
        return QS_ERR_ARG;
    }
    const double lx = cfg->x_max - cfg->x_min, ly = cfg->y_max - cfg->y_min;
    if (!(lx > 0.0) || !(ly > 0.0) || std::fabs(lx - ly) > 1e-12 * lx) {
        snprintf(why, nwhy, "the box must be square with positive extent");
        return QS_ERR_ARG;
    }
    int n = cfg->nx;
    while (n % 2 == 0 && n > 4) n /= 2;
    if (n > 8) {
        snprintf(why, nwhy, "N = %d does not coarsen to a side <= 8", cfg->nx);
        return QS_ERR_ARG;
    }
    if (cfg->n_xi < 1 || !(cfg->xi_max > cfg->xi_min)) {
        snprintf(why, nwhy, "need n_xi >= 1 and xi_max > xi_min");
        return QS_ERR_ARG;
    }
    if (cfg->refine_k < 1 || cfg->refine_k > 1024) {
        snprintf(why, nwhy, "refine_k must be in [1, 1024]");
        return QS_ERR_ARG;
    }
    if (cfg->precision != QS_FP64 && cfg->precision != QS_FP32_REFINED) {
        snprintf(why, nwhy, "unknown precision %d", cfg->precision);
        return QS_ERR_ARG;
    }
    if (!(cfg->mg_tol > 0.0) || cfg->mg_max_vcycles < 1 || !(cfg->psi_floor > 0.0)) {
        snprintf(why, nwhy, "need mg_tol > 0, mg_max_vcycles >= 1, psi_floor > 0");
        return QS_ERR_ARG;
    }
    if (cfg->pre_sweeps < -1 || cfg->post_sweeps < 0 || cfg->pre_sweeps > 8 ||
        cfg->post_sweeps > 8 || (cfg->pre_sweeps == 0 && cfg->post_sweeps == 0)) {
        snprintf(why, nwhy, "sweeps must be in [0, 8] with at least one (pre_sweeps -1: default)");
        return QS_ERR_ARG;
    }
    if (cfg->sort_every < 0) {
        snprintf(why, nwhy, "sort_every must be >= 0");
        return QS_ERR_ARG;
    }
    if (cfg->coarse_block_n < 0 || cfg->coarse_block_n > 4096) {
        snprintf(why, nwhy, "coarse_block_n must be in [0, 4096]");
        return QS_ERR_ARG;
    }
    if (cfg->trace_capacity < 0 || cfg->trace_capacity > (1 << 26)) {
        snprintf(why, nwhy, "trace_capacity must be in [0, 2^26]");
        return QS_ERR_ARG;
    }
    if (cfg->warm_start_order < 0 || cfg->warm_start_order > 2) {
        snprintf(why, nwhy, "warm_start_order must be 0, 1 or 2");
        return QS_ERR_ARG;
    }
    if (cfg->tile_x < 0 || cfg->tile_y < 0 || (cfg->tile_x & 1) || (cfg->tile_y & 1) ||
        cfg->tile_x > 256 || cfg->tile_y > 256 || ((cfg->tile_x == 0) != (cfg->tile_y == 0))) {
        snprintf(why, nwhy, "tile_x, tile_y must both be 0 or even in [2, 256]");
        return QS_ERR_ARG;
    }
    if (cfg->omega_pct != 0 && (cfg->omega_pct < 50 || cfg->omega_pct > 195)) {
        snprintf(why, nwhy, "omega_pct must be 0 or in [50, 195]");
        return QS_ERR_ARG;
    }
    if (cfg->coarse_pre_sweeps < 0 || cfg->coarse_pre_sweeps > 8) {
        snprintf(why, nwhy, "coarse_pre_sweeps must be in [0, 8]");
        return QS_ERR_ARG;
    }
    if (cfg->checkpoint_every < 0) {
        snprintf(why, nwhy, "checkpoint_every must be >= 0");
        return QS_ERR_ARG;
    }
    if (cfg->barrier_wait_cycles < 0) {
        snprintf(why, nwhy, "barrier_wait_cycles must be >= 0");
        return QS_ERR_ARG;
    }
    if (cfg->deposit_band_rows < -1 || (cfg->deposit_band_rows > 0 && cfg->deposit_band_rows < 3)) {
        snprintf(why, nwhy, "deposit_band_rows must be -1, 0 or >= 3");
        return QS_ERR_ARG;
    }
    const int cs = cfg->cluster_size;
    if (cs != 0 && cs != 1 && cs != 8 && cs != 16) {
        snprintf(why, nwhy, "cluster_size must be 0, 1, 8 or 16");
        return QS_ERR_ARG;
    }
    const int cl_max_n = cfg->precision == QS_FP64 ? 128 : 256;
    if (cs > 1 && (cfg->nx % (2 * cs) != 0 || cfg->nx > cl_max_n)) {
        snprintf(why, nwhy, "cluster_size %d needs N <= %d divisible by %d", cs, cl_max_n,
                 2 * cs);
        return QS_ERR_ARG;
    }
    return QS_OK;
}

int create_impl(qs_ctx *c) {
    const qs_config &g = c->cfg;
    CK(cudaGetDevice(&c->dev), "cudaGetDevice");
    c->N = g.nx;
    c->h = (g.x_max - g.x_min) / g.nx;
    int n = c->N;
    c->nlev = 0;
    c->lev_n[c->nlev++] = n;
    while (n % 2 == 0 && n > 4 && c->nlev < QS_MAX_LEV) {
        n /= 2;
        c->lev_n[c->nlev++] = n;
    }
    const size_t nn = (size_t)c->N * c->N;
    auto &L = c->allocs;
    double **grids[] = {&c->n_a, &c->n_b, &c->n_ion, &c->jx,  &c->jy,   &c->txx, &c->txy,
                        &c->tyy, &c->G,   &c->psi,   &c->ez,  &c->bz,   &c->bx,  &c->by,
                        &c->f_psi, &c->f_ez, &c->f_bz, &c->f_bx, &c->f_by, &c->dpx, &c->dpy,
                        &c->jz,  &c->kap, &c->invd0, &c->hist1[0], &c->hist1[1],
                        &c->hist1[2], &c->hist1[3], &c->hist1[4], &c->hist2[0], &c->hist2[1],
                        &c->hist2[2], &c->hist2[3], &c->hist2[4], &c->a2, &c->pondx,
                        &c->pondy};
    for (double **p : grids) AL(L, *p, nn);
    const bool ref = g.precision == QS_FP32_REFINED;
    for (int l = 1; l < c->nlev; ++l) {
        const size_t m = (size_t)c->lev_n[l] * c->lev_n[l];
        if (ref) {
            AL(L, c->lev32[l].u[0], m);
            AL(L, c->lev32[l].u[1], m);
            AL(L, c->lev32[l].f[0], m);
            AL(L, c->lev32[l].f[1], m);
            AL(L, c->lev32[l].k, m);
            AL(L, c->lev32[l].d, m);
        } else {
            AL(L, c->lev[l].u[0], m);
            AL(L, c->lev[l].u[1], m);
            AL(L, c->lev[l].f[0], m);
            AL(L, c->lev[l].f[1], m);
            AL(L, c->lev[l].kap, m);
            AL(L, c->lev[l].d, m);
            AL(L, c->lev[l].s[0], m);  // the staged down legs' pre-smoothed iterate
            AL(L, c->lev[l].s[1], m);
        }
    }
    if (!ref) {  // level 0's scratch pair of the staged float64 cycle
        AL(L, c->lev[0].s[0], nn);
        AL(L, c->lev[0].s[1], nn);
    }
    if (ref)
        for (int k = 0; k < 5; ++k) AL(L, c->f32[k], nn);
    if (ref) {
        float **g32[] = {&c->e32[0],    &c->e32[1],    &c->r32[0][0], &c->r32[0][1],
                         &c->r32[1][0], &c->r32[1][1], &c->k32,       &c->d32,
                         &c->g32[0], &c->g32[1], &c->g32[2], &c->g32[3], &c->g32[4],
                         &c->g32[5]};
        for (float **p : g32) {
            AL(L, *p, nn);
            CK(cudaMemsetAsync(*p, 0, nn * sizeof(float), c->st), "memset");
        }
        AL(L, c->r64[0], nn);
        AL(L, c->r64[1], nn);
    }
    AL(L, c->hist, 5 * (size_t)g.n_xi * nn);
    AL(L, c->jzb, (size_t)g.n_xi * nn);
    AL(L, c->sc, 1);
    AL(L, c->diag_m, (size_t)g.n_xi);
    AL(L, c->d_sched, (size_t)g.n_xi);
    AL(L, c->diag_vmax, (size_t)g.n_xi);
    AL(L, c->diag_charge, (size_t)g.n_xi);
    AL(L, c->s_cursor, nn);
    if (g.sort_every > 0) {
        AL(L, c->l_count, nn);
        AL(L, c->l_offset, nn + 1);
        AL(L, c->l_cursor, nn);
        AL(L, c->l_bsum, (size_t)1024);
    }
    if (g.trace_capacity > 0) AL(L, c->trace, 2 * (size_t)g.trace_capacity);
    // fields start at zero (the warm start of the first slice)
    for (double **p : grids) CK(cudaMemsetAsync(*p, 0, nn * sizeof(double), c->st), "memset");
    CK(cudaMemsetAsync(c->hist, 0, 5 * (size_t)g.n_xi * nn * sizeof(double), c->st), "memset");
    CK(cudaMemsetAsync(c->jzb, 0, (size_t)g.n_xi * nn * sizeof(double), c->st), "memset");
    c->block_level_n = g.coarse_block_n > 0 ? g.coarse_block_n : (ref ? 32 : 16);
    // staged grid levels in both forms: 32 x 16 output tiles by default; the
    // float64 form takes 64 x 32 on grids of 512^2 and more, where a smaller
    // share of each region is recomputed halo (blowout512: +10 %)
    const bool big64 = !ref && c->N >= 512;
    c->tile_x = g.tile_x > 0 ? g.tile_x : (big64 ? 64 : 32);
    c->tile_y = g.tile_y > 0 ? g.tile_y : (big64 ? 32 : 16);
    const int nu = g.pre_sweeps > g.post_sweeps ? g.pre_sweeps : g.post_sweeps;
    c->engine_smem = qs_engine_smem_bytes(c->lev_n, c->nlev, c->block_level_n, g.precision,
                                          c->tile_x, c->tile_y, nu, g.post_sweeps,
                                          &c->block_offset, &c->tile_offset);
    int cs = g.cluster_size;
    if (cs == 0) {
        if (!ref)  // float64: small grids, 16 blocks where the strips keep >= 2 rows
            cs = (c->N <= 64 && c->N % 32 == 0) ? 16 : (c->N <= 64 && c->N % 16 == 0) ? 8 : 1;
        else  // refined: the grid-wide cycles were faster at every size measured
            cs = 1;
    }
    if (cs > 1) {
        // the cluster arrays follow the coarsest inverses; they overlap the
        // shared-memory coarse part and tiles of the grid-wide cycle, which
        // a clustered launch does not use (the adjoint's launch does)
        c->cl_offset = c->block_offset;
        const size_t need =
            c->cl_offset + qs_cluster_smem_bytes(c->lev_n, c->nlev, cs, ref ? 4 : 8) + 256;
        if (need > c->engine_smem) c->engine_smem = need;
    }
    if (g.deposit_band_rows != 0) {
        // privatised deposits: the bands reuse the shared memory of the
        // cycles after the coarsest inverses (free between solves); room for
        // at least 8 rows of the six moments where 200 KB allow it
        const size_t row_m = (size_t)6 * c->N * (ref ? 4 : 8), row_n = (size_t)8 * c->N;
        const size_t want = c->block_offset + 8 * row_m + 256;
        const size_t cap = 200 * 1024;
        if (want > c->engine_smem) c->engine_smem = want < cap ? want : cap;
        const size_t avail = c->engine_smem - 256 - c->block_offset;
        const size_t rm = avail / row_m, rn = avail / row_n;
        const size_t lim = g.deposit_band_rows > 0 ? (size_t)g.deposit_band_rows : (size_t)c->N;
        const size_t cap_m = rm < lim ? rm : lim, cap_n = rn < lim ? rn : lim;
        c->band_rows = g.deposit_band_rows != 0 && cap_m >= 3 ? (int)cap_m : 0;
        c->band_rows_n = g.deposit_band_rows != 0 && cap_n >= 3 ? (int)cap_n : 0;
    }
    if (c->engine_smem > 220 * 1024)
        return fail(c, QS_ERR_ARG,
                    "coarse_block_n = %d with %d x %d tiles needs %zu bytes of shared memory",
                    c->block_level_n, c->tile_x, c->tile_y, c->engine_smem);
    int blocks = 0;
    if (qs_engine_max_blocks(c->dev, g.precision, c->engine_smem, &blocks, cs) != 0 ||
        blocks < cs)
        return fail(c, QS_ERR_CUDA, "slice engine cannot be made resident");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev), "attr");
    c->engine_blocks = blocks < sms ? blocks : sms;
    c->engine_blocks -= c->engine_blocks % cs;  // whole clusters
    c->cl_size = cs;
    CK(cudaEventCreate(&c->ev0), "event");
    CK(cudaEventCreate(&c->ev1), "event");
    CK(cudaStreamSynchronize(c->st), "sync");
    return QS_OK;
}

void free_list(std::vector<void *> &l) {
    for (void *p : l) cudaFree(p);
    l.clear();
}

int check_ctx(qs_ctx *c) { return c ? QS_OK : QS_ERR_ARG; }

}  // namespace

extern "C" {

void qs_config_default(qs_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = cfg->ny = 64;
    cfg->x_min = cfg->y_min = -6.0;
    cfg->x_max = cfg->y_max = 6.0;
    cfg->n_xi = 128;
    cfg->xi_min = 0.0;
    cfg->xi_max = 12.0;
    cfg->refine_k = 8;
    cfg->precision = QS_FP64;
    cfg->mg_tol = 1e-10;
    cfg->mg_max_vcycles = 60;
    cfg->psi_floor = 1e-3;
    cfg->max_psi_guard_hits = -1;
    cfg->sort_every = 16;
    cfg->pre_sweeps = -1;  // the form's default (3 refined, 2 float64)
    cfg->post_sweeps = 2;
    cfg->coarse_pre_sweeps = 1;
    cfg->warm_start_order = 2;
}

int qs_create(const qs_config *cfg, void *cuda_stream, qs_ctx **out) {
    if (!out) return QS_ERR_ARG;
    *out = nullptr;
    char why[256];
    int v = validate(cfg, why, sizeof(why));
    if (v != QS_OK) return v;
    qs_ctx *c = new (std::nothrow) qs_ctx();
    if (!c) return QS_ERR_OOM;
    c->cfg = *cfg;
    // the form's default pre-sweeps: three in the refined form (fewer V-cycles
    // than two, and its float32 sweeps are cheap: blowout256 +4 %), two in
    // the float64 form (three measured 1 % slower there)
    if (c->cfg.pre_sweeps < 0) c->cfg.pre_sweeps = c->cfg.precision == QS_FP32_REFINED ? 3 : 2;
    c->st = static_cast<cudaStream_t>(cuda_stream);
    int r = create_impl(c);
    if (r != QS_OK) {
        free_list(c->allocs);
        if (c->ev0) cudaEventDestroy(c->ev0);
        if (c->ev1) cudaEventDestroy(c->ev1);
        delete c;
        return r;
    }
    *out = c;
    return QS_OK;
}

void qs_destroy(qs_ctx *c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->ckpt) cudaFree(c->ckpt);
    if (c->store) cudaFree(c->store);
    if (c->a2_all) cudaFree(c->a2_all);
    if (c->chi_all) cudaFree(c->chi_all);
    free_list(c->plasma_allocs);
    free_list(c->allocs);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

int qs_init_plasma(qs_ctx *c, int ppc, const double *profile, int n_coef, double r_max) {
    if (check_ctx(c)) return QS_ERR_ARG;
    int s = 1;
    while (s * s < ppc) ++s;
    if (ppc < 1 || s * s != ppc) return fail(c, QS_ERR_ARG, "ppc must be a perfect square");
    if (profile && (n_coef < 1 || !(r_max > 0.0)))
        return fail(c, QS_ERR_ARG, "profile needs n_coef >= 1 and r_max > 0");
    const size_t nn = (size_t)c->N * c->N;
    const int64_t np = (int64_t)nn * ppc;
    if (np > (int64_t)0x7fffffff) return fail(c, QS_ERR_ARG, "too many particles for int32 ids");
    CK(cudaStreamSynchronize(c->st), "sync");
    free_list(c->plasma_allocs);
    c->have_plasma = c->have_step = false;
    c->ckpt_valid = false;
    c->store_valid = false;
    if (np != c->np) {
        // the checkpoints and the slice store are sized by the particle count
        if (c->ckpt) cudaFree(c->ckpt);
        if (c->store) cudaFree(c->store);
        c->ckpt = nullptr;
        c->ckpt_count = 0;
        c->store = nullptr;
        c->store_slots = 0;
    }
    auto &L = c->plasma_allocs;
    AL(L, c->t_x, np);
    AL(L, c->t_y, np);
    AL(L, c->t_px, np);
    AL(L, c->t_py, np);
    AL(L, c->t_w, np);
    AL(L, c->t_id, np);
    AL(L, c->x, np);
    AL(L, c->y, np);
    AL(L, c->px, np);
    AL(L, c->py, np);
    AL(L, c->w, np);
    AL(L, c->id, np);
    if (c->cfg.precision == QS_FP32_REFINED) {
        AL(L, c->px32, np);
        AL(L, c->py32, np);
        AL(L, c->w32, np);
    }
    if (c->cfg.sort_every > 0) {  // the spare set of the in-loop sort
        AL(L, c->l_cell, np);
        AL(L, c->l_order, np);
        AL(L, c->id2, np);
        AL(L, c->x2, np);
        AL(L, c->y2, np);
        if (c->cfg.precision == QS_FP32_REFINED) {
            float *a = nullptr, *b = nullptr, *w = nullptr;
            AL(L, a, np);
            AL(L, b, np);
            AL(L, w, np);
            AL(L, c->wd2, np);
            c->px2 = a;
            c->py2 = b;
            c->w2 = w;
        } else {
            double *a = nullptr, *b = nullptr, *w = nullptr;
            AL(L, a, np);
            AL(L, b, np);
            AL(L, w, np);
            c->px2 = a;
            c->py2 = b;
            c->w2 = w;
        }
    }
    double *d_table = nullptr;
    if (profile) {
        AL(L, d_table, (size_t)n_coef);
        CK(cudaMemcpyAsync(d_table, profile, sizeof(double) * n_coef, cudaMemcpyHostToDevice,
                           c->st),
           "copy profile");
    }
    c->np = np;
    c->ppc = ppc;
    const qs_config &g = c->cfg;
    CK(qs_launch_init_plasma(c->st, c->N, ppc, g.x_min, g.y_min, c->h, d_table, n_coef, r_max,
                             c->t_x, c->t_y, c->t_px, c->t_py, c->t_w, c->t_id),
       "init plasma");
    CK(cudaMemsetAsync(c->n_ion, 0, nn * sizeof(double), c->st), "memset");
    CK(qs_launch_deposit(c->st, c->t_x, c->t_y, c->t_w, np, c->N, g.x_min, g.y_min, c->h,
                         1.0 / (c->h * c->h), c->n_ion),
       "deposit n_ion");
    const size_t bd = np * sizeof(double);
    CK(cudaMemcpyAsync(c->x, c->t_x, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    CK(cudaMemcpyAsync(c->y, c->t_y, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    CK(cudaMemcpyAsync(c->px, c->t_px, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    CK(cudaMemcpyAsync(c->py, c->t_py, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    CK(cudaMemcpyAsync(c->w, c->t_w, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    CK(cudaMemcpyAsync(c->id, c->t_id, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st),
       "copy");
    CK(cudaStreamSynchronize(c->st), "init plasma");
    c->have_plasma = true;
    return QS_OK;
}

// Everything of a 3D step before the slice engine: validation, fresh plasma,
// zeroed fields, the driver current on the base slices, reset diagnostics;
// fills the engine arguments.  Work is queued on `st`.
static int step_prepare(qs_ctx *c, const qs_beam *beams, int n_beams, const int32_t *sched,
                        cudaStream_t st, EngineArgs &a, bool replay = false) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_plasma) return fail(c, QS_ERR_STATE, "qs_init_plasma has not been called");
    if (n_beams < 0 || (n_beams > 0 && !beams)) return fail(c, QS_ERR_ARG, "bad beam list");
    const qs_config &g = c->cfg;
    for (int b = 0; b < n_beams; ++b) {
        const qs_beam &bm = beams[b];
        if (bm.n < 0) return fail(c, QS_ERR_ARG, "beam %d: negative count", b);
        if (bm.n > 0 && (!bm.x || !bm.y || !bm.xi || !bm.px || !bm.py || !bm.pz || !bm.w))
            return fail(c, QS_ERR_ARG, "beam %d: NULL array", b);
    }
    if (sched) {
        for (int j = 0; j < g.n_xi; ++j)
            if (sched[j] < 1 || sched[j] > g.refine_k)
                return fail(c, QS_ERR_ARG, "m_schedule[%d] = %d outside [1, refine_k]", j,
                            sched[j]);
    }
    const size_t nn = (size_t)c->N * c->N;
    const double dxi0 = (g.xi_max - g.xi_min) / g.n_xi;
    // fresh plasma at the head of the window
    const size_t bd = c->np * sizeof(double);
    CK(cudaMemcpyAsync(c->x, c->t_x, bd, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c->y, c->t_y, bd, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c->px, c->t_px, bd, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c->py, c->t_py, bd, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c->w, c->t_w, bd, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c->id, c->t_id, c->np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st),
       "copy");
    CK(cudaMemsetAsync(c->n_a, 0, nn * sizeof(double), st), "memset");
    if (g.precision == QS_FP32_REFINED) {  // float32 momenta and weights of the refined form
        CK(qs_launch_convert(st, c->t_px, c->px32, c->np), "convert");
        CK(qs_launch_convert(st, c->t_py, c->py32, c->np), "convert");
        CK(qs_launch_convert(st, c->t_w, c->w32, c->np), "convert");
    }
    // the wake ahead of the driver is zero: every solve of the first slice
    // starts from zero
    for (double *f : {c->psi, c->ez, c->bz, c->bx, c->by})
        CK(cudaMemsetAsync(f, 0, nn * sizeof(double), st), "memset");
    // driver current on the base slices (a replay for the adjoint keeps the
    // current, the history and the diagnostics of the forward step)
    if (!replay) {
        CK(cudaMemsetAsync(c->jzb, 0, (size_t)g.n_xi * nn * sizeof(double), st), "memset");
        for (int b = 0; b < n_beams; ++b)
            CK(qs_launch_beam_deposit(st, beams[b], c->N, g.x_min, g.x_max, g.y_min, g.y_max,
                                      c->h, g.n_xi, g.xi_min, dxi0, c->jzb),
               "beam deposit");
        CK(cudaMemsetAsync(c->diag_m, 0, g.n_xi * sizeof(int32_t), st), "memset");
        CK(cudaMemsetAsync(c->diag_vmax, 0, g.n_xi * sizeof(double), st), "memset");
        CK(cudaMemsetAsync(c->diag_charge, 0, g.n_xi * sizeof(double), st), "memset");
    }
    CK(cudaMemsetAsync(c->sc, 0, sizeof(DevScalars), st), "memset");
    if (sched)
        CK(cudaMemcpyAsync(c->d_sched, sched, g.n_xi * sizeof(int32_t), cudaMemcpyHostToDevice,
                           st),
           "copy schedule");

    std::memset(&a, 0, sizeof(a));
    a.N = c->N;
    a.h = c->h;
    a.inv_h = 1.0 / c->h;
    a.x_min = g.x_min;
    a.x_max = g.x_max;
    a.y_min = g.y_min;
    a.y_max = g.y_max;
    a.n_xi = g.n_xi;
    a.dxi0 = dxi0;
    a.V0 = c->h / dxi0;
    a.refine_k = g.refine_k;
    a.psi_floor = g.psi_floor;
    a.mg_tol = g.mg_tol;
    a.mg_atol = 1e-15 * c->N;
    a.mg_max_vcycles = g.mg_max_vcycles;
    a.nu1 = g.pre_sweeps;
    a.nu2 = g.post_sweeps;
    a.nu1c = g.coarse_pre_sweeps > 0 ? g.coarse_pre_sweeps : g.pre_sweeps;
    a.omega = (g.omega_pct > 0 ? g.omega_pct : QS_DEFAULT_OMEGA_PCT) / 100.0;
    a.np = c->np;
    a.spin_cycles = g.barrier_wait_cycles > 0 ? (long long)g.barrier_wait_cycles : 4000000000LL;
    a.x = c->x;
    a.y = c->y;
    a.px = c->px;
    a.py = c->py;
    a.w = c->w;
    a.px32 = c->px32;
    a.py32 = c->py32;
    a.w32 = c->w32;
    a.jx32 = c->g32[0];
    a.jy32 = c->g32[1];
    a.txx32 = c->g32[2];
    a.txy32 = c->g32[3];
    a.tyy32 = c->g32[4];
    a.G32 = c->g32[5];
    a.n_a = c->n_a;
    a.n_b = c->n_b;
    a.n_ion = c->n_ion;
    a.jx = c->jx;
    a.jy = c->jy;
    a.txx = c->txx;
    a.txy = c->txy;
    a.tyy = c->tyy;
    a.G = c->G;
    a.psi = c->psi;
    a.ez = c->ez;
    a.bz = c->bz;
    a.bx = c->bx;
    a.by = c->by;
    a.f_psi = c->f_psi;
    a.f_ez = c->f_ez;
    a.f_bz = c->f_bz;
    a.f_bx = c->f_bx;
    a.f_by = c->f_by;
    a.dpx = c->dpx;
    a.dpy = c->dpy;
    a.jz = c->jz;
    a.kap = c->kap;
    a.invd0 = c->invd0;
    for (int f = 0; f < 5; ++f) {
        a.hist1[f] = c->hist1[f];
        a.hist2[f] = c->hist2[f];
    }
    a.ws_order = g.warm_start_order;
    a.nlev = c->nlev;
    for (int l = 0; l < c->nlev; ++l) {
        a.lev_n[l] = c->lev_n[l];
        const double hl = c->h * (double)(1 << l);
        a.lev_h2[l] = hl * hl;
        a.lev_inv_h2[l] = 1.0 / (hl * hl);
        a.lev_h2f[l] = (float)(hl * hl);
        a.lev_inv_h2f[l] = (float)(1.0 / (hl * hl));
        a.lev[l] = c->lev[l];
        a.lev32[l] = c->lev32[l];
    }
    a.block_level_n = c->block_level_n;
    a.cl_size = c->cl_size;
    a.cl_smem_offset = (int)c->cl_offset;
    a.band_rows = c->band_rows;
    a.band_rows_n = c->band_rows_n;
    a.band_off = (int)c->block_offset;
    a.id = c->id;
    if (g.sort_every > 0 && c->x2) {
        a.sort_every = g.sort_every;
        a.id2 = c->id2;
        a.x2 = c->x2;
        a.y2 = c->y2;
        a.wd2 = c->wd2;
        a.px2 = c->px2;
        a.py2 = c->py2;
        a.w2 = c->w2;
        a.s_count = c->l_count;
        a.s_offset = c->l_offset;
        a.s_cursor = c->l_cursor;
        a.s_cell = c->l_cell;
        a.s_order = c->l_order;
        a.s_bsum = c->l_bsum;
    }
    a.tile_x = c->tile_x;
    a.tile_y = c->tile_y;
    a.tile_smem_offset = (int)c->tile_offset;
    a.block_smem_offset = (int)c->block_offset;
    a.precision = g.precision;
    for (int k = 0; k < 2; ++k) {
        a.e32[k] = c->e32[k];
        a.r32[0][k] = c->r32[0][k];
        a.r32[1][k] = c->r32[1][k];
        a.r64[k] = c->r64[k];
    }
    a.k32 = c->k32;
    a.d32 = c->d32;
    a.dpx32 = c->f32[0];
    a.dpy32 = c->f32[1];
    a.bx32 = c->f32[2];
    a.by32 = c->f32[3];
    a.bz32 = c->f32[4];
    a.hist = c->hist;
    a.jzb = c->jzb;
    a.m_sched = sched ? c->d_sched : nullptr;
    a.diag_m = c->diag_m;
    a.diag_vmax = c->diag_vmax;
    a.diag_charge = c->diag_charge;
    a.sc = c->sc;
    a.trace = c->trace;
    a.trace_cap = g.trace_capacity;
    a.j_begin = 0;
    a.j_end = g.n_xi;
    a.ckpt_every = 0;
    a.ckpt = nullptr;
    a.seg_p = a.seg_g = nullptr;
    a.seg_cap = 0;
    if (replay) {
        a.hist = nullptr;
        a.diag_m = nullptr;
        a.diag_vmax = nullptr;
        a.diag_charge = nullptr;
        a.trace = nullptr;
        a.trace_cap = 0;
    }
    return QS_OK;
}

// After the slice engine: read the device scalars, set the status, fill stats.
static int step_finish(qs_ctx *c, qs_step_stats *stats, double gpu_ms) {
    const qs_config &g = c->cfg;
    DevScalars hs;
    CK(cudaMemcpy(&hs, c->sc, sizeof(hs), cudaMemcpyDeviceToHost), "copy scalars");
    c->have_step = true;
    int status = QS_OK;
    if (hs.err != 0) {
        status = hs.err;
        if (hs.err == QS_ERR_CUDA && hs.err_where == -1)
            fail(c, status, "the slice engine ran without its %d-block thread-block clusters",
                 c->cl_size);
        else
            fail(c, status, "device wait timed out at phase %d", hs.err_where);
    } else if (hs.not_converged) {
        status = fail(c, QS_ERR_NOT_CONVERGED, "a multigrid solve reached %d V-cycles (relres %g)",
                      g.mg_max_vcycles, hs.max_relres);
    } else if (g.max_psi_guard_hits >= 0 && (int64_t)hs.guard_hits > g.max_psi_guard_hits) {
        status = fail(c, QS_ERR_PSI_FLOOR, "1+psi clamped %llu times", hs.guard_hits);
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->slices = hs.slices;
        stats->substeps = hs.slices - g.n_xi;
        stats->pushes = hs.pushes;
        for (int k = 0; k < 3; ++k) stats->vcycles[k] = hs.vcycles[k];
        stats->psi_guard_hits = (int64_t)hs.guard_hits;
        stats->sorts = hs.sorts;
        stats->max_relres = hs.max_relres;
        unsigned long long vb = hs.vmax_all_bits;
        double vm;
        std::memcpy(&vm, &vb, sizeof(vm));
        stats->vmax = vm;
        stats->max_m = hs.max_m;
        stats->status = status;
        stats->gpu_ms = gpu_ms;
    }
    return status;
}

static int step_impl(qs_ctx *c, const qs_beam *beams, int n_beams, const int32_t *sched,
                     qs_step_stats *stats, const double *a2 = nullptr, double *chi = nullptr) {
    if (check_ctx(c)) return QS_ERR_ARG;
    EngineArgs a;
    c->ckpt_valid = false;
    int r = step_prepare(c, beams, n_beams, sched, c->st, a);
    if (r != QS_OK) return r;
    c->last_laser = a2 != nullptr;
    if (a2) {
        a.a2_base = a2;
        a.a2 = c->a2;
        a.pondx = c->pondx;
        a.pondy = c->pondy;
        a.chi = chi;
    }
    const int K = c->cfg.checkpoint_every;
    if (K > 0) {  // plasma checkpoints for a later qs_step3d_adjoint
        const size_t need = (size_t)((c->cfg.n_xi + K - 1) / K) * 4 * c->np;
        if (c->ckpt_count < need) {
            if (c->ckpt) cudaFree(c->ckpt);
            c->ckpt = nullptr;
            c->ckpt_count = 0;
            CK(cudaMalloc(&c->ckpt, need * sizeof(double)), "cudaMalloc checkpoints");
            c->ckpt_count = need;
        }
        a.ckpt_every = K;
        a.ckpt = c->ckpt;
    }
    c->store_valid = false;
    if (K >= c->cfg.n_xi) {
        // keep every slice's state (plasma before its push, 12 grids) for the
        // adjoint if it fits in at most 40 % of the free device memory:
        // room for two sub-steps per base slice on average, and the slots
        // already held are reused
        const size_t nn = (size_t)c->N * c->N;
        const size_t per = 4 * (size_t)c->np + SG_COUNT * nn;
        size_t want = (size_t)c->cfg.n_xi * 2;
        if (c->store_slots < want) {
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            const size_t held = c->store_slots * per * sizeof(double);
            if ((want * per * sizeof(double)) <= (size_t)(0.4 * (double)(fr + held))) {
                if (c->store) cudaFree(c->store);
                c->store = nullptr;
                c->store_slots = 0;
                if (cudaMalloc(&c->store, want * per * sizeof(double)) == cudaSuccess)
                    c->store_slots = want;
                else
                    cudaGetLastError();
            }
        }
        if (c->store_slots > 0) {
            a.seg_p = c->store;
            a.seg_g = c->store + c->store_slots * 4 * (size_t)c->np;
            a.seg_cap = (int)c->store_slots;
        }
    }
    CK(cudaEventRecord(c->ev0, c->st), "event");
    CK(qs_launch_engine(c->st, a, c->engine_blocks, c->engine_smem), "slice engine launch");
    CK(cudaEventRecord(c->ev1, c->st), "event");
    CK(cudaStreamSynchronize(c->st), "slice engine");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    r = step_finish(c, stats, ms);
    if (r == QS_OK && K > 0) {
        c->ckpt_valid = true;
        c->ckpt_every = K;
    }
    if (r == QS_OK && a.seg_p) {
        DevScalars hs;
        CK(cudaMemcpy(&hs, c->sc, sizeof(hs), cudaMemcpyDeviceToHost), "copy scalars");
        if (hs.slices <= (unsigned long long)c->store_slots) {
            c->store_valid = true;
            c->store_n_sub = (int)hs.slices;
        }
    }
    return r;
}

int qs_step3d(qs_ctx *c, const qs_beam *beams, int n_beams, qs_step_stats *stats) {
    return step_impl(c, beams, n_beams, nullptr, stats);
}

int qs_step3d_schedule(qs_ctx *c, const qs_beam *beams, int n_beams, const int32_t *m_schedule,
                       qs_step_stats *stats) {
    if (!m_schedule) return fail(c, QS_ERR_ARG, "m_schedule is NULL");
    return step_impl(c, beams, n_beams, m_schedule, stats);
}

int qs_step3d_laser(qs_ctx *c, const qs_beam *beams, int n_beams, const double *a2, double *chi,
                    qs_step_stats *stats) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!a2) return fail(c, QS_ERR_ARG, "a2 is NULL");
    return step_impl(c, beams, n_beams, nullptr, stats, a2, chi);
}

int qs_laser_step3d(qs_ctx *c, qs_laser *laser, const qs_beam *beams, int n_beams,
                    double *envelope, double tol, int max_cycles, qs_step_stats *stats,
                    int64_t *env_cycles, double *env_relres) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!laser || !envelope) return fail(c, QS_ERR_ARG, "NULL laser or envelope");
    const qs_config &g = c->cfg;
    int ln = 0, lxi = 0;
    double lw = 0.0, ldxi = 0.0;
    qs_laser_shape(laser, &ln, &lw, &lxi, &ldxi);
    const double dxi0 = (g.xi_max - g.xi_min) / g.n_xi;
    if (ln != c->N || lxi != g.n_xi || std::fabs(lw - (g.x_max - g.x_min)) > 1e-12 * lw ||
        std::fabs(ldxi - dxi0) > 1e-12 * dxi0)
        return fail(c, QS_ERR_ARG, "the envelope's cells, box, slices or slice spacing "
                                   "differ from the context's");
    const size_t n = (size_t)g.n_xi * c->N * c->N;
    if (!c->a2_all) {
        CK(cudaMalloc(&c->a2_all, n * sizeof(double)), "cudaMalloc |A|^2");
        if (cudaMalloc(&c->chi_all, n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->a2_all);
            c->a2_all = nullptr;
            return fail(c, QS_ERR_OOM, "cudaMalloc chi");
        }
    }
    CK(qs_launch_abs2(c->st, envelope, c->a2_all, (int64_t)n), "|A|^2");
    int r = step_impl(c, beams, n_beams, nullptr, stats, c->a2_all, c->chi_all);
    if (r != QS_OK) return r;  // the step synchronised its stream: chi is complete
    r = qs_laser_advance(laser, c->chi_all, envelope, 1, tol, max_cycles, env_cycles,
                         env_relres);
    if (r != QS_OK) return fail(c, r, "envelope advance: %s", qs_strerror(r));
    return QS_OK;
}

int qs_step3d_batched(qs_ctx **ctxs, int n, const qs_beam *const *beams, const int *n_beams,
                      int team_blocks, qs_step_stats *stats) {
    if (n < 1 || !ctxs) return QS_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return QS_ERR_ARG;
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return fail(ctxs[0], QS_ERR_ARG, "context %d repeated", i);
        if (ctxs[i]->cfg.precision != ctxs[0]->cfg.precision || ctxs[i]->dev != ctxs[0]->dev)
            return fail(ctxs[0], QS_ERR_ARG, "batched contexts need one precision and device");
    }
    qs_ctx *c = ctxs[0];
    if (team_blocks < 0) return fail(c, QS_ERR_ARG, "team_blocks must be >= 0");
    cudaStream_t st = c->st;
    // the device queue hands out instances in list order: largest first
    // (cells x particles x slices), so that the last ones to start are short
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto cost = [&](int i) {
        const qs_ctx *x = ctxs[i];
        return ((double)x->N * x->N + (double)x->np) * (double)x->cfg.n_xi;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<EngineArgs> list(n);
    size_t smem = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        ctxs[i]->ckpt_valid = false;  // the batched step stores no checkpoints
        ctxs[i]->store_valid = false;
        const int r = step_prepare(ctxs[i], beams ? beams[i] : nullptr, n_beams ? n_beams[i] : 0,
                                   nullptr, st, list[k]);
        if (r != QS_OK) {
            if (i > 0) fail(c, r, "context %d: %s", i, ctxs[i]->msg);
            return r;
        }
        list[k].trace = nullptr;
        list[k].trace_cap = 0;
        list[k].cl_size = 1;  // the batched launch has no clusters
        if (ctxs[i]->engine_smem > smem) smem = ctxs[i]->engine_smem;
    }
    int total = 0;
    if (qs_engine_batched_max_blocks(c->dev, c->cfg.precision, smem, &total) != 0 || total < 1)
        return fail(c, QS_ERR_CUDA, "batched slice engine cannot be made resident");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev), "attr");
    if (total > sms) total = sms;
    int team = team_blocks > 0 ? team_blocks : total / n;
    if (team < 1) team = 1;
    if (team > total) team = total;
    int teams = total / team;
    if (teams > QS_MAX_TEAMS) teams = QS_MAX_TEAMS;
    void *dbuf = nullptr;
    const size_t list_bytes = (n * sizeof(EngineArgs) + 255) & ~(size_t)255;
    CK(cudaMallocAsync(&dbuf, list_bytes + sizeof(BatchState), st), "cudaMallocAsync");
    EngineArgs *dlist = static_cast<EngineArgs *>(dbuf);
    BatchState *bs = reinterpret_cast<BatchState *>(static_cast<char *>(dbuf) + list_bytes);
    cudaError_t e = cudaMemcpyAsync(dlist, list.data(), n * sizeof(EngineArgs),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bs, 0, sizeof(BatchState), st);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev0, st);
    if (e == cudaSuccess)
        e = qs_launch_engine_batched(st, dlist, n, c->cfg.precision, team, teams, bs, smem);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, st);
    cudaFreeAsync(dbuf, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched slice engine");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "batched slice engine");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    int status = QS_OK;
    for (int i = 0; i < n; ++i) {
        const int r = step_finish(ctxs[i], stats ? &stats[i] : nullptr, ms);
        if (r != QS_OK && status == QS_OK) status = r;
    }
    return status;
}

// ---------------------------------------------------------------------------
// adjoint of one 3D step (checkpointed reverse slice loop)
// ---------------------------------------------------------------------------
namespace {

// device buffers of one adjoint call, freed on every return path
struct DevBufs {
    std::vector<void *> list;
    ~DevBufs() {
        for (void *p : list) cudaFree(p);
    }
};

int read_scalars(qs_ctx *c, DevScalars &hs, const char *what) {
    CK(cudaMemcpy(&hs, c->sc, sizeof(hs), cudaMemcpyDeviceToHost), "copy scalars");
    if (hs.err != 0) return fail(c, hs.err, "%s: device wait timed out at phase %d", what,
                                 hs.err_where);
    if (hs.not_converged)
        return fail(c, QS_ERR_NOT_CONVERGED, "%s: a multigrid solve reached %d V-cycles", what,
                    c->cfg.mg_max_vcycles);
    return QS_OK;
}

// plasma state of checkpoint k into the working particle arrays
int restore_checkpoint(qs_ctx *c, const double *ck) {
    const int64_t np = c->np;
    const size_t bd = np * sizeof(double);
    CK(cudaMemcpyAsync(c->x, ck, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    CK(cudaMemcpyAsync(c->y, ck + np, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    if (c->cfg.precision == QS_FP32_REFINED) {
        CK(qs_launch_convert(c->st, ck + 2 * np, c->px32, np), "convert");
        CK(qs_launch_convert(c->st, ck + 3 * np, c->py32, np), "convert");
    } else {
        CK(cudaMemcpyAsync(c->px, ck + 2 * np, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
        CK(cudaMemcpyAsync(c->py, ck + 3 * np, bd, cudaMemcpyDeviceToDevice, c->st), "copy");
    }
    return QS_OK;
}

}  // namespace

int qs_step3d_adjoint(qs_ctx *c, const double *d_hist, int checkpoint_every, double *d_jzb,
                      double *d_w, double *d_nion, qs_step_stats *stats) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    if (c->last_laser)
        return fail(c, QS_ERR_STATE, "the adjoint does not cover the laser terms of the last step");
    if (!d_jzb || !d_w || !d_nion) return fail(c, QS_ERR_ARG, "NULL output array");
    if (checkpoint_every < 0) return fail(c, QS_ERR_ARG, "checkpoint_every must be >= 0");
    const qs_config &g = c->cfg;
    const bool stored = c->ckpt_valid && (checkpoint_every == 0 ||
                                          checkpoint_every == c->ckpt_every);
    const int K = stored ? c->ckpt_every : (checkpoint_every > 0 ? checkpoint_every : 32);
    const int nxi = g.n_xi;
    const int64_t np = c->np;
    const size_t nn = (size_t)c->N * c->N;
    cudaStream_t st = c->st;
    // the forward schedule, replayed exactly
    std::vector<int32_t> sched(nxi);
    CK(cudaMemcpy(sched.data(), c->diag_m, nxi * sizeof(int32_t), cudaMemcpyDeviceToHost),
       "copy schedule");
    for (int j = 0; j < nxi; ++j)
        if (sched[j] < 1 || sched[j] > g.refine_k)
            return fail(c, QS_ERR_STATE, "the forward step did not complete");
    int blocks = 0, sms = 0;
    if (qs_adjoint_max_blocks(c->dev, g.precision, c->engine_smem, &blocks) != 0 || blocks < 1)
        return fail(c, QS_ERR_CUDA, "adjoint engine cannot be made resident");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev), "attr");
    if (blocks > sms) blocks = sms;
    const int nseg = (nxi + K - 1) / K;
    int max_sub = 0;
    for (int k = 0; k < nseg; ++k) {
        int n_sub = 0;
        for (int j = k * K; j < std::min(nxi, (k + 1) * K); ++j)
            n_sub += (j == nxi - 1) ? 1 : sched[j];
        max_sub = std::max(max_sub, n_sub);
    }
    // every slice kept by the forward step: no checkpoints, no recompute
    const bool whole = stored && nseg == 1 && c->store_valid && c->store_n_sub == max_sub;
    DevBufs B;
    double *ckpt = nullptr, *seg_p = nullptr, *seg_g = nullptr, *lam = nullptr, *grd = nullptr;
    if (stored) ckpt = c->ckpt;
    else AL(B.list, ckpt, (size_t)nseg * 4 * np);
    if (whole) {
        seg_p = c->store;
        seg_g = c->store + c->store_slots * 4 * (size_t)np;
    } else {
        AL(B.list, seg_p, (size_t)max_sub * 4 * np);
        AL(B.list, seg_g, (size_t)max_sub * SG_COUNT * nn);
    }
    AL(B.list, lam, (size_t)4 * np);
    AL(B.list, grd, (size_t)20 * nn);
    float ms_total = 0.f;
    // forward replay that stores the checkpoints (unless the step stored them)
    EngineArgs a;
    int r;
    if (!stored) {
        r = step_prepare(c, nullptr, 0, sched.data(), st, a, true);
        if (r != QS_OK) return r;
        a.ckpt_every = K;
        a.ckpt = ckpt;
        CK(cudaEventRecord(c->ev0, st), "event");
        CK(qs_launch_engine(st, a, c->engine_blocks, c->engine_smem), "slice engine launch");
        CK(cudaEventRecord(c->ev1, st), "event");
        CK(cudaStreamSynchronize(st), "checkpoint pass");
    }
    if (!stored) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        ms_total += ms;
        DevScalars hs;
        r = read_scalars(c, hs, "checkpoint pass");
        if (r != QS_OK) return r;
    }
    // adjoint state
    CK(cudaMemsetAsync(lam, 0, (size_t)4 * np * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(grd, 0, (size_t)20 * nn * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(d_w, 0, np * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(d_jzb, 0, (size_t)nxi * nn * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(d_nion, 0, nn * sizeof(double), st), "memset");
    AdjArgs d;
    std::memset(&d, 0, sizeof(d));
    d.lx = lam;
    d.ly = lam + np;
    d.lpx = lam + 2 * np;
    d.lpy = lam + 3 * np;
    d.lw = d_w;
    double **gp[] = {&d.g_psi, &d.g_ez, &d.g_bz, &d.g_bx, &d.g_by, &d.g_dpx, &d.g_dpy,
                     &d.g_jx,  &d.g_jy, &d.g_txx, &d.g_txy, &d.g_tyy, &d.g_G, &d.g_n,
                     &d.mu_x,  &d.mu_y, &d.nu_ez, &d.nu_bz, &d.nu_psi, &d.f_nu_psi};
    for (int k = 0; k < 20; ++k) *gp[k] = grd + (size_t)k * nn;
    d.d_hist = d_hist;
    d.d_jzb = d_jzb;
    d.d_nion = d_nion;
    int64_t slices = 0, vc[3] = {0, 0, 0};
    for (int k = nseg - 1; k >= 0; --k) {
        const int j0 = k * K, j1 = std::min(nxi, j0 + K);
        int n_sub = 0;
        for (int j = j0; j < j1; ++j) n_sub += (j == nxi - 1) ? 1 : sched[j];
        // recompute the segment from its checkpoint, storing every slice
        r = step_prepare(c, nullptr, 0, sched.data(), st, a, true);
        if (r != QS_OK) return r;
        a.j_begin = j0;
        a.j_end = j1;
        a.seg_p = seg_p;
        a.seg_g = seg_g;
        a.seg_cap = n_sub;
        DevScalars hs;
        CK(cudaEventRecord(c->ev0, st), "event");
        if (!whole) {
            r = restore_checkpoint(c, ckpt + (size_t)k * 4 * np);
            if (r != QS_OK) return r;
            CK(qs_launch_engine(st, a, c->engine_blocks, c->engine_smem),
               "slice engine launch");
            CK(cudaStreamSynchronize(st), "segment recompute");
            r = read_scalars(c, hs, "segment recompute");
            if (r != QS_OK) return r;
        }
        // the reverse slice loop over the segment
        CK(cudaMemsetAsync(c->sc, 0, sizeof(DevScalars), st), "memset");
        d.j0 = j0;
        d.j1 = j1;
        d.n_sub = n_sub;
        EngineArgs ra = a;
        ra.cl_size = 1;  // the adjoint launch has no clusters: grid-wide solves
        CK(qs_launch_adjoint(st, ra, d, blocks, c->engine_smem), "adjoint engine launch");
        CK(cudaEventRecord(c->ev1, st), "event");
        CK(cudaStreamSynchronize(st), "adjoint engine");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        ms_total += ms;
        r = read_scalars(c, hs, "adjoint engine");
        if (r != QS_OK) return r;
        slices += hs.slices;
        for (int q = 0; q < 3; ++q) vc[q] += hs.vcycles[q];
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->slices = slices;
        stats->substeps = slices - nxi;
        for (int q = 0; q < 3; ++q) stats->vcycles[q] = vc[q];
        stats->status = QS_OK;
        stats->gpu_ms = ms_total;
    }
    return QS_OK;
}

int qs_beam_gain(qs_ctx *c, const qs_beam *beam, double dt, double *gain, double *d_hist) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    if (!beam || !gain || beam->n < 1 || !beam->x || !beam->y || !beam->xi || !beam->px ||
        !beam->py || !beam->pz)
        return fail(c, QS_ERR_ARG, "bad bunch");
    const qs_config &g = c->cfg;
    const double dxi0 = (g.xi_max - g.xi_min) / g.n_xi;
    double *dsum = nullptr;
    CK(cudaMallocAsync(&dsum, sizeof(double), c->st), "cudaMallocAsync");
    cudaError_t e = cudaMemsetAsync(dsum, 0, sizeof(double), c->st);
    if (e == cudaSuccess)
        e = qs_launch_beam_gain(c->st, *beam, c->N, g.x_min, g.x_max, g.y_min, g.y_max, c->h,
                                g.n_xi, g.xi_min, dxi0, c->hist, dt, 1.0 / (double)beam->n,
                                dsum, d_hist);
    double sum = 0.0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&sum, dsum, sizeof(double), cudaMemcpyDeviceToHost, c->st);
    cudaFreeAsync(dsum, c->st);
    const cudaError_t e2 = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "bunch gain");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "bunch gain");
    *gain = sum / (double)beam->n;
    return QS_OK;
}

int qs_beam_deposit_adjoint(qs_ctx *c, const qs_beam *beam, const double *d_jzb, double *d_x,
                            double *d_y, double *d_xi, double *d_w) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    if (!beam || beam->n < 0 || !d_jzb ||
        (beam->n > 0 && (!beam->x || !beam->y || !beam->xi || !beam->px || !beam->py ||
                         !beam->pz || !beam->w || !d_x || !d_y || !d_xi || !d_w)))
        return fail(c, QS_ERR_ARG, "bad bunch or output arrays");
    const qs_config &g = c->cfg;
    const double dxi0 = (g.xi_max - g.xi_min) / g.n_xi;
    CK(qs_launch_beam_deposit_adjoint(c->st, *beam, c->N, g.x_min, g.x_max, g.y_min, g.y_max,
                                      c->h, g.n_xi, g.xi_min, dxi0, d_jzb, d_x, d_y, d_xi, d_w),
       "bunch deposit adjoint");
    return QS_OK;
}

int qs_profile_adjoint(qs_ctx *c, const double *d_w, const double *d_nion, int n_coef,
                       double r_max, double *d_table) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_plasma) return fail(c, QS_ERR_STATE, "qs_init_plasma has not been called");
    if (!d_w || !d_nion || !d_table || n_coef < 1 || n_coef > 4096 || !(r_max > 0.0))
        return fail(c, QS_ERR_ARG, "bad profile-adjoint arguments (n_coef in [1, 4096])");
    const qs_config &g = c->cfg;
    double *dt = nullptr;
    CK(cudaMallocAsync(&dt, n_coef * sizeof(double), c->st), "cudaMallocAsync");
    cudaError_t e = cudaMemsetAsync(dt, 0, n_coef * sizeof(double), c->st);
    if (e == cudaSuccess)
        e = qs_launch_profile_adjoint(c->st, c->N, c->ppc, g.x_min, g.y_min, c->h, n_coef,
                                      r_max, d_w, d_nion, dt);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_table, dt, n_coef * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    cudaFreeAsync(dt, c->st);
    const cudaError_t e2 = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "profile adjoint");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "profile adjoint");
    return QS_OK;
}

int qs_push_beam(qs_ctx *c, qs_beam *beams, int n_beams, double dt) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    if (n_beams < 0 || (n_beams > 0 && !beams)) return fail(c, QS_ERR_ARG, "bad beam list");
    const qs_config &g = c->cfg;
    const double dxi0 = (g.xi_max - g.xi_min) / g.n_xi;
    for (int b = 0; b < n_beams; ++b) {
        const qs_beam &bm = beams[b];
        if (bm.n < 0) return fail(c, QS_ERR_ARG, "beam %d: negative count", b);
        if (bm.n > 0 && (!bm.x || !bm.y || !bm.xi || !bm.px || !bm.py || !bm.pz))
            return fail(c, QS_ERR_ARG, "beam %d: NULL array", b);
        CK(qs_launch_beam_push(c->st, bm, c->N, g.x_min, g.x_max, g.y_min, g.y_max, c->h, g.n_xi,
                               g.xi_min, dxi0, c->hist, dt),
           "beam push");
    }
    return QS_OK;
}

int qs_push_beam_dla(qs_ctx *c, qs_beam *beams, int n_beams, double dt, const double *env_n,
                     const double *env_np1, double k0, int n_sub) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    if (n_beams < 0 || (n_beams > 0 && !beams)) return fail(c, QS_ERR_ARG, "bad beam list");
    if (!env_n || !env_np1) return fail(c, QS_ERR_ARG, "NULL envelope");
    if (!(dt > 0.0) || !(k0 > 0.0) || n_sub < 1)
        return fail(c, QS_ERR_ARG, "need dt > 0, k0 > 0 and n_sub >= 1");
    const qs_config &g = c->cfg;
    const double dxi0 = (g.xi_max - g.xi_min) / g.n_xi;
    for (int b = 0; b < n_beams; ++b) {
        const qs_beam &bm = beams[b];
        if (bm.n < 0) return fail(c, QS_ERR_ARG, "beam %d: negative count", b);
        if (bm.n > 0 && (!bm.x || !bm.y || !bm.xi || !bm.px || !bm.py || !bm.pz))
            return fail(c, QS_ERR_ARG, "beam %d: NULL array", b);
        CK(qs_launch_beam_push_dla(c->st, bm, c->N, g.x_min, g.x_max, g.y_min, g.y_max, c->h,
                                   g.n_xi, g.xi_min, dxi0, c->hist, env_n, env_np1, k0, dt,
                                   n_sub),
           "beam push (laser fields)");
    }
    return QS_OK;
}

int qs_fields(qs_ctx *c, int field_mask, int slice_begin, int slice_end, double *out,
              int out_on_device) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    const qs_config &g = c->cfg;
    if (!out || (field_mask & ~63) || field_mask == 0 || slice_begin < 0 ||
        slice_end > g.n_xi || slice_begin >= slice_end)
        return fail(c, QS_ERR_ARG, "bad field mask or slice range");
    const size_t nn = (size_t)c->N * c->N;
    const size_t cnt = (size_t)(slice_end - slice_begin) * nn;
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t off = 0;
    for (int f = 0; f < 6; ++f) {
        if (!(field_mask & (1 << f))) continue;
        const double *src = (f < 5) ? c->hist + (size_t)f * g.n_xi * nn + slice_begin * nn
                                    : c->jzb + slice_begin * nn;
        CK(cudaMemcpyAsync(out + off, src, cnt * sizeof(double), kind, c->st), "copy fields");
        off += cnt;
    }
    if (!out_on_device) CK(cudaStreamSynchronize(c->st), "sync");
    return QS_OK;
}

int qs_slice_diagnostics(qs_ctx *c, int32_t *m, double *vmax, double *charge) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    const int n = c->cfg.n_xi;
    if (m) CK(cudaMemcpyAsync(m, c->diag_m, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st), "copy");
    if (vmax) CK(cudaMemcpyAsync(vmax, c->diag_vmax, n * sizeof(double), cudaMemcpyDeviceToHost, c->st), "copy");
    if (charge) CK(cudaMemcpyAsync(charge, c->diag_charge, n * sizeof(double), cudaMemcpyDeviceToHost, c->st), "copy");
    CK(cudaStreamSynchronize(c->st), "sync");
    return QS_OK;
}

int64_t qs_plasma_count(const qs_ctx *c) { return (c && c->have_plasma) ? c->np : 0; }

int qs_get_plasma(qs_ctx *c, double *x, double *y, double *px, double *py, double *w,
                  int32_t *id) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_plasma) return fail(c, QS_ERR_STATE, "qs_init_plasma has not been called");
    const size_t bd = c->np * sizeof(double);
    const cudaMemcpyKind k = cudaMemcpyDeviceToHost;
    if (c->have_step && c->cfg.precision == QS_FP32_REFINED) {  // float32 working copy
        CK(qs_launch_widen(c->st, c->px32, c->px, c->np), "widen");
        CK(qs_launch_widen(c->st, c->py32, c->py, c->np), "widen");
        CK(qs_launch_widen(c->st, c->w32, c->w, c->np), "widen");
    }
    if (x) CK(cudaMemcpyAsync(x, c->x, bd, k, c->st), "copy");
    if (y) CK(cudaMemcpyAsync(y, c->y, bd, k, c->st), "copy");
    if (px) CK(cudaMemcpyAsync(px, c->px, bd, k, c->st), "copy");
    if (py) CK(cudaMemcpyAsync(py, c->py, bd, k, c->st), "copy");
    if (w) CK(cudaMemcpyAsync(w, c->w, bd, k, c->st), "copy");
    if (id) CK(cudaMemcpyAsync(id, c->id, c->np * sizeof(int32_t), k, c->st), "copy");
    CK(cudaStreamSynchronize(c->st), "sync");
    return QS_OK;
}

int qs_cell_sort(qs_ctx *c, const double *x, const double *y, const int32_t *id, int64_t n,
                 int32_t *cell, int32_t *count, int32_t *offset, int32_t *perm) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (n < 0 || n > (int64_t)0x7fffffff || !count || !offset ||
        (n > 0 && (!x || !y || !id || !cell || !perm)))
        return fail(c, QS_ERR_ARG, "bad cell-sort arguments");
    const qs_config &g = c->cfg;
    CK(qs_launch_cell_sort(c->st, x, y, id, n, c->N, g.x_min, g.y_min, c->h, cell, count, offset,
                           c->s_cursor, perm),
       "cell sort");
    CK(cudaStreamSynchronize(c->st), "cell sort");
    return QS_OK;
}

int qs_phase_trace(qs_ctx *c, int32_t *where, int64_t *t_ns, int cap) {
    if (check_ctx(c)) return QS_ERR_ARG;
    if (!c->have_step) return fail(c, QS_ERR_STATE, "qs_step3d has not been run");
    if (!c->trace || cap < 0) return 0;
    DevScalars hs;
    CK(cudaMemcpy(&hs, c->sc, sizeof(hs), cudaMemcpyDeviceToHost), "copy scalars");
    long long n = (long long)hs.trace_n;
    if (n > cap) n = cap;
    std::vector<int64_t> buf(2 * (size_t)n);
    if (n > 0)
        CK(cudaMemcpy(buf.data(), c->trace, 2 * n * sizeof(int64_t), cudaMemcpyDeviceToHost),
           "copy trace");
    for (long long k = 0; k < n; ++k) {
        if (where) where[k] = (int32_t)buf[2 * k];
        if (t_ns) t_ns[k] = buf[2 * k + 1];
    }
    return (int)n;
}

const char *qs_strerror(int status) {
    switch (status) {
        case QS_OK: return "ok";
        case QS_ERR_ARG: return "invalid argument";
        case QS_ERR_CUDA: return "CUDA error";
        case QS_ERR_OOM: return "out of device memory";
        case QS_ERR_NOT_CONVERGED: return "multigrid did not converge";
        case QS_ERR_PSI_FLOOR: return "1+psi fell below psi_floor too often";
        case QS_ERR_STATE: return "call out of order";
        case QS_ERR_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *qs_last_error(const qs_ctx *c) { return c ? c->msg : ""; }

}  // extern "C"
