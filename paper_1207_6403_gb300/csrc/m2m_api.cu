// C-ABI of libm2m.so: context, tables, launch sequencing of the M2M step.
//
// The step sequence on the caller's stream (Section 2 of the paper; the
// order is push, scatter, residual, weight update, priors):
//
//   k_pass   [pending update at x_t] + push x_t -> x_{t+1} + scatter w_t
//            at x_{t+1} + S, sum w of w_t      (+ (E, L_z) range if priors due)
//   k_residual  y, Delta, Delta~, coef, chi^2; the record of step t+1 is
//               written by the next pass (or k_record when none follows)
//   -> the update w_t -> w_{t+1} (needs coef of this residual) is carried
//      into the next k_pass, so each particle is read and written once per
//      step; a call ends with an update-only pass so the arrays hold w_{t+1}
//      (lazy updates: left to the next call, or to m2m_finish_update);
//   every `period` steps: update + prior cells pass, cell means, gather;
//   self-consistent SH potential: side sums and node tables every period.
// Kernels are launched with programmatic dependent launch where one kernel
// feeds the next; batches of models run one launch per stage for all models
// from device argument arrays, captured as CUDA graphs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "m2m.h"
#define M2M_COMMON_KERNELS
#include "m2m_kernels.cuh"
#include "m2m_analysis.cuh"
#include "m2m_steps.cuh"

using namespace m2m;
static_assert(SH_ROW == M2M_SH_ROW, "node table row");

namespace {

std::string g_init_error;

struct LaunchShape {
    void *fn;
    int nt;
};

}  // namespace

struct m2m_ctx {
    int prec;
    long long n;
    void *x, *y, *z, *vx, *vy, *vz;
    double *w, *what;
    cudaStream_t st;
    int nsm;
    int threads, bps_req;
    int nsets, nobs, npot;
    SetDev sets[MAXSETS];
    PotDev pot[MAXPOT];
    m2m_params par;
    m2m_prior_desc prior;
    int ncells;
    int edge_len, gh_len;
    void *d_edges, *d_gh;
    int *d_lut = nullptr;            // aperture lookup tables of the LUT sets
    short *d_pmap = nullptr;         // layout 1, aligned grids: set 1's cell of each pixel of set 0
    void *d_psf = nullptr;           // seeing quantile tables (state precision)
    long long epoch = 0;             // pushes the positions have had since m2m_init
    double *d_Y, *d_sigma, *d_isig, *d_Dt, *d_y, *d_Delta, *d_coef_d;
    void *d_coef_r;
    void *d_slots;
    unsigned long long *d_y_acc;   // FP32C exact observable totals (int64)
    int slot_cap;
    double *d_stat_slots, *d_chi_slots;   // stats: two halves of 2*slot_cap doubles (by stat_par)
    unsigned *d_ticket;
    int stat_par;        // half of d_stat_slots the next pass with F_STATS writes
    int stat_prev_nblk;  // blocks of the last pass with F_STATS (its half: stat_par ^ 1)
    // record of the last step, left to the next pass by its residual
    bool rec_pending;
    long long rec_step;
    int rec_chi_nblk, rec_stat_par, rec_stat_nblk;
    unsigned long long *d_rec_ticket;
    unsigned long long rec_base;
    m2m_record *d_ring, *d_last;
    int *d_err;
    void *d_mm_slots;
    int mm_nblocks;
    int *d_cell_ids;
    void *d_cell_acc;
    unsigned *d_cell_cnt;
    double *d_cell_mean;
    int fx_shift;
    double fx_q;
    int cell_shift;      // FP32C prior-cell sums: weight * 2^cell_shift (2^-60 of the initial total)
    long long t;
    bool pending;
    bool lazy_update = false;        // m2m_step leaves the last update pending
    int last_grid;       // grid of the last scatter pass (slots to reduce)
    int layout;          // compiled observable layout of the pass kernel
    int cache_bits;      // bits of the packed per-particle cell cache
    unsigned *d_cell_cache;
    float *d_lnwhat;     // FP32C: ln w_hat per particle, refreshed at init and at every prior recompute
    bool cache_valid;    // cell cache holds the cells of the current positions
    bool pipe;           // use the bulk-copy pipelined pass where it applies
    int fx_atomic;       // FP32C histogram flush: global integer atomics (1) or slots (0)
    // self-consistent expansion potential (kind M2M_POT_SH, or M2M_POT_SH_TRI
    // or M2M_POT_SH_FULL with sh_basis 1 or 2): sh_row table values per node
    bool sh_on;
    int sh_basis;        // 0 axisymmetric, 1 triaxial, 2 full (l <= 4)
    int sh_K, sh_period, sh_row;
    double sh_rmin, sh_rmax;
    int sh_gmode;
    float sh_ga, sh_gb;
    void *d_sh_e2, *d_sh_rn, *d_sh_irn, *d_sh_tab;
    void *d_facc;        // force at the current positions ([3][n], state precision)
    bool facc_valid;     // d_facc holds it for the current positions and node table
    bool facc_off;       // m2m_set_force_cache(0): evaluate the force twice per push
    double *d_sh_rnd;
    unsigned long long *d_sh_sum;
    // persistent multi-step launches (FP32C compiled layouts)
    bool persist = true;             // use them where they apply
    unsigned long long *d_bar = nullptr;   // grid-barrier arrivals
    double *d_st2 = nullptr, *d_chi2 = nullptr;   // per-block partials by step parity
    long long wait_ns = 2000000000ll;      // limit of one grid-barrier wait
    int test_stall = 0;              // test only: the next launch's block 0 skips its first arrival
    long long test_wait_ns = 0;      //   and its barrier waits are limited to this
    // particle shards (m2m_shard_*): this context holds one shard of a model
    bool shard = false;
    bool shard_push = false;         // the last shard scatter pushed
    bool shard_due = false;          // a prior recompute is due after it
    // timing of the library's launches
    bool timing;
    long long kernels_total;
    struct Ev { int kind; cudaEvent_t a, b; long long steps; };
    std::vector<Ev> evs;
    std::vector<cudaEvent_t> ev_free;
    std::string err;
};

namespace {

int set_err(m2m_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_init_error = buf;
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_err(ctx, M2M_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

cudaEvent_t ev_get(m2m_ctx *c) {
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets one launch: kernel counter always, events while timing is on.
struct LaunchTimer {
    m2m_ctx *c;
    int kind;
    long long steps;
    cudaEvent_t a = nullptr;
    LaunchTimer(m2m_ctx *c_, int kind_, long long steps_ = -1) : c(c_), kind(kind_), steps(steps_) {
        c->kernels_total++;
        if (c->timing && (a = ev_get(c))) cudaEventRecord(a, c->st);
    }
    ~LaunchTimer() {
        if (!a) return;
        cudaEvent_t b = ev_get(c);
        if (!b) { c->ev_free.push_back(a); return; }
        cudaEventRecord(b, c->st);
        const long long ns = steps >= 0 ? steps : (kind == M2M_TK_STEP_UPD || kind == M2M_TK_STEP ? 1 : 0);
        c->evs.push_back({kind, a, b, ns});
    }
};

int pass_kind(int flags) {
    if ((flags & F_PUSH) && (flags & F_SCAT)) return (flags & F_UPD) ? M2M_TK_STEP_UPD : M2M_TK_STEP;
    if (flags & F_CELLS) return M2M_TK_PRIOR;
    if (flags == F_UPD) return M2M_TK_UPDATE;
    return M2M_TK_OTHER;
}

float ceil_float(double e) {
    float f = (float)e;
    if ((double)f < e) f = nextafterf(f, INFINITY);
    return f;
}

// Index guess for an edge table: linear or logarithmic if either predicts
// every edge within half a cell, else bisection.
void guess_params(const double *e, int nb, int *mode, float *ga, float *gb) {
    double span = e[nb] - e[0];
    bool lin_ok = span > 0 && isfinite(span);
    if (lin_ok) {
        double a = nb / span, b = -e[0] * a;
        for (int k = 0; k <= nb && lin_ok; ++k)
            if (fabs(a * e[k] + b - k) > 0.01) lin_ok = false;
        if (lin_ok) { *mode = G_LIN; *ga = (float)a; *gb = (float)b; return; }
    }
    if (e[0] > 0) {
        double l0 = log2(e[0]), l1 = log2(e[nb]);
        bool ok = l1 > l0;
        double a = ok ? nb / (l1 - l0) : 0, b = -l0 * a;
        for (int k = 0; k <= nb && ok; ++k)
            if (fabs(a * log2(e[k]) + b - k) > 0.01) ok = false;
        if (ok) { *mode = G_LOG; *ga = (float)a; *gb = (float)b; return; }
    }
    *mode = G_BIS; *ga = 0.f; *gb = 0.f;
}

size_t pass_smem(const m2m_ctx *c, int flags) {
    return pass_smem_bytes(c->prec == M2M_FP32C, c->layout, flags, c->nobs, c->edge_len, c->gh_len,
                           c->sh_on ? c->sh_row * c->sh_K : 0, c->prior.nE, c->prior.nL, c->ncells,
                           c->layout == 1 ? c->sets[1].pmap_len : 0);
}

// Pixels of grid set g0 -> cell of grid set g1, when every edge of g1 is an
// edge of g0 as the floats the cells are decided against (the smallest
// float >= each double edge) and g1's range lies within g0's: then a float
// coordinate's g1 cell is a function of its g0 pixel, and the table gives
// it (-1 outside g1).  Empty when the grids are not so aligned.
std::vector<short> aligned_pixel_map(const SetDev &g0, const SetDev &g1, const std::vector<double> &edges) {
    std::vector<short> none;
    if ((long long)g1.nx * g1.ny >= 32767) return none;
    std::vector<int> ax_of[2];
    for (int ax = 0; ax < 2; ++ax) {
        const int n0 = ax ? g0.ny : g0.nx, n1 = ax ? g1.ny : g1.nx;
        const double *e0 = edges.data() + (ax ? g0.ey_off : g0.ex_off);
        const double *e1 = edges.data() + (ax ? g1.ey_off : g1.ex_off);
        std::vector<float> f0(n0 + 1), f1(n1 + 1);
        for (int k = 0; k <= n0; ++k) f0[k] = ceil_float(e0[k]);
        for (int k = 0; k <= n1; ++k) f1[k] = ceil_float(e1[k]);
        // every g1 edge is a g0 edge: its index in g0
        std::vector<int> at(n1 + 1, -1);
        for (int k = 0, j = 0; k <= n1; ++k) {
            while (j <= n0 && f0[j] < f1[k]) ++j;
            if (j > n0 || f0[j] != f1[k]) return none;
            at[k] = j;
        }
        ax_of[ax].assign(n0, -1);
        for (int k = 0; k < n1; ++k)
            for (int j = at[k]; j < at[k + 1]; ++j) ax_of[ax][j] = k;
    }
    std::vector<short> map((size_t)g0.nx * g0.ny);
    for (int iy = 0; iy < g0.ny; ++iy)
        for (int ix = 0; ix < g0.nx; ++ix) {
            const int a = ax_of[0][ix], b = ax_of[1][iy];
            map[(size_t)iy * g0.nx + ix] = (short)(a >= 0 && b >= 0 ? b * g1.nx + a : -1);
        }
    return map;
}

// The exponent of the fixed-point scale of a sum of weights W: ceil(log2 W),
// with sums within 1e-12 above a power of two taken as that power (a sum of
// N weights 1/N lands a few ulp either side of 1 depending on its order, and
// a context over a whole model and its shards must agree on the scale).
int scale_exp(double W) { return (int)ceil(log2(W * (1.0 - 1e-12))); }

// Compile-time observable layout matching the context's sets (see
// for_each_set); 0 = generic.  Layouts need index guesses good to one cell.
int detect_layout(const m2m_ctx *c) {
    // radial sets need log-uniform edges, grids and lookup tables
    // value-uniform edges
    for (int k = 0; k < c->nsets; ++k) {
        const SetDev &s = c->sets[k];
        const bool two_d = s.geom == M2M_GEOM_GRID || s.geom == M2M_GEOM_LUT;
        if (two_d && (s.gx_mode != G_LIN || s.gy_mode != G_LIN)) return 0;
        if (!two_d && s.gx_mode != G_LOG) return 0;
    }
    if (c->cache_bits > 32) return 0;
    auto is = [&](int k, int g, int q) { return c->sets[k].geom == g && c->sets[k].quant == q; };
    bool seeing = false;
    for (int k = 0; k < c->nsets; ++k) seeing |= c->sets[k].psf_shift != 0;
    if (seeing && !(c->prec == M2M_FP32C && c->nsets == 3 && is(0, M2M_GEOM_GRID, M2M_Q_MASS) &&
                    is(1, M2M_GEOM_LUT, M2M_Q_GH) && is(2, M2M_GEOM_LUT, M2M_Q_GH)))
        return 0;
    if (c->nsets == 2 && is(0, M2M_GEOM_GRID, M2M_Q_MASS) && is(1, M2M_GEOM_GRID, M2M_Q_GH)) return 1;
    if (c->nsets == 2 && is(0, M2M_GEOM_SHELL, M2M_Q_MASS) && is(1, M2M_GEOM_ANNULUS, M2M_Q_GH)) return 2;
    if (c->nsets == 3 && is(0, M2M_GEOM_SHELL, M2M_Q_MASS) && is(1, M2M_GEOM_ANNULUS, M2M_Q_MASS) &&
        is(2, M2M_GEOM_ANNULUS, M2M_Q_VLOS2))
        return 3;
    // lookup-table apertures: compiled for FP32C only (FP64 walks the sets);
    // the one compiled layout that takes seeing
    if (c->prec == M2M_FP32C && c->nsets == 3 && is(0, M2M_GEOM_GRID, M2M_Q_MASS) &&
        is(1, M2M_GEOM_LUT, M2M_Q_GH) && is(2, M2M_GEOM_LUT, M2M_Q_GH))
        return 4;
    return 0;
}

LaunchShape pick_kernel(const m2m_ctx *c) {
    int nt = c->threads;
    if (c->prec == M2M_FP32C) return {pass_kernel_f32(nt, c->layout), nt};
    return {pass_kernel_f64(nt, c->layout), nt};
}

void fill_args(const m2m_ctx *c, PassArgs &a, int flags) {
    memset(&a, 0, sizeof a);
    a.x = c->x; a.y = c->y; a.z = c->z; a.vx = c->vx; a.vy = c->vy; a.vz = c->vz;
    a.w = c->w; a.what = c->what; a.lnwhat = c->d_lnwhat; a.n = c->n; a.flags = flags;
    a.epoch = c->epoch;
    a.nsets = c->nsets; a.nobs = c->nobs; a.npot = c->npot;
    memcpy(a.sets, c->sets, sizeof a.sets);
    memcpy(a.pot, c->pot, sizeof a.pot);
    a.eps_dt = c->par.eps * c->par.dt;
    a.mu = c->par.mu; a.ent_c = c->par.entropy_const;
    a.hdt = 0.5 * c->par.dt; a.dt = c->par.dt;
    a.sin_i = c->par.incl_sin; a.cos_i = c->par.incl_cos;
    a.f_eps_dt = (float)a.eps_dt; a.f_mu = (float)a.mu; a.f_ent_c = (float)a.ent_c;
    a.f_hdt = (float)a.hdt; a.f_dt = (float)a.dt; a.f_sin_i = (float)a.sin_i; a.f_cos_i = (float)a.cos_i;
    a.edge_tab = c->d_edges; a.edge_len = c->edge_len;
    a.gh_tab = c->d_gh; a.gh_len = c->gh_len;
    a.coef = c->d_coef_r;
    a.slots = c->d_slots; a.fx_shift = c->fx_shift; a.y_acc = c->d_y_acc; a.fx_atomic = c->fx_atomic;
    a.cell_shift = c->cell_shift;
    a.stat_slots = c->d_stat_slots + (size_t)2 * c->slot_cap * c->stat_par;
    a.rec_pending = c->rec_pending; a.rec_write_ring = 1; a.rec_step = c->rec_step;
    a.rec_chi = c->d_chi_slots; a.rec_chi_nblk = c->rec_chi_nblk;
    a.rec_stat = c->d_stat_slots + (size_t)2 * c->slot_cap * c->rec_stat_par; a.rec_stat_nblk = c->rec_stat_nblk;
    a.rec_ticket = c->d_rec_ticket; a.rec_base = c->rec_base;
    a.ring = c->d_ring; a.last = c->d_last;
    a.prior_kind = c->prior.kind; a.nE = c->prior.nE; a.nL = c->prior.nL; a.ncells = c->ncells;
    a.pk = c->prior.hernquist_a / c->prior.hernquist_GM;
    a.pgma = c->prior.hernquist_GM * c->prior.hernquist_a;
    a.f_pk = (float)a.pk; a.f_pgma = (float)a.pgma;
    a.mm_slots = c->d_mm_slots; a.mm_nblocks = c->mm_nblocks;
    a.sh_tab = c->sh_on ? c->d_sh_tab : nullptr; a.sh_K = c->sh_K; a.sh_row = c->sh_row;
    a.facc = (c->sh_on && !c->facc_off) ? c->d_facc : nullptr;
    a.facc_read = (flags & F_PUSH) && a.facc && c->facc_valid;
    a.cell_cache = c->d_cell_cache;
    a.cache_read = (flags & F_UPD) && c->cache_valid && c->layout != 0;
    a.cache_write = (flags & F_SCAT) && c->layout != 0;
    a.cell_ids = c->d_cell_ids; a.cell_acc = c->d_cell_acc; a.cell_cnt = c->d_cell_cnt;
    a.err = c->d_err;
}

// A launch that may overlap the end of the preceding kernel of the stream
// (programmatic dependent launch); the pass and residual kernels wait for
// their inputs with griddep_wait.
cudaError_t launch_dependent(const void *fn, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// The potential signature a steady-state kernel is compiled for (PK_ANY:
// the run-time walk over the components).
int potential_signature(const m2m_ctx *c) {
    if (c->npot == 1 && c->pot[0].kind == M2M_POT_HERNQUIST) return PK_HERNQUIST;
    if (c->npot == 1 && c->pot[0].kind == M2M_POT_LOG) return PK_LOG;
    if (c->npot == 1 && c->pot[0].kind == M2M_POT_SH) return PK_SH;
    if (c->npot == 1 && c->pot[0].kind == M2M_POT_SH_TRI) return PK_SH_TRI;
    if (c->npot == 1 && c->pot[0].kind == M2M_POT_SH_FULL) return PK_SH_FULL;
    if (c->npot == 2 && c->pot[0].kind == M2M_POT_HERNQUIST && c->pot[1].kind == M2M_POT_NFW) return PK_HERNQUIST_NFW;
    return PK_ANY;
}

int launch_pass(m2m_ctx *ctx, int flags, int *grid_out = nullptr) {
    PassArgs a;
    fill_args(ctx, a, flags);
    LaunchShape ks = pick_kernel(ctx);
    size_t sm = pass_smem(ctx, flags);
    int occ = 0;
    if (ctx->pipe && ctx->prec == M2M_FP32C && ctx->threads == 1024 && ctx->layout != 0) {
        // block-level bulk-copy pipeline when its stage buffers fit beside the tables
        void *fp = flags == F_STEADY ? pass_kernel_f32_pipe_steady(ctx->layout) : pass_kernel_f32_pipe(ctx->layout);
        size_t smp = sm + (size_t)PIPE_STAGES * Chunk<float, 1024>::BYTES;
        if (fp) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp, 1024, smp));
        if (occ >= 1) { ks = {fp, 1024}; sm = smp; }
    }
    if (occ < 1 && ctx->prec == M2M_FP32C && ctx->threads == 1024) {
        void *f = pass_kernel_f32_compiled(flags, ctx->layout, potential_signature(ctx));
        if (f) ks = {f, 1024};
    }
    if (occ < 1) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ks.fn, ks.nt, sm));
    if (occ < 1) return set_err(ctx, M2M_ERR_ARG, "pass needs %zu B shared memory: does not fit", sm);
    int bps = occ;
    if (ctx->bps_req > 0 && ctx->bps_req < bps) bps = ctx->bps_req;
    long long nch = (ctx->n + (ctx->prec == M2M_FP32C ? 3 : 1)) / (ctx->prec == M2M_FP32C ? 4 : 2);
    long long need = (nch + ks.nt - 1) / ks.nt;
    long long grid = (long long)ctx->nsm * bps;
    if (grid > ctx->slot_cap) grid = ctx->slot_cap;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    void *args[] = {&a};
    {
        LaunchTimer lt(ctx, pass_kind(flags));
        CU(launch_dependent(ks.fn, dim3((unsigned)grid), dim3(ks.nt), args, sm, ctx->st));
    }
    if (flags & F_SCAT) ctx->last_grid = (int)grid;
    if (flags & F_STATS) { ctx->stat_prev_nblk = (int)grid; ctx->stat_par ^= 1; }
    if (a.rec_pending) { ctx->rec_pending = false; ctx->rec_base += (unsigned long long)grid; }
    if (flags & F_MINMAX) ctx->mm_nblocks = (int)grid;
    if (flags & F_SCAT) ctx->cache_valid = ctx->layout != 0;
    else if (flags & F_PUSH) ctx->cache_valid = false;
    if (flags & F_PUSH) ctx->facc_valid = a.facc != nullptr;
    if (flags & F_PUSH) ++ctx->epoch;
    if (grid_out) *grid_out = (int)grid;
    return M2M_OK;
}

// tail 1: the residual's last block writes the step record; 0: the next
// pass (or finish_record) does, from the partials left in place.
int finish_record(m2m_ctx *ctx);

int launch_residual(m2m_ctx *ctx, int mode, long long rec_step, int write_ring, int stat_nblk, int tail = 1) {
    int rc0 = finish_record(ctx);          // its partials are about to be overwritten
    if (rc0) return rc0;
    ResArgs r;
    memset(&r, 0, sizeof r);
    r.slots = ctx->d_slots; r.nblk = ctx->last_grid; r.nobs = ctx->nobs; r.y_acc = ctx->d_y_acc;
    r.fx_atomic = ctx->fx_atomic;
    r.fixed = ctx->prec == M2M_FP32C; r.q = ctx->fx_q;
    r.Y = ctx->d_Y; r.inv_sigma = ctx->d_isig; r.Dt = ctx->d_Dt; r.y = ctx->d_y; r.Delta = ctx->d_Delta;
    r.coef_d = ctx->d_coef_d; r.coef_r = ctx->d_coef_r; r.r_float = ctx->prec == M2M_FP32C;
    r.mode = mode; r.alpha = ctx->par.alpha; r.mu = ctx->par.mu;
    r.stat_slots = ctx->d_stat_slots + (size_t)2 * ctx->slot_cap * (ctx->stat_par ^ 1); r.stat_nblk = stat_nblk;
    r.tail = tail;
    r.chi_slots = ctx->d_chi_slots; r.ticket = ctx->d_ticket;
    r.ring = ctx->d_ring; r.last = ctx->d_last; r.rec_step = rec_step; r.write_ring = write_ring;
    r.err = ctx->d_err;
    const bool direct = r.fixed && r.fx_atomic;
    int nt = direct ? RES_NT_FX : RES_NT;
    int nb = direct ? (ctx->nobs + RES_NT_FX - 1) / RES_NT_FX : (ctx->nobs + 31) / 32;
    void *args[] = {&r};
    ctx->rec_chi_nblk = nb;
    LaunchTimer lt(ctx, M2M_TK_RESIDUAL);
    CU(launch_dependent((void *)k_residual, dim3(nb), dim3(nt), args, 0, ctx->st));
    return M2M_OK;
}

// scatter + residual at the current state
int observe_now(m2m_ctx *ctx, int extra_flags, int mode, long long rec_step, int write_ring) {
    int g = 0;
    int rc = launch_pass(ctx, F_SCAT | F_STATS | extra_flags, &g);
    if (rc) return rc;
    return launch_residual(ctx, mode, rec_step, write_ring, g);
}

int prior_recompute(m2m_ctx *ctx, int pass_flags) {
    // pass_flags: F_UPD to apply a pending update in the same pass
    size_t acc_b = (size_t)ctx->ncells * 8;
    CU(cudaMemsetAsync(ctx->d_cell_acc, 0, acc_b, ctx->st));
    CU(cudaMemsetAsync(ctx->d_cell_cnt, 0, (size_t)ctx->ncells * 4, ctx->st));
    int rc = launch_pass(ctx, F_CELLS | pass_flags);
    if (rc) return rc;
    int nb = (ctx->ncells + 255) / 256;
    {
        LaunchTimer lt(ctx, M2M_TK_PRIOR);
        k_prior_mean<<<nb, 256, 0, ctx->st>>>(ctx->d_cell_acc, ctx->d_cell_cnt, ctx->ncells,
                                              ctx->prec == M2M_FP32C, ldexp(1.0, -ctx->cell_shift),
                                              ctx->d_cell_mean);
        CU(cudaGetLastError());
    }
    int g = ctx->nsm * 8;
    long long need = (ctx->n + 255) / 256;
    if (g > need) g = (int)need;
    {
        LaunchTimer lt(ctx, M2M_TK_PRIOR);
        k_prior_gather<<<g, 256, 0, ctx->st>>>(ctx->d_cell_ids, ctx->d_cell_mean, ctx->what, ctx->d_lnwhat, ctx->n);
        CU(cudaGetLastError());
    }
    return M2M_OK;
}

// The persistent multi-step kernel for this context, or NULL where it does
// not apply (FP64, the run-time set walk, the spherical-harmonic potential,
// the bulk-copy pipeline or per-block histogram slots chosen, a potential
// signature without one, or no room for one block per SM).
void *persistent_kernel(m2m_ctx *ctx, size_t *smem_out, int *grid_out) {
    if (!ctx->persist || ctx->prec != M2M_FP32C || ctx->layout == 0 || ctx->sh_on || ctx->pipe || !ctx->fx_atomic ||
        ctx->threads != 1024)
        return nullptr;
    void *fn = steps_kernel_f32(ctx->layout, potential_signature(ctx));
    if (!fn) return nullptr;
    const size_t sm = pass_smem(ctx, F_STEADY);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 1024, sm) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return nullptr;
    }
    long long grid = ctx->nsm;                       // one block per SM: every block resident
    const long long need = (ctx->n + 1023) / 1024;
    if (grid > need) grid = need;
    if (grid > ctx->slot_cap) grid = ctx->slot_cap;
    *smem_out = sm;
    *grid_out = (int)grid;
    return fn;
}

// m steps in one cooperative launch; the last takes the (E, L_z) range when
// last_range.  Leaves the last step's weight update pending and its record
// written.
int launch_steps(m2m_ctx *ctx, void *fn, size_t sm, int grid, long long m, bool last_range) {
    int rc0 = finish_record(ctx);
    if (rc0) return rc0;
    StepsArgs A;
    memset(&A, 0, sizeof A);
    fill_args(ctx, A.p, F_STEADY);
    A.p.cache_write = 1;
    A.p.rec_pending = 0;
    ResArgs &r = A.r;
    r.nobs = ctx->nobs; r.y_acc = ctx->d_y_acc; r.fx_atomic = 1; r.fixed = 1; r.q = ctx->fx_q;
    r.Y = ctx->d_Y; r.inv_sigma = ctx->d_isig; r.Dt = ctx->d_Dt; r.y = ctx->d_y; r.Delta = ctx->d_Delta;
    r.coef_d = ctx->d_coef_d; r.coef_r = ctx->d_coef_r; r.r_float = 1;
    r.mode = 1; r.alpha = ctx->par.alpha; r.mu = ctx->par.mu;
    r.ring = ctx->d_ring; r.last = ctx->d_last; r.write_ring = 1; r.err = ctx->d_err;
    A.nsteps = m;
    A.t0 = ctx->t;
    A.epoch0 = ctx->epoch;
    A.first_upd = ctx->pending ? 1 : 0;
    A.first_cache = ctx->cache_valid ? 1 : 0;
    A.last_range = last_range ? 1 : 0;
    A.bar = ctx->d_bar;
    A.st2 = ctx->d_st2;
    A.chi2 = ctx->d_chi2;
    A.wait_ns = ctx->test_stall ? ctx->test_wait_ns : ctx->wait_ns;
    A.test_stall = ctx->test_stall;
    ctx->test_stall = 0;
    CU(cudaMemsetAsync(ctx->d_bar, 0, 8, ctx->st));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = ctx->st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {&A};
    {
        LaunchTimer lt(ctx, M2M_TK_STEPS, m);
        CU(cudaLaunchKernelExC(&cfg, fn, args));
    }
    ctx->t += m;
    ctx->epoch += m;
    ctx->pending = true;
    ctx->cache_valid = true;
    ctx->rec_pending = false;
    ctx->last_grid = grid;
    if (last_range) ctx->mm_nblocks = grid;
    return M2M_OK;
}

// Applies a pending weight update with an update-only pass.
int finish_update(m2m_ctx *ctx) {
    if (!ctx->pending) return M2M_OK;
    int rc = launch_pass(ctx, F_UPD);
    if (rc) return rc;
    ctx->pending = false;
    return M2M_OK;
}

// Writes a record still left to a next pass (when no pass follows).
int finish_record(m2m_ctx *ctx) {
    if (!ctx->rec_pending) return M2M_OK;
    LaunchTimer lt(ctx, M2M_TK_RESIDUAL);
    k_record<<<1, 32, 0, ctx->st>>>(ctx->d_chi_slots, ctx->rec_chi_nblk,
                                    ctx->d_stat_slots + (size_t)2 * ctx->slot_cap * ctx->rec_stat_par,
                                    ctx->rec_stat_nblk, ctx->par.mu, ctx->rec_step, 1, ctx->d_ring, ctx->d_last,
                                    ctx->d_err);
    CU(cudaGetLastError());
    ctx->rec_pending = false;
    return M2M_OK;
}

int check_err_word(m2m_ctx *ctx) {
    int h = 0;
    CU(cudaMemcpyAsync(&h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    if (h & ERR_NONFINITE) return set_err(ctx, M2M_ERR_NONFINITE, "a weight or a reduction became non-finite");
    if (h & ERR_OVERFLOW) return set_err(ctx, M2M_ERR_OVERFLOW, "fixed-point histogram range exceeded");
    if (h & ERR_TIMEOUT) return set_err(ctx, M2M_ERR_TIMEOUT, "a bounded device wait ran out (bulk copy or grid barrier; results invalid)");
    return M2M_OK;
}

void free_events(m2m_ctx *c) {
    for (auto &e : c->evs) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    c->evs.clear();
    c->ev_free.clear();
}

void free_all(m2m_ctx *c) {
    free_events(c);
    void *ptrs[] = {c->d_edges, c->d_gh, c->d_Y, c->d_sigma, c->d_isig, c->d_Dt, c->d_y, c->d_Delta, c->d_coef_d,
                    c->d_coef_r, c->d_slots, c->d_stat_slots, c->d_chi_slots, c->d_ticket, c->d_rec_ticket, c->d_ring,
                    c->d_last, c->d_err, c->d_mm_slots, c->d_cell_ids, c->d_cell_acc, c->d_cell_cnt,
                    c->d_cell_mean, c->d_cell_cache, c->d_y_acc, c->d_sh_e2, c->d_sh_rn, c->d_sh_irn,
                    c->d_sh_tab, c->d_sh_rnd, c->d_sh_sum, c->d_facc, c->d_lnwhat, c->d_lut, c->d_pmap, c->d_psf,
                    c->d_bar, c->d_st2, c->d_chi2};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

int build_potential(m2m_ctx *ctx, const m2m_potential_desc *pot, int npot) {
    if (npot < 0 || npot > MAXPOT) return set_err(ctx, M2M_ERR_ARG, "npot=%d out of [0,%d]", npot, MAXPOT);
    if (npot > 0 && !pot) return set_err(ctx, M2M_ERR_ARG, "pot is NULL");
    PotDev tmp[MAXPOT];
    memset(tmp, 0, sizeof tmp);
    for (int k = 0; k < npot; ++k) {
        const double *p = pot[k].p;
        PotDev &d = tmp[k];
        d.kind = pot[k].kind;
        if (pot[k].kind == M2M_POT_HERNQUIST) {
            if (!(p[0] > 0 && p[1] > 0)) return set_err(ctx, M2M_ERR_ARG, "hernquist needs GM>0, a>0");
            d.c[0] = p[0]; d.c[1] = p[1];
        } else if (pot[k].kind == M2M_POT_LOG) {
            if (!(p[0] > 0 && p[1] > 0 && p[2] > 0)) return set_err(ctx, M2M_ERR_ARG, "log needs v0, Rc, q > 0");
            d.c[0] = p[1] * p[1]; d.c[1] = 1.0 / (p[2] * p[2]); d.c[2] = p[0] * p[0]; d.c[3] = 0.5 * p[0] * p[0];
        } else if (pot[k].kind == M2M_POT_NFW) {
            if (!(p[0] > 0 && p[1] > 0)) return set_err(ctx, M2M_ERR_ARG, "nfw needs rho_s>0, r_s>0");
            d.c[0] = 4.0 * M_PI * p[0] * p[1] * p[1] * p[1]; d.c[1] = p[1]; d.c[2] = 1.0 / p[1];
        } else if (pot[k].kind == M2M_POT_SH || pot[k].kind == M2M_POT_SH_TRI || pot[k].kind == M2M_POT_SH_FULL) {
            const int K = (int)p[0];
            if (k != npot - 1) return set_err(ctx, M2M_ERR_ARG, "the spherical-harmonic component must be last");
            if (!((double)K == p[0] && K >= 4 && K <= SH_MAXK && p[1] > 0 && p[2] > p[1] && isfinite(p[2]) &&
                  p[3] >= 1 && p[3] == floor(p[3]) && p[3] < 2147483648.0))
                return set_err(ctx, M2M_ERR_ARG, "sh needs integer K in [4,%d], 0 < rmin < rmax, integer period >= 1",
                               SH_MAXK);
            d.ik = K;
            const double lgc = (K - 1) / log2(p[2] / p[1]);
            d.c[0] = K; d.c[1] = p[1]; d.c[2] = p[2]; d.c[3] = lgc; d.c[4] = -lgc * log2(p[1]); d.c[5] = 1.0 / p[1];
        } else {
            return set_err(ctx, M2M_ERR_ARG, "unknown potential kind %d", pot[k].kind);
        }
    }
    for (int k = 0; k < MAXPOT; ++k)
        for (int j = 0; j < 6; ++j) tmp[k].cf[j] = (float)tmp[k].c[j];
    memcpy(ctx->pot, tmp, sizeof tmp);
    ctx->npot = npot;
    const int lastk = npot > 0 ? pot[npot - 1].kind : 0;
    ctx->sh_basis = lastk == M2M_POT_SH_TRI ? 1 : lastk == M2M_POT_SH_FULL ? 2 : 0;
    ctx->sh_on = lastk == M2M_POT_SH || lastk == M2M_POT_SH_TRI || lastk == M2M_POT_SH_FULL;
    ctx->sh_row = ctx->sh_basis == 1 ? TRI_ROW : ctx->sh_basis == 2 ? FULL_ROW : SH_ROW;
    if (ctx->sh_on) {
        const double *p = pot[npot - 1].p;
        ctx->sh_K = (int)p[0];
        ctx->sh_rmin = p[1];
        ctx->sh_rmax = p[2];
        ctx->sh_period = (int)p[3];
    }
    return M2M_OK;
}

// Side sums of the expansion: 10 per node (A_l, B_l of 5 even l), 30 for
// the triaxial one (A_lm, B_lm of its 15 terms).
size_t sh_sums(const m2m_ctx *c) {
    return (size_t)(c->sh_basis == 1 ? 2 * TriBasis::NT : c->sh_basis == 2 ? 2 * FullBasis::NT : 10) * c->sh_K;
}

// Node tables of the expansion: r_k = rmin (rmax/rmin)^(k/(K-1)), r_(K-1) =
// rmax, and r_k^2 (for R = float the smallest float >= the double square).
int sh_setup(m2m_ctx *ctx) {
    const int K = ctx->sh_K;
    const size_t rs = ctx->prec == M2M_FP32C ? 4 : 8;
    void **bufs[] = {&ctx->d_sh_e2, &ctx->d_sh_rn, &ctx->d_sh_irn, &ctx->d_sh_tab, (void **)&ctx->d_sh_rnd,
                     (void **)&ctx->d_sh_sum};
    for (void **b : bufs)
        if (*b) { cudaFree(*b); *b = nullptr; }
    CU(cudaMalloc(&ctx->d_sh_e2, rs * K));
    CU(cudaMalloc(&ctx->d_sh_rn, rs * K));
    CU(cudaMalloc(&ctx->d_sh_irn, rs * K));
    CU(cudaMalloc(&ctx->d_sh_tab, rs * ctx->sh_row * K));
    CU(cudaMalloc((void **)&ctx->d_sh_rnd, 8 * (size_t)K));
    CU(cudaMalloc((void **)&ctx->d_sh_sum, sh_sums(ctx) * 8));
    if (!ctx->d_facc) CU(cudaMalloc(&ctx->d_facc, rs * 3 * (size_t)ctx->n));
    ctx->facc_valid = false;
    std::vector<double> rn(K), e2(K), irn(K);
    const double ratio = ctx->sh_rmax / ctx->sh_rmin;
    for (int k = 0; k < K; ++k) rn[k] = ctx->sh_rmin * pow(ratio, (double)k / (double)(K - 1));
    rn[K - 1] = ctx->sh_rmax;
    for (int k = 0; k < K; ++k) { e2[k] = rn[k] * rn[k]; irn[k] = 1.0 / rn[k]; }
    for (int k = 1; k < K; ++k)
        if (!(e2[k] > e2[k - 1])) return set_err(ctx, M2M_ERR_ARG, "sh nodes not strictly increasing");
    guess_params(e2.data(), K - 1, &ctx->sh_gmode, &ctx->sh_ga, &ctx->sh_gb);
    std::vector<unsigned char> buf(rs * 3 * K);
    if (rs == 4) {
        float *f = (float *)buf.data();
        for (int k = 0; k < K; ++k) { f[k] = ceil_float(e2[k]); f[K + k] = (float)rn[k]; f[2 * K + k] = (float)irn[k]; }
    } else {
        double *d = (double *)buf.data();
        for (int k = 0; k < K; ++k) { d[k] = e2[k]; d[K + k] = rn[k]; d[2 * K + k] = irn[k]; }
    }
    CU(cudaMemcpy(ctx->d_sh_e2, buf.data(), rs * K, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->d_sh_rn, buf.data() + rs * K, rs * K, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->d_sh_irn, buf.data() + 2 * rs * K, rs * K, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->d_sh_rnd, rn.data(), 8 * (size_t)K, cudaMemcpyHostToDevice));
    return M2M_OK;
}

size_t sh_coef_smem(const m2m_ctx *c) {
    const size_t NS = sh_sums(c);
    return 8 * NS + (c->prec == M2M_FP32C ? 4 : 8) * 3 * (size_t)c->sh_K;
}

// The expansion from the current positions and weights: side sums, then
// the node table the push reads.
int sh_recompute(m2m_ctx *ctx) {
    const int K = ctx->sh_K;
    ctx->facc_valid = false;       // a new node table: the kept forces are of the old one
    CU(cudaMemsetAsync(ctx->d_sh_sum, 0, 8 * sh_sums(ctx), ctx->st));
    ShArgs a;
    memset(&a, 0, sizeof a);
    a.x = ctx->x; a.y = ctx->y; a.z = ctx->z; a.w = ctx->w; a.n = ctx->n;
    a.K = K; a.e2 = ctx->d_sh_e2; a.rn = ctx->d_sh_rn; a.irn = ctx->d_sh_irn;
    a.gmode = ctx->sh_gmode; a.ga = ctx->sh_ga; a.gb = ctx->sh_gb;
    a.sh = ctx->fx_shift + 6;
    a.sum = ctx->d_sh_sum; a.err = ctx->d_err;
    const bool f32 = ctx->prec == M2M_FP32C;
    void *fn = ctx->sh_basis == 1 ? (f32 ? (void *)k_ex_coef<TriBasis, float> : (void *)k_ex_coef<TriBasis, double>)
             : ctx->sh_basis == 2 ? (f32 ? (void *)k_ex_coef<FullBasis, float> : (void *)k_ex_coef<FullBasis, double>)
                                  : (f32 ? (void *)k_sh_coef<float> : (void *)k_sh_coef<double>);
    const size_t sm = sh_coef_smem(ctx);
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 512, sm));
    if (occ < 1) return set_err(ctx, M2M_ERR_ARG, "sh coefficient pass needs %zu B shared memory", sm);
    long long grid = (long long)ctx->nsm * occ, need = (ctx->n + 511) / 512;
    if (grid > need) grid = need;
    {
        void *args[] = {&a};
        LaunchTimer lt(ctx, M2M_TK_SH);
        CU(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(512), args, sm, ctx->st));
    }
    const double q = ldexp(1.0, -a.sh);
    const size_t tsm = ctx->sh_basis ? 8 * sh_sums(ctx) : 160 * (size_t)K;
    if (ctx->sh_basis) {
        LaunchTimer lt(ctx, M2M_TK_SH);
        const long long *sum = (const long long *)ctx->d_sh_sum;
        if (ctx->sh_basis == 1 && f32)
            k_ex_tables<TriBasis, float><<<1, 512, tsm, ctx->st>>>(sum, K, ctx->d_sh_rnd, q, (float *)ctx->d_sh_tab,
                                                                   ctx->d_err);
        else if (ctx->sh_basis == 1)
            k_ex_tables<TriBasis, double><<<1, 512, tsm, ctx->st>>>(sum, K, ctx->d_sh_rnd, q, (double *)ctx->d_sh_tab,
                                                                    ctx->d_err);
        else if (f32)
            k_ex_tables<FullBasis, float><<<1, 512, tsm, ctx->st>>>(sum, K, ctx->d_sh_rnd, q, (float *)ctx->d_sh_tab,
                                                                    ctx->d_err);
        else
            k_ex_tables<FullBasis, double><<<1, 512, tsm, ctx->st>>>(sum, K, ctx->d_sh_rnd, q,
                                                                     (double *)ctx->d_sh_tab, ctx->d_err);
        CU(cudaGetLastError());
    } else {
        LaunchTimer lt(ctx, M2M_TK_SH);
        if (f32)
            k_sh_tables<float><<<1, 256, tsm, ctx->st>>>((const long long *)ctx->d_sh_sum, K, ctx->d_sh_rnd, q,
                                                         (float *)ctx->d_sh_tab, ctx->d_err);
        else
            k_sh_tables<double><<<1, 256, tsm, ctx->st>>>((const long long *)ctx->d_sh_sum, K, ctx->d_sh_rnd, q,
                                                          (double *)ctx->d_sh_tab, ctx->d_err);
        CU(cudaGetLastError());
    }
    return M2M_OK;
}

}  // namespace

namespace m2m {
void note_context_free_error(const char *msg) { g_init_error = msg; }
}  // namespace m2m

extern "C" {

int m2m_init(m2m_ctx **ctx_out, int32_t precision, int64_t n, void *x, void *y, void *z, void *vx,
             void *vy, void *vz, double *w, double *what, const m2m_potential_desc *pot, int32_t npot,
             const m2m_obs_desc *obs, int32_t nsets, const double *Y, const double *sigma,
             const m2m_params *par, const m2m_prior_desc *prior, void *stream) {
    m2m_ctx *ctx = nullptr;
    if (!ctx_out) return set_err(nullptr, M2M_ERR_ARG, "ctx_out is NULL");
    *ctx_out = nullptr;
    if (precision != M2M_FP64 && precision != M2M_FP32C)
        return set_err(nullptr, M2M_ERR_ARG, "precision %d unknown", precision);
    if (n < 1 || n >= (1ll << 31)) return set_err(nullptr, M2M_ERR_ARG, "n=%lld out of [1, 2^31)", (long long)n);
    void *arrs[] = {x, y, z, vx, vy, vz, w, what};
    for (int k = 0; k < 8; ++k)
        if (!arrs[k] || !aligned16(arrs[k]))
            return set_err(nullptr, M2M_ERR_ARG, "particle array %d is NULL or not 16-byte aligned", k);
    if (!par) return set_err(nullptr, M2M_ERR_ARG, "par is NULL");
    if (!(isfinite(par->eps) && isfinite(par->mu) && isfinite(par->dt) && isfinite(par->alpha) &&
          isfinite(par->entropy_const) && isfinite(par->incl_sin) && isfinite(par->incl_cos)))
        return set_err(nullptr, M2M_ERR_ARG, "non-finite parameter");
    if (!(par->alpha > 0 && par->alpha <= 1)) return set_err(nullptr, M2M_ERR_ARG, "alpha must be in (0,1]");
    if (nsets < 1 || nsets > MAXSETS || !obs)
        return set_err(nullptr, M2M_ERR_ARG, "nsets=%d out of [1,%d]", nsets, MAXSETS);

    ctx = new m2m_ctx();   // value-initialised: all pointers NULL
    ctx->prec = precision;
    ctx->n = n;
    ctx->x = x; ctx->y = y; ctx->z = z; ctx->vx = vx; ctx->vy = vy; ctx->vz = vz;
    ctx->w = w; ctx->what = what;
    ctx->st = (cudaStream_t)stream;
    ctx->par = *par;
    ctx->threads = precision == M2M_FP32C ? 1024 : 256;
    ctx->bps_req = 0;
    ctx->pipe = false;
    ctx->fx_atomic = 1;
    int rc = build_potential(ctx, pot, npot);
    if (rc) { g_init_error = ctx->err; delete ctx; return rc; }

    // observable tables
    const bool f32 = precision == M2M_FP32C;
    std::vector<double> edges_d;
    std::vector<double> gh_d;
    std::vector<int> lut_h;                  // the LUT sets' tables, concatenated
    int lut_off[MAXSETS] = {0};
    std::vector<double> psf_h;               // the seeing tables, concatenated
    int psf_off[MAXSETS] = {0};
    int nobs = 0;
    for (int s = 0; s < nsets; ++s) {
        const m2m_obs_desc &o = obs[s];
        SetDev &d = ctx->sets[s];
        memset(&d, 0, sizeof d);
        const bool two_d = o.geom == M2M_GEOM_GRID || o.geom == M2M_GEOM_LUT;
        d.geom = o.geom; d.quant = o.quant; d.nx = o.nx; d.ny = two_d ? o.ny : 1;
        if (o.geom < 1 || o.geom > 4 || o.quant < 1 || o.quant > 3 || o.nx < 1 || d.ny < 1 || !o.edges_x ||
            (two_d && !o.edges_y) || (o.geom == M2M_GEOM_LUT && (!o.lut || o.ncell < 1)) ||
            (long long)d.nx * d.ny > M2M_MAX_LUT_PIXELS) {
            set_err(nullptr, M2M_ERR_ARG, "observable set %d: bad geometry/quantity/sizes/edges", s);
            delete ctx; return M2M_ERR_ARG;
        }
        d.nmom = o.quant == M2M_Q_GH ? 5 : 1;
        d.gx_top = (float)(d.nx - 1);
        d.gy_top = (float)(d.ny - 1);
        long long cells = o.geom == M2M_GEOM_LUT ? o.ncell : (long long)d.nx * d.ny;
        d.ncell = (int)cells;
        if (o.geom == M2M_GEOM_LUT) {
            const long long npx = (long long)d.nx * d.ny;
            if ((long long)lut_h.size() + npx > M2M_MAX_LUT_PIXELS) {
                set_err(nullptr, M2M_ERR_ARG, "more than %d lookup-table pixels in total", M2M_MAX_LUT_PIXELS);
                delete ctx; return M2M_ERR_ARG;
            }
            for (long long k = 0; k < npx; ++k) {
                if (o.lut[k] < -1 || o.lut[k] >= o.ncell) {
                    set_err(nullptr, M2M_ERR_ARG, "observable set %d: lookup-table entry %lld = %d not in [-1, %d)",
                            s, k, o.lut[k], o.ncell);
                    delete ctx; return M2M_ERR_ARG;
                }
            }
            lut_off[s] = (int)lut_h.size();
            lut_h.insert(lut_h.end(), o.lut, o.lut + npx);
        }
        if (o.psf_q) {
            bool ok = o.geom != M2M_GEOM_SHELL && o.psf_bits >= 1 && o.psf_bits <= 16;
            const int len = ok ? 1 << o.psf_bits : 0;
            for (int k = 0; ok && k < len; ++k)
                ok = isfinite(o.psf_q[k]) && (k == 0 || o.psf_q[k] >= o.psf_q[k - 1]);
            if (!ok) {
                set_err(nullptr, M2M_ERR_ARG, "observable set %d: seeing needs a projected set and "
                                              "2^psf_bits (1..16) finite, non-decreasing quantiles", s);
                delete ctx; return M2M_ERR_ARG;
            }
            psf_off[s] = (int)psf_h.size();
            psf_h.insert(psf_h.end(), o.psf_q, o.psf_q + len);
            d.psf_shift = 32 - o.psf_bits;
            d.psf_seed = o.psf_seed;
        }
        d.obs_off = nobs;
        if (nobs + cells * d.nmom > MAXOBS) {
            set_err(nullptr, M2M_ERR_ARG, "more than %d observables", MAXOBS);
            delete ctx; return M2M_ERR_ARG;
        }
        nobs += (int)(cells * d.nmom);
        for (int ax = 0; ax < (two_d ? 2 : 1); ++ax) {
            const double *e = ax == 0 ? o.edges_x : o.edges_y;
            int nb = ax == 0 ? d.nx : d.ny;
            for (int k = 0; k <= nb; ++k) {
                if (!(e[k] == e[k]) || (k > 0 && !(e[k] > e[k - 1]))) {
                    set_err(nullptr, M2M_ERR_ARG, "observable set %d: edges must be strictly increasing", s);
                    delete ctx; return M2M_ERR_ARG;
                }
            }
            int off = (int)edges_d.size();
            edges_d.insert(edges_d.end(), e, e + nb + 1);
            if (ax == 0) { d.ex_off = off; guess_params(e, nb, &d.gx_mode, &d.gx_a, &d.gx_b); }
            else { d.ey_off = off; guess_params(e, nb, &d.gy_mode, &d.gy_a, &d.gy_b); }
        }
        if (o.quant == M2M_Q_GH) {
            if (!o.gh_V || !o.gh_S || !(o.sigma_kernel >= 0)) {
                set_err(nullptr, M2M_ERR_ARG, "observable set %d: GH needs gh_V, gh_S, sigma_kernel>=0", s);
                delete ctx; return M2M_ERR_ARG;
            }
            d.gh_off = (int)gh_d.size();
            d.ghc_off = d.gh_off / 5;
            for (long long c = 0; c < cells; ++c) {
                double S = o.gh_S[c];
                if (!(S > 0) || !isfinite(o.gh_V[c])) {
                    set_err(nullptr, M2M_ERR_ARG, "observable set %d: gh_S must be > 0", s);
                    delete ctx; return M2M_ERR_ARG;
                }
                double sk = o.sigma_kernel / S;
                double d1 = 1.0 + sk * sk;
                gh_d.push_back(o.gh_V[c]);
                gh_d.push_back(1.0 / S);
                gh_d.push_back(1.0 / d1);
                gh_d.push_back(sk * sk / d1);
                gh_d.push_back(2.0 * sqrt(M_PI) / sqrt(2.0 * M_PI * d1));
            }
        }
    }
    ctx->nsets = nsets;
    ctx->nobs = nobs;
    {
        int bits = 0;
        for (int k = 0; k < nsets; ++k) {
            int cells = obs[k].geom == M2M_GEOM_LUT ? obs[k].ncell : ctx->sets[k].nx * ctx->sets[k].ny, b = 1;
            while ((1 << b) < cells + 1) ++b;
            ctx->sets[k].cshift = bits < 32 ? bits : 0;
            ctx->sets[k].cmask = (1 << b) - 1;
            bits += b;
        }
        ctx->cache_bits = bits;
    }
    ctx->layout = detect_layout(ctx);
    ctx->edge_len = (int)edges_d.size();
    ctx->gh_len = (int)gh_d.size();
    std::vector<short> pmap_h;
    if (f32 && ctx->layout == 1) pmap_h = aligned_pixel_map(ctx->sets[0], ctx->sets[1], edges_d);

    // priors
    if (prior && prior->kind != M2M_PRIOR_FLAT) {
        ctx->prior = *prior;
        if ((prior->kind != M2M_PRIOR_E_LC && prior->kind != M2M_PRIOR_E_LZ && prior->kind != M2M_PRIOR_E_L2) ||
            prior->nE < 1 ||
            prior->nL < 1 || prior->period < 1 ||
            (long long)prior->nE * prior->nL + 1 > MAXCELLS ||
            (prior->kind == M2M_PRIOR_E_LC && !(prior->hernquist_GM > 0 && prior->hernquist_a > 0))) {
            set_err(nullptr, M2M_ERR_ARG, "bad prior descriptor");
            delete ctx; return M2M_ERR_ARG;
        }
        ctx->ncells = prior->nE * prior->nL + (prior->kind == M2M_PRIOR_E_LC ? 1 : 0);
    } else {
        memset(&ctx->prior, 0, sizeof ctx->prior);
        ctx->prior.kind = M2M_PRIOR_FLAT;
        ctx->prior.nE = ctx->prior.nL = 1;
        ctx->prior.hernquist_GM = ctx->prior.hernquist_a = 1.0;
        ctx->ncells = 0;
    }

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) {
        set_err(nullptr, M2M_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(ce));
        delete ctx; return M2M_ERR_CUDA;
    }
    ctx->slot_cap = ctx->nsm * 4;

#define ALLOC(ptr, bytes)                                                               \
    do {                                                                                \
        if (cudaMalloc((void **)&(ptr), (bytes) ? (bytes) : 16) != cudaSuccess) {       \
            set_err(nullptr, M2M_ERR_NOMEM, "cudaMalloc(%zu) failed", (size_t)(bytes)); \
            free_all(ctx); delete ctx; return M2M_ERR_NOMEM;                            \
        }                                                                               \
    } while (0)
    size_t rs = f32 ? 4 : 8;
    ALLOC(ctx->d_edges, rs * ctx->edge_len);
    ALLOC(ctx->d_gh, rs * (ctx->gh_len + 1));
    ALLOC(ctx->d_Y, 8 * nobs); ALLOC(ctx->d_sigma, 8 * nobs); ALLOC(ctx->d_Dt, 8 * nobs);
    ALLOC(ctx->d_isig, 8 * nobs);
    ALLOC(ctx->d_y, 8 * nobs); ALLOC(ctx->d_Delta, 8 * nobs); ALLOC(ctx->d_coef_d, 8 * nobs);
    ALLOC(ctx->d_coef_r, rs * nobs);
    ALLOC(ctx->d_slots, (size_t)8 * nobs * ctx->slot_cap);
    ALLOC(ctx->d_y_acc, (size_t)8 * nobs);
    ALLOC(ctx->d_stat_slots, (size_t)32 * ctx->slot_cap);
    ALLOC(ctx->d_rec_ticket, 8);
    ALLOC(ctx->d_chi_slots, (size_t)24 * ((nobs + 31) / 32 + 1));
    ALLOC(ctx->d_bar, 8);
    ALLOC(ctx->d_st2, (size_t)32 * ctx->slot_cap);
    ALLOC(ctx->d_chi2, (size_t)48 * ctx->slot_cap);
    ALLOC(ctx->d_ticket, 4);
    ALLOC(ctx->d_ring, sizeof(m2m_record) * M2M_HISTORY);
    ALLOC(ctx->d_last, sizeof(m2m_record));
    ALLOC(ctx->d_err, 4);
    ALLOC(ctx->d_mm_slots, rs * 4 * ctx->slot_cap);
    ALLOC(ctx->d_cell_cache, 4 * (size_t)n);
    if (!lut_h.empty()) ALLOC(ctx->d_lut, 4 * lut_h.size());
    if (!pmap_h.empty()) ALLOC(ctx->d_pmap, 2 * pmap_h.size());
    if (!psf_h.empty()) ALLOC(ctx->d_psf, rs * psf_h.size());
    if (f32) ALLOC(ctx->d_lnwhat, 4 * (size_t)n);
    if (ctx->ncells) {
        ALLOC(ctx->d_cell_ids, 4 * (size_t)n);
        ALLOC(ctx->d_cell_acc, 8 * (size_t)ctx->ncells);
        ALLOC(ctx->d_cell_cnt, 4 * (size_t)ctx->ncells);
        ALLOC(ctx->d_cell_mean, 8 * (size_t)ctx->ncells);
    }
#undef ALLOC

    // tables: float edges are the smallest float >= the double edge
    {
        std::vector<unsigned char> buf(rs * (edges_d.size() + gh_d.size() + 1));
        if (f32) {
            float *e = (float *)buf.data();
            for (size_t k = 0; k < edges_d.size(); ++k) e[k] = ceil_float(edges_d[k]);
            float *g = e + edges_d.size();
            for (size_t k = 0; k < gh_d.size(); ++k) g[k] = (float)gh_d[k];
        } else {
            double *e = (double *)buf.data();
            memcpy(e, edges_d.data(), 8 * edges_d.size());
            memcpy(e + edges_d.size(), gh_d.data(), 8 * gh_d.size());
        }
        cudaError_t e1 = cudaMemcpy(ctx->d_edges, buf.data(), rs * edges_d.size(), cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(ctx->d_gh, buf.data() + rs * edges_d.size(), rs * gh_d.size(),
                                    cudaMemcpyHostToDevice);
        std::vector<double> zero(nobs, 0.0);
        cudaError_t e3 = cudaMemcpy(ctx->d_Y, Y ? Y : zero.data(), 8 * nobs, cudaMemcpyHostToDevice);
        cudaError_t e4 = cudaMemcpy(ctx->d_sigma, sigma ? sigma : zero.data(), 8 * nobs, cudaMemcpyHostToDevice);
        std::vector<double> isig(nobs, 0.0);
        for (int j = 0; j < nobs && sigma; ++j) isig[j] = sigma[j] > 0 ? 1.0 / sigma[j] : 0.0;
        if (e4 == cudaSuccess) e4 = cudaMemcpy(ctx->d_isig, isig.data(), 8 * nobs, cudaMemcpyHostToDevice);
        cudaError_t e5 = cudaMemset(ctx->d_Dt, 0, 8 * nobs);
        cudaError_t e6 = cudaMemset(ctx->d_ticket, 0, 4);
        if (e6 == cudaSuccess) e6 = cudaMemset(ctx->d_rec_ticket, 0, 8);
        cudaError_t e7 = cudaMemset(ctx->d_err, 0, 4);
        cudaError_t e8 = cudaMemset(ctx->d_coef_r, 0, rs * nobs);
        cudaError_t e9 = cudaMemset(ctx->d_ring, 0, sizeof(m2m_record) * M2M_HISTORY);
        cudaError_t e10 = cudaMemset(ctx->d_y_acc, 0, 8 * (size_t)nobs);
        cudaError_t e11 = lut_h.empty() ? cudaSuccess
                                        : cudaMemcpy(ctx->d_lut, lut_h.data(), 4 * lut_h.size(), cudaMemcpyHostToDevice);
        for (int k = 0; k < nsets; ++k)
            if (ctx->sets[k].geom == M2M_GEOM_LUT) ctx->sets[k].lut = ctx->d_lut + lut_off[k];
        if (e11 == cudaSuccess && !pmap_h.empty()) {
            e11 = cudaMemcpy(ctx->d_pmap, pmap_h.data(), 2 * pmap_h.size(), cudaMemcpyHostToDevice);
            ctx->sets[1].pmap = ctx->d_pmap;
            ctx->sets[1].pmap_len = (int)pmap_h.size();
        }
        // seeing tables in the state precision (FP32C: rounded once to float)
        std::vector<unsigned char> pb(rs * psf_h.size());
        for (size_t k = 0; k < psf_h.size(); ++k) {
            if (f32) ((float *)pb.data())[k] = (float)psf_h[k];
            else ((double *)pb.data())[k] = psf_h[k];
        }
        cudaError_t e12 = psf_h.empty() ? cudaSuccess
                                        : cudaMemcpy(ctx->d_psf, pb.data(), pb.size(), cudaMemcpyHostToDevice);
        for (int k = 0; k < nsets; ++k)
            if (obs[k].psf_q) ctx->sets[k].psf = (const unsigned char *)ctx->d_psf + rs * psf_off[k];
        cudaError_t es[] = {e1, e2, e3, e4, e5, e6, e7, e8, e9, e10, e11, e12};
        for (cudaError_t e : es)
            if (e != cudaSuccess) {
                set_err(nullptr, M2M_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
                free_all(ctx); delete ctx; return M2M_ERR_CUDA;
            }
    }
    // the pass kernels may use more than 48 KB of shared memory
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    std::vector<void *> kfns = {cells_kernel_f32(), cells_kernel_f64(), (void *)k_sh_coef<float>,
                                (void *)k_sh_coef<double>, (void *)k_sh_tables<float>, (void *)k_sh_tables<double>,
                                (void *)k_ex_coef<TriBasis, float>, (void *)k_ex_coef<TriBasis, double>,
                                (void *)k_ex_tables<TriBasis, float>, (void *)k_ex_tables<TriBasis, double>,
                                (void *)k_ex_coef<FullBasis, float>, (void *)k_ex_coef<FullBasis, double>,
                                (void *)k_ex_tables<FullBasis, float>, (void *)k_ex_tables<FullBasis, double>};
    for (int lay = 0; lay < 5; ++lay) {
        for (int nt : {256, 512, 1024}) kfns.push_back(pass_kernel_f32(nt, lay));
        for (int nt : {256, 512}) kfns.push_back(pass_kernel_f64(nt, lay));
        if (lay) kfns.push_back(pass_kernel_f32_pipe(lay));
        for (int pk : {PK_ANY, PK_HERNQUIST, PK_LOG, PK_SH, PK_HERNQUIST_NFW, PK_SH_TRI, PK_SH_FULL})
                for (int fl : {F_STEADY, F_STEADY | F_MINMAX, F_PUSH | F_SCAT | F_STATS,
                               F_PUSH | F_SCAT | F_STATS | F_MINMAX, F_CELLS | F_UPD})
                    if (void *f = pass_kernel_f32_compiled(fl, lay, pk)) kfns.push_back(f);
        if (lay) kfns.push_back(pass_kernel_f32_pipe_steady(lay));
        kfns.push_back(pass_kernel_f32_batch(lay));
        if (lay) kfns.push_back(pass_kernel_f32_batch(lay, true));
        if (lay == 2) kfns.push_back(pass_kernel_f32_batch(lay, true, PK_HERNQUIST_NFW));
        for (int pk : {PK_HERNQUIST, PK_LOG, PK_HERNQUIST_NFW}) kfns.push_back(steps_kernel_f32(lay, pk));
    }
    for (void *f : kfns) {
        if (!f) continue;                    // no such variant compiled
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) {
            set_err(nullptr, M2M_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            free_all(ctx); delete ctx; return M2M_ERR_CUDA;
        }
    }

    if (f32) {
        int gl = ctx->nsm * 8;
        const long long needl = (n + 255) / 256;
        if (gl > needl) gl = (int)needl;
        k_lnwhat<<<gl, 256, 0, ctx->st>>>(what, ctx->d_lnwhat, n);
        if (cudaGetLastError() != cudaSuccess) {
            set_err(nullptr, M2M_ERR_CUDA, "ln w_hat launch failed");
            free_all(ctx); delete ctx; return M2M_ERR_CUDA;
        }
    }
    // fixed-point scale from the particle count and the initial total
    // weight: resolution 2^-25 of the average weight (2^-25 * 2^ceil(log2
    // sum w) / 2^ceil(log2 n)), so that the usual terms w K stay below the
    // 2^31 of the fast histogram path (terms up to ~64 times the average)
    int nbits = 0;
    while ((1ll << nbits) < n) ++nbits;
    ctx->fx_shift = FX_AVG_BITS + nbits;
    ctx->fx_q = ldexp(1.0, -ctx->fx_shift);
    ctx->cell_shift = 60;
    int g = 0;
    rc = launch_pass(ctx, F_STATS, &g);
    if (rc == M2M_OK) {
        std::vector<double> st(2 * g);
        cudaError_t e = cudaMemcpyAsync(st.data(), ctx->d_stat_slots + (size_t)2 * ctx->slot_cap * (ctx->stat_par ^ 1),
                                        16 * g, cudaMemcpyDeviceToHost, ctx->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
        if (e != cudaSuccess) rc = set_err(ctx, M2M_ERR_CUDA, "init reduction: %s", cudaGetErrorString(e));
        double W = 0.0;
        for (int b = 0; b < g; ++b) W += st[2 * b + 1];
        if (rc == M2M_OK && !(W >= 0 && isfinite(W))) rc = set_err(ctx, M2M_ERR_NONFINITE, "sum of weights not finite");
        if (rc == M2M_OK && W > 0) {
            int e2 = scale_exp(W);
            ctx->fx_shift = FX_AVG_BITS + nbits - e2;
            ctx->fx_q = ldexp(1.0, -ctx->fx_shift);
            ctx->cell_shift = 60 - e2;
        }
    }
    if (rc == M2M_OK && ctx->sh_on) rc = sh_setup(ctx);
    if (rc == M2M_OK && ctx->sh_on) rc = sh_recompute(ctx);
    if (rc == M2M_OK) rc = observe_now(ctx, 0, 2, 0, 0);
    if (rc == M2M_OK) rc = check_err_word(ctx);
    if (rc != M2M_OK) {
        g_init_error = ctx->err;
        free_all(ctx); delete ctx; return rc;
    }
    ctx->t = 0;
    ctx->pending = false;
    *ctx_out = ctx;
    return M2M_OK;
}

int m2m_set_targets(m2m_ctx *ctx, const double *Y, const double *sigma) {
    if (!ctx || !Y || !sigma) return set_err(ctx, M2M_ERR_ARG, "NULL argument");
    CU(cudaMemcpyAsync(ctx->d_Y, Y, 8 * (size_t)ctx->nobs, cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(ctx->d_sigma, sigma, 8 * (size_t)ctx->nobs, cudaMemcpyHostToDevice, ctx->st));
    int nb = (ctx->nobs + 255) / 256;
    k_inv_sigma<<<nb, 256, 0, ctx->st>>>(ctx->d_sigma, ctx->d_isig, ctx->nobs);
    CU(cudaGetLastError());
    return M2M_OK;
}

int m2m_potential(m2m_ctx *ctx, const m2m_potential_desc *pot, int32_t npot) {
    if (!ctx) return M2M_ERR_ARG;
    int rc0 = finish_update(ctx);
    if (rc0) return rc0;
    const int oldK = ctx->sh_on ? ctx->sh_K : 0;
    const int oldbasis = ctx->sh_basis;
    const double oldr0 = ctx->sh_rmin, oldr1 = ctx->sh_rmax;
    int rc = build_potential(ctx, pot, npot);
    if (rc || !ctx->sh_on) return rc;
    if (ctx->sh_K != oldK || ctx->sh_basis != oldbasis || ctx->sh_rmin != oldr0 || ctx->sh_rmax != oldr1) {
        rc = sh_setup(ctx);
        if (rc) { ctx->sh_on = false; ctx->npot = 0; return rc; }
    }
    return sh_recompute(ctx);
}

int m2m_get_sh_table(m2m_ctx *ctx, double *out) {
    if (!ctx || !out) return set_err(ctx, M2M_ERR_ARG, "NULL argument");
    if (!ctx->sh_on) return set_err(ctx, M2M_ERR_STATE, "the potential has no SH component");
    const size_t cnt = (size_t)ctx->sh_row * ctx->sh_K;
    if (ctx->prec == M2M_FP32C) {
        std::vector<float> f(cnt);
        CU(cudaMemcpyAsync(f.data(), ctx->d_sh_tab, 4 * cnt, cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
        for (size_t k = 0; k < cnt; ++k) out[k] = f[k];
    } else {
        CU(cudaMemcpyAsync(out, ctx->d_sh_tab, 8 * cnt, cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
    }
    return M2M_OK;
}

int m2m_observe(m2m_ctx *ctx, int32_t mode) {
    if (!ctx || mode < 0 || mode > 2) return set_err(ctx, M2M_ERR_ARG, "bad context or mode");
    int rc = finish_update(ctx);
    if (rc) return rc;
    ctx->facc_valid = false;       // the caller may have moved the particles
    return observe_now(ctx, 0, mode, ctx->t, 0);
}

int m2m_update_weights(m2m_ctx *ctx) {
    if (!ctx) return M2M_ERR_ARG;
    int rc = finish_update(ctx);
    if (rc) return rc;
    return launch_pass(ctx, F_UPD);
}

int m2m_priors(m2m_ctx *ctx) {
    if (!ctx) return M2M_ERR_ARG;
    if (ctx->prior.kind == M2M_PRIOR_FLAT) return set_err(ctx, M2M_ERR_STATE, "priors are flat");
    int rc = finish_update(ctx);
    if (rc) return rc;
    rc = launch_pass(ctx, F_MINMAX);
    if (rc) return rc;
    return prior_recompute(ctx, 0);
}

int m2m_push(m2m_ctx *ctx, int64_t nsteps) {
    if (!ctx || nsteps < 0) return set_err(ctx, M2M_ERR_ARG, "bad argument");
    int rc0 = finish_update(ctx);
    if (rc0) return rc0;
    for (int64_t k = 0; k < nsteps; ++k) {
        int rc = launch_pass(ctx, F_PUSH);
        if (rc) return rc;
    }
    return M2M_OK;
}

int m2m_step(m2m_ctx *ctx, int64_t nsteps) {
    if (!ctx || nsteps < 0) return set_err(ctx, M2M_ERR_ARG, "bad argument");
    if (ctx->shard) return set_err(ctx, M2M_ERR_STATE, "a shard context steps through m2m_shard_*");
    const bool moving = ctx->prior.kind != M2M_PRIOR_FLAT;
    for (int64_t k = 0; k < nsteps; ++k) {
        long long t1 = ctx->t + 1;
        size_t psm = 0;
        int pgrid = 0;
        if (void *pf = persistent_kernel(ctx, &psm, &pgrid)) {
            // the steps up to the next prior recompute (inclusive) in one launch
            long long m = nsteps - k;
            if (moving) {
                const long long due = ((t1 + ctx->prior.period - 1) / ctx->prior.period) * ctx->prior.period;
                if (due - t1 + 1 < m) m = due - t1 + 1;
            }
            const bool range = moving && ((t1 + m - 1) % ctx->prior.period == 0);
            int rc = launch_steps(ctx, pf, psm, pgrid, m, range);
            if (rc) return rc;
            if (range) {
                rc = prior_recompute(ctx, F_UPD);
                if (rc) return rc;
                ctx->pending = false;
            }
            k += m - 1;
            continue;
        }
        bool prior_due = moving && (t1 % ctx->prior.period == 0);
        int fl = F_PUSH | F_SCAT | F_STATS | (ctx->pending ? F_UPD : 0) | (prior_due ? F_MINMAX : 0);
        int g = 0;
        int rc = launch_pass(ctx, fl, &g);
        if (rc) return rc;
        rc = launch_residual(ctx, 1, t1, 1, g, 0);
        if (rc) return rc;
        ctx->rec_pending = true;
        ctx->rec_step = t1;
        ctx->rec_stat_par = ctx->stat_par ^ 1;
        ctx->rec_stat_nblk = ctx->stat_prev_nblk;
        ctx->t = t1;
        ctx->pending = true;
        if (prior_due) {
            rc = prior_recompute(ctx, F_UPD);
            if (rc) return rc;
            ctx->pending = false;
        }
        if (ctx->sh_on && t1 % ctx->sh_period == 0) {
            // the expansion of (x_{t+1}, w_{t+1}): apply the update first
            if (ctx->pending) {
                rc = launch_pass(ctx, F_UPD);
                if (rc) return rc;
                ctx->pending = false;
            }
            rc = sh_recompute(ctx);
            if (rc) return rc;
        }
    }
    if (!ctx->lazy_update) return finish_update(ctx);
    return M2M_OK;
}

int m2m_set_lazy_update(m2m_ctx *ctx, int32_t on) {
    if (!ctx) return M2M_ERR_ARG;
    ctx->lazy_update = on != 0;
    return on ? M2M_OK : finish_update(ctx);
}

int m2m_finish_update(m2m_ctx *ctx) {
    if (!ctx) return M2M_ERR_ARG;
    return finish_update(ctx);
}

int m2m_velocity_moments(m2m_ctx *ctx, const double *r2_edges, int32_t nshell, double *out) {
    if (!ctx || !r2_edges || !out || nshell < 1 || nshell > 1024)
        return set_err(ctx, M2M_ERR_ARG, "bad argument (1 <= nshell <= 1024, non-NULL arrays)");
    for (int k = 0; k <= nshell; ++k)
        if (!(r2_edges[k] == r2_edges[k]) || (k > 0 && !(r2_edges[k] > r2_edges[k - 1])))
            return set_err(ctx, M2M_ERR_ARG, "edges must be strictly increasing");
    int rc = finish_update(ctx);
    if (rc) return rc;
    const size_t eb = 8 * (size_t)(nshell + 1), ob = 32 * (size_t)nshell;
    void *d = nullptr;
    CU(cudaMallocAsync(&d, eb + ob, ctx->st));
    double *de = (double *)d, *dout = de + (nshell + 1);
    cudaError_t e = cudaMemcpyAsync(de, r2_edges, eb, cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, ob, ctx->st);
    if (e == cudaSuccess) {
        const size_t sm = ob + eb;
        int g = ctx->nsm * 4;
        long long need = (ctx->n + 255) / 256;
        if (g > need) g = (int)need;
        if (ctx->prec == M2M_FP32C)
            k_vmoments<float><<<g, 256, sm, ctx->st>>>((const float *)ctx->x, (const float *)ctx->y, (const float *)ctx->z,
                                                        (const float *)ctx->vx, (const float *)ctx->vy,
                                                        (const float *)ctx->vz, ctx->w, ctx->n, de, nshell, dout);
        else
            k_vmoments<double><<<g, 256, sm, ctx->st>>>((const double *)ctx->x, (const double *)ctx->y,
                                                         (const double *)ctx->z, (const double *)ctx->vx,
                                                         (const double *)ctx->vy, (const double *)ctx->vz, ctx->w,
                                                         ctx->n, de, nshell, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, ob, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    cudaFreeAsync(d, ctx->st);
    if (e != cudaSuccess) return set_err(ctx, M2M_ERR_CUDA, "velocity moments: %s", cudaGetErrorString(e));
    return check_err_word(ctx);
}

// ---------------------------------------------------------------- shards
int m2m_shard_init(m2m_ctx *ctx, int64_t global_n, double global_sum_w) {
    if (!ctx) return M2M_ERR_ARG;
    if (global_n < ctx->n || global_n >= (1ll << 40) || !(global_sum_w > 0) || !isfinite(global_sum_w))
        return set_err(ctx, M2M_ERR_ARG, "global_n >= the shard's n and global_sum_w > 0 finite");
    if (ctx->sh_on) return set_err(ctx, M2M_ERR_STATE, "shards: not with the spherical-harmonic potential");
    if (ctx->prec != M2M_FP32C) return set_err(ctx, M2M_ERR_STATE, "shards: FP32C contexts (exact integer totals)");
    int rc = finish_update(ctx);
    if (rc) return rc;
    rc = finish_record(ctx);
    if (rc) return rc;
    int nbits = 0;
    while ((1ll << nbits) < global_n) ++nbits;
    const int e2 = scale_exp(global_sum_w);
    ctx->fx_shift = FX_AVG_BITS + nbits - e2;
    ctx->fx_q = ldexp(1.0, -ctx->fx_shift);
    ctx->cell_shift = 60 - e2;
    ctx->fx_atomic = 1;
    ctx->shard = true;
    return M2M_OK;
}

int m2m_shard_scatter(m2m_ctx *ctx, int32_t push, int32_t *prior_due, int64_t *totals, double *stats, double *range) {
    if (!ctx || !totals || !stats) return set_err(ctx, M2M_ERR_ARG, "NULL buffer");
    if (!ctx->shard) return set_err(ctx, M2M_ERR_STATE, "call m2m_shard_init first");
    const bool moving = ctx->prior.kind != M2M_PRIOR_FLAT;
    const bool due = push && moving && ((ctx->t + 1) % ctx->prior.period == 0);
    if (due && !range) return set_err(ctx, M2M_ERR_ARG, "a prior recompute is due: range buffer needed");
    int rc = finish_record(ctx);
    if (rc) return rc;
    const int fl = F_SCAT | F_STATS | (push ? F_PUSH : 0) | (ctx->pending ? F_UPD : 0) | (due ? F_MINMAX : 0);
    int g = 0;
    rc = launch_pass(ctx, fl, &g);
    if (rc) return rc;
    {
        LaunchTimer lt(ctx, M2M_TK_OTHER);
        const double *ss = ctx->d_stat_slots + (size_t)2 * ctx->slot_cap * (ctx->stat_par ^ 1);
        if (ctx->prec == M2M_FP32C)
            k_shard_pack<float><<<1, 256, 0, ctx->st>>>(ctx->d_y_acc, (long long *)totals, ctx->nobs, ss, g, stats, ctx->d_mm_slots,
                                                        due ? ctx->mm_nblocks : 0, due ? range : nullptr);
        else
            k_shard_pack<double><<<1, 256, 0, ctx->st>>>(ctx->d_y_acc, (long long *)totals, ctx->nobs, ss, g, stats, ctx->d_mm_slots,
                                                         due ? ctx->mm_nblocks : 0, due ? range : nullptr);
        CU(cudaGetLastError());
    }
    ctx->pending = false;                // applied by this pass, if it was
    ctx->shard_push = push != 0;
    ctx->shard_due = due;
    if (prior_due) *prior_due = due ? 1 : 0;
    return M2M_OK;
}

int m2m_shard_residual(m2m_ctx *ctx, int64_t *totals, const double *stats) {
    if (!ctx || !totals || !stats) return set_err(ctx, M2M_ERR_ARG, "NULL buffer");
    if (!ctx->shard) return set_err(ctx, M2M_ERR_STATE, "call m2m_shard_init first");
    ResArgs r;
    memset(&r, 0, sizeof r);
    const bool push = ctx->shard_push;
    const long long t1 = push ? ctx->t + 1 : ctx->t;
    r.nobs = ctx->nobs; r.y_acc = (unsigned long long *)totals; r.fx_atomic = 1;
    r.fixed = ctx->prec == M2M_FP32C; r.q = ctx->fx_q;
    r.Y = ctx->d_Y; r.inv_sigma = ctx->d_isig; r.Dt = ctx->d_Dt; r.y = ctx->d_y; r.Delta = ctx->d_Delta;
    r.coef_d = ctx->d_coef_d; r.coef_r = ctx->d_coef_r; r.r_float = ctx->prec == M2M_FP32C;
    r.mode = push ? 1 : 2; r.alpha = ctx->par.alpha; r.mu = ctx->par.mu;
    r.stat_slots = stats; r.stat_nblk = 1; r.tail = 1;
    r.chi_slots = ctx->d_chi_slots; r.ticket = ctx->d_ticket;
    r.ring = ctx->d_ring; r.last = ctx->d_last; r.rec_step = t1; r.write_ring = push ? 1 : 0;
    r.err = ctx->d_err;
    const int nb = (ctx->nobs + RES_NT_FX - 1) / RES_NT_FX;
    void *args[] = {&r};
    {
        LaunchTimer lt(ctx, M2M_TK_RESIDUAL);
        CU(launch_dependent((void *)k_residual, dim3(nb), dim3(RES_NT_FX), args, 0, ctx->st));
    }
    ctx->rec_chi_nblk = nb;
    if (push) ctx->t = t1;
    ctx->pending = push;                 // the update of this step goes into the next pass
    return M2M_OK;
}

int m2m_shard_prior_cells(m2m_ctx *ctx, const double *range, int64_t *cell_sums, int32_t *cell_counts) {
    if (!ctx || !range || !cell_sums || !cell_counts) return set_err(ctx, M2M_ERR_ARG, "NULL buffer");
    if (!ctx->shard || !ctx->shard_due) return set_err(ctx, M2M_ERR_STATE, "no prior recompute is due");
    {
        LaunchTimer lt(ctx, M2M_TK_PRIOR);
        if (ctx->prec == M2M_FP32C) k_shard_range<float><<<1, 1, 0, ctx->st>>>(range, ctx->d_mm_slots);
        else k_shard_range<double><<<1, 1, 0, ctx->st>>>(range, ctx->d_mm_slots);
        CU(cudaGetLastError());
    }
    ctx->mm_nblocks = 1;
    CU(cudaMemsetAsync(ctx->d_cell_acc, 0, (size_t)ctx->ncells * 8, ctx->st));
    CU(cudaMemsetAsync(ctx->d_cell_cnt, 0, (size_t)ctx->ncells * 4, ctx->st));
    int rc = launch_pass(ctx, F_CELLS | (ctx->pending ? F_UPD : 0));
    if (rc) return rc;
    ctx->pending = false;
    CU(cudaMemcpyAsync(cell_sums, ctx->d_cell_acc, (size_t)ctx->ncells * 8, cudaMemcpyDeviceToDevice, ctx->st));
    CU(cudaMemcpyAsync(cell_counts, ctx->d_cell_cnt, (size_t)ctx->ncells * 4, cudaMemcpyDeviceToDevice, ctx->st));
    return M2M_OK;
}

int m2m_shard_prior_finish(m2m_ctx *ctx, const int64_t *cell_sums, const int32_t *cell_counts) {
    if (!ctx || !cell_sums || !cell_counts) return set_err(ctx, M2M_ERR_ARG, "NULL buffer");
    if (!ctx->shard || !ctx->shard_due) return set_err(ctx, M2M_ERR_STATE, "no prior recompute is due");
    const int nb = (ctx->ncells + 255) / 256;
    {
        LaunchTimer lt(ctx, M2M_TK_PRIOR);
        k_prior_mean<<<nb, 256, 0, ctx->st>>>(cell_sums, (const unsigned *)cell_counts, ctx->ncells,
                                              ctx->prec == M2M_FP32C, ldexp(1.0, -ctx->cell_shift), ctx->d_cell_mean);
        CU(cudaGetLastError());
    }
    int g = ctx->nsm * 8;
    const long long need = (ctx->n + 255) / 256;
    if (g > need) g = (int)need;
    {
        LaunchTimer lt(ctx, M2M_TK_PRIOR);
        k_prior_gather<<<g, 256, 0, ctx->st>>>(ctx->d_cell_ids, ctx->d_cell_mean, ctx->what, ctx->d_lnwhat, ctx->n);
        CU(cudaGetLastError());
    }
    ctx->shard_due = false;
    return M2M_OK;
}

int m2m_philox4x32_10(int64_t n, const uint32_t *counters, const uint32_t *keys, uint32_t *out) {
    if (n < 1 || n > (1 << 24) || !counters || !keys || !out) {
        g_init_error = "m2m_philox4x32_10: 1 <= n <= 2^24 and non-NULL arrays";
        return M2M_ERR_ARG;
    }
    const size_t cb = 16 * (size_t)n, kb = 8 * (size_t)n;
    unsigned *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * cb + kb);
    if (e != cudaSuccess) {
        g_init_error = std::string("m2m_philox4x32_10: ") + cudaGetErrorString(e);
        return M2M_ERR_NOMEM;
    }
    unsigned *dc = d, *dk = d + 4 * n, *dout = dk + 2 * n;
    e = cudaMemcpy(dc, counters, cb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, keys, kb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_philox_words<<<(unsigned)((n + 255) / 256), 256>>>(dc, dk, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, cb, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        g_init_error = std::string("m2m_philox4x32_10: ") + cudaGetErrorString(e);
        return M2M_ERR_CUDA;
    }
    return M2M_OK;
}

int m2m_get_obs(m2m_ctx *ctx, double *y, double *Delta, double *Dt) {
    if (!ctx) return M2M_ERR_ARG;
    size_t b = 8 * (size_t)ctx->nobs;
    if (y) CU(cudaMemcpyAsync(y, ctx->d_y, b, cudaMemcpyDeviceToHost, ctx->st));
    if (Delta) CU(cudaMemcpyAsync(Delta, ctx->d_Delta, b, cudaMemcpyDeviceToHost, ctx->st));
    if (Dt) CU(cudaMemcpyAsync(Dt, ctx->d_Dt, b, cudaMemcpyDeviceToHost, ctx->st));
    return check_err_word(ctx);
}

int m2m_get_record(m2m_ctx *ctx, m2m_record *out) {
    if (!ctx || !out) return set_err(ctx, M2M_ERR_ARG, "NULL argument");
    int rc = finish_record(ctx);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, ctx->d_last, sizeof *out, cudaMemcpyDeviceToHost, ctx->st));
    return check_err_word(ctx);
}

int m2m_get_record_async(m2m_ctx *ctx, m2m_record *out) {
    if (!ctx || !out) return set_err(ctx, M2M_ERR_ARG, "NULL argument");
    int rc = finish_record(ctx);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, ctx->d_last, sizeof *out, cudaMemcpyDeviceToHost, ctx->st));
    return M2M_OK;
}

int m2m_get_history(m2m_ctx *ctx, int64_t first, int64_t count, m2m_record *out) {
    if (!ctx || !out || count < 0) return set_err(ctx, M2M_ERR_ARG, "bad argument");
    long long lo = ctx->t - M2M_HISTORY + 1;
    if (lo < 1) lo = 1;
    if (first < lo || first + count - 1 > ctx->t)
        return set_err(ctx, M2M_ERR_ARG, "records [%lld, %lld) not in the ring [%lld, %lld]", (long long)first,
                       (long long)(first + count), lo, ctx->t);
    int rc = finish_record(ctx);
    if (rc) return rc;
    for (int64_t k = 0; k < count;) {
        long long idx = (first + k) % M2M_HISTORY;
        long long run = M2M_HISTORY - idx;
        if (run > count - k) run = count - k;
        CU(cudaMemcpyAsync(out + k, ctx->d_ring + idx, sizeof(m2m_record) * run, cudaMemcpyDeviceToHost, ctx->st));
        k += run;
    }
    return check_err_word(ctx);
}

int m2m_get_cells(m2m_ctx *ctx, int32_t *obs_cells, int32_t *prior_cells) {
    if (!ctx || !obs_cells) return set_err(ctx, M2M_ERR_ARG, "NULL argument");
    if (prior_cells && ctx->prior.kind == M2M_PRIOR_FLAT) return set_err(ctx, M2M_ERR_STATE, "priors are flat");
    if (prior_cells) {
        int rc = launch_pass(ctx, F_MINMAX);
        if (rc) return rc;
    }
    PassArgs a;
    fill_args(ctx, a, 0);
    size_t rs = ctx->prec == M2M_FP32C ? 4 : 8;
    size_t sm = rs * ((ctx->edge_len + 3) & ~3) + rs * ((ctx->prior.nE + 4) & ~3) + rs * ((ctx->prior.nL + 4) & ~3) + 16;
    int g = ctx->nsm * 4;
    long long need = (ctx->n + 255) / 256;
    if (g > need) g = (int)need;
    void *args[] = {&a, &obs_cells, &prior_cells};
    void *fn = ctx->prec == M2M_FP32C ? cells_kernel_f32() : cells_kernel_f64();
    LaunchTimer lt(ctx, M2M_TK_OTHER);
    CU(cudaLaunchKernel(fn, dim3(g), dim3(256), args, sm, ctx->st));
    return M2M_OK;
}

int64_t m2m_nobs(const m2m_ctx *ctx) { return ctx ? ctx->nobs : -1; }
int64_t m2m_steps_taken(const m2m_ctx *ctx) { return ctx ? ctx->t : -1; }

int m2m_set_launch(m2m_ctx *ctx, int32_t threads, int32_t blocks_per_sm) {
    if (!ctx) return M2M_ERR_ARG;
    bool ok = ctx->prec == M2M_FP32C ? (threads == 256 || threads == 512 || threads == 1024)
                                     : (threads == 256 || threads == 512);
    if (!ok || blocks_per_sm < 0 || blocks_per_sm > 4)
        return set_err(ctx, M2M_ERR_ARG, "launch shape %d threads x %d blocks/SM not supported", threads, blocks_per_sm);
    ctx->threads = threads;
    ctx->bps_req = blocks_per_sm;
    return M2M_OK;
}

int m2m_autotune(m2m_ctx *ctx, int32_t steps_per_trial, const char *cache_path, m2m_tuning *out) {
    if (!ctx || !out || steps_per_trial < 1 || steps_per_trial > 10000)
        return set_err(ctx, M2M_ERR_ARG, "bad argument");
    memset(out, 0, sizeof *out);
    // configuration key: what the best launch depends on
    int dev = 0;
    cudaDeviceProp prop;
    CU(cudaGetDevice(&dev));
    CU(cudaGetDeviceProperties(&prop, dev));
    unsigned long long h = 1469598103934665603ull;      // FNV-1a over the shape of the model
    auto mix = [&](long long v) {
        for (int k = 0; k < 8; ++k) { h ^= (unsigned long long)((v >> (8 * k)) & 0xff); h *= 1099511628211ull; }
    };
    mix(ctx->prec); mix(ctx->n); mix(ctx->layout); mix(potential_signature(ctx)); mix(ctx->nobs);
    mix(ctx->prior.kind); mix(ctx->sh_on ? ctx->sh_K * ctx->sh_row : 0); mix(ctx->edge_len); mix(ctx->gh_len);
    snprintf(out->key, sizeof out->key, "%016llx", h);
    std::string devname(prop.name);
    for (char &ch : devname)
        if (ch == '"' || ch == '\\' || ch == '\n') ch = ' ';
    auto valid = [&](int nt, int pl) {
        if (ctx->prec != M2M_FP32C && (nt == 1024 || (pl & 1) || (pl & 2))) return false;
        if ((pl & 1) && !(nt == 1024 && pass_kernel_f32_pipe(ctx->layout))) return false;
        return true;
    };
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof line, f)) {
                if (!strstr(line, out->key)) continue;
                std::string dn = "\"device\": \"" + devname + "\"";
                if (!strstr(line, dn.c_str())) continue;
                const char *pt = strstr(line, "\"threads\": "), *pp = strstr(line, "\"pipeline\": ");
                int nt = 0, pl = 0;
                if (pt && pp && sscanf(pt + 11, "%d", &nt) == 1 && sscanf(pp + 12, "%d", &pl) == 1 && valid(nt, pl)) {
                    ctx->threads = nt;
                    ctx->bps_req = 0;
                    ctx->pipe = (pl & 1) != 0;
                    ctx->fx_atomic = (pl & 2) ? 0 : 1;
                    out->threads = nt; out->pipeline = pl; out->from_cache = 1;
                }
            }
            fclose(f);
            if (out->from_cache) return M2M_OK;
        }
    }
    if (int rc0 = finish_update(ctx)) return rc0;
    const int shapes[] = {1024, 512, 256};
    const int flushes[] = {4, 2, 4 | 1, 2 | 1};
    const bool was_timing = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return set_err(ctx, M2M_ERR_CUDA, "event"); }
    double best = 1e300;
    int bt = ctx->threads, bp = (ctx->pipe ? 1 : 0) | (ctx->fx_atomic ? 4 : 2);
    int rc = M2M_OK;
    for (int nt : shapes) {
        for (int pl : flushes) {
            if (!valid(nt, pl)) continue;
            ctx->threads = nt;
            ctx->bps_req = 0;
            ctx->pipe = (pl & 1) != 0;
            ctx->fx_atomic = (pl & 2) ? 0 : 1;
            rc = m2m_step(ctx, 1);                      // warm-up in this shape
            if (!rc && cudaEventRecord(e0, ctx->st) != cudaSuccess) rc = set_err(ctx, M2M_ERR_CUDA, "event");
            if (!rc) rc = m2m_step(ctx, steps_per_trial);
            if (!rc && cudaEventRecord(e1, ctx->st) != cudaSuccess) rc = set_err(ctx, M2M_ERR_CUDA, "event");
            float ms = 0.f;
            if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = set_err(ctx, M2M_ERR_CUDA, "event timing");
            if (rc) break;
            ++out->candidates;
            const double us = 1e3 * ms / steps_per_trial;
            if (us < best) { best = us; bt = nt; bp = pl; }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = was_timing;
    ctx->threads = bt;
    ctx->bps_req = 0;
    ctx->pipe = (bp & 1) != 0;
    ctx->fx_atomic = (bp & 2) ? 0 : 1;
    if (rc) return rc;
    out->threads = bt; out->pipeline = bp; out->us_per_step = best;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "{\"device\": \"%s\", \"key\": \"%s\", \"threads\": %d, \"pipeline\": %d, \"us_per_step\": %.3f}\n",
                    devname.c_str(), out->key, bt, bp, best);
            fclose(f);
        }
    }
    return check_err_word(ctx);
}

int m2m_set_layout(m2m_ctx *ctx, int32_t layout) {
    if (!ctx) return M2M_ERR_ARG;
    if (layout < 0) layout = detect_layout(ctx);
    if (layout != 0 && layout != detect_layout(ctx))
        return set_err(ctx, M2M_ERR_ARG, "layout %d does not match the observable sets", layout);
    int rc = finish_update(ctx);
    if (rc) return rc;
    if (layout != ctx->layout) ctx->cache_valid = false;
    ctx->layout = layout;
    return M2M_OK;
}

int m2m_set_pipeline(m2m_ctx *ctx, int32_t enable) {
    if (!ctx) return M2M_ERR_ARG;
    ctx->pipe = (enable & 1) != 0;
    if (enable & 2) ctx->fx_atomic = 0;      // FP32C: per-block slots instead of atomics
    if (enable & 4) ctx->fx_atomic = 1;      // FP32C: global integer atomics (default)
    return M2M_OK;
}

int m2m_set_force_cache(m2m_ctx *ctx, int32_t enable) {
    if (!ctx) return M2M_ERR_ARG;
    ctx->facc_off = enable == 0;
    ctx->facc_valid = false;
    return M2M_OK;
}

int m2m_set_persistent(m2m_ctx *ctx, int32_t enable) {
    if (!ctx) return M2M_ERR_ARG;
    int rc = finish_update(ctx);
    if (rc) return rc;
    ctx->persist = enable != 0;
    return M2M_OK;
}

int m2m_test_barrier_stall(m2m_ctx *ctx, int64_t wait_ns) {
    if (!ctx || wait_ns < 1000 || wait_ns > 2000000000ll)
        return set_err(ctx, M2M_ERR_ARG, "wait_ns out of [1e3, 2e9]");
    ctx->test_stall = 1;
    ctx->test_wait_ns = wait_ns;
    return M2M_OK;
}

int m2m_set_timing(m2m_ctx *ctx, int32_t enable) {
    if (!ctx) return M2M_ERR_ARG;
    ctx->timing = enable != 0;
    return M2M_OK;
}

int m2m_get_timing(m2m_ctx *ctx, m2m_timing *out) {
    if (!ctx || !out) return set_err(ctx, M2M_ERR_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    CU(cudaStreamSynchronize(ctx->st));
    for (auto &e : ctx->evs) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, e.a, e.b));
        out->launches[e.kind]++;
        out->ms[e.kind] += ms;
        out->steps[e.kind] += e.steps;
        ctx->ev_free.push_back(e.a);
        ctx->ev_free.push_back(e.b);
    }
    ctx->evs.clear();
    out->kernels_total = ctx->kernels_total;
    ctx->kernels_total = 0;
    return M2M_OK;
}

const char *m2m_last_error(const m2m_ctx *ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

int m2m_free(m2m_ctx *ctx) {
    if (!ctx) return M2M_OK;
    finish_update(ctx);             // the caller's weights: best effort
    cudaStreamSynchronize(ctx->st);
    free_all(ctx);
    delete ctx;
    return M2M_OK;
}

}  // extern "C"

// ======================================================================
// Batches of models
// ======================================================================
struct m2m_batch {
    int prec = 0, nmodels = 0;
    std::vector<m2m_ctx *> ctx;
    cudaStream_t st = nullptr;
    bool fusable = false;        // one launch per stage is possible
    int layout = 0;
    int pk = 0;                  // common potential signature (PK_ANY if they differ)
    int period = 0;              // common moving-prior period (0: flat)
    PassArgs *d_pass = nullptr;  // per-model arguments
    ResArgs *d_res = nullptr;
    int *d_tab = nullptr;        // pass: model, rank, count | residual: model, rank, count
    int pgrid = 0, rgrid = 0;
    int mult = 1;                // pass blocks = mult * SMs * resident blocks (autotuned)
    std::vector<int> pcount, rcount;
    long long *d_step = nullptr; // step counter read by the batched residual
    void *d_gather = nullptr;    // record gather: source pointers, records, error words
    long long t = 0;
    int last_mode = 0;
    std::map<std::tuple<long long, long long, int>, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

int berr(m2m_batch *b, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    g_init_error = buf;
    return code;
}

__global__ void k_add_step(long long *step, long long n) { *step += n; }

void batch_free_all(m2m_batch *b) {
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    for (m2m_ctx *c : b->ctx) m2m_free(c);
    b->ctx.clear();
    void *ptrs[] = {b->d_pass, b->d_res, b->d_tab, b->d_step, b->d_gather};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

// Upload the models' current arguments (potentials may have changed).
int batch_upload(m2m_batch *b) {
    std::vector<PassArgs> pa(b->nmodels);
    std::vector<ResArgs> ra(b->nmodels);
    for (int m = 0; m < b->nmodels; ++m) {
        m2m_ctx *c = b->ctx[m];
        // a fused batch writes and reads the first half of the stat slots
        // and leaves no record to a next pass
        int rc = finish_record(c);
        if (rc) return berr(b, rc, "model %d record: %s", m, c->err.c_str());
        c->stat_par = 0;
        fill_args(c, pa[m], 0);
        ResArgs &r = ra[m];
        memset(&r, 0, sizeof r);
        r.slots = c->d_slots; r.nblk = b->pcount[m]; r.nobs = c->nobs; r.y_acc = c->d_y_acc;
        r.fx_atomic = 1; r.fixed = 1; r.q = c->fx_q;
        r.Y = c->d_Y; r.inv_sigma = c->d_isig; r.Dt = c->d_Dt; r.y = c->d_y; r.Delta = c->d_Delta;
        r.coef_d = c->d_coef_d; r.coef_r = c->d_coef_r; r.r_float = 1;
        r.alpha = c->par.alpha; r.mu = c->par.mu;
        r.stat_slots = c->d_stat_slots; r.stat_nblk = b->pcount[m];
        r.chi_slots = c->d_chi_slots; r.ticket = c->d_ticket;
        r.ring = c->d_ring; r.last = c->d_last;
        r.tail = 1;
        r.err = c->d_err;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_pass, pa.data(), sizeof(PassArgs) * b->nmodels, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_res, ra.data(), sizeof(ResArgs) * b->nmodels, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);   // host staging buffers go out of scope
    if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "batch upload: %s", cudaGetErrorString(e));
    return M2M_OK;
}

size_t batch_smem(const m2m_batch *b, int flags) {
    size_t sm = 0;
    for (m2m_ctx *c : b->ctx) sm = std::max(sm, pass_smem(c, flags));
    return sm;
}

int batch_pass(m2m_batch *b, int flags, int cache_read) {
    BatchPass bp;
    bp.models = b->d_pass;
    bp.blk_model = b->d_tab;
    bp.blk_rank = b->d_tab + b->pgrid;
    bp.blk_count = b->d_tab + 2 * b->pgrid;
    bp.flags = flags;
    bp.cache_read = cache_read;
    bp.cache_write = 1;
    void *args[] = {&bp};
    const bool steady = flags == F_STEADY && cache_read;
    cudaError_t e = cudaLaunchKernel(pass_kernel_f32_batch(b->layout, steady, b->pk), dim3(b->pgrid), dim3(1024), args,
                                     batch_smem(b, flags), b->st);
    if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "batched pass: %s", cudaGetErrorString(e));
    return M2M_OK;
}

// One fused step sequence of nsteps steps starting at step t0 with the
// models' update pending or not.  Records are numbered from *d_step.
int batch_sequence(m2m_batch *b, long long nsteps, long long t0, bool pending) {
    const int *rtab = b->d_tab + 2 * b->pgrid + b->nmodels;   // see the table layout in m2m_batch_init
    for (long long k = 0; k < nsteps; ++k) {
        const long long t1 = t0 + k + 1;
        const bool prior_due = b->period > 0 && (t1 % b->period == 0);
        int fl = F_PUSH | F_SCAT | F_STATS | (pending ? F_UPD : 0) | (prior_due ? F_MINMAX : 0);
        int rc = batch_pass(b, fl, pending ? 1 : 0);
        if (rc) return rc;
        BatchRes br;
        br.models = b->d_res;
        br.blk_model = rtab;
        br.blk_rank = rtab + b->rgrid;
        br.blk_count = rtab + 2 * b->rgrid;
        br.mode = 1;
        br.write_ring = 1;
        br.rec_step = (long long)(k + 1);     // relative: k_residual_batch adds *d_step
        br.step = b->d_step;
        void *args[] = {&br};
        cudaError_t e = cudaLaunchKernel((void *)k_residual_batch, dim3(b->rgrid), dim3(RES_NT_FX), args, 0, b->st);
        if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "batched residual: %s", cudaGetErrorString(e));
        pending = true;
        if (prior_due) {
            for (int m = 0; m < b->nmodels; ++m) {
                m2m_ctx *c = b->ctx[m];
                c->mm_nblocks = b->pcount[m];
                rc = prior_recompute(c, F_UPD);
                if (rc) return berr(b, rc, "model %d priors: %s", m, c->err.c_str());
            }
            pending = false;
        }
    }
    if (pending) {
        int rc = batch_pass(b, F_UPD, 1);
        if (rc) return rc;
    }
    k_add_step<<<1, 1, 0, b->st>>>(b->d_step, nsteps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "step counter: %s", cudaGetErrorString(e));
    return M2M_OK;
}

// Block plan of the fused batch: mult * (SMs x resident blocks) pass blocks
// in proportion to N_m (at least one per model, largest remainders first),
// one residual block per 128 observables of each model; device tables
// [model | rank | count] for the pass, then for the residual.  Drops the
// captured graphs (their launch shapes change).
int batch_plan(m2m_batch *b, int mult) {
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    m2m_ctx *c0 = b->ctx[0];
    const int nmodels = b->nmodels;
    size_t sm = batch_smem(b, F_UPD | F_PUSH | F_SCAT | F_STATS | F_MINMAX);
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pass_kernel_f32_batch(b->layout), 1024, sm);
    if (e != cudaSuccess || occ < 1) {
        b->fusable = false;
        g_init_error = "batched pass does not fit";
        return M2M_OK;
    }
    long long G = (long long)c0->nsm * occ * mult;
    double tot = 0;
    for (m2m_ctx *c : b->ctx) tot += (double)c->n;
    std::vector<double> share(nmodels);
    int used = 0;
    b->pcount.assign(nmodels, 1);
    for (int m = 0; m < nmodels; ++m) {
        share[m] = G * (double)b->ctx[m]->n / tot;
        b->pcount[m] = std::max(1, (int)share[m]);
        long long need = (b->ctx[m]->n + 1023) / 1024;
        b->pcount[m] = (int)std::min<long long>(std::min<long long>(b->pcount[m], need), b->ctx[m]->slot_cap);
        used += b->pcount[m];
    }
    for (int extra = (int)G - used; extra > 0; --extra) {     // largest remainders first
        int best = -1;
        double bestr = 0;
        for (int m = 0; m < nmodels; ++m) {
            long long need = (b->ctx[m]->n + 1023) / 1024;
            if (b->pcount[m] >= need || b->pcount[m] >= b->ctx[m]->slot_cap) continue;
            double r = share[m] - b->pcount[m];
            if (best < 0 || r > bestr) { best = m; bestr = r; }
        }
        if (best < 0) break;
        ++b->pcount[best];
    }
    b->rcount.assign(nmodels, 1);
    for (int m = 0; m < nmodels; ++m) b->rcount[m] = (b->ctx[m]->nobs + RES_NT_FX - 1) / RES_NT_FX;
    b->pgrid = 0;
    for (int m = 0; m < nmodels; ++m) b->pgrid += b->pcount[m];
    b->rgrid = 0;
    for (int m = 0; m < nmodels; ++m) b->rgrid += b->rcount[m];
    std::vector<int> tab, pm_, pr_, rm_, rr_;
    for (int m = 0; m < nmodels; ++m)
        for (int k = 0; k < b->pcount[m]; ++k) { pm_.push_back(m); pr_.push_back(k); }
    for (int m = 0; m < nmodels; ++m)
        for (int k = 0; k < b->rcount[m]; ++k) { rm_.push_back(m); rr_.push_back(k); }
    tab.insert(tab.end(), pm_.begin(), pm_.end());
    tab.insert(tab.end(), pr_.begin(), pr_.end());
    tab.insert(tab.end(), b->pcount.begin(), b->pcount.end());
    tab.insert(tab.end(), rm_.begin(), rm_.end());
    tab.insert(tab.end(), rr_.begin(), rr_.end());
    tab.insert(tab.end(), b->rcount.begin(), b->rcount.end());
    // table layout: pass [model(pgrid) | rank(pgrid) | count(nmodels)],
    // then residual [model(rgrid) | rank(rgrid) | count(nmodels)]
    if (b->d_tab) { cudaFree(b->d_tab); b->d_tab = nullptr; }
    e = cudaMalloc(&b->d_tab, sizeof(int) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b->d_pass) e = cudaMalloc(&b->d_pass, sizeof(PassArgs) * nmodels);
    if (e == cudaSuccess && !b->d_res) e = cudaMalloc(&b->d_res, sizeof(ResArgs) * nmodels);
    if (e == cudaSuccess && !b->d_step) {
        e = cudaMalloc(&b->d_step, sizeof(long long));
        if (e == cudaSuccess) e = cudaMemset(b->d_step, 0, sizeof(long long));
    }
    if (e != cudaSuccess) {
        g_init_error = cudaGetErrorString(e);
        return M2M_ERR_NOMEM;
    }
    b->mult = mult;
    return M2M_OK;
}

}  // namespace

extern "C" {

int m2m_batch_init(m2m_batch **out, int32_t precision, int32_t nmodels, const m2m_model_desc *models,
                   const m2m_params *par, void *stream) {
    if (!out) return berr(nullptr, M2M_ERR_ARG, "batch_out is NULL");
    *out = nullptr;
    if (nmodels < 1 || nmodels > 1024 || !models || !par)
        return berr(nullptr, M2M_ERR_ARG, "nmodels=%d out of [1,1024] or NULL argument", nmodels);
    m2m_batch *b = new m2m_batch();
    b->prec = precision;
    b->nmodels = nmodels;
    b->st = (cudaStream_t)stream;
    for (int m = 0; m < nmodels; ++m) {
        const m2m_model_desc &d = models[m];
        m2m_params pm = *par;
        pm.eps = d.eps;
        m2m_ctx *c = nullptr;
        int rc = m2m_init(&c, precision, d.n, d.x, d.y, d.z, d.vx, d.vy, d.vz, d.w, d.what, d.pot, d.npot, d.obs,
                          d.nsets, d.Y, d.sigma, &pm, d.prior, stream);
        if (rc) {
            std::string msg = g_init_error;
            batch_free_all(b);
            delete b;
            return berr(nullptr, rc, "model %d: %s", m, msg.c_str());
        }
        b->ctx.push_back(c);
    }
    // one launch per stage needs FP32C, one compiled layout and one prior schedule
    m2m_ctx *c0 = b->ctx[0];
    b->fusable = precision == M2M_FP32C && c0->layout != 0;
    b->layout = c0->layout;
    b->pk = potential_signature(c0);
    b->period = c0->prior.kind == M2M_PRIOR_FLAT ? 0 : c0->prior.period;
    for (m2m_ctx *c : b->ctx)
        if (potential_signature(c) != b->pk) b->pk = PK_ANY;
    for (m2m_ctx *c : b->ctx) {
        const int per = c->prior.kind == M2M_PRIOR_FLAT ? 0 : c->prior.period;
        if (c->layout != b->layout || per != b->period || c->sh_on) b->fusable = false;
        for (int k = 0; k < c->nsets; ++k)
            if (c->sets[k].psf_shift) b->fusable = false;   // seeing draws need each model's push count
    }
    if (b->fusable) {
        int rc = batch_plan(b, 1);
        if (rc) {
            batch_free_all(b);
            delete b;
            return berr(nullptr, rc, "batch tables: %s", g_init_error.c_str());
        }
    }
    *out = b;
    return M2M_OK;
}

int m2m_batch_step(m2m_batch *b, int64_t nsteps) {
    if (!b || nsteps < 0) return berr(b, M2M_ERR_ARG, "bad argument");
    if (nsteps == 0) return M2M_OK;
    bool pending = false;
    for (m2m_ctx *c : b->ctx) pending |= c->pending;
    if (!b->fusable || pending) {
        for (int m = 0; m < b->nmodels; ++m) {
            int rc = m2m_step(b->ctx[m], nsteps);
            if (rc) return berr(b, rc, "model %d: %s", m, b->ctx[m]->err.c_str());
        }
        b->t += nsteps;
        b->last_mode = 0;
        return M2M_OK;
    }
    // cell caches valid for every model (their last pass scattered)?
    bool cache_ok = true;
    for (m2m_ctx *c : b->ctx) cache_ok &= c->cache_valid;
    if (!cache_ok) {
        for (m2m_ctx *c : b->ctx) {     // one scatter at the current state refreshes the caches
            int rc = m2m_observe(c, 0);
            if (rc) return berr(b, rc, "cache refresh: %s", c->err.c_str());
        }
    }
    int rc = batch_upload(b);
    if (rc) return rc;
    // step counter of the records: the models' common step count
    long long t0 = b->ctx[0]->t;
    cudaError_t e = cudaMemcpyAsync(b->d_step, &t0, sizeof t0, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "step counter: %s", cudaGetErrorString(e));
    const bool graphable = b->st != nullptr && b->st != cudaStreamLegacy && b->st != cudaStreamPerThread;
    const auto key = std::make_tuple((long long)nsteps, b->period ? t0 % b->period : 0ll, 0);
    bool launched = false;
    if (graphable) {
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            for (m2m_ctx *c : b->ctx) c->timing = false;   // events are not captured
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = batch_sequence(b, nsteps, t0, false);
                cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
                if (rc) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) {
                b->graphs[key] = ge;
                it = b->graphs.find(key);
            } else {
                cudaGetLastError();
            }
        }
        if (it != b->graphs.end()) {
            e = cudaGraphLaunch(it->second, b->st);
            if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
            launched = true;
            b->last_mode = 2;
        }
    }
    if (!launched) {
        rc = batch_sequence(b, nsteps, t0, false);
        if (rc) return rc;
        b->last_mode = 1;
    }
    for (int m = 0; m < b->nmodels; ++m) {
        m2m_ctx *c = b->ctx[m];
        c->t = t0 + nsteps;
        c->epoch += nsteps;                  // one push per step
        c->pending = false;
        c->cache_valid = true;
        c->last_grid = b->pcount[m];
    }
    b->t += nsteps;
    return M2M_OK;
}

int m2m_batch_autotune(m2m_batch *b, int32_t steps_per_trial, m2m_tuning *out) {
    if (!b || !out || steps_per_trial < 1 || steps_per_trial > 10000) return berr(b, M2M_ERR_ARG, "bad argument");
    memset(out, 0, sizeof *out);
    out->threads = 1024;
    out->pipeline = 4;
    if (!b->fusable) return M2M_OK;           // stepped model by model: nothing to tune here
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return berr(b, M2M_ERR_CUDA, "event");
    }
    double best = 1e300;
    int bm = b->mult, rc = M2M_OK;
    for (int mult : {1, 2, 4}) {
        rc = batch_plan(b, mult);
        if (rc || !b->fusable) break;
        rc = m2m_batch_step(b, steps_per_trial);        // warm-up: captures this plan's graph
        if (!rc && cudaEventRecord(e0, b->st) != cudaSuccess) rc = berr(b, M2M_ERR_CUDA, "event");
        if (!rc) rc = m2m_batch_step(b, steps_per_trial);
        if (!rc && cudaEventRecord(e1, b->st) != cudaSuccess) rc = berr(b, M2M_ERR_CUDA, "event");
        float ms = 0.f;
        if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = berr(b, M2M_ERR_CUDA, "event timing");
        if (rc) break;
        ++out->candidates;
        const double us = 1e3 * ms / steps_per_trial;
        if (us < best) { best = us; bm = mult; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = batch_plan(b, bm);
    if (rc) return berr(b, rc, "batch tables: %s", g_init_error.c_str());
    out->us_per_step = best;
    out->threads = 1024;
    snprintf(out->key, sizeof out->key, "pass blocks x%d", bm);
    return M2M_OK;
}

int m2m_batch_context(m2m_batch *b, int32_t model, m2m_ctx **ctx_out) {
    if (!b || !ctx_out || model < 0 || model >= b->nmodels) return berr(b, M2M_ERR_ARG, "bad model index");
    *ctx_out = b->ctx[model];
    return M2M_OK;
}

int m2m_batch_fused(const m2m_batch *b) { return b ? b->last_mode : -1; }

int m2m_batch_get_records(m2m_batch *b, m2m_record *out) {
    if (!b || !out) return berr(b, M2M_ERR_ARG, "NULL argument");
    const int n = b->nmodels;
    // device scratch: record pointers, error-word pointers, records, error words
    const size_t o_err = 8 * (size_t)n, o_rec = 16 * (size_t)n, o_w = o_rec + sizeof(m2m_record) * n;
    const size_t bytes = o_w + 4 * (size_t)n;
    if (!b->d_gather) {
        if (cudaMalloc(&b->d_gather, bytes) != cudaSuccess) return berr(b, M2M_ERR_NOMEM, "cudaMalloc(%zu)", bytes);
        std::vector<const void *> ptr(2 * (size_t)n);
        for (int m = 0; m < n; ++m) { ptr[m] = b->ctx[m]->d_last; ptr[n + m] = b->ctx[m]->d_err; }
        if (cudaMemcpy(b->d_gather, ptr.data(), 16 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
            return berr(b, M2M_ERR_CUDA, "record gather table");
    }
    for (int m = 0; m < n; ++m) {
        // records a model's next pass would write (models stepped one by one)
        int rc = finish_record(b->ctx[m]);
        if (rc) return berr(b, rc, "model %d record: %s", m, b->ctx[m]->err.c_str());
    }
    unsigned char *g = (unsigned char *)b->d_gather;
    k_gather_records<<<(n + 127) / 128, 128, 0, b->st>>>((const m2m_record *const *)g, (const int *const *)(g + o_err),
                                                         n, (m2m_record *)(g + o_rec), (int *)(g + o_w));
    std::vector<int> errw(n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, g + o_rec, sizeof(m2m_record) * n, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(errw.data(), g + o_w, 4 * (size_t)n, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return berr(b, M2M_ERR_CUDA, "record gather: %s", cudaGetErrorString(e));
    for (int m = 0; m < n; ++m)
        if (errw[m]) return berr(b, check_err_word(b->ctx[m]), "model %d: %s", m, b->ctx[m]->err.c_str());
    return M2M_OK;
}

int m2m_batch_free(m2m_batch *b) {
    if (!b) return M2M_OK;
    cudaStreamSynchronize(b->st);
    batch_free_all(b);
    delete b;
    return M2M_OK;
}

}  // extern "C"
