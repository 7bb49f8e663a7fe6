/*
 * m2m.h -- C-ABI of libm2m.so, a GB300 (sm_103a) implementation of the
 * made-to-measure (M2M) particle-model training step of Morganti & Gerhard
 * (2012, arXiv:1207.6403).
 *
 * Section 2 of the paper: the weights w_i of an N-body model are adapted,
 * while its particles orbit in the potential, until its observables match
 * target values Y_j with errors sigma_j: F = -1/2 chi^2 + mu S (Eq. 1) with
 * S = -sum_i w_i ln(w_i/w_hat_i) (Eq. 2) is maximised.  Section 2.1: the
 * priors w_hat_i are flat (1/N) or moving: the mean weight of the
 * particles that share a cell of integral-of-motion space.
 *
 * One step t -> t+1 (the order every entry point below follows):
 *   1. kick-drift-kick leapfrog push of every particle in the potential;
 *   2. scatter y_j = sum_i w_i K_j(x_i, v_i) at the new positions;
 *   3. Delta_j = (y_j - Y_j)/sigma_j, smoothed Delta~_j <- alpha Delta_j +
 *      (1 - alpha) Delta~_j, chi^2 = sum_j Delta~_j^2;
 *   4. w_i <- w_i exp(eps dt G_i), G_i = mu (-ln(w_i/w_hat_i) - c)
 *      - sum_j K_ij Delta~_j / sigma_j  (c = entropy_const, 1 for Eq. 2);
 *   5. moving priors every `period` steps.
 *
 * Conventions common to all calls
 *  - Every call returns an int status (M2M_OK = 0 or a negative M2M_ERR_*);
 *    nothing aborts or throws across the ABI.  m2m_last_error() gives text.
 *  - Work is enqueued on the stream given to m2m_init; calls return without
 *    synchronising except those that return host values (m2m_get_*).
 *  - Particle arrays are CALLER-OWNED DEVICE memory, borrowed until
 *    m2m_free: positions x,y,z and velocities vx,vy,vz are float (M2M_FP32C)
 *    or double (M2M_FP64) arrays of n elements, each 16-byte aligned; w and
 *    w_hat are double arrays of n elements, 16-byte aligned, w_hat_i > 0.
 *  - Host arrays passed in descriptors (edges, targets, GH parameters) are
 *    copied during the call; the caller may free them afterwards.
 *  - Scratch memory (partial histograms, cell tables) is library-owned,
 *    allocated in m2m_init and freed by m2m_free.
 *  - Errors found by kernels (non-finite weights, fixed-point overflow) are
 *    sticky and reported by the next m2m_get_* call.
 *  - Every scatter records each particle's cells (library-owned, 4 bytes per
 *    particle) so that the next weight update need not look them up again.
 *    A caller that changes x..vz itself (not through m2m_step/m2m_push)
 *    must call m2m_observe before the next m2m_update_weights.
 *  - With a self-consistent expansion potential (SH, SH_TRI) every push
 *    keeps the force at the new positions (library-owned, 3 values of the
 *    state precision per particle) and the next push starts from it instead
 *    of evaluating the expansion again; a recompute of the expansion drops
 *    it.  A caller that changes x..z itself must call m2m_observe (which
 *    drops it too) before the next push.
 *  - M2M_FP32C keeps ln w_hat_i per particle in float (library-owned, 4
 *    bytes per particle) for the weight update; it is taken from w_hat at
 *    m2m_init and rewritten with w_hat at every prior recompute.  A caller
 *    that writes w_hat itself must do so before m2m_init (or call
 *    m2m_priors, which overwrites both).
 */
#ifndef M2M_H
#define M2M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m2m_ctx m2m_ctx;          /* opaque, library-owned */

#define M2M_OK             0
#define M2M_ERR_ARG       -1   /* invalid argument, size or alignment */
#define M2M_ERR_CUDA      -2   /* a CUDA runtime call failed */
#define M2M_ERR_NONFINITE -3   /* a weight became non-finite or negative */
#define M2M_ERR_TIMEOUT   -4   /* a bounded device-side wait ran out */
#define M2M_ERR_STATE     -5   /* call not valid in the context's state */
#define M2M_ERR_NOMEM     -6   /* device allocation failed */
#define M2M_ERR_OVERFLOW  -7   /* fixed-point histogram range exceeded */

/* Arithmetic of the particle path.
 * M2M_FP64:  positions, push, bins and kernels in double; double sums.
 * M2M_FP32C: positions, push, bins and kernels in float; weights stored and
 *   updated in double; histogram sums exact in 64-bit fixed point
 *   (resolution 2^-25 of the initial average weight, i.e. 2^-25 *
 *   2^ceil(log2 sum w) / 2^ceil(log2 n)); chi^2, entropy and the
 *   prior-cell means reduced in double. */
#define M2M_FP64  0
#define M2M_FP32C 1

/* ---- potential: Phi = sum of up to M2M_MAX_POT components (G = 1) ----
 * HERNQUIST p = {GM, a}:        Phi = -GM/(r+a)
 * NFW       p = {rho_s, r_s}:   Phi = -4 pi rho_s r_s^3 ln(1+r/r_s)/r
 * LOG       p = {v0, Rc, q}:    Phi = 1/2 v0^2 ln(Rc^2 + R^2 + z^2/q^2)
 * SH        p = {K, rmin, rmax, period}: the potential of the weighted
 *           particles themselves (Sections 1 and 2: the potential may
 *           also be derived from the moving particles), as the
 *           axisymmetric multipole expansion with even l = 0..8,
 *             Phi = -sum_l P_l(cos theta) [A_l(r)/r^(l+1) + B_l(r) r^l],
 *             A_l(r) = sum_{r_i < r} w_i P_l r_i^l,
 *             B_l(r) = sum_{r <= r_i < rmax} w_i P_l r_i^-(l+1),
 *           tabulated at K (4..512, integer) nodes r_k = rmin
 *           (rmax/rmin)^(k/(K-1)) and interpolated linearly in r between
 *           them (exterior multipole law beyond rmax, interior solution
 *           inside rmin).  Which side of node k a particle is on is decided
 *           by its r^2 against r_k^2, like the shells.  Side sums: FP32C
 *           exact 64-bit fixed point of the float terms (resolution 2^-31
 *           of the initial average weight), FP64 double sums; the tables
 *           are built in double.  Recomputed from
 *           (x_{t+1}, w_{t+1}) after the update of every step t+1 that is a
 *           multiple of `period` (integer >= 1), at m2m_init and by
 *           m2m_potential.  At most one SH component, listed last; added
 *           after the analytic ones.  Errors: M2M_ERR_ARG for bad p.
 *   SH_TRI  p = {K, rmin, rmax, period}: the triaxial generalisation of SH
 *           (Section 2's self-consistent potential for models without a
 *           symmetry axis): the real harmonics of even l <= 8 and even
 *           m >= 0 (the terms a set mirror-symmetric about the three
 *           coordinate planes has), with n = x/r, mu = n_z, u = n_x + i n_y
 *             Y_lm = c_lm Q_l^m(mu) Re u^m,  Q_l^m = d^m P_l/dmu^m,
 *             c_l0 = N_l0, c_lm = sqrt(2) N_lm,
 *             N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
 *             Phi = -sum_lm Y_lm F_lm(r),
 *             F_lm(r) = 4 pi/(2l+1) [A_lm(r)/r^(l+1) + B_lm(r) r^l],
 *           A_lm, B_lm the sums of w_i Y_lm(x_i) r_i^l and w_i Y_lm(x_i)
 *           r_i^-(l+1) inside / outside r; nodes, interpolation, side sums,
 *           schedule and placement as for SH.
 *   SH_FULL p = {K, rmin, rmax, period}: the same for models with no
 *           symmetry: every term up to l = 4, t = l*l + l + m for
 *           m = -l..l (25 terms), Y_lm = c_l|m| Q_l^|m|(mu) C_m with
 *           C_m = Re u^m for m >= 0 and Im u^|m| for m < 0. */
#define M2M_MAX_POT 4
#define M2M_POT_HERNQUIST 1
#define M2M_POT_NFW       2
#define M2M_POT_LOG       3
#define M2M_POT_SH        4
#define M2M_POT_SH_TRI    5
#define M2M_POT_SH_FULL   6
#define M2M_SH_ROW        21   /* values per node in m2m_get_sh_table (SH) */
#define M2M_TRI_ROW       61   /* values per node in m2m_get_sh_table (SH_TRI) */
#define M2M_FULL_ROW      101  /* values per node in m2m_get_sh_table (SH_FULL) */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double p[4];
} m2m_potential_desc;

/* ---- observables: up to M2M_MAX_SETS sets, concatenated ----
 * The observables of Section 1-2 (photometry, absorption-line kinematics).
 * geom SHELL:   3D shells, cells by edges of r^2 = (x*x + y*y) + z*z
 *      ANNULUS: projected annuli, edges of R^2 = X*X + Y*Y
 *      GRID:    sky rectangles (pixels, IFU apertures), edges of X and of Y,
 *               cell = iy*nx + ix
 *      LUT:     sky apertures of any shape (Voronoi-binned IFU spaxels,
 *               long-slit segments): the sky pixel (ix, iy) by the edges of
 *               X and of Y as for GRID, then cell = lut[iy*nx + ix] (-1: no
 *               cell); the apertures are cells 0..ncell-1
 * Sky coordinates for the line of sight s = (0, sin i, cos i):
 *   X = x, Y = z*sin_i - y*cos_i, v_los = vy*sin_i + vz*cos_i.
 * quant MASS:  K = 1;  VLOS2: K = v_los^2;
 *       GH:    K_n, n=0..4 = Gauss-Hermite kernels (van der Marel & Franx
 *              1993 normalisation) about (gh_V, gh_S) of the cell, smoothed
 *              by a Gaussian velocity kernel of width sigma_kernel.
 * Membership: value v is in cell j iff edge_j <= v < edge_{j+1}, compared
 * exactly (float values against the double edges), else in no cell.
 * Observable index inside a set: cell*nmom + n (nmom = 5 for GH, else 1). */
#define M2M_MAX_SETS 4
#define M2M_GEOM_SHELL   1
#define M2M_GEOM_ANNULUS 2
#define M2M_GEOM_GRID    3
#define M2M_GEOM_LUT     4
#define M2M_MAX_LUT_PIXELS (1 << 22)   /* lookup-table pixels of all LUT sets */
#define M2M_Q_MASS  1
#define M2M_Q_VLOS2 2
#define M2M_Q_GH    3
typedef struct {
    int32_t geom, quant;
    int32_t nx, ny;             /* ny = 1 unless GRID or LUT */
    const double *edges_x;      /* host, nx+1 strictly increasing */
    const double *edges_y;      /* host, ny+1 (GRID, LUT) or NULL */
    const double *gh_V;         /* host, one per cell (GH) or NULL */
    const double *gh_S;         /* host, one per cell (GH), > 0, or NULL */
    double sigma_kernel;        /* GH velocity kernel width (>= 0) */
    const int32_t *lut;         /* LUT: host, nx*ny cell ids in [-1, ncell); else NULL */
    int32_t ncell;              /* LUT: number of cells (apertures); else ignored */
    /* Seeing (ANNULUS, GRID, LUT only; NULL = none): a host table of
     * 2^psf_bits displacement quantiles of the PSF along one sky axis
     * (finite, non-decreasing; rounded once to the state precision).  Each
     * time the cells of particle i (its index in the arrays) are evaluated
     * at positions that have had e pushes (e counts every push since
     * m2m_init), its sky position becomes (X + q[u0 >> (32 - psf_bits)],
     * Y + q[u1 >> (32 - psf_bits)]), the sums in the state precision, where
     * (u0, u1, -, -) = Philox4x32-10 (Salmon et al. 2011, 10 rounds) of the
     * counter (i, e mod 2^32, set index, e >> 32) under the key
     * (psf_seed, 0): the same draw for the scatter and for the weight
     * update at those positions.  Sets with a PSF take the run-time set
     * walk. */
    const double *psf_q;
    int32_t psf_bits;           /* 1..16 */
    uint32_t psf_seed;
} m2m_obs_desc;

/* ---- priors (Section 2.1) ----
 * FLAT: w_hat stays as passed.
 * E_LC: every `period` steps, w_hat_i = mean w over i's cell of an nE x nL
 *       grid in (E, L^2/Lc^2(E)) for the Hernquist (GM, a) circular orbit;
 *       E cells uniform on [min E, 0), unbound particles in one extra cell.
 * E_LZ: the same on an nE x nL grid in (E, L_z) uniform on
 *       [min E, max E] x [-max|L_z|, max|L_z|].
 * E_L2: the same on an nE x nL grid in (E, L^2) uniform on
 *       [min E, max E] x [0, max L^2], L^2 = (Lx*Lx + Ly*Ly) + Lz*Lz: cells
 *       of integrals that hold (E) or nearly hold (L^2) where the potential
 *       has no symmetry axis (triaxial models, where L_z is not conserved).
 * E = 1/2 v^2 + Phi(x) in the state precision. */
#define M2M_PRIOR_FLAT 0
#define M2M_PRIOR_E_LC 1
#define M2M_PRIOR_E_LZ 2
#define M2M_PRIOR_E_L2 3
typedef struct {
    int32_t kind, nE, nL, period;
    double hernquist_GM, hernquist_a;
} m2m_prior_desc;

/* ---- step parameters ---- */
typedef struct {
    double eps;             /* weight-adaptation rate (already divided by N if wanted) */
    double mu;              /* entropy weight of Eq. 1 */
    double dt;              /* leapfrog time step */
    double alpha;           /* smoothing: Delta~ <- alpha Delta + (1-alpha) Delta~ */
    double entropy_const;   /* c in dS/dw_i = -ln(w_i/w_hat_i) - c (1 = Eq. 2) */
    double incl_sin, incl_cos;
} m2m_params;

/* One record per step t: chi^2 of Delta~ and of Delta after the step's
 * scatter, and S, sum w of the weights that produced that scatter;
 * F = -1/2 chi2 + mu S. */
typedef struct {
    int64_t step;
    double chi2, chi2_raw, S, sum_w, F;
    double max_abs_dt;       /* max_j |Delta~_j| */
} m2m_record;

/* Create a context.  Validates all sizes and alignments (M2M_ERR_ARG),
 * copies the tables, runs an initial scatter at (x_0, w_0) and sets
 * Delta~ = Delta (as the first step's smoothing state).
 *   ctx_out      receives the context (NULL on error)
 *   precision    M2M_FP64 or M2M_FP32C (type of x..vz)
 *   n            particle count, 1 <= n < 2^31
 *   x..vz, w, what  caller-owned device arrays (see conventions)
 *   pot, npot    potential components (0 <= npot <= M2M_MAX_POT)
 *   obs, nsets   observable sets (1 <= nsets <= M2M_MAX_SETS), total
 *                observables <= 8192
 *   Y, sigma     host arrays of the total observable count, or NULL (all
 *                masked: sigma_j <= 0 masks observable j)
 *   par          step parameters;  prior: NULL means FLAT
 *   stream       cudaStream_t to enqueue on (NULL = default stream)
 * Cites: Section 2, Eq. 1-2; Section 2.1 (priors). */
int m2m_init(m2m_ctx **ctx_out, int32_t precision, int64_t n,
             void *x, void *y, void *z, void *vx, void *vy, void *vz,
             double *w, double *what,
             const m2m_potential_desc *pot, int32_t npot,
             const m2m_obs_desc *obs, int32_t nsets,
             const double *Y, const double *sigma,
             const m2m_params *par, const m2m_prior_desc *prior,
             void *stream);

/* Replace targets and errors (host arrays of the observable count; sigma
 * <= 0 masks).  Cites Section 2 (observables with errors). */
int m2m_set_targets(m2m_ctx *ctx, const double *Y, const double *sigma);

/* Replace the potential (fixed, known potential of Section 2; an SH
 * component is expanded at once from the current positions and weights,
 * after a pending weight update is applied). */
int m2m_potential(m2m_ctx *ctx, const m2m_potential_desc *pot, int32_t npot);

/* Copy the SH node table to host memory as doubles, K rows of M2M_SH_ROW:
 * F_l(r_k) for l = 0,2,4,6,8; the slopes of F_l to node k+1; D_l(r_k) =
 * dF_l/dr; the slopes of D_l; r_k (last row: zero slopes).  Phi =
 * -sum P_l F_l.  out must hold K * M2M_SH_ROW doubles.  For SH_TRI: K rows
 * of M2M_TRI_ROW, the same five blocks with the 15 terms (l, m) = (0,0),
 * (2,0), (2,2), (4,0), .., (8,8) each (F_lm, slopes, D_lm, slopes, r_k);
 * out must hold K * M2M_TRI_ROW doubles.  For SH_FULL: K rows of
 * M2M_FULL_ROW, the blocks of its 25 terms in the order t = l*l + l + m;
 * out must hold K * M2M_FULL_ROW doubles.  Synchronises.
 * M2M_ERR_STATE if the potential has no SH or SH_TRI component. */
int m2m_get_sh_table(m2m_ctx *ctx, double *out);

/* Scatter + residual at the current state, no push and no weight change.
 * mode 0: compute y and Delta only (Delta~ untouched);
 * mode 1: also smooth Delta~ <- alpha Delta + (1-alpha) Delta~;
 * mode 2: also reset Delta~ = Delta.  Writes a record (step unchanged). */
int m2m_observe(m2m_ctx *ctx, int32_t mode);

/* Weight update (step 4) with the current Delta~ at the current positions:
 * w_i <- w_i exp(eps dt G_i).  Cites Eq. 1-2 and the adaptation
 * prescription that follows them. */
int m2m_update_weights(m2m_ctx *ctx);

/* Moving-prior recompute now (step 5) from the current positions and
 * weights; M2M_ERR_STATE for FLAT priors.  Cites Section 2.1. */
int m2m_priors(m2m_ctx *ctx);

/* KDK leapfrog push only, nsteps times (step 1). */
int m2m_push(m2m_ctx *ctx, int64_t nsteps);

/* nsteps full M2M steps (1-5 above).  On return the particle arrays, w and
 * w_hat hold the state after the last step (unless lazy weight updates are
 * on: see m2m_set_lazy_update). */
int m2m_step(m2m_ctx *ctx, int64_t nsteps);

/* Lazy weight updates (on != 0; default off).  The weight update of a step
 * (Eq. 2, at the positions the step's scatter used) is fused into the next
 * step's particle pass; with lazy updates on, m2m_step leaves the update of
 * its last step pending instead of applying it with an update-only pass
 * before it returns, so that a caller stepping once per call (reading each
 * step's record, say) pays one pass per step.  A pending update is applied
 * by the next m2m_step, by m2m_finish_update, and first thing by every call
 * that reads or changes the particle state (m2m_observe,
 * m2m_update_weights, m2m_priors, m2m_push, m2m_potential, m2m_set_layout,
 * m2m_autotune, m2m_free), and when lazy updates are turned off.  Until
 * then the caller's w array holds the weights before that update: call
 * m2m_finish_update before reading it directly.  Records, observables and
 * chi^2 of every step are complete either way, and the state after
 * m2m_finish_update is bit-identical to stepping without lazy updates. */
int m2m_set_lazy_update(m2m_ctx *ctx, int32_t on);

/* Apply a pending weight update now (nothing if none is pending).
 * Asynchronous on the context's stream. */
int m2m_finish_update(m2m_ctx *ctx);

/* Velocity-ellipsoid moments of the weighted particles in spherical shells
 * (an analysis of the model, not a step: the anisotropy beta(r) of the
 * recovery experiment of Section 3).  r2_edges: host, nshell+1 strictly
 * increasing edges of r^2 (1 <= nshell <= 1024; membership as for SHELL
 * sets, r^2 = (x*x + y*y) + z*z in the state precision).  out: host,
 * 4*nshell doubles, per shell sum w, sum w v_r^2, sum w v_theta^2,
 * sum w v_phi^2 with v_r = x.v/r, v_phi = (x vy - y vx)/R, v_theta^2 =
 * v^2 - v_r^2 - v_phi^2 in double from the stored state (v_r = 0 at r = 0,
 * v_phi = 0 at R = 0); the sums are double atomics (order-dependent at
 * rounding level).  Applies a pending weight update first.  Synchronises. */
int m2m_velocity_moments(m2m_ctx *ctx, const double *r2_edges, int32_t nshell, double *out);

/* The counter-based generator of the seeing draws (Philox4x32-10, Salmon
 * et al. 2011; see m2m_obs_desc), evaluated by the same device routine the
 * scatter uses, for n given counters and keys: a check of the device
 * generator against the generator's published known-answer vectors.
 *   counters  host, 4n uint32 (words c0..c3 of draw k at 4k..4k+3)
 *   keys      host, 2n uint32 (k0, k1 of draw k at 2k, 2k+1)
 *   out       host, 4n uint32 (the four output words of each draw)
 * 1 <= n <= 2^24.  Runs on the current device and synchronises; allocates
 * and frees its own device buffers.  Errors: M2M_ERR_ARG, M2M_ERR_NOMEM,
 * M2M_ERR_CUDA (text in m2m_last_error(NULL)). */
int m2m_philox4x32_10(int64_t n, const uint32_t *counters, const uint32_t *keys, uint32_t *out);

/* Host copies (synchronise the stream).  Any pointer may be NULL.
 * y, Delta, Dt: observable count doubles (last scatter).  Returns the
 * sticky kernel error if one was raised. */
int m2m_get_obs(m2m_ctx *ctx, double *y, double *Delta, double *Dt);

/* Last record and the number of records available in the ring
 * (capacity M2M_HISTORY). */
#define M2M_HISTORY 16384
int m2m_get_record(m2m_ctx *ctx, m2m_record *out);

/* The last record, copied on the context's stream without waiting for it:
 * the copy is enqueued after the work of every call made so far, and *out
 * holds the record once the stream has reached it (an event recorded after
 * this call, or a synchronisation).  out should be page-locked host memory
 * (from pageable memory the copy runs synchronously, by CUDA's rules).
 * No error-word check: a sticky kernel error is returned by the next
 * synchronising call (m2m_get_record, m2m_get_obs).  For loops that read
 * each step's record while the next step runs. */
int m2m_get_record_async(m2m_ctx *ctx, m2m_record *out);

/* Records for steps [first, first+count) still in the ring, to host. */
int m2m_get_history(m2m_ctx *ctx, int64_t first, int64_t count, m2m_record *out);

/* Cell index of every particle at the current positions, to caller-owned
 * DEVICE int32 arrays: obs_cells[s*n + i] for set s (-1 = none) and, if
 * prior_cells is not NULL and priors are moving, the prior cell of i from
 * the current positions (grid bounds from the current particles). */
int m2m_get_cells(m2m_ctx *ctx, int32_t *obs_cells, int32_t *prior_cells);

/* Sizes. */
int64_t m2m_nobs(const m2m_ctx *ctx);
int64_t m2m_steps_taken(const m2m_ctx *ctx);

/* Launch shape of the particle kernels: threads per block (FP32C: 256, 512
 * or 1024 (default; the pipelined pass needs 1024); FP64: 256 (default) or
 * 512) and blocks per SM (0 = as many as fit, at most 4).  Takes effect on
 * the next launch. */
int m2m_set_launch(m2m_ctx *ctx, int32_t threads, int32_t blocks_per_sm);

/* Observable layout of the particle kernels: the common set combinations
 * (1: pixels + IFU GH apertures; 2: shells + GH annuli; 3: shells + mass
 * and v_los^2 annuli; 4, FP32C only: pixels + two lookup-table GH sets, with
 * or without seeing) run as code compiled for them when every edge table is
 * uniform in value or in log; anything else, and seeing outside layout 4,
 * walks the sets at run time.  layout -1: automatic (the default); 0:
 * force the run-time walk; 1-4: the compiled layout, only if it matches
 * (else M2M_ERR_ARG).  FP32C results are identical either way. */
int m2m_set_layout(m2m_ctx *ctx, int32_t layout);

/* Streaming and reduction options of the FP32C passes (bit flags):
 *  1: stream the particles of the compiled layouts through a block-level
 *     pipeline: one thread of each block stages the block's next chunk of
 *     1024 consecutive particles into shared memory with one bulk copy
 *     (TMA) per array, completing on an mbarrier, while the block computes
 *     the current chunk (default off: plain loads with a one-particle
 *     register prefetch);
 *  2: flush each block's exact histogram to a per-block slot reduced by the
 *     residual kernel;
 *  4: flush it with 64-bit integer atomics into the totals (default).
 * All combinations give bit-identical results. */
int m2m_set_pipeline(m2m_ctx *ctx, int32_t enable);

/* ---- autotuning (no counterpart in the paper: a property of this
 * implementation) ----
 * Chooses the pass launch shape (1024, 512 or 256 threads; FP64: 512, 256)
 * and the histogram privatisation (per-block shared-memory histograms
 * flushed by global integer atomics, or to per-block slots reduced by the
 * residual) and, FP32C with a compiled layout, the bulk-copy pipeline, by
 * timing real steps of the live model: each candidate advances the model
 * by steps_per_trial steps (1..10000), so the call advances it by
 * out->candidates * steps_per_trial steps in all.  FP32C: every candidate
 * yields the same positions, weights and observables (exact histogram
 * sums); only S and sum w in the records, reduced in float per thread,
 * move at rounding level.  FP64: results move at rounding level.
 * cache_path (may be NULL): a JSON-lines file; an entry with this
 * device's name and the model's configuration key is applied without
 * timing (out->from_cache = 1, nothing is advanced), a new choice is
 * appended.  Synchronises. */
typedef struct {
    int32_t threads;          /* chosen pass block size */
    int32_t pipeline;         /* chosen m2m_set_pipeline flags */
    double us_per_step;       /* its measured time per step (0 from the cache) */
    int32_t candidates;       /* configurations timed */
    int32_t from_cache;       /* 1: taken from cache_path */
    char key[64];             /* the configuration key */
} m2m_tuning;
int m2m_autotune(m2m_ctx *ctx, int32_t steps_per_trial, const char *cache_path, m2m_tuning *out);

/* Keep the force of a self-consistent expansion potential between pushes
 * (default 1; see the conventions at the top): 0 evaluates the expansion
 * twice per push, at the old and at the new positions.  The kept force is
 * the same function of the same positions and node table, so the results
 * are bit-identical either way.  Applies from the next push. */
int m2m_set_force_cache(m2m_ctx *ctx, int32_t enable);

/* Persistent multi-step launches (on by default).  Where they apply -- an
 * M2M_FP32C context with a compiled observable layout and potential
 * signature (m2m_set_layout), no spherical-harmonic component, 1024-thread
 * passes with integer-atomic histogram flushes (m2m_set_launch,
 * m2m_set_pipeline), room for one block per SM -- m2m_step advances the
 * steps up to the next prior recompute in one cooperative launch: one block
 * per SM, each with a fixed range of particles, the residual of each step
 * computed between two grid-wide barriers.  The state equals, bit for bit,
 * that of the same steps taken as separate pass and residual launches
 * (enable = 0).  Every barrier wait is bounded (2 s); a wait that runs out
 * records M2M_ERR_TIMEOUT, returned by the next synchronising call. */
int m2m_set_persistent(m2m_ctx *ctx, int32_t enable);

/* Test only: the next persistent launch runs with its block 0 not arriving
 * at the launch's first grid barrier, and with every barrier wait of that
 * launch limited to wait_ns nanoseconds, so that the other blocks' waits
 * run out: the launch records M2M_ERR_TIMEOUT (its results are invalid) and
 * the next synchronising call returns it.  Nothing waits longer than the
 * limit; no copy or other device operation is left outstanding. */
int m2m_test_barrier_stall(m2m_ctx *ctx, int64_t wait_ns);

/* Device timing of the library's own launches, by kernel class, with CUDA
 * events recorded on the context's stream around every launch while
 * enabled.  Classes: */
#define M2M_TK_STEP_UPD  0   /* step pass that also applies the pending update */
#define M2M_TK_STEP      1   /* step pass without a pending update */
#define M2M_TK_RESIDUAL  2   /* residual / chi^2 / record */
#define M2M_TK_UPDATE    3   /* update-only pass (end of a call, m2m_update_weights) */
#define M2M_TK_PRIOR     4   /* update + prior-cell pass, cell means, gather */
#define M2M_TK_OTHER     5   /* observe, push, range and cell-export passes */
#define M2M_TK_SH        6   /* spherical-harmonic side sums and node table */
#define M2M_TK_STEPS     7   /* persistent multi-step launches (see m2m_set_persistent) */
#define M2M_TK_N         8
typedef struct {
    int64_t launches[M2M_TK_N];  /* launches timed since the last read */
    double ms[M2M_TK_N];         /* summed device milliseconds */
    int64_t steps[M2M_TK_N];     /* M2M steps those launches advanced (a step
                                    pass: 1; a persistent launch: its steps) */
    int64_t kernels_total;       /* all kernels launched since the last read,
                                    timed or not */
} m2m_timing;

/* enable != 0: record events around each launch from now on. */
int m2m_set_timing(m2m_ctx *ctx, int32_t enable);

/* Synchronises, fills *out for the launches since the last call, resets. */
int m2m_get_timing(m2m_ctx *ctx, m2m_timing *out);

/* ---- many models in one launch (trial potentials, Section 4 of the paper:
 * models fitted in a sequence of potentials) ----
 * Each model is an independent M2M problem with its own particles,
 * potential, observables, targets, priors and epsilon; all share the
 * precision, the other step parameters and the stream.  When every model
 * is FP32C with the same compiled observable layout and the same prior
 * schedule, one kernel launch advances all models' particles per stage
 * (blocks shared out in proportion to N) and, on a non-default stream, the
 * launch sequence of m2m_batch_step is captured once into a CUDA graph and
 * replayed; otherwise the models are stepped one after another.  Results
 * are those of stepping each model alone. */
typedef struct {
    int64_t n;
    void *x, *y, *z, *vx, *vy, *vz;   /* device, caller-owned (as m2m_init) */
    double *w, *what;
    const m2m_potential_desc *pot;
    int32_t npot;
    const m2m_obs_desc *obs;
    int32_t nsets;
    const double *Y, *sigma;          /* host, or NULL */
    double eps;                       /* this model's epsilon */
    const m2m_prior_desc *prior;      /* NULL = flat */
} m2m_model_desc;
typedef struct m2m_batch m2m_batch;

/* par supplies mu, dt, alpha, entropy_const and the line of sight (its eps
 * is ignored: each model brings its own).  1 <= nmodels <= 1024. */
int m2m_batch_init(m2m_batch **batch_out, int32_t precision, int32_t nmodels, const m2m_model_desc *models,
                   const m2m_params *par, void *stream);

/* nsteps M2M steps of every model (see m2m_step). */
int m2m_batch_step(m2m_batch *batch, int64_t nsteps);

/* The context of model `model` (owned by the batch: valid until
 * m2m_batch_free; use it for m2m_get_obs, m2m_get_record, ...). */
/* Autotune a fused batch: the number of pass blocks (1, 2 or 4 times the
 * SMs x resident blocks, shared in proportion to N_m), each timed on
 * 2 * steps_per_trial real steps of all models (the models advance; their
 * results do not depend on the choice).  out->key names the choice; a
 * batch that steps model by model has nothing to tune (out->candidates =
 * 0).  Synchronises. */
int m2m_batch_autotune(m2m_batch *b, int32_t steps_per_trial, m2m_tuning *out);

int m2m_batch_context(m2m_batch *batch, int32_t model, m2m_ctx **ctx_out);

/* The last record of every model (out: host array of nmodels records, in
 * model order), gathered on the device and copied in one transfer: the
 * comparison of chi^2 and F across a sequence of trial potentials fitted to
 * the same data (Section 4).  Synchronises; returns the first model's
 * sticky kernel error, if any. */
int m2m_batch_get_records(m2m_batch *batch, m2m_record *out);

/* 1 if the last m2m_batch_step used one launch per stage for all models
 * (2 if also through a CUDA graph), 0 if it stepped them one by one. */
int m2m_batch_fused(const m2m_batch *batch);

int m2m_batch_free(m2m_batch *batch);

/* Observables of a particle set without any device allocation.
 *
 * The paper has no counterpart to this call: it serves callers that cannot
 * allocate device memory when they observe -- code running under an
 * external allocator that owns all device memory, or in allocator-free
 * real-time deployments, and callers that must not incur the implicit
 * synchronisation of cudaMalloc/cudaFree.  It computes what m2m_observe
 * computes for an FP32C context over the same particles (the same scatter
 * kernel, exact fixed-point sums at the same resolution when weight_scale
 * is the context's initial sum of weights), without a context.
 *
 * All scratch memory -- the integer totals, an error word and the edge and
 * Gauss-Hermite tables -- is one fixed device array of
 * M2M_STATIC_SCRATCH_BYTES inside the library, present on every GPU that
 * loads the library until the process exits.  The call allocates nothing
 * (no cudaMalloc/cudaFree, no allocating library routine).
 *   n            particle count, 1 <= n < 2^31
 *   x..vz        device float arrays (the FP32C state), w device double
 *                array; all caller-owned, 16-byte aligned, only read
 *   obs, nsets   observable sets as for m2m_init (host, copied; no LUT
 *                sets, no seeing); at most
 *                M2M_STATIC_MAX_OBS observables, M2M_STATIC_MAX_EDGES edges
 *                in total and M2M_STATIC_MAX_GH_CELLS Gauss-Hermite cells,
 *                else M2M_ERR_ARG with the reason in m2m_last_error(NULL)
 *   incl_sin, incl_cos  line of sight as for m2m_params
 *   weight_scale a value of the order of sum(w) (> 0): the fixed-point
 *                resolution is 2^-25 of the average weight,
 *                2^-25 * 2^ceil(log2(weight_scale)) / 2^ceil(log2(n))
 *   y_out        caller-owned device array of the observable count (double)
 *   stream       cudaStream_t (NULL = default stream); the work is enqueued
 *                on it and the call returns without synchronising
 * The first call on a device (the current device) looks up the array's
 * device address once (cudaGetSymbolAddress) and sets kernel attributes;
 * make that first call before any stream capture.  Every call shares the
 * one array, which keeps the previous call's contents (the totals are
 * cleared at the start of each call): calls that overlap on the GPU -- on
 * different streams or from different host threads -- race and give wrong
 * results.  A fixed-point overflow or a non-finite weight makes every
 * output NaN. */
#define M2M_STATIC_MAX_OBS 8192
#define M2M_STATIC_MAX_EDGES 2048
#define M2M_STATIC_MAX_GH_CELLS 4096
#define M2M_STATIC_SCRATCH_BYTES 163840
int m2m_observe_static(int64_t n, const void *x, const void *y, const void *z, const void *vx,
                       const void *vy, const void *vz, const double *w, const m2m_obs_desc *obs,
                       int32_t nsets, double incl_sin, double incl_cos, double weight_scale,
                       double *y_out, void *stream);

/* ---- particle shards: one model over several GPUs (data parallel) ----
 * Each process holds one context over a contiguous shard of the model's
 * particles (its own n; weights of the whole model).  The push, scatter and
 * weight update of a particle need only that particle, so a step is: every
 * shard scatters (m2m_shard_scatter); the shards' exchange buffers are
 * summed over shards (the observable totals and the entropy / weight sums;
 * at a prior recompute the range takes a minimum); every shard forms the
 * residual from the sums (m2m_shard_residual); at a prior recompute every
 * shard takes its particles' prior cells (m2m_shard_prior_cells), the cell
 * sums and counts are summed over shards, and m2m_shard_prior_finish sets
 * w_hat.  The collective is the caller's (NCCL or any all-reduce).  The
 * observable totals and cell sums are integers (FP32C fixed point at the
 * scale of the whole model), so a model split into shards takes exactly the
 * steps it takes in one context: positions, weights, priors and
 * observables bit for bit.  FP32C only; not with the spherical-harmonic
 * potential; a shard context is stepped only through these calls.
 * Buffers are caller-owned device memory:
 *   totals   int64[m2m_nobs]  sum over shards
 *   stats    double[2]        sum over shards (S, sum w of the scattered weights)
 *   range    double[3]        minimum over shards (min E, -max E, -max |L_z|)
 *   cell_sums int64[ncells], cell_counts int32[ncells]   sum over shards
 *            (ncells = nE*nL, +1 for E_LC)
 *
 * m2m_shard_init: the fixed-point scale of the whole model (global_n
 *   particles, initial sum of weights global_sum_w), as m2m_init sets it
 *   for one context.  Call once, before the first m2m_shard_scatter.
 * m2m_shard_scatter: with push = 1 one step's pass (the pending weight
 *   update, the push, the scatter with the updated weights, their S and sum
 *   w, and the (E, L_z) range when the step ends with a prior recompute:
 *   *prior_due = 1); push = 0 scatters the current state (the initial
 *   smoothing Delta~ := Delta, as at m2m_init).  Fills totals, stats (and
 *   range when due).
 * m2m_shard_residual: Eq. 1 and the smoothing from the summed totals, the
 *   update's coefficients, the step record (from the summed stats); zeroes
 *   totals.
 * m2m_shard_prior_cells / m2m_shard_prior_finish: the prior recompute of a
 *   step that ended with *prior_due = 1, from the summed range and the
 *   summed cell sums and counts. */
int m2m_shard_init(m2m_ctx *ctx, int64_t global_n, double global_sum_w);
int m2m_shard_scatter(m2m_ctx *ctx, int32_t push, int32_t *prior_due, int64_t *totals, double *stats, double *range);
int m2m_shard_residual(m2m_ctx *ctx, int64_t *totals, const double *stats);
int m2m_shard_prior_cells(m2m_ctx *ctx, const double *range, int64_t *cell_sums, int32_t *cell_counts);
int m2m_shard_prior_finish(m2m_ctx *ctx, const int64_t *cell_sums, const int32_t *cell_counts);

/* Text of the last error on this context (or of the last failed m2m_init
 * or m2m_observe_static when ctx is NULL). */
const char *m2m_last_error(const m2m_ctx *ctx);

/* Release library-owned memory.  The particle arrays are left as they are,
 * except that a pending weight update (lazy updates) is applied to w first
 * (best effort: an error there is not reported).  Synchronises. */
int m2m_free(m2m_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* M2M_H */
