/*
 * ptylm.h -- C-ABI of the GB300 (sm_103a) matrix-free Levenberg-Marquardt ptychography
 * library, after arXiv 2103.01767 ("A matrix-free Levenberg-Marquardt algorithm for
 * efficient ptychographic phase retrieval").
 *
 * Model (Sec. 2, Eqs. exit_wave and expected_count):
 *     psi_k = diag(P) S_k O,   psihat_k = F psi_k,   h_k = |psihat_k|^2 + b,
 *     zeta = h^(1/2)           (Sec. 4.1, Eq. magnitude)
 * Error metric (Sec. 4.1, Eq. ell_magnitude), summed over positions k and pixels m:
 *     Gaussian  l = (zeta - y^(1/2))^2 / 2          Poisson  l = zeta^2 - y log zeta^2
 * LM system (Sec. 4.1, Eq. lma_magnitude):  (G + lambda D) dz = -J^T grad_zeta l,
 *     G = J^T Hess_zeta(l) J  (Eq. ggn_magnitude), applied matrix-free (App. A).
 *
 * Conventions shared by every entry point
 *   - Complex arrays are interleaved single precision (ptylm_c64, 8 bytes).  Object O is
 *     row-major [ny][nx], probe P row-major [my][mx], per-position arrays [K][my][mx].
 *   - A complex vector stands for the real coordinates [Re; Im] of Sec. 3: inner products
 *     are sum(re*re + im*im) and gradients are dRe + i dIm (twice the Wirtinger form).
 *   - F is the orthonormal 2D DFT with forward sign -1.
 *   - Positions are int32 [K][2] = (row, col) of each patch's top-left corner; every
 *     position must satisfy 0 <= row <= ny-my and 0 <= col <= nx-mx.
 *   - Supported sizes: square probes with my = mx in {32, 64, 128}; any ny, nx >= my.
 *   - Pointers are device pointers unless an entry point says "host or device"; there the
 *     library detects host memory (pageable or pinned) and stages it through buffers it
 *     owns.  All memory passed in stays owned by the caller; the library never frees it.
 *   - Work is issued on the stream given to lm_init.  Entry points that return host
 *     scalars (f_host, stats) synchronise that stream before returning.
 *   - Errors are reported by return code only; nothing is thrown across the ABI.  A
 *     failed call leaves outputs unspecified.  ptylm_last_error() gives a thread-local
 *     message for the most recent failure on the calling thread.
 *   - A context is not thread-safe: one thread at a time may call into it.
 */
#ifndef PTYLM_H
#define PTYLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } ptylm_c64;

typedef struct ptylm_ctx ptylm_ctx;

typedef enum {
    PTYLM_OK = 0,
    PTYLM_ERR_ARG = 1,        /* invalid argument, size or position; nothing launched   */
    PTYLM_ERR_NOMEM = 2,      /* device allocation failed or workspace budget exceeded  */
    PTYLM_ERR_CUDA = 3,       /* a CUDA runtime call failed                              */
    PTYLM_ERR_NAN = 4,        /* a reduction produced NaN or Inf                         */
    PTYLM_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up                      */
    PTYLM_ERR_STALLED = 6,    /* LM damping overflowed (mu > mu_max) without progress   */
    PTYLM_ERR_STATE = 7,      /* call needs a linearisation point (forward_loss cache=1) */
    PTYLM_WARN_CG_MAXIT = 16  /* a CG solve hit max_cg; the step was still used         */
} ptylm_status;

typedef enum { PTYLM_LOSS_GAUSSIAN = 0, PTYLM_LOSS_POISSON = 1 } ptylm_loss;

typedef struct {
    int ny, nx;               /* object rows, columns                                    */
    int my, mx;               /* probe / detector rows, columns (my == mx, 32/64/128)    */
    int K;                    /* number of scan positions (>= 0)                         */
    int loss;                 /* ptylm_loss                                              */
    float background;         /* b > 0, added to every detector pixel (Eq. expected_count) */
    int joint;                /* 0: object only (SPR, Eq. cdp); 1: object + probe (BPR)  */
    size_t workspace_budget;  /* max bytes the context may allocate; 0 = unlimited       */
    int values_per_thread;    /* FFT tile of the single-problem kernels: 32, or 16 for     */
                              /* probe sides 32 and 64 (teams of S^2/16 threads); 0 picks  */
                              /* 16 when the positions would fill less than half of the   */
                              /* GPU with teams of S^2/32 threads (ignored by batches)     */
} ptylm_desc;

/* Parameters of Algorithm 1 (Sec. 4.2; values used in the paper: Sec. 5). */
typedef struct {
    double mu0;        /* initial damping multiplier (paper: 1e-5)                         */
    double mu_min;     /* lower bound of mu (1e-8)                                         */
    double kappa;      /* mu growth/shrink factor (4)                                      */
    double nu;         /* exponent in lambda = mu ||grad_zeta l||^nu (1)                   */
    double rho_min;    /* acceptance threshold of the gain ratio (1e-4)                    */
    double beta;       /* CG forcing bound, Eq. lma_termination_eta (0.1 Gauss, 0.9 Poisson) */
    double mu_max;     /* give up (PTYLM_ERR_STALLED) when mu exceeds this (1e16)          */
    int max_outer;     /* outer LM iterations                                              */
    int max_cg;        /* CG iterations per solve (PTYLM_WARN_CG_MAXIT when reached)       */
    int fixed_cg;      /* > 0: run exactly this many CG iterations per solve (benchmarking) */
    double target_err; /* stop once the object error <= target_err (needs O_ref; 0: none)  */
    const ptylm_c64* O_ref; /* optional device reference object for the error metric       */
    const uint8_t* mask;    /* optional device [ny][nx] mask of pixels the error compares   */
    int scaled;        /* 1: D = Dg(G) (closed form, App. B), lambda = mu, Jacobi PCG with
                          Dg(G + lambda D) (Sec. 3.3, "PLM"); 0: D = I, lambda = mu ||grad l||^nu */
    int projected;     /* 1: Algorithm 2 after each accepted step (Sec. 4.3)                */
    double radius_O;   /* constraint |O| <= radius_O (Eq. constraints: 1)                   */
    double radius_P;   /* constraint |P| <= radius_P (Eq. constraints: 1e8)                 */
    double gamma;      /* Algorithm 2: accept Pi(z + dz) if f(Pi) - f_min < gamma (f - f_min) (1e-6) */
    double tau_s;      /* Algorithm 2: descent test g.s <= -tau_s ||s||^p_s (1e-8)          */
    double p_s;        /* (2.1)                                                              */
    double sigma;      /* Armijo constant, Eq. armijo_criterion (1e-4)                       */
    int max_ls;        /* Armijo halvings before giving up the move (30)                    */
    double diag_floor; /* Dg(G) is raised to diag_floor * max Dg(G) (1e-6)                  */
    /* App. E surrogate metric (LM-S / PLM-S): outer iteration t uses the expected intensity
     * h = |psihat|^2 + b + s_t (Eq. expected_count_surrogate), s_t falling on an evenly
     * spaced logarithmic grid from surrogate0 at t = 0 to surrogate_end at t = surrogate_T - 1,
     * and s_t = 0 (the true metric) from t = surrogate_T on.  surrogate_T = 0 turns it off
     * (default); the paper's runs use surrogate0 = 1, surrogate_T = 100.  Both levels must be
     * finite and > 0 when surrogate_T > 0. */
    double surrogate0;
    double surrogate_end;
    int surrogate_T;
    /* 0 (default): each CG iteration after its GGN product is one cooperative launch with
     * two grid-wide FP64 reductions inside it (when the device supports cooperative
     * launches); 1: three launches (p.q; x, r and r.z; p and q).  Both give the same
     * results bit for bit.  A bounded grid-wide wait that gives up ends lm_solve with
     * PTYLM_ERR_TIMEOUT. */
    int separate_cg_kernels;
    /* Polls of each bounded grid-wide wait of the single-launch CG iteration before it gives
     * up: 0 (default) about a second (2^24 polls of >= 32 ns); > 0 that many.  A small value
     * exists for fault-injection tests: the waits then run out, every CTA still finishes its
     * in-bounds work and exits, and lm_solve returns PTYLM_ERR_TIMEOUT with the context
     * usable for the next call. */
    int wait_polls;
} ptylm_lm_params;

/* Per-call results of lm_solve.  hist_* point to host arrays of hist_len entries (or are
 * NULL); entry t describes outer iteration t.  Each outer iteration is also an NVTX range
 * ("lm: outer iteration t") with its CG solves and trial points nested inside. */
typedef struct {
    int n_outer;          /* outer iterations run                                         */
    int cg_total;         /* CG iterations (GGN matvecs inside CG) summed over the run    */
    int matvecs_total;    /* all GGN matvecs, including each solve's initial residual     */
    double f_final;       /* error metric at the returned iterate                         */
    double err_final;     /* object error at the returned iterate (NaN without O_ref)     */
    int hist_len;
    double* hist_f;       /* f at the linearisation point of iteration t                  */
    double* hist_gnorm;   /* ||grad f|| there                                             */
    double* hist_mu;      /* mu after iteration t                                         */
    int* hist_cg;         /* CG iterations in iteration t                                 */
    double* hist_err;     /* object error after iteration t (NaN without O_ref)           */
    double* hist_rho;     /* gain ratio of the step that ended iteration t                */
    double* hist_lambda;  /* damping lambda of that step                                  */
    double* hist_time;    /* host wall-clock seconds from the start of the call to the end
                             of iteration t                                               */
} ptylm_lm_stats;

/* Create a context for one reconstruction problem (Sec. 2).
 *   positions_dev: device int32 [K][2], copied into the context (validated on the host:
 *                  out-of-range positions return PTYLM_ERR_ARG with nothing launched).
 *   y_dev:         device float [K][my][mx] measured intensities (y >= 0) in natural DFT
 *                  order (zero frequency at [0][0]); copied into the context's internal
 *                  order, so the caller's buffer may be reused once lm_init returns.
 *   stream:        cudaStream_t (NULL = legacy default stream) all work is issued on.
 * Allocates the frequency-domain cache (8*K*M bytes), the measurement copy (4*K*M bytes)
 * and small workspaces within desc->workspace_budget, else PTYLM_ERR_NOMEM. */
ptylm_status lm_init(ptylm_ctx** ctx, const ptylm_desc* desc, const int32_t* positions_dev,
                     const float* y_dev, void* stream);

/* Replace the measurements y (Sec. 2: the recorded data y_k) with y_dev, device float
 * [K][my][mx] in natural order, copied like in lm_init.  Invalidates the linearisation
 * point (a later jvp / jtvp / ggn_matvec / gradient returns PTYLM_ERR_STATE until
 * forward_loss(cache=1) runs again). */
ptylm_status ptylm_set_measurements(ptylm_ctx* ctx, const float* y_dev);

/* Error metric f = sum_k sum_m l(zeta_km, y_km) at (O, P)  (Eq. error_metric_magnitude).
 *   O: device [ny][nx]; P: device [my][mx].
 *   f_host: host double receiving f (accumulated in FP64).
 *   dl_norm2_host: optional host double receiving ||grad_zeta l||^2 (Algorithm 1's lambda).
 *   cache = 1 makes (O, P) the linearisation point of later jvp / jtvp / ggn_matvec /
 *   gradient calls: it copies O and P into the context, stores the per-pixel factor
 *   a = psihat (Hess_zeta l)^(1/2) / zeta used by ggn_matvec, and computes
 *   grad f = J^T grad_zeta l (App. A step 1) fused in the same kernel.
 *   cache = 0 evaluates f only (Algorithm 1's trial point) and changes no state. */
ptylm_status forward_loss(ptylm_ctx* ctx, const ptylm_c64* O, const ptylm_c64* P,
                          double* f_host, double* dl_norm2_host, int cache);

/* grad f = J^T grad_zeta l at the linearisation point (App. A step 1; Eq. grad_f_obj in
 * real coordinates).  gO: device [ny][nx]; gP: device [my][mx] or NULL.  The probe part is
 * only available for joint contexts (else PTYLM_ERR_ARG when gP != NULL). */
ptylm_status gradient(ptylm_ctx* ctx, ptylm_c64* gO, ptylm_c64* gP);

/* Jacobian-vector product at the current point (forward_loss(cache=1) or forward_magnitude;
 * App. A Eqs. jvp_step_1..3; computed
 * in forward mode from App. B Eq. jac_ampl):
 *     out_km = Re( conj(psihat_km) [F (P . S_k vO + vP . S_k O)]_m ) / zeta_km
 *   vO: device [ny][nx]; vP: device [my][mx] (joint contexts only) or NULL (= 0);
 *   out: device float [K][my][mx], natural order.
 * Uses the stored phasor when forward_magnitude kept one, else recomputes psihat from the
 * stored (O, P); never reads the ggn_matvec cache. */
ptylm_status jvp(ptylm_ctx* ctx, const ptylm_c64* vO, const ptylm_c64* vP, float* out);

/* Transposed-Jacobian product at the linearisation point (App. A Eq. arbitrary_jtvp_sequence):
 *     outO = sum_k S_k^T [conj(P) . F^H(psihat_k w_k / zeta_k)]
 *     outP = sum_k conj(S_k O) . F^H(psihat_k w_k / zeta_k)         (joint contexts)
 *   w: device float [K][my][mx]; outO: device [ny][nx] (overwritten); outP: device [my][mx]
 *   (joint contexts only) or NULL. */
ptylm_status jtvp(ptylm_ctx* ctx, const float* w, ptylm_c64* outO, ptylm_c64* outP);

/* Closed-form diagonal of the GGN in real coordinates at the linearisation point (App. B,
 * Eqs. ggn_diag_elem_final, ggn_diag_mat, ggn_joint_diag; the paper's h ~ |psihat|^2
 * approximation):  D_O[n] = sum_{k: n in patch k} |P[n - r_k]|^2 tr_k / (2M),
 *                  D_P[m] = sum_k |O[r_k + m]|^2 tr_k / (2M),   tr_k = sum_m d2l_km.
 *   D_out: device float [ny*nx] or, for joint contexts, [ny*nx + my*mx].
 *   floor_rel: entries of each block below floor_rel * (that block's max) are raised to
 *   it (0 disables). */
ptylm_status ggn_diag(ptylm_ctx* ctx, float* D_out, double floor_rel);

/* Damped GGN-vector product, the hot path (App. A steps 2-4, Eq. ggn_magnitude_appendix_2):
 *     outO = J^T( Hess_zeta l . J vO ) + lambda D vO
 * One fused kernel per call: patch gather x P, 2D FFT, frequency stage with the cached a
 * (t = Re(conj(a) dpsihat), chihat = a t), inverse 2D FFT, x conj(P), overlap scatter-add.
 *   vO, outO: host or device [ny][nx]; outO is overwritten.
 *   vP, outP: joint contexts: device [my][mx] probe blocks (the joint GGN of Eq. ggn_joint_diag's
 *   block structure, z = (O, P)); both NULL in object-only contexts.
 *   D: device float diagonal scaling over z -- [ny*nx] (object only) or [ny*nx + my*mx]
 *   (object then probe) -- or NULL for the identity.
 * Needs a linearisation point (PTYLM_ERR_STATE otherwise). */
ptylm_status ggn_matvec(ptylm_ctx* ctx, const ptylm_c64* vO, const ptylm_c64* vP, double lambda,
                        const float* D, ptylm_c64* outO, ptylm_c64* outP);

/* Truncated matrix-free LM, Algorithm 1 (Sec. 4.2), on z = O (object-only contexts, the
 * SPR problem) or z = (O, P) (joint contexts, the BPR problem).  prm->scaled selects D = I
 * with lambda = mu ||grad_zeta l||^nu ("LM") or D = Dg(G) with lambda = mu and the Jacobi
 * preconditioner Dg(G + lambda D) ("PLM", Sec. 3.3); prm->projected adds Algorithm 2
 * (Sec. 4.3) with the radial constraints of Eq. constraints.  The inner truncated (P)CG is
 * stopped by Eqs. lma_termination_magnitude / lma_termination_eta with
 * eta = min(beta, ||grad f||^(1/2)) and warm-started from the previous step.  CG vectors are
 * FP32; dot products, lambda, mu, the gain ratio and f are FP64 on the device.  With the
 * single-launch CG iteration (separate_cg_kernels = 0) the stopping test runs on the device
 * and the host queues iterations in batches (as many as the previous solve took), reading
 * the scalars once per batch; iterations queued past the stop return at once.  Object-only
 * unprojected solves evaluate each trial point with the cached forward pass, so that an
 * accepted trial is already the next linearisation; this needs a second loss cache, gradient
 * and point (8 K M + 16 ny nx + K M / 8 bytes), taken once, after every buffer the solve
 * needs, when it fits the workspace budget whole with room left for the PLM scaling and the
 * Algorithm 2 direction (12 ny nx bytes, unless already taken); otherwise none of it is
 * taken and every outer iteration runs its own forward pass.
 *   O_inout: host or device [ny][nx]; initial guess in, final iterate out.
 *   P_inout: host or device [my][mx] probe: read only for object-only contexts, updated
 *   in place for joint contexts.
 *   prm: host parameters; stats: host results (may be NULL).
 * Returns PTYLM_OK, PTYLM_WARN_CG_MAXIT (some solve hit max_cg), or an error. */
ptylm_status lm_solve(ptylm_ctx* ctx, ptylm_c64* O_inout, ptylm_c64* P_inout,
                      const ptylm_lm_params* prm, ptylm_lm_stats* stats);

/* Resumable state of Algorithm 1 (Sec. 4.2) between calls, for checkpointing a long run:
 * with the iterate z = O (or (O, P) for joint contexts) it is everything Algorithm 1 carries
 * from one outer iteration to the next.  The App. E surrogate level s_t follows from t. */
typedef struct {
    int t;             /* outer iterations completed so far (>= 0)                         */
    double mu;         /* damping multiplier (> 0)                                         */
    ptylm_c64* delta;  /* host or device [L] (L = ny*nx, + my*mx for joint contexts): the last
                          CG solution, which warm-starts the next solve; NULL: start from zero
                          and do not return it                                             */
} ptylm_lm_state;

/* lm_solve continued from `state` (host struct, in/out): the run starts at outer iteration
 * state->t with damping state->mu and warm start state->delta, runs prm->max_outer more outer
 * iterations (history entries count from there; the surrogate schedule from state->t), and
 * writes the state after its last outer iteration back (delta overwritten in place).  A run
 * split into two calls with the state handed over follows the uninterrupted run (up to the
 * rounding order of the scatter's float reductions).  lm_solve is lm_solve_resume from
 * t = 0, mu = prm->mu0, delta = 0.  PTYLM_ERR_ARG for state == NULL, t < 0 or mu not finite
 * and > 0; on an error return the state is unspecified. */
ptylm_status lm_solve_resume(ptylm_ctx* ctx, ptylm_c64* O_inout, ptylm_c64* P_inout,
                             const ptylm_lm_params* prm, ptylm_lm_state* state, ptylm_lm_stats* stats);

/* Expected intensities h = |F diag(P) S_k O|^2 + b for every position (Sec. 2,
 * Eq. expected_count), used to simulate measurements.  O: device [ny][nx]; P: device
 * [my][mx]; h_out: device float [K][my][mx] in natural order.  Changes no context state. */
ptylm_status forward_intensity(ptylm_ctx* ctx, const ptylm_c64* O, const ptylm_c64* P, float* h_out);

/* Magnitudes zeta = (|F diag(P) S_k O|^2 + b)^(1/2) for every position (Sec. 4.1,
 * Eq. magnitude) into zeta_out (device float [K][my][mx], natural order), and make (O, P)
 * the point of later jvp / jtvp calls (the loss cache is invalidated: ggn_matvec, gradient
 * and ggn_diag need forward_loss(cache = 1) again).  store_phasor = 1 also keeps the unit
 * phasor psihat / zeta (8 K M bytes, allocated once within the workspace budget, else
 * PTYLM_ERR_NOMEM), so that jvp and jtvp need one 2D FFT per position instead of two;
 * store_phasor = 0 makes them recompute the exit waves. */
ptylm_status forward_magnitude(ptylm_ctx* ctx, const ptylm_c64* O, const ptylm_c64* P, float* zeta_out,
                               int store_phasor);

/* Instrumentation (no counterpart in the paper).  ptylm_profile(ctx, 1) resets the
 * counters and starts timing every launch of the per-position kernels with CUDA events on
 * the context stream; ptylm_profile(ctx, 0) stops.  ptylm_profile_read synchronises the
 * stream and returns, for kernel id `kernel` (PTYLM_KERNEL_*), the summed device time in
 * milliseconds and the number of timed launches; kernel = -1 returns 0 ms and the number
 * of launches of all the library's kernels (vector kernels included) since the reset.
 * PTYLM_KERNEL_CG_ITERATION times, per CG iteration of lm_solve, the vector work after the
 * GGN product (one cooperative launch, or three launches with separate_cg_kernels). */
enum {
    PTYLM_KERNEL_FORWARD_LOSS = 0,
    PTYLM_KERNEL_FORWARD_CACHE = 1,
    PTYLM_KERNEL_GGN_MATVEC = 2,
    PTYLM_KERNEL_JTVP = 3,
    PTYLM_KERNEL_JVP = 4,
    PTYLM_KERNEL_FORWARD_INTENSITY = 5,
    PTYLM_KERNEL_FORWARD_CACHE_JOINT = 6,
    PTYLM_KERNEL_GGN_MATVEC_JOINT = 7,
    PTYLM_KERNEL_JTVP_JOINT = 8,
    PTYLM_KERNEL_JVP_JOINT = 9,
    PTYLM_KERNEL_FORWARD_MAGNITUDE = 10,
    PTYLM_KERNEL_JVP_PHASOR = 11,
    PTYLM_KERNEL_JVP_PHASOR_JOINT = 12,
    PTYLM_KERNEL_JTVP_PHASOR = 13,
    PTYLM_KERNEL_JTVP_PHASOR_JOINT = 14,
    PTYLM_KERNEL_CG_ITERATION = 15
};
ptylm_status ptylm_profile(ptylm_ctx* ctx, int enable);
/* As ptylm_profile(ctx, 1), but times only the sections whose bit is set in mask (bit k:
 * kernel id k, PTYLM_KERNEL_*); the launch count still covers every kernel.  Each timed
 * section adds a pair of event records to the stream, so timing one kernel costs the others
 * nothing.  mask = 0 stops. */
ptylm_status ptylm_profile_select(ptylm_ctx* ctx, unsigned mask);
ptylm_status ptylm_profile_read(ptylm_ctx* ctx, int kernel, double* total_ms, long long* launches);

/* Allocation-free error metric (the paper has no counterpart).  It serves callers that must
 * not allocate device memory: serving or real-time loops that reserve all their memory at
 * start-up, because cudaMalloc and cudaFree can synchronise the device and take unbounded
 * time; plug-ins inside a host framework whose memory pool already holds nearly all of the
 * device memory, so a cudaMalloc of their own would fail; and code whose every device byte
 * must be accounted to another allocator.  It computes the same f = sum_k sum_m
 * l(zeta_km, y_km) (Eq. ell_magnitude) and ||grad_zeta l||^2 as forward_loss(cache = 0),
 * without a context and without allocating: the caller passes all inputs and the output,
 * and the only scratch (twiddle tables, FP64 partial sums, a counter, an error flag) is a
 * file-scope device array of PTYLM_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 *   ny, nx: object size; m: probe side (32, 64 or 128; larger sizes are rejected with
 *   PTYLM_ERR_ARG); K >= 0; loss, background: as in ptylm_desc.
 *   O [ny][nx], P [m][m], positions int32 [K][2] (8-byte aligned), y float [K][m][m] in
 *   natural order: device pointers.  out_dev: device double[2] <- (f, ||grad_zeta l||^2).
 *   stream: cudaStream_t (NULL = legacy default stream).
 * At most PTYLM_NOALLOC_MAX_CTAS CTAs run (fewer positions in flight, same result).
 * The first call on a device, with that device current, looks up the scratch's device
 * address and uploads the twiddle tables there (a synchronous copy).  Every call shares
 * the scratch, which keeps the last call's contents; the counter and the flag are cleared
 * at the start of each call.  Calls whose work overlaps on the GPU (other streams, other
 * threads) race and give wrong results.  Before returning, the call waits for its work on
 * `stream` to finish and reads the error flag: positions outside the object return
 * PTYLM_ERR_ARG. */
#define PTYLM_NOALLOC_MAX_CTAS 2048
#define PTYLM_NOALLOC_SCRATCH_BYTES 35328
ptylm_status ptylm_forward_loss_noalloc(int ny, int nx, int m, int K, int loss, float background,
                                        const ptylm_c64* O, const ptylm_c64* P, const int32_t* positions,
                                        const float* y, double* out_dev, void* stream);

/* Measured FP32 peak of the current device (instrumentation; the paper has no counterpart):
 * `launches` timed launches (after one untimed one) of an FFMA loop that keeps every SM's
 * FP32 pipes busy -- 2048 threads per SM, 8 independent FMA chains per thread, 128 * iters
 * FMAs per thread -- each timed with CUDA events on `stream` (cudaStream_t, NULL = legacy
 * stream).  tflops_host: host double <- 2 x FMAs / median launch time, in TFLOP/s; ms_host:
 * host double <- the median launch time in ms (may be NULL).  The call synchronises
 * `stream`.  PTYLM_ERR_ARG for launches < 1, iters < 1 or tflops_host == NULL. */
ptylm_status ptylm_fp32_peak(int launches, int iters, double* tflops_host, double* ms_host, void* stream);

/* Free the context and everything it allocated (NULL is accepted). */
ptylm_status lm_destroy(ptylm_ctx* ctx);

/* Static description of a status code. */
const char* ptylm_strerror(ptylm_status s);

/* Thread-local message of the most recent failed call on this thread ("" if none). */
const char* ptylm_last_error(void);

/* Fill prm with the paper's Algorithm 1 defaults (Sec. 5) for the given loss. */
void ptylm_default_lm_params(ptylm_lm_params* prm, int loss);

/* ---------------------------------------------------------------------------------------
 * Batches of independent reconstructions.
 *
 * B object-only problems (Sec. 2, Eq. cdp), each with its own object size, probe side
 * (32, 64 or 128), scan, loss and background, share one batch.  Each per-position operator
 * (forward model + error metric [+ cache a and gradient], GGN product; App. A) runs over
 * all problems as ONE persistent kernel launch: 512-thread CTAs take work items (a problem
 * and a group of its positions) from a device counter, so problems of uneven size balance
 * across the SMs.  Batch vectors (objects, gradients, directions) are the problems'
 * objects concatenated in problem order, [ny][nx] row-major each; problem b starts at
 * element ptylm_batch_offset(batch, b).  All pointers are device pointers.
 * --------------------------------------------------------------------------------------- */
typedef struct ptylm_batch ptylm_batch;

/* descs[b]: problem b (joint must be 0; workspace_budget is ignored).  positions_dev[b]:
 * int32 [K][2]; y_dev[b]: float [K][my][mx] in natural DFT order; probes_dev[b]: [my][mx].
 * Everything is copied (positions validated on the host: PTYLM_ERR_ARG when outside).
 * stream: the caller's cudaStream_t (NULL = legacy stream); the batch works on a stream of
 * its own, ordered after `stream` on entry to every call and before it on exit. */
ptylm_status ptylm_batch_init(ptylm_batch** batch, int B, const ptylm_desc* descs,
                              const int32_t* const* positions_dev, const float* const* y_dev,
                              const ptylm_c64* const* probes_dev, void* stream);

/* First element of problem b in batch vectors; b = B gives the total length; -1 if invalid. */
long ptylm_batch_offset(const ptylm_batch* batch, int b);

/* f_b and ||grad_zeta l||^2_b at the batch vector O (Eq. error_metric_magnitude per
 * problem, FP64 sums), into host arrays of B entries (either may be NULL).  cache = 1 also
 * makes O the linearisation point: cache a and gradient of every problem. */
ptylm_status ptylm_batch_forward_loss(ptylm_batch* batch, const ptylm_c64* O, double* f_host,
                                      double* dl_norm2_host, int cache);

/* Copy of the batch gradient at the linearisation point (PTYLM_ERR_STATE without one). */
ptylm_status ptylm_batch_gradient(ptylm_batch* batch, ptylm_c64* g);

/* out = (G_b + lambda_b I) v_b for every problem (App. A, Eq. ggn_magnitude_appendix_2);
 * lambda: host array of B values or NULL (= 0). */
ptylm_status ptylm_batch_ggn_matvec(ptylm_batch* batch, const ptylm_c64* v, ptylm_c64* out,
                                    const double* lambda);

/* Algorithm 1 for every problem, in place on the batch vector O_inout: LM (D = I) or, for
 * problems with prm[b].scaled = 1, PLM (D = Dg(G) from the closed form of App. B at every
 * linearisation, floored at diag_floor times its maximum; lambda = mu; Jacobi PCG with
 * (1 + lambda) D; the predicted reduction with Delta^T D Delta), as lm_solve does for one
 * problem.  prm: B parameter sets (projected must be 0; the App. E surrogate schedule is
 * honoured; O_ref / mask point to problem b's own reference object and mask).  stats: B
 * entries or NULL.  All problems advance together: each outer step linearises the problems
 * whose last step was accepted, runs the truncated CG of all unfinished problems (one CG
 * iteration of all of them is a captured CUDA graph of four launches; converged problems
 * are masked out), evaluates every trial point in one launch and accepts or rejects per
 * problem on the host.  The first call tunes the schedule (ptylm_batch_tune) unless one was
 * set.  Returns the first non-OK problem status (PTYLM_ERR_STALLED, PTYLM_ERR_NAN) after
 * finishing the others, else PTYLM_WARN_CG_MAXIT if any CG solve hit max_cg. */
ptylm_status ptylm_batch_lm_solve(ptylm_batch* batch, ptylm_c64* O_inout, const ptylm_lm_params* prm,
                                  ptylm_lm_stats* stats);

/* Closed-form GGN diagonal of every problem at the batch's linearisation point (App. B, Eqs.
 * ggn_diag_elem_final, ggn_diag_mat; as ggn_diag): D_out[z_off_b + n] = sum over problem b's
 * positions k whose patch holds n of |P_b[n - r_k]|^2 tr_k / (2M_b), tr_k = sum_m d2l_km,
 * then raised to floor_rel times problem b's maximum.  D_out: host or device float [total].
 * PTYLM_ERR_STATE without a linearisation point, PTYLM_ERR_ARG for floor_rel outside [0, 1). */
ptylm_status ptylm_batch_ggn_diag(ptylm_batch* batch, float* D_out, double floor_rel);

/* Autotuner (the paper has no counterpart): times the batch's GGN product (3 launches after a
 * warm-up) under 24 schedules and keeps the fastest.  Schedule c = s + 6 (t32 + 2 t64):
 *   s = 0..5: work items ordered largest patches first (0..2) or round robin over the
 *             problems (3..5), with 1, 2 or 4 positions per team per item;
 *   t32, t64: FFT tile of the problems with 32 x 32 / 64 x 64 probes -- 0: 32 values per
 *             thread (teams of S^2/32 threads), 1: 16 values per thread (teams of S^2/16
 *             threads, half the registers per patch, one more exchange for S = 32).
 * Tiles that no problem of the batch uses are not timed (ms entry -1).  A tile change puts
 * the affected problems' measurements into that tile's team order and recomputes the
 * linearisation (cache, gradient, metric) at the same point.  Needs a linearisation point.
 * choice: index kept; ms: up to n_ms entries of the table (host floats). */
ptylm_status ptylm_batch_tune(ptylm_batch* batch, int* choice, float* ms, int n_ms);

/* Use schedule `choice` (0..23, as in ptylm_batch_tune) without timing; with a linearisation
 * point, a tile change recomputes it as in ptylm_batch_tune. */
ptylm_status ptylm_batch_set_schedule(ptylm_batch* batch, int choice);

/* Kernel launches issued by the batch so far (graph replays count their four kernels). */
ptylm_status ptylm_batch_profile_read(ptylm_batch* batch, long long* launches);

/* Free the batch (NULL is accepted). */
ptylm_status ptylm_batch_destroy(ptylm_batch* batch);

/* ---------------------------------------------------------------------------------------
 * Learned initialisation (not part of the paper): a data-driven initial object for
 * Algorithm 1 from the measured magnitudes, for 128 x 128 patterns.
 *
 * Per pattern k the physics input is e_k = F^-1(sqrt(y_k) u) conj(P) / (|P|^2 + 1e-3 max|P|^2)
 * with u = F(P) / max(|F(P)|, 1e-3 max|F(P)|) (the far-field magnitudes with the probe's own
 * far-field phase, propagated back through the forward model of Sec. 2 and divided by the
 * probe), two channels (Re, Im) of [128][128] float.  A 6-layer convolutional encoder-decoder refines it into the object
 * patch: three 3 x 3 stride-2 convolutions 2 -> C1 -> C2 -> C3 (ReLU), then three x2
 * nearest upsamplings each followed by a 3 x 3 convolution C3 -> C2 -> C1 (ReLU) -> 2
 * (linear).  Weights are bfloat16 copies of FP32 master weights; sums are FP32.  The
 * convolutions run on the tensor cores (tcgen05 MMA, BF16 operands, FP32 accumulation in
 * TMEM): each FP32 activation or gradient is carried as a pair of bfloat16 values
 * (x = hi + lo, exact to 2^-18 relative), so a product with a bfloat16 weight takes two MMAs
 * and a weight-gradient product three (hi.hi + hi.lo + lo.hi).  A convolution kernel whose
 * bounded wait gives up makes the call return PTYLM_ERR_TIMEOUT.  The patch estimates are
 * averaged into the object with weights |P|^2 over
 * their overlaps (1 where no probe reaches).  Parameter layout (flat float array):
 * W1 b1 W2 b2 ... W6 b6, W_l as [c_out][c_in][3][3].  Arrays are device arrays unless named
 * *_host; images are [N][2][128][128] float.
 * --------------------------------------------------------------------------------------- */
typedef struct ptylm_net ptylm_net;

/* m must be 128; widths = {C1, C2, C3}, multiples of 32 in [32, 256] ({64, 128, 256}:
 * 740,226 parameters); max_batch: patterns per forward / training batch; seed: He-normal
 * initial weights, zero biases.  PTYLM_ERR_ARG for other sizes. */
ptylm_status ptylm_net_create(ptylm_net** net, int m, const int* widths, int max_batch, uint64_t seed,
                              void* stream);
/* Number of floats in the flat parameter array (-1 for NULL). */
long ptylm_net_num_params(const ptylm_net* net);
/* Load / read the FP32 master parameters (host arrays); grads_host receives the gradients
 * of the last ptylm_net_loss_grad or training step (either pointer may be NULL). */
ptylm_status ptylm_net_set_params(ptylm_net* net, const float* params_host);
ptylm_status ptylm_net_get_params(ptylm_net* net, float* params_host, float* grads_host);
/* out = network(X) for N <= max_batch images. */
ptylm_status ptylm_net_forward(ptylm_net* net, const float* X, int N, float* out);
/* Output of hidden layer `layer` (1..5, after its ReLU) of the first N images of the last
 * forward pass (ptylm_net_forward, ptylm_net_loss_grad or training), as the FP32 value of
 * the stored bfloat16 pair: out device float [N][C_layer][H_layer][H_layer].  For
 * inspection and for taking the ReLU decisions of a reference evaluation from the network
 * itself (the paper has no counterpart).  Synchronises the network's stream. */
ptylm_status ptylm_net_activation(ptylm_net* net, int layer, int N, float* out);
/* Loss L = sum mask (out - T)^2 / (2 N sum mask) (mask [128][128] broadcast over channels
 * and batch) and its gradients (kept in the network, read with ptylm_net_get_params). */
ptylm_status ptylm_net_loss_grad(ptylm_net* net, const float* X, const float* T, const float* mask, int N,
                                 double* loss_host);
/* Training pairs from a pool of objects [n_obj][side][side] (complex64): samples int32
 * [N][3] = (object, row, column); X = physics input of the noiseless pattern of P times the
 * object patch, T = the patch (Re, Im).  PTYLM_ERR_ARG for samples outside their object. */
ptylm_status ptylm_net_pairs(ptylm_net* net, const ptylm_c64* pool, int side, const int32_t* samples, int N,
                             const ptylm_c64* P, float* X, float* T);
/* `steps` Adam steps (beta 0.9 / 0.999, learning rate lr falling linearly to lr/10) on
 * batches of fresh pairs drawn uniformly from the pool by a splitmix64 stream seeded with
 * `seed`; loss per step into loss_hist_host (steps entries, may be NULL).  The loss mask is
 * the probe's support. */
ptylm_status ptylm_net_train(ptylm_net* net, const ptylm_c64* pool, int n_obj, int side, const ptylm_c64* P,
                             int steps, int batch, double lr, uint64_t seed, double* loss_hist_host);
/* Physics inputs of the context's measurements at positions idx[0..count) (int32 device
 * array) into X [count][2][128][128]. */
ptylm_status ptylm_learned_inputs(ptylm_ctx* ctx, ptylm_net* net, const ptylm_c64* P, const int32_t* idx,
                                  int count, float* X);
/* Initial object O0 [ny][nx] of the context: physics inputs of positions idx[0..count),
 * network, |P|^2-weighted overlap average (chunks of max_batch patterns). */
ptylm_status ptylm_learned_init(ptylm_ctx* ctx, ptylm_net* net, const ptylm_c64* P, const int32_t* idx, int count,
                                ptylm_c64* O0);
/* Free the network (NULL is accepted). */
ptylm_status ptylm_net_destroy(ptylm_net* net);

#ifdef __cplusplus
}
#endif
#endif /* PTYLM_H */
