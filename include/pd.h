/*
 * pd.h -- C ABI of the GB300 randomised primal-dual (PD-R) radio-interferometric
 * imaging library (arXiv:1610.08895, Onose, Carrillo, McEwen & Wiaux).
 *
 * The library solves, one iteration at a time, the constrained problem of
 * Sec. 3 (eq. basic-min-problem):
 *
 *     minimise ||Psi^H x||_1  subject to  x >= 0,  ||y_i - Phi_i x||_2 <= eps_i,
 *
 * with Algorithm 1 (randomised forward-backward PD). Every operation runs in
 * hand-written CUDA kernels on one GPU; nothing here falls back to the CPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are real, row-major [ny][nx]; pixel (iy, ix) sits at centred
 *   coordinates (iy - ny/2, ix - nx/2).
 * - Visibilities are complex (interleaved re, im), in the caller's order
 *   ("user order") unless stated otherwise.
 * - Element type follows the plan's precision: PD_F32 -> float / float2 pairs,
 *   PD_F64 -> double / double2 pairs. Device pointers are typed void*.
 * - "device" pointers must be device-accessible memory of the current CUDA
 *   device; "host" pointers are ordinary host memory read during the call.
 * - The caller owns every buffer it passes. The plan and the state own the
 *   scratch they allocate and free it in their destroy calls.
 * - Calls are asynchronous on the given stream (a cudaStream_t, passed as
 *   void*; NULL = legacy default stream) unless a host output is returned,
 *   in which case the call synchronises that stream before returning.
 * - Every entry point returns a pd_status; nothing aborts or throws across the
 *   ABI. pd_last_error() returns a static description of the last failure on
 *   the calling thread.
 */
#ifndef PD_GB300_H
#define PD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PD_OK = 0,
    PD_EINVAL = 1,      /* invalid argument (sizes, ranges, null pointers) */
    PD_ENOMEM = 2,      /* device or host allocation failed */
    PD_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    PD_ETIMEOUT = 4,    /* a bounded device wait gave up (status word set) */
    PD_ENOTCONV = 5,    /* power iteration did not reach its tolerance */
    PD_ENOTSUP = 6      /* valid but unsupported configuration */
} pd_status;

typedef enum { PD_F32 = 0, PD_F64 = 1 } pd_precision;

typedef struct pd_plan pd_plan;
typedef struct pd_state pd_state;

/*
 * Plan description (host memory, read only during pd_plan_create).
 *
 * nx, ny        image size; powers of two in [16, 8192] (FP32) or [16, 4096] (FP64,
 *               PD_ENOTSUP above: one FFT row of 8192 FP64 values needs 2048 threads).
 * osf           oversampling per axis; must be 2 (the paper's k = 4 total,
 *               Sec. 5 "oversampling ratio k=4"), giving a (2ny) x (2nx) grid.
 * nvis          number of visibilities M >= 1.
 * uv            host [nvis][2] doubles (u, v) in radians per pixel, each in
 *               [-pi, pi). u runs along x (columns), v along y (rows).
 * nblocks       number of data blocks d in [1, 4096] (eq. data-split).
 * block_of_vis  host [nvis] int32, block index of each visibility in [0, d).
 * kernel_width  J, even in [2, 16]: the interpolation kernel of G is J x J
 *               (Sec. 5 uses 8 x 8).
 * kb_beta       Kaiser-Bessel shape; 0 selects pi*sqrt((J/2)^2*1.5^2 - 0.8).
 * nbases        b in [1, 16]; basis_ids host [b]: 0 = Dirac, k = db_k (1..8).
 * levels        wavelet levels 1 <= L <= 13 with nx >> L >= 1 and ny >> L >= 1.
 * precision     PD_F32 (complex64 bulk data, FP64 reductions) or PD_F64.
 * tile          gridding tile edge in cells (power of two, >= J); 0 = choose.
 * g_mode        PD_G_ON_THE_FLY: the interpolation weights of G are evaluated in the
 *               kernels; PD_G_CSR: G is built once at plan time, on the device, as a
 *               sparse matrix in CSR form (Sec. 2: G is sparse with J^2 entries per
 *               row): row m (one visibility) holds J^2 (column, weight) pairs, the
 *               column packing the grid cell as (ky << 16 | kx) and the weight the
 *               FP64 product of the two axis weights rounded once to the working
 *               precision; every row has J^2 entries, so the row pointer is m J^2.
 *               J^2 (4 + sizeof real) bytes per visibility (8.6 GB at 16.8M
 *               visibilities, J = 8, FP32), held by the plan. Both modes apply the
 *               same operator (to rounding); CSR needs J <= 8 (PD_ENOTSUP otherwise).
 * dde_width     0 (or 1 with unit kernels): no direction-dependent effects. Otherwise
 *               the odd width d >= 3 of each visibility's Fourier-domain DDE kernel,
 *               and G is the DDE-aware matrix of Sec. 2 (G "models the compact support
 *               DDEs as a convolution in the Fourier domain"): row m is the J x J
 *               interpolation kernel convolved with the d x d kernel D_m, so it has
 *               (J + d - 1)^2 complex entries, (G b)_m = sum_k D_m[k] sum_c
 *               phi_m(c - k) b[c]. Needs g_mode = PD_G_CSR and J + d - 1 <= 8
 *               (PD_EINVAL / PD_ENOTSUP otherwise); the entries are complex, so the
 *               matrix takes (J + d - 1)^2 (4 + 2 sizeof real) bytes per visibility.
 * dde_kernels   with dde_width >= 3: host complex128 [nvis][d][d] (interleaved re, im),
 *               user visibility order, D_m[i][j] at grid offset (ky, kx) = (i - h, j - h),
 *               h = (d - 1) / 2; read during pd_plan_create only.
 */
typedef struct {
    int32_t nx, ny;
    int32_t osf;
    int64_t nvis;
    const double* uv;
    int32_t nblocks;
    const int32_t* block_of_vis;
    int32_t kernel_width;
    double kb_beta;
    int32_t nbases;
    const int32_t* basis_ids;
    int32_t levels;
    int32_t precision;
    int32_t tile;
    int32_t g_mode;
    int32_t dde_width;
    const double* dde_kernels;
} pd_plan_desc;

typedef enum { PD_G_ON_THE_FLY = 0, PD_G_CSR = 1 } pd_g_mode;

/*
 * Build a plan: validate the description, sort the visibilities by gridding
 * tile and block, derive the Daubechies filters, the deapodisation and twiddle
 * tables, and allocate the plan's device scratch on the current device.
 * Sec. 2 (Phi = G F Z), Sec. 3 (data split, Psi). *out receives the plan.
 * Errors: PD_EINVAL (bad description), PD_ENOMEM, PD_ECUDA.
 */
pd_status pd_plan_create(const pd_plan_desc* desc, pd_plan** out);

/*
 * Autotuner of the gridding tile edge (the tile and bin size of the tile-binned
 * degridding and gridding). For each candidate tile (powers of two >= J) it builds
 * the plan of `desc` with that tile, runs `iters` iterations of Algorithm 1 (after
 * one warm-up) with every block and basis drawn at probability 1/2 on zero data,
 * and times them with CUDA events on `stream`. Host outputs: the fastest tile in
 * *best_tile and, if ms is non-NULL, the mean milliseconds per iteration of each
 * candidate (ms[k] < 0 for a candidate the plan rejects). Allocates and frees the
 * trial plans; synchronises `stream`. Use the result as desc->tile.
 */
pd_status pd_plan_autotune(const pd_plan_desc* desc, const int32_t* candidates, int32_t ncand, int32_t iters,
                           int32_t* best_tile, double* ms, void* stream);
pd_status pd_plan_destroy(pd_plan* plan);

/* Static description of the last error on the calling thread (never NULL). */
const char* pd_last_error(void);

/*
 * Plan facts, host outputs (any pointer may be NULL):
 * grid size (Ky, Kx), the Kaiser-Bessel beta in use, the tile edge, the number
 * of (tile, block) segments, the number of tiles holding visibilities, and
 * bytes of device memory the plan holds.
 */
pd_status pd_plan_info(const pd_plan* plan, int32_t* ky, int32_t* kx, double* beta,
                       int32_t* tile, int64_t* nsegments, int64_t* ntiles_nonempty,
                       int64_t* device_bytes);

/* Daubechies low-pass filter of basis id k (1..8) as derived by the plan,
 * written to host h[2k] (largest tap first, sum sqrt(2)). */
pd_status pd_daubechies_filter(int32_t k, double* h);

/*
 * y = Phi x = G F Z x (Sec. 2) for `batch` images.
 * x: device real [batch][ny][nx]; y: device complex [batch][nvis], user order.
 * Errors: PD_EINVAL (null pointers, batch < 1), PD_ECUDA.
 */
pd_status pd_apply_phi(pd_plan* plan, const void* x, void* y, int32_t batch, void* stream);

/*
 * x = Re(Phi^H y) = Re(Z^T F^H G^T y): the adjoint of Phi as a map from real
 * images to complex visibilities (used in Alg. 1 step 17).
 * y: device complex [batch][nvis], user order; x: device real [batch][ny][nx].
 */
pd_status pd_apply_phi_adj(pd_plan* plan, const void* y, void* x, int32_t batch, void* stream);

/*
 * Analysis coeffs = Psi^H x = b^{-1/2} [Psi_1^T x; ...; Psi_b^T x] (Sec. 3).
 * x: device real [ny][nx]; coeffs: device real [b][ny][nx], each basis in the
 * packed periodic wavelet layout (coarsest approximation top-left).
 */
pd_status pd_apply_psi_adj(pd_plan* plan, const void* x, void* coeffs, void* stream);

/*
 * Psi^H x without a plan and without allocating device memory (the paper has no
 * counterpart; this is a deployment variant of pd_apply_psi_adj). For callers
 * that cannot call cudaMalloc once they are running: code that must keep to a
 * device-memory budget fixed at start-up (a real-time pipeline that reserves all
 * of its memory up front, or a host application whose own pool owns the device
 * memory), where a plan's allocations would break that budget. The output equals
 * pd_apply_psi_adj's for the same image, bases and levels.
 *
 * x: device real [ny][nx]; coeffs: device real [nbases][ny][nx] (packed layout,
 * scaled by nbases^{-1/2}); basis_ids: host [nbases] (0 = Dirac, k = db_k), read
 * during the call only (it travels to the GPU as a kernel argument);
 * precision PD_F32 / PD_F64 selects float / double data; 1 <= levels <= 13.
 * Scratch: the library's file-scope 16 MiB device array (held by every GPU that
 * loads the library until exit). Calls needing more than it holds -- about
 * 2 * nbases * (ny/2) * (nx/2) elements plus the filter tables -- fail with
 * PD_EINVAL and a message naming the size. Every call shares the array, so calls
 * that overlap on the GPU (different streams, or different host threads without
 * ordering) race; order them on one stream. `stream` must belong to the current
 * device (PD_EINVAL otherwise); NULL is the current device's legacy stream.
 * The first call on a device does a one-time set-up: it looks up the array's
 * device address with that device current and writes the Daubechies filter tables
 * into the array with a synchronous copy; make that first call before any stream
 * capture. Later calls copy nothing from host memory. Asynchronous on `stream`.
 */
pd_status pd_apply_psi_adj_noalloc(const void* x, void* coeffs, int32_t nx, int32_t ny, int32_t levels,
                                   const int32_t* basis_ids, int32_t nbases, int32_t precision,
                                   void* stream);

/* Synthesis x = Psi coeffs = b^{-1/2} sum_j Psi_j coeffs_j (Sec. 3). */
pd_status pd_apply_psi(pd_plan* plan, const void* coeffs, void* x, void* stream);

/*
 * Operator norms by the power method (Sec. 5): ||Phi||_S^2 and ||Psi||_S^2,
 * the largest eigenvalues of Re(Phi^H Phi) and Psi Psi^H, from the device
 * start image x0 [ny][nx] (not modified). Norms and the stopping test
 * |lambda_k - lambda_{k-1}| <= tol * lambda_k are FP64. Host outputs; the call
 * synchronises `stream`. PD_ENOTCONV if max_iter is reached first (outputs
 * still hold the last estimate).
 */
pd_status pd_operator_norms(pd_plan* plan, const void* x0, int32_t max_iter, double tol,
                            double* phi_norm2, double* psi_norm2, int32_t* iterations,
                            void* stream);

/*
 * Algorithm 1 state: x, x~, s (b packed coefficient sets), s~ = Psi s, the data
 * duals v (internal order), the gridded dual sum U = G^T v, the block data y and
 * bounds eps, residual norms for the adaptive probabilities, and the iteration
 * counter t. Allocated on the current device by pd_state_create.
 */
pd_status pd_state_create(pd_plan* plan, pd_state** out);
pd_status pd_state_destroy(pd_state* st);

/*
 * Load the measurements and reset the iterate to the paper's start values
 * (x = x~ = s = v = 0, t = 0). y: device complex [nvis], user order; eps: host
 * double [nblocks], eps_i > 0. The residual norms used by the adaptive
 * probabilities start at ||y_i|| (= ||Phi_i x^(0) - y_i||).
 */
pd_status pd_state_set_data(pd_plan* plan, pd_state* st, const void* y, const double* eps,
                            void* stream);

/*
 * Weights of the reweighted analysis prior (SARA, Sec. 2, which cites but does not
 * define it): weights = delta / (delta + |Psi^H x|) per coefficient of the normalised
 * dictionary Psi^H x (the coefficients pd_apply_psi_adj writes), the usual reweighted-l1
 * rule. x: device real [ny][nx]; weights: device real [nbases][ny][nx], caller-owned,
 * written on `stream` (asynchronous). delta > 0 sets the scale below which a coefficient
 * counts as zero; the outer loop that recomputes the weights from the current x and
 * lowers delta between runs of pd_iterate is the caller's. Uses the plan's wavelet
 * scratch like pd_apply_psi_adj. Errors: PD_EINVAL (null, delta <= 0), PD_ECUDA.
 */
pd_status pd_sara_weights(pd_plan* plan, const void* x, double delta, void* weights, void* stream);

/*
 * Start values of Algorithm 1 (step 1: x^(0), x~^(0), s^(0), v^(0) are given), for a
 * warm start or a resumed reconstruction. Call after pd_state_set_data (it keeps y
 * and eps). x0, x_tilde0: device real [ny][nx]; s0: device real [b][ny][nx]
 * (packed layout); v0: device complex [nvis], user order; any of them may be NULL
 * for zeros. Derives the state's s~ = Psi s^(0), U = G^T v^(0) and the adaptive
 * residual norms ||Phi_i x^(0) - y_i||, and resets t to 0. Reads the inputs on
 * `stream` and synchronises it before returning. Errors: PD_EINVAL, PD_ECUDA.
 */
pd_status pd_state_set_start(pd_plan* plan, pd_state* st, const void* x0, const void* x_tilde0,
                             const void* s0, const void* v0, void* stream);

/* Iteration parameters (host memory, read during pd_iterate). */
typedef struct {
    double tau, sigma, varsigma;   /* step sizes (Sec. 3 convergence condition) */
    double kappa;                  /* normalised soft threshold (Alg. 1 step 13) */
    double psi_norm;               /* ||Psi||_S; the threshold is kappa * psi_norm */
    uint64_t seed;                 /* key of the counter-based active-set draws */
    const double* p_block;         /* host [nblocks] selection probabilities in (0, 1] */
    const double* p_basis;         /* host [nbases] basis probabilities in (0, 1] */
    int32_t adaptive;              /* 1: p_block from Sec. 4 eq. prob-choice */
    double adapt_n, adapt_p_min, adapt_p_max;   /* n, p_check, p_hat of eq. prob-choice */
    int32_t use_graph;             /* 1: capture one iteration in a CUDA graph and replay it */
    int32_t profile;               /* 1 (and use_graph = 0): time every kernel phase with CUDA
                                      events on `stream`; synchronises after each iteration */
    int32_t adapt_exact;           /* with adaptive = 1: 0 takes c_i (Sec. 4) from ||G_i b - y_i|| of
                                      the last iteration block i was active (free, lagged); 1 takes
                                      it from ||Phi_i x^(t) - y_i|| of every block after every
                                      iteration (Sec. 4's definition; one extra forward FFT and a
                                      degridding pass over all visibilities per iteration) */
    int32_t per_block;             /* 1: the plain per-block form, for comparison with the batched
                                      one: the host draws the active sets (same Philox draws) and
                                      launches the degridding, ball projection and gridding
                                      (four tile-colour launches) once per active block and the
                                      wavelet analysis and synthesis once per active basis;
                                      same results up to rounding
                                      order. Needs adaptive = 0 and use_graph = 0; synchronises
                                      `stream` after every iteration. */
    const void* sparsity_weights;  /* NULL: the l1 prior of Sec. 2 (problem analysis-l1). Else device
                                      real [nbases][ny][nx], packed like s, caller-owned: the
                                      per-coefficient weights W of the reweighted prior of SARA
                                      (Sec. 2), min ||W Psi^H x||_1, whose step-13 threshold is
                                      kappa * psi_norm * W; values in (0, 1] (pd_sara_weights).
                                      Read by every iteration; a graph is re-captured when the
                                      pointer changes, not when the values do. */
} pd_params;

/*
 * Run `niter` iterations of Algorithm 1 (steps 3-18) on `stream`:
 * active-set draws (step 3; Philox-4x64-10 keyed by (seed, 0), counter
 * (t, stream, index, 0)), FZx~ (step 4), degridding and the l2-ball dual update
 * of active blocks (step 8), gridding of the dual change (step 9), the
 * soft-threshold dual update of active bases (step 13) and its synthesis
 * (step 14), and the primal update with positivity and over-relaxation
 * (steps 17-18). Errors: PD_EINVAL (probabilities outside (0, 1], p_max < n/d,
 * p_min > n/d), PD_ECUDA.
 */
pd_status pd_iterate(pd_plan* plan, pd_state* st, const pd_params* params, int32_t niter,
                     void* stream);

/*
 * The synthesis formulation (Sec. 2 names a synthesis approach beside the analysis
 * problem): x = Psi alpha with alpha the [nbases][ny][nx] coefficients of the same
 * normalised dictionary, minimise kappa ||alpha||_1 subject to ||y_i - Phi_i Psi alpha||
 * <= eps_i for every block and Psi alpha >= 0, by niter iterations of the primal-dual
 * template of Algorithm 1 with the roles of the two non-smooth terms exchanged:
 * draw the active blocks (params->p_block, seed; the same Philox draws), x~ = Psi alpha~,
 * the ball dual update of steps 5-8 for the active blocks, the positivity dual
 * u <- min(u + x~, 0), then alpha <- S_{tau kappa}(alpha - tau Psi^H(sigma u + varsigma
 * Re(Phi^H v))) and alpha~ = 2 alpha_new - alpha. Uses tau, sigma, varsigma, kappa,
 * seed and p_block of params (p_basis is ignored: every coefficient is updated);
 * adaptive, per_block, use_graph and profile must be 0. The state's s holds alpha
 * (pd_state_get_s) and, after the call, x holds Psi alpha (pd_state_get_x); start from
 * pd_state_set_data (zeros). A state iterated in this form must not be passed to
 * pd_iterate before pd_state_set_data resets it. Synchronises `stream` before
 * returning. Errors: PD_EINVAL, PD_ENOMEM, PD_ECUDA.
 */
pd_status pd_synthesis_iterate(pd_plan* plan, pd_state* st, const pd_params* params, int32_t niter,
                               void* stream);

/*
 * One iteration split at its only exchange point, for a problem whose data blocks are
 * spread over several GPUs (Sec. 3: the data blocks are processed in parallel and only
 * sum_i G_i^T v_i travels back to the primal update). Each rank plans its own
 * visibilities with the global block count (its other blocks hold no visibilities), so
 * that the counter-based draws agree on every rank; the primal variables are
 * replicated (every rank runs the same primal update).
 * pd_iterate_dual: steps 3-14 (draws, F Z x~, degridding and the l2-ball update of this
 * rank's active blocks, gridding of their dual change into the state's U, the sparsity
 * dual update). The caller then sums U over the ranks (pd_state_u gives the device
 * pointer of the state's U, complex [Kx/4][Ky][4] column panels, Kx*Ky elements; the
 * sum must go to another buffer, since U keeps this rank's own part).
 * pd_iterate_primal: steps 17-18 with the summed U (device, same layout; NULL = the
 * state's own U). adaptive must be 0 (the residual norms would differ between ranks).
 * Both asynchronous on `stream`; pd_iterate_dual + pd_iterate_primal(NULL) equals one
 * iteration of pd_iterate. Errors: PD_EINVAL, PD_ECUDA.
 */
pd_status pd_iterate_dual(pd_plan* plan, pd_state* st, const pd_params* params, void* stream);
pd_status pd_iterate_primal(pd_plan* plan, pd_state* st, const pd_params* params, const void* u, void* stream);
pd_status pd_state_u(pd_state* st, void** u, int64_t* elements);

/*
 * Per-phase kernel times accumulated by iterations run with params.profile = 1:
 * ms[k] (host) is the summed CUDA-event time of phase k and iterations[k] how
 * many iterations contributed, for k < min(n, 11); reset = 1 clears the sums.
 * Phase names come from pd_phase_name(k) (e.g. "degrid_dual", "fwd_cols").
 */
pd_status pd_state_profile(pd_state* st, double* ms, int64_t* iterations, int32_t n, int32_t reset);
const char* pd_phase_name(int32_t phase);

/* Copies out of the state (device destinations; asynchronous). */
pd_status pd_state_get_x(const pd_state* st, void* x, void* stream);
pd_status pd_state_get_x_tilde(const pd_state* st, void* x_tilde, void* stream);
pd_status pd_state_get_s(const pd_state* st, void* s, void* stream);        /* [b][ny][nx] */
pd_status pd_state_get_v(const pd_plan* plan, const pd_state* st, void* v, void* stream); /* user order */

/*
 * Diagnostics of the last iteration, host outputs (synchronises `stream`):
 * t, ||x^t - x^{t-1}||^2 and ||x^t||^2 (FP64), per-block residual norms
 * ||G_i b~ - y_i|| of the last iteration each block was active (host
 * [nblocks], may be NULL), current block probabilities (host [nblocks], may be
 * NULL) and the activity of the last draw (host int32 [nblocks] and
 * [nbases], may be NULL), and the size of the last iteration's work lists (host
 * int32 [2]: (tile, block) segments of active blocks, tiles holding an active
 * block; may be NULL).
 */
pd_status pd_state_report(const pd_plan* plan, const pd_state* st, int64_t* t, double* dx2,
                          double* x2, double* res_norm, double* p_block, int32_t* block_active,
                          int32_t* basis_active, int32_t* work, void* stream);

/*
 * Checkpoint: the full state as one host byte buffer. pd_state_save writes
 * pd_state_bytes() bytes to host `buf`; pd_state_load restores it (same plan).
 * The counter-based draws make a resumed run identical to an uninterrupted one.
 */
size_t pd_state_bytes(const pd_plan* plan);
pd_status pd_state_save(const pd_plan* plan, const pd_state* st, void* buf, void* stream);
pd_status pd_state_load(const pd_plan* plan, pd_state* st, const void* buf, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PD_GB300_H */
