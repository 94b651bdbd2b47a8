/*
 * libpurify: recursive polynomial purification of the one-particle density
 * matrix D = theta(mu I - F) on one NVIDIA GB300 (sm_103a).
 *
 * Method: E. H. Rubensson, "Non-monotonic recursive polynomial expansions for
 * linear scaling calculation of the density matrix", arXiv:1101.0265.
 *   - the problem: D = theta(mu I - F), introduction;
 *   - the recursion X_0 = f_0(F), X_i = f_i(X_{i-1}): Eq. 1;
 *   - fixed-mu scale-and-fold McWeeny (P_{1,1}): Eq. 2, Eq. 3, Algorithm 1;
 *   - varying-mu scale-and-fold P_{1,0} / P_{0,1}: Eq. 4, Eq. 5, Algorithm 2;
 *   - the alpha = 1 / alpha = 0 reference schemes the paper compares with
 *     (regular grand-canonical McWeeny; second-order trace-correcting).
 *
 * Conventions for every entry point:
 *   - Return value: PURIFY_OK (0) or a negative PURIFY_ERR_* code.  No C++
 *     exception crosses this boundary.  purify_strerror() names a code.
 *   - Matrices are dense, row-major, float64, with a leading dimension
 *     (elements between consecutive rows) >= n.  Only symmetric matrices are
 *     accepted; F's upper triangle (j >= i) is read and mirrored.
 *   - Pointers passed to purify_set_hamiltonian / purify_get_density may be
 *     host memory (pageable or pinned) or device memory of the handle's
 *     device; the library tells them apart with cudaPointerGetAttributes.
 *     The caller keeps ownership; the library copies F and never retains a
 *     caller pointer after the call returns.
 *   - A handle owns all device memory it uses and is NOT thread-safe; separate
 *     handles are independent.  Work is issued on the handle's stream; the
 *     calls that return host-visible results synchronise that stream.
 *   - The purify_k_* entry points run one kernel family on caller-owned
 *     DEVICE pointers, asynchronously on the given stream (NULL = the legacy
 *     default stream), and allocate nothing unless stated.
 */
#ifndef LIBPURIFY_PURIFY_H
#define LIBPURIFY_PURIFY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PURIFY_OK                   0
#define PURIFY_ERR_INVALID_ARG     -1  /* bad pointer, size, scheme or option      */
#define PURIFY_ERR_BOUNDS          -2  /* inconsistent spectral bounds, zero gap,
                                          or a trace that shows occupied and
                                          unoccupied states mixed up              */
#define PURIFY_ERR_NOT_CONVERGED   -3  /* max_iter reached; stats still filled     */
#define PURIFY_ERR_OOM             -4  /* device allocation failed                 */
#define PURIFY_ERR_CUDA            -5  /* a CUDA runtime/driver call failed        */
#define PURIFY_ERR_DEVICE_TIMEOUT  -6  /* a bounded device-side wait ran out       */
#define PURIFY_ERR_STATE           -7  /* call order (e.g. run before set)         */
#define PURIFY_ERR_UNSUPPORTED     -8  /* no sm_103a device / feature not built    */
#define PURIFY_ERR_INTERNAL        -9  /* a consistency check inside a kernel failed
                                          (a library bug; purify_stats_t.device_flag
                                          has the raw flag)                       */

/* ---- schemes (Algorithm 1, Algorithm 2 and their reference forms) ------- */
#define PURIFY_FIXED_MU_SF    0  /* Algorithm 1: P_{1,1}(alpha(X - I/2) + I/2)      */
#define PURIFY_FIXED_MU_MONO  1  /* Algorithm 1 with alpha = 1 (regular McWeeny)     */
#define PURIFY_TC_SF          2  /* Algorithm 2: Eq. 4 / Eq. 5 with scaling alpha    */
#define PURIFY_TC_MONO        3  /* Algorithm 2 with alpha = 0 (trace-correcting)    */
/* The fixed-mu scheme with the higher-order P_{3,3}(x) = x^4 (35 - 84x + 70x^2
 * - 20x^3) (the scheme stated with Algorithm 1 for odd m; alpha >= 1 solves
 * P_{3,3}(alpha(beta - 1/2) + 1/2) = P_{3,3}((1 - alpha)/2) by bisection);
 * five products per iteration. */
#define PURIFY_FIXED_MU_P33_SF   4
#define PURIFY_FIXED_MU_P33_MONO 5  /* the same with alpha = 1                     */
/* Asymmetric P_{i,j} (i, j odd, i != j) scaled about their unstable fixed
 * point c (the paper: for i != j the scaling is about that point rather than
 * 1/2): X_0 = c I + (mu I - F) / gamma, gamma = max((mu - lmin) / (1 - c),
 * (lmax - mu) / c); per iteration alpha = the smaller of the two sides' fold
 * solutions, and beta (unoccupied) and beta_bar (occupied) follow their
 * edges' and folded ends' images.  P_{1,3} = x^2 (10 - 20x + 15x^2 - 4x^3):
 * four products per iteration; P_{3,1} = x^4 (5 - 4x): three. */
#define PURIFY_FIXED_MU_P13_SF   6
#define PURIFY_FIXED_MU_P13_MONO 7
#define PURIFY_FIXED_MU_P31_SF   8
#define PURIFY_FIXED_MU_P31_MONO 9
#define PURIFY_SCHEME_LAST       9

/* ---- arithmetic of the matrix products -------------------------------- */
#define PURIFY_FP64    0  /* float64 FMA on the SIMT pipes                          */
#define PURIFY_MIXED   1  /* float64 values held as integer digit planes in bf16,
                             multiplied exactly on the tcgen05 tensor cores with
                             fp32 accumulation in tensor memory, recombined in
                             float64; number of digits set per step               */

/* ---- branch rule of the varying-mu schemes ---------------------------- */
#define PURIFY_BRANCH_BETA   0  /* Algorithm 2's test: beta + beta_bar > 1 -> P_{1,0} */
#define PURIFY_BRANCH_TRACE  1  /* trace(X_{i-1}) > nocc -> P_{1,0} (Niklasson)       */

typedef struct purify_ctx* purify_t;

/* Spectral landmarks of F: extremal eigenvalues (or bounds of them) and the
 * eigenvalues just below (homo) and above (lumo) the gap (Algorithm 1 and
 * Algorithm 2, "Require" lines).  lmin / lmax may be NaN: they are then
 * estimated on the device (Gershgorin discs tightened by Lanczos).  homo /
 * lumo may be NaN only for PURIFY_TC_MONO with PURIFY_BRANCH_TRACE, which then
 * stops on idempotency.  Loose inner estimates (homo_est >= homo, lumo_est <=
 * lumo) are safe and only slow convergence; homo >= lumo is rejected. */
typedef struct purify_bounds {
    double lmin, lmax, homo, lumo;
} purify_bounds;

typedef struct purify_options {
    int precision;       /* PURIFY_FP64 (default) or PURIFY_MIXED                        */
    int branch_rule;     /* PURIFY_BRANCH_BETA (default) or PURIFY_BRANCH_TRACE          */
    int lanczos_steps;   /* Lanczos steps when lmin/lmax are NaN (default 16, 0 = none):
                            the Ritz values widened by their residuals land within a
                            few per cent of the spectral ends, and a few per cent of
                            width moves an iteration count by log2(1.0x), i.e. not at
                            all in practice                                          */
    int refine_squares;  /* MIXED: extra unscaled McWeeny steps at the finest digit
                            count after the schedule ends (default 0)                  */
    int digits;          /* MIXED: 0 = per-step digit count from the mapped gap
                            (default); 2..6 = fixed count                             */
    int time_products;   /* 1 = bracket every matrix-product launch with CUDA events
                            on the handle's stream and report their total time (a
                            dense run's queue launches: one interval)               */
    int block_sparse;    /* MIXED, Algorithm 2 schemes: keep every iterate as a
                            pattern of 32 x 32 blocks, form products only over
                            nonzero blocks and truncate after every step         */
    int split_k;         /* MIXED dense products: cut the tiles of the persistent
                            grid's last, partial wave into k-ranges that run on
                            the idle SMs and are added in a fixed order (default 1;
                            0 = whole tiles, the grouping the batch engine uses) */
    int refine_fp64;     /* MIXED: float64 McWeeny steps X <- 3X^2 - 2X^3 (two float64
                            products each, on the GPU's float64 pipe) appended to the
                            run, which set the final idempotency (0 = none, default;
                            at most 2); stats.trace and stats.idem_err_fro then
                            describe the last of them                              */
    int bits_floor;      /* MIXED, per-step digit count (digits = 0): the fewest bits a
                            step's operands carry (0 = 30, else 16..43)              */
    int bits_gap;        /* MIXED, per-step digit count: bits beyond log2(1 / mapped
                            gap) that a step's operands carry (0 = 26, else 16..43);
                            a step takes the fewest digits (3..6) whose bits cover
                            max(bits_floor, bits_gap + log2(1 / gap))              */
    int autotune;        /* MIXED dense products: 1 = time the candidate launch shapes
                            (the last wave's tiles split by the rule or whole) at the
                            first product
                            of each digit count and padded size in this process, and
                            launch every later product of that kind with the fastest
                            (0 = the fixed rule, default).  Shapes differ only in the
                            summation order of the inexact digit levels, so results
                            stay within the mixed path's tolerance; within a process
                            one shape per kind is used, so runs are reproducible    */
    int wait_kcycles;    /* MIXED: bound of one device-side work wait of the product
                            kernel (a stage, tensor-memory or work-claim hand-off), in
                            thousands of SM cycles (0 = 2^31 cycles, about one second).
                            A wait that runs out stops the kernel cleanly and the call
                            returns PURIFY_ERR_DEVICE_TIMEOUT; waits for copies and
                            MMAs already in flight at teardown keep the full bound.
                            Short values exist to exercise failure detection; a
                            nonzero value also disables autotune                   */
    int host_schedule;   /* MIXED with PURIFY_BRANCH_TRACE: 1 = decide every step's
                            branch and coefficients on the host (one device-to-host
                            round trip per step); 0 (default) = a one-thread kernel
                            decides them on the device from the previous product's
                            float64 trace and the steps replay from a CUDA graph,
                            with one host read per 16 steps                        */
    int launch_per_product; /* MIXED dense runs (Algorithms 1 and 2 with the beta-based
                            schedule): 0 (default) = the run's products in queue
                            launches (one per run of equal digit counts), consecutive
                            products overlapping: an item waits on the device only for
                            the two row panels of the previous product that it reads
                            (used when a product has at least two waves of tiles;
                            time_products then times the queue launches as one
                            interval); 1 = one launch per product              */
    int reserved;
    double trunc_tau;    /* block_sparse: per-step truncation budget: blocks of
                            smallest Frobenius norm are dropped while the dropped
                            mass (off-diagonal blocks twice) stays <= tau^2       */
    double trunc_budget; /* block_sparse: when > 0, a total budget for all of the
                            run's truncations instead: tau = trunc_budget / (m + 1)
                            for the m scheduled iterations and X_0, so a scheme
                            that needs fewer iterations truncates harder at the
                            same bound on the accumulated truncation (the closing
                            discussion's argument for sparsity)                 */
} purify_options;

typedef struct purify_stats_t {
    int status;                 /* return code of the last purify_run                    */
    int iterations;             /* iterations of the scheme (f_1 .. f_n)                 */
    int multiplications;        /* matrix products: 2 per Algorithm 1 iteration, 1 per
                                   Algorithm 2 iteration, plus refinement products       */
    int refine_multiplications; /* of which refinement                                   */
    double err_bound;           /* max(beta, 1 - beta_bar) after the last iteration: a
                                   bound on ||X_n - D||_2 in exact arithmetic             */
    double trace;               /* trace(X_n)                                            */
    double trace_err;           /* |trace(X_n) - nocc| (NaN when nocc is unknown)        */
    double idem_err_fro;        /* ||X - X^2||_F of the last iterate that was squared
                                   (Algorithm 2 only; NaN otherwise)                     */
    double seconds;             /* device time of the iteration loop                     */
    double lmin, lmax, homo, lumo, mu;  /* landmarks used                              */
    double useful_flops;        /* n^2 (n + 1) per symmetric product                     */
    double tensor_flops;        /* MMA flops issued on the tensor cores (MIXED)          */
    int digit_max;              /* MIXED: largest digit count used                       */
    int kernel_launches;        /* kernels launched by the last set/run call             */
    int product_launches;       /* matrix-product kernels among them (last run)          */
    int nnz_blocks;             /* block_sparse: upper 32 x 32 blocks of the result      */
    int digit_kc;               /* MIXED: k-chunk width of the last product launch        */
    int device_flag;            /* MIXED: device error flag of the last run (0 = none;
                                   bits 1, 2, 4, 16: a TMA-producer, MMA, epilogue or
                                   work-claim wait gave up; bit 8: a tile's k-chunk
                                   count and bitmask disagreed)                         */
    int plane_pool_mib;         /* block_sparse: peak MiB of the pooled digit planes of
                                   the iterates (both pools; 0 otherwise)                */
    int reserved;
    double product_seconds;     /* summed event time of the product launches
                                   (time_products = 1; else NaN)                         */
} purify_stats_t;

/* Fill *opt with the defaults above. */
void purify_options_default(purify_options* opt);

/* Create a handle on CUDA device `device`.  `cuda_stream` is the caller's
 * cudaStream_t (NULL = the legacy default stream).  The handle queues its
 * work on a private non-blocking stream; every call first orders that stream
 * after the work the caller has queued on `cuda_stream` (device inputs
 * produced there are complete when the handle reads them) and, before it
 * returns, orders `cuda_stream` after the handle's work.  `opt` may be NULL
 * (defaults).  Fails with PURIFY_ERR_UNSUPPORTED if the device is not compute
 * capability 10.3. */
int purify_create(purify_t* h, int device, void* cuda_stream, const purify_options* opt);

/* Release the handle and all device memory it owns.  NULL is accepted. */
int purify_destroy(purify_t h);

/* Replace the handle's options (takes effect at the next set/run). */
int purify_set_options(purify_t h, const purify_options* opt);

/* Load F (n x n, leading dimension ld, host or device) and its landmarks.
 * A host F has been read when the call returns; a device F is read on the
 * handle's stream after the work already queued on the caller's stream.
 * nocc < 0 means unknown; mu NaN means mu = (homo + lumo) / 2 (fixed-mu
 * schemes).  When b->lmin or b->lmax is NaN, the bounds are estimated here
 * (Gershgorin discs, then `lanczos_steps` Lanczos steps from a SplitMix64
 * start vector, Ritz values widened by their residuals and clipped to the
 * discs).  The estimate runs on the device; its result is in purify_stats. */
int purify_set_hamiltonian(purify_t h, const double* F, int64_t n, int64_t ld,
                           int64_t nocc, double mu, const purify_bounds* b);

/* Load a sparse symmetric F given as COO triplets (host arrays rows[k],
 * cols[k], vals[k], 0-based, both triangles present) into the handle's dense
 * float64 copy; otherwise as purify_set_hamiltonian.  Duplicates are summed in
 * input order; the summed (i, j) and (j, i) entries must be equal, else
 * PURIFY_ERR_INVALID_ARG (so is an index outside [0, n)).  A handle with
 * block_sparse = 1 and MIXED precision keeps F in CSR form instead (no n x n
 * array; n up to 2^18): the bound estimate and the block-sparse run read the
 * CSR form, and any other path makes the dense copy when it first needs it. */
int purify_set_hamiltonian_coo(purify_t h, int64_t n, int64_t nnz, const int64_t* rows,
                               const int64_t* cols, const double* vals, int64_t nocc, double mu,
                               const purify_bounds* b);

/* Gap edges from the purification (Algorithms 1 and 2 need a lower bound of
 * the gap's lower edge and an upper bound of its upper edge; the paper's
 * discussion points to techniques for interior eigenvalues).  Needs F, nocc
 * (0 < nocc < n) and lmin/lmax from purify_set_hamiltonian.  Runs steps of
 * the alpha = 0 scheme with the trace rule until ||X - X^2||_F < 1 / (4
 * sqrt(n)) and round(trace X) = nocc, then `lanczos_steps` Lanczos steps on
 * X^4 (I - X) and on X (I - X)^4, whose largest eigenvalues belong to the
 * images of homo and lumo; Ritz values raised by their residual norms are
 * mapped back through the steps taken.  The results lie inside the gap
 * (homo <= *homo_est < *lumo_est <= lumo, up to the iterate's rounding on the
 * mixed path) and become the handle's gap bounds for purify_run.  Uses the
 * handle's precision; the handle holds no density afterwards.  Returns
 * PURIFY_ERR_NOT_CONVERGED when the sides are not resolved within 200 steps. */
int purify_estimate_gap(purify_t h, int lanczos_steps, double* homo_est, double* lumo_est);

/* The launch shape that purify_options.autotune measured on `device` for
 * products of `digits` digit planes at size n (padded to 128): k-chunk width
 * (*kc) and the last wave's split (*split_ways: 0 = the rule, 1 = whole
 * tiles).  Host only; a launch setting of this library, not an operation of
 * the paper.  PURIFY_ERR_STATE when nothing was measured for that kind in
 * this process, PURIFY_ERR_INVALID_ARG for null outputs, n <= 0 or digits
 * outside 1..6. */
int purify_tuned_shape(int device, int digits, int64_t n, int* kc, int* split_ways);

/* Block-sparse runs: the number of upper 32 x 32 blocks kept after the
 * truncation of X_0 and of every step (count <= cap entries written). */
int purify_block_history(purify_t h, int* nnz_blocks, int cap, int* count);

/* Block-sparse runs keep the density as its kept 32 x 32 blocks (the blocks
 * that survived the last truncation; purify_get_density expands them into
 * an n x n array).  This copies them out: *count receives the number of kept
 * blocks with I <= J (their (I, J) in row-major order); at most cap of them
 * are written, block_ij[2k], block_ij[2k + 1] = (I, J) and values[1024 k ..
 * 1024 k + 1023] = the block's rows (row-major, entries at rows or columns
 * >= n are 0).  block_ij and values may be host or device memory, either may
 * be NULL.  PURIFY_ERR_STATE unless the last run was block-sparse. */
int purify_get_density_blocks(purify_t h, int32_t* block_ij, double* values, int64_t cap, int64_t* count);

/* Run `scheme` until the bound of the scheme's scalar recursion (beta for
 * Algorithm 1, max(beta, 1 - beta_bar) for Algorithm 2) is <= tol, or, for
 * PURIFY_BRANCH_TRACE without gap bounds, until ||X - X^2||_F <= tol; at most
 * max_iter iterations.  Returns PURIFY_ERR_NOT_CONVERGED (stats filled,
 * density available) when max_iter is reached, and PURIFY_ERR_BOUNDS when
 * nocc >= 0 and the final trace differs from nocc by more than 0.5.
 * PURIFY_BRANCH_TRACE takes each branch from trace(X_{i-1}) on both
 * precisions (one host round trip per step; on the mixed path the trace is
 * reduced in float64 by the previous product's epilogue); it is unsupported
 * with block_sparse. */
int purify_run(purify_t h, int scheme, double tol, int max_iter);

/* Copy the current density matrix (the last X_i, symmetric, n x n) into D
 * (host or device, leading dimension ld >= n). */
int purify_get_density(purify_t h, double* D, int64_t ld);

/* Copy the statistics of the last set/run into *out. */
int purify_stats(purify_t h, purify_stats_t* out);

/* Per-iteration reductions of the last purify_run, as the fused epilogue of
 * each step's product reduced them in float64 (Eq. 1's X_i; for Algorithm 2
 * the square of Eq. 4 / Eq. 5 is X_{i-1}^2):
 *   trace[i] = trace(X_{i+1}) for i = 0 .. iterations-1,
 *   idem[i]  = ||X_i - X_i^2||_F, the idempotency of the iterate that step
 *              i + 1 squared (Algorithm 2 schemes; NaN for the fixed-mu
 *              schemes, whose products square the scaled X_s).
 * Refinement steps are not included.  Either array may be NULL; at most cap
 * entries are written and *count receives the number of iterations.
 * PURIFY_ERR_STATE before a successful run. */
int purify_step_history(purify_t h, double* trace, double* idem, int cap, int* count);

/* Device pointer of the handle's current density (n x n, leading dimension
 * n, float64), valid until the next set/run/destroy; NULL before a run and
 * after a block-sparse run (see purify_get_density_blocks). */
const double* purify_density_device_ptr(purify_t h);

/* Human-readable name of a status code (static string). */
const char* purify_strerror(int code);

/* ---- host-only: the scalar schedule ------------------------------------ */

/* The scalar recursion of a scheme with the beta rule, computed on the host
 * (Algorithm 1: alpha, beta; Algorithm 2: branch, alpha, beta, beta_bar),
 * exactly as purify_run uses it.  Arrays have room for max_iter entries; any
 * of them may be NULL.  branch[i] = 1 for P_{1,0}, 0 for P_{0,1} (0 for
 * Algorithm 1).  *iterations receives the count; returns
 * PURIFY_ERR_NOT_CONVERGED if max_iter is reached first.  Needs no GPU. */
int purify_schedule(int scheme, double lmin, double lmax, double mu, double homo, double lumo,
                    double tol, int max_iter, double* alpha, int* branch, double* beta,
                    double* beta_bar, int* iterations);

/* Eigenvalues of the symmetric tridiagonal matrix with diagonal a[0..m) and
 * off-diagonal b[0..m-1) by cyclic Jacobi rotations; w receives them
 * ascending and, if last_row is not NULL, last_row[j] the last component of
 * the j-th normalised eigenvector (for Ritz residuals).  Needs no GPU. */
int purify_tridiag_eig(const double* a, const double* b, int m, double* w, double* last_row);

/* ---- kernel-level entry points (device pointers, asynchronous) ---------- */

/* C = A B for symmetric A, B whose product is symmetric (in the schemes:
 * polynomials of the same matrix), n x n, leading dimension n, float64.
 * Only tiles on or above the diagonal are computed; each is written twice
 * (itself and its transpose).  The matrix product of every step of Eq. 1. */
int purify_k_symm_product_f64(const double* A, const double* B, double* C, int64_t n,
                              void* stream);

/* One fused scheme step in float64 (the matrix form of Eq. 4, Eq. 5 or the
 * two products of Algorithm 1's P_{1,1}), n x n, leading dimension n:
 *   P = A B (upper tiles),  Y = cP P + cE E + cI I,  C = dY Y + dI I,
 * C written with its mirror; E may equal A and may be NULL when cE == 0.
 * red (device, 3 doubles, accumulated with atomics, NOT cleared here):
 *   red[0] += trace(Y), red[1] += ||E - P||_F^2, red[2] += ||Y||_F^2.
 * C must not alias A, B or E. */
int purify_k_step_f64(const double* A, const double* B, const double* E, double* C, int64_t n,
                      double cP, double cE, double cI, double dY, double dI, double* red,
                      void* stream);

/* Gershgorin interval of symmetric F (n x n, leading dimension ld):
 * lohi[0] = min_i (F_ii - R_i), lohi[1] = max_i (F_ii + R_i),
 * R_i = sum_{j != i} |F_ij|.  lohi is device memory.  Allocates (and frees)
 * a device scratch array of 2 * ceil(n / 8) doubles per call. */
int purify_k_gershgorin_f64(const double* F, int64_t n, int64_t ld, double* lohi, void* stream);

/* ---- many Hamiltonians on one device ----------------------------------- */
/* A batch holds any number of purifications of different sizes, schemes and
 * tolerances (the recursion of Eq. 1 with Algorithm 1 or 2 for each), always
 * on the mixed path.  Each instance's product steps are planned when it is
 * added, from its own scalar schedule; a round advances every active
 * instance by one matrix product, with the tiles of all instances that share
 * a digit count in one persistent tensor-core launch.  Instances retire at
 * their own iteration counts.  Not thread-safe; one stream. */
typedef struct purify_batch* purify_batch_t;

/* Device bytes an instance of size n holds while it is in a batch (F, D and
 * three sets of up to 6 digit planes), for admission control. */
int64_t purify_batch_footprint(int64_t n);

/* Create / destroy a batch on `device`.  `cuda_stream` is the caller's stream
 * (NULL = legacy default), joined as for purify_create; the batch's own
 * private stream is the one its CUDA graph is captured on.  opt->digits fixes
 * the digit count (0: from the mapped gap). */
int purify_batch_create(purify_batch_t* b, int device, void* cuda_stream, const purify_options* opt);
int purify_batch_destroy(purify_batch_t b);

/* Add one instance: F (n x n, leading dimension ld, host or device; copied,
 * a host F before the call returns; upper triangle read), nocc (< 0:
 * unknown), mu (fixed-mu schemes; NaN: the
 * gap centre), all four bounds required, scheme, tol, max_iter.  Allocates
 * the instance's device memory (purify_batch_footprint) and writes its id. */
int purify_batch_add(purify_batch_t b, const double* F, int64_t n, int64_t ld, int64_t nocc, double mu,
                     const purify_bounds* bounds, int scheme, double tol, int max_iter, int* id);

/* One round (continuous batching): queue f_0 for instances added since the
 * last round, advance every active instance by one product, synchronise.
 * *active receives the instances still running, *finished those that
 * completed in this round. */
int purify_batch_step(purify_batch_t b, int* active, int* finished);

/* Continuous batching with fewer host round trips: queue f_0 for instances
 * added since the last call, then advance every active instance by up to
 * max_products products (the rest of its schedule if fewer remain) in one
 * queue launch of the product kernel, in which an instance's products run in
 * order and different instances overlap; synchronise.  *active and *finished
 * as for purify_batch_step.  Densities equal those of a run alone, bit for
 * bit.  A CUDA graph captured by purify_batch_run is dropped (its staging is
 * reused).  INVALID_ARG for max_products < 1. */
int purify_batch_advance(purify_batch_t b, int max_products, int* active, int* finished);

/* Run every instance of the batch from f_0 to completion.
 *
 * mode = PURIFY_BATCH_QUEUE (0): the f_0 splits, then ONE persistent launch of
 *   the product kernel over a device queue holding every product of every
 *   instance (round-major, larger instances first).  An item of product k of
 *   an instance waits on the device, with the bounded wait of
 *   opt->wait_kcycles, until product k-1 of that instance has completed, so
 *   each instance advances on its own and retires on the device.
 * mode | PURIFY_BATCH_GRAPH (1): the launches are captured once into a CUDA
 *   graph and replayed by later calls while the set of instances is
 *   unchanged.
 * mode | PURIFY_BATCH_ROUNDS (2): one grouped launch per round (the next
 *   product of every unfinished instance), ordered by the host.
 * Every mode gives the same densities, bit for bit.  Errors: INVALID_ARG for
 * another mode; TIMEOUT when a device wait ran out (see purify_stats_t
 * device_flag of purify_get_stats for the single-matrix analogue). */
#define PURIFY_BATCH_QUEUE 0
#define PURIFY_BATCH_GRAPH 1
#define PURIFY_BATCH_ROUNDS 2
int purify_batch_run(purify_batch_t b, int mode);

/* 1 when instance `id` has finished, 0 while it is pending or running. */
int purify_batch_status(purify_batch_t b, int id);

/* Copy a finished instance's density (host or device, leading dimension ld). */
int purify_batch_get_density(purify_batch_t b, int id, double* D, int64_t ld);

/* Statistics of one instance (trace, idempotency of Algorithm 2, schedule,
 * work); seconds = device time of the last purify_batch_run. */
int purify_batch_stats(purify_batch_t b, int id, purify_stats_t* st);

/* Free an instance's device memory (its id stays invalid afterwards). */
int purify_batch_release(purify_batch_t b, int id);

/* Device bytes held by the batch's instances. */
int64_t purify_batch_bytes_in_use(purify_batch_t b);

/* Largest n accepted by purify_k_gershgorin_f64_noalloc. */
#define PURIFY_GERSHGORIN_NOALLOC_MAX_N 65536

/* The Gershgorin interval of purify_k_gershgorin_f64, for callers that must
 * not allocate device memory: hosts that hand all device memory to their own
 * pool allocator and do not let libraries call cudaMalloc/cudaFree, callers
 * whose device memory budget is fully committed, and latency-sensitive loops
 * that cannot absorb the device-wide synchronisation of cudaFree.  The paper
 * has no counterpart; this is a library-level variant of the bound kernel.
 *
 * It allocates nothing: the per-block partial results live in one static
 * device array of 2 * ceil(PURIFY_GERSHGORIN_NOALLOC_MAX_N / 8) doubles
 * (128 KiB), which every GPU that loads the library holds until the process
 * exits.  n > PURIFY_GERSHGORIN_NOALLOC_MAX_N is rejected with
 * PURIFY_ERR_INVALID_ARG before anything is launched.  The first call on a
 * device looks up that array's device address (once per device and CUDA
 * context, with the device current; after a device reset or a recreated
 * primary context the next call looks it up again); make that first call
 * before any stream capture begins.
 * The work is queued on `stream` and the call returns without synchronising;
 * lohi (device, 2 doubles) is valid once the stream reaches that point.
 * Every call shares the one array and nothing in it needs to start at zero,
 * but calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race on it: serialise them. */
int purify_k_gershgorin_f64_noalloc(const double* F, int64_t n, int64_t ld, double* lohi,
                                    void* stream);

/* k Lanczos steps on symmetric F (n x n, leading dimension n) from the
 * SplitMix64 start vector q_i = 2 u_i - 1, u_i = (splitmix64(key + i *
 * 0x9E3779B97F4A7C15) >> 11) / 2^53 with key 0x11010265.  Writes the
 * tridiagonal diagonal a[0..k) and off-diagonal b[0..k) (b[k-1] = residual
 * norm) to HOST arrays; synchronises the stream.  Allocates 4 n + 2 k + 2
 * doubles of device scratch per call. */
int purify_k_lanczos_f64(const double* F, int64_t n, int k, double* a, double* b, void* stream);

/* C = A B in the arithmetic of PURIFY_MIXED: A and B (n x n, leading
 * dimension n, float64, symmetric, device) are split into `digits` bf16
 * digit planes of 8 bits with scale 2^eA and 2^eB (|A_ij| <= 2^eA, |B_ij| <=
 * 2^eB are required), multiplied on the tcgen05 tensor cores with exact fp32
 * accumulation of the leading digit levels, and recombined; tiles on or
 * above the diagonal are formed and mirrored, so C holds the upper triangle
 * of A B^T mirrored (= A B when A and B commute).  The product of every step
 * of Eq. 1 on the mixed path.  Allocates and frees 2 * digits * p^2 bf16 of
 * device scratch (p = n rounded up to 128); synchronises the stream. */
int purify_k_digit_product_f64(const double* A, const double* B, double* C, int64_t n, int digits,
                               int eA, int eB, void* stream);

/* The product kernel's work plan for a persistent grid of `ctas` CTAs over
 * `tiles` output tiles of `k_chunks` k-chunks each (host only): whole waves
 * of tiles [0, *split_begin) go round-robin over the CTAs; the tiles of the
 * last, partial wave are cut into *ways ranges of k-chunks (ways = 1: none),
 * at most 4, each of at least 4 k-chunks, and at most `ctas` parts in all.
 * A launch setting of this library, not an operation of the paper (exposed
 * for tests).  PURIFY_ERR_INVALID_ARG for non-positive arguments or null
 * outputs. */
int purify_k_split_plan(int tiles, int ctas, int k_chunks, int* split_begin, int* ways);

#ifdef __cplusplus
}
#endif
#endif /* LIBPURIFY_PURIFY_H */
