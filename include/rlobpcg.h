/*
 * rlobpcg.h -- C ABI of the GB300 (sm_103a) RLOBPCG library.
 *
 * RLOBPCG (Epperly, Park & Nakatsukasa, "Fast, high-accuracy, randomized nullspace computations
 * for tall matrices", arXiv 2602.16797) computes the k smallest singular values of a tall matrix
 * A (m x n, m >> n >> 1) and their right singular vectors (Sec. 1): a SparseStack sketch SA
 * (Sec. 2.2) gives a preconditioner and a starting block, then block LOBPCG on A^H A refines them
 * (Algorithm 2; Algorithm 1 is its b = 1 case).
 *
 * Conventions for every entry point:
 *   - Matrices are dense. A is row-major with leading dimension lda >= n (element (i,j) at
 *     A[i*lda + j]). Complex data is interleaved (re, im) pairs of doubles (numpy complex128).
 *   - "device" pointers must be CUDA device (or managed) memory; entry points documented as
 *     accepting host or device pointers detect which through unified addressing.
 *   - The caller owns every pointer it passes; the library never frees or keeps them past the
 *     call, except a plan, which owns its workspace until rlobpcg_plan_destroy.
 *   - Work is issued on the CUDA stream given at plan time (or per call); entry points return
 *     after the stream has finished unless stated otherwise.
 *   - Return value: RLOBPCG_OK (0), a positive warning, or a negative error code.
 *     rlobpcg_status_string() names it; rlobpcg_last_error() gives the detail of the last error.
 */
#ifndef RLOBPCG_H
#define RLOBPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------- */
#define RLOBPCG_OK 0
#define RLOBPCG_NOT_CONVERGED 1      /* max_iter reached; outputs hold the last (best) iterate  */
#define RLOBPCG_ERR_INVALID_ARG (-1) /* bad size, pointer, leading dimension or option           */
#define RLOBPCG_ERR_OOM (-2)         /* device allocation failed                                  */
#define RLOBPCG_ERR_CUDA (-3)        /* a CUDA runtime call failed (detail in rlobpcg_last_error) */
#define RLOBPCG_ERR_NONFINITE (-4)   /* NaN or Inf met in A or in the iteration                   */
#define RLOBPCG_ERR_TIMEOUT (-5)     /* a bounded device-side wait ran out                        */
#define RLOBPCG_ERR_UNSUPPORTED (-6) /* shape outside what the kernels handle                     */
#define RLOBPCG_ERR_CANCELLED (-7)   /* a queued request dropped by rlobpcg_server_destroy          */

/* ---- element types ------------------------------------------------------------------------ */
#define RLOBPCG_F64 0   /* real double                                */
#define RLOBPCG_C128 1  /* complex double, interleaved (re, im)       */

/* Precision of the sketch SA, its QR factor R, the SVD of R and R^{-1}. The Gram products,
 * residuals, Rayleigh-Ritz and orthogonalisation are always FP64 / complex128.
 *   F64:        SA, its QR and R in FP64 (the paper's form).
 *   F32:        SA summed in FP32 and its QR in FP32. Enough when kappa(A) << 1/u_32 ~ 1.7e7; above
 *               that the FP32 factor cannot see the bottom singular directions (Fact 2 of Sec. 3.1
 *               then gives kappa(A P) ~ u_32 kappa(A)) and LOBPCG needs more iterations.
 *   F32_REFINE: SA in FP64, its QR in FP32 (R_32), then one FP64 Cholesky-QR correction on SA:
 *               Y = SA R_32^{-1}, R_c = chol(Y^H Y + s I) with s = n u max_i (Y^H Y)_ii,
 *               R = R_c R_32. R, R^{-1} and the SVD of R are FP64 and as good a preconditioner as
 *               the F64 form's (kappa(Y) ~ u_32 kappa(SA) stays far below 1/sqrt(u)). An addition
 *               of this library; the paper factors in FP64. */
#define RLOBPCG_SKETCH_F64 0
#define RLOBPCG_SKETCH_F32 1
#define RLOBPCG_SKETCH_F32_REFINE 2

/* Stop reasons reported in rlobpcg_info.stop_reason */
#define RLOBPCG_STOP_CONVERGED 0   /* sketched tolerance (+ stagnation checks) held (Sec. 2.1)   */
#define RLOBPCG_STOP_MAX_ITER 1    /* iteration cap (Alg. 1: 200 for b = 1, Alg. 2: 100)         */
#define RLOBPCG_STOP_FIXED 2       /* fixed_iters iterations were run on request                 */

/* Options. rlobpcg_default_opts fills the paper's defaults (Sec. 2.1-2.2). */
typedef struct {
  uint64_t seed;        /* seed of the SparseStack SplitMix64 stream                               */
  int d;                /* sketch rows; 0 means 4n (Alg. 2 uses 4n, Sec. 2.2 suggests 2n..4n)      */
  int zeta;             /* nonzeros per column of S (8 by default; Alg. 2 uses 4)                  */
  int block;            /* block size b >= k; 0 means b = k                                        */
  int max_iter;         /* 0 means 200 when b = 1 (Alg. 1) and 100 otherwise (Alg. 2)              */
  int check_every;      /* stop-test period; 0 means 5 with stagnation checks, 1 without           */
  int use_stagnation;   /* 1: also require the stagnation checks of Sec. 2.1 (default)             */
  int sketch_prec;      /* RLOBPCG_SKETCH_F64 (default), _F32 or _F32_REFINE (see above)           */
  int fixed_iters;      /* > 0: run exactly this many iterations, no stop test (parity runs)       */
  int residual_refresh_every; /* > 0: every this many iterations recompute A^H (A V) with a pass
                                 over A instead of the recombined A^H A V (drift control)         */
  int exact_sketch_svd; /* 1: full one-sided Jacobi SVD of R for V~(:, n-b+1:n) and Sigma~(1,1).
                           0 (default): only those two, by block inverse iteration with
                           (R^H R)^{-1} (3 steps, block 2b+4) + Rayleigh-Ritz on R Z, and a block
                           power iteration for Sigma~(1,1) (8 steps, block 8: about 1% low on a
                           clustered top spectrum; it only scales the stop tolerance)           */
  int gram_split;       /* 1 (default): run the Gram products on the tensor cores by an exact split
                           of A, W and A W into bf16 digits (rlobpcg_gram_split; about FP64
                           accuracy). Real FP64 with b <= 24 and complex128 with b <= 12
                           (rlobpcg_gram_split_c128) only (ignored otherwise); A is split once per
                           solve into about 16 bytes of device memory per real number of A.
                           0: the FP64 CUDA-core Gram pass (rlobpcg_gram).                    */
  double tau;           /* tolerance of ||R(:,j)|| <= Sigma~(1,1)^2 tau; < 0 means 2 sqrt(n) 2^-52 */
  int orth_mode;        /* orthonormalisation of W after its two block Gram-Schmidt passes against
                           [V X]: RLOBPCG_ORTH_HOUSEHOLDER (default, Orth of Alg. 2) or
                           RLOBPCG_ORTH_SVQB (Stathopoulos & Wu's SVQB, the faster, less stable
                           alternative Sec. 2.1 names)                                          */
  int locking;          /* 1: deflate converged columns (Sec. 2.3): a column whose residual meets the
                           tolerance is locked -- kept in V with its value frozen -- while X and W
                           lose its column and W stays orthogonal to all of V, so Rayleigh-Ritz
                           runs on the active columns; the solve also ends when all are locked.
                           The host reads the residual norms after every iteration to decide (one
                           stream synchronisation per iteration instead of per stop check).      */
  int precond;          /* P of W = P (P^* R): RLOBPCG_PRECOND_SKETCH (default; Alg. 2,
                           P P^* = (R^H R)^{-1} from the sketch), RLOBPCG_PRECOND_DIAG
                           (P = diag(||A(:,i)||^{-1}), the diagonally preconditioned LOBPCG of
                           Sec. 1.1; one more pass over A for the column norms) or
                           RLOBPCG_PRECOND_NONE (P = I, LOBPCG without a preconditioner). Every
                           variant starts from the sketch-and-solve block and stops by the rule
                           of Sec. 2.1, as the comparison of Sec. 1.1 does.                      */
} rlobpcg_opts;

#define RLOBPCG_PRECOND_SKETCH 0
#define RLOBPCG_PRECOND_DIAG 1
#define RLOBPCG_PRECOND_NONE 2

#define RLOBPCG_ORTH_HOUSEHOLDER 0
#define RLOBPCG_ORTH_SVQB 1

/* Per-solve report. */
typedef struct {
  int iters;            /* LOBPCG iterations run                                                   */
  int matvecs;          /* columns multiplied by A (b per iteration plus the start block)           */
  int stop_reason;      /* RLOBPCG_STOP_*                                                           */
  int block;            /* block size b used                                                       */
  double sigma11;       /* Sigma~(1,1), the sketch's estimate of ||A|| used by the stop rule         */
  double ms_sketch;     /* device time of the sketch                                               */
  double ms_factor;     /* QR of SA, SVD of R, R^{-1}, start block                                 */
  double ms_iterate;    /* LOBPCG iterations                                                       */
  double ms_total;      /* whole solve, including host<->device copies done by the call            */
  double ms_gram;       /* device time of the fused Gram passes (CUDA events on the plan's stream)  */
  int gram_passes;      /* number of Gram passes in ms_gram                                         */
  int kernel_launches;  /* CUDA kernels this solve launched                                         */
  int jacobi_sweeps;    /* sweeps of the one-sided Jacobi SVD of R                                  */
  double ms_gram_ab;    /* split Gram plans: device time of the A W kernels (W split + first product) */
  double ms_gram_atb;   /* split Gram plans: device time of the A^T (A W) kernels (+ partial sums)     */
  double ms_split_a;    /* split Gram plans: device time of splitting A into digits (once per solve)   */
  int rr_sweeps;        /* Jacobi sweeps of all Rayleigh-Ritz SVDs of the solve (R_T and the start) */
  int rr_calls;         /* number of those SVDs                                                      */
} rlobpcg_info;

typedef struct rlobpcg_plan_s* rlobpcg_plan_t;

/* Fill *opts with the defaults described above. Returns RLOBPCG_OK, or INVALID_ARG for NULL. */
int rlobpcg_default_opts(rlobpcg_opts* opts);

/*
 * Create a plan for solves of m x n matrices (dtype RLOBPCG_F64 or RLOBPCG_C128) asking for the
 * k smallest singular triplets. Allocates all device workspace the solve needs (its size grows
 * as (m + n) * 3b plus d * n and n * n elements), so solve() itself allocates nothing unless it
 * is given host pointers. The workspace is stream-ordered (cudaMallocAsync on `stream`, from the
 * device's default memory pool), so creating a plan does not synchronise the device.
 * `stream` is a cudaStream_t (NULL = default stream). A plan on the tensor-core Gram path
 * (gram_split) also creates a second, non-blocking stream of its own. Each iteration runs its
 * TSQR merges and Rayleigh-Ritz SVD there, beside the second Gram product. That work starts after
 * an event recorded on `stream`, and `stream` waits for its end before the iteration goes on, so
 * to the caller the solve stays ordered on `stream`.
 * Errors: INVALID_ARG when k < 1, b < k, 3b > n, n > m, d < n, d < zeta or zeta < 1;
 * OOM when the workspace does not fit; CUDA for runtime failures.
 */
int rlobpcg_plan(rlobpcg_plan_t* out, int64_t m, int64_t n, int k, int dtype,
                 const rlobpcg_opts* opts, void* stream);

/*
 * Solve (Algorithm 2): sketch, factorise, start block, LOBPCG iterations, outputs.
 *   A      m x n, leading dimension lda >= n, host or device memory, not modified. Host memory is
 *          copied to a plan-owned device buffer first (allocated on first use).
 *   tol    tolerance tau of the sketched stopping rule (Sec. 2.1); tol < 0 keeps the plan's.
 *   sigma  k doubles, ascending: the k smallest singular value estimates.
 *   V      n x k (row-major, leading dimension k) right singular vectors in the dtype of A,
 *          column j belonging to sigma[j].
 *   U      m x k (row-major, leading dimension k) left vectors A V diag(sigma)^{-1}, or NULL.
 *          Entries are Inf/NaN-free only when sigma[j] > 0; a sigma at rounding level gives a
 *          meaningless column.
 *   resid  k doubles: ||A^H A v_j - sigma_j^2 v_j||, or NULL.
 *   info   per-solve report, or NULL.
 * sigma, V, U and resid may each be host or device memory. Returns OK, NOT_CONVERGED (outputs
 * valid), or an error (outputs undefined).
 */
int rlobpcg_solve(rlobpcg_plan_t plan, const void* A, int64_t lda, double tol, double* sigma,
                  void* V, void* U, double* resid, rlobpcg_info* info);

/* Release a plan and its device workspace. NULL is accepted. */
/* Asynchronous form of rlobpcg_solve (same arguments and results). It returns at once: 0 once the
 * solve has started, INVALID_ARG (bad arguments, or a solve of this plan already in flight) or OOM
 * without starting one. The solve -- its work on the plan's stream and the stopping rule that the
 * host evaluates between iterations -- runs on a host thread of the library with the caller's
 * current device, so the calling thread is free meanwhile. A, the outputs and info must stay valid,
 * and the plan must not be used (solve, history, batch), until rlobpcg_solve_wait returns.
 * rlobpcg_plan_destroy waits for a solve still in flight. */
int rlobpcg_solve_async(rlobpcg_plan_t plan, const void* A, int64_t lda, double tol, double* sigma, void* V,
                        void* U, double* resid, rlobpcg_info* info);

/* Waits for the plan's asynchronous solve; returns what rlobpcg_solve would have returned, with its
 * message in rlobpcg_last_error() on the calling thread. INVALID_ARG when no solve is in flight. */
int rlobpcg_solve_wait(rlobpcg_plan_t plan);

int rlobpcg_plan_destroy(rlobpcg_plan_t plan);

/* Per-iteration history of the plan's last solve (host memory, row-major, b columns, b = the block
 * size, returned in *block): row 0 holds the Ritz values of the start block's Rayleigh-Ritz step
 * and its residual norms, row t >= 1 those after iteration t; within a row, the b smallest Ritz
 * values in descending order (the last is the smallest) and their residual column norms
 * ||A^H A v_j - theta_j^2 v_j|| -- the quantities the stopping rule of Sec. 2.1 reads. *rows
 * receives iterations + 1; at most cap_rows rows are copied into theta and resnorm (either may be
 * NULL). Errors: INVALID_ARG (NULL plan or rows, cap_rows < 0). */
int rlobpcg_history(rlobpcg_plan_t plan, double* theta, double* resnorm, int cap_rows, int* rows, int* block);

/* Device bytes a plan owns (its workspace; a host-A copy made by solve() is not included). */
size_t rlobpcg_plan_device_bytes(rlobpcg_plan_t plan);

/* Device bytes rlobpcg_plan would allocate for these arguments (0 if they are invalid), without
 * allocating anything: what an admission controller charges a solve before it starts. */
size_t rlobpcg_plan_workspace_size(int64_t m, int64_t n, int k, int dtype, const rlobpcg_opts* opts);

/* ---- serving: continuous batching under an HBM budget ------------------------------------ */
/*
 * A server owns `max_active` worker slots on `device`, each with its own CUDA stream. Requests
 * join a FIFO queue; the head is admitted when a slot is free and its device footprint (the plan
 * workspace of rlobpcg_plan_workspace_size plus a device copy of A) fits in what
 * `hbm_budget_bytes` has left. Admitted solves run concurrently on the GPU (their kernels
 * overlap); each keeps its LOBPCG state in device memory between iterations and releases it when
 * it finishes, which admits the next request. Results are those of rlobpcg_solve on the same
 * input (the kernels are deterministic), whatever else is running.
 * The north star of this library asks for this serving mode; the paper has no counterpart.
 */
typedef struct rlobpcg_server_s* rlobpcg_server_t;

/* Creates the max_active worker streams up front; a server is created with all its slots or not
 * at all. Errors: INVALID_ARG (bad budget, max_active outside 1..64, bad device), CUDA (a
 * stream could not be created; nothing is left behind). */
int rlobpcg_server_create(rlobpcg_server_t* out, size_t hbm_budget_bytes, int max_active, int device);

/* Serving modes of rlobpcg_server_create_ex (rlobpcg_server_create is RLOBPCG_SERVE_STREAMS). */
#define RLOBPCG_SERVE_STREAMS 0   /* each admitted solve runs whole on its worker's stream           */
#define RLOBPCG_SERVE_BATCHED 1   /* set-up and outputs per worker; the iterations of every admitted
                                     solve the batched kernels take (see rlobpcg_solve_batch) run
                                     together in one batch engine, solves joining and leaving
                                     between graph replays; other requests run whole             */

/* As rlobpcg_server_create, with a serving mode; max_active may be up to 256 in batched mode
 * (the number of solves iterating together). A batched request's footprint adds the batched
 * iterations' buffers. Each result equals that of rlobpcg_solve (streams mode) or of
 * rlobpcg_solve_batch with that request alone (batched mode), whatever else runs. */
int rlobpcg_server_create_ex(rlobpcg_server_t* out, size_t hbm_budget_bytes, int max_active, int device, int mode);

/* Batched mode: the largest m n b (rows x columns x block) a request may have to iterate in the
 * batch engine; larger requests run whole on their worker, where the Gram products of FP64 and
 * complex128 solves run on the tensor cores (gram_split). Applies to requests submitted afterwards.
 * Default RLOBPCG_SERVE_BATCH_LIMIT_DEFAULT. INVALID_ARG for a negative limit. */
#define RLOBPCG_SERVE_BATCH_LIMIT_DEFAULT ((int64_t)1 << 23)
int rlobpcg_server_set_batch_limit(rlobpcg_server_t s, int64_t max_mnb);

/* Counters of a batched server's engine since creation (all zero in streams mode). */
typedef struct {
  int64_t replays;      /* graph replays (4 iterations of every joined solve each)               */
  int64_t joins;        /* solves that joined the batch                                           */
  int64_t retires;      /* solves handed back                                                     */
  int64_t rebuilds;     /* work-list + graph rebuilds (membership changes)                        */
  double gpu_ms;        /* device time inside replays (CUDA events on the engine stream)          */
  double host_ms;       /* engine thread time outside replays (joins, retires, rebuilds, waits)   */
  double active_mean;   /* solves per replay, averaged over replays                               */
} rlobpcg_engine_stats;
int rlobpcg_server_engine_stats(rlobpcg_server_t s, rlobpcg_engine_stats* out);

/* Queue a solve of the k smallest singular triplets of A (HOST memory, m x n row-major, lda >= n,
 * F64 or C128; it must stay valid until rlobpcg_server_wait returns for this ticket).
 * opts may be NULL (defaults). Errors: INVALID_ARG, OOM when the request alone exceeds the
 * budget (it could never be admitted). */
int rlobpcg_server_submit(rlobpcg_server_t s, const void* A, int64_t m, int64_t n, int64_t lda, int k, int dtype,
                          const rlobpcg_opts* opts, int64_t* ticket);

/* 0 queued, 1 running, 2 done; INVALID_ARG for an unknown ticket. */
int rlobpcg_server_poll(rlobpcg_server_t s, int64_t ticket);

/* Block until the request is done and copy its results to HOST buffers (sigma k, V n x k
 * row-major in the dtype of A, resid k; each may be NULL). latency_ms: submit -> done.
 * Returns the solve's status (OK, NOT_CONVERGED, CANCELLED when the server was destroyed before
 * the request was admitted, or an error). The ticket is released. One thread waits per ticket:
 * a second wait on a ticket that already has a waiter returns INVALID_ARG at once. */
int rlobpcg_server_wait(rlobpcg_server_t s, int64_t ticket, double* sigma, void* V, double* resid,
                        rlobpcg_info* info, double* latency_ms);

/* Completed requests, their p50/p99 latency (submit -> done), completed / (last done - first
 * submit), the peak of admitted device bytes and of concurrently running solves. */
int rlobpcg_server_stats(rlobpcg_server_t s, int64_t* completed, double* p50_ms, double* p99_ms,
                         double* solves_per_s, size_t* peak_bytes, int* peak_running);

/* Stop the server: requests not yet admitted are cancelled (their waiters return
 * RLOBPCG_ERR_CANCELLED), running solves finish, and the call returns once every worker has
 * stopped and every thread inside rlobpcg_server_wait for this server has returned. No other call
 * on this server may start during or after it. */
int rlobpcg_server_destroy(rlobpcg_server_t s);

/*
 * Batched solves (an addition of this library for many small problems; the paper solves one at a
 * time). rlobpcg_solve_batch runs `count` solves, one per plan: plans[i] distinct, each created by
 * rlobpcg_plan for its own (m_i, n_i, k_i) with dtype RLOBPCG_F64, block b_i <= 5, n_i <= 512, and
 * neither locking, SVQB nor residual refresh (else RLOBPCG_ERR_UNSUPPORTED, nothing run). A[i] is
 * a DEVICE pointer to the m_i x n_i row-major matrix with leading dimension lda[i] >= n_i.
 *
 * Each solve's set-up -- sketch, factor, start block and first Rayleigh-Ritz step (Alg. 2) -- runs
 * on its plan's stream (set-ups of different plans overlap, on up to 8 host threads). The LOBPCG
 * iterations of all solves then run together on a stream of the library's own: per iteration two
 * persistent kernels over a device work queue of (solve, row block) items, (1) W = P P^* R with
 * the preconditioner formed once per solve as the n x n matrix (R^H R)^{-1}, then BCGS2 + Orth of
 * W, and (2) the Gram products A W and A^H (A W) by row tiles, each tile also reducing its rows of
 * A_T to a triangular factor, the factors and G partials merged in a fixed two-level order, and
 * Rayleigh-Ritz, the update, the residual and the stopping rule of Sec. 2.1 for a solve in the same
 * launch, by the CTA that finishes its last tile. Four iterations are replayed as one captured
 * CUDA graph; a solve that has stopped takes no further part. Outputs, per solve, as rlobpcg_solve:
 * sigma[i] (k_i, ascending), V[i] (n_i x k_i), U[i] (m_i x k_i; U or U[i] may be NULL), resid[i]
 * (may be NULL); infos and status (count entries each) may be NULL. Host or device output
 * pointers are accepted as in rlobpcg_solve. The stopping decisions are the device's.
 *
 * A solve's arithmetic depends only on its own data and on the tile shape of its (n, b) class
 * (rlobpcg_batch_tile), so it gives the same bits alone and in any batch of one process.
 * Synchronous: returns once every output is written. Returns the first negative per-solve status,
 * else RLOBPCG_OK (RLOBPCG_NOT_CONVERGED is reported per solve in status).
 */
int rlobpcg_solve_batch(int count, rlobpcg_plan_t* plans, const void* const* A, const int64_t* lda,
                        double* const* sigma, void* const* V, void* const* U, double* const* resid,
                        rlobpcg_info* infos, int* status, void* stream);

/* The tile shape the batched kernels use for solves of n columns and block b (n <= 512, b <= 5):
 * trows rows of A per work item and rt rows per shared-memory stage. The class is (the power of
 * two >= max(n, 32), b). On first use of a class the library's autotuner times every shape that
 * fits shared memory on synthetic solves of the class (on `stream`) and keeps the fastest; the
 * choice then stays fixed for the process. */
int rlobpcg_batch_tile(int64_t n, int b, int* trows, int* rt, void* stream);

/* Pin the tile shape of the (n, b) class (one of the candidates the autotuner considers:
 * trows in {256, 512, 1024, 2048}, rt in {8, 16}, within shared memory), e.g. to reproduce
 * results across processes. INVALID_ARG for a shape outside the candidates. */
int rlobpcg_batch_set_tile(int64_t n, int b, int trows, int rt);

/*
 * Health check of the bounded-wait path (an addition of this library; the paper has no
 * counterpart). Every device-side wait of the library gives up after a bounded number of tries,
 * records the timeout, releases what its kernel holds and returns, so that a lost arrival surfaces
 * as RLOBPCG_ERR_TIMEOUT instead of a hung GPU. This call runs a kernel that holds TMEM and waits,
 * at most `spins` tries (1 .. 2^24), on an mbarrier nothing arrives at (kind 0) or on a global
 * flag nothing sets (kind 1). Returns RLOBPCG_ERR_TIMEOUT when the path works (the kernel gave up,
 * released its TMEM and exited; the stream stays usable), INVALID_ARG for a bad kind or spins,
 * CUDA for a runtime failure. Synchronous on `stream`.
 */
int rlobpcg_check_bounded_wait(int kind, int spins, void* stream);

/* Static string naming a status code. */
const char* rlobpcg_status_string(int status);

/* Detail of the most recent error in this thread (static storage, overwritten by the next one). */
const char* rlobpcg_last_error(void);

/* ---- single steps of the path, for callers that compose their own loop (and for tests) ---- */

/*
 * Sketch SA = S A with the SparseStack S of Sec. 2.2 (d rows, zeta nonzeros per column, seeded
 * SplitMix64: entry (row i, piece j) uses output number i*zeta + j; position inside piece j =
 * floor((h >> 32) * len_j / 2^32) with piece j = rows [floor(j d/zeta), floor((j+1) d/zeta));
 * sign -1 when bit 0 of h is set; values +-zeta^{-1/2}). Each output entry is summed over its
 * source rows in ascending order and scaled once at the end, so results are reproducible bit
 * for bit.
 *   A   device, m x n row-major (lda), dtype F64 or C128.
 *   SA  device, d x n COLUMN-major (element (r, j) at SA[j*d + r]); float/complex64 when
 *       sketch_prec is RLOBPCG_SKETCH_F32, double/complex128 otherwise (F32_REFINE keeps the
 *       sketch in FP64).
 * Allocates nothing. Errors: INVALID_ARG (d < zeta, zeta < 1, lda < n, NULL pointers).
 */
int rlobpcg_sketch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int d, int zeta,
                   uint64_t seed, int sketch_prec, void* SA, void* stream);

/*
 * Factorise the sketch (the factorisation step of Alg. 2): Householder QR SA = QR (Q discarded),
 * the SVD R = U~ Sigma~ V~^H by one-sided Jacobi, and R^{-1}. Since SVD(SA) = SVD(R), Sigma~ and
 * V~ are those of SA, and P P^* = V~ Sigma~^{-2} V~^H = (R^H R)^{-1}. With
 * RLOBPCG_SKETCH_F32_REFINE, SA is FP64, the QR runs in FP32 and R is corrected once in FP64 (see
 * the precision constants); R, sigma, V~ and R^{-1} are then FP64.
 *   SA     device, d x n column-major in the sketch precision (overwritten by the QR).
 *   R      device, n x n column-major upper triangular (strict lower part zero), or NULL.
 *   sigma  device, n doubles, Sigma~ descending.
 *   Vt     device, n x n column-major V~ (column j belongs to sigma[j]) in the sketch precision.
 *   Rinv   device, n x n row-major R^{-1} in the sketch precision, or NULL.
 *   work   device scratch of rlobpcg_factor_workspace_size(d, n, dtype, sketch_prec) bytes.
 * Errors: INVALID_ARG (d < n), TIMEOUT (a bounded wait between the QR's CTAs ran out: not seen
 * in normal runs), CUDA.
 */
int rlobpcg_factor(void* SA, int64_t d, int64_t n, int dtype, int sketch_prec, void* R,
                   double* sigma, void* Vt, void* Rinv, void* work, size_t work_bytes,
                   void* stream);
size_t rlobpcg_factor_workspace_size(int64_t d, int64_t n, int dtype, int sketch_prec);

/*
 * Fused Gram pass (the product of Alg. 2 with the trial block): one read of A gives
 *   AW = A W      (m x b, row-major, leading dimension ldaw)
 *   G  = A^H AW   (n x b, row-major, leading dimension ldg)
 * W is n x b row-major (ldw). All device memory, dtype F64 or C128. Rows of A are split over
 * the SMs and the per-SM partial G's are summed in a fixed order (results are deterministic).
 *   work  device scratch of rlobpcg_gram_workspace_size(m, n, b, dtype) bytes.
 * Errors: INVALID_ARG (b < 1, b > 64, leading dimensions too small), UNSUPPORTED (n * b too large
 * for on-chip accumulation), CUDA.
 */
int rlobpcg_gram(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b,
                 int64_t ldw, void* AW, int64_t ldaw, void* G, int64_t ldg, void* work,
                 size_t work_bytes, void* stream);
size_t rlobpcg_gram_workspace_size(int64_t m, int64_t n, int b, int dtype);

/*
 * Allocation-free variant of rlobpcg_gram (the paper has no counterpart; it is an addition of
 * this library). Same arguments, results and errors as rlobpcg_gram, minus the workspace: the
 * split-m scratch is a fixed 16 MiB device buffer inside the library (plus 256 bytes for the
 * error word), held on every GPU that loads the library until the process exits.
 * For callers that cannot let a library allocate device memory: a serving process that has
 * budgeted all of HBM at start-up, or a loop that must avoid cudaMalloc/cudaFree because they
 * synchronise the whole device. This call makes no allocation of any kind.
 *   - The call is synchronous: it reads the device error word back and synchronises `stream`
 *     before it returns.
 *   - The first call on a device looks up the buffer's device address (once per device, with
 *     that device current).
 *   - All calls share the one buffer, which keeps the last call's contents: calls that overlap
 *     on the GPU (other streams, other threads) race and must be serialised by the caller.
 *   - Problems whose partials need more than 16 MiB (about 152 * n * b * 8 bytes for real A,
 *     twice that for complex) are rejected with RLOBPCG_ERR_UNSUPPORTED and a message in
 *     rlobpcg_last_error(); use rlobpcg_gram for those.
 */
int rlobpcg_gram_noalloc(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b,
                         int64_t ldw, void* AW, int64_t ldaw, void* G, int64_t ldg, void* stream);

/*
 * Split-bf16 Gram pass on the tensor cores (real FP64). The paper forms these products in FP64;
 * this is an addition of this library with the same results up to FP64-level rounding: the same
 * AW = A W (m x b) and G = A^T AW (n x b) as rlobpcg_gram, with every operand split exactly into
 * eight signed 7-bit digits (exact in bf16) under a power-of-two scale per group -- a row of A for
 * A W, a column of A within each 128-row chunk for A^T AW, a column of W, a column of AW within
 * each chunk (the Ozaki scheme). Digit products accumulate exactly (as integers below 2^24) in the
 * tensor cores' f32 accumulators and are recombined in FP64; the 43 digit pairs of levels
 * p + q <= 8 are formed (the others weigh below 2^-60 of the leading term). Per product term the
 * error is about 2^-55 times the product of the two group maxima.
 *   rlobpcg_gram_split_prepare: split A (m x n, row-major, lda) once -- it is constant through a
 *     solve -- into prep, rlobpcg_gram_split_prepare_size(m, n) bytes of device memory (about 16
 *     bytes per element of A: one byte per digit, in the layouts of both products). Errors as
 *     below; NONFINITE when A holds Inf or NaN.
 *   rlobpcg_gram_split: one pass; W (n x b, ldw), AW (m x b, ldaw), G (n x b, ldg) row-major,
 *     1 <= b <= 24; work: rlobpcg_gram_split_workspace_size(m, n, b) bytes of device scratch.
 * All pointers are device memory owned by the caller; calls are asynchronous on `stream` and
 * synchronise it before returning. prep also holds a few counters that each pass uses and leaves
 * at zero, so passes on one prep must not overlap. Errors: INVALID_ARG (sizes, NULL, buffers too small),
 * UNSUPPORTED (n above 1,048,560), NONFINITE (W holds Inf or NaN), TIMEOUT (a bounded device wait
 * ran out), CUDA.
 */
size_t rlobpcg_gram_split_prepare_size(int64_t m, int64_t n);
int rlobpcg_gram_split_prepare(const double* A, int64_t m, int64_t n, int64_t lda, void* prep, size_t prep_bytes,
                               void* stream);
size_t rlobpcg_gram_split_workspace_size(int64_t m, int64_t n, int b);
int rlobpcg_gram_split(const void* prep, int64_t m, int64_t n, const double* W, int b, int64_t ldw, double* AW,
                       int64_t ldaw, double* G, int64_t ldg, void* work, size_t work_bytes, void* stream);

/*
 * The same pass for complex128 A (the Gram pass of Alg. 2: AW = A W, G = A^H AW). A complex m x n
 * row-major matrix read as doubles is the real m x 2n row-major matrix B (leading dimension
 * 2 lda; B(i, 2j) = Re A(i, j), B(i, 2j+1) = Im A(i, j)), so
 *   prep: rlobpcg_gram_split_prepare((const double*)A, m, 2 n, 2 lda, ...) -- the split of B,
 *         rlobpcg_gram_split_prepare_size(m, 2 n) bytes;
 *   rlobpcg_gram_split_c128: one pass; W (n x b), AW (m x b), G (n x b), complex128 row-major with
 *         leading dimensions ldw, ldaw, ldg (in complex elements), 1 <= b <= 12; work:
 *         rlobpcg_gram_split_c128_workspace_size(m, n, b) bytes of device scratch (0 when b > 12).
 * Each complex entry w of W becomes the real 2 x 2 block [Re w, Im w; -Im w, Re w] of a 2n x 2b
 * real W', so that B W' is A W in its interleaved storage; the real pass forms B W' and
 * B^T (B W'), and G = A^H AW is combined from the four real products of B^T (B W') in FP64
 * (Re G = Re A^T Re Z + Im A^T Im Z, Im G = Re A^T Im Z - Im A^T Re Z for Z = A W). Error per
 * term as for the real pass, plus one FP64 rounding per entry of G. Pointers, synchronisation and
 * errors as for rlobpcg_gram_split.
 */
size_t rlobpcg_gram_split_c128_workspace_size(int64_t m, int64_t n, int b);
int rlobpcg_gram_split_c128(const void* prep, int64_t m, int64_t n, const void* W, int b, int64_t ldw, void* AW,
                            int64_t ldaw, void* G, int64_t ldg, void* work, size_t work_bytes, void* stream);

/*
 * R factor of a tall block (the TSQR used for Rayleigh-Ritz by SVD of A_T, Alg. 2): X is m x c
 * row-major (ldx), c <= 64; R (c x c, row-major, upper triangular, diag(R) real >= 0) is written
 * to device memory. Householder reflections per row block, then a fixed-order tree of stacked
 * R factors.  work: rlobpcg_tsqr_workspace_size(m, c, dtype) bytes of device scratch.
 */
int rlobpcg_tsqr(const void* X, int64_t m, int c, int64_t ldx, int dtype, void* R, void* work,
                 size_t work_bytes, void* stream);
size_t rlobpcg_tsqr_workspace_size(int64_t m, int c, int dtype);

#ifdef __cplusplus
}
#endif
#endif /* RLOBPCG_H */
