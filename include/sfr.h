/*
 * libsfr — sparse fixed-rank decomposition M = L + S, rank(L) = r, on one GB300 GPU.
 *
 * The library solves the S-FR problem of Ros et al., "Fast and Robust Fixed-Rank
 * Matrix Recovery" (Eq. 1 / Eq. 3): min ||S||_1 s.t. M = L + S, L on the rank-r
 * manifold, by FR-ADM (Algorithm 1), an augmented-Lagrangian iteration (Eq. 4)
 * whose L-step is one FixedRankOptStep (Algorithm 3) in polar form L = U B V^T
 * (U, V Stiefel, B symmetric, Sec. 4.1), and its Nystrom variant FR-Nys
 * (Algorithm 2).
 *
 * Conventions for every entry point:
 *   - All matrices are row-major.  M is m x n with leading dimension ldm >= n
 *     (in elements).  U is m x r, V is n x r, B is r x r, all float64 and dense
 *     (leading dimension r).  S is m x n with leading dimension lds >= n.
 *   - `mem` says where the caller's M, nys_perm, U, B, V and S live:
 *     SFR_MEM_DEVICE (pointers into the context's GPU) or SFR_MEM_HOST
 *     (ordinary or pinned host memory; the library copies in and out).
 *   - The caller owns M and every result buffer; they must stay valid until
 *     the call (sfr_solve) or the request (sfr_submit ... sfr_poll) finishes.
 *     The library owns its workspace (multiplier Y, thin products, r x r
 *     scratch) and frees it in sfr_destroy.
 *   - Functions return an sfr_status and never abort.  A status < 0 is an
 *     error; sfr_last_error(ctx) then holds a one-line message.  A per-problem
 *     outcome is also stored in sfr_result.status.
 *   - A context is not thread-safe: use one context per host thread.
 *   - Launch shapes: the first mixed-precision solve of a size class (m and n by
 *     powers of two, padded rank, dtype of M) times a few grid sizes of the
 *     float32 sweep (r <= 32) before it starts and keeps the fastest for the rest
 *     of the process, so every later solve of that class, in any context or
 *     serving slot, runs the same kernels and gives bit-identical results.
 *     Environment: SFR_AUTOTUNE=0 skips the timing (a fixed default grid);
 *     SFR_TUNE_FILE=path loads the choices from, and saves them to, a JSON file.
 */
#ifndef SFR_H
#define SFR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFR_OK = 0,
  SFR_PENDING = 1,      /* sfr_poll: the request is still running                      */
  SFR_E_INVAL = -1,     /* bad argument (sizes, rank, dtype, null pointer, rho <= 1 ...) */
  SFR_E_NOMEM = -2,     /* device allocation failed or the HBM budget is exceeded        */
  SFR_E_CUDA = -3,      /* a CUDA runtime call failed                                     */
  SFR_E_RANK = -4,      /* P_O met an m x r (or n x r) matrix of rank < r (Eq. 9 assumes full rank) */
  SFR_E_NOCONV = -5,    /* max_iter iterations without reaching tol                       */
  SFR_E_NAN = -6,       /* a non-finite value appeared in the iteration                   */
  SFR_E_TIMEOUT = -7,   /* sfr_poll: timeout elapsed                                      */
  SFR_E_BUSY = -8       /* the request queue is full                                      */
} sfr_status;

typedef enum { SFR_F64 = 0, SFR_F32 = 1, SFR_BF16 = 2 } sfr_dtype;

/* Arithmetic of the m x n sweep.  The r x r projectors and the convergence
 * test are float64 in both modes.
 *   SFR_PREC_FP64:  float64 everywhere (M may be stored f64, f32 or bf16).
 *   SFR_PREC_MIXED: float32 sweep arithmetic and multiplier storage, float64
 *                   factors and r x r steps. */
typedef enum { SFR_PREC_FP64 = 0, SFR_PREC_MIXED = 1 } sfr_precision;

typedef enum { SFR_MEM_DEVICE = 0, SFR_MEM_HOST = 1 } sfr_memspace;

/* Bits of sfr_result.path: which kernels a solve ran. */
typedef enum {
  SFR_PATH_TC = 1           /* the m x n sweep and W pass ran on the tensor cores (tcgen05, TMA):
                               mixed precision with bfloat16 M, 33 <= r <= 64, n and ldm multiples
                               of 8 and a 16-byte aligned M; clear = the SIMT passes            */
} sfr_path_flag;

typedef struct sfr_ctx sfr_ctx;

typedef struct {
  int device;               /* CUDA device ordinal                                         */
  size_t hbm_budget_bytes;  /* cap on workspace bytes the context may hold; 0 = no cap     */
  int max_slots;            /* concurrent requests for sfr_submit; 0 = default (8)         */
  void* cuda_stream;        /* cudaStream_t for sfr_solve; NULL = a stream the ctx creates */
  int profile;              /* 1: time the sweep (or P pass), W-pass and r x r kernels of
                               sfr_solve / sfr_fixed_rank_opt_full with CUDA events on the
                               solve stream (see sfr_stats); 2: time the sweep (or P pass) only,
                               in the first iteration and every fourth after it (an event
                               record splits the iteration's launch chain); 0: no timing  */
  int max_batch;            /* > 0: sfr_submit runs requests on the mixed-precision SIMT path
                               (FR-ADM, device buffers, r <= 32) in a grouped engine with up to
                               this many live problems: every step advances each of them by one
                               iteration with one grouped launch per kernel; results equal
                               sfr_solve's.  Other requests go to the slots.  0: slots only  */
} sfr_config;

/* Kernel classes counted by sfr_stats. */
typedef enum {
  SFR_STAT_SWEEP = 0,       /* fused sweep: L rebuild, S- and Y-steps of Algorithm 1, Delta, next X V */
  SFR_STAT_WPASS = 1,       /* X^T U_bar pass (V-step product of Algorithm 3)                      */
  SFR_STAT_RXR = 2,         /* r x r projector kernels (Eq. 9, Eq. 10)                           */
  SFR_STAT_ALL = 3,         /* every kernel launch of the library (total_ms unused)              */
  SFR_STAT_PPASS = 4,       /* M V pass of sfr_fixed_rank_opt_full (U-step product, Algorithm 4)  */
  SFR_STAT_COUNT = 5
} sfr_stat_kind;

typedef struct {
  int64_t launches;         /* kernel launches (including launches that found the stop flag set) */
  int64_t timed;            /* launches that did work and were timed (profile != 0)              */
  double total_ms;          /* summed event-to-event duration of the timed launches              */
  double bytes;             /* algorithmic DRAM bytes of the timed launches: the m x n operands
                               each must read or write once, given their storage types           */
} sfr_kernel_stat;

typedef struct {
  int64_t m, n, ldm;        /* M is m x n, row-major, leading dimension ldm >= n           */
  int32_t r;                /* target rank, 1 <= r <= min(m, n) and r <= 64                */
  sfr_dtype m_dtype;        /* storage type of M                                           */
  const void* M;            /* the data matrix (read only)                                 */
  double mu0;               /* initial penalty mu_1 (Algorithm 1 uses 1); > 0              */
  double rho;               /* continuation factor, > 1 (Algorithm 1 leaves it open)       */
  double mu_max;            /* penalty cap mu_bar (Algorithm 1 uses 1e9)                   */
  double tol;               /* stop when ||M - L - S||_F / ||M||_F <= tol                  */
  int32_t max_iter;         /* give up (SFR_E_NOCONV) after this many iterations           */
  int32_t fixed_iters;      /* > 0: run exactly this many iterations, ignore tol           */
  sfr_precision precision;
  sfr_memspace mem;         /* where M, nys_perm and the result buffers live               */
  int32_t nys_l;            /* 0: FR-ADM.  > 0: FR-Nys with an m x l column block and an
                               l x n row block (Algorithm 2), r <= l <= min(m, n)          */
  const int64_t* nys_perm;  /* FR-Nys only: row shuffle, shuffled row i = input row perm[i] */
} sfr_problem;

typedef struct {
  double* U;                /* m x r, orthonormal columns; NULL = do not return            */
  double* B;                /* r x r, symmetric (FR-Nys: diagonal, see below)              */
  double* V;                /* n x r, orthonormal columns.  L = U B V^T.  FR-Nys returns its
                               L = U_L Core V_T^T (Algorithm 2, r x r core) in this form through
                               the SVD Core = A diag(sigma) C^T: U = U_L A (rows in M's order),
                               B = diag(sigma) (decreasing), V = V_T C                      */
  void* S;                  /* m x n sparse part; NULL = do not write S                    */
  sfr_dtype s_dtype;        /* SFR_F64 or SFR_F32                                          */
  int64_t lds;              /* leading dimension of S, >= n                                */
  void* L;                  /* optional m x n low-rank part (same dtype/ld as S); NULL = skip */
  int32_t iters;            /* iterations run (FR-Nys: sum over the two block solves, which
                               run concurrently on two streams)                            */
  double rel_residual;      /* ||M - L - S||_F / ||M||_F after the last iteration          */
  double lambda_min_B;      /* smallest eigenvalue of the returned B (SPD diagnostic)      */
  sfr_status status;        /* outcome of this problem                                     */
  int32_t path;             /* sfr_path_flag bits of the kernels this solve ran (FR-Nys: of
                               either block solve)                                           */
} sfr_result;

/* FixedRankOptFull (Algorithm 4, Appendix): FixedRankOptStep (Algorithm 3)
 * iterated on a fixed M, i.e. alternating minimisation of ||M - U B V^T||_F over
 * U in St(m, r), B symmetric, V in St(n, r).  Each iteration computes
 *     U = P_O[M V B],  V = P_O[M^T U B],  B = Sym(U^T M V)      (Eq. 9, Eq. 10),
 * and by Theorem 2 the iterates converge Q-linearly (subspace error shrinking by
 * (sigma_{r+1} / sigma_r)^2 per iteration) to factors of the rank-r truncated SVD
 * of M, whenever rank(M V_0) = r: a TSVD replacement on the same kernels as FR-ADM. */
typedef struct {
  int64_t m, n, ldm;        /* M is m x n, row-major, leading dimension ldm >= n           */
  int32_t r;                /* target rank, 1 <= r <= min(m, n) and r <= 64                */
  sfr_dtype m_dtype;        /* storage type of M                                           */
  const void* M;            /* the data matrix (read only)                                 */
  const double* V0;         /* n x r initial V (orthonormal columns); NULL = I_{n x r}     */
  const double* B0;         /* r x r initial B, symmetric and invertible (Algorithm 4 asks
                               for SPD; Lemma 1 needs only rank r); NULL = I_r.  A
                               nonsymmetric B0 is refused with SFR_E_INVAL               */
  double tol;               /* stop when ||B_i - B_{i-1}||_F <= tol ||B_i||_F (the paper's
                               "until converged" is unspecified); 0 = run exactly max_iter  */
  int32_t max_iter;         /* > 0; with tol > 0, SFR_E_NOCONV after this many iterations  */
  sfr_precision precision;  /* SFR_PREC_MIXED: float32 thin products (bfloat16 M on the
                               tensor cores when r > 32), float64 r x r steps             */
  sfr_memspace mem;         /* where M, V0, B0 and the result buffers live                 */
} sfr_opt_full_problem;

typedef struct {
  double* U;                /* m x r; NULL = do not return                                 */
  double* B;                /* r x r; NULL = do not return                                 */
  double* V;                /* n x r; NULL = do not return                                 */
  int32_t iters;            /* iterations run                                              */
  double rel_change;        /* ||B_K - B_{K-1}||_F / ||B_K||_F of the last iteration       */
  double lambda_min_B;      /* smallest eigenvalue of B_K (B is SPD near the optimum, Lemma 2);
                               NaN when B is not returned                                  */
  sfr_status status;        /* outcome (SFR_E_RANK if rank(M V_i B_i) < r, Eq. 9)          */
} sfr_opt_full_result;

/* Create a context on cfg->device.  *out receives the handle. */
sfr_status sfr_create(sfr_ctx** out, const sfr_config* cfg);

/* Solve one problem and wait for it (FR-ADM, Algorithm 1, or FR-Nys, Algorithm 2).
 * Returns the same status as res->status. */
sfr_status sfr_solve(sfr_ctx* ctx, const sfr_problem* prob, sfr_result* res);

/* Queue one problem; requests run concurrently on the device as slots and HBM
 * budget allow (continuous batching).  *ticket identifies it for sfr_poll.
 * The problem struct is copied; the buffers it points to are not. */
sfr_status sfr_submit(sfr_ctx* ctx, const sfr_problem* prob, sfr_result* res, uint64_t* ticket);

/* Wait up to timeout_us microseconds (< 0: forever, 0: just check) for a ticket.
 * Returns SFR_PENDING if still running, SFR_E_TIMEOUT is never returned for a
 * 0 timeout, otherwise the request's final status (res->status). */
sfr_status sfr_poll(sfr_ctx* ctx, uint64_t ticket, int64_t timeout_us);

/* Finish or cancel outstanding requests, free the workspace and the context. */
sfr_status sfr_destroy(sfr_ctx* ctx);

/* Run FixedRankOptFull (Algorithm 4) on one matrix and wait for it, on the
 * context's stream (the same stream and workspace as sfr_solve).  Returns the same
 * status as res->status; SFR_E_INVAL for bad sizes, dtypes or a null M. */
sfr_status sfr_fixed_rank_opt_full(sfr_ctx* ctx, const sfr_opt_full_problem* prob, sfr_opt_full_result* res);

/* Copy the per-kernel-class counters of sfr_solve and sfr_fixed_rank_opt_full calls
 * on ctx into out[0 .. count) (indexed by sfr_stat_kind); reset != 0 zeroes them
 * afterwards.  Counts do not cover requests run through sfr_submit. */
sfr_status sfr_stats(sfr_ctx* ctx, sfr_kernel_stat* out, int32_t count, int32_t reset);

/* sfr_solve without any device allocation, for callers that cannot allocate:
 * processes whose device memory belongs to a fixed pool or to a framework
 * allocator, and latency-critical paths that may not take the allocator's locks.
 * The paper has no counterpart; this is a library convenience.  It runs the same
 * FR-ADM kernels as sfr_solve (the SIMT passes, sfr_result.path = 0), eagerly on
 * the context's stream, with all workspace taken from one 32 MiB __device__ array
 * built into the library (every GPU that loads libsfr holds it until the process
 * exits).
 *   - FR-ADM only (nys_l == 0) and device buffers only (mem == SFR_MEM_DEVICE).
 *   - A problem whose workspace exceeds the array is refused with SFR_E_NOMEM.
 *     The workspace is about 24 bytes (float64 path) or 12 bytes (mixed path)
 *     per element of M plus the thin and r x r buffers; 500 x 500 at r = 25
 *     in float64 needs about 10 MiB.
 *   - Every call looks up the array's device address (a host query), so a
 *     cudaDeviceReset earlier in the process leaves no stale address behind.
 *   - All calls share the array and it keeps the previous call's contents (the
 *     solve clears what must start at zero).  Calls whose GPU work overlaps --
 *     from two host threads, or two contexts on one device -- race on it.
 * Same arguments and results as sfr_solve. */
sfr_status sfr_solve_noalloc(sfr_ctx* ctx, const sfr_problem* prob, sfr_result* res);

/* The last error message of ctx (or of the last failed sfr_create when ctx is NULL). */
const char* sfr_last_error(const sfr_ctx* ctx);

/* Library version string. */
const char* sfr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SFR_H */
