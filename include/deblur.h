/*
 * libdeblur -- B300 (sm_103a) implementation of the wavelet multilevel
 * V-cycle for l1-regularised deblurring, min ||A x - b||^2 + mu ||L x||_1
 * (Introduction, Eq. (l1b)), with IRLS, MM and Split Bregman outer solvers
 * (Sec. 2, Alg. 1-3), LSQR inner solves and GCV parameter choice (Sec. 3),
 * and Haar / 4-tap Daubechies transfers between levels (Sec. 4, Alg. 4).
 *
 * Conventions (all entry points):
 *  - Images are m x m, stored as vec(X) column-major: pixel (r, c) at
 *    X[r + c*m] (the paper vectorises column-wise, Sec. 5).
 *  - Gradient-domain vectors (L x, IRLS weights, MM shift, SB d and g) are two
 *    m x m planes, also column-major: plane x holds (D X)(r, c) for
 *    r < m-1 (row m-1 is padding, kept 0); plane y holds (X D^T)(r, c) for
 *    c < m-1 (column m-1 is padding, kept 0). D is the forward difference
 *    (Sec. 4.2: L = [I kron D; D kron I]).
 *  - A PSF is S x S (S odd), centred, column-major, psf[(p+R) + (q+R)*S] for
 *    row offset p and column offset q, R = (S-1)/2, acting as
 *    (A X)(r,c) = sum_{p,q} psf(p,q) X(r-p, c-q) with X = 0 outside the image
 *    (the zero-boundary banded Toeplitz blur of Sec. 5).
 *  - Pointers documented "device" must be device memory of the context's
 *    device; "host" pointers are ordinary host memory. The caller owns every
 *    buffer it passes; no call frees or retains caller memory.
 *  - Every call is asynchronous on `stream` unless stated otherwise; calls
 *    that return results to the host synchronise the stream first.
 *  - Errors: DB_EINVAL for bad sizes / enums / null pointers (nothing is
 *    launched), DB_ENOMEM when the context cannot allocate its workspace,
 *    DB_ECUDA for a CUDA runtime error (cudaGetLastError is cleared),
 *    DB_ETIMEOUT when a device-side wait (grid barrier) exceeded its time
 *    limit: the kernel then records the failure, returns, and the context
 *    remains usable.
 */
#ifndef DEBLUR_H
#define DEBLUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* db_stream;   /* a cudaStream_t; NULL = default stream */

typedef enum { DB_IRLS = 0, DB_MM = 1, DB_SB = 2 } db_solver;            /* Alg. 1, 2, 3 */
typedef enum { DB_HAAR = 0, DB_DB4 = 1 } db_wavelet;                     /* Sec. 4 filters */
typedef enum { DB_APPROACH_I = 0, DB_APPROACH_X = 1, DB_APPROACH_D = 2 } db_transfer; /* Sec. 4.1 */
typedef enum { DB_PREC_FP64 = 0, DB_PREC_FP32 = 1, DB_PREC_BF16 = 2 } db_precision;
typedef enum {
  DB_OK = 0, DB_EINVAL = 1, DB_ENOMEM = 2, DB_ECUDA = 3, DB_ETIMEOUT = 4,
  DB_EBUSY = 5, DB_ECANCELLED = 6
} db_status;

/* GCV options (Sec. 3). The paper evaluates the exact GCV functional through
 * the GSVD of the pair. This library does that on small levels (dense pair,
 * exact trace) and otherwise uses a projected form: the numerator is
 * projected onto span{K_k(A^T A, A^T b), D^T c} and the trace term is
 * evaluated for the same pair under periodic boundary conditions, where it
 * has a closed form. k starts at proj_dim and doubles while gamma moves by
 * more than 0.1 %, up to proj_dim_max. */
typedef struct {
  int    grid_points;        /* 50 log-spaced grid points (Sec. 3)            */
  double log10_gamma_lo;     /* -10: grid range [1e-10, 1e2]; the side that   */
  double log10_gamma_hi;     /*   holds the minimum is widened by 4 decades,  */
                             /*   at most twice                               */
  double refine_tol_log10;   /* 1e-5: Brent tolerance on log10(gamma)         */
  int    gcv_estimates;      /* 3: MM/SB estimate gamma at outer k < 3        */
  int    proj_dim;           /* 40                                            */
  int    proj_dim_max;       /* 160                                           */
  double gamma_fixed;        /* > 0: skip GCV and use this gamma everywhere   */
  int    exact_max_pixels;   /* 256: levels with at most this many pixels use */
                             /*   the exact GCV (dense pair, exact trace);    */
                             /*   0..1024, else DB_EINVAL. One block factors  */
                             /*   the dense pencil of each selection in FP64: */
                             /*   its cost grows as n^3 in the level's pixels */
} db_gcv_opts;

typedef struct {
  double tol_fine;           /* 1e-3 RC tolerance on level 0 (Sec. 5)         */
  double tol_coarse;         /* 1e-6 RC tolerance on levels >= 1 (Sec. 5)     */
  int    kmax;               /* 50 outer iterations per level                 */
  double eps_irls;           /* 0.03 (Sec. 5)                                 */
  double eps_mm;             /* 0.03 (Sec. 5)                                 */
  double tau_sb;             /* 0.005 (Sec. 2.3)                              */
  double lsqr_atol, lsqr_btol, lsqr_conlim;   /* 1e-6, 1e-6, 1e8              */
  int    lsqr_maxit;         /* 100                                           */
  int    lsqr_warm_start;    /* 1: LSQR solves for the correction from x^(k)  */
  db_precision precision;    /* storage precision of images and iterates      */
  int    barrier_timeout_us; /* 2,000,000: limit of every device-side wait of */
                             /*   the persistent LSQR launch (its grid        */
                             /*   barriers). A wait that runs out ends the    */
                             /*   launch on every block and the call returns  */
                             /*   DB_ETIMEOUT; the context stays usable. 0    */
                             /*   expires at the first wait (a test setting). */
  int    fine_direct;        /* 1: on level 0 of a separable PSF (odd side    */
                             /*   <= 32, side m >= 64, FP32/BF16 storage) the */
                             /*   LSQR passes apply the blur as a direct      */
                             /*   convolution over TMA-loaded windows; 0: the */
                             /*   band form on every level. Same operator,    */
                             /*   summed in another order.                    */
} db_opts;

typedef struct db_context db_context;

/* Fill defaults (the values in the comments above). */
void db_default_opts(db_opts* opts, db_gcv_opts* gcv);

/* Create a context on CUDA device `device`. `hbm_budget_bytes` caps the
 * device workspace the context may hold (0 = no cap). */
db_status db_context_create(db_context** ctx, int device, size_t hbm_budget_bytes);
db_status db_context_destroy(db_context* ctx);
/* Text of the last error recorded on this context (static storage). */
const char* db_last_error(db_context* ctx);

/* Device workspace one solve of this shape needs (bytes). */
size_t db_footprint_bytes(int m, int levels, int psf_size, db_precision prec,
                          const db_gcv_opts* gcv);

/* ---- the method: one V-cycle solve (Alg. 4) -------------------------------
 * b:   m*m observed image, column-major, float64 (host or device, per
 *      `inputs_on_device`);
 * psf: S*S PSF, column-major, float64, same residence as b;
 * levels = n + 1 >= 1 (1 = Approach I, single level; `transfer` ignored);
 *      m must be a power of two and m / 2^(levels-1) >= filter length.
 * Outputs (residence per `inputs_on_device`, caller-owned):
 *   x[m*m] float64; mu_per_level[levels] (final gamma of each level, finest
 *   first: mu for IRLS/MM, lambda for SB); iters_per_level[levels] (outer
 *   iterations); inner_iters_per_level[levels] (total LSQR iterations; may be
 *   NULL). The call synchronises `stream` before returning. */
db_status deblur_solve(db_context* ctx, const double* b, int m, const double* psf, int psf_size,
                       db_solver solver, db_wavelet wavelet, int levels, db_transfer transfer,
                       const db_gcv_opts* gcv, const db_opts* opts,
                       double* x, double* mu_per_level, int* iters_per_level,
                       int* inner_iters_per_level, int inputs_on_device, db_stream stream);

/* ---- batched solves (an addition of this library, not in the paper) --------
 * `count` independent solves advanced together: at every scheduler step each
 * unfinished problem runs one outer iteration of its current level; all of
 * their LSQR solves share one persistent cooperative launch (problems of any
 * size, level and solver in one tile list), and their GCV evaluations run
 * concurrently on a few internal streams. Results equal those of separate
 * deblur_solve calls (same kernels, same per-problem arithmetic).
 * Per request: b, psf, x as in deblur_solve (residence per
 * `inputs_on_device`); mu/iters/inner outputs are host arrays of `levels`
 * entries (inner may be NULL). All requests share `gcv` and `opts`
 * (precision included). Synchronises `stream`. */
typedef struct {
  const double* b;
  int m;
  const double* psf;
  int psf_size;
  db_solver solver;
  db_wavelet wavelet;
  int levels;
  db_transfer transfer;
  double* x;
  double* mu_per_level;
  int* iters_per_level;
  int* inner_iters_per_level;
} db_request;

db_status deblur_solve_batch(db_context* ctx, int count, const db_request* reqs, const db_gcv_opts* gcv,
                             const db_opts* opts, int inputs_on_device, db_stream stream);

/* ---- serving loop (an addition of this library, not in the paper) ---------
 * Continuous batching of deblur solves: a scheduler thread keeps up to
 * `max_resident` solves resident on the device and advances all of them one
 * outer iteration per step, exactly as deblur_solve_batch does; a submitted
 * request is admitted at the next step boundary once a slot is free and its
 * device footprint (its V-cycle state and its GCV workspace) fits the
 * budget. Each slot keeps its device workspace for the server's lifetime and
 * grows it only when a larger request arrives: once every slot has served a
 * request of the largest size, admitting and retiring requests allocates and
 * frees nothing. Results are identical to a separate deblur_solve of the
 * same request (same kernels and per-problem arithmetic).
 * Requests use host buffers: submit copies b and psf; x, mu, iters (and
 * inner if not NULL) are written into the request's host buffers before the
 * request is reported done; they must stay valid until then. FP32 storage.
 * The server's scheduler thread uses the context: make no other call on the
 * same context while a server created on it is alive (use a second context). */
typedef struct db_server db_server;

typedef struct {
  int    max_resident;       /* solves advanced together (slots), >= 1       */
  int    max_m;              /* largest image side that will be submitted    */
  size_t hbm_budget_bytes;   /* device bytes for resident solves (0 = none)  */
  db_opts opts;
  db_gcv_opts gcv;
} db_server_opts;

db_status db_server_create(db_context* ctx, const db_server_opts* opts, db_server** out);
/* Queue a request; returns at once with a ticket. DB_EINVAL for invalid
 * requests (checked here), DB_EBUSY if the server is shutting down. */
db_status db_server_submit(db_server* srv, const db_request* req, uint64_t* ticket);
/* Wait up to timeout_us (< 0: forever) for a ticket: DB_OK when done (its
 * outputs are written; latency_ms = submit to completion), DB_ETIMEOUT if not
 * yet, or the solve's own error status. A ticket can be polled until done. */
db_status db_server_poll(db_server* srv, uint64_t ticket, int timeout_us, double* latency_ms);
/* Withdraw a request. A queued one leaves the queue at once; a resident one
 * stops at the next scheduler step boundary (its slot and device memory are
 * released). Its poll then returns DB_ECANCELLED and its outputs are not
 * written. A request that has already finished is left as it is (DB_OK; its
 * poll returns its result). DB_EINVAL for an unknown ticket. */
db_status db_server_cancel(db_server* srv, uint64_t ticket);
/* Drain the queue, stop the scheduler and free everything. */
db_status db_server_destroy(db_server* srv);

/* ---- measurement ------------------------------------------------------------
 * Counters a context accumulates over its calls (reset by db_reset_stats):
 * kernel launches it issued, and for the LSQR kernel (the dominant one) its
 * launch count, device time (CUDA events recorded on the launching stream
 * around each launch when db_set_profiling(ctx, 1) is on) and the LSQR
 * iterations x pixels it processed, split by solver family (IRLS reads the
 * weight planes in both passes); with profiling on, also the wall time spent
 * in GCV selections (each ends with a synchronisation of its stream). */
typedef struct {
  uint64_t kernel_launches;
  uint64_t lsqr_launches;
  double   lsqr_ms;
  double   lsqr_pixel_iters_irls;     /* sum over launches of (its + 1) * n */
  double   lsqr_pixel_iters_other;
  uint64_t gcv_calls;
  uint64_t outer_iterations;
  double   gcv_ms;
  /* the same LSQR counters restricted to level 0 (the finest level) of
   * single-image solves */
  uint64_t lsqr_fine_launches;
  double   lsqr_fine_ms;
  double   lsqr_fine_pixel_iters_irls;
  double   lsqr_fine_pixel_iters_other;
  /* LSQR solves (one per problem of a launch) whose level-0 blur took the
   * direct path (db_opts.fine_direct), and launches of the direct
   * standalone blur (GCV Krylov basis, db_apply_blur) */
  uint64_t lsqr_direct_solves;
  uint64_t blur_direct_launches;
} db_stats;

db_status db_set_profiling(db_context* ctx, int on);
/* Launch-shape autotuner (on by default; no counterpart in the paper): the
 * first LSQR launch of a size class (storage type, tile-count bucket, PSF
 * rank one or not, band width) times each shape -- blocks per SM capped at
 * 1 or 2, band-row cache on or off -- as a complete solve on the live inputs
 * and keeps the fastest for the context's life. All shapes compute the same
 * result bit for bit, so tuning changes timing only. on = 0 uses the first
 * shape (2 blocks per SM, cache on) without timing. */
db_status db_set_autotune(db_context* ctx, int on);
db_status db_get_stats(db_context* ctx, db_stats* out);
db_status db_reset_stats(db_context* ctx);

/* ---- operator-level entry points (device pointers, float64 unless noted) --
 * These expose the individual steps of the path for testing and reuse. The
 * precision argument selects the kernel instantiation: inputs/outputs are
 * float64 buffers for DB_PREC_FP64 and float32 for DB_PREC_FP32. */

/* y = A^(level) x or (A^(level))^T x for the hierarchy built from `psf`
 * (level 0 = the PSF's zero-boundary blur, Sec. 5; level i >= 1 =
 * W^T A^(i-1) W, Sec. 4). x, y: m_i*m_i device buffers, m_i = m >> level. */
db_status db_apply_blur(db_context* ctx, const double* psf_host, int psf_size, int m,
                        db_wavelet wavelet, int level, int transpose,
                        const void* x, void* y, db_precision prec, db_stream stream);

/* *out (host) = sum_i x_i^2 over the n-element device vector x (float64,
 * float32 or bfloat16 per `prec`), formed by the reduction that gives the
 * LSQR norms (Sec. 3, the Golub-Kahan scalars alpha and beta): every square
 * enters exactly (float products with their rounding error recovered by an
 * FMA), sums are double-float pairs within a 1024-element tile, and the tile
 * partials are added in tile order. Exposed so that its accuracy against a
 * float64 reduction can be checked directly. Synchronises `stream`. */
db_status db_sumsq(const void* x, size_t n, db_precision prec, double* out, db_stream stream);

/* q = L x (two padded planes, 2*m*m) and x = L^T q (Sec. 4.2). */
db_status db_apply_L(int m, const void* x, void* q, db_precision prec, db_stream stream);
db_status db_apply_Lt(int m, const void* q, void* x, db_precision prec, db_stream stream);

/* Restriction y = W^T x (m x m -> m/2 x m/2) and prolongation x = W y
 * (Sec. 4, W = W1 kron W1, periodic stride-2 filters). m and m_coarse must
 * be powers of two (DB_EINVAL otherwise), m at least the filter length. */
db_status db_restrict(int m, db_wavelet wavelet, const void* x, void* y, db_precision prec, db_stream stream);
db_status db_prolong(int m_coarse, db_wavelet wavelet, const void* y, void* x, db_precision prec, db_stream stream);
/* Approach D blockwise transfer (Sec. 4.2): Qx_f = W~1 Qx_c W1^T,
 * Qy_f = W1 Qy_c W~1^T on padded planes (2*m_c*m_c -> 2*m_f*m_f);
 * m_coarse a power of two. */
db_status db_aux_prolong(int m_coarse, db_wavelet wavelet, const void* qc, void* qf,
                         db_precision prec, db_stream stream);

/* One LSQR solve of the augmented problem of Eq. (augmented) at level 0 of
 * `psf` on an m x m image: min ||[A; sqrt(gamma) D] delta - r0|| with
 * r0 = [b - A x0; sqrt(gamma)(c - D x0)], D = diag(w) L (solver IRLS, w from
 * `aux0` planes) or L (MM: c = aux0; SB: c = aux0 - aux1). Device buffers
 * (precision `prec`); x_out = x0 + delta. iters (host) receives the
 * iteration count. Synchronises `stream`. */
db_status db_lsqr_solve(db_context* ctx, const double* psf_host, int psf_size, int m,
                        db_solver solver, double gamma,
                        const void* b, const void* x0, const void* aux0, const void* aux1,
                        void* x_out, const db_opts* opts, int* iters,
                        db_precision prec, db_stream stream);

/* The same LSQR solve as db_lsqr_solve without a context and without any
 * device allocation. The paper has no counterpart: this exists for callers
 * that must not allocate device memory when they call (a process that gives
 * all of HBM to its own pool, a loop that may not touch the allocator).
 * All workspace comes from one 16 MiB array the library reserves when it is
 * loaded; it limits m to 256 and psf_size to 31, and a problem whose
 * workspace does not fit (e.g. a high-rank PSF) returns DB_EINVAL with a
 * message in db_last_error(NULL); so do larger m or psf_size. Arguments,
 * layouts and results are those of db_lsqr_solve; b, x0 and the auxiliary
 * planes are read in place. The blur is always applied in its band form
 * (opts->fine_direct is not used: the direct path needs tensor maps in
 * device memory), so the result equals db_lsqr_solve's with fine_direct = 0
 * and differs from its direct-path result by float32 summation order. The array is shared by every call on a device:
 * calls that overlap in time race on it and must be serialised by the
 * caller. The first call on a device looks the array up; make it before any
 * stream capture begins. Synchronises `stream`, on success and on error
 * alike: when the call returns, none of its kernels is still running. A
 * problem too large for the array is rejected while none of the call's
 * kernels is in flight. */
db_status db_lsqr_solve_static(const double* psf_host, int psf_size, int m,
                               db_solver solver, double gamma,
                               const void* b, const void* x0, const void* aux0, const void* aux1,
                               void* x_out, const db_opts* opts, int* iters,
                               db_precision prec, db_stream stream);

/* GCV choice of gamma (Sec. 3, projected form above) for the level-0
 * subproblem of the given solver with auxiliaries aux0/aux1 (device planes;
 * NULL = none: unweighted pair with zero shift). gamma_out on the host.
 * Synchronises `stream`. */
db_status db_gcv_select(db_context* ctx, const double* psf_host, int psf_size, int m,
                        db_solver solver, const void* b, const void* aux0, const void* aux1,
                        const db_gcv_opts* gcv, double* gamma_out,
                        db_precision prec, db_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* DEBLUR_H */
