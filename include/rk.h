/*
 * rk.h -- C ABI of the B300 library for mixed-precision, perturbed diagonally
 * implicit Runge-Kutta (DIRK) time stepping of linear 3D PDEs du/dt = L u.
 *
 * Method (arXiv 2412.16638):
 *   one step is u_{n+1} = u_n + tau sum_j b_j k_j                 (Eq. RKstep)
 *   with a tableau split A = A_hi + A_lo into coefficients of high-precision
 *   stage derivatives k_j = f(y_j) and low-precision ones k^eps_j = f^eps(y_j)
 *   (Sec. 2.2, Tables ButchertabA/B/C; Eqs. mpAstep1-5).  Each implicit stage
 *   solves the core system of Sec. 3 (Eq. corelinear) in the stage-derivative
 *   form (I - tau a_ii L) k^eps_i = L r_i with a low-precision preconditioned
 *   Krylov method (CG for heat, restarted GMRES for advection-diffusion,
 *   Sec. 3), followed by the high-precision explicit evaluation
 *   k_i = L (r_i + tau a_ii k^eps_i) (Sec. 2.1 step 2, Sec. 4.2).
 *
 * Grid: n^3 interior nodes of the unit cube, h = 1/(n+1), homogeneous
 * Dirichlet boundary, lexicographic numbering u[i + j n + k n^2] (Sec. 4.2).
 *
 * Conventions for every entry point:
 *   - returns rk_status; on error rk_last_error() gives a thread-local message;
 *   - never traps or aborts on bad input: arguments are checked first;
 *   - host arrays passed in are copied, never retained; the caller keeps
 *     ownership of everything it passes;
 *   - the library owns all device memory it allocates (rk_destroy_* frees it);
 *   - a problem object is not thread-safe; a server object is.
 *   - RK_ERR_NOT_CONVERGED still leaves a valid state and filled statistics.
 */
#ifndef RK_H
#define RK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RK_OK = 0,
  RK_ERR_ARG = 1,            /* invalid argument (null pointer, size, enum)      */
  RK_ERR_OOM = 2,            /* device or host allocation failed / over budget   */
  RK_ERR_CUDA = 3,           /* a CUDA runtime call failed                       */
  RK_ERR_NOT_CONVERGED = 4,  /* a stage solve hit max_iter; state still valid    */
  RK_ERR_NONFINITE = 5,      /* NaN/Inf or Krylov breakdown detected             */
  RK_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                    */
  RK_ERR_BUSY = 7,           /* server queue full / job not finished             */
  RK_ERR_NOT_FOUND = 8       /* unknown job id                                   */
} rk_status;

typedef enum { RK_F64 = 0, RK_F32 = 1, RK_F16 = 2, RK_BF16 = 3 } rk_dtype;

typedef enum {
  RK_OP_HEAT7 = 0,      /* L u = kappa/h^2 * (7-point Laplacian), constant kappa,
                           applied matrix-free (Sec. 5.2.1)                     */
  RK_OP_ADVDIFF_CSR = 1, /* L u = div(kappa(x) grad u) - v.grad u, face kappa =
                           mean of the two nodes, first-order upwind, assembled
                           in CSR (variable-coefficient stand-in for Sec. 5.2.2) */
  RK_OP_ADV_PERIODIC = 2 /* L u = -div(beta u) = -sum_d beta_d D_d u with the
                           second-order central difference D_d, periodic in every
                           direction, nodes x_i = i h, h = 1/n, n >= 3; beta = vel;
                           assembled in CSR (the advection problem of Sec. 5.2.2) */
} rk_op;

typedef enum { RK_KRYLOV_CG = 0, RK_KRYLOV_GMRES = 1 } rk_krylov;

/* Preconditioner of the stage solves.  RK_PREC_BLOCK_JACOBI: x-line blocks of
 * bj_block nodes.  RK_PREC_FDM: the fast-diagonalization preconditioner of
 * Sec. 3 (Eqs. preconbasic, Pinvform, TensorDecomp), exact for the
 * constant-coefficient heat stage matrix; applied as six tensor-core mode
 * products in the storage precision (TF32 for FP32 storage, FP16/BF16 for
 * 16-bit storage, FP32 accumulation).  Needs CG, RK_OP_HEAT7, storage F32,
 * F16 or BF16, n <= 256 and n * (storage bytes) a multiple of 16. */
typedef enum { RK_PREC_BLOCK_JACOBI = 0, RK_PREC_FDM = 1 } rk_precond;

typedef struct {
  int op;                    /* rk_op                                             */
  int n;                     /* nodes per direction, 1 <= n <= 1024 (interior nodes
                                for the Dirichlet operators)                      */
  double kappa;              /* constant diffusivity (RK_OP_HEAT7), > 0           */
  const double* kappa_field; /* RK_OP_ADVDIFF_CSR: n^3 host values at the nodes,
                                lexicographic; copied at creation                 */
  double vel[3];             /* RK_OP_ADVDIFF_CSR, RK_OP_ADV_PERIODIC: constant
                                velocity (vx,vy,vz)                               */
  const double* source;      /* optional forcing f: n^3 host values; the problem is
                                then du/dt = L u + f (Sec. 5.2.1 heat problem);
                                NULL = none; copied at creation                   */
} rk_problem_desc;

typedef struct {
  int krylov;      /* rk_krylov: CG (symmetric heat) or GMRES (advection-diffusion) */
  int restart;     /* GMRES restart length m, 1..64 (30 by default)                 */
  int bj_block;    /* block-Jacobi block size along x: 1, 2, 4, 8, 16 or 32         */
  double tol_rel;  /* stop when ||res||_2 <= tol_rel ||rhs||_2 ...                  */
  double tol_abs;  /* ... or ||res||_2 <= tol_abs (either-or rule of Sec. 5.3)     */
  int max_iter;    /* iteration cap per solve (Sec. 5.3 uses 40)                    */
  int storage;     /* rk_dtype of the Krylov vectors (and CSR values)               */
  int arith;       /* rk_dtype of the Krylov arithmetic: RK_F64 (only with F64
                      storage) or RK_F32                                            */
  int correct;     /* 1: perturbed form, k_i = L y_i re-evaluated in FP64 after the
                      low-precision solve (Sec. 2.1/2.2); 0: plain DIRK, k_i taken
                      from the solve (the FP64 baseline)                            */
  int max_refine;  /* extra refinement solves when the FP64 true residual
                      ||L r_i - (I - tau a_ii L) k^eps_i|| / ||L r_i|| exceeds
                      tol_true (0 disables)                                         */
  double tol_true; /* true-residual acceptance bound (<= 0: report only)            */
  int precond;     /* rk_precond (0 = block-Jacobi)                                 */
  int basis;       /* GMRES Krylov basis dtype: 0 or the storage dtype = same as the
                      other Krylov vectors; RK_BF16 with RK_F32 storage = compressed
                      basis (BF16 vectors, FP32 arithmetic)                        */
  int warm_start;  /* CG only: 1 = start every stage solve of rk_step/rk_integrate
                      from the previous step's solution of the same stage (the
                      stopping rule stays relative to ||rhs||); 0 = from zero, as
                      the paper's description implies.  Not with RK_F16 storage
                      (its right-hand sides are rescaled per solve)                */
  double bj_adapt_tau; /* > 0: adaptive-precision block-Jacobi (CSR operators, FP32
                      storage; the Ginkgo feature named in Sec. 1): each block's
                      inverse is stored in FP16 when its 1-norm condition number
                      kappa_1 satisfies kappa_1 * 2^-11 <= bj_adapt_tau, else in
                      FP32; 0 = every block in the storage precision             */
} rk_solver_desc;

typedef struct {
  long long iters_total; /* Krylov iterations over all solves of the call         */
  int iters_max;         /* largest single-solve iteration count                  */
  int solves;            /* number of stage solves                                */
  int refinements;       /* refinement solves triggered by the true residual      */
  int not_converged;     /* solves that hit max_iter                              */
  double true_res;       /* largest relative FP64 true residual seen (-1 if none) */
  double seconds;        /* wall time of the call                                 */
  double bytes;          /* rk_integrate_batch: algorithmic bytes of its working
                            launches (every vector element a kernel must read or
                            write once); 0 for the other calls, whose per-kernel
                            bytes rk_profile_read reports                        */
} rk_stats;

typedef struct rk_problem rk_problem;
typedef struct rk_server rk_server;

/* ---- problem lifecycle (Sec. 3 problem class; Sec. 5.2 test cases) -------- */

/* Create a problem: allocates and owns the device state (u, stage vectors,
 * Krylov workspace, operator data).  `cuda_stream` is a cudaStream_t (NULL =
 * legacy default stream) on which every later call of this problem runs.
 * Errors: RK_ERR_ARG (bad descriptor), RK_ERR_OOM, RK_ERR_CUDA. */
rk_status rk_create_problem(const rk_problem_desc* desc, const rk_solver_desc* solver,
                            void* cuda_stream, rk_problem** out);

/* Set the split Butcher tableau (Sec. 2.2): q stages (1..8), A_hi and A_lo
 * q*q row-major host arrays, b length q.  A_hi must be strictly lower
 * triangular and A_lo lower triangular (DIRK structure); stage i is implicit
 * iff A_lo[i*q+i] != 0.  Copied.  Errors: RK_ERR_ARG. */
rk_status rk_set_tableau(rk_problem* p, int q, const double* A_hi, const double* A_lo,
                         const double* b);

/* Copy n^3 float64 values into u_n.  is_device_ptr = 1: `u` is a device
 * pointer (e.g. a torch CUDA tensor), else host memory.  Synchronous. */
rk_status rk_set_state(rk_problem* p, const double* u, int is_device_ptr);

/* Copy u_n out (n^3 float64).  Synchronous. */
rk_status rk_get_state(const rk_problem* p, double* u, int is_device_ptr);

/* One time step of size dt (Eq. RKstep).  stats may be NULL. */
rk_status rk_step(rk_problem* p, double dt, rk_stats* stats);

/* nsteps steps of size dt. */
rk_status rk_integrate(rk_problem* p, double dt, int nsteps, rk_stats* stats);

rk_status rk_destroy_problem(rk_problem* p);

/* Failure detection: bound the polls of every bounded device wait in the main
 * loops of this problem's TMA-fed CG sweeps (the waits for each shared-memory
 * tile; a poll is then one non-blocking mbarrier test_wait).  0 restores the
 * default bound of 2^24 blocking try_wait polls.  When a wait runs out, the kernel lets its copies in flight land
 * (always with the default bound), marks the solve and returns; the step then
 * fails with RK_ERR_TIMEOUT, the state u_n is left as it was before the step
 * and the problem stays usable.  Small values exist to exercise that path
 * without a fault; the per-segment sweeps (shapes the TMA sweeps do not take)
 * have no device waits.  Errors: RK_ERR_ARG. */
rk_status rk_set_wait_limit(rk_problem* p, unsigned long long spins);

/* Introspection of a problem: device bytes the library allocated for it, kernel
 * launches issued so far, the block-Jacobi blocks of the last preconditioner
 * set-up on the CSR path with how many of them adaptive precision stored in
 * FP16 (0 / 0 before a set-up and on the heat path), and this problem's own
 * outcome in its last rk_integrate_batch call (RK_OK, RK_ERR_NOT_CONVERGED or
 * RK_ERR_NONFINITE; RK_OK before any): the call returns the worst outcome of
 * its problems, while the other problems' states are advanced correctly. */
typedef struct {
  size_t device_bytes;
  long long launches;
  long long bj_blocks;
  long long bj_half_blocks;
  int batch_status;
} rk_problem_info;

rk_status rk_get_problem_info(const rk_problem* p, rk_problem_info* info);

/* Guard-band check (a stand-in for a device memory checker).  When the
 * environment variable RK_GUARD_BYTES = G > 0 is set while a problem
 * allocates, each of its device blocks gets G bytes (rounded up to 256) of a
 * fixed pattern on both sides.  This call waits for the problem's stream,
 * reads every guard band back and returns in *corrupted_bytes how many pattern
 * bytes were overwritten (0 when no kernel wrote outside its buffers), and in
 * *guarded_blocks (may be NULL) how many blocks carry guards (0 when the
 * problem was created without them).  Errors: RK_ERR_ARG, RK_ERR_CUDA. */
rk_status rk_check_guards(rk_problem* p, long long* corrupted_bytes, int* guarded_blocks);

/* Test hook of the guard check: overwrite byte `offset` (0 <= offset < the
 * guard size) of the leading guard band of the problem's guarded block number
 * `block` (allocation order) with the pattern's complement, from the host.
 * It writes inside the allocation, never into a buffer.  Errors: RK_ERR_ARG
 * (no such block or offset), RK_ERR_CUDA. */
rk_status rk_guard_poke(rk_problem* p, int block, long long offset);

/* ---- single operations of the step (for testing the kernels) ------------- */

/* y = L x in FP64 (the explicit evaluation k = f(y) of Sec. 4.2, without the
 * forcing term of a problem that has one).  x, y: n^3 float64, host or device
 * per is_device_ptr. */
rk_status rk_apply_op(rk_problem* p, const double* x, double* y, int is_device_ptr);

/* Solve (I - shift L) k = g (Eq. corelinear in stage-derivative form) with the
 * problem's Krylov method, preconditioner and precision, from k = 0.  g, k:
 * n^3 float64 (k widened from the storage precision).  stats may be NULL. */
rk_status rk_solve(rk_problem* p, double shift, const double* g, double* k,
                   int is_device_ptr, rk_stats* stats);

/* z = M^{-1} r with M the problem's preconditioner of (I - shift L): the
 * x-line block-Jacobi diagonal, or the fast-diagonalization operator P, in
 * the problem's storage/arithmetic precision (r is rounded to the storage
 * type unscaled, so with FP16 storage |r| must stay below 65504).  r, z: n^3
 * float64. */
rk_status rk_apply_precond(rk_problem* p, double shift, const double* r, double* z,
                           int is_device_ptr);

/* ---- batched stepping (many independent problems per launch) ------------- */

/* Advance `count` problems by nsteps steps of size dt each.  Problems with
 * the same storage, block size, correction mode and tableau step together:
 * every phase of the stage loop is one launch over a work list of
 * (problem, tile) items of all of them, with each problem's reductions summed
 * over its own items in item order, so a problem's result does not depend on
 * the other problems of the batch.  Every problem must
 * be RK_OP_HEAT7 with CG, have a tableau and a state, and share the stream
 * of ps[0].  stats (may be NULL) receives the totals.  The launch shape of the
 * work-list kernels (CTAs per SM) is timed on the call's first steps and
 * cached per batch signature; the environment variable RK_BATCH_GRID_CAP
 * (0 = the occupancy limit, 1..64) fixes it instead.  Results do not depend
 * on the shape. */
rk_status rk_integrate_batch(rk_problem** ps, int count, double dt, int nsteps,
                             rk_stats* stats);

/* ---- serving: continuous batching of time-integration jobs --------------- */

/* Create a server that admits jobs while their device footprint fits
 * hbm_budget_bytes and a slot (of max_slots) is free; it steps all resident
 * jobs together on its own worker thread and stream. */
rk_status rk_server_create(size_t hbm_budget_bytes, int max_slots, rk_server** out);

/* Queue a job: problem + solver descriptors, tableau, host initial state u0
 * (copied), step size and count.  Returns its id.  Non-blocking. */
rk_status rk_submit_job(rk_server* s, const rk_problem_desc* desc, const rk_solver_desc* solver,
                        int q, const double* A_hi, const double* A_lo, const double* b,
                        const double* u0, double dt, int nsteps, uint64_t* job_id);

/* done = 1 when the job has finished (result ready).  Non-blocking. */
rk_status rk_poll_job(rk_server* s, uint64_t job_id, int* done);

/* Block until the job finishes; copy its final state (n^3 float64, host) into
 * u_out (may be NULL) and its statistics into stats (may be NULL); latency_s
 * (may be NULL) receives submit-to-finish seconds.  Frees the job. */
rk_status rk_wait_job(rk_server* s, uint64_t job_id, double* u_out, rk_stats* stats,
                      double* latency_s);

/* Timeline of a finished job, for checking how jobs shared the device.  Times
 * are seconds since rk_server_create; a tick is one round in which the server
 * launches one step of every resident job (the steps of one tick run
 * concurrently on the device).  -1 where the job never got that far. */
typedef struct {
  double t_submit;       /* rk_submit_job returned                             */
  double t_admit;        /* admitted: a slot and budget were free              */
  double t_first_step;   /* the tick of its first step started                 */
  double t_done;         /* finished (result copied to the host)               */
  long long first_tick;  /* first and last tick in which the job was stepped   */
  long long last_tick;
  int steps;             /* steps completed                                    */
} rk_job_info;

/* rk_wait_job, and the job's timeline into info (may be NULL).  Frees the job. */
rk_status rk_wait_job_info(rk_server* s, uint64_t job_id, double* u_out, rk_stats* stats,
                           rk_job_info* info);

rk_status rk_server_destroy(rk_server* s);

/* ---- profiling: CUDA events around every kernel launch of a problem ------ */

typedef struct {
  char name[32];           /* kernel name                                       */
  long long launches;      /* launches that did work                            */
  long long noop_launches; /* sweeps launched after their solve had finished     */
  double ms_total;         /* summed event time of the working launches          */
  double bytes_total;      /* algorithmic bytes (compulsory HBM traffic) of the
                              working launches: every vector element the kernel
                              must read or write once                            */
} rk_kernel_stat;

/* enable = 1: record a CUDA event pair on the problem's stream around every
 * kernel launch from now on; 0: stop.  Either way the counters are cleared. */
rk_status rk_profile(rk_problem* p, int enable);

/* Synchronise the problem's stream and return per-kernel totals since the
 * last rk_profile() call (up to max entries; *count = entries written) and
 * the number of kernel launches the problem issued (profiled or not). */
rk_status rk_profile_read(rk_problem* p, rk_kernel_stat* out, int max, int* count,
                          long long* launches_total);

/* ---- solve without allocating (no counterpart in the paper) -------------- */

/* For callers that may not allocate device memory (a memory pool or arena that
 * owns the device, a host program whose allocator policy forbids cudaMalloc, or
 * code that must not trigger the implicit synchronisation of cudaMalloc/
 * cudaFree): the rk_solve stage solve of the heat operator, (I - shift L) k = g
 * with L = kappa/h^2 * 7-point Laplacian on n^3 nodes, FP32 block-Jacobi CG
 * (blocks of bj_block x-nodes), tolerances and iteration cap as in
 * rk_solver_desc, from k = 0.  g_dev and k_dev are caller-owned device arrays of
 * n^3 float64; *iters (may be NULL) receives the iteration count.
 * The workspace is a fixed device array inside the library (about 5.3 MB), so n
 * is limited to 1..64; larger n returns RK_ERR_ARG with an explanation.  The
 * CUDA runtime places that array (with the library's device code) on a device
 * at its first use there: the FIRST call on a device takes those 5.3 MB and can
 * fail with RK_ERR_CUDA (out of memory) on a full device, so make it before a
 * pool claims the device's memory (or set CUDA_MODULE_LOADING=EAGER); the array
 * then stays until the process exits and later calls allocate nothing.  Every
 * call looks up the array's address on the current device.  The call is
 * synchronous (it reads the solver status back between chunks of sweeps) and
 * must not be made while any stream is being captured.  All calls share the
 * array: calls that overlap on the GPU race and must be serialised by the
 * caller.  No counterpart in the paper.
 * Errors: RK_ERR_ARG, RK_ERR_CUDA, RK_ERR_NOT_CONVERGED, RK_ERR_NONFINITE. */
rk_status rk_heat_solve_noalloc(int n, double kappa, double shift, int bj_block, double tol_rel,
                                double tol_abs, int max_iter, const double* g_dev, double* k_dev,
                                void* cuda_stream, int* iters);

/* Thread-local description of the last error on this thread ("" if none). */
const char* rk_last_error(void);

/* Library version string. */
const char* rk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RK_H */
