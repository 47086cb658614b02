/*
 * pint.h -- C ABI of the GB300 parallel-in-time KKT solver for unsteady
 * Stokes / Oseen distributed optimal control (Heinzelreiter & Pearson,
 * "Diagonalization-Based Parallel-in-Time Preconditioners for Instationary
 * Fluid Flow Control Problems").
 *
 * The library solves the all-at-once optimality system of Sec. 2 (Eq. FinalA)
 * with flexible GMRES (Sec. 3.4), preconditioned by the block-circulant
 * approximation P_C of Sec. 3.1 whose frequency blocks (Eq. SubBlockG) are
 * handled by the Stokes transform and commutator preconditioner (Sec. 3.2,
 * Algorithms 1-2) or the Uzawa-based preconditioner of Sec. 4 (Algorithm 3).
 *
 * Conventions (all entry points)
 *  - Every call returns a pint_status; PINT_OK = 0.  No exception or C++
 *    object crosses the ABI.  On failure pint_last_error(h) (or
 *    pint_last_error(NULL) when no handle exists yet) returns a message that
 *    stays valid until the next call on the same thread.
 *  - Device pointers ("_dev") are CUDA global-memory addresses on the device
 *    that was current at pint_create; host pointers ("_host") are ordinary
 *    host memory.  The caller owns every buffer it passes; the library owns
 *    (allocates at create, frees at destroy) all of its internal workspace.
 *  - All device work is enqueued on the stream given to pint_create.  Entry
 *    points that return numbers to the host (solve, the GMRES loops inside
 *    apply_preconditioner) synchronise that stream.  A handle is not
 *    thread-safe; distinct handles may be used from distinct threads.
 *  - Time-domain all-at-once vectors ("KKT vectors") are real FP64 arrays
 *    [n_t][n_blk], one block per time level t_k = k tau (k = 1..n_t), each
 *    block holding six fields back to back:
 *        v_x, v_y (Q2, n_s = (2N+1)^2 nodes each), p (Q1, n_q = (N+1)^2),
 *        lambda_x, lambda_y (Q2), mu (Q1);
 *    node index = iy * (nodes per side) + ix on the uniform grid over
 *    [x0, x1]^2.  Residual vectors use the same slots: the adjoint-equation
 *    rows (first block row of Eq. FinalA) in the (v, p) slots, the
 *    state-equation rows in the (lambda, mu) slots.  Dirichlet velocity
 *    nodes (the boundary) and the pinned pressure node (the Q1 node at
 *    (x0, x0), index 0) are not unknowns: their input entries are ignored
 *    and their output entries are written as 0.
 *  - Frequency-domain vectors are complex FP64 (interleaved re, im) arrays
 *    [J][n_blk][2] with J = floor(n_t/2) + 1 (the Hermitian half of the
 *    spectrum; frequency n_t - j is the conjugate of j), same slots.
 */
#ifndef PINT_H
#define PINT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pint_ctx* pint_handle;

typedef enum {
  PINT_OK = 0,
  PINT_ERR_ARG = 1,            /* invalid argument or parameter            */
  PINT_ERR_OOM = 2,            /* device or host allocation failed         */
  PINT_ERR_CUDA = 3,           /* a CUDA call failed (message has details) */
  PINT_ERR_NOT_CONVERGED = 4,  /* outer solve hit outer_maxit             */
  PINT_ERR_NONFINITE = 5,      /* NaN/Inf in host input data or in a Krylov vector */
  PINT_ERR_TIMEOUT = 6,        /* a bounded device wait gave up            */
  PINT_ERR_STATE = 7           /* call out of order (e.g. solve before set_data) */
} pint_status;

typedef enum { PINT_STOKES = 0, PINT_OSEEN = 1 } pint_kind;

/* Wind of the Oseen operator (Sec. 2); RECIRC and TWO_VORTEX require
 * x0 = -1, x1 = 1.
 *  RECIRC       w = (2y(1-x^2), -2x(1-y^2)), divergence free and tangential on
 *               the boundary of [-1,1]^2; a polynomial, integrated exactly.
 *  TWO_VORTEX   the wind of the Sec. 5.2 lid-driven cavity: two elliptic
 *               vortices about (1/2, 0) and (-1/2, 0), turning opposite ways
 *               (the printed second branch read as the divergence-free one),
 *               zero outside them.  Not a polynomial: the convection matrices
 *               use the wind at 4 x 4 Gauss points per element and are taken
 *               in skew-symmetric form (N - N^T)/2, on every multigrid level.
 *  NODAL        a caller-given wind: its values at the Q2 nodes of the
 *               finest grid (pint_create_wind), used as their Q2 interpolant
 *               and injected to the nested coarser grids; convection as for
 *               TWO_VORTEX (same Gauss points, skew-symmetric form).  Any
 *               domain; the wind should be (nearly) divergence free with
 *               w . n = 0 on the boundary, as Sec. 2 assumes. */
typedef enum { PINT_WIND_NONE = 0, PINT_WIND_RECIRC = 1, PINT_WIND_TWO_VORTEX = 2, PINT_WIND_NODAL = 3 } pint_wind;

/* Arithmetic of the preconditioner.  The outer FGMRES (Arnoldi,
 * least-squares update, true residual) and the multigrid coarse solve are
 * FP64 in both modes. */
typedef enum { PINT_PREC_FP64 = 0, PINT_PREC_FP32 = 1 } pint_prec;

/* How the FP32 preconditioner evaluates the time DFT and its inverse (the
 * diagonalisation of the circulant C, Sec. 3.1): as a dense real
 * contraction of the n_t x n_t real-DFT matrix with the n_t x n_blk block of
 * time slices.
 *  AUTO     FP32: BF16X6 when n_t <= 256, else CUDA cores.  FP64: CUDA cores.
 *  SIMT     CUDA-core FMA in the preconditioner's precision.
 *  BF16X6   tensor cores (tcgen05, BF16 operands, FP32 accumulation), each
 *           operand split into three BF16 pieces and the six products whose
 *           pieces sum to order <= 2 accumulated: about FP32 accuracy.
 *  TF32X3   tensor cores (tcgen05, TF32 operands, FP32 accumulation), each
 *           operand split into two TF32 pieces, three products.
 * The tensor-core modes need n_t <= 256 and PINT_PREC_FP32; pint_create
 * returns PINT_ERR_ARG otherwise. */
typedef enum { PINT_DFT_AUTO = 0, PINT_DFT_SIMT = 1, PINT_DFT_BF16X6 = 2, PINT_DFT_TF32X3 = 3 } pint_dft_mode;

typedef struct {
  int kind;            /* pint_kind                                          */
  int level;           /* N = 2^level elements per side, 1 <= level <= 10    */
  double x0, x1;       /* square domain [x0, x1]^2                           */
  int n_t;             /* number of time blocks K (size of I_t, E, C; Sec. 2.2) */
  double tau;          /* time step                                          */
  double beta;         /* control regularisation (Eq. OseenOptimization)     */
  double nu;           /* viscosity; L = nu K + N(w)                         */
  int wind;            /* pint_wind                                          */
  int prec;            /* pint_prec                                          */
  int outer_restart;   /* FGMRES restart length m (Sec. 3.4)                 */
  int outer_maxit;     /* total outer iterations allowed                     */
  double outer_tol;    /* stop when ||b - A x||_2 / ||b||_2 <= outer_tol     */
  double inner_tol;    /* inner GMRES tolerance epsilon (Sec. 3.4, 5.1.2)    */
  int inner_maxit;     /* inner GMRES iteration cap (no restart)             */
  int mg_cycles;       /* V-cycles per multigrid application (Sec. 5.1.1: 4) */
  int mg_pre, mg_post; /* multicolour SOR sweeps before / after correction   */
  int cheb_steps;      /* Chebyshev semi-iteration steps (Sec. 5.1.1: 10)    */
  int uzawa_steps;     /* Uzawa steps in Algorithm 3 (Sec. 5.2.1: 6)         */
  double uzawa_mu;     /* Uzawa parameter mu (Sec. 4: 3/4)                   */
  double sor_omega;    /* SOR relaxation (1 = Gauss-Seidel)                  */
  int fixed_inner_its; /* > 0: run exactly this many inner GMRES iterations  */
  int linear;          /* 1: Algorithm 1 (no inner GMRES), 0: Algorithm 2/3  */
  int dft_mode;        /* pint_dft_mode                                      */
  /* SOR relaxation of the Oseen velocity multigrids on Q_j and Q_j^H (Sec. 4); */
  /* 0 = sor_omega.  Values below 1 keep those multigrids convergent on the      */
  /* convection-dominated low-frequency Q_j of large beta.                        */
  double sor_omega_conv;
} pint_params;

typedef struct {
  int outer_iterations;   /* FGMRES iterations taken                         */
  int restarts;
  double relres;          /* true ||b - A x|| / ||b|| at return (FP64)       */
  double relres_history[256]; /* Arnoldi estimates, first 256 iterations     */
  int inner_iterations_total; /* sum over applications and frequencies      */
  int inner_iterations_max;   /* largest per-frequency count in one apply   */
  int precond_applies;
  double ms_precond, ms_matvec, ms_orth, ms_total; /* host wall-clock split */
} pint_solve_info;

typedef struct {
  int N, n_t, J;
  size_t n_s, n_q, n_blk;     /* per-field / per-block sizes (see header)   */
  size_t kkt_len;             /* n_t * n_blk doubles                         */
  size_t freq_len;            /* J * n_blk complex values                    */
  size_t device_bytes;        /* workspace owned by the handle              */
} pint_sizes;

/* Upper estimate of the device memory pint_create would allocate for p
 * (bytes; 0 for invalid parameters).  Computed on the host, no CUDA call. */
size_t pint_estimate_device_bytes(const pint_params* p);

/* Defaults from Sec. 5: FGMRES(30), inner tolerance 1e-2, 4 V-cycles with
 * 2+2 SOR sweeps (omega = 1, also for Q_j: sor_omega_conv = 0), 10
 * Chebyshev steps, 6 Uzawa steps, mu = 3/4,
 * inner cap 100, outer tolerance 1e-8.  Problem fields are set to a Stokes
 * problem on [0,1]^2 with N = 8, n_t = 8, tau = 1/9, beta = 1e-2, nu = 1e-2. */
void pint_default_params(pint_params* p);

/* Create a problem (Sec. 2.2 discretisation, Sec. 3 preconditioner setup).
 * stream: a cudaStream_t (NULL = legacy default stream).  Allocates all
 * device workspace; returns PINT_ERR_ARG for invalid parameters,
 * PINT_ERR_OOM if the workspace does not fit. */
pint_status pint_create(const pint_params* p, void* stream, pint_handle* out);

/* pint_create for p->wind = PINT_WIND_NODAL: wind_host holds the wind at the
 * Q2 nodes of the finest grid, [2][n_s] (component, then node index
 * iy*(2N+1)+ix), read before the call returns.  PINT_ERR_ARG if wind_host is
 * NULL or p->wind is not PINT_WIND_NODAL (pint_create returns PINT_ERR_ARG
 * for PINT_WIND_NODAL); PINT_ERR_NONFINITE on NaN/Inf values. */
pint_status pint_create_wind(const pint_params* p, const double* wind_host, void* stream, pint_handle* out);

/* Frees everything the handle owns.  Accepts NULL. */
pint_status pint_destroy(pint_handle h);

/* Sizes of the handle's vectors and its device workspace (host struct,
 * caller-owned).  PINT_ERR_ARG for a NULL argument. */
pint_status pint_get_sizes(pint_handle h, pint_sizes* s);

/* Problem data (Sec. 2.2 backward-Euler equations): builds the right-hand
 * side b on the device.  vd_host: desired velocity [n_t][2][n_s] at
 * t_k = k tau; f_host: forcing [n_t][2][n_s] or NULL; v0_host: initial
 * velocity [2][n_s] or NULL.  Adjoint rows get tau M v_d(t_k), state rows
 * tau M f(t_k), the first state row also M v_0.  PINT_ERR_NONFINITE on
 * NaN/Inf input. */
pint_status pint_set_data(pint_handle h, const double* vd_host, const double* f_host,
                          const double* v0_host);

/* Problem data with a prescribed (non-zero) boundary velocity, as in the
 * problems of Sec. 5: the closed-form velocity on the boundary in Sec. 5.1,
 * the moving lid in Sec. 5.2.  vd_host, f_host, v0_host as in pint_set_data,
 * but read as nodal interpolants on the whole grid: every load is the
 * full-grid mass row times all nodal values (boundary values included).
 * g_host: [n_t][2][n_s] velocity at t_k = k tau, only its boundary nodes
 * read (the Dirichlet data; interior entries ignored), or NULL for zero.
 * The boundary of v0_host is the Dirichlet data at t_0.  The known boundary
 * columns of the Sec. 2.2 backward-Euler equations are moved to b: adjoint
 * rows get -tau M g_k, state rows -M (g_k - g_{k-1}) - tau L g_k (k = 1 uses
 * v_0 in place of g_0 through its load), divergence rows -tau B g_k.  The
 * adjoint velocity is zero on the boundary.  Solutions keep zero boundary
 * entries: the state velocity at t_k is the solution plus g_k.  Host
 * buffers are read before the call returns.  PINT_ERR_NONFINITE on NaN/Inf
 * input, PINT_ERR_OOM if the temporary device buffers (two KKT vectors
 * when g is given) do not fit. */
pint_status pint_set_data_dirichlet(pint_handle h, const double* vd_host, const double* f_host,
                                    const double* v0_host, const double* g_host);

/* Copy the assembled right-hand side b (KKT vector) to b_dev (caller-owned,
 * n_t * n_blk doubles).  PINT_ERR_STATE before pint_set_data or
 * pint_set_data_dirichlet. */
pint_status pint_get_rhs(pint_handle h, double* b_dev);

/* y = A x with A of Eq. FinalA, FP64, matrix-free.  x_dev, y_dev: KKT
 * vectors (must not overlap); entries of x_dev that are not unknowns are
 * ignored.  Asynchronous on the handle's stream; PINT_ERR_CUDA if a launch
 * fails. */
pint_status pint_kkt_matvec(pint_handle h, const double* x_dev, double* y_dev);

/* z = P^{-1} r: the parallel-in-time preconditioner (Algorithm 1 if
 * params.linear, else Algorithm 2 (Stokes) / the Uzawa variant (Oseen)),
 * in the handle's precision.  r_dev, z_dev: KKT vectors.  PINT_ERR_TIMEOUT
 * if a bounded wait of the tensor-core DFT gave up (the handle stays
 * usable), PINT_ERR_CUDA on launch failure. */
pint_status pint_apply_preconditioner(pint_handle h, const double* r_dev, double* z_dev);

/* Solve A x = b by FP64 FGMRES(m) with the preconditioner.  x_dev: in =
 * initial guess, out = solution (KKT vector).  info may be NULL.  Returns
 * PINT_ERR_NOT_CONVERGED (with x the last iterate) if outer_maxit is hit,
 * PINT_ERR_NONFINITE if a preconditioned Krylov vector is not finite (a
 * diverging inexact preconditioner), PINT_ERR_TIMEOUT as for
 * pint_apply_preconditioner, PINT_ERR_STATE before the data are set. */
pint_status pint_solve(pint_handle h, double* x_dev, pint_solve_info* info);

/* Same as pint_solve with host buffers: copies the initial guess host to
 * device, solves, copies the solution back (synchronous). */
pint_status pint_solve_host(pint_handle h, double* x_host, pint_solve_info* info);

/* ---- component entry points (diagnostics and parity testing) ------------ */

/* xhat = F x along time (Sec. 3.1, F_jk = exp(-2 pi i j k / n_t)) for the
 * Hermitian half j = 0..J-1; x_dev: KKT vector; xhat_dev: frequency vector. */
pint_status pint_dft_forward(pint_handle h, const double* x_dev, double* xhat_dev);

/* x = Re F^{-1} xhat, using the conjugate symmetry of the full spectrum. */
pint_status pint_dft_inverse(pint_handle h, const double* xhat_dev, double* x_dev);

/* y_j = G_j x_j (Eq. SubBlockG) for every frequency of the half spectrum;
 * frequency vectors in the library slot order (rows in the slot order of
 * the residual convention above). */
pint_status pint_freq_block_matvec(pint_handle h, const double* xhat_dev, double* yhat_dev);

/* The frequency part of the preconditioner: for every j, y_j = the block
 * solve of Algorithm 1/2 (Stokes: (T^r)^{-1} Zbar_j^{-1} (T^l)^{-1}) or of
 * Algorithm 3 inside inner GMRES (Oseen), on frequency vectors.
 * inner_its_host: NULL or int[J] receiving the inner GMRES counts. */
pint_status pint_freq_block_solve(pint_handle h, const double* rhat_dev, double* yhat_dev,
                                  int* inner_its_host);

/* Component operators on one frequency's fields (complex FP64 in/out, full
 * grid, interleaved): which =
 *   0  multigrid on W_j  (Q2 field, Sec. 3.2)      1  multigrid on Q_j (Sec. 4)
 *   2  multigrid on Q_j^H                          3  multigrid on K_p (Q1 field)
 *   4  Chebyshev on M (Q2 field)                   5  Chebyshev on M_p (Q1 field)
 *   6  block preconditioner P~_j (Stokes) / P~_j^(UZ) (Oseen), frequency block
 * j selects the frequency (0 <= j < J).  Runs in the handle's precision. */
pint_status pint_component_apply(pint_handle h, int which, int j, const double* in_dev,
                                 double* out_dev);

/* Multigrid solve on one field, like pint_component_apply with which = 0..3,
 * but without allocating anything: no device or host memory is allocated or
 * freed, by this library or any library it calls.  No counterpart in the
 * paper; it exists for callers that cannot call cudaMalloc while they run --
 * for example an application whose memory pool already reserved the device
 * memory, or a latency-critical loop where an allocation would synchronise
 * the device.
 * Scratch comes from one fixed 2 MiB array in device memory that every GPU
 * loading this library keeps until the process exits; a field whose scratch
 * does not fit (staged input, output and V-cycle levels: about N <= 64 for
 * velocity fields) is rejected with PINT_ERR_ARG and a message giving the
 * bytes needed.  The first call on a device looks up the array's device
 * address (make that first call before any stream capture).  All calls
 * share the array: calls that overlap on the GPU race.  Inputs and outputs
 * as in pint_component_apply (complex FP64, full grid, caller-owned: n_s
 * values for which = 0..2, n_q for which = 3; the call takes no length, so
 * shorter buffers are read or written past their end); the device current
 * at the call must be the handle's device.  Unlike pint_component_apply the
 * call is asynchronous: it returns with its work queued on the handle's
 * stream, and in_dev and out_dev must stay valid (and out_dev unread) until
 * that stream is synchronised.  The multigrid autotuner is not consulted
 * (its bookkeeping would allocate): the CTA size is the fixed heuristic. */
pint_status pint_mg_apply_noalloc(pint_handle h, int which, int j, const double* in_dev, double* out_dev);

/* ---- tracing ------------------------------------------------------------
 * Kernel classes of the hot path.  Launch counts are always kept; CUDA-event
 * timing (events recorded on the handle's stream around each launch of a
 * class) is kept for the classes whose bit is set in the mask. */
enum {
  PINT_PROF_MG_Q2 = 0,      /* multigrid on velocity fields (W_j, Q_j, Q_j^H)  */
  PINT_PROF_MG_Q1 = 1,      /* multigrid on pressure fields (K_p)              */
  PINT_PROF_CHEB = 2,       /* Chebyshev semi-iteration (M, M_p)               */
  PINT_PROF_DFT_FWD = 3,    /* forward time DFT                                */
  PINT_PROF_DFT_INV = 4,    /* inverse time DFT                                */
  PINT_PROF_BLOCK_MV = 5,   /* frequency-block matvec (G_j / Z_j)              */
  PINT_PROF_COMBO = 6,      /* operator combinations, transforms, axpys        */
  PINT_PROF_INNER = 7,      /* inner GMRES reductions, Givens, updates         */
  PINT_PROF_KKT_MV = 8,     /* FP64 KKT matvec (Eq. FinalA)                    */
  PINT_PROF_OUTER = 9,      /* outer FGMRES vector kernels                     */
  PINT_PROF_OTHER = 10,     /* masking, conversions, right-hand side           */
  PINT_PROF_APPLY = 11,     /* whole preconditioner applies (timing only: the
                             * events bracket every kernel of an apply, both
                             * streams; its launches are counted in the
                             * classes above)                                  */
  PINT_PROF_CLASSES = 12
};

typedef struct {
  long long launches[PINT_PROF_CLASSES]; /* kernels launched since the reset    */
  long long timed[PINT_PROF_CLASSES];    /* launches covered by event timing    */
  double ms[PINT_PROF_CLASSES];          /* summed event time of timed launches */
  /* Algorithmic bytes of the launches since the reset, counted whether or not
   * the class is timed: the compulsory traffic of each kernel's work, every
   * operand read once and every result written once (b_w bytes per real word
   * of the kernel's precision, c = 2 for complex data, n nodes of a field):
   * multigrid (4 (pre + post) + 8) n c b_w per V-cycle and field, Chebyshev
   * 5 n c b_w per step and field, block matvec 2 n_blk c b_w per frequency,
   * Gram-Schmidt (4 i + 8) n_blk c b_w at inner step i, time DFT
   * 8 n_t n_blk + J n_blk c b_w per transform, KKT matvec 16 n_t n_blk,
   * operator combinations their fields read and written once; only the
   * frequencies still active in the inner GMRES are counted. */
  double bytes[PINT_PROF_CLASSES];
  /* Host synchronisations of the solve path since the reset: one per inner
   * GMRES step (the host reads how many frequencies are still active), two
   * per outer FGMRES step, one per shared batch of a group. */
  long long host_syncs;
} pint_profile;

/* Reset the counters and select the timed classes (bit i = class i). */
pint_status pint_profile_enable(pint_handle h, unsigned mask);
/* Synchronise the handle's stream and copy the counters out. */
pint_status pint_profile_read(pint_handle h, pint_profile* out);

/* ------------------------------------------------------------------------
 * Groups: shared frequency solves of several problems.
 *
 * Handles created in a group (pint_create_in_group) solve like any handle,
 * but the frequency solves of their preconditioner applies (Algorithm 2 /
 * the Uzawa variant over all frequencies of the Hermitian half) run batched
 * with those of the group's other handles: problems that share grid level,
 * domain, wind, nu, precision and the inner-solver settings (inner_tol,
 * inner_maxit, fixed_inner_its, multigrid, Chebyshev and Uzawa counts,
 * mu, sor_omega, sor_omega_conv, linear) form a subgroup whose members'
 * applies, when several are pending, run as ONE set of launches over all
 * their frequencies, each frequency with the constants of its own problem
 * (tau, beta, n_t); a batch waits at most 3 ms for members that are inside
 * pint_solve / pint_solve_host but still in their outer step.  Each handle
 * keeps its outer FGMRES, KKT matvec and time DFT on its own stream.  The
 * frequencies are independent (Sec. 3.1), so every result is bit for bit the
 * one of the same problem solved on an ordinary handle.  Solves on handles
 * of one group share launches only when they run concurrently (one host
 * thread per solve).  No counterpart in the paper (its frequency blocks are
 * distributed over processes, Sec. 5.3).  PINT_WIND_NODAL handles cannot
 * join a group (PINT_ERR_ARG).  A group's shared workspace is allocated
 * when a batch first needs it and grows with the largest batch; it is freed
 * with the group's last handle.  Destroy every handle of a group before the
 * group. */
typedef struct pint_batcher_s* pint_group;
typedef struct {
  long long batches;       /* shared frequency solves run                        */
  long long member_solves; /* preconditioner applies they served (sum of sizes)  */
  long long frequencies;   /* frequencies solved in them                         */
  int max_members;         /* most applies in one batch                          */
} pint_group_stats;
pint_status pint_group_create(pint_group* out);
pint_status pint_create_in_group(pint_group g, const pint_params* p, void* stream, pint_handle* out);
pint_status pint_group_get_stats(pint_group g, pint_group_stats* out);
/* Tracing of a group's shared frequency solves, as pint_profile_enable /
 * pint_profile_read for a handle: counters summed over all batches since the
 * reset, class PINT_PROF_APPLY timing whole batches (the handles' own
 * counters cover their outer solves and time DFTs). */
pint_status pint_group_profile_enable(pint_group g, unsigned mask);
pint_status pint_group_profile_read(pint_group g, pint_profile* out);
pint_status pint_group_destroy(pint_group g);

/* ------------------------------------------------------------------------
 * Serving loop: continuous batching of control problems.
 *
 * A server owns max_active worker slots on the current device.  Requests
 * (any kind, level, n_t, beta, nu, precision) wait in submission order; a
 * free slot admits the oldest waiting request as soon as its estimate
 * pint_estimate_device_bytes(p) fits in what the requests on the GPU leave
 * of the server's budget.  Each admitted request gets its own handle and
 * CUDA stream: data and Krylov state stay resident on the device until it
 * completes, and the kernels of all admitted requests run concurrently.  A
 * request whose handle cannot be created for lack of memory returns to the
 * head of the queue until a running request completes, and fails with
 * PINT_ERR_OOM only on an otherwise idle server.  Results are identical to
 * a solve of the same request alone (the kernels are deterministic).
 * ---------------------------------------------------------------------- */
typedef struct pint_server_s* pint_server;

typedef struct {
  size_t device_budget; /* bytes admitted requests may hold; 0: 90% of free memory */
  int max_active;       /* worker slots (requests on the GPU at once), 1..64      */
  /* 1: batch the frequency solves of the requests on the GPU.  Requests that
   * share grid level, domain, wind, nu, precision and the inner-solver
   * settings form a group; each keeps its own outer FGMRES, KKT matvec and
   * time DFT, and the frequency solves of the members that need a
   * preconditioner apply at about the same time (a batch waits at most 3 ms
   * for members still in their outer step) run in shared launches over all
   * their frequencies, each frequency with its own problem's constants.  The
   * frequencies are independent (Sec. 3.1): every result is the same as in a
   * solve alone.  Admission then counts each request's share of its group's
   * shared workspace.  0: every request solves on its own handle. */
  int share_solves;
} pint_server_params;

typedef struct {
  long long submitted, completed, failed, active, queued;
  size_t budget_bytes, bytes_in_use, bytes_peak; /* by estimate               */
  int active_peak;                               /* most requests at once     */
  /* shared frequency solves (share_solves = 1): batches run, member applies
   * they served (sum of batch sizes), frequencies solved, largest batch */
  long long shared_batches, shared_member_solves, shared_frequencies;
  int shared_max_members;
} pint_server_stats;

/* Start the worker threads.  PINT_ERR_ARG for max_active outside [1, 64]. */
pint_status pint_server_create(const pint_server_params* sp, pint_server* out);
/* Queue a request.  vd (host, [n_t][2][n_s]) is copied, as are the optional
 * f ([n_t][2][n_s]) and v0 ([2][n_s]); the data are those of pint_set_data
 * (zero boundary velocity), and a request's handle is made by pint_create
 * (so PINT_WIND_NODAL is refused by the worker, which reports the failure
 * through pint_server_wait).  PINT_ERR_ARG for invalid params, PINT_ERR_OOM
 * if the estimate exceeds the whole budget. */
pint_status pint_server_submit(pint_server s, const pint_params* p, const double* vd, const double* f,
                               const double* v0, long long* id);
/* Block until request id completes; copy its solution (host, kkt_len
 * doubles, may be null), info and latency (submission to completion, ms).
 * Returns the request's solve status.  Each id is collected once. */
pint_status pint_server_wait(pint_server s, long long id, double* x_host, pint_solve_info* info, double* latency_ms);
pint_status pint_server_get_stats(pint_server s, pint_server_stats* out);
/* Finish every queued and running request, then stop the workers. */
pint_status pint_server_destroy(pint_server s);
/* Message of the last failed server call of the calling thread. */
const char* pint_server_last_error(void);

/* Autotuner of the multigrid launches (on by default, process-wide): for
 * each launch shape (space, grid, number of fields, precision, operator
 * variant) the launches after the first three (untimed: module loading,
 * first touch of the workspaces) run each candidate twice, interleaved,
 * timed by CUDA events on the launch stream; later launches use the fastest
 * on average.  Candidates: 256 and 512 threads per CTA for the kernels
 * with compile-time level sizes (velocity W_j, pressure operators), 256,
 * 512 and 1024 for the general kernels, for the general velocity kernel
 * each with and without the multigrid iterates staged in shared memory.
 * Results do not depend on the choice.  pint_autotune(0) restores the fixed
 * heuristic (1024 threads up to one field per SM, 512 up to two, else 256;
 * the pressure kernel 512 up to one field per SM, else 256; staging
 * whenever it fits), or the choice of pint_mg_launch_config. */
void pint_autotune(int on);
/* The multigrid launch choice used while the tuner is off (pint_autotune(0)),
 * process-wide: threads per CTA (256, 512, 1024; 0 = the fixed heuristic;
 * the kernels with compile-time level sizes take at most 512) and the
 * kernel variant: 1 or -1 = the kernels with compile-time level sizes where
 * they apply (velocity W_j on grids of 4..256 elements per side, pressure
 * operators on grids of 4..64), else the general kernels with the iterates
 * staged in shared memory where they fit; 2 = the same with the general
 * kernels unstaged; 0 = the general kernels only, unstaged.  Results agree
 * bit for bit; PINT_ERR_ARG for other values. */
pint_status pint_mg_launch_config(int threads, int staging);
/* The tuner's decisions as text, one launch shape per line, written to buf
 * (NUL-terminated, truncated to len); returns the size needed. */
size_t pint_autotune_report(char* buf, size_t len);

/* Failure injection for tests (no GPU fault is involved).
 * PINT_INJECT_DFT_STALL: the next tensor-core DFT launch of the handle arms
 * its first pipeline barrier for 16 bytes more than its bulk copy delivers,
 * so that every CTA's bounded wait (1 s) runs out; the kernel then waits
 * (bounded) for its own copies, frees its tensor memory and returns, and the
 * API call that ran it returns PINT_ERR_TIMEOUT.  The handle stays usable.
 * Returns PINT_ERR_ARG for an unknown code or if the handle does not use the
 * tensor-core DFT. */
typedef enum { PINT_INJECT_DFT_STALL = 1 } pint_inject;
pint_status pint_debug_inject(pint_handle h, int what);

/* Host only, no CUDA call: the FP64 convection stencils that pint_create
 * builds for p->wind = PINT_WIND_TWO_VORTEX or PINT_WIND_NODAL on multigrid
 * level l (0 = finest, grids of N / 2^l elements), in node order:
 * q2_out[(2n+1)^2][25] (entry dy*5+dx couples node (ix, iy) to
 * (ix+dx-2, iy+dy-2)), q1_out[(n+1)^2][9] likewise with offsets -1..1, where
 * n = N / 2^l; either output may be NULL.  wind_host: the finest-grid nodal
 * wind for PINT_WIND_NODAL (as in pint_create_wind), else NULL.
 * PINT_ERR_ARG for invalid parameters, another wind or l outside
 * [0, level). */
pint_status pint_convection_stencils(const pint_params* p, const double* wind_host, int l, double* q2_out,
                                     double* q1_out);

const char* pint_last_error(pint_handle h);

#ifdef __cplusplus
}
#endif
#endif /* PINT_H */
