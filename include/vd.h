/*
 * vd.h -- C ABI of the GB300 (sm_103a) variable-density spectral elliptic solver.
 *
 * Method: Reynier, Di Pierro, Alizard, Cadiou, Le Penven, Buffat, "A preconditioning for
 * the spectral solution of incompressible variable-density flows" (arXiv 2403.06654).
 * The library solves the elliptic systems of each semi-implicit second-order time step on
 * a fully periodic (Fourier x Fourier x Fourier) grid:
 *   pressure  L_rho(phi) = div(rho^-1 grad phi) = f             (Eq. VDINSE.Lrho / Lrho.num)
 *   velocity  V_rho(u)   = u - (dt/2) zeta(rho, u) = b            (Eq. VDINSE.zeta, num.momentum.proj;
 *                                                                   1D form Eq. VDINSE.Vrho)
 * by preconditioned CG, GMRES or Richardson Minimal Residual (Sec. 3.1), with the inverse
 * of the constant-density operator as preconditioner (Eq. VDINSE.V for the velocity; the
 * inverse Laplacian with the k = 0 mode removed for the pressure, Sec. 3.2 and the text
 * before Table 2).
 *
 * Conventions shared by every call
 *  - Every call returns a vd_status; VD_OK is 0.  On failure vd_last_error() returns a
 *    message for the calling thread.  No C++ exception crosses the ABI.
 *  - Device buffers are owned by the caller: the library reads and writes them and never
 *    frees them.  Only vd_grid_create allocates device memory of its own (the twiddle
 *    tables, a few KB), released by vd_grid_destroy.
 *  - Calls that take a stream are stream-ordered on it: they enqueue kernels and return;
 *    vd_solve and vd_density_set also synchronise the stream to read convergence flags and
 *    density bounds.  Pass 0 for the legacy default stream.
 *  - Fields are row-major with x fastest: a physical scalar field holds n0*n1*n2 doubles
 *    laid out [n2][n1][n0] (1D: n1 = n2 = 1; 2D: n2 = 1).  A vector field stores its ndim
 *    components back to back.  Every axis length must be even and factor into 2, 3 and 5,
 *    with 4 <= n <= 1024.
 *  - Discretisation: Fourier differentiation D_j = F^-1 diag(i k~_j) F with the Nyquist
 *    wavenumber set to zero, and the Laplacian sum_j D_j D_j (symbol -|k~|^2).  The pressure
 *    operator then has a null space of dimension 2^ndim (the modes whose every index is 0
 *    or n/2); pressure solves return the solution orthogonal to it.
 */
#ifndef VD_H_
#define VD_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vd_grid vd_grid;
typedef struct CUstream_st* vd_stream; /* same type as cudaStream_t */

typedef enum {
  VD_OK = 0,
  VD_ERR_INVALID_ARG = 1,    /* bad size, null pointer, rho <= 0 or non-finite, CG on V_rho */
  VD_ERR_OOM = 2,            /* workspace smaller than the query says, or allocation failed */
  VD_ERR_CUDA = 3,           /* a CUDA runtime call failed; message has the CUDA error */
  VD_ERR_NOT_CONVERGED = 4,  /* max_it reached above tol (x holds the last iterate) */
  VD_ERR_BREAKDOWN = 5,      /* Krylov breakdown (zero curvature / zero search direction) */
  VD_ERR_DIVERGED = 6,       /* RMR: monitored residual grew above 1e3 x the best value */
  VD_ERR_NONFINITE = 7,      /* NaN or Inf met in a reduction */
  VD_ERR_NO_DENSITY = 8,     /* an operator was used before vd_density_set */
  VD_ERR_RHS_NOT_IN_RANGE = 9, /* the part of b outside the operator's range exceeds
                                 vd_solve_params.range_tol ||b|| (only when range_tol > 0) */
  VD_ERR_TIMEOUT = 10        /* a kernel gave up a bounded wait on its own staged transfers
                                (vd_solve reports it; the result is not valid) */
} vd_status;

/*
 * Operators.  VD_OP_PRESSURE: L~_rho phi = sum_j D_j(rho^-1 D_j phi) (Eq. VDINSE.Lrho.num).
 * VD_OP_VELOCITY: V~_rho (Eq. VDINSE.zeta with the Crank--Nicolson factor a).
 * VD_OP_KRHO: the modified-Helmholtz form of the pressure equation (Sec. 4.2, Eq. VDINSE.Krho)
 * for Phi = phi / sqrt(rho): K~ Phi = Lap Phi + c Phi with the full-wavenumber Laplacian
 * (symbol -|k|^2, Nyquist kept) and c = -Lap(w) / w, w = rho^-1/2 -- the paper's coefficient
 * Lap rho / (2 rho) - 3 |grad rho|^2 / (4 rho^2), formed so that K~ w = 0 holds exactly.  Its
 * preconditioner is the pseudo-inverse of that Laplacian (the mean removed); a solve returns
 * the zero-mean Phi for the right-hand side projected onto the w-orthogonal range (pass
 * sqrt(rho) f to solve the pressure equation; phi = sqrt(rho) Phi).  Two scalar transforms
 * per apply instead of 2 ndim.
 */
typedef enum { VD_OP_PRESSURE = 0, VD_OP_VELOCITY = 1, VD_OP_KRHO = 2 } vd_op;
typedef enum { VD_SOLVER_CG = 0, VD_SOLVER_GMRES = 1, VD_SOLVER_RMR = 2 } vd_solver;
typedef enum {
  VD_PREC_FP64 = 0,  /* every transform, product and reduction in IEEE double */
  VD_PREC_MIXED = 1, /* inner Krylov solve with float transforms and preconditioner, double
                        dot products, inside a double iterative-refinement loop whose true
                        residual uses the double operator */
  VD_PREC_MIXED_DD = 2 /* as VD_PREC_MIXED, but the refinement residual b - A x is formed with
                        float-pair transforms (two floats per value, ~2^-48 relative rounding,
                        on the FP32 pipes; storage stays double; the velocity operator's
                        pointwise bracket stays double).  On GB300 double arithmetic runs at
                        1/69 of the float rate, which makes this much faster.  The residual
                        that certifies tol carries the float-pair error, normwise
                        ~2^-47 |A| |x| / |b|. */
} vd_precision;

/* Parameters of the velocity operator: a = dt/(2 Re) (Eq. VDINSE.Vrho), inv_sc = 1/Sc. */
typedef struct {
  double a;
  double inv_sc;
} vd_op_params;

typedef struct {
  double tol;        /* stop when the monitored relative residual <= tol */
  int max_it;        /* limit on operator applications inside the Krylov loop(s) */
  int restart;       /* GMRES restart length m (1..64), default 30 when <= 0 */
  int use_x0;        /* 1: x holds the initial guess (warm start, Sec. 3.1); 0: start from 0 */
  int precision;     /* vd_precision */
  double inner_tol;  /* mixed modes: relative tolerance of each inner float solve (<= 0: 1e-5).
                        A float CG cannot go much below kappa times the float rounding: an inner CG
                        solve below 1e-3 whose residual has not halved in 8 iterations, or has
                        grown 100-fold from its best, ends its sweep and the refinement goes on */
  int check_every;   /* iterations enqueued between host convergence checks (default 1); CG
                        and RMR check one batch behind, so one batch may be launched after
                        convergence: its kernels see the device flag and return at once */
  int coef_pair;     /* VD_PREC_MIXED(_DD), pressure and K_rho operators: arithmetic of the
                        variable-coefficient multiply (1/rho, or c of K_rho) inside the inner float
                        operator.  0 (default): float pairs (hi + lo, ~2^-48, the multiply rounded
                        once to float) when rho_max / rho_min > 10, plain float otherwise;
                        1: always float pairs; -1: always plain float */
  double range_tol;  /* pressure and K_rho right-hand sides lose their part outside the range
                        (its norm is reported in vd_solve_info.rhs_removed).  0 (default): project
                        silently; > 0: refuse with VD_ERR_RHS_NOT_IN_RANGE when that part
                        exceeds range_tol ||b|| (checked before iterating; synchronises stream) */
} vd_solve_params;

typedef struct {
  int iters;           /* operator applications in the Krylov loop(s) */
  int outer_iters;     /* VD_PREC_MIXED: refinement sweeps (0 otherwise) */
  int status;          /* vd_status of the solve */
  double relres;       /* last monitored relative residual */
  double relres_true;  /* ||b - A x|| / ||b|| of the returned x, with the double operator */
  double* hist;        /* optional host array: monitored relres per iteration (hist[0] = initial) */
  int hist_cap;        /* capacity of hist */
  int hist_len;        /* entries written */
  double rhs_removed;  /* ||Pi b - b|| / ||b||: the relative part of the right-hand side outside
                          the operator's range, removed before solving (pressure: the 2^ndim
                          null-space modes; K_rho: the component along w = rho^-1/2; velocity: 0).
                          relres and relres_true are relative to ||Pi b|| */
  int coef_pair;       /* 1 if the inner float operator multiplied by 1/rho (or c) in float pairs */
} vd_solve_info;

/* Last error message of the calling thread (static storage, never null). */
const char* vd_last_error(void);

/* Library version string. */
const char* vd_version(void);

/*
 * Create a periodic grid: ndim in {1,2,3}; n[j] points over length L[j] along axis j
 * (j = 0 is x).  Entries beyond ndim are ignored.  Builds the FFT plans and uploads the
 * twiddle tables (library-owned device memory) on the current device.
 * Errors: VD_ERR_INVALID_ARG for an unsupported size, VD_ERR_CUDA/OOM on allocation.
 */
vd_status vd_grid_create(int ndim, const int n[3], const double L[3], vd_grid** out);
vd_status vd_grid_destroy(vd_grid* grid);

/* Number of points (n0 n1 n2) and of half-spectrum coefficients ((n0/2+1) n1 n2). */
size_t vd_grid_points(const vd_grid* grid);
size_t vd_grid_modes(const vd_grid* grid);

/*
 * Density data: bytes of the caller-owned device buffer that vd_density_set fills with
 * rho, 1/(N rho) (double and float) and, when `op` is VD_OP_VELOCITY, the spectral first
 * and second derivatives D_j rho and D_i D_j rho (reading: the paper does not say how
 * they are formed; they are the Fourier derivatives of the grid density).  With VD_OP_KRHO
 * it also holds the coefficient c/N of K~ (double, float, float-pair) and the normalised
 * spectrum of w = rho^-1/2; the pressure operator stays usable with that buffer.
 */
size_t vd_density_bytes(const vd_grid* grid, vd_op op);

/*
 * Attach the density rho (device, n0 n1 n2 doubles, caller-owned, not retained) to the
 * grid, precomputing into dens_ws (device, vd_density_bytes(grid, op) bytes, caller-owned,
 * must stay alive while the grid uses it).  Checks rho > 0 and finite
 * (VD_ERR_INVALID_ARG otherwise; this synchronises `stream`).  The grid keeps pointers
 * into dens_ws until the next vd_density_set.
 */
vd_status vd_density_set(vd_grid* grid, vd_op op, const double* rho, void* dens_ws, size_t dens_bytes,
                         vd_stream stream);

/* Workspace bytes needed by vd_apply_op / vd_apply_precond / vd_solve (caller-owned). */
size_t vd_workspace_bytes(const vd_grid* grid, vd_op op, vd_solver solver, const vd_solve_params* params);

/*
 * out = A(in) on physical fields, A = L~_rho (pressure, scalar field), K~ (VD_OP_KRHO, scalar
 * field) or V~_rho (velocity, ndim-component field, params required).  in and out may not
 * alias.  Forward transform, spectral apply, inverse transform, all on `stream`.
 */
vd_status vd_apply_op(const vd_grid* grid, vd_op op, const vd_op_params* params, const double* in, double* out,
                      void* ws, size_t ws_bytes, vd_stream stream);

/*
 * out = M(in): the constant-density inverse, diagonal in Fourier space.
 * Pressure: multiply by -1/|k~|^2, 0 on the null-space modes (pseudo-inverse of the
 * Laplacian).  VD_OP_KRHO: multiply by -1/|k|^2 (full wavenumbers), 0 for the mean only.
 * Velocity: multiply every component by 1/(1 + a |k~|^2) (Eq. VDINSE.V).
 */
vd_status vd_apply_precond(const vd_grid* grid, vd_op op, const vd_op_params* params, const double* in, double* out,
                           void* ws, size_t ws_bytes, vd_stream stream);

/*
 * Solve A x = b (physical fields) with the chosen Krylov method, right-preconditioned by
 * M (GMRES, RMR) or split-preconditioned (CG).  Pressure right-hand sides are first
 * projected onto the range of L~ (their null-space modes are removed); x is returned
 * orthogonal to the null space.  VD_OP_KRHO right-hand sides lose their component along
 * w = rho^-1/2 and x is returned zero-mean.  CG with VD_OP_VELOCITY is rejected (VD_ERR_INVALID_ARG:
 * V_rho is not symmetric, Sec. 3.1).  x is input (initial guess if use_x0) and output.
 * info (optional, host) receives iteration counts, residuals and history.  Returns the
 * solve status (VD_OK when converged).
 */
vd_status vd_solve(const vd_grid* grid, vd_op op, vd_solver solver, const vd_op_params* op_params,
                   const vd_solve_params* params, const double* b, double* x, vd_solve_info* info, void* ws,
                   size_t ws_bytes, vd_stream stream);

/*
 * Plain transforms of the F-F-F discretisation (Sec. 3: constant-coefficient problems are
 * diagonal in Fourier space; the transforms are the unit of cost of every apply).
 * vd_fft_r2c: unnormalised forward DFT over every axis of a physical field (n0 n1 n2 reals)
 * into its half spectrum ((n0/2+1) n1 n2 complex values, interleaved re/im, layout
 * [n2][n1][n0/2+1]): out(k) = sum_x in(x) exp(-i k.x).  vd_fft_c2r: the inverse, divided by
 * N = n0 n1 n2 (the imaginary parts of the self-conjugate modes are ignored).
 * prec: VD_PREC_FP64 (double fields, double arithmetic), VD_PREC_MIXED (float fields, float
 * arithmetic), VD_PREC_MIXED_DD (double fields, float-pair arithmetic).  ws: device scratch
 * of vd_transform_ws_bytes(grid, prec) bytes (unused by the double and float r2c and by 1D
 * c2r).  in and out (device, caller-owned) may not alias.  Stream-ordered, no synchronisation.
 */
size_t vd_transform_ws_bytes(const vd_grid* grid, int prec);
vd_status vd_fft_r2c(const vd_grid* grid, int prec, const void* in, void* out, void* ws, size_t ws_bytes,
                     vd_stream stream);
vd_status vd_fft_c2r(const vd_grid* grid, int prec, const void* in, void* out, void* ws, size_t ws_bytes,
                     vd_stream stream);

/* out = sum_j D_j u_j (spectral divergence of an ndim-component physical field). */
vd_status vd_divergence(const vd_grid* grid, const double* u, double* out, void* ws, size_t ws_bytes,
                        vd_stream stream);

/* out_j = D_j phi (spectral gradient; out holds ndim components). */
vd_status vd_gradient(const vd_grid* grid, const double* phi, double* out, void* ws, size_t ws_bytes,
                      vd_stream stream);

/*
 * Semi-implicit second-order step (Sec. 2: Eqs. VDINSE.num.mass.proj, num.momentum.proj,
 * Lrho.num, num.proj, num.gradp.update) on the grid: Crank--Nicolson + Adams--Bashforth 2
 * mass update (diagonal in Fourier), rho_h = (rho^{n+1} + rho^n)/2, velocity predictor solved
 * with V~_{rho_h} (a = dt/(2 Re); warm start u^n), pressure increment L~_{rho_h} phi = div(u*) / dt
 * (warm start: previous phi), projection u = u* - dt grad(phi) / rho_h and the pressure update
 * in the scalar form of Eq. VDINSE.num.p.update (the form the paper's time study marches),
 * kept as its gradient: grad p += grad phi - grad Lap^+ div(rho_h (dt/2) zeta(rho_h,
 * grad phi / rho_h)).  Readings: Euler for the first step's advection terms; gravity along
 * gravity_axis as the periodic body force -Fr^-1 (1 - <rho_h>/rho_h) (the paper's -Fr^-1 e_z
 * with its mean weight removed); -1 for no gravity.
 * Memory: vd_flow_bytes() device bytes (caller-owned) hold the state (rho, u, grad p, phi,
 * Adams--Bashforth history), temporaries, the density data and the solve workspace.  The
 * flow owns its grid's density slot while it steps (vd_flow_step calls vd_density_set).
 * State fields are physical, layout as for every other call; u and grad p have ndim
 * components.  vd_flow_step synchronises the stream (density checks, convergence flags).
 * Errors as in vd_solve; a solve that stops unconverged is reported in info and in the
 * returned status, the step is still completed.
 */
typedef struct vd_flow vd_flow;
typedef struct {
  double Re, Sc, Fr;
  int gravity_axis;   /* axis of gravity (0..ndim-1), -1 for none */
  int vel_solver;     /* VD_SOLVER_GMRES or VD_SOLVER_RMR */
  int pres_solver;    /* any vd_solver */
  double tol;         /* relative tolerance of both solves */
  int max_it, restart, precision;
} vd_flow_params;
typedef struct {
  int vel_iters, pres_iters, vel_status, pres_status;
  double vel_relres, pres_relres;   /* true relative residuals of the two solves */
} vd_step_info;
size_t vd_flow_bytes(vd_grid* grid, const vd_flow_params* params);
vd_status vd_flow_create(vd_grid* grid, const vd_flow_params* params, void* mem, size_t bytes, vd_flow** out);
vd_status vd_flow_destroy(vd_flow* flow);
/* initial state: rho (n points) and u (ndim fields); grad p and phi start at 0 */
vd_status vd_flow_set_state(vd_flow* flow, const double* rho, const double* u, vd_stream stream);
/* optional source terms for the following steps (Sec. 4.1 adds a mass source and a body
 * force so that a manufactured field solves the equations): mass_source (n points) and force
 * (ndim fields), device buffers the flow copies; each step uses them as values at its mid-time
 * t^{n+1/2}: -dt [u.grad rho - S] in the mass update, +dt F in the predictor.  Set them before
 * every step whose sources change; a null pointer removes that term.  Not part of snapshots. */
vd_status vd_flow_set_sources(vd_flow* flow, const double* mass_source, const double* force, vd_stream stream);
/* copy out any of rho, u, grad p, phi (null pointers are skipped) */
vd_status vd_flow_get_state(const vd_flow* flow, double* rho, double* u, double* gradp, double* phi,
                            vd_stream stream);
vd_status vd_flow_step(vd_flow* flow, double dt, vd_step_info* info, vd_stream stream);
/*
 * Checkpoint / resume (not in the paper).  A snapshot is the complete state a step reads:
 * rho, u, grad p, phi (the pressure solve's initial guess) and the previous step's explicit
 * terms of the Adams--Bashforth extrapolation with their presence flag, behind a header that
 * records the grid.  vd_flow_save copies it to a host buffer (synchronises `stream`);
 * vd_flow_load restores it into a flow on a grid of the same sizes (INVALID_ARG otherwise), and
 * the steps that follow are bit-identical to those of the flow that was saved (same kernels in
 * the same order, the same launch shapes).
 */
size_t vd_flow_snapshot_bytes(const vd_flow* flow);
vd_status vd_flow_save(const vd_flow* flow, void* host, size_t bytes, vd_stream stream);
vd_status vd_flow_load(vd_flow* flow, const void* host, size_t bytes, vd_stream stream);

/*
 * Request server (continuous batching; not in the paper).  Pressure solves of different
 * grids, densities and tolerances are submitted at any time, queue in FIFO order, and are
 * admitted as soon as one of max_inflight execution slots is idle and the request's device
 * memory (vd_server_request_bytes) fits in the HBM budget (hbm_budget bytes, 0 = 80% of the
 * free memory at creation).  Admitted requests run concurrently, each on its slot's own CUDA
 * stream; their Krylov state stays in their device workspace until they complete, when the
 * memory returns to the server and the next requests are admitted.  The server allocates
 * request memory itself (stream-ordered allocator).  rho and b are device buffers owned by
 * the caller and must stay valid until the request's completion has been polled.  The
 * solution goes to the caller's x when x is not null; with x null the server keeps it in
 * its own device memory, counted in the request's bytes and in the HBM budget until the
 * caller calls vd_server_fetch (copy out, then free) or vd_server_release (free) with the
 * request's id, so a client never allocates on the submit path.
 * Completions carry steady-clock timestamps (seconds) of submission, start and end.
 * A request's result does not depend on the other requests in flight.
 */
typedef struct vd_server vd_server;
typedef struct {
  int max_inflight;    /* concurrent requests (1..64) */
  size_t hbm_budget;   /* bytes available to admitted requests; 0 = 80% of free memory */
} vd_server_params;
typedef struct {
  unsigned long long id;
  int ndim;
  int n[3];
  double L[3];
  const double* rho;   /* density (n0 n1 n2 doubles, device) */
  const double* b;     /* right-hand side (device) */
  double* x;           /* solution (device, written on completion); null: server-owned */
  int solver;          /* vd_solver */
  double tol;
  int max_it, restart, precision;
} vd_request;
typedef struct {
  unsigned long long id;
  int status;          /* vd_status of the solve */
  int iters;
  double relres_true;
  double t_submit, t_start, t_done;
  const double* x;     /* device address of the solution (the caller's x, or server-owned) */
} vd_completion;
vd_status vd_server_create(const vd_server_params* params, vd_server** out);
/* device bytes a request will hold while running (density data + solve workspace, plus the
 * solution when x is null); 0 on bad sizes */
size_t vd_server_request_bytes(const vd_request* request);
/* enqueue (the request is copied); bytes = vd_server_request_bytes(request) */
vd_status vd_server_submit(vd_server* server, const vd_request* request, size_t bytes);
/* withdraw a request that is still queued (not admitted): it produces no completion.
 * INVALID_ARG if no queued request has this id (unknown, admitted or completed). */
vd_status vd_server_cancel(vd_server* server, unsigned long long id);
/* move up to max completions into out; returns how many */
int vd_server_poll(vd_server* server, vd_completion* out, int max);
/* server-owned solution of completed request id: copy it to dst (n0 n1 n2 doubles, device,
 * ordered on stream) and free it / only free it.  INVALID_ARG if id holds no server-owned
 * solution (unknown, not completed, caller-owned or already released). */
vd_status vd_server_fetch(vd_server* server, unsigned long long id, double* dst, vd_stream stream);
vd_status vd_server_release(vd_server* server, unsigned long long id);
/* block until every submitted request has completed */
vd_status vd_server_drain(vd_server* server);
vd_status vd_server_stats(vd_server* server, long long* submitted, long long* completed, long long* inflight,
                          size_t* reserved, size_t* budget);
/* drains, then stops the workers */
vd_status vd_server_destroy(vd_server* server);

/*
 * Batched solves in one graph launch (not in the paper).  A batch holds `count` independent
 * instances of any grids and densities; each carries a velocity system (V~_rho with its own a
 * and 1/Sc, ndim components; b_vel/x_vel non-null), a pressure system (L~_rho; b_pres/x_pres
 * non-null) or both.  vd_batch_create attaches every density (synchronising `stream`), lays
 * every grid's density data and solve workspace out in the caller's device buffer `mem`
 * (vd_batch_bytes bytes, caller-owned, alive until vd_batch_destroy) and records every solve
 * into one CUDA graph: each system is a branch of its own, and its Krylov
 * loop a conditional WHILE node whose body is one iteration (one restart cycle for GMRES) and
 * whose condition a kernel sets from the device-resident convergence flag.  vd_batch_run
 * replays all solves with a single graph launch on `stream`, reading the right-hand sides
 * and writing the solutions at each run (new right-hand sides need no rebuild; the buffers
 * named at creation must stay valid).  x starts from 0.  vd_batch_info waits for the device
 * and reports one instance's results (iterations, status, monitored and true relative
 * residual).  CG is refused for the velocity system.  The event profiler must be off while
 * recording.
 */
typedef struct vd_batch vd_batch;
typedef struct {
  int ndim;
  int n[3];
  double L[3];
  const double* rho;     /* density (device) */
  const double* b_vel;   /* velocity right-hand side, ndim fields (device), or null */
  double* x_vel;         /* velocity solution, ndim fields (device) */
  double a, inv_sc;      /* velocity operator parameters */
  const double* b_pres;  /* pressure right-hand side (device), or null */
  double* x_pres;        /* pressure solution (device) */
} vd_batch_item;
typedef struct {
  int vel_solver;        /* VD_SOLVER_GMRES or VD_SOLVER_RMR */
  int pres_solver;       /* any vd_solver */
  double tol;
  int max_it, restart;
  int precision;         /* vd_precision: FP64, or the refinement loop recorded into the graph as
                            a conditional WHILE node around the float inner solve */
} vd_batch_params;
size_t vd_batch_bytes(const vd_batch_item* items, int count, const vd_batch_params* params);
vd_status vd_batch_create(const vd_batch_item* items, int count, const vd_batch_params* params, void* mem,
                          size_t bytes, vd_stream stream, vd_batch** out);
vd_status vd_batch_run(vd_batch* batch, vd_stream stream);
vd_status vd_batch_info(vd_batch* batch, int index, vd_solve_info* vel, vd_solve_info* pres);
/* number of nodes of the recorded graph (top level) */
size_t vd_batch_graph_nodes(const vd_batch* batch);
vd_status vd_batch_destroy(vd_batch* batch);

/*
 * Launch-shape autotuner of the transform passes (not in the paper).  For this grid and each
 * arithmetic type in `precisions` (bit 0 double, bit 1 float, bit 2 float-pair), every pass
 * the solvers use (y and z passes in both directions; the x pass forward, inverse and fused)
 * is timed with CUDA events on `scratch` (device, vd_autotune_bytes(grid) bytes, caller-owned,
 * overwritten) for each candidate shape: the register-resident four-step kernel where one
 * exists, and the shared-memory Stockham engine with 1, 2, 4, ... lines per block up to the
 * shared-memory limit.  The fastest shape goes into a process-wide table keyed by (pass, type,
 * length, axis, direction or x-pass form) that every later launch on any grid consults; with
 * the environment variable VD_TUNE_FILE set the table is written to that file, and read from
 * it at the first launch or query of a later process.  Synchronises `stream`.  Shapes change
 * the work distribution only; results stay within the parity bounds.  The event profiler must
 * be off while tuning.
 */
size_t vd_autotune_bytes(const vd_grid* grid);
vd_status vd_autotune(const vd_grid* grid, int precisions, void* scratch, size_t bytes, vd_stream stream);
/* entries of the table, 6 ints each (kind 0 y/z pass or 1 x pass, type 0 double / 1 float /
 * 2 float-pair, length, axis, direction or x-pass form, choice: 0 register kernel, 1..64 lines
 * per block, 128 the register kernel with TMA-staged tiles (float y/z passes of length 128 and
 * 256), 256 the Stockham engine on unpacked float pairs (float-pair passes; the default packed
 * engine gives the same bits); writes at most max entries to out (may be null) and returns the
 * total count */
int vd_autotune_table(int* out, int max);
/* set one entry by hand (choice < 0 erases it); INVALID_ARG on a bad key or choice */
vd_status vd_autotune_set(int kind, int type, int n, int axis, int dir, int choice);

/*
 * out = L~_rho(in) for callers that cannot allocate device memory (the paper has no
 * counterpart; this is an integration convenience).  Such callers include code running
 * inside a host framework whose memory pool owns the device, plugins that must keep a
 * fixed device footprint, and loops that must not synchronise the device through an
 * allocation.  The call takes the grid description directly (ndim, n, L as in
 * vd_grid_create), the density rho and the physical fields in/out (n0 n1 n2 doubles each,
 * device, caller-owned; in and out must not alias), and allocates nothing: it calls no
 * cudaMalloc/cudaFree and no allocating library routine.  Every intermediate lives in one
 * fixed file-scope device array of 32 MiB, held by each GPU that loads the library until
 * the process exits; grids needing more (3D beyond about 64^3, 2D beyond 512 x 1024) are
 * rejected with VD_ERR_INVALID_ARG and a message giving the size.  The first call on a
 * device looks up the array's device address (once per device, with that device current):
 * make that first call before any stream capture.  The address is kept for the life of the
 * process, so the call must not be used across a cudaDeviceReset of that device.  All calls
 * share the array and it keeps the last call's contents, so calls whose kernels overlap on the
 * GPU race: serialise them.  rho must be positive and finite (VD_ERR_INVALID_ARG otherwise):
 * every call reads that check back to the host, so every call synchronises `stream` and
 * blocks the calling thread until the density has been checked.
 */
vd_status vd_apply_pressure_noalloc(int ndim, const int n[3], const double L[3], const double* rho, const double* in,
                                    double* out, vd_stream stream);

/*
 * Instrumentation (not part of the method; used by the benchmark to report achieved
 * bandwidth).  vd_launch_count: kernels launched by this library since it was loaded.
 * vd_profile_enable(1): bracket every transform-pass launch with CUDA events on its stream
 * and accumulate, per class, launches, elapsed ms, algorithmic bytes (every input and
 * output field once) and flops (5 n log2 n per complex line transform).  Classes:
 * 0 strided pass double, 1 strided pass float, 2 x pass double, 3 x pass float,
 * 5 strided pass float-pair, 6 x pass float-pair, 7 Krylov vector kernels on float vectors,
 * 8 Krylov vector kernels on double vectors (4: unused).
 * vd_profile_enable(2): span mode: only each inner float Krylov solve of a mixed-precision
 * refinement sweep is bracketed (two events), with the algorithmic bytes and flops of every
 * launch inside it, into class 9; individual launches are not timed.
 * vd_profile_enable(0) turns profiling off; other values are INVALID_ARG.
 * vd_profile_read synchronises on the recorded events; vd_profile_reset clears the totals.
 */
long long vd_launch_count(void);
/* Measured arithmetic rate of the current GPU (flop/s, an FMA or a float-pair multiply-add
 * counted as 2 flops): kind 0 FP64 FMA, 1 FP32 FMA, 2 float-pair multiply + add.  Eight
 * independent dependency chains per thread, 8 blocks of 256 threads per SM, best of three
 * launches timed with CUDA events on `stream` (synchronised).  The denominators of the
 * ALU-bound rooflines (double and float-pair transform passes). */
vd_status vd_alu_rate(int kind, double* flops_per_s, vd_stream stream);
vd_status vd_profile_enable(int on);
vd_status vd_profile_reset(void);
vd_status vd_profile_read(int cls, long long* launches, double* ms, double* alg_bytes, double* alg_flops);

#ifdef __cplusplus
}
#endif

#endif /* VD_H_ */
