/*
 * libibm: GB300 (sm_103a) implementation of one fractional time step of the
 * discrete-forcing immersed-boundary solver of Sundar, Majumdar, Shah &
 * Sarkar, "Massive parallelization and performance enhancement of an
 * immersed boundary method based unsteady flow solver", arXiv 2402.17337.
 *
 * The paper's problem (Sec. 2.1-2.3): 2-D incompressible laminar flow past
 * a rigid elliptic foil of thickness/chord t/c that plunges sinusoidally,
 * y = h sin(k t), ydot = k h cos(k t) (Eqs. 1-2), governed by the
 * non-dimensional Navier-Stokes equations with momentum forcing f and mass
 * source q (Eqs. 3-4), on a Cartesian staggered grid that is uniform where
 * the body moves and stretched geometrically outward (Sec. 2.3), advanced
 * by a semi-implicit fractional step (Adams-Bashforth convection,
 * Crank-Nicolson diffusion) whose velocity and pressure-correction systems
 * are solved by red-black Gauss-Seidel SOR (Sec. 2.2, Sec. 3.1).
 *
 * Units are non-dimensional: chord, free-stream speed and density are 1.
 *
 * Conventions of every entry point:
 *   - return IBM_OK (0) on success, a negative IBM_E_* code otherwise; the
 *     message of the last failure on the calling thread is returned by
 *     ibm_last_error();
 *   - the context owns all of its device memory; host buffers passed in are
 *     owned by the caller and are only read or written during the call;
 *   - fields cross the boundary in a compact row-major layout, x fastest:
 *       u  (nx+1) x ny   u[j*(nx+1)+i] at (x_f[i], y_c[j])
 *       v  nx x (ny+1)   v[j*nx+i]     at (x_c[i], y_f[j])
 *       p  nx x ny       p[j*nx+i]     at cell centres
 *   - all GPU work of a context runs on the stream given at creation (or on
 *     a stream the context creates); calls that return host data wait for it.
 */
#ifndef IBM_H_
#define IBM_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IBM_OK 0
#define IBM_E_INVAL (-1)    /* bad argument or state */
#define IBM_E_CUDA (-2)     /* a CUDA call failed */
#define IBM_E_NOCONV (-3)   /* an SOR solve hit max_sweeps before its tolerance */
#define IBM_E_DIVERGED (-4) /* a residual norm became NaN or Inf */
#define IBM_E_TIMEOUT (-5)  /* a bounded device-side wait gave up */

typedef struct ibm_ctx ibm_ctx;

/* Grid, flow and solver parameters (Sec. 2.1-2.3).
 *   x0,x1,y0,y1  rectangular domain; the paper uses [-7.5,24] x [-12.5,12.5]
 *   nx,ny        number of cells (>= 4 each, ny <= 8192)
 *   hmin         <= 0: uniform grid; otherwise the spacing of the uniform block
 *                ubox = [bx0,bx1] x [by0,by1]; outside it the spacing grows
 *                geometrically to the domain edge (Sec. 2.3)
 *   bc           0: inflow u = u_in, v = 0 at x0, convective outflow at x1,
 *                   free-slip walls at y0,y1;  1: free-slip walls all round
 *   Re, dt       Reynolds number and time step
 *   precision    0: FP64 throughout;  1: FP32 SOR sweeps inside FP64 defect
 *                correction (residuals, updates, norms and forces in FP64);
 *                2: as 1 with an FP32 inner solver of geometric multigrid
 *                (a variant; the paper's solver is SOR, Sec. 2.2): flexible
 *                conjugate gradients preconditioned by one V(2,2)-cycle per
 *                iteration; the stretched grid is coarsened by merging cell
 *                pairs, every level carries the five-point operator
 *                rediscretised from its faces, residuals are restricted as
 *                volume-weighted averages, corrections prolonged bilinearly,
 *                smoothing is red-black Gauss-Seidel, the coarsest level
 *                (<= 64 cells) is solved by SOR; the same FP64 stopping rule;
 *                sweeps_p then counts V-cycles
 *   poisson_tol  the pressure solve stops when
 *   poisson_rtol ||b - L_p phi||_inf <= max(poisson_tol, poisson_rtol*||b||_inf);
 *                the divergence left in fluid cells is dt times that residual
 *   helm_tol     velocity solves stop when their residual <= helm_tol
 *   check_every_p, check_every_h  residual checked every m full sweeps (<=0: 8, 2)
 *   max_sweeps   cap per solve (<= 0: 1000000)
 *   omega_p      SOR factor of the pressure solve (<= 0: 2/(1+sin(pi/max(nx,ny))))
 *   omega_h      SOR factor of the velocity solves (<= 0: 1)
 *   cuda_stream  cudaStream_t to run on, or NULL for a stream owned by the context */
typedef struct {
  double x0, x1, y0, y1;
  int nx, ny;
  double hmin;
  double ubox[4];
  int bc;
  double u_in;
  double Re, dt;
  int precision;
  double poisson_tol, poisson_rtol, helm_tol;
  int check_every_p, check_every_h;
  int max_sweeps;
  double omega_p, omega_h;
  void* cuda_stream;
} ibm_grid_params;

/* Statistics of one step. */
typedef struct {
  int n;                 /* steps completed */
  double t;              /* time after the step */
  int sweeps_u, sweeps_v, sweeps_p;  /* sweeps per solve (precision 2: sweeps_p counts V-cycles) */
  double res_u, res_v, res_p;
  double div_max;        /* max |div u| over cells whose centre is in the fluid */
  double cl, cd;         /* lift and drag coefficients of the step */
} ibm_step_stats;

/* Builds the grid (Sec. 2.3), allocates the fields on the device, zero
 * interior flow with u = u_in on the inflow face.  *out receives the context.
 * Errors: IBM_E_INVAL for inconsistent parameters, IBM_E_CUDA. */
int ibm_create_grid(const ibm_grid_params* params, ibm_ctx** out);

/* Places an elliptic body (Sec. 2.1): chord along x, semi-axes chord/2 and
 * thickness_ratio*chord/2 (1 = circle), centre (xc, yc + h sin(k t)),
 * plunge velocity k h cos(k t) (Eqs. 1-2).  h = 0 gives a fixed body.
 * Must come before the first step; fails with IBM_E_INVAL otherwise or when
 * the body's swept region does not fit inside the grid. */
int ibm_set_body(ibm_ctx* ctx, double chord, double thickness_ratio, double h, double k, double xc,
                 double yc);

/* Advances nsteps fractional steps (Sec. 2.2): classification of the nodes
 * at t^{n+1}, explicit predictor, implicit velocity solves with the forcing
 * rows, right-hand side with the mass source, pressure solve, projection,
 * forces.  *last (may be NULL) receives the statistics of the last step.
 * On IBM_E_NOCONV / IBM_E_DIVERGED the failing step is not counted. */
int ibm_step(ibm_ctx* ctx, int nsteps, ibm_step_stats* last);

/* Copies the lift and drag histories (one entry per completed step) into
 * cl and cd (either may be NULL), at most cap entries; *n_out = steps done. */
int ibm_forces(const ibm_ctx* ctx, double* cl, double* cd, int cap, int* n_out);

/* Field ids for ibm_get_field / ibm_set_field. */
#define IBM_U 0
#define IBM_V 1
#define IBM_P 2
#define IBM_PHI 3   /* last pressure increment (gauge cell zero) */
#define IBM_B 4     /* last Poisson right-hand side */
#define IBM_UHAT 5  /* last intermediate velocity */
#define IBM_VHAT 6
#define IBM_RU 7    /* last explicit right-hand side of the u system */
#define IBM_RV 8
#define IBM_HU 9    /* last convective term div(u u) */
#define IBM_HV 10
#define IBM_Q 11    /* last mass source */

/* Copies field `which` into host (n must equal the field's size). */
int ibm_get_field(const ibm_ctx* ctx, int which, double* host, size_t n);

/* Overwrites u, v, p or phi from host (n must equal the field's size). */
int ibm_set_field(ibm_ctx* ctx, int which, const double* host, size_t n);

/* Classification of the last step: grid 0 = u nodes, 1 = v nodes (kind
 * 0 fluid, 1 solid, 2 forcing; dir = side of the wall 0 -x, 1 +x, 2 -y, 3 +y;
 * alpha = interpolation weight), grid 2 = cells (1 = centre inside the body;
 * dir and alpha unused).  Full field size n, any of the pointers may be NULL. */
int ibm_get_flags(const ibm_ctx* ctx, int grid, unsigned char* kind, unsigned char* dir, double* alpha,
                  size_t n);

/* Face coordinates x_f (nx+1) and y_f (ny+1). */
int ibm_get_grid(const ibm_ctx* ctx, double* xf, double* yf);

/* Solves L_p phi = b (homogeneous Neumann) by red-black SOR on the
 * context's grid, as inside a step (Sec. 2.2), to
 * ||b - L_p phi||_inf <= tol checked every check_every sweeps (precision 1:
 * FP32 sweeps inside FP64 defect correction, checked in FP64 after whole
 * launches of the tuned tile, so sweep counts and the max_sweeps cap are
 * rounded up to a multiple of the sweeps per launch; check_every is the
 * length of the first run of FP32 sweeps, later runs adapt to the observed
 * convergence rate), then shifts
 * phi so that the cell (nx-1, 0) is zero.  b_dev, phi_dev: device pointers
 * to nx*ny doubles in the compact layout; phi_dev holds the initial guess
 * and receives the result (on IBM_E_NOCONV: the last iterate, unshifted).
 * Uses the context's work arrays, so it must not
 * overlap a step of the same context.  *sweeps and *res (may be NULL)
 * receive the sweep count and the final residual norm. */
int ibm_poisson_solve(ibm_ctx* ctx, const double* b_dev, double* phi_dev, double tol, int check_every,
                      int max_sweeps, int* sweeps, double* res);

/* Pressure solve for callers that cannot allocate device memory.
 *
 * No counterpart in the paper: this is a packaging variant of
 * ibm_poisson_solve for callers that cannot call cudaMalloc, such as an
 * application whose device memory belongs to its own allocator or to a pool
 * sized up front, a framework that forbids allocation on its hot path, or a
 * real-time loop that cannot take the device-wide synchronisation an
 * allocation may cause.  It needs no context: the caller passes the grid's
 * face coordinates and its own buffers, and every scratch value (the 1-D
 * coefficients and the residual-norm accumulator) lives in one fixed-size
 * static device array of the library, which each GPU that loads the library
 * holds (256 KB) until the process exits.
 *
 * Solves L_p phi = b on the grid with face coordinates xf (nx+1 host
 * doubles) and yf (ny+1 host doubles), homogeneous Neumann, by red-black SOR
 * with factor omega, checking ||b - L_p phi||_inf <= tol every check_every
 * sweeps (<= 0: 8), at most max_sweeps sweeps (<= 0: 1e6), then shifts phi
 * so that cell (nx-1, 0) is zero; the iterates equal those of
 * ibm_poisson_solve on an FP64 (precision 0) context of the same grid (the
 * mixed and multigrid contexts iterate differently).  xf and yf must
 * increase strictly (IBM_E_INVAL otherwise).  b_dev and phi_dev are device pointers
 * to nx*ny doubles in the compact layout; phi_dev holds the initial guess
 * and receives the result.  stream is a cudaStream_t (NULL: the default
 * stream); the call returns after the stream has finished its work.
 * *sweeps and *res (may be NULL) receive the sweep count and final residual.
 *
 * Limits and sharing: nx and ny must be at most 8192, larger sizes fail
 * with IBM_E_INVAL and a message in ibm_last_error().  The first call on a
 * device performs a one-time set-up: it looks up the device address of the
 * scratch array (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture begins.  Every call on a device uses
 * the same scratch array, which keeps the last call's contents; each call
 * clears what it needs before use.  Calls whose GPU work overlaps (two host
 * threads, or two streams of one device) race on the scratch: serialise them. */
int ibm_poisson_solve_noalloc(int nx, int ny, const double* xf, const double* yf, const double* b_dev,
                              double* phi_dev, double omega, double tol, int check_every, int max_sweeps,
                              void* stream, int* sweeps, double* res);

/* Counters of a context.  With profiling on, each run of pressure SOR
 * launches between two residual checks is bracketed by CUDA events on the
 * context's stream; sweep_ms is the summed device time of those runs and
 * sweep_launches the number of launches they contain. */
typedef struct {
  long long launches;        /* kernels launched by this context */
  long long sweep_launches;  /* pressure SOR sweep launches inside timed runs */
  double sweep_ms;           /* device time of those runs */
  long long steps;           /* steps completed */
  long long poisson_sweeps;  /* pressure sweeps over all steps */
  long long helm_sweeps;     /* velocity sweeps over all steps (u and v) */
  int sor_shape[3];          /* FP32 sweep tile chosen by the autotuner: rows per tile,
                                half-sweeps per launch, thread rows (0 if not tuned) */
  double sor_us_per_sweep;   /* its measured time per full sweep, microseconds */
  long long sweep_cells;     /* cells covered by the timed sweep launches, summed over launches */
  int sor_form;              /* form of that sweep kernel (3 to 7; 0 if not tuned) */
  long long ws_applied;      /* steps that evaluated the learned warm start */
  long long ws_kept;         /* of those, steps whose learned guess had the smaller residual and was kept */
  int sor_index;             /* index of that shape for ibm_set_sor_shape (-1 if not tuned) */
} ibm_profile;

/* Autotuner of the FP32 sweep kernel (precision 1): times each tile shape on
 * this context's grid and keeps the fastest per sweep.  Runs by itself
 * before the first mixed-precision solve; calling it re-tunes.  A no-op for
 * precision 0.  Uses the context's work arrays: not during a step. */
int ibm_tune(ibm_ctx* ctx);

/* Tile shapes of the FP32 sweep kernel: their number, and a fixed choice
 * for the context (index 0 .. n-1; -1 returns to the autotuner on the next
 * mixed-precision solve).  Every shape performs the same red-black SOR
 * iterates; they differ in speed only. */
int ibm_sor_num_shapes(void);
int ibm_set_sor_shape(ibm_ctx* ctx, int index);

/* Relaxation factor of the pressure SOR (Sec. 2.2 leaves it free) from the
 * observed convergence: red-black SOR runs on the homogeneous pressure
 * system from a pseudo-random start until the residual has fallen by 1e-10
 * or `sweeps` sweeps have run (<= 0: 8 max(nx, ny), clamped to 2048..32768),
 * the asymptotic rate rho over the second half at the context's omega gives
 * the Jacobi spectral radius through Young's relation for consistently
 * ordered matrices, and the optimum 2 / (1 + sqrt(1 - mu^2)) replaces omega
 * if a second run confirms a faster rate.  The optimum depends on the grid
 * only (stretching included), not on the flow.  *omega receives the factor in
 * use.  Uses temporary device memory and the context's stream; not during a
 * step.  FP64 sweeps whatever the precision. */
int ibm_tune_omega(ibm_ctx* ctx, int sweeps, double* omega);

/* Young's relation as used by ibm_tune_omega: the optimal relaxation factor
 * given the convergence factor per sweep rho observed at omega (omega itself
 * when rho <= omega - 1, i.e. omega at or above the optimum).  Host only. */
double ibm_omega_from_rate(double omega, double rho);

/* Turns the event timing of pressure sweeps on (1) or off (0); counters are
 * reset.  Timing adds one event pair per run of sweeps. */
int ibm_set_profiling(ibm_ctx* ctx, int on);

/* Copies the counters. */
int ibm_get_profile(const ibm_ctx* ctx, ibm_profile* out);

/* ---------------------------------------------------------------- U-Net
 * Learned warm start of the pressure solve: a 4-level convolutional U-Net
 * with BF16 weights and activations and FP32 accumulation (tensor cores),
 * trained on the GPU by the library's own forward and backward kernels on
 * samples the solver generates.  widths: channels of the four levels
 * (multiples of 16).  Inputs are 4 FP32 feature channels [H][W][4], the
 * output one FP32 channel [H][W]; H and W must be multiples of 8.  Device
 * pointers; stream may be NULL.  The network owns its device memory
 * (ibm_unet_create allocates the parameters, ibm_unet_destroy frees all);
 * activation buffers are allocated by the first forward or training step
 * at a given H x W and reallocated when the size changes, so a size change
 * must not happen while a stream that uses the network is being captured.
 * The 3x3 convolutions of the forward pass and of the data gradient run on
 * the tcgen05 tensor cores (tensor-memory accumulators, TMA-loaded tiles);
 * their waits are bounded (about 2 s).  The BF16 weights are repacked for
 * those kernels on the stream after every change (creation, new parameters,
 * an Adam step), inside the next forward pass.
 * Errors: IBM_E_INVAL (widths not positive multiples of 16, n different
 * from ibm_unet_num_params, H or W not multiples of 8, NULL pointers),
 * IBM_E_CUDA, IBM_E_TIMEOUT (a convolution kernel gave up a bounded wait;
 * reported by the first forward or training call after it, and by every
 * later one: the device state is then suspect). */
typedef struct ibm_unet ibm_unet;
int ibm_unet_create(const int widths[4], unsigned long long seed, ibm_unet** out);
void ibm_unet_destroy(ibm_unet* net);
long long ibm_unet_num_params(const ibm_unet* net);
/* copies the FP32 master parameters to (set = 0) or from (set = 1) host */
int ibm_unet_params(ibm_unet* net, float* host, long long n, int set);
/* gradient of the last ibm_unet_train_step, to host */
int ibm_unet_grads(const ibm_unet* net, float* host, long long n);
int ibm_unet_forward(ibm_unet* net, const float* feat_dev, int H, int W, float* out_dev, void* stream);
/* one Adam step (apply = 1) on the mean squared error of output channel 0
 * against target_dev [H][W]; apply = 0 only computes the gradient.
 * *loss (may be NULL) receives the loss. */
int ibm_unet_train_step(ibm_unet* net, const float* feat_dev, const float* target_dev, int H, int W, float lr,
                        int apply, double* loss, void* stream);

/* Warm start of the pressure solve of each step (Sec. 2.2 solves it by SOR
 * from a starting guess): mode 0, the previous increment; mode 1, the
 * previous increment plus the U-Net's prediction of its change (the net is
 * borrowed, not owned), kept only if its residual ||b - L_p phi||_inf is
 * below half that of the previous increment (counted in ibm_profile);
 * mode 2, the previous increment and, every step, a training sample
 * recorded for ibm_get_sample.  The network works on the
 * grid coarsened 2x (nx, ny must be divisible by 16) with four features per
 * coarse cell (initial residual b - L_p phi^n, b, body-cell fraction, p^n,
 * each over its infinity norm) and predicts (phi^{n+1} - phi^n) / (s0 c_T),
 * s0 the norm of the residual feature and c_T = target_scale. */
int ibm_set_warmstart(ibm_ctx* ctx, int mode, ibm_unet* net, double target_scale);

/* Base guess of the warm start (any mode): 0, the previous increment
 * phi^n (default); 1, its linear extrapolation in time 2 phi^n - phi^{n-1}
 * (the history starts when the base is set: the first step after it uses
 * phi^n).  The learned form predicts the change from the base guess. */
int ibm_set_warmstart_base(ibm_ctx* ctx, int base);

/* Checkpoint and resume.  A state holds everything a step carries to the
 * next: u, v, p, the last pressure increment (the next solve's start), the
 * AB2 convection history, the momentum inside the body (the added-mass term
 * of the force), the C_l/C_d histories, the step count, the adapted inner
 * run lengths of the FP32 solves and, when the warm start extrapolates in
 * time, the increment before, and the FP32 sweep shape chosen by the
 * autotuner (its sweeps per launch round the inner runs).  ibm_state_bytes
 * gives the size of the context's state; ibm_save_state copies it into the
 * caller's host buffer of at least that size (waits for the stream).  ibm_load_state restores
 * one into a context created with the same grid, Re and dt, with the same
 * body set (and the same warm-start base); stepping on from it repeats the
 * saved run's steps bit for bit.  The layout is the library's own (native
 * byte order).  Errors: IBM_E_INVAL (small buffer, another format, grid,
 * dt, Re or body), IBM_E_CUDA. */
int ibm_state_bytes(const ibm_ctx* ctx, size_t* bytes);
int ibm_save_state(const ibm_ctx* ctx, void* host, size_t bytes);
int ibm_load_state(ibm_ctx* ctx, const void* host, size_t bytes);

/* Preconditioner of the FCG iteration of precision 2 (the multigrid
 * variant; a network used as preconditioner rather than warm start).
 * kind 0: one V(2,2)-cycle (default).  kind 1: a two-level cycle whose
 * coarse level is the U-Net: pre_smooth (0 or 1) launches of two red-black
 * Gauss-Seidel sweeps from zero, the residual restricted (volume-weighted)
 * to the 2x coarsened grid, there replaced by net's prediction from the
 * features of ibm_set_warmstart with channel 0 the restricted residual over
 * its infinity norm s (channels 1-3 taken when the solve starts), the
 * prediction times s * target_scale prolonged bilinearly, two
 * post-smoothing sweeps.  The FP64 defect correction and its tolerance are
 * unchanged, so the result meets the same residual bound whatever the
 * network predicts.  net stays owned by the caller and must outlive its use
 * here; nx and ny divisible by 16.  Errors: IBM_E_INVAL (precision not 2,
 * bad kind, missing net, sizes), IBM_E_CUDA. */
int ibm_set_preconditioner(ibm_ctx* ctx, int kind, ibm_unet* net, double target_scale, int pre_smooth);

/* Last recorded sample (mode 2): feat [Hc][Wc][4] and target [Hc][Wc]
 * (host, FP32); either may be NULL; *Hc, *Wc receive the coarse sizes. */
int ibm_get_sample(const ibm_ctx* ctx, float* feat, float* target, int* Hc, int* Wc);

/* ---------------------------------------------------------------- batch
 * Many independent cases (each a context of its own grid, body and
 * parameters, precision 1) advancing together; the paper runs one case at
 * a time, and this batching of cases has no counterpart in it.  Each step
 * of the batch is one step (Sec. 2.2) of every case: the parts before and
 * after the pressure solve run case by case, and the pressure solves of
 * all cases run as one defect-correction loop whose FP32 sweep launches and
 * FP64 residual launches each cover every case that has not converged yet
 * (cases leave the launches as they reach their tolerance).  The parts
 * before and after the pressure solve (classification, predictor, velocity
 * solves, right-hand side, forces, projection) run as shared launches over
 * all cases too, so the launches of a step do not grow with the number of
 * cases (cases with a learned or extrapolated warm start or a relative
 * pressure tolerance take those parts case by case).  The tile shape is
 * chosen for the whole batch by the autotuner on the first step; see
 * ibm_batch_set_budgets for the rounds of the pressure loop.
 *
 * The contexts are borrowed: they must outlive the batch and must not be
 * used by other calls while ibm_batch_step runs.  The batch owns a stream
 * of its own; a step waits for the work queued on the cases' streams and
 * the cases' streams wait for the step.  Between batch steps a case may be
 * read (ibm_get_field, ibm_forces) or stepped alone. */
typedef struct ibm_batch ibm_batch;

/* cases: n distinct contexts of precision 1.  IBM_E_INVAL otherwise. */
int ibm_batch_create(ibm_ctx* const* cases, int n, ibm_batch** out);

/* Advances every case by nsteps.  last (may be NULL): n entries receiving
 * the statistics of each case's last step.  On an error the message names
 * the case; the cases are then in an unspecified state. */
int ibm_batch_step(ibm_batch* batch, int nsteps, ibm_step_stats* last);

/* The batch's own stream (a cudaStream_t), for timing with events; NULL for
 * a NULL batch. */
void* ibm_batch_stream(const ibm_batch* batch);

/* A fixed FP32 sweep tile shape for the batch (index as for
 * ibm_set_sor_shape; -1: tuned over the batch on the next step). */
int ibm_batch_set_sor_shape(ibm_batch* batch, int index);

/* Sweep budgets of the batched pressure solve: on (1, the default), each
 * round of the defect-correction loop gives every active case the FP32
 * sweeps it predicts for itself (its CTAs skip the launches beyond them),
 * so the loop takes as many rounds as its slowest case, in direct
 * (programmatic dependent) launches; off (0), every active case takes the
 * shortest prediction of the round, and the sweep launches are replayed
 * from CUDA graphs (ibm_batch_set_graphs).  Either way each case stops at
 * its own tolerance; the iterates differ only in where the checks fall. */
int ibm_batch_set_budgets(ibm_batch* batch, int on);

/* CUDA-graph replay of the sweep launches when budgets are off: on (1, the
 * default) or off (0, direct launches of the same sweeps). */
int ibm_batch_set_graphs(ibm_batch* batch, int on);

/* Profiling of the batch (event timing of its sweep runs; counters of the
 * batch and of its cases are reset). */
int ibm_batch_set_profiling(ibm_batch* batch, int on);

/* Counters: launches (the batch's and its cases'), sweep launches and time
 * of the batched runs, steps, pressure sweeps summed over cases, velocity
 * sweeps summed over cases, the batch's tile shape and time per sweep of
 * the whole batch. */
int ibm_batch_get_profile(const ibm_batch* batch, ibm_profile* out);

/* Frees the batch (not its cases). */
void ibm_batch_destroy(ibm_batch* batch);

/* Frees the context and its device memory. */
void ibm_destroy(ibm_ctx* ctx);

/* Message of the last failure on this thread ("" if none). */
const char* ibm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IBM_H_ */
