/*
 * bem.h -- C ABI of the GB300 Laplace-domain elastodynamic BEM frequency-solve library.
 *
 * Method: Xiao, Rong, Ye, Zhang, "An efficient adaptive frequency sampling scheme for
 * large-scale transient boundary element analysis".  The library solves the frequency-domain
 * boundary integral equation of Sec. 2.1, Eq. (bie),
 *     c_ij u_j(x,s) + PV int_G T_ij(x,y,s) u_j(y,s) dG = int_G U_ij(x,y,s) t_j(y,s) dG,
 * discretised by constant-element collocation on flat triangles into A(s) a(s) = b(s)
 * (Eq. (Aa_b)), at many complex frequencies s = sigma + i omega at once, and post-processes the
 * responses by the Fourier series method (Sec. 2.2, Eq. (IDFT-MFT)), vector fitting
 * (Sec. 2.3, Eqs. (vf-f), (vf-td)) and adaptive frequency sampling (Sec. 3, Algorithm AFS).
 *
 * Conventions (all entry points):
 *  - Every function returns 0 (BEM_OK) on success or a negative BEM_ERR_* code; it never
 *    aborts the process.  bem_last_error() gives a one-line message for the last failure.
 *  - SI units.  Complex numbers are interleaved (re, im) IEEE doubles at the ABI.
 *  - Laplace variable s with time factor e^{st}; boundary data are a real spatial pattern times
 *    the Laplace transform of a time profile (BEM_PROFILE_STEP: 1/s, BEM_PROFILE_CONSTANT: 1).
 *  - Input arrays are copied; the caller keeps ownership.  Output arrays are written, never
 *    retained.  A pointer argument may be host memory or device memory of the context's device
 *    (detected with cudaPointerGetAttributes) unless the description says "host".
 *  - Mesh: triangles are counter-clockwise about their unit normal, and that normal points out
 *    of the elastic domain (into cavities, out of finite bodies).  Unknown ordering: element e
 *    owns entries 3e, 3e+1, 3e+2 (x, y, z) of every solution vector.
 *  - A context is bound to one CUDA device and one stream; calls on one context must not
 *    overlap in time (the context is not thread-safe).  All work runs on the context's stream;
 *    functions return after that work completes.
 */
#ifndef BEM_H
#define BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define BEM_OK 0
#define BEM_ERR_INVALID_ARG (-1)   /* bad pointer, size, value or call order              */
#define BEM_ERR_CUDA (-2)          /* a CUDA runtime call failed (message has the reason) */
#define BEM_ERR_NOT_CONVERGED (-3) /* tolerance not met within the iteration limits       */
#define BEM_ERR_OOM (-4)           /* device allocation failed                             */
#define BEM_ERR_BREAKDOWN (-5)     /* GMRES breakdown / NaN in an instance                 */
#define BEM_ERR_NO_MESH (-6)       /* operation needs bem_set_mesh first                   */

/* ------------------------------------------------------------------ enums */
#define BEM_BC_TRACTION 0      /* traction given, displacement unknown (Neumann)   */
#define BEM_BC_DISPLACEMENT 1  /* displacement given, traction unknown (Dirichlet) */

#define BEM_PROFILE_STEP 0     /* Laplace factor 1/s (Heaviside step in time)  */
#define BEM_PROFILE_CONSTANT 1 /* Laplace factor 1 (data already in s-domain)  */

#define BEM_PREC_FP64 0   /* plain FP64: FP64 operator, FP64 GMRES                            */
#define BEM_PREC_MIXED 1  /* FP32 operator + FP32-stored Krylov basis with FP64 dot products,
                             FP64 iterative refinement: every residual r = b - A x, with b
                             formed from the boundary data in the same sweep, is FP64        */
#define BEM_PREC_FP32 2   /* operator-only mode for bem_apply: FP32 far/near kernels          */

#define BEM_APPLY_A 0     /* y = A(s) x : the system operator of Eq. (Aa_b)                  */
#define BEM_APPLY_K 1     /* y = K(s) x : the operator acting on the known boundary data,
                             so that b(s) = K(s) (profile(s) * pattern)                       */

#define BEM_RESID_DF64 0  /* far and near field of the residual in float-float on the FP32 pipes */
#define BEM_RESID_FP64 1  /* far and near field of the residual in native FP64                 */

#define BEM_WARM_ZERO 0     /* GMRES starts from x0 = 0                                       */
#define BEM_WARM_NEAREST 1  /* x0 = alpha * the stored solution at the nearest frequency     */
#define BEM_WARM_MLP 2      /* x0 = a1 POD basis MLP(s) + a2 nearest stored solution, (a1, a2)
                               minimising |b - A x0| (network trained by bem_warm_train)       */
#define BEM_WARM_VF 3       /* inside bem_afs: x0 = a1 x_VF(s) + a2 nearest stored solution, x_VF
                               the rational prediction of every unknown from the current fit's
                               poles (residues identified over the stored solutions, Sec. 2.3);
                               elsewhere the nearest stored solution                           */
#define BEM_WARM_SWEEP 4    /* a frequency list of >= 8 is solved in two passes: every other
                               frequency from x0 = 0, then a vector fit of order J/2 to 8
                               unknowns of those J solutions, then the remaining frequencies
                               from the fit's rational prediction of every unknown combined with
                               the nearest solved frequency, as BEM_WARM_VF (uses and replaces
                               the context's warm-start memory); in bem_afs as BEM_WARM_VF     */

typedef struct bem_ctx bem_ctx;

typedef struct bem_options {
  int32_t precision;   /* BEM_PREC_FP64 or BEM_PREC_MIXED (default MIXED)                   */
  int32_t restart;     /* GMRES restart length m (default 50)                               */
  int32_t max_iters;   /* cap on GMRES iterations per inner solve (default 500)             */
  int32_t max_refine;  /* cap on FP64 refinement steps in MIXED mode (default 8); a frequency
                          whose refinement stalls (< 4x per step) or that exhausts the cap is
                          solved again in plain FP64 from x0 = 0                             */
  double tol;          /* target ||b - A x||_2 / ||b||_2, measured in FP64 (default 1e-6)   */
  double inner_tol;    /* relative reduction asked of each FP32 inner solve (default 1e-6,
                          the FP32 operator's error floor: a first solve relative to |b|,
                          later ones relative to the FP64-class residual; never below 0.8 tol
                          of |b| for a frequency's first inner solve, 0.5 tol for later ones) */
  int32_t warm_start;  /* BEM_WARM_* (default ZERO)                                          */
  int32_t reserved0[2]; /* zero                                                              */
  int32_t residual_mode; /* MIXED refinement residual: BEM_RESID_DF64 (default) or
                            BEM_RESID_FP64                                                    */
  int32_t reserved[6];
} bem_options;

typedef struct bem_solve_stats {
  int32_t* iterations;   /* [ns] total GMRES iterations per frequency (nullable)              */
  int32_t* refinements;  /* [ns] FP64 residual evaluations per frequency (nullable)           */
  double* residual;      /* [ns] final ||b - A x||_2/||b||_2, FP64 (nullable)                  */
  int32_t* status;       /* [ns] 0 converged, else BEM_ERR_NOT_CONVERGED / _BREAKDOWN (null.)  */
  double seconds;        /* out: wall time of the call                                         */
  int64_t fp32_operator_applies; /* out: batched FP32 operator launches (far + near)          */
  int64_t fp64_operator_applies; /* out: batched FP64 operator launches                       */
  int64_t kernel_launches;       /* out: kernels of this library launched by the call        */
} bem_solve_stats;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to run on (the
 * caller keeps it alive), or NULL for a stream the context creates and owns.
 * Errors: INVALID_ARG (out NULL, device out of range), CUDA. */
int bem_create(bem_ctx** out, int device, void* cuda_stream);

/* Release every device and host resource of the context (NULL is a no-op). */
int bem_destroy(bem_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed bem_create if ctx is NULL).
 * The string stays valid until the next call on the same context. */
const char* bem_last_error(const bem_ctx* ctx);

/* Fill *opt with the defaults listed in bem_options. */
int bem_default_options(bem_options* opt);
int bem_set_options(bem_ctx* ctx, const bem_options* opt);

/* ------------------------------------------------------------------ problem statement */

/* Boundary mesh (Sec. 2.1: the boundary G partitioned into n_e triangles).
 * verts: nv x 3 doubles (host); tris: ne x 3 int32 vertex indices (host).
 * Builds on the device the element geometry (centroid collocation points, unit normals,
 * areas, longest edges, 4- and 7-point quadrature points) and the near-source lists
 * (|x_i - c_e| < 2 h_e).  Clears boundary conditions and cached frequency data.
 * Errors: INVALID_ARG (sizes <= 0, index out of range, degenerate triangle), OOM, CUDA. */
int bem_set_mesh(bem_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t ne);

/* Isotropic material (Sec. 2.1): shear modulus mu [Pa], Poisson ratio nu, density rho.
 * Errors: INVALID_ARG (mu <= 0, rho <= 0, nu outside (-1, 0.5)). */
int bem_set_material(bem_ctx* ctx, double mu, double nu, double rho);

/* Boundary conditions (Sec. 2.1, the columns of Eq. (Aa_b)): bc_type[ne] (host, int8,
 * BEM_BC_*), bc_value[ne x 3] (host, doubles: the given traction [Pa] or displacement [m]
 * pattern per element), time_profile BEM_PROFILE_*.
 * Errors: INVALID_ARG (NULL, unknown type/profile), NO_MESH. */
int bem_set_bc(bem_ctx* ctx, const int8_t* bc_type, const double* bc_value, int time_profile);

/* ------------------------------------------------------------------ the frequency solve */

/* Solve A(s_k) a(s_k) = b(s_k) for every frequency s_k (Sec. 2.1, Eq. (Aa_b)), all frequencies
 * batched: matrix-free operator (far field by 4-point quadrature evaluated on the fly, near
 * sources by the 7-point rule, the own element by Duffy + CPV), right block-Jacobi
 * preconditioned GMRES(m), and in MIXED mode FP64 iterative refinement around FP32 inner
 * solves.
 * s: 2 x ns doubles (re, im interleaved, Re s > 0).  x_out: ns x 3ne complex (interleaved
 * doubles), host or device, nullable (then only statistics are produced).
 * Returns NOT_CONVERGED if some frequency missed opt.tol (its status says which); x_out is
 * still written with the best iterate.  Errors: INVALID_ARG, NO_MESH, OOM, CUDA. */
int bem_solve_frequencies(bem_ctx* ctx, const double* s, int64_t ns, double* x_out,
                          bem_solve_stats* stats);

/* Several independent problems in one call: item k solves its context's problem (mesh,
 * material, boundary data and options, set beforehand) at its own ns frequencies s[ns]
 * (complex), with x_out and stats as for bem_solve_frequencies.  The paper solves one problem
 * at a time; batching uneven problems is this library's, to keep the GPU busy when the
 * problems are small.  Up to max_workers host threads (0: one per item) each drive one
 * context through bem_solve_frequencies on that context's own stream, largest problem
 * (ne^2 x ns) first, so kernels of different problems run side by side on the GPU.  Every
 * item needs a distinct context; contexts created with separate streams (the default) run
 * concurrently, contexts sharing a caller stream run one after another.  Out: items[k].status =
 * that solve's return code.  Returns BEM_OK when every item succeeded, else the first failing
 * code (an error other than BEM_ERR_NOT_CONVERGED takes precedence); INVALID_ARG for a null or
 * repeated context or an empty frequency list (nothing is run). */
typedef struct bem_batch_item {
  bem_ctx* ctx;
  const double* s;         /* [ns] complex frequencies (host or device)                  */
  int64_t ns;
  double* x_out;           /* [ns x 3ne] complex (host or device), nullable               */
  bem_solve_stats* stats;  /* nullable                                                     */
  int32_t status;          /* out                                                          */
} bem_batch_item;

int bem_solve_batch(bem_batch_item* items, int32_t n, int32_t max_workers);

/* ------------------------------------------------------------------ time domain (FSM) */

/* Fourier-series-method inverse Laplace transform (step a9; Sec. 2.2, Eqs. (invLap),
 * (IDFT-MFT)), FP64:
 *   out[j][d] = e^{eta t_j}/P [ W_0 Re h_0 + 2 Re sum_{k=1}^{nc-2} W_k h_k e^{i k w t_j}
 *                               + W_{nc-1} Re(h_{nc-1} e^{i (nc-1) w t_j}) ],  w = 2 pi / P,
 * from samples h[k][d] = h_d(eta + i k w), k = 0 .. nc-1 (N_s = 2 (nc - 1) points of the
 * period P; the other half of the spectrum is the complex conjugate).  W_k = Hanning
 * (1 + cos(2 pi k / N_s)) / 2 when window = 1, else 1.  The 1/P factor of the trapezoidal rule,
 * absent from the printed equation, is included; any t is allowed (not only multiples of P/N_s).
 * h: nc x m complex (interleaved), t: nt doubles, out: nt x m doubles; host or device.
 * Errors: INVALID_ARG (nc < 2, m < 1, nt < 1, P <= 0, nc > 12800). */
int bem_fsm_eval(bem_ctx* ctx, const double* h, int64_t nc, int64_t m, double eta, double period,
                 const double* t, int64_t nt, int window, double* out);

/* Frequency-domain approach with the FSM (Sec. 2.2): solves the BEM system at the nc
 * frequencies s_k = eta + i k 2 pi / P (one batched bem_solve_frequencies) and returns the time
 * responses of the requested unknowns at the times t (Hanning window).
 * dofs: ndofs int64 indices into the 3 ne unknowns (host or device); resp_out: nt x ndofs
 * doubles (host or device); stats: as for bem_solve_frequencies (arrays of length nc), nullable.
 * A benchmark grid written s_k = sigma + i k pi / T is this grid with P = 2 T. */
int bem_fsm(bem_ctx* ctx, double period, double eta, int64_t nc, const double* t, int64_t nt,
            const int64_t* dofs, int64_t ndofs, double* resp_out, bem_solve_stats* stats);

/* ------------------------------------------------------------------ allocation-free variant */

/* bem_fsm_eval without any device allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run (a component confined
 * to a fixed memory budget or to buffers handed to it by its host application, or a loop that
 * must not stall on the device-wide synchronisation a cudaMalloc can cause) and therefore
 * cannot create a bem_ctx.
 * Same arithmetic and arguments as bem_fsm_eval, except: h, t and out must be device memory of
 * the calling thread's current device; cuda_stream is the cudaStream_t to run on (NULL = the
 * default stream); the call returns after the work completes.  Its only working memory is a
 * fixed array of BEM_NOALLOC_FSM_TABLE complex doubles (4 MiB) that the library keeps on every
 * device it is loaded on until the process exits, so nt * nc must not exceed
 * BEM_NOALLOC_FSM_TABLE (INVALID_ARG with a message otherwise).  The first call on a device
 * looks up that array's device address, so make it before any stream capture.  All calls share
 * the array: calls that overlap on the GPU race.  Errors: INVALID_ARG (sizes, host pointers,
 * pointers of another device), CUDA; the message is returned by bem_noalloc_last_error(), which
 * keeps one message per calling thread (valid until that thread's next failing call). */
#define BEM_NOALLOC_FSM_TABLE 262144
int bem_fsm_eval_noalloc(const double* h, int64_t nc, int64_t m, double eta, double period,
                         const double* t, int64_t nt, int window, double* out, void* cuda_stream);
const char* bem_noalloc_last_error(void);

/* ------------------------------------------------------------------ learned warm start (a8) */

/* The warm start gives each new frequency solve an initial guess built from solutions already
 * computed (the paper's adaptive sampling solves one new frequency at a time next to solved
 * ones; the warm start itself is not in the paper).  Both modes first pick a direction x^:
 * BEM_WARM_NEAREST the stored solution at the nearest stored frequency; BEM_WARM_MLP
 * x^ = Phi c(s), Phi = the leading left singular vectors (POD) of the stored solutions, c(s)
 * predicted by a 2 -> 128 -> 128 -> 2r MLP (tanh-GELU) trained on the directions of the stored
 * coefficient vectors Phi^H x (unit norm, leading entry real and non-negative); its dense layers
 * run on the tensor cores (FP16 operands, FP32 accumulation), the rest in FP32.  The solve then
 * scales the direction by the complex alpha minimising |b - alpha A x^| (one operator product,
 * which also gives the initial residual), so |r0| <= |b|.  BEM_WARM_MLP combines the learned
 * direction with the nearest stored solution: x0 = a1 x^_MLP + a2 x^_nearest with the (a1, a2)
 * minimising |b - A x0| (two operator products), never worse than either direction alone.  The
 * GMRES tolerance is unchanged: the warm start changes the iteration count, never the accepted
 * accuracy. */
typedef struct bem_warm_params {
  int32_t r_max;    /* POD rank cap (32)                                               */
  double energy_tol; /* POD energy cut: drop modes holding <= energy_tol of sum sigma^2 (1e-10) */
  int32_t steps;    /* Adam steps (2000)                                               */
  double lr;        /* Adam learning rate (1e-3; beta1 0.9, beta2 0.999, eps 1e-8)      */
  uint64_t seed;    /* weight initialisation (uniform +-1/sqrt(fan_in), zero biases)    */
  int32_t reserved[4];
} bem_warm_params;

typedef struct bem_warm_stats {
  int32_t r;             /* out: POD rank                                    */
  int32_t n_snapshots;   /* out: stored solutions used                       */
  double loss_first, loss_last; /* out: training loss at the first/last step */
  double seconds;        /* out                                              */
} bem_warm_stats;

int bem_default_warm_params(bem_warm_params* p);

/* Add ns solutions x[ns x 3ne] complex (host or device) at frequencies s[ns] (host) to the
 * context's warm-start memory (FP64 device copies; at most 256 are used for training). */
int bem_warm_store(bem_ctx* ctx, const double* s, int64_t ns, const double* x);
/* Forget every stored solution and the trained model. */
int bem_warm_clear(bem_ctx* ctx);
/* POD of the stored solutions, then MLP training on the device.  stats nullable.
 * Errors: INVALID_ARG (fewer than 2 or more than 256 stored solutions). */
int bem_warm_train(bem_ctx* ctx, const bem_warm_params* p, bem_warm_stats* stats);
/* The trained POD basis: phi[r x 3ne] complex (host or device, NULL to query r). */
int bem_warm_basis(bem_ctx* ctx, double* phi, int32_t* r);
/* The warm-start direction x^(s) a solve would start from (before its minimal-residual scaling),
 * for ns frequencies s[ns] (complex, host or device): x_out[ns x 3ne] complex (host or device).
 * mode: BEM_WARM_NEAREST (needs stored solutions) or BEM_WARM_MLP (needs bem_warm_train).
 * Errors: INVALID_ARG (other mode, nothing stored or trained, or stored for another mesh). */
int bem_warm_predict(bem_ctx* ctx, int32_t mode, const double* s, int64_t ns, double* x_out);
/* One MLP pass with caller parameters (verification): params (host, float, the layout
 * W1[128x2], b1[128], W2[128x128], b2[128], W3[2r x 128], b3[2r], row-major), inputs U[B x 2],
 * targets T[B x 2r] (nullable: forward only).  Outputs (host): y[B x 2r]; grads[nparams] and
 * *loss (L = sum |y - T|^2 / (2B)) when T is given. */
int bem_mlp_eval(bem_ctx* ctx, int32_t r, const float* params, const float* U, int32_t B,
                 const float* T, float* y, float* grads, double* loss);

/* ------------------------------------------------------------------ vector fitting + AFS */

/* Vector fit (step a10; Sec. 2.3, Eq. (vf-f)) on the host, FP64: f_k(s) ~ sum_m r_km/(s - a_m)
 * with common poles, fitted to K responses sampled at J frequencies.  Pole identification uses
 * the responses listed in fit_cols (NULL = all), starting from pairs -b/100 +- i b with b
 * equally spaced over (0, omega_max] (and -omega_max/100 when M is odd), n_iter relocations
 * (stopping early when the poles move less than 1e-10 omega_max); unstable poles are kept.
 * s: J complex (host); F: J x K complex row-major (host).  Outputs (host): poles[M] complex,
 * conjugate pairs adjacent; residues[K x M] complex.  Errors (bem_last_error(NULL)):
 * INVALID_ARG (M > J, sizes), BREAKDOWN (eigenvalue iteration failed). */
int bem_vf_fit(const double* s, int64_t J, const double* F, int64_t K, const int32_t* fit_cols,
               int32_t n_fit_cols, int32_t M, double omega_max, int32_t n_iter, double* poles,
               double* residues);
/* The fitted responses at n complex frequencies: out[n x K] complex (host). */
int bem_vf_eval(const double* poles, int32_t M, const double* residues, int64_t K, const double* s,
                int64_t n, double* out);
/* Time responses, Eq. (vf-td): out[nt x K] = sum over poles with Re a_m < eta of r_km e^{a_m t}
 * (the inverse Laplace transform of r/(s - a) is r e^{a t}; the printed exponent sign is read
 * as a misprint).  eta: abscissa of the line the samples were taken on -- the Bromwich contour
 * of Eq. (invLap) collects the residues of the poles to its left only; pass +inf to sum all. */
int bem_vf_time(const double* poles, int32_t M, const double* residues, int64_t K, const double* t,
                int64_t nt, double eta, double* out);

typedef struct bem_afs_params {
  double eta;        /* Re s of every sample (Sec. 2.2: eta = kappa ln(10) / T)          */
  double omega_max;  /* frequency band [0, Omega_s]                                       */
  double T;          /* time window of the E1 integrals (Eq. (stop-E1))                   */
  double alpha_H, alpha_L; /* fit orders M = floor(J / alpha) (Eq. (fit-ords); 2.0, 2.3) */
  double E1bar, E2bar;     /* convergence thresholds (Eq. (converge); 1e-4, 2e-3)        */
  int32_t J0;        /* initial Chebyshev frequencies (16)                                */
  int32_t Jc;        /* validation steps after the first converged one (3)                */
  int32_t n_grid;    /* uniform search grid for s_new over [0, Omega_s] (4096)            */
  int32_t nt;        /* time points of the E1 integrals (512)                             */
  int32_t max_samples; /* cap on N_c (400)                                                */
  int32_t vf_iters;  /* pole relocations per fit (20)                                     */
  int32_t batch;     /* new frequencies per step (1: the paper's algorithm).  b > 1 (a
                        variant, to keep the GPU batched): the paper's s_new, then further
                        argmaxes of the same discrepancy curve after masking +-Omega/(2J)
                        around each pick, kept while >= 0.1 of the first; solved together    */
  int32_t warm_retrain; /* with the context's warm_start = BEM_WARM_MLP: retrain the network
                        once this many samples have been added since its last training
                        (0: 4).  Ignored for the other warm-start modes                       */
  int32_t reserved[4];
} bem_afs_params;

typedef struct bem_afs_stats {
  int64_t capacity;  /* in: entries available in each array below                          */
  double* s;         /* [capacity] complex: sampled frequencies in sampling order (null.) */
  int32_t* gmres_iters; /* [capacity] GMRES iterations of each sample's solve (nullable)   */
  double* E1;        /* [capacity] E1 per AFS step (nullable)                             */
  double* E2;        /* [capacity] E2 per AFS step (nullable)                             */
  double* poles;     /* [capacity] complex: poles of the final M_H fit (nullable)         */
  int64_t n_samples; /* out: N_c                                                          */
  int64_t n_steps;   /* out: AFS steps (entries written to E1 / E2)                       */
  int32_t n_poles;   /* out: order of the final fit                                       */
  double seconds_solve, seconds_fit; /* out: time in BEM solves / in fitting             */
  double seconds_train;     /* out: time spent training the warm-start network            */
  int32_t warm_trainings;   /* out: trainings of the warm-start network                   */
  int32_t warm_learned_gains; /* out: MLP- or VF-start solves whose combined start left an initial
                               residual at least 10 % below the nearest stored solution's alone */
} bem_afs_stats;

/* Fill *p with the paper's parameter values (Sec. 3.4) and the defaults above; eta,
 * omega_max and T must still be set. */
int bem_default_afs_params(bem_afs_params* p);

/* Adaptive frequency sampling (Sec. 3, Algorithm AFS): starting from J0 Chebyshev frequencies,
 * repeatedly fits the observation responses (ORFs: unknowns orf[K]) at two orders, solves the
 * BEM system (one batched GPU solve, the context's options) at the frequency where the fits
 * disagree most, and stops when the time-domain change E1 and the fit discrepancy E2 of the
 * test unknowns test[Kt] stay below their thresholds for Jc + 1 consecutive steps.
 * Warm start: when the context's warm_start option is BEM_WARM_NEAREST, BEM_WARM_MLP or BEM_WARM_VF, the call
 * first clears the warm-start memory, then stores every solution it computes (up to 256) and so
 * starts each new frequency's GMRES from the solutions already sampled; with BEM_WARM_MLP it
 * trains the network (default bem_warm_params) after the initial frequencies and again every
 * params->warm_retrain new samples; each learned start is combined with the nearest stored
 * solution (see BEM_WARM_MLP); with BEM_WARM_VF each new frequency's start combines the nearest
 * stored solution with the prediction of the step's order-M_H fit: the residues of every
 * unknown for the fit's poles, identified by least squares over the stored solutions (the
 * paper's residue identification of Sec. 2.3), evaluated at the new frequency.  The GMRES
 * tolerance is unchanged. 
 * resp_out[nt_out x (K + Kt)] (host or device): time responses of the ORFs then the test
 * unknowns at t_out[nt_out] (Eq. (vf-td), final fit); stats nullable.
 * Errors: INVALID_ARG, NOT_CONVERGED (a frequency solve failed), NO_MESH, CUDA. */
int bem_afs(bem_ctx* ctx, const bem_afs_params* params, const int64_t* orf, int64_t K,
            const int64_t* test, int64_t Kt, const double* t_out, int64_t nt_out, double* resp_out,
            bem_afs_stats* stats);

/* ------------------------------------------------------------------ operator-level calls
 * (the steps of one solve, exposed for verification and measurement) */

/* Element geometry (step a1): out[ne x 8] doubles (host or device) =
 * centroid x,y,z, unit normal x,y,z, area, longest edge h_e. */
int bem_geometry(bem_ctx* ctx, double* out);

/* Near-source lists (step a2): CSR over collocation points, sources e != i with
 * |x_i - c_e| < 2 h_e, ascending.  row_ptr[ne+1] (host); cols[cap] (host) may be NULL to
 * query the count, which is returned in *nnz.  Errors: INVALID_ARG (cap too small). */
int bem_near_lists(bem_ctx* ctx, int64_t* row_ptr, int32_t* cols, int64_t cap, int64_t* nnz);

/* Element integral blocks H_ie = int_e T(x_i, y; s) dA, G_ie = int_e U(x_i, y; s) dA
 * (steps a2/a4; Eq. (bie) discretised) for npairs (i, e) pairs at one frequency, FP64, with the
 * same rule selection as the operator (self: Duffy + CPV, near: 7-point, far: 4-point).
 * rows, cols: int32[npairs] (host).  H_out, G_out: npairs x 3 x 3 complex (host or device),
 * row-major [pair][i][j], (re, im) interleaved. */
int bem_element_blocks(bem_ctx* ctx, double s_re, double s_im, const int32_t* rows,
                       const int32_t* cols, int64_t npairs, double* H_out, double* G_out);

/* y = A(s_k) x_k (which = BEM_APPLY_A) or y = K(s_k) x_k (BEM_APPLY_K) for all k (steps
 * a2+a4): x, y: ns x 3ne complex doubles (host or device).  precision: BEM_PREC_FP64 or
 * BEM_PREC_FP32 (inputs rounded to FP32, far and near kernels in FP32, output widened). */
int bem_apply(bem_ctx* ctx, const double* s, int64_t ns, const double* x, double* y,
              int precision, int which);

/* Right-hand sides b(s_k) = K(s_k) (profile(s_k) * bc_value) in FP64 (step a3).
 * b_out: ns x 3ne complex doubles (host or device). */
int bem_rhs(bem_ctx* ctx, const double* s, int64_t ns, double* b_out);

/* Refinement residual (step a7): r_k = b(s_k) - A(s_k) x_k with b formed from the boundary
 * data in the same sweep (r = K k - A x).  mode: BEM_RESID_DF64 or BEM_RESID_FP64 (far field
 * arithmetic; near field and own element are FP64 in both).  x, r: ns x 3ne complex. */
int bem_residual(bem_ctx* ctx, const double* s, int64_t ns, const double* x, double* r, int mode);

/* Block-Jacobi preconditioner (step a5): y_k = D(s_k)^{-1} x_k with D the 3 x 3 diagonal
 * blocks A_ii(s_k) (free term + own-element integral).  FP64.  x, y: ns x 3ne complex. */
int bem_precond_apply(bem_ctx* ctx, const double* s, int64_t ns, const double* x, double* y);

/* ------------------------------------------------------------------ measurement */

/* Kernel classes timed by bem_profile. */
#define BEM_KERNEL_FAR32 0   /* FP32 far-field operator kernel (the hot loop)      */
#define BEM_KERNEL_FAR64 1   /* FP64 far-field operator kernel (RHS, residuals)     */
#define BEM_KERNEL_NEAR32 2  /* FP32 near-field + own-element correction          */
#define BEM_KERNEL_NEAR64 3  /* FP64 near-field + own-element correction          */
#define BEM_KERNEL_SELF 4    /* own-element singular blocks + preconditioner       */
#define BEM_KERNEL_VEC 5     /* GMRES vector kernels of one Arnoldi step            */
#define BEM_KERNEL_RES64 6   /* FP64 residual r = K k - A x (far field, fused U + T) */
#define BEM_KERNEL_HAPPLY 7  /* H-matrix far field: low-rank and dense blocks applied    */
#define BEM_KERNEL_HBUILD 8  /* H-matrix build: cross approximations and factor copies   */

/* Enable (1) or disable (0) CUDA-event timing of the kernel classes above, on the context's
 * stream; resets the totals.  Timing adds two event records per timed launch. */
int bem_profile(bem_ctx* ctx, int enable);

/* Totals since bem_profile(ctx, 1): number of timed launches, summed device milliseconds
 * (events bracket each launch on the launching stream) and, for the operator kernels, the
 * number of frequencies the launches covered (each far/near launch computes the listed active
 * frequencies only).  Any output pointer may be NULL.  Errors: INVALID_ARG (bad kind). */
int bem_kernel_time(bem_ctx* ctx, int kind, int64_t* launches, double* ms, int64_t* freq_launches);

/* ------------------------------------------------------------------ launch tuning
 * The FP32 far-field launch (the operator's hot loop) has three shape parameters:
 *   ft    frequencies one CTA evaluates together (1, 4, 8 or 12): each source point's geometry
 *         is formed once and reused for them;
 *   tiles 32-element source tiles a CTA sums in FP32 before its FP64 atomic add;
 *   waves the source range is split until the grid holds waves x SMs x resident CTAs per SM.
 * The best shape depends on the mesh size and on how many frequencies a launch carries (GMRES
 * retires converged frequencies, so late launches carry few).  Without a table every launch uses
 * ft 12, tiles 2, waves 4.  A table is a list of entries; a launch on a mesh of ne elements with
 * nfl frequencies uses, among the entries with the smallest ne_max >= ne (else the largest
 * ne_max), the one with the smallest nfl_max >= nfl (else the largest nfl_max).  The paper has
 * no counterpart (its solver runs on a CPU). */
typedef struct bem_tune_entry {
  int64_t ne_max;   /* the entry applies to meshes of at most ne_max elements ...            */
  int32_t nfl_max;  /* ... and to launches of at most nfl_max frequencies                    */
  int32_t ft, tiles, waves;
  double ms;        /* bem_autotune output: one operator application's time with this shape */
  double ms_fixed;  /* bem_autotune output: the same with the fixed shape (12, 2, 4)        */
} bem_tune_entry;

/* Autotuner: for the context's mesh (material and boundary conditions set), and for launches of
 * the first nfl[j] frequencies of s (j < n_nfl, each <= ns), times one FP32 operator application
 * (far-field launches + near field) for every shape (ft in {4, 8, 12}, and 1 for launches of at
 * most 2 frequencies; tiles in {1, 2, 4}; waves in {2, 4, 8}; CUDA events, best of 2 after a
 * warm-up) and keeps the fastest.  out[n_nfl] (host): the chosen entries (ne_max = the mesh's
 * ne).  They are also installed in the context (replacing entries with the same ne_max).
 * Errors: INVALID_ARG (sizes, nfl[j] outside [1, ns]), NO_MESH, OOM, CUDA. */
int bem_autotune(bem_ctx* ctx, const double* s, int64_t ns, const int32_t* nfl, int32_t n_nfl,
                 bem_tune_entry* out);
/* Install a table of n entries (host; copied), replacing the context's table; n = 0 restores
 * the fixed shape.  Errors: INVALID_ARG (an entry with ft not 1, 4, 8 or 12, tiles or waves < 1). */
int bem_set_tuning(bem_ctx* ctx, const bem_tune_entry* table, int32_t n);
/* Read a table from a text file (one entry per line: ne_max nfl_max ft tiles waves [ms ms_fixed];
 * '#' starts a comment; ms and ms_fixed are optional) and install it.
 * Errors: INVALID_ARG (unreadable file or bad line). */
int bem_load_tuning(bem_ctx* ctx, const char* path);
/* The shape a far-field launch of nfl frequencies on the context's mesh would use. */
int bem_launch_shape(bem_ctx* ctx, int64_t nfl, int32_t* ft, int32_t* tiles, int32_t* waves);

/* Measured arithmetic peak of the context's device, the denominator of the ALU-bound kernels'
 * rooflines (the paper has no counterpart: the operator and the refinement residual are bound by
 * the FP32 pipes, the plain-FP64 path by the FP64 pipes).  A kernel fills every SM with
 * independent fused multiply-add chains (FFMA for BEM_PEAK_FP32, DFMA for BEM_PEAK_FP64; 2 flops
 * each), iters x 128 steps per chain, launched reps times on the context's stream after one
 * warm-up launch and timed with CUDA events.  Out (host, each nullable): *tflops = the best
 * launch's rate, *ms_best = its duration, *sm_count = the device's multiprocessor count.
 * Errors: INVALID_ARG (kind, iters < 1, reps < 1), OOM, CUDA. */
#define BEM_PEAK_FP32 0
#define BEM_PEAK_FP64 1
#define BEM_PEAK_FP32X2 2  /* FP32 with the paired instruction (two FMAs per thread per FFMA2) */
int bem_measure_peak(bem_ctx* ctx, int kind, int32_t iters, int32_t reps, double* tflops,
                     double* ms_best, int32_t* sm_count);

/* ------------------------------------------------------------------ fast far field (H-matrix)
 *
 * The paper speeds up the matrix-vector product of its iterative solve with a fast multipole
 * method (Sec. 2.1, the paragraph on the fast solver).  This library's fast far field is a
 * hierarchical matrix of the 4-point-rule far-field part A4 of the system operator,
 *     A4[i, e] = sum_q w_q K_e(x_i, y_q)  for e != i  (K_e = T for a traction-given column,
 *                -U for a displacement-given one),   A4[i, i] = 0,
 * the part the FP32 far kernel sums over all sources; the near-field and own-element
 * corrections are applied exactly as without it.  The elements are ordered by a cluster tree
 * (recursive median bisection along the longest side of the centroids' bounding box, ties by
 * element index, first half = size / 2 to the left, until at most `leaf` elements).  A pair of
 * clusters whose vertex bounding boxes satisfy max(diam) <= eta dist, dist > 0, and whose sizes
 * are at most max_block, is a low-rank block (U V^T from a partially pivoted cross approximation
 * to the relative Frobenius tolerance eps, with trial steps from each vector component before it
 * stops, displacement-given columns scaled by mu / D inside it, D the mesh's bounding-box
 * diagonal; FP32 factors); a pair of leaves that is not is a dense block, evaluated on the fly.
 * Other pairs are split, both sides (the non-leaf side when one is a leaf), depth first.
 *
 * When enabled, every FP32 application of A (the inner GMRES operator of BEM_PREC_MIXED solves
 * and bem_apply with BEM_PREC_FP32, BEM_APPLY_A) uses it.  The factors are built on the device
 * at the first such application after the frequency set changes, for all frequencies of the
 * set.  The FP64-class refinement residual stays the exact operator, so a mixed solve still
 * certifies tol against the full discretisation; the approximation only changes how many
 * refinements it takes. */
typedef struct bem_hmatrix_params {
  int32_t enable;     /* 1: use the H-matrix far field; 0: the direct far kernel (default 0)  */
  int32_t leaf;       /* elements per leaf cluster, at most (default 32; 1 .. 128)            */
  int32_t max_block;  /* elements per side of a low-rank block, at most (default 512;
                         leaf .. 1024)                                                        */
  int32_t max_rank;   /* rank cap of one block's cross approximation (default 96; 1 .. 256);
                         a block that reaches it keeps that rank and is counted in `capped`  */
  double eta;         /* admissibility parameter (default 2.0; > 0)                           */
  double eps;         /* cross-approximation tolerance (default 1e-4; 0 < eps < 1); the factors
                         and the residuals of the approximation are FP32, so tolerances below
                         ~1e-5 reach their rounding floor and blocks run to max_rank (capped) */
  int32_t max_freqs;  /* frequencies whose factors are held at once: a bem_solve_frequencies
                         or bem_fsm list longer than this is solved in consecutive chunks of
                         max_freqs frequencies (default 0: the whole list at once; the two
                         passes of BEM_WARM_SWEEP are not chunked)                          */
  int32_t reserved[5];
} bem_hmatrix_params;

typedef struct bem_hmatrix_info {
  int64_t clusters;        /* clusters of the tree                                          */
  int64_t lowrank_blocks;  /* low-rank blocks of the partition                              */
  int64_t dense_blocks;    /* dense blocks                                                  */
  int64_t lowrank_pairs;   /* element pairs the low-rank blocks cover                       */
  int64_t dense_pairs;     /* element pairs the dense blocks cover (the on-the-fly work)    */
  int64_t frequencies;     /* frequencies of the last build                                */
  int64_t factor_bytes;    /* device bytes of the factors of the last build                 */
  int64_t rank_sum;        /* sum of the block ranks over blocks and frequencies            */
  int32_t rank_max;        /* largest block rank                                            */
  int32_t capped;          /* (block, frequency) approximations that reached max_rank       */
  double seconds_build;    /* wall time of the last build (cross approximations + copies)   */
  int64_t builds;          /* builds since the parameters were set                          */
  int64_t reserved[4];
} bem_hmatrix_info;

/* Defaults of bem_hmatrix_params (enable = 0). */
int bem_default_hmatrix_params(bem_hmatrix_params* p);
/* Enable (p->enable = 1), disable (p->enable = 0 or p NULL) or re-parametrise the H-matrix far
 * field; drops any factors held.  Errors: INVALID_ARG (a parameter out of range). */
int bem_set_hmatrix(bem_ctx* ctx, const bem_hmatrix_params* p);
/* Statistics of the partition and of the last build (host struct). */
int bem_get_hmatrix_info(bem_ctx* ctx, bem_hmatrix_info* out);
/* The cluster tree and block partition the H-matrix uses for a mesh (host only, no context and
 * no GPU needed).  verts: nv x 3 doubles, tris: ne x 3 int32 (host).  Outputs (host, each
 * nullable): perm[ne] (tree position -> element), clusters[cap_clusters][2] (first position,
 * size) in depth-first order (a cluster, its left subtree, its right subtree), lowrank and
 * dense [cap][2] (target cluster, source cluster) in the order of the depth-first subdivision
 * of (root, root), target children outer.  counts[3] (host, required) receives the numbers of
 * clusters, low-rank and dense blocks; an array whose capacity is smaller is not written.
 * Errors: INVALID_ARG (sizes, indices or parameters out of range); message in
 * bem_last_error(NULL). */
int bem_hmatrix_partition(const double* verts, int64_t nv, const int32_t* tris, int64_t ne,
                          const bem_hmatrix_params* p, int32_t* perm, int32_t* clusters,
                          int64_t cap_clusters, int32_t* lowrank, int64_t cap_lowrank,
                          int32_t* dense, int64_t cap_dense, int64_t* counts);

#ifdef __cplusplus
}
#endif
#endif /* BEM_H */
