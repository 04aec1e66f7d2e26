/*
 * opf.h -- C ABI of libopf.so, a GB300 (sm_103a) implementation of the
 * pipe-flow Navier-Stokes time step described in Willis (2017), "The
 * Openpipeflow Navier-Stokes solver", SoftwareX 6:124-127.
 *
 * Problem (paper section 2): incompressible flow in the periodic pipe
 * (r, theta, z) in [0,1] x [0, 2pi/m_p) x [0, 2pi/alpha), lengths in units of
 * the radius R and velocities in units of the laminar centre-line speed,
 * Re = U_cl R / nu (= D U_bulk / nu, section 1).  Each field is expanded as in
 * Eq. 1:  A(r,theta,z) = sum_{|k|<K} sum_{|m|<M} A_km(r_n) e^{i(alpha k z + m_p m theta)},
 * n = 1..N radial points, negative m by complex conjugation.
 *
 * STATE LAYOUT (all host/device state buffers below): interleaved complex
 * double, array [3][M][2K-1][N] = (u_r, u_theta, u_z)[m][k + K - 1][n],
 * n fastest, r_N = 1 is the wall.  The state is the TOTAL velocity (the
 * laminar profile 1 - r^2 sits in the (k,m) = (0,0) u_z coefficient).
 * Size in doubles: 2 * 3 * M * (2K-1) * N.
 *
 * ERRORS: every int-returning call returns OPF_OK (0) or a negative code; the
 * reason is available from opf_last_error() (thread-local, library-owned
 * string, valid until the next failing call or state load on the same
 * thread).
 * Buffers passed in are owned by the caller and only read/written during the
 * call.  Calls on one handle must not overlap; different handles are
 * independent.  All compute runs on the CUDA device current at opf_create.
 */
#ifndef OPF_H
#define OPF_H

#ifdef __cplusplus
extern "C" {
#endif

#define OPF_OK 0
#define OPF_EINVAL -1   /* bad argument (NULL, size, unknown option) */
#define OPF_ECUDA -2    /* a CUDA runtime call failed */
#define OPF_ENAN -3     /* non-finite values in a state */
#define OPF_ETIMEOUT -4 /* a bounded device-side wait expired */
#define OPF_ENOMEM -5   /* device or host allocation failed */

typedef struct opf_ctx opf_t; /* opaque; owned by the library */

/* Create a solver for resolution (N, K, M), rotational symmetry m_p, axial
 * wavenumber alpha, Reynolds number Re and time step dt (paper section 2).
 * Builds the radial mesh (Chebyshev-clustered points, section 2), the 9-point
 * finite-difference operators, one banded LU factorisation per radial
 * operator (section 2.2), the influence-matrix boundary data (section 2) and
 * the fixed-flux response, and allocates device memory.  Requires N >= 9,
 * K >= 1, M >= 1, m_p >= 1, alpha > 0, Re > 0, dt > 0, and 3K, 3M with no
 * prime factor other than 2, 3, 5.  Returns NULL on failure (opf_last_error). */
opf_t* opf_create(int N, int K, int M, int m_p, double alpha, double Re, double dt);

/* As opf_create, on a user radial mesh (paper section 2: the radial points
 * may be supplied instead of computed): r holds N strictly increasing points
 * in (0, 1] with r[N-1] = 1 (the wall), host memory, copied; NULL = the
 * default points.  Stencils (9 index-nearest points of the parity-extended
 * mesh), quadrature weights, operators and the influence data are built on
 * these points; states on the handle are sampled there.  NULL on an invalid
 * mesh (opf_last_error). */
opf_t* opf_create_mesh(int N, int K, int M, int m_p, double alpha, double Re, double dt, const double* r);

/* Release the handle and its device memory.  NULL is ignored. */
void opf_destroy(opf_t* h);

/* Reason for the last failing call on this thread ("" if none); after a
 * successful opf_set_state family call, "" or that call's note. */
const char* opf_last_error(void);

/* Load a state from a host buffer (layout above).  The m = 0 coefficients are
 * projected onto Hermitian symmetry A(-k,0) = conj A(k,0) (real fields,
 * section 2).  On success opf_last_error() is "" unless the buffer's m = 0
 * coefficients were not Hermitian to 1e-12 of the largest of them (parts
 * compared separately): then it holds a note with that relative asymmetry,
 * and the call still returns OPF_OK with the projected state loaded.
 * OPF_ENAN if the buffer holds a NaN/Inf (the previous state is kept). */
int opf_set_state(opf_t* h, const double* coeffs);

/* Copy the current state into a host buffer (layout above).  Pinned host
 * buffers (cudaHostAlloc / cudaMallocHost / cudaHostRegister memory) are
 * read (opf_set_state) and written (opf_get_state) by the library's kernels
 * directly; other host memory goes through a device staging copy.  Either
 * way the call is synchronous and the result the same. */
int opf_get_state(opf_t* h, double* coeffs);

/* Same as opf_set_state / opf_get_state with DEVICE pointers (layout above),
 * for callers that keep states resident on the GPU. */
int opf_set_state_device(opf_t* h, const double* d_coeffs);
int opf_get_state_device(opf_t* h, double* d_coeffs);

/* Advance n >= 0 time steps of the second-order predictor-corrector
 * (section 2): per step the nonlinear term u x omega is evaluated
 * pseudo-spectrally on the 3K x 3M grid (section 2.2), then for every Fourier
 * mode a pressure-Poisson solve and implicit viscous solves for
 * u+- = u_r +- i u_theta and u_z (banded LU, section 2.2), the
 * influence-matrix correction that zeroes the boundary vector g (no-slip and
 * wall divergence, section 2), and the fixed-flux correction (section 1).
 * Synchronous: returns when the steps are complete.  OPF_ENAN if the state
 * became non-finite (detected when opf_energy/opf_check runs). */
int opf_step(opf_t* h, int n);

/* Kinetic energy E, energy input I and dissipation D, each normalised by its
 * laminar value (section 3.2, the columns of vel_totEID.dat):
 * out[0] = E/E_lam, out[1] = I/I_lam, out[2] = D/D_lam.  OPF_ENAN if any of
 * them is not finite. */
int opf_energy(opf_t* h, double out[3]);

/* Boundary residuals of the current state: out[0] = max |u(r=1)| over all
 * modes and components, out[1] = max |div u (r=1)| over modes (k,m) != (0,0)
 * (the vector g of section 2). */
int opf_wall_residual(opf_t* h, double out[2]);

/* Evaluate the nonlinear term N = u x omega (+ the base axial forcing 4/Re in
 * the (0,0) mode) of a host state, pseudo-spectrally with 3/2 dealiasing
 * (section 2), writing N in the state layout (N_r, N_theta, N_z) to a host
 * buffer.  The handle's current state is not modified. */
int opf_nonlinear(opf_t* h, const double* coeffs, double* out);

/* Options:
 *   "precision": 0 = FP64 throughout (default), 1 = mixed (FP32 transforms and
 *                product, FP64 radial solves and boundary correction)
 *   "n_corr":    corrector iterations per step (default 1; 0 = the predictor
 *                alone, a first-order step, e.g. to check single solves)
 *   "graph":     1 = replay the step as a CUDA graph (default), 0 = plain launches
 *   "timing":    1 = record per-kernel device times (opf_kernel_times); 2 = only
 *                the kernel named by "timed_kernel" (0 curl, 1 z synthesis,
 *                2 theta product, 3 z analysis, 4 solve; default 4), so the
 *                other kernels run without event records between them
 *   "autotune":  1 = on the next step, time the launch shapes of each kernel
 *                (columns/rows per block of the transforms, modes per block of
 *                the solve) on the current state and keep the fastest; reads
 *                back as 2 once done.  Read-only keys "mcz", "mca", "zc" report
 *                the transforms' shapes in use.
 *   "fused":     mixed precision only: the z synthesis, theta product and z
 *                analysis as one launch -- a cluster of blocks per radial
 *                plane exchanging the half-physical fields through
 *                distributed shared memory -- where the transform lengths
 *                are 48, 72 or 96: 0 = three launches (default), 1 = fused
 *                with the cluster size chosen (4, or 8 for few planes),
 *                2/4/8 = fused with that cluster size; the autotuner times
 *                both forms and keeps the faster.  Results are identical.
 *                Reads back the cluster size in use (0: three launches).
 *   "timed_kernel" (with "timing" 2): 5 = the fused transforms.
 *   "pdl":       launch the kernels of a step with programmatic dependent
 *                launch, so that each kernel's launch and read-only prologue
 *                overlap the end of its predecessor: 0 = plain launches
 *                (default; measured faster), 1 = each kernel signals its
 *                successor at the top of each block, 2 = before each block's
 *                final store phase.  Results do not depend on it.
 *   "tile":      modes per block of the solve: 0 = chosen from the grid size
 *                (default), 4, 8 or 16 (OPF_EINVAL if that block's shared
 *                memory does not fit); reads back the value set or the one the
 *                autotuner chose.  Results do not depend on it.
 *   "spike":     1 = the split solve with 4-mode tiles: each banded system
 *                (section 2.2) is substituted as two halves at once, joined by an
 *                8 x 8 interface system and rank-4 spike corrections (the
 *                factors are built at creation when N is even, N >= 26 and the
 *                grid is at most three 4-mode blocks per SM; elsewhere setting
 *                it is a no-op and it reads back 0).  Default: on where the
 *                grid is at most one block per SM.  It agrees with the
 *                single-chain solve to round-off (not bit for bit); the
 *                autotuner keeps whichever is set.
 *   "rot_x", "rot_y", "rot_z": frame rotation Omega (Cartesian components, pipe
 *                axis z; default 0): the Coriolis force -2 Omega x u joins the
 *                nonlinear term (section 3.1's rotating pipe; a transverse axis
 *                needs m_p = 1).  On an ensemble (opf_ens_set_option) it
 *                applies to every trajectory.
 *   "cfl":       C > 0 switches on automatic time-step control (section 2):
 *                after every step dt = min(dt_max, C / max(|u_r|/dr,
 *                |u_theta|/(r dtheta), |u_z|/dz)) over the 3K x 3M grid, applied
 *                when dt must drop or could rise by more than 10 %; the
 *                dt-dependent operators are then refactored.  0 = off (default).
 *                Single-trajectory handles only.
 *   "dt_max":    upper bound of the controlled dt (default: the initial dt).
 *   "dt":        set the time step now (refactors the dt-dependent operators).
 *   "cfl_number" (read only): max |u| dt / spacing seen in the last step.
 * Unknown keys or out-of-range values: OPF_EINVAL. */
int opf_set_option(opf_t* h, const char* key, double value);
int opf_get_option(opf_t* h, const char* key, double* value);

/* Time step, simulated time, and the excess pressure gradient beta of the
 * last step (driving force (4/Re)(1 + beta), fixed flux). */
int opf_get_dt(opf_t* h, double* dt);
int opf_get_time(opf_t* h, double* t);
int opf_get_beta(opf_t* h, double* beta);

/* Launch subsequent work on this CUDA stream (a cudaStream_t; NULL = the
 * library's own stream).  The caller keeps the stream alive while in use. */
int opf_set_stream(opf_t* h, void* stream);

/* Per-kernel device time of the steps run since the last call with reset=1:
 * names[i] (library-owned) and total_ms[i], launches[i] for i < *count
 * (capacity cap).  Collected only while option "timing" = 1.  In FP64 steps
 * the curl is taken inside the solve launches (its own kernel runs only when
 * a step starts after the state, the work buffers or an option changed, and
 * is not timed then), so "curl" reports no launches there. */
int opf_kernel_times(opf_t* h, int cap, int* count, const char** names,
                     double* total_ms, int* launches, int reset);

/* ---- Ensembles: many independent trajectories stepped together -----------
 * The paper runs one trajectory per job; this batches count trajectories,
 * each with its own resolution and parameters, into one CUDA graph per step:
 * trajectories with equal (N, K, M, m_p, alpha) share every kernel launch
 * (one launch covers all of them), while Re and dt may differ per trajectory
 * (each gets its own radial operators).  Arrays N..dt have count entries;
 * trajectory i's state uses the layout above with its own (N, K, M).
 * NULL on invalid arguments or allocation failure (opf_last_error). */
typedef struct opf_ens opf_ens_t;
opf_ens_t* opf_ens_create(int count, const int* N, const int* K, const int* M, const int* m_p,
                          const double* alpha, const double* Re, const double* dt);
void opf_ens_destroy(opf_ens_t* e);
int opf_ens_count(opf_ens_t* e, int* count);
/* State of trajectory i (host or device buffer, state layout, its own sizes). */
int opf_ens_set_state(opf_ens_t* e, int i, const double* coeffs);
int opf_ens_get_state(opf_ens_t* e, int i, double* coeffs);
int opf_ens_set_state_device(opf_ens_t* e, int i, const double* d_coeffs);
int opf_ens_get_state_device(opf_ens_t* e, int i, double* d_coeffs);
/* Advance every trajectory n steps (same scheme as opf_step); synchronous. */
int opf_ens_step(opf_ens_t* e, int n);
/* E, I, D of trajectory i (as opf_energy) and its simulated time. */
int opf_ens_energy(opf_ens_t* e, int i, double out[3]);
int opf_ens_get_time(opf_ens_t* e, int i, double* t);
/* Same options as opf_set_option, applied to all trajectories. */
int opf_ens_set_option(opf_ens_t* e, const char* key, double value);
int opf_ens_set_stream(opf_ens_t* e, void* stream);
int opf_ens_kernel_times(opf_ens_t* e, int cap, int* count, const char** names,
                         double* total_ms, int* launches, int reset);

/* ---- Newton-Krylov-trust-region solver (paper section 2: Newton utility
 * with a combined Krylov / trust-region "hookstep" method, Viswanath 2007) --
 * opf_nk_core solves F(x) = 0 for count independent problems of size n in
 * lockstep: GMRES (modified Gram-Schmidt, FP64) builds a Krylov basis from
 * Jacobian-vector products, the hookstep minimises the linearised residual
 * inside a trust region via the SVD of the small Hessenberg matrix, and a
 * trial is accepted when it achieves >= 1 % of the predicted reduction.
 * Callbacks see a subset of the problems: idx[j] is the problem index of
 * x[j]; commit = 1 marks points that become the base of the following
 * Jacobian-vector products.  Return non-zero from a callback to abort.
 * x: [count][n] in/out; scale: per problem (|F| <= tol * scale stops it);
 * res_out: final |F| / scale; iters_out: accepted Newton steps. */
typedef int (*opf_nk_residual)(void* ctx, int count, const int* idx, double* const* x,
                               double* const* f, int commit);
typedef int (*opf_nk_jv)(void* ctx, int count, const int* idx, double* const* x,
                         double* const* v, double* const* jv);
typedef struct {
  int max_newton;    /* Newton iterations */
  int max_krylov;    /* Krylov dimension per Newton iteration */
  int max_hook;      /* trust-region trials per Newton iteration */
  double tol;        /* |F| <= tol * scale stops a problem */
  double gmres_tol;  /* GMRES relative residual target */
  double delta0;     /* initial trust radius (<= 0: 0.1 |x|) */
  /* used by opf_nk_solve only: */
  double dt;         /* target time step; steps per period n = ceil(T / dt) */
  double eps;        /* relative size of the finite-difference perturbation */
  int fix_T;         /* 1: period T fixed (no time phase condition) */
  int fix_s;         /* 1: axial shift s fixed (no axial phase condition) */
  int precision;     /* time integrations: 0 FP64, 1 mixed */
  /* physics of the time integrations, as opf_set_forcing and the rot_x/y/z
   * options of a handle (paper section 3.1's forcing hook and Coriolis force): */
  const double* forcing; /* constant body force, state layout, host memory; NULL = none */
  double rot[3];         /* frame rotation (Omega_x, Omega_y, Omega_z); a transverse
                          * axis needs m_p = 1 */
} opf_nk_opts;
int opf_nk_core(int n, int count, double* x, const double* scale, opf_nk_residual F,
                opf_nk_jv JV, void* ctx, const opf_nk_opts* opts, double* res_out,
                int* iters_out);

/* Periodic orbits / relative periodic orbits / travelling waves of the pipe
 * flow: solve sigma_s Phi_T(u) = u, Phi_T the time-T map of opf_step (n steps
 * of dt = T/n) and sigma_s the axial shift by s, for count initial guesses in
 * lockstep (every Krylov step integrates all guesses in one batched launch
 * sequence).  Unknowns: the state's independent coefficients, T and s (unless
 * fixed), with phase conditions <du/dt, du'> = 0 and <du/dz, du'> = 0 closing
 * the system.  states: [count] host states (state layout) in/out; T, s:
 * [count] in/out; residual: [count] final |F| / |u|; iters: [count]. */
int opf_nk_solve(int N, int K, int M, int m_p, double alpha, double Re, int count,
                 double* states, double* T, double* s, const opf_nk_opts* opts,
                 double* residual, int* iters);

/* Multiple shooting (paper section 2: orbits may be split into sections):
 * as opf_nk_solve, with each orbit split into S sections of duration T/S,
 * each integrated as its own trajectory of the batched group.  Unknowns: the
 * S section starts, T and s; residual Phi_{T/S}(u_q) - u_{q+1} (q < S-1) and
 * sigma_s Phi_{T/S}(u_{S-1}) - u_0; phase conditions on u_0.  states:
 * [count][S] host states (section starts, state layout) in/out; residual:
 * |F| / |(u_0 .. u_{S-1})|.  S = 1 is single shooting. */
int opf_nk_solve_ms(int N, int K, int M, int m_p, double alpha, double Re, int count, int S,
                    double* states, double* T, double* s, const opf_nk_opts* opts, double* residual,
                    int* iters);

/* ---- Leading eigenvalues of linear maps: stability of invariant solutions
 * (the paper's Newton utility converges travelling waves and periodic orbits;
 * section 3.2 quotes the leading eigenvalue of one) --------------------------
 * opf_arnoldi_core runs kdim Arnoldi steps (modified Gram-Schmidt applied
 * twice, FP64) for count linear maps of size n in lockstep: each step calls
 * A once for all maps still running (idx[j] names the map of v[j]; write
 * A v[j] to av[j]; return non-zero to abort).  A map stops early when its
 * Krylov space becomes invariant.  Ritz values are the eigenvalues of the
 * Hessenberg matrix (implicit double-shift QR); the nev of largest modulus
 * are returned per map ([count][nev], decreasing modulus) with residual
 * estimates |h_{k+1,k}| |e_k^T y| (y the unit Ritz vector of H; resid may be
 * NULL).  v0: [count][n] starting vectors (non-zero); kused: [count] Krylov
 * dimension reached (may be NULL).  Returns OPF_EINVAL on bad arguments. */
typedef int (*opf_linear_map)(void* ctx, int count, const int* idx, double* const* v, double* const* av);
int opf_arnoldi_core(int n, int count, const double* v0, int kdim, int nev, opf_linear_map A, void* ctx,
                     double* eig_re, double* eig_im, double* resid, int* kused);

/* Floquet multipliers (eigenvalues of the linearised period map
 * dv -> sigma_s DPhi_T(u) dv) of count states of the pipe flow, e.g. periodic
 * orbits or travelling waves returned by opf_nk_solve (for a travelling wave
 * or equilibrium any T > 0 works; the multipliers are then exp(lambda T)).
 * Phi_T: n = ceil(max T / dt) steps of T_i / n; products by finite
 * differences with relative step eps (perturbation eps |u| / |dv|);
 * precision: 0 FP64, 1 mixed time integration; start: [count] starting
 * vectors in the state layout, or NULL for SplitMix64 uniforms from seed (a
 * start inside an invariant subspace, e.g. one Fourier mode of one component,
 * restricts the search to it).  states: [count] host states (state layout);
 * outputs as for opf_arnoldi_core, over the independent coefficients (m = 0
 * with k >= 0, all k for m > 0).  No counterpart call exists in the paper. */
int opf_floquet(int N, int K, int M, int m_p, double alpha, double Re, int count, const double* states,
                const double* T, const double* s, int kdim, int nev, double dt, double eps, int precision,
                unsigned long long seed, const double* start, double* eig_re, double* eig_im, double* resid);

/* ---- Proposal network for Newton-Krylov initial guesses (no counterpart in
 * the paper; the learned-proposal part of this implementation) ---------------
 * A 1-D convolution net over the L radial points of the lowest Fourier modes:
 *   h1 = gelu(conv3(x)), h2 = gelu(conv3(h1)), y = conv3(h2)  ([B][L][cin])
 *   z = Wh mean_l(h2) + bh                                    ([B][nout])
 * conv3: width 3 along r, zero padding.  BF16 operands, FP32 accumulation
 * (tensor-core GEMMs), FP32 master weights, Adam.  Loss:
 * mean((y - ty)^2) + lambda mean((z - tz)^2).  All array arguments of the
 * forward/gradient/train calls are DEVICE pointers to float32; parameters
 * are exchanged in the order W1 [H][3 cin], b1, W2 [H][3H], b2, W3 [cin][3H],
 * b3, Wh [nout][H], bh (W[o][j*C + c] weights input channel c at offset j-1). */
typedef struct opf_net opf_net_t;
opf_net_t* opf_net_create(int cin, int hidden, int L, int nout, unsigned long long seed);
void opf_net_destroy(opf_net_t* n);
int opf_net_param_count(opf_net_t* n, long* total, long* sizes8);
int opf_net_get_params(opf_net_t* n, float* host, int grads); /* grads=1: last gradients */
int opf_net_set_params(opf_net_t* n, const float* host);
int opf_net_forward(opf_net_t* n, const float* d_x, int B, float* d_y, float* d_z);
int opf_net_gradients(opf_net_t* n, const float* d_x, const float* d_ty, const float* d_tz, int B,
                      float lambda, double* loss);
int opf_net_train_step(opf_net_t* n, const float* d_x, const float* d_ty, const float* d_tz, int B,
                       float lambda, float lr, double* loss);
/* Training minibatch with the flow's symmetries applied (data augmentation,
 * on the net's stream, ordered before the next train step): sample b is row
 * idx[b] < rows of the DEVICE sets d_x, d_y ([rows][L][ncomp*nkf*mf*2]
 * float32, channels (component, axial index, azimuthal index, re/im),
 * axial index kidx for k = kidx - (nkf - 1)/2) and d_z ([rows][nz]); each
 * complex channel of its x and y is multiplied by e^{i(ang[2b] k +
 * ang[2b+1] m)} -- an axial shift by a with ang[2b] = alpha a and an
 * azimuthal rotation by phi with ang[2b+1] = m_p phi, both symmetries of
 * pipe flow -- and its z is copied unchanged (period and shift are
 * invariant).  idx and ang are HOST arrays (B and 2B entries, copied);
 * outputs d_bx, d_by ([B][L][...]) and d_bz ([B][nz]) are DEVICE buffers.
 * OPF_EINVAL on bad sizes or an index out of range. */
int opf_net_gather_augment(opf_net_t* n, int B, int L, int ncomp, int nkf, int mf, int nz, const float* d_x,
                           const float* d_y, const float* d_z, long rows, const int* idx, const float* ang,
                           float* d_bx, float* d_by, float* d_bz);

/* No counterpart in the paper: an allocation-free variant of opf_nonlinear
 * for callers that must not allocate device memory when they call (their
 * device memory is all owned by their own pool, cudaMalloc/cudaFree could
 * synchronise the device at a bad moment, or they forbid allocation after
 * start-up).  Same result as opf_nonlinear on a handle created with the same
 * (N, K, M, m_p, alpha, Re), but without a handle: d_state and d_out are
 * DEVICE buffers in the state layout, stream is a cudaStream_t (NULL = the
 * default stream); the call returns when the result is in d_out.  All
 * intermediates (stencils, twiddles, transforms) live in one fixed 16 MiB
 * device array inside the library, held on every GPU that loads it until
 * the process exits; OPF_EINVAL if the resolution needs more (the small
 * N=32, |k|<16, m<16 case needs 6.6 MB).  The first call on a device looks
 * up that array's address there and sets the kernels' shared-memory limits,
 * so make it before any stream capture; CUDA loads modules lazily, so that
 * first call (not loading the library) is also what places the array and the
 * kernels' code on the device: make it at start-up, before the caller's own
 * pool takes the device memory.  The call synchronises its stream before it
 * returns, so on a stream that is being captured it returns OPF_EINVAL
 * without launching anything.  Calls share the array: calls whose GPU work
 * overlaps race.  On success it calls no allocator at all (no cudaMalloc,
 * cudaFree or allocating library routine); a failure only stores its message
 * for opf_last_error. */
int opf_nonlinear_noalloc(int N, int K, int M, int m_p, double alpha, double Re,
                          const double* d_state, double* d_out, void* stream);

/* Constant body force f (paper section 3.1: a user forcing hook; state layout,
 * components (f_r, f_theta, f_z), host memory, copied) added to the nonlinear
 * term at every evaluation; NULL removes it.  A uniform axial force on the
 * (0,0) mode is absorbed by the fixed-flux driving (beta shifts by -f Re / 4). */
int opf_set_forcing(opf_t* h, const double* coeffs);

/* Host-only (no GPU needed): a state of resolution (N1, K1, M1) at another
 * resolution (N2, K2, M2), same m_p (the paper: initial conditions of another
 * resolution are truncated or interpolated automatically).  Fourier modes
 * present in both are copied, the others are zero; radial profiles are
 * interpolated by the 9-point Lagrange interpolant through the nearest nodes
 * of the source mesh extended to negative r with the field's axis parity.
 * in / out: state layout [3][M][2K-1][N] complex (interleaved), caller-owned.
 * OPF_EINVAL for non-positive sizes or N1 < 9. */
int opf_change_resolution(int N1, int K1, int M1, const double* in, int N2, int K2, int M2, int m_p,
                          double* out);

/* Host-only diagnostics (no GPU needed): build the radial setup that
 * opf_create would build for these parameters and copy one array into
 * out[0..cap).  what = "r" (N radial points), "wq" (N quadrature weights,
 * sum wq f ~ int_0^1 f r dr for even f), "d1" / "d2" ([2][N][9] first/second
 * derivative stencils, [0] = even axis parity, [1] = odd, row n against
 * columns clamp(n-4, 0, N-9) + t), "G" (N, fixed-flux response),
 * "basis" ([K][M][6][N] influence-matrix responses), "luH" / "luP" (the
 * banded LU factors as the device reads them, 13 N values per operator:
 * [N][4] L(c+1+t, c), [N][4] L(c+5+t, c), [N] 1/U(c,c),
 * [N][4] U(c-1-t, c) / U(c-1-t, c-1-t), unit-lower L, zeros outside the
 * band; luH is [K][nJ] Helmholtz operators 1/dt - c L_j with the Dirichlet
 * wall row, luP is [K][M] pressure operators with the Neumann wall row plus
 * (0,0) with p(1) = 0 last), "hop" ([M][3] the index j' < nJ of the
 * Helmholtz operator of u+, u-, u_z at each m; section 2.2), "ainv"
 * ([M][2K-1][4][4] complex as (re, im) pairs: the inverse of the influence
 * matrix A, A[i][j] = g_i of basis response j, g = (u+(1), u-(1), u_z(1),
 * div u(1)), responses (pressure, unit u+, u-, u_z wall values); section 2;
 * zero at (0,0)); the two-partition forms of the same operators (even
 * N >= 26 only): "luH2" / "luP2" (per operator the top block's factors,
 * N/2 rows, then the bottom block's, each stored as luH), "spkH" / "spkP"
 * (per operator N rows of 4: T^{-1} H(0:k, k:k+4), then
 * B^{-1} H(k:N, k-4:k), k = N/2), "rH" / "rP" (per operator the 8 x 8
 * inverse of the interface system, row-major).  *len receives the full
 * length; OPF_EINVAL if cap is too small or what is unknown. */
int opf_setup_query(int N, int K, int M, int m_p, double alpha, double Re, double dt,
                    const char* what, double* out, long cap, long* len);
/* Same, on a user radial mesh r (N points as for opf_create_mesh; NULL = the
 * default points). */
int opf_setup_query_mesh(int N, int K, int M, int m_p, double alpha, double Re, double dt, const double* r,
                         const char* what, double* out, long cap, long* len);

/* No counterpart in the paper (measurement support): the device's sustained
 * fused multiply-add rate in TFLOP/s, FP64 (precision 0) or FP32 (precision
 * 1), measured with a kernel of independent FMA recurrences over every SM.
 * It is the denominator of the rooflines of the kernels bound by arithmetic
 * rather than by memory (the radial solves, the transforms).  Runs on the
 * current device; takes ~50 ms.  OPF_EINVAL for another precision or a NULL
 * output. */
int opf_fma_rate(int precision, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* OPF_H */
