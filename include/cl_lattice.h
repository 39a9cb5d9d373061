/*
 * cl_lattice.h -- C ABI of the GB300 lattice evolver for the method of
 * arXiv:2006.15122, "The Art of Simulating the Early Universe -- Part I".
 *
 * The library evolves interacting real scalar fields, or a U(1)-charged
 * complex scalar with a compact Abelian gauge field on link variables, on a
 * periodic N^3 comoving lattice in a self-consistently expanding FLRW
 * background, all in the paper's program variables (section 4.1):
 *   phi~ = phi/f*,  d eta~ = a^-alpha w* dt,  dx~ = w* dx,  V~ = V/(f*^2 w*^2).
 *
 * Conventions shared by every call:
 *  - No exceptions cross this boundary.  Every call returns a cl_status; a
 *    human-readable reason of the last failure is in cl_last_error().
 *  - A handle owns its device memory (cudaMalloc'd at lattice_init, freed at
 *    lattice_destroy).  Host pointers passed in are only read or written
 *    during the call.
 *  - Work is ordered on the CUDA stream given to lattice_init (NULL = the
 *    legacy default stream).  lattice_evolve only enqueues work; the
 *    measure, get and save calls synchronize that stream before returning.
 *  - Fields are stored as a double-precision homogeneous mean plus a
 *    fluctuation array in the handle's precision (CL_FP64 or CL_FP32), laid
 *    out SoA with site index (n3*N + n2)*N + n1 (n1 fastest, section 3.1).
 *    Every field crossing the ABI is the full field (mean + fluctuation) in
 *    double precision.
 *  - Errors: CL_ERR_ARG for invalid arguments (nothing is changed),
 *    CL_ERR_CUDA / CL_ERR_OOM for runtime failures, CL_ERR_UNSTABLE_DT when
 *    the time step exceeds the integrator's linear stability bound,
 *    CL_ERR_NONFINITE once a reduction has seen a NaN/Inf (the handle then
 *    refuses to evolve), CL_ERR_STATE for calls that do not fit the
 *    handle's state, CL_ERR_IO for checkpoint files that cannot be read,
 *    written or verified.
 */
#ifndef CL_LATTICE_H
#define CL_LATTICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status of every call; cl_last_error gives the reason.  CL_ERR_TIMEOUT: a
 * Gauss-Legendre step whose stage equations did not converge (the lattice
 * stops at the last completed step), or a bounded device-side wait that gave
 * up -- a field pass waiting for its tensor copies, a tensor-core GEMM waiting
 * for its MMAs, a training epoch waiting at a grid barrier (none expected);
 * errors found on the device are reported by the next call that synchronizes. */
typedef enum {
    CL_OK = 0,
    CL_ERR_ARG = 1,
    CL_ERR_CUDA = 2,
    CL_ERR_OOM = 3,
    CL_ERR_UNSTABLE_DT = 4,
    CL_ERR_NONFINITE = 5,
    CL_ERR_TIMEOUT = 6,
    CL_ERR_STATE = 7,
    CL_ERR_IO = 8
} cl_status;

/* Model families.
 * CL_MODEL_SU2: a complex doublet Phi = (Phi_1, Phi_2), stored as its four real
 *   components (Re Phi_1, Im Phi_1, Re Phi_2, Im Phi_2) = CL_FIELD(0..3), with
 *   V = (lam/4)(|Phi|^2 - vev2)^2, coupled with g = gauge_e to a compact SU(2)
 *   gauge field in temporal gauge (section 6): links U_i = q0 + i q.sigma as unit
 *   quaternions CL_SU2_LINK(i, c), electric momenta CL_SU2_EMOMENTUM(i, a).
 *   It starts from a homogeneous, uncharged doublet with unit links, plus (with
 *   init->spectrum) vacuum fluctuations of every canonical component sqrt(2) Phi_c,
 *   the total colour charges projected out of pi, and electric momenta from
 *   the Gauss law.
 *   SU(2) x U(1) + chi (the working example of section 8.3): gauge_e_u1 > 0
 *   also charges the doublet under a compact U(1) (link angles CL_LINK(i),
 *   electric momenta CL_EMOMENTUM(i); the parallel transporter of Phi is
 *   exp(-i theta_i) U_i) and n_fields = 2 adds a real singlet chi
 *   (CL_SINGLET, CL_SINGLET_MOMENTUM) with V_int = q |Phi|^2 chi^2.  Such a
 *   model starts from the constrained vacuum draws of section 7.2 (|l| = |r|
 *   per component, one l-r phase difference and one frequency, the mean
 *   curvature of the four components, for all of them), which leave no U(1)
 *   or SU(2) charge; chi starts with zero mean and velocity and the
 *   fluctuations of curvature 2 q |Phi|^2; both Gauss laws are solved for the
 *   electric momenta.  Energies are reported per sector (lattice_measure_means).
 * CL_MODEL_SCALAR: n_fields = 1 or 2 real singlets phi, chi with the program
 *   potential of section 8.1, V = (lam/p)|phi|^p + (q/2) phi^2 chi^2.
 * CL_MODEL_U1: one complex scalar phi = (phi_0 + i phi_1)/sqrt(2) with
 *   V = (lam/4)(|phi|^2 - vev2)^2, coupled with charge e to a compact U(1)
 *   gauge field in temporal gauge (section 5.3), or with noncompact = 1 to the
 *   non-compact one (section 5.2: magnetic term (D_i^+ A_j - D_j^+ A_i)^2, link
 *   angles theta_i = e dx A_i kept unwrapped). */
typedef enum { CL_MODEL_SCALAR = 0, CL_MODEL_U1 = 1, CL_MODEL_SU2 = 2 } cl_model_kind;

/* Integrators (the paper's "switch", section 1.2):
 * CL_INT_LF   staggered leapfrog: scheme III of section 4.2.1 for scalars,
 *             the compact staggered leapfrog of section 5.3.1 for U(1);
 * CL_INT_VV2  velocity-Verlet, section 4.2.3 (scalars) and 5.3.2 (compact U(1));
 * CL_INT_VV4..CL_INT_VV10  Yoshida compositions of VV2 (sections 4.3.2 and
 *             5.3.3, weights of the appendix table; VV4 in closed form);
 * CL_INT_RK4  explicit fourth-order Runge-Kutta in the velocity form of
 *             section 4.3.1 (scalar model, CL_FP64, self-consistent background;
 *             not symplectic: the paper's reference for the others);
 * CL_INT_GL2..CL_INT_GL5  implicit Gauss-Legendre Runge-Kutta with s = 2..5
 *             stages, order 2s (sections 3.4.2, 4.3.3, Scheme II; same
 *             restrictions as RK4; stages solved by fixed-point iteration to a
 *             relative 1e-14). */
typedef enum {
    CL_INT_LF = 0,
    CL_INT_VV2 = 1,
    CL_INT_VV4 = 2,
    CL_INT_VV6 = 3,
    CL_INT_VV8 = 4,
    CL_INT_VV10 = 5,
    CL_INT_RK4 = 6,
    CL_INT_GL2 = 7,
    CL_INT_GL3 = 8,
    CL_INT_GL4 = 9,
    CL_INT_GL5 = 10
} cl_integrator;

typedef enum { CL_FP64 = 0, CL_FP32 = 1 } cl_precision;

/* Expansion (section 4.1).
 * CL_BG_FRIEDMANN: self-consistent, b' = K_a from the volume-averaged energies
 *   (fstar_over_mp = 0 selects a static background, a = a0, b = 0);
 * CL_BG_FLUID: sourced by an external fluid of constant equation of state
 *   fluid_w, a(t) = a0 (1 + hubble0 t / p)^p with p = 2/(3(1 + fluid_w) - 2 alpha)
 *   and hubble0 the program Hubble rate a'/a at t = 0 (scalar model under the
 *   velocity-Verlet integrators; the Hubble constraint is then reported as 0). */
typedef enum { CL_BG_FRIEDMANN = 0, CL_BG_FLUID = 1 } cl_background;

/* Potential of the charged scalar of CL_MODEL_U1 / CL_MODEL_SU2 (|phi|^2 is
 * |phi|^2 for U(1) and Phi^dag Phi for SU(2)):
 *   CL_POT_HIGGS     V = (lam/4)(|phi|^2 - vev2)^2 (sections 5, 6);
 *   CL_POT_MONOMIAL  V = (lam/p)(2|phi|^2)^(p/2), p = pexp: the inflaton of the
 *                    gauge working examples (section 8) as a charged field,
 *                    2|phi|^2 being the squared canonical norm. */
typedef enum { CL_POT_HIGGS = 0, CL_POT_MONOMIAL = 1 } cl_gauge_potential;

typedef struct {
    int32_t kind;            /* cl_model_kind */
    int32_t n_fields;        /* CL_MODEL_SCALAR: 1 or 2; ignored for CL_MODEL_U1 */
    int32_t pexp;            /* p of (lam/p)|phi|^p (scalar) or of the monomial gauge potential: 2, 4 or 6 */
    int32_t background;      /* cl_background */
    double alpha;            /* alpha-time exponent (section 4.1) */
    double fstar_over_mp;    /* f_star/m_p; 0 selects a static background (a = 1, b = 0) */
    double omega_over_fstar; /* w_star/f_star: amplitude factor of the vacuum fluctuations (section 7) */
    double lam;              /* scalar: coefficient of (1/p)|phi|^p; U(1): lam of (lam/4)(|phi|^2 - vev2)^2 */
    double q;                /* scalar, n_fields = 2: coupling of (q/2) phi^2 chi^2 */
    double vev2;             /* U(1): vev2 */
    double gauge_e;          /* U(1): gauge coupling e = g_A Q_A in program units */
    double fluid_w;          /* CL_BG_FLUID: equation of state w of the fluid */
    double hubble0;          /* CL_BG_FLUID: program Hubble rate a'/a at t = 0 */
    int32_t potential;       /* U(1), SU(2): cl_gauge_potential */
    int32_t noncompact;      /* U(1): 1 selects the non-compact gauge kinetics of section 5.2 (0: compact) */
    double gauge_e_u1;       /* SU(2): U(1) coupling eA = g_A Q_A of the doublet (section 8.3); 0: no U(1) sector */
} cl_model;

typedef struct {
    int32_t N;          /* sites per dimension: multiple of 8, 8 <= N <= 2048 (U(1): N^3 < 2^32) */
    int32_t integrator; /* cl_integrator */
    int32_t precision;  /* cl_precision of the fluctuation arrays */
    int32_t force_dt;   /* nonzero: accept dt beyond the stability bound */
    double kIR;         /* infrared momentum k_IR = 2 pi / L in program units (section 3.1) */
    double dt;          /* time step d eta~ (program units) */
} cl_grid;

typedef struct {
    double phi0[4];     /* homogeneous values: scalar fields, or (phi_0, phi_1) of U(1) */
    double dphi0[4];    /* their program-time derivatives */
    uint64_t seed;      /* key of the Philox4x32-10 draws of the fluctuations */
    int32_t spectrum;   /* 0: homogeneous only; 1: vacuum fluctuations (section 7) */
    int32_t reserved;
    double fluct_scale; /* multiplies the fluctuation amplitude (1 = the paper's) */
    double a0;          /* initial scale factor (1 in every configuration of the paper) */
} cl_init;

/* Volume averages and constraints (sections 4.4, 5.4, 8.2.1). */
typedef struct {
    double t;              /* program time */
    double a, b;           /* scale factor and b = a' */
    int64_t step;          /* completed steps */
    double mean[4];        /* <f_c>: scalar fields, or Re/Im of phi for U(1) */
    double mean2[4];       /* <f_c^2> */
    double var[4];         /* <f_c^2> - <f_c>^2 */
    double mean_pi[4];     /* <pi_c> */
    double EK[4];          /* scalar: E_K per field; U(1): {E_K^phi, E_K^A}; SU(2): {E_K^Phi, E_K^B, E_K^A, E_K^chi} */
    double EG[4];          /* scalar: E_G per field; U(1): {E_G^phi, E_G^A}; SU(2): {E_G^Phi, E_G^B, E_G^A, E_G^chi} */
    double EV[4];          /* scalar: {<(lam/p)|phi|^p>, <(q/2)phi^2chi^2>}; U(1): {<V>};
                              SU(2): {<V(|Phi|^2) + q |Phi|^2 chi^2>} */
    double rho;            /* total energy density E_K + E_G + E_V (program units) */
    double w;              /* equation of state p/rho */
    double hubble_violation; /* Delta_e = |b^2 - rhs| / rhs of the Hubble constraint */
    double gauss_violation;  /* U(1), SU(2): Delta_g = rms(G)/sqrt(<lhs^2> + <rhs^2>), sums over every Gauss law */
    double reserved[4];
} cl_means;

typedef struct cl_lattice cl_lattice;

/* Status string of a code; never NULL. */
const char* cl_status_str(cl_status s);
/* Reason of the last failure on this handle (or of the last failed
 * lattice_init when h is NULL); never NULL. */
const char* cl_last_error(const cl_lattice* h);

/* Create a lattice: allocate device memory, draw the initial conditions of
 * section 7 on the device (Rayleigh moduli and uniform phases from
 * Philox4x32-10 keyed by init->seed, inverse DFT by cuFFT), fix b from the
 * Hubble constraint b^2 = (1/3)(f_star/m_p)^2 a^{2(alpha+1)} (E_K+E_G+E_V)
 * (sections 4.1, 4.2.3), and, for U(1), set A = 0 and the electric momenta
 * from the lattice Gauss law (section 7.2).  cuda_stream is a cudaStream_t
 * or NULL.  Rejects dt beyond the linear stability bound of the integrator
 * (omega_max dt < 2 for LF/VV2, < 1.5734 for VV4) unless grid->force_dt.
 * On failure *out is NULL and cl_last_error(NULL) says why. */
cl_status lattice_init(const cl_model* model, const cl_grid* grid, const cl_init* init, void* cuda_stream,
                       cl_lattice** out);

/* Advance nsteps full time steps with the handle's integrator (sections
 * 4.2.1, 4.2.3, 4.3.2, 5.3.1): fused drift / stencil / kick / reduction
 * passes on the device with the Friedmann update between passes, replayed as
 * CUDA graphs.  Asynchronous on the handle's stream.  nsteps >= 0. */
cl_status lattice_evolve(cl_lattice* h, int64_t nsteps);

/* Volume averages, energies, w, Delta_e and (U(1)) Delta_g at the current
 * time; synchronizes the stream.  For CL_INT_LF the momenta live half a step
 * behind the fields, so EK is the kinetic energy at t - dt/2. */
cl_status lattice_measure_means(cl_lattice* h, cl_means* out);

/* Number of spectrum bins, floor(sqrt(3) N/2) + 1. */
int32_t lattice_spectrum_bins(const cl_lattice* h);

/* Power spectrum of section 3.1 / 4.4.2 / 5.4.2,
 * Delta(k) = k^3/(2 pi^2) (dx/N)^3 <|f(n~)|^2>_R, averaged over the modes of
 * each shell |n~| in [b, b+1), with k_b = k_IR times the mean |n~| of the
 * shell.  field: scalar field index, or 0 for the complex U(1) scalar (Re and
 * Im summed), or for SU(2) 0 the doublet (four components summed) and 1 the
 * singlet chi.  what: 0 the field, 1 its momentum.  k, Delta (double) and
 * counts (int64) have lattice_spectrum_bins() entries (host memory).
 * Synchronizes the stream. */
cl_status lattice_measure_spectrum(cl_lattice* h, int32_t field, int32_t what, double* k, double* Delta,
                                   int64_t* counts);

/* Power spectra of the gauge fields (sections 5.4 and 6.3), with the shells,
 * k and normalisation of lattice_measure_spectrum and the components summed:
 *   sector 0: the U(1) field (CL_MODEL_U1, or CL_MODEL_SU2 with gauge_e_u1 > 0);
 *             what 0: E_i = piA_i / a^{1-alpha};
 *             what 1: B_i = sin(theta_jk)/(e dx^2) (compact) or theta_jk/(e dx^2)
 *             = eps_ijk D_j^+ A_k (non-compact), (i, j, k) cyclic, theta_jk the
 *             plaquette angle at n;
 *   sector 1: the SU(2) field (CL_MODEL_SU2); what 0: E_i^a = piB_i^a / a^{1-alpha};
 *             what 1: B_i^a = -2 q_a[U_jk(n)]/(g dx^2), the sigma^a part of the
 *             plaquette quaternion (the trace form of section 6.3).
 * CL_ERR_ARG when the model has no such sector.  Synchronizes the stream. */
cl_status lattice_measure_gauge_spectrum(cl_lattice* h, int32_t sector, int32_t what, double* k, double* Delta,
                                         int64_t* counts);

/* Array indices of get/set: scalar models: 0..n-1 the fields, 4..4+n-1
 * their momenta.  U(1): 0 Re phi, 1 Im phi, 4 Re pi, 5 Im pi, 8..10 the link
 * angles theta_i = e dx A_i (V_i = exp(-i theta_i)), 12..14 the electric
 * momenta piA_i. */
#define CL_FIELD(i) (i)
#define CL_MOMENTUM(i) (4 + (i))
#define CL_LINK(i) (8 + (i))
#define CL_EMOMENTUM(i) (12 + (i))
#define CL_SU2_LINK(i, c) (16 + 4 * (i) + (c))     /* quaternion component c of U_i */
#define CL_SU2_EMOMENTUM(i, a) (28 + 3 * (i) + (a)) /* piB_i^a */
/* CL_MODEL_SU2 with gauge_e_u1 > 0: the U(1) link angles and electric momenta
 * of the doublet are CL_LINK(i) and CL_EMOMENTUM(i); with n_fields = 2 the
 * real singlet chi and its momentum: */
#define CL_SINGLET 37
#define CL_SINGLET_MOMENTUM 38

/* Copy the full array `which` (N^3 doubles) to dst: host memory when
 * on_device = 0, device memory of the handle's device otherwise.
 * Synchronizes the stream. */
cl_status lattice_get_field(cl_lattice* h, int32_t which, double* dst, int32_t on_device);

/* Overwrite array `which` from src (N^3 doubles, host or device).  The
 * handle splits it into its mean and fluctuation.  Ordered on the stream. */
cl_status lattice_set_field(cl_lattice* h, int32_t which, const double* src, int32_t on_device);

/* The stored representation of array `which`, in the handle's precision:
 * N^3 elements (float for CL_FP32, double for CL_FP64) and the FP64
 * homogeneous value they fluctuate about, field = *mean + array (section 4.4's
 * volume average as the mean; the models without a mean split, U(1) and SU(2),
 * have mean 0 and their full arrays).  An FP32 lattice thus crosses the ABI in
 * half the bytes of lattice_get_field, with nothing lost: mean + array is, in
 * FP64, exactly the value lattice_get_field returns, and setting it back
 * reproduces those field values bit for bit.  dst / src are host memory
 * (on_device = 0) or device memory of the handle's device; both calls
 * synchronize the stream.  set rejects a non-finite mean, and a non-zero mean
 * for an array without a homogeneous part (CL_ERR_ARG). */
cl_status lattice_get_stored(cl_lattice* h, int32_t which, void* dst, double* mean, int32_t on_device);
cl_status lattice_set_stored(cl_lattice* h, int32_t which, const void* src, double mean, int32_t on_device);

/* Set the background: scale factor a and b = a' at program time t.  A NaN b
 * is replaced by the positive root of the Hubble constraint of the current
 * fields.  Under CL_BG_FLUID a and b are ignored and follow t.  Marks the
 * state as synchronized (momenta at the fields' time). */
cl_status lattice_set_background(cl_lattice* h, double a, double b, double t);

/* Checkpoint: raw arrays, means and background with a header and a CRC-32;
 * restore refuses files of another geometry, model or precision, or whose
 * CRC does not match (CL_ERR_IO).  Continuation after restore is bitwise
 * identical to uninterrupted evolution. */
cl_status lattice_save(cl_lattice* h, const char* path);
cl_status lattice_restore(cl_lattice* h, const char* path);

/* Free everything the handle owns.  NULL is accepted. */
cl_status lattice_destroy(cl_lattice* h);

/* ------------------------------------------------------------------ ensembles
 * Batched parameter scans (a workload pattern around the paper's method, not a
 * part of it): n independent lattices of the two-field model of section 8.1,
 * V = phi^2/2 + (q/2) phi^2 chi^2 (model->pexp = 2, n_fields = 2), that differ
 * in the coupling q[i], the size N[i] (multiples of 32, up to 1024) and the
 * seed seeds[i], advanced together: one persistent kernel launch per
 * integrator pass covers every member (velocity-Verlet VV2 or VV4, a time step
 * grid->dt common to all members, which must satisfy every member's stability
 * bound).  Each member is an ordinary lattice initialised as by lattice_init;
 * ensemble_member() lends its handle for measurements (do not destroy it).
 *
 * ensemble_observe writes, per member, CL_OBS_SIZE floats: the daughter-field
 * energy fraction (E_K[1] + E_G[1]) / rho, the equation of state w, and log10
 * of the chi power spectrum (section 3.1) at the 32 momenta
 * k_j = k_IR (k_max/k_IR)^((j + 1/2)/32), j = 0..31, interpolated linearly in
 * (log k, log Delta) between the shells.  kmax <= 0 selects k_max = N_min k_IR / 2
 * (N_min the smallest member: its Nyquist momentum along an axis; shells
 * beyond it are incomplete); a positive kmax is used as given, so that
 * ensembles of different sizes observe at the same momenta.  *t (may be NULL)
 * receives the program time.  Synchronizes the stream.
 *
 * q, N and seeds are host arrays of n entries, read during ensemble_init only;
 * obs is a host array of n x CL_OBS_SIZE floats (member-major).  The handle
 * owns every member and its device memory until ensemble_destroy (NULL is
 * accepted).  ensemble_init refuses with CL_ERR_ARG (reason in
 * cl_last_error(NULL), nothing left allocated): n < 1, a NULL array or struct, a
 * model other than the two-field pexp = 2 scalar model, an integrator other
 * than VV2 / VV4, an N that is not a multiple of 32 in [32, 1024], a q < 0 or
 * NaN, and any member that lattice_init would refuse (its reason is passed
 * on); allocation failures give CL_ERR_OOM.  ensemble_member refuses an index
 * outside [0, n). */
typedef struct cl_ensemble cl_ensemble;
#define CL_OBS_SIZE 34
cl_status ensemble_init(int32_t n, const cl_model* model, const double* q, const int32_t* N, const uint64_t* seeds,
                        const cl_grid* grid, const cl_init* init, void* cuda_stream, cl_ensemble** out);
cl_status ensemble_evolve(cl_ensemble* e, int64_t nsteps);
cl_status ensemble_observe(cl_ensemble* e, double kmax, float* obs, double* t);
cl_status ensemble_member(cl_ensemble* e, int32_t i, cl_lattice** out);
cl_status ensemble_destroy(cl_ensemble* e);

/* Tile shape of the ensemble pass, tile = {BX, BY, ZC, S}: a block of BX x BY
 * threads (each thread owns 4 consecutive FP32 or 2 FP64 sites along x) walks
 * ZC planes along z through S shared-memory stages.  Admissible shapes divide
 * every member's N, make whole warps of at most 256 threads, fit the shared
 * memory and 4 <= S <= 6; ensemble_init installs {8, 32, 32, 5} (FP32) or
 * {16, 16, 32, 5} (FP64) and fails with CL_ERR_ARG when that shape does not
 * fit.  set_tile rejects inadmissible shapes with CL_ERR_ARG (nothing
 * changed). */
cl_status ensemble_get_tile(const cl_ensemble* e, int32_t tile[4]);
cl_status ensemble_set_tile(cl_ensemble* e, const int32_t tile[4]);
/* Autotuner: times every admissible shape of a fixed candidate list on the
 * ensemble's own members (one warm-up and three timed integrator passes each,
 * CUDA events on the ensemble's stream), installs the fastest and leaves the
 * ensemble's physical state as it was (the timing passes write only the spare
 * copy of the fields and every member's scalar state is restored).  The first
 * min(n_tried, max_report) shapes tried and their mean pass times in ms go to
 * tiles (4 per shape) and ms when these are not NULL; *n_tried (may be NULL)
 * receives the number tried.  Synchronizes the stream. */
cl_status ensemble_autotune(cl_ensemble* e, int32_t max_report, int32_t* tiles, double* ms, int32_t* n_tried);

/* The CL_OBS_SIZE observables of ensemble_observe for one lattice of the
 * two-field model under a velocity-Verlet integrator (CL_ERR_ARG otherwise),
 * the 32 spectrum momenta spread between k_IR and kmax (kmax <= 0 selects
 * N k_IR / 2).  *t (may be NULL) receives the program time.
 * Synchronizes the stream. */
cl_status lattice_observe(cl_lattice* h, double kmax, float* obs, double* t);

/* Volume-averaged energies and means of caller-owned scalar fields, computed
 * without allocating any device memory.  The paper has no counterpart: this
 * serves callers that cannot call cudaMalloc -- programs that own all device
 * memory themselves (their own pool has claimed the GPU, or a loop must never
 * enter the allocator) -- and that hand over their arrays as they are.
 *
 * phi, pi: device arrays of n_fields x N^3 doubles (full fields, field-major,
 * site index (n3*N + n2)*N + n1), the momenta pi = a^{3-alpha} phi'.  out: a
 * device array of 10 doubles receiving {E_K[0], E_K[1], E_G[0], E_G[1],
 * <(lam/p)|phi|^p>, <(q/2)phi^2chi^2>, <phi_0>, <phi_1>, var[0], var[1]} with
 * the definitions of lattice_measure_means (sums taken about the value at
 * site 0, so a large mean does not cancel the variance).  model->kind must be
 * CL_MODEL_SCALAR; kIR fixes dx = 2 pi/(kIR N); a is the scale factor.
 * Enqueued on cuda_stream (NULL = legacy default stream); nothing is
 * synchronized.
 *
 * Scratch: a fixed device array of CL_NOALLOC_MAX_BLOCKS x 16 partial sums and
 * a counter (about 128 KiB), present on every GPU that loads the library until
 * the process exits.  The first call on a device looks its address up with
 * cudaGetSymbolAddress (that device current) and keeps it; every call then
 * enqueues one memset of the counter and one kernel launch.  All
 * calls share the array and it keeps the last call's contents; the counter is
 * cleared at the start of each call.  Calls that overlap on the GPU race on it.
 * Rejects n_fields > 2, N outside [2, CL_NOALLOC_MAX_N] and NULL pointers with
 * CL_ERR_ARG (reason in cl_last_error(NULL)).  CL_ERR_CUDA when a CUDA error
 * from earlier work is pending on the calling thread (it is left pending), or
 * when the launch fails (reason in cl_last_error(NULL)). */
#define CL_NOALLOC_MAX_BLOCKS 1024
#define CL_NOALLOC_MAX_N 2048
cl_status lattice_energies_noalloc(const cl_model* model, int32_t N, double kIR, double a, const double* phi,
                                   const double* pi, double* out, void* cuda_stream);

/* ------------------------------------------------------------------ surrogate
 * A multilayer perceptron fitted to ensemble observations (a workload pattern
 * around the paper's method, not a part of it): it maps n_in inputs (e.g.
 * log10 q and the program time) to n_out observables (e.g. the CL_OBS_SIZE
 * values of ensemble_observe), so that a parameter scan can be interpolated
 * between the simulated couplings.
 *
 *   H_0 = X,  Z_l = H_l W_l^T + b_l,  H_{l+1} = GELU(Z_l) for the `depth`
 *   hidden layers of `width` units,  Y = Z_depth (linear output),
 *   loss = mean over samples and outputs of (Y - T)^2,
 *   GELU(x) = x/2 (1 + erf(x/sqrt 2)).
 *
 * Every GEMM (forward, input gradient, weight gradient) runs on the tensor
 * cores with BF16 operands and FP32 accumulation; parameters, Adam moments
 * and the bias/GELU epilogues are FP32.  Weights start N(0, 1/fan_in) drawn by
 * Philox4x32-10 keyed by `seed`, biases zero.
 *
 * All array arguments are HOST pointers, row-major: X is n x n_in, Y and T
 * are n x n_out (float).  Calls are enqueued on cuda_stream (NULL = legacy
 * default stream) and synchronize it before returning.  The handle owns its
 * device memory; buffers grow with the largest batch seen.  Invalid sizes or
 * NULL pointers give CL_ERR_ARG (nothing is changed), allocation failures
 * CL_ERR_OOM, runtime failures CL_ERR_CUDA; the reason is in
 * cl_last_error(NULL). */
typedef struct cl_surrogate cl_surrogate;

typedef struct {
    int32_t epochs;      /* passes over the training set (>= 1) */
    int32_t batch;       /* minibatch rows (>= 1; clipped to n) */
    float lr;            /* Adam step size (> 0) */
    float beta1, beta2;  /* Adam decay rates (<= 0 selects 0.9, 0.999) */
    float eps;           /* Adam epsilon (<= 0 selects 1e-8) */
    float weight_decay;  /* L2 coefficient added to the weight gradients (biases exempt) */
    int32_t standardize; /* nonzero: fit on inputs and targets shifted and scaled to zero
                            mean and unit variance per column (the mapping is kept and
                            undone by surrogate_predict) */
    float lr_end;        /* >= 0: cosine decay of the step size from lr to lr_end over the
                            minibatch steps of this call; < 0: constant lr */
    int32_t shuffle;     /* nonzero: a fresh order of the samples every epoch (Fisher-Yates,
                            keyed by the handle's seed and its epoch count); 0: in order */
} cl_train_cfg;

/* n_in, n_out in [1, 1024], width in [1, 4096], depth (hidden layers) in
 * [1, 16].  *out receives the handle. */
cl_status surrogate_create(int32_t n_in, int32_t n_out, int32_t width, int32_t depth, uint64_t seed,
                           void* cuda_stream, cl_surrogate** out);
/* Number of trainable parameters: sum over layers of d_out*d_in + d_out. */
int64_t surrogate_param_count(const cl_surrogate* s);
/* Parameters as doubles in the order W_0 (d_1 x d_0 row-major), b_0, W_1, b_1, ...
 * (surrogate_param_count values).  set rounds them to FP32. */
cl_status surrogate_get_params(cl_surrogate* s, double* theta);
cl_status surrogate_set_params(cl_surrogate* s, const double* theta);
/* Loss and gradient of the raw (unstandardized) mean squared error over the n
 * rows of X and T in one batch, without changing the parameters; grad (may be
 * NULL) receives surrogate_param_count doubles in the order of get_params. */
cl_status surrogate_loss_grad(cl_surrogate* s, const float* X, const float* T, int64_t n, double* loss,
                              double* grad);
/* Adam training on n rows (n <= 2^24).  loss_history (may be NULL) receives
 * cfg->epochs floats: the mean squared error (in standardized units when
 * cfg->standardize) accumulated over each epoch's minibatches. */
cl_status surrogate_train(cl_surrogate* s, const float* X, const float* Y, int64_t n, const cl_train_cfg* cfg,
                          float* loss_history);
/* Y = network(X) for n rows (n <= 2^24), in the targets' original units. */
cl_status surrogate_predict(cl_surrogate* s, const float* X, int64_t n, float* Y);
/* Free everything the handle owns.  NULL is accepted. */
cl_status surrogate_destroy(cl_surrogate* s);

#ifdef __cplusplus
}
#endif

#endif /* CL_LATTICE_H */
