/*
 * droplet.h -- C ABI of the GB300 (sm_103a) implementation of one time step of
 * the VOF droplet-evaporation method of Saufi, Frassoldati, Faravelli & Cuoci,
 * "DropletSMOKE++: a comprehensive multiphase CFD framework for the
 * evaporation of multidimensional fuel droplets" (arXiv 2005.02867).
 *
 * The library advances, on one GPU, an isolated droplet on a uniform 2D
 * axisymmetric (r, z) or 3D Cartesian grid.  One call of droplet_step runs,
 * per time step, the segregated sequence of Sec. 3.1 (Fig. Scheme):
 *   thermodynamics (Sec. 2.5, Eqs. equilibrium / equilibirumyi / densitygas),
 *   evaporation flux (Sec. 2.4, Eqs. massflux, sumoverm, alphafunction),
 *   alpha source (Eq. alphasource), interface advection (Eq. advection),
 *   mixture properties (Sec. 2.7), energy (Eq. Teqn), species
 *   (Eq. speciesequation), momentum with the centripetal force
 *   (Eqs. magneticfield, magneticpotential, NavierStokesModified) and the
 *   variable-density pressure projection (Eq. pequation).
 *
 * Conventions
 *   - Every function returns an int status: 0 = success, < 0 = error
 *     (DROPLET_ERR_*).  droplet_strerror() names it.  No function aborts the
 *     process; a CUDA failure is reported as DROPLET_ERR_CUDA.
 *   - Units are SI.  Fields are FP64 on the host side of this ABI.
 *   - Grid layout: cell (i, j, k) has the linear index i + n0 (j + n1 k)
 *     (index 0 fastest).  Axisymmetric runs use n2 = 1 with axis 0 = r and
 *     axis 1 = z; 3D runs use x, y, z with z the streamwise (gravity / inflow)
 *     axis.  Face velocities of direction a are stored on the faces normal to
 *     a, with n_a + 1 entries along a (same index order).
 *   - The library owns all device memory it allocates; caller buffers are
 *     only read or written during the call that receives them.
 */
#ifndef DROPLET_H
#define DROPLET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DROPLET_OK                 0
#define DROPLET_ERR_ARG           -1  /* invalid configuration or argument            */
#define DROPLET_ERR_CUDA          -2  /* a CUDA runtime call failed                    */
#define DROPLET_ERR_NOT_CONVERGED -3  /* a linear solve hit its iteration cap          */
#define DROPLET_ERR_NONFINITE     -4  /* a non-finite value appeared in the state      */
#define DROPLET_ERR_SIZE          -5  /* host buffer size does not match the field     */
#define DROPLET_ERR_NOMEM         -6  /* device allocation failed                      */
#define DROPLET_ERR_IO            -7  /* checkpoint file could not be written or read  */
#define DROPLET_ERR_TIMEOUT       -8  /* a bounded device wait (grid barrier of a
                                         persistent solve) ran out; the step finished
                                         with that solve stopped where it was          */

/* diagnostic flag bits (droplet_diag_t.flags), accumulated since the last read */
#define DROPLET_FLAG_NO_INTERFACE   1u   /* sum f(alpha) m_raw V = 0: mdot set to 0         */
#define DROPLET_FLAG_MDOT_CAPPED    2u   /* mdot limited to rho_L alpha / dt somewhere     */
#define DROPLET_FLAG_ALPHA_CLIPPED  4u   /* alpha left [0, 1] and was clipped              */
#define DROPLET_FLAG_ADJ_NOT_FOUND  8u   /* an interface cell found no adjacent gas cell   */
#define DROPLET_FLAG_BOILING       16u   /* saturation mole fraction clamped below 1       */
#define DROPLET_FLAG_NONFINITE     32u   /* a NaN or infinity in alpha, T, omega, rho_G, mdot
                                            or a face velocity (seen by the diagnostics)  */

/* physics_mask bits */
#define DROPLET_PHYS_EVAP     1
#define DROPLET_PHYS_ENERGY   2
#define DROPLET_PHYS_SPECIES  4
#define DROPLET_PHYS_FLOW     8
#define DROPLET_PHYS_ALL     15

/* Problem statement of one droplet (Sec. 2, Sec. 3.2 boundary conditions,
 * case tables table1Dcases / tableGravityCases / tableForcedCases).
 * Copied by droplet_init; the caller keeps ownership. */
typedef struct droplet_config {
  int    geom;          /* 0 = 2D axisymmetric r-z, 1 = 3D Cartesian                  */
  int    n[3];          /* cells per axis; n[2] is ignored (taken as 1) when geom = 0  */
  double L[3];          /* domain extent [m]                                           */
  double xc[3];         /* droplet and fibre centre [m]; xc[0] = 0 when geom = 0        */
  double D0;            /* initial droplet diameter [m]                                */
  double T_drop;        /* initial liquid temperature [K]                              */
  double T_amb;         /* ambient (and inflow) temperature [K]                        */
  double P;             /* thermodynamic pressure [Pa]                                 */
  double g[3];          /* gravity per axis [m/s2]                                     */
  double u_inflow;      /* forced-convection inlet velocity along the streamwise axis  */
  int    bc_mode;       /* 0 natural convection (open inlet), 1 forced-convection inlet */
  int    eq_model;      /* 0 Raoult + Clausius-Clapeyron, 1 Peng-Robinson fugacities   */
  double Tb, Lv, M_l, rho_l, cp_l, k_l, mu_l, D_l;   /* liquid fuel                    */
  double M_g, cp_g, cp_v, k_g, mu_g, D_g;            /* inert gas; D_g at 1 bar; cp_v:
                                                        the vapour's heat capacity (the
                                                        gas mixture's c_p, and with
                                                        cp_v != cp_g the species-diffusion
                                                        enthalpy term of Eq. Teqn; the
                                                        adjoint needs cp_v = cp_g)     */
  double Tc, Pc, omega_ac, Tc_g, Pc_g, omega_g, kij; /* Peng-Robinson data            */
  double xi0;           /* centripetal potential intensity [m2/s2] (Eq. magneticpotential) */
  double fiber_radius;  /* D_f [m] (Eq. magneticpotential)                             */
  double dt;            /* time step [s]                                               */
  int    precision;     /* 0 = FP64 throughout, 1 = FP32 multigrid preconditioner     */
  double cg_rtol;       /* pressure solve: relative residual target                    */
  int    cg_maxit;      /* pressure solve: iteration cap                               */
  double helm_rtol;     /* T, omega, momentum solves: relative residual target         */
  int    helm_maxit;    /* T, omega, momentum solves: iteration cap                    */
  unsigned long long seed;  /* initial temperature perturbation seed (SplitMix64)      */
  double T_perturb;     /* relative amplitude of the initial T perturbation            */
  int    const_props_check; /* 1 = constant-property d2-law check mode                 */
  int    physics_mask;  /* DROPLET_PHYS_* bits of the active stages                     */
  double C_alpha;       /* interface-compression coefficient of the alpha flux         */
  int    mg_tile[2];    /* tile (cells along r / x, along z / y) of the temporal blocking of
                           the persistent multigrid smoothing on 2D levels; {0, 0}: 32 x 32,
                           or the autotuner's choice where it runs.  Owned cells get the same
                           values whatever the tile: a pure performance setting.  Each entry
                           0 or 8 .. 256; an odd entry is rounded up to the next even one. */
  int    wait_limit;    /* polls of the arrival counter after which a grid-barrier wait of a
                           persistent (cooperative) solve gives up; 0 = 2^22.  A wait that
                           runs out stops that solve and the step reports DROPLET_ERR_TIMEOUT
                           instead of hanging (a launch whose blocks are not all resident) */
  int    solver_select; /* 0 = by size: persistent solvers for the latency-bound sizes, the
                           launched multi-kernel ones beyond; 1 = the launched solvers at
                           every size (the path of the largest grids, e.g. for checking it
                           on small ones).  The answers agree to the solver tolerance. */
  double co_max;        /* threshold Courant number of the time step (Sec. 3.1: the step is
                           computed from a Courant threshold; the paper gives no value).
                           0 = the fixed step dt.  > 0: each step takes
                           dt^{n+1} = min(dt, co_max h_min / max|u^{n+1}|, 1.2 dt^n) over
                           every face velocity, the configured dt the upper bound, the first
                           step min(dt, co_max h_min / max|u^0|); the clock (diag t) is the
                           sum of the steps taken.  Not available with droplet_adjoint. */
  int    adv_scheme;    /* interface advection (Eq. advection): 0 = upwind + compressive flux
                           with a Zalesak limiter (C_alpha); 1 = geometric, the paper's
                           kind (Sec. 2.1): a plane per partly filled cell (Youngs normal),
                           one sweep per axis passing the liquid of each donor's swept slab,
                           volume-conserving whatever div u; FP64 in both precisions */
  double drho_l_dT;     /* temperature dependence of the liquid density (Sec. 2.7 takes rho_L
                           from correlations in T and lets it change the volume through
                           Eqs. alphasource and pequation): rho_L(T) = rho_l + drho_l_dT
                           (T - T_drop) [kg m^-3 K^-1], entering the mixture density, the
                           evaporation flux, the alpha source and its cap, the Poynting
                           factor, and the continuity source through
                           - alpha/rho_L D(rho_L)/Dt (with the time derivative and the
                           advective term of the gas density's), whose value the next alpha
                           source subtracts again; diag M_liq is then sum rho_L(T) alpha V.
                           0 = the constant rho_l.  Must keep rho_L > 0 at T_amb and Tb.
                           Not available with droplet_adjoint. */
  int    fiber;         /* the spherical fibre the droplet is placed around (Sec. 3.1.1: a
                           sphere of diameter 0.1 mm at the droplet's centre; Table
                           tableboundary, "sphere" row: no slip, zero gradient of alpha, T,
                           omega and p_rgh): 0 = none (the fibre is only the centre of the
                           potential xi), 1 = the cells whose centre lies closer than
                           fiber_radius to xc are solid.  Their faces carry u = 0 (pinned rows of
                           the momentum systems), no flux of alpha, T, omega or pressure, and
                           central differences reaching into them use the fluid cell's own
                           value; the solid cells hold alpha = 0, T = T_drop, omega = 0 and
                           are never interface or adjacent gas cells.  Either precision;
                           requires adv_scheme = 0 and drho_l_dT = 0; not available with
                           droplet_adjoint. */
} droplet_config;

/* Diagnostics of one droplet after the last completed step (Sec. 4 reports
 * the diameter decay, the surface temperature and the vaporisation rate). */
typedef struct droplet_diag_t {
  double t;             /* simulated time [s]                                         */
  long long step;       /* steps taken                                                 */
  double V_l;           /* liquid volume [m3] (2 pi sum alpha V in 2D)                 */
  double d_eq;          /* equivalent diameter (6 V_l / pi)^(1/3) [m]                  */
  double d2;            /* d_eq^2 [m2]                                                 */
  double mdot_tot;      /* evaporation rate of the last step [kg/s]                    */
  double K_norm;        /* K of Eq. alphafunction in the last step                     */
  double T_s_mean;      /* |grad alpha|-weighted mean temperature [K]                  */
  double M_liq, M_vap;  /* liquid and vapour masses [kg]                               */
  double vap_out_cum;   /* vapour mass that left through open boundaries [kg]          */
  double max_u;         /* max |face velocity| [m/s]                                   */
  double alpha_min, alpha_max;
  double clip_mass;     /* cumulative clipped liquid volume [m3]                       */
  int    its_p, its_T, its_w, its_u;   /* iterations of the last step's solves        */
  double res_p;         /* final relative residual of the last pressure solve          */
  unsigned flags;       /* DROPLET_FLAG_* accumulated since the previous droplet_diag  */
} droplet_diag_t;

typedef struct droplet_ctx droplet_ctx;   /* opaque; owns all device memory */

/* field identifiers for droplet_get_field / droplet_set_field */
enum droplet_field {
  DROPLET_F_ALPHA = 0, DROPLET_F_T = 1, DROPLET_F_OMEGA = 2, DROPLET_F_P = 3, DROPLET_F_RHOG = 4,
  DROPLET_F_U0 = 5, DROPLET_F_U1 = 6, DROPLET_F_U2 = 7,
  /* intermediates of the last step (read only) */
  DROPLET_F_MDOT = 8, DROPLET_F_MRAW = 9, DROPLET_F_ALPHA_STAR = 10, DROPLET_F_DP = 11, DROPLET_F_S = 12,
  DROPLET_F_USTAR0 = 13, DROPLET_F_USTAR1 = 14, DROPLET_F_USTAR2 = 15, DROPLET_F_RHOG_OLD = 16,
  DROPLET_F_OMEGA_PINNED = 17,
  /* the liquid's expansion term alpha/rho_L D(rho_L)/Dt of the last continuity source
     (cell field), which the next alpha source subtracts: part of the step's state, and
     writable, with a temperature-dependent liquid density (drho_l_dT != 0) only */
  DROPLET_F_EXPAND = 18,
  DROPLET_F_COUNT = 19
};

/* Create a context for n_droplets independent droplets (cfgs[0..n-1], each
 * with its own grid, conditions and precision) and set the initial state of
 * Sec. 3.3: alpha from sub-cell sampling of the sphere, the steady spherical
 * conduction profile of T, the quasi-steady Stefan profile of the vapour,
 * u = 0, p_rgh = 0.  cuda_stream is a cudaStream_t (NULL = the legacy default
 * stream, replaced by an internal blocking stream) on which every later call
 * orders its work.  A batch (n_droplets > 1) steps all droplets in one CUDA
 * graph per step, one branch per droplet on a stream of its own; at creation
 * an autotuner times a few steps for each candidate block cap of the
 * reduction kernels (the state is restored afterwards) and keeps the fastest.
 * On success *out receives the context.  Errors: DROPLET_ERR_ARG (bad
 * dimensions, droplet not inside the domain, dt <= 0, unsupported option),
 * DROPLET_ERR_SIZE (the pressure multigrid halves the grid while every active
 * dimension is even and above 2; when the level where that stops is too large
 * for the one-block coarse solve's shared memory, e.g. a large grid with an odd
 * dimension, the grid is refused), DROPLET_ERR_NOMEM, DROPLET_ERR_CUDA. */
int droplet_init(const droplet_config* cfgs, int n_droplets, void* cuda_stream, droplet_ctx** out);

/* Advance every droplet by n_steps time steps (the stage list of Sec. 3.1):
 * one launch of the captured step graph per step (captured at the first call;
 * while profiling, the kernels are launched one by one instead).  Returns when
 * the steps have finished (one stream synchronisation per call).
 * DROPLET_ERR_NOT_CONVERGED is returned when a linear solve of any droplet
 * reached its cap, DROPLET_ERR_TIMEOUT (which takes precedence) when a
 * grid-barrier wait of a persistent solve ran out (wait_limit); in both cases
 * the state is still advanced and the context stays usable. */
int droplet_step(droplet_ctx* ctx, int n_steps);

/* Copy the diagnostics of droplet `droplet` into the caller-owned *out
 * (synchronises the stream).  Clears the accumulated flags.  Returns
 * DROPLET_ERR_NONFINITE (with *out filled) when a diagnostic is not finite or
 * DROPLET_FLAG_NONFINITE is set: a NaN or infinity in a state field. */
int droplet_diag(droplet_ctx* ctx, int droplet, droplet_diag_t* out);

/* Number of doubles of field `field_id` (cells, or faces for velocities). */
int droplet_field_size(droplet_ctx* ctx, int droplet, int field_id, size_t* n);

/* Copy a field to the caller-owned host array `host` of exactly n doubles
 * (DROPLET_ERR_SIZE otherwise).  Synchronises the stream. */
int droplet_get_field(droplet_ctx* ctx, int droplet, int field_id, double* host, size_t n);

/* Overwrite a state field (ALPHA, T, OMEGA, P, RHOG, U0..U2) from n host doubles. */
int droplet_set_field(droplet_ctx* ctx, int droplet, int field_id, const double* host, size_t n);

/* Solve one symmetric positive-definite box system of the kind the step
 * assembles for the energy, species and momentum equations (Sec. 3.1: implicit
 * Euler with the orthogonal Laplacian), with the library's Jacobi-preconditioned
 * conjugate gradient.  The unknowns sit on an m[0] x m[1] x m[2] box (index 0
 * fastest); the operator is
 *   y_P = D_P x_P + sum_a [ c_a[P] (x_P - x_{P-e_a}) + c_a[P+e_a] (x_P - x_{P+e_a}) ],
 * i.e. the coupling of each pair of neighbours is stored at its high cell, and
 * c_a[P] is ignored where P_a = 0.  D, c0, c1, b are device arrays of
 * m0*m1*m2 doubles; c2 is NULL when m[2] = 1; x (device) holds the initial guess
 * and receives the solution.  Stops at ||b - A x|| <= rtol ||b|| or after maxit
 * iterations (DROPLET_ERR_NOT_CONVERGED).  Work is enqueued on cuda_stream and
 * the call returns when the solve has finished; *its and *relres (host, may be
 * NULL) receive the iteration count and the final relative residual.
 * Allocates its workspace with cudaMalloc for the duration of the call. */
int droplet_box_solve(const int m[3], const double* D, const double* c0, const double* c1, const double* c2,
                      const double* b, double* x, double rtol, int maxit, void* cuda_stream, int* its,
                      double* relres);

/* droplet_box_solve for callers that cannot allocate device memory: a host
 * framework whose device memory all comes from its own pool or arena, code
 * that must not call cudaMalloc / cudaFree while other streams are in flight
 * (those calls can synchronise the device), or a tight loop where allocation
 * latency matters.  The paper has no counterpart; this is a service of the
 * library.
 *
 * Same arguments, operator, stopping rule and statuses as droplet_box_solve.
 * The solver's work vectors live in one static device array inside the
 * library, sized for at most DROPLET_NOALLOC_MAX_UNKNOWNS unknowns (about
 * 10.5 MB, held by every GPU that loads the library until the process
 * exits); a larger box is rejected with DROPLET_ERR_SIZE before any work is
 * enqueued.  The call makes no cudaMalloc, cudaFree, pinned-memory or other
 * allocating call.  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress, which allocates nothing; no address is
 * kept between calls).  Under lazy module loading (the CUDA default) the array
 * is placed in device memory at the first call on a device: make that first
 * call early if the caller's own pool is to take the rest of the memory.  No
 * call can be captured into a CUDA graph (each reads the solver's state back
 * and synchronises the stream): on a stream under capture the call returns
 * DROPLET_ERR_ARG before anything is enqueued.  Every call reuses the same array and
 * initialises what it needs, so calls must not overlap on the GPU: two solves
 * running at once on different streams would race on the array. */
#define DROPLET_NOALLOC_MAX_UNKNOWNS 262144
int droplet_box_solve_noalloc(const int m[3], const double* D, const double* c0, const double* c1,
                              const double* c2, const double* b, double* x, double rtol, int maxit,
                              void* cuda_stream, int* its, double* relres);

/* Kernel classes timed by droplet_profile (algorithmic bytes per launch in brackets,
 * w = word size of the launch, d = 2 or 3 active axes, N = unknowns of the launch):
 *   0 MG_SMOOTH   red-black Gauss-Seidel half sweep    [(2.5 + d) N w; FP64: (2d + 1) N/2 instructions;
 *                                                        an FP32 level's first half sweep after
 *                                                        the coarse correction also prolongs it:
 *                                                        + N_coarse w, and no MG_PROLONG launch]
 *   1 SPMV        CG operator application + dot        [(3 + d) N w; FP64: (2d + 2) N instructions,
 *                                                        the diagonal form a_P x_P - sum c x_N]
 *   2 UPDATE      CG x/r update + dot                  [Jacobi 8 N w (x, r in and out, p, Ap,
 *                                                        1/diag in, z out); MG-PCG 6 N 8 (+ 4 N
 *                                                        with an FP32 hierarchy); FP64: 5 N
 *                                                        (Jacobi), 3 N]
 *   3 MG_RESTRICT residual + restriction               [(3 + d) N w + N/2^d w; FP64: (4d + 3) N]
 *   4 MG_PROLONG  injection prolongation (FP64 levels) [(2 + 1/2^d) N w; FP64: N]
 *   5 MOM_ASSEMBLE momentum system assembly            [(12 + 2d) N 8]
 *   6 SCALAR_ASSEMBLE energy / species assembly        [(12 + 2d) N 8]
 *   7 PCG_PERSIST the whole Jacobi-preconditioned CG of one to three Helmholtz
 *                 systems in one persistent launch     [setup, then (11 + d) N w per
 *                                                       iteration of each system]
 * (w = 8 for FP64 launches, 4 for FP32 ones.  The FP64 figures count binary64 pipe
 * instructions the arithmetic needs, an FMA once: on GB300 that pipe, not HBM, bounds
 * the FP64 stencils.  The assembly classes carry none: their issued counts come from
 * counter captures.)
 * The Helmholtz systems solve with the persistent kernel of class 7 in mixed
 * precision at every size, in FP64 up to 2^22 cells.  Single droplets of at most
 * 2^22 cells, and the droplets of a batch, solve the pressure with a persistent
 * kernel too: class 0 then times the whole multigrid-preconditioned CG (one launch
 * per solve; bytes: per iteration the level-0 FP64 CG vectors, each grid level's
 * operator, b and x once per smoothing side, the transfers and the coarse tail,
 * times the iterations); classes 2 - 4 then stay empty.                            */
#define DROPLET_KCLASS_COUNT 8

/* Start (enable = 1) or stop (0) timing every launch of the kernel classes above
 * with CUDA events on the context's stream; starting clears the totals. */
int droplet_profile(droplet_ctx* ctx, int enable);

/* Totals since profiling started for one kernel class: summed event time [ms],
 * number of launches, summed algorithmic bytes and summed binary64 instructions
 * (flops64, may be NULL; the figures above, an FMA counted once; launches computing in
 * FP32 add none).  Synchronises. */
int droplet_profile_read(droplet_ctx* ctx, int kclass, double* ms_total, long long* launches, double* bytes_total,
                         double* flops64);

/* Number of kernel launches the library has issued for this context so far. */
int droplet_launch_count(droplet_ctx* ctx, long long* launches);

/* Hand-written discrete adjoint of the step.  Two forms:
 *  - without flow (physics_mask = EVAP | ENERGY | SPECIES): evaporation flux with
 *    the K normalisation of Eq. alphafunction, alpha source of Eq. alphasource,
 *    energy Eq. Teqn, species Eq. speciesequation with the liquid pinned to the
 *    Raoult saturation value, gas density Eq. densitygas; natural boundaries;
 *  - with flow (all four physics terms, adv_scheme 0, either boundary mode): also
 *    the convective part of the evaporation flux, the FCT advection of alpha
 *    (Eq. advection), convection in energy and species, the momentum predictor
 *    with buoyancy and the centripetal force (Eqs. NavierStokesModified,
 *    magneticfield), the Stefan source and the variable-density pressure equation
 *    (Eq. pequation) and the velocity correction; the ambient temperature then
 *    also enters through the energy equation's inflow boundary values.
 * Both: FP64, Raoult, one droplet, constant liquid density, fixed dt.
 * Starting from the initial state of droplet_init (step 0) it runs n_steps
 * forward, keeping the state every ckpt_every steps, and returns
 *   *J = (1/n_steps) sum_n mdot_tot^n   (mean evaporation rate, kg/s)
 * and, through a reverse sweep that recomputes each segment from its
 * checkpoint, the derivatives of J with respect to T_amb (through the initial
 * temperature profile and, with flow, the boundary values), D_g, and the
 * initial temperature field (dJ_dT0, host array of nT0 = cell-count doubles).
 * Any gradient pointer may be NULL; with all three NULL only J is computed.  The
 * branch decisions of the forward step (interface cells, adjacent cells, the
 * mdot cap, upwind sides, minmod, van Leer and limiter choices, clipping, pinned
 * cells) are held fixed.  Every linear system is symmetric: its adjoint is the
 * same system solved again (to a relative residual of 1e-14) for the adjoint
 * right-hand side.  The context is left at the state after n_steps.  Errors:
 * DROPLET_ERR_ARG (another physics mask, precision, equilibrium model,
 * adv_scheme, co_max or drho_l_dT, a batch, or step != 0), DROPLET_ERR_SIZE,
 * DROPLET_ERR_NOMEM (work memory: one state per checkpoint plus
 * ckpt_every + 1 states and about 40 cell and 12 face arrays with flow),
 * DROPLET_ERR_NOT_CONVERGED (a solve reached its cap; results still returned). */
int droplet_adjoint(droplet_ctx* ctx, int n_steps, int ckpt_every, double* J, double* dJ_dTamb, double* dJ_dDg,
                    double* dJ_dT0, size_t nT0);

/* One step of the flow adjoint, for checking it against finite differences: from
 * the context's current state s (which must satisfy the flow form's conditions
 * above, at any step) it takes one step s' = F(s) with the solves started from s
 * alone (as after droplet_set_field) and returns
 *   lam_prev = (dF/ds)^T lam_next + mdot_weight d(mdot_tot)/ds
 * and dpar[0], dpar[1] = the same derivative of <lam_next, F(s)> + mdot_weight
 * mdot_tot with respect to T_amb (boundary values; the initial field is not part of
 * a step) and D_g.  State vectors (host, n doubles): alpha, T, omega, p_rgh (each N
 * cells, field order), then the face velocities of each active direction
 * (droplet_field_size of u0, u1, u2).  dpar may be NULL.  The context is left at
 * s'.  Errors as droplet_adjoint; DROPLET_ERR_SIZE when n is not the state size. */
int droplet_adjoint_vjp(droplet_ctx* ctx, const double* lam_next, double* lam_prev, size_t n, double mdot_weight,
                        double* dpar);

/* Forward check of the flow adjoint's stage formulas: takes one step from the
 * current state (as droplet_adjoint_vjp does) and evaluates, for each stage, the
 * formulas the adjoint differentiates; rel[k] (k < 20, nrel >= 20) receives
 * max |formula - forward kernel| / max |forward kernel| for: the FCT face fluxes
 * (low order, antidiffusive), alpha^L, R+, R-, alpha^{n+1}, m_raw; the diagonal,
 * right-hand side and couplings of the energy, species, momentum (all components)
 * and pressure systems; and the corrected velocities.  The context is left after
 * the step.  Errors as droplet_adjoint_vjp. */
int droplet_adjoint_check(droplet_ctx* ctx, double* rel, int nrel);

/* Checkpoint / resume.  droplet_save writes, for every droplet, its config, time,
 * step count, the accumulated diagnostics (clipped volume, vapour outflow) and the
 * state fields (alpha, T, omega, p_rgh, rho_G and the face velocities, FP64,
 * little-endian) to `path`, followed by the previous step's T, omega and face
 * velocities, from which the next step extrapolates the initial guesses of its
 * Helmholtz solves (a state set with droplet_set_field starts them from itself).  droplet_load reads such a file into a context
 * created with the same configs (byte-identical droplet_config structs, else
 * DROPLET_ERR_ARG) and continues from there: the next steps are bit-identical to
 * those of the saved run.  File errors: DROPLET_ERR_IO. */
int droplet_save(droplet_ctx* ctx, const char* path);
int droplet_load(droplet_ctx* ctx, const char* path);

/* Round n doubles (host array `in`) to binary32 on the device with the integer-pipe
 * conversion the mixed-precision (precision 1) assembly kernels use, and widen the
 * results back to binary64 with their exact integer-pipe widening: out32[i] and
 * back64[i] (host arrays).  The paper has no counterpart: the entry point exists so
 * that the conversion can be checked against IEEE 754 round-to-nearest-even.  Runs
 * on the current device and synchronises.  Errors: DROPLET_ERR_ARG (a NULL array or
 * n > 2^30), DROPLET_ERR_NOMEM, DROPLET_ERR_CUDA. */
int droplet_round_f32(const double* in, float* out32, double* back64, size_t n);

/* The binary64 reciprocal the step kernels use in place of a division (a binary32
 * seed refined by two Newton-Raphson steps; a division outside binary32's normal
 * range), applied on the device to n doubles of the host array `in`, results in the
 * host array `out`.  No counterpart in the paper: it exists so that the reciprocal
 * can be checked against the correctly rounded 1 / x (at most one ulp apart).  Runs
 * on the current device and synchronises.  Errors: DROPLET_ERR_ARG (a NULL array or
 * n > 2^30), DROPLET_ERR_NOMEM, DROPLET_ERR_CUDA. */
int droplet_rcp_f64(const double* in, double* out, size_t n);

/* Measured binary64 fused multiply-add throughput of the current device in TFLOP/s
 * (an FMA counts two operations): eight independent FMA chains per thread on every
 * SM, the best of five timed launches after a warm-up, CUDA events on the legacy
 * default stream.  No counterpart in the paper: it gives the FP64-bound stencil
 * kernels a measured roof (on GB300 the binary64 pipe retires about two FMAs per SM
 * per clock).  Synchronises the device.  Errors: DROPLET_ERR_ARG (NULL),
 * DROPLET_ERR_NOMEM, DROPLET_ERR_CUDA. */
int droplet_fp64_rate(double* tflops);

/* Block until all work enqueued by the context has finished. */
int droplet_sync(droplet_ctx* ctx);

/* Release every device allocation of the context (NULL is accepted). */
void droplet_free(droplet_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* droplet_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* DROPLET_H */
