/*
 * sphvisc: the semi-implicit viscous solve of SPH on one GB300 (sm_103a).
 *
 * C ABI of the library.  It implements the hot path of Bilotta et al.,
 * "A numerically robust, parallel-friendly variant of BiCGSTAB for the
 * semi-implicit integration of the viscous term in Smoothed Particle
 * Hydrodynamics" (arXiv 2206.14780):
 *
 *   A(dt) V = B(dt)            Sec. 3.2, "Shared formulation"
 *
 * one sparse N x N matrix shared by the d = 3 velocity components, applied
 * matrix-free over cell-list neighbours and solved with the restructured
 * BiCGSTAB of Sec. 4.2.
 *
 * Conventions for every entry point:
 *  - Pointers marked (device) are CUDA device pointers owned by the caller;
 *    pointers marked (host) are host memory owned by the caller.  The library
 *    never frees caller memory.
 *  - Arrays are in the caller's particle order.  The library keeps its own
 *    cell-sorted copy inside an opaque sph_neighbors handle.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; entry points that return host-visible
 *    results (reports, counts) synchronise that stream before returning.
 *  - Every call returns an sph_status and never aborts.  On error the
 *    thread-local message sph_last_error() says what failed.  Output buffers
 *    are unspecified after an error.
 *  - Device workspace is allocated by sph_build_neighbors / sph_visc_setup /
 *    the first solve on a handle, and reused afterwards; it is released by
 *    sph_neighbors_destroy.
 */
#ifndef SPHVISC_H
#define SPHVISC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPH_OK = 0,
  SPH_ERR_INVALID = 1,     /* bad argument (null pointer, size, box, option)      */
  SPH_ERR_CUDA = 2,        /* a CUDA runtime call failed                           */
  SPH_ERR_CAPACITY = 3,    /* a particle has more neighbours than max_neighbors    */
  SPH_ERR_NONFINITE = 4,   /* NaN or Inf in an input or in the solver's scalars    */
  SPH_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                   */
  SPH_NOT_CONVERGED = 6,   /* maxit reached, or the true residual stayed above rtol */
  SPH_ERR_NOMEM = 7        /* device allocation failed                             */
} sph_status;

/* particle types (the set F of fluid particles and W of boundary particles) */
enum { SPH_FLUID = 0, SPH_WALL = 1 };
/* boundary model: dummy (Adami; Eq. implicit-system-dummy-full) or dynamic
   (Eq. implicit-system-dyn-full) */
enum { SPH_BC_DUMMY = 0, SPH_BC_DYNAMIC = 1 };
/* average viscosity mubar_ab (Sec. 2.3): harmonic 2 mu_a mu_b/(mu_a+mu_b) or
   arithmetic (mu_a+mu_b)/2 */
enum { SPH_MEAN_HARMONIC = 0, SPH_MEAN_ARITHMETIC = 1 };
/* per-component solver states (Sec. 4.2, "Stopping criterion") */
enum { SPH_CONVERGED = 0, SPH_STALLED = 1, SPH_PROGRESSING = 2 };
/* solve precision */
enum {
  SPH_PREC_MIXED = 0,   /* FP32 operator/vectors, FP64 dots+scalars, FP64 refinement */
  SPH_PREC_FP64 = 1     /* every vector and coefficient in FP64                      */
};

/* One particle set.  All arrays have n entries, caller order, (device). */
typedef struct {
  int64_t n;               /* number of particles (fluid + wall), >= 1          */
  const float* pos;        /* [n][4]: x, y, z (m) and mass m (kg)               */
  const float* rho;        /* [n]: density rho (kg/m^3), > 0                    */
  const float* mu;         /* [n]: dynamic viscosity mu (Pa s), > 0; App. A
                              advises storing mu rather than nu*rho             */
  const uint8_t* ptype;    /* [n]: SPH_FLUID or SPH_WALL                        */
  double lo[3], hi[3];     /* box; on a periodic axis hi-lo is the period and
                              hi-lo >= 3 R h (R h: the kernel's support
                              radius); particles on open axes may lie
                              outside [lo, hi) (they are clamped into the edge
                              cells, which keeps the search exact)              */
  int32_t periodic[3];     /* 1 = periodic axis (minimum image)                 */
  float h;                 /* smoothing length                                  */
  int32_t kernel;          /* SPH_KERNEL_WENDLAND (support radius 2h, default)
                              or SPH_KERNEL_GAUSSIAN (support radius 3h)        */
} sph_scene;

/* Smoothing kernels (Sec. 5.2, "Smoothing kernel choice"), W = w(r/h)/h^3 and
 * the gradient factor |F| = |f(r/h)|/h^5:
 *   SPH_KERNEL_WENDLAND: w = 21/(16 pi) (1 - q/2)^4 (2q + 1),
 *                        |f| = 105/(128 pi) (2 - q)^3, zero for q >= 2;
 *   SPH_KERNEL_GAUSSIAN: the normalised Gaussian truncated at k = 3,
 *                        w = (e^{-q^2} - e^{-9}) / w_G, |f| = 2 e^{-q^2} / w_G,
 *                        w_G = pi^{3/2} erf(3) - (2 pi / 3) e^{-9} 3 (3 + 18);
 *                        about 250 neighbours at h = 1.3 dx (max_neighbors of
 *                        at least 320 or so for jittered particles).
 * The neighbour lists, the coefficients of A(dt), the dummy-wall Shepard rows,
 * the v^n start with its wall closure and the Papanastasiou pass follow the
 * chosen kernel; the on-the-fly apply and the learned warm start's features
 * are written for the Wendland kernel and return SPH_ERR_INVALID otherwise. */
enum { SPH_KERNEL_WENDLAND = 0, SPH_KERNEL_GAUSSIAN = 1 };

/* Opaque neighbour structure: cell-sorted particle copy, permutation and the
   sliced-ELL neighbour lists (Sec. 5.2: a particle sees about 80 neighbours at
   h = 1.3 dp; App. A: relative positions evaluated as one difference). */
typedef struct sph_neighbors sph_neighbors;

/* Build (or rebuild in place, if *handle is non-NULL) the neighbour lists.
 * alpha is a neighbour of beta iff alpha != beta and |r_ab|^2 < (R h)^2, R = 2
 * (Wendland) or 3 (Gaussian), with
 * r_ab the minimum image on periodic axes, decided exactly as in float64 on
 * the float32 positions (a float32 test with a safety band, then a float64
 * recheck inside the band).
 * max_neighbors: capacity per particle, 1..1024; a larger count returns
 *   SPH_ERR_CAPACITY.  The lists are built in one pass into a layout of that
 *   capacity: 4 * max_neighbors bytes of device memory per particle (512 B at
 *   the default 128).
 * Copies pos/rho/mu/ptype into the handle: the scene arrays may be freed after
 * the call returns. */
sph_status sph_build_neighbors(const sph_scene* scene, int32_t max_neighbors,
                               sph_neighbors** handle, void* stream);

/* Host query: number of particles, total neighbour pairs, largest row. */
sph_status sph_neighbors_info(const sph_neighbors* handle, int64_t* n, int64_t* nnz,
                              int32_t* max_count);

/* Export the lists as CSR in caller order with each row ascending.
 * offsets (device) [n+1] int64; idx (device) [nnz] int32.  Synchronises. */
sph_status sph_neighbors_export(const sph_neighbors* handle, int64_t* offsets, int32_t* idx,
                                void* stream);

/* Replace the per-particle viscosity (caller order, device [n]) without
 * rebuilding the lists (the lagged viscosity of Sec. 3.3). */
sph_status sph_set_viscosity(sph_neighbors* handle, const float* mu, void* stream);

sph_status sph_neighbors_destroy(sph_neighbors* handle);

/* Parameters of the viscous matrix A(dt) (Sec. 3.2). */
typedef struct {
  double dt;               /* time step of the implicit system, > 0              */
  int32_t boundary;        /* SPH_BC_DUMMY or SPH_BC_DYNAMIC                      */
  int32_t mean;            /* SPH_MEAN_HARMONIC or SPH_MEAN_ARITHMETIC            */
} sph_visc_params;

/* Compute and cache the matrix coefficients of A(dt) on the handle:
 *   fluid row b:  A_bb = 1 + dt sum_a c_ab,  A_ba = -dt c_ab,
 *                 c_ab = 2 mubar_ab m_a |F_ab| / (rho_a rho_b)   (Eq. kab;
 *                 |F| reading: the printed signs make the rows anti-diffusive)
 *                 a wall neighbour uses mubar = mu_b (the row's own mu)
 *   dummy wall:   A_bb = 1, A_ba = W_ba / sum_{a' fluid} W_ba' over fluid a
 *                 (Eq. implicit-system-dummy-full); an empty sum gives an
 *                 identity row
 *   dynamic wall: identity row (Eq. implicit-system-dyn-full)
 * and the Jacobi diagonal (App. B).  Coefficients are computed in float64 and
 * stored as a float32 pair (hi + lo).  Called implicitly by apply/solve when
 * the parameters change. */
sph_status sph_visc_setup(sph_neighbors* handle, const sph_visc_params* params, void* stream);

/* y = A(dt) v in float32 (the operator of the inner iterations), with the
 * fluid rows in the difference form v_b + dt sum_a c_ab (v_b - v_a).
 * v, y: (device) [n][4] float (xyz, w ignored / written 0), caller order;
 * v and y must not overlap. */
sph_status sph_visc_apply(sph_neighbors* handle, const sph_visc_params* params, const float* v,
                          float* y, void* stream);

/* The same y = A v as sph_visc_apply, with every coefficient recomputed from the
 * particle data inside the apply (the paper's own GPU form, App. A and App. B):
 * c_ab = 2 mubar m_a |F_ab| / (rho_a rho_b) of Eq. kab per neighbour pair in
 * float32, dummy-wall rows by the Shepard sums of Eq. dummyvel, row kinds as in
 * sph_visc_setup.  It streams the 4-byte neighbour list instead of the stored
 * 8-byte (index, coefficient) entries and gathers each neighbour's position,
 * volume and viscosity besides its velocity.  Arguments, layout and errors as
 * sph_visc_apply; the first call after a rebuild or new viscosities packs the
 * per-particle geometry (device memory owned by the handle). */
sph_status sph_visc_apply_otf(sph_neighbors* handle, const sph_visc_params* params, const float* v,
                              float* y, void* stream);

/* Largest particle count sph_visc_apply_noalloc accepts (after rounding n up
 * to a multiple of 32). */
#define SPH_NOALLOC_MAX_ROWS 262144

/* Same result as sph_visc_apply, for callers that must not allocate device
 * memory at the time of the call: e.g. a plugin whose host framework owns all
 * device memory through its own pool (a cudaMalloc would fail or fragment that
 * pool), or a time-step loop that forbids allocation calls.  The paper has no
 * counterpart; this is an interface convenience.
 *  - Allocates nothing: no cudaMalloc/cudaFree and no allocating library call.
 *    Its scratch (the cell-sorted copies of v and y, 32 bytes per row) is a
 *    file-scope device array of 2 * SPH_NOALLOC_MAX_ROWS float4 (8 MiB) that
 *    every GPU loading this library keeps until the process exits.
 *  - The coefficients for `params` must already be on the handle
 *    (sph_visc_setup, or an apply/solve with the same params; those calls may
 *    allocate); otherwise SPH_ERR_INVALID.
 *  - n rounded up to 32 above SPH_NOALLOC_MAX_ROWS: SPH_ERR_INVALID.
 *  - The first call on a device looks up the array's device address there
 *    (cudaGetSymbolAddress, once per device, with that device current); make
 *    that first call before any stream capture.  The address is kept for the
 *    life of the process: after a cudaDeviceReset of that device it is stale,
 *    so a process that resets a device must not call this entry point on it
 *    again.
 *  - v and y must not overlap (any overlap of their n x 16-byte ranges:
 *    SPH_ERR_INVALID).
 *  - All calls share the one array: calls whose work overlaps on the GPU (other
 *    streams, other host threads) race on it.  Every row it reads is written
 *    by the same call first, so stale contents from a previous call are never
 *    used. */
sph_status sph_visc_apply_noalloc(sph_neighbors* handle, const sph_visc_params* params,
                                  const float* v, float* y, void* stream);

/* r = b - A(dt) x in float64 with the float64 coefficients (the true residual).
 * x, b, r: (device) [n][3] double, caller order. */
sph_status sph_visc_residual(sph_neighbors* handle, const sph_visc_params* params,
                             const double* x, const double* b, double* r, void* stream);

typedef struct {
  double rtol;             /* accept when ||b - A x||_2 / ||b||_2 <= rtol (all
                              three components jointly, float64 true residual);
                              default 1e-6                                       */
  double eps_inner;        /* floor of the relative tolerance of one inner
                              BiCGSTAB pass on its Jacobi-scaled recursive
                              residual (the paper's tau^2 = max(eps^2 b.b,
                              FLT_MIN), Sec. 4.1); each pass asks for
                              max(eps_inner, rtol ||b|| / (4 ||r64||)); 0 = 2e-2.
                              Each pass restarts BiCGSTAB from the float64 true
                              residual with a fresh shadow vector r0^, which on
                              stiff systems takes fewer iterations in total than
                              one long float32 recursion near its accuracy
                              limit (~kappa * 2^-24)                             */
  int32_t maxit;           /* cap on inner iterations summed over passes          */
  int32_t max_refine;      /* cap on refinement passes                            */
  int32_t precision;       /* SPH_PREC_MIXED or SPH_PREC_FP64                     */
  int32_t merged_reductions; /* 0: three reductions per iteration, gamma and |r|^2
                              from direct dots as the paper does; 1: two, with
                              gamma' = r0^.r* - w r0^.Ar*, |r|^2 = |r*|^2 - 2w
                              r*.Ar* + w^2 |Ar*|^2                               */
  int32_t chunk;           /* iterations launched between host checks (>= 1)      */
  int32_t jacobi;          /* 1: Jacobi scaling (App. B): left scaling of the
                              BiCGSTAB system, z = D^-1 r in the CG; 0: none
                              (CG only: BiCGSTAB returns SPH_ERR_INVALID)        */
  int32_t apply_form;      /* 0: the autotuner picks the operator apply's row-loop
                              form per phase (default); k = 1..6: use form k - 1
                              (sph_profile_counters.apply_variant numbering)     */
  int32_t launch_mode;     /* 0: the BiCGSTAB loop's kernels are programmatic
                              dependent launches, each launch processed while its
                              predecessor still runs (default); 1: plain
                              stream-ordered launches.  Same results either way   */
  int32_t method;          /* SPH_SOLVER_BICGSTAB (default) or SPH_SOLVER_CG      */
} sph_solve_opts;

/* Inner iteration of sph_visc_solve (sph_solve_opts.method).
 * SPH_SOLVER_BICGSTAB: the restructured BiCGSTAB of Sec. 4.2 on the Jacobi-scaled
 *   system (App. B); needs jacobi = 1.
 * SPH_SOLVER_CG: the rotated conjugate gradient of Sec. 4.1 (second listing: p
 *   update first, beta and the convergence check last, alpha = 0 while r is
 *   not small is a stall, single exit), preconditioned with z = D^-1 r when
 *   jacobi = 1 (App. B).  It needs a symmetric matrix: the dynamic boundary
 *   model (the dummy model returns SPH_ERR_INVALID) with one particle mass, for
 *   which the fluid block is symmetric (Sec. 4).  Identity rows start at x = b,
 *   their exact value, so every residual vanishes on the walls and the
 *   iteration runs on the reduced fluid system of Sec. 4 whatever the wall
 *   velocities.  One operator apply per iteration instead of two.  Mixed
 *   precision only; apply_form 0..4; merged_reductions is ignored. */
enum { SPH_SOLVER_BICGSTAB = 0, SPH_SOLVER_CG = 1 };

typedef struct {
  int32_t status;          /* same value the call returns                        */
  int32_t iters;           /* inner BiCGSTAB iterations, all passes              */
  int32_t refinements;     /* inner passes run (true-residual recomputations - 1)*/
  int8_t state[3];         /* last inner pass, per component (SPH_CONVERGED ...) */
  int8_t stalled_any[3];   /* 1 if the component stalled in any pass             */
  double true_rel_res;     /* ||b - A x||_2 / ||b||_2, float64, all components   */
  double true_rel_res_c[3];/* per component (absolute residual if b_c = 0)       */
} sph_solve_report;

/* Solve A(dt) X = B with the restructured BiCGSTAB (Sec. 4.2): per iteration
 *   p = r + beta p - alpha' A p;  delta = r0^.A p;  alpha = gamma/delta;
 *   r* = r - alpha A p;  x += alpha p;  omega = (r*.Ar*)/(Ar*.Ar*);
 *   r = r* - omega A r*;  x += omega r*;  gamma' = r0^.r;  alpha' = gamma'/delta;
 *   beta = alpha'/omega
 * with the paper's safeguards (delta = 0 sets alpha = alpha' = beta = 0 and the
 * component is stalled; the iteration completes and there is one exit point)
 * and the three per-component states.  In SPH_PREC_MIXED the iterations run in
 * float32 with float64 dots and scalars inside iterative refinement on the
 * float64 true residual.
 * b: (device) [n][3] double, the right-hand side B (Sec. 3.2: u^n + dt(f_P+g)
 *    for fluid rows, 2 u_w for dummy walls, u_w for dynamic walls).
 * x: (device) [n][3] double; in: initial guess, out: solution.
 * report: (host), filled before return.  Synchronises the stream.
 * Returns SPH_OK, or SPH_NOT_CONVERGED (x holds the best iterate; the report
 * says which components stalled). */
sph_status sph_visc_solve(sph_neighbors* handle, const sph_visc_params* params,
                          const sph_solve_opts* opts, const double* b, double* x,
                          sph_solve_report* report, void* stream);

/* Diagnostic for the breakdown safeguards: replays the scalar steps that
 * sph_visc_solve runs after each of its grid reductions (Sec. 4.2, restructured
 * listing and "Stopping criterion"), with the same device code on one warp, on
 * dot products given by the caller instead of computed from a matrix:
 *   after delta = r0^.A p:      alpha = gamma / delta; delta zero or not finite,
 *                               or alpha not finite: alpha = 0, the component
 *                               stalls this iteration;
 *   after r*.Ar* and Ar*.Ar*:   omega = (r*.Ar*) / (Ar*.Ar*), 0 unless the
 *                               denominator is positive and finite and the
 *                               quotient finite;
 *   after gamma' and r.r:       alpha' = gamma' / delta, beta = alpha' / omega
 *                               (both 0 after a stall, for omega = 0, or when
 *                               either is not finite); state converged if
 *                               r.r < tau^2, else stalled on a stall, omega = 0
 *                               or r.r not finite, else progressing.
 * Components that are not progressing are frozen (all scalars 0, state kept);
 * the pass is done when none progresses or the iteration count reaches maxit,
 * after which no further step runs (as in the solver's loop).
 * gamma0: (host) [3] r0.r0 of the pass, which is also the base of
 *   tau^2 = max(eps^2 gamma0, FLT_MIN);
 * dots: (host) [nsteps][15]: delta[3], r*.Ar*[3], Ar*.Ar*[3], gamma'[3], r.r[3];
 * out: (host) [nsteps + 1][20]: row 0 after the pass initialisation, row i
 *   after iteration i: alpha[3], omega[3], alpha'[3], beta[3], state[3],
 *   stalled_any[3], iterations, done (all as doubles).
 * 0 <= nsteps <= 100000, maxit >= 1.  Allocates a small device buffer;
 * synchronises the stream. */
sph_status sph_bicgstab_replay(const double* gamma0, double eps, int32_t maxit, int32_t nsteps, const double* dots,
                               double* out, void* stream);

/* One time step's viscous solve from HOST buffers (no counterpart in the paper;
 * the call a host-side time integrator makes): copies the scene (pos, rho, mu,
 * ptype: HOST pointers here, same layouts as sph_scene), b and either vel or x
 * to library-owned device staging, builds or rebuilds *handle's neighbour
 * lists (as sph_build_neighbors with max_neighbors), starts from
 * x0 = v^n with the dummy-wall closure (as sph_warm_start without a network)
 * when vel is non-NULL, else from x, solves as sph_visc_solve and copies the
 * solution back into x.
 * vel: (host) [n][4] float or NULL; b: (host) [n][3] double; x: (host) [n][3]
 * double, in: the initial guess when vel is NULL, out: the solution.  Pinned
 * (page-locked) host buffers make the copies asynchronous.
 * *handle: NULL on the first call (a handle is created and returned; release it
 * with sph_neighbors_destroy), or a handle from an earlier call.  The staging
 * is allocated on first use and grows with n; it is freed with the handle.
 * report: (host).  Synchronises the stream.  Returns as sph_visc_solve, or the
 * status of the neighbour build. */
sph_status sph_visc_solve_host(const sph_scene* scene, int32_t max_neighbors, const sph_visc_params* params,
                               const sph_solve_opts* opts, const float* vel, const double* b, double* x,
                               sph_neighbors** handle, sph_solve_report* report, void* stream);

/* ---- The semi-implicit time step (Sec. 3.3) ---------------------------------
 * The predictor/corrector step of Sec. 3.3 around the viscous solve, on a
 * particle state kept on the device:
 *   abar^n, drho^n; solve A^n(dt/2) V = B(dt/2) (B_fluid = u^n + dt/2 abar^n,
 *   walls 2 u_w dummy / u_w dynamic) for u^{n+1/2}; r^{n+1/2} = r^n + dt/2 u^n,
 *   rho^{n+1/2} = rho^n + dt/2 drho^n, mu^{n+1/2} (Papanastasiou); abar, drho
 *   there; solve A^{n+1/2}(dt) V = u^n + dt abar^{n+1/2} for u^{n+1};
 *   r^{n+1} = r^n + dt/2 (u^n + u^{n+1}), rho^{n+1} = rho^n + dt drho^{n+1/2}.
 * Pressure: Cole's equation of state (Eq. cole-pressure),
 *   P = c0^2 rho0 / zeta ((rho / rho0)^zeta - 1);
 * dummy walls (Eq. dummyP, walls at constant velocity): P_w = (sum_F P_a W_wa +
 *   g . sum_F rho_a (r_w - r_a) W_wa) / sum_F W_wa, rho_w = EOS^-1(P_w);
 * inviscid acceleration and continuity (Eqs. part_NS, part_continuity), with
 *   grad_b W_ab = |F_ab| (r_a - r_b):
 *   abar_b = g - sum_a m_a (P_a / rho_a^2 + P_b / rho_b^2) |F_ab| (r_a - r_b),
 *   drho_b/dt = sum_a m_a (u_b - u_a) . (r_a - r_b) |F_ab|
 *   (the printed signs, with the printed F <= 0, would make pressure attract;
 *   these are the signs under which it repels and compression raises rho).
 * Fluid rows get abar; fluid and dynamic-wall rows evolve their density; walls
 * move with their prescribed velocity.  Positions and densities are updated in
 * float64 and stored as float32 (periodic axes folded into [lo, hi)). */
typedef struct {
  int64_t n;               /* particles, >= 1                                        */
  float* pos;              /* (device) [n][4] x, y, z, m; in: r^n, out: r^{n+1}       */
  float* vel;              /* (device) [n][4]; fluid rows in: u^n, out: u^{n+1}; wall
                              rows: the prescribed wall velocity u_w (read only)      */
  float* rho;              /* (device) [n]; in/out (dummy walls: set by the closure)  */
  float* mu;               /* (device) [n]; in/out: recomputed from the velocities
                              after each neighbour build when rheology = 1            */
  const uint8_t* ptype;    /* (device) [n] SPH_FLUID / SPH_WALL                      */
  double lo[3], hi[3];     /* box, as sph_scene                                       */
  int32_t periodic[3];
  float h;
  int32_t kernel;          /* SPH_KERNEL_WENDLAND or SPH_KERNEL_GAUSSIAN              */
} sph_state;

typedef struct {
  double dt;               /* time step                                               */
  double rho0, c0, zeta;   /* equation of state: rest density, sound speed, exponent  */
  double g[3];             /* body force per unit mass                                */
  int32_t boundary;        /* SPH_BC_DUMMY or SPH_BC_DYNAMIC                          */
  int32_t mean;            /* SPH_MEAN_HARMONIC or SPH_MEAN_ARITHMETIC                */
  int32_t rheology;        /* 0: Newtonian (mu as given); 1: Papanastasiou (Eq. papa)  */
  double tau0, mu0, m;     /* Papanastasiou yield stress, plastic viscosity, exponent */
  int32_t max_neighbors;   /* capacity of the neighbour lists (0 = 128)               */
  int32_t picard;          /* rheology = 1 only: fixed-point passes that bring the
                              viscosity into the implicit system (the non-linear
                              form Sec. 8 names): after the corrector's solve, mu is
                              recomputed from r^{n+1/2} and the new velocities and
                              the system solved again, at most `picard` times; 0 =
                              the paper's lagged viscosity                           */
  double picard_tol;       /* stop when ||u_k - u_{k-1}|| / ||u_k|| <= picard_tol
                              (0 = 1e-6)                                              */
} sph_step_params;

typedef struct {
  sph_solve_report half;   /* the solve with A^n(dt/2)                                */
  sph_solve_report full;   /* the (last) solve with A^{n+1/2}(dt)                     */
  int32_t picard_passes;   /* fixed-point passes run                                  */
  double picard_change;    /* ||u_k - u_{k-1}|| / ||u_k|| of the last pass            */
} sph_step_report;

/* One step on `state` (device arrays, updated in place).  *handle: NULL on the
 * first call (created and returned; release with sph_neighbors_destroy) or the
 * handle of the previous step; the neighbour lists are rebuilt at r^n and at
 * r^{n+1/2}.  Both solves use opts (its method must suit the boundary model, as
 * for sph_visc_solve).  The step's buffers are owned by the handle.  report:
 * (host).  Synchronises.  Returns SPH_OK, SPH_NOT_CONVERGED when a solve stopped
 * above rtol (the state is still advanced), or the error of a failed call. */
sph_status sph_step(sph_state* state, const sph_step_params* params, const sph_solve_opts* opts,
                    sph_neighbors** handle, sph_step_report* report, void* stream);

/* ---- Batched ensemble solve -------------------------------------------------
 * S independent scenes (each its own handle and A(dt)) solved together: every
 * scene runs the restructured BiCGSTAB of Sec. 4.2 with its own scalars, states
 * and stopping decision, and the float64 refinement of sph_visc_solve.  One
 * refinement pass is one CUDA-graph replay of: the float64 residual of every
 * scene (scenes at rtol drop out on the device), pass set-up, ONE persistent
 * cooperative kernel running the iterations of all active scenes, and x += d.
 * Grid barriers inside the persistent kernel wait a bounded time and report
 * SPH_ERR_TIMEOUT instead of hanging.  A tile is a run of consecutive 32-row
 * slices of one scene taken by one block (16, 32 or 64 slices; the last tile
 * of a scene shorter).  The persistent kernel's row-loop form and block size
 * (256 or 128 threads) are autotuned on the first solve at 32-slice tiles, then
 * the tile length for that form. */
typedef struct sph_batch sph_batch;

/* handles: (host) [nscenes] built handles; params: (host) [nscenes] A(dt)
 * parameters (set up on each handle here; a handle rebuilt or given new
 * viscosities afterwards makes sph_batch_solve fail with SPH_ERR_INVALID).
 * The batch keeps pointers to the handles: destroy it before them. */
sph_status sph_batch_create(sph_neighbors* const* handles, const sph_visc_params* params,
                            int32_t nscenes, sph_batch** batch, void* stream);

/* b, x: (host) arrays of nscenes (device) pointers, each [n_s][3] double in that
 * scene's caller order (x: in guess, out solution); reports: (host) [nscenes].
 * opts as for sph_visc_solve (SPH_PREC_MIXED only; merged_reductions and chunk
 * are ignored: the batch always computes gamma' directly).  Synchronises.
 * Returns SPH_OK when every scene reached rtol. */
sph_status sph_batch_solve(sph_batch* batch, const sph_solve_opts* opts, const double* const* b,
                           double* const* x, sph_solve_report* reports, void* stream);

/* The autotuned persistent-kernel variant (0..7: row-loop form v & 3 as in
 * sph_profile_counters, block size 256 (v < 4) or 128 threads), whether the
 * solve runs as one graph launch whose conditional WHILE node repeats the pass
 * on the device (2), as a captured pass replayed per pass (1) or as direct
 * launches (0), the tuning
 * times (ms, [8]) and the chosen variant's grid size.  Any pointer may be NULL. */
sph_status sph_batch_info(const sph_batch* batch, int32_t* variant, int32_t* graph, float* tune_ms,
                          int32_t* grid);

/* The tile length in slices the batch uses (32 until the first solve has tuned
 * it), the number of tiles, the three candidate lengths (host [3]) and the
 * tuning time (ms, host [3]) of the chosen form at each (0 before tuning).  Any
 * pointer may be NULL. */
sph_status sph_batch_tiles(const sph_batch* batch, int32_t* tile_slices, int32_t* ntiles, int32_t* candidates,
                           float* tune_ms);

/* Fixes the tile length (one of the candidates sph_batch_tiles lists; anything
 * else is SPH_ERR_INVALID and changes nothing): later solves use it and the
 * tuner leaves it.  Synchronises the stream. */
sph_status sph_batch_set_tile(sph_batch* batch, int32_t tile_slices, void* stream);

sph_status sph_batch_destroy(sph_batch* batch);

/* ---- One system over several sub-domains (Sec. 7, Sec. 7.1) -----------------
 * The domain decomposition of the paper's multi-GPU solver: the cells of the
 * neighbour grid are grouped into layers along the longest axis of the box
 * (cell side >= 2h, so neighbours share a layer or sit in adjacent ones), and
 * each of `ranks` sub-domains owns a contiguous run of layers, balanced by
 * particle count.  A sub-domain keeps its own copy of the operator rows of its
 * particles (columns renumbered locally) and of every solver vector, plus a
 * halo: the particles of other sub-domains that its rows reference (the outer
 * edge of Sec. 7.1).  Per BiCGSTAB iteration the halo values of p and of r* are
 * exchanged before the two operator applies (the paper exchanges A p and A r*:
 * the same volume), and the dot products reduce as per-layer partials summed
 * in layer order, so the iterates are bit-identical for any number of
 * sub-domains.  All sub-domains run on the calling GPU (each in its own
 * allocations; the exchange is a device gather and the reduction a device
 * sum, standing for the send/recv and the all-gather of a multi-GPU run). */
typedef struct sph_shard sph_shard;

/* The partition on the host (no GPU needed): rows in layers, numbered layer by
 * layer in their given order with each layer padded to a multiple of 32 rows,
 * and the layers split into `ranks` contiguous runs of about n / ranks rows.
 * layer: (host) [n], each in 0..nlayers-1; virt: (host) [n] out, the new row
 * number of each row; rank_first_layer: (host) [ranks + 1] out; layer_first_virt:
 * (host) [nlayers + 1] out, the first row number of each layer (the last entry
 * is the padded total).  1 <= ranks <= min(64, nlayers). */
sph_status sph_shard_plan(int64_t n, const int32_t* layer, int32_t nlayers, int32_t ranks, int64_t* virt,
                          int32_t* rank_first_layer, int64_t* layer_first_virt);

/* Partition the system of `handle` with the coefficients for params (set up
 * here if needed) over `ranks` sub-domains (1..64, at most the layer count).
 * Copies the operator: the shard does not follow later rebuilds of the handle
 * (sph_shard_solve then fails with SPH_ERR_INVALID).  Synchronises. */
sph_status sph_shard_create(sph_neighbors* handle, const sph_visc_params* params, int32_t ranks,
                            sph_shard** shard, void* stream);

/* axis: the slab axis; layers: cell layers along it; owned, halo: (host)
 * [ranks] rows owned (with layer padding) and halo rows per sub-domain;
 * exchanged: halo rows filled per exchanged vector.  Any pointer may be NULL. */
sph_status sph_shard_info(const sph_shard* shard, int32_t* axis, int32_t* layers, int64_t* owned,
                          int64_t* halo, int64_t* exchanged);

/* As sph_visc_solve (b, x, report in caller order, device) with the mixed
 * precision BiCGSTAB, Jacobi scaling and direct reductions (other options:
 * SPH_ERR_INVALID); the float64 true residual is also recomputed over the
 * sub-domains (halo exchange of x's float32 hi/lo split).  Synchronises. */
sph_status sph_shard_solve(sph_shard* shard, const sph_solve_opts* opts, const double* b, double* x,
                           sph_solve_report* report, void* stream);

/* Striping (off by default; the overlap of transfers with computation that Sec. 7.2
 * and the conclusions name as the remedy for the exchange overhead): per apply,
 * the halo exchange runs on a stream of the shard's own while the interior slices
 * (32-row groups none of whose rows references a halo row) are applied on the
 * solve's stream; the edge slices follow when the exchange is done.  Each slice's
 * result and dots are those of the unstriped order, so the iterates are
 * bit-identical either way.  With every sub-domain on one GPU the exchange is a
 * small gather with nothing to hide, and the split launches and cross-stream
 * events make the solve slower; the overlap pays where the exchange is a
 * transfer between devices.  on: 0 or 1, else SPH_ERR_INVALID. */
sph_status sph_shard_set_striping(sph_shard* shard, int32_t on);

sph_status sph_shard_destroy(sph_shard* shard);

/* ---- Learned warm start ---------------------------------------------------
 * The paper names a better initial guess as future work (Sec. 8).  A
 * per-particle MLP, 16 -> 64 -> 64 -> 64 -> 3 with SiLU (9,603 parameters),
 * predicts delta = (x* - v^n) / U from 16 local features; the solve then starts
 * from x0 = v^n + U delta on fluid rows (walls start at b), and the unchanged
 * BiCGSTAB with its float64 true residual stays the arbiter of the result.
 * Inference and training run on BF16 tensor cores with FP32 accumulation.
 * Parameters are exchanged as 9,603 float32 values, row-major [out][in]:
 * W1 64x16, b1 64, W2 64x64, b2 64, W3 64x64, b3 64, W4 3x64, b4 3. */
typedef struct sph_mlp sph_mlp;

/* params: (host) [9603] float32, or NULL for zeros. */
sph_status sph_mlp_create(const float* params, sph_mlp** mlp);
sph_status sph_mlp_set_params(sph_mlp* mlp, const float* params);   /* (host); resets Adam */
sph_status sph_mlp_get_params(const sph_mlp* mlp, float* params);   /* (host) [9603] */
sph_status sph_mlp_destroy(sph_mlp* mlp);

/* Features (device, [n][16] bf16 bits, caller order) of the particles of
 * `handle` for velocities vel (device, [n][4] float): v/U, the Jacobi-scaled
 * explicit viscous increment D^-1 (v - A v) / U and its second application,
 * log10(mu)/5, log10(1 + dt sum c)/4 (on a wall row: of the mean over its fluid
 * neighbours), nearest wall neighbour / 2h (at most 1), the Shepard sum of W V
 * (W of the handle's kernel), neighbour count / 80, |v| relative to the
 * neighbourhood RMS, and the wall flag.  scale_out (host, may be NULL): U = RMS |v|
 * over the fluid. */
sph_status sph_mlp_features(sph_neighbors* handle, const sph_visc_params* params, const float* vel,
                            uint16_t* feats, double* scale_out, void* stream);

/* Training targets (x* - v) / U (device [n][4] float) and the fluid mask
 * (device [n] u8) from a solution x_star (device [n][3] double); uses the U of
 * the last sph_mlp_features call on the handle. */
sph_status sph_mlp_targets(sph_neighbors* handle, const float* vel, const double* x_star,
                           const uint8_t* ptype, float* targets, uint8_t* mask, void* stream);

/* out (device [m][4] float) = network(feats (device [m][16] bf16)). */
sph_status sph_mlp_forward(const sph_mlp* mlp, const uint16_t* feats, int64_t m, float* out, void* stream);

/* Mean squared error over the masked rows (mask may be NULL = all rows;
 * count = the number of masked rows) and its gradient: grad_out (device
 * [9603] float), loss_out (device [1] float); either may be NULL.  Forward and
 * backward run on the tcgen05 tensor cores (one CTA per SM holding all of its
 * tensor memory); the sums run in a fixed order, so equal inputs give equal
 * gradients.  A tensor-core wait that gives up is reported as SPH_ERR_TIMEOUT by
 * the next sph_mlp_get_params or sph_mlp_train_step with loss_host. */
sph_status sph_mlp_grad(sph_mlp* mlp, const uint16_t* feats, const float* targets, const uint8_t* mask,
                        int64_t m, int64_t count, float* grad_out, float* loss_out, void* stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss; loss_host (may be
 * NULL) receives the loss before the step (synchronises when given). */
sph_status sph_mlp_train_step(sph_mlp* mlp, const uint16_t* feats, const float* targets,
                              const uint8_t* mask, int64_t m, int64_t count, float lr, float* loss_host,
                              void* stream);

/* Network modes (bit flags, sph_mlp_set_mode).  SPH_MLP_HIGHPASS: the fluid
 * correction is y - S y instead of y, where (S y)_b is the Shepard average
 * sum_a W_ab V_a y_a / sum_a W_ab V_a over the fluid neighbours a of b and b
 * itself (V = m / rho): only the part of the correction that varies on the
 * particle scale enters x0, and its smooth part -- which the previous velocity
 * already carries and which the iteration removes slowest -- is left to v. */
#define SPH_MLP_HIGHPASS 1
sph_status sph_mlp_set_mode(sph_mlp* mlp, int32_t mode);

/* Loss options of sph_mlp_residual_targets (bit flags). */
#define SPH_RLOSS_JACOBI 1 /* weight the residual by D^-1 (default: unweighted)      */
#define SPH_RLOSS_LOG 2    /* per-problem log loss log(sum w^2|r|^2 / sum |b|^2)    */

/* Targets for training the warm start on the solver's own starting residual.
 * x0 = v + U net(features) on fluid rows with the dummy-wall closure of
 * sph_warm_start on wall rows; r = b - A x0; w = D^-1 with SPH_RLOSS_JACOBI,
 * else 1.  Loss (fluid rows): L = sum w^2 |r|^2 / (U^2 count), or with
 * SPH_RLOSS_LOG L = log(sum w^2 |r|^2 / sum |b|^2), whose scale does not depend
 * on how stiff or how far from converged a problem is.  dL/dy =
 * -(2 U / (U^2 count)) A^T (w^2 r) (resp. -(2 U / sum w^2|r|^2) A^T (w^2 r)),
 * holding the wall closure fixed.  The fluid block of A is symmetric when all
 * particles have one mass, so A^T z = A z there, and the targets
 * t = y + g A (w^2 r) with g = 1 / U (resp. count U / sum w^2 |r|^2)
 * (device [n][4] float; mask = fluid, device [n] u8) make the mean-squared-error
 * gradient of sph_mlp_grad / sph_mlp_train_step with count = the fluid count
 * equal to dL/dparameters.  feats (device [n][16] bf16) receives the features;
 * loss_host (may be NULL; synchronises) the loss L.  With SPH_MLP_HIGHPASS set
 * on the network, x0 uses y - S y and the targets carry (I - S)^T in front of
 * A (w^2 r), the transpose gathered over the same symmetric neighbour sets.
 * Unknown flags: SPH_ERR_INVALID. */
sph_status sph_mlp_residual_targets(sph_neighbors* handle, const sph_visc_params* params,
                                    const sph_mlp* mlp, const float* vel, const uint8_t* ptype,
                                    const double* b, int flags, uint16_t* feats, float* targets,
                                    uint8_t* mask, double* loss_host, void* stream);

/* x0 (device [n][3] double, caller order) = v + U network(features) on fluid
 * rows (v alone when mlp is NULL: the previous-step start of Sec. 4); on dummy
 * wall rows x0 = b - sum over fluid neighbours of (W / S) x0, which makes the
 * wall rows of b - A x0 vanish (Eq. dummyvel), and x0 = b on dynamic wall rows.
 * vel (device [n][4] float), ptype (device [n] u8), b (device [n][3] double)
 * in caller order. */
sph_status sph_warm_start(sph_neighbors* handle, const sph_visc_params* params, const sph_mlp* mlp,
                          const float* vel, const uint8_t* ptype, const double* b, double* x0,
                          void* stream);

/* Diagonal preconditioner scale: the alternative to the warm start.  The
 * mixed-precision solves precondition from the left by the Jacobi diagonal
 * (App. B); a row scale s > 0 per particle (the three velocity components share
 * the operator, so its diagonal block is one number) makes that S D^-1: the
 * inner BiCGSTAB or CG works on (S D^-1 A) d = S D^-1 r, with the same solution,
 * and the stop stays on the float64 true residual of A x = b.  scale: (device)
 * [n] float, caller order, copied; NULL clears it.  The scale stays with the
 * handle across operator rebuilds and neighbour rebuilds of the same particles
 * until cleared; a neighbour rebuild with another particle count clears it.
 * Values that are not positive
 * finite numbers: SPH_ERR_NONFINITE (synchronises to check).  The batched solve
 * takes each handle's scale as it stands at sph_batch_create (setting or clearing
 * one afterwards makes sph_batch_solve return SPH_ERR_INVALID); the float64 and
 * the sharded solves use the Jacobi diagonal alone and return SPH_ERR_INVALID
 * while a scale is set; sph_visc_apply is not affected. */
sph_status sph_set_row_scale(sph_neighbors* handle, const float* scale, void* stream);

/* norm2 (device [n] float, caller order) = squared Euclidean norm of each row of
 * D^-1 A(dt) for params: 1 + sum (a / D)^2 over a fluid row's coefficients, 1 +
 * sum S^2 over a dummy-wall row's Shepard weights, 1 for an identity row
 * (float32 sums of the stored float32 coefficients). */
sph_status sph_row_norms(sph_neighbors* handle, const sph_visc_params* params, float* norm2, void* stream);

/* The closed-form wall scale: scale (device [n] float, caller order) =
 * factor norm2^-power on dummy-wall (Shepard) rows and 1 on fluid and identity
 * rows, norm2 as in sph_row_norms; 1e-6 <= factor <= 1e6 and 0 <= power <= 64,
 * else SPH_ERR_INVALID.  The dummy-wall rows are interpolation constraints
 * (Eq. dummyvel); weighting them down against the Jacobi-scaled fluid rows
 * shortens the inner iteration on stiff systems. */
sph_status sph_wall_row_scale(sph_neighbors* handle, const sph_visc_params* params, double factor,
                              double power, float* scale, void* stream);

/* The learned scale: the network mlp (the warm start's 16-64-64-64-3 architecture,
 * trained for this use) on the features of sph_mlp_features for velocities vel
 * (device [n][4] float); scale (device [n] float, caller order) = exp(y_0),
 * y_0 clamped to [-8, 2], on wall rows and 1 on fluid rows, ready for
 * sph_set_row_scale.  scale may be NULL: the learned scale then becomes the
 * handle's row scale directly, as sph_set_row_scale would make it, without the
 * check and the synchronisation (its values are positive and finite by
 * construction).  Either kernel (the Shepard feature uses the handle's W). */
sph_status sph_mlp_row_scale(sph_neighbors* handle, const sph_visc_params* params, const sph_mlp* mlp,
                             const float* vel, float* scale, void* stream);

/* Training targets of the learned scale: targets (device [n][4] float, caller
 * order) = (log s, 0, 0, 0) with s the closed-form wall scale of
 * sph_wall_row_scale for factor and power, and mask (device [n] u8) = 1 on wall
 * rows. */
sph_status sph_mlp_scale_targets(sph_neighbors* handle, const sph_visc_params* params, double factor,
                                 double power, float* targets, uint8_t* mask, void* stream);

/* Papanastasiou viscosity from the previous velocities (Sec. 2.4, Eq. papa):
 *   grad u_b = sum_a V_a |F_ab| r_ab (x) u_ab;  gdot = sym(grad u);
 *   D = sqrt(2 gdot:gdot);  mu_b = tau0 Ybar(D) + mu0,
 * Ybar(D) = m T(m D) for m D < 0.5 (T: the paper's 8-term Horner series of
 * (1 - e^-x)/x) and (1 - e^{-m D})/D above.  Wall neighbours contribute their
 * wall velocity.  vel, wall_vel: (device) [n][4] float, caller order;
 * mu_out: (device) [n] float, caller order (fluid rows; wall rows get mu0).
 * Also stores the result as the handle's viscosity when set_handle != 0. */
sph_status sph_mu_papanastasiou(sph_neighbors* handle, const float* vel, const float* wall_vel,
                                double tau0, double mu0, double m, float* mu_out,
                                int32_t set_handle, void* stream);

/* Instrumentation (tracing): launch counts and the device time of the operator
 * apply inside solves, measured with CUDA events recorded on the solve's own
 * stream around the two apply launches of every eighth BiCGSTAB iteration (a
 * sample, so that the event records do not slow the loop they time).  Off by
 * default; enabling it adds two event records per sampled apply. */
typedef struct {
  int64_t launches;        /* kernels this library launched (all handles, all calls) */
  int64_t apply_launches;  /* operator applies timed on this handle (the sample)     */
  double apply_ms;         /* summed device time of those applies (ms)               */
  int64_t apply_bytes;     /* algorithmic bytes of one apply: 8 per stored
                              coefficient (index + value) plus, per row, 16 read of
                              v, 16 write of the result, 16 read of r0^ for the dot
                              and 9 of row data (count, kind, 1/D)                  */
  int64_t op_nnz;          /* stored coefficients of A(dt)                          */
  int64_t phase_launches[2]; /* apply_launches split: [0] A p (delta), [1] A r* (omega) */
  double phase_ms[2];        /* apply_ms split the same way                           */
  int32_t apply_variant[2];  /* row-loop form the autotuner chose per phase: 0..3 =
                                (8 entries, plain), (4, plain), (8, prefetch), (4, prefetch)
                                in registers; 4 = coefficient stream staged in shared
                                memory by bulk asynchronous copies; 5 = each 32-row
                                slice's distinct neighbour vectors gathered once into
                                shared memory                                        */
  float tune_us[3][6];       /* autotuner timings (us) per phase (A p, A r*, A r* with
                                merged dots) and form; 0 where not measured          */
  int64_t standalone_launches[2]; /* sph_visc_apply [0] and sph_visc_apply_otf [1] calls
                                     timed (their apply kernel only; profiling makes
                                     each such call synchronise)                      */
  double standalone_ms[2];        /* summed device time of those apply kernels (ms)    */
  int64_t otf_bytes;         /* algorithmic bytes of one on-the-fly apply: 4 per
                                neighbour-list entry plus, per row, 16 read of v, 16
                                write, 16 of packed geometry, 4 of 1/mu, 4 of R_b, 4
                                of the count and 1 of the kind                        */
  int32_t apply_grid[2];     /* blocks of 256 threads the chosen forms run with, per
                                phase as apply_variant: the full resident grid, or
                                for a register form the smallest grid with the same
                                number of rounds of slices per warp when the tuner
                                measured that faster                                */
} sph_profile_counters;

sph_status sph_profile_enable(sph_neighbors* handle, int32_t on);
/* Reads the counters (synchronises the handle's last stream); reset != 0
 * clears the per-handle timing after reading. */
sph_status sph_profile_read(sph_neighbors* handle, sph_profile_counters* out, int32_t reset);

/* Thread-local description of the last error (empty string if none). */
const char* sph_last_error(void);

/* Library version string. */
const char* sph_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPHVISC_H */
