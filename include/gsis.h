/*
 * gsis.h -- C ABI of the GB300 GSIS steady rarefied-flow solver.
 *
 * Method: general synthetic iterative scheme (GSIS-II) of arXiv 2310.18916,
 * "Efficient parallel solver for rarefied gas flow using GSIS":
 *   - kinetic step over phase space (Section 3.2, Eq. delta_equations and the
 *     point-implicit form that follows it; Algorithm 3 body),
 *   - velocity moments (Eq. getmoment), high-order terms (Eq. full_constitutive),
 *   - FP64 synthetic NSF solve (Section 3.3, Eq. macro, delta_Macroscopic_equations,
 *     res_macro; Algorithm 2 body),
 *   - VDF correction (Eq. updatef) and residual (Eq. convergence_critertion),
 *   - driven by the outer loop of Algorithm 1.
 *
 * Units (nondimensional): lengths in L, velocities in v0 = sqrt(2 R T0), density in rho0,
 * temperature in T0 (so R T -> T/2 and the Maxwellian is rho (pi T)^(-3/2) exp(-|xi-u|^2/T)).
 *
 * Conventions for every entry point:
 *   - return value: GSIS_OK (0) or a negative GSIS_E_* code; no exception crosses the ABI;
 *     gsis_last_error() gives a one-line message for the last failure on a handle;
 *   - pointers named host_* or documented as host point to host memory, owned by the caller
 *     and only read/written during the call;
 *   - all device memory is owned by the handle (allocated at gsis_create through the
 *     caller's allocator callback, or cudaMalloc when none is given) and released by
 *     gsis_destroy;
 *   - one handle is used by one host thread at a time; distinct handles are independent;
 *   - work is issued on the stream given in gsis_options (default stream when NULL);
 *     calls that return host data synchronise that stream.
 */
#ifndef GSIS_H
#define GSIS_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

#define GSIS_OK 0
#define GSIS_E_INVALID (-1)       /* bad argument, mesh or grid */
#define GSIS_E_OOM (-2)           /* allocation failed */
#define GSIS_E_CUDA (-3)          /* CUDA error (message in gsis_last_error) */
#define GSIS_E_DIVERGED (-4)      /* non-finite or non-positive density / temperature */
#define GSIS_E_TIMEOUT (-5)       /* a bounded device-side wait gave up */
#define GSIS_E_NOT_CONVERGED (-6) /* max_outer reached above tol; results are valid */
#define GSIS_E_UNSUPPORTED (-7)   /* valid input outside what the library implements */

enum gsis_bc_type { GSIS_BC_WALL = 1, GSIS_BC_PERIODIC = 2, GSIS_BC_FARFIELD = 3, GSIS_BC_AXIS = 4 };
enum gsis_model { GSIS_SHAKHOV = 0, GSIS_RYKOV = 1 };
enum gsis_precision { GSIS_F64 = 0, GSIS_F32 = 1, GSIS_BF16 = 2 };
enum gsis_mode { GSIS_MODE_GSIS = 0, GSIS_MODE_DVM = 1 };
/* Wall flux of the synthetic solve (Section 3.3).  Both enter as increments on the wall flux the
   kinetic step produced (their values at W^{n+1/2} cancel), so the converged state is the
   kinetic one either way; they differ in how the wall responds to the inner steps. */
enum gsis_wall_flux {
  GSIS_WALL_EQ = 0,   /* the half-range flux of the wall cell's local Maxwellian */
  GSIS_WALL_G13 = 1   /* that of its Grad-13 VDF (Eq. G13_VDF): the cell's rho, u, T of the inner
                         step with the stress and heat fluxes of the kinetic step (Eq.
                         GSIS-DVM-flux) */
};

/* Structured hexahedral block (spatial finite-volume cells of Section 3.2).
 * nodes: (ni+1)(nj+1)(nk+1) x 3 doubles (host), node (I,J,K) at index I + (ni+1)(J + (nj+1)K).
 * bc[side], side = i-, i+, j-, j+, k-, k+ (x-, x+, ... on a rectilinear block):
 *   WALL      isothermal, fully diffuse wall with velocity wall_u[side] (tangential) and
 *             temperature wall_T[side];
 *   PERIODIC  on both sides of an axis.  An axis with one cell must be PERIODIC (it then carries
 *             no transport); with at least 3 cells the axis closes on itself, the two ends being
 *             neighbours (the azimuth of an O-grid: the mesh geometry already joins them), and
 *             GSIS mode and Euler presteps need an even cell count on it;
 *   FARFIELD  free stream of density 1, velocity wall_u[side] and temperature wall_T[side]:
 *             molecules entering through a face carry its Maxwellian where the free stream does
 *             not leave through the face, else the cell's own face value;
 *   AXIS      a degenerate side of zero area (the pole of a spherical grid): no flux.
 * Axes with one cell come after the others.  A rectilinear block (node x depends on I only,
 * y on J, z on K, increasing) with WALL sides and one-cell periodic axes takes the rectilinear
 * kernels; any other block (curvilinear, far field, pole or wrapped sides) takes the general
 * ones, with n_sweeps colour passes per kinetic step, in both modes and velocity-sharded alike.
 * Cells must have positive volume, else GSIS_E_INVALID. */
typedef struct {
  int ni, nj, nk;
  const double *nodes;
  int bc[6];
  double wall_u[6][3];
  double wall_T[6];
  /* Unstructured mesh (ncells > 0; the hexahedral, prismatic, pyramidal and tetrahedral cells
   * of the paper's spatial meshes, Section 5): ni, nj, nk and nodes are then not read.
   *   unodes:     [nnodes][3] node coordinates (host).
   *   cells:      [ncells][8] node ids of each cell as a hexahedron with corner t at the
   *               offsets (t & 1, (t >> 1) & 1, t >> 2) of the block convention above; other
   *               shapes repeat ids (prism a b c c d e f f, pyramid a b c d e e e e, tetrahedron
   *               a b c c d d d d), and a side whose corners span no area carries no flux.
   *   face_patch: [ncells][6] per side (0: corners 0 2 6 4, 1: 1 3 7 5, 2: 0 1 5 4, 3: 2 3 7 6,
   *               4: 0 1 3 2, 5: 4 5 7 6): -1 where the side is shared with another cell (the
   *               two cells list the same node ids on it), else the boundary patch 0..5 whose
   *               bc, wall_u and wall_T above apply.  A PERIODIC patch marks the two faces of a
   *               mesh one cell layer thick in z (faces normal to z): no transport across them
   *               and no z gradient, the unstructured form of a one-cell periodic axis; AXIS
   *               faces carry no flux.
   * The kinetic step sweeps each velocity octant (signs d) in its own upwind order: cells ranked
   * by the mean over their distinct nodes of ((d_x x) + (d_y y)) + (d_z z), ties by index, each
   * cell's colour one more than the largest colour of its face neighbours ranked before it;
   * n_sweeps passes, colour by colour.  The synthetic solve's LU-SGS runs over a greedy
   * colouring of the face graph (cells in index order, each taking the smallest colour none of
   * its neighbours holds).  Least-squares
   * gradients: over the face neighbours on a mesh of hexahedra, over every node-sharing cell on
   * a mesh with prisms, pyramids or tetrahedra; the synthetic solve takes its gradients over
   * the same stencils.  Both modes and the Euler presteps run on every shape.  Faces must be
   * planar to round-off, cells of positive volume; an unmatched side with patch -1, a patch out of
   * range or a shared side with a patch gives GSIS_E_INVALID. */
  int ncells;
  int nnodes;
  const double *unodes;
  const int *cells;
  const int *face_patch;
} gsis_mesh;

/* Discrete velocity set (Section 3.1, velocity-space discretisation), host arrays, copied.
 * Tensor product (npoints = 0): n[d] nodes x[d][.] with quadrature weights w[d][.] per axis d;
 *   the discrete velocity index used by gsis_get_f / gsis_set_f is v = ix + n0 (iy + n1 iz).
 * Unstructured (npoints > 0; the locally refined velocity meshes of the paper's unstructured
 *   velocity-space discretisation): points[v][4] = xi_x, xi_y, xi_z and the quadrature weight
 *   (the volume of the velocity cell of discrete velocity v), v = 0 .. npoints-1 the index of
 *   gsis_get_f / gsis_set_f; n, x and w are not read.  Weights must be positive and finite,
 *   else GSIS_E_INVALID. */
typedef struct {
  int n[3];
  const double *x[3];
  const double *w[3];
  int npoints;
  const double *points;
} gsis_vgrid;

/* Gas model (Section 2): Shakhov (monatomic, Pr = 2/3; the g_0t reference distribution) or
 * the Rykov-type model with d_r internal degrees of freedom, internal collision number Z_r
 * and heat-flux relaxation rates A = (Att, Atr, Art, Arr).  omega: viscosity index. */
typedef struct {
  int model;
  double omega;
  double d_r, Z_r;
  double A[4];
} gsis_gas;

/* Device allocator callback: alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, stream, ctx) releases it.  Both may be NULL (cudaMalloc / cudaFree are used). */
typedef void *(*gsis_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*gsis_free_fn)(void *ptr, void *stream, void *ctx);

/* Sum-all-reduce across the shards of a velocity-sharded solve (see shard_count): replace the
 * count FP64 values at device pointer dev by their sum over all shards, in the order of work on
 * stream (e.g. an NCCL all-reduce on that stream, or a host-synchronising exchange).  Every
 * shard calls it with the same count at the same points of a step; returns 0 on success. */
typedef int (*gsis_allreduce_fn)(double *dev, size_t count, void *stream, void *ctx);

/* Solver options.  Defaults (gsis_default_options): see the comments. */
typedef struct {
  int precision;        /* VDF storage / kinetic arithmetic (default F32): GSIS_F64 (FP64 / FP64),
                           GSIS_F32 (FP32 / FP32), GSIS_BF16 (BF16, rounded to nearest even on
                           store / FP32).  FP32 and BF16 accumulate moments in FP32 with
                           compensated sums.  The synthetic solve, the correction state and the
                           residual are FP64 always. */
  int mode;             /* GSIS_MODE_GSIS (default) or GSIS_MODE_DVM (plain kinetic iteration) */
  int n_sweeps;         /* colour-ordered point-implicit passes per kinetic step (default 1; a
                           rectilinear block is solved exactly by 1 and takes only 1; general
                           blocks take 1..64) */
  int macro_steps;      /* inner synthetic steps per outer step (default 300, Algorithm 1) */
  int macro_sweeps;     /* red-black LU-SGS passes per inner step (default 4, Algorithm 2) */
  double macro_cfl;     /* pseudo-time CFL of the synthetic solve (default 100) */
  double macro_tol;     /* inner early exit on the relative increment (default 1e-10) */
  double kin_inv_dt;    /* 1/dt of the kinetic delta form (default 0: steady).  A pseudo-time step
                           (> 0) damps the kinetic iteration after an impulsive start; only
                           GSIS_MODE_DVM takes it (the synthetic solve needs a steady step). */
  double venkat_K;      /* Venkatakrishnan constant, eps^2 = (K V^(1/3))^3 (default 1) */
  int kinetic_presteps; /* plain kinetic steps before the GSIS loop (default 10, Algorithm 1) */
  const double *init_W; /* optional host array, per cell rho, ux, uy, uz, Tt, Tr; f0 = Maxwellian.
                           NULL: rho = 1, u = 0, Tt = Tr = 1. */
  void *stream;         /* cudaStream_t, NULL = default stream */
  gsis_alloc_fn alloc;
  gsis_free_fn free;
  void *alloc_ctx;
  int macro_sms;        /* SMs the synthetic solve may occupy (default 0: all).  Its blocks hold a
                           whole SM each, so solves that run at the same time on one GPU (serving)
                           each take a share. */
  int shard_count;      /* velocity sharding (the N_v decomposition of Section 4): the discrete
                           velocities, in blocks of 32 of one octant, are split into shard_count
                           contiguous ranges; this handle owns range shard_index and stores f only
                           there (default 1: unsharded).  Per step three partial sums are
                           all-reduced through allreduce: the wall re-emission densities before
                           the kinetic sweeps, the per-cell moments and kinetic flux sums, and the
                           wall fluxes.  Everything after them (the synthetic solve included) is
                           repeated identically on every shard.  gsis_get_f / gsis_set_f then
                           transfer only this shard's velocities (others untouched / ignored). */
  int shard_index;
  gsis_allreduce_fn allreduce;  /* required when shard_count > 1 */
  void *allreduce_ctx;
  int kinetic_ring;     /* where the kinetic sweep keeps the three colours it works on and the
                           face values along walls, per block of 32 velocities (Section 4's
                           colour-ordered sweep).  0 (default): in shared memory, unless the
                           largest colour does not fit there (3D meshes from about 18^3 cells in
                           FP32 and BF16, 12^3 in FP64) or the other placement keeps at least
                           twice as many blocks resident per SM; else in a device scratch of the
                           solver's own, counted by gsis_footprint_bytes.  1: always in the
                           device scratch.  Results are bit-identical either way. */
  int euler_presteps;   /* inner steps of the inviscid synthetic solve (Euler fluxes, slip walls,
                           far field against the free stream) run once at creation, before the
                           kinetic presteps; f then starts as the Maxwellian of their result
                           (the Euler preconditioning of Algorithm 1 for strong shocks).  Default
                           0; general blocks only (GSIS_E_UNSUPPORTED on rectilinear ones). */
  int wall_flux;        /* GSIS_WALL_EQ (default) or GSIS_WALL_G13 */
  int positive_faces;   /* general blocks (body-fitted and unstructured meshes): 1 makes the kinetic
                           step's reconstructed face values keep the sign of the cell value.  Where
                           the limited linear value f_i + d (Section 3.2) falls below f_i, the face
                           takes f_i^2 / (f_i - d), which agrees with it to first order in d / f_i.
                           The linear form lets a VDF's steep fall into a near-vacuum wake
                           reconstruct negative face values, which empties cells behind a body in
                           supersonic flow.  Default 0 (the linear form); GSIS_E_UNSUPPORTED on
                           rectilinear blocks. */
  double relax;         /* general blocks, GSIS mode: the outer step's update of the state is
                           W^{n+1/2} + relax (W^{n+1} - W^{n+1/2}) (in rho, u, T_t, T_r) instead of
                           the synthetic solve's W^{n+1}.  0 or 1 (default 0): the full update of
                           Algorithm 1; values in (0, 1) damp it.  The converged state is the same
                           wherever the discrete reference distribution conserves mass, momentum
                           and energy on the velocity grid; otherwise the two differ by that
                           quadrature error.
                           On O-grids whose cells next to the poles are thin wedges, the full
                           update lets a slowly growing mode in (sphere of 16 x 24 x 48 cells, Kn
                           0.05: eps falls to 7e-5, then grows); 0.5 converges it.
                           GSIS_E_INVALID outside [0, 1]; GSIS_E_UNSUPPORTED below 1 on rectilinear
                           blocks. */
  double visc_jump;     /* general blocks: the weight alpha of the jump term in the synthetic
                           solve's viscous face gradients (Eq. NSF_constitutive at a face between
                           cells i and j, d = x_j - x_i the line between their centres):
                             grad_f = g + alpha (phi_j - phi_i - g.d) d / |d|^2,
                           g the mean of the two cells' least-squares gradients, for u, T_t and
                           T_r.  The mean alone is not dissipative on meshes with prisms, pyramids
                           or tetrahedra (their node-sharing stencils): the synthetic solve's inner
                           iteration diverges there at Kn 0.2 on a 16 x 16 cavity, at every CFL.
                           The full correction (alpha = 1) makes the outer coupling with the
                           kinetic step stall or diverge; 1/4 converges both.  The fixed point does
                           not depend on alpha.  Negative (default -1): 1/4 on meshes with
                           prisms, pyramids or tetrahedra, 0 on others; a value in [0, 1] applies
                           on every general block.  GSIS_E_INVALID above 1 or NaN;
                           GSIS_E_UNSUPPORTED above 0 on rectilinear blocks. */
  int capture_graphs;   /* 1: each outer step runs as a CUDA graph, captured from the solver's
                           stream on the first step of each mode and state buffer (two alternate)
                           and replayed afterwards: one launch per step on the host instead of one
                           per kernel (about 4,500 per GSIS step on a general mesh).  Results are
                           identical to direct launches.  Steps launch directly while profiling
                           (gsis_profile) or with velocity shards, and for good if a capture fails;
                           gsis_set_f drops the graphs.  Default 0; GSIS_E_INVALID unless 0 or 1. */
} gsis_options;

typedef struct gsis_solver *gsis_handle;

/* Fill *opt with the defaults listed above. */
void gsis_default_options(gsis_options *opt);

/* Device bytes a solver of this size would hold (admission by memory footprint).
 * Returns GSIS_OK and writes *bytes, or GSIS_E_INVALID / GSIS_E_UNSUPPORTED. */
int gsis_footprint_bytes(const gsis_mesh *mesh, const gsis_vgrid *vgrid, const gsis_gas *gas,
                         const gsis_options *opt, size_t *bytes);

/* Build a solver: copy the inputs, build geometry and velocity blocks, allocate device state,
 * set f0 = Maxwellian(init_W) and run opt->kinetic_presteps plain kinetic steps
 * (the preconditioning of Algorithm 1).  Kn: Knudsen number, mu(T0)/(p0 L) sqrt(pi R T0/2) (Section 2.1).
 * Ma: Mach number of the problem (Section 5 states each case by its free-stream Mach number):
 * the free stream's speed |wall_u| over its speed of sound for a mesh with FARFIELD sides, else
 * the fastest WALL's speed over the speed of sound at that wall's temperature, with
 * c^2 = gamma T / 2 (speeds in sqrt(2 R T0)) and gamma = (5 + d_r)/(3 + d_r) (5/3 for Shakhov).
 * The speeds themselves come from the mesh; a Ma that disagrees with them by more than
 * 1e-9 max(1, Ma) is refused with GSIS_E_INVALID before anything is allocated.  With
 * opt->euler_presteps > 0 the inviscid presteps run first and f starts from their result.
 * On success *out is a new handle; on failure *out is NULL. */
int gsis_create(const gsis_mesh *mesh, const gsis_vgrid *vgrid, const gsis_gas *gas, double Kn,
                double Ma, const gsis_options *opt, gsis_handle *out);

/* Run outer iterations of Algorithm 1 until eps < tol or max_outer iterations.
 * *outer_done: iterations run by this call; *eps_last: eps of the last one.
 * Returns GSIS_OK (converged), GSIS_E_NOT_CONVERGED (max_outer reached), or an error. */
int gsis_iterate(gsis_handle h, int max_outer, double tol, int *outer_done, double *eps_last);

/* Copy per-cell macroscopic fields to host_out (FP64, layout [cell][field], cell index
 * i + ni (j + nj k)).  field_mask selects, in this order:
 *   GSIS_F_W    : rho, ux, uy, uz, Tt, Tr of the state used by the next kinetic step (6)
 *   GSIS_F_HALF : moments of f^{n+1/2} of the last step: rho, u(3), Tt, Tr,
 *                 sigma(xx,yy,zz,xy,xz,yz), qt(3), qr(3) (18)
 *   GSIS_F_HOT  : HoT of the last GSIS step: sigma(6), qt(3), qr(3) (12)
 * out_len: number of doubles available at host_out. */
#define GSIS_F_W 1u
#define GSIS_F_HALF 2u
#define GSIS_F_HOT 4u
int gsis_moments(gsis_handle h, unsigned field_mask, double *host_out, size_t out_len);

/* eps of Eq. convergence_critertion for the last outer step: eps_by_field[0..2] = rho, u, Tt,
 * eps_by_field[3] = their maximum (n >= 4). */
int gsis_residual(gsis_handle h, double *eps_by_field, int n);

/* One outer step enqueued on the handle's stream without waiting for it (GSIS or DVM as
 * opt.mode), so steps of several handles on different streams overlap on the device.  At most
 * one step may be pending: gsis_step_wait must follow before the next gsis_step_async or any
 * other call on the handle (GSIS_E_INVALID otherwise). */
int gsis_step_async(gsis_handle h);

/* Waits for the pending step of gsis_step_async and returns its status (the same codes as
 * gsis_iterate for one step); *eps_last (may be NULL) receives its eps (maximum over fields).
 * GSIS_E_INVALID when no step is pending. */
int gsis_step_wait(gsis_handle h, double *eps_last);

/* Per wall face (host arrays of length gsis_nwall): cell index, side, re-emitted density
 * rho_w of the last kinetic step and the kinetic wall flux (outward, area-integrated: mass,
 * momentum(3), energy, internal energy). Any pointer may be NULL. */
int gsis_nwall(gsis_handle h);
int gsis_wall(gsis_handle h, int *cell, int *side, double *rho_w, double *flux6);

/* Wall loads (drag and heat-flux coefficients, a10) from the kinetic wall fluxes of the last
 * kinetic step, summed over the wall faces of the sides selected by side_mask (bit s = side s:
 * 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z).  Writes 6 host doubles to out6:
 *   out6[0..2] force on the walls = sum of the outward (gas -> wall) momentum fluxes,
 *   out6[3]    energy flux into the walls,
 *   out6[4]    C_D = (force . dir) / (1/2 rho_ref U_ref^2 A_ref),
 *   out6[5]    C_H = energy flux / (1/2 rho_ref U_ref^3 A_ref),
 * in the solver's units (lengths of the mesh, velocities in sqrt(2RT0), density rho0).
 * dir: 3 host doubles, the reference direction (not normalised by the call).  rho_ref, U_ref,
 * A_ref > 0, else GSIS_E_INVALID.  Synchronises the solver's stream. */
int gsis_wall_loads(gsis_handle h, unsigned side_mask, const double *dir, double rho_ref, double U_ref, double A_ref,
                    double *out6);

/* Per cell the sum over its faces of the outward kinetic face flux of the last kinetic step
 * (mass, momentum(3), energy, internal energy; area-integrated): the kinetic information the
 * synthetic solve uses (Eq. full_constitutive evaluated with the kinetic scheme's own fluxes).
 * host_out holds ncells x 6 doubles.  Rectilinear blocks obtain it from the collision moments
 * (exact there: one colour pass solves the implicit system); general blocks sum the face fluxes
 * in GSIS mode, and in DVM mode report the collision-moment form, which a finite number of
 * colour passes satisfies only approximately. */
int gsis_kinetic_flux_sum(gsis_handle h, double *host_out, size_t out_len);

/* VDF transfer, FP64 host arrays [cell][v] (f1 for the Rykov model only, else NULL).
 * gsis_set_f also resets the per-cell state to the moments of the new f (checkpoint load). */
int gsis_get_f(gsis_handle h, double *host_f0, double *host_f1);
int gsis_set_f(gsis_handle h, const double *host_f0, const double *host_f1);

/* Device-time profile of gsis_iterate, from CUDA events recorded on the solver's stream around
 * each phase of an outer step while enabled.  enable: 1 record from now on, 0 stop.  reset: clear
 * the accumulators first.  ms[0..4] (n >= 5, may be NULL): accumulated milliseconds of
 * [0] wall pre-pass, [1] kinetic step, [2] block reduction and moments, [3] synthetic solve,
 * [4] residual and next state.  *steps: outer steps recorded; *launches: kernels launched by
 * those steps (either may be NULL). */
int gsis_profile(gsis_handle h, int enable, int reset, double *ms, int n, int *steps, int *launches);

/* Counters: outer iterations run so far, inner synthetic steps of the last outer step. */
int gsis_stats(gsis_handle h, int *outer_total, int *macro_iters_last);

/* Step graphs (gsis_options.capture_graphs): the number of captured outer-step graphs the solver
 * holds (0 before the first captured step or without the option), or -1 once a capture has
 * failed and the solver launches its steps directly.  No GPU work; 0 for a NULL handle. */
int gsis_graphs(gsis_handle h);

/* Allocation-free velocity moments of a VDF held by the caller (no counterpart in the paper).
 * For callers that cannot allocate device memory where they need moments: code running inside
 * another framework's memory pool without an allocator handle to pass down, or a
 * latency-critical region where an allocation (and the synchronisation it can imply) is not
 * allowed.  It allocates nothing: its only scratch is a fixed 8 MiB array of static device
 * memory (every GPU that loads this library holds it until the process exits).
 *   f_dev:   device, FP32, [cell][v], v = ix + nx (iy + ny iz) (the layout of gsis_get_f)
 *   vel_dev: device, FP32, 16-byte aligned, [v][4] = xi_x, xi_y, xi_z, quadrature weight
 *   out_dev: device, FP64, [cell][18] = the GSIS_F_HALF fields of gsis_moments: rho, u(3),
 *            Tt, Tr (= Tt), sigma(xx,yy,zz,xy,xz,yz), qt(3), qr(3) (= 0)
 *   stream:  cudaStream_t (NULL = default stream); the call only enqueues work on it.
 * Accuracy: two passes, both summed in FP32 with compensated (Kahan) accumulators and the
 * per-chunk partials combined in FP64 in a fixed order: the mean velocity first, then the
 * moments about it, so fast streams (|u| several times the thermal speed) keep the relative
 * accuracy of slow ones.  out_dev doubles as the store of the mean velocity between passes.
 * Limits: ncells <= 8 MiB / (12 x 8 B) = 87381, else GSIS_E_INVALID (nothing is launched;
 * gsis_last_error(NULL) says why).
 * The first call on a device, with that device current, looks up the scratch's device address
 * (cudaGetSymbolAddress); make that first call before capturing a stream into a graph.
 * Calls share the scratch: two calls whose work overlaps on the GPU (different streams,
 * concurrent host threads) race and must be ordered by the caller.  Each call overwrites all
 * scratch it reads, so no state carries from one call to the next.
 * Returns GSIS_OK, GSIS_E_INVALID or GSIS_E_CUDA. */
int gsis_vdf_moments_noalloc(const float *f_dev, const float *vel_dev, int ncells, int nvel, double *out_dev,
                             void *stream);

/* Release everything held by h.  NULL-safe. */
int gsis_destroy(gsis_handle h);

/* Message of the last error on h (or, when h is NULL, of the last failed gsis_create or
 * gsis_vdf_moments_noalloc on this host thread). */
const char *gsis_last_error(gsis_handle h);

/* Self-test of the bounded device waits, on the current device: which = 0 runs the synthetic
 * solve's grid barrier with one of its two blocks leaving without arriving; which = 1 waits on an
 * mbarrier phase that nothing completes (the kinetic kernel's staging wait).  Each wait gives up
 * after ~2^24 clock cycles (a few ms) and raises the device error flag, which is returned in
 * *device_status (GSIS_E_TIMEOUT when the wait ran out as designed, GSIS_OK if it did not).  The
 * context stays usable.  Uses its own cudaMalloc'd scratch (freed before returning).
 * Returns GSIS_OK, GSIS_E_INVALID (bad which / NULL) or GSIS_E_CUDA. */
int gsis_selftest_wait_timeout(int which, int *device_status);

#ifdef __cplusplus
}
#endif
#endif
