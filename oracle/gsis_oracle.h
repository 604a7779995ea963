/*
 * gsis_oracle.h -- plain, slow, FP64 CPU oracle of the GSIS steady solver
 * (arXiv 2310.18916, "Efficient parallel solver for rarefied gas flow using GSIS").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this file.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code with the CUDA library.
 *
 * Units (nondimensional): lengths in L, velocities in v0 = sqrt(2 R T0), density in
 * rho0, temperature in T0.  Hence R T -> T/2, p = rho T / 2 and the Maxwellian is
 * rho (pi T)^(-3/2) exp(-|xi-u|^2/T).
 */
#ifndef GSIS_ORACLE_H
#define GSIS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* Side conditions.  WALL: diffuse isothermal wall (wall_u, wall_T).  PERIODIC: both sides of
   an axis; with several cells the axis wraps onto itself (a closed mesh such as the azimuth of
   an O-grid, whose geometry already joins the two ends).  FARFIELD: free stream rho = 1,
   u = wall_u, T_t = T_r = wall_T.  AXIS: a degenerate side of zero area (the pole of a
   spherical grid): no flux, no neighbour. */
enum { ORC_BC_WALL = 1, ORC_BC_PERIODIC = 2, ORC_BC_FARFIELD = 3, ORC_BC_AXIS = 4 };
enum { ORC_SHAKHOV = 0, ORC_RYKOV = 1 };
enum { ORC_GSIS = 0, ORC_DVM = 1 };
enum { ORC_SCHED_COLOUR = 0, ORC_SCHED_LEXSGS = 1 };
enum { ORC_OK = 0, ORC_E_INVALID = -1, ORC_E_OOM = -2, ORC_E_DIVERGED = -4 };

typedef struct {
  int ni, nj, nk;
  const double *nodes;  /* (ni+1)(nj+1)(nk+1) x 3, node (I,J,K) at I + (ni+1)(J + (nj+1)K) */
  int bc[6];            /* sides x-, x+, y-, y+, z-, z+ (index space: i-, i+, j-, j+, k-, k+) */
  double wall_u[6][3];
  double wall_T[6];
  /* unstructured mesh (ncells > 0; ni, nj, nk, nodes unused): cells as hexahedra of node ids,
     corner t at offsets (t & 1, (t >> 1) & 1, t >> 2), other shapes repeating ids; per side
     (corners 0 2 6 4 | 1 3 7 5 | 0 1 5 4 | 2 3 7 6 | 0 1 3 2 | 4 5 7 6) -1 when shared with
     another cell, else the boundary patch 0..5 indexing bc, wall_u, wall_T */
  int ncells, nnodes;
  const double *unodes; /* [nnodes][3] */
  const int *cells;     /* [ncells][8] */
  const int *face_patch;/* [ncells][6] */
} orc_mesh;

typedef struct {
  int n[3];
  const double *x[3];   /* nodes per axis */
  const double *w[3];   /* quadrature weights per axis */
  int npoints;          /* > 0: an unstructured set of npoints velocities (n, x, w unused) */
  const double *points; /* [npoints][4]: xi_x, xi_y, xi_z, weight (the velocity cell's volume) */
} orc_vgrid;

typedef struct {
  int model;            /* ORC_SHAKHOV (monatomic) or ORC_RYKOV */
  double omega;         /* viscosity index */
  double Kn;
  double d_r, Z_r;      /* Rykov only */
  double A[4];          /* Att, Atr, Art, Arr (Rykov only) */
} orc_gas;

typedef struct {
  int mode;             /* ORC_GSIS or ORC_DVM */
  int schedule;         /* ORC_SCHED_COLOUR or ORC_SCHED_LEXSGS */
  int n_sweeps;
  int macro_steps, macro_sweeps;
  double macro_cfl, macro_tol;
  double kin_inv_dt, venkat_K;
  int nthreads;         /* OpenMP threads over velocity (results do not depend on it) */
  int wall_flux;        /* wall flux of the synthetic solve, both as increments on the frozen
                           kinetic wall flux: ORC_WALL_EQ (0) the half-range flux of the local
                           Maxwellian, ORC_WALL_G13 (1) that of the Grad-13 reconstruction of
                           Eq. G13_VDF (Section 3.3) */
  int positive_faces;   /* 1: the kinetic face values keep the sign of the cell value (see
                           orc_cell_faces); 0: the linear reconstruction of Section 3.2 */
  double relax;         /* GSIS update W^{n+1/2} + relax (W^{n+1} - W^{n+1/2}); 0 or 1: the full
                           update of Algorithm 1 */
  double visc_jump;     /* weight alpha of the jump along the centre line in the viscous face
                           gradients (see face_nsf); negative: 1/4 on meshes with prisms,
                           pyramids or tetrahedra, 0 on others */
} orc_opts;

enum { ORC_WALL_EQ = 0, ORC_WALL_G13 = 1 };

typedef struct orc_solver orc_solver;

/* W0: per cell (rho, ux, uy, uz, Tt, Tr); Tr ignored for Shakhov.  f0 = Maxwellian(W0). */
int orc_create(const orc_mesh *m, const orc_vgrid *vg, const orc_gas *g, const orc_opts *o,
               const double *W0, orc_solver **out);
void orc_destroy(orc_solver *s);

/* Replace the VDFs (layout [cell][v], v = ix + nx (iy + ny iz)); f1 may be NULL for Shakhov.
   The per-cell state used by the next kinetic step becomes the moments of the new f. */
int orc_set_f(orc_solver *s, const double *f0, const double *f1);
int orc_get_f(const orc_solver *s, double *f0, double *f1);

/* One outer iteration of Algorithm 1 (mode GSIS) or one plain DVM step (mode DVM). */
int orc_step(orc_solver *s);
/* 1/dt of the kinetic delta form and the mode for the following steps. */
void orc_set_kin_inv_dt(orc_solver *s, double inv_dt);
void orc_set_mode(orc_solver *s, int mode);
/* n plain kinetic steps whatever the mode (the preconditioning of Algorithm 1). */
int orc_presteps(orc_solver *s, int n);
/* Euler preconditioning: n inner steps of the inviscid synthetic solve (slip walls, far field
   against the free stream) from the current state; f restarts as the Maxwellian of the result. */
int orc_euler_presteps(orc_solver *s, int n);

/* The outward wall flux (per unit area; rho, momentum, energy, rotational energy) of a cell
   state pr = (rho, u, Tt, Tr) meeting the diffuse wall of boundary patch `patch` along the unit
   normal n: mode ORC_WALL_EQ uses the local Maxwellian, ORC_WALL_G13 the Grad-13 VDF built
   with the stress, translational and rotational heat fluxes of m18 (the layout of
   orc_get_half_moments). */
void orc_wall_flux(const orc_solver *s, int mode, int patch, const double *pr, const double *m18, const double *n,
                   double *F);

/* Parts of one outer step, for timing and unit tests. */
int orc_wall_prepass(orc_solver *s);                       /* rho_w from the current f */
int orc_kinetic_velocities(orc_solver *s, int v0, int v1); /* kinetic update of velocities [v0,v1) */
int orc_macro_from_current(orc_solver *s);                 /* moments, HoT, macro solve on current f */

/* Accessors.  Cell-major arrays. */
int orc_ncells(const orc_solver *s);
int orc_nvel(const orc_solver *s);
int orc_nwall(const orc_solver *s);
double orc_eps(const orc_solver *s);             /* eps of the last step */
double orc_mass_scale(const orc_solver *s);      /* closed-domain mass rescaling of the last kinetic step */
int orc_macro_iters(const orc_solver *s);        /* inner steps used by the last macro solve */
/* state W used by the next kinetic step: per cell rho, ux, uy, uz, Tt, Tr */
void orc_get_W(const orc_solver *s, double *out6);
/* moments of f^{n+1/2} of the last step: per cell rho, u(3), Tt, Tr, sigma(xx,yy,zz,xy,xz,yz), qt(3), qr(3) = 18 */
void orc_get_half_moments(const orc_solver *s, double *out18);
/* HoT of the last GSIS step: per cell sigma(6), qt(3), qr(3) = 12 */
void orc_get_hot(const orc_solver *s, double *out12);
/* per wall face: cell, side, rho_w (from the pre-pass of the last step) and the kinetic
   wall flux (6 components, outward) of the last kinetic step */
void orc_get_wall(const orc_solver *s, int *cell, int *side, double *rho_w, double *flux6);
/* geometry: per cell volume and centre; per cell and side the outward area vector and face
   centre (zeros for absent faces) */
void orc_get_geometry(const orc_solver *s, double *vol, double *centre3, double *S18, double *xf18);

/* LSQ gradient and Venkatakrishnan cell limiter of a cell field q[cell] (pins). */
void orc_cell_gradient(const orc_solver *s, int cell, const double *q, double *grad3);
double orc_cell_limiter(const orc_solver *s, int cell, const double *q);
/* Face values of a cell on its six sides for a field q over cells (the reconstruction the kinetic
   step applies to each velocity's f, orc_opts.positive_faces included). */
void orc_cell_faces(const orc_solver *s, int cell, const double *q, double *out6);
/* NSF stress and heat fluxes (sigma xx yy zz xy xz yz, q_t, q_r) of the synthetic solve at the
   face between `cell` and its neighbour on `side` (the cell itself on a boundary side) for the
   conservative state W [cell][6]. */
int orc_face_nsf(const orc_solver *s, const double *W, int cell, int side, double *out12);
/* per cell and side the outward kinetic face flux (mass, momentum(3), energy, internal
   energy) of the last kinetic step: 36 per cell */
void orc_get_face_flux(const orc_solver *s, double *out36);

/* Model pieces, exposed for the pins. */
double orc_tau(const orc_gas *g, double rho, double Tt);
void orc_conductivity(const orc_gas *g, double mu, double *kt, double *kr);
/* reference distributions g0, g1 at molecular velocity xi for state
   st = (rho, ux, uy, uz, Tt, Tr, qtx, qty, qtz, qrx, qry, qrz) */
void orc_reference(const orc_gas *g, const double *st, const double *xi, double *g0, double *g1);
/* Venkatakrishnan face limiter value for (Delta_max_or_min, Delta_2, eps^2) */
double orc_venkat_face(double dm, double d2, double eps2);

#ifdef __cplusplus
}
#endif
#endif
