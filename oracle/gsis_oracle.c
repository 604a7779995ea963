/*
 * gsis_oracle.c -- plain FP64 CPU oracle of GSIS (arXiv 2310.18916).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference leg of bench.py.  It shares no code, header, table or
 * helper with the CUDA library under paper_2310_18916_gb300/.
 *
 * Every function follows the paper's equations in the paper's order, in plain
 * loops over cells and velocities; the only parallelism is an optional OpenMP loop
 * over independent discrete velocities, and every reduction runs sequentially in a
 * fixed index order, so results do not depend on the thread count.
 *
 * Units: x in L, xi in v0 = sqrt(2 R T0), rho in rho0, T in T0; R T -> T/2.
 *
 * Parity status of each part (pins live in tests/test_oracle_*.py):
 *   geometry, LSQ gradient, Venkatakrishnan limiter, moments, reference
 *   distributions, tau, conductivities, collision conservation, uniform
 *   equilibrium, free-molecular Couette, wall mass balance, NSF limit,
 *   refinement, GSIS-vs-DVM fixed point, O-grid geometry (wrapped azimuth, pole faces),
 *   far field (uniform free stream, collisionless reservoir against a wall), the
 *   free-molecular force on a cylinder, the Euler presteps (mirror symmetry of the converged
 *   inviscid cylinder flow), the jump term of the viscous face gradients on meshes with
 *   simplices (no jump for linear fields, the difference quotient along the centre line at
 *   weight 1, affine in the weight): pinned.
 *   Macro-solver details the paper leaves to its references (face gradient,
 *   Gamma, time step): pinned only through the fixed point (kinetic/GSIS agree).
 */
#include "gsis_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846
#define STENCIL_MAX 80
#define SQRT_PI 1.77245385090551602730

struct orc_solver {
  int ni, nj, nk, nc;
  int nvx, nvy, nvz, nv;
  int active[3];
  int bc[6];
  double wall_u[6][3], wall_T[6];
  orc_gas g;
  orc_opts o;
  int nvdf;              /* 1 (Shakhov) or 2 (Rykov) */
  int nW;                /* 5 (Shakhov) or 6 (Rykov) conservative components */
  double *vx, *vy, *vz, *wx, *wy, *wz;
  double *pts;           /* unstructured velocity set [v][4] (NULL: the tensor product above) */
  /* geometry */
  double *vol, *xc, *S, *xf, *eps2;
  int *nb;               /* per cell and side: >=0 neighbour, -1 wall, -2 absent (inactive axis),
                            -3 axis (zero area), -4 far field */
  int open;              /* a far-field side exists: mass is not conserved by the domain */
  int *wid;              /* per cell and side: wall face id or -1 */
  int nwall;
  int *wcell, *wside;
  double *rho_w;
  /* VDFs, stored velocity-major [v][cell] */
  double *f0, *f1;
  /* per cell state for the reference distribution: rho,u(3),Tt,Tr,qt(3),qr(3) */
  double *st;
  double *Mh;            /* half-step moments, 18 per cell */
  double *hot;           /* 12 per cell */
  double *kin;           /* kinetic sigma(6), qt(3), qr(3) per cell */
  double *fkin;          /* per cell and side: outward kinetic face flux of the last kinetic step (6) */
  double eps;
  int macro_iters;
  int *corder;           /* per octant (8) the cells sorted by colour, then by index */
  /* unstructured meshes: per cell and side the neighbour's side of the shared face and the
     boundary patch; per cell its colour (NULL on structured blocks: side ^ 1, the side itself,
     hyperplanes / red-black) */
  int *nbf, *pat, *colour;
  int ncolour;
  /* unstructured meshes: the least-squares stencil of each cell (-1 padded): on a mesh of
     hexahedra the face neighbours in side order; on a mesh with prisms, pyramids or tetrahedra
     every other cell sharing a node with it, ascending (face neighbours alone leave the
     second-order upwind scheme unstable on simplices) */
  int *sten;
  int simplex;           /* an unstructured mesh with prisms, pyramids or tetrahedra */
  double jump;           /* the weight of the jump term in the viscous face gradients */
  double mass_ref;       /* total mass of the closed domain (set with f) */
  double mass_scale;     /* rescaling applied after the last kinetic step */
};

static int cid(const orc_solver *s, int i, int j, int k) { return i + s->ni * (j + s->nj * k); }
/* the neighbour's side of the face cell i shares through `side`, and the boundary patch of a side */
static int opp_side(const orc_solver *s, int i, int side) { return s->nbf ? s->nbf[6 * i + side] : side ^ 1; }
static int patch_of(const orc_solver *s, int i, int side) { return s->pat ? s->pat[6 * i + side] : side; }

/* discrete velocity v and its quadrature weight (Section 3.1): a node of the tensor product of
   the three axis grids, or point v of an unstructured set with its velocity cell's volume */
static void vel_of(const orc_solver *s, int v, double xi[3], double *w) {
  if (s->pts) {
    const double *q = s->pts + 4 * (size_t)v;
    xi[0] = q[0]; xi[1] = q[1]; xi[2] = q[2];
    *w = q[3];
    return;
  }
  int ix = v % s->nvx, iy = (v / s->nvx) % s->nvy, iz = v / (s->nvx * s->nvy);
  xi[0] = s->vx[ix]; xi[1] = s->vy[iy]; xi[2] = s->vz[iz];
  *w = s->wx[ix] * s->wy[iy] * s->wz[iz];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ---------------- model: Section 2 ---------------- */

/* Maxwellian f^(0) of Section 2.3 in nondimensional form. */
static double maxwellian(double rho, const double *u, double T, const double *xi) {
  double c0 = xi[0] - u[0], c1 = xi[1] - u[1], c2 = xi[2] - u[2];
  return rho * pow(PI * T, -1.5) * exp(-(c0 * c0 + c1 * c1 + c2 * c2) / T);
}

/* tau = mu(Tt)/p_t with mu = mu(T0)(Tt/T0)^omega and Kn = mu(T0)/(p0 L) sqrt(pi R T0/2)
   (Section 2.1); nondimensionally mu = Kn/sqrt(pi) Tt^omega and p_t = rho Tt/2. */
double orc_tau(const orc_gas *g, double rho, double Tt) {
  return 2.0 * g->Kn / SQRT_PI * pow(Tt, g->omega - 1.0) / rho;
}

static double visc(const orc_gas *g, double Tt) { return g->Kn / SQRT_PI * pow(Tt, g->omega); }

/* Eq. mu_kappa: (kt, kr) = (mu R/2) A^{-1} (5, d_r); R = 1/2 nondimensionally.
   The Shakhov (monatomic, Pr = 2/3) case is A_tt = 2/3, d_r = 0. */
void orc_conductivity(const orc_gas *g, double mu, double *kt, double *kr) {
  if (g->model == ORC_SHAKHOV) {
    *kt = mu / 4.0 * (5.0 / (2.0 / 3.0));
    *kr = 0.0;
    return;
  }
  double Att = g->A[0], Atr = g->A[1], Art = g->A[2], Arr = g->A[3];
  double det = Att * Arr - Atr * Art;
  double i00 = Arr / det, i01 = -Atr / det, i10 = -Art / det, i11 = Att / det;
  *kt = mu / 4.0 * (i00 * 5.0 + i01 * g->d_r);
  *kr = mu / 4.0 * (i10 * 5.0 + i11 * g->d_r);
}

/* Reference distributions g_0t, g_0r, g_1t, g_1r of Section 2.2 combined as
   g = (1 - 1/Z_r) g_t + g_r / Z_r (Section 3.2); heat fluxes q0, q1 from the
   2x2 relaxation map of Section 2.2.  Shakhov: g0 = g_0t, no g1. */
void orc_reference(const orc_gas *g, const double *st, const double *xi, double *g0, double *g1) {
  double rho = st[0], Tt = st[4], Tr = st[5];
  const double *u = st + 1, *qt = st + 6, *qr = st + 9;
  double c[3] = {xi[0] - u[0], xi[1] - u[1], xi[2] - u[2]};
  double c2 = dot3(c, c);
  double Mt = rho * pow(PI * Tt, -1.5) * exp(-c2 / Tt);
  /* 2 q.c/(15 R Tt p_t) (c^2/(2 R Tt) - 5/2) with R Tt = Tt/2, p_t = rho Tt/2 */
  double g0t = Mt * (1.0 + 8.0 / (15.0 * rho * Tt * Tt) * dot3(qt, c) * (c2 / Tt - 2.5));
  if (g->model == ORC_SHAKHOV) {
    *g0 = g0t;
    if (g1) *g1 = 0.0;
    return;
  }
  double dr = g->d_r, Zr = g->Z_r;
  double Att = g->A[0], Atr = g->A[1], Art = g->A[2], Arr = g->A[3];
  double T = (3.0 * Tt + dr * Tr) / (3.0 + dr);
  double q0[3], q1[3];
  for (int a = 0; a < 3; ++a) {
    q0[a] = ((2.0 - 3.0 * Att) * Zr + 1.0) * qt[a] - 3.0 * Atr * Zr * qr[a];
    q1[a] = -Art * Zr * qt[a] + (-Arr * Zr + 1.0) * qr[a];
  }
  double MT = rho * pow(PI * T, -1.5) * exp(-c2 / T);
  double g0r = MT * (1.0 + 8.0 / (15.0 * rho * T * T) * dot3(q0, c) * (c2 / T - 2.5));
  /* (d_r/2) R T_r = d_r T_r / 4;  (2 pi R T)^{-3/2} = (pi T)^{-3/2};  q.c/(R T) = 2 q.c/T */
  double g1t = dr * Tr / 4.0 * g0t + pow(PI * Tt, -1.5) * (2.0 * dot3(qr, c) / Tt) * exp(-c2 / Tt);
  double g1r = dr * T / 4.0 * g0r + pow(PI * T, -1.5) * (2.0 * dot3(q1, c) / T) * exp(-c2 / T);
  *g0 = (1.0 - 1.0 / Zr) * g0t + g0r / Zr;
  if (g1) *g1 = (1.0 - 1.0 / Zr) * g1t + g1r / Zr;
}

/* ---------------- geometry ---------------- */

static void node(const orc_mesh *m, int I, int J, int K, double p[3]) {
  const double *q = m->nodes + 3 * ((size_t)I + (size_t)(m->ni + 1) * ((size_t)J + (size_t)(m->nj + 1) * K));
  p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
}

/* quad face: area vector 1/2 (p2-p0) x (p3-p1), centre = mean of the corners */
static void quad(const double p[4][3], double S[3], double x[3]) {
  double a[3], b[3];
  for (int d = 0; d < 3; ++d) { a[d] = p[2][d] - p[0][d]; b[d] = p[3][d] - p[1][d]; }
  S[0] = 0.5 * (a[1] * b[2] - a[2] * b[1]);
  S[1] = 0.5 * (a[2] * b[0] - a[0] * b[2]);
  S[2] = 0.5 * (a[0] * b[1] - a[1] * b[0]);
  for (int d = 0; d < 3; ++d) x[d] = 0.25 * (p[0][d] + p[1][d] + p[2][d] + p[3][d]);
}

static int build_geometry(orc_solver *s, const orc_mesh *m) {
  int n[3] = {s->ni, s->nj, s->nk};
  s->open = 0;
  for (int a = 0; a < 3; ++a) {
    int lo = m->bc[2 * a], hi = m->bc[2 * a + 1];
    s->active[a] = n[a] > 1;
    if (!s->active[a]) {
      if (lo != ORC_BC_PERIODIC || hi != ORC_BC_PERIODIC) return ORC_E_INVALID;
    } else if ((lo == ORC_BC_PERIODIC) != (hi == ORC_BC_PERIODIC)) {
      return ORC_E_INVALID;
    } else if (lo == ORC_BC_PERIODIC && n[a] < 3) {
      return ORC_E_INVALID;  /* a wrapped axis needs distinct neighbours on both sides */
    }
    for (int t = 0; t < 2; ++t) {
      int b = m->bc[2 * a + t];
      if (b < ORC_BC_WALL || b > ORC_BC_AXIS) return ORC_E_INVALID;
      if (b == ORC_BC_FARFIELD) s->open = 1;
    }
  }
  s->nwall = 0;
  for (int k = 0; k < s->nk; ++k)
    for (int j = 0; j < s->nj; ++j)
      for (int i = 0; i < s->ni; ++i) {
        int c = cid(s, i, j, k);
        double corner[8][3];
        int t = 0;
        for (int dk = 0; dk < 2; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) node(m, i + di, j + dj, k + dk, corner[t++]);
        double *xc = s->xc + 3 * c;
        xc[0] = xc[1] = xc[2] = 0.0;
        for (t = 0; t < 8; ++t)
          for (int d = 0; d < 3; ++d) xc[d] += corner[t][d] / 8.0;
        double V = 0.0;
        for (int side = 0; side < 6; ++side) {
          int a = side / 2, hi = side % 2;
          double p[4][3];
          int I0 = i, J0 = j, K0 = k;
          if (a == 0) {
            I0 += hi;
            node(m, I0, J0, K0, p[0]); node(m, I0, J0 + 1, K0, p[1]);
            node(m, I0, J0 + 1, K0 + 1, p[2]); node(m, I0, J0, K0 + 1, p[3]);
          } else if (a == 1) {
            J0 += hi;
            node(m, I0, J0, K0, p[0]); node(m, I0 + 1, J0, K0, p[1]);
            node(m, I0 + 1, J0, K0 + 1, p[2]); node(m, I0, J0, K0 + 1, p[3]);
          } else {
            K0 += hi;
            node(m, I0, J0, K0, p[0]); node(m, I0 + 1, J0, K0, p[1]);
            node(m, I0 + 1, J0 + 1, K0, p[2]); node(m, I0, J0 + 1, K0, p[3]);
          }
          double *S = s->S + 18 * c + 3 * side, *xf = s->xf + 18 * c + 3 * side;
          quad((const double(*)[3])p, S, xf);
          double r[3] = {xf[0] - xc[0], xf[1] - xc[1], xf[2] - xc[2]};
          if (dot3(S, r) < 0) { S[0] = -S[0]; S[1] = -S[1]; S[2] = -S[2]; }
          V += dot3(xf, S) / 3.0;  /* divergence theorem with F = x/3 */
          int idx[3] = {i, j, k};
          idx[a] += hi ? 1 : -1;
          int nbr;
          s->wid[6 * c + side] = -1;
          if (!s->active[a]) nbr = -2;
          else if (idx[a] >= 0 && idx[a] < n[a]) nbr = cid(s, idx[0], idx[1], idx[2]);
          else if (m->bc[side] == ORC_BC_PERIODIC) {
            idx[a] = (idx[a] + n[a]) % n[a];
            nbr = cid(s, idx[0], idx[1], idx[2]);
          } else if (m->bc[side] == ORC_BC_AXIS) nbr = -3;
          else if (m->bc[side] == ORC_BC_FARFIELD) nbr = -4;
          else { nbr = -1; s->wid[6 * c + side] = s->nwall++; }
          s->nb[6 * c + side] = nbr;
        }
        if (!(V > 0)) return ORC_E_INVALID;
        s->vol[c] = V;
        double h = cbrt(V);
        s->eps2[c] = pow(s->o.venkat_K * h, 3.0);
      }
  s->wcell = (int *)malloc(sizeof(int) * (s->nwall + 1));
  s->wside = (int *)malloc(sizeof(int) * (s->nwall + 1));
  s->rho_w = (double *)calloc(s->nwall + 1, sizeof(double));
  if (!s->wcell || !s->wside || !s->rho_w) return ORC_E_OOM;
  for (int c = 0; c < s->nc; ++c)
    for (int side = 0; side < 6; ++side)
      if (s->wid[6 * c + side] >= 0) { s->wcell[s->wid[6 * c + side]] = c; s->wside[s->wid[6 * c + side]] = side; }
  return ORC_OK;
}

/* ---------------- reconstruction (Section 3.2) ---------------- */

/* Least-squares gradient over the face neighbours inside the domain:
   minimise sum_j (q_j - q_i - grad . (x_j - x_i))^2 via its 3x3 normal equations. */
static void lsq_grad(const orc_solver *s, int i, const double *q, int stride, double g[3]) {
  double A[3][3] = {{0}}, b[3] = {0};
  const double *xi = s->xc + 3 * i;
  for (int t = 0; t < (s->sten ? STENCIL_MAX : 6); ++t) {
    int j = s->sten ? s->sten[(size_t)STENCIL_MAX * i + t] : s->nb[6 * i + t];
    if (j < 0) continue;
    double d[3] = {s->xc[3 * j] - xi[0], s->xc[3 * j + 1] - xi[1], s->xc[3 * j + 2] - xi[2]};
    double dq = q[(size_t)j * stride] - q[(size_t)i * stride];
    for (int r = 0; r < 3; ++r) {
      b[r] += d[r] * dq;
      for (int cc = 0; cc < 3; ++cc) A[r][cc] += d[r] * d[cc];
    }
  }
  for (int a = 0; a < 3; ++a)
    if (!s->active[a]) {
      for (int t = 0; t < 3; ++t) A[a][t] = A[t][a] = 0.0;
      A[a][a] = 1.0; b[a] = 0.0;
    }
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (s->colour) {
    /* unstructured: a cell whose neighbours leave the fit undetermined (a corner tetrahedron)
       adds its boundary faces' centres with its own value (rows that change A, not b) */
    double tr = 0.0;
    int nact = 0;
    for (int a = 0; a < 3; ++a)
      if (s->active[a]) { tr += A[a][a]; ++nact; }
    if (!(det > 1e-9 * pow(tr, nact))) {
      for (int side = 0; side < 6; ++side) {
        int j = s->nb[6 * i + side];
        const double *S = s->S + 18 * i + 3 * side, *xf = s->xf + 18 * i + 3 * side;
        if (j >= 0 || j == -2 || !(dot3(S, S) > 0)) continue;
        double r[3] = {xf[0] - xi[0], xf[1] - xi[1], xf[2] - xi[2]};
        for (int a = 0; a < 3; ++a)
          for (int cc = 0; cc < 3; ++cc)
            if (s->active[a] && s->active[cc]) A[a][cc] += r[a] * r[cc];
      }
      det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
            A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    }
  }
  /* Cramer's rule */
  for (int col = 0; col < 3; ++col) {
    double M[3][3];
    memcpy(M, A, sizeof M);
    for (int r = 0; r < 3; ++r) M[r][col] = b[r];
    double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    g[col] = dc / det;
  }
}

/* Venkatakrishnan limiter for one face: (1/D2) [(Dm^2+e^2) D2 + 2 D2^2 Dm] / [Dm^2 + 2 D2^2 + Dm D2 + e^2]. */
double orc_venkat_face(double dm, double d2, double eps2) {
  if (d2 == 0.0) return 1.0;
  double num = (dm * dm + eps2) * d2 + 2.0 * d2 * d2 * dm;
  double den = d2 * (dm * dm + 2.0 * d2 * d2 + dm * d2 + eps2);
  return num / den;
}

/* Cell limiter: minimum over every face of the cell (boundary faces included), capped at 1;
   the bounds are the extremes over the cell and its neighbours inside the domain. */
static double venkat_cell(const orc_solver *s, int i, const double *q, int stride, const double g[3]) {
  double qi = q[(size_t)i * stride], qmax = qi, qmin = qi;
  for (int side = 0; side < 6; ++side) {
    int j = s->nb[6 * i + side];
    if (j < 0) continue;
    double qj = q[(size_t)j * stride];
    if (qj > qmax) qmax = qj;
    if (qj < qmin) qmin = qj;
  }
  double phi = 1.0;
  for (int side = 0; side < 6; ++side) {
    if (s->nb[6 * i + side] == -2 || s->nb[6 * i + side] == -3) continue;
    const double *xf = s->xf + 18 * i + 3 * side, *xc = s->xc + 3 * i;
    double r[3] = {xf[0] - xc[0], xf[1] - xc[1], xf[2] - xc[2]};
    double d2 = dot3(g, r);
    double dm = d2 > 0 ? qmax - qi : (d2 < 0 ? qmin - qi : 0.0);
    double p = orc_venkat_face(dm, d2, s->eps2[i]);
    if (p < phi) phi = p;
  }
  return phi;
}

/* Face values of cell i on each of its sides: q_i + d, d = phi grad q_i . (x_f - x_i).  With
   orc_opts.positive_faces a face value that would fall below the cell value (d < 0) is
   q_i^2 / (q_i - d) instead: positive whenever q_i is, equal to q_i + d to first order in d / q_i
   (the two differ by d^2 / (q_i - d)), and continuous with its first derivative at d = 0.  The
   linear form lets a VDF's steep fall into near-vacuum or into a velocity tail reconstruct
   negative face values; a non-positive q_i keeps its own value. */
static void reconstruct(const orc_solver *s, int i, const double *q, int stride, double out[6]) {
  double g[3];
  lsq_grad(s, i, q, stride, g);
  double phi = venkat_cell(s, i, q, stride, g);
  const double *xc = s->xc + 3 * i, qi = q[(size_t)i * stride];
  for (int side = 0; side < 6; ++side) {
    const double *xf = s->xf + 18 * i + 3 * side;
    double r[3] = {xf[0] - xc[0], xf[1] - xc[1], xf[2] - xc[2]};
    double d = phi * dot3(g, r);
    if (s->o.positive_faces && d < 0)
      out[side] = qi > 0 ? qi * qi / (qi - d) : qi;
    else
      out[side] = qi + d;
  }
}

/* ---------------- walls ---------------- */

static double wall_maxwellian(const orc_solver *s, int side, const double *xi) {
  return maxwellian(1.0, s->wall_u[side], s->wall_T[side], xi);
}

/* Diffuse wall: the re-emitted density rho_w balances the mass flux of the
   molecules reaching the wall, whose face values are the cell's reconstruction. */
int orc_wall_prepass(orc_solver *s) {
#pragma omp parallel for schedule(dynamic) num_threads(s->o.nthreads > 0 ? s->o.nthreads : 1)
  for (int wf = 0; wf < s->nwall; ++wf) {
    int c = s->wcell[wf], side = s->wside[wf];
    const double *S = s->S + 18 * c + 3 * side;
    double num = 0.0, den = 0.0, ff[6], xi[3], w;
    for (int v = 0; v < s->nv; ++v) {
      vel_of(s, v, xi, &w);
      double sn = dot3(xi, S);
      if (sn > 0) {
        reconstruct(s, c, s->f0 + (size_t)v * s->nc, 1, ff);
        num += w * sn * ff[side];
      } else if (sn < 0) {
        den += w * (-sn) * wall_maxwellian(s, patch_of(s, c, side), xi);
      }
    }
    s->rho_w[wf] = num / den;
  }
  return ORC_OK;
}

/* ---------------- kinetic step (Section 3.2, Algorithm 3 body) ---------------- */

typedef struct {
  double *ff, *r, *df, *D;
  double *fl;            /* this velocity's outward face fluxes [cell][side][6] */
} kin_work;

/* A far-field face lets the free stream in unless the stream leaves through it faster than
   sound (U_inf . n > c_inf): a reservoir boundary, except where nothing travels upstream into
   the domain.  c_inf^2 = gamma R T_inf with R T = T/2 and the equilibrium ratio of specific
   heats of the free stream, gamma = (5 + d_r)/(3 + d_r) (5/3 monatomic, 7/5 for d_r = 2). */
static int far_inflow(const orc_solver *s, int i, int side) {
  const int p = patch_of(s, i, side);
  const double *U = s->wall_u[p], *S = s->S + 18 * i + 3 * side;
  double dr = s->nvdf == 2 ? s->g.d_r : 0.0;
  double gam = (5.0 + dr) / (3.0 + dr);
  return dot3(U, S) <= sqrt(0.5 * gam * s->wall_T[p]) * sqrt(dot3(S, S));
}

/* Face values (f, and f1 for Rykov) entering the domain through the boundary face (i, side)
   for velocity xi: at a wall the re-emitted rho_w M_w (f1 = (d_r T_w / 4) f); at a far field
   the free-stream Maxwellian, except where the free stream leaves through the face faster than
   sound, where they carry the cell's own values own[] (zero gradient, first order). */
static void boundary_in(const orc_solver *s, int i, int side, const double *xi, const double own[2], double e[2]) {
  if (s->nb[6 * i + side] == -1) {
    const int p = patch_of(s, i, side);
    double M = s->rho_w[s->wid[6 * i + side]] * wall_maxwellian(s, p, xi);
    e[0] = M;
    e[1] = s->g.d_r * s->wall_T[p] / 4.0 * M;
  } else if (far_inflow(s, i, side)) {
    const int p = patch_of(s, i, side);
    double M = maxwellian(1.0, s->wall_u[p], s->wall_T[p], xi);
    e[0] = M;
    e[1] = s->g.d_r * s->wall_T[p] / 4.0 * M;
  } else {
    e[0] = own[0];
    e[1] = own[1];
  }
}


static void point_implicit(const orc_solver *s, const double *xi, int i, kin_work *wk, int q) {
  double acc = wk->r[(size_t)q * s->nc + i];
  for (int side = 0; side < 6; ++side) {
    int j = s->nb[6 * i + side];
    if (j < 0) continue;  /* wall increments are lagged: Delta f_wall = 0 */
    double sn = dot3(xi, s->S + 18 * i + 3 * side);
    if (sn < 0) acc += (-sn) / s->vol[i] * wk->df[(size_t)q * s->nc + j];
  }
  wk->df[(size_t)q * s->nc + i] = acc / wk->D[i];
}

/* One kinetic step for discrete velocity v: delta-form equation with the
   second-order upwind explicit residual r_i^n and the first-order upwind
   implicit operator, solved by point-implicit sweeps; then f += Delta f. */
static void kinetic_velocity(orc_solver *s, int v, kin_work *wk) {
  int nc = s->nc;
  double xi[3], w;
  vel_of(s, v, xi, &w);
  int sgn[3] = {xi[0] >= 0 ? 1 : -1, xi[1] >= 0 ? 1 : -1, xi[2] >= 0 ? 1 : -1};
  double *fq[2] = {s->f0 + (size_t)v * nc, s->nvdf == 2 ? s->f1 + (size_t)v * nc : NULL};
  for (int q = 0; q < s->nvdf; ++q)
    for (int i = 0; i < nc; ++i) reconstruct(s, i, fq[q], 1, wk->ff + ((size_t)q * nc + i) * 6);
  for (int i = 0; i < nc; ++i) {
    double gq[2];
    orc_reference(&s->g, s->st + 12 * i, xi, &gq[0], &gq[1]);
    double tau = orc_tau(&s->g, s->st[12 * i], s->st[12 * i + 4]);
    double D = s->o.kin_inv_dt + 1.0 / tau;
    double flux[2] = {0.0, 0.0};
    for (int side = 0; side < 6; ++side) {
      int j = s->nb[6 * i + side];
      if (j == -2 || j == -3) continue;
      double sn = dot3(xi, s->S + 18 * i + 3 * side);
      if (sn > 0) {
        D += sn / s->vol[i];
        for (int q = 0; q < s->nvdf; ++q) flux[q] += sn * wk->ff[((size_t)q * nc + i) * 6 + side];
      } else if (sn < 0) {
        if (j >= 0) {
          int opp = opp_side(s, i, side);
          for (int q = 0; q < s->nvdf; ++q) flux[q] += sn * wk->ff[((size_t)q * nc + j) * 6 + opp];
        } else {
          double own[2] = {0.0, 0.0}, e[2];
          for (int q = 0; q < s->nvdf; ++q) own[q] = fq[q][i];
          boundary_in(s, i, side, xi, own, e);
          for (int q = 0; q < s->nvdf; ++q) flux[q] += sn * e[q];
        }
      }
    }
    wk->D[i] = D;
    for (int q = 0; q < s->nvdf; ++q)
      wk->r[(size_t)q * nc + i] = (gq[q] - fq[q][i]) / tau - flux[q] / s->vol[i];
  }
  for (int q = 0; q < s->nvdf; ++q) {
    double *df = wk->df + (size_t)q * nc;
    for (int i = 0; i < nc; ++i) df[i] = 0.0;
    for (int pass = 0; pass < s->o.n_sweeps; ++pass) {
      if (s->o.schedule == ORC_SCHED_COLOUR) {
        /* colours = hyperplanes i'+j'+k' in the upwind order of this velocity's octant;
           cells of one colour never share a face, so their order does not matter */
        const int *ord = s->corder + (size_t)nc * ((sgn[0] < 0) + 2 * (sgn[1] < 0) + 4 * (sgn[2] < 0));
        for (int t = 0; t < nc; ++t) point_implicit(s, xi, ord[t], wk, q);
      } else {
        for (int i = 0; i < nc; ++i) point_implicit(s, xi, i, wk, q);
        for (int i = nc - 1; i >= 0; --i) point_implicit(s, xi, i, wk, q);
      }
    }
  }
  /* Moments of this velocity's face fluxes at the new level: on every face the upwind
     face value of f^n plus the upwind cell's increment (the wall re-emission has no
     increment).  These are exactly the fluxes of the delta-form equation just solved. */
  if (wk->fl) {
    double e2 = 0.5 * dot3(xi, xi);
    for (int i = 0; i < nc; ++i)
      for (int side = 0; side < 6; ++side) {
        double *out = wk->fl + (size_t)36 * i + 6 * side;
        for (int k = 0; k < 6; ++k) out[k] = 0.0;
        int j = s->nb[6 * i + side];
        if (j == -2 || j == -3) continue;
        double sn = dot3(xi, s->S + 18 * i + 3 * side), e[2] = {0.0, 0.0};
        if (sn > 0) {
          for (int q = 0; q < s->nvdf; ++q)
            e[q] = wk->ff[((size_t)q * nc + i) * 6 + side] + wk->df[(size_t)q * nc + i];
        } else if (sn < 0) {
          if (j >= 0) {
            for (int q = 0; q < s->nvdf; ++q)
              e[q] = wk->ff[((size_t)q * nc + j) * 6 + opp_side(s, i, side)] + wk->df[(size_t)q * nc + j];
          } else {
            double own[2] = {0.0, 0.0};
            for (int q = 0; q < s->nvdf; ++q) own[q] = fq[q][i];
            boundary_in(s, i, side, xi, own, e);
            if (s->nvdf == 1) e[1] = 0.0;
          }
        }
        out[0] = w * sn * e[0];
        out[1] = w * sn * xi[0] * e[0];
        out[2] = w * sn * xi[1] * e[0];
        out[3] = w * sn * xi[2] * e[0];
        out[4] = w * sn * (e2 * e[0] + e[1]);
        out[5] = w * sn * e[1];
      }
  }
  for (int q = 0; q < s->nvdf; ++q)
    for (int i = 0; i < nc; ++i) fq[q][i] += wk->df[(size_t)q * nc + i];
}

int orc_kinetic_velocities(orc_solver *s, int v0, int v1) {
  int nc = s->nc, nq = s->nvdf, bad = 0;
  /* velocities are processed in chunks; inside a chunk in parallel, and the chunk's face
     fluxes are then summed in ascending velocity order, independent of the thread count */
  int chunk = (int)(4000000 / (36 * (size_t)nc));
  if (chunk < 1) chunk = 1;
  if (chunk > 256) chunk = 256;
  double *fl = (double *)malloc(sizeof(double) * 36 * (size_t)nc * chunk);
  if (!fl) return ORC_E_OOM;
  if (v0 == 0) memset(s->fkin, 0, sizeof(double) * 36 * (size_t)nc);
  for (int c0 = v0; c0 < v1 && !bad; c0 += chunk) {
    int c1 = c0 + chunk < v1 ? c0 + chunk : v1;
#pragma omp parallel num_threads(s->o.nthreads > 0 ? s->o.nthreads : 1)
    {
      kin_work wk;
      wk.ff = (double *)malloc(sizeof(double) * 6 * (size_t)nc * nq);
      wk.r = (double *)malloc(sizeof(double) * (size_t)nc * nq);
      wk.df = (double *)malloc(sizeof(double) * (size_t)nc * nq);
      wk.D = (double *)malloc(sizeof(double) * (size_t)nc);
      if (!wk.ff || !wk.r || !wk.df || !wk.D) {
#pragma omp atomic write
        bad = 1;
      } else {
#pragma omp for schedule(dynamic, 1)
        for (int v = c0; v < c1; ++v) {
          wk.fl = fl + (size_t)36 * nc * (v - c0);
          kinetic_velocity(s, v, &wk);
        }
      }
      free(wk.ff); free(wk.r); free(wk.df); free(wk.D);
    }
    for (int v = c0; v < c1; ++v) {
      const double *src = fl + (size_t)36 * nc * (v - c0);
      for (size_t t = 0; t < (size_t)36 * nc; ++t) s->fkin[t] += src[t];
    }
  }
  free(fl);
  return bad ? ORC_E_OOM : ORC_OK;
}

/* ---------------- unstructured meshes (Section 5's cell shapes) ---------------- */

/* the six sides of a hexahedron of corners t = (t & 1, (t >> 1) & 1, t >> 2), in cyclic order */
static const int HEX_SIDE[6][4] = {{0, 2, 6, 4}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 3, 7, 6}, {0, 1, 3, 2}, {4, 5, 7, 6}};

typedef struct { int id[4]; int face; } face_key;

static int key_cmp(const void *a, const void *b) {
  const face_key *x = (const face_key *)a, *y = (const face_key *)b;
  for (int t = 0; t < 4; ++t)
    if (x->id[t] != y->id[t]) return x->id[t] < y->id[t] ? -1 : 1;
  return x->face < y->face ? -1 : (x->face > y->face);
}

static void unode(const orc_mesh *m, int id, double p[3]) {
  for (int d = 0; d < 3; ++d) p[d] = m->unodes[3 * (size_t)id + d];
}

/* Cells given as hexahedra of node ids (other shapes repeat ids).  Geometry per side: four
   distinct corners, the quadrilateral of the structured blocks (half the cross product of the
   diagonals, centre the corner mean); three, a triangle (half the cross product of two edges,
   centre their mean); fewer, no area and no flux.  Cell centre: mean of the distinct corners.
   Shared sides: the same set of node ids on two cells.  Other sides take their patch's
   condition; a PERIODIC patch (faces normal to z) makes a one-layer mesh: no transport across
   it and no z gradient.  Colours: greedy, cells in index order, each the smallest colour none of
   its face neighbours already has. */
static int build_geometry_unstructured(orc_solver *s, const orc_mesh *m) {
  int nc = s->nc;
  s->open = 0;
  s->nwall = 0;
  s->active[0] = s->active[1] = s->active[2] = 1;
  s->nbf = (int *)malloc(sizeof(int) * 6 * nc);
  s->pat = (int *)malloc(sizeof(int) * 6 * nc);
  s->colour = (int *)malloc(sizeof(int) * nc);
  face_key *keys = (face_key *)malloc(sizeof(face_key) * 6 * (size_t)nc);
  double *area = (double *)malloc(sizeof(double) * 6 * (size_t)nc);
  if (!s->nbf || !s->pat || !s->colour || !keys || !area) { free(keys); free(area); return ORC_E_OOM; }
  int nk = 0;
  for (int c = 0; c < nc; ++c) {
    const int *ids = m->cells + 8 * (size_t)c;
    int dist[8], nd = 0;
    for (int t = 0; t < 8; ++t) {
      int seen = 0;
      for (int u = 0; u < nd; ++u) seen |= dist[u] == ids[t];
      if (!seen) dist[nd++] = ids[t];
    }
    double *xc = s->xc + 3 * c, p[3];
    xc[0] = xc[1] = xc[2] = 0.0;
    for (int u = 0; u < nd; ++u) {
      unode(m, dist[u], p);
      for (int d = 0; d < 3; ++d) xc[d] += p[d] / nd;
    }
    double V = 0.0;
    for (int side = 0; side < 6; ++side) {
      int q[4], fd[4], nf = 0;
      for (int t = 0; t < 4; ++t) q[t] = ids[HEX_SIDE[side][t]];
      for (int t = 0; t < 4; ++t) {
        int seen = 0;
        for (int u = 0; u < nf; ++u) seen |= fd[u] == q[t];
        if (!seen) fd[nf++] = q[t];
      }
      double *S = s->S + 18 * c + 3 * side, *xf = s->xf + 18 * c + 3 * side;
      S[0] = S[1] = S[2] = xf[0] = xf[1] = xf[2] = 0.0;
      if (nf == 4) {
        double pq[4][3];
        for (int t = 0; t < 4; ++t) unode(m, q[t], pq[t]);
        quad((const double(*)[3])pq, S, xf);
      } else if (nf == 3) {
        double a[3], b[3], c3[3], e1[3], e2[3];
        unode(m, fd[0], a); unode(m, fd[1], b); unode(m, fd[2], c3);
        for (int d = 0; d < 3; ++d) { e1[d] = b[d] - a[d]; e2[d] = c3[d] - a[d]; xf[d] = (a[d] + b[d] + c3[d]) / 3.0; }
        S[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
        S[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
        S[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
      } else {
        for (int t = 0; t < 4; ++t) { unode(m, q[t], p); for (int d = 0; d < 3; ++d) xf[d] += p[d] / 4.0; }
      }
      double r[3] = {xf[0] - xc[0], xf[1] - xc[1], xf[2] - xc[2]};
      if (dot3(S, r) < 0) { S[0] = -S[0]; S[1] = -S[1]; S[2] = -S[2]; }
      V += dot3(xf, S) / 3.0;
      area[6 * c + side] = nf >= 3 ? sqrt(dot3(S, S)) : 0.0;
      s->nb[6 * c + side] = -2;
      s->nbf[6 * c + side] = -1;
      s->pat[6 * c + side] = -1;
      s->wid[6 * c + side] = -1;
      if (area[6 * c + side] > 0) {
        /* sorted distinct ids, padded with -1 */
        for (int t = 0; t < 4; ++t) keys[nk].id[t] = t < nf ? fd[t] : -1;
        for (int t = 1; t < nf; ++t)
          for (int u = t; u > 0 && keys[nk].id[u - 1] > keys[nk].id[u]; --u) {
            int x = keys[nk].id[u]; keys[nk].id[u] = keys[nk].id[u - 1]; keys[nk].id[u - 1] = x;
          }
        keys[nk].face = 6 * c + side;
        ++nk;
      }
    }
    if (!(V > 0)) { free(keys); free(area); return ORC_E_INVALID; }
    s->vol[c] = V;
    s->eps2[c] = pow(s->o.venkat_K * cbrt(V), 3.0);
  }
  qsort(keys, nk, sizeof(face_key), key_cmp);
  for (int t = 0; t + 1 < nk; ++t)
    if (memcmp(keys[t].id, keys[t + 1].id, sizeof keys[t].id) == 0) {
      int f = keys[t].face, g = keys[t + 1].face;
      if (m->face_patch[f] >= 0 || m->face_patch[g] >= 0) { free(keys); free(area); return ORC_E_INVALID; }
      s->nb[f] = g / 6; s->nbf[f] = g % 6;
      s->nb[g] = f / 6; s->nbf[g] = f % 6;
      ++t;
    }
  free(keys);
  int one_layer = 0;
  for (int c = 0; c < nc; ++c)
    for (int side = 0; side < 6; ++side) {
      int f = 6 * c + side;
      if (!(area[f] > 0) || s->nb[f] >= 0) continue;
      int p = m->face_patch[f];
      if (p < 0 || p > 5) { free(area); return ORC_E_INVALID; }
      s->pat[f] = p;
      int b = m->bc[p];
      if (b == ORC_BC_WALL) { s->nb[f] = -1; s->wid[f] = s->nwall++; }
      else if (b == ORC_BC_FARFIELD) { s->nb[f] = -4; s->open = 1; }
      else if (b == ORC_BC_AXIS) s->nb[f] = -3;
      else if (b == ORC_BC_PERIODIC) {
        const double *S = s->S + 18 * c + 3 * side;
        if (fabs(S[2]) < (1.0 - 1e-9) * area[f]) { free(area); return ORC_E_INVALID; }
        s->nb[f] = -2;
        one_layer = 1;
      } else { free(area); return ORC_E_INVALID; }
    }
  free(area);
  s->active[2] = !one_layer;
  /* node-sharing neighbours: cells listed per node, then merged per cell */
  {
    int nn = m->nnodes;
    int *cnt = (int *)calloc(nn + 1, sizeof(int));
    s->sten = (int *)malloc(sizeof(int) * STENCIL_MAX * (size_t)nc);
    if (!cnt || !s->sten) { free(cnt); return ORC_E_OOM; }
    for (int c = 0; c < nc; ++c)
      for (int t = 0; t < 8; ++t) {
        int dup = 0;
        for (int u = 0; u < t; ++u) dup |= m->cells[8 * (size_t)c + u] == m->cells[8 * (size_t)c + t];
        if (!dup) cnt[m->cells[8 * (size_t)c + t] + 1]++;
      }
    for (int v = 0; v < nn; ++v) cnt[v + 1] += cnt[v];
    int *lst = (int *)malloc(sizeof(int) * (cnt[nn] + 1)), *pos = (int *)malloc(sizeof(int) * (nn + 1));
    if (!lst || !pos) { free(cnt); free(lst); free(pos); return ORC_E_OOM; }
    memcpy(pos, cnt, sizeof(int) * (nn + 1));
    for (int c = 0; c < nc; ++c)
      for (int t = 0; t < 8; ++t) {
        int dup = 0;
        for (int u = 0; u < t; ++u) dup |= m->cells[8 * (size_t)c + u] == m->cells[8 * (size_t)c + t];
        if (!dup) lst[pos[m->cells[8 * (size_t)c + t]]++] = c;
      }
    int all_hex = 1;
    for (int c = 0; c < nc; ++c) {
      int ndist = 0;
      for (int t = 0; t < 8; ++t) {
        int dup = 0;
        for (int u = 0; u < t; ++u) dup |= m->cells[8 * (size_t)c + u] == m->cells[8 * (size_t)c + t];
        ndist += !dup;
      }
      if (ndist < 8) all_hex = 0;
    }
    s->simplex = !all_hex;
    for (int c = 0; c < nc; ++c) {
      int *st = s->sten + (size_t)STENCIL_MAX * c, k = 0;
      for (int t = 0; t < STENCIL_MAX; ++t) st[t] = -1;
      if (all_hex) {
        for (int side = 0; side < 6; ++side)
          if (s->nb[6 * c + side] >= 0) st[k++] = s->nb[6 * c + side];
        continue;
      }
      for (int t = 0; t < 8; ++t) {
        int v = m->cells[8 * (size_t)c + t];
        for (int e = cnt[v]; e < cnt[v + 1]; ++e) {
          int o = lst[e], seen = o == c;
          for (int u = 0; u < k && !seen; ++u) seen = st[u] == o;
          if (!seen) {
            if (k == STENCIL_MAX) { free(cnt); free(lst); free(pos); return ORC_E_INVALID; }
            st[k++] = o;
          }
        }
      }
      /* ascending order, so the sums do not depend on the node order */
      for (int a = 1; a < k; ++a)
        for (int b = a; b > 0 && st[b - 1] > st[b]; --b) { int x = st[b]; st[b] = st[b - 1]; st[b - 1] = x; }
    }
    free(cnt); free(lst); free(pos);
  }
  s->ncolour = 0;
  for (int c = 0; c < nc; ++c) {
    int k = 0, clash = 1;
    while (clash) {
      clash = 0;
      for (int side = 0; side < 6; ++side) {
        int j = s->nb[6 * c + side];
        if (j >= 0 && j < c && s->colour[j] == k) clash = 1;
      }
      if (clash) ++k;
    }
    s->colour[c] = k;
    if (k + 1 > s->ncolour) s->ncolour = k + 1;
  }
  s->wcell = (int *)malloc(sizeof(int) * (s->nwall + 1));
  s->wside = (int *)malloc(sizeof(int) * (s->nwall + 1));
  s->rho_w = (double *)calloc(s->nwall + 1, sizeof(double));
  if (!s->wcell || !s->wside || !s->rho_w) return ORC_E_OOM;
  for (int c = 0; c < nc; ++c)
    for (int side = 0; side < 6; ++side)
      if (s->wid[6 * c + side] >= 0) { s->wcell[s->wid[6 * c + side]] = c; s->wside[s->wid[6 * c + side]] = side; }
  return ORC_OK;
}

/* ---------------- moments (Eq. getmoment) ---------------- */

/* out: rho, u(3), Tt, Tr, sigma(xx,yy,zz,xy,xz,yz), qt(3), qr(3) */
static void cell_moments(const orc_solver *s, int i, double *out) {
  double rho = 0, mom[3] = {0, 0, 0}, xi[3], w;
  for (int v = 0; v < s->nv; ++v) {
    vel_of(s, v, xi, &w);
    double f = s->f0[(size_t)v * s->nc + i];
    rho += w * f;
    for (int a = 0; a < 3; ++a) mom[a] += w * xi[a] * f;
  }
  double u[3] = {mom[0] / rho, mom[1] / rho, mom[2] / rho};
  double P[3][3] = {{0}}, E = 0, qt[3] = {0, 0, 0}, e1 = 0, qr[3] = {0, 0, 0};
  for (int v = 0; v < s->nv; ++v) {
    vel_of(s, v, xi, &w);
    double f = s->f0[(size_t)v * s->nc + i];
    double c[3] = {xi[0] - u[0], xi[1] - u[1], xi[2] - u[2]}, c2 = dot3(c, c);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) P[a][b] += w * c[a] * c[b] * f;
    E += w * 0.5 * c2 * f;
    for (int a = 0; a < 3; ++a) qt[a] += w * 0.5 * c2 * c[a] * f;
    if (s->nvdf == 2) {
      double f1 = s->f1[(size_t)v * s->nc + i];
      e1 += w * f1;
      for (int a = 0; a < 3; ++a) qr[a] += w * c[a] * f1;
    }
  }
  out[0] = rho;
  out[1] = u[0]; out[2] = u[1]; out[3] = u[2];
  out[4] = E / (0.75 * rho);                                   /* (3/2) rho R Tt = (3/4) rho Tt */
  out[5] = s->nvdf == 2 ? e1 / (s->g.d_r * rho / 4.0) : out[4]; /* (d_r/2) rho R Tr */
  double tr = (P[0][0] + P[1][1] + P[2][2]) / 3.0;
  out[6] = P[0][0] - tr; out[7] = P[1][1] - tr; out[8] = P[2][2] - tr;
  out[9] = P[0][1]; out[10] = P[0][2]; out[11] = P[1][2];
  out[12] = qt[0]; out[13] = qt[1]; out[14] = qt[2];
  out[15] = qr[0]; out[16] = qr[1]; out[17] = qr[2];
}

static int all_moments(orc_solver *s) {
  int bad = 0;
#pragma omp parallel for num_threads(s->o.nthreads > 0 ? s->o.nthreads : 1)
  for (int i = 0; i < s->nc; ++i) {
    cell_moments(s, i, s->Mh + 18 * i);
    double *m = s->Mh + 18 * i;
    if (!(m[0] > 0) || !(m[4] > 0) || !(m[5] > 0) || !isfinite(m[12])) {
#pragma omp atomic write
      bad = 1;
    }
  }
  return bad ? ORC_E_DIVERGED : ORC_OK;
}

/* ---------------- macroscopic synthetic solve (Section 3.3) ---------------- */

/* conservative W: rho, rho u, rho E, rho E_r;  E = |u|^2/2 + 3Tt/4 + d_r Tr/4 */
static void prim_of(const orc_solver *s, const double *W, double *pr) {
  double rho = W[0];
  double u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
  double Er = s->nW == 6 ? W[5] : 0.0;
  double Tt = (W[4] - 0.5 * rho * dot3(u, u) - Er) / (0.75 * rho);
  double Tr = s->nW == 6 ? Er / (s->g.d_r * rho / 4.0) : Tt;
  pr[0] = rho; pr[1] = u[0]; pr[2] = u[1]; pr[3] = u[2]; pr[4] = Tt; pr[5] = Tr;
}

static void cons_of(const orc_solver *s, const double *pr, double *W) {
  double rho = pr[0];
  W[0] = rho;
  W[1] = rho * pr[1]; W[2] = rho * pr[2]; W[3] = rho * pr[3];
  double Er = s->nW == 6 ? s->g.d_r * rho * pr[5] / 4.0 : 0.0;
  W[4] = 0.5 * rho * dot3(pr + 1, pr + 1) + 0.75 * rho * pr[4] + Er;
  if (s->nW == 6) W[5] = Er;
}

/* Convective (Euler) flux of W along unit normal n: (rho u_n, rho u u_n + p_t n, (rho E + p_t) u_n, rho E_r u_n). */
static void euler_flux(const orc_solver *s, const double *W, const double *n, double *F) {
  double pr[6];
  prim_of(s, W, pr);
  double un = dot3(pr + 1, n), p = 0.5 * pr[0] * pr[4];
  F[0] = W[0] * un;
  for (int a = 0; a < 3; ++a) F[1 + a] = W[1 + a] * un + p * n[a];
  F[4] = (W[4] + p) * un;
  if (s->nW == 6) F[5] = W[5] * un;
}

static double sound(double Tt) { return sqrt(5.0 * Tt / 6.0); }  /* sqrt(5 p_t / (3 rho)) */

/* Wall flux (outward, per unit area) of a gas in local equilibrium at the cell state
   pr = (rho, u, Tt, Tr) meeting a diffuse wall (u_w, T_w): the half of the Maxwellian
   moving towards the wall leaves, the wall re-emits rho_w M(u_w, T_w) with zero net mass
   flux.  Half-range normal moments J_k of N(u_n, T/2) satisfy
   J_k = u_n J_{k-1} + (k-1) (T/2) J_{k-2} + (T/2) M_n(0) [k = 1].
   Used for the increment-based "boundary flux modification" of Section 3.3. */
static void wall_eq_flux(const orc_solver *s, int side, const double *pr, const double *n, double *F) {
  double rho = pr[0], T = pr[4], un = dot3(pr + 1, n), Tw = s->wall_T[side];
  const double *uw = s->wall_u[side];
  double sr = un / sqrt(T);
  double M0 = exp(-sr * sr) / sqrt(PI * T);
  double J0 = 0.5 * (1.0 + erf(sr)), J1 = un * J0 + 0.5 * T * M0;
  double J2 = un * J1 + 0.5 * T * J0, J3 = un * J2 + T * J1;
  double K1 = -sqrt(Tw) / (2.0 * SQRT_PI), K2 = Tw / 4.0, K3 = Tw * K1;
  double rw = -rho * J1 / K1;
  double ut[3], uwt[3];
  for (int a = 0; a < 3; ++a) { ut[a] = pr[1 + a] - un * n[a]; uwt[a] = uw[a] - dot3(uw, n) * n[a]; }
  F[0] = rho * J1 + rw * K1;
  for (int a = 0; a < 3; ++a) F[1 + a] = n[a] * (rho * J2 + rw * K2) + rho * J1 * ut[a] + rw * K1 * uwt[a];
  double ein = 0.5 * rho * (J3 + J1 * (dot3(ut, ut) + T)), eout = 0.5 * rw * (K3 + K1 * (dot3(uwt, uwt) + Tw));
  double rin = 0.0, rout = 0.0;
  if (s->nW == 6) { rin = s->g.d_r * pr[5] / 4.0 * rho * J1; rout = s->g.d_r * Tw / 4.0 * rw * K1; }
  F[4] = ein + eout + rin + rout;
  F[5] = rin + rout;
}

/* Polynomials in one variable of degree <= 6 (coefficients of x^0 .. x^6). */
typedef struct { double c[7]; } poly6;

static poly6 poly_of(int n, const double *c) {
  poly6 p;
  for (int k = 0; k < 7; ++k) p.c[k] = k < n ? c[k] : 0.0;
  return p;
}

static poly6 poly_mul(poly6 a, poly6 b) {
  poly6 r = poly_of(0, NULL);
  for (int i = 0; i < 7; ++i)
    for (int j = 0; i + j < 7; ++j) r.c[i + j] += a.c[i] * b.c[j];
  return r;
}

static poly6 poly_add(poly6 a, double s, poly6 b) { /* a + s b */
  for (int k = 0; k < 7; ++k) a.c[k] += s * b.c[k];
  return a;
}

static double poly_dot(poly6 a, const double *H) {
  double r = 0.0;
  for (int k = 0; k < 7; ++k) r += a.c[k] * H[k];
  return r;
}

/* Wall flux of the Grad-13 reconstruction of Eq. G13_VDF.  In the units of this code (velocity
   in sqrt(2 R T0), p = rho T / 2, sigma = int c c f - p I, q_t = int c^2 c f / 2, q_r = int c f1)
   the 13-moment VDF that reproduces rho, u, T_t, sigma and q_t is
     f0 = M [1 + A:cc + (B.c)(c^2/T - 5/2)],  A = 2 sigma / (rho T^2),  B = 8 q_t / (5 rho T^2),
   M = rho (pi T)^(-3/2) exp(-c^2/T), and the rotational VDF with (d_r/4) rho T_r and q_r is
     f1 = (d_r T_r / 4) f0 + 2 M (q_r.c) / (rho T).
   The half moving into the wall (xi.n > 0) leaves with this VDF; the wall re-emits
   rho_w M(u_w, T_w) with zero net mass flux.  With c = x n + c_t, the tangential Gaussian
   moments are taken in closed form, which leaves per flux a polynomial in x against
   H_k = int_{x > -u_n} x^k g(x) dx, g the one-dimensional Maxwellian of variance T/2:
     H_0 = erfc(-u_n / sqrt T) / 2,  H_k = (k-1) (T/2) H_{k-2} + (T/2) (-u_n)^(k-1) g(-u_n).
   The tangential averages of the bracket Q = f0 / M:
     <Q> = 1 - A_nn T/2 + A_nn x^2 + B_n x (x^2/T - 3/2),
     <c_t Q> = T x A_nt + B_t (x^2/2 - T/4),
     <|c_t|^2 Q> = T - A_nn T^2 + A_nn T x^2 + B_n x (x^2 - T/2),
   A_nn = n.A.n, A_nt and B_t the tangential parts of A n and B. */
static void wall_g13_flux(const orc_solver *s, int patch, const double *pr, const double *m18, const double *n,
                          double *F) {
  const double rho = pr[0], T = pr[4], Tr = pr[5], Tw = s->wall_T[patch];
  const double *u = pr + 1, *uw = s->wall_u[patch];
  const double sig[3][3] = {{m18[6], m18[9], m18[10]}, {m18[9], m18[7], m18[11]}, {m18[10], m18[11], m18[8]}};
  const double *qt = m18 + 12, *qr = m18 + 15;
  double un = dot3(u, n), sn[3];
  for (int a = 0; a < 3; ++a) sn[a] = sig[a][0] * n[0] + sig[a][1] * n[1] + sig[a][2] * n[2];
  const double kA = 2.0 / (rho * T * T), kB = 8.0 / (5.0 * rho * T * T);
  const double snn = dot3(sn, n), qn = dot3(qt, n);
  const double Ann = kA * snn, Bn = kB * qn;
  double Ant[3], Bt[3], ut[3];
  for (int a = 0; a < 3; ++a) {
    Ant[a] = kA * (sn[a] - snn * n[a]);
    Bt[a] = kB * (qt[a] - qn * n[a]);
    ut[a] = u[a] - un * n[a];
  }
  const double cQ0[4] = {1.0 - 0.5 * Ann * T, -1.5 * Bn, Ann, Bn / T};
  const double cQ2[4] = {T - Ann * T * T, -0.5 * Bn * T, Ann * T, Bn};
  const double cL[2] = {un, 1.0};
  poly6 Q0 = poly_of(4, cQ0), Q2 = poly_of(4, cQ2), L = poly_of(2, cL), Qt[3];
  for (int a = 0; a < 3; ++a) {
    const double c[3] = {-0.25 * Bt[a] * T, T * Ant[a], 0.5 * Bt[a]};
    Qt[a] = poly_of(3, c);
  }
  const poly6 mass = poly_mul(L, Q0), normal = poly_mul(L, mass);
  /* the energy bracket (|u|^2/2 + u_n x + x^2/2) <Q> + u_t.<c_t Q> + <|c_t|^2 Q>/2 */
  const double ce[3] = {0.5 * dot3(u, u), un, 0.5};
  poly6 eb = poly_add(poly_mul(poly_of(3, ce), Q0), 0.5, Q2);
  for (int a = 0; a < 3; ++a) eb = poly_add(eb, ut[a], Qt[a]);
  const poly6 energy = poly_mul(L, eb);
  poly6 rot = poly_of(0, NULL);
  if (s->nW == 6) {
    const double cx[2] = {0.0, 2.0 * dot3(qr, n) / (rho * T)};
    rot = poly_add(poly_mul(poly_of(2, cx), L), s->g.d_r * Tr / 4.0, mass);
  }
  /* half-range moments of x */
  const double sr = un / sqrt(T), g0 = exp(-sr * sr) / sqrt(PI * T);
  double H[7];
  H[0] = 0.5 * erfc(-sr);
  H[1] = 0.5 * T * g0;
  for (int k = 2; k < 7; ++k) H[k] = (k - 1) * 0.5 * T * H[k - 2] + 0.5 * T * pow(-un, k - 1) * g0;
  const double min = rho * poly_dot(mass, H), rin = rho * poly_dot(rot, H);
  /* the wall's half (as for the Maxwellian flux) */
  const double K1 = -sqrt(Tw) / (2.0 * SQRT_PI), K2 = Tw / 4.0, K3 = Tw * K1;
  const double rw = -min / K1;
  double uwt[3];
  for (int a = 0; a < 3; ++a) uwt[a] = uw[a] - dot3(uw, n) * n[a];
  F[0] = min + rw * K1;
  for (int a = 0; a < 3; ++a)
    F[1 + a] = rho * (n[a] * poly_dot(normal, H) + ut[a] * poly_dot(mass, H) + poly_dot(poly_mul(L, Qt[a]), H)) +
               n[a] * rw * K2 + rw * K1 * uwt[a];
  const double rout = s->nW == 6 ? s->g.d_r * Tw / 4.0 * rw * K1 : 0.0;
  F[4] = rho * poly_dot(energy, H) + rin + 0.5 * rw * (K3 + K1 * (dot3(uwt, uwt) + Tw)) + rout;
  F[5] = rin + rout;
}

/* the wall flux model of the synthetic solve (orc_opts.wall_flux) */
static void wall_model_flux(const orc_solver *s, int patch, const double *pr, const double *m18, const double *n,
                            double *F) {
  if (s->o.wall_flux == ORC_WALL_G13)
    wall_g13_flux(s, patch, pr, m18, n, F);
  else
    wall_eq_flux(s, patch, pr, n, F);
}

void orc_wall_flux(const orc_solver *s, int mode, int patch, const double *pr, const double *m18, const double *n,
                   double *F) {
  for (int k = 0; k < 6; ++k) F[k] = 0.0;
  if (mode == ORC_WALL_G13)
    wall_g13_flux(s, patch, pr, m18, n, F);
  else
    wall_eq_flux(s, patch, pr, n, F);
}

typedef struct {
  double *pr, *gW, *phW, *gP, *R, *dt, *D, *dW, *mu;
} macro_work;

/* NSF stress and heat fluxes at the face between cells i and j (Eq. NSF_constitutive):
   face gradient = mean of the two cells' LSQ gradients, mu at the face = mean of the
   cells' mu.  Between two different cells, with the weight alpha = s->jump > 0, each field
   phi in (u_x, u_y, u_z, T_t, T_r) replaces the fraction alpha of the mean gradient's change
   along the centre line d = x_j - x_i by the cells' difference:
     grad_f = mean + alpha (phi_j - phi_i - mean . d) d / |d|^2
   (alpha = 1 makes grad_f . d = phi_j - phi_i).  out: sigma(xx,yy,zz,xy,xz,yz), qt(3), qr(3). */
static void face_nsf(const orc_solver *s, const macro_work *m, int i, int j, double *out) {
  double G[3][3], gT[3], gTr[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) G[a][b] = 0.5 * (m->gP[15 * i + 3 * a + b] + m->gP[15 * j + 3 * a + b]);
    gT[a] = 0.5 * (m->gP[15 * i + 9 + a] + m->gP[15 * j + 9 + a]);
    gTr[a] = 0.5 * (m->gP[15 * i + 12 + a] + m->gP[15 * j + 12 + a]);
  }
  if (s->jump > 0.0 && j != i) {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = s->xc[3 * j + a] - s->xc[3 * i + a];
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double *grad[5] = {G[0], G[1], G[2], gT, gTr};
    for (int k = 0; k < 5; ++k) {
      double along = grad[k][0] * d[0] + grad[k][1] * d[1] + grad[k][2] * d[2];
      double jump = m->pr[6 * j + 1 + k] - m->pr[6 * i + 1 + k] - along;
      for (int a = 0; a < 3; ++a) grad[k][a] += s->jump * jump * d[a] / dd;
    }
  }
  double muf = 0.5 * (m->mu[i] + m->mu[j]), kt, kr;
  orc_conductivity(&s->g, muf, &kt, &kr);
  double div = G[0][0] + G[1][1] + G[2][2];
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int t = 0; t < 6; ++t) {
    int a = ia[t], b = ib[t];
    out[t] = -muf * (G[a][b] + G[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
  }
  for (int a = 0; a < 3; ++a) {
    out[6 + a] = -kt * gT[a];
    out[9 + a] = s->nW == 6 ? -kr * gTr[a] : 0.0;
  }
}

static int macro_solve(orc_solver *s, double *W, const double *fkin, int euler, int max_steps, double tol,
                       int *used) {
  int nc = s->nc, nW = s->nW;
  macro_work m;
  m.pr = (double *)malloc(sizeof(double) * 6 * nc);
  m.gW = (double *)malloc(sizeof(double) * 18 * nc);
  m.phW = (double *)malloc(sizeof(double) * 6 * nc);
  m.gP = (double *)malloc(sizeof(double) * 15 * nc);
  m.R = (double *)malloc(sizeof(double) * 6 * nc);
  m.dt = (double *)malloc(sizeof(double) * nc);
  m.D = (double *)malloc(sizeof(double) * 6 * nc);
  m.dW = (double *)malloc(sizeof(double) * 6 * nc);
  m.mu = (double *)malloc(sizeof(double) * nc);
  double *feq0 = (double *)malloc(sizeof(double) * 6 * (size_t)(s->nwall + 1));
  double *corr = (double *)calloc(36 * (size_t)nc, sizeof(double));
  int rc = ORC_OK;
  *used = 0;
  if (!m.pr || !m.gW || !m.phW || !m.gP || !m.R || !m.dt || !m.D || !m.dW || !m.mu || !feq0 || !corr) { rc = ORC_E_OOM; goto done; }
  for (int wf = 0; wf < s->nwall; ++wf) {
    int i = s->wcell[wf], side = s->wside[wf];
    const double *S = s->S + 18 * i + 3 * side;
    double A = sqrt(dot3(S, S)), n[3] = {S[0] / A, S[1] / A, S[2] / A}, pr[6];
    prim_of(s, W + 6 * i, pr);
    wall_model_flux(s, patch_of(s, i, side), pr, s->Mh + 18 * i, n, feq0 + 6 * wf);
  }
  for (int step = 0; step < max_steps; ++step) {
    for (int i = 0; i < nc; ++i) {
      prim_of(s, W + 6 * i, m.pr + 6 * i);
      if (!(m.pr[6 * i] > 0) || !(m.pr[6 * i + 4] > 0) || !(m.pr[6 * i + 5] > 0)) { rc = ORC_E_DIVERGED; goto done; }
      m.mu[i] = visc(&s->g, m.pr[6 * i + 4]);
    }
    /* gradients (LSQ) and limiters of conservative W; gradients of u, Tt, Tr */
    for (int i = 0; i < nc; ++i) {
      for (int k = 0; k < nW; ++k) {
        lsq_grad(s, i, W + k, 6, m.gW + 18 * i + 3 * k);
        m.phW[6 * i + k] = venkat_cell(s, i, W + k, 6, m.gW + 18 * i + 3 * k);
      }
      for (int k = 0; k < 5; ++k) lsq_grad(s, i, m.pr + 1 + k, 6, m.gP + 15 * i + 3 * k);
    }
    /* residual R_i = -(1/V_i) sum_faces F S + Q_i */
    for (int i = 0; i < 6 * nc; ++i) m.R[i] = 0.0;
    for (int i = 0; i < nc; ++i) {
      for (int side = 0; side < 6; ++side) {
        int j = s->nb[6 * i + side];
        const double *S = s->S + 18 * i + 3 * side, *xf = s->xf + 18 * i + 3 * side;
        double A = sqrt(dot3(S, S)), n[3] = {S[0] / A, S[1] / A, S[2] / A};
        if (j == -1) {
          int wf = s->wid[6 * i + side];
          if (euler) {
            double p = 0.5 * m.pr[6 * i] * m.pr[6 * i + 4];
            for (int a = 0; a < 3; ++a) m.R[6 * i + 1 + a] -= p * n[a] * A;
          } else {
            /* frozen kinetic wall flux plus the increment of the model wall flux */
            double feq[6];
            wall_model_flux(s, patch_of(s, i, side), m.pr + 6 * i, s->Mh + 18 * i, n, feq);
            for (int k = 0; k < nW; ++k) m.R[6 * i + k] -= fkin[36 * i + 6 * side + k] + (feq[k] - feq0[6 * wf + k]) * A;
          }
          continue;
        }
        if (j == -2 || j == -3) continue;
        if (j == -4) {
          /* far field: Rusanov flux between the cell's face state and the free stream (a
             dissipative, well-posed weak imposition on inflow and outflow faces alike; at the
             fixed point the high-order correction makes the face flux the kinetic one anyway),
             the NSF part from the cell's own gradients, the correction as on interior faces */
          double WL[6], WR[6], FL[6], FR[6], F[6], pL[6], pR[6];
          const double *xci = s->xc + 3 * i;
          double ri[3] = {xf[0] - xci[0], xf[1] - xci[1], xf[2] - xci[2]};
          for (int k = 0; k < nW; ++k) WL[k] = W[6 * i + k] + m.phW[6 * i + k] * dot3(m.gW + 18 * i + 3 * k, ri);
          prim_of(s, WL, pL);
          if (!(pL[0] > 0) || !(pL[4] > 0) || !(pL[5] > 0)) { memcpy(WL, W + 6 * i, sizeof WL); prim_of(s, WL, pL); }
          const int pp = patch_of(s, i, side);
          double pinf[6] = {1.0, s->wall_u[pp][0], s->wall_u[pp][1], s->wall_u[pp][2], s->wall_T[pp], s->wall_T[pp]};
          cons_of(s, pinf, WR);
          prim_of(s, WR, pR);
          euler_flux(s, WL, n, FL);
          euler_flux(s, WR, n, FR);
          double lL = fabs(dot3(pL + 1, n)) + sound(pL[4]), lR = fabs(dot3(pR + 1, n)) + sound(pR[4]);
          double lam = lL > lR ? lL : lR;
          for (int k = 0; k < nW; ++k) F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (WR[k] - WL[k]);
          if (!euler) {
            double nsf[12], sn[3];
            face_nsf(s, &m, i, i, nsf);
            const int map[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
            for (int a = 0; a < 3; ++a) sn[a] = nsf[map[a][0]] * n[0] + nsf[map[a][1]] * n[1] + nsf[map[a][2]] * n[2];
            for (int a = 0; a < 3; ++a) F[1 + a] += sn[a];
            F[4] += dot3(sn, m.pr + 6 * i + 1) + dot3(nsf + 6, n) + (nW == 6 ? dot3(nsf + 9, n) : 0.0);
            if (nW == 6) F[5] += dot3(nsf + 9, n);
          }
          double *cr = corr + 36 * i + 6 * side;
          if (step == 0)
            for (int k = 0; k < nW; ++k) cr[k] = euler ? 0.0 : fkin[36 * i + 6 * side + k] - F[k] * A;
          for (int k = 0; k < nW; ++k) m.R[6 * i + k] -= F[k] * A + cr[k];
          continue;
        }
        if (j < i) continue;  /* each interior face once, from its lower-index cell */
        double WL[6], WR[6], FL[6], FR[6], F[6];
        const double *xci = s->xc + 3 * i, *xcj = s->xc + 3 * j;
        double ri[3] = {xf[0] - xci[0], xf[1] - xci[1], xf[2] - xci[2]};
        double rj[3] = {xf[0] - xcj[0], xf[1] - xcj[1], xf[2] - xcj[2]};
        for (int k = 0; k < nW; ++k) {
          WL[k] = W[6 * i + k] + m.phW[6 * i + k] * dot3(m.gW + 18 * i + 3 * k, ri);
          WR[k] = W[6 * j + k] + m.phW[6 * j + k] * dot3(m.gW + 18 * j + 3 * k, rj);
        }
        double pL[6], pR[6];
        prim_of(s, WL, pL);
        prim_of(s, WR, pR);
        if (!(pL[0] > 0) || !(pL[4] > 0) || !(pL[5] > 0)) { memcpy(WL, W + 6 * i, sizeof WL); prim_of(s, WL, pL); }
        if (!(pR[0] > 0) || !(pR[4] > 0) || !(pR[5] > 0)) { memcpy(WR, W + 6 * j, sizeof WR); prim_of(s, WR, pR); }
        euler_flux(s, WL, n, FL);
        euler_flux(s, WR, n, FR);
        double lL = fabs(dot3(pL + 1, n)) + sound(pL[4]), lR = fabs(dot3(pR + 1, n)) + sound(pR[4]);
        double lam = lL > lR ? lL : lR;
        for (int k = 0; k < nW; ++k) F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (WR[k] - WL[k]);
        if (!euler) {
          double nsf[12], uf[3];
          face_nsf(s, &m, i, j, nsf);
          for (int a = 0; a < 3; ++a) uf[a] = 0.5 * (m.pr[6 * i + 1 + a] + m.pr[6 * j + 1 + a]);
          const int map[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
          double sn[3];
          for (int a = 0; a < 3; ++a) sn[a] = nsf[map[a][0]] * n[0] + nsf[map[a][1]] * n[1] + nsf[map[a][2]] * n[2];
          for (int a = 0; a < 3; ++a) F[1 + a] += sn[a];
          F[4] += dot3(sn, uf) + dot3(nsf + 6, n) + (nW == 6 ? dot3(nsf + 9, n) : 0.0);
          if (nW == 6) F[5] += dot3(nsf + 9, n);
        }
        /* Eq. full_constitutive evaluated as face fluxes: the high-order part is the kinetic
           face flux of the last kinetic step minus this scheme's face flux at W^{n+1/2},
           frozen over the inner iterations (zero in the Euler preconditioning). */
        double *cr = corr + 36 * i + 6 * side;
        if (step == 0)
          for (int k = 0; k < nW; ++k) cr[k] = euler ? 0.0 : fkin[36 * i + 6 * side + k] - F[k] * A;
        for (int k = 0; k < nW; ++k) {
          m.R[6 * i + k] -= F[k] * A + cr[k];
          m.R[6 * j + k] += F[k] * A + cr[k];
        }
      }
    }
    for (int i = 0; i < nc; ++i) {
      double *pr = m.pr + 6 * i, V = s->vol[i];
      for (int k = 0; k < nW; ++k) m.R[6 * i + k] /= V;
      double srcdiag = 0.0;
      if (nW == 6) {
        /* Q = (d_r rho R/2)(T - Tr)/(Z_r tau), T = (3Tt + d_r Tr)/(3 + d_r) */
        double tau = orc_tau(&s->g, pr[0], pr[4]);
        double T = (3.0 * pr[4] + s->g.d_r * pr[5]) / (3.0 + s->g.d_r);
        m.R[6 * i + 5] += s->g.d_r * pr[0] * (T - pr[5]) / (4.0 * s->g.Z_r * tau);
        srcdiag = 1.0 / (s->g.Z_r * tau);  /* -dQ/d(rho E_r) with tau frozen */
      }
      double lsum = 0.0, gsum = 0.0;
      for (int side = 0; side < 6; ++side) {
        int j = s->nb[6 * i + side];
        if (j == -2 || j == -3) continue;
        const double *S = s->S + 18 * i + 3 * side;
        double A = sqrt(dot3(S, S)), n[3] = {S[0] / A, S[1] / A, S[2] / A};
        double li = fabs(dot3(pr + 1, n)) + sound(pr[4]);
        lsum += li * A;
        double gam;
        if (j >= 0) {
          double lj = fabs(dot3(m.pr + 6 * j + 1, n)) + sound(m.pr[6 * j + 4]);
          gam = li > lj ? li : lj;
          if (!euler) {
            double d[3] = {s->xc[3 * j] - s->xc[3 * i], s->xc[3 * j + 1] - s->xc[3 * i + 1], s->xc[3 * j + 2] - s->xc[3 * i + 2]};
            double ni = m.mu[i] / pr[0], nj = m.mu[j] / m.pr[6 * j];
            gam += 2.0 * (ni > nj ? ni : nj) / fabs(dot3(n, d));
          }
        } else {
          const double *xf = s->xf + 18 * i + 3 * side;
          double d[3] = {xf[0] - s->xc[3 * i], xf[1] - s->xc[3 * i + 1], xf[2] - s->xc[3 * i + 2]};
          gam = li;
          if (!euler) gam += 2.0 * (m.mu[i] / pr[0]) / fabs(dot3(n, d));
        }
        gsum += gam * A;
      }
      m.dt[i] = s->o.macro_cfl * V / lsum;
      for (int k = 0; k < nW; ++k) m.D[6 * i + k] = 1.0 / m.dt[i] + gsum / (2.0 * V) + (k == 5 ? srcdiag : 0.0);
    }
    /* matrix-free LU-SGS, colour ordered: red-black cells, macro_sweeps passes (Eq. res_macro) */
    for (int i = 0; i < 6 * nc; ++i) m.dW[i] = 0.0;
    for (int sw = 0; sw < s->o.macro_sweeps; ++sw)
      for (int col = 0; col < (s->colour ? s->ncolour : 2); ++col)
        for (int i = 0; i < nc; ++i) {
          int ii = i % s->ni, jj = (i / s->ni) % s->nj, kk = i / (s->ni * s->nj);
          if ((s->colour ? s->colour[i] : (ii + jj + kk) & 1) != col) continue;
          double acc[6];
          for (int k = 0; k < nW; ++k) acc[k] = m.R[6 * i + k];
          double V = s->vol[i];
          for (int side = 0; side < 6; ++side) {
            int j = s->nb[6 * i + side];
            if (j < 0) continue;
            const double *S = s->S + 18 * i + 3 * side;
            double A = sqrt(dot3(S, S)), n[3] = {S[0] / A, S[1] / A, S[2] / A};
            double li = fabs(dot3(m.pr + 6 * i + 1, n)) + sound(m.pr[6 * i + 4]);
            double lj = fabs(dot3(m.pr + 6 * j + 1, n)) + sound(m.pr[6 * j + 4]);
            double gam = li > lj ? li : lj;
            if (!euler) {
              double d[3] = {s->xc[3 * j] - s->xc[3 * i], s->xc[3 * j + 1] - s->xc[3 * i + 1], s->xc[3 * j + 2] - s->xc[3 * i + 2]};
              double ni = m.mu[i] / m.pr[6 * i], nj = m.mu[j] / m.pr[6 * j];
              gam += 2.0 * (ni > nj ? ni : nj) / fabs(dot3(n, d));
            }
            double Wn[6], F1[6], F0[6];
            for (int k = 0; k < nW; ++k) Wn[k] = W[6 * j + k] + m.dW[6 * j + k];
            euler_flux(s, Wn, n, F1);
            euler_flux(s, W + 6 * j, n, F0);
            for (int k = 0; k < nW; ++k) acc[k] -= ((F1[k] - F0[k]) - gam * m.dW[6 * j + k]) * A / (2.0 * V);
          }
          for (int k = 0; k < nW; ++k) m.dW[6 * i + k] = acc[k] / m.D[6 * i + k];
        }
    double num[6] = {0}, den[6] = {0};
    for (int i = 0; i < nc; ++i)
      for (int k = 0; k < nW; ++k) {
        W[6 * i + k] += m.dW[6 * i + k];
        num[k] += m.dW[6 * i + k] * m.dW[6 * i + k] * s->vol[i];
        den[k] += W[6 * i + k] * W[6 * i + k] * s->vol[i];
      }
    /* the relative increment of every field that is not identically zero: as for eps, a field
       whose volume-weighted RMS is below 1e-12 (the z momentum of a 2D flow, rounding noise)
       has no relative increment to test */
    double vsum = 0.0, delta = 0.0;
    for (int i = 0; i < nc; ++i) vsum += s->vol[i];
    for (int k = 0; k < nW; ++k)
      if (den[k] > 1e-24 * vsum) {
        double e = sqrt(num[k] / den[k]);
        if (e > delta) delta = e;
      }
    for (int i = 0; i < nc; ++i)
      for (int k = 0; k < nW; ++k)
        if (!isfinite(W[6 * i + k])) { rc = ORC_E_DIVERGED; goto done; }
    *used = step + 1;
    if (delta < tol) break;
  }
done:
  free(m.pr); free(m.gW); free(m.phW); free(m.gP); free(m.R); free(m.dt); free(m.D); free(m.dW); free(m.mu);
  free(feq0);
  free(corr);
  return rc;
}

/* HoT of Eq. full_constitutive: kinetic stress/heat flux of f^{n+1/2} minus their NSF values at W^{n+1/2}. */
static void compute_hot(orc_solver *s) {
  int nc = s->nc;
  for (int i = 0; i < nc; ++i) {
    double G[3][3], gT[3], gTr[3];
    for (int a = 0; a < 3; ++a) lsq_grad(s, i, s->Mh + 1 + a, 18, G[a]);
    lsq_grad(s, i, s->Mh + 4, 18, gT);
    lsq_grad(s, i, s->Mh + 5, 18, gTr);
    const double *m = s->Mh + 18 * i;
    double mu = visc(&s->g, m[4]), kt, kr;
    orc_conductivity(&s->g, mu, &kt, &kr);
    double div = G[0][0] + G[1][1] + G[2][2];
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    double *h = s->hot + 12 * i, *kk = s->kin + 12 * i;
    for (int t = 0; t < 6; ++t) kk[t] = m[6 + t];
    for (int t = 0; t < 3; ++t) { kk[6 + t] = m[12 + t]; kk[9 + t] = s->nvdf == 2 ? m[15 + t] : 0.0; }
    for (int t = 0; t < 6; ++t) {
      int a = ia[t], b = ib[t];
      double nsf = -mu * (G[a][b] + G[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
      h[t] = m[6 + t] - nsf;
    }
    for (int a = 0; a < 3; ++a) {
      h[6 + a] = m[12 + a] - (-kt * gT[a]);
      h[9 + a] = s->nvdf == 2 ? m[15 + a] - (-kr * gTr[a]) : 0.0;
    }
  }
}

/* ---------------- outer loop (Algorithm 1) ---------------- */

/* Eq. convergence_critertion over rho, u (as a vector) and Tt; fields with a zero
   denominator are skipped. */
static double eps_of(const orc_solver *s, const double *Wn, const double *Wo) {
  double num[3] = {0}, den[3] = {0};
  for (int i = 0; i < s->nc; ++i) {
    double V = s->vol[i];
    const double *a = Wn + 6 * i, *b = Wo + 6 * i;
    num[0] += (a[0] - b[0]) * (a[0] - b[0]) * V;
    den[0] += b[0] * b[0] * V;
    for (int d = 1; d <= 3; ++d) {
      num[1] += (a[d] - b[d]) * (a[d] - b[d]) * V;
      den[1] += b[d] * b[d] * V;
    }
    num[2] += (a[4] - b[4]) * (a[4] - b[4]) * V;
    den[2] += b[4] * b[4] * V;
  }
  /* a field whose volume-weighted RMS is below 1e-12 counts as identically zero (rounding noise) */
  double vsum = 0.0;
  for (int i = 0; i < s->nc; ++i) vsum += s->vol[i];
  double e = 0.0;
  for (int k = 0; k < 3; ++k)
    if (den[k] > 1e-24 * vsum) {
      double r = sqrt(num[k] / den[k]);
      if (r > e) e = r;
    }
  return e;
}

static void state_from_moments(orc_solver *s) {
  for (int i = 0; i < s->nc; ++i) {
    const double *m = s->Mh + 18 * i;
    double *st = s->st + 12 * i;
    for (int t = 0; t < 6; ++t) st[t] = m[t];
    for (int t = 0; t < 3; ++t) { st[6 + t] = m[12 + t]; st[9 + t] = m[15 + t]; }
  }
}

static double total_mass(const orc_solver *s) {
  double m = 0.0;
  for (int i = 0; i < s->nc; ++i) m += s->Mh[18 * i] * s->vol[i];
  return m;
}

/* Closed domain (walls and periodic sides only): the re-emitted wall density is lagged,
   so the wall only balances the mass flux once f stops changing; the step therefore
   rescales f^{n+1/2} to the domain's total mass (a factor that tends to 1). */
static int conserve_mass(orc_solver *s) {
  if (s->open) {  /* mass leaves and enters through the far field */
    s->mass_scale = 1.0;
    return ORC_OK;
  }
  double fac = s->mass_ref / total_mass(s);
  s->mass_scale = fac;
  size_t n = (size_t)s->nc * s->nv;
  for (size_t t = 0; t < n; ++t) s->f0[t] *= fac;
  if (s->nvdf == 2)
    for (size_t t = 0; t < n; ++t) s->f1[t] *= fac;
  return all_moments(s);
}

static int run_step(orc_solver *s, int mode) {
  int nc = s->nc, rc;
  orc_wall_prepass(s);
  rc = orc_kinetic_velocities(s, 0, s->nv);
  if (rc) return rc;
  rc = all_moments(s);
  if (rc) return rc;
  rc = conserve_mass(s);
  if (rc) return rc;
  double *Wold = (double *)malloc(sizeof(double) * 6 * nc), *Wnew = (double *)malloc(sizeof(double) * 6 * nc);
  if (!Wold || !Wnew) { free(Wold); free(Wnew); return ORC_E_OOM; }
  for (int i = 0; i < nc; ++i)
    for (int t = 0; t < 6; ++t) Wold[6 * i + t] = s->st[12 * i + t];
  if (mode == ORC_GSIS) {
    compute_hot(s);
    double *Wc = (double *)calloc(6 * (size_t)nc, sizeof(double));
    if (!Wc) { free(Wold); free(Wnew); return ORC_E_OOM; }
    for (int i = 0; i < nc; ++i) cons_of(s, s->Mh + 18 * i, Wc + 6 * i);
    rc = macro_solve(s, Wc, s->fkin, 0, s->o.macro_steps, s->o.macro_tol, &s->macro_iters);
    if (rc) { free(Wc); free(Wold); free(Wnew); return rc; }
    /* Closed domain (no far field): the synthetic solve fixes the density only up to a constant and its
       local-time-step iteration does not conserve mass, so its density is rescaled to the
       domain's total mass (velocity and temperatures unchanged). */
    double mk = s->mass_ref, mm = 0.0;
    for (int i = 0; i < nc; ++i) prim_of(s, Wc + 6 * i, Wnew + 6 * i);
    /* orc_opts.relax < 1: the update is W^{n+1/2} + relax (W^{n+1} - W^{n+1/2}), in primitives */
    if (s->o.relax > 0.0 && s->o.relax < 1.0)
      for (int i = 0; i < nc; ++i)
        for (int t = 0; t < 6; ++t) Wnew[6 * i + t] = s->Mh[18 * i + t] + s->o.relax * (Wnew[6 * i + t] - s->Mh[18 * i + t]);
    for (int i = 0; i < nc; ++i) mm += Wnew[6 * i] * s->vol[i];
    if (!s->open)
      for (int i = 0; i < nc; ++i) Wnew[6 * i] *= mk / mm;
    free(Wc);
    /* Eq. updatef: keep the non-equilibrium part, replace the equilibrium */
#pragma omp parallel for num_threads(s->o.nthreads > 0 ? s->o.nthreads : 1)
    for (int i = 0; i < nc; ++i) {
      const double *a = Wnew + 6 * i, *b = s->Mh + 18 * i;
      double xi[3], w;
      for (int v = 0; v < s->nv; ++v) {
        vel_of(s, v, xi, &w);
        double Ma = maxwellian(a[0], a + 1, a[4], xi), Mb = maxwellian(b[0], b + 1, b[4], xi);
        s->f0[(size_t)v * nc + i] += Ma - Mb;
        if (s->nvdf == 2) s->f1[(size_t)v * nc + i] += s->g.d_r / 4.0 * (a[5] * Ma - b[5] * Mb);
      }
    }
  } else {
    s->macro_iters = 0;
    for (int i = 0; i < nc; ++i)
      for (int t = 0; t < 6; ++t) Wnew[6 * i + t] = s->Mh[18 * i + t];
  }
  s->eps = eps_of(s, Wnew, Wold);
  state_from_moments(s);
  for (int i = 0; i < nc; ++i)
    for (int t = 0; t < 6; ++t) s->st[12 * i + t] = Wnew[6 * i + t];
  free(Wold);
  free(Wnew);
  return ORC_OK;
}

int orc_step(orc_solver *s) { return run_step(s, s->o.mode); }

/* 1/dt of the kinetic delta form for the following steps (a pseudo-time schedule) */
void orc_set_kin_inv_dt(orc_solver *s, double inv_dt) { s->o.kin_inv_dt = inv_dt; }

/* run the next steps in another mode (ORC_GSIS or ORC_DVM) */
void orc_set_mode(orc_solver *s, int mode) { s->o.mode = mode; }

int orc_presteps(orc_solver *s, int n) {
  for (int t = 0; t < n; ++t) {
    int rc = run_step(s, ORC_DVM);
    if (rc) return rc;
  }
  return ORC_OK;
}

int orc_macro_from_current(orc_solver *s) {
  int rc = all_moments(s);
  if (rc) return rc;
  compute_hot(s);
  double *Wc = (double *)calloc(6 * (size_t)s->nc, sizeof(double));
  if (!Wc) return ORC_E_OOM;
  for (int i = 0; i < s->nc; ++i) cons_of(s, s->Mh + 18 * i, Wc + 6 * i);
  rc = macro_solve(s, Wc, s->fkin, 0, s->o.macro_steps, s->o.macro_tol, &s->macro_iters);
  free(Wc);
  return rc;
}

/* ---------------- lifecycle ---------------- */

static double *dup(const double *a, int n) {
  double *b = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  if (b) memcpy(b, a, sizeof(double) * n);
  return b;
}

void orc_destroy(orc_solver *s) {
  if (!s) return;
  free(s->vx); free(s->vy); free(s->vz); free(s->wx); free(s->wy); free(s->wz); free(s->pts);
  free(s->vol); free(s->xc); free(s->S); free(s->xf); free(s->eps2); free(s->nb); free(s->wid);
  free(s->wcell); free(s->wside); free(s->rho_w);
  free(s->f0); free(s->f1); free(s->st); free(s->Mh); free(s->hot); free(s->kin); free(s->fkin); free(s->corder);
  free(s->nbf); free(s->pat); free(s->colour); free(s->sten);
  free(s);
}

/* f = Maxwellian of W (rho, u, T_t, T_r per cell); f1 = (d_r T_r / 4) M */
static void set_maxwellian(orc_solver *s, const double *W) {
  int nc = s->nc;
  for (int i = 0; i < nc; ++i) {
    const double *w0 = W + 6 * i;
    double xi[3], w;
    for (int v = 0; v < s->nv; ++v) {
      vel_of(s, v, xi, &w);
      double M = maxwellian(w0[0], w0 + 1, w0[4], xi);
      s->f0[(size_t)v * nc + i] = M;
      if (s->nvdf == 2) s->f1[(size_t)v * nc + i] = s->g.d_r * w0[5] / 4.0 * M;
    }
  }
}

static int init_state_from_f(orc_solver *s) {
  int rc = all_moments(s);
  if (rc) return rc;
  state_from_moments(s);
  s->mass_ref = total_mass(s);
  s->mass_scale = 1.0;
  return ORC_OK;
}

/* The order in which each velocity octant (signs d of its velocities) sweeps the cells
   (Section 3.2's sweeps in upwind order).  A cell's rank key is the mean over its nodes of
   ((d_x x) + (d_y y)) + (d_z z): its 8 corners on a structured block, its distinct nodes on an
   unstructured mesh, summed in that order; ties go by index.  A cell's colour is one more than
   the largest colour of its face neighbours ranked before it (0 without one), and the octant
   sweeps colour by colour, in index order within a colour.  On a rectilinear block this is the
   hyperplane order i' + j' + k' of the octant; on a curved or unstructured mesh it follows the
   flow, where index-space hyperplanes or a colouring shared by all octants do not. */
static const double *g_sort_key;
static int by_key(const void *pa, const void *pb) {
  int a = *(const int *)pa, b = *(const int *)pb;
  if (g_sort_key[a] < g_sort_key[b]) return -1;
  if (g_sort_key[a] > g_sort_key[b]) return 1;
  return (a > b) - (a < b);
}

static int sweep_orders(orc_solver *s, const orc_mesh *m) {
  int nc = s->nc;
  double *key = (double *)malloc(sizeof(double) * nc);
  int *rank = (int *)malloc(sizeof(int) * nc), *byk = (int *)malloc(sizeof(int) * nc);
  int *kc = (int *)malloc(sizeof(int) * nc), *start = (int *)malloc(sizeof(int) * (nc + 1));
  if (!key || !rank || !byk || !kc || !start) { free(key); free(rank); free(byk); free(kc); free(start); return ORC_E_OOM; }
  int N0 = s->ni + 1, N1 = s->nj + 1;
  for (int oct = 0; oct < 8; ++oct) {
    double d[3] = {oct & 1 ? -1.0 : 1.0, oct & 2 ? -1.0 : 1.0, oct & 4 ? -1.0 : 1.0};
    for (int c = 0; c < nc; ++c) {
      double sum = 0.0;
      int cnt = 0;
      if (m->ncells > 0) {
        const int *ids = m->cells + 8 * (size_t)c;
        for (int t = 0; t < 8; ++t) {
          int dup = 0;
          for (int u = 0; u < t; ++u) dup |= ids[u] == ids[t];
          if (dup) continue;
          const double *x = m->unodes + 3 * (size_t)ids[t];
          sum += ((d[0] * x[0]) + (d[1] * x[1])) + (d[2] * x[2]);
          ++cnt;
        }
      } else {
        int i = c % s->ni, j = (c / s->ni) % s->nj, k = c / (s->ni * s->nj);
        for (int t = 0; t < 8; ++t) {
          int I = i + (t & 1), J = j + (t >> 1 & 1), K = k + (t >> 2);
          const double *x = m->nodes + 3 * ((size_t)I + (size_t)N0 * ((size_t)J + (size_t)N1 * K));
          sum += ((d[0] * x[0]) + (d[1] * x[1])) + (d[2] * x[2]);
          ++cnt;
        }
      }
      key[c] = sum / cnt;
      byk[c] = c;
    }
    g_sort_key = key;
    qsort(byk, (size_t)nc, sizeof(int), by_key);
    for (int r = 0; r < nc; ++r) rank[byk[r]] = r;
    int ncol = 0;
    for (int r = 0; r < nc; ++r) {
      int c = byk[r], k = 0;
      for (int side = 0; side < 6; ++side) {
        int j = s->nb[6 * c + side];
        if (j >= 0 && rank[j] < r && kc[j] + 1 > k) k = kc[j] + 1;
      }
      kc[c] = k;
      if (k + 1 > ncol) ncol = k + 1;
    }
    /* colour by colour, index order within a colour (a counting sort) */
    for (int k = 0; k <= ncol; ++k) start[k] = 0;
    for (int c = 0; c < nc; ++c) ++start[kc[c] + 1];
    for (int k = 0; k < ncol; ++k) start[k + 1] += start[k];
    for (int c = 0; c < nc; ++c) s->corder[(size_t)oct * nc + start[kc[c]]++] = c;
  }
  free(key); free(rank); free(byk); free(kc); free(start);
  return ORC_OK;
}

int orc_create(const orc_mesh *m, const orc_vgrid *vg, const orc_gas *g, const orc_opts *o, const double *W0,
               orc_solver **out) {
  *out = NULL;
  if (m->ncells <= 0 && (m->ni < 1 || m->nj < 1 || m->nk < 1)) return ORC_E_INVALID;
  if (m->ncells > 0 && (!m->unodes || !m->cells || !m->face_patch)) return ORC_E_INVALID;
  if (vg->npoints > 0 ? !vg->points : (vg->n[0] < 1 || vg->n[1] < 1 || vg->n[2] < 1)) return ORC_E_INVALID;
  if (g->model == ORC_RYKOV && !(g->d_r > 0)) return ORC_E_INVALID;
  orc_solver *s = (orc_solver *)calloc(1, sizeof(orc_solver));
  if (!s) return ORC_E_OOM;
  if (m->ncells > 0) { s->ni = m->ncells; s->nj = s->nk = 1; s->nc = m->ncells; }
  else { s->ni = m->ni; s->nj = m->nj; s->nk = m->nk; s->nc = m->ni * m->nj * m->nk; }
  if (vg->npoints > 0) {
    /* one-node placeholders for the unused axis arrays */
    static const double one = 1.0;
    s->nvx = s->nvy = s->nvz = 1;
    s->nv = vg->npoints;
    s->pts = dup(vg->points, 4 * vg->npoints);
    s->vx = dup(&one, 1); s->vy = dup(&one, 1); s->vz = dup(&one, 1);
    s->wx = dup(&one, 1); s->wy = dup(&one, 1); s->wz = dup(&one, 1);
  } else {
    s->nvx = vg->n[0]; s->nvy = vg->n[1]; s->nvz = vg->n[2]; s->nv = s->nvx * s->nvy * s->nvz;
  }
  memcpy(s->bc, m->bc, sizeof s->bc);
  memcpy(s->wall_u, m->wall_u, sizeof s->wall_u);
  memcpy(s->wall_T, m->wall_T, sizeof s->wall_T);
  s->g = *g; s->o = *o;
  if (s->o.n_sweeps < 1) s->o.n_sweeps = 1;
  s->nvdf = g->model == ORC_RYKOV ? 2 : 1;
  s->nW = g->model == ORC_RYKOV ? 6 : 5;
  if (!s->pts) {
    s->vx = dup(vg->x[0], s->nvx); s->vy = dup(vg->x[1], s->nvy); s->vz = dup(vg->x[2], s->nvz);
    s->wx = dup(vg->w[0], s->nvx); s->wy = dup(vg->w[1], s->nvy); s->wz = dup(vg->w[2], s->nvz);
  }
  int nc = s->nc;
  s->vol = (double *)malloc(sizeof(double) * nc);
  s->xc = (double *)malloc(sizeof(double) * 3 * nc);
  s->S = (double *)malloc(sizeof(double) * 18 * nc);
  s->xf = (double *)malloc(sizeof(double) * 18 * nc);
  s->eps2 = (double *)malloc(sizeof(double) * nc);
  s->nb = (int *)malloc(sizeof(int) * 6 * nc);
  s->wid = (int *)malloc(sizeof(int) * 6 * nc);
  s->st = (double *)calloc(12 * (size_t)nc, sizeof(double));
  s->Mh = (double *)calloc(18 * (size_t)nc, sizeof(double));
  s->hot = (double *)calloc(12 * (size_t)nc, sizeof(double));
  s->kin = (double *)calloc(12 * (size_t)nc, sizeof(double));
  s->fkin = (double *)calloc(36 * (size_t)nc, sizeof(double));
  s->f0 = (double *)malloc(sizeof(double) * (size_t)nc * s->nv);
  s->f1 = s->nvdf == 2 ? (double *)malloc(sizeof(double) * (size_t)nc * s->nv) : NULL;
  if (!s->vx || !s->vy || !s->vz || !s->wx || !s->wy || !s->wz || (vg->npoints > 0 && !s->pts) || !s->vol || !s->xc || !s->S || !s->xf ||
      !s->eps2 || !s->nb || !s->wid || !s->st || !s->Mh || !s->hot || !s->kin || !s->fkin || !s->f0 || (s->nvdf == 2 && !s->f1)) {
    orc_destroy(s);
    return ORC_E_OOM;
  }
  int rc = m->ncells > 0 ? build_geometry_unstructured(s, m) : build_geometry(s, m);
  if (rc) { orc_destroy(s); return rc; }
  s->jump = s->o.visc_jump >= 0.0 ? s->o.visc_jump : (s->simplex ? 0.25 : 0.0);
  s->corder = (int *)malloc(sizeof(int) * 8 * (size_t)nc);
  if (!s->corder) { orc_destroy(s); return ORC_E_OOM; }
  rc = sweep_orders(s, m);
  if (rc) { orc_destroy(s); return rc; }
  set_maxwellian(s, W0);
  rc = init_state_from_f(s);
  if (rc) { orc_destroy(s); return rc; }
  *out = s;
  return ORC_OK;
}

/* Euler preconditioning (the presteps of Algorithm 1 for configurations with strong shocks):
   n inner steps of the synthetic solve in its inviscid form (Euler fluxes, slip walls, no
   high-order correction) from the current state, then f restarts as the Maxwellian of the
   result. */
int orc_euler_presteps(orc_solver *s, int n) {
  int nc = s->nc, used = 0;
  double *Wc = (double *)calloc(6 * (size_t)nc, sizeof(double)), *Wp = (double *)malloc(sizeof(double) * 6 * nc);
  if (!Wc || !Wp) { free(Wc); free(Wp); return ORC_E_OOM; }
  for (int i = 0; i < nc; ++i) cons_of(s, s->st + 12 * i, Wc + 6 * i);
  int rc = macro_solve(s, Wc, s->fkin, 1, n, s->o.macro_tol, &used);
  if (!rc) {
    double mm = 0.0;
    for (int i = 0; i < nc; ++i) {
      prim_of(s, Wc + 6 * i, Wp + 6 * i);
      mm += Wp[6 * i] * s->vol[i];
    }
    if (!s->open)
      for (int i = 0; i < nc; ++i) Wp[6 * i] *= s->mass_ref / mm;
    set_maxwellian(s, Wp);
    rc = init_state_from_f(s);
    s->macro_iters = used;
  }
  free(Wc);
  free(Wp);
  return rc;
}

int orc_set_f(orc_solver *s, const double *f0, const double *f1) {
  for (int i = 0; i < s->nc; ++i)
    for (int v = 0; v < s->nv; ++v) {
      s->f0[(size_t)v * s->nc + i] = f0[(size_t)i * s->nv + v];
      if (s->nvdf == 2) s->f1[(size_t)v * s->nc + i] = f1 ? f1[(size_t)i * s->nv + v] : 0.0;
    }
  return init_state_from_f(s);
}

int orc_get_f(const orc_solver *s, double *f0, double *f1) {
  for (int i = 0; i < s->nc; ++i)
    for (int v = 0; v < s->nv; ++v) {
      f0[(size_t)i * s->nv + v] = s->f0[(size_t)v * s->nc + i];
      if (f1 && s->nvdf == 2) f1[(size_t)i * s->nv + v] = s->f1[(size_t)v * s->nc + i];
    }
  return ORC_OK;
}

int orc_ncells(const orc_solver *s) { return s->nc; }
int orc_nvel(const orc_solver *s) { return s->nv; }
int orc_nwall(const orc_solver *s) { return s->nwall; }
double orc_eps(const orc_solver *s) { return s->eps; }
int orc_macro_iters(const orc_solver *s) { return s->macro_iters; }

void orc_get_W(const orc_solver *s, double *out6) {
  for (int i = 0; i < s->nc; ++i)
    for (int t = 0; t < 6; ++t) out6[6 * i + t] = s->st[12 * i + t];
}
void orc_get_half_moments(const orc_solver *s, double *out18) { memcpy(out18, s->Mh, sizeof(double) * 18 * s->nc); }
void orc_get_hot(const orc_solver *s, double *out12) { memcpy(out12, s->hot, sizeof(double) * 12 * s->nc); }
void orc_get_wall(const orc_solver *s, int *cell, int *side, double *rho_w, double *flux6) {
  for (int wf = 0; wf < s->nwall; ++wf) {
    cell[wf] = s->wcell[wf];
    side[wf] = s->wside[wf];
    rho_w[wf] = s->rho_w[wf];
    for (int k = 0; k < 6; ++k) flux6[6 * wf + k] = s->fkin[36 * s->wcell[wf] + 6 * s->wside[wf] + k];
  }
}
void orc_get_geometry(const orc_solver *s, double *vol, double *centre3, double *S18, double *xf18) {
  memcpy(vol, s->vol, sizeof(double) * s->nc);
  memcpy(centre3, s->xc, sizeof(double) * 3 * s->nc);
  for (int i = 0; i < s->nc; ++i)
    for (int side = 0; side < 6; ++side)
      for (int d = 0; d < 3; ++d) {
        int present = s->nb[6 * i + side] != -2;
        S18[18 * i + 3 * side + d] = present ? s->S[18 * i + 3 * side + d] : 0.0;
        xf18[18 * i + 3 * side + d] = present ? s->xf[18 * i + 3 * side + d] : 0.0;
      }
}

/* ---------------- pieces exposed for the pins ---------------- */

void orc_cell_gradient(const orc_solver *s, int i, const double *q, double *g) { lsq_grad(s, i, q, 1, g); }

void orc_cell_faces(const orc_solver *s, int i, const double *q, double *out6) { reconstruct(s, i, q, 1, out6); }

int orc_face_nsf(const orc_solver *s, const double *W, int i, int side, double *out12) {
  int nc = s->nc;
  if (i < 0 || i >= nc || side < 0 || side > 5) return ORC_E_INVALID;
  int j = s->nb[6 * i + side] >= 0 ? s->nb[6 * i + side] : i;
  macro_work m;
  memset(&m, 0, sizeof m);
  m.pr = (double *)malloc(sizeof(double) * 6 * nc);
  m.gP = (double *)calloc(15 * (size_t)nc, sizeof(double));
  m.mu = (double *)malloc(sizeof(double) * nc);
  if (!m.pr || !m.gP || !m.mu) { free(m.pr); free(m.gP); free(m.mu); return ORC_E_OOM; }
  for (int c = 0; c < nc; ++c) {
    prim_of(s, W + 6 * c, m.pr + 6 * c);
    m.mu[c] = visc(&s->g, m.pr[6 * c + 4]);
  }
  for (int k = 0; k < 5; ++k) {
    lsq_grad(s, i, m.pr + 1 + k, 6, m.gP + 15 * i + 3 * k);
    lsq_grad(s, j, m.pr + 1 + k, 6, m.gP + 15 * j + 3 * k);
  }
  face_nsf(s, &m, i, j, out12);
  free(m.pr); free(m.gP); free(m.mu);
  return ORC_OK;
}

double orc_cell_limiter(const orc_solver *s, int i, const double *q) {
  double g[3];
  lsq_grad(s, i, q, 1, g);
  return venkat_cell(s, i, q, 1, g);
}

void orc_get_face_flux(const orc_solver *s, double *out36) { memcpy(out36, s->fkin, sizeof(double) * 36 * s->nc); }

double orc_mass_scale(const orc_solver *s) { return s->mass_scale; }
