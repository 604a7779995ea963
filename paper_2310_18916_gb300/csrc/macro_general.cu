// macro_general.cu -- the FP64 synthetic NSF solve of GSIS (Section 3.3, Algorithm 2) on general
// (curvilinear) structured meshes: O-grids with far-field, pole and wrapped sides.
//
// Per inner step, one thread per cell, one launch per phase:
//   prim     primitives and viscosity of W;
//   grad     least-squares gradients of the conservative fields with their Venkatakrishnan
//            limiters, and of the primitives u, T_t, T_r;
//   face     each interior face flux once (the other cell takes its negative);
//   resid    R_i = -(1/V_i) [K_i + sum_faces (F_f - F_f^0) A_f] + Q_i: K_i the area-integrated
//            outward kinetic flux of the last kinetic step summed over the cell's faces, F_f the
//            face flux of this scheme (Rusanov + NSF between the two reconstructed states; a
//            far-field face against the free stream; a wall face the equilibrium wall flux) and
//            F^0 its value at the first inner step (Eq. full_constitutive as face fluxes: the
//            high-order part is frozen);
//   diag     local time step (CFL) and the LU-SGS diagonal;
//   sweep    red/black point-implicit passes with the matrix-free off-diagonal terms
//            (F(W_j + dW_j) - F(W_j)) . n - gamma dW_j (Eq. res_macro);
//   update   W += dW, the relative increment per field, and the early exit below macro_tol.
// Work is skipped once the early exit has fired, so the whole solve is enqueued at once.
// Euler mode (the presteps of Algorithm 1): Euler fluxes only, slip walls (pressure), no
// high-order correction and no kinetic flux sums.
#include <cuda_runtime.h>

#include <cmath>

#include "gsis_internal.h"
#include "wall_flux.cuh"

namespace gsis {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr int kBlock = 128;

__device__ __forceinline__ double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// primitives rho, u, T_t, T_r of conservative W (rho, rho u, rho E, rho E_r), E = |u|^2/2 +
// 3 T_t / 4 (+ d_r T_r / 4 in rho E_r)
// (one reciprocal of rho: FP64 divisions cost several FP64 instructions each on this GPU)
__device__ void prim_of(const MacroGenArgs &m, const double *W, double *p) {
  const double rho = W[0], ir = 1.0 / rho, u0 = W[1] * ir, u1 = W[2] * ir, u2 = W[3] * ir;
  const double Er = m.nW == 6 ? W[5] : 0.0;
  p[0] = rho;
  p[1] = u0;
  p[2] = u1;
  p[3] = u2;
  p[4] = (W[4] - 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2) - Er) * (ir * (4.0 / 3.0));
  p[5] = m.nW == 6 ? Er * (ir * (4.0 / m.d_r)) : p[4];
}

__device__ void cons_of(const MacroGenArgs &m, const double *p, double *W) {
  const double rho = p[0];
  const double Er = m.nW == 6 ? m.d_r * rho * p[5] / 4.0 : 0.0;
  W[0] = rho;
  W[1] = rho * p[1];
  W[2] = rho * p[2];
  W[3] = rho * p[3];
  W[4] = 0.5 * rho * (p[1] * p[1] + p[2] * p[2] + p[3] * p[3]) + 0.75 * rho * p[4] + Er;
  W[5] = Er;
}

__device__ bool physical(const double *p) { return p[0] > 0.0 && p[4] > 0.0 && p[5] > 0.0; }

// convective flux along the unit normal n
__device__ void euler_flux(const MacroGenArgs &m, const double *W, const double *n, double *F) {
  double p[6];
  prim_of(m, W, p);
  const double un = p[1] * n[0] + p[2] * n[1] + p[3] * n[2], pt = 0.5 * p[0] * p[4];
  F[0] = W[0] * un;
  for (int a = 0; a < 3; ++a) F[1 + a] = W[1 + a] * un + pt * n[a];
  F[4] = (W[4] + pt) * un;
  F[5] = m.nW == 6 ? W[5] * un : 0.0;
}

// the convective flux along each axis, F_a (a = x, y, z): F . n = sum_a F_a n_a
__device__ void axis_fluxes(const MacroGenArgs &m, const double *W, double *Fa) {
  double p[6];
  prim_of(m, W, p);
  const double pt = 0.5 * p[0] * p[4];
  for (int a = 0; a < 3; ++a) {
    const double ua = p[1 + a];
    double *F = Fa + 6 * a;
    F[0] = W[0] * ua;
    for (int b = 0; b < 3; ++b) F[1 + b] = W[1 + b] * ua + (a == b ? pt : 0.0);
    F[4] = (W[4] + pt) * ua;
    F[5] = m.nW == 6 ? W[5] * ua : 0.0;
  }
}

__device__ __forceinline__ double sound(double Tt) { return sqrt(Tt * (5.0 / 6.0)); }

// Eq. mu_kappa with R = 1/2: (kt, kr) = (mu / 4) A^{-1} (5, d_r); Shakhov: A_tt = 2/3, no kr
__device__ void kappas(const MacroGenArgs &m, double mu, double *kt, double *kr) {
  if (m.model == 0) {
    *kt = mu * 15.0 / 8.0;
    *kr = 0.0;
    return;
  }
  const double det = m.A[0] * m.A[3] - m.A[1] * m.A[2];
  *kt = mu / 4.0 * (m.A[3] * 5.0 - m.A[1] * m.d_r) / det;
  *kr = mu / 4.0 * (-m.A[2] * 5.0 + m.A[0] * m.d_r) / det;
}

// Outward flux per unit area of local equilibrium at the cell state p meeting the diffuse wall of
// `side` (u_w, T_w) along the unit normal n: the half moving into the wall leaves with the
// half-range moments J_k of N(u_n, T/2), the wall re-emits rho_w M(u_w, T_w) with zero net mass.
__device__ void wall_eq_flux(const MacroGenArgs &m, int patch, const double *p, const double *n, double *F) {
  const double *uT = m.wall_uT + 4 * patch;
  const double rho = p[0], T = p[4], un = p[1] * n[0] + p[2] * n[1] + p[3] * n[2], Tw = uT[3];
  const double sr = un / sqrt(T);
  const double M0 = exp(-sr * sr) / sqrt(kPi * T);
  const double J0 = 0.5 * (1.0 + erf(sr)), J1 = un * J0 + 0.5 * T * M0;
  const double J2 = un * J1 + 0.5 * T * J0, J3 = un * J2 + T * J1;
  const double K1 = -sqrt(Tw) / (2.0 * kSqrtPi), K2 = Tw / 4.0, K3 = Tw * K1;
  const double rw = -rho * J1 / K1;
  const double uwn = uT[0] * n[0] + uT[1] * n[1] + uT[2] * n[2];
  double ut[3], uwt[3];
  for (int a = 0; a < 3; ++a) {
    ut[a] = p[1 + a] - un * n[a];
    uwt[a] = uT[a] - uwn * n[a];
  }
  F[0] = rho * J1 + rw * K1;
  for (int a = 0; a < 3; ++a) F[1 + a] = n[a] * (rho * J2 + rw * K2) + rho * J1 * ut[a] + rw * K1 * uwt[a];
  const double ein = 0.5 * rho * (J3 + J1 * (dot3(ut, ut) + T));
  const double eout = 0.5 * rw * (K3 + K1 * (dot3(uwt, uwt) + Tw));
  double rin = 0.0, rout = 0.0;
  if (m.nW == 6) {
    rin = m.d_r * p[5] / 4.0 * rho * J1;
    rout = m.d_r * Tw / 4.0 * rw * K1;
  }
  F[4] = ein + eout + rin + rout;
  F[5] = rin + rout;
}

// NSF stress and heat fluxes at a face: gradients and viscosity the means of cells i and j
// (j = i on a far-field face); between two cells, with visc_jump = alpha > 0, each gradient g of
// u, T_t, T_r takes alpha times the jump along the centre line d = x_j - x_i,
// g + alpha (phi_j - phi_i - g.d) d / |d|^2.  out: sigma (xx yy zz xy xz yz), q_t (3), q_r (3).
__device__ void face_nsf(const MacroGenArgs &m, int i, int j, double *out) {
  double G[3][3], gT[3], gTr[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) G[a][b] = 0.5 * (m.gP[15 * (size_t)i + 3 * a + b] + m.gP[15 * (size_t)j + 3 * a + b]);
    gT[a] = 0.5 * (m.gP[15 * (size_t)i + 9 + a] + m.gP[15 * (size_t)j + 9 + a]);
    gTr[a] = 0.5 * (m.gP[15 * (size_t)i + 12 + a] + m.gP[15 * (size_t)j + 12 + a]);
  }
  if (m.visc_jump > 0.0 && j != i) {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = m.xc[3 * (size_t)j + a] - m.xc[3 * (size_t)i + a];
    const double s = m.visc_jump / dot3(d, d);
    double *g[5] = {G[0], G[1], G[2], gT, gTr};
    for (int k = 0; k < 5; ++k) {
      const double c = m.pr[6 * (size_t)j + 1 + k] - m.pr[6 * (size_t)i + 1 + k] - dot3(g[k], d);
      for (int a = 0; a < 3; ++a) g[k][a] += s * c * d[a];
    }
  }
  const double muf = 0.5 * (m.mu[i] + m.mu[j]);
  double kt, kr;
  kappas(m, muf, &kt, &kr);
  const double div = G[0][0] + G[1][1] + G[2][2];
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int t = 0; t < 6; ++t) {
    const int a = ia[t], b = ib[t];
    out[t] = -muf * (G[a][b] + G[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
  }
  for (int a = 0; a < 3; ++a) {
    out[6 + a] = -kt * gT[a];
    out[9 + a] = m.nW == 6 ? -kr * gTr[a] : 0.0;
  }
}

// reconstructed conservative state of cell i at the face centre of `side` (cell state where the
// reconstruction is not physical)
__device__ void face_state(const MacroGenArgs &m, int i, int side, double *Wf, double *pf) {
  const double *r = m.gen[i].f[side].r;
  for (int k = 0; k < 6; ++k) Wf[k] = 0.0;
  for (int k = 0; k < m.nW; ++k)
    Wf[k] = m.W[6 * (size_t)i + k] + m.phW[6 * (size_t)i + k] * dot3(m.gW + 18 * (size_t)i + 3 * k, r);
  prim_of(m, Wf, pf);
  if (!physical(pf)) {
    for (int k = 0; k < m.nW; ++k) Wf[k] = m.W[6 * (size_t)i + k];
    prim_of(m, Wf, pf);
  }
}

// Rusanov + NSF flux per unit area through the face (i, side) along its unit normal n, between
// i's face state and the state on the other side (cell j's face state, or the free stream)
__device__ void face_flux(const MacroGenArgs &m, int i, int side, int j, const double *n, double *F) {
  double WL[6], WR[6], pL[6], pR[6], FL[6], FR[6];
  face_state(m, i, side, WL, pL);
  int jv = i;
  if (j >= 0) {
    face_state(m, j, nb_side(m.gnf, i, side), WR, pR);
    jv = j;
  } else {
    const double *uT = m.wall_uT + 4 * patch_of(m.gpat, i, side);
    const double pinf[6] = {1.0, uT[0], uT[1], uT[2], uT[3], uT[3]};
    cons_of(m, pinf, WR);
    prim_of(m, WR, pR);
  }
  euler_flux(m, WL, n, FL);
  euler_flux(m, WR, n, FR);
  const double lL = fabs(pL[1] * n[0] + pL[2] * n[1] + pL[3] * n[2]) + sound(pL[4]);
  const double lR = fabs(pR[1] * n[0] + pR[2] * n[1] + pR[3] * n[2]) + sound(pR[4]);
  const double lam = lL > lR ? lL : lR;
  for (int k = 0; k < 6; ++k) F[k] = k < m.nW ? 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (WR[k] - WL[k]) : 0.0;
  if (m.euler) return;
  double nsf[12], sn[3], uf[3];
  face_nsf(m, i, jv, nsf);
  for (int a = 0; a < 3; ++a) uf[a] = 0.5 * (m.pr[6 * (size_t)i + 1 + a] + m.pr[6 * (size_t)jv + 1 + a]);
  const int map[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (int a = 0; a < 3; ++a) sn[a] = nsf[map[a][0]] * n[0] + nsf[map[a][1]] * n[1] + nsf[map[a][2]] * n[2];
  for (int a = 0; a < 3; ++a) F[1 + a] += sn[a];
  F[4] += dot3(sn, uf) + dot3(nsf + 6, n) + (m.nW == 6 ? dot3(nsf + 9, n) : 0.0);
  if (m.nW == 6) F[5] += dot3(nsf + 9, n);
}

__device__ __forceinline__ bool done(const MacroGenArgs &m) { return *(volatile int *)m.flag != 0; }

__global__ void init_kernel(MacroGenArgs m) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
    double p[6];
    for (int k = 0; k < 6; ++k) p[k] = m.Mh[(size_t)m.mh_stride * c + k];
    cons_of(m, p, m.W + 6 * (size_t)c);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    m.flag[0] = 0;
    m.flag[1] = 0;
  }
}

__global__ void prim_kernel(MacroGenArgs m) {
  if (done(m)) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
    double *p = m.pr + 6 * (size_t)c;
    prim_of(m, m.W + 6 * (size_t)c, p);
    if (!physical(p)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
    m.mu[c] = m.mu0 * pow(p[4], m.omega);
  }
}

__global__ void grad_kernel(MacroGenArgs m) {
  if (done(m)) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
    const GenCell<double> &g = m.gen[c];
    int nb[6];
    for (int s = 0; s < 6; ++s) nb[s] = m.gnb[6 * (size_t)c + s];
    // conservative fields: gradient and limiter
    for (int k = 0; k < m.nW; ++k) {
      const double qi = m.W[6 * (size_t)c + k];
      double gr[3] = {0.0, 0.0, 0.0}, qmax = qi, qmin = qi;
      for (int s = 0; s < 6; ++s) {
        if (nb[s] < 0) continue;
        const double qj = m.W[6 * (size_t)nb[s] + k], d = qj - qi;
        if (!m.gso)
          for (int a = 0; a < 3; ++a) gr[a] += g.f[s].w[a] * d;
        qmax = qj > qmax ? qj : qmax;
        qmin = qj < qmin ? qj : qmin;
      }
      if (m.gso)
        for (int e = m.gso[c]; e < m.gso[c + 1]; ++e) {
          const double d = m.W[6 * (size_t)m.gsi[e] + k] - qi;
          for (int a = 0; a < 3; ++a) gr[a] += m.gsw[3 * e + a] * d;
        }
      double phi = 1.0;
      for (int s = 0; s < 6; ++s) {
        if (nb[s] == NB_ABSENT || nb[s] == NB_AXIS) continue;
        const double d2 = dot3(gr, g.f[s].r);
        if (d2 == 0.0) continue;
        const double dm = d2 > 0 ? qmax - qi : qmin - qi;
        const double num = (dm * dm + g.eps2) * d2 + 2.0 * d2 * d2 * dm;
        const double den = d2 * (dm * dm + 2.0 * d2 * d2 + dm * d2 + g.eps2);
        const double p = num / den;
        if (p < phi) phi = p;
      }
      for (int a = 0; a < 3; ++a) m.gW[18 * (size_t)c + 3 * k + a] = gr[a];
      m.phW[6 * (size_t)c + k] = phi;
    }
    // primitives u (3), T_t, T_r: gradients only
    for (int k = 0; k < 5; ++k) {
      const double qi = m.pr[6 * (size_t)c + 1 + k];
      double gr[3] = {0.0, 0.0, 0.0};
      if (m.gso) {
        for (int e = m.gso[c]; e < m.gso[c + 1]; ++e) {
          const double d = m.pr[6 * (size_t)m.gsi[e] + 1 + k] - qi;
          for (int a = 0; a < 3; ++a) gr[a] += m.gsw[3 * e + a] * d;
        }
      } else {
        for (int s = 0; s < 6; ++s) {
          if (nb[s] < 0) continue;
          const double d = m.pr[6 * (size_t)nb[s] + 1 + k] - qi;
          for (int a = 0; a < 3; ++a) gr[a] += g.f[s].w[a] * d;
        }
      }
      for (int a = 0; a < 3; ++a) m.gP[15 * (size_t)c + 3 * k + a] = gr[a];
    }
  }
}

// Interior faces once each, from the cell on their lower side (the upper sides 1, 3, 5 of every
// cell of a structured block; on an unstructured mesh the cell of lower index): the flux seen
// from the other cell is its exact negative (opposite normal, swapped states), so each cell's
// residual reads it instead of computing it again.
__global__ void face_kernel(MacroGenArgs m) {
  if (done(m)) return;
  const int per = m.gnf ? 6 : 3;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < per * m.nc; t += gridDim.x * blockDim.x) {
    const int c = t / per, s = m.gnf ? t - 6 * c : 2 * (t - 3 * c) + 1;
    const int nb = m.gnb[6 * (size_t)c + s];
    if (nb < 0 || (m.gnf && nb < c)) continue;
    const double *S = m.gen[c].f[s].S;
    const double A = sqrt(dot3(S, S)), iA = 1.0 / A, n[3] = {S[0] * iA, S[1] * iA, S[2] * iA};
    face_flux(m, c, s, nb, n, m.Ff + 36 * (size_t)c + 6 * s);
  }
}

__global__ void resid_kernel(MacroGenArgs m, int step) {
  if (done(m)) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
    const GenCell<double> &g = m.gen[c];
    double acc[6];
    for (int k = 0; k < 6; ++k) acc[k] = m.euler ? 0.0 : m.K[6 * (size_t)c + k];
    for (int s = 0; s < 6; ++s) {
      const int nb = m.gnb[6 * (size_t)c + s];
      if (nb == NB_ABSENT || nb == NB_AXIS) continue;
      const double *S = g.f[s].S;
      const double A = sqrt(dot3(S, S)), iA = 1.0 / A, n[3] = {S[0] * iA, S[1] * iA, S[2] * iA};
      double F[6];
      if (nb == NB_WALL && m.euler) {
        // slip wall: the pressure of the cell
        const double *pc = m.pr + 6 * (size_t)c;
        const double pt = 0.5 * pc[0] * pc[4];
        for (int k = 0; k < 6; ++k) F[k] = 0.0;
        for (int a = 0; a < 3; ++a) F[1 + a] = pt * n[a];
      } else if (nb == NB_WALL && m.wall_g13) {
        const int pt = patch_of(m.gpat, c, s);
        const double *pc = m.pr + 6 * (size_t)c, *M = m.Mh + 18 * (size_t)c, *uT = m.wall_uT + 4 * pt;
        grad13_wall_flux(m.nW, m.d_r, pc[0], pc + 1, pc[4], pc[5], n, M + 6, M + 12, M + 15, uT, uT[3], F);
      } else if (nb == NB_WALL) {
        wall_eq_flux(m, patch_of(m.gpat, c, s), m.pr + 6 * (size_t)c, n, F);
      } else if (nb >= 0) {
        // each interior face flux is computed once, by its owner (see face_kernel)
        const bool own = m.gnf ? c < nb : (s & 1) != 0;
        const double *Fs = own ? m.Ff + 36 * (size_t)c + 6 * s : m.Ff + 36 * (size_t)nb + 6 * nb_side(m.gnf, c, s);
        for (int k = 0; k < 6; ++k) F[k] = own ? Fs[k] : -Fs[k];
      } else {
        face_flux(m, c, s, nb, n, F);
      }
      if (m.euler) {
        for (int k = 0; k < m.nW; ++k) acc[k] += F[k] * A;
        continue;
      }
      double *F0 = m.F0 + 36 * (size_t)c + 6 * s;
      if (step == 0)
        for (int k = 0; k < 6; ++k) F0[k] = F[k];
      for (int k = 0; k < m.nW; ++k) acc[k] += (F[k] - F0[k]) * A;
    }
    const double V = m.vol[c];
    double *R = m.R + 6 * (size_t)c;
    for (int k = 0; k < m.nW; ++k) R[k] = -acc[k] / V;
    if (m.nW == 6) {
      // Q = (d_r rho R / 2)(T - T_r) / (Z_r tau), T = (3 T_t + d_r T_r) / (3 + d_r)
      const double *p = m.pr + 6 * (size_t)c;
      const double tau = 2.0 * m.mu0 * pow(p[4], m.omega - 1.0) / p[0];
      const double T = (3.0 * p[4] + m.d_r * p[5]) / (3.0 + m.d_r);
      R[5] += m.d_r * p[0] * (T - p[5]) / (4.0 * m.Z_r * tau);
    }
  }
}

// gamma of the face (c, side): spectral radius of the convective Jacobian (the larger of the
// two cells') plus the viscous term 2 max(mu / rho) / |n . d|
__device__ double face_gamma(const MacroGenArgs &m, int c, int s, int nb, const double *n) {
  const double *pc = m.pr + 6 * (size_t)c;
  const double li = fabs(pc[1] * n[0] + pc[2] * n[1] + pc[3] * n[2]) + sound(pc[4]);
  if (nb >= 0) {
    const double *pj = m.pr + 6 * (size_t)nb;
    const double lj = fabs(pj[1] * n[0] + pj[2] * n[1] + pj[3] * n[2]) + sound(pj[4]);
    const double d[3] = {m.xc[3 * (size_t)nb] - m.xc[3 * (size_t)c], m.xc[3 * (size_t)nb + 1] - m.xc[3 * (size_t)c + 1],
                         m.xc[3 * (size_t)nb + 2] - m.xc[3 * (size_t)c + 2]};
    const double ni = m.mu[c] / pc[0], nj = m.mu[nb] / pj[0];
    const double lam = li > lj ? li : lj;
    return m.euler ? lam : lam + 2.0 * (ni > nj ? ni : nj) / fabs(dot3(n, d));
  }
  const double *r = m.gen[c].f[s].r;
  return m.euler ? li : li + 2.0 * (m.mu[c] / pc[0]) / fabs(dot3(n, r));
}

__global__ void diag_kernel(MacroGenArgs m) {
  if (done(m)) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
    const GenCell<double> &g = m.gen[c];
    const double *p = m.pr + 6 * (size_t)c;
    double lsum = 0.0, gsum = 0.0;
    for (int s = 0; s < 6; ++s) {
      const int nb = m.gnb[6 * (size_t)c + s];
      if (nb == NB_ABSENT || nb == NB_AXIS) continue;
      const double *S = g.f[s].S;
      const double A = sqrt(dot3(S, S)), iA = 1.0 / A, n[3] = {S[0] * iA, S[1] * iA, S[2] * iA};
      lsum += (fabs(p[1] * n[0] + p[2] * n[1] + p[3] * n[2]) + sound(p[4])) * A;
      const double gam = face_gamma(m, c, s, nb, n);
      gsum += gam * A;
      if (nb >= 0) m.gam[6 * (size_t)c + s] = gam;  // fixed during the sweeps
    }
    // this cell's axis fluxes at W (the sweeps' base) and at W + dW (dW = 0 until it is updated)
    axis_fluxes(m, m.W + 6 * (size_t)c, m.FW0 + 18 * (size_t)c);
    for (int k = 0; k < 18; ++k) m.FW[18 * (size_t)c + k] = m.FW0[18 * (size_t)c + k];
    const double V = m.vol[c];
    const double dt = m.cfl * V / lsum;
    double srcdiag = 0.0;
    if (m.nW == 6) srcdiag = 1.0 / (m.Z_r * (2.0 * m.mu0 * pow(p[4], m.omega - 1.0) / p[0]));
    // the sweeps multiply by the inverse diagonal
    for (int k = 0; k < 6; ++k) m.D[6 * (size_t)c + k] = 1.0 / (1.0 / dt + gsum / (2.0 * V) + (k == 5 ? srcdiag : 0.0));
    for (int k = 0; k < 6; ++k) m.dW[6 * (size_t)c + k] = 0.0;
  }
}

__global__ void sweep_kernel(MacroGenArgs m, int first, int count) {
  if (done(m)) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    const int c = m.colcells[first + t];
    const GenCell<double> &g = m.gen[c];
    double acc[6];
    for (int k = 0; k < 6; ++k) acc[k] = m.R[6 * (size_t)c + k];
    for (int s = 0; s < 6; ++s) {
      const int nb = m.gnb[6 * (size_t)c + s];
      if (nb < 0) continue;
      const double *S = g.f[s].S;
      const double A = sqrt(dot3(S, S)), iA = 1.0 / A, n[3] = {S[0] * iA, S[1] * iA, S[2] * iA};
      const double gam = m.gam[6 * (size_t)c + s];
      // (F(W_j + dW_j) - F(W_j)) . n from the neighbour's axis fluxes
      const double *F1 = m.FW + 18 * (size_t)nb, *F0 = m.FW0 + 18 * (size_t)nb;
      const double kA = 0.5 * A * g.invV;
      for (int k = 0; k < m.nW; ++k) {
        const double dF = (F1[k] - F0[k]) * n[0] + (F1[6 + k] - F0[6 + k]) * n[1] + (F1[12 + k] - F0[12 + k]) * n[2];
        acc[k] -= (dF - gam * m.dW[6 * (size_t)nb + k]) * kA;
      }
    }
    double Wn[6];
    for (int k = 0; k < 6; ++k) {
      const double d = k < m.nW ? acc[k] * m.D[6 * (size_t)c + k] : 0.0;
      if (k < m.nW) m.dW[6 * (size_t)c + k] = d;
      Wn[k] = m.W[6 * (size_t)c + k] + d;
    }
    axis_fluxes(m, Wn, m.FW + 18 * (size_t)c);
  }
}

// W += dW and the per-block sums of dW^2 V and W^2 V per field (fixed grid, fixed order)
__global__ void update_kernel(MacroGenArgs m) {
  __shared__ double red[2 * 6][kBlock];
  if (done(m)) return;
  double num[6] = {0, 0, 0, 0, 0, 0}, den[6] = {0, 0, 0, 0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.nc; c += gridDim.x * blockDim.x) {
    const double V = m.vol[c];
    for (int k = 0; k < m.nW; ++k) {
      const double d = m.dW[6 * (size_t)c + k];
      const double w = m.W[6 * (size_t)c + k] + d;
      m.W[6 * (size_t)c + k] = w;
      if (!isfinite(w)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
      num[k] += d * d * V;
      den[k] += w * w * V;
    }
  }
  for (int k = 0; k < 6; ++k) {
    red[k][threadIdx.x] = num[k];
    red[6 + k][threadIdx.x] = den[k];
  }
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 12; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 12) m.part[12 * (size_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// the relative increment max_k sqrt(sum dW_k^2 V / sum W_k^2 V); below tol the solve stops.
__global__ void check_kernel(MacroGenArgs m, int nparts, int step) {
  if (done(m)) return;
  if (threadIdx.x != 0) return;
  double num[6] = {0, 0, 0, 0, 0, 0}, den[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nparts; ++b)
    for (int k = 0; k < 6; ++k) {
      num[k] += m.part[12 * (size_t)b + k];
      den[k] += m.part[12 * (size_t)b + 6 + k];
    }
  // fields that are identically zero up to rounding (volume-weighted RMS below 1e-12: the z
  // momentum of a 2D flow) have no relative increment to test
  double delta = 0.0;
  for (int k = 0; k < m.nW; ++k)
    if (den[k] > 1e-24 * m.vsum) {
      const double e = sqrt(num[k] / den[k]);
      if (e > delta) delta = e;
    }
  m.flag[1] = step + 1;
  if (delta < m.tol) m.flag[0] = 1;
}

// W^{n+1} as primitives; a closed domain rescales the density to its total mass
__global__ void final_kernel(MacroGenArgs m) {
  __shared__ double red[256];
  double mm = 0.0;
  for (int c = threadIdx.x; c < m.nc; c += blockDim.x) {
    double *p = m.Wout + 6 * (size_t)c;
    prim_of(m, m.W + 6 * (size_t)c, p);
    if (m.relax < 1.0 && !m.euler) {
      // under-relaxed update: W^{n+1/2} + relax (W^{n+1} - W^{n+1/2}) in primitives
      const double *q = m.Mh + (size_t)m.mh_stride * c;
      for (int k = 0; k < 6; ++k) p[k] = q[k] + m.relax * (p[k] - q[k]);
    }
    mm += p[0] * m.vol[c];
  }
  red[threadIdx.x] = mm;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (m.closed) {
    const double f = m.mass_ref / red[0];
    for (int c = threadIdx.x; c < m.nc; c += blockDim.x) m.Wout[6 * (size_t)c] *= f;
  }
  if (threadIdx.x == 0) *m.iters = m.flag[1];
}

}  // namespace

int macro_general_parts(int nc) {
  int grid = (nc + kBlock - 1) / kBlock;
  return grid > 4096 ? 4096 : grid;
}

cudaError_t run_macro_general(const MacroGenArgs &m, cudaStream_t s) {
  const int grid = macro_general_parts(m.nc);
  init_kernel<<<grid, kBlock, 0, s>>>(m);
  for (int step = 0; step < m.steps; ++step) {
    prim_kernel<<<grid, kBlock, 0, s>>>(m);
    grad_kernel<<<grid, kBlock, 0, s>>>(m);
    face_kernel<<<grid, kBlock, 0, s>>>(m);
    resid_kernel<<<grid, kBlock, 0, s>>>(m, step);
    diag_kernel<<<grid, kBlock, 0, s>>>(m);
    for (int sw = 0; sw < m.sweeps; ++sw) {
      for (int k = 0; k < m.ncolm; ++k)
        sweep_kernel<<<grid, kBlock, 0, s>>>(m, m.colm_off[k], m.colm_off[k + 1] - m.colm_off[k]);
    }
    update_kernel<<<grid, kBlock, 0, s>>>(m);
    check_kernel<<<1, 32, 0, s>>>(m, grid, step);
  }
  final_kernel<<<1, 256, 0, s>>>(m);
  return cudaGetLastError();
}

}  // namespace gsis
