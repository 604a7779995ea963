// macro.cu -- FP64 synthetic NSF solve of GSIS-II on sm_103a (Section 3.2 of arXiv 2310.18916).
//
// One persistent cooperative kernel runs all inner steps (Algorithm 2 body):
//   primitives -> LSQ gradients and Venkatakrishnan limiters -> face fluxes (Rusanov
//   convective + NSF viscous, plus the frozen high-order correction) -> residual R_i
//   (Eq. delta_Macroscopic_equations) -> matrix-free point-implicit sweeps over red/black
//   colours (Eq. res_macro) -> update and inner residual.
// The high-order terms of Eq. full_constitutive enter as face fluxes: the kinetic face flux
// of the last kinetic step minus this scheme's face flux at W^{n+1/2}, frozen over the inner
// steps.  Wall faces carry the kinetic wall flux plus the increment of the equilibrium wall
// flux of the boundary cell (the boundary-flux modification of Section 3.2).
// Phases are separated by a grid barrier whose spin is bounded: on time-out it raises an error
// flag and every block returns.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>

#include "gsis_internal.h"

namespace gsis {

namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr int kBlock = 256;
constexpr long long kSpinLimit = 1LL << 31;  // ~1 s of clock64 cycles at 2 GHz

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) { return *(volatile const unsigned *)p; }

// Sense-reversing grid barrier with a bounded spin.  Returns false when any block has flagged an
// error (including a time-out here), so every caller leaves the kernel together.
__device__ bool grid_sync(unsigned *bar, int *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_volatile(bar + 1);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_volatile(bar + 1) == gen) {
        if (clock64() - t0 > kSpinLimit || *(volatile int *)err != 0) {
          atomicCAS(err, 0, GSIS_ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)err == 0;
}

struct Geo {
  int n0, n1, n2, nc;
  __device__ void nat(int c, int *v) const {
    v[0] = c % n0;
    v[1] = (c / n0) % n1;
    v[2] = c / (n0 * n1);
  }
};

__device__ __forceinline__ void prim_of(const double *W, int nW, double dr, double *p) {
  const double rho = W[0], ir = 1.0 / rho;
  const double ux = W[1] * ir, uy = W[2] * ir, uz = W[3] * ir;
  const double Er = nW == 6 ? W[5] : 0.0;
  const double Tt = (W[4] - 0.5 * rho * (ux * ux + uy * uy + uz * uz) - Er) * (ir * (4.0 / 3.0));
  p[0] = rho;
  p[1] = ux;
  p[2] = uy;
  p[3] = uz;
  p[4] = Tt;
  p[5] = nW == 6 ? Er * ir * (4.0 / dr) : Tt;
}

// Euler flux along n = sg e_a: (rho u_n, rho u u_n + p_t n, (rho E + p_t) u_n, rho E_r u_n)
__device__ __forceinline__ void euler_axis(const double *W, int nW, double dr, int a, double sg, double *F) {
  const double ir = 1.0 / W[0];
  const double un = sg * W[1 + a] * ir;
  const double Er = nW == 6 ? W[5] : 0.0;
  // p_t = rho Tt / 2 = (2/3) (rho E - |rho u|^2 / (2 rho) - rho E_r)
  const double pt = (2.0 / 3.0) * (W[4] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) * ir - Er);
  F[0] = W[0] * un;
  for (int b = 0; b < 3; ++b) F[1 + b] = W[1 + b] * un + (b == a ? sg * pt : 0.0);
  F[4] = (W[4] + pt) * un;
  F[5] = Er * un;
  (void)dr;
}

__device__ __forceinline__ double sound(double Tt) { return sqrt(5.0 * Tt / 6.0); }

__device__ __forceinline__ double visc(const MacroArgs &m, double Tt) { return m.Kn / sqrt(kPi) * pow(Tt, m.omega); }

__device__ __forceinline__ void kappas(const MacroArgs &m, double mu, double *kt, double *kr) {
  if (m.model == 0) {
    *kt = mu * 15.0 / 8.0;
    *kr = 0.0;
    return;
  }
  const double det = m.A[0] * m.A[3] - m.A[1] * m.A[2];
  *kt = mu / 4.0 * (m.A[3] * 5.0 - m.A[1] * m.d_r) / det;
  *kr = mu / 4.0 * (-m.A[2] * 5.0 + m.A[0] * m.d_r) / det;
}

// Outward wall flux per unit area of local equilibrium at the cell state p meeting the diffuse
// wall (u_w, T_w): half-range moments J_k of N(u_n, T/2) for the half moving into the wall,
// re-emission rho_w M(u_w, T_w) with zero net mass flux.  n = sg e_a.
__device__ void equilibrium_wall_flux(const MacroArgs &m, const double *p, int a, double sg, const double *uT,
                                      double *F) {
  const double rho = p[0], T = p[4], un = sg * p[1 + a], Tw = uT[3];
  const double sr = un / sqrt(T);
  const double phi0 = exp(-sr * sr) / sqrt(kPi * T);
  const double J0 = 0.5 * erfc(-sr);
  const double J1 = un * J0 + 0.5 * T * phi0;
  const double J2 = un * J1 + 0.5 * T * J0;
  const double J3 = un * J2 + T * J1;
  const double K1 = -sqrt(Tw) / (2.0 * sqrt(kPi)), K2 = Tw / 4.0, K3 = Tw * K1;
  const double rw = -rho * J1 / K1;
  double ut[3], uwt[3];
  for (int b = 0; b < 3; ++b) {
    ut[b] = b == a ? 0.0 : p[1 + b];
    uwt[b] = b == a ? 0.0 : uT[b];
  }
  const double ut2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  const double uw2 = uwt[0] * uwt[0] + uwt[1] * uwt[1] + uwt[2] * uwt[2];
  F[0] = rho * J1 + rw * K1;
  for (int b = 0; b < 3; ++b) F[1 + b] = (b == a ? sg : 0.0) * (rho * J2 + rw * K2) + rho * J1 * ut[b] + rw * K1 * uwt[b];
  const double rin = m.nW == 6 ? m.d_r * p[5] / 4.0 * rho * J1 : 0.0;
  const double rout = m.nW == 6 ? m.d_r * Tw / 4.0 * rw * K1 : 0.0;
  F[4] = 0.5 * rho * (J3 + J1 * (ut2 + T)) + 0.5 * rw * (K3 + K1 * (uw2 + Tw)) + rin + rout;
  F[5] = rin + rout;
}

__device__ __forceinline__ double venkat_face(double fi, double fmax, double fmin, double d2, double eps2) {
  const double dm = d2 > 0.0 ? fmax - fi : (d2 < 0.0 ? fmin - fi : 0.0);
  return (dm * dm + eps2 + 2.0 * d2 * dm) / (dm * dm + 2.0 * d2 * d2 + dm * d2 + eps2);
}
}  // namespace

__global__ void __launch_bounds__(kBlock) macro_kernel(MacroArgs m) {
  const Geo G{m.g.n[0], m.g.n[1], m.g.n[2], m.g.nc};
  const int nc = G.nc, nW = m.nW;
  // work items are dealt round-robin over the blocks first, so every SM holds cells
  const int tid = blockIdx.x + gridDim.x * threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int cs[3] = {1, G.n0, G.n0 * G.n1};
  const int act[3] = {m.g.act[0], m.g.act[1], m.g.act[2]};
  __shared__ double sred[kBlock];

  // initial conservative state from the moments of f^{n+1/2}
  for (int c = tid; c < nc; c += nthr) {
    const double *M = m.Mh + (size_t)c * 18;
    double *W = m.W + (size_t)c * 6;
    const double rho = M[0];
    W[0] = rho;
    W[1] = rho * M[1];
    W[2] = rho * M[2];
    W[3] = rho * M[3];
    const double Er = nW == 6 ? m.d_r * rho * M[5] / 4.0 : 0.0;
    W[4] = 0.5 * rho * (M[1] * M[1] + M[2] * M[2] + M[3] * M[3]) + 0.75 * rho * M[4] + Er;
    W[5] = Er;
  }
  if (!grid_sync(m.bar, m.err)) return;

  int used = 0;
  for (int step = 0; step < m.steps; ++step) {
    // ---- phase 1: primitives, viscosity
    for (int c = tid; c < nc; c += nthr) {
      double *p = m.pr + (size_t)c * 6;
      prim_of(m.W + (size_t)c * 6, nW, m.d_r, p);
      if (!(p[0] > 0.0) || !(p[4] > 0.0) || !(p[5] > 0.0)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
      m.mu[c] = visc(m, p[4]);
    }
    if (!grid_sync(m.bar, m.err)) return;
    // ---- phase 2: gradients, limiters, axis Euler fluxes, time step and diagonal
    for (int c = tid; c < nc; c += nthr) {
      int nt[3];
      G.nat(c, nt);
      const double *Wi = m.W + (size_t)c * 6, *pi = m.pr + (size_t)c * 6;
      AxisCell<double> gc[3];
      double V = 1.0;
      for (int a = 0; a < 3; ++a) {
        gc[a] = m.ax[a][nt[a]];
        V *= gc[a].h;
      }
      const double eps2 = m.g.K3 * V;
      for (int k = 0; k < nW; ++k) {
        double gr[3] = {0, 0, 0}, fmax = Wi[k], fmin = Wi[k];
        for (int a = 0; a < 3; ++a) {
          if (!act[a]) continue;
          double lo = Wi[k], hi = Wi[k];
          if (nt[a] > 0) { lo = m.W[(size_t)(c - cs[a]) * 6 + k]; fmax = fmax > lo ? fmax : lo; fmin = fmin < lo ? fmin : lo; }
          if (nt[a] < m.g.n[a] - 1) { hi = m.W[(size_t)(c + cs[a]) * 6 + k]; fmax = fmax > hi ? fmax : hi; fmin = fmin < hi ? fmin : hi; }
          gr[a] = gc[a].clo * (lo - Wi[k]) + gc[a].chi * (hi - Wi[k]);
        }
        double phi = 1.0;
        for (int a = 0; a < 3; ++a) {
          if (!act[a]) continue;
          for (int sd = 0; sd < 2; ++sd) {
            const double d2 = gr[a] * (sd ? gc[a].rhi : gc[a].rlo);
            const double pf = venkat_face(Wi[k], fmax, fmin, d2, eps2);
            phi = pf < phi ? pf : phi;
          }
        }
        for (int a = 0; a < 3; ++a) m.gW[((size_t)c * 6 + k) * 3 + a] = gr[a];
        m.phW[(size_t)c * 6 + k] = phi;
      }
      for (int k = 0; k < 5; ++k) {
        double gr[3] = {0, 0, 0};
        const double qi = pi[1 + k];
        for (int a = 0; a < 3; ++a) {
          if (!act[a]) continue;
          const double lo = nt[a] > 0 ? m.pr[(size_t)(c - cs[a]) * 6 + 1 + k] : qi;
          const double hi = nt[a] < m.g.n[a] - 1 ? m.pr[(size_t)(c + cs[a]) * 6 + 1 + k] : qi;
          gr[a] = gc[a].clo * (lo - qi) + gc[a].chi * (hi - qi);
        }
        for (int a = 0; a < 3; ++a) m.gP[((size_t)c * 5 + k) * 3 + a] = gr[a];
      }
      double lsum = 0.0, gsum = 0.0;
      const double ci = sound(pi[4]), nui = m.mu[c] / pi[0];
      for (int a = 0; a < 3; ++a) {
        euler_axis(Wi, nW, m.d_r, a, 1.0, m.Fc + ((size_t)c * 3 + a) * 6);
        if (!act[a]) continue;
        const double A = V * gc[a].invh;
        const double li = fabs(pi[1 + a]) + ci;
        for (int sd = 0; sd < 2; ++sd) {
          const bool inside = sd ? nt[a] < m.g.n[a] - 1 : nt[a] > 0;
          lsum += li * A;
          double gam;
          if (inside) {
            const int j = c + (sd ? cs[a] : -cs[a]);
            const double *pj = m.pr + (size_t)j * 6;
            const double lj = fabs(pj[1 + a]) + sound(pj[4]);
            const double nuj = m.mu[j] / pj[0];
            const AxisCell<double> gj = m.ax[a][nt[a] + (sd ? 1 : -1)];
            const double dx = sd ? (gc[a].rhi - gj.rlo) : (gj.rhi - gc[a].rlo);
            gam = (li > lj ? li : lj) + 2.0 * (nui > nuj ? nui : nuj) / fabs(dx);
            if (sd) m.gam[(size_t)c * 3 + a] = gam;
          } else {
            const double dx = sd ? gc[a].rhi : gc[a].rlo;
            gam = li + 2.0 * nui / fabs(dx);
          }
          gsum += gam * A;
        }
      }
      const double dt = m.cfl * V / lsum;
      double srcdiag = 0.0;
      if (nW == 6) {
        const double tau = 2.0 * m.Kn / sqrt(kPi) * pow(pi[4], m.omega - 1.0) / pi[0];
        srcdiag = 1.0 / (m.Z_r * tau);
      }
      for (int k = 0; k < nW; ++k) m.D[(size_t)c * 6 + k] = 1.0 / dt + gsum / (2.0 * V) + (k == 5 ? srcdiag : 0.0);
    }
    if (!grid_sync(m.bar, m.err)) return;
    // ---- phase 3: face fluxes (interior + faces of each cell, and wall faces)
    for (int t = tid; t < 3 * nc; t += nthr) {
      const int c = t / 3, a = t % 3;
      if (!act[a]) continue;
      int nt[3];
      G.nat(c, nt);
      if (nt[a] >= m.g.n[a] - 1) continue;
      const int j = c + cs[a];
      const AxisCell<double> gi = m.ax[a][nt[a]], gj = m.ax[a][nt[a] + 1];
      double V = 1.0;
      for (int b = 0; b < 3; ++b) V *= m.ax[b][nt[b]].h;
      const double A = V * gi.invh;
      double WL[6], WR[6], pL[6], pR[6];
      for (int k = 0; k < 6; ++k) {
        WL[k] = m.W[(size_t)c * 6 + k];
        WR[k] = m.W[(size_t)j * 6 + k];
      }
      for (int k = 0; k < nW; ++k) {
        WL[k] += m.phW[(size_t)c * 6 + k] * m.gW[((size_t)c * 6 + k) * 3 + a] * gi.rhi;
        WR[k] += m.phW[(size_t)j * 6 + k] * m.gW[((size_t)j * 6 + k) * 3 + a] * gj.rlo;
      }
      prim_of(WL, nW, m.d_r, pL);
      prim_of(WR, nW, m.d_r, pR);
      if (!(pL[0] > 0.0) || !(pL[4] > 0.0) || !(pL[5] > 0.0)) {
        for (int k = 0; k < 6; ++k) WL[k] = m.W[(size_t)c * 6 + k];
        prim_of(WL, nW, m.d_r, pL);
      }
      if (!(pR[0] > 0.0) || !(pR[4] > 0.0) || !(pR[5] > 0.0)) {
        for (int k = 0; k < 6; ++k) WR[k] = m.W[(size_t)j * 6 + k];
        prim_of(WR, nW, m.d_r, pR);
      }
      double FL[6], FR[6], F[6];
      euler_axis(WL, nW, m.d_r, a, 1.0, FL);
      euler_axis(WR, nW, m.d_r, a, 1.0, FR);
      const double lL = fabs(pL[1 + a]) + sound(pL[4]), lR = fabs(pR[1 + a]) + sound(pR[4]);
      const double lam = lL > lR ? lL : lR;
      for (int k = 0; k < 6; ++k) F[k] = k < nW ? 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (WR[k] - WL[k]) : 0.0;
      // NSF viscous and conductive flux with face gradients = mean of the cells' gradients
      double G3[3][3], gT[3], gTr[3], uf[3];
      for (int b = 0; b < 3; ++b) {
        for (int d = 0; d < 3; ++d) G3[b][d] = 0.5 * (m.gP[((size_t)c * 5 + b) * 3 + d] + m.gP[((size_t)j * 5 + b) * 3 + d]);
        gT[b] = 0.5 * (m.gP[((size_t)c * 5 + 3) * 3 + b] + m.gP[((size_t)j * 5 + 3) * 3 + b]);
        gTr[b] = 0.5 * (m.gP[((size_t)c * 5 + 4) * 3 + b] + m.gP[((size_t)j * 5 + 4) * 3 + b]);
        uf[b] = 0.5 * (m.pr[(size_t)c * 6 + 1 + b] + m.pr[(size_t)j * 6 + 1 + b]);
      }
      const double muf = 0.5 * (m.mu[c] + m.mu[j]);
      double kt, kr;
      kappas(m, muf, &kt, &kr);
      const double div = G3[0][0] + G3[1][1] + G3[2][2];
      double sn[3];
      for (int b = 0; b < 3; ++b) sn[b] = -muf * (G3[b][a] + G3[a][b] - (a == b ? 2.0 / 3.0 * div : 0.0));
      for (int b = 0; b < 3; ++b) F[1 + b] += sn[b];
      F[4] += sn[0] * uf[0] + sn[1] * uf[1] + sn[2] * uf[2] - kt * gT[a] - (nW == 6 ? kr * gTr[a] : 0.0);
      if (nW == 6) F[5] += -kr * gTr[a];
      double *Ff = m.Ffc + ((size_t)c * 3 + a) * 6;
      for (int k = 0; k < 6; ++k) Ff[k] = k < nW ? F[k] * A : 0.0;
    }
    for (int wf = tid; wf < m.nwall; wf += nthr) {
      const int c = m.wall_cell[wf], side = m.wall_side[wf], a = side / 2;
      const double sg = (side & 1) ? 1.0 : -1.0;
      int nt[3];
      G.nat(c, nt);
      double V = 1.0;
      for (int b = 0; b < 3; ++b) V *= m.ax[b][nt[b]].h;
      const double A = V * m.ax[a][nt[a]].invh;
      double feq[6];
      equilibrium_wall_flux(m, m.pr + (size_t)c * 6, a, sg, m.wall_uT + 4 * side, feq);
      for (int k = 0; k < 6; ++k) m.wfl[(size_t)wf * 6 + k] = k < nW ? feq[k] * A : 0.0;
    }
    if (!grid_sync(m.bar, m.err)) return;
    // ---- phase 4: residual.  S = sum over the cell's faces of this scheme's outward flux; the
    // high-order correction (frozen) is corr = K - S(W^{n+1/2}) with K the kinetic step's sum of
    // outward face fluxes, so R_i(W^{n+1/2}) is the kinetic step's moment residual.
    for (int c = tid; c < nc; c += nthr) {
      int nt[3];
      G.nat(c, nt);
      double V = 1.0;
      for (int b = 0; b < 3; ++b) V *= m.ax[b][nt[b]].h;
      double S[6] = {0, 0, 0, 0, 0, 0};
      for (int a = 0; a < 3; ++a) {
        if (!act[a]) continue;
        if (nt[a] < m.g.n[a] - 1)
          for (int k = 0; k < nW; ++k) S[k] += m.Ffc[((size_t)c * 3 + a) * 6 + k];
        if (nt[a] > 0)
          for (int k = 0; k < nW; ++k) S[k] -= m.Ffc[((size_t)(c - cs[a]) * 3 + a) * 6 + k];
        const int trn = a == 0 ? nt[1] + G.n1 * nt[2] : (a == 1 ? nt[0] + G.n0 * nt[2] : nt[0] + G.n0 * nt[1]);
        if (nt[a] == 0 && m.g.wall_base[2 * a] >= 0) {
          const int wid = m.g.wall_base[2 * a] + trn;
          for (int k = 0; k < nW; ++k) S[k] += m.wfl[(size_t)wid * 6 + k];
        }
        if (nt[a] == m.g.n[a] - 1 && m.g.wall_base[2 * a + 1] >= 0) {
          const int wid = m.g.wall_base[2 * a + 1] + trn;
          for (int k = 0; k < nW; ++k) S[k] += m.wfl[(size_t)wid * 6 + k];
        }
      }
      double *cr = m.corr + (size_t)c * 6;
      if (step == 0)
        for (int k = 0; k < nW; ++k) cr[k] = m.K[(size_t)c * 6 + k] - S[k];
      double R[6] = {0, 0, 0, 0, 0, 0};
      for (int k = 0; k < nW; ++k) R[k] = -(S[k] + cr[k]) / V;
      if (nW == 6) {
        const double *p = m.pr + (size_t)c * 6;
        const double tau = 2.0 * m.Kn / sqrt(kPi) * pow(p[4], m.omega - 1.0) / p[0];
        const double T = (3.0 * p[4] + m.d_r * p[5]) / (3.0 + m.d_r);
        R[5] += m.d_r * p[0] * (T - p[5]) / (4.0 * m.Z_r * tau);
      }
      for (int k = 0; k < 6; ++k) {
        m.R[(size_t)c * 6 + k] = R[k];
        m.dW[(size_t)c * 6 + k] = 0.0;
      }
    }
    if (!grid_sync(m.bar, m.err)) return;
    // ---- phase 5: red-black point-implicit sweeps
    for (int sw = 0; sw < m.sweeps; ++sw) {
      for (int col = 0; col < 2; ++col) {
        for (int c = tid; c < nc; c += nthr) {
          int nt[3];
          G.nat(c, nt);
          if (((nt[0] + nt[1] + nt[2]) & 1) != col) continue;
          double V = 1.0;
          for (int b = 0; b < 3; ++b) V *= m.ax[b][nt[b]].h;
          double acc[6];
          for (int k = 0; k < nW; ++k) acc[k] = m.R[(size_t)c * 6 + k];
          for (int a = 0; a < 3; ++a) {
            if (!act[a]) continue;
            const double A = V * m.ax[a][nt[a]].invh;
            for (int sd = 0; sd < 2; ++sd) {
              const bool inside = sd ? nt[a] < m.g.n[a] - 1 : nt[a] > 0;
              if (!inside) continue;
              const int j = c + (sd ? cs[a] : -cs[a]);
              const double sg = sd ? 1.0 : -1.0;
              const double gam = sd ? m.gam[(size_t)c * 3 + a] : m.gam[(size_t)j * 3 + a];
              double Wn[6], F1[6];
              for (int k = 0; k < 6; ++k) Wn[k] = m.W[(size_t)j * 6 + k] + m.dW[(size_t)j * 6 + k];
              euler_axis(Wn, nW, m.d_r, a, sg, F1);
              for (int k = 0; k < nW; ++k) {
                const double dF = F1[k] - sg * m.Fc[((size_t)j * 3 + a) * 6 + k];
                acc[k] -= (dF - gam * m.dW[(size_t)j * 6 + k]) * A / (2.0 * V);
              }
            }
          }
          for (int k = 0; k < nW; ++k) m.dW[(size_t)c * 6 + k] = acc[k] / m.D[(size_t)c * 6 + k];
        }
        if (!grid_sync(m.bar, m.err)) return;
      }
    }
    // ---- phase 6: update and inner residual
    double num[6] = {0, 0, 0, 0, 0, 0}, den[6] = {0, 0, 0, 0, 0, 0};
    for (int c = tid; c < nc; c += nthr) {
      int nt[3];
      G.nat(c, nt);
      double V = 1.0;
      for (int b = 0; b < 3; ++b) V *= m.ax[b][nt[b]].h;
      for (int k = 0; k < nW; ++k) {
        double &w = m.W[(size_t)c * 6 + k];
        const double d = m.dW[(size_t)c * 6 + k];
        w += d;
        if (!isfinite(w)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
        num[k] += d * d * V;
        den[k] += w * w * V;
      }
    }
    {
      __shared__ double wsum[kBlock / 32][12];
      const int nwarps = blockDim.x >> 5;
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      for (int k = 0; k < 12; ++k) {
        double v = k < 6 ? num[k] : den[k - 6];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) wsum[wid][k] = v;
      }
      __syncthreads();
      if (threadIdx.x < 12) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += wsum[w][threadIdx.x];
        m.red[(size_t)blockIdx.x * 16 + threadIdx.x] = v;
      }
    }
    if (!grid_sync(m.bar, m.err)) return;
    used = step + 1;
    // the same fixed-order sum in every block (thread 0), broadcast through shared memory
    __shared__ double sdelta;
    if (threadIdx.x == 0) {
      double tot[12];
      for (int k = 0; k < 12; ++k) tot[k] = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b)
        for (int k = 0; k < 12; ++k) tot[k] += ((volatile double *)m.red)[(size_t)b * 16 + k];
      double delta = 0.0;
      for (int k = 0; k < nW; ++k)
        if (tot[6 + k] > 0.0) {
          const double e = sqrt(tot[k] / tot[6 + k]);
          delta = e > delta ? e : delta;
        }
      sdelta = delta;
    }
    // every block has read the partials before any block overwrites them in the next step
    if (!grid_sync(m.bar, m.err)) return;
    if (sdelta < m.tol) break;
  }
  // closed domain: rescale the density to the domain's total mass (velocity, temperatures kept)
  double mloc = 0.0;
  for (int c = tid; c < nc; c += nthr) {
    int nt[3];
    G.nat(c, nt);
    double V = 1.0;
    for (int b = 0; b < 3; ++b) V *= m.ax[b][nt[b]].h;
    mloc += m.W[(size_t)c * 6] * V;
  }
  for (int o = 16; o > 0; o >>= 1) mloc += __shfl_xor_sync(0xffffffffu, mloc, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = mloc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sred[w];
    m.red[(size_t)blockIdx.x * 16] = v;
  }
  if (!grid_sync(m.bar, m.err)) return;
  __shared__ double sfac;
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) mm += ((volatile double *)m.red)[(size_t)b * 16];
    sfac = m.closed ? m.mass_ref / mm : 1.0;
  }
  __syncthreads();
  const double fac = sfac;
  for (int c = tid; c < nc; c += nthr) {
    double p[6];
    prim_of(m.W + (size_t)c * 6, nW, m.d_r, p);
    p[0] *= fac;
    for (int k = 0; k < 6; ++k) m.Wout[(size_t)c * 6 + k] = p[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *m.iters = used;
}

int macro_block_size() { return kBlock; }

// One block per SM (two when the cells do not fit in 256 threads per SM), block size the
// smallest multiple of 32 that covers the cells: FP64 on GB300 runs at 1/58 of FP32, so the
// solve is bound by FP64 issue and latency and every SM must hold cells.
cudaError_t macro_launch_shape(int nc, int *grid, int *block) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int b = 32 * ((nc + 32 * nsm - 1) / (32 * nsm));
  if (b < 32) b = 32;
  if (b > kBlock) b = kBlock;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, macro_kernel, b, 0);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  int g = nsm * (per < 2 ? per : 2);
  if (b < kBlock) g = nsm;
  const int need = (nc + b - 1) / b;
  if (g > need && need >= 1) g = need < nsm ? nsm : need;
  if (g > nc) g = nc > 0 ? nc : 1;
  *grid = g;
  *block = b;
  return cudaSuccess;
}

cudaError_t macro_max_grid(int *grid) {
  int b = 0;
  return macro_launch_shape(1 << 30, grid, &b);
}

cudaError_t launch_macro(const MacroArgs &a, int grid, int block, cudaStream_t s) {
  MacroArgs copy = a;
  void *args[] = {&copy};
  return cudaLaunchCooperativeKernel((void *)macro_kernel, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace gsis
