// macro.cu -- FP64 synthetic NSF solve of GSIS-II on sm_103a (Section 3.2 of arXiv 2310.18916).
//
// One persistent cooperative kernel runs all inner steps (Algorithm 2 body).  FP64 on GB300 is
// 1/58 of the FP32 rate and the problem has O(10^4) cells, so the solve is bound by FP64
// latency: every phase is split into many short work items (per cell and field, per face, per
// cell and neighbour) dealt out warp by warp over all SMs, and per-cell quantities every phase
// needs are computed once per inner step.
//   A (with the update)  primitives, mu, nu = mu/rho, sound speed, |u_a| + c_s, axis Euler fluxes
//   B  per (cell, field): LSQ gradients, Venkatakrishnan limiters; per cell: time step, diagonal
//   C  per face: Rusanov convective + NSF viscous flux; wall faces: equilibrium wall flux
//   D  per cell: residual R_i (Eq. delta_Macroscopic_equations)
//   E  red / black point-implicit sweeps (Eq. res_macro), one lane per (cell, neighbour)
//   F  update, inner residual, then A for the next step
// The high-order terms of Eq. full_constitutive enter through a per-cell frozen correction
// corr = K - S(W^{n+1/2}), K the kinetic step's sum of outward face fluxes and S this scheme's,
// so the residual at W^{n+1/2} is the kinetic step's moment residual.  Wall faces use the
// equilibrium wall flux of the boundary cell (its increment over the inner steps is the
// boundary-flux modification of Section 3.2; its value at W^{n+1/2} cancels in corr).
// Phases are separated by a grid barrier whose spin is bounded: on time-out it raises an error
// flag and every block returns.
#include <cuda_runtime.h>

#include <cmath>

#include "gsis_internal.h"

namespace gsis {

namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr int kBlock = 512;
constexpr long long kSpinLimit = 1LL << 31;  // ~1 s of clock64 cycles at 2 GHz
constexpr int NAUX = 8;                      // mu, nu, c_s, lam_x, lam_y, lam_z

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
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)err == 0;
}

// Work items: warp w (dealt round-robin over the blocks) takes items 32 w .. 32 w + 31.
struct Items {
  int first, stride;
  __device__ Items() {
    first = (blockIdx.x + gridDim.x * (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
    stride = gridDim.x * blockDim.x;
  }
};

__device__ __forceinline__ void nat_of(const KinGeom &g, int c, int *v) {
  v[0] = c % g.n[0];
  v[1] = (c / g.n[0]) % g.n[1];
  v[2] = c / (g.n[0] * g.n[1]);
}

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
__device__ __forceinline__ void euler_axis(const double *W, int nW, int a, double sg, double *F) {
  const double ir = 1.0 / W[0];
  const double un = sg * W[1 + a] * ir;
  const double Er = nW == 6 ? W[5] : 0.0;
  // p_t = rho Tt / 2 = (2/3) (rho E - |rho u|^2 / (2 rho) - rho E_r)
  const double pt = (2.0 / 3.0) * (W[4] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) * ir - Er);
  F[0] = W[0] * un;
  for (int b = 0; b < 3; ++b) F[1 + b] = W[1 + b] * un + (b == a ? sg * pt : 0.0);
  F[4] = (W[4] + pt) * un;
  F[5] = Er * un;
}

__device__ __forceinline__ double sound(double Tt) { return sqrt(5.0 * Tt / 6.0); }

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

__device__ __forceinline__ double cell_volume(const MacroArgs &m, const int *nt) {
  return m.ax[0][nt[0]].h * m.ax[1][nt[1]].h * m.ax[2][nt[2]].h;
}

// A: primitives and the per-cell quantities the later phases read
__device__ void cell_aux(const MacroArgs &m, int c) {
  double *p = m.pr + (size_t)c * 6;
  const double *W = m.W + (size_t)c * 6;
  prim_of(W, m.nW, m.d_r, p);
  if (!(p[0] > 0.0) || !(p[4] > 0.0) || !(p[5] > 0.0)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
  double *x = m.aux + (size_t)c * NAUX;
  const double mu = m.Kn / sqrt(kPi) * pow(p[4], m.omega);
  const double cs = sound(p[4]);
  x[0] = mu;
  x[1] = mu / p[0];
  x[2] = cs;
  for (int a = 0; a < 3; ++a) {
    x[3 + a] = fabs(p[1 + a]) + cs;
    euler_axis(W, m.nW, a, 1.0, m.Fc + ((size_t)c * 3 + a) * 6);
  }
}
}  // namespace

__global__ void __launch_bounds__(kBlock) macro_kernel(MacroArgs m) {
  const KinGeom &g = m.g;
  const int nc = g.nc, nW = m.nW;
  const Items it;
  const int cs[3] = {1, g.n[0], g.n[0] * g.n[1]};
  __shared__ double wsum[kBlock / 32][12];
  __shared__ double sdelta;

  // initial conservative state from the moments of f^{n+1/2}, then A
  for (int c = it.first; c < nc; c += it.stride) {
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
    cell_aux(m, c);
  }
  if (!grid_sync(m.bar, m.err)) return;

  const int nB = nW + 6;  // phase-B items per cell: nW limited fields, 5 primitive gradients, 1 diagonal
  const int G = 2 * g.nact <= 2 ? 2 : (2 * g.nact <= 4 ? 4 : 8);  // lanes per cell in the sweeps
  int used = 0;
  for (int step = 0; step < m.steps; ++step) {
    // ---- B: gradients and limiters per (cell, field); time step and diagonal per cell
    for (int t = it.first; t < nc * nB; t += it.stride) {
      const int c = t / nB, k = t % nB;
      int nt[3];
      nat_of(g, c, nt);
      if (k < nW + 5) {
        const bool lim = k < nW;
        const double *q = lim ? m.W + k : m.pr + 1 + (k - nW);
        const double qi = q[(size_t)c * 6];
        double gr[3] = {0, 0, 0}, qmax = qi, qmin = qi, V = 1.0;
        AxisCell<double> gc[3];
        for (int a = 0; a < 3; ++a) {
          gc[a] = m.ax[a][nt[a]];
          V *= gc[a].h;
          if (!g.act[a]) continue;
          double lo = qi, hi = qi;
          if (nt[a] > 0) { lo = q[(size_t)(c - cs[a]) * 6]; qmax = fmax(qmax, lo); qmin = fmin(qmin, lo); }
          if (nt[a] < g.n[a] - 1) { hi = q[(size_t)(c + cs[a]) * 6]; qmax = fmax(qmax, hi); qmin = fmin(qmin, hi); }
          gr[a] = gc[a].clo * (lo - qi) + gc[a].chi * (hi - qi);
        }
        if (lim) {
          // Venkatakrishnan: min over the faces (and 1) of (Dm^2 + 2 D2 Dm + e^2) / (Dm^2 + D2 Dm + 2 D2^2 + e^2),
          // compared by cross-multiplication and divided once
          const double eps2 = g.K3 * V;
          double bn = 1.0, bd = 1.0;
          for (int a = 0; a < 3; ++a) {
            if (!g.act[a]) continue;
            for (int sd = 0; sd < 2; ++sd) {
              const double d2 = gr[a] * (sd ? gc[a].rhi : gc[a].rlo);
              const double dm = d2 > 0.0 ? qmax - qi : (d2 < 0.0 ? qmin - qi : 0.0);
              const double nn = dm * dm + eps2 + 2.0 * d2 * dm, dd = dm * dm + 2.0 * d2 * d2 + dm * d2 + eps2;
              if (nn * bd < bn * dd) { bn = nn; bd = dd; }
            }
          }
          for (int a = 0; a < 3; ++a) m.gW[((size_t)c * 6 + k) * 3 + a] = gr[a];
          m.phW[(size_t)c * 6 + k] = bn / bd;
        } else {
          for (int a = 0; a < 3; ++a) m.gP[((size_t)c * 5 + (k - nW)) * 3 + a] = gr[a];
        }
      } else {
        // local time step and diagonal D_i = 1/dt_i + (1/2V_i) sum_f Gamma_f A_f (- dQ/dW)
        const double *xi = m.aux + (size_t)c * NAUX;
        const double V = cell_volume(m, nt);
        double lsum = 0.0, gsum = 0.0;
        for (int a = 0; a < 3; ++a) {
          if (!g.act[a]) continue;
          const AxisCell<double> ga = m.ax[a][nt[a]];
          const double A = V * ga.invh, li = xi[3 + a];
          for (int sd = 0; sd < 2; ++sd) {
            const bool inside = sd ? nt[a] < g.n[a] - 1 : nt[a] > 0;
            lsum += li * A;
            double gam;
            if (inside) {
              const int j = c + (sd ? cs[a] : -cs[a]);
              const double *xj = m.aux + (size_t)j * NAUX;
              const double idx = sd ? ga.pad0 : m.ax[a][nt[a] - 1].pad0;  // 1 / centre distance
              gam = fmax(li, xj[3 + a]) + 2.0 * fmax(xi[1], xj[1]) * idx;
              if (sd) m.gam[(size_t)c * 3 + a] = gam;
            } else {
              gam = li + 2.0 * xi[1] * (2.0 * ga.invh);  // wall at half a cell width
            }
            gsum += gam * A;
          }
        }
        const double inv_dt = lsum / (m.cfl * V);
        double srcdiag = 0.0;
        if (nW == 6) {
          const double *p = m.pr + (size_t)c * 6;
          const double tau = 2.0 * m.Kn / sqrt(kPi) * pow(p[4], m.omega - 1.0) / p[0];
          srcdiag = 1.0 / (m.Z_r * tau);
        }
        const double Dt = inv_dt + gsum / (2.0 * V);
        for (int q = 0; q < 6; ++q) m.invD[(size_t)c * 6 + q] = 1.0 / (Dt + (q == 5 ? srcdiag : 0.0));
      }
    }
    if (!grid_sync(m.bar, m.err)) return;
    // ---- C: interior + faces (Rusanov + NSF) and wall faces (equilibrium wall flux)
    for (int t = it.first; t < 3 * nc + m.nwall; t += it.stride) {
      if (t >= 3 * nc) {
        const int wf = t - 3 * nc;
        const int c = m.wall_cell[wf], side = m.wall_side[wf], a = side / 2;
        int nt[3];
        nat_of(g, c, nt);
        const double A = cell_volume(m, nt) * m.ax[a][nt[a]].invh;
        double feq[6];
        equilibrium_wall_flux(m, m.pr + (size_t)c * 6, a, (side & 1) ? 1.0 : -1.0, m.wall_uT + 4 * side, feq);
        for (int k = 0; k < 6; ++k) m.wfl[(size_t)wf * 6 + k] = k < nW ? feq[k] * A : 0.0;
        continue;
      }
      const int c = t / 3, a = t % 3;
      if (!g.act[a]) continue;
      int nt[3];
      nat_of(g, c, nt);
      if (nt[a] >= g.n[a] - 1) continue;
      const int j = c + cs[a];
      const AxisCell<double> gi = m.ax[a][nt[a]], gj = m.ax[a][nt[a] + 1];
      const double A = cell_volume(m, nt) * gi.invh;
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
      euler_axis(WL, nW, a, 1.0, FL);
      euler_axis(WR, nW, a, 1.0, FR);
      const double lam = fmax(fabs(pL[1 + a]) + sound(pL[4]), fabs(pR[1 + a]) + sound(pR[4]));
      for (int k = 0; k < 6; ++k) F[k] = k < nW ? 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (WR[k] - WL[k]) : 0.0;
      // NSF viscous and conductive flux, face gradients = mean of the cells' gradients
      double G3[3][3], gT[3], gTr[3], uf[3];
      for (int b = 0; b < 3; ++b) {
        for (int d = 0; d < 3; ++d) G3[b][d] = 0.5 * (m.gP[((size_t)c * 5 + b) * 3 + d] + m.gP[((size_t)j * 5 + b) * 3 + d]);
        gT[b] = 0.5 * (m.gP[((size_t)c * 5 + 3) * 3 + b] + m.gP[((size_t)j * 5 + 3) * 3 + b]);
        gTr[b] = 0.5 * (m.gP[((size_t)c * 5 + 4) * 3 + b] + m.gP[((size_t)j * 5 + 4) * 3 + b]);
        uf[b] = 0.5 * (m.pr[(size_t)c * 6 + 1 + b] + m.pr[(size_t)j * 6 + 1 + b]);
      }
      const double muf = 0.5 * (m.aux[(size_t)c * NAUX] + m.aux[(size_t)j * NAUX]);
      double kt, kr;
      kappas(m, muf, &kt, &kr);
      const double div = G3[0][0] + G3[1][1] + G3[2][2];
      double sn[3];
      for (int b = 0; b < 3; ++b) sn[b] = -muf * (G3[b][a] + G3[a][b] - (a == b ? 2.0 / 3.0 * div : 0.0));
      for (int b = 0; b < 3; ++b) F[1 + b] += sn[b];
      F[4] += sn[0] * uf[0] + sn[1] * uf[1] + sn[2] * uf[2] - kt * gT[a] - (nW == 6 ? kr * gTr[a] : 0.0);
      if (nW == 6) F[5] += -kr * gTr[a];
      double *Ff = m.Ffc + ((size_t)c * 3 + a) * 6;
      for (int k = 0; k < 6; ++k) Ff[k] = F[k] * A;
    }
    if (!grid_sync(m.bar, m.err)) return;
    // ---- D: residual.  S = sum over the cell's faces of this scheme's outward flux; the frozen
    // correction corr = K - S(W^{n+1/2}) makes R_i(W^{n+1/2}) the kinetic moment residual.
    for (int c = it.first; c < nc; c += it.stride) {
      int nt[3];
      nat_of(g, c, nt);
      const double V = cell_volume(m, nt);
      double S[6] = {0, 0, 0, 0, 0, 0};
      for (int a = 0; a < 3; ++a) {
        if (!g.act[a]) continue;
        if (nt[a] < g.n[a] - 1)
          for (int k = 0; k < nW; ++k) S[k] += m.Ffc[((size_t)c * 3 + a) * 6 + k];
        if (nt[a] > 0)
          for (int k = 0; k < nW; ++k) S[k] -= m.Ffc[((size_t)(c - cs[a]) * 3 + a) * 6 + k];
        const int trn = a == 0 ? nt[1] + g.n[1] * nt[2] : (a == 1 ? nt[0] + g.n[0] * nt[2] : nt[0] + g.n[0] * nt[1]);
        if (nt[a] == 0 && g.wall_base[2 * a] >= 0)
          for (int k = 0; k < nW; ++k) S[k] += m.wfl[(size_t)(g.wall_base[2 * a] + trn) * 6 + k];
        if (nt[a] == g.n[a] - 1 && g.wall_base[2 * a + 1] >= 0)
          for (int k = 0; k < nW; ++k) S[k] += m.wfl[(size_t)(g.wall_base[2 * a + 1] + trn) * 6 + k];
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
    // ---- E: red/black point-implicit sweeps, G lanes per cell (one per neighbour)
    for (int sw = 0; sw < m.sweeps; ++sw) {
      for (int col = 0; col < 2; ++col) {
        const int off = col ? m.ncol0 : 0, cnt = col ? nc - m.ncol0 : m.ncol0;
        // all lanes of a group loop together so the group shuffle is converged
        const int nitems = ((cnt * G + 31) / 32) * 32;
        for (int t = it.first; t < nitems; t += it.stride) {
          const int q = t / G, gl = t % G;
          const bool live = q < cnt;
          const int c = live ? m.colcells[off + q] : 0;
          double acc[6] = {0, 0, 0, 0, 0, 0};
          const int a = gl >> 1, sd = gl & 1;
          if (live && a < 3 && g.act[a]) {
            int nt[3];
            nat_of(g, c, nt);
            const bool inside = sd ? nt[a] < g.n[a] - 1 : nt[a] > 0;
            if (inside) {
              const int j = c + (sd ? cs[a] : -cs[a]);
              const double sg = sd ? 1.0 : -1.0;
              const double gam = sd ? m.gam[(size_t)c * 3 + a] : m.gam[(size_t)j * 3 + a];
              const double half_AoV = 0.5 * m.ax[a][nt[a]].invh;  // A / (2 V) on a rectilinear cell
              double Wn[6], F1[6];
              for (int k = 0; k < 6; ++k) Wn[k] = m.W[(size_t)j * 6 + k] + m.dW[(size_t)j * 6 + k];
              euler_axis(Wn, nW, a, sg, F1);
              for (int k = 0; k < nW; ++k) {
                const double dF = F1[k] - sg * m.Fc[((size_t)j * 3 + a) * 6 + k];
                acc[k] = (dF - gam * m.dW[(size_t)j * 6 + k]) * half_AoV;
              }
            }
          }
          for (int o = 1; o < G; o <<= 1)
            for (int k = 0; k < 6; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o, G);
          if (live && gl == 0)
            for (int k = 0; k < nW; ++k)
              m.dW[(size_t)c * 6 + k] = (m.R[(size_t)c * 6 + k] - acc[k]) * m.invD[(size_t)c * 6 + k];
        }
        if (!grid_sync(m.bar, m.err)) return;
      }
    }
    // ---- F: update, inner residual partials (double buffered), then A for the next step
    double num[6] = {0, 0, 0, 0, 0, 0}, den[6] = {0, 0, 0, 0, 0, 0};
    for (int c = it.first; c < nc; c += it.stride) {
      int nt[3];
      nat_of(g, c, nt);
      const double V = cell_volume(m, nt);
      for (int k = 0; k < nW; ++k) {
        double &w = m.W[(size_t)c * 6 + k];
        const double d = m.dW[(size_t)c * 6 + k];
        w += d;
        if (!isfinite(w)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
        num[k] += d * d * V;
        den[k] += w * w * V;
      }
      cell_aux(m, c);
    }
    double *red = m.red + (size_t)(step & 1) * gridDim.x * 16;
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
      for (int k = 0; k < 12; ++k) {
        double v = k < 6 ? num[k] : den[k - 6];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) wsum[wid][k] = v;
      }
      __syncthreads();
      if (threadIdx.x < 12) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += wsum[w][threadIdx.x];
        red[(size_t)blockIdx.x * 16 + threadIdx.x] = v;
      }
    }
    if (!grid_sync(m.bar, m.err)) return;
    used = step + 1;
    // the same fixed-order sum in every block; the partials of this step are not overwritten
    // before two more barriers, so no barrier is needed after reading them
    if (threadIdx.x == 0) {
      double tot[12];
      for (int k = 0; k < 12; ++k) tot[k] = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b)
        for (int k = 0; k < 12; ++k) tot[k] += ((volatile double *)red)[(size_t)b * 16 + k];
      double delta = 0.0;
      for (int k = 0; k < nW; ++k)
        if (tot[6 + k] > 0.0) delta = fmax(delta, sqrt(tot[k] / tot[6 + k]));
      sdelta = delta;
    }
    __syncthreads();
    if (sdelta < m.tol) break;
  }
  // closed domain: rescale the density to the domain's total mass (velocity, temperatures kept)
  if (!grid_sync(m.bar, m.err)) return;
  double mloc = 0.0;
  for (int c = it.first; c < nc; c += it.stride) {
    int nt[3];
    nat_of(g, c, nt);
    mloc += m.W[(size_t)c * 6] * cell_volume(m, nt);
  }
  for (int o = 16; o > 0; o >>= 1) mloc += __shfl_xor_sync(0xffffffffu, mloc, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5][0] = mloc;
  __syncthreads();
  double *red = m.red + (size_t)2 * gridDim.x * 16;
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += wsum[w][0];
    red[blockIdx.x] = v;
  }
  if (!grid_sync(m.bar, m.err)) return;
  __shared__ double sfac;
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) mm += ((volatile double *)red)[b];
    sfac = m.closed ? m.mass_ref / mm : 1.0;
  }
  __syncthreads();
  const double fac = sfac;
  for (int c = it.first; c < nc; c += it.stride) {
    double p[6];
    prim_of(m.W + (size_t)c * 6, nW, m.d_r, p);
    p[0] *= fac;
    for (int k = 0; k < 6; ++k) m.Wout[(size_t)c * 6 + k] = p[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *m.iters = used;
}

int macro_block_size() { return kBlock; }

// One block of 512 threads per SM: the phases have many short FP64 work items and every SM
// must hold some.  The cooperative launch guarantees the blocks are co-resident.
cudaError_t macro_launch_shape(int nc, int *grid, int *block) {
  (void)nc;
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, macro_kernel, kBlock, 0);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  *grid = nsm;
  *block = kBlock;
  return cudaSuccess;
}

cudaError_t macro_max_grid(int *grid) {
  int b = 0;
  return macro_launch_shape(0, grid, &b);
}

cudaError_t launch_macro(const MacroArgs &a, int grid, int block, cudaStream_t s) {
  MacroArgs copy = a;
  void *args[] = {&copy};
  return cudaLaunchCooperativeKernel((void *)macro_kernel, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace gsis
