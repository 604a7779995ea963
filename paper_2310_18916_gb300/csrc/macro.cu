// macro.cu -- FP64 synthetic NSF solve of GSIS-II on sm_103a (Section 3.3 of arXiv 2310.18916).
//
// One persistent cooperative kernel runs all inner steps (Algorithm 2 body).  FP64 on GB300 is
// 1/58 of the FP32 rate and the problem has O(10^4) cells, so the solve is bound by FP64
// latency: every phase is split into many short work items (per cell and field, per face, per
// cell and face) dealt out warp by warp over all SMs, and per-cell quantities every phase
// needs are computed once per inner step.  Per inner step:
//   B  per (cell, field): LSQ gradients, Venkatakrishnan limiters; per cell: time step, diagonal
//   C  per face: Rusanov convective + NSF viscous flux; wall faces: equilibrium wall flux
//   E  red / black point-implicit sweeps (Eq. res_macro), two lanes per cell.  A cell
//      updated in a pass evaluates its own axis-flux increments F(W + dW) - F(W) once, for the
//      other colour's next pass.  The first pass of each colour also sums the cell's face fluxes
//      into the residual R_i (Eq. delta_Macroscopic_equations); the last one applies the update
//      W += dW, adds to the inner residual and recomputes the cell's primitives, mu, nu, sound
//      speed, |u_a| + c_s and axis Euler fluxes (into the second of two flux buffers: the other
//      colour still reads the fluxes at the start of the step)
// so ten grid barriers per inner step with the default four sweeps.
// The high-order terms of Eq. full_constitutive enter through a per-cell frozen correction
// corr = K - S(W^{n+1/2}), K the kinetic step's sum of outward face fluxes and S this scheme's,
// so the residual at W^{n+1/2} is the kinetic step's moment residual.  Wall faces use the
// equilibrium wall flux of the boundary cell (its increment over the inner steps is the
// boundary-flux modification of Section 3.3; its value at W^{n+1/2} cancels in corr).
// Phases are separated by a grid barrier whose spin is bounded: on time-out it raises an error
// flag and every block returns.
// Per-cell arrays are indexed only by compile-time constants (the field count NW is a template
// parameter, per-axis values are selected, not indexed), so they stay in registers.
#include <cuda_runtime.h>

#include <cmath>

#include "gsis_internal.h"
#include "wall_flux.cuh"

namespace gsis {

namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr int kBlock = 512;
constexpr long long kSpinLimit = 1LL << 31;  // ~1 s of clock64 cycles at 2 GHz
constexpr int NAUX = 8;                      // mu, nu, c_s, lam_x, lam_y, lam_z

constexpr int kBarGroups = 8, kBarStride = 32;  // arrival counters, 128 bytes apart
constexpr int kListCap = 2048;                  // cells per block and last pass evaluated compacted
constexpr size_t kResidualSmem = 12 * kBlock * sizeof(double);  // per-thread inner-residual partials
static_assert(kBarGroups * kBarStride <= MACRO_BAR_WORDS, "barrier words");

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned x) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

// Grid barrier on kBarGroups monotonic arrival counters, each in its own 128-byte line and zero
// at launch.  Block b adds 1 to counter b % kBarGroups with release semantics (publishing the
// block's writes); thread g < kBarGroups of every block waits, with acquire loads, until counter
// g has reached the barrier's epoch (1, 2, ...) times its group size.  Spreading the arrivals
// keeps same-address atomics from serialising on one line.  The spin is bounded: on time-out
// it raises the error flag.  Returns false when any block has flagged an error, so every caller
// leaves the kernel together.
__device__ bool grid_sync(unsigned *bar, unsigned &epoch, int *err, long long limit = kSpinLimit) {
  ++epoch;
  __syncthreads();
  if (threadIdx.x == 0) red_release_add(bar + kBarStride * (blockIdx.x % kBarGroups), 1u);
  if (threadIdx.x < kBarGroups) {
    const unsigned g = threadIdx.x, gsize = (gridDim.x - g + kBarGroups - 1) / kBarGroups;
    const unsigned target = epoch * gsize;
    const long long t0 = clock64();
    for (unsigned i = 0; ld_acquire(bar + kBarStride * g) < target; ++i) {
      if ((i & 15u) == 15u && (clock64() - t0 > limit || *(volatile int *)err != 0)) {
        atomicCAS(err, 0, GSIS_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
  return *(volatile int *)err == 0;
}

// Warp sums of v[0..15] by recursive halving: at each level a lane keeps the half of its vector
// selected by one bit of its lane index and adds the partner's copy of that half (16 adds instead
// of 80).  Afterwards lanes 2i and 2i + 1 hold the warp total of v[i].
__device__ __forceinline__ double transpose_sum16(double *v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 16, n = 8; h > 1; h >>= 1, n >>= 1) {
    const bool up = lane & h;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const double send = up ? v[i] : v[i + n];
      const double keep = up ? v[i + n] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Work items: warp w (dealt round-robin over the blocks) takes items 32 w .. 32 w + 31.
struct Items {
  int first, stride;
  __device__ Items() {
    first = (blockIdx.x + gridDim.x * (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
    stride = gridDim.x * blockDim.x;
  }
};

template <typename T>
__device__ __forceinline__ T pick3(int a, T x, T y, T z) { return a == 0 ? x : (a == 1 ? y : z); }

__device__ __forceinline__ void nat_of(const KinGeom &g, int c, int *v) {
  v[0] = c % g.n[0];
  v[1] = (c / g.n[0]) % g.n[1];
  v[2] = c / (g.n[0] * g.n[1]);
}

// primitives (rho, u, Tt, Tr) of the conservative state W; returns 1 / rho
template <int NW>
__device__ __forceinline__ double prim_of(const double *W, double dr, double *p) {
  const double rho = W[0], ir = __drcp_rn(rho);  // = 1.0 / rho, correctly rounded
  const double ux = W[1] * ir, uy = W[2] * ir, uz = W[3] * ir;
  const double Er = NW == 6 ? W[5] : 0.0;
  const double Tt = (W[4] - 0.5 * rho * (ux * ux + uy * uy + uz * uz) - Er) * (ir * (4.0 / 3.0));
  p[0] = rho;
  p[1] = ux;
  p[2] = uy;
  p[3] = uz;
  p[4] = Tt;
  p[5] = NW == 6 ? Er * ir * (4.0 / dr) : Tt;
  return ir;
}

// FP64 comparisons, min and max run at the FP64 rate on this GPU (a warp instruction holds a
// sub-partition's FP64 pipe for ~64 cycles, like an FMA).  Where the operands are known to be
// non-negative, the order of their bit patterns as integers is their numeric order, so these take
// the integer pipes and give the same results (no NaN reaches them on a physical state).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// x > 0 exactly as the FP64 comparison: +0 < bits <= +inf (negative values, -0 and NaN fail)
__device__ __forceinline__ bool gt0(double x) {
  return (unsigned long long)(dbits(x) - 1) < 0x7ff0000000000000ULL;
}
// x < y and max(x, y) for x, y >= 0
__device__ __forceinline__ bool lt_nn(double x, double y) { return dbits(x) < dbits(y); }
__device__ __forceinline__ double max_nn(double x, double y) { return dbits(x) < dbits(y) ? y : x; }

__device__ __forceinline__ bool physical(const double *p) { return gt0(p[0]) && gt0(p[4]) && gt0(p[5]); }

// Euler flux along n = sg e_a: (rho u_n, rho u u_n + p_t n, (rho E + p_t) u_n, rho E_r u_n)
template <int NW>
__device__ __forceinline__ void euler_axis(const double *W, int a, double sg, double *F) {
  const double ir = __drcp_rn(W[0]);
  const double un = sg * pick3(a, W[1], W[2], W[3]) * ir;
  const double Er = NW == 6 ? W[5] : 0.0;
  // p_t = rho Tt / 2 = (2/3) (rho E - |rho u|^2 / (2 rho) - rho E_r)
  const double pt = (2.0 / 3.0) * (W[4] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) * ir - Er);
  F[0] = W[0] * un;
#pragma unroll
  for (int b = 0; b < 3; ++b) F[1 + b] = W[1 + b] * un + (b == a ? sg * pt : 0.0);
  F[4] = (W[4] + pt) * un;
  F[5] = Er * un;
}

// The same flux from W and its primitives p (no division): u_n = u_a, p_t = rho Tt / 2
template <int NW>
__device__ __forceinline__ void euler_axis_prim(const double *W, const double *p, int a, double *F) {
  const double un = pick3(a, p[1], p[2], p[3]);
  const double pt = 0.5 * p[0] * p[4];
  F[0] = W[0] * un;
#pragma unroll
  for (int b = 0; b < 3; ++b) F[1 + b] = W[1 + b] * un + (b == a ? pt : 0.0);
  F[4] = (W[4] + pt) * un;
  F[5] = (NW == 6 ? W[5] : 0.0) * un;
}

__device__ __forceinline__ double sound(double Tt) { return sqrt(Tt * (5.0 / 6.0)); }

// Venkatakrishnan face function of the two faces of one axis, r_lo < 0 < r_hi.  The increment
// D2 = g r of the face where it is positive meets the bound dp = qmax - qi, the other face dn =
// qmin - qi.  As a function of y = Dm / D2 >= 0, (y^2 + 2y + E) / (y^2 + y + 2 + E) with E =
// e^2 / D2^2 (the same on both faces, |r_lo| = |r_hi|) rises while y < 2 + sqrt(8 + E) and
// exceeds 1 exactly when y > 2, so the minimum of the two faces and 1 is the face with the
// smaller y (up to rounding).  Returns that face's numerator and denominator.
__device__ __forceinline__ void venkat_axis(double g, double rlo, double rhi, double dp, double dn, double eps2,
                                            double &nn, double &dd) {
  const double dh = g * rhi, dl = g * rlo;
  const bool pos = gt0(g);
  const double mh = pos ? dp : dn, ml = pos ? dn : dp;
  const bool hi = !lt_nn(fabs(ml) * fabs(dh), fabs(mh) * fabs(dl));
  // (g = 0: D2 = 0 and the face value is 1, which never lowers the minimum)
  const double d2 = hi ? dh : dl, dm = hi ? mh : ml;
  const double dm2 = fma(dm, dm, eps2);
  nn = fma(2.0 * d2, dm, dm2);
  dd = fma(d2, fma(2.0, d2, dm), dm2);
}

// T^e for T > 0 as exp(e log T)
__device__ __forceinline__ double power(double T, double e) { return exp(e * log(T)); }

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
template <int NW>
__device__ void equilibrium_wall_flux(const MacroArgs &m, const double *p, int a, double sg, const double *uT,
                                      double *F) {
  const double rho = p[0], T = p[4], un = sg * pick3(a, p[1], p[2], p[3]), Tw = uT[3];
  const double sr = un / sqrt(T);
  const double phi0 = exp(-sr * sr) / sqrt(kPi * T);
  const double J0 = 0.5 * erfc(-sr);
  const double J1 = un * J0 + 0.5 * T * phi0;
  const double J2 = un * J1 + 0.5 * T * J0;
  const double J3 = un * J2 + T * J1;
  const double K1 = -sqrt(Tw) / (2.0 * sqrt(kPi)), K2 = Tw / 4.0, K3 = Tw * K1;
  const double rw = -rho * J1 / K1;
  double ut[3], uwt[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    ut[b] = b == a ? 0.0 : p[1 + b];
    uwt[b] = b == a ? 0.0 : uT[b];
  }
  const double ut2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  const double uw2 = uwt[0] * uwt[0] + uwt[1] * uwt[1] + uwt[2] * uwt[2];
  F[0] = rho * J1 + rw * K1;
#pragma unroll
  for (int b = 0; b < 3; ++b) F[1 + b] = (b == a ? sg : 0.0) * (rho * J2 + rw * K2) + rho * J1 * ut[b] + rw * K1 * uwt[b];
  const double rin = NW == 6 ? m.d_r * p[5] / 4.0 * rho * J1 : 0.0;
  const double rout = NW == 6 ? m.d_r * Tw / 4.0 * rw * K1 : 0.0;
  F[4] = 0.5 * rho * (J3 + J1 * (ut2 + T)) + 0.5 * rw * (K3 + K1 * (uw2 + Tw)) + rin + rout;
  F[5] = rin + rout;
}

__device__ __forceinline__ double cell_volume(const MacroArgs &m, const int *nt) {
  return m.ax[0][nt[0]].h * m.ax[1][nt[1]].h * m.ax[2][nt[2]].h;
}

__device__ __forceinline__ double cell_inv_volume(const MacroArgs &m, const int *nt) {
  return m.ax[0][nt[0]].invh * m.ax[1][nt[1]].invh * m.ax[2][nt[2]].invh;
}

__device__ __forceinline__ const AxisCell<double> *axis_cells(const MacroArgs &m, int a) {
  return pick3(a, m.ax[0], m.ax[1], m.ax[2]);
}

// Primitives and the per-cell quantities the later phases read (everything but the fluxes)
template <int NW>
__device__ void cell_prims(const MacroArgs &m, int c, const double *W) {
  double p[6];
  const double ir = prim_of<NW>(W, m.d_r, p);
  if (!physical(p)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
#pragma unroll
  for (int k = 0; k < 6; ++k) m.pr[(size_t)c * 6 + k] = p[k];
  double *x = m.aux + (size_t)c * NAUX;
  const double mu = m.mu0 * power(p[4], m.omega);
  const double cs = sound(p[4]);
  x[0] = mu;
  x[1] = mu * ir;
  x[2] = cs;
  x[3] = fabs(p[1]) + cs;
  x[4] = fabs(p[2]) + cs;
  x[5] = fabs(p[3]) + cs;
}

// B, one cell's limited fields: LSQ gradients of the conservative fields k < NW with their
// Venkatakrishnan limiters.  The neighbours' rows are read once for all fields (a missing
// neighbour reads the cell's own row: difference +0).
template <int NW, int MA>
__device__ void limited_cell(const MacroArgs &m, const int *cs, int c) {
  const KinGeom &g = m.g;
  int nt[3];
  nat_of(g, c, nt);
  AxisCell<double> gc[3];
  double V = 1.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gc[a] = m.ax[a][nt[a]];
    V *= gc[a].h;
  }
  const double eps2 = g.K3 * V;
  const double *Wc = m.W + (size_t)c * 6;
  const double *Wlo[MA], *Whi[MA];
#pragma unroll
  for (int a = 0; a < MA; ++a) {
    const bool act = a < g.nact;
    Wlo[a] = act && nt[a] > 0 ? m.W + (size_t)(c - cs[a]) * 6 : Wc;
    Whi[a] = act && nt[a] < g.n[a] - 1 ? m.W + (size_t)(c + cs[a]) * 6 : Wc;
  }
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const double qi = Wc[k];
    double gr[3] = {0, 0, 0};
    // bounds qmax - qi, qmin - qi as the largest positive and negative neighbour difference
    // (rounding is monotonic, so max fl(q - qi) = fl(max q - qi)): bit patterns of the positive
    // differences and magnitudes of the negative ones, compared as integers
    long long pbits = 0, nmag = 0;
#pragma unroll
    for (int a = 0; a < MA; ++a) {
      if (a >= g.nact) continue;
      const double dlo = Wlo[a][k] - qi, dhi = Whi[a][k] - qi;
      gr[a] = gc[a].clo * dlo + gc[a].chi * dhi;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const long long b = dbits(e ? dhi : dlo), mag = b & 0x7fffffffffffffffLL;
        pbits = b > pbits ? b : pbits;
        nmag = b < 0 && mag > nmag ? mag : nmag;
      }
    }
    // Venkatakrishnan: min over the faces (and 1) of (Dm^2 + 2 D2 Dm + e^2) / (Dm^2 + D2 Dm + 2 D2^2 + e^2),
    // one face per axis (the one with the smaller |Dm| / |D2|), compared by cross-multiplication
    // and divided once
    const double dp = __longlong_as_double(pbits);
    const double dn = nmag ? __longlong_as_double(nmag | (long long)0x8000000000000000ULL) : 0.0;
    double bn = 1.0, bd = 1.0;
#pragma unroll
    for (int a = 0; a < MA; ++a) {
      if (a >= g.nact) continue;
      double nn, dd;
      venkat_axis(gr[a], gc[a].rlo, gc[a].rhi, dp, dn, eps2, nn, dd);
      if (lt_nn(nn * bd, bn * dd)) { bn = nn; bd = dd; }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) m.gW[((size_t)c * 6 + k) * 3 + a] = gr[a];
    m.phW[(size_t)c * 6 + k] = bn / bd;
  }
}

// B, one cell's primitive gradients (u, T_t and for Rykov T_r: the NSF stress and heat flux) and
// its local time step and diagonal D_i = 1/dt_i + (1/2V_i) sum_f Gamma_f A_f (- dQ/dW)
template <int NW, int MA>
__device__ void prim_cell(const MacroArgs &m, const int *cs, double inv_cfl, int c) {
  const KinGeom &g = m.g;
  int nt[3];
  nat_of(g, c, nt);
  constexpr int NP = NW == 6 ? 5 : 4;  // Shakhov: T_r = T_t, whose gradient is not taken twice
  const double *pc = m.pr + (size_t)c * 6;
  AxisCell<double> gc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gc[a] = m.ax[a][nt[a]];
  const double *plo[MA], *phi_[MA];
#pragma unroll
  for (int a = 0; a < MA; ++a) {
    const bool act = a < g.nact;
    plo[a] = act && nt[a] > 0 ? m.pr + (size_t)(c - cs[a]) * 6 : pc;
    phi_[a] = act && nt[a] < g.n[a] - 1 ? m.pr + (size_t)(c + cs[a]) * 6 : pc;
  }
#pragma unroll
  for (int f = 0; f < NP; ++f) {
    const double qi = pc[1 + f];
    double gr[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < MA; ++a) {
      if (a >= g.nact) continue;
      gr[a] = gc[a].clo * (plo[a][1 + f] - qi) + gc[a].chi * (phi_[a][1 + f] - qi);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) m.gP[((size_t)c * 5 + f) * 3 + a] = gr[a];
  }
  const double *xi = m.aux + (size_t)c * NAUX;
  const double V = gc[0].h * gc[1].h * gc[2].h, iV = gc[0].invh * gc[1].invh * gc[2].invh;
  double lsum = 0.0, gsum = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!g.act[a]) continue;
    const AxisCell<double> ga = gc[a];
    const double A = V * ga.invh, li = xi[3 + a];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const bool inside = sd ? nt[a] < g.n[a] - 1 : nt[a] > 0;
      lsum += li * A;
      double gam;
      if (inside) {
        const int j = c + (sd ? cs[a] : -cs[a]);
        const double *xj = m.aux + (size_t)j * NAUX;
        const double idx = sd ? ga.pad0 : m.ax[a][nt[a] - 1].pad0;  // 1 / centre distance
        gam = max_nn(li, xj[3 + a]) + 2.0 * max_nn(xi[1], xj[1]) * idx;
        if (sd) m.gam[(size_t)c * 3 + a] = gam;
      } else {
        gam = li + 2.0 * xi[1] * (2.0 * ga.invh);  // wall at half a cell width
      }
      gsum += gam * A;
    }
  }
  const double inv_dt = lsum * iV * inv_cfl;
  double srcdiag = 0.0;
  if (NW == 6) {
    const double tau = 2.0 * m.mu0 * power(pc[4], m.omega - 1.0) / pc[0];
    srcdiag = 1.0 / (m.Z_r * tau);
  }
  const double Dt = inv_dt + gsum * 0.5 * iV, iD = __drcp_rn(Dt);
#pragma unroll
  for (int q = 0; q < 5; ++q) m.invD[(size_t)c * 6 + q] = iD;
  m.invD[(size_t)c * 6 + 5] = NW == 6 ? 1.0 / (Dt + srcdiag) : iD;
}

// C, one item: Rusanov convective + NSF viscous flux (area-integrated) through the + face of
// cell c along axis a, from the limited linear reconstructions of both sides.
template <int NW>
__device__ void face_item(const MacroArgs &m, const int *cs, int c, int a) {
  const KinGeom &g = m.g;
  int nt[3];
  nat_of(g, c, nt);
  const int na = pick3(a, nt[0], nt[1], nt[2]);
  if (na >= pick3(a, g.n[0], g.n[1], g.n[2]) - 1) return;
  const int j = c + pick3(a, cs[0], cs[1], cs[2]);
  const AxisCell<double> *axa = axis_cells(m, a);
  const double rhi = axa[na].rhi, rlo = axa[na + 1].rlo;
  // face area: the product of the cell's widths along the two other axes
  const double h0 = m.ax[0][nt[0]].h, h1 = m.ax[1][nt[1]].h, h2 = m.ax[2][nt[2]].h;
  const double A = a == 0 ? h1 * h2 : (a == 1 ? h0 * h2 : h0 * h1);
  double WL[6], WR[6], pL[6], pR[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    WL[k] = m.W[(size_t)c * 6 + k];
    WR[k] = m.W[(size_t)j * 6 + k];
  }
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    WL[k] += m.phW[(size_t)c * 6 + k] * m.gW[((size_t)c * 6 + k) * 3 + a] * rhi;
    WR[k] += m.phW[(size_t)j * 6 + k] * m.gW[((size_t)j * 6 + k) * 3 + a] * rlo;
  }
  prim_of<NW>(WL, m.d_r, pL);
  prim_of<NW>(WR, m.d_r, pR);
  if (!physical(pL)) {
#pragma unroll
    for (int k = 0; k < 6; ++k) WL[k] = m.W[(size_t)c * 6 + k];
    prim_of<NW>(WL, m.d_r, pL);
  }
  if (!physical(pR)) {
#pragma unroll
    for (int k = 0; k < 6; ++k) WR[k] = m.W[(size_t)j * 6 + k];
    prim_of<NW>(WR, m.d_r, pR);
  }
  double FL[6], FR[6], F[6];
  euler_axis_prim<NW>(WL, pL, a, FL);
  euler_axis_prim<NW>(WR, pR, a, FR);
  const double lam = max_nn(fabs(pick3(a, pL[1], pL[2], pL[3])) + sound(pL[4]),
                            fabs(pick3(a, pR[1], pR[2], pR[3])) + sound(pR[4]));
  // area-integrated Rusanov flux (A/2) [F_L + F_R - lam (W_R - W_L)]
  const double hA = 0.5 * A;
#pragma unroll
  for (int k = 0; k < 6; ++k) F[k] = k < NW ? hA * fma(-lam, WR[k] - WL[k], FL[k] + FR[k]) : 0.0;
  // NSF viscous and conductive flux with the face gradients, velocity and viscosity the means of
  // the two cells' values: the sums are taken here and the halves folded into q = A mu_f / 2
  // (stress -mu_f (G + G^T - 2/3 div G) with G = S / 2) and the conductivities (linear in mu)
  const double *gPc = m.gP + (size_t)c * 15, *gPj = m.gP + (size_t)j * 15;
  double S3[3][3], us[3];  // S3[b][d] = sum of the cells' d u_b / dx_d
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int d = 0; d < 3; ++d) S3[b][d] = gPc[b * 3 + d] + gPj[b * 3 + d];
    us[b] = m.pr[(size_t)c * 6 + 1 + b] + m.pr[(size_t)j * 6 + 1 + b];
  }
  const double gTs = gPc[9 + a] + gPj[9 + a];
  const double gTrs = NW == 6 ? gPc[12 + a] + gPj[12 + a] : 0.0;
  const double q = 0.25 * A * (m.aux[(size_t)c * NAUX] + m.aux[(size_t)j * NAUX]);
  double qt, qr;  // conductivities at viscosity q: the heat fluxes' coefficients of the gradient sums
  kappas(m, q, &qt, &qr);
  const double divs = S3[0][0] + S3[1][1] + S3[2][2];
  double sn[3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
    sn[b] = -q * (pick3(a, S3[b][0], S3[b][1], S3[b][2]) + pick3(a, S3[0][b], S3[1][b], S3[2][b]) -
                  (a == b ? (2.0 / 3.0) * divs : 0.0));
#pragma unroll
  for (int b = 0; b < 3; ++b) F[1 + b] += sn[b];
  F[4] += fma(0.5, sn[0] * us[0] + sn[1] * us[1] + sn[2] * us[2], -qt * gTs) - (NW == 6 ? qr * gTrs : 0.0);
  if (NW == 6) F[5] += -qr * gTrs;
  double *Ff = m.Ffc + ((size_t)c * 3 + a) * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) Ff[k] = F[k];
}

// C, one wall item: the model wall flux (area-integrated) of wall face wf: local equilibrium or
// the Grad-13 VDF with the kinetic step's stress and heat fluxes
template <int NW>
__device__ void wall_item(const MacroArgs &m, int wf) {
  const int c = m.wall_cell[wf], side = m.wall_side[wf], a = side / 2;
  int nt[3];
  nat_of(m.g, c, nt);
  const double A = cell_volume(m, nt) * axis_cells(m, a)[pick3(a, nt[0], nt[1], nt[2])].invh;
  double p[6], feq[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = m.pr[(size_t)c * 6 + k];
  const double sg = (side & 1) ? 1.0 : -1.0;
  if (m.wall_g13) {
    const double n[3] = {a == 0 ? sg : 0.0, a == 1 ? sg : 0.0, a == 2 ? sg : 0.0};
    const double *M = m.Mh + (size_t)c * 18;
    grad13_wall_flux(NW, m.d_r, p[0], p + 1, p[4], p[5], n, M + 6, M + 12, M + 15, m.wall_uT + 4 * side,
                     m.wall_uT[4 * side + 3], feq);
  } else {
    equilibrium_wall_flux<NW>(m, p, a, sg, m.wall_uT + 4 * side, feq);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) m.wfl[(size_t)wf * 6 + k] = k < NW ? feq[k] * A : 0.0;
}

// E, publishing.  A cell updated in a pass writes, for each of its axes a, the two off-diagonal
// terms its neighbours along a read in the other colour's next pass: the upper neighbour (face
// on its low side) reads -dF - Gamma_hi dW, the lower one (face on its high side) +dF - Gamma_lo dW,
// dF = F_a(W + dW) - F_a(W) and Gamma of the face in question.  A reader then needs one
// five-vector per face, scaled by A / (2V).
template <int NW>
__device__ __forceinline__ void publish_terms(const MacroArgs &m, int c, int a, const double *dF, const double *d,
                                              double gam_lo, double gam_hi) {
  double *G = m.G + ((size_t)c * 3 + a) * 12;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    G[k] = fma(-gam_hi, d[k], -dF[k]);
    G[6 + k] = fma(-gam_lo, d[k], dF[k]);
  }
}

// Gamma of the faces below and above cell c along axis a (zero where the face is a boundary)
__device__ __forceinline__ void face_gammas(const MacroArgs &m, int c, int csa, int na, int n, int a, double &lo,
                                            double &hi) {
  lo = na > 0 ? m.gam[(size_t)(c - csa) * 3 + a] : 0.0;
  hi = na < n - 1 ? m.gam[(size_t)c * 3 + a] : 0.0;
}
}  // namespace

// NW conservative fields (5 Shakhov, 6 Rykov); MA >= the active axis count bounds the per-face
// registers of the sweeps (2 for 1D and 2D meshes, 3 for 3D).
template <int NW, int MA>
__global__ void __launch_bounds__(kBlock) macro_kernel(MacroArgs m) {
  const KinGeom &g = m.g;
  const int nc = g.nc, nact = g.nact;
  const Items it;
  const int cs[3] = {1, g.n[0], g.n[0] * g.n[1]};
  const double inv_cfl = 1.0 / m.cfl;
  unsigned ep = 0;  // grid barriers passed
  static_assert(kBlock >= 12 * 32, "one warp per reduced field");
  __shared__ double wsum[kBlock / 32][12];
  __shared__ int sdone;
  // cells this block updated in a last pass, for the compacted evaluation of their primitives
  // and fluxes (overflow entries are evaluated in place)
  __shared__ int slist[kListCap];
  extern __shared__ double rsd[];  // [12][kBlock] inner-residual partials, value-major
  __shared__ int scount;
  if (threadIdx.x == 0) scount = 0;

  // initial conservative state from the moments of f^{n+1/2}, its primitives and axis fluxes
  for (int c = it.first; c < nc; c += it.stride) {
    const double *M = m.Mh + (size_t)c * 18;
    double W[6];
    const double rho = M[0];
    W[0] = rho;
    W[1] = rho * M[1];
    W[2] = rho * M[2];
    W[3] = rho * M[3];
    const double Er = NW == 6 ? m.d_r * rho * M[5] / 4.0 : 0.0;
    W[4] = 0.5 * rho * (M[1] * M[1] + M[2] * M[2] + M[3] * M[3]) + 0.75 * rho * M[4] + Er;
    W[5] = Er;
#pragma unroll
    for (int k = 0; k < 6; ++k) m.W[(size_t)c * 6 + k] = W[k];
    cell_prims<NW>(m, c, W);
    for (int a = 0; a < nact; ++a) euler_axis<NW>(W, a, 1.0, m.Fc + ((size_t)c * 3 + a) * 6);
  }
  if (!grid_sync(m.bar, ep, m.err)) return;

  // the cell of this thread's first sweep item in each colour (the items are the same every pass)
  const int cell0 = it.first >> 1 < m.ncol0 ? m.colcells[it.first >> 1] : 0;
  const int cell1 = it.first >> 1 < nc - m.ncol0 ? m.colcells[m.ncol0 + (it.first >> 1)] : 0;
  int used = 0;
  for (int step = 0; step < m.steps; ++step) {
    // axis fluxes at the start of this step, and the buffer for those at its end
    const double *Fc = m.Fc + (size_t)(step & 1) * nc * 18;
    double *Fn = m.Fc + (size_t)((step + 1) & 1) * nc * 18;
    // the previous step's inner residual: block k < 12 sums value k (num_k, den_k) of the
    // blocks' partials in fixed order; every block tests them during C
    const bool check = m.tol > 0.0 && step > 0;
    if (check && blockIdx.x < 12 && (threadIdx.x >> 5) == kBlock / 32 - 1) {
      // (the block's last warp, the last one dealt B items)
      const double *red = m.red + (size_t)((step - 1) & 1) * gridDim.x * 16;
      const int lane = threadIdx.x & 31;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < MACRO_MAX_GRID / 32; ++i) {
        const int b = lane + 32 * i;
        if (b < (int)gridDim.x) v += __ldcg(red + (size_t)b * 16 + blockIdx.x);
      }
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) m.red[(size_t)3 * gridDim.x * 16 + ((step - 1) & 1) * 16 + blockIdx.x] = v;
    }
    // ---- B: per cell, the limited fields' gradients and limiters (items [0, nc)), then the
    // primitive gradients, time step and diagonal (items [nc, 2 nc)): one round of items over
    // the GPU, each reading its neighbours' rows once
    for (int t = it.first; t < 2 * nc; t += it.stride) {
      if (t < nc)
        limited_cell<NW, MA>(m, cs, t);
      else
        prim_cell<NW, MA>(m, cs, inv_cfl, t - nc);
    }
    if (!grid_sync(m.bar, ep, m.err)) return;
    // ---- C: interior + faces of the active axes, then the wall faces.  Warp 0 loads the
    // residual sums before its items and tests them after: stop when max_k sqrt(num_k / den_k) <
    // tol, tested as num_k < tol^2 den_k (the state is still that of the previous step's end)
    double rsum = 0.0;
    if (check && threadIdx.x < 12) rsum = __ldcg(m.red + (size_t)3 * gridDim.x * 16 + ((step - 1) & 1) * 16 + threadIdx.x);
    for (int t = it.first; t < nact * nc + m.nwall; t += it.stride) {
      if (t >= nact * nc)
        wall_item<NW>(m, t - nact * nc);
      else
        face_item<NW>(m, cs, t / nact, t % nact);
    }
    if (check && threadIdx.x < 32) {
      const int k = threadIdx.x;
      const double den = __shfl_sync(0xffffffffu, rsum, (k + 6) & 31);
      bool done = !(k < NW && den > m.den_floor && !(rsum < m.tol * m.tol * den));
      done = __all_sync(0xffffffffu, done);
      if (k == 0) sdone = done;
    }
    if (!grid_sync(m.bar, ep, m.err)) return;
    if (check && sdone) break;
    // ---- E: red/black point-implicit sweeps, a pair of lanes per cell: lane sd takes the faces
    // on side sd of every active axis and the axis fluxes of axes sd, sd + 2
    // inner residual partials of this thread, in shared memory (registers are the sweeps')
    double *const num = rsd + threadIdx.x, *const den = rsd + 6 * kBlock + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NW; ++k) num[k * kBlock] = den[k * kBlock] = 0.0;
    for (int sw = 0; sw < m.sweeps; ++sw) {
      const bool first = sw == 0, last = sw == m.sweeps - 1;
      for (int col = 0; col < 2; ++col) {
        const int off = col ? m.ncol0 : 0, cnt = col ? nc - m.ncol0 : m.ncol0;
        // in the first red pass every increment is still zero
        const bool nb_term = !(first && col == 0);
        // both lanes of a pair loop together so the pair shuffles are converged
        const int nitems = ((2 * cnt + 31) / 32) * 32;
        for (int t = it.first; t < nitems; t += it.stride) {
          const int q = t >> 1, sd = t & 1;
          const bool live = q < cnt, upd = live && sd == 0;
          const int c = !live ? 0 : (t == it.first ? (col ? cell1 : cell0) : m.colcells[off + q]);
          int nt[3];
          nat_of(g, c, nt);
          // one wave of loads.  The cell's own data: both lanes W, and for the axes they publish
          // the start-of-step flux and the face Gammas; for the update, lane sd takes the
          // components 3 sd .. 3 sd + 2 (those below NW): their inverse diagonal and R (first pass:
          // K at the first inner step, else corr).  Per face on side sd: the neighbour's published
          // term (and, in the first pass, the face flux).
          const bool pub = live && sd < nact && !(last && col == 1);
          const int k0 = 3 * sd;  // first component of this lane's share of the update
          double Wc[6], iDo[3], Ro[3], Fco[NW], gl = 0.0, gh = 0.0;
#pragma unroll
          for (int k = 0; k < 6; ++k) Wc[k] = live ? m.W[(size_t)c * 6 + k] : 0.0;
#pragma unroll
          for (int k = 0; k < NW; ++k) Fco[k] = 0.0;
          {
            const double *src = first ? (step == 0 ? m.K : m.corr) : m.R;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const bool ok = live && k0 + j < NW;
              iDo[j] = ok ? m.invD[(size_t)c * 6 + k0 + j] : 0.0;
              Ro[j] = ok ? src[(size_t)c * 6 + k0 + j] : 0.0;
            }
          }
          if (pub) {
            if (!last)
#pragma unroll
              for (int k = 0; k < NW; ++k) Fco[k] = Fc[((size_t)c * 3 + sd) * 6 + k];
            face_gammas(m, c, pick3(sd, cs[0], cs[1], cs[2]), pick3(sd, nt[0], nt[1], nt[2]),
                        pick3(sd, g.n[0], g.n[1], g.n[2]), sd, gl, gh);
          }
          double Gn[MA][NW], hA[MA], S[NW];
          bool nbf[MA];
#pragma unroll
          for (int k = 0; k < NW; ++k) S[k] = 0.0;
#pragma unroll
          for (int a = 0; a < MA; ++a) {
            nbf[a] = false;
            hA[a] = 0.0;
#pragma unroll
            for (int k = 0; k < NW; ++k) Gn[a][k] = 0.0;
            if (!live || a >= nact) continue;
            const int na = pick3(a, nt[0], nt[1], nt[2]);
            const bool inside = sd ? na < pick3(a, g.n[0], g.n[1], g.n[2]) - 1 : na > 0;
            const int csa = pick3(a, cs[0], cs[1], cs[2]);
            const int j = sd ? c + csa : c - csa;
            if (inside && nb_term) {
              nbf[a] = true;
              hA[a] = 0.5 * axis_cells(m, a)[na].invh;  // A / (2 V) on a rectilinear cell
              const double *Gj = m.G + ((size_t)j * 3 + a) * 12 + 6 * sd;
#pragma unroll
              for (int k = 0; k < NW; ++k) Gn[a][k] = Gj[k];
            }
            if (first) {
              if (inside) {
#pragma unroll
                for (int k = 0; k < NW; ++k) S[k] += sd ? m.Ffc[((size_t)c * 3 + a) * 6 + k] : -m.Ffc[((size_t)j * 3 + a) * 6 + k];
              } else {
                const int wb = g.wall_base[2 * a + sd];
                if (wb >= 0) {
                  const int trn = pick3(a, nt[1] + g.n[1] * nt[2], nt[0] + g.n[0] * nt[2], nt[0] + g.n[0] * nt[1]);
#pragma unroll
                  for (int k = 0; k < NW; ++k) S[k] += m.wfl[(size_t)(wb + trn) * 6 + k];
                }
              }
            }
          }
          // off-diagonal sum of the lane's faces: (1/2V) A [Delta F_j(n) - Gamma dW_j]
          double acc[NW];
#pragma unroll
          for (int k = 0; k < NW; ++k) acc[k] = 0.0;
#pragma unroll
          for (int a = 0; a < MA; ++a)
            if (nbf[a])
#pragma unroll
              for (int k = 0; k < NW; ++k) acc[k] = fma(Gn[a][k], hA[a], acc[k]);
          // the pair's totals of this lane's components: its own partial plus the partner's
          // (a + b = b + a, so both lanes see the sums a single lane would form)
          auto own = [&](const double *v, int j) { return sd ? (3 + j < NW ? v[3 + j] : 0.0) : v[j]; };
          auto other = [&](const double *v, int j) { return sd ? v[j] : (3 + j < NW ? v[3 + j] : 0.0); };
          double acco[3], So[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            acco[j] = own(acc, j) + __shfl_xor_sync(0xffffffffu, other(acc, j), 1);
            So[j] = first ? own(S, j) + __shfl_xor_sync(0xffffffffu, other(S, j), 1) : 0.0;
          }
          // the update of this lane's components (the point-implicit solve of Eq. res_macro)
          double Rn[3];
          if (first) {
            // residual R_i = -(S + corr) / V, corr = K - S frozen at the first inner step
            const double iV = cell_inv_volume(m, nt);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const bool ok = live && k0 + j < NW;
              if (step == 0) {
                Ro[j] -= So[j];
                if (ok) m.corr[(size_t)c * 6 + k0 + j] = Ro[j];
              }
              Rn[j] = -(So[j] + Ro[j]) * iV;
            }
            if (NW == 6 && live && sd == 1) {
              const double *p = m.pr + (size_t)c * 6;
              const double tau = 2.0 * m.mu0 * power(p[4], m.omega - 1.0) / p[0];
              const double T = (3.0 * p[4] + m.d_r * p[5]) / (3.0 + m.d_r);
              Rn[2] += m.d_r * p[0] * (T - p[5]) / (4.0 * m.Z_r * tau);
            }
            if (!last)
#pragma unroll
              for (int j = 0; j < 3; ++j)
                if (live && k0 + j < NW) m.R[(size_t)c * 6 + k0 + j] = Rn[j];
          } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) Rn[j] = Ro[j];
          }
          double dO[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) dO[j] = (Rn[j] - acco[j]) * iDo[j];
          int here = !last;  // evaluate the axis fluxes (last sweep: and primitives) in this loop
          if (last && live) {
            // the new state; the cell joins the block's list for the compacted evaluation of its
            // primitives, its fluxes for the next step, its published terms (last red pass) and
            // its inner-residual terms after the loop, one item per lane
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              if (k0 + j >= NW) continue;
              const double w = (sd ? Wc[3 + j] : Wc[j]) + dO[j];
              if (!isfinite(w)) atomicCAS(m.err, 0, GSIS_ERR_DIVERGED);
              m.W[(size_t)c * 6 + k0 + j] = w;
              m.dW[(size_t)c * 6 + k0 + j] = dO[j];
            }
            if (upd) {
              const int slot = atomicAdd(&scount, 1);
              if (slot < kListCap) slist[slot] = c;
              else here = 1;
            }
          }
          // both lanes take the whole increment and evaluate the axis fluxes at W + dW of their
          // axes: the increment over the step's start for the other colour's next pass
          // (published with dW) and, in the last sweep when the block's list is full, the fluxes
          // of the next step
          here = __shfl_sync(0xffffffffu, here, t & 30u);
          double d[NW];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double x = __shfl_xor_sync(0xffffffffu, dO[j], 1);
            d[j] = sd ? x : dO[j];
            if (3 + j < NW) d[3 + j] = sd ? dO[j] : x;
          }
          if (last && upd && here) {
            // list overflow: the inner-residual terms here
            const double V = cell_volume(m, nt);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
              num[k * kBlock] += d[k] * d[k] * V;
              den[k * kBlock] += (Wc[k] + d[k]) * (Wc[k] + d[k]) * V;
            }
          }
          if (live && here) {
            double Wnew[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) Wnew[k] = k < NW ? Wc[k] + d[k] : Wc[k];
#pragma unroll
            for (int h = 0; h < (MA > 2 ? 2 : 1); ++h) {
              const int a = sd + 2 * h;
              if (a >= nact) continue;
              double F[6];
              euler_axis<NW>(Wnew, a, 1.0, F);
              const size_t o = ((size_t)c * 3 + a) * 6;
              if (last)
#pragma unroll
                for (int k = 0; k < 6; ++k) Fn[o + k] = F[k];
              if (!(last && col == 1)) {
                double dF[NW], lo = gl, hi = gh;
#pragma unroll
                for (int k = 0; k < NW; ++k) dF[k] = F[k] - (last || h ? Fc[o + k] : Fco[k]);
                if (h) face_gammas(m, c, pick3(a, cs[0], cs[1], cs[2]), pick3(a, nt[0], nt[1], nt[2]), pick3(a, g.n[0], g.n[1], g.n[2]), a, lo, hi);
                publish_terms<NW>(m, c, a, dF, d, lo, hi);
              }
            }
            if (last && upd) cell_prims<NW>(m, c, Wnew);
          }
        }
        if (last) {
          // compacted evaluation for the listed cells: items [0, n) primitives and inner-residual
          // terms, then (cell, axis) fluxes; the block's own W, dW writes are visible after the
          // barrier
          __syncthreads();
          const int n = min(scount, kListCap);
          // warp w runs on sub-partition w % 4: the primitives go to the warps of sub-partitions 0
          // and 1, the axis fluxes to those of 2 and 3, so the two kinds do not share FP64 pipes
          const int wq = threadIdx.x >> 5, rs = blockDim.x >> 1;
          const int r = (((wq >> 2) << 1) | (wq & 1)) * 32 + (threadIdx.x & 31);
          if (!(wq & 2)) {
            for (int t = r; t < n; t += rs) {
              const int c = slist[t];
              double Wl[6];
#pragma unroll
              for (int k = 0; k < 6; ++k) Wl[k] = m.W[(size_t)c * 6 + k];
              cell_prims<NW>(m, c, Wl);
              if (m.tol > 0.0) {
                int nt[3];
                nat_of(g, c, nt);
                const double V = cell_volume(m, nt);
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                  const double d = m.dW[(size_t)c * 6 + k];
                  num[k * kBlock] += d * d * V;
                  den[k * kBlock] += Wl[k] * Wl[k] * V;
                }
              }
            }
          } else {
            for (int t = r; t < n * nact; t += rs) {
              const int q = t / nact, a = t - q * nact;
              const int c = slist[q];
              double Wl[6];
#pragma unroll
              for (int k = 0; k < 6; ++k) Wl[k] = m.W[(size_t)c * 6 + k];
              double F[6];
              euler_axis<NW>(Wl, a, 1.0, F);
              const size_t o = ((size_t)c * 3 + a) * 6;
#pragma unroll
              for (int k = 0; k < 6; ++k) Fn[o + k] = F[k];
              if (col == 0) {
                double dF[NW], dl[NW], lo, hi;
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                  dF[k] = F[k] - Fc[o + k];
                  dl[k] = m.dW[(size_t)c * 6 + k];
                }
                int nt[3];
                nat_of(g, c, nt);
                face_gammas(m, c, pick3(a, cs[0], cs[1], cs[2]), pick3(a, nt[0], nt[1], nt[2]), pick3(a, g.n[0], g.n[1], g.n[2]), a,
                            lo, hi);
                publish_terms<NW>(m, c, a, dF, dl, lo, hi);
              }
            }
          }
          __syncthreads();
          if (threadIdx.x == 0) scount = 0;
        }
        if (last && col == 1 && m.tol > 0.0) {
          // block partials of the inner residual (values 0..5: num_k, 6..11: den_k), double
          // buffered by step.  Only the threads that evaluated listed (or overflowing) cells hold
          // nonzero terms: warps without any skip the FP64 reduction.
          double *red = m.red + (size_t)(step & 1) * gridDim.x * 16;
          const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
          bool nz = false;
#pragma unroll
          for (int k = 0; k < NW; ++k) nz = nz || num[k * kBlock] != 0.0 || den[k * kBlock] != 0.0;
          if (__any_sync(0xffffffffu, nz)) {
            double v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = 0.0;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
              v[k] = num[k * kBlock];
              v[6 + k] = den[k * kBlock];
            }
            const double tot = transpose_sum16(v);
            if (!(lane & 1) && lane < 24) wsum[wid][lane >> 1] = tot;
          } else if (lane < 12) {
            wsum[wid][lane] = 0.0;
          }
          __syncthreads();
          if (threadIdx.x < 24) {
            // lane 2k + h sums value k over warps 8h .. 8h + 7, then the pair adds up
            const int k = threadIdx.x >> 1, h = threadIdx.x & 1;
            double v = 0.0;
#pragma unroll
            for (int w = 0; w < kBlock / 64; ++w) v += wsum[h * (kBlock / 64) + w][k];
            v += __shfl_xor_sync(0x00ffffffu, v, 1);
            if (!h) red[(size_t)blockIdx.x * 16 + k] = v;
          }
        }
        if (!grid_sync(m.bar, ep, m.err)) return;
      }
    }
    used = step + 1;
  }
  // closed domain: rescale the density to the domain's total mass (velocity, temperatures kept)
  if (!grid_sync(m.bar, ep, m.err)) return;
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
  if (!grid_sync(m.bar, ep, m.err)) return;
  __shared__ double sfac;
  if (threadIdx.x < 32) {
    double mm = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) mm += __ldcg(red + b);
    for (int o = 16; o > 0; o >>= 1) mm += __shfl_xor_sync(0xffffffffu, mm, o);
    if (threadIdx.x == 0) sfac = m.closed ? m.mass_ref / mm : 1.0;
  }
  __syncthreads();
  const double fac = sfac;
  for (int c = it.first; c < nc; c += it.stride) {
    double p[6];
    prim_of<NW>(m.W + (size_t)c * 6, m.d_r, p);
    p[0] *= fac;
#pragma unroll
    for (int k = 0; k < 6; ++k) m.Wout[(size_t)c * 6 + k] = p[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *m.iters = used;
}

// One block of 512 threads per SM: the phases have many short FP64 work items and every SM
// must hold some.  The cooperative launch guarantees the blocks are co-resident.
cudaError_t macro_launch_shape(int nc, int max_sms, int *grid, int *block) {
  (void)nc;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  void (*const kernels[])(MacroArgs) = {macro_kernel<5, 2>, macro_kernel<5, 3>, macro_kernel<6, 2>, macro_kernel<6, 3>};
  for (auto k : kernels) {
    int per = 0;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResidualSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kBlock, kResidualSmem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
  }
  if (max_sms > 0 && max_sms < nsm) nsm = max_sms;
  *grid = nsm < MACRO_MAX_GRID ? nsm : MACRO_MAX_GRID;
  *block = kBlock;
  return cudaSuccess;
}

// Self-test of the bounded grid barrier: block 1 of two co-resident blocks leaves without
// arriving, so block 0's wait runs out after `limit` cycles and raises GSIS_ERR_TIMEOUT.
__global__ void barrier_timeout_probe(unsigned *bar, int *err, long long limit) {
  if (blockIdx.x == 1) return;
  unsigned ep = 0;
  grid_sync(bar, ep, err, limit);
}

cudaError_t probe_barrier_timeout(unsigned *bar, int *err, long long limit, cudaStream_t s) {
  void *args[] = {&bar, &err, &limit};
  return cudaLaunchCooperativeKernel((void *)barrier_timeout_probe, dim3(2), dim3(32), args, 0, s);
}

cudaError_t launch_macro(const MacroArgs &a, int grid, int block, cudaStream_t s) {
  MacroArgs copy = a;
  void *args[] = {&copy};
  const bool a3 = a.g.nact > 2;
  void *fn = a.nW == 6 ? (a3 ? (void *)macro_kernel<6, 3> : (void *)macro_kernel<6, 2>)
                       : (a3 ? (void *)macro_kernel<5, 3> : (void *)macro_kernel<5, 2>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, kResidualSmem, s);
}

}  // namespace gsis
