// reduce.cu -- deterministic reductions and per-cell FP64 kernels of one GSIS outer step:
// block partials -> moments (Eq. getmoment) and kinetic face fluxes, moment shift to the mean
// velocity, closed-domain mass scale, HoT (Eq. full_constitutive), the per-cell state of the
// next kinetic step (Eq. updatef applied lazily) and eps (Eq. convergence_critertion).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "gsis_internal.h"

namespace gsis {

namespace {
constexpr double kPi = 3.14159265358979323846;
}  // namespace

// Chunk partials [chunk][cell][np] -> mom [cell][MOM_STRIDE] (raw, about the state velocity:
// f0 then, Rykov, f1) and
//   K [cell][k] = V sum_v w phi_k (g^n - f^{n+1/2}) / tau = sum over the cell's faces of the
//   outward kinetic face flux (mass, momentum, energy, internal energy; the last 0 for Shakhov).
__global__ void reduce_moments_kernel(const double *mp, int nchunks, int nc, int np, const double *vol,
                                      const double *st64, double *mom, double *K) {
  const size_t n = (size_t)nc * np;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int cell = (int)(idx / np), k = (int)(idx % np);
    double acc = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) acc += mp[((size_t)ch * nc + cell) * np + k];
    const double kf = vol[cell] * st64[(size_t)cell * NST + 11];
    if (k < NMOM) {
      mom[(size_t)cell * MOM_STRIDE + k] = acc;
    } else if (k < NMOM + NFF) {
      K[(size_t)cell * 6 + (k - NMOM)] = kf * acc;
      if (k == NMOM && np == NMOM + NFF) K[(size_t)cell * 6 + 5] = 0.0;
    } else if (k == NMOM + NFF) {
      K[(size_t)cell * 6 + 5] = kf * acc;
    } else {
      mom[(size_t)cell * MOM_STRIDE + NMOM + (k - NMOM - NFF - 1)] = acc;
    }
  }
}

// FP64 storage, Shakhov: chunks 0..nchunks-1 hold sum w f (1, xi, xi xi, |xi|^2 xi) about the
// origin, the last chunk sum w phi g^n.  Per cell: K = V/tau (G - F) with F = sum w phi f
// (phi = 1, xi, |xi|^2/2), and the moments about the state velocity u by the binomial shift
//   M1 = S1 - u S0,  M2_ab = S2_ab - u_a S1_b - u_b S1_a + u_a u_b S0,
//   M3_a = S3_a - u_a tr S2 - 2 (S2 u)_a + 2 u_a (u.S1) + |u|^2 S1_a - |u|^2 u_a S0.
__global__ void reduce_origin_kernel(const double *mp, int nrows, int nc, const double *vol, const double *st64,
                                     double *mom, double *K) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= nc) return;
  constexpr int NP = NMOM + NFF;
  double S[NP];
  for (int k = 0; k < NP; ++k) S[k] = 0.0;
  for (int ch = 0; ch < nrows; ++ch) {
    const double *r = mp + ((size_t)ch * nc + cell) * NP;
    for (int k = 0; k < NP; ++k) S[k] += r[k];
  }
  const double *st = st64 + (size_t)cell * NST;
  const double u[3] = {st[0], st[1], st[2]};
  const double kf = vol[cell] * st[11];
  const double S0 = S[0], S1[3] = {S[1], S[2], S[3]};
  const double S2[3][3] = {{S[4], S[7], S[8]}, {S[7], S[5], S[9]}, {S[8], S[9], S[6]}};
  const double trS2 = S[4] + S[5] + S[6];
  double *k6 = K + (size_t)cell * 6;
  k6[0] = kf * (S[NMOM] - S0);
  for (int a = 0; a < 3; ++a) k6[1 + a] = kf * (S[NMOM + 1 + a] - S1[a]);
  k6[4] = kf * (S[NMOM + 4] - 0.5 * trS2);
  k6[5] = 0.0;
  const double uS1 = u[0] * S1[0] + u[1] * S1[1] + u[2] * S1[2];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double M2[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) M2[a][b] = S2[a][b] - u[a] * S1[b] - u[b] * S1[a] + u[a] * u[b] * S0;
  double *M = mom + (size_t)cell * MOM_STRIDE;
  M[0] = S0;
  for (int a = 0; a < 3; ++a) M[1 + a] = S1[a] - u[a] * S0;
  M[4] = M2[0][0];
  M[5] = M2[1][1];
  M[6] = M2[2][2];
  M[7] = M2[0][1];
  M[8] = M2[0][2];
  M[9] = M2[1][2];
  for (int a = 0; a < 3; ++a) {
    const double S2u = S2[a][0] * u[0] + S2[a][1] * u[1] + S2[a][2] * u[2];
    M[10 + a] = S[10 + a] - u[a] * trS2 - 2.0 * S2u + 2.0 * u[a] * uS1 + uu * S1[a] - uu * u[a] * S0;
  }
}

// Outward kinetic wall flux per unit area: the half moving towards the wall from the wall cells'
// block partials (blocks whose octant moves towards this wall), the re-emitted half rho_w Zw.
// General meshes (general = 1): every block's partial already holds both halves along the
// face's outward normal.
template <typename T>
__global__ void reduce_wall_kernel(const T *wpart, const int8_t *boct, int nblocks, int nwall, const int *wall_side,
                                   const double *rho_w, const double *Zw, int emit, int general, double *wf) {
  // one block per wall face, warp m < NWF for moment m: lane l sums the blocks l, l + 32, ... in
  // order, then a fixed butterfly over the lanes
  const int w = blockIdx.x, m = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= nwall || m >= NWF) return;
  const int side = wall_side[w], a = side / 2;
  const bool plus = side & 1;
  double out = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    const bool neg = (boct[b] >> a) & 1;
    if (!general && neg == plus) continue;  // this block's velocities move away from the wall
    out += (double)wpart[((size_t)b * nwall + w) * NWF + m];
  }
  for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
  if (lane == 0) {
    // the re-emitted half once per solve: by one shard of a velocity-sharded solve
    if (general) {
      wf[(size_t)w * 6 + m] = out;
      return;
    }
    const double tot = out + (emit ? rho_w[w] * Zw[6 * side + m] : 0.0);
    wf[(size_t)w * 6 + m] = plus ? tot : -tot;
  }
}

template <typename T>
cudaError_t launch_reduce(const double *mp, int nchunks, int nvdf, const T *wpart, const int8_t *boct, int nblocks,
                          const KinGeom &g, const int *wall_cell, const int *wall_side, int nwall,
                          const double *rho_w, const double *Zw, bool emit, bool general, const double *vol,
                          const double *st64, double *mom, double *K, double *wf, cudaStream_t s, bool origin) {
  (void)wall_cell;
  const int np = moment_len(nvdf);
  const size_t n = (size_t)g.nc * np;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (origin)
    reduce_origin_kernel<<<(g.nc + 127) / 128, 128, 0, s>>>(mp, nchunks + 1, g.nc, vol, st64, mom, K);
  else
    reduce_moments_kernel<<<grid, 256, 0, s>>>(mp, nchunks, g.nc, np, vol, st64, mom, K);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nwall == 0 || wpart == nullptr) return e;
  reduce_wall_kernel<T><<<nwall, 32 * NWF, 0, s>>>(wpart, boct, nblocks, nwall, wall_side, rho_w, Zw, emit ? 1 : 0,
                                                   general ? 1 : 0, wf);
  return cudaGetLastError();
}
template cudaError_t launch_reduce<float>(const double *, int, int, const float *, const int8_t *, int, const KinGeom &,
                                          const int *, const int *, int, const double *, const double *, bool, bool,
                                          const double *, const double *, double *, double *, double *, cudaStream_t,
                                          bool);
template cudaError_t launch_reduce<double>(const double *, int, int, const double *, const int8_t *, int,
                                           const KinGeom &, const int *, const int *, int, const double *,
                                           const double *, bool, bool, const double *, const double *, double *,
                                           double *, double *, cudaStream_t, bool);

// ---------------------------------------------------------------------------------------------
// Raw moments about the state velocity un -> rho, u, Tt, sigma, q about the mean velocity.
// With d = S1/rho (u = un + d):  P = S2 - rho d d^T,  Tt = 2 tr P / (3 rho),
//   q = 1/2 [S3 - tr(S2) d - 2 S2 d + 2 rho |d|^2 d].
// Then the closed-domain mass scale s = mass_ref / sum(rho V) (the last block computes it
// from the per-block partial masses in block order).
__global__ void finalize_kernel(FinalizeArgs a) {
  __shared__ double red[256];
  double mloc = 0.0;
  const int nc = a.g.nc;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < nc; cell += gridDim.x * blockDim.x) {
    const double *S = a.mom + (size_t)cell * MOM_STRIDE;
    const double *un = a.st64 + (size_t)cell * NST;
    const double rho = S[0];
    const double d[3] = {S[1] / rho, S[2] / rho, S[3] / rho};
    const double S2[3][3] = {{S[4], S[7], S[8]}, {S[7], S[5], S[9]}, {S[8], S[9], S[6]}};
    double P[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) P[i][j] = S2[i][j] - rho * d[i] * d[j];
    const double trP = P[0][0] + P[1][1] + P[2][2];
    const double trS2 = S2[0][0] + S2[1][1] + S2[2][2];
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double *M = a.Mh + (size_t)cell * 18;
    M[0] = rho;
    for (int i = 0; i < 3; ++i) M[1 + i] = un[i] + d[i];
    M[4] = 2.0 * trP / (3.0 * rho);
    // Rykov: (d_r / 2) rho R Tr = sum w f1, qr = sum w (c - d) f1 about the mean velocity
    M[5] = a.nvdf == 2 ? S[NMOM] / (a.d_r * rho / 4.0) : M[4];
    M[6] = P[0][0] - trP / 3.0;
    M[7] = P[1][1] - trP / 3.0;
    M[8] = P[2][2] - trP / 3.0;
    M[9] = P[0][1];
    M[10] = P[0][2];
    M[11] = P[1][2];
    for (int i = 0; i < 3; ++i) {
      const double S2d = S2[i][0] * d[0] + S2[i][1] * d[1] + S2[i][2] * d[2];
      M[12 + i] = 0.5 * (S[10 + i] - trS2 * d[i] - 2.0 * S2d + 2.0 * rho * dd * d[i]);
      M[15 + i] = a.nvdf == 2 ? S[NMOM + 1 + i] - d[i] * S[NMOM] : 0.0;
    }
    if (!(rho > 0.0) || !(M[4] > 0.0) || !(M[5] > 0.0) || !isfinite(M[12]) || !isfinite(M[13]) || !isfinite(M[14]))
      atomicCAS(a.err, 0, GSIS_ERR_DIVERGED);
    mloc += rho * a.vol[cell];
  }
  red[threadIdx.x] = mloc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  __shared__ bool lastb;
  if (threadIdx.x == 0) {
    a.scratch[blockIdx.x] = red[0];
    __threadfence();
    const unsigned t = atomicAdd(a.ticket, 1u);
    lastb = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (lastb && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) tot += ((volatile double *)a.scratch)[b];
    a.mass_scale[0] = a.closed ? a.mass_ref / tot : 1.0;
    a.mass_scale[1] = tot;
    *a.ticket = 0u;
  }
}

__global__ void scale_kernel(int nc, double *Mh, const double *mass_scale) {
  const double s = mass_scale[0];
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < nc; cell += gridDim.x * blockDim.x) {
    double *M = Mh + (size_t)cell * 18;
    M[0] *= s;
    for (int q = 6; q < 18; ++q) M[q] *= s;
  }
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s) {
  int grid = (a.g.nc + 255) / 256;
  if (grid > 1024) grid = 1024;
  finalize_kernel<<<grid, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scale_kernel<<<grid, 256, 0, s>>>(a.g.nc, a.Mh, a.mass_scale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// LSQ gradient of a cell field (stride floats apart) on the rectilinear block.
__device__ __forceinline__ void grad_field(const KinGeom &g, const AxisCell<double> *const *ax, const double *q,
                                           int stride, int cell, double *gr) {
  const int nat[3] = {cell % g.n[0], (cell / g.n[0]) % g.n[1], cell / (g.n[0] * g.n[1])};
  const int cs[3] = {1, g.n[0], g.n[0] * g.n[1]};
  const double qi = q[(size_t)cell * stride];
  for (int a = 0; a < 3; ++a) {
    gr[a] = 0.0;
    if (!g.act[a]) continue;
    const AxisCell<double> c = ax[a][nat[a]];
    const double lo = nat[a] > 0 ? q[(size_t)(cell - cs[a]) * stride] : qi;
    const double hi = nat[a] < g.n[a] - 1 ? q[(size_t)(cell + cs[a]) * stride] : qi;
    gr[a] = c.clo * (lo - qi) + c.chi * (hi - qi);
  }
}

__device__ __forceinline__ void conductivities(const CellFieldArgs &c, double mu, double *kt, double *kr) {
  // Eq. mu_kappa with R = 1/2: (kt, kr) = (mu/4) A^{-1} (5, d_r); Shakhov: A_tt = 2/3, d_r = 0.
  if (c.model == 0) {
    *kt = mu * 15.0 / 8.0;
    *kr = 0.0;
    return;
  }
  const double det = c.A[0] * c.A[3] - c.A[1] * c.A[2];
  *kt = mu / 4.0 * (c.A[3] * 5.0 - c.A[1] * c.d_r) / det;
  *kr = mu / 4.0 * (-c.A[2] * 5.0 + c.A[0] * c.d_r) / det;
}

__global__ void hot_kernel(CellFieldArgs c, const double *Mh, double *hot) {
  const int nc = c.g.nc;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < nc; cell += gridDim.x * blockDim.x) {
    double G[3][3], gT[3], gTr[3];
    for (int i = 0; i < 3; ++i) grad_field(c.g, c.ax, Mh + 1 + i, 18, cell, G[i]);
    grad_field(c.g, c.ax, Mh + 4, 18, cell, gT);
    grad_field(c.g, c.ax, Mh + 5, 18, cell, gTr);
    const double *M = Mh + (size_t)cell * 18;
    const double mu = c.Kn / sqrt(kPi) * pow(M[4], c.omega);
    double kt, kr;
    conductivities(c, mu, &kt, &kr);
    const double div = G[0][0] + G[1][1] + G[2][2];
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    double *h = hot + (size_t)cell * 12;
    for (int t = 0; t < 6; ++t) {
      const int i = ia[t], j = ib[t];
      h[t] = M[6 + t] + mu * (G[i][j] + G[j][i] - (i == j ? 2.0 / 3.0 * div : 0.0));
    }
    for (int i = 0; i < 3; ++i) {
      h[6 + i] = M[12 + i] + kt * gT[i];
      h[9 + i] = c.model == 1 ? M[15 + i] + kr * gTr[i] : 0.0;
    }
  }
}

cudaError_t launch_hot(const CellFieldArgs &c, const double *Mh, double *hot, cudaStream_t s) {
  int grid = (c.g.nc + 255) / 256;
  if (grid > 1024) grid = 1024;
  hot_kernel<<<grid, 256, 0, s>>>(c, Mh, hot);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// State of the next kinetic step: reference distribution and collision rate from W^{n+1}
// (heat flux from the kinetic moments of f^{n+1/2}); pending correction
//   f^{n+1} = s f_raw + M(W^{n+1}) - M(W^{n+1/2})   (Eq. updatef).
template <typename T>
__global__ void state_kernel(StateArgs a) {
  const int nc = a.g.nc;
  const double s = a.mass_scale_ptr ? a.mass_scale_ptr[0] : a.mass_scale;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < nc; cell += gridDim.x * blockDim.x) {
    const double *W = a.Wn + (size_t)cell * 6;
    const double *M = a.Mh + (size_t)cell * 18;
    double *st = a.st64 + (size_t)cell * NST;
    // the Maxwellian of the step that just stored f becomes the storage reference of relative
    // VDF storage (f1: times its internal-energy factor)
    for (int q = 0; q < 5; ++q) st[16 + q] = st[q];
    st[21] = st[29];
    const double rho = W[0], Tt = W[4];
    st[0] = W[1];
    st[1] = W[2];
    st[2] = W[3];
    st[3] = 1.0 / Tt;
    st[4] = rho * pow(kPi * Tt, -1.5);
    st[5] = M[1];
    st[6] = M[2];
    st[7] = M[3];
    st[8] = 1.0 / M[4];
    st[9] = M[0] * pow(kPi * M[4], -1.5);
    st[10] = s;
    const double invtau = rho * sqrt(kPi) / (2.0 * a.Kn) * pow(Tt, 1.0 - a.omega);
    st[11] = invtau;
    const double A = 8.0 / (15.0 * rho * Tt * Tt);
    st[12] = A * M[12];
    st[13] = A * M[13];
    st[14] = A * M[14];
    st[15] = a.kin_inv_dt + invtau;
    for (int q = 22; q < NST; ++q) st[q] = 0.0;
    if (a.nvdf == 2) {
      // Rykov (Section 2.2): equilibrium temperature T, heat fluxes q0, q1 from the kinetic
      // qt, qr through the A matrix and Z_r, internal-energy factors d_r T / 4
      const double dr = a.d_r, Zr = a.Z_r, Tr = W[5];
      const double Teq = (3.0 * Tt + dr * Tr) / (3.0 + dr);
      const double *qt = M + 12, *qr = M + 15;
      const double At = 2.0 * pow(kPi * Tt, -1.5) / Tt, AT = 2.0 * pow(kPi * Teq, -1.5) / Teq;
      st[24] = 1.0 / Teq;
      st[25] = rho * pow(kPi * Teq, -1.5);
      const double A0 = 8.0 / (15.0 * rho * Teq * Teq);
      for (int k = 0; k < 3; ++k) {
        const double q0 = ((2.0 - 3.0 * a.A[0]) * Zr + 1.0) * qt[k] - 3.0 * a.A[1] * Zr * qr[k];
        const double q1 = -a.A[2] * Zr * qt[k] + (-a.A[3] * Zr + 1.0) * qr[k];
        st[26 + k] = A0 * q0;
        st[31 + k] = At * qr[k];
        st[34 + k] = AT * q1;
      }
      st[29] = dr * Tr / 4.0;
      st[30] = dr * Teq / 4.0;
      st[37] = 1.0 - 1.0 / Zr;
      st[38] = 1.0 / Zr;
      st[39] = dr * M[5] / 4.0;
    }
    T *out = reinterpret_cast<T *>(a.stT) + (size_t)cell * NST;
    for (int q = 0; q < NST; ++q) out[q] = (T)st[q];
  }
}

cudaError_t launch_state(const StateArgs &a, cudaStream_t s) {
  int grid = (a.g.nc + 255) / 256;
  if (grid > 1024) grid = 1024;
  if (a.is_float) state_kernel<float><<<grid, 256, 0, s>>>(a);
  else state_kernel<double><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// eps over rho, u (as a vector) and Tt; fields whose RMS is below 1e-12 count as zero.
__global__ void eps_kernel(EpsArgs a) {
  __shared__ double red[6][256];
  double loc[6] = {0, 0, 0, 0, 0, 0};
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < a.nc; cell += gridDim.x * blockDim.x) {
    const double *n = a.Wn + (size_t)cell * 6, *o = a.Wo + (size_t)cell * 6;
    const double V = a.vol[cell];
    loc[0] += (n[0] - o[0]) * (n[0] - o[0]) * V;
    loc[1] += o[0] * o[0] * V;
    for (int d = 1; d <= 3; ++d) {
      loc[2] += (n[d] - o[d]) * (n[d] - o[d]) * V;
      loc[3] += o[d] * o[d] * V;
    }
    loc[4] += (n[4] - o[4]) * (n[4] - o[4]) * V;
    loc[5] += o[4] * o[4] * V;
  }
  for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = loc[q];
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + off];
    __syncthreads();
  }
  __shared__ bool lastb;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) a.scratch[7 * blockIdx.x + q] = red[q][0];
    __threadfence();
    lastb = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (lastb && threadIdx.x == 0) {
    __threadfence();
    double tot[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < (int)gridDim.x; ++b)
      for (int q = 0; q < 6; ++q) tot[q] += ((volatile double *)a.scratch)[7 * b + q];
    const double vsum = a.vsum;
    double mx = 0.0;
    for (int f = 0; f < 3; ++f) {
      double e = 0.0;
      if (tot[2 * f + 1] > 1e-24 * vsum) e = sqrt(tot[2 * f] / tot[2 * f + 1]);
      a.eps4[f] = e;
      mx = e > mx ? e : mx;
    }
    a.eps4[3] = mx;
    *a.ticket = 0u;
  }
}

cudaError_t launch_eps(const EpsArgs &a, cudaStream_t s) {
  int grid = (a.nc + 255) / 256;
  if (grid > 256) grid = 256;
  eps_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Wall loads (a10): sums over the wall faces of the selected sides of the kinetic wall flux of
// the last kinetic step (per unit area in wf, times the face area): force on the walls
// (outward momentum flux), energy flux into the walls, and the coefficients
// C_D = F.dir / (1/2 rho U^2 A), C_H = Q / (1/2 rho U^3 A).  One block; each thread sums a fixed
// strided subset, then a fixed-order tree, so the result does not depend on timing.
__global__ void wall_loads_kernel(WallLoadArgs a) {
  constexpr int NT = 256;
  __shared__ double red[4][NT];
  double acc[4] = {0, 0, 0, 0};
  for (int w = threadIdx.x; w < a.nwall; w += NT) {
    const int side = a.wall_side[w];
    if (!((a.mask >> side) & 1u)) continue;
    const int c = a.wall_cell[w], ax = side / 2;
    const int nat[3] = {c % a.n[0], (c / a.n[0]) % a.n[1], c / (a.n[0] * a.n[1])};
    const double area = a.area ? a.area[w]
                               : a.ax[0][nat[0]].h * a.ax[1][nat[1]].h * a.ax[2][nat[2]].h * a.ax[ax][nat[ax]].invh;
    for (int k = 0; k < 4; ++k) acc[k] += a.wf[(size_t)w * 6 + 1 + k] * area;
  }
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double F[3] = {red[0][0], red[1][0], red[2][0]}, Q = red[3][0];
    for (int k = 0; k < 3; ++k) a.out[k] = F[k];
    a.out[3] = Q;
    a.out[4] = (F[0] * a.dir[0] + F[1] * a.dir[1] + F[2] * a.dir[2]) / (0.5 * a.rho_ref * a.U_ref * a.U_ref * a.A_ref);
    a.out[5] = Q / (0.5 * a.rho_ref * a.U_ref * a.U_ref * a.U_ref * a.A_ref);
  }
}

cudaError_t launch_wall_loads(const WallLoadArgs &a, cudaStream_t s) {
  wall_loads_kernel<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gsis
