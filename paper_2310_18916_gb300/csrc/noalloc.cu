// noalloc.cu -- velocity moments of a caller-held VDF without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need moments: code that
// runs inside another framework's memory pool with no allocator handle to pass in, code that
// must not trigger allocation inside a latency-critical region, or hosts whose allocator is
// locked while they run.  gsis_vdf_moments_noalloc serves them: it takes device pointers to
// the VDF, the velocity table and the output, and keeps its only scratch (per-chunk partial
// moments) in a fixed-size array of static device memory that every GPU loading this library
// holds until the process exits.
//
// Two passes over the VDF, both summing in FP32 with compensated (Kahan) accumulators:
//   1. density and momentum -> the mean velocity d of each cell (written to the output row);
//   2. the moments of c = xi - d: c(3), cc(6), |c|^2 c(3).
// Moments taken about d, not the origin, keep their accuracy when |u| is large next to the
// thermal speed: about the origin the second and third moments of a Ma-4 stream are dominated
// by rho u u and rho |u|^2 u, and the stress and heat flux would be their small differences.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/gsis.h"
#include "gsis_internal.h"

namespace {

constexpr int kMom1 = 4;                                     // pass 1: 1, xi(3)
constexpr int kMom2 = 12;                                    // pass 2: c(3), cc(6), |c|^2 c(3) about d
constexpr size_t kScratchBytes = 8u << 20;                   // 8 MiB of chunk partials
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);
constexpr size_t kMaxCells = kScratchDoubles / kMom2;        // 87381: one chunk per cell still fits
constexpr int kMaxDevices = 64;
constexpr int kWarps = 4;                                    // warps per block, one (cell, chunk) each

// Chunk partials [chunk][cell][kMom1 or kMom2].  Shared by every call on a device; each pass
// overwrites every entry its reduction reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

template <int N>
struct Comp {
  float s[N], c[N];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = c[k] = 0.f;
  }
  __device__ void add(const float *x) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const float y = x[k] - c[k];
      const float t = s[k] + y;
      c[k] = (t - s[k]) - y;
      s[k] = t;
    }
  }
};

// One warp per (cell, chunk) item, lanes striding over the chunk's velocities (coalesced reads
// of the cell's row); lane partials are reduced over the warp in FP64 in a fixed order.
// PASS 1 sums w f (1, xi); PASS 2 sums w f (c, cc, |c|^2 c) with c = xi - d, d read from
// out[cell][1..3] where pass 1's reduction left it.
template <int PASS>
__global__ void __launch_bounds__(32 * kWarps)
    noalloc_pass_kernel(const float *__restrict__ f, const float *__restrict__ vel, int nc, int nv, int nchunks,
                        int per_chunk, const double *__restrict__ out, double *part) {
  constexpr int N = PASS == 1 ? kMom1 : kMom2;
  const int lane = threadIdx.x & 31;
  const long long item = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (item >= (long long)nc * nchunks) return;
  const int chunk = (int)(item / nc), cell = (int)(item - (long long)chunk * nc);
  const int v0 = chunk * per_chunk;
  const int v1 = min(nv, v0 + per_chunk);
  float d[3] = {0.f, 0.f, 0.f};
  if (PASS == 2) {
    const double *o = out + (size_t)cell * 18;
    d[0] = (float)o[1];
    d[1] = (float)o[2];
    d[2] = (float)o[3];
  }
  Comp<N> acc;
  acc.zero();
  const float *fc = f + (size_t)cell * nv;
  for (int v = v0 + lane; v < v1; v += 32) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(vel) + v);
    const float wf = q.w * __ldg(fc + v);
    float t[N];
    if constexpr (PASS == 1) {
      t[0] = wf;
      t[1] = wf * q.x;
      t[2] = wf * q.y;
      t[3] = wf * q.z;
    } else {
      const float cx = q.x - d[0], cy = q.y - d[1], cz = q.z - d[2];
      const float c2 = cx * cx + cy * cy + cz * cz;
      t[0] = wf * cx;
      t[1] = wf * cy;
      t[2] = wf * cz;
      t[3] = wf * cx * cx;
      t[4] = wf * cy * cy;
      t[5] = wf * cz * cz;
      t[6] = wf * cx * cy;
      t[7] = wf * cx * cz;
      t[8] = wf * cy * cz;
      t[9] = wf * c2 * cx;
      t[10] = wf * c2 * cy;
      t[11] = wf * c2 * cz;
    }
    acc.add(t);
  }
  double *dst = part + ((size_t)chunk * nc + cell) * N;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double x = (double)acc.s[k] - (double)acc.c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) dst[k] = x;
  }
}

// Pass 1's chunks summed in fixed order: rho and the mean velocity d into out[cell][0..3].
__global__ void noalloc_mean_kernel(const double *part, int nc, int nchunks, double *out) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= nc) return;
  double S[kMom1] = {0.0, 0.0, 0.0, 0.0};
  for (int ch = 0; ch < nchunks; ++ch)
    for (int k = 0; k < kMom1; ++k) S[k] += part[((size_t)ch * nc + cell) * kMom1 + k];
  double *M = out + (size_t)cell * 18;
  M[0] = S[0];
  for (int i = 0; i < 3; ++i) M[1 + i] = (double)(float)(S[1 + i] / S[0]);  // d as pass 2 uses it
}

// Pass 2's chunks summed in fixed order, then the fields of GSIS_F_HALF: rho, u, Tt, Tr (= Tt),
// sigma(6), qt(3), qr(3) = 0.  The moments are about d; the true mean is u = d + e with
// e = S1/rho (rounding of d only), so P = S2 - rho e e^T and
// q = 1/2 [S3 - tr(S2) e - 2 S2 e + 2 rho |e|^2 e], terms that stay small.
__global__ void noalloc_finalize_kernel(const double *part, int nc, int nchunks, double *out) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= nc) return;
  double S[kMom2];
  for (int k = 0; k < kMom2; ++k) S[k] = 0.0;
  for (int ch = 0; ch < nchunks; ++ch)
    for (int k = 0; k < kMom2; ++k) S[k] += part[((size_t)ch * nc + cell) * kMom2 + k];
  double *M = out + (size_t)cell * 18;
  const double rho = M[0];
  const double e[3] = {S[0] / rho, S[1] / rho, S[2] / rho};
  const double S2[3][3] = {{S[3], S[6], S[7]}, {S[6], S[4], S[8]}, {S[7], S[8], S[5]}};
  double P[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[i][j] = S2[i][j] - rho * e[i] * e[j];
  const double trP = P[0][0] + P[1][1] + P[2][2], trS2 = S2[0][0] + S2[1][1] + S2[2][2];
  const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  for (int i = 0; i < 3; ++i) M[1 + i] += e[i];
  M[4] = 2.0 * trP / (3.0 * rho);
  M[5] = M[4];
  M[6] = P[0][0] - trP / 3.0;
  M[7] = P[1][1] - trP / 3.0;
  M[8] = P[2][2] - trP / 3.0;
  M[9] = P[0][1];
  M[10] = P[0][2];
  M[11] = P[1][2];
  for (int i = 0; i < 3; ++i) {
    const double S2e = S2[i][0] * e[0] + S2[i][1] * e[1] + S2[i][2] * e[2];
    M[12 + i] = 0.5 * (S[9 + i] - trS2 * e[i] - 2.0 * S2e + 2.0 * rho * ee * e[i]);
    M[15 + i] = 0.0;
  }
}

// Device address of the static scratch for the current device, looked up once per device.
int scratch_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSIS_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, g_noalloc_scratch) != cudaSuccess || !p) return GSIS_E_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GSIS_OK;
}

}  // namespace

extern "C" int gsis_vdf_moments_noalloc(const float *f_dev, const float *vel_dev, int ncells, int nvel,
                                        double *out_dev, void *stream) {
  if (!f_dev || !vel_dev || !out_dev || ncells < 1 || nvel < 1) {
    gsis::set_handle_free_error("gsis_vdf_moments_noalloc: NULL pointer or a size below 1");
    return GSIS_E_INVALID;
  }
  if ((size_t)ncells > kMaxCells) {
    gsis::set_handle_free_error(("gsis_vdf_moments_noalloc: " + std::to_string(ncells) +
                                 " cells exceed the fixed scratch's maximum of " + std::to_string(kMaxCells))
                                    .c_str());
    return GSIS_E_INVALID;
  }
  if (((size_t)vel_dev & 15) != 0) {
    gsis::set_handle_free_error("gsis_vdf_moments_noalloc: vel_dev must be 16-byte aligned");
    return GSIS_E_INVALID;
  }
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) {
    gsis::set_handle_free_error("gsis_vdf_moments_noalloc: cudaGetSymbolAddress of the scratch failed");
    return rc;
  }
  // Chunks of at least 32 velocities; enough (cell, chunk) warps to fill the GPU; all chunk
  // partials of pass 2 inside the scratch.
  long long nchunks = (long long)(kMaxCells / (size_t)ncells);
  const long long want = (40000 + ncells - 1) / ncells;
  if (nchunks > want) nchunks = want;
  if (nchunks > (nvel + 31) / 32) nchunks = (nvel + 31) / 32;
  if (nchunks < 1) nchunks = 1;
  const int per_chunk = (int)((nvel + nchunks - 1) / nchunks);
  const int nch = (nvel + per_chunk - 1) / per_chunk;
  const long long items = (long long)ncells * nch;  // <= kMaxCells
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((items + kWarps - 1) / kWarps);
  const unsigned cgrid = (unsigned)((ncells + 127) / 128);
  noalloc_pass_kernel<1><<<grid, 32 * kWarps, 0, s>>>(f_dev, vel_dev, ncells, nvel, nch, per_chunk, out_dev, scratch);
  noalloc_mean_kernel<<<cgrid, 128, 0, s>>>(scratch, ncells, nch, out_dev);
  noalloc_pass_kernel<2><<<grid, 32 * kWarps, 0, s>>>(f_dev, vel_dev, ncells, nvel, nch, per_chunk, out_dev, scratch);
  noalloc_finalize_kernel<<<cgrid, 128, 0, s>>>(scratch, ncells, nch, out_dev);
  if (cudaGetLastError() != cudaSuccess) {
    gsis::set_handle_free_error("gsis_vdf_moments_noalloc: kernel launch failed");
    return GSIS_E_CUDA;
  }
  return GSIS_OK;
}
