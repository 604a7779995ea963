// noalloc.cu -- velocity moments of a caller-held VDF without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need moments: code that
// runs inside another framework's memory pool with no allocator handle to pass in, code that
// must not trigger allocation inside a latency-critical region, or hosts whose allocator is
// locked while they run.  gsis_vdf_moments_noalloc serves them: it takes device pointers to
// the VDF, the velocity table and the output, and keeps its only scratch (per-chunk partial
// moments) in a fixed-size array of static device memory that every GPU loading this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/gsis.h"

namespace {

constexpr int kMom = 13;                                     // 1, c(3), cc(6), |c|^2 c(3) about u = 0
constexpr size_t kScratchBytes = 8u << 20;                   // 8 MiB of chunk partials
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

// Chunk partials [chunk][cell][13].  Shared by every call on a device; each call overwrites
// every entry it reads back, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Compensated accumulation of one velocity's contributions (Kahan), FP32 as in the solver.
struct Comp {
  float s[kMom], c[kMom];
  __device__ void add(const float *x) {
#pragma unroll
    for (int k = 0; k < kMom; ++k) {
      const float y = x[k] - c[k];
      const float t = s[k] + y;
      c[k] = (t - s[k]) - y;
      s[k] = t;
    }
  }
};

// One thread per (cell, velocity chunk): raw moments about the origin of f[cell][v] over the
// chunk's velocities (the streaming moments kernel of the solver, on the canonical layout).
__global__ void noalloc_moments_kernel(const float *__restrict__ f, const float *__restrict__ vel, int nc, int nv,
                                       int per_chunk, double *part) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y;
  if (cell >= nc) return;
  const int v0 = chunk * per_chunk;
  const int v1 = min(nv, v0 + per_chunk);
  Comp acc;
#pragma unroll
  for (int k = 0; k < kMom; ++k) acc.s[k] = acc.c[k] = 0.f;
  const float *fc = f + (size_t)cell * nv;
  for (int v = v0; v < v1; ++v) {
    const float x = __ldg(vel + 4 * v), y = __ldg(vel + 4 * v + 1), z = __ldg(vel + 4 * v + 2), w = __ldg(vel + 4 * v + 3);
    const float wf = w * __ldg(fc + v);
    const float c2 = x * x + y * y + z * z;
    const float t[kMom] = {wf, wf * x, wf * y, wf * z, wf * x * x, wf * y * y, wf * z * z,
                           wf * x * y, wf * x * z, wf * y * z, wf * c2 * x, wf * c2 * y, wf * c2 * z};
    acc.add(t);
  }
  double *out = part + ((size_t)chunk * nc + cell) * kMom;
#pragma unroll
  for (int k = 0; k < kMom; ++k) out[k] = (double)acc.s[k] - (double)acc.c[k];
}

// Sum the chunks in fixed order and convert to rho, u, Tt, Tr (= Tt), sigma(6), qt(3), qr(3)
// = 0, the layout of GSIS_F_HALF.  Shift from the origin to the mean velocity d = S1/rho:
// P = S2 - rho d d^T, Tt = 2 tr P / (3 rho), q = 1/2 [S3 - tr(S2) d - 2 S2 d + 2 rho |d|^2 d].
__global__ void noalloc_finalize_kernel(const double *part, int nc, int nchunks, double *out) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= nc) return;
  double S[kMom];
  for (int k = 0; k < kMom; ++k) {
    double a = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) a += part[((size_t)ch * nc + cell) * kMom + k];
    S[k] = a;
  }
  const double rho = S[0];
  const double d[3] = {S[1] / rho, S[2] / rho, S[3] / rho};
  const double S2[3][3] = {{S[4], S[7], S[8]}, {S[7], S[5], S[9]}, {S[8], S[9], S[6]}};
  double P[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[i][j] = S2[i][j] - rho * d[i] * d[j];
  const double trP = P[0][0] + P[1][1] + P[2][2], trS2 = S2[0][0] + S2[1][1] + S2[2][2];
  const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double *M = out + (size_t)cell * 18;
  M[0] = rho;
  for (int i = 0; i < 3; ++i) M[1 + i] = d[i];
  M[4] = 2.0 * trP / (3.0 * rho);
  M[5] = M[4];
  M[6] = P[0][0] - trP / 3.0;
  M[7] = P[1][1] - trP / 3.0;
  M[8] = P[2][2] - trP / 3.0;
  M[9] = P[0][1];
  M[10] = P[0][2];
  M[11] = P[1][2];
  for (int i = 0; i < 3; ++i) {
    const double S2d = S2[i][0] * d[0] + S2[i][1] * d[1] + S2[i][2] * d[2];
    M[12 + i] = 0.5 * (S[10 + i] - trS2 * d[i] - 2.0 * S2d + 2.0 * rho * dd * d[i]);
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
  if (!f_dev || !vel_dev || !out_dev || ncells < 1 || nvel < 1) return GSIS_E_INVALID;
  // at least one chunk per cell must fit in the fixed scratch
  const size_t max_cells = kScratchDoubles / kMom;
  if ((size_t)ncells > max_cells) return GSIS_E_INVALID;
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  int nchunks = (int)(max_cells / (size_t)ncells);
  const int want = (160000 + ncells - 1) / ncells;  // enough (cell, chunk) threads to fill the GPU
  if (nchunks > want) nchunks = want;
  if (nchunks > nvel) nchunks = nvel;
  if (nchunks < 1) nchunks = 1;
  const int per_chunk = (nvel + nchunks - 1) / nchunks;
  nchunks = (nvel + per_chunk - 1) / per_chunk;
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid((ncells + 127) / 128, nchunks);
  noalloc_moments_kernel<<<grid, 128, 0, s>>>(f_dev, vel_dev, ncells, nvel, per_chunk, scratch);
  if (cudaGetLastError() != cudaSuccess) return GSIS_E_CUDA;
  noalloc_finalize_kernel<<<(ncells + 127) / 128, 128, 0, s>>>(scratch, ncells, nchunks, out_dev);
  if (cudaGetLastError() != cudaSuccess) return GSIS_E_CUDA;
  return GSIS_OK;
}
