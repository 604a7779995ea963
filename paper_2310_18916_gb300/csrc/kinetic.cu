// kinetic.cu -- the mesoscopic kinetic step of GSIS on sm_103a (Section 3.2 of arXiv 2310.18916).
//
// One CTA owns one block of VB = 32 discrete velocities of a single octant (one per lane) and
// marches through the spatial cells colour by colour, the colours being the hyperplanes
// i' + j' + k' = const in the upwind order of that octant.  For each cell and velocity it
//   - applies the pending VDF correction of Eq. updatef (and the closed-domain mass scale)
//     while staging f^n into a three-colour shared-memory ring,
//   - builds the reference distribution g (Shakhov g_0t, Section 2.2),
//   - takes the LSQ gradient and the Venkatakrishnan limiter, reconstructs the outflow face
//     value (second-order upwind, Section 3.2),
//   - solves the point-implicit delta form with the first-order upwind implicit operator,
//     taking the inflow value "face value + upwind increment" from the previous colour
//     (exact in one pass on a rectilinear grid: every inflow neighbour has a lower colour),
//   - writes f^{n+1/2} in place, and the outgoing flux moments of its wall faces.
// The velocity moments of f^{n+1/2} are a separate streaming pass (moments_kernel, and
// moments_origin_kernel for FP64 storage on tensor-product grids).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "gsis_internal.h"

namespace gsis {

// VDF element load / store between the storage type S and the arithmetic type T: plain for
// S = T; BF16 storage widens exactly to FP32 on load and rounds to nearest even on store.
template <typename T, typename S>
struct Fio {
  static __device__ __forceinline__ T ld(const S *p) { return *p; }
  static __device__ __forceinline__ void st(S *p, T v) { *p = v; }
};
template <>
struct Fio<float, __nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

__device__ __forceinline__ float dexp(float x) { return __expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float ddiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return a / b; }

// Wall Maxwellian M(xi; u_w, T_w) with unit density, in the arithmetic type (an FP64 pow per
// lane would cost FP64-rate time on this GPU in every CTA's set-up)
template <typename T>
__device__ __forceinline__ T wall_maxwellian(const double *uT, T x, T y, T z) {
  const T ux = (T)uT[0], uy = (T)uT[1], uz = (T)uT[2], Tw = (T)uT[3];
  const T cx = x - ux, cy = y - uy, cz = z - uz;
  const T pT = (T)3.14159265358979323846 * Tw;
  const T norm = (T)1 / (pT * sqrt(pT));  // (pi T_w)^(-3/2)
  return norm * dexp(-(cx * cx + cy * cy + cz * cz) / Tw);
}

// f^n = s f_raw + Cn M(un, Tn) - Co M(uo, To)   (Eq. updatef applied on load)
template <typename T>
__device__ __forceinline__ T corrected(T fraw, const T *st, T x, T y, T z) {
  T cx = x - st[0], cy = y - st[1], cz = z - st[2];
  T mn = st[4] * dexp(-(cx * cx + cy * cy + cz * cz) * st[3]);
  cx = x - st[5]; cy = y - st[6]; cz = z - st[7];
  T mo = st[9] * dexp(-(cx * cx + cy * cy + cz * cz) * st[8]);
  return st[10] * fraw + mn - mo;
}

// BF16 and FP32 storage keep f_raw relative to a per-cell Maxwellian, the Maxwellian of W^n of
// the kinetic step that stored it (state values 16..20): the stored deviation is small next to
// f, and so is its round-off.  FP64 stores f_raw itself (an FP64 exponential per point costs
// more than its round-off is worth).
template <typename S>
struct StoredRelative : std::false_type {};
template <>
struct StoredRelative<__nv_bfloat16> : std::true_type {};
template <>
struct StoredRelative<float> : std::true_type {};

// state values a loader of stored f needs: 24 with the storage reference (FP32, BF16), 12 for
// FP64 storage (slots 0..10, rounded up to whole 16-byte rows)
template <typename S>
__host__ __device__ constexpr int state_len() { return StoredRelative<S>::value ? 24 : 12; }

// f^n from a stored value: f_raw = stored (+ M_r for relative storage), then Eq. updatef
template <typename T, typename S>
__device__ __forceinline__ T corrected_stored(T stored, const T *st, T x, T y, T z) {
  if constexpr (StoredRelative<S>::value) {
    const T cx = x - st[16], cy = y - st[17], cz = z - st[18];
    stored += st[20] * dexp(-(cx * cx + cy * cy + cz * cz) * st[19]);
  }
  return corrected(stored, st, x, y, z);
}

// f^n of the NV reduced VDFs from their stored values, sharing the Maxwellians: f0 as above;
// f1 (Rykov) carries the internal-energy factor d_r T_r / 4 of each Maxwellian (state values
// 21, 29, 39), in its storage reference and in Eq. updatef alike.
template <typename T, typename S, int NV>
__device__ __forceinline__ void corrected_all(const T *stored, const T *st, T x, T y, T z, T *f) {
  T cx = x - st[0], cy = y - st[1], cz = z - st[2];
  const T mn = st[4] * dexp(-(cx * cx + cy * cy + cz * cz) * st[3]);
  cx = x - st[5]; cy = y - st[6]; cz = z - st[7];
  const T mo = st[9] * dexp(-(cx * cx + cy * cy + cz * cz) * st[8]);
  T raw[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) raw[q] = stored[q];
  if constexpr (StoredRelative<S>::value) {
    cx = x - st[16]; cy = y - st[17]; cz = z - st[18];
    const T mr = st[20] * dexp(-(cx * cx + cy * cy + cz * cz) * st[19]);
    raw[0] += mr;
    if constexpr (NV == 2) raw[1] += st[21] * mr;
  }
  f[0] = st[10] * raw[0] + mn - mo;
  if constexpr (NV == 2) f[1] = st[10] * raw[1] + st[29] * mn - st[39] * mo;
}

// Reference distributions of the state W^n (Section 2.2), c = xi - u_n, c2 = |c|^2:
//   Shakhov: g0 = M_t [1 + A q_t.c (c^2/T_t - 5/2)];
//   Rykov:   g_q = (1 - 1/Z_r) g_qt + g_qr / Z_r with the translational (T_t) and equilibrium
//            (T) Maxwellians, heat fluxes q0, q1 and the internal-energy factors (state 24..38).
// mw returns M_t, the Maxwellian relative storage refers to.
template <typename T, int NV>
__device__ __forceinline__ void reference(const T *st, T cx, T cy, T cz, T c2, T &mw, T *g) {
  const T et = dexp(-c2 * st[3]);
  mw = st[4] * et;
  const T g0t = mw * ((T)1 + (st[12] * cx + st[13] * cy + st[14] * cz) * (c2 * st[3] - (T)2.5));
  if constexpr (NV == 1) {
    g[0] = g0t;
  } else {
    const T eT = dexp(-c2 * st[24]);
    const T g0r = st[25] * eT * ((T)1 + (st[26] * cx + st[27] * cy + st[28] * cz) * (c2 * st[24] - (T)2.5));
    const T g1t = st[29] * g0t + (st[31] * cx + st[32] * cy + st[33] * cz) * et;
    const T g1r = st[30] * g0r + (st[34] * cx + st[35] * cy + st[36] * cz) * eT;
    g[0] = st[37] * g0t + st[38] * g0r;
    g[1] = st[37] * g1t + st[38] * g1r;
  }
}

// state values the kinetic kernels read: Rykov 40; Shakhov 16 (24 with relative storage for
// the loaders of stored f)
template <typename S, int NV>
__host__ __device__ constexpr int stage_state_len() { return NV == 2 ? NST_RYKOV : state_len<S>(); }

// Comparisons on the integer pipe for FP64.  On this GPU an FP64 comparison, min or max holds a
// sub-partition's FP64 pipe as long as an FMA; the bit patterns of IEEE doubles order like their
// values once the magnitude bits of negative values are inverted (sign-magnitude to two's
// complement order), so the comparisons below give the same results on the integer pipe.  FP32
// keeps its native comparisons.
__device__ __forceinline__ long long ordered_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool is_greater(double a, double b) { return ordered_key(a) > ordered_key(b); }
__device__ __forceinline__ bool is_greater(float a, float b) { return a > b; }
__device__ __forceinline__ double larger(double a, double b) { return is_greater(a, b) ? a : b; }
__device__ __forceinline__ float larger(float a, float b) { return a > b ? a : b; }
__device__ __forceinline__ double smaller(double a, double b) { return is_greater(a, b) ? b : a; }
__device__ __forceinline__ float smaller(float a, float b) { return a < b ? a : b; }
// a > 0
__device__ __forceinline__ bool is_positive(double a) { return __double_as_longlong(a) > 0; }
__device__ __forceinline__ bool is_positive(float a) { return a > 0.f; }
// a <= b and a < b for a, b >= 0 (non-negative doubles order like their bit patterns)
__device__ __forceinline__ bool nonneg_le(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
__device__ __forceinline__ bool nonneg_le(float a, float b) { return a <= b; }
__device__ __forceinline__ bool nonneg_lt(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool nonneg_lt(float a, float b) { return a < b; }

// Venkatakrishnan limiter of one cell: min over its faces (and 1) of
//   (Dm^2 + 2 D2 Dm + e^2) / (Dm^2 + D2 Dm + 2 D2^2 + e^2),
// the face function with numerator and denominator divided by D2; both are positive, so
// the minimum is taken by cross-multiplication and divided once.  Of the two faces of an axis
// (r_lo < 0 < r_hi) only the one with the smaller y = Dm / D2 >= 0 can give the minimum: with
// E = e^2 / D2^2 (the same on both faces, |r_lo| = |r_hi|) the function (y^2 + 2y + E) /
// (y^2 + y + 2 + E) rises while y < 2 + sqrt(8 + E) and exceeds 1 exactly when y > 2.
template <typename T, int NACT>
__device__ __forceinline__ void venkat_parts(T fi, T fmax, T fmin, const T *gr, const T *rlo, const T *rhi, T eps2,
                                             T &bn, T &bd) {
  const T dp = fmax - fi, dn = fmin - fi;
  bn = (T)1;
  bd = (T)1;
#pragma unroll
  for (int a = 0; a < NACT; ++a) {
    const T dh = gr[a] * rhi[a], dl = gr[a] * rlo[a];
    const bool pos = is_positive(gr[a]);
    const T mh = pos ? dp : dn, ml = pos ? dn : dp;
    const bool hi = nonneg_le(fabs(mh) * fabs(dl), fabs(ml) * fabs(dh));
    // (gr = 0: D2 = 0 and the face value is 1, which never lowers the minimum)
    const T d2 = hi ? dh : dl, dm = hi ? mh : ml;
    const T dm2 = dm * dm + eps2;
    const T n = (T)2 * d2 * dm + dm2;
    const T d = d2 * ((T)2 * d2 + dm) + dm2;
    if (nonneg_lt(n * bd, bn * d)) { bn = n; bd = d; }
  }
}
template <typename T, int NACT>
__device__ __forceinline__ T venkat_phi(T fi, T fmax, T fmin, const T *gr, const T *rlo, const T *rhi, T eps2) {
  T bn, bd;
  venkat_parts<T, NACT>(fi, fmax, fmin, gr, rlo, rhi, eps2, bn, bd);
  return ddiv(bn, bd);
}

// Per-cell state and colour-entry addresses from 32-bit offsets: a 64-bit multiply by a
// non-power-of-two stride would run at the FP64 rate on this GPU (cells * NST < 2^32 is checked
// at creation).
template <typename T>
__device__ __forceinline__ const T *state_of(const T *st, int cell) {
  return st + (unsigned)cell * (unsigned)NST;
}
__device__ __forceinline__ const EntryInfo &entry_of(const EntryInfo *e, int i) {
  return *reinterpret_cast<const EntryInfo *>(reinterpret_cast<const char *>(e) + (unsigned)i * (unsigned)sizeof(EntryInfo));
}

template <int N = 16>
__device__ __forceinline__ void load_state(const float *__restrict__ src, float *st) {
  const float4 *p = reinterpret_cast<const float4 *>(src);
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 v = __ldg(p + q);
    st[4 * q] = v.x;
    st[4 * q + 1] = v.y;
    st[4 * q + 2] = v.z;
    st[4 * q + 3] = v.w;
  }
}
template <int N = 16>
__device__ __forceinline__ void load_state(const double *__restrict__ src, double *st) {
  const double2 *p = reinterpret_cast<const double2 *>(src);
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    const double2 v = __ldg(p + q);
    st[2 * q] = v.x;
    st[2 * q + 1] = v.y;
  }
}

// Sum over the 32 lanes of v[0..31] by recursive halving: at each level a lane keeps the half
// of its vector selected by one bit of its lane index and adds the partner's copy of that half.
// Afterwards lane l holds the warp total of v[l] (31 shuffles instead of 5 per value).
template <typename T>
__device__ __forceinline__ T transpose_reduce(T *v, int lane) {
#pragma unroll
  for (int h = 16; h > 0; h >>= 1) {
    const bool up = lane & h;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- bulk asynchronous copies (TMA) into shared memory, completed on an mbarrier ----
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// the one arrival of a phase, announcing the bytes its copies will deliver
__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of the given parity; false on time-out (about a second)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit = 1LL << 31) {
  const long long t0 = clock64();
  for (unsigned i = 0; !mbar_test(bar, parity); ++i)
    if ((i & 63u) == 63u && clock64() - t0 > limit) return false;
  return true;
}

// Self-test of the bounded mbarrier wait: a phase that no arrival and no copy completes, so the
// wait runs out after `limit` cycles and raises GSIS_ERR_TIMEOUT.
__global__ void mbarrier_timeout_probe(int *err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u, limit);
  if (!ok && threadIdx.x == 0) atomicCAS(err, 0, GSIS_ERR_TIMEOUT);
}

cudaError_t probe_mbarrier_timeout(int *err, long long limit, cudaStream_t s) {
  mbarrier_timeout_probe<<<1, 32, 0, s>>>(err, limit);
  return cudaGetLastError();
}

// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

template <typename T>
__device__ __forceinline__ void load_state_shared(const T *src, T *st, int n) {
#pragma unroll
  for (int q = 0; q < 40; ++q)
    if (q < n) st[q] = src[q];
}

// shared-memory layout of the kinetic kernel: the three-colour ring and the face buffers (T),
// with factored Maxwellians the factor cache of two colours (KFAC_MAX values per cell), the
// bulk-copy staging area for one colour (stored f in S, then the state rows in T), the mbarrier
template <typename T, typename S>
struct KinSmem {
  size_t ring, ebuf, fcache, rawf, rawst, bar, total;
  __host__ __device__ KinSmem(const KinGeom &g, int nv, int sl, bool fx) {
    ring = 0;
    ebuf = ring + (size_t)3 * g.maxcol * nv * VB * sizeof(T);
    fcache = ebuf;
    for (int a = 0; a < 3; ++a) fcache += (size_t)g.ntrans[a] * nv * VB * sizeof(T);
    rawf = fcache + (fx ? (size_t)2 * g.maxcol * KFAC_MAX * sizeof(T) : 0);
    rawf = (rawf + 15) & ~(size_t)15;
    rawst = (rawf + (size_t)g.maxcol * nv * VB * sizeof(S) + 15) & ~(size_t)15;
    bar = (rawst + (size_t)g.maxcol * sl * sizeof(T) + 15) & ~(size_t)15;
    total = bar + 16;
  }
};

// FX: factored Maxwellians (FP64 Shakhov on a tiled velocity grid).  The block's 32 velocities
// are a TX x TY x TZ tile, so exp(-|xi - u|^2 / T) over the block is the product of
// F = TX + TY + TZ one-dimensional factors exp(-(xi_a - u_a)^2 / T).  When a cell is staged, lane
// t < 2F evaluates factor t of the two Maxwellians of Eq. updatef (M(W^n) for t < F, M(W^{n-1/2})
// above), one exponential per lane for the whole warp, and every lane gathers its three
// factors of each by shuffles.  The factors of M(W^n) stay in the factor cache until the cell
// is computed, where M(W^n) is also the Maxwellian of the reference distribution g.  Three
// exponentials per point become one evaluation per 32 points per Maxwellian.
template <typename T, typename S>
__host__ __device__ inline bool factored(const KinGeom &g, int nvdf) {
  return sizeof(T) == 8 && sizeof(S) == 8 && nvdf == 1 && g.tile[0] > 0;
}

// GM: the colour ring and face buffers of a velocity block too large for shared memory (3D
// meshes: a colour of n^3 cells has O(n^2) cells) live in the block's own slice of a global
// scratch (L2-resident where it fits), and each colour is staged with plain loads.  The
// arithmetic and the order of every cell's inputs are those of the shared-memory kernel.
template <typename T, typename S, int NACT, int NV, bool GM, bool FX>
__global__ void kinetic_kernel(const KinArgs<T, S> A) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  const KinGeom &G = A.g;
  constexpr int SL = stage_state_len<S, NV>();
  const KinSmem<T, S> L(G, NV, SL, FX);
  unsigned char *smem_raw = GM ? A.gscratch + (size_t)blockIdx.x * A.gstride : smem_dyn;
  T *ring = reinterpret_cast<T *>(smem_raw + L.ring);
  T *ebuf[3];
  {
    T *p = reinterpret_cast<T *>(smem_raw + L.ebuf);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ebuf[a] = p;
      p += (size_t)G.ntrans[a] * NV * VB;
    }
  }
  S *rawf = reinterpret_cast<S *>(smem_raw + L.rawf);
  T *rawst = reinterpret_cast<T *>(smem_raw + L.rawst);
  T *fcache = reinterpret_cast<T *>(smem_raw + L.fcache);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + L.bar);
  const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int oct = A.boct[b];
  const int sg[3] = {oct & 1 ? -1 : 1, oct & 2 ? -1 : 1, oct & 4 ? -1 : 1};
  const T *vp = A.vel + ((size_t)b * VB + lane) * 4;
  const T xi[3] = {vp[0], vp[1], vp[2]};
  const T wv = vp[3];
  // factored Maxwellians: this lane's tile position (lx, ly, lz), the source lanes of its three
  // factors, and the factor it evaluates: Maxwellian fj (0: W^n, 1: W^{n-1/2}), axis fa, node fx
  int src[3] = {0, 0, 0}, fj = 0, fa = 0, NF = 0;
  bool fon = false;
  T fnode = (T)0;
  if constexpr (FX) {
    const int TX = G.tile[0], TY = G.tile[1];
    NF = G.tile[0] + G.tile[1] + G.tile[2];
    src[0] = lane % TX;
    src[1] = TX + (lane / TX) % TY;
    src[2] = TX + TY + lane / (TX * TY);
    fon = lane < 2 * NF;
    fj = lane >= NF ? 1 : 0;
    const int r = lane - fj * NF;
    fa = r < TX ? 0 : (r < TX + TY ? 1 : 2);
    const int nl = fa == 0 ? r : (fa == 1 ? TX * (r - TX) : TX * TY * (r - TX - TY));
    const T vx = __shfl_sync(0xffffffffu, xi[0], nl & 31), vy = __shfl_sync(0xffffffffu, xi[1], nl & 31),
            vz = __shfl_sync(0xffffffffu, xi[2], nl & 31);
    fnode = fa == 0 ? vx : (fa == 1 ? vy : vz);
  }
  const T e2 = (T)0.5 * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
  T axi[3], Mw[3], Mw1[3];
  int upside[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    axi[a] = fabs(xi[a]);
    upside[a] = 2 * a + (sg[a] > 0 ? 0 : 1);
    Mw[a] = Mw1[a] = (T)0;
    if (a < NACT && G.wall_base[upside[a]] >= 0) {
      Mw[a] = wall_maxwellian<T>(A.wall_uT + 4 * upside[a], xi[0], xi[1], xi[2]);
      // re-emitted f1 = (d_r T_w / 4) f0 at the wall
      if constexpr (NV == 2) Mw1[a] = (T)(A.d_r * A.wall_uT[4 * upside[a] + 3] / 4.0) * Mw[a];
    }
  }
  const int n0 = G.n[0], n1 = G.n[1];
  S *F[NV];
  F[0] = A.f + (size_t)b * G.nc * VB;
  if constexpr (NV == 2) F[NV - 1] = A.f1 + (size_t)b * G.nc * VB;
  const int4 *natcell = A.natcell + (size_t)oct * G.nc;
  const T K3 = (T)G.K3;
  const size_t slot_stride = (size_t)G.maxcol * NV * VB;
  const int tid = threadIdx.x, nthr = blockDim.x;
  // Colour c + 2's stored f rows (VB values per cell and VDF) and state rows are copied into the
  // staging area by bulk copies while colour c is computed; one thread per copy, the cell index
  // loaded before the wait so that its latency is hidden.
  constexpr unsigned kRowBytes = VB * sizeof(S), kStBytes = SL * sizeof(T);
  auto colour_bytes = [&](int c) { return (unsigned)(A.col_off[c + 1] - A.col_off[c]) * (NV * kRowBytes + kStBytes); };
  auto prefetch_cell = [&](int c) {
    if (c >= G.ncol) return 0;
    const int off = A.col_off[c], cnt = A.col_off[c + 1] - off;
    return tid < cnt * (NV + 1) ? __ldg(&natcell[off + tid / (NV + 1)].x) : 0;
  };
  auto issue = [&](int c, int cell0) {
    const int off = A.col_off[c], cnt = A.col_off[c + 1] - off;
    for (int i = tid; i < cnt * (NV + 1); i += nthr) {
      const int p = i / (NV + 1), q = i - p * (NV + 1);
      const int cell = i == tid ? cell0 : __ldg(&natcell[off + p].x);
      if (q < NV)
        bulk_copy(rawf + (size_t)(p * NV + q) * VB, F[q] + (size_t)cell * VB, kRowBytes, bar);
      else
        bulk_copy(rawst + (size_t)p * SL, state_of(A.st, cell), kStBytes, bar);
    }
  };
  // Each colour is one phase of the mbarrier; on a time-out the block flags the error, waits
  // once more (bounded) for its copies in flight and leaves.
  unsigned phase = 0;
  auto await = [&]() {
    const bool ok = mbar_wait(bar, phase & 1u);
    ++phase;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicCAS(A.err, 0, GSIS_ERR_TIMEOUT);
        mbar_wait(bar, (phase - 1) & 1u);
      }
      return false;
    }
    return true;
  };
  auto stage = [&](int c) {
    const int off = A.col_off[c], cnt = A.col_off[c + 1] - off;
    T *slot = ring + (size_t)(c % 3) * slot_stride;
    for (int p = warp; p < cnt; p += nw) {
      T st[SL], stored[NV], f[NV];
      if constexpr (GM) {
        const int cell = __ldg(&natcell[off + p].x);
        load_state<SL>(state_of(A.st, cell), st);
#pragma unroll
        for (int q = 0; q < NV; ++q) stored[q] = Fio<T, S>::ld(F[q] + (size_t)cell * VB + lane);
      } else {
        load_state_shared<T>(rawst + (size_t)p * SL, st, SL);
#pragma unroll
        for (int q = 0; q < NV; ++q) stored[q] = Fio<T, S>::ld(rawf + (size_t)(p * NV + q) * VB + lane);
      }
      if constexpr (FX) {
        // this lane's factor of Maxwellian fj (state slots 0..4: W^n, 5..9: W^{n-1/2})
        const T ua = fa == 0 ? (fj ? st[5] : st[0]) : (fa == 1 ? (fj ? st[6] : st[1]) : (fj ? st[7] : st[2]));
        const T dv = fon ? fnode - ua : (T)0;
        const T e = dexp(-dv * dv * (fj ? st[8] : st[3]));
        if (fon && !fj) fcache[(size_t)((c & 1) * G.maxcol + p) * KFAC_MAX + lane] = e;
        const T mn = st[4] * __shfl_sync(0xffffffffu, e, src[0]) * __shfl_sync(0xffffffffu, e, src[1]) *
                     __shfl_sync(0xffffffffu, e, src[2]);
        const T mo = st[9] * __shfl_sync(0xffffffffu, e, NF + src[0]) * __shfl_sync(0xffffffffu, e, NF + src[1]) *
                     __shfl_sync(0xffffffffu, e, NF + src[2]);
        f[0] = st[10] * stored[0] + mn - mo;
      } else {
        corrected_all<T, S, NV>(stored, st, xi[0], xi[1], xi[2], f);
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) slot[(p * NV + q) * VB + lane] = f[q];
    }
  };

  if constexpr (GM) {
    stage(0);
  } else {
  if (tid == 0) {
    mbar_init(bar);
    mbar_expect(bar, colour_bytes(0));
  }
  __syncthreads();
  issue(0, prefetch_cell(0));
  int pf = prefetch_cell(1);
  if (!await()) return;
  stage(0);
  if (tid == 0 && G.ncol > 1) mbar_expect(bar, colour_bytes(1));
  __syncthreads();
  if (G.ncol > 1) issue(1, pf);
  }
  int pf = 0;
  for (int c = 0; c < G.ncol; ++c) {
    if constexpr (GM) {
      if (c + 1 < G.ncol) stage(c + 1);
      __syncthreads();
    } else {
    pf = prefetch_cell(c + 2);
    if (c + 1 < G.ncol) {
      if (!await()) return;
      stage(c + 1);
      if (tid == 0 && c + 2 < G.ncol) mbar_expect(bar, colour_bytes(c + 2));
    }
    __syncthreads();
    if (c + 2 < G.ncol) issue(c + 2, pf);
    }
    const T *slotm = ring + (size_t)((c + 2) % 3) * slot_stride;
    const T *slot0 = ring + (size_t)(c % 3) * slot_stride;
    const T *slotp = ring + (size_t)((c + 1) % 3) * slot_stride;
    const int off = A.col_off[c], cnt = A.col_off[c + 1] - off;
    for (int p = warp; p < cnt; p += nw) {
      const int4 nc4 = __ldg(&natcell[off + p]);
      const int cell = nc4.x;
      const int nat[3] = {nc4.y, nc4.z, nc4.w};
      const EntryInfo &E = entry_of(A.entry, off + p);
      int nb[6], trn[3];
#pragma unroll
      for (int q = 0; q < 2 * NACT; ++q) nb[q] = __ldg(&E.nb[q]);
#pragma unroll
      for (int q = 0; q < NACT; ++q) trn[q] = __ldg(&E.trn[q]);
      T fi[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) fi[q] = slot0[(p * NV + q) * VB + lane];
      constexpr int CL = NV == 2 ? NST_RYKOV : 16;
      T st[CL];
      load_state<CL>(state_of(A.st, cell), st);
      // gradient (LSQ, decoupled per axis on a rectilinear grid) and bounds, per VDF
      T gr[NV][3], rlo[3], rhi[3], invh[3];
      T fmax[NV], fmin[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) fmax[q] = fmin[q] = fi[q];
      T V = (T)1;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const AxisCell<T> gc = A.ax[a][nat[a]];
        V *= gc.h;
        if (a < NACT) {
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            T fup = fi[q], fdn = fi[q];
            if (nb[2 * a] >= 0) {
              fup = slotm[(nb[2 * a] * NV + q) * VB + lane];
              fmax[q] = larger(fmax[q], fup);
              fmin[q] = smaller(fmin[q], fup);
            }
            if (nb[2 * a + 1] >= 0) {
              fdn = slotp[(nb[2 * a + 1] * NV + q) * VB + lane];
              fmax[q] = larger(fmax[q], fdn);
              fmin[q] = smaller(fmin[q], fdn);
            }
            const T flo = sg[a] > 0 ? fup : fdn, fhi = sg[a] > 0 ? fdn : fup;
            gr[q][a] = gc.clo * (flo - fi[q]) + gc.chi * (fhi - fi[q]);
          }
          rlo[a] = gc.rlo;
          rhi[a] = gc.rhi;
          invh[a] = gc.invh;
        }
      }
      // the implicit diagonal D = 1/dt + 1/tau + the outflow coefficients, then the limiter.  In
      // FP64 one reciprocal r = 1 / (bd D) gives both phi = bn / bd = bn D r and the update's
      // 1 / D = bd r (an FP64 division costs several FP64 instructions on this GPU)
      T D = st[15];
#pragma unroll
      for (int a = 0; a < NACT; ++a) D += axi[a] * invh[a];
      T phi[NV], invD[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if constexpr (std::is_same<T, double>::value) {
          T bn, bd;
          venkat_parts<T, NACT>(fi[q], fmax[q], fmin[q], gr[q], rlo, rhi, K3 * V, bn, bd);
          const T r = (T)1 / (bd * D);
          phi[q] = bn * D * r;
          invD[q] = bd * r;
        } else {
          phi[q] = venkat_phi<T, NACT>(fi[q], fmax[q], fmin[q], gr[q], rlo, rhi, K3 * V);
          invD[q] = (T)0;
        }
      }
      // reference distributions of the state W^n
      const T cx = xi[0] - st[0], cy = xi[1] - st[1], cz = xi[2] - st[2];
      const T c2 = cx * cx + cy * cy + cz * cz;
      T mw, g[NV];  // mw: Maxwellian of W^n
      if constexpr (FX) {
        // M(W^n) from the cached factors (the product the staging formed for Eq. updatef), then
        // the Shakhov g_0t of Section 2.2
        const T *fc = fcache + (size_t)((c & 1) * G.maxcol + p) * KFAC_MAX;
        mw = st[4] * fc[src[0]] * fc[src[1]] * fc[src[2]];
        g[0] = mw * ((T)1 + (st[12] * cx + st[13] * cy + st[14] * cz) * (c2 * st[3] - (T)2.5));
      } else {
        reference<T, NV>(st, cx, cy, cz, c2, mw, g);
      }
      T acc[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = (g[q] - fi[q]) * st[11];
      T fout[NV][3];
#pragma unroll
      for (int a = 0; a < NACT; ++a) {
        const T k = axi[a] * invh[a];
        T rho_w = (T)0;
        if (nb[2 * a] < 0) {
          // upwind boundary: the natural transverse index of the wall face
          const int trw = a == 0 ? nat[1] + n1 * nat[2] : (a == 1 ? nat[0] + n0 * nat[2] : nat[0] + n0 * nat[1]);
          rho_w = (T)A.rho_w[G.wall_base[upside[a]] + trw];
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          fout[q][a] = fi[q] + phi[q] * gr[q][a] * (sg[a] > 0 ? rhi[a] : rlo[a]);
          const T ein = nb[2 * a] >= 0 ? ebuf[a][(trn[a] * NV + q) * VB + lane] : rho_w * (q == 0 ? Mw[a] : Mw1[a]);
          acc[q] -= k * (fout[q][a] - ein);
        }
      }
      T df[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if constexpr (std::is_same<T, double>::value) df[q] = acc[q] * invD[q];
        else df[q] = ddiv(acc[q], D);
        // relative storage keeps the deviation from the reference: M_t for f0, (d_r Tr_n / 4) M_t for f1
        const T ref = q == 0 ? mw : st[NV == 2 ? 29 : 0] * mw;
        Fio<T, S>::st(F[q] + (size_t)cell * VB + lane, StoredRelative<S>::value ? fi[q] + df[q] - ref : fi[q] + df[q]);
      }
#pragma unroll
      for (int a = 0; a < NACT; ++a) {
        T eout[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          eout[q] = fout[q][a] + df[q];
          ebuf[a][(trn[a] * NV + q) * VB + lane] = eout[q];
        }
        if (nb[2 * a + 1] < 0) {
          // outflow face on the domain boundary (a wall): moments of the flux towards the wall
          const int trw = a == 0 ? nat[1] + n1 * nat[2] : (a == 1 ? nat[0] + n0 * nat[2] : nat[0] + n0 * nat[1]);
          const int wid = G.wall_base[2 * a + (sg[a] > 0 ? 1 : 0)] + trw;
          const T fl = wv * xi[a] * eout[0];
          const T e1 = NV == 2 ? wv * xi[a] * eout[NV - 1] : (T)0;
          const T m0 = warp_sum(fl), m1 = warp_sum(fl * xi[0]), m2 = warp_sum(fl * xi[1]);
          const T m3 = warp_sum(fl * xi[2]), m4 = warp_sum(fl * e2 + e1);
          const T m5 = NV == 2 ? warp_sum(e1) : (T)0;
          if (lane == 0) {
            T *W = A.wpart + ((size_t)b * A.nwall + wid) * NWF;
            W[0] = m0;
            W[1] = m1;
            W[2] = m2;
            W[3] = m3;
            W[4] = m4;
            W[5] = m5;
          }
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, typename S>
size_t kinetic_smem_bytes(const KinGeom &g, int nvdf) {
  const int sl = nvdf == 2 ? stage_state_len<S, 2>() : stage_state_len<S, 1>();
  return KinSmem<T, S>(g, nvdf, sl, factored<T, S>(g, nvdf)).total;
}

// the ring and face buffers only (the bulk-copy staging area is not used from global memory),
// rounded to 256 bytes so that every block's slice starts on an aligned boundary
template <typename T, typename S>
size_t kinetic_gscratch_stride(const KinGeom &g, int nvdf) {
  const int sl = nvdf == 2 ? stage_state_len<S, 2>() : stage_state_len<S, 1>();
  return (KinSmem<T, S>(g, nvdf, sl, factored<T, S>(g, nvdf)).rawf + 255) & ~(size_t)255;
}

template <typename T, typename S, bool GM>
static void (*kinetic_fn_gm(int nact, int nvdf, bool fx))(const KinArgs<T, S>) {
  if (nvdf == 2)
    return nact == 1 ? kinetic_kernel<T, S, 1, 2, GM, false>
                     : (nact == 2 ? kinetic_kernel<T, S, 2, 2, GM, false> : kinetic_kernel<T, S, 3, 2, GM, false>);
  if constexpr (std::is_same<T, double>::value && std::is_same<S, double>::value) {
    if (fx)
      return nact == 1 ? kinetic_kernel<T, S, 1, 1, GM, true>
                       : (nact == 2 ? kinetic_kernel<T, S, 2, 1, GM, true> : kinetic_kernel<T, S, 3, 1, GM, true>);
  }
  return nact == 1 ? kinetic_kernel<T, S, 1, 1, GM, false>
                   : (nact == 2 ? kinetic_kernel<T, S, 2, 1, GM, false> : kinetic_kernel<T, S, 3, 1, GM, false>);
}

template <typename T, typename S>
static void (*kinetic_fn(const KinGeom &g, int nvdf, bool gm))(const KinArgs<T, S>) {
  const bool fx = factored<T, S>(g, nvdf);
  return gm ? kinetic_fn_gm<T, S, true>(g.nact, nvdf, fx) : kinetic_fn_gm<T, S, false>(g.nact, nvdf, fx);
}

template <typename T, typename S>
cudaError_t kinetic_shape(const KinGeom &g, int nvdf, bool gm, int want_warps, size_t smem, int *warps,
                          int *ctas_per_sm) {
  void (*k)(const KinArgs<T, S>) = kinetic_fn<T, S>(g, nvdf, gm);
  cudaFuncAttributes attr;
  cudaError_t e = cudaFuncGetAttributes(&attr, k);
  if (e != cudaSuccess) return e;
  *warps = std::max(1, std::min(want_warps, attr.maxThreadsPerBlock / 32));
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, *warps * 32, smem);
}

template <typename T, typename S>
cudaError_t launch_kinetic(const KinArgs<T, S> &a, int nblocks, int nwarps, size_t smem, cudaStream_t s) {
  void (*k)(const KinArgs<T, S>) = kinetic_fn<T, S>(a.g, a.nvdf, a.gscratch != nullptr);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<nblocks, nwarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Diffuse-wall pre-pass: rho_w of each wall face balances the mass flux of the molecules that
// reach the wall, whose face values are the wall cell's limited reconstruction of f^n.

template <typename T, typename S, int NACT>
__global__ void wall_prepass_kernel(const KinArgs<T, S> A, const int *wall_cell, const int *wall_side,
                                    const double *Z0, double *rho_w, int nslots) {
  const KinGeom &G = A.g;
  const int wf = blockIdx.x;
  const int cell = wall_cell[wf], side = wall_side[wf], axn = side / 2;
  const double dir = (side & 1) ? 1.0 : -1.0;
  const int n0 = G.n[0], n1 = G.n[1];
  const int nat[3] = {cell % n0, (cell / n0) % n1, cell / (n0 * n1)};
  const int stride[3] = {1, n0, n0 * n1};
  constexpr int SL = state_len<S>();
  T st[SL], stn[3][2][SL];
  load_state<SL>(A.st + (size_t)cell * NST, st);
  bool has[3][2];
#pragma unroll
  for (int a = 0; a < NACT; ++a) {
    has[a][0] = nat[a] > 0;
    has[a][1] = nat[a] < G.n[a] - 1;
    if (has[a][0]) load_state<SL>(A.st + (size_t)(cell - stride[a]) * NST, stn[a][0]);
    if (has[a][1]) load_state<SL>(A.st + (size_t)(cell + stride[a]) * NST, stn[a][1]);
  }
  AxisCell<T> gc[3];
  T V = (T)1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gc[a] = A.ax[a][nat[a]];
    V *= gc[a].h;
  }
  double acc = 0.0;
  for (int v = threadIdx.x; v < nslots; v += blockDim.x) {
    const T *vp = A.vel + (size_t)v * 4;
    const T x = vp[0], y = vp[1], z = vp[2], w = vp[3];
    const T xa = axn == 0 ? x : (axn == 1 ? y : z);
    // (the direction test and the product in the arithmetic type: FP64 conversions, compares
    // and products per velocity would run at the FP64 rate; dir = +-1 keeps them exact)
    if (!(w > (T)0) || !(xa * (T)dir > (T)0)) continue;
    const int blk = v / VB, ln = v % VB;
    const S *Fb = A.f + (size_t)blk * G.nc * VB;
    const T fi = corrected_stored<T, S>(Fio<T, S>::ld(Fb + (size_t)cell * VB + ln), st, x, y, z);
    T gr[3], rlo[3], rhi[3], fmax = fi, fmin = fi;
#pragma unroll
    for (int a = 0; a < NACT; ++a) {
      T flo = fi, fhi = fi;
      if (has[a][0]) flo = corrected_stored<T, S>(Fio<T, S>::ld(Fb + (size_t)(cell - stride[a]) * VB + ln), stn[a][0], x, y, z);
      if (has[a][1]) fhi = corrected_stored<T, S>(Fio<T, S>::ld(Fb + (size_t)(cell + stride[a]) * VB + ln), stn[a][1], x, y, z);
      if (has[a][0]) { fmax = larger(fmax, flo); fmin = smaller(fmin, flo); }
      if (has[a][1]) { fmax = larger(fmax, fhi); fmin = smaller(fmin, fhi); }
      gr[a] = gc[a].clo * (flo - fi) + gc[a].chi * (fhi - fi);
      rlo[a] = gc[a].rlo;
      rhi[a] = gc[a].rhi;
    }
    const T phi = venkat_phi<T, NACT>(fi, fmax, fmin, gr, rlo, rhi, (T)G.K3 * V);
    const T r = (side & 1) ? rhi[axn] : rlo[axn];
    const T face = fi + phi * gr[axn] * r;
    acc += (double)(w * fabs(xa) * face);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) rho_w[wf] = red[0] / Z0[side];
}

template <typename T, typename S>
cudaError_t launch_wall_prepass(const KinArgs<T, S> &a, const int *wall_cell, const int *wall_side, int nwall,
                                const double *Z0, double *rho_w, int nslots, cudaStream_t s) {
  if (nwall == 0) return cudaSuccess;
  if (a.g.nact == 1) wall_prepass_kernel<T, S, 1><<<nwall, 256, 0, s>>>(a, wall_cell, wall_side, Z0, rho_w, nslots);
  else if (a.g.nact == 2) wall_prepass_kernel<T, S, 2><<<nwall, 256, 0, s>>>(a, wall_cell, wall_side, Z0, rho_w, nslots);
  else wall_prepass_kernel<T, S, 3><<<nwall, 256, 0, s>>>(a, wall_cell, wall_side, Z0, rho_w, nslots);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Wall constants: for each wall side, over the velocities leaving the wall into the gas,
//   Z0 = sum w |xi_n| M_w  and  Zw[m] = sum w xi_a phi_m M_w (signed, +e_a direction),
// phi = 1, xi(3), |xi|^2/2 and the internal-energy factor d_r T_w / 4 (Rykov).
__global__ void wall_constants_kernel(const double *vel64, int nslots, const double *wall_uT, const int *sides,
                                      double *Z0, double *Zw, double d_r) {
  const int side = sides[blockIdx.x], a = side / 2;
  const double dir = (side & 1) ? 1.0 : -1.0;
  const double *uT = wall_uT + 4 * side;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const double norm = pow(3.14159265358979323846 * uT[3], -1.5);
  for (int v = threadIdx.x; v < nslots; v += blockDim.x) {
    const double x = vel64[4 * v], y = vel64[4 * v + 1], z = vel64[4 * v + 2], w = vel64[4 * v + 3];
    const double xa = a == 0 ? x : (a == 1 ? y : z);
    if (!(w > 0.0) || !(xa * dir < 0.0)) continue;
    const double cx = x - uT[0], cy = y - uT[1], cz = z - uT[2];
    const double M = norm * exp(-(cx * cx + cy * cy + cz * cz) / uT[3]);
    const double fl = w * xa * M;
    acc[0] += w * fabs(xa) * M;
    acc[1] += fl;
    acc[2] += fl * x;
    acc[3] += fl * y;
    acc[4] += fl * z;
    acc[5] += fl * (0.5 * (x * x + y * y + z * z) + d_r * uT[3] / 4.0);
    acc[6] += fl * d_r * uT[3] / 4.0;
  }
  __shared__ double red[7][256];
  for (int q = 0; q < 7; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 7; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Z0[side] = red[0][0];
    for (int q = 0; q < 6; ++q) Zw[6 * side + q] = red[1 + q][0];
  }
}

cudaError_t launch_wall_constants(const double *vel64, int nslots, const double *wall_uT, const int *sides,
                                  int nsides, double *Z0, double *Zw, double d_r, cudaStream_t s) {
  if (nsides == 0) return cudaSuccess;
  wall_constants_kernel<<<nsides, 256, 0, s>>>(vel64, nslots, wall_uT, sides, Z0, Zw, d_r);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Moments of the stored f (Eq. getmoment) streamed after the kinetic step: one thread owns one
// cell and a chunk of velocity blocks, reads the block's 32 values of its cell as vectors and
// accumulates, about the state velocity u_n,
//   13 raw moments of f (1, c, cc, |c|^2 c)  and  5 moments of w (g^n - f) (1, xi, |xi|^2/2).
// The second set gives, through the discrete identity of the delta-form equation with 1/dt = 0,
//   sum over the cell's faces of the outward kinetic flux = V sum_v w phi (g^n - f^{n+1/2}) / tau,
// the only kinetic-flux information the synthetic solve needs.  Sums over one block (32 terms)
// are plain, and are added into compensated (Kahan) accumulators across blocks.
template <typename T, int N>
struct MomAcc {
  T s[N], c[N];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = c[k] = (T)0;
  }
  __device__ void add(const T *x) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T y = x[k] - c[k];
      const T t = s[k] + y;
      c[k] = (t - s[k]) - y;
      s[k] = t;
    }
  }
};

template <typename T, typename S>
__device__ __forceinline__ void load_block_f(const S *p, T *f);
template <>
__device__ __forceinline__ void load_block_f<float, float>(const float *p, float *f) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 v = __ldcs(q + i);
    f[4 * i] = v.x;
    f[4 * i + 1] = v.y;
    f[4 * i + 2] = v.z;
    f[4 * i + 3] = v.w;
  }
}
template <>
__device__ __forceinline__ void load_block_f<float, __nv_bfloat16>(const __nv_bfloat16 *p, float *f) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint4 v = __ldcs(q + i);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // a 32-bit word holds two BF16 values, the lower-addressed one in the low half; a BF16
      // value is the upper 16 bits of the FP32 value it widens to
      f[8 * i + 2 * j] = __uint_as_float(w[j] << 16);
      f[8 * i + 2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
    }
  }
}
template <>
__device__ __forceinline__ void load_block_f<double, double>(const double *p, double *f) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const double2 v = __ldcs(q + i);
    f[2 * i] = v.x;
    f[2 * i + 1] = v.y;
  }
}

template <typename T, typename S, int NV>
__global__ void __launch_bounds__(128) moments_kernel(const KinArgs<T, S> A, int blocks_per_chunk, double *mp) {
  constexpr int NP = moment_len(NV);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *svel = reinterpret_cast<T *>(smem_raw);  // [blocks_per_chunk * VB][4]
  const KinGeom &G = A.g;
  const int chunk = blockIdx.y;
  const int b0 = chunk * blocks_per_chunk;
  const int nb = min(blocks_per_chunk, A.nblocks - b0);
  for (int i = threadIdx.x; i < nb * VB * 4; i += blockDim.x) svel[i] = A.vel[(size_t)b0 * VB * 4 + i];
  __syncthreads();
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= G.nc) return;
  constexpr int CL = NV == 2 ? NST_RYKOV : 16;
  T st[CL];
  load_state<CL>(A.st + (size_t)cell * NST, st);
  MomAcc<T, NP> acc;
  acc.zero();
  for (int bb = 0; bb < nb; ++bb) {
    T f[VB], f1[NV == 2 ? VB : 1];
    load_block_f<T, S>(A.f + ((size_t)(b0 + bb) * G.nc + cell) * VB, f);
    if constexpr (NV == 2) load_block_f<T, S>(A.f1 + ((size_t)(b0 + bb) * G.nc + cell) * VB, f1);
    T sum[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) sum[k] = (T)0;
#pragma unroll
    for (int l = 0; l < VB; ++l) {
      const T *v = svel + (bb * VB + l) * 4;
      const T x = v[0], y = v[1], z = v[2], w = v[3];
      const T cx = x - st[0], cy = y - st[1], cz = z - st[2];
      const T c2 = cx * cx + cy * cy + cz * cz;
      T mw, g[NV];  // Maxwellian of W^n (the storage reference of this step) and the reference
      if constexpr (NV == 1) {
        mw = st[4] * dexp(-c2 * st[3]);
      } else {
        reference<T, NV>(st, cx, cy, cz, c2, mw, g);
      }
      const T wf = w * (StoredRelative<S>::value ? f[l] + mw : f[l]);
      sum[0] += wf;
      sum[1] += wf * cx;
      sum[2] += wf * cy;
      sum[3] += wf * cz;
      sum[4] += wf * cx * cx;
      sum[5] += wf * cy * cy;
      sum[6] += wf * cz * cz;
      sum[7] += wf * cx * cy;
      sum[8] += wf * cx * cz;
      sum[9] += wf * cy * cz;
      sum[10] += wf * c2 * cx;
      sum[11] += wf * c2 * cy;
      sum[12] += wf * c2 * cz;
      T d, d1 = (T)0;
      if constexpr (NV == 1) {
        const T shak = (st[12] * cx + st[13] * cy + st[14] * cz) * (c2 * st[3] - (T)2.5);
        // w (g - f): with relative storage g - f = M shak - (f - M) needs no difference of O(1)
        // values (the sum is multiplied by 1/tau, which at small Kn would amplify that round-off)
        d = StoredRelative<S>::value ? w * (mw * shak - f[l]) : w * (mw * ((T)1 + shak)) - wf;
      } else {
        const T wf1 = w * (StoredRelative<S>::value ? f1[l] + st[29] * mw : f1[l]);
        d = w * g[0] - wf;
        d1 = w * g[NV - 1] - wf1;
        sum[NMOM + NFF + 1] += wf1;
        sum[NMOM + NFF + 2] += wf1 * cx;
        sum[NMOM + NFF + 3] += wf1 * cy;
        sum[NMOM + NFF + 4] += wf1 * cz;
        sum[NMOM + NFF] += d1;
      }
      sum[13] += d;
      sum[14] += d * x;
      sum[15] += d * y;
      sum[16] += d * z;
      sum[17] += d * (T)0.5 * (x * x + y * y + z * z) + d1;
    }
    acc.add(sum);
  }
  double *out = mp + ((size_t)chunk * G.nc + cell) * NP;
#pragma unroll
  for (int k = 0; k < NP; ++k) out[k] = (double)acc.s[k] - (double)acc.c[k];
}

template <typename T, typename S>
cudaError_t launch_moments(const KinArgs<T, S> &a, int blocks_per_chunk, int nchunks, double *mp, cudaStream_t s) {
  const size_t smem = (size_t)blocks_per_chunk * VB * 4 * sizeof(T);
  auto k = a.nvdf == 2 ? moments_kernel<T, S, 2> : moments_kernel<T, S, 1>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.g.nc + 127) / 128, nchunks);
  k<<<grid, 128, smem, s>>>(a, blocks_per_chunk, mp);
  return cudaGetLastError();
}

// FP64 storage with the Shakhov model: the 13 moments of the stored f^{n+1/2} about the origin,
// sum_v f_v t_k(v) with the per-slot table t_k = w (1, xi(3), xi_a xi_b (6), |xi|^2 xi(3)) (16
// doubles per slot, the last three 0): one FMA per moment and point and no exponential.  The
// collision sums sum_v w phi (g^n - f) are assembled per cell by the reduction from the closed
// form of sum_v w phi g^n (ref_sums_kernel) and these moments.  Per-block plain sums, compensated
// (Kahan) across the chunk's blocks, as in moments_kernel.
__global__ void __launch_bounds__(128) moments_origin_kernel(const KinArgs<double, double> A, const double *mtab,
                                                             int blocks_per_chunk, double *mp) {
  const int chunk = blockIdx.y;
  const int b0 = chunk * blocks_per_chunk;
  const int nb = min(blocks_per_chunk, A.nblocks - b0);
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= A.g.nc) return;
  MomAcc<double, NMOM> acc;
  acc.zero();
  for (int bb = 0; bb < nb; ++bb) {
    double f[VB];
    load_block_f<double, double>(A.f + ((size_t)(b0 + bb) * A.g.nc + cell) * VB, f);
    const double2 *tb = reinterpret_cast<const double2 *>(mtab + (size_t)(b0 + bb) * VB * 16);
    double sum[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) sum[k] = 0.0;
#pragma unroll
    for (int l = 0; l < VB; ++l) {
      double t[14];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const double2 v = __ldg(tb + l * 8 + q);
        t[2 * q] = v.x;
        t[2 * q + 1] = v.y;
      }
#pragma unroll
      for (int k = 0; k < NMOM; ++k) sum[k] = fma(f[l], t[k], sum[k]);
    }
    acc.add(sum);
  }
  double *out = mp + ((size_t)chunk * A.g.nc + cell) * (NMOM + NFF);
#pragma unroll
  for (int k = 0; k < NMOM; ++k) out[k] = acc.s[k] - acc.c[k];
#pragma unroll
  for (int k = NMOM; k < NMOM + NFF; ++k) out[k] = 0.0;
}

// Closed form of sum_v w phi(xi) g^n(xi), phi = 1, xi(3), |xi|^2/2, for the Shakhov g_0t of
// Section 2.2 on a tensor-product velocity grid: with c = xi - u and
// g = C e^{-|c|^2/T} [1 + a.c (|c|^2/T - 5/2)], every term is a polynomial in c times a product
// of one-dimensional Gaussians, so the sum over the grid factorises into the one-dimensional
// sums m_a[k] = sum_i w_a(i) e^{-c_a(i)^2/T} c_a(i)^k (k <= 5).  One thread per cell writes its
// row of the extra moment chunk (moments 0, collision sums in slots 13..17); emit = 0 (the
// velocity shards other than the first) writes zeros, so the sum over shards counts it once.
__global__ void ref_sums_kernel(int nc, const double *st64, const double *vaxis, int nx, int ny, int nz, int emit,
                                double *row) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= nc) return;
  double *o = row + (size_t)cell * (NMOM + NFF);
#pragma unroll
  for (int k = 0; k < NMOM + NFF; ++k) o[k] = 0.0;
  if (!emit) return;
  const double *st = st64 + (size_t)cell * NST;
  const double u[3] = {st[0], st[1], st[2]}, invT = st[3], C = st[4], aq[3] = {st[12], st[13], st[14]};
  const int n[3] = {nx, ny, nz};
  const double *xs[3] = {vaxis, vaxis + nx, vaxis + nx + ny};
  const double *ws[3] = {vaxis + nx + ny + nz, vaxis + 2 * nx + ny + nz, vaxis + 2 * nx + 2 * ny + nz};
  double m[3][6];
  for (int a = 0; a < 3; ++a) {
    for (int k = 0; k < 6; ++k) m[a][k] = 0.0;
    for (int i = 0; i < n[a]; ++i) {
      const double c = xs[a][i] - u[a];
      double p = ws[a][i] * exp(-c * c * invT);
      for (int k = 0; k < 6; ++k) {
        m[a][k] += p;
        p *= c;
      }
    }
  }
  auto mono = [&](int px, int py, int pz) { return m[0][px] * m[1][py] * m[2][pz]; };
  // sum_v w g c^e for the exponent triple e
  auto G = [&](int px, int py, int pz) {
    double t1 = 0.0;
    for (int b = 0; b < 3; ++b) {
      const int e[3] = {px + (b == 0), py + (b == 1), pz + (b == 2)};
      const double s3 = mono(e[0] + 2, e[1], e[2]) + mono(e[0], e[1] + 2, e[2]) + mono(e[0], e[1], e[2] + 2);
      t1 += aq[b] * (invT * s3 - 2.5 * mono(e[0], e[1], e[2]));
    }
    return C * (mono(px, py, pz) + t1);
  };
  const double g1 = G(0, 0, 0);
  const double gc[3] = {G(1, 0, 0), G(0, 1, 0), G(0, 0, 1)};
  const double gc2 = G(2, 0, 0) + G(0, 2, 0) + G(0, 0, 2);
  o[NMOM] = g1;
  for (int a = 0; a < 3; ++a) o[NMOM + 1 + a] = gc[a] + u[a] * g1;
  o[NMOM + 4] = 0.5 * gc2 + (u[0] * gc[0] + u[1] * gc[1] + u[2] * gc[2]) +
                0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * g1;
}

cudaError_t launch_moments_origin(const KinArgs<double, double> &a, const double *mtab, int blocks_per_chunk,
                                  int nchunks, const double *st64, const double *vaxis, const int *nv_axis, int emit,
                                  double *mp, cudaStream_t s) {
  dim3 grid((a.g.nc + 127) / 128, nchunks);
  moments_origin_kernel<<<grid, 128, 0, s>>>(a, mtab, blocks_per_chunk, mp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ref_sums_kernel<<<(a.g.nc + 127) / 128, 128, 0, s>>>(a.g.nc, st64, vaxis, nv_axis[0], nv_axis[1], nv_axis[2], emit,
                                                       mp + (size_t)nchunks * a.g.nc * (NMOM + NFF));
  return cudaGetLastError();
}

// f_raw = Maxwellian(W0) of each cell at each slot velocity, in the storage precision (the
// per-cell factor rho (pi T)^(-3/2) and 1/T in FP64, the exponential in T).  Relative (BF16,
// FP32) storage writes zero deviations from M(W0), which the initial state names as the
// reference.
__device__ __forceinline__ float accurate_exp(float x) { return expf(x); }
__device__ __forceinline__ double accurate_exp(double x) { return exp(x); }

// One warp per cell: the per-cell factors once (FP64 is scarce on this GPU), then every
// velocity block of the cell, one 128-byte line per block.
template <typename T, typename S>
__global__ void init_maxwellian_kernel(const KinArgs<T, S> A, const double *W0) {
  const KinGeom &G = A.g;
  const int lane = threadIdx.x & 31;
  const int cell = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (cell >= G.nc) return;
  const double *w0 = W0 + 6 * (size_t)cell;
  const T C = (T)(w0[0] * pow(3.14159265358979323846 * w0[4], -1.5)), invT = (T)(1.0 / w0[4]);
  const T ux = (T)w0[1], uy = (T)w0[2], uz = (T)w0[3];
  const T c1 = (T)(A.d_r * w0[5] / 4.0);  // f1 = (d_r Tr / 4) f0 (Rykov)
  for (int b = 0; b < A.nblocks; ++b) {
    const T *vp = A.vel + ((size_t)b * VB + lane) * 4;
    const T cx = vp[0] - ux, cy = vp[1] - uy, cz = vp[2] - uz;
    // relative storage: f is exactly the reference Maxwellian M(W0), stored as a zero deviation
    const T f = StoredRelative<S>::value ? (T)0 : C * accurate_exp(-(cx * cx + cy * cy + cz * cz) * invT);
    Fio<T, S>::st(A.f + ((size_t)b * G.nc + cell) * VB + lane, f);
    if (A.nvdf == 2) Fio<T, S>::st(A.f1 + ((size_t)b * G.nc + cell) * VB + lane, c1 * f);
  }
}

template <typename T, typename S>
cudaError_t launch_init_maxwellian(const KinArgs<T, S> &a, const double *W0, int nblocks, cudaStream_t s) {
  (void)nblocks;
  const int threads = 256;
  const size_t grid = ((size_t)a.g.nc * 32 + threads - 1) / threads;
  init_maxwellian_kernel<T, S><<<(unsigned)grid, threads, 0, s>>>(a, W0);
  return cudaGetLastError();
}

// Canonical [cell][v] FP64 <-> internal [block][cell][lane].  Export applies the pending
// correction (the returned f is the VDF the next kinetic step starts from).
template <typename T, typename S>
__global__ void export_f_kernel(const KinArgs<T, S> A, int q, const int *slot_canon, int nslots, int nv, double *out) {
  const size_t n = (size_t)A.g.nc * nslots;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int slot = (int)(idx % nslots);
    const int cell = (int)(idx / nslots);
    const T *vp = A.vel + (size_t)slot * 4;
    if (!(vp[3] > (T)0)) continue;
    T st[NST_RYKOV];
    load_state<NST_RYKOV>(A.st + (size_t)cell * NST, st);
    const int blk = slot / VB, ln = slot % VB;
    const size_t at = ((size_t)blk * A.g.nc + cell) * VB + ln;
    T stored[2] = {Fio<T, S>::ld(A.f + at), (T)0}, f[2];
    if (A.nvdf == 2) {
      stored[1] = Fio<T, S>::ld(A.f1 + at);
      corrected_all<T, S, 2>(stored, st, vp[0], vp[1], vp[2], f);
    } else {
      corrected_all<T, S, 1>(stored, st, vp[0], vp[1], vp[2], f);
    }
    out[(size_t)cell * nv + slot_canon[slot]] = (double)f[q];
  }
}

template <typename T, typename S>
__global__ void import_f_kernel(const KinArgs<T, S> A, int q, const int *slot_canon, int nslots, int nv, const double *in) {
  const size_t n = (size_t)A.g.nc * nslots;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int slot = (int)(idx % nslots);
    const int cell = (int)(idx / nslots);
    const int blk = slot / VB, ln = slot % VB;
    Fio<T, S>::st((q ? A.f1 : A.f) + ((size_t)blk * A.g.nc + cell) * VB + ln, (T)in[(size_t)cell * nv + slot_canon[slot]]);
  }
}

template <typename T, typename S>
cudaError_t launch_export_f(const KinArgs<T, S> &a, int q, const int *slot_canon, int nslots, int nv, double *out,
                            cudaStream_t s) {
  export_f_kernel<T, S><<<1024, 256, 0, s>>>(a, q, slot_canon, nslots, nv, out);
  return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t launch_import_f(const KinArgs<T, S> &a, int q, const int *slot_canon, int nslots, int nv, const double *in,
                            cudaStream_t s) {
  import_f_kernel<T, S><<<1024, 256, 0, s>>>(a, q, slot_canon, nslots, nv, in);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// General (curvilinear) structured meshes: O-grids with far-field, pole and wrapped sides.
//
// On a curved mesh the upwind side of a face changes with the velocity, so the colour sweeps are
// no longer exact in one pass; the kernel therefore keeps whole-mesh work arrays for its block
// of 32 velocities (in its own slice of a device scratch) and runs the steps of Section 3.2 one
// after another: f^n with the pending correction, the limited LSQ gradient, the second-order
// upwind residual with the implicit diagonal, n_sweeps point-implicit passes over the colours
// of the octant (a cell's inflow increments are the neighbours' latest), the update with the
// wall-face fluxes and, for GSIS, the per-cell kinetic face-flux sums.  A persistent grid walks
// the velocity blocks, one block per CTA at a time.  Far-field faces: the free-stream
// Maxwellian enters unless the stream leaves faster than sound (host flag gin), else the
// cell's own value; pole (AXIS) and absent sides carry no flux.

template <typename T>
__device__ __forceinline__ T dot_xi(const T *S, T x, T y, T z) {
  return x * S[0] + y * S[1] + z * S[2];
}

// The kinetic face value from the cell value fi and its limited increment d = phi grad f . r: fi + d,
// or with positive faces fi^2 / (fi - d) where d < 0 (positive whenever fi is; equal to fi + d to
// first order in d / fi, the two differing by d^2 / (fi - d)); a non-positive fi keeps its value.
template <typename T>
__device__ __forceinline__ T face_value(T fi, T d, int pos) {
  if (pos && d < (T)0) return fi > (T)0 ? ddiv(fi * fi, fi - d) : fi;
  return fi + d;
}

// Venkatakrishnan factor of one cell from its unlimited gradient gr and neighbour bounds: the
// minimum over its faces (not the absent or pole sides) of
//   (Dm^2 + e^2 + 2 D2 Dm) / (Dm^2 + 2 D2^2 + D2 Dm + e^2),  D2 = gr . r,
// Dm the bound on the side of D2; faces with D2 = 0 give 1.  Both parts are positive, so the
// minimum is found by cross-multiplication and divided once.
template <typename T>
__device__ __forceinline__ T venkat_general(const GenCell<T> &g, const int *nb, T fi, T fmax, T fmin, const T *gr) {
  T bn = (T)1, bd = (T)1;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    if (nb[s] == NB_ABSENT || nb[s] == NB_AXIS) continue;
    const T d2 = gr[0] * g.f[s].r[0] + gr[1] * g.f[s].r[1] + gr[2] * g.f[s].r[2];
    if (d2 == (T)0) continue;
    const T dm = d2 > (T)0 ? fmax - fi : fmin - fi;
    const T dm2 = dm * dm + g.eps2;
    const T n = dm2 + (T)2 * d2 * dm;
    const T d = dm2 + d2 * ((T)2 * d2 + dm);
    if (n * bd < bn * d) {
      bn = n;
      bd = d;
    }
  }
  return ddiv(bn, bd);
}

template <typename T, typename S, int NV, int NACT>
__global__ void __launch_bounds__(256) kinetic_general_kernel(const KinArgs<T, S> A) {
  constexpr int NF = 2 * NACT;  // sides of the active axes (the others carry no transport)
  const KinGeom &G = A.g;
  const int nc = G.nc, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int SL = stage_state_len<S, NV>();
  constexpr int CL = NV == 2 ? NST_RYKOV : 16;
  // work arrays of this CTA: f^n, the limited face values of every active side, residual and
  // increment [cell][q][...][VB]; the implicit diagonal [cell][VB]
  T *fc = reinterpret_cast<T *>(A.gscratch + (size_t)blockIdx.x * A.gstride);
  T *ffs = fc + (size_t)nc * NV * VB;
  T *rs = ffs + (size_t)nc * NV * NF * VB;
  T *dfs = rs + (size_t)nc * NV * VB;
  T *ds = dfs + (size_t)nc * NV * VB;
  auto FC = [&](int c, int q) -> T & { return fc[((size_t)c * NV + q) * VB + lane]; };
  auto FF = [&](int c, int q, int s) -> T & { return ffs[(((size_t)c * NV + q) * NF + s) * VB + lane]; };
  auto DF = [&](int c, int q) -> T & { return dfs[((size_t)c * NV + q) * VB + lane]; };
  for (int b = blockIdx.x; b < A.nblocks; b += gridDim.x) {
    const int oct = A.boct[b];
    const T *vp = A.vel + ((size_t)b * VB + lane) * 4;
    const T x = vp[0], y = vp[1], z = vp[2], wv = vp[3];
    const T e2 = (T)0.5 * (x * x + y * y + z * z);
    S *F[NV];
    F[0] = A.f + (size_t)b * nc * VB;
    if constexpr (NV == 2) F[NV - 1] = A.f1 + (size_t)b * nc * VB;
    // f^n of every cell (Eq. updatef applied on load); the increments start at zero
    for (int c = warp; c < nc; c += nw) {
      T st[SL], stored[NV], f[NV];
      load_state<SL>(state_of(A.st, c), st);
#pragma unroll
      for (int q = 0; q < NV; ++q) stored[q] = Fio<T, S>::ld(F[q] + (size_t)c * VB + lane);
      corrected_all<T, S, NV>(stored, st, x, y, z, f);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        FC(c, q) = f[q];
        DF(c, q) = (T)0;
      }
    }
    __syncthreads();
    // limited least-squares reconstruction: the face value of every active side
    for (int c = warp; c < nc; c += nw) {
      const GenCell<T> &g = A.gen[c];
      int nb[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) nb[s] = s < NF ? __ldg(A.gnb + 6 * c + s) : NB_ABSENT;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const T fi = FC(c, q);
        T fj[NF];
#pragma unroll
        for (int s = 0; s < NF; ++s) fj[s] = nb[s] >= 0 ? FC(nb[s], q) : fi;
        T gr[3] = {(T)0, (T)0, (T)0}, fmax = fi, fmin = fi;
#pragma unroll
        for (int s = 0; s < NF; ++s) {
          if (nb[s] < 0) continue;
          if (!A.gso) {
            const T d = fj[s] - fi;
            gr[0] += g.f[s].w[0] * d;
            gr[1] += g.f[s].w[1] * d;
            gr[2] += g.f[s].w[2] * d;
          }
          fmax = larger(fmax, fj[s]);
          fmin = smaller(fmin, fj[s]);
        }
        if (A.gso)
          for (int e = __ldg(A.gso + c); e < __ldg(A.gso + c + 1); ++e) {
            const T d = FC(__ldg(A.gsi + e), q) - fi;
            gr[0] += A.gsw[3 * e] * d;
            gr[1] += A.gsw[3 * e + 1] * d;
            gr[2] += A.gsw[3 * e + 2] * d;
          }
        const T phi = venkat_general<T>(g, nb, fi, fmax, fmin, gr);
#pragma unroll
        for (int s = 0; s < NF; ++s)
          FF(c, q, s) = face_value(fi, phi * (gr[0] * g.f[s].r[0] + gr[1] * g.f[s].r[1] + gr[2] * g.f[s].r[2]), A.pos_faces);
      }
    }
    __syncthreads();
    // residual r = (g - f)/tau - (1/V) sum_faces (xi . S) f_face and the implicit diagonal
    for (int c = warp; c < nc; c += nw) {
      const GenCell<T> &g = A.gen[c];
      T st[CL];
      load_state<CL>(state_of(A.st, c), st);
      const T cx = x - st[0], cy = y - st[1], cz = z - st[2];
      T mw, gq[NV], acc[NV];
      reference<T, NV>(st, cx, cy, cz, cx * cx + cy * cy + cz * cz, mw, gq);
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = (gq[q] - FC(c, q)) * st[11];
      T D = st[15];
#pragma unroll
      for (int s = 0; s < NF; ++s) {
        const int nb = __ldg(A.gnb + 6 * c + s);
        if (nb == NB_ABSENT || nb == NB_AXIS) continue;
        const T sn = dot_xi(g.f[s].S, x, y, z), k = sn * g.invV;
        T e[NV];
        if (sn > (T)0) {
          D += k;
#pragma unroll
          for (int q = 0; q < NV; ++q) e[q] = FF(c, q, s);
        } else if (sn < (T)0) {
          if (nb >= 0) {
#pragma unroll
            for (int q = 0; q < NV; ++q) e[q] = FF(nb, q, nb_side(A.gnf, c, s));
          } else if (nb == NB_WALL || A.gin[6 * c + s]) {
            // the wall's re-emission rho_w M_w, or the free stream entering (f1: (d_r T / 4) M)
            const double *uT = A.wall_uT + 4 * patch_of(A.gpat, c, s);
            const T M = wall_maxwellian<T>(uT, x, y, z) * (nb == NB_WALL ? (T)A.rho_w[__ldg(A.gwid + 6 * c + s)] : (T)1);
            e[0] = M;
            if constexpr (NV == 2) e[NV - 1] = (T)(A.d_r * uT[3] / 4.0) * M;
          } else {
            // far field where the free stream leaves: the cell's own value (zero gradient)
#pragma unroll
            for (int q = 0; q < NV; ++q) e[q] = FC(c, q);
          }
        } else {
          continue;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] -= k * e[q];
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) rs[((size_t)c * NV + q) * VB + lane] = acc[q];
      ds[(size_t)c * VB + lane] = D;
    }
    __syncthreads();
    // point-implicit passes over the colours of this octant
    const int4 *natcell = A.natcell + (size_t)oct * nc;
    for (int pass = 0; pass < A.n_sweeps; ++pass) {
      for (int col = 0; col < G.ncol; ++col) {
        const int *co = A.col_off + (size_t)oct * A.col_stride;
        const int e0 = co[col], e1 = co[col + 1];
        for (int e = e0 + warp; e < e1; e += nw) {
          const int c = __ldg(&natcell[e].x);
          const GenCell<T> &g = A.gen[c];
          T acc[NV];
#pragma unroll
          for (int q = 0; q < NV; ++q) acc[q] = rs[((size_t)c * NV + q) * VB + lane];
#pragma unroll
          for (int s = 0; s < NF; ++s) {
            const int nb = __ldg(A.gnb + 6 * c + s);
            if (nb < 0) continue;  // boundary increments are lagged (zero)
            const T sn = dot_xi(g.f[s].S, x, y, z);
            if (sn < (T)0) {
#pragma unroll
              for (int q = 0; q < NV; ++q) acc[q] += -sn * g.invV * DF(nb, q);
            }
          }
          const T D = ds[(size_t)c * VB + lane];
#pragma unroll
          for (int q = 0; q < NV; ++q) DF(c, q) = ddiv(acc[q], D);
        }
        __syncthreads();
      }
    }
    // f^{n+1/2} = f^n + df (stored relative to M_t of W^n for FP32 / BF16), the outward flux
    // moments of the wall faces per unit area and, in GSIS mode, the kinetic face-flux sums
    for (int c = warp; c < nc; c += nw) {
      const GenCell<T> &g = A.gen[c];
      T fi[NV], df[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        fi[q] = FC(c, q);
        df[q] = DF(c, q);
      }
      if constexpr (StoredRelative<S>::value) {
        const T *st = state_of(A.st, c);
        const T cx = x - st[0], cy = y - st[1], cz = z - st[2];
        const T mw = st[4] * dexp(-(cx * cx + cy * cy + cz * cz) * st[3]);
        const T r1 = NV == 2 ? st[29] : (T)0;
#pragma unroll
        for (int q = 0; q < NV; ++q) Fio<T, S>::st(F[q] + (size_t)c * VB + lane, fi[q] + df[q] - (q == 0 ? mw : r1 * mw));
      } else {
#pragma unroll
        for (int q = 0; q < NV; ++q) Fio<T, S>::st(F[q] + (size_t)c * VB + lane, fi[q] + df[q]);
      }
      if (A.kpart) {
        // outward flux through every face at the new level (upwind face value of f^n plus the
        // upwind cell's increment; boundary values carry none), summed over the faces; then
        // its moments over this block's velocities
        T psi[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) psi[q] = (T)0;
#pragma unroll
        for (int s = 0; s < NF; ++s) {
          const int nb = __ldg(A.gnb + 6 * c + s);
          if (nb == NB_ABSENT || nb == NB_AXIS) continue;
          const T sn = dot_xi(g.f[s].S, x, y, z);
          T e[NV];
          if (sn > (T)0) {
#pragma unroll
            for (int q = 0; q < NV; ++q) e[q] = FF(c, q, s) + df[q];
          } else if (sn < (T)0) {
            if (nb >= 0) {
#pragma unroll
              for (int q = 0; q < NV; ++q) e[q] = FF(nb, q, nb_side(A.gnf, c, s)) + DF(nb, q);
            } else if (nb == NB_WALL || A.gin[6 * c + s]) {
              const double *uT = A.wall_uT + 4 * patch_of(A.gpat, c, s);
              const T M = wall_maxwellian<T>(uT, x, y, z) * (nb == NB_WALL ? (T)A.rho_w[__ldg(A.gwid + 6 * c + s)] : (T)1);
              e[0] = M;
              if constexpr (NV == 2) e[NV - 1] = (T)(A.d_r * uT[3] / 4.0) * M;
            } else {
#pragma unroll
              for (int q = 0; q < NV; ++q) e[q] = fi[q];
            }
          } else {
            continue;
          }
#pragma unroll
          for (int q = 0; q < NV; ++q) psi[q] += sn * e[q];
        }
        const T p0 = wv * psi[0], p1 = NV == 2 ? wv * psi[NV - 1] : (T)0;
        const T m0 = warp_sum(p0), m1 = warp_sum(p0 * x), m2 = warp_sum(p0 * y), m3 = warp_sum(p0 * z);
        const T m4 = warp_sum(p0 * e2 + p1), m5 = NV == 2 ? warp_sum(p1) : (T)0;
        if (lane == 0) {
          double *Kp = A.kpart + ((size_t)blockIdx.x * nc + c) * 6;
          Kp[0] += (double)m0;
          Kp[1] += (double)m1;
          Kp[2] += (double)m2;
          Kp[3] += (double)m3;
          Kp[4] += (double)m4;
          Kp[5] += (double)m5;
        }
      }
      for (int s = 0; s < NF; ++s) {
        const int wid = __ldg(A.gwid + 6 * c + s);
        if (wid < 0) continue;
        const GenFace<T> &fa = g.f[s];
        const T sn = dot_xi(fa.S, x, y, z);
        T e[NV];
        if (sn > (T)0) {
#pragma unroll
          for (int q = 0; q < NV; ++q) e[q] = FF(c, q, s) + df[q];
        } else {
          const double *uT = A.wall_uT + 4 * patch_of(A.gpat, c, s);
          const T M = sn < (T)0 ? wall_maxwellian<T>(uT, x, y, z) * (T)A.rho_w[wid] : (T)0;
          e[0] = M;
          if constexpr (NV == 2) e[NV - 1] = (T)(A.d_r * uT[3] / 4.0) * M;
        }
        const T fl = wv * sn * fa.invA * e[0];
        const T e1 = NV == 2 ? wv * sn * fa.invA * e[NV - 1] : (T)0;
        const T m0 = warp_sum(fl), m1 = warp_sum(fl * x), m2 = warp_sum(fl * y), m3 = warp_sum(fl * z);
        const T m4 = warp_sum(fl * e2 + e1), m5 = NV == 2 ? warp_sum(e1) : (T)0;
        if (lane == 0) {
          T *W = A.wpart + ((size_t)b * A.nwall + wid) * NWF;
          W[0] = m0;
          W[1] = m1;
          W[2] = m2;
          W[3] = m3;
          W[4] = m4;
          W[5] = m5;
        }
      }
    }
    __syncthreads();
  }
}

// Wall pre-pass on general meshes: rho_w of each wall face balances the mass flux of the
// molecules reaching it (the wall cell's limited reconstruction of f^n) against the re-emitted
// flux of M(u_w, T_w) through the face.  One CTA per wall face; warps over velocity blocks,
// FP64 sums in a fixed order.
template <typename T, typename S, int NV>
__global__ void __launch_bounds__(256) wall_prepass_general_kernel(const KinArgs<T, S> A, const int *wall_cell,
                                                                  const int *wall_side, double *rho_w) {
  __shared__ double red[2][8];
  const int w = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int c = wall_cell[w], side = wall_side[w], nc = A.g.nc;
  constexpr int SL = stage_state_len<S, NV>();
  const GenCell<T> &g = A.gen[c];
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) nb[s] = __ldg(A.gnb + 6 * c + s);
  const GenFace<T> &fa = g.f[side];
  const double *uT = A.wall_uT + 4 * patch_of(A.gpat, c, side);
  double num = 0.0, den = 0.0;
  for (int b = warp; b < A.nblocks; b += nw) {
    const T *vp = A.vel + ((size_t)b * VB + lane) * 4;
    const T x = vp[0], y = vp[1], z = vp[2], wv = vp[3];
    const T sn = dot_xi(fa.S, x, y, z);
    if (sn > (T)0) {
      auto fn = [&](int cell) {
        T st[SL], stored[NV], f[NV];
        load_state<SL>(state_of(A.st, cell), st);
#pragma unroll
        for (int q = 0; q < NV; ++q) stored[q] = Fio<T, S>::ld((q == 0 ? A.f : A.f1) + ((size_t)b * nc + cell) * VB + lane);
        corrected_all<T, S, NV>(stored, st, x, y, z, f);
        return f[0];
      };
      const T fi = fn(c);
      T gr[3] = {(T)0, (T)0, (T)0}, fmax = fi, fmin = fi;
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        if (nb[s] < 0) continue;
        const T fj = fn(nb[s]), d = fj - fi;
        if (!A.gso) {
          gr[0] += g.f[s].w[0] * d;
          gr[1] += g.f[s].w[1] * d;
          gr[2] += g.f[s].w[2] * d;
        }
        fmax = larger(fmax, fj);
        fmin = smaller(fmin, fj);
      }
      if (A.gso)
        for (int e = __ldg(A.gso + c); e < __ldg(A.gso + c + 1); ++e) {
          const T d = fn(__ldg(A.gsi + e)) - fi;
          gr[0] += A.gsw[3 * e] * d;
          gr[1] += A.gsw[3 * e + 1] * d;
          gr[2] += A.gsw[3 * e + 2] * d;
        }
      const T phi = venkat_general<T>(g, nb, fi, fmax, fmin, gr);
      const T ff = A.pos_faces ? face_value(fi, phi * (gr[0] * fa.r[0] + gr[1] * fa.r[1] + gr[2] * fa.r[2]), 1)
                               : fi + (phi * gr[0]) * fa.r[0] + (phi * gr[1]) * fa.r[1] + (phi * gr[2]) * fa.r[2];
      num += (double)(wv * sn * ff);
    } else if (sn < (T)0) {
      den += (double)(wv * -sn * wall_maxwellian<T>(uT, x, y, z));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if (lane == 0) {
    red[0][warp] = num;
    red[1][warp] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double n = 0.0, d = 0.0;
    for (int k = 0; k < nw; ++k) {
      n += red[0][k];
      d += red[1][k];
    }
    // a velocity shard holds part of the numerator; the denominator covers every velocity
    rho_w[w] = n / (A.wden ? A.wden[w] : d);
  }
}

template <typename T, typename S>
__global__ void __launch_bounds__(256) wall_den_general_kernel(const KinArgs<T, S> A, const double *vel64, int nslots,
                                                               const int *wall_cell, const int *wall_side,
                                                               double *wden) {
  __shared__ double red[8];
  const int w = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = wall_cell[w], side = wall_side[w];
  const GenFace<T> &fa = A.gen[c].f[side];
  const double *uT = A.wall_uT + 4 * patch_of(A.gpat, c, side);
  double den = 0.0;
  for (int v = threadIdx.x; v < nslots; v += blockDim.x) {
    const T x = (T)vel64[4 * v], y = (T)vel64[4 * v + 1], z = (T)vel64[4 * v + 2], wv = (T)vel64[4 * v + 3];
    const T sn = dot_xi(fa.S, x, y, z);
    if (sn < (T)0) den += (double)(wv * -sn * wall_maxwellian<T>(uT, x, y, z));
  }
  for (int o = 16; o > 0; o >>= 1) den += __shfl_xor_sync(0xffffffffu, den, o);
  if (lane == 0) red[warp] = den;
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int k = 0; k < 8; ++k) d += red[k];
    wden[w] = d;
  }
}

template <typename T, typename S>
cudaError_t launch_wall_den_general(const KinArgs<T, S> &a, const double *vel64, int nslots_all, const int *wall_cell,
                                    const int *wall_side, int nwall, double *wden, cudaStream_t s) {
  if (nwall == 0) return cudaSuccess;
  wall_den_general_kernel<T, S><<<nwall, 256, 0, s>>>(a, vel64, nslots_all, wall_cell, wall_side, wden);
  return cudaGetLastError();
}

__global__ void sum_kpart_kernel(const double *kpart, int nparts, int nc, double *K) {
  const size_t n = (size_t)nc * 6;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int p = 0; p < nparts; ++p) acc += kpart[(size_t)p * n + i];
    K[i] = acc;
  }
}

cudaError_t launch_sum_kpart(const double *kpart, int nparts, int nc, double *K, cudaStream_t s) {
  int grid = (int)(((size_t)nc * 6 + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  sum_kpart_kernel<<<grid, 256, 0, s>>>(kpart, nparts, nc, K);
  return cudaGetLastError();
}

template <typename T, typename S>
size_t kinetic_general_stride(int nc, int nvdf, int nact) {
  return (((size_t)nc * VB * (nvdf * (3 + 2 * nact) + 1)) * sizeof(T) + 255) & ~(size_t)255;
}

template <typename T, typename S>
static void (*kinetic_general_fn(int nvdf, int nact))(const KinArgs<T, S>) {
  if (nvdf == 2)
    return nact == 1 ? kinetic_general_kernel<T, S, 2, 1>
                     : (nact == 2 ? kinetic_general_kernel<T, S, 2, 2> : kinetic_general_kernel<T, S, 2, 3>);
  return nact == 1 ? kinetic_general_kernel<T, S, 1, 1>
                   : (nact == 2 ? kinetic_general_kernel<T, S, 1, 2> : kinetic_general_kernel<T, S, 1, 3>);
}

template <typename T, typename S>
cudaError_t kinetic_general_shape(int nvdf, int nact, int *ctas_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kinetic_general_fn<T, S>(nvdf, nact), 256, 0);
}

template <typename T, typename S>
cudaError_t launch_kinetic_general(const KinArgs<T, S> &a, int grid, cudaStream_t s) {
  kinetic_general_fn<T, S>(a.nvdf, a.g.nact)<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t launch_wall_prepass_general(const KinArgs<T, S> &a, const int *wall_cell, const int *wall_side, int nwall,
                                        double *rho_w, cudaStream_t s) {
  if (nwall == 0) return cudaSuccess;
  if (a.nvdf == 2)
    wall_prepass_general_kernel<T, S, 2><<<nwall, 256, 0, s>>>(a, wall_cell, wall_side, rho_w);
  else
    wall_prepass_general_kernel<T, S, 1><<<nwall, 256, 0, s>>>(a, wall_cell, wall_side, rho_w);
  return cudaGetLastError();
}

#define GSIS_INST(T, S)                                                                                         \
  template cudaError_t launch_kinetic<T, S>(const KinArgs<T, S> &, int, int, size_t, cudaStream_t);             \
  template cudaError_t kinetic_shape<T, S>(const KinGeom &, int, bool, int, size_t, int *, int *);                                       \
  template cudaError_t launch_wall_prepass<T, S>(const KinArgs<T, S> &, const int *, const int *, int,           \
                                                 const double *, double *, int, cudaStream_t);                   \
  template cudaError_t launch_moments<T, S>(const KinArgs<T, S> &, int, int, double *, cudaStream_t);           \
  template cudaError_t launch_init_maxwellian<T, S>(const KinArgs<T, S> &, const double *, int, cudaStream_t);   \
  template cudaError_t launch_export_f<T, S>(const KinArgs<T, S> &, int, const int *, int, int, double *,       \
                                             cudaStream_t);                                                      \
  template cudaError_t launch_import_f<T, S>(const KinArgs<T, S> &, int, const int *, int, int, const double *, \
                                             cudaStream_t);                                                      \
  template cudaError_t launch_kinetic_general<T, S>(const KinArgs<T, S> &, int, cudaStream_t);                   \
  template cudaError_t kinetic_general_shape<T, S>(int, int, int *);                                             \
  template size_t kinetic_general_stride<T, S>(int, int, int);                                                   \
  template cudaError_t launch_wall_prepass_general<T, S>(const KinArgs<T, S> &, const int *, const int *, int,   \
                                                         double *, cudaStream_t);                                \
  template cudaError_t launch_wall_den_general<T, S>(const KinArgs<T, S> &, const double *, int, const int *,    \
                                                     const int *, int, double *, cudaStream_t);
GSIS_INST(float, float)
GSIS_INST(double, double)
GSIS_INST(float, __nv_bfloat16)
template size_t kinetic_smem_bytes<float, float>(const KinGeom &, int);
template size_t kinetic_smem_bytes<double, double>(const KinGeom &, int);
template size_t kinetic_smem_bytes<float, __nv_bfloat16>(const KinGeom &, int);
template size_t kinetic_gscratch_stride<float, float>(const KinGeom &, int);
template size_t kinetic_gscratch_stride<double, double>(const KinGeom &, int);
template size_t kinetic_gscratch_stride<float, __nv_bfloat16>(const KinGeom &, int);

}  // namespace gsis
