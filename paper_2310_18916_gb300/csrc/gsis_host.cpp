// gsis_host.cpp -- host solver object behind the C ABI of include/gsis.h.
//
// Builds the geometry (rectilinear axes, or the per-cell finite-volume geometry of a general
// structured block), the octant-blocked velocity layout, the colour tables and the wall tables,
// owns every device buffer, and sequences one outer iteration of Algorithm 1:
//   wall pre-pass -> kinetic step -> block reduction -> moments (+ closed-domain mass scale)
//   -> [GSIS: FP64 synthetic solve] -> eps -> state of the next step,
// with the rectilinear kernels or the general-mesh ones; plus the Euler presteps at creation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/gsis.h"
#include "gsis_internal.h"

// Evaluates EXPR with T (kinetic arithmetic) and S (VDF storage) bound to the types of the
// precision PREC: F64 -> double/double, F32 -> float/float, BF16 -> float/__nv_bfloat16.
#define GSIS_DISPATCH(PREC, EXPR)                                                          \
  ((PREC) == GSIS_F64    ? [&] { using T = double; using S = double; return EXPR; }()        \
   : (PREC) == GSIS_BF16 ? [&] { using T = float; using S = __nv_bfloat16; return EXPR; }()  \
                         : [&] { using T = float; using S = float; return EXPR; }())

using namespace gsis;

namespace {
thread_local std::string g_create_error;

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};
}  // namespace

struct gsis_solver {
  // options
  gsis_options opt{};
  int prec = GSIS_F32;
  int nvdf = 1;  // reduced VDFs: 1 (Shakhov) or 2 (Rykov)
  double Kn = 0.1, omega = 0.81;
  gsis_gas gas{};
  cudaStream_t stream = nullptr;
  // geometry
  int n[3] = {1, 1, 1}, nc = 0;
  std::vector<double> X[3];
  std::vector<AxisCell<double>> axc[3];
  std::vector<double> vol;
  double vsum = 0.0;
  KinGeom kg{};
  std::vector<int> col_off, col_cell, pos_of;
  int col_stride = 0;  // > 0: per-octant kinetic colour offsets (unstructured meshes)
  std::vector<EntryInfo> entries;
  std::vector<int4> natcell;
  // velocities
  int nvc = 0, nslots = 0, nblocks = 0;
  int nv_axis[3] = {0, 0, 0};
  std::vector<int> slot_canon;
  std::vector<int8_t> boct;
  std::vector<double> vel64;      // this shard's slots [slot][4]
  std::vector<double> vel64_all;  // every slot (wall constants integrate over all velocities)
  int nslots_all = 0;
  std::vector<double> vaxis;      // the 1-D grids: nodes of x, y, z, then their weights
  bool point_set = false;         // an unstructured velocity set (no tensor product)
  // FP64 storage with the Shakhov model: moments about the origin from a per-slot table and the
  // reference distribution's sums in closed form (launch_moments_origin)
  bool origin_mom = false;
  double *d_mtab = nullptr, *d_vaxis = nullptr;
  // walls
  int nwall = 0;
  std::vector<int> wall_cell, wall_side, wall_sides_list;
  double wall_uT[6][4] = {};
  int closed = 1;
  // general (curvilinear) meshes: per-cell geometry, neighbour codes, wall-face ids, far-field
  // inflow sides, wall-face areas; the kinetic kernel's persistent grid
  bool general = false;
  bool simplex = false;  // an unstructured mesh with prisms, pyramids or tetrahedra
  // unstructured meshes: the neighbour's side of each shared face and the boundary patch of each
  // boundary face (both absent on structured blocks, whose opposite side is s ^ 1 and whose
  // patches are the block sides); the synthetic solve's colour offsets into colcells
  bool unstructured = false;
  std::vector<unsigned char> gnf, gpat;
  unsigned char *d_gnf = nullptr, *d_gpat = nullptr;
  std::vector<int> wall_patch;
  int *d_wall_patch = nullptr;
  std::vector<int> gs_off, gs_idx;      // least-squares stencil (CSR) of an unstructured mesh
  std::vector<double> gs_w;             // [entry][3]
  int *d_gso = nullptr, *d_gsi = nullptr;
  void *d_gsw = nullptr;                // in the kinetic precision
  double *d_gsw64 = nullptr;
  std::vector<int> mcol_off;
  std::vector<GenCell<double>> gen64;
  std::vector<int> gnb, gwid;
  std::vector<unsigned char> gin;
  std::vector<double> wall_area;
  void *d_gen = nullptr;
  int *d_gnb = nullptr, *d_gwid = nullptr;
  unsigned char *d_gin = nullptr;
  double *d_wall_area = nullptr;
  std::vector<double> xc64;
  // general meshes, GSIS mode: FP64 geometry and the synthetic solve's work arrays
  GenCell<double> *d_gen64 = nullptr;
  double *d_xc = nullptr, *d_kpart = nullptr, *d_wden = nullptr;
  double *g_W = nullptr, *g_pr = nullptr, *g_mu = nullptr, *g_gW = nullptr, *g_phW = nullptr, *g_gP = nullptr;
  double *g_R = nullptr, *g_D = nullptr, *g_dW = nullptr, *g_F0 = nullptr, *g_part = nullptr;
  double *g_Ff = nullptr, *g_gam = nullptr, *g_FW0 = nullptr, *g_FW = nullptr;
  int *g_flag = nullptr;
  int kin_grid = 0;
  size_t kin_scratch_bytes = 0;
  // device
  std::vector<DevBuf> allocs;
  void *d_f = nullptr, *d_wpart = nullptr, *d_stT = nullptr, *d_vel = nullptr;
  double *d_mp = nullptr, *d_K = nullptr;
  int mom_bpc = 1, mom_nchunks = 1;
  void *d_ax[3] = {nullptr, nullptr, nullptr};
  AxisCell<double> *d_ax64[3] = {nullptr, nullptr, nullptr};
  double *d_vel64 = nullptr, *d_st64 = nullptr, *d_rho_w = nullptr, *d_Z0 = nullptr, *d_Zw = nullptr;
  double *d_wall_uT = nullptr, *d_mom = nullptr, *d_wf = nullptr, *d_Mh = nullptr;
  double *d_hot = nullptr, *d_Wstate = nullptr, *d_Wnew = nullptr, *d_vol = nullptr, *d_mass = nullptr;
  double *d_scratch = nullptr, *d_eps4 = nullptr;
  int8_t *d_boct = nullptr;
  int *d_col_off = nullptr, *d_wall_cell = nullptr;
  int *d_wall_side = nullptr, *d_wall_sides = nullptr, *d_err = nullptr, *d_iters = nullptr;
  EntryInfo *d_entry = nullptr;
  int4 *d_natcell = nullptr;
  unsigned *d_ticket = nullptr, *d_bar = nullptr;
  // macro work
  double *m_W = nullptr, *m_pr = nullptr, *m_gW = nullptr, *m_phW = nullptr, *m_gP = nullptr, *m_aux = nullptr;
  double *m_R = nullptr, *m_invD = nullptr, *m_dW = nullptr, *m_Fc = nullptr, *m_corr = nullptr, *m_gam = nullptr;
  int *d_colcells = nullptr;
  int ncol0 = 0;
  std::vector<int> colcells;
  double *m_red = nullptr, *m_Ffc = nullptr, *m_wfl = nullptr, *m_G = nullptr;
  int macro_grid = 0, macro_block = 256;
  // pinned host words the step's results are copied into, so a step can be enqueued without
  // the host waiting (pageable read-backs would block)
  struct Readback {
    double eps4[4];
    int iters, err;
  };
  Readback *pin = nullptr;
  bool pending = false;
  int pending_mode = 0, pending_launches = 0;
  int kin_warps = 1;
  size_t kin_smem = 0;     // dynamic shared memory of the kinetic kernel (0 with a global ring)
  size_t kin_gstride = 0;  // bytes of global ring scratch per velocity block (0: shared memory)
  void *d_kscratch = nullptr;
  // CUDA graphs of one outer step (opt.capture_graphs): one per mode and current state buffer
  // (the step swaps the state buffers, so two alternate), captured on first use and replayed
  struct StepGraph {
    int mode;
    const double *wstate;
    cudaGraphExec_t exec;
    int launches;
  };
  std::vector<StepGraph> graphs;
  bool graphs_off = false;  // a capture failed: every later step launches directly
  // graphs are captured on and launched into a stream of the solver's own (the caller's stream
  // may be the legacy default stream, which cannot be captured), ordered after the caller's
  // earlier work and before its later work by two events
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {};
  void drop_graphs() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
  void release_graphs() {
    drop_graphs();
    for (auto &e : gev)
      if (e) cudaEventDestroy(e);
    if (gstream) cudaStreamDestroy(gstream);
    gstream = nullptr;
    gev[0] = gev[1] = nullptr;
  }
  // the caller's stream -> the graph stream, launch, graph stream -> the caller's stream
  int launch_graph(cudaGraphExec_t exec) {
    int rc = cuda(cudaEventRecord(gev[0], stream), "event");
    if (!rc) rc = cuda(cudaStreamWaitEvent(gstream, gev[0], 0), "stream wait");
    if (!rc) rc = cuda(cudaGraphLaunch(exec, gstream), "graph launch");
    if (!rc) rc = cuda(cudaEventRecord(gev[1], gstream), "event");
    if (!rc) rc = cuda(cudaStreamWaitEvent(stream, gev[1], 0), "stream wait");
    return rc;
  }
  // profiling
  bool profiling = false;
  cudaEvent_t ev[6] = {};
  double phase_ms[5] = {0, 0, 0, 0, 0};
  int prof_steps = 0, prof_launches = 0;
  // bookkeeping
  double mass_ref = 0.0;
  int outer_total = 0, macro_iters_last = 0;
  double eps4[4] = {0, 0, 0, 0};
  std::string last_error;

  int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    last_error = buf;
    return code;
  }

  template <typename P>
  int alloc(P **out, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (opt.alloc) {
      p = opt.alloc(bytes, (void *)stream, opt.alloc_ctx);
      if (!p) return fail(GSIS_E_OOM, "allocator returned NULL for %zu bytes", bytes);
    } else {
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) return fail(GSIS_E_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    allocs.push_back({p, bytes});
    *out = static_cast<P *>(p);
    return GSIS_OK;
  }

  void mark(int k) {
    if (profiling) cudaEventRecord(ev[k], stream);
  }

  void release() {
    if (!graphs.empty()) cudaStreamSynchronize(stream);
    release_graphs();
    if (pin) {
      cudaFreeHost(pin);
      pin = nullptr;
    }
    if (ev[0])
      for (auto &e : ev) cudaEventDestroy(e);
    if (!allocs.empty()) cudaStreamSynchronize(stream);
    for (auto &b : allocs) {
      if (opt.free) opt.free(b.p, (void *)stream, opt.alloc_ctx);
      else cudaFree(b.p);
    }
    allocs.clear();
  }

  int cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GSIS_OK;
    return fail(GSIS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  }

  template <typename P>
  int upload(P *dst, const void *src, size_t bytes) {
    return cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream), "upload");
  }

  template <typename T, typename S = T>
  KinArgs<T, S> kin_args() const {
    KinArgs<T, S> a{};
    a.g = kg;
    for (int d = 0; d < 3; ++d) a.ax[d] = static_cast<const AxisCell<T> *>(d_ax[d]);
    a.vel = static_cast<const T *>(d_vel);
    a.boct = d_boct;
    a.col_off = d_col_off;
    a.col_stride = col_stride;
    a.entry = d_entry;
    a.natcell = d_natcell;
    a.st = static_cast<const T *>(d_stT);
    a.rho_w = d_rho_w;
    a.wall_uT = d_wall_uT;
    a.f = static_cast<S *>(d_f);
    a.f1 = nvdf == 2 ? static_cast<S *>(d_f) + (size_t)nslots * nc : nullptr;
    a.nvdf = nvdf;
    a.d_r = gas.d_r;
    a.wpart = static_cast<T *>(d_wpart);
    a.nwall = nwall;
    a.nblocks = nblocks;
    a.err = d_err;
    a.gscratch = static_cast<unsigned char *>(d_kscratch);
    a.gstride = kin_gstride;
    a.gen = static_cast<const GenCell<T> *>(d_gen);
    a.gnb = d_gnb;
    a.gwid = d_gwid;
    a.gin = d_gin;
    a.n_sweeps = opt.n_sweeps;
    a.pos_faces = opt.positive_faces;
    a.wden = d_wden;
    a.gnf = d_gnf;
    a.gpat = d_gpat;
    a.gso = d_gso;
    a.gsi = d_gsi;
    a.gsw = static_cast<const T *>(d_gsw);
    return a;
  }

  // the synthetic solve on general meshes: GSIS inner steps from the moments Mh (K set by the
  // caller); Euler mode sets euler, steps, Mh / mh_stride itself
  MacroGenArgs macro_general_args() const {
    MacroGenArgs m{};
    m.nc = (int)nc;
    m.nW = gas.model == GSIS_RYKOV ? 6 : 5;
    m.model = gas.model;
    m.steps = opt.macro_steps;
    m.sweeps = opt.macro_sweeps;
    m.closed = closed;
    m.ncol0 = ncol0;
    m.ncolm = (int)mcol_off.size() - 1;
    for (int c = 0; c <= m.ncolm && c <= MACRO_MAX_COLOURS; ++c) m.colm_off[c] = mcol_off[c];
    m.gnf = d_gnf;
    m.gpat = d_gpat;
    m.gso = d_gso;
    m.gsi = d_gsi;
    m.gsw = d_gsw64;
    m.euler = 0;
    m.mh_stride = 18;
    m.wall_g13 = opt.wall_flux == GSIS_WALL_G13;
    m.relax = opt.relax > 0.0 ? opt.relax : 1.0;
    m.visc_jump = opt.visc_jump >= 0.0 ? opt.visc_jump : (simplex ? 0.25 : 0.0);
    m.mu0 = Kn / std::sqrt(3.14159265358979323846);
    m.omega = omega;
    m.cfl = opt.macro_cfl;
    m.tol = opt.macro_tol;
    m.d_r = gas.d_r;
    m.Z_r = gas.Z_r;
    for (int k = 0; k < 4; ++k) m.A[k] = gas.A[k];
    m.mass_ref = mass_ref;
    m.vsum = vsum;
    m.gen = d_gen64;
    m.gnb = d_gnb;
    m.xc = d_xc;
    m.vol = d_vol;
    m.wall_uT = d_wall_uT;
    m.Mh = d_Mh;
    m.colcells = d_colcells;
    m.W = g_W; m.pr = g_pr; m.mu = g_mu; m.gW = g_gW; m.phW = g_phW; m.gP = g_gP;
    m.R = g_R; m.D = g_D; m.dW = g_dW; m.F0 = g_F0; m.part = g_part; m.flag = g_flag;
    m.Ff = g_Ff;
    m.gam = g_gam;
    m.FW0 = g_FW0;
    m.FW = g_FW;
    m.Wout = d_Wnew;
    m.err = d_err;
    m.iters = d_iters;
    return m;
  }

  // sum over the velocity shards (no-op unsharded)
  int exchange(double *dev, size_t count, const char *what) {
    if (opt.shard_count <= 1 || count == 0) return GSIS_OK;
    if (opt.allreduce(dev, count, (void *)stream, opt.allreduce_ctx) != 0)
      return fail(GSIS_E_CUDA, "allreduce of %s failed", what);
    return GSIS_OK;
  }

  int check_err() {
    int herr = 0;
    int rc = cuda(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream), "read error flag");
    if (rc) return rc;
    rc = cuda(cudaStreamSynchronize(stream), "synchronize");
    if (rc) return rc;
    if (herr == GSIS_ERR_DIVERGED) return fail(GSIS_E_DIVERGED, "non-finite or non-positive density/temperature");
    if (herr == GSIS_ERR_TIMEOUT) return fail(GSIS_E_TIMEOUT, "a bounded device wait timed out");
    if (herr != 0) return fail(GSIS_E_CUDA, "device error flag %d", herr);
    return GSIS_OK;
  }

  // moments of the stored f -> Mh (about the state velocity st64[0..2]), the kinetic flux sum K
  // and the wall fluxes
  template <typename T, typename S>
  int reduce_and_finalize(bool closed_scale) {
    const bool first_shard = opt.shard_count <= 1 || opt.shard_index == 0;
    int rc;
    if constexpr (std::is_same<T, double>::value && std::is_same<S, double>::value) {
      if (origin_mom)
        rc = cuda(launch_moments_origin(kin_args<T, S>(), d_mtab, mom_bpc, mom_nchunks, d_st64, d_vaxis, nv_axis,
                                        first_shard ? 1 : 0, d_mp, stream),
                  "moments");
      else
        rc = cuda(launch_moments<T, S>(kin_args<T, S>(), mom_bpc, mom_nchunks, d_mp, stream), "moments");
    } else {
      rc = cuda(launch_moments<T, S>(kin_args<T, S>(), mom_bpc, mom_nchunks, d_mp, stream), "moments");
    }
    if (rc) return rc;
    rc = cuda(launch_reduce<T>(d_mp, mom_nchunks, nvdf, static_cast<const T *>(d_wpart), d_boct, nblocks, kg, d_wall_cell,
                               d_wall_side, nwall, d_rho_w, d_Zw, first_shard, general, d_vol, d_st64, d_mom, d_K, d_wf,
                               stream, origin_mom),
              "reduce");
    if (!rc) rc = exchange(d_mom, (size_t)nc * MOM_STRIDE, "moments");
    if (!rc) rc = exchange(d_K, (size_t)nc * 6, "kinetic flux sums");
    if (!rc) rc = exchange(d_wf, (size_t)nwall * 6, "wall fluxes");
    if (rc) return rc;
    FinalizeArgs fa{};
    fa.nvdf = nvdf;
    fa.d_r = gas.d_r;
    fa.g = kg;
    fa.mom = d_mom;
    fa.st64 = d_st64;
    fa.vol = d_vol;
    fa.mass_ref = mass_ref;
    fa.closed = closed_scale ? closed : 0;
    fa.Mh = d_Mh;
    fa.mass_scale = d_mass;
    fa.scratch = d_scratch;
    fa.ticket = d_ticket;
    fa.err = d_err;
    return cuda(launch_finalize(fa, stream), "finalize");
  }

  int write_state(const double *Wn) {
    StateArgs sa{};
    sa.nvdf = nvdf;
    sa.d_r = gas.d_r;
    sa.Z_r = gas.Z_r;
    for (int k = 0; k < 4; ++k) sa.A[k] = gas.A[k];
    sa.g = kg;
    sa.Wn = Wn;
    sa.Mh = d_Mh;
    sa.mass_scale_ptr = d_mass;
    sa.Kn = Kn;
    sa.omega = omega;
    sa.kin_inv_dt = opt.kin_inv_dt;
    sa.st64 = d_st64;
    sa.stT = d_stT;
    sa.is_float = prec != GSIS_F64;
    return cuda(launch_state(sa, stream), "state");
  }

  // state <- moments of the current f (after init or set_f); also sets mass_ref.  W0: the
  // initial state when f was just initialised to its Maxwellian (BF16 storage holds f relative
  // to it), else nullptr.
  template <typename T, typename S>
  int state_from_f(const double *W0 = nullptr) {
    // neutral state: corrected f = f_raw, moments about u = 0; with relative storage after
    // initialisation, f_raw = M(W0) is formed from the state's W^n Maxwellian slot
    std::vector<double> st0((size_t)nc * NST, 0.0);
    for (int c = 0; c < nc; ++c) st0[(size_t)c * NST + 10] = 1.0;
    if (W0 && prec != GSIS_F64)
      for (int c = 0; c < nc; ++c) {
        const double *w = W0 + (size_t)c * 6;
        double *st = st0.data() + (size_t)c * NST;
        st[0] = w[1];
        st[1] = w[2];
        st[2] = w[3];
        st[3] = 1.0 / w[4];
        st[4] = w[0] * std::pow(3.14159265358979323846 * w[4], -1.5);
        if (nvdf == 2) st[29] = gas.d_r * w[5] / 4.0;  // f1 = (d_r Tr / 4) M
      }
    std::vector<T> st0T(st0.begin(), st0.end());
    int rc = upload(d_st64, st0.data(), st0.size() * sizeof(double));
    if (!rc) rc = upload(d_stT, st0T.data(), st0T.size() * sizeof(T));
    if (!rc) rc = reduce_and_finalize<T, S>(false);
    if (rc) return rc;
    double m2[2];
    rc = cuda(cudaMemcpyAsync(m2, d_mass, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream), "mass");
    if (!rc) rc = cuda(cudaStreamSynchronize(stream), "sync");
    if (rc) return rc;
    mass_ref = m2[1];
    double one = 1.0;
    rc = upload(d_mass, &one, sizeof(double));
    if (!rc) rc = cuda(cudaMemcpy2DAsync(d_Wstate, 6 * sizeof(double), d_Mh, 18 * sizeof(double), 6 * sizeof(double),
                                         nc, cudaMemcpyDeviceToDevice, stream),
                       "copy W");
    if (!rc) rc = write_state(d_Wstate);
    if (!rc) rc = check_err();
    return rc;
  }

  template <typename T, typename S>
  int step_impl(int mode) {
    int launches = 0;
    mark(0);
    int rc = general ? cuda(launch_wall_prepass_general<T, S>(kin_args<T, S>(), d_wall_cell, d_wall_side, nwall, d_rho_w,
                                                              stream),
                            "wall pre-pass")
                     : cuda(launch_wall_prepass<T, S>(kin_args<T, S>(), d_wall_cell, d_wall_side, nwall, d_Z0, d_rho_w,
                                                      nslots, stream),
                            "wall pre-pass");
    if (!rc) rc = exchange(d_rho_w, (size_t)nwall, "wall densities");
    if (rc) return rc;
    launches += nwall > 0;
    mark(1);
    if (general) {
      KinArgs<T, S> ka = kin_args<T, S>();
      if (mode == GSIS_MODE_GSIS) {
        ka.kpart = d_kpart;
        rc = cuda(cudaMemsetAsync(d_kpart, 0, (size_t)kin_grid * nc * 6 * sizeof(double), stream), "memset");
        if (rc) return rc;
      }
      rc = cuda(launch_kinetic_general<T, S>(ka, kin_grid, stream), "kinetic");
    } else {
      rc = cuda(launch_kinetic<T, S>(kin_args<T, S>(), nblocks, kin_warps, kin_smem, stream), "kinetic");
    }
    if (rc) return rc;
    mark(2);
    rc = reduce_and_finalize<T, S>(true);
    if (rc) return rc;
    launches += 1 + 1 + (nwall > 0) + 2;
    mark(3);
    if (mode == GSIS_MODE_GSIS && general) {
      // the kinetic face fluxes summed per cell, then the general synthetic solve
      rc = cuda(launch_sum_kpart(d_kpart, kin_grid, (int)nc, d_K, stream), "kinetic flux sums");
      if (!rc) rc = exchange(d_K, (size_t)nc * 6, "kinetic flux sums");
      if (rc) return rc;
      MacroGenArgs m = macro_general_args();
      m.K = d_K;
      rc = cuda(run_macro_general(m, stream), "synthetic solve");
      if (rc) return rc;
      launches += 2 + opt.macro_steps * (7 + 2 * opt.macro_sweeps);
    } else if (mode == GSIS_MODE_GSIS) {
      MacroArgs m{};
      m.g = kg;
      for (int d = 0; d < 3; ++d) m.ax[d] = d_ax64[d];
      m.Kn = Kn;
      m.mu0 = Kn / std::sqrt(3.14159265358979323846);
      m.omega = omega;
      m.cfl = opt.macro_cfl;
      m.tol = opt.macro_tol;
      m.model = gas.model;
      m.nW = gas.model == GSIS_RYKOV ? 6 : 5;
      m.steps = opt.macro_steps;
      m.sweeps = opt.macro_sweeps;
      m.d_r = gas.d_r;
      m.Z_r = gas.Z_r;
      for (int k = 0; k < 4; ++k) m.A[k] = gas.A[k];
      m.mass_ref = mass_ref;
      m.den_floor = 1e-24 * vsum;
      m.closed = closed;
      m.Mh = d_Mh;
      m.wall_g13 = opt.wall_flux == GSIS_WALL_G13;
      m.K = d_K;
      m.wall_cell = d_wall_cell;
      m.wall_side = d_wall_side;
      m.nwall = nwall;
      m.wall_uT = d_wall_uT;
      m.colcells = d_colcells;
      m.ncol0 = ncol0;
      m.W = m_W; m.pr = m_pr; m.gW = m_gW; m.phW = m_phW; m.gP = m_gP; m.aux = m_aux; m.R = m_R; m.invD = m_invD;
      m.dW = m_dW; m.Fc = m_Fc; m.corr = m_corr; m.gam = m_gam; m.red = m_red; m.Ffc = m_Ffc;
      m.wfl = m_wfl;
      m.G = m_G;
      m.Wout = d_Wnew;
      m.bar = d_bar;
      m.err = d_err;
      m.iters = d_iters;
      if (opt.macro_steps > 0) {
        rc = cuda(cudaMemsetAsync(d_bar, 0, MACRO_BAR_WORDS * sizeof(unsigned), stream), "memset");
        if (rc) return rc;
        rc = cuda(launch_macro(m, macro_grid, macro_block, stream), "synthetic solve");
        if (rc) return rc;
        ++launches;
      } else {
        rc = cuda(cudaMemcpy2DAsync(d_Wnew, 6 * sizeof(double), d_Mh, 18 * sizeof(double), 6 * sizeof(double), nc,
                                    cudaMemcpyDeviceToDevice, stream),
                  "copy W");
        if (rc) return rc;
      }
    } else {
      rc = cuda(cudaMemcpy2DAsync(d_Wnew, 6 * sizeof(double), d_Mh, 18 * sizeof(double), 6 * sizeof(double), nc,
                                  cudaMemcpyDeviceToDevice, stream),
                "copy W");
      if (rc) return rc;
    }
    mark(4);
    EpsArgs ea{};
    ea.nc = nc;
    ea.vsum = vsum;
    ea.Wn = d_Wnew;
    ea.Wo = d_Wstate;
    ea.vol = d_vol;
    ea.scratch = d_scratch;
    ea.ticket = d_ticket + 1;
    ea.eps4 = d_eps4;
    rc = cuda(launch_eps(ea, stream), "eps");
    if (!rc) rc = write_state(d_Wnew);
    if (rc) return rc;
    launches += 2;
    mark(5);
    std::swap(d_Wstate, d_Wnew);
    pin->iters = 0;
    rc = cuda(cudaMemcpyAsync(pin->eps4, d_eps4, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream), "eps");
    if (!rc && mode == GSIS_MODE_GSIS && opt.macro_steps > 0)
      rc = cuda(cudaMemcpyAsync(&pin->iters, d_iters, sizeof(int), cudaMemcpyDeviceToHost, stream), "iters");
    if (!rc) rc = cuda(cudaMemcpyAsync(&pin->err, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream), "error flag");
    if (rc) return rc;
    pending = true;
    pending_mode = mode;
    pending_launches = launches;
    return GSIS_OK;
  }

  // waits for the enqueued step and takes over its results
  int finish_step() {
    if (!pending) return fail(GSIS_E_INVALID, "no step is pending");
    pending = false;
    int rc = cuda(cudaStreamSynchronize(stream), "synchronize");
    if (rc) return rc;
    if (pin->err == GSIS_ERR_DIVERGED) return fail(GSIS_E_DIVERGED, "non-finite or non-positive density/temperature");
    if (pin->err == GSIS_ERR_TIMEOUT) return fail(GSIS_E_TIMEOUT, "a bounded device wait timed out");
    if (pin->err != 0) return fail(GSIS_E_CUDA, "device error flag %d", pin->err);
    for (int k = 0; k < 4; ++k) eps4[k] = pin->eps4[k];
    macro_iters_last = pin->iters;
    ++outer_total;
    if (profiling) {
      for (int k = 0; k < 5; ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
        phase_ms[k] += t;
      }
      ++prof_steps;
      prof_launches += pending_launches;
    }
    return GSIS_OK;
  }

  int enqueue_step(int mode) {
    if (pending) return fail(GSIS_E_INVALID, "a step is pending: call gsis_step_wait first");
    // direct launches: no graphs asked for, profiling (the phase events are recorded per step),
    // velocity shards (the host all-reduce callback runs inside the step) or a failed capture
    if (!opt.capture_graphs || profiling || opt.shard_count > 1 || graphs_off)
      return GSIS_DISPATCH(prec, (step_impl<T, S>(mode)));
    for (const StepGraph &g : graphs)
      if (g.mode == mode && g.wstate == d_Wstate) {
        // the host side of step_impl: the read-back word the step may leave alone, the buffer swap
        pin->iters = 0;
        int rc = launch_graph(g.exec);
        if (rc) return rc;
        std::swap(d_Wstate, d_Wnew);
        pending = true;
        pending_mode = mode;
        pending_launches = g.launches;
        return GSIS_OK;
      }
    cudaError_t ce = cudaSuccess;
    if (!gstream) {
      ce = cudaStreamCreateWithFlags(&gstream, cudaStreamNonBlocking);
      for (auto &e : gev)
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    }
    double *ws = d_Wstate, *wn = d_Wnew;
    cudaStream_t user = stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = GSIS_OK;
    const char *where = "stream or event creation";
    if (ce == cudaSuccess) {
      where = "begin capture";
      ce = cudaStreamBeginCapture(gstream, cudaStreamCaptureModeThreadLocal);
    }
    if (ce == cudaSuccess) {
      stream = gstream;  // step_impl enqueues on the capturing stream
      rc = GSIS_DISPATCH(prec, (step_impl<T, S>(mode)));
      stream = user;
      where = "end capture";
      ce = cudaStreamEndCapture(gstream, &graph);
      if (!rc && ce == cudaSuccess && graph) {
        where = "instantiate";
        ce = cudaGraphInstantiate(&exec, graph, 0);
      }
      if (graph) cudaGraphDestroy(graph);
    }
    if (rc || ce != cudaSuccess || !exec) {
      // nothing of the captured step ran: undo its host bookkeeping and launch it directly
      const std::string why = rc ? last_error : std::string(where) + ": " + cudaGetErrorString(ce);
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      d_Wstate = ws;
      d_Wnew = wn;
      pending = false;
      graphs_off = true;
      rc = GSIS_DISPATCH(prec, (step_impl<T, S>(mode)));
      if (!rc) last_error = "CUDA graph capture failed, steps launch directly (" + why + ")";
      return rc;
    }
    graphs.push_back({mode, ws, exec, pending_launches});
    rc = launch_graph(exec);
    if (rc) pending = false;
    return rc;
  }
  int step(int mode) {
    int rc = enqueue_step(mode);
    return rc ? rc : finish_step();
  }
};

// ---------------------------------------------------------------------------------------------

extern "C" void gsis_default_options(gsis_options *o) {
  std::memset(o, 0, sizeof *o);
  o->precision = GSIS_F32;
  o->mode = GSIS_MODE_GSIS;
  o->n_sweeps = 1;
  o->macro_steps = 300;
  o->macro_sweeps = 4;
  o->macro_cfl = 100.0;
  o->macro_tol = 1e-10;
  o->kin_inv_dt = 0.0;
  o->venkat_K = 1.0;
  o->kinetic_presteps = 10;
  o->visc_jump = -1.0;
}

namespace {

// A mesh takes the general (curvilinear) path when its nodes are not a rectilinear product or
// a side is a far field, a pole, or a wrapped axis with several cells.
bool rectilinear_nodes(const gsis_mesh *m) {
  const int N0 = m->ni + 1, N1 = m->nj + 1, N2 = m->nk + 1;
  auto node = [&](int I, int J, int K, int d) { return m->nodes[3 * ((size_t)I + (size_t)N0 * ((size_t)J + (size_t)N1 * K)) + d]; };
  for (int K = 0; K < N2; ++K)
    for (int J = 0; J < N1; ++J)
      for (int I = 0; I < N0; ++I)
        if (node(I, J, K, 0) != node(I, 0, 0, 0) || node(I, J, K, 1) != node(0, J, 0, 1) || node(I, J, K, 2) != node(0, 0, K, 2))
          return false;
  return true;
}

bool needs_general(const gsis_mesh *m) {
  if (m->ncells > 0) return true;
  const int n[3] = {m->ni, m->nj, m->nk};
  for (int side = 0; side < 6; ++side) {
    const int b = m->bc[side];
    if (b == GSIS_BC_FARFIELD || b == GSIS_BC_AXIS || (b == GSIS_BC_PERIODIC && n[side / 2] > 1)) return true;
  }
  return !rectilinear_nodes(m);
}

int validate(const gsis_mesh *m, const gsis_vgrid *vg, const gsis_gas *g, double Kn, const gsis_options *o,
             std::string &why) {
  if (!m || !vg || !g || !o) { why = "NULL argument"; return GSIS_E_INVALID; }
  if (m->ncells < 0) { why = "ncells must be >= 0"; return GSIS_E_INVALID; }
  if (m->ncells > 0) {
    if (!m->unodes || !m->cells || !m->face_patch || m->nnodes < 4) {
      why = "an unstructured mesh needs unodes, cells, face_patch and at least 4 nodes";
      return GSIS_E_INVALID;
    }
    if ((double)m->ncells * NST >= 4294967296.0) { why = "too many cells"; return GSIS_E_UNSUPPORTED; }
    for (size_t t = 0; t < (size_t)8 * m->ncells; ++t)
      if (m->cells[t] < 0 || m->cells[t] >= m->nnodes) { why = "cell node id out of range"; return GSIS_E_INVALID; }
    for (size_t t = 0; t < (size_t)6 * m->ncells; ++t) {
      const int p = m->face_patch[t];
      if (p < -1 || p > 5) { why = "face patch out of range"; return GSIS_E_INVALID; }
      if (p >= 0 && (m->bc[p] < GSIS_BC_WALL || m->bc[p] > GSIS_BC_AXIS)) { why = "bad boundary condition"; return GSIS_E_INVALID; }
      if (p >= 0 && (m->bc[p] == GSIS_BC_WALL || m->bc[p] == GSIS_BC_FARFIELD) && !(m->wall_T[p] > 0)) {
        why = "wall and free-stream temperatures must be positive";
        return GSIS_E_INVALID;
      }
    }
    for (size_t t = 0; t < (size_t)3 * m->nnodes; ++t)
      if (!std::isfinite(m->unodes[t])) { why = "node coordinates must be finite"; return GSIS_E_INVALID; }
  } else {
    if (!m->nodes) { why = "NULL argument"; return GSIS_E_INVALID; }
    if (m->ni < 1 || m->nj < 1 || m->nk < 1 || m->ni > 1023 || m->nj > 1023 || m->nk > 1023) {
      why = "cell counts must be in [1, 1023]";
      return GSIS_E_INVALID;
    }
  }
  if (m->ncells == 0 && (double)m->ni * m->nj * m->nk * NST >= 4294967296.0) {  // 32-bit state offsets in the kernels
    why = "too many cells";
    return GSIS_E_UNSUPPORTED;
  }
  if (vg->npoints > 0) {
    if (!vg->points) { why = "npoints > 0 needs points"; return GSIS_E_INVALID; }
    for (int v = 0; v < vg->npoints; ++v) {
      const double *q = vg->points + 4 * (size_t)v;
      if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) || !(q[3] > 0) || !std::isfinite(q[3])) {
        why = "velocity points must be finite with positive weights";
        return GSIS_E_INVALID;
      }
    }
  } else {
    if (vg->npoints < 0) { why = "npoints must be >= 0"; return GSIS_E_INVALID; }
    for (int d = 0; d < 3; ++d)
      if (vg->n[d] < 1 || !vg->x[d] || !vg->w[d]) { why = "bad velocity grid"; return GSIS_E_INVALID; }
  }
  if (!(Kn > 0)) { why = "Kn must be positive"; return GSIS_E_INVALID; }
  if (!(o->venkat_K > 0)) { why = "venkat_K must be positive"; return GSIS_E_INVALID; }
  if (o->precision != GSIS_F32 && o->precision != GSIS_F64 && o->precision != GSIS_BF16) {
    why = "bad precision";
    return GSIS_E_INVALID;
  }
  if (o->mode != GSIS_MODE_GSIS && o->mode != GSIS_MODE_DVM) { why = "bad mode"; return GSIS_E_INVALID; }
  if (o->kinetic_ring != 0 && o->kinetic_ring != 1) { why = "kinetic_ring must be 0 or 1"; return GSIS_E_INVALID; }
  if (o->euler_presteps < 0) { why = "euler_presteps must be >= 0"; return GSIS_E_INVALID; }
  if (o->wall_flux != GSIS_WALL_EQ && o->wall_flux != GSIS_WALL_G13) { why = "bad wall_flux"; return GSIS_E_INVALID; }
  if (o->positive_faces != 0 && o->positive_faces != 1) { why = "positive_faces must be 0 or 1"; return GSIS_E_INVALID; }
  if (o->capture_graphs != 0 && o->capture_graphs != 1) { why = "capture_graphs must be 0 or 1"; return GSIS_E_INVALID; }
  if (!(o->relax >= 0.0 && o->relax <= 1.0)) { why = "relax must be in [0, 1]"; return GSIS_E_INVALID; }
  if (!(o->visc_jump <= 1.0)) { why = "visc_jump must be at most 1"; return GSIS_E_INVALID; }
  if (o->shard_count > 1 && (o->shard_index < 0 || o->shard_index >= o->shard_count || !o->allreduce)) {
    why = "velocity sharding needs 0 <= shard_index < shard_count and an allreduce callback";
    return GSIS_E_INVALID;
  }
  if (g->model == GSIS_RYKOV && (!(g->d_r > 0) || !(g->Z_r > 0))) {
    why = "Rykov needs d_r > 0 and Z_r > 0";
    return GSIS_E_INVALID;
  }
  if (g->model != GSIS_SHAKHOV && g->model != GSIS_RYKOV) { why = "bad model"; return GSIS_E_INVALID; }
  if (!(o->kin_inv_dt >= 0.0) || !std::isfinite(o->kin_inv_dt)) { why = "kin_inv_dt must be finite and >= 0"; return GSIS_E_INVALID; }
  if (o->kin_inv_dt != 0.0 && o->mode == GSIS_MODE_GSIS) {
    why = "the synthetic solve takes the face fluxes of a steady kinetic step: kin_inv_dt must be 0 in GSIS mode";
    return GSIS_E_UNSUPPORTED;
  }
  const bool general = needs_general(m);
  if (!general && o->n_sweeps != 1) {
    why = "rectilinear colour sweeps are exact in one pass: n_sweeps must be 1";
    return GSIS_E_UNSUPPORTED;
  }
  if (general && (o->n_sweeps < 1 || o->n_sweeps > 64)) { why = "n_sweeps must be in [1, 64]"; return GSIS_E_INVALID; }
  if (m->ncells > 0) return GSIS_OK;  // faces, volumes and colours are checked when the mesh is built
  const int n[3] = {m->ni, m->nj, m->nk};
  bool seen_inactive = false;
  for (int a = 0; a < 3; ++a) {
    const bool active = n[a] > 1;
    const int lo = m->bc[2 * a], hi = m->bc[2 * a + 1];
    for (int t = 0; t < 2; ++t)
      if (m->bc[2 * a + t] < GSIS_BC_WALL || m->bc[2 * a + t] > GSIS_BC_AXIS) { why = "bad boundary condition"; return GSIS_E_INVALID; }
    if (!active) {
      if (lo != GSIS_BC_PERIODIC || hi != GSIS_BC_PERIODIC) {
        why = "an axis with one cell must be periodic on both sides";
        return GSIS_E_INVALID;
      }
      seen_inactive = true;
    } else {
      if (seen_inactive) { why = "active axes must come first (x, then y, then z)"; return GSIS_E_UNSUPPORTED; }
      if ((lo == GSIS_BC_PERIODIC) != (hi == GSIS_BC_PERIODIC)) {
        why = "a periodic axis is periodic on both sides";
        return GSIS_E_INVALID;
      }
      if (lo == GSIS_BC_PERIODIC && n[a] < 3) { why = "a wrapped axis needs at least 3 cells"; return GSIS_E_INVALID; }
      // the synthetic solve updates red and black cells (i+j+k even / odd) in parallel: across
      // the wrap of an odd axis two neighbours share a colour
      if (lo == GSIS_BC_PERIODIC && (n[a] & 1) && (o->mode == GSIS_MODE_GSIS || o->euler_presteps > 0)) {
        why = "the synthetic solve needs an even number of cells on a wrapped axis";
        return GSIS_E_UNSUPPORTED;
      }
    }
  }
  for (int s = 0; s < 6; ++s)
    if ((m->bc[s] == GSIS_BC_WALL || m->bc[s] == GSIS_BC_FARFIELD) && !(m->wall_T[s] > 0)) {
      why = "wall and free-stream temperatures must be positive";
      return GSIS_E_INVALID;
    }
  if (!general && o->euler_presteps > 0) {
    why = "Euler presteps are built on general meshes only";
    return GSIS_E_UNSUPPORTED;
  }
  if (!general && o->positive_faces) {
    why = "positive face values are built on general meshes only";
    return GSIS_E_UNSUPPORTED;
  }
  if (!general && o->relax > 0.0 && o->relax < 1.0) {
    why = "the relaxed GSIS update is built on general meshes only";
    return GSIS_E_UNSUPPORTED;
  }
  if (!general && o->visc_jump > 0.0) {
    why = "the viscous face-gradient jump term is built on general meshes only";
    return GSIS_E_UNSUPPORTED;
  }
  if (general) return GSIS_OK;  // volumes are checked when the geometry is built
  const int N0 = m->ni + 1, N1 = m->nj + 1, N2 = m->nk + 1;
  auto node = [&](int I, int J, int K, int d) { return m->nodes[3 * ((size_t)I + (size_t)N0 * ((size_t)J + (size_t)N1 * K)) + d]; };
  (void)N2;
  for (int I = 1; I < N0; ++I) if (!(node(I, 0, 0, 0) > node(I - 1, 0, 0, 0))) { why = "x nodes must increase"; return GSIS_E_INVALID; }
  for (int J = 1; J < N1; ++J) if (!(node(0, J, 0, 1) > node(0, J - 1, 0, 1))) { why = "y nodes must increase"; return GSIS_E_INVALID; }
  for (int K = 1; K < N2; ++K) if (!(node(0, 0, K, 2) > node(0, 0, K - 1, 2))) { why = "z nodes must increase"; return GSIS_E_INVALID; }
  return GSIS_OK;
}

// Tile shape (TX, TY, TZ), TX TY TZ = VB, that splits every octant of a tensor-product grid
// exactly: each axis's count of negative and of non-negative nodes is a multiple of its tile
// extent.  Only shapes with TX + TY + TZ <= KFAC_MAX per-axis factors qualify; {0, 0, 0} if none.
static void choose_tile(const gsis_vgrid *vg, int tile[3]) {
  static const int shapes[3][3] = {{4, 4, 2}, {4, 2, 4}, {2, 4, 4}};
  tile[0] = tile[1] = tile[2] = 0;
  int neg[3], pos[3];
  for (int a = 0; a < 3; ++a) {
    neg[a] = pos[a] = 0;
    for (int i = 0; i < vg->n[a]; ++i) (vg->x[a][i] < 0 ? neg[a] : pos[a])++;
  }
  for (const auto &t : shapes) {
    bool ok = t[0] + t[1] + t[2] <= KFAC_MAX;
    for (int a = 0; a < 3 && ok; ++a) ok = neg[a] % t[a] == 0 && pos[a] % t[a] == 0;
    if (ok) {
      for (int a = 0; a < 3; ++a) tile[a] = t[a];
      return;
    }
  }
}

// Velocity slots: velocities grouped by octant (sign of each component, 0 counted +).  With a
// tile shape each block of VB slots is one TX x TY x TZ tile of its octant, lane
// lx + TX (ly + TY lz) at the tile's node (lx, ly, lz), so that a Maxwellian over the block is a
// product of TX + TY + TZ one-dimensional factors; otherwise each octant is listed x-fastest and
// padded to a multiple of VB with weight-0 copies of its first velocity.
void build_slots(const gsis_vgrid *vg, const int tile[3], std::vector<int> &slot_canon, std::vector<int8_t> &boct,
                 std::vector<double> &vel64) {
  slot_canon.clear();
  boct.clear();
  vel64.clear();
  if (vg->npoints > 0) {
    // an unstructured set: each octant's points in input order, padded with weight-0 copies
    for (int oct = 0; oct < 8; ++oct) {
      std::vector<int> list;
      for (int v = 0; v < vg->npoints; ++v) {
        const double *q = vg->points + 4 * (size_t)v;
        const int o = (q[0] < 0 ? 1 : 0) | (q[1] < 0 ? 2 : 0) | (q[2] < 0 ? 4 : 0);
        if (o == oct) list.push_back(v);
      }
      if (list.empty()) continue;
      const size_t padded = (list.size() + VB - 1) / VB * VB;
      for (size_t t = 0; t < padded; ++t) {
        const bool real = t < list.size();
        const double *q = vg->points + 4 * (size_t)(real ? list[t] : list[0]);
        slot_canon.push_back(real ? list[t] : list[0]);
        vel64.insert(vel64.end(), {q[0], q[1], q[2], real ? q[3] : 0.0});
      }
      for (size_t b = 0; b < padded / VB; ++b) boct.push_back((int8_t)oct);
    }
    return;
  }
  const int nx = vg->n[0], ny = vg->n[1], nz = vg->n[2];
  for (int oct = 0; oct < 8; ++oct) {
    std::vector<int> ax[3];
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < vg->n[a]; ++i)
        if ((vg->x[a][i] < 0) == (((oct >> a) & 1) != 0)) ax[a].push_back(i);
    std::vector<int> list;
    if (tile[0] > 0) {
      // nodes by increasing |xi| on each axis, so that mirror-image octants list mirror-image
      // velocities in the same lane order
      for (int a = 0; a < 3; ++a)
        if ((oct >> a) & 1) std::reverse(ax[a].begin(), ax[a].end());
      const int T0 = tile[0], T1 = tile[1], T2 = tile[2];
      for (size_t bz = 0; bz < ax[2].size(); bz += T2)
        for (size_t by = 0; by < ax[1].size(); by += T1)
          for (size_t bx = 0; bx < ax[0].size(); bx += T0)
            for (int lz = 0; lz < T2; ++lz)
              for (int ly = 0; ly < T1; ++ly)
                for (int lx = 0; lx < T0; ++lx)
                  list.push_back(ax[0][bx + lx] + nx * (ax[1][by + ly] + ny * ax[2][bz + lz]));
    } else {
      for (int iz : ax[2])
        for (int iy : ax[1])
          for (int ix : ax[0]) list.push_back(ix + nx * (iy + ny * iz));
    }
    if (list.empty()) continue;
    const size_t padded = (list.size() + VB - 1) / VB * VB;
    for (size_t t = 0; t < padded; ++t) {
      const bool real = t < list.size();
      const int v = real ? list[t] : list[0];
      const int ix = v % nx, iy = (v / nx) % ny, iz = v / (nx * ny);
      slot_canon.push_back(v);
      vel64.push_back(vg->x[0][ix]);
      vel64.push_back(vg->x[1][iy]);
      vel64.push_back(vg->x[2][iz]);
      vel64.push_back(real ? vg->w[0][ix] * vg->w[1][iy] * vg->w[2][iz] : 0.0);
    }
    for (size_t b = 0; b < padded / VB; ++b) boct.push_back((int8_t)oct);
  }
}

template <typename T>
std::vector<GenCell<T>> cast_gen(const std::vector<GenCell<double>> &in) {
  std::vector<GenCell<T>> out(in.size());
  for (size_t c = 0; c < in.size(); ++c) {
    for (int s = 0; s < 6; ++s) {
      for (int d = 0; d < 3; ++d) {
        out[c].f[s].S[d] = (T)in[c].f[s].S[d];
        out[c].f[s].r[d] = (T)in[c].f[s].r[d];
        out[c].f[s].w[d] = (T)in[c].f[s].w[d];
      }
      out[c].f[s].invA = (T)in[c].f[s].invA;
    }
    out[c].invV = (T)in[c].invV;
    out[c].eps2 = (T)in[c].eps2;
  }
  return out;
}

template <typename T>
std::vector<AxisCell<T>> cast_axis(const std::vector<AxisCell<double>> &in) {
  std::vector<AxisCell<T>> out(in.size());
  for (size_t i = 0; i < in.size(); ++i)
    out[i] = {(T)in[i].invh, (T)in[i].rlo, (T)in[i].rhi, (T)in[i].clo, (T)in[i].chi, (T)in[i].h, (T)in[i].pad0, (T)0};
  return out;
}

}  // namespace

// Finite-volume geometry of a general structured block (Section 3.2): a face's area vector is
// half the cross product of its diagonals, oriented out of the cell; its centre the mean of its
// corners; a cell's centre the mean of its 8 corners and its volume (1/3) sum x_f . S_f
// (divergence theorem with F = x / 3).  Least squares: the unweighted normal equations over
// the in-domain neighbours, with the components of one-cell axes fixed to zero, inverted once
// per cell into per-side weights.  Wall faces are numbered cell by cell, side by side.
static int build_general(gsis_solver *s, const gsis_mesh *m) {
  const int n[3] = {m->ni, m->nj, m->nk}, nc = s->nc;
  const int N0 = m->ni + 1, N1 = m->nj + 1;
  auto P = [&](int I, int J, int K, double *p) {
    const double *q = m->nodes + 3 * ((size_t)I + (size_t)N0 * ((size_t)J + (size_t)N1 * K));
    p[0] = q[0];
    p[1] = q[1];
    p[2] = q[2];
  };
  s->gen64.assign(nc, GenCell<double>{});
  s->gnb.assign((size_t)6 * nc, NB_ABSENT);
  s->gwid.assign((size_t)6 * nc, -1);
  s->gin.assign((size_t)6 * nc, 0);
  s->vol.assign(nc, 0.0);
  s->xc64.assign((size_t)3 * nc, 0.0);
  std::vector<double> &xc = s->xc64;
  s->vsum = 0.0;
  s->nwall = 0;
  s->wall_cell.clear();
  s->wall_side.clear();
  s->wall_area.clear();
  s->closed = 1;
  for (int side = 0; side < 6; ++side)
    if (m->bc[side] == GSIS_BC_FARFIELD) s->closed = 0;
  const double K3 = s->opt.venkat_K * s->opt.venkat_K * s->opt.venkat_K;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        const int c = i + n[0] * (j + n[1] * k);
        double cen[3] = {0, 0, 0}, p[3];
        for (int t = 0; t < 8; ++t) {
          P(i + (t & 1), j + ((t >> 1) & 1), k + (t >> 2), p);
          for (int d = 0; d < 3; ++d) cen[d] += p[d] / 8.0;
        }
        for (int d = 0; d < 3; ++d) xc[3 * (size_t)c + d] = cen[d];
        GenCell<double> &g = s->gen64[c];
        double V = 0.0;
        for (int side = 0; side < 6; ++side) {
          const int a = side / 2, hi = side & 1;
          // the face's corners in cyclic order: the two tangential index directions
          const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
          double q[4][3];
          for (int t = 0; t < 4; ++t) {
            int idx[3] = {i, j, k};
            idx[a] += hi;
            idx[t1] += (t == 1 || t == 2);
            idx[t2] += (t >= 2);
            P(idx[0], idx[1], idx[2], q[t]);
          }
          double d1[3], d2[3], S[3], xf[3];
          for (int d = 0; d < 3; ++d) {
            d1[d] = q[2][d] - q[0][d];
            d2[d] = q[3][d] - q[1][d];
            xf[d] = 0.25 * (q[0][d] + q[1][d] + q[2][d] + q[3][d]);
          }
          S[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
          S[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
          S[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
          double r[3] = {xf[0] - cen[0], xf[1] - cen[1], xf[2] - cen[2]};
          if (S[0] * r[0] + S[1] * r[1] + S[2] * r[2] < 0)
            for (int d = 0; d < 3; ++d) S[d] = -S[d];
          V += (xf[0] * S[0] + xf[1] * S[1] + xf[2] * S[2]) / 3.0;
          const double A = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
          for (int d = 0; d < 3; ++d) {
            g.f[side].S[d] = S[d];
            g.f[side].r[d] = r[d];
          }
          g.f[side].invA = A > 0 ? 1.0 / A : 0.0;
          int idx[3] = {i, j, k};
          idx[a] += hi ? 1 : -1;
          int nb;
          const int b = m->bc[side];
          if (n[a] == 1) nb = NB_ABSENT;
          else if (idx[a] >= 0 && idx[a] < n[a]) nb = idx[0] + n[0] * (idx[1] + n[1] * idx[2]);
          else if (b == GSIS_BC_PERIODIC) {
            idx[a] = (idx[a] + n[a]) % n[a];
            nb = idx[0] + n[0] * (idx[1] + n[1] * idx[2]);
          } else if (b == GSIS_BC_AXIS) nb = NB_AXIS;
          else if (b == GSIS_BC_FARFIELD) {
            nb = NB_FAR;
            // a reservoir boundary: the free stream enters unless it leaves through the face
            // faster than sound, c^2 = gamma R T with gamma = (5 + d_r) / (3 + d_r) of the
            // free stream in equilibrium (5/3 monatomic, 7/5 for d_r = 2) and R T = T / 2
            const double *U = m->wall_u[side];
            const double un = U[0] * S[0] + U[1] * S[1] + U[2] * S[2];
            const double dr = s->gas.model == GSIS_RYKOV ? s->gas.d_r : 0.0;
            const double gam = (5.0 + dr) / (3.0 + dr);
            s->gin[6 * (size_t)c + side] = un <= std::sqrt(0.5 * gam * m->wall_T[side]) * A;
          } else {
            nb = NB_WALL;
            s->gwid[6 * (size_t)c + side] = s->nwall++;
            s->wall_cell.push_back(c);
            s->wall_side.push_back(side);
            s->wall_area.push_back(A);
          }
          s->gnb[6 * (size_t)c + side] = nb;
        }
        if (!(V > 0)) return s->fail(GSIS_E_INVALID, "cell %d has volume %g", c, V);
        s->vol[c] = V;
        s->vsum += V;
        g.invV = 1.0 / V;
        g.eps2 = K3 * V;
      }
  // least-squares weights
  for (int c = 0; c < nc; ++c) {
    GenCell<double> &g = s->gen64[c];
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dv[6][3];
    for (int side = 0; side < 6; ++side) {
      const int nb = s->gnb[6 * (size_t)c + side];
      for (int d = 0; d < 3; ++d) dv[side][d] = nb >= 0 ? xc[3 * (size_t)nb + d] - xc[3 * (size_t)c + d] : 0.0;
      for (int a = 0; a < 3; ++a)
        if (n[a] == 1) dv[side][a] = 0.0;
      for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) A[r][q] += dv[side][r] * dv[side][q];
    }
    for (int a = 0; a < 3; ++a)
      if (n[a] == 1) A[a][a] = 1.0;
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(std::fabs(det) > 0)) return s->fail(GSIS_E_INVALID, "cell %d: singular least-squares system", c);
    double inv[3][3];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        // adjugate / det: cofactor of (q, r)
        const int r1 = (q + 1) % 3, r2 = (q + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
        inv[r][q] = (A[r1][c1] * A[r2][c2] - A[r1][c2] * A[r2][c1]) / det;
      }
    for (int side = 0; side < 6; ++side)
      for (int r = 0; r < 3; ++r)
        g.f[side].w[r] = inv[r][0] * dv[side][0] + inv[r][1] * dv[side][1] + inv[r][2] * dv[side][2];
  }
  return GSIS_OK;
}

// The kinetic sweeps of general meshes, per velocity octant (signs d): the cells ranked by the
// mean over their nodes of ((d_x x) + (d_y y)) + (d_z z) (a structured cell's 8 corners, an
// unstructured cell's distinct nodes, summed in that order), ties by index, which places a cell
// after the cells its flow comes from.  A cell's colour is one more than the largest colour of
// its face neighbours ranked before it (0 without one): a colour's cells share no face, and the
// octant sweeps colour by colour, in index order within a colour, from per-octant offsets
// (col_stride).  On curved blocks the index-space hyperplanes do not follow the flow (near a
// sphere's poles they run across it, and GSIS there grew instead of converging), and a greedy
// colouring shared by every octant carries information one cell against the flow per pass.
static void octant_sweeps(gsis_solver *s, const gsis_mesh *m) {
  const int nc = (int)s->nc;
  KinGeom &g = s->kg;
  std::vector<std::vector<int>> korder(8), koff(8);
  int kmax = 0;
  std::vector<double> pkey(nc);
  std::vector<int> byk(nc), rank(nc), kc(nc);
  const size_t N0 = (size_t)m->ni + 1, N1 = (size_t)m->nj + 1;
  for (int oct = 0; oct < 8; ++oct) {
    const double d[3] = {oct & 1 ? -1.0 : 1.0, oct & 2 ? -1.0 : 1.0, oct & 4 ? -1.0 : 1.0};
    for (int c = 0; c < nc; ++c) {
      double sum = 0.0;
      int cnt = 0;
      if (m->ncells > 0) {
        const int *ids = m->cells + 8 * (size_t)c;
        for (int t = 0; t < 8; ++t) {
          bool dup = false;
          for (int u = 0; u < t; ++u) dup = dup || ids[u] == ids[t];
          if (dup) continue;
          const double *x = m->unodes + 3 * (size_t)ids[t];
          sum += ((d[0] * x[0]) + (d[1] * x[1])) + (d[2] * x[2]);
          ++cnt;
        }
      } else {
        const int i = c % m->ni, j = (c / m->ni) % m->nj, k = c / (m->ni * m->nj);
        for (int t = 0; t < 8; ++t) {
          const size_t I = i + (t & 1), J = j + (t >> 1 & 1), K = k + (t >> 2);
          const double *x = m->nodes + 3 * (I + N0 * (J + N1 * K));
          sum += ((d[0] * x[0]) + (d[1] * x[1])) + (d[2] * x[2]);
          ++cnt;
        }
      }
      pkey[c] = sum / cnt;
      byk[c] = c;
    }
    std::sort(byk.begin(), byk.end(), [&](int a, int b) { return pkey[a] < pkey[b] || (pkey[a] == pkey[b] && a < b); });
    for (int r = 0; r < nc; ++r) rank[byk[r]] = r;
    int nk = 0;
    for (int r = 0; r < nc; ++r) {
      const int c = byk[r];
      int k = 0;
      for (int side = 0; side < 6; ++side) {
        const int nb = s->gnb[6 * (size_t)c + side];
        if (nb >= 0 && rank[nb] < r) k = std::max(k, kc[nb] + 1);
      }
      kc[c] = k;
      nk = std::max(nk, k + 1);
    }
    std::vector<int> cnt(nk + 1, 0);
    for (int c = 0; c < nc; ++c) ++cnt[kc[c] + 1];
    for (int k = 0; k < nk; ++k) cnt[k + 1] += cnt[k];
    koff[oct] = cnt;
    korder[oct].assign(nc, 0);
    for (int c = 0; c < nc; ++c) korder[oct][cnt[kc[c]]++] = c;  // index order within a colour
    kmax = std::max(kmax, nk);
  }
  s->col_stride = kmax + 1;
  s->col_off.assign((size_t)8 * s->col_stride, 0);
  g.ncol = kmax;
  g.maxcol = 0;
  s->natcell.assign((size_t)8 * nc, int4{0, 0, 0, 0});
  for (int oct = 0; oct < 8; ++oct) {
    const int nk = (int)koff[oct].size() - 1;
    for (int k = 0; k <= kmax; ++k) s->col_off[(size_t)oct * s->col_stride + k] = koff[oct][std::min(k, nk)];
    for (int k = 0; k < nk; ++k) g.maxcol = std::max(g.maxcol, koff[oct][k + 1] - koff[oct][k]);
    for (int e = 0; e < nc; ++e) s->natcell[(size_t)oct * nc + e] = int4{korder[oct][e], 0, 0, 0};
  }
}

// Unstructured meshes: every cell a hexahedron of node ids (other shapes repeat ids), its six
// sides with corners in cyclic order; a side's geometry as on structured blocks (a quadrilateral:
// half the cross product of its diagonals, centre the corner mean), a side with three distinct
// corners a triangle (half the cross product of two edges, centre their mean), fewer: no area.
static const int kHexSide[6][4] = {{0, 2, 6, 4}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 3, 7, 6}, {0, 1, 3, 2}, {4, 5, 7, 6}};

static int setup_unstructured_mesh(gsis_solver *s, const gsis_mesh *m) {
  const int nc = m->ncells;
  s->unstructured = true;
  s->general = true;
  s->nc = nc;
  s->n[0] = nc;
  s->n[1] = s->n[2] = 1;
  for (int a = 0; a < 3; ++a) {
    // placeholders: the axis arrays serve rectilinear blocks only
    s->X[a] = {0.0, 1.0};
    AxisCell<double> c{};
    c.h = 1.0;
    c.invh = 1.0;
    s->axc[a].assign(1, c);
  }
  KinGeom &g = s->kg;
  g = KinGeom{};
  g.nc = nc;
  g.n[0] = nc;
  g.n[1] = g.n[2] = 1;
  for (int a = 0; a < 3; ++a) g.act[a] = 1;
  g.nact = 3;
  g.K3 = s->opt.venkat_K * s->opt.venkat_K * s->opt.venkat_K;
  for (int side = 0; side < 6; ++side) g.wall_base[side] = -1;
  for (int p = 0; p < 6; ++p) {
    for (int d = 0; d < 3; ++d) s->wall_uT[p][d] = m->wall_u[p][d];
    s->wall_uT[p][3] = m->wall_T[p];
  }
  s->nwall = 0;
  s->wall_cell.clear();
  s->wall_side.clear();
  s->wall_area.clear();
  s->wall_patch.clear();
  s->wall_sides_list.clear();
  s->closed = 1;
  s->gen64.assign(nc, GenCell<double>{});
  s->gnb.assign((size_t)6 * nc, NB_ABSENT);
  s->gwid.assign((size_t)6 * nc, -1);
  s->gin.assign((size_t)6 * nc, 0);
  s->gnf.assign((size_t)6 * nc, 255);
  s->gpat.assign((size_t)6 * nc, 255);
  s->vol.assign(nc, 0.0);
  s->xc64.assign((size_t)3 * nc, 0.0);
  s->vsum = 0.0;
  const double K3 = g.K3;
  auto X = [&](int id, int d) { return m->unodes[3 * (size_t)id + d]; };
  std::vector<double> area((size_t)6 * nc, 0.0);
  std::vector<std::array<int, 4>> key((size_t)6 * nc);
  for (int c = 0; c < nc; ++c) {
    const int *ids = m->cells + 8 * (size_t)c;
    std::vector<int> dist;
    for (int t = 0; t < 8; ++t)
      if (std::find(dist.begin(), dist.end(), ids[t]) == dist.end()) dist.push_back(ids[t]);
    double cen[3] = {0, 0, 0};
    for (int id : dist)
      for (int d = 0; d < 3; ++d) cen[d] += X(id, d) / dist.size();
    for (int d = 0; d < 3; ++d) s->xc64[3 * (size_t)c + d] = cen[d];
    GenCell<double> &gc = s->gen64[c];
    double V = 0.0;
    for (int side = 0; side < 6; ++side) {
      int q[4];
      for (int t = 0; t < 4; ++t) q[t] = ids[kHexSide[side][t]];
      std::vector<int> fd;
      for (int t = 0; t < 4; ++t)
        if (std::find(fd.begin(), fd.end(), q[t]) == fd.end()) fd.push_back(q[t]);
      double S[3] = {0, 0, 0}, xf[3] = {0, 0, 0};
      if (fd.size() == 4) {
        double d1[3], d2[3];
        for (int d = 0; d < 3; ++d) {
          d1[d] = X(q[2], d) - X(q[0], d);
          d2[d] = X(q[3], d) - X(q[1], d);
          xf[d] = 0.25 * (X(q[0], d) + X(q[1], d) + X(q[2], d) + X(q[3], d));
        }
        S[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
        S[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
        S[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
      } else if (fd.size() == 3) {
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) {
          e1[d] = X(fd[1], d) - X(fd[0], d);
          e2[d] = X(fd[2], d) - X(fd[0], d);
          xf[d] = (X(fd[0], d) + X(fd[1], d) + X(fd[2], d)) / 3.0;
        }
        S[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
        S[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
        S[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
      } else {
        for (int t = 0; t < 4; ++t)
          for (int d = 0; d < 3; ++d) xf[d] += 0.25 * X(q[t], d);
      }
      double r[3] = {xf[0] - cen[0], xf[1] - cen[1], xf[2] - cen[2]};
      if (S[0] * r[0] + S[1] * r[1] + S[2] * r[2] < 0)
        for (int d = 0; d < 3; ++d) S[d] = -S[d];
      V += (xf[0] * S[0] + xf[1] * S[1] + xf[2] * S[2]) / 3.0;
      const double A = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
      for (int d = 0; d < 3; ++d) {
        gc.f[side].S[d] = S[d];
        gc.f[side].r[d] = r[d];
      }
      gc.f[side].invA = A > 0 ? 1.0 / A : 0.0;
      area[6 * (size_t)c + side] = fd.size() >= 3 ? A : 0.0;
      std::sort(fd.begin(), fd.end());
      std::array<int, 4> k{-1, -1, -1, -1};
      for (size_t t = 0; t < fd.size(); ++t) k[t] = fd[t];
      key[6 * (size_t)c + side] = k;
    }
    if (!(V > 0)) return s->fail(GSIS_E_INVALID, "cell %d has volume %g", c, V);
    s->vol[c] = V;
    s->vsum += V;
    gc.invV = 1.0 / V;
    gc.eps2 = K3 * V;
  }
  // shared sides: the same node set on two cells
  std::map<std::array<int, 4>, int> open;
  for (int c = 0; c < nc; ++c)
    for (int side = 0; side < 6; ++side) {
      const size_t f = 6 * (size_t)c + side;
      if (!(area[f] > 0)) continue;
      auto it = open.find(key[f]);
      if (it == open.end()) {
        open.emplace(key[f], (int)f);
        continue;
      }
      const int o = it->second, oc = o / 6, os = o % 6;
      open.erase(it);
      if (m->face_patch[f] >= 0 || m->face_patch[o] >= 0)
        return s->fail(GSIS_E_INVALID, "cell %d side %d is shared with cell %d but has a boundary patch", c, side, oc);
      s->gnb[f] = oc;
      s->gnf[f] = (unsigned char)os;
      s->gnb[o] = c;
      s->gnf[o] = (unsigned char)side;
    }
  // boundary sides, walls numbered cell by cell, side by side
  bool one_layer = false;
  const double dr = s->gas.model == GSIS_RYKOV ? s->gas.d_r : 0.0;
  const double gam = (5.0 + dr) / (3.0 + dr);
  for (int c = 0; c < nc; ++c)
    for (int side = 0; side < 6; ++side) {
      const size_t f = 6 * (size_t)c + side;
      if (!(area[f] > 0) || s->gnb[f] >= 0) continue;
      const int p = m->face_patch[f];
      if (p < 0) return s->fail(GSIS_E_INVALID, "cell %d side %d is neither shared nor on a boundary patch", c, side);
      s->gpat[f] = (unsigned char)p;
      const double *S = s->gen64[c].f[side].S;
      const double A = area[f];
      switch (m->bc[p]) {
        case GSIS_BC_WALL:
          s->gnb[f] = NB_WALL;
          s->gwid[f] = s->nwall++;
          s->wall_cell.push_back(c);
          s->wall_side.push_back(side);
          s->wall_area.push_back(A);
          s->wall_patch.push_back(p);
          break;
        case GSIS_BC_FARFIELD: {
          s->gnb[f] = NB_FAR;
          s->closed = 0;
          const double *U = m->wall_u[p];
          s->gin[f] = U[0] * S[0] + U[1] * S[1] + U[2] * S[2] <= std::sqrt(0.5 * gam * m->wall_T[p]) * A;
          break;
        }
        case GSIS_BC_PERIODIC:
          if (std::fabs(S[2]) < (1.0 - 1e-9) * A)
            return s->fail(GSIS_E_UNSUPPORTED, "PERIODIC patches of an unstructured mesh must be normal to z (cell %d)", c);
          s->gnb[f] = NB_ABSENT;
          one_layer = true;
          break;
        default:
          s->gnb[f] = NB_AXIS;
      }
    }
  // Least-squares stencils (no z component on a one-layer mesh): on a mesh of hexahedra a cell
  // fits its face neighbours; on a mesh with prisms, pyramids or tetrahedra every other cell
  // sharing a node with it (the second-order upwind scheme with face neighbours only is unstable
  // on simplices).  A cell
  // whose stencil does not determine a gradient (a corner tetrahedron) also fits the centres of
  // its boundary faces, each carrying the cell's own value: rows of the normal matrix that add
  // nothing to the gradient sum.
  const bool active[3] = {true, true, !one_layer};
  const int nact = one_layer ? 2 : 3;
  auto det3 = [](const double A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  };
  std::vector<std::vector<int>> node_cells(m->nnodes);
  std::vector<int> ndist(nc, 0);
  for (int c = 0; c < nc; ++c) {
    const int *ids = m->cells + 8 * (size_t)c;
    for (int t = 0; t < 8; ++t) {
      bool dup = false;
      for (int u = 0; u < t; ++u) dup = dup || ids[u] == ids[t];
      if (!dup) {
        node_cells[ids[t]].push_back(c);
        ++ndist[c];
      }
    }
  }
  // (a mesh with any simplex cell takes node-sharing stencils everywhere: face stencils on its
  // hexahedra next to simplices' node stencils left the mixed scheme unstable too)
  const bool all_hex = std::all_of(ndist.begin(), ndist.end(), [](int k) { return k == 8; });
  s->simplex = !all_hex;
  s->gs_off.assign(nc + 1, 0);
  s->gs_idx.clear();
  s->gs_w.clear();
  for (int c = 0; c < nc; ++c) {
    std::vector<int> st;
    if (all_hex) {
      for (int side = 0; side < 6; ++side)
        if (s->gnb[6 * (size_t)c + side] >= 0) st.push_back(s->gnb[6 * (size_t)c + side]);
    } else {
      for (int t = 0; t < 8; ++t)
        for (int o : node_cells[m->cells[8 * (size_t)c + t]])
          if (o != c && std::find(st.begin(), st.end(), o) == st.end()) st.push_back(o);
      std::sort(st.begin(), st.end());
      if (st.size() > 80) return s->fail(GSIS_E_UNSUPPORTED, "cell %d: %d stencil cells (at most 80)", c, (int)st.size());
    }
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    std::vector<std::array<double, 3>> dv(st.size());
    for (size_t e = 0; e < st.size(); ++e) {
      for (int d = 0; d < 3; ++d)
        dv[e][d] = active[d] ? s->xc64[3 * (size_t)st[e] + d] - s->xc64[3 * (size_t)c + d] : 0.0;
      for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) A[r][q] += dv[e][r] * dv[e][q];
    }
    for (int a = 0; a < 3; ++a)
      if (!active[a]) A[a][a] = 1.0;
    double tr = 0.0;
    for (int a = 0; a < 3; ++a)
      if (active[a]) tr += A[a][a];
    if (!(det3(A) > 1e-9 * std::pow(tr, nact)))
      for (int side = 0; side < 6; ++side) {
        const size_t f = 6 * (size_t)c + side;
        if (!(area[f] > 0) || s->gnb[f] >= 0 || s->gnb[f] == NB_ABSENT) continue;
        const double *r = s->gen64[c].f[side].r;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (active[a] && active[b]) A[a][b] += r[a] * r[b];
      }
    const double det = det3(A);
    if (!(std::fabs(det) > 0)) return s->fail(GSIS_E_INVALID, "cell %d: singular least-squares system", c);
    double inv[3][3];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        const int r1 = (q + 1) % 3, r2 = (q + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
        inv[r][q] = (A[r1][c1] * A[r2][c2] - A[r1][c2] * A[r2][c1]) / det;
      }
    for (size_t e = 0; e < st.size(); ++e) {
      s->gs_idx.push_back(st[e]);
      for (int r = 0; r < 3; ++r) s->gs_w.push_back(inv[r][0] * dv[e][0] + inv[r][1] * dv[e][1] + inv[r][2] * dv[e][2]);
    }
    s->gs_off[c + 1] = (int)s->gs_idx.size();
  }
  // greedy colouring of the face graph, cells in index order
  std::vector<int> colour(nc, -1);
  int ncol = 0;
  for (int c = 0; c < nc; ++c) {
    unsigned long long used = 0;
    for (int side = 0; side < 6; ++side) {
      const int nb = s->gnb[6 * (size_t)c + side];
      if (nb >= 0 && colour[nb] >= 0) used |= 1ull << colour[nb];
    }
    int k = 0;
    while (used >> k & 1ull) ++k;
    colour[c] = k;
    ncol = std::max(ncol, k + 1);
  }
  if (ncol > MACRO_MAX_COLOURS) return s->fail(GSIS_E_UNSUPPORTED, "%d colours (at most %d)", ncol, MACRO_MAX_COLOURS);
  std::vector<int> order;
  s->col_off.assign(ncol + 1, 0);
  g.ncol = ncol;
  g.maxcol = 0;
  for (int k = 0; k < ncol; ++k) {
    for (int c = 0; c < nc; ++c)
      if (colour[c] == k) order.push_back(c);
    s->col_off[k + 1] = (int)order.size();
    g.maxcol = std::max(g.maxcol, s->col_off[k + 1] - s->col_off[k]);
  }
  s->col_cell = order;
  s->pos_of.assign(nc, 0);
  s->entries.assign(nc, EntryInfo{});
  // the synthetic solve's LU-SGS passes over the greedy colours
  s->colcells = order;
  s->mcol_off = s->col_off;
  s->ncol0 = s->col_off[1];
  octant_sweeps(s, m);
  return GSIS_OK;
}

static int setup_mesh(gsis_solver *s, const gsis_mesh *m);
static int setup_velocities(gsis_solver *s, const gsis_vgrid *vg);

static int setup(gsis_solver *s, const gsis_mesh *m, const gsis_vgrid *vg) {
  int rc0 = m->ncells > 0 ? setup_unstructured_mesh(s, m) : setup_mesh(s, m);
  if (rc0) return rc0;
  return setup_velocities(s, vg);
}

// structured blocks
static int setup_mesh(gsis_solver *s, const gsis_mesh *m) {
  s->n[0] = m->ni;
  s->n[1] = m->nj;
  s->n[2] = m->nk;
  s->nc = m->ni * m->nj * m->nk;
  const int N0 = m->ni + 1, N1 = m->nj + 1;
  for (int a = 0; a < 3; ++a) {
    s->X[a].resize(s->n[a] + 1);
    for (int I = 0; I <= s->n[a]; ++I) {
      const size_t idx = a == 0 ? (size_t)I : (a == 1 ? (size_t)N0 * I : (size_t)N0 * N1 * I);
      s->X[a][I] = m->nodes[3 * idx + a];
    }
    const int na = s->n[a];
    std::vector<double> xc(na), h(na);
    for (int i = 0; i < na; ++i) {
      xc[i] = 0.5 * (s->X[a][i] + s->X[a][i + 1]);
      h[i] = s->X[a][i + 1] - s->X[a][i];
    }
    s->axc[a].resize(na);
    for (int i = 0; i < na; ++i) {
      AxisCell<double> c{};
      c.h = h[i];
      c.invh = 1.0 / h[i];
      c.rlo = s->X[a][i] - xc[i];
      c.rhi = s->X[a][i + 1] - xc[i];
      // unweighted least squares over the axis neighbours inside the domain
      const double dlo = i > 0 ? xc[i - 1] - xc[i] : 0.0, dhi = i < na - 1 ? xc[i + 1] - xc[i] : 0.0;
      const double den = dlo * dlo + dhi * dhi;
      c.clo = den > 0 ? dlo / den : 0.0;
      c.chi = den > 0 ? dhi / den : 0.0;
      c.pad0 = i < na - 1 ? 1.0 / (xc[i + 1] - xc[i]) : 0.0;
      c.pad1 = 0.0;
      s->axc[a][i] = c;
    }
  }
  s->vol.resize(s->nc);
  s->vsum = 0.0;
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j)
      for (int i = 0; i < s->n[0]; ++i) {
        const double V = s->axc[0][i].h * s->axc[1][j].h * s->axc[2][k].h;
        s->vol[i + s->n[0] * (j + s->n[1] * k)] = V;
        s->vsum += V;
      }
  KinGeom &g = s->kg;
  g = KinGeom{};
  g.nc = s->nc;
  g.nact = 0;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = s->n[a];
    g.act[a] = s->n[a] > 1;
    g.nact += g.act[a];
  }
  g.ntrans[0] = g.act[0] ? s->n[1] * s->n[2] : 0;
  g.ntrans[1] = g.act[1] ? s->n[0] * s->n[2] : 0;
  g.ntrans[2] = g.act[2] ? s->n[0] * s->n[1] : 0;
  g.K3 = s->opt.venkat_K * s->opt.venkat_K * s->opt.venkat_K;
  // colour tables: hyperplanes i'+j'+k' of the transformed (upwind-first) coordinates
  g.ncol = s->n[0] + s->n[1] + s->n[2] - 2;
  s->col_off.assign(g.ncol + 1, 0);
  s->col_cell.resize(s->nc);
  s->pos_of.resize(s->nc);
  std::vector<std::vector<int>> lists(g.ncol);
  for (int k = 0; k < s->n[2]; ++k)
    for (int j = 0; j < s->n[1]; ++j)
      for (int i = 0; i < s->n[0]; ++i) lists[i + j + k].push_back(i | (j << 10) | (k << 20));
  g.maxcol = 0;
  for (int c = 0; c < g.ncol; ++c) {
    s->col_off[c + 1] = s->col_off[c] + (int)lists[c].size();
    g.maxcol = std::max(g.maxcol, (int)lists[c].size());
    for (size_t p = 0; p < lists[c].size(); ++p) {
      const int tp = lists[c][p];
      s->col_cell[s->col_off[c] + p] = tp;
      const int i = tp & 1023, j = (tp >> 10) & 1023, k = tp >> 20;
      s->pos_of[i + s->n[0] * (j + s->n[1] * k)] = (int)p;
    }
  }
  // per colour entry: neighbour positions in the adjacent colours and transformed transverse
  // indices (octant independent); per octant: the natural cell of every entry
  s->entries.assign(s->nc, EntryInfo{});
  s->natcell.assign((size_t)8 * s->nc, int4{0, 0, 0, 0});
  {
    const int n0 = s->n[0], n1 = s->n[1], n2 = s->n[2];
    for (int e = 0; e < s->nc; ++e) {
      const int tp = s->col_cell[e];
      const int tc[3] = {tp & 1023, (tp >> 10) & 1023, tp >> 20};
      const int t = tc[0] + n0 * (tc[1] + n1 * tc[2]);
      const int st[3] = {1, n0, n0 * n1};
      EntryInfo &E = s->entries[e];
      for (int a = 0; a < 3; ++a) {
        E.nb[2 * a] = tc[a] > 0 ? s->pos_of[t - st[a]] : -1;
        E.nb[2 * a + 1] = tc[a] < s->n[a] - 1 ? s->pos_of[t + st[a]] : -1;
      }
      E.trn[0] = tc[1] + n1 * tc[2];
      E.trn[1] = tc[0] + n0 * tc[2];
      E.trn[2] = tc[0] + n0 * tc[1];
      for (int oct = 0; oct < 8; ++oct) {
        const int nat[3] = {oct & 1 ? n0 - 1 - tc[0] : tc[0], oct & 2 ? n1 - 1 - tc[1] : tc[1], oct & 4 ? n2 - 1 - tc[2] : tc[2]};
        s->natcell[(size_t)oct * s->nc + e] = int4{nat[0] + n0 * (nat[1] + n1 * nat[2]), nat[0], nat[1], nat[2]};
      }
    }
  }
  // walls
  s->nwall = 0;
  s->wall_cell.clear();
  s->wall_side.clear();
  s->wall_sides_list.clear();
  s->closed = 1;
  for (int side = 0; side < 6; ++side) {
    const int a = side / 2;
    g.wall_base[side] = -1;
    for (int d = 0; d < 3; ++d) s->wall_uT[side][d] = m->wall_u[side][d];
    s->wall_uT[side][3] = m->wall_T[side];
    if (m->bc[side] != GSIS_BC_WALL) continue;
    g.wall_base[side] = s->nwall;
    s->wall_sides_list.push_back(side);
    const int fixed = (side & 1) ? s->n[a] - 1 : 0;
    const int ntr = a == 0 ? s->n[1] * s->n[2] : (a == 1 ? s->n[0] * s->n[2] : s->n[0] * s->n[1]);
    for (int t = 0; t < ntr; ++t) {
      int nat[3];
      if (a == 0) { nat[0] = fixed; nat[1] = t % s->n[1]; nat[2] = t / s->n[1]; }
      else if (a == 1) { nat[1] = fixed; nat[0] = t % s->n[0]; nat[2] = t / s->n[0]; }
      else { nat[2] = fixed; nat[0] = t % s->n[0]; nat[1] = t / s->n[0]; }
      s->wall_cell.push_back(nat[0] + s->n[0] * (nat[1] + s->n[1] * nat[2]));
      s->wall_side.push_back(side);
    }
    s->nwall += ntr;
  }
  s->general = needs_general(m);
  if (s->general) {
    for (int side = 0; side < 6; ++side) g.wall_base[side] = -1;
    const int rc = build_general(s, m);
    if (rc) return rc;
    octant_sweeps(s, m);
  }
  // red/black cell lists of the synthetic solve's sweeps
  s->colcells.clear();
  for (int col = 0; col < 2; ++col) {
    for (int c = 0; c < s->nc; ++c) {
      const int i = c % s->n[0], j = (c / s->n[0]) % s->n[1], k = c / (s->n[0] * s->n[1]);
      if (((i + j + k) & 1) == col) s->colcells.push_back(c);
    }
    if (col == 0) s->ncol0 = (int)s->colcells.size();
  }
  s->mcol_off = {0, s->ncol0, (int)s->nc};
  s->wall_patch = s->wall_side;
  return GSIS_OK;
}

static int setup_velocities(gsis_solver *s, const gsis_vgrid *vg) {
  s->point_set = vg->npoints > 0;
  for (int a = 0; a < 3; ++a) s->nv_axis[a] = s->point_set ? 0 : vg->n[a];
  s->nvc = s->point_set ? vg->npoints : vg->n[0] * vg->n[1] * vg->n[2];
  // only the FP64 Shakhov kinetic kernel uses tiles (factored Maxwellians); FP32 and BF16 keep
  // the x-fastest octant order
  if (s->prec == GSIS_F64 && s->nvdf == 1 && !s->point_set) choose_tile(vg, s->kg.tile);
  else s->kg.tile[0] = s->kg.tile[1] = s->kg.tile[2] = 0;
  build_slots(vg, s->kg.tile, s->slot_canon, s->boct, s->vel64);
  s->vaxis.clear();
  if (!s->point_set) {
    for (int a = 0; a < 3; ++a) s->vaxis.insert(s->vaxis.end(), vg->x[a], vg->x[a] + vg->n[a]);
    for (int a = 0; a < 3; ++a) s->vaxis.insert(s->vaxis.end(), vg->w[a], vg->w[a] + vg->n[a]);
  }
  s->vel64_all = s->vel64;
  s->nslots_all = (int)s->slot_canon.size();
  const int K = s->opt.shard_count > 1 ? s->opt.shard_count : 1;
  if (K > 1) {
    // this shard's contiguous range of velocity blocks
    const int nb = s->nslots_all / VB, k = s->opt.shard_index;
    if (K > nb) return s->fail(GSIS_E_INVALID, "%d shards for %d velocity blocks", K, nb);
    const int b0 = (int)((long long)k * nb / K), b1 = (int)((long long)(k + 1) * nb / K);
    s->slot_canon = std::vector<int>(s->slot_canon.begin() + (size_t)b0 * VB, s->slot_canon.begin() + (size_t)b1 * VB);
    s->boct = std::vector<int8_t>(s->boct.begin() + b0, s->boct.begin() + b1);
    s->vel64 = std::vector<double>(s->vel64.begin() + (size_t)b0 * VB * 4, s->vel64.begin() + (size_t)b1 * VB * 4);
  }
  s->nslots = (int)s->slot_canon.size();
  s->nblocks = s->nslots / VB;
  return GSIS_OK;
}

// Kinetic launch shape and ring placement.  One warp per cell of a colour, up to 16 warps (8 in
// FP64), within the register file.  The ring stays in shared memory unless the largest colour
// does not fit there, or the global-scratch kernel keeps at least twice as many blocks resident
// per SM (3D meshes: a colour ring of ~100 KB or more leaves room for one block per SM, and the
// scratch stays in L2).  Without a device (footprint queries on a host with no GPU) the
// placement follows the shared-memory limit of the sm_100 family, 227 KB.
template <typename T, typename S>
static int plan_kinetic(gsis_solver *s) {
  if (s->general) {
    // persistent grid of 8-warp CTAs over the velocity blocks, as many as the SMs hold (the
    // kernel is latency-bound) while their whole-mesh work arrays, one set per CTA for its
    // block of 32 velocities, stay within 144 GB (half of the GPU's memory: a 100,000-cell
    // mesh with two reduced VDFs takes 243 MB per CTA, four CTAs per SM)
    s->kin_smem = 0;
    s->kin_warps = 8;
    s->kin_gstride = kinetic_general_stride<T, S>(s->nc, s->nvdf, s->kg.nact);
    int dev = 0, sms = 152, occ = 2;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      const int rc = s->cuda(kinetic_general_shape<T, S>(s->nvdf, s->kg.nact, &occ), "kinetic shape");
      if (rc) return rc;
    } else {
      cudaGetLastError();
    }
    const size_t budget = (size_t)144 << 30;
    const int by_mem = (int)std::max<size_t>(1, budget / ((size_t)sms * s->kin_gstride));
    s->kin_grid = std::max(1, std::min(s->nblocks, std::max(1, std::min(occ, by_mem)) * sms));
    s->kin_scratch_bytes = (size_t)s->kin_grid * s->kin_gstride;
    return GSIS_OK;
  }
  const size_t smem = kinetic_smem_bytes<T, S>(s->kg, s->nvdf);
  const size_t gstride = kinetic_gscratch_stride<T, S>(s->kg, s->nvdf);
  int want = std::max(1, std::min(16, s->kg.maxcol / 4));
  if (sizeof(T) == 8) want = std::min(want, 8);
  int dev = 0, optin = 0;
  const bool have_dev = cudaGetDevice(&dev) == cudaSuccess &&
                        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess;
  if (!have_dev) {
    cudaGetLastError();
    optin = 227 * 1024;
  }
  bool gm = s->opt.kinetic_ring == 1 || smem > (size_t)optin;
  int warps_sh = want, warps_gm = want;
  if (have_dev) {
    int occ_sh = 0, occ_gm = 0;
    int rc = s->cuda(kinetic_shape<T, S>(s->kg, s->nvdf, true, want, 0, &warps_gm, &occ_gm), "kinetic shape");
    if (!rc && !gm) rc = s->cuda(kinetic_shape<T, S>(s->kg, s->nvdf, false, want, smem, &warps_sh, &occ_sh), "kinetic shape");
    if (rc) return rc;
    if (!gm && occ_gm >= 2 * occ_sh) gm = true;
  }
  s->kin_smem = gm ? 0 : smem;
  s->kin_gstride = gm ? gstride : 0;
  s->kin_warps = gm ? warps_gm : warps_sh;
  s->kin_scratch_bytes = (size_t)s->nblocks * s->kin_gstride;
  return GSIS_OK;
}

static size_t footprint(const gsis_solver *s) {
  const size_t T = s->prec == GSIS_F64 ? 8 : 4;                             // kinetic arithmetic
  const size_t Sb = s->prec == GSIS_F64 ? 8 : (s->prec == GSIS_BF16 ? 2 : 4);  // VDF storage
  const size_t nc = s->nc;
  size_t b = 0;
  b += (size_t)s->nvdf * s->nslots * nc * Sb;  // f (f0, f1)
  b += (size_t)s->nblocks * (s->nwall + 1) * NWF * T;  // wall partials
  b += s->kin_scratch_bytes;                          // kinetic ring or work arrays in global memory
  if (s->general) b += nc * (sizeof(GenCell<double>) + 6 * (2 * sizeof(int) + 1)) + (size_t)s->nwall * 8;
  if (s->unstructured) b += 14 * nc + (nc + 1) * 4 + s->gs_idx.size() * (4 + 3 * (T + 8));
  if (s->general && (s->opt.mode == GSIS_MODE_GSIS || s->opt.euler_presteps > 0))
    b += nc * (sizeof(GenCell<double>) + (3 + 6 * (size_t)s->kin_grid + 6 + 6 + 1 + 18 + 6 + 15 + 6 + 6 + 6 + 36 + 36 + 6 + 36) * 8) +
         12 * 8 * (size_t)macro_general_parts((int)nc);
  b += (size_t)nc * moment_len(s->nvdf) * 8 * 16;  // moment chunks (bounded)
  if (Sb == 8 && s->nvdf == 1 && !s->point_set)     // FP64 origin moments: the extra chunk, the table
    b += (size_t)nc * moment_len(1) * 8 + (size_t)s->nslots * 16 * 8 + s->vaxis.size() * 8;
  b += nc * NST * (T + 8);                    // states
  b += nc * (13 + 18 + 18 + 12 + 6 + 6 + 1) * 8;
  b += nc * (6 + 6 + 18 + 6 + 15 + 1 + 6 + 6 + 6 + 36 + 6 + 3 + 18 + 8 + 36) * 8;  // synthetic-solve work
  b += (size_t)s->nslots * 4 * (T + 8) + (size_t)s->nwall * 32 * 8 + 3 * nc * 4 + (1 << 20);
  return b;
}

template <typename T, typename S>
static int allocate_and_upload(gsis_solver *s) {
  const size_t nc = s->nc;
  int rc = 0;
#define A(ptr, bytes) \
  if (!rc) rc = s->alloc(&(ptr), (bytes))
  A(s->d_f, (size_t)s->nvdf * s->nslots * nc * sizeof(S));
  // moment chunks: enough (cell, chunk) threads to fill the GPU, at most 64 blocks per chunk
  {
    const int want = std::max(1, (int)((160000 + nc - 1) / nc));
    s->mom_bpc = std::max(1, std::min(64, (s->nblocks + want - 1) / want));
    s->mom_nchunks = (s->nblocks + s->mom_bpc - 1) / s->mom_bpc;
  }
  s->origin_mom = std::is_same<T, double>::value && s->nvdf == 1 && !s->point_set;
  A(s->d_mp, (size_t)(s->mom_nchunks + (s->origin_mom ? 1 : 0)) * nc * moment_len(s->nvdf) * sizeof(double));
  if (s->origin_mom) {
    A(s->d_mtab, (size_t)s->nslots * 16 * sizeof(double));
    A(s->d_vaxis, s->vaxis.size() * sizeof(double));
  }
  A(s->d_wpart, (size_t)s->nblocks * (s->nwall + 1) * NWF * sizeof(T));
  if (s->kin_scratch_bytes) A(s->d_kscratch, s->kin_scratch_bytes);
  if (s->general) {
    A(s->d_gen, nc * sizeof(GenCell<T>));
    A(s->d_gnb, 6 * nc * sizeof(int));
    A(s->d_gwid, 6 * nc * sizeof(int));
    A(s->d_gin, 6 * nc);
    A(s->d_wall_area, (size_t)(s->nwall + 1) * sizeof(double));
    A(s->d_wden, (size_t)(s->nwall + 1) * sizeof(double));
    if (s->opt.mode == GSIS_MODE_GSIS || s->opt.euler_presteps > 0) {
      A(s->d_gen64, nc * sizeof(GenCell<double>));
      A(s->d_xc, 3 * nc * sizeof(double));
      A(s->d_kpart, (size_t)s->kin_grid * nc * 6 * sizeof(double));
      A(s->g_W, 6 * nc * sizeof(double));
      A(s->g_pr, 6 * nc * sizeof(double));
      A(s->g_mu, nc * sizeof(double));
      A(s->g_gW, 18 * nc * sizeof(double));
      A(s->g_phW, 6 * nc * sizeof(double));
      A(s->g_gP, 15 * nc * sizeof(double));
      A(s->g_R, 6 * nc * sizeof(double));
      A(s->g_D, 6 * nc * sizeof(double));
      A(s->g_dW, 6 * nc * sizeof(double));
      A(s->g_F0, 36 * nc * sizeof(double));
      A(s->g_Ff, 36 * nc * sizeof(double));
      A(s->g_gam, 6 * nc * sizeof(double));
      A(s->g_FW0, 18 * nc * sizeof(double));
      A(s->g_FW, 18 * nc * sizeof(double));
      A(s->g_part, 12 * (size_t)macro_general_parts((int)nc) * sizeof(double));
      A(s->g_flag, 2 * sizeof(int));
    }
  }
  A(s->d_K, nc * 6 * sizeof(double));
  A(s->d_stT, nc * NST * sizeof(T));
  A(s->d_st64, nc * NST * sizeof(double));
  A(s->d_vel, (size_t)s->nslots * 4 * sizeof(T));
  A(s->d_vel64, (size_t)s->nslots_all * 4 * sizeof(double));
  for (int a = 0; a < 3; ++a) {
    A(s->d_ax[a], s->axc[a].size() * sizeof(AxisCell<T>));
    A(s->d_ax64[a], s->axc[a].size() * sizeof(AxisCell<double>));
  }
  A(s->d_boct, s->boct.size());
  A(s->d_col_off, s->col_off.size() * sizeof(int));
  A(s->d_entry, nc * sizeof(EntryInfo));
  A(s->d_natcell, 8 * nc * sizeof(int4));
  A(s->d_rho_w, (size_t)(s->nwall + 1) * sizeof(double));
  A(s->d_Z0, 6 * sizeof(double));
  A(s->d_Zw, 36 * sizeof(double));
  A(s->d_wall_uT, 24 * sizeof(double));
  A(s->d_wall_cell, (size_t)(s->nwall + 1) * sizeof(int));
  A(s->d_wall_side, (size_t)(s->nwall + 1) * sizeof(int));
  A(s->d_wall_patch, (size_t)(s->nwall + 1) * sizeof(int));
  if (s->unstructured) {
    A(s->d_gnf, 6 * nc);
    A(s->d_gpat, 6 * nc);
    A(s->d_gso, (nc + 1) * sizeof(int));
    A(s->d_gsi, (s->gs_idx.size() + 1) * sizeof(int));
    A(s->d_gsw, (s->gs_idx.size() + 1) * 3 * sizeof(T));
    A(s->d_gsw64, (s->gs_idx.size() + 1) * 3 * sizeof(double));
  }
  A(s->d_wall_sides, 6 * sizeof(int));
  A(s->d_mom, nc * MOM_STRIDE * sizeof(double));
  A(s->d_wf, (size_t)(s->nwall + 1) * 6 * sizeof(double));
  A(s->d_Mh, nc * 18 * sizeof(double));
  A(s->d_hot, nc * 12 * sizeof(double));
  A(s->d_Wstate, nc * 6 * sizeof(double));
  A(s->d_Wnew, nc * 6 * sizeof(double));
  A(s->d_vol, nc * sizeof(double));
  A(s->d_mass, 2 * sizeof(double));
  A(s->d_scratch, 8192 * sizeof(double));
  A(s->d_eps4, 4 * sizeof(double));
  A(s->d_ticket, 4 * sizeof(unsigned));
  A(s->d_bar, MACRO_BAR_WORDS * sizeof(unsigned));
  A(s->d_err, sizeof(int));
  if (!rc && cudaHostAlloc((void **)&s->pin, sizeof(gsis_solver::Readback), cudaHostAllocDefault) != cudaSuccess)
    rc = s->fail(GSIS_E_OOM, "pinned host read-back words");
  A(s->d_iters, sizeof(int));
  A(s->m_W, nc * 6 * sizeof(double));
  A(s->m_pr, nc * 6 * sizeof(double));
  A(s->m_gW, nc * 18 * sizeof(double));
  A(s->m_phW, nc * 6 * sizeof(double));
  A(s->m_gP, nc * 15 * sizeof(double));
  A(s->m_aux, nc * 8 * sizeof(double));
  A(s->d_colcells, nc * sizeof(int));
  A(s->m_R, nc * 6 * sizeof(double));
  A(s->m_invD, nc * 6 * sizeof(double));
  A(s->m_dW, nc * 6 * sizeof(double));
  A(s->m_Fc, nc * 36 * sizeof(double));  // two buffers: start and end of an inner step
  A(s->m_corr, nc * 6 * sizeof(double));
  A(s->m_gam, nc * 3 * sizeof(double));
  A(s->m_Ffc, nc * 18 * sizeof(double));
  A(s->m_G, nc * 36 * sizeof(double));
  A(s->m_wfl, (size_t)(s->nwall + 1) * 6 * sizeof(double));
#undef A
  if (rc) return rc;
  rc = s->cuda(macro_launch_shape((int)nc, s->opt.macro_sms, &s->macro_grid, &s->macro_block), "occupancy");
  if (rc) return rc;
  rc = s->alloc(&s->m_red, ((size_t)3 * s->macro_grid * 16 + 32) * sizeof(double));
  if (rc) return rc;
  std::vector<T> velT(s->vel64.begin(), s->vel64.end());
  rc = s->upload(s->d_vel, velT.data(), velT.size() * sizeof(T));
  std::vector<double> mtab;
  if (s->origin_mom) {
    // per slot: w (1, x, y, z, xx, yy, zz, xy, xz, yz, |xi|^2 x, |xi|^2 y, |xi|^2 z), padded to 16
    mtab.assign((size_t)s->nslots * 16, 0.0);
    for (int v = 0; v < s->nslots; ++v) {
      const double x = s->vel64[4 * v], y = s->vel64[4 * v + 1], z = s->vel64[4 * v + 2], w = s->vel64[4 * v + 3];
      const double q2 = x * x + y * y + z * z;
      const double t[NMOM] = {w, w * x, w * y, w * z, w * x * x, w * y * y, w * z * z, w * x * y, w * x * z, w * y * z,
                              w * q2 * x, w * q2 * y, w * q2 * z};
      for (int k = 0; k < NMOM; ++k) mtab[(size_t)v * 16 + k] = t[k];
    }
    if (!rc) rc = s->upload(s->d_mtab, mtab.data(), mtab.size() * sizeof(double));
    if (!rc) rc = s->upload(s->d_vaxis, s->vaxis.data(), s->vaxis.size() * sizeof(double));
    if (!rc) rc = s->cuda(cudaStreamSynchronize(s->stream), "sync");  // mtab leaves scope
  }
  if (!rc) rc = s->upload(s->d_vel64, s->vel64_all.data(), s->vel64_all.size() * sizeof(double));
  for (int a = 0; a < 3 && !rc; ++a) {
    auto cv = cast_axis<T>(s->axc[a]);
    rc = s->upload(s->d_ax[a], cv.data(), cv.size() * sizeof(AxisCell<T>));
    if (!rc) rc = s->upload(s->d_ax64[a], s->axc[a].data(), s->axc[a].size() * sizeof(AxisCell<double>));
  }
  if (!rc) rc = s->upload(s->d_boct, s->boct.data(), s->boct.size());
  if (!rc) rc = s->upload(s->d_col_off, s->col_off.data(), s->col_off.size() * sizeof(int));
  if (!rc) rc = s->upload(s->d_entry, s->entries.data(), nc * sizeof(EntryInfo));
  if (!rc) rc = s->upload(s->d_natcell, s->natcell.data(), 8 * nc * sizeof(int4));
  if (!rc && s->nwall) rc = s->upload(s->d_wall_cell, s->wall_cell.data(), s->nwall * sizeof(int));
  if (!rc && s->nwall) rc = s->upload(s->d_wall_side, s->wall_side.data(), s->nwall * sizeof(int));
  if (!rc && s->nwall) rc = s->upload(s->d_wall_patch, s->wall_patch.data(), s->nwall * sizeof(int));
  if (!rc && s->unstructured) rc = s->upload(s->d_gnf, s->gnf.data(), 6 * nc);
  if (!rc && s->unstructured) rc = s->upload(s->d_gpat, s->gpat.data(), 6 * nc);
  std::vector<T> gswT(s->gs_w.begin(), s->gs_w.end());
  if (!rc && s->unstructured) rc = s->upload(s->d_gso, s->gs_off.data(), (nc + 1) * sizeof(int));
  if (!rc && s->unstructured && !s->gs_idx.empty()) {
    rc = s->upload(s->d_gsi, s->gs_idx.data(), s->gs_idx.size() * sizeof(int));
    if (!rc) rc = s->upload(s->d_gsw, gswT.data(), gswT.size() * sizeof(T));
    if (!rc) rc = s->upload(s->d_gsw64, s->gs_w.data(), s->gs_w.size() * sizeof(double));
    if (!rc) rc = s->cuda(cudaStreamSynchronize(s->stream), "sync");  // gswT leaves scope
  }
  if (!rc && !s->wall_sides_list.empty())
    rc = s->upload(s->d_wall_sides, s->wall_sides_list.data(), s->wall_sides_list.size() * sizeof(int));
  if (!rc) rc = s->upload(s->d_wall_uT, &s->wall_uT[0][0], 24 * sizeof(double));
  if (!rc) rc = s->upload(s->d_vol, s->vol.data(), nc * sizeof(double));
  if (!rc) rc = s->upload(s->d_colcells, s->colcells.data(), nc * sizeof(int));
  if (!rc && s->general) {
    const std::vector<GenCell<T>> gT = cast_gen<T>(s->gen64);
    rc = s->upload(s->d_gen, gT.data(), nc * sizeof(GenCell<T>));
    if (!rc) rc = s->upload(s->d_gnb, s->gnb.data(), 6 * nc * sizeof(int));
    if (!rc) rc = s->upload(s->d_gwid, s->gwid.data(), 6 * nc * sizeof(int));
    if (!rc) rc = s->upload(s->d_gin, s->gin.data(), 6 * nc);
    if (!rc && s->nwall) rc = s->upload(s->d_wall_area, s->wall_area.data(), s->nwall * sizeof(double));
    if (!rc && s->nwall)
      rc = s->cuda(launch_wall_den_general<T, S>(s->kin_args<T, S>(), s->d_vel64, s->nslots_all, s->d_wall_cell,
                                                 s->d_wall_side, s->nwall, s->d_wden, s->stream),
                   "wall denominators");
    if (!rc && s->d_gen64) rc = s->upload(s->d_gen64, s->gen64.data(), nc * sizeof(GenCell<double>));
    if (!rc && s->d_xc) rc = s->upload(s->d_xc, s->xc64.data(), 3 * nc * sizeof(double));
  }
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_ticket, 0, 4 * sizeof(unsigned), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_rho_w, 0, (s->nwall + 1) * sizeof(double), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_K, 0, nc * 6 * sizeof(double), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_wf, 0, (s->nwall + 1) * 6 * sizeof(double), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_hot, 0, nc * 12 * sizeof(double), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_Z0, 0, 6 * sizeof(double), s->stream), "memset");
  if (!rc) rc = s->cuda(cudaMemsetAsync(s->d_Zw, 0, 36 * sizeof(double), s->stream), "memset");
  if (!rc)
    rc = s->cuda(launch_wall_constants(s->d_vel64, s->nslots_all, s->d_wall_uT, s->d_wall_sides,
                                       (int)s->wall_sides_list.size(), s->d_Z0, s->d_Zw,
                                       s->nvdf == 2 ? s->gas.d_r : 0.0, s->stream),
                 "wall constants");
  if (rc) return rc;
  return GSIS_OK;
}

extern "C" int gsis_footprint_bytes(const gsis_mesh *mesh, const gsis_vgrid *vgrid, const gsis_gas *gas,
                                    const gsis_options *opt, size_t *bytes) {
  std::string why;
  gsis_options o;
  if (opt) o = *opt;
  else gsis_default_options(&o);
  int rc = validate(mesh, vgrid, gas, 1.0, &o, why);
  if (rc) return rc;
  gsis_solver tmp;
  tmp.opt = o;
  tmp.prec = o.precision;
  tmp.nvdf = gas->model == GSIS_RYKOV ? 2 : 1;
  rc = setup(&tmp, mesh, vgrid);
  if (!rc) rc = GSIS_DISPATCH(tmp.prec, (plan_kinetic<T, S>(&tmp)));
  if (rc) return rc;
  *bytes = footprint(&tmp);
  return GSIS_OK;
}

static int init_state_from(gsis_solver *s, std::vector<double> &W0);

static int init_state(gsis_solver *s) {
  const size_t nc = s->nc;
  std::vector<double> W0(nc * 6);
  for (size_t c = 0; c < nc; ++c) {
    if (s->opt.init_W) {
      for (int k = 0; k < 6; ++k) W0[c * 6 + k] = s->opt.init_W[c * 6 + k];
    } else {
      W0[c * 6 + 0] = 1.0;
      W0[c * 6 + 1] = W0[c * 6 + 2] = W0[c * 6 + 3] = 0.0;
      W0[c * 6 + 4] = W0[c * 6 + 5] = 1.0;
    }
    if (!(W0[c * 6] > 0) || !(W0[c * 6 + 4] > 0)) return s->fail(GSIS_E_INVALID, "initial state must have rho, T > 0");
  }
  return init_state_from(s, W0);
}

// Euler preconditioning on general meshes: the inviscid synthetic solve from the current state
// W^n for euler_presteps inner steps, then f restarts as the Maxwellian of its result
static int euler_presteps(gsis_solver *s) {
  MacroGenArgs m = s->macro_general_args();
  m.euler = 1;
  m.wall_g13 = 0;
  m.relax = 1.0;
  m.visc_jump = 0.0;
  m.steps = s->opt.euler_presteps;
  m.Mh = s->d_Wstate;
  m.mh_stride = 6;
  m.K = nullptr;
  int rc = s->cuda(run_macro_general(m, s->stream), "Euler presteps");
  std::vector<double> W((size_t)s->nc * 6);
  if (!rc) rc = s->cuda(cudaMemcpyAsync(W.data(), s->d_Wnew, W.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream), "W");
  if (!rc) rc = s->cuda(cudaStreamSynchronize(s->stream), "sync");
  if (!rc) rc = s->check_err();
  if (rc) return rc;
  return init_state_from(s, W);
}

static int init_state_from(gsis_solver *s, std::vector<double> &W0) {
  const size_t nc = s->nc;
  double *dW0 = nullptr;
  int rc = s->cuda(cudaMalloc(&dW0, nc * 6 * sizeof(double)), "temporary");
  if (rc) return rc;
  rc = s->upload(dW0, W0.data(), nc * 6 * sizeof(double));
  if (!rc)
    rc = GSIS_DISPATCH(s->prec, (s->cuda(launch_init_maxwellian<T, S>(s->kin_args<T, S>(), dW0, s->nblocks, s->stream),
                                         "init f")));
  if (!rc) rc = s->cuda(cudaStreamSynchronize(s->stream), "sync");
  cudaFree(dW0);
  if (rc) return rc;
  return GSIS_DISPATCH(s->prec, (s->state_from_f<T, S>(W0.data())));
}

// Mach number the mesh's boundary data describe: the free stream's (far-field sides) or, without
// a far field, the fastest wall's, each over the speed of sound at its own temperature,
// c^2 = gamma R T with R T = T / 2 and gamma = (5 + d_r) / (3 + d_r) (Section 2.1: internal
// energy d_r R T_r / 2 beside the translational 3 R T_t / 2).
static double mesh_mach(const gsis_mesh *m, const gsis_gas *g) {
  const double dr = g->model == GSIS_RYKOV ? g->d_r : 0.0;
  const double gam = (5.0 + dr) / (3.0 + dr);
  // the sides of a block, or the patches an unstructured mesh uses
  bool used[6] = {true, true, true, true, true, true};
  if (m->ncells > 0) {
    for (int s = 0; s < 6; ++s) used[s] = false;
    for (size_t t = 0; t < (size_t)6 * m->ncells; ++t)
      if (m->face_patch[t] >= 0) used[m->face_patch[t]] = true;
  }
  bool far = false;
  for (int s = 0; s < 6; ++s) far = far || (used[s] && m->bc[s] == GSIS_BC_FARFIELD);
  double ma = 0.0;
  for (int s = 0; s < 6; ++s) {
    if (!used[s] || m->bc[s] != (far ? GSIS_BC_FARFIELD : GSIS_BC_WALL)) continue;
    const double *u = m->wall_u[s];
    ma = std::max(ma, std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / std::sqrt(0.5 * gam * m->wall_T[s]));
  }
  return ma;
}

extern "C" int gsis_create(const gsis_mesh *mesh, const gsis_vgrid *vgrid, const gsis_gas *gas, double Kn, double Ma,
                           const gsis_options *opt, gsis_handle *out) {
  if (out) *out = nullptr;
  if (!out) { g_create_error = "out is NULL"; return GSIS_E_INVALID; }
  gsis_options o;
  if (opt) o = *opt;
  else gsis_default_options(&o);
  std::string why;
  int rc = validate(mesh, vgrid, gas, Kn, &o, why);
  if (rc) { g_create_error = why; return rc; }
  {
    const double ma_mesh = mesh_mach(mesh, gas);
    if (!std::isfinite(Ma) || !(Ma >= 0.0) || std::fabs(Ma - ma_mesh) > 1e-9 * std::max(1.0, ma_mesh)) {
      char buf[200];
      std::snprintf(buf, sizeof buf, "Ma = %.9g disagrees with the %s speed of the mesh (Ma = %.9g)", Ma,
                    ma_mesh > 0 || Ma > 0 ? "free-stream or wall" : "zero", ma_mesh);
      g_create_error = buf;
      return GSIS_E_INVALID;
    }
  }
  gsis_solver *s = new (std::nothrow) gsis_solver();
  if (!s) { g_create_error = "out of host memory"; return GSIS_E_OOM; }
  s->opt = o;
  s->prec = o.precision;
  s->nvdf = gas->model == GSIS_RYKOV ? 2 : 1;
  s->Kn = Kn;
  s->omega = gas->omega;
  s->gas = *gas;
  s->stream = (cudaStream_t)o.stream;
  rc = setup(s, mesh, vgrid);
  if (!rc) rc = GSIS_DISPATCH(s->prec, (plan_kinetic<T, S>(s)));
  if (!rc) rc = GSIS_DISPATCH(s->prec, (allocate_and_upload<T, S>(s)));
  if (!rc) rc = init_state(s);
  if (!rc && o.euler_presteps > 0) rc = euler_presteps(s);
  for (int t = 0; !rc && t < o.kinetic_presteps; ++t) rc = s->step(GSIS_MODE_DVM);
  if (rc) {
    g_create_error = s->last_error;
    s->release();
    delete s;
    return rc;
  }
  s->outer_total = 0;
  *out = s;
  return GSIS_OK;
}

#define GSIS_NOT_PENDING(h) \
  if ((h)->pending) return (h)->fail(GSIS_E_INVALID, "a step is pending: call gsis_step_wait first")

extern "C" int gsis_step_async(gsis_handle h) {
  if (!h) return GSIS_E_INVALID;
  return h->enqueue_step(h->opt.mode);
}

extern "C" int gsis_step_wait(gsis_handle h, double *eps_last) {
  if (!h) return GSIS_E_INVALID;
  const int rc = h->finish_step();
  if (!rc && eps_last) *eps_last = h->eps4[3];
  return rc;
}

extern "C" int gsis_iterate(gsis_handle h, int max_outer, double tol, int *outer_done, double *eps_last) {
  if (!h) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  if (outer_done) *outer_done = 0;
  for (int t = 0; t < max_outer; ++t) {
    int rc = h->step(h->opt.mode);
    if (rc) return rc;
    if (outer_done) *outer_done = t + 1;
    if (eps_last) *eps_last = h->eps4[3];
    if (h->eps4[3] < tol) return GSIS_OK;
  }
  return max_outer > 0 ? GSIS_E_NOT_CONVERGED : GSIS_OK;
}

extern "C" int gsis_moments(gsis_handle h, unsigned mask, double *host_out, size_t out_len) {
  if (!h || !host_out) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  const size_t nc = h->nc;
  size_t per = 0;
  if (mask & GSIS_F_W) per += 6;
  if (mask & GSIS_F_HALF) per += 18;
  if (mask & GSIS_F_HOT) per += 12;
  if (per == 0 || out_len < per * nc) return h->fail(GSIS_E_INVALID, "out_len too small");
  std::vector<double> W(nc * 6), M(nc * 18), H(nc * 12);
  int rc = 0;
  if (mask & GSIS_F_HOT) {
    CellFieldArgs c{};
    c.g = h->kg;
    for (int d = 0; d < 3; ++d) c.ax[d] = h->d_ax64[d];
    c.Kn = h->Kn;
    c.omega = h->omega;
    c.model = h->gas.model;
    c.d_r = h->gas.d_r;
    c.Z_r = h->gas.Z_r;
    for (int k = 0; k < 4; ++k) c.A[k] = h->gas.A[k];
    rc = h->cuda(launch_hot(c, h->d_Mh, h->d_hot, h->stream), "hot");
  }
  if (!rc) rc = h->cuda(cudaMemcpyAsync(W.data(), h->d_Wstate, nc * 6 * 8, cudaMemcpyDeviceToHost, h->stream), "W");
  if (!rc) rc = h->cuda(cudaMemcpyAsync(M.data(), h->d_Mh, nc * 18 * 8, cudaMemcpyDeviceToHost, h->stream), "Mh");
  if (!rc) rc = h->cuda(cudaMemcpyAsync(H.data(), h->d_hot, nc * 12 * 8, cudaMemcpyDeviceToHost, h->stream), "hot");
  if (!rc) rc = h->cuda(cudaStreamSynchronize(h->stream), "sync");
  if (rc) return rc;
  for (size_t c = 0; c < nc; ++c) {
    double *o = host_out + c * per;
    if (mask & GSIS_F_W) { std::memcpy(o, &W[c * 6], 6 * 8); o += 6; }
    if (mask & GSIS_F_HALF) { std::memcpy(o, &M[c * 18], 18 * 8); o += 18; }
    if (mask & GSIS_F_HOT) { std::memcpy(o, &H[c * 12], 12 * 8); o += 12; }
  }
  return GSIS_OK;
}

extern "C" int gsis_residual(gsis_handle h, double *eps, int n) {
  if (!h || !eps || n < 4) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  for (int k = 0; k < 4; ++k) eps[k] = h->eps4[k];
  return GSIS_OK;
}

extern "C" int gsis_nwall(gsis_handle h) { return h ? h->nwall : 0; }

static double face_area(const gsis_solver *s, int cell, int a) {
  const int nat[3] = {cell % s->n[0], (cell / s->n[0]) % s->n[1], cell / (s->n[0] * s->n[1])};
  return s->vol[cell] / s->axc[a][nat[a]].h;
}

extern "C" int gsis_wall(gsis_handle h, int *cell, int *side, double *rho_w, double *flux6) {
  if (!h) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  const int nw = h->nwall;
  std::vector<double> rw(nw + 1), wf((size_t)(nw + 1) * 6);
  int rc = h->cuda(cudaMemcpyAsync(rw.data(), h->d_rho_w, (nw + 1) * 8, cudaMemcpyDeviceToHost, h->stream), "rho_w");
  if (!rc) rc = h->cuda(cudaMemcpyAsync(wf.data(), h->d_wf, (nw + 1) * 48, cudaMemcpyDeviceToHost, h->stream), "wf");
  if (!rc) rc = h->cuda(cudaStreamSynchronize(h->stream), "sync");
  if (rc) return rc;
  for (int w = 0; w < nw; ++w) {
    if (cell) cell[w] = h->wall_cell[w];
    if (side) side[w] = h->wall_side[w];
    if (rho_w) rho_w[w] = rw[w];
    if (flux6) {
      const double A = h->general ? h->wall_area[w] : face_area(h, h->wall_cell[w], h->wall_side[w] / 2);
      for (int k = 0; k < 6; ++k) flux6[6 * w + k] = wf[6 * w + k] * A;
    }
  }
  return GSIS_OK;
}

extern "C" int gsis_wall_loads(gsis_handle h, unsigned side_mask, const double *dir, double rho_ref, double U_ref,
                               double A_ref, double *out6) {
  if (!h || !dir || !out6) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  if (!(rho_ref > 0.0) || !(U_ref > 0.0) || !(A_ref > 0.0) || (side_mask & ~63u) != 0)
    return h->fail(GSIS_E_INVALID, "wall loads need rho_ref, U_ref, A_ref > 0 and a 6-bit side mask");
  WallLoadArgs a{};
  a.wf = h->d_wf;
  a.wall_cell = h->d_wall_cell;
  a.wall_side = h->d_wall_patch;  // the mask selects sides (patches of an unstructured mesh)
  a.nwall = h->nwall;
  a.area = h->general ? h->d_wall_area : nullptr;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = h->n[d];
    a.ax[d] = h->d_ax64[d];
    a.dir[d] = dir[d];
  }
  a.mask = side_mask;
  a.rho_ref = rho_ref;
  a.U_ref = U_ref;
  a.A_ref = A_ref;
  a.out = h->d_scratch;
  int rc = h->cuda(launch_wall_loads(a, h->stream), "wall loads");
  if (!rc) rc = h->cuda(cudaMemcpyAsync(out6, h->d_scratch, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "out");
  if (!rc) rc = h->cuda(cudaStreamSynchronize(h->stream), "sync");
  return rc;
}

extern "C" int gsis_kinetic_flux_sum(gsis_handle h, double *out, size_t out_len) {
  if (!h || !out) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  const size_t nc = h->nc;
  if (out_len < nc * 6) return h->fail(GSIS_E_INVALID, "out_len too small");
  int rc = h->cuda(cudaMemcpyAsync(out, h->d_K, nc * 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "K");
  if (!rc) rc = h->cuda(cudaStreamSynchronize(h->stream), "sync");
  return rc;
}

extern "C" int gsis_get_f(gsis_handle h, double *f0, double *f1) {
  if (!h || !f0) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  const size_t bytes = (size_t)h->nc * h->nvc * sizeof(double);
  double *tmp = nullptr;
  int *canon = nullptr;
  int rc = h->cuda(cudaMalloc(&tmp, bytes), "temporary");
  if (!rc) rc = h->cuda(cudaMalloc(&canon, h->nslots * sizeof(int)), "temporary");
  if (!rc) rc = h->upload(canon, h->slot_canon.data(), h->nslots * sizeof(int));
  double *outs[2] = {f0, h->nvdf == 2 ? f1 : nullptr};
  for (int q = 0; q < 2 && !rc; ++q) {
    if (!outs[q]) continue;
    rc = GSIS_DISPATCH(h->prec, (h->cuda(launch_export_f<T, S>(h->kin_args<T, S>(), q, canon, h->nslots, h->nvc, tmp,
                                                                 h->stream),
                                         "export")));
    if (!rc) rc = h->cuda(cudaMemcpyAsync(outs[q], tmp, bytes, cudaMemcpyDeviceToHost, h->stream), "copy f");
    if (!rc) rc = h->cuda(cudaStreamSynchronize(h->stream), "sync");
  }
  cudaFree(tmp);
  cudaFree(canon);
  return rc;
}

extern "C" int gsis_set_f(gsis_handle h, const double *f0, const double *f1) {
  if (!h || !f0) return GSIS_E_INVALID;
  GSIS_NOT_PENDING(h);
  const size_t bytes = (size_t)h->nc * h->nvc * sizeof(double);
  double *tmp = nullptr;
  int *canon = nullptr;
  int rc = h->cuda(cudaMalloc(&tmp, bytes), "temporary");
  if (!rc) rc = h->cuda(cudaMalloc(&canon, h->nslots * sizeof(int)), "temporary");
  if (!rc) rc = h->upload(canon, h->slot_canon.data(), h->nslots * sizeof(int));
  const double *ins[2] = {f0, f1};
  for (int q = 0; q < h->nvdf && !rc; ++q) {
    if (ins[q]) rc = h->upload(tmp, ins[q], bytes);
    else rc = h->cuda(cudaMemsetAsync(tmp, 0, bytes, h->stream), "memset");  // f1 = 0 when not given
    if (!rc)
      rc = GSIS_DISPATCH(h->prec, (h->cuda(launch_import_f<T, S>(h->kin_args<T, S>(), q, canon, h->nslots, h->nvc,
                                                                   tmp, h->stream),
                                           "import")));
    if (!rc) rc = h->cuda(cudaStreamSynchronize(h->stream), "sync");
  }
  cudaFree(tmp);
  cudaFree(canon);
  if (rc) return rc;
  h->drop_graphs();  // the step's arguments include the new f's mass reference
  return GSIS_DISPATCH(h->prec, (h->state_from_f<T, S>()));
}

extern "C" int gsis_profile(gsis_handle h, int enable, int reset, double *ms, int n, int *steps, int *launches) {
  if (!h) return GSIS_E_INVALID;
  if (!h->ev[0])
    for (auto &e : h->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return h->fail(GSIS_E_CUDA, "cudaEventCreate");
  if (reset) {
    for (double &t : h->phase_ms) t = 0.0;
    h->prof_steps = h->prof_launches = 0;
  }
  if (ms)
    for (int k = 0; k < n && k < 5; ++k) ms[k] = h->phase_ms[k];
  if (steps) *steps = h->prof_steps;
  if (launches) *launches = h->prof_launches;
  h->profiling = enable != 0;
  return GSIS_OK;
}

extern "C" int gsis_stats(gsis_handle h, int *outer_total, int *macro_iters_last) {
  if (!h) return GSIS_E_INVALID;
  if (outer_total) *outer_total = h->outer_total;
  if (macro_iters_last) *macro_iters_last = h->macro_iters_last;
  return GSIS_OK;
}

extern "C" int gsis_graphs(gsis_handle h) {
  if (!h) return 0;
  return h->graphs_off ? -1 : (int)h->graphs.size();
}

extern "C" int gsis_destroy(gsis_handle h) {
  if (!h) return GSIS_OK;
  h->release();
  delete h;
  return GSIS_OK;
}

void gsis::set_handle_free_error(const char *msg) { g_create_error = msg; }

extern "C" const char *gsis_last_error(gsis_handle h) {
  if (!h) return g_create_error.c_str();
  return h->last_error.c_str();
}

extern "C" int gsis_selftest_wait_timeout(int which, int *device_status) {
  if ((which != 0 && which != 1) || !device_status) return GSIS_E_INVALID;
  unsigned *bar = nullptr;
  int *err = nullptr;
  cudaError_t e = cudaMalloc(&bar, MACRO_BAR_WORDS * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(bar, 0, MACRO_BAR_WORDS * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  const long long limit = 1LL << 24;
  if (e == cudaSuccess) e = which == 0 ? probe_barrier_timeout(bar, err, limit, nullptr) : probe_mbarrier_timeout(err, limit, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (bar) cudaFree(bar);
  if (err) cudaFree(err);
  if (e != cudaSuccess) return GSIS_E_CUDA;
  *device_status = h;
  return GSIS_OK;
}
