// gsis_internal.h -- structures shared by the host solver object and the CUDA kernels.
// Not part of the public ABI (include/gsis.h is).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gsis {

constexpr int VB = 32;          // discrete velocities per block (one per lane)
constexpr int NMOM = 13;        // raw moments of f0 about the state velocity: 1, c(3), cc(6), |c|^2 c(3)
constexpr int NMOM1 = 4;        // raw moments of f1 (Rykov) about the state velocity: 1, c(3)
constexpr int NFF = 5;          // kinetic flux sums: mass, momentum(3), energy (with f1)
constexpr int NWF = 6;          // wall-flux moments: NFF and the internal energy (f1; 0 for Shakhov)
// per-cell moment vector of the moments kernel: f0 moments, flux sums, then for Rykov the f1
// flux sum and the f1 moments
__host__ __device__ constexpr int moment_len(int nvdf) { return nvdf == 2 ? NMOM + NFF + 1 + NMOM1 : NMOM + NFF; }
constexpr int NST = 48;         // per-cell kinetic state values:
                                //  [0..2] u_n, [3] 1/T_n, [4] rho_n (pi T_n)^-3/2 (Maxwellian of W^n),
                                //  [5..7] u_o, [8] 1/T_o, [9] rho_o (pi T_o)^-3/2 (of W^{n+1/2}),
                                //  [10] mass scale s, [11] 1/tau, [12..14] Shakhov heat-flux factor,
                                //  [15] diagonal, [16..18] u_r, [19] 1/T_r, [20] rho_r (pi T_r)^-3/2:
                                //  the Maxwellian an FP32/BF16 VDF is stored relative to,
                                //  [21] d_r T_r,r / 4 (the f1 reference factor), [22..23] unused,
                                //  Rykov: [24] 1/T, [25] rho (pi T)^-3/2 with T = (3Tt + d_r Tr)/(3 + d_r),
                                //  [26..28] 8 q0 / (15 rho T^2), [29] d_r Tr_n / 4, [30] d_r T / 4,
                                //  [31..33] 2 (pi Tt)^-3/2 qr / Tt, [34..36] 2 (pi T)^-3/2 q1 / T,
                                //  [37] 1 - 1/Z_r, [38] 1/Z_r, [39] d_r Tr_o / 4, [40..47] unused
constexpr int NST_RYKOV = 40;   // state values a Rykov kinetic step reads
constexpr int GSIS_ERR_DIVERGED = -4;  // same values as GSIS_E_DIVERGED / GSIS_E_TIMEOUT
constexpr int GSIS_ERR_TIMEOUT = -5;

// Per-axis geometry of one cell of a rectilinear block (natural orientation).
//   gradient along the axis: g = clo (q[i-1] - q[i]) + chi (q[i+1] - q[i])  (missing neighbour: 0)
//   face offsets from the cell centre: rlo = X[i] - xc[i] < 0, rhi = X[i+1] - xc[i] > 0
//   pad0 = 1 / (xc[i+1] - xc[i]) (0 for the last cell), pad1 unused
template <typename T>
struct alignas(8 * sizeof(T)) AxisCell {
  T invh, rlo, rhi, clo, chi, h, pad0, pad1;
};

// Per colour entry (octant independent): position inside the previous / next colour of the
// transformed upwind and downwind neighbour along each axis (-1 if none) and the transformed
// transverse index of the entry for each axis (index of its e-buffer slot).
struct alignas(16) EntryInfo {
  int nb[6];    // up x, dn x, up y, dn y, up z, dn z
  int trn[3];
  int pad[3];
};

// Per-cell kinetic state (values in the precision of the kinetic kernel):
//  [0..2] un       velocity of the state W^n (reference distribution, correction, moments)
//  [3]    invTn    1/Tt of W^n
//  [4]    Cn       rho (pi Tt)^(-3/2) of W^n
//  [5..7] uo       velocity of W^{n-1/2} (the moments the pending correction removes)
//  [8]    invTo
//  [9]    Co
//  [10]   s        closed-domain mass scale of the stored f
//  [11]   invtau   1/tau(W^n)
//  [12..14] Aq     8/(15 rho Tt^2) q_t (Shakhov heat-flux coefficient times q)
//  [15]   D0       1/dt + 1/tau
//  [16..19] reserved
// The stored f is f_raw; the VDF the step starts from is
//   f^n = s f_raw + Cn exp(-|xi-un|^2 invTn) - Co exp(-|xi-uo|^2 invTo)   (Eq. updatef, lazily).

struct KinGeom {
  int n[3];
  int nc;
  int act[3];
  int nact;
  int ncol, maxcol;
  int ntrans[3];        // transverse face count per axis (0 if inactive)
  int wall_base[6];     // first wall-face id of each side, -1 if not a wall
  double K3;            // venkat K^3: eps^2 = K^3 V
  int tile[3];          // velocity blocks as TX x TY x TZ tiles of their octant ({0,0,0}: not tiled)
};
constexpr int KFAC_MAX = 10;    // one-dimensional Maxwellian factors per tiled block at most

// General (curvilinear) structured meshes.  Per cell and side: the outward area vector S, the
// vector r from the cell centre to the face centre, the least-squares weight w (gradient =
// sum over the in-domain neighbours of w (q_j - q_i)) and 1/|S|; per cell 1/V and the
// Venkatakrishnan eps^2 = (K V^(1/3))^3.  Neighbour codes: >= 0 a cell, or one of the NB_*.
template <typename T>
struct GenFace {
  T S[3], r[3], w[3], invA;
};
template <typename T>
struct GenCell {
  GenFace<T> f[6];
  T invV, eps2;
};
constexpr int NB_WALL = -1, NB_ABSENT = -2, NB_AXIS = -3, NB_FAR = -4;

// T: kinetic arithmetic (float or double); S: VDF storage (T, or __nv_bfloat16 with T = float)
template <typename T, typename S = T>
struct KinArgs {
  KinGeom g;
  const AxisCell<T> *ax[3];
  const T *vel;          // [slot][4]: xi_x, xi_y, xi_z, w
  const int8_t *boct;    // octant of each block: bit a set => xi_a < 0
  const int *col_off;    // [ncol+1], or per octant [8][col_stride] when col_stride > 0
  int col_stride;        // 0: one colour list for every octant (general kernel)
  const EntryInfo *entry;  // [entry] neighbour positions and transverse indices
  const int4 *natcell;     // [octant][entry]: cell index and natural coordinates
  const T *st;           // [cell][NST]
  const double *rho_w;   // [nwall]
  const double *wall_uT; // [6][4]: u_w(3), T_w
  S *f;                  // [block][cell][VB] f_raw, updated in place
  S *f1;                 // Rykov: the second reduced VDF, same layout (nullptr for Shakhov)
  int nvdf;              // 1 (Shakhov) or 2 (Rykov)
  double d_r;            // rotational degrees of freedom (Rykov)
  T *wpart;              // [block][wall face][NWF] outgoing wall-flux moments (wall cells only)
  int nwall;
  int nblocks;
  int *err;              // device error flag (a bounded wait that timed out)
  unsigned char *gscratch;  // ring and face buffers in global memory (nullptr: shared memory);
                            // general meshes: the per-CTA work arrays of the kinetic kernel
  size_t gstride;           // bytes of gscratch per velocity block (general meshes: per CTA)
  // general meshes (nullptr otherwise)
  const GenCell<T> *gen;    // [cell]
  const int *gnb;           // [cell][6] neighbour codes
  const int *gwid;          // [cell][6] wall-face id, -1 if the side is not a wall
  const unsigned char *gin; // [cell][6] far-field sides: 1 where the free stream enters
  int n_sweeps;             // point-implicit passes over the colours
  int pos_faces;            // general meshes: face values that keep the sign of the cell value
  double *kpart;            // [CTA][cell][6] per-CTA sums of the outward kinetic face fluxes
                            // (area-integrated, over the cell's faces); nullptr: not wanted
  const double *wden;       // [wall face] re-emission flux of M(u_w, T_w) over every velocity
                            // (all shards), the denominator of rho_w
  // unstructured meshes (nullptr on structured blocks): per cell and side the neighbour's side
  // of the shared face (else the opposite side s ^ 1), the boundary patch (else the side s)
  const unsigned char *gnf;
  const unsigned char *gpat;
  // unstructured meshes: the least-squares stencil as CSR (cell c: entries gso[c] .. gso[c+1]-1
  // of neighbour gsi[e] with weight gsw[e][3]; gradient = sum_e w_e (q_j - q_c)); nullptr: the
  // per-side weights of GenCell over the face neighbours
  const int *gso;
  const int *gsi;
  const T *gsw;
};
// the neighbour's side of the face a cell shares through side s, and the boundary patch of side s
__host__ __device__ inline int nb_side(const unsigned char *gnf, int c, int s) { return gnf ? gnf[6 * c + s] : (s ^ 1); }
__host__ __device__ inline int patch_of(const unsigned char *gpat, int c, int s) { return gpat ? gpat[6 * c + s] : s; }

// ---- launchers (defined in the .cu files) ----
template <typename T, typename S>
cudaError_t launch_kinetic(const KinArgs<T, S> &a, int nblocks, int nwarps, size_t smem, cudaStream_t s);
template <typename T, typename S>
size_t kinetic_smem_bytes(const KinGeom &g, int nvdf);
// bytes of global scratch per velocity block when the ring and face buffers live there
template <typename T, typename S>
size_t kinetic_gscratch_stride(const KinGeom &g, int nvdf);
template <typename T, typename S>
cudaError_t launch_wall_prepass(const KinArgs<T, S> &a, const int *wall_cell, const int *wall_side, int nwall,
                                const double *Z0, double *rho_w, int nslots, cudaStream_t s);
template <typename T, typename S>
cudaError_t launch_moments(const KinArgs<T, S> &a, int blocks_per_chunk, int nchunks, double *mp, cudaStream_t s);
// FP64 storage, Shakhov: moments about the origin from the per-slot table mtab [slot][16] into
// chunks 0..nchunks-1 of mp, and the closed-form sums of w phi g^n (from the 1-D grids in vaxis:
// nodes of x, y, z, then their weights) into chunk nchunks (zeros unless emit)
cudaError_t launch_moments_origin(const KinArgs<double, double> &a, const double *mtab, int blocks_per_chunk,
                                  int nchunks, const double *st64, const double *vaxis, const int *nv_axis, int emit,
                                  double *mp, cudaStream_t s);
template <typename T, typename S>
cudaError_t launch_init_maxwellian(const KinArgs<T, S> &a, const double *W0, int nblocks, cudaStream_t s);
template <typename T, typename S>
cudaError_t launch_export_f(const KinArgs<T, S> &a, int q, const int *slot_canon, int nslots, int nv, double *out,
                            cudaStream_t s);
template <typename T, typename S>
cudaError_t launch_import_f(const KinArgs<T, S> &a, int q, const int *slot_canon, int nslots, int nv, const double *in,
                            cudaStream_t s);
// general meshes: the kinetic step as a persistent kernel over the velocity blocks (grid CTAs of
// 8 warps, each with gstride bytes of work arrays), and the wall pre-pass
template <typename T, typename S>
cudaError_t launch_kinetic_general(const KinArgs<T, S> &a, int grid, cudaStream_t s);
template <typename T, typename S>
cudaError_t kinetic_general_shape(int nvdf, int nact, int *ctas_per_sm);
template <typename T, typename S>
size_t kinetic_general_stride(int nc, int nvdf, int nact);
// general meshes: per wall face, the flux of the wall Maxwellian leaving the wall summed over
// every velocity slot (nslots_all of vel64, all shards), the denominator of rho_w
template <typename T, typename S>
cudaError_t launch_wall_den_general(const KinArgs<T, S> &a, const double *vel64, int nslots_all, const int *wall_cell,
                                    const int *wall_side, int nwall, double *wden, cudaStream_t s);
// K [cell][6] = sum over the CTAs of kpart (fixed order)
cudaError_t launch_sum_kpart(const double *kpart, int nparts, int nc, double *K, cudaStream_t s);
template <typename T, typename S>
cudaError_t launch_wall_prepass_general(const KinArgs<T, S> &a, const int *wall_cell, const int *wall_side, int nwall,
                                        double *rho_w, cudaStream_t s);

// launch shape of the kinetic kernel (gm: ring in global scratch): warps = want_warps capped by
// the kernel's registers, and the blocks of that size and dynamic shared memory an SM holds
template <typename T, typename S>
cudaError_t kinetic_shape(const KinGeom &g, int nvdf, bool gm, int want_warps, size_t smem, int *warps,
                          int *ctas_per_sm);

cudaError_t launch_wall_constants(const double *vel64, int nslots, const double *wall_uT, const int *sides,
                                  int nsides, double *Z0, double *Zw, double d_r, cudaStream_t s);

// per-chunk moment partials [chunk][cell][18] -> mom [cell][13] and kinetic flux sum
// K [cell][6] (outward, area-integrated, via the delta-form identity); per-block wall partials
// -> wf [wall][6] outward kinetic wall flux per unit area.
// origin: the chunks hold FP64 moments about the origin and, in the last chunk, the sums of
// w phi g^n (launch_moments_origin); the reduction forms the collision sums and shifts the
// moments to the state velocity.
template <typename T>
cudaError_t launch_reduce(const double *mp, int nchunks, int nvdf, const T *wpart, const int8_t *boct, int nblocks,
                          const KinGeom &g, const int *wall_cell, const int *wall_side, int nwall,
                          const double *rho_w, const double *Zw, bool emit, bool general, const double *vol,
                          const double *st64, double *mom, double *K, double *wf, cudaStream_t s,
                          bool origin = false);
constexpr int MOM_STRIDE = NMOM + NMOM1;  // per-cell raw moments: f0 then f1

struct FinalizeArgs {
  KinGeom g;
  const double *mom;     // [cell][MOM_STRIDE] raw moments about the state velocity
  int nvdf;
  double d_r;
  const double *st64;    // [cell][NST] FP64 copy of the state (un at [0..2])
  const double *vol;     // [cell]
  double mass_ref;
  int closed;
  double *Mh;            // out [cell][18]
  double *mass_scale;    // out [1]
  double *scratch;       // >= 2 * nblocks doubles
  unsigned *ticket;      // zero-initialised counter
  int *err;
};
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s);

struct CellFieldArgs {
  KinGeom g;
  const AxisCell<double> *ax[3];
  double Kn, omega;
  int model;
  double d_r, Z_r, A[4];
};
// HoT (Eq. full_constitutive) for reporting, per cell from Mh
cudaError_t launch_hot(const CellFieldArgs &c, const double *Mh, double *hot, cudaStream_t s);

struct StateArgs {
  KinGeom g;
  const double *Wn;       // [cell][6] prim state for the next step
  const double *Mh;       // [cell][18] moments of f^{n+1/2} (after mass scaling)
  double mass_scale;      // device value read inside via pointer below
  const double *mass_scale_ptr;
  double Kn, omega, kin_inv_dt;
  double *st64;           // out FP64 state
  void *stT;              // out state in kernel precision
  int is_float;
  int nvdf;               // Rykov (2): the state carries the Rykov values
  double d_r, Z_r, A[4];
};
cudaError_t launch_state(const StateArgs &a, cudaStream_t s);

struct EpsArgs {
  int nc;
  double vsum;                  // total volume
  const double *Wn, *Wo, *vol;  // prim [cell][6]
  double *scratch;              // >= 7 * nblocks
  unsigned *ticket;
  double *eps4;                 // out: rho, u, Tt, max
};
cudaError_t launch_eps(const EpsArgs &a, cudaStream_t s);

struct WallLoadArgs {
  const double *wf;            // [wall face][6] kinetic wall flux per unit area (outward)
  const int *wall_cell, *wall_side;
  int nwall;
  int n[3];
  const AxisCell<double> *ax[3];
  const double *area;          // general meshes: [wall face] area (nullptr: from ax)
  unsigned mask;               // bit s selects wall side s
  double dir[3], rho_ref, U_ref, A_ref;
  double *out;                 // [6] force(3), energy flux, C_D, C_H
};
cudaError_t launch_wall_loads(const WallLoadArgs &a, cudaStream_t s);

struct MacroArgs {
  KinGeom g;
  const AxisCell<double> *ax[3];
  double Kn, omega, cfl, tol;
  double mu0;              // Kn / sqrt(pi): mu = mu0 T^omega
  int model, nW, steps, sweeps;
  double d_r, Z_r, A[4];
  double mass_ref;
  double den_floor;        // 1e-24 x total volume: fields with sum W_k^2 V below it count as zero
  int closed;
  const double *Mh;        // [cell][18] initial state W^{n+1/2}
  int wall_g13;            // wall flux increments of the Grad-13 VDF (else of the local Maxwellian)
  const double *K;         // [cell][6] sum over the cell's faces of the outward kinetic flux (area-integrated)
  const int *wall_cell, *wall_side;
  int nwall;
  const double *wall_uT;   // [6][4]
  // work (device, sized by the host)
  const int *colcells;     // red cells (i+j+k even) then black cells
  int ncol0;               // number of red cells
  double *W, *pr, *aux, *gW, *phW, *gP, *R, *invD, *dW, *Fc, *corr, *gam, *red, *Ffc, *wfl;
  double *G;               // [cell][3][2][6] off-diagonal terms a cell publishes for its neighbours
                           // along each axis: [0] for the upper one, [1] for the lower one
  double *Wout;            // [cell][6] prim W^{n+1}
  unsigned *bar;           // barrier counter, generation; zero at launch
  int *err;
  int *iters;              // out
};
// The synthetic solve on general meshes (one thread per cell, one launch per phase)
constexpr int MACRO_MAX_COLOURS = 32;  // colours of the synthetic solve's sweeps at most
struct MacroGenArgs {
  int nc, nW, model, steps, sweeps, closed, ncol0;
  int ncolm;                   // colours of the LU-SGS passes (cells of colour k: colcells[colm_off[k] ..])
  int colm_off[MACRO_MAX_COLOURS + 1];
  const unsigned char *gnf, *gpat;  // unstructured meshes (see KinArgs), else nullptr
  const int *gso, *gsi;             // least-squares stencil (see KinArgs), else nullptr
  const double *gsw;
  int euler;                   // 1: the inviscid presteps (slip walls, no correction, K unused)
  int wall_g13;                // wall flux of the Grad-13 VDF (needs mh_stride 18: the moments)
  double relax;                // GSIS update W^{n+1/2} + relax (W^{n+1} - W^{n+1/2}) (1: the full one)
  double visc_jump;            // weight of the jump term in the viscous face gradients (0: the mean)
  int mh_stride;               // doubles per cell of Mh (18: the moments; 6: a primitive state)
  double mu0, omega, cfl, tol, d_r, Z_r, A[4], mass_ref;
  double vsum;                 // total volume (fields with sum W_k^2 V <= 1e-24 vsum count as zero)
  const GenCell<double> *gen;  // [cell] FP64 geometry
  const int *gnb;              // [cell][6]
  const double *xc, *vol;      // [cell][3], [cell]
  const double *wall_uT;       // [6][4]: wall u, T; far field: free-stream u, T
  const double *Mh;            // [cell][mh_stride] initial primitives rho, u, T_t, T_r
  const double *K;             // [cell][6] area-integrated outward kinetic flux summed over the faces
  const int *colcells;         // red cells then black cells
  // work
  double *W, *pr, *mu, *gW, *phW, *gP, *R, *D, *dW, *F0, *part;  // D: the inverse LU-SGS diagonal
  double *Ff;                  // [cell][6][6]: interior face fluxes
  double *gam;                 // [cell][6] gamma of each interior face for the sweeps
  double *FW0, *FW;            // [cell][3][6] axis fluxes at W and at W + dW for the sweeps
  int *flag;                   // [0] early exit fired, [1] inner steps used
  double *Wout;                // [cell][6] prim W^{n+1}
  int *err, *iters;
};
int macro_general_parts(int nc);  // blocks of the per-cell launches (rows of `part`)
cudaError_t run_macro_general(const MacroGenArgs &a, cudaStream_t s);

constexpr int MACRO_MAX_GRID = 512;  // blocks of the synthetic-solve kernel at most
constexpr int MACRO_BAR_WORDS = 512;  // barrier words, cleared before each launch
cudaError_t launch_macro(const MacroArgs &a, int grid, int block, cudaStream_t s);
// self-tests of the bounded device waits (each raises GSIS_ERR_TIMEOUT in *err after `limit` cycles)
cudaError_t probe_barrier_timeout(unsigned *bar, int *err, long long limit, cudaStream_t s);
cudaError_t probe_mbarrier_timeout(int *err, long long limit, cudaStream_t s);
cudaError_t macro_launch_shape(int nc, int max_sms, int *grid, int *block);

// message returned by gsis_last_error(NULL) for a failed call that has no handle
void set_handle_free_error(const char *msg);

}  // namespace gsis
