// Internal declarations of the GB300 Helmholtz multigrid library.
//
// Device storage per level (all vectors in the TILED layout of hmg.h:
// tiles of 32 columns, layer-major inside a tile, so that one warp holding
// 32 columns reads one layer of all of them with a single coalesced access):
//   nbr   int4[ncp]      three neighbour columns (w unused)
//   gh    double4_32a[ncp]   horizontal couplings g_k = w_c^2 / Mh_ff of the three
//                        lateral faces and their sum G (layer independent)
//   d, e  double[Np]     diagonal of H^ and the vertical off-diagonal
//                        H^[(c,l),(c,l-1)] (e = 0 at l = 0)
//   lo, w double[Np]     twisted factorisation N D N^T of H^_z (twist at
//                        layer `twist`): multipliers and omega / D_l
//   mt    double[ncp]    the second multiplier of the twist row
//   los, mts             the same multipliers scaled to the pivot of their
//                        own row (e/D_l), for the forward recurrence of the
//                        twisted tile sweep in z = (omega / D) y
//   *32                  FP32 copies for the mixed-precision cycle (lo32,
//                        w32, mt32: the factorisation twisted at `twist32`,
//                        computed in FP64 and rounded once)
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hmg.h"

namespace hmg {

constexpr int TW = 32;                 // columns per tile
constexpr int SMALL_LEVEL_TILES = 160;  // levels with at most this many tiles are latency bound
constexpr int FUSED_PROLONG_MAX_TILES = 160;  // FP64 levels up to this size fuse prolongation into the sweep
// The coarse end of the V-cycle, from the first level of at most
// CC_MAX_TILES tiles (below the finest) down, runs as one cooperative kernel.
constexpr int CC_MAX_TILES = 160;
constexpr int CC_MAX_LEVELS = 8;
constexpr int RED_MAX_BLOCKS = 16384;  // partial sums of one reduction (>= tiles of the finest level)
constexpr int GMRES_MAX_RESTART = HMG_GMRES_MAX_RESTART;
constexpr int GS_MAX_BLOCKS = 1216;    // blocks of one Gram-Schmidt pass (8 per SM)

struct HostLevel {
  int refinement = 0;
  int ncols = 0;
  std::vector<double> verts;      // ncols * 9: three unit-sphere vertices per column
  std::vector<double> centroid;   // ncols * 3
  std::vector<int32_t> nbr;       // ncols * 3
};

std::vector<HostLevel> build_mesh_hierarchy(int refinement, int nlevels);

// Horizontal domain decomposition (partition.cpp).  One part of one
// partitioned level: owned columns [begin, end) in the global numbering;
// local numbering = owned columns (c - begin), padded to n_own_pad, then the
// ghost columns in ghost order, sorted by (owner part, global column).
struct PartLevel {
  int32_t begin = 0, end = 0, n_own = 0, n_own_pad = 0;
  std::vector<int32_t> ghost_col, ghost_owner, ghost_owner_local;
  std::vector<int32_t> local_nbr;            // n_own * 3 local indices
  std::vector<int32_t> send_col, send_to;    // sorted by (to, position in the receiver's ghost list)
};
struct PartitionPlan {
  int nparts = 0;
  int nlevels = 0;                           // partitioned levels 0 .. nlevels - 1
  std::vector<std::vector<PartLevel>> lv;    // [level][part]
};
// Levels split over the parts: all but the coarsest (gathered on one part),
// or the only one.
int partitioned_levels(int nlevels);
PartitionPlan build_partition(const std::vector<std::vector<int32_t>>& nbr, const std::vector<int>& ncols,
                              int nparts);
PartitionPlan build_partition_for_mesh(int refinement, int nlevels, int nparts);

struct Level {
  int refinement = 0, nc = 0, ncp = 0, nz = 0;
  // twist rows of the column factorisations.  FP64 factors (lo, w, mt):
  // nz / 2 on every level (the FP64 sweep relaxes each half column on its own
  // warp).  FP32 factors (lo32, w32, mt32): nz / 2 on small levels (two
  // half-length recurrences, latency bound), nz - 1 elsewhere (one recurrence:
  // the plain L D L^T of the register-column FP32 sweep).
  int twist = 0;
  int twist32 = 0;
  int64_t N = 0, Np = 0;
  std::vector<double> centroid_host;
  std::vector<int32_t> nbr_host;
  std::vector<double> verts_host;   // nc * 9
  // geometry
  int4* nbr = nullptr;
  double* verts = nullptr;    // ncp * 9
  double* A1 = nullptr;       // ncp, unit-sphere flat-triangle area
  double4_32a* sigma = nullptr;   // ncp, RT0 shape factors of the three edges
  // coefficients
  double4_32a* gh = nullptr;
  float4* gh32 = nullptr;
  double *d = nullptr, *e = nullptr, *lo = nullptr, *w = nullptr, *mt = nullptr;
  double *los = nullptr, *mts = nullptr;   // Np, ncp: scaled multipliers (FP64 factors)
  float *d32 = nullptr, *e32 = nullptr, *lo32 = nullptr, *w32 = nullptr, *mt32 = nullptr;
  double* theta = nullptr;    // Np
  // cycle work vectors
  // b: right-hand side of this level (restricted residual); ua, ub: smoother
  // ping-pong; ux: result of this level's cycle (the coarse correction)
  double *b64 = nullptr, *ua64 = nullptr, *ub64 = nullptr, *ux64 = nullptr;
  float *b32 = nullptr, *ua32 = nullptr, *ub32 = nullptr, *ux32 = nullptr;
};

// Slots of the Krylov scalars kept on the device.
enum Scalar {
  S_BB = 0, S_RZ, S_PQ, S_RR, S_ALPHA, S_BETA, S_ZQ, S_RZNEW, S_TRUE, S_FLAG, S_COUNT = 16
};
// Flag bits raised by reduction epilogues.
enum { F_NONFINITE = 1, F_BREAKDOWN = 2 };
// What the last block of a reduction does with the sums.
enum Epilogue {
  EPI_STORE0 = 0,   // sc[slot] = s0
  EPI_ALPHA,        // sc[PQ] = s0; sc[ALPHA] = sc[RZ] / s0
  EPI_RR,           // sc[RR] = s0 (flag non-finite)
  EPI_BETA_CG,      // sc[BETA] = s0 / sc[RZ]; sc[RZ] = s0
  EPI_BETA_FCG,     // sc[BETA] = -sc[ALPHA] * s1 / sc[RZ]; sc[RZ] = s0
  EPI_INIT_RZ       // sc[RZ] = s0 (flag non-positive)
};

struct Reduce {
  double* partials = nullptr;   // RED_MAX_BLOCKS * 2
  unsigned int* counter = nullptr;
  double* sc = nullptr;         // S_COUNT scalars
  int epilogue = EPI_STORE0;
  int slot = 0;
};

struct Phys {
  double R = 0, dz = 0, wc2 = 0, vfac = 0, omega = 0.8;
  double a = 0, c2 = 0, wn2 = 0;   // dt / 2, c^2, w_N^2 (velocity-pressure system)
};

// The velocity-pressure system of the finest level (mixed.cu).  Vectors hold
// [horizontal faces | vertical faces | cells]: horizontal faces tiled like
// cells with edges in place of columns ((e / 32) * 32 * nz + l * 32 + e % 32,
// nep = edges padded to 32); vertical faces in the cell tiling, row l being
// the face between layers l and l + 1 (row nz - 1 zero); cells tiled.
struct MixedSys {
  bool ready = false;
  int ne = 0, nep = 0;
  int64_t nh = 0, n = 0;              // nep * nz; nh + 2 * Np
  std::vector<int32_t> edges_host;    // ne x (t, k, tn, kn), t < tn
  int4* edge = nullptr;               // nep: t, k, tn, kn
  int4* enb = nullptr;                // nep: the four coupled edges
  double4_32a* ecoef = nullptr;       // nep: their M2^h entries
  double* emass = nullptr;            // nep: M2^h diagonal
  double* einv = nullptr;             // nep: its reciprocal
  int4* cedge = nullptr;              // ncp: edges of local edges 0..2, sign bits in w
  double* zd = nullptr;               // Np: dz / (3 A_K)
  double* m3 = nullptr;               // Np: |K|
  double* zsi = nullptr;              // Np: 1 / M2^z diagonal of the face above the cell
  double *b = nullptr, *x = nullptr, *t1 = nullptr, *t2 = nullptr;   // n entries each
};
void launch_mixed_coeffs(const Level& L, const MixedSys& M, const Phys& ph, cudaStream_t s);
void launch_mixed_apply(const Level& L, const MixedSys& M, const Phys& ph, const double* x, double* y,
                        cudaStream_t s);
void launch_mixed_pre_lower(const Level& L, const MixedSys& M, const Phys& ph, const double* r, double* rp,
                            cudaStream_t s);  // rp = r_P - a c^2 D M2inv r_U
void launch_mixed_pre_upper(const Level& L, const MixedSys& M, const Phys& ph, const double* r, double* z,
                            cudaStream_t s);  // z_U = M2inv (r_U + a D^T z_P)
void launch_mixed_layout(const Level& L, const MixedSys& M, bool to_tiled, const double* u_col, const double* p_col,
                         double* tiled, double* u_out, double* p_out, cudaStream_t s);

// ---- next-to-lowest order (nlo_setup.cpp: host assembly; nlo.cu: kernels)
// Column blocks of the NLO operator per cell (6 x 6, row-major, unknown
// u = 2 j + m): diag = H^[(c,l),(c,l)], sub = H^[(c,l),(c,l-1)]; nbr =
// H^[(c,l),(n_k,l)] per column and local edge k (layer independent).
struct NloHost {
  int nc = 0, nz = 0;
  std::vector<double> diag, sub, nbr;
  // nbr = nbr3 (x) Z2 with Z2 = [[5, 4], [4, 5]] / 12 (the vertical DG1
  // factor): nbr3[(3 c + k) * 9 + 3 j + j'] is the horizontal factor
  std::vector<double> nbr3;
};
NloHost nlo_assemble_host(const std::vector<double>& verts, const std::vector<int32_t>& nbr, int nc, int nz,
                          const Phys& ph);
// Block L D L^T of the column part: Lf[cell] = L_l (zero at l = 0),
// Dinv[cell] = omega Dt_l^-1.
void nlo_factor_host(const NloHost& H, double omega, std::vector<double>& Lf, std::vector<double>& Dinv);

// CSR matrix (host or device arrays)
struct Csr {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};
// The NLO velocity-pressure system on the host: A (n x n), D (np x nu),
// D^T (nu x np) and the diagonal of M2~ (nu), in the NLO mixed COLUMN layout.
struct NloMixedHost {
  int64_t nue = 0, nui = 0, nuz = 0, nu = 0, np = 0, n = 0;
  Csr A, D, Dt;
  std::vector<double> m2diag;
};
NloMixedHost nlo_mixed_assemble_host(const std::vector<double>& verts, const std::vector<int32_t>& nbr,
                                     const std::vector<int32_t>& edges, int nc, int nz, const Phys& ph);

// A CSR matrix on the device.
struct DevCsr {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int64_t* ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};
// y = (y0 + alpha A x) * s, elementwise s and y0 optional (nlo_mixed.cu)
void launch_csr_spmv(const DevCsr& A, const double* x, double alpha, const double* y0, const double* s, double* y,
                     cudaStream_t st);
void launch_mul(int64_t n, const double* a, const double* b, double* y, cudaStream_t st);   // y = a * b
// the same product with FP32 values and x, accumulated in FP32 (FP64 y0, s, y)
void launch_csr_spmv32(const DevCsr& A, const float* val32, const float* x, double alpha, const double* y0,
                       const double* s, double* y, cudaStream_t st);
void launch_mul32(int64_t n, const double* a, const double* b, float* y, cudaStream_t st);  // y = a * b in FP32
// The NLO velocity-pressure system on the device (NLO mixed COLUMN layout).
struct NloMixedSys {
  bool ready = false;
  int64_t nue = 0, nui = 0, nuz = 0, nu = 0, np = 0, n = 0;
  DevCsr A, D, Dt;
  double* m2inv = nullptr;                                      // nu
  double *b = nullptr, *x = nullptr, *t1 = nullptr, *t2 = nullptr;   // n
  // mixed form: FP32 values of D and D^T and FP32 operands of their products
  float *Dval32 = nullptr, *Dtval32 = nullptr, *tu32 = nullptr, *zp32 = nullptr;
};

constexpr int NLO_TILE = 5;   // columns per warp: lanes 6 c5 + u, lanes 30 and 31 padding
// The NLO system of the finest mesh.  Vectors: tiles of 5 columns, one row
// of 32 doubles per (tile, layer), index (t * nz + l) * 32 + 6 c5 + u
// (columns 5 t + c5); padding lanes zero.  Coefficients: 6 rows of 32 per
// (tile, layer), index ((t * nz + l) * 6 + e) * 32 + lane = entry (u, e) of
// the lane's cell: Ad the diagonal block, Cs the sub-diagonal block, Cu the
// super-diagonal block (C_(l+1)^T), Lf the forward multipliers L_l, Di
// omega Dt_l^-1, Lb the backward multipliers L_(l+1)^T.  Nb: 3 rows of 32 per
// (tile, edge k): row j' holds, in lane 6 c5 + 2 j + m, entry (j, j') of the
// horizontal factor of the neighbour block (the block is that factor times
// Z2 = [[5, 4], [4, 5]] / 12 over (m, m')); nb: per (tile, edge k, lane) the
// offset of the neighbour column's row 0 plus its 6 c5.
struct NloSys {
  bool ready = false;        // coefficients of the current assembly uploaded
  bool allocated = false;
  int nt = 0;
  int64_t n = 0;             // nt * nz * 32
  double *Ad = nullptr, *Cs = nullptr, *Cu = nullptr, *Lf = nullptr, *Di = nullptr, *Lb = nullptr;
  double* Nb = nullptr;
  int* nb = nullptr;
  double *b = nullptr, *x = nullptr, *t1 = nullptr, *t2 = nullptr, *w = nullptr, *ua = nullptr, *ub = nullptr;
  // FP32 copies for the mixed form, and its FP32 work vectors
  float *Ad32 = nullptr, *Cs32 = nullptr, *Cu32 = nullptr, *Lf32 = nullptr, *Di32 = nullptr, *Lb32 = nullptr;
  float* Nb32 = nullptr;
  float *b32 = nullptr, *w32 = nullptr, *ua32 = nullptr, *ub32 = nullptr;
};
void nlo_pack_host(const NloHost& H, const std::vector<double>& Lf, const std::vector<double>& Dinv,
                   const std::vector<int32_t>& nbr, std::vector<double>* Ad, std::vector<double>* Cs,
                   std::vector<double>* Cu, std::vector<double>* Lft, std::vector<double>* Dit,
                   std::vector<double>* Lb, std::vector<double>* Nb, std::vector<int>* nb);
void launch_nlo_layout(const NloSys& X, int nz, bool to_tiled, const double* src, double* dst, cudaStream_t s);
void launch_nlo_apply(const NloSys& X, int nz, const double* x, double* y, cudaStream_t s);   // FP64
// bc (lowest-order level L0, TILED, type bc_dt) = P^T (b - H^ u), P the
// embedding DG0 -> DG1; b and u of type dt
void launch_nlo_resid_restrict(const NloSys& X, const Level& L0, int dt, const void* b, const void* u, void* bc,
                               int bc_dt, cudaStream_t s);
// uo = u + omega H^_z^-1 (b - H^ u) in type dt (u == nullptr: from u = 0);
// b of type b_dt (FP64 with dt FP32 only from zero, then copied to bcopy if
// given), uo of type uo_dt
void launch_nlo_sweep(const NloSys& X, int nz, int dt, const void* b, int b_dt, void* bcopy, const void* u,
                      void* uo, int uo_dt, double omega, cudaStream_t s);
// u (type dt) += P ec, ec on the lowest-order level L0 (TILED, type ec_dt)
void launch_nlo_prolong(const NloSys& X, const Level& L0, int dt, void* u, const void* ec, int ec_dt,
                        cudaStream_t s);

// ---- assembly (assemble.cu)
void launch_geometry(const Level& L, cudaStream_t s);
void launch_couplings(const Level& L, double wc2_dz, cudaStream_t s);
void launch_bands(const Level& L, const Phys& ph, cudaStream_t s);
void launch_ldl(const Level& L, double omega, cudaStream_t s);
void launch_to_fp32(const Level& L, cudaStream_t s);
void launch_theta_restrict(const Level& fine, const Level& coarse, cudaStream_t s);
void launch_theta_grad(const Level& L, const Phys& ph, const double* p_col, const double* lam_col,
                       double* grad_col, cudaStream_t s);

// ---- cycle kernels (cycle.cu); dt = HMG_FP64 or HMG_FP32 names the type of
// each void* buffer.
void launch_sweep0(const Level& L, int dt, const void* b, int b_dt, void* u, float* bcopy,
                   double omega, cudaStream_t s);
// Optional dot products fused into a sweep: s0 = a . u', s1 = u' . c (c may be null).
struct SweepDot {
  const double* a = nullptr;
  const double* c = nullptr;
  Reduce red{};
};
void launch_sweep(const Level& L, int dt, const void* b, const void* u, void* uo, int uo_dt, const void* ec,
                  int ec_dt, double omega, const SweepDot* dot, cudaStream_t s);
void launch_prolong(const Level& L, int dt, void* u, const void* ec, int ec_dt, cudaStream_t s);
// Halo exchange and column copies of the domain decomposition (halo.cu).
constexpr int MAX_PARTS = 16;
struct PartPtrs {
  void* p[MAX_PARTS];
};
// buf[e][l] = v.p[part[e]] at (col[e], l), e < n (tiled layout of the part)
void launch_halo_pack(int n, int nz, const int32_t* part, const int32_t* col, const PartPtrs& v, void* buf, int dt,
                      cudaStream_t s);
// v.p[part[e]] at (col[e], l) = buf[e][l]
void launch_halo_unpack(int n, int nz, const int32_t* part, const int32_t* col, const PartPtrs& v,
                        const void* buf, int dt, cudaStream_t s);
// dst column dst0 + c = src column src0 + c, c < ncols, every layer
void launch_copy_cols(int ncols, int nz, const void* src, int src0, void* dst, int dst0, int dt, cudaStream_t s);

// The V-cycle from level ls (b_in: its right-hand side, out: its result,
// both of its type) down to level nlev - 1 and back, as one cooperative
// kernel (cycle.cu, k_coarse_cycle).  Returns the launch's error.
cudaError_t launch_coarse_cycle(const Level* lv, int ls, int nlev, int nu_pre, int nu_post, int n_coarse,
                                double omega, bool mixed, const void* b_in, void* out, cudaStream_t s);
void launch_resid_restrict(const Level& L, int dt, const void* b, const void* u, void* bc, int bc_dt,
                           cudaStream_t s);
void launch_apply(const Level& L, int dt, const void* x, void* y, const Reduce* red, cudaStream_t s);

// ---- Krylov vector kernels (krylov.cu), FP64, tiled layout of level L
void launch_to_tiled(const Level& L, int dt, const void* col, void* tiled, cudaStream_t s);
void launch_to_column(const Level& L, int dt, const void* tiled, void* col, cudaStream_t s);
// tile transpose of nitems columns of nzc values (COLUMN) <-> nz tiled rows (rows >= nzc zero)
void launch_transpose64(bool to_tiled, int nitems, int nz, int nzc, const double* src, double* dst, cudaStream_t s);
void launch_dot(const Level& L, const double* a, const double* b, const double* c, const double* d,
                const Reduce& red, cudaStream_t s);  // s0 = a.b, s1 = c.d (c may be null)
void launch_update_p(const Level& L, double* p, const double* z, const double* sc, cudaStream_t s);
// Device-side CG loop state: the iteration k, its limit, rtol^2 and the
// relative residual after each iteration (at most CG_LOOP_HIST iterations;
// longer solves run the host-side loop).
constexpr int CG_LOOP_HIST = 1024;
struct CgLoop {
  double rtol2;
  double rr;          // ||r_k||^2 and the reduction flags seen by the last test
  int flag;
  int max_iter;
  int k;
  double hist[CG_LOOP_HIST];
};
void launch_cg_loop_init(CgLoop* loop, double rtol2, int max_iter, cudaStream_t s);
// FP64 FMA throughput of this device in TFLOP/s (krylov.cu, k_fp64_fma_probe);
// synchronises the stream.
double measure_fp64_fma_rate(double* sink, cudaStream_t s);
void launch_cg_control(CgLoop* loop, const double* sc, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_update_xr(const Level& L, double* x, double* r, const double* p, const double* q,
                      const Reduce& red, cudaStream_t s);
void launch_resid_sq(const Level& L, const double* b, const double* q, const Reduce& red,
                     cudaStream_t s);  // s0 = |b - q|^2
void launch_check_finite(const Level& L, const double* v, const Reduce& red, cudaStream_t s);

int reduce_grid(int64_t n);

// GMRES (gmres.cu).  Basis vectors are contiguous FP64 tiled vectors, vector
// i at V + i * ld; nv <= GMRES_MAX_RESTART.
struct GsWork {
  double* part = nullptr;       // (GMRES_MAX_RESTART + 1) * GS_MAX_BLOCKS block partials
  unsigned int* counter = nullptr;
  double* h = nullptr;          // GMRES_MAX_RESTART: first-pass coefficients
  double* h2 = nullptr;         // GMRES_MAX_RESTART + 1: second-pass coefficients (if any), then |w|^2
  double* hn = nullptr;         // 1: h_(j+1,j)
};
void launch_gs_dots(int64_t n, const double* V, int64_t ld, int nv, const double* w, const GsWork& ws,
                    cudaStream_t s);  // h = V^T w
void launch_gs_update(int64_t n, const double* V, int64_t ld, int nv, bool second_dots, double* w,
                      const GsWork& ws, cudaStream_t s);  // w -= V h; |w|^2 (second_dots: h2 = V^T w first)
void launch_gs_final(int64_t n, const double* V, int64_t ld, int nv, double* w, const GsWork& ws,
                     cudaStream_t s);  // w -= V h2; w /= hn
void launch_gmres_x(int64_t n, double* x, const double* Z, int64_t ld, int nv, const double* y,
                    cudaStream_t s);  // x += Z y
void launch_sub_norm(int64_t n, const double* b, const double* q, double* v, const Reduce& red,
                     cudaStream_t s);  // v = b - q; s0 = |v|^2
void launch_normalise(int64_t n, const double* a, double* v, const double* nrm2, cudaStream_t s);
void launch_dot_n(int64_t n, const double* a, const double* b, const Reduce& red, cudaStream_t s);  // s0 = a.b
// FP64 -> FP32 (round to nearest even) or FP32 -> FP64 on the integer pipe
void launch_convert(int64_t n, const void* src, int src_dt, void* dst, cudaStream_t s);


}  // namespace hmg

namespace hmg {
struct ProfRec {
  int kernel, level;
  size_t ev;  // index of the start event in the pool; the end event follows
};
// Events recorded as nodes of a captured graph (re-recorded at every replay).
struct GraphProf {
  int kernel, level;
  cudaEvent_t a, b;
};
}  // namespace hmg

struct hmg_ctx;
namespace hmg {
// Dynamic shared memory above 48 KB needs a per-kernel opt-in, and the
// attribute belongs to the device that is current when it is set.  One
// SmemOptIn per kernel instantiation records, per device ordinal, the largest
// size set so far; the mutex keeps host threads from racing on it.
struct SmemOptIn {
  std::mutex m;
  size_t bytes[64] = {};
};
template <typename K>
cudaError_t allow_smem(K kern, size_t smem, SmemOptIn& st) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(st.m);
  size_t& cur = st.bytes[dev & 63];
  if (cur >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) cur = smem;
  return e;
}

// Bracket a launch with the tracing events of hmg_profile_start when tracing
// selects (kernel, level); trace_begin returns the record to hand to
// trace_end (-1: not traced).  Both may throw on a CUDA error.
int trace_begin(hmg_ctx* c, int kernel, int level, cudaStream_t s);
void trace_end(hmg_ctx* c, int rec, cudaStream_t s);
}  // namespace hmg

struct hmg_ctx {
  // caller's device allocator (both null: the CUDA runtime's)
  hmg_alloc_fn alloc_fn = nullptr;
  hmg_release_fn release_fn = nullptr;
  void* alloc_user = nullptr;
  hmg_mesh_params mp{};
  hmg_op_params op{};
  hmg::Phys ph{};
  bool assembled = false;
  bool has_theta = false;
  bool fuse_coarse = false;       // hmg_set_coarse_fusion (off: measured slower inside solves)
  std::vector<hmg::Level> lv;
  // Krylov vectors on the finest level (tiled) and a column-layout staging buffer
  double *kx = nullptr, *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr, *kb = nullptr;
  double *kcol = nullptr, *kcol2 = nullptr;
  hmg::Reduce red{};
  double* host_sc = nullptr;      // page-locked copy of the scalars
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void*> allocations;
  std::string err;
  // tracing
  bool prof_on = false;
  unsigned prof_kmask = 0, prof_lmask = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<hmg::ProfRec> prof;
  std::vector<hmg_kernel_stat> prof_agg;          // accumulated records
  bool capturing = false;
  std::vector<hmg::GraphProf> capture_prof;       // events of the graph being captured
  int64_t launches = 0;
  // relative recursive residual after each iteration of the last solve
  std::vector<double> history;
  // CUDA graphs of the Krylov iteration body, one per cycle configuration
  struct BodyGraph {
    int64_t key = -1;
    unsigned long long trace = 0;   // tracing masks the graph was captured with (0: none)
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    int first_kernels = 0;          // device-side CG loop: launches before the while node
    std::vector<hmg::GraphProf> prof;
  };
  std::vector<BodyGraph> graphs;
  cudaStream_t capture_stream = nullptr;  // graphs are captured here, launched on the caller's stream

  // GMRES workspace: basis V (gm_m + 1 vectors) and preconditioned
  // directions Z (gm_m vectors), allocated by the first GMRES solve that
  // needs them; gm_small holds h, h2, hn and the least-squares solution y.
  int gm_m = 0;
  int64_t gm_n = 0;               // entries per basis vector
  double* gm_V = nullptr;
  double* gm_Z = nullptr;
  hmg::GsWork gm{};
  double* gm_y = nullptr;
  double* gm_host = nullptr;      // page-locked copy of gm_small
  // K-part horizontal domain decomposition emulated on this device
  // (hmg_partition): per partitioned level, each part's level view and local
  // vectors, and the halo exchange tables; per part, the landing arrays of
  // the coarsest level's gather and scatter.
  struct PartSet {
    std::vector<hmg::Level> part;              // [part]: owned columns, local neighbours, local work vectors
    std::vector<int32_t> begin;                // [part] first owned column (global)
    int n_send = 0, n_recv = 0;
    int32_t *pack_part = nullptr, *pack_col = nullptr, *unpack_part = nullptr, *unpack_col = nullptr;
    std::vector<int64_t> copy_src, copy_dst, copy_n;   // segment moves between parts, in entries
    void* send64 = nullptr;                    // n_send x nz entries (FP64 and FP32 buffers)
    void* recv64 = nullptr;
    void* send32 = nullptr;
    void* recv32 = nullptr;
  };
  int nparts = 1;
  std::vector<PartSet> psets;                  // [partitioned level]
  std::vector<double*> land_b, land_x;         // [part] coarsest-level landing arrays (FP64)

  // device-side CG loop: its state (device, through the context's allocator)
  // and a page-locked copy read once after the loop
  hmg::CgLoop* cg_loop = nullptr;
  hmg::CgLoop* cg_loop_host = nullptr;

  hmg::MixedSys mx;               // velocity-pressure system, set up by its first use
  hmg::NloSys nlo;                // next-to-lowest-order system, set up by its first use
  hmg::NloMixedSys nlomx;         // next-to-lowest-order velocity-pressure system, set up by its first use
};
