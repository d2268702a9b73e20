// C ABI of the library (include/hmg.h): context life cycle, assembly driver,
// V-cycle driver (Algorithm 1, recursive correction scheme) and the
// preconditioned CG / flexible CG / restarted flexible GMRES loops (Sec. 5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <functional>
#include <new>
#include <string>

#include "hmg_internal.h"

using namespace hmg;

namespace {

std::string g_build_error;

struct Fail {
  hmg_status st;
  std::string msg;
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    throw Fail{HMG_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e)};
  }
  throw Fail{HMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

void launched(const char* what) { cuda_ok(cudaGetLastError(), what); }

// Device memory of a context: the caller's allocator when one was given,
// else cudaMalloc; zero-filled.
void* raw_alloc(hmg_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(bytes, c->alloc_user);
    if (!p) throw Fail{HMG_ERR_OOM, "the caller's allocator returned NULL for " + std::to_string(bytes) + " bytes"};
  } else {
    cuda_ok(cudaMalloc(&p, bytes), "cudaMalloc");
  }
  return p;
}

void raw_free(hmg_ctx* c, void* p) {
  if (c->release_fn) c->release_fn(p, c->alloc_user);
  else cudaFree(p);
}

template <typename T>
T* dalloc(hmg_ctx* c, size_t count) {
  if (count == 0) count = 1;
  void* p = raw_alloc(c, count * sizeof(T));
  c->allocations.push_back(p);
  cuda_ok(cudaMemset(p, 0, count * sizeof(T)), "cudaMemset");
  return static_cast<T*>(p);
}

void dfree(hmg_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
  if (it != c->allocations.end()) c->allocations.erase(it);
  raw_free(c, p);
}

void destroy_graph_prof(std::vector<GraphProf>& v) {
  for (auto& gp : v) {
    if (gp.a) cudaEventDestroy(gp.a);
    if (gp.b) cudaEventDestroy(gp.b);
  }
  v.clear();
}

void release(hmg_ctx* c) {
  for (void* p : c->allocations) raw_free(c, p);
  c->allocations.clear();
  if (c->host_sc) cudaFreeHost(c->host_sc);
  c->host_sc = nullptr;
  if (c->gm_host) cudaFreeHost(c->gm_host);
  c->gm_host = nullptr;
  if (c->cg_loop_host) cudaFreeHost(c->cg_loop_host);
  c->cg_loop_host = nullptr;
  c->cg_loop = nullptr;   // device memory: freed with the allocations
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  c->ev0 = c->ev1 = nullptr;
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    destroy_graph_prof(g.prof);
  }
  c->graphs.clear();
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  c->capture_stream = nullptr;
}

template <typename F>
hmg_status guarded(hmg_ctx* c, F&& f) {
  try {
    f();
    if (c) c->err.clear();
    return HMG_OK;
  } catch (const Fail& e) {
    if (c) c->err = e.msg;
    else g_build_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    else g_build_error = "host allocation failed";
    return HMG_ERR_OOM;
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    else g_build_error = e.what();
    return HMG_ERR_INVALID_ARG;
  }
}

void require(bool ok, const std::string& msg) {
  if (!ok) throw Fail{HMG_ERR_INVALID_ARG, msg};
}

// ------------------------------------------------------------ tracing

cudaEvent_t pool_event(hmg_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cuda_ok(cudaEventCreate(&e), "event");
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

// Returns -1 (not traced), a record index >= 0 (direct launch), or
// -2 - i for event pair i of the graph being captured.
int prof_begin(hmg_ctx* c, int kernel, int level, cudaStream_t s) {
  if (!c->prof_on || !((c->prof_kmask >> kernel) & 1u) || level < 0 || level > 31 ||
      !((c->prof_lmask >> level) & 1u))
    return -1;
  if (c->capturing) {
    GraphProf gp{kernel, level, nullptr, nullptr};
    cuda_ok(cudaEventCreate(&gp.a), "event");
    cuda_ok(cudaEventCreate(&gp.b), "event");
    c->capture_prof.push_back(gp);
    cuda_ok(cudaEventRecordWithFlags(gp.a, s, cudaEventRecordExternal), "event");
    return -2 - ((int)c->capture_prof.size() - 1);
  }
  size_t idx = c->ev_used;
  cudaEvent_t a = pool_event(c);
  pool_event(c);
  cuda_ok(cudaEventRecord(a, s), "event");
  c->prof.push_back(ProfRec{kernel, level, idx});
  return (int)c->prof.size() - 1;
}

void prof_end(hmg_ctx* c, int rec, cudaStream_t s) {
  if (rec == -1) return;
  if (rec <= -2) {
    cuda_ok(cudaEventRecordWithFlags(c->capture_prof[-2 - rec].b, s, cudaEventRecordExternal), "event");
    return;
  }
  cuda_ok(cudaEventRecord(c->ev_pool[c->prof[rec].ev + 1], s), "event");
}

void prof_add(hmg_ctx* c, int kernel, int level, double ms) {
  for (auto& st : c->prof_agg)
    if (st.kernel == kernel && st.level == level) {
      st.launches += 1;
      st.total_ms += ms;
      return;
    }
  c->prof_agg.push_back(hmg_kernel_stat{kernel, level, 1, ms});
}

// Launch `call` (one or more kernels), check the launch, count it and, when
// tracing selects (kernel, level), bracket it with events.
#define LAUNCHN(C, K, LEV, S, NK, CALL)              \
  do {                                               \
    int rec_ = prof_begin((C), (K), (LEV), (S));     \
    CALL;                                            \
    launched(#CALL);                                 \
    prof_end((C), rec_, (S));                        \
    (C)->launches += (NK);                           \
  } while (0)
#define LAUNCH(C, K, LEV, S, CALL) LAUNCHN(C, K, LEV, S, 1, CALL)

// ------------------------------------------------------------ V-cycle driver

struct CycleCfg {
  int nu_pre = 2, nu_post = 2, n_coarse = 2;
  int nlev = 1;          // levels used: 0 .. nlev - 1 (nlev = 1: single-level line relaxation)
  bool mixed = false;
  bool fuse = false;     // coarse end of the cycle as one cooperative kernel
  double omega = 0.8;
};

CycleCfg make_cfg(const hmg_ctx* c, int nu_pre, int nu_post, int n_coarse, int levels, int precision) {
  CycleCfg cfg;
  cfg.nu_pre = nu_pre;
  cfg.nu_post = nu_post;
  cfg.n_coarse = n_coarse;
  cfg.nlev = levels > 0 ? levels : (int)c->lv.size();
  cfg.mixed = precision == HMG_PRECISION_MIXED;
  cfg.omega = c->ph.omega;
  cfg.fuse = c->fuse_coarse;
  return cfg;
}

int level_dt(const hmg_ctx* c, const CycleCfg& cfg, int lev) {
  (void)c;
  return (cfg.mixed && lev < cfg.nlev - 1) ? HMG_FP32 : HMG_FP64;
}

void* work(Level& L, int dt, int which) {
  if (dt == HMG_FP64) return which == 0 ? (void*)L.ua64 : (which == 1 ? (void*)L.ub64 : (void*)L.b64);
  return which == 0 ? (void*)L.ua32 : (which == 1 ? (void*)L.ub32 : (void*)L.b32);
}

// Whether the cycle from level lev down runs as the fused coarse-level
// kernel: lev is below the finest, has at most CC_MAX_TILES tiles, and the
// levels from it down fit the kernel's argument block.
bool fused_from(const hmg_ctx* c, const CycleCfg& cfg, int lev) {
  return cfg.fuse && lev >= 1 && lev < cfg.nlev && c->lv[lev].ncp / TW <= CC_MAX_TILES &&
         cfg.nlev - lev <= CC_MAX_LEVELS;
}

// ------------------------------------------------------------ domain decomposition
//
// A context partitioned into K parts (hmg_partition) runs every level-0
// V-cycle and level-0 FP64 operator application as K parts, as K processes
// would: each pass once per part on the part's owned columns, and every pass
// that reads neighbour columns preceded by a halo exchange (pack, move the
// (sender, receiver) segments, unpack).  The coarsest level is gathered, solved
// once and scattered back.  On one device the moves are device copies; each
// part's passes are the same kernels with the same per-cell arithmetic as the
// unpartitioned cycle.

size_t dt_size(int dt) { return dt == HMG_FP64 ? sizeof(double) : sizeof(float); }

void cycle(hmg_ctx* c, const CycleCfg& cfg, int lev, const void* b, int b_dt, void* out, int out_dt,
           cudaStream_t s, const SweepDot* dot);

void exchange(hmg_ctx* c, int lev, int dt, const PartPtrs& v, cudaStream_t s) {
  hmg_ctx::PartSet& ps = c->psets[lev];
  if (ps.n_send == 0) return;
  const int nz = c->lv[lev].nz;
  void* sb = dt == HMG_FP64 ? ps.send64 : ps.send32;
  void* rb = dt == HMG_FP64 ? ps.recv64 : ps.recv32;
  const size_t es = dt_size(dt) * (size_t)nz;
  LAUNCH(c, HMG_K_HALO, lev, s, launch_halo_pack(ps.n_send, nz, ps.pack_part, ps.pack_col, v, sb, dt, s));
  for (size_t i = 0; i < ps.copy_n.size(); ++i)
    cuda_ok(cudaMemcpyAsync(static_cast<char*>(rb) + ps.copy_dst[i] * es,
                            static_cast<const char*>(sb) + ps.copy_src[i] * es, ps.copy_n[i] * es,
                            cudaMemcpyDeviceToDevice, s),
            "halo move");
  LAUNCH(c, HMG_K_HALO, lev, s, launch_halo_unpack(ps.n_recv, nz, ps.unpack_part, ps.unpack_col, v, rb, dt, s));
}

// The cycle of cycle() on partitioned level lev; b, out: each part's owned
// tiles of the right-hand side and of the result.
void pcycle(hmg_ctx* c, const CycleCfg& cfg, int lev, const PartPtrs& b, int b_dt, const PartPtrs& out,
            int out_dt, cudaStream_t s) {
  hmg_ctx::PartSet& ps = c->psets[lev];
  const int K = c->nparts;
  const int dt = level_dt(c, cfg, lev);
  const bool coarsest = lev == cfg.nlev - 1;
  const int npre = coarsest ? cfg.n_coarse : cfg.nu_pre;
  PartPtrs A{}, B{}, bl{};
  for (int p = 0; p < K; ++p) {
    Level& P = ps.part[p];
    A.p[p] = work(P, dt, 0);
    B.p[p] = work(P, dt, 1);
    float* bcopy = (dt == HMG_FP32 && b_dt == HMG_FP64) ? P.b32 : nullptr;
    bl.p[p] = bcopy ? (void*)bcopy : b.p[p];
    const bool direct = coarsest && npre == 1 && out_dt == dt && !bcopy;
    LAUNCH(c, HMG_K_SWEEP0, lev, s,
           launch_sweep0(P, dt, b.p[p], b_dt, direct ? out.p[p] : A.p[p], bcopy, cfg.omega, s));
  }
  if (coarsest && npre == 1) {
    if (out_dt != dt || dt == HMG_FP32) throw Fail{HMG_ERR_INVALID_ARG, "unsupported coarsest-level configuration"};
    return;
  }
  PartPtrs cur = A, nxt = B;
  for (int i = 1; i < npre; ++i) {
    const bool last = coarsest && i == npre - 1;
    exchange(c, lev, dt, cur, s);
    for (int p = 0; p < K; ++p)
      LAUNCH(c, HMG_K_SWEEP, lev, s,
             launch_sweep(ps.part[p], dt, bl.p[p], cur.p[p], last ? out.p[p] : nxt.p[p], last ? out_dt : dt,
                          nullptr, dt, cfg.omega, nullptr, s));
    if (last) return;
    std::swap(cur, nxt);
  }
  if (coarsest) throw Fail{HMG_ERR_INVALID_ARG, "unsupported coarsest-level configuration"};
  // residual, restricted into the parts of the next level, or into the
  // landing arrays of the gathered coarsest level
  const int cdt = level_dt(c, cfg, lev + 1);
  const bool land = lev + 1 >= (int)c->psets.size();
  PartPtrs bc{}, ec{};
  for (int p = 0; p < K; ++p) {
    if (land) {
      bc.p[p] = c->land_b[p];
      ec.p[p] = c->land_x[p];
    } else {
      Level& Q = c->psets[lev + 1].part[p];
      bc.p[p] = work(Q, cdt, 2);
      ec.p[p] = cdt == HMG_FP64 ? (void*)Q.ux64 : (void*)Q.ux32;
    }
  }
  exchange(c, lev, dt, cur, s);
  for (int p = 0; p < K; ++p)
    LAUNCH(c, HMG_K_RESID_RESTRICT, lev, s,
           launch_resid_restrict(ps.part[p], dt, bl.p[p], cur.p[p], bc.p[p], cdt, s));
  if (land) {
    if (cdt != HMG_FP64) throw Fail{HMG_ERR_INVALID_ARG, "the gathered coarsest level must be FP64"};
    Level& C = c->lv[lev + 1];
    for (int p = 0; p < K; ++p)
      LAUNCH(c, HMG_K_HALO, lev + 1, s,
             launch_copy_cols(ps.part[p].nc / 4, C.nz, c->land_b[p], 0, C.b64, ps.begin[p] / 4, HMG_FP64, s));
    cycle(c, cfg, lev + 1, C.b64, HMG_FP64, C.ux64, HMG_FP64, s, nullptr);
    for (int p = 0; p < K; ++p)
      LAUNCH(c, HMG_K_HALO, lev + 1, s,
             launch_copy_cols(ps.part[p].nc / 4, C.nz, C.ux64, ps.begin[p] / 4, c->land_x[p], 0, HMG_FP64, s));
  } else {
    pcycle(c, cfg, lev + 1, bc, cdt, ec, cdt, s);
  }
  // post-smoothing: the prolonged correction is added by its own pass (the
  // sweeps then read it, with the neighbours' values, after an exchange)
  for (int p = 0; p < K; ++p)
    LAUNCH(c, HMG_K_PROLONG, lev, s, launch_prolong(ps.part[p], dt, cur.p[p], ec.p[p], cdt, s));
  for (int i = 0; i < cfg.nu_post; ++i) {
    const bool last = i == cfg.nu_post - 1;
    exchange(c, lev, dt, cur, s);
    for (int p = 0; p < K; ++p)
      LAUNCH(c, HMG_K_SWEEP, lev, s,
             launch_sweep(ps.part[p], dt, bl.p[p], cur.p[p], last ? out.p[p] : nxt.p[p], last ? out_dt : dt,
                          nullptr, cdt, cfg.omega, nullptr, s));
    std::swap(cur, nxt);
  }
}

// Free the device side of a partition; the graphs hold its pointers, so they go too.
void drop_partition(hmg_ctx* c) {
  for (auto& ps : c->psets) {
    for (Level& P : ps.part)
      for (void* v : {(void*)P.nbr, (void*)P.ua64, (void*)P.ub64, (void*)P.b64, (void*)P.ux64, (void*)P.ua32,
                      (void*)P.ub32, (void*)P.b32, (void*)P.ux32})
        dfree(c, v);
    for (void* v : {(void*)ps.pack_part, (void*)ps.pack_col, (void*)ps.unpack_part, (void*)ps.unpack_col,
                    ps.send64, ps.recv64, ps.send32, ps.recv32})
      dfree(c, v);
  }
  for (double* v : c->land_b) dfree(c, v);
  for (double* v : c->land_x) dfree(c, v);
  c->psets.clear();
  c->land_b.clear();
  c->land_x.clear();
  c->nparts = 1;
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    destroy_graph_prof(g.prof);
  }
  c->graphs.clear();
}

template <typename T>
T* upload(hmg_ctx* c, const std::vector<T>& h) {
  T* d = dalloc<T>(c, h.size());
  if (!h.empty()) cuda_ok(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return d;
}

// The device side of a K-part partition: each part's view of every
// partitioned level (its owned columns of the level's coefficient arrays,
// which are whole tiles, a local neighbour table and local work vectors with
// room for the ghost columns), the exchange tables, and the landing arrays
// of the gathered coarsest level.
void build_partition_dev(hmg_ctx* c, int K) {
  std::vector<std::vector<int32_t>> nbr;
  std::vector<int> ncols;
  for (const Level& L : c->lv) {
    nbr.push_back(L.nbr_host);
    ncols.push_back(L.nc);
  }
  const PartitionPlan plan = build_partition(nbr, ncols, K);
  c->nparts = K;
  c->psets.resize(plan.nlevels);
  for (int l = 0; l < plan.nlevels; ++l) {
    const Level& G = c->lv[l];
    hmg_ctx::PartSet& ps = c->psets[l];
    ps.part.resize(K);
    ps.begin.resize(K);
    std::vector<int32_t> pk_part, pk_col, up_part, up_col;
    std::vector<int64_t> send_off(K + 1, 0), recv_off(K + 1, 0);
    for (int p = 0; p < K; ++p) {
      const PartLevel& pl = plan.lv[l][p];
      send_off[p + 1] = send_off[p] + (int64_t)pl.send_col.size();
      recv_off[p + 1] = recv_off[p] + (int64_t)pl.ghost_col.size();
    }
    for (int p = 0; p < K; ++p) {
      const PartLevel& pl = plan.lv[l][p];
      ps.begin[p] = pl.begin;
      Level& P = ps.part[p];
      P.refinement = G.refinement;
      P.nc = pl.n_own;
      P.ncp = pl.n_own_pad;
      P.nz = G.nz;
      P.twist = G.twist;
      P.twist32 = G.twist32;
      P.N = (int64_t)P.nc * P.nz;
      P.Np = (int64_t)P.ncp * P.nz;
      const int64_t cell0 = (int64_t)pl.begin * G.nz;   // whole tiles: the part's tiles start here
      P.gh = G.gh + pl.begin;
      P.gh32 = G.gh32 + pl.begin;
      P.mt = G.mt + pl.begin;
      P.mts = G.mts + pl.begin;
      P.los = G.los + cell0;
      P.mt32 = G.mt32 + pl.begin;
      P.d = G.d + cell0;
      P.e = G.e + cell0;
      P.lo = G.lo + cell0;
      P.w = G.w + cell0;
      P.d32 = G.d32 + cell0;
      P.e32 = G.e32 + cell0;
      P.lo32 = G.lo32 + cell0;
      P.w32 = G.w32 + cell0;
      std::vector<int4> nb(P.ncp);
      for (int col = 0; col < P.ncp; ++col)
        nb[col] = col < P.nc ? make_int4(pl.local_nbr[3 * col], pl.local_nbr[3 * col + 1], pl.local_nbr[3 * col + 2], 0)
                             : make_int4(col, col, col, 0);
      P.nbr = upload(c, nb);
      const int64_t ghost_tiles = ((int64_t)pl.ghost_col.size() + TW - 1) / TW;
      const int64_t with_ghosts = (P.ncp + ghost_tiles * TW) * P.nz;
      P.ua64 = dalloc<double>(c, with_ghosts);
      P.ub64 = dalloc<double>(c, with_ghosts);
      P.ua32 = dalloc<float>(c, with_ghosts);
      P.ub32 = dalloc<float>(c, with_ghosts);
      P.b64 = dalloc<double>(c, P.Np);
      P.ux64 = dalloc<double>(c, P.Np);
      P.b32 = dalloc<float>(c, P.Np);
      P.ux32 = dalloc<float>(c, P.Np);
      for (size_t i = 0; i < pl.send_col.size(); ++i) {
        pk_part.push_back(p);
        pk_col.push_back(pl.send_col[i] - pl.begin);
      }
      for (size_t i = 0; i < pl.ghost_col.size(); ++i) {
        up_part.push_back(p);
        up_col.push_back(pl.n_own_pad + (int32_t)i);
      }
      // the (p -> q) segments: p's send list is grouped by receiver, q's
      // ghosts by owner, both in q's ghost order
      for (int q = 0; q < K; ++q) {
        if (q == p) continue;
        const auto s0 = std::find(pl.send_to.begin(), pl.send_to.end(), q);
        const int64_t n = std::count(pl.send_to.begin(), pl.send_to.end(), q);
        if (n == 0) continue;
        const PartLevel& ql = plan.lv[l][q];
        const auto g0 = std::find(ql.ghost_owner.begin(), ql.ghost_owner.end(), p);
        ps.copy_src.push_back(send_off[p] + (s0 - pl.send_to.begin()));
        ps.copy_dst.push_back(recv_off[q] + (g0 - ql.ghost_owner.begin()));
        ps.copy_n.push_back(n);
      }
    }
    ps.n_send = (int)pk_part.size();
    ps.n_recv = (int)up_part.size();
    require(ps.n_send == ps.n_recv, "partition: send and receive lists differ in length");
    ps.pack_part = upload(c, pk_part);
    ps.pack_col = upload(c, pk_col);
    ps.unpack_part = upload(c, up_part);
    ps.unpack_col = upload(c, up_col);
    const size_t entries = (size_t)std::max(ps.n_send, 1) * G.nz;
    ps.send64 = dalloc<double>(c, entries);
    ps.recv64 = dalloc<double>(c, entries);
    ps.send32 = dalloc<float>(c, entries);
    ps.recv32 = dalloc<float>(c, entries);
  }
  if (plan.nlevels < (int)c->lv.size()) {   // landing arrays of the gathered coarsest level
    const Level& C = c->lv[plan.nlevels];
    for (int p = 0; p < K; ++p) {
      const int ncl = c->psets.back().part[p].nc / 4;
      const size_t cells = (size_t)((ncl + TW - 1) / TW) * TW * C.nz;
      c->land_b.push_back(dalloc<double>(c, cells));
      c->land_x.push_back(dalloc<double>(c, cells));
    }
  }
}

// Each part's owned tiles of a level-0 tiled vector.
PartPtrs part_slices(const hmg_ctx* c, const void* v, int dt) {
  PartPtrs r{};
  const hmg_ctx::PartSet& ps = c->psets[0];
  for (int p = 0; p < c->nparts; ++p)
    r.p[p] = static_cast<char*>(const_cast<void*>(v)) + (size_t)ps.begin[p] * c->lv[0].nz * dt_size(dt);
  return r;
}

// y = H^ x on level 0 (FP64, tiled), partitioned when the context is; with
// red, x.y is reduced as well (over all parts: the allreduce of the dot).
void apply_fine(hmg_ctx* c, const double* x, double* y, const Reduce* red, cudaStream_t s) {
  Level& L = c->lv[0];
  if (c->nparts <= 1) {
    LAUNCH(c, HMG_K_APPLY, 0, s, launch_apply(L, HMG_FP64, x, y, red, s));
    return;
  }
  hmg_ctx::PartSet& ps = c->psets[0];
  PartPtrs xl{};
  const PartPtrs xs = part_slices(c, x, HMG_FP64), ys = part_slices(c, y, HMG_FP64);
  for (int p = 0; p < c->nparts; ++p) {
    Level& P = ps.part[p];
    xl.p[p] = P.ua64;
    cuda_ok(cudaMemcpyAsync(P.ua64, xs.p[p], (size_t)P.Np * sizeof(double), cudaMemcpyDeviceToDevice, s),
            "part operand");
  }
  exchange(c, 0, HMG_FP64, xl, s);
  for (int p = 0; p < c->nparts; ++p)
    LAUNCH(c, HMG_K_APPLY, 0, s, launch_apply(ps.part[p], HMG_FP64, xl.p[p], ys.p[p], nullptr, s));
  if (red) LAUNCH(c, HMG_K_DOT, 0, s, launch_dot(L, x, y, nullptr, nullptr, *red, s));
}

// out <- V_lev b (zero initial guess).  b has type b_dt, out has type out_dt;
// out must not be one of the level's work buffers ua / ub.  `dot` (optional)
// is fused into the last sweep of this level.
void cycle(hmg_ctx* c, const CycleCfg& cfg, int lev, const void* b, int b_dt, void* out, int out_dt,
           cudaStream_t s, const SweepDot* dot = nullptr) {
  if (lev == 0 && c->nparts > 1) {
    if (dot) throw Fail{HMG_ERR_INVALID_ARG, "a fused dot product is not available on a partitioned cycle"};
    pcycle(c, cfg, 0, part_slices(c, b, b_dt), b_dt, part_slices(c, out, out_dt), out_dt, s);
    return;
  }
  Level& L = c->lv[lev];
  const int nlev = cfg.nlev;
  const int dt = level_dt(c, cfg, lev);
  const bool coarsest = lev == nlev - 1;
  const int npre = coarsest ? cfg.n_coarse : cfg.nu_pre;
  void* A = work(L, dt, 0);
  void* B = work(L, dt, 1);
  float* bcopy = (dt == HMG_FP32 && b_dt == HMG_FP64) ? L.b32 : nullptr;

  if (coarsest && npre == 1 && out_dt == dt && !bcopy && !dot) {
    LAUNCH(c, HMG_K_SWEEP0, lev, s, launch_sweep0(L, dt, b, b_dt, out, nullptr, cfg.omega, s));
    return;
  }
  LAUNCH(c, HMG_K_SWEEP0, lev, s, launch_sweep0(L, dt, b, b_dt, A, bcopy, cfg.omega, s));
  const void* bl = bcopy ? (const void*)bcopy : b;
  void* cur = A;
  void* nxt = B;
  for (int i = 1; i < npre; ++i) {
    bool last = coarsest && i == npre - 1;
    LAUNCH(c, HMG_K_SWEEP, lev, s,
           launch_sweep(L, dt, bl, cur, last ? out : nxt, last ? out_dt : dt, nullptr, dt, cfg.omega,
                        last ? dot : nullptr, s));
    if (last) return;
    std::swap(cur, nxt);
  }
  if (coarsest)  // n_coarse == 1 with a dot or a change of type: not produced by any caller
    throw Fail{HMG_ERR_INVALID_ARG, "unsupported coarsest-level configuration"};
  // residual, restricted to the next coarser level
  Level& C = c->lv[lev + 1];
  const int cdt = level_dt(c, cfg, lev + 1);
  void* bc = work(C, cdt, 2);
  LAUNCH(c, HMG_K_RESID_RESTRICT, lev, s, launch_resid_restrict(L, dt, bl, cur, bc, cdt, s));
  void* ec = cdt == HMG_FP64 ? (void*)C.ux64 : (void*)C.ux32;
  if (fused_from(c, cfg, lev + 1))
    LAUNCH(c, HMG_K_COARSE, lev + 1, s,
           cuda_ok(launch_coarse_cycle(c->lv.data(), lev + 1, nlev, cfg.nu_pre, cfg.nu_post, cfg.n_coarse,
                                       cfg.omega, cfg.mixed, bc, ec, s),
                   "coarse cycle"));
  else
    cycle(c, cfg, lev + 1, bc, cdt, ec, cdt, s);
  // post-smoothing; the coarse correction is added by its own pass first on
  // large FP64 levels (1 instead of 4 FP64 operations per cell) and on small
  // FP32 levels (whose staged sweep takes no fused prolongation), and is
  // prolonged inside the first sweep elsewhere.
  const void* ec_in = ec;
  const bool small = L.ncp / TW <= FUSED_PROLONG_MAX_TILES;
  if ((dt == HMG_FP64 && !small) || (dt == HMG_FP32 && small)) {
    LAUNCH(c, HMG_K_PROLONG, lev, s, launch_prolong(L, dt, cur, ec, cdt, s));
    ec_in = nullptr;
  }
  for (int i = 0; i < cfg.nu_post; ++i) {
    bool last = i == cfg.nu_post - 1;
    LAUNCH(c, HMG_K_SWEEP, lev, s,
           launch_sweep(L, dt, bl, cur, last ? out : nxt, last ? out_dt : dt, i == 0 ? ec_in : nullptr, cdt,
                        cfg.omega, last ? dot : nullptr, s));
    std::swap(cur, nxt);
  }
}

void check_cycle_params(int nu_pre, int nu_post, int n_coarse) {
  require(nu_pre >= 1 && nu_pre <= 64, "nu_pre must be in [1, 64]");
  require(nu_post >= 1 && nu_post <= 64, "nu_post must be in [1, 64]");
  require(n_coarse >= 1 && n_coarse <= 64, "n_coarse must be in [1, 64]");
}

// ------------------------------------------------------------ Krylov driver

void read_scalars(hmg_ctx* c, cudaStream_t s) {
  cuda_ok(cudaMemcpyAsync(c->host_sc, c->red.sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s),
          "scalar read");
  cuda_ok(cudaStreamSynchronize(s), "solve");
}

Reduce red_with(const hmg_ctx* c, int epi, int slot = 0) {
  Reduce r = c->red;
  r.epilogue = epi;
  r.slot = slot;
  return r;
}

// One Krylov iteration after the first: z = V r, beta (device), p = z + beta p,
// q = H^ p with alpha (device), x += alpha p, r -= alpha q with r.r, and the
// scalars copied to page-locked host memory.
// The dots r.z (and z.q) that form beta are fused into the last sweep of the
// V-cycle when it has one (nu_post >= 1 always, so it does).
SweepDot beta_dot(const hmg_ctx* c, bool flexible) {
  SweepDot d;
  d.a = c->kr;
  d.c = flexible ? c->kq : nullptr;
  d.red = red_with(c, flexible ? EPI_BETA_FCG : EPI_BETA_CG);
  return d;
}

// Whether the beta dots ride on the V-cycle's last sweep: the FP64 cycle with
// a last sweep (not a lone sweep0); the FP32 register sweeps take no dots
// (holding their outputs for the dots costs the registers that let the
// column recurrence run ahead of its loads).
bool fused_beta(const hmg_ctx* c, const CycleCfg& cfg) {
  return !cfg.mixed && (cfg.nlev > 1 || cfg.n_coarse > 1) && c->nparts <= 1;
}

void iteration_body(hmg_ctx* c, const CycleCfg& cfg, bool flexible, cudaStream_t s, bool read_back = true) {
  Level& L = c->lv[0];
  if (fused_beta(c, cfg)) {
    SweepDot d = beta_dot(c, flexible);
    cycle(c, cfg, 0, c->kr, HMG_FP64, c->kz, HMG_FP64, s, &d);
  } else {
    cycle(c, cfg, 0, c->kr, HMG_FP64, c->kz, HMG_FP64, s);
    LAUNCH(c, HMG_K_DOT, 0, s,
           launch_dot(L, c->kr, c->kz, flexible ? c->kz : nullptr, c->kq,
                      red_with(c, flexible ? EPI_BETA_FCG : EPI_BETA_CG), s));
  }
  LAUNCH(c, HMG_K_UPDATE_P, 0, s, launch_update_p(L, c->kp, c->kz, c->red.sc, s));
  Reduce ra = red_with(c, EPI_ALPHA);
  apply_fine(c, c->kp, c->kq, &ra, s);
  LAUNCH(c, HMG_K_UPDATE_XR, 0, s, launch_update_xr(L, c->kx, c->kr, c->kp, c->kq, red_with(c, EPI_RR), s));
  if (read_back)
    cuda_ok(cudaMemcpyAsync(c->host_sc, c->red.sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s),
            "scalar read");
}

// Graph keys: the cycle configuration, the Krylov method and, for GMRES, the
// Arnoldi step j within a restart cycle (its vectors are baked in).
int64_t graph_key(const CycleCfg& cfg, bool flexible, int gmres_step = -1) {
  const int64_t base =
      ((((((cfg.fuse ? 1 : 0) * 2 + (cfg.mixed ? 1 : 0)) * 2 + (flexible ? 1 : 0)) * 65 + cfg.nu_pre) * 65 +
        cfg.nu_post) * 65 + cfg.n_coarse) * 33 + cfg.nlev;
  return base * (GMRES_MAX_RESTART + 1) + (gmres_step + 1);
}

// Replay (capturing it the first time) the iteration body as a CUDA graph.
// With tracing on, the graph carries event nodes around the traced kernels;
// harvest_body() reads them after the replay has completed.
template <typename Body>
hmg_ctx::BodyGraph* run_graph(hmg_ctx* c, int64_t key, Body&& body, cudaStream_t s) {
  const unsigned long long trace =
      c->prof_on ? (((unsigned long long)c->prof_kmask << 32) | c->prof_lmask) | (1ull << 63) : 0ull;
  hmg_ctx::BodyGraph* g = nullptr;
  for (auto& bg : c->graphs)
    if (bg.key == key && bg.trace == trace) g = &bg;
  if (!g) {
    cudaGraph_t graph = nullptr;
    const int64_t before = c->launches;
    cudaStream_t cs = c->capture_stream;
    c->capture_prof.clear();
    cuda_ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    c->capturing = true;
    try {
      body(cs);
    } catch (...) {
      c->capturing = false;
      cudaStreamEndCapture(cs, &graph);
      if (graph) cudaGraphDestroy(graph);
      destroy_graph_prof(c->capture_prof);
      throw;
    }
    c->capturing = false;
    cuda_ok(cudaStreamEndCapture(cs, &graph), "end capture");
    hmg_ctx::BodyGraph bg;
    bg.key = key;
    bg.trace = trace;
    bg.kernels = (int)(c->launches - before);
    bg.prof.swap(c->capture_prof);
    c->launches = before;
    cudaError_t e = cudaGraphInstantiate(&bg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) destroy_graph_prof(bg.prof);
    cuda_ok(e, "graph instantiate");
    c->graphs.push_back(std::move(bg));
    g = &c->graphs.back();
  }
  cuda_ok(cudaGraphLaunch(g->exec, s), "graph launch");
  c->launches += g->kernels;
  return g;
}

hmg_ctx::BodyGraph* run_body(hmg_ctx* c, const CycleCfg& cfg, bool flexible, cudaStream_t s) {
  return run_graph(c, graph_key(cfg, flexible), [&](cudaStream_t cs) { iteration_body(c, cfg, flexible, cs); }, s);
}

// After the replay of g has completed: add its traced kernels to the records.
void harvest_body(hmg_ctx* c, const hmg_ctx::BodyGraph* g) {
  if (!c->prof_on || !g) return;
  for (const GraphProf& gp : g->prof) {
    float ms = 0.f;
    cuda_ok(cudaEventElapsedTime(&ms, gp.a, gp.b), "event time");
    prof_add(c, gp.kernel, gp.level, ms);
  }
}

// The first CG iteration: z = V r with r.z, p = z, q = H^ p with alpha,
// x += alpha p, r -= alpha q with r.r.
void first_iteration(hmg_ctx* c, const CycleCfg& cfg, cudaStream_t s) {
  Level& L = c->lv[0];
  if (fused_beta(c, cfg)) {
    SweepDot d;
    d.a = c->kr;
    d.red = red_with(c, EPI_INIT_RZ);
    cycle(c, cfg, 0, c->kr, HMG_FP64, c->kz, HMG_FP64, s, &d);
  } else {
    cycle(c, cfg, 0, c->kr, HMG_FP64, c->kz, HMG_FP64, s);
    LAUNCH(c, HMG_K_DOT, 0, s, launch_dot(L, c->kr, c->kz, nullptr, nullptr, red_with(c, EPI_INIT_RZ), s));
  }
  cuda_ok(cudaMemcpyAsync(c->kp, c->kz, (size_t)L.Np * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  Reduce ra = red_with(c, EPI_ALPHA);
  apply_fine(c, c->kp, c->kq, &ra, s);
  LAUNCH(c, HMG_K_UPDATE_XR, 0, s, launch_update_xr(L, c->kx, c->kr, c->kp, c->kq, red_with(c, EPI_RR), s));
}

// The CG iterations as one CUDA graph: the first iteration, a stopping-test
// kernel (k_cg_control), then a while node whose body is one iteration
// followed by the same test, so the whole loop runs without the host.  The
// test sets the node's condition; it ends the loop at max_iter at the
// latest, so the graph always terminates.  Graphs with a conditional node
// cannot hold event nodes, so traced solves take the host-side loop.
hmg_ctx::BodyGraph* run_loop(hmg_ctx* c, const CycleCfg& cfg, bool flexible, cudaStream_t s) {
  const int64_t key = graph_key(cfg, flexible) + (int64_t(1) << 60);
  hmg_ctx::BodyGraph* g = nullptr;
  for (auto& bg : c->graphs)
    if (bg.key == key && bg.trace == 0) g = &bg;
  if (!g) {
    if (!c->cg_loop) c->cg_loop = dalloc<CgLoop>(c, 1);
    cudaStream_t cs = c->capture_stream;
    cudaGraph_t graph = nullptr;
    cuda_ok(cudaGraphCreate(&graph, 0), "graph create");
    int body_kernels = 0, first_kernels = 0;
    try {
      cudaGraphConditionalHandle hnd;
      cuda_ok(cudaGraphConditionalHandleCreate(&hnd, graph, 0, cudaGraphCondAssignDefault), "conditional handle");
      // the first iteration and the first test, then the while node after them
      cudaGraph_t body = nullptr;
      const int64_t before0 = c->launches;
      cuda_ok(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
              "begin capture");
      c->capturing = true;
      try {
        first_iteration(c, cfg, cs);
        launch_cg_control(c->cg_loop, c->red.sc, hnd, cs);
        launched("k_cg_control");
        c->launches += 1;
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cuda_ok(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps), "capture info");
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hnd;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode = nullptr;
        cuda_ok(cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &np), "while node");
        cuda_ok(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies),
                "capture dependencies");
        body = np.conditional.phGraph_out[0];
      } catch (...) {
        c->capturing = false;
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(cs, &dummy);
        c->launches = before0;
        throw;
      }
      c->capturing = false;
      first_kernels = (int)(c->launches - before0);
      c->launches = before0;
      cudaGraph_t same = nullptr;
      cuda_ok(cudaStreamEndCapture(cs, &same), "end capture");
      const int64_t before = c->launches;
      cuda_ok(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
              "begin capture");
      c->capturing = true;
      try {
        iteration_body(c, cfg, flexible, cs, false);
        launch_cg_control(c->cg_loop, c->red.sc, hnd, cs);
        launched("k_cg_control");
        c->launches += 1;
      } catch (...) {
        c->capturing = false;
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(cs, &dummy);
        c->launches = before;
        throw;
      }
      c->capturing = false;
      body_kernels = (int)(c->launches - before);
      c->launches = before;
      cudaGraph_t body_same = nullptr;
      cuda_ok(cudaStreamEndCapture(cs, &body_same), "end capture");
    } catch (...) {
      cudaGraphDestroy(graph);
      throw;
    }
    hmg_ctx::BodyGraph bg;
    bg.key = key;
    bg.trace = 0;
    bg.kernels = body_kernels;
    bg.first_kernels = first_kernels;
    cudaError_t e = cudaGraphInstantiate(&bg.exec, graph, 0);
    cudaGraphDestroy(graph);
    cuda_ok(e, "graph instantiate");
    c->graphs.push_back(std::move(bg));
    g = &c->graphs.back();
  }
  cuda_ok(cudaGraphLaunch(g->exec, s), "graph launch");
  return g;
}

hmg_status solve_gmres(hmg_ctx* c, const hmg_solve_params& p, hmg_solve_info* info, cudaStream_t s);

// The solve on the tiled vectors kb (right-hand side) and kx (solution).
hmg_status solve_tiled(hmg_ctx* c, const hmg_solve_params& p, hmg_solve_info* info, cudaStream_t s) {
  if (p.krylov == HMG_KRYLOV_GMRES) return solve_gmres(c, p, info, s);
  Level& L = c->lv[0];
  const CycleCfg cfg = make_cfg(c, p.nu_pre, p.nu_post, p.n_coarse, p.levels, p.precision);
  const bool flexible = cfg.mixed || p.krylov == HMG_KRYLOV_FCG;
  const size_t bytes = (size_t)L.Np * sizeof(double);
  hmg_solve_info inf{};
  c->history.clear();

  cuda_ok(cudaEventRecord(c->ev0, s), "event");
  cuda_ok(cudaMemsetAsync(c->red.sc, 0, S_COUNT * sizeof(double), s), "memset");
  cuda_ok(cudaMemsetAsync(c->kx, 0, bytes, s), "memset");
  cuda_ok(cudaMemcpyAsync(c->kr, c->kb, bytes, cudaMemcpyDeviceToDevice, s), "copy");
  LAUNCH(c, HMG_K_DOT, 0, s, launch_dot(L, c->kr, c->kr, nullptr, nullptr, red_with(c, EPI_STORE0, S_BB), s));
  read_scalars(c, s);
  const double bb = c->host_sc[S_BB];
  if (((int)c->host_sc[S_FLAG] & F_NONFINITE) || !std::isfinite(bb)) {
    if (info) *info = inf;
    throw Fail{HMG_ERR_NONFINITE, "right-hand side is not finite"};
  }
  hmg_status st = HMG_ERR_NOT_CONVERGED;
  hmg_ctx::BodyGraph* loop_graph = nullptr;   // set when the device-side loop ran
  if (bb == 0.0) {
    inf.converged = 1;
    st = HMG_OK;
  } else {
    const double stop2 = p.rtol * p.rtol * bb;
    if (!c->prof_on && p.max_iter <= CG_LOOP_HIST) {
      // device-side loop: one graph launch; its state is read with the
      // true residual's scalars at the end
      if (!c->cg_loop_host)
        cuda_ok(cudaHostAlloc((void**)&c->cg_loop_host, sizeof(CgLoop), cudaHostAllocDefault), "host alloc");
      if (!c->cg_loop) c->cg_loop = dalloc<CgLoop>(c, 1);
      launch_cg_loop_init(c->cg_loop, p.rtol * p.rtol, p.max_iter, s);
      launched("k_cg_loop_init");
      c->launches += 1;
      loop_graph = run_loop(c, cfg, flexible, s);
      cuda_ok(cudaMemcpyAsync(c->cg_loop_host, c->cg_loop, sizeof(CgLoop), cudaMemcpyDeviceToHost, s), "loop read");
    } else {
      first_iteration(c, cfg, s);
      read_scalars(c, s);
      for (int k = 1;; ++k) {
        inf.iterations = k;
        const int flag = (int)c->host_sc[S_FLAG];
        const double rr = c->host_sc[S_RR];
        inf.rel_residual = std::sqrt(rr / bb);
        c->history.push_back(inf.rel_residual);
        if (flag & F_NONFINITE) {
          st = HMG_ERR_NONFINITE;
          break;
        }
        if (flag & F_BREAKDOWN) {
          st = HMG_ERR_BREAKDOWN;
          break;
        }
        if (rr < stop2) {
          inf.converged = 1;
          st = HMG_OK;
          break;
        }
        if (k == p.max_iter) break;
        hmg_ctx::BodyGraph* g = run_body(c, cfg, flexible, s);
        cuda_ok(cudaStreamSynchronize(s), "solve");
        harvest_body(c, g);
      }
    }
  }
  // true residual ||b - H^ x|| / ||b||
  apply_fine(c, c->kx, c->kq, nullptr, s);
  LAUNCH(c, HMG_K_RESID_SQ, 0, s, launch_resid_sq(L, c->kb, c->kq, red_with(c, EPI_STORE0, S_TRUE), s));
  cuda_ok(cudaEventRecord(c->ev1, s), "event");
  read_scalars(c, s);
  if (loop_graph) {
    const CgLoop& lh = *c->cg_loop_host;
    const int k = lh.k;
    if (k < 1 || k > p.max_iter) throw Fail{HMG_ERR_CUDA, "device loop returned an invalid iteration count"};
    c->launches += loop_graph->first_kernels + (int64_t)(k - 1) * loop_graph->kernels;
    inf.iterations = k;
    c->history.assign(lh.hist, lh.hist + k);
    inf.rel_residual = c->history.back();
    if (lh.flag & F_NONFINITE) st = HMG_ERR_NONFINITE;
    else if (lh.flag & F_BREAKDOWN) st = HMG_ERR_BREAKDOWN;
    else if (lh.rr < p.rtol * p.rtol * bb) {
      inf.converged = 1;
      st = HMG_OK;
    }
  }
  inf.true_rel_residual = bb > 0 ? std::sqrt(c->host_sc[S_TRUE] / bb) : 0.0;
  float ms = 0.f;
  cuda_ok(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "event time");
  inf.solve_ms = ms;
  if (info) *info = inf;
  return st;
}

// ------------------------------------------------------------ GMRES

// Offsets in gm_small (device) and gm_host (page-locked): the step results
// h, h2 (with |w|^2 after them) and hn are read back together; y is staged.
constexpr int GM_H = 0, GM_H2 = GMRES_MAX_RESTART, GM_HN = 2 * GMRES_MAX_RESTART + 1, GM_READ = GM_HN + 1,
              GM_Y = 3 * GMRES_MAX_RESTART, GM_SMALL = 4 * GMRES_MAX_RESTART;

// Basis storage for restart length m on vectors of n entries (kept across
// solves; a longer restart or longer vectors reallocate it and drop the
// graphs that hold the old vectors).
void ensure_gmres(hmg_ctx* c, int m, int64_t n) {
  if (!c->gm_host) {
    double* small = dalloc<double>(c, GM_SMALL);
    c->gm.h = small + GM_H;
    c->gm.h2 = small + GM_H2;
    c->gm.hn = small + GM_HN;
    c->gm_y = small + GM_Y;
    c->gm.part = dalloc<double>(c, (size_t)(GMRES_MAX_RESTART + 1) * GS_MAX_BLOCKS);
    c->gm.counter = dalloc<unsigned int>(c, 1);
    cuda_ok(cudaMallocHost(&c->gm_host, GM_SMALL * sizeof(double)), "cudaMallocHost");
  }
  if (m <= c->gm_m && n <= c->gm_n) return;
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    destroy_graph_prof(g.prof);
  }
  c->graphs.clear();
  dfree(c, c->gm_V);
  dfree(c, c->gm_Z);
  c->gm_V = c->gm_Z = nullptr;
  const int mm = std::max(m, c->gm_m);
  const int64_t nn = std::max(n, c->gm_n);
  c->gm_m = 0;
  c->gm_n = 0;
  c->gm_V = dalloc<double>(c, (size_t)(mm + 1) * nn);
  c->gm_Z = dalloc<double>(c, (size_t)mm * nn);
  c->gm_m = mm;
  c->gm_n = nn;
}

// A linear system for the GMRES driver: n entries per vector (tiled layouts,
// padding entries zero), the right-hand side b and the iterate x (device),
// y = A x and z = P^-1 r launched on a stream, and the graph key of its
// first Arnoldi step (step j uses key + j; the top bits name the system).
struct KrylovSystem {
  int64_t n = 0;
  const double* b = nullptr;
  double* x = nullptr;
  double* tmp = nullptr;      // n entries of scratch
  std::function<void(const double*, double*, cudaStream_t)> apply;
  std::function<void(const double*, double*, cudaStream_t)> precond;
  int64_t key = 0;
  int orth = 1;               // classical Gram-Schmidt passes: 1 or 2
};

// Arnoldi step j: z_j = P^-1 v_j, w = A z_j into v_(j+1), two Gram-Schmidt
// passes against v_0..v_j and the normalisation, results copied to the host.
void gmres_step(hmg_ctx* c, const KrylovSystem& sys, int j, cudaStream_t s) {
  const int64_t ld = sys.n;
  double* vj = c->gm_V + j * ld;
  double* zj = c->gm_Z + j * ld;
  double* w = c->gm_V + (j + 1) * ld;
  sys.precond(vj, zj, s);
  sys.apply(zj, w, s);
  const int nd2 = sys.orth == 2 ? j + 1 : 0;
  LAUNCH(c, HMG_K_ORTHO, 0, s, launch_gs_dots(ld, c->gm_V, ld, j + 1, w, c->gm, s));
  LAUNCH(c, HMG_K_ORTHO, 0, s, launch_gs_update(ld, c->gm_V, ld, j + 1, nd2 > 0, w, c->gm, s));
  LAUNCH(c, HMG_K_ORTHO, 0, s, launch_gs_final(ld, c->gm_V, ld, nd2, w, c->gm, s));
  cuda_ok(cudaMemcpyAsync(c->gm_host, c->gm.h, GM_READ * sizeof(double), cudaMemcpyDeviceToHost, s),
          "GMRES read");
}

// Restarted flexible GMRES(m) with right preconditioning on `sys`, x_0 = 0.
hmg_status gmres_run(hmg_ctx* c, const KrylovSystem& sys, const hmg_solve_params& p, hmg_solve_info* info,
                     cudaStream_t s) {
  const int m = p.restart;
  const int64_t ld = sys.n;
  ensure_gmres(c, m, ld);
  hmg_solve_info inf{};
  c->history.clear();

  cuda_ok(cudaEventRecord(c->ev0, s), "event");
  cuda_ok(cudaMemsetAsync(c->red.sc, 0, S_COUNT * sizeof(double), s), "memset");
  cuda_ok(cudaMemsetAsync(sys.x, 0, (size_t)ld * sizeof(double), s), "memset");
  LAUNCH(c, HMG_K_DOT, 0, s, launch_dot_n(ld, sys.b, sys.b, red_with(c, EPI_STORE0, S_BB), s));
  read_scalars(c, s);
  const double bb = c->host_sc[S_BB];
  if (((int)c->host_sc[S_FLAG] & F_NONFINITE) || !std::isfinite(bb)) {
    if (info) *info = inf;
    throw Fail{HMG_ERR_NONFINITE, "right-hand side is not finite"};
  }
  hmg_status st = HMG_ERR_NOT_CONVERGED;
  if (bb == 0.0) {
    inf.converged = 1;
    st = HMG_OK;
  } else {
    const double r0 = std::sqrt(bb);
    LAUNCH(c, HMG_K_ORTHO, 0, s, launch_normalise(ld, sys.b, c->gm_V, c->red.sc + S_BB, s));
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    double beta = r0;
    int k = 0;
    bool stop = false;
    while (!stop) {
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jend = 0;
      for (int j = 0; j < m; ++j) {
        hmg_ctx::BodyGraph* gr =
            run_graph(c, sys.key + j, [&](cudaStream_t cs) { gmres_step(c, sys, j, cs); }, s);
        cuda_ok(cudaStreamSynchronize(s), "solve");
        harvest_body(c, gr);
        const double* hh = c->gm_host;
        const int nd2 = sys.orth == 2 ? j + 1 : 0;
        bool finite = std::isfinite(hh[GM_HN]) && std::isfinite(hh[GM_H2 + nd2]);
        for (int i = 0; i <= j; ++i) {
          Hij(i, j) = hh[GM_H + i] + (i < nd2 ? hh[GM_H2 + i] : 0.0);
          finite = finite && std::isfinite(Hij(i, j));
        }
        Hij(j + 1, j) = hh[GM_HN];
        if (!finite) {
          st = HMG_ERR_NONFINITE;
          stop = true;
          break;
        }
        for (int i = 0; i < j; ++i) {  // earlier rotations on column j
          const double a = Hij(i, j), bv = Hij(i + 1, j);
          Hij(i, j) = cs[i] * a + sn[i] * bv;
          Hij(i + 1, j) = -sn[i] * a + cs[i] * bv;
        }
        const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
        if (!(den > 0.0)) {
          st = HMG_ERR_BREAKDOWN;
          stop = true;
          break;
        }
        cs[j] = Hij(j, j) / den;
        sn[j] = Hij(j + 1, j) / den;
        Hij(j, j) = den;
        Hij(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++k;
        jend = j + 1;
        inf.iterations = k;
        inf.rel_residual = std::fabs(g[j + 1]) / r0;
        c->history.push_back(inf.rel_residual);
        if (inf.rel_residual < p.rtol) {
          inf.converged = 1;
          st = HMG_OK;
          stop = true;
          break;
        }
        if (k >= p.max_iter) {
          stop = true;
          break;
        }
      }
      if (jend > 0) {  // y = R^-1 g; x += Z y
        for (int i = jend - 1; i >= 0; --i) {
          double t = g[i];
          for (int l = i + 1; l < jend; ++l) t -= Hij(i, l) * y[l];
          y[i] = t / Hij(i, i);
        }
        std::copy(y.begin(), y.begin() + jend, c->gm_host + GM_Y);
        cuda_ok(cudaMemcpyAsync(c->gm_y, c->gm_host + GM_Y, jend * sizeof(double), cudaMemcpyHostToDevice, s),
                "GMRES y");
        LAUNCH(c, HMG_K_ORTHO, 0, s, launch_gmres_x(ld, sys.x, c->gm_Z, ld, jend, c->gm_y, s));
      }
      if (stop) break;
      // restart from the residual of the new iterate: v_0 = (b - A x) / beta
      sys.apply(sys.x, sys.tmp, s);
      LAUNCH(c, HMG_K_ORTHO, 0, s, launch_sub_norm(ld, sys.b, sys.tmp, c->gm_V, red_with(c, EPI_STORE0, S_RR), s));
      read_scalars(c, s);
      const double rr = c->host_sc[S_RR];
      if (!std::isfinite(rr)) {
        st = HMG_ERR_NONFINITE;
        break;
      }
      if (rr == 0.0) {  // exact solution
        inf.converged = 1;
        inf.rel_residual = 0.0;
        st = HMG_OK;
        break;
      }
      beta = std::sqrt(rr);
      LAUNCH(c, HMG_K_ORTHO, 0, s, launch_normalise(ld, c->gm_V, c->gm_V, c->red.sc + S_RR, s));
    }
  }
  // true residual ||b - A x|| / ||b||
  sys.apply(sys.x, sys.tmp, s);
  LAUNCH(c, HMG_K_RESID_SQ, 0, s, launch_sub_norm(ld, sys.b, sys.tmp, sys.tmp, red_with(c, EPI_STORE0, S_TRUE), s));
  cuda_ok(cudaEventRecord(c->ev1, s), "event");
  read_scalars(c, s);
  inf.true_rel_residual = bb > 0 ? std::sqrt(c->host_sc[S_TRUE] / bb) : 0.0;
  float ms = 0.f;
  cuda_ok(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "event time");
  inf.solve_ms = ms;
  if (info) *info = inf;
  return st;
}

// GMRES(m) on H^ x = b (tiled kb, kx), preconditioned by the V-cycle.
hmg_status solve_gmres(hmg_ctx* c, const hmg_solve_params& p, hmg_solve_info* info, cudaStream_t s) {
  Level& L = c->lv[0];
  const CycleCfg cfg = make_cfg(c, p.nu_pre, p.nu_post, p.n_coarse, p.levels, p.precision);
  KrylovSystem sys;
  sys.n = L.Np;
  sys.b = c->kb;
  sys.x = c->kx;
  sys.tmp = c->kq;
  sys.apply = [c](const double* x, double* y, cudaStream_t st) {
    apply_fine(c, x, y, nullptr, st);
  };
  sys.precond = [c, cfg](const double* r, double* z, cudaStream_t st) {
    cycle(c, cfg, 0, r, HMG_FP64, z, HMG_FP64, st);
  };
  sys.orth = p.orth == 2 ? 2 : 1;
  sys.key = (1LL << 60) + (sys.orth == 2 ? (1LL << 59) : 0) + graph_key(cfg, true, 0);
  return gmres_run(c, sys, p, info, s);
}

// ------------------------------------------------------------ velocity-pressure system

// Edge list (t, k, tn, kn with t < tn, ordered by t then k), per-column edge
// table and the coefficient arrays of the finest level; built on first use.
void mixed_edges_host(hmg_ctx* c, std::vector<int4>* cedge_out) {
  MixedSys& M = c->mx;
  const Level& L = c->lv[0];
  const std::vector<int32_t>& nbr = L.nbr_host;
  std::vector<int32_t> edges;
  std::vector<int4> cedge(L.ncp, make_int4(0, 0, 0, 0));
  for (int t = 0; t < L.nc; ++t)
    for (int k = 0; k < 3; ++k) {
      const int tn = nbr[3 * t + k];
      if (t < tn) {
        int kn = 0;
        while (kn < 3 && nbr[3 * tn + kn] != t) ++kn;
        require(kn < 3, "mesh neighbours are not symmetric");
        const int e = (int)(edges.size() / 4);
        edges.insert(edges.end(), {t, k, tn, kn});
        int* ct = &cedge[t].x;
        ct[k] = e;
        int* cn = &cedge[tn].x;
        cn[kn] = e;
        cedge[tn].w |= 1 << kn;   // -1 on the higher-numbered column
      }
    }
  M.ne = (int)(edges.size() / 4);
  M.nep = (M.ne + TW - 1) / TW * TW;
  M.nh = (int64_t)M.nep * L.nz;
  M.n = M.nh + 2 * L.Np;
  M.edges_host = edges;
  if (cedge_out) cedge_out->swap(cedge);
}

void ensure_mixed(hmg_ctx* c, cudaStream_t s) {
  MixedSys& M = c->mx;
  if (M.ready) return;
  const Level& L = c->lv[0];
  std::vector<int4> cedge;
  mixed_edges_host(c, &cedge);
  const std::vector<int32_t>& edges = M.edges_host;
  std::vector<int4> ed(M.nep, make_int4(0, 0, 0, 0));
  for (int e = 0; e < M.ne; ++e) ed[e] = make_int4(edges[4 * e], edges[4 * e + 1], edges[4 * e + 2], edges[4 * e + 3]);
  M.edge = dalloc<int4>(c, M.nep);
  M.enb = dalloc<int4>(c, M.nep);
  M.ecoef = dalloc<double4_32a>(c, M.nep);
  M.emass = dalloc<double>(c, M.nep);
  M.einv = dalloc<double>(c, M.nep);
  M.cedge = dalloc<int4>(c, L.ncp);
  M.zd = dalloc<double>(c, L.Np);
  M.m3 = dalloc<double>(c, L.Np);
  M.zsi = dalloc<double>(c, L.Np);
  M.b = dalloc<double>(c, M.n);
  M.x = dalloc<double>(c, M.n);
  M.t1 = dalloc<double>(c, M.n);
  M.t2 = dalloc<double>(c, M.n);
  cuda_ok(cudaMemcpy(M.edge, ed.data(), ed.size() * sizeof(int4), cudaMemcpyHostToDevice), "upload");
  cuda_ok(cudaMemcpy(M.cedge, cedge.data(), cedge.size() * sizeof(int4), cudaMemcpyHostToDevice), "upload");
  Phys geo;   // geometry only: the coefficients do not depend on the operator parameters
  geo.R = c->mp.radius_m;
  geo.dz = c->mp.thickness_m / c->mp.nlayers;
  LAUNCHN(c, HMG_K_ASSEMBLY, 0, s, 2, launch_mixed_coeffs(L, M, geo, s));
  cuda_ok(cudaStreamSynchronize(s), "mixed setup");
  M.ready = true;
}

// GMRES(m) on the velocity-pressure system (tiled mx.b, mx.x) with the
// Schur-complement preconditioner; H^^-1 is one V-cycle of the given form.
hmg_status solve_mixed_tiled(hmg_ctx* c, const hmg_solve_params& p, hmg_solve_info* info, cudaStream_t s) {
  Level& L = c->lv[0];
  MixedSys& M = c->mx;
  const CycleCfg cfg = make_cfg(c, p.nu_pre, p.nu_post, p.n_coarse, p.levels, p.precision);
  const int64_t off_p = M.nh + L.Np;   // cell part of a vector
  KrylovSystem sys;
  sys.n = M.n;
  sys.b = M.b;
  sys.x = M.x;
  sys.tmp = M.t1;
  sys.apply = [c, &L, &M](const double* x, double* y, cudaStream_t st) {
    LAUNCHN(c, HMG_K_APPLY, 0, st, 2, launch_mixed_apply(L, M, c->ph, x, y, st));
  };
  sys.precond = [c, &L, &M, cfg, off_p](const double* r, double* z, cudaStream_t st) {
    LAUNCH(c, HMG_K_ORTHO, 0, st, launch_mixed_pre_lower(L, M, c->ph, r, M.t2, st));
    cycle(c, cfg, 0, M.t2, HMG_FP64, z + off_p, HMG_FP64, st);
    LAUNCHN(c, HMG_K_ORTHO, 0, st, 2, launch_mixed_pre_upper(L, M, c->ph, r, z, st));
  };
  sys.orth = p.orth == 2 ? 2 : 1;
  sys.key = (2LL << 60) + (sys.orth == 2 ? (1LL << 59) : 0) + graph_key(cfg, true, 0);
  return gmres_run(c, sys, p, info, s);
}

// ------------------------------------------------------------ next-to-lowest order

Phys make_phys(const hmg_mesh_params& mp, const hmg_op_params& p) {
  const double dx = p.dx_m > 0 ? p.dx_m : 90.0e3 * std::ldexp(1.0, 6 - mp.refinement);
  const double dt = p.nu_cfl * dx / p.c;
  const double wc = 0.5 * p.c * dt, wn = 0.5 * p.N * dt;
  Phys ph;
  ph.R = mp.radius_m;
  ph.dz = mp.thickness_m / mp.nlayers;
  ph.wc2 = wc * wc;
  ph.vfac = wc * wc / (1.0 + wn * wn);
  ph.omega = p.omega;
  ph.a = 0.5 * dt;
  ph.c2 = p.c * p.c;
  ph.wn2 = wn * wn;
  return ph;
}

void check_op_params(const hmg_op_params* p) {
  require(p != nullptr, "params is NULL");
  require(p->c > 0 && std::isfinite(p->c), "c must be positive");
  require(p->N >= 0 && std::isfinite(p->N), "N must be >= 0");
  require(p->nu_cfl > 0 && std::isfinite(p->nu_cfl), "nu_cfl must be positive");
  require(p->omega > 0 && p->omega < 2, "omega must be in (0, 2)");
}

// Coefficient tables of the NLO level for the current assembly (host
// assembly and factorisation, one upload).
void ensure_nlo(hmg_ctx* c) {
  NloSys& X = c->nlo;
  if (X.ready) return;
  const Level& L = c->lv[0];
  require(L.nc % NLO_TILE == 0, "NLO needs a multiple of 5 columns");
  if (!X.allocated) {
    X.nt = L.nc / NLO_TILE;
    X.n = (int64_t)X.nt * L.nz * 32;
    const size_t cw = (size_t)X.n * 6;
    X.Ad = dalloc<double>(c, cw);
    X.Cs = dalloc<double>(c, cw);
    X.Cu = dalloc<double>(c, cw);
    X.Lf = dalloc<double>(c, cw);
    X.Di = dalloc<double>(c, cw);
    X.Lb = dalloc<double>(c, cw);
    X.Nb = dalloc<double>(c, (size_t)X.nt * 3 * 3 * 32);
    X.nb = dalloc<int>(c, (size_t)X.nt * 3 * 32);
    for (double** v : {&X.b, &X.x, &X.t1, &X.t2, &X.w, &X.ua, &X.ub}) *v = dalloc<double>(c, X.n);
    for (float** v : {&X.Ad32, &X.Cs32, &X.Cu32, &X.Lf32, &X.Di32, &X.Lb32}) *v = dalloc<float>(c, cw);
    X.Nb32 = dalloc<float>(c, (size_t)X.nt * 3 * 3 * 32);
    for (float** v : {&X.b32, &X.w32, &X.ua32, &X.ub32}) *v = dalloc<float>(c, X.n);
    X.allocated = true;
  }
  const NloHost H = nlo_assemble_host(L.verts_host, L.nbr_host, L.nc, L.nz, c->ph);
  std::vector<double> Lf, Dinv;
  nlo_factor_host(H, c->ph.omega, Lf, Dinv);
  std::vector<double> Ad, Cs, Cu, Lft, Dit, Lb, Nb;
  std::vector<int> nb;
  nlo_pack_host(H, Lf, Dinv, L.nbr_host, &Ad, &Cs, &Cu, &Lft, &Dit, &Lb, &Nb, &nb);
  auto up = [](void* dst, const void* src, size_t bytes) {
    cuda_ok(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), "NLO upload");
  };
  // FP64 tables and their FP32 copies (rounded to nearest)
  std::vector<float> f32;
  auto up2 = [&](double* d64, float* d32, const std::vector<double>& v) {
    up(d64, v.data(), v.size() * sizeof(double));
    f32.assign(v.begin(), v.end());
    up(d32, f32.data(), f32.size() * sizeof(float));
  };
  up2(X.Ad, X.Ad32, Ad);
  up2(X.Cs, X.Cs32, Cs);
  up2(X.Cu, X.Cu32, Cu);
  up2(X.Lf, X.Lf32, Lft);
  up2(X.Di, X.Di32, Dit);
  up2(X.Lb, X.Lb32, Lb);
  up2(X.Nb, X.Nb32, Nb);
  up(X.nb, nb.data(), nb.size() * sizeof(int));
  X.ready = true;
}

// The lowest-order cycle configuration below the NLO level: levels = 0 all,
// 1 none (the NLO smoother alone), k > 1 the first k - 1.
CycleCfg nlo_cfg(const hmg_ctx* c, int nu_pre, int nu_post, int n_coarse, int levels, int precision) {
  CycleCfg cfg = make_cfg(c, nu_pre, nu_post, n_coarse, levels > 1 ? levels - 1 : 0, precision);
  if (levels == 1) cfg.nlev = 0;
  return cfg;
}

// out <- V b on the NLO level (tiled NLO FP64 vectors, zero initial guess);
// out must not be one of the NLO work vectors.  The mixed form runs the NLO
// level in FP32 unless it is the only level (the coarsest level stays FP64,
// as in the lowest-order cycle).
void nlo_cycle(hmg_ctx* c, const CycleCfg& cfg, const double* b, double* out, cudaStream_t s) {
  NloSys& X = c->nlo;
  Level& L0 = c->lv[0];
  const int nz = L0.nz;
  const bool single = cfg.nlev == 0;
  const int dt = (cfg.mixed && !single) ? HMG_FP32 : HMG_FP64;
  const int npre = single ? cfg.n_coarse : cfg.nu_pre;
  if (single && npre == 1) {
    LAUNCH(c, HMG_K_NLO_SWEEP0, 0, s,
           launch_nlo_sweep(X, nz, dt, b, HMG_FP64, nullptr, nullptr, out, HMG_FP64, cfg.omega, s));
    return;
  }
  void* A = dt == HMG_FP64 ? (void*)X.ua : (void*)X.ua32;
  void* B = dt == HMG_FP64 ? (void*)X.ub : (void*)X.ub32;
  const void* bl = dt == HMG_FP64 ? (const void*)b : (const void*)X.b32;
  LAUNCH(c, HMG_K_NLO_SWEEP0, 0, s,
         launch_nlo_sweep(X, nz, dt, b, HMG_FP64, dt == HMG_FP32 ? X.b32 : nullptr, nullptr, A, dt, cfg.omega, s));
  void* cur = A;
  void* nxt = B;
  for (int i = 1; i < npre; ++i) {
    const bool last = single && i == npre - 1;
    LAUNCH(c, HMG_K_NLO_SWEEP, 0, s,
           launch_nlo_sweep(X, nz, dt, bl, dt, nullptr, cur, last ? (void*)out : nxt, last ? HMG_FP64 : dt,
                            cfg.omega, s));
    if (last) return;
    std::swap(cur, nxt);
  }
  const int cdt = level_dt(c, cfg, 0);
  void* bc = work(L0, cdt, 2);
  void* ec = cdt == HMG_FP64 ? (void*)L0.ux64 : (void*)L0.ux32;
  if (L0.ncp > L0.nc)
    cuda_ok(cudaMemsetAsync(bc, 0, (size_t)L0.Np * (cdt == HMG_FP64 ? sizeof(double) : sizeof(float)), s),
            "memset");
  LAUNCH(c, HMG_K_NLO_RESID, 0, s, launch_nlo_resid_restrict(X, L0, dt, bl, cur, bc, cdt, s));
  cycle(c, cfg, 0, bc, cdt, ec, cdt, s);
  LAUNCH(c, HMG_K_PROLONG, 0, s, launch_nlo_prolong(X, L0, dt, cur, ec, cdt, s));
  for (int i = 0; i < cfg.nu_post; ++i) {
    const bool last = i == cfg.nu_post - 1;
    LAUNCH(c, HMG_K_NLO_SWEEP, 0, s,
           launch_nlo_sweep(X, nz, dt, bl, dt, nullptr, cur, last ? (void*)out : nxt, last ? HMG_FP64 : dt,
                            cfg.omega, s));
    std::swap(cur, nxt);
  }
}

// GMRES(m) on the NLO system (tiled nlo.b, nlo.x), right-preconditioned by
// one NLO V-cycle.
hmg_status solve_nlo_tiled(hmg_ctx* c, const hmg_solve_params& p, hmg_solve_info* info, cudaStream_t s) {
  NloSys& X = c->nlo;
  const int nz = c->lv[0].nz;
  const CycleCfg cfg = nlo_cfg(c, p.nu_pre, p.nu_post, p.n_coarse, p.levels, p.precision);
  KrylovSystem sys;
  sys.n = X.n;
  sys.b = X.b;
  sys.x = X.x;
  sys.tmp = X.t1;
  sys.apply = [c, &X, nz](const double* x, double* y, cudaStream_t st) {
    LAUNCH(c, HMG_K_NLO_APPLY, 0, st, launch_nlo_apply(X, nz, x, y, st));
  };
  sys.precond = [c, cfg](const double* r, double* z, cudaStream_t st) { nlo_cycle(c, cfg, r, z, st); };
  sys.orth = p.orth == 2 ? 2 : 1;
  sys.key = (3LL << 60) + (sys.orth == 2 ? (1LL << 59) : 0) + graph_key(cfg, true, 0);
  return gmres_run(c, sys, p, info, s);
}

// ------------------------------------------------------------ NLO velocity-pressure system

// Upload a host CSR matrix; the device arrays are allocated by the first
// upload and reused afterwards (the sparsity depends on the mesh only), so
// CUDA graphs that captured them stay valid.
void upload_csr(hmg_ctx* c, const Csr& h, DevCsr& d) {
  if (!d.ptr) {
    d.nrows = h.nrows;
    d.ncols = h.ncols;
    d.nnz = (int64_t)h.col.size();
    d.ptr = dalloc<int64_t>(c, h.ptr.size());
    d.col = dalloc<int32_t>(c, h.col.size());
    d.val = dalloc<double>(c, h.val.size());
  }
  require(d.nrows == h.nrows && d.nnz == (int64_t)h.col.size(), "NLO system sparsity changed");
  cuda_ok(cudaMemcpy(d.ptr, h.ptr.data(), h.ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "upload");
  cuda_ok(cudaMemcpy(d.col, h.col.data(), h.col.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "upload");
  cuda_ok(cudaMemcpy(d.val, h.val.data(), h.val.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
}

// The assembled system of the current assembly (host CSR assembly, one upload).
void ensure_nlo_mixed(hmg_ctx* c) {
  ensure_nlo(c);
  NloMixedSys& M = c->nlomx;
  if (M.ready) return;
  const Level& L = c->lv[0];
  if (c->mx.edges_host.empty()) mixed_edges_host(c, nullptr);
  const NloMixedHost H = nlo_mixed_assemble_host(L.verts_host, L.nbr_host, c->mx.edges_host, L.nc, L.nz, c->ph);
  M.nue = H.nue;
  M.nui = H.nui;
  M.nuz = H.nuz;
  M.nu = H.nu;
  M.np = H.np;
  M.n = H.n;
  upload_csr(c, H.A, M.A);
  upload_csr(c, H.D, M.D);
  upload_csr(c, H.Dt, M.Dt);
  if (!M.m2inv) {
    M.m2inv = dalloc<double>(c, M.nu);
    for (double** v : {&M.b, &M.x, &M.t1, &M.t2}) *v = dalloc<double>(c, M.n);
    M.Dval32 = dalloc<float>(c, H.D.val.size());
    M.Dtval32 = dalloc<float>(c, H.Dt.val.size());
    M.tu32 = dalloc<float>(c, M.nu);
    M.zp32 = dalloc<float>(c, M.np);
  }
  {
    const std::vector<float> d32(H.D.val.begin(), H.D.val.end()), dt32(H.Dt.val.begin(), H.Dt.val.end());
    cuda_ok(cudaMemcpy(M.Dval32, d32.data(), d32.size() * sizeof(float), cudaMemcpyHostToDevice), "upload");
    cuda_ok(cudaMemcpy(M.Dtval32, dt32.data(), dt32.size() * sizeof(float), cudaMemcpyHostToDevice), "upload");
  }
  std::vector<double> inv(H.m2diag.size());
  for (size_t i = 0; i < inv.size(); ++i) inv[i] = 1.0 / H.m2diag[i];
  cuda_ok(cudaMemcpy(M.m2inv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
  M.ready = true;
}

// GMRES(m) on the NLO velocity-pressure system (nlomx.b, nlomx.x) with the
// Schur-complement preconditioner; H^^-1 is one NLO V-cycle.
hmg_status solve_nlo_mixed(hmg_ctx* c, const hmg_solve_params& p, hmg_solve_info* info, cudaStream_t s) {
  NloMixedSys& M = c->nlomx;
  NloSys& X = c->nlo;
  const int nz = c->lv[0].nz;
  const CycleCfg cfg = nlo_cfg(c, p.nu_pre, p.nu_post, p.n_coarse, p.levels, p.precision);
  KrylovSystem sys;
  sys.n = M.n;
  sys.b = M.b;
  sys.x = M.x;
  sys.tmp = M.t1;
  sys.apply = [c, &M](const double* x, double* y, cudaStream_t st) {
    LAUNCH(c, HMG_K_APPLY, 0, st, launch_csr_spmv(M.A, x, 1.0, nullptr, nullptr, y, st));
  };
  // The mixed form also runs the two outer factors' products with FP32
  // values and operands (on the FP32 pipe); their sums and the FP64 right-hand
  // sides they update stay FP64.
  sys.precond = [c, &M, &X, cfg, nz](const double* r, double* z, cudaStream_t st) {
    const double ac2 = c->ph.a * c->ph.c2;
    if (cfg.mixed) {
      LAUNCH(c, HMG_K_ORTHO, 0, st, launch_mul32(M.nu, r, M.m2inv, M.tu32, st));       // M2inv r_U
      LAUNCH(c, HMG_K_ORTHO, 0, st,
             launch_csr_spmv32(M.D, M.Dval32, M.tu32, -ac2, r + M.nu, nullptr, M.t2 + M.nu, st));
    } else {
      LAUNCH(c, HMG_K_ORTHO, 0, st, launch_mul(M.nu, r, M.m2inv, M.t2, st));           // M2inv r_U
      LAUNCH(c, HMG_K_ORTHO, 0, st, launch_csr_spmv(M.D, M.t2, -ac2, r + M.nu, nullptr, M.t2 + M.nu, st));
    }
    LAUNCH(c, HMG_K_LAYOUT, 0, st, launch_nlo_layout(X, nz, true, M.t2 + M.nu, X.t1, st));
    nlo_cycle(c, cfg, X.t1, X.t2, st);
    LAUNCH(c, HMG_K_LAYOUT, 0, st, launch_nlo_layout(X, nz, false, X.t2, z + M.nu, st));
    if (cfg.mixed) {
      LAUNCH(c, HMG_K_LAYOUT, 0, st, launch_convert(M.np, z + M.nu, HMG_FP64, M.zp32, st));
      LAUNCH(c, HMG_K_ORTHO, 0, st, launch_csr_spmv32(M.Dt, M.Dtval32, M.zp32, c->ph.a, r, M.m2inv, z, st));
    } else {
      LAUNCH(c, HMG_K_ORTHO, 0, st, launch_csr_spmv(M.Dt, z + M.nu, c->ph.a, r, M.m2inv, z, st));
    }
  };
  sys.orth = p.orth == 2 ? 2 : 1;
  sys.key = (4LL << 60) + (sys.orth == 2 ? (1LL << 59) : 0) + graph_key(cfg, true, 0);
  return gmres_run(c, sys, p, info, s);
}

void check_solve_params(const hmg_solve_params* p) {
  require(p != nullptr, "params is NULL");
  require(p->precision == HMG_PRECISION_FP64 || p->precision == HMG_PRECISION_MIXED, "bad precision");
  require(p->krylov == HMG_KRYLOV_CG || p->krylov == HMG_KRYLOV_FCG || p->krylov == HMG_KRYLOV_GMRES,
          "bad krylov");
  require(p->krylov != HMG_KRYLOV_GMRES || (p->restart >= 1 && p->restart <= GMRES_MAX_RESTART),
          "GMRES restart must be in [1, " + std::to_string(GMRES_MAX_RESTART) + "]");
  require(p->levels >= 0, "levels must be >= 0");
  require(p->orth >= 0 && p->orth <= 2, "orth must be 0, 1 or 2");
  require(p->rtol > 0.0 && p->rtol < 1.0, "rtol must be in (0, 1)");
  require(p->max_iter >= 1 && p->max_iter <= 100000, "max_iter must be in [1, 100000]");
  check_cycle_params(p->nu_pre, p->nu_post, p->n_coarse);
}

void need_assembled(const hmg_ctx* c) {
  if (!c->assembled) throw Fail{HMG_ERR_STATE, "operator not assembled (call hmg_assemble_helmholtz)"};
}

}  // namespace

namespace hmg {
// Tracing hooks for entry points defined in other files (see LAUNCH above).
int trace_begin(hmg_ctx* c, int kernel, int level, cudaStream_t s) { return prof_begin(c, kernel, level, s); }
void trace_end(hmg_ctx* c, int rec, cudaStream_t s) { prof_end(c, rec, s); }
}  // namespace hmg

extern "C" {

const char* hmg_status_string(hmg_status s) {
  switch (s) {
    case HMG_OK: return "ok";
    case HMG_ERR_INVALID_ARG: return "invalid argument";
    case HMG_ERR_CUDA: return "CUDA error";
    case HMG_ERR_OOM: return "out of memory";
    case HMG_ERR_NOT_CONVERGED: return "not converged";
    case HMG_ERR_BREAKDOWN: return "Krylov breakdown";
    case HMG_ERR_NONFINITE: return "non-finite value";
    case HMG_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* hmg_last_error(const hmg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_build_error.c_str();
}

static hmg_status build_hierarchy(const hmg_mesh_params* p, hmg_alloc_fn alloc, hmg_release_fn rel, void* user,
                                  hmg_ctx** out) {
  if (!out) {
    g_build_error = "out is NULL";
    return HMG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  hmg_ctx* c = nullptr;
  hmg_status st = guarded(nullptr, [&] {
    require(p != nullptr, "params is NULL");
    require((alloc == nullptr) == (rel == nullptr), "alloc and release must both be given");
    require(p->refinement >= 0 && p->refinement <= 10, "refinement must be in [0, 10]");
    require(p->nlayers >= 1 && p->nlayers <= 256, "nlayers must be in [1, 256]");
    require(p->nlevels >= 1 && p->nlevels <= p->refinement + 1, "nlevels must be in [1, refinement + 1]");
    require(p->radius_m > 0 && std::isfinite(p->radius_m), "radius_m must be positive");
    require(p->thickness_m > 0 && std::isfinite(p->thickness_m), "thickness_m must be positive");
    std::vector<HostLevel> host = build_mesh_hierarchy(p->refinement, p->nlevels);
    c = new hmg_ctx();
    c->alloc_fn = alloc;
    c->release_fn = rel;
    c->alloc_user = user;
    c->mp = *p;
    c->lv.resize(host.size());
    for (size_t k = 0; k < host.size(); ++k) {
      Level& L = c->lv[k];
      HostLevel& H = host[k];
      L.refinement = H.refinement;
      L.nc = H.ncols;
      L.ncp = (H.ncols + TW - 1) / TW * TW;
      L.nz = p->nlayers;
      L.N = (int64_t)L.nc * L.nz;
      L.Np = (int64_t)L.ncp * L.nz;
      // FP64: half columns on two warps everywhere; FP32: twisted two-chain
      // column solves on the small (latency-bound) levels, the same tile
      // threshold as the staged FP32 sweep of cycle.cu
      L.twist = L.nz / 2;
      L.twist32 = (L.ncp / TW <= SMALL_LEVEL_TILES) ? L.nz / 2 : L.nz - 1;
      L.centroid_host = H.centroid;
      L.nbr_host = H.nbr;
      L.verts_host = H.verts;
      std::vector<int4> nb(L.ncp);
      for (int col = 0; col < L.ncp; ++col) {
        if (col < L.nc) nb[col] = make_int4(H.nbr[3 * col], H.nbr[3 * col + 1], H.nbr[3 * col + 2], 0);
        else nb[col] = make_int4(col, col, col, 0);
      }
      std::vector<double> verts((size_t)L.ncp * 9, 0.0);
      std::copy(H.verts.begin(), H.verts.end(), verts.begin());
      L.nbr = dalloc<int4>(c, L.ncp);
      L.verts = dalloc<double>(c, (size_t)L.ncp * 9);
      cuda_ok(cudaMemcpy(L.nbr, nb.data(), nb.size() * sizeof(int4), cudaMemcpyHostToDevice), "upload");
      cuda_ok(cudaMemcpy(L.verts, verts.data(), verts.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
      L.A1 = dalloc<double>(c, L.ncp);
      L.sigma = dalloc<double4_32a>(c, L.ncp);
      L.gh = dalloc<double4_32a>(c, L.ncp);
      L.gh32 = dalloc<float4>(c, L.ncp);
      L.d = dalloc<double>(c, L.Np);
      L.e = dalloc<double>(c, L.Np);
      L.lo = dalloc<double>(c, L.Np);
      L.w = dalloc<double>(c, L.Np);
      L.d32 = dalloc<float>(c, L.Np);
      L.e32 = dalloc<float>(c, L.Np);
      L.lo32 = dalloc<float>(c, L.Np);
      L.w32 = dalloc<float>(c, L.Np);
      L.mt = dalloc<double>(c, L.ncp);
      L.los = dalloc<double>(c, L.Np);
      L.mts = dalloc<double>(c, L.ncp);
      L.mt32 = dalloc<float>(c, L.ncp);
      L.theta = dalloc<double>(c, L.Np);
      L.b64 = dalloc<double>(c, L.Np);
      L.ua64 = dalloc<double>(c, L.Np);
      L.ub64 = dalloc<double>(c, L.Np);
      L.ux64 = dalloc<double>(c, L.Np);
      L.b32 = dalloc<float>(c, L.Np);
      L.ua32 = dalloc<float>(c, L.Np);
      L.ub32 = dalloc<float>(c, L.Np);
      L.ux32 = dalloc<float>(c, L.Np);
    }
    const int64_t Np0 = c->lv[0].Np;
    c->kx = dalloc<double>(c, Np0);
    c->kr = dalloc<double>(c, Np0);
    c->kz = dalloc<double>(c, Np0);
    c->kp = dalloc<double>(c, Np0);
    c->kq = dalloc<double>(c, Np0);
    c->kb = dalloc<double>(c, Np0);
    c->kcol = dalloc<double>(c, Np0);
    c->kcol2 = dalloc<double>(c, Np0);
    c->red.partials = dalloc<double>(c, 2 * RED_MAX_BLOCKS);
    c->red.counter = dalloc<unsigned int>(c, 4);
    c->red.sc = dalloc<double>(c, S_COUNT);
    cuda_ok(cudaHostAlloc((void**)&c->host_sc, S_COUNT * sizeof(double), cudaHostAllocDefault), "host alloc");
    cuda_ok(cudaEventCreate(&c->ev0), "event");
    cuda_ok(cudaEventCreate(&c->ev1), "event");
    cuda_ok(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "stream");
    cuda_ok(cudaDeviceSynchronize(), "build");
  });
  if (st != HMG_OK) {
    if (c) {
      g_build_error = g_build_error.empty() ? c->err : g_build_error;
      release(c);
      delete c;
    }
    return st;
  }
  *out = c;
  return HMG_OK;
}

hmg_status hmg_build_hierarchy(const hmg_mesh_params* p, hmg_ctx** out) {
  return build_hierarchy(p, nullptr, nullptr, nullptr, out);
}

hmg_status hmg_build_hierarchy_with_allocator(const hmg_mesh_params* p, hmg_alloc_fn alloc, hmg_release_fn release,
                                              void* user, hmg_ctx** out) {
  if (!alloc || !release) {
    g_build_error = "alloc and release must be non-NULL";
    return HMG_ERR_INVALID_ARG;
  }
  return build_hierarchy(p, alloc, release, user, out);
}

hmg_status hmg_destroy(hmg_ctx* ctx) {
  if (!ctx) return HMG_OK;
  cudaDeviceSynchronize();
  release(ctx);
  delete ctx;
  return HMG_OK;
}

hmg_status hmg_get_level_info(const hmg_ctx* ctx, int level, hmg_level_info* out) {
  if (!ctx || !out || level < 0 || level >= (int)ctx->lv.size()) return HMG_ERR_INVALID_ARG;
  const Level& L = ctx->lv[level];
  out->refinement = L.refinement;
  out->ncols = L.nc;
  out->ncols_padded = L.ncp;
  out->nlayers = L.nz;
  out->ncells = L.N;
  out->ncells_padded = L.Np;
  return HMG_OK;
}

hmg_status hmg_export_mesh(const hmg_ctx* ctx, int level, double* centroids, int32_t* nbr) {
  if (!ctx || level < 0 || level >= (int)ctx->lv.size()) return HMG_ERR_INVALID_ARG;
  const Level& L = ctx->lv[level];
  if (centroids) std::memcpy(centroids, L.centroid_host.data(), L.centroid_host.size() * sizeof(double));
  if (nbr) std::memcpy(nbr, L.nbr_host.data(), L.nbr_host.size() * sizeof(int32_t));
  return HMG_OK;
}

hmg_status hmg_assemble_helmholtz(hmg_ctx* ctx, const hmg_op_params* p, const double* theta, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    check_op_params(p);
    cudaStream_t s = as_stream(stream);
    ctx->assembled = false;
    ctx->nlo.ready = false;
    ctx->nlomx.ready = false;
    ctx->op = *p;
    const Phys& ph = (ctx->ph = make_phys(ctx->mp, *p));
    ctx->has_theta = theta != nullptr;
    if (theta) {
      LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_tiled(ctx->lv[0], HMG_FP64, theta, ctx->lv[0].theta, s));
      for (size_t k = 1; k < ctx->lv.size(); ++k)
        LAUNCH(ctx, HMG_K_ASSEMBLY, (int)k, s, launch_theta_restrict(ctx->lv[k - 1], ctx->lv[k], s));
    }
    for (size_t k = 0; k < ctx->lv.size(); ++k) {
      Level& L = ctx->lv[k];
      const int lev = (int)k;
      double* th = L.theta;
      if (!theta) L.theta = nullptr;  // bands use theta = 1
      LAUNCH(ctx, HMG_K_ASSEMBLY, lev, s, launch_geometry(L, s));
      LAUNCH(ctx, HMG_K_ASSEMBLY, lev, s, launch_couplings(L, ph.wc2 * ph.dz, s));
      LAUNCH(ctx, HMG_K_ASSEMBLY, lev, s, launch_bands(L, ph, s));
      L.theta = th;
      LAUNCHN(ctx, HMG_K_ASSEMBLY, lev, s, 2, launch_ldl(L, ph.omega, s));
      LAUNCHN(ctx, HMG_K_ASSEMBLY, lev, s, 3, launch_to_fp32(L, s));
    }
    cuda_ok(cudaStreamSynchronize(s), "assemble");
    ctx->assembled = true;
  });
}

hmg_status hmg_apply(hmg_ctx* ctx, int level, int dtype, int layout, const void* x, void* y, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(level >= 0 && level < (int)ctx->lv.size(), "bad level");
    require(dtype == HMG_FP64 || dtype == HMG_FP32, "bad dtype");
    require(layout == HMG_LAYOUT_COLUMN || layout == HMG_LAYOUT_TILED, "bad layout");
    require(x && y && x != y, "x and y must be distinct non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    Level& L = ctx->lv[level];
    // level 0 in FP64 runs partitioned on a partitioned context
    const bool part = level == 0 && dtype == HMG_FP64 && ctx->nparts > 1;
    if (layout == HMG_LAYOUT_TILED) {
      if (part) apply_fine(ctx, (const double*)x, (double*)y, nullptr, s);
      else LAUNCH(ctx, HMG_K_APPLY, level, s, launch_apply(L, dtype, x, y, nullptr, s));
      return;
    }
    LAUNCH(ctx, HMG_K_LAYOUT, level, s, launch_to_tiled(L, dtype, x, ctx->kcol, s));
    if (part) apply_fine(ctx, ctx->kcol, ctx->kcol2, nullptr, s);
    else LAUNCH(ctx, HMG_K_APPLY, level, s, launch_apply(L, dtype, ctx->kcol, ctx->kcol2, nullptr, s));
    LAUNCH(ctx, HMG_K_LAYOUT, level, s, launch_to_column(L, dtype, ctx->kcol2, y, s));
  });
}

hmg_status hmg_vcycle(hmg_ctx* ctx, int precision, int layout, const void* r, void* z, int nu_pre, int nu_post,
                      int n_coarse, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(precision == HMG_PRECISION_FP64 || precision == HMG_PRECISION_MIXED, "bad precision");
    require(layout == HMG_LAYOUT_COLUMN || layout == HMG_LAYOUT_TILED, "bad layout");
    require(r && z && r != z, "r and z must be distinct non-NULL device pointers");
    check_cycle_params(nu_pre, nu_post, n_coarse);
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    const CycleCfg cfg = make_cfg(ctx, nu_pre, nu_post, n_coarse, 0, precision);
    Level& L = ctx->lv[0];
    if (layout == HMG_LAYOUT_TILED) {
      cycle(ctx, cfg, 0, r, HMG_FP64, z, HMG_FP64, s);
      return;
    }
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_tiled(L, HMG_FP64, r, ctx->kcol, s));
    cycle(ctx, cfg, 0, ctx->kcol, HMG_FP64, ctx->kcol2, HMG_FP64, s);
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_column(L, HMG_FP64, ctx->kcol2, z, s));
  });
}

hmg_status hmg_solve(hmg_ctx* ctx, const double* b, double* x, const hmg_solve_params* params,
                     hmg_solve_info* info, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  hmg_status result = HMG_OK;
  hmg_status st = guarded(ctx, [&] {
    check_solve_params(params);
    require(params->levels <= (int)ctx->lv.size(), "levels exceeds the hierarchy's level count");
    require(b && x, "b and x must be non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    Level& L = ctx->lv[0];
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_tiled(L, HMG_FP64, b, ctx->kb, s));
    result = solve_tiled(ctx, *params, info, s);
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_column(L, HMG_FP64, ctx->kx, x, s));
    cuda_ok(cudaStreamSynchronize(s), "solve");
  });
  if (st != HMG_OK) return st;
  if (result == HMG_ERR_NOT_CONVERGED) ctx->err = "maximum number of iterations reached";
  if (result == HMG_ERR_BREAKDOWN) ctx->err = "CG breakdown: p.q <= 0 or r.z <= 0";
  if (result == HMG_ERR_NONFINITE) ctx->err = "non-finite residual";
  return result;
}

// The device address of page-locked (registered or cudaHostAlloc'd) host
// memory, or null for any other pointer (pageable host memory, device
// memory), which the caller then copies.
static const void* device_address(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // clear the error of an unknown pointer
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

hmg_status hmg_solve_host(hmg_ctx* ctx, const double* b_host, double* x_host, const hmg_solve_params* params,
                          hmg_solve_info* info, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  hmg_status result = HMG_OK;
  hmg_status st = guarded(ctx, [&] {
    check_solve_params(params);
    require(params->levels <= (int)ctx->lv.size(), "levels exceeds the hierarchy's level count");
    require(b_host && x_host, "b_host and x_host must be non-NULL");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    Level& L = ctx->lv[0];
    // Page-locked host buffers that the device addresses directly are read
    // and written by the layout kernels over the host link, with no staging
    // copy; other host memory goes through cudaMemcpyAsync and a device buffer.
    const void* b_dev = device_address(b_host);
    void* x_dev = const_cast<void*>(device_address(x_host));
    if (b_dev) {
      LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_tiled(L, HMG_FP64, b_dev, ctx->kb, s));
    } else {
      cuda_ok(cudaMemcpyAsync(ctx->kcol, b_host, (size_t)L.N * sizeof(double), cudaMemcpyHostToDevice, s), "H2D");
      LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_tiled(L, HMG_FP64, ctx->kcol, ctx->kb, s));
    }
    result = solve_tiled(ctx, *params, info, s);
    if (x_dev) {
      LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_column(L, HMG_FP64, ctx->kx, x_dev, s));
    } else {
      LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_to_column(L, HMG_FP64, ctx->kx, ctx->kcol, s));
      cuda_ok(cudaMemcpyAsync(x_host, ctx->kcol, (size_t)L.N * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    }
    cuda_ok(cudaStreamSynchronize(s), "solve");
  });
  if (st != HMG_OK) return st;
  return result;
}

hmg_status hmg_mixed_sizes(const hmg_ctx* ctx, int64_t* n_hfaces, int64_t* n_vfaces, int64_t* n_cells) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  const Level& L = ctx->lv[0];
  const int64_t ne = (int64_t)L.nc * 3 / 2;
  if (n_hfaces) *n_hfaces = ne * L.nz;
  if (n_vfaces) *n_vfaces = (int64_t)L.nc * (L.nz - 1);
  if (n_cells) *n_cells = L.N;
  return HMG_OK;
}

hmg_status hmg_export_edges(hmg_ctx* ctx, int32_t* edges) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(edges != nullptr, "edges is NULL");
    if (ctx->mx.edges_host.empty()) mixed_edges_host(ctx, nullptr);
    std::memcpy(edges, ctx->mx.edges_host.data(), ctx->mx.edges_host.size() * sizeof(int32_t));
  });
}

hmg_status hmg_mixed_apply(hmg_ctx* ctx, const double* u, const double* p, double* yu, double* yp, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(u && p && yu && yp, "u, p, yu and yp must be non-NULL device pointers");
    require(u != yu && p != yp, "outputs must differ from inputs");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_mixed(ctx, s);
    Level& L = ctx->lv[0];
    MixedSys& M = ctx->mx;
    LAUNCHN(ctx, HMG_K_LAYOUT, 0, s, 3, launch_mixed_layout(L, M, true, u, p, M.t1, nullptr, nullptr, s));
    LAUNCHN(ctx, HMG_K_APPLY, 0, s, 2, launch_mixed_apply(L, M, ctx->ph, M.t1, M.t2, s));
    LAUNCHN(ctx, HMG_K_LAYOUT, 0, s, 3, launch_mixed_layout(L, M, false, nullptr, nullptr, M.t2, yu, yp, s));
  });
}

hmg_status hmg_mixed_solve(hmg_ctx* ctx, const double* bu, const double* bp, double* u, double* p,
                           const hmg_solve_params* params, hmg_solve_info* info, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  hmg_status result = HMG_OK;
  hmg_status st = guarded(ctx, [&] {
    check_solve_params(params);
    require(params->levels <= (int)ctx->lv.size(), "levels exceeds the hierarchy's level count");
    require(params->restart >= 1 && params->restart <= GMRES_MAX_RESTART,
            "GMRES restart must be in [1, " + std::to_string(GMRES_MAX_RESTART) + "]");
    require(bu && bp && u && p, "bu, bp, u and p must be non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_mixed(ctx, s);
    Level& L = ctx->lv[0];
    MixedSys& M = ctx->mx;
    LAUNCHN(ctx, HMG_K_LAYOUT, 0, s, 3, launch_mixed_layout(L, M, true, bu, bp, M.b, nullptr, nullptr, s));
    result = solve_mixed_tiled(ctx, *params, info, s);
    LAUNCHN(ctx, HMG_K_LAYOUT, 0, s, 3, launch_mixed_layout(L, M, false, nullptr, nullptr, M.x, u, p, s));
    cuda_ok(cudaStreamSynchronize(s), "solve");
  });
  if (st != HMG_OK) return st;
  if (result == HMG_ERR_NOT_CONVERGED) ctx->err = "maximum number of iterations reached";
  if (result == HMG_ERR_BREAKDOWN) ctx->err = "GMRES breakdown";
  if (result == HMG_ERR_NONFINITE) ctx->err = "non-finite residual";
  return result;
}

hmg_status hmg_nlo_size(const hmg_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return HMG_ERR_INVALID_ARG;
  *n = 6 * ctx->lv[0].N;
  return HMG_OK;
}

hmg_status hmg_export_vertices(const hmg_ctx* ctx, int level, double* verts) {
  if (!ctx || !verts || level < 0 || level >= (int)ctx->lv.size()) return HMG_ERR_INVALID_ARG;
  const Level& L = ctx->lv[level];
  std::memcpy(verts, L.verts_host.data(), L.verts_host.size() * sizeof(double));
  return HMG_OK;
}

hmg_status hmg_nlo_host_blocks(const hmg_mesh_params* mesh, const hmg_op_params* op, double* diag, double* sub,
                               double* nbr_blocks, int32_t* nbr, double* verts) {
  hmg_status st = guarded(nullptr, [&] {
    require(mesh != nullptr, "mesh is NULL");
    require(mesh->refinement >= 0 && mesh->refinement <= 8, "refinement must be in [0, 8]");
    require(mesh->nlayers >= 1 && mesh->nlayers <= 256, "nlayers must be in [1, 256]");
    require(mesh->radius_m > 0 && mesh->thickness_m > 0, "radius_m and thickness_m must be positive");
    check_op_params(op);
    require(diag && sub && nbr_blocks, "diag, sub and nbr_blocks must be non-NULL host buffers");
    std::vector<HostLevel> host = build_mesh_hierarchy(mesh->refinement, 1);
    const HostLevel& H = host[0];
    const NloHost B = nlo_assemble_host(H.verts, H.nbr, H.ncols, mesh->nlayers, make_phys(*mesh, *op));
    std::memcpy(diag, B.diag.data(), B.diag.size() * sizeof(double));
    std::memcpy(sub, B.sub.data(), B.sub.size() * sizeof(double));
    std::memcpy(nbr_blocks, B.nbr.data(), B.nbr.size() * sizeof(double));
    if (nbr) std::memcpy(nbr, H.nbr.data(), H.nbr.size() * sizeof(int32_t));
    if (verts) std::memcpy(verts, H.verts.data(), H.verts.size() * sizeof(double));
  });
  return st;
}

hmg_status hmg_nlo_apply(hmg_ctx* ctx, const double* x, double* y, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(x && y && x != y, "x and y must be distinct non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_nlo(ctx);
    NloSys& X = ctx->nlo;
    const int nz = ctx->lv[0].nz;
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_nlo_layout(X, nz, true, x, X.t1, s));
    LAUNCH(ctx, HMG_K_NLO_APPLY, 0, s, launch_nlo_apply(X, nz, X.t1, X.t2, s));
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_nlo_layout(X, nz, false, X.t2, y, s));
  });
}

hmg_status hmg_nlo_vcycle(hmg_ctx* ctx, int precision, const double* r, double* z, int nu_pre, int nu_post,
                          int n_coarse, int levels, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(precision == HMG_PRECISION_FP64 || precision == HMG_PRECISION_MIXED, "bad precision");
    require(r && z && r != z, "r and z must be distinct non-NULL device pointers");
    check_cycle_params(nu_pre, nu_post, n_coarse);
    require(levels >= 0 && levels <= (int)ctx->lv.size() + 1, "levels must be in [0, nlevels + 1]");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_nlo(ctx);
    NloSys& X = ctx->nlo;
    const int nz = ctx->lv[0].nz;
    const CycleCfg cfg = nlo_cfg(ctx, nu_pre, nu_post, n_coarse, levels, precision);
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_nlo_layout(X, nz, true, r, X.t1, s));
    nlo_cycle(ctx, cfg, X.t1, X.t2, s);
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_nlo_layout(X, nz, false, X.t2, z, s));
  });
}

hmg_status hmg_nlo_solve(hmg_ctx* ctx, const double* b, double* x, const hmg_solve_params* params,
                         hmg_solve_info* info, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  hmg_status result = HMG_OK;
  hmg_status st = guarded(ctx, [&] {
    check_solve_params(params);
    require(params->krylov == HMG_KRYLOV_GMRES, "the NLO solve runs GMRES (krylov = HMG_KRYLOV_GMRES)");
    require(params->levels <= (int)ctx->lv.size() + 1, "levels must be in [0, nlevels + 1]");
    require(b && x, "b and x must be non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_nlo(ctx);
    NloSys& X = ctx->nlo;
    const int nz = ctx->lv[0].nz;
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_nlo_layout(X, nz, true, b, X.b, s));
    result = solve_nlo_tiled(ctx, *params, info, s);
    LAUNCH(ctx, HMG_K_LAYOUT, 0, s, launch_nlo_layout(X, nz, false, X.x, x, s));
    cuda_ok(cudaStreamSynchronize(s), "solve");
  });
  if (st != HMG_OK) return st;
  if (result == HMG_ERR_NOT_CONVERGED) ctx->err = "maximum number of iterations reached";
  if (result == HMG_ERR_BREAKDOWN) ctx->err = "GMRES breakdown";
  if (result == HMG_ERR_NONFINITE) ctx->err = "non-finite residual";
  return result;
}

hmg_status hmg_nlo_mixed_sizes(const hmg_ctx* ctx, int64_t* n_hedge, int64_t* n_hint, int64_t* n_vert,
                               int64_t* n_p) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  const Level& L = ctx->lv[0];
  const int64_t ne = (int64_t)L.nc * 3 / 2;
  if (n_hedge) *n_hedge = ne * L.nz * 4;
  if (n_hint) *n_hint = (int64_t)L.nc * L.nz * 6;
  if (n_vert) *n_vert = (int64_t)L.nc * 3 * (2 * L.nz - 1);
  if (n_p) *n_p = (int64_t)L.nc * L.nz * 6;
  return HMG_OK;
}

hmg_status hmg_nlo_mixed_host_csr(const hmg_mesh_params* mesh, const hmg_op_params* op, int64_t* n, int64_t* nnz,
                                  int64_t* ptr, int32_t* col, double* val, int32_t* edges) {
  return guarded(nullptr, [&] {
    require(mesh != nullptr, "mesh is NULL");
    require(mesh->refinement >= 0 && mesh->refinement <= 5, "refinement must be in [0, 5]");
    require(mesh->nlayers >= 1 && mesh->nlayers <= 256, "nlayers must be in [1, 256]");
    require(mesh->radius_m > 0 && mesh->thickness_m > 0, "radius_m and thickness_m must be positive");
    check_op_params(op);
    require(n && nnz, "n and nnz must be non-NULL");
    std::vector<HostLevel> host = build_mesh_hierarchy(mesh->refinement, 1);
    const HostLevel& H = host[0];
    std::vector<int32_t> el;   // edge list (t, k, tn, kn), t < tn, by t then k
    for (int t = 0; t < H.ncols; ++t)
      for (int k = 0; k < 3; ++k) {
        const int tn = H.nbr[3 * t + k];
        if (t < tn) {
          int kn = 0;
          while (kn < 3 && H.nbr[3 * tn + kn] != t) ++kn;
          require(kn < 3, "mesh neighbours are not symmetric");
          el.insert(el.end(), {t, k, tn, kn});
        }
      }
    const NloMixedHost X = nlo_mixed_assemble_host(H.verts, H.nbr, el, H.ncols, mesh->nlayers, make_phys(*mesh, *op));
    *n = X.n;
    *nnz = (int64_t)X.A.col.size();
    if (ptr) std::memcpy(ptr, X.A.ptr.data(), X.A.ptr.size() * sizeof(int64_t));
    if (col) std::memcpy(col, X.A.col.data(), X.A.col.size() * sizeof(int32_t));
    if (val) std::memcpy(val, X.A.val.data(), X.A.val.size() * sizeof(double));
    if (edges) std::memcpy(edges, el.data(), el.size() * sizeof(int32_t));
  });
}

hmg_status hmg_nlo_mixed_apply(hmg_ctx* ctx, const double* x, double* y, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(x && y && x != y, "x and y must be distinct non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_nlo_mixed(ctx);
    LAUNCH(ctx, HMG_K_APPLY, 0, s, launch_csr_spmv(ctx->nlomx.A, x, 1.0, nullptr, nullptr, y, s));
  });
}

hmg_status hmg_nlo_mixed_solve(hmg_ctx* ctx, const double* b, double* x, const hmg_solve_params* params,
                               hmg_solve_info* info, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  hmg_status result = HMG_OK;
  hmg_status st = guarded(ctx, [&] {
    check_solve_params(params);
    require(params->levels <= (int)ctx->lv.size() + 1, "levels must be in [0, nlevels + 1]");
    require(b && x, "b and x must be non-NULL device pointers");
    need_assembled(ctx);
    cudaStream_t s = as_stream(stream);
    ensure_nlo_mixed(ctx);
    NloMixedSys& M = ctx->nlomx;
    cuda_ok(cudaMemcpyAsync(M.b, b, (size_t)M.n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    result = solve_nlo_mixed(ctx, *params, info, s);
    cuda_ok(cudaMemcpyAsync(x, M.x, (size_t)M.n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    cuda_ok(cudaStreamSynchronize(s), "solve");
  });
  if (st != HMG_OK) return st;
  if (result == HMG_ERR_NOT_CONVERGED) ctx->err = "maximum number of iterations reached";
  if (result == HMG_ERR_BREAKDOWN) ctx->err = "GMRES breakdown";
  if (result == HMG_ERR_NONFINITE) ctx->err = "non-finite residual";
  return result;
}

hmg_status hmg_theta_grad(hmg_ctx* ctx, const double* p, const double* lambda, double* grad, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(p && lambda && grad, "p, lambda and grad must be non-NULL device pointers");
    need_assembled(ctx);
    Level& L = ctx->lv[0];
    double* th = L.theta;
    if (!ctx->has_theta) L.theta = nullptr;
    LAUNCH(ctx, HMG_K_THETA_GRAD, 0, as_stream(stream), launch_theta_grad(L, ctx->ph, p, lambda, grad, as_stream(stream)));
    L.theta = th;
  });
}

hmg_status hmg_to_layout(hmg_ctx* ctx, int level, int src_layout, const double* src, int dst_layout, double* dst,
                         void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(level >= 0 && level < (int)ctx->lv.size(), "bad level");
    require(src && dst && src != dst, "src and dst must be distinct non-NULL device pointers");
    require((src_layout == HMG_LAYOUT_COLUMN && dst_layout == HMG_LAYOUT_TILED) ||
                (src_layout == HMG_LAYOUT_TILED && dst_layout == HMG_LAYOUT_COLUMN),
            "layouts must differ");
    Level& L = ctx->lv[level];
    if (src_layout == HMG_LAYOUT_COLUMN)
      LAUNCH(ctx, HMG_K_LAYOUT, level, as_stream(stream), launch_to_tiled(L, HMG_FP64, src, dst, as_stream(stream)));
    else
      LAUNCH(ctx, HMG_K_LAYOUT, level, as_stream(stream), launch_to_column(L, HMG_FP64, src, dst, as_stream(stream)));
  });
}

const char* hmg_kernel_name(int kernel) {
  static const char* names[HMG_K_COUNT] = {"sweep0", "sweep",     "prolong",  "resid_restrict", "apply",
                                           "dot",    "update_xr", "update_p", "layout",         "resid_sq",
                                           "assembly", "theta_grad", "ortho",    "nlo_sweep",      "nlo_resid",
                                           "nlo_apply", "nlo_sweep0", "coarse_cycle", "halo"};
  return (kernel >= 0 && kernel < HMG_K_COUNT) ? names[kernel] : "?";
}

static const PartLevel& partition_part(int refinement, int nlevels, int nparts, int part, int level,
                                       PartitionPlan& keep) {
  require(refinement >= 0 && refinement <= 9, "refinement must be in [0, 9]");
  require(nlevels >= 1 && nlevels <= refinement + 1, "nlevels must be in [1, refinement + 1]");
  keep = build_partition_for_mesh(refinement, nlevels, nparts);
  require(part >= 0 && part < nparts, "part must be in [0, nparts)");
  require(level >= 0 && level < keep.nlevels, "level is not a partitioned level");
  return keep.lv[level][part];
}

hmg_status hmg_partition_info(int refinement, int nlevels, int nparts, int part, int level, hmg_part_info* out) {
  return guarded(nullptr, [&] {
    require(out != nullptr, "out must not be NULL");
    PartitionPlan plan;
    const PartLevel& pl = partition_part(refinement, nlevels, nparts, part, level, plan);
    out->col_begin = pl.begin;
    out->col_end = pl.end;
    out->ncols_padded = pl.n_own_pad;
    out->n_ghost = (int32_t)pl.ghost_col.size();
    out->n_send = (int32_t)pl.send_col.size();
  });
}

hmg_status hmg_partition_tables(int refinement, int nlevels, int nparts, int part, int level, int32_t* ghost_col,
                                int32_t* ghost_owner, int32_t* ghost_owner_local, int32_t* local_nbr,
                                int32_t* send_col, int32_t* send_to) {
  return guarded(nullptr, [&] {
    PartitionPlan plan;
    const PartLevel& pl = partition_part(refinement, nlevels, nparts, part, level, plan);
    auto put = [](const std::vector<int32_t>& v, int32_t* dst) {
      if (dst) std::copy(v.begin(), v.end(), dst);
    };
    put(pl.ghost_col, ghost_col);
    put(pl.ghost_owner, ghost_owner);
    put(pl.ghost_owner_local, ghost_owner_local);
    put(pl.local_nbr, local_nbr);
    put(pl.send_col, send_col);
    put(pl.send_to, send_to);
  });
}

hmg_status hmg_partition(hmg_ctx* ctx, int nparts) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    require(nparts >= 1 && nparts <= MAX_PARTS, "nparts must be in [1, 16]");
    cuda_ok(cudaDeviceSynchronize(), "partition");
    drop_partition(ctx);
    if (nparts > 1) {
      try {
        build_partition_dev(ctx, nparts);
      } catch (...) {
        drop_partition(ctx);
        throw;
      }
    }
  });
}

hmg_status hmg_measure_fp64_rate(hmg_ctx* ctx, double* tflops, void* stream) {
  if (!ctx || !tflops) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    *tflops = measure_fp64_fma_rate(ctx->red.partials, as_stream(stream));
    launched("k_fp64_fma_probe");
    ctx->launches += 2;
  });
}

hmg_status hmg_set_coarse_fusion(hmg_ctx* ctx, int enable) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  ctx->fuse_coarse = enable != 0;
  ctx->err.clear();
  return HMG_OK;
}

hmg_status hmg_profile_start(hmg_ctx* ctx, unsigned kernel_mask, unsigned level_mask) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    ctx->prof.clear();
    ctx->prof_agg.clear();
    ctx->ev_used = 0;
    ctx->prof_kmask = kernel_mask;
    ctx->prof_lmask = level_mask;
    ctx->prof_on = true;
  });
}

hmg_status hmg_profile_stop(hmg_ctx* ctx, hmg_kernel_stat* out, int capacity, int* count) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] {
    if (!ctx->prof_on) throw Fail{HMG_ERR_STATE, "tracing was not started"};
    for (const ProfRec& r : ctx->prof) {
      cudaEvent_t a = ctx->ev_pool[r.ev], b = ctx->ev_pool[r.ev + 1];
      cuda_ok(cudaEventSynchronize(b), "event sync");
      float ms = 0.f;
      cuda_ok(cudaEventElapsedTime(&ms, a, b), "event time");
      prof_add(ctx, r.kernel, r.level, ms);
    }
    ctx->prof_on = false;
    std::vector<hmg_kernel_stat> agg;
    agg.swap(ctx->prof_agg);
    ctx->prof.clear();
    ctx->ev_used = 0;
    if (count) *count = (int)agg.size();
    for (int i = 0; out && i < capacity && i < (int)agg.size(); ++i) out[i] = agg[i];
  });
}

hmg_status hmg_residual_history(const hmg_ctx* ctx, double* out, int capacity, int* count) {
  if (!ctx || !count || capacity < 0 || (capacity > 0 && !out)) return HMG_ERR_INVALID_ARG;
  *count = (int)ctx->history.size();
  const size_t k = std::min(ctx->history.size(), (size_t)capacity);
  if (k) std::memcpy(out, ctx->history.data(), k * sizeof(double));
  return HMG_OK;
}

hmg_status hmg_launch_count(const hmg_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return HMG_ERR_INVALID_ARG;
  *count = ctx->launches;
  return HMG_OK;
}

hmg_status hmg_convert_fp64_to_fp32(const double* src, float* dst, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!src || !dst))) return HMG_ERR_INVALID_ARG;
  if (n == 0) return HMG_OK;
  launch_convert(n, src, HMG_FP64, dst, as_stream(stream));
  return cudaGetLastError() == cudaSuccess ? HMG_OK : HMG_ERR_CUDA;
}

hmg_status hmg_convert_fp32_to_fp64(const float* src, double* dst, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!src || !dst))) return HMG_ERR_INVALID_ARG;
  if (n == 0) return HMG_OK;
  launch_convert(n, src, HMG_FP32, dst, as_stream(stream));
  return cudaGetLastError() == cudaSuccess ? HMG_OK : HMG_ERR_CUDA;
}

hmg_status hmg_sync(hmg_ctx* ctx, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  return guarded(ctx, [&] { cuda_ok(cudaStreamSynchronize(as_stream(stream)), "sync"); });
}

}  // extern "C"
