// Horizontal domain decomposition of the column hierarchy (the paper's
// parallel design, Sec. 5: the horizontal domain is split over processes,
// each parallel loop is preceded by a halo exchange of the columns a process
// reads but does not own, and the Krylov solver's dot products are reduced
// over all processes).
//
// Parts are contiguous ranges of the hierarchical column order.  The split is
// made on the coarsest partitioned level, in whole tiles of 32 columns, and
// finer levels inherit it: the children 4C..4C+3 of an owned column C are
// owned by the same part, so restriction and prolongation never leave a
// part.  The coarsest level (below the partitioned ones) is gathered on one
// part.  Everything here is host code.
#include <algorithm>
#include <stdexcept>
#include <string>

#include "hmg_internal.h"

namespace hmg {

namespace {

int owner_of(const std::vector<int32_t>& bounds, int32_t col) {
  // bounds[p] = first column of part p, bounds[K] = ncols
  auto it = std::upper_bound(bounds.begin(), bounds.end(), col);
  return (int)(it - bounds.begin()) - 1;
}

}  // namespace

int partitioned_levels(int nlevels) { return nlevels > 1 ? nlevels - 1 : 1; }

PartitionPlan build_partition(const std::vector<std::vector<int32_t>>& nbr, const std::vector<int>& ncols,
                              int nparts) {
  const int nlev = (int)ncols.size();
  const int P = partitioned_levels(nlev);
  const int top = P - 1;   // coarsest partitioned level: the split is made here
  const int ntiles = (ncols[top] + TW - 1) / TW;
  if (nparts < 1 || nparts > ntiles)
    throw std::invalid_argument("nparts must be in [1, " + std::to_string(ntiles) +
                                "] (tiles of 32 columns on the coarsest partitioned level)");
  PartitionPlan plan;
  plan.nparts = nparts;
  plan.nlevels = P;
  plan.lv.resize(P);
  for (int l = 0; l < P; ++l) {
    const int64_t scale = int64_t(1) << (2 * (top - l));   // 4^(top - l)
    std::vector<int32_t> bounds(nparts + 1);
    for (int p = 0; p <= nparts; ++p) {
      const int64_t t = (int64_t)p * ntiles / nparts;
      bounds[p] = (int32_t)std::min<int64_t>((int64_t)ncols[l], t * TW * scale);
    }
    std::vector<PartLevel>& parts = plan.lv[l];
    parts.resize(nparts);
    for (int p = 0; p < nparts; ++p) {
      PartLevel& pl = parts[p];
      pl.begin = bounds[p];
      pl.end = bounds[p + 1];
      pl.n_own = pl.end - pl.begin;
      pl.n_own_pad = (pl.n_own + TW - 1) / TW * TW;
      // ghosts: neighbours outside the range, sorted by (owner, column)
      std::vector<std::pair<int, int32_t>> g;
      for (int32_t c = pl.begin; c < pl.end; ++c)
        for (int k = 0; k < 3; ++k) {
          const int32_t n = nbr[l][(size_t)c * 3 + k];
          if (n < pl.begin || n >= pl.end) g.emplace_back(owner_of(bounds, n), n);
        }
      std::sort(g.begin(), g.end());
      g.erase(std::unique(g.begin(), g.end()), g.end());
      pl.ghost_col.resize(g.size());
      pl.ghost_owner.resize(g.size());
      pl.ghost_owner_local.resize(g.size());
      for (size_t i = 0; i < g.size(); ++i) {
        pl.ghost_owner[i] = g[i].first;
        pl.ghost_col[i] = g[i].second;
        pl.ghost_owner_local[i] = g[i].second - bounds[g[i].first];
      }
      pl.local_nbr.resize((size_t)pl.n_own * 3);
      for (int32_t c = pl.begin; c < pl.end; ++c)
        for (int k = 0; k < 3; ++k) {
          const int32_t n = nbr[l][(size_t)c * 3 + k];
          int32_t loc;
          if (n >= pl.begin && n < pl.end) {
            loc = n - pl.begin;
          } else {
            const auto key = std::make_pair(owner_of(bounds, n), n);
            const size_t i = (size_t)(std::lower_bound(g.begin(), g.end(), key) - g.begin());
            loc = pl.n_own_pad + (int32_t)i;
          }
          pl.local_nbr[(size_t)(c - pl.begin) * 3 + k] = loc;
        }
    }
    // send lists: part p sends to each q, in q's ghost order, the columns of
    // q's ghost list that p owns
    for (int p = 0; p < nparts; ++p) {
      PartLevel& pl = parts[p];
      for (int q = 0; q < nparts; ++q) {
        if (q == p) continue;
        const PartLevel& ql = parts[q];
        for (size_t i = 0; i < ql.ghost_col.size(); ++i)
          if (ql.ghost_owner[i] == p) {
            pl.send_col.push_back(ql.ghost_col[i]);
            pl.send_to.push_back(q);
          }
      }
    }
  }
  return plan;
}

PartitionPlan build_partition_for_mesh(int refinement, int nlevels, int nparts) {
  const std::vector<HostLevel> hl = build_mesh_hierarchy(refinement, nlevels);
  std::vector<std::vector<int32_t>> nbr;
  std::vector<int> ncols;
  for (const HostLevel& h : hl) {
    nbr.push_back(h.nbr);
    ncols.push_back(h.ncols);
  }
  return build_partition(nbr, ncols, nparts);
}

}  // namespace hmg
