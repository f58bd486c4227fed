// Gather-scatter halo of one rank under an element partition (host only).
//
// Sec. 3.1 partitions the elements across ranks, one rank per GPU, and Sec. 2
// sums the values of shared element faces across them.  This build runs one
// GPU (replicas for several), but keeps the multi-rank split of QQ^T defined
// and testable: for a partition elem_rank[E] and one rank, the nodes whose
// copies lie on that rank and on others, with every copy (its rank and its
// index in that rank's local vector) in ascending global local index.  A rank
// that receives the other ranks' copy values of these nodes and sums every
// node's copies in that order gets QQ^T bit for bit as on one rank; nodes
// whose copies all lie on the rank need no exchange.
#include <cstring>
#include <vector>

#include "sem_internal.h"

using namespace sem;

extern "C" sem_status sem_gs_halo(int64_t E, int N, const int64_t* vert, const int32_t* elem_rank, int rank,
                                  int64_t* n_nodes, int64_t* n_copies, int64_t* node_gid, int64_t* node_ptr,
                                  int32_t* copy_rank, int64_t* copy_local) {
  SEM_TRACE("sem_gs_halo");
  if (!vert || !elem_rank || !n_nodes || !n_copies || E < 1) {
    set_error("sem_gs_halo: null argument or no elements");
    return SEM_ERR_INVALID;
  }
  const bool fill = node_gid != nullptr;
  if (fill && (!node_ptr || !copy_rank || !copy_local)) {
    set_error("sem_gs_halo: output arrays must all be given");
    return SEM_ERR_INVALID;
  }
  Topology t;
  sem_status st = build_numbering(E, N, vert, t);
  if (st != SEM_OK) return st;
  const int64_t n3 = (int64_t)(N + 1) * (N + 1) * (N + 1);
  // position of every element in its rank's local vector
  std::vector<int64_t> pos(E);
  {
    std::vector<int64_t> seen;
    for (int64_t e = 0; e < E; ++e) {
      const int32_t r = elem_rank[e];
      if (r < 0) {
        set_error("sem_gs_halo: negative rank");
        return SEM_ERR_INVALID;
      }
      if ((size_t)r >= seen.size()) seen.resize((size_t)r + 1, 0);
      pos[e] = seen[r]++;
    }
  }
  // per node: on `rank`?  on another rank?  number of copies
  std::vector<uint8_t> on_me(t.n_global, 0), on_other(t.n_global, 0);
  std::vector<int32_t> cnt(t.n_global, 0);
  for (int64_t l = 0; l < t.n_local; ++l) {
    const int64_t g = t.glo[l];
    if (elem_rank[l / n3] == rank) on_me[g] = 1;
    else on_other[g] = 1;
    cnt[g]++;
  }
  int64_t nn = 0, nc = 0;
  std::vector<int64_t> slot(t.n_global, -1);
  for (int64_t g = 0; g < t.n_global; ++g)
    if (on_me[g] && on_other[g]) {
      slot[g] = nn++;
      nc += cnt[g];
    }
  *n_nodes = nn;
  *n_copies = nc;
  if (!fill) return SEM_OK;
  // ascending global id, copies in ascending global local index
  node_ptr[0] = 0;
  {
    int64_t k = 0;
    for (int64_t g = 0; g < t.n_global; ++g)
      if (slot[g] >= 0) {
        node_gid[k] = g;
        node_ptr[k + 1] = node_ptr[k] + cnt[g];
        ++k;
      }
  }
  std::vector<int64_t> fillp(nn);
  for (int64_t k = 0; k < nn; ++k) fillp[k] = node_ptr[k];
  for (int64_t l = 0; l < t.n_local; ++l) {
    const int64_t s = slot[t.glo[l]];
    if (s < 0) continue;
    const int64_t e = l / n3;
    copy_rank[fillp[s]] = elem_rank[e];
    copy_local[fillp[s]] = pos[e] * n3 + (l - e * n3);
    ++fillp[s];
  }
  return SEM_OK;
}
