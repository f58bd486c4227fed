// Direct stiffness summation QQ^T over shared GLL nodes (Sec. 2: the
// "exchange of element face values" between neighbouring elements), then the
// Dirichlet mask.
//
// Nodes are grouped by their number of copies m: for m = 2..8 a node is a
// fixed tuple of m local indices (ascending), so a thread loads its tuples
// and then the values -- one dependent step, no segment-pointer stream --
// for several nodes at once.  Nodes with more copies use a CSR class; Dirichlet
// nodes with a single copy only need zeroing.  The copies are summed in
// ascending local index, left to right, with explicit round-to-nearest adds
// (no contraction, no reordering), so the result is bit-identical to the
// same sum written as a plain loop.
#include <type_traits>

#include "kernels.h"

namespace sem {

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

constexpr int kGsThreads = 256;

struct GsLaunch {
  GsDev g;
  int64_t blk[10];  // first block of each class; blk[9] = grid size
};

// Nodes per thread of class m (one: more nodes per thread throttled the
// load/store queue on GB300 and ran slower).
__host__ __device__ constexpr int gs_npt(int) { return 1; }

// The m indices of one node; tuples of 2, 4, 6 and 8 are 8-byte aligned
// (every class starts 16-byte aligned) and load as int2 / int4 vectors.
template <int M>
__device__ __forceinline__ void load_tuple(const int32_t* __restrict__ id, int32_t (&ix)[M]) {
  if constexpr (M % 4 == 0) {
#pragma unroll
    for (int c = 0; c < M; c += 4) {
      const int4 q = *reinterpret_cast<const int4*>(id + c);
      ix[c] = q.x; ix[c + 1] = q.y; ix[c + 2] = q.z; ix[c + 3] = q.w;
    }
  } else if constexpr (M % 2 == 0) {
#pragma unroll
    for (int c = 0; c < M; c += 2) {
      const int2 q = *reinterpret_cast<const int2*>(id + c);
      ix[c] = q.x; ix[c + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < M; ++c) ix[c] = id[c];
  }
}

// NPT nodes of m = M copies each: node q at id + q * stride * M.
template <typename T, int M, int NPT>
__device__ __forceinline__ void gs_tuples(T* __restrict__ v, const int32_t* __restrict__ id, int64_t first_node,
                                          int64_t count, int apply_mask) {
  int32_t ix[NPT][M];
  bool ok[NPT];
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int64_t node = first_node + (int64_t)q * kGsThreads;
    ok[q] = node < count;
    if (ok[q]) load_tuple<M>(id + node * M, ix[q]);
  }
  T val[NPT][M];
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    if (!ok[q]) continue;
    const bool dir = ix[q][0] < 0;
    ix[q][0] &= 0x7fffffff;
    if (apply_mask && dir) {
      ok[q] = false;
#pragma unroll
      for (int c = 0; c < M; ++c) v[ix[q][c]] = T(0);
      continue;
    }
#pragma unroll
    for (int c = 0; c < M; ++c) val[q][c] = v[ix[q][c]];
  }
#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    if (!ok[q]) continue;
    T acc = val[q][0];
#pragma unroll
    for (int c = 1; c < M; ++c) acc = add_rn(acc, val[q][c]);
#pragma unroll
    for (int c = 0; c < M; ++c) v[ix[q][c]] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs(T* __restrict__ v, const GsLaunch L, int apply_mask,
                                                   const PcgState* __restrict__ st) {
  if (st && st->done) return;  // inside a CG chunk that already finished
  const int64_t b = blockIdx.x;
  int c = 0;
  while (c < 8 && b >= L.blk[c + 1]) ++c;
  const int64_t rel = b - L.blk[c];
  const int32_t* base = L.g.idx + L.g.off[c];
  const int64_t cnt = L.g.cnt[c];
#define GS_CASE(CLS, M)                                                                             \
  case CLS: {                                                                                       \
    constexpr int NPT = gs_npt(M);                                                                  \
    gs_tuples<T, M, NPT>(v, base, rel * kGsThreads * NPT + threadIdx.x, cnt, apply_mask);           \
    break;                                                                                          \
  }
  switch (c) {
    GS_CASE(0, 2)
    GS_CASE(1, 3)
    GS_CASE(2, 4)
    GS_CASE(3, 5)
    GS_CASE(4, 6)
    GS_CASE(5, 7)
    GS_CASE(6, 8)
    case 7: {  // more than 8 copies
      const int64_t t = rel * kGsThreads + threadIdx.x;
      if (t >= cnt) break;
      const int32_t b0 = L.g.gptr[t], e0 = L.g.gptr[t + 1];
      const int32_t first = base[b0];
      const bool dir = first < 0;
      if (apply_mask && dir) {
        v[first & 0x7fffffff] = T(0);
        for (int32_t q = b0 + 1; q < e0; ++q) v[base[q]] = T(0);
        break;
      }
      T acc = v[first & 0x7fffffff];
      for (int32_t q = b0 + 1; q < e0; ++q) acc = add_rn(acc, v[base[q]]);
      v[first & 0x7fffffff] = acc;
      for (int32_t q = b0 + 1; q < e0; ++q) v[base[q]] = acc;
      break;
    }
    default: {  // Dirichlet node with one copy
      const int64_t t = rel * kGsThreads + threadIdx.x;
      if (t < cnt && apply_mask) v[base[t] & 0x7fffffff] = T(0);
      break;
    }
  }
#undef GS_CASE
}

template <typename T>
cudaError_t launch_gs(T* v, const GsDev& g, int apply_mask, const PcgState* st, cudaStream_t s) {
  GsLaunch L;
  L.g = g;
  int64_t nb = 0;
  for (int c = 0; c < 9; ++c) {
    L.blk[c] = nb;
    const int64_t per_block = (int64_t)kGsThreads * (c < 7 ? gs_npt(c + 2) : 1);
    nb += (g.cnt[c] + per_block - 1) / per_block;
  }
  L.blk[9] = nb;
  if (nb == 0) return cudaSuccess;
  k_gs<T><<<(unsigned)nb, kGsThreads, 0, s>>>(v, L, apply_mask, st);
  return cudaGetLastError();
}

template cudaError_t launch_gs<double>(double*, const GsDev&, int, const PcgState*, cudaStream_t);
template cudaError_t launch_gs<float>(float*, const GsDev&, int, const PcgState*, cudaStream_t);

}  // namespace sem
