// Direct stiffness summation QQ^T over shared GLL nodes (Sec. 2: the
// "exchange of element face values" between neighbouring elements), then the
// Dirichlet mask.
//
// One thread per node.  Nodes are grouped by their number of copies m: for
// m = 2..8 a node is a fixed tuple of m local indices (ascending), so a
// thread loads its tuple and then the values -- one dependent step, no
// segment-pointer stream.  Nodes with more copies use a CSR class; Dirichlet
// nodes with a single copy only need zeroing.  The copies are summed in
// ascending local index, left to right, with explicit round-to-nearest adds
// (no contraction, no reordering), so the result is bit-identical to the
// same sum written as a plain loop.
#include "kernels.h"

namespace sem {

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

constexpr int kGsThreads = 256;

struct GsLaunch {
  GsDev g;
  int64_t blk[10];  // first block of each class; blk[9] = grid size
};

template <typename T, int M>
__device__ __forceinline__ void gs_tuple(T* __restrict__ v, const int32_t* __restrict__ id, int apply_mask) {
  int32_t ix[M];
#pragma unroll
  for (int c = 0; c < M; ++c) ix[c] = id[c];
  const bool dir = ix[0] < 0;
  ix[0] &= 0x7fffffff;
  if (apply_mask && dir) {
#pragma unroll
    for (int c = 0; c < M; ++c) v[ix[c]] = T(0);
    return;
  }
  T val[M];
#pragma unroll
  for (int c = 0; c < M; ++c) val[c] = v[ix[c]];
  T acc = val[0];
#pragma unroll
  for (int c = 1; c < M; ++c) acc = add_rn(acc, val[c]);
#pragma unroll
  for (int c = 0; c < M; ++c) v[ix[c]] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs(T* __restrict__ v, const GsLaunch L, int apply_mask,
                                                   const PcgState* __restrict__ st) {
  if (st && st->done) return;  // inside a CG chunk that already finished
  const int64_t b = blockIdx.x;
  int c = 0;
  while (c < 8 && b >= L.blk[c + 1]) ++c;
  const int64_t t = (b - L.blk[c]) * kGsThreads + threadIdx.x;
  if (t >= L.g.cnt[c]) return;
  const int32_t* base = L.g.idx + L.g.off[c];
  switch (c) {
    case 0: gs_tuple<T, 2>(v, base + 2 * t, apply_mask); break;
    case 1: gs_tuple<T, 3>(v, base + 3 * t, apply_mask); break;
    case 2: gs_tuple<T, 4>(v, base + 4 * t, apply_mask); break;
    case 3: gs_tuple<T, 5>(v, base + 5 * t, apply_mask); break;
    case 4: gs_tuple<T, 6>(v, base + 6 * t, apply_mask); break;
    case 5: gs_tuple<T, 7>(v, base + 7 * t, apply_mask); break;
    case 6: gs_tuple<T, 8>(v, base + 8 * t, apply_mask); break;
    case 7: {  // more than 8 copies
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
    default:  // Dirichlet node with one copy
      if (apply_mask) v[base[t] & 0x7fffffff] = T(0);
      break;
  }
}

template <typename T>
cudaError_t launch_gs(T* v, const GsDev& g, int apply_mask, const PcgState* st, cudaStream_t s) {
  GsLaunch L;
  L.g = g;
  int64_t nb = 0;
  for (int c = 0; c < 9; ++c) {
    L.blk[c] = nb;
    nb += (g.cnt[c] + kGsThreads - 1) / kGsThreads;
  }
  L.blk[9] = nb;
  if (nb == 0) return cudaSuccess;
  k_gs<T><<<(unsigned)nb, kGsThreads, 0, s>>>(v, L, apply_mask, st);
  return cudaGetLastError();
}

template cudaError_t launch_gs<double>(double*, const GsDev&, int, const PcgState*, cudaStream_t);
template cudaError_t launch_gs<float>(float*, const GsDev&, int, const PcgState*, cudaStream_t);

}  // namespace sem
