// Direct stiffness summation QQ^T over shared GLL nodes (Sec. 2: the
// "exchange of element face values" between neighbouring elements), then the
// Dirichlet mask.
//
// Nodes are grouped by their number of copies m: for m = 2..8 a node is a
// fixed tuple of m local indices (ascending), so a thread loads its tuple and
// then the values -- one dependent step, no segment-pointer stream.  Nodes with more copies use a CSR class; Dirichlet
// nodes with a single copy only need zeroing.  The copies are summed in
// ascending local index, left to right, with explicit round-to-nearest adds
// (no contraction, no reordering), so the result is bit-identical to the
// same sum written as a plain loop.
#include <type_traits>

#include "kernels.h"
#include "sem_internal.h"

namespace sem {

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

constexpr int kGsThreads = kGsUnitNodes;

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

// One node of m = M copies: load its tuple, then the values, sum in ascending
// local index, write the sum to every copy (or zero a Dirichlet node).
template <typename T, int M>
__device__ __forceinline__ void gs_tuple(T* __restrict__ v, const int32_t* __restrict__ id, int apply_mask) {
  int32_t ix[M];
  load_tuple<M>(id, ix);
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

// One CTA per work unit of the plan, one node per thread.  CTAs start in
// unit order, so the units in flight at any time cover about one window of
// global ids -- a few neighbouring element layers -- whose sectors stay in L2
// while their face, edge and vertex nodes are summed (measured on the
// E = 262,144 pipe: 20% less time in FP64 than class-by-class order; a
// persistent grid walking the same units was slower).
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs(T* __restrict__ v, const GsDev g, int apply_mask,
                                                   const PcgState* __restrict__ st) {
  if (st && st->done) return;  // inside a CG chunk that already finished
  {
    const int64_t u = blockIdx.x;
    const int4 w = g.units[u];
    if ((int)threadIdx.x >= w.z) return;
    const int c = w.x;
    const int64_t t = (int64_t)w.y + threadIdx.x;  // node within class c
    const int32_t* base = g.idx + g.off[c];
    switch (c) {
      case 0: gs_tuple<T, 2>(v, base + t * 2, apply_mask); break;
      case 1: gs_tuple<T, 3>(v, base + t * 3, apply_mask); break;
      case 2: gs_tuple<T, 4>(v, base + t * 4, apply_mask); break;
      case 3: gs_tuple<T, 5>(v, base + t * 5, apply_mask); break;
      case 4: gs_tuple<T, 6>(v, base + t * 6, apply_mask); break;
      case 5: gs_tuple<T, 7>(v, base + t * 7, apply_mask); break;
      case 6: gs_tuple<T, 8>(v, base + t * 8, apply_mask); break;
      case 7: {  // more than 8 copies
        const int32_t b0 = g.gptr[t], e0 = g.gptr[t + 1];
        const int32_t first = base[b0];
        if (apply_mask && first < 0) {
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
}

template <typename T>
cudaError_t launch_gs(T* v, const GsDev& g, int apply_mask, const PcgState* st, cudaStream_t s) {
  if (g.nunits == 0) return cudaSuccess;
  k_gs<T><<<(unsigned)g.nunits, kGsThreads, 0, s>>>(v, g, apply_mask, st);
  return cudaGetLastError();
}

template cudaError_t launch_gs<double>(double*, const GsDev&, int, const PcgState*, cudaStream_t);
template cudaError_t launch_gs<float>(float*, const GsDev&, int, const PcgState*, cudaStream_t);

}  // namespace sem
