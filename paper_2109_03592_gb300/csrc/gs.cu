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

constexpr int kGsThreads = kGsUnitNodes;  // nodes per work unit
// Two nodes per thread, their loads interleaved: measured on GB300
// (E = 262,144, N = 7) 0.46 -> 0.36 ms FP32 and 0.59 -> 0.50 ms FP64 against
// one node per thread; four per thread was no faster.

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


// Two nodes of m = M copies, their loads interleaved (both tuples, then all
// values); sums in ascending local index, written to every copy (a Dirichlet
// node is zeroed instead when the mask applies).
template <typename T, int M>
__device__ __forceinline__ void gs_tuple2(T* __restrict__ v, const int32_t* __restrict__ ida,
                                          const int32_t* __restrict__ idb, bool hb, int apply_mask) {
  int32_t xa[M], xb[M];
  load_tuple<M>(ida, xa);
  if (hb) load_tuple<M>(idb, xb);
  const bool da = xa[0] < 0, db = hb && xb[0] < 0;
  xa[0] &= 0x7fffffff;
  if (hb) xb[0] &= 0x7fffffff;
  const bool ga = !(apply_mask && da), gb = hb && !(apply_mask && db);
  T va[M], vb[M];
#pragma unroll
  for (int c = 0; c < M; ++c) va[c] = ga ? v[xa[c]] : T(0);
#pragma unroll
  for (int c = 0; c < M; ++c) vb[c] = gb ? v[xb[c]] : T(0);
  T sa = va[0], sb = vb[0];
#pragma unroll
  for (int c = 1; c < M; ++c) {
    sa = add_rn(sa, va[c]);
    sb = add_rn(sb, vb[c]);
  }
#pragma unroll
  for (int c = 0; c < M; ++c) v[xa[c]] = ga ? sa : T(0);
  if (hb) {
#pragma unroll
    for (int c = 0; c < M; ++c) v[xb[c]] = gb ? sb : T(0);
  }
}

// One CTA per work unit of the plan (kGsThreads nodes), two nodes per thread
// (the unit's nodes tid and tid + kGsThreads / 2).  CTAs start in unit order,
// so the units in flight at any time cover about one window of global ids --
// a few neighbouring element layers -- whose sectors stay in L2 while their
// face, edge and vertex nodes are summed (measured on the E = 262,144 pipe:
// 20% less time in FP64 than class-by-class order; a persistent grid walking
// the same units was slower).
template <typename T>
__global__ void __launch_bounds__(kGsThreads / 2) k_gs(T* __restrict__ v, const GsDev g, int apply_mask,
                                                       const PcgState* __restrict__ st) {
  if (st && st->done) return;  // inside a CG chunk that already finished
  const int4 w = g.units[blockIdx.x];
  const int c = w.x, ja = threadIdx.x, jb = threadIdx.x + kGsThreads / 2;
  if (ja >= w.z) return;
  const bool hb = jb < w.z;
  const int64_t ta = (int64_t)w.y + ja, tb = (int64_t)w.y + jb;  // nodes within class c
  const int32_t* base = g.idx + g.off[c];
  switch (c) {
    case 0: gs_tuple2<T, 2>(v, base + ta * 2, base + tb * 2, hb, apply_mask); break;
    case 1: gs_tuple2<T, 3>(v, base + ta * 3, base + tb * 3, hb, apply_mask); break;
    case 2: gs_tuple2<T, 4>(v, base + ta * 4, base + tb * 4, hb, apply_mask); break;
    case 3: gs_tuple2<T, 5>(v, base + ta * 5, base + tb * 5, hb, apply_mask); break;
    case 4: gs_tuple2<T, 6>(v, base + ta * 6, base + tb * 6, hb, apply_mask); break;
    case 5: gs_tuple2<T, 7>(v, base + ta * 7, base + tb * 7, hb, apply_mask); break;
    case 6: gs_tuple2<T, 8>(v, base + ta * 8, base + tb * 8, hb, apply_mask); break;
    default:
      for (int r = 0; r < 2; ++r) {
        if (r == 1 && !hb) break;
        const int64_t t = r ? tb : ta;
        if (c == 7) {  // more than 8 copies
          const int32_t b0 = g.gptr[t], e0 = g.gptr[t + 1];
          const int32_t first = base[b0];
          if (apply_mask && first < 0) {
            v[first & 0x7fffffff] = T(0);
            for (int32_t q = b0 + 1; q < e0; ++q) v[base[q]] = T(0);
            continue;
          }
          T acc = v[first & 0x7fffffff];
          for (int32_t q = b0 + 1; q < e0; ++q) acc = add_rn(acc, v[base[q]]);
          v[first & 0x7fffffff] = acc;
          for (int32_t q = b0 + 1; q < e0; ++q) v[base[q]] = acc;
        } else if (apply_mask) {  // Dirichlet node with one copy
          v[base[t] & 0x7fffffff] = T(0);
        }
      }
  }
}

template <typename T>
cudaError_t launch_gs(T* v, const GsDev& g, int apply_mask, const PcgState* st, cudaStream_t s) {
  if (g.nunits == 0) return cudaSuccess;
  k_gs<T><<<(unsigned)g.nunits, kGsThreads / 2, 0, s>>>(v, g, apply_mask, st);
  return cudaGetLastError();
}

template cudaError_t launch_gs<double>(double*, const GsDev&, int, const PcgState*, cudaStream_t);
template cudaError_t launch_gs<float>(float*, const GsDev&, int, const PcgState*, cudaStream_t);

}  // namespace sem
