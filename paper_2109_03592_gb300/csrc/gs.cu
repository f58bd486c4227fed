// Direct stiffness summation QQ^T over shared GLL nodes (Sec. 2: the
// "exchange of element face values" between neighbouring elements), then the
// Dirichlet mask.
//
// One thread per segment (a global node with several copies or on a
// Dirichlet face).  The copies are summed in ascending local index, left to
// right, with explicit round-to-nearest adds (no contraction, no reordering),
// so the result is bit-identical to the same sum written as a plain loop.
#include "kernels.h"

namespace sem {

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

template <typename T>
__global__ void k_gs(T* __restrict__ v, const int32_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_idx,
                     const uint8_t* __restrict__ seg_dir, int64_t nseg, int apply_mask,
                     const PcgState* __restrict__ st) {
  if (st && st->done) return;  // inside a CG chunk that already finished
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = seg_ptr[s], e = seg_ptr[s + 1];
    if (apply_mask && seg_dir[s]) {
      for (int32_t q = b; q < e; ++q) v[seg_idx[q]] = T(0);
      continue;
    }
    if (e - b < 2) continue;
    T acc = v[seg_idx[b]];
    for (int32_t q = b + 1; q < e; ++q) acc = add_rn(acc, v[seg_idx[q]]);
    for (int32_t q = b; q < e; ++q) v[seg_idx[q]] = acc;
  }
}

template <typename T>
cudaError_t launch_gs(T* v, const int32_t* seg_ptr, const int32_t* seg_idx, const uint8_t* seg_dir, int64_t nseg,
                      int apply_mask, const PcgState* st, cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  int64_t grid = (nseg + 255) / 256;
  if (grid > 152LL * 64) grid = 152LL * 64;
  k_gs<T><<<(unsigned)grid, 256, 0, s>>>(v, seg_ptr, seg_idx, seg_dir, nseg, apply_mask, st);
  return cudaGetLastError();
}

template cudaError_t launch_gs<double>(double*, const int32_t*, const int32_t*, const uint8_t*, int64_t, int,
                                       const PcgState*, cudaStream_t);
template cudaError_t launch_gs<float>(float*, const int32_t*, const int32_t*, const uint8_t*, int64_t, int,
                                      const PcgState*, cudaStream_t);

}  // namespace sem
