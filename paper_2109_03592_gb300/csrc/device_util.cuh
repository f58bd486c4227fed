// Small device helpers shared by the kernels: deterministic block reductions
// and the "last block finishes the grid reduction" pattern.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sem {

// Scalars of one CG run, resident in device memory so that a whole iteration
// runs without a host round trip (Sec. 3: hand-written reduction kernels,
// data kept on the device).
struct PcgState {
  double rho;    // <r, z> of the current iterate
  double alpha;  // rho / <p, A p>
  double beta;   // rho_new / rho_old (0 before the first direction)
  double pAp;
  double rr;     // <r, r>
  double bb;     // <b, b> of the system being solved
  double tol2;   // tol^2
  double aux;    // scratch scalar (outer residual norms)
  double rr_max; // largest <r, r> since the last reliable update
  double delta2; // reliable-update trigger: pause when <r,r> <= delta2 * rr_max (0 = never)
  double cz;     // pressure CG: mean of D^-1 r (aux holds the mean of E q)
  double alpha_prev;  // CG with x updated every second iteration: alpha of the pending direction
  int last;      // pressure CG: iteration of the last residual replacement
  int xpend;     // 1 while x lacks alpha_prev times the last direction
  int iter;
  int maxit;
  int done;      // 1 once converged / failed / paused: later kernels of the chunk return at once
  int ru;        // 1 when paused for a reliable update (FP64 residual replacement)
  int status;    // sem_status of the run
  unsigned int cnt[4];  // arrival counters of the grid reductions
};

#ifdef __CUDACC__
// Sum over a block in a fixed order (warp shuffles, then one warp over the
// per-warp sums).  Deterministic for a fixed blockDim.  `sbuf` needs
// blockDim.x / 32 entries.  The result is valid in thread 0.
template <typename A>
__device__ __forceinline__ A warp_sum_prefix(A v, int nact) {
  // lanes >= nact do not exist (a partial last warp): their values are not added
  const unsigned mask = nact >= 32 ? 0xffffffffu : ((1u << nact) - 1u);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const A other = __shfl_down_sync(mask, v, o);
    if (lane + o < nact) v += other;
  }
  return v;
}

template <typename A>
__device__ __forceinline__ A block_sum(A v, A* sbuf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const int nact = min(32, (int)blockDim.x - wid * 32);
  v = warp_sum_prefix(v, nact);
  __syncthreads();  // sbuf may still be read by a previous call
  if (lane == 0) sbuf[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < nw ? sbuf[lane] : A(0);
    v = warp_sum_prefix(v, nact);
  }
  return v;
}

// Called by every thread after thread 0 wrote this block's partial(s) with
// plain stores.  Returns true in exactly one block (the last to arrive);
// that block then sees every other block's partials.
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Fixed-order sum of partials[0..count) with stride `stride` by one block.
__device__ __forceinline__ double sum_partials(const double* partials, int count, int stride, int offset,
                                               double* sbuf) {
  double v = 0.0;
  for (int q = threadIdx.x; q < count; q += blockDim.x) v += __ldcg(partials + (size_t)q * stride + offset);
  return block_sum(v, sbuf);
}
#endif  // __CUDACC__

}  // namespace sem
