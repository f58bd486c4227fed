// FP32 local operator (Alg. 1 + h2 B u) as a persistent kernel fed by the
// Blackwell bulk-copy (TMA) engine.
//
// The plain FP32 kernel (ax_impl.cuh) moves exactly the algorithmic bytes
// but is latency bound: each thread waits on its own global loads of u and
// the six factors, and register pressure caps the resident warps.  Here
// every CTA is persistent and walks tiles of EPB consecutive elements.  The
// tile's inputs are contiguous in HBM (u or z,p: EPB n^3 floats; G:
// EPB 6 n^3 floats), so one thread issues them as 1-D bulk copies
// (cp.async.bulk ... mbarrier::complete_tx) into a ring of STAGES shared
// buffers, STAGES tiles ahead of the compute.  Consumers wait on the
// stage's mbarrier (bounded spin: after kSpinLimit polls the kernel records
// SEM_ERR_DEVICE_TIMEOUT in *err, drains what it issued and returns) and
// read u and G from shared memory.
//
// Requirements: n = N+1 even (n^3 floats per element is a multiple of 16
// bytes, so every copy starts 16-byte aligned), FP32 data.
#pragma once

#include "kernels.h"
#include "tma_util.cuh"

namespace sem {
namespace tma {

template <int N, int EPB, bool FUSED>
struct Layout {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int in_vec = FUSED ? 2 : 1;                   // u, or z and p
  static constexpr int stage_floats = in_vec * EPB * n3 + EPB * 6 * n3;
  static constexpr size_t stage_bytes = sizeof(float) * stage_floats;
  static constexpr int work_floats = n * n + 2 * EPB * n3;        // D, wr, ws
};

template <int N, int EPB, int STAGES, bool FUSED>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1)) k_ax_tma(const AxParams<float> P, int* err) {
  using Lay = Layout<N, EPB, FUSED>;
  constexpr int n = Lay::n, n2 = Lay::n2, n3 = Lay::n3;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  float* sD = stage0 + STAGES * Lay::stage_floats;  // D[a][b] at a*n + b
  float* swr = sD + n * n;
  float* sws = swr + EPB * n3;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sws + EPB * n3);  // 8-byte aligned (even float count above)
  __shared__ double sred[32];
  __shared__ int sflag;

  const int tid = threadIdx.x;
  if (FUSED) {
    if (tid == 0) sflag = P.st->done;
    __syncthreads();
    if (sflag) return;
  }
  const int64_t ntiles = (P.E + EPB - 1) / EPB;
  for (int q = tid; q < n2; q += blockDim.x) sD[q] = P.D[q];
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    sflag = 0;
  }
  __syncthreads();

  // one thread issues the copies of a tile into a stage
  auto issue = [&](int s, int64_t tile) {
    const int64_t e0 = tile * EPB;
    const int ne = (int)min((int64_t)EPB, P.E - e0);
    float* st = stage0 + s * Lay::stage_floats;
    const uint32_t bu = (uint32_t)(ne * n3 * sizeof(float)), bg = 6u * bu;
    mbar_expect_tx(&bars[s], Lay::in_vec * bu + bg);
    if (FUSED) {
      bulk_g2s(st, P.z + e0 * n3, bu, &bars[s]);
      bulk_g2s(st + EPB * n3, P.p + e0 * n3, bu, &bars[s]);
    } else {
      bulk_g2s(st, P.u + e0 * n3, bu, &bars[s]);
    }
    bulk_g2s(st + Lay::in_vec * EPB * n3, P.G + e0 * 6 * n3, bg, &bars[s]);
  };
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      const int64_t tile = blockIdx.x + (int64_t)s * gridDim.x;
      if (tile < ntiles) issue(s, tile);
    }
  }

  const int le = tid / n2, ij = tid - le * n2, i = ij % n, j = ij / n;
  const float beta = FUSED ? (float)P.st->beta : 0.f;
  float pw = 0.f;
  int64_t it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = (int)(it % STAGES);
    const uint32_t parity = (uint32_t)((it / STAGES) & 1);
    if (!mbar_wait(&bars[s], parity)) sflag = 1;  // benign race: every writer stores 1
    __syncthreads();
    if (sflag) break;
    float* st = stage0 + s * Lay::stage_floats;
    float* su = st + le * n3;  // u, or z then overwritten by p = z + beta p
    const float* sG = st + Lay::in_vec * EPB * n3 + le * 6 * n3;
    const int64_t e = tile * EPB + le;
    const bool act = e < P.E;
    const int64_t base = e * n3 + ij;

    // h2 B u: B does not go through the copy ring (the Poisson operator
    // needs no room for it).  Its n values are loaded here, before any store
    // of this tile, so that their latency overlaps the contractions; loaded
    // next to the stores of w, each load waited in turn (3x the time).
    float rb[n];
#pragma unroll
    for (int k = 0; k < n; ++k) rb[k] = (act && P.helm) ? __ldg(P.B + base + k * n2) : 0.f;

    float ru[n];
    if (act) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        float v = su[k * n2 + ij];
        if (FUSED) {
          v += beta * st[EPB * n3 + le * n3 + k * n2 + ij];
          su[k * n2 + ij] = v;
          (P.pout ? P.pout : P.p)[base + k * n2] = v;
        }
        ru[k] = v;
      }
    }
    if (FUSED) __syncthreads();

    float rw[n];
#pragma unroll
    for (int k = 0; k < n; ++k) rw[k] = 0.f;
    if (act) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const float g1 = sG[k * n2 + ij], g2 = sG[n3 + k * n2 + ij], g3 = sG[2 * n3 + k * n2 + ij];
        const float g4 = sG[3 * n3 + k * n2 + ij], g5 = sG[4 * n3 + k * n2 + ij], g6 = sG[5 * n3 + k * n2 + ij];
        float ur = 0.f, us = 0.f, ut = 0.f;
#pragma unroll
        for (int l = 0; l < n; ++l) {
          ur += sD[i * n + l] * su[k * n2 + j * n + l];
          us += sD[j * n + l] * su[k * n2 + l * n + i];
          ut += sD[k * n + l] * ru[l];
        }
        const float wr = g1 * ur + g4 * us + g5 * ut;
        const float ws = g4 * ur + g2 * us + g6 * ut;
        const float wt = g5 * ur + g6 * us + g3 * ut;
        swr[le * n3 + k * n2 + ij] = wr;
        sws[le * n3 + k * n2 + ij] = ws;
#pragma unroll
        for (int k2 = 0; k2 < n; ++k2) rw[k2] += sD[k * n + k2] * wt;
      }
    }
    __syncthreads();
    // the stage is free: refill it with the tile STAGES ahead
    if (tid == 0) {
      const int64_t next = tile + (int64_t)STAGES * gridDim.x;
      if (next < ntiles) {
        fence_async_smem();
        issue(s, next);
      }
    }
    if (act) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        float acc = rw[k];
#pragma unroll
        for (int l = 0; l < n; ++l)
          acc += sD[l * n + i] * swr[le * n3 + k * n2 + j * n + l] + sD[l * n + j] * sws[le * n3 + k * n2 + l * n + i];
        float out = P.h1 * acc;
        if (P.helm) out += P.h2 * rb[k] * ru[k];
        P.w[base + k * n2] = out;
        if (FUSED) pw += ru[k] * out;
      }
    }
    __syncthreads();  // swr / sws are rewritten by the next tile
  }

  if (sflag) {
    // drain the copies this CTA issued and still owns (bounded), record the error
    if (tid == 0) {
      atomicExch(err, 7);  // SEM_ERR_DEVICE_TIMEOUT
      for (int64_t k = 0; k < STAGES; ++k) {
        const int64_t t2 = blockIdx.x + (it + k) * gridDim.x;
        if (t2 < ntiles) mbar_wait(&bars[(it + k) % STAGES], (uint32_t)(((it + k) / STAGES) & 1));
      }
      if (FUSED) {
        P.st->status = 7;
        P.st->done = 1;
      }
    }
    return;
  }

  if (FUSED) {
    const double s = block_sum((double)pw, sred);
    if (tid == 0) P.partial[blockIdx.x] = s;
    if (last_block(&P.st->cnt[0])) {
      const double pAp = sum_partials(P.partial, gridDim.x, 1, 0, sred);
      if (tid == 0) {
        PcgState* stt = P.st;
        stt->pAp = pAp;
        if (stt->done) {
          // a CTA timed out above; keep its status
        } else if (!(pAp > 0.0)) {
          stt->done = 1;
          stt->status = 5;  // SEM_ERR_BREAKDOWN
        } else {
          stt->alpha = stt->rho / pAp;
        }
        stt->cnt[0] = 0;
      }
    }
  }
}

template <int N, int EPB, int STAGES, bool FUSED>
size_t tma_smem_bytes() {
  using Lay = Layout<N, EPB, FUSED>;
  return STAGES * Lay::stage_bytes + sizeof(float) * Lay::work_floats + STAGES * sizeof(uint64_t);
}

// Persistent grid: as many CTAs as fit on the device (at most one per tile).
template <int N, int EPB, int STAGES, bool FUSED>
cudaError_t launch_ax_tma_t(const AxParams<float>& p, int* err, cudaStream_t s, int* grid_out) {
  constexpr int n = N + 1;
  const size_t smem = tma_smem_bytes<N, EPB, STAGES, FUSED>();
  static DeviceOnce once;  // CTAs per device, computed once per device
  int grid_cap = 0;
  cudaError_t oerr = once.get(
      [&](int dev, int* cap) {
        cudaError_t e = cudaFuncSetAttribute(k_ax_tma<N, EPB, STAGES, FUSED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_tma<N, EPB, STAGES, FUSED>, EPB * n * n,
                                                          smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        *cap = per_sm * sms;
        return cudaSuccess;
      },
      &grid_cap);
  if (oerr != cudaSuccess) return oerr;
  const int64_t ntiles = (p.E + EPB - 1) / EPB;
  const int grid = (int)std::min<int64_t>(ntiles, grid_cap);
  if (grid_out) *grid_out = grid;
  if (p.E == 0) return cudaSuccess;
  k_ax_tma<N, EPB, STAGES, FUSED><<<grid, EPB * n * n, smem, s>>>(p, err);
  return cudaGetLastError();
}

}  // namespace tma
}  // namespace sem
