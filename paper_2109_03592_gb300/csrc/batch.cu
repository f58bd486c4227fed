// Batched mixed-precision PCG: one CUDA graph advances every active request
// of one polynomial order by kChunk CG iterations.
//
// Requests (ragged element counts, own meshes, own h1/h2 and tolerances) sit
// in the slots of a device table.  The four batched kernels of an iteration
// read sizes and pointers from that table, so the captured graph stays
// valid while requests join, pause and leave:
//   k_bax     persistent, bulk-copy pipelined FP32 A_L over the concatenated
//             element tiles of all live requests (p <- z + beta p fused),
//             one <p, A_L p> partial per tile
//   k_balpha  one block per request: fixed-order sum of its tile partials,
//             alpha = rho / pAp
//   k_bgs     QQ^T + mask over (request, multiplicity class) virtual blocks
//   k_bupdate x, r, z update over per-request virtual blocks; the last
//             block of a request reduces <r,z>, <r,r> in fixed order and
//             applies the stop / reliable-update test
// Every reduction runs over one request's own tiles or blocks in a fixed
// order, so a request's result does not depend on what else is batched.
// The FP64 parts of the reliable-update scheme (x += x32, r = b - A64 x,
// residual replacement) run per request between graph launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "ax_impl.cuh"
#include "kernels.h"
#include "sem_internal.h"
#include "batch.h"
#include "solver.h"

namespace sem {
namespace batch {

constexpr int kMaxSlots = 32;
constexpr int kChunk = 8;
constexpr int kVecThreads = 256;
constexpr int kVecW = 8;  // floats per thread per virtual block (two 16-byte vectors)
constexpr int kTileGroup = 8;  // consecutive tiles of one request per <p, A p> partial
constexpr int kVecPts = kVecThreads * kVecW;
constexpr int kGsThreads = 256;

struct Slot {
  const float* G;
  const float* B;
  const float* D;
  const uint8_t* wm;
  const int32_t* gs_idx;
  const int32_t* gs_ptr;
  int64_t gs_off[9];
  int64_t gs_cnt[9];
  float* x;
  float* r;
  float* z;
  float* p;
  float* w;
  const float* minv;
  PcgState* st;
  float h1, h2;
  int helm;
  int active;
  int64_t E, n_local;
};

struct Table {
  int nslots;
  const float* D;  // derivative matrix of the table's order (any active request's copy)
  Slot s[kMaxSlots];
  int64_t tile_off[kMaxSlots + 1];
  int64_t grp_off[kMaxSlots + 1];  // tile groups (kTileGroup tiles) per request, prefix
  int64_t gs_vb[kMaxSlots * 9 + 1];
  int64_t vec_vb[kMaxSlots + 1];
  unsigned int cnt[kMaxSlots];
};

__device__ __forceinline__ int find_slot(const int64_t* off, int n, int64_t t) {
  int lo = 0, hi = n;  // off[lo] <= t < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool live(const Slot& s) { return s.active && !s.st->done; }

// ---- batched fused FP32 local operator (even n) ------------------------------
template <int N, int EPB, int STAGES>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1)) k_bax(const Table* __restrict__ T, double* part_tile,
                                                                 int* err) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  using Lay = tma::Layout<N, EPB, true>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  float* sD = stage0 + STAGES * Lay::stage_floats;
  float* swr = sD + n * n;
  float* sws = swr + EPB * n3;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sws + EPB * n3);
  __shared__ int slive[kMaxSlots];
  __shared__ int64_t stoff[kMaxSlots + 1];
  __shared__ int64_t sgoff[kMaxSlots + 1];
  __shared__ int snslots, sflag;
  __shared__ double sred[32];

  const int tid = threadIdx.x;
  if (tid == 0) {
    snslots = T->nslots;
    sflag = 0;
  }
  __syncthreads();
  const int ns = snslots;
  int any = 0;
  for (int r = tid; r < ns; r += blockDim.x) any |= (slive[r] = live(T->s[r]));
  // every request paused or finished (the rest of a chunk after its last
  // iteration): return before any set-up
  if (!__syncthreads_or(any)) return;
  for (int r = tid; r <= ns; r += blockDim.x) {
    stoff[r] = T->tile_off[r];
    sgoff[r] = T->grp_off[r];
  }
  for (int q = tid; q < n2; q += blockDim.x) sD[q] = T->D[q];  // one order per table
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) tma::mbar_init(&bars[s], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  // Work comes in tile groups: kTileGroup consecutive tiles of one request,
  // taken by the CTAs in grid strides.  A group's <p, A p> partial is summed
  // by the one CTA that runs it, in tile order, so it does not depend on the
  // other requests in the table (a request's result is the same alone and in
  // a batch) and costs one block reduction per group instead of per tile.
  const int64_t gtotal = sgoff[ns];
  auto next_group = [&](int64_t g) {
    while (g < gtotal && !slive[find_slot(sgoff, ns, g)]) g += gridDim.x;
    return g;
  };
  auto group_tiles = [&](int64_t g, int64_t& t0) {  // first tile and tile count of group g
    const int r = find_slot(sgoff, ns, g);
    const int64_t lt = (g - sgoff[r]) * kTileGroup;
    t0 = stoff[r] + lt;
    return (int)min((int64_t)kTileGroup, stoff[r + 1] - stoff[r] - lt);
  };
  auto issue = [&](int s, int64_t t) {
    const int r = find_slot(stoff, ns, t);
    const Slot& sl = T->s[r];
    const int64_t e0 = (t - stoff[r]) * EPB;
    const int ne = (int)min((int64_t)EPB, sl.E - e0);
    float* st = stage0 + s * Lay::stage_floats;
    const uint32_t bu = (uint32_t)(ne * n3 * sizeof(float)), bg = 6u * bu;
    tma::mbar_expect_tx(&bars[s], 2 * bu + bg);
    tma::bulk_g2s(st, sl.z + e0 * n3, bu, &bars[s]);
    tma::bulk_g2s(st + EPB * n3, sl.p + e0 * n3, bu, &bars[s]);
    tma::bulk_g2s(st + 2 * EPB * n3, sl.G + e0 * 6 * n3, bg, &bars[s]);
  };
  // producer cursor (thread 0): group pg, tile pk of pn in it, from tile pt0
  int64_t pg = next_group(blockIdx.x), pt0 = 0;
  int pk = 0, pn = pg < gtotal ? group_tiles(pg, pt0) : 0;
  auto padvance = [&]() {
    if (++pk < pn) return;
    pg = next_group(pg + gridDim.x);
    pk = 0;
    pn = pg < gtotal ? group_tiles(pg, pt0) : 0;
  };
  int64_t nissued = 0;  // tiles issued so far (thread 0)
  if (tid == 0) {
    for (int s = 0; s < STAGES && pg < gtotal; ++s) {
      issue(s, pt0 + pk);
      ++nissued;
      padvance();
    }
  }

  const int le = tid / n2, ij = tid - le * n2, i = ij % n, j = ij / n;
  int64_t it = 0;
  int64_t cg = next_group(blockIdx.x), ct0 = 0;
  int ck = 0, cn = cg < gtotal ? group_tiles(cg, ct0) : 0;
  double pwg = 0.0;  // this thread's part of the group's <p, A p>
  // the group's request, its fields in registers: read once per group, and
  // before any store through its pointers (which could alias the table)
  float *slp = nullptr, *slw = nullptr;
  const float* slB = nullptr;
  float h1 = 0.f, h2 = 0.f, beta = 0.f;
  int helm = 0;
  int64_t sE = 0, sT0 = 0;
  for (; cg < gtotal; ++it) {
    const int64_t tile = ct0 + ck;
    const int s = (int)(it % STAGES);
    if (ck == 0) {
      const int r = find_slot(stoff, ns, tile);
      const Slot& sl = T->s[r];
      slp = sl.p;
      slw = sl.w;
      slB = sl.B;
      h1 = sl.h1;
      h2 = sl.h2;
      helm = sl.helm;
      sE = sl.E;
      sT0 = stoff[r];
      beta = (float)sl.st->beta;
    }
    if (!tma::mbar_wait(&bars[s], (uint32_t)((it / STAGES) & 1))) sflag = 1;
    __syncthreads();
    if (sflag) break;
    float* st = stage0 + s * Lay::stage_floats;
    float* su = st + le * n3;
    const float* sG = st + 2 * EPB * n3 + le * 6 * n3;
    const int64_t e = (tile - sT0) * EPB + le;
    const bool act = e < sE;
    const int64_t base = e * n3 + ij;
    // B loaded ahead of the stores of this tile (see the single-mesh kernel)
    float rb[n];
#pragma unroll
    for (int k = 0; k < n; ++k) rb[k] = (act && helm) ? __ldg(slB + base + k * n2) : 0.f;

    float ru[n];
    if (act) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const float v = su[k * n2 + ij] + beta * st[EPB * n3 + le * n3 + k * n2 + ij];
        su[k * n2 + ij] = v;
        slp[base + k * n2] = v;
        ru[k] = v;
      }
    }
    __syncthreads();
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
        swr[le * n3 + k * n2 + ij] = g1 * ur + g4 * us + g5 * ut;
        sws[le * n3 + k * n2 + ij] = g4 * ur + g2 * us + g6 * ut;
        const float wt = g5 * ur + g6 * us + g3 * ut;
#pragma unroll
        for (int k2 = 0; k2 < n; ++k2) rw[k2] += sD[k * n + k2] * wt;
      }
    }
    __syncthreads();
    if (tid == 0 && pg < gtotal) {
      tma::fence_async_smem();
      issue(s, pt0 + pk);
      ++nissued;
      padvance();
    }
    float pw = 0.f;
    if (act) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        float acc = rw[k];
#pragma unroll
        for (int l = 0; l < n; ++l)
          acc += sD[l * n + i] * swr[le * n3 + k * n2 + j * n + l] + sD[l * n + j] * sws[le * n3 + k * n2 + l * n + i];
        float out = h1 * acc;
        if (helm) out += h2 * rb[k] * ru[k];
        slw[base + k * n2] = out;
        pw += ru[k] * out;
      }
    }
    pwg += (double)pw;
    if (++ck == cn) {  // the group's last tile: its partial
      const double bs = block_sum(pwg, sred);
      if (tid == 0) part_tile[cg] = bs;
      pwg = 0.0;
      cg = next_group(cg + gridDim.x);
      ck = 0;
      cn = cg < gtotal ? group_tiles(cg, ct0) : 0;
    }
    __syncthreads();
  }
  if (sflag && tid == 0) {
    atomicExch(err, 7);  // SEM_ERR_DEVICE_TIMEOUT; drain the copies this CTA issued (bounded waits)
    for (int64_t k = it; k < nissued; ++k) tma::mbar_wait(&bars[k % STAGES], (uint32_t)((k / STAGES) & 1));
    for (int r = 0; r < ns; ++r)
      if (slive[r]) {
        T->s[r].st->status = 7;
        T->s[r].st->done = 1;
      }
  }
}

// ---- alpha per request ----------------------------------------------------------
__global__ void __launch_bounds__(256) k_balpha(const Table* __restrict__ T, const double* __restrict__ part_tile) {
  __shared__ double sred[32];
  const int r = blockIdx.x;
  if (r >= T->nslots) return;
  const Slot& sl = T->s[r];
  if (!sl.active || sl.st->done) return;
  const int64_t b = T->grp_off[r], e = T->grp_off[r + 1];
  double v = 0.0;
  for (int64_t q = b + threadIdx.x; q < e; q += blockDim.x) v += part_tile[q];
  const double pAp = block_sum(v, sred);
  if (threadIdx.x == 0) {
    PcgState* st = sl.st;
    st->pAp = pAp;
    if (!(pAp > 0.0)) {
      st->done = 1;
      st->status = 5;  // SEM_ERR_BREAKDOWN
    } else {
      st->alpha = st->rho / pAp;
    }
  }
}

// ---- gather-scatter ---------------------------------------------------------------
__device__ __forceinline__ void bgs_node(float* __restrict__ v, const int32_t* __restrict__ id, int M) {
  const int32_t first = id[0];
  float acc = v[first & 0x7fffffff];
  for (int c = 1; c < M; ++c) acc = __fadd_rn(acc, v[id[c]]);
  v[first & 0x7fffffff] = acc;
  for (int c = 1; c < M; ++c) v[id[c]] = acc;
}

// Live flags and the slots' virtual-block offsets staged in shared memory
// once per CTA; false when no request is live (the CTA returns at once).
// A dead slot's virtual blocks are skipped in whole grid strides.
__device__ __forceinline__ int64_t skip_dead(const int64_t* off, int r, int64_t vb) {
  const int64_t end = off[r + 1];
  return vb + ((end - vb - 1) / gridDim.x) * gridDim.x;  // this CTA's last block before end
}

__global__ void __launch_bounds__(kGsThreads) k_bgs(const Table* __restrict__ T) {
  __shared__ int64_t svb[kMaxSlots * 9 + 1];
  __shared__ int slive[kMaxSlots];
  const int ns = T->nslots;
  int any = 0;
  for (int r = threadIdx.x; r < ns; r += blockDim.x) any |= (slive[r] = live(T->s[r]));
  if (!__syncthreads_or(any)) return;
  for (int q = threadIdx.x; q <= ns * 9; q += blockDim.x) svb[q] = T->gs_vb[q];
  __syncthreads();
  const int64_t total = svb[ns * 9];
  for (int64_t vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int rc = find_slot(svb, ns * 9, vb);
    const int r = rc / 9, c = rc % 9;
    if (!slive[r]) {
      vb = skip_dead(svb, rc, vb);
      continue;
    }
    const Slot& sl = T->s[r];
    const int64_t t = (vb - svb[rc]) * kGsThreads + threadIdx.x;
    if (t >= sl.gs_cnt[c]) continue;
    float* const w = sl.w;
    const int32_t* base = sl.gs_idx + sl.gs_off[c];
    if (c < 7) {
      const int M = c + 2;
      const int32_t* id = base + t * M;
      if (id[0] < 0) {  // Dirichlet node: masked to zero
        w[id[0] & 0x7fffffff] = 0.f;
        for (int q = 1; q < M; ++q) w[id[q]] = 0.f;
      } else {
        bgs_node(w, id, M);
      }
    } else if (c == 7) {
      const int32_t* gp = sl.gs_ptr;
      const int32_t b0 = gp[t], e0 = gp[t + 1];
      if (base[b0] < 0) {
        w[base[b0] & 0x7fffffff] = 0.f;
        for (int32_t q = b0 + 1; q < e0; ++q) w[base[q]] = 0.f;
      } else {
        bgs_node(w, base + b0, e0 - b0);
      }
    } else {
      w[base[t] & 0x7fffffff] = 0.f;
    }
  }
}

// ---- update + stop / reliable-update test ------------------------------------------
struct AccF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

__global__ void __launch_bounds__(kVecThreads, 4) k_bupdate(Table* __restrict__ T, double* part_vec) {
  __shared__ double sred[32];
  __shared__ float sinv[128];
  __shared__ bool is_last;
  __shared__ int64_t svb[kMaxSlots + 1];
  __shared__ int slive[kMaxSlots];
  const int ns = T->nslots;
  int any = 0;
  for (int r = threadIdx.x; r < ns; r += blockDim.x) any |= (slive[r] = live(T->s[r]));
  if (!__syncthreads_or(any)) return;
  for (int r = threadIdx.x; r <= ns; r += blockDim.x) svb[r] = T->vec_vb[r];
  for (int m = threadIdx.x; m < 128; m += blockDim.x) sinv[m] = m ? 1.f / (float)m : 0.f;
  __syncthreads();
  const int64_t total = svb[ns];
  for (int64_t vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int r = find_slot(svb, ns, vb);
    if (!slive[r]) {
      vb = skip_dead(svb, r, vb);
      continue;
    }
    // the slot's fields in registers before the first store (see k_bax)
    Slot& sl = T->s[r];
    float4* const x = reinterpret_cast<float4*>(sl.x);
    float4* const rv = reinterpret_cast<float4*>(sl.r);
    float4* const z = reinterpret_cast<float4*>(sl.z);
    const float4* const p = reinterpret_cast<const float4*>(sl.p);
    const float4* const w = reinterpret_cast<const float4*>(sl.w);
    const float4* const minv = reinterpret_cast<const float4*>(sl.minv);
    const uchar4* const wm = reinterpret_cast<const uchar4*>(sl.wm);
    const int64_t nl = sl.n_local;
    const float alpha = (float)sl.st->alpha;
    // kVecW / 4 16-byte vectors per thread, each of 4 consecutive points (n_local
    // is a multiple of 8 for every odd order, and the vectors are 16-byte
    // aligned); all loads issued before the first store
    const int64_t q0 = (vb - svb[r]) * (kVecPts / 4) + threadIdx.x;
    constexpr int U = kVecW / 4;
    AccF rz, rr;
    float4 pv[U], wv[U], mv[U], xv[U], rq[U];
    uchar4 mk[U];
    bool in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = q0 + (int64_t)u * kVecThreads;
      in[u] = 4 * q < nl;
      if (in[u]) {
        pv[u] = p[q];
        wv[u] = w[q];
        mv[u] = minv[q];
        xv[u] = x[q];
        rq[u] = rv[q];
        mk[u] = wm[q];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!in[u]) continue;
      const int64_t q = q0 + (int64_t)u * kVecThreads;
      float4 a = xv[u], b = rq[u];
      a.x += alpha * pv[u].x; a.y += alpha * pv[u].y; a.z += alpha * pv[u].z; a.w += alpha * pv[u].w;
      b.x -= alpha * wv[u].x; b.y -= alpha * wv[u].y; b.z -= alpha * wv[u].z; b.w -= alpha * wv[u].w;
      const float4 zq = make_float4(mv[u].x * b.x, mv[u].y * b.y, mv[u].z * b.z, mv[u].w * b.w);
      x[q] = a;
      rv[q] = b;
      z[q] = zq;
      const float i0 = sinv[mk[u].x & 0x7f], i1 = sinv[mk[u].y & 0x7f], i2 = sinv[mk[u].z & 0x7f],
                  i3 = sinv[mk[u].w & 0x7f];
      rz.add(b.x * zq.x * i0);
      rz.add(b.y * zq.y * i1);
      rz.add(b.z * zq.z * i2);
      rz.add(b.w * zq.w * i3);
      rr.add(b.x * b.x * i0);
      rr.add(b.y * b.y * i1);
      rr.add(b.z * b.z * i2);
      rr.add(b.w * b.w * i3);
    }
    const double a = block_sum(rz.get(), sred);
    const double b = block_sum(rr.get(), sred);
    if (threadIdx.x == 0) {
      part_vec[2 * vb] = a;
      part_vec[2 * vb + 1] = b;
      __threadfence();
      const unsigned int nvb = (unsigned int)(svb[r + 1] - svb[r]);
      is_last = atomicAdd(&T->cnt[r], 1u) == nvb - 1;
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      double vz = 0.0, vr = 0.0;
      for (int64_t q = svb[r] + threadIdx.x; q < svb[r + 1]; q += blockDim.x) {
        vz += __ldcg(part_vec + 2 * q);
        vr += __ldcg(part_vec + 2 * q + 1);
      }
      const double rz_t = block_sum(vz, sred);
      const double rr_t = block_sum(vr, sred);
      if (threadIdx.x == 0) {
        PcgState* st = sl.st;
        st->iter += 1;
        st->rr = rr_t;
        if (rr_t != rr_t || rz_t != rz_t) {
          st->done = 1;
          st->status = 5;
        } else if (rr_t <= st->tol2 * st->bb) {
          st->done = 1;
          st->status = 0;
        } else if (st->iter >= st->maxit) {
          st->done = 1;
          st->status = 4;
        } else if (st->delta2 > 0.0 && rr_t <= st->delta2 * st->rr_max) {
          st->done = 1;
          st->ru = 1;
        } else {
          if (rr_t > st->rr_max) st->rr_max = rr_t;
          st->beta = rz_t / st->rho;
          st->rho = rz_t;
        }
        T->cnt[r] = 0;
      }
    }
    __syncthreads();
  }
}

// ---- host engine ---------------------------------------------------------------------

template <int N>
cudaError_t launch_bax(const Table* T, double* part, int* err, int variant, cudaStream_t s, int* grid_cap) {
  constexpr int n = N + 1;
  constexpr int EPB = epb_for(N, 1), STAGES = 3;
  (void)variant;
  const size_t smem = tma::tma_smem_bytes<N, EPB, STAGES, true>();
  static DeviceOnce once;  // CTAs per device, computed once per device
  int cap = 0;
  cudaError_t oerr = once.get(
      [&](int dev, int* c) {
        cudaError_t e =
            cudaFuncSetAttribute(k_bax<N, EPB, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bax<N, EPB, STAGES>, EPB * n * n, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        *c = per_sm * sms;
        return cudaSuccess;
      },
      &cap);
  if (oerr != cudaSuccess) return oerr;
  if (grid_cap) *grid_cap = EPB;
  k_bax<N, EPB, STAGES><<<cap, EPB * n * n, smem, s>>>(T, part, err);
  return cudaGetLastError();
}

cudaError_t dispatch_bax(int N, const Table* T, double* part, int* err, cudaStream_t s, int* epb) {
  switch (N) {
    case 1: return launch_bax<1>(T, part, err, 0, s, epb);
    case 3: return launch_bax<3>(T, part, err, 0, s, epb);
    case 5: return launch_bax<5>(T, part, err, 0, s, epb);
    case 7: return launch_bax<7>(T, part, err, 0, s, epb);
    case 9: return launch_bax<9>(T, part, err, 0, s, epb);
    case 11: return launch_bax<11>(T, part, err, 0, s, epb);
    default: return cudaErrorNotSupported;
  }
}


constexpr double kGamma = 0.2;  // the FP32 residual must undershoot gamma * tol (see solver.cpp)

class EngineImpl {
 public:
  explicit EngineImpl(int N) : N_(N) {}
  ~EngineImpl() { release(); }
  int order() const { return N_; }

  // Order the engine's stream after the caller's (at init, and each time a
  // cached engine serves another call).
  sem_status attach(cudaStream_t user) {
    SEM_CUDA(cudaEventRecord(eu_, user));
    SEM_CUDA(cudaStreamWaitEvent(s_, eu_, 0));
    return SEM_OK;
  }

  sem_status init(cudaStream_t user) {
    SEM_CUDA(cudaStreamCreateWithFlags(&s_, cudaStreamNonBlocking));
    SEM_CUDA(cudaEventCreateWithFlags(&eu_, cudaEventDisableTiming));
    sem_status st = attach(user);
    if (st != SEM_OK) return st;
    SEM_CUDA(cudaMallocHost((void**)&h_tab_, sizeof(Table)));
    SEM_CUDA(cudaMalloc((void**)&d_tab_, sizeof(Table)));
    SEM_CUDA(cudaMallocHost((void**)&h_st_, kMaxSlots * sizeof(PcgState)));
    SEM_CUDA(cudaMalloc((void**)&d_err_, sizeof(int)));
    SEM_CUDA(cudaMemsetAsync(d_err_, 0, sizeof(int), s_));
    SEM_CUDA(cudaMalloc((void**)&done_state_, sizeof(PcgState)));
    PcgState d;
    std::memset(&d, 0, sizeof(d));
    d.done = 1;
    SEM_CUDA(cudaMemcpyAsync(done_state_, &d, sizeof(d), cudaMemcpyHostToDevice, s_));
    SEM_CUDA(cudaStreamSynchronize(s_));  // d is on this thread's stack
    std::memset(h_tab_, 0, sizeof(Table));
    return SEM_OK;
  }

  // FP64 set-up of requests and their activation in free slots, in two
  // phases so that the requests' FP64 work overlaps on the GPU: every
  // request's initial residual is launched on its own stream with an
  // asynchronous copy of its state, then each state is read and the request
  // either finishes (b = 0, or x0 already meets tol) or starts its FP32 CG.
  // Requests beyond the free slots are not taken (*taken counts those that were).
  sem_status add_many(Req* const* qs, int count, int* taken) {
    *taken = 0;
    int free_slots = 0;
    for (Req* o : slots_)
      if (!o) ++free_slots;
    const int k = std::min(count, free_slots);
    for (int t = 0; t < k; ++t) {
      sem_status st = add_begin(qs[t]);
      if (st != SEM_OK) return st;
      *taken = t + 1;
    }
    for (int t = 0; t < k; ++t) {
      sem_status st = add_end(qs[t]);
      if (st != SEM_OK) return st;
    }
    return SEM_OK;
  }

  void abandon() {
    if (s_) cudaStreamSynchronize(s_);
    auto drop = [](Req* q) {
      if (q->ws) {
        cudaStreamSynchronize(q->ws->s);
        if (q->own_ws) q->m->spare_ws.push_back(q->ws);
      }
      q->ws = nullptr;
      q->own_ws = false;
      q->slot = -1;
    };
    for (Req*& q : slots_) {
      if (q) drop(q);
      q = nullptr;
    }
    for (Req* q : pending_) drop(q);
    pending_.clear();
    dirty_ = true;
  }

  sem_status add(Req* q) {
    int taken = 0;
    sem_status st = add_many(&q, 1, &taken);
    if (st != SEM_OK) return st;
    return taken ? SEM_OK : SEM_ERR_BUSY;
  }

 private:
  // A request's state written from the pinned slot sth[1] (sth[0] receives
  // the reads); the host rewrites sth[1] only after a read of the same
  // stream has completed, so no synchronisation is needed here.
  sem_status put_state_async(Workspace* ws, double tol, int maxit) {
    PcgState h;
    std::memset(&h, 0, sizeof(h));
    h.tol2 = tol * tol;
    h.maxit = maxit;
    ws->sth[1] = h;
    SEM_CUDA(cudaMemcpyAsync(ws->st, &ws->sth[1], sizeof(PcgState), cudaMemcpyHostToDevice, ws->s));
    return SEM_OK;
  }

  // the FP64 residual r = b - A x of a request on its stream, then its state copied to sth[0] (event ev[0])
  sem_status launch_residual_read(Req* q, int set_bb) {
    Workspace* ws = q->ws;
    sem_mesh* m = q->m;
    SEM_CUDA(ax64_exact(m, ws->x, ws->w, q->o.h1, q->o.h2, ws->s));
    SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, nullptr, ws->s));
    SEM_CUDA(launch_residual(ws->r, ws->b, ws->w, m->wm, ws->n, ws->st, ws->part_vec, set_bb, ws->s));
    count_launches(3);
    SEM_CUDA(cudaMemcpyAsync(&ws->sth[0], ws->st, sizeof(PcgState), cudaMemcpyDeviceToHost, ws->s));
    SEM_CUDA(cudaEventRecord(ws->ev[0], ws->s));
    return SEM_OK;
  }

  sem_status read_async_state(Workspace* ws, PcgState& out) {
    SEM_CUDA(cudaEventSynchronize(ws->ev[0]));
    out = ws->sth[0];
    return SEM_OK;
  }

  sem_status add_begin(Req* q) {
    sem_mesh* m = q->m;
    if (!m->ws) {
      sem_status st = alloc_ws(m, &m->ws);
      if (st != SEM_OK) return st;
    }
    // the mesh's workspace, or a fresh one when another request of this
    // batch (another right-hand side on the same mesh) already holds it
    bool taken = false;
    for (Req* o : slots_)
      if (o && o->ws == m->ws) taken = true;
    for (Req* o : pending_)
      if (o->ws == m->ws) taken = true;
    if (taken) {
      Workspace* own = nullptr;
      if (!m->spare_ws.empty()) {  // one kept from an earlier batch on this mesh
        own = m->spare_ws.back();
        m->spare_ws.pop_back();
      } else {
        sem_status st = alloc_ws(m, &own);
        if (st != SEM_OK) return st;
      }
      q->ws = own;
      q->own_ws = true;
    } else {
      q->ws = m->ws;
      q->own_ws = false;
    }
    pending_.push_back(q);
    Workspace* ws = q->ws;
    const size_t bytes = (size_t)ws->n * sizeof(double);
    // the request's own stream ws->s does its FP64 work; order it after ours
    SEM_CUDA(cudaEventRecord(eu_, s_));
    SEM_CUDA(cudaStreamWaitEvent(ws->s, eu_, 0));
    // a fresh state (zero arrival counters) before the first reduction kernel
    sem_status st0 = put_state_async(ws, q->o.tol, q->o.maxit);
    if (st0 != SEM_OK) return st0;
    SEM_CUDA(cudaMemcpyAsync(ws->b, q->b, bytes, cudaMemcpyDeviceToDevice, ws->s));
    SEM_CUDA(cudaMemcpyAsync(ws->x, q->x, bytes, cudaMemcpyDeviceToDevice, ws->s));
    launch_mask(ws->x, m->wm, ws->n, ws->s);
    launch_minv(ws->minv, ws->minv32, m->opdK(), m->opdB(), m->wm, q->o.h1, q->o.h2, ws->n, ws->s);
    ws->minv_h1 = q->o.h1;
    ws->minv_h2 = q->o.h2;
    count_launches(2);
    return launch_residual_read(q, 1);
  }

  sem_status add_end(Req* q) {
    pending_.erase(std::find(pending_.begin(), pending_.end(), q));
    Workspace* ws = q->ws;
    sem_mesh* m = q->m;
    const size_t bytes = (size_t)ws->n * sizeof(double);
    PcgState s0;
    sem_status st = read_async_state(ws, s0);
    if (st != SEM_OK) return st;
    if (s0.bb == 0.0) {
      SEM_CUDA(cudaMemsetAsync(ws->x, 0, bytes, ws->s));
      return finish(q, SEM_OK, 0.0, 0);
    }
    q->bnorm = std::sqrt(s0.bb);
    q->scale = 1.0 / q->bnorm;
    const double rel = std::sqrt(s0.aux) / q->bnorm;
    if (rel <= q->o.tol) return finish(q, SEM_OK, rel, 0);
    st = put_state_async(ws, kGamma * q->o.tol, q->o.maxit);
    if (st != SEM_OK) return st;
    launch_scale_to_f32(ws->r32, ws->r, q->scale, ws->n, ws->s);
    launch_zero_f32(ws->x32, ws->n, ws->s);
    VecParams<float> v{ws->x32, ws->r32, ws->z32, ws->p32, ws->w32, ws->minv32, ws->r32, m->wm, ws->n, ws->st,
                       ws->part_vec};
    SEM_CUDA(launch_pcg_init<float>(v, ws->s));
    launch_set_bb(ws->st, 1.0, q->o.delta * q->o.delta, ws->s);
    count_launches(4);
    SEM_CUDA(cudaEventRecord(eu_, ws->s));
    SEM_CUDA(cudaStreamWaitEvent(s_, eu_, 0));
    int slot = -1;
    for (int r = 0; r < kMaxSlots; ++r)
      if (!slots_[r]) {
        slot = r;
        break;
      }
    q->slot = slot;
    slots_[slot] = q;
    dirty_ = true;
    return SEM_OK;
  }

 public:
  bool idle() const {
    for (auto* q : slots_)
      if (q) return false;
    return true;
  }

  // One graph launch (kChunk iterations of every live request), then the
  // per-request FP64 work of the requests that paused.
  sem_status step() {
    sem_status st = sync_table();
    if (st != SEM_OK) return st;
    st = ensure_graph();
    if (st != SEM_OK) return st;
    SEM_CUDA(cudaGraphLaunch(graph_, s_));
    count_launches(4 * kChunk);
    for (int r = 0; r < kMaxSlots; ++r)
      if (slots_[r])
        SEM_CUDA(cudaMemcpyAsync(&h_st_[r], slots_[r]->ws->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s_));
    SEM_CUDA(cudaStreamSynchronize(s_));
    int err = 0;
    SEM_CUDA(cudaMemcpyAsync(&err, d_err_, sizeof(int), cudaMemcpyDeviceToHost, s_));
    SEM_CUDA(cudaStreamSynchronize(s_));
    // the paused requests' FP64 residuals first (each on its own stream, so
    // they overlap), then their decisions
    std::vector<std::pair<Req*, PcgState>> waiting;
    for (int r = 0; r < kMaxSlots; ++r) {
      Req* q = slots_[r];
      if (!q || !h_st_[r].done) continue;
      bool launched = false;
      st = pause_begin(q, h_st_[r], err, &launched);
      if (st != SEM_OK) return st;
      if (launched) waiting.push_back({q, h_st_[r]});
    }
    for (auto& w : waiting) {
      st = pause_end(w.first, w.second);
      if (st != SEM_OK) return st;
    }
    return SEM_OK;
  }

 private:
  // x += x32 ||b|| for a paused request; a finished one (error, breakdown,
  // maxit) completes here, any other gets its FP64 residual launched (*launched).
  sem_status pause_begin(Req* q, const PcgState& fin, int err, bool* launched) {
    *launched = false;
    Workspace* ws = q->ws;
    SEM_CUDA(cudaEventRecord(eu_, s_));
    SEM_CUDA(cudaStreamWaitEvent(ws->s, eu_, 0));
    launch_accumulate(ws->x, ws->x32, q->bnorm, ws->n, ws->s);
    launch_zero_f32(ws->x32, ws->n, ws->s);
    count_launches(2);
    if (err || fin.status == SEM_ERR_DEVICE_TIMEOUT) return finish(q, SEM_ERR_DEVICE_TIMEOUT, 0.0, fin.iter);
    if (fin.status == SEM_ERR_BREAKDOWN || fin.status == SEM_ERR_NOT_CONVERGED)
      return finish(q, (sem_status)fin.status, std::sqrt(fin.rr), fin.iter);
    *launched = true;
    return launch_residual_read(q, 0);
  }

  // The replacement's decision: finish at tol (or maxit), else r32 = r / ||b||
  // and CG continues with its direction.
  sem_status pause_end(Req* q, const PcgState& fin) {
    Workspace* ws = q->ws;
    sem_mesh* m = q->m;
    PcgState s1;
    sem_status st = read_async_state(ws, s1);
    if (st != SEM_OK) return st;
    q->outer += 1;
    const double rel = std::sqrt(s1.aux) / q->bnorm;
    if (rel <= q->o.tol) return finish(q, SEM_OK, rel, fin.iter);
    if (fin.iter >= q->o.maxit) return finish(q, SEM_ERR_NOT_CONVERGED, rel, fin.iter);
    launch_scale_to_f32(ws->r32, ws->r, q->scale, ws->n, ws->s);
    VecParams<float> v{ws->x32, ws->r32, ws->z32, ws->p32, ws->w32, ws->minv32, ws->r32, m->wm, ws->n, ws->st,
                       ws->part_vec};
    SEM_CUDA(launch_pcg_restart<float>(v, ws->s));
    count_launches(2);
    SEM_CUDA(cudaEventRecord(eu_, ws->s));
    SEM_CUDA(cudaStreamWaitEvent(s_, eu_, 0));
    return SEM_OK;
  }

  sem_status finish(Req* q, sem_status status, double rel, int iters) {
    Workspace* ws = q->ws;
    SEM_CUDA(cudaMemcpyAsync(q->x, ws->x, (size_t)ws->n * sizeof(double), cudaMemcpyDeviceToDevice, ws->s));
    SEM_CUDA(cudaStreamSynchronize(ws->s));
    if (q->own_ws) {  // kept on the mesh for its next batch
      q->m->spare_ws.push_back(ws);
      q->ws = nullptr;
      q->own_ws = false;
    }
    q->finished = true;
    q->status = status;
    if (q->out) {
      q->out->iters = iters;
      q->out->outer_iters = q->outer;
      q->out->rel_res = rel;
      q->out->ms = 0.0;
      q->out->status = status;
    }
    if (q->slot >= 0) {
      slots_[q->slot] = nullptr;
      dirty_ = true;
    }
    return SEM_OK;
  }

  // Rebuild the slot table (prefix offsets) after requests joined or left.
  sem_status sync_table() {
    if (!dirty_) return SEM_OK;
    SEM_CUDA(cudaStreamSynchronize(s_));  // the previous table copy has landed
    Table& T = *h_tab_;
    std::memset(&T, 0, sizeof(Table));
    int ns = 0;
    for (int r = 0; r < kMaxSlots; ++r)
      if (slots_[r]) ns = r + 1;
    T.nslots = ns;
    const int epb = ax_elems_per_block(N_, 1);
    int64_t tiles = 0, groups = 0, gvb = 0, vvb = 0;
    for (int r = 0; r < ns; ++r) {
      T.tile_off[r] = tiles;
      T.grp_off[r] = groups;
      T.vec_vb[r] = vvb;
      Req* q = slots_[r];
      Slot& sl = T.s[r];
      for (int c = 0; c < 9; ++c) T.gs_vb[r * 9 + c] = gvb + 0;
      if (q) {
        sem_mesh* m = q->m;
        Workspace* ws = q->ws;
        sl.G = m->opG32();
        sl.B = m->opB32();
        sl.D = m->D32;
        if (!T.D) T.D = m->D32;
        sl.wm = m->wm;
        sl.gs_idx = m->gs_idx;
        sl.gs_ptr = m->gs_ptr;
        for (int c = 0; c < 9; ++c) {
          sl.gs_off[c] = m->gs_off[c];
          sl.gs_cnt[c] = m->gs_cnt[c];
        }
        sl.x = ws->x32;
        sl.r = ws->r32;
        sl.z = ws->z32;
        sl.p = ws->p32;
        sl.w = ws->w32;
        sl.minv = ws->minv32;
        sl.st = ws->st;
        sl.h1 = (float)q->o.h1;
        sl.h2 = (float)q->o.h2;
        sl.helm = q->o.h2 != 0.0;
        sl.active = 1;
        sl.E = m->E;
        sl.n_local = m->n_local;
        const int64_t nt = (m->E + epb - 1) / epb;
        tiles += nt;
        groups += (nt + kTileGroup - 1) / kTileGroup;
        vvb += (m->n_local + kVecPts - 1) / kVecPts;
        for (int c = 0; c < 9; ++c) {
          T.gs_vb[r * 9 + c] = gvb;
          gvb += (m->gs_cnt[c] + kGsThreads - 1) / kGsThreads;
        }
      } else {
        // an empty slot: no tiles, no blocks; st points at a done state
        sl.active = 0;
        sl.st = done_state_;
      }
    }
    T.tile_off[ns] = tiles;
    T.grp_off[ns] = groups;
    T.vec_vb[ns] = vvb;
    T.gs_vb[ns * 9] = gvb;
    if (tiles > cap_tiles_ || vvb > cap_vb_) {
      if (part_tile_) cudaFree(part_tile_);
      if (part_vec_) cudaFree(part_vec_);
      part_tile_ = nullptr;
      part_vec_ = nullptr;
      cap_tiles_ = std::max<int64_t>(tiles, 2 * cap_tiles_);
      cap_vb_ = std::max<int64_t>(vvb, 2 * cap_vb_);
      SEM_CUDA(cudaMalloc((void**)&part_tile_, (size_t)std::max<int64_t>(cap_tiles_, 1) * sizeof(double)));
      SEM_CUDA(cudaMalloc((void**)&part_vec_, 2 * (size_t)std::max<int64_t>(cap_vb_, 1) * sizeof(double)));
      if (graph_) {
        cudaGraphExecDestroy(graph_);
        graph_ = nullptr;
      }
    }
    SEM_CUDA(cudaMemcpyAsync(d_tab_, h_tab_, sizeof(Table), cudaMemcpyHostToDevice, s_));
    dirty_ = false;
    return SEM_OK;
  }

  sem_status launch_iteration() {
    int epb = 0;
    SEM_CUDA(dispatch_bax(N_, d_tab_, part_tile_, d_err_, s_, &epb));
    k_balpha<<<kMaxSlots, 256, 0, s_>>>(d_tab_, part_tile_);
    SEM_CUDA(cudaGetLastError());
    k_bgs<<<152 * 16, kGsThreads, 0, s_>>>(d_tab_);
    SEM_CUDA(cudaGetLastError());
    k_bupdate<<<152 * 4, kVecThreads, 0, s_>>>(d_tab_, part_vec_);
    SEM_CUDA(cudaGetLastError());
    return SEM_OK;
  }

  sem_status ensure_graph() {
    if (graph_) return SEM_OK;
    // one eager pass on an empty table sets the kernels' attributes outside the capture
    Table* empty = nullptr;
    SEM_CUDA(cudaMalloc((void**)&empty, sizeof(Table)));
    SEM_CUDA(cudaMemsetAsync(empty, 0, sizeof(Table), s_));
    Table* keep = d_tab_;
    d_tab_ = empty;
    sem_status st = launch_iteration();
    d_tab_ = keep;
    SEM_CUDA(cudaStreamSynchronize(s_));
    cudaFree(empty);
    if (st != SEM_OK) return st;
    count_launches(4);
    cudaGraph_t g = nullptr;
    SEM_CUDA(cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < kChunk && st == SEM_OK; ++k) st = launch_iteration();
    cudaError_t e = cudaStreamEndCapture(s_, &g);
    if (st != SEM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&graph_, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return SEM_OK;
  }

  void release() {
    if (s_) cudaStreamSynchronize(s_);
    if (graph_) cudaGraphExecDestroy(graph_);
    for (void* p : {(void*)d_tab_, (void*)part_tile_, (void*)part_vec_, (void*)d_err_, (void*)done_state_})
      if (p) cudaFree(p);
    if (h_tab_) cudaFreeHost(h_tab_);
    if (h_st_) cudaFreeHost(h_st_);
    if (eu_) cudaEventDestroy(eu_);
    if (s_) cudaStreamDestroy(s_);
  }

  int N_;
  cudaStream_t s_ = nullptr;
  cudaEvent_t eu_ = nullptr;
  Table* h_tab_ = nullptr;
  Table* d_tab_ = nullptr;
  PcgState* h_st_ = nullptr;
  PcgState* done_state_ = nullptr;
  double* part_tile_ = nullptr;
  double* part_vec_ = nullptr;
  int64_t cap_tiles_ = 0, cap_vb_ = 0;
  int* d_err_ = nullptr;
  cudaGraphExec_t graph_ = nullptr;
  Req* slots_[kMaxSlots] = {nullptr};
  std::vector<Req*> pending_;  // between add_begin and add_end
  bool dirty_ = true;
};


Engine::Engine(int N) : impl_(new EngineImpl(N)) {}
Engine::~Engine() { delete impl_; }
sem_status Engine::init(cudaStream_t user) { return impl_->init(user); }
sem_status Engine::attach(cudaStream_t user) { return impl_->attach(user); }
sem_status Engine::add(Req* q) { return impl_->add(q); }
sem_status Engine::add_many(Req* const* qs, int count, int* taken) { return impl_->add_many(qs, count, taken); }
sem_status Engine::step() { return impl_->step(); }
bool Engine::idle() const { return impl_->idle(); }
void Engine::abandon() { impl_->abandon(); }
int Engine::order() const { return impl_->order(); }

}  // namespace batch
}  // namespace sem

using namespace sem;

namespace {
// Idle engines of sem_pcg_solve_batch by (device, order): a later call reuses
// one with its buffers and captured graph instead of building and capturing
// anew.  Never destroyed: freeing CUDA resources during static destruction at
// exit is not safe, and the driver reclaims them with the process.
std::mutex g_engine_mutex;
auto* g_idle_engines = new std::vector<std::pair<std::pair<int, int>, batch::Engine*>>();

batch::Engine* take_idle_engine(int dev, int N) {
  std::lock_guard<std::mutex> lk(g_engine_mutex);
  for (size_t k = 0; k < g_idle_engines->size(); ++k)
    if ((*g_idle_engines)[k].first == std::make_pair(dev, N)) {
      batch::Engine* e = (*g_idle_engines)[k].second;
      g_idle_engines->erase(g_idle_engines->begin() + k);
      return e;
    }
  return nullptr;
}

void put_idle_engine(int dev, int N, batch::Engine* e) {
  std::lock_guard<std::mutex> lk(g_engine_mutex);
  g_idle_engines->push_back({{dev, N}, e});
}
}  // namespace

extern "C" sem_status sem_pcg_solve_batch(const sem_mesh* const* meshes, const double* const* b_dev,
                                          double* const* x_dev, const sem_solve_opts* opts,
                                          sem_solve_result* results, int count, void* stream) {
  SEM_TRACE("sem_pcg_solve_batch");
  if (count < 0 || (count > 0 && (!meshes || !b_dev || !x_dev || !opts))) {
    set_error("sem_pcg_solve_batch: null argument");
    return SEM_ERR_INVALID;
  }
  if (count == 0) return SEM_OK;
  const int N = meshes[0] ? meshes[0]->N : -1;
  if (N < 1 || (N + 1) % 2 != 0) {
    set_error("sem_pcg_solve_batch: batched kernels need an odd polynomial order N (even n = N + 1)");
    return SEM_ERR_INVALID;
  }
  std::vector<batch::Req> reqs(count);
  for (int k = 0; k < count; ++k) {
    const sem_mesh* m = meshes[k];
    if (!m || !b_dev[k] || !x_dev[k] || m->N != N) {
      set_error("sem_pcg_solve_batch: every request needs a mesh of the same order and b, x");
      return SEM_ERR_INVALID;
    }
    sem_solve_opts o = opts[k];
    if (o.prec != SEM_MIXED || o.refine != 0) {
      set_error("sem_pcg_solve_batch: batches run the mixed-precision reliable-update solver (prec = SEM_MIXED)");
      return SEM_ERR_INVALID;
    }
    if (!(o.h1 >= 0.0) || !(o.h2 >= 0.0) || (o.h1 == 0.0 && o.h2 == 0.0)) {
      set_error("sem_pcg_solve_batch: need h1 >= 0, h2 >= 0, not both zero");
      return SEM_ERR_INVALID;
    }
    if (!(o.tol > 0.0)) o.tol = 1e-10;
    if (o.maxit <= 0) o.maxit = 20000;
    if (!(o.delta > 0.0)) o.delta = 0.1;
    reqs[k].m = const_cast<sem_mesh*>(m);
    reqs[k].b = b_dev[k];
    reqs[k].x = x_dev[k];
    reqs[k].o = o;
    reqs[k].out = results ? &results[k] : nullptr;
  }
  // each distinct mesh locked once (a mesh may carry several right-hand
  // sides), in address order so that concurrent callers cannot deadlock
  std::vector<sem_mesh*> distinct;
  for (auto& q : reqs) distinct.push_back(q.m);
  std::sort(distinct.begin(), distinct.end());
  distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
  std::vector<std::unique_lock<std::mutex>> locks;
  for (sem_mesh* m : distinct) locks.emplace_back(m->ws_mutex);
  int dev = 0;
  SEM_CUDA(cudaGetDevice(&dev));
  std::unique_ptr<batch::Engine> held(take_idle_engine(dev, N));
  sem_status st;
  if (held) {
    st = held->attach((cudaStream_t)stream);
  } else {
    held.reset(new batch::Engine(N));
    st = held->init((cudaStream_t)stream);
  }
  if (st != SEM_OK) return st;
  batch::Engine& eng = *held;
  // a failure leaves the requests unfinished: the engine lets go of them (and
  // of the meshes) before it is destroyed
  auto fail = [&](sem_status s) {
    eng.abandon();
    return s;
  };
  size_t next = 0;
  const int max_steps = 1 << 20;
  for (int step = 0; step < max_steps; ++step) {
    // continuous admission: fill free slots from the queue (their FP64 set-up overlaps)
    if (next < reqs.size()) {
      std::vector<batch::Req*> qs;
      for (size_t k = next; k < reqs.size(); ++k) qs.push_back(&reqs[k]);
      int taken = 0;
      st = eng.add_many(qs.data(), (int)qs.size(), &taken);
      if (st != SEM_OK) return fail(st);
      next += taken;
    }
    if (eng.idle() && next == reqs.size()) break;
    st = eng.step();
    if (st != SEM_OK) return fail(st);
  }
  if (!eng.idle() || next < reqs.size()) {
    set_error("sem_pcg_solve_batch: the batch did not finish within its step limit");
    return fail(SEM_ERR_DEVICE_TIMEOUT);
  }
  put_idle_engine(dev, N, held.release());  // kept with its captured graph
  sem_status first_bad = SEM_OK;
  for (auto& q : reqs)
    if (q.status != SEM_OK && first_bad == SEM_OK) first_bad = q.status;
  return first_bad;
}
