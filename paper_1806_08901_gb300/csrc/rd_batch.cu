// rd_batch.cu -- the batched estimate (rd_select_batch): three persistent
// passes over the work items of every field of a batch.
//   range: runs of a field's values; the CTA that ends a field's last item
//     (a counter in the field's workspace, fenced on both sides) derives VR,
//     eb_abs and the precision exponent (Algorithm 1 line 2);
//   sampled blocks: runs of a field's sampled blocks, one thread per block:
//     the block and its one-cell low halo are read once; the SZ residuals
//     of its points (which do not depend on the bin width) are stored, and
//     the ZFP estimator terms accumulated (lines 3-6); the CTA that ends a
//     field's last item derives delta (line 7);
//   SZ histogram: the stored residuals, quantised at delta, coalesced
//     (line 8).
// The sampled blocks are scattered: each block row costs a whole DRAM
// fetch, so one pass that serves both estimators reads about a third of the
// field where two passes read about six tenths.
// CTAs stride over the items of their pass; the passes are stream-ordered
// launches, so no CTA waits on another.
#include <math.h>
#include <stdint.h>

#include "rd_delta.cuh"
#include "rd_device.cuh"
#include "rd_range_dev.cuh"
#include "rd_sz_dev.cuh"
#include "rd_zfp_dev.cuh"

namespace rdk {

constexpr int kBatchRangeThreads = 512;
constexpr int kBatchBlockThreads = 128;
constexpr int kBatchSzThreads = 256;

// ---------------------------------------------------------------------------
// Range
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBatchRangeThreads) k_batch_range(const BatchField* __restrict__ bf,
                                                                    const BatchItem* __restrict__ items,
                                                                    int nitems) {
  __shared__ int s_last;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem item = items[it];
    const BatchField& F = bf[item.field];
    RangeAcc acc;
    range_span(F.f.x, item.begin, item.end, threadIdx.x, blockDim.x, acc);
    range_commit(acc, F.ws);
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(&F.ws->sc.done[0], 1u) == F.items_range - 1u;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      prepare_field(F.p, F.ws);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Sampled blocks: ZFP estimate and SZ residuals from one read
// ---------------------------------------------------------------------------
// Block bx of the field's lattice and its low halo, (4+1)^d values, into
// cube (index 0 of each axis: the halo plane / row / column).  Coordinates
// below zero read zero (the Lorenzo zero padding); coordinates past the far
// edges read the last valid sample (the replication load_block does for the
// ZFP transform; for the SZ residuals they feed only points past the
// extent).  All the loads are independent.
template <int D>
__device__ __forceinline__ void load_cube(const FieldDev& f, const int* o, float* cube) {
  const int nx = f.n[D - 1];
  const int x0 = o[D - 1];
  constexpr int NR = D == 3 ? 25 : D == 2 ? 5 : 1;
#pragma unroll
  for (int rr = 0; rr < NR; rr++) {
    const int iz = D == 3 ? rr / 5 : 0, iy = D >= 2 ? rr % 5 : 0;
    bool in = true;
    long long row = 0;
    if (D == 3) {
      const int z = o[0] - 1 + iz, y = o[1] - 1 + iy;
      in = z >= 0 && y >= 0;
      row = (long long)min(z, f.n[0] - 1) * f.n[1] + min(y, f.n[1] - 1);
    } else if (D == 2) {
      const int y = o[0] - 1 + iy;
      in = y >= 0;
      row = min(y, f.n[0] - 1);
    }
    float* c = cube + rr * 5;
    if (!in) {
#pragma unroll
      for (int k = 0; k < 5; k++) c[k] = 0.0f;
      continue;
    }
    const float* p = f.x + row * nx;
    c[0] = x0 > 0 ? __ldg(p + x0 - 1) : 0.0f;
    if (f.vec_ok && x0 + 4 <= nx) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p + x0));
      c[1] = q.x;
      c[2] = q.y;
      c[3] = q.z;
      c[4] = q.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++) c[k + 1] = __ldg(p + min(x0 + k, nx - 1));
    }
  }
}

// One thread per sampled block: the SZ residuals of the block's points (the
// float32 nested differences of est_residual; NaN past the extent) are
// stored for the histogram pass, and the ZFP estimator terms of the block
// (Alg. 1 lines 4-6) are accumulated.
template <int D>
__device__ __forceinline__ void sampled_blocks_item(const BatchField& F, long long b0, long long b1,
                                                    int minexp, unsigned long long& my_s2,
                                                    unsigned long long* s_lo,
                                                    unsigned long long* s_hi) {
  constexpr int NB = 1 << (2 * D);
  constexpr int NC = D == 3 ? 125 : D == 2 ? 25 : 5;
  const FieldDev& f = F.f;
  const bool ec_all = F.p.ec_mode == RD_EC_ALL;
  for (long long sb = b0 + threadIdx.x; sb < b1; sb += blockDim.x) {
    int o[3] = {0, 0, 0};
    sampled_block_origin<D>(f, sb, o);
    float cube[NC];
    load_cube<D>(f, o, cube);
    // SZ residuals
    float r[NB];
#pragma unroll
    for (int t = 0; t < NB; t++) {
      const int k = t & 3, j = D >= 2 ? (t >> 2) & 3 : 0, i = D == 3 ? t >> 4 : 0;
      Nbr nb;
#pragma unroll
      for (int m = 0; m < (1 << D); m++) {
        const int bx = m & 1, by = (m >> 1) & 1, bz = (m >> 2) & 1;
        const int cz = D == 3 ? i + 1 - bz : 0, cy = D >= 2 ? j + 1 - by : 0, cx = k + 1 - bx;
        nb.v[m] = cube[(cz * 5 + cy) * 5 + cx];
      }
      bool ok = o[D - 1] + k < f.n[D - 1];
      if (D >= 2) ok = ok && o[D - 2] + j < f.n[D - 2];
      if (D == 3) ok = ok && o[0] + i < f.n[0];
      r[t] = ok ? est_residual<D>(nb) : __int_as_float(0x7fc00000);
    }
    float* dst = F.res + sb * NB;
    if (D == 1) {
#pragma unroll
      for (int t = 0; t < NB; t++) dst[t] = r[t];
    } else {
#pragma unroll
      for (int t = 0; t < NB; t += 4)
        *reinterpret_cast<float4*>(dst + t) = make_float4(r[t], r[t + 1], r[t + 2], r[t + 3]);
    }
    // ZFP: the block's values (with far-edge replication) are the cube's
    // entries with every index >= 1
    float v[NB];
#pragma unroll
    for (int t = 0; t < NB; t++) {
      const int k = t & 3, j = D >= 2 ? (t >> 2) & 3 : 0, i = D == 3 ? t >> 4 : 0;
      v[t] = cube[((D == 3 ? i + 1 : 0) * 5 + (D >= 2 ? j + 1 : 0)) * 5 + k + 1];
    }
    BlockWork<D> w;
    w.forward(v, minexp);
    zfp_est_accumulate<D>(w, ec_all, my_s2, s_lo, s_hi);
  }
}

__global__ void __launch_bounds__(kBatchBlockThreads) k_batch_blocks(const BatchField* __restrict__ bf,
                                                                     const BatchItem* __restrict__ items,
                                                                     int nitems) {
  __shared__ unsigned long long s_lo[kMseBins], s_hi[kMseBins];
  __shared__ unsigned long long s_s2;
  __shared__ int s_last;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem item = items[it];
    const BatchField& F = bf[item.field];
    Workspace* ws = F.ws;
    const bool live = ws->sc.status == RD_OK && !ws->sc.constant;
    for (int i = threadIdx.x; i < kMseBins; i += blockDim.x) {
      s_lo[i] = 0ull;
      s_hi[i] = 0ull;
    }
    if (threadIdx.x == 0) s_s2 = 0ull;
    __syncthreads();
    if (live) {
      unsigned long long my_s2 = 0ull;
      const int minexp = ws->sc.minexp;
      switch (F.f.d) {
        case 1: sampled_blocks_item<1>(F, item.begin, item.end, minexp, my_s2, s_lo, s_hi); break;
        case 2: sampled_blocks_item<2>(F, item.begin, item.end, minexp, my_s2, s_lo, s_hi); break;
        default: sampled_blocks_item<3>(F, item.begin, item.end, minexp, my_s2, s_lo, s_hi); break;
      }
      my_s2 = warp_sum(my_s2);
      if ((threadIdx.x & 31) == 0 && my_s2) atomicAdd(&s_s2, my_s2);
    }
    __syncthreads();
    if (live) {
      if (threadIdx.x == 0 && s_s2) atomicAdd(&ws->sc.s2, s_s2);
      for (int i = threadIdx.x; i < kMseBins; i += blockDim.x)
        if (s_lo[i] | s_hi[i]) atomic_add_u128(&ws->sc.mse_lo[i], &ws->sc.mse_hi[i], s_lo[i], s_hi[i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(&ws->sc.done[1], 1u) == F.items_zfp - 1u;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
      __threadfence();
      delta_warp(F.p, ws, DELTA_FROM_MSE, 0.0, 1, F.need_gt, F.ncoeff, F.npoints);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// SZ histogram of the stored residuals (Alg. 1 line 8), coalesced
// ---------------------------------------------------------------------------
// the shared window of the residual histogram: +-8192 codes around zero
// (the residuals of rough fields at fine bounds spread over thousands of
// codes; outside the window a code takes a global atomic)
constexpr int kWideWin = 16384;
constexpr int kWideWinLo = kCenter - kWideWin / 2;

__global__ void __launch_bounds__(kBatchSzThreads) k_batch_sz_hist(const BatchField* __restrict__ bf,
                                                                   const BatchItem* __restrict__ items,
                                                                   int nitems) {
  extern __shared__ uint32_t s_win[];  // kWideWin counters
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem item = items[it];
    const BatchField& F = bf[item.field];
    Workspace* ws = F.ws;
    if (ws->sc.status != RD_OK || ws->sc.constant) continue;  // uniform over the CTA
    for (int i = threadIdx.x; i < kWideWin; i += blockDim.x) s_win[i] = 0u;
    __syncthreads();
    const float inv = ws->sc.inv;
    const int R = F.p.R;
    const long long nb = 1ll << (2 * F.f.d);  // a multiple of 4: float4 granules
    const float4* r4 = reinterpret_cast<const float4*>(F.res + item.begin * nb);
    const int n4 = (int)((item.end - item.begin) * nb / 4);
    constexpr int U = 4;  // independent 16-byte loads in flight per thread
    const float nan = __int_as_float(0x7fc00000);
    for (int i0 = threadIdx.x; i0 - (int)threadIdx.x < n4; i0 += U * kBatchSzThreads) {
      float4 q[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        const int i = i0 + k * kBatchSzThreads;
        q[k] = i < n4 ? __ldcs(r4 + i) : make_float4(nan, nan, nan, nan);
      }
#pragma unroll
      for (int k = 0; k < U; k++) {
        const float rv[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const bool ok = !isnan(rv[c]);
          hist_add_sorted(s_win, kWideWinLo, kWideWin, ws->hist[0], ok ? est_symbol(rv[c], inv, R) : 0, ok);
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWideWin; i += blockDim.x) {
      const uint32_t c = s_win[i];
      if (c) atomicAdd(&ws->hist[0][kWideWinLo + i], c);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int grid_for(int nitems, int ctas) {
  const int g = nitems < ctas ? nitems : ctas;
  return g < 1 ? 1 : g;
}

cudaError_t launch_batch_range(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                               cudaStream_t s) {
  k_batch_range<<<grid_for(nitems, ctas), kBatchRangeThreads, 0, s>>>(bf, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_batch_blocks(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                cudaStream_t s) {
  k_batch_blocks<<<grid_for(nitems, ctas), kBatchBlockThreads, 0, s>>>(bf, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_batch_sz_hist(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                 cudaStream_t s) {
  k_batch_sz_hist<<<grid_for(nitems, ctas), kBatchSzThreads, kWideWin * sizeof(uint32_t), s>>>(
      bf, items, nitems);
  return cudaGetLastError();
}

static int occupancy(const void* fn, int threads, int num_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess || per < 1)
    per = 1;
  return per * num_sms;
}

void batch_occupancy(int num_sms, int* range_ctas, int* zfp_ctas, int* sz_ctas) {
  *range_ctas = occupancy((const void*)k_batch_range, kBatchRangeThreads, num_sms);
  *zfp_ctas = occupancy((const void*)k_batch_blocks, kBatchBlockThreads, num_sms);
  cudaFuncSetAttribute(k_batch_sz_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kWideWin * (int)sizeof(uint32_t));
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_batch_sz_hist, kBatchSzThreads,
                                                    kWideWin * sizeof(uint32_t)) != cudaSuccess ||
      per < 1)
    per = 1;
  *sz_ctas = per * num_sms;
}

}  // namespace rdk
