// rd_batch.cu -- the batched estimate (rd_select_batch): three persistent
// passes over the work items of every field of a batch.
//   range: runs of a field's values; the CTA that ends a field's last item
//     (a counter in the field's workspace, fenced on both sides) derives VR,
//     eb_abs and the precision exponent (Algorithm 1 line 2);
//   ZFP estimate: runs of a field's sampled blocks, one thread per block
//     (lines 3-6); the CTA that ends a field's last item derives delta
//     (line 7);
//   SZ estimate: runs of a field's sampled blocks, one thread per block
//     (line 8).
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
constexpr int kBatchZfpThreads = 128;
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
// ZFP estimate
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBatchZfpThreads) k_batch_zfp_est(const BatchField* __restrict__ bf,
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
        case 1: zfp_est_item<1>(F.f, F.p, minexp, item.begin, item.end, my_s2, s_lo, s_hi); break;
        case 2: zfp_est_item<2>(F.f, F.p, minexp, item.begin, item.end, my_s2, s_lo, s_hi); break;
        default: zfp_est_item<3>(F.f, F.p, minexp, item.begin, item.end, my_s2, s_lo, s_hi); break;
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
// SZ estimate, one thread per sampled block (sz_est_block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBatchSzThreads) k_batch_sz_est(const BatchField* __restrict__ bf,
                                                                  const BatchItem* __restrict__ items,
                                                                  int nitems) {
  __shared__ uint32_t s_win[kHistWin];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem item = items[it];
    const BatchField& F = bf[item.field];
    Workspace* ws = F.ws;
    if (ws->sc.status != RD_OK || ws->sc.constant) continue;  // uniform over the CTA
    for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) s_win[i] = 0u;
    __syncthreads();
    const float inv = ws->sc.inv;
    switch (F.f.d) {
      case 1: sz_est_item<1>(F.f, F.p.R, inv, ws->hist[0], item.begin, item.end, s_win); break;
      case 2: sz_est_item<2>(F.f, F.p.R, inv, ws->hist[0], item.begin, item.end, s_win); break;
      default: sz_est_item<3>(F.f, F.p.R, inv, ws->hist[0], item.begin, item.end, s_win); break;
    }
    __syncthreads();
    hist_flush(s_win, ws->hist[0]);
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

cudaError_t launch_batch_zfp_est(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                 cudaStream_t s) {
  k_batch_zfp_est<<<grid_for(nitems, ctas), kBatchZfpThreads, 0, s>>>(bf, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_batch_sz_est(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                cudaStream_t s) {
  k_batch_sz_est<<<grid_for(nitems, ctas), kBatchSzThreads, 0, s>>>(bf, items, nitems);
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
  *zfp_ctas = occupancy((const void*)k_batch_zfp_est, kBatchZfpThreads, num_sms);
  *sz_ctas = occupancy((const void*)k_batch_sz_est, kBatchSzThreads, num_sms);
}

}  // namespace rdk
