// rd_batch.cu -- the batched estimate (rd_select_batch): three persistent
// passes over the work items of every field of a batch.
//   range: runs of a field's values; the CTA that ends a field's last item
//     (a counter in the field's workspace, fenced on both sides) derives VR,
//     eb_abs and the precision exponent (Algorithm 1 line 2);
//   sampled blocks (one launch per dimensionality): runs of a field's
//     sampled blocks, one thread per block: the block and its one-cell low
//     halo are read once; the SZ residuals of its points (which do not
//     depend on the bin width) are stored, and the ZFP estimator terms
//     accumulated (lines 3-6); the CTA that ends a field's last item
//     derives delta (line 7);
//   SZ histogram: the stored residuals, quantised at delta, coalesced
//     (line 8).
// The sampled blocks are scattered: each block row costs a whole DRAM
// fetch, so one pass that serves both estimators reads about a third of the
// field where two passes read about six tenths.
// CTAs take contiguous ranges of the items of their pass (so that the items
// of one field share a CTA's accumulators); the passes are stream-ordered
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
constexpr int kBatchSzThreads = 1024;

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
      F.ws->sc.clean = 0u;  // the histogram pass writes the tables from here on
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

// Order-preserving 32-bit key of a residual; NaN (a point past the extent)
// gets all ones, after every valid key.
__device__ __forceinline__ uint32_t res_key(float r) {
  const uint32_t b = __float_as_uint(r);
  return isnan(r) ? 0xffffffffu : (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_res(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// One thread per sampled block: the SZ residuals of the block's points (the
// float32 nested differences of est_residual; NaN past the extent) are
// stored for the histogram pass as order-preserving keys, and the block's
// ZFP estimator terms (Alg. 1 lines 4-6) accumulated, the exact error sums
// per block exponent added per warp.
template <int D>
__device__ __forceinline__ void sampled_blocks_item(const BatchField& F, long long b0, long long b1,
                                                    int minexp, unsigned long long& my_s2,
                                                    unsigned long long* s_lo,
                                                    unsigned long long* s_hi) {
  constexpr int NB = 1 << (2 * D);
  constexpr int NC = D == 3 ? 125 : D == 2 ? 25 : 5;
  constexpr EcPositions<D> EC{};
  const FieldDev& f = F.f;
  const bool ec_all = F.p.ec_mode == RD_EC_ALL;
  for (long long base = b0; base < b1; base += blockDim.x) {  // warp-uniform trips
    const long long sb = base + threadIdx.x;
    bool has = false;
    int bin = 0;
    unsigned long long lo = 0ull, hi = 0ull;
    if (sb < b1) {
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
      uint4* dst = reinterpret_cast<uint4*>(F.res + sb * NB);
#pragma unroll
      for (int t = 0; t < NB; t += 4)
        dst[t / 4] = make_uint4(res_key(r[t]), res_key(r[t + 1]), res_key(r[t + 2]), res_key(r[t + 3]));
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
      long long s2;
      zfp_est_terms<D>(w.bi.kmin, ec_all, [&](int j) { return ec_all ? w.u[j] : w.u[EC.pos[j]]; }, s2,
                       lo, hi);
      my_s2 += (unsigned long long)s2;
      has = !w.bi.all_zero && (lo | hi);
      bin = mse_bin<D>(w.bi.emax);
    }
    mse_add_warp(has, bin, lo, hi, s_lo, s_hi);
  }
}

// The items [i0, i1) a CTA takes: contiguous, so that consecutive items of
// one field share the CTA's accumulators and their flush.
__device__ __forceinline__ void cta_items(int nitems, int& i0, int& i1) {
  const int per = (nitems + (int)gridDim.x - 1) / (int)gridDim.x;
  i0 = min(nitems, (int)blockIdx.x * per);
  i1 = min(nitems, i0 + per);
}

// Adds the CTA's ZFP terms of field F (cnt items) to its workspace; the CTA
// that brings the field's item count to items_zfp derives delta.
__device__ __forceinline__ void zfp_commit(const BatchField& F, uint32_t cnt,
                                           unsigned long long my_s2, unsigned long long* s_lo,
                                           unsigned long long* s_hi, unsigned long long* s_s2,
                                           int* s_last) {
  Workspace* ws = F.ws;
  my_s2 = warp_sum(my_s2);
  if ((threadIdx.x & 31) == 0 && my_s2) atomicAdd(s_s2, my_s2);
  __syncthreads();
  if (threadIdx.x == 0 && *s_s2) atomicAdd(&ws->sc.s2, *s_s2);
  for (int i = threadIdx.x; i < kMseBins; i += blockDim.x)
    if (s_lo[i] | s_hi[i]) atomic_add_u128(&ws->sc.mse_lo[i], &ws->sc.mse_hi[i], s_lo[i], s_hi[i]);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *s_last = atomicAdd(&ws->sc.done[1], cnt) + cnt == F.items_zfp;
  }
  __syncthreads();
  if (*s_last && threadIdx.x < 32) {
    __threadfence();
    delta_warp(F.p, ws, DELTA_FROM_MSE, 0.0, 1, F.need_gt, F.ncoeff, F.npoints);
  }
  __syncthreads();
}

// One launch per dimensionality (the items of d-dimensional fields): the
// registers of the 3D form would otherwise set the occupancy of all.
template <int D>
__global__ void __launch_bounds__(kBatchBlockThreads) k_batch_blocks(const BatchField* __restrict__ bf,
                                                                     const BatchItem* __restrict__ items,
                                                                     int nitems) {
  __shared__ unsigned long long s_lo[kMseBins], s_hi[kMseBins];
  __shared__ unsigned long long s_s2;
  __shared__ int s_last;
  int i0, i1;
  cta_items(nitems, i0, i1);
  int cur = -1;  // the field the accumulators hold
  uint32_t cnt = 0u;
  unsigned long long my_s2 = 0ull;
  for (int it = i0; it < i1; it++) {
    const BatchItem item = items[it];
    if (item.field != cur) {  // uniform over the CTA
      if (cur >= 0) zfp_commit(bf[cur], cnt, my_s2, s_lo, s_hi, &s_s2, &s_last);
      for (int i = threadIdx.x; i < kMseBins; i += blockDim.x) {
        s_lo[i] = 0ull;
        s_hi[i] = 0ull;
      }
      if (threadIdx.x == 0) s_s2 = 0ull;
      __syncthreads();
      cur = item.field;
      cnt = 0u;
      my_s2 = 0ull;
    }
    const BatchField& F = bf[item.field];
    Workspace* ws = F.ws;
    cnt++;
    if (ws->sc.status != RD_OK || ws->sc.constant) continue;  // uniform over the CTA
    sampled_blocks_item<D>(F, item.begin, item.end, ws->sc.minexp, my_s2, s_lo, s_hi);
  }
  if (cur >= 0) zfp_commit(bf[cur], cnt, my_s2, s_lo, s_hi, &s_s2, &s_last);
}

// ---------------------------------------------------------------------------
// SZ histogram of the stored residuals (Alg. 1 line 8), coalesced
// ---------------------------------------------------------------------------

// Counts two keys of the residual list (one lane): each key's code adds one
// to its 16-bit counter (raising *s_hot when the counter reaches
// kHotCount).  All-ones keys (points past the extent, or past the list)
// count nothing.  (Merging runs of equal codes within a warp first, with
// ballots, cost more than it saved: 0.240 against 0.206 ms on the snapshot.)
__device__ __forceinline__ void hist_add2(uint32_t* s_win, uint32_t ka, uint32_t kb, float inv, int R,
                                          int* s_hot) {
  if (ka != 0xffffffffu) packed_add(s_win, est_symbol(key_res(ka), inv, R), 1u, s_hot);
  if (kb != 0xffffffffu) packed_add(s_win, est_symbol(key_res(kb), inv, R), 1u, s_hot);
}


__global__ void __launch_bounds__(kBatchSzThreads, 1) k_batch_sz_hist(const BatchField* __restrict__ bf,
                                                                   const BatchItem* __restrict__ items,
                                                                   int nitems) {
  extern __shared__ uint32_t s_win[];  // kPackWords words of two counters
  __shared__ int s_hot;                // a counter reached kHotCount
  int i0, i1;
  cta_items(nitems, i0, i1);
  for (int i = threadIdx.x; i < kPackWords; i += blockDim.x) s_win[i] = 0u;
  if (threadIdx.x == 0) s_hot = 0;
  __syncthreads();
  int cur = -1;  // the field the window holds
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = kBatchSzThreads / 32;
  constexpr int U = 4;  // independent 8-byte loads in flight per lane
  for (int it = i0; it < i1; it++) {
    const BatchItem item = items[it];
    const BatchField& F = bf[item.field];
    Workspace* ws = F.ws;
    if (item.field != cur) {  // uniform over the CTA
      if (cur >= 0) window_flush(s_win, bf[cur].ws->hist[0]);
      cur = item.field;
    }
    if (ws->sc.status != RD_OK || ws->sc.constant) continue;
    const float inv = ws->sc.inv;
    const int R = F.p.R;
    const long long nb = 1ll << (2 * F.f.d);
    // the item's keys as pairs, in rounds of kRoundPoints keys; a warp
    // takes 64 consecutive keys (2 per lane) at a time
    const uint2* k2 = reinterpret_cast<const uint2*>(F.res + item.begin * nb);
    const long long npts = (item.end - item.begin) * nb;
    for (long long r0 = 0; r0 < npts; r0 += kRoundPoints) {
      const long long rn = npts - r0 < kRoundPoints ? npts - r0 : kRoundPoints;
      const uint2* q2 = k2 + r0 / 2;
      const int n2 = (int)(rn / 2);
      const int nchunks = (n2 + 31) >> 5;
      for (int c0 = warp; c0 < nchunks; c0 += U * W) {  // warp-uniform
        uint2 q[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
          const int c = c0 + k * W;
          const int g = 32 * c + lane;
          q[k] = (c < nchunks && g < n2) ? __ldcs(q2 + g) : make_uint2(0xffffffffu, 0xffffffffu);
        }
#pragma unroll
        for (int k = 0; k < U; k++) hist_add2(s_win, q[k].x, q[k].y, inv, R, &s_hot);
      }
      __syncthreads();
      if (s_hot) {  // uniform after the barrier
        window_flush(s_win, ws->hist[0]);
        if (threadIdx.x == 0) s_hot = 0;
        __syncthreads();
      }
    }
  }
  if (cur >= 0) window_flush(s_win, bf[cur].ws->hist[0]);
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

cudaError_t launch_batch_blocks(const BatchField* bf, const BatchItem* items, int nitems, int d,
                                int ctas, cudaStream_t s) {
  const int g = grid_for(nitems, ctas);
  if (d == 1)
    k_batch_blocks<1><<<g, kBatchBlockThreads, 0, s>>>(bf, items, nitems);
  else if (d == 2)
    k_batch_blocks<2><<<g, kBatchBlockThreads, 0, s>>>(bf, items, nitems);
  else
    k_batch_blocks<3><<<g, kBatchBlockThreads, 0, s>>>(bf, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_batch_sz_hist(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                 cudaStream_t s) {
  k_batch_sz_hist<<<grid_for(nitems, ctas), kBatchSzThreads, kPackWords * sizeof(uint32_t), s>>>(
      bf, items, nitems);
  return cudaGetLastError();
}

static int occupancy(const void* fn, int threads, int num_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess || per < 1)
    per = 1;
  return per * num_sms;
}

void batch_occupancy(int num_sms, int* range_ctas, int* blocks_ctas, int* sz_ctas) {
  *range_ctas = occupancy((const void*)k_batch_range, kBatchRangeThreads, num_sms);
  blocks_ctas[0] = occupancy((const void*)k_batch_blocks<1>, kBatchBlockThreads, num_sms);
  blocks_ctas[1] = occupancy((const void*)k_batch_blocks<2>, kBatchBlockThreads, num_sms);
  blocks_ctas[2] = occupancy((const void*)k_batch_blocks<3>, kBatchBlockThreads, num_sms);
  cudaFuncSetAttribute(k_batch_sz_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kPackWords * (int)sizeof(uint32_t));
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_batch_sz_hist, kBatchSzThreads,
                                                    kPackWords * sizeof(uint32_t)) != cudaSuccess ||
      per < 1)
    per = 1;
  *sz_ctas = per * num_sms;
}

}  // namespace rdk
