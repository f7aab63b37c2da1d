// rd_reduce.cu -- the small kernels of one rate-distortion call: workspace
// reset, value range (Algorithm 1 line 2), the bin width delta from the exact
// MSE_sp (line 7), the entropy and Huffman cost of the code histograms
// (lines 8-9 and the SZ ground truth) and the final selection (lines 10-12).
#include <math.h>
#include <stdint.h>

#include "rd_delta.cuh"
#include "rd_finish.cuh"
#include "rd_device.cuh"
#include "rd_range_dev.cuh"

namespace rdk {

// ---------------------------------------------------------------------------
// Reset: zero accumulators and histograms of the workspace.
// ---------------------------------------------------------------------------
__device__ void reset_ws(Workspace* ws, int tid, int nth, int which_mask) {
#pragma unroll 1
  for (int w = 0; w < 2; w++) {
    if (!((which_mask >> w) & 1)) continue;
    uint4* h = reinterpret_cast<uint4*>(ws->hist[w]);
    uint4* cc = reinterpret_cast<uint4*>(ws->count_of[w]);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < kNsym / 4; i += nth) {
      h[i] = z;
      cc[i] = z;
    }
    uint32_t* pr = ws->present[w];
    for (int i = tid; i < kNsym / 32; i += nth) pr[i] = 0u;
  }
  unsigned long long* lo = ws->sc.mse_lo;
  unsigned long long* hi = ws->sc.mse_hi;
  for (int i = tid; i < kMseBins; i += nth) {
    lo[i] = 0ull;
    hi[i] = 0ull;
  }
  if (tid == 0) {
    Scalars& s = ws->sc;
    s.status = RD_OK;
    s.flags = 0u;
    s.constant = 0;
    s.minexp = 0;
    s.min_key = 0xffffffffu;
    s.max_key = 0u;
    s.nonfinite = 0u;
    s.done[0] = s.done[1] = 0u;
    s.vmin = s.vmax = s.amax = 0.0f;
    s.w = s.inv = s.tau = 0.0f;
    s.vr = s.eb_abs = s.delta = s.mse_sp = 0.0;
    s.s2 = 0ull;
    s.zfp_bits = 0ull;
    s.zfp_maxerr = 0u;
    s.sz_maxerr = 0u;
    s.log_maxabs = 0u;
    s.huff_done = 0u;
    s.zfp_done = 0u;
    for (int w = 0; w < 2; w++) {
      ws->nbig[w] = 0u;
      ws->huff[w].ns = 0ull;
      ws->huff[w].cost = 0ull;
      ws->huff[w].nsym = 0u;
      ws->huff[w].plogp = 0.0;
    }
    unsigned char* r = reinterpret_cast<unsigned char*>(&ws->res);
    for (size_t i = 0; i < sizeof(rd_result); i++) r[i] = 0;
    unsigned char* t = reinterpret_cast<unsigned char*>(&ws->truth);
    for (size_t i = 0; i < sizeof(rd_truth); i++) t[i] = 0;
  }
}

__global__ void k_reset(Workspace* ws) {
  reset_ws(ws, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, 3);
}

cudaError_t launch_reset(Workspace* ws, cudaStream_t s) {
  k_reset<<<128, 256, 0, s>>>(ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Value range: min / max over every value, with a non-finite test.  Rows are
// read as float4 where the pointer allows it.
// ---------------------------------------------------------------------------
// The CTA that ends last (a counter, fenced on both sides) derives VR,
// eb_abs and minexp (Algorithm 1 line 2).
// With kCopy, x is the field in host memory the device can address (pinned)
// and every value is also stored at copy (the device staging buffer): the
// host-to-device transfer is the range pass's own read.
template <bool kCopy>
__global__ void __launch_bounds__(512) k_range(const float* __restrict__ x, long long n,
                                               ParamsDev p, Workspace* ws, float* __restrict__ copy) {
  __shared__ int s_last;
  RangeAcc acc;
  range_span<kCopy>(x, 0, n, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x, acc, copy);
  range_commit(acc, ws);
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ws->sc.done[0], 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    prepare_field(p, ws);
  }
}

cudaError_t launch_range(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                         cudaStream_t s, const float* host_src) {
  long long want = (f.N / 4 + 511) / 512;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (host_src)
    k_range<true><<<g, 512, 0, s>>>(host_src, f.N, p, ws, const_cast<float*>(f.x));
  else
    k_range<false><<<g, 512, 0, s>>>(f.x, f.N, p, ws, nullptr);
  return cudaGetLastError();
}

// Bin width delta (Algorithm 1 line 7): one warp.
__global__ void k_delta(ParamsDev p, Workspace* ws, int mode, double arg, int need_quant,
                        int need_gt, unsigned long long ncoeff, unsigned long long npoints) {
  delta_warp(p, ws, mode, arg, need_quant, need_gt, ncoeff, npoints);
}

cudaError_t launch_delta(const ParamsDev& p, Workspace* ws, int mode, double arg, int need_quant,
                         int need_gt, unsigned long long ncoeff, unsigned long long npoints,
                         cudaStream_t s) {
  k_delta<<<1, 32, 0, s>>>(p, ws, mode, arg, need_quant, need_gt, ncoeff, npoints);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Code statistics of the histograms (Algorithm 1 lines 8-9 and the SZ ground
// truth), in two launches: k_code_prep spreads each histogram over
// kEntropyCtas CTAs (entropy partials, count-of-counts), k_huffman runs one
// CTA per histogram for the Huffman cost.
//
// Huffman cost (sum of internal-node weights = coded bits).  The nonzero
// counts are sorted ascending (a counting sort by count value; the rare
// counts of 2^16 or more by a bitonic network).  The two-queue method
// consumes leaves and internal nodes in ascending order and pairs them
// consecutively; it runs here in phases: with a0 <= a1 the two smallest
// remaining items, every item below T = a0 + a1 is consumed before any new
// node (new nodes are >= T), so all such items are paired at once, in merged
// order, and the new nodes (non-decreasing, as in the sequential method) are
// appended to the internal queue.  The result equals the sequential merge.
// ---------------------------------------------------------------------------
__device__ void bitonic_sort(uint32_t* a, int n) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    // first stage of each merge compares mirrored partners
    for (int q = threadIdx.x; q < P / 2; q += blockDim.x) {
      int half = k >> 1;
      int i = (q / half) * k + (q % half);
      int j = i ^ (k - 1);
      if (j < n) {
        uint32_t x = a[i], y = a[j];
        if (x > y) { a[i] = y; a[j] = x; }
      }
    }
    __syncthreads();
    for (int jj = k >> 2; jj > 0; jj >>= 1) {
      for (int q = threadIdx.x; q < P / 2; q += blockDim.x) {
        int i = (q / jj) * (2 * jj) + (q % jj);
        int j = i + jj;
        if (j < n) {
          uint32_t x = a[i], y = a[j];
          if (x > y) { a[i] = y; a[j] = x; }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int kPrepThreads = 256;   // code-statistics prep CTAs (1024 bins each)
constexpr int kHuffThreads = 1024;  // Huffman CTA
constexpr uint32_t kMinPairs = 1;   // fewest pairs per thread in a Huffman phase

// Numbers of elements below T of the sorted a[0..na) and b[0..nb), found
// together by one warp: each round tests 128 evenly spaced elements of every
// range still wider than 128 (four per lane, loaded together) and keeps the
// gap holding the answer; a range of at most 128 is answered by one round
// of four ballots.  T < 2^33; a T of 2^32 or more exceeds every 32-bit
// element.
template <class VA, class VB>
__device__ __forceinline__ void warp_count_below2(const VA& a, uint32_t na, const VB& b, uint32_t nb,
                                                  unsigned long long T, uint32_t& ra,
                                                  uint32_t& rb) {
  if (T > 0xffffffffull) {
    ra = na;
    rb = nb;
    return;
  }
  const uint32_t t = (uint32_t)T;
  const uint32_t lane = threadIdx.x & 31u;
  constexpr uint32_t kOpen = 0xffffffffu;
  constexpr uint32_t kProbes = 128u;
  uint32_t alo = 0u, ahi = na, blo = 0u, bhi = nb;
  ra = kOpen;
  rb = kOpen;
  while (ra == kOpen || rb == kOpen) {
    const bool wa = ahi - alo > kProbes, wb = bhi - blo > kProbes;
    const uint32_t sa = wa ? (ahi - alo + kProbes - 1u) / kProbes : 1u;
    const uint32_t sb = wb ? (bhi - blo + kProbes - 1u) / kProbes : 1u;
    bool pa[4], pb[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t q = (uint32_t)u * 32u + lane;
      const uint32_t ia = alo + q * sa, ib = blo + q * sb;
      pa[u] = ra == kOpen && ia < ahi && a[ia] < t;
      pb[u] = rb == kOpen && ib < bhi && b[ib] < t;
    }
    uint32_t ca = 0u, cb = 0u;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      ca += (uint32_t)__popc(__ballot_sync(0xffffffffu, pa[u]));
      cb += (uint32_t)__popc(__ballot_sync(0xffffffffu, pb[u]));
    }
    if (ra == kOpen) {
      if (!wa) {
        ra = alo + ca;
      } else if (ca == 0u) {
        ra = alo;
      } else {
        const uint32_t nh = alo + ca * sa;
        alo += (ca - 1u) * sa + 1u;
        ahi = nh < ahi ? nh : ahi;
      }
    }
    if (rb == kOpen) {
      if (!wb) {
        rb = blo + cb;
      } else if (cb == 0u) {
        rb = blo;
      } else {
        const uint32_t nh = blo + cb * sb;
        blo += (cb - 1u) * sb + 1u;
        bhi = nh < bhi ? nh : bhi;
      }
    }
  }
}

// The internal-node queue of the run-length form (below) as a ring of cap
// words: element k of the queue from position off.
struct RingView {
  const uint32_t* q;
  uint32_t off, cap;
  __device__ __forceinline__ uint32_t operator[](uint32_t k) const {
    const uint32_t p = off + k;  // off < cap and k < cap
    return q[p >= cap ? p - cap : p];
  }
};

// The run holding leaf o: the last r with rs[r] <= o (rs[0] = 0).
__device__ __forceinline__ uint32_t run_of(const uint32_t* rs, uint32_t R, uint32_t o) {
  uint32_t lo = 0u, hi = R;
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (rs[mid] <= o) lo = mid; else hi = mid;
  }
  return lo;
}

// The merge split (the number of leaves among the first d items of the
// merged order, ties from the leaves first) with the leaves in run-length
// form: A[i] is leaf lh + i, run r
// holding leaves rs[r] .. rs[r+1]-1, all of weight rv[r].  The predicate
// A[i] <= B[d-1-i] is tested first at the starts of runs, then inside the
// one run where it turns false.  Returns the split and, in run, the run of
// leaf lh + split.
template <class VB>
__device__ __forceinline__ uint32_t merge_split_runs(const uint32_t* rv, const uint32_t* rs,
                                                     uint32_t R, uint32_t lh, uint32_t na,
                                                     const VB& B, uint32_t nb, uint32_t d,
                                                     uint32_t& run) {
  const uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  const uint32_t r0 = run_of(rs, R, lh + lo);
  run = r0;
  if (lo == hi || rv[r0] > B[d - 1 - lo]) return lo;
  // the last run whose first leaf in [lo, hi) still satisfies the predicate
  uint32_t a = r0, b = R;
  while (b - a > 1u) {
    const uint32_t mid = (a + b) >> 1;
    const uint32_t s = rs[mid] - lh;  // > lo: mid is past the run of lo
    if (s < hi && rv[mid] <= B[d - 1 - s]) a = mid; else b = mid;
  }
  const uint32_t v = rv[a];
  const uint32_t end = rs[a + 1] - lh;
  uint32_t l2 = (a == r0 ? lo : rs[a] - lh) + 1u, h2 = end < hi ? end : hi;
  while (l2 < h2) {
    const uint32_t mid = (l2 + h2) >> 1;
    if (v <= B[d - 1 - mid]) l2 = mid + 1u; else h2 = mid;
  }
  run = l2 < end ? a : a + 1u;
  return l2;
}

// ---------------------------------------------------------------------------
// Table of v log2 v for the entropy (v < 2^16), filled once per context.
// ---------------------------------------------------------------------------
__global__ void k_init_xlogx(double* xlogx) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < kNsym) xlogx[v] = v > 1 ? (double)v * log2((double)v) : 0.0;
}

cudaError_t launch_init_tables(double* xlogx, cudaStream_t s) {
  k_init_xlogx<<<kNsym / 256, 256, 0, s>>>(xlogx);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prep (kEntropyCtas CTAs per histogram, 1024 bins each): the multiplicity
// of every count value below 2^16 (a counting sort of the counts; lanes
// holding equal counts merge into one atomic), a bitmap of the count values
// present, the counts of 2^16 or more (at most N / 2^16 of them) appended
// to a list, and the slice's shares of N_s = sum c and of the entropy sum
// sum c log2 c (from the table below 2^16), each summed in a fixed order.
// ---------------------------------------------------------------------------
// With kClear, every nonzero bin read is set back to zero, except bin 0 (the
// escape count, read by the finish step).
template <bool kClear>
__device__ __forceinline__ void code_prep_slice(Workspace* ws, int which, int slice,
                                                const double* __restrict__ xlogx) {
  __shared__ double part[kPrepThreads / 32];
  __shared__ unsigned long long npart[kPrepThreads / 32];
  if (ws->sc.status != RD_OK || ws->sc.constant) return;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint32_t* cc = ws->count_of[which];
  uint32_t* present = ws->present[which];
  uint32_t* big = ws->node_scratch[which];
  double v = 0.0;
  unsigned long long nsum = 0ull;
  constexpr int kPer = 1024 / kPrepThreads;
  // the bins and their table entries loaded together, ahead of the atomics
  uint32_t cs[kPer];
  double xs[kPer];
#pragma unroll
  for (int k = 0; k < kPer; k++) cs[k] = ws->hist[which][slice * 1024 + k * kPrepThreads + threadIdx.x];
#pragma unroll
  for (int k = 0; k < kPer; k++) xs[k] = (cs[k] != 0u && cs[k] < (uint32_t)kNsym) ? xlogx[cs[k]] : 0.0;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int bin = slice * 1024 + k * kPrepThreads + threadIdx.x;
    const uint32_t c = cs[k];
    if (kClear && c != 0u && bin != 0) ws->hist[which][bin] = 0u;
    const bool small = c != 0u && c < (uint32_t)kNsym;
    const bool large = c >= (uint32_t)kNsym;
    nsum += c;
    v += xs[k];
    const unsigned ms = __ballot_sync(0xffffffffu, small);
    const unsigned mb = __ballot_sync(0xffffffffu, large);
    if (small) {
      const unsigned same = __match_any_sync(ms, c);
      if (lane == __ffs(same) - 1) {
        if (atomicAdd(&cc[c], (uint32_t)__popc(same)) == 0u)
          atomicOr(&present[c >> 5], 1u << (c & 31u));
      }
    }
    if (mb) {
      uint32_t base = 0u;
      if (lane == __ffs(mb) - 1) base = atomicAdd(&ws->nbig[which], (uint32_t)__popc(mb));
      base = __shfl_sync(0xffffffffu, base, __ffs(mb) - 1);
      if (large) {
        big[base + __popc(mb & lt_mask)] = c;
        v += (double)c * log2((double)c);
      }
    }
  }
  v = warp_sum(v);
  nsum = warp_sum(nsum);
  if (lane == 0) {
    part[threadIdx.x >> 5] = v;
    npart[threadIdx.x >> 5] = nsum;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = threadIdx.x < kPrepThreads / 32;
    const double t = warp_sum(in ? part[threadIdx.x] : 0.0);
    const unsigned long long nt = warp_sum(in ? npart[threadIdx.x] : 0ull);
    if (threadIdx.x == 0) {
      ws->ent_part[which][slice] = t;
      ws->ns_part[which][slice] = nt;
    }
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_code_prep(Workspace* ws, int which_mask,
                                                            const double* __restrict__ xlogx) {
  const int first = (which_mask & 1) ? 0 : 1;
  code_prep_slice<false>(ws, first + blockIdx.x / kEntropyCtas, blockIdx.x % kEntropyCtas, xlogx);
}

// Block-wide scans and sums for kHuffThreads threads (32 warps); s_w holds
// 32 words of scratch.  Each ends with a barrier, so s_w can be reused.
__device__ uint32_t block_excl_sum(uint32_t v, uint32_t* s_w, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += t;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = s_w[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += t;
    }
    s_w[lane] = w;
  }
  __syncthreads();
  const uint32_t base = wid ? s_w[wid - 1] : 0u;
  *total = s_w[31];
  __syncthreads();
  return base + inc - v;
}

// exclusive running maximum
__device__ uint32_t block_excl_max(uint32_t v, uint32_t* s_w) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc = max(inc, t);
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = s_w[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w = max(w, t);
    }
    s_w[lane] = w;
  }
  __syncthreads();
  uint32_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) ex = 0u;
  if (wid) ex = max(ex, s_w[wid - 1]);
  __syncthreads();
  return ex;
}

// fixed-order block sums, valid in every thread
__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* s_w) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  const unsigned long long t = warp_sum(s_w[threadIdx.x & 31]);
  __syncthreads();
  return t;
}

// The Huffman phases once every remaining item lies below the threshold
// (the sum of the two smallest).  Then every later phase pairs all of its
// items in order: for a sorted list Q with Q[L-1] < Q[0] + Q[1] the next
// list (the last item when L is odd, then the pair sums) is sorted again, and
// again all below its threshold, since Q[L-3] + Q[L-2] < (Q[0] + Q[1]) +
// Q[L-1] and Q[L-2] + Q[L-1] < 2 (Q[0] + Q[1]).  So a phase needs neither
// the threshold search nor a merge.  The list is the front item f (when fv),
// then n queue words from position base; new nodes go from position it on.
// at(p, k) is the queue word k places after position p, nxt(p, k) its
// position.  One barrier per phase: a phase reads the words the one before
// wrote and writes past them.  Returns this thread's share of the cost.
template <class At, class Nxt>
__device__ __forceinline__ unsigned long long huffman_tail(At at, Nxt nxt, bool fv, uint32_t f,
                                                           uint32_t base, uint32_t n, uint32_t it) {
  unsigned long long cost = 0ull;
  const uint32_t tid = threadIdx.x;
  for (;;) {
    const uint32_t L = n + (fv ? 1u : 0u);
    if (L <= 1u) break;
    const uint32_t np = L >> 1;
    for (uint32_t j = tid; j < np; j += kHuffThreads) {
      const uint32_t v0 = fv ? (j == 0u ? f : at(base, 2u * j - 1u)) : at(base, 2u * j);
      const uint32_t v1 = fv ? at(base, 2u * j) : at(base, 2u * j + 1u);
      const uint32_t sum = v0 + v1;
      at(it, j) = sum;
      cost += sum;
    }
    const bool odd = (L & 1u) != 0u;
    const uint32_t last = odd ? at(base, n - 1u) : 0u;  // the list's last item
    __syncthreads();
    fv = odd;
    f = last;
    base = it;
    n = np;
    it = nxt(it, np);
  }
  return cost;
}

// Phases of the two-queue merge with the leaves in run-length form, for
// alphabets past the linear shared-memory form: the ascending leaves are
// runs of equal weight (rv[r], first leaf rs[r]; the D distinct small
// counts, then the large counts one run each), and the internal nodes live
// in a ring of C words.  Before a phase the L live nodes are disjoint
// subtrees of at least two leaves each, so L <= lh / 2 and the phase's new
// nodes np <= ((K - lh) + L) / 2; L + np <= 3K/4 < C, so new nodes never
// overwrite a node still to be read.  Returns this thread's share of the
// cost.
__device__ unsigned long long huffman_runs(const uint32_t* dv, uint32_t D, const uint32_t* big,
                                           uint32_t nbig, uint32_t nsmall, uint32_t K,
                                           uint32_t* s_w) {
  // the runs and the ring in shared memory, addressed as such (every phase
  // is a chain of dependent loads)
  extern __shared__ uint32_t s_dyn[];
  const uint32_t tid = threadIdx.x;
  const uint32_t R = D + nbig;
  const uint32_t C = (3u * K + 3u) / 4u + 1u;
  uint32_t* rv = s_dyn;
  uint32_t* rs = s_dyn + R;
  uint32_t* ring = s_dyn + 2u * R + 1u;
  {
    const uint32_t Cd = (D + kHuffThreads - 1) / kHuffThreads;
    const uint32_t e0 = min(D, tid * Cd), e1 = min(D, e0 + Cd);
    uint32_t mloc = 0u;
    for (uint32_t d = e0; d < e1; d++) mloc += (dv[d] & 0xffffu) + 1u;
    uint32_t tot;
    uint32_t start = block_excl_sum(mloc, s_w, &tot);
    for (uint32_t d = e0; d < e1; d++) {
      const uint32_t q = dv[d];
      rv[d] = q >> 16;
      rs[d] = start;
      start += (q & 0xffffu) + 1u;
    }
    for (uint32_t i = tid; i < nbig; i += kHuffThreads) rv[D + i] = big[i];
    __syncthreads();
    bitonic_sort(rv + D, (int)nbig);
    for (uint32_t i = tid; i < nbig; i += kHuffThreads) rs[D + i] = nsmall + i;
    if (tid == 0) rs[R] = K;
    __syncthreads();
  }
  unsigned long long cost = 0ull;
  uint32_t lh = 0u, ih = 0u, it = 0u;  // leaf head, node head, node tail
  uint32_t ihr = 0u, itr = 0u;         // ring positions of ih and it
  for (;;) {
    if ((K - lh) + (it - ih) <= 1u) break;
    if (tid < 32) {
      const RingView B{ring, ihr, C};
      unsigned long long c4[4] = {~0ull, ~0ull, ~0ull, ~0ull};
      if (lh < K) {
        const uint32_t r = run_of(rs, R, lh);
        c4[0] = rv[r];
        if (lh + 1u < K) c4[1] = lh + 1u < rs[r + 1u] ? rv[r] : rv[r + 1u];
      }
      if (ih < it) c4[2] = B[0];
      if (ih + 1u < it) c4[3] = B[1];
      const unsigned long long m01 = min(c4[0], c4[1]), x01 = max(c4[0], c4[1]);
      const unsigned long long m23 = min(c4[2], c4[3]), x23 = max(c4[2], c4[3]);
      const unsigned long long a0 = min(m01, m23);
      const unsigned long long a1 = m01 < m23 ? min(x01, m23) : min(x23, m01);
      // runs of weight below T end at leaf rs[rc]
      uint32_t rc, mi;
      warp_count_below2(rv, R, B, it - ih, a0 + a1, rc, mi);
      const uint32_t first = rs[rc];
      const uint32_t ml = first > lh ? first - lh : 0u;
      uint32_t cl = ml;
      if ((ml + mi) & 1u) {
        if (mi == 0u || (ml > 0u && rv[rc - 1u] > B[mi - 1u])) cl = ml - 1u;
      }
      if (tid == 0) {
        s_w[0] = ml;
        s_w[1] = mi;
        s_w[2] = cl;
      }
    }
    __syncthreads();
    const uint32_t ml = s_w[0], mi = s_w[1], cl = s_w[2];
    const uint32_t np = (ml + mi) >> 1;
    const bool all_below = ml + mi == (K - lh) + (it - ih);
    const uint32_t per_t = max(kMinPairs, (np + kHuffThreads - 1) / kHuffThreads);
    const uint32_t j0 = tid * per_t;
    const uint32_t j1 = min(np, j0 + per_t);
    if (j0 < j1) {
      const RingView B{ring, ihr, C};
      uint32_t r;
      uint32_t i = merge_split_runs(rv, rs, R, lh, ml, B, mi, 2u * j0, r);
      uint32_t k = 2u * j0 - i;
      uint32_t vA = r < R ? rv[r] : 0u;
      uint32_t endA = r < R ? rs[r + 1u] - lh : 0xffffffffu;
      uint32_t bp = ihr + k;
      if (bp >= C) bp -= C;
      uint32_t wp = itr + j0;
      if (wp >= C) wp -= C;
      for (uint32_t j = j0; j < j1; j++) {
        uint32_t e[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          if (i < ml && (k >= mi || vA <= ring[bp])) {
            e[u] = vA;
            if (++i == endA) {
              r++;
              vA = r < R ? rv[r] : 0u;
              endA = r < R ? rs[r + 1u] - lh : 0xffffffffu;
            }
          } else {
            e[u] = ring[bp];
            k++;
            if (++bp == C) bp = 0u;
          }
        }
        const uint32_t sum = e[0] + e[1];
        ring[wp] = sum;
        if (++wp == C) wp = 0u;
        cost += sum;
      }
    }
    __syncthreads();
    const uint32_t used = 2u * np - cl;  // nodes consumed
    lh += cl;
    ih += used;
    ihr += used;
    if (ihr >= C) ihr -= C;
    it += np;
    itr += np;
    if (itr >= C) itr -= C;
    if (all_below) {
      // what is left: a leaf (odd count), then the nodes from ring position ihr
      const bool fv = lh < K;
      const uint32_t f = fv ? rv[run_of(rs, R, lh)] : 0u;
      auto at = [&](uint32_t p, uint32_t k) -> uint32_t& {
        uint32_t q = p + k;  // p < C, k < C
        if (q >= C) q -= C;
        return ring[q];
      };
      auto nxt = [&](uint32_t p, uint32_t k) {
        uint32_t q = p + k;
        return q >= C ? q - C : q;
      };
      cost += huffman_tail(at, nxt, fv, f, ihr, it - ih, itr);
      break;
    }
  }
  return cost;
}

// Keys of queue items for the windowed merge: the weight doubled, plus one
// for an internal node, so that key order is weight order with leaves first
// among equal weights (weights are below 2^31: fields hold fewer points).
__device__ __forceinline__ uint32_t hkey_leaf(uint32_t v) { return v << 1; }
__device__ __forceinline__ uint32_t hkey_node(uint32_t v) { return (v << 1) | 1u; }

// Number of A items among the first d of merge(A, B) (ties from A first),
// found by one warp: the predicate A[i] <= B[d-1-i] holds for a prefix of i
// in [lo, hi); each round tests 128 evenly spaced i (four per lane) and
// keeps the gap holding the first failure.
template <class VA, class VB>
__device__ __forceinline__ uint32_t warp_merge_split(const VA& A, uint32_t na, const VB& B, uint32_t nb,
                                                     uint32_t d) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t n = hi - lo;
    const uint32_t st = n > 128u ? (n + 127u) / 128u : 1u;
    bool pr[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t i = lo + ((uint32_t)u * 32u + lane) * st;
      pr[u] = i < hi && A[i] <= B[d - 1u - i];
    }
    uint32_t c = 0u;
#pragma unroll
    for (int u = 0; u < 4; u++) c += (uint32_t)__popc(__ballot_sync(0xffffffffu, pr[u]));
    if (st == 1u) return lo + c;  // every i of the range tested
    if (c == 0u) return lo;
    const uint32_t nh = lo + c * st;
    lo += (c - 1u) * st + 1u;
    hi = nh < hi ? nh : hi;
  }
  return lo;
}

// The 64 smallest of 64 rising keys a (a0 at lane l is item l, a1 item
// 32 + l) and 64 rising keys b (the same layout), in rising order as r0
// (item l) and r1 (item 32 + l): a half-cleaner on a followed by b reversed
// (a bitonic sequence) keeps the lower half, then a bitonic sort of it.
__device__ __forceinline__ void window_merge64(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1,
                                               uint32_t& r0, uint32_t& r1) {
  const uint32_t lane = threadIdx.x & 31u;
  // item e of the lower half: min(a[e], b[63 - e])
  uint32_t u0 = min(a0, __shfl_sync(0xffffffffu, b1, 31u - lane));
  uint32_t u1 = min(a1, __shfl_sync(0xffffffffu, b0, 31u - lane));
  r0 = min(u0, u1);
  r1 = max(u0, u1);
#pragma unroll
  for (uint32_t dist = 16u; dist >= 1u; dist >>= 1) {
    const uint32_t p0 = __shfl_xor_sync(0xffffffffu, r0, dist);
    const uint32_t p1 = __shfl_xor_sync(0xffffffffu, r1, dist);
    const bool upper = (lane & dist) != 0u;
    r0 = upper ? max(r0, p0) : min(r0, p0);
    r1 = upper ? max(r1, p1) : min(r1, p1);
  }
}

// Steps 2 and 3 of the Huffman cost with both queues linear: the leaves
// (the small counts expanded from the distinct list, then the large ones
// sorted), then the phases.  kSmem: K <= kHuffSmemKeys, both queues in shared
// memory (addressed as such: every phase is a chain of dependent loads),
// else in the workspace.  Returns this thread's share of the cost.
template <bool kSmem>
__device__ __forceinline__ unsigned long long huffman_linear(Workspace* ws, int which,
                                                             const uint32_t* dv_ws, uint32_t D,
                                                             const uint32_t* big, uint32_t nbig,
                                                             uint32_t nsmall, uint32_t K,
                                                             unsigned long long ns, uint32_t* s_w) {
  extern __shared__ uint32_t s_dyn[];
  const int tid = threadIdx.x;
  unsigned long long cost = 0ull;
  // with the queues in shared memory the distinct list (D <= K) is there too
  const uint32_t* dv = kSmem ? s_dyn + kHuffSmemKeys : dv_ws;
  uint32_t* leaves = kSmem ? s_dyn : ws->sort_scratch[which];
  // the nodes overwrite the distinct list, or the large counts once copied
  uint32_t* nodes = kSmem ? s_dyn + kHuffSmemKeys : ws->node_scratch[which];
  const uint32_t Cd = (D + kHuffThreads - 1) / kHuffThreads;
  const uint32_t e0 = min(D, (uint32_t)tid * Cd), e1 = min(D, e0 + Cd);
  uint32_t mloc = 0u;
  for (uint32_t d = e0; d < e1; d++) mloc += (dv[d] & 0xffffu) + 1u;
  uint32_t tot;
  uint32_t start = block_excl_sum(mloc, s_w, &tot);
  for (uint32_t o = tid; o < nsmall; o += kHuffThreads) leaves[o] = 0u;
  __syncthreads();
  for (uint32_t d = e0; d < e1; d++) {
    const uint32_t q = dv[d];
    leaves[start] = q >> 16;
    start += (q & 0xffffu) + 1u;
  }
  for (uint32_t i = tid; i < nbig; i += kHuffThreads) leaves[nsmall + i] = big[i];
  __syncthreads();
  {
    const uint32_t C = (nsmall + kHuffThreads - 1) / kHuffThreads;
    const uint32_t o0 = min(nsmall, (uint32_t)tid * C), o1 = min(nsmall, o0 + C);
    uint32_t run = 0u;
    for (uint32_t o = o0; o < o1; o++) run = max(run, leaves[o]);
    uint32_t carry = block_excl_max(run, s_w);
    for (uint32_t o = o0; o < o1; o++) {
      carry = max(carry, leaves[o]);
      leaves[o] = carry;
    }
  }
  __syncthreads();
  bitonic_sort(leaves + nsmall, (int)nbig);

  // 3. phases
  if (K == 1) {
    cost = (tid == 0) ? ns : 0ull;
  } else if (K > 1) {
    const uint32_t lane = (uint32_t)tid & 31u;
    // the phase reports carry their phase number: a report not written in
    // this phase is never read as one
    if (tid == 0) s_w[2] = s_w[6] = 0xffffffffu;
    __syncthreads();
    uint32_t lh = 0u, ih = 0u, it = 0u;  // leaf head, node head, node tail
    for (uint32_t ph = 0u;; ph++) {
      const uint32_t na = K - lh, nb = it - ih, L = na + nb;
      if (L <= 1u) break;
      const uint32_t* A = leaves + lh;
      const uint32_t* B = nodes + ih;
      // T: the two smallest items (every thread reads the queue heads)
      unsigned long long c4[4] = {~0ull, ~0ull, ~0ull, ~0ull};
      if (na > 0u) c4[0] = A[0];
      if (na > 1u) c4[1] = A[1];
      if (nb > 0u) c4[2] = B[0];
      if (nb > 1u) c4[3] = B[1];
      const unsigned long long m01 = min(c4[0], c4[1]), x01 = max(c4[0], c4[1]);
      const unsigned long long m23 = min(c4[2], c4[3]), x23 = max(c4[2], c4[3]);
      const unsigned long long T = min(m01, m23) + (m01 < m23 ? min(x01, m23) : min(x23, m01));
      // every item below T: this phase pairs them all, then the tail follows
      const uint32_t topa = na > 0u ? A[na - 1u] : 0u, topb = nb > 0u ? B[nb - 1u] : 0u;
      const bool all_below = (unsigned long long)max(topa, topb) < T;
      // windows of 32 pairs: warp w takes windows w, w + 32, ... while they
      // pair all 32; the window where pairing stops writes (np, cl)
      uint32_t* s_res = s_w + 4u * (ph & 1u);
      for (uint32_t win = (uint32_t)tid >> 5;; win += kHuffThreads / 32) {
        const uint32_t d = 64u * win;  // merged position of the window's first item
        if (d >= L) {
          // all L items paired (L even): the phase ends exactly here
          if (d == L && all_below && lane == 0u) {
            s_res[0] = L / 2u;
            s_res[1] = na;
            s_res[2] = ph;
          }
          break;
        }
        {
          // skip a window that provably holds no pair and does not end the
          // phase: at most d - 1 items lie below T when A[a] >= T and
          // B[b] >= T (or a queue is shorter) with a + b = d - 1
          if (d > 0u) {
            const uint32_t ia = (d - 1u) >> 1, ib = d - 1u - ia;
            const bool fa = ia >= na || (unsigned long long)A[ia] >= T;
            const bool fb = ib >= nb || (unsigned long long)B[ib] >= T;
            if (fa && fb) break;
          }
        }
        const uint32_t i0 = warp_merge_split(A, na, B, nb, d);
        const uint32_t k0 = d - i0;
        const uint32_t a0k = i0 + lane < na ? hkey_leaf(A[i0 + lane]) : ~0u;
        const uint32_t a1k = i0 + 32u + lane < na ? hkey_leaf(A[i0 + 32u + lane]) : ~0u;
        const uint32_t b0k = k0 + lane < nb ? hkey_node(B[k0 + lane]) : ~0u;
        const uint32_t b1k = k0 + 32u + lane < nb ? hkey_node(B[k0 + 32u + lane]) : ~0u;
        uint32_t r0, r1;
        window_merge64(a0k, a1k, b0k, b1k, r0, r1);
        // lane l's pair: merged items 2l and 2l + 1 of the window
        const uint32_t src = (2u * lane) & 31u;
        const uint32_t x0 = __shfl_sync(0xffffffffu, r0, src), x1 = __shfl_sync(0xffffffffu, r0, src + 1u);
        const uint32_t y0 = __shfl_sync(0xffffffffu, r1, src), y1 = __shfl_sync(0xffffffffu, r1, src + 1u);
        const uint32_t e0 = lane < 16u ? x0 : y0, e1 = lane < 16u ? x1 : y1;
        // a pair forms when its larger item is below T (a prefix of the lanes)
        const bool valid = d + 2u * lane + 1u < L && (unsigned long long)(e1 >> 1) < T;
        if (valid) {
          const uint32_t sum = (e0 >> 1) + (e1 >> 1);
          nodes[it + d / 2u + lane] = sum;
          cost += sum;
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (vm != 0xffffffffu) {
          const uint32_t v = (uint32_t)__popc(vm);
          // this window ends the phase when the item before it is below T
          bool prev_ok = true;
          if (d > 0u) {
            const uint32_t pa = i0 > 0u ? A[i0 - 1u] : 0u, pb = k0 > 0u ? B[k0 - 1u] : 0u;
            prev_ok = (unsigned long long)max(pa, pb) < T;
          }
          // leaves among the window's first 2v items
          const unsigned la = __ballot_sync(0xffffffffu, lane < v && (e0 & 1u) == 0u);
          const unsigned lb = __ballot_sync(0xffffffffu, lane < v && (e1 & 1u) == 0u);
          if (prev_ok && lane == 0u) {
            s_res[0] = d / 2u + v;
            s_res[1] = i0 + (uint32_t)__popc(la) + (uint32_t)__popc(lb);
            s_res[2] = ph;
          }
          break;
        }
      }
      __syncthreads();
      const uint32_t np = s_res[0], cl = s_res[1];
      // exactly one window reports, with at least one pair (the two smallest
      // items are below T); a missing or inconsistent report would stall the
      // loop, so it ends the call instead
      if (s_res[2] != ph || np == 0u || 2u * np > L || cl > na || 2u * np - cl > nb) {
        if (tid == 0) atomicCAS((int*)&ws->sc.status, RD_OK, RD_ERR_TIMEOUT);
        break;
      }
      lh += cl;
      ih += 2u * np - cl;
      it += np;
      if (all_below) {
        // what is left: a leaf (odd count), then the nodes from ih
        const bool fv = lh < K;
        const uint32_t f = fv ? leaves[lh] : 0u;
        auto at = [&](uint32_t p, uint32_t k) -> uint32_t& { return nodes[p + k]; };
        auto nxt = [](uint32_t p, uint32_t k) { return p + k; };
        cost += huffman_tail(at, nxt, fv, f, ih, it - ih, it);
        break;
      }
    }
  }
  return cost;
}

// ---------------------------------------------------------------------------
// Huffman cost and entropy sum (one CTA per histogram).
//  1. The bitmap of present count values gives each its rank d in ascending
//     order; the D distinct values and their multiplicities (packed as
//     v << 16 | (m - 1)) are gathered in that order.  N_s and the entropy
//     sum are the code prep's per-slice shares added in a fixed order.
//  2. The ascending leaf array: the first position of every distinct value
//     is marked with the value and a running maximum over positions fills
//     each run; the large counts follow, sorted by a bitonic network.
//  3. The phased two-queue merge (nodes are written only above the queue
//     tail, which no thread reads until the next barrier).  With both
//     queues linear, every warp takes windows of 64 consecutive items of
//     the merged order (the window's start by a 128-way search for the
//     split, then the 64 smallest of the next 64 leaves and 64 nodes sorted
//     by a bitonic network) and forms the window's pairs whose larger item
//     lies below the phase threshold; the window where pairing stops
//     reports the phase's numbers of pairs and of leaves consumed, so a
//     phase has one barrier.  In run-length form one warp finds the numbers
//     of leaves and nodes below the threshold first, then the threads pair
//     contiguous runs of the merged order.  Once every remaining item lies
//     below the threshold the phases need no search at all (huffman_tail).
// Up to kHuffSmemKeys symbols both queues are linear in shared memory.
// Larger alphabets keep the leaves as runs of equal weight and the nodes in
// a ring, in shared memory (huffman_runs), when the runs fit; otherwise the
// linear queues live in the workspace in global memory.
// ---------------------------------------------------------------------------
__device__ void huffman_cta(Workspace* ws, int which) {
  extern __shared__ uint32_t s_dyn[];
  __shared__ uint32_t s_w[32];
  __shared__ unsigned long long s_w64[32];
  __shared__ double s_wd[32];
  __shared__ int s_skip;
  // one reading of the status for the whole CTA (the other histogram's CTA,
  // or a kernel running beside this launch, may change it)
  if (threadIdx.x == 0) s_skip = (__ldcg(&ws->sc.status) != RD_OK || __ldcg(&ws->sc.constant)) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;
  const int tid = threadIdx.x;
  const uint32_t* cc = ws->count_of[which];

  // 1. distinct values in ascending order
  const uint2 pw = reinterpret_cast<const uint2*>(ws->present[which])[tid];
  const uint32_t nbig = ws->nbig[which];
  const double ent = tid < kEntropyCtas ? ws->ent_part[which][tid] : 0.0;
  const unsigned long long nsum = tid < kEntropyCtas ? ws->ns_part[which][tid] : 0ull;
  uint32_t D;
  const uint32_t dbase = block_excl_sum(__popc(pw.x) + __popc(pw.y), s_w, &D);
  uint32_t* dv = (D <= (uint32_t)kHuffSmemKeys) ? s_dyn + kHuffSmemKeys : ws->distinct[which];
  {
    uint32_t d = dbase;
    for (uint32_t w = pw.x; w; w &= w - 1u) dv[d++] = 64u * tid + (uint32_t)(__ffs(w) - 1);
    for (uint32_t w = pw.y; w; w &= w - 1u) dv[d++] = 64u * tid + 32u + (uint32_t)(__ffs(w) - 1);
  }
  __syncthreads();
  uint32_t msum = 0u;
  for (uint32_t d0 = tid; d0 < D; d0 += 4u * kHuffThreads) {
    uint32_t vv[4], mm[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t d = d0 + (uint32_t)u * kHuffThreads;
      vv[u] = d < D ? dv[d] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t d = d0 + (uint32_t)u * kHuffThreads;
      mm[u] = d < D ? cc[vv[u]] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t d = d0 + (uint32_t)u * kHuffThreads;
      if (d < D) {
        dv[d] = (vv[u] << 16) | (mm[u] - 1u);
        msum += mm[u];
      }
    }
  }
  const uint32_t* big = ws->node_scratch[which];
  // the number of small symbols, N_s and the entropy sum: one fixed-order
  // block reduction of the three
  uint32_t nsmall;
  unsigned long long ns;
  double plogp;
  {
    static_assert(kEntropyCtas % 32 == 0 && kEntropyCtas <= 32 * 32, "whole warps of slices");
    constexpr int kSliceWarps = kEntropyCtas / 32;
    const uint32_t a = warp_sum(msum);
    // the slices' shares are held by the first warps alone (float64 is
    // a narrow pipe: the other warps skip it)
    if (tid < kEntropyCtas) {
      const unsigned long long b = warp_sum(nsum);
      const double c = warp_sum(ent);
      if ((tid & 31) == 0) {
        s_w64[tid >> 5] = b;
        s_wd[tid >> 5] = c;
      }
    }
    if ((tid & 31) == 0) s_w[tid >> 5] = a;
    __syncthreads();
    nsmall = warp_sum(s_w[tid & 31]);
    ns = 0ull;
    plogp = 0.0;
#pragma unroll
    for (int i = 0; i < kSliceWarps; i++) {
      ns += s_w64[i];
      plogp += s_wd[i];
    }
    __syncthreads();
  }
  const uint32_t K = nsmall + nbig;

  unsigned long long cost = 0ull;
  const uint32_t R = D + nbig;
  const bool runs = K > (uint32_t)kHuffSmemKeys && 2u * R + 1u <= (uint32_t)kHuffSmemKeys &&
                    2u * R + 1u + (3u * K + 3u) / 4u + 1u <= 2u * (uint32_t)kHuffSmemKeys;
  if (runs) {
    cost = huffman_runs(dv, D, big, nbig, nsmall, K, s_w);
  } else if (K <= (uint32_t)kHuffSmemKeys) {
    cost = huffman_linear<true>(ws, which, dv, D, big, nbig, nsmall, K, ns, s_w);
  } else {
    cost = huffman_linear<false>(ws, which, dv, D, big, nbig, nsmall, K, ns, s_w);
  }
  cost = block_sum_u64(cost, s_w64);
  if (tid == 0) {
    ws->huff[which].ns = ns;
    ws->huff[which].cost = cost;
    ws->huff[which].nsym = K;
    ws->huff[which].plogp = plogp;
  }
}

__global__ void __launch_bounds__(kHuffThreads) k_huffman(Workspace* ws, int which0) {
  huffman_cta(ws, which0 + blockIdx.x);
}

cudaError_t launch_code_prep(Workspace* ws, int which_mask, const double* xlogx, cudaStream_t s) {
  const int nh = (which_mask == 3) ? 2 : 1;
  k_code_prep<<<nh * kEntropyCtas, kPrepThreads, 0, s>>>(ws, which_mask, xlogx);
  return cudaGetLastError();
}

cudaError_t launch_huffman(Workspace* ws, int which_mask, cudaStream_t s) {
  const int smem = 2 * kHuffSmemKeys * (int)sizeof(uint32_t);
  const int nh = (which_mask == 3) ? 2 : 1;
  k_huffman<<<nh, kHuffThreads, smem, s>>>(ws, (which_mask & 1) ? 0 : 1);
  return cudaGetLastError();
}

cudaError_t launch_code_stats(Workspace* ws, int which_mask, const double* xlogx, cudaStream_t s) {
  cudaError_t e = launch_code_prep(ws, which_mask, xlogx, s);
  if (e == cudaSuccess) e = launch_huffman(ws, which_mask, s);
  return e;
}

__global__ void __launch_bounds__(kHuffThreads) k_batch_final(const BatchField* __restrict__ bf,
                                                              rd_result* res, int32_t* status);

__global__ void __launch_bounds__(kHuffThreads) k_huffman_finish(Workspace* ws, int which0,
                                                                 FinishArgs fa);

cudaError_t prepare_code_stats() {
  const int smem = 2 * kHuffSmemKeys * (int)sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_huffman, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_huffman_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_final, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

// ---------------------------------------------------------------------------
// Finish: SZ rates, ground-truth rates, PSNRs and the selection
// (rd_finish.cuh).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFinishThreads) k_finish(ParamsDev p, Workspace* ws, int passes,
                                                           int zfp_parts, int sz_parts,
                                                           long long npoints_all,
                                                           unsigned long long zfp_npoints,
                                                           OutRecords* out) {
  finish_cta(p, ws, passes, zfp_parts, sz_parts, npoints_all, zfp_npoints);
  if (out) write_out(ws, out);
}

// One CTA per histogram; the CTA that ends last (a counter, fenced on both
// sides) runs the finish step.
__global__ void __launch_bounds__(kHuffThreads) k_huffman_finish(Workspace* ws, int which0,
                                                                 FinishArgs fa) {
  __shared__ int s_last;
  // a launch waiting on this one as its programmatic dependent (the truth's
  // ZFP pass of the evaluate step) may start now
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // with a join the truth's ZFP pass finishes the ZFP truth itself
  const int passes = fa.join ? (fa.passes & ~P_ZFP_GT) : fa.passes;
  // the finish step's first part needs no Huffman cost: the first CTA does
  // it before its own histogram
  if (blockIdx.x == 0 && (passes & (P_ZFP_GT | P_SZ_GT))) {  // nothing to do without a truth
    finish_pre(ws, passes, fa.zfp_parts, fa.sz_parts, fa.npoints_all);
    __syncthreads();
  }
  huffman_cta(ws, which0 + blockIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ws->sc.huff_done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  finish_post(fa.p, ws, passes, fa.npoints_all, fa.zfp_npoints);
  if (!fa.join && fa.out) write_out(ws, fa.out);  // with a join the ZFP pass writes
}

cudaError_t launch_huffman_finish(Workspace* ws, int which_mask, const FinishArgs& fa,
                                  cudaStream_t s) {
  const int smem = 2 * kHuffSmemKeys * (int)sizeof(uint32_t);
  const int nh = (which_mask == 3) ? 2 : 1;
  k_huffman_finish<<<nh, kHuffThreads, smem, s>>>(ws, (which_mask & 1) ? 0 : 1, fa);
  return cudaGetLastError();
}

cudaError_t launch_finish(const ParamsDev& p, Workspace* ws, int passes, int zfp_parts,
                          int sz_parts, long long npoints_all, unsigned long long zfp_npoints,
                          OutRecords* out, cudaStream_t s) {
  k_finish<<<1, kFinishThreads, 0, s>>>(p, ws, passes, zfp_parts, sz_parts, npoints_all, zfp_npoints,
                                        out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched estimate (rd_select_batch): the reset, the count-of-counts of every
// field, and the final pass (one CTA per field: Huffman cost and entropy,
// then the rates, PSNRs and selection; the field's record and status are
// gathered).
// ---------------------------------------------------------------------------
// The estimate's tables (hist[0], count_of[0], present[0]) are cleared only
// when the call before left them dirty: the batched passes that read them
// clear what they read (code prep: the histogram; the final pass: the
// count-of-counts and the bitmap), and the final pass marks them clean.
__global__ void k_batch_reset(const BatchField* __restrict__ bf, int need_gt) {
  const BatchField& F = bf[blockIdx.x];
  const int est = F.ws->sc.clean == kCleanTables ? 0 : 1;
  reset_ws(F.ws, threadIdx.x, blockDim.x, est | (need_gt ? 2 : 0));
}

cudaError_t launch_batch_reset(const BatchField* bf, int n, int need_gt, cudaStream_t s) {
  // one CTA per field: with clean tables only the scalars and the exponent
  // bins are left to clear
  k_batch_reset<<<n, 1024, 0, s>>>(bf, need_gt);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kPrepThreads) k_batch_code_prep(const BatchField* __restrict__ bf,
                                                                  const double* __restrict__ xlogx) {
  code_prep_slice<true>(bf[blockIdx.x / kEntropyCtas].ws, 0, blockIdx.x % kEntropyCtas, xlogx);
}

cudaError_t launch_batch_code_prep(const BatchField* bf, int n, const double* xlogx, cudaStream_t s) {
  k_batch_code_prep<<<n * kEntropyCtas, kPrepThreads, 0, s>>>(bf, xlogx);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kHuffThreads) k_batch_final(const BatchField* __restrict__ bf,
                                                              rd_result* res, int32_t* status) {
  const BatchField& F = bf[blockIdx.x];
  Workspace* ws = F.ws;
  huffman_cta(ws, 0);
  __syncthreads();
  finish_cta(F.p, ws, P_ZFP_EST | P_SZ_EST, 0, 0, F.f.N, F.npoints);
  __syncthreads();
  // gather the record (word-wise) and the status
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&ws->res);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&res[blockIdx.x]);
  for (int i = threadIdx.x; i < (int)(sizeof(rd_result) / 4); i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) status[blockIdx.x] = ws->sc.status;
  // leave the tables zero for the next call: the count-of-counts entries of
  // the present values, the bitmap and the escape bin (code prep cleared the
  // other bins); a field that stopped early is left for the reset to clear
  const bool used = ws->sc.status == RD_OK && !ws->sc.constant;  // uniform over the CTA
  __syncthreads();
  if (used) {
    uint32_t* cc = ws->count_of[0];
    uint32_t* pr = ws->present[0];
    for (int i = threadIdx.x; i < kNsym / 32; i += blockDim.x) {
      const uint32_t word = pr[i];
      if (!word) continue;
      for (uint32_t b = word; b; b &= b - 1u) cc[32 * i + __ffs(b) - 1] = 0u;
      pr[i] = 0u;
    }
    if (threadIdx.x == 0) ws->hist[0][0] = 0u;
    __syncthreads();
  }
  if (threadIdx.x == 0) ws->sc.clean = used ? kCleanTables : 0u;
}

cudaError_t launch_batch_final(const BatchField* bf, int n, rd_result* res, int32_t* status,
                               cudaStream_t s) {
  const int smem = 2 * kHuffSmemKeys * (int)sizeof(uint32_t);
  k_batch_final<<<n, kHuffThreads, smem, s>>>(bf, res, status);
  return cudaGetLastError();
}

__global__ void k_batch_truth(const BatchField* __restrict__ bf, rd_truth* truth, int32_t* status) {
  const Workspace* ws = bf[blockIdx.x].ws;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&ws->truth);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&truth[blockIdx.x]);
  for (int i = threadIdx.x; i < (int)(sizeof(rd_truth) / 4); i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) status[blockIdx.x] = ws->sc.status;
}

cudaError_t launch_batch_truth(const BatchField* bf, int n, rd_truth* truth, int32_t* status,
                               cudaStream_t s) {
  k_batch_truth<<<n, 64, 0, s>>>(bf, truth, status);
  return cudaGetLastError();
}

}  // namespace rdk
