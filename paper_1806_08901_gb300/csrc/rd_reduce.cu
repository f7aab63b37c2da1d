// rd_reduce.cu -- the small kernels of one rate-distortion call: workspace
// reset, value range (Algorithm 1 line 2), the bin width delta from the exact
// MSE_sp (line 7), the entropy and Huffman cost of the code histograms
// (lines 8-9 and the SZ ground truth) and the final selection (lines 10-12).
#include <math.h>
#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

// ---------------------------------------------------------------------------
// Reset: zero accumulators and histograms of the workspace.
// ---------------------------------------------------------------------------
__global__ void k_reset(Workspace* ws) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  uint32_t* h = &ws->hist[0][0];
  for (int i = tid; i < 2 * kNsym; i += nth) h[i] = 0u;
  uint32_t* cc = &ws->count_of[0][0];
  for (int i = tid; i < 2 * kNsym; i += nth) cc[i] = 0u;
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
    s.vmin = s.vmax = s.amax = 0.0f;
    s.w = s.inv = s.tau = 0.0f;
    s.vr = s.eb_abs = s.delta = s.mse_sp = 0.0;
    s.s2 = 0ull;
    s.zfp_bits = 0ull;
    s.zfp_maxerr = 0u;
    s.sz_maxerr = 0u;
    for (int w = 0; w < 2; w++) {
      ws->nbig[w] = 0u;
      ws->huff[w].ns = 0ull;
      ws->huff[w].cost = 0ull;
      ws->huff[w].nsym = 0u;
    }
    unsigned char* r = reinterpret_cast<unsigned char*>(&ws->res);
    for (size_t i = 0; i < sizeof(rd_result); i++) r[i] = 0;
    unsigned char* t = reinterpret_cast<unsigned char*>(&ws->truth);
    for (size_t i = 0; i < sizeof(rd_truth); i++) t[i] = 0;
  }
}

cudaError_t launch_reset(Workspace* ws, cudaStream_t s) {
  k_reset<<<128, 256, 0, s>>>(ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Value range: min / max over every value, with a non-finite test.  Rows are
// read as float4 where the pointer allows it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_range(const float* __restrict__ x, long long n,
                                               Workspace* ws) {
  unsigned kmin = 0xffffffffu, kmax = 0u, bad = 0u;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  // scalar head up to a 16-byte boundary
  long long head = (long long)((16u - ((uintptr_t)x & 15u)) & 15u) / 4;
  if (head > n) head = n;
  if (((uintptr_t)x & 3u) != 0) head = n;  // not even 4-byte aligned: all scalar
  for (long long i = tid; i < head; i += nth) {
    float v = x[i];
    unsigned b = __float_as_uint(v);
    bad |= ((b & 0x7f800000u) == 0x7f800000u);
    unsigned k = float_key(v);
    kmin = min(kmin, k);
    kmax = max(kmax, k);
  }
  const long long nvec = (n - head) / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x + head);
  for (long long i = tid; i < nvec; i += nth) {
    float4 q = __ldg(x4 + i);
    float v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      unsigned b = __float_as_uint(v[j]);
      bad |= ((b & 0x7f800000u) == 0x7f800000u);
      unsigned k = float_key(v[j]);
      kmin = min(kmin, k);
      kmax = max(kmax, k);
    }
  }
  for (long long i = head + nvec * 4 + tid; i < n; i += nth) {
    float v = x[i];
    unsigned b = __float_as_uint(v);
    bad |= ((b & 0x7f800000u) == 0x7f800000u);
    unsigned k = float_key(v);
    kmin = min(kmin, k);
    kmax = max(kmax, k);
  }
  // warp, then CTA, then one update per CTA of the shared keys
  __shared__ unsigned s_min[16], s_max[16], s_bad[16];
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  bad = __reduce_or_sync(0xffffffffu, bad);
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_min[wid] = kmin;
    s_max[wid] = kmax;
    s_bad[wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    unsigned a = threadIdx.x < nw ? s_min[threadIdx.x] : 0xffffffffu;
    unsigned b = threadIdx.x < nw ? s_max[threadIdx.x] : 0u;
    unsigned c = threadIdx.x < nw ? s_bad[threadIdx.x] : 0u;
    a = __reduce_min_sync(0xffffffffu, a);
    b = __reduce_max_sync(0xffffffffu, b);
    c = __reduce_or_sync(0xffffffffu, c);
    if (threadIdx.x == 0) {
      atomicMin(&ws->sc.min_key, a);
      atomicMax(&ws->sc.max_key, b);
      if (c) atomicOr(&ws->sc.nonfinite, 1u);
    }
  }
}

cudaError_t launch_range(const FieldDev& f, Workspace* ws, int ctas, cudaStream_t s) {
  long long want = (f.N / 4 + 511) / 512;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  k_range<<<g, 512, 0, s>>>(f.x, f.N, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prepare: value range VR, eb_abs (Eq. psnr-sz: eb_rel = eb_abs / VR) and
// floor(log2 eb_abs) for the ZFP precision rule.
// ---------------------------------------------------------------------------
__global__ void k_prepare(ParamsDev p, Workspace* ws) {
  Scalars& s = ws->sc;
  if (s.nonfinite) {
    s.status = RD_ERR_NONFINITE;
    return;
  }
  s.vmin = key_float(s.min_key);
  s.vmax = key_float(s.max_key);
  s.amax = fmaxf(fabsf(s.vmin), fabsf(s.vmax));
  s.vr = (double)s.vmax - (double)s.vmin;
  s.eb_abs = (p.eb_mode == RD_EB_REL) ? p.eb * s.vr : p.eb;
  ws->res.vmin = s.vmin;
  ws->res.vmax = s.vmax;
  ws->res.vr = s.vr;
  ws->res.eb_abs = s.eb_abs;
  if (s.vr == 0.0) {
    s.constant = 1;
    s.flags |= RD_F_CONSTANT;
    return;
  }
  if (!(s.eb_abs > 0.0) || !isfinite(s.eb_abs)) {
    s.status = RD_ERR_INVALID_ARG;
    return;
  }
  int e;
  frexp(s.eb_abs, &e);
  s.minexp = e - 1;
  ws->res.minexp = s.minexp;
}

cudaError_t launch_prepare(const ParamsDev& p, Workspace* ws, cudaStream_t s) {
  k_prepare<<<1, 1, 0, s>>>(p, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bin width.  MSE_sp is the exact sum of (2^d d)^2 4^(emax-30) over the
// EC-sampled coefficients, held as 64-bit limbs with the least significant
// bit at 2^-312 and rounded once to nearest-even; delta = sqrt(12 MSE_sp)
// (PSNR_sz = PSNR_zfp in Eq. psnr-pdf-linear), clamped to 2 eb_abs.
// ---------------------------------------------------------------------------
constexpr int kLimbs = 12;  // 768 bits

__device__ void limbs_add(unsigned long long* a, unsigned long long v, int off) {
  int w = off >> 6, sh = off & 63;
  unsigned long long lo = v << sh;
  unsigned long long hi = sh ? (v >> (64 - sh)) : 0ull;
  unsigned long long carry = 0ull;
  for (int i = w; i < kLimbs; i++) {
    unsigned long long add = (i == w) ? lo : (i == w + 1) ? hi : 0ull;
    unsigned long long t = a[i] + add;
    unsigned long long c1 = t < add;
    unsigned long long t2 = t + carry;
    unsigned long long c2 = t2 < carry;
    a[i] = t2;
    carry = c1 + c2;
    if (i > w + 1 && carry == 0ull) break;
  }
}

// Round the limb integer times 2^-312 to the nearest double (ties to even):
// the 53 bits below the leading one, a round bit and a sticky bit.
__device__ double limbs_to_double(const unsigned long long* a) {
  int ti = kLimbs - 1;
  while (ti >= 0 && a[ti] == 0ull) ti--;
  if (ti < 0) return 0.0;
  const int top = ti * 64 + 63 - __clzll((long long)a[ti]);
  if (top <= 52) return ldexp((double)a[0], -312);  // exact
  const int shift = top - 52;
  const int w = shift >> 6, o = shift & 63;
  unsigned long long m = a[w] >> o;
  if (o && w + 1 < kLimbs) m |= a[w + 1] << (64 - o);
  m &= (1ull << 53) - 1ull;
  const int rb = shift - 1;
  const int round = (int)((a[rb >> 6] >> (rb & 63)) & 1ull);
  bool sticky = (a[rb >> 6] & ((1ull << (rb & 63)) - 1ull)) != 0ull;
  for (int i = 0; i < (rb >> 6) && !sticky; i++) sticky = a[i] != 0ull;
  if (round && (sticky || (m & 1ull))) m += 1ull;
  return ldexp((double)m, shift - 312);
}

// Launched with one warp: the lanes sum disjoint exponent bins into their own
// limb integers, a butterfly adds the 32 integers (exact, so the order does
// not matter), and lane 0 finishes.
__global__ void k_delta(ParamsDev p, Workspace* ws, int mode, double arg, int need_quant,
                        int need_gt, unsigned long long ncoeff, unsigned long long npoints) {
  Scalars& s = ws->sc;
  if (s.status != RD_OK || s.constant) return;
  rd_result& r = ws->res;
  const int lane = threadIdx.x;
  unsigned long long acc[kLimbs];
  if (mode == DELTA_FROM_MSE) {
#pragma unroll
    for (int i = 0; i < kLimbs; i++) acc[i] = 0ull;
    for (int i = lane; i < kMseBins; i += 32) {
      const unsigned long long lo = s.mse_lo[i], hi = s.mse_hi[i];
      if (lo) limbs_add(acc, lo, 2 * i);
      if (hi) limbs_add(acc, hi, 2 * i + 64);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long carry = 0ull;
#pragma unroll
      for (int j = 0; j < kLimbs; j++) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, acc[j], o);
        const unsigned long long u = acc[j] + t;
        const unsigned long long c1 = u < t;
        const unsigned long long v = u + carry;
        const unsigned long long c2 = v < carry;
        acc[j] = v;
        carry = c1 + c2;
      }
    }
  }
  if (lane != 0) return;
  double delta;
  if (mode == DELTA_FROM_MSE) {
    double num = limbs_to_double(acc);
    s.mse_sp = num / (double)ncoeff;
    r.mse_sp = s.mse_sp;
    r.zfp_s2 = s.s2;
    r.br_zfp = (double)s.s2 / (2.0 * (double)npoints);
    r.psnr_zfp = s.mse_sp > 0.0 ? 20.0 * log10(s.vr) - 10.0 * log10(s.mse_sp) : INFINITY;
    if (s.mse_sp == 0.0) {
      delta = 2.0 * s.eb_abs;
      s.flags |= RD_F_MSE_ZERO;
    } else {
      delta = sqrt(12.0 * s.mse_sp);
      if (delta > 2.0 * s.eb_abs) {
        delta = 2.0 * s.eb_abs;
        s.flags |= RD_F_DELTA_CLAMPED;
      }
    }
  } else if (mode == DELTA_EXPLICIT) {
    delta = arg > 0.0 ? arg : 2.0 * s.eb_abs;
  } else {
    delta = 2.0 * arg;
  }
  s.delta = delta;
  r.delta = delta;
  r.psnr_sz = 20.0 * log10(s.vr / delta) + 10.0 * log10(12.0);
  if (!need_quant) return;
  // float quantiser: w = float(delta), 1/w, and tau = the largest float not
  // above (delta / 2)(1 - 2^-23), so that a float |x - xhat| <= tau proves
  // |x - xhat| <= delta / 2
  float w = (float)delta;
  if (!(w >= 1.17549435e-38f) || isinf(w)) {
    s.status = RD_ERR_RANGE;
    return;
  }
  float inv = __fdiv_rn(1.0f, w);
  if (isinf(inv) || !(inv >= 1.17549435e-38f)) {
    s.status = RD_ERR_RANGE;
    return;
  }
  double t = (delta / 2.0) * (1.0 - 1.1920928955078125e-07);
  float tau = __double2float_rz(t);
  s.w = w;
  s.inv = inv;
  s.tau = tau;
  if (need_gt) {
    if (__fmul_rn(s.amax, inv) > 134217728.0f) s.status = RD_ERR_RANGE;
  }
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

// number of A elements among the first d of merge(A, B), ties from A first
__device__ __forceinline__ uint32_t merge_split(const uint32_t* A, uint32_t na, const uint32_t* B,
                                                uint32_t nb, uint32_t d) {
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  return lo;
}


constexpr int kPrepThreads = 256;   // code-statistics prep CTAs (1024 bins each)
constexpr int kHuffThreads = 1024;  // Huffman CTA

// Number of elements of the sorted a[0..n) below T, found by one warp: each
// round tests 32 evenly spaced elements and keeps the gap holding the answer.
__device__ uint32_t warp_count_below(const uint32_t* a, uint32_t n, unsigned long long T) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 32u) {
    const uint32_t step = (hi - lo + 31u) / 32u;
    const uint32_t idx = lo + (uint32_t)lane * step;
    const bool p = idx < hi && (unsigned long long)a[idx] < T;
    const int c = __popc(__ballot_sync(0xffffffffu, p));
    if (c == 0) return lo;
    const uint32_t nl = lo + (uint32_t)(c - 1) * step + 1u;
    const uint32_t nh = lo + (uint32_t)c * step;
    lo = nl;
    hi = nh < hi ? nh : hi;
  }
  const uint32_t idx = lo + (uint32_t)lane;
  const bool p = idx < hi && (unsigned long long)a[idx] < T;
  return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, p));
}

// Number of A elements among the first d of merge(A, B) (ties: A first),
// found by one warp: the predicate A[i] <= B[d-1-i] holds for a prefix of i.
__device__ uint32_t warp_merge_split(const uint32_t* A, uint32_t na, const uint32_t* B,
                                     uint32_t nb, uint32_t d) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;  // answer in [lo, hi]
  while (hi - lo > 32u) {
    const uint32_t step = (hi - lo + 31u) / 32u;
    const uint32_t i = lo + (uint32_t)lane * step;
    const bool p = i < hi && A[i] <= B[d - 1 - i];
    const int c = __popc(__ballot_sync(0xffffffffu, p));
    if (c == 0) return lo;
    const uint32_t nl = lo + (uint32_t)(c - 1) * step + 1u;
    const uint32_t nh = lo + (uint32_t)c * step;
    lo = nl;
    hi = nh < hi ? nh : hi;
  }
  const uint32_t i = lo + (uint32_t)lane;
  const bool p = i < hi && A[i] <= B[d - 1 - i];
  return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, p));
}

// ---------------------------------------------------------------------------
// Prep (many CTAs, 1024 bins each): the slice's sum of h log2 h for the
// entropy; the multiplicity of every count value below 2^16 (a counting sort
// of the counts, lanes with equal counts merged into one atomic); counts of
// 2^16 or more (at most N / 2^16 of them) appended to a list.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPrepThreads) k_code_prep(Workspace* ws, int which_mask) {
  __shared__ double part[kPrepThreads / 32];
  if (ws->sc.status != RD_OK || ws->sc.constant) return;
  const int first = (which_mask & 1) ? 0 : 1;
  const int which = first + blockIdx.x / kEntropyCtas;
  const int slice = blockIdx.x % kEntropyCtas;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint32_t* cc = ws->count_of[which];
  uint32_t* big = ws->node_scratch[which];
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 1024 / kPrepThreads; k++) {
    const uint32_t c = ws->hist[which][slice * 1024 + k * kPrepThreads + threadIdx.x];
    if (c) v += (double)c * log2((double)c);
    const bool small = c != 0u && c < (uint32_t)kNsym;
    const bool large = c >= (uint32_t)kNsym;
    const unsigned ms = __ballot_sync(0xffffffffu, small);
    const unsigned mb = __ballot_sync(0xffffffffu, large);
    if (small) {
      const unsigned same = __match_any_sync(ms, c);
      if (lane == __ffs(same) - 1) atomicAdd(&cc[c], (uint32_t)__popc(same));
    }
    if (mb) {
      uint32_t base = 0u;
      if (lane == __ffs(mb) - 1) base = atomicAdd(&ws->nbig[which], (uint32_t)__popc(mb));
      base = __shfl_sync(0xffffffffu, base, __ffs(mb) - 1);
      if (large) big[base + __popc(mb & lt_mask)] = c;
    }
  }
  v = warp_sum(v);
  if (lane == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double t = warp_sum(threadIdx.x < kPrepThreads / 32 ? part[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) ws->ent_part[which][slice] = t;
  }
}

// ---------------------------------------------------------------------------
// Huffman cost (one CTA per histogram).  The ascending leaf array is the
// counting-sorted small counts followed by the sorted large ones.  Then the
// two-queue method in phases: with a0 <= a1 the two smallest remaining
// items, every item below T = a0 + a1 is consumed before any new node (new
// nodes are >= T), so all of them are paired at once in merged order (ties:
// leaves first); the new nodes, non-decreasing as in the sequential method,
// are appended to the internal queue.  Cost = sum of internal-node weights.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kHuffThreads) k_huffman(Workspace* ws, int which0) {
  extern __shared__ uint32_t s_dyn[];
  __shared__ uint32_t s_pre[kHuffThreads];   // per-thread small-count totals, scanned
  __shared__ unsigned long long s_red[kHuffThreads / 32];
  __shared__ uint32_t s_wmax[32];
  __shared__ uint32_t s_state[8];
  if (ws->sc.status != RD_OK || ws->sc.constant) return;
  const int which = which0 + blockIdx.x;
  const int tid = threadIdx.x;
  const uint32_t* cc = ws->count_of[which];
  constexpr int vper = kNsym / kHuffThreads;  // 64 count values per thread

  // multiplicities of this thread's values and their contribution to N_s
  uint32_t tot = 0u;
  unsigned long long nsum = 0ull;
  {
    const uint4* c4 = reinterpret_cast<const uint4*>(cc + tid * vper);
#pragma unroll
    for (int k = 0; k < vper / 4; k++) {
      const uint4 q = c4[k];
      const uint32_t v0 = (uint32_t)(tid * vper + 4 * k);
      tot += q.x + q.y + q.z + q.w;
      nsum += (unsigned long long)q.x * v0 + (unsigned long long)q.y * (v0 + 1) +
              (unsigned long long)q.z * (v0 + 2) + (unsigned long long)q.w * (v0 + 3);
    }
  }
  const uint32_t nbig = ws->nbig[which];
  const uint32_t* big = ws->node_scratch[which];
  for (uint32_t i = tid; i < nbig; i += kHuffThreads) nsum += big[i];
  s_pre[tid] = tot;
  nsum = warp_sum(nsum);
  if ((tid & 31) == 0) s_red[tid >> 5] = nsum;
  __syncthreads();
  for (int off = 1; off < kHuffThreads; off <<= 1) {
    const uint32_t t = tid >= off ? s_pre[tid - off] : 0u;
    __syncthreads();
    s_pre[tid] += t;
    __syncthreads();
  }
  const uint32_t nsmall = s_pre[kHuffThreads - 1];
  const uint32_t K = nsmall + nbig;
  unsigned long long ns = 0ull;
  if (tid < 32) ns = warp_sum(s_red[tid]);

  uint32_t* leaves;
  uint32_t* nodes;
  if (K <= (uint32_t)kHuffSmemKeys) {
    leaves = s_dyn;
    nodes = s_dyn + kHuffSmemKeys;
  } else {
    leaves = ws->sort_scratch[which];
    nodes = ws->node_scratch[which];  // free once the large counts are copied
  }
  // expansion of the small counts in ascending order: the first position of
  // every present value is marked with the value, then a running maximum
  // over positions fills each run (values ascend with position, 0 is absent)
  for (uint32_t o = tid; o < nsmall; o += kHuffThreads) leaves[o] = 0u;
  __syncthreads();
  {
    uint32_t o = s_pre[tid] - tot;
    const uint4* c4 = reinterpret_cast<const uint4*>(cc + tid * vper);
#pragma unroll 4
    for (int k = 0; k < vper / 4; k++) {
      const uint4 q = c4[k];
      const uint32_t v0 = (uint32_t)(tid * vper + 4 * k);
      if (q.x) { leaves[o] = v0; o += q.x; }
      if (q.y) { leaves[o] = v0 + 1; o += q.y; }
      if (q.z) { leaves[o] = v0 + 2; o += q.z; }
      if (q.w) { leaves[o] = v0 + 3; o += q.w; }
    }
  }
  // the large counts follow (in the global layout they move from the node
  // scratch to the leaf array)
  for (uint32_t i = tid; i < nbig; i += kHuffThreads) leaves[nsmall + i] = big[i];
  __syncthreads();
  {
    const uint32_t C = (nsmall + kHuffThreads - 1) / kHuffThreads;
    const uint32_t o0 = min(nsmall, (uint32_t)tid * C), o1 = min(nsmall, o0 + C);
    uint32_t run = 0u;
    for (uint32_t o = o0; o < o1; o++) run = max(run, leaves[o]);
    // exclusive running maximum over the threads' chunks
    const int lane = tid & 31;
    uint32_t inc = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc = max(inc, t);
    }
    if (lane == 31) s_wmax[tid >> 5] = inc;
    __syncthreads();
    if (tid < 32) {
      uint32_t w = s_wmax[tid];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, w, off);
        if (tid >= off) w = max(w, t);
      }
      s_wmax[tid] = w;
    }
    __syncthreads();
    uint32_t carry = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) carry = 0u;
    if (tid >= 32) carry = max(carry, s_wmax[(tid >> 5) - 1]);
    for (uint32_t o = o0; o < o1; o++) {
      carry = max(carry, leaves[o]);
      leaves[o] = carry;
    }
  }
  __syncthreads();
  bitonic_sort(leaves + nsmall, (int)nbig);

  unsigned long long cost = 0ull;
  if (K == 1) {
    cost = (tid == 0) ? ns : 0ull;
  } else if (K > 1) {
    // s_state: 0 lh, 1 ih, 2 it, 3 ml, 4 mi, 5 cl, 6 np, 7 done
    if (tid == 0) {
      s_state[0] = s_state[1] = s_state[2] = 0u;
      s_state[7] = 0u;
    }
    __syncthreads();
    for (;;) {
      if (tid < 32) {
        const uint32_t lh = s_state[0], ih = s_state[1], it = s_state[2];
        if ((K - lh) + (it - ih) <= 1u) {
          if (tid == 0) s_state[7] = 1u;
        } else {
          unsigned long long c4[4] = {~0ull, ~0ull, ~0ull, ~0ull};
          if (lh < K) c4[0] = leaves[lh];
          if (lh + 1 < K) c4[1] = leaves[lh + 1];
          if (ih < it) c4[2] = nodes[ih];
          if (ih + 1 < it) c4[3] = nodes[ih + 1];
          const unsigned long long m01 = min(c4[0], c4[1]), x01 = max(c4[0], c4[1]);
          const unsigned long long m23 = min(c4[2], c4[3]), x23 = max(c4[2], c4[3]);
          const unsigned long long a0 = min(m01, m23);
          const unsigned long long a1 = m01 < m23 ? min(x01, m23) : min(x23, m01);
          const unsigned long long T = a0 + a1;
          const uint32_t ml = warp_count_below(leaves + lh, K - lh, T);
          const uint32_t mi = warp_count_below(nodes + ih, it - ih, T);
          const uint32_t np = (ml + mi) >> 1;
          const uint32_t cl = warp_merge_split(leaves + lh, ml, nodes + ih, mi, 2u * np);
          if (tid == 0) {
            s_state[3] = ml;
            s_state[4] = mi;
            s_state[5] = cl;
            s_state[6] = np;
          }
        }
      }
      __syncthreads();
      if (s_state[7]) break;
      const uint32_t lh = s_state[0], ih = s_state[1], it = s_state[2];
      const uint32_t ml = s_state[3], mi = s_state[4], np = s_state[6];
      const uint32_t* A = leaves + lh;
      const uint32_t* B = nodes + ih;
      // each thread pairs a contiguous run of the merged order
      const uint32_t per_t = (np + kHuffThreads - 1) / kHuffThreads;
      const uint32_t j0 = (uint32_t)tid * per_t;
      const uint32_t j1 = min(np, j0 + per_t);
      if (j0 < j1) {
        uint32_t i = merge_split(A, ml, B, mi, 2u * j0);
        uint32_t k = 2u * j0 - i;
        for (uint32_t j = j0; j < j1; j++) {
          uint32_t e0, e1;
          if (i < ml && (k >= mi || A[i] <= B[k])) e0 = A[i++]; else e0 = B[k++];
          if (i < ml && (k >= mi || A[i] <= B[k])) e1 = A[i++]; else e1 = B[k++];
          const uint32_t s = e0 + e1;
          nodes[it + j] = s;
          cost += s;
        }
      }
      __syncthreads();
      if (tid == 0) {
        s_state[0] = lh + s_state[5];
        s_state[1] = ih + (2u * np - s_state[5]);
        s_state[2] = it + np;
      }
    }
  }
  __syncthreads();
  cost = warp_sum(cost);
  if ((tid & 31) == 0) s_red[tid >> 5] = cost;
  __syncthreads();
  if (tid < 32) {
    const unsigned long long c = warp_sum(s_red[tid]);
    if (tid == 0) {
      ws->huff[which].ns = ns;
      ws->huff[which].cost = c;
      ws->huff[which].nsym = K;
    }
  }
}

cudaError_t launch_code_prep(Workspace* ws, int which_mask, cudaStream_t s) {
  const int nh = (which_mask == 3) ? 2 : 1;
  k_code_prep<<<nh * kEntropyCtas, kPrepThreads, 0, s>>>(ws, which_mask);
  return cudaGetLastError();
}

cudaError_t launch_huffman(Workspace* ws, int which_mask, cudaStream_t s) {
  const int smem = 2 * kHuffSmemKeys * (int)sizeof(uint32_t);
  const int nh = (which_mask == 3) ? 2 : 1;
  k_huffman<<<nh, kHuffThreads, smem, s>>>(ws, (which_mask & 1) ? 0 : 1);
  return cudaGetLastError();
}

cudaError_t launch_code_stats(Workspace* ws, int which_mask, cudaStream_t s) {
  cudaError_t e = launch_code_prep(ws, which_mask, s);
  if (e == cudaSuccess) e = launch_huffman(ws, which_mask, s);
  return e;
}

cudaError_t prepare_code_stats() {
  const int smem = 2 * kHuffSmemKeys * (int)sizeof(uint32_t);
  return cudaFuncSetAttribute(k_huffman, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// ---------------------------------------------------------------------------
// Finish: SZ rates, ground-truth rates, PSNRs and the selection.
// ---------------------------------------------------------------------------
constexpr int kFinishThreads = 256;

// Fixed-order block sum (strided per-thread sums, then a fixed tree); the
// result is valid in thread 0.
__device__ double block_sum_parts(const double* a, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += a[i];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kFinishThreads) k_finish(ParamsDev p, Workspace* ws, int passes,
                                                           int zfp_parts, int sz_parts,
                                                           long long npoints_all,
                                                           unsigned long long zfp_npoints) {
  __shared__ double red[kFinishThreads / 32];
  Scalars& s = ws->sc;
  if (s.status != RD_OK) return;
  rd_result& r = ws->res;
  rd_truth& t = ws->truth;
  double zsse = 0.0, ssse = 0.0, plogp = 0.0;
  if (!s.constant) {
    if (passes & P_ZFP_GT) zsse = block_sum_parts(ws->zfp_sse, zfp_parts, red);
    if (passes & P_SZ_GT) ssse = block_sum_parts(ws->sz_sse, sz_parts, red);
    if (passes & P_SZ_EST) plogp = block_sum_parts(ws->ent_part[0], kEntropyCtas, red);
  }
  if (threadIdx.x != 0) return;
  if (s.constant) {
    r.flags = s.flags;
    r.psnr_zfp = INFINITY;
    r.psnr_sz = INFINITY;
    r.selection = 1;
    t.flags = s.flags;
    t.psnr_sz_gt = INFINITY;
    t.psnr_zfp_gt = INFINITY;
    t.best_gt = 1;
    return;
  }
  double lvr = 20.0 * log10(s.vr);
  if (passes & P_SZ_EST) {
    const HuffOut& hh = ws->huff[0];
    double ns = (double)hh.ns;
    double H = log2(ns) - plogp / ns;
    if (H < 0.0) H = 0.0;
    uint32_t h0 = ws->hist[0][0];
    r.entropy = H;
    r.br_sz = H + p.sz_offset;
    r.sz_ns = hh.ns;
    r.sz_huff_bits = hh.cost;
    r.sz_nsym = hh.nsym;
    r.sz_nesc = h0;
    r.br_sz_huff = (double)(hh.cost + 32ull * h0) / ns;
    if (passes & P_ZFP_EST) {
      if (p.sel_rule == RD_SEL_PAPER) {
        double diff = r.br_sz - r.br_zfp;
        if (fabs(diff) <= 1e-9) {
          s.flags |= RD_F_TIE_BAND;
          r.selection = 1;
        } else {
          r.selection = diff < 0.0 ? 0 : 1;
        }
      } else {
        // 2 (Huff + 32 h0) N_z < S2 N_s, in 128-bit integers
        unsigned long long a = 2ull * (hh.cost + 32ull * h0);
        unsigned long long alo = a * zfp_npoints, ahi = __umul64hi(a, zfp_npoints);
        unsigned long long blo = s.s2 * hh.ns, bhi = __umul64hi(s.s2, hh.ns);
        bool lt = ahi < bhi || (ahi == bhi && alo < blo);
        r.selection = lt ? 0 : 1;
      }
    }
  }
  r.flags = s.flags;
  if (passes & P_ZFP_GT) {
    t.zfp_bits_gt = s.zfp_bits;
    t.br_zfp_gt = (double)s.zfp_bits / (double)npoints_all;
    t.sse_zfp = zsse;
    t.maxerr_zfp = (double)__uint_as_float(s.zfp_maxerr);
    double mse = zsse / (double)npoints_all;
    t.psnr_zfp_gt = mse > 0.0 ? lvr - 10.0 * log10(mse) : INFINITY;
  }
  if (passes & P_SZ_GT) {
    const HuffOut& hg = ws->huff[1];
    uint32_t h0 = ws->hist[1][0];
    t.delta = s.delta;
    t.eb_sz = s.delta / 2.0;
    t.sz_huff_gt = hg.cost;
    t.sz_nsym_gt = hg.nsym;
    t.sz_nesc_gt = h0;
    t.sz_bits_gt = hg.cost + 32ull * h0 + 22ull * hg.nsym + 64ull;
    t.br_sz_gt = (double)t.sz_bits_gt / (double)npoints_all;
    t.sse_sz = ssse;
    t.maxerr_sz = (double)__uint_as_float(s.sz_maxerr);
    double mse = ssse / (double)npoints_all;
    t.psnr_sz_gt = mse > 0.0 ? lvr - 10.0 * log10(mse) : INFINITY;
    if (passes & P_ZFP_GT) t.best_gt = t.br_sz_gt < t.br_zfp_gt ? 0 : 1;
  }
  t.flags = s.flags & (RD_F_DELTA_CLAMPED | RD_F_MSE_ZERO | RD_F_CONSTANT);
}

cudaError_t launch_finish(const ParamsDev& p, Workspace* ws, int passes, int zfp_parts,
                          int sz_parts, long long npoints_all, unsigned long long zfp_npoints,
                          cudaStream_t s) {
  k_finish<<<1, kFinishThreads, 0, s>>>(p, ws, passes, zfp_parts, sz_parts, npoints_all, zfp_npoints);
  return cudaGetLastError();
}

}  // namespace rdk
