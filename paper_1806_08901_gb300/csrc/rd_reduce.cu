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
  uint32_t* pr = &ws->present[0][0];
  for (int i = tid; i < 2 * (kNsym / 32); i += nth) pr[i] = 0u;
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
      ws->huff[w].plogp = 0.0;
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

// Round the limb integer times 2^-312 to the nearest double (ties to even):
// the 53 bits below the leading one, a round bit and a sticky bit.  Every
// limb index is a compile-time constant, so the limbs stay in registers.
__device__ __forceinline__ double limbs_to_double(const unsigned long long (&a)[kLimbs]) {
  // rolling window (w2, w1, w0) = limbs i, i-1, i-2 and the OR of the
  // limbs below it, captured at the highest nonzero limb
  unsigned long long w2 = 0ull, w1 = 0ull, w0 = 0ull;
  bool bl = false;
  unsigned long long h = 0ull, m = 0ull, l = 0ull;
  bool below = false;
  int ti = -1;
#pragma unroll
  for (int i = 0; i < kLimbs; i++) {
    bl = bl || (w0 != 0ull);
    w0 = w1;
    w1 = w2;
    w2 = a[i];
    if (w2) {
      h = w2;
      m = w1;
      l = w0;
      below = bl;
      ti = i;
    }
  }
  if (ti < 0) return 0.0;
  // normalise the 192-bit window h:m:l so that bit 63 of h is the leading one
  const int lz = __clzll((long long)h);
  if (lz) {
    h = (h << lz) | (m >> (64 - lz));
    m = (m << lz) | (l >> (64 - lz));
    l <<= lz;
  }
  unsigned long long mant = h >> 11;  // 53 bits
  const bool round = (h >> 10) & 1ull;
  const bool sticky = (h & 0x3ffull) || m || l || below;
  if (round && (sticky || (mant & 1ull))) mant += 1ull;  // 2^53 stays exact
  const int lead = ti * 64 + 63 - lz;  // bit index of the leading one
  return ldexp((double)mant, lead - 52 - 312);
}

// Launched with one warp.  Bin i holds a 128-bit sum at bit offset 2i, so
// the bins of lane l (i = l + 32k) all sit at shift 2l within limb k: each
// lane adds its bins as one multi-limb integer, shifts it by 2l, and a
// butterfly adds the 32 integers (exact, so the order does not matter).
// The logarithms of the PSNRs run in separate lanes.
__global__ void k_delta(ParamsDev p, Workspace* ws, int mode, double arg, int need_quant,
                        int need_gt, unsigned long long ncoeff, unsigned long long npoints) {
  Scalars& s = ws->sc;
  if (s.status != RD_OK || s.constant) return;
  rd_result& r = ws->res;
  const int lane = threadIdx.x;
  double delta, mse_sp = 0.0;
  bool clamped = false;
  if (mode == DELTA_FROM_MSE) {
    unsigned long long acc[kLimbs];
    unsigned long long lo[9], hi[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const int i = lane + 32 * k;
      lo[k] = i < kMseBins ? s.mse_lo[i] : 0ull;
      hi[k] = i < kMseBins ? s.mse_hi[i] : 0ull;
    }
    unsigned long long carry = 0ull;
#pragma unroll
    for (int k = 0; k < 10; k++) {
      const unsigned long long a0 = k < 9 ? lo[k] : 0ull;
      const unsigned long long a1 = k >= 1 ? hi[k - 1] : 0ull;
      const unsigned long long t = a0 + a1;
      const unsigned long long c1 = t < a0;
      const unsigned long long u = t + carry;
      const unsigned long long c2 = u < carry;
      acc[k] = u;
      carry = c1 + c2;
    }
    acc[10] = carry;
    acc[11] = 0ull;
    const int sh = 2 * lane;
    if (sh) {
#pragma unroll
      for (int j = kLimbs - 1; j > 0; j--) acc[j] = (acc[j] << sh) | (acc[j - 1] >> (64 - sh));
      acc[0] <<= sh;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long c = 0ull;
#pragma unroll
      for (int j = 0; j < kLimbs; j++) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, acc[j], o);
        const unsigned long long u = acc[j] + t;
        const unsigned long long c1 = u < t;
        const unsigned long long v = u + c;
        const unsigned long long c2 = v < c;
        acc[j] = v;
        c = c1 + c2;
      }
    }
    mse_sp = limbs_to_double(acc) / (double)ncoeff;
    if (mse_sp == 0.0) {
      delta = 2.0 * s.eb_abs;
    } else {
      delta = sqrt(12.0 * mse_sp);
      clamped = delta > 2.0 * s.eb_abs;
      if (clamped) delta = 2.0 * s.eb_abs;
    }
  } else if (mode == DELTA_EXPLICIT) {
    delta = arg > 0.0 ? arg : 2.0 * s.eb_abs;
  } else {
    delta = 2.0 * arg;
  }
  // lane 0: log10 VR, lane 1: log10 MSE_sp, lane 2: log10 (VR / delta),
  // lane 3: log10 12
  const double larg = lane == 0 ? s.vr : lane == 1 ? mse_sp : lane == 2 ? s.vr / delta : 12.0;
  const double lg = log10(larg);
  const double l_vr = __shfl_sync(0xffffffffu, lg, 0);
  const double l_mse = __shfl_sync(0xffffffffu, lg, 1);
  const double l_vd = __shfl_sync(0xffffffffu, lg, 2);
  const double l_12 = __shfl_sync(0xffffffffu, lg, 3);
  if (lane != 0) return;
  if (mode == DELTA_FROM_MSE) {
    s.mse_sp = mse_sp;
    r.mse_sp = mse_sp;
    r.zfp_s2 = s.s2;
    r.br_zfp = (double)s.s2 / (2.0 * (double)npoints);
    r.psnr_zfp = mse_sp > 0.0 ? 20.0 * l_vr - 10.0 * l_mse : INFINITY;
    if (mse_sp == 0.0) s.flags |= RD_F_MSE_ZERO;
    if (clamped) s.flags |= RD_F_DELTA_CLAMPED;
  }
  s.delta = delta;
  r.delta = delta;
  r.psnr_sz = 20.0 * l_vd + 10.0 * l_12;
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

// Number of A elements among the first d of merge(A, B), ties from A first:
// the predicate A[i] <= B[d-1-i] holds for a prefix of i in [lo, hi].  A
// 4-way search (three probes per step, loaded together) shortens the chain
// of dependent loads, then binary steps finish.
__device__ __forceinline__ uint32_t merge_split(const uint32_t* A, uint32_t na, const uint32_t* B,
                                                uint32_t nb, uint32_t d) {
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (hi - lo > 3u) {
    const uint32_t q = (hi - lo) >> 2;
    const uint32_t m1 = lo + q, m2 = lo + 2u * q, m3 = lo + 3u * q;
    const bool p1 = A[m1] <= B[d - 1 - m1];
    const bool p2 = A[m2] <= B[d - 1 - m2];
    const bool p3 = A[m3] <= B[d - 1 - m3];
    if (!p1) {
      hi = m1;
    } else if (!p2) {
      lo = m1 + 1u;
      hi = m2;
    } else if (!p3) {
      lo = m2 + 1u;
      hi = m3;
    } else {
      lo = m3 + 1u;
    }
  }
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  return lo;
}


constexpr int kPrepThreads = 256;   // code-statistics prep CTAs (1024 bins each)
constexpr int kHuffThreads = 1024;  // Huffman CTA
constexpr uint32_t kMinPairs = 1;   // fewest pairs per thread in a Huffman phase

// Numbers of elements below T of the sorted a[0..na) and b[0..nb), found
// together by one warp: each round tests 32 evenly spaced elements of every
// range still wider than 32 and keeps the gap holding the answer; a range of
// at most 32 is answered by one ballot.  T < 2^33; a T of 2^32 or more
// exceeds every 32-bit element.
__device__ __forceinline__ void warp_count_below2(const uint32_t* a, uint32_t na,
                                                  const uint32_t* b, uint32_t nb,
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
  uint32_t alo = 0u, ahi = na, blo = 0u, bhi = nb;
  ra = kOpen;
  rb = kOpen;
  while (ra == kOpen || rb == kOpen) {
    const bool wa = ahi - alo > 32u, wb = bhi - blo > 32u;
    const uint32_t sa = wa ? (ahi - alo + 31u) >> 5 : 1u;
    const uint32_t sb = wb ? (bhi - blo + 31u) >> 5 : 1u;
    const uint32_t ia = alo + lane * sa, ib = blo + lane * sb;
    const bool pa = ra == kOpen && ia < ahi && a[ia] < t;
    const bool pb = rb == kOpen && ib < bhi && b[ib] < t;
    const uint32_t ca = (uint32_t)__popc(__ballot_sync(0xffffffffu, pa));
    const uint32_t cb = (uint32_t)__popc(__ballot_sync(0xffffffffu, pb));
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

// ---------------------------------------------------------------------------
// Table of v log2 v for the entropy (v < 2^16), filled once per workspace.
// ---------------------------------------------------------------------------
__global__ void k_init_xlogx(Workspace* ws) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < kNsym) ws->xlogx[v] = v > 1 ? (double)v * log2((double)v) : 0.0;
}

cudaError_t launch_init_tables(Workspace* ws, cudaStream_t s) {
  k_init_xlogx<<<kNsym / 256, 256, 0, s>>>(ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prep (kEntropyCtas CTAs per histogram, 1024 bins each, integer work only):
// the multiplicity of every count value below 2^16 (a counting sort of the
// counts; lanes holding equal counts merge into one atomic), a bitmap of the
// count values present, and the counts of 2^16 or more (at most N / 2^16 of
// them) appended to a list, with their share c log2 c of the entropy sum.
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
  uint32_t* present = ws->present[which];
  uint32_t* big = ws->node_scratch[which];
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 1024 / kPrepThreads; k++) {
    const uint32_t c = ws->hist[which][slice * 1024 + k * kPrepThreads + threadIdx.x];
    const bool small = c != 0u && c < (uint32_t)kNsym;
    const bool large = c >= (uint32_t)kNsym;
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
  if (lane == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double t = warp_sum(threadIdx.x < kPrepThreads / 32 ? part[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) ws->ent_part[which][slice] = t;
  }
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

__device__ double block_sum_f64(double v, double* s_w) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  const double t = warp_sum(s_w[threadIdx.x & 31]);
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// Huffman cost and entropy sum (one CTA per histogram).
//  1. The bitmap of present count values gives each its rank d in ascending
//     order; the D distinct values and their multiplicities (packed as
//     v << 16 | (m - 1)) are gathered in that order.  The entropy sum is
//     sum m v log2 v over them, from the table, plus the large counts' share.
//  2. The ascending leaf array: the first position of every distinct value
//     is marked with the value and a running maximum over positions fills
//     each run; the large counts follow, sorted by a bitonic network.
//  3. The phased two-queue merge: one warp finds the phase threshold and
//     the numbers of leaves and nodes below it, then the threads pair
//     contiguous runs of the merged order (nodes are written only above the
//     queue tail, which no thread reads until the next barrier).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kHuffThreads) k_huffman(Workspace* ws, int which0) {
  extern __shared__ uint32_t s_dyn[];
  __shared__ uint32_t s_w[32];
  __shared__ unsigned long long s_w64[32];
  __shared__ double s_wd[32];
  if (ws->sc.status != RD_OK || ws->sc.constant) return;
  const int which = which0 + blockIdx.x;
  const int tid = threadIdx.x;
  const uint32_t* cc = ws->count_of[which];

  // 1. distinct values in ascending order
  const uint2 pw = reinterpret_cast<const uint2*>(ws->present[which])[tid];
  const uint32_t nbig = ws->nbig[which];
  double ent = tid < kEntropyCtas ? ws->ent_part[which][tid] : 0.0;
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
  unsigned long long nsum = 0ull;
  for (uint32_t d0 = tid; d0 < D; d0 += 4u * kHuffThreads) {
    uint32_t vv[4], mm[4];
    double xl[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t d = d0 + (uint32_t)u * kHuffThreads;
      vv[u] = d < D ? dv[d] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t d = d0 + (uint32_t)u * kHuffThreads;
      mm[u] = d < D ? cc[vv[u]] : 0u;
      xl[u] = d < D ? ws->xlogx[vv[u]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t d = d0 + (uint32_t)u * kHuffThreads;
      if (d < D) {
        dv[d] = (vv[u] << 16) | (mm[u] - 1u);
        msum += mm[u];
        nsum += (unsigned long long)mm[u] * vv[u];
        ent += (double)mm[u] * xl[u];
      }
    }
  }
  const uint32_t* big = ws->node_scratch[which];
  for (uint32_t i = tid; i < nbig; i += kHuffThreads) nsum += big[i];
  uint32_t nsmall;
  (void)block_excl_sum(msum, s_w, &nsmall);
  const unsigned long long ns = block_sum_u64(nsum, s_w64);
  const double plogp = block_sum_f64(ent, s_wd);
  const uint32_t K = nsmall + nbig;

  // 2. leaves
  uint32_t* leaves;
  uint32_t* nodes;
  if (K <= (uint32_t)kHuffSmemKeys) {
    leaves = s_dyn;
    nodes = s_dyn + kHuffSmemKeys;  // the distinct list lives here until the phases
  } else {
    leaves = ws->sort_scratch[which];
    nodes = ws->node_scratch[which];  // free once the large counts are copied
  }
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
  unsigned long long cost = 0ull;
  if (K == 1) {
    cost = (tid == 0) ? ns : 0ull;
  } else if (K > 1) {
    uint32_t lh = 0u, ih = 0u, it = 0u;  // leaf head, node head, node tail
    for (;;) {
      if ((K - lh) + (it - ih) <= 1u) break;
      if (tid < 32) {
        unsigned long long c4[4] = {~0ull, ~0ull, ~0ull, ~0ull};
        if (lh < K) c4[0] = leaves[lh];
        if (lh + 1 < K) c4[1] = leaves[lh + 1];
        if (ih < it) c4[2] = nodes[ih];
        if (ih + 1 < it) c4[3] = nodes[ih + 1];
        const unsigned long long m01 = min(c4[0], c4[1]), x01 = max(c4[0], c4[1]);
        const unsigned long long m23 = min(c4[2], c4[3]), x23 = max(c4[2], c4[3]);
        const unsigned long long a0 = min(m01, m23);
        const unsigned long long a1 = m01 < m23 ? min(x01, m23) : min(x23, m01);
        uint32_t ml, mi;
        warp_count_below2(leaves + lh, K - lh, nodes + ih, it - ih, a0 + a1, ml, mi);
        // leaves among the 2 np paired items: all ml, unless the count is
        // odd and the last item below T in merged order (ties: leaves
        // first) is a leaf; that item waits for the next phase
        uint32_t cl = ml;
        if ((ml + mi) & 1u) {
          if (mi == 0u || (ml > 0u && leaves[lh + ml - 1] > nodes[ih + mi - 1])) cl = ml - 1u;
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
      const uint32_t* A = leaves + lh;
      const uint32_t* B = nodes + ih;
      // each thread pairs a contiguous run of the merged order (at least
      // kMinPairs, so that few warps search when the phase is small)
      const uint32_t per_t = max(kMinPairs, (np + kHuffThreads - 1) / kHuffThreads);
      const uint32_t j0 = (uint32_t)tid * per_t;
      const uint32_t j1 = min(np, j0 + per_t);
      if (j0 < j1) {
        uint32_t i = merge_split(A, ml, B, mi, 2u * j0);
        uint32_t k = 2u * j0 - i;
        for (uint32_t j = j0; j < j1; j++) {
          uint32_t e0v, e1v;
          if (i < ml && (k >= mi || A[i] <= B[k])) e0v = A[i++]; else e0v = B[k++];
          if (i < ml && (k >= mi || A[i] <= B[k])) e1v = A[i++]; else e1v = B[k++];
          const uint32_t sum = e0v + e1v;
          nodes[it + j] = sum;
          cost += sum;
        }
      }
      __syncthreads();
      lh += cl;
      ih += 2u * np - cl;
      it += np;
    }
  }
  cost = block_sum_u64(cost, s_w64);
  if (tid == 0) {
    ws->huff[which].ns = ns;
    ws->huff[which].cost = cost;
    ws->huff[which].nsym = K;
    ws->huff[which].plogp = plogp;
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
  double zsse = 0.0, ssse = 0.0;
  if (!s.constant) {
    if (passes & P_ZFP_GT) zsse = block_sum_parts(ws->zfp_sse, zfp_parts, red);
    if (passes & P_SZ_GT) ssse = block_sum_parts(ws->sz_sse, sz_parts, red);
  }
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  // the logarithms in separate lanes: 0 VR, 1 N_s, 2 ZFP truth MSE, 3 SZ truth MSE
  const double ns_d = (double)ws->huff[0].ns;
  const double mse_z = zsse / (double)npoints_all;
  const double mse_s = ssse / (double)npoints_all;
  const double larg = lane == 0 ? s.vr : lane == 1 ? ns_d : lane == 2 ? mse_z : mse_s;
  const double lg2 = log2(larg);
  const double kLog10of2 = 0.30102999566398119521;
  const double l_vr = __shfl_sync(0xffffffffu, lg2, 0) * kLog10of2;
  const double l_ns = __shfl_sync(0xffffffffu, lg2, 1);
  const double l_mz = __shfl_sync(0xffffffffu, lg2, 2) * kLog10of2;
  const double l_ms = __shfl_sync(0xffffffffu, lg2, 3) * kLog10of2;
  if (lane != 0) return;
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
  const double lvr = 20.0 * l_vr;
  if (passes & P_SZ_EST) {
    const HuffOut& hh = ws->huff[0];
    double ns = (double)hh.ns;
    double H = l_ns - hh.plogp / ns;
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
    t.psnr_zfp_gt = mse_z > 0.0 ? lvr - 10.0 * l_mz : INFINITY;
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
    t.psnr_sz_gt = mse_s > 0.0 ? lvr - 10.0 * l_ms : INFINITY;
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
