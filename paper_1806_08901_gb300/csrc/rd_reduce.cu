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
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&ws->sc.min_key, kmin);
    atomicMax(&ws->sc.max_key, kmax);
    if (bad) atomicOr(&ws->sc.nonfinite, 1u);
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

__device__ int limbs_bit(const unsigned long long* a, int pos) {
  return (int)((a[pos >> 6] >> (pos & 63)) & 1ull);
}

// Round the limb integer times 2^-312 to the nearest double (ties to even).
__device__ double limbs_to_double(const unsigned long long* a) {
  int top = -1;
  for (int i = kLimbs - 1; i >= 0 && top < 0; i--)
    if (a[i]) top = i * 64 + 63 - __clzll((long long)a[i]);
  if (top < 0) return 0.0;
  if (top <= 52) {
    unsigned long long m = a[0];  // fits in the lowest limb
    return ldexp((double)m, -312);
  }
  int shift = top - 52;
  unsigned long long m = 0ull;
  for (int b = 52; b >= 0; b--) m = (m << 1) | (unsigned long long)limbs_bit(a, shift + b);
  int round = limbs_bit(a, shift - 1);
  int sticky = 0;
  for (int b = shift - 2; b >= 0 && !sticky; b--) sticky = limbs_bit(a, b);
  if (round && (sticky || (m & 1ull))) m += 1ull;
  return ldexp((double)m, shift - 312);
}

__global__ void k_delta(ParamsDev p, Workspace* ws, int mode, double arg, int need_quant,
                        int need_gt, unsigned long long ncoeff, unsigned long long npoints) {
  Scalars& s = ws->sc;
  if (s.status != RD_OK || s.constant) return;
  rd_result& r = ws->res;
  double delta;
  if (mode == DELTA_FROM_MSE) {
    unsigned long long acc[kLimbs];
    for (int i = 0; i < kLimbs; i++) acc[i] = 0ull;
    for (int i = 0; i < kMseBins; i++) {
      if (s.mse_lo[i]) limbs_add(acc, s.mse_lo[i], 2 * i);
      if (s.mse_hi[i]) limbs_add(acc, s.mse_hi[i], 2 * i + 64);
    }
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
  k_delta<<<1, 1, 0, s>>>(p, ws, mode, arg, need_quant, need_gt, ncoeff, npoints);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Entropy partials: sum of h log2 h per 1024-bin slice (fixed order).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_entropy(Workspace* ws, int which_mask) {
  __shared__ double part[32];
  for (int which = 0; which < 2; which++) {
    if (!((which_mask >> which) & 1)) continue;
    if (ws->sc.status != RD_OK || ws->sc.constant) return;
    uint32_t h = ws->hist[which][blockIdx.x * 1024 + threadIdx.x];
    double v = h ? (double)h * log2((double)h) : 0.0;
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = warp_sum(part[threadIdx.x]);
      if (threadIdx.x == 0) ws->ent_part[which][blockIdx.x] = t;
    }
    __syncthreads();
  }
}

cudaError_t launch_entropy(Workspace* ws, int which_mask, cudaStream_t s) {
  k_entropy<<<kEntropyCtas, 1024, 0, s>>>(ws, which_mask);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Huffman cost of a histogram: the nonzero counts are compacted, sorted
// ascending (bitonic network with virtual +inf padding, shared memory when
// they fit, else global scratch), then merged with the two-queue method; the
// internal node j is stored in the consumed leaf slot j.  Total cost = sum of
// internal-node weights = coded bits.
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

__global__ void __launch_bounds__(1024) k_huffman(Workspace* ws, int which0) {
  extern __shared__ uint32_t s_keys[];
  __shared__ uint32_t s_cnt[1024];
  __shared__ unsigned long long s_tot[32];
  __shared__ uint32_t s_base;
  const int which = which0 + blockIdx.x;
  if (ws->sc.status != RD_OK || ws->sc.constant) return;
  const uint32_t* h = ws->hist[which];
  const int per = kNsym / 1024;  // 64 bins per thread
  const int b0 = threadIdx.x * per;
  uint32_t nz = 0;
  unsigned long long tot = 0ull;
  for (int i = 0; i < per; i++) {
    uint32_t c = h[b0 + i];
    nz += (c != 0u);
    tot += c;
  }
  // exclusive scan of nonzero counts over the threads
  s_cnt[threadIdx.x] = nz;
  unsigned long long wt = warp_sum(tot);
  if ((threadIdx.x & 31) == 0) s_tot[threadIdx.x >> 5] = wt;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t v = threadIdx.x >= (unsigned)off ? s_cnt[threadIdx.x - off] : 0u;
    __syncthreads();
    s_cnt[threadIdx.x] += v;
    __syncthreads();
  }
  const uint32_t K = s_cnt[1023];
  const uint32_t start = s_cnt[threadIdx.x] - nz;
  unsigned long long ns = 0ull;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 32; i++) ns += s_tot[i];
    s_base = 0;
  }
  uint32_t* keys = (K <= (uint32_t)kHuffSmemKeys) ? s_keys : ws->sort_scratch[which];
  uint32_t o = start;
  for (int i = 0; i < per; i++) {
    uint32_t c = h[b0 + i];
    if (c) keys[o++] = c;
  }
  __syncthreads();
  bitonic_sort(keys, (int)K);
  if (threadIdx.x == 0) {
    unsigned long long cost = 0ull;
    if (K == 1) {
      cost = ns;
    } else if (K > 1) {
      uint32_t lh = 0, nh = 0, nt = 0;
      for (uint32_t step = 0; step + 1 < K; step++) {
        uint32_t pick[2];
        for (int j = 0; j < 2; j++) {
          if (lh < K && (nh >= nt || keys[lh] <= keys[nh]))
            pick[j] = keys[lh++];
          else
            pick[j] = keys[nh++];
        }
        uint32_t sum = pick[0] + pick[1];
        keys[nt++] = sum;  // slot nt was consumed: lh >= nt + 1
        cost += sum;
      }
    }
    ws->huff[which].ns = ns;
    ws->huff[which].cost = cost;
    ws->huff[which].nsym = K;
  }
}

cudaError_t launch_huffman(Workspace* ws, int which_mask, cudaStream_t s) {
  static bool attr = false;
  const int smem = kHuffSmemKeys * (int)sizeof(uint32_t);
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_huffman, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int first = (which_mask & 1) ? 0 : 1;
  int count = (which_mask == 3) ? 2 : 1;
  k_huffman<<<count, 1024, smem, s>>>(ws, first);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Finish: SZ rates, ground-truth rates, PSNRs and the selection.
// ---------------------------------------------------------------------------
__device__ double sum_parts(const double* a, int n) {
  // fixed-order: each lane sums a strided subset, then a fixed butterfly
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) v += a[i];
  return warp_sum(v);
}

__global__ void k_finish(ParamsDev p, Workspace* ws, int passes, int zfp_parts, int sz_parts,
                         long long npoints_all, unsigned long long zfp_npoints) {
  Scalars& s = ws->sc;
  if (s.status != RD_OK) return;
  rd_result& r = ws->res;
  rd_truth& t = ws->truth;
  double zsse = 0.0, ssse = 0.0;
  if (!s.constant) {
    if (passes & P_ZFP_GT) zsse = sum_parts(ws->zfp_sse, zfp_parts);
    if (passes & P_SZ_GT) ssse = sum_parts(ws->sz_sse, sz_parts);
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
    double plogp = 0.0;
    for (int i = 0; i < kEntropyCtas; i++) plogp += ws->ent_part[0][i];
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
  k_finish<<<1, 32, 0, s>>>(p, ws, passes, zfp_parts, sz_parts, npoints_all, zfp_npoints);
  return cudaGetLastError();
}

}  // namespace rdk
