// rd_zfp.cu -- ZFP block pass.  One thread owns one 4^d block in registers:
// exponent alignment, block-floating-point cast, lifting transform along
// every axis, sequency order, negabinary bit planes (Sections "Block
// Orthogonal Transformation" and "Estimation Based on Dynamic
// Quantization"), then
//   estimator (sampled blocks, Alg. 1 lines 3-6): n_sb at the EC-sampled
//     coefficients, piecewise-linear interpolation, doubled sum S2; truncation
//     errors d, summed exactly per block exponent for MSE_sp;
//   ground truth (every block): exact group-test embedded-coding bits,
//     truncation, inverse transform, reconstruction, SSE and max error.
#include <stdint.h>

#include "rd_delta.cuh"
#include "rd_device.cuh"

namespace rdk {

constexpr int kZfpThreads = 128;

// Load a 4^D block with edge clamping (partial blocks replicate the last
// valid sample along each axis).
template <int D>
__device__ __forceinline__ void load_block(const FieldDev& f, const int* b, float* v) {
  const float* __restrict__ x = f.x;
  constexpr int NR = (1 << (2 * D)) / 4;  // rows along the fastest axis
  const int nf = f.n[D - 1];
  const int x0 = 4 * b[D - 1];
#pragma unroll
  for (int r = 0; r < NR; r++) {
    long long row = 0;
    if constexpr (D == 2) {
      int y = min(4 * b[0] + r, f.n[0] - 1);
      row = (long long)y * nf;
    } else if constexpr (D == 3) {
      int z = min(4 * b[0] + (r >> 2), f.n[0] - 1);
      int y = min(4 * b[1] + (r & 3), f.n[1] - 1);
      row = ((long long)z * f.n[1] + y) * nf;
    }
    const float* p = x + row;
    if (f.vec_ok) {
      float4 q = __ldg(reinterpret_cast<const float4*>(p + x0));
      v[4 * r + 0] = q.x;
      v[4 * r + 1] = q.y;
      v[4 * r + 2] = q.z;
      v[4 * r + 3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++) v[4 * r + j] = __ldg(p + min(x0 + j, nf - 1));
    }
  }
}

struct BlockInfo {
  int emax;      // block exponent (-127 for an all-zero block)
  int prec;      // coded planes P
  int kmin;      // lowest coded plane, 32 - P
  int all_zero;
};

// Exponent and precision (zfp fixed-accuracy rule): emax = largest frexp
// exponent of the block's values (>= -126), P = clamp(emax - minexp +
// 2(d+1), 0, 32).
template <int D>
__device__ __forceinline__ BlockInfo block_info(const float* v, int minexp) {
  constexpr int NB = 1 << (2 * D);
  unsigned ebits = 0u, nz = 0u;
#pragma unroll
  for (int t = 0; t < NB; t++) {
    unsigned b = __float_as_uint(v[t]);
    ebits = max(ebits, (b >> 23) & 0xffu);
    nz |= b & 0x7fffffffu;
  }
  BlockInfo bi;
  bi.all_zero = nz == 0u;
  // frexp exponent of a normal float is E - 126; subnormals clamp to -126
  bi.emax = bi.all_zero ? -127 : (ebits == 0u ? -126 : (int)ebits - 126);
  int p = bi.emax - minexp + 2 * (D + 1);
  bi.prec = bi.all_zero ? 0 : min(32, max(0, p));
  bi.kmin = 32 - bi.prec;
  return bi;
}

// Exact group-test embedded-coding cost of the planes 31..kmin, from the
// leading-one position c_j of each coefficient (-1 when below kmin).  With
// M_j the suffix maximum of c, plane k starts with n_k = #{j : M_j > k}
// significant coefficients and finds the ones at positions where c_j = M_j.
// Summed over planes: sum_j max(0, M_j - kmin + 1)  (verbatim bits)
//   + #{planes whose group test ends with 0}       = 31 - max(kmin-1, c_last)
//   + #{j : c_j >= kmin, c_j = M_j}                 (one bit per found one)
//   - [c_last >= kmin]                              (the implied last one).
template <int D>
__device__ __forceinline__ unsigned ec_bits(const int* c, int kmin) {
  constexpr int NB = 1 << (2 * D);
  int M = -1;
  int verbatim = 0, found = 0;
#pragma unroll
  for (int p = NB - 1; p >= 0; p--) {
    M = max(M, c[p]);
    verbatim += max(0, M - kmin + 1);
    found += (c[p] >= kmin && c[p] == M) ? 1 : 0;
  }
  const int last = c[NB - 1];
  int tests = 31 - max(kmin - 1, last);
  return 9u + (unsigned)(verbatim + tests + found - (last >= kmin ? 1 : 0));
}

// The full per-block computation shared by the pass and the inspector.
template <int D>
struct BlockWork {
  static constexpr int NB = 1 << (2 * D);
  unsigned u[NB];    // negabinary, sequency order
  BlockInfo bi;

  __device__ __forceinline__ void forward(const float* v, int minexp) {
    constexpr Sequency<D> S{};
    bi = block_info<D>(v, minexp);
    int c[NB];
    const int sh = 30 - bi.emax;
#pragma unroll
    for (int t = 0; t < NB; t++) c[t] = bi.all_zero ? 0 : cast_scaled(v[t], sh);
    if (!bi.all_zero) fwd_xform<D>(c);
#pragma unroll
    for (int p = 0; p < NB; p++) {
      u[p] = to_negabinary(c[S.perm[p]]);
    }
  }
  __device__ __forceinline__ unsigned keep_mask() const {
    return bi.kmin >= 32 ? 0u : (0xffffffffu << bi.kmin);
  }
  __device__ __forceinline__ unsigned bits() const {
    if (bi.prec == 0) return 1u;
    int c[NB];
#pragma unroll
    for (int p = 0; p < NB; p++) {
      int b = 31 - __clz((int)u[p]);
      c[p] = b >= bi.kmin ? b : -1;
    }
    return ec_bits<D>(c, bi.kmin);
  }
  // Reconstruction of the block (block order) from the truncated planes.
  __device__ __forceinline__ void reconstruct(float* xr) const {
    constexpr Sequency<D> S{};
    if (bi.prec == 0) {
#pragma unroll
      for (int t = 0; t < NB; t++) xr[t] = 0.0f;
      return;
    }
    const unsigned keep = keep_mask();
    int c[NB];
#pragma unroll
    for (int p = 0; p < NB; p++) c[S.perm[p]] = from_negabinary(u[p] & keep);
    inv_xform<D>(c);
    const int e = bi.emax - 30;
#pragma unroll
    for (int t = 0; t < NB; t++) xr[t] = scale_pow2(__int2float_rn(c[t]), e);
  }
};

// Valid-point mask of a (possibly partial) block, bit t for block index t.
template <int D>
__device__ __forceinline__ unsigned long long valid_mask(const FieldDev& f, const int* b) {
  constexpr int NB = 1 << (2 * D);
  int v[3] = {4, 4, 4};
#pragma unroll
  for (int k = 0; k < D; k++) v[k] = min(4, f.n[k] - 4 * b[k]);
  unsigned long long m = 0ull;
#pragma unroll
  for (int t = 0; t < NB; t++) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; k++) ok = ok && (((t >> (2 * (D - 1 - k))) & 3) < v[k]);
    if (ok) m |= 1ull << t;
  }
  return m;
}

template <int D>
__device__ __forceinline__ void decode_block(const FieldDev& f, long long u, bool sampled_only,
                                             int* b) {
  if (sampled_only) {
    long long r = u;
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
      int l = (int)(r % f.L[k]);
      r /= f.L[k];
      b[k] = l * f.s[k];
    }
  } else {
    long long r = u;
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
      b[k] = (int)(r % f.B[k]);
      r /= f.B[k];
    }
  }
}

// Estimator terms of one sampled block (Alg. 1 lines 4-6): the doubled
// interpolated n_sb sum into s2, and the exact squared truncation errors at
// the EC-sampled coefficients into the 128-bit bin of the block exponent.
template <int D>
__device__ __forceinline__ void zfp_est_accumulate(const BlockWork<D>& w, bool ec_all,
                                                   unsigned long long& my_s2,
                                                   unsigned long long* s_lo,
                                                   unsigned long long* s_hi) {
  constexpr int NB = 1 << (2 * D);
  constexpr EcPositions<D> EC{};
  // n_sb at the sampled positions, interpolated in sequency index
  auto nsb = [&](int q) {
    int bb = 31 - __clz((int)w.u[q]);
    return bb >= w.bi.kmin ? bb - w.bi.kmin + 1 : 0;
  };
  long long s2 = 0;
  unsigned long long lo = 0ull, hi = 0ull;
  const unsigned keep = w.keep_mask();
  if (ec_all) {
#pragma unroll
    for (int q = 0; q < NB; q++) {
      s2 += 2 * nsb(q);
      long long d = (long long)from_negabinary(w.u[q]) - (long long)from_negabinary(w.u[q] & keep);
      unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
      unsigned long long sq = ad * ad;  // |d| < 2^32
      lo += sq;
      hi += (lo < sq);
    }
  } else {
#pragma unroll
    for (int j = 0; j < EcPositions<D>::M; j++) {
      const int q = EC.pos[j];
      if (j + 1 < EcPositions<D>::M) {
        const int L = EC.pos[j + 1] - q;
        s2 += (long long)(L + 1) * nsb(q) + (long long)(L - 1) * nsb(EC.pos[j + 1]);
      } else {
        s2 += 2 * nsb(q);
      }
      long long d = (long long)from_negabinary(w.u[q]) - (long long)from_negabinary(w.u[q] & keep);
      unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
      unsigned long long sq = ad * ad;  // |d| < 2^32
      lo += sq;
      hi += (lo < sq);
    }
  }
  my_s2 += (unsigned long long)s2;
  if (!w.bi.all_zero && (lo | hi)) {
    const int bin = w.bi.emax + D + 126;  // exponent of the 2^d-rescaled error
    unsigned long long old = atomicAdd(&s_lo[bin], lo);
    unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&s_hi[bin], hi + carry);
  }
}

template <int D, bool GT, bool EST>
__global__ void __launch_bounds__(kZfpThreads) k_zfp(FieldDev f, ParamsDev p, Workspace* ws) {
  constexpr int NB = 1 << (2 * D);
  __shared__ unsigned long long s_lo[kMseBins], s_hi[kMseBins];
  __shared__ unsigned long long s_acc[2];
  __shared__ double s_sse[kZfpThreads / 32];
  __shared__ float s_max[kZfpThreads / 32];
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  const int minexp = sc.minexp;
  if (EST) {
    for (int i = threadIdx.x; i < kMseBins; i += blockDim.x) {
      s_lo[i] = 0ull;
      s_hi[i] = 0ull;
    }
  }
  if (threadIdx.x < 2) s_acc[threadIdx.x] = 0ull;
  __syncthreads();

  const long long units = GT ? f.nblocks : f.nsampled;
  unsigned long long my_s2 = 0ull, my_bits = 0ull;
  double my_sse = 0.0;
  float my_max = 0.0f;
  const bool ec_all = p.ec_mode == RD_EC_ALL;

  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    int b[3] = {0, 0, 0};
    decode_block<D>(f, u, !GT, b);
    bool sampled = true;
    if (GT) {
#pragma unroll
      for (int k = 0; k < D; k++) sampled = sampled && (b[k] % f.s[k] == 0);
    }
    float v[NB];
    load_block<D>(f, b, v);
    BlockWork<D> w;
    w.forward(v, minexp);

    if (EST && sampled) zfp_est_accumulate<D>(w, ec_all, my_s2, s_lo, s_hi);

    if (GT) {
      my_bits += w.bits();
      float xr[NB];
      w.reconstruct(xr);
      float e2[NB];
      float emx = 0.0f;
      bool interior = true;
#pragma unroll
      for (int k = 0; k < D; k++) interior = interior && (4 * b[k] + 4 <= f.n[k]);
      if (interior) {
#pragma unroll
        for (int t = 0; t < NB; t++) {
          e2[t] = __fsub_rn(v[t], xr[t]);
          emx = fmaxf(emx, fabsf(e2[t]));
        }
      } else {
        const unsigned long long vm = valid_mask<D>(f, b);
#pragma unroll
        for (int t = 0; t < NB; t++) {
          float e = __fsub_rn(v[t], xr[t]);
          e2[t] = ((vm >> t) & 1ull) ? e : 0.0f;
          emx = fmaxf(emx, fabsf(e2[t]));
        }
      }
      my_max = fmaxf(my_max, emx);
      if (emx > 0.0f) {
        // scale by 2^k (exact) so the largest error is in [1, 2): squares
        // of errors far below eb_abs neither underflow nor lose the sum
        const unsigned E = (__float_as_uint(emx) >> 23) & 0xffu;
        const int k = E ? 127 - (int)E : 149;
        if (k <= 127 && k >= -126) {
          const float sc = pow2f(k);
#pragma unroll
          for (int t = 0; t < NB; t++) {
            const float es = __fmul_rn(e2[t], sc);
            e2[t] = __fmul_rn(es, es);
          }
        } else {
#pragma unroll
          for (int t = 0; t < NB; t++) {
            const float es = mul_pow2(e2[t], k);
            e2[t] = __fmul_rn(es, es);
          }
        }
        // pairwise sum of the block's scaled squared errors in float
#pragma unroll
        for (int w2 = NB / 2; w2 >= 1; w2 >>= 1) {
#pragma unroll
          for (int t = 0; t < w2; t++) e2[t] = __fadd_rn(e2[t], e2[t + w2]);
        }
        my_sse += (double)e2[0] * __longlong_as_double((long long)(1023 - 2 * k) << 52);
      }
    }
  }

  // reductions: warp, then CTA, then one global update per CTA
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (EST) {
    unsigned long long t = warp_sum(my_s2);
    if (lane == 0 && t) atomicAdd(&s_acc[0], t);
  }
  if (GT) {
    unsigned long long t = warp_sum(my_bits);
    if (lane == 0) atomicAdd(&s_acc[1], t);
    double ss = warp_sum(my_sse);
    float mm = warp_max(my_max);
    if (lane == 0) {
      s_sse[wid] = ss;
      s_max[wid] = mm;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (EST && s_acc[0]) atomicAdd(&ws->sc.s2, s_acc[0]);
    if (GT) {
      atomicAdd(&ws->sc.zfp_bits, s_acc[1]);
      double ss = 0.0;
      float mm = 0.0f;
      for (int i = 0; i < kZfpThreads / 32; i++) {
        ss += s_sse[i];
        mm = fmaxf(mm, s_max[i]);
      }
      ws->zfp_sse[blockIdx.x] = ss;
      atomicMax(&ws->sc.zfp_maxerr, __float_as_uint(mm));
    }
  }
  if (EST) {
    for (int i = threadIdx.x; i < kMseBins; i += blockDim.x)
      if (s_lo[i] | s_hi[i]) atomic_add_u128(&ws->sc.mse_lo[i], &ws->sc.mse_hi[i], s_lo[i], s_hi[i]);
  }
}

template <int D>
static cudaError_t launch_zfp_d(const FieldDev& f, const ParamsDev& p, int passes, Workspace* ws,
                                int ctas, cudaStream_t s, int* grid_used) {
  const bool gt = passes & P_ZFP_GT, est = passes & P_ZFP_EST;
  long long units = gt ? f.nblocks : f.nsampled;
  long long want = (units + kZfpThreads - 1) / kZfpThreads;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (grid_used) *grid_used = g;
  if (gt && est)
    k_zfp<D, true, true><<<g, kZfpThreads, 0, s>>>(f, p, ws);
  else if (gt)
    k_zfp<D, true, false><<<g, kZfpThreads, 0, s>>>(f, p, ws);
  else
    k_zfp<D, false, true><<<g, kZfpThreads, 0, s>>>(f, p, ws);
  return cudaGetLastError();
}

cudaError_t launch_zfp(const FieldDev& f, const ParamsDev& p, int passes, Workspace* ws, int ctas,
                       cudaStream_t s, int* grid_used) {
  switch (f.d) {
    case 1: return launch_zfp_d<1>(f, p, passes, ws, ctas, s, grid_used);
    case 2: return launch_zfp_d<2>(f, p, passes, ws, ctas, s, grid_used);
    default: return launch_zfp_d<3>(f, p, passes, ws, ctas, s, grid_used);
  }
}

// Number of CTAs of the pass that the SMs hold at once (a grid-stride pass
// is sized to that; extra CTAs only add tail).
int zfp_occupancy(int d, int num_sms) {
  int per = 0;
  const void* fn = nullptr;
  if (d == 1) fn = (const void*)k_zfp<1, true, true>;
  else if (d == 2) fn = (const void*)k_zfp<2, true, true>;
  else fn = (const void*)k_zfp<3, true, true>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kZfpThreads, 0) != cudaSuccess || per < 1)
    per = 1;
  long long g = (long long)per * num_sms;
  return (int)(g > kMaxGrid ? kMaxGrid : g);
}

// ---------------------------------------------------------------------------
// Batched estimate: sampled blocks of many fields.  Each work item is a run
// of sampled blocks of one field, accumulated in shared memory and added to
// the field's exact sums when the item ends; the CTA that finishes a field's
// last item then derives the bin width delta of that field (one warp).
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void zfp_est_item(const FieldDev& f, const ParamsDev& p, int minexp,
                                             long long u0, long long u1,
                                             unsigned long long& my_s2, unsigned long long* s_lo,
                                             unsigned long long* s_hi) {
  constexpr int NB = 1 << (2 * D);
  const bool ec_all = p.ec_mode == RD_EC_ALL;
  for (long long u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    int b[3] = {0, 0, 0};
    decode_block<D>(f, u, true, b);
    float v[NB];
    load_block<D>(f, b, v);
    BlockWork<D> w;
    w.forward(v, minexp);
    zfp_est_accumulate<D>(w, ec_all, my_s2, s_lo, s_hi);
  }
}

__global__ void __launch_bounds__(kZfpThreads) k_batch_zfp_est(const BatchField* __restrict__ bf,
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

cudaError_t launch_batch_zfp_est(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                 cudaStream_t s) {
  int g = nitems < ctas ? nitems : ctas;
  if (g < 1) g = 1;
  k_batch_zfp_est<<<g, kZfpThreads, 0, s>>>(bf, items, nitems);
  return cudaGetLastError();
}

int batch_zfp_occupancy(int num_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_batch_zfp_est, kZfpThreads, 0) !=
          cudaSuccess ||
      per < 1)
    per = 1;
  return per * num_sms;
}

// ---------------------------------------------------------------------------
// Inspector: per-block records through the same block code.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_zfp_inspect(FieldDev f, int minexp, int32_t* emax, int32_t* prec,
                              uint64_t* bits, uint32_t* coeffs) {
  constexpr int NB = 1 << (2 * D);
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < f.nblocks;
       u += (long long)gridDim.x * blockDim.x) {
    int b[3] = {0, 0, 0};
    decode_block<D>(f, u, false, b);
    float v[NB];
    load_block<D>(f, b, v);
    BlockWork<D> w;
    w.forward(v, minexp);
    if (emax) emax[u] = w.bi.emax;
    if (prec) prec[u] = w.bi.prec;
    if (bits) bits[u] = w.bits();
    if (coeffs) {
#pragma unroll
      for (int q = 0; q < NB; q++) coeffs[u * NB + q] = w.u[q];
    }
  }
}

cudaError_t launch_zfp_inspect(const FieldDev& f, double eb_abs, int32_t* emax, int32_t* prec,
                               uint64_t* bits, uint32_t* coeffs, cudaStream_t s) {
  int e;
  frexp(eb_abs, &e);
  const int minexp = e - 1;
  long long g = (f.nblocks + 127) / 128;
  if (g > 65535) g = 65535;
  if (g < 1) g = 1;
  switch (f.d) {
    case 1: k_zfp_inspect<1><<<(int)g, 128, 0, s>>>(f, minexp, emax, prec, bits, coeffs); break;
    case 2: k_zfp_inspect<2><<<(int)g, 128, 0, s>>>(f, minexp, emax, prec, bits, coeffs); break;
    default: k_zfp_inspect<3><<<(int)g, 128, 0, s>>>(f, minexp, emax, prec, bits, coeffs); break;
  }
  return cudaGetLastError();
}

}  // namespace rdk
