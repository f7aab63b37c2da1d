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
#include "rd_zfp_dev.cuh"

namespace rdk {

template <int D, bool GT, bool EST>
__global__ void __launch_bounds__(kZfpThreads) k_zfp(FieldDev f, ParamsDev p, DeltaArgs da,
                                                      Workspace* ws) {
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

  constexpr EcPositions<D> EC{};
  // warp-uniform trip count: the estimator's bin sums are added per warp
  for (long long base = (long long)blockIdx.x * blockDim.x; base < units;
       base += (long long)gridDim.x * blockDim.x) {
    const long long u = base + threadIdx.x;
    bool est_has = false;
    int est_bin = 0;
    unsigned long long est_lo = 0ull, est_hi = 0ull;
    if (u < units) {
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

    if (EST && sampled) {
      long long s2;
      zfp_est_terms<D>(w.bi.kmin, ec_all, [&](int j) { return ec_all ? w.u[j] : w.u[EC.pos[j]]; },
                       s2, est_lo, est_hi);
      my_s2 += (unsigned long long)s2;
      est_has = !w.bi.all_zero && (est_lo | est_hi);
      est_bin = mse_bin<D>(w.bi.emax);
    }

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
    if (EST) mse_add_warp(est_has, est_bin, est_lo, est_hi, s_lo, s_hi);
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
  if (da.on) {
    // the CTA that ends last derives delta (Algorithm 1 line 7)
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(&ws->sc.done[1], 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
      __threadfence();
      delta_warp(p, ws, da.mode, da.arg, da.need_quant, da.need_gt, da.ncoeff, da.npoints);
    }
  }
}

template <int D>
static cudaError_t launch_zfp_d(const FieldDev& f, const ParamsDev& p, int passes,
                                const DeltaArgs& da, Workspace* ws, int ctas, cudaStream_t s,
                                int* grid_used) {
  const bool gt = passes & P_ZFP_GT, est = passes & P_ZFP_EST;
  long long units = gt ? f.nblocks : f.nsampled;
  long long want = (units + kZfpThreads - 1) / kZfpThreads;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (grid_used) *grid_used = g;
  if (gt && est)
    k_zfp<D, true, true><<<g, kZfpThreads, 0, s>>>(f, p, da, ws);
  else if (gt)
    k_zfp<D, true, false><<<g, kZfpThreads, 0, s>>>(f, p, da, ws);
  else
    k_zfp<D, false, true><<<g, kZfpThreads, 0, s>>>(f, p, da, ws);
  return cudaGetLastError();
}

// 3D fields go to the four-lanes-per-block pass (rd_zfp3.cu); 1D and 2D
// blocks (4 and 16 values) fit one thread each.
cudaError_t launch_zfp(const FieldDev& f, const ParamsDev& p, int passes, const DeltaArgs& da,
                       Workspace* ws, int ctas, cudaStream_t s, int* grid_used) {
  switch (f.d) {
    case 1: return launch_zfp_d<1>(f, p, passes, da, ws, ctas, s, grid_used);
    case 2: return launch_zfp_d<2>(f, p, passes, da, ws, ctas, s, grid_used);
    default: return launch_zfp3(f, p, passes, da, ws, ctas, s, grid_used);
  }
}

// Number of CTAs of the pass that the SMs hold at once (a grid-stride pass
// is sized to that; extra CTAs only add tail).
int zfp_occupancy(int d, int num_sms) {
  if (d == 3) return zfp3_occupancy(num_sms);
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
