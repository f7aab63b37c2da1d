// rd_sz_log.cu -- the log-scale quantisation estimate (Section "Estimation
// Based on Static Quantization", log-scale case): the residuals of the
// linear SZ estimate (Lorenzo prediction from the original neighbours at the
// points of the sampled blocks) binned on a logarithmic scale.
//
// Bins, with magnitudes in units of u = eb_abs and n = quant_radius: the
// central bin |r| < A[1] (code 0, width 2 A[1]) and, for |r| >= A[1], code
// sign(r) k with k the number of edges A[1..n-1] at or below |r| (the bin
// [A[k], A[k+1]), width A[k+1] - A[k]); A[k] = u pow(b, k), b the smallest
// double >= 1 with A[n] above the largest |r|.  The edge table is computed on
// the host in float64 (a library power function is not the same on the
// device); the device compares each |r|, a float, with the smallest float at
// or above each edge, which decides exactly as the float64 comparison.
//
// Passes: the largest |r| (one atomic maximum per warp); the host derives b
// and the tables; the histogram (binary search over the edges, one global
// atomic per point: the log bins spread the codes evenly); Huffman cost and
// entropy sums of that histogram (the linear estimate's code statistics);
// the finish: the bin model's MSE (Eq. mse-pdf) summed in a fixed order,
// entropy (Eq. bit-rate-pdf), PSNR (Eq. psnr-pdf).
#include <math.h>
#include <stdint.h>

#include "rd_sz_dev.cuh"

namespace rdk {

constexpr int kLogThreads = 256;
constexpr int kLogFinishThreads = 1024;

template <int D>
__global__ void __launch_bounds__(kLogThreads) k_sz_log_max(FieldDev f, Workspace* ws) {
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  float m = 0.0f;
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < f.nsampled;
       b0 += (long long)gridDim.x * blockDim.x) {
    const long long sb = b0 + threadIdx.x;
    sz_block_residuals<D>(f, sb, sb < f.nsampled, [&](float r) { m = fmaxf(m, fabsf(r)); },
                          [] {});
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&ws->sc.log_maxabs, __float_as_uint(m));
}

// F[i - 1] = the smallest float >= A[i], i = 1 .. n-1, non-decreasing.
template <int D>
__global__ void __launch_bounds__(kLogThreads) k_sz_log_hist(FieldDev f, int n,
                                                             const float* __restrict__ F,
                                                             Workspace* ws) {
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  uint32_t* g = ws->hist[0];
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < f.nsampled;
       b0 += (long long)gridDim.x * blockDim.x) {
    const long long sb = b0 + threadIdx.x;
    sz_block_residuals<D>(
        f, sb, sb < f.nsampled,
        [&](float r) {
          const float a = fabsf(r);
          int lo = 0, hi = n - 1;  // the count of edges <= a, in [0, n-1]
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(F + mid - 1) <= a)
              lo = mid;
            else
              hi = mid - 1;
          }
          atomicAdd(&g[kCenter + (r < 0.0f ? -lo : lo)], 1u);
        },
        [] {});
  }
}

// One CTA.  A[0..n] holds u and the edges.
__global__ void __launch_bounds__(kLogFinishThreads) k_sz_log_finish(ParamsDev p,
                                                                     const double* __restrict__ A,
                                                                     Workspace* ws,
                                                                     rd_log_result* out) {
  __shared__ double red[kLogFinishThreads / 32];
  const Scalars& s = ws->sc;
  if (s.status != RD_OK || s.constant) return;
  const uint32_t* h = ws->hist[0];
  double part = 0.0;
  for (int sym = threadIdx.x; sym < kNsym; sym += blockDim.x) {
    const uint32_t c = h[sym];
    if (c) {
      const int k = sym >= kCenter ? sym - kCenter : kCenter - sym;
      const double w = k == 0 ? 2.0 * A[1] : A[k + 1] - A[k];
      part += (double)c * (w * w);
    }
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  double t = threadIdx.x < (kLogFinishThreads / 32) ? red[threadIdx.x] : 0.0;
  t = warp_sum(t);
  if (threadIdx.x != 0) return;
  const HuffOut& hh = ws->huff[0];
  const double ns = (double)hh.ns;
  double H = log2(ns) - hh.plogp / ns;
  if (H < 0.0) H = 0.0;
  rd_log_result& r = *out;
  r.vr = s.vr;
  r.eb_abs = s.eb_abs;
  r.entropy = H;
  r.br_log = H + p.sz_offset;
  r.ns = hh.ns;
  r.huff_bits = hh.cost;
  r.nsym = hh.nsym;
  r.br_log_huff = (double)hh.cost / ns;
  r.mse_log = t / (12.0 * ns);
  r.psnr_log = r.mse_log > 0.0 ? 20.0 * log10(s.vr) - 10.0 * log10(r.mse_log) : INFINITY;
  r.flags = s.flags;
}

cudaError_t launch_sz_log_max(const FieldDev& f, Workspace* ws, int ctas, cudaStream_t s) {
  long long want = (f.nsampled + kLogThreads - 1) / kLogThreads;
  const int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  switch (f.d) {
    case 1: k_sz_log_max<1><<<g, kLogThreads, 0, s>>>(f, ws); break;
    case 2: k_sz_log_max<2><<<g, kLogThreads, 0, s>>>(f, ws); break;
    default: k_sz_log_max<3><<<g, kLogThreads, 0, s>>>(f, ws); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sz_log_hist(const FieldDev& f, int n, const float* F, Workspace* ws, int ctas,
                               cudaStream_t s) {
  long long want = (f.nsampled + kLogThreads - 1) / kLogThreads;
  const int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  switch (f.d) {
    case 1: k_sz_log_hist<1><<<g, kLogThreads, 0, s>>>(f, n, F, ws); break;
    case 2: k_sz_log_hist<2><<<g, kLogThreads, 0, s>>>(f, n, F, ws); break;
    default: k_sz_log_hist<3><<<g, kLogThreads, 0, s>>>(f, n, F, ws); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sz_log_finish(const ParamsDev& p, const double* A, Workspace* ws,
                                 rd_log_result* out, cudaStream_t s) {
  k_sz_log_finish<<<1, kLogFinishThreads, 0, s>>>(p, A, ws, out);
  return cudaGetLastError();
}

}  // namespace rdk
