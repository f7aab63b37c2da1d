// rd_sz.cu -- SZ passes.
//   estimator (Alg. 1 line 8; Sections "Prediction-Based Transformation" and
//     "Estimation Based on Static Quantization"): every valid point of every
//     sampled block, Lorenzo residual from its ORIGINAL neighbours (zero
//     outside the domain) evaluated in float32 as nested first differences,
//     last axis first; code q = rint(r * (1/delta)); symbol q + 32768 when
//     |q| < R, else the escape symbol 0; 65536-bin histogram.
//   ground truth (every point, bound delta/2): prequantised code
//     Q = rint(x * (1/w)), reconstruction float(Q) * w, escape when the float
//     error exceeds tau or the integer Lorenzo residual of Q reaches R;
//     histogram of residual symbols, SSE and max error.
#include <stdint.h>

#include "rd_sz_dev.cuh"

namespace rdk {

// Estimator: grid-strided, one CTA of up to 1024 threads per SM with the
// whole-alphabet 16-bit window (codes of fine bounds spread over tens of
// thousands of bins); the 2H+1 codes around the centre are counted in
// registers.  Two work units: with few sampled blocks (their rows fill the
// resident threads at most four times) one thread per row of four points
// (sz_est_row: a row's residuals need only its own four row loads, so the
// gather latency is paid once); otherwise one thread per block
// (sz_est_block: five planes in turn, each row loaded once).  A round is
// one pass of the CTA's threads over rows, or one plane of its 3D blocks,
// or one of its 2D / 1D blocks: at most kRoundPoints points.
constexpr int kSzEstThreads = 1024;
static_assert(kSzEstThreads * 16 <= kRoundPoints, "a round adds at most kRoundPoints");

template <int D, bool ROWS>
__global__ void __launch_bounds__(kSzEstThreads, 1) k_sz_est(FieldDev f, ParamsDev p, Workspace* ws) {
  extern __shared__ uint32_t s_win[];  // kPackWords words of two counters
  __shared__ int s_hot;
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;  // uniform over the grid
  for (int i = threadIdx.x; i < kPackWords; i += blockDim.x) s_win[i] = 0u;
  if (threadIdx.x == 0) s_hot = 0;
  __syncthreads();
  const float inv = sc.inv;
  uint32_t* g_hist = ws->hist[0];
  HotBins<2> hot;
  hot.clear();
  auto add = [&](int sym) {
    if (!hot.take(sym - kCenter)) packed_add(s_win, sym, 1u, &s_hot);
  };
  auto round_end = [&]() {
    __syncthreads();
    if (s_hot) {  // uniform after the barrier
      window_flush(s_win, g_hist);
      if (threadIdx.x == 0) s_hot = 0;
      __syncthreads();
    }
  };
  if (ROWS) {
    constexpr int kRows = est_rows<D>();
    const long long nrows = f.nsampled * kRows;
    for (long long q0 = (long long)blockIdx.x * blockDim.x; q0 < nrows;
         q0 += (long long)gridDim.x * blockDim.x) {  // uniform trip count over the CTA
      const long long q = q0 + threadIdx.x;
      sz_est_row<D>(f, q / kRows, (int)(q % kRows), q < nrows, inv, p.R, add);
      round_end();
    }
  } else {
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < f.nsampled;
         b0 += (long long)gridDim.x * blockDim.x) {  // uniform trip count over the CTA
      const long long sb = b0 + threadIdx.x;
      sz_est_block<D>(f, sb, sb < f.nsampled, inv, p.R, add, round_end);
      if (D < 3) round_end();
    }
  }
  hot.flush_global(g_hist);
  window_flush(s_win, g_hist);
}

// ---------------------------------------------------------------------------
// Ground truth over every point, with the estimator fused for points of
// sampled blocks when requested.
// ---------------------------------------------------------------------------
template <int D, bool EST>
__global__ void __launch_bounds__(kSzThreads) k_sz_gt(FieldDev f, ParamsDev p, Workspace* ws) {
  __shared__ uint32_t s_gt[kHistWin];
  __shared__ uint32_t s_est[EST ? kHistWin : 1];
  __shared__ double s_sse[kSzThreads / 32];
  __shared__ float s_max[kSzThreads / 32];
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) {
    s_gt[i] = 0u;
    if (EST) s_est[i] = 0u;
  }
  __syncthreads();
  const float w = sc.w, inv = sc.inv, tau = sc.tau;
  const int R = p.R;
  double my_sse = 0.0;
  float my_max = 0.0f;
  for (long long u0 = (long long)blockIdx.x * blockDim.x; u0 < f.N;
       u0 += (long long)gridDim.x * blockDim.x) {
    const long long u = u0 + threadIdx.x;
    const bool ok = u < f.N;
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (!ok) continue;
    int g[3] = {0, 0, 0};
    point_coords<D>(f, u, g);
    Nbr c = gather_cell<D>(f, g);
    const float x = c.v[0];
    const int q = __float2int_rn(__fmul_rn(x, inv));
    const float xh = __fmul_rn(__int2float_rn(q), w);
    const float e = __fsub_rn(x, xh);
    const int r = gt_residual<D>(c, inv);
    const bool esc = fabsf(e) > tau || r >= R || r <= -R;
    hist_add(s_gt, ws->hist[1], esc ? 0 : r + kCenter, mask);
    if (!esc) {
      const double de = (double)e;  // squares of subnormal errors need float64
      my_sse += de * de;
      my_max = fmaxf(my_max, fabsf(e));
    }
    if (EST) {
      const bool smp = in_sampled_block<D>(f, g);
      const unsigned m2 = __ballot_sync(mask, smp);
      if (smp) hist_add(s_est, ws->hist[0], est_symbol(est_residual<D>(c), inv, R), m2);
    }
  }
  // per-CTA partials
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double ss = warp_sum(my_sse);
  float mm = warp_max(my_max);
  if (lane == 0) {
    s_sse[wid] = ss;
    s_max[wid] = mm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    float m = 0.0f;
    for (int i = 0; i < kSzThreads / 32; i++) {
      t += s_sse[i];
      m = fmaxf(m, s_max[i]);
    }
    ws->sz_sse[blockIdx.x] = t;
    atomicMax(&ws->sc.sz_maxerr, __float_as_uint(m));
  }
  hist_flush(s_gt, ws->hist[1]);
  if (EST) hist_flush(s_est, ws->hist[0]);
}

template <int D>
static cudaError_t launch_est_d(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                                cudaStream_t s) {
  // one CTA per SM (ctas); rows as work units when they fill the resident
  // threads at most four times (on a 100x500x500 field 2.1 rounds of rows
  // took 26.5 us against 30.6 for blocks; on 512^3 fields 10.5 rounds of
  // rows took 88 us against 66), else blocks; fewer threads per CTA when
  // there are fewer units than the CTAs' threads, so that every SM takes a
  // share
  const long long nrows = f.nsampled * est_rows<D>();
  const bool rows = nrows <= 4ll * ctas * kSzEstThreads;
  const long long units = rows ? nrows : f.nsampled;
  long long per = (units + ctas - 1) / ctas;
  per = (per + 31) / 32 * 32;
  const int threads = (int)(per < 128 ? 128 : per > kSzEstThreads ? kSzEstThreads : per);
  long long want = (units + threads - 1) / threads;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (rows)
    k_sz_est<D, true><<<g, threads, kPackWords * sizeof(uint32_t), s>>>(f, p, ws);
  else
    k_sz_est<D, false><<<g, threads, kPackWords * sizeof(uint32_t), s>>>(f, p, ws);
  return cudaGetLastError();
}

cudaError_t launch_sz_est(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                          cudaStream_t s) {
  switch (f.d) {
    case 1: return launch_est_d<1>(f, p, ws, ctas, s);
    case 2: return launch_est_d<2>(f, p, ws, ctas, s);
    default: return launch_est_d<3>(f, p, ws, ctas, s);
  }
}

template <int D>
static cudaError_t launch_gt_d(const FieldDev& f, const ParamsDev& p, int with_est, Workspace* ws,
                               int ctas, cudaStream_t s, int* grid_used) {
  long long want = (f.N + kSzThreads - 1) / kSzThreads;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (grid_used) *grid_used = g;
  if (with_est)
    k_sz_gt<D, true><<<g, kSzThreads, 0, s>>>(f, p, ws);
  else
    k_sz_gt<D, false><<<g, kSzThreads, 0, s>>>(f, p, ws);
  return cudaGetLastError();
}

cudaError_t launch_sz_gt(const FieldDev& f, const ParamsDev& p, int with_est, Workspace* ws,
                         int ctas, cudaStream_t s, int* grid_used) {
  switch (f.d) {
    case 1: return launch_gt_d<1>(f, p, with_est, ws, ctas, s, grid_used);
    case 2: return launch_gt_d<2>(f, p, with_est, ws, ctas, s, grid_used);
    default: return launch_gt_d<3>(f, p, with_est, ws, ctas, s, grid_used);
  }
}

cudaError_t prepare_sz_est() {
  const int smem = kPackWords * (int)sizeof(uint32_t);
  const void* fns[6] = {(const void*)k_sz_est<1, false>, (const void*)k_sz_est<2, false>,
                        (const void*)k_sz_est<3, false>, (const void*)k_sz_est<1, true>,
                        (const void*)k_sz_est<2, true>,  (const void*)k_sz_est<3, true>};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; i++)
    e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

int sz_est_occupancy(int d, int num_sms) {
  int per = 0;
  const void* fn = d == 1 ? (const void*)k_sz_est<1, false>
                 : d == 2 ? (const void*)k_sz_est<2, false> : (const void*)k_sz_est<3, false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kSzEstThreads,
                                                    kPackWords * sizeof(uint32_t)) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    per = 1;
  }
  long long g = (long long)per * num_sms;
  return (int)(g > kMaxGrid ? kMaxGrid : g);
}

int sz_occupancy(int d, int num_sms) {
  int per = 0;
  const void* fn = d == 1 ? (const void*)k_sz_gt<1, true>
                 : d == 2 ? (const void*)k_sz_gt<2, true> : (const void*)k_sz_gt<3, true>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kSzThreads, 0) != cudaSuccess || per < 1)
    per = 1;
  long long g = (long long)per * num_sms;
  return (int)(g > kMaxGrid ? kMaxGrid : g);
}

// ---------------------------------------------------------------------------
// Inspector: per-point symbols and reconstruction through the same helpers.
// ---------------------------------------------------------------------------
// With qws, the quantiser (w, 1/w, tau) is the one that workspace holds.
template <int D>
__global__ void k_sz_inspect(FieldDev f, float w, float inv, float tau, int R, int use_strides,
                             int32_t* est_sym, int32_t* gt_sym, float* recon, const Workspace* qws) {
  if (qws) {
    w = qws->sc.w;
    inv = qws->sc.inv;
    tau = qws->sc.tau;
  }
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < f.N;
       u += (long long)gridDim.x * blockDim.x) {
    int g[3] = {0, 0, 0};
    point_coords<D>(f, u, g);
    Nbr c = gather_cell<D>(f, g);
    const float x = c.v[0];
    if (est_sym) est_sym[u] = (use_strides && in_sampled_block<D>(f, g))
                                  ? est_symbol(est_residual<D>(c), inv, R) : -1;
    const int q = __float2int_rn(__fmul_rn(x, inv));
    const float xh = __fmul_rn(__int2float_rn(q), w);
    const float e = __fsub_rn(x, xh);
    const int r = gt_residual<D>(c, inv);
    const bool esc = fabsf(e) > tau || r >= R || r <= -R;
    if (gt_sym) gt_sym[u] = esc ? 0 : r + kCenter;
    if (recon) recon[u] = esc ? x : xh;
  }
}

cudaError_t launch_sz_inspect_q(const FieldDev& f, float w, float inv, float tau, int R,
                                int32_t* est_sym, int32_t* gt_sym, float* recon, int use_strides,
                                cudaStream_t s, const Workspace* qws) {
  long long g = (f.N + 255) / 256;
  if (g > 65535) g = 65535;
  if (g < 1) g = 1;
  switch (f.d) {
    case 1: k_sz_inspect<1><<<(int)g, 256, 0, s>>>(f, w, inv, tau, R, use_strides, est_sym, gt_sym, recon, qws); break;
    case 2: k_sz_inspect<2><<<(int)g, 256, 0, s>>>(f, w, inv, tau, R, use_strides, est_sym, gt_sym, recon, qws); break;
    default: k_sz_inspect<3><<<(int)g, 256, 0, s>>>(f, w, inv, tau, R, use_strides, est_sym, gt_sym, recon, qws); break;
  }
  return cudaGetLastError();
}

}  // namespace rdk
