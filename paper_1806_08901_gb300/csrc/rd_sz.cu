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

#include "rd_device.cuh"

namespace rdk {

constexpr int kSzThreads = 256;

struct Nbr {
  // the 2^D corner values of the Lorenzo cell ending at a point; index bit k
  // set = one step back along axis D-1-k (bit 0 = fastest axis)
  float v[8];
};

template <int D>
__device__ __forceinline__ Nbr gather_cell(const FieldDev& f, const int* g) {
  Nbr c;
  constexpr int NC = 1 << D;
#pragma unroll
  for (int m = 0; m < NC; m++) {
    long long idx = 0;
    bool inside = true;
#pragma unroll
    for (int k = 0; k < D; k++) {
      int back = (m >> (D - 1 - k)) & 1;
      int gk = g[k] - back;
      inside = inside && gk >= 0;
      idx = idx * f.n[k] + gk;
    }
    c.v[m] = inside ? __ldg(f.x + idx) : 0.0f;
  }
  return c;
}

// x - Lorenzo(x) as nested float32 differences, last axis first:
//   1D: v0 - v1
//   2D: (v00 - v01) - (v10 - v11)
//   3D: 2D form on the current plane minus the 2D form on the plane behind.
template <int D>
__device__ __forceinline__ float est_residual(const Nbr& c) {
  if constexpr (D == 1) {
    return __fsub_rn(c.v[0], c.v[1]);
  } else if constexpr (D == 2) {
    return __fsub_rn(__fsub_rn(c.v[0], c.v[1]), __fsub_rn(c.v[2], c.v[3]));
  } else {
    float p0 = __fsub_rn(__fsub_rn(c.v[0], c.v[1]), __fsub_rn(c.v[2], c.v[3]));
    float p1 = __fsub_rn(__fsub_rn(c.v[4], c.v[5]), __fsub_rn(c.v[6], c.v[7]));
    return __fsub_rn(p0, p1);
  }
}

__device__ __forceinline__ int est_symbol(float r, float inv, int R) {
  float q = rintf(__fmul_rn(r, inv));
  return fabsf(q) < (float)R ? (int)q + kCenter : 0;
}

// Integer Lorenzo residual of the prequantised codes: sum over the cell's
// corners of (-1)^(steps back) Q.
template <int D>
__device__ __forceinline__ int gt_residual(const Nbr& c, float inv) {
  int r = 0;
#pragma unroll
  for (int m = 0; m < (1 << D); m++) {
    int q = __float2int_rn(__fmul_rn(c.v[m], inv));
    r += (__popc(m) & 1) ? -q : q;
  }
  return r;
}

template <int D>
__device__ __forceinline__ void point_coords(const FieldDev& f, long long u, int* g) {
  long long r = u;
#pragma unroll
  for (int k = D - 1; k >= 0; k--) {
    g[k] = (int)(r % f.n[k]);
    r /= f.n[k];
  }
}

template <int D>
__device__ __forceinline__ bool in_sampled_block(const FieldDev& f, const int* g) {
  bool s = true;
#pragma unroll
  for (int k = 0; k < D; k++) s = s && (((g[k] >> 2) % f.s[k]) == 0);
  return s;
}

// ---------------------------------------------------------------------------
// Estimator over the points of sampled blocks only: one thread per sampled
// block.  The thread reads the block with its one-cell halo on the low side
// ((4+1)^d values, zero outside the domain), a plane at a time: the 2D
// nested difference of each of the 16 points of a plane, minus that of the
// plane behind, is the 3D residual, in the same float32 operations and
// order as est_residual.
// ---------------------------------------------------------------------------
// Row y of plane z, values x0-1 .. x0+3 (zero outside the domain; values past
// the far edges feed no valid point and read as zero).
__device__ __forceinline__ void load_halo_row(const FieldDev& f, long long row, bool row_ok, int x0,
                                              float* v) {
  const int nx = f.n[f.d - 1];
  if (!row_ok) {
#pragma unroll
    for (int k = 0; k < 5; k++) v[k] = 0.0f;
    return;
  }
  const float* __restrict__ p = f.x + row * nx;
  v[0] = x0 > 0 ? __ldg(p + x0 - 1) : 0.0f;
  if (f.vec_ok && x0 + 4 <= nx) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p + x0));
    v[1] = q.x;
    v[2] = q.y;
    v[3] = q.z;
    v[4] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++) v[k + 1] = x0 + k < nx ? __ldg(p + x0 + k) : 0.0f;
  }
}

// Lattice index of a sampled block -> its first point per axis.
template <int D>
__device__ __forceinline__ void sampled_block_origin(const FieldDev& f, long long sb, int* o) {
  long long r = sb;
#pragma unroll
  for (int k = D - 1; k >= 0; k--) {
    const int l = (int)(r % f.L[k]);
    r /= f.L[k];
    o[k] = 4 * l * f.s[k];
  }
}

template <int D>
__device__ __forceinline__ void sz_est_block(const FieldDev& f, long long sb, bool active, float inv,
                                             int R, uint32_t* s_win, uint32_t* g_hist) {
  int o[3] = {0, 0, 0};
  if (active) sampled_block_origin<D>(f, sb, o);
  if constexpr (D == 1) {
    float v[5];
    load_halo_row(f, 0, active, o[0], v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool ok = active && o[0] + k < f.n[0];
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) hist_add(s_win, g_hist, est_symbol(__fsub_rn(v[k + 1], v[k]), inv, R), mask);
    }
  } else {
    const int ny = f.n[D - 2], nx = f.n[D - 1];
    const int y0 = o[D - 2], x0 = o[D - 1];
    // 2D nested differences of the 16 points of plane z (rows y0-1 .. y0+3)
    auto plane = [&](int z, bool z_ok, float* d2) {
      float v[5][5];
#pragma unroll
      for (int r = 0; r < 5; r++) {
        const int y = y0 - 1 + r;
        const bool ok = z_ok && y >= 0 && y < ny;
        const long long row = (D == 3 ? (long long)z * ny : 0ll) + y;
        load_halo_row(f, row, ok, x0, v[r]);
      }
#pragma unroll
      for (int j = 0; j < 4; j++)
#pragma unroll
        for (int k = 0; k < 4; k++)
          d2[4 * j + k] = __fsub_rn(__fsub_rn(v[j + 1][k + 1], v[j + 1][k]),
                                    __fsub_rn(v[j][k + 1], v[j][k]));
    };
    float prev[16];
    const int nz = D == 3 ? f.n[0] : 1;
    const int z0 = D == 3 ? o[0] : 0;
    if (D == 3) plane(z0 - 1, active && z0 > 0, prev);
#pragma unroll 1
    for (int i = 0; i < (D == 3 ? 4 : 1); i++) {
      const int z = z0 + i;
      const bool z_ok = active && z < nz;
      float cur[16];
      plane(z, z_ok, cur);
#pragma unroll
      for (int t = 0; t < 16; t++) {
        const int j = t >> 2, k = t & 3;
        const bool ok = z_ok && y0 + j < ny && x0 + k < nx;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        const float r = D == 3 ? __fsub_rn(cur[t], prev[t]) : cur[t];
        if (ok) hist_add(s_win, g_hist, est_symbol(r, inv, R), mask);
      }
      if (D == 3) {
#pragma unroll
        for (int t = 0; t < 16; t++) prev[t] = cur[t];
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kSzThreads) k_sz_est(FieldDev f, ParamsDev p, Workspace* ws) {
  __shared__ uint32_t s_win[kHistWin];
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) s_win[i] = 0u;
  __syncthreads();
  const float inv = sc.inv;
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < f.nsampled;
       b0 += (long long)gridDim.x * blockDim.x) {
    const long long sb = b0 + threadIdx.x;
    sz_est_block<D>(f, sb, sb < f.nsampled, inv, p.R, s_win, ws->hist[0]);
  }
  __syncthreads();
  hist_flush(s_win, ws->hist[0]);
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
  long long want = (f.nsampled + kSzThreads - 1) / kSzThreads;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  k_sz_est<D><<<g, kSzThreads, 0, s>>>(f, p, ws);
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
// Batched estimate: the sampled blocks of many fields.  Each work item is a
// run of sampled blocks of one field; its histogram window lives in shared
// memory and is added to the field's histogram when the item ends.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void sz_est_item(const FieldDev& f, int R, float inv, uint32_t* g_hist,
                                            long long u0, long long u1, uint32_t* s_win) {
  for (long long b0 = u0; b0 < u1; b0 += blockDim.x) {
    const long long sb = b0 + threadIdx.x;
    sz_est_block<D>(f, sb, sb < u1, inv, R, s_win, g_hist);
  }
}

__global__ void __launch_bounds__(kSzThreads) k_batch_sz_est(const BatchField* __restrict__ bf,
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

cudaError_t launch_batch_sz_est(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                cudaStream_t s) {
  int g = nitems < ctas ? nitems : ctas;
  if (g < 1) g = 1;
  k_batch_sz_est<<<g, kSzThreads, 0, s>>>(bf, items, nitems);
  return cudaGetLastError();
}

int batch_sz_occupancy(int num_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_batch_sz_est, kSzThreads, 0) !=
          cudaSuccess ||
      per < 1)
    per = 1;
  return per * num_sms;
}

// ---------------------------------------------------------------------------
// Inspector: per-point symbols and reconstruction through the same helpers.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_sz_inspect(FieldDev f, float w, float inv, float tau, int R, int use_strides,
                             int32_t* est_sym, int32_t* gt_sym, float* recon) {
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
                                cudaStream_t s) {
  long long g = (f.N + 255) / 256;
  if (g > 65535) g = 65535;
  if (g < 1) g = 1;
  switch (f.d) {
    case 1: k_sz_inspect<1><<<(int)g, 256, 0, s>>>(f, w, inv, tau, R, use_strides, est_sym, gt_sym, recon); break;
    case 2: k_sz_inspect<2><<<(int)g, 256, 0, s>>>(f, w, inv, tau, R, use_strides, est_sym, gt_sym, recon); break;
    default: k_sz_inspect<3><<<(int)g, 256, 0, s>>>(f, w, inv, tau, R, use_strides, est_sym, gt_sym, recon); break;
  }
  return cudaGetLastError();
}

}  // namespace rdk
