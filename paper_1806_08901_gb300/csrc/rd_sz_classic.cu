// rd_sz_classic.cu -- classic SZ ground truth (Section "Prediction-Based
// Transformation"): every point is predicted by the Lorenzo predictor from
// the *reconstructed* values of its preceding neighbours, as compression and
// decompression must predict alike; the residual is quantised with bin
// w = 2 eb_sz, and the reconstruction pred + q w is kept when |q| < R and it
// lies within tau of the value, else the value escapes (stored exactly,
// symbol 0).
//
// A point depends on the reconstruction of the points before it on its
// stencil, so the field is walked in wavefronts:
//  * 1D: one chain, one thread, the previous reconstruction in a register;
//  * 2D: tiles of 32 rows x 128 columns, one warp each, lane r taking row r
//    one step behind lane r-1 (its upper neighbours come by shuffle, the
//    tile's halo row and column from the tiles before it); a launch per
//    anti-diagonal of tiles;
//  * 3D: a launch per wavefront i + j + k = s of points, a thread per (i, j).
// The reconstruction is kept in a field-sized buffer; a last pass sums the
// squared errors in fixed order.
#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

constexpr int kClassicThreads = 256;
constexpr int kTileRows = 32;    // one warp: a lane per row
constexpr int kTileCols = 128;

// The code of one point with prediction pred: its symbol, and rec, the
// value a decompressor reconstructs.
__device__ __forceinline__ int classic_code(float x, float pred, float w, float inv, float tau,
                                            float Rf, float& rec) {
  const float q = rintf(__fmul_rn(__fsub_rn(x, pred), inv));
  rec = x;
  if (fabsf(q) < Rf) {
    const float cand = __fadd_rn(pred, __fmul_rn(q, w));
    if (fabsf(__fsub_rn(x, cand)) <= tau) {
      rec = cand;
      return (int)q + kCenter;
    }
  }
  return 0;
}

// One histogram increment per active lane, equal codes of a warp merged
// into one atomic.  Every lane of the warp calls it.
__device__ __forceinline__ void classic_hist(uint32_t* hist, bool act, int sym) {
  const unsigned m = __ballot_sync(0xffffffffu, act);
  if (act) {
    const unsigned same = __match_any_sync(m, sym);
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[sym], (uint32_t)__popc(same));
  }
}

// 1D: pred = 0 + xhat[i-1] (xhat[-1] = 0).
__global__ void k_classic_chain(FieldDev f, ParamsDev p, float* xh, Workspace* ws) {
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  const float w = sc.w, inv = sc.inv, tau = sc.tau, Rf = (float)p.R;
  float prev = 0.0f;
  for (int i = 0; i < f.n[0]; i++) {
    const float pred = __fadd_rn(0.0f, prev);
    float rec;
    const int sym = classic_code(f.x[i], pred, w, inv, tau, Rf, rec);
    xh[i] = rec;
    prev = rec;
    atomicAdd(&ws->hist[1][sym], 1u);
  }
}

// 2D tile (a, b) with a + b = u, a = a_lo + blockIdx.x.  The prediction of
// (i, j) is 0 + xhat(i, j-1) + xhat(i-1, j) - xhat(i-1, j-1), in that order.
// Lane r computes (i0 + r, j0 + t - r) at step t: its left neighbour is its
// own result of step t-1, its upper neighbours lane r-1's results of steps
// t-1 and t-2.
__global__ void __launch_bounds__(kTileRows) k_classic_tile2(FieldDev f, ParamsDev p, int u, int a_lo,
                                                             float* xh, Workspace* ws) {
  __shared__ float s_t[kTileRows][kTileCols + 2];  // the tile (row pitch 130: the skewed
                                                   // accesses of a step fall in 32 banks)
  __shared__ float s_up[kTileCols + 1];             // xhat(i0-1, j0-1+c), c = 0..kTileCols
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  const int lane = threadIdx.x;
  const int a = a_lo + blockIdx.x, b = u - a;
  const int n0 = f.n[0], n1 = f.n[1];
  const int i0 = a * kTileRows, j0 = b * kTileCols;
  const float* __restrict__ x = f.x;
  for (int r = 0; r < kTileRows; r++) {
    const int i = i0 + r;
    if (i >= n0) break;
#pragma unroll
    for (int q = 0; q < kTileCols / 32; q++) {
      const int c = lane + 32 * q, j = j0 + c;
      s_t[r][c] = j < n1 ? x[(long long)i * n1 + j] : 0.0f;
    }
  }
  for (int c = lane; c <= kTileCols; c += 32) {
    const int j = j0 - 1 + c;
    s_up[c] = (i0 > 0 && j >= 0 && j < n1) ? xh[(long long)(i0 - 1) * n1 + j] : 0.0f;
  }
  const int i = i0 + lane;
  const float left0 = (j0 > 0 && i < n0) ? xh[(long long)i * n1 + j0 - 1] : 0.0f;
  float upleft0 = __shfl_up_sync(0xffffffffu, left0, 1);  // xhat(i-1, j0-1)
  __syncwarp();
  if (lane == 0) upleft0 = s_up[0];
  const float w = sc.w, inv = sc.inv, tau = sc.tau, Rf = (float)p.R;
  float last = 0.0f, last2 = 0.0f;  // this lane's results of the two steps before
  for (int t = 0; t < kTileCols + kTileRows - 1; t++) {
    const int c = t - lane;
    const float up_l = __shfl_up_sync(0xffffffffu, last, 1);
    const float ul_l = __shfl_up_sync(0xffffffffu, last2, 1);
    const bool act = c >= 0 && c < kTileCols && i < n0 && j0 + c < n1;
    float rec = 0.0f;
    int sym = 0;
    if (act) {
      const float left = c > 0 ? last : left0;
      const float up = lane > 0 ? up_l : s_up[1 + c];
      const float ul = c == 0 ? upleft0 : lane > 0 ? ul_l : s_up[c];
      float pred = __fadd_rn(0.0f, left);
      pred = __fadd_rn(pred, up);
      pred = __fsub_rn(pred, ul);
      sym = classic_code(s_t[lane][c], pred, w, inv, tau, Rf, rec);
      s_t[lane][c] = rec;
    }
    last2 = last;
    last = rec;
    classic_hist(ws->hist[1], act, sym);
  }
  __syncwarp();
  for (int r = 0; r < kTileRows; r++) {
    const int ii = i0 + r;
    if (ii >= n0) break;
#pragma unroll
    for (int q = 0; q < kTileCols / 32; q++) {
      const int c = lane + 32 * q, j = j0 + c;
      if (j < n1) xh[(long long)ii * n1 + j] = s_t[r][c];
    }
  }
}

// 3D wavefront s: thread t takes (i, j) = (t / n1, t % n1) and k = s - i - j.
// The seven neighbours idx - e for the nonzero subsets e of the axes (bit b
// of e steps back along axis 2-b) are added when e has an odd number of axes
// and subtracted when even, in increasing order of e; outside the field they
// are zero.
__global__ void __launch_bounds__(kClassicThreads) k_classic_wave3(FieldDev f, ParamsDev p, int s,
                                                                   float* xh, Workspace* ws) {
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;  // uniform over the grid
  const int n0 = f.n[0], n1 = f.n[1], n2 = f.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t / n1), j = (int)(t % n1), k = s - i - j;
  const bool act = i < n0 && k >= 0 && k < n2;
  int sym = 0;
  if (act) {
    const long long pl = (long long)n1 * n2;
    const long long l = (long long)i * pl + (long long)j * n2 + k;
    float pred = 0.0f;
#pragma unroll
    for (int e = 1; e < 8; e++) {
      const int di = (e >> 2) & 1, dj = (e >> 1) & 1, dk = e & 1;
      const bool odd = ((di + dj + dk) & 1) != 0;
      const bool inside = i >= di && j >= dj && k >= dk;
      const float v = inside ? xh[l - di * pl - dj * n2 - dk] : 0.0f;
      pred = odd ? __fadd_rn(pred, v) : __fsub_rn(pred, v);
    }
    float rec;
    sym = classic_code(f.x[l], pred, sc.w, sc.inv, sc.tau, (float)p.R, rec);
    xh[l] = rec;
  }
  classic_hist(ws->hist[1], act, sym);
}

// Squared errors (the difference of two floats, exact in double) and the
// largest error against the reconstruction: per-CTA fixed-order partials in
// sz_sse, as the other truth passes leave them.
__global__ void __launch_bounds__(kClassicThreads) k_classic_err(FieldDev f, const float* xh,
                                                                 Workspace* ws) {
  __shared__ double s_sse[kClassicThreads / 32];
  __shared__ float s_max[kClassicThreads / 32];
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  double my_sse = 0.0;
  float my_max = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < f.N;
       i += (long long)gridDim.x * blockDim.x) {
    const double e = (double)f.x[i] - (double)xh[i];
    my_sse += e * e;
    my_max = fmaxf(my_max, (float)fabs(e));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double ss = warp_sum(my_sse);
  const float mm = warp_max(my_max);
  if (lane == 0) {
    s_sse[wid] = ss;
    s_max[wid] = mm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    float m = 0.0f;
    for (int q = 0; q < kClassicThreads / 32; q++) {
      tot += s_sse[q];
      m = fmaxf(m, s_max[q]);
    }
    ws->sz_sse[blockIdx.x] = tot;
    atomicMax(&ws->sc.sz_maxerr, __float_as_uint(m));
  }
}

namespace {
int tiles(int n, int t) { return (n + t - 1) / t; }
}  // namespace

long long classic_launches(const FieldDev& f) {
  if (f.d == 1) return 1;
  if (f.d == 2) return tiles(f.n[0], kTileRows) + tiles(f.n[1], kTileCols) - 1;
  return (long long)f.n[0] + f.n[1] + f.n[2] - 2;
}

cudaError_t launch_classic_waves(const FieldDev& f, const ParamsDev& p, float* xh, Workspace* ws,
                                 cudaStream_t st) {
  if (f.d == 1) {
    k_classic_chain<<<1, 1, 0, st>>>(f, p, xh, ws);
    return cudaGetLastError();
  }
  if (f.d == 2) {
    const int na = tiles(f.n[0], kTileRows), nb = tiles(f.n[1], kTileCols);
    for (int u = 0; u < na + nb - 1; u++) {
      const int a_lo = u - (nb - 1) > 0 ? u - (nb - 1) : 0;
      const int a_hi = u < na - 1 ? u : na - 1;
      k_classic_tile2<<<a_hi - a_lo + 1, kTileRows, 0, st>>>(f, p, u, a_lo, xh, ws);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const int n0 = f.n[0], n1 = f.n[1];
  const int waves = f.n[0] + f.n[1] + f.n[2] - 2;
  for (int s = 0; s < waves; s++) {
    // rows i <= s only
    const long long rows = s + 1 < n0 ? s + 1 : n0;
    const long long th = rows * n1;
    const int g = (int)((th + kClassicThreads - 1) / kClassicThreads);
    k_classic_wave3<<<g, kClassicThreads, 0, st>>>(f, p, s, xh, ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_classic_err(const FieldDev& f, const float* xh, Workspace* ws, int ctas,
                               cudaStream_t st, int* grid_used) {
  const long long want = (f.N + kClassicThreads - 1) / kClassicThreads;
  long long g = want < ctas ? want : ctas;
  if (g < 1) g = 1;
  if (g > kMaxGrid) g = kMaxGrid;
  if (grid_used) *grid_used = (int)g;
  k_classic_err<<<(int)g, kClassicThreads, 0, st>>>(f, xh, ws);
  return cudaGetLastError();
}

}  // namespace rdk
