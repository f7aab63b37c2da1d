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
//  * 2D and 3D: tiles of 32 rows x 32 columns of one plane, one warp each,
//    lane r taking row r one step behind lane r-1 (its upper neighbours come
//    by shuffle, the tile's halo row and column and the previous plane from
//    the tiles before it); a launch per wavefront of tiles, plane + row tile
//    + column tile = w.
// The reconstruction is kept in a field-sized buffer; a last pass sums the
// squared errors in fixed order.
#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

constexpr int kClassicThreads = 256;
constexpr int kTileRows = 32;    // one warp: a lane per row
constexpr int kTileWin = 256;   // per-tile shared histogram of the codes near zero
constexpr int kTileCols = 32;   // the tile wavefront's critical path is
                                 // (planes + row tiles + column tiles) x
                                 // (rows + columns of a tile) steps

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

// Four bytes from global to shared memory without a register round trip
// (cp.async); zeros when !valid (source size 0: nothing is read, src only
// has to be a valid address).  All of a tile's copies are in flight at once.
__device__ __forceinline__ void copy4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void copy_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

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

// A tile of 32 rows x 32 columns of one plane (3D: plane p along axis 0,
// rows along axis 1, columns along axis 2; 2D: the one plane), one warp.
// Lane r computes (row i0 + r, column j0 + t - r) at step t: its left
// neighbour is its own result of step t-1, its upper and upper-left
// neighbours lane r-1's results of steps t-1 and t-2; the tile's halo row
// and column, and in 3D the previous plane, come from tiles finished by
// earlier launches.  The prediction adds the neighbours in the order of the
// subsets e = 1 .. 2^D - 1 (bit b of e steps back along axis D-1-b): left,
// up, -upper-left, and in 3D then +P, -P left, -P up, +P upper-left from
// the previous plane.  The tiles of one launch are those with p + a + b = w
// (2D: a = a_lo + blockIdx.x, b = w - a; 3D: (a, b) from blockIdx.x, the
// others return at once).
template <int D>
__global__ void __launch_bounds__(kTileRows) k_classic_tile(FieldDev f, ParamsDev p, int w, int a_lo,
                                                            float* xh, Workspace* ws) {
  constexpr int kPitch = kTileCols + 2;  // 34: the skewed accesses of a step hit 32 banks
  __shared__ float s_x[kTileRows][kPitch];                       // values, then reconstructions
  __shared__ float s_prev[D == 3 ? kTileRows + 1 : 1][kPitch];   // 3D: plane p-1, rows i0-1..,
                                                                 // columns j0-1..
  __shared__ unsigned short s_sym[kTileRows][kPitch];
  __shared__ float s_up[kTileCols + 1];  // xhat of row i0-1, columns j0-1 ..
  __shared__ unsigned s_win[kTileWin];   // codes |q| < kTileWin / 2 of the tile
  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  const int nr = f.n[D - 2], nc = f.n[D - 1];
  int a, b, pl;
  if (D == 3) {
    const int nb = (nc + kTileCols - 1) / kTileCols;
    a = blockIdx.x / nb;
    b = blockIdx.x - a * nb;
    pl = w - a - b;
    if (pl < 0 || pl >= f.n[0]) return;  // uniform over the CTA
  } else {
    a = a_lo + blockIdx.x;
    b = w - a;
    pl = 0;
  }
  const int lane = threadIdx.x;
  const int i0 = a * kTileRows, j0 = b * kTileCols;
  const long long plane = (long long)nr * nc;
  const long long base = (long long)pl * plane;
  const float* __restrict__ x = f.x + base;
  float* xp = xh + base;
  // the tile, its halo row and (3D) the previous plane: every copy issued
  // before the first wait; out-of-field cells read as zero
  for (int r = 0; r < kTileRows; r++) {
    const int i = i0 + r;
#pragma unroll
    for (int q = 0; q < kTileCols / 32; q++) {
      const int c = lane + 32 * q, j = j0 + c;
      const bool ok = i < nr && j < nc;
      copy4(&s_x[r][c], ok ? x + (long long)i * nc + j : x, ok);
    }
  }
  for (int c = lane; c <= kTileCols; c += 32) {
    const int j = j0 - 1 + c;
    const bool ok = i0 > 0 && j >= 0 && j < nc;
    copy4(&s_up[c], ok ? xp + (long long)(i0 - 1) * nc + j : xp, ok);
  }
  if (D == 3) {
    const float* pp = pl > 0 ? xp - plane : xp;
    for (int r = 0; r <= kTileRows; r++) {
      const int i = i0 - 1 + r;
      for (int c = lane; c <= kTileCols; c += 32) {
        const int j = j0 - 1 + c;
        const bool ok = pl > 0 && i >= 0 && i < nr && j >= 0 && j < nc;
        copy4(&s_prev[r][c], ok ? pp + (long long)i * nc + j : xp, ok);
      }
    }
  }
  const int i = i0 + lane;
  const bool row_ok = i < nr;
  const float left0 = (j0 > 0 && row_ok) ? xp[(long long)i * nc + j0 - 1] : 0.0f;
  float upleft0 = __shfl_up_sync(0xffffffffu, left0, 1);  // xhat(i-1, j0-1)
  for (int k = lane; k < kTileWin; k += 32) s_win[k] = 0u;
  copy_wait_all();
  __syncwarp();
  if (lane == 0) upleft0 = s_up[0];
  const float w_ = sc.w, inv = sc.inv, tau = sc.tau, Rf = (float)p.R;
  float last = 0.0f, last2 = 0.0f;  // this lane's results of the two steps before
  for (int t = 0; t < kTileCols + kTileRows - 1; t++) {
    const int c = t - lane;
    const float up_l = __shfl_up_sync(0xffffffffu, last, 1);
    const float ul_l = __shfl_up_sync(0xffffffffu, last2, 1);
    const bool act = c >= 0 && c < kTileCols && row_ok && j0 + c < nc;
    float rec = 0.0f;
    if (act) {
      const float left = c > 0 ? last : left0;
      const float up = lane > 0 ? up_l : s_up[1 + c];
      const float ul = c == 0 ? upleft0 : lane > 0 ? ul_l : s_up[c];
      float pred = __fadd_rn(0.0f, left);
      pred = __fadd_rn(pred, up);
      pred = __fsub_rn(pred, ul);
      if (D == 3) {
        pred = __fadd_rn(pred, s_prev[lane + 1][c + 1]);
        pred = __fsub_rn(pred, s_prev[lane + 1][c]);
        pred = __fsub_rn(pred, s_prev[lane][c + 1]);
        pred = __fadd_rn(pred, s_prev[lane][c]);
      }
      const int sym = classic_code(s_x[lane][c], pred, w_, inv, tau, Rf, rec);
      s_sym[lane][c] = (unsigned short)sym;
      s_x[lane][c] = rec;
    }
    last2 = last;
    last = rec;
  }
  __syncwarp();
  // reconstructions out, row by row; the codes: equal codes of 32 merged,
  // those near zero counted in shared memory (every tile of a launch hits
  // the same few hot codes), the rest with global atomics
  constexpr int kWinLo = kCenter - kTileWin / 2;
  for (int r = 0; r < kTileRows; r++) {
    const int ii = i0 + r;
    if (ii >= nr) break;
#pragma unroll
    for (int q = 0; q < kTileCols / 32; q++) {
      const int c = lane + 32 * q;
      const bool ok = j0 + c < nc;
      if (ok) xp[(long long)ii * nc + j0 + c] = s_x[r][c];
      const int sym = ok ? (int)s_sym[r][c] : 0;
      const bool inw = ok && (unsigned)(sym - kWinLo) < (unsigned)kTileWin;
      const unsigned mw = __ballot_sync(0xffffffffu, inw);
      if (inw) {
        const unsigned same = __match_any_sync(mw, sym);
        if (lane == __ffs(same) - 1) atomicAdd(&s_win[sym - kWinLo], (unsigned)__popc(same));
      }
      classic_hist(ws->hist[1], ok && !inw, sym);
    }
  }
  __syncwarp();
  for (int k = lane; k < kTileWin; k += 32) {
    const unsigned v = s_win[k];
    if (v) atomicAdd(&ws->hist[1][kWinLo + k], v);
  }
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
  const int na = tiles(f.n[f.d - 2], kTileRows), nb = tiles(f.n[f.d - 1], kTileCols);
  return (long long)(f.d == 3 ? f.n[0] : 1) + na + nb - 2;
}

cudaError_t launch_classic_waves(const FieldDev& f, const ParamsDev& p, float* xh, Workspace* ws,
                                 cudaStream_t st) {
  if (f.d == 1) {
    k_classic_chain<<<1, 1, 0, st>>>(f, p, xh, ws);
    return cudaGetLastError();
  }
  const int na = tiles(f.n[f.d - 2], kTileRows), nb = tiles(f.n[f.d - 1], kTileCols);
  const long long waves = classic_launches(f);
  for (long long w = 0; w < waves; w++) {
    if (f.d == 2) {
      const int a_lo = w - (nb - 1) > 0 ? (int)w - (nb - 1) : 0;
      const int a_hi = w < na - 1 ? (int)w : na - 1;
      k_classic_tile<2><<<a_hi - a_lo + 1, kTileRows, 0, st>>>(f, p, (int)w, a_lo, xh, ws);
    } else {
      k_classic_tile<3><<<na * nb, kTileRows, 0, st>>>(f, p, (int)w, 0, xh, ws);
    }
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
