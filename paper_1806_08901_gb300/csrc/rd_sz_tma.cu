// rd_sz_tma.cu -- the SZ pass over every point as a TMA-fed march (fields
// whose rows are 16-byte aligned; others take the gather kernel in rd_sz.cu).
//
// A field is walked as (Z, Y, X): 3D fields as they are, 2D fields as
// (rows, 1, cols).  A CTA owns an X x Y tile and marches down a chunk of Z;
// each step is one or more planes of the tile plus a one-element halo on the
// low sides (x0-1, y0-1) brought into shared memory by cp.async.bulk.tensor
// with mbarrier completion, several steps in flight.  Out-of-range elements
// are zero-filled by the tensor copy, which is exactly the zero padding of
// the Lorenzo stencil.  The first plane of a chunk is its z-1 halo.
//
// Per point (Section "Prediction-Based Transformation"; Eq. psnr-sz bound):
//   ground truth: Q = rint(x / w) in float, reconstruction float(Q) * w,
//     escape if the float error exceeds tau or the integer Lorenzo residual
//     d3 = dz dy dx Q reaches R; residual symbol histogram, SSE, max error;
//   estimator (points of sampled blocks): the float residual as nested
//     differences, last axis first, code rint(r * (1/w)), symbol histogram.
// The mixed differences are carried in registers: along x from the plane in
// shared memory, along y from the thread's previous row, along z from the
// thread's previous plane.
#include <cuda.h>
#include <stdint.h>

#include "rd_device.cuh"
#include "rd_tma.cuh"

namespace rdk {

struct MarchGeom {
  int X, Y, Z;        // extents, x fastest
  int sX, sY, sZ;     // block sampling strides along each walked axis
  int tilesX, tilesY, chunksZ, ZC;
  long long ntiles;
};

// Shared histogram windows of the ground truth and of the estimator; codes
// outside a window go to the global histogram.  Their sizes and the stages
// fit four CTAs per SM: the ground truth codes every point, the estimator
// only the sampled ones, so the estimator's window is the small one.
constexpr int kGtWin = 8192;
constexpr int kGtWinLo = kCenter - kGtWin / 2;
constexpr int kEstWin = 1024;
constexpr int kEstWinLo = kCenter - kEstWin / 2;
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

// TY > 1: 3D fields, a (TY+1)-row plane with the y0-1 halo row, rank-3 map.
// TY == 1: 2D fields walked row by row, no y axis: the row above is zero and
// the stage holds PZ consecutive rows from a rank-2 map.
template <int TX, int TY, int R, int PZ, int NST>
struct MarchCfg {
  static constexpr int kHY = TY > 1 ? 1 : 0;           // halo row in shared memory
  static constexpr int kThreads = TX * (TY / R);
  static constexpr int kRowW = TX + 4;                 // x0-4 .. x0+TX-1
  static constexpr int kPlane = (TY + kHY) * kRowW;    // floats per plane
  static constexpr int kStageBytes = PZ * kPlane * 4;
  static constexpr int kStageStride = (kStageBytes + 127) / 128 * 128;
  static constexpr int kSmem = NST * kStageStride + (kGtWin + kEstWin) * 4 + 128;
};

// Per-thread march state: the previous plane's y-x differences of the codes
// (integer) and of the values (float) for each of the thread's R rows.
template <int R>
struct MarchState {
  int d2pp[R];
  float p0pp[R];
  float ssum, scomp, emax;
  float tiny;  // squares of the tiny errors, at scale (scl * 2^64)^2
  unsigned esc_gt, esc_est;
};

// One plane of a tile for one thread.  FAST: every |x / w| < 2^22, so codes
// are rounded with the 1.5 * 2^23 constant (exactly rint) and need no
// conversion instructions; otherwise the conversion instructions are used.
template <int TX, int TY, int R, int PZ, int NST, bool EST, bool FAST>
__device__ __forceinline__ void march_plane(const float* plane, MarchState<R>& ms, bool halo,
                                            bool xin, int yvalid, bool xz_samp, unsigned ysamp,
                                            float w, float inv, float tau, float scl, int Rq,
                                            uint32_t* s_gt, uint32_t* s_est, Workspace* ws) {
  using Cfg = MarchCfg<TX, TY, R, PZ, NST>;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int yr0 = ty * R;
  auto quant = [&](float v, float& qf) -> int {
    const float t = __fmul_rn(v, inv);
    if (FAST) return round_small(t, qf);
    const int q = __float2int_rn(t);
    qf = __int2float_rn(q);
    return q;
  };
  float vprev = 0.0f, vwprev = 0.0f;
  if (Cfg::kHY) {
    const float* rowp = plane + yr0 * Cfg::kRowW + 4 + tx;  // the row above the strip
    vprev = rowp[0];
    vwprev = rowp[-1];
  }
  float qfd;
  int d1prev = quant(vprev, qfd) - quant(vwprev, qfd);
  float rfprev = __fsub_rn(vprev, vwprev);
  float blocksum = 0.0f;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const float* rp = plane + (yr0 + r + Cfg::kHY) * Cfg::kRowW + 4 + tx;
    const float v = rp[0];
    const float vw = rp[-1];
    float qf, qwf;
    const int q = quant(v, qf);
    const int d1 = q - quant(vw, qwf);
    const float rf = __fsub_rn(v, vw);
    const int d2 = d1 - d1prev;
    const float p0 = __fsub_rn(rf, rfprev);
    d1prev = d1;
    rfprev = rf;
    if (!halo && xin && r < yvalid) {
      const int d3 = d2 - ms.d2pp[r];
      const float xh = __fmul_rn(qf, w);
      const float e = __fsub_rn(v, xh);
      const bool esc = fabsf(e) > tau || d3 >= Rq || d3 <= -Rq;
      if (esc) {
        ms.esc_gt++;
      } else {
        const int sym = d3 + kCenter;
        const int wi = sym - kGtWinLo;
        if ((unsigned)wi < (unsigned)kGtWin)
          atomicAdd(&s_gt[wi], 1u);
        else
          atomicAdd(&ws->hist[1][sym], 1u);
        ms.emax = fmaxf(ms.emax, fabsf(e));
        // squares in float at two power-of-two scales: errors within 2^-60
        // of tau at scl, smaller ones at scl * 2^64 (no float64 per point)
        const float es = __fmul_rn(e, scl);
        const bool big = fabsf(es) >= 8.673617e-19f;  // 2^-60
        const float et = __fmul_rn(es, 1.8446744e19f);  // 2^64
        blocksum = __fadd_rn(blocksum, big ? __fmul_rn(es, es) : 0.0f);
        ms.tiny = __fadd_rn(ms.tiny, big ? 0.0f : __fmul_rn(et, et));
      }
      if (EST && xz_samp && ((ysamp >> r) & 1u)) {
        const float t = __fmul_rn(__fsub_rn(p0, ms.p0pp[r]), inv);
        bool ok;
        int qe;
        if (FAST) {
          ok = fabsf(t) < 4194304.0f;  // beyond 2^22 the code escapes anyway
          float dummy;
          qe = ok ? round_small(t, dummy) : 0;
          ok = ok && qe < Rq && qe > -Rq;
        } else {
          const float qq = rintf(t);
          ok = fabsf(qq) < (float)Rq;
          qe = ok ? (int)qq : 0;
        }
        if (ok) {
          const int sym = qe + kCenter;
          const int wi = sym - kEstWinLo;
          if ((unsigned)wi < (unsigned)kEstWin)
            atomicAdd(&s_est[wi], 1u);
          else
            atomicAdd(&ws->hist[0][sym], 1u);
        } else {
          ms.esc_est++;
        }
      }
    }
    ms.d2pp[r] = d2;
    ms.p0pp[r] = p0;
  }
  // Kahan-compensated accumulation of the per-plane subtotals
  const float yk = __fsub_rn(blocksum, ms.scomp);
  const float tk = __fadd_rn(ms.ssum, yk);
  ms.scomp = __fsub_rn(__fsub_rn(tk, ms.ssum), yk);
  ms.ssum = tk;
}

template <int TX, int TY, int R, int PZ, int NST, bool EST>
__global__ void __launch_bounds__(MarchCfg<TX, TY, R, PZ, NST>::kThreads)
    k_sz_march(const __grid_constant__ CUtensorMap tmap, MarchGeom g, ParamsDev p, Workspace* ws) {
  using Cfg = MarchCfg<TX, TY, R, PZ, NST>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* stages = reinterpret_cast<float*>(smem);
  uint32_t* s_gt = reinterpret_cast<uint32_t*>(smem + NST * Cfg::kStageStride);
  uint32_t* s_est = s_gt + kGtWin;
  __shared__ uint64_t bars[NST];
  __shared__ double s_red[Cfg::kThreads / 32];
  __shared__ float s_fred[Cfg::kThreads / 32];
  __shared__ unsigned long long s_esc[2];
  __shared__ int s_abort;

  const Scalars& sc = ws->sc;
  if (sc.status != RD_OK || sc.constant) return;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const float w = sc.w, inv = sc.inv, tau = sc.tau;
  const int Rq = p.R;
  const bool fast = __fmul_rn(sc.amax, inv) < 4194304.0f;  // every |x / w| < 2^22
  // power-of-two scale putting tau near [1, 2): squares of errors far below
  // tau stay in float range
  const unsigned Et = (__float_as_uint(tau) >> 23) & 0xffu;
  const int ksc = max(-126, 127 - (int)(Et ? Et : 1u));
  const float scl = pow2f(ksc);

  for (int i = tid; i < kGtWin; i += Cfg::kThreads) s_gt[i] = 0u;
  for (int i = tid; i < kEstWin; i += Cfg::kThreads) s_est[i] = 0u;
  if (tid < 2) s_esc[tid] = 0ull;
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < NST; i++) mbar_init(&bars[i], 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int G = (g.ZC + 1 + PZ - 1) / PZ;  // steps per tile (chunk + halo plane)
  const long long mytiles =
      blockIdx.x < g.ntiles ? (g.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long J = mytiles * G;

  // tile of the CTA's lt-th assignment (32-bit: fields hold < 2^31 points)
  auto tile_coords = [&](int lt, int& x0, int& y0, int& zc0, int& zc1) {
    const int t = (int)blockIdx.x + lt * (int)gridDim.x;
    const int itx = t % g.tilesX;
    const int rest = t / g.tilesX;
    const int ity = rest % g.tilesY;
    const int icz = rest / g.tilesY;
    x0 = itx * TX;
    y0 = ity * TY;
    zc0 = icz * g.ZC;
    zc1 = min(zc0 + g.ZC, g.Z);
  };
  auto item_coords = [&](long long j, int& x0, int& y0, int& zc0, int& zc1, int& gi) {
    gi = (int)(j % G);
    tile_coords((int)(j / G), x0, y0, zc0, zc1);
  };
  auto issue = [&](long long j) {
    int x0, y0, zc0, zc1, gi;
    item_coords(j, x0, y0, zc0, zc1, gi);
    const int st = (int)(j % NST);
    mbar_expect_tx(&bars[st], (uint32_t)Cfg::kStageBytes);
    if (Cfg::kHY)
      tma_load_3d(stages + st * (Cfg::kStageStride / 4), &tmap, x0 - 4, y0 - 1, zc0 - 1 + gi * PZ,
                  &bars[st]);
    else
      tma_load_2d(stages + st * (Cfg::kStageStride / 4), &tmap, x0 - 4, zc0 - 1 + gi * PZ, &bars[st]);
  };
  if (tid == 0) {
    for (long long j = 0; j < J && j < NST; j++) issue(j);
  }

  MarchState<R> ms;
#pragma unroll
  for (int r = 0; r < R; r++) {
    ms.d2pp[r] = 0;
    ms.p0pp[r] = 0.0f;
  }
  ms.ssum = ms.scomp = ms.emax = 0.0f;
  ms.tiny = 0.0f;
  ms.esc_gt = ms.esc_est = 0u;
  // tile-constant per-thread facts, refreshed when a tile starts
  bool xin = false, xsamp = false;
  int yvalid = 0;
  unsigned ysamp = 0u;
  int zmod = 0;  // (z >> 2) mod sZ of the current plane

  long long j = 0;
  int gi = 0, lt = 0;  // step within the tile, tile ordinal: advanced incrementally
  int x0 = 0, y0 = 0, zc0 = 0, zc1 = 0;
  for (; j < J; j++) {
    const int st = (int)(j % NST);
    const uint32_t parity = (uint32_t)((j / NST) & 1);
    // every thread waits for the stage itself; a wait that runs out marks
    // the call failed, and the CTA leaves at the barrier below (the planes
    // it counts meanwhile do not matter: the call's results are discarded)
    if (!mbar_wait(&bars[st], parity)) {
      atomicCAS((int*)&ws->sc.status, RD_OK, RD_ERR_TIMEOUT);
      s_abort = 1;
    }
    if (gi == 0) {
      tile_coords(lt, x0, y0, zc0, zc1);
      const int x = x0 + tx;
      xin = x < g.X;
      xsamp = ((x >> 2) % g.sX) == 0;
      const int yb = y0 + ty * R;
      yvalid = min(R, max(0, g.Y - yb));
      ysamp = 0u;
#pragma unroll
      for (int r = 0; r < R; r++)
        if ((((yb + r) >> 2) % g.sY) == 0) ysamp |= 1u << r;
      zmod = (zc0 >> 2) % g.sZ;
    }
    const float* sbase = stages + st * (Cfg::kStageStride / 4);
#pragma unroll
    for (int pz = 0; pz < PZ; pz++) {
      const int z = zc0 - 1 + gi * PZ + pz;
      if (z >= zc1) break;
      const bool halo = (z == zc0 - 1);
      if (!halo && z > zc0 && (z & 3) == 0) zmod = (zmod + 1 == g.sZ) ? 0 : zmod + 1;
      const bool xz = xsamp && zmod == 0;
      const float* plane = sbase + pz * Cfg::kPlane;
      if (fast)
        march_plane<TX, TY, R, PZ, NST, EST, true>(plane, ms, halo, xin, yvalid, xz, ysamp, w, inv,
                                                   tau, scl, Rq, s_gt, s_est, ws);
      else
        march_plane<TX, TY, R, PZ, NST, EST, false>(plane, ms, halo, xin, yvalid, xz, ysamp, w,
                                                    inv, tau, scl, Rq, s_gt, s_est, ws);
    }
    __syncthreads();  // every thread is done with this stage
    if (s_abort) break;  // copies j .. j + NST - 1 may still be in flight
    if (tid == 0 && j + NST < J) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j + NST);
    }
    if (++gi == G) {
      gi = 0;
      lt++;
    }
  }
  if (s_abort && tid == 0) {
    // bounded wait for copies still in flight before the CTA leaves
    for (long long k = j; k < J && k < j + NST; k++) mbar_wait(&bars[k % NST], (uint32_t)((k / NST) & 1));
  }

  // reductions: SSE (fixed order), max error, escapes, histogram windows
  double sse = ((double)ms.ssum - (double)ms.scomp) *
                   __longlong_as_double((long long)(1023 - 2 * ksc) << 52) +
               (double)ms.tiny * __longlong_as_double((long long)(1023 - 2 * ksc - 128) << 52);
  sse = warp_sum(sse);
  const float mm = warp_max(ms.emax);
  const unsigned eg = warp_sum(ms.esc_gt);
  const unsigned ee = warp_sum(ms.esc_est);
  if ((tid & 31) == 0) {
    s_red[tid >> 5] = sse;
    s_fred[tid >> 5] = mm;
    if (eg) atomicAdd(&s_esc[0], (unsigned long long)eg);
    if (ee) atomicAdd(&s_esc[1], (unsigned long long)ee);
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    float m = 0.0f;
    for (int i = 0; i < Cfg::kThreads / 32; i++) {
      t += s_red[i];
      m = fmaxf(m, s_fred[i]);
    }
    ws->sz_sse[blockIdx.x] = t;
    atomicMax(&ws->sc.sz_maxerr, __float_as_uint(m));
    if (s_esc[0]) atomicAdd(&ws->hist[1][0], (unsigned)s_esc[0]);
    if (EST && s_esc[1]) atomicAdd(&ws->hist[0][0], (unsigned)s_esc[1]);
  }
  for (int i = tid; i < kGtWin; i += Cfg::kThreads)
    if (s_gt[i]) atomicAdd(&ws->hist[1][kGtWinLo + i], s_gt[i]);
  if (EST)
    for (int i = tid; i < kEstWin; i += Cfg::kThreads)
      if (s_est[i]) atomicAdd(&ws->hist[0][kEstWinLo + i], s_est[i]);
}

// ---------------------------------------------------------------------------
// Host side: tensor map, tiling, grid.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 3D fields: 64 x 16 tiles, 4 rows per thread, two planes per step, two
// steps in flight (one barrier per step); 55 KB of shared memory per CTA,
// four CTAs per SM.
// 2D fields (walked as rows x 1 x cols): 128-column tiles, 16 rows per step
// (a tensor box spans at most 256 elements per axis).
constexpr int k3TX = 64, k3TY = 16, k3R = 4, k3PZ = 2, k3NST = 2;
using Cfg3 = MarchCfg<k3TX, k3TY, k3R, k3PZ, k3NST>;
using Cfg2 = MarchCfg<128, 1, 1, 16, 4>;

template <int TX, int TY, int R, int PZ, int NST, bool EST>
static cudaError_t set_smem() {
  using Cfg = MarchCfg<TX, TY, R, PZ, NST>;
  return cudaFuncSetAttribute(k_sz_march<TX, TY, R, PZ, NST, EST>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
}

cudaError_t prepare_sz_march() {
  cudaError_t e = set_smem<k3TX, k3TY, k3R, k3PZ, k3NST, true>();
  if (e == cudaSuccess) e = set_smem<k3TX, k3TY, k3R, k3PZ, k3NST, false>();
  if (e == cudaSuccess) e = set_smem<128, 1, 1, 16, 4, true>();
  if (e == cudaSuccess) e = set_smem<128, 1, 1, 16, 4, false>();
  return e;
}

bool sz_march_supported(const FieldDev& f) {
  return f.d >= 2 && f.vec_ok && encode_fn() != nullptr;
}

template <int TX, int TY, int R, int PZ, int NST, bool EST>
static int march_ctas(int num_sms) {
  using Cfg = MarchCfg<TX, TY, R, PZ, NST>;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sz_march<TX, TY, R, PZ, NST, EST>,
                                                    Cfg::kThreads, Cfg::kSmem) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    per = 1;
  }
  long long g = (long long)per * num_sms;
  return (int)(g > kMaxGrid ? kMaxGrid : g);
}

cudaError_t launch_sz_march(const FieldDev& f, const ParamsDev& p, int with_est, Workspace* ws,
                            int num_sms, cudaStream_t s, int* grid_used) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  MarchGeom g;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  int TX, TY, PZ;
  if (f.d == 3) {
    g.Z = f.n[0]; g.Y = f.n[1]; g.X = f.n[2];
    g.sZ = f.s[0]; g.sY = f.s[1]; g.sX = f.s[2];
    TX = k3TX; TY = k3TY; PZ = k3PZ;
  } else {
    g.Z = f.n[0]; g.Y = 1; g.X = f.n[1];
    g.sZ = f.s[0]; g.sY = 1; g.sX = f.s[1];
    TX = 128; TY = 1; PZ = 16;
  }
  cuuint32_t rank;
  if (f.d == 3) {  // (x, y, z) with the y0-1 halo row in the box
    rank = 3;
    dims[0] = (cuuint64_t)g.X;
    dims[1] = (cuuint64_t)g.Y;
    dims[2] = (cuuint64_t)g.Z;
    strides[0] = (cuuint64_t)g.X * 4;
    strides[1] = (cuuint64_t)g.X * g.Y * 4;
    box[0] = (cuuint32_t)(TX + 4);
    box[1] = (cuuint32_t)(TY + 1);
    box[2] = (cuuint32_t)PZ;
  } else {  // (x, row): PZ rows per step
    rank = 2;
    dims[0] = (cuuint64_t)g.X;
    dims[1] = (cuuint64_t)g.Z;
    strides[0] = (cuuint64_t)g.X * 4;
    box[0] = (cuuint32_t)(TX + 4);
    box[1] = (cuuint32_t)PZ;
  }
  alignas(64) CUtensorMap map;
  CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(f.x), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  g.tilesX = (g.X + TX - 1) / TX;
  g.tilesY = (g.Y + TY - 1) / TY;
  const long long xy = (long long)g.tilesX * g.tilesY;
  int ctas = 0;
  if (f.d == 3)
    ctas = with_est ? march_ctas<k3TX, k3TY, k3R, k3PZ, k3NST, true>(num_sms)
                    : march_ctas<k3TX, k3TY, k3R, k3PZ, k3NST, false>(num_sms);
  else
    ctas = with_est ? march_ctas<128, 1, 1, 16, 4, true>(num_sms) : march_ctas<128, 1, 1, 16, 4, false>(num_sms);
  // z chunks: enough tiles to fill the resident CTAs about twice, each chunk
  // long enough that its halo plane stays a small overhead
  int chunks = (int)((2LL * ctas + xy - 1) / xy);
  if (chunks < 1) chunks = 1;
  int zc = (g.Z + chunks - 1) / chunks;
  if (zc < 16) zc = g.Z < 16 ? g.Z : 16;
  g.ZC = zc;
  g.chunksZ = (g.Z + zc - 1) / zc;
  g.ntiles = xy * g.chunksZ;
  int grid = (int)(g.ntiles < ctas ? g.ntiles : ctas);
  if (grid_used) *grid_used = grid;
  if (f.d == 3) {
    if (with_est)
      k_sz_march<k3TX, k3TY, k3R, k3PZ, k3NST, true><<<grid, Cfg3::kThreads, Cfg3::kSmem, s>>>(map, g, p, ws);
    else
      k_sz_march<k3TX, k3TY, k3R, k3PZ, k3NST, false><<<grid, Cfg3::kThreads, Cfg3::kSmem, s>>>(map, g, p, ws);
  } else {
    if (with_est)
      k_sz_march<128, 1, 1, 16, 4, true><<<grid, Cfg2::kThreads, Cfg2::kSmem, s>>>(map, g, p, ws);
    else
      k_sz_march<128, 1, 1, 16, 4, false><<<grid, Cfg2::kThreads, Cfg2::kSmem, s>>>(map, g, p, ws);
  }
  return cudaGetLastError();
}

}  // namespace rdk
