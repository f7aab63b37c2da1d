// rd_zfp3.cu -- the ZFP pass over a 3D field with four lanes per 4x4x4 block
// (Sections "Block Orthogonal Transformation" and "Estimation Based on
// Dynamic Quantization"; the ground truth of the same blocks).
//
// One thread holding a whole 4^3 block needs its 64 values and 64
// coefficients in registers (about 250 of them), which leaves one SM eight
// resident warps and nothing to hide the latency of the integer chains.
// Here the four lanes of a quad share a block, in the slice, line and rank
// layouts of rd_zfp3_dev.cuh.  A warp takes eight consecutive blocks (eight
// quads) per step, so each of its 16-byte loads reads four whole 128-byte
// rows.  Every integer result (exponents, coefficients, bits, the
// estimator's sums) is the one thread-per-block computation's, term for
// term; only the float32 sum of squared errors is added in another order.
#include <stdint.h>
#include <string.h>

#include "rd_delta.cuh"
#include "rd_finish.cuh"
#include "rd_zfp3_dev.cuh"

namespace rdk {

constexpr int kZ3Threads = 256;
constexpr int kZ3Warps = kZ3Threads / 32;
static_assert(kZ3Threads >= kFinishThreads, "the last CTA runs the finish step's sums");

// The evaluate step's truth pass beside the Huffman launch: the CTA that
// ends last (its own counter, fenced on both sides) waits for the Huffman
// launch to complete (the programmatic dependency's wait; so this pass also
// completes after it), finishes the ZFP truth (squared-error sum over the
// CTAs' partials in a fixed order, MSE, PSNR, rate), compares the truths and
// writes the records.  Every thread of every CTA calls it.
__device__ __forceinline__ void zfp_finish_last(Workspace* ws, const FinishArgs& fa) {
  __shared__ int s_lastz;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_lastz = atomicAdd(&ws->sc.zfp_done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_lastz) return;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __threadfence();
  finish_pre(ws, fa.passes & ~P_SZ_GT, (int)gridDim.x, fa.sz_parts, fa.npoints_all);
  finish_combine(ws, fa.passes, fa.out);
}

template <bool GT, bool EST>
__global__ void __launch_bounds__(kZ3Threads) k_zfp3(FieldDev f, ParamsDev p, DeltaArgs da,
                                                      Workspace* ws, FinishArgs fa) {
  __shared__ unsigned long long s_lo[kMseBins], s_hi[kMseBins];
  __shared__ unsigned long long s_acc[2];
  __shared__ double s_sse[kZ3Warps];
  __shared__ float s_max[kZ3Warps];
  __shared__ __align__(16) int s_tr[kZ3Warps][8 * kZ3BlockWords];
  __shared__ __align__(16) unsigned char s_rk[kZ3Warps][8 * kZ3RankBytes];
  const Scalars& sc = ws->sc;
  {
    // one reading of the status for the whole CTA (with a join, the Huffman
    // launch runs beside this pass and may change it)
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (__ldcg(&sc.status) != RD_OK || __ldcg(&sc.constant)) ? 1 : 0;
    __syncthreads();
    if (s_skip) {
      // the evaluate step's records still come from this pass's last CTA
      if (GT && fa.join) zfp_finish_last(ws, fa);
      return;
    }
  }
  const int minexp = sc.minexp;
  if (EST) {
    for (int i = threadIdx.x; i < kMseBins; i += blockDim.x) {
      s_lo[i] = 0ull;
      s_hi[i] = 0ull;
    }
  }
  if (threadIdx.x < 2) s_acc[threadIdx.x] = 0ull;
  __syncthreads();

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int q = lane & 3, g = lane >> 2;
  // the layouts' per-lane constants, by q: ranks (4 words), S2 weights (4
  // words) and the EC mask, read from shared memory where used
  __shared__ uint32_t s_tab[4][12];
  quad_fill_tables(s_tab, p.ec_mode == RD_EC_ALL);
  __syncthreads();
  const uint32_t* tab = s_tab[q];

  int* tr = &s_tr[wid][g * kZ3BlockWords];
  unsigned char* rb = &s_rk[wid][g * kZ3RankBytes];

  // units: every block (ground truth) or the sampled blocks (estimate
  // alone), in raster order; the warp walks its first unit and the stride
  // of all warps as digits of the block (or lattice) grid (fewer than 2^31
  // units: the field has fewer than 2^31 points)
  const int* R = GT ? f.B : f.L;
  const int units = (int)(GT ? f.nblocks : f.nsampled);
  const int w0 = (blockIdx.x * kZ3Warps + wid) * 8;
  const int wstep = gridDim.x * kZ3Warps * 8;
  Radix3 pos, step;
  pos.set(w0 < units ? w0 : 0, R);
  step.set(wstep, R);

  unsigned long long my_s2 = 0ull, my_bits = 0ull;
  double my_sse = 0.0;
  float my_max = 0.0f;

  for (int base = w0; base < units; base += wstep) {
    const bool act = base + g < units;
    // this lane's unit: the warp's position plus g along the fastest digit
    int l2 = pos.a2 + g, l1 = pos.a1, l0 = pos.a0;
    if (l2 >= R[2]) {  // a carry (several when the grid is narrower than 8)
      l1 += l2 / R[2];
      l2 %= R[2];
      if (l1 >= R[1]) {
        l0 += l1 / R[1];
        l1 %= R[1];
      }
    }
    pos.add(step, R);
    int b0 = l0, b1 = l1, b2 = l2;
    if (!GT) {
      b0 *= f.s[0];
      b1 *= f.s[1];
      b2 *= f.s[2];
    }
    const bool sampled = act && (!GT || (on_stride(f, 0, b0) && on_stride(f, 1, b1) &&
                                          on_stride(f, 2, b2)));
    const bool interior = 4 * b0 + 4 <= f.n[0] && 4 * b1 + 4 <= f.n[1] && 4 * b2 + 4 <= f.n[2];

    int c[16];
    int emax;
    {
      float v[16];
      load_slice(f, b0, b1, b2, q, act, interior, v);
      emax = quad_emax(v);
      quad_cast(v, emax, c);
    }
    const bool all_zero = emax == -127;
    const int prec = all_zero ? 0 : min(32, max(0, emax - minexp + 8));
    const int kmin = 32 - prec;
    unsigned uu[16];
    quad_transform(c, q, tr, uu);

    // estimator: exact squared truncation errors of the EC-sampled
    // coefficients, binned by the block exponent
    bool est_has = false;
    unsigned long long lo = 0ull, hi = 0ull;
    if (EST && sampled) {
      quad_est_err(uu, kmin, tab[8], lo, hi);
      est_has = !all_zero && (lo | hi);
    }
    if (EST) mse_add_warp(est_has, mse_bin<3>(emax), lo, hi, s_lo, s_hi);

    // truncation to the coded planes, then the rank layout
    int cr[16];
    const int seed = quad_rank(uu, kmin, q, tab, rb, cr);

    if (EST && sampled) my_s2 += quad_s2(cr, kmin, tab);

    if (GT) {
      // exact group-test embedded-coding cost (the suffix-maximum closed
      // form of the thread-per-block pass, split over the quad's ranks).
      // c' of a truncated coefficient is 0 or above kmin.  With Mk the
      // suffix maximum of c' floored at k1 = max(kmin, 1), the verbatim bits
      // sum (Mk - kmin) less, when kmin = 0, one per rank whose suffix
      // holds no one at all; a one is found where c' equals Mk (c' >= 1).
      const int k1 = max(kmin, 1);
      int Mk = max(seed, k1);
      unsigned sumM = 0u, found = 0u;
#pragma unroll
      for (int j = 15; j >= 0; j--) {
        Mk = max(Mk, cr[j]);
        sumM += (unsigned)Mk;
        found += cr[j] == Mk ? 1u : 0u;
      }
      unsigned bits = sumM - 16u * (unsigned)kmin + found;
      if (kmin == 0) {
        // ranks with an empty suffix: above the quad's highest nonzero c'
        int hi = -1;
#pragma unroll
        for (int j = 0; j < 16; j++) hi = cr[j] ? j : hi;
        const int top = seed > 0 ? 16 : hi + 1;  // ranks of this lane with a nonzero suffix
        bits -= (unsigned)(16 - top);
      }
      if (q == 3) {
        const int last = cr[15];  // rank 63
        bits += 9u + (unsigned)(32 - max(kmin, last)) - (last > kmin ? 1u : 0u);
      }
      if (prec == 0) bits = q == 0 ? 1u : 0u;
      my_bits += act ? bits : 0u;

      // inverse lifting z (line layout), back to the slice layout, inverse
      // lifting y and x
#pragma unroll
      for (int i = 0; i < 16; i++) c[i] = from_negabinary(uu[i]);
#pragma unroll
      for (int x = 0; x < 4; x++) inv_lift(c[x], c[4 + x], c[8 + x], c[12 + x]);
#pragma unroll
      for (int z = 0; z < 4; z++)
        *reinterpret_cast<int4*>(tr + z * kZ3SliceWords + 4 * q) =
            make_int4(c[4 * z], c[4 * z + 1], c[4 * z + 2], c[4 * z + 3]);
      __syncwarp();
#pragma unroll
      for (int y = 0; y < 4; y++) {
        const int4 t = *reinterpret_cast<const int4*>(tr + q * kZ3SliceWords + 4 * y);
        c[4 * y] = t.x;
        c[4 * y + 1] = t.y;
        c[4 * y + 2] = t.z;
        c[4 * y + 3] = t.w;
      }
      __syncwarp();
#pragma unroll
      for (int x = 0; x < 4; x++) inv_lift(c[x], c[4 + x], c[8 + x], c[12 + x]);
#pragma unroll
      for (int y = 0; y < 4; y++) inv_lift(c[4 * y], c[4 * y + 1], c[4 * y + 2], c[4 * y + 3]);

      // reconstruction and errors at the valid points (the values read
      // again: they stay in L1 between the two reads)
      float v[16];
      load_slice(f, b0, b1, b2, q, act, interior, v);
      // x-hat = float(i) 2^(emax - 30): one exact factor, or two below 2^-126
      // (an inactive lane has v = 0 and i = 0: no error)
      const int e = emax - 30;
      float e2[16];
      if (e >= -126) {
        const float scl = pow2f(e);
#pragma unroll
        for (int i = 0; i < 16; i++) e2[i] = __fsub_rn(v[i], __fmul_rn(__int2float_rn(c[i]), scl));
      } else {
        const float scl = pow2f(e + 64);
#pragma unroll
        for (int i = 0; i < 16; i++)
          e2[i] = __fsub_rn(v[i], __fmul_rn(__fmul_rn(__int2float_rn(c[i]), scl), pow2f(-64)));
      }
      if (!interior) {
        const bool zin = 4 * b0 + q < f.n[0];
#pragma unroll
        for (int i = 0; i < 16; i++) {
          const bool ok = zin && (4 * b1 + (i >> 2) < f.n[1]) && (4 * b2 + (i & 3) < f.n[2]);
          e2[i] = ok ? e2[i] : 0.0f;
        }
      }
      float emx = 0.0f;
#pragma unroll
      for (int i = 0; i < 16; i++) emx = fmaxf(emx, fabsf(e2[i]));
      my_max = fmaxf(my_max, emx);
      if (emx > 0.0f) {
        // scale by 2^k (exact) so the largest error is in [1, 2): squares of
        // errors far below eb_abs neither underflow nor lose the sum
        const unsigned Ex = (__float_as_uint(emx) >> 23) & 0xffu;
        const int k = Ex ? 127 - (int)Ex : 149;
        if (k <= 127 && k >= -126) {
          const float scl = pow2f(k);
#pragma unroll
          for (int i = 0; i < 16; i++) e2[i] = __fmul_rn(e2[i], scl);
        } else {
#pragma unroll
          for (int i = 0; i < 16; i++) e2[i] = mul_pow2(e2[i], k);
        }
        // squares summed pairwise in float (the first level as a fused
        // multiply-add of two squares)
#pragma unroll
        for (int i = 0; i < 8; i++) e2[i] = __fmaf_rn(e2[i], e2[i], __fmul_rn(e2[i + 8], e2[i + 8]));
#pragma unroll
        for (int w2 = 4; w2 >= 1; w2 >>= 1) {
#pragma unroll
          for (int i = 0; i < w2; i++) e2[i] = __fadd_rn(e2[i], e2[i + w2]);
        }
        // the partial (>= 1, a normal float) times 2^-2k, built as a double
        // exactly with integer operations (one float64 add per slice)
        const unsigned fb = __float_as_uint(e2[0]);
        const unsigned dexp = (fb >> 23) - 127u + 1023u - (unsigned)(2 * k);
        const int hiw = (int)((dexp << 20) | ((fb & 0x7fffffu) >> 3));
        const int low = (int)((fb & 7u) << 29);
        my_sse += __hiloint2double(hiw, low);
      }
    }
  }

  // reductions: warp, then CTA, then one global update per CTA
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
      for (int i = 0; i < kZ3Warps; i++) {
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
  if (GT && fa.join) zfp_finish_last(ws, fa);
}

cudaError_t launch_zfp3(const FieldDev& f, const ParamsDev& p, int passes, const DeltaArgs& da,
                        Workspace* ws, int ctas, cudaStream_t s, int* grid_used, const FinishArgs* join) {
  FinishArgs fa;
  memset(&fa, 0, sizeof(fa));
  if (join) fa = *join;
  const bool gt = passes & P_ZFP_GT, est = passes & P_ZFP_EST;
  const long long units = gt ? f.nblocks : f.nsampled;
  const long long per_cta = 8LL * kZ3Warps;
  const long long want = (units + per_cta - 1) / per_cta;
  int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (grid_used) *grid_used = g;
  if (gt && est)
    k_zfp3<true, true><<<g, kZ3Threads, 0, s>>>(f, p, da, ws, fa);
  else if (gt)
    k_zfp3<true, false><<<g, kZ3Threads, 0, s>>>(f, p, da, ws, fa);
  else
    k_zfp3<false, true><<<g, kZ3Threads, 0, s>>>(f, p, da, ws, fa);
  return cudaGetLastError();
}

cudaError_t launch_zfp3_after_huffman(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                                      const FinishArgs& fa, cudaStream_t s, int* grid_used) {
  const long long per_cta = 8LL * kZ3Warps;
  const long long want = (f.nblocks + per_cta - 1) / per_cta;
  const int g = (int)(want < ctas ? (want < 1 ? 1 : want) : ctas);
  if (grid_used) *grid_used = g;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(g, 1, 1);
  cfg.blockDim = dim3(kZ3Threads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_zfp3<true, false>, f, p, DeltaArgs{}, ws, fa);
}

int zfp3_occupancy(int num_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_zfp3<true, true>,
                                                    kZ3Threads, 0) != cudaSuccess ||
      per < 1)
    per = 1;
  long long g = (long long)per * num_sms;
  return (int)(g > kMaxGrid ? kMaxGrid : g);
}

}  // namespace rdk
