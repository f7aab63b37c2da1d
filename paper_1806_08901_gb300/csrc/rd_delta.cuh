// rd_delta.cuh -- the bin width delta from the exact MSE_sp (Algorithm 1
// line 7) and the estimated PSNRs, as a device function run by one warp:
// shared by the per-field launch and the batched ZFP pass, whose last CTA of
// a field runs it.
#pragma once

#include <math.h>
#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

// ---------------------------------------------------------------------------
// Bin width.  MSE_sp is the exact sum of (2^d d)^2 4^(emax-30) over the
// EC-sampled coefficients, held as 64-bit limbs with the least significant
// bit at 2^-312 and rounded once to nearest-even; delta = sqrt(12 MSE_sp)
// (PSNR_sz = PSNR_zfp in Eq. psnr-pdf-linear), clamped to 2 eb_abs.
// ---------------------------------------------------------------------------
constexpr int kLimbs = 12;  // 768 bits

// Round the limb integer times 2^-312 to the nearest double (ties to even):
// the 53 bits below the leading one, a round bit and a sticky bit.  Every
// limb index is a compile-time constant, so the limbs stay in registers.
__device__ __forceinline__ double limbs_to_double(const unsigned long long (&a)[kLimbs]) {
  // rolling window (w2, w1, w0) = limbs i, i-1, i-2 and the OR of the
  // limbs below it, captured at the highest nonzero limb
  unsigned long long w2 = 0ull, w1 = 0ull, w0 = 0ull;
  bool bl = false;
  unsigned long long h = 0ull, m = 0ull, l = 0ull;
  bool below = false;
  int ti = -1;
#pragma unroll
  for (int i = 0; i < kLimbs; i++) {
    bl = bl || (w0 != 0ull);
    w0 = w1;
    w1 = w2;
    w2 = a[i];
    if (w2) {
      h = w2;
      m = w1;
      l = w0;
      below = bl;
      ti = i;
    }
  }
  if (ti < 0) return 0.0;
  // normalise the 192-bit window h:m:l so that bit 63 of h is the leading one
  const int lz = __clzll((long long)h);
  if (lz) {
    h = (h << lz) | (m >> (64 - lz));
    m = (m << lz) | (l >> (64 - lz));
    l <<= lz;
  }
  unsigned long long mant = h >> 11;  // 53 bits
  const bool round = (h >> 10) & 1ull;
  const bool sticky = (h & 0x3ffull) || m || l || below;
  if (round && (sticky || (mant & 1ull))) mant += 1ull;  // 2^53 stays exact
  const int lead = ti * 64 + 63 - lz;  // bit index of the leading one
  return ldexp((double)mant, lead - 52 - 312);
}

// Launched with one warp.  Bin i holds a 128-bit sum at bit offset 2i, so
// the bins of lane l (i = l + 32k) all sit at shift 2l within limb k: each
// lane adds its bins as one multi-limb integer, shifts it by 2l, and a
// butterfly adds the 32 integers (exact, so the order does not matter).
// The logarithms of the PSNRs run in separate lanes.
__device__ __forceinline__ void delta_warp(const ParamsDev& p, Workspace* ws, int mode, double arg,
                                           int need_quant, int need_gt, unsigned long long ncoeff,
                                           unsigned long long npoints) {
  Scalars& s = ws->sc;
  if (s.status != RD_OK || s.constant) return;
  rd_result& r = ws->res;
  const int lane = threadIdx.x & 31;
  double delta, mse_sp = 0.0;
  bool clamped = false;
  if (mode == DELTA_FROM_MSE) {
    unsigned long long acc[kLimbs];
    unsigned long long lo[9], hi[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const int i = lane + 32 * k;
      lo[k] = i < kMseBins ? __ldcg(&s.mse_lo[i]) : 0ull;
      hi[k] = i < kMseBins ? __ldcg(&s.mse_hi[i]) : 0ull;
    }
    unsigned long long carry = 0ull;
#pragma unroll
    for (int k = 0; k < 10; k++) {
      const unsigned long long a0 = k < 9 ? lo[k] : 0ull;
      const unsigned long long a1 = k >= 1 ? hi[k - 1] : 0ull;
      const unsigned long long t = a0 + a1;
      const unsigned long long c1 = t < a0;
      const unsigned long long u = t + carry;
      const unsigned long long c2 = u < carry;
      acc[k] = u;
      carry = c1 + c2;
    }
    acc[10] = carry;
    acc[11] = 0ull;
    const int sh = 2 * lane;
    if (sh) {
#pragma unroll
      for (int j = kLimbs - 1; j > 0; j--) acc[j] = (acc[j] << sh) | (acc[j - 1] >> (64 - sh));
      acc[0] <<= sh;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long c = 0ull;
#pragma unroll
      for (int j = 0; j < kLimbs; j++) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, acc[j], o);
        const unsigned long long u = acc[j] + t;
        const unsigned long long c1 = u < t;
        const unsigned long long v = u + c;
        const unsigned long long c2 = v < c;
        acc[j] = v;
        c = c1 + c2;
      }
    }
    mse_sp = limbs_to_double(acc) / (double)ncoeff;
    if (mse_sp == 0.0) {
      delta = 2.0 * s.eb_abs;
    } else {
      delta = sqrt(12.0 * mse_sp);
      clamped = delta > 2.0 * s.eb_abs;
      if (clamped) delta = 2.0 * s.eb_abs;
    }
  } else if (mode == DELTA_EXPLICIT) {
    delta = arg > 0.0 ? arg : 2.0 * s.eb_abs;
  } else {
    delta = 2.0 * arg;
  }
  // lane 0: log10 VR, lane 1: log10 MSE_sp, lane 2: log10 (VR / delta),
  // lane 3: log10 12
  const double larg = lane == 0 ? s.vr : lane == 1 ? mse_sp : lane == 2 ? s.vr / delta : 12.0;
  const double lg = log10(larg);
  const double l_vr = __shfl_sync(0xffffffffu, lg, 0);
  const double l_mse = __shfl_sync(0xffffffffu, lg, 1);
  const double l_vd = __shfl_sync(0xffffffffu, lg, 2);
  const double l_12 = __shfl_sync(0xffffffffu, lg, 3);
  if (lane != 0) return;
  if (mode == DELTA_FROM_MSE) {
    s.mse_sp = mse_sp;
    r.mse_sp = mse_sp;
    const unsigned long long s2 = __ldcg(&s.s2);
    r.zfp_s2 = s2;
    r.br_zfp = (double)s2 / (2.0 * (double)npoints);
    r.psnr_zfp = mse_sp > 0.0 ? 20.0 * l_vr - 10.0 * l_mse : INFINITY;
    if (mse_sp == 0.0) s.flags |= RD_F_MSE_ZERO;
    if (clamped) s.flags |= RD_F_DELTA_CLAMPED;
  }
  s.delta = delta;
  r.delta = delta;
  r.psnr_sz = 20.0 * l_vd + 10.0 * l_12;
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


}  // namespace rdk
