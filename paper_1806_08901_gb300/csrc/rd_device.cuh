// rd_device.cuh -- device helpers of the rate-distortion kernels: the ZFP
// block transform in 32-bit two's complement, the sequency permutation,
// negabinary coding, power-of-two float scaling and histogram updates.
#pragma once

#include <stdint.h>

#include "rd_internal.cuh"

namespace rdk {

// ---------------------------------------------------------------------------
// 32-bit wrapping integer arithmetic (the transform is defined modulo 2^32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wadd(int a, int b) { return (int)((unsigned)a + (unsigned)b); }
__device__ __forceinline__ int wsub(int a, int b) { return (int)((unsigned)a - (unsigned)b); }
__device__ __forceinline__ int wdbl(int a) { return (int)((unsigned)a << 1); }
__device__ __forceinline__ int asr1(int a) { return a >> 1; }  // floor(a / 2)

// ZFP's decorrelating 4-point transform (zfp publication, Lindstrom 2014):
// forward matrix (1/16)[[4,4,4,4],[5,1,-1,-5],[-4,4,4,-4],[-2,6,-6,2]] as a
// lifting scheme (Section "Block Orthogonal Transformation" applies it along
// every axis of a 4^d block).
__device__ __forceinline__ void fwd_lift(int& a, int& b, int& c, int& d) {
  a = asr1(wadd(a, d)); d = wsub(d, a);   // outer pair: mean, half-difference
  c = asr1(wadd(c, b)); b = wsub(b, c);   // inner pair
  a = asr1(wadd(a, c)); c = wsub(c, a);   // the two means
  d = asr1(wadd(d, b)); b = wsub(b, d);   // the two differences
  d = wadd(d, asr1(b)); b = wsub(b, asr1(d));  // rotate the odd terms
}

// Exact inverse of every lifting step, applied in reverse order.
__device__ __forceinline__ void inv_lift(int& a, int& b, int& c, int& d) {
  b = wadd(b, asr1(d)); d = wsub(d, asr1(b));
  b = wadd(b, d); d = wsub(wdbl(d), b);
  c = wadd(c, a); a = wsub(wdbl(a), c);
  b = wadd(b, c); c = wsub(wdbl(c), b);
  d = wadd(d, a); a = wsub(wdbl(a), d);
}

// Apply the transform along axis `A` of a 4^D block held in registers
// (block index t = sum_k t_k 4^(D-1-k), last axis fastest).
template <int D, int A, bool INV>
__device__ __forceinline__ void lift_axis(int* c) {
  constexpr int NB = 1 << (2 * D);
  constexpr int ST = 1 << (2 * (D - 1 - A));
#pragma unroll
  for (int t = 0; t < NB; t++) {
    if (((t / ST) & 3) == 0) {
      if (INV)
        inv_lift(c[t], c[t + ST], c[t + 2 * ST], c[t + 3 * ST]);
      else
        fwd_lift(c[t], c[t + ST], c[t + 2 * ST], c[t + 3 * ST]);
    }
  }
}

// Forward: fastest axis first.  Inverse: slowest axis first.
template <int D>
__device__ __forceinline__ void fwd_xform(int* c) {
  lift_axis<D, D - 1, false>(c);
  if constexpr (D >= 2) lift_axis<D, D - 2, false>(c);
  if constexpr (D >= 3) lift_axis<D, D - 3, false>(c);
}

template <int D>
__device__ __forceinline__ void inv_xform(int* c) {
  if constexpr (D >= 3) lift_axis<D, D - 3, true>(c);
  if constexpr (D >= 2) lift_axis<D, D - 2, true>(c);
  lift_axis<D, D - 1, true>(c);
}

// ---------------------------------------------------------------------------
// Sequency order, built at compile time: block indices ordered by the sum of
// their per-axis indices, then the sum of squares, then lexicographically
// with the slowest axis first.
// ---------------------------------------------------------------------------
template <int D>
struct Sequency {
  static constexpr int NB = 1 << (2 * D);
  int perm[NB];  // perm[p] = block index of the coefficient at sequency p

  static constexpr int digit(int t, int k) { return (t >> (2 * (D - 1 - k))) & 3; }
  static constexpr bool before(int a, int b) {
    int sa = 0, sb = 0, qa = 0, qb = 0;
    for (int k = 0; k < D; k++) {
      sa += digit(a, k); sb += digit(b, k);
      qa += digit(a, k) * digit(a, k); qb += digit(b, k) * digit(b, k);
    }
    if (sa != sb) return sa < sb;
    if (qa != qb) return qa < qb;
    for (int k = 0; k < D; k++)
      if (digit(a, k) != digit(b, k)) return digit(a, k) < digit(b, k);
    return false;
  }
  constexpr Sequency() : perm() {
    for (int t = 0; t < NB; t++) perm[t] = t;
    for (int i = 1; i < NB; i++) {
      int v = perm[i];
      int j = i - 1;
      while (j >= 0 && before(v, perm[j])) {
        perm[j + 1] = perm[j];
        j--;
      }
      perm[j + 1] = v;
    }
  }
};

// Embedded-coding sample positions: m of the 4^D sequency positions spread
// evenly, p_j = floor((j (NB-1) + floor((m-1)/2)) / (m-1)); m = 3/9/16.
template <int D>
struct EcPositions {
  static constexpr int NB = 1 << (2 * D);
  static constexpr int M = D == 1 ? 3 : D == 2 ? 9 : 16;
  int pos[M];
  constexpr EcPositions() : pos() {
    for (int j = 0; j < M; j++) pos[j] = (j * (NB - 1) + (M - 1) / 2) / (M - 1);
  }
};

// Negabinary: base -2 digits of a two's complement integer.
__device__ __forceinline__ unsigned int to_negabinary(int i) {
  return ((unsigned)i + 0xaaaaaaaau) ^ 0xaaaaaaaau;
}
__device__ __forceinline__ int from_negabinary(unsigned int u) {
  return (int)((u ^ 0xaaaaaaaau) - 0xaaaaaaaau);
}

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// x * 2^e rounded once, for -156 <= e <= 127 (a two-step product whose first
// factor keeps the intermediate in the normal range).
__device__ __forceinline__ float scale_pow2(float x, int e) {
  if (e >= -126) return __fmul_rn(x, pow2f(e));
  return __fmul_rn(__fmul_rn(x, pow2f(e + 64)), pow2f(-64));
}

// x * 2^k for -252 <= k <= 254 (two products outside the normal range of 2^k).
__device__ __forceinline__ float mul_pow2(float x, int k) {
  if (k > 127) return __fmul_rn(__fmul_rn(x, pow2f(127)), pow2f(k - 127));
  if (k < -126) return __fmul_rn(__fmul_rn(x, pow2f(-126)), pow2f(k + 126));
  return __fmul_rn(x, pow2f(k));
}

// trunc(x * 2^e) for the block-floating-point cast, -98 <= e <= 156, where
// |x * 2^e| < 2^30.  Results below one may round but truncate to zero.
__device__ __forceinline__ int cast_scaled(float x, int e) {
  float y = (e <= 127) ? __fmul_rn(x, pow2f(e))
                       : __fmul_rn(__fmul_rn(x, pow2f(127)), pow2f(e - 127));
  return __float2int_rz(y);
}

// ---------------------------------------------------------------------------
// Conversion-free integer/float helpers.  On this GPU the F2I / I2F / FRND
// conversions issue on the narrow float64 pipe, so the per-value paths use
// integer bit operations and float adds instead; each helper gives exactly
// the result of the conversion it replaces.
// ---------------------------------------------------------------------------

// trunc(x * 2^s) when |x * 2^s| < 2^30 (the block-floating-point cast):
// x = m * 2^(E-150) with the 24-bit significand m, so x * 2^s = m * 2^(E-150+s).
__device__ __forceinline__ int cast_bits(float x, int s) {
  const unsigned b = __float_as_uint(x);
  int E = (int)((b >> 23) & 0xffu);
  unsigned m = b & 0x7fffffu;
  if (E) m |= 0x800000u; else E = 1;  // subnormal: no hidden bit, exponent of E = 1
  const int sh = E - 150 + s;
  const unsigned mag = sh >= 0 ? (m << sh) : (m >> min(-sh, 31));
  return (b >> 31) ? -(int)mag : (int)mag;
}

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

// float(k) for |k| < 2^22, exactly.
__device__ __forceinline__ float small_int_to_float(int k) {
  return __fsub_rn(__int_as_float(k + kMagicBits), kMagic);
}

// float(i) rounded to nearest even for any int: i = hi * 2^16 + lo with both
// halves exact in float, summed by one fused multiply-add (one rounding).
__device__ __forceinline__ float int_to_float_rn(int i) {
  const float fh = small_int_to_float(i >> 16);
  const float fl = small_int_to_float(i & 0xffff);
  return __fmaf_rn(fh, 65536.0f, fl);
}

// rint(t) for |t| < 2^22: adding 1.5 * 2^23 rounds t to the nearest integer
// (ties to even) in the low bits; returns the integer and its exact float.
__device__ __forceinline__ int round_small(float t, float& tf) {
  const float a = __fadd_rn(t, kMagic);
  tf = __fsub_rn(a, kMagic);
  return __float_as_int(a) - kMagicBits;
}

// Ordered unsigned key of a float: monotone in the float's value.
__device__ __forceinline__ unsigned int float_key(float v) {
  unsigned int b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k) {
  unsigned int b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

// Histogram update: bins near the centre go to a per-CTA shared window, the
// rest straight to global memory.  Lanes of a warp with the same symbol are
// merged into one atomic.
__device__ __forceinline__ void hist_add(uint32_t* s_win, uint32_t* g_hist, int sym,
                                         unsigned mask) {
  unsigned same = __match_any_sync(mask, sym);
  int leader = __ffs(same) - 1;
  if ((int)(threadIdx.x & 31) == leader) {
    unsigned cnt = __popc(same);
    int wi = sym - kHistWinLo;
    if ((unsigned)wi < (unsigned)kHistWin)
      atomicAdd(&s_win[wi], cnt);
    else
      atomicAdd(&g_hist[sym], cnt);
  }
}

// Warp-aggregated histogram insert without warp matching (whose unit runs it
// at a low rate on this GPU), two symbols per lane: each lane packs two
// 16-bit symbols into one word, and the warp sorts both 32-symbol sequences
// at once with a bitonic network of shuffles and paired 16-bit min/max (the
// network does not depend on the data, so both halves come out sorted).
// The first lane of every run of equal symbols in a half adds the run's
// length with one atomic (shared window [win_lo, win_lo + win), else the
// global histogram): sorted runs land on consecutive words, so the atomics
// of a warp rarely meet in a bank.  Lanes whose symbol is not valid carry
// 0xffff, which sorts last, and are taken off that symbol's run.  Every lane
// of the warp calls.
__device__ __forceinline__ void hist_add_sorted2(uint32_t* s_win, int win_lo, int win,
                                                 uint32_t* g_hist, uint32_t keys, bool ok_lo,
                                                 bool ok_hi) {
  const int lane = threadIdx.x & 31;
  const unsigned bad_lo = __popc(__ballot_sync(0xffffffffu, !ok_lo));
  const unsigned bad_hi = __popc(__ballot_sync(0xffffffffu, !ok_hi));
  uint32_t key = keys;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint32_t other = __shfl_xor_sync(0xffffffffu, key, j);
      const bool up = (lane & k) == 0;
      const bool low = (lane & j) == 0;
      key = (low == up) ? __vminu2(key, other) : __vmaxu2(key, other);
    }
  }
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const uint32_t kh = (key >> (16 * h)) & 0xffffu, ph = (prev >> (16 * h)) & 0xffffu;
    const bool head = lane == 0 || kh != ph;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    if (head) {
      const unsigned later = heads & ~((2u << lane) - 1u);  // heads after this lane
      const int next = later ? __ffs(later) - 1 : 32;
      unsigned cnt = (unsigned)(next - lane);
      if (kh == 0xffffu) cnt -= h ? bad_hi : bad_lo;
      if (cnt) {
        const int wi = (int)kh - win_lo;
        if ((unsigned)wi < (unsigned)win)
          atomicAdd(&s_win[wi], cnt);
        else
          atomicAdd(&g_hist[kh], cnt);
      }
    }
  }
}

// A code histogram over the whole alphabet in shared memory (128 KB):
// 65536 16-bit counters, code s in half s >> 15 of word s & 0x7fff (so
// neighbouring codes, which a warp often hits together, fall in different
// words).  The residuals of rough fields at fine bounds spread over tens of
// thousands of codes: a partial window sent most of them to global atomics,
// which set the pace.  A counter cannot pass 65535 between flushes: an add
// that takes a counter to kHotCount or more raises a flag, and the CTA
// flushes at the end of the round of at most kRoundPoints points in
// progress.  Wide code distributions, whose counters stay low, flush only
// when the CTA is done with the field.
constexpr int kPackWords = 32768;
constexpr long long kRoundPoints = 16384;  // points between flush checks (a multiple of 4)
constexpr uint32_t kHotCount = 65535u - (uint32_t)kRoundPoints;

// Adds cnt to the counter of code sym; raises *s_hot when it reaches
// kHotCount.
__device__ __forceinline__ void packed_add(uint32_t* s_win, int sym, unsigned cnt, int* s_hot) {
  const int sh = (sym >> 15) << 4;
  const uint32_t old = atomicAdd(&s_win[sym & 0x7fff], cnt << sh);
  if (((old >> sh) & 0xffffu) + cnt >= kHotCount) *s_hot = 1;
}

// Adds the window's counters to the global histogram and clears them; every
// thread of the CTA calls.
__device__ __forceinline__ void window_flush(uint32_t* s_win, uint32_t* g_hist) {
  __syncthreads();
  uint4* w4 = reinterpret_cast<uint4*>(s_win);
  for (int i = threadIdx.x; i < kPackWords / 4; i += blockDim.x) {
    const uint4 c = w4[i];
    if (c.x | c.y | c.z | c.w) {
      const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (cw[k] & 0xffffu) atomicAdd(&g_hist[4 * i + k], cw[k] & 0xffffu);
        if (cw[k] >> 16) atomicAdd(&g_hist[4 * i + k + 32768], cw[k] >> 16);
      }
      w4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  __syncthreads();
}

// Per-thread register counters of the 2H+1 symbols around the centre, where
// nearly every code of a smooth field falls: counting them costs a few
// predicated adds and no atomics (contended shared-memory atomics on a few
// hot bins, or warp matching, would set the pace).  Other symbols take a
// plain atomic on the shared window (or the global histogram outside it).
template <int H>
struct HotBins {
  uint32_t c[2 * H + 1];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int k = 0; k < 2 * H + 1; k++) c[k] = 0u;
  }
  // d = symbol - kCenter; true when counted here
  __device__ __forceinline__ bool take(int d) {
#pragma unroll
    for (int k = 0; k < 2 * H + 1; k++) c[k] += d == k - H ? 1u : 0u;
    return (unsigned)(d + H) <= (unsigned)(2 * H);
  }
  // count symbol sym: a hot bin, else the window at win_lo (width win), else
  // the global histogram
  __device__ __forceinline__ void add(int sym, uint32_t* s_win, int win_lo, int win,
                                      uint32_t* g_hist) {
    if (take(sym - kCenter)) return;
    const int wi = sym - win_lo;
    if ((unsigned)wi < (unsigned)win)
      atomicAdd(&s_win[wi], 1u);
    else
      atomicAdd(&g_hist[sym], 1u);
  }
  // add the warp's counters to the global histogram; every lane of the warp
  // calls
  __device__ __forceinline__ void flush_global(uint32_t* g_hist) {
#pragma unroll
    for (int k = 0; k < 2 * H + 1; k++) {
      uint32_t v = c[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(&g_hist[kCenter - H + k], v);
    }
    clear();
  }
  // add the warp's counters to the window; every lane of the warp calls
  __device__ __forceinline__ void flush_warp(uint32_t* s_win, int win_lo) {
#pragma unroll
    for (int k = 0; k < 2 * H + 1; k++) {
      uint32_t v = c[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_win[kCenter - H + k - win_lo], v);
    }
    clear();
  }
};

__device__ __forceinline__ void hist_flush(const uint32_t* s_win, uint32_t* g_hist) {
  for (int i = threadIdx.x; i < kHistWin; i += blockDim.x) {
    uint32_t c = s_win[i];
    if (c) atomicAdd(&g_hist[kHistWinLo + i], c);
  }
}

// 128-bit add with carry into a (lo, hi) pair of 64-bit words.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* lo, unsigned long long* hi,
                                                unsigned long long vlo, unsigned long long vhi) {
  unsigned long long old = atomicAdd(lo, vlo);
  unsigned long long carry = (old + vlo < old) ? 1ull : 0ull;
  if (vhi + carry) atomicAdd(hi, vhi + carry);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace rdk
