// rd_zfp3_dev.cuh -- the ZFP block code of a 4x4x4 block shared by the four
// lanes q = 0..3 of a quad (Sections "Block Orthogonal Transformation" and
// "Estimation Based on Dynamic Quantization"), used by the 3D ZFP pass:
//   slice layout  lane q holds the plane z = q (16 values, x fastest): the
//                 lifting along x and y runs in its registers;
//   line layout   lane q holds the row y = q of every plane (z, q, 0..3):
//                 the lifting along z runs in its registers.  A transpose in
//                 shared memory (four 16-byte stores and loads per lane)
//                 turns one layout into the other;
//   rank layout   the embedded-coding cost and the estimator's interpolated
//                 sum walk the coefficients in sequency order: each lane
//                 writes the leading-one position of its 16 coefficients as
//                 bytes at their sequency ranks, and lane q reads ranks
//                 16q .. 16q+15 back in one 16-byte load.  The suffix maximum
//                 over ranks is the lane's own running maximum seeded with
//                 the maxima of the lanes above it (two shuffles).
// Every function is called by all four lanes of the quad, and every lane of
// the warp (the shuffles and warp barriers span the warp).
#pragma once

#include <stdint.h>

#include "rd_zfp_dev.cuh"

namespace rdk {

constexpr int kZ3SliceWords = 20;  // a 4x4 slice plus 4 words of padding (no bank conflicts)
constexpr int kZ3BlockWords = 4 * kZ3SliceWords;
// a block's 64 rank bytes plus 16 bytes of padding: the eight blocks of a
// warp start 20 words apart, so byte stores of one rank by the eight quads
// fall in different banks
constexpr int kZ3RankBytes = 80;
constexpr unsigned kFull = 0xffffffffu;

// Per-lane constants of the layouts, built at compile time from the
// sequency order and the EC sample positions of a 3D block.
struct Z3Tables {
  uint32_t rank[4][4];    // [q][z]: byte x = sequency rank of block index 16z + 4q + x
  uint32_t wpaper[4][4];  // [q][k]: byte b = weight of rank 16q + 4k + b in the doubled S2 sum
  uint32_t ecmask[4];     // [q]: bit 4z + x set when block index 16z + 4q + x is EC-sampled
  constexpr Z3Tables() : rank(), wpaper(), ecmask() {
    const Sequency<3> S{};
    const EcPositions<3> EC{};
    int rk[64] = {};
    for (int p = 0; p < 64; p++) rk[S.perm[p]] = p;
    int w[64] = {};
    bool isec[64] = {};
    // S2 = sum_j [(L_j + 1) n(p_j) + (L_j - 1) n(p_{j+1})] + 2 n(p_last):
    // each EC position's weight is its share of the interpolated sum
    for (int j = 0; j < EcPositions<3>::M; j++) {
      int wt = j + 1 < EcPositions<3>::M ? EC.pos[j + 1] - EC.pos[j] + 1 : 2;
      if (j > 0) wt += EC.pos[j] - EC.pos[j - 1] - 1;
      w[EC.pos[j]] = wt;
      isec[EC.pos[j]] = true;
    }
    for (int q = 0; q < 4; q++) {
      uint32_t m = 0u;
      for (int z = 0; z < 4; z++) {
        uint32_t word = 0u;
        for (int x = 0; x < 4; x++) {
          const int r = rk[16 * z + 4 * q + x];
          word |= (uint32_t)r << (8 * x);
          if (isec[r]) m |= 1u << (4 * z + x);
        }
        rank[q][z] = word;
      }
      ecmask[q] = m;
      for (int k = 0; k < 4; k++) {
        uint32_t word = 0u;
        for (int b = 0; b < 4; b++) word |= (uint32_t)w[16 * q + 4 * k + b] << (8 * b);
        wpaper[q][k] = word;
      }
    }
  }
};

__device__ __forceinline__ uint32_t pick_q(int q, uint32_t a0, uint32_t a1, uint32_t a2,
                                           uint32_t a3) {
  return q == 0 ? a0 : q == 1 ? a1 : q == 2 ? a2 : a3;
}

// A position in a 3-axis mixed radix (slowest first), advanced by a fixed
// stride without divisions.
struct Radix3 {
  int a0, a1, a2;
  __device__ __forceinline__ void set(long long u, const int* R) {
    a2 = (int)(u % R[2]);
    u /= R[2];
    a1 = (int)(u % R[1]);
    a0 = (int)(u / R[1]);
  }
  // add a stride given as digits (each below its radix)
  __device__ __forceinline__ void add(const Radix3& s, const int* R) {
    a2 += s.a2;
    int c = a2 >= R[2];
    a2 -= c ? R[2] : 0;
    a1 += s.a1 + c;
    c = a1 >= R[1];
    a1 -= c ? R[1] : 0;
    a0 += s.a0 + c;
  }
};

// Load plane z = 4 b0 + q of a block (clamped to the last plane, rows and
// columns clamped likewise: partial blocks replicate their last sample).
__device__ __forceinline__ void load_slice(const FieldDev& f, int b0, int b1, int b2, int q,
                                           bool act, bool interior, float* v) {
  if (!act) {
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = 0.0f;
    return;
  }
  const float* __restrict__ x = f.x;
  const int z = min(4 * b0 + q, f.n[0] - 1);
  const int y0 = 4 * b1, x0 = 4 * b2;
  if (interior && f.vec_ok) {
    // point indices stay below 2^31
    const float* p0 = x + ((z * f.n[1] + y0) * f.n[2] + x0);
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p0 + r * f.n[2]));
      v[4 * r + 0] = t.x;
      v[4 * r + 1] = t.y;
      v[4 * r + 2] = t.z;
      v[4 * r + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int y = min(y0 + r, f.n[1] - 1);
      const long long row = ((long long)z * f.n[1] + y) * f.n[2];
#pragma unroll
      for (int j = 0; j < 4; j++) v[4 * r + j] = __ldg(x + row + min(x0 + j, f.n[2] - 1));
    }
  }
}

// Block coordinate b is on axis k's sampling lattice (a multiple of s[k]).
__device__ __forceinline__ bool on_stride(const FieldDev& f, int k, int b) {
  if (f.ssh[k] < 0) return true;
  const unsigned qt = __umulhi((unsigned)b, f.smag[k]) >> f.ssh[k];
  return (int)qt * f.s[k] == b;
}

// The quad tables by q (ranks: words 0..3, S2 weights: 4..7, EC mask: 8),
// written by the first 48 threads of the CTA; a barrier must follow.
__device__ __forceinline__ void quad_fill_tables(uint32_t (*s_tab)[12], bool ec_all) {
  if (threadIdx.x < 48) {
    constexpr Z3Tables T{};
    const int tq = threadIdx.x / 12, k = threadIdx.x % 12;
    uint32_t v = 0u;
#pragma unroll
    for (int a = 0; a < 4; a++) {
#pragma unroll
      for (int z = 0; z < 4; z++) {
        if (a == tq && z == k) v = T.rank[a][z];
        if (a == tq && z + 4 == k) v = ec_all ? 0x02020202u : T.wpaper[a][z];
      }
      if (a == tq && k == 8) v = ec_all ? 0xffffu : T.ecmask[a];
    }
    s_tab[tq][k] = v;
  }
}

// Block exponent (zfp fixed-accuracy rule): the largest magnitude's exponent
// field over the quad; -127 for an all-zero block.
__device__ __forceinline__ int quad_emax(const float* v) {
  float am = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; i++) am = fmaxf(am, fabsf(v[i]));
  am = fmaxf(am, __shfl_xor_sync(kFull, am, 1));
  am = fmaxf(am, __shfl_xor_sync(kFull, am, 2));
  const unsigned m = __float_as_uint(am);
  const unsigned E = m >> 23;
  return m == 0u ? -127 : (E == 0u ? -126 : (int)E - 126);
}

// Block-floating-point cast trunc(x 2^sh), sh = 30 - emax: 2^sh as one
// factor, or two when sh > 127.
__device__ __forceinline__ void quad_cast(const float* v, int emax, int* c) {
  const int sh = 30 - emax;
  if (emax == -127) {
#pragma unroll
    for (int i = 0; i < 16; i++) c[i] = 0;
  } else if (sh <= 127) {
    const float scl = pow2f(sh);
#pragma unroll
    for (int i = 0; i < 16; i++) c[i] = __float2int_rz(__fmul_rn(v[i], scl));
  } else {
    const float scl = pow2f(sh - 127);
#pragma unroll
    for (int i = 0; i < 16; i++) c[i] = __float2int_rz(__fmul_rn(__fmul_rn(v[i], pow2f(127)), scl));
  }
}

// Lifting along x and y (slice layout), the transpose to the line layout
// through tr (the quad's kZ3BlockWords words), lifting along z, negabinary:
// uu[4z + x] is the coefficient of block index 16z + 4q + x.
__device__ __forceinline__ void quad_transform(int* c, int q, int* tr, unsigned* uu) {
#pragma unroll
  for (int y = 0; y < 4; y++) fwd_lift(c[4 * y], c[4 * y + 1], c[4 * y + 2], c[4 * y + 3]);
#pragma unroll
  for (int x = 0; x < 4; x++) fwd_lift(c[x], c[4 + x], c[8 + x], c[12 + x]);
#pragma unroll
  for (int y = 0; y < 4; y++)
    *reinterpret_cast<int4*>(tr + q * kZ3SliceWords + 4 * y) =
        make_int4(c[4 * y], c[4 * y + 1], c[4 * y + 2], c[4 * y + 3]);
  __syncwarp();
#pragma unroll
  for (int z = 0; z < 4; z++) {
    const int4 t = *reinterpret_cast<const int4*>(tr + z * kZ3SliceWords + 4 * q);
    c[4 * z] = t.x;
    c[4 * z + 1] = t.y;
    c[4 * z + 2] = t.z;
    c[4 * z + 3] = t.w;
  }
  __syncwarp();
#pragma unroll
  for (int x = 0; x < 4; x++) fwd_lift(c[x], c[4 + x], c[8 + x], c[12 + x]);
#pragma unroll
  for (int i = 0; i < 16; i++) uu[i] = to_negabinary(c[i]);
}

// Exact squared truncation errors of the lane's EC-sampled coefficients
// (mask ecm over the line layout), added to the 128-bit (lo, hi) pair.
__device__ __forceinline__ void quad_est_err(const unsigned* uu, int kmin, uint32_t ecm,
                                             unsigned long long& lo, unsigned long long& hi) {
#pragma unroll
  for (int i = 0; i < 16; i++)
    if ((ecm >> i) & 1u) zfp_add_err(uu[i], kmin, lo, hi);
}

// Truncation to the coded planes (in place: a coefficient whose leading one
// is below them counts as zero in every sum that follows), then the rank
// layout through rb (the quad's kZ3RankBytes bytes): cr[j] = leading-one
// position + 1 of rank 16q + j (0 for a zero coefficient).  Returns the
// maximum of cr over the ranks above this lane's (lanes q+1 .. 3).
__device__ __forceinline__ int quad_rank(unsigned* uu, int kmin, int q, const uint32_t* tab,
                                         unsigned char* rb, int* cr) {
  const unsigned keep = kmin >= 32 ? 0u : (0xffffffffu << kmin);
#pragma unroll
  for (int i = 0; i < 16; i++) uu[i] &= keep;
#pragma unroll
  for (int z = 0; z < 4; z++) {
    const uint32_t rz = tab[z];
#pragma unroll
    for (int x = 0; x < 4; x++)
      rb[(rz >> (8 * x)) & 0xffu] = (unsigned char)(32 - __clz((int)uu[4 * z + x]));
  }
  __syncwarp();
  const uint4 cw = *reinterpret_cast<const uint4*>(rb + 16 * q);
  __syncwarp();
  const uint32_t cws[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
  for (int j = 0; j < 16; j++) cr[j] = (int)((cws[j >> 2] >> (8 * (j & 3))) & 0xffu);
  int lmax = 0;
#pragma unroll
  for (int j = 0; j < 16; j += 2) lmax = max(lmax, max(cr[j], cr[j + 1]));
  int s1 = __shfl_down_sync(kFull, lmax, 1);
  s1 = q < 3 ? s1 : 0;
  int s2 = __shfl_down_sync(kFull, max(lmax, s1), 2);
  s2 = q < 2 ? s2 : 0;
  return max(s1, s2);
}

// The lane's share of the doubled interpolated n_sb sum: every rank's weight
// times its n_sb = max(0, cr - kmin).
__device__ __forceinline__ unsigned quad_s2(const int* cr, int kmin, const uint32_t* tab) {
  unsigned s2sum = 0u;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t wk = tab[4 + k];
#pragma unroll
    for (int b = 0; b < 4; b++)
      s2sum += ((wk >> (8 * b)) & 0xffu) * (unsigned)max(0, cr[4 * k + b] - kmin);
  }
  return s2sum;
}

}  // namespace rdk
