// rd_zfp_dev.cuh -- the ZFP block computation shared by the ZFP pass, the
// fused batched estimate and the inspector: one thread owns one 4^d block in
// registers (Sections "Block Orthogonal Transformation" and "Estimation
// Based on Dynamic Quantization").
#pragma once

#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

constexpr int kZfpThreads = 128;

// Load a 4^D block with edge clamping (partial blocks replicate the last
// valid sample along each axis).
template <int D>
__device__ __forceinline__ void load_block(const FieldDev& f, const int* b, float* v) {
  const float* __restrict__ x = f.x;
  constexpr int NR = (1 << (2 * D)) / 4;  // rows along the fastest axis
  const int nf = f.n[D - 1];
  const int x0 = 4 * b[D - 1];
#pragma unroll
  for (int r = 0; r < NR; r++) {
    long long row = 0;
    if constexpr (D == 2) {
      int y = min(4 * b[0] + r, f.n[0] - 1);
      row = (long long)y * nf;
    } else if constexpr (D == 3) {
      int z = min(4 * b[0] + (r >> 2), f.n[0] - 1);
      int y = min(4 * b[1] + (r & 3), f.n[1] - 1);
      row = ((long long)z * f.n[1] + y) * nf;
    }
    const float* p = x + row;
    if (f.vec_ok) {
      float4 q = __ldg(reinterpret_cast<const float4*>(p + x0));
      v[4 * r + 0] = q.x;
      v[4 * r + 1] = q.y;
      v[4 * r + 2] = q.z;
      v[4 * r + 3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++) v[4 * r + j] = __ldg(p + min(x0 + j, nf - 1));
    }
  }
}

struct BlockInfo {
  int emax;      // block exponent (-127 for an all-zero block)
  int prec;      // coded planes P
  int kmin;      // lowest coded plane, 32 - P
  int all_zero;
};

// Exponent and precision (zfp fixed-accuracy rule): emax = largest frexp
// exponent of the block's values (>= -126), P = clamp(emax - minexp +
// 2(d+1), 0, 32).
template <int D>
__device__ __forceinline__ BlockInfo block_info(const float* v, int minexp) {
  constexpr int NB = 1 << (2 * D);
  unsigned ebits = 0u, nz = 0u;
#pragma unroll
  for (int t = 0; t < NB; t++) {
    unsigned b = __float_as_uint(v[t]);
    ebits = max(ebits, (b >> 23) & 0xffu);
    nz |= b & 0x7fffffffu;
  }
  BlockInfo bi;
  bi.all_zero = nz == 0u;
  // frexp exponent of a normal float is E - 126; subnormals clamp to -126
  bi.emax = bi.all_zero ? -127 : (ebits == 0u ? -126 : (int)ebits - 126);
  int p = bi.emax - minexp + 2 * (D + 1);
  bi.prec = bi.all_zero ? 0 : min(32, max(0, p));
  bi.kmin = 32 - bi.prec;
  return bi;
}

// Exact group-test embedded-coding cost of the planes 31..kmin, from the
// leading-one position c_j of each coefficient (-1 when below kmin).  With
// M_j the suffix maximum of c, plane k starts with n_k = #{j : M_j > k}
// significant coefficients and finds the ones at positions where c_j = M_j.
// Summed over planes: sum_j max(0, M_j - kmin + 1)  (verbatim bits)
//   + #{planes whose group test ends with 0}       = 31 - max(kmin-1, c_last)
//   + #{j : c_j >= kmin, c_j = M_j}                 (one bit per found one)
//   - [c_last >= kmin]                              (the implied last one).
template <int D>
__device__ __forceinline__ unsigned ec_bits(const int* c, int kmin) {
  constexpr int NB = 1 << (2 * D);
  int M = -1;
  int verbatim = 0, found = 0;
#pragma unroll
  for (int p = NB - 1; p >= 0; p--) {
    M = max(M, c[p]);
    verbatim += max(0, M - kmin + 1);
    found += (c[p] >= kmin && c[p] == M) ? 1 : 0;
  }
  const int last = c[NB - 1];
  int tests = 31 - max(kmin - 1, last);
  return 9u + (unsigned)(verbatim + tests + found - (last >= kmin ? 1 : 0));
}

// The full per-block computation shared by the pass and the inspector.
template <int D>
struct BlockWork {
  static constexpr int NB = 1 << (2 * D);
  unsigned u[NB];    // negabinary, sequency order
  BlockInfo bi;

  __device__ __forceinline__ void forward(const float* v, int minexp) {
    constexpr Sequency<D> S{};
    bi = block_info<D>(v, minexp);
    int c[NB];
    const int sh = 30 - bi.emax;
#pragma unroll
    for (int t = 0; t < NB; t++) c[t] = bi.all_zero ? 0 : cast_scaled(v[t], sh);
    if (!bi.all_zero) fwd_xform<D>(c);
#pragma unroll
    for (int p = 0; p < NB; p++) {
      u[p] = to_negabinary(c[S.perm[p]]);
    }
  }
  __device__ __forceinline__ unsigned keep_mask() const {
    return bi.kmin >= 32 ? 0u : (0xffffffffu << bi.kmin);
  }
  __device__ __forceinline__ unsigned bits() const {
    if (bi.prec == 0) return 1u;
    int c[NB];
#pragma unroll
    for (int p = 0; p < NB; p++) {
      int b = 31 - __clz((int)u[p]);
      c[p] = b >= bi.kmin ? b : -1;
    }
    return ec_bits<D>(c, bi.kmin);
  }
  // Reconstruction of the block (block order) from the truncated planes.
  __device__ __forceinline__ void reconstruct(float* xr) const {
    constexpr Sequency<D> S{};
    if (bi.prec == 0) {
#pragma unroll
      for (int t = 0; t < NB; t++) xr[t] = 0.0f;
      return;
    }
    const unsigned keep = keep_mask();
    int c[NB];
#pragma unroll
    for (int p = 0; p < NB; p++) c[S.perm[p]] = from_negabinary(u[p] & keep);
    inv_xform<D>(c);
    const int e = bi.emax - 30;
#pragma unroll
    for (int t = 0; t < NB; t++) xr[t] = scale_pow2(__int2float_rn(c[t]), e);
  }
};

// Valid-point mask of a (possibly partial) block, bit t for block index t.
template <int D>
__device__ __forceinline__ unsigned long long valid_mask(const FieldDev& f, const int* b) {
  constexpr int NB = 1 << (2 * D);
  int v[3] = {4, 4, 4};
#pragma unroll
  for (int k = 0; k < D; k++) v[k] = min(4, f.n[k] - 4 * b[k]);
  unsigned long long m = 0ull;
#pragma unroll
  for (int t = 0; t < NB; t++) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; k++) ok = ok && (((t >> (2 * (D - 1 - k))) & 3) < v[k]);
    if (ok) m |= 1ull << t;
  }
  return m;
}

template <int D>
__device__ __forceinline__ void decode_block(const FieldDev& f, long long u, bool sampled_only,
                                             int* b) {
  if (sampled_only) {
    long long r = u;
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
      int l = (int)(r % f.L[k]);
      r /= f.L[k];
      b[k] = l * f.s[k];
    }
  } else {
    long long r = u;
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
      b[k] = (int)(r % f.B[k]);
      r /= f.B[k];
    }
  }
}

// Estimator terms of one sampled block (Alg. 1 lines 4-6): the doubled
// interpolated n_sb sum (s2), and the exact sum of the squared truncation
// errors at the EC-sampled coefficients as a 128-bit (lo, hi) pair, which
// belongs to the bin of the block exponent (mse_bin).  uj(j) is the j-th
// sampled coefficient (negabinary): coefficient j of the sequency order
// when every coefficient is sampled, else the one at EC position j.
// Significant bits of coefficient u in the planes kmin..31.
__device__ __forceinline__ int zfp_nsb(unsigned u, int kmin) {
  const int bb = 31 - __clz((int)u);
  return bb >= kmin ? bb - kmin + 1 : 0;
}

// Squared truncation error of coefficient u (planes below kmin dropped)
// added to the 128-bit (lo, hi) pair.
__device__ __forceinline__ void zfp_add_err(unsigned u, int kmin, unsigned long long& lo,
                                            unsigned long long& hi) {
  const unsigned keep = kmin >= 32 ? 0u : (0xffffffffu << kmin);
  long long d = (long long)from_negabinary(u) - (long long)from_negabinary(u & keep);
  unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
  unsigned long long sq = ad * ad;  // |d| < 2^32
  lo += sq;
  hi += (lo < sq);
}

template <int D, class UJ>
__device__ __forceinline__ void zfp_est_terms(int kmin, bool ec_all, UJ uj, long long& s2,
                                              unsigned long long& lo, unsigned long long& hi) {
  constexpr int NB = 1 << (2 * D);
  constexpr EcPositions<D> EC{};
  auto nsb = [&](unsigned u) { return zfp_nsb(u, kmin); };
  s2 = 0;
  lo = 0ull;
  hi = 0ull;
  auto add_err = [&](unsigned u) { zfp_add_err(u, kmin, lo, hi); };
  if (ec_all) {
#pragma unroll
    for (int q = 0; q < NB; q++) {
      const unsigned u = uj(q);
      s2 += 2 * nsb(u);
      add_err(u);
    }
  } else {
#pragma unroll
    for (int j = 0; j < EcPositions<D>::M; j++) {
      const unsigned u = uj(j);
      if (j + 1 < EcPositions<D>::M) {
        const int L = EC.pos[j + 1] - EC.pos[j];
        s2 += (long long)(L + 1) * nsb(u) + (long long)(L - 1) * nsb(uj(j + 1));
      } else {
        s2 += 2 * nsb(u);
      }
      add_err(u);
    }
  }
}

// Bin of the exponent of the 2^d-rescaled error of a block with exponent emax.
template <int D>
__device__ __forceinline__ int mse_bin(int emax) { return emax + D + 126; }

// Adds each lane's 128-bit error sum (when has) to its bin of the shared
// (s_lo, s_hi) arrays.  Every lane of the warp calls.  The blocks of a warp
// share few exponents: for each bin present, the warp sums its lanes' pairs
// with shuffles and one lane adds the total (lanes adding 64-bit words of
// one bin one by one would be serialised).
__device__ __forceinline__ void mse_add_warp(bool has, int bin, unsigned long long lo,
                                             unsigned long long hi, unsigned long long* s_lo,
                                             unsigned long long* s_hi) {
  unsigned pending = __ballot_sync(0xffffffffu, has);
  while (pending) {  // warp-uniform
    const int leader = __ffs(pending) - 1;
    const int b = __shfl_sync(0xffffffffu, bin, leader);
    const bool mine = has && bin == b;
    pending &= ~__ballot_sync(0xffffffffu, mine);
    unsigned long long l = mine ? lo : 0ull, h = mine ? hi : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, l, o);
      const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, h, o);
      const unsigned long long sum = l + l2;
      h += h2 + (sum < l ? 1ull : 0ull);
      l = sum;
    }
    if ((int)(threadIdx.x & 31) == leader) atomic_add_u128(&s_lo[b], &s_hi[b], l, h);
  }
}

}  // namespace rdk
