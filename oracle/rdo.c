/*
 * rdo.c -- CPU oracle for online SZ-vs-ZFP rate-distortion estimation
 *          (Tao et al., arXiv 1806.08901).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct statement of
 * the per-field hot path (Algorithm 1, lines 2-12) and of the full-field
 * ground truth that judges it.  Only the test suite, the package's smoke
 * check and the benchmark's CPU-baseline leg may load this library; the CUDA
 * product path never does, and the two share no code.
 *
 * Numerics: every floating-point step is written in the order stated here, in
 * IEEE round-to-nearest-even, with contraction disabled (-ffp-contract=off).
 * Quantisation decisions (SZ codes, escape tests) are taken in float32, the
 * precision of the data (the paper fixes none): the plain definition is
 * q = floor(v / delta + 0.5), and the tests bound this evaluation against
 * it in float64 (a code may differ by one bin, only within float32 rounding
 * of a bin edge).  Sums of squared errors, value range and PSNR are in
 * float64.  Integer work (ZFP coefficients, bit counts, histograms) is
 * exact.
 *
 * Parity unpinned (no implementation to compare against): bit-compatibility
 * with zfp-0.5.0 and SZ-1.4.11 themselves.  The ZFP rules marked (Z) are
 * readings of the zfp publication (Lindstrom, IEEE TVCG 2014) and its
 * documentation, restated here; the sequency order is this project's rule.
 */
#include "rdo.h"

#include <float.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Field geometry                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d;          /* number of axes */
  int64_t n[3];   /* n[0] slowest ... n[d-1] fastest */
  int64_t N;      /* number of points */
  const float* x;
} field_t;

static int field_init(field_t* f, const float* x, int ndim,
                      const int64_t* shape) {
  if (!x || !shape || ndim < 1 || ndim > 3) return RDO_ERR_INVALID_ARG;
  f->d = ndim;
  f->x = x;
  f->N = 1;
  for (int k = 0; k < 3; k++) f->n[k] = 1;
  for (int k = 0; k < ndim; k++) {
    if (shape[k] < 1) return RDO_ERR_INVALID_ARG;
    f->n[k] = shape[k];
    f->N *= shape[k];
    if (f->N > 2147483647LL) return RDO_ERR_INVALID_ARG;
  }
  return RDO_OK;
}

static int64_t lin_index(const field_t* f, const int64_t* idx) {
  int64_t l = 0;
  for (int k = 0; k < f->d; k++) l = l * f->n[k] + idx[k];
  return l;
}

/* Value at idx, zero when any coordinate is negative (the Lorenzo stencil
 * reads only preceding neighbours; outside the domain they are zero). */
static float value_or_zero(const field_t* f, const int64_t* idx) {
  for (int k = 0; k < f->d; k++)
    if (idx[k] < 0) return 0.0f;
  return f->x[lin_index(f, idx)];
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 line 2: value range and absolute error bound                 */
/* (Eq. psnr-sz: eb_rel = eb_abs / VR, value-range relative).               */
/* ------------------------------------------------------------------------ */

static int value_range(const field_t* f, float* vmin, float* vmax) {
  float lo = INFINITY, hi = -INFINITY;
  for (int64_t i = 0; i < f->N; i++) {
    float v = f->x[i];
    if (!isfinite(v)) return RDO_ERR_NONFINITE;
    if (v < lo) lo = v;
    if (v > hi) hi = v;
  }
  *vmin = lo;
  *vmax = hi;
  return RDO_OK;
}

/* floor(log2(e)) for e > 0, read from frexp: e = f * 2^k with 1/2 <= f < 1. */
static int floor_log2(double e) {
  int k;
  frexp(e, &k);
  return k - 1;
}

/* ------------------------------------------------------------------------ */
/* Section "Data Sampling for Compression-Quality Estimation": blocks are    */
/* sampled at a fixed distance per axis, different across axes, so that the  */
/* sampled blocks spread uniformly.  Reading: S = round(1/r_sp) is split     */
/* into primes; each prime, largest first, multiplies the stride of the     */
/* axis whose stride is smallest (ties: the faster axis).  A block is        */
/* sampled when every block coordinate is a multiple of its axis' stride.    */
/* ------------------------------------------------------------------------ */

static void sampling_strides(int d, double r_sp, int32_t* s) {
  int64_t S = (int64_t)floor(1.0 / r_sp + 0.5);
  if (S < 1) S = 1;
  int64_t primes[64];
  int np = 0;
  int64_t m = S;
  for (int64_t p = 2; p * p <= m; p++)
    while (m % p == 0) {
      primes[np++] = p;
      m /= p;
    }
  if (m > 1) primes[np++] = m;
  for (int k = 0; k < 3; k++) s[k] = 1;
  for (int i = np - 1; i >= 0; i--) { /* ascending list: walk from largest */
    int best = d - 1;
    for (int k = d - 2; k >= 0; k--)
      if (s[k] < s[best]) best = k;
    s[best] = (int32_t)(s[best] * primes[i]);
  }
}

static int64_t blocks_along(int64_t n) { return (n + 3) / 4; }

static int block_is_sampled(const field_t* f, const int64_t* b,
                            const int32_t* s) {
  for (int k = 0; k < f->d; k++)
    if (b[k] % s[k] != 0) return 0;
  return 1;
}

static int block_has_valid(const field_t* f, const int64_t* b, int t) {
  /* local tuple t (last axis fastest) lies inside the domain? */
  for (int k = f->d - 1; k >= 0; k--) {
    int tk = t & 3;
    t >>= 2;
    if (4 * b[k] + tk >= f->n[k]) return 0;
  }
  return 1;
}

/* Iterate block coordinates in block order (last axis fastest). */
static int next_block(const field_t* f, int64_t* b) {
  for (int k = f->d - 1; k >= 0; k--) {
    if (++b[k] < blocks_along(f->n[k])) return 1;
    b[k] = 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* ZFP block transform.  Section "Block Orthogonal Transformation" (BOT)     */
/* describes the per-axis 4-point transform applied along D_1..D_n; ZFP's    */
/* own transform (Z) is the non-orthogonal lifting scheme of the zfp         */
/* publication, whose forward matrix is                                      */
/*   (1/16) [[4,4,4,4],[5,1,-1,-5],[-4,4,4,-4],[-2,6,-6,2]],                 */
/* computed with integer adds and arithmetic shifts in 32-bit two's          */
/* complement.                                                               */
/* ------------------------------------------------------------------------ */

static int32_t wrap32(int64_t v) { return (int32_t)(uint32_t)(uint64_t)v; }
static int32_t add32(int32_t a, int32_t b) { return wrap32((int64_t)a + b); }
static int32_t sub32(int32_t a, int32_t b) { return wrap32((int64_t)a - b); }
/* arithmetic shift right by one = floor(a / 2) */
static int32_t half32(int32_t a) { return (int32_t)(((int64_t)a - (a & 1)) / 2); }
static int32_t twice32(int32_t a) { return wrap32(2 * (int64_t)a); }

void rdo_fwd_lift(int32_t* v) {
  int32_t a = v[0], b = v[1], c = v[2], d = v[3];
  /* outer pair and inner pair: averages and half-differences */
  a = half32(add32(a, d));
  d = sub32(d, a);
  c = half32(add32(c, b));
  b = sub32(b, c);
  /* combine the two averages, and the two differences */
  a = half32(add32(a, c));
  c = sub32(c, a);
  d = half32(add32(d, b));
  b = sub32(b, d);
  /* final rotation of the two odd-sequency terms */
  d = add32(d, half32(b));
  b = sub32(b, half32(d));
  v[0] = a; v[1] = b; v[2] = c; v[3] = d;
}

void rdo_inv_lift(int32_t* v) {
  int32_t a = v[0], b = v[1], c = v[2], d = v[3];
  /* undo each forward step, last step first */
  b = add32(b, half32(d));
  d = sub32(d, half32(b));
  b = add32(b, d);
  d = sub32(twice32(d), b);
  c = add32(c, a);
  a = sub32(twice32(a), c);
  b = add32(b, c);
  c = sub32(twice32(c), b);
  d = add32(d, a);
  a = sub32(twice32(a), d);
  v[0] = a; v[1] = b; v[2] = c; v[3] = d;
}

static void lift_axis(int32_t* blk, int d, int axis, int inverse) {
  int nb = 1 << (2 * d);
  int stride = 1 << (2 * (d - 1 - axis));
  for (int t = 0; t < nb; t++) {
    if (((t / stride) & 3) != 0) continue;
    int32_t v[4];
    for (int j = 0; j < 4; j++) v[j] = blk[t + j * stride];
    if (inverse)
      rdo_inv_lift(v);
    else
      rdo_fwd_lift(v);
    for (int j = 0; j < 4; j++) blk[t + j * stride] = v[j];
  }
}

/* Sequency order (this project's rule): index tuples (i_0..i_{d-1}), i_0
 * slowest, sorted by the sum of indices, then the sum of squares, then
 * lexicographically with i_0 first. */
static int g_seq_d;
static int seq_key_cmp(const void* pa, const void* pb) {
  int a = *(const int*)pa, b = *(const int*)pb;
  int ta[3], tb[3];
  for (int k = g_seq_d - 1; k >= 0; k--) {
    ta[k] = a & 3; a >>= 2;
    tb[k] = b & 3; b >>= 2;
  }
  int sa = 0, sb = 0, qa = 0, qb = 0;
  for (int k = 0; k < g_seq_d; k++) {
    sa += ta[k]; sb += tb[k];
    qa += ta[k] * ta[k]; qb += tb[k] * tb[k];
  }
  if (sa != sb) return sa < sb ? -1 : 1;
  if (qa != qb) return qa < qb ? -1 : 1;
  for (int k = 0; k < g_seq_d; k++)
    if (ta[k] != tb[k]) return ta[k] < tb[k] ? -1 : 1;
  return 0;
}

int rdo_sequency(int ndim, int32_t* perm) {
  if (ndim < 1 || ndim > 3 || !perm) return RDO_ERR_INVALID_ARG;
  int nb = 1 << (2 * ndim);
  int idx[64];
  for (int t = 0; t < nb; t++) idx[t] = t;
  g_seq_d = ndim;
  qsort(idx, (size_t)nb, sizeof(int), seq_key_cmp);
  for (int p = 0; p < nb; p++) perm[p] = idx[p];
  return RDO_OK;
}

/* Negabinary (Z): u = (i + M) xor M with M = 0xaaaaaaaa, modulo 2^32. */
uint32_t rdo_int2nb(int32_t i) {
  const uint32_t M = 0xaaaaaaaau;
  return ((uint32_t)i + M) ^ M;
}
int32_t rdo_nb2int(uint32_t u) {
  const uint32_t M = 0xaaaaaaaau;
  return (int32_t)((u ^ M) - M);
}

static int msb32(uint32_t u) {
  int b = -1;
  for (int k = 0; k < 32; k++)
    if (u >> k & 1u) b = k;
  return b;
}

/* Section "Estimation Based on Dynamic Quantization": r_sp^ec takes 3 of 4
 * (1D), 9 of 16 (2D), 16 of 64 (3D) coefficients per block.  Reading: the m
 * positions spread evenly over the sequency order,
 *   p_j = floor((j*(Nb-1) + floor((m-1)/2)) / (m-1)),  j = 0..m-1. */
int rdo_ec_positions(int ndim, int32_t ec_mode, int32_t* pos, int32_t* m) {
  if (ndim < 1 || ndim > 3 || !pos || !m) return RDO_ERR_INVALID_ARG;
  int nb = 1 << (2 * ndim);
  int mm = (ec_mode == RDO_EC_ALL) ? nb : (ndim == 1 ? 3 : ndim == 2 ? 9 : 16);
  for (int j = 0; j < mm; j++)
    pos[j] = (j * (nb - 1) + (mm - 1) / 2) / (mm - 1);
  *m = mm;
  return RDO_OK;
}

/* Group-test embedded coding, simulated bit by bit (Z).  For each bit plane
 * from the top down to kmin: the bits of the n coefficients already found
 * significant go out verbatim; then, while coefficients remain, one bit says
 * whether any remaining coefficient has a one in this plane; if so, bits are
 * sent one by one up to and including that one (the last coefficient's one
 * is implied), and everything up to it becomes significant. */
static uint64_t ec_bits_emitter(const uint32_t* u, int nb, int kmin) {
  uint64_t bits = 0;
  int n = 0;
  for (int k = 31; k >= kmin; k--) {
    int x[64];
    for (int j = 0; j < nb; j++) x[j] = (int)(u[j] >> k & 1u);
    bits += (uint64_t)n; /* verbatim bits of significant coefficients */
    int pos = n;
    while (pos < nb) {
      int any = 0;
      for (int j = pos; j < nb; j++) any |= x[j];
      bits += 1; /* group test */
      if (!any) break;
      while (pos < nb - 1) {
        bits += 1;
        if (x[pos]) break;
        pos++;
      }
      pos++;
      n = pos;
    }
  }
  return bits;
}

/* The same cost per plane in closed form: with n significant, m ones at
 * positions >= n, the highest at p:  m == 0 -> n + [n < nb];
 * p == nb-1 -> m + p;  otherwise m + p + 2; then n = p + 1. */
static uint64_t ec_bits_closed(const uint32_t* u, int nb, int kmin) {
  uint64_t bits = 0;
  int n = 0;
  for (int k = 31; k >= kmin; k--) {
    int m = 0, p = -1;
    for (int j = n; j < nb; j++)
      if (u[j] >> k & 1u) {
        m++;
        p = j;
      }
    if (m == 0)
      bits += (uint64_t)(n + (n < nb ? 1 : 0));
    else if (p == nb - 1)
      bits += (uint64_t)(m + p);
    else
      bits += (uint64_t)(m + p + 2);
    if (m > 0) n = p + 1;
  }
  return bits;
}

/* One ZFP block: exponent alignment, block-floating-point cast, lifting,
 * sequency order, negabinary, bit planes and embedded-coding bit count,
 * the estimator's n_sb and truncation error, and the reconstruction. */
int rdo_zfp_block(const float* v, int ndim, int32_t minexp, int32_t ec_mode,
                  rdo_block_out* o) {
  if (!v || !o || ndim < 1 || ndim > 3) return RDO_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  int nb = 1 << (2 * ndim);

  /* (Z) block exponent: largest frexp exponent of a nonzero value,
   * clamped at -126 (subnormal floats). */
  int all_zero = 1, emax = -127;
  for (int t = 0; t < nb; t++) {
    if (v[t] != 0.0f) {
      int e;
      frexp((double)v[t], &e);
      if (e < -126) e = -126;
      if (all_zero || e > emax) emax = e;
      all_zero = 0;
    }
  }
  /* (Z) precision for the absolute error bound 2^minexp:
   * P = clamp(emax - minexp + 2(d+1), 0, 32); planes 31..32-P are coded. */
  int prec = 0;
  if (!all_zero) {
    prec = emax - minexp + 2 * (ndim + 1);
    if (prec < 0) prec = 0;
    if (prec > 32) prec = 32;
  }
  int kmin = 32 - prec;
  o->emax = emax;
  o->prec = prec;
  o->kmin = kmin;
  o->all_zero = all_zero;

  int32_t blk[64];
  if (all_zero) {
    for (int t = 0; t < nb; t++) blk[t] = 0;
  } else {
    /* (Z) block floating point: i = trunc(x * 2^(30 - emax)), exact in
     * double because the factor is a power of two. */
    for (int t = 0; t < nb; t++)
      blk[t] = (int32_t)trunc(ldexp((double)v[t], 30 - emax));
    /* BOT along each axis, fastest axis first. */
    for (int a = ndim - 1; a >= 0; a--) lift_axis(blk, ndim, a, 0);
  }

  int32_t perm[64];
  rdo_sequency(ndim, perm);
  uint32_t u[64], ut[64];
  uint32_t keep = (kmin >= 32) ? 0u : (0xffffffffu << kmin);
  for (int p = 0; p < nb; p++) {
    o->coeff_int[p] = blk[perm[p]];
    u[p] = rdo_int2nb(blk[perm[p]]);
    o->coeff_nb[p] = u[p];
    ut[p] = u[p] & keep; /* planes below kmin are dropped */
    o->d[p] = (int64_t)rdo_nb2int(u[p]) - (int64_t)rdo_nb2int(ut[p]);
    /* n_sb: bits from the leading one down to the last coded plane */
    int b = msb32(u[p]);
    o->nsb[p] = (b >= kmin) ? b - kmin + 1 : 0;
  }

  /* Ground-truth bit count: 1 bit for an empty block, else 1 + 8 exponent
   * bits plus the embedded-coded planes (Z). */
  if (prec == 0) {
    o->bits_emitter = 1;
    o->bits_closed = 1;
  } else {
    o->bits_emitter = 9 + ec_bits_emitter(u, nb, kmin);
    o->bits_closed = 9 + ec_bits_closed(u, nb, kmin);
  }

  /* Estimator: n_sb at the EC-sampled positions, interpolated linearly in
   * sequency index between samples, summed (doubled to stay an integer):
   * a segment [p_j, p_j+L) contributes (L+1)*v_j + (L-1)*v_{j+1}; the last
   * sample contributes 2*v. */
  int32_t pos[64], m;
  rdo_ec_positions(ndim, ec_mode, pos, &m);
  int64_t s2 = 0;
  for (int j = 0; j + 1 < m; j++) {
    int64_t L = pos[j + 1] - pos[j];
    s2 += (L + 1) * o->nsb[pos[j]] + (L - 1) * o->nsb[pos[j + 1]];
  }
  s2 += 2 * (int64_t)o->nsb[pos[m - 1]];
  o->s2_block = s2;

  /* Reconstruction (Z): truncated coefficients, inverse order, inverse
   * lifting slowest axis first, then x = round_float(round_float(i) *
   * 2^(emax-30)). */
  if (all_zero) {
    for (int t = 0; t < nb; t++) o->recon[t] = 0.0f;
  } else {
    int32_t rb[64];
    for (int p = 0; p < nb; p++) rb[perm[p]] = rdo_nb2int(ut[p]);
    for (int a = 0; a < ndim; a++) lift_axis(rb, ndim, a, 1);
    for (int t = 0; t < nb; t++) {
      float fi = (float)rb[t];
      o->recon[t] = (float)ldexp((double)fi, emax - 30);
    }
  }
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact accumulation of the ZFP estimator's squared truncation errors,      */
/* Section "Estimation of compression error" (embedded coding): each sampled */
/* coefficient's error is its truncated integer error scaled by its block's  */
/* exponent.  Theorem 1 carries the error through an ORTHONORMAL BOT; zfp's  */
/* lifting computes 2^-1 times a near-orthonormal 4-point transform per axis */
/* (the 1/2 of the parametric T of Section "Block Orthogonal                 */
/* Transformation"), so a d-dimensional coefficient is rescaled by 2^d       */
/* before squaring.  Term = d^2 * 4^(e-30) with e = emax + d; the sum is     */
/* held as a wide integer with its least significant bit at 2^-312 and      */
/* rounded once to double.                                                  */
/* ------------------------------------------------------------------------ */

#define BIG_LIMBS 24
typedef struct { uint32_t w[BIG_LIMBS]; } big_t;

static void big_add_u32(big_t* a, uint32_t v, int off) {
  int w = off / 32, s = off % 32;
  uint64_t t = (uint64_t)v << s;
  uint64_t carry = 0;
  for (int i = w; i < BIG_LIMBS; i++) {
    uint64_t add = (i == w) ? (t & 0xffffffffu) : (i == w + 1) ? (t >> 32) : 0;
    uint64_t sum = (uint64_t)a->w[i] + add + carry;
    a->w[i] = (uint32_t)sum;
    carry = sum >> 32;
    if (i > w + 1 && carry == 0) break;
  }
}

static void big_add_term(big_t* a, int64_t d, int e) {
  uint64_t m = (uint64_t)(d < 0 ? -d : d);
  /* d^2 fits 64 bits because |d| < 2^32 */
  uint64_t sq = m * m;
  int off = 2 * (e + 126); /* 2(e - 30) + 312 */
  big_add_u32(a, (uint32_t)sq, off);
  big_add_u32(a, (uint32_t)(sq >> 32), off + 32);
}

static double big_to_double(const big_t* a) {
  /* hexadecimal float literal of the exact value; strtod rounds it once
   * to nearest-even */
  char buf[BIG_LIMBS * 8 + 32];
  char* p = buf;
  p += sprintf(p, "0x");
  int top = BIG_LIMBS - 1;
  while (top > 0 && a->w[top] == 0) top--;
  for (int i = top; i >= 0; i--) p += sprintf(p, "%08x", a->w[i]);
  sprintf(p, "p-312");
  return strtod(buf, NULL);
}

int rdo_mse_numerator(const int32_t* emax, const int64_t* d, int64_t n,
                      double* out) {
  if (!emax || !d || !out || n < 0) return RDO_ERR_INVALID_ARG;
  big_t acc;
  memset(&acc, 0, sizeof(acc));
  for (int64_t i = 0; i < n; i++) {
    if (emax[i] < -126 || emax[i] > 131) return RDO_ERR_INVALID_ARG;
    if (d[i] >= 4294967296LL || d[i] <= -4294967296LL) return RDO_ERR_INVALID_ARG;
    big_add_term(&acc, d[i], emax[i]);
  }
  *out = big_to_double(&acc);
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Huffman code cost (Stage III entropy coding).  The total coded length of  */
/* a Huffman code equals the sum of the weights of the internal nodes of its */
/* tree; built here with the two-queue method on sorted counts.              */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : x > y ? 1 : 0;
}

int rdo_huffman_cost(const uint64_t* counts, int64_t n, uint64_t* cost) {
  if (!counts || !cost || n < 0) return RDO_ERR_INVALID_ARG;
  int64_t K = 0;
  for (int64_t i = 0; i < n; i++)
    if (counts[i]) K++;
  *cost = 0;
  if (K == 0) return RDO_OK;
  uint64_t* leaf = (uint64_t*)malloc((size_t)K * sizeof(uint64_t));
  uint64_t* node = (uint64_t*)malloc((size_t)K * sizeof(uint64_t));
  if (!leaf || !node) {
    free(leaf);
    free(node);
    return RDO_ERR_INVALID_ARG;
  }
  int64_t k = 0;
  for (int64_t i = 0; i < n; i++)
    if (counts[i]) leaf[k++] = counts[i];
  if (K == 1) { /* a single symbol still costs one bit per occurrence */
    *cost = leaf[0];
    free(leaf);
    free(node);
    return RDO_OK;
  }
  qsort(leaf, (size_t)K, sizeof(uint64_t), cmp_u64);
  int64_t lh = 0, nh = 0, nt = 0;
  uint64_t total = 0;
  for (int64_t step = 0; step < K - 1; step++) {
    uint64_t pick[2];
    for (int j = 0; j < 2; j++) {
      if (lh < K && (nh >= nt || leaf[lh] <= node[nh]))
        pick[j] = leaf[lh++];
      else
        pick[j] = node[nh++];
    }
    node[nt++] = pick[0] + pick[1];
    total += pick[0] + pick[1];
  }
  *cost = total;
  free(leaf);
  free(node);
  return RDO_OK;
}

/* Eq. (entropy) with Eq. (bitrate-sz): for linear quantisation with the PDF
 * taken from the histogram, P(m_i) = h_i / (N delta), so the bit-rate
 * reduces to the discrete entropy of the bin frequencies. */
static double entropy_bits(const uint32_t* h, uint64_t ns) {
  double H = 0.0;
  for (int s = 0; s < RDO_NSYM; s++) {
    if (!h[s]) continue;
    double p = (double)h[s] / (double)ns;
    H -= p * log2(p);
  }
  return H;
}

static void huffman_of_hist(const uint32_t* h, uint64_t* cost, uint32_t* K) {
  uint64_t* c = (uint64_t*)malloc(RDO_NSYM * sizeof(uint64_t));
  uint32_t k = 0;
  for (int s = 0; s < RDO_NSYM; s++) {
    c[s] = h[s];
    if (h[s]) k++;
  }
  rdo_huffman_cost(c, RDO_NSYM, cost);
  *K = k;
  free(c);
}

/* ------------------------------------------------------------------------ */
/* Parameters                                                               */
/* ------------------------------------------------------------------------ */

static int check_params(const rdo_params* p) {
  if (!p) return RDO_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return RDO_ERR_INVALID_ARG;
  if (p->eb_mode != RDO_EB_REL && p->eb_mode != RDO_EB_ABS)
    return RDO_ERR_INVALID_ARG;
  if (p->ec_mode != RDO_EC_PAPER && p->ec_mode != RDO_EC_ALL)
    return RDO_ERR_INVALID_ARG;
  if (!(p->r_sp >= 1e-6 && p->r_sp <= 1.0)) return RDO_ERR_INVALID_ARG;
  if (p->quant_radius < 1 || p->quant_radius > 32768) return RDO_ERR_INVALID_ARG;
  if (p->sel_rule != RDO_SEL_PAPER && p->sel_rule != RDO_SEL_HUFFMAN)
    return RDO_ERR_INVALID_ARG;
  if (!isfinite(p->sz_offset)) return RDO_ERR_INVALID_ARG;
  return RDO_OK;
}

/* Sampled blocks and the valid points inside them, by enumeration. */
static void sampling_counts(const field_t* f, const int32_t* strides,
                            uint64_t* nsb, uint64_t* npts) {
  int64_t b[3] = {0, 0, 0};
  int nb = 1 << (2 * f->d);
  *nsb = 0;
  *npts = 0;
  do {
    if (!block_is_sampled(f, b, strides)) continue;
    (*nsb)++;
    for (int t = 0; t < nb; t++) *npts += (uint64_t)block_has_valid(f, b, t);
  } while (next_block(f, b));
}

int rdo_sampling(int ndim, const int64_t* shape, double r_sp,
                 int32_t* strides, uint64_t* n_sampled_blocks,
                 uint64_t* n_points) {
  static const float dummy = 0.0f;
  field_t f;
  int rc = field_init(&f, &dummy, ndim, shape);
  if (rc) return rc;
  if (!(r_sp >= 1e-6 && r_sp <= 1.0) || !strides) return RDO_ERR_INVALID_ARG;
  sampling_strides(ndim, r_sp, strides);
  uint64_t nsb = 0, npts = 0;
  sampling_counts(&f, strides, &nsb, &npts);
  if (n_sampled_blocks) *n_sampled_blocks = nsb;
  if (n_points) *n_points = npts;
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* SZ residuals.  Section "Prediction-Based Transformation" (PBT): the        */
/* Lorenzo predictor uses 1/3/7 preceding neighbours in 1D/2D/3D; on the     */
/* sampled points it reads the ORIGINAL neighbours (sampling section).  The  */
/* residual x - pred equals the mixed first difference along every axis;     */
/* it is evaluated here in float32 as nested differences, last axis first:  */
/*   1D: x[j] - x[j-1]                                                      */
/*   2D: (x[i,j]-x[i,j-1]) - (x[i-1,j]-x[i-1,j-1])                           */
/*   3D: the 2D form on plane k minus the 2D form on plane k-1.             */
/* ------------------------------------------------------------------------ */

static float est_residual(const field_t* f, const int64_t* idx) {
  int64_t q[3];
  if (f->d == 1) {
    q[0] = idx[0] - 1;
    return f->x[idx[0]] - value_or_zero(f, q);
  }
  if (f->d == 2) {
    int64_t a[2] = {idx[0], idx[1]};
    int64_t b[2] = {idx[0], idx[1] - 1};
    int64_t c[2] = {idx[0] - 1, idx[1]};
    int64_t e[2] = {idx[0] - 1, idx[1] - 1};
    float row = value_or_zero(f, a) - value_or_zero(f, b);
    float up = value_or_zero(f, c) - value_or_zero(f, e);
    return row - up;
  }
  float plane[2];
  for (int z = 0; z < 2; z++) {
    int64_t k = idx[0] - z;
    int64_t a[3] = {k, idx[1], idx[2]};
    int64_t b[3] = {k, idx[1], idx[2] - 1};
    int64_t c[3] = {k, idx[1] - 1, idx[2]};
    int64_t e[3] = {k, idx[1] - 1, idx[2] - 1};
    float row = value_or_zero(f, a) - value_or_zero(f, b);
    float up = value_or_zero(f, c) - value_or_zero(f, e);
    plane[z] = row - up;
  }
  return plane[0] - plane[1];
}

/* Linear quantisation (Section "Detailed analysis", linear case): bins of
 * width delta centred on zero, code q = round(r / delta) taken as
 * rint(r * (1/delta)) in float32; |q| < R gives symbol q + 32768, else the
 * escape symbol 0. */
static int32_t est_symbol(float r, float inv, int32_t R) {
  float q = rintf(r * inv);
  if (fabsf(q) < (float)R) return (int32_t)q + 32768;
  return 0;
}

/* Integer Lorenzo residual of the prequantised codes, zero outside. */
static int64_t q_at(const field_t* f, const int32_t* Q, const int64_t* idx) {
  for (int k = 0; k < f->d; k++)
    if (idx[k] < 0) return 0;
  return Q[lin_index(f, idx)];
}

static int64_t gt_residual(const field_t* f, const int32_t* Q,
                           const int64_t* idx) {
  /* x - pred(x) = sum over subsets S of the axes of (-1)^|S| Q(idx - e_S) */
  int64_t r = 0;
  for (int sub = 0; sub < (1 << f->d); sub++) {
    int64_t j[3];
    int odd = 0;
    for (int k = 0; k < f->d; k++) {
      int in = (sub >> k) & 1;
      j[k] = idx[k] - in;
      odd ^= in;
    }
    r += odd ? -q_at(f, Q, j) : q_at(f, Q, j);
  }
  return r;
}

typedef struct {
  float w, inv, tau;
} sz_quant_t;

/* Quantiser constants for bin width delta: w = float(delta), 1/w in float,
 * and the escape threshold tau = the largest float <= (delta/2)(1 - 2^-23),
 * so that a float-evaluated |x - xhat| <= tau proves |x - xhat| <= delta/2. */
static int sz_quant_init(double delta, sz_quant_t* q) {
  float w = (float)delta;
  if (!(w >= FLT_MIN) || !isfinite(w)) return RDO_ERR_RANGE;
  float inv = 1.0f / w;
  if (!isfinite(inv) || !(inv >= FLT_MIN)) return RDO_ERR_RANGE;
  double t = (delta / 2.0) * (1.0 - ldexp(1.0, -23));
  float tau = (float)t;
  if ((double)tau > t) tau = nextafterf(tau, 0.0f);
  q->w = w;
  q->inv = inv;
  q->tau = tau;
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* PSNR (Eq. psnr-pdf): PSNR = -20 log10(NRMSE), NRMSE = sqrt(MSE)/VR.       */
/* ------------------------------------------------------------------------ */

static double psnr_of(double vr, double mse) {
  if (mse <= 0.0) return INFINITY;
  return 20.0 * log10(vr) - 10.0 * log10(mse);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, lines 2-12, for one field.                                  */
/* ------------------------------------------------------------------------ */

/* Alg. 1 line 8: histogram of quantised Lorenzo residuals of every valid
 * point of every sampled block (strides in r->strides); line 9: Eq.
 * (bitrate-sz) = entropy, plus the 0.5-bit offset of the evaluation section,
 * and the Huffman-coded cost of the same histogram.  h is zeroed by caller. */
static void sz_estimate(const field_t* f, const rdo_params* p, float inv,
                        rdo_result* r, uint32_t* h) {
  int nb = 1 << (2 * f->d);
  int64_t bb[3] = {0, 0, 0};
  do {
    if (!block_is_sampled(f, bb, r->strides)) continue;
    for (int t = 0; t < nb; t++) {
      if (!block_has_valid(f, bb, t)) continue;
      int64_t idx[3];
      int tt = t;
      for (int k = f->d - 1; k >= 0; k--) {
        idx[k] = 4 * bb[k] + (tt & 3);
        tt >>= 2;
      }
      h[est_symbol(est_residual(f, idx), inv, p->quant_radius)]++;
    }
  } while (next_block(f, bb));
  uint64_t ns = 0;
  for (int s = 0; s < RDO_NSYM; s++) ns += h[s];
  r->sz_ns = ns;
  r->entropy = entropy_bits(h, ns);
  r->br_sz = r->entropy + p->sz_offset;
  huffman_of_hist(h, &r->sz_huff_bits, &r->sz_nsym);
  r->sz_nesc = h[0];
  r->br_sz_huff = (double)(r->sz_huff_bits + 32ull * h[0]) / (double)ns;
}

/* SZ estimate alone at an explicit bin width (delta <= 0: 2 eb_abs, SZ's own
 * bin, for which Eq. (psnr-sz) gives the PSNR). */
int rdo_estimate_sz(const float* x, int ndim, const int64_t* shape,
                    const rdo_params* p, double delta, rdo_result* r,
                    uint32_t* hist_est) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (!r || isnan(delta)) return RDO_ERR_INVALID_ARG;
  memset(r, 0, sizeof(*r));
  if (hist_est) memset(hist_est, 0, RDO_NSYM * sizeof(uint32_t));
  float vmin, vmax;
  if ((rc = value_range(&f, &vmin, &vmax))) return rc;
  r->vmin = vmin;
  r->vmax = vmax;
  r->vr = (double)vmax - (double)vmin;
  r->eb_abs = (p->eb_mode == RDO_EB_REL) ? p->eb * r->vr : p->eb;
  for (int k = 0; k < f.d; k++)
    if (f.n[k] % 4) r->flags |= RDO_F_PARTIAL_BLOCKS;
  uint64_t nblocks = 1;
  for (int k = 0; k < f.d; k++) nblocks *= (uint64_t)blocks_along(f.n[k]);
  r->n_blocks = nblocks;
  sampling_strides(f.d, p->r_sp, r->strides);
  if (r->vr == 0.0) {
    r->flags |= RDO_F_CONSTANT;
    r->psnr_zfp = INFINITY;
    r->psnr_sz = INFINITY;
    r->selection = 1;
    return RDO_OK;
  }
  if (!(r->eb_abs > 0.0) || !isfinite(r->eb_abs)) return RDO_ERR_INVALID_ARG;
  r->minexp = floor_log2(r->eb_abs);
  uint64_t nsb = 0, npts = 0;
  sampling_counts(&f, r->strides, &nsb, &npts);
  r->n_sampled_blocks = nsb;
  r->r_sp_eff = (double)nsb / (double)nblocks;
  r->zfp_npoints = npts;
  r->delta = delta > 0.0 ? delta : 2.0 * r->eb_abs;
  r->psnr_sz = 20.0 * log10(r->vr / r->delta) + 10.0 * log10(12.0);
  sz_quant_t qz;
  if ((rc = sz_quant_init(r->delta, &qz))) return rc;
  uint32_t* h = (uint32_t*)calloc(RDO_NSYM, sizeof(uint32_t));
  if (!h) return RDO_ERR_INVALID_ARG;
  sz_estimate(&f, p, qz.inv, r, h);
  if (hist_est) memcpy(hist_est, h, RDO_NSYM * sizeof(uint32_t));
  free(h);
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Section "Estimation Based on Static Quantization", log-scale case.  The   */
/* paper's bins: the central bin n (width 2b) holds the values the rule     */
/* floor(log_b |x|) sends there, bin n +- i the values with                 */
/* floor(log_b |x|) = i, up to bin 2n-1, so b must carry the largest        */
/* magnitude into the outermost bin.  Its formula for b is garbled; reading: */
/* magnitudes in units of u = eb_abs (so the central bin (-b u, b u) is     */
/* SZ's zero bin (-eb_abs, eb_abs) widened by b, and its width 2b in units   */
/* of u is the paper's delta_n), b the smallest double >= 1 whose edge      */
/* u b^n lies above max|r|, the edges taken                                 */
/* as the doubles u * pow(b, k), and bin n +- k spanning [u b^k, u b^(k+1))  */
/* (the printed width b^i - b^(i-1) is read as the width of the bin that    */
/* floor(log_b) reaches, one index on).                                     */
/* ------------------------------------------------------------------------ */

static double log_edge(double u, double b, int k) { return u * pow(b, (double)k); }

static double log_base(double u, double M, int n) {
  double b = 1.0;
  if (M >= u) {
    b = pow(M / u, 1.0 / (double)n);
    if (!(b >= 1.0)) b = 1.0;
  }
  while (!(log_edge(u, b, n) > M)) b = nextafter(b, INFINITY);
  while (b > 1.0 && log_edge(u, nextafter(b, 0.0), n) > M) b = nextafter(b, 0.0);
  return b;
}

/* Code of residual r: 0 in the central bin, else sign(r) times the number of
 * edges A[1..n-1] at or below |r| (A[0] unused), found by bisection over the
 * non-decreasing table. */
static int32_t log_code(float r, const double* A, int n) {
  double a = fabs((double)r);
  int lo = 0, hi = n - 1; /* answer in [0, n-1] */
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (A[mid] <= a)
      lo = mid;
    else
      hi = mid - 1;
  }
  return r < 0.0f ? -lo : lo;
}

int rdo_estimate_sz_log(const float* x, int ndim, const int64_t* shape,
                        const rdo_params* p, rdo_log_result* r, uint32_t* hist,
                        double* edges) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (!r) return RDO_ERR_INVALID_ARG;
  memset(r, 0, sizeof(*r));
  if (hist) memset(hist, 0, RDO_NSYM * sizeof(uint32_t));
  float vmin, vmax;
  if ((rc = value_range(&f, &vmin, &vmax))) return rc;
  r->vr = (double)vmax - (double)vmin;
  r->eb_abs = (p->eb_mode == RDO_EB_REL) ? p->eb * r->vr : p->eb;
  for (int k = 0; k < f.d; k++)
    if (f.n[k] % 4) r->flags |= RDO_F_PARTIAL_BLOCKS;
  if (r->vr == 0.0) {
    r->flags |= RDO_F_CONSTANT;
    r->psnr_log = INFINITY;
    return RDO_OK;
  }
  if (!(r->eb_abs > 0.0) || !isfinite(r->eb_abs)) return RDO_ERR_INVALID_ARG;
  const int n = p->quant_radius;
  int32_t strides[3];
  sampling_strides(f.d, p->r_sp, strides);
  /* the residuals of every valid point of every sampled block, as the
   * linear estimate computes them */
  int nb = 1 << (2 * f.d);
  float* res = NULL;
  int64_t nres = 0, cap = 0;
  int64_t bb[3] = {0, 0, 0};
  do {
    if (!block_is_sampled(&f, bb, strides)) continue;
    for (int t = 0; t < nb; t++) {
      if (!block_has_valid(&f, bb, t)) continue;
      int64_t idx[3];
      int tt = t;
      for (int k = f.d - 1; k >= 0; k--) {
        idx[k] = 4 * bb[k] + (tt & 3);
        tt >>= 2;
      }
      if (nres == cap) {
        cap = cap ? 2 * cap : 4096;
        float* nr = (float*)realloc(res, (size_t)cap * sizeof(float));
        if (!nr) {
          free(res);
          return RDO_ERR_INVALID_ARG;
        }
        res = nr;
      }
      res[nres++] = est_residual(&f, idx);
    }
  } while (next_block(&f, bb));
  double M = 0.0;
  for (int64_t i = 0; i < nres; i++)
    if (fabs((double)res[i]) > M) M = fabs((double)res[i]);
  const double u = r->eb_abs;
  const double b = log_base(u, M, n);
  double* A = (double*)malloc((size_t)(n + 1) * sizeof(double));
  uint32_t* h = (uint32_t*)calloc(RDO_NSYM, sizeof(uint32_t));
  if (!A || !h) {
    free(A);
    free(h);
    free(res);
    return RDO_ERR_INVALID_ARG;
  }
  A[0] = u;
  for (int k = 1; k <= n; k++) A[k] = log_edge(u, b, k);
  for (int k = 2; k <= n; k++)
    if (A[k] < A[k - 1]) { /* a table the bisection cannot use */
      free(A);
      free(h);
      free(res);
      return RDO_ERR_RANGE;
    }
  for (int64_t i = 0; i < nres; i++) h[log_code(res[i], A, n) + 32768]++;
  uint64_t ns = 0;
  for (int s = 0; s < RDO_NSYM; s++) ns += h[s];
  /* Eq. (mse-pdf) with P(m_i) = h_i / (N delta_i): sum h_i delta_i^2 / (12 N) */
  double sum = 0.0;
  for (int s = 0; s < RDO_NSYM; s++) {
    if (!h[s]) continue;
    int k = s >= 32768 ? s - 32768 : 32768 - s;
    double w = k == 0 ? 2.0 * A[1] : A[k + 1] - A[k];
    sum += (double)h[s] * (w * w);
  }
  r->unit = u;
  r->max_abs = M;
  r->base = b;
  r->ns = ns;
  r->entropy = entropy_bits(h, ns);
  r->br_log = r->entropy + p->sz_offset;
  huffman_of_hist(h, &r->huff_bits, &r->nsym);
  r->br_log_huff = ns ? (double)r->huff_bits / (double)ns : 0.0;
  r->mse_log = ns ? sum / (12.0 * (double)ns) : 0.0;
  r->psnr_log = psnr_of(r->vr, r->mse_log);
  if (hist) memcpy(hist, h, RDO_NSYM * sizeof(uint32_t));
  if (edges)
    for (int k = 1; k <= n; k++) edges[k - 1] = A[k];
  free(A);
  free(h);
  free(res);
  return RDO_OK;
}

static uint64_t u128_lt(uint64_t a_hi, uint64_t a_lo, uint64_t b_hi,
                        uint64_t b_lo) {
  return a_hi < b_hi || (a_hi == b_hi && a_lo < b_lo);
}

static void mul64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 r = (unsigned __int128)a * b;
  *hi = (uint64_t)(r >> 64);
  *lo = (uint64_t)r;
}

int rdo_select(const float* x, int ndim, const int64_t* shape,
               const rdo_params* p, rdo_result* r, uint32_t* hist_est) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (!r) return RDO_ERR_INVALID_ARG;
  memset(r, 0, sizeof(*r));
  if (hist_est) memset(hist_est, 0, RDO_NSYM * sizeof(uint32_t));

  /* line 2: value range and eb */
  float vmin, vmax;
  if ((rc = value_range(&f, &vmin, &vmax))) return rc;
  r->vmin = vmin;
  r->vmax = vmax;
  r->vr = (double)vmax - (double)vmin;
  r->eb_abs = (p->eb_mode == RDO_EB_REL) ? p->eb * r->vr : p->eb;
  for (int k = 0; k < f.d; k++)
    if (f.n[k] % 4) r->flags |= RDO_F_PARTIAL_BLOCKS;
  uint64_t nblocks = 1;
  for (int k = 0; k < f.d; k++) nblocks *= (uint64_t)blocks_along(f.n[k]);
  r->n_blocks = nblocks;
  sampling_strides(f.d, p->r_sp, r->strides);
  if (r->vr == 0.0) {
    /* constant field: nothing to estimate; both rates 0, tie -> ZFP */
    r->flags |= RDO_F_CONSTANT;
    r->psnr_zfp = INFINITY;
    r->psnr_sz = INFINITY;
    r->selection = 1;
    return RDO_OK;
  }
  if (!(r->eb_abs > 0.0) || !isfinite(r->eb_abs)) return RDO_ERR_INVALID_ARG;
  r->minexp = floor_log2(r->eb_abs);

  /* lines 3-6: ZFP on the sampled blocks and EC-sampled coefficients */
  int nb = 1 << (2 * f.d);
  int32_t pos[64], m;
  rdo_ec_positions(f.d, p->ec_mode, pos, &m);
  big_t mse_acc;
  memset(&mse_acc, 0, sizeof(mse_acc));
  uint64_t s2 = 0, npts = 0, nsb = 0;
  int64_t b[3] = {0, 0, 0};
  do {
    if (!block_is_sampled(&f, b, r->strides)) continue;
    float v[64];
    for (int t = 0; t < nb; t++) {
      int64_t idx[3];
      int tt = t;
      for (int k = f.d - 1; k >= 0; k--) {
        int64_t g = 4 * b[k] + (tt & 3);
        tt >>= 2;
        idx[k] = g < f.n[k] ? g : f.n[k] - 1; /* partial block: clamp */
      }
      v[t] = f.x[lin_index(&f, idx)];
      npts += (uint64_t)block_has_valid(&f, b, t);
    }
    rdo_block_out o;
    rdo_zfp_block(v, f.d, r->minexp, p->ec_mode, &o);
    if (o.bits_emitter != o.bits_closed) {
      fprintf(stderr, "rdo: embedded-coding bit counters disagree\n");
      abort();
    }
    s2 += (uint64_t)o.s2_block;
    if (!o.all_zero)
      for (int j = 0; j < m; j++)
        big_add_term(&mse_acc, o.d[pos[j]], o.emax + f.d);
    nsb++;
  } while (next_block(&f, b));
  r->n_sampled_blocks = nsb;
  r->r_sp_eff = (double)nsb / (double)nblocks;
  r->zfp_s2 = s2;
  r->zfp_npoints = npts;
  r->zfp_ncoeff = nsb * (uint64_t)m;
  r->br_zfp = (double)s2 / (2.0 * (double)npts);
  r->mse_sp = big_to_double(&mse_acc) / (double)r->zfp_ncoeff;
  r->psnr_zfp = psnr_of(r->vr, r->mse_sp);

  /* line 7: PSNR_sz = PSNR_zfp in Eq. (psnr-pdf-linear) gives
   * delta^2 = 12 MSE_sp (VR cancels); clamped at 2 eb_abs (SZ's own bin). */
  double delta;
  if (r->mse_sp == 0.0) {
    delta = 2.0 * r->eb_abs;
    r->flags |= RDO_F_MSE_ZERO;
  } else {
    delta = sqrt(12.0 * r->mse_sp);
    if (delta > 2.0 * r->eb_abs) {
      delta = 2.0 * r->eb_abs;
      r->flags |= RDO_F_DELTA_CLAMPED;
    }
  }
  r->delta = delta;
  r->psnr_sz = 20.0 * log10(r->vr / delta) + 10.0 * log10(12.0);
  sz_quant_t qz;
  if ((rc = sz_quant_init(delta, &qz))) return rc;

  /* lines 8-9 */
  uint32_t* h = (uint32_t*)calloc(RDO_NSYM, sizeof(uint32_t));
  if (!h) return RDO_ERR_INVALID_ARG;
  sz_estimate(&f, p, qz.inv, r, h);
  uint64_t ns = r->sz_ns;

  /* lines 10-12: SZ iff its estimated bit-rate is lower; equal -> ZFP */
  if (p->sel_rule == RDO_SEL_PAPER) {
    double diff = r->br_sz - r->br_zfp;
    if (fabs(diff) <= 1e-9) {
      r->flags |= RDO_F_TIE_BAND;
      r->selection = 1;
    } else {
      r->selection = diff < 0.0 ? 0 : 1;
    }
  } else {
    /* (Huff + 32 h0)/N_s < S2/(2 N_z)  <=>  2 (Huff + 32 h0) N_z < S2 N_s */
    uint64_t ahi, alo, bhi, blo;
    mul64(2 * (r->sz_huff_bits + 32ull * h[0]), npts, &ahi, &alo);
    mul64(s2, ns, &bhi, &blo);
    r->selection = u128_lt(ahi, alo, bhi, blo) ? 0 : 1;
  }
  if (hist_est) memcpy(hist_est, h, RDO_NSYM * sizeof(uint32_t));
  free(h);
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Ground truth: full ZFP fixed-accuracy pass and full SZ pass.             */
/* ------------------------------------------------------------------------ */

int rdo_zfp_blocks(const float* x, int ndim, const int64_t* shape,
                   double eb_abs, int32_t* emax, int32_t* prec,
                   uint64_t* bits, uint32_t* coeffs) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if (!(eb_abs > 0.0) || !isfinite(eb_abs)) return RDO_ERR_INVALID_ARG;
  int minexp = floor_log2(eb_abs);
  int nb = 1 << (2 * f.d);
  int64_t b[3] = {0, 0, 0};
  int64_t bi = 0;
  do {
    float v[64];
    for (int t = 0; t < nb; t++) {
      int64_t idx[3];
      int tt = t;
      for (int k = f.d - 1; k >= 0; k--) {
        int64_t g = 4 * b[k] + (tt & 3);
        tt >>= 2;
        idx[k] = g < f.n[k] ? g : f.n[k] - 1;
      }
      v[t] = f.x[lin_index(&f, idx)];
    }
    rdo_block_out o;
    rdo_zfp_block(v, f.d, minexp, RDO_EC_PAPER, &o);
    if (emax) emax[bi] = o.emax;
    if (prec) prec[bi] = o.prec;
    if (bits) bits[bi] = o.bits_closed;
    if (coeffs)
      for (int j = 0; j < nb; j++) coeffs[bi * nb + j] = o.coeff_nb[j];
    bi++;
  } while (next_block(&f, b));
  return RDO_OK;
}

int rdo_sz_symbols(const float* x, int ndim, const int64_t* shape,
                   double delta, int32_t quant_radius, const int32_t* strides,
                   int32_t* est_sym, int32_t* gt_sym, float* recon) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if (quant_radius < 1 || quant_radius > 32768) return RDO_ERR_INVALID_ARG;
  sz_quant_t qz;
  if ((rc = sz_quant_init(delta, &qz))) return rc;
  int32_t* Q = (int32_t*)malloc((size_t)f.N * sizeof(int32_t));
  if (!Q) return RDO_ERR_INVALID_ARG;
  for (int64_t i = 0; i < f.N; i++) Q[i] = (int32_t)rintf(f.x[i] * qz.inv);
  for (int64_t i = 0; i < f.N; i++) {
    int64_t idx[3], rem = i;
    for (int k = f.d - 1; k >= 0; k--) {
      idx[k] = rem % f.n[k];
      rem /= f.n[k];
    }
    if (est_sym) {
      int in = strides != NULL;
      for (int k = 0; k < f.d && in; k++)
        if ((idx[k] / 4) % strides[k]) in = 0;
      est_sym[i] = in ? est_symbol(est_residual(&f, idx), qz.inv, quant_radius)
                      : -1;
    }
    float xh = (float)Q[i] * qz.w;
    float e = f.x[i] - xh;
    int64_t rr = gt_residual(&f, Q, idx);
    int esc = fabsf(e) > qz.tau || rr >= quant_radius || rr <= -quant_radius;
    if (gt_sym) gt_sym[i] = esc ? 0 : (int32_t)(rr + 32768);
    if (recon) recon[i] = esc ? f.x[i] : xh;
  }
  free(Q);
  return RDO_OK;
}

int rdo_ground_truth(const float* x, int ndim, const int64_t* shape,
                     const rdo_params* p, double eb_sz, rdo_truth* t,
                     uint32_t* hist_gt) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (!t) return RDO_ERR_INVALID_ARG;
  memset(t, 0, sizeof(*t));
  if (hist_gt) memset(hist_gt, 0, RDO_NSYM * sizeof(uint32_t));
  if (!(eb_sz > 0.0) && !(eb_sz <= 0.0)) return RDO_ERR_INVALID_ARG; /* NaN */

  float vmin, vmax;
  if ((rc = value_range(&f, &vmin, &vmax))) return rc;
  double vr = (double)vmax - (double)vmin;
  double eb_abs = (p->eb_mode == RDO_EB_REL) ? p->eb * vr : p->eb;
  if (vr == 0.0) {
    t->flags |= RDO_F_CONSTANT;
    t->psnr_sz_gt = INFINITY;
    t->psnr_zfp_gt = INFINITY;
    t->best_gt = 1;
    return RDO_OK;
  }
  if (!(eb_abs > 0.0) || !isfinite(eb_abs)) return RDO_ERR_INVALID_ARG;
  double delta;
  if (eb_sz > 0.0) {
    delta = 2.0 * eb_sz;
  } else {
    rdo_result r;
    if ((rc = rdo_select(x, ndim, shape, p, &r, NULL))) return rc;
    delta = r.delta;
    t->flags |= r.flags & (RDO_F_DELTA_CLAMPED | RDO_F_MSE_ZERO);
  }
  t->delta = delta;
  t->eb_sz = delta / 2.0;
  int minexp = floor_log2(eb_abs);

  /* ZFP fixed accuracy at eb_abs over every block */
  int nb = 1 << (2 * f.d);
  uint64_t zbits = 0;
  double zsse = 0.0, zmax = 0.0;
  int64_t b[3] = {0, 0, 0};
  do {
    float v[64];
    for (int tt0 = 0; tt0 < nb; tt0++) {
      int64_t idx[3];
      int tt = tt0;
      for (int k = f.d - 1; k >= 0; k--) {
        int64_t g = 4 * b[k] + (tt & 3);
        tt >>= 2;
        idx[k] = g < f.n[k] ? g : f.n[k] - 1;
      }
      v[tt0] = f.x[lin_index(&f, idx)];
    }
    rdo_block_out o;
    rdo_zfp_block(v, f.d, minexp, RDO_EC_PAPER, &o);
    if (o.bits_emitter != o.bits_closed) {
      fprintf(stderr, "rdo: embedded-coding bit counters disagree\n");
      abort();
    }
    zbits += o.bits_closed;
    for (int tt0 = 0; tt0 < nb; tt0++) {
      if (!block_has_valid(&f, b, tt0)) continue;
      double e = (double)v[tt0] - (double)o.recon[tt0];
      zsse += e * e;
      if (fabs(e) > zmax) zmax = fabs(e);
    }
  } while (next_block(&f, b));
  t->zfp_bits_gt = zbits;
  t->br_zfp_gt = (double)zbits / (double)f.N;
  t->sse_zfp = zsse;
  t->maxerr_zfp = zmax;
  t->psnr_zfp_gt = psnr_of(vr, zsse / (double)f.N);

  /* SZ at eb_sz = delta/2: prequantise every point, code the integer
   * Lorenzo residuals, escape what the float reconstruction cannot bound */
  sz_quant_t qz;
  if ((rc = sz_quant_init(delta, &qz))) return rc;
  float amax = fabsf(vmin) > fabsf(vmax) ? fabsf(vmin) : fabsf(vmax);
  if (amax * qz.inv > 134217728.0f) return RDO_ERR_RANGE;
  int32_t* sym = (int32_t*)malloc((size_t)f.N * sizeof(int32_t));
  float* rec = (float*)malloc((size_t)f.N * sizeof(float));
  uint32_t* h = (uint32_t*)calloc(RDO_NSYM, sizeof(uint32_t));
  if (!sym || !rec || !h) {
    free(sym);
    free(rec);
    free(h);
    return RDO_ERR_INVALID_ARG;
  }
  rdo_sz_symbols(x, ndim, shape, delta, p->quant_radius, NULL, NULL, sym, rec);
  double ssse = 0.0, smax = 0.0;
  for (int64_t i = 0; i < f.N; i++) {
    h[sym[i]]++;
    double e = (double)f.x[i] - (double)rec[i];
    ssse += e * e;
    if (fabs(e) > smax) smax = fabs(e);
  }
  uint64_t huff;
  uint32_t K;
  huffman_of_hist(h, &huff, &K);
  t->sz_huff_gt = huff;
  t->sz_nsym_gt = K;
  t->sz_nesc_gt = h[0];
  /* stream cost (reading): Huffman payload + 32 bits per escaped value +
   * 22 bits per table entry + a 64-bit header */
  t->sz_bits_gt = huff + 32ull * h[0] + 22ull * K + 64ull;
  t->br_sz_gt = (double)t->sz_bits_gt / (double)f.N;
  t->sse_sz = ssse;
  t->maxerr_sz = smax;
  t->psnr_sz_gt = psnr_of(vr, ssse / (double)f.N);
  t->best_gt = t->br_sz_gt < t->br_zfp_gt ? 0 : 1;
  if (hist_gt) memcpy(hist_gt, h, RDO_NSYM * sizeof(uint32_t));
  free(sym);
  free(rec);
  free(h);
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* Classic SZ ground truth (Section "Prediction-Based Transformation"):      */
/* every point, in storage order, is predicted by the Lorenzo predictor from */
/* the *reconstructed* values of its preceding neighbours (zero outside the  */
/* field), as compression and decompression must predict alike.  The         */
/* residual is quantised with bin w = 2 eb_sz; the reconstruction            */
/* pred + q w is kept when |q| < R and it lies within tau of the value,      */
/* otherwise the value escapes (stored exactly, symbol 0).  Stream cost and  */
/* PSNR as in rdo_ground_truth.                                              */
/* ------------------------------------------------------------------------ */

/* Lorenzo prediction at idx from the reconstruction xh: the neighbours
 * idx - s for the nonzero subsets s of the axes, added when s has an odd
 * number of axes and subtracted when even, in increasing order of s (bit k
 * of s steps back along axis d-1-k), as float operations. */
static float classic_pred(const field_t* f, const float* xh, const int64_t* idx) {
  float pred = 0.0f;
  for (int s = 1; s < (1 << f->d); s++) {
    int64_t j[3];
    int odd = 0, inside = 1;
    for (int k = 0; k < f->d; k++) j[k] = idx[k];
    for (int b = 0; b < f->d; b++) {
      if ((s >> b) & 1) {
        j[f->d - 1 - b] -= 1;
        odd ^= 1;
      }
    }
    for (int k = 0; k < f->d; k++)
      if (j[k] < 0) inside = 0;
    float v = inside ? xh[lin_index(f, j)] : 0.0f;
    pred = odd ? pred + v : pred - v;
  }
  return pred;
}

int rdo_classic_sz(const float* x, int ndim, const int64_t* shape, const rdo_params* p,
                   double eb_sz, rdo_truth* t, uint32_t* hist, int32_t* sym_out, float* recon) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (!t || !(eb_sz > 0.0) || !isfinite(eb_sz)) return RDO_ERR_INVALID_ARG;
  memset(t, 0, sizeof(*t));
  float vmin, vmax;
  if ((rc = value_range(&f, &vmin, &vmax))) return rc;
  double vr = (double)vmax - (double)vmin;
  double delta = 2.0 * eb_sz;
  if (vr == 0.0) {
    /* nothing to quantise: the record holds the flag and PSNR only, as
     * rdo_ground_truth's does */
    t->flags |= RDO_F_CONSTANT;
    t->psnr_sz_gt = INFINITY;
    return RDO_OK;
  }
  t->delta = delta;
  t->eb_sz = eb_sz;
  sz_quant_t qz;
  if ((rc = sz_quant_init(delta, &qz))) return rc;
  float* xh = (float*)malloc((size_t)f.N * sizeof(float));
  uint32_t* h = (uint32_t*)calloc(RDO_NSYM, sizeof(uint32_t));
  if (!xh || !h) {
    free(xh);
    free(h);
    return RDO_ERR_INVALID_ARG;
  }
  const float R = (float)p->quant_radius;
  for (int64_t i = 0; i < f.N; i++) {
    int64_t idx[3], rem = i;
    for (int k = f.d - 1; k >= 0; k--) {
      idx[k] = rem % f.n[k];
      rem /= f.n[k];
    }
    const float pred = classic_pred(&f, xh, idx);
    const float q = rintf((f.x[i] - pred) * qz.inv);
    int sym = 0;
    float rec = f.x[i];
    if (fabsf(q) < R) {
      const float cand = pred + q * qz.w;
      if (fabsf(f.x[i] - cand) <= qz.tau) {
        sym = (int)q + 32768;
        rec = cand;
      }
    }
    xh[i] = rec;
    h[sym]++;
    if (sym_out) sym_out[i] = sym;
  }
  double sse = 0.0, smax = 0.0;
  for (int64_t i = 0; i < f.N; i++) {
    double e = (double)f.x[i] - (double)xh[i];
    sse += e * e;
    if (fabs(e) > smax) smax = fabs(e);
  }
  uint64_t huff;
  uint32_t K;
  huffman_of_hist(h, &huff, &K);
  t->sz_huff_gt = huff;
  t->sz_nsym_gt = K;
  t->sz_nesc_gt = h[0];
  t->sz_bits_gt = huff + 32ull * h[0] + 22ull * K + 64ull;
  t->br_sz_gt = (double)t->sz_bits_gt / (double)f.N;
  t->sse_sz = sse;
  t->maxerr_sz = smax;
  t->psnr_sz_gt = psnr_of(vr, sse / (double)f.N);
  if (hist) memcpy(hist, h, RDO_NSYM * sizeof(uint32_t));
  if (recon) memcpy(recon, xh, (size_t)f.N * sizeof(float));
  free(xh);
  free(h);
  return RDO_OK;
}

/* ------------------------------------------------------------------------ */
/* SZ stream: the stream whose size both SZ ground truths report (the      */
/* paper does not lay out SZ's stream; this project's reading costs it as   */
/* Huffman payload + 32 bits per escaped value + 22 bits per table entry +  */
/* a 64-bit header).  Layout, bits written MSB first:                       */
/*   header   K (32 bits), number of escapes (32 bits)                      */
/*   table    K entries in ascending symbol order: symbol (16), length (6)  */
/*   payload  the canonical Huffman code of every point's symbol, in order */
/*   escapes  the 32-bit pattern of every escaped value (symbol 0), in order*/
/* Code lengths are the leaf depths of a Huffman tree built with a binary   */
/* heap of (weight, node) pairs -- not the two-queue merge that computes    */
/* the cost -- so that the payload length pins that cost.  One symbol alone */
/* gets length 1 (the cost model's one bit per occurrence).                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t w;
  int32_t node;
} heap_item;

static int heap_less(const heap_item* a, const heap_item* b) {
  return a->w < b->w || (a->w == b->w && a->node < b->node);
}

static void heap_push(heap_item* h, int64_t* n, heap_item v) {
  int64_t i = (*n)++;
  h[i] = v;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!heap_less(&h[i], &h[p])) break;
    heap_item t = h[i];
    h[i] = h[p];
    h[p] = t;
    i = p;
  }
}

static heap_item heap_pop(heap_item* h, int64_t* n) {
  heap_item top = h[0];
  h[0] = h[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *n && heap_less(&h[l], &h[m])) m = l;
    if (r < *n && heap_less(&h[r], &h[m])) m = r;
    if (m == i) break;
    heap_item t = h[i];
    h[i] = h[m];
    h[m] = t;
    i = m;
  }
  return top;
}

/* len[s] for every symbol with h[s] > 0 (0 elsewhere); returns K, or -1 on
 * allocation failure or a length above 63 (the table's 6-bit field). */
static int64_t huffman_lengths(const uint32_t* h, uint8_t* len) {
  int64_t K = 0;
  for (int s = 0; s < RDO_NSYM; s++) {
    len[s] = 0;
    if (h[s]) K++;
  }
  if (K == 0) return 0;
  if (K == 1) {
    for (int s = 0; s < RDO_NSYM; s++)
      if (h[s]) len[s] = 1;
    return 1;
  }
  /* nodes 0..K-1 are leaves (symbol in leaf_sym), K..2K-2 internal */
  int32_t* parent = (int32_t*)malloc((size_t)(2 * K) * sizeof(int32_t));
  int32_t* leaf_sym = (int32_t*)malloc((size_t)K * sizeof(int32_t));
  heap_item* heap = (heap_item*)malloc((size_t)K * sizeof(heap_item));
  if (!parent || !leaf_sym || !heap) {
    free(parent);
    free(leaf_sym);
    free(heap);
    return -1;
  }
  int64_t hn = 0, k = 0;
  for (int s = 0; s < RDO_NSYM; s++) {
    if (!h[s]) continue;
    leaf_sym[k] = s;
    heap_item it = {h[s], (int32_t)k};
    heap_push(heap, &hn, it);
    k++;
  }
  int32_t next = (int32_t)K;
  while (hn > 1) {
    heap_item a = heap_pop(heap, &hn), b = heap_pop(heap, &hn);
    parent[a.node] = next;
    parent[b.node] = next;
    heap_item c = {a.w + b.w, next};
    heap_push(heap, &hn, c);
    next++;
  }
  parent[next - 1] = -1; /* the root */
  int ok = 1;
  for (int64_t i = 0; i < K; i++) {
    int d = 0;
    for (int32_t v = (int32_t)i; parent[v] >= 0; v = parent[v]) d++;
    if (d > 63) ok = 0;
    len[leaf_sym[i]] = (uint8_t)d;
  }
  free(parent);
  free(leaf_sym);
  free(heap);
  return ok ? K : -1;
}

/* Canonical codes: symbols in ascending (length, symbol) order take
 * consecutive code values, shifted left whenever the length grows. */
static void canonical_codes(const uint8_t* len, uint64_t* code) {
  uint64_t c = 0;
  int prev = 0, first = 1;
  for (int L = 1; L <= 63; L++) {
    for (int s = 0; s < RDO_NSYM; s++) {
      if (len[s] != L) continue;
      if (first) {
        c = 0;
        first = 0;
      } else {
        c = (c + 1) << (L - prev);
      }
      prev = L;
      code[s] = c;
    }
  }
}

typedef struct {
  uint8_t* buf;
  uint64_t cap_bits, pos;
} bit_writer;

static void put_bits(bit_writer* w, uint64_t v, int nb) {
  for (int i = nb - 1; i >= 0; i--) {
    if (w->buf && w->pos < w->cap_bits) {
      uint8_t bit = (uint8_t)((v >> i) & 1u);
      w->buf[w->pos >> 3] |= (uint8_t)(bit << (7 - (w->pos & 7)));
    }
    w->pos++;
  }
}

int rdo_sz_stream_encode(const int32_t* sym, const float* x, int64_t n, uint8_t* out,
                         uint64_t cap_bytes, uint64_t* nbits) {
  if (!sym || !x || n < 0 || !nbits) return RDO_ERR_INVALID_ARG;
  uint32_t* h = (uint32_t*)calloc(RDO_NSYM, sizeof(uint32_t));
  uint8_t* len = (uint8_t*)malloc(RDO_NSYM);
  uint64_t* code = (uint64_t*)calloc(RDO_NSYM, sizeof(uint64_t));
  if (!h || !len || !code) {
    free(h);
    free(len);
    free(code);
    return RDO_ERR_INVALID_ARG;
  }
  int rc = RDO_OK;
  uint32_t nesc = 0;
  for (int64_t i = 0; i < n; i++) {
    if (sym[i] < 0 || sym[i] >= RDO_NSYM) {
      rc = RDO_ERR_INVALID_ARG;
      break;
    }
    h[sym[i]]++;
    if (sym[i] == 0) nesc++;
  }
  int64_t K = rc ? 0 : huffman_lengths(h, len);
  if (K < 0) rc = RDO_ERR_RANGE;
  if (rc == RDO_OK) {
    canonical_codes(len, code);
    if (out) memset(out, 0, (size_t)cap_bytes);
    bit_writer w = {out, out ? cap_bytes * 8u : 0u, 0u};
    put_bits(&w, (uint64_t)K, 32);
    put_bits(&w, nesc, 32);
    for (int s = 0; s < RDO_NSYM; s++) {
      if (!h[s]) continue;
      put_bits(&w, (uint64_t)s, 16);
      put_bits(&w, len[s], 6);
    }
    for (int64_t i = 0; i < n; i++) put_bits(&w, code[sym[i]], len[sym[i]]);
    for (int64_t i = 0; i < n; i++) {
      if (sym[i] != 0) continue;
      uint32_t b;
      memcpy(&b, &x[i], sizeof(b));
      put_bits(&w, b, 32);
    }
    *nbits = w.pos;
    if (out && w.pos > w.cap_bits) rc = RDO_ERR_RANGE; /* buffer too small */
  }
  free(h);
  free(len);
  free(code);
  return rc;
}

static int get_bits(const uint8_t* buf, uint64_t nbits, uint64_t* pos, int nb, uint64_t* v) {
  if (*pos + (uint64_t)nb > nbits) return 0;
  uint64_t r = 0;
  for (int i = 0; i < nb; i++, (*pos)++) r = (r << 1) | ((buf[*pos >> 3] >> (7 - (*pos & 7))) & 1u);
  *v = r;
  return 1;
}

/* Reads a stream of n symbols back: sym[n], and the escaped values' bit
 * patterns into esc[] (capacity esc_cap; *n_esc their number).  Returns
 * RDO_ERR_INVALID_ARG for a stream that does not parse or has bits left. */
int rdo_sz_stream_decode(const uint8_t* in, uint64_t nbits, int64_t n, int32_t* sym,
                         uint32_t* esc, uint64_t esc_cap, uint64_t* n_esc) {
  if (!in || !sym || n < 0 || !n_esc) return RDO_ERR_INVALID_ARG;
  uint64_t pos = 0, K, ne, v;
  if (!get_bits(in, nbits, &pos, 32, &K) || !get_bits(in, nbits, &pos, 32, &ne)) return RDO_ERR_INVALID_ARG;
  if (K > RDO_NSYM || (K == 0 && n > 0)) return RDO_ERR_INVALID_ARG;
  uint8_t* len = (uint8_t*)calloc(RDO_NSYM, 1);
  uint64_t* code = (uint64_t*)calloc(RDO_NSYM, sizeof(uint64_t));
  if (!len || !code) {
    free(len);
    free(code);
    return RDO_ERR_INVALID_ARG;
  }
  int rc = RDO_OK;
  for (uint64_t k = 0; k < K && rc == RDO_OK; k++) {
    uint64_t s, L;
    if (!get_bits(in, nbits, &pos, 16, &s) || !get_bits(in, nbits, &pos, 6, &L) || L == 0)
      rc = RDO_ERR_INVALID_ARG;
    else
      len[s] = (uint8_t)L;
  }
  if (rc == RDO_OK) canonical_codes(len, code);
  /* the symbols of each length in ascending order hold consecutive codes
   * from the length's smallest: a code c of length L is symbol
   * bylen[first[L] + c - lo[L]] when c - lo[L] < nlen[L] */
  int32_t bylen[RDO_NSYM];
  int64_t first[64], nlen[64];
  uint64_t lo[64];
  int64_t m = 0;
  for (int L = 0; L < 64; L++) {
    first[L] = m;
    nlen[L] = 0;
    lo[L] = 0;
    for (int s = 0; s < RDO_NSYM; s++)
      if (L > 0 && len[s] == L) {
        if (nlen[L] == 0) lo[L] = code[s];
        bylen[m++] = s;
        nlen[L]++;
      }
  }
  /* decode by growing the code one bit at a time */
  for (int64_t i = 0; i < n && rc == RDO_OK; i++) {
    uint64_t c = 0;
    int L = 0, found = -1;
    while (found < 0 && rc == RDO_OK) {
      if (!get_bits(in, nbits, &pos, 1, &v) || ++L > 63) {
        rc = RDO_ERR_INVALID_ARG;
        break;
      }
      c = (c << 1) | v;
      if (nlen[L] > 0 && c >= lo[L] && c - lo[L] < (uint64_t)nlen[L]) found = bylen[first[L] + (int64_t)(c - lo[L])];
    }
    if (rc == RDO_OK) sym[i] = found;
  }
  uint64_t cnt = 0;
  for (int64_t i = 0; i < n && rc == RDO_OK; i++) {
    if (sym[i] != 0) continue;
    if (!get_bits(in, nbits, &pos, 32, &v)) {
      rc = RDO_ERR_INVALID_ARG;
      break;
    }
    if (esc && cnt < esc_cap) esc[cnt] = (uint32_t)v;
    cnt++;
  }
  if (rc == RDO_OK && (cnt != ne || pos != nbits)) rc = RDO_ERR_INVALID_ARG;
  *n_esc = cnt;
  free(len);
  free(code);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* ZFP stream (fixed accuracy; the stream the ZFP ground-truth bit count    */
/* costs).  Blocks in the order of rdo_zfp_blocks; per block: one bit, 0    */
/* for a block with no coded plane (P = 0); else 1, the exponent emax + 127 */
/* (8 bits), and the group-test embedded coding of planes 31 .. kmin of the */
/* negabinary coefficients in sequency order, bits written as the emitter  */
/* above decides them.  The decoder needs the field's shape and eb_abs.     */
/* ------------------------------------------------------------------------ */

static void ec_emit(const uint32_t* u, int nb, int kmin, bit_writer* w) {
  int n = 0;
  for (int k = 31; k >= kmin; k--) {
    int x[64];
    for (int j = 0; j < nb; j++) x[j] = (int)(u[j] >> k & 1u);
    for (int j = 0; j < n; j++) put_bits(w, (uint64_t)x[j], 1); /* verbatim */
    int pos = n;
    while (pos < nb) {
      int any = 0;
      for (int j = pos; j < nb; j++) any |= x[j];
      put_bits(w, (uint64_t)any, 1); /* group test */
      if (!any) break;
      while (pos < nb - 1) {
        put_bits(w, (uint64_t)x[pos], 1);
        if (x[pos]) break;
        pos++;
      }
      pos++;
      n = pos;
    }
  }
}

int rdo_zfp_stream_encode(const float* x, int ndim, const int64_t* shape, double eb_abs,
                          uint8_t* out, uint64_t cap_bytes, uint64_t* nbits) {
  field_t f;
  int rc = field_init(&f, x, ndim, shape);
  if (rc) return rc;
  if (!(eb_abs > 0.0) || !isfinite(eb_abs) || !nbits) return RDO_ERR_INVALID_ARG;
  int minexp = floor_log2(eb_abs);
  int nb = 1 << (2 * f.d);
  if (out) memset(out, 0, (size_t)cap_bytes);
  bit_writer w = {out, out ? cap_bytes * 8u : 0u, 0u};
  int64_t b[3] = {0, 0, 0};
  do {
    float v[64];
    for (int t = 0; t < nb; t++) {
      int64_t idx[3];
      int tt = t;
      for (int k = f.d - 1; k >= 0; k--) {
        int64_t g = 4 * b[k] + (tt & 3);
        tt >>= 2;
        idx[k] = g < f.n[k] ? g : f.n[k] - 1;
      }
      v[t] = f.x[lin_index(&f, idx)];
    }
    rdo_block_out o;
    rdo_zfp_block(v, f.d, minexp, RDO_EC_PAPER, &o);
    if (o.prec == 0) {
      put_bits(&w, 0u, 1);
    } else {
      put_bits(&w, 1u, 1);
      put_bits(&w, (uint64_t)(o.emax + 127), 8);
      ec_emit(o.coeff_nb, nb, o.kmin, &w);
    }
  } while (next_block(&f, b));
  *nbits = w.pos;
  if (out && w.pos > w.cap_bits) return RDO_ERR_RANGE;
  return RDO_OK;
}

/* Reads a fixed-accuracy ZFP stream back into the field it encodes: per
 * block the flag, the exponent and the coded planes (the group tests read
 * as the emitter wrote them), then the block's reconstruction -- the
 * truncated coefficients through the inverse steps of rdo_zfp_block --
 * written to recon at the block's in-field points.  Returns
 * RDO_ERR_INVALID_ARG for a stream that does not parse or has bits left. */
int rdo_zfp_stream_decode(const uint8_t* in, uint64_t nbits, int ndim, const int64_t* shape,
                          double eb_abs, float* recon) {
  if (!in || !recon || !shape || ndim < 1 || ndim > 3) return RDO_ERR_INVALID_ARG;
  if (!(eb_abs > 0.0) || !isfinite(eb_abs)) return RDO_ERR_INVALID_ARG;
  field_t f;
  int rc = field_init(&f, recon, ndim, shape); /* geometry only; recon is written */
  if (rc) return rc;
  const int minexp = floor_log2(eb_abs);
  const int nb = 1 << (2 * f.d);
  int32_t perm[64];
  rdo_sequency(f.d, perm);
  uint64_t pos = 0, v;
  int64_t b[3] = {0, 0, 0};
  do {
    uint32_t u[64];
    for (int j = 0; j < nb; j++) u[j] = 0u;
    int emax = 0, coded = 0;
    if (!get_bits(in, nbits, &pos, 1, &v)) return RDO_ERR_INVALID_ARG;
    if (v) {
      coded = 1;
      if (!get_bits(in, nbits, &pos, 8, &v)) return RDO_ERR_INVALID_ARG;
      emax = (int)v - 127;
      int prec = emax - minexp + 2 * (f.d + 1);
      if (prec < 0) prec = 0;
      if (prec > 32) prec = 32;
      const int kmin = 32 - prec;
      int n = 0;
      for (int k = 31; k >= kmin; k--) {
        for (int j = 0; j < n; j++) {
          if (!get_bits(in, nbits, &pos, 1, &v)) return RDO_ERR_INVALID_ARG;
          u[j] |= (uint32_t)v << k;
        }
        int p = n;
        while (p < nb) {
          if (!get_bits(in, nbits, &pos, 1, &v)) return RDO_ERR_INVALID_ARG;
          if (!v) break;
          while (p < nb - 1) {
            if (!get_bits(in, nbits, &pos, 1, &v)) return RDO_ERR_INVALID_ARG;
            if (v) break;
            p++;
          }
          u[p] |= 1u << k;
          p++;
          n = p;
        }
      }
    }
    float xr[64];
    if (!coded) {
      for (int t = 0; t < nb; t++) xr[t] = 0.0f;
    } else {
      int32_t rb[64];
      for (int p = 0; p < nb; p++) rb[perm[p]] = rdo_nb2int(u[p]);
      for (int a = 0; a < f.d; a++) lift_axis(rb, f.d, a, 1);
      for (int t = 0; t < nb; t++) xr[t] = (float)ldexp((double)(float)rb[t], emax - 30);
    }
    for (int t = 0; t < nb; t++) {
      int64_t idx[3];
      int tt = t, in_field = 1;
      for (int k = f.d - 1; k >= 0; k--) {
        int64_t g = 4 * b[k] + (tt & 3);
        tt >>= 2;
        if (g >= f.n[k]) in_field = 0;
        idx[k] = g;
      }
      if (in_field) recon[lin_index(&f, idx)] = xr[t];
    }
  } while (next_block(&f, b));
  return pos == nbits ? RDO_OK : RDO_ERR_INVALID_ARG;
}
