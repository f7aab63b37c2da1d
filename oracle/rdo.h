/*
 * rdo.h -- CPU oracle for online SZ-vs-ZFP rate-distortion estimation
 *          (Tao et al., "Optimizing Lossy Compression Rate-Distortion from
 *          Automatic Online Selection between SZ and ZFP", arXiv 1806.08901).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, single-threaded
 * statement of what the GPU path must compute.  Only the test suite, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no header, helper, table or constant generator with the CUDA library:
 * every struct here is declared again, independently, from the paper.
 *
 * All functions take HOST pointers.  Fields are float32, row-major, the last
 * axis fastest; ndim is 1, 2 or 3.  Return value 0 = ok, negative = error
 * (the codes below).
 *
 * Parity unpinned: agreement with the zfp-0.5.0 and SZ-1.4.11 libraries
 * themselves (neither is available); the ZFP-internal rules (precision rule,
 * header bits, lifting steps, sequency order, decode rounding) follow the zfp
 * publication and documentation, and the SZ ground-truth stream costs (escape
 * payload, table and header bits) are this project's readings.
 */
#ifndef RDO_H
#define RDO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RDO_OK 0
#define RDO_ERR_INVALID_ARG (-1)
#define RDO_ERR_NONFINITE (-2)
#define RDO_ERR_RANGE (-7)

#define RDO_EB_REL 0
#define RDO_EB_ABS 1
#define RDO_EC_PAPER 0
#define RDO_EC_ALL 1
#define RDO_SEL_PAPER 0
#define RDO_SEL_HUFFMAN 1

#define RDO_F_CONSTANT 1u
#define RDO_F_DELTA_CLAMPED 2u
#define RDO_F_MSE_ZERO 4u
#define RDO_F_TIE_BAND 8u
#define RDO_F_PARTIAL_BLOCKS 16u

#define RDO_NSYM 65536

typedef struct {
  double eb;            /* error bound: relative to the value range, or absolute */
  int32_t eb_mode;      /* RDO_EB_REL | RDO_EB_ABS */
  int32_t ec_mode;      /* RDO_EC_PAPER (3/9/16 per block) | RDO_EC_ALL */
  double r_sp;          /* block sampling rate, (0, 1] */
  int32_t quant_radius; /* R: |code| < R is coded, else escape; 1..32768 */
  int32_t sel_rule;     /* RDO_SEL_PAPER | RDO_SEL_HUFFMAN */
  double sz_offset;     /* bits/value added to the SZ entropy (0.5) */
} rdo_params;

typedef struct {
  float vmin, vmax;
  double vr, eb_abs, r_sp_eff;
  int32_t strides[3];          /* block sampling strides per axis */
  int32_t minexp;              /* floor(log2 eb_abs) */
  uint64_t n_blocks, n_sampled_blocks;
  /* ZFP estimate */
  double br_zfp, psnr_zfp, mse_sp;
  uint64_t zfp_s2;             /* doubled, interpolated n_sb sum */
  uint64_t zfp_npoints;        /* valid points in sampled blocks */
  uint64_t zfp_ncoeff;         /* EC-sampled coefficients */
  /* SZ estimate */
  double delta, br_sz, br_sz_huff, psnr_sz, entropy;
  uint64_t sz_ns, sz_huff_bits, sz_nesc;
  uint32_t sz_nsym;
  int32_t selection;           /* 0 = SZ, 1 = ZFP */
  uint32_t flags;
} rdo_result;

typedef struct {
  double eb_sz, delta;
  double br_sz_gt, psnr_sz_gt, sse_sz, maxerr_sz;
  uint64_t sz_bits_gt, sz_huff_gt, sz_nesc_gt;
  uint32_t sz_nsym_gt;
  double br_zfp_gt, psnr_zfp_gt, sse_zfp, maxerr_zfp;
  uint64_t zfp_bits_gt;
  int32_t best_gt;             /* 0 = SZ, 1 = ZFP */
  uint32_t flags;
} rdo_truth;

typedef struct {
  int32_t emax, prec, kmin, all_zero;
  int32_t coeff_int[64];       /* after lifting, sequency order */
  uint32_t coeff_nb[64];       /* negabinary, sequency order */
  uint64_t bits_emitter;       /* bit-by-bit group-test simulation */
  uint64_t bits_closed;        /* per-plane closed form */
  int64_t s2_block;            /* doubled interpolated n_sb sum */
  int32_t nsb[64];             /* n_sb for every coefficient */
  int64_t d[64];               /* truncation error, sequency order */
  float recon[64];             /* reconstructed block, block order */
} rdo_block_out;

/* Log-scale quantisation estimate (Section "Estimation Based on Static
 * Quantization", log-scale case), on the same residuals as the linear
 * estimate.  Magnitudes are measured against the unit u = eb_abs (the
 * half-width of SZ's zero bin); with n = quant_radius, the edges are
 * A[k] = u * pow(b, k), k = 1..n, where b is the smallest double >= 1 with
 * A[n] > max |r|.  A residual r gets code 0 when |r| < A[1] (the central bin,
 * width 2 A[1]) and otherwise sign(r) k with k = the number of edges
 * A[1..n-1] at or below |r| (the bin [A[k], A[k+1]), width A[k+1] - A[k]).
 * Symbol = code + 32768 (2n-1 bins, no escapes). */
typedef struct {
  double vr, eb_abs, unit;     /* unit u = eb_abs */
  double max_abs;              /* largest |r| over the sampled points */
  double base;                 /* b */
  double entropy;              /* Eq. (bit-rate-pdf) with P(m_i) = h_i / (N delta_i) */
  double br_log;               /* entropy + sz_offset */
  double br_log_huff;          /* Huffman-coded bits per point */
  double mse_log;              /* Eq. (mse-pdf): sum h_i delta_i^2 / (12 N) */
  double psnr_log;             /* Eq. (psnr-pdf) */
  uint64_t ns, huff_bits;
  uint32_t nsym, flags;
} rdo_log_result;

int rdo_estimate_sz_log(const float* x, int ndim, const int64_t* shape,
                        const rdo_params* p, rdo_log_result* r, uint32_t* hist,
                        double* edges);

/* Algorithm 1 lines 2-12 for one field. hist_est: 65536 counts or NULL. */
int rdo_select(const float* x, int ndim, const int64_t* shape,
               const rdo_params* p, rdo_result* r, uint32_t* hist_est);

/* SZ estimate alone (Alg. 1 lines 8-9) at bin width delta; delta <= 0 uses
 * 2 eb_abs.  Fills the SZ, range and sampling fields of r. */
int rdo_estimate_sz(const float* x, int ndim, const int64_t* shape,
                    const rdo_params* p, double delta, rdo_result* r,
                    uint32_t* hist_est);

/* Full-field ground truth. eb_sz > 0: SZ runs at that bound; eb_sz <= 0: at
 * delta/2 from rdo_select on the same field and params. */
int rdo_ground_truth(const float* x, int ndim, const int64_t* shape,
                     const rdo_params* p, double eb_sz, rdo_truth* t,
                     uint32_t* hist_gt);

/* Classic SZ at the absolute bound eb_sz > 0: prediction from the
 * reconstructed neighbours, point by point in storage order.  Fills the SZ
 * fields of t (eb_sz, delta, sz_*, br_sz_gt, sse_sz, maxerr_sz, psnr_sz_gt);
 * hist: 65536 counts, sym: N symbols (0 = escaped), recon: N floats; each
 * may be NULL. */
int rdo_classic_sz(const float* x, int ndim, const int64_t* shape, const rdo_params* p,
                   double eb_sz, rdo_truth* t, uint32_t* hist, int32_t* sym, float* recon);

/* Per-block ZFP records over all blocks (block order, last axis fastest). */
int rdo_zfp_blocks(const float* x, int ndim, const int64_t* shape,
                   double eb_abs, int32_t* emax, int32_t* prec,
                   uint64_t* bits, uint32_t* coeffs /* nblocks*4^d or NULL */);

/* Per-point SZ symbols.  est_sym: estimator symbol of points inside sampled
 * blocks (strides), -1 elsewhere; gt_sym: ground-truth symbol; recon: the
 * ground-truth reconstruction.  Any output may be NULL. */
int rdo_sz_symbols(const float* x, int ndim, const int64_t* shape,
                   double delta, int32_t quant_radius,
                   const int32_t* strides, int32_t* est_sym, int32_t* gt_sym,
                   float* recon);

int rdo_zfp_block(const float* v, int ndim, int32_t minexp, int32_t ec_mode,
                  rdo_block_out* o);

/* SZ stream of n symbols (0 = escape, stored as the 32-bit pattern of x[i]):
 * header (K, escapes: 32 bits each), table (symbol 16 + code length 6 bits
 * per used symbol, ascending), canonical Huffman payload, escaped values.
 * encode: *nbits = its length; out (cap_bytes, zero-filled first) may be
 * NULL to size it.  decode: sym[n] and the escaped values' bit patterns. */
int rdo_sz_stream_encode(const int32_t* sym, const float* x, int64_t n, uint8_t* out,
                         uint64_t cap_bytes, uint64_t* nbits);
/* ZFP fixed-accuracy stream of a field at eb_abs: per block (the order of
 * rdo_zfp_blocks) a flag bit, then for coded blocks emax + 127 (8 bits) and
 * the group-test embedded coding of the coded planes. */
int rdo_zfp_stream_encode(const float* x, int ndim, const int64_t* shape, double eb_abs,
                          uint8_t* out, uint64_t cap_bytes, uint64_t* nbits);
/* The field a ZFP stream encodes (recon: N floats), from the stream, the
 * shape and eb_abs. */
int rdo_zfp_stream_decode(const uint8_t* in, uint64_t nbits, int ndim, const int64_t* shape,
                          double eb_abs, float* recon);
int rdo_sz_stream_decode(const uint8_t* in, uint64_t nbits, int64_t n, int32_t* sym,
                         uint32_t* esc, uint64_t esc_cap, uint64_t* n_esc);
int rdo_huffman_cost(const uint64_t* counts, int64_t n, uint64_t* cost);
void rdo_fwd_lift(int32_t* v4);
void rdo_inv_lift(int32_t* v4);
uint32_t rdo_int2nb(int32_t i);
int32_t rdo_nb2int(uint32_t u);
int rdo_sequency(int ndim, int32_t* perm);
int rdo_ec_positions(int ndim, int32_t ec_mode, int32_t* pos, int32_t* m);
int rdo_sampling(int ndim, const int64_t* shape, double r_sp,
                 int32_t* strides, uint64_t* n_sampled_blocks,
                 uint64_t* n_points);
/* Exact sum of d[i]^2 * 4^(e[i]-30), e in [-126, 131], rounded once to
 * double (the estimator passes e = block exponent + ndim). */
int rdo_mse_numerator(const int32_t* emax, const int64_t* d, int64_t n,
                      double* out);

#ifdef __cplusplus
}
#endif
#endif
