/*
 * rdsel.h -- C ABI of the GB300 library for online rate-distortion
 * estimation and SZ-vs-ZFP selection (Tao et al., "Optimizing Lossy
 * Compression Rate-Distortion from Automatic Online Selection between SZ and
 * ZFP", arXiv 1806.08901).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Fields are float32, row-major with shape[ndim-1] the fastest axis,
 *    ndim in {1,2,3}, every extent >= 1 and at most 2^31-1 points.  The
 *    caller owns the field memory; the library never writes or frees it.
 *    rd_field.location says whether `data` is a DEVICE pointer (the normal
 *    case) or a HOST pointer, which the library then copies into a staging
 *    buffer it owns inside the context.  For rd_select, rd_ground_truth,
 *    rd_ground_truth_classic, rd_evaluate and rd_rd_curve, a host field in
 *    page-locked (pinned) memory whose address is 16-byte aligned is not
 *    copied separately: the value-range pass reads it from host memory and
 *    stores it into the staging buffer as it goes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is stream-ordered; every entry point synchronises that
 *    stream before it returns and writes its result structs to caller-owned
 *    host memory.
 *  - Return value: RD_OK (0) or a negative RD_ERR_* code; on error the output
 *    structs are zeroed except where stated.  Non-fatal conditions are
 *    reported in the `flags` word of the outputs (RD_F_*).
 *  - One context per host thread; calls on one context must not overlap.
 *  - Every numeric output equals the CPU oracle's bit for bit, except the
 *    float64 sums, which are added in another order: PSNR within 1e-6
 *    relative, entropy and BR_sz within 1e-10 relative, SSE within 1e-6
 *    relative, the largest error within 2^-22 relative.
 */
#ifndef RDSEL_H
#define RDSEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define RD_OK 0
#define RD_ERR_INVALID_ARG (-1) /* bad pointer, shape, or parameter */
#define RD_ERR_NONFINITE (-2)   /* the field holds a NaN or an infinity */
#define RD_ERR_OOM (-3)         /* a device or pinned allocation failed */
#define RD_ERR_BUDGET (-4)      /* the request exceeds the context's HBM budget */
#define RD_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define RD_ERR_TIMEOUT (-6)     /* a bounded device wait ran out */
#define RD_ERR_RANGE (-7)       /* bin width not representable, or codes
                                   would overflow (|x|/bin >= 2^27) */

/* ---- parameter values ------------------------------------------------ */
#define RD_EB_REL 0   /* eb is relative to the value range (Eq. psnr-sz) */
#define RD_EB_ABS 1   /* eb is absolute */
#define RD_EC_PAPER 0 /* 3 / 9 / 16 EC samples per 1D/2D/3D block */
#define RD_EC_ALL 1   /* every coefficient of a sampled block */
#define RD_SEL_PAPER 0   /* SZ iff entropy + offset < mean n_sb (Alg. 1 l.10) */
#define RD_SEL_HUFFMAN 1 /* SZ iff Huffman bits/value < mean n_sb (exact) */
#define RD_LOC_DEVICE 0
#define RD_LOC_HOST 1

/* ---- flags ----------------------------------------------------------- */
#define RD_F_CONSTANT 1u        /* value range 0: nothing estimated, ZFP */
#define RD_F_DELTA_CLAMPED 2u   /* sqrt(12 MSE_sp) > 2 eb_abs: bin = 2 eb_abs */
#define RD_F_MSE_ZERO 4u        /* MSE_sp = 0: bin = 2 eb_abs */
#define RD_F_TIE_BAND 8u        /* |BR_sz - BR_zfp| <= 1e-9: tie, ZFP */
#define RD_F_PARTIAL_BLOCKS 16u /* some extent is not a multiple of 4 */

#define RD_NSYM 65536 /* code alphabet: 0 = escape, q + 32768 otherwise */

typedef struct rd_context rd_context;

typedef struct {
  const float* data;  /* field values (see location) */
  int32_t ndim;       /* 1, 2 or 3 */
  int32_t location;   /* RD_LOC_DEVICE | RD_LOC_HOST */
  int64_t shape[3];   /* shape[0] slowest; entries >= ndim are ignored */
} rd_field;

/* Inputs of Algorithm 1: error bound eb_abs or eb_rel, sampling rates r_sp
 * and r_sp^ec. */
typedef struct {
  double eb;            /* > 0; relative (RD_EB_REL) or absolute */
  int32_t eb_mode;      /* RD_EB_REL | RD_EB_ABS */
  int32_t ec_mode;      /* RD_EC_PAPER | RD_EC_ALL */
  double r_sp;          /* block sampling rate in [1e-6, 1]; paper default 0.05 */
  int32_t quant_radius; /* R in [1, 32768]: codes with |q| >= R escape */
  int32_t sel_rule;     /* RD_SEL_PAPER | RD_SEL_HUFFMAN */
  double sz_offset;     /* bits/value added to the SZ entropy; paper: 0.5 */
} rd_params;

/* Estimates of Algorithm 1 lines 2-12 for one field. */
typedef struct {
  float vmin, vmax;
  double vr, eb_abs, r_sp_eff;
  int32_t strides[3];          /* block sampling strides per axis */
  int32_t minexp;              /* floor(log2 eb_abs) */
  uint64_t n_blocks, n_sampled_blocks;
  double br_zfp, psnr_zfp, mse_sp;  /* ZFP: mean n_sb, PSNR_sp, MSE_sp */
  uint64_t zfp_s2;             /* doubled interpolated n_sb sum */
  uint64_t zfp_npoints;        /* valid points in sampled blocks */
  uint64_t zfp_ncoeff;         /* EC-sampled coefficients */
  double delta;                /* SZ bin width from PSNR_sz = PSNR_zfp */
  double br_sz, br_sz_huff, psnr_sz, entropy;
  uint64_t sz_ns, sz_huff_bits, sz_nesc;
  uint32_t sz_nsym;
  int32_t selection;           /* s_i of Alg. 1 l.15: 0 = SZ, 1 = ZFP */
  uint32_t flags;
} rd_result;

/* Full-field ground truth that judges the estimates. */
typedef struct {
  double eb_sz, delta;         /* SZ bound (= delta/2) and bin width */
  double br_sz_gt, psnr_sz_gt, sse_sz, maxerr_sz;
  uint64_t sz_bits_gt, sz_huff_gt, sz_nesc_gt;
  uint32_t sz_nsym_gt;
  double br_zfp_gt, psnr_zfp_gt, sse_zfp, maxerr_zfp;
  uint64_t zfp_bits_gt;        /* exact fixed-accuracy bits, all blocks */
  int32_t best_gt;             /* 0 = SZ, 1 = ZFP (lower measured bit-rate) */
  uint32_t flags;
} rd_truth;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget bounds the device
 * memory the context may hold (0 = no bound); the fixed workspace (about
 * 2 MB) is allocated here.  Errors: RD_ERR_INVALID_ARG (out NULL or bad
 * device), RD_ERR_OOM, RD_ERR_BUDGET, RD_ERR_CUDA. */
int32_t rd_context_create(int32_t device, size_t hbm_budget, rd_context** out);
int32_t rd_context_destroy(rd_context* ctx);

/* ---- the hot path (Algorithm 1 lines 2-12, and the ground truth) ---- */

/* ZFP estimate, Alg. 1 lines 2-7 (Sections "Estimation Based on Dynamic
 * Quantization" and "Estimation of compression error"): value range, block
 * sampling at r_sp, per 4^d block exponent alignment, lifting transform,
 * sequency order, negabinary bit planes; BR_zfp = mean interpolated n_sb
 * over r_sp^ec-sampled coefficients; PSNR_zfp from the exact MSE_sp; and the
 * SZ bin delta = sqrt(12 MSE_sp) from Eq. (psnr-pdf-linear).  Fills the ZFP
 * fields, delta, vr, eb_abs and the sampling fields of *out. */
int32_t rd_estimate_zfp(rd_context* ctx, const rd_field* field,
                        const rd_params* params, rd_result* out, void* stream);

/* SZ estimate, Alg. 1 lines 8-9 (Sections "Prediction-Based
 * Transformation" and "Estimation Based on Static Quantization"): Lorenzo
 * residuals of the points of sampled blocks from their original neighbours,
 * linear quantisation with bin `delta` (<= 0: 2 eb_abs, SZ's own bin),
 * 65536-symbol histogram, BR_sz = entropy + sz_offset (Eq. bitrate-sz),
 * Huffman-coded bits, PSNR_sz (Eq. psnr-pdf-linear).  Fills the SZ fields,
 * vr, eb_abs, delta and the sampling fields of *out. */
int32_t rd_estimate_sz(rd_context* ctx, const rd_field* field,
                       const rd_params* params, double delta, rd_result* out,
                       void* stream);

/* Algorithm 1 lines 2-12: both estimates and the selection s_i (SZ iff its
 * estimated bit-rate is lower at the matched PSNR; ties go to ZFP). */
int32_t rd_select(rd_context* ctx, const rd_field* field,
                  const rd_params* params, rd_result* out, void* stream);

/* Ground truth over every point: ZFP fixed accuracy at eb_abs (exact
 * embedded-coding bits, reconstruction, SSE, max error) and SZ at the
 * absolute bound eb_sz (prequantised codes, integer Lorenzo residuals,
 * escapes, Huffman-coded bits, SSE, max error).  eb_sz <= 0 runs the ZFP
 * estimate first and uses eb_sz = delta/2 (Alg. 1 l.13, read as delta/2). */
int32_t rd_ground_truth(rd_context* ctx, const rd_field* field,
                        const rd_params* params, double eb_sz,
                        rd_truth* out, void* stream);

/* Classic SZ ground truth (Section "Prediction-Based Transformation"):
 * every point predicted by the Lorenzo predictor from the RECONSTRUCTED
 * values of its preceding neighbours (zero outside the field), the residual
 * quantised with bin w = float(2 eb_sz), the reconstruction pred + q w kept
 * when |q| < quant_radius and |x - (pred + q w)| <= tau (the largest float
 * not above eb_sz (1 - 2^-23)), else the value escapes (symbol 0, stored
 * exactly).  The stream is costed as in rd_ground_truth (Huffman bits +
 * 32 bits per escape + 22 bits per distinct symbol + 64).  This is the
 * serial predictor that rd_ground_truth's prequantised codes stand in for:
 * it measures how far that stand-in is from what a sequential SZ writes.
 *  - eb_sz: the absolute bound, > 0 and finite (else RD_ERR_INVALID_ARG).
 *  - Fills the SZ fields of *out (delta = 2 eb_sz, eb_sz, sz_huff_gt,
 *    sz_nsym_gt, sz_nesc_gt, sz_bits_gt, br_sz_gt, sse_sz, maxerr_sz,
 *    psnr_sz_gt) and flags; the ZFP fields stay 0.  A constant field has
 *    nothing to quantise: flags RD_F_CONSTANT, psnr_sz_gt = +inf, every
 *    other field 0.
 *  - recon: NULL, or DEVICE memory for N floats (caller-owned, the field's
 *    row-major order) that receives the reconstruction a decompressor
 *    would produce (for a constant field: the field itself).
 *  - Device work: the points are taken in dependency wavefronts (1D: one
 *    chain; 2D and 3D: 32x32 tiles of a plane, one launch per wavefront of
 *    tiles, plane + row tile + column tile = w), so the call is far slower than
 *    rd_ground_truth.  The context keeps an N-float reconstruction buffer,
 *    counted against its memory budget (RD_ERR_BUDGET when it would not fit).
 *  - Codes, histogram, escapes, bits and the reconstruction do not depend
 *    on the launch shape (each decision is a fixed sequence of float32
 *    operations); the SSE is a fixed-order float64 sum, so it differs from a
 *    sequential sum by rounding order only.
 *  - Returns once the work on `stream` has finished (the call synchronises
 *    it). */
int32_t rd_ground_truth_classic(rd_context* ctx, const rd_field* field,
                                const rd_params* params, double eb_sz,
                                rd_truth* out, float* recon, void* stream);

/* rd_select followed by rd_ground_truth at delta/2, fused into three passes
 * over the field (range; ZFP estimate + ZFP truth; SZ estimate + SZ truth).
 * Either output may be NULL. */
int32_t rd_evaluate(rd_context* ctx, const rd_field* field,
                    const rd_params* params, rd_result* est,
                    rd_truth* truth, void* stream);

/* rd_select for callers that may not allocate memory.  The paper has no
 * counterpart: this exists for code that runs under a device-memory budget
 * it does not own (an in-situ simulation holding the GPU's memory, a
 * framework whose allocator must serve every allocation) or that cannot take
 * the synchronisation an allocation may imply.  It needs no context and
 * calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating routine:
 * its scratch is fixed arrays inside the library (2.75 MiB of workspace and
 * a 0.5 MiB table), held by every GPU that loads the library until the
 * process exits.
 *  - field: DEVICE memory only (location RD_LOC_HOST is rejected, since a
 *    host field would need a staging buffer), at most 2^31-1 points; larger
 *    or malformed shapes return RD_ERR_INVALID_ARG.  The scratch does not
 *    grow with the field, so no other size limit applies.
 *  - The first call on a device (the current device) resolves the array's
 *    device address, sizes the grids and fills a constant table in the
 *    array (one kernel on the legacy default stream, then a wait for it);
 *    make that first call before any stream capture.  The first call in a
 *    new CUDA context of the device (after cudaDeviceReset, say) does this
 *    set-up again, since the library's device code is loaded afresh there.
 *  - Synchronous: the call waits for its work on `stream` and copies the
 *    record back before it returns.
 *  - Every call shares the array and leaves its contents behind; each call
 *    clears what must start at zero.  Calls that overlap on the GPU (other
 *    streams or host threads) race on the array: serialise them.
 *  - Results equal rd_select's on the same field and parameters (the same
 *    kernels, lattice and record fix-up code). */
int32_t rd_select_static(const rd_field* field, const rd_params* params,
                         rd_result* out, void* stream);

/* ---- log-scale quantisation ------------------------------------------ */

/* Section "Estimation Based on Static Quantization", the log-scale case: the
 * residuals of the linear SZ estimate (the points of the sampled blocks at
 * r_sp, Lorenzo prediction from the original neighbours) binned on a
 * logarithmic scale of 2n-1 bins, n = quant_radius.  The paper's base
 * formula is garbled; the reading taken: magnitudes in units of
 * u = eb_abs, edges A[k] = u * pow(b, k) (float64, k = 1..n) with b the
 * smallest double >= 1 for which A[n] exceeds the largest |r|; code 0 for
 * |r| < A[1] (width 2 A[1]), else sign(r) * k with k the number of edges
 * A[1..n-1] at or below |r| (the bin [A[k], A[k+1])).  No value escapes. */
typedef struct {
  double vr, eb_abs;
  double unit;        /* u = eb_abs */
  double max_abs;     /* largest |r| over the sampled points */
  double base;        /* b */
  double entropy;     /* Eq. (bit-rate-pdf) with the histogram as the PDF */
  double br_log;      /* entropy + params->sz_offset */
  double br_log_huff; /* Huffman-coded bits per sampled point */
  double mse_log;     /* Eq. (mse-pdf): sum h_i delta_i^2 / (12 N_s) */
  double psnr_log;    /* Eq. (psnr-pdf) */
  uint64_t ns, huff_bits;
  uint32_t nsym, flags;
} rd_log_result;

/* The log-scale estimate of one field.  The edge table is derived on the
 * host from the largest residual (one device-to-host copy and wait in the
 * middle of the call); the binning compares each residual with it exactly,
 * so codes, histogram, base and edges equal the CPU oracle's.  A constant
 * field returns RD_F_CONSTANT and an infinite PSNR.  The histogram is left
 * in the context (rd_copy_histograms, the estimate's slot).  Errors as
 * rd_estimate_sz. */
int32_t rd_estimate_sz_log(rd_context* ctx, const rd_field* field,
                           const rd_params* params, rd_log_result* out,
                           void* stream);

/* ---- rate-distortion sweep ------------------------------------------- */

/* One error bound of a sweep (rd_rd_curve). */
typedef struct {
  double eb;            /* the bound, in params->eb_mode */
  rd_result est;        /* Algorithm 1 at eb: selection based on rate-distortion */
  rd_truth truth;       /* ground truth at the matched PSNR (SZ at delta/2, ZFP at
                           eb_abs); truth.best_gt is the "optimum" choice */
  rd_result est_eb;     /* SZ estimate at bin 2 eb_abs: both compressors at the
                           same maximum error */
  rd_truth truth_eb;    /* ground truth at the same maximum error (SZ and ZFP at
                           eb_abs) */
  int32_t selection_eb; /* selection based on error bound, from the estimates:
                           0 = SZ iff its bit-rate (sel_rule) is below br_zfp */
  int32_t best_eb_gt;   /* the same from the ground truth */
} rd_rd_point;

/* Rate-distortion points of one field over the bounds eb[0..n) (evaluation
 * section, "Analysis of Adaptability between Selection Methods Based on
 * Fixed-PSNR vs. Fixed-Maximum-Error", Fig. f9, and the "optimum bar" of
 * Fig. f5): at each bound, rd_evaluate (Algorithm 1 and its ground truth at
 * the matched PSNR), and the selection based on error bound that the paper
 * compares against: SZ with bin 2 eb_abs against ZFP at eb_abs, by
 * estimates and by ground truth (rd_estimate_sz with delta <= 0,
 * rd_ground_truth at eb_sz = eb_abs).  params->eb is ignored; every other
 * parameter applies to every bound.
 *  - field as for rd_select (host fields are copied in for each call);
 *    eb: n host doubles > 0; out: n records, written in order.
 *  - Return: RD_OK, or the first error (out[i..] zeroed from the failing
 *    bound on). */
int32_t rd_rd_curve(rd_context* ctx, const rd_field* field, const rd_params* params,
                    const double* eb, int32_t n, rd_rd_point* out, void* stream);

/* ---- batched estimate ------------------------------------------------ */

/* Work split of the batched estimate.  The results do not depend on it. */
typedef struct {
  int64_t range_values; /* values per range work item (rounded up to a multiple of 4) */
  int32_t zfp_blocks;   /* sampled blocks of a 3D field per work item of the block
                           passes (4^(3-d) times as many for d dimensions) */
  int32_t sz_blocks;    /* the same for the SZ histogram */
  int32_t ctas;         /* cap on each pass's CTAs; 0 = every CTA the SMs hold at once */
  int32_t tuned;        /* output: 1 when the autotuner chose this split */
} rd_batch_config;

/* Algorithm 1 lines 2-12 for n fields at once, e.g. every field of a
 * simulation snapshot, of uneven 2D/3D sizes (the paper's algorithm loops
 * over the fields of a snapshot).  Five launches plus one per dimensionality
 * present cover all fields: a reset; persistent passes over work items of
 * every field (runs of a field's values for the range; runs of its sampled
 * blocks, read once for both estimators, one launch per dimensionality,
 * for the ZFP estimate and the SZ residuals; the stored residuals for the
 * SZ histogram; the CTA that ends a field's last range item derives VR and
 * eb_abs, the one that ends its last block item derives delta); the
 * count-of-counts; one CTA per field for the Huffman cost, entropy, rates,
 * PSNRs and selection.
 *  - fields[i]: DEVICE memory only (RD_ERR_INVALID_ARG otherwise);
 *    params[i]: the parameters of field i.  n >= 1.
 *  - results[n] is required; truths[n] may be NULL, else each field's ground
 *    truth at delta/2 is added as in rd_evaluate; status[n] may be NULL, else
 *    it receives each field's status.
 *  - Return: RD_OK when every field succeeded; else the status of the first
 *    failing field (whose records are zeroed; the others stay valid), or a
 *    call-level error (RD_ERR_INVALID_ARG, _OOM, _BUDGET, _CUDA) with every
 *    record zeroed.
 *  - The context holds one workspace per field (about 2.7 MB each) and caches
 *    a plan per distinct set of fields and parameters, with the stored SZ
 *    residuals of its sampled blocks (4^d words per sampled block: about 5%
 *    of the fields' bytes at r_sp = 0.05, counted against the HBM budget):
 *    the plan's first call runs the autotuner (three work-item sizes, each
 *    run twice, the passes timed, the fastest kept) unless rd_batch_set_config forced a
 *    split; its second call captures a CUDA graph that later calls replay.
 *  - Each field's records equal those of rd_select (and of rd_evaluate for
 *    the truth) on that field alone. */
int32_t rd_select_batch(rd_context* ctx, const rd_field* fields,
                        const rd_params* params, int32_t n, rd_result* results,
                        rd_truth* truths, int32_t* status, void* stream);
/* Force the work split of later batch calls (NULL: autotune, the default).
 * Zero item sizes take the middle of the autotuner's candidates. */
int32_t rd_batch_set_config(rd_context* ctx, const rd_batch_config* cfg);
/* The work split of the last batch call. */
int32_t rd_batch_get_config(rd_context* ctx, rd_batch_config* out);

/* ---- serving loop ----------------------------------------------------- */

/* An in-situ request loop: per-field selection requests (rd_select on one
 * field each) arrive at any time and are served by `slots` host threads,
 * each with its own context and CUDA stream, so that the work of requests
 * in different slots overlaps on the device.  A free slot takes the first
 * admissible request among the first `window` pending ones (continuous
 * admission).  A request on a HOST field keeps a device copy of its field
 * resident under the caller's field key: it is admitted when the key is
 * resident (a hit), or when the HBM budget has room after evicting unpinned
 * resident fields, least recently used first; key 0 makes the copy
 * transient.  A request on a DEVICE field uses the caller's memory and does
 * not count against the budget.  The paper has no serving loop; this is the
 * in-situ deployment of its selection. */
typedef struct rd_server rd_server;

typedef struct {
  int32_t device;
  int32_t slots;        /* concurrent requests on the device, 1..64 */
  int32_t window;       /* pending requests a free slot considers, >= 1 */
  int32_t pad;
  uint64_t hbm_budget;  /* bytes of resident host fields; 0 = no bound */
} rd_server_config;

typedef struct {
  uint64_t request_id, tag;
  int32_t status;        /* RD_OK or the rd_select / copy error of the request */
  int32_t resident_hit;  /* 1: the field was already resident */
  double queue_ms;       /* submission to start of service */
  double service_ms;     /* start of service to completion (copy + estimate) */
  double latency_ms;     /* submission to completion */
  rd_result result;
} rd_server_completion;

typedef struct {
  uint64_t submitted, completed, rejected, pending;
  uint64_t resident_hits, evictions, resident_fields, resident_bytes;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* latency of completed requests */
} rd_server_stats;

/* Start the slots; returns once every slot has reported whether it could
 * create its context and stream.  A slot that could not takes no work (and
 * rd_server_poll then returns RD_ERR_CUDA beside the completions); when no
 * slot could start, the server is torn down and RD_ERR_CUDA returned.
 * Errors: RD_ERR_INVALID_ARG, RD_ERR_CUDA, RD_ERR_OOM. */
int32_t rd_server_create(const rd_server_config* cfg, rd_server** out);
/* Queue a request.  The field memory (host or device) must stay valid and
 * unchanged until the request completes; field_key != 0 names a host field
 * whose device copy may stay resident (the same key must mean the same
 * values).  RD_ERR_BUDGET: a host field larger than the whole budget. */
int32_t rd_server_submit(rd_server* srv, const rd_field* field,
                         const rd_params* params, uint64_t field_key,
                         uint64_t tag, uint64_t* request_id);
/* Take up to max completions (waiting up to wait_ms for the first). */
int32_t rd_server_poll(rd_server* srv, rd_server_completion* out,
                       int32_t max, int32_t wait_ms, int32_t* n);
/* Counters and latency percentiles (nearest rank) since the last reset. */
int32_t rd_server_get_stats(rd_server* srv, rd_server_stats* out);
int32_t rd_server_reset_stats(rd_server* srv);
/* Serve every pending request, stop the slots, free resident copies. */
int32_t rd_server_destroy(rd_server* srv);

/* ---- inspection (same kernels, per-element outputs) ------------------ */

/* Copy the histograms of the last SZ estimate / SZ ground truth run on this
 * context into host arrays of RD_NSYM counts (either may be NULL). */
int32_t rd_copy_histograms(rd_context* ctx, uint32_t* est_hist,
                           uint32_t* gt_hist);

/* Per-block ZFP records for every block (block order, last axis fastest)
 * at absolute bound eb_abs, written to DEVICE arrays owned by the caller:
 * emax[nblocks], prec[nblocks], bits[nblocks], and (optional, may be NULL)
 * the negabinary coefficients in sequency order coeffs[nblocks * 4^ndim]. */
int32_t rd_zfp_blocks(rd_context* ctx, const rd_field* field, double eb_abs,
                      int32_t* emax, int32_t* prec, uint64_t* bits,
                      uint32_t* coeffs, void* stream);

/* Per-point SZ symbols at bin width delta, written to DEVICE arrays of N
 * entries owned by the caller (each may be NULL): est_sym = estimator symbol
 * for points of blocks sampled with `strides` (int32[ndim]), -1 elsewhere;
 * gt_sym = ground-truth symbol; recon = ground-truth reconstruction. */
int32_t rd_sz_symbols(rd_context* ctx, const rd_field* field, double delta,
                      int32_t quant_radius, const int32_t* strides,
                      int32_t* est_sym, int32_t* gt_sym, float* recon,
                      void* stream);

/* ---- profiling ------------------------------------------------------- */

/* Record CUDA events around every kernel launch of this context (off by
 * default).  rd_kernel_stat reports, for i = 0, 1, ..., the kernel's name,
 * its accumulated device time in milliseconds and its launch count since
 * the last reset; RD_ERR_INVALID_ARG past the last kernel. */
int32_t rd_set_profiling(rd_context* ctx, int32_t on);
int32_t rd_reset_profile(rd_context* ctx);
int32_t rd_kernel_stat(rd_context* ctx, int32_t i, const char** name,
                       double* total_ms, int64_t* launches);
/* Kernel launches made by this context since creation. */
int64_t rd_launch_count(rd_context* ctx);

const char* rd_status_string(int32_t status);

#ifdef __cplusplus
}
#endif
#endif /* RDSEL_H */
