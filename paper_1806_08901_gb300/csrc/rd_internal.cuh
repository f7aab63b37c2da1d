// rd_internal.cuh -- shared declarations of the rate-distortion estimation
// library's CUDA translation units (device workspace, field descriptor,
// kernel launchers).  Not part of the public ABI (include/rdsel.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include "rdsel.h"

namespace rdk {

constexpr int kNsym = RD_NSYM;
constexpr int kCenter = 32768;       // symbol of code 0
constexpr int kMseBins = 272;        // bin index e + 126, e = emax + d in [-126, 131]
constexpr int kMaxGrid = 4096;       // upper bound of CTAs of a reducing pass
constexpr int kHistWin = 4096;       // shared-memory window of histogram bins
constexpr int kHistWinLo = kCenter - kHistWin / 2;
constexpr int kEntropyCtas = kNsym / 1024;
constexpr int kHuffSmemKeys = 28672; // Huffman with linear queues in shared memory up to this many symbols

// Scalars produced and consumed on the device within one call: nothing
// data-dependent (value range, bin width, error flags) leaves the device
// until the final result copy.
struct Scalars {
  int32_t status;        // RD_OK or an RD_ERR_* code raised on the device
  uint32_t flags;        // RD_F_*
  int32_t constant;      // value range is zero
  int32_t minexp;        // floor(log2 eb_abs)
  uint32_t min_key, max_key, nonfinite;
  uint32_t clean;        // batched estimate: kCleanTables while hist[0], count_of[0] and
                         // present[0] are all zero (the passes that read them clear them)
  uint32_t done[2];       // batched passes: range / ZFP work items finished (last-CTA detection)
  float vmin, vmax, amax;  // amax = max(|vmin|, |vmax|)
  float w, inv, tau;       // SZ quantiser: bin, 1/bin, escape threshold
  double vr, eb_abs, delta, mse_sp;
  unsigned long long s2;         // doubled interpolated n_sb sum
  unsigned long long zfp_bits;   // exact ZFP fixed-accuracy bits
  unsigned int zfp_maxerr;       // float bits of max |x - xhat|
  unsigned int sz_maxerr;
  unsigned int log_maxabs;       // float bits of max |residual| (log-scale estimate)
  uint32_t huff_done;            // Huffman CTAs finished (the last one runs the finish step)
  uint32_t zfp_done;             // CTAs of the truth's ZFP pass finished (the last one writes
                                 // the evaluate step's records)
  unsigned long long mse_lo[kMseBins];  // 128-bit sums of d^2 per exponent
  unsigned long long mse_hi[kMseBins];
};

constexpr uint32_t kCleanTables = 0x6c65616eu;

struct HuffOut {
  unsigned long long ns;    // total count
  unsigned long long cost;  // Huffman-coded bits (sum of internal weights)
  double plogp;             // sum of h log2 h over the bins
  uint32_t nsym;            // nonzero symbols
  uint32_t pad;
};

// The arrays are 16-byte aligned: kernels clear and read them as uint4.
struct Workspace {
  Scalars sc;
  alignas(16) uint32_t hist[2][kNsym];          // 0 = SZ estimate, 1 = SZ ground truth
  double ent_part[2][kEntropyCtas];             // partial sums of h log2 h
  unsigned long long ns_part[2][kEntropyCtas];  // partial sums of h
  HuffOut huff[2];
  double zfp_sse[kMaxGrid];                     // per-CTA partial sums (fixed order)
  double sz_sse[kMaxGrid];
  alignas(16) uint32_t count_of[2][kNsym];      // multiplicity of each count value below 2^16
  alignas(16) uint32_t present[2][kNsym / 32];  // bitmap of the count values present
  uint32_t nbig[2];                             // counts of 2^16 or more
  alignas(16) uint32_t distinct[2][kNsym];      // sorted distinct counts when there are many
  alignas(16) uint32_t sort_scratch[2][kNsym];  // Huffman leaves when K is large
  alignas(16) uint32_t node_scratch[2][kNsym];  // counts >= 2^16, then Huffman internal nodes
  rd_result res;
  rd_truth truth;
};
static_assert(offsetof(Workspace, hist) % 16 == 0 && offsetof(Workspace, count_of) % 16 == 0 &&
                  offsetof(Workspace, present) % 16 == 0 && sizeof(Workspace) % 16 == 0,
              "workspace arrays must be 16-byte aligned");

// Field geometry, passed by value to every kernel.  Axis 0 is the slowest;
// only the first d entries are meaningful.
struct FieldDev {
  const float* x;
  int d;
  int vec_ok;           // rows along the fastest axis are 16-byte aligned
  int n[3];             // extents
  int B[3];             // blocks per axis, ceil(n / 4)
  int s[3];             // block sampling strides
  int L[3];             // sampled blocks per axis, ceil(B / s)
  long long N;          // points
  long long nblocks;    // blocks
  long long nsampled;   // sampled blocks
  // b is a multiple of s[k] iff b == s[k] * (umulhi(b, smag[k]) >> ssh[k])
  // for 0 <= b < 2^31 (ssh[k] < 0: s[k] == 1, every b)
  uint32_t smag[3];
  int32_t ssh[3];
};

struct ParamsDev {
  double eb;
  int eb_mode;
  int ec_mode;
  int R;
  int sel_rule;
  double sz_offset;
};

// One field of a batched call (rd_select_batch), in device memory.
struct BatchField {
  FieldDev f;
  ParamsDev p;
  Workspace* ws;                 // the field's own workspace
  float* res;                    // SZ residuals of the sampled blocks' points (4^d per block)
  unsigned long long ncoeff;     // EC-sampled coefficients (denominator of MSE_sp)
  unsigned long long npoints;    // valid points of the sampled blocks
  uint32_t items_range;          // range work items of the field
  uint32_t items_zfp;            // sampled-block work items of the field
  int32_t need_gt;               // the quantiser is also prepared for the ground truth
  int32_t pad;
};

// A work item of a batched pass: units [begin, end) of one field (values
// for the range pass, sampled blocks for the estimates).
struct BatchItem {
  int32_t field;
  int32_t pad;
  long long begin, end;
};

// Grid bounds computed once per context from the occupancy calculator.
struct LaunchCfg {
  int num_sms;
  int zfp_ctas;   // resident CTAs of the ZFP pass (all SMs)
  int sz_ctas;
  int range_ctas;
};

enum KernelId {
  K_RESET = 0,
  K_RANGE,
  K_ZFP,
  K_DELTA,
  K_SZ_EST,
  K_SZ_GT,
  K_CODE_PREP,
  K_HUFFMAN,
  K_FINISH,
  K_ZFP_INSPECT,
  K_SZ_INSPECT,
  K_B_RESET,
  K_B_RANGE,
  K_B_ZFP,
  K_B_SZ,
  K_B_PREP,
  K_B_FINAL,
  K_B_TRUTH,
  K_SZ_CLASSIC,
  K_SZ_CLASSIC_ERR,
  K_SZ_LOG,
  K_ZFP_EST,
  K_COUNT
};

// Passes of one call, as flags.
enum PassFlags : int {
  P_ZFP_EST = 1,   // ZFP estimate over sampled blocks
  P_ZFP_GT = 2,    // ZFP truth over every block
  P_SZ_EST = 4,    // SZ estimate over points of sampled blocks
  P_SZ_GT = 8,     // SZ truth over every point
  P_SZ_CLASSIC = 16,  // classic SZ truth (prediction from reconstructed values)
};

enum DeltaMode { DELTA_FROM_MSE = 0, DELTA_EXPLICIT = 1, DELTA_FROM_EB_SZ = 2 };

// The bin-width step (delta_warp) that the last CTA of the ZFP pass runs
// when on is set, with the arguments of a separate k_delta launch.
struct DeltaArgs {
  int on, mode;
  double arg;
  int need_quant, need_gt;
  unsigned long long ncoeff, npoints;
};

// ---- launchers (each returns the cudaError_t of the launch) ----
// the table v log2 v (v < 2^16) of the entropy sums, kNsym doubles (once)
cudaError_t launch_init_tables(double* xlogx, cudaStream_t s);
cudaError_t launch_reset(Workspace* ws, cudaStream_t s);
// value range; the CTA that ends last derives VR, eb_abs and minexp.  With
// host_src (pinned host memory holding the field) the pass reads the field
// there and stores it at f.x as it goes.
cudaError_t launch_range(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                         cudaStream_t s, const float* host_src = nullptr);
// ZFP pass; with da.on, its last CTA derives delta
cudaError_t launch_zfp(const FieldDev& f, const ParamsDev& p, int passes, const DeltaArgs& da,
                       Workspace* ws, int ctas, cudaStream_t s, int* grid_used);
cudaError_t launch_delta(const ParamsDev& p, Workspace* ws, int mode, double arg,
                         int need_quant, int need_gt, unsigned long long ncoeff,
                         unsigned long long npoints, cudaStream_t s);
// SZ estimate; ctas from sz_est_occupancy, prepare_sz_est() once per
// device first (128 KB of dynamic shared memory per CTA)
cudaError_t launch_sz_est(const FieldDev& f, const ParamsDev& p, Workspace* ws,
                          int ctas, cudaStream_t s);
cudaError_t prepare_sz_est();
int sz_est_occupancy(int d, int num_sms);
// classic SZ truth: the wavefront launches over the field (their number is
// classic_launches(f)), which write the reconstruction to xh (N floats) and
// the codes to the truth histogram, then the error pass (per-CTA partials)
long long classic_launches(const FieldDev& f);
cudaError_t launch_classic_waves(const FieldDev& f, const ParamsDev& p, float* xh, Workspace* ws,
                                 cudaStream_t s);
cudaError_t launch_classic_err(const FieldDev& f, const float* xh, Workspace* ws, int ctas,
                               cudaStream_t s, int* grid_used);
cudaError_t launch_sz_gt(const FieldDev& f, const ParamsDev& p, int with_est,
                         Workspace* ws, int ctas, cudaStream_t s, int* grid_used);
// Entropy partials and count-of-counts (launch_code_prep), then the Huffman
// cost (launch_huffman), of the histograms in which_mask (bit 0 = estimate,
// bit 1 = ground truth); launch_code_stats issues both.  prepare_code_stats()
// once per device first.
cudaError_t launch_code_prep(Workspace* ws, int which_mask, const double* xlogx, cudaStream_t s);
cudaError_t launch_huffman(Workspace* ws, int which_mask, cudaStream_t s);
cudaError_t launch_code_stats(Workspace* ws, int which_mask, const double* xlogx, cudaStream_t s);
cudaError_t prepare_code_stats();
// The result records and the status of one call, where the host reads them.
struct OutRecords {
  rd_result res;
  rd_truth truth;
  int32_t status;
};
// The finish step; with out (device-visible pinned host memory, or NULL)
// it also writes the records and the status there.
cudaError_t launch_finish(const ParamsDev& p, Workspace* ws, int passes,
                          int zfp_parts, int sz_parts, long long npoints_all,
                          unsigned long long zfp_npoints, OutRecords* out, cudaStream_t s);
// The arguments of the finish step, for the launch that fuses it.
struct FinishArgs {
  ParamsDev p;
  int passes, zfp_parts, sz_parts;
  long long npoints_all;
  unsigned long long zfp_npoints;
  OutRecords* out;
  // 1: the evaluate step with the truth's ZFP pass launched beside the
  // Huffman launch (programmatic dependent launch): the Huffman launch
  // finishes the estimates and the SZ truth only; the ZFP pass's last CTA
  // waits for it, finishes the ZFP truth and writes the records
  int join;
};
// Huffman cost and entropy of the histograms in which_mask, then the finish
// step by the CTA that ends last (one launch fewer than launch_huffman and
// launch_finish).
cudaError_t launch_huffman_finish(Workspace* ws, int which_mask, const FinishArgs& fa,
                                  cudaStream_t s);
cudaError_t launch_zfp_inspect(const FieldDev& f, double eb_abs, int32_t* emax,
                               int32_t* prec, uint64_t* bits, uint32_t* coeffs,
                               cudaStream_t s);
cudaError_t launch_sz_inspect_q(const FieldDev& f, float w, float inv, float tau, int R,
                                int32_t* est_sym, int32_t* gt_sym, float* recon,
                                int use_strides, cudaStream_t s, const Workspace* qws = nullptr);
// SZ pass as a TMA-fed march (2D/3D fields with 16-byte aligned rows);
// prepare_sz_march() once per device first.
bool sz_march_supported(const FieldDev& f);
cudaError_t prepare_sz_march();
cudaError_t launch_sz_march(const FieldDev& f, const ParamsDev& p, int with_est, Workspace* ws,
                            int num_sms, cudaStream_t s, int* grid_used);
int zfp_occupancy(int d, int num_sms);
// the 3D ZFP pass, four lanes per block (launch_zfp dispatches to it)
cudaError_t launch_zfp3(const FieldDev& f, const ParamsDev& p, int passes, const DeltaArgs& da,
                        Workspace* ws, int ctas, cudaStream_t s, int* grid_used,
                        const FinishArgs* join = nullptr);
// The truth's ZFP pass (3D) of the evaluate step, launched right after the
// Huffman launch as its programmatic dependent (it starts once the Huffman
// CTAs run and its last CTA waits for them to complete).
cudaError_t launch_zfp3_after_huffman(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                                      const FinishArgs& fa, cudaStream_t s, int* grid_used);
int zfp3_occupancy(int num_sms);

// ---- log-scale quantisation estimate (rd_sz_log.cu) ----
cudaError_t launch_sz_log_max(const FieldDev& f, Workspace* ws, int ctas, cudaStream_t s);
cudaError_t launch_sz_log_hist(const FieldDev& f, int n, const float* F, Workspace* ws, int ctas,
                               cudaStream_t s);
cudaError_t launch_sz_log_finish(const ParamsDev& p, const double* A, Workspace* ws,
                                 rd_log_result* out, cudaStream_t s);

// ---- batched estimate (rd_select_batch) ----
cudaError_t launch_batch_reset(const BatchField* bf, int n, int need_gt, cudaStream_t s);
// range; the CTA ending a field's last item derives VR, eb_abs, minexp
cudaError_t launch_batch_range(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                               cudaStream_t s);
// sampled blocks of d-dimensional fields (ZFP estimate, stored SZ
// residuals); the CTA ending a field's last item derives delta
cudaError_t launch_batch_blocks(const BatchField* bf, const BatchItem* items, int nitems, int d,
                                int ctas, cudaStream_t s);
// SZ histogram of the stored residuals
cudaError_t launch_batch_sz_hist(const BatchField* bf, const BatchItem* items, int nitems, int ctas,
                                 cudaStream_t s);
// resident CTAs of the item-based passes
// (blocks_ctas: one count per dimensionality 1..3)
void batch_occupancy(int num_sms, int* range_ctas, int* blocks_ctas, int* sz_ctas);
cudaError_t launch_batch_code_prep(const BatchField* bf, int n, const double* xlogx, cudaStream_t s);
// Huffman cost, entropy and finish of every field; result records and
// statuses gathered into res[n] and status[n]
cudaError_t launch_batch_final(const BatchField* bf, int n, rd_result* res, int32_t* status,
                               cudaStream_t s);
// ground-truth records and final statuses of a batch, gathered
cudaError_t launch_batch_truth(const BatchField* bf, int n, rd_truth* truth, int32_t* status,
                               cudaStream_t s);

int sz_occupancy(int d, int num_sms);

// ---------------------------------------------------------------------------
// Host-side argument checks and field geometry, shared by every entry point
// (the context calls, the batch and the static-scratch estimate), so that
// each derives the same lattice and result fields from the same code.
// ---------------------------------------------------------------------------

inline int check_params(const rd_params* p) {
  if (!p) return RD_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return RD_ERR_INVALID_ARG;
  if (p->eb_mode != RD_EB_REL && p->eb_mode != RD_EB_ABS) return RD_ERR_INVALID_ARG;
  if (p->ec_mode != RD_EC_PAPER && p->ec_mode != RD_EC_ALL) return RD_ERR_INVALID_ARG;
  if (!(p->r_sp >= 1e-6 && p->r_sp <= 1.0)) return RD_ERR_INVALID_ARG;
  if (p->quant_radius < 1 || p->quant_radius > 32768) return RD_ERR_INVALID_ARG;
  if (p->sel_rule != RD_SEL_PAPER && p->sel_rule != RD_SEL_HUFFMAN) return RD_ERR_INVALID_ARG;
  if (!isfinite(p->sz_offset)) return RD_ERR_INVALID_ARG;
  return RD_OK;
}

inline ParamsDev params_dev(const rd_params* p) {
  ParamsDev d;
  d.eb = p->eb;
  d.eb_mode = p->eb_mode;
  d.ec_mode = p->ec_mode;
  d.R = p->quant_radius;
  d.sel_rule = p->sel_rule;
  d.sz_offset = p->sz_offset;
  return d;
}

// Block sampling lattice (Section "Data Sampling"): S = round(1/r_sp) is
// factored into primes; each prime, largest first, multiplies the stride of
// the axis with the smallest stride so far (ties: the faster axis).
inline void sampling_strides(int d, double r_sp, int* s) {
  long long S = (long long)floor(1.0 / r_sp + 0.5);
  if (S < 1) S = 1;
  long long f[64];
  int nf = 0;
  long long m = S;
  for (long long q = 2; q * q <= m; q++)
    while (m % q == 0) {
      f[nf++] = q;
      m /= q;
    }
  if (m > 1) f[nf++] = m;
  for (int k = 0; k < 3; k++) s[k] = 1;
  for (int i = nf - 1; i >= 0; i--) {
    int a = d - 1;
    for (int k = d - 2; k >= 0; k--)
      if (s[k] < s[a]) a = k;
    s[a] = (int)(s[a] * f[i]);
  }
}

// EC-sampled coefficients per block: 3/9/16 for 1D/2D/3D, or all 4^d.
inline int ec_count(int d, int ec_mode) {
  if (ec_mode == RD_EC_ALL) return 1 << (2 * d);
  return d == 1 ? 3 : d == 2 ? 9 : 16;
}

// Multiplier and shift that divide any 0 <= b < 2^31 by d exactly:
// with l = ceil(log2 d) and m = floor(2^(31+l) / d) + 1 < 2^32,
// floor(b / d) = floor(b m / 2^(31+l)) = umulhi(b, m) >> (l - 1).
inline void stride_magic(int d, uint32_t* m, int32_t* sh) {
  if (d <= 1) {
    *m = 0u;
    *sh = -1;
    return;
  }
  int l = 0;
  while ((1LL << l) < d) l++;
  *m = (uint32_t)(((unsigned long long)1 << (31 + l)) / (unsigned long long)d + 1ull);
  *sh = l - 1;
}

// Geometry of a field whose values are at x (device): extents (at most
// 2^31 - 1 points), blocks, sampling strides (given, or from r_sp) and
// the valid points of the sampled blocks.
struct FieldGeom {
  FieldDev f;
  unsigned long long npoints_sampled;  // valid points of sampled blocks
  int partial;                         // some extent is not a multiple of 4
};

inline int field_geometry(const rd_field* fld, const float* x, const int* strides_or_null,
                          double r_sp, FieldGeom* g) {
  if (!fld || fld->ndim < 1 || fld->ndim > 3 || !x) return RD_ERR_INVALID_ARG;
  FieldDev& f = g->f;
  memset(&f, 0, sizeof(f));
  f.d = fld->ndim;
  long long N = 1;
  for (int k = 0; k < 3; k++) f.n[k] = 1;
  for (int k = 0; k < f.d; k++) {
    if (fld->shape[k] < 1 || fld->shape[k] > 2147483647LL) return RD_ERR_INVALID_ARG;
    f.n[k] = (int)fld->shape[k];
    N *= fld->shape[k];
    if (N > 2147483647LL) return RD_ERR_INVALID_ARG;
  }
  f.N = N;
  f.x = x;
  f.vec_ok = (((uintptr_t)x & 15u) == 0) && (f.n[f.d - 1] % 4 == 0);
  int st[3] = {1, 1, 1};
  if (strides_or_null) {
    for (int k = 0; k < f.d; k++) {
      if (strides_or_null[k] < 1) return RD_ERR_INVALID_ARG;
      st[k] = strides_or_null[k];
    }
  } else {
    sampling_strides(f.d, r_sp, st);
  }
  f.nblocks = 1;
  f.nsampled = 1;
  g->npoints_sampled = 1;
  g->partial = 0;
  for (int k = 0; k < f.d; k++) {
    f.B[k] = (f.n[k] + 3) / 4;
    f.s[k] = st[k];
    f.L[k] = (f.B[k] + st[k] - 1) / st[k];
    f.nblocks *= f.B[k];
    f.nsampled *= f.L[k];
    stride_magic(st[k], &f.smag[k], &f.ssh[k]);
    unsigned long long pts = 0;
    for (int b = 0; b < f.B[k]; b += st[k])
      pts += (unsigned long long)(f.n[k] - 4 * b < 4 ? f.n[k] - 4 * b : 4);
    g->npoints_sampled *= pts;
    if (f.n[k] % 4) g->partial = 1;
  }
  return RD_OK;
}

// The geometry fields of a result record, which the host fills in after the
// device wrote the rest: strides, block counts, sampling rate and sample
// sizes (a constant field keeps its zeros), and the partial-block flag.
inline void record_geometry(rd_result* r, const FieldGeom& g, bool zfp_est, int ec_mode) {
  const FieldDev& f = g.f;
  for (int k = 0; k < 3; k++) r->strides[k] = k < f.d ? f.s[k] : 0;
  r->n_blocks = (uint64_t)f.nblocks;
  if (!(r->flags & RD_F_CONSTANT)) {
    r->n_sampled_blocks = (uint64_t)f.nsampled;
    r->r_sp_eff = (double)f.nsampled / (double)f.nblocks;
    r->zfp_npoints = g.npoints_sampled;
    if (zfp_est) r->zfp_ncoeff = (unsigned long long)f.nsampled * ec_count(f.d, ec_mode);
  }
  if (g.partial) r->flags |= RD_F_PARTIAL_BLOCKS;
}

}  // namespace rdk
