// rd_internal.cuh -- shared declarations of the rate-distortion estimation
// library's CUDA translation units (device workspace, field descriptor,
// kernel launchers).  Not part of the public ABI (include/rdsel.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

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
// value range; the CTA that ends last derives VR, eb_abs and minexp
cudaError_t launch_range(const FieldDev& f, const ParamsDev& p, Workspace* ws, int ctas,
                         cudaStream_t s);
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
cudaError_t launch_code_prep(Workspace* ws, int which_mask, cudaStream_t s);
cudaError_t launch_huffman(Workspace* ws, int which_mask, const double* xlogx, cudaStream_t s);
cudaError_t launch_code_stats(Workspace* ws, int which_mask, const double* xlogx, cudaStream_t s);
cudaError_t prepare_code_stats();
cudaError_t launch_finish(const ParamsDev& p, Workspace* ws, int passes,
                          int zfp_parts, int sz_parts, long long npoints_all,
                          unsigned long long zfp_npoints, cudaStream_t s);
cudaError_t launch_zfp_inspect(const FieldDev& f, double eb_abs, int32_t* emax,
                               int32_t* prec, uint64_t* bits, uint32_t* coeffs,
                               cudaStream_t s);
cudaError_t launch_sz_inspect_q(const FieldDev& f, float w, float inv, float tau, int R,
                                int32_t* est_sym, int32_t* gt_sym, float* recon,
                                int use_strides, cudaStream_t s);
// SZ pass as a TMA-fed march (2D/3D fields with 16-byte aligned rows);
// prepare_sz_march() once per device first.
bool sz_march_supported(const FieldDev& f);
cudaError_t prepare_sz_march();
cudaError_t launch_sz_march(const FieldDev& f, const ParamsDev& p, int with_est, Workspace* ws,
                            int num_sms, cudaStream_t s, int* grid_used);
int zfp_occupancy(int d, int num_sms);

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
cudaError_t launch_batch_code_prep(const BatchField* bf, int n, cudaStream_t s);
// Huffman cost, entropy and finish of every field; result records and
// statuses gathered into res[n] and status[n]
cudaError_t launch_batch_final(const BatchField* bf, int n, const double* xlogx, rd_result* res,
                               int32_t* status, cudaStream_t s);
// ground-truth records and final statuses of a batch, gathered
cudaError_t launch_batch_truth(const BatchField* bf, int n, rd_truth* truth, int32_t* status,
                               cudaStream_t s);

int sz_occupancy(int d, int num_sms);

}  // namespace rdk
