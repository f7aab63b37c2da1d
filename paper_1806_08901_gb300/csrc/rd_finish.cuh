// rd_finish.cuh -- the finish step of a call (Algorithm 1 lines 10-12 and
// the truth's records): sums of the per-CTA squared errors in a fixed order,
// MSEs and PSNRs, rates, the selection, and the records written into mapped
// host memory.  Shared by the Huffman launch and the truth's ZFP pass, which
// finish their own parts when the evaluate step runs them side by side.
#pragma once

#include <math.h>
#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

constexpr int kFinishThreads = 256;

// Fixed-order block sum (strided per-thread sums, then a fixed tree); the
// result is valid in thread 0.
// Fixed-order sum of a[0..n) by the first kFinishThreads threads of the CTA
// (every thread calls it): the same order whatever the CTA's size, and few
// warps on the SM's narrow float64 pipe.
__device__ inline double block_sum_parts(const double* a, int n, double* red) {
  if (threadIdx.x < kFinishThreads) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += kFinishThreads) v += a[i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kFinishThreads / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// The finish step in two parts.  finish_pre (every thread of the CTA): the
// fields that need no Huffman cost — the truth's squared-error sums (fixed
// order), MSEs and PSNRs, the ZFP truth's rates.  finish_post (warp 0):
// the entropy, rates and selection from the Huffman costs, the SZ truth's
// sizes, the flags.  finish_cta runs both; the fused Huffman launch runs
// the first part in its first CTA before that CTA's own Huffman work.
__device__ inline void finish_pre(Workspace* ws, int passes, int zfp_parts, int sz_parts,
                           long long npoints_all) {
  __shared__ double red[32];
  __shared__ int s_skip;
  Scalars& s = ws->sc;
  // one reading of the status for the whole CTA (a kernel running beside
  // this one may change it)
  if (threadIdx.x == 0) s_skip = (__ldcg(&s.status) != RD_OK || __ldcg(&s.constant)) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;
  rd_truth& t = ws->truth;
  double zsse = 0.0, ssse = 0.0;
  if (passes & P_ZFP_GT) zsse = block_sum_parts(ws->zfp_sse, zfp_parts, red);
  if (passes & P_SZ_GT) ssse = block_sum_parts(ws->sz_sse, sz_parts, red);
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  // the logarithms in separate lanes: 0 VR, 2 ZFP truth MSE, 3 SZ truth MSE
  const double mse_z = zsse / (double)npoints_all;
  const double mse_s = ssse / (double)npoints_all;
  const double larg = lane == 0 ? s.vr : lane == 2 ? mse_z : mse_s;
  const double lg2 = log2(larg);
  const double kLog10of2 = 0.30102999566398119521;
  const double l_vr = __shfl_sync(0xffffffffu, lg2, 0) * kLog10of2;
  const double l_mz = __shfl_sync(0xffffffffu, lg2, 2) * kLog10of2;
  const double l_ms = __shfl_sync(0xffffffffu, lg2, 3) * kLog10of2;
  if (lane != 0) return;
  const double lvr = 20.0 * l_vr;
  if (passes & P_ZFP_GT) {
    t.zfp_bits_gt = s.zfp_bits;
    t.br_zfp_gt = (double)s.zfp_bits / (double)npoints_all;
    t.sse_zfp = zsse;
    t.maxerr_zfp = (double)__uint_as_float(s.zfp_maxerr);
    t.psnr_zfp_gt = mse_z > 0.0 ? lvr - 10.0 * l_mz : INFINITY;
  }
  if (passes & P_SZ_GT) {
    t.delta = s.delta;
    t.eb_sz = s.delta / 2.0;
    t.sse_sz = ssse;
    t.maxerr_sz = (double)__uint_as_float(s.sz_maxerr);
    t.psnr_sz_gt = mse_s > 0.0 ? lvr - 10.0 * l_ms : INFINITY;
  }
}

__device__ inline void finish_post(const ParamsDev& p, Workspace* ws, int passes, long long npoints_all,
                            unsigned long long zfp_npoints) {
  Scalars& s = ws->sc;
  if (s.status != RD_OK || threadIdx.x != 0) return;
  rd_result& r = ws->res;
  rd_truth& t = ws->truth;
  if (s.constant) {
    r.flags = s.flags;
    r.psnr_zfp = INFINITY;
    r.psnr_sz = INFINITY;
    r.selection = 1;
    t.flags = s.flags;
    t.psnr_sz_gt = INFINITY;
    t.psnr_zfp_gt = INFINITY;
    t.best_gt = 1;
    return;
  }
  if (passes & P_SZ_EST) {
    const HuffOut& hh = ws->huff[0];
    double ns = (double)hh.ns;
    double H = log2(ns) - hh.plogp / ns;
    if (H < 0.0) H = 0.0;
    uint32_t h0 = ws->hist[0][0];
    r.entropy = H;
    r.br_sz = H + p.sz_offset;
    r.sz_ns = hh.ns;
    r.sz_huff_bits = hh.cost;
    r.sz_nsym = hh.nsym;
    r.sz_nesc = h0;
    r.br_sz_huff = (double)(hh.cost + 32ull * h0) / ns;
    if (passes & P_ZFP_EST) {
      if (p.sel_rule == RD_SEL_PAPER) {
        double diff = r.br_sz - r.br_zfp;
        if (fabs(diff) <= 1e-9) {
          s.flags |= RD_F_TIE_BAND;
          r.selection = 1;
        } else {
          r.selection = diff < 0.0 ? 0 : 1;
        }
      } else {
        // 2 (Huff + 32 h0) N_z < S2 N_s, in 128-bit integers
        unsigned long long a = 2ull * (hh.cost + 32ull * h0);
        unsigned long long alo = a * zfp_npoints, ahi = __umul64hi(a, zfp_npoints);
        unsigned long long blo = s.s2 * hh.ns, bhi = __umul64hi(s.s2, hh.ns);
        bool lt = ahi < bhi || (ahi == bhi && alo < blo);
        r.selection = lt ? 0 : 1;
      }
    }
  }
  r.flags = s.flags;
  if (passes & P_SZ_GT) {
    const HuffOut& hg = ws->huff[1];
    uint32_t h0 = ws->hist[1][0];
    t.sz_huff_gt = hg.cost;
    t.sz_nsym_gt = hg.nsym;
    t.sz_nesc_gt = h0;
    t.sz_bits_gt = hg.cost + 32ull * h0 + 22ull * hg.nsym + 64ull;
    t.br_sz_gt = (double)t.sz_bits_gt / (double)npoints_all;
    if (passes & P_ZFP_GT) t.best_gt = t.br_sz_gt < t.br_zfp_gt ? 0 : 1;
  }
  t.flags = s.flags & (RD_F_DELTA_CLAMPED | RD_F_MSE_ZERO | RD_F_CONSTANT);
}

__device__ inline void finish_cta(const ParamsDev& p, Workspace* ws, int passes, int zfp_parts,
                           int sz_parts, long long npoints_all, unsigned long long zfp_npoints) {
  finish_pre(ws, passes, zfp_parts, sz_parts, npoints_all);
  __syncthreads();
  finish_post(p, ws, passes, npoints_all, zfp_npoints);
}

// The records and the status, word by word, straight into host memory (all
// threads of the CTA, after the finish step).
__device__ inline void write_out(const Workspace* ws, OutRecords* out) {
  __syncthreads();
  const uint32_t* rs = reinterpret_cast<const uint32_t*>(&ws->res);
  const uint32_t* ts = reinterpret_cast<const uint32_t*>(&ws->truth);
  uint32_t* rd = reinterpret_cast<uint32_t*>(&out->res);
  uint32_t* td = reinterpret_cast<uint32_t*>(&out->truth);
  for (int i = threadIdx.x; i < (int)(sizeof(rd_result) / 4); i += blockDim.x) rd[i] = __ldcg(rs + i);
  for (int i = threadIdx.x; i < (int)(sizeof(rd_truth) / 4); i += blockDim.x) td[i] = __ldcg(ts + i);
  if (threadIdx.x == 0) out->status = __ldcg(&ws->sc.status);
}

// The evaluate step with the truth's ZFP pass beside the Huffman launch:
// the Huffman launch finishes the estimates and the SZ truth, the ZFP pass's
// last CTA (after the Huffman launch has completed) the ZFP truth; then that
// CTA compares the two truths and writes the records.  Every thread of the
// CTA calls it.
__device__ inline void finish_combine(Workspace* ws, int passes, OutRecords* out) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const Scalars& s = ws->sc;
    rd_truth& t = ws->truth;
    if (__ldcg(&s.status) == RD_OK && !__ldcg(&s.constant) && (passes & P_ZFP_GT) && (passes & P_SZ_GT))
      t.best_gt = __ldcg(&t.br_sz_gt) < __ldcg(&t.br_zfp_gt) ? 0 : 1;
  }
  if (out) write_out(ws, out);
}


}  // namespace rdk
