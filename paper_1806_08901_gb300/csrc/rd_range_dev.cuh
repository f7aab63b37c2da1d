// rd_range_dev.cuh -- value range (Algorithm 1 line 2) and the derived
// scalars, shared by the per-field range pass and the fused batched
// estimate.
#pragma once

#include <math.h>
#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

struct RangeAcc {
  unsigned kmin = 0xffffffffu, kmax = 0u, bad = 0u;
  __device__ __forceinline__ void add(float v) {
    const unsigned b = __float_as_uint(v);
    bad |= ((b & 0x7f800000u) == 0x7f800000u);
    const unsigned k = float_key(v);
    kmin = min(kmin, k);
    kmax = max(kmax, k);
  }
};

// Values [begin, end) of x, thread tid of nth: a scalar head up to a 16-byte
// boundary, float4 loads, a scalar tail.  With kCopy every value is also
// stored at the same index of copy (whose address has x's alignment modulo
// 16), through L2, where the next pass finds it.
template <bool kCopy = false>
__device__ __forceinline__ void range_span(const float* __restrict__ x, long long begin,
                                           long long end, long long tid, long long nth,
                                           RangeAcc& acc, float* __restrict__ copy = nullptr) {
  const float* xb = x + begin;
  float* cb = kCopy ? copy + begin : nullptr;
  const long long n = end - begin;
  long long head = (long long)((16u - ((uintptr_t)xb & 15u)) & 15u) / 4;
  if (head > n) head = n;
  if (((uintptr_t)xb & 3u) != 0) head = n;  // not even 4-byte aligned: all scalar
  for (long long i = tid; i < head; i += nth) {
    const float v = xb[i];
    if (kCopy) __stcg(cb + i, v);
    acc.add(v);
  }
  const long long nvec = (n - head) / 4;
  const float4* x4 = reinterpret_cast<const float4*>(xb + head);
  float4* c4 = kCopy ? reinterpret_cast<float4*>(cb + head) : nullptr;
  long long i = tid;
  // four independent 16-byte loads in flight per thread
  for (; i + 3 * nth < nvec; i += 4 * nth) {
    float4 q[4];
#pragma unroll
    for (int u = 0; u < 4; u++) q[u] = __ldg(x4 + i + u * nth);
#pragma unroll
    for (int u = 0; u < 4; u++) {
      if (kCopy) __stcg(c4 + i + u * nth, q[u]);
      acc.add(q[u].x);
      acc.add(q[u].y);
      acc.add(q[u].z);
      acc.add(q[u].w);
    }
  }
  for (; i < nvec; i += nth) {
    const float4 q = __ldg(x4 + i);
    if (kCopy) __stcg(c4 + i, q);
    acc.add(q.x);
    acc.add(q.y);
    acc.add(q.z);
    acc.add(q.w);
  }
  for (long long i = head + nvec * 4 + tid; i < n; i += nth) {
    const float v = xb[i];
    if (kCopy) __stcg(cb + i, v);
    acc.add(v);
  }
}

// Warp, then CTA, then one update per CTA of the field's shared keys.  All
// threads of the CTA call it (up to 1024 threads).
__device__ __forceinline__ void range_commit(RangeAcc acc, Workspace* ws) {
  __shared__ unsigned s_min[32], s_max[32], s_bad[32];
  unsigned kmin = __reduce_min_sync(0xffffffffu, acc.kmin);
  unsigned kmax = __reduce_max_sync(0xffffffffu, acc.kmax);
  unsigned bad = __reduce_or_sync(0xffffffffu, acc.bad);
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_min[wid] = kmin;
    s_max[wid] = kmax;
    s_bad[wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    unsigned a = threadIdx.x < nw ? s_min[threadIdx.x] : 0xffffffffu;
    unsigned b = threadIdx.x < nw ? s_max[threadIdx.x] : 0u;
    unsigned c = threadIdx.x < nw ? s_bad[threadIdx.x] : 0u;
    a = __reduce_min_sync(0xffffffffu, a);
    b = __reduce_max_sync(0xffffffffu, b);
    c = __reduce_or_sync(0xffffffffu, c);
    if (threadIdx.x == 0) {
      atomicMin(&ws->sc.min_key, a);
      atomicMax(&ws->sc.max_key, b);
      if (c) atomicOr(&ws->sc.nonfinite, 1u);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Prepare: value range VR, eb_abs (Eq. psnr-sz: eb_rel = eb_abs / VR) and
// floor(log2 eb_abs) for the ZFP precision rule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prepare_field(const ParamsDev& p, Workspace* ws) {
  Scalars& s = ws->sc;
  if (__ldcg(&s.nonfinite)) {
    s.status = RD_ERR_NONFINITE;
    return;
  }
  s.vmin = key_float(__ldcg(&s.min_key));
  s.vmax = key_float(__ldcg(&s.max_key));
  s.amax = fmaxf(fabsf(s.vmin), fabsf(s.vmax));
  s.vr = (double)s.vmax - (double)s.vmin;
  s.eb_abs = (p.eb_mode == RD_EB_REL) ? p.eb * s.vr : p.eb;
  ws->res.vmin = s.vmin;
  ws->res.vmax = s.vmax;
  ws->res.vr = s.vr;
  ws->res.eb_abs = s.eb_abs;
  if (s.vr == 0.0) {
    s.constant = 1;
    s.flags |= RD_F_CONSTANT;
    return;
  }
  if (!(s.eb_abs > 0.0) || !isfinite(s.eb_abs)) {
    s.status = RD_ERR_INVALID_ARG;
    return;
  }
  int e;
  frexp(s.eb_abs, &e);
  s.minexp = e - 1;
  ws->res.minexp = s.minexp;
}

}  // namespace rdk
