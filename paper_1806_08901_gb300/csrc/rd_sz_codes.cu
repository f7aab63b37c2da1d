// rd_sz_codes.cu -- the code table of the SZ stream, built on the device
// (Algorithm 1's last step writes SZ's stream; its Huffman code is an
// optimal prefix code of the truth's symbol histogram): code lengths from a
// Huffman tree, canonical codes, and the stream's header and table.
//
// One CTA of kCodeThreads threads, in steps separated by barriers:
//  1. the present symbols in symbol order (a block scan over the bins);
//  2. a stable LSD radix sort of (count, symbol) by count, 8 bits a pass,
//     so that equal counts keep symbol order (the leaves' order, and with it
//     the code, is the same on every run);
//  3. the two-queue Huffman merge in phases (every item below the sum of
//     the two smallest is paired at once, in merged order, ties leaves
//     first), each new node recording itself as the parent of its two
//     items; the queues live in shared memory up to kHuffSmemKeys symbols;
//  4. node depths from the root down, a phase at a time in reverse, then
//     every leaf's depth is its symbol's code length;
//  5. canonical codes: ascending (length, symbol) take consecutive values
//     from the first code of each length (the count of shorter codes);
//  6. the header (K, the escape count; 32 bits each) and the table (per
//     present symbol in symbol order: symbol 16 bits, length 6 bits) ORed
//     into the stream from bit 0.
// A single symbol gets length 1.  A length above 63 (the table's field)
// sets *status to RD_ERR_RANGE.
#include <stdint.h>

#include "rd_sz_stream.cuh"

namespace rdk {

namespace {

constexpr int kCodeThreads = 1024;
constexpr int kCodeWarps = kCodeThreads / 32;
constexpr int kMaxPhases = 64;

__device__ __forceinline__ unsigned long long cbswap64(unsigned long long v) {
  const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
  return ((unsigned long long)__byte_perm(lo, 0u, 0x0123) << 32) | __byte_perm(hi, 0u, 0x0123);
}

// ORs the low nb bits of v (1 <= nb <= 32) into the big-endian bit stream at
// bit p (stream bit p is bit 63 - p % 64 of 64-bit word p / 64, stored
// byte-swapped).
__device__ __forceinline__ void or_bits(unsigned long long* out, unsigned long long p, unsigned long long v,
                                        int nb) {
  const unsigned long long w = p >> 6;
  const int off = (int)(p & 63);
  if (off + nb <= 64) {
    atomicOr(out + w, cbswap64(v << (64 - off - nb)));
  } else {
    atomicOr(out + w, cbswap64(v >> (off + nb - 64)));
    atomicOr(out + w + 1, cbswap64(v << (128 - off - nb)));
  }
}

// Block-wide exclusive sum (every thread of the CTA calls); *total gets the
// sum.  s_w: kCodeWarps words.
__device__ uint32_t code_excl_sum(uint32_t v, uint32_t* s_w, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += t;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t x = s_w[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += t;
    }
    s_w[lane] = x;
  }
  __syncthreads();
  const uint32_t base = wid ? s_w[wid - 1] : 0u;
  *total = s_w[kCodeWarps - 1];
  __syncthreads();
  return base + inc - v;
}

// Number of elements below t in the ascending a[0..n).
__device__ __forceinline__ uint32_t count_below(const uint32_t* a, uint32_t n, unsigned long long t) {
  uint32_t lo = 0u, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((unsigned long long)a[mid] < t) lo = mid + 1u; else hi = mid;
  }
  return lo;
}

// Number of A elements among the first d of merge(A, B), ties from A first.
__device__ __forceinline__ uint32_t split_at(const uint32_t* A, uint32_t na, const uint32_t* B, uint32_t nb,
                                             uint32_t d) {
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1u; else hi = mid;
  }
  return lo;
}

}  // namespace

__global__ void __launch_bounds__(kCodeThreads, 1)
    k_sz_code_table(const uint32_t* __restrict__ h, CodeScratch sc, uint8_t* __restrict__ len,
                    unsigned long long* __restrict__ code, unsigned long long* __restrict__ out,
                    int32_t* status) {
  // dynamic shared memory: the two queues of step 3 (up to kHuffSmemKeys
  // symbols), and before and after them the per-warp counts of steps 2 and
  // 5 and the per-warp code offsets of step 5
  extern __shared__ __align__(16) uint32_t s_dyn[];
  uint32_t(*s_cnt)[256] = reinterpret_cast<uint32_t(*)[256]>(s_dyn);
  unsigned long long(*s_off)[64] =
      reinterpret_cast<unsigned long long(*)[64]>(s_dyn + kCodeWarps * 256);
  __shared__ uint32_t s_w[kCodeWarps];
  __shared__ unsigned long long s_first[64];
  __shared__ uint32_t s_nlen[64];
  __shared__ uint32_t s_ph[kMaxPhases + 1];
  __shared__ uint32_t s_m[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  constexpr int kPer = kNsym / kCodeThreads;  // bins per thread, consecutive

  // 1. present symbols in symbol order; every length cleared
  uint32_t mine = 0u, mx = 0u;
  for (int k = 0; k < kPer; k++) {
    const uint32_t c = h[tid * kPer + k];
    len[tid * kPer + k] = 0;
    mine += c ? 1u : 0u;
    mx = max(mx, c);
  }
  uint32_t K;
  uint32_t at = code_excl_sum(mine, s_w, &K);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) s_w[wid] = mx;
  __syncthreads();
  if (tid < 32) {
    const uint32_t m = __reduce_max_sync(0xffffffffu, s_w[tid]);
    if (tid == 0) s_m[3] = m;
  }
  for (int k = 0; k < kPer; k++) {
    const uint32_t s = (uint32_t)(tid * kPer + k);
    const uint32_t c = h[s];
    if (c) {
      sc.sym0[at] = s;
      sc.keyA[at] = c;
      sc.symA[at] = s;
      at++;
    }
  }
  __syncthreads();
  mx = s_m[3];
  if (K == 0u) return;

  uint32_t* kin = sc.keyA;
  uint32_t* sin = sc.symA;
  if (K == 1u) {
    if (tid == 0) len[sc.sym0[0]] = 1;
  } else {
    // 2. stable radix sort of (count, symbol) by count
    uint32_t* kout = sc.keyB;
    uint32_t* sout = sc.symB;
    const int passes = (mx >> 24) ? 4 : (mx >> 16) ? 3 : (mx >> 8) ? 2 : 1;
    const uint32_t seg = (K + kCodeWarps - 1) / kCodeWarps;
    const uint32_t w0 = min(K, (uint32_t)wid * seg), w1 = min(K, w0 + seg);
    for (int pass = 0; pass < passes; pass++) {
      const int shift = 8 * pass;
      for (int d = lane; d < 256; d += 32) s_cnt[wid][d] = 0u;
      __syncwarp();
      for (uint32_t b = w0; b < w1; b += 32) {
        const uint32_t i = b + lane;
        const bool ok = i < w1;
        const uint32_t dg = ok ? (kin[i] >> shift) & 255u : 0u;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const unsigned same = __match_any_sync(act, dg);
          if (lane == __ffs(same) - 1) s_cnt[wid][dg] += (uint32_t)__popc(same);
        }
        __syncwarp();
      }
      __syncthreads();
      // offsets, digit-major and warp-minor
      uint32_t tot = 0u;
      if (tid < 256)
        for (int w = 0; w < kCodeWarps; w++) tot += s_cnt[w][tid];
      uint32_t all;
      uint32_t run = code_excl_sum(tid < 256 ? tot : 0u, s_w, &all);
      if (tid < 256)
        for (int w = 0; w < kCodeWarps; w++) {
          const uint32_t t = s_cnt[w][tid];
          s_cnt[w][tid] = run;
          run += t;
        }
      __syncthreads();
      for (uint32_t b = w0; b < w1; b += 32) {
        const uint32_t i = b + lane;
        const bool ok = i < w1;
        const uint32_t key = ok ? kin[i] : 0u;
        const uint32_t sym = ok ? sin[i] : 0u;
        const uint32_t dg = (key >> shift) & 255u;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        unsigned same = 0u;
        if (ok) {
          same = __match_any_sync(act, dg);
          const uint32_t pos = s_cnt[wid][dg] + (uint32_t)__popc(same & lt_mask);
          kout[pos] = key;
          sout[pos] = sym;
        }
        __syncwarp();
        if (ok && lane == __ffs(same) - 1) s_cnt[wid][dg] += (uint32_t)__popc(same);
        __syncwarp();
      }
      __syncthreads();
      uint32_t* t = kin;
      kin = kout;
      kout = t;
      t = sin;
      sin = sout;
      sout = t;
    }

    // 3. Huffman phases, recording parents
    uint32_t* leaves = kin;
    uint32_t* nodes = sc.nodes;
    if (K <= (uint32_t)kHuffSmemKeys) {
      leaves = s_dyn;
      nodes = s_dyn + kHuffSmemKeys;
      for (uint32_t i = tid; i < K; i += kCodeThreads) leaves[i] = kin[i];
      __syncthreads();
    }
    uint32_t lh = 0u, ih = 0u, it = 0u;
    int nph = 0;
    for (;;) {
      if ((K - lh) + (it - ih) <= 1u) break;
      if (tid == 0) {
        unsigned long long c4[4] = {~0ull, ~0ull, ~0ull, ~0ull};
        if (lh < K) c4[0] = leaves[lh];
        if (lh + 1u < K) c4[1] = leaves[lh + 1u];
        if (ih < it) c4[2] = nodes[ih];
        if (ih + 1u < it) c4[3] = nodes[ih + 1u];
        const unsigned long long m01 = min(c4[0], c4[1]), x01 = max(c4[0], c4[1]);
        const unsigned long long m23 = min(c4[2], c4[3]), x23 = max(c4[2], c4[3]);
        const unsigned long long a0 = min(m01, m23);
        const unsigned long long a1 = m01 < m23 ? min(x01, m23) : min(x23, m01);
        const uint32_t ml = count_below(leaves + lh, K - lh, a0 + a1);
        const uint32_t mi = count_below(nodes + ih, it - ih, a0 + a1);
        uint32_t cl = ml;
        if ((ml + mi) & 1u) {
          if (mi == 0u || (ml > 0u && leaves[lh + ml - 1u] > nodes[ih + mi - 1u])) cl = ml - 1u;
        }
        s_m[0] = ml;
        s_m[1] = mi;
        s_m[2] = cl;
        if (nph < kMaxPhases) s_ph[nph] = it;
      }
      __syncthreads();
      const uint32_t ml = s_m[0], mi = s_m[1], cl = s_m[2];
      const uint32_t np = (ml + mi) >> 1;
      const uint32_t per_t = max(1u, (np + kCodeThreads - 1) / kCodeThreads);
      const uint32_t j0 = (uint32_t)tid * per_t, j1 = min(np, j0 + per_t);
      if (j0 < j1 && nph < kMaxPhases) {
        const uint32_t* A = leaves + lh;
        const uint32_t* B = nodes + ih;
        uint32_t i = split_at(A, ml, B, mi, 2u * j0);
        uint32_t k = 2u * j0 - i;
        for (uint32_t j = j0; j < j1; j++) {
          uint32_t sum = 0u;
#pragma unroll
          for (int u = 0; u < 2; u++) {
            if (i < ml && (k >= mi || A[i] <= B[k])) {
              sum += A[i];
              sc.leafpar[lh + i] = it + j;
              i++;
            } else {
              sum += B[k];
              sc.nodepar[ih + k] = it + j;
              k++;
            }
          }
          nodes[it + j] = sum;
        }
      }
      __syncthreads();
      lh += cl;
      ih += 2u * np - cl;
      it += np;
      nph++;
    }
    if (nph > kMaxPhases) {  // cannot happen below 2^32 points (each phase
      if (tid == 0) atomicExch(status, RD_ERR_RANGE);  // at least doubles the threshold)
      return;
    }

    // 4. depths: the root (the last node) is 0; each phase's nodes from
    // their parents, made in later phases; then the leaves
    const uint32_t root = it - 1u;
    if (tid == 0) {
      sc.ndepth[root] = 0u;
      s_ph[nph] = it;
    }
    __syncthreads();
    for (int p = nph - 1; p >= 0; p--) {
      for (uint32_t n = s_ph[p] + tid; n < s_ph[p + 1]; n += kCodeThreads)
        if (n != root) sc.ndepth[n] = sc.ndepth[sc.nodepar[n]] + 1u;
      __syncthreads();
    }
    for (uint32_t i = tid; i < K; i += kCodeThreads) {
      const uint32_t d = sc.ndepth[sc.leafpar[i]] + 1u;
      if (d > 63u) atomicExch(status, RD_ERR_RANGE);
      len[sin[i]] = (uint8_t)min(d, 63u);
    }
    __syncthreads();
  }

  // 5. canonical codes: counts per length, the first code of each length,
  // then consecutive codes in symbol order within a length
  if (tid < 64) s_nlen[tid] = 0u;
  __syncthreads();
  const uint32_t seg = (K + kCodeWarps - 1) / kCodeWarps;
  const uint32_t w0 = min(K, (uint32_t)wid * seg), w1 = min(K, w0 + seg);
  for (int L = lane; L < 64; L += 32) s_cnt[wid][L] = 0u;
  __syncwarp();
  for (uint32_t b = w0; b < w1; b += 32) {
    const uint32_t i = b + lane;
    const bool ok = i < w1;
    const uint32_t L = ok ? len[sc.sym0[i]] : 0u;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const unsigned same = __match_any_sync(act, L);
      if (lane == __ffs(same) - 1) s_cnt[wid][L] += (uint32_t)__popc(same);
    }
    __syncwarp();
  }
  __syncthreads();
  if (tid < 64) {
    uint32_t t = 0u;
    for (int w = 0; w < kCodeWarps; w++) t += s_cnt[w][tid];
    s_nlen[tid] = t;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long cv = 0ull;
    int prev = 0;
    for (int L = 1; L < 64; L++) {
      s_first[L] = 0ull;
      if (!s_nlen[L]) continue;
      cv = prev ? (cv + s_nlen[prev]) << (L - prev) : 0ull;
      s_first[L] = cv;
      prev = L;
    }
  }
  __syncthreads();
  if (tid < 64) {
    unsigned long long run = s_first[tid];
    for (int w = 0; w < kCodeWarps; w++) {
      s_off[w][tid] = run;
      run += s_cnt[w][tid];
    }
  }
  __syncthreads();
  for (uint32_t b = w0; b < w1; b += 32) {
    const uint32_t i = b + lane;
    const bool ok = i < w1;
    const uint32_t s = ok ? sc.sym0[i] : 0u;
    const uint32_t L = ok ? len[s] : 0u;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    unsigned same = 0u;
    if (ok) {
      same = __match_any_sync(act, L);
      code[s] = s_off[wid][L] + (unsigned long long)__popc(same & lt_mask);
    }
    __syncwarp();
    if (ok && lane == __ffs(same) - 1) s_off[wid][L] += (unsigned long long)__popc(same);
    __syncwarp();
  }

  // 6. header and table
  if (tid == 0) {
    or_bits(out, 0ull, K, 32);
    or_bits(out, 32ull, h[0], 32);
  }
  for (uint32_t r = tid; r < K; r += kCodeThreads) {
    const uint32_t s = sc.sym0[r];
    or_bits(out, 64ull + 22ull * r, ((unsigned long long)s << 6) | len[s], 22);
  }
}

cudaError_t prepare_sz_code_table() {
  return cudaFuncSetAttribute(k_sz_code_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              2 * kHuffSmemKeys * (int)sizeof(uint32_t));
}

cudaError_t launch_sz_code_table(const uint32_t* h, const CodeScratch& sc, uint8_t* len,
                                 unsigned long long* code, unsigned long long* out, int32_t* status,
                                 cudaStream_t s) {
  k_sz_code_table<<<1, kCodeThreads, 2 * kHuffSmemKeys * sizeof(uint32_t), s>>>(h, sc, len, code, out,
                                                                                status);
  return cudaGetLastError();
}

}  // namespace rdk
