// rd_sz_stream.cu -- the SZ stream of the prequantised ground truth
// (Algorithm 1's last step compresses each field with the selected
// compressor; this writes SZ's stream): the canonical Huffman code of every
// point's symbol, then the 32-bit pattern of every escaped value, each at
// its bit offset.  Offsets are exclusive scans of the code lengths and
// escape flags in storage order: per-CTA totals, one scan over the CTAs,
// then each CTA re-scans its chunk and writes.  The header and code table
// are written by the code-table kernel (rd_sz_codes.cu).
#include <stdint.h>

#include "rd_sz_stream.cuh"

namespace rdk {

namespace {

// The chunk of points of this thread: kStreamPer consecutive points.
__device__ __forceinline__ long long chunk_begin() {
  return (long long)blockIdx.x * kStreamChunk + (long long)threadIdx.x * kStreamPer;
}

template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T t = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += t;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < kStreamThreads / 32 ? s_warp[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T t = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += t;
    }
    if (lane < kStreamThreads / 32) s_warp[lane] = w;
  }
  __syncthreads();
  const T base = wid ? s_warp[wid - 1] : T(0);
  *total = s_warp[kStreamThreads / 32 - 1];
  __syncthreads();
  return base + inc - v;
}

__device__ __forceinline__ unsigned long long bswap64(unsigned long long v) {
  const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
  return ((unsigned long long)__byte_perm(lo, 0u, 0x0123) << 32) | __byte_perm(hi, 0u, 0x0123);
}

// ORs the low nb bits of v (1 <= nb <= 63) into the stream at bit p, most
// significant bit first: bit p of the stream is bit 7 - p % 8 of byte p / 8,
// i.e. bit 63 - p % 64 of the big-endian 64-bit word p / 64.
__device__ __forceinline__ void put_bits(unsigned long long* out, unsigned long long p,
                                         unsigned long long v, int nb) {
  const unsigned long long w = p >> 6;
  const int off = (int)(p & 63);
  if (off + nb <= 64) {
    atomicOr(out + w, bswap64(v << (64 - off - nb)));
  } else {
    atomicOr(out + w, bswap64(v >> (off + nb - 64)));
    atomicOr(out + w + 1, bswap64(v << (128 - off - nb)));
  }
}

}  // namespace

__global__ void __launch_bounds__(kStreamThreads) k_stream_count(const int32_t* __restrict__ sym, long long n,
                                                                 const uint8_t* __restrict__ len,
                                                                 unsigned long long* cta_bits,
                                                                 unsigned* cta_esc) {
  __shared__ unsigned long long s_b[kStreamThreads / 32];
  __shared__ unsigned s_e[kStreamThreads / 32];
  const long long i0 = chunk_begin();
  unsigned long long bits = 0ull;
  unsigned esc = 0u;
#pragma unroll
  for (int k = 0; k < kStreamPer; k++) {
    const long long i = i0 + k;
    if (i < n) {
      const int s = sym[i];
      bits += len[s];
      esc += s == 0 ? 1u : 0u;
    }
  }
  unsigned long long tb;
  unsigned te;
  (void)block_excl_scan(bits, s_b, &tb);
  (void)block_excl_scan(esc, s_e, &te);
  if (threadIdx.x == 0) {
    cta_bits[blockIdx.x] = tb;
    cta_esc[blockIdx.x] = te;
  }
}

__global__ void __launch_bounds__(1024) k_stream_scan(unsigned long long* cta_bits, unsigned* cta_esc,
                                                      int nctas, unsigned long long* totals) {
  __shared__ unsigned long long s_b[32];
  __shared__ unsigned long long s_e[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long carry_b = 0ull, carry_e = 0ull;
  for (int base = 0; base < nctas; base += 1024) {
    const int i = base + (int)threadIdx.x;
    const unsigned long long vb = i < nctas ? cta_bits[i] : 0ull;
    const unsigned long long ve = i < nctas ? cta_esc[i] : 0ull;
    unsigned long long ib = vb, ie = ve;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long tb = __shfl_up_sync(0xffffffffu, ib, off);
      const unsigned long long te = __shfl_up_sync(0xffffffffu, ie, off);
      if (lane >= off) {
        ib += tb;
        ie += te;
      }
    }
    if (lane == 31) {
      s_b[wid] = ib;
      s_e[wid] = ie;
    }
    __syncthreads();
    if (wid == 0) {
      unsigned long long wb = s_b[lane], we = s_e[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long tb = __shfl_up_sync(0xffffffffu, wb, off);
        const unsigned long long te = __shfl_up_sync(0xffffffffu, we, off);
        if (lane >= off) {
          wb += tb;
          we += te;
        }
      }
      s_b[lane] = wb;
      s_e[lane] = we;
    }
    __syncthreads();
    const unsigned long long pb = (wid ? s_b[wid - 1] : 0ull) + ib - vb;
    const unsigned long long pe = (wid ? s_e[wid - 1] : 0ull) + ie - ve;
    if (i < nctas) {
      cta_bits[i] = carry_b + pb;
      cta_esc[i] = (unsigned)(carry_e + pe);
    }
    carry_b += s_b[31];
    carry_e += s_e[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    totals[0] = carry_b;
    totals[1] = carry_e;
  }
}

__global__ void __launch_bounds__(kStreamThreads) k_stream_pack(
    const int32_t* __restrict__ sym, const float* __restrict__ x, long long n,
    const uint8_t* __restrict__ len, const unsigned long long* __restrict__ code,
    const unsigned long long* __restrict__ cta_bits, const unsigned* __restrict__ cta_esc,
    const unsigned long long* __restrict__ totals, unsigned long long payload_base,
    unsigned long long* out) {
  __shared__ unsigned long long s_b[kStreamThreads / 32];
  __shared__ unsigned s_e[kStreamThreads / 32];
  const long long i0 = chunk_begin();
  int s_loc[kStreamPer];
  unsigned long long bits = 0ull;
  unsigned esc = 0u;
#pragma unroll
  for (int k = 0; k < kStreamPer; k++) {
    const long long i = i0 + k;
    s_loc[k] = i < n ? sym[i] : -1;
    if (s_loc[k] >= 0) {
      bits += len[s_loc[k]];
      esc += s_loc[k] == 0 ? 1u : 0u;
    }
  }
  unsigned long long tb;
  unsigned te;
  const unsigned long long my_b = block_excl_scan(bits, s_b, &tb);
  const unsigned my_e = block_excl_scan(esc, s_e, &te);
  unsigned long long p = payload_base + cta_bits[blockIdx.x] + my_b;
  unsigned long long q = payload_base + totals[0] + 32ull * ((unsigned long long)cta_esc[blockIdx.x] + my_e);
#pragma unroll
  for (int k = 0; k < kStreamPer; k++) {
    const int s = s_loc[k];
    if (s < 0) continue;
    const int L = len[s];
    if (L == 0) continue;  // not in the table: the length check refuses the stream
    put_bits(out, p, code[s], L);
    p += (unsigned long long)L;
    if (s == 0) {
      put_bits(out, q, (unsigned long long)__float_as_uint(x[i0 + k]), 32);
      q += 32ull;
    }
  }
}

cudaError_t launch_stream_count(const int32_t* sym, long long n, const uint8_t* len,
                                unsigned long long* cta_bits, unsigned* cta_esc, cudaStream_t s) {
  k_stream_count<<<stream_ctas(n), kStreamThreads, 0, s>>>(sym, n, len, cta_bits, cta_esc);
  return cudaGetLastError();
}

cudaError_t launch_stream_scan(unsigned long long* cta_bits, unsigned* cta_esc, int nctas,
                               unsigned long long* totals, cudaStream_t s) {
  k_stream_scan<<<1, 1024, 0, s>>>(cta_bits, cta_esc, nctas, totals);
  return cudaGetLastError();
}

cudaError_t launch_stream_pack(const int32_t* sym, const float* x, long long n, const uint8_t* len,
                               const unsigned long long* code, const unsigned long long* cta_bits,
                               const unsigned* cta_esc, const unsigned long long* totals,
                               unsigned long long payload_base, unsigned long long* out,
                               cudaStream_t s) {
  k_stream_pack<<<stream_ctas(n), kStreamThreads, 0, s>>>(sym, x, n, len, code, cta_bits, cta_esc,
                                                          totals, payload_base, out);
  return cudaGetLastError();
}

}  // namespace rdk
