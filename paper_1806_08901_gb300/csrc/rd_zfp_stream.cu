// rd_zfp_stream.cu -- the ZFP fixed-accuracy stream of a field (Algorithm
// 1's last step compresses each field with the selected compressor; this
// writes ZFP's stream): per block, in raster block order (last axis
// fastest), a flag bit (0: no plane coded), else 1, the block exponent + 127
// in 8 bits and the group-test embedded coding of planes 31 .. 32-P of the
// negabinary coefficients in sequency order.  Its length is the ZFP ground
// truth's bit count.
//
// Passes: the bits of every block (the block code of the ZFP pass, one
// thread per block) and their sum per chunk of kZsChunk blocks; one CTA
// scans the chunk sums; each chunk's CTA scans its blocks' bits and every
// thread writes its blocks at their offsets.  A block's bits are gathered in
// a 64-bit word per stream word and ORed into the stream (zeroed first), so
// the words a block shares with its neighbours are merged exactly.
#include <stdint.h>

#include "rd_sz_stream.cuh"
#include "rd_zfp_dev.cuh"

namespace rdk {

constexpr int kZsThreads = 256;
constexpr int kZsPer = 4;                          // blocks per thread
constexpr int kZsChunk = kZsThreads * kZsPer;      // blocks per CTA
constexpr int kZsScanThreads = 1024;

namespace {

__device__ __forceinline__ unsigned long long zs_bswap64(unsigned long long v) {
  const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
  return ((unsigned long long)__byte_perm(lo, 0u, 0x0123) << 32) | __byte_perm(hi, 0u, 0x0123);
}

// Bits written most significant first: stream bit p is bit 63 - p % 64 of
// the big-endian 64-bit word p / 64.  The word under construction is held
// in `acc` and ORed into the stream when the writer leaves it.
struct BitWriter {
  unsigned long long* out;
  unsigned long long pos;  // next bit
  unsigned long long acc;  // bits of word pos / 64 so far
  __device__ __forceinline__ void flush() {
    if (acc) atomicOr(out + (pos >> 6), zs_bswap64(acc));
    acc = 0ull;
  }
  // the low nb bits of v, 1 <= nb <= 64
  __device__ __forceinline__ void put(unsigned long long v, int nb) {
    while (nb > 0) {
      const int off = (int)(pos & 63);
      const int take = min(nb, 64 - off);
      const unsigned long long chunk =
          (take == 64 ? v : (v >> (nb - take)) & ((1ull << take) - 1ull));
      acc |= (take == 64 ? chunk : chunk << (64 - off - take));
      nb -= take;
      if (off + take == 64) {
        flush();
        pos += take;
      } else {
        pos += take;
      }
    }
  }
  // nz zero bits then a one
  __device__ __forceinline__ void zeros_then_one(int nz) {
    while (nz >= 64) {
      put(0ull, 64);
      nz -= 64;
    }
    put(1ull, nz + 1);
  }
};

// The group-test embedded coding of planes 31 .. kmin of the NB
// coefficients u (sequency order): per plane, the bits of the n coefficients
// already significant verbatim, then group tests: a 1 when a one remains
// among the rest, followed by the scanned bits up to and including it (the
// last coefficient's bit implied), until a test reads 0 or no coefficient is
// left.
template <int NB>
__device__ __forceinline__ void emit_planes(const unsigned* u, int kmin, BitWriter& w) {
  int n = 0;
  for (int k = 31; k >= kmin; k--) {
    unsigned long long x = 0ull;  // bit j: plane k of coefficient j
#pragma unroll
    for (int j = 0; j < NB; j++) x |= (unsigned long long)((u[j] >> k) & 1u) << j;
    if (n > 0) w.put(__brevll(x) >> (64 - n), n);  // x[0] first
    int pos = n;
    while (pos < NB) {
      const unsigned long long rest = pos < 64 ? x >> pos : 0ull;
      if (!rest) {
        w.put(0ull, 1);  // no one left in the plane
        break;
      }
      const int p = pos + __ffsll((long long)rest) - 1;
      if (p == NB - 1) {
        // the test, then the zeros before the last coefficient, whose one
        // is implied
        w.put(1ull, 1);
        if (NB - 1 - pos > 0) {
          int nz = NB - 1 - pos;
          while (nz > 0) {
            const int t = min(nz, 64);
            w.put(0ull, t);
            nz -= t;
          }
        }
        pos = NB;
      } else {
        w.put(1ull, 1);
        w.zeros_then_one(p - pos);
        pos = p + 1;
      }
      n = pos;
    }
  }
}

}  // namespace

// Bits of every block; per-chunk sums (one chunk per CTA).
template <int D>
__global__ void __launch_bounds__(kZsThreads) k_zfp_enc_bits(FieldDev f, int minexp,
                                                             uint32_t* __restrict__ bits,
                                                             unsigned long long* __restrict__ csum) {
  __shared__ unsigned long long s_sum[kZsThreads / 32];
  constexpr int NB = 1 << (2 * D);
  unsigned long long mine = 0ull;
#pragma unroll 1
  for (int i = 0; i < kZsPer; i++) {
    const long long u = (long long)blockIdx.x * kZsChunk + (long long)i * kZsThreads + threadIdx.x;
    if (u >= f.nblocks) break;
    int b[3] = {0, 0, 0};
    decode_block<D>(f, u, false, b);
    float v[NB];
    load_block<D>(f, b, v);
    BlockWork<D> w;
    w.forward(v, minexp);
    const unsigned nb = w.bits();
    bits[u] = nb;
    mine += nb;
  }
  mine = warp_sum(mine);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0ull;
    for (int i = 0; i < kZsThreads / 32; i++) t += s_sum[i];
    csum[blockIdx.x] = t;
  }
}

// Exclusive scan of the chunk sums in place (one CTA, in rounds of
// kZsScanThreads); total[0] = the stream's length.
__global__ void __launch_bounds__(kZsScanThreads) k_zfp_enc_scan(unsigned long long* csum, int n,
                                                                 unsigned long long* total) {
  __shared__ unsigned long long s_warp[kZsScanThreads / 32];
  __shared__ unsigned long long s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (int base = 0; base < n; base += kZsScanThreads) {
    const int i = base + threadIdx.x;
    const unsigned long long v = i < n ? csum[i] : 0ull;
    unsigned long long inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += t;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      unsigned long long x = s_warp[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += t;
      }
      s_warp[lane] = x;
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    const unsigned long long before = carry + (wid ? s_warp[wid - 1] : 0ull) + inc - v;
    if (i < n) csum[i] = before;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_warp[kZsScanThreads / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) total[0] = s_carry;
}

// Each chunk's CTA: exclusive scan of its blocks' bits, then every thread
// writes its blocks.
template <int D>
__global__ void __launch_bounds__(kZsThreads) k_zfp_enc_pack(FieldDev f, int minexp,
                                                             const uint32_t* __restrict__ bits,
                                                             const unsigned long long* __restrict__ coff,
                                                             unsigned long long* __restrict__ out) {
  __shared__ unsigned long long s_warp[kZsThreads / 32];
  constexpr int NB = 1 << (2 * D);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // this thread's kZsPer consecutive blocks of the chunk
  const long long u0 = (long long)blockIdx.x * kZsChunk + (long long)threadIdx.x * kZsPer;
  unsigned long long mine = 0ull;
#pragma unroll
  for (int i = 0; i < kZsPer; i++)
    if (u0 + i < f.nblocks) mine += bits[u0 + i];
  unsigned long long inc = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += t;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned long long x = lane < kZsThreads / 32 ? s_warp[lane] : 0ull;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += t;
    }
    if (lane < kZsThreads / 32) s_warp[lane] = x;
  }
  __syncthreads();
  BitWriter w;
  w.out = out;
  w.pos = coff[blockIdx.x] + (wid ? s_warp[wid - 1] : 0ull) + inc - mine;
  w.acc = 0ull;
#pragma unroll 1
  for (int i = 0; i < kZsPer; i++) {
    const long long u = u0 + i;
    if (u >= f.nblocks) break;
    int b[3] = {0, 0, 0};
    decode_block<D>(f, u, false, b);
    float v[NB];
    load_block<D>(f, b, v);
    BlockWork<D> bw;
    bw.forward(v, minexp);
    if (bw.bi.prec == 0) {
      w.put(0ull, 1);
    } else {
      w.put(1ull, 1);
      w.put((unsigned long long)(bw.bi.emax + 127), 8);
      emit_planes<NB>(bw.u, bw.bi.kmin, w);
    }
  }
  w.flush();
}

int zfp_stream_chunks(long long nblocks) { return (int)((nblocks + kZsChunk - 1) / kZsChunk); }

cudaError_t launch_zfp_stream(const FieldDev& f, int minexp, uint32_t* bits,
                              unsigned long long* csum, unsigned long long* total,
                              unsigned long long* out, cudaStream_t s) {
  const int nch = zfp_stream_chunks(f.nblocks);
  switch (f.d) {
    case 1: k_zfp_enc_bits<1><<<nch, kZsThreads, 0, s>>>(f, minexp, bits, csum); break;
    case 2: k_zfp_enc_bits<2><<<nch, kZsThreads, 0, s>>>(f, minexp, bits, csum); break;
    default: k_zfp_enc_bits<3><<<nch, kZsThreads, 0, s>>>(f, minexp, bits, csum); break;
  }
  k_zfp_enc_scan<<<1, kZsScanThreads, 0, s>>>(csum, nch, total);
  if (out) {
    switch (f.d) {
      case 1: k_zfp_enc_pack<1><<<nch, kZsThreads, 0, s>>>(f, minexp, bits, csum, out); break;
      case 2: k_zfp_enc_pack<2><<<nch, kZsThreads, 0, s>>>(f, minexp, bits, csum, out); break;
      default: k_zfp_enc_pack<3><<<nch, kZsThreads, 0, s>>>(f, minexp, bits, csum, out); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace rdk
