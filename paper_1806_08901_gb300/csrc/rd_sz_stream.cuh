// rd_sz_stream.cuh -- launchers of the SZ stream encoder (rd_sz_compress).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rd_internal.cuh"

namespace rdk {

// Points per CTA of the counting and packing passes.
constexpr int kStreamThreads = 256;
constexpr int kStreamPer = 16;  // consecutive points per thread
constexpr long long kStreamChunk = (long long)kStreamThreads * kStreamPer;

inline int stream_ctas(long long n) { return (int)((n + kStreamChunk - 1) / kStreamChunk); }

// Per-CTA totals of code bits (len[sym]) and escapes (sym == 0) over the
// CTA's chunk of points.
cudaError_t launch_stream_count(const int32_t* sym, long long n, const uint8_t* len,
                                unsigned long long* cta_bits, unsigned* cta_esc, cudaStream_t s);
// Exclusive scans of the per-CTA totals in place (one CTA); the grand
// totals go to totals[0] (bits) and totals[1] (escapes).
cudaError_t launch_stream_scan(unsigned long long* cta_bits, unsigned* cta_esc, int nctas,
                               unsigned long long* totals, cudaStream_t s);
// Writes every point's code at payload_base + its bit offset and every
// escaped value's 32-bit pattern after the payload, by 64-bit ORs into out
// (zeroed, 8-byte aligned, big-endian bit order within the byte stream).
cudaError_t launch_stream_pack(const int32_t* sym, const float* x, long long n, const uint8_t* len,
                               const unsigned long long* code, const unsigned long long* cta_bits,
                               const unsigned* cta_esc, const unsigned long long* totals,
                               unsigned long long payload_base, unsigned long long* out,
                               cudaStream_t s);

// ZFP fixed-accuracy stream (rd_zfp_stream.cu): every block's bits into
// bits[nblocks], per-chunk sums into csum[zfp_stream_chunks(nblocks)] (then
// scanned in place; total[0] = the stream's length); with out, every block
// written at its offset by 64-bit ORs into out (zeroed, 8-byte aligned).
int zfp_stream_chunks(long long nblocks);
cudaError_t launch_zfp_stream(const FieldDev& f, int minexp, uint32_t* bits,
                              unsigned long long* csum, unsigned long long* total,
                              unsigned long long* out, cudaStream_t s);

}  // namespace rdk
