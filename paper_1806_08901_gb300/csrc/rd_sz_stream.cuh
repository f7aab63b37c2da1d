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

// Device scratch of the code table (rd_sz_codes.cu): kNsym words each.
struct CodeScratch {
  uint32_t* sym0;     // present symbols in symbol order
  uint32_t* keyA;     // radix sort: counts and symbols, two buffers
  uint32_t* symA;
  uint32_t* keyB;
  uint32_t* symB;
  uint32_t* nodes;    // Huffman nodes' weights (above kHuffSmemKeys symbols)
  uint32_t* leafpar;  // parent node of every leaf (sorted order)
  uint32_t* nodepar;  // parent node of every node
  uint32_t* ndepth;   // depth of every node
};
constexpr int kCodeScratchWords = 9 * kNsym;

// From the histogram h (kNsym bins): the code length len[s] and canonical
// code code[s] of every symbol (length 0: absent) of an optimal prefix
// code, with the stream's header (present symbols K, h[0] escapes; 32 bits
// each) and table (per present symbol in symbol order: symbol 16 bits,
// length 6 bits) ORed into out (zeroed) from bit 0, so that the payload
// starts at bit 64 + 22 K.  *status (RD_OK on entry) gets RD_ERR_RANGE when
// a length would exceed 63.  One CTA.
cudaError_t prepare_sz_code_table();
cudaError_t launch_sz_code_table(const uint32_t* h, const CodeScratch& sc, uint8_t* len,
                                 unsigned long long* code, unsigned long long* out, int32_t* status,
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
