/* rdsel_stream.h -- compressed streams of the selected compressor
 * (Algorithm 1, the step after the selection: each field is compressed by
 * the compressor chosen for it).  Types and error codes are those of
 * rdsel.h.
 */
#ifndef RDSEL_STREAM_H
#define RDSEL_STREAM_H

#include <stdint.h>

#include "rdsel.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The SZ stream of the prequantised ground truth at the absolute bound
 * eb_sz (the stream whose size rd_ground_truth reports as sz_bits_gt).
 * Layout, bits most significant first within each byte:
 *   header   K, the number of distinct symbols (32 bits); the number of
 *            escapes (32 bits)
 *   table    K entries in ascending symbol order: symbol (16 bits), code
 *            length (6 bits)
 *   payload  the canonical Huffman code of every point's symbol in the
 *            field's row-major order (canonical: symbols in ascending
 *            (length, symbol) order take consecutive code values)
 *   escapes  the 32-bit pattern of every escaped value (symbol 0), in order
 * A decoder rebuilds the field from the stream, the shape, eb_sz and
 * quant_radius: a non-escaped point's code Q is its residual (symbol -
 * 32768) plus the integer Lorenzo prediction from the codes of its decoded
 * neighbours, its value float(Q) * float(2 eb_sz); an escaped point's value
 * is the stored one and its code rint(value / w) as in the quantiser.
 *  - field, params: as for rd_ground_truth (params->quant_radius is R).
 *  - eb_sz > 0 and finite; a constant field has nothing to quantise
 *    (RD_ERR_INVALID_ARG).
 *  - out: DEVICE memory, 8-byte aligned, cap_bytes >= 8 * ceil(*nbits / 64)
 *    (RD_ERR_RANGE otherwise); the bytes past the stream's last bit are
 *    zero.  out = NULL: only *nbits is computed (the ground truth's bit
 *    count), nothing is written.
 *  - *nbits: the stream's length in bits.
 *  - Device work: the ground truth (histogram, quantiser, status); the
 *    code table (the symbols sorted by count, stably, a Huffman tree over at
 *    most 65536 symbols, the code lengths, canonical codes, the header and
 *    table written into out); the per-point symbols, per-CTA sums of code
 *    lengths and escapes, one scan over the CTAs, then each CTA writes its
 *    points' codes and escaped values at their offsets (64-bit ORs).  The
 *    context keeps a scratch of 4 N bytes + 2.9 MB, counted against its
 *    memory budget.
 *  - Equal counts keep symbol order in the tree's leaves, so the same
 *    histogram gives the same code on every call; the code is one optimal
 *    code (its payload length is the same for every optimal code).
 *  - Returns once the work on `stream` has finished. */
int32_t rd_sz_compress(rd_context* ctx, const rd_field* field, const rd_params* params,
                       double eb_sz, void* out, uint64_t cap_bytes, uint64_t* nbits,
                       void* stream);

/* The ZFP fixed-accuracy stream of the field at eb_abs (from params: eb and
 * eb_mode), the stream whose size rd_ground_truth reports as zfp_bits_gt.
 * Layout, bits most significant first within each byte, one block after
 * another in row-major block order (the last axis fastest):
 *   flag      1 bit: 0 when the block codes no plane (precision 0: the
 *             block is all zero, or far below the bound), and nothing more;
 *   exponent  the block exponent emax + 127 (8 bits);
 *   planes    planes 31 .. 32-P of the block's negabinary coefficients in
 *             sequency order (P = clamp(emax - floor(log2 eb_abs) + 2(d+1),
 *             0, 32)), each as: the bits of the coefficients already
 *             significant, verbatim; then group tests, a 1 when a one remains
 *             among the others followed by their bits up to and including
 *             that one (the last coefficient's bit implied), until a test
 *             reads 0 or no coefficient is left.
 * A decoder rebuilds the field from the stream, the shape and eb_abs (the
 * truncated coefficients through the inverse transform).
 *  - out: DEVICE memory, 8-byte aligned, cap_bytes >= 8 * ceil(*nbits /
 *    64) (RD_ERR_RANGE otherwise); the bytes past the last bit are zero.
 *    out = NULL: only *nbits is computed.
 *  - A constant field under a value-range-relative bound has no bound to
 *    code at: RD_ERR_INVALID_ARG.
 *  - Device work: the ZFP truth (bit count), then every block's bits and
 *    their sums per chunk of 1024 blocks, one scan over the chunks, and
 *    each block written at its offset by 64-bit ORs.  The context keeps a
 *    scratch of 4 bytes per block, counted against its memory budget.
 *  - Returns once the work on `stream` has finished. */
int32_t rd_zfp_compress(rd_context* ctx, const rd_field* field, const rd_params* params,
                        void* out, uint64_t cap_bytes, uint64_t* nbits, void* stream);

/* Algorithm 1 for one field, to the end: the selection s_i (rd_select),
 * then the compressed bytes C_i of the compressor it picks -- SZ's stream
 * (rd_sz_compress) at eb_sz = delta / 2 when s_i = 0, ZFP's stream
 * (rd_zfp_compress) at eb_abs when s_i = 1.
 *  - *selection: s_i (0 = SZ, 1 = ZFP); *nbits: the length of C_i; est:
 *    the selection's record, or NULL.
 *  - out = NULL: the selection and the length only; otherwise as the two
 *    stream calls (device memory, 8-byte aligned, large enough).
 *  - A constant field: RD_ERR_INVALID_ARG (est, when given, holds its
 *    record). */
int32_t rd_compress(rd_context* ctx, const rd_field* field, const rd_params* params, void* out,
                    uint64_t cap_bytes, uint64_t* nbits, int32_t* selection, rd_result* est,
                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RDSEL_STREAM_H */
