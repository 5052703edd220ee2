/*
 * rans.h -- C ABI of the B300 interleaved streaming rANS library
 *           (libinterleaved_rans_b300.so).
 *
 * The library encodes and decodes byte streams with static-model streaming
 * rANS, N coders interleaved into one bitstream without metadata, following
 * F. Giesen, "Interleaved entropy coders" (arXiv:1402.3392):
 *
 *   - coding function C(s,x) = floor(x/f_s)*M + B_s + (x mod f_s) and its
 *     inverse D (Section 2; the paper's worked example in Section 2.1 is this
 *     function with M = 4), B_s = f_0 + ... + f_{s-1};
 *   - streaming with the normalized interval I = [L, bL) (Section 2,
 *     Algorithm 1); the encoder runs over the message backwards and writes
 *     backwards, the decoder runs forwards; the final encoder states are
 *     transmitted (Section 2);
 *   - N coders share one word buffer, symbol i is coded by coder i mod N
 *     (Section 3);
 *   - L = 2^16, b = 2^16 (16-bit words), M = 2^12, 32-bit states: b >= M, so
 *     every symbol needs at most one renormalization step and the bitstream
 *     does not depend on how many coders run in parallel (Section 5).  On the
 *     GPU one coder is one warp lane; the renormalization reads and writes of
 *     a step are placed by a warp ballot and prefix population counts
 *     (Section 6).
 *
 * Message format (little endian; the paper defines no container):
 *   bytes 0..31  header: u32 magic 0x534E4152 ("RANS"), u32 version 1,
 *                u32 n_lanes N, u32 log2_M (12; 13 or 14 for version 1),
 *                u64 n_symbols,
 *                u32 chunk_symbols, u32 n_chunks = ceil(n_symbols/chunk_symbols)
 *   u32 offsets[n_chunks + 1]: start of chunk c in bytes, relative to the
 *                data region; offsets[0] = 0, offsets[n_chunks] = data bytes
 *   zero padding up to data0 = round_up(32 + 4*(n_chunks+1), 16)
 *   data region: the chunks back to back; chunk c codes symbols
 *                [c*chunk_symbols, min(n_symbols, (c+1)*chunk_symbols)) as
 *                u32 state[N] (final encoder state of coder 0..N-1) followed
 *                by the u16 words in decoder read order
 *   zero padding up to a multiple of 16 bytes (the message size).
 * Chunks are independent streams, so a message of many chunks keeps every SM
 * busy.  The frequency table is not stored: like the model of Section 3 it
 * is agreed out of band.
 *
 * Conventions for every call:
 *   - Ownership: the caller allocates and frees every buffer.  Pointers named
 *     d_* are device pointers; h_* are host pointers.  The library keeps no
 *     pointer after a call returns.
 *   - Streams: work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and the call returns without synchronizing.
 *   - Errors: argument errors are returned synchronously and enqueue
 *     nothing.  Errors found in the data (a corrupt or truncated message, a
 *     symbol without probability) are written to a device status word and
 *     never trap.  RANS_ERR_CUDA means a CUDA call failed (launch error).
 *   - Device code runs on the current CUDA device, which must be sm_103.
 */
#ifndef INTERLEAVED_RANS_B300_H_
#define INTERLEAVED_RANS_B300_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rans_stream_t; /* same type as cudaStream_t */

/* Status codes (return values and device status words). */
#define RANS_OK                   0
#define RANS_ERR_INVALID_ARG      1  /* bad argument, alignment or size */
#define RANS_ERR_ZERO_FREQ        2  /* input holds a symbol with f_s = 0 or s >= n_alpha */
#define RANS_ERR_BUFFER_TOO_SMALL 3  /* output or scratch capacity too small */
#define RANS_ERR_CORRUPT          4  /* message header, offsets or chunk contents inconsistent */
#define RANS_ERR_TIMEOUT          5  /* a bounded device-side wait gave up */
#define RANS_ERR_CUDA             6  /* a CUDA runtime call or launch failed */
#define RANS_ERR_OOM              7  /* an admission or allocation budget was exceeded */

/* Fixed coding parameters (Section 5 of the paper: b >= M). */
#define RANS_LOG2_M        12
#define RANS_M             4096u
#define RANS_L             65536u      /* I = [2^16, 2^32) */
#define RANS_LOG2_B        16
#define RANS_LOG2_M_MAX    14          /* plain messages: M = 2^12, 2^13 or 2^14 */
#define RANS_MAX_ALPHABET  256
#define RANS_MAX_LANES     32
#define RANS_MAGIC         0x534E4152u
#define RANS_VERSION       1u
#define RANS_VERSION_BYPASS 2u         /* messages with raw words (rans_encode_bypass) */
#define RANS_VERSION_BYTES 3u          /* byte-wise messages (rans_encode_bytes) */
#define RANS_VERSION_ADAPTIVE 4u       /* adaptive binary messages (rans_encode_adaptive) */
#define RANS_VERSION_PREFIX 5u         /* prefix-code messages (rans_encode_prefix) */
#define RANS_VERSION_ADAPTIVE_N 6u     /* adaptive n-symbol messages (rans_encode_adaptive_n) */
#define RANS_PREFIX_MAX_LEN 12         /* longest prefix code */

typedef struct {
    uint32_t n_lanes;        /* N interleaved coders per chunk, 1..32 */
    uint32_t chunk_symbols;  /* symbols per chunk, >= 1 */
} rans_params;

/* Library version (RANS_VERSION of the format it writes). */
uint32_t rans_version(void);

/* Short English text for a status code (static storage). */
const char *rans_status_string(int status);

/*
 * rans_quantize_table -- static order-0 model: integer weights -> integer
 * frequencies f_s with sum f_s = 2^log2_M.  The paper assumes a static
 * probability model per file (Section 7) but does not say how it is
 * quantized; this is the rule the library uses:
 *   1. f_s = floor(w_s * M / W), W = sum w; raised to 1 where w_s > 0;
 *   2. while sum f < M: +1 to the symbols with w_s > 0 in decreasing order
 *      of the remainder w_s*M mod W (ties: lower index), repeating the
 *      order if needed;
 *   3. while sum f > M: -1 from the symbol with the largest f_s > 1
 *      (ties: lower index).
 * Hence f_s >= 1 exactly when w_s > 0.
 * weights: host, n entries.  freq_out: host, n entries.
 * n in [1, 4096], log2_M in [1, 15], sum w < 2^64, at most M nonzero weights;
 * the coders need n <= 256 and log2_M = 12 (12, 13 or 14 for the plain
 * rans_encode / rans_decode family).
 * Returns RANS_OK or RANS_ERR_INVALID_ARG (freq_out untouched).  Host only.
 */
int rans_quantize_table(const uint64_t *weights, uint32_t n, uint32_t log2_M,
                        uint16_t *freq_out);

/* Worst-case message size in bytes for n_symbols symbols (one 16-bit word
 * per symbol, Section 5, plus header, offsets, states and padding).
 * 0 if the parameters are invalid. */
uint64_t rans_max_encoded_size(uint64_t n_symbols, const rans_params *params);

/* Scratch bytes rans_encode needs for n_symbols symbols.  0 if invalid. */
uint64_t rans_encode_scratch_size(uint64_t n_symbols, const rans_params *params);

/*
 * rans_encode -- encode n_symbols bytes into one message (format above).
 *
 * d_symbols : device, n_symbols bytes, symbol values < n_alpha.
 * h_freq    : host, n_alpha frequencies (rans_quantize_table) with sum M =
 *             2^12 = RANS_M, or 2^13 or 2^14: with b = 2^16 >= M a symbol still
 *             needs at most one renormalization (Section 5's 12-14 bits of
 *             probability resolution).  The sum selects M; the header's log2_M
 *             field records it (the 2^13/2^14 tables cost the decoder a
 *             second table lookup per symbol).
 * n_alpha   : 1..256.
 * params    : host; n_lanes 1..32, chunk_symbols >= 1.
 * d_out     : device, 16-byte aligned, out_cap bytes; out_cap must be at
 *             least rans_max_encoded_size(n_symbols, params).
 * d_out_size: device, one u64: the message size in bytes (a multiple of 16),
 *             or 0 if the data was rejected.
 * d_status  : device, one u32: RANS_OK, or RANS_ERR_ZERO_FREQ if some symbol
 *             has f_s = 0 (the message is then not valid), or RANS_ERR_TIMEOUT.
 * d_scratch : device, 16-byte aligned, scratch_cap bytes,
 *             >= rans_encode_scratch_size(n_symbols, params).
 * The worst-case message (every chunk's offsets must fit in u32) must stay
 * below 4 GiB.  Returns RANS_OK, RANS_ERR_INVALID_ARG,
 * RANS_ERR_BUFFER_TOO_SMALL or RANS_ERR_CUDA.
 */
int rans_encode(const uint8_t *d_symbols, uint64_t n_symbols, const uint16_t *h_freq,
                uint32_t n_alpha, const rans_params *params, uint8_t *d_out,
                uint64_t out_cap, uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                uint64_t scratch_cap, rans_stream_t stream);

/*
 * rans_decode -- decode a message produced by rans_encode (or the same
 * format from any encoder that follows the paper's interleaving).
 *
 * d_msg     : device, 16-byte aligned, msg_size bytes (a multiple of 16).
 * h_freq, n_alpha, params : the model and layout the message was encoded
 *             with (the header is checked against them, log2_M included).
 * d_symbols : device, n_symbols bytes of output.
 * d_status  : device, one u32, set to RANS_OK, or RANS_ERR_CORRUPT if the
 *             header, the offsets or any chunk is inconsistent (a chunk must
 *             end with every coder back at its initial state L and with its
 *             words consumed exactly), or RANS_ERR_TIMEOUT.  On RANS_ERR_CORRUPT
 *             the output of the bad chunks is unspecified.
 * Returns RANS_OK, RANS_ERR_INVALID_ARG or RANS_ERR_CUDA.
 */
int rans_decode(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream);

/*
 * rans_decode_host -- rans_decode with the message and the symbols in host
 * memory.  The message is split into pieces of whole chunks; each piece's
 * bytes are copied to the device on one internal stream, decoded on `stream`,
 * and its symbols copied back on another internal stream, so copies in both
 * directions overlap each other and the decoding (this needs page-locked host
 * buffers; pageable ones work but copy synchronously).  The two internal
 * streams are created on a device's first call and kept.
 *
 * h_msg, msg_size, h_freq, n_alpha, params, n_symbols : as in rans_decode,
 *             with h_msg in host memory (no alignment required).
 * h_symbols : host, n_symbols bytes of output.
 * h_status  : host u32, set like rans_decode's d_status (RANS_OK,
 *             RANS_ERR_CORRUPT or RANS_ERR_TIMEOUT) by the enqueued work.
 * d_work    : device, 16-byte aligned, work_cap >=
 *             rans_decode_host_work_size(msg_size, n_symbols) bytes: the
 *             message, the symbols and the status word on the device.
 * Returns RANS_OK, RANS_ERR_INVALID_ARG, RANS_ERR_BUFFER_TOO_SMALL or
 * RANS_ERR_CUDA.  The work is ordered after what `stream` holds, and later
 * work on `stream` runs after it; h_symbols and h_status are valid, and the
 * host buffers may be reused, once `stream` has reached that point.
 */
/*
 * rans_encode_host -- rans_encode with the symbols and the message in host
 * memory.  The symbols are copied in by pieces of whole chunks on one
 * internal stream, coded on `stream`, and each piece's chunks are given
 * their final offsets (a running total on the device) and packed into the
 * output on another internal stream, so the copies overlap the coding.  A
 * page-locked, 16-byte aligned h_out is written directly by the device,
 * piece by piece; any other h_out receives the message in one copy at the
 * end, and then the call waits for `stream` before it returns.
 *
 * h_symbols, n_symbols, h_freq, n_alpha, params : as in rans_encode, with
 *             h_symbols in host memory.
 * h_out     : host, out_cap >= rans_max_encoded_size(n_symbols, params).
 * h_out_size: host u64: the message size (0 if the encode failed).
 * h_status  : host u32: RANS_OK or RANS_ERR_ZERO_FREQ (or RANS_ERR_TIMEOUT).
 * d_work    : device, 16-byte aligned, work_cap >=
 *             rans_encode_host_work_size(n_symbols, params): the symbols, the
 *             encode scratch, the offsets and a worst-case message.
 * Returns RANS_OK, RANS_ERR_INVALID_ARG, RANS_ERR_BUFFER_TOO_SMALL or
 * RANS_ERR_CUDA.  h_out, *h_out_size and *h_status are valid, and the host
 * buffers may be reused, once `stream` has reached the end of the work.
 */
uint64_t rans_encode_host_work_size(uint64_t n_symbols, const rans_params *params);
int rans_encode_host(const uint8_t *h_symbols, uint64_t n_symbols, const uint16_t *h_freq,
                     uint32_t n_alpha, const rans_params *params, uint8_t *h_out,
                     uint64_t out_cap, uint64_t *h_out_size, uint32_t *h_status, void *d_work,
                     uint64_t work_cap, rans_stream_t stream);
uint64_t rans_decode_host_work_size(uint64_t msg_size, uint64_t n_symbols);
int rans_decode_host(const uint8_t *h_msg, uint64_t msg_size, const uint16_t *h_freq,
                     uint32_t n_alpha, const rans_params *params, uint8_t *h_symbols,
                     uint64_t n_symbols, uint32_t *h_status, void *d_work, uint64_t work_cap,
                     rans_stream_t stream);

/*
 * Bypass (raw) words interleaved with the coded symbols -- Section 3 of the
 * paper (bypass coding): because encoder and decoder run in lockstep, raw
 * data can be written into the same stream at agreed points with no
 * metadata and no coder state change.  Here the agreed point is a per-symbol
 * flag of the model: raw_words[s] in {0, 1} is the number of raw 16-bit
 * words symbol s carries.  The encoder sends a symbol's raw word right before
 * it encodes the symbol; the decoder reads it right after it has decoded the
 * symbol and renormalized.  Within a step of N coders, each coder's
 * renormalization word is followed by its raw word, coders in order.
 * A bypass message is a version-2 container (RANS_VERSION_BYPASS); the model
 * (frequencies and raw_words) is not stored in it.
 *
 * rans_encode_bypass -- as rans_encode, plus:
 *   d_raw       : device, n_symbols u16 (2-byte aligned): d_raw[i] is sent
 *                 after symbol i when h_raw_words[symbol i] == 1, ignored
 *                 otherwise.
 *   h_raw_words : host, n_alpha bytes, each 0 or 1.
 *   out_cap     : >= rans_max_encoded_size_bypass(n_symbols, params).
 *   scratch_cap : >= rans_encode_scratch_size_bypass(n_symbols, params).
 * rans_decode_bypass -- as rans_decode, plus:
 *   h_raw_words : as above (must equal the encoder's).
 *   d_raw       : device, n_symbols u16 (2-byte aligned): d_raw[i] = the raw
 *                 word after symbol i, or 0 when its symbol carries none.
 * A bypass message is decoded with one chunk per warp.  Messages of one kind
 * given to the other kind's decoder are reported RANS_ERR_CORRUPT (version).
 */
uint64_t rans_max_encoded_size_bypass(uint64_t n_symbols, const rans_params *params);
uint64_t rans_encode_scratch_size_bypass(uint64_t n_symbols, const rans_params *params);
int rans_encode_bypass(const uint8_t *d_symbols, const uint16_t *d_raw, uint64_t n_symbols,
                       const uint16_t *h_freq, const uint8_t *h_raw_words, uint32_t n_alpha,
                       const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                       uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                       uint64_t scratch_cap, rans_stream_t stream);
int rans_decode_bypass(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                       const uint8_t *h_raw_words, uint32_t n_alpha, const rans_params *params,
                       uint8_t *d_symbols, uint16_t *d_raw, uint64_t n_symbols,
                       uint32_t *d_status, rans_stream_t stream);

/*
 * Byte-wise messages -- Section 5 of the paper: with 8-bit digits (b = 2^8 <
 * M = 2^12) a coder can need two renormalization digits for one symbol, and
 * a SIMD/GPU decoder with one lane per coder reads a step's digits
 * breadth-first (one digit for every lane that needs one, lanes in order,
 * then the second digits).  The stream therefore depends on N (N is "baked
 * in"): a byte-wise message must be decoded with the N it was encoded with,
 * which the header records.  L = 2^23, b = 2^8, I = [2^23, 2^31); chunks
 * are [u32 state[N]][bytes][zeros up to a multiple of 4]; version 3
 * (RANS_VERSION_BYTES).
 *
 * rans_encode_bytes / rans_decode_bytes: arguments, buffers and statuses as
 * rans_encode / rans_decode; out_cap >= rans_max_encoded_size_bytes(...),
 * scratch_cap >= rans_encode_scratch_size(...).  Decoded one chunk per warp.
 */
uint64_t rans_max_encoded_size_bytes(uint64_t n_symbols, const rans_params *params);
int rans_encode_bytes(const uint8_t *d_symbols, uint64_t n_symbols, const uint16_t *h_freq,
                      uint32_t n_alpha, const rans_params *params, uint8_t *d_out,
                      uint64_t out_cap, uint64_t *d_out_size, uint32_t *d_status,
                      void *d_scratch, uint64_t scratch_cap, rans_stream_t stream);
int rans_decode_bytes(const uint8_t *d_msg, uint64_t msg_size, const uint16_t *h_freq,
                      uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                      uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream);

/*
 * Adaptive binary messages -- Section 5 of the paper: adaptive models still
 * vectorize when no two lanes update the same model, e.g. with one context
 * per lane.  Symbols are bytes 0 or 1.  Coder j keeps its own context p (the
 * probability of a 0, scaled to M = 2^12, starting at M/2 in every chunk);
 * a symbol is coded with f_0 = p, f_1 = M - p and afterwards p moves towards
 * it by (target - p) >> 5.  Coder j's context sees only its own symbols, so
 * the stream depends on N like the rest of the container.  L = b = 2^16,
 * 16-bit words, version 4 (RANS_VERSION_ADAPTIVE).  No model table is passed.
 *
 * rans_encode_adaptive: as rans_encode without the model; out_cap >=
 *   rans_max_encoded_size(...), scratch_cap >=
 *   rans_encode_scratch_size_adaptive(...) (the plain scratch plus about 4
 *   bytes per 16 steps of each coder: the encoder runs the contexts forwards,
 *   storing a checkpoint and the symbols' bits for every 16 steps, then codes
 *   backwards from those alone).
 *   A symbol other than 0 or 1 gives RANS_ERR_ZERO_FREQ.
 * rans_decode_adaptive: as rans_decode without the model.
 */
uint64_t rans_encode_scratch_size_adaptive(uint64_t n_symbols, const rans_params *params);
int rans_encode_adaptive(const uint8_t *d_symbols, uint64_t n_symbols, const rans_params *params,
                         uint8_t *d_out, uint64_t out_cap, uint64_t *d_out_size,
                         uint32_t *d_status, void *d_scratch, uint64_t scratch_cap,
                         rans_stream_t stream);
int rans_decode_adaptive(const uint8_t *d_msg, uint64_t msg_size, const rans_params *params,
                         uint8_t *d_symbols, uint64_t n_symbols, uint32_t *d_status,
                         rans_stream_t stream);

/*
 * Adaptive messages over n symbols (2 <= n <= RANS_ADAPTIVE_N_MAX) -- Section 5
 * of the paper: adaptive models vectorize as long as every lane updates only
 * its own model.  Symbols are bytes 0..n-1.  Coder j keeps its own cumulative
 * frequencies C_0 = 0 < C_1 < ... < C_n = M (M = 2^12; f_s = C_{s+1} - C_s,
 * B_s = C_s), starting at C_i = floor(i M / n) in every chunk.  After coding
 * symbol s it moves every interior boundary a 1/32 part of the way (rounded
 * down) towards i when i <= s and towards M - n + i when i > s:
 *     i <= s:  C_i -= (C_i - i) >> 5      i > s:  C_i += (M - n + i - C_i) >> 5
 * so s's interval widens and every f stays >= 1.  Coder j sees only its own
 * symbols, so the stream depends on N like the rest of the container.
 * L = b = 2^16, 16-bit words, version 6 (RANS_VERSION_ADAPTIVE_N); the
 * header's log2_M field holds 12 | n << 16.  No model table is passed.
 *
 * rans_encode_adaptive_n: as rans_encode with the alphabet size n_alpha in
 *   place of the model; out_cap >= rans_max_encoded_size(...), scratch_cap >=
 *   rans_encode_scratch_size_adaptive_n(...) (the plain scratch plus 4 bytes
 *   per symbol: the encoder runs every coder's model forwards and stores each
 *   symbol's (B_s, f_s), then codes backwards from those).  A symbol >= n
 *   gives RANS_ERR_ZERO_FREQ; n_alpha outside [2, 16] RANS_ERR_INVALID_ARG.
 * rans_decode_adaptive_n: as rans_decode with n_alpha in place of the model;
 *   a header whose n differs from n_alpha is corrupt.
 */
#define RANS_ADAPTIVE_N_MAX 16u
uint64_t rans_encode_scratch_size_adaptive_n(uint64_t n_symbols, const rans_params *params);
int rans_encode_adaptive_n(const uint8_t *d_symbols, uint64_t n_symbols, uint32_t n_alpha,
                           const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                           uint64_t *d_out_size, uint32_t *d_status, void *d_scratch,
                           uint64_t scratch_cap, rans_stream_t stream);
int rans_decode_adaptive_n(const uint8_t *d_msg, uint64_t msg_size, uint32_t n_alpha,
                           const rans_params *params, uint8_t *d_symbols, uint64_t n_symbols,
                           uint32_t *d_status, rans_stream_t stream);

/*
 * Interleaving arbitrary coders -- Section 4 of the paper: any entropy
 * coder's streams can be interleaved without metadata if the encoder runs
 * (an instrumented copy of) the decoder and lays the words down in the order
 * the decoder will read them.  The coder here is a canonical prefix code.
 *
 * Code: lengths l_s in 0..RANS_PREFIX_MAX_LEN (0 = symbol not in the code)
 * with sum 2^-l_s <= 1; codes assigned in order of (length, symbol), each
 * length's codes consecutive (the canonical rule of RFC 1951, 3.2.2).
 * Coder j of a chunk takes symbols j, j+N, ... and writes their codes MSB
 * first into 32-bit words.  Its decoder holds up to 43 bits and, before each
 * symbol, reads one word when it holds fewer than 12 bits; the reads of one
 * step are taken in lane order.  The message lays every word where that
 * read finds it.  A chunk ends with every coder's leftover bits zero and
 * every word read.  Container as rans.h's plain one, version 5
 * (RANS_VERSION_PREFIX), log2_M field 12; chunk c = u32 little-endian words
 * only (no states), so offsets are multiples of 4.
 *
 * rans_prefix_lengths: host.  Optimal code lengths <= max_len (1..12) for
 *   weights[0..n_alpha) (0 = unused), by package-merge; ties between equal
 *   weights go to the lower symbol index first.  One used symbol gets
 *   length 1.  Returns RANS_OK, or RANS_ERR_INVALID_ARG (no used symbol,
 *   more than 2^max_len used symbols, bad pointers or sizes).
 * rans_prefix_codes: host.  The canonical codes of lengths[0..n_alpha)
 *   (codes_out[s], right-aligned; 0 for unused symbols).  RANS_ERR_INVALID_ARG
 *   if a length exceeds 12, no symbol is used, or Kraft's sum exceeds 1.
 * rans_encode_prefix: as rans_encode with code lengths (host, n_alpha <=
 *   256) instead of a frequency table; out_cap >=
 *   rans_max_encoded_size_prefix(...), scratch_cap >=
 *   rans_encode_scratch_size_prefix(...).  A symbol without a code gives
 *   RANS_ERR_ZERO_FREQ.
 * rans_decode_prefix: as rans_decode with the same code lengths.
 */
int rans_prefix_lengths(const uint64_t *weights, uint32_t n_alpha, uint32_t max_len,
                        uint8_t *lengths_out);
int rans_prefix_codes(const uint8_t *lengths, uint32_t n_alpha, uint16_t *codes_out);
uint64_t rans_max_encoded_size_prefix(uint64_t n_symbols, const rans_params *params);
uint64_t rans_encode_scratch_size_prefix(uint64_t n_symbols, const rans_params *params);
int rans_encode_prefix(const uint8_t *d_symbols, uint64_t n_symbols, const uint8_t *h_lengths,
                       uint32_t n_alpha, const rans_params *params, uint8_t *d_out,
                       uint64_t out_cap, uint64_t *d_out_size, uint32_t *d_status,
                       void *d_scratch, uint64_t scratch_cap, rans_stream_t stream);
int rans_decode_prefix(const uint8_t *d_msg, uint64_t msg_size, const uint8_t *h_lengths,
                       uint32_t n_alpha, const rans_params *params, uint8_t *d_symbols,
                       uint64_t n_symbols, uint32_t *d_status, rans_stream_t stream);

/*
 * Batched decoding: many independent messages ("streams"), each with its own
 * model, layout and size, decoded by one persistent launch.  A CTA takes one
 * work item at a time -- up to 16 chunks of one stream -- from a device-side
 * counter, builds that stream's slot table in shared memory (only when the
 * model changes) and decodes two chunks per warp side by side.  Uneven stream sizes balance
 * themselves because items are handed out dynamically.  The call enqueues
 * kernels only (no allocation, no host synchronization), so it can be
 * captured in a CUDA graph and replayed.
 */
typedef struct {
    const uint8_t *msg;       /* device, 16-byte aligned: the stream's message */
    uint64_t msg_size;        /* its size in bytes (a multiple of 16) */
    uint8_t *symbols;         /* device: n_symbols bytes of output */
    uint64_t n_symbols;       /* symbols in the stream */
    uint32_t table;           /* index of the stream's model in d_freqs */
    uint32_t n_lanes;         /* N the stream was encoded with, 1..32 */
    uint32_t chunk_symbols;   /* chunk size it was encoded with, >= 1 */
    uint32_t reserved;        /* set to 0 */
} rans_stream;                /* 48 bytes */

/* Scratch bytes rans_decode_batch needs for n_streams streams. */
uint64_t rans_decode_batch_scratch_size(uint32_t n_streams);

/*
 * rans_decode_batch -- decode n_streams messages.
 *
 * d_streams : device, n_streams descriptors (read only).
 * d_freqs   : device, n_tables models of 256 u16 frequencies each (zero for
 *             symbols outside the alphabet); each must sum to RANS_M.
 * d_status  : device, n_streams u32: per stream RANS_OK, RANS_ERR_INVALID_ARG
 *             (bad descriptor or model; the stream is skipped),
 *             RANS_ERR_CORRUPT or RANS_ERR_TIMEOUT (as in rans_decode).
 * d_scratch : device, 16-byte aligned, >= rans_decode_batch_scratch_size().
 * Returns RANS_OK, RANS_ERR_INVALID_ARG, RANS_ERR_BUFFER_TOO_SMALL or
 * RANS_ERR_CUDA; per-stream problems go to d_status only.
 */
int rans_decode_batch(const rans_stream *d_streams, uint32_t n_streams, const uint16_t *d_freqs,
                      uint32_t n_tables, uint32_t *d_status, void *d_scratch,
                      uint64_t scratch_cap, rans_stream_t stream);

/*
 * Batched encoding: the mirror image of rans_decode_batch.  Every stream is
 * encoded into its own message (format above) with its own model and layout.
 */
typedef struct {
    const uint8_t *symbols;   /* device: n_symbols bytes, values < the model's alphabet */
    uint64_t n_symbols;
    uint8_t *out;             /* device, 16-byte aligned: the stream's message */
    uint64_t out_cap;         /* >= rans_max_encoded_size(n_symbols, {n_lanes, chunk_symbols}) */
    uint64_t scratch_offset;  /* byte offset of the stream's scratch in d_scratch
                                 (filled in by rans_encode_batch_plan) */
    uint32_t table;           /* index of the stream's model in d_freqs */
    uint32_t n_lanes;         /* N, 1..32 */
    uint32_t chunk_symbols;   /* >= 1 */
    uint32_t reserved;        /* set to 0 */
} rans_encode_stream;         /* 56 bytes */

/*
 * rans_encode_batch_plan -- host: give every stream its scratch region
 * (h_streams[i].scratch_offset, 16-byte aligned, after a work area of the
 * batch) and return the scratch size rans_encode_batch needs, or 0 if a
 * stream's n_lanes or chunk_symbols is out of range.
 */
uint64_t rans_encode_batch_plan(rans_encode_stream *h_streams, uint32_t n_streams);

/*
 * rans_encode_batch -- encode n_streams streams.
 *
 * d_streams  : device, n_streams descriptors planned by rans_encode_batch_plan.
 * d_freqs    : device, n_tables models of 256 u16 frequencies each.
 * d_out_sizes: device, n_streams u64: message sizes (0 when a stream failed).
 * d_status   : device, n_streams u32: RANS_OK, RANS_ERR_INVALID_ARG (bad
 *              descriptor, model or scratch range; skipped) or RANS_ERR_ZERO_FREQ.
 * d_scratch  : device, 16-byte aligned, >= the planned size.
 * Returns RANS_OK, RANS_ERR_INVALID_ARG or RANS_ERR_CUDA.
 */
int rans_encode_batch(const rans_encode_stream *d_streams, uint32_t n_streams,
                      const uint16_t *d_freqs, uint32_t n_tables, uint64_t *d_out_sizes,
                      uint32_t *d_status, void *d_scratch, uint64_t scratch_cap,
                      rans_stream_t stream);

/*
 * Serving: a continuous-batching request loop.  The server owns a device
 * arena (the caller's HBM budget) and a few CUDA streams ("slots").  It
 * replays a trace of encode and decode requests in real time: a request is
 * pending from its arrival time; pending requests are admitted in arrival
 * order while their device input and output fit in the arena; admitted
 * requests form the next batch in an idle slot -- copies of the inputs to the
 * device, one rans_encode_batch and/or rans_decode_batch launch, copies of the
 * outputs back -- while later arrivals are admitted into the other slots as
 * memory frees up, so the batches overlap on the device.  The models stay
 * resident on the device for the server's lifetime.
 */
#define RANS_REQ_ENCODE 0u
#define RANS_REQ_DECODE 1u
/* Or'ed into kind: input and output are device memory (a message input and
 * an encode output 16-byte aligned).  The coders then read and write them in
 * place: no copies, and only the batch's scratch and descriptors take arena
 * memory.  The request is done when its kernels are. */
#define RANS_REQ_DEVICE_MEMORY 0x100u

typedef struct {
    uint32_t kind;            /* RANS_REQ_ENCODE or RANS_REQ_DECODE, optionally
                                 | RANS_REQ_DEVICE_MEMORY */
    uint32_t table;           /* model index in the server's d_freqs */
    uint32_t n_lanes;         /* N of the message (made or read) */
    uint32_t chunk_symbols;   /* chunk size of the message */
    const uint8_t *input;     /* host (page-locked for overlap), or device with
                                 RANS_REQ_DEVICE_MEMORY: symbols (encode) or a
                                 message (decode) */
    uint64_t input_size;      /* bytes: = n_symbols (encode), message size (decode) */
    uint64_t n_symbols;       /* symbols in the request */
    uint8_t *output;          /* host (device with RANS_REQ_DEVICE_MEMORY): receives
                                 the message (encode) or symbols (decode) */
    uint64_t output_cap;      /* >= rans_max_encoded_size (encode), >= n_symbols (decode) */
    double arrival_s;         /* arrival, seconds after rans_server_run starts;
                                 non-decreasing along the trace */
} rans_request;

typedef struct {
    uint64_t output_size;     /* bytes written to output */
    uint32_t status;          /* RANS_OK, the coder's error, or RANS_ERR_OOM when the
                                 request can never fit the budget */
    uint32_t batch;           /* index of the batch that served it */
    double admit_s;           /* admission time, seconds after the start */
    double done_s;            /* completion (output in host memory, or in the
                                 device output for RANS_REQ_DEVICE_MEMORY) */
} rans_result;

typedef struct rans_server rans_server;

/*
 * rans_server_create -- d_freqs: device models (n_tables x 256 u16, kept
 * resident); d_arena: device memory of arena_bytes (16-byte aligned) that
 * bounds everything the server places on the device; max_batch: requests per
 * batch; n_slots: batches in flight at once (1..16).  Creates CUDA streams,
 * events and page-locked staging; allocates no device memory.  The arena is
 * the server's budget, not the process's whole device footprint: the
 * library's fixed RANS_STATIC_SCRATCH_BYTES array (see
 * rans_encode_static_scratch), held by every GPU that loads the library,
 * comes on top of it.
 */
int rans_server_create(const uint16_t *d_freqs, uint32_t n_tables, void *d_arena,
                       uint64_t arena_bytes, uint32_t max_batch, uint32_t n_slots,
                       rans_server **out);

/*
 * rans_server_run -- serve n requests (host array, sorted by arrival) in real
 * time; blocks until every request is done and fills results[0..n).
 * Returns RANS_OK, RANS_ERR_INVALID_ARG (a malformed request; nothing runs)
 * or RANS_ERR_CUDA.
 */
int rans_server_run(rans_server *server, const rans_request *reqs, uint32_t n,
                    rans_result *results);

void rans_server_destroy(rans_server *server);

/*
 * rans_encode_static_scratch -- rans_encode for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a service of the
 * library, not a step of the method.
 *
 * Who needs it: code that runs where cudaMalloc is not allowed or not wanted
 * -- for example a host that has reserved the whole device up front and hands
 * out only fixed buffers, a real-time pipeline that forbids allocation once
 * it is running, or a plugin that is given input and output buffers by its
 * host and nothing else.  Such a caller still passes its own input and
 * output; only the encoder's scratch is taken from a fixed array inside the
 * library.
 *
 * Arguments, output format and status codes are those of rans_encode,
 * without d_scratch/scratch_cap; the model may sum to 2^12, 2^13 or 2^14 as
 * there.  The scratch is a file-scope device array of
 * RANS_STATIC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  An input whose scratch need,
 * rans_encode_scratch_size(n_symbols, params), exceeds that returns
 * RANS_ERR_BUFFER_TOO_SMALL and enqueues nothing (at 64 KiB chunks: about
 * 32 Mi symbols).
 *
 * - The first call on a device, with that device current, looks up the
 *   array's device address (cudaGetSymbolAddress); make that first call
 *   before any stream capture.  No call allocates device memory.  The
 *   address is kept until the process exits, so after a reset of the
 *   device's context (cudaDeviceReset) this entry point must not be called
 *   again in the same process.
 * - The array counts against the device's memory on top of any budget the
 *   caller manages (for example rans_server_create's arena).
 * - Every call on a device shares the one array and leaves its contents
 *   behind; nothing in it needs to start at zero.  Calls whose work overlaps
 *   on the GPU (different streams, or different host threads without
 *   ordering) race on the array and corrupt each other's output: order them
 *   on one stream or otherwise serialize them.
 */
#define RANS_STATIC_SCRATCH_BYTES (64u << 20)
int rans_encode_static_scratch(const uint8_t *d_symbols, uint64_t n_symbols,
                               const uint16_t *h_freq, uint32_t n_alpha,
                               const rans_params *params, uint8_t *d_out, uint64_t out_cap,
                               uint64_t *d_out_size, uint32_t *d_status,
                               rans_stream_t stream);

/*
 * rans_check_bounded_wait -- diagnostic of the failure path; no step of the
 * paper's method.  Launches one warp that waits, with the same bounded wait
 * the coder kernels use for their bulk copies (at most 200 ms of
 * %globaltimer), on a shared-memory mbarrier that nothing ever completes.
 * The wait gives up, the kernel writes RANS_ERR_TIMEOUT to *d_status and
 * returns, and the context stays usable: this is how a copy that never
 * lands ends a coder kernel with a status instead of a hang.
 *
 * d_status : device u32, overwritten (RANS_ERR_TIMEOUT once the kernel ends).
 * Returns RANS_OK when the kernel was enqueued, RANS_ERR_INVALID_ARG for a
 * null d_status, RANS_ERR_CUDA on a launch error.  The kernel takes about
 * 200 ms of GPU time.
 */
int rans_check_bounded_wait(uint32_t *d_status, rans_stream_t stream);

/*
 * rans_check_lookback_wait -- diagnostic of the failure path; no step of the
 * paper's method.  rans_encode (and the other whole-message encoders) find
 * each chunk's offset by waiting, bounded, for the sizes of the chunks
 * before it.  This launches one warp that runs that look-back for chunk 1 of
 * a two-chunk message whose chunk 0 never publishes its size, with a 200 ms
 * bound: the look-back gives up, marks its chunk failed (so that later
 * chunks give up at once), and the kernel writes RANS_ERR_TIMEOUT to
 * *d_status (RANS_OK if the look-back ended any other way).
 *
 * d_status : device u32, overwritten.  Returns RANS_OK when the kernel was
 * enqueued, RANS_ERR_INVALID_ARG for a null d_status, RANS_ERR_CUDA on a
 * launch error.  The kernel takes about 200 ms of GPU time; calls must not
 * overlap (they share one small device array).
 */
int rans_check_lookback_wait(uint32_t *d_status, rans_stream_t stream);

/*
 * rans_check_division -- diagnostic of the encoders' exact division; no step
 * of the paper's method, but C(s, x) = floor(x / f_s) * M + B_s + (x mod f_s)
 * (Section 2) needs floor(x / f_s) exactly, and the encoders compute it
 * without a divide.  Enqueues one kernel that runs the encoders' own division
 * code over every frequency f in [1, M - 1] (M = 2^log2m) and every state x
 * in the range it is applied to, the precursor set I_s = [f L / M, f b L / M)
 * of Section 2 (L = b = 2^16), and checks each quotient q against the
 * definition q * f <= x < (q + 1) * f in 64-bit integers.
 *
 * method   : 0 = the 64-bit multiply-add by the table's reciprocal (static
 *            models, log2m 12, 13 or 14); 1 = the adaptive coder's float estimate and
 *            one correction (log2m 12; the remainder is checked too).
 * d_result : device, 8-byte aligned, 4 u64, overwritten: [0] states checked,
 *            [1] wrong quotients, [2] the smallest f << 32 | x that was wrong
 *            (~0 if none), [3] 0.
 * Returns RANS_OK when the kernels were enqueued, RANS_ERR_INVALID_ARG for a
 * bad method/log2m or pointer, RANS_ERR_CUDA on a launch error.  It takes
 * seconds of GPU time (about 9e12 states at log2m 12, 3.5e13 at 14).
 */
int rans_check_division(uint32_t method, uint32_t log2m, uint64_t *d_result,
                        rans_stream_t stream);

/*
 * rans_check_gather_ceiling -- diagnostic of what bounds the table decoder; no
 * step of the paper's method.  The decode step of Section 6 puts three
 * accesses through the SM's L1/shared-memory pipe: the slot-table lookup (32
 * random entries of a 4096-entry table in shared memory), the read of the
 * step's words (a contiguous window of the word ring) and the store of the
 * step's 32 symbols.  This enqueues one kernel that does only those three
 * accesses per step, in the plain decoder's shape (CTAs of 12 warps, 3 per SM,
 * one 16 KiB table per CTA, a 4 KiB ring per warp), each lane's next slot
 * taken from a multiply-add of the two values it loaded, so that each warp's
 * steps form a chain as the decoder's do.  Every warp runs `steps` steps; the
 * kernel's time for rans_check_gather_ceiling_warps() * steps warp-steps is
 * the pipe's rate for the decode step's access mix, to set beside the
 * decoder's own steps per second.
 *
 * steps  : warp-steps per warp, a positive multiple of 16.
 * d_out  : device, out_size >= rans_check_gather_ceiling_warps() * 4096 bytes,
 *          overwritten (4 KiB per warp, written cyclically).
 * d_sink : device u32, incremented only by a lane whose state reaches 0 (it
 *          keeps the chain live; almost never).
 * Returns RANS_OK when the kernel was enqueued, RANS_ERR_INVALID_ARG for a bad
 * steps or pointer, RANS_ERR_BUFFER_TOO_SMALL for a small d_out, RANS_ERR_CUDA
 * on a launch error.
 *
 * rans_check_gather_ceiling_warps -- the number of warps that kernel runs on
 * the current device (resident CTAs x 12), 0 on a CUDA error.
 */
int rans_check_gather_ceiling(uint32_t steps, uint8_t *d_out, uint64_t out_size,
                              uint32_t *d_sink, rans_stream_t stream);
uint64_t rans_check_gather_ceiling_warps(void);

/*
 * rans_check_cta_warps -- the launch rule the placing encoders apply to a
 * message whose chunks all start at once, exposed for host-side tests (no
 * CUDA call, no step of the paper's method).  With one chunk per warp at a
 * time, the message is done when the SM given the most warps is: of the CTA
 * sizes w = 1 .. max_warps, the one whose ceil(n_units / w) CTAs, spread
 * evenly over sms SMs, give the busiest SM the fewest warps, the larger w of
 * equal ones.
 *
 * n_units   : chunks of the launch.
 * sms       : SMs of the device.
 * per_sm    : host, max_warps + 1 entries; per_sm[w] = w-warp CTAs an SM
 *             holds (0: none fits); per_sm[0] unused.  A launch of more than
 *             per_sm[max_warps] * sms * max_warps units keeps max_warps.
 * max_warps : 1 .. 32.
 * Returns the chosen warps per CTA, or 0 for a null per_sm or a max_warps
 * out of range.
 */
uint32_t rans_check_cta_warps(uint64_t n_units, uint32_t sms, const int32_t *per_sm,
                              uint32_t max_warps);

/*
 * Checked builds (a test build compiled with -DRANS_CHECKED; the library
 * built normally answers RANS_ERR_INVALID_ARG to both calls).  The kernels
 * then test their invariants as they run and count the ones that fail (the
 * access a failed check guards is skipped):
 *   - decoder: before each group of steps, every byte the group can read lies
 *     in ring segments whose copies have completed and that no later copy has
 *     taken over (the ring's ordering, i.e. no read of stale or in-flight data);
 *   - encoder: the staged words fit the chunk's slot and every bulk store
 *     lands inside it; the prefix encoder stores only to positions its
 *     decoder's reads were given, inside the slot.
 * rans_debug_checks: host.  Waits for the device, then stores the number of
 *   failed checks since the last call in *failures and clears the counters.
 * rans_debug_check_selftest: enqueues a kernel whose one check fails on
 *   purpose (the next rans_debug_checks then reports at least one).
 */
int rans_debug_checks(uint64_t *failures);
int rans_debug_check_selftest(rans_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* INTERLEAVED_RANS_B300_H_ */
