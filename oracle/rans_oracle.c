/*
 * rans_oracle.c -- CPU ORACLE for interleaved streaming rANS.
 *
 * TEST INFRASTRUCTURE.  This file is the independent, plain, slow reference
 * that the CUDA library is checked against.  Only tests/, the smoke check in
 * __graft_entry__.py and the cpu_baseline leg of bench.py may load it.  The
 * product package never includes, links or calls it, and it includes nothing
 * from the product (no shared header, table, constant or helper).
 *
 * What it computes, following F. Giesen, "Interleaved entropy coders"
 * (arXiv:1402.3392):
 *
 *   - Section 2: the coding function C(s,x) and its inverse D(x) with
 *     C(D(x)) = x.  The paper leaves the concrete C open ("rANS/rABS"); its
 *     worked example in Section 2.1 is the range variant with M = 4.  The
 *     general range form used here is
 *         C(s,x) = floor(x / f_s) * M + B_s + (x mod f_s),  B_s = sum_{t<s} f_t
 *         D(x)   = (s, f_s * floor(x / M) + (x mod M) - B_s)
 *     where s is the unique symbol with B_s <= x mod M < B_s + f_s.
 *     The symbol search in D is a linear scan on purpose (no slot table).
 *   - Section 2, Algorithm 1: streaming encode / decode with the normalized
 *     interval I = [L, bL).  Both loops are literal `while` loops:
 *         Encode: while C(s,x) not in I: emit(x mod b); x = floor(x / b)
 *                 x = C(s,x)
 *         Decode: (s,x) = D(x); while x not in I: x = b*x + read()
 *     The encoder walks the message backwards and the emitted words are
 *     reversed at the end, so the decoder reads them forwards (Section 2,
 *     the stack property and the backwards-encoding convention).  The final
 *     encoder states are transmitted (Section 2).
 *   - Section 3: N coders interleaved into one buffer with no metadata.
 *     Symbol i of a message is handled by coder (i mod N); encoder and
 *     decoder use the same coder sequence.
 *   - Section 5, more than one renormalization digit per symbol (b < M):
 *     a SIMD decoder reads the digits of a step breadth-first across its N
 *     lanes, which bakes N into the stream; orc_*_wide and the byte-wise
 *     container (b = 2^8) follow that order.
 *   - Section 5, adaptive models: they vectorize when every lane has its own
 *     context; orc_*_adaptive codes binary symbols with one adaptive
 *     probability per coder.
 *   - Section 3, bypass: raw digits interleaved with the coded data.  A
 *     symbol may carry raw base-b digits that no coder touches; the encoder
 *     sends them right before encoding the symbol, the decoder reads them
 *     right after decoding it, and the two stay in lockstep.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - initial encoder state x0 = L for every coder;
 *   - symbol i -> coder i mod N;
 *   - production parameters L = 2^16, b = 2^16, M = 2^12 (so b >= M and at
 *     most one renormalization per symbol, Section 5);
 *   - the chunked container (header, offset table, chunk layout) and the
 *     weight -> frequency quantizer are not in the paper at all.
 *
 * Generic entry points take (f[], n, L, b) so the paper's own example
 * (L=16, b=2, M=4) runs through the same code as the production parameters.
 * State arithmetic is done in unsigned __int128 so that C(s,x) inside the
 * encoder's loop test never wraps.
 *
 * Compile-time ORACLE_MUTANT=k plants one deliberate mistake (tests only use
 * this to show that the pins catch it); the default build has none.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

typedef unsigned __int128 u128;

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,       /* bad parameters */
    ORC_ERR_SYMBOL = 2,    /* symbol outside the alphabet or with f_s = 0 */
    ORC_ERR_SPACE = 3,     /* output buffer too small */
    ORC_ERR_CORRUPT = 4,   /* decoder: bad start state, ran out of words,
                              did not end in x0 = L, or left words unread */
    ORC_ERR_INVARIANT = 5  /* x left I after a step (never expected) */
};

#define ORC_MAX_ALPHA 4096u

typedef struct {
    u128 L, b, M;
    uint32_t n;
    u128 f[ORC_MAX_ALPHA];
    u128 B[ORC_MAX_ALPHA];
} orc_model;

/* Build the model: M = sum f_s, B_s = sum_{t<s} f_t (Section 2: the C/D pair
 * of the range variant).  Requires b >= 2 and L >= 1 (Section 2). */
static int model_init(orc_model *m, const uint64_t *f, uint32_t n, uint64_t L, uint64_t b)
{
    if (n == 0 || n > ORC_MAX_ALPHA || L == 0 || b < 2) return ORC_ERR_ARG;
    m->L = L;
    m->b = b;
    m->n = n;
    u128 acc = 0;
    for (uint32_t s = 0; s < n; ++s) {
        m->B[s] = acc;
        m->f[s] = f[s];
        acc += f[s];
    }
    m->M = acc;
    if (acc == 0) return ORC_ERR_ARG;
    return ORC_OK;
}

static int in_I(const orc_model *m, u128 x)
{
    return x >= m->L && x < m->b * m->L;
}

/* C(s,x) = floor(x/f_s)*M + B_s + (x mod f_s). */
static u128 C(const orc_model *m, uint32_t s, u128 x)
{
    u128 f = m->f[s];
#if ORACLE_MUTANT == 1
    return (x / f) * m->M + (x % f);                 /* drops B_s */
#elif ORACLE_MUTANT == 2
    return (x / m->M) * f + m->B[s] + (x % f);       /* M and f swapped */
#else
    return (x / f) * m->M + m->B[s] + (x % f);
#endif
}

/* D(x) = (s, f_s*floor(x/M) + (x mod M) - B_s), s found by a linear scan
 * over the cumulative frequencies. */
static u128 D(const orc_model *m, u128 x, uint32_t *s_out)
{
    u128 r = x % m->M;
    uint32_t s = 0;
    for (s = 0; s < m->n; ++s) {
#if ORACLE_MUTANT == 7
        if (m->B[s] < r && r <= m->B[s] + m->f[s]) break;  /* off by one */
#else
        if (m->B[s] <= r && r < m->B[s] + m->f[s]) break;
#endif
    }
    if (s == m->n) s = m->n - 1;  /* only reachable under a mutant */
    *s_out = s;
    return m->f[s] * (x / m->M) + r - m->B[s];
}

static uint32_t coder_of(uint64_t i, uint32_t N)
{
#if ORACLE_MUTANT == 4
    return (uint32_t)((i + 1) % N);
#else
    return (uint32_t)(i % N);
#endif
}

static u128 initial_state(const orc_model *m)
{
#if ORACLE_MUTANT == 6
    return m->L + 1;
#else
    return m->L;
#endif
}

/* ---------------------------------------------------------------------- */
/* Generic coder: Algorithm 1 run by N interleaved coders (Sections 2, 3). */
/* ---------------------------------------------------------------------- */

static void trace_push(uint64_t *ts, uint32_t *tl, uint64_t cap, uint64_t *nt,
                       uint32_t lane, u128 x)
{
    if (ts && *nt < cap) {
        ts[*nt] = (uint64_t)x;
        if (tl) tl[*nt] = lane;
    }
    if (ts) ++*nt;
}

/*
 * Encode sym[0..n) with N interleaved coders sharing one output buffer.
 * The message is processed backwards (i = n-1 .. 0); coder (i mod N) runs
 * Encode(s_i) of Algorithm 1.  Words go into one shared buffer in emission
 * order; at the end the buffer is reversed so that words[0] is the first
 * word the decoder reads.  states[j] receives coder j's final state.
 *
 * Raw (bypass) digits, Section 3: when r is given, symbol s carries r[s]
 * raw base-b digits that no coder touches.  raw[0..n_raw) holds them in
 * message order (symbol i's digits, first digit first).  The encoder sends a
 * symbol's raw digits right before it encodes the symbol -- in its backwards
 * emission order, last digit first -- so that after the final reversal the
 * decoder finds them right after the words it reads when decoding that
 * symbol.  r = NULL: no raw digits.
 *
 * trace (optional): every state a coder passes through, in encoder order,
 * starting with the N initial states.
 * max_iters (optional): the largest number of renormalization iterations
 * any single symbol needed.
 */
static int encode_impl(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
                       const uint32_t *sym, uint64_t n_sym, const uint32_t *r,
                       const uint64_t *raw, uint64_t n_raw,
                       uint64_t *words, uint64_t word_cap, uint64_t *n_words,
                       uint64_t *states,
                       uint64_t *trace_state, uint32_t *trace_lane, uint64_t trace_cap,
                       uint64_t *n_trace, uint32_t *max_iters)
{
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    if (!mp) return ORC_ERR_ARG;
    int rc = model_init(mp, f, n_alpha, L, b);
    if (rc || N == 0) { free(mp); return rc ? rc : ORC_ERR_ARG; }

    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    if (!x) { free(mp); return ORC_ERR_ARG; }
    uint64_t nt = 0, W = 0, raw_end = n_raw;
    uint32_t worst = 0;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = initial_state(mp);
        trace_push(trace_state, trace_lane, trace_cap, &nt, j, x[j]);
    }

    rc = ORC_OK;
    for (uint64_t i = n_sym; i-- > 0;) {
        uint32_t j = coder_of(i, N);
        uint32_t s = sym[i];
        if (s >= mp->n || mp->f[s] == 0) { rc = ORC_ERR_SYMBOL; break; }
        uint32_t nr = r ? r[s] : 0;
        if (nr > raw_end) { rc = ORC_ERR_ARG; break; }
        raw_end -= nr;
#if ORACLE_MUTANT != 9
        /* Raw digits first: the decoder reads them after decoding s_i. */
        for (uint32_t k = nr; k-- > 0;) {
            if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
            if (raw[raw_end + k] >= (uint64_t)mp->b) { rc = ORC_ERR_ARG; goto done; }
            words[W++] = raw[raw_end + k];
        }
#endif
        uint32_t iters = 0;
        /* Algorithm 1, Encode: renormalize while C(s,x) would leave I. */
        while (!in_I(mp, C(mp, s, x[j]))) {
            if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
#if ORACLE_MUTANT == 3
            words[W++] = (uint64_t)(x[j] / mp->b);      /* wrong digit */
#else
            words[W++] = (uint64_t)(x[j] % mp->b);
#endif
            x[j] = x[j] / mp->b;
            ++iters;
            trace_push(trace_state, trace_lane, trace_cap, &nt, j, x[j]);
            if (x[j] == 0) { rc = ORC_ERR_INVARIANT; goto done; }
        }
        x[j] = C(mp, s, x[j]);
        trace_push(trace_state, trace_lane, trace_cap, &nt, j, x[j]);
        if (!in_I(mp, x[j])) { rc = ORC_ERR_INVARIANT; goto done; }
        if (iters > worst) worst = iters;
#if ORACLE_MUTANT == 9
        /* planted mistake: raw digits sent after the symbol is encoded */
        for (uint32_t k = nr; k-- > 0;) {
            if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
            words[W++] = raw[raw_end + k];
        }
#endif
    }
    if (rc == ORC_OK && raw_end != 0) rc = ORC_ERR_ARG;   /* raw digits left over */
done:
    if (rc == ORC_OK) {
#if ORACLE_MUTANT != 5
        /* Reverse: the encoder wrote backwards, the decoder reads forwards. */
        for (uint64_t a = 0, z = W; a + 1 < z; ++a, --z) {
            uint64_t t = words[a];
            words[a] = words[z - 1];
            words[z - 1] = t;
        }
#endif
        for (uint32_t j = 0; j < N; ++j) states[j] = (uint64_t)x[j];
        *n_words = W;
        if (n_trace) *n_trace = nt;
        if (max_iters) *max_iters = worst;
    }
    free(x);
    free(mp);
    return rc;
}

int orc_encode(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
               const uint32_t *sym, uint64_t n_sym,
               uint64_t *words, uint64_t word_cap, uint64_t *n_words,
               uint64_t *states,
               uint64_t *trace_state, uint32_t *trace_lane, uint64_t trace_cap,
               uint64_t *n_trace, uint32_t *max_iters)
{
    return encode_impl(f, n_alpha, L, b, N, sym, n_sym, NULL, NULL, 0, words, word_cap, n_words,
                       states, trace_state, trace_lane, trace_cap, n_trace, max_iters);
}

int orc_encode_bypass(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
                      const uint32_t *sym, uint64_t n_sym, const uint32_t *r,
                      const uint64_t *raw, uint64_t n_raw,
                      uint64_t *words, uint64_t word_cap, uint64_t *n_words, uint64_t *states,
                      uint64_t *trace_state, uint32_t *trace_lane, uint64_t trace_cap,
                      uint64_t *n_trace)
{
    if (!r) return ORC_ERR_ARG;
    return encode_impl(f, n_alpha, L, b, N, sym, n_sym, r, raw, n_raw, words, word_cap, n_words,
                       states, trace_state, trace_lane, trace_cap, n_trace, NULL);
}

/*
 * Decode n_sym symbols.  Coder (i mod N) runs Decode of Algorithm 1 for
 * symbol i, all coders reading the one shared word buffer in order
 * (Section 3); with r given, the r[s_i] raw digits of symbol i are read
 * right after it (Section 3, bypass) into raw_out (message order).
 * states_in are the transmitted final encoder states.  consumed: words
 * read.  states_out: coder states at the end (equal to the encoder's initial
 * states for a well-formed stream).
 */
static int decode_impl(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
                       const uint64_t *words, uint64_t n_words, const uint64_t *states_in,
                       uint64_t n_sym, const uint32_t *r, uint32_t *sym_out,
                       uint64_t *raw_out, uint64_t raw_cap, uint64_t *n_raw_out,
                       uint64_t *consumed, uint64_t *states_out,
                       uint64_t *trace_state, uint32_t *trace_lane, uint64_t trace_cap,
                       uint64_t *n_trace, uint32_t *max_iters)
{
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    if (!mp) return ORC_ERR_ARG;
    int rc = model_init(mp, f, n_alpha, L, b);
    if (rc || N == 0) { free(mp); return rc ? rc : ORC_ERR_ARG; }
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    if (!x) { free(mp); return ORC_ERR_ARG; }

    uint64_t nt = 0, rp = 0, nr_out = 0;
    uint32_t worst = 0;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = states_in[j];
        if (!in_I(mp, x[j])) rc = ORC_ERR_CORRUPT;   /* Algorithm 1 requires x in I */
        trace_push(trace_state, trace_lane, trace_cap, &nt, j, x[j]);
    }
    if (rc) goto out;

    for (uint64_t i = 0; i < n_sym; ++i) {
        uint32_t j = coder_of(i, N);
        uint32_t s;
        x[j] = D(mp, x[j], &s);
        sym_out[i] = s;
        trace_push(trace_state, trace_lane, trace_cap, &nt, j, x[j]);
        uint32_t iters = 0;
        while (!in_I(mp, x[j])) {
            if (rp >= n_words || x[j] >= mp->L * mp->b) { rc = ORC_ERR_CORRUPT; goto out; }
            x[j] = mp->b * x[j] + words[rp++];
            ++iters;
            trace_push(trace_state, trace_lane, trace_cap, &nt, j, x[j]);
        }
        if (iters > worst) worst = iters;
        for (uint32_t k = 0; r && k < r[s]; ++k) {
            if (rp >= n_words) { rc = ORC_ERR_CORRUPT; goto out; }
            if (nr_out >= raw_cap) { rc = ORC_ERR_SPACE; goto out; }
            raw_out[nr_out++] = words[rp++];
        }
    }
    for (uint32_t j = 0; j < N; ++j) states_out[j] = (uint64_t)x[j];
    *consumed = rp;
    if (n_raw_out) *n_raw_out = nr_out;
    if (n_trace) *n_trace = nt;
    if (max_iters) *max_iters = worst;
out:
    free(x);
    free(mp);
    return rc;
}

int orc_decode(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
               const uint64_t *words, uint64_t n_words, const uint64_t *states_in,
               uint64_t n_sym, uint32_t *sym_out, uint64_t *consumed, uint64_t *states_out,
               uint64_t *trace_state, uint32_t *trace_lane, uint64_t trace_cap,
               uint64_t *n_trace, uint32_t *max_iters)
{
    return decode_impl(f, n_alpha, L, b, N, words, n_words, states_in, n_sym, NULL, sym_out,
                       NULL, 0, NULL, consumed, states_out, trace_state, trace_lane, trace_cap,
                       n_trace, max_iters);
}

int orc_decode_bypass(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
                      const uint64_t *words, uint64_t n_words, const uint64_t *states_in,
                      uint64_t n_sym, const uint32_t *r, uint32_t *sym_out,
                      uint64_t *raw_out, uint64_t raw_cap, uint64_t *n_raw_out,
                      uint64_t *consumed, uint64_t *states_out,
                      uint64_t *trace_state, uint32_t *trace_lane, uint64_t trace_cap,
                      uint64_t *n_trace)
{
    if (!r) return ORC_ERR_ARG;
    return decode_impl(f, n_alpha, L, b, N, words, n_words, states_in, n_sym, r, sym_out,
                       raw_out, raw_cap, n_raw_out, consumed, states_out, trace_state,
                       trace_lane, trace_cap, n_trace, NULL);
}

/* ---------------------------------------------------------------------- */
/* Width-baked interleaving (Section 5): several renormalization digits    */
/* per symbol, read breadth-first across the N lanes of a step.            */
/* ---------------------------------------------------------------------- */

/*
 * Symbols go in steps of N (step t holds symbols tN .. tN+N-1, symbol tN+j
 * on lane j = coder j; the last step may be partial).  Decoder, per step:
 * every lane decodes its symbol (D); then in rounds r = 1, 2, ... every lane
 * still below L reads one digit, lanes in order, until all lanes are in I.
 * That is the order of a SIMD decoder with one lane per coder; it differs
 * from Algorithm 1's depth-first order as soon as a lane needs two digits,
 * so N is part of the stream.  The encoder gives the same order: per step it
 * renormalizes and codes every lane (lanes are independent coders), then
 * lays the step's digits out round by round -- lane j's digits in the order
 * its decoder reads them, high digit first.  With N = 1 this is Algorithm 1.
 */
#define ORC_WIDE_MAX_DIGITS 128u
int orc_encode_wide(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
                    const uint32_t *sym, uint64_t n_sym, uint64_t *words, uint64_t word_cap,
                    uint64_t *n_words, uint64_t *states)
{
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    if (!mp) return ORC_ERR_ARG;
    int rc = model_init(mp, f, n_alpha, L, b);
    if (rc || N == 0) { free(mp); return rc ? rc : ORC_ERR_ARG; }
    uint64_t T = (n_sym + N - 1) / N;
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    uint64_t *dig = (uint64_t *)malloc(sizeof(uint64_t) * N * ORC_WIDE_MAX_DIGITS);
    uint32_t *k = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (word_cap ? word_cap : 1));
    uint64_t *bstart = (uint64_t *)malloc(sizeof(uint64_t) * (T ? T : 1));
    uint64_t *blen = (uint64_t *)malloc(sizeof(uint64_t) * (T ? T : 1));
    if (!x || !dig || !k || !tmp || !bstart || !blen) { rc = ORC_ERR_ARG; goto done; }
    for (uint32_t j = 0; j < N; ++j) x[j] = initial_state(mp);
    uint64_t W = 0;
    for (uint64_t t = T; t-- > 0;) {
        uint32_t lanes = (t == T - 1 && n_sym % N) ? (uint32_t)(n_sym % N) : N;
        uint32_t kmax = 0;
        for (uint32_t j = 0; j < lanes; ++j) {
            uint32_t s = sym[t * N + j];
            if (s >= mp->n || mp->f[s] == 0) { rc = ORC_ERR_SYMBOL; goto done; }
            k[j] = 0;
            while (!in_I(mp, C(mp, s, x[j]))) {            /* Algorithm 1, Encode */
                if (k[j] >= ORC_WIDE_MAX_DIGITS) { rc = ORC_ERR_ARG; goto done; }
                dig[(uint64_t)j * ORC_WIDE_MAX_DIGITS + k[j]++] = (uint64_t)(x[j] % mp->b);
                x[j] = x[j] / mp->b;
            }
            x[j] = C(mp, s, x[j]);
            if (!in_I(mp, x[j])) { rc = ORC_ERR_INVARIANT; goto done; }
            if (k[j] > kmax) kmax = k[j];
        }
        bstart[t] = W;
#if ORACLE_MUTANT == 10
        /* planted mistake: depth-first (lane by lane) instead of round by round */
        for (uint32_t j = 0; j < lanes; ++j)
            for (uint32_t r = 1; r <= k[j]; ++r) {
                if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
                tmp[W++] = dig[(uint64_t)j * ORC_WIDE_MAX_DIGITS + k[j] - r];
            }
#else
        for (uint32_t r = 1; r <= kmax; ++r)               /* round r: lanes in order */
            for (uint32_t j = 0; j < lanes; ++j)
                if (k[j] >= r) {
                    if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
                    tmp[W++] = dig[(uint64_t)j * ORC_WIDE_MAX_DIGITS + k[j] - r];
                }
#endif
        blen[t] = W - bstart[t];
    }
    {
        uint64_t o = 0;                                     /* steps in decoder order */
        for (uint64_t t = 0; t < T; ++t)
            for (uint64_t q = 0; q < blen[t]; ++q) words[o++] = tmp[bstart[t] + q];
    }
    for (uint32_t j = 0; j < N; ++j) states[j] = (uint64_t)x[j];
    *n_words = W;
    rc = ORC_OK;
done:
    free(x); free(dig); free(k); free(tmp); free(bstart); free(blen); free(mp);
    return rc;
}

int orc_decode_wide(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
                    const uint64_t *words, uint64_t n_words, const uint64_t *states_in,
                    uint64_t n_sym, uint32_t *sym_out, uint64_t *consumed, uint64_t *states_out)
{
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    if (!mp) return ORC_ERR_ARG;
    int rc = model_init(mp, f, n_alpha, L, b);
    if (rc || N == 0) { free(mp); return rc ? rc : ORC_ERR_ARG; }
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    if (!x) { free(mp); return ORC_ERR_ARG; }
    uint64_t rp = 0, T = (n_sym + N - 1) / N;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = states_in[j];
        if (!in_I(mp, x[j])) rc = ORC_ERR_CORRUPT;
    }
    for (uint64_t t = 0; !rc && t < T; ++t) {
        uint32_t lanes = (t == T - 1 && n_sym % N) ? (uint32_t)(n_sym % N) : N;
        for (uint32_t j = 0; j < lanes; ++j) {
            uint32_t s;
            x[j] = D(mp, x[j], &s);
            sym_out[t * N + j] = s;
        }
        for (int any = 1; any && !rc;) {                    /* rounds */
            any = 0;
            for (uint32_t j = 0; j < lanes; ++j)
                if (!in_I(mp, x[j])) {
                    if (rp >= n_words || x[j] >= mp->L * mp->b) { rc = ORC_ERR_CORRUPT; break; }
                    x[j] = mp->b * x[j] + words[rp++];
                    any = 1;
                }
        }
    }
    if (!rc) {
        for (uint32_t j = 0; j < N; ++j) states_out[j] = (uint64_t)x[j];
        *consumed = rp;
    }
    free(x);
    free(mp);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Adaptive binary models, one context per coder (Section 5: adaptive      */
/* models vectorize when no two lanes update the same model).              */
/* ---------------------------------------------------------------------- */

/*
 * Binary alphabet {0, 1}.  Coder j keeps its own probability p_j of a 0,
 * scaled to M (1 <= p_j <= M-1), starting at p0.  Symbol s is coded with
 * f_0 = p, f_1 = M - p, B_0 = 0, B_1 = p (the range form of Section 2), and
 * afterwards the coder's context moves towards s:
 *     s = 0:  p += (M - p) >> R        s = 1:  p -= p >> R
 * Coder j's context sees only its own symbols j, j+N, j+2N, ...  The
 * decoder updates after decoding; the encoder, which runs backwards, first
 * runs every context forwards to know the p each symbol was coded with.
 */
static void adapt(u128 *p, uint32_t s, u128 M, uint32_t R)
{
    if (s == 0) *p += (M - *p) >> R;
    else *p -= *p >> R;
}

static int adaptive_model(orc_model *m, u128 p, u128 M, uint64_t L, uint64_t b)
{
    uint64_t f[2] = {(uint64_t)p, (uint64_t)(M - p)};
    return model_init(m, f, 2, L, b);
}

int orc_encode_adaptive(uint64_t M, uint64_t L, uint64_t b, uint32_t N, uint32_t R, uint64_t p0,
                        const uint32_t *sym, uint64_t n_sym, uint64_t *words, uint64_t word_cap,
                        uint64_t *n_words, uint64_t *states)
{
    if (N == 0 || M < 2 || p0 < 1 || p0 >= M || R == 0 || R > 30) return ORC_ERR_ARG;
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    u128 *ctx = (u128 *)malloc(sizeof(u128) * N);
    u128 *pi = (u128 *)malloc(sizeof(u128) * (n_sym ? n_sym : 1));
    int rc = ORC_OK;
    uint64_t W = 0;
    if (!mp || !x || !ctx || !pi) { rc = ORC_ERR_ARG; goto done; }
    /* forward: the probability every symbol is coded with */
    for (uint32_t j = 0; j < N; ++j) ctx[j] = p0;
    for (uint64_t i = 0; i < n_sym; ++i) {
        uint32_t j = coder_of(i, N);
        if (sym[i] > 1) { rc = ORC_ERR_SYMBOL; goto done; }
#if ORACLE_MUTANT == 11
        adapt(&ctx[j], sym[i], M, R);          /* planted mistake: update before coding */
        pi[i] = ctx[j];
#else
        pi[i] = ctx[j];
        adapt(&ctx[j], sym[i], M, R);
#endif
    }
    /* backwards: Algorithm 1 with symbol i's model */
    if ((rc = adaptive_model(mp, p0, M, L, b)) != ORC_OK) goto done;
    for (uint32_t j = 0; j < N; ++j) x[j] = initial_state(mp);
    for (uint64_t i = n_sym; i-- > 0;) {
        uint32_t j = coder_of(i, N), s = sym[i];
        if ((rc = adaptive_model(mp, pi[i], M, L, b)) != ORC_OK) goto done;
        while (!in_I(mp, C(mp, s, x[j]))) {
            if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
            words[W++] = (uint64_t)(x[j] % mp->b);
            x[j] = x[j] / mp->b;
        }
        x[j] = C(mp, s, x[j]);
        if (!in_I(mp, x[j])) { rc = ORC_ERR_INVARIANT; goto done; }
    }
    for (uint64_t a = 0, z = W; a + 1 < z; ++a, --z) {
        uint64_t t = words[a];
        words[a] = words[z - 1];
        words[z - 1] = t;
    }
    for (uint32_t j = 0; j < N; ++j) states[j] = (uint64_t)x[j];
    *n_words = W;
done:
    free(mp); free(x); free(ctx); free(pi);
    return rc;
}

int orc_decode_adaptive(uint64_t M, uint64_t L, uint64_t b, uint32_t N, uint32_t R, uint64_t p0,
                        const uint64_t *words, uint64_t n_words, const uint64_t *states_in,
                        uint64_t n_sym, uint32_t *sym_out, uint64_t *consumed,
                        uint64_t *states_out)
{
    if (N == 0 || M < 2 || p0 < 1 || p0 >= M || R == 0 || R > 30) return ORC_ERR_ARG;
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    u128 *ctx = (u128 *)malloc(sizeof(u128) * N);
    int rc = ORC_OK;
    uint64_t rp = 0;
    if (!mp || !x || !ctx) { rc = ORC_ERR_ARG; goto done; }
    if ((rc = adaptive_model(mp, p0, M, L, b)) != ORC_OK) goto done;
    for (uint32_t j = 0; j < N; ++j) {
        x[j] = states_in[j];
        ctx[j] = p0;
        if (!in_I(mp, x[j])) rc = ORC_ERR_CORRUPT;
    }
    for (uint64_t i = 0; !rc && i < n_sym; ++i) {
        uint32_t j = coder_of(i, N), s;
        if ((rc = adaptive_model(mp, ctx[j], M, L, b)) != ORC_OK) break;
        x[j] = D(mp, x[j], &s);
        sym_out[i] = s;
        while (!in_I(mp, x[j])) {
            if (rp >= n_words || x[j] >= mp->L * mp->b) { rc = ORC_ERR_CORRUPT; break; }
            x[j] = mp->b * x[j] + words[rp++];
        }
        adapt(&ctx[j], s, M, R);
    }
    if (!rc) {
        for (uint32_t j = 0; j < N; ++j) states_out[j] = (uint64_t)x[j];
        *consumed = rp;
    }
done:
    free(mp); free(x); free(ctx);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Adaptive models over n symbols, one per coder (Section 5: the lanes'    */
/* models must evolve independently for the coders to vectorize).         */
/* ---------------------------------------------------------------------- */

/*
 * Alphabet {0..n-1}, 2 <= n <= ORC_ADAPT_NMAX.  Coder j keeps its own
 * cumulative frequencies C_0 = 0 < C_1 < ... < C_n = M, so f_s = C_{s+1} - C_s
 * and B_s = C_s (the range form of Section 2), starting from
 * C_i = floor(i * M / n).  After coding symbol s every interior boundary
 * 1 <= i <= n-1 moves a 2^-R part of the way to its target, rounded down:
 *     i <= s:  C_i -= (C_i - i) >> R            (target i)
 *     i >  s:  C_i += (M - n + i - C_i) >> R    (target M - n + i)
 * so symbol s's interval [C_s, C_{s+1}) widens and the others narrow.
 * Every f stays >= 1 and every boundary within [i, M - n + i]:
 *   - two boundaries below s: with a_i = C_i - i, a_{i+1} >= a_i (since
 *     f_i >= 1), and a -> a - (a >> R) is non-decreasing, so the new
 *     a_{i+1} >= a_i again, i.e. the new f_i >= 1;
 *   - two above s: the same with u_i = M - n + i - C_i (u_{i+1} <= u_i);
 *   - across s: C_s moves down and C_{s+1} up.
 * The decoder updates after decoding; the encoder, which runs backwards,
 * first runs every coder's model forwards to know each symbol's (B_s, f_s).
 * (The binary contexts above use a different rounding; n = 2 here is its
 * own model, not the same as them.)
 */
#define ORC_ADAPT_NMAX 16u

static void cdf_init(u128 *c, uint32_t n, u128 M)
{
    for (uint32_t i = 0; i <= n; ++i) c[i] = (u128)i * M / n;
}

static void cdf_adapt(u128 *c, uint32_t n, u128 M, uint32_t R, uint32_t s)
{
    for (uint32_t i = 1; i < n; ++i) {
#if ORACLE_MUTANT == 15
        if (i < s)                                  /* planted mistake: C_s moves up */
#else
        if (i <= s)
#endif
            c[i] -= (c[i] - i) >> R;
        else
            c[i] += (M - n + i - c[i]) >> R;
    }
}

/* The model a coder's cumulative frequencies give (model_init's form). */
static int cdf_model(orc_model *m, const u128 *c, uint32_t n, uint64_t L, uint64_t b)
{
    uint64_t f[ORC_ADAPT_NMAX];
    for (uint32_t s = 0; s < n; ++s) f[s] = (uint64_t)(c[s + 1] - c[s]);
    return model_init(m, f, n, L, b);
}

static int adapt_n_args(uint64_t M, uint32_t N, uint32_t R, uint32_t n)
{
    return N == 0 || n < 2 || n > ORC_ADAPT_NMAX || M < n || R == 0 || R > 30;
}

/* The cumulative frequencies of one context over sym[0..n_sym): row k of
 * cdf_out ((n_sym + 1) x (n + 1) values) is the model symbol k is coded
 * with; row n_sym the model after the last symbol. */
int orc_adaptive_n_trace(uint64_t M, uint32_t R, uint32_t n, const uint32_t *sym, uint64_t n_sym,
                         uint64_t *cdf_out)
{
    if (adapt_n_args(M, 1, R, n)) return ORC_ERR_ARG;
    u128 c[ORC_ADAPT_NMAX + 1];
    cdf_init(c, n, M);
    for (uint64_t k = 0; k <= n_sym; ++k) {
        for (uint32_t i = 0; i <= n; ++i) cdf_out[k * (n + 1) + i] = (uint64_t)c[i];
        if (k == n_sym) break;
        if (sym[k] >= n) return ORC_ERR_SYMBOL;
        cdf_adapt(c, n, M, R, sym[k]);
    }
    return ORC_OK;
}

int orc_encode_adaptive_n(uint64_t M, uint64_t L, uint64_t b, uint32_t N, uint32_t R, uint32_t n,
                          const uint32_t *sym, uint64_t n_sym, uint64_t *words, uint64_t word_cap,
                          uint64_t *n_words, uint64_t *states)
{
    if (adapt_n_args(M, N, R, n)) return ORC_ERR_ARG;
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    u128 *cdf = (u128 *)malloc(sizeof(u128) * N * (ORC_ADAPT_NMAX + 1));
    u128 *Bi = (u128 *)malloc(sizeof(u128) * (n_sym ? n_sym : 1));
    u128 *fi = (u128 *)malloc(sizeof(u128) * (n_sym ? n_sym : 1));
    int rc = ORC_OK;
    uint64_t W = 0;
    if (!mp || !x || !cdf || !Bi || !fi) { rc = ORC_ERR_ARG; goto done; }
    /* forward: the (B_s, f_s) every symbol is coded with */
    for (uint32_t j = 0; j < N; ++j) cdf_init(cdf + j * (ORC_ADAPT_NMAX + 1), n, M);
    for (uint64_t i = 0; i < n_sym; ++i) {
        uint32_t j = coder_of(i, N), s = sym[i];
        u128 *c = cdf + j * (ORC_ADAPT_NMAX + 1);
        if (s >= n) { rc = ORC_ERR_SYMBOL; goto done; }
#if ORACLE_MUTANT == 14
        cdf_adapt(c, n, M, R, s);                   /* planted mistake: update before coding */
        Bi[i] = c[s];
        fi[i] = c[s + 1] - c[s];
#else
        Bi[i] = c[s];
        fi[i] = c[s + 1] - c[s];
        cdf_adapt(c, n, M, R, s);
#endif
    }
    /* backwards: Algorithm 1 with symbol i's model.  C(s, x) needs only M,
     * B_s and f_s, so the three-part model [B_s, f_s, M - B_s - f_s] with the
     * symbol in the middle gives the same C as the coder's full model. */
    if ((rc = cdf_model(mp, cdf, n, L, b)) != ORC_OK) goto done;
    for (uint32_t j = 0; j < N; ++j) x[j] = initial_state(mp);
    for (uint64_t i = n_sym; i-- > 0;) {
        uint32_t j = coder_of(i, N);
        uint64_t part[3] = {(uint64_t)Bi[i], (uint64_t)fi[i], (uint64_t)(M - Bi[i] - fi[i])};
        if ((rc = model_init(mp, part, 3, L, b)) != ORC_OK) goto done;
        while (!in_I(mp, C(mp, 1, x[j]))) {
            if (W >= word_cap) { rc = ORC_ERR_SPACE; goto done; }
            words[W++] = (uint64_t)(x[j] % mp->b);
            x[j] = x[j] / mp->b;
        }
        x[j] = C(mp, 1, x[j]);
        if (!in_I(mp, x[j])) { rc = ORC_ERR_INVARIANT; goto done; }
    }
    for (uint64_t a = 0, z = W; a + 1 < z; ++a, --z) {
        uint64_t t = words[a];
        words[a] = words[z - 1];
        words[z - 1] = t;
    }
    for (uint32_t j = 0; j < N; ++j) states[j] = (uint64_t)x[j];
    *n_words = W;
done:
    free(mp); free(x); free(cdf); free(Bi); free(fi);
    return rc;
}

int orc_decode_adaptive_n(uint64_t M, uint64_t L, uint64_t b, uint32_t N, uint32_t R, uint32_t n,
                          const uint64_t *words, uint64_t n_words, const uint64_t *states_in,
                          uint64_t n_sym, uint32_t *sym_out, uint64_t *consumed,
                          uint64_t *states_out)
{
    if (adapt_n_args(M, N, R, n)) return ORC_ERR_ARG;
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    u128 *x = (u128 *)malloc(sizeof(u128) * N);
    u128 *cdf = (u128 *)malloc(sizeof(u128) * N * (ORC_ADAPT_NMAX + 1));
    int rc = ORC_OK;
    uint64_t rp = 0;
    if (!mp || !x || !cdf) { rc = ORC_ERR_ARG; goto done; }
    for (uint32_t j = 0; j < N; ++j) {
        cdf_init(cdf + j * (ORC_ADAPT_NMAX + 1), n, M);
        x[j] = states_in[j];
        if (x[j] < L || x[j] >= (u128)L * b) rc = ORC_ERR_CORRUPT;   /* x must be in I */
    }
    for (uint64_t i = 0; !rc && i < n_sym; ++i) {
        uint32_t j = coder_of(i, N), s;
        u128 *c = cdf + j * (ORC_ADAPT_NMAX + 1);
        if ((rc = cdf_model(mp, c, n, L, b)) != ORC_OK) break;
        x[j] = D(mp, x[j], &s);
        sym_out[i] = s;
        while (!in_I(mp, x[j])) {
            if (rp >= n_words || x[j] >= mp->L * mp->b) { rc = ORC_ERR_CORRUPT; break; }
            x[j] = mp->b * x[j] + words[rp++];
        }
        cdf_adapt(c, n, M, R, s);
    }
    if (!rc) {
        for (uint32_t j = 0; j < N; ++j) states_out[j] = (uint64_t)x[j];
        *consumed = rp;
    }
done:
    free(mp); free(x); free(cdf);
    return rc;
}

/* Single coding-function evaluations, for checking the oracle against the
 * paper's printed example (Section 2.1).  *ok = 0 on bad input. */
uint64_t orc_C(const uint64_t *f, uint32_t n_alpha, uint32_t s, uint64_t x, int *ok)
{
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    *ok = 0;
    if (!mp) return 0;
    if (model_init(mp, f, n_alpha, 1, 2) || s >= n_alpha || f[s] == 0) { free(mp); return 0; }
    u128 r = C(mp, s, x);
    free(mp);
    if (r >> 64) return 0;
    *ok = 1;
    return (uint64_t)r;
}

uint64_t orc_D(const uint64_t *f, uint32_t n_alpha, uint64_t x, uint32_t *s_out, int *ok)
{
    orc_model *mp = (orc_model *)malloc(sizeof(orc_model));
    *ok = 0;
    if (!mp) return 0;
    if (model_init(mp, f, n_alpha, 1, 2)) { free(mp); return 0; }
    u128 r = D(mp, x, s_out);
    free(mp);
    *ok = 1;
    return (uint64_t)r;
}

/* ---------------------------------------------------------------------- */
/* Container with the production parameters (not in the paper).          */
/*                                                                        */
/*   L = 2^16, b = 2^16, M = 2^12, 32-bit states, 16-bit words.           */
/*   header (32 bytes, little endian):                                    */
/*     u32 magic 0x534E4152, u32 version 1, u32 N, u32 log2_M (12),       */
/*     u64 n_symbols, u32 chunk_symbols, u32 n_chunks                     */
/*   u32 offsets[n_chunks+1], chunk start byte offsets within the data    */
/*     region, offsets[0] = 0, offsets[n_chunks] = data bytes             */
/*   zero padding to 16 bytes; data region; zero padding to 16 bytes.    */
/*   chunk c = symbols [c*chunk_symbols, min(n, (c+1)*chunk_symbols)):    */
/*     u32 state[N] (coder order) then u16 word[W_c] in decoder order.    */
/* ---------------------------------------------------------------------- */

#define ORC_MAGIC 0x534E4152u
#define ORC_VERSION 1u
#define ORC_VERSION_BYPASS 2u  /* messages with raw words (Section 3, bypass) */
#define ORC_VERSION_BYTES 3u   /* byte-wise, width-baked messages (Section 5) */
#define ORC_VERSION_ADAPTIVE 4u /* adaptive binary contexts, one per coder */
#define ORC_ADAPT_RATE 5u      /* adaptive messages: p moves by (target - p) >> 5 */
#define ORC_ADAPT_P0 2048u     /* ... from p = M/2 at the start of every chunk */
#define ORC_VERSION_ADAPTIVE_N 6u /* adaptive models over n <= 16 symbols, one per coder;
                                     the header's log2_M word holds 12 | n << 16 */
#define ORC_L8 (1ull << 23)    /* byte-wise: L = 2^23, b = 2^8, I = [2^23, 2^31) */
#define ORC_B8 (1ull << 8)
#define ORC_L (1ull << 16)
#define ORC_B (1ull << 16)
#define ORC_LOG2_M 12u
#define ORC_LOG2_M_MAX 14u     /* plain messages: M = 2^12, 2^13 or 2^14 */

static void put_u32(uint8_t *p, uint32_t v)
{
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static void put_u16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static uint32_t get_u32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint32_t get_u16(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint64_t round16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

static int prod_table(const uint16_t *freq, uint32_t n_alpha, uint64_t *f64)
{
    if (n_alpha == 0 || n_alpha > 256) return ORC_ERR_ARG;
    uint64_t sum = 0;
    for (uint32_t s = 0; s < n_alpha; ++s) { f64[s] = freq[s]; sum += freq[s]; }
    return sum == (1ull << ORC_LOG2_M) ? ORC_OK : ORC_ERR_ARG;
}

/* Plain messages may also use M = 2^13 or 2^14 (Section 5: with b = 2^16 a
 * coder in 32-bit integers keeps one renormalization per symbol at 12-14
 * bits of probability resolution, since b >= M); M is the table's sum and
 * the header records log2(M).  Other kinds keep M = 2^12. */
static int plain_table(const uint16_t *freq, uint32_t n_alpha, uint64_t *f64, int wide_ok,
                       uint32_t *log2_m)
{
    if (n_alpha == 0 || n_alpha > 256) return ORC_ERR_ARG;
    uint64_t sum = 0;
    for (uint32_t s = 0; s < n_alpha; ++s) { f64[s] = freq[s]; sum += freq[s]; }
    for (uint32_t lm = ORC_LOG2_M; lm <= (wide_ok ? ORC_LOG2_M_MAX : ORC_LOG2_M); ++lm)
        if (sum == (1ull << lm)) { *log2_m = lm; return ORC_OK; }
    return ORC_ERR_ARG;
}

/* Worst case: one word per symbol, since b >= M allows at most one
 * renormalization per symbol (Section 5); with raw words, one more word per
 * symbol at most. */
static uint64_t max_size(uint64_t n_sym, uint32_t N, uint32_t chunk_symbols, uint64_t per_sym)
{
    if (chunk_symbols == 0 || N == 0) return 0;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    return round16(32 + 4 * (n_chunks + 1)) + round16(4ull * N * n_chunks + per_sym * n_sym);
}
uint64_t orc_max_message_size(uint64_t n_sym, uint32_t N, uint32_t chunk_symbols)
{
    return max_size(n_sym, N, chunk_symbols, 2);
}
uint64_t orc_max_message_size_bypass(uint64_t n_sym, uint32_t N, uint32_t chunk_symbols)
{
    return max_size(n_sym, N, chunk_symbols, 4);
}

/* Raw-word flags of a bypass model: rawf[s] in {0, 1} is the number of raw
 * 16-bit words symbol s carries (one base-2^16 digit at most). */
static int raw_counts(const uint8_t *rawf, uint32_t n_alpha, uint32_t *r)
{
    for (uint32_t s = 0; s < n_alpha; ++s) {
        if (rawf[s] > 1) return ORC_ERR_ARG;
        r[s] = rawf[s];
    }
    return ORC_OK;
}

/* One chunk: [u32 state[N]][u16 words in decoder order].  rawf != NULL: a
 * bypass chunk, symbol i followed by raw16[i] when rawf[sym[i]] = 1. */
static int chunk_encode(const uint8_t *sym, const uint16_t *raw16, uint64_t n_c,
                        const uint16_t *freq, const uint8_t *rawf, uint32_t n_alpha, uint32_t N,
                        uint8_t *out, uint64_t cap, uint64_t *size)
{
    uint64_t f64[256];
    uint32_t r[256], lm;
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    int rc = plain_table(freq, n_alpha, f64, rawf == NULL, &lm);
    if (!rc && rawf) rc = raw_counts(rawf, n_alpha, r);
    if (rc) return rc;
    uint64_t cap_w = 3 * (n_c ? n_c : 1);
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * cap_w);
    uint64_t *raw = (uint64_t *)malloc(sizeof(uint64_t) * (n_c ? n_c : 1));
    if (!s32 || !w || !raw) { free(s32); free(w); free(raw); return ORC_ERR_ARG; }
    uint64_t n_raw = 0;
    for (uint64_t i = 0; i < n_c; ++i) {
        s32[i] = sym[i];
        if (rawf && sym[i] < n_alpha && r[sym[i]]) raw[n_raw++] = raw16[i];
    }
    uint64_t st[32], W = 0;
    rc = encode_impl(f64, n_alpha, ORC_L, ORC_B, N, s32, n_c, rawf ? r : NULL, raw, n_raw, w,
                     cap_w, &W, st, NULL, NULL, 0, NULL, NULL);
    if (rc == ORC_OK) {
        uint64_t need = 4ull * N + 2ull * W;
        if (need > cap) rc = ORC_ERR_SPACE;
        else {
            for (uint32_t j = 0; j < N; ++j) put_u32(out + 4 * j, (uint32_t)st[j]);
            for (uint64_t k = 0; k < W; ++k) put_u16(out + 4ull * N + 2 * k, (uint32_t)w[k]);
            *size = need;
        }
    }
    free(s32);
    free(w);
    free(raw);
    return rc;
}

/* raw_out[i] = the raw word of symbol i, or 0 for a symbol without one. */
static int chunk_decode(const uint8_t *chunk, uint64_t size, const uint16_t *freq,
                        const uint8_t *rawf, uint32_t n_alpha, uint32_t N, uint8_t *sym_out,
                        uint16_t *raw_out, uint64_t n_c)
{
    uint64_t f64[256];
    uint32_t r[256], lm;
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    int rc = plain_table(freq, n_alpha, f64, rawf == NULL, &lm);
    if (!rc && rawf) rc = raw_counts(rawf, n_alpha, r);
    if (rc) return rc;
    if (size < 4ull * N || ((size - 4ull * N) & 1)) return ORC_ERR_CORRUPT;
    uint64_t W = (size - 4ull * N) / 2;
    uint64_t st[32], st_end[32], used = 0, n_raw = 0;
    for (uint32_t j = 0; j < N; ++j) st[j] = get_u32(chunk + 4 * j);
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (W ? W : 1));
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    uint64_t *raw = (uint64_t *)malloc(sizeof(uint64_t) * (n_c ? n_c : 1));
    if (!w || !s32 || !raw) { free(w); free(s32); free(raw); return ORC_ERR_ARG; }
    for (uint64_t k = 0; k < W; ++k) w[k] = get_u16(chunk + 4ull * N + 2 * k);
    rc = decode_impl(f64, n_alpha, ORC_L, ORC_B, N, w, W, st, n_c, rawf ? r : NULL, s32, raw,
                     n_c ? n_c : 1, &n_raw, &used, st_end, NULL, NULL, 0, NULL, NULL);
    if (rc == ORC_OK) {
        /* A well-formed chunk ends with every coder back at x0 = L and every
         * word consumed (the decoder unwinds the encoder exactly, Section 3). */
        for (uint32_t j = 0; j < N; ++j)
            if (st_end[j] != ORC_L) rc = ORC_ERR_CORRUPT;
        if (used != W) rc = ORC_ERR_CORRUPT;
        uint64_t k = 0;
        for (uint64_t i = 0; i < n_c; ++i) {
            sym_out[i] = (uint8_t)s32[i];
            if (raw_out) raw_out[i] = (rawf && r[s32[i]]) ? (uint16_t)raw[k++] : 0;
        }
    }
    free(w);
    free(s32);
    free(raw);
    return rc;
}

int orc_encode_chunk(const uint8_t *sym, uint64_t n_c, const uint16_t *freq, uint32_t n_alpha,
                     uint32_t N, uint8_t *out, uint64_t cap, uint64_t *size)
{
    return chunk_encode(sym, NULL, n_c, freq, NULL, n_alpha, N, out, cap, size);
}
int orc_decode_chunk(const uint8_t *chunk, uint64_t size, const uint16_t *freq, uint32_t n_alpha,
                     uint32_t N, uint8_t *sym_out, uint64_t n_c)
{
    return chunk_decode(chunk, size, freq, NULL, n_alpha, N, sym_out, NULL, n_c);
}
int orc_encode_chunk_bypass(const uint8_t *sym, const uint16_t *raw16, uint64_t n_c,
                            const uint16_t *freq, const uint8_t *rawf, uint32_t n_alpha,
                            uint32_t N, uint8_t *out, uint64_t cap, uint64_t *size)
{
    if (!rawf || !raw16) return ORC_ERR_ARG;
    return chunk_encode(sym, raw16, n_c, freq, rawf, n_alpha, N, out, cap, size);
}
int orc_decode_chunk_bypass(const uint8_t *chunk, uint64_t size, const uint16_t *freq,
                            const uint8_t *rawf, uint32_t n_alpha, uint32_t N, uint8_t *sym_out,
                            uint16_t *raw_out, uint64_t n_c)
{
    if (!rawf || !raw_out) return ORC_ERR_ARG;
    return chunk_decode(chunk, size, freq, rawf, n_alpha, N, sym_out, raw_out, n_c);
}

/* Byte-wise chunk (version 3): [u32 state[N]][u8 digits, breadth-first per
 * step][zero bytes up to a multiple of 4].  b = 2^8 < M = 2^12, so a lane
 * can read two digits for one symbol (Section 5); N is part of the stream. */
static uint64_t round4(uint64_t v) { return (v + 3u) & ~(uint64_t)3u; }

static int chunk_encode_bytes(const uint8_t *sym, uint64_t n_c, const uint16_t *freq,
                              uint32_t n_alpha, uint32_t N, uint8_t *out, uint64_t cap,
                              uint64_t *size)
{
    uint64_t f64[256];
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    int rc = prod_table(freq, n_alpha, f64);
    if (rc) return rc;
    uint64_t cap_w = 2 * (n_c ? n_c : 1) + 8;
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * cap_w);
    if (!s32 || !w) { free(s32); free(w); return ORC_ERR_ARG; }
    for (uint64_t i = 0; i < n_c; ++i) s32[i] = sym[i];
    uint64_t st[32], W = 0;
    rc = orc_encode_wide(f64, n_alpha, ORC_L8, ORC_B8, N, s32, n_c, w, cap_w, &W, st);
    if (rc == ORC_OK) {
        uint64_t need = round4(4ull * N + W);
        if (need > cap) rc = ORC_ERR_SPACE;
        else {
            for (uint32_t j = 0; j < N; ++j) put_u32(out + 4 * j, (uint32_t)st[j]);
            for (uint64_t q = 0; q < W; ++q) out[4ull * N + q] = (uint8_t)w[q];
            for (uint64_t q = 4ull * N + W; q < need; ++q) out[q] = 0;
            *size = need;
        }
    }
    free(s32);
    free(w);
    return rc;
}

static int chunk_decode_bytes(const uint8_t *chunk, uint64_t size, const uint16_t *freq,
                              uint32_t n_alpha, uint32_t N, uint8_t *sym_out, uint64_t n_c)
{
    uint64_t f64[256];
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    int rc = prod_table(freq, n_alpha, f64);
    if (rc) return rc;
    if (size < 4ull * N || (size & 3)) return ORC_ERR_CORRUPT;
    uint64_t W = size - 4ull * N;
    uint64_t st[32], st_end[32], used = 0;
    for (uint32_t j = 0; j < N; ++j) st[j] = get_u32(chunk + 4 * j);
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (W ? W : 1));
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    if (!w || !s32) { free(w); free(s32); return ORC_ERR_ARG; }
    for (uint64_t q = 0; q < W; ++q) w[q] = chunk[4ull * N + q];
    rc = orc_decode_wide(f64, n_alpha, ORC_L8, ORC_B8, N, w, W, st, n_c, s32, &used, st_end);
    if (rc == ORC_OK) {
        /* every coder back at L, every digit read, then only zero padding */
        for (uint32_t j = 0; j < N; ++j)
            if (st_end[j] != ORC_L8) rc = ORC_ERR_CORRUPT;
        if (round4(4ull * N + used) != size) rc = ORC_ERR_CORRUPT;
        for (uint64_t q = used; q < W; ++q)
            if (w[q] != 0) rc = ORC_ERR_CORRUPT;
        for (uint64_t i = 0; i < n_c; ++i) sym_out[i] = (uint8_t)s32[i];
    }
    free(w);
    free(s32);
    return rc;
}

uint64_t orc_max_message_size_bytes(uint64_t n_sym, uint32_t N, uint32_t chunk_symbols)
{
    if (chunk_symbols == 0 || N == 0) return 0;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    return round16(32 + 4 * (n_chunks + 1)) + round16(n_chunks * (4ull * N + 3) + 2ull * n_sym);
}
int orc_encode_chunk_bytes(const uint8_t *sym, uint64_t n_c, const uint16_t *freq,
                           uint32_t n_alpha, uint32_t N, uint8_t *out, uint64_t cap, uint64_t *size)
{
    return chunk_encode_bytes(sym, n_c, freq, n_alpha, N, out, cap, size);
}
int orc_decode_chunk_bytes(const uint8_t *chunk, uint64_t size, const uint16_t *freq,
                           uint32_t n_alpha, uint32_t N, uint8_t *sym_out, uint64_t n_c)
{
    return chunk_decode_bytes(chunk, size, freq, n_alpha, N, sym_out, n_c);
}

/* Adaptive chunk (version 4): [u32 state[N]][u16 words], M = 2^12, L = b =
 * 2^16, binary symbols, per-coder contexts from p = M/2, rate 5. */
static int chunk_encode_adaptive(const uint8_t *sym, uint64_t n_c, uint32_t N, uint8_t *out,
                                 uint64_t cap, uint64_t *size)
{
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (n_c ? n_c : 1) * 2);
    if (!s32 || !w) { free(s32); free(w); return ORC_ERR_ARG; }
    for (uint64_t i = 0; i < n_c; ++i) s32[i] = sym[i];
    uint64_t st[32], W = 0;
    int rc = orc_encode_adaptive(1ull << ORC_LOG2_M, ORC_L, ORC_B, N, ORC_ADAPT_RATE, ORC_ADAPT_P0,
                                 s32, n_c, w, 2 * (n_c ? n_c : 1), &W, st);
    if (rc == ORC_OK) {
        uint64_t need = 4ull * N + 2ull * W;
        if (need > cap) rc = ORC_ERR_SPACE;
        else {
            for (uint32_t j = 0; j < N; ++j) put_u32(out + 4 * j, (uint32_t)st[j]);
            for (uint64_t k = 0; k < W; ++k) put_u16(out + 4ull * N + 2 * k, (uint32_t)w[k]);
            *size = need;
        }
    }
    free(s32);
    free(w);
    return rc;
}

static int chunk_decode_adaptive(const uint8_t *chunk, uint64_t size, uint32_t N,
                                 uint8_t *sym_out, uint64_t n_c)
{
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    if (size < 4ull * N || ((size - 4ull * N) & 1)) return ORC_ERR_CORRUPT;
    uint64_t W = (size - 4ull * N) / 2;
    uint64_t st[32], st_end[32], used = 0;
    for (uint32_t j = 0; j < N; ++j) st[j] = get_u32(chunk + 4 * j);
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (W ? W : 1));
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    if (!w || !s32) { free(w); free(s32); return ORC_ERR_ARG; }
    for (uint64_t k = 0; k < W; ++k) w[k] = get_u16(chunk + 4ull * N + 2 * k);
    int rc = orc_decode_adaptive(1ull << ORC_LOG2_M, ORC_L, ORC_B, N, ORC_ADAPT_RATE,
                                 ORC_ADAPT_P0, w, W, st, n_c, s32, &used, st_end);
    if (rc == ORC_OK) {
        for (uint32_t j = 0; j < N; ++j)
            if (st_end[j] != ORC_L) rc = ORC_ERR_CORRUPT;
        if (used != W) rc = ORC_ERR_CORRUPT;
        for (uint64_t i = 0; i < n_c; ++i) sym_out[i] = (uint8_t)s32[i];
    }
    free(w);
    free(s32);
    return rc;
}

int orc_encode_chunk_adaptive(const uint8_t *sym, uint64_t n_c, uint32_t N, uint8_t *out,
                              uint64_t cap, uint64_t *size)
{
    return chunk_encode_adaptive(sym, n_c, N, out, cap, size);
}
int orc_decode_chunk_adaptive(const uint8_t *chunk, uint64_t size, uint32_t N, uint8_t *sym_out,
                              uint64_t n_c)
{
    return chunk_decode_adaptive(chunk, size, N, sym_out, n_c);
}

/* Adaptive n-symbol chunk (version 6): [u32 state[N]][u16 words], M = 2^12,
 * L = b = 2^16, per-coder models from the uniform start, rate 5. */
static int chunk_encode_adaptive_n(const uint8_t *sym, uint64_t n_c, uint32_t n, uint32_t N,
                                   uint8_t *out, uint64_t cap, uint64_t *size)
{
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (n_c ? n_c : 1) * 2);
    if (!s32 || !w) { free(s32); free(w); return ORC_ERR_ARG; }
    for (uint64_t i = 0; i < n_c; ++i) s32[i] = sym[i];
    uint64_t st[32], W = 0;
    int rc = orc_encode_adaptive_n(1ull << ORC_LOG2_M, ORC_L, ORC_B, N, ORC_ADAPT_RATE, n, s32,
                                   n_c, w, 2 * (n_c ? n_c : 1), &W, st);
    if (rc == ORC_OK) {
        uint64_t need = 4ull * N + 2ull * W;
        if (need > cap) rc = ORC_ERR_SPACE;
        else {
            for (uint32_t j = 0; j < N; ++j) put_u32(out + 4 * j, (uint32_t)st[j]);
            for (uint64_t k = 0; k < W; ++k) put_u16(out + 4ull * N + 2 * k, (uint32_t)w[k]);
            *size = need;
        }
    }
    free(s32);
    free(w);
    return rc;
}

static int chunk_decode_adaptive_n(const uint8_t *chunk, uint64_t size, uint32_t n, uint32_t N,
                                   uint8_t *sym_out, uint64_t n_c)
{
    if (N == 0 || N > 32) return ORC_ERR_ARG;
    if (size < 4ull * N || ((size - 4ull * N) & 1)) return ORC_ERR_CORRUPT;
    uint64_t W = (size - 4ull * N) / 2;
    uint64_t st[32], st_end[32], used = 0;
    for (uint32_t j = 0; j < N; ++j) st[j] = get_u32(chunk + 4 * j);
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (W ? W : 1));
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_c ? n_c : 1));
    if (!w || !s32) { free(w); free(s32); return ORC_ERR_ARG; }
    for (uint64_t k = 0; k < W; ++k) w[k] = get_u16(chunk + 4ull * N + 2 * k);
    int rc = orc_decode_adaptive_n(1ull << ORC_LOG2_M, ORC_L, ORC_B, N, ORC_ADAPT_RATE, n, w, W,
                                   st, n_c, s32, &used, st_end);
    if (rc == ORC_OK) {
        for (uint32_t j = 0; j < N; ++j)
            if (st_end[j] != ORC_L) rc = ORC_ERR_CORRUPT;
        if (used != W) rc = ORC_ERR_CORRUPT;
        for (uint64_t i = 0; i < n_c; ++i) sym_out[i] = (uint8_t)s32[i];
    }
    free(w);
    free(s32);
    return rc;
}

int orc_encode_chunk_adaptive_n(const uint8_t *sym, uint64_t n_c, uint32_t n, uint32_t N,
                                uint8_t *out, uint64_t cap, uint64_t *size)
{
    return chunk_encode_adaptive_n(sym, n_c, n, N, out, cap, size);
}
int orc_decode_chunk_adaptive_n(const uint8_t *chunk, uint64_t size, uint32_t n, uint32_t N,
                                uint8_t *sym_out, uint64_t n_c)
{
    return chunk_decode_adaptive_n(chunk, size, n, N, sym_out, n_c);
}

/* Message = header + offsets + chunks; version 2 marks a bypass message,
 * version 3 a byte-wise one (bytes == 1), 4 adaptive binary contexts
 * (bytes == 2), 6 adaptive n-symbol models (bytes == 3, n = n_alpha). */
static int message_encode(const uint8_t *sym, const uint16_t *raw16, uint64_t n_sym,
                          const uint16_t *freq, const uint8_t *rawf, uint32_t n_alpha, uint32_t N,
                          uint32_t chunk_symbols, uint8_t *out, uint64_t cap, uint64_t *size,
                          int bytes)
{
    if (N == 0 || N > 32 || chunk_symbols == 0) return ORC_ERR_ARG;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    if (n_chunks > 0xFFFFFFFEull) return ORC_ERR_ARG;
    uint64_t data0 = round16(32 + 4 * (n_chunks + 1));
    if (cap < data0) return ORC_ERR_SPACE;
    memset(out, 0, data0);
    put_u32(out + 0, ORC_MAGIC);
    put_u32(out + 4, bytes == 3 ? ORC_VERSION_ADAPTIVE_N : bytes == 2 ? ORC_VERSION_ADAPTIVE
                     : bytes ? ORC_VERSION_BYTES : rawf ? ORC_VERSION_BYPASS : ORC_VERSION);
    put_u32(out + 8, N);
    uint32_t lm = ORC_LOG2_M;
    if (bytes == 0 && !rawf) {
        uint64_t f64[256];
        int rc0 = plain_table(freq, n_alpha, f64, 1, &lm);
        if (rc0) return rc0;
    }
    if (bytes == 3) {
        if (n_alpha < 2 || n_alpha > ORC_ADAPT_NMAX) return ORC_ERR_ARG;
        lm |= n_alpha << 16;
    }
    put_u32(out + 12, lm);
    put_u32(out + 16, (uint32_t)n_sym);
    put_u32(out + 20, (uint32_t)(n_sym >> 32));
    put_u32(out + 24, chunk_symbols);
    put_u32(out + 28, (uint32_t)n_chunks);
    uint64_t pos = 0;
    for (uint64_t c = 0; c < n_chunks; ++c) {
        uint64_t first = c * chunk_symbols;
        uint64_t n_c = n_sym - first < chunk_symbols ? n_sym - first : chunk_symbols;
        if (pos > 0xFFFFFFFFull) return ORC_ERR_ARG;
        put_u32(out + 32 + 4 * c, (uint32_t)pos);
        uint64_t sz = 0;
        if (data0 + pos > cap) return ORC_ERR_SPACE;
        int rc = bytes == 3 ? chunk_encode_adaptive_n(sym + first, n_c, n_alpha, N,
                                                      out + data0 + pos, cap - data0 - pos, &sz)
                 : bytes == 2 ? chunk_encode_adaptive(sym + first, n_c, N, out + data0 + pos,
                                                      cap - data0 - pos, &sz)
                 : bytes ? chunk_encode_bytes(sym + first, n_c, freq, n_alpha, N,
                                              out + data0 + pos, cap - data0 - pos, &sz)
                         : chunk_encode(sym + first, raw16 ? raw16 + first : NULL, n_c, freq,
                                        rawf, n_alpha, N, out + data0 + pos, cap - data0 - pos,
                                        &sz);
        if (rc) return rc;
        pos += sz;
    }
    if (pos > 0xFFFFFFFFull) return ORC_ERR_ARG;
    put_u32(out + 32 + 4 * n_chunks, (uint32_t)pos);
    uint64_t total = data0 + round16(pos);
    if (total > cap) return ORC_ERR_SPACE;
    memset(out + data0 + pos, 0, round16(pos) - pos);
    *size = total;
    return ORC_OK;
}

static int message_decode(const uint8_t *msg, uint64_t size, const uint16_t *freq,
                          const uint8_t *rawf, uint32_t n_alpha, uint32_t N,
                          uint32_t chunk_symbols, uint8_t *sym_out, uint16_t *raw_out,
                          uint64_t n_sym, int bytes)
{
    if (N == 0 || N > 32 || chunk_symbols == 0) return ORC_ERR_ARG;
    if (size < 48 || (size & 15)) return ORC_ERR_CORRUPT;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    uint64_t hdr_n = (uint64_t)get_u32(msg + 16) | ((uint64_t)get_u32(msg + 20) << 32);
    uint32_t version = bytes == 3 ? ORC_VERSION_ADAPTIVE_N : bytes == 2 ? ORC_VERSION_ADAPTIVE
                       : bytes ? ORC_VERSION_BYTES : rawf ? ORC_VERSION_BYPASS : ORC_VERSION;
    uint32_t lm = ORC_LOG2_M;
    if (bytes == 0 && !rawf) {
        uint64_t f64[256];
        int rc0 = plain_table(freq, n_alpha, f64, 1, &lm);
        if (rc0) return rc0;
    }
    if (bytes == 3) {
        if (n_alpha < 2 || n_alpha > ORC_ADAPT_NMAX) return ORC_ERR_ARG;
        lm |= n_alpha << 16;
    }
    if (get_u32(msg) != ORC_MAGIC || get_u32(msg + 4) != version ||
        get_u32(msg + 8) != N || get_u32(msg + 12) != lm || hdr_n != n_sym ||
        get_u32(msg + 24) != chunk_symbols || get_u32(msg + 28) != n_chunks)
        return ORC_ERR_CORRUPT;
    uint64_t data0 = round16(32 + 4 * (n_chunks + 1));
    if (data0 > size) return ORC_ERR_CORRUPT;
    uint64_t data_bytes = size - data0;
    if (get_u32(msg + 32) != 0) return ORC_ERR_CORRUPT;
    uint64_t end_all = get_u32(msg + 32 + 4 * n_chunks);
    if (round16(end_all) != data_bytes) return ORC_ERR_CORRUPT;
    int rc_all = ORC_OK;
    for (uint64_t c = 0; c < n_chunks; ++c) {
        uint64_t a = get_u32(msg + 32 + 4 * c), z = get_u32(msg + 32 + 4 * (c + 1));
        uint64_t first = c * chunk_symbols;
        uint64_t n_c = n_sym - first < chunk_symbols ? n_sym - first : chunk_symbols;
        if (z < a || z > end_all) return ORC_ERR_CORRUPT;
        int rc = bytes == 3 ? chunk_decode_adaptive_n(msg + data0 + a, z - a, n_alpha, N,
                                                      sym_out + first, n_c)
                 : bytes == 2 ? chunk_decode_adaptive(msg + data0 + a, z - a, N, sym_out + first,
                                                      n_c)
                 : bytes ? chunk_decode_bytes(msg + data0 + a, z - a, freq, n_alpha, N,
                                              sym_out + first, n_c)
                         : chunk_decode(msg + data0 + a, z - a, freq, rawf, n_alpha, N,
                                        sym_out + first, raw_out ? raw_out + first : NULL, n_c);
        if (rc && !rc_all) rc_all = rc;
    }
    return rc_all;
}

int orc_encode_message(const uint8_t *sym, uint64_t n_sym, const uint16_t *freq, uint32_t n_alpha,
                       uint32_t N, uint32_t chunk_symbols, uint8_t *out, uint64_t cap,
                       uint64_t *size)
{
    return message_encode(sym, NULL, n_sym, freq, NULL, n_alpha, N, chunk_symbols, out, cap, size,
                          0);
}
int orc_decode_message(const uint8_t *msg, uint64_t size, const uint16_t *freq, uint32_t n_alpha,
                       uint32_t N, uint32_t chunk_symbols, uint8_t *sym_out, uint64_t n_sym)
{
    return message_decode(msg, size, freq, NULL, n_alpha, N, chunk_symbols, sym_out, NULL, n_sym,
                          0);
}
int orc_encode_message_bypass(const uint8_t *sym, const uint16_t *raw16, uint64_t n_sym,
                              const uint16_t *freq, const uint8_t *rawf, uint32_t n_alpha,
                              uint32_t N, uint32_t chunk_symbols, uint8_t *out, uint64_t cap,
                              uint64_t *size)
{
    if (!rawf || !raw16) return ORC_ERR_ARG;
    return message_encode(sym, raw16, n_sym, freq, rawf, n_alpha, N, chunk_symbols, out, cap, size,
                          0);
}
int orc_decode_message_bypass(const uint8_t *msg, uint64_t size, const uint16_t *freq,
                              const uint8_t *rawf, uint32_t n_alpha, uint32_t N,
                              uint32_t chunk_symbols, uint8_t *sym_out, uint16_t *raw_out,
                              uint64_t n_sym)
{
    if (!rawf || !raw_out) return ORC_ERR_ARG;
    return message_decode(msg, size, freq, rawf, n_alpha, N, chunk_symbols, sym_out, raw_out,
                          n_sym, 0);
}
int orc_encode_message_adaptive(const uint8_t *sym, uint64_t n_sym, uint32_t N,
                                uint32_t chunk_symbols, uint8_t *out, uint64_t cap, uint64_t *size)
{
    return message_encode(sym, NULL, n_sym, NULL, NULL, 0, N, chunk_symbols, out, cap, size, 2);
}
int orc_decode_message_adaptive(const uint8_t *msg, uint64_t size, uint32_t N,
                                uint32_t chunk_symbols, uint8_t *sym_out, uint64_t n_sym)
{
    return message_decode(msg, size, NULL, NULL, 0, N, chunk_symbols, sym_out, NULL, n_sym, 2);
}
int orc_encode_message_adaptive_n(const uint8_t *sym, uint64_t n_sym, uint32_t n, uint32_t N,
                                  uint32_t chunk_symbols, uint8_t *out, uint64_t cap,
                                  uint64_t *size)
{
    return message_encode(sym, NULL, n_sym, NULL, NULL, n, N, chunk_symbols, out, cap, size, 3);
}
int orc_decode_message_adaptive_n(const uint8_t *msg, uint64_t size, uint32_t n, uint32_t N,
                                  uint32_t chunk_symbols, uint8_t *sym_out, uint64_t n_sym)
{
    return message_decode(msg, size, NULL, NULL, n, N, chunk_symbols, sym_out, NULL, n_sym, 3);
}
int orc_encode_message_bytes(const uint8_t *sym, uint64_t n_sym, const uint16_t *freq,
                             uint32_t n_alpha, uint32_t N, uint32_t chunk_symbols, uint8_t *out,
                             uint64_t cap, uint64_t *size)
{
    return message_encode(sym, NULL, n_sym, freq, NULL, n_alpha, N, chunk_symbols, out, cap, size,
                          1);
}
int orc_decode_message_bytes(const uint8_t *msg, uint64_t size, const uint16_t *freq,
                             uint32_t n_alpha, uint32_t N, uint32_t chunk_symbols,
                             uint8_t *sym_out, uint64_t n_sym)
{
    return message_decode(msg, size, freq, NULL, n_alpha, N, chunk_symbols, sym_out, NULL, n_sym,
                          1);
}

/* ---------------------------------------------------------------------- */
/* Quantizer: weights w_s -> integer f_s with sum f_s = M (not in the      */
/* paper; the paper only assumes a static model, Section 7).              */
/*   1. f_s = floor(w_s * M / W), W = sum w; raised to 1 where w_s > 0.    */
/*   2. While sum f < M: +1 to symbols with w_s > 0 in order of decreasing */
/*      remainder (w_s * M mod W), ties to the lower index, cycling.       */
/*   3. While sum f > M: -1 from the symbol with the largest f_s > 1,      */
/*      ties to the lower index.                                          */
/* ---------------------------------------------------------------------- */
int orc_quantize(const uint64_t *w, uint32_t n, uint32_t log2_M, uint16_t *f_out)
{
    if (n == 0 || n > 4096 || log2_M == 0 || log2_M > 15) return ORC_ERR_ARG;
    const u128 M = (u128)1 << log2_M;
    u128 W = 0;
    uint32_t nz = 0;
    for (uint32_t s = 0; s < n; ++s) { W += w[s]; nz += w[s] != 0; }
    if (W == 0 || W >> 64 || nz > (uint32_t)M) return ORC_ERR_ARG;
    u128 *rem = (u128 *)malloc(sizeof(u128) * n);
    uint32_t *fv = (uint32_t *)malloc(sizeof(uint32_t) * n);
    unsigned char *used = (unsigned char *)malloc(n);
    if (!rem || !fv || !used) { free(rem); free(fv); free(used); return ORC_ERR_ARG; }
    u128 sum = 0;
    for (uint32_t s = 0; s < n; ++s) {
        u128 num = (u128)w[s] * M;
        fv[s] = (uint32_t)(num / W);
        rem[s] = num % W;
        if (w[s] > 0 && fv[s] == 0) fv[s] = 1;
        sum += fv[s];
    }
    while (sum < M) {
        /* one pass in decreasing-remainder order, ties to the lower index */
        memset(used, 0, n);
        for (uint32_t k = 0; k < nz && sum < M; ++k) {
            int best = -1;
            for (uint32_t s = 0; s < n; ++s) {
                if (w[s] == 0 || used[s]) continue;
#if ORACLE_MUTANT == 8
                if (best < 0 || rem[s] >= rem[best]) best = (int)s;   /* ties to higher index */
#else
                if (best < 0 || rem[s] > rem[best]) best = (int)s;
#endif
            }
            used[best] = 1;
            fv[best] += 1;
            sum += 1;
        }
    }
    while (sum > M) {
        int best = -1;
        for (uint32_t s = 0; s < n; ++s)
            if (fv[s] > 1 && (best < 0 || fv[s] > fv[best])) best = (int)s;
        fv[best] -= 1;
        sum -= 1;
    }
    for (uint32_t s = 0; s < n; ++s) f_out[s] = (uint16_t)fv[s];
    free(rem);
    free(fv);
    free(used);
    return ORC_OK;
}
