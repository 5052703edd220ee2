/*
 * mux_oracle.c -- CPU ORACLE for Section 4 of F. Giesen, "Interleaved
 * entropy coders" (arXiv:1402.3392): interleaving arbitrary entropy coders.
 *
 * TEST INFRASTRUCTURE, built into the same library as rans_oracle.c and
 * under the same rules: only tests/, the smoke check in __graft_entry__.py
 * and the CPU legs of bench.py may load it; it shares nothing with the
 * product.
 *
 * Section 4's method.  Every coder writes its own buffer.  The single
 * output stream is made by running the decoders, in the order the receiver
 * will run them, in an instrumented form: whenever a decoder reads a word
 * from its coder's buffer, that word is also appended to the output.  The
 * receiver runs the plain decoders on the output and meets every word in
 * exactly the order it was appended, so no metadata is needed.
 *
 * The mux is generic over the coder family (struct family).  Two families
 * go through it here:
 *   - rANS, Algorithm 1 with one coder per buffer.  Its decoder first reads
 *     its state as base-b digits (least significant first), then decodes
 *     and renormalizes.  Muxing N such buffers, coder i mod N taking symbol
 *     i, gives exactly the interleaved stream of Section 3 (pinned).
 *   - a canonical prefix code.  Code lengths are at most 12; codes are
 *     assigned in order of (length, symbol), the rule of RFC 1951 Section
 *     3.2.2; bits go MSB first into 32-bit words.  The decoder reads one
 *     word whenever it holds fewer than 12 bits before decoding a symbol
 *     (so at most one word per symbol).  The encoder's flush pads the last
 *     word with zero bits and appends one zero word, which covers the
 *     decoder's read-ahead (it holds at most 43 bits); words the decoder
 *     never reads are not part of the output and must be padding.
 *
 * Also here:
 *   - the coroutine form of the mux (Section 4): encoders and instrumented
 *     decoder run together and the largest number of words buffered between
 *     them is measured.  A periodic flush cuts the message into segments of
 *     F symbols, each flushed and muxed on its own (decoders restart), which
 *     bounds the buffering at some cost in size;
 *   - optimal length-limited code lengths by package-merge (L. L. Larmore
 *     and D. S. Hirschberg, "A fast algorithm for optimal length-limited
 *     Huffman codes", J. ACM 37(3), 1990);
 *   - the version-5 container: the chunked container of rans_oracle.c with
 *     each chunk the prefix-code mux of its symbols (coder i mod N).
 *
 * ORACLE_MUTANT (see rans_oracle.c) plants mistakes 12 and 13 here.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

typedef unsigned __int128 u128;

enum { MX_OK = 0, MX_ERR_ARG = 1, MX_ERR_SYMBOL = 2, MX_ERR_SPACE = 3, MX_ERR_CORRUPT = 4 };

#define PFX_MAXLEN 12u   /* longest code; also the decoder's refill threshold */
#define PFX_ALPHA 256u

/* Single rANS coding steps from rans_oracle.c (Section 2's D). */
uint64_t orc_D(const uint64_t *f, uint32_t n_alpha, uint64_t x, uint32_t *s_out, int *ok);
int orc_encode(const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t N,
               const uint32_t *sym, uint64_t n_sym, uint64_t *words, uint64_t word_cap,
               uint64_t *n_words, uint64_t *states, uint64_t *trace_state, uint32_t *trace_lane,
               uint64_t trace_cap, uint64_t *n_trace, uint32_t *max_iters);

/* ---------------------------------------------------------------------- */
/* Reading words: instrumented (from coder j's own buffer, copied to the   */
/* output) or receiving (from the one stream).                             */
/* ---------------------------------------------------------------------- */

typedef struct {
    /* instrumented mode: own != NULL */
    uint64_t *const *own;
    const uint64_t *own_len;
    uint64_t *own_pos;
    uint64_t *out;
    uint64_t out_cap, out_len;
    /* receiving mode */
    const uint64_t *in;
    uint64_t in_len, in_pos;
} reader;

static int read_word(reader *r, uint32_t j, uint64_t *w)
{
    if (r->own) {
        if (r->own_pos[j] >= r->own_len[j]) return MX_ERR_CORRUPT;
        *w = r->own[j][r->own_pos[j]++];
        if (r->out_len >= r->out_cap) return MX_ERR_SPACE;
        r->out[r->out_len++] = *w;   /* the instrumentation: copy what was read */
        return MX_OK;
    }
    if (r->in_pos >= r->in_len) return MX_ERR_CORRUPT;
    *w = r->in[r->in_pos++];
    return MX_OK;
}

/* A coder family: its decoder's start, one symbol, and end check. */
typedef struct {
    size_t state_words;   /* u64 words of decoder state per coder */
    int (*start)(const void *param, uint64_t *st, uint32_t j, reader *r);
    int (*step)(const void *param, uint64_t *st, uint32_t j, reader *r, uint32_t *sym);
    int (*end)(const void *param, const uint64_t *st);
} family;

static uint32_t lane_at(const uint32_t *lane_of, uint64_t i, uint32_t N)
{
    return lane_of ? lane_of[i] : (uint32_t)(i % N);
}

/* Run the N decoders in the receiver's order: every coder starts (coder 0
 * first), symbol i is decoded by coder lane_of[i] (i mod N if NULL), then
 * every coder's end check. */
static int run_decoders(const family *fam, const void *param, uint32_t N,
                        const uint32_t *lane_of, uint64_t n_sym, reader *r, uint32_t *sym_out)
{
    uint64_t *st = (uint64_t *)calloc((size_t)N * fam->state_words, sizeof(uint64_t));
    if (!st) return MX_ERR_ARG;
    int rc = MX_OK;
    for (uint32_t j = 0; j < N && !rc; ++j) rc = fam->start(param, st + j * fam->state_words, j, r);
    for (uint64_t i = 0; i < n_sym && !rc; ++i) {
        uint32_t j = lane_at(lane_of, i, N), s = 0;
        if (j >= N) { rc = MX_ERR_ARG; break; }
        rc = fam->step(param, st + j * fam->state_words, j, r, &s);
        if (!rc && sym_out) sym_out[i] = s;
    }
    for (uint32_t j = 0; j < N && !rc; ++j) rc = fam->end(param, st + j * fam->state_words);
    free(st);
    return rc;
}

/* Section 4: the instrumented decoders copy every word they read from the
 * coders' buffers own[j] into out, in read order.  Words left unread in a
 * coder's buffer must be zero (flush padding). */
static int mux(const family *fam, const void *param, uint32_t N, const uint32_t *lane_of,
               uint64_t n_sym, uint64_t *const *own, const uint64_t *own_len, uint64_t *out,
               uint64_t cap, uint64_t *n_out)
{
    uint64_t *pos = (uint64_t *)calloc(N, sizeof(uint64_t));
    if (!pos) return MX_ERR_ARG;
    reader r;
    memset(&r, 0, sizeof r);
    r.own = own;
    r.own_len = own_len;
    r.own_pos = pos;
    r.out = out;
    r.out_cap = cap;
    int rc = MX_OK;
#if ORACLE_MUTANT == 12
    /* planted mistake: the buffers concatenated, coder by coder */
    (void)fam; (void)param; (void)lane_of; (void)n_sym;
    for (uint32_t j = 0; j < N && !rc; ++j)
        for (uint64_t k = 0; k < own_len[j]; ++k) {
            if (r.out_len >= cap) { rc = MX_ERR_SPACE; break; }
            out[r.out_len++] = own[j][k];
        }
#else
    rc = run_decoders(fam, param, N, lane_of, n_sym, &r, NULL);
    for (uint32_t j = 0; j < N && !rc; ++j)
        for (uint64_t k = pos[j]; k < own_len[j]; ++k)
            if (own[j][k] != 0) rc = MX_ERR_CORRUPT;
#endif
    free(pos);
    if (!rc) *n_out = r.out_len;
    return rc;
}

/* The receiver: the plain decoders on the one stream; every word must be
 * read. */
static int demux(const family *fam, const void *param, uint32_t N, const uint32_t *lane_of,
                 uint64_t n_sym, const uint64_t *in, uint64_t n_in, uint32_t *sym_out)
{
    reader r;
    memset(&r, 0, sizeof r);
    r.in = in;
    r.in_len = n_in;
    int rc = run_decoders(fam, param, N, lane_of, n_sym, &r, sym_out);
    if (!rc && r.in_pos != n_in) rc = MX_ERR_CORRUPT;
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Family 1: rANS, Algorithm 1 with one coder per buffer.                 */
/* ---------------------------------------------------------------------- */

typedef struct {
    const uint64_t *f;
    uint32_t n_alpha;
    uint64_t L, b;
    uint32_t state_digits;   /* base-b digits of a state in [L, bL) */
} rans_param;

static int rans_start(const void *pv, uint64_t *st, uint32_t j, reader *r)
{
    const rans_param *p = (const rans_param *)pv;
    u128 x = 0, scale = 1;
    for (uint32_t k = 0; k < p->state_digits; ++k) {
        uint64_t w;
        int rc = read_word(r, j, &w);
        if (rc) return rc;
        x += (u128)w * scale;
        scale *= p->b;
    }
    if (x < p->L || x >= (u128)p->L * p->b) return MX_ERR_CORRUPT;
    st[0] = (uint64_t)x;
    return MX_OK;
}

static int rans_step(const void *pv, uint64_t *st, uint32_t j, reader *r, uint32_t *sym)
{
    const rans_param *p = (const rans_param *)pv;
    int ok = 0;
    uint64_t x = orc_D(p->f, p->n_alpha, st[0], sym, &ok);   /* Algorithm 1, Decode */
    if (!ok) return MX_ERR_ARG;
    while (x < p->L) {
        uint64_t w;
        int rc = read_word(r, j, &w);
        if (rc) return rc;
        x = x * p->b + w;
    }
    st[0] = x;
    return MX_OK;
}

static int rans_end(const void *pv, const uint64_t *st)
{
    return st[0] == ((const rans_param *)pv)->L ? MX_OK : MX_ERR_CORRUPT;
}

static const family RANS_FAMILY = {1, rans_start, rans_step, rans_end};

static int rans_param_init(rans_param *p, const uint64_t *f, uint32_t n_alpha, uint64_t L,
                           uint64_t b)
{
    if (L == 0 || b < 2 || n_alpha == 0) return MX_ERR_ARG;
    p->f = f;
    p->n_alpha = n_alpha;
    p->L = L;
    p->b = b;
    p->state_digits = 0;
    u128 top = (u128)L * b, span = 1;
    while (span < top) { span *= b; ++p->state_digits; }
    return MX_OK;
}

/* Coder j of N encodes its own symbols (j, j+N, ...) alone with Algorithm 1;
 * its buffer is its final state as digits, least significant first, then
 * its words in decode order.  The mux of the N buffers is the output. */
int orc_mux_rans(const uint32_t *sym, uint64_t n_sym, uint32_t N, const uint64_t *f,
                 uint32_t n_alpha, uint64_t L, uint64_t b, uint64_t *out, uint64_t cap,
                 uint64_t *n_out)
{
    rans_param p;
    if (N == 0 || rans_param_init(&p, f, n_alpha, L, b)) return MX_ERR_ARG;
    uint64_t **own = (uint64_t **)calloc(N, sizeof(uint64_t *));
    uint64_t *len = (uint64_t *)calloc(N, sizeof(uint64_t));
    uint32_t *sub = (uint32_t *)malloc(sizeof(uint32_t) * (n_sym / N + 1));
    int rc = (own && len && sub) ? MX_OK : MX_ERR_ARG;
    for (uint32_t j = 0; j < N && !rc; ++j) {
        uint64_t m = 0;
        for (uint64_t i = j; i < n_sym; i += N) sub[m++] = sym[i];
        uint64_t wcap = m * 64 + 8, W = 0, state = 0;
        own[j] = (uint64_t *)malloc(sizeof(uint64_t) * (wcap + p.state_digits));
        if (!own[j]) { rc = MX_ERR_ARG; break; }
        rc = orc_encode(f, n_alpha, L, b, 1, sub, m, own[j] + p.state_digits, wcap, &W, &state,
                        NULL, NULL, 0, NULL, NULL);
        if (rc) break;
        u128 x = state;
        for (uint32_t k = 0; k < p.state_digits; ++k) {
            own[j][k] = (uint64_t)(x % b);
            x /= b;
        }
        len[j] = p.state_digits + W;
    }
    if (!rc) rc = mux(&RANS_FAMILY, &p, N, NULL, n_sym, own, len, out, cap, n_out);
    for (uint32_t j = 0; own && j < N; ++j) free(own[j]);
    free(own);
    free(len);
    free(sub);
    return rc;
}

int orc_demux_rans(const uint64_t *in, uint64_t n_in, uint64_t n_sym, uint32_t N,
                   const uint64_t *f, uint32_t n_alpha, uint64_t L, uint64_t b, uint32_t *sym_out)
{
    rans_param p;
    if (N == 0 || rans_param_init(&p, f, n_alpha, L, b)) return MX_ERR_ARG;
    return demux(&RANS_FAMILY, &p, N, NULL, n_sym, in, n_in, sym_out);
}

/* ---------------------------------------------------------------------- */
/* Family 2: a canonical prefix code.                                     */
/* ---------------------------------------------------------------------- */

typedef struct {
    uint32_t n_alpha;
    uint8_t len[PFX_ALPHA];
    uint32_t code[PFX_ALPHA];
} pfx_param;

/* Canonical codes from code lengths (RFC 1951 Section 3.2.2): count the
 * codes of each length; the first code of length l is (first code of length
 * l-1 + count of length l-1) shifted left by one; codes of one length go to
 * the symbols in increasing order.  Length 0 = unused symbol.  The lengths
 * must satisfy Kraft's inequality sum 2^-l <= 1. */
int orc_prefix_codes(const uint8_t *len, uint32_t n_alpha, uint32_t *code)
{
    if (n_alpha == 0 || n_alpha > PFX_ALPHA) return MX_ERR_ARG;
    uint32_t count[PFX_MAXLEN + 1] = {0}, next[PFX_MAXLEN + 2] = {0};
    uint64_t kraft = 0;   /* in units of 2^-PFX_MAXLEN */
    for (uint32_t s = 0; s < n_alpha; ++s) {
        if (len[s] > PFX_MAXLEN) return MX_ERR_ARG;
        if (len[s]) {
            ++count[len[s]];
            kraft += 1ull << (PFX_MAXLEN - len[s]);
        }
    }
    if (kraft == 0 || kraft > (1ull << PFX_MAXLEN)) return MX_ERR_ARG;
    uint32_t c = 0;
    for (uint32_t l = 1; l <= PFX_MAXLEN; ++l) {
        c = (c + count[l - 1]) << 1;
        next[l] = c;
    }
#if ORACLE_MUTANT == 13
    /* planted mistake: codes of one length handed out in decreasing symbol order */
    for (uint32_t s = n_alpha; s-- > 0;)
#else
    for (uint32_t s = 0; s < n_alpha; ++s)
#endif
        code[s] = len[s] ? next[len[s]]++ : 0u;
    return MX_OK;
}

static int pfx_param_init(pfx_param *p, const uint8_t *len, uint32_t n_alpha)
{
    memset(p, 0, sizeof *p);
    if (n_alpha == 0 || n_alpha > PFX_ALPHA) return MX_ERR_ARG;
    p->n_alpha = n_alpha;
    memcpy(p->len, len, n_alpha);
    return orc_prefix_codes(len, n_alpha, p->code);
}

/* Decoder state: st[0] = bit buffer, bits left-aligned; st[1] = bit count. */
static int pfx_start(const void *pv, uint64_t *st, uint32_t j, reader *r)
{
    (void)pv; (void)j; (void)r;
    st[0] = 0;
    st[1] = 0;
    return MX_OK;
}

static int pfx_step(const void *pv, uint64_t *st, uint32_t j, reader *r, uint32_t *sym)
{
    const pfx_param *p = (const pfx_param *)pv;
    uint64_t bb = st[0], nb = st[1];
    if (nb < PFX_MAXLEN) {   /* refill: one 32-bit word */
        uint64_t w;
        int rc = read_word(r, j, &w);
        if (rc) return rc;
        if (w >> 32) return MX_ERR_CORRUPT;
        bb |= w << (32 - nb);
        nb += 32;
    }
    /* The one symbol whose code is a prefix of the buffered bits (linear
     * search on purpose). */
    for (uint32_t s = 0; s < p->n_alpha; ++s) {
        uint32_t l = p->len[s];
        if (l && l <= nb && (bb >> (64 - l)) == p->code[s]) {
            *sym = s;
            st[0] = bb << l;
            st[1] = nb - l;
            return MX_OK;
        }
    }
    return MX_ERR_CORRUPT;
}

static int pfx_end(const void *pv, const uint64_t *st)
{
    (void)pv;
    return st[0] == 0 ? MX_OK : MX_ERR_CORRUPT;   /* what is left is zero padding */
}

static const family PFX_FAMILY = {2, pfx_start, pfx_step, pfx_end};

/* One coder's own buffer: codes of its symbols, MSB first, in 32-bit words;
 * flush: zero bits to the word's end, then one zero word. */
static int pfx_encode_own(const pfx_param *p, const uint8_t *sym, const uint32_t *lane_of,
                          uint64_t n_sym, uint32_t N, uint32_t j, uint64_t *words,
                          uint64_t cap, uint64_t *n_words)
{
    uint64_t acc = 0, W = 0;
    uint32_t na = 0;
    for (uint64_t i = 0; i < n_sym; ++i) {
        if (lane_at(lane_of, i, N) != j) continue;
        uint32_t s = sym[i];
        if (s >= p->n_alpha || p->len[s] == 0) return MX_ERR_SYMBOL;
        acc = (acc << p->len[s]) | p->code[s];
        na += p->len[s];
        if (na >= 32) {
            if (W >= cap) return MX_ERR_SPACE;
            words[W++] = (acc >> (na - 32)) & 0xFFFFFFFFull;
            na -= 32;
            acc &= (1ull << na) - 1;
        }
    }
    if (W + 2 > cap) return MX_ERR_SPACE;
    if (na) words[W++] = (acc << (32 - na)) & 0xFFFFFFFFull;
    words[W++] = 0;
    *n_words = W;
    return MX_OK;
}

static int pfx_mux_u64(const pfx_param *p, const uint8_t *sym, uint64_t n_sym, uint32_t N,
                       const uint32_t *lane_of, uint64_t *out, uint64_t cap, uint64_t *n_out)
{
    uint64_t **own = (uint64_t **)calloc(N, sizeof(uint64_t *));
    uint64_t *len = (uint64_t *)calloc(N, sizeof(uint64_t));
    int rc = (own && len) ? MX_OK : MX_ERR_ARG;
    for (uint32_t j = 0; j < N && !rc; ++j) {
        uint64_t wcap = n_sym * PFX_MAXLEN / 32 + 4;
        own[j] = (uint64_t *)malloc(sizeof(uint64_t) * wcap);
        if (!own[j]) { rc = MX_ERR_ARG; break; }
        rc = pfx_encode_own(p, sym, lane_of, n_sym, N, j, own[j], wcap, &len[j]);
    }
    if (!rc) rc = mux(&PFX_FAMILY, p, N, lane_of, n_sym, own, len, out, cap, n_out);
    for (uint32_t j = 0; own && j < N; ++j) free(own[j]);
    free(own);
    free(len);
    return rc;
}

/* Prefix-code mux: coder lane_of[i] (i mod N if NULL) takes symbol i. */
int orc_mux_prefix(const uint8_t *sym, uint64_t n_sym, uint32_t N, const uint32_t *lane_of,
                   const uint8_t *len, uint32_t n_alpha, uint32_t *out, uint64_t cap,
                   uint64_t *n_out)
{
    pfx_param p;
    if (N == 0 || pfx_param_init(&p, len, n_alpha)) return MX_ERR_ARG;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (cap ? cap : 1));
    if (!tmp) return MX_ERR_ARG;
    uint64_t n = 0;
    int rc = pfx_mux_u64(&p, sym, n_sym, N, lane_of, tmp, cap, &n);
    if (!rc) {
        for (uint64_t k = 0; k < n; ++k) out[k] = (uint32_t)tmp[k];
        *n_out = n;
    }
    free(tmp);
    return rc;
}

int orc_demux_prefix(const uint32_t *in, uint64_t n_in, uint64_t n_sym, uint32_t N,
                     const uint32_t *lane_of, const uint8_t *len, uint32_t n_alpha,
                     uint8_t *sym_out)
{
    pfx_param p;
    if (N == 0 || pfx_param_init(&p, len, n_alpha)) return MX_ERR_ARG;
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (n_in ? n_in : 1));
    uint32_t *s32 = (uint32_t *)malloc(sizeof(uint32_t) * (n_sym ? n_sym : 1));
    int rc = (w && s32) ? MX_OK : MX_ERR_ARG;
    for (uint64_t k = 0; k < n_in && !rc; ++k) w[k] = in[k];
    if (!rc) rc = demux(&PFX_FAMILY, &p, N, lane_of, n_sym, w, n_in, s32);
    if (!rc)
        for (uint64_t i = 0; i < n_sym; ++i) sym_out[i] = (uint8_t)s32[i];
    free(w);
    free(s32);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* The coroutine form (Section 4) and periodic flushing.                  */
/* ---------------------------------------------------------------------- */

/* Encoders and the instrumented decoder run together on the prefix family:
 * the decoder decodes as far as the words it needs exist; when it waits,
 * the encoders take the next symbol (or, at the end of a segment, flush).
 * Buffered = words the encoders have finished that the mux has not taken
 * yet; *peak is its maximum.  segment = F > 0: every F symbols all coders
 * flush and the decoders restart (segments muxed one after another);
 * segment = 0: one segment.  *total = words in the output. */
int orc_mux_prefix_peak(const uint8_t *sym, uint64_t n_sym, uint32_t N, const uint32_t *lane_of,
                        const uint8_t *len, uint32_t n_alpha, uint64_t segment, uint64_t *peak,
                        uint64_t *total)
{
    pfx_param p;
    if (N == 0 || pfx_param_init(&p, len, n_alpha)) return MX_ERR_ARG;
    uint64_t seg = segment ? segment : (n_sym ? n_sym : 1);
    /* per coder: encoder bits (acc, na), words produced (kept), decoder
     * bits (bb, nb) and words taken */
    uint64_t *acc = (uint64_t *)calloc(N, 8), *na = (uint64_t *)calloc(N, 8);
    uint64_t *bb = (uint64_t *)calloc(N, 8), *nb = (uint64_t *)calloc(N, 8);
    uint64_t *made = (uint64_t *)calloc(N, 8), *taken = (uint64_t *)calloc(N, 8);
    uint64_t **words = (uint64_t **)calloc(N, sizeof(uint64_t *));
    uint64_t wcap = n_sym * PFX_MAXLEN / 32 + 4;
    int rc = (acc && na && bb && nb && made && taken && words) ? MX_OK : MX_ERR_ARG;
    for (uint32_t j = 0; j < N && !rc; ++j)
        if (!(words[j] = (uint64_t *)malloc(8 * wcap))) rc = MX_ERR_ARG;
    uint64_t buffered = 0, pk = 0, out = 0;
    for (uint64_t a = 0; a < n_sym && !rc; a += seg) {
        uint64_t z = a + seg < n_sym ? a + seg : n_sym, e = a, d = a;
        int flushed = 0;
        for (uint32_t j = 0; j < N; ++j) acc[j] = na[j] = bb[j] = nb[j] = made[j] = taken[j] = 0;
        while (d < z && !rc) {
            uint32_t j = lane_at(lane_of, d, N);
            if (j >= N) { rc = MX_ERR_ARG; break; }
            if (nb[j] < PFX_MAXLEN && taken[j] >= made[j]) {
                /* the decoder waits: the encoders move on */
                if (e < z) {
                    uint32_t k = lane_at(lane_of, e, N), s = sym[e];
                    if (k >= N) { rc = MX_ERR_ARG; break; }
                    if (s >= p.n_alpha || p.len[s] == 0) { rc = MX_ERR_SYMBOL; break; }
                    acc[k] = (acc[k] << p.len[s]) | p.code[s];
                    na[k] += p.len[s];
                    if (na[k] >= 32) {
                        words[k][made[k]++] = (acc[k] >> (na[k] - 32)) & 0xFFFFFFFFull;
                        na[k] -= 32;
                        acc[k] &= (1ull << na[k]) - 1;
                        ++buffered;
                    }
                    ++e;
                } else if (!flushed) {
                    for (uint32_t k = 0; k < N; ++k) {
                        if (na[k]) {
                            words[k][made[k]++] = (acc[k] << (32 - na[k])) & 0xFFFFFFFFull;
                            ++buffered;
                        }
                        words[k][made[k]++] = 0;
                        ++buffered;
                    }
                    flushed = 1;
                } else {
                    rc = MX_ERR_CORRUPT;   /* nothing left to wait for */
                }
                if (buffered > pk) pk = buffered;
                continue;
            }
            if (nb[j] < PFX_MAXLEN) {
                bb[j] |= words[j][taken[j]++] << (32 - nb[j]);
                nb[j] += 32;
                --buffered;
                ++out;
            }
            uint32_t s = 0;
            for (s = 0; s < p.n_alpha; ++s)
                if (p.len[s] && (bb[j] >> (64 - p.len[s])) == p.code[s]) break;
            if (s == p.n_alpha || s != sym[d]) { rc = MX_ERR_CORRUPT; break; }
            bb[j] <<= p.len[s];
            nb[j] -= p.len[s];
            ++d;
        }
        /* words the decoders never take (flush padding) are dropped; the
         * mux's words do not depend on when the flush came */
        for (uint32_t j = 0; j < N && !rc; ++j) buffered -= made[j] - taken[j];
    }
    for (uint32_t j = 0; words && j < N; ++j) free(words[j]);
    free(words); free(acc); free(na); free(bb); free(nb); free(made); free(taken);
    if (!rc) {
        *peak = pk;
        *total = out;
    }
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Optimal length-limited code lengths: package-merge.                    */
/* ---------------------------------------------------------------------- */

/*
 * The coin-collector form.  Every used symbol (weight > 0) is a coin of
 * each denomination 2^-1 .. 2^-max_len whose value is its weight; the
 * lengths of an optimal code with lengths <= max_len are the numbers of
 * each symbol's coins in a cheapest set of total denomination n - 1 (n used
 * symbols).  The lists, from the smallest denomination up:
 *   list_max = the used symbols sorted by (weight, index);
 *   list_d   = the used symbols merged with the packages of list_{d+1}
 *              (items 0+1, 2+3, ...: weight the sum, an odd last item
 *              dropped), by weight, a symbol before a package of equal
 *              weight, packages in the order they were made;
 * and the first 2(n-1) items of list_1 are taken.  Each item carries how
 * many coins of every symbol it holds.  One used symbol gets length 1.
 */
int orc_prefix_lengths(const uint64_t *w, uint32_t n_alpha, uint32_t max_len, uint8_t *len_out)
{
    if (n_alpha == 0 || n_alpha > PFX_ALPHA || max_len == 0 || max_len > 16) return MX_ERR_ARG;
    uint32_t used[PFX_ALPHA], n = 0;
    for (uint32_t s = 0; s < n_alpha; ++s) {
        len_out[s] = 0;
        if (w[s]) used[n++] = s;
    }
    if (n == 0 || (max_len < 32 && (uint64_t)n > (1ull << max_len))) return MX_ERR_ARG;
    if (n == 1) {
        len_out[used[0]] = 1;
        return MX_OK;
    }
    /* used symbols sorted by (weight, index): insertion sort */
    for (uint32_t a = 1; a < n; ++a) {
        uint32_t v = used[a], k = a;
        while (k > 0 && (w[used[k - 1]] > w[v] || (w[used[k - 1]] == w[v] && used[k - 1] > v))) {
            used[k] = used[k - 1];
            --k;
        }
        used[k] = v;
    }
    uint32_t cap = 2 * n;
    u128 *pw = (u128 *)malloc(sizeof(u128) * cap), *cw = (u128 *)malloc(sizeof(u128) * cap);
    uint16_t *pc = (uint16_t *)calloc((size_t)cap * n, 2), *cc = (uint16_t *)calloc((size_t)cap * n, 2);
    if (!pw || !cw || !pc || !cc) { free(pw); free(cw); free(pc); free(cc); return MX_ERR_ARG; }
    uint32_t pn = 0;   /* items in the previous (finer) list */
    for (uint32_t d = max_len; d >= 1; --d) {
        uint32_t cn = 0, li = 0, pk = 0, n_pk = pn / 2;
        while (li < n || pk < n_pk) {
            u128 lw = li < n ? (u128)w[used[li]] : 0;
            u128 kw = pk < n_pk ? pw[2 * pk] + pw[2 * pk + 1] : 0;
            uint16_t *dst = cc + (size_t)cn * n;
            if (li < n && (pk >= n_pk || lw <= kw)) {
                memset(dst, 0, 2 * n);
                dst[li] = 1;
                cw[cn++] = lw;
                ++li;
            } else {
                const uint16_t *x = pc + (size_t)(2 * pk) * n, *y = x + n;
                for (uint32_t k = 0; k < n; ++k) dst[k] = (uint16_t)(x[k] + y[k]);
                cw[cn++] = kw;
                ++pk;
            }
        }
        u128 *tw = pw; pw = cw; cw = tw;
        uint16_t *tc = pc; pc = cc; cc = tc;
        pn = cn;
    }
    uint32_t take = 2 * (n - 1);
    for (uint32_t i = 0; i < take && i < pn; ++i)
        for (uint32_t k = 0; k < n; ++k) len_out[used[k]] = (uint8_t)(len_out[used[k]] + pc[(size_t)i * n + k]);
    free(pw); free(cw); free(pc); free(cc);
    return MX_OK;
}

/* ---------------------------------------------------------------------- */
/* Version-5 container: chunks of the prefix-code mux.                    */
/*   header as in rans_oracle.c with version 5 and 12 (the longest code)  */
/*   in the log2_M field; chunk c = the mux (coder i mod N takes symbol i */
/*   of the chunk) of its symbols as u32 little-endian words.             */
/* ---------------------------------------------------------------------- */

#define MX_MAGIC 0x534E4152u
#define MX_VERSION_PREFIX 5u

static void wr32(uint8_t *p, uint32_t v)
{
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static uint32_t rd32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t rnd16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

/* Worst case: per chunk, 12 bits a symbol plus a padded word and the
 * read-ahead word for each coder. */
uint64_t orc_max_message_size_prefix(uint64_t n_sym, uint32_t N, uint32_t chunk_symbols)
{
    if (N == 0 || chunk_symbols == 0) return 0;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    return rnd16(32 + 4 * (n_chunks + 1)) +
           rnd16(4 * ((n_sym * PFX_MAXLEN + 31) / 32 + n_chunks * (uint64_t)(2 * N + 1)));
}

int orc_encode_chunk_prefix(const uint8_t *sym, uint64_t n_c, const uint8_t *len,
                            uint32_t n_alpha, uint32_t N, uint8_t *out, uint64_t cap,
                            uint64_t *size)
{
    pfx_param p;
    if (N == 0 || N > 32 || pfx_param_init(&p, len, n_alpha)) return MX_ERR_ARG;
    uint64_t wcap = (n_c * PFX_MAXLEN + 31) / 32 + 2 * N + 1;
    uint64_t *w = (uint64_t *)malloc(8 * wcap), n = 0;
    if (!w) return MX_ERR_ARG;
    int rc = pfx_mux_u64(&p, sym, n_c, N, NULL, w, wcap, &n);
    if (!rc && 4 * n > cap) rc = MX_ERR_SPACE;
    if (!rc) {
        for (uint64_t k = 0; k < n; ++k) wr32(out + 4 * k, (uint32_t)w[k]);
        *size = 4 * n;
    }
    free(w);
    return rc;
}

int orc_decode_chunk_prefix(const uint8_t *chunk, uint64_t size, const uint8_t *len,
                            uint32_t n_alpha, uint32_t N, uint8_t *sym_out, uint64_t n_c)
{
    pfx_param p;
    if (N == 0 || N > 32 || pfx_param_init(&p, len, n_alpha)) return MX_ERR_ARG;
    if (size & 3) return MX_ERR_CORRUPT;
    uint64_t n = size / 4;
    uint64_t *w = (uint64_t *)malloc(8 * (n ? n : 1));
    uint32_t *s32 = (uint32_t *)malloc(4 * (n_c ? n_c : 1));
    int rc = (w && s32) ? MX_OK : MX_ERR_ARG;
    for (uint64_t k = 0; k < n && !rc; ++k) w[k] = rd32(chunk + 4 * k);
    if (!rc) rc = demux(&PFX_FAMILY, &p, N, NULL, n_c, w, n, s32);
    if (!rc)
        for (uint64_t i = 0; i < n_c; ++i) sym_out[i] = (uint8_t)s32[i];
    free(w);
    free(s32);
    return rc;
}

int orc_encode_message_prefix(const uint8_t *sym, uint64_t n_sym, const uint8_t *len,
                              uint32_t n_alpha, uint32_t N, uint32_t chunk_symbols, uint8_t *out,
                              uint64_t cap, uint64_t *size)
{
    if (N == 0 || N > 32 || chunk_symbols == 0) return MX_ERR_ARG;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    if (n_chunks > 0xFFFFFFFEull) return MX_ERR_ARG;
    uint64_t data0 = rnd16(32 + 4 * (n_chunks + 1));
    if (cap < data0) return MX_ERR_SPACE;
    memset(out, 0, data0);
    wr32(out + 0, MX_MAGIC);
    wr32(out + 4, MX_VERSION_PREFIX);
    wr32(out + 8, N);
    wr32(out + 12, PFX_MAXLEN);
    wr32(out + 16, (uint32_t)n_sym);
    wr32(out + 20, (uint32_t)(n_sym >> 32));
    wr32(out + 24, chunk_symbols);
    wr32(out + 28, (uint32_t)n_chunks);
    uint64_t pos = 0;
    for (uint64_t c = 0; c < n_chunks; ++c) {
        uint64_t first = c * chunk_symbols;
        uint64_t n_c = n_sym - first < chunk_symbols ? n_sym - first : chunk_symbols;
        if (pos > 0xFFFFFFFFull) return MX_ERR_ARG;
        wr32(out + 32 + 4 * c, (uint32_t)pos);
        uint64_t sz = 0;
        if (data0 + pos > cap) return MX_ERR_SPACE;
        int rc = orc_encode_chunk_prefix(sym + first, n_c, len, n_alpha, N, out + data0 + pos,
                                         cap - data0 - pos, &sz);
        if (rc) return rc;
        pos += sz;
    }
    if (pos > 0xFFFFFFFFull) return MX_ERR_ARG;
    wr32(out + 32 + 4 * n_chunks, (uint32_t)pos);
    uint64_t total = data0 + rnd16(pos);
    if (total > cap) return MX_ERR_SPACE;
    memset(out + data0 + pos, 0, rnd16(pos) - pos);
    *size = total;
    return MX_OK;
}

int orc_decode_message_prefix(const uint8_t *msg, uint64_t size, const uint8_t *len,
                              uint32_t n_alpha, uint32_t N, uint32_t chunk_symbols,
                              uint8_t *sym_out, uint64_t n_sym)
{
    if (N == 0 || N > 32 || chunk_symbols == 0) return MX_ERR_ARG;
    if (size < 48 || (size & 15)) return MX_ERR_CORRUPT;
    uint64_t n_chunks = (n_sym + chunk_symbols - 1) / chunk_symbols;
    uint64_t hdr_n = (uint64_t)rd32(msg + 16) | ((uint64_t)rd32(msg + 20) << 32);
    if (rd32(msg) != MX_MAGIC || rd32(msg + 4) != MX_VERSION_PREFIX || rd32(msg + 8) != N ||
        rd32(msg + 12) != PFX_MAXLEN || hdr_n != n_sym || rd32(msg + 24) != chunk_symbols ||
        rd32(msg + 28) != n_chunks)
        return MX_ERR_CORRUPT;
    uint64_t data0 = rnd16(32 + 4 * (n_chunks + 1));
    if (data0 > size) return MX_ERR_CORRUPT;
    if (rd32(msg + 32) != 0) return MX_ERR_CORRUPT;
    uint64_t end_all = rd32(msg + 32 + 4 * n_chunks);
    if (rnd16(end_all) != size - data0) return MX_ERR_CORRUPT;
    int rc_all = MX_OK;
    for (uint64_t c = 0; c < n_chunks; ++c) {
        uint64_t a = rd32(msg + 32 + 4 * c), z = rd32(msg + 32 + 4 * (c + 1));
        uint64_t first = c * chunk_symbols;
        uint64_t n_c = n_sym - first < chunk_symbols ? n_sym - first : chunk_symbols;
        if (z < a || z > end_all) return MX_ERR_CORRUPT;
        int rc = orc_decode_chunk_prefix(msg + data0 + a, z - a, len, n_alpha, N, sym_out + first,
                                         n_c);
        if (rc && !rc_all) rc_all = rc;
    }
    return rc_all;
}
