"""Pins that tie the CPU oracle to what the paper and the mathematics fix.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError
if the oracle disagrees with:

  * values the paper prints for its worked example (Section 2.1, and the
    bypass-coding paragraph of Section 3), read from tests/golden/;
  * properties the paper states: C(D(x)) = x (Section 2), encoder and decoder
    pass through the same states in opposite order (Section 2.1, Section 3),
    b-uniqueness of the precursor sets (Section 2), at most one
    renormalization per symbol when b >= M (Section 5), and identical
    bitstreams for the serial interleaved coder and the vectorised
    packed-load / packed-store coder (Sections 5 and 6);
  * closed forms derived here: the power-of-two uniform table, where C is a
    bit-field insertion; infinite-precision ANS (no renormalization); the
    coded-size bound around the model's information content;
  * brute force on tiny inputs (unique decodability).

tests/test_oracle_pins.py runs every pin on the real oracle;
tests/test_oracle_mutants.py runs them on copies with planted mistakes and
requires each copy to fail at least one pin.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
L16 = 1 << 16
B16 = 1 << 16
M12 = 1 << 12


def read_golden(name: str) -> dict:
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            vals[k] = v.split()
    return vals


PAPER = read_golden("paper_example_babba.txt")
PAPER_FREQ = [1, 3]          # a -> f=1, B=0 ; b -> f=3, B=1 ; M = 4
PAPER_SYM = {"a": 0, "b": 1}


def paper_C(s: int, x: int) -> int:
    """The paper's printed coding function (Section 2.1)."""
    return 4 * x if s == 0 else 4 * (x // 3) + (x % 3) + 1


def paper_D(x: int):
    """The paper's printed decoding function (Section 2.1)."""
    return (0, x // 4) if x % 4 == 0 else (1, 3 * (x // 4) + (x % 4) - 1)


def cum_of(freq):
    f = np.asarray(freq, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(f)[:-1]])


# ----------------------------------------------------------------------------
# Worked example of Section 2.1
# ----------------------------------------------------------------------------

def pin_paper_C_D(o):
    for x in range(0, 600):
        assert o.C(PAPER_FREQ, 0, x) == paper_C(0, x), ("C(a,x)", x)
        assert o.C(PAPER_FREQ, 1, x) == paper_C(1, x), ("C(b,x)", x)
    for x in range(1, 600):
        assert o.D(PAPER_FREQ, x) == paper_D(x), ("D", x)


def pin_paper_precursor_sets(o):
    L, b = int(PAPER["L"][0]), int(PAPER["b"][0])
    lo, hi = (int(v) for v in PAPER["I"])
    assert (lo, hi) == (L, b * L - 1)
    for s, key in ((0, "precursor_a"), (1, "precursor_b")):
        got = [x for x in range(0, 200) if L <= o.C(PAPER_FREQ, s, x) < b * L]
        assert got == [int(v) for v in PAPER[key]], key


def _paper_message():
    return [PAPER_SYM[c] for c in PAPER["message"]]


def pin_paper_state_30(o):
    L, b = int(PAPER["L"][0]), int(PAPER["b"][0])
    msg = _paper_message()
    enc = o.encode(PAPER_FREQ, msg, N=1, L=L, b=b)
    # Decoding the first two symbols ("b", then the first "a") leaves the
    # decoder in the state the paper names.
    dec2 = o.decode(PAPER_FREQ, enc["words"], enc["states"], 2, N=1, L=L, b=b)
    assert list(dec2["symbols"]) == msg[:2]
    assert int(dec2["states_end"][0]) == int(PAPER["state_after_first_a"][0])
    full = o.decode(PAPER_FREQ, enc["words"], enc["states"], len(msg), N=1, L=L, b=b)
    assert list(full["symbols"]) == msg
    assert full["consumed"] == len(enc["words"])
    assert int(full["states_end"][0]) == L


def pin_paper_lockstep(o):
    L, b = int(PAPER["L"][0]), int(PAPER["b"][0])
    msg = _paper_message()
    enc = o.encode(PAPER_FREQ, msg, N=1, L=L, b=b, trace=True)
    dec = o.decode(PAPER_FREQ, enc["words"], enc["states"], len(msg), N=1, L=L, b=b,
                   trace=True)
    assert list(dec["trace_state"]) == list(enc["trace_state"][::-1])
    assert 30 in list(dec["trace_state"])
    assert enc["max_iters"] == 2        # b = 2 < M = 4: two bits at once happen


# ----------------------------------------------------------------------------
# Properties stated in Sections 2, 3, 5
# ----------------------------------------------------------------------------

def pin_lockstep_interleaved(o):
    """Encoder and decoder pass through the same (coder, state) sequence in
    opposite order, for several interleaved coders (Sections 2.1 and 3)."""
    rng = np.random.default_rng(7)
    for N, (L, b, freq) in itertools.product(
            (1, 2, 3, 5), ((16, 2, PAPER_FREQ), (L16, B16, [1000, 3000, 96]))):
        msg = rng.integers(0, len(freq), size=int(rng.integers(1, 40)))
        enc = o.encode(freq, msg, N=N, L=L, b=b, trace=True)
        dec = o.decode(freq, enc["words"], enc["states"], msg.size, N=N, L=L, b=b,
                       trace=True)
        assert list(dec["symbols"]) == list(msg)
        # Each trace starts with the N states a coder holds at the start, then
        # records (coder, state) after every step.  Per coder, the decoder's
        # states are the encoder's in reverse order ...
        for j in range(N):
            e_j = [int(v) for v, c in zip(enc["trace_state"], enc["trace_lane"]) if c == j]
            d_j = [int(v) for v, c in zip(dec["trace_state"], dec["trace_lane"]) if c == j]
            assert d_j == e_j[::-1], (N, j)
        # ... and the coders take their steps in exactly the reverse order.
        assert list(dec["trace_lane"][N:]) == list(enc["trace_lane"][N:][::-1])


def pin_inverse_exhaustive(o):
    """D is C's inverse: C(D(x)) = x and D(C(s,x)) = (s,x) (Section 2)."""
    rng = np.random.default_rng(11)
    for freq in ([16], [1, 15], [3, 5, 8], list(rng.integers(1, 9, size=6))):
        n = len(freq)
        for x in range(1, 1500):
            s, y = o.D(freq, x)
            assert o.C(freq, s, y) == x
            for t in range(n):
                assert o.D(freq, o.C(freq, t, x)) == (t, x)


def pin_precursor_rans_b_unique(o):
    """For the range coder with M | L the precursor set of every symbol is
    {k, ..., b*k - 1} with k = f_s * L / M, i.e. b-unique (Section 2)."""
    for freq, L, b in (([1, 3], 16, 2), ([2, 5, 9], 32, 4), ([1, 1, 6], 64, 3),
                       ([5, 11], 16, 5)):
        M = sum(freq)
        assert L % M == 0
        for s, f in enumerate(freq):
            got = [x for x in range(0, b * L + 1) if L <= o.C(freq, s, x) < b * L]
            k = f * L // M
            assert got == list(range(k, b * k)), (freq, s)


def pin_one_renorm_production(o):
    """With b = 2^16 >= M = 2^12 no symbol needs more than one
    renormalization step (Section 5)."""
    rng = np.random.default_rng(3)
    for trial in range(6):
        n = int(rng.integers(1, 256))
        freq = o.quantize(rng.integers(1, 1 << 20, size=n).astype(np.uint64))
        if trial == 0:
            freq = np.zeros(n, dtype=np.uint16)
            freq[0] = M12 - (n - 1)
            freq[1:] = 1
        p = freq / freq.sum()
        msg = rng.choice(n, size=3000, p=p)
        msg[:50] = n - 1                      # rarest symbol, largest state jumps
        enc = o.encode(freq, msg, N=int(rng.integers(1, 33)))
        assert enc["max_iters"] <= 1


# ----------------------------------------------------------------------------
# Closed forms
# ----------------------------------------------------------------------------

def bit_insertion_stream(symbols, k, N):
    """Stream for the uniform table over 2^k symbols (f_s = 2^(12-k),
    B_s = s * 2^(12-k)).  With power-of-two frequencies the coding function
    inserts the symbol's k bits at bit (12-k) of the state and moves the bits
    above up by k; renormalization moves the low 16 bits out once the state
    reaches 2^(32-k) = f_s * 2^20.  Only shifts and masks are used here."""
    lo_bits = 12 - k
    x = [L16] * N
    emitted = []
    n = len(symbols)
    for i in range(n - 1, -1, -1):
        j = i % N
        s = int(symbols[i])
        if x[j] >= 1 << (32 - k):
            emitted.append(x[j] & 0xFFFF)
            x[j] >>= 16
        x[j] = ((x[j] >> lo_bits) << 12) | (s << lo_bits) | (x[j] & ((1 << lo_bits) - 1))
    return emitted[::-1], x


def bitlength_word_count(counts, k):
    """Words emitted by a coder that codes c symbols of k bits each: the
    state's bit length starts at 16 (x0 = 2^16), grows by exactly k per
    symbol and drops by exactly 16 per emitted word, emitting whenever it
    has reached 32 - k before a symbol."""
    total = 0
    for c in counts:
        e = 16
        for _ in range(c):
            if e >= 32 - k:
                e -= 16
                total += 1
            e += k
    return total


def pin_uniform_closed_form(o):
    rng = np.random.default_rng(5)
    for k, N in itertools.product((1, 2, 4, 8), (1, 7, 32)):
        freq = [1 << (12 - k)] * (1 << k)
        n = int(rng.integers(1, 700))
        msg = rng.integers(0, 1 << k, size=n)
        enc = o.encode(freq, msg, N=N)
        words, states = bit_insertion_stream(msg, k, N)
        assert list(enc["words"]) == words, (k, N)
        assert list(enc["states"]) == states, (k, N)
        counts = [len(range(j, n, N)) for j in range(N)]
        assert len(words) == bitlength_word_count(counts, k)
        if k == 8:
            assert len(words) == sum(c // 2 for c in counts)


def pin_single_symbol(o):
    """f_s = M makes C the identity: nothing is emitted and every coder
    keeps x0 = L."""
    for freq, s in (([M12], 0), ([0, M12, 0], 1)):
        msg = [s] * 77
        enc = o.encode(freq, msg, N=5)
        assert len(enc["words"]) == 0
        assert list(enc["states"]) == [L16] * 5
        dec = o.decode(freq, [], enc["states"], 77, N=5)
        assert list(dec["symbols"]) == msg


def pin_infinite_precision_paper(o):
    """With an interval so wide that no renormalization happens, streaming
    ANS is infinite-precision ANS: the final state is the nested coding
    function of the whole message (Section 1), here with the paper's
    printed C (Section 2.1)."""
    L, b = 1 << 20, 1 << 40
    for n in range(0, 13):
        for msg in itertools.islice(itertools.product((0, 1), repeat=n), 40):
            X = L
            for s in reversed(msg):
                X = paper_C(s, X)
            enc = o.encode(PAPER_FREQ, list(msg), N=1, L=L, b=b)
            assert len(enc["words"]) == 0
            assert int(enc["states"][0]) == X
            # Decoding the big state with the paper's D recovers the message.
            got = []
            for _ in msg:
                s, X = paper_D(X)
                got.append(s)
            assert tuple(got) == msg and X == L


def pin_infinite_precision_general(o):
    rng = np.random.default_rng(9)
    L, b = 1 << 16, 1 << 44
    for _ in range(40):
        n = int(rng.integers(2, 4))
        freq = [int(v) for v in rng.integers(1, 6, size=n)]
        M = sum(freq)
        B = [sum(freq[:s]) for s in range(n)]
        msg = [int(v) for v in rng.integers(0, n, size=int(rng.integers(1, 10)))]
        X = L
        for s in reversed(msg):
            X = (X // freq[s]) * M + B[s] + X % freq[s]
        if not (L <= X < b * L):
            continue
        enc = o.encode(freq, msg, N=1, L=L, b=b)
        assert len(enc["words"]) == 0 and int(enc["states"][0]) == X


def pin_size_bound(o):
    """Coded size against the model's information content.

    For one coding step write x = q f + r (0 <= r < f); then
    x' = q M + B + r lies in [qM, (q+1)M), so
        (M/f) (x - f) < x' < (M/f) (x + f).
    After renormalization x is in the precursor set [16 f, 2^20 f), hence
        log2(M/f) + log2(15/16) < log2(x'/x) < log2(M/f) + log2(17/16).
    An emitted word divides x by 2^16 and drops a remainder < 2^16, and the
    state left behind is >= 16, so each word removes between 16 and
    16 + log2(17/16) bits.  Telescoping each coder from x0 = L:
        bits := 16 W + sum_j log2(x_j / L)
        bits <  sum_i log2(M / f_{s_i}) + n log2(17/16)
        bits >  sum_i log2(M / f_{s_i}) + n log2(15/16) - W log2(17/16)
    """
    rng = np.random.default_rng(13)
    up, dn = math.log2(17 / 16), math.log2(15 / 16)
    for trial in range(10):
        n_alpha = int(rng.integers(2, 257))
        p = rng.dirichlet(np.full(n_alpha, 0.3 if trial % 2 else 1.0))
        freq = o.quantize(np.maximum(np.rint(p * 2.0 ** 32), 1).astype(np.uint64))
        q = freq / freq.sum()
        n = int(rng.integers(1, 5000))
        msg = rng.choice(n_alpha, size=n, p=q)
        N = int(rng.integers(1, 33))
        enc = o.encode(freq, msg, N=N)
        W = len(enc["words"])
        bits = 16 * W + sum(math.log2(int(x) / L16) for x in enc["states"])
        info = float(np.sum(np.log2(M12 / freq[msg].astype(np.float64))))
        assert bits < info + n * up + 1e-9
        assert bits > info + n * dn - W * up - 1e-9


# ----------------------------------------------------------------------------
# Brute force
# ----------------------------------------------------------------------------

def pin_brute_force_unique(o):
    """Every message up to length 8 over the paper's alphabet maps to a
    different (states, words) pair and decodes back (paper parameters)."""
    L, b = int(PAPER["L"][0]), int(PAPER["b"][0])
    for N in (1, 2):
        seen = {}
        for n in range(0, 9):
            for msg in itertools.product((0, 1), repeat=n):
                enc = o.encode(PAPER_FREQ, list(msg), N=N, L=L, b=b)
                key = (tuple(int(v) for v in enc["states"]), tuple(int(v) for v in enc["words"]))
                assert key not in seen, (msg, seen.get(key))
                seen[key] = msg
                dec = o.decode(PAPER_FREQ, enc["words"], enc["states"], n, N=N, L=L, b=b)
                assert tuple(int(v) for v in dec["symbols"]) == msg
                assert dec["consumed"] == len(enc["words"])
                assert all(int(v) == L for v in dec["states_end"])


# ----------------------------------------------------------------------------
# Serial interleaved == vectorised packed I/O (Sections 5, 6)
# ----------------------------------------------------------------------------

def packed_store_encode(freq, msg, N, L=L16, b=B16):
    """All N coders advance together one step at a time (from the last step
    to the first).  Per step each coder renormalizes at most once -- the
    `if` form of Section 5 -- using the precursor-set bound x >= b f L / M,
    and the words of one step are stored packed, in descending coder order
    (the mirror image of the decoder's packed load)."""
    freq = np.asarray(freq, dtype=np.uint64)
    M = int(freq.sum())
    cum = cum_of(freq).astype(np.uint64)
    n = len(msg)
    msg = np.asarray(msg, dtype=np.int64)
    x = np.full(N, L, dtype=np.uint64)
    out = []
    T = -(-n // N)
    lanes = np.arange(N)
    for t in range(T - 1, -1, -1):
        idx = t * N + lanes
        act = idx < n
        s = np.where(act, msg[np.minimum(idx, n - 1)], 0)
        f = np.where(act, freq[s], np.uint64(1))
        B = cum[s]
        xmax = np.uint64(L // M * b) * f
        emit = act & (x >= xmax)
        for j in np.nonzero(emit)[0][::-1]:
            out.append(int(x[j] % np.uint64(b)))
        x = np.where(emit, x // np.uint64(b), x)
        xc = (x // f) * np.uint64(M) + B + x % f
        x = np.where(act, xc, x)
    return out[::-1], [int(v) for v in x]


def packed_load_decode(freq, words, states, n, N, L=L16, b=B16):
    """Vectorised decoder in the GPU form of Section 6: D from a slot table,
    renorm_mask = (x < L), each renormalizing coder reads the word at
    read_pos + (number of renormalizing coders before it), then read_pos
    advances by the mask's population count."""
    freq = np.asarray(freq, dtype=np.int64)
    M = int(freq.sum())
    cum = cum_of(freq)
    slot_sym = np.repeat(np.arange(len(freq)), freq)
    x = np.asarray(states, dtype=np.int64).copy()
    w = np.asarray(words, dtype=np.int64)
    out = np.zeros(n, dtype=np.int64)
    rp = 0
    lanes = np.arange(N)
    for t in range(-(-n // N)):
        idx = t * N + lanes
        act = idx < n
        slot = x % M
        s = slot_sym[slot]
        xn = freq[s] * (x // M) + slot - cum[s]
        x = np.where(act, xn, x)
        out[idx[act]] = s[act]
        mask = act & (x < L)
        offs = np.cumsum(mask) - mask
        pos = rp + offs
        assert pos[mask].size == 0 or pos[mask].max() < w.size
        x = np.where(mask, x * b + w[np.where(mask, pos, 0)] if w.size else x, x)
        rp += int(mask.sum())
    return out, rp, [int(v) for v in x]


def pin_packed_io_equivalence(o):
    rng = np.random.default_rng(17)
    for trial in range(8):
        n_alpha = int(rng.integers(1, 257))
        p = rng.dirichlet(np.full(n_alpha, 0.5))
        freq = o.quantize(np.maximum(np.rint(p * 2.0 ** 32), 1).astype(np.uint64))
        q = freq / freq.sum()
        n = int(rng.integers(0, 3000))
        N = (1, 4, 13, 32, 32, 31, 2, 32)[trial]
        msg = rng.choice(n_alpha, size=n, p=q)
        enc = o.encode(freq, msg, N=N)
        w2, st2 = packed_store_encode(freq, msg, N)
        assert [int(v) for v in enc["words"]] == w2
        assert [int(v) for v in enc["states"]] == st2
        sym, rp, st_end = packed_load_decode(freq, enc["words"], enc["states"], n, N)
        assert list(sym) == list(msg)
        assert rp == len(w2) and st_end == [L16] * N


# ----------------------------------------------------------------------------
# Container (production format) and quantizer
# ----------------------------------------------------------------------------

def pin_round_trip_edges(o):
    rng = np.random.default_rng(19)
    freqs = {
        1: np.array([M12], dtype=np.uint16),
        2: np.array([1, M12 - 1], dtype=np.uint16),
        256: o.quantize(rng.integers(1, 1 << 30, size=256).astype(np.uint64)),
    }
    for n_alpha, N, cs in itertools.product((1, 2, 256), (1, 5, 32), (1, 7, 64, 4096)):
        fr = freqs[n_alpha]
        for n in sorted({0, 1, N - 1, N, N + 1, cs, cs + 1, 3 * cs - 1, 2 * N * 7 + 3}):
            if n < 0 or n > 20000:
                continue
            msg = rng.choice(n_alpha, size=n, p=fr / fr.sum()).astype(np.uint8)
            blob = o.encode_message(msg, fr, N=N, chunk_symbols=cs)
            assert blob.size % 16 == 0
            back = o.decode_message(blob, n, fr, N=N, chunk_symbols=cs)
            assert np.array_equal(back, msg)


def pin_container_layout(o):
    rng = np.random.default_rng(23)
    fr = o.quantize(rng.integers(1, 1 << 30, size=200).astype(np.uint64))
    for n, N, cs in ((0, 32, 64), (1000, 32, 64), (999, 7, 100), (5, 3, 1)):
        msg = rng.choice(200, size=n, p=fr / fr.sum()).astype(np.uint8)
        blob = o.encode_message(msg, fr, N=N, chunk_symbols=cs)
        h = blob[:32].view(np.uint32)
        n_chunks = -(-n // cs)
        assert list(h[:4]) == [0x534E4152, 1, N, 12]
        assert int(h[4]) | (int(h[5]) << 32) == n
        assert list(h[6:8]) == [cs, n_chunks]
        offs = blob[32:32 + 4 * (n_chunks + 1)].view(np.uint32).astype(np.int64)
        data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
        assert offs[0] == 0 and np.all(np.diff(offs) >= 4 * N)
        assert blob.size == data0 + (int(offs[-1]) + 15) // 16 * 16
        assert not blob[32 + 4 * (n_chunks + 1):data0].any()
        assert not blob[data0 + int(offs[-1]):].any()
        for c in range(n_chunks):
            a, z = data0 + offs[c], data0 + offs[c + 1]
            one = o.encode_chunk(msg[c * cs:(c + 1) * cs], fr, N=N)
            assert np.array_equal(blob[a:z], one)
            assert (z - a - 4 * N) % 2 == 0


def pin_quantize(o):
    rng = np.random.default_rng(29)
    # Hand-worked cases of the stated rule.
    assert list(o.quantize([1, 1, 1], log2_M=2)) == [2, 1, 1]          # tie -> lower index
    assert list(o.quantize([5, 3], log2_M=2)) == [3, 1]                # remainders tie (4, 4)
    assert list(o.quantize([1_000_000, 1, 1, 1], log2_M=2)) == [1, 1, 1, 1]  # excess removed
    assert list(o.quantize([0, 7, 0, 1], log2_M=3)) == [0, 7, 0, 1]     # exact
    assert list(o.quantize([3, 0, 1], log2_M=4)) == [12, 0, 4]
    for _ in range(200):
        n = int(rng.integers(1, 257))
        w = rng.integers(0, 1 << int(rng.integers(1, 55)), size=n).astype(np.uint64)
        w[rng.random(n) < 0.2] = 0
        if not w.any():
            w[0] = 1
        f = o.quantize(w)
        assert int(f.sum()) == M12
        assert np.array_equal(f > 0, w > 0)
        # exact proportional weights are reproduced
        g = o.quantize(f.astype(np.uint64) * np.uint64(rng.integers(1, 1000)))
        assert np.array_equal(g, f)


# ----------------------------------------------------------------------------
# Bypass: raw digits interleaved with the coded symbols (Section 3)
# ----------------------------------------------------------------------------

def pin_bypass_paper_example(o):
    """The paper's bypass example: each a of "babba" carries two raw bits
    (its subtype), sent before the a is encoded and read right after it is
    decoded.  The bits sit in the stream exactly where the plain decoder has
    just finished the a (state 30 for the first one), and no coder state
    changes: the state traces with and without the raw bits are equal."""
    L, b = int(PAPER["L"][0]), int(PAPER["b"][0])
    nbits = int(PAPER["bypass_bits_per_a"][0])
    msg = _paper_message()
    counts = [nbits, 0]
    subtypes = [[1, 0], [1, 1]]                       # a_2 and a_3, first bit first
    raw = [bit for st in subtypes for bit in st]
    plain = o.encode(PAPER_FREQ, msg, N=1, L=L, b=b, trace=True)
    byp = o.encode_bypass(PAPER_FREQ, msg, counts, raw, N=1, L=L, b=b, trace=True)
    assert list(byp["trace_state"]) == list(plain["trace_state"])
    assert list(byp["states"]) == list(plain["states"])
    # where the plain decoder stands after each a
    a_at = [i for i, c in enumerate(msg) if c == PAPER_SYM["a"]]
    cut = [o.decode(PAPER_FREQ, plain["words"], plain["states"], i + 1, N=1, L=L, b=b)["consumed"]
           for i in a_at]
    first = o.decode(PAPER_FREQ, plain["words"], plain["states"], a_at[0] + 1, N=1, L=L, b=b)
    assert int(first["states_end"][0]) == int(PAPER["state_after_first_a"][0])
    w, expect, prev = list(plain["words"]), [], 0
    for c, st in zip(cut, subtypes):
        expect += w[prev:c] + st
        prev = c
    expect += w[prev:]
    assert list(byp["words"]) == expect
    dec = o.decode_bypass(PAPER_FREQ, byp["words"], byp["states"], len(msg), counts, N=1, L=L,
                          b=b, trace=True)
    assert list(dec["symbols"]) == msg and list(dec["raw"]) == raw
    assert dec["consumed"] == len(expect) and int(dec["states_end"][0]) == L
    assert list(dec["trace_state"]) == list(plain["trace_state"][::-1])


def pin_bypass_without_raw_is_plain(o):
    """No symbol carries raw digits: the bypass coder is the plain coder, and
    a bypass message differs from the plain one only in its version field."""
    rng = np.random.default_rng(11)
    for N in (1, 5, 32):
        freq = o.quantize(np.maximum(1, rng.integers(0, 1000, size=40)).astype(np.uint64))
        msg = rng.choice(40, size=777, p=freq / freq.sum())
        plain = o.encode(freq, msg, N=N)
        byp = o.encode_bypass(freq, msg, np.zeros(40, np.uint32), [], N=N)
        assert np.array_equal(plain["words"], byp["words"])
        assert np.array_equal(plain["states"], byp["states"])
        m_plain = o.encode_message(msg.astype(np.uint8), freq, N=N, chunk_symbols=300)
        m_byp = o.encode_message_bypass(msg.astype(np.uint8), np.zeros(777, np.uint16), freq,
                                        np.zeros(40, np.uint8), N=N, chunk_symbols=300)
        assert m_plain.size == m_byp.size
        diff = np.nonzero(m_plain != m_byp)[0]
        assert list(diff) == [4], diff                 # version 1 -> 2
        assert m_byp[4] == 2 and m_plain[4] == 1


def pin_bypass_interleaved(o):
    """Production parameters, N interleaved coders, random raw-word flags:
    the raw words change no coder state (same encoder trace as without
    them), add exactly one word each, and decode back, words and symbols."""
    rng = np.random.default_rng(13)
    for N, n in ((1, 50), (3, 401), (32, 3000), (32, 31)):
        k = int(rng.integers(2, 60))
        freq = o.quantize(np.maximum(1, rng.integers(0, 1000, size=k)).astype(np.uint64))
        flags = (rng.random(k) < 0.5).astype(np.uint32)
        msg = rng.choice(k, size=n, p=freq / freq.sum())
        raw = rng.integers(0, 1 << 16, size=int(flags[msg].sum()))
        plain = o.encode(freq, msg, N=N, trace=True)
        byp = o.encode_bypass(freq, msg, flags, raw, N=N, trace=True)
        assert np.array_equal(plain["trace_state"], byp["trace_state"])
        assert byp["words"].size == plain["words"].size + raw.size
        dec = o.decode_bypass(freq, byp["words"], byp["states"], n, flags, N=N)
        assert np.array_equal(dec["symbols"], msg) and np.array_equal(dec["raw"], raw)
        assert dec["consumed"] == byp["words"].size
        assert all(int(v) == L16 for v in dec["states_end"])
        # container: per-position raw words, zero where a symbol has none
        r16 = np.zeros(n, np.uint16)
        r16[flags[msg] == 1] = raw
        m = o.encode_message_bypass(msg.astype(np.uint8), r16, freq, flags.astype(np.uint8), N=N,
                                    chunk_symbols=200)
        sym2, raw2 = o.decode_message_bypass(m, n, freq, flags.astype(np.uint8), N=N,
                                             chunk_symbols=200)
        assert np.array_equal(sym2, msg) and np.array_equal(raw2, r16)


# ----------------------------------------------------------------------------
# Several renormalization digits per symbol, width-baked order (Section 5)
# ----------------------------------------------------------------------------

L23 = 1 << 23
B8 = 1 << 8


def digits_per_symbol(o, freq, msg, N, L, b):
    """k_i = renormalization digits the serial decoder reads for symbol i,
    from its state trace: per symbol one entry after D, then one per digit
    (consecutive symbols sit on different lanes when N >= 2)."""
    enc = o.encode(freq, msg, N=N, L=L, b=b)
    dec = o.decode(freq, enc["words"], enc["states"], len(msg), N=N, L=L, b=b, trace=True)
    lanes = list(dec["trace_lane"][N:])
    k, i = [], 0
    while i < len(lanes):
        j = i + 1
        while j < len(lanes) and lanes[j] == lanes[i]:
            j += 1
        k.append(j - i - 1)
        i = j
    assert len(k) == len(msg)
    return enc, k


def pin_wide_one_lane_is_algorithm1(o):
    """With N = 1 the width-baked coder is Algorithm 1 itself."""
    rng = np.random.default_rng(17)
    for L, b in ((16, 2), (L23, B8), (1 << 14, 4)):
        freq = [1, 3] if L == 16 else o.quantize(
            np.maximum(1, rng.integers(0, 1000, size=30)).astype(np.uint64))
        msg = _paper_message() if L == 16 else rng.choice(30, size=500, p=np.asarray(freq) / np.sum(freq))
        a = o.encode(freq, msg, N=1, L=L, b=b)
        w = o.encode_wide(freq, msg, N=1, L=L, b=b)
        assert list(a["words"]) == list(w["words"]) and list(a["states"]) == list(w["states"])


def pin_wide_breadth_first(o):
    """The SIMD order of Section 5: within a step of N symbols the decoder
    reads first one digit for every lane that needs one (lanes in order),
    then a second digit for every lane that needs two, and so on -- the
    paper's two-lane example: lane 0's first byte, lane 1's byte, lane 0's
    second byte.  Built here from the serial (depth-first) stream of
    Algorithm 1 and compared with the width-baked coder; states are equal."""
    rng = np.random.default_rng(19)
    saw_example = False
    for N in (2, 5, 32):
        freq = o.quantize(np.maximum(1, rng.integers(0, 1000, size=64)).astype(np.uint64))
        msg = rng.choice(64, size=40 * N + 3, p=freq / freq.sum())
        ser, k = digits_per_symbol(o, freq, msg, N, L23, B8)
        pos, per_sym = 0, []
        for ki in k:
            per_sym.append(list(ser["words"][pos:pos + ki]))
            pos += ki
        expect = []
        for t0 in range(0, len(msg), N):
            syms = list(range(t0, min(len(msg), t0 + N)))
            for r in range(max(k[i] for i in syms)):
                expect += [per_sym[i][r] for i in syms if k[i] > r]
            if N >= 2 and len(syms) >= 2 and k[syms[0]] == 2 and k[syms[1]] == 1:
                saw_example = True
        wide = o.encode_wide(freq, msg, N=N, L=L23, b=B8)
        assert list(wide["words"]) == expect, N
        assert list(wide["states"]) == list(ser["states"])
        dec = o.decode_wide(freq, wide["words"], wide["states"], len(msg), N=N, L=L23, b=B8)
        assert list(dec["symbols"]) == list(msg) and dec["consumed"] == len(expect)
        assert all(int(v) == L23 for v in dec["states_end"])
    assert saw_example


def pin_bytes_container(o):
    """Byte-wise messages: version 3, chunks of [N states][digits][zeros to
    a multiple of 4]; round trip; a chunk equals the width-baked coder's
    output for its symbols."""
    rng = np.random.default_rng(23)
    freq = o.quantize(np.maximum(1, rng.integers(0, 1000, size=100)).astype(np.uint64))
    msg = rng.choice(100, size=5000, p=freq / freq.sum()).astype(np.uint8)
    N, CS = 7, 1000
    m = o.encode_message_bytes(msg, freq, N=N, chunk_symbols=CS)
    assert int.from_bytes(m[4:8].tobytes(), "little") == 3
    n_chunks = 5
    data0 = (32 + 4 * (n_chunks + 1) + 15) // 16 * 16
    offs = m[32:32 + 4 * (n_chunks + 1)].view(np.uint32)
    for c in range(n_chunks):
        ch = m[data0 + offs[c]:data0 + offs[c + 1]]
        assert ch.size % 4 == 0
        w = o.encode_wide(freq, msg[c * CS:(c + 1) * CS], N=N, L=L23, b=B8)
        assert list(ch[:4 * N].view(np.uint32)) == list(w["states"])
        body = ch[4 * N:]
        assert list(body[:w["words"].size]) == list(w["words"])
        assert not body[w["words"].size:].any()
    assert np.array_equal(o.decode_message_bytes(m, msg.size, freq, N=N, chunk_symbols=CS), msg)


# ----------------------------------------------------------------------------
# Adaptive binary contexts, one per coder (Section 5)
# ----------------------------------------------------------------------------

def pin_adaptive_lanes_independent(o):
    """Separate contexts per lane: with N coders, coder j's final state is
    exactly that of a single coder run on symbols j, j+N, j+2N, ... alone, and
    the interleaved stream decodes back."""
    rng = np.random.default_rng(29)
    for N in (2, 3, 8):
        msg = (rng.random(40 * N + 5) < rng.uniform(0.02, 0.5)).astype(np.uint32)
        enc = o.encode_adaptive(msg, N=N)
        for j in range(N):
            solo = o.encode_adaptive(msg[j::N], N=1)
            assert int(enc["states"][j]) == int(solo["states"][0]), (N, j)
        dec = o.decode_adaptive(enc["words"], enc["states"], msg.size, N=N)
        assert np.array_equal(dec["symbols"], msg) and dec["consumed"] == enc["words"].size
        assert all(int(v) == L16 for v in dec["states_end"])


def pin_adaptive_brute_force(o):
    """All binary messages up to 10 symbols, N = 1..3: distinct messages get
    distinct encodings, and every one decodes back."""
    for N in (1, 2, 3):
        seen = {}
        for n in range(0, 11):
            for bits in itertools.product((0, 1), repeat=n):
                enc = o.encode_adaptive(list(bits), N=N)
                key = (n, tuple(enc["words"]), tuple(int(v) for v in enc["states"]))
                assert key not in seen
                seen[key] = bits
                dec = o.decode_adaptive(enc["words"], enc["states"], n, N=N)
                assert tuple(dec["symbols"]) == bits


def pin_adaptive_size_and_learning(o):
    """The coded size stays within the derived bound around the information
    content of the probabilities the contexts give (reading 13, per symbol);
    a long run of one bit costs a small fraction of a bit per symbol once the
    context has learned it; the context never leaves [1, M-1] (else coding
    would fail)."""
    rng = np.random.default_rng(31)
    M, R = 1 << 12, 5
    for N, msg in ((1, (rng.random(3000) < 0.1).astype(np.uint32)),
                   (4, (rng.random(4000) < 0.3).astype(np.uint32)),
                   (2, np.concatenate([np.zeros(6000, np.uint32), np.ones(6000, np.uint32)]))):
        ctx = [2048] * N
        info = 0.0
        for i, s in enumerate(msg):
            j = i % N
            f = ctx[j] if s == 0 else M - ctx[j]
            info += math.log2(M / f)
            ctx[j] = ctx[j] + ((M - ctx[j]) >> R) if s == 0 else ctx[j] - (ctx[j] >> R)
            assert 1 <= ctx[j] <= M - 1
        enc = o.encode_adaptive(msg, N=N)
        W = enc["words"].size
        bits = 16 * W + sum(math.log2(int(x) / L16) for x in enc["states"])
        n = msg.size
        lo = info + n * math.log2(15 / 16) - W * math.log2(17 / 16) - 1e-6
        hi = info + n * math.log2(17 / 16) + 1e-6
        assert lo <= bits <= hi, (N, lo, bits, hi)
    assert bits / msg.size < 0.2      # the runs: far below 1 bit per symbol


def pin_adaptive_container(o):
    rng = np.random.default_rng(37)
    msg = (rng.random(5000) < 0.2).astype(np.uint8)
    m = o.encode_message_adaptive(msg, N=7, chunk_symbols=999)
    assert int.from_bytes(m[4:8].tobytes(), "little") == 4
    assert np.array_equal(o.decode_message_adaptive(m, msg.size, N=7, chunk_symbols=999), msg)
    data0 = (32 + 4 * 7 + 15) // 16 * 16
    offs = m[32:32 + 4 * 7].view(np.uint32)
    enc = o.encode_adaptive(msg[:999].astype(np.uint32), N=7)
    ch = m[data0 + offs[0]:data0 + offs[1]]
    assert list(ch[:28].view(np.uint32)) == list(enc["states"])
    assert list(ch[28:].view(np.uint16)) == list(enc["words"])


# ----------------------------------------------------------------------------
# Adaptive models over n symbols, one per coder (Section 5)
# ----------------------------------------------------------------------------

def pin_adaptive_n_worked_example(o):
    """The model update worked out by hand for two small cases.

    (a) M = 16, n = 3, R = 1, start floor(i*16/3) = [0, 5, 10, 16]; targets
        i below and at the coded symbol, 13 + i above it:
        s=2: C1 = 5-((5-1)>>1) = 3, C2 = 10-((10-2)>>1) = 6
        s=0: C1 = 3+((14-3)>>1) = 8, C2 = 6+((15-6)>>1) = 10
        s=1: C1 = 8-((8-1)>>1) = 5, C2 = 10+((15-10)>>1) = 12
        s=1: C1 = 5-2 = 3, C2 = 12+1 = 13
        s=2: C1 = 3-1 = 2, C2 = 13-5 = 8
        s=2: C1 = 2-0 = 2, C2 = 8-3 = 5
        s=0: C1 = 2+6 = 8, C2 = 5+5 = 10
    (b) M = 4096, n = 4, R = 5, start [0, 1024, 2048, 3072, 4096]:
        s=0: +(3069>>5)=95, +(2046>>5)=63, +(1023>>5)=31 -> 1119 2111 3103
        s=3: -(1118>>5)=34, -(2109>>5)=65, -(3100>>5)=96 -> 1085 2046 3007"""
    rows = [[0, 5, 10, 16], [0, 3, 6, 16], [0, 8, 10, 16], [0, 5, 12, 16], [0, 3, 13, 16],
            [0, 2, 8, 16], [0, 2, 5, 16], [0, 8, 10, 16]]
    tr = o.adaptive_n_trace([2, 0, 1, 1, 2, 2, 0], 3, M=16, R=1)
    assert tr.tolist() == rows
    tr = o.adaptive_n_trace([0, 3], 4, M=4096, R=5)
    assert tr.tolist() == [[0, 1024, 2048, 3072, 4096], [0, 1119, 2111, 3103, 4096],
                           [0, 1085, 2046, 3007, 4096]]


def pin_adaptive_n_invariants(o):
    """Along long random sequences every model is a valid one (C_0 = 0,
    C_n = M, every f >= 1, boundary i within [i, M - n + i]); coding a
    symbol never narrows its own interval nor widens another's; and a
    symbol coded over and over settles: each boundary below it within
    2^R - 1 of its target, where the update stops moving it."""
    rng = np.random.default_rng(41)
    M = 1 << 12
    for n in (2, 5, 16):
        seq = rng.integers(0, n, size=3000).astype(np.uint32)
        seq[1000:1600] = 1
        tr = o.adaptive_n_trace(seq, n)
        i = np.arange(n + 1)
        assert (tr[:, 0] == 0).all() and (tr[:, n] == M).all()
        f = np.diff(tr, axis=1)
        assert (f >= 1).all()
        assert (tr >= i).all() and (tr <= M - n + i).all()
        for k, s in enumerate(seq):
            grow = f[k + 1] - f[k]
            assert grow[s] >= 0 and (np.delete(grow, s) <= 0).all(), (n, k)
        # a long run of the last symbol: every boundary settles within 2^R - 1
        # of its lower target i (the shift no longer moves it), after which
        # the model is fixed
        run = o.adaptive_n_trace(np.full(5000, n - 1, np.uint32), n)
        a = run[-1][1:n] - np.arange(1, n)
        assert (a >= 0).all() and (a >> 5 == 0).all()
        assert np.array_equal(run[-1], run[-2])
        assert M - run[-1][n - 1] >= M - (n - 1) - 31


def pin_adaptive_n_static_limit(o):
    """With R = 30 no boundary ever moves (every distance is below 2^30), so
    each coder keeps the uniform start model and the stream is the static
    Algorithm-1 coder's with f = diff(floor(i*M/n))."""
    rng = np.random.default_rng(43)
    for n, N in ((3, 1), (7, 4), (16, 5)):
        msg = rng.integers(0, n, size=2000).astype(np.uint32)
        freq = np.diff([(i * M12) // n for i in range(n + 1)])
        a = o.encode_adaptive_n(msg, n, N=N, R=30)
        s = o.encode(freq, msg, N=N)
        assert np.array_equal(a["words"], s["words"])
        assert np.array_equal(a["states"], s["states"])


def pin_adaptive_n_lanes_independent(o):
    """Separate models per lane: coder j's final state equals that of one
    coder run on symbols j, j+N, ... alone, and the stream decodes back."""
    rng = np.random.default_rng(47)
    for n, N in ((4, 2), (9, 3), (16, 8)):
        p = rng.dirichlet(np.full(n, 0.4))
        msg = rng.choice(n, size=60 * N + 7, p=p).astype(np.uint32)
        enc = o.encode_adaptive_n(msg, n, N=N)
        for j in range(N):
            solo = o.encode_adaptive_n(msg[j::N], n, N=1)
            assert int(enc["states"][j]) == int(solo["states"][0]), (n, N, j)
        dec = o.decode_adaptive_n(enc["words"], enc["states"], msg.size, n, N=N)
        assert np.array_equal(dec["symbols"], msg) and dec["consumed"] == enc["words"].size
        assert all(int(v) == L16 for v in dec["states_end"])


def pin_adaptive_n_brute_force(o):
    """All messages over 3 symbols up to length 6, N = 1 and 2: distinct
    messages get distinct encodings, and every one decodes back."""
    for N in (1, 2):
        seen = set()
        for k in range(0, 7):
            for msg in itertools.product(range(3), repeat=k):
                enc = o.encode_adaptive_n(list(msg), 3, N=N)
                key = (k, tuple(enc["words"]), tuple(int(v) for v in enc["states"]))
                assert key not in seen
                seen.add(key)
                dec = o.decode_adaptive_n(enc["words"], enc["states"], k, 3, N=N)
                assert tuple(dec["symbols"]) == msg


def pin_adaptive_n_size(o):
    """The coded size stays within the derived per-symbol bound (reading 13)
    around the information content of the models the contexts give; on data
    the models can learn (a skewed source with a burst of one symbol) it is
    well below log2 n bits per symbol."""
    rng = np.random.default_rng(53)
    n, N = 8, 4
    p = np.array([0.6, 0.2, 0.1, 0.05, 0.02, 0.01, 0.01, 0.01])
    msg = rng.choice(n, size=8000, p=p).astype(np.uint32)
    msg[3000:5000] = 2
    info = 0.0
    for j in range(N):
        sub = msg[j::N]
        tr = o.adaptive_n_trace(sub, n)
        f = tr[np.arange(sub.size), sub + 1] - tr[np.arange(sub.size), sub]
        info += float(np.sum(np.log2(M12 / f)))
    enc = o.encode_adaptive_n(msg, n, N=N)
    W = enc["words"].size
    bits = 16 * W + sum(math.log2(int(x) / L16) for x in enc["states"])
    lo = info + msg.size * math.log2(15 / 16) - W * math.log2(17 / 16) - 1e-6
    hi = info + msg.size * math.log2(17 / 16) + 1e-6
    assert lo <= bits <= hi, (lo, bits, hi)
    assert bits / msg.size < 0.75 * math.log2(n)


def pin_adaptive_n_container(o):
    rng = np.random.default_rng(59)
    msg = rng.integers(0, 11, size=5000).astype(np.uint8)
    m = o.encode_message_adaptive_n(msg, 11, N=7, chunk_symbols=999)
    h = m[:32].view(np.uint32)
    assert int(h[1]) == 6 and int(h[3]) == 12 | (11 << 16)
    assert np.array_equal(o.decode_message_adaptive_n(m, msg.size, 11, N=7, chunk_symbols=999),
                          msg)
    data0 = (32 + 4 * 7 + 15) // 16 * 16
    offs = m[32:32 + 4 * 7].view(np.uint32)
    enc = o.encode_adaptive_n(msg[:999].astype(np.uint32), 11, N=7)
    ch = m[data0 + offs[0]:data0 + offs[1]]
    assert list(ch[:28].view(np.uint32)) == list(enc["states"])
    assert list(ch[28:].view(np.uint16)) == list(enc["words"])


# ----------------------------------------------------------------------------
# Section 4: interleaving arbitrary coders by running an instrumented decoder
# ----------------------------------------------------------------------------

RFC1951 = read_golden("rfc1951_canonical_codes.txt")


def pin_mux_rans_is_section3_interleaving(o):
    """Section 4 applied to rANS: N coders each encode their own symbols
    into their own buffer; the instrumented decoders' mux of those buffers
    is exactly the interleaved stream Section 3's encoder writes directly
    (the production chunk, and the paper's own L = 16, b = 2 model), and it
    decodes back."""
    rng = np.random.default_rng(41)
    for alpha, n, N in ((6, 700, 1), (6, 700, 2), (40, 2000, 5), (3, 901, 32)):
        freq = o.quantize(rng.integers(1, 1000, size=alpha).astype(np.uint64))
        sym = rng.choice(alpha, size=n, p=freq / freq.sum()).astype(np.uint8)
        words = o.mux_rans(sym, freq.astype(np.uint64), N)
        chunk = o.encode_chunk(sym, freq, N=N)
        assert np.array_equal(words.astype(np.uint16).view(np.uint8), chunk), (alpha, N)
        assert np.array_equal(o.demux_rans(words, n, freq.astype(np.uint64), N), sym)
    # the paper's model, two coders: state digits (5 binary digits each, low
    # first, coder 0 then coder 1), then the interleaved words
    msg = [PAPER_SYM[c] for c in "babbaabbbabbab"]
    enc = o.encode(PAPER_FREQ, msg, N=2, L=16, b=2)
    digits = [(int(x) >> k) & 1 for x in enc["states"] for k in range(5)]
    words = o.mux_rans(msg, np.array(PAPER_FREQ, dtype=np.uint64), 2, L=16, b=2)
    assert list(words) == digits + [int(w) for w in enc["words"]]


def pin_prefix_codes_rfc1951(o):
    """Canonical codes: the RFC 1951 worked example (golden file), and for
    random length vectors the prefix property and Kraft's inequality."""
    lengths = np.array([int(v) for v in RFC1951["lengths"]], dtype=np.uint8)
    want = [int(c, 2) for c in RFC1951["codes"]]
    assert list(o.prefix_codes(lengths)) == want
    rng = np.random.default_rng(43)
    for _ in range(30):
        n = int(rng.integers(2, 40))
        w = rng.integers(1, 1 << 20, size=n).astype(np.uint64)
        ln = o.prefix_lengths(w, 12)
        codes = o.prefix_codes(ln)
        words = [format(int(c), "b").zfill(int(l)) for c, l in zip(codes, ln)]
        for a in range(n):
            for b in range(n):
                if a != b:
                    assert not words[b].startswith(words[a])
    bad = np.array([1, 1, 1], dtype=np.uint8)          # Kraft sum 3/2
    try:
        o.prefix_codes(bad)
        raise AssertionError("over-full code accepted")
    except oracle.OracleError:
        pass


def _huffman_cost(w):
    """Textbook Huffman (repeatedly merge the two lightest): total cost."""
    import heapq
    h = [int(x) for x in w if x]
    if len(h) == 1:
        return h[0]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def pin_prefix_lengths_optimal(o):
    """Package-merge lengths: optimal among all codes with lengths <= the
    limit (brute force on small alphabets), a complete code (Kraft sum 1),
    heavier symbols never longer, and without a binding limit the cost of a
    textbook Huffman code."""
    rng = np.random.default_rng(47)
    for n, lim in ((2, 1), (3, 2), (4, 2), (5, 3), (6, 3), (6, 4), (7, 3), (7, 5)):
        for _ in range(12):
            w = rng.integers(1, 60, size=n).astype(np.uint64)
            if rng.random() < 0.3:
                w = (2 ** rng.integers(0, 12, size=n)).astype(np.uint64)  # skewed
            ln = o.prefix_lengths(w, lim)
            assert ln.max() <= lim and ln.min() >= 1
            assert sum(2.0 ** -int(l) for l in ln) == 1.0
            best = min(sum(int(a) * b for a, b in zip(w, ls))
                       for ls in itertools.product(range(1, lim + 1), repeat=n)
                       if sum(2.0 ** -b for b in ls) <= 1.0)
            assert sum(int(a) * int(b) for a, b in zip(w, ln)) == best, (w, lim, ln)
            for a in range(n):
                for b in range(n):
                    if w[a] > w[b]:
                        assert ln[a] <= ln[b]
    for _ in range(20):
        n = int(rng.integers(2, 200))
        w = rng.integers(1, 1000, size=n).astype(np.uint64)
        w[rng.random(n) < 0.2] = 0                      # unused symbols get length 0
        if np.count_nonzero(w) < 2:
            continue
        ln = o.prefix_lengths(w, 16)
        assert all((ln[i] == 0) == (w[i] == 0) for i in range(n))
        assert sum(int(a) * int(b) for a, b in zip(w, ln)) == _huffman_cost(w)


def _schedule(o, sym, lengths, N):
    """Bit-length bookkeeping of the prefix decoder's reads (it takes a word
    whenever it holds fewer than 12 bits before a symbol): the (step, lane)
    of every read, in read order."""
    held = [0] * N
    reads = []
    for i, s in enumerate(sym):
        j = i % N
        if held[j] < 12:
            reads.append(j)
            held[j] += 32
        held[j] -= int(lengths[s])
    return reads


def pin_prefix_mux_lane_streams(o):
    """Split the prefix-code mux by the reading coder (schedule from bit
    counts): coder j's words, in order, are its own symbols' codes
    concatenated MSB first, zero-padded -- every word the receiver needs and
    nothing else -- and the mux decodes back."""
    rng = np.random.default_rng(53)
    for n_alpha, n, N in ((2, 300, 1), (5, 999, 3), (17, 4000, 8), (60, 3001, 32)):
        w = rng.integers(1, 5000, size=n_alpha).astype(np.uint64)
        ln = o.prefix_lengths(w, 12)
        codes = o.prefix_codes(ln)
        sym = rng.choice(n_alpha, size=n, p=w / w.sum()).astype(np.uint8)
        mux = o.mux_prefix(sym, ln, N)
        reads = _schedule(o, sym, ln, N)
        assert mux.size == len(reads)
        for j in range(N):
            mine = [int(x) for x, r in zip(mux, reads) if r == j]
            bits = "".join(format(int(codes[s]), "b").zfill(int(ln[s])) for s in sym[j::N])
            bits = bits.ljust(32 * len(mine), "0")
            assert mine == [int(bits[32 * k:32 * k + 32], 2) for k in range(len(mine))], (N, j)
        assert np.array_equal(o.demux_prefix(mux, n, ln, N), sym)


def pin_prefix_mux_brute_force(o):
    """All messages of up to 6 symbols over a 3-symbol code, 1..3 coders:
    distinct messages give distinct muxes, and each decodes back."""
    ln = np.array([1, 2, 2], dtype=np.uint8)
    for N in (1, 2, 3):
        seen = {}
        for n in range(0, 7):
            for msg in itertools.product(range(3), repeat=n):
                m = np.array(msg, dtype=np.uint8)
                mux = tuple(int(x) for x in o.mux_prefix(m, ln, N))
                assert (n, mux) not in seen
                seen[(n, mux)] = msg
                assert tuple(o.demux_prefix(np.array(mux, dtype=np.uint32), n, ln, N)) == msg


def pin_mux_coroutine_and_flush(o):
    """Section 4's catch: coder 0 takes the first symbol and coder 1 all the
    rest; a coroutine mux then waits on coder 0 until it flushes, so nearly
    every word is buffered.  Flushing every F symbols bounds the buffer
    (about F symbols' words) at a small cost in size; with coders taking
    symbols in turn the buffer stays at a few words per coder."""
    rng = np.random.default_rng(59)
    ln = np.array([2, 3, 3, 2, 4, 4, 3], dtype=np.uint8)      # Kraft sum 1
    n = 30_000
    sym = rng.integers(0, 7, size=n).astype(np.uint8)
    lane = np.ones(n, dtype=np.uint32)
    lane[0] = 0
    peak, total = o.mux_prefix_peak(sym, ln, 2, lane, 0)
    assert peak >= 0.95 * total
    for F in (500, 3000):
        pk, tot = o.mux_prefix_peak(sym, ln, 2, lane, F)
        assert pk <= F * 4 // 32 + 8, (F, pk)
        assert total <= tot <= total + 2 * 3 * (n // F + 1)
    for N in (2, 7, 32):
        pk, tot = o.mux_prefix_peak(sym, ln, N, None, 0)
        assert pk <= 3 * N, (N, pk)
        assert tot == o.mux_prefix(sym, ln, N).size


def pin_prefix_container(o):
    """Version-5 container: chunk c is the mux of its symbols (coder i mod N),
    u32 little-endian words; round trip."""
    rng = np.random.default_rng(61)
    w = rng.integers(1, 100, size=30).astype(np.uint64)
    ln = o.prefix_lengths(w, 12)
    sym = rng.choice(30, size=5000, p=w / w.sum()).astype(np.uint8)
    m = o.encode_message_prefix(sym, ln, N=7, chunk_symbols=999)
    h = m[:32].view(np.uint32)
    assert list(h[:4]) == [0x534E4152, 5, 7, 12] and list(h[6:8]) == [999, 6]
    data0 = (32 + 4 * 7 + 15) // 16 * 16
    offs = m[32:32 + 4 * 7].view(np.uint32)
    for c in range(6):
        ch = m[data0 + offs[c]:data0 + offs[c + 1]]
        assert list(ch.view(np.uint32)) == list(o.mux_prefix(sym[999 * c:999 * (c + 1)], ln, 7))
    assert np.array_equal(o.decode_message_prefix(m, sym.size, ln, N=7, chunk_symbols=999), sym)


def pin_wide_resolution(o):
    """Section 5: with b = 2^16 a coder in 32-bit integers keeps one
    renormalization per symbol at 12-14 bits of probability resolution.  For
    M = 2^13 and 2^14 (the table's sum): no symbol needs more than one
    renormalization, each container chunk is the generic Algorithm-1 coder's
    stream at the production L and b, the header records log2(M), messages
    decode back, and a table of any other sum is refused (as is a wide table
    by the byte-wise container, which keeps M = 2^12)."""
    rng = np.random.default_rng(67)
    for lm in (13, 14):
        for alpha in (2, 40, 256):
            w = rng.integers(1, 1 << 20, size=alpha).astype(np.uint64)
            freq = o.quantize(w, lm)
            assert int(freq.astype(np.int64).sum()) == 1 << lm
            sym = rng.integers(0, alpha, size=3000).astype(np.uint8)   # rare symbols too
            for N in (1, 7, 32):
                enc = o.encode(freq.astype(np.uint64), sym, N=N)
                assert enc["max_iters"] <= 1
                ref = np.concatenate([enc["states"].astype("<u4").view(np.uint8),
                                      enc["words"].astype("<u2").view(np.uint8)])
                assert np.array_equal(o.encode_chunk(sym, freq, N=N), ref), (lm, alpha, N)
            m = o.encode_message(sym, freq, N=7, chunk_symbols=999)
            assert int.from_bytes(m[12:16].tobytes(), "little") == lm
            assert np.array_equal(o.decode_message(m, sym.size, freq, N=7, chunk_symbols=999), sym)
    sym = rng.integers(0, 256, size=100).astype(np.uint8)
    for bad in (np.full(256, 128, dtype=np.uint16),                 # sum 2^15
                np.full(256, 24, dtype=np.uint16)):                 # sum 6144
        try:
            o.encode_message(sym, bad, N=32, chunk_symbols=64)
            raise AssertionError("a table of sum %d was accepted" % int(bad.sum()))
        except oracle.OracleError:
            pass
    wide = o.quantize(np.ones(256, dtype=np.uint64), 14)
    try:
        o.encode_message_bytes(sym, wide, N=32, chunk_symbols=64)
        raise AssertionError("the byte-wise container took M = 2^14")
    except oracle.OracleError:
        pass


ALL_PINS = [
    pin_paper_C_D, pin_paper_precursor_sets, pin_paper_state_30, pin_paper_lockstep,
    pin_lockstep_interleaved, pin_inverse_exhaustive, pin_precursor_rans_b_unique,
    pin_one_renorm_production, pin_uniform_closed_form, pin_single_symbol,
    pin_infinite_precision_paper, pin_infinite_precision_general, pin_size_bound,
    pin_brute_force_unique, pin_packed_io_equivalence, pin_round_trip_edges,
    pin_container_layout, pin_quantize, pin_bypass_paper_example,
    pin_bypass_without_raw_is_plain, pin_bypass_interleaved, pin_wide_one_lane_is_algorithm1,
    pin_wide_breadth_first, pin_bytes_container, pin_adaptive_lanes_independent,
    pin_adaptive_brute_force, pin_adaptive_size_and_learning, pin_adaptive_container,
    pin_mux_rans_is_section3_interleaving, pin_prefix_codes_rfc1951, pin_prefix_lengths_optimal,
    pin_prefix_mux_lane_streams, pin_prefix_mux_brute_force, pin_mux_coroutine_and_flush,
    pin_prefix_container, pin_wide_resolution, pin_adaptive_n_worked_example,
    pin_adaptive_n_invariants, pin_adaptive_n_static_limit, pin_adaptive_n_lanes_independent,
    pin_adaptive_n_brute_force, pin_adaptive_n_size, pin_adaptive_n_container,
]
