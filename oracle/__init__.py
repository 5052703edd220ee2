"""CPU oracle for interleaved streaming rANS -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The product package
(``paper_1402_3392_b300``) never imports it, and the two share no code.

The arithmetic lives in ``rans_oracle.c`` (plain scalar C, Algorithm 1 of
Giesen, "Interleaved entropy coders", run by N round-robin coders, Section 3)
and ``mux_oracle.c`` (Section 4: interleaving arbitrary coders by running an
instrumented decoder, with rANS and a canonical prefix code as the coders).
This module compiles both with gcc on first use and wraps them with ctypes.

``load(mutant=k)`` builds a copy with one planted mistake (k >= 1); the pin
tests use those copies to show that each plausible mistake is caught.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "rans_oracle.c"), os.path.join(_HERE, "mux_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, C.CDLL] = {}

# Oracle status codes (its own, independent of the library's).
OK, ERR_ARG, ERR_SYMBOL, ERR_SPACE, ERR_CORRUPT, ERR_INVARIANT = range(6)

# Production parameters of the container (readings of the paper, Section 5).
L_PROD = 1 << 16
B_PROD = 1 << 16
LOG2_M_PROD = 12
M_PROD = 1 << LOG2_M_PROD

_u64p = C.POINTER(C.c_uint64)
_u32p = C.POINTER(C.c_uint32)
_u16p = C.POINTER(C.c_uint16)
_u8p = C.POINTER(C.c_uint8)


def lib_path(mutant: int = 0) -> str:
    name = "librans_oracle.so" if mutant == 0 else f"librans_oracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (gcc -O2) into oracle/_build/ and return the path."""
    out = lib_path(mutant)
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(out) >= os.path.getmtime(src) for src in _SRCS)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-Wall", "-Wextra", "-shared", "-fPIC",
           f"-DORACLE_MUTANT={mutant}", "-o", tmp, *_SRCS]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutant: int = 0) -> C.CDLL:
    with _LOCK:
        if mutant in _LIBS:
            return _LIBS[mutant]
        lib = C.CDLL(build(mutant))
        lib.orc_encode.argtypes = [_u64p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32,
                                   _u32p, C.c_uint64, _u64p, C.c_uint64, _u64p, _u64p,
                                   _u64p, _u32p, C.c_uint64, _u64p, _u32p]
        lib.orc_encode.restype = C.c_int
        lib.orc_decode.argtypes = [_u64p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32,
                                   _u64p, C.c_uint64, _u64p, C.c_uint64, _u32p, _u64p, _u64p,
                                   _u64p, _u32p, C.c_uint64, _u64p, _u32p]
        lib.orc_decode.restype = C.c_int
        lib.orc_C.argtypes = [_u64p, C.c_uint32, C.c_uint32, C.c_uint64, C.POINTER(C.c_int)]
        lib.orc_C.restype = C.c_uint64
        lib.orc_D.argtypes = [_u64p, C.c_uint32, C.c_uint64, _u32p, C.POINTER(C.c_int)]
        lib.orc_D.restype = C.c_uint64
        lib.orc_max_message_size.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        lib.orc_max_message_size.restype = C.c_uint64
        lib.orc_encode_chunk.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                         _u8p, C.c_uint64, _u64p]
        lib.orc_encode_chunk.restype = C.c_int
        lib.orc_decode_chunk.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                         _u8p, C.c_uint64]
        lib.orc_decode_chunk.restype = C.c_int
        lib.orc_encode_message.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                           C.c_uint32, _u8p, C.c_uint64, _u64p]
        lib.orc_encode_message.restype = C.c_int
        lib.orc_decode_message.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                           C.c_uint32, _u8p, C.c_uint64]
        lib.orc_decode_message.restype = C.c_int
        lib.orc_quantize.argtypes = [_u64p, C.c_uint32, C.c_uint32, _u16p]
        lib.orc_quantize.restype = C.c_int
        lib.orc_encode_bypass.argtypes = [_u64p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32,
                                          _u32p, C.c_uint64, _u32p, _u64p, C.c_uint64, _u64p,
                                          C.c_uint64, _u64p, _u64p, _u64p, _u32p, C.c_uint64,
                                          _u64p]
        lib.orc_encode_bypass.restype = C.c_int
        lib.orc_decode_bypass.argtypes = [_u64p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32,
                                          _u64p, C.c_uint64, _u64p, C.c_uint64, _u32p, _u32p,
                                          _u64p, C.c_uint64, _u64p, _u64p, _u64p, _u64p, _u32p,
                                          C.c_uint64, _u64p]
        lib.orc_decode_bypass.restype = C.c_int
        lib.orc_max_message_size_bypass.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        lib.orc_max_message_size_bypass.restype = C.c_uint64
        lib.orc_encode_chunk_bypass.argtypes = [_u8p, _u16p, C.c_uint64, _u16p, _u8p, C.c_uint32,
                                                C.c_uint32, _u8p, C.c_uint64, _u64p]
        lib.orc_encode_chunk_bypass.restype = C.c_int
        lib.orc_decode_chunk_bypass.argtypes = [_u8p, C.c_uint64, _u16p, _u8p, C.c_uint32,
                                                C.c_uint32, _u8p, _u16p, C.c_uint64]
        lib.orc_decode_chunk_bypass.restype = C.c_int
        lib.orc_encode_message_bypass.argtypes = [_u8p, _u16p, C.c_uint64, _u16p, _u8p,
                                                  C.c_uint32, C.c_uint32, C.c_uint32, _u8p,
                                                  C.c_uint64, _u64p]
        lib.orc_encode_message_bypass.restype = C.c_int
        lib.orc_decode_message_bypass.argtypes = [_u8p, C.c_uint64, _u16p, _u8p, C.c_uint32,
                                                  C.c_uint32, C.c_uint32, _u8p, _u16p,
                                                  C.c_uint64]
        lib.orc_decode_message_bypass.restype = C.c_int
        lib.orc_encode_wide.argtypes = [_u64p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32,
                                        _u32p, C.c_uint64, _u64p, C.c_uint64, _u64p, _u64p]
        lib.orc_encode_wide.restype = C.c_int
        lib.orc_decode_wide.argtypes = [_u64p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32,
                                        _u64p, C.c_uint64, _u64p, C.c_uint64, _u32p, _u64p, _u64p]
        lib.orc_decode_wide.restype = C.c_int
        lib.orc_max_message_size_bytes.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        lib.orc_max_message_size_bytes.restype = C.c_uint64
        lib.orc_encode_chunk_bytes.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                               _u8p, C.c_uint64, _u64p]
        lib.orc_encode_chunk_bytes.restype = C.c_int
        lib.orc_decode_chunk_bytes.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                               _u8p, C.c_uint64]
        lib.orc_decode_chunk_bytes.restype = C.c_int
        lib.orc_encode_message_bytes.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                                 C.c_uint32, _u8p, C.c_uint64, _u64p]
        lib.orc_encode_message_bytes.restype = C.c_int
        lib.orc_decode_message_bytes.argtypes = [_u8p, C.c_uint64, _u16p, C.c_uint32, C.c_uint32,
                                                 C.c_uint32, _u8p, C.c_uint64]
        lib.orc_decode_message_bytes.restype = C.c_int
        lib.orc_encode_adaptive.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                            C.c_uint32, C.c_uint64, _u32p, C.c_uint64, _u64p,
                                            C.c_uint64, _u64p, _u64p]
        lib.orc_encode_adaptive.restype = C.c_int
        lib.orc_decode_adaptive.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                            C.c_uint32, C.c_uint64, _u64p, C.c_uint64, _u64p,
                                            C.c_uint64, _u32p, _u64p, _u64p]
        lib.orc_decode_adaptive.restype = C.c_int
        lib.orc_encode_chunk_adaptive.argtypes = [_u8p, C.c_uint64, C.c_uint32, _u8p, C.c_uint64,
                                                  _u64p]
        lib.orc_encode_chunk_adaptive.restype = C.c_int
        lib.orc_decode_chunk_adaptive.argtypes = [_u8p, C.c_uint64, C.c_uint32, _u8p, C.c_uint64]
        lib.orc_decode_chunk_adaptive.restype = C.c_int
        lib.orc_encode_message_adaptive.argtypes = [_u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                                    _u8p, C.c_uint64, _u64p]
        lib.orc_encode_message_adaptive.restype = C.c_int
        lib.orc_decode_message_adaptive.argtypes = [_u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                                    _u8p, C.c_uint64]
        lib.orc_decode_message_adaptive.restype = C.c_int
        lib.orc_adaptive_n_trace.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, _u32p,
                                             C.c_uint64, _u64p]
        lib.orc_adaptive_n_trace.restype = C.c_int
        lib.orc_encode_adaptive_n.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                              C.c_uint32, C.c_uint32, _u32p, C.c_uint64, _u64p,
                                              C.c_uint64, _u64p, _u64p]
        lib.orc_encode_adaptive_n.restype = C.c_int
        lib.orc_decode_adaptive_n.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                              C.c_uint32, C.c_uint32, _u64p, C.c_uint64, _u64p,
                                              C.c_uint64, _u32p, _u64p, _u64p]
        lib.orc_decode_adaptive_n.restype = C.c_int
        lib.orc_encode_chunk_adaptive_n.argtypes = [_u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                                    _u8p, C.c_uint64, _u64p]
        lib.orc_encode_chunk_adaptive_n.restype = C.c_int
        lib.orc_decode_chunk_adaptive_n.argtypes = [_u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                                    _u8p, C.c_uint64]
        lib.orc_decode_chunk_adaptive_n.restype = C.c_int
        lib.orc_encode_message_adaptive_n.argtypes = [_u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                                      C.c_uint32, _u8p, C.c_uint64, _u64p]
        lib.orc_encode_message_adaptive_n.restype = C.c_int
        lib.orc_decode_message_adaptive_n.argtypes = [_u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                                      C.c_uint32, _u8p, C.c_uint64]
        lib.orc_decode_message_adaptive_n.restype = C.c_int
        # Section 4: instrumented-decoder mux (mux_oracle.c)
        lib.orc_mux_rans.argtypes = [_u32p, C.c_uint64, C.c_uint32, _u64p, C.c_uint32,
                                     C.c_uint64, C.c_uint64, _u64p, C.c_uint64, _u64p]
        lib.orc_demux_rans.argtypes = [_u64p, C.c_uint64, C.c_uint64, C.c_uint32, _u64p,
                                       C.c_uint32, C.c_uint64, C.c_uint64, _u32p]
        lib.orc_prefix_codes.argtypes = [_u8p, C.c_uint32, _u32p]
        lib.orc_prefix_lengths.argtypes = [_u64p, C.c_uint32, C.c_uint32, _u8p]
        lib.orc_mux_prefix.argtypes = [_u8p, C.c_uint64, C.c_uint32, _u32p, _u8p, C.c_uint32,
                                       _u32p, C.c_uint64, _u64p]
        lib.orc_demux_prefix.argtypes = [_u32p, C.c_uint64, C.c_uint64, C.c_uint32, _u32p, _u8p,
                                         C.c_uint32, _u8p]
        lib.orc_mux_prefix_peak.argtypes = [_u8p, C.c_uint64, C.c_uint32, _u32p, _u8p,
                                            C.c_uint32, C.c_uint64, _u64p, _u64p]
        lib.orc_max_message_size_prefix.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        lib.orc_max_message_size_prefix.restype = C.c_uint64
        lib.orc_encode_chunk_prefix.argtypes = [_u8p, C.c_uint64, _u8p, C.c_uint32, C.c_uint32,
                                                _u8p, C.c_uint64, _u64p]
        lib.orc_decode_chunk_prefix.argtypes = [_u8p, C.c_uint64, _u8p, C.c_uint32, C.c_uint32,
                                                _u8p, C.c_uint64]
        lib.orc_encode_message_prefix.argtypes = [_u8p, C.c_uint64, _u8p, C.c_uint32,
                                                  C.c_uint32, C.c_uint32, _u8p, C.c_uint64,
                                                  _u64p]
        lib.orc_decode_message_prefix.argtypes = [_u8p, C.c_uint64, _u8p, C.c_uint32,
                                                  C.c_uint32, C.c_uint32, _u8p, C.c_uint64]
        for fn in ("orc_mux_rans", "orc_demux_rans", "orc_prefix_codes", "orc_prefix_lengths",
                   "orc_mux_prefix", "orc_demux_prefix", "orc_mux_prefix_peak",
                   "orc_encode_chunk_prefix", "orc_decode_chunk_prefix",
                   "orc_encode_message_prefix", "orc_decode_message_prefix"):
            getattr(lib, fn).restype = C.c_int
        _LIBS[mutant] = lib
        return lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class Oracle:
    """ctypes front end of one build of the oracle (mutant 0 = the real one)."""

    def __init__(self, mutant: int = 0):
        self.mutant = mutant
        self.lib = load(mutant)

    # -- generic coder (any L, b, M; words are base-b digits) ----------------
    def encode(self, freq, symbols, N=1, L=L_PROD, b=B_PROD, trace=False):
        """Algorithm 1 encoder, N interleaved coders.

        Returns dict(words, states, max_iters[, trace_state, trace_lane]).
        ``words`` is in decoder read order."""
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        n = s.size
        cap = max(1, 64 * n + 64)
        words = np.zeros(cap, dtype=np.uint64)
        states = np.zeros(N, dtype=np.uint64)
        nw = C.c_uint64(0)
        it = C.c_uint32(0)
        tcap = (64 * n + N + 64) if trace else 0
        ts = np.zeros(max(tcap, 1), dtype=np.uint64)
        tl = np.zeros(max(tcap, 1), dtype=np.uint32)
        nt = C.c_uint64(0)
        rc = self.lib.orc_encode(_p(f, _u64p), f.size, L, b, N, _p(s, _u32p), n,
                                 _p(words, _u64p), cap, C.byref(nw), _p(states, _u64p),
                                 _p(ts, _u64p) if trace else None,
                                 _p(tl, _u32p) if trace else None, tcap,
                                 C.byref(nt), C.byref(it))
        if rc != OK:
            raise OracleError(rc, "encode")
        out = dict(words=words[: nw.value].copy(), states=states, max_iters=it.value)
        if trace:
            assert nt.value <= tcap
            out["trace_state"] = ts[: nt.value].copy()
            out["trace_lane"] = tl[: nt.value].copy()
        return out

    def decode(self, freq, words, states, n_sym, N=1, L=L_PROD, b=B_PROD, trace=False):
        """Algorithm 1 decoder, N interleaved coders reading one buffer.

        Returns dict(symbols, consumed, states_end, max_iters[, trace...])."""
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        w = np.ascontiguousarray(words, dtype=np.uint64)
        st = np.ascontiguousarray(states, dtype=np.uint64)
        assert st.size == N
        sym = np.zeros(max(1, n_sym), dtype=np.uint32)
        st_end = np.zeros(N, dtype=np.uint64)
        used = C.c_uint64(0)
        it = C.c_uint32(0)
        tcap = (64 * n_sym + N + 64) if trace else 0
        ts = np.zeros(max(tcap, 1), dtype=np.uint64)
        tl = np.zeros(max(tcap, 1), dtype=np.uint32)
        nt = C.c_uint64(0)
        rc = self.lib.orc_decode(_p(f, _u64p), f.size, L, b, N, _p(w, _u64p), w.size,
                                 _p(st, _u64p), n_sym, _p(sym, _u32p), C.byref(used),
                                 _p(st_end, _u64p),
                                 _p(ts, _u64p) if trace else None,
                                 _p(tl, _u32p) if trace else None, tcap,
                                 C.byref(nt), C.byref(it))
        if rc != OK:
            raise OracleError(rc, "decode")
        out = dict(symbols=sym[:n_sym].copy(), consumed=used.value, states_end=st_end,
                   max_iters=it.value)
        if trace:
            out["trace_state"] = ts[: nt.value].copy()
            out["trace_lane"] = tl[: nt.value].copy()
        return out

    def C(self, freq, s, x):
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        ok = C.c_int(0)
        r = self.lib.orc_C(_p(f, _u64p), f.size, s, x, C.byref(ok))
        if not ok.value:
            raise OracleError(ERR_ARG, "C")
        return int(r)

    def D(self, freq, x):
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        ok = C.c_int(0)
        s = C.c_uint32(0)
        r = self.lib.orc_D(_p(f, _u64p), f.size, x, C.byref(s), C.byref(ok))
        if not ok.value:
            raise OracleError(ERR_ARG, "D")
        return int(s.value), int(r)

    # -- production container (L = b = 2^16, M = 2^12, u16 words) -----------
    def max_message_size(self, n_sym, N, chunk_symbols):
        return int(self.lib.orc_max_message_size(n_sym, N, chunk_symbols))

    def encode_message(self, symbols, freq, N=32, chunk_symbols=65536):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        cap = self.max_message_size(s.size, N, chunk_symbols)
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_message(_p(s, _u8p), s.size, _p(fr, _u16p), fr.size, N,
                                         chunk_symbols, _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_message")
        return out[: size.value].copy()

    def decode_message(self, msg, n_sym, freq, N=32, chunk_symbols=65536):
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_message(_p(m, _u8p), m.size, _p(fr, _u16p), fr.size, N,
                                         chunk_symbols, _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_message")
        return out[:n_sym].copy()

    def encode_chunk(self, symbols, freq, N=32):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        cap = 4 * N + 2 * s.size
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_chunk(_p(s, _u8p), s.size, _p(fr, _u16p), fr.size, N,
                                       _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_chunk")
        return out[: size.value].copy()

    def decode_chunk(self, chunk, n_sym, freq, N=32):
        c = np.ascontiguousarray(chunk, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_chunk(_p(c, _u8p), c.size, _p(fr, _u16p), fr.size, N,
                                       _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_chunk")
        return out[:n_sym].copy()

    # -- bypass: raw digits interleaved with the coded symbols (Section 3) ----
    def encode_bypass(self, freq, symbols, raw_counts, raw, N=1, L=L_PROD, b=B_PROD,
                      trace=False):
        """Algorithm 1 encoder where symbol s carries raw_counts[s] raw base-b
        digits; raw holds them in message order.  Returns dict(words, states
        [, trace_state, trace_lane])."""
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        r = np.ascontiguousarray(raw_counts, dtype=np.uint32)
        rw = np.ascontiguousarray(raw, dtype=np.uint64)
        n = s.size
        cap = max(1, 64 * n + rw.size + 64)
        words = np.zeros(cap, dtype=np.uint64)
        states = np.zeros(N, dtype=np.uint64)
        nw = C.c_uint64(0)
        tcap = (64 * n + N + 64) if trace else 0
        ts = np.zeros(max(tcap, 1), dtype=np.uint64)
        tl = np.zeros(max(tcap, 1), dtype=np.uint32)
        nt = C.c_uint64(0)
        rc = self.lib.orc_encode_bypass(_p(f, _u64p), f.size, L, b, N, _p(s, _u32p), n,
                                        _p(r, _u32p), _p(rw, _u64p) if rw.size else None, rw.size,
                                        _p(words, _u64p), cap, C.byref(nw), _p(states, _u64p),
                                        _p(ts, _u64p) if trace else None,
                                        _p(tl, _u32p) if trace else None, tcap, C.byref(nt))
        if rc != OK:
            raise OracleError(rc, "encode_bypass")
        out = dict(words=words[: nw.value].copy(), states=states)
        if trace:
            out["trace_state"] = ts[: nt.value].copy()
            out["trace_lane"] = tl[: nt.value].copy()
        return out

    def decode_bypass(self, freq, words, states, n_sym, raw_counts, N=1, L=L_PROD, b=B_PROD,
                      trace=False):
        """Decoder reading raw_counts[s] raw digits after each symbol s.
        Returns dict(symbols, raw, consumed, states_end[, trace...])."""
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        w = np.ascontiguousarray(words, dtype=np.uint64)
        st = np.ascontiguousarray(states, dtype=np.uint64)
        r = np.ascontiguousarray(raw_counts, dtype=np.uint32)
        sym = np.zeros(max(1, n_sym), dtype=np.uint32)
        rcap = max(1, w.size)
        raw = np.zeros(rcap, dtype=np.uint64)
        nraw = C.c_uint64(0)
        st_end = np.zeros(N, dtype=np.uint64)
        used = C.c_uint64(0)
        tcap = (64 * n_sym + N + 64) if trace else 0
        ts = np.zeros(max(tcap, 1), dtype=np.uint64)
        tl = np.zeros(max(tcap, 1), dtype=np.uint32)
        nt = C.c_uint64(0)
        rc = self.lib.orc_decode_bypass(_p(f, _u64p), f.size, L, b, N, _p(w, _u64p), w.size,
                                        _p(st, _u64p), n_sym, _p(r, _u32p), _p(sym, _u32p),
                                        _p(raw, _u64p), rcap, C.byref(nraw), C.byref(used),
                                        _p(st_end, _u64p),
                                        _p(ts, _u64p) if trace else None,
                                        _p(tl, _u32p) if trace else None, tcap, C.byref(nt))
        if rc != OK:
            raise OracleError(rc, "decode_bypass")
        out = dict(symbols=sym[:n_sym].copy(), raw=raw[: nraw.value].copy(),
                   consumed=used.value, states_end=st_end)
        if trace:
            out["trace_state"] = ts[: nt.value].copy()
            out["trace_lane"] = tl[: nt.value].copy()
        return out

    def max_message_size_bypass(self, n_sym, N, chunk_symbols):
        return int(self.lib.orc_max_message_size_bypass(n_sym, N, chunk_symbols))

    def encode_message_bypass(self, symbols, raw16, freq, raw_words, N=32, chunk_symbols=65536):
        """Bypass message: symbol i is followed by raw16[i] when
        raw_words[symbols[i]] == 1."""
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        rw = np.ascontiguousarray(raw16, dtype=np.uint16)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        rf = np.ascontiguousarray(raw_words, dtype=np.uint8)
        assert rw.size == s.size and rf.size == fr.size
        cap = self.max_message_size_bypass(s.size, N, chunk_symbols)
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_message_bypass(_p(s, _u8p), _p(rw, _u16p), s.size,
                                                _p(fr, _u16p), _p(rf, _u8p), fr.size, N,
                                                chunk_symbols, _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_message_bypass")
        return out[: size.value].copy()

    def decode_message_bypass(self, msg, n_sym, freq, raw_words, N=32, chunk_symbols=65536):
        """Returns (symbols, raw16) with raw16[i] = 0 where symbol i has none."""
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        rf = np.ascontiguousarray(raw_words, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        raw = np.zeros(max(1, n_sym), dtype=np.uint16)
        rc = self.lib.orc_decode_message_bypass(_p(m, _u8p), m.size, _p(fr, _u16p),
                                                _p(rf, _u8p), fr.size, N, chunk_symbols,
                                                _p(out, _u8p), _p(raw, _u16p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_message_bypass")
        return out[:n_sym].copy(), raw[:n_sym].copy()

    def encode_chunk_bypass(self, symbols, raw16, freq, raw_words, N=32):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        rw = np.ascontiguousarray(raw16, dtype=np.uint16)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        rf = np.ascontiguousarray(raw_words, dtype=np.uint8)
        cap = 4 * N + 4 * s.size
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_chunk_bypass(_p(s, _u8p), _p(rw, _u16p), s.size, _p(fr, _u16p),
                                              _p(rf, _u8p), fr.size, N, _p(out, _u8p), cap,
                                              C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_chunk_bypass")
        return out[: size.value].copy()

    def decode_chunk_bypass(self, chunk, n_sym, freq, raw_words, N=32):
        c = np.ascontiguousarray(chunk, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        rf = np.ascontiguousarray(raw_words, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        raw = np.zeros(max(1, n_sym), dtype=np.uint16)
        rc = self.lib.orc_decode_chunk_bypass(_p(c, _u8p), c.size, _p(fr, _u16p), _p(rf, _u8p),
                                              fr.size, N, _p(out, _u8p), _p(raw, _u16p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_chunk_bypass")
        return out[:n_sym].copy(), raw[:n_sym].copy()

    # -- width-baked interleaving: digits read breadth-first per step (Section 5)
    def encode_wide(self, freq, symbols, N=1, L=L_PROD, b=B_PROD):
        """Returns dict(words, states); words in decoder read order."""
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        cap = max(1, 64 * s.size + 64)
        words = np.zeros(cap, dtype=np.uint64)
        states = np.zeros(N, dtype=np.uint64)
        nw = C.c_uint64(0)
        rc = self.lib.orc_encode_wide(_p(f, _u64p), f.size, L, b, N, _p(s, _u32p), s.size,
                                      _p(words, _u64p), cap, C.byref(nw), _p(states, _u64p))
        if rc != OK:
            raise OracleError(rc, "encode_wide")
        return dict(words=words[: nw.value].copy(), states=states)

    def decode_wide(self, freq, words, states, n_sym, N=1, L=L_PROD, b=B_PROD):
        """Returns dict(symbols, consumed, states_end)."""
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        w = np.ascontiguousarray(words, dtype=np.uint64)
        st = np.ascontiguousarray(states, dtype=np.uint64)
        sym = np.zeros(max(1, n_sym), dtype=np.uint32)
        st_end = np.zeros(N, dtype=np.uint64)
        used = C.c_uint64(0)
        rc = self.lib.orc_decode_wide(_p(f, _u64p), f.size, L, b, N, _p(w, _u64p), w.size,
                                      _p(st, _u64p), n_sym, _p(sym, _u32p), C.byref(used),
                                      _p(st_end, _u64p))
        if rc != OK:
            raise OracleError(rc, "decode_wide")
        return dict(symbols=sym[:n_sym].copy(), consumed=used.value, states_end=st_end)

    def max_message_size_bytes(self, n_sym, N, chunk_symbols):
        return int(self.lib.orc_max_message_size_bytes(n_sym, N, chunk_symbols))

    def encode_message_bytes(self, symbols, freq, N=32, chunk_symbols=65536):
        """Byte-wise (version 3) message: L = 2^23, b = 2^8, digits breadth-first."""
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        cap = self.max_message_size_bytes(s.size, N, chunk_symbols)
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_message_bytes(_p(s, _u8p), s.size, _p(fr, _u16p), fr.size, N,
                                               chunk_symbols, _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_message_bytes")
        return out[: size.value].copy()

    def decode_message_bytes(self, msg, n_sym, freq, N=32, chunk_symbols=65536):
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_message_bytes(_p(m, _u8p), m.size, _p(fr, _u16p), fr.size, N,
                                               chunk_symbols, _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_message_bytes")
        return out[:n_sym].copy()

    def encode_chunk_bytes(self, symbols, freq, N=32):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        cap = 4 * N + 2 * s.size + 8
        out = np.zeros(cap, dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_chunk_bytes(_p(s, _u8p), s.size, _p(fr, _u16p), fr.size, N,
                                             _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_chunk_bytes")
        return out[: size.value].copy()

    def decode_chunk_bytes(self, chunk, n_sym, freq, N=32):
        c = np.ascontiguousarray(chunk, dtype=np.uint8)
        fr = np.ascontiguousarray(freq, dtype=np.uint16)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_chunk_bytes(_p(c, _u8p), c.size, _p(fr, _u16p), fr.size, N,
                                             _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_chunk_bytes")
        return out[:n_sym].copy()

    # -- adaptive binary contexts, one per coder (Section 5) ---------------------
    ADAPT_RATE = 5
    ADAPT_P0 = 2048

    def encode_adaptive(self, symbols, N=1, M=1 << 12, L=L_PROD, b=B_PROD, R=5, p0=2048):
        """Binary symbols, coder j with its own adaptive probability.  Returns
        dict(words, states)."""
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        cap = max(1, 64 * s.size + 64)
        words = np.zeros(cap, dtype=np.uint64)
        states = np.zeros(N, dtype=np.uint64)
        nw = C.c_uint64(0)
        rc = self.lib.orc_encode_adaptive(M, L, b, N, R, p0, _p(s, _u32p), s.size,
                                          _p(words, _u64p), cap, C.byref(nw), _p(states, _u64p))
        if rc != OK:
            raise OracleError(rc, "encode_adaptive")
        return dict(words=words[: nw.value].copy(), states=states)

    def decode_adaptive(self, words, states, n_sym, N=1, M=1 << 12, L=L_PROD, b=B_PROD, R=5,
                        p0=2048):
        w = np.ascontiguousarray(words, dtype=np.uint64)
        st = np.ascontiguousarray(states, dtype=np.uint64)
        sym = np.zeros(max(1, n_sym), dtype=np.uint32)
        st_end = np.zeros(N, dtype=np.uint64)
        used = C.c_uint64(0)
        rc = self.lib.orc_decode_adaptive(M, L, b, N, R, p0, _p(w, _u64p), w.size, _p(st, _u64p),
                                          n_sym, _p(sym, _u32p), C.byref(used),
                                          _p(st_end, _u64p))
        if rc != OK:
            raise OracleError(rc, "decode_adaptive")
        return dict(symbols=sym[:n_sym].copy(), consumed=used.value, states_end=st_end)

    def encode_message_adaptive(self, symbols, N=32, chunk_symbols=65536):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        cap = self.max_message_size(s.size, N, chunk_symbols)
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_message_adaptive(_p(s, _u8p), s.size, N, chunk_symbols,
                                                  _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_message_adaptive")
        return out[: size.value].copy()

    def decode_message_adaptive(self, msg, n_sym, N=32, chunk_symbols=65536):
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_message_adaptive(_p(m, _u8p), m.size, N, chunk_symbols,
                                                  _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_message_adaptive")
        return out[:n_sym].copy()

    def encode_chunk_adaptive(self, symbols, N=32):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        cap = 4 * N + 2 * s.size
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_chunk_adaptive(_p(s, _u8p), s.size, N, _p(out, _u8p), cap,
                                                C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_chunk_adaptive")
        return out[: size.value].copy()

    def decode_chunk_adaptive(self, chunk, n_sym, N=32):
        c = np.ascontiguousarray(chunk, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_chunk_adaptive(_p(c, _u8p), c.size, N, _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_chunk_adaptive")
        return out[:n_sym].copy()

    # -- adaptive models over n <= 16 symbols, one per coder (Section 5) -------
    def adaptive_n_trace(self, symbols, n, M=1 << 12, R=5):
        """The cumulative frequencies of one context: row k = the model symbol
        k is coded with, row len(symbols) = the model after the last."""
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        out = np.zeros((s.size + 1) * (n + 1), dtype=np.uint64)
        rc = self.lib.orc_adaptive_n_trace(M, R, n, _p(s, _u32p), s.size, _p(out, _u64p))
        if rc != OK:
            raise OracleError(rc, "adaptive_n_trace")
        return out.reshape(s.size + 1, n + 1).astype(np.int64)

    def encode_adaptive_n(self, symbols, n, N=1, M=1 << 12, L=L_PROD, b=B_PROD, R=5):
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        cap = max(1, 64 * s.size + 64)
        words = np.zeros(cap, dtype=np.uint64)
        states = np.zeros(N, dtype=np.uint64)
        nw = C.c_uint64(0)
        rc = self.lib.orc_encode_adaptive_n(M, L, b, N, R, n, _p(s, _u32p), s.size,
                                            _p(words, _u64p), cap, C.byref(nw), _p(states, _u64p))
        if rc != OK:
            raise OracleError(rc, "encode_adaptive_n")
        return dict(words=words[: nw.value].copy(), states=states)

    def decode_adaptive_n(self, words, states, n_sym, n, N=1, M=1 << 12, L=L_PROD, b=B_PROD, R=5):
        w = np.ascontiguousarray(words, dtype=np.uint64)
        st = np.ascontiguousarray(states, dtype=np.uint64)
        sym = np.zeros(max(1, n_sym), dtype=np.uint32)
        st_end = np.zeros(N, dtype=np.uint64)
        used = C.c_uint64(0)
        rc = self.lib.orc_decode_adaptive_n(M, L, b, N, R, n, _p(w, _u64p), w.size,
                                            _p(st, _u64p), n_sym, _p(sym, _u32p), C.byref(used),
                                            _p(st_end, _u64p))
        if rc != OK:
            raise OracleError(rc, "decode_adaptive_n")
        return dict(symbols=sym[:n_sym].copy(), consumed=used.value, states_end=st_end)

    def encode_message_adaptive_n(self, symbols, n, N=32, chunk_symbols=65536):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        cap = self.max_message_size(s.size, N, chunk_symbols)
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_message_adaptive_n(_p(s, _u8p), s.size, n, N, chunk_symbols,
                                                    _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_message_adaptive_n")
        return out[: size.value].copy()

    def decode_message_adaptive_n(self, msg, n_sym, n, N=32, chunk_symbols=65536):
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_message_adaptive_n(_p(m, _u8p), m.size, n, N, chunk_symbols,
                                                    _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_message_adaptive_n")
        return out[:n_sym].copy()

    def encode_chunk_adaptive_n(self, symbols, n, N=32):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        cap = 4 * N + 2 * s.size
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_chunk_adaptive_n(_p(s, _u8p), s.size, n, N, _p(out, _u8p), cap,
                                                  C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_chunk_adaptive_n")
        return out[: size.value].copy()

    def decode_chunk_adaptive_n(self, chunk, n_sym, n, N=32):
        c = np.ascontiguousarray(chunk, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_chunk_adaptive_n(_p(c, _u8p), c.size, n, N, _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_chunk_adaptive_n")
        return out[:n_sym].copy()

    # -- Section 4: interleaving arbitrary coders by an instrumented decoder --

    def mux_rans(self, symbols, freq, N, L=L_PROD, b=B_PROD):
        """Coder j encodes symbols j, j+N, ... alone (Algorithm 1); the
        instrumented decoders mux the N buffers.  Returns the words (u64)."""
        s = np.ascontiguousarray(symbols, dtype=np.uint32)
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        cap = 64 * s.size + 8 * N + 8
        out = np.zeros(cap, dtype=np.uint64)
        n = C.c_uint64(0)
        rc = self.lib.orc_mux_rans(_p(s, _u32p), s.size, N, _p(f, _u64p), f.size, L, b,
                                   _p(out, _u64p), cap, C.byref(n))
        if rc != OK:
            raise OracleError(rc, "mux_rans")
        return out[: n.value].copy()

    def demux_rans(self, words, n_sym, freq, N, L=L_PROD, b=B_PROD):
        w = np.ascontiguousarray(words, dtype=np.uint64)
        f = np.ascontiguousarray(freq, dtype=np.uint64)
        out = np.zeros(max(1, n_sym), dtype=np.uint32)
        rc = self.lib.orc_demux_rans(_p(w, _u64p), w.size, n_sym, N, _p(f, _u64p), f.size, L, b,
                                     _p(out, _u32p))
        if rc != OK:
            raise OracleError(rc, "demux_rans")
        return out[:n_sym].copy()

    def prefix_codes(self, lengths):
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        code = np.zeros(max(1, ln.size), dtype=np.uint32)
        rc = self.lib.orc_prefix_codes(_p(ln, _u8p), ln.size, _p(code, _u32p))
        if rc != OK:
            raise OracleError(rc, "prefix_codes")
        return code[: ln.size].copy()

    def prefix_lengths(self, weights, max_len=12):
        w = np.ascontiguousarray(weights, dtype=np.uint64)
        ln = np.zeros(max(1, w.size), dtype=np.uint8)
        rc = self.lib.orc_prefix_lengths(_p(w, _u64p), w.size, max_len, _p(ln, _u8p))
        if rc != OK:
            raise OracleError(rc, "prefix_lengths")
        return ln[: w.size].copy()

    @staticmethod
    def _lanes(lane_of):
        if lane_of is None:
            return None, None
        a = np.ascontiguousarray(lane_of, dtype=np.uint32)
        return a, _p(a, _u32p)

    def mux_prefix(self, symbols, lengths, N, lane_of=None):
        """Prefix-code mux: coder lane_of[i] (i mod N) takes symbol i.
        Returns the u32 words in the receiver's read order."""
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        keep, lp = self._lanes(lane_of)
        cap = (12 * s.size) // 32 + 2 * N + 8
        out = np.zeros(cap, dtype=np.uint32)
        n = C.c_uint64(0)
        rc = self.lib.orc_mux_prefix(_p(s, _u8p), s.size, N, lp, _p(ln, _u8p), ln.size,
                                     _p(out, _u32p), cap, C.byref(n))
        del keep
        if rc != OK:
            raise OracleError(rc, "mux_prefix")
        return out[: n.value].copy()

    def demux_prefix(self, words, n_sym, lengths, N, lane_of=None):
        w = np.ascontiguousarray(words, dtype=np.uint32)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        keep, lp = self._lanes(lane_of)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_demux_prefix(_p(w, _u32p), w.size, n_sym, N, lp, _p(ln, _u8p),
                                       ln.size, _p(out, _u8p))
        del keep
        if rc != OK:
            raise OracleError(rc, "demux_prefix")
        return out[:n_sym].copy()

    def mux_prefix_peak(self, symbols, lengths, N, lane_of=None, segment=0):
        """Coroutine mux (Section 4): (peak words buffered, words output)."""
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        keep, lp = self._lanes(lane_of)
        peak, total = C.c_uint64(0), C.c_uint64(0)
        rc = self.lib.orc_mux_prefix_peak(_p(s, _u8p), s.size, N, lp, _p(ln, _u8p), ln.size,
                                          segment, C.byref(peak), C.byref(total))
        del keep
        if rc != OK:
            raise OracleError(rc, "mux_prefix_peak")
        return peak.value, total.value

    def max_message_size_prefix(self, n_sym, N, chunk_symbols):
        return int(self.lib.orc_max_message_size_prefix(n_sym, N, chunk_symbols))

    def encode_chunk_prefix(self, symbols, lengths, N=32):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        cap = 4 * ((12 * s.size + 31) // 32 + 2 * N + 1)
        out = np.zeros(cap, dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_chunk_prefix(_p(s, _u8p), s.size, _p(ln, _u8p), ln.size, N,
                                              _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_chunk_prefix")
        return out[: size.value].copy()

    def decode_chunk_prefix(self, chunk, n_sym, lengths, N=32):
        c = np.ascontiguousarray(chunk, dtype=np.uint8)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_chunk_prefix(_p(c, _u8p), c.size, _p(ln, _u8p), ln.size, N,
                                              _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_chunk_prefix")
        return out[:n_sym].copy()

    def encode_message_prefix(self, symbols, lengths, N=32, chunk_symbols=65536):
        s = np.ascontiguousarray(symbols, dtype=np.uint8)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        cap = self.max_message_size_prefix(s.size, N, chunk_symbols)
        out = np.zeros(max(cap, 1), dtype=np.uint8)
        size = C.c_uint64(0)
        rc = self.lib.orc_encode_message_prefix(_p(s, _u8p), s.size, _p(ln, _u8p), ln.size, N,
                                                chunk_symbols, _p(out, _u8p), cap, C.byref(size))
        if rc != OK:
            raise OracleError(rc, "encode_message_prefix")
        return out[: size.value].copy()

    def decode_message_prefix(self, msg, n_sym, lengths, N=32, chunk_symbols=65536):
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        ln = np.ascontiguousarray(lengths, dtype=np.uint8)
        out = np.zeros(max(1, n_sym), dtype=np.uint8)
        rc = self.lib.orc_decode_message_prefix(_p(m, _u8p), m.size, _p(ln, _u8p), ln.size, N,
                                                chunk_symbols, _p(out, _u8p), n_sym)
        if rc != OK:
            raise OracleError(rc, "decode_message_prefix")
        return out[:n_sym].copy()

    def quantize(self, weights, log2_M=LOG2_M_PROD):
        w = np.ascontiguousarray(weights, dtype=np.uint64)
        f = np.zeros(w.size, dtype=np.uint16)
        rc = self.lib.orc_quantize(_p(w, _u64p), w.size, log2_M, _p(f, _u16p))
        if rc != OK:
            raise OracleError(rc, "quantize")
        return f


_DEFAULT: Oracle | None = None


def default() -> Oracle:
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle(0)
    return _DEFAULT
