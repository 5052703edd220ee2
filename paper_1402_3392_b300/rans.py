"""Thin ctypes binding of the C ABI declared in include/rans.h.

Every function here only marshals arguments: device buffers are torch CUDA
tensors (or raw device addresses), host tables are numpy arrays, and the work
runs in the CUDA kernels of libinterleaved_rans_b300.so.  There is no CPU
fallback: if the shared library is missing the import fails with an error
that says how to build it.

Names follow the C ABI (``rans_encode`` ...).  ``encode``/``decode`` are
small conveniences that allocate the output and scratch tensors with torch
and call the same entry points.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "RansError", "RANS_OK", "RANS_ERR_INVALID_ARG", "RANS_ERR_ZERO_FREQ",
    "RANS_ERR_BUFFER_TOO_SMALL", "RANS_ERR_CORRUPT", "RANS_ERR_TIMEOUT", "RANS_ERR_CUDA",
    "RANS_ERR_OOM", "RANS_M", "RANS_L", "RANS_LOG2_M", "library_path", "lib",
    "rans_version", "rans_status_string", "rans_quantize_table", "rans_max_encoded_size",
    "rans_encode_scratch_size", "rans_encode", "rans_decode", "rans_encode_static_scratch",
    "RANS_STATIC_SCRATCH_BYTES", "encode", "decode", "STREAM_DTYPE", "ENCODE_STREAM_DTYPE",
    "rans_decode_batch_scratch_size", "rans_decode_batch", "rans_encode_batch_plan",
    "rans_encode_batch", "REQUEST_DTYPE", "RESULT_DTYPE", "RANS_REQ_ENCODE", "RANS_REQ_DECODE", "RANS_REQ_DEVICE_MEMORY",
    "Server", "rans_check_bounded_wait", "rans_check_lookback_wait", "rans_check_division", "rans_decode_host",
    "rans_decode_host_work_size", "decode_host", "rans_max_encoded_size_bypass", "rans_encode_scratch_size_bypass",
    "rans_encode_bypass", "rans_decode_bypass", "encode_bypass", "decode_bypass",
    "rans_max_encoded_size_bytes", "rans_encode_bytes", "rans_decode_bytes", "encode_bytes",
    "decode_bytes",
]

RANS_OK = 0
RANS_ERR_INVALID_ARG = 1
RANS_ERR_ZERO_FREQ = 2
RANS_ERR_BUFFER_TOO_SMALL = 3
RANS_ERR_CORRUPT = 4
RANS_ERR_TIMEOUT = 5
RANS_ERR_CUDA = 6
RANS_ERR_OOM = 7
RANS_LOG2_M = 12
RANS_M = 1 << RANS_LOG2_M
RANS_L = 1 << 16
RANS_STATIC_SCRATCH_BYTES = 64 << 20
RANS_PREFIX_MAX_LEN = 12


# Layouts of rans_stream and rans_encode_stream (include/rans.h).
STREAM_DTYPE = np.dtype([("msg", "<u8"), ("msg_size", "<u8"), ("symbols", "<u8"),
                         ("n_symbols", "<u8"), ("table", "<u4"), ("n_lanes", "<u4"),
                         ("chunk_symbols", "<u4"), ("reserved", "<u4")])
ENCODE_STREAM_DTYPE = np.dtype([("symbols", "<u8"), ("n_symbols", "<u8"), ("out", "<u8"),
                                ("out_cap", "<u8"), ("scratch_offset", "<u8"), ("table", "<u4"),
                                ("n_lanes", "<u4"), ("chunk_symbols", "<u4"),
                                ("reserved", "<u4")])
REQUEST_DTYPE = np.dtype([("kind", "<u4"), ("table", "<u4"), ("n_lanes", "<u4"),
                          ("chunk_symbols", "<u4"), ("input", "<u8"), ("input_size", "<u8"),
                          ("n_symbols", "<u8"), ("output", "<u8"), ("output_cap", "<u8"),
                          ("arrival_s", "<f8")])
RESULT_DTYPE = np.dtype([("output_size", "<u8"), ("status", "<u4"), ("batch", "<u4"),
                         ("admit_s", "<f8"), ("done_s", "<f8")])
RANS_REQ_ENCODE = 0
RANS_REQ_DECODE = 1
RANS_REQ_DEVICE_MEMORY = 0x100
assert STREAM_DTYPE.itemsize == 48 and ENCODE_STREAM_DTYPE.itemsize == 56
assert REQUEST_DTYPE.itemsize == 64 and RESULT_DTYPE.itemsize == 32


class RansParams(C.Structure):
    _fields_ = [("n_lanes", C.c_uint32), ("chunk_symbols", C.c_uint32)]


def library_path() -> str:
    """The CUDA library to load: the normal build, or with
    RANS_LIB_VARIANT=checked the checked test build (rans_debug_checks)."""
    if os.environ.get("RANS_LIB_VARIANT") == "checked":
        return _build.LIB_PATH_CHECKED
    return _build.LIB_PATH


def _load() -> C.CDLL:
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -m paper_1402_3392_b300.build); there is no CPU fallback")
    lib = C.CDLL(path)
    vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
    pp = C.POINTER(RansParams)
    sig = {
        "rans_version": (u32, []),
        "rans_status_string": (C.c_char_p, [i32]),
        "rans_quantize_table": (i32, [vp, u32, u32, vp]),
        "rans_max_encoded_size": (u64, [u64, pp]),
        "rans_encode_scratch_size": (u64, [u64, pp]),
        "rans_encode": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp]),
        "rans_encode_static_scratch": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp, vp]),
        "rans_check_bounded_wait": (i32, [vp, vp]),
        "rans_check_lookback_wait": (i32, [vp, vp]),
        "rans_check_division": (i32, [u32, u32, vp, vp]),
        "rans_check_gather_ceiling": (i32, [u32, vp, u64, vp, vp]),
        "rans_check_gather_ceiling_warps": (u64, []),
        "rans_check_cta_warps": (u32, [u64, u32, vp, u32]),
        "rans_debug_checks": (i32, [vp]),
        "rans_debug_check_selftest": (i32, [vp]),
        "rans_decode_host_work_size": (u64, [u64, u64]),
        "rans_max_encoded_size_bypass": (u64, [u64, pp]),
        "rans_encode_scratch_size_bypass": (u64, [u64, pp]),
        "rans_encode_bypass": (i32, [vp, vp, u64, vp, vp, u32, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode_bypass": (i32, [vp, u64, vp, vp, u32, pp, vp, vp, u64, vp, vp]),
        "rans_max_encoded_size_bytes": (u64, [u64, pp]),
        "rans_encode_bytes": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode_bytes": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp]),
        "rans_prefix_lengths": (i32, [vp, u32, u32, vp]),
        "rans_prefix_codes": (i32, [vp, u32, vp]),
        "rans_max_encoded_size_prefix": (u64, [u64, pp]),
        "rans_encode_scratch_size_prefix": (u64, [u64, pp]),
        "rans_encode_prefix": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode_prefix": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp]),
        "rans_encode_scratch_size_adaptive": (u64, [u64, pp]),
        "rans_encode_adaptive": (i32, [vp, u64, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode_adaptive": (i32, [vp, u64, pp, vp, u64, vp, vp]),
        "rans_encode_scratch_size_adaptive_n": (u64, [u64, pp]),
        "rans_encode_adaptive_n": (i32, [vp, u64, u32, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode_adaptive_n": (i32, [vp, u64, u32, pp, vp, u64, vp, vp]),
        "rans_decode_host": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp, u64, vp]),
        "rans_encode_host_work_size": (u64, [u64, pp]),
        "rans_encode_host": (i32, [vp, u64, vp, u32, pp, vp, u64, vp, vp, vp, u64, vp]),
        "rans_decode_batch_scratch_size": (u64, [u32]),
        "rans_decode_batch": (i32, [vp, u32, vp, u32, vp, vp, u64, vp]),
        "rans_encode_batch_plan": (u64, [vp, u32]),
        "rans_encode_batch": (i32, [vp, u32, vp, u32, vp, vp, vp, u64, vp]),
        "rans_server_create": (i32, [vp, u32, vp, u64, u32, u32, C.POINTER(vp)]),
        "rans_server_run": (i32, [vp, vp, u32, vp]),
        "rans_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class RansError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {rans_status_string(code)} ({code})")
        self.code = code


def _check(code: int, what: str) -> int:
    if code != RANS_OK:
        raise RansError(code, what)
    return code


def _ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _params(n_lanes: int, chunk_symbols: int) -> RansParams:
    return RansParams(int(n_lanes), int(chunk_symbols))


def _freq(freq) -> np.ndarray:
    return np.ascontiguousarray(freq, dtype=np.uint16)


def rans_version() -> int:
    return int(lib.rans_version())


def rans_status_string(code: int) -> str:
    return lib.rans_status_string(int(code)).decode()


def rans_quantize_table(weights, log2_M: int = RANS_LOG2_M) -> np.ndarray:
    w = np.ascontiguousarray(weights, dtype=np.uint64)
    out = np.zeros(w.size, dtype=np.uint16)
    _check(lib.rans_quantize_table(w.ctypes.data, w.size, log2_M, out.ctypes.data),
           "rans_quantize_table")
    return out


def rans_max_encoded_size(n_symbols: int, n_lanes: int = 32, chunk_symbols: int = 65536) -> int:
    p = _params(n_lanes, chunk_symbols)
    return int(lib.rans_max_encoded_size(int(n_symbols), C.byref(p)))


def rans_encode_scratch_size(n_symbols: int, n_lanes: int = 32,
                             chunk_symbols: int = 65536) -> int:
    p = _params(n_lanes, chunk_symbols)
    return int(lib.rans_encode_scratch_size(int(n_symbols), C.byref(p)))


def rans_encode(d_symbols, n_symbols, freq, n_lanes, chunk_symbols, d_out, out_cap, d_out_size,
                d_status, d_scratch, scratch_cap, stream=None, check=True) -> int:
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode(_ptr(d_symbols), int(n_symbols), f.ctypes.data, f.size, C.byref(p),
                         _ptr(d_out), int(out_cap), _ptr(d_out_size), _ptr(d_status),
                         _ptr(d_scratch), int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode") if check else rc


def _raw_words(raw_words, n_alpha: int) -> np.ndarray:
    r = np.ascontiguousarray(raw_words, dtype=np.uint8)
    if r.size != n_alpha:
        raise ValueError("raw_words needs one entry per alphabet symbol")
    return r


def rans_max_encoded_size_bypass(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_max_encoded_size_bypass(int(n_symbols), C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_scratch_size_bypass(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_encode_scratch_size_bypass(int(n_symbols),
                                                   C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_bypass(d_symbols, d_raw, n_symbols, freq, raw_words, n_lanes, chunk_symbols, d_out,
                       out_cap, d_out_size, d_status, d_scratch, scratch_cap, stream=None,
                       check=True) -> int:
    """rans_encode with raw 16-bit words after the symbols whose raw_words
    entry is 1 (bypass, Section 3)."""
    f = _freq(freq)
    r = _raw_words(raw_words, f.size)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_bypass(_ptr(d_symbols), _ptr(d_raw), int(n_symbols), f.ctypes.data,
                                r.ctypes.data, f.size, C.byref(p), _ptr(d_out), int(out_cap),
                                _ptr(d_out_size), _ptr(d_status), _ptr(d_scratch),
                                int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode_bypass") if check else rc


def rans_decode_bypass(d_msg, msg_size, freq, raw_words, n_lanes, chunk_symbols, d_symbols, d_raw,
                       n_symbols, d_status, stream=None, check=True) -> int:
    f = _freq(freq)
    r = _raw_words(raw_words, f.size)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode_bypass(_ptr(d_msg), int(msg_size), f.ctypes.data, r.ctypes.data, f.size,
                                C.byref(p), _ptr(d_symbols), _ptr(d_raw), int(n_symbols),
                                _ptr(d_status), _stream(stream))
    return _check(rc, "rans_decode_bypass") if check else rc


def encode_bypass(symbols, raw, freq, raw_words, n_lanes: int = 32, chunk_symbols: int = 65536,
                  stream=None, sync: bool = True):
    """Encode CUDA tensors symbols (uint8) and raw (int16/uint16 view, one
    per symbol).  Returns (message, size, status) like encode()."""
    import torch

    dev = symbols.device
    n = symbols.numel()
    cap = rans_max_encoded_size_bypass(n, n_lanes, chunk_symbols)
    scap = rans_encode_scratch_size_bypass(n, n_lanes, chunk_symbols)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(max(scap, 16), dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_encode_bypass(symbols, raw, n, freq, raw_words, n_lanes, chunk_symbols, out, cap, size,
                       status, scratch, scratch.numel(), stream)
    if not sync:
        return out, size, status
    torch.cuda.synchronize(dev)
    st = int(status.item())
    if st != RANS_OK:
        raise RansError(st, "rans_encode_bypass (device status)")
    return out[: int(size.item())], size, status


def decode_bypass(msg, n_symbols: int, freq, raw_words, n_lanes: int = 32,
                  chunk_symbols: int = 65536, stream=None, sync: bool = True):
    """Decode a bypass message.  Returns (symbols, raw, status), raw as an
    int16 tensor holding the u16 raw words (0 where a symbol has none)."""
    import torch

    dev = msg.device
    out = torch.empty(max(1, n_symbols), dtype=torch.uint8, device=dev)
    raw = torch.empty(max(1, n_symbols), dtype=torch.int16, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_decode_bypass(msg, msg.numel(), freq, raw_words, n_lanes, chunk_symbols, out, raw,
                       n_symbols, status, stream)
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st != RANS_OK:
            raise RansError(st, "rans_decode_bypass (device status)")
    return out[:n_symbols], raw[:n_symbols], status


def rans_max_encoded_size_bytes(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_max_encoded_size_bytes(int(n_symbols), C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_bytes(d_symbols, n_symbols, freq, n_lanes, chunk_symbols, d_out, out_cap,
                      d_out_size, d_status, d_scratch, scratch_cap, stream=None, check=True) -> int:
    """Byte-wise (b = 2^8, digits breadth-first per step, Section 5) encode."""
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_bytes(_ptr(d_symbols), int(n_symbols), f.ctypes.data, f.size, C.byref(p),
                               _ptr(d_out), int(out_cap), _ptr(d_out_size), _ptr(d_status),
                               _ptr(d_scratch), int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode_bytes") if check else rc


def rans_decode_bytes(d_msg, msg_size, freq, n_lanes, chunk_symbols, d_symbols, n_symbols,
                      d_status, stream=None, check=True) -> int:
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode_bytes(_ptr(d_msg), int(msg_size), f.ctypes.data, f.size, C.byref(p),
                               _ptr(d_symbols), int(n_symbols), _ptr(d_status), _stream(stream))
    return _check(rc, "rans_decode_bytes") if check else rc


def encode_bytes(symbols, freq, n_lanes: int = 32, chunk_symbols: int = 65536, stream=None,
                 sync: bool = True):
    """Encode a CUDA uint8 tensor as a byte-wise message; (message, size, status)."""
    import torch

    dev = symbols.device
    n = symbols.numel()
    cap = rans_max_encoded_size_bytes(n, n_lanes, chunk_symbols)
    scap = rans_encode_scratch_size(n, n_lanes, chunk_symbols)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(max(scap, 16), dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_encode_bytes(symbols, n, freq, n_lanes, chunk_symbols, out, cap, size, status, scratch,
                      scratch.numel(), stream)
    if not sync:
        return out, size, status
    torch.cuda.synchronize(dev)
    st = int(status.item())
    if st != RANS_OK:
        raise RansError(st, "rans_encode_bytes (device status)")
    return out[: int(size.item())], size, status


def decode_bytes(msg, n_symbols: int, freq, n_lanes: int = 32, chunk_symbols: int = 65536,
                 stream=None, sync: bool = True):
    """Decode a byte-wise message; (symbols, status)."""
    import torch

    dev = msg.device
    out = torch.empty(max(1, n_symbols), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_decode_bytes(msg, msg.numel(), freq, n_lanes, chunk_symbols, out, n_symbols, status,
                      stream)
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st != RANS_OK:
            raise RansError(st, "rans_decode_bytes (device status)")
    return out[:n_symbols], status


def rans_encode_scratch_size_adaptive(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_encode_scratch_size_adaptive(int(n_symbols),
                                                     C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_adaptive(d_symbols, n_symbols, n_lanes, chunk_symbols, d_out, out_cap, d_out_size,
                         d_status, d_scratch, scratch_cap, stream=None, check=True) -> int:
    """Adaptive binary encode: one context per coder (Section 5)."""
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_adaptive(_ptr(d_symbols), int(n_symbols), C.byref(p), _ptr(d_out),
                                  int(out_cap), _ptr(d_out_size), _ptr(d_status), _ptr(d_scratch),
                                  int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode_adaptive") if check else rc


def rans_decode_adaptive(d_msg, msg_size, n_lanes, chunk_symbols, d_symbols, n_symbols, d_status,
                         stream=None, check=True) -> int:
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode_adaptive(_ptr(d_msg), int(msg_size), C.byref(p), _ptr(d_symbols),
                                  int(n_symbols), _ptr(d_status), _stream(stream))
    return _check(rc, "rans_decode_adaptive") if check else rc


def encode_adaptive(symbols, n_lanes: int = 32, chunk_symbols: int = 65536, stream=None,
                    sync: bool = True):
    """Encode a CUDA uint8 tensor of bits (0/1) as an adaptive message; (message, size, status)."""
    import torch

    dev = symbols.device
    n = symbols.numel()
    cap = rans_max_encoded_size(n, n_lanes, chunk_symbols)
    scap = rans_encode_scratch_size_adaptive(n, n_lanes, chunk_symbols)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(max(scap, 16), dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_encode_adaptive(symbols, n, n_lanes, chunk_symbols, out, cap, size, status, scratch,
                         scratch.numel(), stream)
    if not sync:
        return out, size, status
    torch.cuda.synchronize(dev)
    st = int(status.item())
    if st != RANS_OK:
        raise RansError(st, "rans_encode_adaptive (device status)")
    return out[: int(size.item())], size, status


def decode_adaptive(msg, n_symbols: int, n_lanes: int = 32, chunk_symbols: int = 65536,
                    stream=None, sync: bool = True):
    """Decode an adaptive message; (bits, status)."""
    import torch

    dev = msg.device
    out = torch.empty(max(1, n_symbols), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_decode_adaptive(msg, msg.numel(), n_lanes, chunk_symbols, out, n_symbols, status, stream)
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st != RANS_OK:
            raise RansError(st, "rans_decode_adaptive (device status)")
    return out[:n_symbols], status


RANS_ADAPTIVE_N_MAX = 16


def rans_encode_scratch_size_adaptive_n(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_encode_scratch_size_adaptive_n(int(n_symbols),
                                                       C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_adaptive_n(d_symbols, n_symbols, n_alpha, n_lanes, chunk_symbols, d_out, out_cap,
                           d_out_size, d_status, d_scratch, scratch_cap, stream=None,
                           check=True) -> int:
    """Adaptive encode over n_alpha <= 16 symbols: one model per coder (Section 5)."""
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_adaptive_n(_ptr(d_symbols), int(n_symbols), int(n_alpha), C.byref(p),
                                    _ptr(d_out), int(out_cap), _ptr(d_out_size), _ptr(d_status),
                                    _ptr(d_scratch), int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode_adaptive_n") if check else rc


def rans_decode_adaptive_n(d_msg, msg_size, n_alpha, n_lanes, chunk_symbols, d_symbols, n_symbols,
                           d_status, stream=None, check=True) -> int:
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode_adaptive_n(_ptr(d_msg), int(msg_size), int(n_alpha), C.byref(p),
                                    _ptr(d_symbols), int(n_symbols), _ptr(d_status),
                                    _stream(stream))
    return _check(rc, "rans_decode_adaptive_n") if check else rc


def encode_adaptive_n(symbols, n_alpha: int, n_lanes: int = 32, chunk_symbols: int = 65536,
                      stream=None, sync: bool = True):
    """Encode a CUDA uint8 tensor of symbols < n_alpha with per-coder adaptive
    models; (message, size, status)."""
    import torch

    dev = symbols.device
    n = symbols.numel()
    cap = rans_max_encoded_size(n, n_lanes, chunk_symbols)
    scap = rans_encode_scratch_size_adaptive_n(n, n_lanes, chunk_symbols)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(max(scap, 16), dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_encode_adaptive_n(symbols, n, n_alpha, n_lanes, chunk_symbols, out, cap, size, status,
                           scratch, scratch.numel(), stream)
    if not sync:
        return out, size, status
    torch.cuda.synchronize(dev)
    st = int(status.item())
    if st != RANS_OK:
        raise RansError(st, "rans_encode_adaptive_n (device status)")
    return out[: int(size.item())], size, status


def decode_adaptive_n(msg, n_symbols: int, n_alpha: int, n_lanes: int = 32,
                      chunk_symbols: int = 65536, stream=None, sync: bool = True):
    """Decode an adaptive-n message; (symbols, status)."""
    import torch

    dev = msg.device
    out = torch.empty(max(1, n_symbols), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_decode_adaptive_n(msg, msg.numel(), n_alpha, n_lanes, chunk_symbols, out, n_symbols,
                           status, stream)
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st != RANS_OK:
            raise RansError(st, "rans_decode_adaptive_n (device status)")
    return out[:n_symbols], status


def rans_prefix_lengths(weights, max_len: int = RANS_PREFIX_MAX_LEN) -> np.ndarray:
    """Optimal code lengths <= max_len (package-merge, host)."""
    w = np.ascontiguousarray(weights, dtype=np.uint64)
    out = np.zeros(max(1, w.size), dtype=np.uint8)
    _check(lib.rans_prefix_lengths(w.ctypes.data, w.size, max_len, out.ctypes.data),
           "rans_prefix_lengths")
    return out[: w.size]


def rans_prefix_codes(lengths) -> np.ndarray:
    """Canonical codes of the given code lengths (host)."""
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(max(1, ln.size), dtype=np.uint16)
    _check(lib.rans_prefix_codes(ln.ctypes.data, ln.size, out.ctypes.data), "rans_prefix_codes")
    return out[: ln.size]


def rans_max_encoded_size_prefix(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_max_encoded_size_prefix(int(n_symbols), C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_scratch_size_prefix(n_symbols: int, n_lanes: int, chunk_symbols: int) -> int:
    return int(lib.rans_encode_scratch_size_prefix(int(n_symbols),
                                                   C.byref(_params(n_lanes, chunk_symbols))))


def _lengths(lengths) -> np.ndarray:
    return np.ascontiguousarray(lengths, dtype=np.uint8)


def rans_encode_prefix(d_symbols, n_symbols, lengths, n_lanes, chunk_symbols, d_out, out_cap,
                       d_out_size, d_status, d_scratch, scratch_cap, stream=None, check=True) -> int:
    """Prefix-code coders muxed in their decoders' read order (Section 4)."""
    ln = _lengths(lengths)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_prefix(_ptr(d_symbols), int(n_symbols), ln.ctypes.data, ln.size,
                                C.byref(p), _ptr(d_out), int(out_cap), _ptr(d_out_size),
                                _ptr(d_status), _ptr(d_scratch), int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode_prefix") if check else rc


def rans_decode_prefix(d_msg, msg_size, lengths, n_lanes, chunk_symbols, d_symbols, n_symbols,
                       d_status, stream=None, check=True) -> int:
    ln = _lengths(lengths)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode_prefix(_ptr(d_msg), int(msg_size), ln.ctypes.data, ln.size, C.byref(p),
                                _ptr(d_symbols), int(n_symbols), _ptr(d_status), _stream(stream))
    return _check(rc, "rans_decode_prefix") if check else rc


def encode_prefix(symbols, lengths, n_lanes: int = 32, chunk_symbols: int = 65536, stream=None,
                  sync: bool = True):
    """Encode a CUDA uint8 tensor as a prefix-code message; (message, size, status)."""
    import torch

    dev = symbols.device
    n = symbols.numel()
    cap = rans_max_encoded_size_prefix(n, n_lanes, chunk_symbols)
    scap = rans_encode_scratch_size_prefix(n, n_lanes, chunk_symbols)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    scratch = torch.empty(max(scap, 16), dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_encode_prefix(symbols, n, lengths, n_lanes, chunk_symbols, out, cap, size, status,
                       scratch, scratch.numel(), stream)
    if not sync:
        return out, size, status
    torch.cuda.synchronize(dev)
    st = int(status.item())
    if st != RANS_OK:
        raise RansError(st, "rans_encode_prefix (device status)")
    return out[: int(size.item())], size, status


def decode_prefix(msg, n_symbols: int, lengths, n_lanes: int = 32, chunk_symbols: int = 65536,
                  stream=None, sync: bool = True):
    """Decode a prefix-code message; (symbols, status)."""
    import torch

    dev = msg.device
    out = torch.empty(max(1, n_symbols), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_decode_prefix(msg, msg.numel(), lengths, n_lanes, chunk_symbols, out, n_symbols, status,
                       stream)
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st != RANS_OK:
            raise RansError(st, "rans_decode_prefix (device status)")
    return out[:n_symbols], status


def rans_decode_host_work_size(msg_size: int, n_symbols: int) -> int:
    return int(lib.rans_decode_host_work_size(int(msg_size), int(n_symbols)))


def rans_decode_host(h_msg, msg_size, freq, n_lanes, chunk_symbols, h_symbols, n_symbols,
                     h_status, d_work, work_cap, stream=None, check=True) -> int:
    """rans_decode from and to host memory (pointers or CPU tensors, page-locked
    for overlap), copies in both directions overlapped with the decoding."""
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode_host(_ptr(h_msg), int(msg_size), f.ctypes.data, f.size, C.byref(p),
                              _ptr(h_symbols), int(n_symbols), _ptr(h_status), _ptr(d_work),
                              int(work_cap), _stream(stream))
    return _check(rc, "rans_decode_host") if check else rc


def decode_host(msg, n_symbols: int, freq, n_lanes: int = 32, chunk_symbols: int = 65536,
                device=None, stream=None, out=None, work=None):
    """Decode a host (CPU, ideally pinned) uint8 message tensor into a host
    tensor of n_symbols bytes through rans_decode_host.  Returns (symbols,
    status) after synchronizing."""
    import torch

    device = device or torch.device("cuda", torch.cuda.current_device())
    cap = rans_decode_host_work_size(msg.numel(), n_symbols)
    if work is None or work.numel() < cap:
        work = torch.empty(cap, dtype=torch.uint8, device=device)
    if out is None:
        out = torch.empty(max(1, n_symbols), dtype=torch.uint8, pin_memory=True)
    status = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    rans_decode_host(msg, msg.numel(), freq, n_lanes, chunk_symbols, out, n_symbols, status,
                     work, work.numel(), stream)
    if stream is not None:
        stream.synchronize()
    else:
        torch.cuda.current_stream(device).synchronize()
    return out[:n_symbols], int(status.item())


def rans_encode_host_work_size(n_symbols: int, n_lanes: int = 32, chunk_symbols: int = 65536) -> int:
    return int(lib.rans_encode_host_work_size(int(n_symbols),
                                              C.byref(_params(n_lanes, chunk_symbols))))


def rans_encode_host(h_symbols, n_symbols, freq, n_lanes, chunk_symbols, h_out, out_cap,
                     h_out_size, h_status, d_work, work_cap, stream=None, check=True) -> int:
    """rans_encode from and to host memory (pointers or CPU tensors; a
    page-locked, 16-byte aligned output is written by the device directly)."""
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_host(_ptr(h_symbols), int(n_symbols), f.ctypes.data, f.size, C.byref(p),
                              _ptr(h_out), int(out_cap), _ptr(h_out_size), _ptr(h_status),
                              _ptr(d_work), int(work_cap), _stream(stream))
    return _check(rc, "rans_encode_host") if check else rc


def encode_host(symbols, freq, n_lanes: int = 32, chunk_symbols: int = 65536, device=None,
                stream=None, out=None, work=None):
    """Encode a host (CPU, ideally pinned) uint8 tensor through
    rans_encode_host.  Returns (message, status) after synchronizing; the
    message is a view of the output buffer."""
    import torch

    device = device or torch.device("cuda", torch.cuda.current_device())
    n = symbols.numel()
    cap = rans_max_encoded_size(n, n_lanes, chunk_symbols)
    wcap = rans_encode_host_work_size(n, n_lanes, chunk_symbols)
    if work is None or work.numel() < wcap:
        work = torch.empty(wcap, dtype=torch.uint8, device=device)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    size = torch.zeros(1, dtype=torch.int64, pin_memory=True)
    status = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    rans_encode_host(symbols, n, freq, n_lanes, chunk_symbols, out, out.numel(), size, status,
                     work, work.numel(), stream)
    if stream is not None:
        stream.synchronize()
    else:
        torch.cuda.current_stream(device).synchronize()
    return out[: int(size.item())], int(status.item())


def rans_debug_checks() -> int:
    """Checked builds: failed kernel invariants since the last call (the
    counters are cleared); RansError(RANS_ERR_INVALID_ARG) otherwise."""
    v = C.c_uint64(0)
    _check(lib.rans_debug_checks(C.byref(v)), "rans_debug_checks")
    return int(v.value)


def rans_debug_check_selftest(stream=None) -> int:
    return _check(lib.rans_debug_check_selftest(_stream(stream)), "rans_debug_check_selftest")


def rans_check_bounded_wait(d_status, stream=None, check=True) -> int:
    """Diagnostic: a kernel whose bounded wait on a barrier that nothing
    completes gives up after about 200 ms and writes RANS_ERR_TIMEOUT."""
    rc = lib.rans_check_bounded_wait(_ptr(d_status), _stream(stream))
    return _check(rc, "rans_check_bounded_wait") if check else rc


def rans_check_lookback_wait(d_status, stream=None, check=True) -> int:
    """Diagnostic: the encoder's look-back for a chunk whose predecessor never
    publishes gives up after about 200 ms and writes RANS_ERR_TIMEOUT."""
    rc = lib.rans_check_lookback_wait(_ptr(d_status), _stream(stream))
    return _check(rc, "rans_check_lookback_wait") if check else rc


def rans_check_division(method: int, log2m: int, d_result, stream=None, check=True) -> int:
    """Diagnostic: the encoders' division (method 0: reciprocal multiply-high,
    method 1: the adaptive coder's float estimate) checked on the device for
    every frequency below M = 2^log2m and every state it divides; d_result is
    a device tensor of 4 u64 (checked, wrong, first wrong f << 32 | x, 0)."""
    rc = lib.rans_check_division(int(method), int(log2m), _ptr(d_result), _stream(stream))
    return _check(rc, "rans_check_division") if check else rc


def rans_check_gather_ceiling_warps() -> int:
    return int(lib.rans_check_gather_ceiling_warps())


def rans_check_cta_warps(n_units: int, sms: int, per_sm, max_warps: int) -> int:
    """The placing encoders' CTA size for n_units chunks that all start at
    once (host logic only); per_sm[w] = w-warp CTAs an SM holds, w = 0 ..
    max_warps (entry 0 unused)."""
    a = np.ascontiguousarray(per_sm, dtype=np.int32)
    if a.size < max_warps + 1:
        raise ValueError("per_sm needs max_warps + 1 entries")
    return int(lib.rans_check_cta_warps(int(n_units), int(sms), a.ctypes.data, int(max_warps)))


def rans_check_gather_ceiling(steps: int, d_out, out_size: int, d_sink, stream=None,
                              check=True) -> int:
    """Diagnostic: the table decoder's data-pipe work (slot-table gather, ring
    window read, 32-byte symbol store per step) without its arithmetic, in the
    plain decoder's shape; every one of rans_check_gather_ceiling_warps()
    warps runs `steps` steps (a multiple of 16)."""
    rc = lib.rans_check_gather_ceiling(int(steps), _ptr(d_out), int(out_size), _ptr(d_sink),
                                       _stream(stream))
    return _check(rc, "rans_check_gather_ceiling") if check else rc


def rans_encode_static_scratch(d_symbols, n_symbols, freq, n_lanes, chunk_symbols, d_out,
                               out_cap, d_out_size, d_status, stream=None, check=True) -> int:
    """rans_encode without a scratch argument: for callers that cannot
    allocate device memory, the library's fixed scratch array is used (see
    include/rans.h for the size limit and the rule that calls on one device
    must not overlap)."""
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_encode_static_scratch(_ptr(d_symbols), int(n_symbols), f.ctypes.data, f.size,
                                        C.byref(p), _ptr(d_out), int(out_cap), _ptr(d_out_size),
                                        _ptr(d_status), _stream(stream))
    return _check(rc, "rans_encode_static_scratch") if check else rc


def rans_decode(d_msg, msg_size, freq, n_lanes, chunk_symbols, d_symbols, n_symbols, d_status,
                stream=None, check=True) -> int:
    f = _freq(freq)
    p = _params(n_lanes, chunk_symbols)
    rc = lib.rans_decode(_ptr(d_msg), int(msg_size), f.ctypes.data, f.size, C.byref(p),
                         _ptr(d_symbols), int(n_symbols), _ptr(d_status), _stream(stream))
    return _check(rc, "rans_decode") if check else rc


def rans_decode_batch_scratch_size(n_streams: int) -> int:
    return int(lib.rans_decode_batch_scratch_size(int(n_streams)))


def rans_decode_batch(d_streams, n_streams, d_freqs, n_tables, d_status, d_scratch, scratch_cap,
                      stream=None, check=True) -> int:
    rc = lib.rans_decode_batch(_ptr(d_streams), int(n_streams), _ptr(d_freqs), int(n_tables),
                               _ptr(d_status), _ptr(d_scratch), int(scratch_cap), _stream(stream))
    return _check(rc, "rans_decode_batch") if check else rc


def rans_encode_batch_plan(h_streams: np.ndarray) -> int:
    """Fill h_streams["scratch_offset"] in place (ENCODE_STREAM_DTYPE array)
    and return the scratch bytes rans_encode_batch needs."""
    assert h_streams.dtype == ENCODE_STREAM_DTYPE and h_streams.flags.c_contiguous
    total = int(lib.rans_encode_batch_plan(h_streams.ctypes.data, h_streams.size))
    if h_streams.size and total == 0:
        raise RansError(RANS_ERR_INVALID_ARG, "rans_encode_batch_plan")
    return total


def rans_encode_batch(d_streams, n_streams, d_freqs, n_tables, d_out_sizes, d_status, d_scratch,
                      scratch_cap, stream=None, check=True) -> int:
    rc = lib.rans_encode_batch(_ptr(d_streams), int(n_streams), _ptr(d_freqs), int(n_tables),
                               _ptr(d_out_sizes), _ptr(d_status), _ptr(d_scratch),
                               int(scratch_cap), _stream(stream))
    return _check(rc, "rans_encode_batch") if check else rc


class Server:
    """rans_server_create / rans_server_run / rans_server_destroy.

    tables_dev: device [n_tables, 256] u16 models (kept resident);
    arena: torch uint8 device tensor = the server's HBM budget."""

    def __init__(self, tables_dev, arena, max_batch: int = 64, n_slots: int = 3):
        self._tables, self._arena = tables_dev, arena
        h = C.c_void_p()
        _check(lib.rans_server_create(_ptr(tables_dev), tables_dev.shape[0], _ptr(arena),
                                      arena.numel(), max_batch, n_slots, C.byref(h)),
               "rans_server_create")
        self._h = h

    def run(self, reqs: np.ndarray) -> np.ndarray:
        assert reqs.dtype == REQUEST_DTYPE and reqs.flags.c_contiguous
        res = np.zeros(reqs.size, dtype=RESULT_DTYPE)
        _check(lib.rans_server_run(self._h, reqs.ctypes.data, reqs.size, res.ctypes.data),
               "rans_server_run")
        return res

    def close(self):
        if self._h:
            lib.rans_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- conveniences: allocate with torch, call the entry points -----------------

def encode(symbols, freq, n_lanes: int = 32, chunk_symbols: int = 65536, stream=None,
           out=None, scratch=None, sync: bool = True):
    """Encode a CUDA uint8 tensor.  Returns (message, size, status) where
    ``message`` is the output buffer (trimmed to the size when sync=True),
    and ``size``/``status`` are the device words the library wrote."""
    import torch

    dev = symbols.device
    n = symbols.numel()
    cap = rans_max_encoded_size(n, n_lanes, chunk_symbols)
    scap = rans_encode_scratch_size(n, n_lanes, chunk_symbols)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=dev)
    if scratch is None:
        scratch = torch.empty(scap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_encode(symbols, n, freq, n_lanes, chunk_symbols, out, out.numel(), size, status,
                scratch, scratch.numel(), stream)
    if not sync:
        return out, size, status
    torch.cuda.synchronize(dev)
    st = int(status.item())
    if st != RANS_OK:
        raise RansError(st, "rans_encode (device status)")
    return out[: int(size.item())], size, status


def decode(msg, n_symbols: int, freq, n_lanes: int = 32, chunk_symbols: int = 65536,
           stream=None, out=None, sync: bool = True):
    """Decode a CUDA uint8 message tensor into n_symbols bytes.  Returns
    (symbols, status)."""
    import torch

    dev = msg.device
    if out is None:
        out = torch.empty(max(1, n_symbols), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rans_decode(msg, msg.numel(), freq, n_lanes, chunk_symbols, out, n_symbols, status, stream)
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st != RANS_OK:
            raise RansError(st, "rans_decode (device status)")
    return out[:n_symbols], status
