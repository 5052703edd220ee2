"""B300-native interleaved streaming rANS (Giesen, "Interleaved entropy coders").

The coder itself runs in hand-written CUDA kernels behind the C ABI declared
in include/rans.h; ``paper_1402_3392_b300.rans`` is the thin ctypes binding.
The binding is loaded on first use of one of its names so that the synthetic
workload generators (``paper_1402_3392_b300.workloads``) import without it.
"""
_BINDING = frozenset({
    "RansError", "rans_version", "rans_status_string", "rans_quantize_table",
    "rans_max_encoded_size", "rans_encode_scratch_size", "rans_encode", "rans_decode",
    "rans_encode_static_scratch", "encode", "decode", "rans_decode_batch",
    "rans_decode_batch_scratch_size", "rans_encode_batch", "rans_encode_batch_plan",
    "rans_check_bounded_wait", "rans_check_lookback_wait", "rans_decode_host", "rans_decode_host_work_size", "decode_host",
    "rans_max_encoded_size_bypass", "rans_encode_scratch_size_bypass", "rans_encode_bypass",
    "rans_decode_bypass", "encode_bypass", "decode_bypass", "rans_max_encoded_size_bytes",
    "rans_encode_bytes", "rans_decode_bytes", "encode_bytes", "decode_bytes",
    "rans_encode_scratch_size_adaptive", "rans_encode_adaptive", "rans_decode_adaptive",
    "encode_adaptive", "decode_adaptive", "rans_prefix_lengths", "rans_prefix_codes",
    "rans_max_encoded_size_prefix", "rans_encode_scratch_size_prefix", "rans_encode_prefix",
    "rans_decode_prefix", "encode_prefix", "decode_prefix", "rans_encode_host_work_size",
    "rans_encode_host", "encode_host", "rans_debug_checks", "rans_debug_check_selftest",
})


def __getattr__(name):
    if name in _BINDING:
        from . import rans

        return getattr(rans, name)
    raise AttributeError(name)
