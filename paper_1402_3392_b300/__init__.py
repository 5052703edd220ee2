"""B300-native interleaved streaming rANS (Giesen, "Interleaved entropy coders").

The coder itself runs in hand-written CUDA kernels behind the C ABI declared
in include/rans.h; ``paper_1402_3392_b300.rans`` is the thin ctypes binding.
The binding is loaded on first use of one of its names so that the synthetic
workload generators (``paper_1402_3392_b300.workloads``) import without it.
"""
_BINDING_NAMES = None


def __getattr__(name):
    global _BINDING_NAMES
    from . import rans

    if _BINDING_NAMES is None:
        _BINDING_NAMES = set(rans.__all__)
    if name in _BINDING_NAMES:
        return getattr(rans, name)
    raise AttributeError(name)
