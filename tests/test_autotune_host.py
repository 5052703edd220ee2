"""The batched coder's layout candidates (autotune.chunk_sizes) -- host logic,
no GPU.  The 10,000-stream workload asks for chunks of 16-256 KiB: every
chunk a layout gives, but a stream's last, must lie in that range, and a
stream never has more chunks than one work item of the batched decoder
holds unless the candidate size itself is reached."""
import numpy as np
import pytest

from paper_1402_3392_b300 import workloads as wl

CHUNKS = (16 << 10, 32 << 10, 64 << 10, 128 << 10, 256 << 10)


@pytest.mark.parametrize("policy", ["fixed", "fill"])
@pytest.mark.parametrize("chunk", CHUNKS)
def test_chunk_sizes_stay_in_the_candidate_range(rlib, policy, chunk):
    from paper_1402_3392_b300 import autotune   # imports the binding: after rlib built it

    assert autotune.CHUNKS == CHUNKS and policy in autotune.POLICIES
    cfg = wl.WORKLOADS["batched"]
    sizes = wl.log_uniform_sizes(wl.rng_for("batched"), cfg["n_streams"], cfg["size_lo"],
                                 cfg["size_hi"])
    cs = autotune.chunk_sizes(sizes, chunk, policy)
    assert cs.shape == sizes.shape
    lo, hi = autotune.CHUNKS[0], autotune.CHUNKS[-1]
    assert (cs >= lo).all() and (cs <= hi).all()
    assert (cs <= chunk).all()
    if policy == "fixed":
        assert (cs == chunk).all()
    else:
        # a stream is cut into at most ITEM_CHUNKS chunks while the chunk
        # size is below the candidate, and the chunk size never goes below
        # what that needs
        n_chunks = -(-sizes // cs)
        short = cs < chunk
        assert (n_chunks[short] <= autotune.ITEM_CHUNKS).all()
        assert (cs % 1024 == 0).all()
