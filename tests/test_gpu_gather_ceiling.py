"""rans_check_gather_ceiling: the table decoder's data-pipe work (slot-table
gather, ring window read, 32-byte symbol store per step) without its
arithmetic, the ceiling bench.py sets beside the decoder's rate.  The test
checks that it runs through the C ABI on every warp it reports, writes its
output, and refuses bad arguments without launching."""
import pytest

pytestmark = pytest.mark.gpu


def test_gather_ceiling_runs_and_checks_its_arguments(rlib, cuda):
    import torch

    warps = rlib.rans_check_gather_ceiling_warps()
    assert warps > 0 and warps % 12 == 0
    need = warps * 4096
    out = torch.zeros(need, dtype=torch.uint8, device=cuda)
    sink = torch.zeros(1, dtype=torch.int32, device=cuda)
    rlib.rans_check_gather_ceiling(256, out, need, sink)
    torch.cuda.synchronize()
    # every warp stored 256 steps x 32 bytes cyclically over its 4 KiB: all of it
    written = out.view(warps, 4096)
    assert bool((written != 0).any(dim=1).all())
    assert int(sink.item()) == 0
    for steps, size in ((17, need), (0, need), (256, need - 1)):
        rc = rlib.rans_check_gather_ceiling(steps, out, size, sink, check=False)
        assert rc == (rlib.RANS_ERR_BUFFER_TOO_SMALL if size < need else
                      rlib.RANS_ERR_INVALID_ARG)
    assert rlib.rans_check_gather_ceiling(256, None, need, sink,
                                          check=False) == rlib.RANS_ERR_INVALID_ARG
