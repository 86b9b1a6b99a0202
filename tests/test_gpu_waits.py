"""Bounded device waits: a look-back whose predecessor never publishes gives up
after its poll limit, records GS_ERR_TIMEOUT in the workspace's status word,
and the kernel returns; nothing traps or hangs, and the context stays usable.
The stall is made on the host (tile 0 of a radix pass is withheld: no CTA ever
takes it), not by a fault."""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_18764_gb300 as gs
from paper_2505_18764_gb300 import _lib

pytestmark = pytest.mark.gpu


def _keys(n, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << 20, size=n, dtype=np.uint64).astype(np.uint32)
    return torch.from_numpy(k.view(np.int32)).cuda(), torch.arange(n, dtype=torch.int32, device="cuda")


def test_lookback_wait_gives_up_and_reports_timeout():
    from paper_2505_18764_gb300 import build
    build.build_library()
    n = 50000
    ws = gs.Workspace(n, 16, 16, gs.RasterOpts())
    keys, vals = _keys(n, 1)
    gs.stalled_sort_selftest(ws, keys, vals, spin_limit=10000)
    with pytest.raises(gs.GsError) as e:
        gs.check_status(ws)
    assert e.value.code == _lib.GS_ERR_TIMEOUT
    # the context is still usable: an ordinary sort on the same workspace is exact
    kr, vr = gs.sort_pairs(ws, keys, vals, 24)
    gs.check_status(ws)
    order = oracle.stable_sort_u32(keys.cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(vr.cpu().numpy(), order)


def test_selftest_argument_checks():
    ws = gs.Workspace(4096, 16, 16, gs.RasterOpts())
    keys, vals = _keys(2048, 2)
    with pytest.raises(gs.GsError):                     # one tile: nothing to withhold
        gs.stalled_sort_selftest(ws, keys, vals, spin_limit=100)
    keys, vals = _keys(4096, 3)
    with pytest.raises(gs.GsError):                     # limit beyond the library's own
        gs.stalled_sort_selftest(ws, keys, vals, spin_limit=1 << 23)
