"""The allocation-free pair sort against the workspace pair sort.

gs_sort_pairs_noalloc serves callers that cannot hand the library any device
scratch (a host that owns every device allocation, or a service whose memory
budget is fixed at start-up); it keeps its scratch in a fixed array inside the
library.  Two calls in a row must each give exactly what gs_sort_pairs gives
on the same input, including the first call of the process, which also sets
the array up.  This file sorts last so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2505_18764_gb300 as gs
from paper_2505_18764_gb300 import _lib

pytestmark = pytest.mark.gpu


def _inputs(n, bits, seed, full_range=False):
    rng = np.random.default_rng(seed)
    hi = 2 ** bits if full_range else min(2 ** bits, max(2, n // 5))
    keys = rng.integers(0, hi, size=n, dtype=np.uint64).astype(np.uint32)
    return (torch.from_numpy(keys.view(np.int32)).cuda(),
            torch.arange(n, dtype=torch.int32, device="cuda"))


def _noalloc_via_c_abi(keys, vals, bits):
    """Direct C-ABI call (no Python-side workspace exists for this entry point)."""
    lib = _lib.load()
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.gs_sort_pairs_noalloc(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                   ctypes.c_void_p(ko.data_ptr()), ctypes.c_void_p(vo.data_ptr()),
                                   keys.numel(), bits, ctypes.c_void_p(stream))
    assert rc == _lib.GS_OK, lib.gs_last_error()
    assert lib.gs_sort_pairs_noalloc_status(ctypes.c_void_p(stream)) == _lib.GS_OK, lib.gs_last_error()
    return ko, vo


def _check_against_workspace_sort(n, bits, seed, full_range=False):
    keys, vals = _inputs(n, bits, seed, full_range)
    ko, vo = _noalloc_via_c_abi(keys, vals, bits)
    ws = gs.Workspace(max(n, 1), 16, 16, gs.RasterOpts())
    kr, vr = gs.sort_pairs(ws, keys, vals, bits)
    gs.check_status(ws)
    torch.cuda.synchronize()
    assert torch.equal(ko, kr) and torch.equal(vo, vr)
    # and both are the stable sort
    order = oracle.stable_sort_u32(keys.cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(vo.cpu().numpy(), order)


def test_noalloc_sort_matches_workspace_sort_twice():
    assert torch.cuda.is_available()
    from paper_2505_18764_gb300 import build
    build.build_library()
    # two calls in a row, different sizes and keys
    for n, bits, seed in [(200003, 24, 1), (131071, 13, 2)]:
        _check_against_workspace_sort(n, bits, seed)


@pytest.mark.parametrize("n,bits,full", [
    (150001, 32, True),                             # four passes over keys that fill 32 bits
    (_lib.GS_SORT_NOALLOC_MAX_PAIRS, 32, True),     # exactly the maximum
    (_lib.GS_SORT_NOALLOC_MAX_PAIRS, 17, False),
    (0, 32, False),                                 # empty
])
def test_noalloc_sort_edge_sizes(n, bits, full):
    _check_against_workspace_sort(n, bits, 11 + n % 7, full_range=full)


def test_noalloc_sort_rejects_more_than_its_maximum():
    lib = _lib.load()
    n = _lib.GS_SORT_NOALLOC_MAX_PAIRS + 1
    rc = lib.gs_sort_pairs_noalloc(None, None, None, None, n, 32, None)  # refused on the host
    assert rc == _lib.GS_ERR_INVALID_ARG
    assert b"GS_SORT_NOALLOC_MAX_PAIRS" in lib.gs_last_error()


def test_noalloc_sort_rejects_host_memory():
    lib = _lib.load()
    keys = np.zeros(4096, dtype=np.uint32)
    p = keys.ctypes.data_as(ctypes.c_void_p)
    rc = lib.gs_sort_pairs_noalloc(p, p, p, p, keys.size, 32, None)
    assert rc == _lib.GS_ERR_INVALID_ARG, lib.gs_last_error()


def test_noalloc_sort_reports_a_wait_that_gave_up():
    """A radix pass over the library's array with tile 0 withheld: its look-back
    waits give up after 1e4 polls, the status query says GS_ERR_TIMEOUT, and the
    next ordinary call (which clears the status) is correct again."""
    keys, vals = _inputs(20000, 16, 5)
    gs.stalled_sort_selftest(None, keys, vals, spin_limit=10000)
    with pytest.raises(gs.GsError) as e:
        gs.sort_pairs_noalloc_status()
    assert e.value.code == _lib.GS_ERR_TIMEOUT
    _check_against_workspace_sort(20000, 16, 6)
