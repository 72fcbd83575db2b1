"""gamer_hydro_dt_noalloc: the dt / conservation reduction for callers that
cannot allocate device memory (for example a host AMR code whose device memory
all belongs to its own allocator).  It must give the results of
gamer_hydro_dt with a caller-provided workspace, call after call, although its
scratch array keeps whatever the previous call left in it.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1007_3818_gb300 import native as n
    assert n.gamer_device_check() == 0
    return n


def _inputs(rng, N, L):
    part = np.column_stack([rng.uniform(0.1, 3.0, N), rng.standard_normal((N, 5))])
    level = rng.integers(0, L, N).astype(np.int32)
    dh_level = 1.0 / (256.0 * 2.0 ** np.arange(L))
    return part, level, dh_level


def _run(native, noalloc, part, level, dh_level, cfl):
    import torch
    d = lambda a, t=torch.float64: torch.as_tensor(a, device="cuda", dtype=t)
    N, L = len(part), len(dh_level)
    dt_out = torch.full((L,), -1.0, device="cuda", dtype=torch.float64)
    tot = torch.full((5,), -1.0, device="cuda", dtype=torch.float64)
    dt_group = torch.full((N,), -1.0, device="cuda", dtype=torch.float64)
    args = (d(part), d(level, torch.int32), d(dh_level), cfl, dt_out, tot, dt_group)
    if noalloc:
        native.gamer_hydro_dt_noalloc(*args)
    else:
        ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(N, L), device="cuda",
                         dtype=torch.uint8)
        native.gamer_hydro_dt(*args, ws)
    torch.cuda.synchronize()
    return dt_out.cpu().numpy(), tot.cpu().numpy(), dt_group.cpu().numpy()


def test_noalloc_matches_workspace_version_on_consecutive_calls(native):
    rng = np.random.default_rng(2024)
    # two calls in a row with different sizes: the second must not see the
    # first one's leftovers in the shared scratch array
    for N, L in ((5000, 3), (1700, 2), (40000, 1)):
        part, level, dh_level = _inputs(rng, N, L)
        ref = _run(native, False, part, level, dh_level, 0.5)
        got = _run(native, True, part, level, dh_level, 0.5)
        assert np.array_equal(got[0], ref[0])                      # dt per level
        assert np.allclose(got[1], ref[1], rtol=1e-13,
                           atol=1e-13 * np.abs(part[:, 1:]).sum())  # totals
        assert np.array_equal(got[2], ref[2])                      # dt per group


def test_noalloc_rejects_sizes_beyond_its_scratch(native):
    import torch
    N = 200000
    # buffers sized for the call, so that even a regressed size check could
    # not read or write out of bounds
    part = torch.zeros((N, 6), device="cuda", dtype=torch.float64)
    level = torch.zeros(N, device="cuda", dtype=torch.int32)
    dh = torch.ones(64, device="cuda", dtype=torch.float64)
    out = torch.zeros(64, device="cuda", dtype=torch.float64)
    dt_group = torch.zeros(N, device="cuda", dtype=torch.float64)
    # 64 levels and 200,000 groups need more than the 64 KiB scratch; the call
    # is rejected on the host before anything is launched
    rc = native.lib().gamer_hydro_dt_noalloc(ctypes.c_void_p(part.data_ptr()), N,
                                             ctypes.c_void_p(level.data_ptr()), 64,
                                             ctypes.c_void_p(dh.data_ptr()), 0.5,
                                             ctypes.c_void_p(out.data_ptr()), None,
                                             ctypes.c_void_p(dt_group.data_ptr()), None)
    assert rc == -7  # GAMER_E_WORKSPACE
    torch.cuda.synchronize()
    assert not out.any() and not dt_group.any()
