"""The library's host-side ghost fill (CPU threads, used by the streamed level
step) reproduces the oracle's fill bit for bit.  Host code only: no GPU."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1007_3818_gb300 import build as cuda_build
from paper_1007_3818_gb300 import native


@pytest.fixture(scope="module", autouse=True)
def _lib():
    cuda_build.build()
    native.lib()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("dims", [(3, 2, 4), (1, 1, 1), (5, 1, 2)])
def test_host_fill_matches_oracle(dtype, bc, dims):
    gx, gy, gz = dims
    G = gx * gy * gz
    rng = np.random.default_rng(G + bc)
    level = rng.standard_normal((G, 5, 16, 16, 16)).astype(dtype)
    out = np.full((G, 5, 20, 20, 20), np.nan, dtype=dtype)
    native.gamer_fill_ghosts_uniform_host(level, out, gx, gy, gz, bc, nthreads=3)
    ref = oracle.fill_ghosts_uniform(level.astype(np.float64), gx, gy, gz, bc)
    assert np.array_equal(out.astype(np.float64), ref)


def test_host_fill_rejects_bad_arguments():
    lv = np.zeros((8, 5, 16, 16, 16), np.float32)
    out = np.zeros((8, 5, 20, 20, 20), np.float32)
    with pytest.raises(native.GamerError):
        native.gamer_fill_ghosts_uniform_host(lv, out, 2, 2, 2, 5)
    with pytest.raises(native.GamerError):
        native.gamer_fill_ghosts_uniform_host(lv, out.astype(np.float64), 2, 2, 2, 0)
