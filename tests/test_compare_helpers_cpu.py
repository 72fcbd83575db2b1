"""The GPU-vs-oracle comparison helpers themselves, on planted differences
(CPU only): the element-wise bound catches one wrong value that the summed
relative L1 lets pass, names the value, and accepts exact or rounding-level
agreement; the per-field relative L1 is the plain definition."""
from __future__ import annotations

import numpy as np

from gpu_util import (EPS_F32, ELEM_C_F32, elementwise_excess, flux_rel_l1, rel_l1_fields,
                      rel_l1_per_field)

F32, F64 = 0, 2


def _state(n=7, seed=3):
    rng = np.random.default_rng(seed)
    b = rng.uniform(0.5, 2.0, (n, 5, 16, 16, 16))
    b[:, 1:4] = rng.normal(0.0, 0.3, (n, 3, 16, 16, 16))
    return b


def test_one_wrong_value_passes_the_sum_but_not_the_element_bound():
    b = _state()
    a = b.copy()
    a[3, 4, 5, 6, 7] *= 1.1                       # one energy value off by 10 %
    assert rel_l1_fields(a, b) < 1e-5              # the summed norm lets it pass
    r, idx, av, bv = elementwise_excess(a, b, F32)
    assert r > 1e2 and idx == (3, 4, 5, 6, 7) and av == 1.1 * bv


def test_rounding_level_differences_pass():
    b = _state()
    rng = np.random.default_rng(1)
    scale = np.abs(b).reshape(7, 5, -1).max(axis=2)[:, :, None, None, None]
    a = b + 8 * EPS_F32 * scale * rng.uniform(-1, 1, b.shape)
    assert elementwise_excess(a, b, F32)[0] <= 8 / ELEM_C_F32 * 1.01
    assert elementwise_excess(b, b, F64)[0] == 0.0
    # FP64: 1e-12 of the scale
    a64 = b + 0.5e-12 * scale
    assert elementwise_excess(a64, b, F64)[0] <= 0.5
    assert elementwise_excess(b + 3e-12 * scale, b, F64)[0] > 1.0


def test_momentum_scale_is_the_momentum_magnitude():
    b = _state()
    b[:, 3] = 0.0                                 # rho w identically zero ...
    a = b.copy()
    a[0, 3, 0, 0, 0] = 1e-9                       # ... yet judged against |m|: a value
    # 1e-9 of the momentum magnitude passes, one at 1e-3 of it does not
    assert elementwise_excess(a, b, F32)[0] < 1.0
    a[0, 3, 0, 0, 0] = 1e-3
    assert elementwise_excess(a, b, F32)[0] > 1.0


def test_zero_field_must_match_exactly_and_nan_fails():
    b = _state()
    b[:, 1:4] = 0.0                               # a state at rest: momenta identically 0
    a = b.copy()
    a[2, 2, 1, 1, 1] = 1e-30
    assert elementwise_excess(a, b, F32)[0] == np.inf
    a = b.copy()
    a[1, 0, 2, 2, 2] = np.nan
    assert elementwise_excess(a, b, F32)[0] == np.inf


def test_face_flux_layout_is_compared_per_field():
    rng = np.random.default_rng(4)
    b = rng.uniform(0.5, 2.0, (3, 6, 5, 16, 16))
    a = b.copy()
    a[1, 4, 2, 3, 5] *= 1.001                     # face 4 (-z), field 2
    r, idx, _, _ = elementwise_excess(a, b, F32, state=False)
    assert r > 1.0 and idx[:2] == (1, 2)           # group 1, field 2
    assert flux_rel_l1(a, b) < 1e-5


def test_per_field_rel_l1_definition():
    b = np.zeros((2, 3, 4))
    b[:, 0] = 1.0
    b[:, 1] = 2.0
    a = b.copy()
    a[0, 0, 0] += 0.8                              # field 0: 0.8 / 8
    a[1, 1, :] += 0.4                              # field 1: 1.6 / 16
    got = rel_l1_per_field(a, b)
    assert np.allclose(got, [0.1, 0.1, 0.0])
    a[0, 2, 0] = 1e-20                             # field 2 is zero in b only
    assert rel_l1_per_field(a, b)[2] == np.inf
