"""Seeded generators: determinism, shapes and the stated workload structure."""
import numpy as np
import pytest

from paper_2511_15629_b300 import instances as I


def _same(a, b):
    for name in ("price", "trans", "cost", "terminal", "mu0"):
        assert getattr(a, name).tobytes() == getattr(b, name).tobytes(), name


@pytest.mark.parametrize("fn", [I.config1, I.config2, I.config5])
def test_seed_determinism(fn):
    _same(fn(), fn())


def test_config4_assets_deterministic_and_ranges():
    for j in (0, 7, 255):
        a, b = I.config4_asset(j), I.config4_asset(j)
        _same(a, b)
        assert 201 <= a.N <= 4001 and 41 <= a.A <= 401 and a.A % 2 == 1
        assert 8 <= a.K <= 40 and 0.85 <= a.eta_c <= 0.97 and 0.85 <= a.eta_d <= 0.97
        assert a.T == 288


def test_config_shapes():
    c1 = I.config1()
    assert (c1.T, c1.N, c1.K, c1.A) == (24, 101, 5, 51) and c1.evals == 24 * 101 * 5 * 51
    assert (c1.price < 0).sum() == 3           # -$20 on the lowest node in 3 hours
    c2 = I.config2()
    assert (c2.T, c2.N, c2.K, c2.A, c2.n_modes) == (288, 1001, 20, 201, 2)
    lo, hi = c2.meta["negative_stretch"]
    assert hi - lo == 72 and np.all(c2.price[lo:hi, :4] < -30)
    c5 = I.config5()
    assert (c5.T, c5.N, c5.K, c5.A, c5.s0) == (288, 2001, 32, 201, 1000)


def test_rows_stochastic():
    for inst in (I.config1(), I.config2(), I.random_instance(3, 5, 9, 4, 2, 2)):
        P = inst.trans.astype(np.float64)
        assert np.all(P >= 0)
        np.testing.assert_allclose(P.sum(axis=2), 1.0, atol=1e-6)


def test_tauchen_moments():
    x, P = I.tauchen(41, 0.9, 0.2)
    # conditional mean of the next node is close to phi * x away from the edges
    mid = slice(10, 31)
    np.testing.assert_allclose((P @ x)[mid], 0.9 * x[mid], atol=0.02)
