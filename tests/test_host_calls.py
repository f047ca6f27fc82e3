"""Host-only calls of the library (no GPU needed): the bound widening after a
penalty verdict (Eq. 5, penalty passage of Sec. "Determination of the
eigenvalue bounds and polynomial degree") and the bracket a network output
proposes (the scaling of Eq. 2 undone)."""
import math

import numpy as np
import pytest

L = pytest.importorskip("paper_1704_00512_gb300._lib")


@pytest.mark.parametrize("verdict,expect", [(0, (-2.0, 3.0)), (-1, (-2.5, 3.0)), (1, (-2.0, 3.5)),
                                            (2, (-2.5, 3.5))])
def test_widen_moves_the_named_bound_by_a_fraction_of_the_width(verdict, expect):
    assert L.widen_bounds((-2.0, 3.0), verdict, 0.1) == pytest.approx(expect, abs=0)


@pytest.mark.parametrize("bounds,verdict,frac", [((1.0, 0.0), 1, 0.1), ((0.0, 1.0), 3, 0.1),
                                                 ((0.0, 1.0), -2, 0.1), ((0.0, 1.0), 1, -0.1)])
def test_widen_refuses_bad_arguments(bounds, verdict, frac):
    with pytest.raises(L.ChebError) as e:
        L.widen_bounds(bounds, verdict, frac)
    assert e.value.code == L.ERR_INVALID


def test_bracket_maps_the_scaled_guess_back_through_eq2():
    rng = np.random.default_rng(3)
    for _ in range(50):
        e0 = rng.uniform(-10, -1)
        e1 = rng.uniform(1, 10)
        kT = rng.uniform(0.002, 0.05)
        o = np.array([rng.uniform(-1, 1), rng.uniform(-9, 0)], dtype=np.float32)
        mu, half = L.mlp_bracket(o, e0, e1, kT, 0.05, 1.0)
        # Eq. 2: x~ = (e - tau) * 2 / (emax - emin); the guess is the level whose
        # scaled value is out[0]
        assert (mu - 0.5 * (e0 + e1)) * 2.0 / (e1 - e0) == pytest.approx(float(o[0]), rel=1e-12, abs=1e-15)
        raw = math.exp(float(o[1])) * (e1 - e0) / 2.0
        assert half == pytest.approx(min(max(raw, 0.05 * kT), kT), rel=1e-12)
        assert 0.05 * kT <= half <= kT


def test_bracket_refuses_an_empty_interval():
    with pytest.raises(L.ChebError):
        L.mlp_bracket([0.0, 0.0], 1.0, 1.0, 0.01, 0.05, 1.0)
    with pytest.raises(L.ChebError):
        L.mlp_bracket([0.0, 0.0], 0.0, 1.0, 0.01, 2.0, 1.0)


def test_hilbert_reference_visits_face_adjacent_cells():
    # the reference order used by the GPU test of cheb_locality_order: the first
    # 16^3 indices of a Hilbert curve fill the corner cube, one face step apart
    from hilbert_ref import hilbert_keys_ref
    g = np.stack(np.meshgrid(*[np.arange(16)] * 3, indexing="ij"), -1).reshape(-1, 3)
    k = hilbert_keys_ref(g + 0.5, 1024.0)
    o = np.argsort(k)
    assert np.array_equal(k[o], np.arange(16 ** 3))
    assert np.all(np.abs(np.diff(g[o], axis=0)).sum(axis=1) == 1)
