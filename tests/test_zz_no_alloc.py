"""cheb_mu_search_noalloc against cheb_mu_search (GPU, through the C ABI).

The workspace-free entry point keeps its count weights in the library's static
device scratch; it must give the same mu search result as the workspace
version on consecutive calls with different inputs, and refuse expansions
longer than its scratch before launching anything.
"""

import numpy as np
import pytest
import torch

import paper_1704_00512_gb300 as cg
from paper_1704_00512_gb300 import _lib


def _spectral_moments(n_terms: int, n_levels: int, seed: int) -> np.ndarray:
    """g_k = sum_j T_k(x_j) for levels x_j in (-0.95, 0.95): the trace moments of
    a diagonal operator with S = I, so N(mu) counts levels below mu."""
    x = np.random.default_rng(seed).uniform(-0.95, 0.95, n_levels)
    k = np.arange(n_terms)[:, None]
    return np.cos(k * np.arccos(x)[None, :]).sum(axis=1)


def _both(g: np.ndarray, N_e: float, kT: float, kind: int, bracket=None):
    dev = torch.device("cuda:0")
    gd = torch.as_tensor(g, dtype=torch.float64, device=dev)
    n = g.shape[0]
    tol_N = 1e-8 * N_e
    ref = cg.decode_mu_result(cg.mu_search(gd, n, -1.0, 1.0, kind, kT, N_e, tol_N, bracket=bracket))
    got = cg.decode_mu_result(cg.mu_search_noalloc(gd, n, -1.0, 1.0, kind, kT, N_e, tol_N, bracket=bracket))
    return ref, got


def _assert_same(ref: dict, got: dict):
    assert got["iters"] == ref["iters"]
    assert got["converged"] == ref["converged"]
    assert got["bits"] == ref["bits"]
    assert got["mu"] == pytest.approx(ref["mu"], abs=1e-13)
    assert got["N"] == pytest.approx(ref["N"], rel=1e-12, abs=1e-12)


@pytest.mark.gpu
def test_noalloc_mu_search_matches_workspace_version_on_consecutive_calls():
    # first call on the device sets up the scratch address; the second reuses it
    g1 = _spectral_moments(2048, 300, seed=11)
    ref1, got1 = _both(g1, 150.0, 0.01, cg.FERMI)
    g2 = _spectral_moments(3000, 500, seed=12)
    ref2, got2 = _both(g2, 137.0, 0.02, cg.ERFC, bracket=(-0.9, 0.9))
    _assert_same(ref1, got1)
    _assert_same(ref2, got2)
    assert ref1["converged"] and ref2["converged"]
    # the two inputs differ, so a stale scratch would show up here
    assert abs(got1["mu"] - got2["mu"]) > 1e-6


@pytest.mark.gpu
def test_noalloc_mu_search_at_the_scratch_limit_and_beyond():
    n = _lib.MU_SEARCH_NOALLOC_MAX_TERMS
    g = _spectral_moments(n, 64, seed=13)
    ref, got = _both(g, 32.0, 0.005, cg.FERMI)
    _assert_same(ref, got)
    gd = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(cg.ChebError) as e:
        cg.mu_search_noalloc(gd, n + 1, -1.0, 1.0, cg.FERMI, 0.01, 1.0, 1e-6)
    assert e.value.code == _lib.ERR_INVALID
    assert "static scratch" in str(e.value)
