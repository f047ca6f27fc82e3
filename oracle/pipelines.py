"""Oracle versions of the solve sequences -- TEST INFRASTRUCTURE ONLY.

Same steps as the paper describes (Sec. "Fermi Operator Expansion", Sec. "Matrix
powers"), each by the plain functions of ``oracle.ref``.  Spectral bounds and
term counts can be passed in so that an expansion parity test does not depend on
the rounding of a Lanczos run (the two sides' Lanczos runs are compared on
their own).
"""

from __future__ import annotations

import numpy as np

from . import ref


def system_mats(sysm, r_buf: float):
    """S, H on P_H and the pattern P_out (r_c + r_buf) for a synth.System."""
    S = ref.Bsr(sysm.row_ptr, sysm.col_idx, sysm.S)
    H = ref.Bsr(sysm.row_ptr, sysm.col_idx, sysm.H)
    rp, ci = ref.pattern(sysm.xyz, sysm.L, sysm.r_cut + r_buf)
    return S, H, ref.Bsr(rp, ci, None)


def lanczos_start(n_rows: int) -> np.ndarray:
    """The all-ones start vector (the C ABI's default)."""
    return np.ones(n_rows)


def powers(S: ref.Bsr, P_out: ref.Bsr, exponents, bounds, n_terms: int, newton_schulz: bool = False):
    e0, e1 = bounds
    St = ref.scale(S, e0, e1)
    coeffs = np.stack([ref.cheb_coeffs(ref.Func(ref.KIND_POWER, a=a), n_terms, e0, e1) for a in exponents])
    ex = ref.chebyshev_expand(St, P_out, coeffs)
    out = {"acc": ex.acc, "moments": ex.t}
    if newton_schulz and -1.0 in exponents:
        out["inv_ns"] = ref.newton_schulz(S, ex.acc[list(exponents).index(-1.0)], P_out)
    return out


def foe(S: ref.Bsr, H: ref.Bsr, P_out: ref.Bsr, kT: float, N_e: float, bounds_S, n_S: int, bounds_H, n_H: int,
        tol_N: float, kind: int = ref.KIND_FERMI, max_iter: int = 100):
    """FOE with the S^-1/2 transformation and bisection on the trace functional."""
    A = powers(S, P_out, (-0.5,), bounds_S, n_S)["acc"][0]
    Hp = ref.orthogonalise(H, A, P_out)
    e0, e1 = bounds_H
    Hpt = ref.scale(Hp, e0, e1)
    G = ref.trace_functional_matrix(A, S, P_out)
    ex0 = ref.chebyshev_expand(Hpt, P_out, np.zeros((1, n_H)), G=G)
    ms = ref.mu_bisect(ex0.g, kind, kT, e0, e1, N_e, tol_N, max_iter)
    c = ref.cheb_coeffs(ref.Func(kind, mu=ms.mu, kT=kT), n_H, e0, e1)
    ex = ref.chebyshev_expand(Hpt, P_out, c[None])
    F = ref.postprocess(ex.acc[0], A, P_out)
    return {"F": F, "p": ex.acc[0], "A": A, "Hp": Hp, "G": G, "mu": ms, "moments": ex0.t, "gmoments": ex0.g,
            "trace_FS": ref.trace_product(F, S)}
