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
    """The C ABI's default start vector: v_i = 1 + u_i / 2 with u_i the top 53
    bits of SplitMix64(i) over 2^53 (a positive vector with a component along
    every eigenvector; the all-ones vector can lie in a small invariant subspace)."""
    from .mlp import splitmix64
    u = (splitmix64(np.arange(n_rows, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    return 1.0 + 0.5 * u


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
        tol_N: float, kind: int = ref.KIND_FERMI, max_iter: int = 100, energy: bool = False):
    """FOE with the S^-1/2 transformation and bisection on the trace functional.

    energy: the second pass also collects the energy moments e_k = <T_k, G_H>."""
    A = powers(S, P_out, (-0.5,), bounds_S, n_S)["acc"][0]
    Hp = ref.orthogonalise(H, A, P_out)
    e0, e1 = bounds_H
    Hpt = ref.scale(Hp, e0, e1)
    G = ref.trace_functional_matrix(A, S, P_out)
    ex0 = ref.chebyshev_expand(Hpt, P_out, np.zeros((1, n_H)), G=G)
    ms = ref.mu_bisect(ex0.g, kind, kT, e0, e1, N_e, tol_N, max_iter)
    c = ref.cheb_coeffs(ref.Func(kind, mu=ms.mu, kT=kT), n_H, e0, e1)
    GH = ref.trace_functional_matrix(A, H, P_out) if energy else None
    ex = ref.chebyshev_expand(Hpt, P_out, c[None], G=GH)
    F = ref.postprocess(ex.acc[0], A, P_out)
    return {"F": F, "p": ex.acc[0], "A": A, "Hp": Hp, "G": G, "mu": ms, "moments": ex0.t, "gmoments": ex0.g,
            "trace_FS": ref.trace_product(F, S), "G_H": GH, "emoments": ex.g if energy else None,
            "kT": kT, "kind": kind, "bounds_H": (e0, e1), "n_terms": n_H, "N_e": N_e, "tol_N": tol_N}


def energy_pair(r: dict, kT_prime: float, max_iter: int = 100) -> dict:
    """E = Tr(K H) of a solve with energy moments, and E' = Tr(K' H) of the
    kernel with the wider smearing kT_prime at its own mu' (Tr(K' S) = N_e by
    the same bisection on the same trace moments); both are re-sums."""
    e0, e1 = r["bounds_H"]
    E = ref.energy(r["emoments"], ref.Func(r["kind"], mu=r["mu"].mu, kT=r["kT"]), e0, e1)
    msp = ref.mu_bisect(r["gmoments"], r["kind"], kT_prime, e0, e1, r["N_e"], r["tol_N"], max_iter)
    Ep = ref.energy(r["emoments"], ref.Func(r["kind"], mu=msp.mu, kT=kT_prime), e0, e1)
    return {"E": E, "E_prime": Ep, "mu_prime": msp}


def foe_auto_kT(S: ref.Bsr, H: ref.Bsr, P_out: ref.Bsr, kT0: float, N_e: float, dE_tol: float, bounds_S, n_S: int,
                bounds_H, tol: float, n_max: int, tol_N: float, widen: float = 1.25, shrink: float = 0.5,
                kT_min: float = 1e-4, max_rounds: int = 8, kind: int = ref.KIND_FERMI):
    """The smearing chosen on the fly (Sec. "Fermi Operator Expansion"): solve at
    kT with the degree of Eq. 6; compare E with E' at widen*kT; accept when
    |E - E'| <= dE_tol, else repeat at shrink*kT.  Returns the accepted solve
    with the history [(kT, n, E, E', accepted)] under "rounds"."""
    e0, e1 = bounds_H
    rounds = []
    kT = kT0
    while True:
        n = ref.choose_degree(ref.Func(kind, mu=0.5 * (e0 + e1), kT=kT), e0, e1, tol, n_max)
        r = foe(S, H, P_out, kT, N_e, bounds_S, n_S, bounds_H, n, tol_N, kind, energy=True)
        ep = energy_pair(r, widen * kT)
        ok = abs(ep["E"] - ep["E_prime"]) <= dE_tol
        rounds.append((kT, n, ep["E"], ep["E_prime"], ok))
        if ok or len(rounds) == max_rounds or shrink * kT < kT_min:
            r.update(ep)
            r.update({"rounds": rounds, "accepted": ok})
            return r
        kT *= shrink
