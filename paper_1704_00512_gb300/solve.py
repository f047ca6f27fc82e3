"""Solve sequences built from the C ABI (every numerical step runs in libcheb.so).

``powers``: matrix powers S^a from one shared recursion (Sec. "Matrix
powers"), optionally followed by one FP64 Newton-Schulz step for S^-1.

``foe``: the Fermi-operator expansion with the S^-1/2 transformation and the
mu search (Sec. "Fermi Operator Expansion"):
  1. block patterns P_H (cutoff r_c) and P_out (r_c + r_buf) from the atoms;
  2. S^-1/2 by a power expansion of S on P_out, and the trace functional
     G = (P_out(S^-1/2 P_out(S S^-1/2)))^T, so that Tr(F(mu) S) =
     sum_k c_k(mu) <T_k, G> (``overlap_setup``: both depend on S only, so a
     sequence of solves with one overlap matrix computes them once);
  3. H' = P_H(S^-1/2 P_out(H S^-1/2));
  4. Lanczos bounds of H', degree for the occupation function at the interval
     centre (the hardest position for a Chebyshev fit);
  5. pass 1: the recursion on H~' collecting Tr T_k (for the penalty check of
     Eq. 5, which widens a failing bound once and otherwise reports
     CHEB_ERR_BOUNDS) and g_k = <T_k, G>;
  6. bisection for Tr(F S) = N_e on g (no new products);
  7. pass 2: the recursion again, accumulating p at mu*;
  8. F = P_out(S^-1/2 P_out(p S^-1/2)) and Tr(FS).
The form "mu4" runs pass 1 over the first half of the terms only; the
bisection on those moments brackets mu* (the truncated series is a smoothed
Fermi function of the same filling), pass 2 accumulates p at the 4 Chebyshev
points of a bracket of half-width mu_half_kT * kT (the 4 simultaneous mu) and
collects all g_k, the bisection on all of them gives mu* exactly as in the
two-pass form, and p(mu*) is the Lagrange interpolant of the 4 accumulators
when mu* lies in the bracket (else a third pass runs at mu*).
Host code only sequences calls and moves a few scalars (bounds, degree, mu).
"""

from __future__ import annotations

import time

import numpy as np
import torch

from . import _lib as L


def _bsr_to_device(row_ptr, col_idx, vals, device) -> L.Bsr:
    return L.Bsr(torch.as_tensor(row_ptr, dtype=torch.int64, device=device),
                 torch.as_tensor(col_idx, dtype=torch.int32, device=device),
                 None if vals is None else torch.as_tensor(np.ascontiguousarray(vals), dtype=torch.float64,
                                                          device=device))


class Problem:
    """Device-resident inputs of one system: atoms, P_H with S and H, and P_out.

    order="hilbert" relabels the atoms along a Hilbert curve (cheb_locality_order)
    so that the column kernel's panels of consecutive columns hold atoms that lie
    close together; the patterns, S, H and every result are then in the new
    labelling, and set_H / to_caller_out move values from and to the caller's
    labelling (the patterns built from the caller's atoms)."""

    def __init__(self, xyz: np.ndarray, L_box: float, r_c: float, r_buf: float, S_vals: np.ndarray,
                 H_vals: np.ndarray, device, precision: int = L.F64, op_lists: bool = True,
                 order: str | None = None):
        self.device = torch.device(device)
        self.L = float(L_box)
        self.r_c = float(r_c)
        self.r_out = float(r_c + r_buf)
        self.xyz_caller = torch.as_tensor(np.ascontiguousarray(xyz), dtype=torch.float64, device=self.device)
        self.S_host = S_vals
        self.H_host = H_vals
        self.precision = precision
        self.op_lists = op_lists
        if order not in (None, "hilbert"):
            raise ValueError(f"unknown order {order!r}")
        self.perm = None
        if order == "hilbert":
            self.perm = L.locality_order(self.xyz_caller, self.L)
            self.xyz = L.gather_rows(self.xyz_caller.reshape(-1), self.perm, 3).view(-1, 3)
        else:
            self.xyz = self.xyz_caller
        self.build_patterns()
        S = torch.as_tensor(np.ascontiguousarray(S_vals), dtype=torch.float64, device=self.device)
        H = torch.as_tensor(np.ascontiguousarray(H_vals), dtype=torch.float64, device=self.device)
        if self.perm is not None:
            rp, ci = L.pattern_build(self.xyz_caller, self.L, self.r_c)
            self.P_H_caller = L.Bsr(rp, ci)
            rp, ci = L.pattern_build(self.xyz_caller, self.L, self.r_out)
            self.P_out_caller = L.Bsr(rp, ci)
            self.map_H = L.position_map(self.P_H, self.P_H_caller, self.perm)
            self.map_out = L.position_map(self.P_out, self.P_out_caller, self.perm)
            S = L.gather_rows(S.reshape(-1), self.map_H, 16).view(S.shape)
            H = L.gather_rows(H.reshape(-1), self.map_H, 16).view(H.shape)
        self.S = self.P_H.with_vals(S)
        self.H = self.P_H.with_vals(H)

    def set_H(self, vals: torch.Tensor):
        """New Hamiltonian values given in the caller's labelling (device, P_H order)."""
        if self.perm is None:
            self.H.vals.copy_(vals.view(self.H.vals.shape))
        else:
            L.gather_rows(vals.reshape(-1), self.map_H, 16, out=self.H.vals.view(-1))

    def to_caller_out(self, F: torch.Tensor) -> torch.Tensor:
        """Values on P_out (this problem's labelling) in the caller's labelling."""
        if self.perm is None:
            return F
        out = torch.zeros_like(F)
        return L.scatter_rows(F.reshape(-1), self.map_out, 16, out.view(-1)).view(F.shape)

    def build_patterns(self):
        rp, ci = L.pattern_build(self.xyz, self.L, self.r_c)
        self.P_H = L.Bsr(rp, ci)
        rp, ci = L.pattern_build(self.xyz, self.L, self.r_out)
        self.P_out = L.Bsr(rp, ci)
        self.plan64 = L.Plan(self.P_out, L.F64)
        self.planX = self.plan64 if self.precision == L.F64 else L.Plan(self.P_out, self.precision)
        if self.op_lists:
            # gather plan of the recursions on S~ and H~' (both on P_H)
            self.plan64.attach_operator(self.P_H)
            if self.planX is not self.plan64:
                self.planX.attach_operator(self.P_H)

    @property
    def n_rows(self) -> int:
        return 4 * (self.P_H.nbr)

    def zeros_out(self) -> torch.Tensor:
        return torch.zeros((self.P_out.nnzb, 4, 4), dtype=torch.float64, device=self.device)


def problem_from_system(sysm, r_buf: float, device, precision: int = L.F64, op_lists: bool = True,
                        order: str | None = None) -> Problem:
    return Problem(sysm.xyz, sysm.L, sysm.r_cut, r_buf, sysm.S, sysm.H, device, precision, op_lists, order)


def powers(pb: Problem, exponents=(-1.0, 0.5, -0.5), tol: float = 1e-10, n_max: int = 512,
           lanczos_k: int = 40, bounds_S=None, n_terms=None, newton_schulz: bool = False,
           precision: int | None = None, stepwise: bool | None = None) -> dict:
    """S^a for every a in exponents from one recursion on S~ (Sec. "Matrix powers").

    stepwise: one launch per step (None: above 1,000 block rows, where it was
    measured faster than the one-launch resident form on GB300, e.g. 56 vs 68
    ms per FP64 step at 10,000 atoms)."""
    prec = pb.precision if precision is None else precision
    plan = pb.plan64 if prec == L.F64 else pb.planX
    if bounds_S is None:
        e0, e1 = L.bounds_spd(pb.S, lanczos_k)
    else:
        e0, e1 = bounds_S
    St = pb.S.with_vals(L.scale(pb.S, e0, e1))
    funcs = [{"kind": L.POWER, "a": a} for a in exponents]
    if n_terms is None:
        n, c = L.coeffs(funcs, e0, e1, tol, n_max, rel=True, device=pb.device)
    else:
        n, c = L.coeffs(funcs, e0, e1, 0.0, n_terms, device=pb.device)
    accs = [pb.zeros_out() for _ in exponents]
    t = torch.zeros(n, dtype=torch.float64, device=pb.device)
    if stepwise is None:
        stepwise = pb.P_out.nbr > 1000
    L.expand(plan, St, n, c, accs, moments=t, precision=prec, stepwise=stepwise)
    out = {"bounds": (e0, e1), "n_terms": n, "coeffs": c, "acc": accs, "moments": t}
    if newton_schulz and -1.0 in exponents:
        X0 = accs[list(exponents).index(-1.0)]
        X1 = pb.zeros_out()
        tmp = pb.zeros_out()
        L.newton_schulz(pb.plan64, pb.S, X0, X1, tmp)
        out["inv_ns"] = X1
    return out


def orthogonalise(pb: Problem, A: torch.Tensor, energy: bool = False):
    """H' = P_H(A P_out(H A)), A = S^-1/2 on P_out.

    energy=True also returns the energy functional G_H = Z^T of the same
    product Z = P_out(A P_out(H A)) (<X, G_H> = Tr(P_out(A P_out(X A)) H))."""
    Y = pb.zeros_out()
    Z = pb.zeros_out()
    L.masked_product(pb.plan64, pb.H, A, Y)
    L.masked_product(pb.plan64, pb.P_out.with_vals(A), Y, Z)
    Hp = pb.P_H.with_vals(L.restrict(pb.P_out.with_vals(Z), pb.P_H))
    return (Hp, L.transpose(pb.plan64, Z)) if energy else Hp


def trace_functional(pb: Problem, A: torch.Tensor, M: L.Bsr | None = None) -> torch.Tensor:
    """G with <X, G> = Tr(P_out(A P_out(X A)) M): the transpose of P_out(A P_out(M A)).

    M = S (default) gives the electron count Tr(F S); M = H gives the energy
    Tr(F H) of the same kernel (M symmetric, its pattern within P_out)."""
    Y = pb.zeros_out()
    Z = pb.zeros_out()
    L.masked_product(pb.plan64, pb.S if M is None else M, A, Y)
    L.masked_product(pb.plan64, pb.P_out.with_vals(A), Y, Z)
    return L.transpose(pb.plan64, Z)


def postprocess(pb: Problem, A: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """F = P_out(A P_out(p A))."""
    Y = pb.zeros_out()
    F = pb.zeros_out()
    L.masked_product(pb.plan64, pb.P_out.with_vals(p), A, Y)
    L.masked_product(pb.plan64, pb.P_out.with_vals(A), Y, F)
    return F


def overlap_setup(pb: Problem, tol_S: float = 1e-10, lanczos_k: int = 40, bounds_S=None, n_S=None,
                  isqrt: str = "f64") -> dict:
    """S^-1/2 (A) and the trace-functional matrix G: the parts of the FOE that
    depend on the overlap only (steps 2 of the module docstring).

    isqrt: "f64" expands S^-1/2 in FP64; "f32ns" expands it in the problem's
    reduced precision and applies one FP64 Newton-Schulz correction."""
    if isqrt == "f32ns" and pb.precision != L.F64:
        pw = powers(pb, exponents=(-0.5,), tol=tol_S, bounds_S=bounds_S, n_terms=n_S, precision=pb.precision,
                    lanczos_k=lanczos_k)
        A = pb.zeros_out()
        L.newton_schulz_isqrt(pb.plan64, pb.S, pw["acc"][0], A, pb.zeros_out(), pb.zeros_out())
    else:
        pw = powers(pb, exponents=(-0.5,), tol=tol_S, bounds_S=bounds_S, n_terms=n_S, precision=L.F64,
                    lanczos_k=lanczos_k)
        A = pw["acc"][0]
    G = trace_functional(pb, A)
    return {"A": A, "G": G, "bounds_S": pw["bounds"], "n_S": pw["n_terms"]}


def penalty(t: torch.Tensor, m: int, alpha: float = -200.0, threshold: float = 1.0, terms: int = 512):
    """Eq. 5 on the first min(m, terms) traces t_k = Tr T_k of an expansion:
    (verdict, value), verdict 0 when the spectrum lies in the bounds, -1 / +1
    for the lower / upper bound, 2 for a non-finite trace.  |alpha| (scaled
    variable) is capped by the library at 2/5 of the terms, so that the penalty
    polynomial resolves it."""
    return L.penalty_check(t, min(m, terms), alpha, threshold)


def widen(bounds: tuple[float, float], verdict: int, frac: float) -> tuple[float, float]:
    """The bound the penalty verdict names, moved out by frac of the interval width."""
    return L.widen_bounds(bounds, verdict, frac)


def foe(pb: Problem, kT: float, N_e: float, tol: float = 1e-10, kind: int = L.FERMI, n_max: int = 16384,
        lanczos_k: int = 40, tol_N: float | None = None, bounds_S=None, n_S=None, bounds_H=None, n_H=None,
        max_iter: int = 100, form: str = "twopass", n_mu: int = 4, mu_half_kT: float = 0.02,
        overlap: dict | None = None, tol_S: float | None = None, penalty_alpha: float = -200.0,
        penalty_threshold: float = 1.0, penalty_widen: float = 0.05, penalty_terms: int = 512,
        energy: bool = False, stepwise: bool = True, isqrt: str = "f64", timings: dict | None = None) -> dict:
    """Density matrix F with Tr(F S) = N_e (see the module docstring for the steps).

    form: "twopass" (moment pass, bisection, accumulation pass) or "mu4" (a
    half-length moment pass brackets mu*, one pass accumulates n_mu mu at
    once and collects all moments, interpolation at mu*).  overlap: the
    result of overlap_setup for this problem's S (computed here if None).
    The penalty check (Eq. 5) runs on the first penalty_terms Tr T_k of pass 1
    with alpha = penalty_alpha in the scaled variable (|alpha| capped at 2/5 of
    the terms it is expanded in, so that the penalty polynomial resolves it):
    a failing bound is widened by penalty_widen of the interval width and pass
    1 repeated once; a second failure raises ChebError(ERR_BOUNDS).
    energy (two-pass form only): the accumulation pass also collects the
    energy moments e_k = <T_k, G_H> (G_H the energy functional of the overlap
    setup), so that Tr(K H) of any kernel re-summed from the same polynomials
    costs no new products (the beta check of Sec. "Fermi Operator Expansion").
    """
    if form not in ("twopass", "mu4"):
        raise ValueError(f"foe: unknown form {form!r}")
    if energy and form != "twopass":
        raise ValueError("foe: the energy moments ride on the second pass of the two-pass form")
    tm = {} if timings is None else timings
    t0 = time.perf_counter()
    tS = tol if tol_S is None else tol_S
    ov = overlap_setup(pb, tS, lanczos_k, bounds_S, n_S, isqrt) if overlap is None else overlap
    A, G = ov["A"], ov["G"]
    Hp, GH = orthogonalise(pb, A, True) if energy else (orthogonalise(pb, A), None)
    if bounds_H is None:
        e0, e1, _ = L.bounds(Hp, lanczos_k)
    else:
        e0, e1 = bounds_H
    if tol_N is None:
        tol_N = 1e-9 * N_e if pb.precision in (L.F64, L.F64X) else 1e-6 * N_e
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ws = None
    checks = []
    for attempt in range(2):
        Hpt = Hp.with_vals(L.scale(Hp, e0, e1))
        if n_H is None:
            n, _ = L.coeffs([{"kind": kind, "mu": 0.5 * (e0 + e1), "kT": kT}], e0, e1, tol, n_max, device=pb.device)
        else:
            n = n_H
        m = n // 2 if form == "mu4" else n
        tm["setup_s"] = time.perf_counter() - t0
        t = torch.zeros(m, dtype=torch.float64, device=pb.device)
        g = torch.zeros(m, dtype=torch.float64, device=pb.device)
        ev[0].record()
        ws = L.expand(pb.planX, Hpt, m, None, [], moments=t, G=G, gmoments=g, precision=pb.precision, ws=ws,
                      stepwise=stepwise)
        ev[1].record()
        verdict, value = penalty(t, m, penalty_alpha, penalty_threshold, penalty_terms)
        checks.append((verdict, value, (e0, e1)))
        if verdict == 0:
            break
        if attempt == 1:
            raise L.ChebError(L.ERR_BOUNDS, f"penalty check (Eq. 5) failed twice: trace {value:g} on [{e0}, {e1}]")
        e0, e1 = widen((e0, e1), verdict, penalty_widen)
    passes = 1
    em = None
    if form == "twopass":
        res = L.mu_search(g, n, e0, e1, kind, kT, N_e, tol_N, max_iter)
        r = L.decode_mu_result(res)
        mu = r["mu"]
        _, c = L.coeffs([{"kind": kind, "mu": mu, "kT": kT}], e0, e1, 0.0, n, device=pb.device)
        p = pb.zeros_out()
        em = torch.zeros(n, dtype=torch.float64, device=pb.device) if energy else None
        ev[2].record()
        L.expand(pb.planX, Hpt, n, c, [p], G=GH, gmoments=em, precision=pb.precision, ws=ws, stepwise=stepwise)
        ev[3].record()
        passes = 2
        mus, gm = [mu], g
        r_half = None
    else:
        r_half = L.decode_mu_result(L.mu_search(g, m, e0, e1, kind, kT, N_e, tol_N, max_iter))
        mus = L.mu_nodes(r_half["mu"], mu_half_kT * kT, n_mu)
        _, c = L.coeffs([{"kind": kind, "mu": x, "kT": kT} for x in mus], e0, e1, 0.0, n, device=pb.device)
        accs = [pb.zeros_out() for _ in mus]
        gm = torch.zeros(n, dtype=torch.float64, device=pb.device)
        ev[2].record()
        L.expand(pb.planX, Hpt, n, c, accs, G=G, gmoments=gm, precision=pb.precision, ws=ws, stepwise=stepwise)
        ev[3].record()
        passes = 2
        r = L.decode_mu_result(L.mu_search(gm, n, e0, e1, kind, kT, N_e, tol_N, max_iter))
        mu = r["mu"]
        p = pb.zeros_out()
        ev[4].record()
        if abs(mu - r_half["mu"]) <= mu_half_kT * kT:
            L.lincomb(L.lagrange_weights(mus, mu), accs, p)
        else:
            _, c3 = L.coeffs([{"kind": kind, "mu": mu, "kT": kT}], e0, e1, 0.0, n, device=pb.device)
            L.expand(pb.planX, Hpt, n, c3, [p], precision=pb.precision, ws=ws, stepwise=stepwise)
            passes = 3
        ev[5].record()
    F = postprocess(pb, A, p)
    trFS = L.trace(pb.P_out.with_vals(F), pb.S)
    tm["events"] = ev
    tm["form"] = form
    return {"F": F, "p": p, "mus": mus, "A": A, "Hp": Hp, "G": G, "mu": mu, "mu_result": r, "mu_half": r_half,
            "moments": t, "gmoments": gm, "n_terms": n, "n_pass1": m, "passes": passes, "bounds_H": (e0, e1),
            "bounds_S": ov["bounds_S"], "n_S": ov["n_S"], "trace_FS": trFS, "penalty": checks,
            "emoments": em, "G_H": GH, "kT": kT, "kind": kind, "N_e": N_e, "tol_N": tol_N}


def energy_pair(pb: Problem, r: dict, kT_prime: float, max_iter: int = 100) -> dict:
    """E = Tr(K H) of a two-pass solve r (foe with energy=True) and E' = Tr(K' H)
    of the kernel K' with the wider smearing kT_prime, both re-summed from r's
    moments: K' takes its own mu' (bisection on the same trace moments, so that
    Tr(K' S) = N_e too) and its coefficient set, and no new products."""
    em = r.get("emoments")
    if em is None:
        raise ValueError("energy_pair: the solve did not collect energy moments (foe(..., energy=True))")
    n, (e0, e1), kind = r["n_terms"], r["bounds_H"], r["kind"]
    _, c = L.coeffs([{"kind": kind, "mu": r["mu"], "kT": r["kT"]}], e0, e1, 0.0, n, device=pb.device)
    rp = L.decode_mu_result(L.mu_search(r["gmoments"], n, e0, e1, kind, kT_prime, r["N_e"], r["tol_N"], max_iter))
    _, cp = L.coeffs([{"kind": kind, "mu": rp["mu"], "kT": kT_prime}], e0, e1, 0.0, n, device=pb.device)
    E = L.series_value(c[0], em, n)
    Ep = L.series_value(cp[0], em, n)
    return {"E": E, "E_prime": Ep, "mu_prime": rp["mu"], "mu_prime_result": rp}


def foe_auto_kT(pb: Problem, kT0: float, N_e: float, dE_tol: float, widen: float = 1.25, shrink: float = 0.5,
                kT_min: float = 1e-4, max_rounds: int = 8, **kw) -> dict:
    """Smearing chosen on the fly (Sec. "Fermi Operator Expansion"): solve with
    kT, compare E = Tr(K H) with E' = Tr(K' H) of the same polynomials at
    kT' = widen kT; accept when |E - E'| <= dE_tol, otherwise solve again with
    kT <- shrink kT (more terms) until kT_min.  kw goes to foe (two-pass form,
    energy moments on); the overlap setup and the bounds of H are kept across
    rounds.  Returns the accepted solve with "kT", "E", "E_prime" and the
    "rounds" history [(kT, n_terms, E, E', accepted)]."""
    if not (widen > 1.0 and 0.0 < shrink < 1.0 and dE_tol > 0.0):
        raise ValueError("foe_auto_kT: need widen > 1, 0 < shrink < 1, dE_tol > 0")
    kw = dict(kw)
    if kw.pop("n_H", None) is not None:
        raise ValueError("foe_auto_kT: the term count follows kT (Eq. 6); n_H cannot be fixed")
    kw["form"], kw["energy"] = "twopass", True
    if kw.get("overlap") is None:
        tS = kw.get("tol_S") or kw.get("tol", 1e-10)
        kw["overlap"] = overlap_setup(pb, tS, kw.get("lanczos_k", 40), kw.get("bounds_S"), kw.get("n_S"),
                                      kw.get("isqrt", "f64"))
    rounds = []
    kT = kT0
    while True:
        r = foe(pb, kT, N_e, **kw)
        kw["bounds_H"] = r["bounds_H"]
        ep = energy_pair(pb, r, widen * kT, kw.get("max_iter", 100))
        E, Ep = float(ep["E"].item()), float(ep["E_prime"].item())
        ok = abs(E - Ep) <= dE_tol
        rounds.append((kT, r["n_terms"], E, Ep, ok))
        if ok or len(rounds) == max_rounds or shrink * kT < kT_min:
            r.update(ep)
            r.update({"E": E, "E_prime": Ep, "rounds": rounds, "accepted": ok})
            return r
        kT *= shrink


def selected_eigenvalues(pb: Problem, kT: float, intervals=(), levels=(), tol: float = 1e-9, n_max: int = 16384,
                         lanczos_k: int = 40, tol_S: float = 1e-10, bounds_S=None, n_S=None, bounds_H=None,
                         tol_N: float = 1e-10) -> dict:
    """Sec. "Extraction of selected eigenvalues": eigenvalue counts and levels.

    For each interval (lo, hi) the projector Q = f_FD(H; hi) - f_FD(H; lo) is
    accumulated (one FP64 accumulator each, all in one recursion) and post-
    processed like F; Tr(Q S) counts the eigenvalues in (lo, hi).  For each
    level N the bisection on the trace functional of the same recursion finds
    the mu with Tr(F(mu) S) = N - 1/2, which lies at the N-th eigenvalue when
    kT is small against the gaps around it."""
    pw = powers(pb, exponents=(-0.5,), tol=tol_S, bounds_S=bounds_S, n_terms=n_S, precision=L.F64)
    A = pw["acc"][0]
    Hp = orthogonalise(pb, A)
    e0, e1 = L.bounds(Hp, lanczos_k)[:2] if bounds_H is None else bounds_H
    Hpt = Hp.with_vals(L.scale(Hp, e0, e1))
    G = trace_functional(pb, A)
    funcs = [{"kind": L.INTERVAL, "lo": lo, "hi": hi, "kT": kT} for lo, hi in intervals]
    fdeg = funcs + [{"kind": L.FERMI, "mu": 0.5 * (e0 + e1), "kT": kT}]
    n, _ = L.coeffs(fdeg, e0, e1, tol, n_max, device=pb.device)
    c = L.coeffs(funcs, e0, e1, 0.0, n, device=pb.device)[1] if funcs else None
    accs = [pb.zeros_out() for _ in funcs]
    g = torch.zeros(n, dtype=torch.float64, device=pb.device)
    L.expand(pb.plan64, Hpt, n, c, accs, G=G, gmoments=g, precision=L.F64, stepwise=True)
    counts, Qs = [], []
    for Q in accs:
        Qp = postprocess(pb, A, Q)
        Qs.append(Qp)
        counts.append(float(L.trace(pb.P_out.with_vals(Qp), pb.S).item()))
    eigs = []
    for N in levels:
        r = L.decode_mu_result(L.mu_search(g, n, e0, e1, L.FERMI, kT, N - 0.5, tol_N, 128))
        eigs.append(r["mu"])
    return {"counts": counts, "Q": Qs, "eigenvalues": eigs, "n_terms": n, "bounds_H": (e0, e1),
            "bounds_S": pw["bounds"], "n_S": pw["n_terms"], "gmoments": g}


def foe_solve(sysm, r_buf: float, kT: float, N_e: float, tol: float = 1e-10, precision: int = L.F64,
              device="cuda", order: str | None = None, **kw) -> dict:
    """foe() on a synthetic system, with host copies of the main results (F_host
    in the caller's labelling)."""
    pb = problem_from_system(sysm, r_buf, device, precision, order=order)
    out = foe(pb, kT, N_e, tol=tol, **kw)
    torch.cuda.synchronize(pb.device)
    out["problem"] = pb
    out["F_host"] = pb.to_caller_out(out["F"]).cpu().numpy()
    out["trace_FS"] = float(out["trace_FS"].item())
    return out
