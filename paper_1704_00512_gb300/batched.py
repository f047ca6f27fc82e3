"""Batched density matrices: many independent systems of uneven size.

Each system follows the FOE of Sec. "Fermi Operator Expansion" with its own
spectral bounds, degree and mu; the recursions of all systems run in one
persistent launch per pass (columns are independent, Sec. "Expansion in
Chebyshev polynomials", so the block-diagonal concatenation of the systems is
expanded panel by panel, no panel straddling two systems):

  1. patterns P_H_i, P_out_i and S_i, H_i of every system, concatenated
     block-diagonally (cheb_block_diag);
  2. bounds of every S_i (Lanczos), S^-1/2 of all systems by one batched FP64
     power expansion (each system with its own bounds and degree);
  3. H' = P_H(S^-1/2 P_out(H S^-1/2)) on the concatenation, bounds of every
     H'_i, H~'_i scaled with its own bounds, degree n_i at the centre of its
     interval, and the trace functional G;
  4. pass 1: one batched launch with G gives g_k of every system, then every
     system's bisection for Tr(F_i S_i) = N_e,i on its own g;
  5. coefficients of every system at its mu*_i (host calls, between passes);
  6. pass 2: one batched launch accumulating every p_i, post-processing
     F = P_out(S^-1/2 P_out(p S^-1/2)) and Tr(F_i S_i) per system.

The expansion of pass 4 and all of pass 6 are captured in CUDA graphs on the
first solve and replayed on later solves of the same batch (same patterns,
degrees and buffers; new H values, as in the iterations of a self-consistent
loop); the bisections run outside the graphs, since each takes its system's
bounds, kT and N_e as launch arguments.  The tile shape of
the batched launch is chosen by `autotune_tile`, which times every shape of
the library's table on the batch and caches the fastest.

Every numerical step runs in libcheb.so; this module sequences calls.
"""

from __future__ import annotations

import time

import numpy as np
import torch

from . import _lib as L
from . import solve


def _slice_bsr(pattern: L.Bsr, vals: torch.Tensor, b0: int) -> L.Bsr:
    """System view: its own pattern with its contiguous block range of the concatenated values."""
    return L.Bsr(pattern.row_ptr, pattern.col_idx, vals[b0:b0 + pattern.nnzb])


_TILE_CACHE: dict = {}


def autotune_tile(P_out: L.Bsr, starts, precision: int, Mt: L.Bsr, probe_terms: int = 24, reps: int = 2,
                  log=None) -> int:
    """Fastest tile shape of the batched launch on this batch (CUDA-event timing).

    Every tile of the precision's table whose plan can be built is timed on a
    probe_terms-term moment expansion of Mt; the result is cached per (pattern
    size, system starts, precision)."""
    key = (P_out.nbr, P_out.nnzb, tuple(int(x) for x in starts), precision)
    if key in _TILE_CACHE:
        return _TILE_CACHE[key]
    nsys = len(starts) - 1
    dev = Mt.vals.device
    n_terms = torch.full((nsys,), probe_terms, dtype=torch.int32, device=dev)
    mom = torch.zeros((nsys, probe_terms), dtype=torch.float64, device=dev)
    best, best_ms, timings = None, float("inf"), {}
    for tile in range(len(L.tile_shapes(precision))):
        try:
            plan = L.BatchedPlan(P_out, starts, precision, tile)
        except L.ChebError as e:
            timings[tile] = f"unavailable ({e})"
            continue
        ws = L.expand_batched(plan, Mt, probe_terms, n_terms, None, None, 0, [], moments=mom,
                              moment_stride=probe_terms, precision=precision)
        ms = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            L.expand_batched(plan, Mt, probe_terms, n_terms, None, None, 0, [], moments=mom,
                             moment_stride=probe_terms, precision=precision, ws=ws)
            e1.record()
            e1.synchronize()
            ms = min(ms, e0.elapsed_time(e1))
        timings[tile] = ms
        if ms < best_ms:
            best, best_ms = tile, ms
        del plan, ws
    if best is None:
        raise L.ChebError(L.ERR_NOSPACE, f"no tile shape fits this batch: {timings}")
    if log:
        log(f"autotune precision={precision}: " + ", ".join(
            f"{t}{L.tile_shapes(precision)[t]}={v if isinstance(v, str) else f'{v:.2f} ms'}"
            for t, v in timings.items()) + f" -> tile {best}")
    _TILE_CACHE[key] = best
    return best


class BatchedProblem:
    """Device-resident batch of independent synthetic systems (synth.System)."""

    def __init__(self, systems, r_buf: float, device, precision: int = L.F32, tune: bool = True, log=None):
        self.device = torch.device(device)
        self.systems = systems
        self.precision = precision
        self.nsys = len(systems)
        self.PH, self.Pout = [], []
        Sp, Hp = [], []
        for s in systems:
            xyz = torch.as_tensor(np.ascontiguousarray(s.xyz), dtype=torch.float64, device=self.device)
            rp, ci = L.pattern_build(xyz, s.L, s.r_cut)
            ph = L.Bsr(rp, ci)
            rp, ci = L.pattern_build(xyz, s.L, s.r_cut + r_buf)
            self.PH.append(ph)
            self.Pout.append(L.Bsr(rp, ci))
            Sp.append(ph.with_vals(torch.as_tensor(np.ascontiguousarray(s.S), dtype=torch.float64,
                                                   device=self.device)))
            Hp.append(ph.with_vals(torch.as_tensor(np.ascontiguousarray(s.H), dtype=torch.float64,
                                                   device=self.device)))
        self.S = L.block_diag(Sp)
        self.H = self.S.with_vals(L.block_diag(Hp).vals)
        self.P_H = L.Bsr(self.S.row_ptr, self.S.col_idx)
        self.P_out = L.block_diag(self.Pout, with_vals=False)
        self.starts = [0]
        for s in systems:
            self.starts.append(self.starts[-1] + s.n_atoms)
        self.hoff = np.concatenate([[0], np.cumsum([p.nnzb for p in self.PH])]).astype(np.int64)
        self.ooff = np.concatenate([[0], np.cumsum([p.nnzb for p in self.Pout])]).astype(np.int64)
        self.plan64 = L.Plan(self.P_out, L.F64)
        self.tune = tune
        self.log = log
        self.tiles = {}
        self.graphs = {}

    def zeros_out(self) -> torch.Tensor:
        return torch.zeros((self.P_out.nnzb, 4, 4), dtype=torch.float64, device=self.device)

    def batched_plan(self, precision: int, Mt: L.Bsr) -> L.BatchedPlan:
        if precision not in self.tiles:
            self.tiles[precision] = (autotune_tile(self.P_out, self.starts, precision, Mt, log=self.log)
                                     if self.tune else -1)
        plan = L.BatchedPlan(self.P_out, self.starts, precision, self.tiles[precision])
        # every batched expansion here runs on an operator with the pattern of P_H
        return plan.attach_operator(self.P_H)


def _pack_coeffs(funcs_per_sys, bounds, n_terms, device) -> tuple[torch.Tensor, torch.Tensor]:
    """One coefficient vector per system at offsets [sum of earlier n_i] (Eq. 4, given degrees)."""
    off = np.concatenate([[0], np.cumsum(n_terms)]).astype(np.int64)
    buf = torch.zeros(int(off[-1]), dtype=torch.float64, device=device)
    for i, (f, (e0, e1), n) in enumerate(zip(funcs_per_sys, bounds, n_terms)):
        L.coeffs([f], e0, e1, 0.0, int(n), device=device, out=buf[off[i]:off[i + 1]])
    return buf, torch.as_tensor(off[:-1], dtype=torch.int64, device=device)


def prepare_batched(bp: BatchedProblem, kT, tol: float = 1e-7, tol_S: float = 1e-10, kind: int = L.FERMI,
                    lanczos_k: int = 40, n_max: int = 16384, bounds_H=None) -> dict:
    """Steps 2-3 of the module docstring: S^-1/2, H~', per-system bounds and degrees, G.

    kT: one smearing for every system, or a list with one per system (it sets
    each system's degree).  bounds_H: per-system bounds of H' to use instead of
    Lanczos (a warm start, e.g. the previous step's; None entries run Lanczos)."""
    dev = bp.device
    nsys = bp.nsys
    kTs = list(kT) if isinstance(kT, (list, tuple, np.ndarray)) else [kT] * nsys
    # --- S^-1/2 of every system: one batched FP64 power expansion
    bS = []
    for i in range(nsys):
        bS.append(L.bounds_spd(_slice_bsr(bp.PH[i], bp.S.vals, bp.hoff[i]), lanczos_k))
    St = torch.empty_like(bp.S.vals)
    for i in range(nsys):
        L.scale(_slice_bsr(bp.PH[i], bp.S.vals, bp.hoff[i]), *bS[i], out=St[bp.hoff[i]:bp.hoff[i + 1]])
    St = bp.S.with_vals(St)
    fS = {"kind": L.POWER, "a": -0.5}
    nS = [L.coeffs([fS], e0, e1, tol_S, 512, rel=True, device=dev)[0] for e0, e1 in bS]
    cS, oS = _pack_coeffs([fS] * nsys, bS, nS, dev)
    plan64 = bp.batched_plan(L.F64, St)
    A = bp.zeros_out()
    L.expand_batched(plan64, St, max(nS), torch.as_tensor(nS, dtype=torch.int32, device=dev), cS, oS, 0, [A],
                     precision=L.F64)
    # --- H' on the concatenation, per-system bounds, scaling and degree
    Y, Z = bp.zeros_out(), bp.zeros_out()
    L.masked_product(bp.plan64, bp.H, A, Y)
    L.masked_product(bp.plan64, bp.P_out.with_vals(A), Y, Z)
    Hp_vals = L.restrict(bp.P_out.with_vals(Z), bp.P_H)
    bH, nH = [], []
    Hpt = torch.empty_like(Hp_vals)
    for i in range(nsys):
        Hi = _slice_bsr(bp.PH[i], Hp_vals, bp.hoff[i])
        if bounds_H is not None and bounds_H[i] is not None:
            e0, e1 = bounds_H[i]
        else:
            e0, e1, _ = L.bounds(Hi, lanczos_k)
        bH.append((e0, e1))
        L.scale(Hi, e0, e1, out=Hpt[bp.hoff[i]:bp.hoff[i + 1]])
        nH.append(L.coeffs([{"kind": kind, "mu": 0.5 * (e0 + e1), "kT": kTs[i]}], e0, e1, tol, n_max,
                           device=dev)[0])
    Hpt = bp.P_H.with_vals(Hpt)
    # trace functional G = transpose of P_out(A P_out(S A))
    L.masked_product(bp.plan64, bp.S, A, Y)
    L.masked_product(bp.plan64, bp.P_out.with_vals(A), Y, Z)
    G = L.transpose(bp.plan64, Z)
    return {"A": A, "Hpt": Hpt, "G": G, "bounds_S": bS, "n_S": nS, "bounds_H": bH, "n_terms": nH}


def foe_batched(bp: BatchedProblem, kT: float, N_e: list[float], tol: float = 1e-7, tol_S: float = 1e-10,
                kind: int = L.FERMI, lanczos_k: int = 40, n_max: int = 16384, max_iter: int = 100,
                tol_N: list[float] | None = None, use_graphs: bool = True, bounds_H=None,
                penalty_alpha: float = -200.0, penalty_threshold: float = 1.0, penalty_terms: int = 512,
                timings: dict | None = None) -> dict:
    """Density matrices of every system of the batch (see the module docstring).

    Pass 1 also collects every system's Tr T_k; the penalty check of Eq. 5 runs
    on them before the bisections, and a system whose spectrum leaves its bounds
    raises ChebError(ERR_BOUNDS) naming the system and the bound (the plain
    solve.foe widens and retries; a batch shares its passes).  bounds_H: as in
    prepare_batched."""
    tm = {} if timings is None else timings
    dev = bp.device
    t0 = time.perf_counter()
    nsys = bp.nsys
    pr = prepare_batched(bp, kT, tol, tol_S, kind, lanczos_k, n_max, bounds_H)
    A, Hpt, G, bS, nS, bH, nH = (pr[k] for k in ("A", "Hpt", "G", "bounds_S", "n_S", "bounds_H", "n_terms"))
    torch.cuda.synchronize(dev)
    tm["setup_s"] = time.perf_counter() - t0

    kmax = max(nH)
    planX = bp.batched_plan(bp.precision, Hpt)
    key = (tuple(nH), bp.precision)
    st = bp.graphs.get(key)
    if st is None or not use_graphs:
        # buffers the captured passes read and write (kept for replays)
        st = {"nt": torch.as_tensor(nH, dtype=torch.int32, device=dev),
              "Hpt": Hpt.vals.clone(), "A": A.clone(), "G": G.clone(),
              "g": torch.zeros((nsys, kmax), dtype=torch.float64, device=dev),
              "t": torch.zeros((nsys, kmax), dtype=torch.float64, device=dev),
              "res": torch.zeros((nsys, 48), dtype=torch.uint8, device=dev),
              "mws": [L._ws(8 * n, dev) for n in nH],
              "c": torch.zeros(int(sum(nH)), dtype=torch.float64, device=dev),
              "coff": torch.as_tensor(np.concatenate([[0], np.cumsum(nH)[:-1]]), dtype=torch.int64, device=dev),
              "p": bp.zeros_out(), "Y": bp.zeros_out(), "F": bp.zeros_out(),
              "tr": torch.zeros(nsys, dtype=torch.float64, device=dev),
              "planX": planX}
        tws_need = max(L._trace_ws_bytes(bp.PH[i]) for i in range(nsys))
        st["tws"] = L._ws(tws_need, dev)
        st["wsA"] = L._ws(L.expand_workspace_size(planX, Hpt, bp.precision, kmax), dev)
        st["wsB"] = L._ws(L.expand_workspace_size(planX, Hpt, bp.precision, kmax), dev)
        st["graphs"] = None
        if use_graphs:
            bp.graphs[key] = st
    else:
        st["Hpt"].copy_(Hpt.vals)
        st["A"].copy_(A)
        st["G"].copy_(G)
    Hst = bp.P_H.with_vals(st["Hpt"])
    tolN = [1e-6 * n for n in N_e] if tol_N is None else tol_N

    # The captured passes hold only launches whose arguments stay fixed for the
    # batch (buffers, term counts); each system's bisection takes its bounds,
    # kT and N_e as kernel arguments, which change with H, so it runs outside.
    def pass1():
        st["g"].zero_()
        st["t"].zero_()
        L.expand_batched(st["planX"], Hst, kmax, st["nt"], None, None, 0, [], moments=st["t"], G=st["G"],
                         gmoments=st["g"], moment_stride=kmax, precision=bp.precision, ws=st["wsA"])

    def check_bounds():
        for i in range(nsys):
            verdict, value = solve.penalty(st["t"][i], nH[i], penalty_alpha, penalty_threshold, penalty_terms)
            if verdict != 0:
                side = {-1: "lower", 1: "upper"}.get(verdict, "a")
                raise L.ChebError(L.ERR_BOUNDS, f"penalty check (Eq. 5): system {i} leaves its {side} bound "
                                                f"(trace {value:g} on [{bH[i][0]}, {bH[i][1]}])")

    def searches():
        for i in range(nsys):
            L.mu_search(st["g"][i], nH[i], bH[i][0], bH[i][1], kind, kT, N_e[i], tolN[i], max_iter,
                        result=st["res"][i], ws=st["mws"][i])

    def pass2():
        st["p"].zero_()
        L.expand_batched(st["planX"], Hst, kmax, st["nt"], st["c"], st["coff"], 0, [st["p"]],
                         precision=bp.precision, ws=st["wsB"])
        L.masked_product(bp.plan64, bp.P_out.with_vals(st["p"]), st["A"], st["Y"])
        L.masked_product(bp.plan64, bp.P_out.with_vals(st["A"]), st["Y"], st["F"])
        for i in range(nsys):
            L.trace(_slice_bsr(bp.Pout[i], st["F"], bp.ooff[i]), _slice_bsr(bp.PH[i], bp.S.vals, bp.hoff[i]),
                    out=st["tr"][i:i + 1], ws=st["tws"])

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    captured = False
    if use_graphs and st["graphs"] is None:
        # first solve of this batch: run eagerly, then capture both passes
        ev[0].record()
        pass1()
        ev[1].record()
        check_bounds()
        searches()
        res = L.decode_mu_batch(st["res"])
        mus = [r["mu"] for r in res]
        _fill_pass2_coeffs(st, kind, kT, mus, bH, nH, dev)
        ev[2].record()
        pass2()
        ev[3].record()
        torch.cuda.synchronize(dev)
        gA, gB = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gA):
            pass1()
        with torch.cuda.graph(gB):
            pass2()
        st["graphs"] = (gA, gB)
        captured = True
    elif use_graphs:
        gA, gB = st["graphs"]
        ev[0].record()
        gA.replay()
        ev[1].record()
        check_bounds()
        searches()
        res = L.decode_mu_batch(st["res"])
        mus = [r["mu"] for r in res]
        _fill_pass2_coeffs(st, kind, kT, mus, bH, nH, dev)
        ev[2].record()
        gB.replay()
        ev[3].record()
    else:
        ev[0].record()
        pass1()
        ev[1].record()
        check_bounds()
        searches()
        res = L.decode_mu_batch(st["res"])
        mus = [r["mu"] for r in res]
        _fill_pass2_coeffs(st, kind, kT, mus, bH, nH, dev)
        ev[2].record()
        pass2()
        ev[3].record()
    torch.cuda.synchronize(dev)
    tm["pass1_ms"] = ev[0].elapsed_time(ev[1])
    tm["pass2_ms"] = ev[2].elapsed_time(ev[3])
    tm["total_s"] = time.perf_counter() - t0
    return {"F": st["F"], "p": st["p"], "A": st["A"], "G": st["G"], "gmoments": st["g"], "mu": mus,
            "mu_result": res, "n_terms": nH, "n_S": nS, "bounds_H": bH, "bounds_S": bS,
            "trace_FS": st["tr"].cpu().numpy(), "captured": captured, "graphs": use_graphs,
            "tiles": dict(bp.tiles)}


def _fill_pass2_coeffs(st, kind, kT, mus, bH, nH, dev):
    off = np.concatenate([[0], np.cumsum(nH)]).astype(np.int64)
    for i, (mu, (e0, e1), n) in enumerate(zip(mus, bH, nH)):
        L.coeffs([{"kind": kind, "mu": mu, "kT": kT}], e0, e1, 0.0, int(n), device=dev,
                 out=st["c"][off[i]:off[i + 1]])


def moment_pass_batched(bp: BatchedProblem, kT, N_e: list[float], n_moments: int = 32, tol: float = 1e-7,
                        tol_S: float = 1e-10, kind: int = L.FERMI, max_iter: int = 100,
                        tol_N: list[float] | None = None) -> dict:
    """Pass 1 only, for every system: the first n_moments traces t_k = Tr T_k of
    H~'_i, the trace functional moments g_k and each system's bisection result
    (used to label training instances of the learned mu proposal)."""
    dev = bp.device
    nsys = bp.nsys
    kTs = list(kT) if isinstance(kT, (list, tuple, np.ndarray)) else [kT] * nsys
    pr = prepare_batched(bp, kTs, tol, tol_S, kind)
    nH, bH = pr["n_terms"], pr["bounds_H"]
    kmax = max(nH)
    planX = bp.batched_plan(bp.precision, pr["Hpt"])
    g = torch.zeros((nsys, kmax), dtype=torch.float64, device=dev)
    t = torch.zeros((nsys, kmax), dtype=torch.float64, device=dev)
    L.expand_batched(planX, pr["Hpt"], kmax, torch.as_tensor(nH, dtype=torch.int32, device=dev), None, None, 0,
                     [], moments=t, G=pr["G"], gmoments=g, moment_stride=kmax, precision=bp.precision)
    res = torch.zeros((nsys, 48), dtype=torch.uint8, device=dev)
    tolN = [1e-6 * n for n in N_e] if tol_N is None else tol_N
    for i in range(nsys):
        L.mu_search(g[i], nH[i], bH[i][0], bH[i][1], kind, kTs[i], N_e[i], tolN[i], max_iter, result=res[i])
    out = dict(pr)
    out.update({"t": t[:, :n_moments].contiguous(), "g": g, "mu_result": L.decode_mu_batch(res)})
    out["mu"] = [r["mu"] for r in out["mu_result"]]
    return out
