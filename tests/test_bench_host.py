"""Host-side logic of bench.py and the shipped proposal weights (no GPU)."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import mlp as omlp  # noqa: E402


def test_workloads_carry_what_their_arm_reads():
    for name, cfg in bench.WORKLOADS.items():
        assert cfg["precision"] in ("f32", "f64", "f64x"), name
        if cfg.get("batched"):
            assert {"n_sys", "atoms_lo", "atoms_hi", "r_c", "r_buf", "kT", "tol", "tol_S"} <= set(cfg), name
        elif cfg.get("powers"):
            assert {"n_atoms", "r_c", "r_buf", "tol", "exponents", "n_mu"} <= set(cfg), name
        else:
            assert {"n_atoms", "r_c", "r_buf", "kT", "N_e", "tol", "tol_S", "n_mu"} <= set(cfg), name
            if cfg.get("form") == "learned":
                assert cfg["n_mu"] <= 8 and 0 < cfg["max_half_kT"] <= 1.0
            if cfg.get("form") == "autokT":
                assert cfg["dE_tol"] > 0 and cfg["widen"] > 1 and 0 < cfg["shrink"] < 1, name
    assert bench.DEFAULT_WORKLOAD in bench.WORKLOADS


def test_batched_sizes_are_seeded_and_in_range():
    cfg = bench.WORKLOADS["foe_batched_64"]
    a, b = bench.batched_sizes(cfg), bench.batched_sizes(cfg)
    assert a == b and len(a) == cfg["n_sys"]
    assert min(a) >= cfg["atoms_lo"] and max(a) <= cfg["atoms_hi"]


def test_step_bytes_counts_each_stream_once():
    # T_k, T_{k-1} read and T_{k+1} written (FP32), the operator (FP32), each
    # accumulator read and written (8 bytes per element), G read (8 bytes)
    assert bench.col_step_bytes(10, 4, 0, False) == 10 * 16 * 4 * 3 + 4 * 16 * 4
    assert bench.col_step_bytes(10, 4, 2, True) == 10 * 16 * 4 * 3 + 4 * 16 * 4 + 10 * 16 * 8 * 2 * 2 + 10 * 16 * 8


def test_solve_step_equivalents():
    # a half-length moment pass, a full accumulation pass, four P_out products
    assert bench.solve_step_equivalents(100, 50, 30, 10) == 48 + 98 + 12
    assert bench.solve_step_equivalents(100, 100, 10, 10) == 98 + 98 + 4


def test_default_workload_is_the_mixed_40k_solve_with_four_mu():
    cfg = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert cfg["n_atoms"] == 10000 and cfg["precision"] == "f32" and cfg["kT"] == 0.005
    assert cfg["n_mu"] == 4 and cfg["form"] == "mu4"


def test_oracle_threads_follow_omp_setting(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.oracle_threads() == 3
    monkeypatch.delenv("OMP_NUM_THREADS")
    assert bench.oracle_threads() == (os.cpu_count() or 1)


def test_shipped_proposal_weights_match_the_network():
    path = os.path.join(ROOT, "paper_1704_00512_gb300", "weights", "mu_proposal.npz")
    with np.load(path) as d:
        theta = d["theta"]
        X, xstar, scale = d["features"], d["xstar"], d["scale"]
    assert theta.shape == (omlp.N_PARAMS,) and np.all(np.isfinite(theta))
    # the FP64 restatement of the network on the stored training inputs gives
    # finite outputs of the expected shape
    out, _ = omlp.forward(theta.astype(np.float64), X[:8].astype(np.float64))
    assert out.shape == (8, 2) and np.all(np.isfinite(out))
    assert X.shape[1] == omlp.N_IN and len(xstar) == len(scale) == len(X)


def test_traffic_scales_with_blocks_and_is_tied_to_the_measured_source():
    order = bench.COL_TRAFFIC["order"]
    t = bench.col_traffic_per_launch("mu4", 4, [100, 200], bench.COL_TRAFFIC["blocks_P_out"] * 2, measured=True,
                                     order=order)
    want = 2 * (bench.COL_TRAFFIC["pass1_bytes"] * 100 + bench.COL_TRAFFIC["pass2_4acc_bytes"] * 200) / 300
    assert t == int(want)
    # measured in one atom order: another order's solve reports no figure
    other = None if order == "hilbert" else "hilbert"
    assert bench.col_traffic_per_launch("mu4", 4, [100, 200], 10, measured=True, order=other) is None
    assert bench.col_traffic_per_launch("twopass", 1, [100, 100], 10, measured=True) is None
    assert bench.col_traffic_per_launch("mu4", 4, [100, 200], 10, measured=False) is None
    # any change to the kernel text before the host section drops the figure
    assert not bench.col_kernel_measured("__global__ void k() {}\n" + bench.COL_KERNEL_END)
