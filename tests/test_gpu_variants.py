"""GPU: every per-step tile variant computes the same head, and the step
tuner keeps a variant set that is at least as fast and still exact.

The workload is the full 30-qubit, 14-cycle one (all 64 slices), compared
amplitude by amplitude with the O1 state vector stored by
tests/golden/make_sliced30_golden.py; tolerances as in the parity tests
(relative L2 <= 1e-5, 1e-4 for the BF16x3 form)."""
import os

import numpy as np
import pytest

import circuit_inputs as ci
import oracle as O

pytestmark = pytest.mark.gpu

_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sliced30_o1.npz")
ENGINES = [1, 3, 4]
IDS = ["tc3xtf32", "bf16x3", "fp16x3"]


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def _tol(gemm):
    return 1e-4 if gemm == 3 else 1e-5


def _read_head(tn, head, cfg):
    tails, oq = cfg["tails"], cfg["open_qubits"]
    h = len(oq)
    bits = np.array([O.bitstring_index(int(t), oq, mu) for t in tails for mu in range(1 << h)], dtype=np.uint64)
    return tn.tn_amplitudes(head, bits).reshape(len(tails), 1 << h)


def _assert_close(H, ref, tol):
    err = float(np.linalg.norm(H - ref) / np.linalg.norm(ref))
    assert err <= tol, err
    assert np.abs(H - ref).max() <= 2 * tol * np.abs(ref).max()


@pytest.mark.parametrize("gemm", ENGINES, ids=IDS)
def test_every_step_variant_matches_stored_o1(tn, gemm):
    """Variant v of every step at once (v past a step's count: its last), for
    every v: all 65,536 amplitudes of the 64-slice sum, plain launches and a
    captured graph (recaptured after the variants change)."""
    g = np.load(_GOLDEN)
    cfg = ci.config_sliced30()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                      order_trials=2048)
    ns = tn.tn_plan_get_stats(plan)["n_launches"] - 1
    counts = [tn.tn_plan_step_variants(plan, i)[0] for i in range(ns)]
    assert max(counts) >= 4
    for v in range(max(counts)):
        for i in range(ns):
            tn.tn_plan_set_step_variant(plan, i, min(v, counts[i] - 1))
        head = tn.tn_head_create(plan)
        tn.tn_contract_slices(plan, 0, 64, head)
        _assert_close(_read_head(tn, head, cfg), g["H_full"], _tol(gemm))
        hg = tn.tn_head_create(plan)
        tn.tn_contract_slices_graph(plan, 0, 64, hg)
        _assert_close(_read_head(tn, hg, cfg), g["H_full"], _tol(gemm))


@pytest.mark.parametrize("gemm", ENGINES, ids=IDS)
def test_step_tuner_keeps_the_faster_set_and_stays_exact(tn, gemm):
    g = np.load(_GOLDEN)
    cfg = ci.config_sliced30()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                      order_trials=2048)
    t0, t1 = tn.tn_plan_tune_steps(plan, reps=2)
    assert t0 > 0 and t1 > 0
    st = tn.tn_plan_get_stats(plan)
    assert (st["tune_default_ms"], st["tune_tuned_ms"]) == (t0, t1)
    d = tn.tn_plan_describe(plan)
    assert st["n_tuned_steps"] == sum(s["variant"] != 0 for s in d["steps"])
    if t1 >= t0:
        assert st["n_tuned_steps"] == 0          # the starting (default) set is kept
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices_graph(plan, 0, 64, head)
    _assert_close(_read_head(tn, head, cfg), g["H_full"], _tol(gemm))
    # the autotuner tunes the steps of the plan it keeps (a slice is ~10 ms)
    ap = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], n_candidates=2,
                             order_trials=2048, gemm=gemm)
    sa = tn.tn_plan_get_stats(ap)
    assert sa["tune_default_ms"] > 0 and sa["tune_tuned_ms"] > 0
    assert sa["measured_slice_ms"] == min(sa["tune_default_ms"], sa["tune_tuned_ms"])
    ap2 = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], n_candidates=1,
                              order_trials=2048, gemm=gemm, tune_steps=-1)
    s2 = tn.tn_plan_get_stats(ap2)
    assert s2["n_tuned_steps"] == 0 and s2["tune_default_ms"] == 0
