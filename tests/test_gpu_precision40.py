"""The 40-qubit precision workload: 5x8 grid, 12 open qubits and one tail
(2^12 head amplitudes), 10 sliced edges on the inputs of 5 fSim gates of the
middle cycle (2^10 slices), of which the kept prefix [0, 128) is summed
(kept fraction 1/8; Results, summing a fraction of the sub-tasks).

- 10 cycles, every engine: the 2^10-amplitude subset (q28 = 1, q29 = 0)
  against the FP64 O2 amplitudes stored by
  tests/golden/make_precision40_golden.py, in the launch configuration the
  bench uses (the kept slices replayed as one captured graph).  Tolerance:
  relative L2 <= 1e-5 (3xTF32, FP16x3, CUDA-core FP32) or 1e-4 (BF16x3), and
  every element within twice that of the largest.
- 16 cycles (the full workload: 2.4e14 complex MACs per slice, intermediates
  up to 2^32 elements): one slice of O2 would take days of NumPy, so there
  the split forms are compared with 3xTF32 on one slice, within the sum of
  the two bounds, and the fidelity estimate of the kept prefix is checked.
"""
import gc
import math
import os

import numpy as np
import pytest

import circuit_inputs as ci

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "precision40_m10_o2.npz")
TOL = {1: 1e-5, 2: 1e-5, 3: 1e-4, 4: 1e-5}


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("gemm", [1, 2, 3, 4], ids=["tc3xtf32", "simt", "bf16x3", "fp16x3"])
def test_precision40_reduced_depth_subset_vs_oracle(tn, gemm):
    g = np.load(GOLDEN)
    cfg = ci.config_precision40(int(g["cycles"]))
    assert [tuple(e) for e in g["edges"]] == [(a, b) for (a, b, _, _) in cfg["edges"]]
    bits = ci.subset_bitstrings(cfg)
    assert np.array_equal(bits, g["bitstrings"])
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm, order_trials=256,
                      order_seed=1, max_log2_elements=32, auto_slice=24)
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices_graph(plan, 0, cfg["kept"], head)
    f_est, done = tn.tn_head_fidelity(head)
    assert done == cfg["kept"] and math.isclose(f_est, 1 / 8)
    got = tn.tn_amplitudes(head, bits)
    ref = g["H_subset"]
    tol = TOL[gemm]
    assert _rel(got, ref) <= tol, _rel(got, ref)
    assert np.abs(got - ref).max() <= 2 * tol * np.abs(ref).max()
    # the head outside the subset: a sparse state of 2^12 amplitudes with the
    # subset's magnitude (a quarter of the norm, within sampling noise)
    assert 0.15 < np.vdot(got, got).real / tn.tn_head_norm(head) < 0.35


def test_precision40_full_depth_engines_agree(tn):
    cfg = ci.config_precision40(16)
    bits = ci.subset_bitstrings(cfg)
    res = {}
    for gemm in (1, 4, 3):                          # one plan (up to 189 GB of workspace) at a time
        plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                          order_trials=4096, order_seed=1, max_log2_elements=32, auto_slice=24)
        st = tn.tn_plan_get_stats(plan)
        assert st["max_log2_elements"] <= 32 and st["tc_macs"] > 1e14
        head = tn.tn_head_create(plan)
        tn.tn_contract_slices(plan, 0, 1, head)
        f_est, done = tn.tn_head_fidelity(head)
        assert done == 1 and math.isclose(f_est, 1 / 1024)
        res[gemm] = tn.tn_amplitudes(head, bits)
        assert np.isfinite(res[gemm]).all() and np.abs(res[gemm]).max() > 0
        del head, plan
        gc.collect()
    for gemm in (4, 3):
        assert _rel(res[gemm], res[1]) <= TOL[gemm] + TOL[1], (gemm, _rel(res[gemm], res[1]))
