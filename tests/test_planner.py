"""Host planner (no GPU): the plan replayed on the CPU matches the oracle.

The library is built for sm_103a and loaded; plans are made host_only, so no
device call is made.
"""
import numpy as np
import pytest

import circuit_inputs as ci
import oracle as O
from tests.plan_emulator import emulate


@pytest.fixture(scope="module")
def tn():
    import paper_2111_03011_gb300 as m
    return m


def _edges(cfg):
    return [(g, l, k, v) for (g, l, k, v) in cfg["edges"]]


def _oracle_H(cfg, slice_range=None, pins=()):
    se = [(g, l) for (g, l, k, v) in cfg["edges"] if k == 0]
    psi = O.sliced_statevector(cfg["circuit"], se, pins=pins, slice_range=slice_range)
    return O.sparse_state_from_vector(psi, cfg["open_qubits"], cfg["tails"])


def test_library_exports_every_declared_symbol(tn):
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "tn_gb300.h")).read()
    declared = set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", hdr))
    for name in declared:
        assert hasattr(tn.lib, name), name
    assert declared == set(tn.EXPORTED)


@pytest.mark.parametrize("case", [
    dict(r=3, c=4, m=6, seed=5, n_open=4, L=6, cut=1),
    dict(r=3, c=3, m=8, seed=8, n_open=9, L=1, cut=0),
    dict(r=2, c=4, m=8, seed=6, n_open=0, L=5, cut=1),
    dict(r=4, c=4, m=8, seed=11, n_open=6, L=8, cut=2),
])
@pytest.mark.parametrize("absorb", [0, 2])
def test_plan_replay_matches_oracle(tn, case, absorb):
    cfg = ci.config_small(case["r"], case["c"], case["m"], seed=case["seed"], n_open=case["n_open"],
                          L=case["L"], n_cut_gates=case["cut"])
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                      max_host_absorb_log2=absorb)
    d = tn.tn_plan_describe(plan, with_data=True)
    k = d["n_sliced"]
    H = emulate(d, cfg["tails"], cfg["open_qubits"], range(1 << k))
    ref = _oracle_H(cfg)
    assert np.abs(H - ref).max() < 1e-12
    st = tn.tn_plan_get_stats(plan)
    assert st["n_sliced"] == k and st["n_tails"] == case["L"]
    assert st["tc_macs"] > 0 or st["n_contractions"] == 0


def test_slice_range_and_pins_replay(tn):
    c = ci.make_grid_circuit(3, 4, 8, seed=2)
    cut = ci.mid_circuit_cut_edges(c, 2)            # 4 edges on 2 gates
    open_q = [8, 9, 10, 11]
    tails = ci.draw_tails(12, open_q, 4, seed=3)
    edges = [cut[0], cut[1], (cut[2][0], cut[2][1], tn.TN_EDGE_PIN, 1), (cut[3][0], cut[3][1], tn.TN_EDGE_PIN, 0)]
    plan = tn.tn_plan(c, open_q, tails, edges, host_only=True)
    d = tn.tn_plan_describe(plan, with_data=True)
    assert d["n_sliced"] == 2 and d["n_pinned"] == 2
    H = emulate(d, tails, open_q, [1, 2])
    psi = O.sliced_statevector(c, [(cut[0][0], cut[0][1]), (cut[1][0], cut[1][1])],
                               pins=[(cut[2][0], cut[2][1], 1), (cut[3][0], cut[3][1], 0)], slice_range=(1, 3))
    ref = O.sparse_state_from_vector(psi, open_q, tails)
    assert np.abs(H - ref).max() < 1e-13


def test_hole_is_removed_exactly(tn):
    """Both inputs of an fSim pinned to 0: the host splits the rank-one
    remainder into two vectors (Method case (i)); the result is exact."""
    c = ci.make_grid_circuit(3, 3, 6, seed=12)
    gi = ci.mid_circuit_cut_edges(c, 1)[0][0]
    edges = [(gi, 0, tn.TN_EDGE_PIN, 0), (gi, 1, tn.TN_EDGE_PIN, 0)]
    open_q = list(range(9))
    tails = np.zeros(1, np.uint64)
    plan = tn.tn_plan(c, open_q, tails, edges, host_only=True)
    d = tn.tn_plan_describe(plan, with_data=True)
    H = emulate(d, tails, open_q, [0])
    psi = O.statevector(c, [(gi, 0, 0), (gi, 1, 0)])
    assert np.abs(H[0] - psi).max() < 1e-13


def test_user_order_roundtrip_and_random_order(tn):
    cfg = ci.config_small(3, 4, 6, seed=5, n_open=4, L=6, n_cut_gates=1)
    p1 = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True)
    order = tn.tn_plan_order(p1)
    p2 = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), order=order, host_only=True)
    assert (tn.tn_plan_order(p2) == order).all()
    d1 = tn.tn_plan_describe(p1)
    n_leaves = len(d1["leaves"])
    # a different valid order: contract leaf 0 with every other leaf in turn
    o = np.array([[0, j] for j in range(1, n_leaves)], dtype=np.int32)
    p3 = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), order=o, host_only=True,
                    max_log2_elements=30)
    d3 = tn.tn_plan_describe(p3, with_data=True)
    H = emulate(d3, cfg["tails"], cfg["open_qubits"], range(4))
    assert np.abs(H - _oracle_H(cfg)).max() < 1e-12
    with pytest.raises(tn.TNError):
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), order=[[0, 0]], host_only=True)


def test_sparse_state_worked_example_patterns(tn):
    """Supplement worked example: targets {111, 010, 000}; merging the final
    legs of qubits 2 and 3 (0-based 1 and 2) keeps the 3 patterns {11, 10, 00}."""
    import json, os
    ex = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))["sparse_state_example"]
    c = ci.make_random_2q_circuit(3, 2, seed=1)
    tails = np.array([int(t[::-1], 2) for t in ex["targets"]], dtype=np.uint64)
    plan0 = tn.tn_plan(c, [], tails, host_only=True, max_host_absorb_log2=1, host_fold_log2=-1)
    d0 = tn.tn_plan_describe(plan0)
    ids = {lf["tq"]: i for i, lf in enumerate(d0["leaves"]) if lf["tq"] in (2, 4)}
    assert set(ids) == {2, 4}
    plan = tn.tn_plan(c, [], tails, order=[[ids[2], ids[4]]], host_only=True, max_host_absorb_log2=1,
                      host_fold_log2=-1)
    d = tn.tn_plan_describe(plan, with_data=True)
    merged = [v for v in d["vts"] if v["tq"] == 6]
    assert merged and merged[0]["P"] == 3
    pats = sorted(set(int(t) & 6 for t in tails))
    assert [format(p >> 1, "02b")[::-1] for p in pats] == sorted(ex["unique_patterns"], key=lambda s: int(s[::-1], 2))
    H = emulate(d, tails, [], [0])
    psi = O.statevector(c)
    assert np.abs(H[:, 0] - psi[tails.astype(np.int64)]).max() < 1e-13


def test_invalid_inputs_rejected(tn):
    c = ci.make_grid_circuit(2, 2, 2, seed=1)
    t = np.zeros(1, np.uint64)
    for kw in [dict(open_qubits=[5]), dict(open_qubits=[0, 0])]:
        with pytest.raises(tn.TNError) as e:
            tn.tn_plan(c, kw["open_qubits"], t, host_only=True)
        assert e.value.code == tn.TN_ERR_INVALID
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(c, [0], t, [(0, 0, 0, 0), (0, 0, 0, 0)], host_only=True)
    assert e.value.code == tn.TN_ERR_INVALID
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(c, [0], t, [(0, 0, tn.TN_EDGE_COMPANION, 0)], host_only=True)   # gate 0 is single-qubit
    assert e.value.code == tn.TN_ERR_INVALID
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(c, [0], np.zeros(0, np.uint64), host_only=True)
    assert e.value.code == tn.TN_ERR_INVALID


def test_injected_allocation_failure(tn, monkeypatch):
    """Host-side fault injection: with TN_FAULT_INJECT=alloc the plan's device
    upload fails with TN_ERR_OOM before any CUDA call (so this runs without a
    GPU); host-only planning is unaffected, and disarming restores it."""
    cfg = ci.config_small(3, 4, 6, seed=5, n_open=4, L=6, n_cut_gates=1)
    monkeypatch.setenv("TN_FAULT_INJECT", "alloc")
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"])
    assert e.value.code == tn.TN_ERR_OOM and "injected" in str(e.value)
    p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True)
    assert tn.tn_plan_get_stats(p)["n_sliced"] == 2
    monkeypatch.delenv("TN_FAULT_INJECT")
    try:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"])   # succeeds on a GPU
    except tn.TNError as e:
        assert e.code == tn.TN_ERR_CUDA          # without a device the real upload fails in CUDA


def test_size_cap_enforced(tn):
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=16, L=1, n_cut_gates=0)
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], host_only=True, max_log2_elements=10)
    assert e.value.code == tn.TN_ERR_OOM


def test_companion_cuts_replay_and_fidelity_estimate(tn):
    """Companion cuts (Method case (ii)): the replayed plan equals the oracle
    with the partner outputs fixed, and F_est carries (1 + sin^2 theta)/2 per
    companion (the fidelity-estimate equation)."""
    import math
    import oracle as O
    c = ci.make_grid_circuit(3, 4, 8, seed=15)
    cut = ci.mid_circuit_cut_edges(c, 2)
    g0, g1 = cut[0][0], cut[2][0]
    edges = [(g0, 0, tn.TN_EDGE_COMPANION, 0), (g1, 1, tn.TN_EDGE_COMPANION, 0), (cut[3][0], 0, tn.TN_EDGE_SLICE, 0)]
    oq = [8, 9, 10, 11]
    tails = ci.draw_tails(12, oq, 6, seed=3)
    plan = tn.tn_plan(c, oq, tails, edges, host_only=True)
    d = tn.tn_plan_describe(plan, with_data=True)
    assert d["n_sliced"] == 3
    H = emulate(d, tails, oq, range(8))
    se = [(g0, 0, True), (g1, 1, True), (cut[3][0], 0)]
    ref = O.sparse_state_from_vector(O.sliced_statevector(c, se), oq, tails)
    assert np.abs(H - ref).max() < 1e-13
    # the plan's companion factor, visible through F_est once a head exists, is
    # checked on the GPU; here the formula itself
    f = O.companion_factor(c.gates[g0].theta) * O.companion_factor(c.gates[g1].theta)
    assert 0.9 < f <= 1.0


def _auto_cfg():
    return ci.config_small(4, 5, 10, seed=13, n_open=8, L=24, n_cut_gates=1)


def test_automatic_slicing_is_exact_per_user_slice(tn):
    """With a cap no order meets, the planner slices extra wires (Supplement,
    slicing and contraction order: the sliced edges are those that cut the
    largest intermediates) and sums them inside every user slice, so user
    slice s replays to the oracle's slice s."""
    cfg = _auto_cfg()
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                   max_log2_elements=13)
    assert e.value.code == tn.TN_ERR_OOM
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                      max_log2_elements=13, auto_slice=16)
    st = tn.tn_plan_get_stats(plan)
    d = tn.tn_plan_describe(plan, with_data=True)
    k, ni = st["n_sliced"], st["n_internal_sliced"]
    assert k == 2 and ni >= 1 and d["n_internal"] == ni and len(d["internal_edges"]) == ni
    assert st["max_log2_elements"] <= 13 + 1e-9
    # the extra edges are wires of the circuit: (gate, input leg)
    for g, leg in d["internal_edges"]:
        assert 0 <= g < len(cfg["circuit"].gates) and leg in (0, 1)
        assert leg < cfg["circuit"].gates[g].arity
    for s in (1, 2):
        H = emulate(d, cfg["tails"], cfg["open_qubits"], [s | (t << k) for t in range(1 << ni)])
        ref = _oracle_H(cfg, slice_range=(s, s + 1))
        assert np.abs(H - ref).max() < 1e-12
    # the internal slices alone are the oracle with those wires cut as well
    se = [(g, l) for (g, l, kk, v) in cfg["edges"]] + [tuple(x) for x in d["internal_edges"]]
    sub = 5 << k
    H = emulate(d, cfg["tails"], cfg["open_qubits"], [sub])
    ref = O.sparse_state_from_vector(O.sliced_statevector(cfg["circuit"], se, slice_range=(sub, sub + 1)),
                                     cfg["open_qubits"], cfg["tails"])
    assert np.abs(H - ref).max() < 1e-12


def test_automatic_slicing_counts_and_limits(tn):
    cfg = _auto_cfg()
    base = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                      max_log2_elements=13, auto_slice=16)
    st = tn.tn_plan_get_stats(base)
    ni = st["n_internal_sliced"]
    # per-user-slice figures count every internal pass
    assert st["n_launches"] % (1 << ni) == 0
    # a budget below what the cap needs is an error, not a silent over-cap plan
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                   max_log2_elements=13, auto_slice=1 if ni > 1 else 0)
    assert e.value.code == tn.TN_ERR_OOM
    # open legs cannot be sliced: 16 open qubits never fit 2^10
    big = ci.config_small(4, 4, 8, seed=11, n_open=16, L=1, n_cut_gates=0)
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(big["circuit"], big["open_qubits"], big["tails"], host_only=True, max_log2_elements=10,
                   auto_slice=20)
    assert e.value.code == tn.TN_ERR_OOM
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True, auto_slice=25)
    assert e.value.code == tn.TN_ERR_INVALID
    # without need, automatic slicing adds nothing
    p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True, auto_slice=8)
    assert tn.tn_plan_get_stats(p)["n_internal_sliced"] == 0


def test_fp16_engine_scale_slots(tn):
    """The FP16x3 engine scales each GEMM operand by a power of two from its
    maximum.  Every fp16 GEMM step reads two distinct slots: a leaf operand's
    maximum is a static slot computed on the host; an intermediate's slot is
    written, earlier in the pass, either by the epilogue of the step that
    produced it (tensor-core GEMM or small-operand step) or by an operand-max
    step -- exactly one writer each.  The other engines use no slots, and
    unitarity is not required (a gate scaled by 2^-40 plans the same way)."""
    import copy
    cfg = _auto_cfg()
    for small in (-1, 0):
        plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                          gemm=tn.TN_GEMM_TC_FP16X3, small_max_bits=small)
        steps = tn.tn_plan_describe(plan)["steps"]
        gemms = [i for i, s_ in enumerate(steps) if s_["kind"] == 3 and s_["h16"] == 2]
        assert gemms
        seen = set()
        for gi in gemms:
            g = steps[gi]
            for sl, consumer_kind in ((g["slot"], 1), (g["slotB"], 2)):
                assert sl != -1 and sl not in seen
                seen.add(sl)
                users = [i for i, s_ in enumerate(steps[:gi]) if s_["kind"] == consumer_kind and s_["slot"] == sl]
                assert len(users) == 1
                if sl <= -2:
                    continue
                writers = [i for i, s_ in enumerate(steps) if (s_["kind"] == 6 and s_["slot"] == sl) or
                           (s_["kind"] in (0, 3) and s_["max_slot"] == sl)]
                assert len(writers) == 1 and writers[0] < users[0]
        assert any(s_["max_slot"] >= 0 for s_ in steps)
    for eng in (tn.TN_GEMM_TC_3XTF32, tn.TN_GEMM_TC_BF16X3, tn.TN_GEMM_SIMT_FP32):
        p2 = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True, gemm=eng)
        assert all(s_["kind"] != 6 and s_["max_slot"] == -1 and s_["slot"] == -1
                   for s_ in tn.tn_plan_describe(p2)["steps"])
    bad = copy.deepcopy(cfg["circuit"])
    bad.gates[3].U = bad.gates[3].U * 2.0 ** -40
    tn.tn_plan(bad, cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True, gemm=tn.TN_GEMM_TC_FP16X3)


def test_sycamore53_topology_replay_matches_oracle(tn):
    """53-qubit Sycamore-topology circuit at 6 cycles (reduced depth): the
    replayed plan equals the O2 network oracle on two groups."""
    circ = ci.make_sycamore_circuit(6, seed=5)
    n = circ.n_qubits
    assert n == 53
    oq = list(range(n - 6, n))
    tails = ci.draw_tails(n, oq, 8, seed=55)
    plan = tn.tn_plan(circ, oq, tails, host_only=True, max_log2_elements=24, auto_slice=8)
    d = tn.tn_plan_describe(plan, with_data=True)
    H = emulate(d, tails, oq, [t << d["n_sliced"] for t in range(1 << d["n_internal"])])
    ref = O.network_amplitudes(circ, oq, tails, [], groups=[0, 5])
    assert np.abs(H[[0, 5]] - ref).max() <= 1e-10 * np.abs(ref).max()


def test_automatic_slicing_of_a_given_order(tn):
    """A caller's order over the cap is sliced to fit (same leaves, same order)
    and still replays to the oracle slice by slice; without auto_slice the
    same order is refused with TN_ERR_OOM."""
    cfg = _auto_cfg()
    free = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), host_only=True,
                      max_log2_elements=30)
    order = tn.tn_plan_order(free)
    big = tn.tn_plan_get_stats(free)["max_log2_elements"]
    cap = big - 2
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), order=order, host_only=True,
                   max_log2_elements=cap)
    assert e.value.code == tn.TN_ERR_OOM
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], _edges(cfg), order=order, host_only=True,
                      max_log2_elements=cap, auto_slice=8)
    st = tn.tn_plan_get_stats(plan)
    assert st["n_internal_sliced"] >= 1 and st["max_log2_elements"] <= cap + 1e-9
    assert np.array_equal(tn.tn_plan_order(plan), order)
    d = tn.tn_plan_describe(plan, with_data=True)
    k, ni = st["n_sliced"], st["n_internal_sliced"]
    H = emulate(d, cfg["tails"], cfg["open_qubits"], [3 | (t << k) for t in range(1 << ni)])
    assert np.abs(H - _oracle_H(cfg, slice_range=(3, 4))).max() < 1e-12


@pytest.mark.parametrize("case", range(16))
def test_random_plans_replay_to_the_oracle(tn, case):
    """Seeded random cases over everything the host planner combines: generic
    two-qubit gates in both orientations, random open sets and tail counts,
    SLICE / PIN / COMPANION edges on random gates, host absorption caps, the
    small-operand threshold, engines (leaf variants and, for FP16x3, scale
    slots), host folding thresholds, automatic slicing under a tight cap --
    each replayed on the host and compared with the state-vector oracle over a
    random slice range."""
    rng = np.random.default_rng(1000 + case)
    n = int(rng.integers(4, 9))
    circ = ci.make_random_2q_circuit(n, int(rng.integers(2, 5)), seed=2000 + case)
    n_open = int(rng.integers(0, min(n, 5) + 1))
    oq = sorted(int(q) for q in rng.choice(n, n_open, replace=False))
    L = int(rng.integers(1, min(8, 1 << (n - n_open)) + 1))
    tails = ci.draw_tails(n, oq, L, seed=3000 + case)
    twoq = [i for i, g in enumerate(circ.gates) if g.arity == 2]
    picks = rng.choice(len(twoq), min(len(twoq), int(rng.integers(0, 4))), replace=False)
    edges, used = [], set()
    for p in picks:
        g = twoq[int(p)]
        leg = int(rng.integers(0, 2))
        kind = int(rng.choice([tn.TN_EDGE_SLICE, tn.TN_EDGE_PIN, tn.TN_EDGE_COMPANION]))
        if (g, leg) in used:
            continue
        used.add((g, leg))
        edges.append((g, leg, kind, int(rng.integers(0, 2)) if kind == tn.TN_EDGE_PIN else 0))
    gemm = int(rng.choice([tn.TN_GEMM_TC_3XTF32, tn.TN_GEMM_TC_FP16X3, tn.TN_GEMM_TC_BF16X3, tn.TN_GEMM_SIMT_FP32]))
    kw = dict(host_only=True, gemm=gemm, max_host_absorb_log2=int(rng.choice([0, 2, 12])),
              small_max_bits=int(rng.choice([-1, 2, 4])), host_fold_log2=int(rng.choice([-1, 3, 5, 12])))
    free = tn.tn_plan(circ, oq, tails, edges, **dict(kw, host_fold_log2=-1))   # caps are on the unfolded network
    big = tn.tn_plan_get_stats(free)["max_log2_elements"]
    leaves = tn.tn_plan_describe(free)["leaves"]
    floor = max([np.log2(len(set(int(t) for t in tails))) + n_open] +
                [np.log2(lf["P"]) + len(lf["dev_legs"]) for lf in leaves])
    cap = max(float(np.ceil(floor)), big - float(rng.integers(0, 3)))
    plan = tn.tn_plan(circ, oq, tails, edges, max_log2_elements=cap, auto_slice=12, **kw)
    st = tn.tn_plan_get_stats(plan)
    d = tn.tn_plan_describe(plan, with_data=True)
    k, ni = st["n_sliced"], st["n_internal_sliced"]
    b = int(rng.integers(0, 1 << k))
    e = int(rng.integers(b + 1, (1 << k) + 1))
    H = emulate(d, tails, oq, [s | (t << k) for s in range(b, e) for t in range(1 << ni)])
    se = [(g, l, True) if kd == tn.TN_EDGE_COMPANION else (g, l) for (g, l, kd, v) in edges
          if kd != tn.TN_EDGE_PIN]
    pins = [(g, l, v) for (g, l, kd, v) in edges if kd == tn.TN_EDGE_PIN]
    ref = O.sparse_state_from_vector(O.sliced_statevector(circ, se, pins=pins, slice_range=(b, e)), oq, tails)
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.abs(H - ref).max() <= 1e-11 * scale


@pytest.mark.parametrize("fold", [0, 4, 8, 16])
def test_host_folding_equals_the_device_contraction(tn, fold):
    """Host folding: contractions of host tensors with small results are done
    at plan time and become leaves (with a variant per value of their slice
    bits, the two ends of a cut merged into one variant axis).  The folded
    plan replays to the same amplitudes as the unfolded one and the oracle,
    over every slice, with slice, pin and companion cuts; it launches fewer
    kernels; at 2^16 the whole 16-qubit network folds into one leaf."""
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    c = cfg["circuit"]
    twoq = c.two_qubit_gates()
    edges = list(cfg["edges"][:3]) + [(twoq[4], 1, tn.TN_EDGE_COMPANION, 0), (twoq[9], 0, tn.TN_EDGE_PIN, 1)]
    cfg = dict(cfg, edges=edges)
    base = tn.tn_plan(c, cfg["open_qubits"], cfg["tails"], edges, host_only=True, host_fold_log2=-1)
    plan = tn.tn_plan(c, cfg["open_qubits"], cfg["tails"], edges, host_only=True, host_fold_log2=fold)
    sb, sp = tn.tn_plan_get_stats(base), tn.tn_plan_get_stats(plan)
    assert sp["n_sliced"] == sb["n_sliced"] == 4 and sp["n_pinned"] == 1
    assert sp["n_launches"] <= sb["n_launches"]
    if fold == 16:
        assert sp["n_leaves"] == 1 and sp["n_contractions"] == 0 and sp["n_launches"] == 1
    if fold >= 8:
        assert sp["n_launches"] < sb["n_launches"]
    H = emulate(tn.tn_plan_describe(plan, with_data=True), cfg["tails"], cfg["open_qubits"], range(16))
    Hb = emulate(tn.tn_plan_describe(base, with_data=True), cfg["tails"], cfg["open_qubits"], range(16))
    se = [(g, l, True) if kd == tn.TN_EDGE_COMPANION else (g, l) for (g, l, kd, v) in edges if kd != tn.TN_EDGE_PIN]
    pins = [(g, l, v) for (g, l, kd, v) in edges if kd == tn.TN_EDGE_PIN]
    ref = O.sparse_state_from_vector(O.sliced_statevector(c, se, pins=pins), cfg["open_qubits"], cfg["tails"])
    assert np.abs(H - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(H - Hb).max() < 1e-12 * np.abs(ref).max()
    # the user-visible order is still over the simplified leaves: planning
    # again with it gives the same folded plan
    again = tn.tn_plan(c, cfg["open_qubits"], cfg["tails"], edges, order=tn.tn_plan_order(plan), host_only=True,
                       host_fold_log2=fold)
    assert tn.tn_plan_get_stats(again)["n_launches"] == sp["n_launches"]


def test_companion_fixing_an_open_qubit_final_wire(tn):
    """A companion cut on a qubit pair's last gate fixes the partner's output --
    here an open qubit's final wire: the amplitudes whose open bit differs from
    the slice's value vanish in that slice (oracle: the post-gate projector)."""
    c = ci.make_random_2q_circuit(5, 3, seed=77)
    last = max(i for i, g in enumerate(c.gates) if g.arity == 2)
    g = c.gates[last]
    oq = sorted({g.q0, g.q1})                       # both outputs of the last gate are open
    tails = ci.draw_tails(5, oq, 3, seed=5)
    edges = [(last, 0, tn.TN_EDGE_COMPANION, 0)]
    plan = tn.tn_plan(c, oq, tails, edges, host_only=True)
    d = tn.tn_plan_describe(plan, with_data=True)
    for s in (0, 1):
        H = emulate(d, tails, oq, [s])
        ref = O.sparse_state_from_vector(O.sliced_statevector(c, [(last, 0, True)], slice_range=(s, s + 1)),
                                         oq, tails)
        assert np.abs(H - ref).max() < 1e-12
        j = oq.index(g.q1)                          # the partner of leg 0 is q1
        assert all(abs(H[gi, mu]) < 1e-15 for gi in range(len(tails)) for mu in range(1 << len(oq))
                   if ((mu >> j) & 1) != s)


def test_cut_on_a_wire_fixed_by_a_companion_is_rejected(tn):
    """A companion cut fixes the partner qubit's output wire; a second cut on
    that same wire (the next gate's input) is a conflicting request and is
    refused with TN_ERR_INVALID rather than silently decoupling the wire."""
    c = ci.make_random_2q_circuit(4, 3, seed=9)
    twoq = [i for i, g in enumerate(c.gates) if g.arity == 2]
    g0 = twoq[0]
    partner = c.gates[g0].q1
    nxt = next(i for i in range(g0 + 1, len(c.gates)) if partner in (c.gates[i].q0, c.gates[i].q1))
    leg = 0 if c.gates[nxt].q0 == partner else 1
    oq = [0, 1]
    tails = ci.draw_tails(4, oq, 2, seed=1)
    for kind in (tn.TN_EDGE_SLICE, tn.TN_EDGE_PIN):
        with pytest.raises(tn.TNError) as e:
            tn.tn_plan(c, oq, tails, [(g0, 0, tn.TN_EDGE_COMPANION, 0), (nxt, leg, kind, 0)], host_only=True)
        assert e.value.code == tn.TN_ERR_INVALID
    tn.tn_plan(c, oq, tails, [(g0, 0, tn.TN_EDGE_COMPANION, 0)], host_only=True)
