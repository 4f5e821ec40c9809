"""The paper's validation sweeps on the 30-qubit, 14-cycle workload (the
Supplement's validation section uses an n = 30, m = 14 circuit).

For K broken edges -- the kept prefix [0, 64 / 2^K) of the 64 slices, whose
top K slice bits are fixed to 0 -- the GPU head has the fidelity estimate
2^-K.  Against the exact amplitudes stored by tests/golden/make_sliced30_golden.py
(the O1 state vector), it is compared with the head's fidelity on the sparse
state, with the expected linear XEB of one-sample-per-group sampling, with the
linear and logarithmic XEB of samples drawn by the GPU sampler, and with the
entropy of the sampling law against its sample estimate (Supplement,
validation: fidelity, XEB and log-XEB against K; entropy figure).  The XEB as a
function of the group size l (Supplement, XEB against l) is taken from the
same heads by splitting groups into sub-groups.
"""
import math
import os

import numpy as np
import pytest

import circuit_inputs as ci
import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sliced30_o1.npz")


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def _bits(cfg):
    oq, tails = cfg["open_qubits"], cfg["tails"]
    return np.array([O.bitstring_index(int(t), oq, mu) for t in tails for mu in range(1 << len(oq))], np.uint64)


def test_fidelity_xeb_entropy_against_broken_edges(tn):
    g = np.load(GOLDEN)
    cfg = ci.config_sliced30()
    n, L, h = 30, len(cfg["tails"]), len(cfg["open_qubits"])
    oq = cfg["open_qubits"]
    H = g["H_full"]
    P = np.abs(H) ** 2                                  # exact probabilities of the sparse-state bitstrings
    plan = tn.tn_plan(cfg["circuit"], oq, cfg["tails"], cfg["edges"], gemm=tn.TN_GEMM_TC_FP16X3, order_trials=2048,
                      order_seed=1)
    bits = _bits(cfg)
    exact = tn.tn_head_create(plan)                     # all 64 slices: the exact amplitudes on the GPU
    tn.tn_contract_slices_graph(plan, 0, 64, exact)
    R = 512                                             # samples per group
    rows = []
    for K in range(0, 7):
        kept = 64 >> K
        head = tn.tn_head_create(plan)
        tn.tn_contract_slices_graph(plan, 0, kept, head)
        f_est, _ = tn.tn_head_fidelity(head)
        assert math.isclose(f_est, 2.0 ** -K) and math.isclose(f_est, O.f_estimate(0, kept, 64))
        Hh = tn.tn_amplitudes(head, bits).reshape(L, 1 << h)
        F_S = O.subset_fidelity(H, Hh)
        xeb_exact = O.expected_group_sampler_xeb(Hh, P, n)
        s = tn.tn_sample(head, L * R, 0.0, 1000 + K)
        grp = np.arange(L * R) % L
        mu = np.zeros(L * R, dtype=np.int64)
        for j, q in enumerate(oq):
            mu |= ((s >> np.uint64(q)) & np.uint64(1)).astype(np.int64) << j
        x = 2.0 ** n * P[grp, mu]
        xeb = O.linear_xeb(n, P[grp, mu])
        lxeb = O.log_xeb(n, P[grp, mu])
        # the same benchmarks reduced in FP64 on the GPU against the GPU's exact head
        g_lin, g_log = tn.tn_xeb(exact, s)
        assert abs(g_lin - xeb) < 1e-4 * max(1.0, abs(xeb)), (K, g_lin, xeb)
        assert abs(g_log - lxeb) < 1e-4, (K, g_log, lxeb)
        q = O.group_sampling_law(Hh)
        ent, ent_s = O.entropy(q), O.entropy_from_samples(q[grp, mu])
        y = -np.log(q[grp, mu])
        rows.append((K, f_est, F_S, xeb_exact, xeb, lxeb, ent, ent_s))
        # samples: unbiased for the exact expectation and for the entropy
        assert abs(xeb - xeb_exact) < 4 * x.std() / math.sqrt(x.size), (K, xeb, xeb_exact)
        assert abs(ent_s - ent) < 4 * y.std() / math.sqrt(y.size), (K, ent_s, ent)
        # the kept fraction tracks the fidelity, and the XEB tracks both
        assert 0.8 < F_S / f_est < 1.25, (K, F_S, f_est)
        assert 0.75 < xeb_exact / F_S < 1.25, (K, xeb_exact, F_S)
    for kept in g["prefixes"]:       # the sparse-state fidelity against the full-space one (O1)
        K = 6 - (int(kept).bit_length() - 1)
        assert abs(rows[K][2] / float(g[f"F_true_{int(kept)}"]) - 1) < 0.1
    print("\nK  F_est     F_S       E[XEB]    XEB       logXEB    H         H_samples")
    for r in rows:
        print("%d  " % r[0] + "  ".join("%.6f" % v for v in r[1:]))


def test_xeb_against_group_size(tn):
    """Supplement, XEB against l: with the exact head the expected XEB of one
    draw per group of l follows (l - 1)/(l + 1) (Porter-Thomas), so groups of
    l = 64 already give 97% of the l = 1024 value; with 3 broken edges the
    curve is that shape times the fidelity."""
    g = np.load(GOLDEN)
    cfg = ci.config_sliced30()
    n, L, h = 30, len(cfg["tails"]), len(cfg["open_qubits"])
    P = np.abs(g["H_full"]) ** 2
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=tn.TN_GEMM_TC_FP16X3,
                      order_trials=2048, order_seed=1)
    bits = _bits(cfg)
    for kept in (64, 8):
        head = tn.tn_head_create(plan)
        tn.tn_contract_slices_graph(plan, 0, kept, head)
        Hh = tn.tn_amplitudes(head, bits).reshape(L, 1 << h)
        F_S = O.subset_fidelity(g["H_full"], Hh)
        curve = [O.expected_subgroup_xeb(Hh, P, n, 1 << b) for b in range(1, h + 1)]
        assert all(a < b for a, b in zip(curve, curve[1:]))
        for b, v in zip(range(1, h + 1), curve):
            l = 1 << b
            assert abs(v / (F_S * (l - 1) / (l + 1)) - 1) < 0.2, (kept, l, v, F_S)
        assert curve[5] / curve[-1] > 0.93                 # l = 64 against l = 1024


def test_xeb_reduction_rejects_samples_outside_the_sparse_state(tn):
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"])
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 16, head)
    s = tn.tn_sample(head, 64, 0.0, 3)
    lin, lg = tn.tn_xeb(head, s)
    psi = O.sliced_statevector(cfg["circuit"], [(g, l) for (g, l, k, v) in cfg["edges"]])
    P = np.abs(psi) ** 2
    assert abs(lin - O.linear_xeb(16, P[s.astype(np.int64)])) < 1e-4
    assert abs(lg - O.log_xeb(16, P[s.astype(np.int64)])) < 1e-4
    bad = s.copy()
    bad[7] ^= np.uint64(1)                               # flip a tail bit: not a group
    with pytest.raises(tn.TNError) as e:
        tn.tn_xeb(head, bad)
    assert e.value.code == tn.TN_ERR_NOT_IN_STATE
