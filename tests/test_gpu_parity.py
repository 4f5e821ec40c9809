"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: the complex64 contraction must match the complex128 oracle to
relative L2 <= 1e-5 over the whole head tensor (and every element to within
2e-5 of the largest amplitude); integer work (lookup, sampling decisions) is
bit-exact except where an FP64 prefix sum sits within rounding of a draw.
"""
import math
import os

import numpy as np
import pytest

import circuit_inputs as ci
import oracle as O

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def contract_all(tn, cfg, slice_range=None, **plan_kw):
    # host folding off unless asked for: these small circuits would otherwise
    # fold mostly on the host and leave little for the kernels under test
    plan_kw.setdefault("host_fold_log2", -1)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], **plan_kw)
    head = tn.tn_head_create(plan)
    k = tn.tn_plan_get_stats(plan)["n_sliced"]
    b, e = slice_range if slice_range else (0, 1 << k)
    tn.tn_contract_slices(plan, b, e, head)
    return plan, head


def read_head(tn, plan, head, cfg):
    """All L x 2^h amplitudes through tn_amplitudes (complex128 out)."""
    tails, oq = cfg["tails"], cfg["open_qubits"]
    h = len(oq)
    bits = np.array([O.bitstring_index(int(t), oq, mu) for t in tails for mu in range(1 << h)], dtype=np.uint64)
    out = tn.tn_amplitudes(head, bits)
    return out.reshape(len(tails), 1 << h)


def oracle_head(cfg, slice_range=None):
    se = [(g, l) for (g, l, k, v) in cfg["edges"] if k == ci.EDGE_SLICE]
    pins = [(g, l, v) for (g, l, k, v) in cfg["edges"] if k == ci.EDGE_PIN]
    psi = O.sliced_statevector(cfg["circuit"], se, pins=pins, slice_range=slice_range)
    return O.sparse_state_from_vector(psi, cfg["open_qubits"], cfg["tails"])


REL_L2_BF16 = 1e-4   # bound of the bf16x3 precision form


def assert_close(H, ref, tol=REL_L2):
    assert rel_l2(H, ref) <= tol, rel_l2(H, ref)
    assert np.abs(H - ref).max() <= 2 * tol * np.abs(ref).max()


ENGINES = [dict(gemm=0), dict(gemm=2), dict(gemm=0, small_max_bits=-1), dict(gemm=2, small_max_bits=-1),
           dict(gemm=0, small_max_bits=2), dict(gemm=3), dict(gemm=3, small_max_bits=-1), dict(gemm=4),
           dict(gemm=4, small_max_bits=-1), dict(gemm=4, host_fold_log2=0), dict(gemm=0, host_fold_log2=8)]
ENGINE_IDS = ["tc", "simt", "tc-allgemm", "simt-allgemm", "tc-small2", "bf16", "bf16-allgemm", "fp16",
              "fp16-allgemm", "fp16-fold", "tc-fold8"]


def tol_of(eng):
    return REL_L2_BF16 if eng.get("gemm") == 3 else REL_L2


@pytest.mark.parametrize("eng", ENGINES, ids=ENGINE_IDS)
def test_tiny_grid_all_amplitudes(tn, eng):
    """12-qubit 3x4 grid, 8 cycles, all qubits open: every amplitude."""
    cfg = ci.config_tiny()
    plan, head = contract_all(tn, cfg, **eng)
    H = read_head(tn, plan, head, cfg)
    ref = O.statevector(cfg["circuit"]).reshape(1, -1)
    assert_close(H, ref, tol_of(eng))


CASES = [dict(r=3, c=4, m=6, seed=5, n_open=4, L=6, cut=1),
         dict(r=4, c=4, m=8, seed=11, n_open=6, L=8, cut=2),
         dict(r=2, c=4, m=8, seed=6, n_open=0, L=5, cut=1),
         dict(r=4, c=5, m=10, seed=13, n_open=8, L=24, cut=2),
         dict(r=3, c=5, m=12, seed=17, n_open=5, L=64, cut=3)]


@pytest.mark.parametrize("case", CASES, ids=[f"{c['r']}x{c['c']}m{c['m']}L{c['L']}" for c in CASES])
@pytest.mark.parametrize("eng", ENGINES, ids=ENGINE_IDS)
def test_sliced_sparse_state_parity(tn, case, eng):
    cfg = ci.config_small(case["r"], case["c"], case["m"], seed=case["seed"], n_open=case["n_open"], L=case["L"],
                          n_cut_gates=case["cut"])
    plan, head = contract_all(tn, cfg, **eng)
    H = read_head(tn, plan, head, cfg)
    assert_close(H, oracle_head(cfg), tol_of(eng))


@pytest.mark.parametrize("seed", [1, 2])
def test_generic_two_qubit_gates_all_gemm(tn, seed):
    """Random (non-symmetric) 2q unitaries on random pairs, both orientations."""
    c = ci.make_random_2q_circuit(10, 4, seed=seed)
    twoq = c.two_qubit_gates()
    oq = [1, 4, 7]
    tails = ci.draw_tails(10, oq, 16, seed=seed)
    edges = [(twoq[5], 0, 0, 0), (twoq[9], 1, 0, 0), (twoq[12], 0, 1, 1)]
    cfg = dict(circuit=c, open_qubits=oq, tails=tails, edges=edges)
    for eng in (dict(gemm=0, small_max_bits=-1), dict(gemm=0)):
        plan, head = contract_all(tn, cfg, **eng)
        H = read_head(tn, plan, head, cfg)
        assert_close(H, oracle_head(cfg))


def test_slice_ranges_additive_and_fidelity(tn):
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)   # 16 slices
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 4, head)
    f, done = tn.tn_head_fidelity(head)
    assert done == 4 and math.isclose(f, 4 / 16)
    H = read_head(tn, plan, head, cfg)
    assert_close(H, oracle_head(cfg, (0, 4)))
    with pytest.raises(tn.TNError):
        tn.tn_contract_slices(plan, 3, 6, head)          # overlaps [0, 4)
    tn.tn_contract_slices(plan, 9, 16, head)
    tn.tn_contract_slices(plan, 4, 9, head)
    H = read_head(tn, plan, head, cfg)
    assert_close(H, oracle_head(cfg))
    with pytest.raises(tn.TNError):
        tn.tn_contract_slices(plan, 0, 17, head)


def test_pinned_edges_fidelity_estimate_and_parity(tn):
    """Method, edge breaking: each PIN edge halves F_est, so a head over a kept
    range reports F_est = 2^-n_pinned * kept / 2^k; its amplitudes are the
    oracle's with the same pins and kept slices."""
    c = ci.make_grid_circuit(4, 4, 8, seed=11)
    cut = ci.mid_circuit_cut_edges(c, 3)
    edges = [(g, l, ci.EDGE_PIN, 0) for (g, l, _, _) in cut[:3]] + \
            [(g, l, ci.EDGE_SLICE, 0) for (g, l, _, _) in cut[3:]]
    oq = [12, 13, 14, 15]
    cfg = dict(circuit=c, open_qubits=oq, tails=ci.draw_tails(16, oq, 8, seed=3), edges=edges)
    for gemm in (1, 4):
        plan, head = contract_all(tn, cfg, slice_range=(0, 5), gemm=gemm)
        st = tn.tn_plan_get_stats(plan)
        assert st["n_pinned"] == 3 and st["n_sliced"] == 3
        f, done = tn.tn_head_fidelity(head)
        assert done == 5 and math.isclose(f, 2.0 ** -3 * 5 / 8, rel_tol=1e-15)
        assert math.isclose(f, O.f_estimate(3, 5, 8), rel_tol=1e-15)
        assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg, (0, 5)))


def test_slice_shares_sum_to_the_full_head(tn):
    """The multi-GPU split on one GPU: three heads over bench.py's contiguous
    shares of the 16 slices, summed on the host, equal the full contraction
    (and the oracle); each head's F_est counts its own share."""
    from paper_2111_03011_gb300.shard import slice_share
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=4, host_fold_log2=-1)
    total = 0
    parts = []
    for r in range(3):
        b, e = slice_share(0, 16, r, 3)
        h = tn.tn_head_create(plan)
        tn.tn_contract_slices_graph(plan, b, e, h)
        assert tn.tn_head_fidelity(h) == ((e - b) / 16, e - b)
        parts.append(read_head(tn, plan, h, cfg))
        total += e - b
    assert total == 16
    full = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 16, full)
    Hf = read_head(tn, plan, full, cfg)
    assert_close(sum(parts), Hf, 1e-6)
    assert_close(sum(parts), oracle_head(cfg))


def test_amplitudes_lookup_dtypes_and_missing(tn):
    import torch
    cfg = ci.config_small(3, 4, 6, seed=5, n_open=4, L=6, n_cut_gates=1)
    plan, head = contract_all(tn, cfg)
    ref = oracle_head(cfg)
    rng = np.random.default_rng(0)
    g = rng.integers(0, 6, 100)
    mu = rng.integers(0, 16, 100)
    bits = np.array([O.bitstring_index(int(cfg["tails"][a]), cfg["open_qubits"], int(b)) for a, b in zip(g, mu)],
                    dtype=np.uint64)
    out128 = tn.tn_amplitudes(head, bits, dtype=tn.TN_C128)
    out64 = tn.tn_amplitudes(head, bits, dtype=tn.TN_C64)
    exp = ref[g, mu]
    assert np.abs(out128 - exp).max() <= 2e-5 * np.abs(ref).max()
    assert np.array_equal(out64, out128.astype(np.complex64))
    # device input and output
    dbits = torch.from_numpy(bits.view(np.int64)).cuda()
    dout = torch.zeros(100, dtype=torch.complex128, device="cuda")
    tn.tn_amplitudes(head, dbits, out=dout, dtype=tn.TN_C128)
    assert np.array_equal(dout.cpu().numpy(), out128)
    # a bitstring outside the sparse state
    bad = bits.copy()
    all_tails = set(int(t) for t in cfg["tails"])
    x = 0
    while (x & ~sum(1 << q for q in cfg["open_qubits"])) in all_tails:
        x += 1
    bad[37] = x
    with pytest.raises(tn.TNError) as e:
        tn.tn_amplitudes(head, bad)
    assert e.value.code == tn.TN_ERR_NOT_IN_STATE and "37" in str(e.value)


def _synthetic_head(tn, L, h, seed, n_qubits=30):
    import torch
    oq = list(range(n_qubits - h, n_qubits))
    tails = ci.draw_tails(n_qubits, oq, L, seed=seed)
    c = ci.make_grid_circuit(2, 2, 1, seed=1)       # plan only carries the sparse-state layout here
    c.n_qubits = n_qubits
    plan = tn.tn_plan(c, oq, tails, host_fold_log2=-1)
    H = ci.synthetic_head(L, h, seed)
    buf = torch.from_numpy(H.copy()).cuda()
    head = tn.tn_head_create(plan, buf)              # zeroes the buffer
    buf.copy_(torch.from_numpy(H))
    torch.cuda.synchronize()
    return plan, head, buf, H, tails, oq


def test_norms_fp64(tn):
    plan, head, buf, H, tails, oq = _synthetic_head(tn, 64, 10, seed=3)
    N, Z = tn.tn_head_norm(head, with_groups=True)
    w = np.abs(H) ** 2
    assert abs(N - w.sum()) <= 1e-12 * w.sum()
    assert np.allclose(Z, w.sum(axis=1), rtol=1e-13, atol=0)


def _match_with_boundaries(s_gpu, s_ref, H, tails, oq, seed, n):
    """Samples must agree; a disagreement is allowed only where the draw lies
    within 1e-12 (relative) of the boundary between the two members."""
    bad = np.nonzero(s_gpu != s_ref)[0]
    L = H.shape[0]
    for i in bad:
        g = i % L
        w = np.abs(H[g]) ** 2
        cdf = np.cumsum(w)
        r = O.philox4x32_10((i & 0xFFFFFFFF, i >> 32, 0, 0), (seed & 0xFFFFFFFF, seed >> 32))
        u = (((r[3] << 32) | r[2]) >> 11) * 2.0 ** -53
        t = u * cdf[-1]
        assert np.min(np.abs(cdf - t)) <= 1e-12 * cdf[-1], (i, s_gpu[i], s_ref[i])
    return len(bad)


@pytest.mark.parametrize("L,h,n", [(64, 10, 64), (64, 10, 1000), (300, 6, 300), (1, 12, 5000)])
def test_sampler_matches_oracle(tn, L, h, n):
    plan, head, buf, H, tails, oq = _synthetic_head(tn, L, h, seed=L + h)
    seed = 0x1234_5678_9ABC
    s = tn.tn_sample(head, n, 0.0, seed)
    ref = O.sample_groups(H, tails, oq, 30, n, 0.0, 1.0, seed)
    assert _match_with_boundaries(s, ref, H, tails, oq, seed, n) <= 1


def test_sampler_uniform_mixing_matches_oracle(tn):
    plan, head, buf, H, tails, oq = _synthetic_head(tn, 64, 10, seed=9)
    tn.tn_head_set_fidelity(head, 0.5)
    seed = 77
    s = tn.tn_sample(head, 4000, 0.2, seed)
    ref = O.sample_groups(H, tails, oq, 30, 4000, 0.2, 0.5, seed)
    assert _match_with_boundaries(s, ref, H, tails, oq, seed, 4000) <= 1
    with pytest.raises(tn.TNError):
        tn.tn_sample(head, 10, 0.9, 1)


def test_tiny_grid_sampling_xeb(tn):
    """10^4 samples of the exact 12-qubit state: XEB within 3 sigma of the
    exact expectation 2^n sum P^2 - 1 (validation section's XEB)."""
    cfg = ci.config_tiny()
    plan, head = contract_all(tn, cfg)
    f, done = tn.tn_head_fidelity(head)
    assert f == 1.0 and done == 1
    s = tn.tn_sample(head, cfg["n_samples"], 0.0, cfg["sample_seed"])
    psi = O.statevector(cfg["circuit"])
    P = np.abs(psi) ** 2
    x = 2 ** 12 * P[s.astype(np.int64)]
    expect = 2 ** 12 * (P * P).sum() - 1
    assert abs(x.mean() - 1 - expect) < 3 * x.std() / math.sqrt(x.size)


def test_sliced30_full_size_properties(tn):
    """The 30-qubit, 14-cycle, 64-slice workload at full size: the exact sparse
    state (all slices) is normalised like a Porter-Thomas sample (E|psi|^2 =
    2^-n), the partial sums track the kept fraction, and amplitudes are
    consistent between the tensor-core and CUDA-core engines."""
    cfg = ci.config_sliced30()
    plan = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], n_candidates=4,
                               order_trials=2048)
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 16, head)
    N16 = tn.tn_head_norm(head)
    tn.tn_contract_slices(plan, 16, 64, head)
    N = tn.tn_head_norm(head)
    l = 2 ** 10 * 64
    x = N * 2 ** 30 / l
    assert 0.9 < x < 1.1, x
    assert 0.15 < N16 / N < 0.4
    H = read_head(tn, plan, head, cfg)
    p = np.abs(H) ** 2 * 2 ** 30
    assert O.porter_thomas_ks(p / p.mean()) < 0.02


_SLICED30_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sliced30_o1.npz")


@pytest.mark.parametrize("gemm", [1, 3, 4], ids=["tc3xtf32", "bf16x3", "fp16x3"])
def test_sliced30_all_amplitudes_vs_stored_o1(tn, gemm):
    """The full 30-qubit, 14-cycle workload in the bench's launch
    configuration (the autotuned plan, all 64 slices replayed as one captured
    graph): every one of the 65,536 sparse-state amplitudes against the O1
    state vector stored by tests/golden/make_sliced30_golden.py (by the
    slice-sum identity, the uncut circuit).  The kept prefixes [0, 32) and
    [0, 16) are compared with the O1 runs that pin the top slice bits to 0,
    and their fidelity estimates with O1's exact fidelity."""
    g = np.load(_SLICED30_GOLDEN)
    cfg = ci.config_sliced30()
    assert np.array_equal(g["tails"], np.asarray(cfg["tails"], dtype=np.uint64))
    assert list(g["open_qubits"]) == list(cfg["open_qubits"])
    assert [tuple(e) for e in g["edges"]] == [(a, b) for (a, b, _, _) in cfg["edges"]]
    tol = tol_of(dict(gemm=gemm))
    plan = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], n_candidates=4,
                               order_trials=2048, gemm=gemm)
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices_graph(plan, 0, 64, head)
    assert_close(read_head(tn, plan, head, cfg), g["H_full"], tol)
    for kept in g["prefixes"]:
        kept = int(kept)
        h = tn.tn_head_create(plan)
        tn.tn_contract_slices_graph(plan, 0, kept, h)
        assert_close(read_head(tn, plan, h, cfg), g[f"H_{kept}"], tol)
        f_est, done = tn.tn_head_fidelity(h)
        assert done == kept and math.isclose(f_est, kept / 64)
        assert abs(float(g[f"F_true_{kept}"]) / f_est - 1) < 0.05     # the kept fraction tracks the fidelity


_SLICED30_REF = {}


@pytest.mark.parametrize("gemm", [1, 3, 4], ids=["tc3xtf32", "bf16x3", "fp16x3"])
def test_sliced30_full_size_sampled_groups_vs_oracle(tn, gemm):
    """Full-size workload in the bench's launch configuration (same plan, same
    kernels): one slice contracted for all 64 groups; two sampled groups
    checked element by element against the O2 network oracle."""
    cfg = ci.config_sliced30()
    # the plan bench.py times: the autotuner over 4 candidates of 2048 restarts
    plan = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], n_candidates=4,
                               order_trials=2048, gemm=gemm)
    assert tn.tn_plan_get_stats(plan)["autotune_candidates"] >= 1
    head = tn.tn_head_create(plan)
    s = 5
    tn.tn_contract_slices(plan, s, s + 1, head)
    H = read_head(tn, plan, head, cfg)
    se = [(g, l) for (g, l, k, v) in cfg["edges"]]
    groups = [0, 37]
    if "ref" not in _SLICED30_REF:
        _SLICED30_REF["ref"] = O.network_amplitudes(cfg["circuit"], cfg["open_qubits"], cfg["tails"], se,
                                                    slice_range=(s, s + 1), groups=groups)
    ref = _SLICED30_REF["ref"]
    for i, g in enumerate(groups):
        assert_close(H[g:g + 1], ref[i:i + 1], REL_L2_BF16 if gemm == 3 else REL_L2)


def test_profile_and_reset(tn):
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
    head = tn.tn_head_create(plan)
    ms = tn.tn_profile_slices(plan, 0, 16, head)
    st = tn.tn_plan_get_stats(plan)
    assert ms.shape == (st["n_launches"],) and (ms > 0).all()
    assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg))
    tn.tn_head_reset(head)
    assert tn.tn_head_fidelity(head) == (0.0, 0)
    tn.tn_contract_slices(plan, 0, 16, head)
    assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg))
    kinds = [tn.tn_plan_step_info(plan, i)[0] for i in range(st["n_launches"])]
    assert kinds[-1] == -1 and set(kinds[:-1]) <= {0, 1, 2, 3, 4, 5, 6}


@pytest.mark.parametrize("gemm", [0, 3, 4], ids=["tc", "bf16", "fp16"])
def test_companion_cuts_parity_and_f_est(tn, gemm):
    """Companion cuts on the GPU path vs the oracle with the partner outputs
    fixed; F_est = prod (1 + sin^2 theta)/2 over the companions."""
    import math
    c = ci.make_grid_circuit(4, 4, 10, seed=17)
    cut = ci.mid_circuit_cut_edges(c, 3)
    g0, g1, g2 = cut[0][0], cut[2][0], cut[4][0]
    edges = [(g0, 0, tn.TN_EDGE_COMPANION, 0), (g1, 1, tn.TN_EDGE_COMPANION, 0), (g2, 0, tn.TN_EDGE_SLICE, 0)]
    oq = list(range(10, 16))
    tails = ci.draw_tails(16, oq, 12, seed=5)
    cfg = dict(circuit=c, open_qubits=oq, tails=tails, edges=edges)
    plan, head = contract_all(tn, cfg, gemm=gemm)
    H = read_head(tn, plan, head, cfg)
    se = [(g0, 0, True), (g1, 1, True), (g2, 0)]
    ref = O.sparse_state_from_vector(O.sliced_statevector(c, se), oq, tails)
    assert_close(H, ref, REL_L2_BF16 if gemm == 3 else REL_L2)
    f, done = tn.tn_head_fidelity(head)
    expect = O.companion_factor(c.gates[g0].theta) * O.companion_factor(c.gates[g1].theta)
    assert done == 8 and abs(f - expect) < 1e-12


@pytest.mark.parametrize("L,h,n,T", [(64, 6, 256, 64), (16, 10, 64, 300), (1, 8, 500, 40)])
def test_metropolis_sampler_matches_oracle_bit_exact(tn, L, h, n, T):
    """In-group Metropolis chain: both sides draw the same Philox stream and
    compare round-to-nearest FP64 weights, so every sample must agree."""
    plan, head, buf, H, tails, oq = _synthetic_head(tn, L, h, seed=L + 3 * h)
    seed = 0xABCDEF12345
    s = tn.tn_sample_ex(head, n, 0.0, seed, tn.TN_SAMPLE_METROPOLIS, T)
    ref = O.sample_groups_mcmc(H, tails, oq, 30, n, 0.0, 1.0, seed, "metropolis", T)
    assert np.array_equal(s, ref)


@pytest.mark.parametrize("L,h,n,M", [(64, 6, 256, 10), (32, 10, 64, 4)])
def test_frugal_sampler_matches_oracle(tn, L, h, n, M):
    """Frugal rejection: same stream on both sides; the group sum Z is summed
    in a different order, so a draw may differ only when it sits within 1e-12
    (relative) of its acceptance threshold."""
    plan, head, buf, H, tails, oq = _synthetic_head(tn, L, h, seed=L + h + 1)
    seed = 4242
    s = tn.tn_sample_ex(head, n, 0.0, seed, tn.TN_SAMPLE_FRUGAL, M)
    ref = O.sample_groups_mcmc(H, tails, oq, 30, n, 0.0, 1.0, seed, "frugal", M)
    bad = np.nonzero(s != ref)[0]
    assert len(bad) <= 1
    for i in bad:
        lo_ref = O.sample_groups_mcmc(H * (1 + 1e-12), tails, oq, 30, i + 1, 0.0, 1.0, seed, "frugal", M)[i]
        hi_ref = O.sample_groups_mcmc(H * (1 - 1e-12), tails, oq, 30, i + 1, 0.0, 1.0, seed, "frugal", M)[i]
        assert s[i] in (lo_ref, hi_ref)


def test_sampler_methods_mixing_and_errors(tn):
    plan, head, buf, H, tails, oq = _synthetic_head(tn, 64, 6, seed=2)
    tn.tn_head_set_fidelity(head, 0.5)
    s = tn.tn_sample_ex(head, 300, 0.1, 9, tn.TN_SAMPLE_METROPOLIS, 32)
    ref = O.sample_groups_mcmc(H, tails, oq, 30, 300, 0.1, 0.5, 9, "metropolis", 32)
    assert np.array_equal(s, ref)
    with pytest.raises(tn.TNError):
        tn.tn_sample_ex(head, 10, 0.0, 1, 7, 0)


def _heads_array(tn, plan, head, cfg):
    return read_head(tn, plan, head, cfg)


def test_graph_replay_equals_plain_launches(tn):
    """Batched form: the slice range captured as a CUDA graph and replayed
    gives bit-identical heads to the plain launches (same kernels, order)."""
    cfg = ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
    h1 = tn.tn_head_create(plan)
    h2 = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 16, h1)
    tn.tn_contract_slices_graph(plan, 0, 16, h2)
    A, B = read_head(tn, plan, h1, cfg), read_head(tn, plan, h2, cfg)
    assert np.array_equal(A, B)
    assert_close(B, oracle_head(cfg))
    tn.tn_head_reset(h2)
    tn.tn_contract_slices_graph(plan, 0, 16, h2)        # replay of the cached graph
    assert np.array_equal(read_head(tn, plan, h2, cfg), A)
    with pytest.raises(tn.TNError):
        tn.tn_contract_slices_graph(plan, 0, 4, h2)      # already accumulated


def test_batch_of_mixed_circuits_in_one_graph(tn):
    """Many small circuits of uneven step shapes as parallel branches of one
    graph: each head equals its own plain contraction and the oracle."""
    shapes = [(3, 3, 6, 3, 4, 0), (3, 4, 8, 4, 6, 1), (4, 4, 6, 6, 8, 1), (2, 5, 8, 5, 4, 0),
              (4, 5, 8, 6, 16, 2), (3, 5, 10, 5, 8, 1)]
    cfgs, plans, heads, refs, plain = [], [], [], [], []
    for i, (r, c, m, h, L, cut) in enumerate(shapes):
        cfg = ci.config_small(r, c, m, seed=40 + i, n_open=h, L=L, n_cut_gates=cut)
        p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
        cfgs.append(cfg)
        plans.append(p)
        heads.append(tn.tn_head_create(p))
        hp = tn.tn_head_create(p)
        k = tn.tn_plan_get_stats(p)["n_sliced"]
        tn.tn_contract_slices(p, 0, 1 << k, hp)
        plain.append(read_head(tn, p, hp, cfg))
    ranges = [(0, 1 << tn.tn_plan_get_stats(p)["n_sliced"]) for p in plans]
    tn.tn_contract_batch(plans, ranges, heads)
    for cfg, p, hd, pl in zip(cfgs, plans, heads, plain):
        H = read_head(tn, p, hd, cfg)
        assert np.array_equal(H, pl)
        assert_close(H, oracle_head(cfg))
    for hd in heads:
        tn.tn_head_reset(hd)
    tn.tn_contract_batch(plans, ranges, heads)             # cached graph replay
    for cfg, p, hd, pl in zip(cfgs, plans, heads, plain):
        assert np.array_equal(read_head(tn, p, hd, cfg), pl)
    with pytest.raises(tn.TNError):
        tn.tn_contract_batch(plans[:2], ranges[:2], [heads[0], heads[0]])
    # the cached graph is keyed on handle identity: freed plans and heads whose
    # addresses come back for new ones (same ranges) must not replay it
    del plans, heads
    import gc
    gc.collect()
    cfgs2 = [ci.config_small(r, c, m, seed=70 + i, n_open=h, L=L, n_cut_gates=cut)
             for i, (r, c, m, h, L, cut) in enumerate(shapes)]
    plans2 = [tn.tn_plan(cf["circuit"], cf["open_qubits"], cf["tails"], cf["edges"], host_fold_log2=-1) for cf in cfgs2]
    heads2 = [tn.tn_head_create(p) for p in plans2]
    tn.tn_contract_batch(plans2, [(0, 1 << tn.tn_plan_get_stats(p)["n_sliced"]) for p in plans2], heads2)
    for cf, p, hd in zip(cfgs2, plans2, heads2):
        assert_close(read_head(tn, p, hd, cf), oracle_head(cf))


def _server_cases(tn):
    shapes = [(3, 4, 8, 4, 16, 1), (4, 4, 8, 6, 32, 2), (3, 5, 10, 5, 64, 1)]
    out = []
    for i, (r, c, m, h, L, cut) in enumerate(shapes):
        cfg = ci.config_small(r, c, m, seed=60 + i, n_open=h, L=L, n_cut_gates=cut)
        plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
        k = tn.tn_plan_get_stats(plan)["n_sliced"]
        kept = (0, max(1, (1 << k) // 2))                  # kept fraction 1/2 (1 when k = 0)
        out.append((cfg, plan, kept))
    return out


def _requests(cases, rng):
    reqs = []
    for j in range(24):
        ci_ = j % len(cases)
        cfg = cases[ci_][0]
        if j % 3 == 2:
            reqs.append(dict(circuit=ci_, kind=1, n=int(rng.integers(10, 200)), seed=int(rng.integers(1 << 40)),
                             method=int(j % 9 // 3)))
        else:
            oq, tails = cfg["open_qubits"], cfg["tails"]
            g = rng.integers(0, len(tails), 300)
            mu = rng.integers(0, 1 << len(oq), 300)
            bits = np.array([O.bitstring_index(int(tails[a]), oq, int(b)) for a, b in zip(g, mu)], np.uint64)
            reqs.append(dict(circuit=ci_, kind=0, bits=bits))
    return reqs


def _submit(tn, sv, q):
    if q["kind"] == 0:
        return tn.tn_server_submit(sv, q["circuit"], tn.TN_REQ_AMPLITUDES, 0, bitstrings=q["bits"])
    return tn.tn_server_submit(sv, q["circuit"], tn.TN_REQ_SAMPLE, q["n"], seed=q["seed"], method=q["method"],
                               param=16 if q["method"] == 1 else 0)


def test_server_results_same_alone_and_in_the_mix(tn):
    """Serving: every request's result equals the plain API on a directly
    contracted head, whether it ran alone or admitted into a busy server
    (continuous admission, overlapping slots, LRU head eviction)."""
    cases = _server_cases(tn)
    rng = np.random.default_rng(7)
    reqs = _requests(cases, rng)
    # expected: plain calls on heads built directly
    expect = []
    heads = []
    for cfg, plan, kept in cases:
        hd = tn.tn_head_create(plan)
        tn.tn_contract_slices(plan, kept[0], kept[1], hd)
        heads.append(hd)
    for q in reqs:
        hd = heads[q["circuit"]]
        if q["kind"] == 0:
            expect.append(tn.tn_amplitudes(hd, q["bits"]))
        else:
            expect.append(tn.tn_sample_ex(hd, q["n"], 0.0, q["seed"], q["method"], 16 if q["method"] == 1 else 0))
    del heads
    for mode in ("alone", "mix"):
        # heads of 4, 32 and 32 KiB: a 40 kB budget holds two at a time, forcing evictions
        sv = tn.tn_server_create(n_slots=4, hbm_budget_bytes=(64 << 30) if mode == "alone" else 40_000)
        for cfg, plan, kept in cases:
            tn.tn_server_add_circuit(sv, plan, kept[0], kept[1])
        got = []
        if mode == "alone":
            for q in reqs:
                got.append(tn.tn_server_wait(sv, _submit(tn, sv, q))[0])
        else:
            tickets = [_submit(tn, sv, q) for q in reqs]
            got = [tn.tn_server_wait(sv, t)[0] for t in tickets]
        st = tn.tn_server_get_stats(sv)
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert 0 < st["p50_us"] <= st["p99_us"]
        if mode == "mix":
            assert st["evictions"] > 0
        for q, a, b in zip(reqs, got, expect):
            assert np.array_equal(a, b), (mode, q["kind"])
        tn.tn_server_free(sv)


def test_server_merges_waiting_amplitude_requests(tn):
    """Continuous batching: with one slot busy, amplitude requests that queue
    on the same ready circuit run merged into one launch per slot; each still
    gets exactly its own amplitudes (complex64 and complex128 requests are
    batched separately), and a request with a bitstring outside the sparse
    state fails alone, reporting its own index."""
    cfg, plan, kept = _server_cases(tn)[1]
    hd = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, kept[0], kept[1], hd)
    oq, tails = cfg["open_qubits"], cfg["tails"]
    rng = np.random.default_rng(19)

    def bits(k):
        g = rng.integers(0, len(tails), k)
        mu = rng.integers(0, 1 << len(oq), k)
        return np.array([O.bitstring_index(int(tails[a]), oq, int(b)) for a, b in zip(g, mu)], dtype=np.uint64)

    sv = tn.tn_server_create(n_slots=1)
    tn.tn_server_add_circuit(sv, plan, kept[0], kept[1])
    tn.tn_server_wait(sv, tn.tn_server_submit(sv, 0, tn.TN_REQ_AMPLITUDES, 0, bitstrings=bits(4)))   # build the head
    reqs = []
    for j in range(40):
        b = bits(int(rng.integers(1, 300)))
        dt = tn.TN_C64 if j % 4 == 3 else tn.TN_C128
        bad = j == 13
        if bad:
            b[3] ^= np.uint64(1 << 0)      # tail bit 0 flipped: not one of the tails
            assert not any((int(b[3]) & ~sum(1 << q for q in oq)) == (int(t) & ~sum(1 << q for q in oq))
                           for t in tails)
        reqs.append((b, dt, bad, tn.tn_server_submit(sv, 0, tn.TN_REQ_AMPLITUDES, 0, bitstrings=b, dtype=dt)))
    for b, dt, bad, t in reqs:
        if bad:
            with pytest.raises(tn.TNError) as e:
                tn.tn_server_wait(sv, t)
            assert e.value.code == tn.TN_ERR_NOT_IN_STATE and "bitstring 3 " in str(e.value)
            continue
        got = tn.tn_server_wait(sv, t)[0]
        assert np.array_equal(got, tn.tn_amplitudes(hd, b, dtype=dt))
    st = tn.tn_server_get_stats(sv)
    assert st["completed"] == 40 and st["failed"] == 1
    tn.tn_server_free(sv)


@pytest.mark.parametrize("gemm", [3, 4], ids=["bf16x3", "fp16x3"])
def test_side_stream_bprep_bitwise_equal(tn, gemm):
    """B-prep steps launched on the side stream beside an earlier GEMM give the
    same head, bit for bit, as every step in order on one stream: in plain
    launches, in a captured graph, and against tn_profile_slices (which runs in
    order)."""
    cfg = ci.config_sliced30()
    heads = {}
    for side in (1, 0):
        plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                          order_trials=2048, order_seed=1, side_bprep=side)
        assert (tn.tn_plan_get_stats(plan)["n_side_bprep"] >= 1) == (side == 1)
        h1 = tn.tn_head_create(plan)
        tn.tn_contract_slices(plan, 0, 3, h1)
        h2 = tn.tn_head_create(plan)
        tn.tn_contract_slices_graph(plan, 0, 3, h2)
        h3 = tn.tn_head_create(plan)
        tn.tn_profile_slices(plan, 0, 3, h3)
        heads[side] = [read_head(tn, plan, h, cfg) for h in (h1, h2, h3)]
    ref = heads[0][2]
    for side in (1, 0):
        for h in heads[side]:
            assert np.array_equal(h, ref)


def test_autotuned_plan_parity(tn):
    """The autotuner times distinct candidate orders and keeps the fastest;
    whatever it keeps computes the same amplitudes."""
    cfg = ci.config_small(4, 5, 10, seed=13, n_open=8, L=24, n_cut_gates=2)
    plan = tn.tn_plan_autotune(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], n_candidates=3,
                               order_trials=16)
    st = tn.tn_plan_get_stats(plan)
    assert 1 <= st["autotune_candidates"] <= 3 and st["measured_slice_ms"] > 0
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 1 << st["n_sliced"], head)
    assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg))


@pytest.mark.parametrize("gemm", [0, 3, 4], ids=["tc", "bf16", "fp16"])
def test_automatic_slicing_parity_f_est_profile_and_graph(tn, gemm):
    """A cap that no order meets: the planner slices extra wires, runs every
    internal value inside each user slice, and the head, F_est, the profile
    and the graph replay are those of the user's slicing."""
    cfg = ci.config_small(4, 5, 10, seed=13, n_open=8, L=24, n_cut_gates=1)
    tol = REL_L2_BF16 if gemm == 3 else REL_L2
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=gemm,
                      max_log2_elements=15, auto_slice=16)
    st = tn.tn_plan_get_stats(plan)
    assert st["n_sliced"] == 2 and st["n_internal_sliced"] >= 1 and st["max_log2_elements"] <= 15 + 1e-9
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 1, 3, head)
    assert tn.tn_head_fidelity(head) == (0.5, 2)
    assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg, slice_range=(1, 3)), tol)
    tn.tn_contract_slices(plan, 0, 1, head)
    tn.tn_contract_slices_graph(plan, 3, 4, head)
    assert tn.tn_head_fidelity(head) == (1.0, 4)
    assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg), tol)
    h2 = tn.tn_head_create(plan)
    ms = tn.tn_profile_slices(plan, 0, 4, h2)
    assert ms.shape == (st["n_launches"] >> st["n_internal_sliced"],) and (ms > 0).all()
    assert_close(read_head(tn, plan, h2, cfg), oracle_head(cfg), tol)


def _sycamore_case(cycles, n_tails):
    circ = ci.make_sycamore_circuit(cycles, seed=5)
    n = circ.n_qubits
    oq = list(range(n - 6, n))
    return circ, oq, ci.draw_tails(n, oq, n_tails, seed=55)


@pytest.mark.parametrize("gemm", [1, 4], ids=["tc3xtf32", "fp16x3"])
def test_sycamore53_reduced_depth_parity(tn, gemm):
    """53-qubit Sycamore topology (reduced depth): 6 cycles against O2 live,
    8 cycles (auto-sliced to a 2^28 cap) against stored O2 amplitudes written
    by tests/golden/make_sycamore53_golden.py."""
    import os
    circ, oq, tails = _sycamore_case(6, 8)
    plan = tn.tn_plan(circ, oq, tails, [], gemm=gemm)
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 1, head)
    cfg = dict(circuit=circ, open_qubits=oq, tails=tails, edges=[])
    H = read_head(tn, plan, head, cfg)
    assert_close(H[[0, 5]], O.network_amplitudes(circ, oq, tails, [], groups=[0, 5]))
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "sycamore53_m8_o2.npz"))
    circ, oq, tails = _sycamore_case(int(g["cycles"]), len(g["tails"]))
    assert np.array_equal(np.asarray(tails, dtype=np.uint64), g["tails"])
    plan = tn.tn_plan(circ, oq, tails, [], gemm=gemm, max_log2_elements=28, auto_slice=12)
    st = tn.tn_plan_get_stats(plan)
    assert st["n_internal_sliced"] >= 1
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices_graph(plan, 0, 1, head)
    H = read_head(tn, plan, head, dict(circuit=circ, open_qubits=oq, tails=tails, edges=[]))
    assert_close(H[list(g["groups"])], g["H"])
    assert tn.tn_head_fidelity(head) == (1.0, 1)


@pytest.mark.parametrize("scale_exp", [-40, -16, 16])
def test_fp16_engine_dynamic_range(tn, scale_exp):
    """FP16x3 with per-operand power-of-two scaling keeps complex64 accuracy
    whatever the magnitude of the network's entries: two gates scaled by
    2^scale_exp (and so every amplitude by 2^(2 scale_exp)) -- far outside the
    fp16 range unscaled -- match the oracle at 1e-5."""
    import copy
    cfg = ci.config_small(4, 5, 10, seed=13, n_open=8, L=24, n_cut_gates=1)
    circ = copy.deepcopy(cfg["circuit"])
    for gi in (5, len(circ.gates) // 2):
        circ.gates[gi].U = circ.gates[gi].U * 2.0 ** scale_exp
    cfg = dict(cfg, circuit=circ)
    plan, head = contract_all(tn, cfg, gemm=tn.TN_GEMM_TC_FP16X3, small_max_bits=-1)
    assert_close(read_head(tn, plan, head, cfg), oracle_head(cfg))
