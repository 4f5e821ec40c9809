"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each test names the passage or the mathematics it checks against.
"""
import json
import math
import os

import numpy as np
import pytest

import circuit_inputs as ci
import oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


# ---------------- gates (fSim equation; Supplement, sliced fSim) ----------------

def test_gates_unitary_and_square_roots():
    for k, U in ci.SQRT_GATES.items():
        assert np.allclose(U.conj().T @ U, np.eye(2), atol=1e-14)
        G = {"sx": np.array([[0, 1], [1, 0]]), "sy": np.array([[0, -1j], [1j, 0]]),
             "sw": (np.array([[0, 1], [1, 0]]) + np.array([[0, -1j], [1j, 0]])) / math.sqrt(2)}[k]
        # (I - iG)/sqrt 2 squares to -iG: a square root of G up to a global phase
        assert np.allclose(U @ U, -1j * G, atol=1e-14)
    U = ci.fsim(1.3, 0.4)
    assert np.allclose(U.conj().T @ U, np.eye(4), atol=1e-14)


@pytest.mark.parametrize("theta", [math.pi / 2, math.pi / 2 + 0.1, math.pi / 2 - 0.07, 1.0])
@pytest.mark.parametrize("leg,v", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_pinned_fsim_singular_values_fix_companion_factor(theta, leg, v):
    """Supplement, singular values of the sliced fSim: pinning one input of the
    fSim leaves squared singular values {1 + sin^2 theta, cos^2 theta} across
    the partner qubit's output (the companion edge); the kept share of the
    norm is the companion factor."""
    G = ci.fsim(theta, 0.5).reshape(2, 2, 2, 2)           # [o0, o1, i0, i1]
    T = G[:, :, v, :] if leg == 0 else G[:, :, :, v]      # [o0, o1, free input]
    if leg == 0:       # companion = partner output o1: group (free input, o0) vs o1
        M = np.transpose(T, (2, 0, 1)).reshape(4, 2)
    else:              # companion = partner output o0
        M = np.transpose(T, (2, 1, 0)).reshape(4, 2)
    s2 = np.sort(np.linalg.svd(M, compute_uv=False) ** 2)[::-1]
    assert np.allclose(s2, [1 + math.sin(theta) ** 2, math.cos(theta) ** 2], atol=1e-13)
    assert math.isclose(s2[0] / s2.sum(), O.companion_factor(theta), rel_tol=1e-13)


def test_double_pin_is_rank_one_product():
    """Method case (i): both inputs pinned to 0 gives B = (1,0) x (1,0)."""
    G = ci.fsim(math.pi / 2 + 0.05, math.pi / 6).reshape(2, 2, 2, 2)
    B = G[:, :, 0, 0]
    assert np.allclose(B, np.outer([1, 0], [1, 0]), atol=1e-15)


# ---------------- simulator ----------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_statevector_matches_brute_force(seed):
    c = ci.make_random_2q_circuit(5, 3, seed=seed)
    twoq = c.two_qubit_gates()
    cuts = [(twoq[1], 0, 1), (twoq[3], 1, 0)]
    for cc in ([], cuts):
        a = O.statevector(c, cc)
        b = O.brute_force_state(c, cc)
        assert np.abs(a - b).max() < 1e-13


def test_statevector_grid_brute_force_and_norm():
    c = ci.make_grid_circuit(2, 3, 5, seed=9)
    a = O.statevector(c)
    assert abs(np.linalg.norm(a) - 1.0) < 1e-13      # unitary network
    assert np.abs(a - O.brute_force_state(c)).max() < 1e-13


def test_bitstring_index_convention():
    # qubit q is bit q; open qubit j takes bit j of mu
    assert O.bitstring_index(0b1010, [0, 2], 0b11) == 0b1111
    assert O.bitstring_index(0b1111, [1], 0) == 0b1101


# ---------------- O1 vs O2 (two independent routes) ----------------

@pytest.mark.parametrize("case", [dict(r=3, c=4, m=6, seed=5, n_open=4, L=6, cut=1),
                                  dict(r=2, c=4, m=8, seed=6, n_open=0, L=5, cut=1),
                                  dict(r=3, c=3, m=5, seed=8, n_open=9, L=1, cut=0)])
def test_statevector_matches_network(case):
    cfg = ci.config_small(case["r"], case["c"], case["m"], seed=case["seed"], n_open=case["n_open"],
                          L=case["L"], n_cut_gates=case["cut"])
    circ = cfg["circuit"]
    se = [(g, l) for (g, l, k, v) in cfg["edges"]]
    psi = O.sliced_statevector(circ, se, slice_range=(1, 3) if se else None)
    H1 = O.sparse_state_from_vector(psi, cfg["open_qubits"], cfg["tails"])
    H2 = O.network_amplitudes(circ, cfg["open_qubits"], cfg["tails"], se, slice_range=(1, 3) if se else None)
    assert np.abs(H1 - H2).max() <= 1e-12 * max(1e-300, np.abs(H1).max())


def test_generic_gates_network_matches_statevector():
    c = ci.make_random_2q_circuit(6, 3, seed=4)
    tails = ci.draw_tails(6, [1, 4], 5, seed=1)
    twoq = c.two_qubit_gates()
    se = [(twoq[2], 0), (twoq[4], 1)]
    pins = [(twoq[5], 0, 1)]
    psi = O.sliced_statevector(c, se, pins=pins)
    H1 = O.sparse_state_from_vector(psi, [1, 4], tails)
    H2 = O.network_amplitudes(c, [1, 4], tails, se, pins=pins)
    assert np.abs(H1 - H2).max() < 1e-13


# ---------------- slicing identities (Supplement, slicing) ----------------

def test_slice_sum_equals_unsliced():
    c = ci.make_grid_circuit(3, 4, 8, seed=2)
    se = [(g, l) for (g, l, k, v) in ci.mid_circuit_cut_edges(c, 3)]      # 2^6 slices
    full = O.statevector(c)
    summed = O.sliced_statevector(c, se)
    assert np.abs(full - summed).max() < 1e-14


def test_prefix_kept_range_equals_pinned_top_bits():
    """Keeping slices [0, 2^(k-t)) is the same as pinning the top t sliced
    edges to 0 and summing the others (kept fraction 2^-t)."""
    c = ci.make_grid_circuit(3, 3, 7, seed=4)
    se = [(g, l) for (g, l, k, v) in ci.mid_circuit_cut_edges(c, 2)]      # k = 4
    kept = O.sliced_statevector(c, se, slice_range=(0, 4))
    pinned = O.sliced_statevector(c, se[:2], pins=[(g, l, 0) for (g, l) in se[2:]])
    assert np.abs(kept - pinned).max() < 1e-14


def test_hole_equals_gate_removed_and_outputs_projected():
    """Method case (i): pinning both inputs of an fSim to 0 acts like the
    product of (1,0) vectors: the gate disappears and both wires are |0><0|."""
    c = ci.make_grid_circuit(3, 3, 6, seed=12)
    gi = ci.mid_circuit_cut_edges(c, 1)[0][0]
    a = O.statevector(c, [(gi, 0, 0), (gi, 1, 0)])
    c2 = ci.Circuit(c.n_qubits, list(c.gates), c.rows, c.cols, c.cycles, c.seed, c.cycle_first_gate)
    g = c.gates[gi]
    c2.gates[gi] = ci.Gate(2, g.q0, g.q1, np.diag([1.0, 0, 0, 0]).astype(np.complex128), kind="proj00")
    b = O.statevector(c2)
    assert np.abs(a - b).max() < 1e-15


# ---------------- fidelity and statistics ----------------

def test_kept_fraction_tracks_fidelity_and_norm():
    """Method (path-integral view) and Supplement (slicing): summing a fraction
    f of the slices gives fidelity ~ f and squared norm ~ f (Results, norm vs
    summed fraction).  Bands measured on this seeded circuit."""
    c = ci.make_grid_circuit(4, 4, 12, seed=21)
    se = [(g, l) for (g, l, k, v) in ci.mid_circuit_cut_edges(c, 2)]      # k = 4
    psi = O.statevector(c)
    for kept in (2, 4, 8):
        hat = O.sliced_statevector(c, se, slice_range=(0, kept))
        f = kept / 16
        F = O.fidelity(psi, hat)
        nrm = np.vdot(hat, hat).real
        assert 0.6 * f < F < 1.5 * f, (kept, F)
        assert 0.6 * f < nrm < 1.5 * f, (kept, nrm)
        assert math.isclose(O.f_estimate(0, kept, 16), f)


def test_porter_thomas_and_exact_sampling_xeb():
    """Results (Porter-Thomas histogram) and the validation section's XEB: the
    exact state of a deep random circuit is close to Porter-Thomas and exact
    one-group sampling has E[XEB] = 2^n sum P^2 - 1 ~ 1."""
    c = ci.make_grid_circuit(4, 4, 14, seed=31)
    n = 16
    psi = O.statevector(c)
    P = np.abs(psi) ** 2
    assert O.porter_thomas_ks(P * 2 ** n) < 0.03
    H = psi.reshape(1, -1)                              # one group, all qubits open
    samples = O.sample_groups(H, np.zeros(1, np.uint64), list(range(n)), n, 20000, 0.0, 1.0, seed=7)
    x = 2 ** n * P[samples.astype(np.int64)]
    expect = O.expected_group_sampler_xeb(H, P.reshape(1, -1), n)
    assert abs(expect - ((2 ** n) * (P * P).sum() - 1)) < 1e-12
    assert abs(x.mean() - 1 - expect) < 3 * x.std() / math.sqrt(x.size)
    assert 0.8 < expect < 1.2


def test_group_sampler_xeb_dirichlet_closed_form():
    """For Porter-Thomas weights, one exact draw per group of size l has
    E[XEB] = (l - 1)/(l + 1) (Dirichlet(1,...,1) weights, Gamma(l) sum)."""
    L, h = 20000, 4
    l = 1 << h
    H = ci.synthetic_head(L, h, seed=5)
    n = 30
    P = np.abs(H) ** 2 / 2 ** n                        # ideal = approximate, mean 2^-n
    s = O.sample_groups(H, np.arange(L, dtype=np.uint64) << np.uint64(h), list(range(h)), n, L, 0.0, 1.0,
                        seed=11)
    mu = (s & np.uint64(l - 1)).astype(np.int64)
    x = 2 ** n * P[np.arange(L), mu]
    closed = (l - 1) / (l + 1)
    assert abs(x.mean() - 1 - closed) < 3 * x.std() / math.sqrt(L) + 0.01


def test_sampler_categorical_frequencies_and_mixing():
    H = ci.synthetic_head(1, 3, seed=2)
    w = np.abs(H[0]) ** 2
    w /= w.sum()
    n = 20000
    s = O.sample_groups(H, np.zeros(1, np.uint64), [0, 1, 2], 3, n, 0.0, 1.0, seed=3)
    cnt = np.bincount(s.astype(np.int64), minlength=8)
    chi2 = ((cnt - n * w) ** 2 / (n * w)).sum()
    assert chi2 < 24.3                                 # chi2(7) 99.9% quantile
    # mixing: fraction 1 - f/F_head of draws replaced by uniform 20-qubit strings
    s = O.sample_groups(H, np.zeros(1, np.uint64), [0, 1, 2], 20, n, 0.25, 1.0, seed=4)
    frac_high = np.mean(s >= 8)                        # exact draws never set bits >= 3
    assert abs(frac_high - 0.75 * (1 - 8 / 2 ** 20)) < 0.02


def test_philox_known_answer_vectors():
    """Philox-4x32-10 against the published known-answer vectors of the
    Random123 distribution (Salmon et al., SC'11): counter and key all zero,
    all ones, and the pi-digit counter/key."""
    kat = [((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
           ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
           ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
            (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for ctr, key, want in kat:
        assert O.philox4x32_10(ctr, key) == want


def test_linear_xeb_formula():
    """F_XEB = 2^n <P(s_i)> - 1 (Supplement, validation section) through
    oracle.linear_xeb, pinned by three closed forms: a computational-basis
    state sampled exactly scores 2^n - 1; uniformly random bitstrings score 0
    in expectation; exact samples of a random 16-qubit state score
    2^n sum P^2 - 1 in expectation (samples drawn with NumPy's own
    categorical sampler, not the oracle's)."""
    n = 16
    P = np.zeros(1 << n)
    P[12345] = 1.0
    assert O.linear_xeb(n, P[[12345] * 10]) == 2.0 ** n - 1
    c = ci.make_grid_circuit(4, 4, 14, seed=31)
    P = np.abs(O.statevector(c)) ** 2
    rng = np.random.default_rng(17)
    N = 40000
    u = rng.integers(0, 1 << n, N)
    x = 2.0 ** n * P[u]
    assert abs(O.linear_xeb(n, P[u])) < 3 * x.std() / math.sqrt(N)
    s = rng.choice(1 << n, size=N, p=P / P.sum())
    x = 2.0 ** n * P[s]
    expect = 2.0 ** n * (P * P).sum() - 1
    assert abs(O.linear_xeb(n, P[s]) - expect) < 3 * x.std() / math.sqrt(N)
    assert 0.8 < expect < 1.2


def test_log_xeb_closed_forms():
    """Logarithmic XEB through oracle.log_xeb: 1 for exact sampling and 0 for
    uniform sampling of a Porter-Thomas state (E[log x] = 1 - gamma and
    -gamma for x = 2^n P), n log 2 + gamma for a basis state sampled exactly;
    the samples come from NumPy's categorical and uniform generators."""
    n = 16
    P = np.zeros(1 << n)
    P[7] = 1.0
    assert math.isclose(O.log_xeb(n, P[[7, 7, 7]]), n * math.log(2) + O.EULER_GAMMA, rel_tol=1e-14)
    c = ci.make_grid_circuit(4, 4, 14, seed=31)
    P = np.abs(O.statevector(c)) ** 2
    rng = np.random.default_rng(5)
    N = 60000
    s = rng.choice(1 << n, size=N, p=P / P.sum())
    u = rng.integers(0, 1 << n, N)
    for samples, want in ((s, 1.0), (u, 0.0)):
        y = np.log(2.0 ** n * P[samples])
        assert abs(O.log_xeb(n, P[samples]) - want) < 3 * y.std() / math.sqrt(N) + 0.02


def test_entropy_closed_forms_and_sample_estimate():
    """Entropy of a uniform law over 2^k outcomes is k log 2; a Porter-Thomas
    law over N outcomes has entropy log N - 1 + gamma (to O(1/sqrt N)); the
    sample estimate -<log p(s_i)> of samples drawn from p (NumPy's sampler)
    matches the exact entropy within its standard error."""
    for k in (1, 5, 12):
        assert math.isclose(O.entropy(np.ones(1 << k)), k * math.log(2), rel_tol=1e-13)
    assert O.entropy([0.5, 0.5, 0.0]) == math.log(2)
    c = ci.make_grid_circuit(4, 4, 14, seed=31)
    P = np.abs(O.statevector(c)) ** 2
    Nn = P.size
    assert abs(O.entropy(P) - (math.log(Nn) - 1 + O.EULER_GAMMA)) < 0.02
    rng = np.random.default_rng(9)
    s = rng.choice(Nn, size=50000, p=P / P.sum())
    y = -np.log(P[s])
    assert abs(O.entropy_from_samples(P[s]) - O.entropy(P)) < 3 * y.std() / math.sqrt(s.size)


def test_subgroup_xeb_dirichlet_closed_form():
    """XEB of one exact draw per sub-group of size l from Porter-Thomas
    weights is (l - 1)/(l + 1) (the Dirichlet form); the sub-group split of a
    head equals building the smaller groups directly, and l = 1 gives 0."""
    L, h = 256, 10
    H = ci.synthetic_head(L, h, seed=12)
    P = np.abs(H) ** 2 / 2 ** 30
    for l in (2, 8, 64, 1024):
        x = O.expected_subgroup_xeb(H, P, 30, l)
        assert abs(x - (l - 1) / (l + 1)) < 0.02, (l, x)
        assert math.isclose(x, O.expected_group_sampler_xeb(H.reshape(-1, l), P.reshape(-1, l), 30), rel_tol=1e-12)
    assert abs(O.expected_subgroup_xeb(H, P, 30, 1) - (P.mean() * 2 ** 30 - 1)) < 1e-12


def test_group_sampling_law_matches_sampler_frequencies():
    """The law of one-sample-per-group draws: each group equally often, inside
    a group |H|^2 normalised; checked against the oracle sampler's counts
    (chi-squared) and against its closed-form expected XEB."""
    H = ci.synthetic_head(4, 3, seed=8)
    q = O.group_sampling_law(H)
    assert abs(q.sum() - 1) < 1e-14 and np.allclose(q.sum(axis=1), 0.25)
    n = 40000
    s = O.sample_groups(H, np.arange(4, dtype=np.uint64) << np.uint64(3), [0, 1, 2], 5, n, 0.0, 1.0, seed=3)
    cnt = np.bincount(s.astype(np.int64), minlength=32).reshape(4, 8)
    chi2 = ((cnt - n * q) ** 2 / (n * q)).sum()
    assert chi2 < 61.1                                   # chi2(31) 99.9%
    Pid = np.abs(ci.synthetic_head(4, 3, seed=9)) ** 2 / 2 ** 5
    assert math.isclose((q * Pid).sum() * 2 ** 5 - 1, O.expected_group_sampler_xeb(H, Pid, 5), rel_tol=1e-12)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_pinned_edges_halve_fidelity(seed):
    """Method, edge breaking: each broken (pinned) edge halves the fidelity, so
    K pins give F_true ~ f_estimate(K, 1, 1) = 2^-K; the squared norm of the
    pinned state also tracks 2^-K.  Bands measured on these seeded 16-qubit
    circuits (ratios 0.95-1.06 for K <= 6); a dropped or doubled factor 2
    falls far outside them."""
    c = ci.make_grid_circuit(4, 4, 12, seed=seed)
    edges = [(g, l) for (g, l, k, v) in ci.mid_circuit_cut_edges(c, 3)]
    psi = O.statevector(c)
    for K in range(1, 7):
        hat = O.statevector(c, [(g, l, 0) for (g, l) in edges[:K]])
        f = O.f_estimate(K, 1, 1)
        assert 0.85 < O.fidelity(psi, hat) / f < 1.15, K
        assert 0.85 < np.vdot(hat, hat).real / f < 1.15, K
    # with slices: K pins and a kept fraction multiply
    se = edges[2:4]
    hat = O.sliced_statevector(c, se, pins=[(g, l, 0) for (g, l) in edges[:2]], slice_range=(0, 2))
    f = O.f_estimate(2, 2, 4)
    assert math.isclose(f, 2 ** -2 * 0.5)
    assert 0.75 < O.fidelity(psi, hat) / f < 1.3


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_c_statevector_matches_numpy_and_brute_force(seed):
    """The in-place C route of O1 (used for the 30-qubit golden values) equals
    the NumPy route with cuts and companion cuts, and the brute-force
    Kronecker route on small circuits; norm 1 without cuts."""
    from oracle.statevector_c import overlap, statevector_inplace
    c = ci.make_random_2q_circuit(6, 5, seed=seed)
    twoq = c.two_qubit_gates()
    cuts = [(twoq[2], 0, 1), (twoq[4], 1, 0)]
    a = statevector_inplace(c, cuts)
    assert np.abs(a - O.brute_force_state(c, cuts)).max() < 1e-13
    g = ci.make_grid_circuit(4, 4, 10, seed=seed)
    e = [(gg, l, v) for (gg, l, k, v) in ci.mid_circuit_cut_edges(g, 2, value=1)]
    post = [(e[0][0], 1, 1)]
    assert np.abs(statevector_inplace(g, e[:3], post) - O.statevector(g, e[:3], post)).max() < 1e-13
    psi = statevector_inplace(g)
    ov, nn = overlap(psi, psi)
    assert abs(nn - 1) < 1e-12 and abs(ov - 1) < 1e-12


def test_sliced30_golden_file_identities():
    """The stored 30-qubit O1 results obey what the mathematics fixes: the
    uncut state has norm 1 (unitarity); a kept prefix fixes slice bits to 0,
    a projection inside a unitary circuit, so <psi|psi_hat> = <psi_hat|psi_hat>
    and F_true equals the prefix's squared norm exactly; the sparse state's
    mean |psi|^2 is 2^-30 to a few percent (Porter-Thomas sample of 65,536);
    its inputs are those of the 30-qubit workload."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "sliced30_o1.npz"))
    cfg = ci.config_sliced30()
    assert np.array_equal(g["tails"], np.asarray(cfg["tails"], dtype=np.uint64))
    assert list(g["open_qubits"]) == cfg["open_qubits"]
    assert abs(float(g["norm2_full"]) - 1) < 1e-12
    for kept in g["prefixes"]:
        assert abs(float(g[f"F_true_{kept}"]) - float(g[f"norm2_{kept}"])) < 1e-12
        assert abs(float(g[f"F_true_{kept}"]) / (kept / 64) - 1) < 0.05
    m = (np.abs(g["H_full"]) ** 2).mean() * 2 ** 30
    assert abs(m - 1) < 0.05
    assert O.porter_thomas_ks((np.abs(g["H_full"]) ** 2 * 2 ** 30).ravel()) < 0.02


def test_philox_words_uniform():
    words = []
    for i in range(4000):
        words.extend(O.philox4x32_10((i, 0, 0, 0), (123, 456)))
    w = np.array(words, dtype=np.uint64)
    bits = np.unpackbits(w.astype(">u4").view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    hist = np.bincount((w >> np.uint64(28)).astype(np.int64), minlength=16)
    e = w.size / 16
    assert ((hist - e) ** 2 / e).sum() < 37.7          # chi2(15) 99.9%
    # different keys / counters give different streams
    assert O.philox4x32_10((0, 0, 0, 0), (0, 0)) != O.philox4x32_10((0, 0, 0, 0), (1, 0))
    assert O.philox4x32_10((0, 0, 0, 0), (0, 0)) != O.philox4x32_10((1, 0, 0, 0), (0, 0))


def test_normalisation_mean_one():
    H = ci.synthetic_head(64, 6, seed=1)
    p = O.normalised_probabilities(H, 30)
    assert abs(p.mean() * 2 ** 30 - 1.0) < 1e-12


# ---------------- the paper's printed numbers ----------------

def test_paper_efficiency_numbers():
    e = GOLDEN["efficiency"]
    P = e["v100_fp32_peak_flops"]
    assert abs(O.gpu_efficiency(e["Tc_head_branch_merged"], P, e["t_head_s"]) - e["eff_head"]) < 0.005
    assert abs(O.gpu_efficiency(e["Tc_tail_branch_merged"], P, e["t_tail_s"]) - e["eff_tail"]) < 0.005
    tot = e["Tc_head_branch_merged"] + e["Tc_tail_branch_merged"]
    assert abs(O.gpu_efficiency(tot, P, e["t_subtask_s"]) - e["eff_overall"]) < 0.005


def test_paper_complexity_and_walltime():
    c = GOLDEN["complexity"]
    tot = 2 ** c["subtasks_log2"] * (c["Tc_head"] + c["Tc_tail"])
    assert abs(tot / c["Tc_overall"] - 1) < 0.001
    assert abs(8 * c["Tc_overall"] / c["flops_overall"] - 1) < 0.01
    w = GOLDEN["wall_time"]
    hours = 2 ** c["subtasks_log2"] * GOLDEN["efficiency"]["t_subtask_s"] / w["gpus"] / 3600
    assert abs(hours - w["hours"]) < 0.5


def test_paper_fidelity_estimate():
    f = GOLDEN["fidelity"]
    # the paper's estimate through the oracle's own formula: K broken edges and
    # 21 companion edges whose factors multiply to the printed rank-one factor
    # (equal thetas, solved from ((1 + sin^2 theta)/2)^21 = factor)
    per = f["rank_one_factor"] ** (1.0 / f["n_companions"])
    th = math.asin(math.sqrt(2 * per - 1))
    F = O.f_estimate(f["K_broken_edges"], 1, 1, [th] * f["n_companions"])
    assert math.isclose(F, 2.0 ** -f["K_broken_edges"] * f["rank_one_factor"], rel_tol=1e-12)
    assert abs(F - f["F_estimate"]) < 0.00005
    # the estimate's structure: 2^-K, kept fraction, companion factors
    th = [math.pi / 2 - 0.1] * 3
    assert math.isclose(O.f_estimate(8, 1, 1, th), 2 ** -8 * ((math.sin(th[0]) ** 2 + 1) / 2) ** 3)
    # companions at theta = pi/2 cost nothing (cos^2 theta = 0: the cut is exact)
    assert O.companion_factor(math.pi / 2) == 1.0


def test_paper_sparse_state_example_amplitudes():
    """Supplement worked example: the sparse state {111, 010, 000} of a 3-qubit
    circuit is the 3 requested amplitudes (L = 3 groups, no open qubit)."""
    ex = GOLDEN["sparse_state_example"]
    c = ci.make_random_2q_circuit(3, 2, seed=1)
    tails = np.array([int(t[::-1], 2) for t in ex["targets"]], dtype=np.uint64)   # char i = qubit i
    psi = O.statevector(c)
    H = O.sparse_state_from_vector(psi, [], tails)
    H2 = O.network_amplitudes(c, [], tails)
    assert H.shape == (3, 1)
    assert np.abs(H - H2).max() < 1e-14
    for g, t in enumerate(tails):
        assert H[g, 0] == psi[int(t)]


# ---------------- companion cuts (Method case (ii)) ----------------

def _with_theta(c, gi, theta):
    g = c.gates[gi]
    c2 = ci.Circuit(c.n_qubits, list(c.gates), c.rows, c.cols, c.cycles, c.seed, c.cycle_first_gate)
    c2.gates[gi] = ci.Gate(2, g.q0, g.q1, ci.fsim(theta, g.phi), kind="fsim", theta=theta, phi=g.phi)
    return c2


def test_companion_cut_exact_at_theta_half_pi():
    """cos(theta) = 0 makes the dropped singular value zero: slicing an input of
    fSim(pi/2, phi) with its companion and summing all slices is exact."""
    c = ci.make_grid_circuit(3, 3, 6, seed=14)
    gi = ci.mid_circuit_cut_edges(c, 1)[0][0]
    c = _with_theta(c, gi, math.pi / 2)
    exact = O.statevector(c)
    for leg in (0, 1):
        hat = O.sliced_statevector(c, [(gi, leg, True)])
        assert np.abs(hat - exact).max() < 1e-14


def test_companion_matches_between_oracle_routes():
    c = ci.make_grid_circuit(3, 4, 6, seed=15)
    cut = ci.mid_circuit_cut_edges(c, 2)
    se = [(cut[0][0], 0, True), (cut[2][0], 1, True), (cut[3][0], 0)]
    oq = [8, 9, 10, 11]
    tails = ci.draw_tails(12, oq, 5, seed=2)
    H1 = O.sparse_state_from_vector(O.sliced_statevector(c, se), oq, tails)
    H2 = O.network_amplitudes(c, oq, tails, se)
    assert np.abs(H1 - H2).max() < 1e-14


def test_companion_fidelity_tracks_estimate():
    """One companion cut at theta = pi/2 - 0.3 keeps fidelity ~ (1+sin^2)/2."""
    c = ci.make_grid_circuit(4, 4, 12, seed=16)
    gi = ci.mid_circuit_cut_edges(c, 1)[0][0]
    th = math.pi / 2 - 0.3
    c = _with_theta(c, gi, th)
    psi = O.statevector(c)
    hat = O.sliced_statevector(c, [(gi, 0, True)])
    F = O.fidelity(psi, hat)
    assert abs(F - O.companion_factor(th)) < 0.03, (F, O.companion_factor(th))


# ---------------- in-group Markov chain and frugal sampling ----------------

def test_metropolis_chain_converges_to_group_law():
    """The Metropolis chain with uniform proposals has the categorical law
    w/Z as its stationary law (Method, last paragraph)."""
    H = ci.synthetic_head(1, 3, seed=8)
    w = np.abs(H[0]) ** 2
    w /= w.sum()
    n = 6000
    s = O.sample_groups_mcmc(H, np.zeros(1, np.uint64), [0, 1, 2], 3, n, 0.0, 1.0, 5, "metropolis", 64)
    cnt = np.bincount(s.astype(np.int64), minlength=8)
    chi2 = ((cnt - n * w) ** 2 / (n * w)).sum()
    assert chi2 < 24.3                                  # chi2(7) 99.9%


def test_frugal_sampling_exact_when_bound_holds_and_xeb():
    """Frugal rejection is exact when M bounds l*w/Z; under Porter-Thomas
    with l = 64 and M = 10 its XEB matches the Dirichlet closed form
    (l-1)/(l+1) (Supplement: frugal sampling is near-perfect at l = 64)."""
    H = ci.synthetic_head(1, 3, seed=9)
    w = np.abs(H[0]) ** 2
    M = 8.0 * w.max() / w.mean()                        # bound holds
    n = 6000
    s = O.sample_groups_mcmc(H, np.zeros(1, np.uint64), [0, 1, 2], 3, n, 0.0, 1.0, 6, "frugal", int(np.ceil(M)))
    cnt = np.bincount(s.astype(np.int64), minlength=8)
    p = w / w.sum()
    assert ((cnt - n * p) ** 2 / (n * p)).sum() < 24.3
    L, h = 3000, 6
    l = 1 << h
    H = ci.synthetic_head(L, h, seed=10)
    n_q = 30
    P = np.abs(H) ** 2 / 2 ** n_q
    s = O.sample_groups_mcmc(H, np.arange(L, dtype=np.uint64) << np.uint64(h), list(range(h)), n_q, L, 0.0, 1.0,
                             7, "frugal", 10)
    mu = (s & np.uint64(l - 1)).astype(np.int64)
    x = 2 ** n_q * P[np.arange(L), mu]
    assert abs(x.mean() - 1 - (l - 1) / (l + 1)) < 3 * x.std() / math.sqrt(L) + 0.01


@pytest.mark.parametrize("case", range(8))
def test_random_cases_two_oracle_routes_agree(case):
    """O1 (state vector with projectors) and O2 (its own network builder and
    tensordot order) agree on seeded random circuits with random open sets,
    tails, sliced edges on one- and two-qubit gates, pins and companion cuts,
    over a random slice range."""
    rng = np.random.default_rng(90000 + case)
    n = int(rng.integers(3, 7))
    c = ci.make_random_2q_circuit(n, int(rng.integers(1, 4)), seed=91000 + case)
    n_open = int(rng.integers(0, n))
    oq = sorted(int(q) for q in rng.choice(n, n_open, replace=False))
    tails = ci.draw_tails(n, oq, int(rng.integers(1, min(5, 1 << (n - n_open)) + 1)), seed=92000 + case)
    se, pins, used = [], [], set()
    for _ in range(int(rng.integers(1, 5))):
        g = int(rng.integers(0, len(c.gates)))
        leg = int(rng.integers(0, c.gates[g].arity))
        if (g, leg) in used:
            continue
        used.add((g, leg))
        r = rng.random()
        if r < 0.3:
            pins.append((g, leg, int(rng.integers(0, 2))))
        elif r < 0.6 and c.gates[g].arity == 2 and (g, 1 - leg) not in used:
            se.append((g, leg, True))
        else:
            se.append((g, leg))
    b = int(rng.integers(0, 1 << len(se)))
    e = int(rng.integers(b + 1, (1 << len(se)) + 1))
    H1 = O.sparse_state_from_vector(O.sliced_statevector(c, se, pins=pins, slice_range=(b, e)), oq, tails)
    H2 = O.network_amplitudes(c, oq, tails, se, pins=pins, slice_range=(b, e))
    assert np.abs(H1 - H2).max() <= 1e-12 * max(np.abs(H1).max(), 1e-300)
