"""Fidelity, XEB, Porter-Thomas and efficiency formulas of the paper.

Test infrastructure (see the package docstring); never imported by the library.
"""
from __future__ import annotations

import math

import numpy as np


def fidelity(psi: np.ndarray, psi_hat: np.ndarray) -> float:
    """|<psi|psi_hat>|^2 / (<psi|psi> <psi_hat|psi_hat>): the fidelity of the
    approximate state used in the Supplement's validation section."""
    num = abs(np.vdot(psi, psi_hat)) ** 2
    den = np.vdot(psi, psi).real * np.vdot(psi_hat, psi_hat).real
    return float(num / den)


def companion_factor(theta: float) -> float:
    """Fidelity factor (sin^2 theta + 1)/2 of one companion-edge rank-one cut
    (Method, case (ii); Supplement, singular values of the sliced fSim)."""
    return (math.sin(theta) ** 2 + 1.0) / 2.0


def f_estimate(n_broken_edges: int, kept_slices: int, total_slices: int, companion_thetas=()) -> float:
    """F_est = 2^-K * (kept fraction of slices) * prod (sin^2 theta_i + 1)/2.

    2^-K for K broken edges (Method, edge breaking); a kept fraction f of the
    slices gives fidelity f (Supplement, slicing and fidelity); each companion
    edge multiplies by its factor (the fidelity-estimate equation)."""
    f = 2.0 ** (-n_broken_edges) * (kept_slices / total_slices)
    for th in companion_thetas:
        f *= companion_factor(th)
    return f


def linear_xeb(n_qubits: int, ideal_probs) -> float:
    """F_XEB = 2^n / N_s * sum_i P(s_i) - 1 (Supplement, validation section)."""
    p = np.asarray(ideal_probs, dtype=np.float64)
    return float((2.0 ** n_qubits) * p.mean() - 1.0)


EULER_GAMMA = 0.5772156649015329


def log_xeb(n_qubits: int, ideal_probs) -> float:
    """Logarithmic XEB, log(2^n) + gamma + <log P(s_i)> (the logarithmic
    cross-entropy benchmark the Supplement's validation figure reports beside
    the linear one).  With x = 2^n P Porter-Thomas distributed, samples drawn
    from P have E[log x] = 1 - gamma and uniform samples E[log x] = -gamma, so
    the benchmark is 1 for ideal sampling and 0 for uniform guessing."""
    p = np.asarray(ideal_probs, dtype=np.float64)
    return float(n_qubits * math.log(2.0) + EULER_GAMMA + np.log(p).mean())


def entropy(p) -> float:
    """Shannon entropy -sum p log p (natural log) of a distribution; zero
    entries contribute nothing.  The input is normalised first."""
    p = np.asarray(p, dtype=np.float64).ravel()
    p = p / p.sum()
    nz = p[p > 0]
    return float(-(nz * np.log(nz)).sum())


def entropy_from_samples(probs_at_samples) -> float:
    """Entropy estimated from samples s_i of a distribution p: -<log p(s_i)>,
    whose expectation over s_i ~ p is the entropy of p (the sample estimate of
    the Supplement's entropy figure)."""
    q = np.asarray(probs_at_samples, dtype=np.float64)
    return float(-np.log(q).mean())


def group_sampling_law(H: np.ndarray) -> np.ndarray:
    """Probability of each sparse-state member under one-sample-per-group
    sampling, each group drawn equally often: |H[g][mu]|^2 / (L sum_nu
    |H[g][nu]|^2)."""
    w = np.abs(np.asarray(H)) ** 2
    return w / (w.sum(axis=1, keepdims=True) * w.shape[0])


def expected_group_sampler_xeb(H: np.ndarray, P_ideal: np.ndarray, n_qubits: int) -> float:
    """Exact expectation of the linear XEB of one-sample-per-group sampling:
    each group g drawn once with weights |H[g][mu]|^2 / sum_nu |H[g][nu]|^2,
    scored with the ideal probabilities P_ideal[g][mu]."""
    w = np.abs(H) ** 2
    w = w / w.sum(axis=1, keepdims=True)
    return float((2.0 ** n_qubits) * (w * P_ideal).sum(axis=1).mean() - 1.0)


def expected_subgroup_xeb(H: np.ndarray, P_ideal: np.ndarray, n_qubits: int, l: int) -> float:
    """expected_group_sampler_xeb with every group of the head split into
    consecutive sub-groups of l members (the open index mu's high bits fixed),
    each sampled once: the linear XEB of the paper's group sampling as a
    function of the group size l (Supplement, XEB against group size)."""
    L, lh = H.shape
    assert lh % l == 0
    return expected_group_sampler_xeb(H.reshape(L * (lh // l), l), P_ideal.reshape(L * (lh // l), l), n_qubits)


def subset_fidelity(psi, psi_hat) -> float:
    """fidelity() restricted to the amplitudes given (here the sparse state):
    |<psi|psi_hat>|^2 / (<psi|psi> <psi_hat|psi_hat>) over that subset, an
    estimate of the full fidelity when the subset is a random sample of
    bitstrings."""
    return fidelity(np.asarray(psi).ravel(), np.asarray(psi_hat).ravel())


def normalised_probabilities(H: np.ndarray, n_qubits: int) -> np.ndarray:
    """p(s) = |psi_hat(s)|^2 / (N * 2^n / (L l)), N = sum |psi_hat|^2 over the
    sparse state: the normalisation of the Results section read as 2^n/(L l) N
    (2^27 N for n = 53, L l = 2^26)."""
    w = np.abs(H) ** 2
    N = w.sum()
    return w / (N * (2.0 ** n_qubits) / w.size)


def porter_thomas_ks(x: np.ndarray) -> float:
    """Kolmogorov-Smirnov distance between the empirical law of x = 2^n p and
    the Porter-Thomas law P(x) = e^{-x} (Results, probability histogram)."""
    xs = np.sort(np.asarray(x, dtype=np.float64).ravel())
    n = xs.size
    cdf = 1.0 - np.exp(-xs)
    hi = np.arange(1, n + 1) / n - cdf
    lo = cdf - np.arange(0, n) / n
    return float(max(hi.max(), lo.max()))


def gpu_efficiency(T_c: float, peak_flops: float, seconds: float) -> float:
    """8 T_c / (P t): the GPU-efficiency definition of the complexity table
    (8 real flops per complex multiply-add)."""
    return 8.0 * T_c / (peak_flops * seconds)
