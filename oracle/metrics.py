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


def expected_group_sampler_xeb(H: np.ndarray, P_ideal: np.ndarray, n_qubits: int) -> float:
    """Exact expectation of the linear XEB of one-sample-per-group sampling:
    each group g drawn once with weights |H[g][mu]|^2 / sum_nu |H[g][nu]|^2,
    scored with the ideal probabilities P_ideal[g][mu]."""
    w = np.abs(H) ** 2
    w = w / w.sum(axis=1, keepdims=True)
    return float((2.0 ** n_qubits) * (w * P_ideal).sum(axis=1).mean() - 1.0)


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
