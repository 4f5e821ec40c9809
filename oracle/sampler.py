"""One-sample-per-group sampler and its counter-based generator.

Test infrastructure (see the package docstring); never imported by the library.

Sampling (Method, last paragraph; Supplement, bitstring choice): the L groups are
independent, so one bitstring drawn per group is an uncorrelated sample.  Inside
a group the draw is the exact categorical law |H[g][mu]|^2 / sum_nu |H[g][nu]|^2,
the stationary law of the paper's Metropolis chain; it is taken by inverse CDF
over the inclusive prefix sums in float64.  With target fidelity 0 < f < F_head
each draw is replaced, with probability 1 - f/F_head, by a uniform bitstring:
the noisy-state mixture rho = f|psi><psi| + (1-f) I/2^n of the Supplement's
slicing section.

Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), written from its definition: a 4x32-bit
counter and 2x32-bit key, 10 rounds of two 32x32->64 multiplies with the
multipliers 0xD2511F53 and 0xCD9E8D57, key bumped by the Weyl constants
0x9E3779B9 and 0xBB67AE85 between rounds.

Stream use per sample i (counter words (i_lo, i_hi, c2, 0), key = (seed_lo, seed_hi)):
  c2 = 0 -> r0..r3: u_mix from (r1:r0), u_pick from (r3:r2), each the top 53
            bits of the 64-bit word times 2^-53;
  c2 = 1 -> r0..r3: the uniform bitstring's bits (r1:r0), masked to n qubits.
Group of sample i: i mod L.
"""
from __future__ import annotations

import numpy as np

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """One Philox-4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c0, c1, c2, c3 = (int(x) & _MASK for x in ctr)
    k0, k1 = (int(x) & _MASK for x in key)
    for r in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        if r != 9:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def _u53(lo, hi):
    return ((hi << 32) | lo) >> 11


def sample_groups(H, tails, open_qubits, n_qubits, n_samples, target_fidelity, f_head, seed):
    """Reference sampler; returns uint64 bitstrings (see the module docstring)."""
    H = np.asarray(H)
    L, l = H.shape
    w = np.abs(H) ** 2
    seed = int(seed)
    key = (seed & _MASK, (seed >> 32) & _MASK)
    mix = 0.0
    if target_fidelity > 0.0 and f_head > 0.0 and target_fidelity < f_head:
        mix = 1.0 - target_fidelity / f_head
    full = (1 << n_qubits) - 1 if n_qubits < 64 else (1 << 64) - 1
    open_mask = 0
    for q in open_qubits:
        open_mask |= 1 << int(q)
    out = np.zeros(n_samples, dtype=np.uint64)
    for i in range(n_samples):
        g = i % L
        r0, r1, r2, r3 = philox4x32_10((i & _MASK, (i >> 32) & _MASK, 0, 0), key)
        u_mix = _u53(r0, r1) * 2.0 ** -53
        u_pick = _u53(r2, r3) * 2.0 ** -53
        if mix > 0.0 and u_mix < mix:
            b0, b1, _, _ = philox4x32_10((i & _MASK, (i >> 32) & _MASK, 1, 0), key)
            out[i] = ((b1 << 32) | b0) & full
            continue
        cdf = np.cumsum(w[g])
        Z = cdf[-1]
        if Z > 0.0:
            t = u_pick * Z
            mu = int(np.searchsorted(cdf, t, side="right"))
            mu = min(mu, l - 1)
        else:
            mu = int(u_pick * l)
        s = int(tails[g]) & ~open_mask
        for j, q in enumerate(open_qubits):
            s |= ((mu >> j) & 1) << int(q)
        out[i] = s
    return out


def _weights_rn(Hg):
    # |h|^2 as re*re + im*im, each operation rounded to nearest
    return Hg.real * Hg.real + Hg.imag * Hg.imag


def _emit(tail, open_qubits, open_mask, mu):
    s = int(tail) & ~open_mask
    for j, q in enumerate(open_qubits):
        s |= ((mu >> j) & 1) << int(q)
    return s


def sample_groups_mcmc(H, tails, open_qubits, n_qubits, n_samples, target_fidelity, f_head, seed,
                       method, param):
    """In-group Markov chain (method "metropolis", param = chain length T) or
    frugal rejection (method "frugal", param = bound M), one sample per group
    (Method; Supplement, bitstring choice and validation).  Random numbers from
    Philox-4x32-10 with counter words (i_lo, i_hi, c2, t): c2 = 0 mixing and
    pick, c2 = 1 uniform bitstring, c2 = 2 chain step t, c2 = 3 frugal round t.

    Metropolis: start at member 0; propose mu' = low bits of word 0, accept when
    u * w(mu) < w(mu') (u from words 2-3), which leaves the law w/Z stationary.
    Frugal: candidate mu = low bits of word 0, accepted when
    (u * M) * Z < w(mu) * l; after 64 M rounds the last candidate is kept."""
    H = np.asarray(H)
    L, l = H.shape
    seed = int(seed)
    key = (seed & _MASK, (seed >> 32) & _MASK)
    mix = 0.0
    if target_fidelity > 0.0 and f_head > 0.0 and target_fidelity < f_head:
        mix = 1.0 - target_fidelity / f_head
    full = (1 << n_qubits) - 1 if n_qubits < 64 else (1 << 64) - 1
    open_mask = 0
    for q in open_qubits:
        open_mask |= 1 << int(q)
    out = np.zeros(n_samples, dtype=np.uint64)
    for i in range(n_samples):
        g = i % L
        lo, hi = i & _MASK, (i >> 32) & _MASK
        r0, r1, _, _ = philox4x32_10((lo, hi, 0, 0), key)
        if mix > 0.0 and _u53(r0, r1) * 2.0 ** -53 < mix:
            b0, b1, _, _ = philox4x32_10((lo, hi, 1, 0), key)
            out[i] = ((b1 << 32) | b0) & full
            continue
        w = _weights_rn(H[g])
        if method == "metropolis":
            cur, wc = 0, w[0]
            for t in range(int(param)):
                q0, _, q2, q3 = philox4x32_10((lo, hi, 2, t), key)
                prop = q0 & (l - 1)
                u = _u53(q2, q3) * 2.0 ** -53
                if u * wc < w[prop]:
                    cur, wc = prop, w[prop]
            mu = cur
        elif method == "frugal":
            M = float(param)
            Z = float(np.sum(w))
            bound = M * Z
            cand = 0
            for t in range(64 * int(param)):
                q0, _, q2, q3 = philox4x32_10((lo, hi, 3, t), key)
                cand = q0 & (l - 1)
                u = _u53(q2, q3) * 2.0 ** -53
                if u * bound < w[cand] * l:
                    break
            mu = cand
        else:
            raise ValueError(method)
        out[i] = _emit(tails[g], open_qubits, open_mask, mu)
    return out
