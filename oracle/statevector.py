"""O1: complex128 state-vector simulation of a circuit with cut edges.

Test infrastructure (see the package docstring); never imported by the library.

Conventions: qubit q is bit q of a basis-state index (LSB = qubit 0); a gate's
matrix has row = output, column = input, two-qubit basis |q0 q1> with q0 high.

A cut edge (gate g, leg j, value v) is the wire entering gate g on its j-th
qubit.  Fixing it to v is the projector |v><v| on that qubit just before the
gate: the edge-breaking insertion E = (1,0) x (1,0) of the Method section for
v = 0, and its mirror for v = 1.  Slicing (Supplement, "Slicing and contraction
order") fixes the k sliced edges to the bits of a slice id s -- edge j takes
(s >> j) & 1 -- and the result of the network is the sum over slices, so the
sum over all 2^k slices equals the unsliced circuit because sum_v |v><v| = I.
"""
from __future__ import annotations

import numpy as np


def _axis(n: int, q: int) -> int:
    # C-order reshape to [2]*n puts the most significant bit (qubit n-1) first
    return n - 1 - q


def apply_1q(psi: np.ndarray, n: int, q: int, U: np.ndarray) -> np.ndarray:
    t = psi.reshape([2] * n)
    ax = _axis(n, q)
    t = np.tensordot(U, t, axes=([1], [ax]))          # new axis 0 = output
    t = np.moveaxis(t, 0, ax)
    return t.reshape(-1)


def apply_2q(psi: np.ndarray, n: int, q0: int, q1: int, U: np.ndarray) -> np.ndarray:
    t = psi.reshape([2] * n)
    a0, a1 = _axis(n, q0), _axis(n, q1)
    G = U.reshape(2, 2, 2, 2)                         # [out0, out1, in0, in1]
    t = np.tensordot(G, t, axes=([2, 3], [a0, a1]))   # axes 0,1 = out0, out1
    t = np.moveaxis(t, [0, 1], [a0, a1])
    return t.reshape(-1)


def project(psi: np.ndarray, n: int, q: int, v: int) -> np.ndarray:
    t = psi.reshape([2] * n).copy()
    idx = [slice(None)] * n
    idx[_axis(n, q)] = 1 - v
    t[tuple(idx)] = 0
    return t.reshape(-1)


def statevector(circ, cuts=(), post_cuts=()) -> np.ndarray:
    """Final state of `circ` from |0...0> with every edge in `cuts` fixed.

    cuts: iterable of (gate_index, leg, value), the wire entering the gate;
    post_cuts: iterable of (gate_index, leg, value), the wire leaving the gate
    on that leg's qubit (the companion edge of Method case (ii))."""
    n = circ.n_qubits
    by_gate = {}
    for (g, leg, v) in cuts:
        by_gate.setdefault(int(g), []).append((int(leg), int(v)))
    after = {}
    for (g, leg, v) in post_cuts:
        after.setdefault(int(g), []).append((int(leg), int(v)))
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for gi, gate in enumerate(circ.gates):
        for (leg, v) in by_gate.get(gi, ()):
            q = gate.q0 if leg == 0 else gate.q1
            psi = project(psi, n, q, v)
        if gate.arity == 1:
            psi = apply_1q(psi, n, gate.q0, gate.U)
        else:
            psi = apply_2q(psi, n, gate.q0, gate.q1, gate.U)
        for (leg, v) in after.get(gi, ()):
            q = gate.q0 if leg == 0 else gate.q1
            psi = project(psi, n, q, v)
    return psi


def sliced_statevector(circ, sliced_edges, pins=(), slice_range=None) -> np.ndarray:
    """Sum over slices s in slice_range of the state with sliced edge j fixed to
    (s >> j) & 1 and every pin fixed (Supplement, slicing figure).

    A sliced edge (gate, leg, True) is a companion cut: in slice s the partner
    qubit's output of that gate is fixed to the same value (Method case (ii):
    the rank-one approximation keeps the partner output at the pinned value)."""
    k = len(sliced_edges)
    if slice_range is None:
        slice_range = (0, 1 << k)
    acc = np.zeros(1 << circ.n_qubits, dtype=np.complex128)
    for s in range(*slice_range):
        cuts, post = [], []
        for j, e in enumerate(sliced_edges):
            g, leg = e[0], e[1]
            v = (s >> j) & 1
            cuts.append((g, leg, v))
            if len(e) > 2 and e[2]:
                post.append((g, 1 - leg, v))
        cuts += [(g, leg, v) for (g, leg, v) in pins]
        acc += statevector(circ, cuts, post)
    return acc


def bitstring_index(tail: int, open_qubits, mu: int) -> int:
    """Basis index of the group member (tail, mu): open qubit open_qubits[j]
    takes bit j of mu, every other qubit takes its tail bit."""
    s = int(tail)
    for j, q in enumerate(open_qubits):
        s &= ~(1 << q)
        s |= ((mu >> j) & 1) << q
    return s


def sparse_state_from_vector(psi: np.ndarray, open_qubits, tails) -> np.ndarray:
    """The sparse state H[g][mu] = psi(tails[g] with open bits = mu) of the
    sparse-state section of the Supplement (L groups x 2^h members)."""
    h = len(open_qubits)
    H = np.empty((len(tails), 1 << h), dtype=np.complex128)
    for g, t in enumerate(tails):
        for mu in range(1 << h):
            H[g, mu] = psi[bitstring_index(int(t), open_qubits, mu)]
    return H


# ---- brute force: the full 2^n x 2^n unitary from Kronecker products ----

def _embed_1q(n, q, U):
    M = np.array([[1.0 + 0j]])
    for p in range(n - 1, -1, -1):                   # kron's first factor = highest bit
        M = np.kron(M, U if p == q else np.eye(2))
    return M


def _embed_2q(n, q0, q1, U):
    full = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    E = [[np.array([[1, 0], [0, 0]]), np.array([[0, 1], [0, 0]])],
         [np.array([[0, 0], [1, 0]]), np.array([[0, 0], [0, 1]])]]   # E[a][c] = |a><c|
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    coef = U[2 * a + b, 2 * c + d]
                    if coef == 0:
                        continue
                    M = np.array([[1.0 + 0j]])
                    for p in range(n - 1, -1, -1):
                        if p == q0:
                            f = E[a][c]
                        elif p == q1:
                            f = E[b][d]
                        else:
                            f = np.eye(2)
                        M = np.kron(M, f)
                    full += coef * M
    return full


def brute_force_state(circ, cuts=()) -> np.ndarray:
    """Same as `statevector` via explicit full-size matrices (n <= 8)."""
    n = circ.n_qubits
    assert n <= 8
    by_gate = {}
    for (g, leg, v) in cuts:
        by_gate.setdefault(int(g), []).append((int(leg), int(v)))
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for gi, gate in enumerate(circ.gates):
        for (leg, v) in by_gate.get(gi, ()):
            q = gate.q0 if leg == 0 else gate.q1
            P = np.zeros((2, 2))
            P[v, v] = 1.0
            psi = _embed_1q(n, q, P) @ psi
        if gate.arity == 1:
            psi = _embed_1q(n, gate.q0, gate.U) @ psi
        else:
            psi = _embed_2q(n, gate.q0, gate.q1, gate.U) @ psi
    return psi
