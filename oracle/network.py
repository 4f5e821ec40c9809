"""O2: tensor-network contraction of the circuit, one group at a time.

Test infrastructure (see the package docstring); never imported by the library.

Builds the network of the Method section from scratch -- |0> vectors on the
initial boundary, a matrix per single-qubit gate, a four-way tensor per
two-qubit gate -- with every cut edge (value v) replaced by the projector
|v><v| inserted on that wire (the edge-breaking matrix E of the Method
section).  The final boundary of one group is the product of basis vectors
|tail bit> on the tail qubits, with the open qubits' final wires left open:
the batch contraction of the Supplement's simulation taxonomy, run once per
group, which is the plain definition the sparse-state contraction has to
reproduce.  A slice range sums over the sliced edges' values, each slice a
separate contraction.

Contraction: repeated pairwise ``numpy.tensordot`` over shared labels, the pair
picked greedily (smallest size(C) - size(A) - size(B)).
"""
from __future__ import annotations

import numpy as np


class _Net:
    def __init__(self):
        self.tensors = {}   # id -> (array, [labels])
        self.next_id = 0
        self.next_label = 0

    def label(self):
        self.next_label += 1
        return self.next_label - 1

    def add(self, arr, labels):
        assert arr.ndim == len(labels)
        self.tensors[self.next_id] = (np.asarray(arr, dtype=np.complex128), list(labels))
        self.next_id += 1


def _build(circ, cuts, open_qubits, tail):
    n = circ.n_qubits
    net = _Net()
    wire = []
    for q in range(n):
        e = net.label()
        net.add(np.array([1.0, 0.0]), [e])
        wire.append(e)
    by_gate = {}
    for (g, leg, v) in cuts:
        by_gate.setdefault(int(g), []).append((int(leg), int(v)))
    for gi, gate in enumerate(circ.gates):
        for (leg, v) in by_gate.get(gi, ()):
            q = gate.q0 if leg == 0 else gate.q1
            P = np.zeros((2, 2))
            P[v, v] = 1.0
            e = net.label()
            net.add(P, [e, wire[q]])               # [out, in]
            wire[q] = e
        if gate.arity == 1:
            e = net.label()
            net.add(gate.U, [e, wire[gate.q0]])
            wire[gate.q0] = e
        else:
            e0, e1 = net.label(), net.label()
            net.add(gate.U.reshape(2, 2, 2, 2), [e0, e1, wire[gate.q0], wire[gate.q1]])
            wire[gate.q0], wire[gate.q1] = e0, e1
    open_set = set(int(q) for q in open_qubits)
    for q in range(n):
        if q in open_set:
            continue
        b = (int(tail) >> q) & 1
        vec = np.zeros(2)
        vec[b] = 1.0
        net.add(vec, [wire[q]])
    out_labels = [wire[q] for q in open_qubits]
    return net, out_labels


def _contract(net, out_labels):
    T = net.tensors
    out_set = set(out_labels)
    while len(T) > 1:
        where = {}
        for tid, (_, labs) in T.items():
            for l in labs:
                where.setdefault(l, []).append(tid)
        best = None
        for l, tids in where.items():
            if len(tids) != 2:
                continue
            a, b = tids
            la, lb = T[a][1], T[b][1]
            shared = set(la) & set(lb)
            size_c = 2 ** (len(la) + len(lb) - 2 * len(shared))
            score = size_c - T[a][0].size - T[b][0].size
            key = (score, size_c, min(a, b), max(a, b))
            if best is None or key < best[0]:
                best = (key, a, b)
        if best is None:                              # disconnected: outer product of two smallest
            ids = sorted(T, key=lambda t: T[t][0].size)
            a, b = ids[0], ids[1]
        else:
            a, b = best[1], best[2]
        A, la = T.pop(a)
        B, lb = T.pop(b)
        shared = [l for l in la if l in lb and l not in out_set]
        ia = [la.index(l) for l in shared]
        ib = [lb.index(l) for l in shared]
        C = np.tensordot(A, B, axes=(ia, ib))
        lc = [l for l in la if l not in shared] + [l for l in lb if l not in shared]
        net.add(C, lc)
    (arr, labs), = T.values()
    return arr, labs


def network_amplitudes(circ, open_qubits, tails, sliced_edges=(), pins=(), slice_range=None,
                       groups=None) -> np.ndarray:
    """H[g][mu] for the selected groups (all by default), mu bit j = open_qubits[j].

    sliced_edges: [(gate, leg)] enumerated as slice id bits; pins: [(gate, leg, value)]."""
    h = len(open_qubits)
    k = len(sliced_edges)
    if slice_range is None:
        slice_range = (0, 1 << k)
    if groups is None:
        groups = range(len(tails))
    groups = list(groups)
    H = np.zeros((len(groups), 1 << h), dtype=np.complex128)
    for gi, g in enumerate(groups):
        for s in range(*slice_range):
            cuts = [(ge, leg, (s >> j) & 1) for j, (ge, leg) in enumerate(sliced_edges)] + list(pins)
            net, out_labels = _build(circ, cuts, open_qubits, tails[g])
            arr, labs = _contract(net, out_labels)
            # order axes as (open[h-1], ..., open[0]) so C-order flattening gives mu
            perm = [labs.index(out_labels[j]) for j in range(h - 1, -1, -1)]
            arr = np.transpose(arr, perm) if h else arr
            H[gi] += np.asarray(arr).reshape(-1)
    return H
