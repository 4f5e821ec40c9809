"""O2: tensor-network contraction of the circuit, one group at a time.

Test infrastructure (see the package docstring); never imported by the library.

Builds the network of the Method section from scratch -- |0> vectors on the
initial boundary, a matrix per single-qubit gate, a four-way tensor per
two-qubit gate -- with every cut edge (value v) replaced by the projector
|v><v| on that wire, written as the pair of vectors <v| and |v> (the
edge-breaking insertion E = (1,0) x (1,0) of the Method section for v = 0).  The final boundary of one group is the product of basis vectors
|tail bit> on the tail qubits, with the open qubits' final wires left open:
the batch contraction of the Supplement's simulation taxonomy, run once per
group, which is the plain definition the sparse-state contraction has to
reproduce.  A slice range sums over the sliced edges' values, each slice a
separate contraction.

Contraction: repeated pairwise ``numpy.tensordot`` over shared labels, in an
order chosen on the label lists alone by randomised greedy restarts (smallest
largest intermediate wins).
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


def _build(circ, cuts, open_qubits, tail, post_cuts=()):
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
    after = {}
    for (g, leg, v) in post_cuts:
        after.setdefault(int(g), []).append((int(leg), int(v)))
    for gi, gate in enumerate(circ.gates):
        for (leg, v) in by_gate.get(gi, ()):
            # |v><v| on the wire written as its two factors: the wire ends in
            # <v| and a fresh wire starts from |v> (E = (1,0) x (1,0) for v = 0)
            q = gate.q0 if leg == 0 else gate.q1
            vec = np.zeros(2)
            vec[v] = 1.0
            net.add(vec, [wire[q]])
            e = net.label()
            net.add(vec.copy(), [e])
            wire[q] = e
        if gate.arity == 1:
            e = net.label()
            net.add(gate.U, [e, wire[gate.q0]])
            wire[gate.q0] = e
        else:
            e0, e1 = net.label(), net.label()
            net.add(gate.U.reshape(2, 2, 2, 2), [e0, e1, wire[gate.q0], wire[gate.q1]])
            wire[gate.q0], wire[gate.q1] = e0, e1
        for (leg, v) in after.get(gi, ()):
            q = gate.q0 if leg == 0 else gate.q1
            vec = np.zeros(2)
            vec[v] = 1.0
            net.add(vec, [wire[q]])
            e = net.label()
            net.add(vec.copy(), [e])
            wire[q] = e
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


def _find_order(shapes, out_set, trials=24, seed=0):
    """Pairwise order for tensors given only their label lists: randomised
    greedy restarts (score size(C) - size(A) - size(B) plus noise), keeping the
    order with the smallest largest intermediate, then the fewest flops."""
    rng = np.random.default_rng(seed)
    best = None
    for trial in range(trials):
        T = {i: list(l) for i, l in shapes.items()}
        nxt = max(T) + 1 if T else 0
        order, mx, flops = [], 0, 0.0
        tau = 0.0 if trial == 0 else rng.uniform(0.05, 1.0)
        while len(T) > 1:
            where = {}
            for tid, labs in T.items():
                for l in labs:
                    where.setdefault(l, []).append(tid)
            cand = set()
            for l, tids in where.items():
                if len(tids) == 2:
                    cand.add((min(tids), max(tids)))
            if cand:
                keys = []
                for (a, b) in cand:
                    la, lb = T[a], T[b]
                    sh = set(la) & set(lb)
                    lc = len(la) + len(lb) - 2 * len(sh)
                    sc = 2.0 ** lc - 2.0 ** len(la) - 2.0 ** len(lb)
                    k = np.sign(sc) * np.log2(1 + abs(sc))
                    if tau:
                        k -= tau * np.log(-np.log(rng.uniform(1e-12, 1)))
                    keys.append((k, a, b))
                _, a, b = min(keys)
            else:
                ids = sorted(T, key=lambda t: len(T[t]))
                a, b = ids[0], ids[1]
            la, lb = T.pop(a), T.pop(b)
            sh = [l for l in la if l in lb and l not in out_set]
            lc = [l for l in la if l not in sh] + [l for l in lb if l not in sh]
            mx = max(mx, len(lc))
            flops += 2.0 ** (len(la) + len(lb) - len(sh))
            T[nxt] = lc
            order.append((a, b, nxt))
            nxt += 1
        key = (mx, flops)
        if best is None or key < best[0]:
            best = (key, order)
    return best[1]


def _pairwise(A, la, B, lb, out_set, stats=None):
    shared = [l for l in la if l in lb and l not in out_set]
    C = np.tensordot(A, B, axes=([la.index(l) for l in shared], [lb.index(l) for l in shared]))
    if stats is not None:     # complex multiply-adds of this tensordot: |A| |B| / |shared|
        stats["complex_macs"] = stats.get("complex_macs", 0.0) + float(A.size) * float(B.size) / float(
            np.prod([A.shape[la.index(l)] for l in shared]) if shared else 1.0)
    return C, [l for l in la if l not in shared] + [l for l in lb if l not in shared]


def _absorb_small(T, out_set, stats=None):
    """Contract every tensor with at most two labels into a neighbour (exact)."""
    changed = True
    while changed and len(T) > 1:
        changed = False
        where = {}
        for tid, (_, labs) in T.items():
            for l in labs:
                where.setdefault(l, []).append(tid)
        for tid in list(T):
            if tid not in T or len(T[tid][1]) > 2:
                continue
            nbrs = [o for l in T[tid][1] for o in where.get(l, []) if o != tid and o in T]
            if not nbrs:
                continue
            o = min(nbrs, key=lambda x: T[x][0].size)
            A, la = T.pop(o)
            B, lb = T.pop(tid)
            T[o] = _pairwise(A, la, B, lb, out_set, stats)
            changed = True
            break


_ORDER_CACHE = {}


def _contract(net, out_labels, stats=None):
    T = net.tensors
    out_set = set(out_labels)
    _absorb_small(T, out_set, stats)
    # The order depends on the label lists alone, which are the same for every
    # slice of one network (only the cut vectors' entries change), so it is
    # found once per label structure.
    key = (tuple(sorted((i, tuple(l)) for i, (_, l) in T.items())), tuple(sorted(out_set)))
    order = _ORDER_CACHE.get(key)
    if order is None:
        order = _ORDER_CACHE[key] = _find_order({i: l for i, (_, l) in T.items()}, out_set)
    for (a, b, c) in order:
        A, la = T.pop(a)
        B, lb = T.pop(b)
        T[c] = _pairwise(A, la, B, lb, out_set, stats)
    (arr, labs), = T.values()
    return arr, labs


def network_amplitudes(circ, open_qubits, tails, sliced_edges=(), pins=(), slice_range=None,
                       groups=None, stats=None) -> np.ndarray:
    """H[g][mu] for the selected groups (all by default), mu bit j = open_qubits[j].

    sliced_edges: [(gate, leg)] or [(gate, leg, companion)] enumerated as slice id
    bits (a companion also fixes the partner output, as in sliced_statevector);
    pins: [(gate, leg, value)].  stats: optional dict; its "complex_macs" entry
    is increased by the complex multiply-adds of every tensordot."""
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
            cuts, post = [], []
            for j, e in enumerate(sliced_edges):
                v = (s >> j) & 1
                cuts.append((e[0], e[1], v))
                if len(e) > 2 and e[2]:
                    post.append((e[0], 1 - e[1], v))
            cuts += list(pins)
            net, out_labels = _build(circ, cuts, open_qubits, tails[g], post)
            arr, labs = _contract(net, out_labels, stats)
            # order axes as (open[h-1], ..., open[0]) so C-order flattening gives mu
            perm = [labs.index(out_labels[j]) for j in range(h - 1, -1, -1)]
            arr = np.transpose(arr, perm) if h else arr
            H[gi] += np.asarray(arr).reshape(-1)
    return H
