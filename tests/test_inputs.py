"""Seeded input generators (no method arithmetic): the circuit families have
the structure the input recipe states."""
import numpy as np

import circuit_inputs as ci


def test_sycamore_lattice_structure():
    """53 qubits on the staggered 9 x 6 lattice minus one site, 86 couplers in
    four patterns, each pattern a matching, every qubit of degree <= 4 and the
    coupler graph connected."""
    n, _, pats = ci.sycamore_couplers()
    assert n == 53
    edges = [e for v in pats.values() for e in v]
    assert len(edges) == 86 and len(set(map(frozenset, edges))) == 86
    for v in pats.values():
        qs = [q for e in v for q in e]
        assert len(qs) == len(set(qs))
    deg = np.zeros(n, int)
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
    assert deg.max() <= 4 and deg.min() >= 1
    seen, stack = {0}, [0]
    adj = {q: [] for q in range(n)}
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    while stack:
        for r in adj[stack.pop()]:
            if r not in seen:
                seen.add(r)
                stack.append(r)
    assert len(seen) == n


def test_circuit_layers_and_gates():
    """Each cycle: one single-qubit layer on every qubit (never repeating the
    previous gate on a qubit), then the two-qubit gates of the cycle's pattern;
    a final single-qubit layer; every gate unitary."""
    for circ in (ci.make_grid_circuit(3, 4, 8, seed=1), ci.make_sycamore_circuit(8, seed=5)):
        n = circ.n_qubits
        ones = [g for g in circ.gates if g.arity == 1]
        twos = [g for g in circ.gates if g.arity == 2]
        assert len(ones) == n * (circ.cycles + 1)
        last = {}
        for g in ones:
            key = np.round(g.U, 12).tobytes()
            assert last.get(g.q0) != key
            last[g.q0] = key
        for g in circ.gates:
            d = 2 if g.arity == 1 else 4
            assert np.allclose(g.U.conj().T @ g.U, np.eye(d), atol=1e-13)
        assert len(twos) > 0


def test_tails_distinct_and_seeded():
    oq = [8, 9, 10, 11]
    t1 = ci.draw_tails(12, oq, 64, seed=3)
    t2 = ci.draw_tails(12, oq, 64, seed=3)
    assert np.array_equal(t1, t2)
    mask = sum(1 << q for q in oq)
    assert len(set(int(t) & ~mask for t in t1)) == 64
    assert all(int(t) & mask == 0 for t in t1)
