"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module only *generates data*: random circuits written out as explicit gate
matrices, random tail bitstrings, sliced-edge selections and synthetic head
tensors.  It contains none of the contraction, sampling or fidelity arithmetic
of the method, so the oracle and the CUDA path stay independent: both read the
same numbers and compute everything else on their own.

Circuit model (the paper's Sycamore-style random circuits, Sec. "Method" and the
fSim equation; gate-set details that the paper leaves to its data files are a
documented reading):

* qubits on an R x C grid, qubit q = r*C + c;
* each cycle = a layer of single-qubit gates on every qubit, drawn uniformly
  from {sqrt(X), sqrt(Y), sqrt(W)} excluding the previous one on that qubit,
  followed by one layer of fSim gates on the couplers of one pattern;
* couplers: A = horizontal bonds with even column, B = horizontal with odd
  column, C = vertical with even row, D = vertical with odd row; cycle t uses
  pattern "ABCDCDAB"[t mod 8];
* a final layer of single-qubit gates after the last cycle;
* fSim(theta, phi) per the paper's fSim equation, theta = pi/2 + U(-0.11, 0.11)
  and phi = pi/6 + U(-0.05, 0.05), fixed per coupler.

Gate matrix convention: row = output, column = input; for two-qubit gates the
basis is |q0 q1> with q0 the high bit.  Bitstrings are uint64 with qubit q at
bit q.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

PATTERN_ABCD = "ABCDCDAB"

# kinds of a cut edge (match the C ABI's TN_EDGE_* values)
EDGE_SLICE = 0
EDGE_PIN = 1
EDGE_COMPANION = 2


@dataclass
class Gate:
    arity: int
    q0: int
    q1: int          # -1 for single-qubit gates
    U: np.ndarray    # (2,2) or (4,4) complex128, row = output, column = input
    kind: str = ""   # "sx", "sy", "sw", "fsim"
    theta: float = 0.0
    phi: float = 0.0


@dataclass
class Circuit:
    n_qubits: int
    gates: list
    rows: int = 0
    cols: int = 0
    cycles: int = 0
    seed: int = 0
    cycle_first_gate: list = field(default_factory=list)  # index of each cycle's first 2q gate

    def two_qubit_gates(self):
        return [i for i, g in enumerate(self.gates) if g.arity == 2]


def _sqrt_gate(G):
    # (I - iG)/sqrt(2): a square root of G up to a global phase
    return (np.eye(2, dtype=np.complex128) - 1j * G) / math.sqrt(2.0)


_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_W = (_X + _Y) / math.sqrt(2.0)
SQRT_GATES = {"sx": _sqrt_gate(_X), "sy": _sqrt_gate(_Y), "sw": _sqrt_gate(_W)}


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) in the basis |q0 q1> (q0 high bit), as printed in the
    paper's fSim equation."""
    c, s = math.cos(theta), math.sin(theta)
    U = np.zeros((4, 4), dtype=np.complex128)
    U[0, 0] = 1.0
    U[1, 1] = c
    U[1, 2] = -1j * s
    U[2, 1] = -1j * s
    U[2, 2] = c
    U[3, 3] = np.exp(-1j * phi)
    return U


def grid_couplers(rows: int, cols: int):
    """Coupler lists of the four patterns A, B, C, D on an R x C grid."""
    pats = {"A": [], "B": [], "C": [], "D": []}
    for r in range(rows):
        for c in range(cols - 1):
            pats["A" if c % 2 == 0 else "B"].append((r * cols + c, r * cols + c + 1))
    for r in range(rows - 1):
        for c in range(cols):
            pats["C" if r % 2 == 0 else "D"].append((r * cols + c, (r + 1) * cols + c))
    return pats


def make_grid_circuit(rows: int, cols: int, cycles: int, seed: int,
                      sequence: str = PATTERN_ABCD) -> Circuit:
    """Seeded Sycamore-like circuit on an R x C grid (see the module docstring)."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    pats = grid_couplers(rows, cols)
    params = {}
    for p in pats.values():
        for cp in p:
            params[cp] = (math.pi / 2 + rng.uniform(-0.11, 0.11),
                          math.pi / 6 + rng.uniform(-0.05, 0.05))
    gates = []
    prev = [None] * n
    names = ["sx", "sy", "sw"]

    def single_layer():
        for q in range(n):
            choices = [k for k in names if k != prev[q]]
            k = choices[rng.integers(len(choices))]
            prev[q] = k
            gates.append(Gate(1, q, -1, SQRT_GATES[k].copy(), kind=k))

    first = []
    for t in range(cycles):
        single_layer()
        first.append(len(gates))
        for (a, b) in pats[sequence[t % len(sequence)]]:
            th, ph = params[(a, b)]
            gates.append(Gate(2, a, b, fsim(th, ph), kind="fsim", theta=th, phi=ph))
    single_layer()
    return Circuit(n, gates, rows, cols, cycles, seed, first)


def sycamore_couplers(rows: int = 9, cols: int = 6, removed=((8, 5),)):
    """Couplers of a Sycamore-like staggered diagonal lattice: sites (r, c),
    minus `removed`; site (r, c) couples down-right to (r+1, c + (r % 2)) and
    down-left to (r+1, c - 1 + (r % 2)).  Pattern A = down-right from even
    rows, B = down-right from odd rows, C = down-left from even rows,
    D = down-left from odd rows (each pattern is a matching).  Returns
    (number of qubits, qubit index of each site, {pattern: [(a, b), ...]})."""
    sites = [(r, c) for r in range(rows) for c in range(cols) if (r, c) not in set(removed)]
    index = {rc: i for i, rc in enumerate(sites)}
    pats = {"A": [], "B": [], "C": [], "D": []}
    for (r, c) in sites:
        for kind, dc in (("R", r % 2), ("L", -1 + r % 2)):
            nb = (r + 1, c + dc)
            if nb in index:
                key = {("R", 0): "A", ("R", 1): "B", ("L", 0): "C", ("L", 1): "D"}[(kind, r % 2)]
                pats[key].append((index[(r, c)], index[nb]))
    return len(sites), index, pats


def make_sycamore_circuit(cycles: int, seed: int, sequence: str = PATTERN_ABCD) -> Circuit:
    """Seeded 53-qubit Sycamore-topology circuit: the grid circuit's gate
    distribution on the staggered lattice of `sycamore_couplers`."""
    rng = np.random.default_rng(seed)
    n, _, pats = sycamore_couplers()
    params = {}
    for p in pats.values():
        for cp in p:
            params[cp] = (math.pi / 2 + rng.uniform(-0.11, 0.11), math.pi / 6 + rng.uniform(-0.05, 0.05))
    gates, prev, names, first = [], [None] * n, ["sx", "sy", "sw"], []

    def single_layer():
        for q in range(n):
            choices = [k for k in names if k != prev[q]]
            k = choices[rng.integers(len(choices))]
            prev[q] = k
            gates.append(Gate(1, q, -1, SQRT_GATES[k].copy(), kind=k))

    for t in range(cycles):
        single_layer()
        first.append(len(gates))
        for (a, b) in pats[sequence[t % len(sequence)]]:
            th, ph = params[(a, b)]
            gates.append(Gate(2, a, b, fsim(th, ph), kind="fsim", theta=th, phi=ph))
    single_layer()
    return Circuit(n, gates, 9, 6, cycles, seed, first)


def make_random_2q_circuit(n: int, depth: int, seed: int) -> Circuit:
    """Circuit of random (Haar-ish) 1q and generic 2q unitaries on random qubit
    pairs, both orientations; exercises conventions the symmetric fSim cannot."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(depth):
        for q in range(n):
            Z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
            Q, _ = np.linalg.qr(Z)
            gates.append(Gate(1, q, -1, Q, kind="u1"))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            a, b = int(perm[i]), int(perm[i + 1])
            Z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
            Q, _ = np.linalg.qr(Z)
            gates.append(Gate(2, a, b, Q, kind="u2"))
    return Circuit(n, gates, 0, 0, depth, seed, [])


def draw_tails(n_qubits: int, open_qubits, L: int, seed: int, distinct: bool = True) -> np.ndarray:
    """L uniformly random tail bitstrings (uint64, open-qubit bits zero), drawn by
    coin flips and, when `distinct`, without repetition (duplicates redrawn)."""
    rng = np.random.default_rng(seed)
    open_mask = 0
    for q in open_qubits:
        open_mask |= 1 << int(q)
    full = (1 << n_qubits) - 1
    tail_mask = full & ~open_mask
    n_tail = n_qubits - len(open_qubits)
    if distinct and L > (1 << n_tail):
        raise ValueError("more distinct tails requested than tail patterns exist")
    out, seen = [], set()
    while len(out) < L:
        bits = rng.integers(0, 2, size=n_qubits)
        v = 0
        for q in range(n_qubits):
            if bits[q]:
                v |= 1 << q
        v &= tail_mask
        if distinct and v in seen:
            continue
        seen.add(v)
        out.append(v)
    return np.array(out, dtype=np.uint64)


def mid_circuit_cut_edges(circ: Circuit, n_gates: int, kind: int = EDGE_SLICE, cycle: int | None = None,
                          value: int = 0):
    """Input edges of `n_gates` fSim gates of one middle cycle, spread over the
    layer (two edges per gate, leg 0 = input of q0, leg 1 = input of q1).
    Returns a list of (gate_index, leg, kind, value)."""
    if cycle is None:
        cycle = circ.cycles // 2
    start = circ.cycle_first_gate[cycle]
    end = circ.cycle_first_gate[cycle + 1] if cycle + 1 < len(circ.cycle_first_gate) else len(circ.gates)
    layer = [i for i in range(start, end) if circ.gates[i].arity == 2]
    if len(layer) < n_gates:
        raise ValueError("not enough two-qubit gates in the chosen cycle")
    pick = np.linspace(0, len(layer) - 1, n_gates).round().astype(int)
    edges = []
    for j in pick:
        gi = layer[int(j)]
        edges.append((gi, 0, kind, value))
        edges.append((gi, 1, kind, value))
    return edges


def synthetic_head(L: int, h: int, seed: int) -> np.ndarray:
    """Seeded complex128 head tensor [L][2^h] with Porter-Thomas-like magnitudes
    (complex Gaussian entries), for sampler tests that need no contraction."""
    rng = np.random.default_rng(seed)
    H = (rng.normal(size=(L, 1 << h)) + 1j * rng.normal(size=(L, 1 << h))) / math.sqrt(2.0)
    return H.astype(np.complex128)


# ---- the five workloads (shapes of the paper's experiments, synthetic data) ----

def config_tiny():
    """12-qubit 3x4 grid, 8 cycles, all qubits open, one group, no slicing."""
    circ = make_grid_circuit(3, 4, 8, seed=1)
    open_q = list(range(12))
    tails = np.zeros(1, dtype=np.uint64)
    return dict(circuit=circ, open_qubits=open_q, tails=tails, edges=[], n_samples=10_000,
                sample_seed=2, name="grid3x4_m8_open12")


def config_sliced30():
    """30-qubit 5x6 grid, 14 cycles; 10 open qubits (the last two rows) x 64
    distinct tails; 6 sliced edges = inputs of 3 mid-circuit fSim gates."""
    circ = make_grid_circuit(5, 6, 14, seed=3)
    open_q = list(range(20, 30))
    tails = draw_tails(30, open_q, 64, seed=33)
    edges = mid_circuit_cut_edges(circ, 3, EDGE_SLICE)
    return dict(circuit=circ, open_qubits=open_q, tails=tails, edges=edges, n_samples=64,
                sample_seed=4, name="grid5x6_m14_open10_L64_k6")


def config_precision40(cycles: int = 16):
    """40-qubit 5x8 grid (seed 4), `cycles` cycles (16 for the full workload);
    12 open qubits (q28..q39) and one tail (seed 44): 2^12 head amplitudes;
    10 sliced edges = inputs of 5 fSim gates of the middle cycle (2^10 slices),
    of which the kept prefix [0, 128) is summed (kept fraction 1/8).  The
    2^10-amplitude subset has q28 = 1, q29 = 0 (`subset_bitstrings`)."""
    circ = make_grid_circuit(5, 8, cycles, seed=4)
    open_q = list(range(28, 40))
    tails = draw_tails(40, open_q, 1, seed=44)
    edges = mid_circuit_cut_edges(circ, 5, EDGE_SLICE)
    return dict(circuit=circ, open_qubits=open_q, tails=tails, edges=edges, kept=128, n_samples=4096,
                sample_seed=8, name=f"grid5x8_m{cycles}_open12_L1_k10_kept128")


def subset_bitstrings(cfg) -> np.ndarray:
    """The 2^10 bitstrings of the precision workload's error subset: the tail,
    q28 = 1, q29 = 0, and q30..q39 = mu (bit j of mu on q30+j), mu = 0..1023."""
    base = int(cfg["tails"][0]) | (1 << 28)
    return np.array([base | (mu << 30) for mu in range(1 << 10)], dtype=np.uint64)


def config_grid25():
    """25-qubit 5x5 grid, 10 cycles, all qubits open, one group, no slicing: a
    small case with the same step kernels (operands above L2, ~2 GB on device)."""
    circ = make_grid_circuit(5, 5, 10, seed=21)
    return dict(circuit=circ, open_qubits=list(range(25)), tails=np.zeros(1, dtype=np.uint64), edges=[],
                n_samples=1000, sample_seed=6, name="grid5x5_m10_open25")


def serving_mix(seed=5, n_circuits=6):
    """Seeded mix of 20-25 qubit grid circuits (8-12 cycles, 6-8 open qubits,
    32-256 tails, 0-2 cut gates) for the serving workload."""
    rng = np.random.default_rng(seed)
    shapes = [(4, 5), (4, 6), (5, 5), (4, 5), (5, 5), (4, 6)]
    out = []
    for i in range(n_circuits):
        r, c = shapes[i % len(shapes)]
        m = int(rng.integers(8, 13))
        h = int(rng.integers(6, 9))
        L = int(2 ** rng.integers(5, 9))
        cut = int(rng.integers(0, 3))
        cfg = config_small(r, c, m, seed=100 + i, n_open=h, L=L, n_cut_gates=cut, tail_seed=200 + i)
        cfg["name"] = f"grid{r}x{c}_m{m}_h{h}_L{L}_k{2 * cut}"
        out.append(cfg)
    return out


def batch_mix(n_circuits=256, seed=7, n_open=6, L=16):
    """Seeded batch of grid circuits of 16-28 qubits and 8-16 cycles (seeds
    100, 101, ...), each with `n_open` open qubits and `L` tails, no cut
    edges: the many-small-circuits batched workload."""
    rng = np.random.default_rng(seed)
    shapes = [(4, 4), (3, 6), (4, 5), (3, 7), (4, 6), (5, 5), (4, 7)]
    out = []
    for i in range(n_circuits):
        r, c = shapes[int(rng.integers(len(shapes)))]
        m = int(rng.integers(8, 17))
        cfg = config_small(r, c, m, seed=100 + i, n_open=n_open, L=L, n_cut_gates=0, tail_seed=1000 + i)
        cfg["name"] = f"grid{r}x{c}_m{m}"
        out.append(cfg)
    return out


def poisson_requests(n_requests, rate_per_s, n_circuits, seed=9):
    """Seeded request stream: arrival times (Poisson), circuit ids, kinds
    (70 % amplitude batches, 30 % sampling) and log-uniform sizes."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n_requests))
    circ = rng.integers(0, n_circuits, n_requests)
    kind = (rng.random(n_requests) < 0.3).astype(int)
    size = np.where(kind == 0, 10 ** rng.uniform(3, 5, n_requests), 10 ** rng.uniform(2, 4, n_requests)).astype(int)
    seeds = rng.integers(0, 1 << 40, n_requests)
    return [dict(t=float(t[i]), circuit=int(circ[i]), kind=int(kind[i]), n=int(size[i]), seed=int(seeds[i]))
            for i in range(n_requests)]


def config_small(rows=4, cols=4, cycles=8, seed=11, n_open=6, L=8, n_cut_gates=2, tail_seed=12):
    """Scaled-down sliced sparse-state case used by parity tests."""
    circ = make_grid_circuit(rows, cols, cycles, seed=seed)
    n = rows * cols
    open_q = list(range(n - n_open, n))
    tails = draw_tails(n, open_q, L, seed=tail_seed)
    edges = mid_circuit_cut_edges(circ, n_cut_gates, EDGE_SLICE) if n_cut_gates else []
    return dict(circuit=circ, open_qubits=open_q, tails=tails, edges=edges, n_samples=L,
                sample_seed=5, name=f"grid{rows}x{cols}_m{cycles}")
