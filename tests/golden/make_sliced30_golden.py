"""Writes sliced30_o1.npz: the exact sparse state of the 30-qubit, 14-cycle
5x6 grid workload (seed 3; open qubits 20..29; 64 coin-flip tails, seed 33;
6 sliced edges on the inputs of 3 fSim gates of cycle 7) from the O1 state
vector, together with two kept prefixes of its slices.

By the slice-sum identity (Supplement, slicing: sum_v |v><v| = I on every cut
edge) the sum of all 64 slices is the uncut circuit, so one uncut O1 run gives
all 65,536 amplitudes.  A kept prefix [0, 2^(6-j)) fixes the top j slice bits
to 0, i.e. it is one O1 run with those j edges pinned to 0.  For each prefix
the file also holds F_true = |<psi|psi_hat>|^2 / (<psi|psi> <psi_hat|psi_hat>)
over the full 2^30 state (the fidelity of the Supplement's validation section)
and <psi_hat|psi_hat>.

Calls only the oracle (O1, in place through oracle/sv.c: two 16 GiB states)
and the seeded input generators; about an hour on 8 cores:

    python tests/golden/make_sliced30_golden.py
"""
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
import circuit_inputs as ci  # noqa: E402
import oracle as O  # noqa: E402
from oracle.statevector_c import overlap, statevector_inplace  # noqa: E402

PREFIXES = (32, 16)     # kept slices [0, kept) of 64


def main():
    cfg = ci.config_sliced30()
    circ, oq, tails, edges = cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"]
    k = len(edges)
    t0 = time.time()
    psi = statevector_inplace(circ)
    _, nn = overlap(psi, psi)
    H_full = O.sparse_state_from_vector(psi, oq, tails)
    print(f"full state: norm^2 {nn:.15f} ({time.time() - t0:.0f} s)", flush=True)
    out = dict(H_full=H_full, norm2_full=nn, tails=np.asarray(tails, dtype=np.uint64), open_qubits=np.array(oq),
               edges=np.array([(g, l) for (g, l, _, _) in edges]), prefixes=np.array(PREFIXES))
    hat = np.empty_like(psi)
    for kept in PREFIXES:
        j = k - (kept.bit_length() - 1)                       # top j slice bits pinned to 0
        pins = [(g, l, 0) for (g, l, _, _) in edges[k - j:]]
        statevector_inplace(circ, cuts=pins, out=hat)
        ov, hh = overlap(psi, hat)
        F = abs(ov) ** 2 / (nn * hh)
        out[f"H_{kept}"] = O.sparse_state_from_vector(hat, oq, tails)
        out[f"F_true_{kept}"] = F
        out[f"norm2_{kept}"] = hh
        print(f"kept {kept}/64: F_true {F:.6f}, norm^2 {hh:.6f} ({time.time() - t0:.0f} s)", flush=True)
    path = os.path.join(os.path.dirname(__file__), "sliced30_o1.npz")
    np.savez(path, **out)
    print(path)


if __name__ == "__main__":
    main()
