"""Writes sycamore53_m8_o2.npz: amplitudes of the O2 network oracle for the
53-qubit Sycamore-topology circuit at 8 cycles (seed 5), open qubits 47..52,
8 seeded tails (seed 55), groups 0 and 5.  Calls only the oracle and the
seeded input generators (about five minutes on 16 cores):

    python tests/golden/make_sycamore53_golden.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
import circuit_inputs as ci  # noqa: E402
import oracle as O  # noqa: E402

CYCLES, SEED, TAIL_SEED, N_TAILS, GROUPS = 8, 5, 55, 8, [0, 5]


def main():
    circ = ci.make_sycamore_circuit(CYCLES, seed=SEED)
    n = circ.n_qubits
    oq = list(range(n - 6, n))
    tails = ci.draw_tails(n, oq, N_TAILS, seed=TAIL_SEED)
    H = O.network_amplitudes(circ, oq, tails, [], groups=GROUPS)
    out = os.path.join(os.path.dirname(__file__), "sycamore53_m8_o2.npz")
    np.savez(out, H=H, groups=np.array(GROUPS), tails=np.asarray(tails, dtype=np.uint64),
             open_qubits=np.array(oq), cycles=CYCLES, seed=SEED)
    print(out, H.shape, float(np.linalg.norm(H)))


if __name__ == "__main__":
    main()
