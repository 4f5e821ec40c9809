"""Writes precision40_m10_o2.npz: FP64 amplitudes of the 40-qubit 5x8 grid
precision workload at reduced depth (10 cycles; everything else as in
circuit_inputs.config_precision40: 12 open qubits, one tail, 10 sliced edges
on the inputs of 5 fSim gates of the middle cycle) on its 2^10-amplitude
subset (q28 = 1, q29 = 0, q30..q39 = mu), summed over the kept prefix
[0, 128) of the 2^10 slices.

The kept prefix fixes slice bits 7..9 to 0: those three edges are pinned to
|0><0| (edge breaking, Method) and the other seven are summed slice by slice
(Supplement, slicing), 128 O2 contractions of about 1.4e9 complex
multiply-adds each.  A 40-qubit state vector (2^40 amplitudes) does not fit
in host memory, so O2 is the oracle here.

Calls only the oracle (O2) and the seeded input generators; a few minutes on
8 cores:

    python tests/golden/make_precision40_golden.py
"""
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
import circuit_inputs as ci  # noqa: E402
import oracle as O  # noqa: E402

CYCLES = 10


def main():
    cfg = ci.config_precision40(CYCLES)
    circ, edges, kept = cfg["circuit"], cfg["edges"], cfg["kept"]
    k = len(edges)
    j = k - (kept.bit_length() - 1)                        # top j slice bits fixed to 0
    summed = [(g, l) for (g, l, _, _) in edges[:k - j]]
    pins = [(g, l, 0) for (g, l, _, _) in edges[k - j:]]
    sub_open = list(range(30, 40))
    sub_tail = np.array([int(cfg["tails"][0]) | (1 << 28)], dtype=np.uint64)
    t0 = time.time()
    st = {}
    H = O.network_amplitudes(circ, sub_open, sub_tail, sliced_edges=summed, pins=pins, slice_range=(0, kept),
                             stats=st)[0]
    print(f"{kept} slices, {st['complex_macs']:.3e} complex MACs, {time.time() - t0:.0f} s, "
          f"|H|^2 = {np.vdot(H, H).real:.6e}", flush=True)
    path = os.path.join(os.path.dirname(__file__), "precision40_m10_o2.npz")
    np.savez(path, H_subset=H, cycles=CYCLES, kept=kept, bitstrings=ci.subset_bitstrings(cfg),
             edges=np.array([(g, l) for (g, l, _, _) in edges]))
    print(path)


if __name__ == "__main__":
    main()
