"""Replays a plan's contraction list on the CPU (numpy, complex128).

Used by the planner tests: it checks the host planner's network, pins, slice
variants, sparse-state patterns, order and final mapping against the oracle
without a GPU.  It re-derives the pattern lists from the tails on its own.
"""
import string

import numpy as np

LETTERS = string.ascii_letters


def _pats(tails_masked, tq):
    return sorted(set(int(t) & tq for t in tails_masked))


def emulate(desc, tails, open_qubits, slices, on_tensor=None):
    """Sum over `slices` of the replayed plan; `on_tensor(array)` (optional)
    sees every leaf variant and every intermediate."""
    n = desc["n_qubits"]
    tail_mask = desc["tail_mask"]
    tm = [int(t) & tail_mask for t in tails]
    L = len(tails)
    h = len(open_qubits)
    H = np.zeros((L, 1 << h), dtype=np.complex128)
    leaves = desc["leaves"]
    vts = desc["vts"]
    # contraction list in order: (vt_a, vt_b, vt_c)
    seen, contr = set(), []
    for st in desc["steps"]:
        if st["contraction"] not in seen:
            seen.add(st["contraction"])
            contr.append((st["vt_a"], st["vt_b"], st["vt_c"]))
    for s in slices:
        T = {}
        for i, lf in enumerate(leaves):
            v = 0
            for t, b in enumerate(lf["var_slice_bits"]):
                v |= ((s >> b) & 1) << t
            size = lf["size"]
            re = np.array(lf["re"][v * size:(v + 1) * size])
            im = np.array(lf["im"][v * size:(v + 1) * size])
            T[i] = (re + 1j * im).reshape(lf["P"], -1)
            if on_tensor:
                on_tensor(T[i])
        for (a, b, c) in contr:
            A, B = T[a], T[b]
            la, lb, lc = vts[a]["legs"], vts[b]["legs"], vts[c]["legs"]
            tqa, tqb, tqc = vts[a]["tq"], vts[b]["tq"], vts[c]["tq"]
            pa, pb, pc = _pats(tm, tqa), _pats(tm, tqb), _pats(tm, tqc)
            assert len(pc) == vts[c]["P"]
            mA = [pa.index(x & tqa) for x in pc]
            mB = [pb.index(x & tqb) for x in pc]
            letter = {}
            for l in la + lb:
                if l not in letter:
                    letter[l] = LETTERS[len(letter)]
            # bit i <-> legs[i]; reshape [P] + [2]*r puts bit r-1 first
            At = A[mA].reshape([len(pc)] + [2] * len(la))
            Bt = B[mB].reshape([len(pc)] + [2] * len(lb))
            sa = "Z" + "".join(letter[l] for l in reversed(la))
            sb = "Z" + "".join(letter[l] for l in reversed(lb))
            sc = "Z" + "".join(letter[l] for l in reversed(lc))
            assert "Z" not in "".join(letter.values())
            Ct = np.einsum(f"{sa},{sb}->{sc}", At, Bt)
            T[c] = Ct.reshape(len(pc), -1)
            if on_tensor:
                on_tensor(T[c])
        F = T[desc["final"]["vt"]]
        fp = _pats(tm, tail_mask)
        op = desc["final"]["open_pos"]
        for g in range(L):
            row = F[fp.index(tm[g])]
            for mu in range(1 << h):
                off = 0
                for j in range(h):
                    if (mu >> j) & 1:
                        off |= 1 << op[j]
                H[g, mu] += row[off]
    return H
