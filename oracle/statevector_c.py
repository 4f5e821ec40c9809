"""O1 for large states: the gate loop of ``statevector`` over in-place C kernels.

Test infrastructure (see the package docstring); never imported by the library.

``statevector`` (NumPy) makes a new array per gate, so a 30-qubit state
(16 GiB) would need two to three times that.  This module runs the same
definitions in place through ``sv.c`` (plain C, OpenMP over independent
amplitude groups): the same conventions, gates in time order, cut edges as
|v><v| projectors before the gate, companion (post) cuts after it.  It is
checked against ``statevector`` and the brute-force Kronecker route on small
circuits.  The shared object is compiled on first use with gcc into
``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv.c")
_LIB = os.path.join(_HERE, "_build", "libsv.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile sv.c (gcc -O2 -fopenmp) unless the shared object is up to date."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp, vp = C.POINTER(C.c_double), C.c_void_p
        lib.sv_apply_1q.argtypes = [vp, C.c_int, C.c_int, dp, dp]
        lib.sv_apply_2q.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, dp]
        lib.sv_project.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        lib.sv_overlap.argtypes = [vp, vp, C.c_int, dp, dp, dp]
        for f in (lib.sv_apply_1q, lib.sv_apply_2q, lib.sv_project, lib.sv_overlap):
            f.restype = None
        _lib = lib
    return _lib


def _mat(U):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    re = np.ascontiguousarray(U.real.ravel())
    im = np.ascontiguousarray(U.imag.ravel())
    return re, im


def statevector_inplace(circ, cuts=(), post_cuts=(), out=None) -> np.ndarray:
    """Same result as ``statevector.statevector(circ, cuts, post_cuts)``.

    cuts: (gate_index, leg, value), the wire entering the gate fixed to value;
    post_cuts: (gate_index, leg, value), the wire leaving the gate on that
    leg's qubit.  `out` (complex128, 2^n) is reused if given."""
    lib = _get()
    n = circ.n_qubits
    psi = out if out is not None else np.empty(1 << n, dtype=np.complex128)
    assert psi.dtype == np.complex128 and psi.size == (1 << n) and psi.flags.c_contiguous
    psi[:] = 0
    psi[0] = 1.0
    before, after = {}, {}
    for (g, leg, v) in cuts:
        before.setdefault(int(g), []).append((int(leg), int(v)))
    for (g, leg, v) in post_cuts:
        after.setdefault(int(g), []).append((int(leg), int(v)))
    ptr = psi.ctypes.data
    dp = C.POINTER(C.c_double)
    for gi, gate in enumerate(circ.gates):
        for (leg, v) in before.get(gi, ()):
            lib.sv_project(ptr, n, gate.q0 if leg == 0 else gate.q1, v)
        re, im = _mat(gate.U)
        if gate.arity == 1:
            lib.sv_apply_1q(ptr, n, gate.q0, re.ctypes.data_as(dp), im.ctypes.data_as(dp))
        else:
            lib.sv_apply_2q(ptr, n, gate.q0, gate.q1, re.ctypes.data_as(dp), im.ctypes.data_as(dp))
        for (leg, v) in after.get(gi, ()):
            lib.sv_project(ptr, n, gate.q0 if leg == 0 else gate.q1, v)
    return psi


def overlap(a: np.ndarray, b: np.ndarray):
    """(<a|b>, <b|b>) of two complex128 states of equal size."""
    lib = _get()
    n = int(a.size).bit_length() - 1
    assert a.size == b.size == (1 << n)
    r, i, bb = C.c_double(), C.c_double(), C.c_double()
    lib.sv_overlap(a.ctypes.data, b.ctypes.data, n, C.byref(r), C.byref(i), C.byref(bb))
    return complex(r.value, i.value), bb.value
