"""Python binding of the sliced sparse-state contraction library (libtn_gb300.so).

Argument marshalling only: every step of the contraction, accumulation,
lookup and sampling runs in the library's CUDA kernels.  The functions carry
the names of the C ABI (include/tn_gb300.h) and raise TNError on a non-zero
return code.  The library is built in-tree for sm_103a by ``build.build()``;
importing this package builds it if stale and fails loudly if it cannot be
built or loaded.
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

from .buildlib import LIBPATH, build

TN_OK, TN_ERR_INVALID, TN_ERR_OOM, TN_ERR_NOT_IN_STATE, TN_ERR_TIMEOUT, TN_ERR_CUDA, TN_ERR_UNSUPPORTED = range(7)
TN_EDGE_SLICE, TN_EDGE_PIN, TN_EDGE_COMPANION = 0, 1, 2
TN_C64, TN_C128 = 0, 1
TN_SAMPLE_EXACT, TN_SAMPLE_METROPOLIS, TN_SAMPLE_FRUGAL = 0, 1, 2
TN_REQ_AMPLITUDES, TN_REQ_SAMPLE = 0, 1
TN_GEMM_AUTO, TN_GEMM_TC_3XTF32, TN_GEMM_SIMT_FP32, TN_GEMM_TC_BF16X3, TN_GEMM_TC_FP16X3 = 0, 1, 2, 3, 4


class TNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[tn error {code}] {msg}")
        self.code = code


class tn_gate(C.Structure):
    _fields_ = [("arity", C.c_int), ("q0", C.c_int), ("q1", C.c_int),
                ("re", C.c_double * 16), ("im", C.c_double * 16)]


class tn_circuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_gates", C.c_int), ("gates", C.POINTER(tn_gate))]


class tn_open_spec(C.Structure):
    _fields_ = [("open_qubits", C.POINTER(C.c_int)), ("n_open", C.c_int),
                ("tails", C.POINTER(C.c_uint64)), ("n_tails", C.c_int64)]


class tn_edge(C.Structure):
    _fields_ = [("gate", C.c_int), ("leg", C.c_int), ("kind", C.c_int), ("value", C.c_int)]


class tn_range(C.Structure):
    _fields_ = [("begin", C.c_int64), ("end", C.c_int64)]


class tn_plan_opts(C.Structure):
    _fields_ = [("max_log2_elements", C.c_double), ("gemm", C.c_int), ("host_only", C.c_int),
                ("order_trials", C.c_int), ("order_seed", C.c_uint64), ("max_host_absorb_log2", C.c_int),
                ("small_max_bits", C.c_int), ("auto_slice", C.c_int), ("host_fold_log2", C.c_int),
                ("gemm_pair", C.c_int), ("side_bprep", C.c_int), ("tune_steps", C.c_int)]


class tn_server_opts(C.Structure):
    _fields_ = [("n_slots", C.c_int), ("hbm_budget_bytes", C.c_int64)]


class tn_request(C.Structure):
    _fields_ = [("circuit", C.c_int), ("kind", C.c_int), ("bitstrings", C.c_void_p), ("n", C.c_int64),
                ("out", C.c_void_p), ("dtype", C.c_int), ("target_fidelity", C.c_double), ("seed", C.c_uint64),
                ("method", C.c_int), ("param", C.c_int64)]


class tn_request_result(C.Structure):
    _fields_ = [("status", C.c_int), ("latency_us", C.c_double), ("queue_us", C.c_double)]


class tn_server_stats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("in_flight", C.c_int64), ("queued", C.c_int64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("mean_us", C.c_double),
                ("heads_cached", C.c_int64), ("head_bytes", C.c_int64), ("evictions", C.c_int64),
                ("wall_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tn_plan_stats(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_open", C.c_int), ("n_tails", C.c_int64), ("n_patterns", C.c_int64),
                ("n_sliced", C.c_int), ("n_pinned", C.c_int), ("n_leaves", C.c_int), ("n_contractions", C.c_int),
                ("n_launches", C.c_int), ("tc_macs", C.c_double), ("alg_bytes", C.c_double),
                ("max_log2_elements", C.c_double), ("workspace_bytes", C.c_int64),
                ("n_gemm_tc", C.c_int), ("n_gemm_simt", C.c_int), ("n_small", C.c_int), ("n_permute", C.c_int),
                ("measured_slice_ms", C.c_double), ("autotune_candidates", C.c_int),
                ("n_internal_sliced", C.c_int), ("gemm_pair", C.c_int), ("n_side_bprep", C.c_int),
                ("n_tuned_steps", C.c_int), ("tune_default_ms", C.c_double), ("tune_tuned_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    try:
        build()          # no-op when the in-tree library is up to date
    except Exception as e:  # no compiler: only an existing library can be used
        if not os.path.exists(LIBPATH):
            raise ImportError(f"libtn_gb300.so is missing and could not be built: {e}") from e
    lib = C.CDLL(LIBPATH)
    vp, i64, i32p = C.c_void_p, C.c_int64, C.POINTER(C.c_int32)
    lib.tn_plan.argtypes = [C.POINTER(tn_circuit), C.POINTER(tn_open_spec), C.POINTER(tn_edge), C.c_int, i32p, i64,
                            C.POINTER(tn_plan_opts), C.POINTER(vp)]
    lib.tn_plan_autotune.argtypes = [C.POINTER(tn_circuit), C.POINTER(tn_open_spec), C.POINTER(tn_edge), C.c_int,
                                     C.POINTER(tn_plan_opts), C.c_int, vp, C.POINTER(vp)]
    lib.tn_plan_free.argtypes = [vp]
    lib.tn_plan_free.restype = None
    lib.tn_plan_get_stats.argtypes = [vp, C.POINTER(tn_plan_stats)]
    lib.tn_plan_order.argtypes = [vp, i32p, i64, C.POINTER(i64)]
    lib.tn_plan_describe.argtypes = [vp, C.c_int]
    lib.tn_plan_describe.restype = C.c_char_p
    lib.tn_head_create.argtypes = [vp, vp, C.POINTER(vp)]
    lib.tn_head_free.argtypes = [vp]
    lib.tn_head_free.restype = None
    lib.tn_head_data.argtypes = [vp]
    lib.tn_head_data.restype = vp
    lib.tn_head_reset.argtypes = [vp, vp]
    lib.tn_head_fidelity.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64)]
    lib.tn_head_set_fidelity.argtypes = [vp, C.c_double]
    lib.tn_contract_slices.argtypes = [vp, tn_range, vp, vp]
    lib.tn_amplitudes.argtypes = [vp, vp, i64, vp, C.c_int, vp]
    lib.tn_sample.argtypes = [vp, i64, C.c_double, C.c_uint64, vp, vp]
    lib.tn_head_norm.argtypes = [vp, C.POINTER(C.c_double), vp, vp]
    lib.tn_contract_slices_graph.argtypes = [vp, tn_range, vp, vp]
    lib.tn_contract_batch.argtypes = [C.POINTER(vp), C.POINTER(tn_range), C.POINTER(vp), C.c_int, vp]
    lib.tn_server_create.argtypes = [C.POINTER(tn_server_opts), C.POINTER(vp)]
    lib.tn_server_add_circuit.argtypes = [vp, vp, tn_range, C.POINTER(C.c_int)]
    lib.tn_server_submit.argtypes = [vp, C.POINTER(tn_request), C.POINTER(C.c_uint64)]
    lib.tn_server_wait.argtypes = [vp, C.c_uint64, C.POINTER(tn_request_result)]
    lib.tn_server_get_stats.argtypes = [vp, C.POINTER(tn_server_stats)]
    lib.tn_server_free.argtypes = [vp]
    lib.tn_server_free.restype = None
    lib.tn_sample_ex.argtypes = [vp, i64, C.c_double, C.c_uint64, C.c_int, i64, vp, vp]
    lib.tn_profile_slices.argtypes = [vp, tn_range, vp, vp, C.POINTER(C.c_double), i64]
    lib.tn_plan_step_info.argtypes = [vp, i64, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.tn_plan_step_variants.argtypes = [vp, i64, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.tn_plan_set_step_variant.argtypes = [vp, i64, C.c_int]
    lib.tn_plan_tune_steps.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.tn_head_norm_noalloc.argtypes = [vp, i64, C.c_int, vp, vp]
    lib.tn_xeb.argtypes = [vp, vp, i64, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.tn_gemm_c64.argtypes = [C.c_int, vp, vp, vp, i64, i64, i64, i64, i64, i64, i32p, i32p, C.c_int, vp]
    lib.tn_last_error.restype = C.c_char_p
    lib.tn_version.restype = C.c_char_p
    for name in ("tn_plan", "tn_plan_autotune", "tn_plan_get_stats", "tn_plan_order", "tn_head_create", "tn_head_fidelity",
                 "tn_head_set_fidelity", "tn_contract_slices", "tn_amplitudes", "tn_sample", "tn_head_norm",
                 "tn_profile_slices", "tn_plan_step_info", "tn_plan_step_variants", "tn_plan_set_step_variant",
                 "tn_plan_tune_steps", "tn_head_reset", "tn_head_norm_noalloc", "tn_sample_ex",
                 "tn_contract_slices_graph", "tn_contract_batch", "tn_server_create", "tn_server_add_circuit",
                 "tn_server_submit", "tn_server_wait", "tn_server_get_stats"):
        getattr(lib, name).restype = C.c_int
    return lib


_lib = _load()
lib = _lib

EXPORTED = ["tn_plan", "tn_plan_autotune", "tn_plan_free", "tn_plan_get_stats", "tn_plan_order", "tn_plan_describe",
            "tn_head_create", "tn_head_free", "tn_head_data", "tn_head_reset", "tn_head_fidelity", "tn_head_set_fidelity",
            "tn_contract_slices", "tn_contract_slices_graph", "tn_contract_batch", "tn_amplitudes", "tn_sample", "tn_sample_ex", "tn_head_norm", "tn_profile_slices",
            "tn_plan_step_info", "tn_plan_step_variants", "tn_plan_set_step_variant", "tn_plan_tune_steps",
            "tn_head_norm_noalloc", "tn_server_create", "tn_server_add_circuit",
            "tn_server_submit", "tn_server_wait", "tn_server_get_stats", "tn_server_free", "tn_last_error",
            "tn_gemm_c64", "tn_xeb", "tn_version"]


def _check(rc):
    if rc != TN_OK:
        raise TNError(rc, _lib.tn_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device)."""
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(int(x))


def gates_to_c(circuit):
    """tn_gate array from a circuit with .n_qubits and .gates (arity, q0, q1, U)."""
    arr = (tn_gate * max(1, len(circuit.gates)))()
    for i, g in enumerate(circuit.gates):
        arr[i].arity = int(g.arity)
        arr[i].q0 = int(g.q0)
        arr[i].q1 = int(g.q1) if g.arity == 2 else -1
        U = np.asarray(g.U, dtype=np.complex128).reshape(-1)
        for e in range(U.size):
            arr[i].re[e] = float(U[e].real)
            arr[i].im[e] = float(U[e].imag)
    return arr


class Plan:
    """Owns a tn_plan_t handle (and keeps its inputs alive)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_plan_free(self.handle)
            self.handle = None


class Head:
    def __init__(self, handle, plan, buf):
        self.handle = handle
        self.plan = plan
        self._buf = buf

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_head_free(self.handle)
            self.handle = None


def tn_plan(circuit, open_qubits, tails, edges=(), order=None, max_log2_elements=0.0, gemm=TN_GEMM_AUTO,
            host_only=False, order_trials=0, order_seed=0, max_host_absorb_log2=0, small_max_bits=0,
            auto_slice=0, host_fold_log2=0, gemm_pair=0, side_bprep=0) -> Plan:
    gates = gates_to_c(circuit)
    circ = tn_circuit(int(circuit.n_qubits), len(circuit.gates), gates)
    oq = (C.c_int * max(1, len(open_qubits)))(*[int(q) for q in open_qubits])
    t = np.ascontiguousarray(np.asarray(tails, dtype=np.uint64))
    spec = tn_open_spec(oq, len(open_qubits), t.ctypes.data_as(C.POINTER(C.c_uint64)), int(t.size))
    ed = (tn_edge * max(1, len(edges)))()
    for i, e in enumerate(edges):
        g, leg, kind, val = (list(e) + [TN_EDGE_SLICE, 0])[:4] if len(e) < 4 else e
        ed[i] = tn_edge(int(g), int(leg), int(kind), int(val))
    opts = tn_plan_opts(float(max_log2_elements), int(gemm), int(bool(host_only)), int(order_trials),
                        int(order_seed), int(max_host_absorb_log2), int(small_max_bits), int(auto_slice),
                        int(host_fold_log2), int(gemm_pair), int(side_bprep), 0)
    h = C.c_void_p()
    if order is not None:
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int32).reshape(-1))
        _check(_lib.tn_plan(C.byref(circ), C.byref(spec), ed, len(edges), o.ctypes.data_as(C.POINTER(C.c_int32)),
                            o.size // 2, C.byref(opts), C.byref(h)))
    else:
        _check(_lib.tn_plan(C.byref(circ), C.byref(spec), ed, len(edges), None, 0, C.byref(opts), C.byref(h)))
    return Plan(h, (gates, oq, t, ed))


def tn_plan_autotune(circuit, open_qubits, tails, edges=(), n_candidates=4, max_log2_elements=0.0,
                     gemm=TN_GEMM_AUTO, order_trials=0, order_seed=0, max_host_absorb_log2=0, small_max_bits=0,
                     stream=None, auto_slice=0, host_fold_log2=0, gemm_pair=0, side_bprep=0,
                     tune_steps=0) -> Plan:
    gates = gates_to_c(circuit)
    circ = tn_circuit(int(circuit.n_qubits), len(circuit.gates), gates)
    oq = (C.c_int * max(1, len(open_qubits)))(*[int(q) for q in open_qubits])
    t = np.ascontiguousarray(np.asarray(tails, dtype=np.uint64))
    spec = tn_open_spec(oq, len(open_qubits), t.ctypes.data_as(C.POINTER(C.c_uint64)), int(t.size))
    ed = (tn_edge * max(1, len(edges)))()
    for i, e in enumerate(edges):
        g, leg, kind, val = (list(e) + [TN_EDGE_SLICE, 0])[:4] if len(e) < 4 else e
        ed[i] = tn_edge(int(g), int(leg), int(kind), int(val))
    opts = tn_plan_opts(float(max_log2_elements), int(gemm), 0, int(order_trials), int(order_seed),
                        int(max_host_absorb_log2), int(small_max_bits), int(auto_slice), int(host_fold_log2),
                        int(gemm_pair), int(side_bprep), int(tune_steps))
    h = C.c_void_p()
    _check(_lib.tn_plan_autotune(C.byref(circ), C.byref(spec), ed, len(edges), C.byref(opts), int(n_candidates),
                                 _stream(stream), C.byref(h)))
    return Plan(h, (gates, oq, t, ed))


def tn_plan_get_stats(plan: Plan) -> dict:
    s = tn_plan_stats()
    _check(_lib.tn_plan_get_stats(plan.handle, C.byref(s)))
    return s.as_dict()


def tn_plan_step_variants(plan: Plan, i: int):
    """(number of tile variants of step i, the chosen one)."""
    n, c = C.c_int(), C.c_int()
    _check(_lib.tn_plan_step_variants(plan.handle, int(i), C.byref(n), C.byref(c)))
    return n.value, c.value


def tn_plan_set_step_variant(plan: Plan, i: int, variant: int) -> None:
    _check(_lib.tn_plan_set_step_variant(plan.handle, int(i), int(variant)))


def tn_plan_tune_steps(plan: Plan, reps=3, stream=None):
    """Tune every step's tile variant; returns (slice ms before, slice ms with the chosen variants)."""
    a, b = C.c_double(), C.c_double()
    _check(_lib.tn_plan_tune_steps(plan.handle, int(reps), _stream(stream), C.byref(a), C.byref(b)))
    return a.value, b.value


def tn_plan_order(plan: Plan) -> np.ndarray:
    n = C.c_int64()
    _check(_lib.tn_plan_order(plan.handle, None, 0, C.byref(n)))
    buf = np.zeros(2 * max(1, n.value), dtype=np.int32)
    _check(_lib.tn_plan_order(plan.handle, buf.ctypes.data_as(C.POINTER(C.c_int32)), n.value, C.byref(n)))
    return buf[: 2 * n.value].reshape(-1, 2)


def tn_plan_describe(plan: Plan, with_data=False) -> dict:
    return json.loads(_lib.tn_plan_describe(plan.handle, int(bool(with_data))).decode())


def tn_head_create(plan: Plan, buffer=None) -> Head:
    h = C.c_void_p()
    _check(_lib.tn_head_create(plan.handle, _ptr(buffer) if buffer is not None else None, C.byref(h)))
    return Head(h, plan, buffer)


def tn_head_free(head: Head):
    if head.handle:
        _lib.tn_head_free(head.handle)
        head.handle = None


def tn_head_data(head: Head) -> int:
    return _lib.tn_head_data(head.handle)


def tn_head_reset(head: Head, stream=None):
    _check(_lib.tn_head_reset(head.handle, _stream(stream)))


def tn_head_fidelity(head: Head):
    f = C.c_double()
    n = C.c_int64()
    _check(_lib.tn_head_fidelity(head.handle, C.byref(f), C.byref(n)))
    return f.value, n.value


def tn_head_set_fidelity(head: Head, f: float):
    _check(_lib.tn_head_set_fidelity(head.handle, float(f)))


def tn_contract_slices(plan: Plan, begin: int, end: int, head: Head, stream=None):
    _check(_lib.tn_contract_slices(plan.handle, tn_range(int(begin), int(end)), head.handle, _stream(stream)))


def tn_contract_slices_graph(plan: Plan, begin: int, end: int, head: Head, stream=None):
    _check(_lib.tn_contract_slices_graph(plan.handle, tn_range(int(begin), int(end)), head.handle,
                                         _stream(stream)))


def tn_contract_batch(plans, ranges, heads, stream=None):
    """plans, heads: lists of Plan / Head; ranges: list of (begin, end)."""
    n = len(plans)
    P = (C.c_void_p * max(1, n))(*[p.handle for p in plans])
    R = (tn_range * max(1, n))(*[tn_range(int(b), int(e)) for (b, e) in ranges])
    Hh = (C.c_void_p * max(1, n))(*[h.handle for h in heads])
    _check(_lib.tn_contract_batch(P, R, Hh, n, _stream(stream)))


def tn_amplitudes(head: Head, bitstrings, out=None, dtype=TN_C128, stream=None):
    """bitstrings: numpy uint64 (host) or torch uint64/int64 tensor (device).
    Returns `out` (allocated as numpy complex128/complex64 when None)."""
    n = int(bitstrings.numel() if hasattr(bitstrings, "numel") else np.asarray(bitstrings).size)
    if not hasattr(bitstrings, "data_ptr"):
        bitstrings = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64))
    if out is None:
        out = np.zeros(n, dtype=np.complex128 if dtype == TN_C128 else np.complex64)
    _check(_lib.tn_amplitudes(head.handle, _ptr(bitstrings), n, _ptr(out), int(dtype), _stream(stream)))
    return out


def tn_sample(head: Head, n: int, target_fidelity=0.0, seed=0, out=None, stream=None):
    if out is None:
        out = np.zeros(int(n), dtype=np.uint64)
    _check(_lib.tn_sample(head.handle, int(n), float(target_fidelity), int(seed), _ptr(out), _stream(stream)))
    return out


def tn_sample_ex(head: Head, n: int, target_fidelity=0.0, seed=0, method=TN_SAMPLE_EXACT, param=0, out=None,
                 stream=None):
    if out is None:
        out = np.zeros(int(n), dtype=np.uint64)
    _check(_lib.tn_sample_ex(head.handle, int(n), float(target_fidelity), int(seed), int(method), int(param),
                             _ptr(out), _stream(stream)))
    return out


def tn_xeb(ideal: Head, samples, stream=None):
    """(linear XEB, log XEB) of the samples against the exact head `ideal`."""
    if not hasattr(samples, "data_ptr"):
        samples = np.ascontiguousarray(np.asarray(samples, dtype=np.uint64))
    n = int(samples.numel() if hasattr(samples, "numel") else samples.size)
    lin, lg = C.c_double(), C.c_double()
    _check(_lib.tn_xeb(ideal.handle, _ptr(samples), n, C.byref(lin), C.byref(lg), _stream(stream)))
    return lin.value, lg.value


def tn_head_norm(head: Head, with_groups=False, stream=None):
    N = C.c_double()
    L = int(tn_plan_get_stats(head.plan)["n_tails"])
    Z = np.zeros(L, dtype=np.float64) if with_groups else None
    _check(_lib.tn_head_norm(head.handle, C.byref(N), _ptr(Z) if Z is not None else None, _stream(stream)))
    return (N.value, Z) if with_groups else N.value


def tn_profile_slices(plan: Plan, begin: int, end: int, head: Head, stream=None) -> np.ndarray:
    """Contract [begin, end) into head, returning summed ms per launch of one
    pass (summed over every pass: 2^n_internal_sliced per slice)."""
    st = tn_plan_get_stats(plan)
    n = int(st["n_launches"]) >> int(st["n_internal_sliced"])
    ms = np.zeros(n, dtype=np.float64)
    _check(_lib.tn_profile_slices(plan.handle, tn_range(int(begin), int(end)), head.handle, _stream(stream),
                                  ms.ctypes.data_as(C.POINTER(C.c_double)), n))
    return ms


def tn_plan_step_info(plan: Plan, i: int):
    """(kind, algorithmic complex MACs, algorithmic HBM bytes) of launch i."""
    k = C.c_int()
    m = C.c_double()
    b = C.c_double()
    _check(_lib.tn_plan_step_info(plan.handle, int(i), C.byref(k), C.byref(m), C.byref(b)))
    return k.value, m.value, b.value


def tn_gemm_c64(a, b, c, engine=TN_GEMM_AUTO, map_a=None, map_b=None, pair=0, stream=None):
    """c[p] = a[map_a(p)] @ b[map_b(p)] on the device (torch complex64 tensors of
    shapes [PA, M, K], [PB, K, N], [PC, M, N]); maps are sequences of PC ints
    or None."""
    PA, M, K = (int(x) for x in a.shape)
    PB, K2, N = (int(x) for x in b.shape)
    PC = int(c.shape[0])
    assert K2 == K and tuple(c.shape[1:]) == (M, N)
    i32p = C.POINTER(C.c_int32)
    ma = np.ascontiguousarray(np.asarray(map_a, dtype=np.int32)) if map_a is not None else None
    mb = np.ascontiguousarray(np.asarray(map_b, dtype=np.int32)) if map_b is not None else None
    _check(_lib.tn_gemm_c64(int(engine), _ptr(a), _ptr(b), _ptr(c), M, N, K, PA, PB, PC,
                            ma.ctypes.data_as(i32p) if ma is not None else None,
                            mb.ctypes.data_as(i32p) if mb is not None else None, int(pair), _stream(stream)))
    return c


def tn_head_norm_noalloc(head_buffer, n_groups: int, n_open: int, norm_out, stream=None):
    """FP64 squared norm of a device complex128 head buffer into the device
    double `norm_out`, with no device allocation (asynchronous on `stream`)."""
    _check(_lib.tn_head_norm_noalloc(_ptr(head_buffer), int(n_groups), int(n_open), _ptr(norm_out),
                                     _stream(stream)))


class Server:
    """Owns a tn_server_t; keeps registered plans and in-flight buffers alive."""

    def __init__(self, handle):
        self.handle = handle
        self.plans = []
        self.inflight = {}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_server_free(self.handle)
            self.handle = None


def tn_server_create(n_slots=0, hbm_budget_bytes=0) -> Server:
    h = C.c_void_p()
    _check(_lib.tn_server_create(C.byref(tn_server_opts(int(n_slots), int(hbm_budget_bytes))), C.byref(h)))
    return Server(h)


def tn_server_add_circuit(server: Server, plan: Plan, begin: int, end: int) -> int:
    cid = C.c_int()
    _check(_lib.tn_server_add_circuit(server.handle, plan.handle, tn_range(int(begin), int(end)), C.byref(cid)))
    server.plans.append(plan)
    return cid.value


def tn_server_submit(server: Server, circuit: int, kind: int, n: int, bitstrings=None, out=None, dtype=TN_C128,
                     target_fidelity=0.0, seed=0, method=TN_SAMPLE_EXACT, param=0) -> int:
    """Queue a request; returns its ticket.  `out` (allocated when None) and the
    bitstrings are kept alive until tn_server_wait."""
    if kind == TN_REQ_AMPLITUDES:
        bitstrings = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64))
        n = bitstrings.size
        if out is None:
            out = np.zeros(n, dtype=np.complex128 if dtype == TN_C128 else np.complex64)
    elif out is None:
        out = np.zeros(int(n), dtype=np.uint64)
    req = tn_request(int(circuit), int(kind), bitstrings.ctypes.data if bitstrings is not None else None, int(n),
                     out.ctypes.data, int(dtype), float(target_fidelity), int(seed), int(method), int(param))
    t = C.c_uint64()
    _check(_lib.tn_server_submit(server.handle, C.byref(req), C.byref(t)))
    server.inflight[t.value] = (bitstrings, out)
    return t.value


def tn_server_wait(server: Server, ticket: int):
    """Blocks for the request; returns (out, latency_us)."""
    res = tn_request_result()
    rc = _lib.tn_server_wait(server.handle, int(ticket), C.byref(res))
    bufs = server.inflight.pop(int(ticket), (None, None))
    _check(rc)
    return bufs[1], res.latency_us


def tn_server_get_stats(server: Server) -> dict:
    st = tn_server_stats()
    _check(_lib.tn_server_get_stats(server.handle, C.byref(st)))
    return st.as_dict()


def tn_server_free(server: Server):
    if server.handle:
        _lib.tn_server_free(server.handle)
        server.handle = None


def tn_last_error() -> str:
    return _lib.tn_last_error().decode(errors="replace")


def tn_version() -> str:
    return _lib.tn_version().decode()
