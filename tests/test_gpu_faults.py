"""Failure handling on the GPU without a GPU fault: host-side injection
(TN_FAULT_INJECT) of a failed allocation, a failure at a given slice and a
device status word set as a bounded wait that gave up would set it; the
bookkeeping of slice ranges around those failures; the bounded graph cache."""
import math

import numpy as np
import pytest

import circuit_inputs as ci
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def _cfg():
    return ci.config_small(4, 4, 8, seed=11, n_open=6, L=8, n_cut_gates=2)    # 16 slices


def _head(tn, cfg, head):
    tails, oq = cfg["tails"], cfg["open_qubits"]
    bits = np.array([O.bitstring_index(int(t), oq, mu) for t in tails for mu in range(1 << len(oq))], np.uint64)
    return tn.tn_amplitudes(head, bits).reshape(len(tails), -1)


def _oracle(cfg, r=None):
    se = [(g, l) for (g, l, k, v) in cfg["edges"]]
    return O.sparse_state_from_vector(O.sliced_statevector(cfg["circuit"], se, slice_range=r), cfg["open_qubits"],
                                      cfg["tails"])


def _close(H, ref):
    assert np.linalg.norm(H - ref) <= 1e-5 * np.linalg.norm(ref)


def test_injected_allocation_failure_on_device(tn, monkeypatch):
    cfg = _cfg()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
    monkeypatch.setenv("TN_FAULT_INJECT", "alloc")
    for make in (lambda: tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1),
                 lambda: tn.tn_head_create(plan)):
        with pytest.raises(tn.TNError) as e:
            make()
        assert e.value.code == tn.TN_ERR_OOM
    monkeypatch.delenv("TN_FAULT_INJECT")
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 16, head)
    _close(_head(tn, cfg, head), _oracle(cfg))


def test_failure_at_slice_keeps_completed_slices(tn, monkeypatch):
    """A failure before slice 5 of [0, 16): slices 0-4 stay recorded, a retry
    of [5, 16) is accepted, a retry of [0, 16) is not, and the sum is exact."""
    cfg = _cfg()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=4, host_fold_log2=-1)
    head = tn.tn_head_create(plan)
    monkeypatch.setenv("TN_FAULT_INJECT", "slice:5")
    with pytest.raises(tn.TNError) as e:
        tn.tn_contract_slices(plan, 0, 16, head)
    assert e.value.code == tn.TN_ERR_CUDA and "[0, 5)" in str(e.value)
    monkeypatch.delenv("TN_FAULT_INJECT")
    assert tn.tn_head_fidelity(head) == (5 / 16, 5)
    _close(_head(tn, cfg, head), _oracle(cfg, (0, 5)))
    with pytest.raises(tn.TNError):
        tn.tn_contract_slices(plan, 0, 16, head)
    tn.tn_contract_slices(plan, 5, 16, head)
    assert tn.tn_head_fidelity(head) == (1.0, 16)
    _close(_head(tn, cfg, head), _oracle(cfg))


def test_failure_inside_a_slice_invalidates_the_head(tn, monkeypatch):
    """With automatic slicing a user slice runs several passes; a failure
    after the first pass leaves the slice partly in H, so the head refuses
    every call until it is reset."""
    cfg = ci.config_small(4, 5, 10, seed=13, n_open=8, L=24, n_cut_gates=1)
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], max_log2_elements=15, host_fold_log2=-1,
                      auto_slice=16)
    assert tn.tn_plan_get_stats(plan)["n_internal_sliced"] >= 1
    head = tn.tn_head_create(plan)
    monkeypatch.setenv("TN_FAULT_INJECT", "slice:2:1")
    with pytest.raises(tn.TNError) as e:
        tn.tn_contract_slices(plan, 0, 4, head)
    assert "invalid" in str(e.value)
    monkeypatch.delenv("TN_FAULT_INJECT")
    for call in (lambda: tn.tn_contract_slices(plan, 2, 4, head), lambda: _head(tn, cfg, head),
                 lambda: tn.tn_head_norm(head), lambda: tn.tn_sample(head, 4, 0.0, 1)):
        with pytest.raises(tn.TNError) as e:
            call()
        assert e.value.code == tn.TN_ERR_INVALID
    tn.tn_head_reset(head)
    tn.tn_contract_slices(plan, 0, 4, head)
    _close(_head(tn, cfg, head), _oracle(cfg))


def test_device_status_word_reports_timeout(tn, monkeypatch):
    """A set device status word (here set from the host, as a bounded mbarrier
    wait that gave up sets it) surfaces as TN_ERR_TIMEOUT at the next
    synchronising call; the head is then invalid until reset, and the word is
    cleared."""
    cfg = _cfg()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], gemm=4, host_fold_log2=-1)
    for read in (lambda h: _head(tn, cfg, h), lambda h: tn.tn_head_norm(h), lambda h: tn.tn_sample(h, 4, 0.0, 1)):
        head = tn.tn_head_create(plan)
        monkeypatch.setenv("TN_FAULT_INJECT", "status")
        tn.tn_contract_slices(plan, 0, 16, head)
        monkeypatch.delenv("TN_FAULT_INJECT")
        with pytest.raises(tn.TNError) as e:
            read(head)
        assert e.value.code == tn.TN_ERR_TIMEOUT
        with pytest.raises(tn.TNError) as e:
            read(head)
        assert e.value.code == tn.TN_ERR_INVALID
        tn.tn_head_reset(head)
        tn.tn_contract_slices(plan, 0, 16, head)
        _close(_head(tn, cfg, head), _oracle(cfg))


def test_empty_batch_item_keeps_the_range_record(tn):
    """An empty range in a batch records nothing: [0, 4) stays accumulated and
    contracting it again is still rejected."""
    cfg = _cfg()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
    head = tn.tn_head_create(plan)
    tn.tn_contract_slices(plan, 0, 4, head)
    tn.tn_contract_batch([plan], [(0, 0)], [head])
    tn.tn_contract_batch([plan], [(4, 4)], [head])
    assert tn.tn_head_fidelity(head) == (4 / 16, 4)
    with pytest.raises(tn.TNError):
        tn.tn_contract_slices(plan, 0, 4, head)
    tn.tn_contract_slices(plan, 4, 16, head)
    _close(_head(tn, cfg, head), _oracle(cfg))


def test_graph_cache_is_bounded_and_replays_correctly(tn):
    """More distinct captured ranges than the per-plan cache holds: the oldest
    graphs are dropped and every replay still adds exactly its slices."""
    cfg = _cfg()
    plan = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_fold_log2=-1)
    heads = [tn.tn_head_create(plan) for _ in range(2)]
    for rep in range(2):
        for h in heads:
            tn.tn_head_reset(h)
            for s in range(16):                 # 16 ranges per head: 32 distinct (range, head) graphs
                tn.tn_contract_slices_graph(plan, s, s + 1, h)
        for h in heads:
            assert tn.tn_head_fidelity(h) == (1.0, 16)
            _close(_head(tn, cfg, h), _oracle(cfg))
    assert math.isfinite(tn.tn_head_norm(heads[0]))
