"""tn_head_norm_noalloc: the FP64 head norm for callers that cannot allocate
device memory (code inside a framework that owns all device memory, loops
where cudaMalloc is not allowed).  Its scratch is a fixed array inside the
library; the result must match tn_head_norm, call after call."""
import numpy as np
import pytest

import circuit_inputs as ci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def _head(tn, L, h, seed, n_qubits=30):
    import torch
    oq = list(range(n_qubits - h, n_qubits))
    tails = ci.draw_tails(n_qubits, oq, L, seed=seed)
    c = ci.make_grid_circuit(2, 2, 1, seed=1)
    c.n_qubits = n_qubits
    plan = tn.tn_plan(c, oq, tails)
    buf = torch.zeros((L, 1 << h), dtype=torch.complex128, device="cuda")
    head = tn.tn_head_create(plan, buf)
    buf.copy_(torch.from_numpy(ci.synthetic_head(L, h, seed)))
    torch.cuda.synchronize()
    return plan, head, buf


def test_noalloc_norm_matches_head_norm_twice(tn):
    import torch
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    # two calls in a row on different heads: the shared scratch keeps the first
    # call's partial sums, which the second call must not pick up
    for (L, h, seed) in [(1000, 10, 3), (64, 6, 4)]:
        plan, head, buf = _head(tn, L, h, seed)
        ref = tn.tn_head_norm(head)
        tn.tn_head_norm_noalloc(buf, L, h, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_noalloc_norm_rejects_too_many_groups(tn):
    import torch
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    buf = torch.zeros((4,), dtype=torch.complex128, device="cuda")
    with pytest.raises(tn.TNError) as e:
        tn.tn_head_norm_noalloc(buf, 131072 + 1, 0, out)
    assert e.value.code == tn.TN_ERR_INVALID
