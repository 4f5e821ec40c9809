"""The complex GEMM step on its own (tn_gemm_c64), against NumPy complex128.

Each engine runs the production split permute, B preparation and GEMM kernels.
The shapes cover every GEMM path:
- the one-CTA 128-row tiles of every width;
- the CTA-pair 256 x 256 tiles (16-bit engines, M >= 256) with one B box per
  CTA, and the same shapes on one-CTA tiles (pair = -1);
- 2, 4, 8 and 16 patterns folded side by side, with a ragged last group;
- ragged K (one k-block and chunks of several);
- gather tables for both operands;
- K = 2, which the 16-bit engines run in tf32;
- a partial last wave of pair tiles (80 tiles on 76 clusters) and fewer
  tiles than clusters.

Tolerance: relative L2 <= 1e-5 (3xTF32, FP16x3, CUDA-core FP32) or 1e-4
(BF16x3), and every element within twice that of the largest.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ENGINES = {1: 1e-5, 2: 1e-5, 3: 1e-4, 4: 1e-5}

# (M, N, K, PA, PB, PC, mapA, mapB)
SHAPES = [
    (256, 128, 64, 1, 1, 1, None, None),        # one pair tile, 2N = 256
    (1024, 1024, 512, 1, 1, 1, None, None),     # pair tiles, 8 n-tiles
    (512, 64, 256, 1, 5, 5, None, None),        # 2N = 128: 2 patterns per tile, ragged last group
    (256, 32, 128, 1, 7, 7, None, None),        # 2N = 64: 4 patterns per tile
    (512, 16, 64, 1, 9, 9, None, None),         # 2N = 32: 8 patterns per tile
    (256, 8, 32, 1, 20, 20, None, None),        # 2N = 16: 16 patterns per tile
    (128, 256, 128, 1, 1, 1, None, None),       # M < 256: one-CTA 256-wide tile
    (2048, 4, 16, 1, 1, 1, None, None),         # narrow: 16-wide tile
    (64, 32, 2048, 1, 1, 1, None, None),        # long K, single m-tile
    (256, 64, 2, 1, 1, 1, None, None),          # K = 2 (tf32 kernel for the 16-bit engines)
    (128, 32, 64, 3, 4, 7, [0, 2, 1, 2, 0, 1, 2], [3, 0, 1, 2, 3, 3, 0]),   # gather tables
    (512, 128, 128, 2, 6, 6, [0, 1, 0, 1, 0, 1], None),   # A gathered: no fold
    (4096, 64, 1024, 1, 10, 10, None, None),    # 80 pair tiles on 76 clusters: a 4-tile last wave
    (2048, 128, 1024, 1, 1, 1, None, None),     # 8 pair tiles, fewer than the clusters
]


@pytest.fixture(scope="module")
def tn():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2111_03011_gb300 as m
    return m


def _rand(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2 * shape[-1])


@pytest.mark.parametrize("pair", [0, -1], ids=["pairs", "one-cta"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"M{s[0]}N{s[1]}K{s[2]}P{s[3]}x{s[4]}x{s[5]}" for s in SHAPES])
@pytest.mark.parametrize("engine", list(ENGINES), ids=["tf32x3", "simt", "bf16x3", "fp16x3"])
def test_complex_gemm_against_numpy(tn, engine, shape, pair):
    import torch
    M, N, K, PA, PB, PC, ma, mb = shape
    rng = np.random.default_rng(M * 7 + N * 3 + K + PA + 5 * PB + PC)
    A = _rand(rng, (PA, M, K))
    B = _rand(rng, (PB, K, N))
    ia = ma if ma is not None else ([0] * PC if PA == 1 else list(range(PC)))
    ib = mb if mb is not None else ([0] * PC if PB == 1 else list(range(PC)))
    ref = np.stack([A[ia[p]] @ B[ib[p]] for p in range(PC)])
    a = torch.from_numpy(A.astype(np.complex64)).cuda()
    b = torch.from_numpy(B.astype(np.complex64)).cuda()
    c = torch.full((PC, M, N), float("nan"), dtype=torch.complex64, device="cuda")
    tn.tn_gemm_c64(a, b, c, engine=engine, map_a=ma, map_b=mb, pair=pair)
    got = c.cpu().numpy().astype(np.complex128)
    tol = ENGINES[engine]
    assert np.isfinite(got).all()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol, err
    assert np.abs(got - ref).max() <= 2 * tol * np.abs(ref).max()


def test_complex_gemm_rejects_bad_arguments(tn):
    import torch
    a = torch.zeros((1, 96, 32), dtype=torch.complex64, device="cuda")
    b = torch.zeros((1, 32, 16), dtype=torch.complex64, device="cuda")
    c = torch.zeros((1, 96, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(tn.TNError):                  # M not a power of two
        tn.tn_gemm_c64(a, b, c)
    a = torch.zeros((2, 64, 32), dtype=torch.complex64, device="cuda")
    c = torch.zeros((3, 64, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(tn.TNError):                  # PA differs from PC and no map
        tn.tn_gemm_c64(a, b, c)
    with pytest.raises(tn.TNError):                  # map entry out of range
        tn.tn_gemm_c64(a, b, c, map_a=[0, 1, 2])
