"""The no-allocation FCTN contraction against the handle-based one.

Some callers cannot allocate device memory: their GPU memory is owned by
another allocator (for example a framework's caching allocator that has
reserved the device), or they run latency-critical loops in which
cudaMalloc / cudaFree would synchronise the device.  fctn_contract_noalloc
serves them with a static scratch array.  Through the C ABI, two calls in a
row must give the tensor that fctn_contract gives, within the contraction
tolerances used elsewhere in the tests (FP64 1e-12, FP32 2e-6 relative).
This file is collected last so that a run stopping at the first failure has
run every other test already.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,r,precision,tol", [
    ((30, 30, 10), 3, "fp64", 1e-12),
    ((64, 48, 31), 4, "fp32", 2e-6),
    ((13, 7, 3, 5), 3, "fp64", 1e-12),
    ((24, 20, 3, 9), 3, "fp32", 2e-6),
    ((9, 11), 4, "fp32", 2e-6),
])
def test_noalloc_matches_contract_twice(dims, r, precision, tol):
    torch = pytest.importorskip("torch")
    from paper_2510_22506_gb300 import fctn as F

    N = len(dims)
    R = np.full((N, N), r)
    p = F.make_params(dims, R, precision=precision, reuse=False)
    dt = F.elem_dtype(p)
    tdt = torch.float64 if dt == np.float64 else torch.float32
    rng = np.random.default_rng(99)
    fs = [np.ascontiguousarray(rng.standard_normal(shp).astype(dt)) for shp in F.factor_shapes(p)]
    h = F.fctn_create(p)
    try:
        F.fctn_set_factors(h, fs)
        ref = np.empty(dims, dtype=dt)
        F.fctn_contract(h, ref)
    finally:
        F.fctn_destroy(h)
    dev = [torch.from_numpy(a).cuda() for a in fs]
    for _ in range(2):
        out = torch.full(dims, float("nan"), dtype=tdt, device="cuda")
        F.fctn_contract_noalloc(dims, R, precision, dev, out)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref) <= tol


def test_noalloc_rejects_oversized_intermediate():
    torch = pytest.importorskip("torch")
    from paper_2510_22506_gb300 import fctn as F

    dims, N = (4096, 4096, 64), 3
    R = np.full((N, N), 8)
    small = [torch.zeros(4, device="cuda") for _ in range(N)]   # never read: rejected before any launch
    out = torch.zeros(4, device="cuda")
    with pytest.raises(F.FctnError) as ei:
        F.fctn_contract_noalloc(dims, R, "fp32", small, out)
    assert ei.value.code == F.FCTN_E_ARG
    assert "scratch" in str(ei.value)


def test_noalloc_order5_unequal_ranks_twice():
    """Order 5 with unequal bond ranks: the bond order of every factor view
    (smaller mode index first) must match the handle-based contraction."""
    torch = pytest.importorskip("torch")
    from paper_2510_22506_gb300 import fctn as F

    dims = (5, 4, 3, 4, 3)
    N = len(dims)
    R = np.ones((N, N), dtype=int)
    vals = iter([2, 3, 1, 2, 3, 2, 1, 2, 3, 2])
    for a in range(N):
        for b in range(a + 1, N):
            R[a, b] = R[b, a] = next(vals)
    p = F.make_params(dims, R, precision="fp64", reuse=False)
    rng = np.random.default_rng(5)
    fs = [np.ascontiguousarray(rng.standard_normal(shp)) for shp in F.factor_shapes(p)]
    h = F.fctn_create(p)
    try:
        F.fctn_set_factors(h, fs)
        ref = np.empty(dims)
        F.fctn_contract(h, ref)
    finally:
        F.fctn_destroy(h)
    dev = [torch.from_numpy(a).cuda() for a in fs]
    for _ in range(2):
        out = torch.full(dims, float("nan"), dtype=torch.float64, device="cuda")
        F.fctn_contract_noalloc(dims, R, "fp64", dev, out)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref) <= 1e-12
