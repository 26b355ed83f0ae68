"""The C-ABI library loads and exports every entry point that include/fctn.h
declares; host-side validation and footprint arithmetic work without a GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fctn_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def F():
    from paper_2510_22506_gb300 import build
    build.build()
    from paper_2510_22506_gb300 import fctn
    return fctn


def test_every_declared_symbol_is_exported(F):
    decl = _declared()
    assert {"fctn_create", "fctn_contract", "fctn_pam_sweep", "fctn_complete"} <= decl
    for name in decl:
        assert hasattr(F.lib, name), name
    assert set(F.EXPORTED) >= decl - {"fctn_params"}


def test_version_and_error_buffer(F):
    assert "sm_103a" in F.fctn_version()
    assert isinstance(F.fctn_last_error(), str)


def _params(F, dims, r=3, **kw):
    N = len(dims)
    R = np.full((N, N), r)
    return F.make_params(dims, R, **kw)


def test_footprint_scales_with_size(F):
    a = F.fctn_footprint_bytes(_params(F, (30, 30, 10), precision="fp64"))
    b = F.fctn_footprint_bytes(_params(F, (256, 256, 31), r=8, precision="fp32"))
    assert 0 < a < b
    # X (4 B/elt) + merged tensor dominate the c2-sized handle
    assert b > 4 * 256 * 256 * 31


@pytest.mark.parametrize("bad", [
    dict(dims=(30, 0, 10)),            # empty mode
    dict(dims=(30,)),                  # order 1
    dict(rho=0.0),
    dict(precision=9),
    dict(order_policy=5),
    dict(refine_steps=99),
    dict(rhs_ctas=-1),
    dict(rhs_ctas=5000),
    dict(tile_code=-1),
    dict(tile_code=256),
    dict(eig_tol=1.5),
    dict(finish_fp32_at=-1.0),
    dict(solve_method=3),
])
def test_invalid_params_rejected(F, bad):
    dims = bad.pop("dims", (30, 30, 10))
    N = len(dims)
    R = np.full((max(N, 2), max(N, 2)), 3)
    p = F.make_params(dims, R, **bad) if N >= 1 else None
    if N == 1:
        p.order = 1
    with pytest.raises(F.FctnError) as ei:
        F.fctn_footprint_bytes(p)
    assert ei.value.code in (F.FCTN_E_ARG,)


def test_reuse_beyond_order_four_is_planned(F):
    """N >= 5 reuse keeps two half intermediates: more memory than no reuse."""
    on = F.fctn_footprint_bytes(_params(F, (6, 5, 4, 5, 4), r=2, reuse=True))
    off = F.fctn_footprint_bytes(_params(F, (6, 5, 4, 5, 4), r=2, reuse=False))
    assert on > 0 and off > 0


def test_rhs_ctas_sets_the_split(F):
    """A larger right-hand-side CTA budget splits M_k's columns more finely:
    more per-split partials, so a larger footprint; 0 is the built-in rule.
    (Merged tensors formed per factor: reuse off.)"""
    kw = dict(r=8, precision="fp32", reuse=False)
    small = F.fctn_footprint_bytes(_params(F, (256, 256, 31), rhs_ctas=16, **kw))
    rule = F.fctn_footprint_bytes(_params(F, (256, 256, 31), **kw))
    large = F.fctn_footprint_bytes(_params(F, (256, 256, 31), rhs_ctas=2432, **kw))
    assert small < large
    assert small <= rule <= large


@pytest.mark.parametrize("bad", [dict(sweeps=0), dict(sweeps=1001), dict(candidates=(-1,)), dict(candidates=(5000,)),
                                 dict(candidates=tuple(range(1, 66)))])
def test_autotune_rejects_bad_arguments_before_any_launch(F, bad):
    """fctn_autotune validates its arguments on the host (FCTN_E_ARG) before
    it creates a probe handle, so these calls need no GPU."""
    dims = (6, 5, 4)
    p = _params(F, dims, r=2, precision="fp32")
    Y = np.zeros(dims, dtype=np.float32)
    mask = np.ones(dims, dtype=np.uint8)
    facs = [np.zeros(F.factor_shapes(p)[k], dtype=np.float32) for k in range(3)]
    kw = dict(candidates=(96,), sweeps=1)
    kw.update(bad)
    with pytest.raises(F.FctnError) as ei:
        F.fctn_autotune(p, Y, mask, facs, **kw)
    assert ei.value.code == F.FCTN_E_ARG


def test_order8_planning_stays_in_bounds(F):
    """Order 8, every rank 1: chain intermediates carry up to 20 labels.  The
    footprint planner and the no-allocation contraction plan them without
    overrunning their label arrays and answer with status codes; the
    no-allocation call is rejected by its scratch limit before it touches
    the device (its pointers are never dereferenced)."""
    import ctypes
    dims = (16,) * 8
    N = 8
    R = np.ones((N, N), dtype=int)
    assert F.fctn_footprint_bytes(F.make_params(dims, R, precision="fp32")) > 4 * 16 ** 8
    d = (ctypes.c_int64 * N)(*dims)
    r = (ctypes.c_int32 * (N * N))(*([1] * (N * N)))
    fake = (ctypes.c_void_p * N)(*([ctypes.c_void_p(256)] * N))
    rc = F.lib.fctn_contract_noalloc(N, d, r, F.FCTN_FP32, fake, ctypes.c_void_p(256), None)
    assert rc == F.FCTN_E_ARG
    assert "scratch" in F.fctn_last_error()


@pytest.mark.parametrize("kw", [dict(precision="fp64", solve_method="chol"),
                                dict(precision="fp32", solve_method="chol", r=17)])
def test_cholesky_solve_limits(F, kw):
    """The Cholesky solve is FP32 with s_k <= 256: FP64, or s = 17^2 = 289,
    is a valid request that it does not serve (AUTO takes Eq. 8 there)."""
    r = kw.pop("r", 3)
    with pytest.raises(F.FctnError) as ei:
        F.fctn_footprint_bytes(_params(F, (40, 36, 30), r=r, **kw))
    assert ei.value.code == F.FCTN_E_UNSUPPORTED
    assert F.fctn_footprint_bytes(_params(F, (40, 36, 30), r=17, precision="fp32")) > 0
    assert F.fctn_footprint_bytes(_params(F, (40, 36, 30), r=16, precision="fp32", solve_method="chol")) > 0
