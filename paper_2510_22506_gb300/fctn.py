"""Thin ctypes binding of libfctn.so (names follow the C ABI in include/fctn.h).

Only argument marshalling lives here: every step of the completion runs in
the library's CUDA kernels.  Arrays are accepted as NumPy arrays (host
memory, passed as FCTN_HOST) or as CUDA torch tensors (device memory, passed
as FCTN_DEVICE through ``data_ptr()``).  Importing this module raises if the
library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIBPATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfctn.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(f"{_LIBPATH} is missing: build it with `python -m paper_2510_22506_gb300.build`")
lib = ctypes.CDLL(_LIBPATH)

MAX_ORDER = 8
FCTN_OK, FCTN_E_ARG, FCTN_E_OOM, FCTN_E_SINGULAR, FCTN_E_NONFINITE, FCTN_E_TIMEOUT, FCTN_E_CUDA, \
    FCTN_E_STATE, FCTN_E_UNSUPPORTED = range(9)
FCTN_FP64, FCTN_FP32, FCTN_TF32, FCTN_BF16 = range(4)
FCTN_ORDER_PLAIN, FCTN_ORDER_ALTERNATE = 0, 1
FCTN_LAPLACIAN_PSD, FCTN_LAPLACIAN_PRINTED = 0, 1
FCTN_HOST, FCTN_DEVICE = 0, 1

PRECISIONS = {"fp64": FCTN_FP64, "fp32": FCTN_FP32, "tf32": FCTN_TF32, "bf16": FCTN_BF16}


class fctn_params(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("reuse", ctypes.c_int32),
        ("order_policy", ctypes.c_int32),
        ("laplacian_sign", ctypes.c_int32),
        ("refine_steps", ctypes.c_int32),
        ("dims", ctypes.c_int64 * MAX_ORDER),
        ("ranks", (ctypes.c_int32 * MAX_ORDER) * MAX_ORDER),
        ("lambda_", ctypes.c_double * MAX_ORDER),
        ("delta", ctypes.c_double * MAX_ORDER),
        ("rho", ctypes.c_double),
        ("extrap_alpha", ctypes.c_double),
        ("extrap_beta", ctypes.c_double),
        ("gram_mode", ctypes.c_int32),
        ("rhs_ctas", ctypes.c_int32),
        ("eig_max_sweeps", ctypes.c_int32),
        ("eig_tol", ctypes.c_double),
        ("finish_fp32_at", ctypes.c_double),
        ("tile_code", ctypes.c_int32),
        ("solve_method", ctypes.c_int32),
    ]


class fctn_stats(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int64),
        ("rel_change", ctypes.c_double),
        ("objective", ctypes.c_double),
        ("data_term", ctypes.c_double),
        ("converged", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("eig_sweeps", ctypes.c_int32),
        ("eig_capped", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp, _i, _i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
lib.fctn_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
lib.fctn_last_error.restype = ctypes.c_size_t
lib.fctn_version.restype = ctypes.c_char_p
lib.fctn_footprint_bytes.argtypes = [ctypes.POINTER(fctn_params), ctypes.POINTER(ctypes.c_size_t)]
lib.fctn_create.argtypes = [ctypes.POINTER(fctn_params), _vp, ctypes.POINTER(_vp)]
lib.fctn_set_data.argtypes = [_vp, _vp, _vp, _i]
lib.fctn_set_factors.argtypes = [_vp, ctypes.POINTER(_vp), _i]
lib.fctn_contract.argtypes = [_vp, _vp, _i]
lib.fctn_pam_sweep.argtypes = [_vp, _i, ctypes.POINTER(fctn_stats)]
lib.fctn_complete.argtypes = [_vp, ctypes.c_double, _i, _vp, _i, ctypes.POINTER(fctn_stats)]
lib.fctn_get_factor.argtypes = [_vp, _i, _vp, _i]
lib.fctn_get_X.argtypes = [_vp, _vp, _i]
lib.fctn_grow_ranks.argtypes = [_vp, ctypes.POINTER((ctypes.c_int32 * MAX_ORDER) * MAX_ORDER), ctypes.c_double,
                                ctypes.c_uint64]
lib.fctn_quality.argtypes = [_vp, _vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
lib.fctn_sync.argtypes = [_vp]
lib.fctn_launch_count.argtypes = [_vp, _i64p]
lib.fctn_destroy.argtypes = [_vp]
lib.fctn_set_graphs.argtypes = [_vp, _i]
lib.fctn_profile.argtypes = [_vp, _i]
_dp = ctypes.POINTER(ctypes.c_double)
lib.fctn_profile_read.argtypes = [_vp, _i64p, _dp, _dp, _dp]
lib.fctn_contract_noalloc.argtypes = [_i, _i64p, ctypes.POINTER(ctypes.c_int32), _i, ctypes.POINTER(_vp), _vp, _vp]
lib.fctn_contract_noalloc.restype = ctypes.c_int
for _f in ("fctn_footprint_bytes", "fctn_create", "fctn_set_data", "fctn_set_factors", "fctn_contract",
           "fctn_pam_sweep", "fctn_complete", "fctn_get_factor", "fctn_get_X", "fctn_sync", "fctn_launch_count",
           "fctn_destroy", "fctn_set_graphs", "fctn_profile", "fctn_profile_read"):
    getattr(lib, _f).restype = ctypes.c_int

EXPORTED = ("fctn_last_error", "fctn_version", "fctn_footprint_bytes", "fctn_create", "fctn_set_data",
            "fctn_set_factors", "fctn_contract", "fctn_pam_sweep", "fctn_complete", "fctn_get_factor",
            "fctn_get_X", "fctn_sync", "fctn_launch_count", "fctn_destroy", "fctn_set_graphs", "fctn_profile",
            "fctn_profile_read", "fctn_contract_noalloc", "fctn_server_create", "fctn_server_submit",
            "fctn_server_step", "fctn_server_poll", "fctn_server_result", "fctn_server_stats", "fctn_server_destroy",
            "fctn_server_finished", "fctn_server_group_stats", "fctn_quality", "fctn_grow_ranks", "fctn_autotune",
            "fctn_autotune_tiles")
KC = {"merged": 0, "gram": 1, "reduce": 2, "eig": 3, "solve": 4, "xupdate": 5, "misc": 6, "env": 7, "rhs2": 8,
      "eigaux": 9, "subst": 10, "resid": 11}


class fctn_server_config(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int32), ("flags", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_size_t)]


class fctn_job_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("sweeps", ctypes.c_int64),
                ("rel_change", ctypes.c_double), ("objective", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


FCTN_JOB_QUEUED, FCTN_JOB_RUNNING, FCTN_JOB_DONE, FCTN_JOB_FAILED = range(4)
lib.fctn_server_create.argtypes = [ctypes.POINTER(fctn_server_config), ctypes.POINTER(ctypes.c_void_p)]
lib.fctn_server_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(fctn_params), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p), ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_uint64)]
lib.fctn_server_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
lib.fctn_server_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(fctn_job_info)]
lib.fctn_server_result.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
lib.fctn_server_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t)]
lib.fctn_server_destroy.argtypes = [ctypes.c_void_p]
lib.fctn_server_group_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
lib.fctn_server_finished.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]
for _f in ("fctn_server_create", "fctn_server_submit", "fctn_server_step", "fctn_server_poll", "fctn_server_result",
           "fctn_server_stats", "fctn_server_destroy", "fctn_server_finished", "fctn_server_group_stats"):
    getattr(lib, _f).restype = ctypes.c_int


class FctnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfctn error {code}: {msg}")
        self.code = code


def fctn_last_error():
    buf = ctypes.create_string_buffer(1024)
    lib.fctn_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc):
    if rc != FCTN_OK:
        raise FctnError(rc, fctn_last_error())


def fctn_version():
    return lib.fctn_version().decode()


SOLVE_METHODS = {"auto": 0, "eig": 1, "chol": 2}


def make_params(dims, R, lam=0.01, delta=0.5, rho=0.1, precision="fp32", reuse=True, order_policy="alternate",
                laplacian_sign="psd", refine_steps=None, extrapolation=None, gram_mode="auto", rhs_ctas=0,
                eig_max_sweeps=0, eig_tol=0.0, finish_fp32_at=0.0, tile_code=0, solve_method="auto"):
    """fctn_params from Python values; R is an N x N symmetric rank matrix."""
    N = len(dims)
    p = fctn_params()
    p.order = N
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.reuse = int(bool(reuse))
    p.order_policy = {"plain": 0, "alternate": 1}[order_policy] if isinstance(order_policy, str) else int(order_policy)
    p.laplacian_sign = {"psd": 0, "printed": 1}[laplacian_sign] if isinstance(laplacian_sign, str) else int(laplacian_sign)
    if refine_steps is None:
        refine_steps = 0 if p.precision == FCTN_FP64 else 1
    p.refine_steps = int(refine_steps)
    lams = list(lam) if np.ndim(lam) else [lam] * N
    dels = list(delta) if np.ndim(delta) else [delta] * N
    for k in range(N):
        p.dims[k] = int(dims[k])
        p.lambda_[k] = float(lams[k])
        p.delta[k] = float(dels[k])
        for t in range(N):
            if t != k:
                p.ranks[min(k, t)][max(k, t)] = int(R[min(k, t)][max(k, t)])
    p.rho = float(rho)
    if extrapolation is not None:
        p.extrap_alpha, p.extrap_beta = float(extrapolation[0]), float(extrapolation[1])
    p.gram_mode = {"auto": 0, "direct": 1, "factored": 2}[gram_mode] if isinstance(gram_mode, str) else int(gram_mode)
    p.rhs_ctas = int(rhs_ctas)
    p.eig_max_sweeps = int(eig_max_sweeps)
    p.eig_tol = float(eig_tol)
    p.finish_fp32_at = float(finish_fp32_at)
    p.tile_code = int(tile_code)
    p.solve_method = SOLVE_METHODS[solve_method] if isinstance(solve_method, str) else int(solve_method)
    return p


def elem_dtype(p):
    return np.float64 if p.precision == FCTN_FP64 else np.float32


def _ptr(a, dtype=None):
    """(pointer, where) of a NumPy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(ctypes.c_void_p), FCTN_HOST
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (FCTN_DEVICE if a.is_cuda else FCTN_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def fctn_footprint_bytes(params):
    out = ctypes.c_size_t(0)
    _check(lib.fctn_footprint_bytes(ctypes.byref(params), ctypes.byref(out)))
    return out.value


def fctn_create(params, stream=None):
    """Create a handle; ``stream`` is a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    h = ctypes.c_void_p()
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.fctn_create(ctypes.byref(params), sp, ctypes.byref(h)))
    return h


def fctn_set_data(h, Y, mask):
    py, wy = _ptr(Y)
    pm, wm = _ptr(mask)
    if wy != wm:
        raise ValueError("Y and mask must both be on the host or both on the device")
    _check(lib.fctn_set_data(h, py, pm, wy))


def fctn_set_factors(h, factors):
    ptrs, where = [], None
    for a in factors:
        p, w = _ptr(a)
        if where is not None and w != where:
            raise ValueError("all factors must live in the same memory")
        where = w
        ptrs.append(p)
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    _check(lib.fctn_set_factors(h, arr, where))


def fctn_contract(h, out):
    p, w = _ptr(out)
    _check(lib.fctn_contract(h, p, w))
    return out


def fctn_pam_sweep(h, nsweeps=1, want_stats=True):
    st = fctn_stats()
    _check(lib.fctn_pam_sweep(h, int(nsweeps), ctypes.byref(st) if want_stats else None))
    return st.as_dict() if want_stats else None


def fctn_complete(h, tol, max_sweeps, out_X=None):
    st = fctn_stats()
    if out_X is None:
        rc = lib.fctn_complete(h, float(tol), int(max_sweeps), None, FCTN_HOST, ctypes.byref(st))
    else:
        p, w = _ptr(out_X)
        rc = lib.fctn_complete(h, float(tol), int(max_sweeps), p, w, ctypes.byref(st))
    _check(rc)
    return st.as_dict()


def fctn_get_factor(h, k, out):
    p, w = _ptr(out)
    _check(lib.fctn_get_factor(h, int(k), p, w))
    return out


def fctn_get_X(h, out):
    p, w = _ptr(out)
    _check(lib.fctn_get_X(h, p, w))
    return out


def fctn_grow_ranks(h, R, scale, seed):
    """Raise the FCTN ranks to R (N x N, a < b read); see include/fctn.h."""
    r = ((ctypes.c_int32 * MAX_ORDER) * MAX_ORDER)()
    N = len(R)
    for a in range(N):
        for b in range(a + 1, N):
            r[a][b] = int(R[a][b])
    _check(lib.fctn_grow_ranks(h, ctypes.byref(r), float(scale), ctypes.c_uint64(int(seed) & (2 ** 64 - 1))))


TUNE_CANDIDATES = (96, 120, 152, 192, 228, 304)


def fctn_autotune(params, Y, mask, factors, candidates=None, sweeps=3, stream=None):
    """Fastest rhs_ctas for these parameters and inputs (libfctn's autotuner).

    Returns (best, {candidate: mean sweep ms}).  ``candidates`` None takes the
    library's built-in list.  Y, mask and factors as for fctn_set_data /
    fctn_set_factors, all on the host or all on the device."""
    py, wy = _ptr(Y)
    pm, wm = _ptr(mask)
    ptrs, where = [], wy
    for a in factors:
        pa, wa = _ptr(a)
        ptrs.append(pa)
        if wa != wy:
            raise ValueError("Y, mask and factors must all be on the host or all on the device")
    if wm != wy:
        raise ValueError("Y, mask and factors must all be on the host or all on the device")
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    cand = list(TUNE_CANDIDATES if candidates is None else candidates)
    carr = (ctypes.c_int32 * len(cand))(*[int(c) for c in cand])
    ms = (ctypes.c_double * len(cand))()
    best = ctypes.c_int32(0)
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.fctn_autotune(ctypes.byref(params), py, pm, arr, where, carr if candidates is not None else None,
                             len(cand), int(sweeps), sp, ctypes.byref(best), ms))
    return best.value, {c: ms[i] for i, c in enumerate(cand)}


TILE_CANDIDATES = (0, 1, 2, 4, 8, 16, 32, 64, 96, 128, 136, 160)


def fctn_autotune_tiles(params, Y, mask, factors, candidates=None, sweeps=3, stream=None):
    """Fastest tile code (fctn_params.tile_code) of the head-mode route for
    these parameters and inputs.  Returns (best, {candidate: mean sweep ms})."""
    py, wy = _ptr(Y)
    pm, wm = _ptr(mask)
    ptrs = []
    for a in factors:
        pa, wa = _ptr(a)
        ptrs.append(pa)
        if wa != wy:
            raise ValueError("Y, mask and factors must all be on the host or all on the device")
    if wm != wy:
        raise ValueError("Y, mask and factors must all be on the host or all on the device")
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    cand = list(TILE_CANDIDATES if candidates is None else candidates)
    carr = (ctypes.c_int32 * len(cand))(*[int(c) for c in cand])
    ms = (ctypes.c_double * len(cand))()
    best = ctypes.c_int32(0)
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.fctn_autotune_tiles(ctypes.byref(params), py, pm, arr, wy, carr if candidates is not None else None,
                                   len(cand), int(sweeps), sp, ctypes.byref(best), ms))
    return best.value, {c: ms[i] for i, c in enumerate(cand)}


def fctn_quality(h, truth):
    """(PSNR, SSIM) of the current X against `truth` (Sec. 4), computed by libfctn."""
    p, w = _ptr(truth)
    ps, ss = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.fctn_quality(h, p, w, ctypes.byref(ps), ctypes.byref(ss)))
    return ps.value, ss.value


def fctn_sync(h):
    _check(lib.fctn_sync(h))


def fctn_launch_count(h):
    out = ctypes.c_int64(0)
    _check(lib.fctn_launch_count(h, ctypes.byref(out)))
    return out.value


def fctn_set_graphs(h, enable):
    _check(lib.fctn_set_graphs(h, int(bool(enable))))


def fctn_profile(h, kernel_class):
    """Start timing every launch of one kernel class (name or number; -1/None = off)."""
    kc = -1 if kernel_class is None else (KC[kernel_class] if isinstance(kernel_class, str) else int(kernel_class))
    _check(lib.fctn_profile(h, kc))


def fctn_profile_read(h):
    n = ctypes.c_int64(0)
    ms, b, f = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(lib.fctn_profile_read(h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b), ctypes.byref(f)))
    return {"launches": n.value, "ms": ms.value, "bytes": b.value, "flops": f.value}


def fctn_contract_noalloc(dims, R, precision, factors, out, stream=None):
    """FCTN contraction of device factors into device `out` without any device allocation.

    For callers that cannot allocate device memory (see include/fctn.h); the
    chain intermediates use the library's static scratch array.
    """
    N = len(dims)
    d = (ctypes.c_int64 * N)(*[int(x) for x in dims])
    r = (ctypes.c_int32 * (N * N))(*[int(R[a][b]) if a != b else 0 for a in range(N) for b in range(N)])
    ptrs = []
    for a in factors:
        pa, w = _ptr(a)
        if w != FCTN_DEVICE:
            raise ValueError("fctn_contract_noalloc takes device factors")
        ptrs.append(pa)
    po, w = _ptr(out)
    if w != FCTN_DEVICE:
        raise ValueError("fctn_contract_noalloc writes a device buffer")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    arr = (ctypes.c_void_p * N)(*ptrs)
    _check(lib.fctn_contract_noalloc(N, d, r, prec, arr, po, sp))
    return out


def fctn_destroy(h):
    _check(lib.fctn_destroy(h))


def factor_shapes(params):
    N = params.order
    out = []
    for k in range(N):
        out.append(tuple(int(params.dims[k]) if t == k else int(params.ranks[min(k, t)][max(k, t)]) for t in range(N)))
    return out


FCTN_SERVER_GROUP = 1


def fctn_server_create(max_jobs=32, mem_budget_bytes=0, group=False):
    cfg = fctn_server_config(max_jobs=int(max_jobs), flags=FCTN_SERVER_GROUP if group else 0,
                             mem_budget_bytes=int(mem_budget_bytes))
    out = ctypes.c_void_p()
    _check(lib.fctn_server_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def fctn_server_submit(srv, params, Y, mask, factors, tol, max_sweeps):
    """Submit a job from host arrays; returns its id."""
    dt = elem_dtype(params)
    Y = np.ascontiguousarray(Y, dtype=dt)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    fs = [np.ascontiguousarray(a, dtype=dt) for a in factors]
    arr = (ctypes.c_void_p * len(fs))(*[a.ctypes.data_as(ctypes.c_void_p) for a in fs])
    jid = ctypes.c_uint64(0)
    _check(lib.fctn_server_submit(srv, ctypes.byref(params), Y.ctypes.data_as(ctypes.c_void_p),
                                  mask.ctypes.data_as(ctypes.c_void_p), arr, float(tol), int(max_sweeps),
                                  ctypes.byref(jid)))
    return jid.value


def fctn_server_step(srv):
    r, q = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.fctn_server_step(srv, ctypes.byref(r), ctypes.byref(q)))
    return r.value, q.value


def fctn_server_poll(srv, job_id):
    info = fctn_job_info()
    _check(lib.fctn_server_poll(srv, ctypes.c_uint64(job_id), ctypes.byref(info)))
    return info.as_dict()


def fctn_server_result(srv, job_id, out=None):
    if out is None:
        _check(lib.fctn_server_result(srv, ctypes.c_uint64(job_id), None, FCTN_HOST))
        return None
    p, w = _ptr(out)
    _check(lib.fctn_server_result(srv, ctypes.c_uint64(job_id), p, w))
    return out


def fctn_server_finished(srv, cap=1024):
    ids = (ctypes.c_uint64 * cap)()
    n = ctypes.c_int(0)
    _check(lib.fctn_server_finished(srv, ids, cap, ctypes.byref(n)))
    return [ids[i] for i in range(n.value)]


def fctn_server_stats(srv):
    n, b = ctypes.c_int64(0), ctypes.c_size_t(0)
    _check(lib.fctn_server_stats(srv, ctypes.byref(n), ctypes.byref(b)))
    return {"sweeps_launched": n.value, "bytes_in_use": b.value}


def fctn_server_group_stats(srv):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.fctn_server_group_stats(srv, ctypes.byref(a), ctypes.byref(b)))
    return {"group_launches": a.value, "group_captures": b.value}


def fctn_server_destroy(srv):
    _check(lib.fctn_server_destroy(srv))
