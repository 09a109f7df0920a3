"""Thin ctypes binding of libgf.so (C ABI declared in include/gf.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Functions keep the C names; a field argument may be a torch
tensor (CUDA or CPU, complex128 of shape (Lt, Lz, Ly, Lx, 4, 3, 3) or float64
with a trailing 2), a numpy array, or a raw address (int).

The library is built in-tree (``paper_1209_4008_gb300/_build/libgf.so``) by
``paper_1209_4008_gb300.build``; if it is missing the binding raises -- there
is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

GF_OK, GF_EINVAL, GF_ECUDA, GF_ETIMEOUT, GF_ENOTCONVERGED, GF_ENOMEM, GF_EREJECT, GF_ESTATE = range(8)
GF_LANDAU, GF_COULOMB, GF_MAG = 0, 1, 2
GF_FP64, GF_MIXED, GF_FP32 = 0, 1, 2

_lock = threading.Lock()
_lib = None


class GFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_name(code)}: {msg}")
        self.code = code


def _name(code: int) -> str:
    names = ["GF_OK", "GF_EINVAL", "GF_ECUDA", "GF_ETIMEOUT", "GF_ENOTCONVERGED", "GF_ENOMEM",
             "GF_EREJECT", "GF_ESTATE"]
    return names[code] if 0 <= code < len(names) else f"code {code}"


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)

# name -> (restype, argtypes)
SIGNATURES = {
    "gf_create": (C.c_int, [_ip, C.c_int, C.POINTER(_vp)]),
    "gf_destroy": (C.c_int, [_vp]),
    "gf_last_error": (C.c_char_p, [_vp]),
    "gf_error_string": (C.c_char_p, [C.c_int]),
    "gf_set_stream": (C.c_int, [_vp, _vp]),
    "gf_set_option": (C.c_int, [_vp, C.c_char_p, C.c_double]),
    "gf_get_option": (C.c_int, [_vp, C.c_char_p, _dp]),
    "gf_get_stat": (C.c_int, [_vp, C.c_char_p, _dp]),
    "gf_overrelax": (C.c_int, [_vp, _vp, C.c_double, C.c_double, C.c_int, _ip, _dp, _dp]),
    "gf_anneal": (C.c_int, [_vp, _vp, C.c_double, C.c_double, C.c_int, C.c_uint64]),
    "gf_functional": (C.c_int, [_vp, _vp, _dp]),
    "gf_theta": (C.c_int, [_vp, _vp, _dp]),
    "gf_plaquette": (C.c_int, [_vp, _vp, _dp]),
    "gf_upload": (C.c_int, [_vp, _vp, C.c_int]),
    "gf_download": (C.c_int, [_vp, _vp]),
    "gf_or_half_sweep": (C.c_int, [_vp, C.c_int, C.c_double]),
    "gf_or_sweeps": (C.c_int, [_vp, C.c_double, C.c_int]),
    "gf_sa_half_sweep": (C.c_int, [_vp, C.c_int, C.c_double, C.c_uint64, C.c_uint32]),
    "gf_measure": (C.c_int, [_vp, _dp, _dp]),
    "gf_measure_timeslices": (C.c_int, [_vp, _dp, _dp]),
    "gf_wilson_update": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_uint32]),
    "gf_generate": (C.c_int, [_vp, _vp, C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32]),
    "gf_sr_half_sweep": (C.c_int, [_vp, C.c_int, C.c_double, C.c_uint64, C.c_uint32]),
    "gf_reunitarize": (C.c_int, [_vp]),
    "gf_autotune": (C.c_int, [_vp, _ip, _ip]),
    "gf_measure_noalloc": (C.c_int, [_ip, C.c_int, _vp, _vp, _vp]),
    "gf_fma_peak": (C.c_int, [C.c_int, C.c_int, _dp, _dp]),
    "gf_batch_create": (C.c_int, [C.c_int, _ip, C.c_int, C.POINTER(_vp)]),
    "gf_batch_destroy": (C.c_int, [_vp]),
    "gf_batch_last_error": (C.c_char_p, [_vp]),
    "gf_batch_set_stream": (C.c_int, [_vp, _vp]),
    "gf_batch_set_option": (C.c_int, [_vp, C.c_char_p, C.c_double]),
    "gf_batch_get_stat": (C.c_int, [_vp, C.c_char_p, _dp]),
    "gf_batch_overrelax": (C.c_int, [_vp, C.POINTER(_vp), C.c_double, C.c_double, C.c_int, _ip, _dp,
                                     _dp]),
    "gf_batch_autotune": (C.c_int, [_vp, C.POINTER(_vp), _ip, _ip]),
    "gf_overrelax_batched": (C.c_int, [C.c_int, _ip, C.POINTER(_vp), C.c_double, C.c_double, C.c_int, _ip, _dp,
                                       _dp]),
    "gf_net_param_count": (C.c_size_t, []),
    "gf_net_create": (C.c_int, [_ip, C.POINTER(_vp)]),
    "gf_net_destroy": (C.c_int, [_vp]),
    "gf_net_last_error": (C.c_char_p, [_vp]),
    "gf_net_set_stream": (C.c_int, [_vp, _vp]),
    "gf_net_set_params": (C.c_int, [_vp, _vp]),
    "gf_net_get_params": (C.c_int, [_vp, _vp]),
    "gf_net_forward": (C.c_int, [_vp, _vp, _vp]),
    "gf_net_gradient": (C.c_int, [_vp, _vp, _vp, _vp, _dp]),
    "gf_net_train_step": (C.c_int, [_vp, _vp, _vp, C.c_float, _dp]),
    "gf_net_set_option": (C.c_int, [_vp, C.c_char_p, C.c_double]),
    "gf_gauge_reset": (C.c_int, [_vp]),
    "gf_get_gauge": (C.c_int, [_vp, _vp]),
    "gf_converge": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int, _ip, _dp, _dp]),
    "gf_apply_tracked_gauge": (C.c_int, [_vp, _vp]),
    "gf_features": (C.c_int, [_vp, C.c_double, _vp]),
    "gf_gauge_algebra": (C.c_int, [_vp, C.c_double, _vp]),
    "gf_apply_algebra": (C.c_int, [_vp, _vp, C.c_double]),
    "gf_set_net": (C.c_int, [_vp, _vp]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libgf.so (building it first if asked and it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"libgf.so not built ({path}); run paper_1209_4008_gb300.build")
                _build.build()
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def _ptr(x) -> int:
    """Address of a field/buffer argument."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported field argument {type(x)}")


def _check_field(ctx: "Context", U) -> None:
    if hasattr(U, "shape") and not isinstance(U, int):
        n = 1
        for s in U.shape:
            n *= int(s)
        itemsize = U.element_size() if hasattr(U, "element_size") else U.itemsize
        if n * itemsize != ctx.volume * 4 * 9 * 16:
            raise ValueError(f"field has {n * itemsize} bytes, lattice needs {ctx.volume * 576}")


class Context:
    """Owns a gf_ctx handle; the C functions below take it as first argument."""

    def __init__(self, dims, gauge: int = GF_LANDAU):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.volume = 1
        for d in self.dims:
            self.volume *= d
        arr = (C.c_int * 4)(*self.dims)
        h = _vp()
        rc = self.lib.gf_create(arr, int(gauge), C.byref(h))
        if rc != GF_OK:
            raise GFError(rc, f"gf_create{self.dims} gauge={gauge}")
        self.handle = h
        self.gauge = gauge

    def check(self, rc: int, what: str, ok=(GF_OK,)) -> int:
        if rc not in ok:
            msg = self.lib.gf_last_error(self.handle)
            raise GFError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.gf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------
def gf_create(dims, gauge: int = GF_LANDAU) -> Context:
    return Context(dims, gauge)


def gf_destroy(ctx: Context) -> None:
    ctx.close()


def gf_set_stream(ctx: Context, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
    s = getattr(stream, "cuda_stream", stream)
    ctx.check(ctx.lib.gf_set_stream(ctx.handle, s or None), "gf_set_stream")


def gf_set_option(ctx: Context, key: str, value: float) -> None:
    ctx.check(ctx.lib.gf_set_option(ctx.handle, key.encode(), float(value)), f"option {key}")


def gf_get_option(ctx: Context, key: str) -> float:
    v = C.c_double()
    ctx.check(ctx.lib.gf_get_option(ctx.handle, key.encode(), C.byref(v)), f"option {key}")
    return v.value


def gf_get_stat(ctx: Context, key: str) -> float:
    v = C.c_double()
    ctx.check(ctx.lib.gf_get_stat(ctx.handle, key.encode(), C.byref(v)), f"stat {key}")
    return v.value


def gf_overrelax(ctx: Context, U, omega: float, theta_target: float, max_iter: int):
    """Returns (converged, sweeps, F, theta); U is fixed in place."""
    _check_field(ctx, U)
    it, F, th = C.c_int(), C.c_double(), C.c_double()
    rc = ctx.check(ctx.lib.gf_overrelax(ctx.handle, _ptr(U), omega, theta_target, int(max_iter),
                                        C.byref(it), C.byref(F), C.byref(th)),
                   "gf_overrelax", ok=(GF_OK, GF_ENOTCONVERGED))
    return rc == GF_OK, it.value, F.value, th.value


def gf_anneal(ctx: Context, U, T0: float, T1: float, steps: int, seed: int, allow_reject=False) -> int:
    _check_field(ctx, U)
    ok = (GF_OK, GF_EREJECT) if allow_reject else (GF_OK,)
    return ctx.check(ctx.lib.gf_anneal(ctx.handle, _ptr(U), T0, T1, int(steps), int(seed)),
                     "gf_anneal", ok=ok)


def gf_functional(ctx: Context, U) -> float:
    _check_field(ctx, U)
    v = C.c_double()
    ctx.check(ctx.lib.gf_functional(ctx.handle, _ptr(U), C.byref(v)), "gf_functional")
    return v.value


def gf_theta(ctx: Context, U) -> float:
    _check_field(ctx, U)
    v = C.c_double()
    ctx.check(ctx.lib.gf_theta(ctx.handle, _ptr(U), C.byref(v)), "gf_theta")
    return v.value


def gf_plaquette(ctx: Context, U) -> float:
    _check_field(ctx, U)
    v = C.c_double()
    ctx.check(ctx.lib.gf_plaquette(ctx.handle, _ptr(U), C.byref(v)), "gf_plaquette")
    return v.value


def gf_upload(ctx: Context, U, precision: int = GF_FP64) -> None:
    _check_field(ctx, U)
    ctx.check(ctx.lib.gf_upload(ctx.handle, _ptr(U), int(precision)), "gf_upload")


def gf_download(ctx: Context, U) -> None:
    _check_field(ctx, U)
    ctx.check(ctx.lib.gf_download(ctx.handle, _ptr(U)), "gf_download")


def gf_or_half_sweep(ctx: Context, parity: int, omega: float) -> None:
    ctx.check(ctx.lib.gf_or_half_sweep(ctx.handle, int(parity), omega), "gf_or_half_sweep")


def gf_or_sweeps(ctx: Context, omega: float, nsweeps: int) -> None:
    ctx.check(ctx.lib.gf_or_sweeps(ctx.handle, omega, int(nsweeps)), "gf_or_sweeps")


def gf_sa_half_sweep(ctx: Context, parity: int, T: float, seed: int, sweep: int) -> None:
    ctx.check(ctx.lib.gf_sa_half_sweep(ctx.handle, int(parity), T, int(seed), int(sweep)),
              "gf_sa_half_sweep")


def gf_sr_half_sweep(ctx: Context, parity: int, p: float, seed: int, sweep: int) -> None:
    ctx.check(ctx.lib.gf_sr_half_sweep(ctx.handle, int(parity), float(p), int(seed), int(sweep)),
              "gf_sr_half_sweep")


def gf_measure(ctx: Context):
    F, th = C.c_double(), C.c_double()
    ctx.check(ctx.lib.gf_measure(ctx.handle, C.byref(F), C.byref(th)), "gf_measure")
    return F.value, th.value


def gf_measure_timeslices(ctx: Context):
    """(F_t, theta_t) of every timeslice of the resident field (numpy arrays)."""
    import numpy as np
    Lt = int(ctx.dims[3])
    F = np.zeros(Lt)
    th = np.zeros(Lt)
    ctx.check(ctx.lib.gf_measure_timeslices(ctx.handle, F.ctypes.data_as(_dp), th.ctypes.data_as(_dp)),
              "gf_measure_timeslices")
    return F, th


def gf_wilson_update(ctx: Context, mu: int, parity: int, beta: float, mode: int, seed: int, sweep: int) -> None:
    ctx.check(ctx.lib.gf_wilson_update(ctx.handle, int(mu), int(parity), float(beta), int(mode), int(seed),
                                       int(sweep)), "gf_wilson_update")


def gf_generate(ctx: Context, U, beta: float, n_sweeps: int, n_or: int, seed: int, sweep0: int = 0,
                allow_reject=False) -> int:
    """Wilson-action heatbath + overrelaxation sweeps on U in place."""
    _check_field(ctx, U)
    ok = (GF_OK, GF_EREJECT) if allow_reject else (GF_OK,)
    return ctx.check(ctx.lib.gf_generate(ctx.handle, _ptr(U), float(beta), int(n_sweeps), int(n_or), int(seed),
                                         int(sweep0)), "gf_generate", ok=ok)


def gf_reunitarize(ctx: Context) -> None:
    ctx.check(ctx.lib.gf_reunitarize(ctx.handle), "gf_reunitarize")


def gf_autotune(ctx: Context):
    t, b = C.c_int(), C.c_int()
    ctx.check(ctx.lib.gf_autotune(ctx.handle, C.byref(t), C.byref(b)), "gf_autotune")
    return t.value, b.value


def gf_measure_noalloc(dims, gauge: int, U, out, stream=None) -> int:
    """F and theta of a device field into the device buffer out (2 doubles),
    without any allocation; returns the C return code.  Tensors are checked
    here first (the library sees only addresses): U must hold the lattice's
    float64 links and out at least two float64 values."""
    lib = load()
    dims = [int(d) for d in dims]
    if hasattr(U, "element_size") or hasattr(out, "element_size"):
        import torch
        vol = 1
        for d in dims:
            vol *= d
        for name, t, need in (("U", U, vol * 72), ("out", out, 2)):
            if not isinstance(t, torch.Tensor):
                continue
            if t.dtype not in (torch.float64, torch.complex128):
                raise ValueError(f"{name} must be float64 (or complex128), got {t.dtype}")
            n = t.numel() * (2 if t.dtype == torch.complex128 else 1)
            if (n != need) if name == "U" else (n < need):
                raise ValueError(f"{name} holds {n} float64 values, needs {'' if name == 'U' else 'at least '}{need}")
    arr = (C.c_int * 4)(*dims)
    s = getattr(stream, "cuda_stream", stream)
    return lib.gf_measure_noalloc(arr, int(gauge), _ptr(U), _ptr(out), s or None)


def gf_fma_peak(fp64: bool, iters: int):
    """Measured FMA rate of the current device: (TFLOP/s, ms per launch)."""
    lib = load()
    t, ms = C.c_double(), C.c_double()
    rc = lib.gf_fma_peak(1 if fp64 else 0, int(iters), C.byref(t), C.byref(ms))
    if rc != GF_OK:
        raise GFError(rc, "gf_fma_peak")
    return t.value, ms.value


class Batch:
    """Owns a gf_batch handle (n lattices gauge-fixed in one persistent launch)."""

    def __init__(self, dims_list, gauge: int = GF_LANDAU):
        self.lib = load()
        self.n = len(dims_list)
        flat = [int(d) for dims in dims_list for d in dims]
        arr = (C.c_int * len(flat))(*flat)
        h = _vp()
        rc = self.lib.gf_batch_create(self.n, arr, int(gauge), C.byref(h))
        if rc != GF_OK:
            raise GFError(rc, "gf_batch_create")
        self.handle = h

    def check(self, rc: int, what: str, ok=(GF_OK,)) -> int:
        if rc not in ok:
            msg = self.lib.gf_batch_last_error(self.handle)
            raise GFError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.gf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gf_batch_create(dims_list, gauge: int = GF_LANDAU) -> Batch:
    return Batch(dims_list, gauge)


def gf_batch_destroy(b: Batch) -> None:
    b.close()


def gf_batch_set_stream(b: Batch, stream) -> None:
    s = getattr(stream, "cuda_stream", stream)
    b.check(b.lib.gf_batch_set_stream(b.handle, s or None), "gf_batch_set_stream")


def gf_batch_set_option(b: Batch, key: str, value: float) -> None:
    b.check(b.lib.gf_batch_set_option(b.handle, key.encode(), float(value)), f"option {key}")


def gf_batch_get_stat(b: Batch, key: str) -> float:
    v = C.c_double()
    b.check(b.lib.gf_batch_get_stat(b.handle, key.encode(), C.byref(v)), f"stat {key}")
    return v.value


def _ptr_array(fields):
    return (_vp * len(fields))(*[_ptr(u) for u in fields])


def gf_batch_overrelax(b: Batch, fields, omega: float, theta_target: float, max_iter: int,
                       raise_on_error: bool = True):
    """Returns (rc, iters, F, theta) with per-lattice lists; fields fixed in place."""
    n = b.n
    it = (C.c_int * n)()
    F = (C.c_double * n)()
    th = (C.c_double * n)()
    rc = b.lib.gf_batch_overrelax(b.handle, _ptr_array(fields), omega, theta_target, int(max_iter),
                                  it, F, th)
    if raise_on_error:
        b.check(rc, "gf_batch_overrelax", ok=(GF_OK, GF_ENOTCONVERGED))
    return rc, list(it), list(F), list(th)


def gf_overrelax_batched(dims_list, fields, omega: float, theta_target: float, max_iter: int):
    """One-call batched solve (Landau gauge, default batch options).
    Returns (rc, iters, F, theta) with per-lattice lists; fields fixed in place."""
    lib = load()
    n = len(dims_list)
    if len(fields) != n:
        raise ValueError("one field per lattice")
    flat = [int(d) for dims in dims_list for d in dims]
    if len(flat) != 4 * n:
        raise ValueError("four extents per lattice")
    it = (C.c_int * n)()
    F = (C.c_double * n)()
    th = (C.c_double * n)()
    rc = lib.gf_overrelax_batched(n, (C.c_int * len(flat))(*flat), _ptr_array(fields), float(omega),
                                  float(theta_target), int(max_iter), it, F, th)
    if rc not in (GF_OK, GF_ENOTCONVERGED):
        raise GFError(rc, "gf_overrelax_batched")
    return rc, list(it), list(F), list(th)


def gf_batch_autotune(b: Batch, fields):
    t, k = C.c_int(), C.c_int()
    b.check(b.lib.gf_batch_autotune(b.handle, _ptr_array(fields), C.byref(t), C.byref(k)),
            "gf_batch_autotune")
    return t.value, k.value


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------
GF_NET_CIN, GF_NET_COUT = 80, 8
NET_CHANNELS = (80, 32, 32, 32, 8)


def gf_net_param_count() -> int:
    return int(load().gf_net_param_count())


class Net:
    """Owns a gf_net handle."""

    def __init__(self, dims):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        h = _vp()
        rc = self.lib.gf_net_create((C.c_int * 4)(*self.dims), C.byref(h))
        if rc != GF_OK:
            raise GFError(rc, "gf_net_create")
        self.handle = h

    def check(self, rc: int, what: str) -> int:
        if rc != GF_OK:
            msg = self.lib.gf_net_last_error(self.handle)
            raise GFError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.gf_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gf_net_create(dims) -> Net:
    return Net(dims)


def gf_net_destroy(n: Net) -> None:
    n.close()


def gf_net_set_stream(n: Net, stream) -> None:
    s = getattr(stream, "cuda_stream", stream)
    n.check(n.lib.gf_net_set_stream(n.handle, s or None), "gf_net_set_stream")


def gf_net_set_option(n: Net, key: str, value: float) -> None:
    n.check(n.lib.gf_net_set_option(n.handle, key.encode(), float(value)), f"option {key}")


def gf_net_set_params(n: Net, params) -> None:
    n.check(n.lib.gf_net_set_params(n.handle, _ptr(params)), "gf_net_set_params")


def gf_net_get_params(n: Net, params) -> None:
    n.check(n.lib.gf_net_get_params(n.handle, _ptr(params)), "gf_net_get_params")


def gf_net_forward(n: Net, features, out) -> None:
    n.check(n.lib.gf_net_forward(n.handle, _ptr(features), _ptr(out)), "gf_net_forward")


def gf_net_gradient(n: Net, features, target, grad=None) -> float:
    loss = C.c_double()
    n.check(n.lib.gf_net_gradient(n.handle, _ptr(features), _ptr(target), _ptr(grad), C.byref(loss)),
            "gf_net_gradient")
    return loss.value


def gf_net_train_step(n: Net, features, target, lr: float) -> float:
    loss = C.c_double()
    n.check(n.lib.gf_net_train_step(n.handle, _ptr(features), _ptr(target), float(lr), C.byref(loss)),
            "gf_net_train_step")
    return loss.value


def gf_gauge_reset(ctx: Context) -> None:
    ctx.check(ctx.lib.gf_gauge_reset(ctx.handle), "gf_gauge_reset")


def gf_get_gauge(ctx: Context, g) -> None:
    ctx.check(ctx.lib.gf_get_gauge(ctx.handle, _ptr(g)), "gf_get_gauge")


def gf_converge(ctx: Context, omega: float, theta_target: float, max_iter: int):
    it, F, th = C.c_int(), C.c_double(), C.c_double()
    rc = ctx.check(ctx.lib.gf_converge(ctx.handle, omega, theta_target, int(max_iter), C.byref(it),
                                       C.byref(F), C.byref(th)), "gf_converge",
                   ok=(GF_OK, GF_ENOTCONVERGED))
    return rc == GF_OK, it.value, F.value, th.value


def gf_apply_tracked_gauge(ctx: Context, U) -> None:
    _check_field(ctx, U)
    ctx.check(ctx.lib.gf_apply_tracked_gauge(ctx.handle, _ptr(U)), "gf_apply_tracked_gauge")


def gf_features(ctx: Context, scale: float, features) -> None:
    ctx.check(ctx.lib.gf_features(ctx.handle, float(scale), _ptr(features)), "gf_features")


def gf_gauge_algebra(ctx: Context, scale: float, c) -> None:
    ctx.check(ctx.lib.gf_gauge_algebra(ctx.handle, float(scale), _ptr(c)), "gf_gauge_algebra")


def gf_apply_algebra(ctx: Context, c, scale: float) -> None:
    ctx.check(ctx.lib.gf_apply_algebra(ctx.handle, _ptr(c), float(scale)), "gf_apply_algebra")


def gf_set_net(ctx: Context, net) -> None:
    ctx.check(ctx.lib.gf_set_net(ctx.handle, net.handle if net is not None else None), "gf_set_net")
