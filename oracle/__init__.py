"""Plain FP64 CPU oracle for SU(3) gauge fixing by checkerboard overrelaxation.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it; the oracle is the slow, obviously
correct reference that the library's results are compared against.

The arithmetic lives in ``gf_oracle.c`` (plain C, FP64, compiled without FMA
contraction) and ``conv_oracle.c``; this module compiles them with gcc on first
use into ``oracle/_build/`` and wraps them with ctypes over numpy arrays.

Field layout (the library's canonical layout as well): a complex128 array of
shape (Lt, Lz, Ly, Lx, 4, 3, 3) -- x fastest among the sites, then the link
direction mu = x, y, z, t, then the 3x3 matrix row-major.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_SOURCE_DIR (tests only): build from another copy of the C sources; the
# mutation tests plant mistakes in such a copy and check that the pins fail
_SRC_DIR = os.environ.get("ORACLE_SOURCE_DIR") or _HERE
_BUILD = os.path.join(_SRC_DIR, "_build")
_SOURCES = ["gf_oracle.c", "conv_oracle.c"]
_lock = threading.Lock()
_libs: dict[str, C.CDLL] = {}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_long)
_u32p = C.POINTER(C.c_uint32)


def _compile(name: str, extra: list[str]) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, name)
    srcs = [os.path.join(_SRC_DIR, s) for s in _SOURCES]
    if os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wno-unused-function", *extra, *srcs, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build() -> None:
    """Compile both oracle builds (OpenMP, and single-thread flop counting)."""
    with _lock:
        _compile("liboracle.so", ["-fopenmp"])
        _compile("liboracle_count.so", ["-DORACLE_COUNT_FLOPS"])


def _declare(lib: C.CDLL) -> C.CDLL:
    d = lib
    d.oracle_or_half_sweep.argtypes = [_dp, _ip, C.c_int, C.c_double, C.c_int]
    d.oracle_or_sweeps.argtypes = [_dp, _ip, C.c_double, C.c_int, C.c_int]
    d.oracle_or_update_sites.argtypes = [_dp, _ip, _lp, C.c_long, C.c_double, C.c_int, _dp]
    d.oracle_block_quaternion.argtypes = [_dp, _dp]
    d.oracle_block_quaternion.restype = None
    d.oracle_overrelax_quaternion.argtypes = [_dp, C.c_double, _dp]
    d.oracle_set_sa_draw.argtypes = [C.c_int]
    d.oracle_set_sa_draw.restype = C.c_int
    d.oracle_set_or_variant.argtypes = [C.c_int]
    d.oracle_mag_half_sweep.argtypes = [_dp, _ip, C.c_int, C.c_double]
    d.oracle_mag_functional.argtypes = [_dp, _ip]
    d.oracle_mag_functional.restype = C.c_double
    d.oracle_mag_theta.argtypes = [_dp, _ip]
    d.oracle_mag_theta.restype = C.c_double
    d.oracle_mag_local_matrix.argtypes = [_dp, _ip, C.c_long, C.c_int, _dp]
    d.oracle_mag_maximiser.argtypes = [_dp, _dp]
    d.oracle_wilson_update.argtypes = [_dp, _ip, C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint64,
                                       C.c_uint32, C.c_int]
    d.oracle_wilson_update.restype = C.c_long
    d.oracle_staple.argtypes = [_dp, _ip, C.c_long, C.c_int, _dp]
    d.oracle_site_quaternion.argtypes = [_dp, _ip, C.c_long, C.c_int, C.c_int, _dp]
    d.oracle_site_rotate.argtypes = [_dp, _ip, C.c_long, C.c_int, _dp]
    for f in ("oracle_functional", "oracle_theta", "oracle_theta_from_M"):
        getattr(d, f).argtypes = [_dp, _ip, C.c_int]
        getattr(d, f).restype = C.c_double
    d.oracle_timeslices.argtypes = [_dp, _ip, C.c_int, _dp, _dp]
    d.oracle_plaquette.argtypes = [_dp, _ip]
    d.oracle_plaquette.restype = C.c_double
    d.oracle_gauge_transform.argtypes = [_dp, _dp, _ip]
    d.oracle_reunitarize.argtypes = [_dp, C.c_long]
    d.oracle_reunitarize.restype = None
    d.oracle_overrelax.argtypes = [_dp, _ip, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                   _ip, _dp, _dp]
    d.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    d.oracle_philox4x32_10.restype = None
    d.oracle_heatbath_quaternion.argtypes = [_dp, C.c_double, C.c_uint32, C.c_uint32, C.c_int,
                                             C.c_int, C.c_uint64, _dp]
    d.oracle_sa_half_sweep.argtypes = [_dp, _ip, C.c_int, C.c_double, C.c_int, C.c_uint64,
                                       C.c_uint32, C.c_int]
    d.oracle_sa_half_sweep.restype = C.c_long
    d.oracle_anneal.argtypes = [_dp, _ip, C.c_int, C.c_double, C.c_double, C.c_int, C.c_uint64,
                                C.c_uint32, C.c_int]
    d.oracle_anneal.restype = C.c_long
    d.oracle_sa_update_sites.argtypes = [_dp, _ip, _lp, C.c_long, C.c_double, C.c_int,
                                         C.c_uint64, C.c_uint32, C.c_int, _dp]
    d.oracle_conv_forward.argtypes = [_dp, _dp, _dp, _ip, C.c_int, C.c_int, _dp]
    d.oracle_conv_forward.restype = None
    d.oracle_conv_backward_data.argtypes = [_dp, _dp, _ip, C.c_int, C.c_int, _dp]
    d.oracle_conv_backward_data.restype = None
    d.oracle_conv_backward_weights.argtypes = [_dp, _dp, _ip, C.c_int, C.c_int, _dp, _dp]
    d.oracle_conv_backward_weights.restype = None
    d.oracle_net_loss.argtypes = [_dp, _dp, _dp, _ip, _ip, _dp, _dp]
    d.oracle_net_loss.restype = C.c_double
    d.oracle_sr_half_sweep.argtypes = [_dp, _ip, C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_uint32]
    d.oracle_features.argtypes = [_dp, _ip, C.c_double, _dp]
    d.oracle_expmap.argtypes = [_dp, C.c_double, _dp, C.c_long]
    d.oracle_expmap.restype = None
    d.oracle_algebra_log.argtypes = [_dp, C.c_double, _dp, C.c_long]
    d.oracle_algebra_log.restype = None
    d.oracle_flops.restype = C.c_ulonglong
    d.oracle_reset_flops.restype = None
    d.oracle_num_threads.restype = C.c_int
    return d


def lib(counting: bool = False) -> C.CDLL:
    """The compiled oracle (``counting=True``: the flop-counting build)."""
    name = "liboracle_count.so" if counting else "liboracle.so"
    with _lock:
        if name not in _libs:
            path = _compile(name, ["-DORACLE_COUNT_FLOPS"] if counting else ["-fopenmp"])
            _libs[name] = _declare(C.CDLL(path))
        return _libs[name]


# ---------------------------------------------------------------------------
# array helpers
# ---------------------------------------------------------------------------
def _field(U: np.ndarray) -> np.ndarray:
    if not (isinstance(U, np.ndarray) and U.dtype == np.complex128 and U.flags.c_contiguous
            and U.ndim == 7 and U.shape[4:] == (4, 3, 3)):
        raise TypeError("field must be a C-contiguous complex128 array (Lt,Lz,Ly,Lx,4,3,3)")
    return U


def dims_of(U: np.ndarray) -> np.ndarray:
    Lt, Lz, Ly, Lx = U.shape[:4]
    return np.array([Lx, Ly, Lz, Lt], dtype=np.intc)


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


# ---------------------------------------------------------------------------
# overrelaxation (Alg. 1)
# ---------------------------------------------------------------------------
def set_or_variant(v: int) -> None:
    """Reading of g -> g^omega for every later overrelaxation call of this
    process: 0 = the 19-flop rational form (default), 1 = first order,
    2 = the exact power (Sec. 2 leaves the order of the exponent open)."""
    _check(lib().oracle_set_or_variant(int(v)), "or variant")
    with _lock:
        counting = _libs.get("liboracle_count.so")
    if counting is not None:
        _check(counting.oracle_set_or_variant(int(v)), "or variant")


def set_sa_draw(fp32: int) -> None:
    """Precision of the annealing heatbath draw for every later call: 0 the
    FP64 definition (default), 1 the FP32 reading (see gf_oracle.c)."""
    _check(lib().oracle_set_sa_draw(int(fp32)), "sa draw")


def or_half_sweep(U, parity: int, omega: float, gauge: int = 0, counting: bool = False) -> None:
    U = _field(U)
    _check(lib(counting).oracle_or_half_sweep(_d(U), _i(dims_of(U)), parity, omega, gauge),
           "half sweep")


def or_sweeps(U, omega: float, gauge: int = 0, n: int = 1) -> None:
    U = _field(U)
    _check(lib().oracle_or_sweeps(_d(U), _i(dims_of(U)), omega, gauge, n), "sweeps")


def or_update_sites(U, sites, omega: float, gauge: int = 0) -> np.ndarray:
    """New links of each listed site after its OR update, from unmodified U.

    Returns (n, 8, 3, 3) complex: U_0..3(x) then U_0..3(x - mu).
    """
    U = _field(U)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((len(s), 8, 3, 3), dtype=np.complex128)
    _check(lib().oracle_or_update_sites(_d(U), _i(dims_of(U)), s.ctypes.data_as(_lp), len(s),
                                        omega, gauge, _d(out)), "update sites")
    return out


def block_quaternion(w: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.complex128).reshape(2, 2)
    k = np.zeros(4)
    lib().oracle_block_quaternion(_d(w), _d(k))
    return k


def overrelax_quaternion(k, omega: float):
    k = np.ascontiguousarray(k, dtype=np.float64)
    r = np.zeros(4)
    ok = lib().oracle_overrelax_quaternion(_d(k), omega, _d(r))
    return r if ok else None


def site_quaternion(U, site: int, gauge: int, sg: int) -> np.ndarray:
    U = _field(U)
    k = np.zeros(4)
    _check(lib().oracle_site_quaternion(_d(U), _i(dims_of(U)), site, gauge, sg, _d(k)), "quat")
    return k


def site_rotate(U, site: int, sg: int, r) -> None:
    U = _field(U)
    r = np.ascontiguousarray(r, dtype=np.float64)
    _check(lib().oracle_site_rotate(_d(U), _i(dims_of(U)), site, sg, _d(r)), "rotate")


# ---------------------------------------------------------------------------
# observables
# ---------------------------------------------------------------------------
def functional(U, gauge: int = 0) -> float:
    U = _field(U)
    return lib().oracle_functional(_d(U), _i(dims_of(U)), gauge)


def theta(U, gauge: int = 0) -> float:
    U = _field(U)
    return lib().oracle_theta(_d(U), _i(dims_of(U)), gauge)


def timeslices(U, gauge: int = 1):
    """(F_t, theta_t) of every timeslice t (arrays of length Lt)."""
    U = _field(U)
    Lt = U.shape[0]
    F = np.zeros(Lt)
    th = np.zeros(Lt)
    _check(lib().oracle_timeslices(_d(U), _i(dims_of(U)), gauge, _d(F), _d(th)), "timeslices")
    return F, th


def theta_from_M(U, gauge: int = 0) -> float:
    U = _field(U)
    return lib().oracle_theta_from_M(_d(U), _i(dims_of(U)), gauge)


def plaquette(U) -> float:
    U = _field(U)
    return lib().oracle_plaquette(_d(U), _i(dims_of(U)))


def gauge_transform(U, g) -> None:
    """U_mu(x) <- g(x) U_mu(x) g(x+mu)^dagger (eq. 1); g: (Lt,Lz,Ly,Lx,3,3)."""
    U = _field(U)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    if g.shape != U.shape[:4] + (3, 3):
        raise TypeError("gauge field shape mismatch")
    _check(lib().oracle_gauge_transform(_d(U), _d(g), _i(dims_of(U))), "gauge transform")


def reunitarize(M) -> None:
    if not (M.dtype == np.complex128 and M.flags.c_contiguous and M.shape[-2:] == (3, 3)):
        raise TypeError("need C-contiguous complex128 (...,3,3)")
    lib().oracle_reunitarize(_d(M), M.size // 9)


def overrelax(U, gauge: int, omega: float, theta_target: float, max_iter: int,
              check_every: int):
    """Alg. 1 with the stopping rule; returns (converged, sweeps, F, theta)."""
    U = _field(U)
    it = C.c_int(0)
    F = C.c_double(0)
    th = C.c_double(0)
    rc = lib().oracle_overrelax(_d(U), _i(dims_of(U)), gauge, omega, theta_target, max_iter,
                                check_every, C.byref(it), C.byref(F), C.byref(th))
    if rc < 0:
        raise ValueError("oracle overrelax rejected its arguments")
    return rc == 0, it.value, F.value, th.value


# ---------------------------------------------------------------------------
# random numbers and simulated annealing
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p),
                               out.ctypes.data_as(_u32p))
    return out


def heatbath_quaternion(k, T: float, site: int, sweep: int, sg: int, cap: int, seed: int):
    k = np.ascontiguousarray(k, dtype=np.float64)
    r = np.zeros(4)
    st = lib().oracle_heatbath_quaternion(_d(k), T, site, sweep, sg, cap, seed, _d(r))
    return st, r


def sa_half_sweep(U, parity: int, T: float, gauge: int, seed: int, sweep: int,
                  cap: int = 64) -> int:
    U = _field(U)
    f = lib().oracle_sa_half_sweep(_d(U), _i(dims_of(U)), parity, T, gauge, seed, sweep, cap)
    if f < 0:
        raise ValueError("oracle heatbath rejected its arguments")
    return f


def anneal(U, gauge: int, T0: float, T1: float, steps: int, seed: int, sweep_offset: int = 0,
           cap: int = 64) -> int:
    U = _field(U)
    f = lib().oracle_anneal(_d(U), _i(dims_of(U)), gauge, T0, T1, steps, seed, sweep_offset, cap)
    if f < 0:
        raise ValueError("oracle anneal rejected its arguments")
    return f


def sr_half_sweep(U, parity: int, p: float, gauge: int, seed: int, sweep: int) -> None:
    """Stochastic relaxation half-sweep: r* or, with probability p, r*^2."""
    U = _field(U)
    _check(lib().oracle_sr_half_sweep(_d(U), _i(dims_of(U)), parity, p, gauge, seed, sweep), "sr")


def sa_update_sites(U, sites, T: float, gauge: int, seed: int, sweep: int,
                    cap: int = 64) -> np.ndarray:
    U = _field(U)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((len(s), 8, 3, 3), dtype=np.complex128)
    _check(lib().oracle_sa_update_sites(_d(U), _i(dims_of(U)), s.ctypes.data_as(_lp), len(s), T,
                                        gauge, seed, sweep, cap, _d(out)), "sa update sites")
    return out


# ---------------------------------------------------------------------------
# flop counting build
# ---------------------------------------------------------------------------
def count_flops_half_sweep(U, parity: int, omega: float, gauge: int = 0) -> int:
    L = lib(counting=True)
    L.oracle_reset_flops()
    or_half_sweep(U, parity, omega, gauge, counting=True)
    return int(L.oracle_flops())


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ---------------------------------------------------------------------------
# learned warm start: periodic 3^4 convolutions and the four-layer network
# ---------------------------------------------------------------------------
def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims4(dims) -> np.ndarray:
    return np.array([int(d) for d in dims], dtype=np.intc)


def conv_forward(X, W, b, dims):
    """Y[s][co] = b[co] + sum_k sum_ci W[k][co][ci] X[s + d(k)][ci] (periodic)."""
    X, W = _f64(X), _f64(W)
    cout, cin = W.shape[1], W.shape[2]
    V = int(np.prod(dims))
    Y = np.zeros((V, cout))
    bb = _f64(b) if b is not None else None
    lib().oracle_conv_forward(_d(X), _d(W), _d(bb) if bb is not None else None, _i(_dims4(dims)), cin,
                              cout, _d(Y))
    return Y


def conv_backward_data(dY, W, dims):
    dY, W = _f64(dY), _f64(W)
    cout, cin = W.shape[1], W.shape[2]
    V = int(np.prod(dims))
    dX = np.zeros((V, cin))
    lib().oracle_conv_backward_data(_d(dY), _d(W), _i(_dims4(dims)), cin, cout, _d(dX))
    return dX


def conv_backward_weights(dY, X, dims, cin, cout):
    dY, X = _f64(dY), _f64(X)
    dW = np.zeros((81, cout, cin))
    db = np.zeros(cout)
    lib().oracle_conv_backward_weights(_d(dY), _d(X), _i(_dims4(dims)), cin, cout, _d(dW), _d(db))
    return dW, db


def features(U, scale: float) -> np.ndarray:
    """Network inputs (V, 80): forward-link reals, then tr(lambda_a Delta)/scale."""
    U = _field(U)
    V = int(np.prod(U.shape[:4]))
    f = np.zeros((V, 80))
    _check(lib().oracle_features(_d(U), _i(dims_of(U)), scale, _d(f)), "features")
    return f


def expmap(c, scale: float = 1.0) -> np.ndarray:
    """exp(i scale sum_a c_a lambda_a / 2) for c of shape (n, 8) -> (n, 3, 3) complex."""
    c = _f64(c).reshape(-1, 8)
    g = np.zeros((c.shape[0], 3, 3), dtype=np.complex128)
    lib().oracle_expmap(_d(c), scale, _d(g), c.shape[0])
    return g


def algebra_log(g, scale: float = 1.0) -> np.ndarray:
    """First-order algebra coefficients tr(lambda_a (g - g^+)/2i)/scale, (n, 8)."""
    g = np.ascontiguousarray(g, dtype=np.complex128).reshape(-1, 3, 3)
    c = np.zeros((g.shape[0], 8))
    lib().oracle_algebra_log(_d(g), scale, _d(c), g.shape[0])
    return c


def net_param_count(channels) -> int:
    return sum(81 * channels[l + 1] * channels[l] + channels[l + 1] for l in range(4))


def net_loss(f, target, params, dims, channels, want_grad=True):
    """Loss (and gradient w.r.t. the flat parameter vector, and the output)."""
    f, target, params = _f64(f), _f64(target), _f64(params)
    c = np.array(channels, dtype=np.intc)
    assert params.size == net_param_count(channels)
    grad = np.zeros_like(params) if want_grad else None
    V = int(np.prod(dims))
    out = np.zeros((V, channels[4]))
    loss = lib().oracle_net_loss(_d(f), _d(target), _d(params), _i(_dims4(dims)), _i(c),
                                 _d(grad) if grad is not None else None, _d(out))
    return loss, grad, out


# ---------------------------------------------------------------------------
# site helpers (canonical lexicographic order)
# ---------------------------------------------------------------------------
def site_index(dims, x, y, z, t) -> int:
    Lx, Ly, Lz, _ = dims
    return int(x + Lx * (y + Ly * (z + Lz * t)))


def site_parity(dims, i: int) -> int:
    Lx, Ly, Lz, _ = dims
    x = i % Lx
    y = (i // Lx) % Ly
    z = (i // (Lx * Ly)) % Lz
    t = i // (Lx * Ly * Lz)
    return (x + y + z + t) & 1


def backward_site(dims, i: int, mu: int) -> int:
    Lx, Ly, Lz, Lt = dims
    c = [i % Lx, (i // Lx) % Ly, (i // (Lx * Ly)) % Lz, i // (Lx * Ly * Lz)]
    c[mu] = (c[mu] - 1) % dims[mu]
    return site_index(dims, *c)


# ---------------------------------------------------------------------------
# maximally Abelian gauge (Sec. 6)
# ---------------------------------------------------------------------------
def mag_half_sweep(U, parity: int, omega: float) -> None:
    U = _field(U)
    _check(lib().oracle_mag_half_sweep(_d(U), _i(dims_of(U)), parity, omega), "mag half sweep")


def mag_sweeps(U, omega: float, n: int = 1) -> None:
    for _ in range(n):
        mag_half_sweep(U, 0, omega)
        mag_half_sweep(U, 1, omega)


def mag_functional(U) -> float:
    U = _field(U)
    return lib().oracle_mag_functional(_d(U), _i(dims_of(U)))


def mag_theta(U) -> float:
    U = _field(U)
    return lib().oracle_mag_theta(_d(U), _i(dims_of(U)))


def mag_local_matrix(U, site: int, sg: int) -> np.ndarray:
    U = _field(U)
    A = np.zeros(16)
    _check(lib().oracle_mag_local_matrix(_d(U), _i(dims_of(U)), site, sg, _d(A)), "mag local matrix")
    return A.reshape(4, 4)


def mag_maximiser(A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(16)
    r = np.zeros(4)
    lib().oracle_mag_maximiser(_d(A), _d(r))
    return r


# ---------------------------------------------------------------------------
# Wilson-action gauge-field generation (thermalised inputs, Sec. 5)
# ---------------------------------------------------------------------------
def wilson_update(U, mu: int, parity: int, beta: float, mode: int, seed: int, sweep: int,
                  cap: int = 64) -> int:
    """mode 0 heatbath, 1 overrelaxation, for the links U_mu(x), x of one parity;
    returns the number of heatbath draws that hit the rejection cap."""
    U = _field(U)
    f = lib().oracle_wilson_update(_d(U), _i(dims_of(U)), mu, parity, beta, mode, seed, sweep, cap)
    if f < 0:
        raise ValueError("oracle wilson update rejected its arguments")
    return f


def wilson_sweep(U, beta: float, mode: int, seed: int, sweep: int) -> int:
    """All links once: directions 0..3, parities 0, 1."""
    f = 0
    for mu in range(4):
        for p in (0, 1):
            f += wilson_update(U, mu, p, beta, mode, seed, sweep)
    return f


def staple(U, site: int, mu: int) -> np.ndarray:
    U = _field(U)
    out = np.zeros((3, 3), dtype=np.complex128)
    _check(lib().oracle_staple(_d(U), _i(dims_of(U)), site, mu, _d(out)), "staple")
    return out
