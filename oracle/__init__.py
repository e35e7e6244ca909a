"""FP64 CPU oracle of the MP-PIC parcel-grid coupling step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and its
Python binding) never does, and the two share no code: this wrapper has its own
config struct and its own build of ``mppic_oracle.cpp``.

What each function computes is stated, with the passage of Woo et al.
(arXiv 2211.15605) it follows, in ``mppic_oracle.cpp``.

Functions without an independent pin: none. The pins live in
``tests/test_oracle_pins.py`` (closed forms, invariants, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppic_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libmppic_oracle.so")
_SRC_MT = os.path.join(_HERE, "mppic_oracle_mt.cpp")
_LIB_MT = os.path.join(_HERE, "_build", "libmppic_oracle_mt.so")
_lock = threading.Lock()
_lib = None
_lib_mt = None


def _compile(src, lib, extra=()):
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(src))
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", *extra, "-o", tmp, src])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FMA contraction off: binning is the plain IEEE product)."""
    if force and os.path.exists(_LIB):
        os.remove(_LIB)
    return _compile(_SRC, _LIB)


def build_mt() -> str:
    """Compile the multithreaded driver (OpenMP) used by the benchmark's all-core baseline."""
    return _compile(_SRC_MT, _LIB_MT, ("-fopenmp",))


class OrcConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("reserved0", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("mu_g", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("gradp", ctypes.c_double * 3),
                ("rho_p", ctypes.c_double), ("Ps", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps_cp", ctypes.c_double), ("alpha", ctypes.c_double),
                ("eps_g_min", ctypes.c_double), ("e_wall", ctypes.c_double),
                ("drag_mult", ctypes.c_double), ("dscale", ctypes.c_double),
                ("u_in", ctypes.c_double), ("dt", ctypes.c_double),
                ("drag_model", ctypes.c_int), ("coupling_iters", ctypes.c_int)]

# drag closures: Wen-Yu, Syamlal-O'Brien, Gidaspow (switch at eps_g = 0.8), Gidaspow blend
DRAG_MODELS = {"wen_yu": 0, "syamlal_obrien": 1, "gidaspow": 2, "gidaspow_blend": 3}


def make_config(p: dict) -> OrcConfig:
    c = OrcConfig()
    for name, _ in OrcConfig._fields_:
        if name == "reserved0":
            continue
        if name in ("drag_model", "coupling_iters"):
            setattr(c, name, int(p.get(name, 0)))
            continue
        v = p[name]
        if name in ("g", "gradp"):
            getattr(c, name)[:] = [float(t) for t in v]
        elif name in ("nx", "ny", "nz"):
            setattr(c, name, int(v))
        else:
            setattr(c, name, float(v))
    return c


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            cp = ctypes.POINTER(OrcConfig)
            L.orc_bin.argtypes = [cp, ctypes.c_long, dp, dp, dp, ip, dp, dp, dp]
            L.orc_deposit_volume.argtypes = [cp, ctypes.c_long, dp, dp, dp, dp, dp, dp]
            L.orc_node_fields.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_interp.argtypes = [cp, ctypes.c_long] + [dp] * 11 + [dp]
            L.orc_drag.argtypes = [cp, ctypes.c_long] + [dp] * 9
            L.orc_step.argtypes = ([cp, ctypes.c_long] + [dp] * 8 + [ip] + [dp] * 6
                                   + [ctypes.c_int] + [dp] * 6)
            L.orc_step.restype = ctypes.c_int
            L.orc_step_tangent.argtypes = ([cp, ctypes.c_long] + [dp] * 8 + [dp] * 6
                                           + [ctypes.c_int, dp])
            L.orc_step_tangent.restype = ctypes.c_int
            L.orc_step_sample.argtypes = ([cp, ctypes.c_long] + [dp] * 8 + [dp] * 3
                                          + [ctypes.c_long, ctypes.POINTER(ctypes.c_long), dp, ip, dp])
            L.orc_step_sample.restype = ctypes.c_int
            L.orc_couple.argtypes = [cp, ctypes.c_long] + [dp] * 24
            L.orc_couple.restype = None
            _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def grid_shape(p: dict):
    return int(p["nx"]), int(p["ny"]), int(p["nz"])


def nnode(p: dict) -> int:
    nx, ny, nz = grid_shape(p)
    return (nx + 1) * (ny + 1) * (nz + 1)


def bin(p, x, y, z):
    """Cell id and in-cell coordinates (xi, eta, zeta) of each parcel."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.size
    cell = np.empty(n, np.int32)
    xi, eta, zeta = np.empty(n), np.empty(n), np.empty(n)
    c = make_config(p)
    lib().orc_bin(ctypes.byref(c), n, _d(x), _d(y), _d(z),
                  cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(xi), _d(eta), _d(zeta))
    return cell, xi, eta, zeta


def deposit_volume(p, x, y, z, d, omega):
    """Deposited solids volume Vs at every node."""
    x, y, z, d, omega = map(_f64, (x, y, z, d, omega))
    Vs = np.empty(nnode(p))
    c = make_config(p)
    lib().orc_deposit_volume(ctypes.byref(c), x.size, _d(x), _d(y), _d(z), _d(d), _d(omega),
                             _d(Vs))
    return Vs


def node_fields(p, Vs, U=(None, None, None)):
    """(eps_s, ug[3], tau) at nodes from a deposited volume."""
    Vs = _f64(Vs)
    U = [_f64(a) for a in U]
    nn = nnode(p)
    es, ux, uy, uz, tau = (np.empty(nn) for _ in range(5))
    c = make_config(p)
    lib().orc_node_fields(ctypes.byref(c), _d(Vs), _d(U[0]), _d(U[1]), _d(U[2]), _d(es),
                          _d(ux), _d(uy), _d(uz), _d(tau))
    return es, np.stack([ux, uy, uz]), tau


def interp(p, x, y, z, eps_s, ug, tau, gradp=None):
    """Interpolated (eps_s, ug[3], gradp[3], gradtau[3]) as a (10, np) array."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    es, tau = _f64(eps_s), _f64(tau)
    ugs = [_f64(ug[a]) for a in range(3)]
    gps = [None] * 3 if gradp is None else [_f64(gradp[a]) for a in range(3)]
    out = np.empty((10, x.size))
    c = make_config(p)
    lib().orc_interp(ctypes.byref(c), x.size, _d(x), _d(y), _d(z), _d(es), _d(ugs[0]),
                     _d(ugs[1]), _d(ugs[2]), _d(gps[0]), _d(gps[1]), _d(gps[2]), _d(tau),
                     _d(out))
    return out


def drag(p, d, eps_s_p, ug_p, u, v, w):
    """Acceleration coefficient D_p per parcel of the configured drag closure."""
    d, es = _f64(d), _f64(eps_s_p)
    ug = [_f64(ug_p[a]) for a in range(3)]
    u, v, w = _f64(u), _f64(v), _f64(w)
    D = np.empty(d.size)
    c = make_config(p)
    lib().orc_drag(ctypes.byref(c), d.size, _d(d), _d(es), _d(ug[0]), _d(ug[1]), _d(ug[2]),
                   _d(u), _d(v), _d(w), _d(D))
    return D


def couple(p, state: dict, U=(None, None, None), gradp=None):
    """The coupling at the start of a step without moving the parcels: deposit, node fields
    and, with p["coupling_iters"] = K > 0, the K gas iterations of implicit coupling.

    Returns a dict with Vs, eps_s, ug (3, Nn) after the iterations, tau, and the drag sums
    A, B (3, Nn) of the last gas iteration (zero when K = 0)."""
    a = {k: _f64(state[k]) for k in ("x", "y", "z", "u", "v", "w", "d", "omega")}
    nn = nnode(p)
    out = {k: np.empty(nn) for k in ("Vs", "eps_s", "tau", "A")}
    ug, B = np.empty((3, nn)), np.empty((3, nn))
    U = [_f64(t) for t in U]
    gps = [None] * 3 if gradp is None else [_f64(gradp[i]) for i in range(3)]
    c = make_config(p)
    lib().orc_couple(ctypes.byref(c), a["x"].size, *[_d(a[k]) for k in
                     ("x", "y", "z", "u", "v", "w", "d", "omega")],
                     _d(U[0]), _d(U[1]), _d(U[2]), _d(gps[0]), _d(gps[1]), _d(gps[2]),
                     _d(out["Vs"]), _d(out["eps_s"]), _d(ug[0]), _d(ug[1]), _d(ug[2]),
                     _d(out["tau"]), _d(out["A"]), _d(B[0]), _d(B[1]), _d(B[2]))
    out.update(ug=ug, B=B)
    return out


def step(p, state: dict, nsteps: int, U=(None, None, None), gradp=None, outputs=True):
    """Advance ``nsteps`` coupling steps on a copy of ``state``.

    ``state`` holds x, y, z, u, v, w, d, omega arrays. Returns
    (new_state, extras, status) where extras has 'cell', 'obj' (nsteps, 2) and,
    if ``outputs``, the last step's node arrays 'Vs', 'A', 'B' (3, Nn).
    """
    s = {k: np.array(state[k], dtype=np.float64, copy=True) for k in
         ("x", "y", "z", "u", "v", "w")}
    d, om = _f64(state["d"]), _f64(state["omega"])
    n = s["x"].size
    nn = nnode(p)
    cell = np.empty(n, np.int32)
    obj = np.empty((max(nsteps, 1), 2))
    Vs = A = None
    B = None
    if outputs:
        Vs, A, B = np.empty(nn), np.empty(nn), np.empty((3, nn))
    U = [_f64(a) for a in U]
    gps = [None] * 3 if gradp is None else [_f64(gradp[a]) for a in range(3)]
    c = make_config(p)
    st = lib().orc_step(ctypes.byref(c), n, _d(s["x"]), _d(s["y"]), _d(s["z"]), _d(s["u"]),
                        _d(s["v"]), _d(s["w"]), _d(d), _d(om),
                        cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        _d(U[0]), _d(U[1]), _d(U[2]), _d(gps[0]), _d(gps[1]), _d(gps[2]),
                        int(nsteps), _d(Vs), _d(A),
                        _d(B[0]) if B is not None else None,
                        _d(B[1]) if B is not None else None,
                        _d(B[2]) if B is not None else None, _d(obj))
    s["d"], s["omega"] = d.copy(), om.copy()
    extras = {"cell": cell, "obj": obj[:nsteps]}
    if outputs:
        extras.update(Vs=Vs, A=A, B=B)
    return s, extras, int(st)


def step_tangent(p, state: dict, nsteps: int, U=(None, None, None), gradp=None):
    """Forward-mode oracle gradient over ``nsteps`` steps.

    Returns (means, grads, status): means = (<dP>, <H>), grads is a (2, 3) array
    d(<dP>, <H>)/d(drag_mult, dscale, u_in).
    """
    s = {k: np.array(state[k], dtype=np.float64, copy=True) for k in
         ("x", "y", "z", "u", "v", "w")}
    d, om = _f64(state["d"]), _f64(state["omega"])
    U = [_f64(a) for a in U]
    gps = [None] * 3 if gradp is None else [_f64(gradp[a]) for a in range(3)]
    out = np.empty(8)
    c = make_config(p)
    st = lib().orc_step_tangent(ctypes.byref(c), s["x"].size, _d(s["x"]), _d(s["y"]),
                                _d(s["z"]), _d(s["u"]), _d(s["v"]), _d(s["w"]), _d(d), _d(om),
                                _d(U[0]), _d(U[1]), _d(U[2]), _d(gps[0]), _d(gps[1]),
                                _d(gps[2]), int(nsteps), _d(out))
    return out[:2].copy(), np.stack([out[2:5], out[5:8]]), int(st)


def step_sample(p, state: dict, sample, U=(None, None, None)):
    """One step of the sampled parcels with node fields deposited by all parcels.

    Returns (new (6, ns) array of x, y, z, u, v, w; cell ids; f per parcel; status)."""
    arrs = {k: _f64(state[k]) for k in ("x", "y", "z", "u", "v", "w", "d", "omega")}
    idx = np.ascontiguousarray(sample, dtype=np.int64)
    ns = idx.size
    out = np.empty((6, ns))
    cell = np.empty(ns, np.int32)
    f = np.empty(ns)
    U = [_f64(a) for a in U]
    c = make_config(p)
    st = lib().orc_step_sample(ctypes.byref(c), arrs["x"].size, *[_d(arrs[k]) for k in
                               ("x", "y", "z", "u", "v", "w", "d", "omega")],
                               _d(U[0]), _d(U[1]), _d(U[2]), ns,
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _d(out),
                               cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(f))
    return out, cell, f, int(st)


def lib_mt():
    global _lib_mt
    with _lock:
        if _lib_mt is None:
            L = ctypes.CDLL(build_mt())
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_step_mt.argtypes = ([ctypes.POINTER(OrcConfig), ctypes.c_long] + [dp] * 8
                                      + [dp] * 3 + [ctypes.c_int, dp, ctypes.c_int])
            L.orc_step_mt.restype = ctypes.c_int
            L.orc_max_threads.restype = ctypes.c_int
            _lib_mt = L
    return _lib_mt


def max_threads() -> int:
    return int(lib_mt().orc_max_threads())


def step_mt(p, state: dict, nsteps: int, U=(None, None, None), nthreads: int = 0):
    """``step`` on ``nthreads`` OpenMP threads (0: all), for timing the oracle on every core:
    the same functions over fixed per-thread parcel ranges, reduced in thread order.
    Returns (new_state, (nsteps, 2) objectives, status)."""
    s = {k: np.array(state[k], dtype=np.float64, copy=True) for k in
         ("x", "y", "z", "u", "v", "w")}
    d, om = _f64(state["d"]), _f64(state["omega"])
    U = [_f64(a) for a in U]
    obj = np.empty((max(nsteps, 1), 2))
    c = make_config(p)
    st = lib_mt().orc_step_mt(ctypes.byref(c), s["x"].size, _d(s["x"]), _d(s["y"]), _d(s["z"]),
                              _d(s["u"]), _d(s["v"]), _d(s["w"]), _d(d), _d(om), _d(U[0]),
                              _d(U[1]), _d(U[2]), int(nsteps), _d(obj), int(nthreads))
    s["d"], s["omega"] = d.copy(), om.copy()
    return s, obj[:nsteps], int(st)
