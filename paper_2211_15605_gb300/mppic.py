"""Thin Python binding of libmppic (the C ABI of include/mppic.h).

Argument marshalling only: every step of the coupling runs in the CUDA kernels of the
library. PyTorch provides device memory and the stream. If the library has not been
built, the first call raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_DOMAIN, ERR_TIMEOUT, ERR_RANGE = range(7)
_NAMES = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "OOM", 4: "DOMAIN", 5: "TIMEOUT", 6: "RANGE"}
PARCEL_FIELDS = ("x", "y", "z", "u", "v", "w", "d", "omega")


class MppicError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mppic {_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("precision", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("mu_g", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("gradp", ctypes.c_double * 3),
                ("rho_p", ctypes.c_double), ("Ps", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps_cp", ctypes.c_double), ("alpha", ctypes.c_double),
                ("eps_g_min", ctypes.c_double), ("e_wall", ctypes.c_double),
                ("drag_mult", ctypes.c_double), ("dscale", ctypes.c_double),
                ("u_in", ctypes.c_double), ("dt", ctypes.c_double),
                ("sort_every", ctypes.c_int), ("drag_model", ctypes.c_int),
                ("coupling_iters", ctypes.c_int), ("reserved", ctypes.c_int)]

# drag closures (mppic_config.drag_model)
DRAG_MODELS = {"wen_yu": 0, "syamlal_obrien": 1, "gidaspow": 2, "gidaspow_blend": 3}


class Parcels(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in PARCEL_FIELDS] + [
        ("cell", ctypes.c_void_p), ("pid", ctypes.c_void_p), ("np", ctypes.c_longlong)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 7), ("launches", ctypes.c_longlong * 7),
                ("total_launches", ctypes.c_longlong), ("active_bricks", ctypes.c_longlong),
                ("parcels", ctypes.c_longlong)]


PHASES = ("sort", "deposit", "finalize", "step", "reduce", "other", "couple")


class Gas(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p * 3), ("gradp", ctypes.c_void_p * 3)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libmppic; raise if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmppic is not built ({path} missing): call "
                               "paper_2211_15605_gb300.build.build() first")
        L = ctypes.CDLL(path)
        H = ctypes.c_void_p
        st = ctypes.c_int
        L.mppic_create.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(H)]
        L.mppic_create.restype = st
        L.mppic_bin.argtypes = [H, ctypes.POINTER(Parcels), ctypes.c_int]
        L.mppic_bin.restype = st
        L.mppic_deposit.argtypes = [H, ctypes.POINTER(Parcels), ctypes.POINTER(Gas),
                                    ctypes.c_void_p, ctypes.c_void_p]
        L.mppic_deposit.restype = st
        L.mppic_interp.argtypes = [H, ctypes.POINTER(Parcels), ctypes.POINTER(Gas),
                                   ctypes.c_void_p]
        L.mppic_interp.restype = st
        L.mppic_step.argtypes = [H, ctypes.POINTER(Parcels), ctypes.POINTER(Gas), ctypes.c_int,
                                 ctypes.c_void_p]
        L.mppic_step.restype = st
        L.mppic_drag_sums.argtypes = [H] + [ctypes.c_void_p] * 4
        L.mppic_drag_sums.restype = st
        L.mppic_step_volume.argtypes = [H, ctypes.c_void_p]
        L.mppic_step_volume.restype = st
        L.mppic_check.argtypes = [H]
        L.mppic_check.restype = st
        L.mppic_set_params.argtypes = [H, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.mppic_set_params.restype = st
        L.mppic_checkpoint.argtypes = [H, ctypes.c_int]
        L.mppic_checkpoint.restype = st
        L.mppic_backward.argtypes = [H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.mppic_backward.restype = st
        L.mppic_tune.argtypes = [H, ctypes.c_int, ctypes.c_int]
        L.mppic_step_graph.argtypes = [H, ctypes.POINTER(Parcels), ctypes.POINTER(Gas),
                                       ctypes.c_int, ctypes.c_void_p]
        L.mppic_step_graph.restype = st
        L.mppic_tune.restype = st
        L.mppic_profile_enable.argtypes = [H, ctypes.c_int]
        L.mppic_profile_enable.restype = st
        L.mppic_profile_read.argtypes = [H, ctypes.POINTER(Profile)]
        L.mppic_profile_read.restype = st
        L.mppic_num_nodes.argtypes = [H]
        L.mppic_num_nodes.restype = ctypes.c_longlong
        L.mppic_destroy.argtypes = [H]
        L.mppic_destroy.restype = None
        L.mppic_last_error.argtypes = [H]
        L.mppic_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def make_config(params: dict, precision: int = 32, sort_every: int = 10) -> Config:
    c = Config()
    for name, _ in Config._fields_:
        if name in ("precision", "sort_every", "reserved"):
            continue
        if name in ("drag_model", "coupling_iters"):
            setattr(c, name, int(params.get(name, 0)))
            continue
        v = params[name]
        if name in ("g", "gradp"):
            getattr(c, name)[:] = [float(t) for t in v]
        elif name in ("nx", "ny", "nz"):
            setattr(c, name, int(v))
        else:
            setattr(c, name, float(v))
    c.precision = int(precision)
    c.sort_every = int(sort_every)
    return c


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def dtype_of(precision: int):
    return torch.float32 if precision == 32 else torch.float64


def parcels_to_device(parcels: dict, precision: int, device="cuda", with_pid=False) -> dict:
    """Copy a dict of numpy parcel arrays to contiguous device tensors of the precision."""
    dt = dtype_of(precision)
    out = {k: torch.as_tensor(parcels[k]).to(device=device, dtype=dt).contiguous()
           for k in PARCEL_FIELDS}
    n = out["x"].numel()
    out["cell"] = torch.zeros(n, dtype=torch.int32, device=device)
    if with_pid:
        out["pid"] = torch.arange(n, dtype=torch.int32, device=device)
    return out


def gas_to_device(U=(None, None, None), gradp=None, precision=32, device="cuda") -> dict:
    dt = dtype_of(precision)
    conv = lambda a: None if a is None else torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
    return {"U": [conv(a) for a in U],
            "gradp": None if gradp is None else [conv(a) for a in gradp]}


class Bed:
    """One bed: a libmppic handle bound to the current device and stream."""

    def __init__(self, params: dict, precision: int = 32, sort_every: int = 10, stream=None):
        self.L = load()
        self.params = dict(params)
        self.precision = precision
        self.dtype = dtype_of(precision)
        self.cfg = make_config(params, precision, sort_every)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = ctypes.c_void_p()
        st = self.L.mppic_create(ctypes.byref(self.cfg), 1, None, None,
                                 ctypes.c_void_p(s.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise MppicError(st, self.L.mppic_last_error(None).decode())
        self.h = h
        self.nnode = int(self.L.mppic_num_nodes(h))

    # -- marshalling
    def _parcels(self, p: dict) -> Parcels:
        s = Parcels()
        for k in PARCEL_FIELDS:
            t = p[k]
            assert t.dtype == self.dtype and t.is_cuda and t.is_contiguous(), k
            setattr(s, k, t.data_ptr())
        s.cell = p["cell"].data_ptr() if p.get("cell") is not None else None
        s.pid = p["pid"].data_ptr() if p.get("pid") is not None else None
        s.np = p["x"].numel()
        return s

    def _gas(self, g: dict | None):
        if g is None:
            return None
        s = Gas()
        for a in range(3):
            U = g["U"][a] if g.get("U") else None
            s.U[a] = None if U is None else U.data_ptr()
            gp = g["gradp"][a] if g.get("gradp") else None
            s.gradp[a] = None if gp is None else gp.data_ptr()
        return s

    def _check_obj(self, obj, nsteps):
        nb = getattr(self, "nbeds", 1)
        if (obj is None or obj.dtype != torch.float64 or not obj.is_cuda or not obj.is_contiguous()
                or obj.numel() < 2 * nb * nsteps):
            raise ValueError(f"obj must be a contiguous float64 device tensor of at least "
                             f"{nsteps} x {nb} x 2 values")

    def _ok(self, st):
        if st != OK:
            raise MppicError(st, self.L.mppic_last_error(self.h).decode())

    # -- API
    def bin(self, parcels: dict, do_sort: bool = False):
        ps = self._parcels(parcels)
        self._ok(self.L.mppic_bin(self.h, ctypes.byref(ps), int(do_sort)))

    def deposit(self, parcels: dict, gas: dict | None = None):
        """Deposited solids volume (double, nnode) and node fields (5, nnode)."""
        ps = self._parcels(parcels)
        gs = self._gas(gas)
        Vs = torch.empty(self.nnode, dtype=torch.float64, device=parcels["x"].device)
        fl = torch.empty((5, self.nnode), dtype=self.dtype, device=parcels["x"].device)
        self._ok(self.L.mppic_deposit(self.h, ctypes.byref(ps),
                                      ctypes.byref(gs) if gs is not None else None,
                                      _ptr(Vs), _ptr(fl)))
        return Vs, fl

    def interp(self, parcels: dict, gas: dict | None = None):
        """(10, np): eps_s, u_g[3], grad p[3], grad tau[3] at every parcel."""
        ps = self._parcels(parcels)
        gs = self._gas(gas)
        out = torch.empty((10, ps.np), dtype=self.dtype, device=parcels["x"].device)
        self._ok(self.L.mppic_interp(self.h, ctypes.byref(ps),
                                     ctypes.byref(gs) if gs is not None else None, _ptr(out)))
        return out

    def step(self, parcels: dict, gas: dict | None, nsteps: int, obj: torch.Tensor | None = None):
        """Advance nsteps in place; returns the (nsteps, 2) device tensor of (dP, H)."""
        ps = self._parcels(parcels)
        gs = self._gas(gas)
        if obj is None:
            obj = torch.empty((max(nsteps, 1), 2), dtype=torch.float64,
                              device=parcels["x"].device)
        self._check_obj(obj, nsteps)
        self._ok(self.L.mppic_step(self.h, ctypes.byref(ps),
                                   ctypes.byref(gs) if gs is not None else None,
                                   int(nsteps), _ptr(obj)))
        return obj[:nsteps]

    def drag_sums(self, device="cuda"):
        A = torch.empty(self.nnode, dtype=torch.float64, device=device)
        B = torch.empty((3, self.nnode), dtype=torch.float64, device=device)
        self._ok(self.L.mppic_drag_sums(self.h, _ptr(A), _ptr(B[0]), _ptr(B[1]), _ptr(B[2])))
        return A, B

    def step_volume(self, device="cuda"):
        """Solids volume (double, nnode) the last step deposited for the final positions."""
        Vs = torch.empty(self.nnode, dtype=torch.float64, device=device)
        self._ok(self.L.mppic_step_volume(self.h, _ptr(Vs)))
        return Vs

    def tune(self, grid_per_sm: int, sort_every: int = -1):
        """Persistent CTAs per SM of the step and deposit kernels (0 = all that fit) and,
        if >= 0, a new sort period."""
        self._ok(self.L.mppic_tune(self.h, int(grid_per_sm), int(sort_every)))

    def step_graph(self, parcels: dict, gas, nsteps: int, obj: torch.Tensor):
        """nsteps steps as one captured CUDA graph (captured on the first call with these
        arguments, relaunched afterwards). obj must be a preallocated device tensor."""
        ps = self._parcels(parcels)
        gs = self._gas(gas)
        self._check_obj(obj, nsteps)
        self._ok(self.L.mppic_step_graph(self.h, ctypes.byref(ps),
                                         ctypes.byref(gs) if gs is not None else None,
                                         int(nsteps), _ptr(obj)))
        return obj

    def set_params(self, drag_mult: float, dscale: float, u_in: float):
        """Set the three differentiable parameters (C, s_d, u_in) for later calls."""
        self._ok(self.L.mppic_set_params(self.h, float(drag_mult), float(dscale), float(u_in)))

    def checkpoint(self, every: int):
        """Save the parcel state every `every` steps in later step calls (0 = off)."""
        self._ok(self.L.mppic_checkpoint(self.h, int(every)))

    def backward(self, dL_ddP: float, dL_dH: float):
        """Gradient of dL_ddP <dP> + dL_dH <H> over the last checkpointed step call with
        respect to (C, s_d, u_in), as a tuple of three floats."""
        dl = (ctypes.c_double * 2)(float(dL_ddP), float(dL_dH))
        g = (ctypes.c_double * 3)()
        self._ok(self.L.mppic_backward(self.h, dl, g))
        return (g[0], g[1], g[2])

    def profile(self, enable: bool = True):
        """Enable or disable per-phase CUDA-event timing inside the library (resets counters)."""
        self._ok(self.L.mppic_profile_enable(self.h, int(enable)))

    def profile_read(self) -> dict:
        pr = Profile()
        self._ok(self.L.mppic_profile_read(self.h, ctypes.byref(pr)))
        return {"ms": {PHASES[i]: pr.ms[i] for i in range(len(PHASES))},
                "launches": {PHASES[i]: int(pr.launches[i]) for i in range(len(PHASES))},
                "total_launches": int(pr.total_launches),
                "active_bricks": int(pr.active_bricks), "parcels": int(pr.parcels)}

    def check(self):
        self._ok(self.L.mppic_check(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.L.mppic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BedObjectives(torch.autograd.Function):
    """Time-averaged (dP, H) of nsteps coupling steps as a differentiable function of
    theta = (drag multiplier C, diameter scale s_d, inflow velocity u_in).

    forward runs mppic_step with checkpointing on a copy of the parcel state; backward
    calls mppic_backward (hand-written adjoint kernels). theta is a CPU or CUDA tensor of
    3 values; the result is a float64 tensor (<dP>, <H>) on the parcels' device.
    """

    @staticmethod
    def forward(ctx, theta, bed: "Bed", parcels: dict, gas, nsteps: int, every: int = 20):
        th = [float(t) for t in theta.detach().cpu().tolist()]
        bed.set_params(*th)
        bed.checkpoint(every)
        state = {k: v.clone() for k, v in parcels.items()}
        obj = bed.step(state, gas, nsteps)
        ctx.bed = bed
        return obj.mean(0)

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().double().cpu().tolist()
        grad = ctx.bed.backward(g[0], g[1])
        return torch.tensor(grad, dtype=torch.float64), None, None, None, None, None


class Batch(Bed):
    """Many independent beds advanced together by one handle (one sort, one persistent
    launch per kernel and step). Parcels, and node arrays of the gas, are concatenated in
    bed order; step() returns the (nsteps, nbeds, 2) objectives."""

    def __init__(self, params_list, np_list, precision: int = 32, sort_every: int = 10,
                 stream=None):
        self.L = load()
        self.precision = precision
        self.dtype = dtype_of(precision)
        self.nbeds = len(params_list)
        cfgs = (Config * self.nbeds)(*[make_config(p, precision, sort_every) for p in params_list])
        self.cfg = make_config(params_list[0], precision, sort_every)
        offs = [0]
        for n in np_list:
            offs.append(offs[-1] + int(n))
        self.offsets = offs
        off_arr = (ctypes.c_longlong * (self.nbeds + 1))(*offs)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = ctypes.c_void_p()
        st = self.L.mppic_create(ctypes.byref(self.cfg), self.nbeds, off_arr, cfgs,
                                 ctypes.c_void_p(s.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise MppicError(st, self.L.mppic_last_error(None).decode())
        self.h = h
        self.nnode = int(self.L.mppic_num_nodes(h))
        self.params = list(params_list)

    def step(self, parcels: dict, gas, nsteps: int, obj=None):
        ps = self._parcels(parcels)
        gs = self._gas(gas)
        if obj is None:
            obj = torch.empty((max(nsteps, 1), self.nbeds, 2), dtype=torch.float64,
                              device=parcels["x"].device)
        self._check_obj(obj, nsteps)
        self._ok(self.L.mppic_step(self.h, ctypes.byref(ps),
                                   ctypes.byref(gs) if gs is not None else None,
                                   int(nsteps), _ptr(obj)))
        return obj[:nsteps]


def concat_beds(beds, precision, device="cuda", with_pid=False):
    """Concatenate synthetic beds (synth.Bed) into one parcel dict and one gas dict for Batch."""
    import numpy as np
    parcels = {k: np.concatenate([b.parcels[k] for b in beds]) for k in PARCEL_FIELDS}
    dev = parcels_to_device(parcels, precision, device=device, with_pid=with_pid)
    gas = None
    if any(u is not None for b in beds for u in b.U):
        U = []
        for a in range(3):
            parts = []
            for b in beds:
                nn = (b.params["nx"] + 1) * (b.params["ny"] + 1) * (b.params["nz"] + 1)
                parts.append(b.U[a] if b.U[a] is not None else np.zeros(nn))
            U.append(np.concatenate(parts))
        gas = gas_to_device(U, None, precision, device=device)
    return dev, gas
