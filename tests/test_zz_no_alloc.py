"""The allocation-free deposit entry point (mppic_deposit_static) against mppic_deposit.

Some callers of this library may not allocate device memory while they run it: a host
simulation code that owns a fixed device pool, or a solve phase where a cudaMalloc (and
the device synchronisation it implies) is not allowed. mppic_deposit_static serves them
from a static device array. This test calls it through the C ABI twice in a row and checks
each result against the handle-based mppic_deposit, within the parity tolerances used
everywhere else (1e-12 for FP64, 2e-5 for FP32, normwise). The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2211_15605_gb300 import mppic, synth

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 2e-5}


def _lib():
    from paper_2211_15605_gb300 import build
    build.build()
    L = mppic.load()
    L.mppic_deposit_static.argtypes = [ctypes.POINTER(mppic.Config), ctypes.POINTER(mppic.Parcels),
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.mppic_deposit_static.restype = ctypes.c_int
    return L


def _normwise(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", [32, 64])
def test_static_deposit_matches_handle_deposit_twice(prec):
    L = _lib()
    bed = synth.fourier_bed(n=50_000, nx=20, ny=16, nz=40, nsteps=1)
    dev = mppic.parcels_to_device(bed.parcels, prec)
    b = mppic.Bed(bed.params, precision=prec)
    Vs_ref, _ = b.deposit(dev, None)
    b.check()
    ref = Vs_ref.cpu().numpy()
    cfg = mppic.make_config(bed.params, prec, 0)
    ps = b._parcels(dev)
    stream = torch.cuda.current_stream()
    outs = []
    for _ in range(2):                      # the scratch is reused: the second call must not see the first
        out = torch.full((b.nnode,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.mppic_deposit_static(ctypes.byref(cfg), ctypes.byref(ps),
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == mppic.OK, L.mppic_last_error(None)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for o in outs:
        assert np.all(np.isfinite(o))
        assert _normwise(o, ref) <= TOL[prec]
    assert np.array_equal(outs[0], outs[1])
    # and against the oracle, with its total equal to the parcels' volumes
    dt = np.float32 if prec == 32 else np.float64
    q = {k: np.asarray(bed.parcels[k], dt).astype(np.float64) for k in ("x", "y", "z", "d", "omega")}
    Vs_orc = oracle.deposit_volume(bed.params, q["x"], q["y"], q["z"], q["d"], q["omega"])
    assert _normwise(outs[0], Vs_orc) <= TOL[prec]
    d, om = np.asarray(bed.parcels["d"], dt), np.asarray(bed.parcels["omega"], dt)
    total = float(np.sum((om * (d * d * d) * dt(np.pi / 6)).astype(np.float64)))
    assert abs(float(outs[0].sum()) - total) <= 1e-12 * total
    b.close()


@pytest.mark.parametrize("bad", ["nan_diameter", "outside_box"])
def test_static_deposit_flags_bad_parcels_with_nan(bad):
    """A parcel that the deposit cannot place (a non-finite value, or a position outside the
    box) turns every output into NaN instead of a finite wrong sum; the next call is clean."""
    L = _lib()
    bed = synth.settle_bed(n=2000, nx=8, ny=8, nz=16)
    parcels = {k: v.copy() for k, v in bed.parcels.items()}
    if bad == "nan_diameter":
        parcels["d"][17] = np.nan
    else:
        parcels["z"][17] = 1.0                   # the box is 16 cm tall
    cfg = mppic.make_config(bed.params, 32, 0)
    nn = 9 * 9 * 17
    for p_, expect_nan in ((parcels, True), (bed.parcels, False)):
        dev = mppic.parcels_to_device(p_, 32)
        ps = mppic.Parcels()
        for k in mppic.PARCEL_FIELDS:
            setattr(ps, k, dev[k].data_ptr())
        ps.np = dev["x"].numel()
        out = torch.zeros(nn, dtype=torch.float64, device="cuda")
        st = L.mppic_deposit_static(ctypes.byref(cfg), ctypes.byref(ps), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == mppic.OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isnan(o)) if expect_nan else np.all(np.isfinite(o))


def test_static_deposit_rejects_grids_above_its_limit():
    L = _lib()
    p = synth.make_params(128, 128, 64)          # 129*129*65 nodes > MPPIC_STATIC_MAX_NODES
    cfg = mppic.make_config(p, 32, 0)
    ps = mppic.Parcels()
    ps.np = 0
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = L.mppic_deposit_static(ctypes.byref(cfg), ctypes.byref(ps), ctypes.c_void_p(out.data_ptr()),
                                None)
    assert st == mppic.ERR_INVALID
    assert b"static scratch limit" in L.mppic_last_error(None)
