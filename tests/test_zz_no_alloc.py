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
    b.close()


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
