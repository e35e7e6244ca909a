"""Parity at full workload sizes, multi-step statistics, and the adjoint at the size of the
differentiation bed.

* The 128x128x512 dense bed with 32M parcels, in the launch configuration bench.py times
  (persistent kernels, sort every 10 steps), one step: 3000 sampled parcels against the
  oracle, which deposits all 32M parcels and pushes the sample; per field within the form's
  tolerance, cell ids bit-exact.
* Multi-step runs compared through time-averaged pressure drop and bed height (the
  statistics the paper's Sec. 3 compares runs by), within 1%: FP32 and FP64 forms against
  the oracle on a reduced polydisperse bed; the FP32 form against the FP64 form on the full
  4M-parcel polydisperse bed (1000 steps) and on the 32M-parcel dense bed (500 steps).
* 500k parcels, 200 steps, checkpoints every 20: reverse-mode gradients against central
  differences of the GPU forward (h = 1e-4 relative), FP64, on the bed lifted clear of the
  floor; on the bed as drawn, whose bottom parcels bounce, against h = 1e-6 (see the test);
  the FP32 adjoint against the FP64 one.
"""
import functools
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2211_15605_gb300 import mppic, synth

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 2e-5}


def rounded(parcels, prec):
    dt = np.float32 if prec == 32 else np.float64
    return {k: np.asarray(v, dtype=dt).astype(np.float64) for k, v in parcels.items()}


@functools.lru_cache(maxsize=1)
def _dense():
    return synth.dense_bed()


@pytest.mark.parametrize("prec", [32, 64])
def test_full_size_dense_bed_sampled(prec):
    bed = _dense()
    state = rounded(bed.parcels, prec)
    b = mppic.Bed(bed.params, precision=prec, sort_every=10)
    dev = mppic.parcels_to_device(state, prec, with_pid=True)
    b.step(dev, None, 1)
    b.check()
    pid = dev["pid"].cpu().numpy()
    rng = np.random.default_rng(0)
    pos = np.sort(rng.choice(bed.np, 3000, replace=False))     # positions in device order
    out, _, _, st = oracle.step_sample(bed.params, state, pid[pos])
    assert st == 0
    at = torch.as_tensor(pos, device="cuda")
    got = np.stack([dev[k][at].double().cpu().numpy() for k in ("x", "y", "z", "u", "v", "w")])
    for a in range(3):
        err = np.max(np.abs(got[a] - out[a])) / np.max(np.abs(out[a]))
        assert err <= TOL[prec], ("xyz"[a], err)
    err = np.max(np.abs(got[3:6] - out[3:6])) / np.max(np.abs(out[3:6]))
    assert err <= TOL[prec], ("velocity", err)
    cref, *_ = oracle.bin(bed.params, got[0], got[1], got[2])
    assert np.array_equal(dev["cell"][at].cpu().numpy(), cref)
    b.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_full_size_dense_bed_node_arrays(prec):
    """The 32M-parcel dense bed, one step in the bench's launch configuration (sorted every 2
    steps): every node of the drag sums A and B[3] against the oracle's full step (all 32M
    parcels), and of the solids volume the step deposited for the new positions against the
    oracle's deposit of those positions, normwise per field and element-wise wherever the
    value is not a near-cancellation (|ref| > 1e-3 max); the new volume adds up to the
    parcels' volumes to 1e-12."""
    bed = _dense()
    state = rounded(bed.parcels, prec)
    _, ex, st = oracle.step(bed.params, state, 1)
    assert st == 0
    b = mppic.Bed(bed.params, precision=prec, sort_every=2)
    dev = mppic.parcels_to_device(state, prec)
    b.step(dev, None, 1)
    A, B = b.drag_sums()
    Vs = b.step_volume()
    b.check()
    hs = {k: dev[k].double().cpu().numpy() for k in ("x", "y", "z", "d", "omega")}
    Vs_ref = oracle.deposit_volume(bed.params, hs["x"], hs["y"], hs["z"], hs["d"], hs["omega"])
    got = {"Vs": Vs.cpu().numpy(), "A": A.cpu().numpy()}
    ref = {"Vs": Vs_ref, "A": ex["A"]}
    for a in range(3):
        got[f"B{a}"] = B[a].cpu().numpy()
        ref[f"B{a}"] = ex["B"][a]
    for k in got:
        scale = np.max(np.abs(ref[k]))
        err = np.abs(got[k] - ref[k])
        if scale == 0.0:                 # B_x, B_y of parcels at rest: exactly zero
            assert np.max(np.abs(got[k])) == 0.0, k
            continue
        assert np.max(err) / scale <= TOL[prec], (k, np.max(err) / scale)
        big = np.abs(ref[k]) > 1e-3 * scale
        assert np.max(err[big] / np.abs(ref[k][big])) <= 10 * TOL[prec], k
    dt = np.float32 if prec == 32 else np.float64
    d, om = np.asarray(state["d"], dt), np.asarray(state["omega"], dt)
    total = float(np.sum((om * (d * d * d) * dt(np.pi / 6)).astype(np.float64)))
    assert abs(float(got["Vs"].sum()) - total) <= 1e-12 * total
    b.close()


def _gpu_means(bed, prec, steps, U=None):
    state = rounded(bed.parcels, prec)
    U = bed.U if U is None else U
    U = [None if u is None else np.asarray(u, np.float32 if prec == 32 else np.float64)
         for u in U]
    b = mppic.Bed(bed.params, precision=prec, sort_every=10)
    dev = mppic.parcels_to_device(state, prec)
    gas = mppic.gas_to_device(U, None, prec)
    obj = b.step(dev, gas, steps).double().cpu().numpy()
    b.check()
    b.close()
    assert np.all(np.isfinite(obj))
    return obj.mean(0)


def _within(m, ref, rel=0.01):
    return abs(m[0] - ref[0]) <= rel * abs(ref[0]) and abs(m[1] - ref[1]) <= rel * abs(ref[1])


def test_multistep_statistics_against_oracle():
    bed = synth.fourier_bed(n=200_000, nx=32, ny=32, nz=64, nsteps=150)
    steps = 150
    for prec in (32, 64):
        U = [np.asarray(u, np.float32 if prec == 32 else np.float64).astype(np.float64)
             for u in bed.U]
        _, ex, st = oracle.step(bed.params, rounded(bed.parcels, prec), steps, U=U, outputs=False)
        assert st == 0
        ref = ex["obj"].mean(0)
        m = _gpu_means(bed, prec, steps)
        assert _within(m, ref), (prec, m, ref)


def test_multistep_fp32_against_fp64_polydisperse_4m():
    bed = synth.fourier_bed()                       # 64x64x256, 4M parcels
    steps = 1000
    m64 = _gpu_means(bed, 64, steps)
    m32 = _gpu_means(bed, 32, steps)
    assert _within(m32, m64), (m32, m64)


def test_multistep_fp32_against_fp64_dense_32m():
    bed = _dense()
    steps = 500
    m64 = _gpu_means(bed, 64, steps)
    m32 = _gpu_means(bed, 32, steps)
    assert _within(m32, m64), (m32, m64)


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grad_bed_tangent.json")
PARAMS = ("drag_mult", "dscale", "u_in")
BEDS = {"as_drawn": 0.0, "lifted_2cm": 0.02}    # floor clearance of the differentiation bed


@functools.lru_cache(maxsize=4)
def _adjoint(which, prec, steps=200, every=20):
    """Means and reverse-mode gradients (objective x parameter) of the 500k-parcel
    differentiation bed over 200 steps with checkpoints every 20."""
    bed = synth.grad_bed(floor_clearance=BEDS[which])
    b = mppic.Bed(bed.params, precision=prec, sort_every=10)
    dev = mppic.parcels_to_device(bed.parcels, prec)
    b.checkpoint(every)
    m = b.step(dev, None, steps).mean(0).double().cpu().numpy()
    g = np.array([b.backward(1.0, 0.0), b.backward(0.0, 1.0)])
    b.check()
    b.close()
    return m, g


def _central_difference(which, name, rel_h, steps=200):
    bed = synth.grad_bed(floor_clearance=BEDS[which])
    p = bed.params
    h = rel_h * p[name]
    vals = []
    for sgn in (1, -1):
        q = dict(p)
        q[name] = p[name] + sgn * h
        b = mppic.Bed(q, precision=64, sort_every=10)
        dev = mppic.parcels_to_device(bed.parcels, 64)
        vals.append(b.step(dev, None, steps).mean(0).cpu().numpy())
        b.check()
        b.close()
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("which", list(BEDS))
def test_adjoint_matches_stored_oracle_gradient_at_full_size(which):
    """Against the oracle's forward-mode (dual number) gradient of the same 200 steps,
    stored by tests/golden/make_grad_bed_tangent.py."""
    ref = json.load(open(GOLDEN))[which]
    m, g = _adjoint(which, 64)
    np.testing.assert_allclose(m, ref["means"], rtol=1e-10)
    for o in range(2):
        go = np.asarray(ref["grads"][o])
        np.testing.assert_allclose(g[o], go, rtol=1e-6, atol=1e-9 * np.max(np.abs(go)))


def test_adjoint_matches_central_differences_at_full_size():
    """Parcels lifted 2 cm off the floor (no wall contact within 20 ms): rel 1e-4 against
    central differences with h = 1e-4 relative."""
    _, g = _adjoint("lifted_2cm", 64)
    for k, name in enumerate(PARAMS):
        fd = _central_difference("lifted_2cm", name, 1e-4)
        for o in range(2):
            assert abs(g[o, k] - fd[o]) <= 1e-4 * abs(fd[o]), (name, o, g[o, k], fd[o])


def test_adjoint_with_wall_contact_at_full_size():
    """The differentiation bed as drawn: about 0.3% of the parcels start within 2 mm of the
    floor and bounce off it. Specular reflection makes the time-discrete map jump (the
    normal velocity changes sign in the step the parcel crosses the wall), so a central
    difference whose two runs put a bounce in different steps picks up a term of order
    (jump)/h that does not shrink with h. With h = 1e-6 no bounce moves and the difference
    is the derivative; with h = 1e-4 a few bounces move and the agreement is 1e-3."""
    _, g = _adjoint("as_drawn", 64)
    for k, name in enumerate(PARAMS):
        fd6 = _central_difference("as_drawn", name, 1e-6)
        fd4 = _central_difference("as_drawn", name, 1e-4)
        for o in range(2):
            assert abs(g[o, k] - fd6[o]) <= 1e-4 * abs(fd6[o]), (name, o, g[o, k], fd6[o])
            assert abs(g[o, k] - fd4[o]) <= 1e-3 * abs(fd4[o]), (name, o, g[o, k], fd4[o])


def test_fp32_adjoint_matches_fp64_at_full_size():
    _, g64 = _adjoint("as_drawn", 64)
    _, g32 = _adjoint("as_drawn", 32)
    np.testing.assert_allclose(g32, g64, rtol=1e-5)


@pytest.mark.parametrize("prec", [32, 64])
def test_adjoint_bitwise_reproducible_at_full_size(prec):
    """Two reverse sweeps of the 500k-parcel, 200-step forward give identical bits (integer
    node sums, fixed-tree block sums: no result depends on thread timing)."""
    bed = synth.grad_bed()
    b = mppic.Bed(bed.params, precision=prec, sort_every=10)
    b.checkpoint(20)
    b.step(mppic.parcels_to_device(bed.parcels, prec), None, 200)
    g1 = np.array(b.backward(1.0, 0.5))
    g2 = np.array(b.backward(1.0, 0.5))
    b.check()
    b.close()
    assert np.array_equal(g1, g2), (g1, g2)
