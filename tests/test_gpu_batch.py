"""Batched beds (one handle, one sort, one persistent launch per kernel) against the same
beds run one by one, and against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_15605_gb300 import mppic, synth

pytestmark = pytest.mark.gpu


def _beds():
    rng = np.random.default_rng(3)
    beds = []
    for k, (g, n) in enumerate((((9, 8, 16), 3000), ((16, 16, 20), 9000), ((5, 13, 11), 700),
                                ((8, 8, 4), 0), ((20, 7, 33), 12000))):
        b = synth.settle_bed(n=n, nx=g[0], ny=g[1], nz=g[2], seed=100 + k)
        b.params["u_in"] = float(rng.uniform(0.2, 1.0))
        synth.random_velocities(b, 0.3, seed=200 + k)
        beds.append(b)
    return beds


@pytest.mark.parametrize("prec", [32, 64])
def test_batch_equals_beds_run_alone(prec):
    beds = _beds()
    steps = 7
    batch = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=prec, sort_every=3)
    dev, gas = mppic.concat_beds(beds, prec)
    obj = batch.step(dev, gas, steps).cpu().numpy()
    batch.check()
    off = batch.offsets
    for k, b in enumerate(beds):
        one = mppic.Bed(b.params, precision=prec, sort_every=3)
        d1 = mppic.parcels_to_device(b.parcels, prec)
        o1 = one.step(d1, None, steps).cpu().numpy()
        one.check()
        for f in ("x", "y", "z", "u", "v", "w", "d", "omega"):
            assert torch.equal(dev[f][off[k]:off[k + 1]], d1[f]), (k, f)
        assert torch.equal(dev["cell"][off[k]:off[k + 1]], d1["cell"])
        np.testing.assert_allclose(obj[:, k, :], o1, rtol=1e-12, atol=0)


def test_batch_matches_oracle():
    beds = _beds()
    steps = 3
    batch = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=64, sort_every=1)
    dev, gas = mppic.concat_beds(beds, 64, with_pid=True)
    obj = batch.step(dev, gas, steps).cpu().numpy()
    batch.check()
    pid = dev["pid"].cpu().numpy()
    off = batch.offsets
    for k, b in enumerate(beds):
        if b.np == 0:
            assert np.all(obj[:, k, :] == 0)
            continue
        ref, ex, st = oracle.step(b.params, b.parcels, steps)
        assert st == 0
        order = pid[off[k]:off[k + 1]] - off[k]
        for f in ("x", "z", "w"):
            got = np.empty(b.np)
            got[order] = dev[f][off[k]:off[k + 1]].double().cpu().numpy()
            scale = np.max(np.abs(ref[f])) if f != "w" else max(np.max(np.abs(ref[c])) for c in "uvw")
            assert np.max(np.abs(got - ref[f])) <= 1e-12 * scale, (k, f)
        np.testing.assert_allclose(obj[:, k, 0], ex["obj"][:, 0], rtol=1e-11)
        np.testing.assert_allclose(obj[:, k, 1], ex["obj"][:, 1], rtol=1e-12)


def test_graph_replay_equals_eager_and_tuning_keeps_results():
    from paper_2211_15605_gb300 import tune
    beds = _beds()
    steps = 6
    ref = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=32, sort_every=3)
    d_ref, gas = mppic.concat_beds(beds, 32)
    o_ref = ref.step(d_ref, gas, steps)
    o_ref2 = ref.step(d_ref, gas, steps).clone()
    ref.check()
    g = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=32, sort_every=3)
    d_g, gas_g = mppic.concat_beds(beds, 32)
    obj = torch.empty((steps, len(beds), 2), dtype=torch.float64, device="cuda")
    g.tune(1, 3)                                       # a different persistent grid
    g.step_graph(d_g, gas_g, steps, obj)               # capture + launch
    o1 = obj.clone()
    g.step_graph(d_g, gas_g, steps, obj)               # relaunch
    g.check()
    for f in ("x", "y", "z", "u", "v", "w"):
        assert torch.equal(d_g[f], d_ref[f]), f
    assert torch.allclose(o1, o_ref, rtol=1e-12, atol=0) and torch.allclose(obj, o_ref2, rtol=1e-12, atol=0)
    res = tune.autotune(g, d_g, gas_g, steps=3, grids=(0, 1), sorts=(3, 6))
    assert res["best"] in res["ms_per_step"]


def test_graph_replay_with_gas_fields_equals_eager():
    """A batch with prescribed gas velocity fields: the sort and the step upload the same
    per-bed parameters, so a captured multi-step call (sorts included) replays as eager."""
    beds = [synth.fourier_bed(n=n, nx=g[0], ny=g[1], nz=g[2], nsteps=1, seed=300 + k)
            for k, (g, n) in enumerate((((16, 16, 24), 20000), ((9, 13, 20), 7000), ((24, 8, 16), 12000)))]
    steps = 6
    ref = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=32, sort_every=2)
    d_ref, gas = mppic.concat_beds(beds, 32)
    assert gas is not None
    o_ref = ref.step(d_ref, gas, steps).clone()
    ref.check()
    g = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=32, sort_every=2)
    d_g, gas_g = mppic.concat_beds(beds, 32)
    obj = torch.empty((steps, len(beds), 2), dtype=torch.float64, device="cuda")
    g.step_graph(d_g, gas_g, steps, obj)
    g.check()
    for f in ("x", "y", "z", "u", "v", "w"):
        assert torch.equal(d_g[f], d_ref[f]), f
    assert torch.allclose(obj, o_ref, rtol=1e-12, atol=0)
