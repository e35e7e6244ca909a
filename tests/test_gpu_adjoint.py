"""Reverse-mode gradients (mppic_backward) against the oracle's forward-mode gradient and
against central finite differences of the GPU forward, in FP64; the FP32 adjoint against
the FP64 one. Objectives: time averages of the drag-borne pressure drop and the bed height;
parameters: drag multiplier C, diameter scale s_d, inflow velocity u_in."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_15605_gb300 import mppic, synth

pytestmark = pytest.mark.gpu


def _bed(n=4000, steps=12):
    rng = np.random.default_rng(17)
    p = synth.make_params(8, 8, 16, u_in=0.4, dt=1e-4)
    Lx, Ly, Lz = 0.08, 0.08, 0.16
    st = dict(x=rng.uniform(0.01, Lx - 0.01, n), y=rng.uniform(0.01, Ly - 0.01, n),
              z=rng.uniform(0.3 * Lz, 0.6 * Lz, n), u=0.05 * rng.standard_normal(n),
              v=0.05 * rng.standard_normal(n), w=0.05 * rng.standard_normal(n),
              d=np.full(n, 150e-6), omega=np.full(n, 200.0))
    return p, st, steps


def _gpu_grad(p, st, steps, prec, every, weights):
    b = mppic.Bed(p, precision=prec, sort_every=3)
    dev = mppic.parcels_to_device(st, prec)
    b.checkpoint(every)
    obj = b.step(dev, None, steps)
    g = b.backward(*weights)
    b.check()
    return obj.mean(0).cpu().numpy(), np.array(g)


@pytest.mark.parametrize("every", [5, 12])
def test_adjoint_matches_oracle_tangent(every):
    p, st, steps = _bed()
    means, grads, status = oracle.step_tangent(p, st, steps)
    assert status == 0
    for o, weights in enumerate(((1.0, 0.0), (0.0, 1.0))):
        m, g = _gpu_grad(p, st, steps, 64, every, weights)
        np.testing.assert_allclose(m, means, rtol=1e-10)
        scale = np.max(np.abs(grads[o]))
        np.testing.assert_allclose(g, grads[o], rtol=1e-6, atol=1e-9 * scale)


def test_adjoint_matches_central_differences():
    """North-star check: gradients agree with central differences (h = 1e-4 relative) to 1e-4."""
    p, st, steps = _bed()
    m, g_dp = _gpu_grad(p, st, steps, 64, 4, (1.0, 0.0))
    _, g_h = _gpu_grad(p, st, steps, 64, 4, (0.0, 1.0))
    for k, name in enumerate(("drag_mult", "dscale", "u_in")):
        base = p[name]
        h = 1e-4 * base
        vals = []
        for sgn in (1, -1):
            q = dict(p)
            q[name] = base + sgn * h
            b = mppic.Bed(q, precision=64, sort_every=3)
            dev = mppic.parcels_to_device(st, 64)
            vals.append(b.step(dev, None, steps).mean(0).cpu().numpy())
            b.check()
        fd = (vals[0] - vals[1]) / (2 * h)
        for o, g in enumerate((g_dp, g_h)):
            scale = max(abs(fd[o]), 1e-3 * abs(m[o]) / base)
            assert abs(g[k] - fd[o]) <= 1e-4 * scale, (name, o, g[k], fd[o])


def test_fp32_adjoint_close_to_fp64():
    p, st, steps = _bed()
    _, g64 = _gpu_grad(p, st, steps, 64, 6, (1.0, 0.5))
    _, g32 = _gpu_grad(p, st, steps, 32, 6, (1.0, 0.5))
    np.testing.assert_allclose(g32, g64, rtol=2e-3, atol=2e-3 * np.max(np.abs(g64)))


def test_autograd_function():
    p, st, steps = _bed(n=2000, steps=6)
    b = mppic.Bed(p, precision=64, sort_every=3)
    dev = mppic.parcels_to_device(st, 64)
    theta = torch.tensor([1.0, 1.0, 0.4], dtype=torch.float64, requires_grad=True)
    out = mppic.BedObjectives.apply(theta, b, dev, None, steps, 3)
    loss = out[0] + 2.0 * out[1]
    loss.backward()
    means, grads, _ = oracle.step_tangent(p, st, steps)
    np.testing.assert_allclose(theta.grad.numpy(), grads[0] + 2.0 * grads[1], rtol=1e-6)


@pytest.mark.parametrize("prec", [32, 64])
def test_adjoint_is_bitwise_reproducible(prec):
    """Node adjoints are integer sums and every block sum is a fixed tree: two reverse sweeps
    of the same forward run, and of a second identical forward run, give identical bits."""
    p, st, steps = _bed()
    b = mppic.Bed(p, precision=prec, sort_every=3)
    b.checkpoint(5)
    b.step(mppic.parcels_to_device(st, prec), None, steps)
    g1 = np.array(b.backward(1.0, 0.5))
    g2 = np.array(b.backward(1.0, 0.5))
    b.check()
    _, g3 = _gpu_grad(p, st, steps, prec, 5, (1.0, 0.5))
    assert np.array_equal(g1, g2) and np.array_equal(g1, g3), (g1, g2, g3)
