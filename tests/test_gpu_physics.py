"""GPU parity (through the C ABI) for the regimes and forms beyond the dilute Wen-Yu step:
the other drag laws (Syamlal-O'Brien, Gidaspow, Gidaspow blend), implicit coupling, the
Newton regime of Wen-Yu drag (Re_m >= 1000), a dense pocket above close packing (the alpha
branch of Eq. 5 and the voidage floor of the drag), and the FP32 form's exact conservation
of the deposited solids volume.

Tolerances as in test_gpu_parity: FP64 form 1e-12, FP32 form 2e-5, normwise per field;
conservation 1e-12 relative in both forms.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2211_15605_gb300 import mppic, synth

from test_gpu_parity import TOL, host, normwise, rounded, state_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15605_gb300 import build
    build.build()
    oracle.build()


def graded_bed(n, nx, ny, nz, es_lo, es_hi, seed, vel=0.3):
    """Parcels uniform in the lower 60% of the box whose volumes grade the solids fraction
    from es_lo at the floor to es_hi at the top of the fill (lognormal d, median 150 um)."""
    rng = np.random.default_rng(seed)
    p = synth.make_params(nx, ny, nz, u_in=0.6, alpha=0.01)
    L = np.array([nx, ny, nz]) * 0.01
    x, y = rng.uniform(0, L[0], n), rng.uniform(0, L[1], n)
    z = rng.uniform(0, 0.6 * L[2], n)
    target = es_lo + (es_hi - es_lo) * z / (0.6 * L[2])
    vfill = L[0] * L[1] * 0.6 * L[2]
    V = target * vfill / n
    d = 150e-6 * np.exp(0.3 * np.clip(rng.standard_normal(n), -4, 4))
    omega = V / (math.pi / 6 * d ** 3)
    st = dict(x=x, y=y, z=z, u=vel * rng.standard_normal(n), v=vel * rng.standard_normal(n),
              w=vel * rng.standard_normal(n), d=d, omega=omega)
    return p, st


def run_compare(p, parcels, prec, nsteps=1, sort_every=1, U=(None, None, None)):
    parcels = rounded(parcels, prec)
    dt = np.float32 if prec == 32 else np.float64
    U = [None if u is None else np.asarray(u, dtype=dt).astype(np.float64) for u in U]
    ref, ex, st = oracle.step(p, parcels, nsteps, U=U)
    assert st == 0
    b = mppic.Bed(p, precision=prec, sort_every=sort_every)
    dev = mppic.parcels_to_device(parcels, prec, with_pid=True)
    gas = mppic.gas_to_device(U, None, prec)
    obj = host(b.step(dev, gas, nsteps))
    A, B = b.drag_sums()
    Vs = b.step_volume()
    b.check()
    out = dict(obj=obj, A=host(A), B=host(B), Vs=host(Vs))
    b.close()
    return ref, ex, dev, out, parcels


def assert_step_parity(ref, ex, dev, out, prec, tol_mult=1.0):
    tol = TOL[prec] * tol_mult
    for k, err in state_errors(dev, ref).items():
        assert err <= tol, (k, err)
    assert normwise(out["A"], ex["A"]) <= tol
    for a in range(3):
        assert normwise(out["B"][a], ex["B"][a]) <= tol, ("B", a)
    assert normwise(out["obj"][:, 0], ex["obj"][:, 0]) <= tol
    assert normwise(out["obj"][:, 1], ex["obj"][:, 1]) <= tol


def interpolated_eps_s(p, parcels):
    Vs = oracle.deposit_volume(p, parcels["x"], parcels["y"], parcels["z"], parcels["d"],
                               parcels["omega"])
    es, ug, tau = oracle.node_fields(p, Vs)
    return oracle.interp(p, parcels["x"], parcels["y"], parcels["z"], es, ug, tau)[0]


# ------------------------------------------------------------- drag laws --

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", [1, 2, 3])
def test_drag_law_single_step(prec, model):
    """One step of a bed graded from dilute (eps_s 0.05) to dense (0.5), so that Gidaspow
    takes both of its branches, with each drag law against the oracle."""
    p, st = graded_bed(60_000, 16, 12, 30, 0.05, 0.5, seed=31 + model)
    p.update(drag_model=model)
    es = interpolated_eps_s(p, rounded(st, prec))
    # Gidaspow's switch at eps_s = 0.2 is a hard conditional that each form decides in its own
    # precision; the FP32 interpolated eps_s is within about 2e-8 of the FP64 one, so with no
    # parcel within 1e-6 of the switch both forms take the oracle's branch (the seeds are
    # chosen so: the test checks its own premise)
    assert np.min(np.abs(es - 0.2)) > 1e-6
    assert np.mean(es > 0.2) > 0.3 and np.mean(es < 0.2) > 0.1
    ref, ex, dev, out, _ = run_compare(p, st, prec)
    assert_step_parity(ref, ex, dev, out, prec)


@pytest.mark.parametrize("prec", [32, 64])
def test_drag_laws_in_a_batch_equal_single_beds(prec):
    """Beds of a batch with different drag laws in one launch equal the same beds run alone."""
    beds = []
    for m in range(4):
        p, st = graded_bed(8_000 + 3_000 * m, 8 + 4 * m, 12, 20, 0.05, 0.45, seed=50 + m)
        p.update(drag_model=m)
        beds.append(synth.Bed(p, rounded(st, prec)))
    batch = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=prec, sort_every=1)
    parcels, gas = mppic.concat_beds(beds, prec, with_pid=True)
    batch.step(parcels, gas, 2)
    batch.check()
    offs = batch.offsets
    for i, bd in enumerate(beds):
        b = mppic.Bed(bd.params, precision=prec, sort_every=1)
        dev = mppic.parcels_to_device(bd.parcels, prec, with_pid=True)
        b.step(dev, None, 2)
        b.check()
        order = host(dev["pid"]).astype(np.int64)
        seg = slice(offs[i], offs[i + 1])
        border = host(parcels["pid"][seg]).astype(np.int64) - offs[i]     # pids are global
        for k in ("x", "w"):
            got = np.empty(bd.np)
            got[border] = host(parcels[k][seg])
            want = np.empty(bd.np)
            want[order] = host(dev[k])
            assert np.array_equal(got, want), (i, k)
        b.close()


# ------------------------------------------------------ implicit coupling --

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", [0, 1])
def test_implicit_coupling_steps(prec, model):
    """Implicit coupling with 3 gas iterations per step, two steps, against the oracle."""
    p, st = graded_bed(50_000, 12, 16, 24, 0.05, 0.45, seed=61)
    p.update(drag_model=model, coupling_iters=3, dt=2e-4)
    ref, ex, dev, out, _ = run_compare(p, st, prec, nsteps=2)
    assert_step_parity(ref, ex, dev, out, prec, tol_mult=2.0)


def test_implicit_coupling_changes_the_step():
    """The gas iterations matter: the drag sums and pressure drop of an implicit step differ
    from the explicit one by more than the tolerance (so the test above is not vacuous)."""
    p, st = graded_bed(30_000, 10, 10, 20, 0.1, 0.45, seed=62)
    outs = []
    for K in (0, 3):
        q = dict(p, coupling_iters=K, dt=2e-4)
        _, _, _, out, _ = run_compare(q, st, 64)
        outs.append(out)
    assert normwise(outs[1]["A"], outs[0]["A"]) > 1e-3
    assert abs(outs[1]["obj"][0, 0] - outs[0]["obj"][0, 0]) > 1e-3 * abs(outs[0]["obj"][0, 0])


@pytest.mark.parametrize("prec", [32, 64])
def test_implicit_coupling_batch_equals_single_beds(prec):
    beds = []
    for m in range(3):
        p, st = graded_bed(6_000 + 4_000 * m, 8 + 4 * m, 8, 16, 0.05, 0.4, seed=70 + m)
        p.update(coupling_iters=2, dt=2e-4, drag_model=m)
        beds.append(synth.Bed(p, rounded(st, prec)))
    cfg_params = dict(beds[0].params)
    batch = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=prec, sort_every=1)
    parcels, gas = mppic.concat_beds(beds, prec, with_pid=True)
    obj = host(batch.step(parcels, gas, 2))
    batch.check()
    offs = batch.offsets
    for i, bd in enumerate(beds):
        b = mppic.Bed(bd.params, precision=prec, sort_every=1)
        dev = mppic.parcels_to_device(bd.parcels, prec, with_pid=True)
        o = host(b.step(dev, None, 2))
        b.check()
        # the parcel state is the same bit for bit (exact integer deposits); the objectives
        # are reduced over bricks in a different tree in a batch, so they agree to rounding
        seg = slice(offs[i], offs[i + 1])
        border = host(parcels["pid"][seg]).astype(np.int64) - offs[i]
        order = host(dev["pid"]).astype(np.int64)
        for k in ("x", "y", "z", "u", "v", "w"):
            got = np.empty(bd.np)
            got[border] = host(parcels[k][seg])
            want = np.empty(bd.np)
            want[order] = host(dev[k])
            assert np.array_equal(got, want), (i, k)
        np.testing.assert_allclose(obj[:, i, :], o, rtol=1e-13 if prec == 64 else 1e-6)
        b.close()
    assert cfg_params["coupling_iters"] == 2


# ------------------------------------------------------------- regimes --

@pytest.mark.parametrize("prec", [32, 64])
def test_wen_yu_newton_regime(prec):
    """3 mm parcels with slips of 6 to 15 m/s: Re_m > 1000, the constant-Cd branch of
    Wen-Yu drag, against the oracle."""
    rng = np.random.default_rng(81)
    n = 4000
    p = synth.make_params(10, 10, 20, u_in=0.5, dt=2e-5)
    L = np.array([10, 10, 20]) * 0.01
    st = dict(x=rng.uniform(0.02, L[0] - 0.02, n), y=rng.uniform(0.02, L[1] - 0.02, n),
              z=rng.uniform(0.02, L[2] - 0.02, n), d=np.full(n, 3e-3), omega=np.ones(n))
    speed = rng.uniform(6.0, 15.0, n)
    direc = rng.standard_normal((n, 3))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    st.update(u=speed * direc[:, 0], v=speed * direc[:, 1], w=speed * direc[:, 2])
    rem = 1.2 * 3e-3 * speed / 1.8e-5                 # eps_g ~ 1 in this dilute bed
    assert np.min(rem) > 1000 * 1.1
    ref, ex, dev, out, _ = run_compare(p, st, prec)
    assert_step_parity(ref, ex, dev, out, prec)


def pocket_bed(prec):
    """A 4x4x4-cell block packed to eps_s = 0.75 (above close packing 0.6, voidage 0.25 below
    the floor 0.3) in a 6x6x8 box, lattice-seeded, inside a dilute random cloud; alpha = 1e-7."""
    p = synth.make_params(6, 6, 8, Ps=1.0, alpha=1e-7, u_in=0.3, dt=2e-5)
    per = 4
    s = 0.01 / per
    ax = (np.arange(4 * per) + 0.5) * s + 0.01
    Z, Y, X = np.meshgrid(ax + 0.01, ax, ax, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    d = 200e-6
    om_block = 0.75 * 1e-6 / per ** 3 / (math.pi / 6 * d ** 3)
    rng = np.random.default_rng(91)
    m = 3000
    L = np.array([6, 6, 8]) * 0.01
    xr, yr, zr = (rng.uniform(0, L[a], m) for a in range(3))
    st = dict(x=np.concatenate([x, xr]), y=np.concatenate([y, yr]), z=np.concatenate([z, zr]),
              d=np.full(x.size + m, d), omega=np.concatenate([np.full(x.size, om_block),
                                                                np.full(m, 10.0)]))
    nn = x.size + m
    st.update(u=0.05 * rng.standard_normal(nn), v=0.05 * rng.standard_normal(nn),
              w=0.05 * rng.standard_normal(nn))
    return p, st


@pytest.mark.parametrize("prec", [32, 64])
def test_dense_pocket_above_close_packing(prec):
    """Nodes above close packing take the alpha branch of Eq. 5 and parcels there the voidage
    floor of the drag; one step against the oracle."""
    p, st = pocket_bed(prec)
    parcels = rounded(st, prec)
    Vs = oracle.deposit_volume(p, parcels["x"], parcels["y"], parcels["z"], parcels["d"],
                               parcels["omega"])
    es, _, tau = oracle.node_fields(p, Vs)
    assert np.max(es) > 0.7 and np.sum(es > p["eps_cp"]) >= 27    # alpha branch and floor
    assert np.max(tau) > 1e6
    esp = interpolated_eps_s(p, parcels)
    assert np.sum(1 - esp < p["eps_g_min"]) > 100                  # drag at the floor
    ref, ex, dev, out, _ = run_compare(p, st, prec)
    assert_step_parity(ref, ex, dev, out, prec)


# --------------------------------------------------------- conservation --

def fp_volumes(parcels, prec, dscale=1.0):
    """Each parcel's volume as the form computes it: om * (d d d) * (pi/6 s_d^3), rounded
    to the form's precision at every product."""
    dt = np.float32 if prec == 32 else np.float64
    d = np.asarray(parcels["d"], dt)
    om = np.asarray(parcels["omega"], dt)
    vcoef = dt(math.pi / 6.0 * dscale ** 3)
    return (om * (d * d * d) * vcoef).astype(np.float64)


@pytest.mark.parametrize("prec", [32, 64])
def test_volume_conservation_exact(prec):
    """The deposited solids volume adds up to the parcels' volumes to 1e-12 relative (FP32
    form: exactly, in fixed point), for a deposit call, for the new positions of a step, and
    for a step whose parcels drifted off their sorted cells (sorted every 5 steps)."""
    bed = synth.fourier_bed(n=400_000, nx=40, ny=36, nz=70, nsteps=1)
    synth.random_velocities(bed, 0.3, seed=101)
    parcels = rounded(bed.parcels, prec)
    total = float(np.sum(fp_volumes(parcels, prec)))
    b = mppic.Bed(bed.params, precision=prec, sort_every=5)
    dev = mppic.parcels_to_device(parcels, prec)
    gas = mppic.gas_to_device(bed.U, None, prec)
    Vs, _ = b.deposit(dev, gas)
    b.check()
    assert abs(float(host(Vs).sum()) - total) <= 1e-12 * total
    for nsteps in (1, 3):
        b.step(dev, gas, nsteps)
        Vs = host(b.step_volume())
        b.check()
        assert abs(float(Vs.sum()) - total) <= 1e-12 * total, nsteps
    b.close()


def test_volume_conservation_drifted_dense_bed():
    """A dense polydisperse bed in which many parcels change cell between sorts (the off-cell
    path) conserves the FP32 volume exactly."""
    p, st = graded_bed(300_000, 24, 24, 40, 0.3, 0.55, seed=111, vel=0.5)
    p.update(dt=1e-3)
    parcels = rounded(st, 32)
    total = float(np.sum(fp_volumes(parcels, 32)))
    b = mppic.Bed(p, precision=32, sort_every=0)
    dev = mppic.parcels_to_device(parcels, 32)
    b.step(dev, None, 4)
    Vs = host(b.step_volume())
    b.check()
    assert abs(float(Vs.sum()) - total) <= 1e-12 * total
    b.close()
