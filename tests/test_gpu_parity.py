"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 form 1e-12 and FP32 form 2e-5, normwise per field (max |gpu - ref| /
max |ref|), cell ids bit-exact. The FP32 bound is the FP32 position/velocity rounding
(about 1e-7) times the few dozen operations of a step, with margin; the FP64 bound is
the same argument at 1e-16. Gradient-like fields (grad tau) are normwise because they
are differences of node values (element-wise error is unbounded where they vanish).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_15605_gb300 import mppic, synth

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 2e-5}


def normwise(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(got))) if got.size else 0.0
    return float(np.max(np.abs(got - ref)) / scale)


def host(t):
    return t.detach().double().cpu().numpy()


VEL = ("u", "v", "w")


def state_errors(dev, ref):
    """Normwise error of each state field of the device (re-ordered to the original parcel
    order by pid: mppic_step sorts the caller's arrays) against the oracle. Velocity
    components share one scale, the largest velocity magnitude of the reference."""
    order = dev["pid"].cpu().numpy()
    vscale = max(float(np.max(np.abs(ref[k]))) for k in VEL)
    out = {}
    for k in ("x", "y", "z", "u", "v", "w"):
        got = np.empty_like(ref[k])
        got[order] = host(dev[k])
        if k in VEL:
            out[k] = float(np.max(np.abs(got - ref[k]))) / max(vscale, 1e-300)
        else:
            out[k] = normwise(got, ref[k])
    return out


def rounded(parcels, prec):
    """The parcel state as the device stores it (FP32 form: rounded to float), in float64."""
    dt = np.float32 if prec == 32 else np.float64
    return {k: np.asarray(v, dtype=dt).astype(np.float64) for k, v in parcels.items()}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_15605_gb300 import build
    build.build()
    oracle.build()


# ---------------------------------------------------------------- binning --

@pytest.mark.parametrize("prec", [32, 64])
def test_binning_bit_exact_including_faces(prec):
    p = synth.make_params(13, 7, 21, dx=0.013, dy=0.021, dz=0.0071)
    rng = np.random.default_rng(10)
    n = 200_000
    L = np.array([13 * 0.013, 7 * 0.021, 21 * 0.0071])
    pos = rng.uniform(0, 1, (n, 3)) * L
    # a quarter of the parcels sit within a few ulps of a cell face
    k = n // 4
    for a, (nn, h) in enumerate(((13, 0.013), (7, 0.021), (21, 0.0071))):
        faces = rng.integers(0, nn + 1, k) * h
        pos[:k, a] = np.clip(faces * (1 + rng.integers(-3, 4, k) * 1e-7), 0, L[a])
    parcels = dict(x=pos[:, 0], y=pos[:, 1], z=pos[:, 2], u=np.zeros(n), v=np.zeros(n),
                   w=np.zeros(n), d=np.full(n, 1e-4), omega=np.ones(n))
    parcels = rounded(parcels, prec)
    b = mppic.Bed(p, precision=prec)
    dev = mppic.parcels_to_device(parcels, prec)
    b.bin(dev, do_sort=False)
    cell_ref, *_ = oracle.bin(p, parcels["x"], parcels["y"], parcels["z"])
    assert np.array_equal(dev["cell"].cpu().numpy(), cell_ref)


def check_level_layout(cell, orig, nx, ny, nz):
    """The layout rule of a sort. The cell kernel runs 128 threads per brick; thread u walks
    the parcels of two cells, lower-half cell u and an upper-half cell B(u), first those of
    cell u, then those of B(u). B(u) = u + 128 (the natural pairing), unless pairing by
    counts lowers the largest per-thread count by more than a tenth (tried only where the
    natural pairing's largest count exceeds the mean ceil(N/128) by more than a tenth): then
    the lower-half cells ranked by count descending take the upper-half cells ranked by
    count ascending (ties by cell index in both). The parcels of each warp (threads
    32w..32w+31) are stored level by level: the r-th parcel of every thread's sequence that
    has one, in thread order, then level r+1; within a cell parcels keep their order before
    the sort (`orig`: each parcel's index before it). Returns which bricks were paired by
    count."""
    n = cell.size
    i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    nbx, nby, nbz = -(-nx // 8), -(-ny // 8), -(-nz // 4)
    brick = (i // 8) + nbx * ((j // 8) + nby * (k // 4))
    local = (i % 8) + 8 * ((j % 8) + 8 * (k % 4))
    key = brick * 256 + local
    counts = np.bincount(key, minlength=nbx * nby * nbz * 256).reshape(-1, 256)
    lo, up = counts[:, :128], counts[:, 128:]
    mx_nat = (lo + up).max(axis=1)
    tot = counts.sum(axis=1)
    tried = 10 * (-(-tot // 128)) < 9 * mx_nat
    idx = np.broadcast_to(np.arange(128), lo.shape)
    olo = np.lexsort((idx, -lo), axis=-1)          # lower half: count descending, then index
    oup = np.lexsort((idx, up), axis=-1)           # upper half: count ascending, then index
    pb = np.empty_like(olo)
    np.put_along_axis(pb, olo, oup + 128, axis=-1)
    mx_cnt = (lo + np.take_along_axis(counts, pb, axis=-1)).max(axis=1)
    paired = tried & (10 * mx_cnt < 9 * mx_nat)
    B = np.where(paired[:, None], pb, idx + 128)
    inv = np.empty_like(B)                         # thread of each upper-half cell
    np.put_along_axis(inv, B - 128, idx, axis=-1)
    # rank of each parcel within its cell, in the order before the sort
    o = np.lexsort((orig, key))
    first = np.searchsorted(key[o], key[o], side="left")
    lvl = np.empty(n, np.int64)
    lvl[o] = np.arange(n) - first
    upper = local >= 128
    u = np.where(upper, inv[brick, np.where(upper, local - 128, 0)], local)
    s = np.where(upper, counts[brick, u] + lvl, lvl)
    t = np.stack([brick, u // 32, s, u], axis=1)
    d = np.diff(t, axis=0)
    inc = np.zeros(len(d), bool)
    eq = np.ones(len(d), bool)
    for c in range(t.shape[1]):
        inc |= eq & (d[:, c] > 0)
        eq &= d[:, c] == 0
    assert np.all(inc)
    return paired


@pytest.mark.parametrize("prec", [32, 64])
def test_sort_is_a_stable_level_permutation(prec):
    bed = synth.settle_bed(n=50_000, nx=20, ny=12, nz=9)   # grid not a multiple of the brick
    b = mppic.Bed(bed.params, precision=prec)
    dev = mppic.parcels_to_device(bed.parcels, prec, with_pid=True)
    x0 = host(dev["x"]).copy()
    b.bin(dev, do_sort=True)
    pid = dev["pid"].cpu().numpy()
    assert np.array_equal(np.sort(pid), np.arange(bed.np))
    np.testing.assert_array_equal(host(dev["x"]), x0[pid])        # arrays moved together
    paired = check_level_layout(dev["cell"].cpu().numpy(), pid, 20, 12, 9)
    assert paired.any() and not paired.all()       # the bed exercises both choices


FIELDS = ("x", "y", "z", "u", "v", "w", "d", "omega", "pid")


def _move(dev, params, moves, seed):
    """Move the parcels on the device: 'near' by up to 0.4 cell per axis; 'far' the same plus
    5% of the parcels anywhere in the box; 'shuffled' a random permutation of the arrays."""
    rng = np.random.default_rng(seed)
    n = dev["x"].numel()
    if moves == "shuffled":
        perm = torch.from_numpy(rng.permutation(n)).to(dev["x"].device)
        for f in FIELDS:
            dev[f].copy_(dev[f][perm])
        return
    h = np.array([params["dx"], params["dy"], params["dz"]])
    L = h * np.array([params["nx"], params["ny"], params["nz"]])
    pos = np.stack([host(dev[a]) for a in "xyz"], axis=1)
    pos += rng.uniform(-0.4, 0.4, (n, 3)) * h
    if moves == "far":
        sel = rng.random(n) < 0.05
        pos[sel] = rng.uniform(0.0, 1.0, (int(sel.sum()), 3)) * L
    pos = np.clip(pos, 0.0, L * (1 - 1e-6))
    for a, c in enumerate("xyz"):
        dev[c].copy_(torch.from_numpy(pos[:, a]).to(dev[c].dtype))


def _copy(dev):
    return {k: v.clone() for k, v in dev.items()}


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("moves", ["near", "far", "shuffled"])
@pytest.mark.parametrize("grid", [(50_000, 20, 12, 9), (20_000, 8, 8, 4), (60_000, 24, 8, 4)])
def test_local_resort_equals_full_sort(prec, moves, grid):
    """A sort that starts from the previous sort's layout re-sorts each brick from its own
    range and its 26 neighbours' (mppic_resort.cuh). Its result must be exactly the full
    radix sort's (a fresh handle, same input order): for parcels that stayed near, for
    parcels that moved anywhere ('far'), for an order unrelated to the layout ('shuffled'),
    and for bricks whose parcels exceed the shared-memory permutation (the 1-brick grid; the
    3-brick row, where shuffling also sends parcels beyond the neighbours)."""
    n, nx, ny, nz = grid
    bed = synth.settle_bed(n=n, nx=nx, ny=ny, nz=nz, seed=41)
    b = mppic.Bed(bed.params, precision=prec)
    dev = mppic.parcels_to_device(bed.parcels, prec, with_pid=True)
    b.bin(dev, do_sort=True)                       # first sort: the full radix sort
    _move(dev, bed.params, moves, seed=5)
    before = _copy(dev)
    b.bin(dev, do_sort=True)                       # second sort: local
    b.check()
    fresh = mppic.Bed(bed.params, precision=prec)
    full = _copy(before)
    fresh.bin(full, do_sort=True)
    fresh.check()
    for f in FIELDS + ("cell",):
        assert torch.equal(dev[f], full[f]), f
    pre = before["pid"].cpu().numpy()
    inv = np.empty_like(pre)
    inv[pre] = np.arange(n)
    orig = inv[dev["pid"].cpu().numpy()]
    np.testing.assert_array_equal(host(dev["x"]), host(before["x"])[orig])
    check_level_layout(dev["cell"].cpu().numpy(), orig, nx, ny, nz)


@pytest.mark.parametrize("moves", ["near", "far"])
def test_local_resort_batch_equals_full_sort(moves):
    """The same for a batch: brick neighbours never cross beds."""
    beds = [synth.settle_bed(n=n, nx=g[0], ny=g[1], nz=g[2], seed=60 + k)
            for k, (g, n) in enumerate((((9, 8, 16), 3000), ((16, 16, 20), 9000), ((8, 8, 4), 0),
                                        ((20, 7, 33), 12000)))]
    batch = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=32)
    dev, _ = mppic.concat_beds(beds, 32, with_pid=True)
    batch.bin(dev, do_sort=True)
    off = batch.offsets
    for k, bd in enumerate(beds):                  # move each bed's parcels in its own box
        if bd.np == 0:
            continue
        part = {f: dev[f][off[k]:off[k + 1]] for f in FIELDS}
        _move(part, bd.params, moves, seed=70 + k)
    before = _copy(dev)
    batch.bin(dev, do_sort=True)
    batch.check()
    fresh = mppic.Batch([b.params for b in beds], [b.np for b in beds], precision=32)
    full = _copy(before)
    fresh.bin(full, do_sort=True)
    fresh.check()
    for f in FIELDS + ("cell",):
        assert torch.equal(dev[f], full[f]), f


# --------------------------------------------------------------- deposit --

@pytest.mark.parametrize("prec", [32, 64])
def test_deposit_and_node_fields(prec):
    bed = synth.fourier_bed(n=60_000, nx=16, ny=16, nz=40, nsteps=1)
    parcels = rounded(bed.parcels, prec)
    p = bed.params
    b = mppic.Bed(p, precision=prec)
    dev = mppic.parcels_to_device(parcels, prec)
    gas = mppic.gas_to_device(bed.U, None, prec)
    Vs, fields = b.deposit(dev, gas)
    b.check()
    Vs_ref = oracle.deposit_volume(p, parcels["x"], parcels["y"], parcels["z"], parcels["d"],
                                   parcels["omega"])
    assert normwise(host(Vs), Vs_ref) <= TOL[prec]
    U = [np.asarray(u, dtype=np.float32 if prec == 32 else np.float64).astype(np.float64)
         for u in bed.U]
    es, ug, tau = oracle.node_fields(p, Vs_ref, U)
    f = host(fields)
    assert normwise(f[0], es) <= TOL[prec]
    for a in range(3):
        assert normwise(f[1 + a], ug[a]) <= TOL[prec]
    assert normwise(f[4], tau) <= TOL[prec]
    # conservation: total deposited volume equals total parcel volume
    total = float(np.sum(parcels["omega"] * np.pi / 6 * parcels["d"] ** 3))
    assert abs(float(host(Vs).sum()) - total) <= (1e-13 if prec == 64 else 1e-6) * total


@pytest.mark.parametrize("prec", [32, 64])
def test_interp(prec):
    bed = synth.fourier_bed(n=40_000, nx=12, ny=20, nz=33, nsteps=1)
    parcels = rounded(bed.parcels, prec)
    p = dict(bed.params, Ps=50.0)      # a visible stress gradient
    b = mppic.Bed(p, precision=prec)
    dev = mppic.parcels_to_device(parcels, prec)
    gas = mppic.gas_to_device(bed.U, None, prec)
    out = host(b.interp(dev, gas))
    b.check()
    Vs = oracle.deposit_volume(p, parcels["x"], parcels["y"], parcels["z"], parcels["d"],
                               parcels["omega"])
    U = [np.asarray(u, dtype=np.float32 if prec == 32 else np.float64).astype(np.float64)
         for u in bed.U]
    es, ug, tau = oracle.node_fields(p, Vs, U)
    ref = oracle.interp(p, parcels["x"], parcels["y"], parcels["z"], es, ug, tau)
    names = ["eps_s", "ugx", "ugy", "ugz", "gpx", "gpy", "gpz", "gtx", "gty", "gtz"]
    for r in range(10):
        assert normwise(out[r], ref[r]) <= TOL[prec], (names[r], normwise(out[r], ref[r]))


# ------------------------------------------------------------------ step --

def _step_compare(bed, prec, nsteps=1, sort_every=1, gradp_field=False):
    parcels = rounded(bed.parcels, prec)
    p = bed.params
    gp = None
    if gradp_field:
        nn = oracle.nnode(p)
        rng = np.random.default_rng(5)
        gp = [np.asarray(p["gradp"][a] + rng.normal(0, 2.0, nn),
                         dtype=np.float32 if prec == 32 else np.float64).astype(np.float64)
              for a in range(3)]
    U = [None if u is None else
         np.asarray(u, dtype=np.float32 if prec == 32 else np.float64).astype(np.float64)
         for u in bed.U]
    ref, ex, st = oracle.step(p, parcels, nsteps, U=U, gradp=gp)
    assert st == 0
    b = mppic.Bed(p, precision=prec, sort_every=sort_every)
    dev = mppic.parcels_to_device(parcels, prec, with_pid=True)
    gas = mppic.gas_to_device(U, gp, prec)
    obj = host(b.step(dev, gas, nsteps))
    A, B = b.drag_sums()
    b.check()
    return ref, ex, dev, obj, host(A), host(B)


@pytest.mark.parametrize("prec", [32, 64])
def test_single_step_all_fields(prec):
    bed = synth.fourier_bed(n=80_000, nx=16, ny=24, nz=40, nsteps=1)
    synth.random_velocities(bed, 0.3, seed=21)
    ref, ex, dev, obj, A, B = _step_compare(bed, prec)
    for k, err in state_errors(dev, ref).items():
        assert err <= TOL[prec], (k, err)
    assert normwise(A, ex["A"]) <= TOL[prec]
    for a in range(3):
        assert normwise(B[a], ex["B"][a]) <= TOL[prec]
    assert normwise(obj[:, 0], ex["obj"][:, 0]) <= TOL[prec]
    assert normwise(obj[:, 1], ex["obj"][:, 1]) <= TOL[prec]
    # binning of the new positions: the device cell ids equal the oracle's formula on the
    # positions the device stored
    cell_ref, *_ = oracle.bin(bed.params, host(dev["x"]), host(dev["y"]), host(dev["z"]))
    assert np.array_equal(dev["cell"].cpu().numpy(), cell_ref)


@pytest.mark.parametrize("prec", [32, 64])
def test_single_step_with_node_pressure_gradient_and_stress(prec):
    bed = synth.settle_bed(n=30_000, nx=9, ny=17, nz=20)
    bed.params.update(Ps=20.0)
    synth.random_velocities(bed, 0.2, seed=4)
    ref, ex, dev, obj, A, B = _step_compare(bed, prec, gradp_field=True)
    for k, err in state_errors(dev, ref).items():
        assert err <= TOL[prec], (k, err)


@pytest.mark.parametrize("prec", [32, 64])
def test_few_steps_sort_schedules(prec):
    """Several steps with sorting every step, every 3 steps and never: all match the oracle
    (the deposit is exact integer arithmetic, so stale orders cost time, not accuracy)."""
    bed = synth.settle_bed(n=20_000, nx=16, ny=16, nz=32)
    synth.random_velocities(bed, 0.5, seed=8)
    bed.params["dt"] = 5e-3          # parcels cross cells between sorts
    for every in (1, 3, 0):
        ref, ex, dev, obj, A, B = _step_compare(bed, prec, nsteps=6, sort_every=every)
        for k, err in state_errors(dev, ref).items():
            assert err <= 10 * TOL[prec], (every, k, err)
        assert normwise(obj[:, 0], ex["obj"][:, 0]) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("every,nsteps", [(1, 5), (2, 6), (2, 7), (3, 7)])
def test_permutation_sorts_equal_gathered_sorts(prec, every, nsteps):
    """A re-sort inside a step call writes only the permutation when no identity array travels
    with the parcels (the next step reads its parcels through it into the other buffer); with
    a pid array it moves the values. Both give the same layout and the same arithmetic, so the
    caller's arrays, objectives and drag sums must agree bit for bit, for sort periods and step
    counts that leave the values in either buffer at the end of the call."""
    bed = synth.settle_bed(n=20_000, nx=16, ny=16, nz=32)
    synth.random_velocities(bed, 0.5, seed=10)
    bed.params["dt"] = 5e-3          # parcels cross cells between sorts
    outs = []
    for with_pid in (True, False):
        b = mppic.Bed(bed.params, precision=prec, sort_every=every)
        dev = mppic.parcels_to_device(bed.parcels, prec, with_pid=with_pid)
        obj = b.step(dev, None, nsteps)
        obj2 = b.step(dev, None, 2)              # a second call from the layout left behind
        A, B = b.drag_sums()
        b.check()
        outs.append([host(dev[k]) for k in mppic.PARCEL_FIELDS] + [host(obj), host(obj2), host(A), host(B)])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("every", [1, 2])
def test_permutation_sorts_equal_gathered_sorts_batch(every):
    beds = synth.batched_beds(nbeds=6, np_lo=2_000, np_hi=20_000, seed=23)
    outs = []
    for with_pid in (True, False):
        dev, gas = mppic.concat_beds(beds, 32, with_pid=with_pid)
        b = mppic.Batch([x.params for x in beds], [x.np for x in beds], precision=32, sort_every=every)
        obj = b.step(dev, gas, 5)
        b.check()
        outs.append([host(dev[k]) for k in mppic.PARCEL_FIELDS] + [host(obj)])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("prec", [32, 64])
def test_step_is_deterministic(prec):
    bed = synth.settle_bed(n=40_000, nx=16, ny=16, nz=32)
    synth.random_velocities(bed, 0.5, seed=9)
    outs = []
    for _ in range(2):
        b = mppic.Bed(bed.params, precision=prec, sort_every=2)
        dev = mppic.parcels_to_device(bed.parcels, prec)
        obj = b.step(dev, None, 5)
        A, B = b.drag_sums()
        b.check()
        outs.append([host(dev[k]) for k in ("x", "w")] + [host(obj), host(A), host(B)])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


# ------------------------------------------------------------ edge cases --

@pytest.mark.parametrize("prec", [32, 64])
def test_empty_and_single_parcel(prec):
    p = synth.make_params(5, 3, 7, u_in=0.3)
    b = mppic.Bed(p, precision=prec)
    empty = {k: np.zeros(0) for k in mppic.PARCEL_FIELDS}
    dev = mppic.parcels_to_device(empty, prec)
    obj = host(b.step(dev, None, 2))
    b.check()
    assert np.all(obj == 0.0)
    one = dict(x=np.array([0.025]), y=np.array([0.015]), z=np.array([0.035]), u=np.zeros(1),
               v=np.zeros(1), w=np.array([-0.2]), d=np.array([2e-4]), omega=np.array([10.0]))
    one = rounded(one, prec)
    ref, ex, st = oracle.step(p, one, 3)
    dev = mppic.parcels_to_device(one, prec, with_pid=True)
    b2 = mppic.Bed(p, precision=prec)
    obj = host(b2.step(dev, None, 3))
    b2.check()
    for k, err in state_errors(dev, ref).items():
        assert err <= TOL[prec], (k, err)


@pytest.mark.parametrize("prec", [32, 64])
def test_parcels_on_walls_and_nodes(prec):
    """Parcels exactly on the far walls, on interior nodes and at the origin."""
    p = synth.make_params(4, 4, 4, dx=0.25, dy=0.25, dz=0.25, u_in=0.2)
    pos = np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0], [0.5, 0.25, 0.75], [1.0, 0.5, 0.0],
                    [0.125, 0.999, 0.5]])
    n = len(pos)
    parcels = dict(x=pos[:, 0], y=pos[:, 1], z=pos[:, 2], u=np.zeros(n), v=np.zeros(n),
                   w=np.zeros(n), d=np.full(n, 1e-3), omega=np.full(n, 100.0))
    ref, ex, st = oracle.step(p, parcels, 1)
    b = mppic.Bed(p, precision=prec)
    dev = mppic.parcels_to_device(parcels, prec, with_pid=True)
    b.step(dev, None, 1)
    b.check()
    for k, err in state_errors(dev, ref).items():
        assert err <= TOL[prec], (k, err)


@pytest.mark.parametrize("prec", [32, 64])
def test_domain_error_is_reported_not_trapped(prec):
    """A parcel thrown faster than one box length per step cannot be reflected back: the
    device flags it and mppic_check reports DOMAIN; the context stays usable."""
    p = synth.make_params(4, 4, 4, drag_mult=0.0)
    parcels = dict(x=np.array([0.02]), y=np.array([0.02]), z=np.array([0.02]),
                   u=np.array([1e5]), v=np.zeros(1), w=np.zeros(1), d=np.array([1e-4]),
                   omega=np.ones(1))
    b = mppic.Bed(p, precision=prec)
    dev = mppic.parcels_to_device(parcels, prec)
    b.step(dev, None, 1)
    with pytest.raises(mppic.MppicError) as e:
        b.check()
    assert e.value.status == mppic.ERR_DOMAIN
    b.check()                                 # flag cleared, context fine
    torch.cuda.synchronize()
