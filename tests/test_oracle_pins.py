"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: exact rational
arithmetic, partition of unity and linear reproduction of trilinear weights,
volume conservation of the deposit (Sec. 2.1: V_parcel = w V_particle), closed-form
node values of Eq. 5, the continuous terminal velocity that the semi-implicit drag
update must reach (Eq. 4 at steady state), drag-free ballistic motion (Eqs. 3-4
with F_P = 0), the bed-weight balance of a uniformly fluidised bed (the paper's
Sec. 3.2 observation that the pressure drop is close to the bed weight), and
central finite differences for the tangent (oracle-gradient) mode.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2211_15605_gb300 import synth


def P(nx=4, ny=3, nz=5, **over):
    return synth.make_params(nx, ny, nz, **over)


# --------------------------------------------------------------- binning --

def test_bin_matches_exact_rationals():
    """The in-cell coordinate is x/dx - i to within one FP64 rounding of the product."""
    p = P(7, 5, 9, dx=0.013, dy=0.021, dz=0.0071)
    rng = np.random.default_rng(1)
    L = np.array([7 * 0.013, 5 * 0.021, 9 * 0.0071])
    pos = rng.uniform(0, 1, (200, 3)) * L
    cell, xi, eta, zeta = oracle.bin(p, pos[:, 0], pos[:, 1], pos[:, 2])
    n = (7, 5, 9)
    h = (0.013, 0.021, 0.0071)
    for q in range(200):
        idx = []
        for a, frac in enumerate((xi, eta, zeta)):
            exact = Fraction(pos[q, a]) / Fraction(h[a])   # exact real x/h
            i = min(max(math.floor(exact), 0), n[a] - 1)
            idx.append(i)
            # one rounding of x * fl(1/h): relative error <= 2^-52 of x/h
            assert abs(Fraction(frac[q]) + i - exact) <= Fraction(2) ** -50 * max(exact, 1)
        assert cell[q] == idx[0] + n[0] * (idx[1] + n[1] * idx[2])


def test_bin_special_positions():
    """Power-of-two spacing: nodes, faces and the far wall bin exactly."""
    p = P(4, 4, 4, dx=0.25, dy=0.25, dz=0.25)
    x = np.array([0.0, 0.25, 0.5, 1.0, 0.125, 0.999999])
    cell, xi, _, _ = oracle.bin(p, x, np.zeros_like(x), np.zeros_like(x))
    assert list(cell) == [0, 1, 2, 3, 0, 3]
    assert list(xi[:5]) == [0.0, 0.0, 0.0, 1.0, 0.5]    # x = L clamps to the last cell, xi = 1


# --------------------------------------------------------------- weights --

def _node_coords(p):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return (i.reshape(-1) * p["dx"], j.reshape(-1) * p["dy"], k.reshape(-1) * p["dz"])


def test_interp_reproduces_linear_fields_and_gradients():
    p = P(6, 4, 5, dx=0.02, dy=0.03, dz=0.01)
    rng = np.random.default_rng(2)
    L = np.array([6 * 0.02, 4 * 0.03, 5 * 0.01])
    pos = rng.uniform(0, 1, (300, 3)) * L
    X, Y, Z = _node_coords(p)
    a, b = 0.7, np.array([1.5, -2.0, 3.25])
    lin = a + b[0] * X + b[1] * Y + b[2] * Z
    ug = np.stack([lin, 2 * lin, -lin])
    out = oracle.interp(p, pos[:, 0], pos[:, 1], pos[:, 2], lin, ug, lin)
    expect = a + pos @ b
    np.testing.assert_allclose(out[0], expect, rtol=1e-13, atol=1e-14)        # eps_s slot
    np.testing.assert_allclose(out[3], -expect, rtol=1e-13, atol=1e-14)       # u_g,z
    for ax in range(3):                                                        # grad tau = b
        np.testing.assert_allclose(out[7 + ax], b[ax], rtol=1e-12)
    const = np.full_like(X, 4.2)
    out = oracle.interp(p, pos[:, 0], pos[:, 1], pos[:, 2], const, ug, const)
    np.testing.assert_allclose(out[0], 4.2, rtol=1e-15)
    assert np.max(np.abs(out[7:10])) < 1e-11                                   # grad of a constant
    np.testing.assert_allclose(out[4:7].T, np.tile(p["gradp"], (300, 1)))      # uniform grad p


# --------------------------------------------------------------- deposit --

def test_deposit_conserves_parcel_volume():
    p = P(5, 6, 7)
    rng = np.random.default_rng(3)
    n = 5000
    L = np.array([5, 6, 7]) * 0.01
    pos = rng.uniform(0, 1, (n, 3)) * L
    d = rng.uniform(50e-6, 400e-6, n)
    om = rng.uniform(1, 30, n)
    Vs = oracle.deposit_volume(p, pos[:, 0], pos[:, 1], pos[:, 2], d, om)
    total = float(np.sum(om * (4.0 / 3.0) * math.pi * (d / 2) ** 3))   # w * sphere volume
    assert abs(Vs.sum() - total) <= 1e-14 * total * 10
    assert Vs.min() >= 0.0


def _lattice(p, per_axis=2):
    """Parcels on a regular lattice, per_axis per cell along each axis, offset symmetric."""
    axes = []
    for n, h in ((p["nx"], p["dx"]), (p["ny"], p["dy"]), (p["nz"], p["dz"])):
        s = h / per_axis
        axes.append((np.arange(n * per_axis) + 0.5) * s)
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1)


def test_uniform_lattice_gives_uniform_solids_fraction():
    p = P(4, 5, 6)
    x, y, z = _lattice(p, 2)
    d = np.full(x.size, 300e-6)
    om = np.full(x.size, 20.0)
    Vs = oracle.deposit_volume(p, x, y, z, d, om)
    es, _, _ = oracle.node_fields(p, Vs)
    vpar = 20 * math.pi / 6 * (300e-6) ** 3
    expect = 8 * vpar / (0.01 ** 3)      # 8 parcels per cell, every node control volume
    np.testing.assert_allclose(es, expect, rtol=1e-13)


def test_deposit_interp_duality():
    """<deposit(V), phi>_nodes == <V, interp(phi)>_parcels: the two are transposes."""
    p = P(5, 4, 6)
    rng = np.random.default_rng(4)
    n = 3000
    L = np.array([5, 4, 6]) * 0.01
    pos = rng.uniform(0, 1, (n, 3)) * L
    d = rng.uniform(100e-6, 300e-6, n)
    om = rng.uniform(1, 10, n)
    phi = rng.standard_normal(oracle.nnode(p))
    Vs = oracle.deposit_volume(p, pos[:, 0], pos[:, 1], pos[:, 2], d, om)
    zero = np.zeros_like(phi)
    ip = oracle.interp(p, pos[:, 0], pos[:, 1], pos[:, 2], phi, [zero] * 3, zero)[0]
    V = om * (4.0 / 3.0) * math.pi * (d / 2) ** 3
    lhs, rhs = float(Vs @ phi), float(V @ ip)
    assert abs(lhs - rhs) <= 1e-13 * float(np.abs(Vs) @ np.abs(phi))


# ----------------------------------------------------------- node fields --

def test_node_fields_closed_forms():
    """Eq. 5 and u_g = U/eps_g at hand-computed solids fractions."""
    p = P(2, 2, 2, Ps=1.0, beta=2.0, eps_cp=0.6, alpha=1e-7, u_in=0.3)
    nn = oracle.nnode(p)
    # interior node (1,1,1) has the full cell volume 1e-6
    node = 1 + 3 * (1 + 3 * 1)
    for eps, tau_expect, ug_expect in ((0.0, 0.0, 0.3),
                                        (0.3, 0.3, 0.3 / 0.7),
                                        (0.5, 2.5, 0.6),
                                        (0.75, 0.5625 / 2.5e-8, 0.3 / 0.3)):
        Vs = np.zeros(nn)
        Vs[node] = eps * 1e-6
        es, ug, tau = oracle.node_fields(p, Vs)
        assert es[node] == pytest.approx(eps, rel=1e-15, abs=1e-18)
        assert tau[node] == pytest.approx(tau_expect, rel=1e-12)
        assert ug[2, node] == pytest.approx(ug_expect, rel=1e-12)
        assert ug[0, node] == 0.0
    # boundary corner node (0,0,0) has an eighth of the cell volume
    Vs = np.zeros(nn)
    Vs[0] = 0.3 * 1e-6 / 8
    es, _, _ = oracle.node_fields(p, Vs)
    assert es[0] == pytest.approx(0.3, rel=1e-14)


# -------------------------------------------------------------- drag/push --

def _terminal_velocity(d, rho_p, rho_g, mu, g, eps_g=1.0):
    """Continuous terminal velocity of Wen-Yu drag: D(u) u = g (1 - rho_g/rho_p), bisection."""
    target = g * (1 - rho_g / rho_p)

    def accel(u):
        rem = eps_g * rho_g * d * u / mu
        if rem < 1000:
            cd = 24 / rem * (1 + 0.15 * rem ** 0.687)
        else:
            cd = 0.44
        return 0.75 * cd * rho_g * u * u * eps_g ** -1.65 / (d * rho_p)

    lo, hi = 1e-9, 1e3
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if accel(mid) < target else (lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("d,ut_table", [(200e-6, 1.41999), (150e-6, 0.98773), (100e-6, 0.55319),
                                        (80e-6, 0.38821), (250e-6, 1.83716), (3e-3, None)])
def test_terminal_settling_velocity(d, ut_table):
    """One parcel in still gas with a hydrostatic gradient settles at the continuous
    terminal velocity: the fixed point of the semi-implicit update is D(u) u = g(1 - rho_g/rho_p)."""
    p = P(1, 1, 40, dx=1.0, dy=1.0, dz=1.0, rho_p=2500.0, Ps=0.0, u_in=0.0, dt=1e-2)
    ut = _terminal_velocity(d, 2500.0, 1.2, 1.8e-5, 9.81)
    if ut_table is not None:
        assert ut == pytest.approx(ut_table, abs=1.5e-5)
    else:   # Newton regime closed form
        assert ut == pytest.approx(math.sqrt(9.81 * (1 - 1.2 / 2500) * d * 2500 / (0.33 * 1.2)),
                                   rel=1e-9)
    if d >= 1e-3:   # fast, slowly relaxing parcel: a tall box and a longer step
        p.update(dz=20.0, dt=0.05)
    st = dict(x=np.array([0.5]), y=np.array([0.5]), z=np.array([p["dz"] * 39.5]),
              u=np.zeros(1), v=np.zeros(1), w=np.zeros(1), d=np.array([d]),
              omega=np.array([1e-9]))
    nsteps = 1500 if d < 1e-3 else 800
    s, ex, status = oracle.step(p, st, nsteps)
    assert status == 0
    assert -s["w"][0] == pytest.approx(ut, rel=1e-10)
    assert s["u"][0] == 0.0 and s["v"][0] == 0.0


def test_ballistic_closed_form():
    """Drag off (C = 0), no stress, no pressure gradient: x_n = x0 + n dt u0 + g dt^2 n(n+1)/2."""
    p = P(10, 10, 10, dx=0.1, dy=0.1, dz=0.1, drag_mult=0.0, Ps=0.0, gradp=(0.0, 0.0, 0.0),
          dt=1e-3)
    rng = np.random.default_rng(5)
    n = 50
    x0 = rng.uniform(0.3, 0.7, (n, 3))
    u0 = rng.uniform(-0.5, 0.5, (n, 3))
    st = dict(x=x0[:, 0], y=x0[:, 1], z=x0[:, 2], u=u0[:, 0], v=u0[:, 1], w=u0[:, 2],
              d=np.full(n, 1e-4), omega=np.ones(n))
    steps = 100
    s, _, status = oracle.step(p, st, steps)
    assert status == 0
    g = np.array([0.0, 0.0, -9.81])
    dt = 1e-3
    xe = x0 + steps * dt * u0 + g * dt * dt * steps * (steps + 1) / 2
    ue = u0 + steps * g * dt
    got_x = np.stack([s["x"], s["y"], s["z"]], 1)
    got_u = np.stack([s["u"], s["v"], s["w"]], 1)
    np.testing.assert_allclose(got_x, xe, rtol=0, atol=1e-13)
    np.testing.assert_allclose(got_u, ue, rtol=0, atol=1e-13)


def test_specular_reflection_mirror():
    """With e = 1 a parcel crossing x = 0 continues on the mirrored free trajectory."""
    p = P(10, 10, 10, dx=0.1, dy=0.1, dz=0.1, drag_mult=0.0, Ps=0.0, gradp=(0.0, 0.0, 0.0),
          g=(0.0, 0.0, 0.0), dt=1e-3, e_wall=1.0)
    st = dict(x=np.array([0.0105, 0.9905]), y=np.array([0.5, 0.5]), z=np.array([0.5, 0.5]),
              u=np.array([-1.0, 1.0]), v=np.zeros(2), w=np.zeros(2), d=np.full(2, 1e-4),
              omega=np.ones(2))
    s, _, status = oracle.step(p, st, 20)
    assert status == 0
    np.testing.assert_allclose(s["x"], [abs(0.0105 - 0.02), 1.0 - abs(0.9905 + 0.02 - 1.0)],
                               atol=1e-15)
    np.testing.assert_allclose(s["u"], [1.0, -1.0])
    # restitution e = 0.5 halves the normal velocity
    p["e_wall"] = 0.5
    s, _, _ = oracle.step(p, st, 20)
    np.testing.assert_allclose(s["u"], [0.5, -0.5])


def _balance_velocity(eps_g, d, rho_p, rho_g, mu, g):
    """Superficial U at which Wen-Yu drag on a uniform bed carries its buoyant weight."""
    target = g * (1 - rho_g / rho_p)

    def accel(U):
        s = U / eps_g
        rem = eps_g * rho_g * d * s / mu
        cd = 24 / rem * (1 + 0.15 * rem ** 0.687) if rem < 1000 else 0.44
        return 0.75 * cd * rho_g * s * s * eps_g ** -1.65 / (d * rho_p)

    lo, hi = 1e-9, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if accel(mid) < target else (lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("eps_g,U_table", [(0.4, 0.0911), (0.5, 0.1880), (0.6, 0.3312)])
def test_uniform_fluidisation_pressure_drop_equals_bed_weight(eps_g, U_table):
    """A uniform lattice bed at rest, fluidised at the balance velocity, has a drag-borne
    pressure drop equal to its buoyant weight (1 - eps_g)(rho_p - rho_g) g H."""
    d, rho_p = 200e-6, 2500.0
    U = _balance_velocity(eps_g, d, rho_p, 1.2, 1.8e-5, 9.81)
    assert U == pytest.approx(U_table, abs=6e-5)
    p = P(3, 3, 4, Ps=0.0, u_in=U, rho_p=rho_p, eps_g_min=0.05)
    x, y, z = _lattice(p, 2)
    vcell = 1e-6
    omega = (1 - eps_g) * vcell / 8 / (math.pi / 6 * d ** 3)
    st = dict(x=x, y=y, z=z, u=np.zeros_like(x), v=np.zeros_like(x), w=np.zeros_like(x),
              d=np.full(x.size, d), omega=np.full(x.size, omega))
    _, ex, status = oracle.step(p, st, 1)
    assert status == 0
    H = 4 * 0.01
    weight = (1 - eps_g) * (rho_p - 1.2) * 9.81 * H
    assert ex["obj"][0, 0] == pytest.approx(weight, rel=1e-12)
    assert ex["obj"][0, 1] == pytest.approx(H, rel=1e-13)     # H = 2 * mean height of a full box


def test_drag_sums_match_pressure_drop():
    """Partition of unity: sum over nodes of (A u_g - B)_z equals sum_p f_p s_z (= dP * area)."""
    bed = synth.settle_bed(n=4000, nx=8, ny=8, nz=16)
    synth.random_velocities(bed, 0.2, 11)
    p = bed.params
    _, ex, st = oracle.step(p, bed.parcels, 1)
    assert st == 0
    Vs, A, B = ex["Vs"], ex["A"], ex["B"]
    _, ug, _ = oracle.node_fields(p, Vs)
    # sum_n (A_n u_g,n - B_n) = sum_p f_p (sum_q W u_g,n - u_p) = sum_p f_p s_p
    lhs = float(np.sum(A * ug[2] - B[2]))
    area = p["nx"] * p["dx"] * p["ny"] * p["dy"]
    assert lhs == pytest.approx(ex["obj"][0, 0] * area, rel=1e-12)


# ---------------------------------------------------------------- tangent --

def test_tangent_matches_central_differences():
    """Oracle gradient (forward mode) of the time-averaged dP and H w.r.t. (C, s_d, u_in)
    against central finite differences with h = 1e-4 relative, in FP64."""
    rng = np.random.default_rng(7)
    p = P(8, 8, 16, u_in=0.4, dt=1e-4)
    n = 2000
    Lx, Ly, Lz = 0.08, 0.08, 0.16
    st = dict(x=rng.uniform(0.01, Lx - 0.01, n), y=rng.uniform(0.01, Ly - 0.01, n),
              z=rng.uniform(0.3 * Lz, 0.6 * Lz, n), u=0.05 * rng.standard_normal(n),
              v=0.05 * rng.standard_normal(n), w=0.05 * rng.standard_normal(n),
              d=np.full(n, 150e-6), omega=np.full(n, 200.0))
    steps = 10
    means, grads, status = oracle.step_tangent(p, st, steps)
    assert status == 0
    for k, name in enumerate(("drag_mult", "dscale", "u_in")):
        base = p[name]
        h = 1e-4 * base
        vals = []
        for sgn in (+1, -1):
            q = dict(p)
            q[name] = base + sgn * h
            _, ex, s2 = oracle.step(q, st, steps, outputs=False)
            assert s2 == 0
            vals.append(ex["obj"].mean(0))
        fd = (vals[0] - vals[1]) / (2 * h)
        for o in range(2):
            scale = max(abs(fd[o]), 1e-12 * abs(means[o]) / base)
            assert abs(grads[o, k] - fd[o]) <= 1e-5 * scale + 1e-10 * abs(means[o]) / base, \
                (name, o, grads[o, k], fd[o])
    _, ex, _ = oracle.step(p, st, steps, outputs=False)
    np.testing.assert_allclose(means, ex["obj"].mean(0), rtol=1e-14)


def test_step_sample_agrees_with_full_step():
    """The sampled-step routine computes, for the sampled parcels, exactly what the full
    step computes (it shares the step's functions; this pins the sampling bookkeeping)."""
    bed = synth.fourier_bed(n=3000, nx=8, ny=8, nz=16, nsteps=1)
    synth.random_velocities(bed, 0.2, seed=12)
    ref, ex, st = oracle.step(bed.params, bed.parcels, 1, U=bed.U)
    assert st == 0
    sample = np.array([0, 7, 123, 2999, 1500])
    out, cell, f, st2 = oracle.step_sample(bed.params, bed.parcels, sample, U=bed.U)
    assert st2 == 0
    for a, k in enumerate(("x", "y", "z", "u", "v", "w")):
        np.testing.assert_array_equal(out[a], ref[k][sample])
    np.testing.assert_array_equal(cell, ex["cell"][sample])


# ------------------------------------------------ branches pinned later on --

def test_interp_reproduces_a_linear_node_pressure_gradient():
    """The node pressure-gradient path of the interpolation: a linear grad p field given at
    the nodes is reproduced exactly at every parcel, each component on its own axis."""
    p = P(6, 5, 4, dx=0.02, dy=0.015, dz=0.01)
    rng = np.random.default_rng(21)
    L = np.array([6 * 0.02, 5 * 0.015, 4 * 0.01])
    pos = rng.uniform(0, 1, (400, 3)) * L
    X, Y, Z = _node_coords(p)
    zero = np.zeros_like(X)
    coef = np.array([[3.0, 1.0, -2.0, 0.5], [-7.0, 0.25, 4.0, -1.0], [11.0, -3.0, 0.0, 2.0]])
    gp = [c[0] + c[1] * X + c[2] * Y + c[3] * Z for c in coef]
    out = oracle.interp(p, pos[:, 0], pos[:, 1], pos[:, 2], zero, [zero] * 3, zero, gradp=gp)
    for a in range(3):
        expect = coef[a, 0] + pos @ coef[a, 1:]
        np.testing.assert_allclose(out[4 + a], expect, rtol=1e-13, atol=1e-13)


def test_drag_sums_partition_of_unity_every_component():
    """Every component of the drag sums: sum_n (A u_g,n - B_n)_a equals sum_p f_p s_p,a, with
    f_p and the slip s_p from the interpolation and drag functions (pinned above), for random
    parcel velocities in all three directions and a non-uniform gas field."""
    bed = synth.fourier_bed(n=4000, nx=8, ny=6, nz=12, nsteps=1)
    synth.random_velocities(bed, 0.3, 13)
    p = bed.params
    st = bed.parcels
    _, ex, status = oracle.step(p, st, 1, U=bed.U)
    assert status == 0
    Vs, A, B = ex["Vs"], ex["A"], ex["B"]
    es, ug, tau = oracle.node_fields(p, Vs, U=bed.U)
    I = oracle.interp(p, st["x"], st["y"], st["z"], es, ug, tau)
    D = oracle.drag(p, st["d"], I[0], I[1:4], st["u"], st["v"], st["w"])
    V = st["omega"] * math.pi / 6 * st["d"] ** 3
    f = p["rho_p"] * V * D
    for a, k in enumerate(("u", "v", "w")):
        lhs = float(np.sum(A * ug[a] - B[a]))
        rhs = float(np.sum(f * (I[1 + a] - st[k])))
        scale = float(np.sum(np.abs(f * (I[1 + a] - st[k]))))
        assert abs(lhs - rhs) <= 1e-12 * scale, (a, lhs, rhs)


def test_drag_voidage_floor_substitutes_eps_g_min():
    """Below eps_g_min the drag takes eps_g = eps_g_min: at eps_s = 0.8 and 0.95 (eps_g 0.2,
    0.05) it equals the drag at eps_s = 0.75 (eps_g = 0.25 = eps_g_min, exact in binary), and
    the unfloored drag at eps_g = 0.25 (a config whose floor is lower), for every drag law."""
    for model in range(4):
        p = P(2, 2, 2, eps_g_min=0.25, drag_model=model)
        q = dict(p, eps_g_min=0.01)
        n = 5
        d = np.full(n, 150e-6)
        ug = [np.zeros(n), np.zeros(n), np.linspace(0.1, 2.0, n)]
        zero = np.zeros(n)
        Dfloor = [oracle.drag(p, d, np.full(n, es), ug, zero, zero, zero) for es in (0.8, 0.95, 0.75)]
        Dref = oracle.drag(q, d, np.full(n, 0.75), ug, zero, zero, zero)
        np.testing.assert_array_equal(Dfloor[0], Dfloor[2])
        np.testing.assert_array_equal(Dfloor[1], Dfloor[2])
        np.testing.assert_array_equal(Dfloor[2], Dref)
        Dabove = oracle.drag(p, d, np.full(n, 0.5), ug, zero, zero, zero)
        assert np.all(Dabove != Dfloor[2])


# ------------------------------------------------------- other drag laws --

def _dallavalle_terminal_velocity(d, rho_p, rho_g, mu, g):
    """Single-particle terminal velocity with Dallavalle's drag coefficient
    C_D = (0.63 + 4.8 / sqrt(Re))^2: 3/4 C_D rho_g u^2 / (d rho_p) = g (1 - rho_g/rho_p)."""
    target = g * (1 - rho_g / rho_p)

    def accel(u):
        re = rho_g * d * u / mu
        cd = (0.63 + 4.8 / math.sqrt(re)) ** 2
        return 0.75 * cd * rho_g * u * u / (d * rho_p)

    lo, hi = 1e-9, 1e3
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if accel(mid) < target else (lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("d", [100e-6, 200e-6, 400e-6])
def test_syamlal_obrien_single_particle_settles_at_dallavalle_velocity(d):
    """In an unbounded dilute suspension (eps_g -> 1) the Syamlal-O'Brien velocity ratio is 1
    and the drag is Dallavalle's: one parcel in still gas settles at that terminal velocity."""
    dz = 1.0 if d < 300e-6 else 2.0      # room to settle for 15 s
    p = P(1, 1, 40, dx=1.0, dy=1.0, dz=dz, rho_p=2500.0, Ps=0.0, u_in=0.0, dt=1e-2,
          drag_model=1)
    ut = _dallavalle_terminal_velocity(d, 2500.0, 1.2, 1.8e-5, 9.81)
    st = dict(x=np.array([0.5]), y=np.array([0.5]), z=np.array([39.5 * dz]),
              u=np.zeros(1), v=np.zeros(1), w=np.zeros(1), d=np.array([d]),
              omega=np.array([1e-9]))
    s, _, status = oracle.step(p, st, 1500)
    assert status == 0
    assert -s["w"][0] == pytest.approx(ut, rel=1e-9)


@pytest.mark.parametrize("eps_g", [0.45, 0.7, 0.85, 0.9, 0.99])
def test_syamlal_obrien_creeping_and_inertial_limits(eps_g):
    """The velocity ratio V_r tends to A = eps_g^4.14 as Re -> 0 and to B (0.8 eps_g^1.28 up
    to eps_g = 0.85, eps_g^2.65 above) as Re -> infinity, so D tends to
    17.28 mu eps_g / (A d^2 rho_p) and to 0.297675 eps_g rho_g |s| / (B^2 d rho_p)."""
    p = P(2, 2, 2, drag_model=1, eps_g_min=0.05)
    d, mu, rho_g, rho_p = 1e-4, 1.8e-5, 1.2, 2500.0
    A = eps_g ** 4.14
    B = 0.8 * eps_g ** 1.28 if eps_g <= 0.85 else eps_g ** 2.65
    one = np.ones(1)
    zero = np.zeros(1)
    for slip, expect in ((1e-16, 17.28 * mu * eps_g / (A * d * d * rho_p)),
                         (1e18, 0.75 * 0.63 ** 2 * eps_g * rho_g * 1e18 / (B * B * d * rho_p))):
        D = oracle.drag(p, d * one, (1 - eps_g) * one, [zero, zero, slip * one], zero, zero, zero)
        assert D[0] == pytest.approx(expect, rel=2e-7), (slip, D[0], expect)


@pytest.mark.parametrize("eps_g,U", [(0.45, 0.05), (0.5, 0.2), (0.6, 0.4), (0.75, 0.8)])
def test_gidaspow_dense_bed_pressure_gradient_is_ergun(eps_g, U):
    """A uniform lattice bed at rest below a voidage of 0.8 under Gidaspow drag: with the
    steady, uniform gas momentum balance of Eq. 2 (0 = -eps_g grad p - F), the drag-borne
    pressure gradient dP / (eps_g H) is Ergun's equation
    150 mu U (1-eps)^2 / (eps^3 d^2) + 1.75 rho_g U^2 (1-eps) / (eps^3 d)."""
    d, rho_p, mu, rho_g = 200e-6, 2500.0, 1.8e-5, 1.2
    p = P(3, 3, 4, Ps=0.0, u_in=U, rho_p=rho_p, eps_g_min=0.05, drag_model=2)
    x, y, z = _lattice(p, 2)
    omega = (1 - eps_g) * 1e-6 / 8 / (math.pi / 6 * d ** 3)
    st = dict(x=x, y=y, z=z, u=np.zeros_like(x), v=np.zeros_like(x), w=np.zeros_like(x),
              d=np.full(x.size, d), omega=np.full(x.size, omega))
    _, ex, status = oracle.step(p, st, 1)
    assert status == 0
    H = 4 * 0.01
    ergun = (150 * mu * U * (1 - eps_g) ** 2 / (eps_g ** 3 * d * d)
             + 1.75 * rho_g * U * U * (1 - eps_g) / (eps_g ** 3 * d))
    assert ex["obj"][0, 0] / (eps_g * H) == pytest.approx(ergun, rel=1e-12)


def test_gidaspow_switch_and_blend():
    """Gidaspow takes Wen-Yu at and above eps_g = 0.8 and Ergun below; the blend weights the
    two equally at eps_s = 0.2 (phi = 1/2) and lies between them in the dense range."""
    n = 4
    d = np.full(n, 180e-6)
    ug = [np.zeros(n), np.full(n, 0.1), np.linspace(0.2, 1.5, n)]
    zero = np.zeros(n)
    q = {m: P(2, 2, 2, drag_model=m, eps_g_min=0.05) for m in range(4)}
    D = lambda m, es: oracle.drag(q[m], d, np.full(n, es), ug, zero, zero, zero)
    for es in (0.0, 0.1, 0.2):
        np.testing.assert_array_equal(D(2, es), D(0, es))
    for es in (0.2 + 1e-9, 0.3, 0.55):
        assert np.all(D(2, es) != D(0, es))
    ergun_at = D(2, 0.2 + 1e-12)              # the Ergun branch, continuous in eps_s
    np.testing.assert_allclose(D(3, 0.2), 0.5 * (ergun_at + D(0, 0.2)), rtol=1e-9)
    for es in (0.25, 0.4, 0.6):               # Gidaspow is Ergun here
        b = D(3, es)
        lo, hi = np.minimum(D(0, es), D(2, es)), np.maximum(D(0, es), D(2, es))
        assert np.all(b >= lo * (1 - 1e-12)) and np.all(b <= hi * (1 + 1e-12))


# ----------------------------------------------------- implicit coupling --

def _moving_lattice(p, vel, per_axis=2, d=200e-6, eps_s=0.3):
    x, y, z = _lattice(p, per_axis)
    omega = eps_s * p["dx"] * p["dy"] * p["dz"] / per_axis ** 3 / (math.pi / 6 * d ** 3)
    n = x.size
    return dict(x=x, y=y, z=z, u=np.full(n, vel[0]), v=np.full(n, vel[1]), w=np.full(n, vel[2]),
                d=np.full(n, d), omega=np.full(n, omega))


def test_implicit_coupling_limits():
    """The gas iteration of implicit coupling: with negligible gas inertia (dt -> infinity)
    one iteration drags the node gas velocity to the f-weighted mean parcel velocity, which
    for parcels all moving with v is v itself; with dt -> 0 the gas velocity stays U/eps_g;
    with no iteration (explicit coupling) the node fields are those of the deposit alone."""
    vel = (0.3, -0.2, 0.7)
    base = P(3, 4, 5, u_in=0.4, Ps=0.0, eps_g_min=0.05)
    st = _moving_lattice(base, vel)
    explicit = oracle.couple(dict(base, coupling_iters=0), st)
    es, ug0, _ = oracle.node_fields(base, explicit["Vs"])
    np.testing.assert_array_equal(explicit["ug"], ug0)
    assert np.all(explicit["A"] == 0) and np.all(explicit["B"] == 0)
    heavy = oracle.couple(dict(base, coupling_iters=1, dt=1e12), st)
    for a in range(3):
        np.testing.assert_allclose(heavy["ug"][a], vel[a], rtol=1e-9, atol=1e-12)
    light = oracle.couple(dict(base, coupling_iters=3, dt=1e-20), st)
    np.testing.assert_allclose(light["ug"], ug0, rtol=1e-9, atol=1e-12)


def test_implicit_coupling_uniform_bed_follows_the_scalar_recurrence():
    """A uniform lattice bed at rest (every node at the same eps_s, f uniform): each gas
    iteration is the scalar recurrence u' = m u0 / (m + rho_p eps_s D(u)) per unit volume,
    m = rho_g eps_g / dt, with D from the drag function; K iterations of the oracle equal
    K steps of the recurrence at every node, for every drag law."""
    for model in range(4):
        p = P(3, 3, 4, u_in=0.5, Ps=0.0, eps_g_min=0.05, dt=2e-3, drag_model=model)
        st = _moving_lattice(p, (0.0, 0.0, 0.0), eps_s=0.35)
        K = 4
        out = oracle.couple(dict(p, coupling_iters=K), st)
        es = 0.35
        eg = 1 - es
        u0 = 0.5 / eg
        m = p["rho_g"] * eg / p["dt"]
        u = u0
        one, zero = np.ones(1), np.zeros(1)
        for _ in range(K):
            D = oracle.drag(p, 200e-6 * one, es * one, [zero, zero, u * one], zero, zero, zero)[0]
            u = m * u0 / (m + p["rho_p"] * es * D)
        np.testing.assert_allclose(out["eps_s"], es, rtol=1e-12)
        np.testing.assert_allclose(out["ug"][2], u, rtol=1e-11)
        np.testing.assert_allclose(out["ug"][0], 0.0, atol=1e-15)


def test_multithreaded_driver_equals_the_oracle():
    """The all-core driver of the CPU baseline runs the oracle's own functions: on one thread
    it is the oracle bit for bit; on several threads it matches to rounding."""
    bed = synth.fourier_bed(n=5000, nx=8, ny=8, nz=16, nsteps=1)
    synth.random_velocities(bed, 0.2, seed=14)
    p = dict(bed.params, coupling_iters=2, drag_model=1)
    ref, ex, st = oracle.step(p, bed.parcels, 3, U=bed.U, outputs=False)
    one, obj1, st1 = oracle.step_mt(p, bed.parcels, 3, U=bed.U, nthreads=1)
    assert st == st1 == 0
    for k in ("x", "y", "z", "u", "v", "w"):
        np.testing.assert_array_equal(one[k], ref[k])
    np.testing.assert_array_equal(obj1, ex["obj"])
    four, obj4, st4 = oracle.step_mt(p, bed.parcels, 3, U=bed.U, nthreads=4)
    assert st4 == 0
    for k in ("x", "w"):
        np.testing.assert_allclose(four[k], ref[k], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(obj4, ex["obj"], rtol=1e-12)
