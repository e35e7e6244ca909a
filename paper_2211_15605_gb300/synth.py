"""Seeded synthetic inputs for the MP-PIC coupling step.

This module only draws inputs: parcel positions, velocities, diameters and
statistical weights, and prescribed gas fields at the mesh nodes. It holds no
step arithmetic (no binning, weights, drag or push), so both the CUDA path and
the CPU oracle can consume what it returns without sharing method code.

The beds mimic the fluidised-bed workloads of Woo et al. (arXiv 2211.15605):
a walled box with gravity along -z, parcels filling the lower part, uniform or
smoothly varying upward gas flow (Sec. 3 and Sec. 4 describe the paper's own
beds; their data is not published, so these are stand-ins with the same kind of
shapes, densities and flow rates).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2211_15605

# Air-like gas, glass-bead-like solids; Snider stress constants of the workloads.
_BASE = dict(
    dx=0.01, dy=0.01, dz=0.01,
    rho_g=1.2, mu_g=1.8e-5,
    g=(0.0, 0.0, -9.81),
    rho_p=2500.0,
    Ps=1.0, beta=2.0, eps_cp=0.6, alpha=1e-7,
    eps_g_min=0.3, e_wall=1.0,
    drag_mult=1.0, dscale=1.0,
    dt=1e-4,
    drag_model=0,          # 0 Wen-Yu, 1 Syamlal-O'Brien, 2 Gidaspow, 3 Gidaspow blend
    coupling_iters=0,      # 0 explicit coupling; K > 0 implicit with K gas iterations
)


def hydrostatic(rho_g, g):
    """Hydrostatic pressure gradient rho_g * g for a gas at rest."""
    return tuple(rho_g * gi for gi in g)


@dataclass
class Bed:
    """One synthetic bed: physical parameters, parcel SoA (float64) and gas fields."""
    params: dict
    parcels: dict
    U: tuple = (None, None, None)      # superficial gas velocity at nodes (before u_in)
    gradp: tuple | None = None         # node pressure gradient; None = uniform
    nsteps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def np(self) -> int:
        return int(self.parcels["x"].size)


def make_params(nx, ny, nz, **over) -> dict:
    p = dict(_BASE)
    p.update(nx=int(nx), ny=int(ny), nz=int(nz))
    p.update(over)
    if "gradp" not in over:
        p["gradp"] = hydrostatic(p["rho_g"], p["g"])
    p.setdefault("u_in", 0.0)
    return p


def _lognormal_d(rng, n, median, sigma):
    z = np.clip(rng.standard_normal(n), -4.0, 4.0)
    return median * np.exp(sigma * z)


def _uniform_positions(rng, n, p, zfrac_lo, zfrac_hi):
    Lx, Ly, Lz = p["nx"] * p["dx"], p["ny"] * p["dy"], p["nz"] * p["dz"]
    x = rng.uniform(0.0, Lx, n)
    y = rng.uniform(0.0, Ly, n)
    z = rng.uniform(zfrac_lo * Lz, zfrac_hi * Lz, n)
    return x, y, z


def fourier_gas(rng, p, mean_w, amp=0.1, modes=3):
    """Smooth random superficial velocity: (0,0,mean_w) + sum_m amp a_m sin(2 pi k_m.x/L + phi_m).

    a_m is a random unit vector, k_m has random integer components in {1,2,3},
    phi_m ~ U[0, 2 pi). Returned as three node arrays and the mean put in u_in.
    """
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    xs = np.arange(nx + 1) * p["dx"] / (nx * p["dx"])
    ys = np.arange(ny + 1) * p["dy"] / (ny * p["dy"])
    zs = np.arange(nz + 1) * p["dz"] / (nz * p["dz"])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")   # node index i fastest
    U = [np.zeros_like(X) for _ in range(3)]
    for _ in range(modes):
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        k = rng.integers(1, 4, size=3)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        s = np.sin(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + phi)
        for c in range(3):
            U[c] += amp * a[c] * s
    return tuple(np.ascontiguousarray(u.reshape(-1)) for u in U), float(mean_w)


def settle_bed(n=20_000, nx=16, ny=16, nz=32, seed=SEED_BASE + 1) -> Bed:
    """Dilute settling cloud: 200 um, 2500 kg/m3, w = 10 parcels uniform in the lower
    half of a 16x16x32 box of 1 cm cells, upward superficial gas 0.3 m/s, dt 1e-4, 100 steps."""
    rng = np.random.default_rng(seed)
    p = make_params(nx, ny, nz, u_in=0.3)
    x, y, z = _uniform_positions(rng, n, p, 0.0, 0.5)
    zeros = np.zeros(n)
    parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(),
                   d=np.full(n, 200e-6), omega=np.full(n, 10.0))
    return Bed(p, parcels, nsteps=100, meta=dict(workload="settle_16x16x32"))


def fourier_bed(n=4_000_000, nx=64, ny=64, nz=256, seed=SEED_BASE + 2, nsteps=1000) -> Bed:
    """Polydisperse bed in a smooth random gas field: lognormal d (median 150 um, sigma 0.3),
    w ~ U[5, 20], parcels uniform in the lower half; gas 0.5 m/s mean plus three 0.1 m/s modes."""
    rng = np.random.default_rng(seed)
    p = make_params(nx, ny, nz)
    x, y, z = _uniform_positions(rng, n, p, 0.0, 0.5)
    zeros = np.zeros(n)
    parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(),
                   d=_lognormal_d(rng, n, 150e-6, 0.3), omega=rng.uniform(5.0, 20.0, n))
    U, mean = fourier_gas(rng, p, 0.5)
    p["u_in"] = mean
    return Bed(p, parcels, U=U, nsteps=nsteps, meta=dict(workload=f"fourier_{nx}x{ny}x{nz}"))


def dense_bed(n=32_000_000, nx=128, ny=128, nz=512, seed=SEED_BASE + 3, eps_s=0.5,
              zfrac=0.25, nsteps=500, jitter=0.25) -> Bed:
    """Dense bottom bed at mean solids fraction eps_s in z < zfrac*Lz; inflow 0.8 m/s.

    Diameters are lognormal (median 100 um, sigma 0.4). Each parcel's statistical weight is
    chosen so that all parcels have the same volume, and parcels sit one per randomly chosen
    sub-cell of a 2x2x4 split of every bed cell, at the sub-cell centre jittered by up to
    +-jitter of its size (a jittered lattice, as MP-PIC beds are usually seeded). Uniform
    random placement at 0.5 would leave cloud-in-cell noise of about +-0.05 in the node
    solids fraction, i.e. nodes above close packing where the Eq. 5 stress explodes."""
    rng = np.random.default_rng(seed)
    # alpha = 0.01: with 1e-7 the explicit stress update diverges as soon as clustering lifts a
    # node above eps_cp (tau ~ 1e7 Pa); 0.01 bounds tau there and leaves it unchanged below.
    p = make_params(nx, ny, nz, u_in=0.8, alpha=0.01)
    kz = max(1, int(round(zfrac * nz)))
    sub = (2, 2, 4)
    nsub = nx * sub[0] * ny * sub[1] * kz * sub[2]
    if n > nsub:
        raise ValueError(f"{n} parcels do not fit {nsub} sub-cells")
    pick = rng.choice(nsub, size=n, replace=False)
    hx, hy, hz = p["dx"] / sub[0], p["dy"] / sub[1], p["dz"] / sub[2]
    ix = pick % (nx * sub[0])
    r = pick // (nx * sub[0])
    iy = r % (ny * sub[1])
    iz = r // (ny * sub[1])
    x = (ix + 0.5 + jitter * rng.uniform(-1.0, 1.0, n)) * hx
    y = (iy + 0.5 + jitter * rng.uniform(-1.0, 1.0, n)) * hy
    z = (iz + 0.5 + jitter * rng.uniform(-1.0, 1.0, n)) * hz
    d = _lognormal_d(rng, n, 100e-6, 0.4)
    bed_volume = (nx * p["dx"]) * (ny * p["dy"]) * (kz * p["dz"])
    vpar = eps_s * bed_volume / n                       # common parcel volume
    omega = vpar / (math.pi / 6.0 * d ** 3)
    zeros = np.zeros(n)
    parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(), d=d, omega=omega)
    return Bed(p, parcels, nsteps=nsteps, meta=dict(workload=f"dense_{nx}x{ny}x{nz}"))


def _lattice_fill(rng, n, p, kz, sub, jitter):
    """n parcel positions, one per randomly chosen sub-cell of a sub[0] x sub[1] x sub[2] split
    of every cell in the bottom kz layers, at the sub-cell centre jittered by up to +-jitter
    of its size (a jittered lattice, as MP-PIC beds are usually seeded)."""
    nx, ny = p["nx"], p["ny"]
    nsub = nx * sub[0] * ny * sub[1] * kz * sub[2]
    if n > nsub:
        raise ValueError(f"{n} parcels do not fit {nsub} sub-cells")
    pick = rng.choice(nsub, size=n, replace=False)
    hx, hy, hz = p["dx"] / sub[0], p["dy"] / sub[1], p["dz"] / sub[2]
    ix = pick % (nx * sub[0])
    r = pick // (nx * sub[0])
    iy = r % (ny * sub[1])
    iz = r // (ny * sub[1])
    x = (ix + 0.5 + jitter * rng.uniform(-1.0, 1.0, n)) * hx
    y = (iy + 0.5 + jitter * rng.uniform(-1.0, 1.0, n)) * hy
    z = (iz + 0.5 + jitter * rng.uniform(-1.0, 1.0, n)) * hz
    return x, y, z


def paper_verification_bed(n=2_983_447, seed=SEED_BASE + 6, u_in=0.5, nsteps=500) -> Bed:
    """The shape of the paper's verification bed (Sec. 3): a 12 x 72 x 12 cm box of 27 x 162 x
    27 cells (4.44 mm), gas of 1.093 kg/m3 and 1.9e-5 Pa s, 400 um particles of 2000 kg/m3,
    statistical weight 10, an initial bed 12 cm tall at a gas fraction of 0.42 (2,983,447
    parcels, the paper's count), inlet velocity in the paper's 0.3-1.0 m/s range. The paper's
    vertical axis (y) is z here, so the grid is 27 x 27 x 162 with gravity along -z. The
    parcels fill the bed as a jittered lattice (one per chosen sub-cell of a 6x6x6 split of
    each bed cell), all with the paper's diameter and the common volume that gives the bed's
    solids fraction (statistical weight 10.03). The paper does not state the Snider constants:
    Ps = 1 Pa, beta = 2, eps_cp = 0.6, alpha = 0.01 as for the dense bed."""
    rng = np.random.default_rng(seed)
    h = 0.12 / 27
    p = make_params(27, 27, 162, dx=h, dy=h, dz=h, rho_g=1.093, mu_g=1.9e-5, rho_p=2000.0,
                    u_in=u_in, alpha=0.01)
    kz = 27                                        # 12 cm of 4.44 mm cells
    x, y, z = _lattice_fill(rng, n, p, kz, (6, 6, 6), 0.25)
    d = np.full(n, 400e-6)
    vpar = 0.58 * (27 * h) * (27 * h) * (kz * h) / n
    omega = np.full(n, vpar / (math.pi / 6.0 * 400e-6 ** 3))
    zeros = np.zeros(n)
    parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(), d=d, omega=omega)
    return Bed(p, parcels, nsteps=nsteps, meta=dict(workload="paper_sec3_27x27x162"))


def paper_scaling_bed(n=47_853_435, seed=SEED_BASE + 7, nsteps=500) -> Bed:
    """The shape of the paper's strong-scaling bed (Sec. 4, 4.1): a 12 x 12 x 36 cm box of 150
    x 150 x 450 cells (0.8 mm), gravity along -z, gas of 1.0 kg/m3 and 1.8e-5 Pa s, 200 um
    particles of 2000 kg/m3, an initial bed 12 cm tall (150 layers) at a gas fraction of 0.42,
    inlet velocity 0.15 m/s, 47,853,435 parcels (the paper's count; statistical weight 5).
    Jittered lattice seeding (2x2x4 sub-cells per bed cell, 89% filled); Snider constants as
    for the dense bed."""
    rng = np.random.default_rng(seed)
    h = 0.0008
    p = make_params(150, 150, 450, dx=h, dy=h, dz=h, rho_g=1.0, mu_g=1.8e-5, rho_p=2000.0,
                    u_in=0.15, alpha=0.01)
    kz = 150
    x, y, z = _lattice_fill(rng, n, p, kz, (2, 2, 4), 0.25)
    d = np.full(n, 200e-6)
    vpar = 0.58 * (150 * h) * (150 * h) * (kz * h) / n
    omega = np.full(n, vpar / (math.pi / 6.0 * 200e-6 ** 3))
    zeros = np.zeros(n)
    parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(), d=d, omega=omega)
    return Bed(p, parcels, nsteps=nsteps, meta=dict(workload="paper_sec4_150x150x450"))


def grad_bed(n=500_000, nx=32, ny=32, nz=128, seed=SEED_BASE + 5, nsteps=200,
             floor_clearance=0.0) -> Bed:
    """Differentiation bed: d = 150 um, 2500 kg/m3, w = 10, lower-half fill, inflow 0.4 m/s.

    floor_clearance > 0 maps the fill's z range [0, Lz/2] affinely onto
    [floor_clearance, Lz/2] (same draws), so that no parcel reaches the floor early on."""
    rng = np.random.default_rng(seed)
    p = make_params(nx, ny, nz, u_in=0.4)
    x, y, z = _uniform_positions(rng, n, p, 0.0, 0.5)
    if floor_clearance > 0.0:
        half = 0.5 * nz * p["dz"]
        z = floor_clearance + z * (half - floor_clearance) / half
    zeros = np.zeros(n)
    parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(),
                   d=np.full(n, 150e-6), omega=np.full(n, 10.0))
    return Bed(p, parcels, nsteps=nsteps, meta=dict(workload=f"grad_{nx}x{ny}x{nz}"))


def batched_beds(nbeds=256, seed=SEED_BASE + 4, np_lo=5_000, np_hi=200_000, nsteps=200):
    """Many independent beds of uneven size: grids uniform in 8..32 x 8..32 x 16..64,
    parcel counts log-uniform in [np_lo, np_hi], inflow U[0.2, 1.0], median d U[80, 250] um."""
    rng = np.random.default_rng(seed)
    beds = []
    for _ in range(nbeds):
        nx, ny = int(rng.integers(8, 33)), int(rng.integers(8, 33))
        nz = int(rng.integers(16, 65))
        n = int(round(math.exp(rng.uniform(math.log(np_lo), math.log(np_hi)))))
        uin = float(rng.uniform(0.2, 1.0))
        dmed = float(rng.uniform(80e-6, 250e-6))
        p = make_params(nx, ny, nz, u_in=uin)
        x, y, z = _uniform_positions(rng, n, p, 0.0, 0.5)
        zeros = np.zeros(n)
        parcels = dict(x=x, y=y, z=z, u=zeros.copy(), v=zeros.copy(), w=zeros.copy(),
                       d=_lognormal_d(rng, n, dmed, 0.3), omega=np.full(n, 10.0))
        beds.append(Bed(p, parcels, nsteps=nsteps, meta=dict(workload="batched")))
    return beds


def random_velocities(bed: Bed, scale: float, seed: int) -> Bed:
    """Give every parcel a Gaussian velocity of the given scale (for single-step parity)."""
    rng = np.random.default_rng(seed)
    for k in ("u", "v", "w"):
        bed.parcels[k] = scale * rng.standard_normal(bed.np)
    return bed


def parcel_count(eps_s: float, bed_volume: float, d: float, omega: float) -> float:
    """Parcels needed to fill a bed volume at solids fraction eps_s with parcels of
    omega spheres of diameter d (the setup arithmetic of the paper's Sec. 3 bed)."""
    return eps_s * bed_volume / (omega * math.pi / 6.0 * d ** 3)
