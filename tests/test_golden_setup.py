"""Golden setup counts printed in the paper (Sec. 3 and Sec. 4.1) against the generator."""
import os

import pytest

from paper_2211_15605_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_setup_counts.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = int(v)
    return out


def test_mesh_counts():
    g = _golden()
    assert (27 + 2) * (162 + 2) * (27 + 2) == g["verification_cells_total"]
    assert 150 * 150 * 450 == g["scaling_cells"]


def test_parcel_counts_from_bed_recipe():
    g = _golden()
    bed = 0.12 * 0.12 * 0.12
    n_ver = synth.parcel_count(1 - 0.42, bed, 400e-6, 10.0)
    assert n_ver == pytest.approx(g["verification_parcels"], rel=3e-3)
    n_scal = synth.parcel_count(1 - 0.42, bed, 200e-6, 5.0)
    assert n_scal == pytest.approx(g["scaling_parcels"], rel=1e-4)


def test_paper_verification_bed_matches_the_printed_setup():
    """The Sec. 3 bed as generated: the paper's parcel count, 400 um particles of 2000 kg/m3,
    statistical weight 10 (to the rounding of the count), a 12 cm bed at gas fraction 0.42 in
    a 12 x 72 x 12 cm box of 27 x 162 x 27 cells (vertical axis z here)."""
    import math
    import numpy as np
    g = _golden()
    b = synth.paper_verification_bed()
    p = b.params
    assert b.np == g["verification_parcels"]
    assert (p["nx"], p["ny"], p["nz"]) == (27, 27, 162)
    assert p["nz"] * p["dz"] == pytest.approx(0.72) and p["nx"] * p["dx"] == pytest.approx(0.12)
    assert np.all(b.parcels["d"] == 400e-6) and p["rho_p"] == 2000.0
    assert b.parcels["omega"][0] == pytest.approx(10.0, rel=3e-3)
    es = np.sum(b.parcels["omega"] * math.pi / 6 * b.parcels["d"] ** 3) / 0.12 ** 3
    assert es == pytest.approx(0.58, rel=1e-12)
    assert b.parcels["z"].max() < 0.12 and b.parcels["z"].min() > 0.0
