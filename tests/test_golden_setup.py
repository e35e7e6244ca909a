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
