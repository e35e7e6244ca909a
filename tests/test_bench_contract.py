"""Host-side logic of bench.py (CPU): the timed window it reports and the bed sample its
reference arm times."""
import argparse

import numpy as np

import bench
from paper_2211_15605_gb300 import synth


def _args(steps, warmup=3, run_steps=500):
    return argparse.Namespace(steps=steps, warmup=warmup, run_steps=run_steps)


def test_default_window_is_the_whole_run():
    a = _args(500)
    assert bench.settle_steps(a) == 0
    t0 = bench.settle_steps(a) + a.warmup
    assert (t0, t0 + a.steps) == (3, 503)


def test_short_window_is_centred_in_the_run():
    for steps in (10, 20, 50, 100, 250):
        a = _args(steps)
        t0 = bench.settle_steps(a) + a.warmup
        mid = t0 + steps / 2
        assert abs(mid - 250) <= 1, (steps, t0)
        assert t0 >= a.warmup


def test_window_never_settles_negatively():
    a = _args(600, warmup=10)
    assert bench.settle_steps(a) == 0


def test_run_lengths_cover_every_workload():
    for w in ("dense", "fourier", "settle", "grad", "batched", "paper_sec3", "paper_sec4"):
        assert bench.RUN_STEPS[w] > 0


def test_reference_sample_is_a_column_of_the_bed():
    bed = synth.fourier_bed(n=20_000, nx=12, ny=10, nz=16, nsteps=1)
    col = bench.sub_column(bed, 5)
    p, q = bed.params, col.params
    assert (q["nx"], q["ny"], q["nz"]) == (5, 5, p["nz"])
    assert q["dx"] == p["dx"] and q["dz"] == p["dz"]
    # exactly the parcels inside the column, in their order
    keep = (bed.parcels["x"] < 5 * p["dx"]) & (bed.parcels["y"] < 5 * p["dy"])
    assert col.np == int(keep.sum()) > 0
    for k in bed.parcels:
        np.testing.assert_array_equal(col.parcels[k], bed.parcels[k][keep])
    # the gas fields on the column's nodes
    for a in range(3):
        full = np.asarray(bed.U[a]).reshape(p["nz"] + 1, p["ny"] + 1, p["nx"] + 1)
        sub = np.asarray(col.U[a]).reshape(q["nz"] + 1, q["ny"] + 1, q["nx"] + 1)
        np.testing.assert_array_equal(sub, full[:, :6, :6])


def test_reference_sample_clamps_to_the_grid():
    bed = synth.settle_bed(n=2_000, nx=4, ny=3, nz=8)
    col = bench.sub_column(bed, 50)
    assert (col.params["nx"], col.params["ny"]) == (4, 3)
    assert col.np == bed.np


def test_cpu_baseline_reports_single_thread_and_all_cores():
    """The CPU leg times the oracle single-threaded and on every core, on columns of the bed,
    and states the host's CPU model and core count."""
    bed = synth.fourier_bed(n=40_000, nx=16, ny=16, nz=24, nsteps=1)
    cpu = bench.cpu_baseline(bed, seconds=0.6, steps=2)
    assert cpu["kind"] == "oracle" and cpu["nproc"] >= 1 and cpu["cpu_model"]
    st, mt = cpu["legs"]["single_thread"], cpu["legs"]["all_cores"]
    assert st["cores"] == 1 and st["value"] > 0
    assert mt["cores"] >= 1 and mt["value"] > 0
    assert cpu["value"] == mt["value"] and cpu["cores"] == mt["cores"]
