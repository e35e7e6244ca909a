"""Write grad_bed_tangent.json: the oracle's forward-mode gradient on the 500k-parcel
differentiation bed (32x32x128 cells, 200 steps), as drawn and lifted 2 cm off the floor.

Calls only the oracle and the seeded input generator; takes several minutes per bed on one
core. Run from the repository root: python tests/golden/make_grad_bed_tangent.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2211_15605_gb300 import synth  # noqa: E402

STEPS = 200


def main():
    out = {"steps": STEPS, "objectives": ["dP", "H"], "params": ["drag_mult", "dscale", "u_in"]}
    for name, bed in (("as_drawn", synth.grad_bed()), ("lifted_2cm", synth.grad_bed(floor_clearance=0.02))):
        t = time.time()
        means, grads, st = oracle.step_tangent(bed.params, bed.parcels, STEPS)
        assert st == 0, st
        out[name] = {"means": means.tolist(), "grads": grads.tolist(),
                     "seconds": round(time.time() - t, 1)}
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "grad_bed_tangent.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
