"""Write the oracle snapshots that the long GPU parity tests compare against.

    python tests/golden/make_oracle_fixtures.py            # all cases (about 25 min, 3 processes)
    python tests/golden/make_oracle_fixtures.py couette    # one case

The FP64 CPU oracle takes about 1.4 s per step on a 32^3 grid, too slow to
run 1000 steps inside a GPU test, so its states are computed once here and
stored.  This script calls only the oracle and the seeded input generators;
nothing in it comes from the CUDA path.  Every case runs in parity mode
(pressure tolerance 1e-13) from the workload's initial state; each file holds
phi, the face velocities and p at the listed step counts.

Cases:
  drop3d_32_noise   the 3D drop of the 256^3 workload at 32^3 (density and
                    viscosity ratio 10, theta_eq 60 deg, uniform noise 1e-3,
                    seed 12345), dt from stable_dt; steps 200 and 1000
  drop3d_32_smooth  the same without the noise; steps 200 and 1000
  couette_128x32    the two-phase Couette workload cut to 128x32 (walls at
                    -/+0.1, slip length dx, Ca 0.05); steps 1000
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
TOL = 1e-13


def cases():
    from paper_2412_16843_gb300 import inputs
    d_noise = inputs.drop_3d(32)
    d_smooth = inputs.drop_3d(32, noise=0.0)
    c = inputs.couette_2d(128, 32, 1.0)
    return {
        "drop3d_32_noise": (d_noise, inputs.stable_dt(d_noise), (200, 1000), None),
        "drop3d_32_smooth": (d_smooth, inputs.stable_dt(d_smooth), (200, 1000), None),
        "couette_128x32": (c, c.dt, (1000,), None),
    }


def path(name):
    return os.path.join(HERE, "oracle_%s.npz" % name)


def run(name):
    sys.path.insert(0, ROOT)
    import oracle
    wl, dt, marks, reg = cases()[name]
    o = oracle.from_workload(wl, tol=TOL)
    if reg is not None:
        o.set_regularisation(*reg)
    out = {"dt": dt, "tol": TOL, "steps": np.array(marks), "mass0": o.mass()}
    done = 0
    for m in marks:
        o.step(dt, m - done)
        done = m
        phi, vel, p = o.get_state()
        out["phi_%d" % m] = phi
        for a, v in enumerate(vel):
            out["u%d_%d" % (a, m)] = v
        out["p_%d" % m] = p
        out["mass_%d" % m] = o.mass()
    np.savez_compressed(path(name), **out)
    return name


def main(argv):
    sys.path.insert(0, ROOT)
    names = argv[1:] or list(cases())
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(names)) as pool:
        for n in pool.imap_unordered(run, names):
            print("wrote", path(n), flush=True)


if __name__ == "__main__":
    main(sys.argv)
