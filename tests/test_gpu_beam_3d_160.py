"""The 3D beam workload at its full size, in the launch configuration the
benchmark times, against the oracle on the whole grid.

128^3 physical cells + 16-cell PML on every face (160^3), 4,194,304
macroparticles in the relativistic beam (Gaussian, sigma 4 / 4 / 8 cells,
u ~ N(50, 0.5) along the beam axis, 1 nC) centred 24 cells before the +z
interface, damped-current PML, dt = 0.99 x Courant limit, FP32 fields with
IEEE FP64 PML split parts, sorted before the first step; the GPU uses the
launch shapes its autotuner picks (as the benchmark does).  Order-1 shapes at normal incidence for 100 steps (by then
the beam's head has crossed the damped PML and left through the outer
wall); order 1 at 15 degrees and order 3 at 0 and 30 degrees (the other
incidences and shape of the workload) for 20 steps.  After 10 steps and at
the end every field component on every node is compared with the FP64
oracle (combined field scale, FP32 tolerance), and the live particles'
positions as sets.  The oracle runs threaded (its loops split over the
host's cores).
"""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, max_field_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("order,theta,steps", [(1, 0.0, 100), (1, 15.0, 20), (3, 0.0, 20), (3, 30.0, 20)],
                         ids=["o1-0deg-100", "o1-15deg-20", "o3-0deg-20", "o3-30deg-20"])
def test_beam_3d_160_full_size(order, theta, steps):
    import torch
    import bench
    from paper_2201_09084_gb300.api import Sim, pack_particles
    parts = I.beam(3, bench.NPART, bench.NPHYS, bench.PML, bench.beam_center(), theta_deg=theta)[0]
    dt = O.yee_dt(bench.D, 0.99, 3)
    gpu = Sim(3, bench.NPHYS, bench.D, bench.PML, dt=dt, order=order, prec="fp32", alpha_mode="damped",
              split_fp64=True)
    pos, mom = pack_particles(parts["cell"], parts["off"], parts["u"], parts["w"], "fp32")
    gpu.add_species(pos, mom, bench.NPART, parts["q"], parts["m"])
    gpu.sort()
    tuning = gpu.autotune(steps=2)
    ora = O.OracleSim(3, bench.NPHYS, bench.PML, bench.D, dt, order=order, alpha_mode="damped")
    X = I.absolute(parts["cell"], parts["off"])
    u = parts["u"].astype(np.float64)
    assert ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2],
                             parts["w"].astype(np.float64), parts["q"], parts["m"], False) == 0
    O.set_threads(None)
    try:
        gpu.step(10)
        ora.step(10)
        torch.cuda.synchronize()
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL["fp32"], (10, err, tuning)
        gpu.step(steps - 10)
        ora.step(steps - 10)
        torch.cuda.synchronize()
    finally:
        O.set_threads(1)
    err = max_field_err(ora, gpu)
    assert max(err.values()) < TOL["fp32"], (steps, err, tuning)
    # the live particles agree as sets (the GPU reorders them when sorting):
    # per axis, the sorted coordinates differ by at most the largest
    # per-particle difference (sorting is 1-Lipschitz in the max norm)
    pg = gpu.particles(0)
    po = ora.particles()
    assert int(pg["alive"].sum()) == int(po["alive"].sum())
    Xg = (pg["cell"] + pg["off"].astype(np.float64))[pg["alive"]]
    Xo = np.stack([po["X"], po["Y"], po["Z"]], 1)[po["alive"]]
    for a in range(3):
        assert np.abs(np.sort(Xg[:, a]) - np.sort(Xo[:, a])).max() < 1e-5
    if steps >= 100:
        assert int(po["alive"].sum()) < bench.NPART, "part of the beam has left through the PML"
    print(f"\nfull-size beam, order {order}, {theta} deg, {steps} steps, tuning {tuning}: max rel field error "
          f"{max(err.values()):.3e}, {int(po['alive'].sum())} of {bench.NPART} particles left")
