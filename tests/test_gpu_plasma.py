"""Plasma + drifting beam (the precision-study workload, reduced to a size
the oracle steps in seconds): a neutral electron-proton plasma, 8
macroparticles per cell and species with Maxwellian u_th = 0.01 and Debye
length = cell size, plus an electron beam at u_z = 5 heading for the +z PML
(neutralised at t = 0 by immobile ions, so Gauss's law holds from the start),
damped-current PML of 8 cells on every face, order 1, all stages and the sort
every 5 steps.

The plasma is chaotic, so the FP32 gate holds for the first 20 steps (after
that FP32 and FP64 trajectories separate physically).  Checked against the
oracle after 10 and 20 steps: the relative field error of FP32 (float-float
PML parts), FP32 with int64 deterministic deposition, and FP64; and the
Gauss-law residual of the FP64 path relative to max |rho/eps0|.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, max_field_err

pytestmark = pytest.mark.gpu

D = (1e-6, 1e-6, 1e-6)
NPHYS = (24, 24, 48)
PML = (8,) * 6


def _parts():
    return I.plasma(NPHYS, PML, D[0], beam_radius=4.0, beam_length=12.0)


@pytest.fixture(scope="module")
def oracle_fields():
    dt = O.yee_dt(D, 0.99, 3)
    ora = O.OracleSim(3, NPHYS, PML, D, dt, order=1, alpha_mode="damped")
    for sp in _parts():
        X = I.absolute(sp["cell"], sp["off"])
        u = sp["u"].astype(np.float64)
        assert ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2],
                                 sp["w"].astype(np.float64), sp["q"], sp["m"], sp["immobile"]) == 0
    out = {}
    for n in (10, 20):
        ora.step(10)
        out[n] = {k: ora.field(k) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    return out, dt


class _Frozen:
    def __init__(self, f):
        self.f = f

    def field(self, k):
        return self.f[k]


@pytest.mark.parametrize("prec", ["fp32", "fixed64", "fp64"])
def test_plasma_beam_first_20_steps(prec, oracle_fields):
    from paper_2201_09084_gb300.api import Sim, pack_particles
    ref, dt = oracle_fields
    gpu = Sim(3, NPHYS, D, PML, dt=dt, order=1, prec=prec, alpha_mode="damped", sort_every=5)
    keep = []
    for sp in _parts():
        pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], prec)
        gpu.add_species(pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"])
        keep.append((pos, mom))
    for n in (10, 20):
        gpu.step(10)
        err = max_field_err(_Frozen(ref[n]), gpu)
        assert max(err.values()) < TOL[prec], (n, err)
    dg = gpu.diag()
    assert dg["rho_scale"] > 0
    if prec == "fp64":
        assert dg["gauss"] <= 1e-10 * dg["rho_scale"], dg
    print(f"\n{prec}: max rel field error after 20 steps {max(err.values()):.3e}, "
          f"Gauss residual {dg['gauss'] / dg['rho_scale']:.3e} of max|rho/eps0|")
