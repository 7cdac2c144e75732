"""Zeroed-field (perfect conductor) cells on the GPU (pic_set_conductor)
against the oracle's (OracleSim.set_conductor), and the cavity run of
Sec. III in small.

A pillbox cavity on a beam pipe is carved out of a box with damped-current
PMLs on its z faces only (conducting x and y walls).  The field of a pulse
started in the cavity, and then the field of a relativistic proton beam
injected continuously inside the undamped entry face's PML and leaving
through the damped exit face (the paper's suggestion for this run, Sec. III),
agree with the oracle within the tolerance of each form.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, make_pair, max_field_err

pytestmark = pytest.mark.gpu

D = (1e-3, 1e-3, 1e-3)
NPHYS = (20, 18, 30)
PML = (0, 0, 0, 0, 6, 6)


def _mask():
    return I.cavity_mask(NPHYS, PML, pipe_radius=4, cavity_radius=8, cavity_z=(10, 20))


@pytest.mark.parametrize("solver", ["yee", "ck"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_conductor_cavity_pulse_matches_oracle(prec, solver):
    ora, gpu = make_pair(3, NPHYS, PML, D, [], prec=prec, solver=solver, delta=10.0)
    m = _mask()
    ora.set_conductor(m)
    gpu.set_conductor(m)
    nx, ny, nz = ora.nn
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = 1e5 * np.exp(-(((i - nx / 2) / 3.0) ** 2 + ((j - ny / 2) / 3.0) ** 2 + ((k - nz / 2) / 4.0) ** 2))
    for s in (ora, gpu):
        s.set_field("Ex", f)
        s.set_field("Ez", 0.5 * np.roll(f, 2, axis=2))
    for _ in range(3):
        ora.step(20)
        gpu.step(20)
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL[prec], err
    # nothing inside the conductor: an E node surrounded by conductor cells on all sides stays zero
    ex = gpu.field("Ex").cpu().numpy()
    assert np.abs(ex[m.shape[0] // 2, 1, 1]) == 0.0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cavity_injected_beam_matches_oracle(prec):
    import torch
    from paper_2201_09084_gb300.api import pack_particles
    faces = ["damped", "damped", "damped", "damped", "one", "damped"]
    ora, gpu = make_pair(3, NPHYS, PML, D, [], prec=prec, alpha_mode="damped", face_alpha=faces, delta=10.0,
                         cfl=0.99)
    m = _mask()
    ora.set_conductor(m)
    gpu.set_conductor(m)
    shift = O.C_LIGHT * gpu.dt / D[2] * np.sqrt(1 - 1 / 479.0 ** 2)
    nsl, per = 24, 40
    b = I.cavity_beam_slices(NPHYS, PML, nsl, per, shift, sigma=1.2, charge=40e-9 * (nsl * per) / 2e5)
    cap = nsl * per
    pos0, mom0 = pack_particles(np.zeros((cap, 3), np.int64), np.zeros((cap, 3), np.float32),
                                np.zeros((cap, 3), np.float32), np.zeros(cap, np.float32), prec)
    sid = gpu.add_species(pos0, mom0, 0, O.Q_E, O.M_P)
    pos, mom = pack_particles(b["cell"], b["off"], b["u"], b["w"], prec)
    Xa = I.absolute(b["cell"], b["off"])
    ua = b["u"].astype(np.float64)
    for st in range(40):
        if st < nsl:
            sl = slice(st * per, (st + 1) * per)
            gpu.inject(sid, pos[sl], mom[sl])
            assert ora.add_particles(Xa[sl, 0], Xa[sl, 1], Xa[sl, 2], ua[sl, 0], ua[sl, 1], ua[sl, 2],
                                     b["w"][sl].astype(np.float64), O.Q_E, O.M_P) == 0
        ora.step(1)
        gpu.step(1)
    torch.cuda.synchronize()
    gpu.sync()
    err = max_field_err(ora, gpu)
    print(f"\ncavity + injected beam ({prec}): max rel field error {max(err.values()):.3e}")
    assert max(err.values()) < TOL[prec], err
