"""pic_diag_static, the diagnostic entry point that allocates no device memory.

Callers that cannot allocate while they run -- a device whose memory belongs
to a pool allocator, a real-time loop -- call pic_diag_static instead of
pic_diag, which allocates its charge-density scratch on first use.  The static variant keeps that
scratch in a file-scope device array shared by all calls, so each call must
clear it: two calls in a row must both agree with pic_diag.

This file is named to run last, so a failure here comes after every other
test has run.  It only needs the library (no oracle).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

D3 = (1e-6, 1.1e-6, 0.9e-6)


def _sim(nphys, pml, npart=400, steps=20):
    import torch
    from paper_2201_09084_gb300 import build as B
    from paper_2201_09084_gb300 import inputs as I
    from paper_2201_09084_gb300.api import Sim, pack_particles
    B.build()
    sim = Sim(3, nphys, D3, pml, cfl=0.95, order=3, prec="fp64", alpha_mode="damped")
    lo = [p + 4 for p in pml[::2]]
    hi = [p + n - 4 for p, n in zip(pml[::2], nphys)]
    parts = I.random_particles(3, npart, lo, hi, u_rms=0.3, seed=3)[0]
    pos, mom = pack_particles(parts["cell"], parts["off"], parts["u"], parts["w"], "fp64")
    sim.add_species(pos, mom, npart, parts["q"], parts["m"])
    pos2, mom2 = pack_particles(parts["cell"], parts["off"], 0 * parts["u"], parts["w"], "fp64")
    sim.add_species(pos2, mom2, npart, -parts["q"], parts["m"], immobile=True)
    sim.step(steps)
    torch.cuda.synchronize()
    return sim


def _static_diag(sim):
    from paper_2201_09084_gb300 import _lib as L
    g, r, e = C.c_double(), C.c_double(), C.c_double()
    rc = L.load().pic_diag_static(sim.ctx, C.byref(g), C.byref(r), C.byref(e))
    L.check(rc, sim.ctx)
    return dict(gauss=g.value, rho_scale=r.value, energy=e.value)


def test_static_diag_matches_pic_diag_on_two_calls():
    sim = _sim((24, 20, 28), (6,) * 6)
    ref = sim.diag()
    assert ref["rho_scale"] > 0 and ref["energy"] > 0
    for _ in range(2):
        got = _static_diag(sim)
        # FP64 atomics sum in a different order on each call
        assert got["rho_scale"] == pytest.approx(ref["rho_scale"], rel=1e-12)
        assert got["energy"] == pytest.approx(ref["energy"], rel=1e-12)
        assert abs(got["gauss"] - ref["gauss"]) <= 1e-12 * ref["rho_scale"]
    # the state moves on: both entry points follow it
    sim.step(5)
    ref2 = sim.diag()
    got2 = _static_diag(sim)
    assert got2["energy"] == pytest.approx(ref2["energy"], rel=1e-12)
    assert got2["rho_scale"] == pytest.approx(ref2["rho_scale"], rel=1e-12)


def test_static_diag_rejects_grids_beyond_its_scratch():
    from paper_2201_09084_gb300 import _lib as L
    sim = _sim((200, 200, 200), (6,) * 6, npart=16, steps=0)
    with pytest.raises(L.PicError) as ei:
        _static_diag(sim)
    assert ei.value.code == -1
    assert "static scratch" in str(ei.value)
