"""Failure detection on the GPU, with the failures made on the host: bad
particle records (NaN momentum, infinite weight, a cell outside the allowed
cells) are removed before they touch the fields and reported at pic_sync; a
fixed-point weight beyond the accumulator's range is reported; a checkpoint
resumes bit-identically in deterministic mode.  Nothing here faults, traps or
hangs the GPU."""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, make_pair, max_field_err, gpu_positions

pytestmark = pytest.mark.gpu

D3 = (1e-6, 1.1e-6, 0.9e-6)
PIC_EPARTICLE = -9
PIC_EOVERFLOW = -5


def _parts(n, seed):
    return I.random_particles(3, n, [6, 6, 6], [14, 14, 16], u_rms=1.0, seed=seed)[0]


@pytest.mark.parametrize("ppt", [1, 4])
@pytest.mark.parametrize("what", ["nan_u", "inf_w", "cell"])
def test_bad_record_is_removed_and_reported(what, ppt):
    """One bad record among ordinary ones: the run's fields equal the oracle's
    without that particle, it is marked removed, and pic_sync reports it."""
    from paper_2201_09084_gb300 import _lib as L
    from paper_2201_09084_gb300.api import pack_particles
    nphys, pml = (10, 10, 12), (4,) * 6
    good = _parts(200, 7)
    ora, gpu = make_pair(3, nphys, pml, D3, [good], order=1, prec="fp32", alpha_mode="damped")
    gpu.set_tuning(ppt, 1)
    # the GPU species gets one more record, the bad one, in the middle
    cell = np.concatenate([good["cell"][:100], [[10, 10, 10]], good["cell"][100:]])
    off = np.concatenate([good["off"][:100], [[0.5, 0.5, 0.5]], good["off"][100:]]).astype(np.float32)
    u = np.concatenate([good["u"][:100], [[0.1, 0.2, 0.3]], good["u"][100:]]).astype(np.float32)
    w = np.concatenate([good["w"][:100], [1.0], good["w"][100:]]).astype(np.float32)
    if what == "nan_u":
        u[100, 1] = np.nan
    elif what == "inf_w":
        w[100] = np.inf
    else:
        cell[100] = [1, 10, 10]      # inside the outer margin of the PML: not allowed
    from paper_2201_09084_gb300.api import Sim
    gpu = Sim(3, nphys, D3, pml, dt=ora.dt, order=1, prec="fp32", alpha_mode="damped")
    gpu.set_tuning(ppt, 1)
    pos, mom = pack_particles(cell, off, u, w, "fp32")
    gpu.add_species(pos, mom, len(w), -O.Q_E, O.M_E)
    ora.step(4)
    gpu.step(4)
    with pytest.raises(L.PicError) as e:
        gpu.sync()
    assert e.value.code == PIC_EPARTICLE
    err = max_field_err(ora, gpu)
    assert max(err.values()) < TOL["fp32"], err
    X, _, alive = gpu_positions(gpu, 0)
    assert not alive[100]
    assert np.array_equal(np.delete(alive, 100), ora.particles()["alive"])


def test_fixed_point_weight_overflow_is_reported():
    """|w q/e| above 2^32 cannot be represented by the deterministic
    accumulator: the deposit skips it and pic_sync reports PIC_EOVERFLOW."""
    from paper_2201_09084_gb300 import _lib as L
    from paper_2201_09084_gb300.api import Sim, pack_particles
    gpu = Sim(3, (10, 10, 12), D3, (4,) * 6, order=1, prec="fixed64")
    p = _parts(20, 9)
    w = p["w"].copy()
    w[5] = 1e10
    pos, mom = pack_particles(p["cell"], p["off"], p["u"], w, "fixed64")
    gpu.add_species(pos, mom, len(w), -O.Q_E, O.M_E)
    gpu.step(1)
    with pytest.raises(L.PicError) as e:
        gpu.sync()
    assert e.value.code == PIC_EOVERFLOW


def test_checkpoint_resumes_bit_identically_in_fixed_point():
    """N steps straight, against N/2 steps, a checkpoint of the fields (and
    a copy of the caller-owned particles) taken into a fresh context, and N/2
    more steps: bit-identical fields in deterministic mode."""
    import torch
    from paper_2201_09084_gb300.api import Sim, pack_particles
    nphys, pml = (12, 10, 14), (5,) * 6
    p = I.random_particles(3, 3000, [6, 6, 6], [16, 14, 18], u_rms=1.5, seed=13)[0]

    def fresh(pos, mom, n):
        s = Sim(3, nphys, D3, pml, order=1, prec="fixed64", alpha_mode="damped")
        s.add_species(pos, mom, n, -O.Q_E, O.M_E)
        return s

    pos, mom = pack_particles(p["cell"], p["off"], p["u"], p["w"], "fixed64")
    a = fresh(pos.clone(), mom.clone(), 3000)
    a.step(12)
    b = fresh(pos.clone(), mom.clone(), 3000)
    b.step(6)
    st = b.get_state()
    n = b.num_particles(0)
    bpos, bmom = b.species[0]
    c = fresh(bpos.clone(), bmom.clone(), n)
    c.set_state(st)
    c.step(6)
    torch.cuda.synchronize()
    for f in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        assert torch.equal(a.field(f), c.field(f)), f
