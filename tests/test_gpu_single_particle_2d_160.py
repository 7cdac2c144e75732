"""The 2D FP64 single-particle workload at its full size, against the oracle.

128 x 128 physical cells of 1 um with a 16-cell PML on all four sides; an
electron with u_z = 10 (gamma = sqrt(101)) and its motionless partner at the
centre, moving at normal incidence into the +z PML (App. A single-particle
setup); shape order 1, dt = 0.99 x the Yee Courant limit, 400 steps.
- The CUDA FP64 path matches the oracle element by element on the whole grid
  (combined field scale, 1e-11) at several times, with the damped current.
- Eq. error against a PML-free 512 x 512 reference run (the physical box at
  nodes (192, 144) of it, conducting outer walls that no signal reaches
  within the compared region in 400 steps) is the same number on the GPU and
  in the oracle, for the damped scheme and for Berenger's alpha = 0.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, make_pair, max_field_err

pytestmark = pytest.mark.gpu

D = (1e-6, 1e-6, 1e-6)
NPHYS = (128, 0, 128)
PML = (16, 16, 0, 0, 16, 16)
GAMMA = float(np.sqrt(101.0))
REF_N = (512, 0, 512)
REF_OFFSET = (192 - 16, 0, 144 - 16)   # reference node index of the damped box's node 0


class _Host:
    """numpy view of a GPU Sim for oracle.rel_error."""

    def __init__(self, s):
        self.s, self.n, self.pml, self.dim = s, s.n, s.pml, s.dim

    def field(self, name):
        return self.s.field(name).cpu().numpy()


def _pair(nphys, pml, start=None, mode="damped"):
    parts = I.single_pair(2, nphys, pml, gamma=GAMMA, start=start)
    return make_pair(2, nphys, pml, D, parts, order=1, prec="fp64", alpha_mode=mode)


@pytest.mark.parametrize("mode", ["damped", "zero"])
def test_single_particle_2d_160_full_size(mode):
    start = np.array([PML[0] + 64.3, 0.0, PML[4] + 64.2])
    ora, gpu = _pair(NPHYS, PML, start=start, mode=mode)
    for _ in range(4):
        ora.step(100)
        gpu.step(100)
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL["fp64"], err
    ref_start = start + np.array(REF_OFFSET, dtype=np.float64)
    ora_ref, gpu_ref = _pair(REF_N, (0,) * 6, start=ref_start)
    ora_ref.step(400)
    gpu_ref.step(400)
    e_ora = O.rel_error(ora, ora_ref, REF_OFFSET)
    e_gpu = O.rel_error(_Host(gpu), _Host(gpu_ref), REF_OFFSET)
    assert np.isfinite(e_ora) and e_ora > 0
    assert abs(e_gpu - e_ora) <= 1e-6 * e_ora, (e_gpu, e_ora)
    print(f"\nEq. error at step 400, alpha {mode}: oracle {e_ora:.6e}, GPU {e_gpu:.6e}")
