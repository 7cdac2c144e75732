"""The diagnostics of the CUDA path (pic_diag: charge density, Gauss-law
residual, field energy; FP64 reductions) against the same quantities
computed by the oracle on the same state.

Both sides step the same seeded particles (a moving species and its
immobile opposite-charge partners, so the box starts neutral and Gauss's law
holds), then:
  rho_scale = max |rho/eps0| over the nodes at least one cell inside the
              physical region (the oracle's rho() of the live particles),
  gauss     = max |div E - rho/eps0| over the same nodes (the oracle's
              divE()),
  energy    = sum over the whole grid of (eps0 E^2 + B^2/mu0)/2 times the cell
              volume, B at the integer time.
With the binomial current filter (App. A) the field conserves the filtered
charge, so div E - rho/eps0 is of the order of rho/eps0 itself and the
residual is compared as a value, not only bounded; without the filter it is
round-off on both sides.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import make_pair

pytestmark = pytest.mark.gpu

D3 = (1e-6, 1.1e-6, 0.9e-6)
D2 = (1e-6, 1e-6, 1e-6)


def _parts(dim, nphys, pml, n, seed):
    lo = [pml[0] + 3, (pml[2] + 3) if dim == 3 else 0, pml[4] + 3]
    hi = [pml[0] + nphys[0] - 3, (pml[2] + nphys[1] - 3) if dim == 3 else 1, pml[4] + nphys[2] - 3]
    mov = I.random_particles(dim, n, lo, hi, u_rms=0.4, seed=seed)[0]
    if dim == 2:
        mov["cell"][:, 1] = 0
        mov["off"][:, 1] = 0.0
        mov["u"][:, 1] = 0.0
    still = dict(mov, u=np.zeros_like(mov["u"]), q=-mov["q"], immobile=True)
    return [mov, still]


def _oracle_diag(ora, dim):
    rho = ora.rho() / O.EPS0
    div = ora.divE()
    lo = [ora.pml[0], ora.pml[2], ora.pml[4]]
    n = [ora.n[0], ora.n[1], ora.n[2]]
    sl = []
    for a in (2, 1, 0):   # arrays are [k, j, i]
        if dim == 2 and a == 1:
            sl.append(slice(0, 1))
        else:
            sl.append(slice(lo[a] + 1, lo[a] + n[a]))
    sl = tuple(sl)
    res = float(np.abs(div[sl] - rho[sl]).max())
    scale = float(np.abs(rho[sl]).max())
    vol = ora.d[0] * ora.d[2] * (ora.d[1] if dim == 3 else 1.0)
    e2 = sum((ora.field("E" + c) ** 2).sum() for c in "xyz")
    b2 = sum(((O.C_LIGHT * ora.field("B" + c)) ** 2).sum() for c in "xyz")
    energy = float(0.5 * O.EPS0 * (e2 + b2) * vol)
    return res, scale, energy


@pytest.mark.parametrize("prec,filt", [("fp64", 0), ("fp64", 1), ("fp32", 0), ("fp32", 1)])
@pytest.mark.parametrize("dim,order", [(3, 1), (3, 3), (2, 3)])
def test_diag_matches_oracle_on_the_same_state(dim, order, prec, filt):
    nphys = (14, 12, 16) if dim == 3 else (22, 0, 26)
    pml = (6,) * 6 if dim == 3 else (6, 6, 0, 0, 6, 6)
    d = D3 if dim == 3 else D2
    parts = _parts(dim, nphys, pml, 600, seed=40 + order + 3 * dim)
    ora, gpu = make_pair(dim, nphys, pml, d, parts, order=order, prec=prec, alpha_mode="damped",
                         filter_passes=filt, split_fp64=True)
    ora.step(15)
    gpu.step(15)
    res, scale, energy = _oracle_diag(ora, dim)
    dg = gpu.diag()
    assert scale > 0 and energy > 0
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert dg["rho_scale"] == pytest.approx(scale, rel=tol)
    assert dg["energy"] == pytest.approx(energy, rel=tol)
    if filt:
        assert res > 1e-3 * scale, "the filtered current leaves a residual of the order of rho/eps0"
        assert abs(dg["gauss"] - res) <= tol * scale, (dg["gauss"], res, scale)
    else:
        assert res <= 1e-10 * scale
        assert dg["gauss"] <= (1e-10 if prec == "fp64" else 1e-5) * scale, (dg["gauss"], scale)
