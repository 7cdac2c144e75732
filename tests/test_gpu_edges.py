"""Edge cases of the GPU path against the oracle: uneven and missing PML
faces, degenerate particles (on nodes, at rest, zero weight), empty species,
and the largest grids the packed cell index allows."""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, make_pair, max_field_err, gpu_positions

pytestmark = pytest.mark.gpu

D3 = (1e-6, 1.1e-6, 0.9e-6)


@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_uneven_and_missing_pml_faces(prec, order):
    """PML widths differ per face and two faces have none (a PEC wall right at
    the physical box)."""
    nphys = (14, 12, 16)
    pml = (0, 5, 3, 0, 7, 2)
    parts = I.random_particles(3, 400, [4.0, 4.0, 9.0], [13.0, 11.0, 21.0], u_rms=1.5, seed=5 + order)
    ora, gpu = make_pair(3, nphys, pml, D3, parts, order=order, prec=prec, alpha_mode="damped")
    for _ in range(2):
        ora.step(6)
        gpu.step(6)
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL[prec], err
    X, u, alive = gpu_positions(gpu, 0)
    assert np.array_equal(alive, ora.particles()["alive"])


@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_degenerate_particles(prec, order):
    """Particles exactly on nodes (offset 0), at rest, and with weight 0,
    mixed with ordinary ones; a charge at rest on a node deposits nothing."""
    nphys = (12, 12, 12)
    pml = (4,) * 6
    rng = np.random.default_rng(9 + order)
    n = 300
    X = np.floor(rng.uniform(6, 14, (n, 3)))            # on nodes
    X[::3] += rng.random((len(X[::3]), 3))              # a third off the nodes
    u = rng.normal(0, 1.0, (n, 3))
    u[1::4] = 0.0                                        # at rest
    w = np.ones(n)
    w[2::5] = 0.0                                        # zero weight
    cell, off = I.split_position(X)
    parts = [dict(cell=cell, off=off, u=u.astype(np.float32), w=w.astype(np.float32), q=-O.Q_E, m=O.M_E,
                  immobile=False)]
    ora, gpu = make_pair(3, nphys, pml, D3, parts, order=order, prec=prec, alpha_mode="damped")
    for _ in range(2):
        ora.step(5)
        gpu.step(5)
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL[prec], err
    Xg, ug, alive = gpu_positions(gpu, 0)
    po = ora.particles()
    assert np.array_equal(alive, po["alive"])
    Xo = np.stack([po["X"], po["Y"], po["Z"]], 1)
    assert np.max(np.abs(Xg[alive] - Xo[alive])) < (1e-5 if prec == "fp32" else 1e-10)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_empty_species_and_no_particles(prec):
    """Species with no live particles (capacity > 0 and capacity 0) next to
    an ordinary one; a box with only empty species keeps zero fields."""
    import torch
    from paper_2201_09084_gb300.api import Sim, pack_particles
    nphys = (10, 10, 12)
    pml = (4,) * 6
    parts = I.random_particles(3, 100, [6, 6, 6], [12, 12, 14], u_rms=1.0, seed=3)
    ora, gpu = make_pair(3, nphys, pml, D3, parts, order=1, prec=prec, alpha_mode="damped")
    z = np.zeros((16, 3))
    pos, mom = pack_particles(z.astype(np.int64), z.astype(np.float32), z.astype(np.float32),
                              np.zeros(16, np.float32), prec)
    gpu.add_species(pos, mom, 0, O.Q_E, O.M_P)
    pos0, mom0 = pack_particles(np.zeros((0, 3), np.int64), np.zeros((0, 3), np.float32),
                                np.zeros((0, 3), np.float32), np.zeros(0, np.float32), prec)
    gpu.add_species(pos0, mom0, 0, O.Q_E, O.M_P)
    ora.step(6)
    gpu.step(6)
    err = max_field_err(ora, gpu)
    assert max(err.values()) < TOL[prec], err
    empty = Sim(3, nphys, D3, pml, prec=prec)
    empty.add_species(pos, mom, 0, O.Q_E, O.M_P)
    empty.step(3)
    for f in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        assert float(empty.field(f).abs().max()) == 0.0, f


def test_largest_packed_grid_is_accepted_and_one_more_cell_rejected():
    """The cell index packs i, j < 1024 and k < 2048: a grid of 1023 x 1 x
    2047 cells in total (x, z here in 2D: 1023 x 2047) is accepted; one more
    cell along x is rejected before any allocation."""
    from paper_2201_09084_gb300 import _lib as L
    from paper_2201_09084_gb300.api import Sim
    d = (1e-6, 1e-6, 1e-6)
    ok = Sim(2, (1023 - 8, 0, 2047 - 8), d, (4, 4, 0, 0, 4, 4), prec="fp32")
    ok.step(1)
    with pytest.raises(L.PicError) as e:
        Sim(2, (1024 - 8, 0, 2047 - 8), d, (4, 4, 0, 0, 4, 4), prec="fp32")
    assert e.value.code == -1
