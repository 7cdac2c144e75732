"""Host checks of the seeded input generators (no GPU).

- The plane-by-plane plasma draws each z-plane of cells from its own stream,
  so a plane is the same however the planes are grouped, and it has the
  distributions of the one-piece generator: ppc particles in every cell,
  offsets uniform in [0, 1), Maxwellian momenta of width u_th, the weight
  n0 d^3 / ppc, protons on top of their electrons.
- The benchmark's streamed packing puts every plane's records, in plane
  order, into one array per species (cell index packed i | j << 10 | k << 20).
"""
import os
import sys

import numpy as np
import pytest

from paper_2201_09084_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

NPHYS = (34, 34, 66)
PML = (16,) * 6
D = 1e-6


def test_plasma_planes_are_per_plane_streams():
    _, planes_a = I.plasma_planes(NPHYS, PML, D)
    _, planes_b = I.plasma_planes(NPHYS, PML, D)
    a = {k: (el, pr) for k, el, pr in planes_a if k in (0, 5, 65)}
    b = {}
    for k, el, pr in planes_b:
        if k == 5:
            b[k] = (el, pr)
            break
    for key in ("cell", "off", "u", "w"):
        assert np.array_equal(a[5][0][key], b[5][0][key])
        assert np.array_equal(a[5][1][key], b[5][1][key])
    assert not np.array_equal(a[0][0]["off"], a[5][0]["off"])


def test_plasma_planes_distributions():
    beam, planes = I.plasma_planes(NPHYS, PML, D)
    w0 = I.plasma_density(0.01, D) * D ** 3 / 8
    offs, us = [], []
    for k, el, pr in planes:
        assert np.array_equal(el["cell"], pr["cell"]) and np.array_equal(el["off"], pr["off"])
        assert np.all(el["cell"][:, 2] == PML[4] + k)
        ij = el["cell"][:, 0].astype(np.int64) * 1000 + el["cell"][:, 1]
        _, counts = np.unique(ij, return_counts=True)
        assert len(counts) == NPHYS[0] * NPHYS[1] and np.all(counts == 8)
        assert np.all((el["off"] >= 0) & (el["off"] < 1))
        assert np.allclose(el["w"], w0, rtol=1e-6)
        assert el["q"] < 0 < pr["q"] and pr["m"] > el["m"]
        if k < 8:
            offs.append(el["off"])
            us.append(el["u"])
    offs = np.concatenate(offs)
    us = np.concatenate(us)
    assert abs(offs.mean() - 0.5) < 0.005
    assert abs(offs.var() - 1.0 / 12.0) < 0.002
    assert abs(us.mean()) < 2e-4 and abs(us.std() / 0.01 - 1.0) < 0.01
    bm, bi = beam
    assert len(bm["w"]) == len(bi["w"]) > 0 and bi["immobile"] and not bm["immobile"]
    assert np.all(bm["u"][:, 2] == 5.0) and np.array_equal(bm["cell"], bi["cell"])


def test_streamed_species_hold_every_plane_in_order(monkeypatch):
    torch = pytest.importorskip("torch")
    import bench
    monkeypatch.setattr(bench, "STREAM_PARTICLES", 0)
    species = bench.plasma_species(NPHYS, "cpu")
    assert len(species) == 4
    per_plane = NPHYS[0] * NPHYS[1] * 8
    _, planes = I.plasma_planes(NPHYS, PML, D)
    el_pos, el_mom, n, q, m, imm = species[0]
    assert n == per_plane * NPHYS[2] and q < 0 and not imm
    cell = el_mom.view(torch.int32)[:, 3].numpy().astype(np.int64)
    k = (cell >> 20) - PML[4]
    assert np.array_equal(k, np.repeat(np.arange(NPHYS[2]), per_plane))
    for kk, el, pr in planes:
        if kk == 7:
            sl = slice(7 * per_plane, 8 * per_plane)
            assert np.array_equal(el_pos[sl, :3].numpy(), el["off"])
            assert np.array_equal(species[1][1][sl, :3].numpy(), pr["u"])
            break
    assert species[3][5] and species[2][2] == species[3][2]
