"""Deterministic (int64 fixed-point) deposition through the C ABI, 3D.

- Deposit stage in isolation: prescribed moves (old positions set through
  pic_set_old_positions, new ones as the species' records) of two species
  with different charges, orders 1 and 3, spread over the whole grid
  including the PML: the int64 sums equal the oracle's integer replay BIT FOR
  BIT, and the damped FP32 current written for the field update equals
  alpha_c K Jq with alpha from the oracle's own tables.
- Determinism of whole steps: a beam run twice, the second time with its
  particles in a different order (and sorted every few steps), gives
  bit-identical fields and integer currents; FP32 atomics would not.
- Whole steps against the FP64 oracle: the beam exiting through the damped
  PML stays within the FP32 tolerance.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, make_pair, max_field_err

pytestmark = pytest.mark.gpu

D3 = (1e-6, 1.1e-6, 0.9e-6)


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_deposit_bit_exact(order):
    import torch
    from paper_2201_09084_gb300.api import Sim, pack_particles
    nphys = (37, 21, 45)
    pml = (6, 9, 5, 7, 8, 10)
    N = (nphys[0] + 15, nphys[1] + 12, nphys[2] + 18)
    margin = 2 if order == 1 else 3
    lo = [margin + 1] * 3
    hi = [N[a] - margin - 1 for a in range(3)]
    dt = O.yee_dt(D3, 0.99, 3)
    gpu = Sim(3, nphys, D3, pml, dt=dt, order=order, prec="fixed64", alpha_mode="damped")
    nn = gpu.nn
    species = [(-O.Q_E, O.M_E, 7000, 101), (2 * O.Q_E, O.M_P, 3001, 202)]
    expect = [np.zeros((nn[2], nn[1], nn[0]), np.int64) for _ in range(3)]
    keep = []
    for q, m, n, seed in species:
        c0, f0, c1, f1, w = I.random_moves(n, lo, hi, seed=seed + order)
        assert c1.min() >= margin and all(c1[:, a].max() <= N[a] - margin - 1 for a in range(3))
        pos, mom = pack_particles(c1, f1, np.zeros((n, 3), np.float32), w, "fixed64")
        sid = gpu.add_species(pos, mom, n, q, m)
        keep.append(gpu.set_old_positions(sid, c0, f0))
        J = O.fixed_deposit3d(order, c0, f0, c1, f1, w, q / O.Q_E, nn)
        for c in range(3):
            expect[c] += J[c]
    gpu.deposit()
    gpu.sync()
    for c in range(3):
        got = gpu.current_fixed(c).cpu().numpy()
        assert np.count_nonzero(expect[c]) > 1000
        assert np.array_equal(got, expect[c]), (c, int(np.count_nonzero(got != expect[c])))
    # the damped current handed to the field update
    ora = O.OracleSim(3, nphys, pml, D3, dt, order=order, alpha_mode="damped")
    an = [ora.table("a_node", a) for a in range(3)]
    ac = [ora.table("a_cent", a) for a in range(3)]
    area = (D3[1] * D3[2], D3[0] * D3[2], D3[0] * D3[1])
    for c, name in enumerate("xyz"):
        al = [ac[a] if a == c else an[a] for a in range(3)]
        alpha = al[2][:, None, None] * al[1][None, :, None] * al[0][None, None, :]
        ref = -(O.Q_E / (area[c] * dt)) * expect[c].astype(np.float64) / O.FIXED_UNIT * alpha
        got = gpu.field("J" + name).cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-6 * scale, name
    del keep


def _beam_pair(order, permute, sort_every, prec="fixed64"):
    nphys = (22, 19, 26)
    pml = (6,) * 6
    center = (6 + 11.3, 6 + 9.6, 6 + 18.2)
    parts = I.beam(3, 3000, nphys, pml, center, sigma=(1.5, 1.5, 2.5), theta_deg=15.0, clip=3.0)
    if permute:
        p = parts[0]
        idx = np.random.default_rng(5).permutation(len(p["w"]))
        parts = [dict(p, cell=p["cell"][idx], off=p["off"][idx], u=p["u"][idx], w=p["w"][idx])]
    return make_pair(3, nphys, pml, D3, parts, order=order, prec=prec, alpha_mode="damped",
                     sort_every=sort_every)


@pytest.mark.parametrize("tuning", ["default", "tile"])
@pytest.mark.parametrize("order", [1, 3])
def test_fixed_steps_are_order_independent(order, tuning):
    """With the tile kernel's deterministic form selected, the sorted run
    pushes its particles in the tile kernel and the unsorted one in the
    one-thread kernel: the fields and integer currents still agree bit for
    bit."""
    if tuning == "tile" and order != 1:
        pytest.skip("the tile kernel serves order 1")
    _, a = _beam_pair(order, permute=False, sort_every=0)
    _, b = _beam_pair(order, permute=True, sort_every=4)
    if tuning == "tile":
        a.set_tuning(2, 1)
        b.set_tuning(2, 1)
    a.step(20)
    b.step(20)
    for name in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        fa, fb = a.field(name).cpu().numpy(), b.field(name).cpu().numpy()
        assert np.abs(fa).max() > 0
        assert np.array_equal(fa, fb), name
    for c in range(3):
        assert np.array_equal(a.current_fixed(c).cpu().numpy(), b.current_fixed(c).cpu().numpy())


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_beam_exit_matches_oracle(order):
    ora, gpu = _beam_pair(order, permute=False, sort_every=5)
    for _ in range(2):
        ora.step(12)
        gpu.step(12)
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL["fixed64"], err


D2 = (1e-6, 1.0, 0.9e-6)


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_deposit_bit_exact_2d(order):
    """2D boxes: the int64 sums of prescribed moves (J_x, J_z in-plane, J_y
    from the momenta's v_y) equal the oracle's 2D replay bit for bit, and the
    damped current handed to the field update is alpha_c K Jq."""
    from paper_2201_09084_gb300.api import Sim, pack_particles
    nphys = (41, 0, 37)
    pml = (6, 9, 0, 0, 8, 7)
    N = (nphys[0] + 15, 0, nphys[2] + 15)
    margin = 2 if order == 1 else 3
    lo = [margin + 1, 0, margin + 1]
    hi = [N[0] - margin - 1, 0.5, N[2] - margin - 1]
    dt = O.yee_dt(D2, 0.99, 2)
    gpu = Sim(2, nphys, D2, pml, dt=dt, order=order, prec="fixed64", alpha_mode="damped")
    nn = gpu.nn
    expect = [np.zeros((nn[2], nn[0]), np.int64) for _ in range(3)]
    keep = []
    rng = np.random.default_rng(17 + order)
    for q, m, n, seed in [(-O.Q_E, O.M_E, 5000, 31), (2 * O.Q_E, O.M_P, 2001, 47)]:
        c0, f0, c1, f1, w = I.random_moves(n, lo, hi, seed=seed + order)
        for a in (c0, c1):
            a[:, 1] = 0
        f0[:, 1] = 0.0
        f1[:, 1] = 0.0
        u = rng.normal(0.0, 1.5, (n, 3)).astype(np.float32)
        pos, mom = pack_particles(c1, f1, u, w, "fixed64")
        sid = gpu.add_species(pos, mom, n, q, m)
        keep.append(gpu.set_old_positions(sid, c0, f0))
        J = O.fixed_deposit2d(order, c0, f0, c1, f1, w, u, q / O.Q_E, (nn[0], nn[2]))
        for c in range(3):
            expect[c] += J[c]
    gpu.deposit()
    gpu.sync()
    for c in range(3):
        got = gpu.current_fixed(c).cpu().numpy()[:, 0, :]
        assert np.count_nonzero(expect[c]) > 500
        assert np.array_equal(got, expect[c]), (c, int(np.count_nonzero(got != expect[c])))
    ora = O.OracleSim(2, nphys, pml, D2, dt, order=order, alpha_mode="damped")
    an = [ora.table("a_node", a) for a in (0, 2)]
    ac = [ora.table("a_cent", a) for a in (0, 2)]
    conv = {"x": -(O.Q_E / (D2[2] * dt)), "y": O.Q_E * O.C_LIGHT / (D2[0] * D2[2]), "z": -(O.Q_E / (D2[0] * dt))}
    for c, name in enumerate("xyz"):
        ax = ac[0] if c == 0 else an[0]
        az = ac[1] if c == 2 else an[1]
        ref = conv[name] * expect[c].astype(np.float64) / O.FIXED_UNIT * az[:, None] * ax[None, :]
        got = gpu.field("J" + name).cpu().numpy()[:, 0, :]
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-6 * scale, name
    del keep


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_2d_whole_steps_order_independent_and_near_oracle(order):
    """2D single particles exiting through the damped PML: the deterministic
    run is bit-identical with its particles permuted, and within the FP32
    tolerance of the FP64 oracle."""
    import torch
    from paper_2201_09084_gb300.api import Sim, pack_particles
    nphys = (40, 0, 44)
    pml = (8, 8, 0, 0, 8, 8)
    rng = np.random.default_rng(5 + order)
    n = 60
    X = np.stack([8 + rng.uniform(10, 30, n), np.zeros(n), 8 + rng.uniform(14, 34, n)], 1)
    u = np.stack([rng.normal(0, 2, n), rng.normal(0, 2, n), rng.normal(0, 3, n)], 1).astype(np.float32)
    cell, off = I.split_position(X)
    w = np.ones(n, np.float32)
    dt = O.yee_dt(D2, 0.99, 2)
    parts = [dict(cell=cell, off=off, u=u, w=w, q=-O.Q_E, m=O.M_E, immobile=False),
             dict(cell=cell, off=off, u=np.zeros_like(u), w=w, q=O.Q_E, m=O.M_E, immobile=True)]
    ora, gpu = make_pair(2, nphys, pml, D2, parts, order=order, prec="fixed64", alpha_mode="damped")
    perm = rng.permutation(n)
    p2 = [dict(parts[0], cell=cell[perm], off=off[perm], u=u[perm]), dict(parts[1], cell=cell[perm], off=off[perm])]
    _, gpu2 = make_pair(2, nphys, pml, D2, p2, order=order, prec="fixed64", alpha_mode="damped")
    for _ in range(3):
        ora.step(10)
        gpu.step(10)
        gpu2.step(10)
        err = max_field_err(ora, gpu)
        assert max(err.values()) < TOL["fixed64"], err
    torch.cuda.synchronize()
    for f in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        assert torch.equal(gpu.field(f), gpu2.field(f)), f
