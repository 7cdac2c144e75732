"""The tile-resident particle kernel (PIC_TUNING_TILE: 3D FP32 boxes of shape
order 1 whose species are sorted by tile) against the FP64 oracle, through the
C ABI.

The kernel gathers from a TMA-loaded field box, keeps the Esirkepov current of
in-cell moves in two register runs per thread (a move in a third cell flushes
the run used less recently), queues moves across cell faces per warp, adds
the runs and the queue to the grid with global reductions and alpha, and sends
particles outside the box (or moving 1/16 cell or more) through global memory.
These tests put every one of those paths on ragged grids (tile and unit counts
that do not divide the grid), with particles inside the damped PML, particles
removed at the outer edge, units whose species take several passes, records
injected after the last sort (the unsorted tail) and a species added after
it.  Particles are matched to the oracle's by a unique FP32
weight, since the sort permutes them.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL, make_pair, max_field_err

pytestmark = pytest.mark.gpu

D3 = (1e-6, 1.1e-6, 0.9e-6)
TILE = 2   # PIC_TUNING_TILE


def _tag(parts, base):
    """Unique FP32 weights base + i 2^-15 (exact), to find each particle again."""
    for k, sp in enumerate(parts):
        n = len(sp["w"])
        assert n < 32768
        sp["w"] = (np.float32(base + k) + np.arange(n, dtype=np.float32) * np.float32(2.0 ** -15)).astype(np.float32)
    return parts


def _pulse(nn, amp):
    nx, ny, nz = nn
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = ((i - nx / 2) / 6.0) ** 2 + ((j - ny / 2) / 5.0) ** 2 + ((k - nz / 2) / 7.0) ** 2
    f = amp * np.exp(-r2)
    f[:, :, 0] = f[:, :, -1] = 0
    f[0] = f[-1] = 0
    f[:, 0] = f[:, -1] = 0
    return f


def _set_fields(sims, nn):
    f = _pulse(nn, 1.0)
    for s in sims:
        s.set_field("Ex", 3e11 * f)
        s.set_field("Ey", 1e11 * np.roll(f, 2, axis=1))
        s.set_field("Ez", -2e11 * np.roll(f, 3, axis=2))
        s.set_field("Bhy", 1e3 * f)
        s.set_field("Bpy", 0.8e3 * f)
        s.set_field("Bhz", 0.5e3 * np.roll(f, 2, axis=0))
        s.set_field("Bpx", 0.3e3 * np.roll(f, -2, axis=0))


def _match(gpu, sid, po, sel):
    """GPU records of species sid ordered like the oracle's records `sel`,
    matched by weight (every weight is unique)."""
    p = gpu.particles(sid)
    order = np.argsort(p["w"])
    wo = po["w"][sel]
    oo = np.argsort(wo)
    assert np.array_equal(p["w"][order].astype(np.float64), wo[oo]), "weights changed"
    inv = np.empty_like(oo)
    inv[oo] = np.arange(len(oo))
    idx = order[inv]
    X = p["cell"][idx].astype(np.float64) + p["off"][idx].astype(np.float64)
    return X, p["u"][idx].astype(np.float64), p["alive"][idx]


def test_tile_one_step_matches_oracle():
    """One fused push + deposit in smooth nonzero fields on a ragged grid:
    slow particles (moves of a few hundredths of a cell: the threads' runs),
    fast ones (moves across faces: the warps' queues), particles in every PML
    face (damped flush) and near the outer edge (removed)."""
    nphys = (37, 21, 30)
    pml = (6, 7, 5, 8, 6, 9)
    N = (nphys[0] + 13, nphys[1] + 13, nphys[2] + 15)
    lo, hi = [2.2, 2.2, 2.2], [N[0] - 2.2, N[1] - 2.2, N[2] - 2.2]
    slow = I.random_particles(3, 24000, lo, hi, u_rms=0.05, seed=301)
    fast = I.random_particles(3, 6000, lo, hi, u_rms=1.5, seed=302)
    parts = _tag(slow + fast, 1.0)
    ora, gpu = make_pair(3, nphys, pml, D3, parts, order=1, prec="fp32", alpha_mode="damped")
    _set_fields((ora, gpu), ora.nn)
    gpu.sort()
    gpu.set_tuning(TILE, 1)
    l0 = gpu.launch_count()
    ora.push()
    ora.deposit()
    gpu.push_deposit()
    # B was set from outside the field step: one launch forms B^n, then one
    # tile-kernel launch pushes both species
    assert gpu.launch_count() - l0 == 2, "B^n average + one tile-kernel launch for both species"
    err = max_field_err(ora, gpu, ("Jx", "Jy", "Jz"))
    print(f"\ncurrent error (of max |J|): {err}")
    assert max(err.values()) < TOL["fp32"], err
    po = ora.particles()
    n0 = len(slow[0]["w"])
    for sid, sel in ((0, slice(0, n0)), (1, slice(n0, None))):
        X, u, alive = _match(gpu, sid, po, sel)
        assert np.array_equal(alive, po["alive"][sel])
        Xo = np.stack([po["X"][sel], po["Y"][sel], po["Z"][sel]], 1)
        uo = np.stack([po["ux"][sel], po["uy"][sel], po["uz"][sel]], 1)
        a = alive
        assert np.abs(X[a] - Xo[a]).max() < 2e-6
        assert np.abs(u[a] - uo[a]).max() < 1e-5 * np.abs(uo).max()
    assert (~po["alive"]).sum() > 0, "some particles should leave through the outer edge"


def test_tile_dense_units_take_several_passes():
    """Two species packed into eight units (about 94 and 56 particles per
    cell): each unit's species take several passes of at most 12 particles
    per thread, whose extra particles rotate over the warps from pass to
    pass and from species to species; one fused push + deposit against the
    oracle, every particle pushed once."""
    nphys = (40, 12, 12)
    pml = (4,) * 6
    lo, hi = [6.0, 5.0, 5.0], [26.0, 9.0, 9.0]
    a = I.random_particles(3, 30000, lo, hi, u_rms=0.05, seed=321)
    b = I.random_particles(3, 18000, lo, hi, u_rms=0.2, seed=322, q=O.Q_E, m=O.M_P * 0.05)
    parts = _tag(a + b, 1.0)
    ora, gpu = make_pair(3, nphys, pml, D3, parts, order=1, prec="fp32", alpha_mode="damped")
    _set_fields((ora, gpu), ora.nn)
    gpu.sort()
    gpu.set_tuning(TILE, 1)
    ps0 = gpu.particle_steps()
    ora.push()
    ora.deposit()
    gpu.push_deposit()
    assert gpu.particle_steps() - ps0 == 48000
    err = max_field_err(ora, gpu, ("Jx", "Jy", "Jz"))
    print(f"\ndense units, current error (of max |J|): {err}")
    assert max(err.values()) < TOL["fp32"], err
    po = ora.particles()
    for sid, sel in ((0, slice(0, 30000)), (1, slice(30000, None))):
        X, u, alive = _match(gpu, sid, po, sel)
        assert np.array_equal(alive, po["alive"][sel])
        Xo = np.stack([po["X"][sel], po["Y"][sel], po["Z"][sel]], 1)
        uo = np.stack([po["ux"][sel], po["uy"][sel], po["uz"][sel]], 1)
        assert np.abs(X - Xo).max() < 2e-6
        assert np.abs(u - uo).max() < 1e-5 * np.abs(uo).max()


@pytest.fixture(scope="module")
def plasma_ref():
    D = (1e-6, 1e-6, 1e-6)
    nphys, pml = (24, 24, 48), (8,) * 6
    parts = I.plasma(nphys, pml, D[0], beam_radius=4.0, beam_length=12.0)
    dt = O.yee_dt(D, 0.99, 3)
    ora = O.OracleSim(3, nphys, pml, D, dt, order=1, alpha_mode="damped")
    for sp in parts:
        X = I.absolute(sp["cell"], sp["off"])
        u = sp["u"].astype(np.float64)
        assert ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], sp["w"].astype(np.float64),
                                 sp["q"], sp["m"], sp["immobile"]) == 0
    out = {}
    for n in (10, 20):
        ora.step(10)
        out[n] = {k: ora.field(k) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    return dict(D=D, nphys=nphys, pml=pml, parts=parts, dt=dt, ref=out)


class _Frozen:
    def __init__(self, f):
        self.f = f

    def field(self, k):
        return self.f[k]


@pytest.mark.parametrize("form", ["fp32", "fp32-splitfp64", "fixed64"])
def test_tile_plasma_beam_first_20_steps(plasma_ref, form):
    """The plasma + beam workload (reduced): whole steps with the tile kernel,
    sorted every 5 steps, one particle launch per step for the three mobile
    species; fields within the FP32 tolerance after 10 and 20 steps."""
    from paper_2201_09084_gb300.api import Sim, pack_particles
    r = plasma_ref
    split_fp64 = form == "fp32-splitfp64"
    prec = "fixed64" if form == "fixed64" else "fp32"
    gpu = Sim(3, r["nphys"], r["D"], r["pml"], dt=r["dt"], order=1, prec=prec, alpha_mode="damped",
              sort_every=5, split_fp64=split_fp64)
    keep = []
    for sp in r["parts"]:
        pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], prec)
        gpu.add_species(pos, mom, len(sp["w"]), sp["q"], sp["m"], sp["immobile"])
        keep.append((pos, mom))
    gpu.set_tuning(TILE, 1)
    gpu.step(1)                     # sorts, then the first step
    l0 = gpu.launch_count()
    gpu.step(1)                     # no sort: one particle launch + the E and B passes
    assert gpu.launch_count() - l0 == (4 if prec == "fixed64" else 3)   # (+ the fixed-point flush)
    gpu.step(8)
    err = max_field_err(_Frozen(r["ref"][10]), gpu)
    assert max(err.values()) < TOL["fp32"], (10, err)
    gpu.step(10)
    err = max_field_err(_Frozen(r["ref"][20]), gpu)
    print(f"\ntile kernel, {form}: max rel field error after 20 steps {max(err.values()):.3e}")
    assert max(err.values()) < TOL[prec], (20, err)
    gpu.sync()


def test_tile_tail_and_unsorted_species():
    """Records injected after the last sort (the kernel's unsorted tail, one
    thread per particle through global memory) and a species registered
    after the sort (one-thread kernel) step together with sorted species."""
    import torch
    from paper_2201_09084_gb300.api import pack_particles
    nphys = (14, 12, 16)
    pml = (6, 6, 6, 6, 6, 6)
    N = (26, 24, 28)
    lo, hi = [2.5, 2.5, 2.5], [N[0] - 2.5, N[1] - 2.5, N[2] - 2.5]
    base = I.random_particles(3, 8000, lo, hi, u_rms=0.05, seed=311)
    ora, gpu = make_pair(3, nphys, pml, D3, [], order=1, prec="fp32", alpha_mode="damped")
    cap = 8000 + 600
    sp = base[0]
    pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], "fp32", capacity=cap)
    sid = gpu.add_species(pos, mom, 8000, sp["q"], sp["m"])
    X = I.absolute(sp["cell"], sp["off"])
    u = sp["u"].astype(np.float64)
    assert ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], sp["w"].astype(np.float64),
                             sp["q"], sp["m"]) == 0
    _set_fields((ora, gpu), ora.nn)
    gpu.sort()
    gpu.set_tuning(TILE, 1)
    rng = np.random.default_rng(312)
    late = None
    for step in range(6):
        if step in (1, 3):   # injected after the sort: the tail
            k = 300
            Xi = np.stack([rng.uniform(lo[a], hi[a], k) for a in range(3)], 1)
            ui = rng.normal(0, 0.8, (k, 3)).astype(np.float32)
            c, o = I.split_position(Xi)
            ip, im = pack_particles(c, o, ui, np.full(k, 0.7, np.float32), "fp32")
            gpu.inject(sid, ip, im)
            Xa = I.absolute(c, o)
            ua = ui.astype(np.float64)
            assert ora.add_particles(Xa[:, 0], Xa[:, 1], Xa[:, 2], ua[:, 0], ua[:, 1], ua[:, 2], np.full(k, 0.7),
                                     -O.Q_E, O.M_E) == 0
        if step == 2:        # a species added after the sort (not tile-sorted)
            late = I.random_particles(3, 2000, lo, hi, u_rms=0.3, seed=313, q=O.Q_E, m=O.M_P * 0.01)[0]
            lp, lm = pack_particles(late["cell"], late["off"], late["u"], late["w"], "fp32")
            gpu.add_species(lp, lm, 2000, late["q"], late["m"])
            Xl = I.absolute(late["cell"], late["off"])
            ul = late["u"].astype(np.float64)
            assert ora.add_particles(Xl[:, 0], Xl[:, 1], Xl[:, 2], ul[:, 0], ul[:, 1], ul[:, 2],
                                     late["w"].astype(np.float64), late["q"], late["m"]) == 0
        ora.step(1)
        gpu.step(1)
    torch.cuda.synchronize()
    gpu.sync()
    err = max_field_err(ora, gpu)
    print(f"\ntail + late species: max rel field error {max(err.values()):.3e}")
    assert max(err.values()) < TOL["fp32"], err
    assert gpu.num_particles(sid) == 8600
