"""The benchmark's default workload at its full size, in the launch
configuration the benchmark times: the thermal plasma + drifting beam in
256 x 256 x 512 physical cells + a 16-cell PML on every face (288 x 288 x 544
cells), electrons and protons 8 per cell (536,870,912) plus the u_z = 5 beam,
FP32 fields with IEEE FP64 PML parts, the tile kernel, a sort every 20 steps;
and the precision-study workload, the same at 128 x 128 x 256 (67 M
particles), in FP32 and in the deterministic int64 form.

No oracle box of this size runs; the checks are the ones that hold at any
size or that the oracle can make one particle at a time:
- sampled particles (every species, drawn at random): their push in one
  tile-kernel launch against the FP64 oracle's gather, Boris push and move of
  the same record in a 7 x 7 x 7-cell oracle box holding the GPU's own fields
  around the particle (E^n, B^{n+1/2}, B^{n-1/2}; the particle in its cell 3,
  inside the oracle's two-cell margin);
- charge conservation (Esirkepov): after whole steps the Gauss residual
  max |div E - rho/eps0| stays at FP32 round-off of max |rho/eps0|, and the
  live particles are all pushed every step.
"""
import os
import sys

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

NSAMPLE = 200   # particles per mobile species


def _neighbourhood(fields, c):
    """The 8 x 8 x 8 nodes c - 3 .. c + 4 of each device field, as numpy
    arrays indexed [k, j, i]."""
    sl = (slice(c[2] - 3, c[2] + 5), slice(c[1] - 3, c[1] + 5), slice(c[0] - 3, c[0] + 5))
    return {n: a[sl].cpu().numpy() for n, a in fields.items()}


@pytest.mark.parametrize("cells,prec", [((256, 256, 512), "fp32"), ((128, 128, 256), "fp32"),
                                        ((128, 128, 256), "fixed64")], ids=["537M-fp32", "67M-fp32", "67M-fixed64"])
def test_headline_full_size_sampled_push_and_gauss(cells, prec):
    import torch
    import bench
    from paper_2201_09084_gb300.api import Sim
    recs = bench.headline_records(cells, "cuda")
    sim = Sim(3, cells, bench.D, bench.PML, cfl=0.99, order=1, prec=prec, alpha_mode="damped",
              sort_every=bench.SORT_EVERY, split_fp64=True)
    for pos, mom, n, q, m, imm in recs:
        sim.add_species(pos, mom, n, q, m, imm)
    sim.set_tuning(2, 1)   # the tile kernel, as the benchmark's autotuner chooses on this workload
    dt = sim.dt
    sim.step(3)            # (sorts first) non-trivial fields for the sampled pushes
    torch.cuda.synchronize()

    # ---- sampled particles: state before one push, the fields around them ----
    names = {"Ex": "Ex", "Ey": "Ey", "Ez": "Ez", "Bhx": "Bhx", "Bhy": "Bhy", "Bhz": "Bhz",
             "Bpx": "Bpx", "Bpy": "Bpy", "Bpz": "Bpz"}
    fields = {n: sim.field(g) for n, g in names.items()}
    rng = np.random.default_rng(2201)
    samples = []
    for sid, (pos, mom, n, q, m, imm) in enumerate(recs):
        if imm:
            continue
        idx = torch.as_tensor(np.unique(rng.integers(0, n, size=2 * NSAMPLE))[:NSAMPLE], device="cuda")
        p0 = pos[idx].cpu().numpy().astype(np.float64)
        m0 = mom[idx].cpu().numpy()
        cw = m0[:, 3].view(np.int32).astype(np.int64)
        for k in range(len(idx)):
            if cw[k] < 0:
                continue
            c = (int(cw[k] & 1023), int((cw[k] >> 10) & 1023), int(cw[k] >> 20))
            samples.append(dict(sid=sid, idx=int(idx[k]), c=c, off=p0[k, :3], w=p0[k, 3],
                                u=m0[k, :3].astype(np.float64), q=q, m=m, nb=_neighbourhood(fields, c)))
    del fields
    torch.cuda.empty_cache()
    sim.push_deposit()
    torch.cuda.synchronize()
    checked = 0
    for s in samples:
        pos, mom = recs[s["sid"]][0], recs[s["sid"]][1]
        p1 = pos[s["idx"]].cpu().numpy().astype(np.float64)
        m1 = mom[s["idx"]].cpu().numpy()
        cw1 = int(m1[3:4].view(np.int32)[0])
        assert cw1 >= 0, "a sampled particle was removed"
        c1 = np.array([cw1 & 1023, (cw1 >> 10) & 1023, cw1 >> 20], dtype=np.float64)
        X_gpu = c1 + p1[:3]
        u_gpu = m1[:3].astype(np.float64)
        # the oracle's push of the same record in a 7^3-cell box with the GPU's fields
        ora = O.OracleSim(3, (7, 7, 7), (0,) * 6, bench.D, dt, order=1, alpha_mode="one")
        for n, a in s["nb"].items():
            ora.set_field(n, a)
        X_loc = 3.0 + s["off"]
        assert ora.add_particles([X_loc[0]], [X_loc[1]], [X_loc[2]], [s["u"][0]], [s["u"][1]], [s["u"][2]],
                                 [s["w"]], s["q"], s["m"]) == 0
        ora.push()
        po = ora.particles()
        X_ora = np.array([po["X"][0], po["Y"][0], po["Z"][0]]) - 3.0 + np.array(s["c"], dtype=np.float64)
        u_ora = np.array([po["ux"][0], po["uy"][0], po["uz"][0]])
        du = u_ora - s["u"]
        # FP32 record and FP32 push: the momentum to ~10 FP32 ulps of |u| plus
        # FP32 round-off of the increment; the position to 1e-5 cell
        tol_u = 1e-6 * np.abs(u_ora).max() + 1e-4 * np.abs(du).max() + 1e-12
        assert np.abs(u_gpu - u_ora).max() <= tol_u, (s["sid"], s["idx"], u_gpu, u_ora, s["u"])
        assert np.abs(X_gpu - X_ora).max() < 1e-5, (s["sid"], s["idx"], X_gpu, X_ora)
        checked += 1
    assert checked >= 2 * NSAMPLE
    sim.field_step()

    # ---- whole steps: every live particle pushed, Gauss's law to FP32 round-off ----
    live = sum(sim.num_particles(s) for s in range(len(recs)) if not recs[s][5])
    thermal = sim.num_particles(0) + sim.num_particles(1)
    ps0 = sim.particle_steps()
    sim.step(5)
    torch.cuda.synchronize()
    pushed = sim.particle_steps() - ps0
    assert 5 * thermal <= pushed <= 5 * live   # (beam particles may leave through the outer wall)
    dg = sim.diag()
    assert dg["rho_scale"] > 0
    assert dg["gauss"] <= 1e-5 * dg["rho_scale"], dg
    sim.sync()
    print(f"\n{cells} {prec}: {checked} sampled pushes against the oracle, "
          f"Gauss residual {dg['gauss'] / dg['rho_scale']:.2e} of max rho/eps0")
