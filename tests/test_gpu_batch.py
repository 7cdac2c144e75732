"""Parity of the batched 2D runs (one persistent launch per step, replayed
from a CUDA graph) with one FP64 oracle box per run.  Runs of different
sizes, PML widths, angles and Lorentz factors (a small copy of the paper's
single-particle sweep); same seeded inputs on both sides."""
import numpy as np
import pytest

import oracle as O
from paper_2201_09084_gb300 import inputs as I
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu

D2 = (1e-6, 1e-6, 1e-6)


def _runs(n, seed):
    return I.batched_runs(n, size_range=(20, 44), pml_range=(6, 12), gamma_range=(1.5, 30.0), seed=seed)


# per-face schemes on the faces the runs' particles leave through: +x removes
# at its interface, +z deposits undamped
FACES = {"faces": ["damped", "zero", "damped", "damped", "damped", "one"]}


@pytest.mark.parametrize("mode", ["damped", "weight", "faces"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("order", [1, 3])
def test_batched_runs_match_single_oracle_boxes(order, prec, mode):
    import torch
    from paper_2201_09084_gb300.api import Batch, pack_particles
    r = _runs(7, seed=31 + order)
    dt = O.yee_dt(D2, 0.99, 2)
    alpha, faces = ("damped", FACES[mode]) if mode in FACES else (mode, None)
    pos, mom = pack_particles(r["cell"], r["off"], r["u"], r["w"], prec)
    b = Batch(r["nx"], r["nz"], r["npml"], (D2[0], D2[2]), pos, mom, r["q"], r["m"], dt=dt, order=order,
              prec=prec, alpha_mode=alpha, face_alpha=faces)
    oras = []
    for k in range(7):
        p = int(r["npml"][k])
        s = O.OracleSim(2, (int(r["nx"][k]), 0, int(r["nz"][k])), (p, p, 0, 0, p, p), D2, dt, order=order,
                        alpha_mode=alpha, face_alpha=faces)
        X = I.absolute(r["cell"][k:k + 1], r["off"][k:k + 1])
        u = r["u"][k].astype(np.float64)
        s.add_particles(X[:, 0], X[:, 1], X[:, 2], [u[0]], [u[1]], [u[2]], [1.0], r["q"], r["m"])
        oras.append(s)
    for blk in range(3):
        b.step(25)                   # odd counts exercise the single-launch path too
        for s in oras:
            s.step(25)
        torch.cuda.synchronize()
        for k, s in enumerate(oras):
            names = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
            unit = {n: O.C_LIGHT if n[0] == "B" else 1.0 for n in names}
            a = {n: s.field(n) * unit[n] for n in names}
            g = {n: b.field(k, n).cpu().numpy() * unit[n] for n in names}
            scale = max(np.abs(v).max() for v in a.values())
            err = max(float(np.abs(a[n] - g[n]).max()) for n in names) / scale
            assert err < TOL[prec], (blk, k, err)
    b.sync()
    assert b.particle_steps() > 0


def test_batched_runs_full_size_sampled():
    """The benchmark's batch itself -- 4096 runs of 64-256 cells per side with
    8-24-cell PMLs, FP32, order 3, its autotuned block shape, steps replayed
    from the CUDA graph -- with six of its runs (the smallest, the largest,
    the widest PML and three drawn at random) compared with one FP64 oracle
    box each after 50 steps."""
    import torch
    from paper_2201_09084_gb300.api import Batch, pack_particles
    r = I.batched_runs(4096)
    dt = O.yee_dt(D2, 0.99, 2)
    pos, mom = pack_particles(r["cell"], r["off"], r["u"], r["w"], "fp32")
    b = Batch(r["nx"], r["nz"], r["npml"], (D2[0], D2[2]), pos, mom, r["q"], r["m"], dt=dt, order=3,
              prec="fp32", alpha_mode="damped")
    cells = (r["nx"] + 2 * r["npml"]) * (r["nz"] + 2 * r["npml"])
    rng = np.random.default_rng(77)
    pick = sorted({int(np.argmin(cells)), int(np.argmax(cells)), int(np.argmax(r["npml"]))} |
                  {int(v) for v in rng.choice(4096, 3, replace=False)})
    oras = {}
    for k in pick:
        p = int(r["npml"][k])
        s = O.OracleSim(2, (int(r["nx"][k]), 0, int(r["nz"][k])), (p, p, 0, 0, p, p), D2, dt, order=3,
                        alpha_mode="damped")
        X = I.absolute(r["cell"][k:k + 1], r["off"][k:k + 1])
        u = r["u"][k].astype(np.float64)
        s.add_particles(X[:, 0], X[:, 1], X[:, 2], [u[0]], [u[1]], [u[2]], [1.0], r["q"], r["m"])
        oras[k] = s
    b.step(50)
    for s in oras.values():
        s.step(50)
    torch.cuda.synchronize()
    names = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
    unit = {n: O.C_LIGHT if n[0] == "B" else 1.0 for n in names}
    for k, s in oras.items():
        a = {n: s.field(n) * unit[n] for n in names}
        g = {n: b.field(k, n).cpu().numpy() * unit[n] for n in names}
        scale = max(np.abs(v).max() for v in a.values())
        err = max(float(np.abs(a[n] - g[n]).max()) for n in names) / scale
        assert err < TOL["fp32"], (k, int(r["nx"][k]), int(r["nz"][k]), int(r["npml"][k]), err)
    b.sync()
