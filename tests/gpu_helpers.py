"""Shared set-up for the GPU parity tests: one oracle box and one CUDA box built
from the same seeded inputs (paper_2201_09084_gb300.inputs)."""
import numpy as np

import oracle as O
from paper_2201_09084_gb300 import inputs as I

# Tolerances on the relative field error: max |GPU - oracle| over a component
# divided by the field scale max(max|E|, c max|B|) over all six components of
# the oracle (E and cB share units; Eq. error weighs them the same way), and
# for the currents by max |J| over the three components.  FP32 kernels: 1e-5
# (the target accuracy of the FP32 form against the FP64 oracle); FP64
# kernels: 1e-11 (only summation orders differ from the oracle).  The
# deterministic int64 deposition carries the FP32 target (its shape quantum
# 2^-20 moves a current by about 1e-6 of its scale).
TOL = {"fp32": 1e-5, "fp64": 1e-11, "fixed64": 1e-5}


def make_pair(dim, nphys, pml, d, parts, order=1, prec="fp32", alpha_mode="damped", cfl=0.99,
              sigma_coef=4.0, delta=6.0, exponent=2.0, v_assumed=O.C_LIGHT, prescribed=False, sort_every=0,
              split_fp64=False, face_alpha=None, filter_passes=0, solver="yee", dt=None):
    import torch
    from paper_2201_09084_gb300.api import Sim, pack_particles
    if dt is None:
        dt = O.ck_dt(d, cfl, dim) if solver == "ck" else O.yee_dt(d, cfl, dim)
    ora = O.OracleSim(dim, nphys, pml, d, dt, order=order, alpha_mode=alpha_mode, sig_coef=sigma_coef,
                      delta=delta, sig_exp=exponent, v_assumed=v_assumed, face_alpha=face_alpha,
                      filter_passes=filter_passes, solver=solver)
    gpu = Sim(dim, nphys, d, pml, dt=dt, order=order, prec=prec, alpha_mode=alpha_mode,
              sigma_coef=sigma_coef, delta=delta, exponent=exponent, v_assumed=v_assumed,
              sort_every=sort_every, split_fp64=split_fp64, face_alpha=face_alpha,
              filter_passes=filter_passes, solver=solver)
    for sp in parts:
        X = I.absolute(sp["cell"], sp["off"])
        u = sp["u"].astype(np.float64)
        w = sp["w"].astype(np.float64)
        refused = ora.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], w,
                                    sp["q"], sp["m"], sp["immobile"])
        assert refused == 0
        pos, mom = pack_particles(sp["cell"], sp["off"], sp["u"], sp["w"], prec)
        gpu.add_species(pos, mom, len(w), sp["q"], sp["m"], sp["immobile"])
    if prescribed:
        ora.set_prescribed(True)
        gpu.set_prescribed(True)
    torch.cuda.synchronize()
    return ora, gpu


def _unit(name):
    return O.C_LIGHT if name[0] == "B" else 1.0


def max_field_err(ora, gpu, names=("Ex", "Ey", "Ez", "Bx", "By", "Bz")):
    """Per-component max |GPU - oracle| over the common field scale."""
    a = {n: ora.field(n) * _unit(n) for n in names}
    b = {n: gpu.field(n).cpu().numpy() * _unit(n) for n in names}
    scale = max(np.abs(v).max() for v in a.values())
    if scale == 0:
        return {n: float(np.abs(b[n]).max()) for n in names}
    return {n: float(np.abs(a[n] - b[n]).max() / scale) for n in names}


def gpu_positions(gpu, sid):
    p = gpu.particles(sid)
    X = p["cell"].astype(np.float64) + p["off"].astype(np.float64)
    return X, p["u"].astype(np.float64), p["alive"]
