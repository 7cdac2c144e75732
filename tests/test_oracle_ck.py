"""Pins of the oracle's Cole-Karkkainen (CK) field solver (the solver of the
paper's single-particle and LWFA runs, App. A; scheme of Cole 1997/2002 and
Karkkainen et al. 2006: Faraday's-law differences of E averaged over the two
transverse axes with weights (1/4, 1/2, 1/4) each, Ampere's law as in Yee).

- A PEC cavity eigenmode (mode numbers m) is an exact discrete eigenmode and
  oscillates at the frequency of the CK dispersion relation
    sin^2(w dt/2) = (c dt)^2 sum_a s_a^2 prod_{b != a} cos^2(k_b d_b/2),
  s_a = sin(k_a d_a/2)/d_a, with B^{n+1/2} from the CK curl of E (the Yee
  curl with the derivative along a scaled by prod_{b != a} cos^2(k_b d_b/2)).
  Checked below the Courant limit on uneven cells and at the limit itself,
  c dt = d on cubic cells, for a short-wavelength mode.
- At c dt = d (cubic cells) the CK scheme stays bounded while Yee, whose
  limit is d / sqrt(3), blows up.
- A divergence-free closed-form mode whose transverse wavenumbers vanish is
  not possible in a closed conducting box, so the axial property (no
  dispersion along an axis at c dt = d) is pinned through the relation above:
  with k_b = 0 for b != a it reads sin(w dt/2) = sin(k_a d/2).
"""
import numpy as np
import pytest

import oracle as O

C = O.C_LIGHT


def _coords(sim):
    nx, ny, nz = sim.nn
    return np.arange(nx)[None, None, :], np.arange(ny)[None, :, None], np.arange(nz)[:, None, None]


def _ck_mode(sim, N, d, A, dim, m):
    """Closed-form PEC cavity mode (m_x, m_y, m_z) on the Yee grid, its CK
    curl at the B locations, and the CK eigenvalue sum_a kt_a^2 F_a."""
    kk = [m[a] * np.pi / (N[a] * d[a]) if N[a] else 0.0 for a in range(3)]
    kt = [2.0 / d[a] * np.sin(kk[a] * d[a] / 2) for a in range(3)]
    cs = [np.cos(kk[a] * d[a] / 2) ** 2 for a in range(3)]
    if dim == 2:
        kt[1], cs[1] = 0.0, 1.0
    F = [cs[1] * cs[2], cs[0] * cs[2], cs[0] * cs[1]]
    ktt = [kt[a] * F[a] for a in range(3)]            # CK derivative factors
    i, j, k = _coords(sim)
    x_n, y_n, z_n = i * d[0], j * d[1], k * d[2]
    x_c, y_c, z_c = (i + 0.5) * d[0], (j + 0.5) * d[1], (k + 0.5) * d[2]
    s, c_ = np.sin, np.cos
    one = np.ones_like(y_n, dtype=float)
    Sy_n = s(kk[1] * y_n) if dim == 3 else one
    Cy_c = c_(kk[1] * y_c) if dim == 3 else one
    E = [A[0] * c_(kk[0] * x_c) * Sy_n * s(kk[2] * z_n),
         A[1] * s(kk[0] * x_n) * Cy_c * s(kk[2] * z_n),
         A[2] * s(kk[0] * x_n) * Sy_n * c_(kk[2] * z_c)]
    Cx = (ktt[1] * A[2] - ktt[2] * A[1]) * s(kk[0] * x_n) * Cy_c * c_(kk[2] * z_c)
    Cy = (ktt[2] * A[0] - ktt[0] * A[2]) * c_(kk[0] * x_c) * Sy_n * c_(kk[2] * z_c)
    Cz = (ktt[0] * A[1] - ktt[1] * A[0]) * c_(kk[0] * x_c) * Cy_c * s(kk[2] * z_n)
    shape = (sim.nn[2], sim.nn[1], sim.nn[0])
    E = [np.broadcast_to(e, shape).astype(float) for e in E]
    Cu = [np.broadcast_to(e, shape).astype(float) for e in (Cx, Cy, Cz)]
    lam = sum(kt[a] * ktt[a] for a in range(3))
    return E, Cu, lam, kt


def _masks(E, Cu, N, dim):
    Ex_m = np.zeros_like(E[0]); Ex_m[:, :, :N[0]] = 1
    Ey_m = np.ones_like(E[1])
    Ez_m = np.zeros_like(E[2]); Ez_m[:N[2], :, :] = 1
    Bx_m = np.ones_like(Cu[0]); Bx_m[N[2]:, :, :] = 0
    By_m = np.ones_like(Cu[1]); By_m[N[2]:, :, :] = 0; By_m[:, :, N[0]:] = 0
    Bz_m = np.ones_like(Cu[2]); Bz_m[:, :, N[0]:] = 0
    if dim == 3:
        Ey_m[:, N[1]:, :] = 0
        Bx_m[:, N[1]:, :] = 0
        Bz_m[:, N[1]:, :] = 0
    return [e * mk for e, mk in zip(E, (Ex_m, Ey_m, Ez_m))], [c * mk for c, mk in zip(Cu, (Bx_m, By_m, Bz_m))]


@pytest.mark.parametrize("case", ["3d-uneven", "2d-uneven", "3d-cubic-at-limit", "2d-cubic-at-limit"])
def test_ck_cavity_mode_frequency(case):
    dim = 3 if case.startswith("3d") else 2
    if "uneven" in case:
        N = (12, 10, 14) if dim == 3 else (12, 0, 14)
        d = (1.0e-6, 1.3e-6, 0.8e-6)
        dt = O.ck_dt(d, 0.95, dim)
        m = (1, 1, 1)
    else:
        N = (12, 10, 14) if dim == 3 else (12, 0, 14)
        d = (1.0e-6, 1.0e-6, 1.0e-6)
        dt = O.ck_dt(d, 1.0, dim)
        m = (5, 1, 2)
    sim = O.OracleSim(dim, N, (0,) * 6, d, dt, alpha_mode="one", solver="ck")
    kt = [2.0 / d[a] * np.sin(m[a] * np.pi / (N[a] * d[a]) * d[a] / 2) if N[a] else 0.0 for a in range(3)]
    if dim == 3:
        A = np.cross(kt, [1.0, 0.3, -0.7])   # Yee-divergence-free amplitude: A . kt = 0
    else:
        A = np.array([kt[2], 0.6 * np.hypot(kt[0], kt[2]), -kt[0]])
    A = A / np.abs(A).max()
    E0, Cu, lam, _ = _ck_mode(sim, N, d, A, dim, m)
    E0, Cu = _masks(E0, Cu, N, dim)
    for c, n in enumerate("xyz"):
        sim.set_field("E" + n, E0[c])
        sim.set_field("Bh" + n, -0.5 * dt * Cu[c])
        sim.set_field("Bp" + n, +0.5 * dt * Cu[c])
    arg = C * dt / 2 * np.sqrt(lam)
    assert arg < 1.0
    w = 2.0 / dt * np.arcsin(arg)
    nsteps = 41
    sim.step(nsteps)
    scale = max(np.abs(e).max() for e in E0)
    for c, n in enumerate("xyz"):
        expect = np.cos(w * nsteps * dt) * E0[c]
        got = sim.field("E" + n)
        assert np.abs(got - expect).max() < 1e-10 * scale, (n, np.abs(got - expect).max() / scale)
    bscale = max(np.abs(cc).max() for cc in Cu) * dt
    for c, n in enumerate("xyz"):
        expect = -0.5 * dt * Cu[c] * np.sin(w * (nsteps + 0.5) * dt) / np.sin(w * dt / 2)
        got = sim.field("Bh" + n)
        assert np.abs(got - expect).max() < 1e-9 * bscale, (n, np.abs(got - expect).max() / bscale)
    # the Yee frequency of the same mode differs: the pin sees the CK curl
    lam_yee = sum(k * k for k in kt)
    assert abs(lam_yee - lam) > 1e-3 * lam


def test_ck_dispersion_relation_is_exact_along_an_axis_at_the_limit():
    """With the transverse wavenumbers zero, the CK relation at c dt = d gives
    w = c k for every k along the axis (no numerical dispersion), which Yee
    only reaches in 1D; evaluated from the eigenvalue the cavity pin checks."""
    d = 1.0e-6
    dt = d / C
    for kd in np.linspace(0.1, 3.0, 7):
        s2 = np.sin(kd / 2) ** 2 / d ** 2            # s_x^2; cos^2 factors of k_y = k_z = 0 are 1
        w = 2.0 / dt * np.arcsin(C * dt * np.sqrt(s2))
        assert abs(w - C * kd / d) < 1e-12 * C * kd / d


@pytest.mark.parametrize("dim", [3, 2])
def test_ck_stable_at_c_dt_equal_d_where_yee_is_not(dim):
    N = (10, 9, 11) if dim == 3 else (14, 0, 16)
    d = (1e-6,) * 3
    dt = d[0] / C
    rng = np.random.default_rng(9)

    def run(solver):
        sim = O.OracleSim(dim, N, (0,) * 6, d, dt, alpha_mode="one", solver=solver)
        nx, ny, nz = sim.nn
        for c in "xyz":
            f = rng.standard_normal((nz, ny, nx))
            f[:, :, 0] = f[:, :, -1] = 0
            f[0] = f[-1] = 0
            if dim == 3:
                f[:, 0] = f[:, -1] = 0
            sim.set_field("E" + c, f)
        e0 = max(np.abs(sim.field("E" + c)).max() for c in "xyz")
        sim.step(400)
        return max(np.abs(sim.field("E" + c)).max() for c in "xyz") / e0

    assert run("ck") < 10.0
    grow = run("yee")
    assert not np.isfinite(grow) or grow > 1e6
