"""Pins of the oracle's field update (Yee leapfrog + split-field PML).

- A cavity eigenmode of a perfectly conducting box oscillates at exactly the
  frequency of the Yee dispersion relation (Sec. II.B: the alpha terms leave
  the usual FDTD discretisation unchanged).  Initial data are closed forms.
- With a vanishing conductivity and alpha = 1 the split-field equations
  (Eqs. MaxwellE, MaxwellB, MaxwellSum) reduce to Maxwell's equations: the
  split path equals the plain path (Sec. II.A, alpha = 0 / sigma = 0 remark).
- A well-resolved plane pulse entering a weak PML decays as
  exp(-int sigma/(eps0 c) dz), the continuum PML attenuation (Berenger).
- The PML of App. A absorbs an incident pulse; a bare conductor reflects it.
- Oblique incidence: a waveguide mode between conducting x-walls (two plane
  waves at +-theta) entering a conductor-backed weak z-PML returns with the
  energy fraction exp(-4 cos(theta) int sigma/(eps0 c) dz), the round trip of
  the split-field PML's matched attenuation (Sec. II.A); B_z, which only
  oblique waves carry, must stay undamped by sigma_z for this to hold.
"""
import numpy as np
import pytest

import oracle as O

C = O.C_LIGHT


def _grid_coords(sim):
    nx, ny, nz = sim.nn
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    return i, j, k


def _mode_fields(sim, N, d, A, dim):
    """Closed-form (1,1,1) PEC cavity mode on the Yee grid, and its discrete curl."""
    kk = [np.pi / (N[a] * d[a]) if N[a] else 0.0 for a in range(3)]
    kt = [2.0 / d[a] * np.sin(kk[a] * d[a] / 2) for a in range(3)]
    i, j, k = _grid_coords(sim)
    x_n, y_n, z_n = i * d[0], j * d[1], k * d[2]
    x_c, y_c, z_c = (i + 0.5) * d[0], (j + 0.5) * d[1], (k + 0.5) * d[2]
    s, c_ = np.sin, np.cos
    if dim == 3:
        Sy_n, Cy_n, Cy_c, Sy_c = s(kk[1] * y_n), c_(kk[1] * y_n), c_(kk[1] * y_c), s(kk[1] * y_c)
        kty = kt[1]
    else:
        # d/dy = 0: the y factor is 1 and y-derivatives vanish
        Sy_n = Cy_n = Cy_c = Sy_c = np.ones_like(y_n, dtype=float)
        kty = 0.0
    E = [A[0] * c_(kk[0] * x_c) * Sy_n * s(kk[2] * z_n),
         A[1] * s(kk[0] * x_n) * (Cy_c if dim == 3 else 1.0) * s(kk[2] * z_n),
         A[2] * s(kk[0] * x_n) * Sy_n * c_(kk[2] * z_c)]
    # discrete curl of E at the B locations
    Cx = (kty * A[2] - kt[2] * A[1]) * s(kk[0] * x_n) * (Cy_c if dim == 3 else 1.0) * c_(kk[2] * z_c)
    Cy = (kt[2] * A[0] - kt[0] * A[2]) * c_(kk[0] * x_c) * Sy_n * c_(kk[2] * z_c)
    Cz = (kt[0] * A[1] - kty * A[0]) * c_(kk[0] * x_c) * (Cy_c if dim == 3 else 1.0) * s(kk[2] * z_n)
    shape = (sim.nn[2], sim.nn[1], sim.nn[0])
    E = [np.broadcast_to(e, shape).astype(float) for e in E]
    Cu = [np.broadcast_to(e, shape).astype(float) for e in (Cx, Cy, Cz)]
    ktot2 = kt[0] ** 2 + kty ** 2 + kt[2] ** 2
    return E, Cu, ktot2, kt


@pytest.mark.parametrize("dim", [3, 2])
def test_cavity_mode_frequency(dim):
    N = (12, 10, 14) if dim == 3 else (12, 0, 14)
    d = (1.0e-6, 1.3e-6, 0.8e-6)
    dt = O.yee_dt(d, 0.95, dim)
    sim = O.OracleSim(dim, N, (0,) * 6, d, dt, alpha_mode="one")
    if dim == 3:
        kt = [2.0 / d[a] * np.sin(np.pi / (N[a] * d[a]) * d[a] / 2) for a in range(3)]
        A = np.cross(kt, [1.0, 0.3, -0.7])  # divergence-free amplitude: A . kt = 0
    else:
        kt = [2.0 / d[a] * np.sin(np.pi / (N[a] * d[a]) * d[a] / 2) if N[a] else 0 for a in range(3)]
        A = np.array([kt[2], 0.6 * np.hypot(kt[0], kt[2]), -kt[0]])
    A = A / np.abs(A).max()
    E0, Cu, k2, _ = _mode_fields(sim, N, d, A, dim)
    # only the staggered locations inside the box carry a field: drop the rest
    Ex_mask = np.zeros_like(E0[0]); Ex_mask[:, :, :N[0]] = 1
    Ey_mask = np.zeros_like(E0[1]); Ey_mask[...] = 1
    if dim == 3:
        Ey_mask[:, N[1]:, :] = 0
    Ez_mask = np.zeros_like(E0[2]); Ez_mask[:N[2], :, :] = 1
    masks_E = [Ex_mask, Ey_mask, Ez_mask]
    E0 = [e * m for e, m in zip(E0, masks_E)]
    Bx_mask = np.ones_like(Cu[0]); Bx_mask[N[2]:, :, :] = 0
    By_mask = np.ones_like(Cu[1]); By_mask[N[2]:, :, :] = 0; By_mask[:, :, N[0]:] = 0
    Bz_mask = np.ones_like(Cu[2]); Bz_mask[:, :, N[0]:] = 0
    if dim == 3:
        Bx_mask[:, N[1]:, :] = 0
        Bz_mask[:, N[1]:, :] = 0
    Cu = [cc * m for cc, m in zip(Cu, (Bx_mask, By_mask, Bz_mask))]
    for c, n in enumerate("xyz"):
        sim.set_field("E" + n, E0[c])
        sim.set_field("Bh" + n, -0.5 * dt * Cu[c])
        sim.set_field("Bp" + n, +0.5 * dt * Cu[c])
    # Yee dispersion: sin(w dt/2) = (c dt/2) |k~|
    w = 2.0 / dt * np.arcsin(C * dt / 2 * np.sqrt(k2))
    nsteps = 37
    sim.step(nsteps)
    scale = max(np.abs(e).max() for e in E0)
    for c, n in enumerate("xyz"):
        expect = np.cos(w * nsteps * dt) * E0[c]
        got = sim.field("E" + n)
        assert np.abs(got - expect).max() < 1e-10 * scale, (n, np.abs(got - expect).max())
    # B^{n+1/2} = -(dt/2) C sin(w (n+1/2) dt) / sin(w dt/2)
    bscale = max(np.abs(cc).max() for cc in Cu) * dt
    for c, n in enumerate("xyz"):
        expect = -0.5 * dt * Cu[c] * np.sin(w * (nsteps + 0.5) * dt) / np.sin(w * dt / 2)
        got = sim.field("Bh" + n)
        assert np.abs(got - expect).max() < 1e-9 * bscale, (n, np.abs(got - expect).max() / bscale)


def _random_run(dim, pml, coef, steps=25, mode="one"):
    N_int = (10, 9, 11)
    d = (1e-6, 1.1e-6, 0.9e-6)
    dt = O.yee_dt(d, 0.9, dim)
    sim = O.OracleSim(dim, N_int, pml, d, dt, order=1, alpha_mode=mode, sig_coef=coef)
    rng = np.random.default_rng(5)
    nx, ny, nz = sim.nn
    # a smooth initial E that vanishes on the outer planes
    i, j, k = _grid_coords(sim)
    Nt = [nx - 1, ny - 1, nz - 1]
    fx = np.sin(np.pi * i / Nt[0]) ; fz = np.sin(np.pi * k / Nt[2])
    fy = np.sin(np.pi * j / Nt[1]) if dim == 3 else 1.0
    shape = (nz, ny, nx)
    sim.set_field("Ey", np.broadcast_to(fx * fz * 1e3, shape))
    # moving particles (prescribed) that stay in the interior
    n = 6
    lo = np.array([pml[0], pml[2], pml[4]]) + 3.0
    X = lo[0] + rng.random(n) * 4
    Y = lo[1] + rng.random(n) * 3 if dim == 3 else np.zeros(n)
    Z = lo[2] + rng.random(n) * 4
    u = rng.normal(size=(3, n)) * 0.3
    sim.add_particles(X, Y, Z, u[0], u[1], u[2], np.ones(n), -O.Q_E, O.M_E)
    sim.set_prescribed(True)
    sim.step(steps)
    return sim


@pytest.mark.parametrize("dim", [3, 2])
def test_split_equals_unsplit_for_vanishing_sigma(dim):
    # total grid identical: 3-cell PML with sigma ~ 0 on each face vs plain cells
    pml = (3, 3, 3, 3, 3, 3)
    a = _random_run(dim, pml, 1e-20)
    # same total size with no PML: physical cells grow by the PML cells
    N_int = (10 + 6, 9 + 6, 11 + 6)
    d = (1e-6, 1.1e-6, 0.9e-6)
    dt = O.yee_dt(d, 0.9, dim)
    b = O.OracleSim(dim, N_int, (0,) * 6, d, dt, order=1, alpha_mode="one")
    nx, ny, nz = b.nn
    i, j, k = _grid_coords(b)
    fx = np.sin(np.pi * i / (nx - 1)); fz = np.sin(np.pi * k / (nz - 1))
    b.set_field("Ey", np.broadcast_to(fx * fz * 1e3, (nz, ny, nx)))
    rng = np.random.default_rng(5)
    n = 6
    lo = np.array([3, 3, 3]) + 3.0
    X = lo[0] + rng.random(n) * 4
    Y = lo[1] + rng.random(n) * 3 if dim == 3 else np.zeros(n)
    Z = lo[2] + rng.random(n) * 4
    u = rng.normal(size=(3, n)) * 0.3
    b.add_particles(X, Y, Z, u[0], u[1], u[2], np.ones(n), -O.Q_E, O.M_E)
    b.set_prescribed(True)
    b.step(25)
    for f in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        fa, fb = a.field(f), b.field(f)
        scale = np.abs(fb).max()
        assert scale > 0
        assert np.abs(fa - fb).max() <= 1e-12 * scale, (f, np.abs(fa - fb).max() / scale)


def _pulse_run(coef, delta, p, pml_cells, steps, probes, width=15.0, nz_phys=200):
    """x-uniform plane pulse (Ex, By) travelling along +z in 2D between
    conducting x-walls, entering a +z PML."""
    d = (1e-6, 1e-6, 1e-6)
    dt = O.yee_dt(d, 0.99, 2)
    nx = 4
    sim = O.OracleSim(2, (nx, 0, nz_phys), (0, 0, 0, 0, pml_cells, pml_cells), d, dt,
                      alpha_mode="one", sig_coef=coef, delta=delta, sig_exp=p)
    _, _, nzt = sim.nn
    z0 = pml_cells + nz_phys * 0.5
    k = np.arange(nzt)[:, None, None] * 1.0
    f = lambda z: np.exp(-((z - z0) / width) ** 2)
    shape = (nzt, 1, nx + 1)
    Ex = np.broadcast_to(f(k), shape).copy()
    Ex[:, :, nx:] = 0
    Ex[0] = Ex[-1] = 0
    s = C * dt / d[2]
    Bh = np.broadcast_to(f(k + 0.5 - 0.5 * s) / C, shape).copy()
    Bp = np.broadcast_to(f(k + 0.5 + 0.5 * s) / C, shape).copy()
    for a in (Bh, Bp):
        a[:, :, nx:] = 0
        a[-1] = 0
    sim.set_field("Ex", Ex)
    sim.set_field("Bhy", Bh)
    sim.set_field("Bpy", Bp)
    rec = np.zeros((steps, len(probes)))
    for n in range(steps):
        sim.step(1)
        ex = sim.field("Ex")[:, 0, 1]
        rec[n] = ex[probes]
    return sim, rec, z0


def test_pml_plane_wave_attenuation():
    # weak profile: int_0^60 sigma/(eps0 c) dz = coef * 60^3/(3 delta^2) = 4
    coef, delta, p, L = 0.2, 60.0, 2.0, 60
    depths = np.array([0, 10, 20, 30, 40, 50])
    probes = 60 + 200 + depths
    sim, rec, z0 = _pulse_run(coef, delta, p, L, 330, probes)
    peak = np.abs(rec).max(axis=0)
    for dd, pk in zip(depths, peak):
        expect = np.exp(-coef * dd ** 3 / (3 * delta ** 2))
        assert pk / peak[0] == pytest.approx(expect, rel=0.02), (dd, pk / peak[0], expect)


def test_pml_absorbs_pec_reflects():
    # App. A profile, 16 cells; probe sits in the physical region on the way back
    probe = np.array([16 + 150])
    _, rec_pml, _ = _pulse_run(4.0, 6.0, 2.0, 16, 330, probe)
    _, rec_pec, _ = _pulse_run(0.0, 6.0, 2.0, 16, 330, probe)
    first = np.abs(rec_pml[:150]).max()
    back_pml = np.abs(rec_pml[200:]).max()
    back_pec = np.abs(rec_pec[200:]).max()
    assert first > 0.9
    assert back_pec > 0.9 * first
    assert back_pml < 1e-3 * first



def _guide_mode_run(dim, orient, nt, coef, L, nz=400, z0=200.0, width=60.0, lam=32.0):
    """Waveguide mode between conducting walls entering a z-PML of L cells
    on both sides.  orient "x": E_y ~ sin(pi x / (nt dx)) with B_x, B_z
    (2D, or 3D uniform along y over 2 cells); orient "y" (3D): E_x ~
    sin(pi y / (nt dy)) with B_y, B_z, uniform along x.  The envelope is a
    Gaussian of carrier wavelength lam cells.  E(z) at t = 0 is decomposed
    into Fourier modes along z; each gets the B of the discrete Yee plane wave
    travelling towards +z (discrete wavenumbers 2/d sin(k d/2), frequency from
    the Yee dispersion relation) at B's own staggered points and at
    t = +-dt/2.  Returns the oracle run, a function giving the Yee energy
    (eps0 E^n.E^n + B^{n-1/2}.B^{n+1/2}/mu0)/2 over the physical z range, the
    carrier's angle to the z axis and dt."""
    d = (1e-6, 1e-6, 1e-6)
    dt = O.yee_dt(d, 0.99, dim)
    if dim == 2:
        n = (nt, 0, nz)
    else:
        n = (nt, 2, nz) if orient == "x" else (2, nt, nz)
    sim = O.OracleSim(dim, n, (0, 0, 0, 0, L, L), d, dt, alpha_mode="one",
                      sig_coef=coef, delta=float(L), sig_exp=2.0)
    NZ = sim.nn[2]
    dz = d[2]
    kt = np.pi / (nt * d[0])
    kz0 = 2 * np.pi / (lam * dz)
    z = np.arange(NZ) * dz
    zc = (L + z0) * dz
    E = np.exp(-((z - zc) / (width * dz)) ** 2) * np.cos(kz0 * (z - zc))
    Ek = np.fft.fft(E)
    k = 2 * np.pi * np.fft.fftfreq(NZ, d=dz)
    sg = np.sign(k)
    ktt = 2 / d[0] * np.sin(kt * d[0] / 2)
    ktz = 2 / dz * np.sin(k * dz / 2)
    wt = C * np.sqrt(ktt ** 2 + ktz ** 2)             # 2/dt sin(w dt/2)
    w = 2 / dt * np.arcsin(wt * dt / 2)
    s_node = np.sin(kt * np.arange(nt + 1) * d[0])    # transverse profile at nodes
    s_node[0] = s_node[-1] = 0.0
    c_half = np.cos(kt * (np.arange(nt + 1) + 0.5) * d[0])   # at half nodes
    c_half[-1] = 0.0
    if dim == 2:
        u_half = np.ones(1)                           # no y staggering in 2D
    else:
        u_half = np.ones(3)                           # uniform axis, half nodes
        u_half[-1] = 0.0

    def place(zp, tp):
        if orient == "x":
            return zp[:, None, None] * u_half[None, :, None] * tp[None, None, :]
        return zp[:, None, None] * tp[None, :, None] * u_half[None, None, :]

    # orient x: E_y, B_x = -(k_z/w) E, B_z ~ +(k_x/w); orient y: E_x, B_y = +(k_z/w) E, B_z ~ -(k_y/w)
    sgn = -1.0 if orient == "x" else 1.0
    sim.set_field("Ey" if orient == "x" else "Ex", place(E, s_node))
    for t, tag in ((dt / 2, "h"), (-dt / 2, "p")):
        ph = np.exp(-1j * sg * w * t)
        bt = np.real(np.fft.ifft(sgn * (np.abs(ktz) / wt) * Ek * np.exp(1j * k * dz / 2) * ph))
        bt[-1] = 0.0
        bz = np.real(np.fft.ifft(sgn * 1j * sg * (ktt / wt) * Ek * ph))
        sim.set_field("B" + tag + orient, place(bt, s_node))
        sim.set_field("B" + tag + "z", place(bz, c_half))

    def energy():
        e = sum((sim.field("E" + c) ** 2)[L:L + nz + 1].sum() for c in "xyz")
        b = sum((sim.field("Bh" + c) * sim.field("Bp" + c))[L:L + nz + 1].sum() for c in "xyz")
        return 0.5 * O.EPS0 * e + 0.5 * b * O.EPS0 * C * C

    return sim, energy, np.arctan2(kt, kz0), dt


@pytest.mark.parametrize("dim,orient,nt", [(2, "x", 28), (2, "x", 16), (2, "x", 9), (3, "x", 16),
                                           (3, "y", 9)])
def test_pml_oblique_reflection_coefficient(dim, orient, nt):
    # weak profile, delta = L = 60 cells: int sigma/(eps0 c) dz = coef * L / 3 = 1
    coef, L = 0.05, 60
    sim, energy, theta, dt = _guide_mode_run(dim, orient, nt, coef, L)
    w0 = energy()
    # the carrier's centre goes 260 cells to the conductor and back at the
    # guide's group velocity c cos(theta); the pulse is then back inside
    steps = int(round(2 * 260e-6 / (C * np.cos(theta)) / dt))
    sim.step(steps)
    r2 = energy() / w0
    expect = np.exp(-4 * np.cos(theta) * coef * L / 3)
    assert r2 == pytest.approx(expect, rel=0.03), (np.degrees(theta), r2, expect)
    # an angle-blind attenuation would give exp(-4) = 0.018 at every angle
    if nt == 9:
        assert r2 > 5 * np.exp(-4 * coef * L / 3)


def test_guide_mode_travels_forward_and_conserves_energy_without_pml_loss():
    """The set-up of the oblique test is a pure +z wave: with sigma = 0 the
    Yee energy is conserved, and the pulse's centre moves at the group
    velocity c cos(theta) of the guide."""
    sim, energy, theta, dt = _guide_mode_run(3, "x", 16, 0.0, 60)
    w0 = energy()

    def centre():
        e = (sim.field("Ey") ** 2).sum(axis=(1, 2))
        return (np.arange(len(e)) * e).sum() / e.sum()

    z0 = centre()
    steps = 100          # the pulse (+-150 cells around cell 200) stays inside the 400 cells
    sim.step(steps)
    assert energy() / w0 == pytest.approx(1.0, abs=1e-3)
    moved = centre() - z0
    assert moved == pytest.approx(steps * C * dt * np.cos(theta) / 1e-6, rel=0.03)
