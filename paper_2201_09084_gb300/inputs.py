"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

Only random draws and unit bookkeeping live here (no step of the PIC method):
each generator returns particles as an int cell index per axis plus an FP32
in-cell offset, FP32 momenta u = p/(mc) and FP32 weights.  The oracle reads
the same numbers as absolute FP64 positions cell + offset (exact), the CUDA
path packs them into its particle records, so both start from bit-identical
inputs.

Workloads (the paper's single-particle studies, App. A, and the beam/plasma
shapes of the benchmark configurations) are synthetic stand-ins: the paper
used WarpX runs whose inputs and data are not available here.
"""
from __future__ import annotations

import numpy as np

Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
M_P = 1.67262192369e-27
SEED_BASE = 20220121


def split_position(X):
    """Absolute positions (cell units, float64, shape (n,3)) -> (cell int32,
    offset float32 in [0,1)), exactly representable on both sides."""
    X = np.asarray(X, dtype=np.float64)
    cell = np.floor(X).astype(np.int64)
    off = (X - cell).astype(np.float32)
    bump = off >= np.float32(1.0)
    cell[bump] += 1
    off[bump] = 0.0
    return cell.astype(np.int32), off


def absolute(cell, off):
    """cell + offset as FP64 (what the oracle consumes)."""
    return np.asarray(cell, dtype=np.float64) + np.asarray(off, dtype=np.float64)


def _pack(X, u, w, dim):
    X = np.array(X, dtype=np.float64, ndmin=2)
    if dim == 2:
        X[:, 1] = 0.0
    cell, off = split_position(X)
    if dim == 2:
        cell[:, 1] = 0
        off[:, 1] = 0.0
    return dict(cell=cell, off=off, u=np.asarray(u, dtype=np.float32).reshape(-1, 3),
                w=np.asarray(w, dtype=np.float32).reshape(-1))


def single_pair(dim, nphys, pml, gamma, theta_deg=0.0, start=None, q=-Q_E, m=M_E):
    """One macroparticle of Lorentz factor gamma moving in the x-z plane at
    theta_deg from +z, and its motionless opposite-charge partner at the same
    place (App. A, single-particle simulations).  start: absolute position in
    cells (default: centre of the physical box, off the nodes)."""
    lo = np.array([pml[0], pml[2], pml[4]], dtype=np.float64)
    if start is None:
        start = lo + 0.5 * np.array([nphys[0], nphys[1] if dim == 3 else 0, nphys[2]]) + [0.3, 0.1, 0.2]
    u = np.sqrt(gamma ** 2 - 1.0)
    th = np.radians(theta_deg)
    mover = _pack([start], [[u * np.sin(th), 0.0, u * np.cos(th)]], [1.0], dim)
    partner = _pack([start], [[0.0, 0.0, 0.0]], [1.0], dim)
    return [dict(mover, q=q, m=m, immobile=False), dict(partner, q=-q, m=m, immobile=True)]


def beam(dim, n_particles, nphys, pml, center, sigma=(4.0, 4.0, 8.0), uz_mean=50.0, uz_rms=0.5,
         theta_deg=0.0, total_charge=1e-9, seed=SEED_BASE + 1, clip=3.5, q=-Q_E, m=M_E):
    """Relativistic Gaussian electron beam: rms sizes `sigma` (cells, along
    x, y and the beam axis), u along the beam axis ~ N(uz_mean, uz_rms), the
    beam axis rotated by theta_deg from +z towards +x.  Draws beyond `clip`
    standard deviations are redrawn.  Weights give `total_charge` coulombs."""
    rng = np.random.default_rng(seed)
    sig = np.asarray(sigma, dtype=np.float64)
    P = np.empty((0, 3))
    while len(P) < n_particles:
        d = rng.standard_normal((n_particles, 3))
        d = d[np.all(np.abs(d) <= clip, axis=1)]
        P = np.concatenate([P, d * sig])
    P = P[:n_particles]
    uz = rng.normal(uz_mean, uz_rms, n_particles)
    th = np.radians(theta_deg)
    c, s = np.cos(th), np.sin(th)
    X = np.empty_like(P)
    X[:, 0] = center[0] + c * P[:, 0] + s * P[:, 2]
    X[:, 1] = center[1] + P[:, 1]
    X[:, 2] = center[2] - s * P[:, 0] + c * P[:, 2]
    u = np.zeros((n_particles, 3))
    u[:, 0] = s * uz
    u[:, 2] = c * uz
    if dim == 2:
        u[:, 1] = 0.0
    w = np.full(n_particles, total_charge / (Q_E * n_particles))
    key = (np.floor(X[:, 2]) * 4096 + np.floor(X[:, 1])) * 4096 + np.floor(X[:, 0])
    order = np.argsort(key, kind="stable")   # cell-ordered start
    out = _pack(X[order], u[order], w, dim)
    return [dict(out, q=q, m=m, immobile=False)]


def random_particles(dim, n_particles, lo, hi, u_rms=0.5, seed=SEED_BASE + 7, q=-Q_E, m=M_E, w=1.0):
    """Uniform positions in the box [lo, hi) (cells), Gaussian momenta."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    X = lo + rng.random((n_particles, 3)) * (hi - lo)
    u = rng.normal(0.0, u_rms, (n_particles, 3))
    out = _pack(X, u, np.full(n_particles, w), dim)
    return [dict(out, q=q, m=m, immobile=False)]


EPS0 = 8.8541878128e-12
C_LIGHT = 299792458.0


def clustered_runs(dim, n_particles, lo, hi, run=4, u_rms=0.5, p_scatter=0.15, seed=SEED_BASE + 11,
                   q=-Q_E, m=M_E, w=1.0):
    """Particles in an order that no sort produces: consecutive runs of
    `run` * k particles (k ~ U{1..24}) each sit in a 2-cell cube at a random
    place of the box [lo, hi), and with probability p_scatter a single run of
    `run` particles is scattered over the whole box instead.  Kept unsorted,
    they give chunks whose cells span the box while short stretches of
    consecutive particles stay compact.  Gaussian momenta."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    X = np.empty((n_particles, 3))
    i = 0
    while i < n_particles:
        if rng.random() < p_scatter:
            k = min(run, n_particles - i)
            X[i:i + k] = lo + rng.random((k, 3)) * (hi - lo)
        else:
            k = min(run * int(rng.integers(1, 25)), n_particles - i)
            corner = lo + rng.random(3) * (hi - lo - 2.0)
            X[i:i + k] = corner + 2.0 * rng.random((k, 3))
        i += k
    u = rng.normal(0.0, u_rms, (n_particles, 3))
    out = _pack(X, u, np.full(n_particles, w), dim)
    return [dict(out, q=q, m=m, immobile=False)]


def plasma_density(u_th, d):
    """Density n0 whose Debye length u_th c / omega_p equals the cell size d:
    omega_p = u_th c / d, n0 = eps0 m_e omega_p^2 / e^2."""
    wp = u_th * C_LIGHT / d
    return EPS0 * M_E * wp * wp / (Q_E * Q_E)


def plasma(nphys, pml, d, ppc=8, u_th=0.01, beam_uz=5.0, beam_radius=16.0, beam_length=64.0,
           beam_density=0.1, seed=SEED_BASE + 3, box=None):
    """Neutral electron-proton plasma filling the physical box (3D), ppc
    macroparticles per cell and species, uniform in each cell; every proton
    starts at its electron's position (zero charge density at t = 0).
    Momenta are Maxwellian with u_th (as p/(mc)) for both species.  Density
    n0 with Debye length = cell size; weight n0 d^3 / ppc.  Plus a drifting
    electron beam (cylinder of radius beam_radius and length beam_length
    cells along z, density beam_density n0, u_z = beam_uz) whose front sits
    beam_length cells before the +z interface, with immobile neutralising
    ions at the beam electrons' starting positions (so the charge density is
    zero at t = 0 and Gauss's law holds from the start).  box: optional
    (lo, hi) absolute cell range the plasma is restricted to (default: the
    physical box).  Returns [electrons, protons, beam, beam ions] species."""
    rng = np.random.default_rng(seed)
    lo = np.array([pml[0], pml[2], pml[4]], dtype=np.float64)
    hi = lo + np.array(nphys, dtype=np.float64)
    if box is not None:
        lo, hi = np.asarray(box[0], dtype=np.float64), np.asarray(box[1], dtype=np.float64)
    ncell = np.round(hi - lo).astype(np.int64)
    n0 = plasma_density(u_th, d)
    w = n0 * d ** 3 / ppc
    cells = np.stack(np.meshgrid(np.arange(ncell[0]), np.arange(ncell[1]), np.arange(ncell[2]),
                                 indexing="ij"), -1).reshape(-1, 3)
    cells = np.repeat(cells, ppc, axis=0)
    X = lo + cells + rng.random(cells.shape)
    n = len(X)
    ue = rng.normal(0.0, u_th, (n, 3))
    up = rng.normal(0.0, u_th, (n, 3))
    el = _pack(X, ue, np.full(n, w), 3)
    pr = _pack(X, up, np.full(n, w), 3)
    bm, bi = _beam_cylinder(rng, lo, ncell, ppc, w, beam_uz, beam_radius, beam_length, beam_density)
    return [dict(el, q=-Q_E, m=M_E, immobile=False), dict(pr, q=Q_E, m=M_P, immobile=False), bm, bi]


def _beam_cylinder(rng, lo, ncell, ppc, w, beam_uz, beam_radius, beam_length, beam_density):
    """The drifting electron beam of `plasma` (a cylinder along z whose front
    sits beam_length cells before the +z interface) and its immobile ions."""
    zf = lo[2] + ncell[2] - beam_length
    cx, cy = lo[0] + ncell[0] / 2, lo[1] + ncell[1] / 2
    vol = np.pi * beam_radius ** 2 * beam_length
    nb = int(round(vol * ppc * beam_density))
    r = beam_radius * np.sqrt(rng.random(nb))
    ph = 2 * np.pi * rng.random(nb)
    Xb = np.stack([cx + r * np.cos(ph), cy + r * np.sin(ph), zf - beam_length * rng.random(nb)], 1)
    ub = np.zeros((nb, 3))
    ub[:, 2] = beam_uz
    bm = _pack(Xb, ub, np.full(nb, w), 3)
    bi = _pack(Xb, np.zeros((nb, 3)), np.full(nb, w), 3)
    return dict(bm, q=-Q_E, m=M_E, immobile=False), dict(bi, q=Q_E, m=M_P, immobile=True)


def plasma_planes(nphys, pml, d, ppc=8, u_th=0.01, beam_uz=5.0, beam_radius=16.0, beam_length=64.0,
                  beam_density=0.1, seed=SEED_BASE + 13):
    """The plasma + beam workload of `plasma`, drawn one z-plane of physical
    cells at a time for boxes whose particles do not fit the host at once.
    Plane k comes from its own stream (seed, k) and the beam from
    (seed, nz), so the draws do not depend on how planes are grouped, and
    host memory holds one plane.  Same distributions as `plasma` (other
    draws).  Returns (beam species, generator of (k, electrons, protons))."""
    lo = np.array([pml[0], pml[2], pml[4]], dtype=np.float64)
    ncell = np.asarray(nphys, dtype=np.int64)
    w = plasma_density(u_th, d) * d ** 3 / ppc
    beam = _beam_cylinder(np.random.default_rng([seed, int(ncell[2])]), lo, ncell, ppc, w, beam_uz,
                          beam_radius, beam_length, beam_density)
    ij = np.stack(np.meshgrid(np.arange(ncell[0]), np.arange(ncell[1]), indexing="ij"), -1).reshape(-1, 2)
    ij = np.repeat(ij, ppc, axis=0)
    n = len(ij)

    def planes():
        for k in range(int(ncell[2])):
            rng = np.random.default_rng([seed, k])
            cells = np.column_stack([ij, np.full(n, k)])
            X = lo + cells + rng.random((n, 3))
            ue = rng.normal(0.0, u_th, (n, 3))
            up = rng.normal(0.0, u_th, (n, 3))
            yield (k, dict(_pack(X, ue, np.full(n, w), 3), q=-Q_E, m=M_E, immobile=False),
                   dict(_pack(X, up, np.full(n, w), 3), q=Q_E, m=M_P, immobile=False))

    return list(beam), planes()


def plasma_device(nphys, pml, d, ppc=8, u_th=0.01, species=("e", "p"), seed=SEED_BASE + 17, device="cuda"):
    """The thermal plasma of `plasma` drawn on the device, for boxes whose
    hundreds of millions of particles would take minutes to draw on the host:
    electrons and protons, ppc per physical cell each, uniform in the cell
    (protons on their electrons), Maxwellian u_th for both, weight
    n0 d^3 / ppc.  Draws come from torch's counter-based generator on
    `device` seeded with `seed` (species k uses seed + k for its momenta), so
    a run is reproducible on the same software stack.  Cells are in x-fastest
    order, ppc consecutive particles per cell.  Returns a list of dicts
    (cell (n, 3) int32, off (n, 3) float32, u (n, 3) float32, w scalar, q,
    m) of torch tensors on `device`.  The beam of `plasma` is drawn on the
    host (`plasma_beam`)."""
    import torch
    lo = [int(pml[0]), int(pml[2]), int(pml[4])]
    nx, ny, nz = (int(v) for v in nphys)
    n = nx * ny * nz * ppc
    w = plasma_density(u_th, d) * d ** 3 / ppc
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    idx = torch.arange(n, device=device, dtype=torch.int64) // ppc
    cell = torch.stack([idx % nx + lo[0], (idx // nx) % ny + lo[1], idx // (nx * ny) + lo[2]], 1).to(torch.int32)
    del idx
    off = torch.rand((n, 3), generator=g, device=device, dtype=torch.float32)
    out = []
    for k, sp in enumerate(species):
        g.manual_seed(int(seed) + 1 + k)
        u = torch.randn((n, 3), generator=g, device=device, dtype=torch.float32) * u_th
        q, m = (-Q_E, M_E) if sp == "e" else (Q_E, M_P)
        out.append(dict(cell=cell, off=off, u=u, w=w, q=q, m=m, immobile=False))
    return out


def plasma_beam(nphys, pml, d, ppc=8, u_th=0.01, beam_uz=5.0, beam_radius=16.0, beam_length=64.0,
                beam_density=0.1, seed=SEED_BASE + 19):
    """The drifting beam of `plasma` (and its immobile ions) alone, drawn on
    the host: the companion of `plasma_device`."""
    lo = np.array([pml[0], pml[2], pml[4]], dtype=np.float64)
    ncell = np.asarray(nphys, dtype=np.int64)
    w = plasma_density(u_th, d) * d ** 3 / ppc
    return list(_beam_cylinder(np.random.default_rng(seed), lo, ncell, ppc, w, beam_uz, beam_radius, beam_length,
                               beam_density))


def cavity_mask(nphys, pml, pipe_radius, cavity_radius, cavity_z):
    """Zeroed-field cells of a pillbox cavity on a beam pipe along z (the
    cavity run of Sec. III; the paper gives no geometry): every cell whose
    centre lies farther from the box's axis than the pipe radius, or than the
    cavity radius for physical z cells in cavity_z = (z0, z1), is a
    conductor; the pipe continues through the z PMLs.  Radii in cells.
    Returns a uint8 mask of shape (Nz, Ny, Nx) over the whole grid."""
    N = [n + pml[2 * a] + pml[2 * a + 1] for a, n in enumerate(nphys)]
    cx, cy = N[0] / 2.0, N[1] / 2.0
    i = np.arange(N[0])[None, None, :] + 0.5
    j = np.arange(N[1])[None, :, None] + 0.5
    k = np.arange(N[2])[:, None, None]
    r = np.sqrt((i - cx) ** 2 + (j - cy) ** 2)
    zin = (k >= pml[4] + cavity_z[0]) & (k < pml[4] + cavity_z[1])
    radius = np.where(zin, float(cavity_radius), float(pipe_radius))
    return np.broadcast_to(r > radius, (N[2], N[1], N[0])).astype(np.uint8)


def cavity_beam_slices(nphys, pml, steps, per_step, shift, sigma=2.0, gamma=479.0, charge=40e-9,
                       z_start=3.0, seed=SEED_BASE + 23):
    """The proton beam of the cavity run (Sec. III: 40 nC, gamma = 479,
    injected continuously on one side): `steps` slices of `per_step`
    macroparticles, slice s to be injected before step s.  Each slice is the
    stretch of a uniform-current beam that enters in one step: z uniform in
    [z_start, z_start + shift) cells (inside the entry face's PML; shift =
    the distance the beam moves in a step), transverse Gaussian of rms sigma
    cells about the axis (redrawn beyond 3 sigma), u along +z.  Weights give
    the total charge over all slices.  Returns dict(cell, off, u, w) of
    steps * per_step records, slices consecutive."""
    rng = np.random.default_rng(seed)
    n = steps * per_step
    N = [v + pml[2 * a] + pml[2 * a + 1] for a, v in enumerate(nphys)]
    d = rng.standard_normal((n, 2))
    bad = np.any(np.abs(d) > 3.0, axis=1)
    while bad.any():
        d[bad] = rng.standard_normal((int(bad.sum()), 2))
        bad = np.any(np.abs(d) > 3.0, axis=1)
    X = np.empty((n, 3))
    X[:, 0] = N[0] / 2.0 + sigma * d[:, 0]
    X[:, 1] = N[1] / 2.0 + sigma * d[:, 1]
    X[:, 2] = z_start + shift * rng.random(n)
    u = np.zeros((n, 3))
    u[:, 2] = np.sqrt(gamma * gamma - 1.0)
    w = np.full(n, charge / (Q_E * n))
    return _pack(X, u, w, 3)


def random_moves(n, lo, hi, max_step=0.95, seed=SEED_BASE + 9, w_range=(0.5, 4.0)):
    """Prescribed one-step moves for depositing in isolation: start positions
    uniform in [lo, hi) (cells, 3D), displacements uniform in +-max_step per
    axis, weights uniform in w_range.  Returns (cell0, off0, cell1, off1, w)
    with int32 cells and FP32 offsets / weights."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    X0 = lo + rng.random((n, 3)) * (hi - lo)
    c0, f0 = split_position(X0)
    X1 = absolute(c0, f0) + rng.uniform(-max_step, max_step, (n, 3))
    c1, f1 = split_position(X1)
    w = rng.uniform(w_range[0], w_range[1], n).astype(np.float32)
    return c0, f0, c1, f1, w


def batched_runs(nruns, size_range=(64, 256), pml_range=(8, 24), theta_max_deg=80.0,
                 gamma_range=(1.1, 100.0), seed=SEED_BASE + 5, q=-Q_E, m=M_E):
    """Independent 2D single-particle runs (the angle / gamma sweeps of the
    paper's single-particle studies): physical sizes nx, nz ~ U{lo..hi},
    PML width ~ U{lo..hi}, one electron at the box centre moving at an angle
    ~ U[0, theta_max] from +z with gamma log-uniform in gamma_range.
    Particle cells are relative to each run's own grid."""
    rng = np.random.default_rng(seed)
    nx = rng.integers(size_range[0], size_range[1] + 1, nruns)
    nz = rng.integers(size_range[0], size_range[1] + 1, nruns)
    npml = rng.integers(pml_range[0], pml_range[1] + 1, nruns)
    theta = rng.uniform(0.0, theta_max_deg, nruns)
    gamma = np.exp(rng.uniform(np.log(gamma_range[0]), np.log(gamma_range[1]), nruns))
    X = np.stack([npml + 0.5 * nx + rng.uniform(0.1, 0.9, nruns), np.zeros(nruns),
                  npml + 0.5 * nz + rng.uniform(0.1, 0.9, nruns)], axis=1)
    u = np.sqrt(gamma ** 2 - 1.0)
    th = np.radians(theta)
    U = np.stack([u * np.sin(th), np.zeros(nruns), u * np.cos(th)], axis=1)
    out = _pack(X, U, np.ones(nruns), 2)
    return dict(out, nx=nx, nz=nz, npml=npml, theta=theta, gamma=gamma, q=q, m=m)
