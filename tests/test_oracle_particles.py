"""Pins of the oracle's particle stages: gather, Boris push, Esirkepov deposit.

- Esirkepov deposition satisfies the discrete continuity equation exactly
  (App. A cites the charge-conserving Esirkepov scheme): checked against the
  oracle's node charge density, which is computed by a separate routine.
- For linear shapes and a straight move inside one cell, the current equals
  q w v times the time-averaged transverse shape, computed here by Gauss
  quadrature of the shape function along the trajectory.
- The summed current moment equals q w dX/dt for any shape order; a particle
  at rest deposits nothing.
- The gather reproduces uniform and linear fields exactly at the staggered
  Yee locations (partition of unity and first moment of the B-splines).
- Boris: in a uniform B the rotation per step is 2 atan(|t|) with |u| kept;
  a uniform E alone adds q E dt/(m c) to u; crossed E, B drift at E x B / B^2.
"""
import numpy as np
import pytest

import oracle as O

C = O.C_LIGHT


def _sim(dim, order, n=(12, 12, 12), pml=(0,) * 6, d=(1e-6, 1.2e-6, 0.9e-6)):
    dt = O.yee_dt(d, 0.9, dim)
    return O.OracleSim(dim, n, pml, d, dt, order=order, alpha_mode="one"), d, dt


def _rho_of(dim, order, X, qw, n=(12, 12, 12), d=(1e-6, 1.2e-6, 0.9e-6)):
    s, _, _ = _sim(dim, order, n=n, d=d)
    s.add_particles([X[0]], [X[1]], [X[2]], [0], [0], [0], [1.0], qw, O.M_E)
    return s.rho()


def _divJ(s, d, dim):
    Jx, Jy, Jz = s.field("Jx"), s.field("Jy"), s.field("Jz")
    div = np.zeros_like(Jx)
    div[:, :, 1:] += (Jx[:, :, 1:] - Jx[:, :, :-1]) / d[0]
    div[1:, :, :] += (Jz[1:, :, :] - Jz[:-1, :, :]) / d[2]
    if dim == 3:
        div[:, 1:, :] += (Jy[:, 1:, :] - Jy[:, :-1, :]) / d[1]
    return div


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("order", [1, 3])
def test_esirkepov_continuity(dim, order):
    rng = np.random.default_rng(11 + dim + order)
    for trial in range(20):
        s, d, dt = _sim(dim, order)
        X0 = np.array([4 + 3 * rng.random(), 4 + 3 * rng.random() if dim == 3 else 0.0, 4 + 3 * rng.random()])
        dX = rng.uniform(-0.95, 0.95, 3)
        if dim == 2:
            dX[1] = 0.0
        X1 = X0 + dX
        qw = -O.Q_E * 3.0
        s.esirkepov(X0, X1, qw, vy=0.37 * C)
        r0 = _rho_of(dim, order, X0, qw, d=d)
        r1 = _rho_of(dim, order, X1, qw, d=d)
        resid = (r1 - r0) / dt + _divJ(s, d, dim)
        scale = np.abs(r1 - r0).max() / dt
        assert np.abs(resid).max() < 1e-13 * scale, np.abs(resid).max() / scale


def _gl(n=12):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


@pytest.mark.parametrize("dim", [3, 2])
def test_linear_shape_flux_equals_time_averaged_shape(dim):
    rng = np.random.default_rng(3)
    t, wq = _gl()
    S = lambda r: max(0.0, 1 - abs(r))
    for trial in range(10):
        s, d, dt = _sim(dim, 1)
        base = np.array([5.0, 5.0 if dim == 3 else 0.0, 6.0])
        f0 = rng.uniform(0.05, 0.95, 3)
        f1 = rng.uniform(0.05, 0.95, 3)
        if dim == 2:
            f0[1] = f1[1] = 0.0
        X0, X1 = base + f0, base + f1
        qw = O.Q_E
        vy = -0.2 * C
        s.esirkepov(X0, X1, qw, vy=vy)
        Jx = s.field("Jx")
        V = d[0] * d[2] * (d[1] if dim == 3 else 1.0)
        vx = (X1[0] - X0[0]) * d[0] / dt
        ys = [5, 6] if dim == 3 else [0]
        for jj in ys:
            for kk in (6, 7):
                # time average of S(y(t)-j) S(z(t)-k) along the straight move
                avg = 0.0
                for tt, ww in zip(t, wq):
                    X = X0 + tt * (X1 - X0)
                    sy = S(X[1] - jj) if dim == 3 else 1.0
                    avg += ww * sy * S(X[2] - kk)
                expect = qw * vx * avg / V
                assert Jx[kk, jj, 5] == pytest.approx(expect, rel=1e-12, abs=1e-12 * abs(qw * vx / V))
        if dim == 2:
            Jy = s.field("Jy")
            for ii in (5, 6):
                for kk in (6, 7):
                    avg = 0.0
                    for tt, ww in zip(t, wq):
                        X = X0 + tt * (X1 - X0)
                        avg += ww * S(X[0] - ii) * S(X[2] - kk)
                    assert Jy[kk, 0, ii] == pytest.approx(qw * vy * avg / V, rel=1e-12)


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("order", [1, 3])
def test_current_moment_and_rest(dim, order):
    rng = np.random.default_rng(7)
    s, d, dt = _sim(dim, order)
    X0 = np.array([5.3, 5.6 if dim == 3 else 0.0, 6.1])
    dX = np.array([0.7, -0.4 if dim == 3 else 0.0, -0.9])
    qw = -O.Q_E
    s.esirkepov(X0, X0 + dX, qw)
    V = d[0] * d[2] * (d[1] if dim == 3 else 1.0)
    for c, a in enumerate("xyz"):
        if dim == 2 and a == "y":
            continue
        tot = s.field("J" + a).sum() * V
        assert tot == pytest.approx(qw * dX[c] * d[c] / dt, rel=1e-13)
    s2, d, dt = _sim(dim, order)
    s2.esirkepov(X0, X0, qw)
    for a in "xyz":
        assert np.abs(s2.field("J" + a)).max() == 0.0


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("order", [1, 3])
def test_gather_reproduces_linear_fields(dim, order):
    s, d, dt = _sim(dim, order)
    nx, ny, nz = s.nn
    i = np.arange(nx)[None, None, :] * 1.0
    j = np.arange(ny)[None, :, None] * 1.0
    k = np.arange(nz)[:, None, None] * 1.0
    shp = (nz, ny, nx)
    coef = {"x": (1.0, 0.3, -0.2, 0.5), "y": (2.0, -0.1, 0.4, 0.2), "z": (-1.0, 0.25, 0.1, -0.3)}
    stagE = {"x": (0.5, 0, 0), "y": (0, 0.5, 0), "z": (0, 0, 0.5)}
    stagB = {"x": (0, 0.5, 0.5), "y": (0.5, 0, 0.5), "z": (0.5, 0.5, 0)}
    if dim == 2:
        stagE = {a: (o[0], 0, o[2]) for a, o in stagE.items()}
        stagB = {a: (o[0], 0, o[2]) for a, o in stagB.items()}

    def lin(a, st):
        c0, cx, cy, cz = coef[a]
        return np.broadcast_to(c0 + cx * (i + st[0]) + cy * (j + st[1]) * (dim == 3) + cz * (k + st[2]), shp)

    for a in "xyz":
        s.set_field("E" + a, lin(a, stagE[a]))
        s.set_field("Bh" + a, 2 * lin(a, stagB[a]))
        s.set_field("Bp" + a, 0 * lin(a, stagB[a]))
    rng = np.random.default_rng(1)
    for _ in range(10):
        X = np.array([4 + 4 * rng.random(), 4 + 4 * rng.random() if dim == 3 else 0.0, 4 + 4 * rng.random()])
        E, B = s.gather(X)
        for c, a in enumerate("xyz"):
            c0, cx, cy, cz = coef[a]
            expect = c0 + cx * X[0] + cy * X[1] * (dim == 3) + cz * X[2]
            assert E[c] == pytest.approx(expect, rel=1e-13, abs=1e-13)
            # B^n is the mean of the two half-step arrays (2 L and 0)
            assert B[c] == pytest.approx(expect, rel=1e-13, abs=1e-13)


def test_boris_uniform_B_rotation():
    q, m, dt = -O.Q_E, O.M_E, 1e-15
    B = np.array([0.0, 0.0, 50.0])
    u = np.array([0.8, 0.0, 0.3])
    g = np.sqrt(1 + u @ u)
    u1 = O.boris(u, [0, 0, 0], B, q, m, dt)
    tmag = abs(q * dt * B[2] / (2 * m * g))
    angle = np.arctan2(u1[1], u1[0]) - np.arctan2(u[1], u[0])
    # electrons gyrate counter-clockwise about +z (q < 0)
    assert abs(angle) == pytest.approx(2 * np.arctan(tmag), rel=1e-12)
    assert np.sign(angle) == -np.sign(q * B[2])
    assert np.linalg.norm(u1) == pytest.approx(np.linalg.norm(u), rel=1e-14)
    assert u1[2] == u[2]


def test_boris_uniform_E_kick():
    q, m, dt = O.Q_E, O.M_P, 2e-15
    E = np.array([1e9, -3e8, 2e9])
    u = np.array([0.1, 0.2, -0.3])
    u1 = O.boris(u, E, [0, 0, 0], q, m, dt)
    np.testing.assert_allclose(u1, u + q * E * dt / (m * C), rtol=1e-14)


def test_boris_ExB_drift():
    q, m = O.Q_E, O.M_P
    B = np.array([0.0, 0.0, 1.0])
    E = np.array([1e5, 0.0, 0.0])  # drift speed E/B = 1e5 m/s, along -y
    wc = q * B[2] / m
    dt = 0.02 / wc
    u = np.zeros(3)
    uavg = np.zeros(3)
    nper = int(round(2 * np.pi / (wc * dt)))
    n = nper * 40
    for _ in range(n):
        u = O.boris(u, E, B, q, m, dt)
        uavg += u
    uavg /= n
    vd = np.cross(E, B) / (B @ B)
    np.testing.assert_allclose(uavg * C, vd, rtol=2e-3, atol=2e-3 * np.linalg.norm(vd))


def test_threaded_oracle_equals_serial_up_to_summation_order():
    """The oracle's threaded loops (per-thread current arrays summed in thread
    order) give the serial result up to the order of the floating-point sums,
    and the same bits on a repeat with the same thread count."""
    import oracle as O
    from paper_2201_09084_gb300 import inputs as I
    D = (1e-6, 1.1e-6, 0.9e-6)
    nphys, pml = (12, 10, 14), (4,) * 6
    parts = I.random_particles(3, 3000, [3, 3, 3], [17, 15, 19], u_rms=0.6, seed=21)[0]
    dt = O.yee_dt(D, 0.95, 3)
    out = {}
    try:
        for label, T in (("serial", 1), ("t4", 4), ("t4b", 4)):
            O.set_threads(T)
            s = O.OracleSim(3, nphys, pml, D, dt, order=3, alpha_mode="damped")
            X = I.absolute(parts["cell"], parts["off"])
            u = parts["u"].astype(np.float64)
            s.add_particles(X[:, 0], X[:, 1], X[:, 2], u[:, 0], u[:, 1], u[:, 2], parts["w"].astype(np.float64),
                            parts["q"], parts["m"])
            s.step(8)
            out[label] = {k: s.field(k) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx")}
    finally:
        O.set_threads(1)
    for k, a in out["serial"].items():
        scale = np.abs(a).max()
        assert scale > 0
        assert np.abs(out["t4"][k] - a).max() <= 1e-12 * scale, k
        assert np.array_equal(out["t4"][k], out["t4b"][k]), k
