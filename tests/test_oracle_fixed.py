"""Pins of the oracle's deterministic (int64 fixed-point) deposition, 3D.

The integer currents are Esirkepov's decomposition (App. A) evaluated in
integers on FP32 shape values quantised to 2^-20.  They are pinned by:
- the quantised shapes against the FP64 B-spline of the oracle's own
  floating-point path (a separate routine): within 0.75 quantum per node for
  order 1 and 2.25 for order 3 (one node per axis takes the remainder of the
  partition of unity, collecting the other nodes' rounding);
- the continuity equation, which the integer decomposition must satisfy
  EXACTLY: sum of the backward differences of the raw currents equals the
  change of the integer node charge 6 S S S, for random moves crossing cells
  on every axis, orders 1 and 3;
- the FP64 Esirkepov current of the floating-point oracle for the same moves,
  after conversion to A/m^2: equal within the quantisation error;
- sign and translation: qn -> -qn negates every integer; shifting the moves
  by whole cells shifts the currents by the same cells, bit for bit.
"""
import numpy as np
import pytest

import oracle as O

NN = (14, 13, 12)


def _moves(rng, n, order, lo=4, hi=7):
    cell0 = rng.integers(lo, hi, size=(n, 3))
    off0 = rng.random((n, 3)).astype(np.float32)
    d = rng.uniform(-0.95, 0.95, size=(n, 3))
    x1 = cell0 + off0.astype(np.float64) + d
    cell1 = np.floor(x1).astype(np.int64)
    off1 = (x1 - cell1).astype(np.float32)
    # an FP32 offset that rounded up to 1.0 belongs to the next cell
    up = off1 >= 1.0
    cell1[up] += 1
    off1[up] = 0.0
    return cell0, off0, cell1, off1


def _bspline_weights(order, f):
    """FP64 node weights of an offset f from the oracle's shape function."""
    if order == 1:
        return [O.shape(1, f), O.shape(1, 1.0 - f)]
    return [O.shape(3, 1.0 + f), O.shape(3, f), O.shape(3, 1.0 - f), O.shape(3, 2.0 - f)]


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_shapes_match_fp64_bspline(order):
    rng = np.random.default_rng(5 + order)
    q = 2.0 ** O.FIXED_SHAPE_BITS
    lo = 1 if order == 3 else 0
    for _ in range(40):
        cell = np.array([[5, 6, 4]])
        off = rng.random((1, 3)).astype(np.float32)
        rho = O.fixed_rho3d(order, cell, off, NN)
        w = [_bspline_weights(order, float(off[0, a])) for a in range(3)]
        exp = np.zeros(NN[::-1])
        for tk in range(order + 1):
            for tj in range(order + 1):
                for ti in range(order + 1):
                    exp[4 - lo + tk, 6 - lo + tj, 5 - lo + ti] = 6 * q ** 3 * w[0][ti] * w[1][tj] * w[2][tk]
        # each quantised shape is within e quanta: the product within 3 e q^2
        e = 0.75 if order == 1 else 2.25
        assert np.max(np.abs(rho - exp)) <= 6 * 3 * e * q * q
        assert np.sum(rho) == 6 * 2 ** (3 * O.FIXED_SHAPE_BITS)
        assert np.count_nonzero(exp) == (order + 1) ** 3


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_continuity_exact(order):
    rng = np.random.default_rng(17 + order)
    c0, f0, c1, f1 = _moves(rng, 25, order)
    # every axis sees crossings in both directions among the moves
    assert all(np.any(c1[:, a] > c0[:, a]) and np.any(c1[:, a] < c0[:, a]) for a in range(3))
    w = np.ones(len(c0), np.float32)
    Jx, Jy, Jz = O.fixed_deposit3d(order, c0, f0, c1, f1, w, 1.0, NN, raw=True)
    r0 = O.fixed_rho3d(order, c0, f0, NN)
    r1 = O.fixed_rho3d(order, c1, f1, NN)
    div = np.zeros_like(Jx)
    div[:, :, 0] += Jx[:, :, 0]
    div[:, :, 1:] += Jx[:, :, 1:] - Jx[:, :, :-1]
    div[:, 0, :] += Jy[:, 0, :]
    div[:, 1:, :] += Jy[:, 1:, :] - Jy[:, :-1, :]
    div[0, :, :] += Jz[0, :, :]
    div[1:, :, :] += Jz[1:, :, :] - Jz[:-1, :, :]
    assert np.array_equal(div, r1 - r0)
    assert np.count_nonzero(Jx) and np.count_nonzero(Jy) and np.count_nonzero(Jz)


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_matches_fp64_esirkepov(order):
    rng = np.random.default_rng(29 + order)
    d = (1e-6, 1.2e-6, 0.9e-6)
    dt = O.yee_dt(d, 0.9, 3)
    n = (NN[0] - 1, NN[1] - 1, NN[2] - 1)
    s = O.OracleSim(3, n, (0,) * 6, d, dt, order=order, alpha_mode="one")
    c0, f0, c1, f1 = _moves(rng, 12, order)
    w = rng.uniform(0.5, 3.0, len(c0)).astype(np.float32)
    qn = -1.0
    for p in range(len(c0)):
        X0 = c0[p] + f0[p].astype(np.float64)
        X1 = c1[p] + f1[p].astype(np.float64)
        s.esirkepov(X0, X1, qn * O.Q_E * float(w[p]))
    J = O.fixed_deposit3d(order, c0, f0, c1, f1, w, qn, NN)
    area = (d[1] * d[2], d[0] * d[2], d[0] * d[1])
    for c, name in enumerate("xyz"):
        ref = s.field("J" + name)
        got = -(O.Q_E / (area[c] * dt)) * J[c].astype(np.float64) / O.FIXED_UNIT
        scale = np.max(np.abs(ref))
        assert scale > 0
        assert np.max(np.abs(got - ref)) <= 2e-5 * scale, name


def test_fixed_sign_and_translation():
    rng = np.random.default_rng(41)
    for order in (1, 3):
        c0, f0, c1, f1 = _moves(rng, 10, order)
        w = rng.uniform(0.1, 10.0, len(c0)).astype(np.float32)
        a = O.fixed_deposit3d(order, c0, f0, c1, f1, w, 2.0, NN)
        b = O.fixed_deposit3d(order, c0, f0, c1, f1, w, -2.0, NN)
        for x, y in zip(a, b):
            assert np.array_equal(x, -y)
        sh = np.array([1, 2, -1])
        t = O.fixed_deposit3d(order, c0 + sh, f0, c1 + sh, f1, w, 2.0, NN)
        for x, y in zip(a, t):
            assert np.array_equal(np.roll(x, (-1, 2, 1), axis=(0, 1, 2)), y)


def test_fixed_weighted_is_rounded_raw():
    """One particle: the weighted integers are the raw ones times w qn 2^-36,
    rounded once."""
    rng = np.random.default_rng(53)
    c0, f0, c1, f1 = _moves(rng, 1, 3)
    w = np.array([0.37], np.float32)
    raw = O.fixed_deposit3d(3, c0, f0, c1, f1, w, 1.0, NN, raw=True)
    val = O.fixed_deposit3d(3, c0, f0, c1, f1, w, 3.0, NN)
    for r, v in zip(raw, val):
        exact = r.astype(np.float64) * (float(w[0]) * 3.0) * 2.0 ** -36
        assert np.max(np.abs(v - exact)) <= 0.5 + 1e-9 * np.max(np.abs(exact))


# 2D (x, z) boxes: J_x, J_z from the in-plane integer sums, J_y from the
# mid-move shape product times v_y/c (formed in FP64 from the FP32 momentum)

NN2 = (14, 13)   # nodes along x, z


def _moves2d(rng, n, order):
    c0, f0, c1, f1 = _moves(rng, n, order)
    for a in (c0, c1):
        a[:, 1] = 0
    f0[:, 1] = 0.0
    f1[:, 1] = 0.0
    return c0, f0, c1, f1


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_continuity_exact_2d(order):
    rng = np.random.default_rng(61 + order)
    c0, f0, c1, f1 = _moves2d(rng, 25, order)
    assert all(np.any(c1[:, a] > c0[:, a]) and np.any(c1[:, a] < c0[:, a]) for a in (0, 2))
    w = np.ones(len(c0), np.float32)
    u = np.zeros((len(c0), 3), np.float32)
    Jx, Jy, Jz = O.fixed_deposit2d(order, c0, f0, c1, f1, w, u, 1.0, NN2, raw=True)
    r0 = O.fixed_rho2d(order, c0, f0, NN2)
    r1 = O.fixed_rho2d(order, c1, f1, NN2)
    div = np.zeros_like(Jx)
    div[:, 0] += Jx[:, 0]
    div[:, 1:] += Jx[:, 1:] - Jx[:, :-1]
    div[0, :] += Jz[0, :]
    div[1:, :] += Jz[1:, :] - Jz[:-1, :]
    assert np.array_equal(div, r1 - r0)
    assert np.count_nonzero(Jx) and np.count_nonzero(Jz)
    # the raw out-of-plane values: the mid-move shape sums to 6 2^40 per move
    assert Jy.sum() == 6 * 2 ** (2 * O.FIXED_SHAPE_BITS) * len(c0)


@pytest.mark.parametrize("order", [1, 3])
def test_fixed_matches_fp64_esirkepov_2d(order):
    rng = np.random.default_rng(71 + order)
    d = (1e-6, 1.0, 0.9e-6)
    dt = O.yee_dt(d, 0.9, 2)
    n = (NN2[0] - 1, 0, NN2[1] - 1)
    s = O.OracleSim(2, n, (0,) * 6, d, dt, order=order, alpha_mode="one")
    c0, f0, c1, f1 = _moves2d(rng, 12, order)
    w = rng.uniform(0.5, 3.0, len(c0)).astype(np.float32)
    u = rng.normal(0.0, 2.0, (len(c0), 3)).astype(np.float32)
    qn = -1.0
    for p in range(len(c0)):
        X0 = c0[p] + f0[p].astype(np.float64)
        X1 = c1[p] + f1[p].astype(np.float64)
        ud = u[p].astype(np.float64)
        vyc = ud[1] / np.sqrt(((1.0 + ud[0] * ud[0]) + ud[1] * ud[1]) + ud[2] * ud[2])
        s.esirkepov(X0, X1, qn * O.Q_E * float(w[p]), O.C_LIGHT * vyc)
    Jx, Jy, Jz = O.fixed_deposit2d(order, c0, f0, c1, f1, w, u, qn, NN2)
    got = {"x": -(O.Q_E / (d[2] * dt)) * Jx / O.FIXED_UNIT,
           "z": -(O.Q_E / (d[0] * dt)) * Jz / O.FIXED_UNIT,
           "y": (O.Q_E * O.C_LIGHT / (d[0] * d[2])) * Jy / O.FIXED_UNIT}
    for c in "xyz":
        ref = s.field("J" + c)[:, 0, :]
        scale = np.max(np.abs(ref))
        assert scale > 0
        assert np.max(np.abs(got[c] - ref)) <= 2e-5 * scale, c


def test_fixed_2d_sign_translation_and_order():
    rng = np.random.default_rng(83)
    for order in (1, 3):
        c0, f0, c1, f1 = _moves2d(rng, 10, order)
        w = rng.uniform(0.1, 10.0, len(c0)).astype(np.float32)
        u = rng.normal(0.0, 1.0, (len(c0), 3)).astype(np.float32)
        a = O.fixed_deposit2d(order, c0, f0, c1, f1, w, u, 2.0, NN2)
        b = O.fixed_deposit2d(order, c0, f0, c1, f1, w, u, -2.0, NN2)
        for x, y in zip(a, b):
            assert np.array_equal(x, -y)
        sh = np.array([2, 0, -1])
        t = O.fixed_deposit2d(order, c0 + sh, f0, c1 + sh, f1, w, u, 2.0, NN2)
        for x, y in zip(a, t):
            assert np.array_equal(np.roll(x, (-1, 2), axis=(0, 1)), y)
        perm = rng.permutation(len(c0))
        r = O.fixed_deposit2d(order, c0[perm], f0[perm], c1[perm], f1[perm], w[perm], u[perm], 2.0, NN2)
        for x, y in zip(a, r):
            assert np.array_equal(x, y)
