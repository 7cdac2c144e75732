"""Pins of the oracle's binomial current filter (App. A: a binomial filter is
applied to the deposited current before the field update; Birdsall and
Langdon's (1, 2, 1)/4 stencil, one pass per axis).

- impulse response: a unit value spreads into the binomial weights
  (1, 2, 1)/4 along every active axis (their outer product), nothing else;
- transfer function: a cosine of wavenumber k along x keeps its shape and is
  scaled by (1 + cos k dx)/2 = cos^2(k dx / 2) per pass, away from the edges;
- filter_passes = 2 equals two single passes;
- Gauss law with the filter: the filtered current conserves the filtered
  charge, so div E = F(rho)/eps0 in the interior to round-off, while div E
  differs from rho/eps0 itself.
"""
import numpy as np
import pytest

import oracle as O

D3 = (1e-6, 1.1e-6, 0.9e-6)


def _box(dim=3, passes=0, n=(12, 10, 14), pml=(0,) * 6, mode="one", order=1):
    dt = O.yee_dt(D3, 0.95, dim)
    return O.OracleSim(dim, n, pml, D3, dt, order=order, alpha_mode=mode, sig_coef=1e-20, filter_passes=passes)


@pytest.mark.parametrize("dim", [3, 2])
def test_impulse_response_is_binomial(dim):
    s = _box(dim)
    nn = s.nn
    for comp in "xyz":
        J = np.zeros((nn[2], nn[1], nn[0]))
        k, j, i = 6, (5 if dim == 3 else 0), 4
        J[k, j, i] = 1.0
        s.set_field("J" + comp, J)
        s.filter_J()
        out = s.field("J" + comp)
        w = np.array([0.25, 0.5, 0.25])
        exp = np.zeros_like(J)
        for dk in range(3):
            for dj in (range(3) if dim == 3 else [1]):
                for di in range(3):
                    wy = w[dj] if dim == 3 else 1.0
                    exp[k + dk - 1, j + dj - 1 if dim == 3 else 0, i + di - 1] = w[dk] * wy * w[di]
        assert np.allclose(out, exp, rtol=0, atol=1e-15), comp
        assert out.sum() == pytest.approx(1.0, abs=1e-14)


def test_transfer_function_of_a_cosine():
    s = _box(3)
    nn = s.nn
    kdx = 2 * np.pi / 7.0
    i = np.arange(nn[0])
    J = np.broadcast_to(np.cos(kdx * i)[None, None, :], (nn[2], nn[1], nn[0])).copy()
    s.set_field("Jz", J)
    s.filter_J()
    out = s.field("Jz")
    # away from every edge (zero padding there) the pattern is scaled
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.allclose(out[inner], np.cos(kdx / 2) ** 2 * J[inner], rtol=0, atol=1e-14)


def test_two_passes_are_two_filters():
    rng = np.random.default_rng(4)
    a = _box(3)
    nn = a.nn
    J = rng.normal(size=(nn[2], nn[1], nn[0]))
    a.set_field("Jy", J)
    a.filter_J()
    a.filter_J()
    b = _box(3)
    b.set_field("Jy", J)
    b.filter_J()
    c = _box(3)
    c.set_field("Jy", b.field("Jy"))
    c.filter_J()
    assert np.array_equal(a.field("Jy"), c.field("Jy"))


def _binomial(r, dim):
    """The filter applied to a node array [k, j, i] with zero padding."""
    out = r.copy()
    for ax in ((0, 1, 2) if dim == 3 else (0, 2)):
        p = np.pad(out, [(1, 1) if a == ax else (0, 0) for a in range(3)])
        sl = lambda o: tuple(slice(1 + o, p.shape[a] - 1 + o) if a == ax else slice(None) for a in range(3))
        out = 0.25 * p[sl(-1)] + 0.5 * p[sl(0)] + 0.25 * p[sl(1)]
    return out


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("order", [1, 3])
def test_gauss_law_holds_for_the_filtered_charge(dim, order):
    s = _box(dim, passes=1, n=(14, 12, 16), pml=(4,) * 6, order=order)
    rng = np.random.default_rng(dim + 7 * order)
    for _ in range(4):
        X = np.array([8 + 6 * rng.random(), (8 + 4 * rng.random()) if dim == 3 else 0.0, 8 + 6 * rng.random()])
        u = rng.normal(size=3) * 0.4
        s.add_particles([X[0]], [X[1]], [X[2]], [u[0]], [u[1]], [u[2]], [1.0], -O.Q_E, O.M_E)
        s.add_particles([X[0]], [X[1]], [X[2]], [0.0], [0.0], [0.0], [1.0], O.Q_E, O.M_E, True)
    s.step(12)
    assert s.particles()["alive"].all()
    rho = s.rho() / O.EPS0
    scale = np.abs(rho).max()
    r_f = s.divE() - _binomial(rho, dim)
    r_0 = s.divE() - rho
    cut = (slice(2, -2), slice(2, -2) if dim == 3 else slice(None), slice(2, -2))
    assert np.abs(r_f[cut]).max() < 1e-10 * scale
    assert np.abs(r_0[cut]).max() > 1e-2 * scale
