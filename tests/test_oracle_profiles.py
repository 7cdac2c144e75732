"""Pins of the oracle's PML profiles: Eq. conductivity and Eq. alpha.

Checked against what the paper fixes rather than against the oracle's own
formulas: the closed-form consequences of Eq. alpha for the App. A profile,
the defining ODE d(alpha)/dz = -sigma alpha/(eps0 v) with alpha(0) = 1
(App. B, condition on alpha), evaluated by finite differences, and the
Fourier-space statement that the ansatz fields of Eq. PMLfield solve the PML
equations only when chi = 1 (App. B).
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "app_a_profiles.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            name, coef, delta, p, cells = line.split()
            rows.append((name, float(coef), float(delta), float(p), int(cells)))
    return rows


def test_alpha_closed_form_values():
    # App. A profile sigma = (4 eps0 c/dz)(z/6dz)^2 with v = c gives
    # alpha(d) = exp(-d^3/27): alpha(3 cells) = 1/e, alpha(6 cells) = e^-8.
    assert O.alpha(0.0) == 1.0
    assert abs(O.alpha(3.0) - np.exp(-1.0)) < 1e-15
    assert abs(O.alpha(6.0) - np.exp(-8.0)) < 1e-17
    assert abs(O.alpha(1.0) - 0.9636404443012863) < 1e-15
    # monotonically decreasing from 1 at the interface towards 0 (Sec. II.A)
    vals = [O.alpha(d) for d in np.linspace(0, 16, 200)]
    assert all(a > b for a, b in zip(vals[:-1], vals[1:]))
    assert vals[-1] < 1e-60


@pytest.mark.parametrize("name,coef,delta,p,cells", _golden())
def test_app_a_profiles(name, coef, delta, p, cells):
    """Golden fixture: the three PML profiles of App. A.  alpha at every
    quarter cell equals exp(-int sigma/(eps0 c) dz) computed by adaptive
    quadrature of the conductivity (Eq. alpha with v = c)."""
    from scipy.integrate import quad
    Delta = 1e-6
    for dcells in np.arange(0.25, cells + 0.01, 0.25):
        integral, _ = quad(lambda zc: O.sigma_over_eps0(zc, Delta, coef, delta, p) * Delta / O.C_LIGHT,
                           0.0, dcells, epsabs=0, epsrel=1e-13)
        a = O.alpha(dcells, coef=coef, delta=delta, p=p)
        assert a == pytest.approx(np.exp(-integral), rel=1e-10)
    # sigma itself: coef eps0 c/dz at depth delta
    assert O.sigma_over_eps0(delta, Delta, coef, delta, p) == pytest.approx(coef * O.C_LIGHT / Delta, rel=1e-15)


@pytest.mark.parametrize("coef,delta,p,vfrac", [(4, 6, 2, 1.0), (4, 10, 2, 1.0),
                                                (4, 6, 2, 0.3), (2.5, 8, 3, 0.7)])
def test_alpha_solves_defining_ode(coef, delta, p, vfrac):
    # d alpha/dz = -sigma(z) alpha(z) / (eps0 v), alpha(0) = 1  (App. B)
    Delta = 1e-6
    v = vfrac * O.C_LIGHT
    h = 1e-5
    for d in np.linspace(0.3, 9.0, 25):
        a = O.alpha(d, coef, delta, p, v)
        dadz = (O.alpha(d + h, coef, delta, p, v) - O.alpha(d - h, coef, delta, p, v)) / (2 * h * Delta)
        s = O.sigma_over_eps0(d, Delta, coef, delta, p)
        rhs = -s * a / v
        assert dadz == pytest.approx(rhs, rel=1e-6, abs=1e-300)


def test_sigma_profile_eq_conductivity():
    # sigma(z) = (4 eps0 c/dz) (z/(6 dz))^2: at depth 6 cells sigma/eps0 = 4c/dz
    Delta = 1e-6
    assert O.sigma_over_eps0(6.0, Delta) == pytest.approx(4 * O.C_LIGHT / Delta, rel=1e-15)
    assert O.sigma_over_eps0(3.0, Delta) == pytest.approx(O.C_LIGHT / Delta, rel=1e-15)
    assert O.sigma_over_eps0(0.0, Delta) == 0.0
    assert O.sigma_over_eps0(-2.0, Delta) == 0.0


def test_alpha_modes():
    assert O.alpha(2.0, mode="zero") == 0.0 and O.alpha(0.0, mode="zero") == 1.0
    assert O.alpha(2.0, mode="one") == 1.0


def _ansatz_residuals(alpha_fn, sigma_fn, v, gamma, kx, ky, w, z, h):
    """Residuals of the Fourier-space PML equations (App. B) for the ansatz
    fields of Eq. FourierPMLfield with splits of Eqs. FourierSplitE/B.
    Uses the field expressions as printed in App. B; returns the largest
    relative residual of the split-sum equations (Eq. FourierMaxwellSum) and
    of the z-derivative equations."""
    q, eps0, c = 1.0, 1.0, 1.0

    def a(zz):
        return alpha_fn(zz)

    def dadz(zz):
        return (a(zz + h) - a(zz - h)) / (2 * h)

    def common(zz):
        return np.exp(1j * w * zz / v) / (kx ** 2 + ky ** 2 + w ** 2 / (gamma * v) ** 2)

    def chi(zz):
        return (1j * w + v / a(zz) * dadz(zz)) / (1j * w - sigma_fn(zz) / eps0)

    def E(zz):
        f = -1j * a(zz) * q / (eps0 * v) * common(zz)
        return f * np.array([kx, ky, w / (gamma ** 2 * v)])

    def B(zz):
        f = -1j * a(zz) * q / (eps0 * c ** 2) * common(zz)
        return f * np.array([-ky, kx, 0.0])

    def splitE(zz):
        f = -1j * a(zz) * q / (eps0 * v) * common(zz)
        ch = chi(zz)
        return f * np.array([0.0, ch * kx, ch * ky, 0.0])  # xy, xz, yz, yx

    def splitB(zz):
        f = -1j * a(zz) * q / (eps0 * v ** 2) * common(zz)
        ch = chi(zz)
        return f * np.array([ky / gamma ** 2, -ch * ky, ch * kx, -kx / gamma ** 2])

    res = []
    Ez, Ez_ = E(z), splitE(z)
    Bz_, Bs = B(z), splitB(z)
    # Eq. FourierMaxwellSum: E_x = E_xy + E_xz, E_y = E_yz + E_yx, B likewise
    res.append(abs(Ez[0] - (Ez_[0] + Ez_[1])) / abs(Ez[0]))
    res.append(abs(Ez[1] - (Ez_[2] + Ez_[3])) / abs(Ez[1]))
    res.append(abs(Bz_[0] - (Bs[0] + Bs[1])) / abs(Bz_[0]))
    res.append(abs(Bz_[1] - (Bs[2] + Bs[3])) / abs(Bz_[1]))
    # z-derivative equation for E_xz: -iw E_xz = -c^2 dBy/dz - sigma/eps0 E_xz
    dBy = (B(z + h)[1] - B(z - h)[1]) / (2 * h)
    lhs = -1j * w * Ez_[1]
    rhs = -c ** 2 * dBy - sigma_fn(z) / eps0 * Ez_[1]
    res.append(abs(lhs - rhs) / abs(lhs))
    # and for B_yz: -iw B_yz = -dEx/dz - sigma/eps0 B_yz
    dEx = (E(z + h)[0] - E(z - h)[0]) / (2 * h)
    lhs = -1j * w * Bs[2]
    rhs = -dEx - sigma_fn(z) / eps0 * Bs[2]
    res.append(abs(lhs - rhs) / abs(lhs))
    return max(res)


@pytest.mark.parametrize("vfrac", [1.0, 0.6])
def test_fourier_ansatz_requires_eq_alpha(vfrac):
    """App. B: with alpha of Eq. alpha, chi = 1 and the ansatz solves the PML
    equations; with a mismatched alpha (velocity halved) it does not."""
    # dimensionless units: c = eps0 = 1, Delta = 1
    v = vfrac
    gamma = 1.0 / np.sqrt(1 - v ** 2) if v < 1 else 10.0
    if v >= 1:
        v = np.sqrt(1 - 1 / gamma ** 2)
    Delta = 1.0
    sig = lambda zz: O.sigma_over_eps0(zz / Delta, Delta) / O.C_LIGHT  # c = 1 units
    good = lambda zz: O.alpha(zz / Delta, v=v * O.C_LIGHT)
    bad = lambda zz: O.alpha(zz / Delta, v=0.5 * v * O.C_LIGHT)
    for z in (0.7, 2.0, 4.5):
        for (kx, ky, w) in ((0.3, 0.2, 0.5), (1.1, -0.4, 2.0)):
            r_good = _ansatz_residuals(good, sig, v, gamma, kx, ky, w, z, 1e-5)
            r_bad = _ansatz_residuals(bad, sig, v, gamma, kx, ky, w, z, 1e-5)
            assert r_good < 1e-7, r_good
            assert r_bad > 1e-2, r_bad


def test_tables_staggering():
    """Sec. II.B: alpha and sigma at nodes and cell centres; the interface is
    the last physical node (depth 0)."""
    d = (1e-6, 1e-6, 1e-6)
    s = O.OracleSim(3, (10, 12, 14), (4, 5, 0, 3, 6, 8), d, 1e-16)
    pl, n = 6, 14  # z axis: 6 cells low, 14 physical, 8 high
    an = s.table("a_node", 2)
    ac = s.table("a_cent", 2)
    sn = s.table("s_node", 2)
    assert len(an) == pl + n + 8 + 1
    for i in range(len(an)):
        dn = max(pl - i, i - (pl + n), 0)
        assert an[i] == pytest.approx(np.exp(-dn ** 3 / 27.0), rel=1e-14)
        assert sn[i] == pytest.approx(4 * O.C_LIGHT / 1e-6 * (dn / 6.0) ** 2, rel=1e-14)
    for i in range(len(ac) - 1):
        x = i + 0.5
        dc = max(pl - x, x - (pl + n), 0)
        assert ac[i] == pytest.approx(np.exp(-dc ** 3 / 27.0), rel=1e-14)
    # y axis: no PML at -y, 3 cells at +y
    an_y = s.table("a_node", 1)
    assert np.all(an_y[:13] == 1.0) and an_y[13] < 1.0
