"""Pins of the oracle's zeroed-field (perfect conductor) cells.

The cavity run of Sec. III has cells where the fields are zero; the paper
gives no geometry, so a conductor is a set of marked cells whose 12 edges
carry E = 0 after every E update.  A cavity carved out of a larger box by
conductor cells then obeys exactly the equations of the same cavity bounded by
the box's own conducting walls (tangential E zero on its faces): the Yee
update of every field inside uses the same neighbours with the same values.
So a random field evolves bit for bit the same in both, and the field inside
the conductor stays zero.
"""
import numpy as np
import pytest

import oracle as O

D = (1e-6, 1.1e-6, 0.9e-6)


def _valid(comp, N, dim):
    """Index ranges (i, j, k) of a component's staggered points in the closed
    box of N cells, with E tangential to a wall left out (it is zero there)."""
    n0, n1, n2 = N
    e_in = lambda n: (1, n - 1)        # interior nodes of an axis
    node = lambda n: (0, n)            # all nodes
    cent = lambda n: (0, n - 1)        # cell centres
    y = (lambda f: (0, 0)) if dim == 2 else (lambda f: f(n1))
    r = {"Ex": (cent(n0), y(e_in), e_in(n2)),
         "Ey": (e_in(n0), y(cent), e_in(n2)),
         "Ez": (e_in(n0), y(e_in), cent(n2)),
         "Bx": (node(n0), y(cent), cent(n2)),
         "By": (cent(n0), y(node), cent(n2)),
         "Bz": (cent(n0), y(cent), node(n2))}[comp]
    return [slice(a, b + 1) for a, b in r]


def _random_fields(N, dim, shape, rng, offset=(0, 0, 0)):
    out = {}
    for comp in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        a = np.zeros(shape)
        si, sj, sk = _valid(comp, N, dim)
        sl = (slice(sk.start + offset[2], sk.stop + offset[2]), slice(sj.start + offset[1], sj.stop + offset[1]),
              slice(si.start + offset[0], si.stop + offset[0]))
        a[sl] = rng.normal(size=a[sl].shape) * (1.0 if comp[0] == "E" else 1.0 / O.C_LIGHT)
        out[comp] = a
    return out


@pytest.mark.parametrize("dim", [3, 2])
def test_conductor_cavity_equals_walled_box_bit_for_bit(dim):
    N = (8, 7, 9) if dim == 3 else (8, 0, 9)
    lo, hi = (2, 3, 2), (3, 2, 4)
    if dim == 2:
        lo, hi = (2, 0, 2), (3, 0, 4)
    big = tuple(n + a + b for n, a, b in zip(N, lo, hi))
    dt = O.yee_dt(D, 0.95, dim)
    a = O.OracleSim(dim, N, (0,) * 6, D, dt, order=1, alpha_mode="one")
    b = O.OracleSim(dim, big, (0,) * 6, D, dt, order=1, alpha_mode="one")
    rng = np.random.default_rng(5)
    fa = _random_fields(N, dim, (a.nn[2], a.nn[1], a.nn[0]), rng)
    # the same values at the cavity's place in the big box
    fb = {}
    for comp, arr in fa.items():
        x = np.zeros((b.nn[2], b.nn[1], b.nn[0]))
        x[lo[2]:lo[2] + a.nn[2], lo[1]:lo[1] + a.nn[1], lo[0]:lo[0] + a.nn[0]] = arr
        fb[comp] = x
    for sim, f in ((a, fa), (b, fb)):
        for comp in ("Ex", "Ey", "Ez"):
            sim.set_field(comp, f[comp])
        for comp in ("Bx", "By", "Bz"):
            sim.set_field("Bh" + comp[1], f[comp])
            sim.set_field("Bp" + comp[1], f[comp])
    ny = big[1] if dim == 3 else 1
    mask = np.ones((big[2], ny, big[0]), dtype=bool)
    mask[lo[2]:lo[2] + N[2], lo[1]:lo[1] + max(N[1], 1), lo[0]:lo[0] + N[0]] = False
    b.set_conductor(mask)
    for _ in range(3):
        a.step(10)
        b.step(10)
        for comp in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
            si, sj, sk = _valid(comp, N, dim)
            A = a.field(comp)[sk, sj, si]
            B = b.field(comp)[lo[2]:, lo[1]:, lo[0]:][sk, sj, si]
            assert np.array_equal(A, B), comp
    # inside the conductor, away from the cavity, everything is still zero
    for comp in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        F = b.field(comp)
        assert np.all(F[:, :, :lo[0] - 1] == 0) and np.all(F[:lo[2] - 1] == 0), comp
    # and the cavity field is alive (the check is not vacuous)
    assert np.abs(a.field("Ex")).max() > 0.1


def test_conductor_can_be_removed():
    N = (6, 0, 6)
    dt = O.yee_dt(D, 0.95, 2)
    s = O.OracleSim(2, N, (0,) * 6, D, dt, order=1, alpha_mode="one")
    t = O.OracleSim(2, N, (0,) * 6, D, dt, order=1, alpha_mode="one")
    rng = np.random.default_rng(9)
    f = _random_fields(N, 2, (s.nn[2], s.nn[1], s.nn[0]), rng)
    for sim in (s, t):
        sim.set_field("Ey", f["Ey"])
        sim.set_field("Bhx", f["Bx"])
        sim.set_field("Bpx", f["Bx"])
    s.set_conductor(np.ones((6, 1, 6), dtype=bool))
    s.set_conductor(None)
    s.step(5)
    t.step(5)
    assert np.array_equal(s.field("Ey"), t.field("Ey"))
