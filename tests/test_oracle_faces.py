"""Pins of the oracle's per-face deposition schemes (the cavity discussion of
Sec. III: the undamped scheme on the face where particles enter, the damped
one where they leave).

- alpha tables: below the physical box an axis carries its low face's mode,
  above it its high face's mode, 1 inside; each side equals the table of a
  box run in that mode throughout (a swapped face or axis fails);
- a deposited and damped move inside one face's PML equals the same move in
  a box whose every face uses that face's mode;
- a face in mode zero removes particles at its own interface only;
- every face in the box's own mode reproduces the box bit for bit;
- weight damping takes no per-face modes.
"""
import numpy as np
import pytest

import oracle as O

D3 = (1e-6, 1.2e-6, 0.9e-6)
N = (10, 9, 12)
PML = (6, 7, 5, 6, 7, 6)


def _box(mode="damped", faces=None, order=1):
    dt = O.yee_dt(D3, 0.9, 3)
    return O.OracleSim(3, N, PML, D3, dt, order=order, alpha_mode=mode, face_alpha=faces)


FACES = ["zero", "damped", "one", "zero", "one", "damped"]


def test_alpha_tables_follow_each_face():
    mixed = _box(faces=FACES)
    uni = {m: _box(m) for m in ("zero", "one", "damped")}
    for a in range(3):
        lo, nph = PML[2 * a], N[a]
        for which, shift in (("a_node", 0.0), ("a_cent", 0.5)):
            t = mixed.table(which, a)
            x = np.arange(len(t)) + shift
            below, above = x < lo, x > lo + nph
            inside = ~below & ~above
            assert np.all(t[inside] == 1.0)
            assert np.array_equal(t[below], uni[FACES[2 * a]].table(which, a)[below]), (a, which)
            assert np.array_equal(t[above], uni[FACES[2 * a + 1]].table(which, a)[above]), (a, which)
            # every face of this layout has some alpha < 1 or = 1 as its mode says
            if FACES[2 * a] != "one":
                assert np.any(t[below] < 1.0)
            if FACES[2 * a + 1] != "one":
                assert np.any(t[above] < 1.0)


@pytest.mark.parametrize("order", [1, 3])
def test_damped_move_in_each_face_matches_that_faces_mode(order):
    # moves 2-3 cells deep in the -z PML (mode one) and in the +z PML (damped)
    lo_z, hi_z = PML[4], PML[4] + N[2]
    moves = {"-z": (np.array([6 + 4.3, 5 + 4.2, lo_z - 2.6]), np.array([6 + 4.6, 5 + 4.0, lo_z - 2.1])),
             "+z": (np.array([6 + 4.3, 5 + 4.2, hi_z + 2.2]), np.array([6 + 4.5, 5 + 4.5, hi_z + 2.8]))}
    for side, mode in (("-z", "one"), ("+z", "damped")):
        X0, X1 = moves[side]
        a = _box(faces=FACES, order=order)
        b = _box(FACES[4] if side == "-z" else FACES[5], order=order)
        for s in (a, b):
            s.esirkepov(X0, X1, -O.Q_E * 2.0)
            s.damp_J()
        for c in "xyz":
            ja, jb = a.field("J" + c), b.field("J" + c)
            assert np.array_equal(ja, jb), (side, c)
        assert np.max(np.abs(a.field("Jz"))) > 0


def test_zero_face_removes_at_its_own_interface():
    faces = ["damped", "damped", "damped", "damped", "damped", "zero"]
    s = _box(faces=faces)
    lo_z, hi_z = PML[4], PML[4] + N[2]
    X = [6 + 5.3, 5 + 4.1]
    uz = 3.0
    # one electron about to cross the -z interface outward, one the +z interface
    s.add_particles([X[0], X[0]], [X[1], X[1]], [lo_z + 0.2, hi_z - 0.2], [0.0, 0.0], [0.0, 0.0], [-uz, uz],
                    [1.0, 1.0], -O.Q_E, O.M_E)
    s.set_prescribed(True)
    s.step(2)
    alive = s.particles()["alive"]
    assert alive[0] and not alive[1]
    assert s.particles()["Z"][0] < lo_z


def test_uniform_faces_reproduce_the_box():
    rng = np.random.default_rng(3)
    X = [6 + rng.uniform(0, 10, 40), 5 + rng.uniform(0, 9, 40), 7 + rng.uniform(0, 12, 40)]
    u = rng.normal(0, 2.0, (3, 40))
    a = _box("damped", faces=["damped"] * 6)
    b = _box("damped")
    for s in (a, b):
        s.add_particles(X[0], X[1], X[2], u[0], u[1], u[2], np.ones(40), -O.Q_E, O.M_E)
    a.step(15)
    b.step(15)
    for f in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        assert np.array_equal(a.field(f), b.field(f)), f


def test_weight_mode_takes_no_face_modes():
    with pytest.raises(ValueError):
        _box("weight", faces=["damped"] * 6)
    with pytest.raises(ValueError):
        _box("damped", faces=["weight"] * 6)
