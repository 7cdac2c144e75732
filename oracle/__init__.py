"""FP64 CPU oracle of the damped-current PML PIC step (arXiv:2201.09084).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2201_09084_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``picpml_oracle.c`` (plain loops, FP64), compiled with
gcc into ``liboracle_picpml.so`` next to it; this module only marshals numpy
arrays.  Each C function cites the passage of the paper it follows.

Functions without an independent pin: none at present; the pins are the
``tests/test_oracle_*.py`` files (listed in the C file's header).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "picpml_oracle.c")
LIB = os.path.join(HERE, "liboracle_picpml.so")

C_LIGHT = 299792458.0
EPS0 = 8.8541878128e-12
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
M_P = 1.67262192369e-27

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (no FMA contraction, portable flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
             "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def set_threads(n=None):
    """Host threads of the oracle's particle and field loops (None: every
    core; 1: the serial loops, the default).  Returns the number in use."""
    return int(lib().ora_set_threads(0 if n is None else int(n)))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.ora_create.restype = C.c_void_p
            L.ora_create.argtypes = [C.c_int, ip, ip, dp, C.c_double, C.c_int, C.c_int,
                                     C.c_double, C.c_double, C.c_double, C.c_double]
            L.ora_destroy.argtypes = [C.c_void_p]
            L.ora_set_prescribed.argtypes = [C.c_void_p, C.c_int]
            L.ora_set_filter.argtypes = [C.c_void_p, C.c_int]
            L.ora_set_solver.argtypes = [C.c_void_p, C.c_int]
            L.ora_set_conductor.argtypes = [C.c_void_p, C.c_void_p]
            L.ora_filter_J.argtypes = [C.c_void_p]
            L.ora_set_face_alpha.argtypes = [C.c_void_p, ip]
            L.ora_set_face_alpha.restype = C.c_int
            L.ora_add_particles.restype = C.c_long
            L.ora_add_particles.argtypes = [C.c_void_p, C.c_long] + [dp] * 7 + [C.c_double, C.c_double, C.c_int]
            L.ora_num_particles.restype = C.c_long
            L.ora_num_particles.argtypes = [C.c_void_p]
            L.ora_get_particles.argtypes = [C.c_void_p] + [dp] * 6 + [ip]
            L.ora_get_weights.argtypes = [C.c_void_p, dp]
            L.ora_weight_integral.restype = C.c_double
            L.ora_weight_integral.argtypes = [C.c_void_p, dp, dp]
            for f in ("ora_push", "ora_deposit", "ora_deposit_raw", "ora_damp_J", "ora_zero_J",
                      "ora_field_E", "ora_field_B"):
                getattr(L, f).argtypes = [C.c_void_p]
            L.ora_step.argtypes = [C.c_void_p, C.c_int]
            L.ora_get_field.argtypes = [C.c_void_p, C.c_int, dp]
            L.ora_get_field.restype = C.c_int
            L.ora_set_field.argtypes = [C.c_void_p, C.c_int, dp]
            L.ora_set_field.restype = C.c_int
            L.ora_rho.argtypes = [C.c_void_p, dp]
            L.ora_divE.argtypes = [C.c_void_p, dp]
            L.ora_get_table.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
            L.ora_dims.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
            L.ora_sigma_over_eps0.restype = C.c_double
            L.ora_sigma_over_eps0.argtypes = [C.c_double] * 4 + [C.c_double]
            L.ora_alpha.restype = C.c_double
            L.ora_alpha.argtypes = [C.c_double] * 5 + [C.c_int]
            L.ora_shape.restype = C.c_double
            L.ora_shape.argtypes = [C.c_int, C.c_double]
            L.ora_boris.argtypes = [dp, dp, dp, C.c_double, C.c_double, C.c_double]
            L.ora_esirkepov.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_double]
            L.ora_gather.argtypes = [C.c_void_p, dp, dp, dp]
            ip_ = C.POINTER(C.c_int)
            fp_ = C.POINTER(C.c_float)
            lp_ = C.POINTER(C.c_longlong)
            L.ora_fixed_deposit3d.argtypes = [C.c_int, C.c_longlong, ip_, fp_, ip_, fp_, fp_, C.c_double,
                                              C.c_int, C.c_longlong, C.c_longlong, C.c_longlong, lp_, lp_, lp_]
            L.ora_fixed_rho3d.argtypes = [C.c_int, C.c_longlong, ip_, fp_,
                                          C.c_longlong, C.c_longlong, C.c_longlong, lp_]
            L.ora_fixed_deposit2d.argtypes = [C.c_int, C.c_longlong, ip_, fp_, ip_, fp_, fp_, fp_, C.c_double,
                                              C.c_int, C.c_longlong, C.c_longlong, lp_, lp_, lp_]
            L.ora_fixed_rho2d.argtypes = [C.c_int, C.c_longlong, ip_, fp_, C.c_longlong, C.c_longlong, lp_]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


ALPHA_MODES = {"zero": 0, "one": 1, "damped": 2, "weight": 3}


def alpha(dcells, coef=4.0, delta=6.0, p=2.0, v=C_LIGHT, mode="damped"):
    """Eq. alpha at depth ``dcells`` (cells) into a face."""
    return lib().ora_alpha(float(dcells), coef, delta, p, v, ALPHA_MODES[mode])


def sigma_over_eps0(dcells, Delta, coef=4.0, delta=6.0, p=2.0):
    """Eq. conductivity divided by eps0, at depth ``dcells`` (cells)."""
    return lib().ora_sigma_over_eps0(float(dcells), Delta, coef, delta, p)


def shape(order, r):
    return lib().ora_shape(int(order), float(r))


def boris(u, E, B, q, m, dt):
    """One Boris rotation of u = p/(mc) (returns the new u)."""
    u = _f64(u).copy()
    lib().ora_boris(_dp(u), _dp(_f64(E)), _dp(_f64(B)), q, m, dt)
    return u


FIXED_SHAPE_BITS = 20
FIXED_UNIT = 6.0 * 2.0 ** 24   # integer current units per elementary charge crossing a face


def fixed_deposit3d(order, cell0, off0, cell1, off1, w, qn, nn, raw=False):
    """Integer currents of the deterministic deposition mode (3D) for the
    given moves: returns (Jx, Jy, Jz) int64 arrays indexed [k, j, i]; see
    ``ora_fixed_deposit3d`` for the arithmetic and units.  cell*: (n, 3) int
    cells (i, j, k); off*: (n, 3) float32 offsets; w: (n,) float32 weights;
    qn: charge in units of the elementary charge."""
    c0 = np.ascontiguousarray(cell0, dtype=np.int32).reshape(-1)
    c1 = np.ascontiguousarray(cell1, dtype=np.int32).reshape(-1)
    f0 = np.ascontiguousarray(off0, dtype=np.float32).reshape(-1)
    f1 = np.ascontiguousarray(off1, dtype=np.float32).reshape(-1)
    wf = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
    out = [np.zeros(nn[0] * nn[1] * nn[2], dtype=np.int64) for _ in range(3)]
    ip, fp, lp = C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_longlong)
    lib().ora_fixed_deposit3d(int(order), len(wf), c0.ctypes.data_as(ip), f0.ctypes.data_as(fp),
                              c1.ctypes.data_as(ip), f1.ctypes.data_as(fp), wf.ctypes.data_as(fp),
                              float(qn), int(bool(raw)), nn[0], nn[1], nn[2],
                              *[o.ctypes.data_as(lp) for o in out])
    return [o.reshape(nn[2], nn[1], nn[0]) for o in out]


def fixed_rho3d(order, cell, off, nn):
    """Integer node charge 6 S S S (units 2^-60 of a particle's charge)."""
    c = np.ascontiguousarray(cell, dtype=np.int32).reshape(-1)
    f = np.ascontiguousarray(off, dtype=np.float32).reshape(-1)
    out = np.zeros(nn[0] * nn[1] * nn[2], dtype=np.int64)
    ip, fp, lp = C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_longlong)
    lib().ora_fixed_rho3d(int(order), len(c) // 3, c.ctypes.data_as(ip), f.ctypes.data_as(fp),
                          nn[0], nn[1], nn[2], out.ctypes.data_as(lp))
    return out.reshape(nn[2], nn[1], nn[0])


def fixed_deposit2d(order, cell0, off0, cell1, off1, w, u, qn, nn, raw=False):
    """Integer currents of the deterministic deposition mode for 2D (x, z)
    boxes: returns (Jx, Jy, Jz) int64 arrays indexed [k, i] (nn = (nx, nz)
    nodes); see ``ora_fixed_deposit2d``.  u: (n, 3) float32 momenta (J_y
    carries v_y/c)."""
    c0 = np.ascontiguousarray(cell0, dtype=np.int32).reshape(-1)
    c1 = np.ascontiguousarray(cell1, dtype=np.int32).reshape(-1)
    f0 = np.ascontiguousarray(off0, dtype=np.float32).reshape(-1)
    f1 = np.ascontiguousarray(off1, dtype=np.float32).reshape(-1)
    wf = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
    uf = np.ascontiguousarray(u, dtype=np.float32).reshape(-1)
    out = [np.zeros(nn[0] * nn[1], dtype=np.int64) for _ in range(3)]
    ip, fp, lp = C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_longlong)
    lib().ora_fixed_deposit2d(int(order), len(wf), c0.ctypes.data_as(ip), f0.ctypes.data_as(fp),
                              c1.ctypes.data_as(ip), f1.ctypes.data_as(fp), wf.ctypes.data_as(fp),
                              uf.ctypes.data_as(fp), float(qn), int(bool(raw)), nn[0], nn[1],
                              *[o.ctypes.data_as(lp) for o in out])
    return [o.reshape(nn[1], nn[0]) for o in out]


def fixed_rho2d(order, cell, off, nn):
    """Integer node charge 6 S S of a 2D box (units 2^-40), indexed [k, i]."""
    c = np.ascontiguousarray(cell, dtype=np.int32).reshape(-1)
    f = np.ascontiguousarray(off, dtype=np.float32).reshape(-1)
    out = np.zeros(nn[0] * nn[1], dtype=np.int64)
    ip, fp, lp = C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_longlong)
    lib().ora_fixed_rho2d(int(order), len(c) // 3, c.ctypes.data_as(ip), f.ctypes.data_as(fp), nn[0], nn[1],
                          out.ctypes.data_as(lp))
    return out.reshape(nn[1], nn[0])


def ck_dt(d, cfl, dim):
    """dt = cfl * Courant limit of the Cole-Karkkainen scheme, min(d)/c."""
    axes = (0, 1, 2) if dim == 3 else (0, 2)
    return cfl * min(d[a] for a in axes) / C_LIGHT


def yee_dt(d, cfl, dim):
    """dt = cfl * Courant limit of the Yee scheme, 1/(c sqrt(sum 1/d_i^2))."""
    axes = (0, 1, 2) if dim == 3 else (0, 2)
    return cfl / (C_LIGHT * np.sqrt(sum(1.0 / d[a] ** 2 for a in axes)))


class OracleSim:
    """One FP64 simulation box: physical cells plus PML cells on every face.

    n: physical cells (nx, ny, nz) (ny ignored in 2D); pml: cells on the
    (-x, +x, -y, +y, -z, +z) faces; d: cell sizes in metres.
    """

    def __init__(self, dim, n, pml, d, dt, order=1, alpha_mode="damped",
                 sig_coef=4.0, delta=6.0, sig_exp=2.0, v_assumed=C_LIGHT, face_alpha=None, filter_passes=0,
                 solver="yee"):
        L = lib()
        self.dim = dim
        n3 = (C.c_int * 3)(*[int(v) for v in n])
        p6 = (C.c_int * 6)(*[int(v) for v in pml])
        d3 = (C.c_double * 3)(*[float(v) for v in d])
        mode = ALPHA_MODES[alpha_mode] if isinstance(alpha_mode, str) else int(alpha_mode)
        self._h = L.ora_create(dim, n3, p6, d3, float(dt), int(order), mode,
                               float(sig_coef), float(delta), float(sig_exp), float(v_assumed))
        if not self._h:
            raise ValueError("oracle: bad grid description")
        nn = (C.c_long * 3)()
        L.ora_dims(self._h, nn)
        self.nn = (nn[0], nn[1], nn[2])
        self.n = tuple(n)
        self.pml = tuple(pml)
        self.d = tuple(float(v) for v in d)
        self.dt = float(dt)
        self.order = order
        if face_alpha is not None:
            self.set_face_alpha(face_alpha)
        if filter_passes:
            lib().ora_set_filter(self._h, int(filter_passes))
        if solver not in ("yee", "ck"):
            raise ValueError("solver is 'yee' or 'ck'")
        self.solver = solver
        lib().ora_set_solver(self._h, int(solver == "ck"))

    def set_conductor(self, mask):
        """Zeroed-field (perfect conductor) cells: mask of shape (Nz, Ny, Nx)
        over the cells of the whole grid (Ny = 1 in 2D), True where the cell
        is a conductor; None removes them.  Every E component on a marked
        cell's edges is zero after each E update."""
        if mask is None:
            lib().ora_set_conductor(self._h, None)
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        ny = self.nn[1] - 1 if self.dim == 3 else 1
        assert m.shape == (self.nn[2] - 1, ny, self.nn[0] - 1), m.shape
        self._cond = m
        lib().ora_set_conductor(self._h, m.ctypes.data_as(C.c_void_p))

    def filter_J(self):
        """One binomial pass per axis on the deposited current (App. A)."""
        lib().ora_filter_J(self._h)

    def set_face_alpha(self, modes):
        """Per-face scheme, faces (-x, +x, -y, +y, -z, +z): "zero", "one" or
        "damped" (the cavity discussion of Sec. III: undamped where particles
        enter, damped where they leave)."""
        m6 = (C.c_int * 6)(*[ALPHA_MODES[m] if isinstance(m, str) else int(m) for m in modes])
        if lib().ora_set_face_alpha(self._h, m6) != 0:
            raise ValueError("oracle: per-face alpha modes are zero, one or damped, and not in weight mode")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_destroy(h)
            self._h = None

    # particles -----------------------------------------------------------
    def add_particles(self, X, Y, Z, ux, uy, uz, w, q, m, immobile=False):
        n = len(X)
        arrs = [_f64(a) for a in (X, Y, Z, ux, uy, uz, w)]
        r = lib().ora_add_particles(self._h, n, *[_dp(a) for a in arrs], float(q), float(m),
                                    int(bool(immobile)))
        if r < 0:
            raise ValueError("oracle: bad particles")
        return r

    def set_prescribed(self, flag=True):
        lib().ora_set_prescribed(self._h, int(bool(flag)))

    def particles(self):
        n = lib().ora_num_particles(self._h)
        out = [np.zeros(n) for _ in range(6)]
        alive = np.zeros(n, dtype=np.int32)
        lib().ora_get_particles(self._h, *[_dp(a) for a in out],
                                alive.ctypes.data_as(C.POINTER(C.c_int)))
        w = np.zeros(n)
        lib().ora_get_weights(self._h, _dp(w))
        return dict(X=out[0], Y=out[1], Z=out[2], ux=out[3], uy=out[4], uz=out[5],
                    alive=alive.astype(bool), w=w)

    def weight_integral(self, X0, X1):
        """The step's damping exponent int sigma/eps0 dt (weight mode)."""
        return lib().ora_weight_integral(self._h, _dp(_f64(X0)), _dp(_f64(X1)))

    # stepping ------------------------------------------------------------
    def step(self, n=1):
        lib().ora_step(self._h, int(n))

    def push(self):
        lib().ora_push(self._h)

    def deposit(self):
        lib().ora_deposit(self._h)

    def deposit_raw(self):
        lib().ora_deposit_raw(self._h)

    def damp_J(self):
        lib().ora_damp_J(self._h)

    def zero_J(self):
        lib().ora_zero_J(self._h)

    def field_E(self):
        lib().ora_field_E(self._h)

    def field_B(self):
        lib().ora_field_B(self._h)

    def esirkepov(self, X0, X1, qw, vy=0.0):
        lib().ora_esirkepov(self._h, _dp(_f64(X0)), _dp(_f64(X1)), float(qw), float(vy))

    def gather(self, X):
        E = np.zeros(3)
        B = np.zeros(3)
        lib().ora_gather(self._h, _dp(_f64(X)), _dp(E), _dp(B))
        return E, B

    # fields ------------------------------------------------------------
    def _shape3(self, a):
        # arrays are laid out i + nx (j + ny k): return as [k, j, i]
        return a.reshape(self.nn[2], self.nn[1], self.nn[0])

    def field(self, which):
        """which: 'Ex'..'Bz' (B at integer time), 'Jx'..'Jz', 'Bhx'.. (B^{n+1/2}),
        'Bpx'.. (B^{n-1/2}).  Returns an array indexed [k, j, i]."""
        base = {"E": 0, "B": 3, "J": 6, "Bh": 9, "Bp": 12}[which[:-1]]
        c = "xyz".index(which[-1])
        out = np.zeros(self.nn[0] * self.nn[1] * self.nn[2])
        lib().ora_get_field(self._h, base + c, _dp(out))
        return self._shape3(out)

    def set_field(self, which, arr):
        base = {"E": 0, "J": 6, "Bh": 9, "Bp": 12}[which[:-1]]
        c = "xyz".index(which[-1])
        a = _f64(np.asarray(arr)).reshape(-1)
        assert a.size == self.nn[0] * self.nn[1] * self.nn[2]
        if lib().ora_set_field(self._h, base + c, _dp(a)) != 0:
            raise ValueError(which)

    def rho(self):
        out = np.zeros(self.nn[0] * self.nn[1] * self.nn[2])
        lib().ora_rho(self._h, _dp(out))
        return self._shape3(out)

    def divE(self):
        out = np.zeros(self.nn[0] * self.nn[1] * self.nn[2])
        lib().ora_divE(self._h, _dp(out))
        return self._shape3(out)

    def table(self, which, axis):
        """which: 's_node', 's_cent', 'a_node', 'a_cent' (sigma/eps0 or alpha)."""
        k = ["s_node", "s_cent", "a_node", "a_cent"].index(which)
        out = np.zeros(self.nn[axis])
        lib().ora_get_table(self._h, k, axis, _dp(out))
        return out


def rel_error(sim, ref, offset=(0, 0, 0), parts=False):
    """Eq. error: int[(E-Eref)^2 + c^2 (B-Bref)^2] / int[Eref^2 + c^2 Bref^2]
    over the physical cells of ``sim``; ``offset`` is the node index of sim's
    node (0,0,0) inside ``ref``.  Every component is sampled at its own
    staggered points that lie in the closed physical box.  parts=True
    returns (numerator, denominator) instead of their ratio."""
    num = 0.0
    den = 0.0
    lo = [sim.pml[0], sim.pml[2], sim.pml[4]]
    hi = [lo[0] + sim.n[0], lo[1] + (sim.n[1] if sim.dim == 3 else 0), lo[2] + sim.n[2]]
    # staggered along its own axis for E, along the two others for B
    for fam, scale in (("E", 1.0), ("B", C_LIGHT ** 2)):
        for c in "xyz":
            a = sim.field(fam + c)
            b = ref.field(fam + c)
            ax = "xyz".index(c)
            stag = [0, 0, 0]
            if fam == "E":
                stag[ax] = 1
            else:
                stag = [1, 1, 1]
                stag[ax] = 0
            if sim.dim == 2:
                stag[1] = 0
            sl = []
            slr = []
            for q, (l, h) in enumerate(zip(lo, hi)):
                top = h - 1 if stag[q] else h
                sl.append(slice(l, top + 1))
                slr.append(slice(l + offset[q], top + 1 + offset[q]))
            A = a[sl[2], sl[1], sl[0]]
            Bv = b[slr[2], slr[1], slr[0]]
            num += scale * np.sum((A - Bv) ** 2)
            den += scale * np.sum(Bv ** 2)
    return (num, den) if parts else num / den
