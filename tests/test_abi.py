"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/picpml.h declares; the binding covers the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "picpml.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?(?:int|void|const char\s*\*|char\s*\*)\s*\*?\s*(\w+)\s*\(", txt, flags=re.M))
    names |= set(re.findall(r"\bint\s+(pic_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2201_09084_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pic_init", "pml_init", "deposit", "push", "field_step", "step_n"):
        assert n in names, n


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2201_09084_gb300 import _lib as L
    assert _declared() == set(L.SIGNATURES), _declared() ^ set(L.SIGNATURES)


def test_init_rejects_bad_descriptions_without_gpu(lib):
    """Host-side validation runs before any device work."""
    from paper_2201_09084_gb300 import _lib as L
    L.load()
    ctx = ctypes.c_void_p()
    g = L.GridDesc()
    g.dim = 4
    assert L.load().pic_init(ctypes.byref(ctx), ctypes.byref(g), None) == -1
    g.dim, g.shape_order, g.prec = 3, 2, 0
    assert L.load().pic_init(ctypes.byref(ctx), ctypes.byref(g), None) == -1
    g.shape_order = 1
    for a in range(3):
        g.n[a] = 16
        g.d[a] = 1e-6
    g.dt = 1e-14   # above the Courant limit 1.9e-15 s
    assert L.load().pic_init(ctypes.byref(ctx), ctypes.byref(g), None) == -4
    assert b"Courant" in L.load().pic_last_error(None)


def test_init_rejects_each_bad_field_without_gpu(lib):
    """Every descriptor check answers PIC_EINVAL with its own message before
    any device work: precision, filter passes, cell counts and sizes, and a
    Courant fraction outside (0, 1] when dt is left to the library."""
    from paper_2201_09084_gb300 import _lib as L
    lb = L.load()
    ctx = ctypes.c_void_p()

    def good():
        g = L.GridDesc()
        g.dim, g.shape_order, g.prec = 3, 1, 0
        for a in range(3):
            g.n[a] = 16
            g.d[a] = 1e-6
        g.dt, g.cfl = 0.0, 0.9
        return g

    cases = [("prec", 7, b"prec"), ("filter_passes", 9, b"filter_passes"),
             ("filter_passes", -1, b"filter_passes"), ("cfl", 1.5, b"cfl"), ("cfl", 0.0, b"cfl")]
    for field, value, msg in cases:
        g = good()
        setattr(g, field, value)
        assert lb.pic_init(ctypes.byref(ctx), ctypes.byref(g), None) == -1, field
        assert msg in lb.pic_last_error(None), (field, lb.pic_last_error(None))
    for a, (n, d) in enumerate([(0, 1e-6), (16, 0.0), (16, -1e-6)]):
        g = good()
        g.n[a], g.d[a] = n, d
        assert lb.pic_init(ctypes.byref(ctx), ctypes.byref(g), None) == -1
        assert b"positive" in lb.pic_last_error(None)
    # in 2D the y extent is ignored
    g = good()
    g.dim, g.n[1], g.d[1], g.prec = 2, 0, 0.0, 7
    assert lb.pic_init(ctypes.byref(ctx), ctypes.byref(g), None) == -1
    assert b"prec" in lb.pic_last_error(None)
    assert lb.pic_init(None, ctypes.byref(g), None) == -1


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field
    offsets (a C program compiled against include/picpml.h prints them)."""
    import subprocess
    from paper_2201_09084_gb300 import _lib as L
    structs = {"pic_grid_desc": L.GridDesc, "pml_desc": L.PmlDesc, "pic_species": L.SpeciesDesc,
               "pic_batch_desc": L.BatchDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "picpml.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, cls in structs.items():
        assert int(got[f"{cname} size"]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname} {fname}"]) == getattr(cls, fname).offset, (cname, fname)
