"""Python face of libpicpml: a Sim object that owns one library context.

PyTorch provides the device memory (particle arrays, field read-back buffers)
and the CUDA stream; every computation is a call into the C ABI.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

FIELDS = {f"{fam}{c}": base + i for fam, base in (("E", 0), ("B", 3), ("J", 6), ("Bh", 9), ("Bp", 12))
          for i, c in enumerate("xyz")}


def pack_particles(cell, off, u, w, prec="fp32", capacity=None, device="cuda"):
    """Packs (cell index (n,3) int, offsets (n,3), u (n,3), weight (n,)) into
    the pos/mom records of include/picpml.h on the device.  Returns (pos, mom)
    tensors of shape (capacity, 4)."""
    n = len(w)
    cap = n if capacity is None else capacity
    dt = torch.float64 if prec == "fp64" else torch.float32
    cell = np.asarray(cell, dtype=np.int64)
    packed = (cell[:, 0] | (cell[:, 1] << 10) | (cell[:, 2] << 20)).astype(np.int64)
    pos = torch.zeros((cap, 4), dtype=dt)
    mom = torch.zeros((cap, 4), dtype=dt)
    pos[:n, :3] = torch.from_numpy(np.asarray(off)).to(dt)
    pos[:n, 3] = torch.from_numpy(np.asarray(w)).to(dt)
    mom[:n, :3] = torch.from_numpy(np.asarray(u)).to(dt)
    if dt == torch.float32:
        mom.view(torch.int32)[:n, 3] = torch.from_numpy(packed.astype(np.int32))
    else:
        mom.view(torch.int64)[:n, 3] = torch.from_numpy(packed)
    return pos.to(device), mom.to(device)


def unpack_particles(pos, mom, n):
    """Inverse of pack_particles (host numpy): cell (n,3), off (n,3), u, w, alive."""
    pos = pos[:n].cpu()
    mom = mom[:n].cpu()
    if pos.dtype == torch.float32:
        packed = mom.view(torch.int32)[:, 3].numpy().astype(np.int64)
    else:
        packed = mom.view(torch.int64)[:, 3].numpy()
    alive = packed >= 0
    cell = np.stack([packed & 1023, (packed >> 10) & 1023, (packed >> 20) & 2047], axis=1)
    cell[~alive] = -1
    return dict(cell=cell, off=pos[:, :3].numpy(), w=pos[:, 3].numpy(), u=mom[:, :3].numpy(), alive=alive)


class Sim:
    """One GPU simulation box (physical cells + PML cells on every face)."""

    def __init__(self, dim, n, d, pml, *, dt=0.0, cfl=0.99, order=1, prec="fp32", sort_every=0,
                 alpha_mode="damped", sigma_coef=4.0, delta=6.0, exponent=2.0, v_assumed=0.0,
                 split_fp64=False, stream=None):
        self.lib = L.load()
        self.prec = prec
        self.dim = dim
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = L.GridDesc()
        g.dim = dim
        for a in range(3):
            g.n[a] = int(n[a])
            g.d[a] = float(d[a])
        g.dt, g.cfl, g.shape_order, g.prec, g.sort_every = float(dt), float(cfl), int(order), L.PREC[prec], int(sort_every)
        g.split_fp64 = int(bool(split_fp64))
        ctx = C.c_void_p()
        L.check(self.lib.pic_init(C.byref(ctx), C.byref(g), C.c_void_p(self.stream.cuda_stream)))
        self.ctx = ctx
        p = L.PmlDesc()
        for i in range(6):
            p.ncell[i] = int(pml[i])
        p.sigma_max_coef, p.delta_cells, p.exponent = float(sigma_coef), float(delta), float(exponent)
        p.alpha_mode = L.ALPHA[alpha_mode] if isinstance(alpha_mode, str) else int(alpha_mode)
        p.v_assumed = float(v_assumed)
        self._call(self.lib.pml_init, C.byref(p))
        nn = (C.c_int * 3)()
        dtv = C.c_double()
        self._call(self.lib.pic_grid_info, nn, C.byref(dtv))
        self.nn = (nn[0], nn[1], nn[2])
        self.dt = dtv.value
        self.n = tuple(n)
        self.pml = tuple(pml)
        self.d = tuple(d)
        self.species = []

    def _call(self, fn, *args):
        L.check(fn(self.ctx, *args), self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # particles --------------------------------------------------------
    def add_species(self, pos, mom, n, q, m, immobile=False):
        want = torch.float64 if self.prec == "fp64" else torch.float32
        assert pos.is_cuda and mom.is_cuda and pos.dtype == want and mom.dtype == want
        assert pos.shape == mom.shape and pos.shape[1] == 4 and pos.is_contiguous() and mom.is_contiguous()
        s = L.SpeciesDesc()
        s.pos, s.mom = pos.data_ptr(), mom.data_ptr()
        s.n, s.capacity, s.q, s.m, s.immobile = int(n), int(pos.shape[0]), float(q), float(m), int(bool(immobile))
        sid = C.c_int()
        self._call(self.lib.pic_add_species, C.byref(s), C.byref(sid))
        self.species.append((pos, mom))
        return sid.value

    def num_particles(self, sid):
        n = C.c_longlong()
        self._call(self.lib.pic_num_particles, int(sid), C.byref(n))
        return n.value

    def particles(self, sid):
        pos, mom = self.species[sid]
        return unpack_particles(pos, mom, self.num_particles(sid))

    def set_prescribed(self, flag=True):
        self._call(self.lib.pic_set_prescribed, int(bool(flag)))

    # stepping ---------------------------------------------------------
    def push(self):
        self._call(self.lib.push)

    def deposit(self):
        self._call(self.lib.deposit)

    def field_step(self):
        self._call(self.lib.field_step)

    def push_deposit(self):
        self._call(self.lib.push_deposit)

    def launch_count(self):
        n = C.c_longlong()
        self._call(self.lib.pic_launch_count, C.byref(n))
        return n.value

    def particle_steps(self):
        n = C.c_longlong()
        self._call(self.lib.pic_particle_steps, C.byref(n))
        return n.value

    def step(self, n=1):
        self._call(self.lib.step_n, int(n))

    def sort(self):
        self._call(self.lib.pic_sort)

    def sync(self):
        self._call(self.lib.pic_sync)

    # fields -----------------------------------------------------------
    def field(self, name, dtype=torch.float64):
        out = torch.empty(self.nn[2] * self.nn[1] * self.nn[0], dtype=dtype, device="cuda")
        self._call(self.lib.pic_get_field, FIELDS[name], C.c_void_p(out.data_ptr()), int(dtype == torch.float64))
        return out.view(self.nn[2], self.nn[1], self.nn[0])

    def set_field(self, name, arr):
        t = torch.as_tensor(arr, dtype=torch.float64).contiguous().cuda()
        assert t.numel() == self.nn[0] * self.nn[1] * self.nn[2]
        self._call(self.lib.pic_set_field, FIELDS[name], C.c_void_p(t.data_ptr()), 1)
        self.stream.synchronize()

    def diag(self):
        g, r, e = C.c_double(), C.c_double(), C.c_double()
        self._call(self.lib.pic_diag, C.byref(g), C.byref(r), C.byref(e))
        return dict(gauss=g.value, rho_scale=r.value, energy=e.value)

    def get_state(self):
        nb = C.c_longlong()
        self._call(self.lib.pic_state_size, C.byref(nb))
        buf = np.empty(nb.value, dtype=np.uint8)
        self._call(self.lib.pic_get_state, C.c_void_p(buf.ctypes.data))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._call(self.lib.pic_set_state, C.c_void_p(buf.ctypes.data))
