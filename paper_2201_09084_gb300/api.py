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


def pack_records(cell, off, u, w, capacity=None):
    """FP32 pos/mom records (include/picpml.h) from device tensors: cell (n, 3)
    int32, off (n, 3) and u (n, 3) float32, w a scalar or (n,) tensor.
    Returns (pos, mom) of shape (capacity, 4) on the tensors' device."""
    n = cell.shape[0]
    cap = n if capacity is None else capacity
    pos = torch.zeros((cap, 4), dtype=torch.float32, device=cell.device)
    mom = torch.zeros((cap, 4), dtype=torch.float32, device=cell.device)
    pos[:n, :3] = off
    pos[:n, 3] = w
    mom[:n, :3] = u
    packed = cell[:, 0] | (cell[:, 1] << 10) | (cell[:, 2] << 20)
    mom.view(torch.int32)[:n, 3] = packed.to(torch.int32)
    return pos, mom


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


def _set_face_alpha(p, face_alpha):
    """Per-face schemes (faces -x, +x, -y, +y, -z, +z): "zero", "one" or
    "damped" each, or None for the box's alpha_mode on every face."""
    if face_alpha is None:
        p.face_alpha_set = 0
        return
    if len(face_alpha) != 6:
        raise ValueError("face_alpha needs six modes (-x, +x, -y, +y, -z, +z)")
    p.face_alpha_set = 1
    for f, m in enumerate(face_alpha):
        p.face_alpha[f] = L.ALPHA[m] if isinstance(m, str) else int(m)


class Sim:
    """One GPU simulation box (physical cells + PML cells on every face)."""

    def __init__(self, dim, n, d, pml, *, dt=0.0, cfl=0.99, order=1, prec="fp32", sort_every=0,
                 alpha_mode="damped", sigma_coef=4.0, delta=6.0, exponent=2.0, v_assumed=0.0,
                 split_fp64=False, face_alpha=None, filter_passes=0, solver="yee", stream=None):
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
        g.filter_passes = int(filter_passes)
        g.solver = L.SOLVER[solver]
        ctx = C.c_void_p()
        L.check(self.lib.pic_init(C.byref(ctx), C.byref(g), C.c_void_p(self.stream.cuda_stream)))
        self.ctx = ctx
        p = L.PmlDesc()
        for i in range(6):
            p.ncell[i] = int(pml[i])
        p.sigma_max_coef, p.delta_cells, p.exponent = float(sigma_coef), float(delta), float(exponent)
        p.alpha_mode = L.ALPHA[alpha_mode] if isinstance(alpha_mode, str) else int(alpha_mode)
        p.v_assumed = float(v_assumed)
        _set_face_alpha(p, face_alpha)
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

    def inject(self, sid, pos, mom, count=None):
        """Appends particles (device tensors in the species' layout) after the
        live ones of species sid (pic_inject); keeps the tensors alive until
        the stream has copied them."""
        want = torch.float64 if self.prec == "fp64" else torch.float32
        assert pos.is_cuda and mom.is_cuda and pos.dtype == want and mom.dtype == want
        assert pos.shape == mom.shape and pos.shape[1] == 4 and pos.is_contiguous() and mom.is_contiguous()
        n = int(pos.shape[0]) if count is None else int(count)
        self._call(self.lib.pic_inject, int(sid), C.c_void_p(pos.data_ptr()), C.c_void_p(mom.data_ptr()), n)
        self._inflight = (pos, mom)

    def num_particles(self, sid):
        n = C.c_longlong()
        self._call(self.lib.pic_num_particles, int(sid), C.byref(n))
        return n.value

    def particles(self, sid):
        pos, mom = self.species[sid]
        return unpack_particles(pos, mom, self.num_particles(sid))

    def set_prescribed(self, flag=True):
        self._call(self.lib.pic_set_prescribed, int(bool(flag)))

    def set_conductor(self, mask):
        """Zeroed-field cells: a mask of shape (Nz, Ny, Nx) over the cells of
        the whole grid (Ny = 1 in 2D), True for a conductor cell; None
        removes them."""
        if mask is None:
            self._call(self.lib.pic_set_conductor, None)
            return
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        ny = self.nn[1] - 1 if self.dim == 3 else 1
        assert m.shape == (self.nn[2] - 1, ny, self.nn[0] - 1), m.shape
        self._call(self.lib.pic_set_conductor, m.ctypes.data_as(C.c_void_p))

    def set_old_positions(self, sid, cell, off):
        """Sets x^n (what push() saves) of species sid from host (n, 3) cells
        and offsets, so deposit() deposits the moves to the current positions.
        Returns the device buffer, which must live until the deposit ran."""
        pos, _ = self.species[sid]
        cap = pos.shape[0]
        dt = torch.float64 if self.prec == "fp64" else torch.float32
        n = len(off)
        cell = np.asarray(cell, dtype=np.int64)
        packed = np.full(cap, -1, dtype=np.int64)
        packed[:n] = cell[:, 0] | (cell[:, 1] << 10) | (cell[:, 2] << 20)
        buf = torch.zeros((cap, 4), dtype=dt)
        buf[:n, :3] = torch.from_numpy(np.asarray(off)).to(dt)
        if dt == torch.float32:
            buf.view(torch.int32)[:, 3] = torch.from_numpy(packed.astype(np.int32))
        else:
            buf.view(torch.int64)[:, 3] = torch.from_numpy(packed)
        buf = buf.to("cuda")
        self._call(self.lib.pic_set_old_positions, int(sid), C.c_void_p(buf.data_ptr()))
        self._keep = buf
        return buf

    def current_fixed(self, comp):
        """int64 current sums of the last deposit (fixed64 contexts), as a
        device tensor indexed [k, j, i]."""
        out = torch.empty(self.nn[2] * self.nn[1] * self.nn[0], dtype=torch.int64, device="cuda")
        self._call(self.lib.pic_get_current_fixed, int(comp), C.c_void_p(out.data_ptr()))
        return out.view(self.nn[2], self.nn[1], self.nn[0])

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

    def autotune(self, steps=3):
        p, k = C.c_int(), C.c_int()
        self._call(self.lib.pic_autotune, int(steps), C.byref(p), C.byref(k))
        return {"particles_per_thread": p.value, "z_nodes_per_thread": k.value}

    def set_tuning(self, particles_per_thread=0, z_nodes_per_thread=1):
        self._call(self.lib.pic_set_tuning, int(particles_per_thread), int(z_nodes_per_thread))

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


class Batch:
    """Many independent 2D runs advanced together (pic_batch_* of the C ABI)."""

    def __init__(self, nx, nz, npml, d, pos, mom, q, m, *, dt=0.0, cfl=0.99, order=1, prec="fp32",
                 alpha_mode="damped", sigma_coef=4.0, delta=6.0, exponent=2.0, v_assumed=0.0, face_alpha=None,
                 stream=None):
        self.lib = L.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n = len(nx)
        self._nx = np.ascontiguousarray(nx, dtype=np.int32)
        self._nz = np.ascontiguousarray(nz, dtype=np.int32)
        self._np = np.ascontiguousarray(npml, dtype=np.int32)
        d_ = L.BatchDesc()
        d_.nruns = self.n
        ip = C.POINTER(C.c_int)
        d_.nx = self._nx.ctypes.data_as(ip)
        d_.nz = self._nz.ctypes.data_as(ip)
        d_.npml = self._np.ctypes.data_as(ip)
        d_.d[0], d_.d[1] = float(d[0]), float(d[1])
        d_.dt, d_.cfl, d_.shape_order, d_.prec = float(dt), float(cfl), int(order), L.PREC[prec]
        d_.pml.sigma_max_coef, d_.pml.delta_cells, d_.pml.exponent = float(sigma_coef), float(delta), float(exponent)
        d_.pml.alpha_mode = L.ALPHA[alpha_mode] if isinstance(alpha_mode, str) else int(alpha_mode)
        d_.pml.v_assumed = float(v_assumed)
        _set_face_alpha(d_.pml, face_alpha)
        d_.q, d_.m = float(q), float(m)
        want = torch.float64 if prec == "fp64" else torch.float32
        assert pos.is_cuda and pos.dtype == want and tuple(pos.shape) == (self.n, 4)
        d_.pos, d_.mom = pos.data_ptr(), mom.data_ptr()
        self.pos, self.mom = pos, mom
        h = C.c_void_p()
        rc = self.lib.pic_batch_init(C.byref(h), C.byref(d_), C.c_void_p(self.stream.cuda_stream))
        self.h = h
        if rc != 0:
            msg = self.lib.pic_batch_last_error(h).decode()
            self.close()
            raise L.PicError(rc, msg)
        dtv, cells = C.c_double(), C.c_longlong()
        self._call(self.lib.pic_batch_info, C.byref(dtv), C.byref(cells))
        self.dt, self.cells = dtv.value, cells.value

    def _call(self, fn, *args):
        rc = fn(self.h, *args)
        if rc != 0:
            raise L.PicError(rc, self.lib.pic_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        self._call(self.lib.pic_batch_step, int(n))

    def sync(self):
        self._call(self.lib.pic_batch_sync)

    def set_prescribed(self, flag=True):
        self._call(self.lib.pic_batch_set_prescribed, int(bool(flag)))

    def particle_steps(self):
        n = C.c_longlong()
        self._call(self.lib.pic_batch_particle_steps, C.byref(n))
        return n.value

    def tuning(self):
        t, mb = C.c_int(), C.c_int()
        ms = (C.c_float * 7)()
        self._call(self.lib.pic_batch_tuning, C.byref(t), C.byref(mb), ms, 7)
        return {"threads": t.value, "min_blocks_per_sm": mb.value, "candidate_ms_per_step": list(ms)}

    def field(self, run, name, dtype=torch.float64):
        nn0 = int(self._nx[run] + 2 * self._np[run] + 1)
        nn2 = int(self._nz[run] + 2 * self._np[run] + 1)
        out = torch.empty(nn0 * nn2, dtype=dtype, device="cuda")
        self._call(self.lib.pic_batch_get_field, int(run), FIELDS[name], C.c_void_p(out.data_ptr()),
                   int(dtype == torch.float64))
        return out.view(nn2, 1, nn0)
