"""GB300-native X2C / DLU relativistic one-electron Hamiltonian (sm_103a CUDA behind a C ABI).

Python side: `x2c_*` functions with the names of include/x2c.h that marshal torch CUDA
tensors into the library calls.  Every step of the computation runs in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import abi
from .abi import (DLU_FREE_ATOM, DLU_MOLECULAR_BLOCK, LOCAL_DLH, LOCAL_DLU, PREC_FP64,  # noqa: F401
                  PREC_SPLIT_BF16, X2CError)

C_LIGHT = 137.035999
DEC_X2C, DEC_BSS = 0, 1  # x2c_decoupling; an integer n = 2..14 selects DKHn
_MAT_KEYS = ("S", "T", "V", "W0", "Wx", "Wy", "Wz")


def _torch():
    import torch
    return torch


class Context:
    """A library context on one CUDA device (x2c_ctx_create / x2c_ctx_destroy)."""

    def __init__(self, device: int = 0):
        self.lib = abi.load()
        h = ctypes.c_void_p()
        abi.check(self.lib.x2c_ctx_create(int(device), ctypes.byref(h)), "x2c_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self.lib.x2c_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        """x2c_ctx_status: synchronise the stream and raise on a latched device error."""
        abi.check(self.lib.x2c_ctx_status(self.handle, _stream(stream)), "device status", self.handle)

    def set_timing(self, enable: bool):
        """x2c_ctx_set_timing: bracket every kernel launch with CUDA events (clears totals)."""
        abi.check(self.lib.x2c_ctx_set_timing(self.handle, int(bool(enable))), "x2c_ctx_set_timing")

    def set_autotune(self, enable: bool):
        """x2c_ctx_set_autotune: time the candidate tensor-core tiles once per workload shape."""
        abi.check(self.lib.x2c_ctx_set_autotune(self.handle, int(bool(enable))), "x2c_ctx_set_autotune")

    def set_split_variant(self, variant: int):
        """x2c_ctx_set_split_variant: force a split-kernel candidate (-1 = automatic)."""
        abi.check(self.lib.x2c_ctx_set_split_variant(self.handle, int(variant)), "x2c_ctx_set_split_variant")

    def set_graphs(self, enable: bool):
        """x2c_ctx_set_graphs: capture a build the second time its launch plan is seen and
        replay the CUDA graph on every later identical call."""
        abi.check(self.lib.x2c_ctx_set_graphs(self.handle, int(bool(enable))), "x2c_ctx_set_graphs")

    def graph_stats(self):
        """x2c_ctx_graph_stats: graphs captured, builds replayed, graphs held, last call replayed."""
        g = abi.GraphStats()
        abi.check(self.lib.x2c_ctx_graph_stats(self.handle, ctypes.byref(g)), "x2c_ctx_graph_stats")
        return dict(captures=g.captures, replays=g.replays, cached=g.cached, last_replayed=bool(g.last_replayed))

    def tuning_log(self) -> str:
        """x2c_ctx_tuning_log: the autotuner's decisions, one line each."""
        return self.lib.x2c_ctx_tuning_log(self.handle).decode()

    def kernel_times(self, max_entries: int = 64, with_flops: bool = False):
        """x2c_ctx_kernel_times: {kernel name: (total ms, launches)} since timing was enabled,
        or (total ms, launches, algorithmic flops) with with_flops=True."""
        names = ctypes.create_string_buffer(32 * max_entries)
        ms = (ctypes.c_double * max_entries)()
        cnt = (ctypes.c_int64 * max_entries)()
        fl = (ctypes.c_double * max_entries)()
        n = ctypes.c_int32()
        abi.check(self.lib.x2c_ctx_kernel_times(self.handle, max_entries, names, ms, cnt, fl, ctypes.byref(n)),
                  "x2c_ctx_kernel_times", self.handle)
        raw = names.raw
        out = {}
        for i in range(n.value):
            key = raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
            out[key] = (ms[i], cnt[i], fl[i]) if with_flops else (ms[i], cnt[i])
        return out

    def counters(self):
        c = abi.Counters()
        abi.check(self.lib.x2c_ctx_counters(self.handle, ctypes.byref(c)), "x2c_ctx_counters")
        return dict(pair_blocks=c.pair_blocks, atomic_solves=c.atomic_solves,
                    kernel_launches=c.kernel_launches, credited_flops=c.credited_flops)


def _stream(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def options(two_component=False, c=None, precision=PREC_FP64, dlu_potential=DLU_FREE_ATOM,
            so_same_atom_only=True, n_slices=0, local_approx=LOCAL_DLU, h_upper_only=False,
            decoupling=DEC_X2C) -> abi.Options:
    """x2c_options.  decoupling: DEC_X2C (0), DEC_BSS (1) or the DKH order n (2..14)."""
    o = abi.Options()
    o.h_upper_only = int(bool(h_upper_only))
    o.decoupling = int(decoupling)
    o.local_approx = int(local_approx)
    o.c = float(c) if c else C_LIGHT
    o.two_component = int(bool(two_component))
    o.precision = int(precision)
    o.dlu_potential = int(dlu_potential)
    o.so_same_atom_only = int(bool(so_same_atom_only))
    o.n_slices = int(n_slices)
    return o


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, n, device_expected=True):
    torch = _torch()
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("matrices must be contiguous float64 torch tensors")
    if t.shape != (n, n):
        raise ValueError(f"expected shape {(n, n)}, got {tuple(t.shape)}")
    if device_expected and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")


def mats_struct(m: dict, two_component: bool) -> abi.Mats:
    n = m["S"].shape[0]
    s = abi.Mats()
    s.n = n
    for k in _MAT_KEYS:
        t = m.get(k) if (two_component or k in ("S", "T", "V", "W0")) else None
        _check_tensor(t, n)
        setattr(s, k, _ptr(t).value if t is not None else None)
    return s


def _alloc_parts(n, nc, device, like=None):
    torch = _torch()
    return [torch.empty((n, n), dtype=torch.float64, device=device) for _ in range(nc)]


def _hout(parts):
    h = abi.HOut()
    for q, t in enumerate(parts):
        h.h[q] = t.data_ptr()
    return h


def x2c_build_full(ctx: Context, m: dict, two_component=False, c=None, want_U=False, stream=None,
                   out=None, U_out=None, decoupling=DEC_X2C):
    """Full X2C: returns dict(h=[h0..], UL=[..], US=[..]) of CUDA tensors (quaternion parts).
    out / U_out = (UL parts, US parts): caller-owned outputs instead of new tensors."""
    nc = 4 if two_component else 1
    ms = mats_struct(m, two_component)
    dev = m["S"].device
    h = out if out is not None else _alloc_parts(ms.n, nc, dev)
    U = None
    out = dict(h=h)
    if want_U or U_out is not None:
        UL, US = U_out if U_out is not None else (_alloc_parts(ms.n, nc, dev), _alloc_parts(ms.n, nc, dev))
        U = abi.UOut()
        for q in range(nc):
            U.UL[q] = UL[q].data_ptr()
            U.US[q] = US[q].data_ptr()
        out.update(UL=UL, US=US)
    o = options(two_component, c, decoupling=decoupling)
    ho = _hout(h)
    abi.check(ctx.lib.x2c_build_full(ctx.handle, ctypes.byref(o), ctypes.byref(ms), ctypes.byref(ho),
                                     ctypes.byref(U) if U is not None else None, _stream(stream)),
              "x2c_build_full", ctx.handle)
    return out


class LayoutHolder:
    """Keeps the host arrays of an x2c_layout alive."""

    def __init__(self, offsets, atom_kind=None, kinds=None, two_component=False):
        self.off = np.ascontiguousarray(offsets, dtype=np.int32)
        self.kind = None if atom_kind is None else np.ascontiguousarray(atom_kind, dtype=np.int32)
        self.kinds = kinds or []
        self.kind_structs = (abi.Mats * max(1, len(self.kinds)))()
        for i, k in enumerate(self.kinds):
            self.kind_structs[i] = mats_struct(k, two_component) if isinstance(k, dict) else k
        self.s = abi.Layout()
        self.s.n_atoms = len(self.off) - 1
        self.s.atom_offset = self.off.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        self.s.atom_kind = (self.kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
                            if self.kind is not None else None)
        self.s.n_kinds = len(self.kinds)
        self.s.kinds = ctypes.cast(self.kind_structs, ctypes.POINTER(abi.Mats)) if self.kinds else None


def x2c_build_dlu(ctx: Context, m: dict, offsets, atom_kind=None, kinds=None, two_component=False,
                  c=None, precision=PREC_FP64, dlu_potential=DLU_FREE_ATOM, so_same_atom_only=True,
                  n_slices=0, local_approx=LOCAL_DLU, out=None, stream=None, decoupling=DEC_X2C):
    """DLU build.  m: molecular matrices (CUDA tensors); kinds: list of free-atom input dicts
    (FREE_ATOM mode) indexed by atom_kind.  Returns the list of h parts."""
    nc = 4 if two_component else 1
    ms = mats_struct(m, two_component)
    h = out if out is not None else _alloc_parts(ms.n, nc, m["S"].device)
    lay = LayoutHolder(offsets, atom_kind, kinds, two_component)
    o = options(two_component, c, precision, dlu_potential, so_same_atom_only, n_slices, local_approx,
                decoupling=decoupling)
    ho = _hout(h)
    abi.check(ctx.lib.x2c_build_dlu(ctx.handle, ctypes.byref(o), ctypes.byref(lay.s), ctypes.byref(ms),
                                    ctypes.byref(ho), _stream(stream)), "x2c_build_dlu", ctx.handle)
    return h


def neighbour_mask(coords, cutoff: float):
    """Atoms within `cutoff` (bohr) of each other, as the n_atoms x n_atoms byte mask of
    x2c_build_dlu_nab."""
    xyz = np.asarray(coords, dtype=np.float64)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)
    return np.ascontiguousarray(d <= cutoff, dtype=np.uint8)


def x2c_build_dlu_nab(ctx: Context, m: dict, offsets, atom_kind, kinds, neighbours, two_component=False, c=None,
                      precision=PREC_FP64, so_same_atom_only=True, n_slices=0, out=None, stream=None,
                      decoupling=DEC_X2C):
    """x2c_build_dlu_nab: DLU blocks for neighbouring atoms (mask `neighbours`, n_atoms x
    n_atoms), T + V on every other block."""
    nc = 4 if two_component else 1
    ms = mats_struct(m, two_component)
    L = len(offsets) - 1
    nbr = np.ascontiguousarray(neighbours, dtype=np.uint8)
    if nbr.shape != (L, L):
        raise ValueError("neighbours must be n_atoms x n_atoms")
    h = out if out is not None else _alloc_parts(ms.n, nc, m["S"].device)
    lay = LayoutHolder(offsets, atom_kind, kinds, two_component)
    o = options(two_component, c, precision, DLU_FREE_ATOM, so_same_atom_only, n_slices, decoupling=decoupling)
    ho = _hout(h)
    abi.check(ctx.lib.x2c_build_dlu_nab(ctx.handle, ctypes.byref(o), ctypes.byref(lay.s), ctypes.byref(ms),
                                        nbr.ctypes.data, ctypes.byref(ho), _stream(stream)),
              "x2c_build_dlu_nab", ctx.handle)
    return h


def x2c_dlu_partition(offsets, rank: int, world: int):
    """x2c_dlu_partition: the row atoms [a_begin, a_end) of rank `rank` of `world` in a
    pair-list partitioned DLU build (host-only; no device, no context)."""
    lay = LayoutHolder(offsets)
    a0, a1 = ctypes.c_int32(), ctypes.c_int32()
    abi.check(abi.load().x2c_dlu_partition(ctypes.byref(lay.s), int(rank), int(world), ctypes.byref(a0),
                                           ctypes.byref(a1)), "x2c_dlu_partition")
    return a0.value, a1.value


def x2c_build_dlu_rows(ctx: Context, m: dict, offsets, atom_kind, kinds, a_begin: int, a_end: int, two_component=False,
                       c=None, precision=PREC_FP64, dlu_potential=DLU_FREE_ATOM, so_same_atom_only=True, n_slices=0,
                       out=None, stream=None, decoupling=DEC_X2C):
    """x2c_build_dlu_rows: one rank's share of a partitioned DLU build (the pair blocks whose
    row atom lies in [a_begin, a_end)); other blocks of `out` are left as they were."""
    nc = 4 if two_component else 1
    ms = mats_struct(m, two_component)
    h = out if out is not None else _alloc_parts(ms.n, nc, m["S"].device)
    lay = LayoutHolder(offsets, atom_kind, kinds, two_component)
    o = options(two_component, c, precision, dlu_potential, so_same_atom_only, n_slices, decoupling=decoupling)
    ho = _hout(h)
    abi.check(ctx.lib.x2c_build_dlu_rows(ctx.handle, ctypes.byref(o), ctypes.byref(lay.s), ctypes.byref(ms),
                                         ctypes.byref(ho), int(a_begin), int(a_end), _stream(stream)),
              "x2c_build_dlu_rows", ctx.handle)
    return h


def gather_dlu_rows(h_parts: list, offsets, group=None, dst: int = 0):
    """Collect a pair-list partitioned DLU h on rank `dst` (torch.distributed; gloo or NCCL).

    Every rank passes its h parts (torch tensors, N x N, holding at least its own blocks: the
    rows of its atom range on and right of the diagonal block, as x2c_build_dlu_rows writes
    them).  Rank `dst` receives the other ranks' row bands, keeps the upper block triangle of
    each and mirrors it (h0 symmetric, h1..h3 antisymmetric) into the lower one; it returns
    the complete parts, the other ranks return None.  This is the optional gather of a
    partitioned build: the build itself exchanges nothing."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    offs = np.asarray(offsets, dtype=np.int64)
    N = int(offs[-1])
    atom = np.repeat(np.arange(len(offs) - 1), np.diff(offs))
    rows = [x2c_dlu_partition(offsets, r, world) for r in range(world)]
    out = []
    for q, hq in enumerate(h_parts):
        bands = []
        for r, (a0, a1) in enumerate(rows):
            r0, r1 = int(offs[a0]), int(offs[a1])
            if r1 == r0:
                continue
            if r == rank:
                band = hq[r0:r1].contiguous()
                if rank != dst:
                    dist.send(band, dst=dst, group=group)
            else:
                if rank != dst:
                    continue
                band = torch.empty((r1 - r0, N), dtype=hq.dtype, device=hq.device)
                dist.recv(band, src=r, group=group)
            bands.append(band)
        if rank != dst:
            continue
        full = torch.cat(bands, 0)
        keep = torch.from_numpy(atom[:, None] <= atom[None, :]).to(full.device)
        upper = torch.where(keep, full, torch.zeros_like(full))
        out.append(torch.where(keep, full, upper.transpose(0, 1) * (1.0 if q == 0 else -1.0)))
    return out if rank == dst else None


def x2c_build_dlu_batched(ctx: Context, mols: list, layouts: list, two_component=False, c=None,
                          precision=PREC_FP64, dlu_potential=DLU_FREE_ATOM, so_same_atom_only=True,
                          n_slices=0, local_approx=LOCAL_DLU, outs=None, stream=None, decoupling=DEC_X2C):
    """Batched DLU over several molecules.  mols: list of matrix dicts; layouts: list of
    (offsets, atom_kind, kinds) tuples.  Returns a list of h-part lists."""
    nc = 4 if two_component else 1
    n_mol = len(mols)
    ms = (abi.Mats * n_mol)()
    ls = (abi.Layout * n_mol)()
    hs = (abi.HOut * n_mol)()
    holders, outs_ = [], []
    for i, (m, lay) in enumerate(zip(mols, layouts)):
        ms[i] = mats_struct(m, two_component)
        holder = LayoutHolder(*lay, two_component=two_component)
        holders.append(holder)
        ls[i] = holder.s
        h = outs[i] if outs is not None else _alloc_parts(ms[i].n, nc, m["S"].device)
        outs_.append(h)
        hs[i] = _hout(h)
    o = options(two_component, c, precision, dlu_potential, so_same_atom_only, n_slices, local_approx,
                decoupling=decoupling)
    abi.check(ctx.lib.x2c_build_dlu_batched(ctx.handle, ctypes.byref(o), n_mol, ls, ms, hs, _stream(stream)),
              "x2c_build_dlu_batched", ctx.handle)
    return outs_


def x2c_atomic_transforms(ctx: Context, inputs: list, two_component=False, c=None, stream=None, out=None,
                          decoupling=DEC_X2C):
    """Decoupling transforms of independent input sets: list of (UL parts, US parts)
    (`out`: caller-owned list of the same form)."""
    nc = 4 if two_component else 1
    k = len(inputs)
    ms = (abi.Mats * k)()
    us = (abi.UOut * k)()
    res = []
    for i, m in enumerate(inputs):
        ms[i] = mats_struct(m, two_component)
        if out is not None:
            UL, US = out[i]
        else:
            UL, US = _alloc_parts(ms[i].n, nc, m["S"].device), _alloc_parts(ms[i].n, nc, m["S"].device)
        for q in range(nc):
            us[i].UL[q] = UL[q].data_ptr()
            us[i].US[q] = US[q].data_ptr()
        res.append((UL, US))
    o = options(two_component, c, decoupling=decoupling)
    abi.check(ctx.lib.x2c_atomic_transforms(ctx.handle, ctypes.byref(o), k, ms, us, _stream(stream)),
              "x2c_atomic_transforms", ctx.handle)
    return res


def x2c_atomic_transforms_noalloc(inputs: list, two_component=False, c=None, out=None, stream=None):
    """x2c_atomic_transforms_noalloc: the batched decoupling solve with no device allocation
    inside the library (fixed scratch array, no context).  Output tensors are allocated here
    by torch unless `out` (list of (UL parts, US parts)) is given.  Synchronous."""
    nc = 4 if two_component else 1
    k = len(inputs)
    ms = (abi.Mats * k)()
    us = (abi.UOut * k)()
    res = []
    for i, m in enumerate(inputs):
        ms[i] = mats_struct(m, two_component)
        if out is not None:
            UL, US = out[i]
        else:
            UL, US = _alloc_parts(ms[i].n, nc, m["S"].device), _alloc_parts(ms[i].n, nc, m["S"].device)
        for q in range(nc):
            us[i].UL[q] = UL[q].data_ptr()
            us[i].US[q] = US[q].data_ptr()
        res.append((UL, US))
    o = options(two_component, c)
    abi.check(abi.load().x2c_atomic_transforms_noalloc(ctypes.byref(o), k, ms, us, _stream(stream)),
              "x2c_atomic_transforms_noalloc")
    return res


def x2c_build_dlu_host(ctx: Context, m: dict, offsets, atom_kind=None, kinds=None, two_component=False,
                       c=None, precision=PREC_FP64, dlu_potential=DLU_FREE_ATOM, so_same_atom_only=True,
                       n_slices=0, local_approx=LOCAL_DLU, out=None, stream=None, h_upper_only=False,
                       decoupling=DEC_X2C):
    """DLU build from HOST arrays (numpy float64 or CPU torch tensors, pinned or not);
    h parts are written into `out` (host arrays) or new numpy arrays.  h_upper_only: the
    upper block triangle of each part is written (blocks below the diagonal keep what `out`
    held, except a few near the diagonal, which receive their values)."""
    nc = 4 if two_component else 1
    n = m["S"].shape[0]

    def hp(a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("host matrices must be C-contiguous float64")
            return a.ctypes.data
        return a.data_ptr()

    def hmats(d, nn):
        s = abi.Mats()
        s.n = nn
        for k in _MAT_KEYS:
            t = d.get(k) if (two_component or k in ("S", "T", "V", "W0")) else None
            setattr(s, k, hp(t))
        return s

    ms = hmats(m, n)
    kind_structs = [hmats(k, k["S"].shape[0]) for k in (kinds or [])]
    lay = LayoutHolder(offsets, atom_kind, kind_structs, two_component)
    if out is None:
        out = [np.empty((n, n)) for _ in range(nc)]
    ho = abi.HOut()
    for q in range(nc):
        ho.h[q] = hp(out[q])
    o = options(two_component, c, precision, dlu_potential, so_same_atom_only, n_slices, local_approx,
                h_upper_only, decoupling)
    abi.check(ctx.lib.x2c_build_dlu_host(ctx.handle, ctypes.byref(o), ctypes.byref(lay.s), ctypes.byref(ms),
                                         ctypes.byref(ho), _stream(stream)), "x2c_build_dlu_host", ctx.handle)
    return out


def x2c_s_integrals(nuc_xyz, nuc_z, bf_xyz, bf_alpha, want=("S", "T", "V", "W0"), stream=None):
    """S, T, V, W0 over primitive s Gaussians computed on the device (x2c_s_integrals).
    Arguments: CUDA float64 tensors (nuclei (L, 3) and (L,), basis centres (n, 3) and
    exponents (n,)).  Returns a dict of n x n CUDA tensors for the requested matrices."""
    torch = _torch()
    args = [nuc_xyz, nuc_z, bf_xyz, bf_alpha]
    for t in args:
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError("expected contiguous float64 tensors")
    # the kernel takes n from bf_alpha and the nucleus count from nuc_z: every other array
    # must have exactly the matching shape, or it would be read out of bounds
    if bf_alpha.dim() != 1 or bf_alpha.shape[0] < 1 or tuple(bf_xyz.shape) != (bf_alpha.shape[0], 3):
        raise ValueError("bf_xyz must be (n, 3) and bf_alpha (n,) with n >= 1")
    if nuc_z.dim() != 1 or tuple(nuc_xyz.shape) != (nuc_z.shape[0], 3):
        raise ValueError("nuc_xyz must be (L, 3) and nuc_z (L,)")
    if not all(t.is_cuda for t in args) or len({t.device for t in args}) != 1:
        raise ValueError("all four tensors must be on the same CUDA device")
    n = int(bf_alpha.shape[0])
    b = abi.SBasis()
    b.n_nuc = int(nuc_z.shape[0])
    b.n = n
    b.nuc_xyz, b.nuc_z, b.bf_xyz, b.bf_alpha = (t.data_ptr() for t in args)
    out = {k: torch.empty((n, n), dtype=torch.float64, device=bf_alpha.device) for k in want}
    ptr = [out[k].data_ptr() if k in out else None for k in ("S", "T", "V", "W0")]
    abi.check(abi.load().x2c_s_integrals(ctypes.byref(b), *ptr, _stream(stream)), "x2c_s_integrals")
    return out


def x2c_quaternion_to_dense(h_parts: list, stream=None):
    """Dense spin-blocked complex 2n x 2n matrix (complex128 CUDA tensor) from h parts."""
    torch = _torch()
    n = h_parts[0].shape[0]
    out = torch.empty((2 * n, 2 * n), dtype=torch.complex128, device=h_parts[0].device)
    arr = (ctypes.c_void_p * 4)(*[(h_parts[q].data_ptr() if q < len(h_parts) else None) for q in range(4)])
    abi.check(abi.load().x2c_quaternion_to_dense(arr, n, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
              "x2c_quaternion_to_dense")
    return out


def x2c_build_dlu_with_transforms(ctx: Context, m: dict, offsets, atom_kind, kinds_U, kind_sizes,
                                  two_component=False, c=None, precision=PREC_FP64, so_same_atom_only=True,
                                  n_slices=0, local_approx=LOCAL_DLU, out=None, stream=None):
    """DLU build (free-atom mode) from given per-kind transforms: kinds_U is a list of
    (UL parts, US parts) CUDA tensors (e.g. from x2c_atomic_transforms), kind_sizes the
    kinds' basis sizes.  Returns the list of h parts."""
    nc = 4 if two_component else 1
    ms = mats_struct(m, two_component)
    h = out if out is not None else _alloc_parts(ms.n, nc, m["S"].device)
    kind_structs = []
    for n in kind_sizes:
        k = abi.Mats()
        k.n = int(n)
        kind_structs.append(k)
    lay = LayoutHolder(offsets, atom_kind, kind_structs, two_component)
    us = (abi.UOut * len(kinds_U))()
    for i, (UL, US) in enumerate(kinds_U):
        for q in range(nc):
            us[i].UL[q] = UL[q].data_ptr()
            us[i].US[q] = US[q].data_ptr()
    o = options(two_component, c, precision, DLU_FREE_ATOM, so_same_atom_only, n_slices, local_approx)
    ho = _hout(h)
    abi.check(ctx.lib.x2c_build_dlu_with_transforms(ctx.handle, ctypes.byref(o), ctypes.byref(lay.s), us,
                                                    ctypes.byref(ms), ctypes.byref(ho), _stream(stream)),
              "x2c_build_dlu_with_transforms", ctx.handle)
    return h



def x2c_picture_change(ctx: Context, P_LL, P_SS, offsets, atom_kind, kinds_U, kind_sizes, two_component=False,
                       precision=PREC_FP64, so_same_atom_only=True, n_slices=0, out=None, stream=None):
    """Picture-change transformation P2c = U^L+ P^LL U^L + U^S+ P^SS U^S of a property
    operator without large-small coupling.  P_LL: CUDA tensor (n x n); P_SS: one tensor
    (spin-free) or a list of the quaternion parts [SS0, SS1, SS2, SS3] (SS1..3 may be None);
    the transforms as in x2c_build_dlu_with_transforms (one "atom" spanning the basis for
    full-X2C transforms).  Returns the list of P2c parts."""
    nc = 4 if two_component else 1
    ss = list(P_SS) if isinstance(P_SS, (list, tuple)) else [P_SS]
    ss += [None] * (4 - len(ss))
    n = int(P_LL.shape[0])
    for t in [P_LL] + ss:
        _check_tensor(t, n)
    p = abi.Property()
    p.n = n
    p.LL = P_LL.data_ptr()
    for q in range(4):
        p.SS[q] = ss[q].data_ptr() if ss[q] is not None else None
    h = out if out is not None else _alloc_parts(n, nc, P_LL.device)
    kind_structs = []
    for kn in kind_sizes:
        k = abi.Mats()
        k.n = int(kn)
        kind_structs.append(k)
    lay = LayoutHolder(offsets, atom_kind, kind_structs, two_component)
    us = (abi.UOut * len(kinds_U))()
    for i, (UL, US) in enumerate(kinds_U):
        for q in range(nc):
            us[i].UL[q] = UL[q].data_ptr()
            us[i].US[q] = US[q].data_ptr()
    o = options(two_component, None, precision, DLU_FREE_ATOM, so_same_atom_only, n_slices)
    ho = _hout(h)
    abi.check(ctx.lib.x2c_picture_change(ctx.handle, ctypes.byref(o), ctypes.byref(lay.s), us, ctypes.byref(p),
                                         ctypes.byref(ho), _stream(stream)), "x2c_picture_change", ctx.handle)
    return h

def x2c_query_workspace(ctx: Context, m: dict, offsets=None, atom_kind=None, kinds=None, two_component=False,
                        precision=PREC_FP64, dlu_potential=DLU_FREE_ATOM, full=False):
    """x2c_query_workspace: device workspace bytes a DLU (or, with full=True, a full X2C)
    build of these inputs would need (nothing runs)."""
    ms = mats_struct(m, two_component)
    o = options(two_component, None, precision, dlu_potential)
    out = ctypes.c_size_t()
    if full:
        abi.check(ctx.lib.x2c_query_workspace(ctx.handle, ctypes.byref(o), 0, None, ctypes.byref(ms),
                                              ctypes.byref(out)), "x2c_query_workspace")
    else:
        lay = LayoutHolder(offsets, atom_kind, kinds, two_component)
        abi.check(ctx.lib.x2c_query_workspace(ctx.handle, ctypes.byref(o), 1, ctypes.byref(lay.s), ctypes.byref(ms),
                                              ctypes.byref(out)), "x2c_query_workspace")
    return out.value


# ---- serving ------------------------------------------------------------------------------

REQ_DLU, REQ_FULL = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
STATE_QUEUED, STATE_RUNNING, STATE_DONE = 0, 1, 2


class _DeviceView:
    """__cuda_array_interface__ of a float64 n x n matrix the server owns (no ownership here)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n, n), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _mat_ptr_ld(a, host):
    """(address, leading dimension) of a row-major float64 matrix or a row-major view of one."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not host:
            raise ValueError("numpy arrays are host memory")
        if a.dtype != np.float64 or a.ndim != 2 or a.strides[1] != 8:
            raise ValueError("host matrices must be float64 with unit column stride")
        return a.ctypes.data, a.strides[0] // 8
    torch = _torch()
    if not isinstance(a, torch.Tensor) or a.dtype != torch.float64 or a.dim() != 2 or a.stride(1) != 1:
        raise ValueError("matrices must be float64 tensors with unit column stride")
    if a.is_cuda == host:
        raise ValueError("device request needs CUDA tensors, host request CPU tensors")
    return a.data_ptr(), a.stride(0)


class Server:
    """x2c_server_*: continuous-batching X2C/DLU server on one GPU.

    Requests keep references to their input (and host output) arrays until release(); the
    arrays must not change until the request is DONE."""

    def __init__(self, device=0, max_inflight=4, max_batch=16, hbm_budget_bytes=0):
        self.lib = abi.load()
        o = abi.ServerOptions()
        o.device, o.max_inflight, o.max_batch = int(device), int(max_inflight), int(max_batch)
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        h = ctypes.c_void_p()
        abi.check(self.lib.x2c_server_create(ctypes.byref(o), ctypes.byref(h)), "x2c_server_create")
        self.handle = h
        self.device = device
        self._keep = {}
        self._shape = {}

    def close(self):
        if self.handle:
            self.lib.x2c_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def now(self):
        t = ctypes.c_double()
        abi.check(self.lib.x2c_server_now(self.handle, ctypes.byref(t)), "x2c_server_now")
        return t.value

    def _submit(self, req, keep, n, nc):
        t = ctypes.c_uint64()
        abi.check(self.lib.x2c_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)), "x2c_server_submit")
        self._keep[t.value] = (req,) + tuple(keep)
        self._shape[t.value] = (n, nc)
        return t.value

    def _mats(self, m, two_component, host):
        s = abi.Mats()
        lds = set()
        n = None
        for k in _MAT_KEYS:
            a = m.get(k) if (two_component or k in ("S", "T", "V", "W0")) else None
            p, ld = _mat_ptr_ld(a, host)
            setattr(s, k, p)
            if a is not None:
                lds.add(ld)
                n = a.shape[0] if n is None else n
                if tuple(a.shape) != (n, n):
                    raise ValueError("all matrices must be n x n")
        if len(lds) != 1:
            raise ValueError("all molecular matrices must share one leading dimension")
        s.n = n
        return s, lds.pop()

    def submit_dlu(self, m, offsets, atom_kind, kinds, kind_keys=None, two_component=False, c=None,
                   precision=PREC_FP64, n_slices=0, local_approx=LOCAL_DLU, so_same_atom_only=True,
                   dlu_potential=DLU_FREE_ATOM, out=None, host=False, t_arrival=-1.0, decoupling=DEC_X2C):
        """Queue a DLU build.  m: molecular matrices (CUDA tensors, or host arrays with
        host=True; row-major views such as big[:n, :n] are allowed); kinds: free-atom input
        dicts; kind_keys: one integer cache key per kind (0 = not cached); out: result
        buffers (device, or host with host=True), None = server-allocated device result."""
        nc = 4 if two_component else 1
        req = abi.Request()
        req.opt = options(two_component, c, precision, dlu_potential, so_same_atom_only, n_slices, local_approx,
                          decoupling=decoupling)
        req.kind, req.memory = REQ_DLU, (MEM_HOST if host else MEM_DEVICE)
        req.mol, ld = self._mats(m, two_component, host)
        req.ld = ld
        kstructs = []
        for k in (kinds or []):
            ks, _ = self._mats(k, two_component, host)
            kstructs.append(ks)
        lay = LayoutHolder(offsets, atom_kind, kstructs, two_component)
        req.layout = lay.s
        keys = None
        if kind_keys is not None:
            keys = (ctypes.c_uint64 * len(kind_keys))(*[int(k) for k in kind_keys])
            req.kind_key = ctypes.cast(keys, ctypes.POINTER(ctypes.c_uint64))
        outs = []
        if out is not None:
            for q in range(nc):
                p, _ = _mat_ptr_ld(out[q], host)
                req.out.h[q] = p
            outs = list(out)
        req.t_arrival = float(t_arrival)
        return self._submit(req, (m, kinds, lay, keys, outs), req.mol.n, nc)

    def submit_full(self, m, two_component=False, c=None, out=None, host=False, t_arrival=-1.0,
                    decoupling=DEC_X2C):
        """Queue a full X2C build of the whole system (see submit_dlu for the arguments)."""
        nc = 4 if two_component else 1
        req = abi.Request()
        req.opt = options(two_component, c, decoupling=decoupling)
        req.kind, req.memory = REQ_FULL, (MEM_HOST if host else MEM_DEVICE)
        req.mol, ld = self._mats(m, two_component, host)
        req.ld = ld
        outs = []
        if out is not None:
            for q in range(nc):
                p, _ = _mat_ptr_ld(out[q], host)
                req.out.h[q] = p
            outs = list(out)
        req.t_arrival = float(t_arrival)
        return self._submit(req, (m, outs), req.mol.n, nc)

    def _result(self, ticket, r):
        d = {k: getattr(r, k) for k in ("state", "status", "t_arrival", "t_submit", "t_admit", "t_start", "t_end",
                                        "batch_size", "cache_hits", "cache_misses", "slot")}
        d["h_ptr"] = [r.h[q] for q in range(4)]
        return d

    def poll(self, ticket):
        r = abi.Result()
        abi.check(self.lib.x2c_server_poll(self.handle, int(ticket), ctypes.byref(r)), "x2c_server_poll")
        return self._result(ticket, r)

    def wait(self, ticket, timeout_ms=120000):
        """Wait for a request; returns its result dict (status X2C_ERR_TIMEOUT = 9 is raised)."""
        r = abi.Result()
        abi.check(self.lib.x2c_server_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(r)),
                  "x2c_server_wait")
        return self._result(ticket, r)

    def result_tensors(self, ticket, res=None):
        """The device result of a DONE request as torch tensors viewing server memory (valid
        until release)."""
        torch = _torch()
        res = res or self.poll(ticket)
        n, nc = self._shape[ticket]
        return [torch.as_tensor(_DeviceView(res["h_ptr"][q], n), device=f"cuda:{self.device}") for q in range(nc)]

    def cancel(self, ticket):
        abi.check(self.lib.x2c_server_cancel(self.handle, int(ticket)), "x2c_server_cancel")

    def release(self, ticket):
        abi.check(self.lib.x2c_server_release(self.handle, int(ticket)), "x2c_server_release")
        self._keep.pop(ticket, None)
        self._shape.pop(ticket, None)

    def stats(self):
        s = abi.ServerStats()
        abi.check(self.lib.x2c_server_get_stats(self.handle, ctypes.byref(s)), "x2c_server_get_stats")
        return {k: getattr(s, k) for k, _ in abi.ServerStats._fields_ if k != "reserved"}

    def reset_stats(self):
        abi.check(self.lib.x2c_server_reset_stats(self.handle), "x2c_server_reset_stats")
