"""Pair-list partition of a DLU build over several GPUs (Sec. III.A: the pair blocks h_AB of
Eqs. 42-43 are independent), on the CPU:

* x2c_dlu_partition gives every rank a consecutive range of row atoms; the ranges are
  disjoint, cover every atom, and share the upper-triangle work about equally;
* two gloo ranks each assemble only their pair blocks (the oracle's pair-block formula
  stands in for the GPU assembly here) and gather_dlu_rows collects them on rank 0, which
  must reproduce the one-rank DLU h."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import paper_1303_4446_gb300 as x  # noqa: E402
from paper_1303_4446_gb300 import workload as w  # noqa: E402


def _work(offsets, a0, a1):
    n = np.diff(np.asarray(offsets, dtype=float))
    return sum(n[a] * n[b] * (n[a] + n[b]) for a in range(a0, a1) for b in range(a, len(n)))


@pytest.mark.parametrize("offsets", [w.silver_cluster(309, "s48").offsets, w.silver_cluster(4, "s30").offsets,
                                     np.concatenate([[0], np.cumsum([30, 48, 48, 30, 7, 48, 30, 1, 48])])])
def test_partition_is_disjoint_complete_and_balanced(offsets):
    L = len(offsets) - 1
    total = _work(offsets, 0, L)
    for world in (1, 2, 3, 4, 8, 16):
        ranges = [x.x2c_dlu_partition(offsets, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == L
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0 and a0 <= a1
        if L >= 8 * world:  # enough rows to balance: no share far above the mean
            share = max(_work(offsets, a0, a1) for a0, a1 in ranges)
            assert share <= 1.15 * total / world, (world, share / (total / world))
    with pytest.raises(x.X2CError):
        x.x2c_dlu_partition(offsets, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, two_c, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    mol = w.silver_cluster(5, "s30")
    m = w.molecule_inputs(mol, two_c)
    kind = w.atomic_inputs(47.0, "s30", two_c)
    r = O.x2c_full(kind)
    offs = mol.offsets
    N = mol.nbf
    a0, a1 = x.x2c_dlu_partition(offs, rank, world)
    nc = 4 if two_c else 1
    h = [torch.full((N, N), float("nan"), dtype=torch.float64) for _ in range(nc)]
    keys = ("V", "T", "W0") + (("Wx", "Wy", "Wz") if two_c else ())
    for A in range(a0, a1):  # this rank's pair blocks only
        for B in range(A, mol.natoms):
            ra, rb = slice(offs[A], offs[A + 1]), slice(offs[B], offs[B + 1])
            blk = O.dlu_pair_block({k: m[k][ra, rb] for k in keys}, r["UL"], r["US"], r["UL"], r["US"])
            parts = O.quaternion_parts(blk) if two_c else [blk]
            for q in range(nc):
                h[q][ra, rb] = torch.from_numpy(np.ascontiguousarray(parts[q]))
    full = x.gather_dlu_rows(h, offs)
    if rank == 0:
        ref = O.x2c_dlu(m, offs, [kind] * mol.natoms)["h"]
        ref = O.quaternion_parts(ref) if two_c else [ref]
        scale = max(np.abs(p).max() for p in ref)
        out["err"] = max(np.abs(f.numpy() - p).max() for f, p in zip(full, ref)) / scale
        out["ranges"] = [x.x2c_dlu_partition(offs, q, world) for q in range(world)]
    else:
        out[f"none{rank}"] = full is None
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("two_c", [False, True])
def test_two_ranks_assemble_and_gather_the_one_rank_h(two_c):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, two_c, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert res["none1"]
    assert res["ranges"][0][1] == res["ranges"][1][0] and 0 < res["ranges"][0][1] < 5
    assert res["err"] <= 1e-13, res["err"]
