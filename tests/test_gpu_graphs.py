"""CUDA-graph replay of repeated builds (x2c_ctx_set_graphs).

A replayed build launches exactly the kernels the eager build enqueues, with the same
autotuned choices and the same deterministic reductions, so its h must be bit-identical to
an eager build of the same inputs; the eager builds themselves are held to the oracle by the
parity tests.  The inputs are read when the graph runs, so a replay after the matrices change
in place must give the eager result of the new matrices."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eager():
    c = x.Context(0)
    yield c
    c.close()


@pytest.fixture()
def gctx():
    c = x.Context(0)
    c.set_graphs(True)
    yield c
    c.close()


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


def poison(parts):
    for p in parts:
        p.fill_(float("nan"))


def same(a, b):
    return all(torch.equal(p, q) for p, q in zip(a, b))


@pytest.mark.parametrize("prec", [x.PREC_SPLIT_BF16, x.PREC_FP64])
def test_replay_is_bit_identical_and_reads_new_contents(eager, gctx, prec):
    mol = w.silver_cluster(13, "s30")
    m, kind = w.molecule_inputs(mol, True), w.atomic_inputs(47.0, "s30", True)
    g, gk = dev(m), dev(kind)
    L = mol.natoms
    args = (mol.offsets, [0] * L, [gk])
    for _ in range(2):  # the second eager build runs the tuned kernels only
        ref = x.x2c_build_dlu(eager, g, *args, two_component=True, precision=prec)
    eager.status()
    out = [torch.empty_like(p) for p in ref]
    for i in range(4):
        poison(out)
        x.x2c_build_dlu(gctx, g, *args, two_component=True, precision=prec, out=out)
        gctx.status()
        assert same(out, ref), i
        st = gctx.graph_stats()
        assert st["last_replayed"] == (i >= 1), (i, st)
        assert gctx.counters()["pair_blocks"] == L * (L + 1) // 2
    assert st["captures"] == 1 and st["replays"] == 3 and st["cached"] == 1
    assert gctx.counters()["kernel_launches"] == eager.counters()["kernel_launches"]
    # new contents behind the same pointers: the graph reads them when it runs
    g["V"].mul_(1.001)
    g["W0"].mul_(0.999)
    ref2 = x.x2c_build_dlu(eager, g, *args, two_component=True, precision=prec)
    poison(out)
    x.x2c_build_dlu(gctx, g, *args, two_component=True, precision=prec, out=out)
    gctx.status()
    assert gctx.graph_stats()["last_replayed"]
    assert same(out, ref2) and not same(ref, ref2)
    # the replayed result still meets the oracle (pair blocks on the same-atom diagonal)
    mv = {k: v.cpu().numpy() for k, v in g.items()}
    r = O.x2c_full(kind)
    a = slice(int(mol.offsets[0]), int(mol.offsets[1]))
    blk = O.dlu_pair_block({k: mv[k][a, a] for k in ("V", "T", "W0", "Wx", "Wy", "Wz")},
                           r["UL"], r["US"], r["UL"], r["US"])
    got = O.from_quaternion(*[p[a, a].cpu().numpy() for p in out])
    tol = 1e-9 if prec == x.PREC_SPLIT_BF16 else 1e-10
    assert np.abs(got - blk).max() <= tol * np.abs(blk).max()


def test_batched_size_groups_on_side_streams(eager, gctx):
    # two kinds of different size in molecular-block mode: one solve group per atom size,
    # the groups forked onto the context's side streams inside the capture
    pool = w.batched_molecules(count=16, lo=2, hi=9)
    mols = [mo for mo in pool if mo.basis[0] == "s30"][:3] + [mo for mo in pool if mo.basis[0] == "s48"][:3]
    ms = [dev(w.molecule_inputs(mo, False)) for mo in mols]
    lays = [(mo.offsets, None, None) for mo in mols]
    kw = dict(precision=x.PREC_FP64, dlu_potential=x.DLU_MOLECULAR_BLOCK)
    ref = x.x2c_build_dlu_batched(eager, ms, lays, **kw)
    eager.status()
    outs = [[torch.empty_like(p) for p in r] for r in ref]
    for i in range(3):
        for o in outs:
            poison(o)
        x.x2c_build_dlu_batched(gctx, ms, lays, outs=outs, **kw)
        gctx.status()
        assert all(same(o, r) for o, r in zip(outs, ref)), i
    assert gctx.graph_stats()["replays"] == 2
    assert len({b for mo in mols for b in mo.basis}) == 2


def test_full_x2c_and_transforms_with_U(eager, gctx):
    mol = w.silver_cluster(2, "s30")
    m = dev(w.molecule_inputs(mol, True))
    ref = x.x2c_build_full(eager, m, two_component=True, want_U=True)
    eager.status()
    h = [torch.empty_like(p) for p in ref["h"]]
    U = ([torch.empty_like(p) for p in ref["UL"]], [torch.empty_like(p) for p in ref["US"]])
    for i in range(3):
        poison(h + U[0] + U[1])
        x.x2c_build_full(gctx, m, two_component=True, out=h, U_out=U)
        gctx.status()
        assert same(h, ref["h"]) and same(U[0], ref["UL"]) and same(U[1], ref["US"]), i
    kinds = [dev(w.atomic_inputs(47.0, b, False)) for b in ("s30", "s48")]
    tref = x.x2c_atomic_transforms(eager, kinds)
    eager.status()
    tout = [([torch.empty_like(p) for p in a], [torch.empty_like(p) for p in b]) for a, b in tref]
    for i in range(3):
        for a, b in tout:
            poison(a + b)
        x.x2c_atomic_transforms(gctx, kinds, out=tout)
        gctx.status()
        assert all(same(a, ra) and same(b, rb) for (a, b), (ra, rb) in zip(tout, tref)), i
    st = gctx.graph_stats()
    assert st["captures"] == 2 and st["replays"] == 4


def test_timing_sees_inside_replays(gctx):
    mol = w.silver_cluster(4, "s30")
    g, gk = dev(w.molecule_inputs(mol, True)), dev(w.atomic_inputs(47.0, "s30", True))
    args = (mol.offsets, [0] * mol.natoms, [gk])
    kw = dict(two_component=True, precision=x.PREC_SPLIT_BF16)
    plain = x.Context(0)
    for c in (plain, gctx):  # no tuning runs: every call launches the same kernels
        c.set_autotune(False)
    plain.set_timing(True)
    x.x2c_build_dlu(plain, g, *args, **kw)
    once = plain.kernel_times()
    plain.close()
    gctx.set_timing(True)
    out = [torch.empty_like(g["V"]) for _ in range(4)]
    for _ in range(3):  # eager, capture + launch, replay
        x.x2c_build_dlu(gctx, g, *args, out=out, **kw)
    gctx.status()
    assert gctx.graph_stats()["replays"] == 2
    times = gctx.kernel_times()
    assert set(times) == set(once)
    for name, (ms, n) in times.items():
        assert n == 3 * once[name][1], name
        assert ms > 0, name


def test_workspace_growth_drops_graphs_and_off_switch(eager, gctx):
    small = w.silver_cluster(2, "s30")
    big = w.silver_cluster(13, "s48")
    gs, gb = dev(w.molecule_inputs(small, False)), dev(w.molecule_inputs(big, False))
    ks, kb = dev(w.atomic_inputs(47.0, "s30", False)), dev(w.atomic_inputs(47.0, "s48", False))
    ref = x.x2c_build_dlu(eager, gs, small.offsets, [0] * small.natoms, [ks])
    eager.status()
    out = [torch.empty_like(ref[0])]
    for _ in range(2):
        x.x2c_build_dlu(gctx, gs, small.offsets, [0] * small.natoms, [ks], out=out)
    assert gctx.graph_stats()["captures"] == 1
    x.x2c_build_dlu(gctx, gb, big.offsets, [0] * big.natoms, [kb])  # grows the workspace
    poison(out)
    x.x2c_build_dlu(gctx, gs, small.offsets, [0] * small.natoms, [ks], out=out)
    gctx.status()
    assert same(out, ref)
    st = gctx.graph_stats()
    assert st["captures"] == 2 and st["cached"] == 1 and st["last_replayed"]
    gctx.set_graphs(False)
    assert gctx.graph_stats()["cached"] == 0
    poison(out)
    x.x2c_build_dlu(gctx, gs, small.offsets, [0] * small.natoms, [ks], out=out)
    gctx.status()
    assert same(out, ref) and not gctx.graph_stats()["last_replayed"]
