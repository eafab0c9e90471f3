"""The row-range DLU build (x2c_build_dlu_rows), one GPU standing in for the ranks of a
pair-list partition: the ranks' builds, run one after another into the same h, give the
one-call build bit for bit (FP64 and split precision), and a rank's call leaves the blocks of
other ranks untouched."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
@pytest.mark.parametrize("world", [2, 3, 7])
def test_ranks_rebuild_the_whole_h(prec, world):
    mol = w.silver_cluster(13, "s30")
    m = {k: torch.from_numpy(v).cuda() for k, v in w.molecule_inputs(mol, True).items()}
    kind = {k: torch.from_numpy(v).cuda() for k, v in w.atomic_inputs(47.0, "s30", True).items()}
    ctx = x.Context(0)
    try:
        ref = x.x2c_build_dlu(ctx, m, mol.offsets, [0] * 13, [kind], two_component=True, precision=prec)
        N = mol.nbf
        h = [torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda") for _ in range(4)]
        for r in range(world):
            a0, a1 = x.x2c_dlu_partition(mol.offsets, r, world)
            if a1 > a0:
                x.x2c_build_dlu_rows(ctx, m, mol.offsets, [0] * 13, [kind], a0, a1, two_component=True,
                                     precision=prec, out=h)
            if r == 0:  # only rank 0's rows (and their mirrors) are written so far
                ctx.status()
                o0, o1 = int(mol.offsets[a0]), int(mol.offsets[a1])
                assert torch.isnan(h[0][o1:, o1:]).all()
                assert not torch.isnan(h[0][o0:o1, o0:]).any()
        ctx.status()
        for a, b in zip(h, ref):
            assert torch.equal(a, b)
    finally:
        ctx.close()
