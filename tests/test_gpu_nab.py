"""GPU parity of the neighbouring-atomic-blocks approximation (x2c_build_dlu_nab): DLU blocks
for neighbouring atoms, T + V elsewhere, against the oracle (x2c_nab), FP64 and split-precision
assembly; all-neighbours equals x2c_build_dlu and no-neighbours equals DLH bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
@pytest.mark.parametrize("two_c", [False, True])
@pytest.mark.parametrize("cutoff", [5.5, 7.8])
def test_nab_matches_oracle(prec, two_c, cutoff):
    mol = w.silver_cluster(13, "s30")
    m = w.molecule_inputs(mol, two_c)
    kind = w.atomic_inputs(47.0, "s30", two_c)
    nb = x.neighbour_mask(mol.coords, cutoff)
    ref = O.x2c_nab(m, mol.offsets, nb.astype(bool), [kind] * 13)
    ctx = x.Context(0)
    try:
        h = x.x2c_build_dlu_nab(ctx, dev(m), mol.offsets, [0] * 13, [dev(kind)], nb, two_component=two_c,
                                precision=prec)
        ctx.status()
        parts = O.quaternion_parts(ref) if two_c else [ref]
        err = max(np.abs(g.cpu().numpy() - r).max() for g, r in zip(h, parts)) / np.abs(ref).max()
        assert err <= (1e-10 if prec == x.PREC_FP64 else 1e-9), err
        L = 13
        g = dev(m)
        k = [dev(kind)]
        full = x.x2c_build_dlu_nab(ctx, g, mol.offsets, [0] * L, k, np.ones((L, L)),
                                   two_component=two_c, precision=prec)
        dlu = x.x2c_build_dlu(ctx, g, mol.offsets, [0] * L, k, two_component=two_c, precision=prec)
        none = x.x2c_build_dlu_nab(ctx, g, mol.offsets, [0] * L, k, np.zeros((L, L)), two_component=two_c,
                                   precision=prec)
        dlh = x.x2c_build_dlu(ctx, g, mol.offsets, [0] * L, k, two_component=two_c, precision=prec,
                              local_approx=x.LOCAL_DLH)
        ctx.status()
        for a, b in zip(full, dlu):
            assert torch.equal(a, b)
        for a, b in zip(none, dlh):
            assert torch.equal(a, b)
    finally:
        ctx.close()
