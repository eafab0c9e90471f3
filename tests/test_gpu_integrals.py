"""GPU parity of x2c_s_integrals (the input matrices computed on the device) with the
workload's host integral generator, and a DLU build fed by them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu


def gpu_ints(mol):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    return x.x2c_s_integrals(d(mol.coords), d(mol.Z), d(mol.bf_xyz), d(mol.bf_alpha))


@pytest.mark.parametrize("case", ["ag4", "mixed"])
def test_device_integrals_match_generator(case):
    if case == "ag4":
        mol = w.silver_cluster(4, "s30")
    else:
        mol = w.Molecule(np.array([[0.0, 0.0, 0.0], [3.86, 3.86, 0.0], [1.2, -0.7, 2.9]]),
                         np.array([47.0, 47.0, 1.0]), ["s48", "s30", "s30"])
    got = gpu_ints(mol)
    torch.cuda.synchronize()
    ref = w.integrals(mol)
    for k in ("S", "T", "V", "W0"):
        g = got[k].cpu().numpy()
        assert np.array_equal(g, g.T), k
        assert np.abs(g - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max(), k


def test_dlu_from_device_integrals():
    mol = w.silver_cluster(4, "s30")
    ctx = x.Context(0)
    try:
        m_host = w.molecule_inputs(mol, False)
        kind = {k: torch.from_numpy(v).cuda() for k, v in w.atomic_inputs(47.0, "s30", False).items()}
        ref = x.x2c_build_dlu(ctx, {k: torch.from_numpy(v).cuda() for k, v in m_host.items()}, mol.offsets,
                              [0] * 4, [kind])
        g = gpu_ints(mol)
        h = x.x2c_build_dlu(ctx, g, mol.offsets, [0] * 4, [kind])
        ctx.status()
        assert (h[0] - ref[0]).abs().max().item() <= 1e-11 * ref[0].abs().max().item()
    finally:
        ctx.close()
