"""GPU checks of x2c_s_integrals (the input matrices computed on the device) against
independent pins (tests/integral_pins.py: one-centre closed forms, scipy's incomplete gamma
function, finite differences of the device's own S and V, quadrature), element by element;
a consistency check with the workload's host generator; and a DLU build fed by them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import integral_pins as P
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def ints(nuc_xyz, nuc_z, bf_xyz, bf_alpha):
    """The device routine as a callable on numpy arrays."""
    out = x.x2c_s_integrals(_d(np.reshape(nuc_xyz, (-1, 3))), _d(nuc_z), _d(np.reshape(bf_xyz, (-1, 3))), _d(bf_alpha))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def gpu_ints(mol):
    return x.x2c_s_integrals(_d(mol.coords), _d(mol.Z), _d(mol.bf_xyz), _d(mol.bf_alpha))


def _mixed():
    return w.Molecule(np.array([[0.0, 0.0, 0.0], [3.86, 3.86, 0.0], [1.2, -0.7, 2.9]]),
                      np.array([47.0, 47.0, 1.0]), ["s48", "s30", "s30"])


def test_one_centre_closed_forms():
    P.check_one_centre(ints)


def test_boys_function_through_V():
    P.check_boys_through_V(ints)


@pytest.mark.parametrize("case", ["ag4", "mixed"])
def test_elementwise_S_T_V_against_closed_forms(case):
    mol = w.silver_cluster(4, "s30") if case == "ag4" else _mixed()
    P.check_elementwise_V(ints, mol.coords, mol.Z, mol.bf_xyz, mol.bf_alpha)


def test_T_and_W0_are_gradients_of_S_and_V():
    P.check_finite_differences(ints)


@pytest.mark.parametrize("case", ["ag4", "mixed"])
def test_W0_elementwise_by_finite_differences(case):
    mol = w.silver_cluster(4, "s30") if case == "ag4" else _mixed()
    P.check_W0_elementwise_fd(ints, mol.coords, mol.Z, mol.bf_xyz, mol.bf_alpha)


def test_V_by_quadrature():
    P.check_quadrature(ints)


def test_consistent_with_the_workload_generator():
    """Element by element; W0 relative to max(|W0|, (a + b) |V|), the size of the terms it is
    summed from (some W0 elements nearly cancel, and the two routines round differently)."""
    mol = _mixed()
    got = ints(mol.coords, mol.Z, mol.bf_xyz, mol.bf_alpha)
    ref = w.integrals(mol)
    p = mol.bf_alpha[:, None] + mol.bf_alpha[None, :]
    for k in ("S", "T", "V", "W0"):
        scale = np.abs(ref[k]) if k != "W0" else np.maximum(np.abs(ref[k]), p * np.abs(ref["V"]))
        big = scale > 1e-290
        rel = np.abs(got[k] - ref[k])[big] / scale[big]
        assert rel.max() <= 1e-12, (k, rel.max())


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
