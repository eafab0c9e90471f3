"""CPU checks of the C ABI: the library exports every declared function, the ctypes
structs match the header's layout, and the quaternion sign tables of the kernels give
the product of the two-component matrices of Eq. 5 (checked against complex arithmetic)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1303_4446_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "x2c.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(x2c_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return ctypes.CDLL(build.LIB_PATH)


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(abi.exported_symbols()) == names


def test_ctypes_structs_match_header(tmp_path):
    exe = tmp_path / "abi_layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "abi_layout.c"), "-o", str(exe)])
    out = dict((l.split()[0], list(map(int, l.split()[1:]))) for l in
               subprocess.check_output([str(exe)], text=True).splitlines())
    O = abi.Options
    assert out["options"] == [ctypes.sizeof(O), O.two_component.offset, O.precision.offset,
                              O.so_same_atom_only.offset, O.n_slices.offset, O.local_approx.offset,
                              O.h_upper_only.offset, O.decoupling.offset]
    assert out["property"] == [ctypes.sizeof(abi.Property), abi.Property.LL.offset, abi.Property.SS.offset]
    assert out["mats"] == [ctypes.sizeof(abi.Mats), abi.Mats.S.offset, abi.Mats.Wz.offset]
    assert out["hout"] == [ctypes.sizeof(abi.HOut)]
    assert out["uout"] == [ctypes.sizeof(abi.UOut), abi.UOut.US.offset]
    L = abi.Layout
    assert out["layout"] == [ctypes.sizeof(L), L.atom_offset.offset, L.n_kinds.offset, L.kinds.offset]
    assert out["counters"] == [ctypes.sizeof(abi.Counters), abi.Counters.credited_flops.offset]
    SO, R, Re, SS = abi.ServerOptions, abi.Request, abi.Result, abi.ServerStats
    assert out["server_options"] == [ctypes.sizeof(SO), SO.hbm_budget_bytes.offset, SO.reserved.offset]
    assert out["request"] == [ctypes.sizeof(R), R.kind.offset, R.layout.offset, R.kind_key.offset, R.mol.offset,
                              R.ld.offset, R.out.offset, R.t_arrival.offset]
    assert out["result"] == [ctypes.sizeof(Re), Re.h.offset, Re.t_end.offset, Re.slot.offset]
    assert out["server_stats"] == [ctypes.sizeof(SS), SS.latency_p50_ms.offset, SS.bytes_in_use.offset,
                                   SS.max_concurrent.offset]
    G = abi.GraphStats
    assert out["graph_stats"] == [ctypes.sizeof(G), G.cached.offset, G.last_replayed.offset]


def _spinor(parts):
    sig = (np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]]))
    return np.kron(np.eye(2), parts[0]) + 1j * sum(np.kron(s, p) for s, p in zip(sig, parts[1:]))


def test_quaternion_tables_reproduce_spinor_products(tmp_path):
    exe = tmp_path / "quat"
    subprocess.check_call(["nvcc", "-std=c++17", "-o", str(exe),
                           os.path.join(ROOT, "tests", "native", "quat_tables.cu")])
    m = 3
    rng = np.random.default_rng(7)
    A = rng.standard_normal((4, m, m))
    B = rng.standard_normal((4, m, m))
    fmt = lambda X: "\n".join("%.17g" % v for v in X.ravel())
    inp = f"{m}\n" + fmt(A) + "\n" + fmt(B) + "\n"
    vals = np.array(subprocess.check_output([str(exe)], input=inp, text=True).split(), float)
    prod, prod_adj = vals[:4 * m * m].reshape(4, m, m), vals[4 * m * m:].reshape(4, m, m)
    ref = _spinor(A) @ _spinor(B)
    ref_adj = _spinor(A).conj().T @ _spinor(B)
    assert np.abs(_spinor(prod) - ref).max() < 1e-12
    assert np.abs(_spinor(prod_adj) - ref_adj).max() < 1e-12


def test_s_integrals_binding_rejects_bad_shapes_before_any_launch():
    """x2c_s_integrals takes n from bf_alpha and the nucleus count from nuc_z; arrays of any
    other shape (or on different devices) would be read out of bounds, so the binding refuses
    them before it reaches the library (checked on CPU tensors: shapes come first)."""
    torch = pytest.importorskip("torch")
    import paper_1303_4446_gb300 as x

    f = lambda *s: torch.zeros(*s, dtype=torch.float64)
    good = dict(nuc_xyz=f(2, 3), nuc_z=f(2), bf_xyz=f(5, 3), bf_alpha=f(5))
    bad = [dict(good, bf_xyz=f(4, 3)), dict(good, bf_xyz=f(15)), dict(good, nuc_xyz=f(3, 3)),
           dict(good, nuc_z=f(2, 1)), dict(good, bf_alpha=f(0)), dict(good, bf_alpha=f(0), bf_xyz=f(0, 3))]
    for kw in bad:
        with pytest.raises(ValueError, match="must be"):
            x.x2c_s_integrals(**kw)
    with pytest.raises(ValueError, match="CUDA"):
        x.x2c_s_integrals(**good)  # right shapes, but not on a GPU
    with pytest.raises(ValueError):
        x.x2c_s_integrals(**dict(good, bf_alpha=torch.zeros(5, dtype=torch.float32)))
