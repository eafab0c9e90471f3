"""The device integral formulas (integrals_math.cuh, compiled here for the host) against
independent pins (tests/integral_pins.py: closed forms, scipy's incomplete gamma function,
finite differences of the routine's own S and V, quadrature), and, as a consistency check,
against the workload's generator."""
import os
import subprocess

import numpy as np
import pytest

import integral_pins as P
from paper_1303_4446_gb300 import workload as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ints(tmp_path_factory):
    out = tmp_path_factory.mktemp("sints") / "s_integrals_check"
    subprocess.check_call(["nvcc", "-std=c++17", "-O2", "-o", str(out),
                           os.path.join(ROOT, "tests", "native", "s_integrals_check.cu")])

    def run(nuc_xyz, nuc_z, bf_xyz, bf_alpha):
        nuc_xyz, bf_xyz = np.asarray(nuc_xyz, float).reshape(-1, 3), np.asarray(bf_xyz, float).reshape(-1, 3)
        n = len(bf_alpha)
        lines = [str(len(nuc_z))]
        lines += ["%.17g %.17g %.17g %.17g" % (*nuc_xyz[c], nuc_z[c]) for c in range(len(nuc_z))]
        lines += [str(n)]
        lines += ["%.17g %.17g %.17g %.17g" % (*bf_xyz[i], bf_alpha[i]) for i in range(n)]
        res = subprocess.run([str(out)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        got = np.array(res.stdout.split(), dtype=np.float64).reshape(n, n, 4)
        return {k: got[:, :, q].copy() for q, k in enumerate(("S", "T", "V", "W0"))}

    return run


def _mixed():
    return w.Molecule(np.array([[0.0, 0.0, 0.0], [3.86, 3.86, 0.0], [1.2, -0.7, 2.9]]), np.array([47.0, 47.0, 1.0]),
                      ["s30", "s30", "s30"])


def test_one_centre_closed_forms(ints):
    P.check_one_centre(ints)


def test_boys_function_through_V(ints):
    P.check_boys_through_V(ints)


def test_cluster_elementwise_against_closed_forms(ints):
    mol = _mixed()
    P.check_elementwise_V(ints, mol.coords, mol.Z, mol.bf_xyz, mol.bf_alpha)


def test_T_and_W0_are_gradients_of_S_and_V(ints):
    P.check_finite_differences(ints)


def test_W0_elementwise_by_finite_differences(ints):
    # a two-atom cut of the s30 basis (every third exponent) keeps the number of calls small
    mol = w.Molecule(np.array([[0.0, 0.0, 0.0], [2.2, -1.4, 3.1]]), np.array([47.0, 8.0]), ["s30", "s30"])
    keep = np.arange(0, mol.nbf, 3)
    P.check_W0_elementwise_fd(ints, mol.coords, mol.Z, mol.bf_xyz[keep], mol.bf_alpha[keep])


def test_V_by_quadrature(ints):
    P.check_quadrature(ints)


def test_consistent_with_the_workload_generator(ints):
    mol = _mixed()
    got = ints(mol.coords, mol.Z, mol.bf_xyz, mol.bf_alpha)
    ref = w.integrals(mol)
    for k in ("S", "T", "V", "W0"):
        err = np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-13, (k, err)
