"""The device integral formulas (integrals_math.cuh, compiled here for the host) against the
workload's closed-form integral generator, which the integral pins of
test_workload_integrals.py hold to finite differences, quadrature and one-centre forms."""
import os
import subprocess

import numpy as np
import pytest

from paper_1303_4446_gb300 import workload as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("sints") / "s_integrals_check"
    subprocess.check_call(["nvcc", "-std=c++17", "-O2", "-o", str(out),
                           os.path.join(ROOT, "tests", "native", "s_integrals_check.cu")])
    return str(out)


def test_host_build_of_device_formulas_matches_generator(exe):
    mol = w.Molecule(np.array([[0.0, 0.0, 0.0], [3.86, 3.86, 0.0], [1.2, -0.7, 2.9]]), np.array([47.0, 47.0, 1.0]),
                     ["s30", "s30", "s30"])
    lines = [str(mol.natoms)]
    lines += ["%.17g %.17g %.17g %.17g" % (*mol.coords[c], mol.Z[c]) for c in range(mol.natoms)]
    lines += [str(mol.nbf)]
    lines += ["%.17g %.17g %.17g %.17g" % (*mol.bf_xyz[i], mol.bf_alpha[i]) for i in range(mol.nbf)]
    res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    got = np.array([[float(v) for v in l.split()] for l in res.stdout.splitlines()]).reshape(mol.nbf, mol.nbf, 4)
    ref = w.integrals(mol)
    for q, k in enumerate(("S", "T", "V", "W0")):
        err = np.abs(got[:, :, q] - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-13, (k, err)
