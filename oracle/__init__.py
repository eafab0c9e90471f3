"""CPU FP64 oracle for the X2C / DLU one-electron Hamiltonian.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or execute anything in this
package.  It shares no code with the CUDA path (``paper_1303_4446_gb300``); both take
their inputs from the seeded workload generator ``paper_1303_4446_gb300.workload``,
which holds none of the decoupling arithmetic.

The X2C oracle (x2c.py) follows the paper's *non-orthogonal* formulation (the definition
of the method), while the CUDA path uses an orthonormalised, GEMM-only formulation; the
paper's appendix proves the two equal.  BSS and DKHn (fw.py) are defined through the
orthonormal kinetic basis and the free-particle transformation, and follow Sec. II.B-C
step by step.
"""
from .x2c import (  # noqa: F401
    C_LIGHT,
    spinor_inputs,
    x2c_full,
    x2c_dlu,
    dlu_from_transforms,
    x2c_dlh,
    x2c_nab,
    picture_change,
    dlu_atomic_transforms,
    dlu_pair_block,
    quaternion_parts,
    from_quaternion,
    dirac_ground_state,
    electronic_eigenvalues,
)
from . import fw  # noqa: F401  BSS and DKHn (Sec. II.B, II.C)
