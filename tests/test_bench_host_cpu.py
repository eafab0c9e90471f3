"""Host logic of bench.py that needs no GPU: the choice of the roofline kernel and the pair
flop model it uses."""
import pytest

import bench


def test_dominant_kernel_skips_kernels_without_known_work():
    # {name: (ms, launches, library flops)}: the sign-iteration products are the slowest here
    # but report no flops (the device decides how many run), so they cannot carry a roofline
    kt = {"solve_sign_gemm": (9.0, 40, 0.0), "split_stage2": (7.0, 5, 0.0), "splitk_reduce": (8.0, 60, 0.0),
          "solve_quat_gemm": (2.0, 30, 1e9)}
    assert bench.dominant_kernel(kt)[0] == "split_stage2"
    kt = {"solve_sign_gemm": (9.0, 40, 0.0), "solve_quat_gemm": (2.0, 30, 1e9), "gemm_f64": (1.0, 3, 1e8)}
    assert bench.dominant_kernel(kt)[0] == "solve_quat_gemm"
    # nothing with known work: fall back to the slowest
    assert bench.dominant_kernel({"a": (1.0, 1, 0.0), "b": (2.0, 1, 0.0)})[0] == "b"


@pytest.mark.parametrize("n", [30, 48])
def test_pair_flop_model_matches_the_credited_counts(n):
    # stage 1 + stage 2 + same-atom spin-orbit of a two-component pair: 96 n^3 off the diagonal,
    # 120 n^3 on it (the credited counts of the paper's scalar-structure rule)
    off = sum(bench.kernel_flops(k, n, n, 4, False) for k in ("split_stage1", "split_stage2", "split_spin_orbit"))
    diag = sum(bench.kernel_flops(k, n, n, 4, True) for k in ("split_stage1", "split_stage2", "split_spin_orbit"))
    assert off == 96.0 * n ** 3 and diag == 120.0 * n ** 3
    sf = sum(bench.kernel_flops(k, n, n, 1, False) for k in ("dlu_stage1", "dlu_stage2"))
    assert sf == 12.0 * n ** 3
