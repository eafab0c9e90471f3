"""Host-only checks of the server's scheduling policy (first come, first served batching under
a memory budget, nearest-rank percentiles, least-recently-used eviction), compiled with g++."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_serve_policy(tmp_path):
    exe = tmp_path / "serve_policy_check"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-o", str(exe),
                           os.path.join(ROOT, "tests", "native", "serve_policy_check.cpp")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"
