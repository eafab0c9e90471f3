"""The device's DKHn operation list (dkh_plan.h, host C++) needs exactly the P(n) matrix
products of Table I ("this work" column) for n = 2..14."""
import json
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plan_products_match_table_I(tmp_path):
    exe = tmp_path / "dkh_plan_check"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-o", str(exe),
                           os.path.join(ROOT, "tests", "native", "dkh_plan_check.cpp")])
    rows = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)], text=True).splitlines()]
    P = json.load(open(os.path.join(ROOT, "tests", "golden", "dkh_mult_counts.json")))["P"]
    assert [r[0] for r in rows] == list(range(2, 15))
    for n, products, ops, hp in rows:
        assert products == P[str(n)] == hp, n
        assert ops >= products
