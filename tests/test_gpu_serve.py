"""GPU tests of the serving layer (x2c_server_*) and of DLU from given atomic transforms.

Every result must be the same alone, in a batch and in the serving mix: the server runs the
same kernels on the same inputs (a request's cached transforms were computed by the same
solve), so the bar against single builds is 1e-13 relative, and the oracle decides one case
of each kind at the parity tolerances (1e-10 FP64, 1e-9 split)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w
from paper_1303_4446_gb300.abi import X2CError

pytestmark = pytest.mark.gpu
SAME_TOL = 1e-13


@pytest.fixture(scope="module")
def ctx():
    c = x.Context(0)
    yield c
    c.close()


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


def rel(a, b):
    scale = max(float(t.abs().max()) for t in b)
    return max(float((p - q).abs().max()) for p, q in zip(a, b)) / scale


KEY = {("s30", False): 11, ("s48", False): 12, ("s30", True): 21, ("s48", True): 22}


def kinds_for(two_c):
    return {b: w.atomic_inputs(47.0, b, two_c) for b in ("s30", "s48")}


def test_dlu_with_transforms_equals_dlu(ctx):
    for two_c in (False, True):
        mol = w.Molecule(w.fcc_sites(3), np.full(3, 47.0), ["s30", "s48", "s30"])
        g = dev(w.molecule_inputs(mol, two_c))
        ks = kinds_for(two_c)
        gk = [dev(ks["s30"]), dev(ks["s48"])]
        idx = [0, 1, 0]
        ref = x.x2c_build_dlu(ctx, g, mol.offsets, idx, gk, two_component=two_c)
        U = x.x2c_atomic_transforms(ctx, gk, two_component=two_c)
        h = x.x2c_build_dlu_with_transforms(ctx, g, mol.offsets, idx, U, [30, 48], two_component=two_c)
        ctx.status()
        assert rel(h, ref) <= SAME_TOL


def _mix():
    """A mixed request set: sizes, bases, sf/2c, FP64/split, one full X2C, host and device
    inputs, and a molecule given as a view into a larger one's matrices (leading dimension)."""
    out = []
    rng = np.random.default_rng(5)
    for i in range(14):
        L = int(rng.integers(2, 8))
        two_c = bool(i % 3 == 0)
        basis = ["s30" if rng.random() < 0.5 else "s48" for _ in range(L)]
        prec = x.PREC_SPLIT_BF16 if i % 4 == 1 else x.PREC_FP64
        host = i % 5 == 2
        out.append(dict(kind="dlu", mol=w.Molecule(w.fcc_sites(L), np.full(L, 47.0), basis), two_c=two_c,
                        prec=prec, host=host))
    out.append(dict(kind="full", mol=w.silver_cluster(2, "s30"), two_c=False, prec=x.PREC_FP64, host=False))
    out.append(dict(kind="full", mol=w.silver_cluster(2, "s30"), two_c=True, prec=x.PREC_FP64, host=True))
    return out


def _single(ctx, r, g, ks_dev):
    mol = r["mol"]
    if r["kind"] == "full":
        return x.x2c_build_full(ctx, g, two_component=r["two_c"])["h"]
    idx = [0 if b == "s30" else 1 for b in mol.basis]
    return x.x2c_build_dlu(ctx, g, mol.offsets, idx, ks_dev[r["two_c"]], two_component=r["two_c"],
                           precision=r["prec"])


def test_serving_mix_same_as_alone(ctx):
    reqs = _mix()
    ks = {tc: kinds_for(tc) for tc in (False, True)}
    ks_dev = {tc: [dev(ks[tc]["s30"]), dev(ks[tc]["s48"])] for tc in (False, True)}
    inputs = [w.molecule_inputs(r["mol"], r["two_c"]) for r in reqs]
    alone = []
    for r, m in zip(reqs, inputs):
        alone.append([t.clone() for t in _single(ctx, r, dev(m), ks_dev)])
    ctx.status()

    # everything the requests read, prepared before the first submission so that requests
    # queue up behind the running ones and form batches
    prepared = []
    for i, (r, m) in enumerate(zip(reqs, inputs)):
        two_c, mol = r["two_c"], r["mol"]
        nc = 4 if two_c else 1
        if r["host"]:
            mm = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in m.items()}
            kk = [{k: torch.from_numpy(v).pin_memory() for k, v in ks[two_c][b].items()} for b in ("s30", "s48")]
            out = [torch.empty((mol.nbf, mol.nbf), dtype=torch.float64).pin_memory() for _ in range(nc)]
        else:
            mm, kk, out = dev(m), ks_dev[two_c], None
        prepared.append((mm, kk, out))
    # one more: a molecule given as the leading block of a larger one's matrices (views with
    # a leading dimension), against a build on a contiguous copy
    big = w.Molecule(w.fcc_sites(5), np.full(5, 47.0), ["s30"] * 5)
    gb = dev(w.molecule_inputs(big, False))
    view = {k: v[:90, :90] for k, v in gb.items()}
    ref_view = x.x2c_build_dlu(ctx, {k: v.contiguous() for k, v in view.items()}, big.offsets[:4], [0, 0, 0],
                               [ks_dev[False][0]])
    ctx.status()

    # a DLH request from host memory: the server must copy all of T and V for it
    dmol = w.silver_cluster(3, "s30")
    dm = w.molecule_inputs(dmol, True)
    ref_dlh = x.x2c_build_dlu(ctx, dev(dm), dmol.offsets, [0] * 3, [ks_dev[True][0]], two_component=True,
                              local_approx=x.LOCAL_DLH)
    ctx.status()
    dm_h = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in dm.items()}
    dk_h = {k: torch.from_numpy(v).pin_memory() for k, v in ks[True]["s30"].items()}
    dlh_out = [torch.empty((dmol.nbf, dmol.nbf), dtype=torch.float64).pin_memory() for _ in range(4)]

    srv = x.Server(0, max_inflight=3, max_batch=4, hbm_budget_bytes=8 << 30)
    try:
        tickets, host_out = [], {}
        for i, (r, (mm, kk, out)) in enumerate(zip(reqs, prepared)):
            two_c, mol = r["two_c"], r["mol"]
            if out is not None:
                host_out[i] = out
            if r["kind"] == "full":
                t = srv.submit_full(mm, two_component=two_c, out=out, host=r["host"])
            else:
                idx = [0 if b == "s30" else 1 for b in mol.basis]
                keys = [KEY[("s30", two_c)], KEY[("s48", two_c)]]
                t = srv.submit_dlu(mm, mol.offsets, idx, kk, kind_keys=keys, two_component=two_c,
                                   precision=r["prec"], out=out, host=r["host"])
            tickets.append(t)
        t_view = srv.submit_dlu(view, big.offsets[:4], [0, 0, 0], [ks_dev[False][0]], kind_keys=[KEY[("s30", False)]])
        t_dlh = srv.submit_dlu(dm_h, dmol.offsets, [0] * 3, [dk_h], kind_keys=[KEY[("s30", True)]], two_component=True,
                               local_approx=x.LOCAL_DLH, out=dlh_out, host=True)
        results = [srv.wait(t) for t in tickets]
        for i, (r, res) in enumerate(zip(reqs, results)):
            assert res["state"] == x.STATE_DONE and res["status"] == 0, (i, res)
            got = host_out[i] if i in host_out else srv.result_tensors(tickets[i], res)
            got = [t.cuda() for t in got]
            assert rel(got, alone[i]) <= SAME_TOL, i
            assert 0 <= res["t_arrival"] <= res["t_admit"] <= res["t_end"]
            assert res["t_start"] <= res["t_end"]
        rv = srv.wait(t_view)
        assert rv["status"] == 0 and rel(srv.result_tensors(t_view, rv), ref_view) <= SAME_TOL
        srv.release(t_view)
        rd = srv.wait(t_dlh)
        assert rd["status"] == 0 and rel([t.cuda() for t in dlh_out], ref_dlh) <= SAME_TOL
        srv.release(t_dlh)
        st = srv.stats()
        assert st["completed"] == len(reqs) + 2 and st["failed"] == 0
        assert st["cache_hits"] > 0 and st["cache_misses"] <= 4
        assert st["peak_bytes"] <= st["budget_bytes"]
        assert max(res["batch_size"] for res in results) > 1
        assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
        for t in tickets:
            srv.release(t)
        assert srv.stats()["bytes_in_use"] < st["peak_bytes"]
    finally:
        srv.close()

    # the oracle decides one spin-free FP64 DLU and the spin-free full X2C case (the split and
    # two-component paths have their own parity tests)
    for i, r in enumerate(reqs):
        if r["kind"] == "dlu" and not r["two_c"] and r["prec"] == x.PREC_FP64:
            break
    mol = reqs[i]["mol"]
    ref = O.x2c_dlu(inputs[i], mol.offsets, [ks[False][b] for b in mol.basis])["h"]
    assert np.abs(alone[i][0].cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    j = len(reqs) - 2
    ref = O.x2c_full(inputs[j])["h"]
    assert np.abs(alone[j][0].cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_serving_errors_and_cancellation():
    two_c = False
    ks = kinds_for(two_c)
    kd = [dev(ks["s30"]), dev(ks["s48"])]
    mol = w.silver_cluster(6, "s48")
    g = dev(w.molecule_inputs(mol, two_c))
    idx = [1] * 6
    keys = [KEY[("s30", False)], KEY[("s48", False)]]

    srv = x.Server(0, max_inflight=1, max_batch=1, hbm_budget_bytes=4 << 30)
    try:
        # invalid request: bad offsets
        with pytest.raises(X2CError) as e:
            srv.submit_dlu(g, np.array([0, 10, 20]), [1, 1], kd, kind_keys=keys)
        assert e.value.code == 1
        # unknown ticket
        with pytest.raises(X2CError) as e:
            srv.release(123456)
        assert e.value.code == 11
        # queue several; the last ones are still queued right after submission
        ts = [srv.submit_dlu(g, mol.offsets, idx, kd, kind_keys=keys) for _ in range(8)]
        with pytest.raises(X2CError) as e:
            srv.wait(ts[-1], timeout_ms=0)
        assert e.value.code == 9
        srv.cancel(ts[-1])
        r = srv.wait(ts[-1])
        assert r["status"] == 10
        for t in ts[:-1]:
            assert srv.wait(t)["status"] == 0
        with pytest.raises(X2CError) as e:
            srv.cancel(ts[0])  # already finished
        assert e.value.code == 1
        # a kind whose S is not positive definite fails its requests only
        bad = dict(ks["s48"])
        bad["S"] = -bad["S"]
        bd = [kd[0], dev(bad)]
        t_bad = srv.submit_dlu(g, mol.offsets, idx, bd, kind_keys=[keys[0], 999])
        t_ok = srv.submit_dlu(g, mol.offsets, idx, kd, kind_keys=keys)
        assert srv.wait(t_bad)["status"] == 4
        assert srv.wait(t_ok)["status"] == 0
        # the failed transforms were not cached: the same key fails again, by its own solve
        t_bad2 = srv.submit_dlu(g, mol.offsets, idx, bd, kind_keys=[keys[0], 999])
        r2 = srv.wait(t_bad2)
        assert r2["status"] == 4 and r2["cache_misses"] == 1
        st = srv.stats()
        assert st["failed"] == 2 and st["cancelled"] == 1
    finally:
        srv.close()


def test_serving_admission_and_eviction():
    two_c = False
    mol = w.silver_cluster(4, "s48")
    m = w.molecule_inputs(mol, two_c)
    g = dev(m)
    ks = kinds_for(two_c)
    kd = dev(ks["s48"])
    # a budget smaller than one request's own memory: refused at submission
    srv = x.Server(0, max_inflight=1, max_batch=1, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(X2CError) as e:
            srv.submit_dlu(g, mol.offsets, [0] * 4, [kd], kind_keys=[5])
        assert e.value.code == 8
    finally:
        srv.close()
    # distinct kind keys with a budget that holds only a few cached transforms: least recently
    # used entries are evicted and every request still completes with the right result
    ctx = x.Context(0)
    ref = x.x2c_build_dlu(ctx, g, mol.offsets, [0] * 4, [kd])
    ctx.status()
    ctx.close()
    # what one request holds at most: workspace, one cached transform, its output
    srv = x.Server(0, max_inflight=1, max_batch=1)
    try:
        t = srv.submit_dlu(g, mol.offsets, [0] * 4, [kd], kind_keys=[99])
        assert srv.wait(t)["status"] == 0
        one = srv.stats()["bytes_in_use"]
    finally:
        srv.close()
    entry = 2 * 48 * 48 * 8  # U^L and U^S of one 48-function kind
    srv = x.Server(0, max_inflight=1, max_batch=1, hbm_budget_bytes=one + 2 * entry)
    try:
        for i in range(10):
            t = srv.submit_dlu(g, mol.offsets, [0] * 4, [kd], kind_keys=[100 + i])
            r = srv.wait(t)
            assert r["status"] == 0 and r["cache_misses"] == 1
            assert rel(srv.result_tensors(t, r), ref) <= SAME_TOL
            srv.release(t)
        st = srv.stats()
        assert st["cache_evictions"] >= 7 and st["cache_entries"] <= 3
        assert st["peak_bytes"] <= st["budget_bytes"]
    finally:
        srv.close()
