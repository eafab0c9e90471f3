"""Benchmark: X2C Hamiltonian builds/s of the two-component DLU scheme on Ag309.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ag309_2c] [--precision fp64|split]

One step = one complete DLU build (per-kind atomic decoupling solve + assembly of all
A <= B pair blocks) of the workload, inputs resident in HBM (they are larger than L2, so
no flush is needed).  Prints one JSON line.  Under torchrun every rank builds its own copy
of the workload (independent problems, weak scaling); rank 0 prints.

--impl reference times the CPU oracle (the plain FP64 definition of the method) on a
bounded sample of the same workload: the atomic solve plus a seeded sample of pair blocks,
extrapolated to the full pair list.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1303_4446_gb300 import workload as w  # noqa: E402

METRIC = "X2C h builds/s & FP64-equiv TFLOP/s (Ag309 2c DLU) vs plain FP64; p99 latency"
# FP64 FMA peak: a DFMA throughput probe on this GB300 measured 1.193 TFLOP/s at 1995 MHz,
# i.e. 2 DFMA per clock per SM; at the 2070 MHz maximum SM clock that is
# 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.2586 TFLOP/s.  (FP64 mma.sync measured 1.046.)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per two-component 48 x 48 pair block of the split kernels, from
# one ncu capture of the Ag55 two-component build (1540 pairs, the same per-pair shapes as
# Ag309); a launch's traffic is this times its pairs.  Set an entry to None when its kernel
# changes.
PROFILED_DRAM_BYTES_PER_PAIR = {("split_stage1", "trm"): 238.5e3, ("split_stage2", "nt96"): 302.0e3}
WORKLOADS = {
    "ag309_2c": dict(L=309, basis="s48", two_c=True),
    # 64 uneven spin-free clusters, n ~ U[2, 43], basis s30/s48 50/50, one batched launch
    "batch64_sf": dict(L=None, basis=None, two_c=False, batch=64),
    # 2000 Poisson requests at 50/s through the server: Ag_n, n log-uniform in [2, 147],
    # s30/s48, 30 % two-component; inputs are leading blocks of the Ag147 matrices in pinned
    # host memory (copied in by the server), results stay on the device
    "serving": dict(L=None, basis=None, two_c=None, serving=2000),
    "ag55_2c": dict(L=55, basis="s48", two_c=True),
    "ag55_sf": dict(L=55, basis="s48", two_c=False),
    "ag4_sf": dict(L=4, basis="s30", two_c=False),
    # DLU with the paper-literal atomic potential (molecular diagonal blocks): one decoupling
    # solve per atom, batched over all 309 atoms
    "ag309_2c_mb": dict(L=309, basis="s48", two_c=True, mb=True),
    # full X2C of the whole cluster (blocked factorisation, Newton-Schulz sign function)
    "ag55_sf_full": dict(L=55, basis="s48", two_c=False, full=True),
    "ag55_2c_full": dict(L=55, basis="s48", two_c=True, full=True),
    "ag13_2c_full": dict(L=13, basis="s48", two_c=True, full=True),
    # DLU with DKH2 (Sec. II.C) or BSS (Sec. II.B) atomic transforms instead of X2C ones
    "ag309_2c_dkh2": dict(L=309, basis="s48", two_c=True, decoupling=2),
    "ag309_2c_bss": dict(L=309, basis="s48", two_c=True, decoupling=1),
}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def clock_matched(roof, peaks, clocks):
    """A tensor-bound fraction at equal SM clocks: the measured BF16 peak was taken at the
    median clock of its own run (a seconds-long loop under the power cap), the kernel at the
    clock sampled during the timed region; both rates scale with the SM clock, so
    frac_clock_matched = frac x (peak run's clock / this run's clock)."""
    if roof.get("bound") != "tensor":
        return
    pk = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    run = (clocks or {}).get("sm_mhz")
    if pk and run:
        roof["peak_clock_mhz"] = pk
        roof["run_clock_mhz"] = run
        roof["frac_clock_matched"] = roof["frac"] * pk / run
        roof["clock_note"] = (f"peak measured at a median {pk:g} MHz, kernel timed at {run:g} MHz; "
                              "frac_clock_matched compares the two at the same clock")


def pair_list(L):
    return [(a, b) for a in range(L) for b in range(a, L)]


MODEL_KERNELS = ("dlu_stage1", "split_stage1", "dlu_stage2", "split_stage2", "dlu_spin_orbit", "split_spin_orbit",
                 "split_slice_mid")


def dominant_kernel(ktimes):
    """The kernel with the largest total time among those whose work is known: a pair-assembly
    kernel of the model below, or one the library reports flops for (the decoupling-solve
    products whose count the device decides, the split-K reductions and the small helpers
    report none)."""
    known = {k: v for k, v in ktimes.items() if k in MODEL_KERNELS or v[2] > 0}
    return max((known or ktimes).items(), key=lambda kv: kv[1][0])


def kernel_flops(name, nA, nB, nc, diag):
    """Algorithmic FP64-equivalent flops of one pair block in each assembly kernel (the
    split kernels compute the same products, as digit-slice products on the tensor cores)."""
    if name in ("dlu_stage1", "split_stage1"):
        return 8.0 * nc * nA * nB * nB
    if name in ("dlu_stage2", "split_stage2"):
        return 4.0 * nc * nc * nA * nA * nB
    if name in ("dlu_spin_orbit", "split_spin_orbit"):
        return 24.0 * nA * nB * nB if diag else 0.0
    return 0.0


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_inputs(cfg, seed=w.DEFAULT_SEED):
    if cfg.get("batch"):
        mols = w.batched_molecules(count=cfg["batch"], lo=2, hi=43, seed=seed)
        ms = [w.molecule_inputs(m, False, seed) for m in mols]
        kinds = {b: w.atomic_inputs(47.0, b, False, seed) for b in ("s30", "s48")}
        return mols, ms, kinds
    mol = w.silver_cluster(cfg["L"], cfg["basis"])
    m = w.molecule_inputs(mol, cfg["two_c"], seed)
    kind = w.atomic_inputs(47.0, cfg["basis"], cfg["two_c"], seed)
    return mol, m, kind


def cpu_oracle_rate(mol, m, kind, two_c, budget_s, seed=1, solves=1, decoupling=0):
    """Oracle builds/s from the atomic solve (times `solves` per build) plus a timed seeded
    sample of pair blocks, extrapolated to all pair blocks.  Returns (builds/s,
    n_sampled_pairs, seconds)."""
    import oracle
    from oracle import fw

    t0 = time.perf_counter()
    if decoupling == 0:
        r = oracle.x2c_full(kind)
    elif decoupling == 1:
        r = fw.bss_full(kind)
    else:
        r = fw.dkh_transforms(kind, decoupling)
    t_atom = (time.perf_counter() - t0) * solves
    UL, US = r["UL"], r["US"]
    pairs = pair_list(mol.natoms)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(pairs))
    keys = ("V", "T", "W0") + (("Wx", "Wy", "Wz") if two_c else ())
    t_pairs, n = 0.0, 0
    for idx in order:
        A, B = pairs[idx]
        ra = slice(mol.offsets[A], mol.offsets[A + 1])
        rb = slice(mol.offsets[B], mol.offsets[B + 1])
        blocks = {k: m[k][ra, rb] for k in keys}
        t0 = time.perf_counter()
        oracle.dlu_pair_block(blocks, UL, US, UL, US)
        t_pairs += time.perf_counter() - t0
        n += 1
        if t_pairs + t_atom > budget_s and n >= 8:
            break
    per_build = t_atom + t_pairs / n * len(pairs)
    return 1.0 / per_build, n, t_atom + t_pairs


def run_reference(args, cfg):
    """CPU oracle arm: each step times the atomic solve and a bounded pair-block sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mol = w.silver_cluster(cfg["L"], cfg["basis"])
    kind = w.atomic_inputs(47.0, cfg["basis"], cfg["two_c"])
    pairs = pair_list(mol.natoms)
    rng = np.random.default_rng(7)
    # pair blocks for the samples are generated on demand (input generation, not timed)
    so = w.so_blocks(47.0, cfg["basis"]) if cfg["two_c"] else None

    def block(A, B):
        ra = slice(int(mol.offsets[A]), int(mol.offsets[A + 1]))
        rb = slice(int(mol.offsets[B]), int(mol.offsets[B + 1]))
        b = w.integrals_block(mol, ra, rb, want=("T", "V", "W0"))
        if cfg["two_c"]:
            for k, name in enumerate(("Wx", "Wy", "Wz")):
                b[name] = so[k].copy() if A == B else np.zeros_like(b["T"])
        return b

    import oracle
    per_step = 64
    rates = []
    for step in range(args.warmup + args.steps):
        sample = [pairs[i] for i in rng.choice(len(pairs), per_step, replace=False)]
        blocks = [block(A, B) for A, B in sample]
        t0 = time.perf_counter()
        r = oracle.x2c_full(kind)
        t_atom = time.perf_counter() - t0
        t0 = time.perf_counter()
        for b in blocks:
            oracle.dlu_pair_block(b, r["UL"], r["US"], r["UL"], r["US"])
        t_p = time.perf_counter() - t0
        if step >= args.warmup:
            rates.append(1.0 / (t_atom + t_p / per_step * len(pairs)))
    v = float(np.mean(rates))
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "builds/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Ag{cfg['L']} {'two-component' if cfg['two_c'] else 'spin-free'} DLU, "
                                   f"{cfg['basis']} primitives per atom, N={mol.nbf}",
                       "pairs": len(pairs)},
            "cpu_baseline": {"value": v, "unit": "builds/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step: atomic solve + {per_step} seeded pair blocks, "
                                       f"extrapolated to {len(pairs)} pair blocks"},
            "e2e": {"value": v, "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, cfg):
    """64 uneven molecules per step through one x2c_build_dlu_batched launch."""
    import torch
    import paper_1303_4446_gb300 as x

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    mols, ms, kinds = make_inputs(cfg)
    t_gen = time.perf_counter() - t_gen
    order = ["s30", "s48"]
    gk = [{k: torch.from_numpy(v).to(dev) for k, v in kinds[b].items()} for b in order]
    gs = [{k: torch.from_numpy(v).to(dev) for k, v in m.items()} for m in ms]
    lays = [(m.offsets, [order.index(b) for b in m.basis], gk) for m in mols]
    outs = [[torch.empty((m.nbf, m.nbf), dtype=torch.float64, device=dev)] for m in mols]
    ctx = x.Context(local)
    ctx.set_graphs(bool(args.graphs))
    prec = x.PREC_SPLIT_BF16 if args.precision == "split" else x.PREC_FP64
    stream = torch.cuda.current_stream(dev)

    def build():
        x.x2c_build_dlu_batched(ctx, gs, lays, precision=prec, n_slices=args.slices, outs=outs, stream=stream)

    # with graphs the warm-up's second build captures the step the timed region replays
    for _ in range(args.warmup):
        build()
    ctx.status(stream)
    counters = ctx.counters()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            build()
        ev1.record(stream)
        torch.cuda.synchronize()
    ctx.status(stream)
    ms_step = ev0.elapsed_time(ev1) / args.steps
    ktimes = kernel_pass(ctx, build, args.steps, stream)
    credited = counters["credited_flops"]
    n_mol = len(mols)
    dom_name, (dom_ms, dom_l, lib_flops) = dominant_kernel(ktimes)
    dom_flops = 0.0
    for m in mols:
        sz = np.diff(m.offsets)
        dom_flops += sum(kernel_flops(dom_name, sz[a], sz[b], 1, a == b) for a, b in pair_list(m.natoms))
    dom_flops *= args.steps
    peaks = measured_peaks()
    if args.precision == "split" and dom_name.startswith("split_stage"):
        S = args.slices or 5
        roof = {"bound": "tensor", "achieved": dom_flops * S * (S + 1) / 2 / (dom_ms * 1e-3) / 1e12,
                "peak": peaks.get("bf16_tflops_sustained", 1730.2), "unit": "TFLOP/s",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured"}
    else:
        # FP64 kernels: pair-assembly flop model, or the flops the library counts per launch
        # (2 m n k per GEMM product; the per-kind decoupling solve GEMMs)
        fl = dom_flops if dom_flops > 0 else lib_flops
        roof = {"bound": "alu", "achieved": fl / (dom_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "152 SMs x 2 DFMA/clk x 2.07 GHz"}
    roof.update(kernel=dom_name, frac=roof["achieved"] / roof["peak"], traffic=None, launches=int(dom_l))
    clk_sum = clk.summary()
    clock_matched(roof, peaks, clk_sum)
    npairs = sum(len(pair_list(m.natoms)) for m in mols)
    line = {"metric": METRIC, "value": n_mol * 1e3 / ms_step, "unit": "builds/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16x-split",
            "data": "synthetic",
            "config": {"workload": f"{n_mol} spin-free Ag_n DLU builds per launch, n ~ U[2,43], s30/s48",
                       "sizes": [m.natoms for m in mols], "pairs": npairs, "precision": args.precision,
                       "inputs": "resident, 1.6 GB total (L2 flushed by the size of the step)"},
            "fp64_equiv_tflops": credited / (ms_step * 1e-3) / 1e12, "credited_flops_per_step": credited,
            "gpu_launches": int(counters["kernel_launches"]) * args.steps, "roofline": roof,
            "clocks": clk_sum,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in sorted(ktimes.items(), key=lambda kv: -kv[1][0])},
            "kernel_launches_per_step": {k: v[1] // args.steps for k, v in ktimes.items()},
            "graphs": ctx.graph_stats(), "kernel_timing": KERNEL_TIMING, "input_generation_s": t_gen}
    if not args.no_e2e:
        pin = [{k: torch.from_numpy(v).pin_memory() for k, v in m.items()} for m in ms]
        hpin = [torch.empty((m.nbf, m.nbf), dtype=torch.float64).pin_memory() for m in mols]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for g, p_ in zip(gs, pin):
                for k in g:
                    g[k].copy_(p_[k], non_blocking=True)
            build()
            for o, hp in zip(outs, hpin):
                hp.copy_(o[0], non_blocking=True)
            torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / args.e2e_steps
        h2d = sum(8 * len(m) * mol.nbf ** 2 for m, mol in zip(ms, mols))
        d2h = sum(8 * mol.nbf ** 2 for mol in mols)
        line["e2e"] = {"value": n_mol / t_e2e, "unit": "builds/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                       "path": "pinned H2D of every molecule's S, T, V, W0 + x2c_build_dlu_batched + D2H of h"}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        done = 0
        for m, mol in zip(ms, mols):
            oracle.x2c_dlu(m, mol.offsets, [kinds[b] for b in mol.basis])
            done += 1
            if time.perf_counter() - t0 > args.cpu_budget:
                break
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "builds/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"dense oracle DLU of the first {done} of {n_mol} molecules ({dt:.1f} s)"}
    ctx.close()
    print(json.dumps(line), flush=True)


KERNEL_TIMING = ("kernel_ms_per_step and the roofline's launch times: a second pass of the same steps with "
                 "a CUDA event pair around every launch; value: the timed region without them")


def kernel_pass(ctx, build, steps, stream):
    """Per-kernel device times of `steps` more builds, each launch bracketed by CUDA events on
    its own stream: {name: (ms, launches, library flops)}.  Run after the timed region, which
    has no per-launch events (on small builds they cost up to a third of the step)."""
    ctx.set_timing(True)
    for _ in range(2):  # with graphs: an eager build, then the capture of the instrumented step
        build()
    ctx.status(stream)
    ctx.set_timing(True)  # drops those two builds' times
    for _ in range(steps):
        build()
    ctx.status(stream)
    kt = ctx.kernel_times(with_flops=True)
    ctx.set_timing(False)
    return kt


def max_over_ranks(value, dist=None, device="cpu"):
    """The maximum of a per-rank value over all ranks (each step is timed on every rank and
    the slowest rank counts); the value itself on one process."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, seconds_per_step):
    """Whole-job builds/s: every rank completes one independent build per step."""
    return world / seconds_per_step


def pct(v, p):
    """Nearest-rank percentile (None for no samples)."""
    if not v:
        return None
    v = sorted(v)
    k = max(0, min(len(v) - 1, int(np.ceil(p / 100.0 * len(v))) - 1))
    return v[k]


def serving_inputs(seed=w.DEFAULT_SEED):
    """Pinned host matrices of Ag147 per basis (two-component set; spin-free requests use S,
    T, V, W0) and the free-atom kinds, host and device."""
    import torch
    big, kinds = {}, {}
    for b in ("s30", "s48"):
        mol = w.silver_cluster(147, b)
        m = w.molecule_inputs(mol, True, seed)
        big[b] = {k: torch.from_numpy(v).pin_memory() for k, v in m.items()}
        for tc in (False, True):
            kinds[(b, tc)] = {k: torch.from_numpy(v).pin_memory()
                              for k, v in w.atomic_inputs(47.0, b, tc, seed).items()}
    return big, kinds


def serve_stream(srv, reqs, big, kinds, precision, n_slices, t_lead=0.05):
    """Open-loop submission at the scheduled arrival times (server clock) of every request;
    latency is counted from the scheduled arrival.  Results are released as they complete."""
    import threading
    import paper_1303_4446_gb300 as x
    keys = {(b, tc): 1 + 2 * ("s30", "s48").index(b) + int(tc) for b in ("s30", "s48") for tc in (False, True)}
    pending = []
    lock = threading.Condition()
    done = {"n": 0, "failed": 0, "wait_ms": [], "service_ms": [], "slowest": []}
    meta = {}
    h2d = [0]

    def reaper():
        # waits for the requests in submission order and releases their results
        while True:
            with lock:
                while not pending and not done.get("stop"):
                    lock.wait(0.05)
                if not pending:
                    return
                t = pending.pop(0)
            r = srv.wait(t, timeout_ms=600000)
            if r["status"] != 0:
                done["failed"] += 1
            else:
                done["wait_ms"].append((r["t_start"] - r["t_arrival"]) * 1e3)
                done["service_ms"].append((r["t_end"] - r["t_start"]) * 1e3)
                done["slowest"].append(((r["t_end"] - r["t_start"]) * 1e3, meta.get(t)))
            srv.release(t)
            done["n"] += 1

    th = threading.Thread(target=reaper, daemon=True)
    th.start()
    t0 = srv.now() + t_lead
    for rq in reqs:
        b, tc, L = rq["basis"], rq["two_component"], rq["natoms"]
        nb = w.BASES[b][2]
        N = L * nb
        m = {k: v[:N, :N] for k, v in big[b].items() if tc or k in ("S", "T", "V", "W0")}
        target = t0 + rq["t_arrive"]
        while True:
            dt = target - srv.now()
            if dt <= 0:
                break
            time.sleep(dt - 0.0005 if dt > 0.001 else 0)
        offs = np.arange(L + 1, dtype=np.int32) * nb
        t = srv.submit_dlu(m, offs, [0] * L, [kinds[(b, tc)]], kind_keys=[keys[(b, tc)]], two_component=tc,
                           precision=precision, n_slices=n_slices, host=True, t_arrival=target)
        # what the server copies: the upper block triangle of T, V, W0 (pairs A <= B) and the
        # same-atom blocks of Wx, Wy, Wz
        h2d[0] += 8 * nb * nb * (3 * L * (L + 1) // 2 + (3 * L if tc else 0))
        meta[t] = f"Ag{L} {b} {'2c' if tc else 'sf'}"
        with lock:
            pending.append(t)
            lock.notify()
    with lock:
        done["stop"] = True
        lock.notify()
    th.join()
    return done, h2d[0]


def run_full(args, cfg):
    """Full X2C of a whole cluster (x2c_build_full), with the oracle's full build timed beside it."""
    import torch
    import paper_1303_4446_gb300 as x

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    mol = w.silver_cluster(cfg["L"], cfg["basis"])
    two_c = cfg["two_c"]
    m = w.molecule_inputs(mol, two_c)
    t_gen = time.perf_counter() - t_gen
    g = {k: torch.from_numpy(v).to(dev) for k, v in m.items()}
    ctx = x.Context(local)
    stream = torch.cuda.current_stream(dev)
    warm, steps = max(1, args.warmup), max(1, args.steps)
    for _ in range(warm):
        out = x.x2c_build_full(ctx, g, two_component=two_c, stream=stream)
    ctx.status(stream)
    counters = ctx.counters()
    ctx.set_timing(True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            out = x.x2c_build_full(ctx, g, two_component=two_c, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    ctx.status(stream)
    ms = ev0.elapsed_time(ev1) / steps
    kt = ctx.kernel_times(with_flops=True)
    ctx.set_timing(False)
    dom_name, (dom_ms, dom_l, dom_fl) = dominant_kernel(kt)
    roof = {"bound": "alu", "achieved": dom_fl / (dom_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "kernel": dom_name, "frac": dom_fl / (dom_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
            "launches": int(dom_l), "peak_source": "152 SMs x 2 DFMA/clk x 2.07 GHz",
            "flops": "2 m n k per real product the kernel computes (upper triangles of Hermitian products)"}
    line = {"metric": METRIC, "value": world * 1e3 / ms, "unit": "builds/s", "n_gpus": world, "steps": steps,
            "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"full X2C of Ag{cfg['L']} {'two-component' if two_c else 'spin-free'}, "
                                   f"{cfg['basis']} primitives per atom, N={mol.nbf}",
                       "inputs": "resident", "parallelism": f"independent replicas x{world}"},
            "fp64_equiv_tflops": world * counters["credited_flops"] / (ms * 1e-3) / 1e12,
            "credited_flops_per_build": counters["credited_flops"],
            "gpu_launches": int(counters["kernel_launches"]) * steps, "roofline": roof, "clocks": clk.summary(),
            "kernel_ms_per_step": {k: v[0] / steps for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])[:10]},
            "input_generation_s": t_gen}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        r = oracle.x2c_full(m)
        dt = time.perf_counter() - t0
        ref = list(oracle.quaternion_parts(r["h"])) if two_c else [r["h"]]
        err = max(float(np.abs(a.cpu().numpy() - b).max()) for a, b in zip(out["h"], ref)) / float(np.abs(r["h"]).max())
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "builds/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"one whole oracle build ({dt:.1f} s)"}
        line["max_abs_err_rel_to_max_h"] = err
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serving(args, cfg):
    """The serving workload: continuous batching of a Poisson request stream (x2c_server_*)."""
    import torch
    import paper_1303_4446_gb300 as x

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    big, kinds = serving_inputs()
    reqs = w.serving_requests(count=args.requests or cfg["serving"], rate=args.rate, seed=w.DEFAULT_SEED + rank)
    t_gen = time.perf_counter() - t_gen
    prec = x.PREC_SPLIT_BF16 if args.precision == "split" else x.PREC_FP64
    srv = x.Server(local, max_inflight=args.slots, max_batch=16, hbm_budget_bytes=150 * 10 ** 9)
    # warm-up: a few requests of every (basis, spin) kind through the server (the transforms
    # cache fills, the slots' workspaces grow), then the statistics are cleared
    combos = [(n, b, tc) for n in (147, 24, 5) for b in ("s30", "s48") for tc in (False, True)]
    warm = [dict(t_arrive=0.002 * i, natoms=n, basis=b, two_component=tc) for i, (n, b, tc) in enumerate(combos)]
    serve_stream(srv, warm, big, kinds, prec, args.slices)
    srv.reset_stats()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        done, h2d = serve_stream(srv, reqs, big, kinds, prec, args.slices)
    st = srv.stats()
    srv.close()
    n_ok = st["completed"]
    line = {"metric": METRIC, "value": world * st["builds_per_s"], "unit": "builds/s", "n_gpus": world,
            "steps": len(reqs), "warmup": len(warm), "ms_per_step": 1e3 / st["builds_per_s"] if st["builds_per_s"] else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "bf16x-split", "data": "synthetic",
            "config": {"workload": f"serving: {len(reqs)} Poisson requests at {args.rate:g}/s, Ag_n DLU, n log-uniform "
                                   "in [2,147], s30/s48, 30% two-component, 150 GB budget",
                       "slots": args.slots, "max_batch": 16, "precision": args.precision,
                       "inputs": "leading n x n blocks of the Ag147 matrices, pinned host memory, "
                                 "copied in by the server; results stay on the device",
                       "parallelism": f"independent replicas x{world}"},
            "serving": {"p50_ms": st["latency_p50_ms"], "p99_ms": st["latency_p99_ms"],
                        "mean_ms": st["latency_mean_ms"], "max_ms": st["latency_max_ms"],
                        "completed": n_ok, "failed": st["failed"], "builds_launched": st["builds_launched"],
                        "cache_hits": st["cache_hits"], "cache_misses": st["cache_misses"],
                        "peak_bytes": st["peak_bytes"], "max_concurrent": st["max_concurrent"],
                        "latency": "completion (device event) - scheduled arrival",
                        "wait_p50_ms": pct(done["wait_ms"], 50), "wait_p99_ms": pct(done["wait_ms"], 99),
                        "service_p50_ms": pct(done["service_ms"], 50), "service_p99_ms": pct(done["service_ms"], 99),
                        "slowest_service": [[round(v, 2), k] for v, k in sorted(done["slowest"], key=lambda x: -x[0])[:8]],
                        "split": "wait = device start - scheduled arrival (submission, admission, queueing); "
                                 "service = device start to completion (input copies + build)"},
            "gpu_launches": int(st["kernel_launches"]), "roofline": None,
            "roofline_note": "latency-bound request stream; kernel rooflines are on the Ag309 line",
            "clocks": clk.summary(), "input_generation_s": t_gen,
            "e2e": {"value": world * st["builds_per_s"], "unit": "builds/s",
                    "h2d_bytes_per_step": int(h2d / max(1, len(reqs))), "d2h_bytes_per_step": 0,
                    "path": "x2c_server_submit with pinned host inputs (H2D inside each request)"}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        cnt = 0
        for rq in reqs:
            b, tc, L = rq["basis"], rq["two_component"], rq["natoms"]
            if L > 40:
                continue  # the dense oracle of the largest requests alone takes minutes
            nb = w.BASES[b][2]
            N = L * nb
            m = {k: v[:N, :N].numpy().copy() for k, v in big[b].items() if tc or k in ("S", "T", "V", "W0")}
            kd = {k: v.numpy() for k, v in kinds[(b, tc)].items()}
            oracle.x2c_dlu(m, np.arange(L + 1) * nb, [kd] * L)
            cnt += 1
            if time.perf_counter() - t0 > args.cpu_budget:
                break
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": cnt / dt, "unit": "builds/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"dense oracle DLU of the first {cnt} requests of the stream with n <= 40 atoms "
                                          f"({dt:.1f} s; larger requests are skipped, so this favours the oracle)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ag309_2c", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="split", choices=["fp64", "split"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="split runs: also time this many plain FP64 builds and compare h")
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay the build step from a captured CUDA graph (1) or enqueue it eagerly (0)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=0, help="serving: requests in the stream (0 = 2000)")
    ap.add_argument("--rate", type=float, default=50.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent builds")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "pairs"],
                    help="N > 1: every rank builds the whole molecule (replicas, weak scaling) or the ranks "
                         "split one build's pair list (pairs, strong scaling)")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="default workload: requests of the short serving run reported as 'serving' (0 = none)")
    args = ap.parse_args()
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, cfg)
    if cfg.get("batch"):
        return run_batched(args, cfg)
    if cfg.get("serving"):
        return run_serving(args, cfg)
    if cfg.get("full"):
        return run_full(args, cfg)
    if cfg.get("mb"):
        # one transform per atom: the split assembly shares operands per atom kind, so the
        # molecular-block mode runs on the FP64 path
        args.precision, args.fp64_steps = "fp64", 0

    import torch
    import paper_1303_4446_gb300 as x

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    t_gen = time.perf_counter()
    mol, m, kind = make_inputs(cfg)
    t_gen = time.perf_counter() - t_gen
    two_c = cfg["two_c"]
    nc = 4 if two_c else 1
    dev = torch.device("cuda", local)
    g = {k: torch.from_numpy(v).to(dev) for k, v in m.items()}
    gk = {k: torch.from_numpy(v).to(dev) for k, v in kind.items()}
    N = mol.nbf
    out = [torch.empty((N, N), dtype=torch.float64, device=dev) for _ in range(nc)]
    ctx = x.Context(local)
    ctx.set_graphs(bool(args.graphs))
    prec = x.PREC_SPLIT_BF16 if args.precision == "split" else x.PREC_FP64
    stream = torch.cuda.current_stream(dev)
    kinds = [0] * mol.natoms
    dlu_pot = x.DLU_MOLECULAR_BLOCK if cfg.get("mb") else x.DLU_FREE_ATOM

    dec = cfg.get("decoupling", 0)
    # --shard pairs (N > 1): the ranks split one build's pair list (x2c_dlu_partition) and each
    # assembles its row atoms' blocks; otherwise every rank builds the whole molecule
    shard = world > 1 and args.shard == "pairs"
    rows = x.x2c_dlu_partition(mol.offsets, rank, world) if shard else (0, mol.natoms)

    def build():
        if shard:
            if rows[1] > rows[0]:
                x.x2c_build_dlu_rows(ctx, g, mol.offsets, kinds, [gk], rows[0], rows[1], two_component=two_c,
                                     precision=prec, dlu_potential=dlu_pot, n_slices=args.slices, out=out,
                                     stream=stream, decoupling=dec)
            return
        x.x2c_build_dlu(ctx, g, mol.offsets, kinds, [gk], two_component=two_c, precision=prec, dlu_potential=dlu_pot,
                        n_slices=args.slices, out=out, stream=stream, decoupling=dec)

    # with graphs the warm-up's second build captures the step the timed region replays
    for _ in range(args.warmup):
        build()
    ctx.status(stream)
    counters = ctx.counters()
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            build()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ctx.status(stream)
    ms = ev0.elapsed_time(ev1) / args.steps
    ktimes = kernel_pass(ctx, build, args.steps, stream)
    ms_max = max_over_ranks(ms, dist, dev)
    clocks = clk.summary()
    credited = counters["credited_flops"]
    # roofline of the dominant kernel (largest total time in the timed region)
    dom_name, (dom_ms, dom_launches, dom_lib_flops) = dominant_kernel(ktimes)
    pairs = pair_list(mol.natoms)
    sizes = np.diff(mol.offsets)
    dom_flops = sum(kernel_flops(dom_name, sizes[a], sizes[b], nc, a == b) for a, b in pairs) * args.steps
    peaks = measured_peaks()
    S_sl = args.slices or 5
    if dom_name in ("split_slice_r", "split_slice_mid"):
        # memory-bound digit slicers: algorithmic bytes read + written per pair block
        KPb = lambda n: (2 * n + 31) // 32 * 32
        def slice_bytes(nA, nB):
            if dom_name == "split_slice_mid":
                return 3 * nA * nB * 8 + 2 * nA * KPb(nB) * S_sl * 2
            return nc * nB * 2 * nA * 8 + nc * nB * KPb(nA) * S_sl * 2
        byt = sum(slice_bytes(sizes[a], sizes[b]) for a, b in pairs) * args.steps
        hbm = peaks.get("hbm_gbs", 6684.8)
        roof = {"bound": "hbm", "achieved": byt / (dom_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "kernel": dom_name, "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"}
    elif args.precision == "fp64" or not dom_name.startswith("split_"):
        # FP64 kernels: the pair-assembly flop model, or the flops the library counts for
        # each FP64 GEMM launch (the decoupling solves)
        fl = dom_flops if dom_flops > 0 else dom_lib_flops
        roof = {"bound": "alu", "achieved": fl / (dom_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "kernel": dom_name,
                "peak_source": "152 SMs x 2 DFMA/clk (measured DFMA rate) x 2.07 GHz max clock"}
    else:
        # tensor-core work of the split kernels: S(S+1)/2 BF16 digit products per FP64 product
        S = args.slices or 5
        bf16_flops = dom_flops * S * (S + 1) / 2
        roof = {"bound": "tensor", "achieved": bf16_flops / (dom_ms * 1e-3) / 1e12,
                "peak": peaks.get("bf16_tflops_sustained", 1730.2), "unit": "TFLOP/s", "kernel": dom_name,
                "fp64_equiv_achieved": dom_flops / (dom_ms * 1e-3) / 1e12,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    clock_matched(roof, peaks, clocks)
    log = ctx.tuning_log()
    variant = {"split_stage1": "trm" if "-> transposed" in log else ("nt96" if "-> NT 96" in log else None),
               "split_stage2": "nt96" if ("-> transposed" in log or "-> NT 96" in log) else None}.get(dom_name)
    per_pair = PROFILED_DRAM_BYTES_PER_PAIR.get((dom_name, variant)) if two_c and cfg["basis"] == "s48" else None
    # per launch, like `achieved`: the pairs of all timed launches over their count
    roof["traffic"] = per_pair * len(pairs) * args.steps / dom_launches if per_pair else None
    if per_pair:
        roof["traffic_source"] = "ncu dram__bytes_read+write of the Ag55 2c capture, per pair x pairs per launch"
    roof["launches"] = int(dom_launches)
    roof["avg_launch_ms"] = dom_ms / max(1, dom_launches)

    if shard:  # one build is the union of the ranks' shares: whole-job work of one build
        tot = torch.tensor([credited], dtype=torch.float64, device=dev)
        dist.all_reduce(tot)
        credited = float(tot.item())
    line = {"metric": METRIC, "value": job_rate(1 if shard else world, ms_max * 1e-3), "unit": "builds/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "strong" if shard else "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "bf16x-split",
            "data": "synthetic",
            "config": {"workload": f"Ag{cfg['L']} {'two-component' if two_c else 'spin-free'} "
                                   f"{({0: '', 1: 'BSS-'}.get(dec, f'DKH{dec}-'))}DLU "
                                   f"({'molecular-block U per atom' if cfg.get('mb') else 'free-atom U per kind'}), "
                                   f"{cfg['basis']} primitives per atom, N={N}",
                       "pairs": len(pairs), "precision": args.precision, "inputs": "larger than L2 (no flush)",
                       "parallelism": (f"pair-list partition x{world} (rows {rows[0]}..{rows[1]} on rank {rank})"
                                       if shard else f"independent replicas x{world}")},
            "fp64_equiv_tflops": (1 if shard else world) * credited / (ms_max * 1e-3) / 1e12,
            "credited_flops_per_build": credited,
            "gpu_launches": int(counters["kernel_launches"]) * args.steps,
            "roofline": roof, "clocks": clocks,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in sorted(ktimes.items(), key=lambda kv: -kv[1][0])},
            "autotune": ctx.tuning_log().strip().splitlines(),
            "graphs": ctx.graph_stats(), "kernel_timing": KERNEL_TIMING, "input_generation_s": t_gen}

    if args.precision == "split" and args.fp64_steps > 0:
        # the plain FP64 path on the same inputs: its rate, and the split path's error in h
        # on every element against it (FP64 path parity: tests/test_gpu_parity.py)
        h_split = [t.clone() for t in out]
        prec64 = x.PREC_FP64

        def build64():
            x.x2c_build_dlu(ctx, g, mol.offsets, kinds, [gk], two_component=two_c, precision=prec64, dlu_potential=dlu_pot,
                            out=out, stream=stream, decoupling=dec)

        build64()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            build64()
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.status(stream)
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        scale = max(t.abs().max().item() for t in out)
        err = max((a - b).abs().max().item() for a, b in zip(h_split, out)) / scale
        line["fp64_path"] = {"value": 1e3 / ms64, "unit": "builds/s", "ms_per_step": ms64,
                             "fp64_equiv_tflops": credited / (ms64 * 1e-3) / 1e12, "steps": args.fp64_steps}
        line["speedup_vs_fp64_path"] = ms64 / ms_max
        line["split_max_abs_err_rel_to_max_h"] = err
        line["split_slices"] = args.slices or 5
        del h_split

    if not args.no_e2e:
        # end to end through the host-buffer entry point: H2D of the inputs the method reads,
        # build, D2H of h, every step, from pinned host memory
        pin = {k: torch.from_numpy(v).pin_memory() for k, v in m.items()}
        pink = {k: torch.from_numpy(v).pin_memory() for k, v in kind.items()}
        hout = [torch.empty((N, N), dtype=torch.float64).pin_memory() for _ in range(nc)]
        # h comes back as the upper block triangle of each part (h0 symmetric, h1..h3
        # antisymmetric: the rest follows); free-atom builds run as a copy/compute pipeline
        e2e_args = dict(two_component=two_c, precision=prec, n_slices=args.slices, out=hout, stream=stream,
                        dlu_potential=dlu_pot, h_upper_only=True, decoupling=dec)
        # two warm calls: the first runs eagerly (and tunes), the second captures the chunk
        # plans' CUDA graphs, every later call replays them
        for _ in range(2):
            x.x2c_build_dlu_host(ctx, pin, mol.offsets, kinds, [pink], **e2e_args)
        torch.cuda.synchronize()
        barrier()
        t_calls = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            x.x2c_build_dlu_host(ctx, pin, mol.offsets, kinds, [pink], **e2e_args)
            t_calls.append(time.perf_counter() - t0)
        t_e2e = sum(t_calls) / len(t_calls)  # the mean (an occasional slow call counts in full)
        t_e2e_max = max_over_ranks(t_e2e, dist, dev)
        sz = np.diff(mol.offsets)
        # what x2c_build_dlu_host copies: the upper block triangle of T, V, W0, the same-atom
        # blocks of Wx..Wz (and of S in molecular-block mode), the kind matrices
        upper = int((sz * (N - np.asarray(mol.offsets[:-1]))).sum())
        diag = int((sz * sz).sum())
        kinds_h2d = 0 if cfg.get("mb") else (3 + (4 if two_c else 1)) * len(kind["S"]) ** 2
        h2d = 8 * (3 * upper + (3 * diag if two_c else 0) + (diag if cfg.get("mb") else 0) + kinds_h2d)
        line["e2e"] = {"value": job_rate(world, t_e2e_max), "unit": "builds/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(8 * nc * upper), "steps": args.e2e_steps,
                       "call_ms": [round(1e3 * t, 2) for t in t_calls],
                       "median_call_ms": round(1e3 * statistics.median(t_calls), 2),
                       "path": "x2c_build_dlu_host from pinned host buffers (h_upper_only: the upper block "
                               "triangle of every h part comes back)"}
        del pin, hout

    if rank == 0 and not args.no_cpu_baseline:
        v, n, secs = cpu_oracle_rate(mol, m, kind, two_c, args.cpu_budget, solves=mol.natoms if cfg.get("mb") else 1,
                                     decoupling=dec)
        line["cpu_baseline"] = {"value": v, "unit": "builds/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"atomic solve + {n} seeded pair blocks ({secs:.1f} s), "
                                          f"extrapolated to {len(pairs)} pair blocks"}
    ctx.close()
    if args.serving_requests > 0:
        # p99 latency of the metric: the configured serving stream (2000 Poisson requests at
        # 50/s) on the same GPU; `--workload serving` runs it alone with more detail
        del g, out
        torch.cuda.empty_cache()
        big, kinds_s = serving_inputs()
        reqs = w.serving_requests(count=args.serving_requests, rate=args.rate, seed=w.DEFAULT_SEED + rank)
        srv = x.Server(local, max_inflight=args.slots, max_batch=16, hbm_budget_bytes=150 * 10 ** 9)
        combos = [(n, b, tc) for n in (147, 24, 5) for b in ("s30", "s48") for tc in (False, True)]
        serve_stream(srv, [dict(t_arrive=0.002 * i, natoms=n, basis=b, two_component=tc)
                           for i, (n, b, tc) in enumerate(combos)], big, kinds_s, prec, args.slices)
        srv.reset_stats()
        done_s, _ = serve_stream(srv, reqs, big, kinds_s, prec, args.slices)
        st = srv.stats()
        srv.close()
        line["serving"] = {"requests": len(reqs), "rate_per_s": args.rate, "p50_ms": st["latency_p50_ms"],
                           "p99_ms": st["latency_p99_ms"], "max_ms": st["latency_max_ms"],
                           "service_p99_ms": pct(done_s["service_ms"], 99), "wait_p99_ms": pct(done_s["wait_ms"], 99),
                           "builds_per_s": st["builds_per_s"], "completed": st["completed"], "failed": st["failed"],
                           "precision": args.precision,
                           "workload": "Ag_n DLU, n log-uniform in [2,147], s30/s48, 30% two-component, "
                                       "pinned host inputs; latency = completion - scheduled arrival"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
