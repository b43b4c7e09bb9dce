"""Benchmark: lattice-cell updates per second of the fused stream-collide step
on the channel workload D2V33 (S^{D2V33}_{Q9E132}), Hermite order 4,
Nx = 4096 periodic x Ny = 512 between diffuse walls, seeded density
1 + 1e-3 N(0, 1), body force for Ma ~ 1e-3.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One benchmark step = --lb-steps (default 1000) lattice-Boltzmann time steps,
one kernel launch each.  `value` is device-resident throughput (GLUPS) over K
steps timed with CUDA events on the solver's stream; `e2e` is the same metric
through the C ABI with the density field copied from pinned host memory and
the mass flow read back every step.  With N > 1 (torchrun) every rank runs
its own channel (independent replicas, weak scaling); rank 0 prints one JSON
line.  `--impl reference` times the fp64 CPU oracle instead (rank 0 only).
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GLUPS & %HBM roofline"
# algorithmic fp64 operations of one node update: ~20 V after pairing the +-e
# populations (moments, equilibrium and force of each pair evaluated once)
FP64_FLOPS_PER_NODE_PER_V = 20
UNIT = "GLUPS"
DVM, ORDER, NX, NY, SEED = "D2V33", 4, 4096, 512, 20151029
WORKLOAD = ("channel D2V33 (S^{D2V33}_{Q9E132}), Hermite order 4, Nx=4096 periodic x "
            "Ny=512 diffuse Maxwell walls, rho=1+1e-3 N(0,1) seed 20151029, Ma~1e-3 force")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--lb-steps", type=int, default=1000)
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    p.add_argument("--kn", type=float, default=0.1)
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-config1", action="store_true")
    p.add_argument("--no-dvm-generator", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=8.0)
    p.add_argument("--serve-saturated-only", action="store_true",
                   help="serving section: only the saturated-capacity run")
    return p.parse_args()


def dist_env():
    from paper_1510_08886_gb300 import replicas
    return replicas.env()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1510_08886_gb300", "csrc")
    for fn in ("lbm_kernels.cuh", "lbm_internal.h", "k_fp32.cu", "k_fp64.cu"):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(precision):
    """DRAM bytes per launch from the committed ncu summary of this kernel,
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"stream_collide_{precision}_D2V33_4096x512.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    hsh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not hsh or hsh.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    """(logical cores, CPU model name) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def cpu_baseline(precision, Kn):
    """The fp64 oracle as it stands on the host cores: its OpenMP build (the
    same per-node arithmetic, nodes in parallel) on every logical core, best of
    3 timings of 5 full-size time steps of the benchmark workload; and one
    single-thread time step for context."""
    import oracle
    from lbm_inputs import rho_field
    ncores, model = host_cpu()
    rho = rho_field(NX, NY, seed=SEED)
    ch = oracle.channel(DVM, ORDER, NX, NY, Kn, oracle.force_for_mach(Kn)).init(rho)
    t0 = time.perf_counter()
    ch.step(1)
    dt1 = time.perf_counter() - t0
    threads = oracle.use_openmp(ncores) or 1
    ch.init(rho)
    ch.step(1)                                   # thread start-up
    times = []
    steps = 5
    for _ in range(3):
        t0 = time.perf_counter()
        ch.step(steps)
        times.append(time.perf_counter() - t0)
    best = min(times)
    return {"value": NX * NY * steps / best / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle", "host_cores": ncores, "cpu_model": model,
            "sample": f"{steps} time steps of the full {NX}x{NY} workload, fp64 C oracle "
                      f"(OpenMP build), {threads} threads, best of 3: "
                      + ", ".join(f"{t:.2f}" for t in times) + " s",
            "single_thread": {"value": NX * NY / dt1 / 1e9, "unit": UNIT,
                              "sample": f"1 time step, 1 thread ({dt1:.2f} s)"}}


def batched_section(lbm, torch):
    """Config-4 workload: 256 channels of uneven sizes, D2V33 (N=4) and the
    D3V107 (x, z) marginal (N=3), fp32, in the engine (persistent kernel per
    velocity set, CUDA-graph chunks, autotuned) vs the same channels stepped
    one solve at a time through the single-solve API."""
    from lbm_inputs import batch_workload
    work = batch_workload(256)
    sets = {n: lbm.dvm(n) for n in {it["dvm"] for it in work}}
    cells = sum(it["Nx"] * it["Ny"] for it in work)
    # algorithmic bytes of one step: every node reads and writes its V fp32 populations
    step_bytes = sum(2 * len(sets[it["dvm"]][1]) * 4 * it["Nx"] * it["Ny"] for it in work)
    need = sum(lbm.Engine.solve_bytes(*sets[it["dvm"]], it["Nx"], it["Ny"], "fp32") for it in work)
    eng = lbm.Engine("fp32", max_solves=256, arena_bytes=need + (64 << 20), chunk=100)
    tiled_slot = {}
    for it in work:
        e, w, c = sets[it["dvm"]]
        slot = eng.add(e, w, c, it["order"], it["Nx"], it["Ny"], it["Kn"], lbm.force_for_mach(it["Kn"]))
        assert slot is not None
        if it["Nx"] > 1:
            tiled_slot.setdefault(it["dvm"], slot)
    eng.autotune()
    schedule = {d: eng.schedule(sl) for d, sl in tiled_slot.items()}
    eng.run(2)
    torch.cuda.synchronize()
    chunks = 10
    t0 = time.perf_counter()
    eng.run(chunks)
    dt = time.perf_counter() - t0
    batched = cells * chunks * eng.chunk / dt / 1e9
    eng.close()
    # same channels, one solve at a time (launch per solve per step)
    solvers = []
    for it in work:
        e, w, c = sets[it["dvm"]]
        solvers.append(lbm.Solver(e, w, c, it["order"], it["Nx"], it["Ny"], it["Kn"],
                                  lbm.force_for_mach(it["Kn"]), precision="fp32").init())
    steps = 20
    for s in solvers:
        s.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in solvers:
        s.step(steps)
    torch.cuda.synchronize()
    dt1 = time.perf_counter() - t0
    per_solve = cells * steps / dt1 / 1e9
    for s in solvers:
        s.close()
    return {"workload": "256 channels, seed 20151030: Ny U{16..512}, Nx {1,64,256}, Kn log-U[0.01,1], "
                        "D2V33 N=4 / D3V107xz N=3, fp32",
            "cells": cells, "GLUPS_engine": batched, "GLUPS_per_solve_api": per_solve,
            "autotuned_schedule": schedule,
            "speedup": batched / per_solve, "timed_steps": chunks * 100,
            "bytes_per_step": step_bytes,
            "achieved_GBs": step_bytes * batched * 1e9 / cells / 1e9,
            "hbm_frac": step_bytes * batched / cells / measured_peaks()[0],
            "hbm_peak_kind": measured_peaks()[1]}


def torch_stream():
    import torch
    return torch.cuda.Stream()


def dvm_generator_section(lbm, with_oracle=True):
    """Host-side DVM generator (Sect. III-IV): from the velocities of every
    printed stencil alone, the lattice speed c* (scan [0.8 c, 1.2 c]) and the
    weights, or the W_zxx-augmented weights of the two augmented S3 sets;
    errors against the printed values and the time taken by the library and,
    on a subset, by the oracle."""
    from lbm_inputs import DVM_TABLES, TEXTBOOK_TABLES
    tables = {**DVM_TABLES, **TEXTBOOK_TABLES}
    augmented = ("D3V77", "D3V107")
    worst_c = worst_w = 0.0
    t_lib = 0.0
    for name, t in tables.items():
        e, w, c = lbm.dvm_from_groups(t)
        t0 = time.perf_counter()
        if name in augmented:
            k = [lbm.dvm_nontrivial_moments(3, t["Q"]).index((2, 0, 1))]
            ws, _ = lbm.dvm_augment(e, c, t["Q"], k)
        else:
            cs = lbm.dvm_find_c(e, t["Q"], 0.8 * c, 1.2 * c)
            ws, _ = lbm.dvm_weights(e, cs, t["Q"])
            worst_c = max(worst_c, abs(cs / c - 1))
        t_lib += time.perf_counter() - t0
        worst_w = max(worst_w, float(np.max(np.abs(ws / w - 1))))
    out = {"stencils": len(tables), "library_s": t_lib,
           "max_rel_err_c_vs_printed": worst_c, "max_rel_err_w_vs_printed": worst_w}
    if with_oracle:
        import oracle.dvm as odvm
        subset = ("D2V16", "D2V33", "D3V15", "D2Q9", "D3Q19")
        t0 = time.perf_counter()
        for name in subset:
            e, _, c = odvm.expand(tables[name])
            cs = odvm.find_c(e, tables[name]["Q"], 0.8 * c, 1.2 * c)
            odvm.solve_weights(e, cs, tables[name]["Q"])
        t_or = time.perf_counter() - t0
        t0 = time.perf_counter()
        for name in subset:
            e, _, c = lbm.dvm_from_groups(tables[name])
            lbm.dvm_weights(e, lbm.dvm_find_c(e, tables[name]["Q"], 0.8 * c, 1.2 * c),
                            tables[name]["Q"])
        out["subset"] = list(subset)
        out["subset_library_s"] = time.perf_counter() - t0
        out["subset_oracle_s"] = t_or
    return out


def config1_section(lbm):
    """Config 1: D2V16, N=3, Nx=1 x Ny=64, Kn=0.1, Ma 1e-3, rho=1, run until
    max|du| < 1e-10 tested every 100 steps (<= 50k steps): wall time to steady
    state on the GPU and with the fp64 CPU oracle.  fp64: resident chunks on one
    thread-block cluster (the default for so small a channel), on the default
    stream and as CUDA-graph chunks on a side stream, and one launch per step
    (resident off, graph chunks); fp32: resident chunks, default stream and graph
    chunks."""
    import oracle
    Kn = 0.1
    g = lbm.force_for_mach(Kn)
    e, w, c = lbm.dvm("D2V16")
    out = {}
    side = torch_stream()
    variants = (("fp64", "fp64", None, True), ("fp64_graphs", "fp64", side, True),
                ("fp64_per_step_graphs", "fp64", side, False), ("fp32", "fp32", None, True),
                ("fp32_graphs", "fp32", side, True))
    for label, prec, stream, resident in variants:
        s = lbm.Solver(e, w, c, 3, 1, 64, Kn, g, precision=prec, stream=stream)
        s.set_resident(resident).init()
        s.run_to_steady(1e-10, 2000)            # warm-up (first launches, clocks)
        s.init()
        t0 = time.perf_counter()
        conv, steps, du = s.run_to_steady(1e-10, 50000)
        dt = time.perf_counter() - t0
        out[label] = {"converged": conv, "steps": steps, "seconds": dt, "steps_per_s": steps / dt,
                      "resident_ctas": s.resident_ctas(), "mdot": s.mass_flow(),
                      "us": s.slip_velocity()}
        s.close()
    ch = oracle.channel("D2V16", 3, 1, 64, Kn, g).init()
    t0 = time.perf_counter()
    conv, steps, du = ch.run_to_steady(1e-10, 50000)
    dt = time.perf_counter() - t0
    out["oracle_cpu_1thread"] = {"converged": conv, "steps": steps, "seconds": dt,
                                 "steps_per_s": steps / dt, "mdot": ch.mass_flow()}
    out["mdot_rel_err_fp64_gpu_vs_oracle"] = abs(out["fp64"]["mdot"] / ch.mass_flow() - 1)
    out["mdot_rel_err_fp32_gpu_vs_oracle"] = abs(out["fp32"]["mdot"] / ch.mass_flow() - 1)
    return out


def _serve(lbm, items, sets, lanes, realtime, route=None, chunk=100, max_solves=1024):
    """Play the request list through engines of the given precisions
    (lanes: name -> precision) and return (stats, requests by id)."""
    from paper_1510_08886_gb300.serving import ContinuousBatcher, requests_from_workload
    engines = {name: lbm.Engine(prec, max_solves=max_solves,
                                arena_bytes=(4 << 30) if prec == "fp64" else (2 << 30), chunk=chunk)
               for name, prec in lanes.items()}
    reqs = requests_from_workload(items)
    b = ContinuousBatcher(engines if len(engines) > 1 else next(iter(engines.values())), sets,
                          route=route)
    st = b.serve(reqs, realtime=realtime)
    for e in engines.values():
        e.close()
    return st, {r.rid: r for r in b.done}


def _gate(served, ref, tol=1e-4):
    """Relative mass-flow error of every served request against the fp64
    reference at its own tolerance test; the gate holds when all are <= tol."""
    errs = {rid: abs(r.mdot / ref[rid].mdot - 1) for rid, r in served.items()
            if rid in ref and r.status == 0 and ref[rid].status == 0}
    bad = [rid for rid, e in errs.items() if e > tol]
    worst = sorted(bad, key=lambda rid: -errs[rid])[:5]
    return errs, {"max": max(errs.values()) if errs else None,
                  "median": float(np.median(list(errs.values()))) if errs else None,
                  "requests": len(errs), "failing": len(bad), "gate_1e-4": not bad,
                  "worst": [{"Ny": served[rid].Ny, "Kn": round(served[rid].Kn, 4),
                             "tol": served[rid].tol, "steps": served[rid].steps,
                             "steps_fp64": ref[rid].steps, "err": errs[rid],
                             "lane": served[rid].lane} for rid in worst]}


def _passing_stats(served, errs, wall, tol=1e-4):
    ok = [r for rid, r in served.items() if rid in errs and errs[rid] <= tol]
    lat = np.array([r.latency for r in ok]) if ok else np.array([math.nan])
    return {"solves_per_s": len(ok) / wall, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "requests": len(ok)}


def _first_check_stops(ref, first=100):
    """Requests whose fp64 reference met its test max|du| < tol at the first
    check (step `first`), by tolerance: the per-step change of a wide, slowly
    relaxing channel at Ma ~ 1e-3 is below 1e-6 from the start, so the rule
    as stated stops it in its start-up transient."""
    ok = [r for r in ref.values() if r.status == 0]
    by_tol = {}
    for r in ok:
        d = by_tol.setdefault(f"tol_{r.tol:g}", {"stopped": 0, "of": 0})
        d["stopped"] += int(r.steps <= first)
        d["of"] += 1
    return {"check_steps": first, "stopped": sum(int(r.steps <= first) for r in ok),
            "of": len(ok), "by_tol": dict(sorted(by_tol.items()))}


def _beyond_first_check(done, ref, wall, errs=None, first=100, tol=1e-4):
    """Rate and latencies over the completed requests whose fp64 reference ran
    past its first test (and, given errs, that pass the accuracy gate): the
    solves that reach the relaxation phase, over the run's whole wall time."""
    keep = [r for rid, r in done.items()
            if rid in ref and ref[rid].status == 0 and ref[rid].steps > first
            and (errs is None or (rid in errs and errs[rid] <= tol))]
    lat = np.array([r.latency for r in keep]) if keep else np.array([math.nan])
    return {"solves_per_s": len(keep) / wall, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "requests": len(keep)}


def _equal_steps(lbm, served, sets, sample):
    """fp64 engine advanced by exactly the served step count of each sampled
    request: the precision error alone (no stopping-rule effect)."""
    e, w, c = sets["D2V16"]
    eng = lbm.Engine("fp64", max_solves=len(sample) + 1, arena_bytes=4 << 30, chunk=100)
    slots = {}
    for rid in sample:
        r = served[rid]
        slots[eng.add(e, w, c, r.order, r.Nx, r.Ny, r.Kn, r.force)] = rid
    out = {}
    steps = 0
    while slots:
        res = eng.run(1)
        steps += 100
        for sl in [sl for sl, rid in slots.items() if served[rid].steps <= steps]:
            rid = slots.pop(sl)
            out[rid] = abs(served[rid].mdot / float(res[sl, 1]) - 1)
            eng.remove(sl)
    eng.close()
    return out


def serving_section(lbm, seconds, saturated_only=False):
    """Config-5 stream (Poisson 200/s, D2V16 N=3, Nx=1, Ny U{16..2048}, Kn
    log-U[0.01,1], tol in {1e-6,1e-8}) for `seconds` of arrivals.

    Reference: every request solved at its own tolerance by the fp64 engine
    (fp64 storage and arithmetic, matching the single-solve fp64 path to
    rounding; checked on the requests the plain path finishes).  Served:
    continuous batching with precision routing (fp32 engine, and an fp64
    engine for the requests whose stopping chunk fp32 could flip), in real
    time and saturated; the same with fp32 only; an fp16-storage arm
    (saturated).  Baseline: the plain per-solve fp64 path in real time.
    Accuracy gate: relative mass-flow error <= 1e-4 against the reference,
    per request; rates and latencies are also given over the passing
    requests only."""
    from lbm_inputs import serving_workload
    from paper_1510_08886_gb300.serving import (PrecisionRouter, requests_from_workload,
                                                serve_plain)
    items = serving_workload(duration_s=seconds)
    sets = {"D2V16": lbm.dvm("D2V16")}
    router = PrecisionRouter(sets)
    lanes = {"fp32": "fp32", "fp64": "fp64"}
    out = {"stream": f"{len(items)} requests in {seconds:.0f} s (Poisson 200/s, seed 20151031)"}
    ref_st, ref = _serve(lbm, items, sets, {"fp64": "fp64"}, realtime=False)
    out["reference_fp64_engine_saturated"] = ref_st.as_dict()
    sat_st, sat = _serve(lbm, items, sets, lanes, realtime=False, route=router)
    errs_sat, gate_sat = _gate(sat, ref)
    out["first_check_stops"] = _first_check_stops(ref)
    out["served_routed_saturated"] = {**sat_st.as_dict(), "accuracy": gate_sat,
                                      "fp64_routed": sum(r.lane == "fp64" for r in sat.values()),
                                      "passing": _passing_stats(sat, errs_sat, sat_st.wall_s),
                                      "passing_beyond_first_check": _beyond_first_check(
                                          sat, ref, sat_st.wall_s, errs_sat)}
    sat32_st, sat32 = _serve(lbm, items, sets, {"fp32": "fp32"}, realtime=False)
    out["served_fp32_only_saturated"] = {**sat32_st.as_dict(), "accuracy": _gate(sat32, ref)[1]}
    sat16_st, sat16 = _serve(lbm, items, sets, {"fp16": "fp16"}, realtime=False)
    out["served_fp16_only_saturated"] = {**sat16_st.as_dict(), "accuracy": _gate(sat16, ref)[1]}
    if saturated_only:
        return out
    st, served = _serve(lbm, items, sets, lanes, realtime=True, route=router)
    errs, gate = _gate(served, ref)
    out["served_routed_realtime"] = {**st.as_dict(), "accuracy": gate,
                                     "fp64_routed": sum(r.lane == "fp64" for r in served.values()),
                                     "passing": _passing_stats(served, errs, st.wall_s),
                                     "passing_beyond_first_check": _beyond_first_check(
                                         served, ref, st.wall_s, errs)}
    st32, served32 = _serve(lbm, items, sets, {"fp32": "fp32"}, realtime=True)
    errs32, gate32 = _gate(served32, ref)
    out["served_fp32_only_realtime"] = {**st32.as_dict(), "accuracy": gate32,
                                        "passing": _passing_stats(served32, errs32, st32.wall_s)}
    e, w, c = sets["D2V16"]

    def make(r):
        return lbm.Solver(e, w, c, r.order, r.Nx, r.Ny, r.Kn, r.force, precision="fp64").init()

    plain_reqs = requests_from_workload(items)
    plain = serve_plain(plain_reqs, make, realtime=True, time_limit=max(seconds, 1.0))
    done = [r for r in plain_reqs if not math.isnan(r.t_done) and r.status == 0]
    out["plain_fp64_per_solve"] = plain.as_dict()
    out["plain_vs_fp64_engine_max_rel"] = max(
        (abs(r.mdot / ref[r.rid].mdot - 1) for r in done if r.rid in ref), default=None)
    out["plain_vs_fp64_engine_same_steps"] = sum(r.steps == ref[r.rid].steps for r in done
                                                 if r.rid in ref)
    out["plain_completed"] = len(done)
    out["plain_fp64_beyond_first_check"] = _beyond_first_check(
        {r.rid: r for r in done}, ref, plain.wall_s)
    # precision alone, stratified over Ny and Kn, on fp32-served requests
    fp32_served = [r for r in served.values() if r.lane == "fp32" and r.status == 0]
    strata = {}
    for r in fp32_served:
        key = (min(3, r.Ny // 512), 0 if r.Kn < 0.1 else 1)
        strata.setdefault(key, []).append(r)
    sample = []
    for key, rs in sorted(strata.items()):
        rs.sort(key=lambda r: (-r.Ny, r.Kn))
        sample += [r.rid for r in rs[:3]]
    eq = _equal_steps(lbm, served, sets, sample)
    out["fp32_equal_steps_precision"] = {
        "max": max(eq.values()) if eq else None, "requests": len(eq),
        "strata": {f"Ny{k[0] * 512}-{k[0] * 512 + 511}_Kn{'<' if k[1] == 0 else '>='}0.1":
                   len(v) for k, v in sorted(strata.items())}}
    p = out["plain_fp64_per_solve"]["solves_per_s"]
    out["solves_per_s_ratio_passing"] = out["served_routed_realtime"]["passing"]["solves_per_s"] / \
        max(p, 1e-12)
    out["saturated_passing_vs_plain"] = out["served_routed_saturated"]["passing"]["solves_per_s"] / \
        max(p, 1e-12)
    pb = out["plain_fp64_beyond_first_check"]["solves_per_s"]
    out["solves_per_s_ratio_beyond_first_check"] = \
        out["served_routed_realtime"]["passing_beyond_first_check"]["solves_per_s"] / max(pb, 1e-12)
    out["saturated_vs_plain_beyond_first_check"] = \
        out["served_routed_saturated"]["passing_beyond_first_check"]["solves_per_s"] / max(pb, 1e-12)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from lbm_inputs import rho_field
    # each step: one full-size time step of the workload, the oracle as it
    # stands (its OpenMP build: same per-node arithmetic) on every host core
    ncores, model = host_cpu()
    threads = oracle.use_openmp(ncores) or 1
    rho = rho_field(NX, NY, seed=SEED)
    ch = oracle.channel(DVM, ORDER, NX, NY, args.kn, oracle.force_for_mach(args.kn)).init(rho)
    for _ in range(args.warmup):
        ch.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ch.step(1)
    dt = time.perf_counter() - t0
    v = NX * NY * args.steps / dt / 1e9
    sample = (f"1 full-size time step ({NX}x{NY}) per step, fp64 C oracle (OpenMP build), "
              f"{threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "lb_steps_per_step": 1, "sample_cells": NX * NY,
                   "parallelism": f"{threads} host threads"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "host_cores": ncores, "cpu_model": model, "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    from paper_1510_08886_gb300 import replicas
    dist = replicas.init("nccl", torch.device("cuda", local))
    if ws > 1:      # scaling runs time the headline workload only
        args.no_variants = args.no_batched = args.no_serving = True
        args.no_dvm_generator = True

    import __graft_entry__
    __graft_entry__.build_library()
    import paper_1510_08886_gb300 as lbm
    from paper_1510_08886_gb300 import _lib
    from lbm_inputs import rho_field

    e, w, c = lbm.dvm(DVM)
    V = len(w)
    ncell = NX * NY
    g = lbm.force_for_mach(args.kn)
    stream = torch.cuda.Stream()
    rho_host = rho_field(NX, NY, seed=replicas.replica_seed(SEED, rank))
    rho_dev = torch.tensor(rho_host, device="cuda")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_run(precision, Kn, lb, steps, warmup, sample_clocks=False, force=True):
        s = lbm.Solver(e, w, c, ORDER, NX, NY, Kn, lbm.force_for_mach(Kn) if force else 0.0,
                       precision=precision, stream=stream)
        s.init(rho_dev)
        for _ in range(warmup):
            s.step(lb)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.__enter__()
        ev0.record(stream)
        for _ in range(steps):
            s.step(lb)
        ev1.record(stream)
        ev1.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        barrier()
        ms = ev0.elapsed_time(ev1)
        st = s.status()
        mdot = s.mass_flow()
        s.close()
        return ms, (sampler.summary() if sampler else None), st, mdot

    # ---- headline: device-resident throughput ------------------------------
    ms, clocks, status, mdot = timed_run(args.precision, args.kn, args.lb_steps, args.steps,
                                         args.warmup, sample_clocks=True)
    launches = args.steps * args.lb_steps
    value, s_max = replicas.aggregate_rate(ncell * launches / 1e9, ms * 1e-3, dist, "cuda")
    ms_max = s_max * 1e3
    ELEM = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
    elem = ELEM[args.precision]
    bytes_per_launch = 2 * V * elem * ncell          # read + write every population once
    avg_launch_s = ms * 1e-3 / launches
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / avg_launch_s / 1e9
    traffic = ncu_traffic(args.precision)
    if args.precision != "fp64":
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind}
    else:
        # fp64: bound by GB300's fp64 pipe; the peak is measured live (FMA chains
        # on every SM, lbm_fma_rate), the flops are the algorithmic 20 V per node
        flops = FP64_FLOPS_PER_NODE_PER_V * V * ncell / avg_launch_s / 1e12
        alu_peak = lbm.fma_rate("fp64", stream) / 1e12
        roofline = {"bound": "alu", "achieved": flops, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": flops / alu_peak, "traffic": traffic,
                    "peak_kind": "measured: independent DFMA chains on every SM (lbm_fma_rate)",
                    "flops_per_node": FP64_FLOPS_PER_NODE_PER_V * V,
                    "hbm_achieved_GBs": achieved, "hbm_frac": achieved / peak}
    roofline.update({"kernel": "k_step_ct<SetD2V33, N=4> (fused pull-stream + walls + collide)",
                     "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6})

    # ---- e2e through the C ABI with host buffers ---------------------------
    pinned = torch.empty((NY, NX), dtype=torch.float64, pin_memory=True)
    pinned.numpy()[:] = rho_host
    s = lbm.Solver(e, w, c, ORDER, NX, NY, args.kn, g, precision=args.precision, stream=stream)
    L = _lib.lib()
    res = np.zeros(2)
    host_ptr = ctypes.cast(pinned.data_ptr(), _lib.c_double_p)
    mptr = res.ctypes.data_as(_lib.c_double_p)

    def e2e_step():
        _lib.check(L.lbm_init(s.handle, host_ptr), "lbm_init")
        _lib.check(L.lbm_step(s.handle, args.lb_steps), "lbm_step")
        _lib.check(L.lbm_mass_flow(s.handle, mptr, None), "lbm_mass_flow")

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ev1.record(stream)
    ev1.synchronize()
    wall = time.perf_counter() - t0
    e2e_ms = wall * 1e3          # host wall clock: copies, launches and reads included
    s.close()
    e2e_value, _ = replicas.aggregate_rate(ncell * args.steps * args.lb_steps / 1e9,
                                           e2e_ms * 1e-3, dist, "cuda")

    # ---- variants: both precisions, Kn in {0.01, 0.1, 1.0}; g = 0 ------------
    variants = []
    if not args.no_variants:
        runs = [(prec, Kn, True) for prec, kns in (("fp64", (0.01, 0.1, 1.0)),
                                                   ("fp32", (0.01, 0.1, 1.0)),
                                                   ("fp16", (0.1,)), ("bf16", (0.1,)))
                for Kn in kns]
        runs += [("fp64", 0.1, False), ("fp32", 0.1, False)]   # force-free specialisation
        for prec, Kn, force in runs:
            lb = 200
            vms, _, vst, vm = timed_run(prec, Kn, lb, 1, 1, force=force)
            el = ELEM[prec]
            variants.append({
                "precision": prec, "Kn": Kn, "g": "8 tau 1e-3" if force else 0.0, "lb_steps": lb,
                "GLUPS": ncell * lb / (vms * 1e-3) / 1e9,
                "achieved_GBs": 2 * V * el * ncell * lb / (vms * 1e-3) / 1e9,
                "mdot": vm if force else None, "status": vst})

    batched = None if args.no_batched else batched_section(lbm, torch)
    serving = None if args.no_serving else serving_section(lbm, args.serve_seconds,
                                                           args.serve_saturated_only)
    config1 = None if (args.no_config1 or ws > 1) else config1_section(lbm)
    dvmgen = None if (args.no_dvm_generator or rank != 0) else dvm_generator_section(
        lbm, with_oracle=not args.no_cpu_baseline)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.precision, args.kn)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (f16 storage)",
                      "bf16": "f32 (bf16 storage)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "Kn": args.kn, "lb_steps_per_step": args.lb_steps,
                       "cells": ncell, "velocities": V,
                       "storage": {"fp32": "fp32 deviations fbar - w",
                                   "fp64": "fp64 deviations fbar - w",
                                   "fp16": "fp16 (fbar - w)/(w S)",
                                   "bf16": "bf16 (fbar - w)/(w S)"}[args.precision],
                       "l2": "inputs larger than L2 (two lattices of "
                             f"{V * elem * ncell / 1e6:.0f} MB each)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": ncell * 8,
                    "d2h_bytes_per_step": 4 * 8 + 4},
            "gpu_launches": launches,
            "clocks": clocks,
            "status": status, "mdot": mdot,
            "variants": variants,
            "batched": batched,
            "serving": serving,
            "config1": config1,
            "dvm_generator": dvmgen,
        }))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
