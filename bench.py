#!/usr/bin/env python3
"""Benchmark of the H-matrix DD-BEM hot path on one GB300 (or N replicas).

A step is one H-matrix product y = E x (FP32 factors, one right-hand side) of the
51,468-element disk fault (256 x 256 grid, r < 1; leaf 64, eta 2, ACA eps 1e-6), the
operator that every GMRES iteration applies.  The H-matrix is assembled once before the
timed region (setup, reported apart).  value = algorithmic bytes of the product (stored
near-field entries x 4 B + factor entries x 4 B + x and y) / time, summed over ranks.
The coefficients (4.3 GB) are far larger than L2 (129 MB), so consecutive products read
them from HBM; no L2 flush is needed.

Also reported: the per-phase roofline of the dominant kernel (CUDA events on the
launching stream), the end-to-end rate through hm_matvec_host (host vectors, copies in
the timed region), GMRES time-to-1e-8 for the plain FP64 and the mixed BF16 + FP64
refinement solvers, clocks sampled during the timed region, and the CPU oracle timed on
this machine's host cores on a bounded sample of rows.

`--impl reference` times the CPU FP64 oracle (the dense product, row-sampled) on the
host cores with the same metric and prints the reference line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H-matvec GB/s (% HBM peak); GMRES time-to-1e-8 residual, mixed vs plain FP64"
WORKLOAD = "disk fault r<1 on 256x256 grid: N=51468 rectangular DD elements, 154404 DOFs, leaf 64, eta 2, ACA eps 1e-6"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--storage", default="f32", choices=["f32", "bf16"])
    p.add_argument("--no-gmres", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--grid", type=int, default=256, help="disk grid size (256: the 51,468-element fault)")
    p.add_argument("--planes-grid", type=int, default=300,
                   help="grid of each plane of the planes workload (300: 270,000 elements)")
    p.add_argument("--lp-h", type=float, default=0.01, help="element size of the crack + fault (learned workload)")
    p.add_argument("--lp-train", type=int, default=2000, help="training systems (learned workload)")
    p.add_argument("--workload", default="fault",
                   choices=["fault", "faults64", "planes", "learned", "ilu", "interface", "coupled", "triangles"],
                   help="fault: the 51,468-element disk fault (default); faults64: 64 independent faults, "
                        "batched product vs per-fault launches; planes: three intersecting 300x300 planes, "
                        "16 right-hand sides")
    p.add_argument("--batch-storage", default="bf16", choices=["f32", "bf16"],
                   help="factor storage of the 64-fault batch (BF16 factors, FP32 near field)")
    p.add_argument("--tune", action="store_true", help="also run the leaf-size autotuner on the workload")
    p.add_argument("--record-dir", default=None,
                   help="write the operator summary (entry counts, algorithmic bytes) of the fault as JSON here")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)[kernel]
        src = open(os.path.join(ROOT, "paper_2605_14397_gb300", "csrc", "matvec.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != d["matvec_cu_sha256_16"]:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


def product_bytes(info, storage):
    """Algorithmic bytes of one single-RHS product (every stored near-field entry, 4 B,
    and factor entry, 4 B or 2 B for BF16, once; x read and y written once) and of its
    two streaming kernels: phase 2 (near entries + U factors + operands + y) and phase 1
    (V factors + x + partials)."""
    fb = 2 if storage == "bf16" else 4
    n = info["n_dof"]
    total = 4 * info["near_entries"] + fb * (info["u_entries"] + info["v_entries"]) + 2 * 4 * n
    phase2 = 4 * info["near_entries"] + fb * info["u_entries"] + 4 * n + 4 * info["tb_len"] + 4 * n
    phase1 = fb * info["v_entries"] + 4 * n + 4 * info["p_len"]
    return total, phase2, phase1


def oracle_rows_rate(el, E, nu, budget_s=15.0, max_rows=None):
    """Oracle dense rows per second on this host (all cores), on a seeded row sample."""
    import numpy as np
    from oracle import oracle as O
    from paper_2605_14397_gb300 import synth
    x = synth.rhs_shear_plus_bump(el)
    rng = np.random.default_rng(1603)
    probe = np.sort(rng.choice(el.N, size=16, replace=False))
    t0 = time.perf_counter()
    O.dense_matvec_rows(el, E, nu, x, probe)
    per_row = (time.perf_counter() - t0) / 16
    rows = int(max(16, min(el.N, budget_s / max(per_row, 1e-9))))
    if max_rows:
        rows = min(rows, max_rows)
    sample = np.sort(rng.choice(el.N, size=rows, replace=False))
    t0 = time.perf_counter()
    O.dense_matvec_rows(el, E, nu, x, sample)
    dt = time.perf_counter() - t0
    return rows / dt, rows, dt


def time_gmres(H, el, dev, torch, reps=3):
    """GMRES time-to-1e-8 on the same fault: (E) x = b, b = uniform shear + Gaussian
    pressure bump, leaf block-Jacobi, restart 50, x0 = 0.  Plain: FP64 Krylov with every
    product compensated FP64 on the FP32 factors.  IR FP32: FP64 refinement of
    corrections solved with the FP32 factors and FP32 products.  Mixed: the same
    refinement with the BF16 factors.  All three stop on the residual of the FP32-factor
    operator recomputed in compensated FP64 (<= 1e-8 ||b||).  The paper's point (3x3)
    Jacobi preconditioner is timed with the plain solver beside leaf block-Jacobi."""
    from paper_2605_14397_gb300 import synth
    b = torch.from_numpy(synth.rhs_shear_plus_bump(el)).to(dev)
    x = torch.zeros_like(b)
    out = {"tol": 1e-8, "restart": 50, "precond": "leaf block-Jacobi", "rhs": "shear + Gaussian bump"}
    for key, mode, pc in (("plain_fp64", "f64", "blockj"), ("ir_fp32", "plain32", "blockj"),
                          ("mixed_bf16_ir", "mixed", "blockj"), ("plain_fp64_point_jacobi", "f64", "jacobi3")):
        times, info = [], None
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = H.solve(b, x, mode=mode, tol=1e-8, restart=50, precond=pc, maxit=3000)[0]
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        out[key] = {"seconds": statistics.median(times), "iters": info["iters"], "outer": info["outer"],
                    "relres": info["relres"]}
    out["speedup_mixed_over_plain"] = out["plain_fp64"]["seconds"] / out["mixed_bf16_ir"]["seconds"]
    out["speedup_ir_fp32_over_plain"] = out["plain_fp64"]["seconds"] / out["ir_fp32"]["seconds"]
    out["speedup_mixed_over_ir_fp32"] = out["ir_fp32"]["seconds"] / out["mixed_bf16_ir"]["seconds"]
    return out


def run_faults64(args, dev, torch, hmat, synth):
    """64 independent disk faults (log-uniform 2k-40k elements, seeded normals and nu,
    795,192 elements in all): one batched H-matrix (one work list, 5 launches per
    product; also replayed from a CUDA graph) against per-fault products (64 x 5
    launches; also 64 graph replays).  value = algorithmic bytes of all 64 products /
    time of the batched product."""
    import numpy as np
    els, nus = synth.config_faults_batch()
    E, eps = 1.0, 1e-6
    t0 = time.perf_counter()
    parts = []
    for el, nu in zip(els, nus):
        T = hmat.ClusterTree(el, 64, 2.0)
        parts.append(hmat.HMatrix(T, el, E, float(nu), eps, args.batch_storage))
        del T
    torch.cuda.synchronize()
    t_parts = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = hmat.HMatrix.batch(parts)
    t_merge = time.perf_counter() - t0
    info = B.info()
    Bytes, _, _ = product_bytes(info, args.batch_storage)
    nd = info["n_dof"]
    x = torch.as_tensor(synth.rhs_normal(nd, 1604), dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    offs = np.cumsum([0] + [3 * el.N for el in els])
    xs = [x[offs[f]:offs[f + 1]] for f in range(len(els))]
    ys = [y[offs[f]:offs[f + 1]] for f in range(len(els))]
    stream = torch.cuda.current_stream()

    def batched():
        B.matvec(x, y, stream)

    def batched_graph():
        B.matvec_graph(x, y, stream)

    def per_fault():
        for H, a, b in zip(parts, xs, ys):
            H.matvec(a, b, stream)

    def per_fault_graph():
        for H, a, b in zip(parts, xs, ys):
            H.matvec_graph(a, b, stream)

    res = {}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for name, fn in (("batched", batched), ("batched_graph", batched_graph), ("per_fault", per_fault),
                     ("per_fault_graph", per_fault_graph)):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            fn()
        ev1.record(stream)
        ev1.synchronize()
        res[name] = ev0.elapsed_time(ev1) / args.steps
    # tile shape of the batched product: every candidate timed, the fastest kept
    tune = B.tune_tile_shape(reps=20)
    for _ in range(max(3, args.warmup)):
        batched()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        batched()
    ev1.record(stream)
    ev1.synchronize()
    res["batched_tuned_shape"] = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop()
    B.timing(True)
    for _ in range(10):
        B.matvec(x, y, stream)
    B.timing(False)
    ph = B.timing_read()
    B.check(stream)
    for H in parts:
        H.check(stream)
    hbm, peak_kind = peaks()
    best_ms = min(res["batched"], res["batched_tuned_shape"])
    value = Bytes / (best_ms * 1e-3) / 1e9
    Ns = [el.N for el in els]
    line = {"metric": "batched H-matvec GB/s over 64 independent faults", "value": value, "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": best_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "tile_shape": {"tuned": tune["best"], "candidates": tune["candidates"],
                           "gain_over_default": res["batched"] / res["batched_tuned_shape"]},
            "dtype": "f32" if args.batch_storage == "f32" else "bf16 factors, f32 accumulation",
            "data": "synthetic (seeded meshes and right-hand side)",
            "config": {"workload": "64 disk faults, N_f log-uniform in [2k, 40k] (%d..%d), %d elements, h = 2/256, "
                                   "nu_f ~ U[0.2, 0.3], leaf 64, eta 2, ACA eps 1e-6" % (min(Ns), max(Ns), sum(Ns)),
                       "nrhs": 1, "storage": args.batch_storage + " factors, f32 near field",
                       "bytes_per_product": Bytes,
                       "assemble_parts_s": t_parts, "merge_s": t_merge,
                       "l2": "operator %.1f GB >> 129 MB L2: no flush" % (Bytes / 1e9)},
            "frac_of_hbm_peak": value / hbm, "peak_source": peak_kind,
            "ms_per_product": res, "speedup_batched_over_per_fault": res["per_fault"] / best_ms,
            "launches_per_product": {"batched": 5, "per_fault": 5 * len(parts)}, "clocks": clocks,
            "batched_phases_ms": {k: ph[k] / max(ph["count"], 1) for k in ("gather", "phase1", "reduce", "phase2",
                                                                           "scatter")}}
    if args.tune:
        line["autotune_largest_fault"] = hmat.autotune(els[int(np.argmax(Ns))], E, float(nus[int(np.argmax(Ns))]),
                                                       eps, "f32", leaves=(32, 48, 64, 96, 128), etas=(2.0,),
                                                       budget_ms=120000)
    print(json.dumps(line), flush=True)


def run_planes(args, dev, torch, hmat, synth):
    """Three intersecting square planes (300 x 300 each, N = 270,000, 810,000 DOFs;
    leaf 64, eta 2, ACA eps 1e-5), 16 seeded N(0, 1) right-hand sides: the product with
    16 RHS per pass of the coefficient streams (FP32 and BF16 factors) against 16
    single-RHS products, and GMRES to 1e-8 on all 16 at once (restart 30) against 16
    sequential solves."""
    import numpy as np
    el = synth.config_three_planes(args.planes_grid)
    E, nu, eps, nr = 1.0, 0.25, 1e-5, 16
    t0 = time.perf_counter()
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, E, nu, eps, "both")
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    info = H.info()
    nd = info["n_dof"]
    X = torch.as_tensor(synth.rhs_normal(nd, 1603, nrhs=nr), dtype=torch.float32, device=dev).contiguous()
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()
    res = {}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()

    def timeit(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    res["f32_16rhs_ms"] = timeit(lambda: H.matvec(X, Y, stream), args.steps)
    res["f32_1rhs_x16_ms"] = 16 * timeit(lambda: H.matvec(X[0], Y[0], stream), args.steps)
    res["bf16_16rhs_ms"] = timeit(lambda: H.matvec(X, Y, stream, factors="bf16"), args.steps)
    res["bf16_1rhs_x16_ms"] = 16 * timeit(lambda: H.matvec(X[0], Y[0], stream, factors="bf16"), args.steps)
    phases = {}
    for nrk, xa, ya in ((16, X, Y), (1, X[0], Y[0])):
        for fac in ("f32", "bf16"):
            H.timing(True)
            for _ in range(5):
                H.matvec(xa, ya, stream, factors=fac)
            H.timing(False)
            ph = H.timing_read()
            phases["%s_%drhs" % (fac, nrk)] = {k: ph[k] / max(ph["count"], 1)
                                               for k in ("gather", "phase1", "reduce", "phase2", "scatter")}
    clocks = sampler.stop()
    H.check(stream)
    # algorithmic bytes of one 16-RHS product: every stored near entry (4 B) and factor
    # entry (4 B FP32, 2 B BF16) once, x read and y written once per right-hand side
    n_coef_near = info["near_entries"]
    n_fac = info["u_entries"] + info["v_entries"]
    vec16 = nr * 2 * 4 * nd
    b16_f32 = 4 * n_coef_near + 4 * n_fac + vec16
    b16_bf16 = 4 * n_coef_near + 2 * n_fac + vec16
    # phase 2 of the BF16 product: near tiles + U slices + x and t operands + y
    ph2_bf16 = 4 * n_coef_near + 2 * info["u_entries"] + nr * 4 * (2 * nd + info["tb_len"])
    ph1_bf16 = 2 * info["v_entries"] + nr * 4 * (nd + info["p_len"])
    flops16 = 2.0 * nr * (n_coef_near + n_fac)  # 2 flops per stored coefficient and RHS
    hbm, peak_kind = peaks()
    t16 = res["bf16_16rhs_ms"] * 1e-3
    tf = res["f32_16rhs_ms"] * 1e-3
    pb = phases["bf16_16rhs"]
    ach = ph2_bf16 / (pb["phase2"] * 1e-3) / 1e9
    line = {"metric": "16-RHS H-matvec GB/s (BF16 factors, FP32 near field); GMRES time-to-1e-8, 16 RHS batched "
                      "vs sequential",
            "value": b16_bf16 / t16 / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["bf16_16rhs_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 factors x bf16 hi+lo vectors on tensor cores, f32 near field and accumulation",
            "data": "synthetic (seeded mesh and right-hand sides)",
            "config": {"workload": "three intersecting %dx%d planes (third shifted h/4): N=%d, %d DOFs, "
                                   "leaf 64, eta 2, ACA eps 1e-5, 16 RHS N(0,1)" % (args.planes_grid, args.planes_grid,
                                                                                    el.N, 3 * el.N),
                       "setup_s": t_setup, "rank_mean": info["rank_mean"], "rank_max": info["rank_max"],
                       "stored_bytes": info["stored_bytes"], "bytes_16rhs_bf16": b16_bf16,
                       "bytes_16rhs_f32": b16_f32,
                       "l2": "operator %.1f GB >> 129 MB L2: no flush" % (b16_bf16 / 1e9)},
            "frac_of_hbm_peak": b16_bf16 / t16 / 1e9 / hbm, "peak_source": peak_kind,
            "roofline": {"bound": "hbm", "kernel": "k_phase2 (16 RHS, BF16 U slices on tensor cores)",
                         "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "algorithmic_bytes_per_launch": ph2_bf16, "launch_ms": pb["phase2"],
                         "phase1_GBs": ph1_bf16 / (pb["phase1"] * 1e-3) / 1e9, "traffic": None},
            "f32_factors_16rhs": {"ms": res["f32_16rhs_ms"], "GBs": b16_f32 / tf / 1e9,
                                  "tflops": flops16 / tf / 1e12},
            "tflops_16rhs_bf16": flops16 / t16 / 1e12, "ms": res,
            "speedup_16rhs_over_16x1": {"bf16": res["bf16_1rhs_x16_ms"] / res["bf16_16rhs_ms"],
                                        "f32": res["f32_1rhs_x16_ms"] / res["f32_16rhs_ms"]},
            "clocks": clocks, "phases_ms": phases}
    if not args.no_gmres:
        # the tangent A = E - diag(k), k log-uniform in [1e-3, 1e2] E/h per element: the bare
        # E of three intersecting planes is indefinite and nearly singular (GMRES with
        # block-Jacobi stalls on it even at a few thousand elements), the tangent is not
        k = torch.as_tensor(synth.k_loguniform(el.N, 1605, E=E, h=2.0 / args.planes_grid), device=dev)
        B = torch.as_tensor(synth.rhs_normal(nd, 1603, nrhs=nr), dtype=torch.float64, device=dev).contiguous()
        Xs = torch.zeros_like(B)
        g = {"system": "E - diag(k), k ~ logU[1e-3, 1e2] E/h (seed 1605)", "restart": 50, "maxit": 1000,
             "tol": 1e-8, "precond": "leaf block-Jacobi"}

        def solve(b, x, mode):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            inf = H.solve(b, x, k, mode=mode, tol=1e-8, restart=50, maxit=1000, precond="blockj",
                          raise_on_error=False)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, inf

        for mode in ("f64", "mixed"):
            t1, i1 = solve(B[0], Xs[0], mode)
            r = {"single_s": t1, "single_iters": i1[0]["iters"], "single_status": i1[0]["status"]}
            if i1[0]["status"] == 0 and t1 < 30.0:
                tb, ib = solve(B, Xs, mode)
                r.update({"batched_s": tb, "iters_batched_max": max(i["iters"] for i in ib),
                          "relres_max": max(i["relres"] for i in ib),
                          "all_converged": all(i["status"] == 0 for i in ib)})
                if t1 < 5.0:
                    ts = 0.0
                    its = []
                    for q in range(nr):
                        dt, iq = solve(B[q], Xs[q], mode)
                        ts += dt
                        its.append(iq[0]["iters"])
                    r.update({"sequential_s": ts, "iters_sequential_max": max(its), "sequential": "measured"})
                else:
                    r.update({"sequential_s": nr * t1, "sequential": "16 x the first right-hand side's time"})
                r["speedup_batched_over_sequential"] = r["sequential_s"] / tb
            g[mode] = r
        line["gmres_16rhs"] = g
    print(json.dumps(line), flush=True)


def run_learned(args, dev, torch, hmat, synth):
    """Learned corrections of leaf block-Jacobi on the crack crossing a fault (h = 0.01:
    40,000 + 160,000 elements): tangent systems A = E - diag(k), k log-uniform in
    [1e-3, 1e2] E/h per element, a fresh draw per system, N(0, 1) right-hand sides.  Two
    networks are trained on the same solved systems (seeds 1605000 + i; 2,000 by default,
    one RHS each, x by block-Jacobi GMRES to 1e-8), 500 Adam steps each: the scaling
    M = D B^-1 and the near correction M = B^-1 - gamma D B^-1 N B^-1.  Validation on 4
    more systems picks gamma (from 0.6 to 1.0) and decides each fallback (plain
    block-Jacobi unless the learned correction takes fewer iterations); the same near
    correction with the untrained network (d = 1) and its own gamma is the control that
    shows what training adds; test: 8 held-out systems (seeds 1606000 + i), GMRES to 1e-8,
    restart 50, plain FP64 mode.  value = the block-Jacobi time over the trained near
    correction's time on the held-out systems."""
    import numpy as np
    h = args.lp_h
    el = synth.config_crack_fault(h=h)
    E, nu, eps = 1.0, 0.25, 1e-6
    t0 = time.perf_counter()
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, E, nu, eps, "f32")
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    nd = 3 * el.N

    def system(seed, nrhs=1):
        k = torch.as_tensor(synth.k_loguniform(el.N, seed, E=E, h=h), device=dev)
        b = torch.as_tensor(synth.rhs_normal(nd, seed, nrhs=nrhs), device=dev).contiguous()
        if nrhs == 1:
            b = b.reshape(-1)
        return k, b

    def solve(k, b, precond, model=None, tol=1e-8):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.perf_counter()
        info = H.solve(b, x, k, precond=precond, model=model, tol=tol, restart=50, maxit=3000, raise_on_error=False)
        torch.cuda.synchronize()
        return x, info[0], time.perf_counter() - t

    models = {"scale": hmat.LearnedCorrection(synth.lp_initial_weights(32, seed=1607), hidden=32),
              "near": hmat.LearnedCorrection(synth.lp_initial_weights(32, seed=1607), hidden=32)}
    models["near"].set_kind("near", 1.0)
    t0 = time.perf_counter()
    for i in range(args.lp_train):
        k, b = system(1605000 + i, nrhs=1)
        x = torch.zeros_like(b)
        H.solve(b, x, k, precond="blockj", tol=1e-8, restart=50, maxit=3000, raise_on_error=False)
        for m in models.values():
            m.add_system(H, k, b, x)
    t_data = time.perf_counter() - t0
    loss, t_train = {}, {}
    for name, m in models.items():
        l0, _ = m.loss_grad()
        t0 = time.perf_counter()
        l1 = m.train(500, lr=3e-3)
        torch.cuda.synchronize()
        t_train[name] = time.perf_counter() - t0
        l2, _ = m.loss_grad()
        loss[name] = {"initial": l0, "before_last_step": l1, "final": l2}
    vsys = [system(1605500 + i) for i in range(4)]
    val = {"blockj": [solve(k, b, "blockj")[1]["iters"] for k, b in vsys],
           "scale": [solve(k, b, "learned", models["scale"])[1]["iters"] for k, b in vsys]}
    # the same near correction with the untrained network (zero output layer: d = 1), its
    # gamma picked the same way: what the trained network adds beyond the damping
    models["near_untrained"] = hmat.LearnedCorrection(synth.lp_initial_weights(32, seed=1607), hidden=32)
    gammas, gbest = {}, {}
    for name in ("near", "near_untrained"):
        gammas[name] = {}
        for g in (0.6, 0.7, 0.8, 0.9, 1.0):
            models[name].set_kind("near", g)
            gammas[name][g] = [solve(k, b, "learned", models[name])[1]["iters"] for k, b in vsys]
        gbest[name] = min(gammas[name], key=lambda g: (float(np.mean(gammas[name][g])), g))
        models[name].set_kind("near", gbest[name])
        val[name] = gammas[name][gbest[name]]
    fallback = {name: float(np.mean(val[name])) >= float(np.mean(val["blockj"])) for name in models}
    for name, m in models.items():
        m.set_fallback(fallback[name])
    test = {pc: {"iters": [], "s": [], "relres": []} for pc in ("blockj", "scale", "near", "near_untrained")}
    for i in range(8):
        k, b = system(1606000 + i)
        for pc in test:
            _, inf, dt = solve(k, b, "blockj" if pc == "blockj" else "learned", None if pc == "blockj" else models[pc])
            test[pc]["iters"].append(inf["iters"])
            test[pc]["s"].append(dt)
            test[pc]["relres"].append(inf["relres"])
    tb, tn = sum(test["blockj"]["s"]), sum(test["near"]["s"])
    line = {"metric": "GMRES time-to-1e-8 on held-out tangent systems, learned near correction vs block-Jacobi",
            "value": tb / tn, "unit": "x (block-Jacobi time / learned time)", "n_gpus": 1, "steps": 8, "warmup": 0,
            "ms_per_step": 1e3 * tn / 8, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 Krylov, f32 preconditioner and network", "data": "synthetic (seeded k, right-hand sides)",
            "config": {"workload": "crack x in [-2,2], z in [-0.5,0.5] crossing a 4x4 fault, h=%g: N=%d; "
                                   "k ~ logU[1e-3, 1e2] E/h per element" % (h, el.N),
                       "setup_s": t_setup, "train_systems": args.lp_train, "train_rhs_per_system": 1,
                       "train_targets": "x = A^-1 b by block-Jacobi GMRES to 1e-8",
                       "adam_steps": 500, "lr": 3e-3, "hidden": 32},
            "loss": loss, "data_s": t_data, "train_s": t_train, "validation_iters": val,
            "gamma_scan": {name: {str(g): v for g, v in gs.items()} for name, gs in gammas.items()}, "gamma": gbest,
            "fallback": fallback,
            "test": test, "mean_iters": {pc: float(np.mean(test[pc]["iters"])) for pc in test},
            "time_ratio_vs_blockj": {pc: tb / sum(test[pc]["s"]) for pc in test}}
    print(json.dumps(line), flush=True)


def run_ilu(args, dev, torch, hmat, synth):
    """The ILU(0) preconditioner of Sec. 3.3.1 against leaf block-Jacobi and the paper's
    point Jacobi: GMRES(50) iterations and time to 1e-8 on tangent systems
    A = E - diag(k), k log-uniform in [1e-3, 1e2] E/h per element (seed 1605), one
    N(0, 1) right-hand side (seed 1606), x0 = 0, plain FP64 and mixed modes, on the
    51,468-element fault (eps 1e-6) and the crack crossing a fault (h = 0.01: 200,000
    elements, eps 1e-6).  The first ILU solve of a fraction p also builds the pattern
    (reported apart); every solve factors for its k."""
    import numpy as np
    out = {"metric": "GMRES time-to-1e-8 on tangent systems: ILU(0) (Sec. 3.3.1) vs leaf block-Jacobi",
           "unit": "s", "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 Krylov; f32 H-matrix, f64 ILU", "data": "synthetic (seeded k, right-hand side)",
           "cases": {}}
    for name, el, h in (("fault256", synth.config_fault(256), 2.0 / 256),
                        ("crackfault_h0.01", synth.config_crack_fault(h=0.01), 0.01)):
        T = hmat.ClusterTree(el, 64, 2.0)
        H = hmat.HMatrix(T, el, 1.0, 0.25, 1e-6, "both")
        k = torch.as_tensor(synth.k_loguniform(el.N, 1605, E=1.0, h=h), device=dev)
        b = torch.as_tensor(synth.rhs_normal(3 * el.N, 1606), device=dev)
        res = {"N": el.N}
        for mode in ("f64", "mixed"):
            for pc, p, meth in (("blockj", 0.0, "fgmres"), ("jacobi3", 0.0, "fgmres"), ("ilu", 0.01, "fgmres"),
                                ("ilu", 0.05, "fgmres"), ("jacobi3", 0.0, "bicgstab"), ("ilu", 0.01, "bicgstab")):
                key = "%s_%s%s%s" % (mode, pc, "_p%.2f" % p if pc == "ilu" else "",
                                     "_bicgstab" if meth == "bicgstab" else "")
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                inf = H.solve(b, x, k, precond=pc, mode=mode, ilu_p=p, maxit=3000, raise_on_error=False,
                              method=meth)[0]
                torch.cuda.synchronize()
                first = time.perf_counter() - t0
                times = []
                for _ in range(3):
                    x.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    inf = H.solve(b, x, k, precond=pc, mode=mode, ilu_p=p, maxit=3000, raise_on_error=False,
                                  method=meth)[0]
                    torch.cuda.synchronize()
                    times.append(time.perf_counter() - t0)
                res[key] = {"seconds": statistics.median(times), "first_call_s": first, "iters": inf["iters"],
                            "outer": inf["outer"], "relres": inf["relres"], "status": inf["status"]}
        for mode in ("f64", "mixed"):
            bj = res["%s_blockj" % mode]["seconds"]
            for p in (0.01, 0.05):
                res["%s_speedup_ilu_p%.2f_over_blockj" % (mode, p)] = bj / res["%s_ilu_p%.2f" % (mode, p)]["seconds"]
        out["cases"][name] = res
        del H, T
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_interface(args, dev, torch, hmat, synth):
    """The interface constitutive update and its consistent tangent (Sec. 2.2, 3.1.1,
    eq. jac_mech) at 4,000,000 seeded points (the softening joint; about 70 % of the
    points return plastically).  Bytes per point: the state and increment read (4 x 24 B)
    and the new state, C^ep and mode written (3 x 24 + 72 + 4 B) = 244 B; inputs far larger
    than L2 (976 MB)."""
    import numpy as np
    n = 4_000_000
    kw = synth.INTERFACE_PARAMS["softening"]
    T, dp, chi, dd = (torch.as_tensor(a, device=dev) for a in synth.interface_states(n, 1608))
    T1, dp1, chi1 = torch.empty_like(T), torch.empty_like(dp), torch.empty_like(chi)
    st = torch.cuda.current_stream()
    res = {}
    for label, tangent in (("with_tangent", True), ("values_only", False)):
        for _ in range(max(3, args.warmup)):
            hmat.interface_update(kw, T, dp, chi, dd, T1, dp1, chi1, tangent=tangent, stream=st)
        out = hmat.interface_update(kw, T, dp, chi, dd, T1, dp1, chi1, tangent=tangent, stream=st)
        reps = max(5, min(args.steps, 50))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            hmat.interface_update(kw, T, dp, chi, dd, T1, dp1, chi1, tangent=tangent, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nbytes = n * (96 + 72 + (72 if tangent else 0) + 4)
        res[label] = {"ms": ms, "points_per_s": n / (ms * 1e-3), "GBs": nbytes / (ms * 1e-3) / 1e9,
                      "bytes_per_point": nbytes // n}
    mc = np.bincount(out[4].cpu().numpy(), minlength=512)
    modes = dict(zip(hmat.INTERFACE_MODES, (int(c) for c in mc[:5])))
    modes["unresolved"] = int(mc[256:].sum())
    peak, src = peaks()
    line = {"metric": "interface constitutive update + consistent tangent, points/s", "unit": "points/s",
            "value": res["with_tangent"]["points_per_s"], "n_gpus": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded states)",
            "config": {"workload": "4,000,000 interface points, softening joint (Ks 10, Kn 20, f 0.6 -> 0.3, "
                                   "psi 0.1, dc 0.2, c 0.1, sigma_t 0.5, wc 0.4)", "modes": modes,
                       "l2": "inputs 976 MB >> 129 MB L2: no flush"},
            "results": res, "frac_of_hbm_peak": res["with_tangent"]["GBs"] / peak, "peak_source": src}
    print(json.dumps(line), flush=True)


def run_coupled(args, dev, torch, hmat, synth):
    """The coupled hydro-mechanical Jacobian solve of Sec. 3.3.1 on the 51,468-element
    fault (52,156 pressure nodes): FGMRES with the upper block triangular preconditioner
    P_up, nested A11 solves (leaf block-Jacobi FGMRES, or the paper's BiCGSTAB with the
    ILU of Sec. 3.3.1), the Schur complement with diag(A11); k log-uniform in
    [1e-2, 1e1] E/h, shift 0.3 E/h, opening U[0, 0.25] h, Delta p and p^n - p^o N(0, 0.1),
    mu 0.8, M 4, w0 0.25 h, dt 0.1; the right-hand side J x* of an N(0, 1) x*; to 1e-8."""
    import numpy as np
    el = synth.config_fault(256)
    h = 2.0 / 256
    conn, nn = synth.node_connectivity(el)
    t0 = time.perf_counter()
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, 1.0, 0.25, 1e-6, "both")
    fl = hmat.Flow(conn, nn, el.a, el.b)
    rng = np.random.default_rng(1609)
    dn = torch.as_tensor(rng.uniform(0.0, 0.25 * h, el.N), device=dev)
    dp = torch.as_tensor(rng.normal(size=nn) * 0.1, device=dev)
    pn = torch.as_tensor(rng.normal(size=nn) * 0.1, device=dev)
    par = dict(mu=0.8, M=4.0, w0=0.25 * h, dt=0.1)
    fl.assemble(par, dn, dp, pn)
    k = torch.as_tensor(np.exp(rng.uniform(np.log(1e-2), np.log(1e1), size=el.N)) / h, device=dev)
    # a consistent right-hand side b = J x* with x* ~ N(0, 1) in both blocks: unknowns of
    # order one, as the paper's scaling of unknowns makes them (Sec. 3.3.2); an N(0, 1)
    # b would call for pressures of order 1 / S~ ~ 1e7 and cancel seven digits in A11 x1
    xs = torch.as_tensor(rng.normal(size=3 * el.N + nn), device=dev)
    b = torch.empty_like(xs)
    fl.matvec(H, xs, b, k, shift=0.3 / h)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    res = {}
    for label, pc, meth in (("blockj_fgmres", "blockj", "fgmres"), ("ilu_bicgstab", "ilu", "bicgstab"),
                            ("jacobi3_bicgstab", "jacobi3", "bicgstab")):
        x = torch.zeros_like(b)
        inf = fl.solve(H, b, x, k, shift=0.3 / h, inner_precond=pc, inner_method=meth, ilu_p=0.01,
                       raise_on_error=False)
        times = []
        for _ in range(2):
            x.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            inf = fl.solve(H, b, x, k, shift=0.3 / h, inner_precond=pc, inner_method=meth, ilu_p=0.01,
                           raise_on_error=False)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        res[label] = {**inf, "seconds": min(times),
                      "rel_error_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))}
    line = {"metric": "coupled hydro-mechanical Jacobian solve, time to 1e-8 (Sec. 3.3.1 P_up)", "unit": "s",
            "value": min(r["seconds"] for r in res.values()), "n_gpus": 1, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 Krylov; f32 H-matrix",
            "data": "synthetic (seeded state, right-hand side)",
            "config": {"workload": "disk fault 256x256: N=51468 elements (154,404 DD) + %d pressure nodes" % nn,
                       "setup_s": setup}, "results": res}
    print(json.dumps(line), flush=True)


def run_triangles(args, dev, torch, hmat, synth):
    """The paper's element: a triangulated disk fault of 50,880 triangles (a 180 x 180
    lattice with seeded vertex jitter of 0.2 h, cells with r < 1 split in two), leaf 64,
    eta 2, eps 1e-6, FP32 + BF16 factors: assembly time and blocks per second, the FP32
    product (F32 vectors) against the HBM peak, and GMRES time to 1e-8 under a uniform
    unit pressure (leaf block-Jacobi, plain FP64 and mixed BF16 + FP64 refinement) with
    the error of the opening against Sneddon's solution; and the coupled hydro-mechanical
    Jacobian solve on it with linear pressure on the triangles (the state and right-hand
    side recipe of the coupled workload, h = 2/180)."""
    import numpy as np
    el = synth.tri_disk_mesh(180)
    t0 = time.perf_counter()
    T = hmat.ClusterTree(el, 64, 2.0)
    H = hmat.HMatrix(T, el, 1.0, 0.25, 1e-6, "both")
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    info = H.info()
    B, B2, B1 = product_bytes(info, "f32")
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(synth.rhs_shear_plus_bump(el)).to(dev, torch.float32)
    y = torch.empty_like(x)
    for _ in range(5):
        H.matvec(x, y, stream)
    H.check(stream)
    steps = min(args.steps, 1000)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        H.matvec(x, y, stream)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    hbm, peak_kind = peaks()
    b = np.zeros((el.N, 3))
    b[:, 2] = -1.0
    bt = torch.as_tensor(b.ravel(), device=dev)
    k0 = torch.zeros(el.N, dtype=torch.float64, device=dev)
    gm = {}
    for mode in ("f64", "mixed"):
        xs = torch.zeros_like(bt)
        H.solve(bt, xs, k0, precond="blockj", mode=mode)
        times = []
        for _ in range(3):
            xs.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            inf = H.solve(bt, xs, k0, precond="blockj", mode=mode)[0]
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        r = np.linalg.norm(el.c, axis=1)
        nu = 0.25
        exact = 8.0 * (1.0 - nu * nu) / (np.pi * 1.0) * np.sqrt(np.maximum(1.0 - r * r, 0.0))
        opening = xs.cpu().numpy().reshape(-1, 3)[:, 2]
        gm[mode] = {"seconds": min(times), "iters": inf["iters"], "relres": inf["relres"],
                    "sneddon_rel_error": float(np.linalg.norm(opening - exact) / np.linalg.norm(exact))}
    conn, nn = synth.node_connectivity(el)
    h = 2.0 / 180
    fl = hmat.Flow(conn, nn, el.a, el.b, el.shape, el.tri)
    rng = np.random.default_rng(1609)
    fl.assemble(dict(mu=0.8, M=4.0, w0=0.25 * h, dt=0.1), torch.as_tensor(rng.uniform(0.0, 0.25 * h, el.N), device=dev),
                torch.as_tensor(rng.normal(size=nn) * 0.1, device=dev), torch.as_tensor(rng.normal(size=nn) * 0.1, device=dev))
    kc = torch.as_tensor(np.exp(rng.uniform(np.log(1e-2), np.log(1e1), size=el.N)) / h, device=dev)
    xstar = torch.as_tensor(rng.normal(size=3 * el.N + nn), device=dev)
    bc = torch.empty_like(xstar)
    fl.matvec(H, xstar, bc, kc, shift=0.3 / h)
    xc = torch.zeros_like(bc)
    fl.solve(H, bc, xc, kc, shift=0.3 / h, raise_on_error=False)
    ct = []
    for _ in range(2):
        xc.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        cinf = fl.solve(H, bc, xc, kc, shift=0.3 / h, raise_on_error=False)
        torch.cuda.synchronize()
        ct.append(time.perf_counter() - t1)
    coupled = {**cinf, "seconds": min(ct), "pressure_nodes": nn,
               "rel_error_vs_xstar": float(torch.linalg.norm(xc - xstar) / torch.linalg.norm(xstar))}
    line = {"metric": "H-matrix product of triangular elements, effective HBM bandwidth", "unit": "GB/s",
            "value": B / (ms * 1e-3) / 1e9, "ms_per_product": ms, "n_gpus": 1, "steps": steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 factors, f32 vectors", "data": "synthetic (seeded triangulation)",
            "config": {"workload": "triangulated disk fault 180x180 lattice: N=%d triangles" % el.N,
                       "setup_s": setup, "stored_bytes": B, "algorithmic_bytes_per_product": B,
                       "hbm_peak_gbs": hbm, "peak_source": peak_kind},
            "frac_of_hbm": B / (ms * 1e-3) / 1e9 / hbm, "gmres_uniform_pressure": gm, "coupled_solve": coupled,
            "assembly": {"seconds": info["assemble_seconds"], "coeff_blocks": info["coeff_blocks"],
                         "blocks_per_s": info["coeff_blocks"] / info["assemble_seconds"],
                         "rank_mean": info["rank_mean"], "rank_max": info["rank_max"]}}
    print(json.dumps(line), flush=True)


def max_over_ranks(dist, value, device):
    """The largest of the ranks' values (each rank passes its own; None: one process)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world, bytes_per_product, seconds):
    """Whole-job rate of `world` replicas that each stream bytes_per_product in
    `seconds` (the slowest rank's time)."""
    return world * bytes_per_product / seconds / 1e9


def cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm: dense FP64 rows of E times x, row-sampled."""
    if rank != 0:
        return
    from oracle import build as oracle_build
    oracle_build.build()  # the oracle only: this arm loads nothing of the CUDA library
    from paper_2605_14397_gb300 import synth
    el = synth.config_fault(256)
    import numpy as np
    from oracle import oracle as O
    x = synth.rhs_shear_plus_bump(el)
    rng = np.random.default_rng(1603)
    # calibrate so the whole run stays within about two minutes
    probe = np.sort(rng.choice(el.N, size=8, replace=False))
    t0 = time.perf_counter()
    O.dense_matvec_rows(el, 1.0, 0.25, x, probe)
    per_row = (time.perf_counter() - t0) / 8
    rows_per_step = int(max(1, min(256, 100.0 / max(per_row * (args.steps + args.warmup), 1e-9))))
    for _ in range(args.warmup):
        O.dense_matvec_rows(el, 1.0, 0.25, x, np.sort(rng.choice(el.N, size=rows_per_step, replace=False)))
    times = []
    for _ in range(args.steps):
        rows = np.sort(rng.choice(el.N, size=rows_per_step, replace=False))
        t0 = time.perf_counter()
        O.dense_matvec_rows(el, 1.0, 0.25, x, rows)
        times.append(time.perf_counter() - t0)
    t_step = sum(times) / len(times)
    # same metric: the H-matrix product's algorithmic bytes per full product
    n = 3 * el.N
    ref_bytes = _reference_bytes()
    full = t_step * el.N / rows_per_step
    val = ref_bytes / full / 1e9
    sample = "%d seeded receiver rows x %d source elements per step (dense FP64 rows of E times x)" % (
        rows_per_step, el.N)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nrhs": 1, "storage": "dense FP64 (oracle)"},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


OPERATOR_RECORD = os.path.join(ROOT, "profiles", "operator_fault256.json")


def _reference_bytes():
    """Algorithmic bytes of one FP32 H-matrix product of this workload (leaf 64, eta 2,
    eps 1e-6) as recorded from an assembly by the GPU arm (profiles/operator_fault256.json),
    so that the oracle's throughput is stated in the same unit."""
    with open(OPERATOR_RECORD) as f:
        return int(json.load(f)["algorithmic_bytes_per_product"])


def record_operator(info, B, out_dir):
    """Write the assembled operator's sizes for the reference arm's unit."""
    rec = {"workload": WORKLOAD, "algorithmic_bytes_per_product": int(B), "stored_bytes": int(info["stored_bytes"]),
           "near_entries": int(info["near_entries"]), "u_entries": int(info["u_entries"]),
           "v_entries": int(info["v_entries"]), "rank_mean": info["rank_mean"], "rank_max": info["rank_max"],
           "recorded": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    os.makedirs(out_dir, exist_ok=True)
    with open(os.path.join(out_dir, "operator_fault256.json"), "w") as f:
        json.dump(rec, f, indent=1)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    from __graft_entry__ import build
    build()
    from paper_2605_14397_gb300 import hmat, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.workload == "faults64":
        run_faults64(args, dev, torch, hmat, synth)
        return
    if args.workload == "planes":
        run_planes(args, dev, torch, hmat, synth)
        return
    if args.workload == "learned":
        run_learned(args, dev, torch, hmat, synth)
        return
    if args.workload == "ilu":
        run_ilu(args, dev, torch, hmat, synth)
        return
    if args.workload == "interface":
        run_interface(args, dev, torch, hmat, synth)
        return
    if args.workload == "coupled":
        run_coupled(args, dev, torch, hmat, synth)
        return
    if args.workload == "triangles":
        run_triangles(args, dev, torch, hmat, synth)
        return
    el = synth.config_fault(args.grid)
    E, nu, eps = 1.0, 0.25, 1e-6
    t0 = time.perf_counter()
    T = hmat.ClusterTree(el, 64, 2.0)
    # FP32 and BF16 copies of the factors: the product times the FP32 ones (or the BF16
    # ones with --storage bf16), the mixed-precision solver needs both
    H = hmat.HMatrix(T, el, E, nu, eps, "both" if (args.storage == "f32" and not args.no_gmres) else args.storage)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    info = H.info()
    B, B2, B1 = product_bytes(info, args.storage)

    x = torch.from_numpy(synth.rhs_shear_plus_bump(el)).to(dev, torch.float32)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        H.matvec(x, y, stream)
    H.check(stream)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        H.matvec(x, y, stream)
    ev1.record(stream)
    ev1.synchronize()
    clocks = sampler.stop()
    # per-phase times from a separate run: the events recorded between the kernels would
    # otherwise sit inside the timed products
    H.timing(True)
    for _ in range(min(args.steps, 200)):
        H.matvec(x, y, stream)
    H.timing(False)
    ph = H.timing_read()
    H.check(stream)
    barrier()
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1) / args.steps, dev)
    value = whole_job_gbs(world, B, ms * 1e-3)
    hbm, peak_kind = peaks()
    cnt = max(ph["count"], 1)
    t2 = ph["phase2"] / cnt * 1e-3
    t1 = ph["phase1"] / cnt * 1e-3
    ach = B2 / t2 / 1e9
    roofline = {"bound": "hbm", "kernel": "k_phase2 ([D|U] z per row leaf)", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "peak_source": peak_kind,
                "traffic": recorded_traffic("k_phase2"),
                "algorithmic_bytes_per_launch": B2, "launch_ms": t2 * 1e3,
                "phases_ms": {k: ph[k] / cnt for k in ("gather", "phase1", "reduce", "phase2", "scatter")},
                "phase1_GBs": B1 / t1 / 1e9 if t1 > 0 else None}

    # the compensated product (FP64 vectors, the same FP32 factors): the operator of the
    # plain FP64 solver, accurate to the ACA tolerance whatever the cancellation in E x
    x64 = torch.from_numpy(synth.rhs_shear_plus_bump(el)).to(dev)
    y64 = torch.empty_like(x64)
    for _ in range(5):
        H.matvec(x64, y64, stream)
    k64 = min(args.steps, 500)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k64):
        H.matvec(x64, y64, stream)
    e1.record(stream)
    e1.synchronize()
    ms64 = e0.elapsed_time(e1) / k64
    B64 = B + 2 * 4 * info["n_dof"]  # x and y are 8 bytes per entry
    f64_vectors = {"ms_per_product": ms64, "GBs": B64 / (ms64 * 1e-3) / 1e9, "bytes_per_product": B64,
                   "frac_of_hbm_peak": B64 / (ms64 * 1e-3) / 1e9 / peaks()[0]}

    # end to end through the host-vector entry point
    xh = torch.from_numpy(synth.rhs_shear_plus_bump(el).astype(np.float32)).pin_memory().numpy()
    yh = torch.empty(xh.shape, dtype=torch.float32).pin_memory().numpy()
    ke = min(args.steps, 200)
    for _ in range(3):
        H.matvec_host(xh, yh, stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        H.matvec_host(xh, yh, stream)
    te = max_over_ranks(dist, (time.perf_counter() - t0) / ke, dev)
    e2e = {"value": whole_job_gbs(world, B, te), "unit": "GB/s", "h2d_bytes_per_step": int(xh.nbytes),
           "d2h_bytes_per_step": int(yh.nbytes), "ms_per_step": te * 1e3}

    gmres = None
    if not args.no_gmres and args.storage == "f32":
        gmres = time_gmres(H, el, dev, torch)

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else "bf16",
            "data": "synthetic (seeded mesh and right-hand side)",
            "config": {"workload": WORKLOAD if args.grid == 256 else "disk fault on %dx%d grid: N=%d" % (
                           args.grid, args.grid, el.N), "nrhs": 1, "storage": args.storage,
                       "trunc_factor": "library default (30: blocks recompressed to 15 eps relative)",
                       "stored_bytes": info["stored_bytes"], "ms_per_product": ms,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "operator 4.3 GB >> 129 MB L2: inputs larger than L2, no flush",
                       "setup_s": t_setup, "assemble_s": info["assemble_seconds"],
                       "assemble_pairs_per_s": info["coeff_blocks"] / info["assemble_seconds"],
                       "assemble_coeff_blocks": info["coeff_blocks"],
                       "rank_mean": info["rank_mean"], "rank_max": info["rank_max"],
                       "bytes_per_product": B, "frac_of_hbm_peak": value / world / hbm},
            "roofline": roofline, "e2e": e2e, "gpu_launches": 5 * args.steps, "clocks": clocks,
            "f64_vectors_compensated": f64_vectors}
    if gmres is not None:
        line["gmres"] = gmres
    if args.tune:
        line["autotune"] = hmat.autotune(el, E, nu, eps, "f32", leaves=(32, 48, 64, 96, 128), etas=(1.5, 2.0, 3.0),
                                         budget_ms=180000)

    if rank == 0 and args.record_dir and args.grid == 256 and args.storage == "f32":
        os.makedirs(args.record_dir, exist_ok=True)
        record_operator(info, B, args.record_dir)
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, rows, dt = oracle_rows_rate(el, E, nu)
        full = el.N / rate
        line["cpu_baseline"] = {"value": B / full / 1e9, "unit": "GB/s", "cores": cores(), "kind": "oracle",
                                "sample": "%d seeded receiver rows of the dense FP64 product (%.1f s), "
                                          "extrapolated to a full product (%.1f s)" % (rows, dt, full)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
