#!/usr/bin/env python
"""Throughput of the steady-state crossbar solve on one GB300.

Workload: the 1024 x 1024 memristor crossbar (2.1M unknowns), log-uniform device
conductances in [1e-6, 1e-4] S, top wires 1 S, bottom wires 0.5 S, 10 ohm drivers and
sense, 1 kohm terminations, sinh devices (b = 2), V_in ~ U[0, 0.3] V.  One step solves
--handles handles of --batch input vectors each, concurrently (mca_solve_many, one host
thread and stream per handle), to a relative KCL residual ||F||/||Y|| <= 1e-8 with Newton +
flexible GMRES(30) preconditioned by the Kronecker/block preconditioner (tensor-core BF16
transforms, split back transforms); value = solves per second.

The JSON line also carries: the end-to-end figure through the C ABI with host buffers,
the roofline of the dominant kernel family (CUDA events on the solve stream, in a pass of
one handle alone), the same workload in the two all-FP64 GPU forms (the exact eigenbasis
preconditioner with FP64 transforms, and the paper's M_hat applied by tridiagonal solves)
at the same batching, the 2048 x 2048 crossbar with an oracle-recomputed residual, the
preconditioner TFLOP/s (dense eigenbasis count 8 m n (m + n) per apply), the batched
statistical-characterisation workload, and the CPU oracle on the host cores (the 1024^2
workload, plus the 32^2 and 256^2 configurations single-threaded and on all cores).

--impl reference times the CPU oracle itself on the same workload (the reference arm).
--profile-precond applies the preconditioner alone (for ncu captures of its GEMMs).
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import mca_inputs as mi  # noqa: E402

METRIC = "solves/s at 1e-8 rel. KCL residual (1024² MCA) vs plain FP64; precond TFLOP/s"
TOL = 1e-8


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=64, help="vectors per handle pass (<= 64)")
    ap.add_argument("--handles", type=int, default=2,
                    help="handles solved concurrently per step (mca_solve_many, one host "
                         "thread and stream each)")
    ap.add_argument("--precision", default="bf16split",
                    choices=["bf16split", "bf16", "fp64", "mhat"])
    ap.add_argument("--device", default="sinh", choices=["sinh", "yakopcic"],
                    help="memristor I-V law; yakopcic: a2/a1 = --neg-ratio below zero, "
                         "inputs of both signs")
    ap.add_argument("--neg-ratio", type=float, default=0.5)
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-2048", action="store_true", help="skip the 2048^2 leg")
    ap.add_argument("--restart", type=int, default=30, help="GMRES restart length")
    ap.add_argument("--profile-precond", type=int, default=0, metavar="REPS",
                    help="only apply the preconditioner REPS times to --batch random vectors "
                         "of a --size^2 handle (between cudaProfilerStart/Stop)")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="(internal) time the oracle on the 32^2 and 256^2 configurations "
                         "and print one JSON line; bench.py runs it in child processes")
    ap.add_argument("--batch-profile", choices=["c4", "small"], default=None,
                    help="only the persistent batched launch on the statistical mix (c4) "
                         "or its {64,128} subset (small), with per-phase timers")
    ap.add_argument("--e2e-breakdown", action="store_true",
                    help="only time one end-to-end call of the headline workload with device "
                         "or host buffers, one or two passes per handle, with and without "
                         "the voltage outputs, and the output copies alone")
    ap.add_argument("--table1", action="store_true",
                    help="GPU version of the paper's Table 1 (GMRES steps per preconditioner)")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        if shutil.which("nvidia-smi") is None:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(
            ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
             "-lms", "200", "-i", str(self.gpu)], stdout=self.fh, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                     hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        sm = sorted(r["sm"] for r in rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0]["smax"],
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def job_time(t, pg):
    """Elapsed time of the whole job: the maximum of the ranks' times (replicas run
    independently; the slowest one ends the job).  No collective without a process group."""
    if not pg:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64)
    pg.all_reduce(tt, op=pg.ReduceOp.MAX)
    return float(tt[0])


def replica_seeds(rank):
    """Each rank solves its own crossbars (no data is shared between ranks): rank r takes
    the four crossbars of seeds 4r .. 4r + 3 (rank 0: seeds 0-3, the 1024^2 workload's)."""
    return tuple(range(4 * rank, 4 * rank + 4))


def oracle_solves(ws, count, start=0, tol=TOL):
    """Time `count` oracle solves (Newton + preconditioned GMRES, FP64, NumPy/SciPy) of
    the workload's vectors start, start + 1, ... (each on its own crossbar's map)."""
    from oracle import mca_oracle as O
    t0 = time.perf_counter()
    for v in range(start, start + count):
        v %= len(ws.vin)
        r = O.newton_solve(ws.params, ws.gmaps[ws.map_index[v]], ws.vin[v], tol=tol,
                           linear="pgmres")
        assert r.rel_residual <= tol
    return time.perf_counter() - t0


def secondary_leg(out, key, fn):
    """out[key] = fn() for a figure reported beside the headline (the all-FP64 forms, the
    2048^2 leg, the batched workload, extra oracle timings).  An exception there is recorded
    as out[key] = {"error": ...} instead of ending the run, so the line with the headline,
    which is complete by then, is still printed."""
    try:
        out[key] = fn()
    except Exception as e:  # noqa: BLE001 - any failure of a side figure is reported in-line
        out[key] = {"error": f"{type(e).__name__}: {e}"[:400]}


def oracle_once(size, seed=0):
    """Seconds of one oracle solve (Newton + FP64 preconditioned GMRES, NumPy/SciPy, BLAS on
    every core) of the size^2 crossbar of seed `seed` with the workload's wiring, input
    vector 0."""
    from oracle import mca_oracle as O
    ws = mi.config_large_set(size, seeds=(seed,), nvec=1)
    t0 = time.perf_counter()
    r = O.newton_solve(ws.params, ws.gmaps[0], ws.vin[0], tol=TOL, linear="pgmres")
    t = time.perf_counter() - t0
    assert r.rel_residual <= TOL
    return t


def workload_config(args, batch):
    dev = ("sinh devices b=2, V_in~U[0,0.3] V" if getattr(args, "device", "sinh") == "sinh" else
           f"Yakopcic-form devices b=2 a2/a1={args.neg_ratio:g}, V_in~U[-0.3,0.3] V")
    return {
        "workload": f"{args.size}x{args.size} MCA, log-uniform g in [1e-6,1e-4] S "
                    f"(crossbar seeds 0-3, vectors interleaved over them), wires "
                    f"1 S top / 0.5 S bottom, {dev}, "
                    f"Newton to {TOL:g} rel. KCL residual, FGMRES({args.restart})",
        "rows": args.size, "cols": args.size, "batch_per_step": batch,
        "precision": args.precision, "newton_rtol": TOL,
        "cache": "inputs larger than L2: the Krylov basis of one solve is ~1 GB",
    }


def step_config(args):
    """The `config` both arms print: one step solves --handles x --batch vectors of the
    workload (the reference arm times a bounded sample of that step's solves)."""
    H, B = max(1, args.handles), args.batch
    return dict(workload_config(args, H * B), handles=H, batch_per_handle=B,
                profile_pass="kernel_breakdown and roofline: one handle alone")


def make_workload(args, rank, nvec):
    """The timed crossbars: four log-uniform crossbars with sinh devices and V_in >= 0
    (seeds 4r .. 4r + 3), or one Yakopcic-form crossbar (a2/a1 = --neg-ratio) with inputs
    of both signs."""
    if getattr(args, "device", "sinh") == "sinh":
        return mi.config_large_set(args.size, seeds=replica_seeds(rank), nvec=nvec)
    cb = mi.make_crossbar(args.size, args.size, replica_seeds(rank)[0], nvec=nvec,
                          g_wire_bot=0.5, vmin=-0.3, neg_ratio=args.neg_ratio)
    return mi.CrossbarSet(params=cb.params, gmaps=cb.gmap[None], vin=cb.vin,
                          map_index=np.zeros(nvec, np.int32), seeds=(cb.seed,))


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    ws = make_workload(args, 0, args.warmup + args.steps)
    oracle_solves(ws, args.warmup)
    t = oracle_solves(ws, args.steps, start=args.warmup)
    value = args.steps / t
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(args),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle solves of the {args.size}^2 crossbars, "
                                   "one input vector each (one solve per step out of the "
                                   "step's handles x batch)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def params_for(mca, p, prec, B, restart=30, tol=TOL, device_model=None):
    """Library parameters of a workload's wiring at one precision and batch."""
    return mca.default_params(p.rows, p.cols, g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot,
                              g_src=p.g_src, g_term_top_right=p.g_term_top_right,
                              g_term_bot_top=p.g_term_bot_top, g_sense=p.g_sense, b=p.b,
                              precision=prec, newton_rtol=tol, max_batch=B,
                              gmres_restart=restart,
                              device_model=(mca.DEVICE_SINH if device_model is None
                                            else device_model),
                              neg_ratio=p.neg_ratio)


def solve_step(mca, solvers, vin_d, map_d, first, outs, check=None):
    """One step: handle h solves vectors first + h*B .. first + (h+1)*B (each with its
    crossbar's map), all handles concurrently through mca_solve_many (which returns when
    every handle is done).  Every solve must reach the tolerance."""
    B = outs[0][0].shape[0]
    nv = vin_d.shape[0]
    vins, maps = [], []
    for h in range(len(solvers)):
        a = (first + h * B) % nv
        if a + B <= nv:             # a view: no copy inside a timed step
            vins.append(vin_d[a:a + B])
            maps.append(map_d[a:a + B])
        else:
            idx = [(a + j) % nv for j in range(B)]
            vins.append(vin_d[idx])
            maps.append(map_d[idx])
    res = mca.solve_many(solvers, vins, map_indices=maps, n_threads=len(solvers), outs=outs)
    for r in res:
        for st in r[3]:
            assert st["status"] == 0 and st["rel_residual"] <= TOL, st
            if check is not None:
                check.append((st["newton_iters"], st["gmres_iters"], st["rel_residual"]))
    return res


def time_form(mca, torch, ws, prec, H, B, steps, first, restart=30, device_model=None,
              grab=None):
    """Solves/s of the workload in another preconditioner form: H handles of B vectors,
    one untimed step, then `steps` timed steps (CUDA events around the synchronous
    mca_solve_many calls), device-resident inputs and outputs.  grab = j also returns the
    node voltages of vector j of the last step's first handle (host) and its index."""
    dev = torch.device("cuda", torch.cuda.current_device())
    params = params_for(mca, ws.params, prec, B, restart, device_model=device_model)
    solvers = [mca.Solver(params, ws.gmaps) for _ in range(H)]
    try:
        m, n = ws.params.rows, ws.params.cols
        vin_d = torch.as_tensor(ws.vin, device=dev)
        outs = [(torch.empty(B, m, n, dtype=torch.float64, device=dev),
                 torch.empty(B, m, n, dtype=torch.float64, device=dev),
                 torch.empty(B, n, dtype=torch.float64, device=dev)) for _ in range(H)]
        solve_step(mca, solvers, vin_d, ws.map_index, first, outs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        chk = []
        e0.record()
        for i in range(steps):
            solve_step(mca, solvers, vin_d, ws.map_index, first + (i + 1) * H * B, outs, chk)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        it = np.array([(a, b_) for a, b_, _ in chk])
        got = None
        if grab is not None:
            v = (first + steps * H * B + grab) % vin_d.shape[0]
            got = (v, outs[0][0][grab].cpu().numpy(), outs[0][1][grab].cpu().numpy())
        return got, {"value": steps * H * B / t, "unit": "solves/s", "handles": H,
                "batch_per_handle": B, "solves": steps * H * B,
                "newton_iters_per_solve": float(it[:, 0].mean()),
                "gmres_iters_per_solve": float(it[:, 1].mean()),
                "max_rel_residual": float(max(r for _, _, r in chk))}
    finally:
        for s_ in solvers:
            s_.close()
        torch.cuda.empty_cache()


def run_2048(mca, torch, args, rank, B=16, steps=3):
    """The 2048 x 2048 crossbars (8.4M unknowns) in the headline's precision: one handle of
    B vectors over the four crossbars, and the oracle's FP64 KCL residual of one of the
    returned solutions."""
    from oracle import mca_oracle as O
    ws = mi.config_large_set(2048, seeds=replica_seeds(rank), nvec=(steps + 1) * B)
    (v, vt, vb), r = time_form(mca, torch, ws, mca.PREC_BF16_SPLIT, 1, B, steps, 0,
                               args.restart, grab=B - 1)
    # one solution of the last timed pass recomputed by the oracle
    g = ws.gmaps[ws.map_index[v]]
    Ft, Fb = O.residual(ws.params, g, ws.vin[v], vt.ravel(), vb.ravel())
    Yt, _ = O.source_vector(ws.params, ws.vin[v])
    rel = float(np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt))
    assert rel <= TOL * 1.01, rel
    r["oracle_rel_residual"] = rel
    r["oracle_checked_vector"] = int(v)
    r["workload"] = ("2048x2048 MCA, crossbar seeds 0-3, same wiring, devices and precision "
                     "as the headline")
    return r


def oracle_configs():
    """Oracle timings on the two small configurations, in this process' BLAS threading:
    32^2 (seed 0, Newton to 1e-10) with the banded direct solve and with preconditioned
    GMRES, each repeated for about a second; 256^2 bimodal (seeds 0-7, one vector each,
    Newton to 1e-8) with preconditioned GMRES on every seed and the banded solve on seed 0
    (about 10 s per solve: the LAPACK band LU of a 131k x 131k matrix of bandwidth 512)."""
    from oracle import mca_oracle as O
    out = {}

    def rate(fn, min_s=1.0):
        k, t = 0, 0.0
        while t < min_s or k == 0:
            a = time.perf_counter()
            fn()
            t += time.perf_counter() - a
            k += 1
        return {"value": k / t, "unit": "solves/s", "solves": k, "seconds": t}

    c1 = mi.config_small(0)
    for lin in ("banded", "pgmres"):
        out[f"c1_32_{lin}"] = rate(lambda: O.newton_solve(c1.params, c1.gmap, c1.vin[0],
                                                          tol=1e-10, linear=lin))
    c2 = [mi.config_bimodal(sd) for sd in range(8)]
    a = time.perf_counter()
    for cb in c2:
        r = O.newton_solve(cb.params, cb.gmap, cb.vin[0], tol=TOL, linear="pgmres")
        assert r.rel_residual <= TOL
    t = time.perf_counter() - a
    out["c2_256_pgmres"] = {"value": 8 / t, "unit": "solves/s", "solves": 8, "seconds": t,
                            "seeds": "0-7"}
    a = time.perf_counter()
    r = O.newton_solve(c2[0].params, c2[0].gmap, c2[0].vin[0], tol=TOL, linear="banded")
    t = time.perf_counter() - a
    assert r.rel_residual <= TOL
    out["c2_256_banded"] = {"value": 1 / t, "unit": "solves/s", "solves": 1, "seconds": t,
                            "seeds": "0"}
    return out


def oracle_configs_in_children():
    """oracle_configs() in two child processes: BLAS limited to one thread, and BLAS on
    every core (the children import no CUDA)."""
    res = {}
    for name, threads in (("single_thread", 1), ("all_cores", os.cpu_count())):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-configs"],
                           env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            res[name] = {"error": r.stderr[-300:]}
            continue
        res[name] = dict(json.loads(r.stdout.strip().splitlines()[-1]), threads=threads)
    return res


def run_profile_precond(args):
    """Apply the preconditioner alone, for ncu captures of its GEMMs: a --size^2 handle
    with max_batch --batch and restart --restart (the tile autotuner runs at create), then
    --profile-precond applies to --batch random vectors between cudaProfilerStart/Stop."""
    import torch
    import paper_2109_07929_gb300 as mca
    prec = {"bf16split": mca.PREC_BF16_SPLIT, "bf16": mca.PREC_BF16}[args.precision]
    ws = mi.config_large_set(args.size, nvec=args.batch)
    B, m, n = args.batch, args.size, args.size
    with mca.Solver(params_for(mca, ws.params, prec, B, args.restart), ws.gmaps) as s:
        r = torch.as_tensor(np.random.default_rng(0).standard_normal((B, 2 * m * n)),
                            device="cuda")
        z = torch.empty_like(r)
        a = np.full(B, 2e-5)
        s.precond_apply(a, r, z)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        for _ in range(args.profile_precond):
            s.precond_apply(a, r, z)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profile_precond": args.profile_precond, "batch": B, "size": m,
                          "tiles": gemm_tiles(s)}), flush=True)


def run_ours(args):
    import torch
    import paper_2109_07929_gb300 as mca

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    prec = {"bf16split": mca.PREC_BF16_SPLIT, "bf16": mca.PREC_BF16,
            "fp64": mca.PREC_FP64, "mhat": mca.PREC_MHAT}[args.precision]
    B = args.batch
    H = max(1, args.handles)
    S = H * B                       # solves per step
    W, K = args.warmup, args.steps
    m = n = args.size
    ws = make_workload(args, rank, (W + max(K, 2 * E2E_PASSES)) * S)
    p = ws.params
    params = params_for(mca, p, prec, B, args.restart,
                        device_model=(mca.DEVICE_SINH if args.device == "sinh"
                                      else mca.DEVICE_YAKOPCIC))
    solvers = [mca.Solver(params, ws.gmaps) for _ in range(H)]
    solver = solvers[0]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    vin = torch.as_tensor(ws.vin, device=dev)
    outs = [(torch.empty(B, m, n, dtype=torch.float64, device=dev),
             torch.empty(B, m, n, dtype=torch.float64, device=dev),
             torch.empty(B, n, dtype=torch.float64, device=dev)) for _ in range(H)]

    def step(i, check):
        # one step: H handles of B vectors each, solved concurrently
        solve_step(mca, solvers, vin, ws.map_index, i * S, outs, check)

    warm = []
    for i in range(W):
        step(i, warm)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = mca.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    timed = []
    for i in range(W, W + K):
        step(i, timed)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = mca.kernel_launches() - launches0
    clocks = sampler.stop()
    t = job_time(ev0.elapsed_time(ev1) / 1000.0, pg)
    if pg:
        pg.barrier()
    value = world * K * S / t

    # ---- end to end through the C ABI with host buffers (pinned), copies included.  One
    # call gives each handle P passes of B vectors: the library runs them as passes of B and
    # overlaps each pass' device->host output copies with the next pass' kernels.
    P = max(2, min(E2E_PASSES, E2E_SOLVES // S))
    vin_h = torch.as_tensor(ws.vin).pin_memory()
    outs_h = [(torch.empty(P * B, m, n, dtype=torch.float64).pin_memory(),
               torch.empty(P * B, m, n, dtype=torch.float64).pin_memory(),
               torch.empty(P * B, n, dtype=torch.float64).pin_memory()) for _ in range(H)]

    def step_host(i):
        base = i * S
        vins = [vin_h[base + h * P * B:base + (h + 1) * P * B] for h in range(H)]
        maps = [ws.map_index[base + h * P * B:base + (h + 1) * P * B] for h in range(H)]
        for r in mca.solve_many(solvers, vins, map_indices=maps, n_threads=H, outs=outs_h):
            for st_ in r[3]:
                assert st_["status"] == 0 and st_["rel_residual"] <= TOL, st_

    step_host(0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ke = max(1, K // (2 * P))
    call_ms = []
    e0.record(stream)
    for i in range(ke):
        c0 = time.perf_counter()
        step_host(W + i * P)
        call_ms.append(round(1e3 * (time.perf_counter() - c0), 1))
    e1.record(stream)
    torch.cuda.synchronize()
    te = job_time(e0.elapsed_time(e1) / 1000.0, pg)
    e2e = {"value": world * ke * P * S / te, "unit": "solves/s",
           "h2d_bytes_per_step": P * S * (m * 8 + 4),
           "d2h_bytes_per_step": P * S * (2 * m * n + n) * 8 + P * S * mca.ctypes.sizeof(mca.Stats),
           "solves_per_call": P * S, "calls": ke, "call_ms": call_ms,
           "d2h_gbs_of_this_host": d2h_rate(torch, dev)}

    # ---- per-family kernel timing (CUDA events on the solve stream, separate pass of one
    # handle alone: the concurrent handles' kernels overlap, which per-launch events cannot
    # apportion)
    st1 = (mca.Stats * B)()
    sp1 = mca.ctypes.cast(st1, mca.ctypes.c_void_p)
    vt, vb, io = outs[0]
    solver.profile(True)
    for i in range(W, W + min(K, 4)):
        mi_ = np.ascontiguousarray(ws.map_index[i * S:i * S + B])
        rc = solver.solve_multi_raw(vin[i * S:i * S + B].data_ptr(), mi_.ctypes.data, B,
                                    vt.data_ptr(), vb.data_ptr(), io.data_ptr(), sp1, stream)
        if rc != 0:
            raise RuntimeError(f"solve failed with status {rc}")
    prof = solver.profile_read()
    solver.profile(False)
    peaks, peak_src = load_peaks()
    fam = max(prof, key=lambda f: prof[f]["ms"])
    fp = prof[fam]
    gemm = fam.startswith("precond")
    tc = prec in (mca.PREC_BF16, mca.PREC_BF16_SPLIT)
    if gemm and tc:
        ach = fp["flops"] / (fp["ms"] / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s"}
    else:
        # FP64 kernels: the binding one of the HBM and the FP64-ALU rooflines
        gbs = fp["bytes"] / (fp["ms"] / 1e3) / 1e9
        tfs = fp["flops"] / (fp["ms"] / 1e3) / 1e12
        if gbs / peaks["hbm_gbs"] >= tfs / FP64_PEAK_TFLOPS:
            roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
        else:
            roof = {"bound": "alu", "achieved": tfs, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "hbm_frac": gbs / peaks["hbm_gbs"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = fam
    roof["launches"] = fp["launches"]
    roof["avg_launch_us"] = 1e3 * fp["ms"] / max(1, fp["launches"])
    roof["peak_source"] = {"tensor": f"{peak_src} sustained bf16", "hbm": f"{peak_src} hbm",
                           "alu": "FP64 DFMA: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz"}[roof["bound"]]
    roof["traffic"] = committed_traffic(fam, fp)
    total_ms = sum(v["ms"] for v in prof.values())
    breakdown = {f: {"share": v["ms"] / total_ms, "launches": v["launches"],
                     "GB/s": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else 0.0,
                     "TFLOP/s": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["ms"] > 0 else 0.0}
                 for f, v in prof.items() if v["launches"] > 0}
    # both ceilings of every CUDA-core family: algorithmic bytes against the measured HBM
    # copy rate, algorithmic FP64 flops against the FP64 pipe (152 SMs x 2 DFMA/clk x 2.07 GHz)
    for f, b in breakdown.items():
        if not f.startswith("precond"):
            b["hbm_frac"] = b["GB/s"] / peaks["hbm_gbs"]
            b["fp64_frac"] = b["TFLOP/s"] / FP64_PEAK_TFLOPS
    # precond TFLOP/s in the dense eigenbasis count, 8 m n (m + n) per apply
    pc_ms = sum(prof[f]["ms"] for f in ("precond_1", "precond_2", "precond_3", "precond_4"))
    applies = prof["precond_1"]["flops"] / (4.0 * m * n * n) if prof["precond_1"]["flops"] else 0
    precond_tflops = (applies * 8.0 * m * n * (m + n) / (pc_ms / 1e3) / 1e12
                      if pc_ms and prec != mca.PREC_MHAT else None)
    precond_frac = None
    if precond_tflops:
        precond_frac = {"of_sustained": precond_tflops / peaks.get("bf16_tflops_sustained", 1700.0),
                        "of_burst": precond_tflops / peaks.get("bf16_tflops", 1900.0),
                        "peak_source": peak_src}

    iters = np.array([(a, b_) for a, b_, _ in timed])
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": 1000 * t / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+bf16" if prec in (mca.PREC_BF16, mca.PREC_BF16_SPLIT) else "f64",
        "data": "synthetic",
        "config": step_config(args),
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
        "precond_tflops": precond_tflops, "precond_frac": precond_frac,
        "kernel_breakdown": breakdown,
        # summed device time of the timed kernels per step (profile pass) over the timed
        # step: what is left is host-side gaps (Newton checks, graph launches)
        "kernel_ms_per_step": total_ms / min(K, 4) * H,
        "gpu_busy_frac": (total_ms / min(K, 4) * H) / (1000 * t / K),
        "gemm_tiles": gemm_tiles(solver),
        "newton_iters_per_solve": float(iters[:, 0].mean()),
        "gmres_iters_per_solve": float(iters[:, 1].mean()),
        "max_rel_residual": float(max(r for _, _, r in timed)),
    }
    for s_ in solvers:
        s_.close()
    del vt, vb, io, outs, outs_h
    torch.cuda.empty_cache()

    # ---- the same workload in the all-FP64 GPU forms, at the headline's batching where it
    # is affordable: the exact eigenbasis preconditioner with FP64 transforms (CUDA-core
    # FP64 GEMMs; one handle of B vectors) and the paper's M_hat (eq. (block) with
    # tridiagonal solves; H handles of B vectors, as the headline)
    if not args.no_fp64_form and prec not in (mca.PREC_FP64, mca.PREC_MHAT):
        def fp64_forms():
            _, f64 = time_form(mca, torch, ws, mca.PREC_FP64, 1, B, 1, 0, args.restart,
                               params.device_model)
            _, mh = time_form(mca, torch, ws, mca.PREC_MHAT, H, B, 2, 0, args.restart,
                              params.device_model)
            out["fp64_form"] = f64
            out["mhat_form"] = mh
            best = max(f64["value"], mh["value"])
            return {"value": value / best,
                    "against": "mhat_form" if mh["value"] >= f64["value"] else "fp64_form",
                    "note": "device solves/s of the headline over the faster all-FP64 GPU "
                            "form"}
        secondary_leg(out, "speedup_of_mixed", fp64_forms)

    # ---- 2048 x 2048 crossbars, with an oracle-recomputed residual
    if not args.no_2048 and args.size == 1024 and prec == mca.PREC_BF16_SPLIT:
        secondary_leg(out, "size_2048", lambda: run_2048(mca, torch, args, rank))

    # ---- the batched statistical-characterisation workload (secondary figure)
    if not args.no_batched and args.size == 1024:
        secondary_leg(out, "batched_c4", lambda: run_batched_c4(mca, torch))

    # ---- CPU oracle on the host cores (rank 0, one GPU only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a bounded sample: whole oracle solves until about 10 s of CPU work (at most 25)
        ncpu, tcpu = 0, 0.0
        while ncpu < 25 and (ncpu == 0 or tcpu < 10.0):
            tcpu += oracle_solves(ws, 1, start=ncpu)
            ncpu += 1
        out["cpu_baseline"] = {"value": ncpu / tcpu, "unit": "solves/s", "cores": os.cpu_count(),
                               "kind": "oracle",
                               "sample": f"{ncpu} oracle solves (Newton + FP64 preconditioned "
                                         f"GMRES, NumPy/SciPy) of the {m}^2 workload, vectors "
                                         f"0-{ncpu - 1} (crossbars 0-3), {tcpu:.1f} s",
                               "configs": oracle_configs_in_children()}
        if not args.no_2048 and args.size == 1024:
            def oracle_2048():
                t2 = oracle_once(2048)
                return {"value": 1.0 / t2, "unit": "solves/s", "solves": 1, "seconds": t2,
                        "seeds": "0", "threads": os.cpu_count()}
            secondary_leg(out["cpu_baseline"], "c3_2048_pgmres", oracle_2048)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


def batch_workload(mca, torch, cbs, nvec, restart=16):
    """Crossbars of one shape as one multi-map Solver each (max_batch: the group's vectors,
    at most 64), their input vectors and output buffers on the device, and the items of a
    persistent launch (one per crossbar and input vector)."""
    groups = {}
    for k, cb in enumerate(cbs):
        groups.setdefault((cb.params.rows, cb.params.cols), []).append(k)
    solvers, vins, maps = [], [], []
    for (m, n), ks in sorted(groups.items()):
        p = cbs[ks[0]].params
        B = min(64, len(ks) * nvec)   # one pass per shape group where it fits
        solvers.append(mca.Solver(params_for(mca, p, mca.PREC_BF16_SPLIT, B, restart=restart),
                                  np.stack([cbs[k].gmap for k in ks])))
        vins.append(np.concatenate([cbs[k].vin for k in ks]))
        maps.append(np.repeat(np.arange(len(ks)), nvec))
    dev = torch.device("cuda", torch.cuda.current_device())
    vins_d = [torch.as_tensor(v, device=dev) for v in vins]
    outs_d = [(torch.empty(v.shape[0], s.m, s.n, dtype=torch.float64, device=dev),
               torch.empty(v.shape[0], s.m, s.n, dtype=torch.float64, device=dev),
               torch.empty(v.shape[0], s.n, dtype=torch.float64, device=dev))
              for s, v in zip(solvers, vins)]
    hs, mp_, vi, vt, vb, io = [], [], [], [], [], []
    for k in range(len(solvers)):
        for r in range(vins_d[k].shape[0]):
            hs.append(k)
            mp_.append(int(maps[k][r]))
            vi.append(vins_d[k][r])
            vt.append(outs_d[k][0][r])
            vb.append(outs_d[k][1][r])
            io.append(outs_d[k][2][r])
    items = mca.Batch.items(hs, mp_, vi, vt, vb, io)
    return dict(groups=groups, solvers=solvers, maps=maps, vins=vins_d, outs=outs_d,
                items=items)


def run_batch_profile(args):
    """--batch-profile MIX: the persistent launch alone on the statistical mix (c4: 128
    crossbars from {64,128,256,512}; small: 32 crossbars from {64,128}; 16 input vectors
    each, restart 16, Newton to 1e-8): wall time of one launch (best of 3, after a warm-up),
    then one launch with the per-phase timers (CTA-milliseconds summed over the CTAs).  One
    JSON line."""
    import torch
    import paper_2109_07929_gb300 as mca
    torch.cuda.set_device(0)
    if args.batch_profile == "small":
        cbs = mi.config_batched(count=32, nvec=16, base_seed=5000, sizes=(64, 128))
    else:
        cbs = mi.config_batched(count=128, nvec=16)
    W = batch_workload(mca, torch, cbs, 16)
    try:
        with mca.Batch(W["solvers"]) as b:
            b.solve_items(W["items"])
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                st = b.solve_items(W["items"])
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            b.profile(True)
            b.solve_items(W["items"])
            torch.cuda.synchronize()
            prof = b.profile_read()
    finally:
        for s in W["solvers"]:
            s.close()
    tot = sum(prof.values())
    cells = sum(cb.params.rows * cb.params.cols for cb in cbs) * 16
    print(json.dumps({"batch_profile": args.batch_profile, "solves": len(st),
                      "cells_solved": cells, "ms": min(ts) * 1e3,
                      "solves_per_s": len(st) / min(ts),
                      "gmres_iters_per_solve": float(np.mean([x["gmres_iters"] for x in st])),
                      "max_rel_residual": max(x["rel_residual"] for x in st),
                      "phase_cta_ms": {k: round(v, 1) for k, v in prof.items()},
                      "phase_share": {k: round(v / tot, 4) for k, v in prof.items()}}))


def run_batched_c4(mca, torch, count=128, nvec=16, threads=4):
    """Statistical characterisation: `count` crossbars with rows/cols drawn from
    {64,128,256,512}, log-uniform g with lognormal 0.1 variation, `nvec` input vectors
    each, solved to 1e-8.  Crossbars of one shape share a multi-map handle (one
    eigenbasis).  The value is one persistent launch over all solves (mca_batch_solve:
    one (crossbar, vector) item per CTA at a time, largest first).  Compared with: the
    shape groups as batched passes run concurrently on `threads` streams with CUDA-graph
    replay and autotuned tiles (mca_solve_many), and one handle per crossbar solved one
    after the other.  Wall-clock time of the solves only (handles and the batch object
    are created beforehand)."""
    cbs = mi.config_batched(count=count, nvec=nvec)
    W = batch_workload(mca, torch, cbs, nvec)
    groups, solvers, maps, vins_d, outs_d = (W["groups"], W["solvers"], W["maps"], W["vins"],
                                              W["outs"])
    mca.solve_many(solvers, vins_d, map_indices=maps, n_threads=threads, outs=outs_d)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = mca.solve_many(solvers, vins_d, map_indices=maps, n_threads=threads, outs=outs_d)
    torch.cuda.synchronize()
    t_groups = time.perf_counter() - t0
    # one persistent launch over every (crossbar, vector) item
    with mca.Batch(solvers) as batch:
        items = W["items"]
        batch.solve_items(items)                                        # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = batch.solve_items(items)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        # one more launch with the per-phase timers (not timed)
        batch.profile(True)
        batch.solve_items(items)
        torch.cuda.synchronize()
        prof = batch.profile_read()
    ptot = sum(prof.values())
    worst = max(x["rel_residual"] for x in st)
    its = float(np.mean([x["gmres_iters"] for x in st]))
    newton = float(np.mean([x["newton_iters"] for x in st]))
    worst_groups = max(x["rel_residual"] for o in out for x in o[3])
    for s in solvers:
        s.close()
    # baseline: one handle per crossbar, sequential (a sample of 16 crossbars, scaled)
    dev = torch.device("cuda", torch.cuda.current_device())
    sample = list(range(0, count, max(1, count // 16)))
    tb = 0.0
    for k in sample:
        cb = cbs[k]
        with mca.Solver(params_for(mca, cb.params, mca.PREC_BF16_SPLIT, nvec, restart=16),
                        cb.gmap) as s1:
            vin_d = torch.as_tensor(cb.vin, device=dev)
            vt = torch.empty(nvec, s1.m, s1.n, dtype=torch.float64, device=dev)
            vb = torch.empty_like(vt)
            io = torch.empty(nvec, s1.n, dtype=torch.float64, device=dev)
            s1.solve(vin_d, vt, vb, io)
            torch.cuda.synchronize()
            a = time.perf_counter()
            s1.solve(vin_d, vt, vb, io)
            torch.cuda.synchronize()
            tb += time.perf_counter() - a
    return {"value": count * nvec / t, "unit": "solves/s", "solves": count * nvec,
            "launches": 1, "form": "one persistent launch (mca_batch_solve)",
            "crossbars": count, "shape_groups": len(groups),
            "max_rel_residual": worst, "gmres_iters_per_solve": its,
            "newton_iters_per_solve": newton,
            "phase_share": {k: round(v / ptot, 4) for k, v in prof.items()},
            "grouped_handles_value": count * nvec / t_groups, "grouped_handles_threads": threads,
            "grouped_handles_max_rel_residual": worst_groups,
            "one_handle_per_crossbar_value": len(sample) * nvec / tb,
            "workload": "128 crossbars, rows/cols from {64,128,256,512}, 16 V_in each, "
                        "log-uniform g x lognormal(0.1), BF16-split preconditioner, "
                        "restart 16, device-resident inputs and outputs, wall clock of the "
                        "solves"}


def gemm_tiles(solver):
    """Tile configuration the autotuner picked for the four tensor-core transforms."""
    names = ("X Q_r", "Q_c^T T1 + modes", "Y Q_r^T", "Q_c E")
    out = {}
    for name, (ws, bn, lp) in zip(names, solver.tile_config()):
        if ws < 0:
            return None
        kind = {0: "tile-per-cta", 1: "persistent", 2: "persistent, CTA pairs (cta_group::2)"}
        out[name] = {"kernel": kind.get(ws, str(ws)), "tile": f"{256 if ws == 2 else 128}x{bn}",
                     "layers_per_tile": lp}
    return out


def d2h_rate(torch, dev, nbytes=1 << 30):
    """Device-to-host copy rate of this machine into pinned memory (GB/s): the end-to-end figure
    moves every solve's node voltages to the host, so where this link is slow it bounds e2e."""
    d = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
    h = torch.empty(nbytes // 8, dtype=torch.float64).pin_memory()
    st = torch.cuda.current_stream()
    h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(2):
        h.copy_(d, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    return round(2 * nbytes / (e0.elapsed_time(e1) * 1e6), 1)


# Batches per end-to-end call (see the e2e block in run_bench).
E2E_PASSES = 8
E2E_SOLVES = 256     # solves per end-to-end call


# FP64 CUDA-core peak used for the FP64 form: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def committed_traffic(fam, fp):
    """Per-launch DRAM bytes of this family from the committed ncu summary, if it was
    taken on the current kernels; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(fam)
    if not ent:
        return None
    # the capture is keyed to the sources of the kernel (their bytes in order)
    import hashlib
    h = hashlib.sha1()
    for name in ent.get("sources", [ent.get("source", "")]):
        src = os.path.join(ROOT, "paper_2109_07929_gb300", "csrc", name)
        if not os.path.exists(src):
            return None
        with open(src, "rb") as f:
            h.update(f.read())
    if h.hexdigest() != ent.get("sha1"):
        return None
    if "ratio_to_algorithmic" in ent:
        return ent["ratio_to_algorithmic"] * fp["bytes"] / max(1, fp["launches"])
    return ent.get("bytes_per_launch")


def run_e2e_breakdown(args, reps=3):
    """Where an end-to-end call spends its time: solve_many on --handles x --batch vectors
    per pass (the headline's handles), outputs in device memory or pinned host memory, one
    or two passes per handle per call, with and without the node-voltage outputs; then the
    device-to-host copy of one call's voltages alone (one stream per handle).  Median
    wall time of `reps` calls after one warm-up call, each call returning with its outputs
    in place."""
    import torch
    import paper_2109_07929_gb300 as mca
    torch.cuda.set_device(0)
    B, H, m, n = args.batch, max(1, args.handles), args.size, args.size
    ws = make_workload(args, 0, H * 2 * B)
    params = params_for(mca, ws.params, mca.PREC_BF16_SPLIT, B, args.restart)
    solvers = [mca.Solver(params, ws.gmaps) for _ in range(H)]
    dev = torch.device("cuda", 0)
    vin = {"device": torch.as_tensor(ws.vin, device=dev),
           "host": torch.as_tensor(ws.vin).pin_memory()}
    out = {"host_loadavg": os.getloadavg(), "host_cpus": os.cpu_count()}

    def call(name, P, where, volt=True):
        nv = P * B
        vins = [vin[where][h * nv:(h + 1) * nv] for h in range(H)]
        maps = [ws.map_index[h * nv:(h + 1) * nv] for h in range(H)]
        if where == "device":
            mk = lambda *s: torch.empty(*s, dtype=torch.float64, device=dev)
        else:
            mk = lambda *s: torch.empty(*s, dtype=torch.float64).pin_memory()
        outs = [((mk(nv, m, n) if volt else None), (mk(nv, m, n) if volt else None),
                 mk(nv, n)) for _ in range(H)]
        ts = []
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = mca.solve_many(solvers, vins, map_indices=maps, n_threads=H, outs=outs)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            for r in res:
                for st in r[3]:
                    assert st["status"] == 0 and st["rel_residual"] <= TOL, st
        t = float(np.median(ts[1:]))
        out[name] = {"ms_per_call": round(1e3 * t, 2), "solves_per_s": round(H * nv / t, 1),
                     "solves_per_call": H * nv}
        del outs

    call("device_1_pass", 1, "device")
    call("device_2_passes", 2, "device")
    call("host_1_pass", 1, "host")
    call("host_2_passes", 2, "host")
    call("host_2_passes_currents_only", 2, "host", volt=False)
    # the voltages of one two-pass call (both layers), device -> pinned host, alone
    d = torch.empty(H, 2 * B, 2, m * n, dtype=torch.float64, device=dev)
    hb = torch.empty(H, 2 * B, 2, m * n, dtype=torch.float64).pin_memory()
    streams = [torch.cuda.Stream() for _ in range(H)]
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for h in range(H):
            with torch.cuda.stream(streams[h]):
                hb[h].copy_(d[h], non_blocking=True)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    out["voltage_copies_alone"] = {"ms": round(1e3 * t, 1), "bytes": d.numel() * 8,
                                   "GB/s": round(d.numel() * 8 / t / 1e9, 1)}
    for s_ in solvers:
        s_.close()
    print(json.dumps({"e2e_breakdown": step_config(args), "results": out}), flush=True)


def run_table1(args):
    """Table 1 of the paper on the GPU: GMRES iterations (and time) to relative residual
    1e-6 on the first Newton system J x = Y in the paper's normalised regime (wires and
    terminations g = 1, linear devices with g_ij ~ U[0, 0.4]), per preconditioner."""
    import torch
    import paper_2109_07929_gb300 as mca
    from oracle import mca_oracle as O   # source vector only (rhs of the linear system)
    precs = [("none", mca.PREC_NONE), ("jacobi", mca.PREC_JACOBI), ("paper_mhat", mca.PREC_MHAT),
             ("exact_fp64", mca.PREC_FP64), ("exact_bf16split", mca.PREC_BF16_SPLIT)]
    out = {}
    for n in (16, 32, 64, 128, 256, 512):
        cb = mi.config_paper_regime(n, 0)
        p = cb.params
        g = np.maximum(cb.gmap, 1e-12)
        Yt, Yb = O.source_vector(p, cb.vin[0])
        rhs = torch.as_tensor(np.concatenate([Yt, Yb])[None], device="cuda")
        D = torch.as_tensor(g.ravel()[None], device="cuda")
        row = {}
        for name, prec in precs:
            params = mca.default_params(n, n, g_wire_top=1.0, g_wire_bot=1.0, g_src=1.0,
                                        g_term_top_right=1.0, g_term_bot_top=1.0, g_sense=1.0,
                                        b=0.0, precision=prec, max_batch=1)
            with mca.Solver(params, g) as s:
                dx = torch.empty(1, 2 * n * n, dtype=torch.float64, device="cuda")
                s.gmres_solve(D, [g.mean()], rhs, dx, 1e-6, max_iters=60000)
                torch.cuda.synchronize()
                t = time.perf_counter()
                its, res = s.gmres_solve(D, [g.mean()], rhs, dx, 1e-6, max_iters=60000)
                torch.cuda.synchronize()
                row[name] = {"steps": int(its[0]), "ms": 1e3 * (time.perf_counter() - t),
                             "converged": bool(res[0] <= 1e-6 * float(rhs.norm()) * 1.01)}
        out[str(n)] = row
        print(json.dumps({"n": n, **row}), file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "table1_gpu", "restart": 30, "rtol": 1e-6,
                      "regime": "g = 1 wires and terminations, linear devices U[0,0.4]",
                      "results": out}), flush=True)


def main():
    args = parse_args()
    if args.oracle_configs:
        print(json.dumps(oracle_configs()), flush=True)
        return
    if args.batch_profile:
        return run_batch_profile(args)
    if args.table1:
        run_table1(args)
        return
    if args.e2e_breakdown:
        run_e2e_breakdown(args)
        return
    if args.profile_precond:
        run_profile_precond(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
