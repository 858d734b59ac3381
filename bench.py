"""Throughput benchmark of the fused D3Q19 MRT sweep with the single-node curved-wall
scheme (arXiv:1712.08288, Eqs. 2.10/2.13) on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload: body-force driven flow in a circular pipe of radius 0.4 L whose axis
(16, 4, 3) is tilted off the lattice axes, L = 256 (16.8M nodes, 8.8M fluid), wall
fractions from the exact cylinder, periodic along the axis through a skewed x-wrap,
l = gamma, b = 1.  One step = one fused collide/stream/boundary sweep over the grid
(one kernel launch).  The headline value is fluid-node updates per second (MLUPS)
with FP32 deviation storage; FP64 storage is timed on the same workload beside it,
and the accuracy of both against the analytic Hagen-Poiseuille profile is reported
after an untimed run.  The populations (1.27 GB in FP32) exceed L2 (129 MB), so
no flush is needed between steps.

Untimed-for-the-headline sections of the same JSON line (rank 0; each can be turned
off with its flag): "d3q15" (the same pipe with the paper's D3Q15), "accuracy"
(E_r of FP32 and FP64 after 20000 steps at L = 128), "ensemble" (96 uneven Couette
instances, one batched graph launch per step against one launch per instance),
"refinement" (curved-wall Couette to steady state, n = 32..512, order; D2Q9
throughput at n = 2048), "taylor_green" (the moving-wall disc of Sec. 3.2, order),
"adjoint" (128^3 sphere, 2000 steps, backward/forward time and central-difference
check), "e2e" (the headline through the C-ABI with host buffers), "cpu_baseline".

--impl reference times the FP64 CPU oracle (the only reference implementation of
this method: the paper ships no code) on the host cores, on a bounded sample of
the same workload family.

Under torchrun (N > 1) every rank runs the same workload on its own GPU (replicas,
weak scaling; the method needs no exchange between independent problems) and the
slowest rank's time is reported.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 MRT+curved-BC MLUPS & % HBM roofline, FP32 vs FP64 at matched L2 err"
WORKLOAD = ("D3Q19 MRT body-force Poiseuille flow in a tilted periodic pipe, L=256 "
            "(16.8M nodes), R=0.4L, axis (16,4,3), skewed x-wrap, single-node scheme l=gamma b=1")
SCHEME = (0.0, 1.0, 0.0, 1.0)
BYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}
PROFILE = os.path.join(ROOT, "profiles", "sweep_d3q19_f32_pipe192.txt")
PROFILE_F64 = os.path.join(ROOT, "profiles", "sweep_d3q19_f64_ops_pipe128.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1712_08288_gb300", "csrc", f)
                  for f in ("sweep.cuh", "common.cuh", "lattice.h", "lbm_internal.h")]


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_field(path, key):
    """A figure from a committed ncu summary (key: value lines), or None when the
    summary is absent or the kernel source changed since it was taken."""
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic():
    """DRAM bytes per launch of the FP32 sweep at the bench's size (ncu summary)."""
    return _profile_field(PROFILE, "dram_bytes_per_launch_full_size")


def profiled_fp64_flops():
    """FP64 operations per fluid-node update of the FP64 sweep (ncu: DADD + DMUL +
    2 DFMA thread instructions per launch over the fluid nodes)."""
    return _profile_field(PROFILE_F64, "fp64_flops_per_fluid_node")


def profiled_fp64_instructions():
    """FP64 pipe instructions (DADD + DMUL + DFMA) per fluid-node update of the FP64
    sweep (same ncu summary)."""
    return _profile_field(PROFILE_F64, "fp64_instructions_per_fluid_node")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
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

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        top = sorted(sm)[len(sm) // 4:]          # samples under load
        return {"sm_mhz": statistics.median(top), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    """The slowest rank's value (timings are taken as the maximum over ranks)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(fluid_per_rank, steps, world, total_ms):
    """Whole-job throughput of independent replicas (weak scaling): every rank
    advances its own copy, the job takes as long as the slowest rank."""
    return fluid_per_rank * steps * world / (total_ms * 1e-3) / 1e6


def build_sim(w, precision, torch, stream):
    from paper_1712_08288_gb300 import binding as B
    sim = B.from_workload(w, precision, SCHEME)
    sim.set_stream(stream.cuda_stream)
    return sim


def time_steps(sim, torch, stream, steps, warmup, per_launch=True):
    """Warm-up, then K single-sweep launches bracketed by events; returns
    (total ms, list of per-launch ms).  The warm-up count is rounded up to an even
    number, so that the first timed launch is an even step."""
    sim.step(warmup + (warmup & 1))
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)] if per_launch else []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        if per_launch:
            ev[k][0].record(stream)
        sim.step(1)
        if per_launch:
            ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    launches = [a.elapsed_time(b) for a, b in ev]
    return total, launches


def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    from paper_1712_08288_gb300 import workloads as W

    L = args.L
    w = W.tilted_pipe_3d(L)
    n_fluid = int((~w["solid"]).sum())
    Q = 19

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- FP32 deviation storage: the headline --------------------------------
    sim = build_sim(w, "f32", torch, stream)
    sim.init_equilibrium(None, np.nan_to_num(w["u_exact"]))
    barrier()
    with ClockSampler(local) as clk:
        total_ms, launches = time_steps(sim, torch, stream, args.steps, args.warmup)
        barrier()
    total_ms = max_over_ranks(total_ms, world, "cuda")
    mlups = job_mlups(n_fluid, args.steps, world, total_ms)
    launch_ms = float(np.mean(launches))
    hbm, peak_kind = peaks()
    alg_bytes = 2 * Q * BYTES["f32"] * n_fluid          # populations read + written
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic()
    status32 = sim.error_norms(None, check=False)["status"]
    del sim

    # ---- the other storage precisions on the same workload ---------------------
    prec_lines = {"f32": {"even_us": round(float(np.mean(launches[0::2])) * 1e3, 1),
                          "odd_us": round(float(np.mean(launches[1::2])) * 1e3, 1),
                          "mlups": round(mlups, 1), "frac_of_hbm": round(achieved / hbm, 4)}}
    fp64_peak = None
    for prec in ("f64", "bf16", "f16"):
        sim = build_sim(w, prec, torch, stream)
        sim.init_equilibrium(None, np.nan_to_num(w["u_exact"]))
        kp = max(10, args.steps // 8) if prec == "f64" else max(20, args.steps // 2)
        kp += kp & 1                                   # even and odd steps alike
        tot_p, ls_p = time_steps(sim, torch, stream, kp, min(args.warmup, 5))
        lm = float(np.mean(ls_p))
        gbs = 2 * Q * BYTES[prec] * n_fluid / (lm * 1e-3) / 1e9
        line_p = {"mlups": round(n_fluid * kp / (tot_p * 1e-3) / 1e6, 1), "steps": kp,
                  "even_us": round(float(np.mean(ls_p[0::2])) * 1e3, 1),
                  "odd_us": round(float(np.mean(ls_p[1::2])) * 1e3, 1),
                  "bytes_per_node": 2 * Q * BYTES[prec], "achieved_GBs": round(gbs, 1),
                  "frac_of_hbm": round(gbs / hbm, 4)}
        if prec == "f64":
            # the FP64 sweep is bound by the FP64 pipe on this GPU: report it against
            # the measured FMA rate, with the FP64 operations per fluid node counted
            # by ncu on the same kernel (profiles/)
            from paper_1712_08288_gb300 import binding as B
            fp64_peak = B.probe_fp64_rate()
            fl_per_node = profiled_fp64_flops()
            line_p["fp64_peak_gflops"] = round(fp64_peak, 1)
            if fl_per_node:
                ach_fl = fl_per_node * n_fluid / (lm * 1e-3) / 1e9
                line_p["roofline"] = {"bound": "fp64", "flops_per_node": fl_per_node,
                                      "achieved_gflops": round(ach_fl, 1),
                                      "frac_of_fp64_peak": round(ach_fl / fp64_peak, 4)}
                # the FP64 pipe issues one DADD, DMUL or DFMA per slot: the sweep's FP64
                # instructions per second against the probe's DFMA issue rate (half its
                # flop rate)
                in_per_node = profiled_fp64_instructions()
                if in_per_node:
                    ach_in = in_per_node * n_fluid / (lm * 1e-3) / 1e9
                    line_p["roofline"].update({
                        "fp64_instructions_per_node": in_per_node,
                        "achieved_ginst_per_s": round(ach_in, 1),
                        "frac_of_fp64_issue_rate": round(ach_in / (fp64_peak / 2), 4)})
        prec_lines[prec] = line_p
        del sim
    mlups64 = prec_lines["f64"]["mlups"]
    k64 = prec_lines["f64"]["steps"]

    # ---- D3Q15 (the paper's own 3D lattice) on the same workload --------------
    d15 = None
    if args.d3q15_steps > 0:
        w15 = W.tilted_pipe_3d(L, lattice="D3Q15")
        nf15 = int((~w15["solid"]).sum())
        d15 = {"workload": "the same pipe, D3Q15 (Appendix velocities, M and S)"}
        for prec, k in (("f32", args.d3q15_steps), ("f64", max(10, args.d3q15_steps // 8))):
            sim = build_sim(w15, prec, torch, stream)
            sim.init_equilibrium(None, np.nan_to_num(w15["u_exact"]))
            tot, ls = time_steps(sim, torch, stream, k, min(args.warmup, 10))
            lm = float(np.mean(ls))
            gbs = 2 * 15 * BYTES[prec] * nf15 / (lm * 1e-3) / 1e9
            d15[prec] = {"mlups": round(nf15 * k / (tot * 1e-3) / 1e6, 1), "steps": k,
                         "achieved_GBs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 4)}
            del sim

    # ---- e2e through the C-ABI with host buffers ------------------------------
    sim = build_sim(w, "f32", torch, stream)
    N = L ** 3
    u0 = torch.from_numpy(np.ascontiguousarray(np.nan_to_num(w["u_exact"]))).pin_memory().numpy()
    rho_h = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    u_h = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
    sim.step(2)
    barrier()
    e0 = time.perf_counter()
    sim.init_equilibrium(None, u0)                 # H2D of the initial field
    sim.step(args.steps)
    sim._check(sim._lib.lbm_moments(sim.h, rho_h.ctypes.data_as(__import__("ctypes").c_void_p),
                                    u_h.ctypes.data_as(__import__("ctypes").c_void_p)))   # D2H
    e_ms = (time.perf_counter() - e0) * 1e3
    e2e = {"value": n_fluid * args.steps * world / (e_ms * 1e-3) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": u0.nbytes / args.steps,
           "d2h_bytes_per_step": (rho_h.nbytes + u_h.nbytes) / args.steps,
           "note": "one job: initial field H2D, K sweeps, rho and u D2H; bytes per sweep"}
    del sim

    # ---- accuracy: every precision against the analytic profile (untimed) ------
    acc = None
    if args.accuracy_steps > 0 and rank == 0:
        acc = run_accuracy(args, torch, stream)

    # ---- ensemble: batched persistent graph launch vs one launch per instance --
    ens = None
    if args.ensemble_steps > 0 and rank == 0:
        ens = run_ensemble(args, torch, stream)

    # ---- grid refinement of the 2D curved-wall problem (order of convergence) ---
    ref = None
    if args.refine_max > 0 and rank == 0:
        ref = run_refinement(args, torch, stream)

    # ---- moving curved wall: Taylor-Green in a disc (order of convergence) ------
    tg = None
    if args.tg_max > 0 and rank == 0:
        tg = run_taylor_green(args, torch, stream)

    # ---- adjoint: gradients through the whole run, sqrt(N) checkpointing --------
    adj = None
    if args.adjoint_steps > 0 and rank == 0:
        adj = run_adjoint(args, torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_L, args.cpu_steps)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("L=256", "L=%d" % L), "lattice": "D3Q19",
                       "L": L, "nodes": N, "fluid_nodes": n_fluid, "links": len(w["links"]["node"]),
                       "storage": "f32 deviations (f - w rho0), f32 arithmetic",
                       "l2_policy": "inputs larger than L2 (%.2f GB populations)" % (Q * 4 * N / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                         "traffic": traffic, "kernel": "sweep_kernel<D3Q19,float>",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "launch_ms": launch_ms},
            "precisions": prec_lines,
            "d3q15": d15,
            "accuracy": acc,
            "ensemble": ens,
            "refinement": ref,
            "taylor_green": tg,
            "adjoint": adj,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "status_f32": status32,
        }
        line["summary"] = summary(line)      # last: the compact digest ends the line
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def summary(line):
    """A compact digest of the sections (roofline fractions per precision, errors
    and orders, adjoint and ensemble figures), placed at the end of the line."""
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r(v, n=4):
        return None if v is None else (round(v, n) if isinstance(v, float) else v)
    pr = line.get("precisions") or {}
    out = {"frac_hbm": {p: g(pr, p, "frac_of_hbm") for p in ("f32", "bf16", "f16", "f64")},
           "mlups": {p: g(pr, p, "mlups") for p in ("f32", "bf16", "f16", "f64")},
           "f64_frac_of_fp64_peak": g(pr, "f64", "roofline", "frac_of_fp64_peak"),
           "f64_frac_of_fp64_issue_rate": g(pr, "f64", "roofline", "frac_of_fp64_issue_rate")}
    acc = line.get("accuracy")
    if acc:
        out["pipe_E_r"] = {"L": acc["L"], **{p: ["%.4g" % v for v in acc[p]] for p in ("f64", "f32", "bf16", "f16")}}
        out["pipe_order"] = {p: r(acc.get("order_" + p), 3) for p in ("f64", "f32", "bf16", "f16")}
    ref = line.get("refinement")
    if ref:
        out["couette_order"] = {"f64": r(ref.get("order_f64"), 3), "f32": r(ref.get("order_f32"), 3),
                                "sizes": ref.get("sizes")}
    tg = line.get("taylor_green")
    if tg:
        out["tg_order"] = {k: r(v.get("order"), 3) for k, v in tg.items() if isinstance(v, dict)}
    adj = line.get("adjoint")
    if adj:
        out["adjoint"] = {"bwd_over_fwd_f32": g(adj, "f32", "backward_over_forward"),
                          "fwd_over_step_f32": g(adj, "f32", "forward_over_lbm_step"),
                          "fd_rel_f64": r(g(adj, "f64", "rel_err_vs_fd"), 10)}
    ens = line.get("ensemble")
    if ens:
        out["ensemble"] = {"mlups": ens.get("batched_graph_mlups"), "frac_hbm": ens.get("frac_of_hbm"),
                           "speedup": ens.get("speedup")}
    return out


def run_accuracy(args, torch, stream):
    """The D3Q19 tilted pipe at L = 64, 128, 256 from the analytic-equilibrium start,
    args.accuracy_steps steps in every storage precision: E_r against the analytic
    Hagen-Poiseuille parabola, the least-squares order over L per precision, and
    which precisions match FP64's error (within 10 %, the metric's matched-error
    rule) at each size."""
    from paper_1712_08288_gb300 import workloads as W
    sizes = [int(v) for v in args.accuracy_sizes.split(",") if v]
    precs = ("f64", "f32", "bf16", "f16")
    out = {"workload": "D3Q19 tilted pipe, analytic start, %d steps" % args.accuracy_steps,
           "L": sizes, "steps": args.accuracy_steps}
    t_start = time.perf_counter()
    for prec in precs:
        out[prec] = []
    for L in sizes:
        wa = W.tilted_pipe_3d(L)
        ue = np.nan_to_num(wa["u_exact"])
        for prec in precs:
            s2 = build_sim(wa, prec, torch, stream)
            s2.init_equilibrium(None, ue)
            s2.step(args.accuracy_steps)
            out[prec].append(s2.error_norms(ue, check=False)["l2_rel"])
            del s2
    for prec in precs:
        e = out[prec]
        out["order_" + prec] = (float(-np.polyfit(np.log(sizes), np.log(e), 1)[0])
                                if len(sizes) > 1 else None)
        out["matched_" + prec] = [bool(abs(a - b) <= 0.1 * b) for a, b in zip(e, out["f64"])]
    out["seconds"] = round(time.perf_counter() - t_start, 1)
    return out


def run_ensemble(args, torch, stream):
    """96 circular Couette instances of uneven size (seed 0), D2Q9, FP32 deviation
    storage: aggregate fluid MLUPS of one persistent batched launch per step replayed
    from a CUDA graph (tuned order and blocks per SM) against the same instances
    stepped with one launch each."""
    from paper_1712_08288_gb300 import binding as B
    from paper_1712_08288_gb300 import workloads as W
    ws = [W.ensemble_member(p) for p in W.couette_ensemble(args.ensemble_count, 0)]
    nf = sum(int((~w["solid"]).sum()) for w in ws)
    nodes = sum(w["shape"][0] * w["shape"][1] for w in ws)

    def fresh():
        sims = []
        for w in ws:
            s = build_sim(w, "f32", torch, stream)
            s.init_equilibrium()
            sims.append(s)
        return sims

    K = args.ensemble_steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # one launch per instance per step
    sims = fresh()
    for s in sims:
        s.step(4)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    del sims
    # batched, graph-replayed
    sims = fresh()
    batch = B.Batch(sims)
    batch.set_stream(stream.cuda_stream)
    order, blocks, split, tile_w = batch.tune(20)
    batch.step(4)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    q = batch.query()
    batch.close()
    del sims
    return {"instances": len(ws), "nodes": nodes, "fluid_nodes": nf, "steps": K,
            "batched_graph_mlups": round(nf * K / (ms_batch * 1e-3) / 1e6, 1),
            "one_launch_per_instance_mlups": round(nf * K / (ms_single * 1e-3) / 1e6, 1),
            "speedup": round(ms_single / ms_batch, 2),
            "alg_GBs": round(2 * 9 * 4 * nf * K / (ms_batch * 1e-3) / 1e9, 1),
            "frac_of_hbm": round(2 * 9 * 4 * nf * K / (ms_batch * 1e-3) / 1e9 / peaks()[0], 4),
            "tuned": {"order": B.Batch.ORDERS[order], "blocks_per_sm": blocks, "split_by_class": bool(split),
                      "tile_w": tile_w,
                      "launches_per_step": q["launches_per_step"], "tiles": q["tiles"]},
            "workload": "D2Q9 circular Couette ensemble, seed 0, n ~ U{48..768}, FP32 deviations"}


def run_refinement(args, torch, stream):
    """Grid refinement of the circular Couette problem (D2Q9, curved walls, the 64^2
    configuration scaled by n/64 in diffusive scaling) to a steady state.

    Each n first runs with FP32 deviation storage from the analytic-equilibrium
    start for ten diffusion times tau = (R2 - R1)^2 / (pi^2 nu) (the slowest decay
    time of the annulus), which leaves the start's transient below FP32's own
    rounding; its E_r and residual are the FP32 result.  FP64 storage then starts
    from the FP32 end state (all populations copied) and steps until the relative
    change of u over 200 steps is below 1e-10; its E_r is the FP64 result.  A
    steady state does not depend on the start, and the FP32 run only removes most
    of the O(tau) spin-up from the FP64 run.  Orders by least squares of log E_r
    against log n; throughput at n = 2048 is timed separately (fixed step counts)."""
    from paper_1712_08288_gb300 import workloads as W
    sizes = [n for n in (32, 64, 128, 256, 512, 1024, 2048) if n <= args.refine_max]
    chunk, tol = 200, 1e-10
    out = {"sizes": sizes, "steady_tol": tol, "chunk": chunk, "f64": {}, "f32": {}}
    t_start = time.perf_counter()
    for n in sizes:
        w = W.couette_config(n)
        ue = np.nan_to_num(w["u_exact"])
        r1, r2 = 10.0 * n / 64, 28.0 * n / 64
        tau = (r2 - r1) ** 2 / (np.pi ** 2 * w["nu"])
        n32 = int(np.ceil(10 * tau / chunk)) * chunk
        s32 = build_sim(w, "f32", torch, stream)
        s32.init_equilibrium(None, ue)
        s32.step(n32 - chunk)
        s32.error_norms(ue, check=False)
        s32.step(chunk)
        nrm = s32.error_norms(ue, check=False)
        out["f32"][str(n)] = {"E_r": nrm["l2_rel"], "steps": n32, "residual": nrm["residual"]}
        f = s32.get_populations()
        del s32
        s64 = build_sim(w, "f64", torch, stream)
        s64.set_populations(f)
        s64.error_norms(ue, check=False)
        steps, res = 0, 1.0
        while res >= tol and steps < args.refine_max_steps:
            s64.step(chunk)
            steps += chunk
            res = s64.error_norms(ue, check=False)["residual"]
        e64 = s64.error_norms(ue, check=False)["l2_rel"]
        del s64
        out["f64"][str(n)] = {"E_r": e64, "steps_after_f32": steps, "residual": res,
                              "converged": bool(res < tol)}

    def order(prec, ns):
        e = [out[prec][str(n)]["E_r"] for n in ns]
        return float(-np.polyfit(np.log(ns), np.log(e), 1)[0]) if len(ns) > 1 else None
    out["order_f64"] = order("f64", sizes)
    out["order_f32"] = order("f32", sizes)
    out["order_f64_to_512"] = order("f64", [n for n in sizes if n <= 512])
    # the size from which FP32's error leaves FP64's by more than 10 %
    out["f32_matched"] = {str(n): bool(abs(out["f32"][str(n)]["E_r"] - out["f64"][str(n)]["E_r"])
                                       <= 0.1 * out["f64"][str(n)]["E_r"]) for n in sizes}
    out["seconds"] = round(time.perf_counter() - t_start, 1)
    if args.refine_mlups_n > 0:
        w = W.couette_config(args.refine_mlups_n)
        nf = int((~w["solid"]).sum())
        ue = np.nan_to_num(w["u_exact"])
        out["throughput_n"] = args.refine_mlups_n
        for prec, k in (("f32", 2000), ("f64", 500)):
            sim = build_sim(w, prec, torch, stream)
            sim.init_equilibrium(None, ue)
            total, _ = time_steps(sim, torch, stream, k, 20, per_launch=False)
            out[prec + "_mlups_at_n"] = round(nf * k / (total * 1e-3) / 1e6, 1)
            del sim
    out["workload"] = "D2Q9 circular Couette, 64^2 configuration scaled to n (diffusive scaling)"
    return out


def run_taylor_green(args, torch, stream):
    """The paper's Taylor-Green vortex in a disc (Sec. 3.2; D2Q9, moving curved wall
    through lbm_set_wall_factor, l = gamma): E_r at T = 1/U0 for h = 1/40 .. 1/200 at
    s_nu = 1 and 1.99, FP64, and the least-squares order.  With several disc shifts
    against the lattice (--tg-shifts) every h is run at each shift, and the order is
    also fitted to the mean E_r over the shifts (the cut fractions q change with the
    disc's position against the nodes; the mean separates that scatter from the trend
    in h)."""
    from paper_1712_08288_gb300 import workloads as W
    sizes = [int(n) for n in args.tg_sizes.split(",") if n and int(n) <= args.tg_max]
    shifts = [tuple(float(v) for v in p.split(",")) for p in args.tg_shifts.split(";") if p]
    out = {"workload": "Taylor-Green vortex in the disc of Sec. 3.2, nu 0.002, U0 0.05, T = 1/U0",
           "inv_h": sizes, "shifts": shifts}
    t_start = time.perf_counter()

    def slope(e):
        return float(np.polyfit(np.log(1.0 / np.array(sizes)), np.log(e), 1)[0]) if len(sizes) > 1 else None
    for s_nu in [float(v) for v in args.tg_snu.split(",") if v]:
        per_shift, steps = [], []
        for sh in shifts:
            errs = []
            for n in sizes:
                w = W.taylor_green_disc(n, s_nu, shift=sh)
                sim = build_sim(w, "f64", torch, stream)
                sim.init_equilibrium(w["rho_init"], np.nan_to_num(w["u_exact"]))
                sim.set_wall_factor(1.0, w["decay"])
                sim.step(w["steps"])
                ue = np.nan_to_num(w["u_exact"]) * w["decay"] ** w["steps"]
                errs.append(sim.error_norms(ue, check=False)["l2_rel"])
                if len(steps) < len(sizes):
                    steps.append(w["steps"])
                del sim
            per_shift.append(errs)
        rec = {"E_r": per_shift[0] if len(shifts) == 1 else per_shift, "steps": steps,
               "order": slope(per_shift[0])}
        if len(shifts) > 1:
            mean = np.mean(np.array(per_shift), axis=0)
            rec["E_r_mean"] = mean.tolist()
            rec["order_of_mean"] = slope(mean)
            rec["order_per_shift"] = [slope(e) for e in per_shift]
        out["s_nu_%g" % s_nu] = rec
    out["seconds"] = round(time.perf_counter() - t_start, 1)
    return out


def run_adjoint(args, torch, stream):
    """Adjoint of the sphere-in-a-periodic-box problem (D3Q19, 128^3, sphere R=20 at
    (64.37, 63.71, 64.13), body force 1e-6 along x, s_nu = 1): loss = sum over the slab
    96 <= x < 104 of |u - u_target|^2 after K steps from rest, u_target from a run with
    every wall fraction raised by 0.05 (clamped to 1) and s_nu scaled by 1.02.
    Timing (after one warm-up call that allocates the workspace): the forward half
    lbm_adjoint_forward against lbm_step over the same K steps, and the backward
    half lbm_adjoint_backward against the forward half.  FP64 check: dJ/ds_nu (sum
    over the viscous rows) against central differences with h = 1e-4."""
    from paper_1712_08288_gb300 import workloads as W
    n, K = args.adjoint_L, args.adjoint_steps
    c = (64.37 * n / 128, 63.71 * n / 128, 64.13 * n / 128)
    w = W.sphere_3d(n, 20.0 * n / 128, c, s_nu=1.0, force=(1e-6, 0.0, 0.0))
    N = n ** 3
    x = np.arange(N) % n
    mask = (x >= 96 * n // 128) & (x < 104 * n // 128)
    viscous = [9, 11, 13, 14, 15]
    wt = dict(w)
    wt["links"] = dict(w["links"], q=np.minimum(w["links"]["q"] + 0.05, 1.0))
    wt["S"] = w["S"].copy()
    wt["S"][viscous] *= 1.02
    tgt = build_sim(wt, "f64", torch, stream)
    tgt.init_equilibrium()
    tgt.step(K)
    _, ut = tgt.moments()
    ut = np.nan_to_num(ut)
    del tgt
    out = {"workload": "D3Q19 sphere R=%g in a periodic %d^3 box, %d steps" % (20.0 * n / 128, n, K)}
    for prec in ("f32", "f64"):
        sim = build_sim(w, prec, torch, stream)
        sim.init_equilibrium()
        sim.step(2)
        sim.init_equilibrium()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(K)
        torch.cuda.synchronize()
        t_step = time.perf_counter() - t0
        sim.init_equilibrium()
        sim.adjoint(K, mask, ut)                # warm-up: allocates the adjoint's workspace
        sim.init_equilibrium()
        torch.cuda.synchronize()
        # the two halves the autograd Function calls: lbm_adjoint_forward (the
        # checkpointed run and the loss) and lbm_adjoint_backward (recompute and
        # adjoint sweep)
        t0 = time.perf_counter()
        J = sim.adjoint_forward(K, mask, ut)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        gs, gq, gp = sim.adjoint_backward()
        torch.cuda.synchronize()
        t_bwd = time.perf_counter() - t0
        out[prec] = {"J": J, "dJ_ds_nu": float(gs[viscous].sum()),
                     "lbm_step_s": round(t_step, 4), "forward_s": round(t_fwd, 4),
                     "backward_s": round(t_bwd, 4),
                     "forward_over_lbm_step": round(t_fwd / t_step, 3),
                     "backward_over_forward": round(t_bwd / t_fwd, 2),
                     "checkpoints": int(np.ceil(K / np.ceil(np.sqrt(K))))}
        if prec == "f64":
            h = 1e-4

            def J_of(sv):
                s2 = build_sim(w, "f64", torch, stream)
                S = w["S"].copy()
                S[viscous] = sv
                s2.set_relaxation(S)
                s2.init_equilibrium()
                s2.step(K)
                _, u = s2.moments()
                d = u[mask] - ut[mask]
                return float(np.nansum(d * d))
            fd = (J_of(1.0 + h) - J_of(1.0 - h)) / (2 * h)
            out["f64"]["fd_dJ_ds_nu"] = fd
            out["f64"]["rel_err_vs_fd"] = abs(fd - out["f64"]["dJ_ds_nu"]) / abs(fd) if fd else None
        del sim
    ref = out["f64"]["dJ_ds_nu"]
    out["f32"]["rel_err_vs_f64"] = abs(out["f32"]["dJ_ds_nu"] - ref) / abs(ref) if ref else None
    return out


_ORACLE_RUN = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import lattices as OL, lbm as O
from paper_1712_08288_gb300 import workloads as W
w = W.tilted_pipe_3d(%d)
sim = O.Simulation(OL.D3Q19, w['shape'], w['S'], 1.0, w['solid'], w['links'], scheme=%r,
                   force=w['force'], skew=w['skew'])
sim.init_equilibrium(None, np.nan_to_num(w['u_exact']))
sim.step(%d)
start_at = %r
while start_at and time.time() < start_at:
    time.sleep(0.01)
t0 = time.time(); p0 = time.perf_counter(); sim.step(%d); dt = time.perf_counter() - p0
nf = int((~w['solid']).sum())
print(json.dumps({'mlups': nf * %d / dt / 1e6, 'seconds': dt, 'fluid': nf, 't0': t0, 't1': t0 + dt}))
"""


def _oracle_procs(L, steps, warmup, nproc):
    """Run the oracle in nproc fresh single-threaded processes started together
    (each steps its own copy of the sample); returns their JSON records."""
    start_at = time.time() + 20.0 if nproc > 1 else 0.0
    code = _ORACLE_RUN % (ROOT, L, SCHEME, warmup, start_at, steps, steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for _ in range(nproc)]
    out = []
    for pr in procs:
        so, se = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(se[-2000:])
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def _oracle_rate(L, steps, warmup):
    """Run the oracle in one fresh single-threaded process; returns its record."""
    return _oracle_procs(L, steps, warmup, 1)[0]


def cpu_baseline(L, steps):
    """The oracle as it stands on the host cores: one single-threaded process, and
    one process per core (nproc) stepping its own copy of the same sample at the
    same time (whole-host throughput)."""
    one = _oracle_rate(L, steps, 1)
    ncores = os.cpu_count() or 1
    many = _oracle_procs(L, steps, 1, ncores)
    wall = max(r["t1"] for r in many) - min(r["t0"] for r in many)
    agg = sum(r["fluid"] * steps for r in many) / wall / 1e6
    return {"value": round(agg, 4), "unit": "MLUPS", "cores": ncores, "kind": "oracle",
            "sample": "FP64 numpy oracle, same pipe recipe at L=%d (%d fluid nodes), %d steps per "
                      "process, %d single-threaded processes at once (nproc), %.1f s wall"
                      % (L, one["fluid"], steps, ncores, wall),
            "single_thread": {"value": round(one["mlups"], 4), "cores": 1,
                              "seconds": round(one["seconds"], 2)}}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    # a sample size whose (steps + warmup) oracle steps end within ~2 minutes
    per_node_s = 0.8e-6
    budget = 120.0 / max(1, args.steps + args.warmup)
    L = 16
    for cand in (64, 48, 32, 16):
        if cand ** 3 * per_node_s <= budget:
            L = cand
            break
    res = _oracle_rate(L, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": round(res["mlups"], 4), "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["seconds"] * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("L=256", "L=%d" % args.L), "lattice": "D3Q19",
                       "L": args.L},
            "cpu_baseline": {"value": round(res["mlups"], 4), "unit": "MLUPS", "cores": 1,
                             "kind": "oracle",
                             "sample": "each step: one oracle step of the same pipe recipe at "
                                       "L=%d (%d fluid nodes), single thread" % (L, res["fluid"])},
            "e2e": {"value": round(res["mlups"], 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--accuracy-sizes", default="64,128,256")
    ap.add_argument("--accuracy-steps", type=int, default=20000)
    ap.add_argument("--adjoint-L", type=int, default=128)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--d3q15-steps", type=int, default=1000)
    ap.add_argument("--refine-max", type=int, default=1024)
    ap.add_argument("--tg-max", type=int, default=200)
    ap.add_argument("--tg-sizes", default="40,80,120,160,200")
    ap.add_argument("--tg-snu", default="1,1.99")
    ap.add_argument("--tg-shifts", default="0,0")
    ap.add_argument("--refine-max-steps", type=int, default=1500000)
    ap.add_argument("--refine-mlups-n", type=int, default=2048)
    ap.add_argument("--ensemble-count", type=int, default=96)
    ap.add_argument("--ensemble-steps", type=int, default=400)
    ap.add_argument("--cpu-L", type=int, default=48)
    ap.add_argument("--cpu-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
