#!/usr/bin/env python3
"""Benchmark of the OK-action W-form hot path on one GB300 (or N independent replicas).

A step is one pass of the whole path over the 16^3 x 32 workload (random SU(3) links, eps 0.2,
am0 0.5, Gaussian source), with inputs resident in HBM:
  precompute W from the links (mean plaquette / u0, clover, W matrices; an FP64-accurate
  double-float copy and an FP32 copy), BiCGStab solve of M x = b to a true FP64 residual
  |b - M x| / |b| < 1e-10 (FP32 iteration with reliable updates whose FP64-accurate residuals run
  in double-float arithmetic on the FP32 pipes), release of W.
`value` is the step's algorithmic HBM traffic (each byte a kernel must move, counted once; the
FP64-accurate work at FP64 bytes whatever its representation) divided by the step time, in GB/s:
a throughput of the whole step, not of the apply alone.  `roofline` describes the dominant kernel
(the FP32 application of M inside the solve, the metric's M.psi GB/s) timed with CUDA events on
its own stream during the timed steps.  `e2e` repeats the step through the public API with the
links and the source copied from pinned host memory and the solution copied back inside the timed
region.

Two further keys time the solve forms the metric compares with plain FP64 BiCGStab, outside the
timed steps: `multi_rhs` (20^3 x 64, the 12 spin-colour point sources of one propagator in one
lockstep solve on the tensor cores) and `large` (28^3 x 96, the same at 2.1 M sites, with the device
memory in use); each against plain FP64 BiCGStab timed on two of the sources and scaled to twelve.

--impl reference times the oracle (plain FP64 numpy CPU code) on the same workload and metric: each
step is one oracle application of M on the full lattice, its W evaluated once beforehand.
--oracle-solve times the oracle's BiCGStab on the 16^3 x 32 workload once (minutes of CPU).

Multi-GPU: one process per GPU under torch.distributed; each rank solves its own replica (its own
source), so the work per GPU is fixed ("scaling": "weak") and no data moves between ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("M·ψ HBM GB/s (% peak); time to 1e-10 solve, chosen form vs plain FP64 BiCGStab")
WORKLOAD = "16^3x32"
TOL = 1e-10
DELTA = 1e-4        # reliable-update threshold of the mixed solver (tuned on this workload)
CHECK_EVERY = 4

# Algorithmic bytes per site (each stored byte read once, each output written once).  FP64-accurate
# work is charged at FP64 bytes whatever representation carries it (the double-float copy holds
# each FP64 number as two floats; that is an implementation choice, not algorithmic traffic).
W64_BYTES = 43 * 9 * 16          # stored FP64 W per site
W32_BYTES = 43 * 9 * 8           # stored FP32 W per site
W16_BYTES = 43 * 9 * 4           # stored FP16 W per site
WTC_BYTES = 3216                 # the tensor-core FP16 copy per site (expanded blocks)
SPINOR64, SPINOR32 = 192, 96
LINKS64 = 4 * 9 * 16
APPLY64 = W64_BYTES + 2 * SPINOR64            # 6576: W + psi in + out
APPLY32 = W32_BYTES + 2 * SPINOR32            # 3288
RESID64 = APPLY64 + SPINOR64                  # true residual also reads b
PRECOMPUTE = {"mixed": LINKS64 + W64_BYTES + W32_BYTES,  # links in, the FP64-accurate and FP32 W out
              "f64": LINKS64 + W64_BYTES}
# FP32 vector traffic per BiCGStab iteration: <rhat, v> reads rhat (1); s = r - a v (3);
# x += a p + w s, r = s - w t with two dots (5 reads + 2 writes); p = r + b (p - w v) (4).
ITER_VEC32 = (1 + 3 + 7 + 4) * SPINOR32
ITER_VEC64 = (1 + 3 + 7 + 4) * SPINOR64
# Mixed-precision reliable update: x64 += x32 and x32 = 0 (2 + 2 vectors, one of each width),
# demotion r64 -> r32 with <rhat, r> (3), update of p (4 FP32 vectors).
RELIABLE32 = 2 * SPINOR64 + 2 * SPINOR32 + (SPINOR64 + 2 * SPINOR32) + 4 * SPINOR32
RESTART64 = 3 * SPINOR64
# The tensor-core multi-RHS apply, per site for nrhs right-hand sides: FP16 W (the compact 1548
# bytes of the stored set) + FP32 fields in and out.
def tc_apply_bytes(nrhs):
    return W16_BYTES + nrhs * 2 * SPINOR32


def solve_bytes(V, info, mode):
    """Algorithmic bytes of one solve from its counters."""
    it = info["iters"]
    if mode == "mixed":
        per_iter = 2 * APPLY32 + ITER_VEC32
        extra = info["fp64_applies"] * RESID64 + (info["reliable_updates"] + info["restarts"] + 1) * RELIABLE32
    else:
        per_iter = 2 * APPLY64 + ITER_VEC64
        extra = info["fp64_applies"] * RESID64 + (info["restarts"] + 1) * RESTART64
    return V * (it * per_iter + extra)


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["mixed", "f64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-forms", action="store_true", help="skip the multi_rhs and large solve-form keys")
    ap.add_argument("--oracle-solve", action="store_true", help="time the oracle's BiCGStab on 16^3 x 32 and exit")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- distributed
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def reduce_max_sum(times_ms, units, device=None):
    """(max over ranks of times_ms, sum over ranks of units); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(times_ms), float(units)
    t = torch.tensor([float(times_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock and throttle samples (every 200 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if _isnum(r[3]))
                if any(_isnum(r[3]) for r in rows) else None}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# ----------------------------------------------------------------------------- roofline inputs
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def apply_source_hash():
    h = hashlib.sha256()
    for f in ("ok_apply.cu", "ok_hops.cuh", "ok_pair.cuh", "ok_internal.cuh", "ok_reduce.cuh", "ok_launch.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1311_5029_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """DRAM bytes per launch recorded by the committed ncu summary, if it still matches the source."""
    path = os.path.join(ROOT, "profiles", "apply_f32_split_16x16x16x32.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_src = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(rf"{kernel_key}_dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_src or not m_b or m_src.group(1) != apply_source_hash():
        return None
    return float(m_b.group(1))


def roofline(trace, infos, key, bytes_per_launch, peak, peak_kind, traffic):
    """The roofline record of the apply class `key` from the trace ({class: (launches, ms)}) and the
    solves' info records.  Every executed iteration applies M twice (v = M p and t = M s; the classes
    key, key_dot and key_ts: plain or with a fused reduction); the other launches belong to
    iterations enqueued after the state halted, which return at once, so the classes' whole time is
    charged to the 2 x iterations launches that do the work.  Only the solves' applies are counted:
    the timed steps apply M nowhere else."""
    names = (key, key + "_dot", key + "_ts")
    n_apply = sum(v[0] for k, v in trace.items() if k in names)
    ms_apply = sum(v[1] for k, v in trace.items() if k in names)
    n_work = 2 * sum(i["iters"] for i in infos)
    avg_us = ms_apply / n_work * 1e3 if n_work else None
    achieved = bytes_per_launch / (avg_us * 1e-6) / 1e9 if n_work else None
    return {"kernel": key, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_source": peak_kind,
            "unit": "GB/s", "frac": achieved / peak if achieved else None, "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_per_launch, "launches": n_work,
            "launches_after_halt": n_apply - n_work, "avg_launch_us": avg_us}


# ----------------------------------------------------------------------------- oracle timing
def host_cpu():
    """(logical CPUs, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    import platform
    return os.cpu_count(), model or platform.processor() or platform.machine()


def oracle_quads(U, c):
    """The oracle's 27 W blocks of Eq. minFlopForm, evaluated once (outside any timed region)."""
    from oracle import wform
    return wform.quads(U, c)


def oracle_sample(quads_, b):
    """One oracle application of M with W already evaluated: (seconds, threads used)."""
    from oracle import wform
    c0 = time.process_time()
    t0 = time.perf_counter()
    wform.apply_quads(quads_, b, (1, 1, 1, 1))
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return wall, (max(1, round(cpu / wall)) if wall > 0 else 1)


def cpu_baseline(U, c, b, V, reps=5):
    """The oracle's W-form apply on the host cores: median of `reps` applications, W evaluated once."""
    q = oracle_quads(U, c)
    walls, cores = [], 1
    for _ in range(reps):
        w, cores = oracle_sample(q, b)
        walls.append(w)
    med = statistics.median(walls)
    nproc, model = host_cpu()
    return {"value": APPLY64 * V / med / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "nproc": nproc, "cpu_model": model, "seconds": [round(w, 3) for w in walls],
            "sample": f"median of {reps} oracle applications of M (FP64 numpy, W evaluated once beforehand, "
                      f"not timed) on the full {WORKLOAD} lattice, {med:.2f} s each, counted as one FP64 apply "
                      f"({APPLY64} B/site); {cores} of {nproc} host threads used"}


def oracle_solve():
    """The oracle's BiCGStab (FP64 numpy) on the 16^3 x 32 workload to a true residual of 1e-10."""
    import synth
    from oracle import bicgstab, wform
    dims, U, c, b = synth.workload_inputs(WORKLOAD)
    t0 = time.perf_counter()
    q = oracle_quads(U, c)
    tq = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, info = bicgstab.solve(lambda v: wform.apply_quads(q, v, (1, 1, 1, 1)), b, tol=TOL)
    ts = time.perf_counter() - t0
    nproc, model = host_cpu()
    return {"impl": "oracle", "workload": WORKLOAD, "tol": TOL, "solve_s": ts, "w_eval_s": tq,
            "iters": info["iters"], "true_relres": info["true_relres"], "nproc": nproc, "cpu_model": model}


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import synth
    import paper_1311_5029_gb300 as ok

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    dev = torch.device("cuda", local)
    ok.load()
    dims, U, c, b = synth.workload_inputs(WORKLOAD, source_seed=7 + rank)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    bc = (1, 1, 1, 1)
    U_d = torch.from_numpy(U).to(dev)
    b_d = torch.from_numpy(b).to(dev)
    precs = (ok.W_DF64 | ok.W_F32) if args.mode == "mixed" else ok.W_F64
    mode = ok.SOLVE_MIXED if args.mode == "mixed" else ok.SOLVE_F64

    def step(links, src):
        W = ok.precompute_W(links, c, bc, precs)
        x = torch.zeros_like(src)
        x, info = ok.bicgstab(W, src, x, tol=TOL, mode=mode, delta=DELTA, check_every=CHECK_EVERY)
        W.free()
        return x, info

    # plain FP64 BiCGStab on the same system: the comparison the metric names (untimed here;
    # its own time to solution comes from CUDA events around the call)
    plain = None
    if not args.no_plain and args.mode == "mixed":
        W = ok.precompute_W(U_d, c, bc, ok.W_F64)
        ok.bicgstab(W, b_d, tol=TOL, mode=ok.SOLVE_F64)         # warm-up (module loading, pools)
        times = []
        for _ in range(5):
            ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev_a.record()
            _, pinfo = ok.bicgstab(W, b_d, tol=TOL, mode=ok.SOLVE_F64, check_every=CHECK_EVERY)
            ev_b.record()
            torch.cuda.synchronize()
            times.append(ev_a.elapsed_time(ev_b))
        plain = {"solve_ms": statistics.median(times), "solve_ms_all": [round(t, 3) for t in times],
                 "timed_solves": len(times), "iters": pinfo["iters"], "true_relres": pinfo["true_relres"],
                 "residuals": "native FP64 W on the FP64 pipe"}
        W.free()

    for _ in range(args.warmup):
        step(U_d, b_d)
    torch.cuda.synchronize()

    ok.trace_reset()
    ok.trace_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    n0 = ok.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tot_bytes, infos = 0, []
    for _ in range(args.steps):
        _, info = step(U_d, b_d)
        infos.append(info)
        tot_bytes += V * PRECOMPUTE[args.mode] + solve_bytes(V, info, args.mode)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    launches = ok.launch_count() - n0
    clk = clocks.stop()
    ok.trace_enable(False)
    trace = ok.trace_read()
    local_ms = e0.elapsed_time(e1)
    ms_all, bytes_all = reduce_max_sum(local_ms, tot_bytes, dev)
    value = bytes_all / (ms_all * 1e-3) / 1e9
    ms_per_step = ms_all / args.steps

    # dominant kernel: the FP32 (or FP64) application of M inside the solve
    key = "apply_f32" if args.mode == "mixed" else "apply_f64"
    per_launch = APPLY32 if args.mode == "mixed" else APPLY64
    peak, peak_kind = measured_peaks()
    roof = roofline(trace, infos, key, per_launch * V, peak, peak_kind, ncu_traffic(key))
    step_ms = sum(v[1] for v in trace.values())
    shares = {k: round(v[1] / step_ms, 4) for k, v in sorted(trace.items(), key=lambda kv: -kv[1][1])} if step_ms else {}

    # end to end through the public API, host buffers in and out
    e2e = None
    if not args.no_e2e:
        U_h = torch.from_numpy(U).pin_memory()
        b_h = torch.from_numpy(b).pin_memory()
        x_h = torch.empty_like(b_h).pin_memory()
        U_e = torch.empty_like(U_d)
        b_e = torch.empty_like(b_d)
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        e2e_bytes = 0
        for _ in range(args.steps):
            U_e.copy_(U_h, non_blocking=True)
            b_e.copy_(b_h, non_blocking=True)
            x, info = step(U_e, b_e)
            x_h.copy_(x, non_blocking=True)
            e2e_bytes += V * PRECOMPUTE[args.mode] + solve_bytes(V, info, args.mode)
        f1.record()
        torch.cuda.synchronize()
        barrier()
        e_ms, e_bytes = reduce_max_sum(f0.elapsed_time(f1), e2e_bytes, dev)
        e2e = {"value": e_bytes / (e_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": e_ms / args.steps,
               "h2d_bytes_per_step": U_h.numel() * U_h.element_size() + b_h.numel() * b_h.element_size(),
               "d2h_bytes_per_step": x_h.numel() * x_h.element_size()}

    forms = {} if args.no_forms else run_forms(ok, torch, dev, peak, peak_kind)

    if rank != 0:
        return None
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(U, c, b, V)
    iters = [i["iters"] for i in infos]
    solve_ms = statistics.median(i["time_ms"] for i in infos)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+df64" if args.mode == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice_xyzt": list(dims), "sites": V, "links_eps": 0.2, "am0": 0.5,
                   "source": "gaussian", "tol": TOL,
                   "solver": (f"BiCGStab FP32 + FP64 reliable updates (delta {DELTA})" if args.mode == "mixed"
                             else "BiCGStab FP64"),
                   "step": ("precompute W (double-float FP64 + FP32) + solve to 1e-10 true residual + free W"
                            if args.mode == "mixed" else "precompute W (FP64) + solve to 1e-10 true residual + free W"),
                   "l2": "inputs larger than L2 (W = %.2f GB per step)" % (
                       V * ((2 * W64_BYTES + W32_BYTES) if args.mode == "mixed" else W64_BYTES) / 1e9),
                   "parallelism": f"replicas x{world}"},
        "value_is": ("algorithmic HBM bytes of the whole step (precompute + solve to 1e-10 + release) per second; "
                     "the M.psi GB/s of the dominant apply is roofline.achieved"),
        "roofline": roof,
        "percent_of_hbm_peak": 100.0 * value / peak,
        "kernel_time_shares": shares,
        "solve": {"iters_median": statistics.median(iters), "solve_ms_median": solve_ms,
                  "reliable_updates": infos[-1]["reliable_updates"], "true_relres": infos[-1]["true_relres"]},
        "plain_fp64": plain,
        "time_to_solution_ratio_plain_over_chosen": (plain["solve_ms"] / solve_ms) if plain else None,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
    }
    line.update(forms)
    return line


# ----------------------------------------------------------------------------- solve forms
def _spin_colour_sources(torch, dims, dev):
    """The 12 unit sources at site 0 (spin s, colour c -> source 3 s + c), [12, ..., 4, 3] complex128."""
    import synth
    V = dims[0] * dims[1] * dims[2] * dims[3]
    b = torch.zeros((12, V, 12), dtype=torch.complex128, device=dev)
    for k in range(12):
        b[k, 0, k] = 1.0
    return b.reshape((12,) + synth.lattice_shape(dims) + (4, 3))


def _events_ms(torch, fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def solve_form(ok, torch, dev, name, dims, eps, seed, am0, peak, peak_kind, delta=1e-4, tc_roofline=False):
    """Time to a true FP64 residual below 1e-10 for the 12 spin-colour point sources of one
    propagator: one lockstep multi-RHS solve on the tensor cores (FP16 operands, FP32 accumulation
    and vectors, an outer FP64 defect correction with double-float residuals, graph-captured
    iterations) against plain FP64 BiCGStab, timed on two of the sources and scaled to twelve."""
    import synth
    V = dims[0] * dims[1] * dims[2] * dims[3]
    c = synth.placeholder_coeffs(am0)
    bc = (1, 1, 1, 1)
    U = synth.device_random_links(dims, eps, seed, device=dev)
    b = _spin_colour_sources(torch, dims, dev)
    free0, total = torch.cuda.mem_get_info()
    Wc = ok.precompute_W(U, c, bc, ok.W_DF64 | ok.W_F16_TC)
    mode = ok.SOLVE_MIXED_TC | ok.SOLVE_DEFECT
    ok.bicgstab_multi(Wc, b[:2].contiguous(), tol=1e-2, mode=mode, delta=delta)   # warm-up
    ok.trace_reset()
    ok.trace_enable(True)
    ms, (x, infos) = _events_ms(torch, lambda: ok.bicgstab_multi(Wc, b, tol=TOL, mode=mode, delta=delta, check_every=8))
    ok.trace_enable(False)
    trace = ok.trace_read()
    free1, _ = torch.cuda.mem_get_info()
    resid = [ok.true_residual(Wc, b[k].contiguous(), x[k].contiguous()) for k in range(12)]
    del x
    Wc.free()
    Wp = ok.precompute_W(U, c, bc, ok.W_F64)
    ok.bicgstab(Wp, b[0].contiguous(), tol=1e-2, mode=ok.SOLVE_F64)                             # warm-up
    plain_ms, plain_it = [], []
    for k in (0, 11):
        t, (_, pinfo) = _events_ms(torch, lambda: ok.bicgstab(Wp, b[k].contiguous(), tol=TOL, mode=ok.SOLVE_F64,
                                                              check_every=CHECK_EVERY))
        plain_ms.append(t)
        plain_it.append(pinfo["iters"])
    Wp.free()
    plain12 = 6.0 * sum(plain_ms)
    out = {"workload": name, "sites": V, "links_eps": eps, "am0": am0, "sources": 12, "tol": TOL,
           "links": "drawn on the device (torch seeded generator, the host recipe's distribution)",
           "form": "multi-RHS tensor-core BiCGStab (FP16 operands, FP32 accumulation and vectors) inside an outer "
                   f"FP64 defect correction on the double-float W (delta {delta}), graph-captured iterations",
           "chosen_ms": ms, "iters": [i["iters"] for i in infos], "reliable_updates": [i["reliable_updates"] for i in infos],
           "true_relres_max": max(resid),
           "plain_fp64_ms": [round(t, 3) for t in plain_ms], "plain_fp64_iters": plain_it,
           "plain_fp64_timed_solves": 2, "plain_fp64_ms_12_scaled": plain12,
           "ratio_plain_over_chosen": plain12 / ms,
           "device_memory_in_use_gb": round((total - min(free0, free1)) / 1e9, 2) if free1 < free0 else None,
           "device_memory_held_by_solve_gb": round((free0 - free1) / 1e9, 2)}
    if tc_roofline:
        names = ("apply_tc_dot", "apply_tc_ts")
        n = sum(v[0] for k, v in trace.items() if k in names)
        t_ms = sum(v[1] for k, v in trace.items() if k in names)
        if n:
            us = t_ms / n * 1e3
            ach = tc_apply_bytes(12) * V / (us * 1e-6) / 1e9
            out["roofline_tc"] = {"kernel": "apply_tc (12 right-hand sides)", "bound": "hbm", "achieved": ach,
                                  "peak": peak, "peak_source": peak_kind, "unit": "GB/s", "frac": ach / peak,
                                  "traffic": None, "algorithmic_bytes_per_launch": tc_apply_bytes(12) * V,
                                  "stored_w_bytes_per_site": WTC_BYTES, "launches": n, "avg_launch_us": us,
                                  "timed": "CUDA events around the directly launched iterations of the solve "
                                           "(before its graph replays)"}
    return out


def run_forms(ok, torch, dev, peak, peak_kind):
    return {"multi_rhs": solve_form(ok, torch, dev, "20^3x64", (20, 20, 20, 64), 0.2, 13115031, 1.0, peak, peak_kind,
                                    tc_roofline=True),
            "large": solve_form(ok, torch, dev, "28^3x96", (28, 28, 28, 96), 0.15, 13115032, 0.8, peak, peak_kind)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    import synth
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    dims, U, c, b = synth.workload_inputs(WORKLOAD)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    q = oracle_quads(U, c)
    for _ in range(args.warmup):
        oracle_sample(q, b)
    walls, cores = [], 1
    for _ in range(args.steps):
        w, cores = oracle_sample(q, b)
        walls.append(w)
    total = sum(walls)
    value = args.steps * APPLY64 * V / total / 1e9
    nproc, model = host_cpu()
    sample = (f"each step one oracle application of M (FP64 numpy, W evaluated once before the steps) on the full "
              f"{WORKLOAD} lattice, counted as one FP64 apply ({APPLY64} B/site)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice_xyzt": list(dims), "sites": V},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "nproc": nproc, "cpu_model": model},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    if args.oracle_solve:
        print(json.dumps(oracle_solve()), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            dist.destroy_process_group()
    except Exception:
        pass


if __name__ == "__main__":
    main()
