#!/usr/bin/env python
"""Benchmark: effective TFLOPS and seconds per 2^k-amplitude batch of the sliced contraction.

One step = one tn_contract over all 16 slices of the 30-qubit 5x6-grid 14-cycle Sycamore-shaped
circuit (10 open qubits: one batch of 1024 amplitudes), inputs resident in HBM.  Effective
TFLOPS = sum over slices and steps of T_cc (8 flops per complex multiply-add, Eq. T_cc) / time.
The headline runs the FP16-scaled tensor-core path; the complex64 CUDA-core path is timed in the
same run for comparison ("mixed vs c64").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode M]

Under torchrun every rank contracts its own amplitude batch (the same circuit with different
seeded closed bits: same work, weak scaling); the time is the maximum over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective TFLOPS & s per 2^k-amplitude batch, mixed vs c64, at XEB err ≤1e-3"
WORKLOAD = "sycamore_5x6_c14_open10_s4"
TC_SOURCE = os.path.join(ROOT, "paper_2310_03978_gb300", "csrc", "tn_gemm_tc.cu")
SIMT_SOURCE = os.path.join(ROOT, "paper_2310_03978_gb300", "csrc", "tn_gemm_simt.cu")
PROFILE_SUMMARY = {"gemm_tc": os.path.join(ROOT, "profiles", "gemm_tc_" + WORKLOAD + ".md"),
                   "gemm_simt": os.path.join(ROOT, "profiles", "gemm_simt_" + WORKLOAD + ".md")}
FP32_LANES_PER_SM = 128
NUM_SMS = 152


SA_SEED = 7  # annealing seed of the optimised-path measurement

def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fp16_scaled")
    ap.add_argument("--gemm-form", default="auto",
                    help="auto, 4m or 3m (the single-step microbench takes a comma list)")
    ap.add_argument("--tc-bk", type=int, default=0, choices=[0, 32, 64])
    ap.add_argument("--tc-bn", type=int, default=0, choices=[0, 128, 256])
    ap.add_argument("--mixed-topk", type=int, default=0,
                    help="mode mixed: tensor-core steps (largest T_cc first) kept single-pass FP16")
    ap.add_argument("--eps-budget", type=float, default=0.0,
                    help="predicted amplitude error budget of the precision policy (0 = the "
                         "mode's default)")
    ap.add_argument("--c64-steps", type=int, default=2)
    ap.add_argument("--bf16-steps", type=int, default=2,
                    help="steps of the BF16-scaled arm (error-budgeted policy); 0 = skip")
    ap.add_argument("--split-steps", type=int, default=2,
                    help="steps of the compensated FP16 (3xFP16) tensor-core arm; 0 = skip")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: plans time every tensor-core variant on their first batch")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: each rank contracts its own amplitude batch; strong: the ranks "
                         "split one batch's slices and sum-reduce the amplitudes (FP64)")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: time the headline steps as CUDA-graph replays and measure the "
                         "dominant kernel in a separate profiled pass of the same steps")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--sa-alpha", type=float, default=512.0,
                    help="weight of the memory term T_mc in the annealing score (multiply-adds "
                         "per element moved)")
    ap.add_argument("--small-steps", type=int, default=50,
                    help="also time the 12-qubit circuit (64 amplitudes, complex64); 0 = skip")
    ap.add_argument("--sycamore53", type=int, default=0,
                    help="time this many batches of slices of the 53-qubit 16-cycle circuit "
                         "(annealed path, slices capped at 2^30 elements) and extrapolate to "
                         "all slices; prints its own JSON line")
    ap.add_argument("--sycamore53-modes", default="",
                    help="comma-separated precision modes for --sycamore53 (default: --mode)")
    ap.add_argument("--table3", action="store_true",
                    help="the Table 3 shape on the 45-qubit 14-cycle circuit (time and eps_L2^2 "
                         "against the number of single-pass dense steps; error budgets)")
    ap.add_argument("--table3-slices", type=int, default=1024,
                    help="contiguous slices timed per row of --table3")
    ap.add_argument("--c53-cycles", type=int, default=16, choices=[16, 20],
                    help="cycles of the 53-qubit circuit for --sycamore53 / --step-profile")
    ap.add_argument("--config4-batches", type=int, default=2,
                    help="53-qubit 16-cycle circuit: batches of slices timed per mode in the "
                         "default run (0 = skip)")
    ap.add_argument("--config4-modes", default="fp16_scaled:0.001,fp16_scaled,split_bf16,c64",
                    help="precision modes of the 53-qubit 16-cycle arms; mode:budget gives the "
                         "precision policy an error budget")
    ap.add_argument("--config5-slices", type=int, default=256,
                    help="53-qubit 20-cycle circuit: contiguous slices timed for the first mode "
                         "(a quarter of them for the others, one batch for complex64; 0 = skip)")
    ap.add_argument("--config5-modes", default="fp16_scaled:0.001,fp16_scaled,c64")
    ap.add_argument("--sycamore53-compare", type=int, default=8,
                    help="contributing slices compared with complex64 under --sycamore53")
    ap.add_argument("--sparse-only", action="store_true",
                    help="run only the sparse-state measurement and print its JSON line")
    ap.add_argument("--sparse-steps", type=int, default=3,
                    help="also time a sparse-state contraction (24-qubit circuit, all qubits "
                         "open, 4096 sampled bitstrings); 0 = skip")
    ap.add_argument("--sa-greedy-trials", type=int, default=20,
                    help="random greedy initial trees per annealing chain of the annealed path")
    ap.add_argument("--sa-budget", type=float, default=1e-3,
                    help="predicted amplitude error budget of the annealed path's plan")
    ap.add_argument("--sa-steps", type=int, default=3,
                    help="also time the bench circuit along an annealed path with dynamic "
                         "slicing (same amplitudes, less work); 0 = skip")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--feed-tc", action="store_true",
                    help="single-step microbench: the step's result feeds a second tensor-core "
                         "step, so it is written as scaled planar 16-bit numbers")
    ap.add_argument("--step-profile", type=int, default=0,
                    help="per-step roofline of the circuit workload: print the N slowest steps")
    ap.add_argument("--thin-tc", type=int, default=0, choices=[-1, 0, 1],
                    help="streaming steps on the tensor cores: 0 automatic, 1 all that fit, "
                         "-1 none")
    ap.add_argument("--step", default=None,
                    help="single-step microbench 'lm,ln,lk' (log2 of m, n, k) instead of the "
                         "circuit: one random dense contraction with shuffled label orders")
    return ap.parse_args()


def peaks():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------------- workload
def dominant_step(wl):
    from paper_2310_03978_gb300 import workload as W
    steps = W.replay_path(wl.network.labels, wl.network.open_labels, wl.path, wl.sliced)
    return max(range(len(steps)), key=lambda i: steps[i].tcc), steps


# ---------------------------------------------------------------------------------- CPU oracle
def oracle_sample(wl, seconds):
    """Time the CPU oracle on a bounded sample of the workload: the dominant contraction step
    (random operands with its labels) restricted to a sub-block of its output by fixing all but
    `keep` of the free labels of A and B, with `keep` grown until the sample takes about
    `seconds`."""
    from oracle import oracle as O
    di, steps = dominant_step(wl)
    st = steps[di]
    rng = np.random.default_rng(12345)
    lk = len(st.k_labels)
    fa = [l for l in st.labels_a if l not in st.k_labels]
    fb = [l for l in st.labels_b if l not in st.k_labels]
    order = [x for pair in zip(fa, fb) for x in pair] + fa[len(fb):] + fb[len(fa):]

    def run(keep):
        kept = set(order[:keep])
        la = [l for l in st.labels_a if l in kept or l in st.k_labels]
        lb = [l for l in st.labels_b if l in kept or l in st.k_labels]
        A = rng.standard_normal((2,) * len(la)) + 1j * rng.standard_normal((2,) * len(la))
        B = rng.standard_normal((2,) * len(lb)) + 1j * rng.standard_normal((2,) * len(lb))
        out = [l for l in st.labels_out if l in kept]
        t0 = time.perf_counter()
        O.einsum_pair(A, la, B, lb, out)
        dt = time.perf_counter() - t0
        return dt, 8.0 * 2 ** len(out) * 2 ** lk, 2 ** len(out)

    keep = 3
    dt, fl, outs = run(keep)
    while dt < 0.5 and keep < len(order):
        keep += 1
        dt, fl, outs = run(keep)
    rate = fl / dt
    while keep < len(order) and fl * 2 / rate <= seconds:
        keep += 1
        fl *= 2
    dt, fl, outs = run(keep)
    rate = fl / dt
    return {"seconds": dt, "flops": fl, "rate": rate, "outputs": outs,
            "fixed_labels": len(order) - keep, "step": di, "threads": O.num_threads(),
            "shape": "m=2^%d n=2^%d k=2^%d" % (len(st.m_labels), len(st.n_labels), lk)}


def oracle_small_circuit(repeats):
    """The whole oracle contraction of the 12-qubit 3x4 8-cycle circuit (its 64 amplitudes, the
    plain complex64 configuration): seconds of each of ``repeats`` runs."""
    from oracle import oracle as O
    from paper_2310_03978_gb300 import workload as W
    wl = W.small_workload()
    O.contract_network(wl.network, wl.path)  # warm
    out = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        O.contract_network(wl.network, wl.path)
        out.append(time.perf_counter() - t0)
    return out


def oracle_child(task, threads):
    """Run an oracle timing (``task``: {"kind": "sample", "seconds": s} or {"kind": "small",
    "repeats": r}) in a child process with OMP_NUM_THREADS = ``threads`` (None: all cores), so
    the oracle's thread pool is sized at load; returns the child's JSON result."""
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child",
                        json.dumps(task)], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_child(spec):
    from oracle import oracle as O
    from paper_2310_03978_gb300 import workload as W
    task = json.loads(spec)
    if task["kind"] == "sample":
        smp = oracle_sample(W.bench_workload(), task["seconds"])
        print(json.dumps({"rate": smp["rate"], "seconds": smp["seconds"],
                          "outputs": smp["outputs"], "threads": smp["threads"],
                          "shape": smp["shape"]}))
    else:
        secs = oracle_small_circuit(task["repeats"])
        print(json.dumps({"seconds": secs, "median_s": statistics.median(secs),
                          "threads": O.num_threads()}))


# ---------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "tn_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------- helpers
def profile_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    path = PROFILE_SUMMARY.get(kernel)
    src = TC_SOURCE if kernel == "gemm_tc" else SIMT_SOURCE
    if not path or not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    traffic, src_sha = None, None
    for line in open(path):
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1].split()[0])
        if line.startswith("source_sha256_16:"):
            src_sha = line.split(":", 1)[1].strip()
    return traffic if src_sha == sha else None


# ---------------------------------------------------------------------------------- accuracy
# Stored expected amplitudes (tests/golden, written by tests/golden/make_golden.py from the CPU
# oracle's state vector) and the error measures the lines report; the oracle itself runs here only
# in the CPU-baseline leg and the reference arm.
def golden_amps(name):
    path = os.path.join(ROOT, "tests", "golden", name + ".amps.txt")
    if not os.path.exists(path):
        return None
    rows = np.loadtxt(path, comments="#")
    return rows[:, 0] + 1j * rows[:, 1]


def read_golden():
    return golden_amps(WORKLOAD)


def rel_l2(a, ref):
    """||a - ref||_2 / ||ref||_2 over the batch."""
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    ref = np.asarray(ref, dtype=np.complex128).reshape(-1)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def max_entry_err(a, ref):
    """max |a - ref| / max |ref|: the largest error of one amplitude, relative to the largest
    amplitude."""
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    ref = np.asarray(ref, dtype=np.complex128).reshape(-1)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def eps_l2sq(a, ref):
    """Relative error of the squared L2 norm (Eq. l2_squared_error)."""
    l2 = float(np.sum(np.abs(np.asarray(ref).reshape(-1)) ** 2))
    return abs(l2 - float(np.sum(np.abs(np.asarray(a).reshape(-1)) ** 2))) / l2


def xeb_ideal(amps, n_qubits):
    """XEB of ideal samples from the amplitudes: 2^n sum p^2 / sum p - 1, p = |amplitude|^2."""
    p = np.abs(np.asarray(amps).reshape(-1)) ** 2
    return float(2.0 ** n_qubits * np.sum(p * p) / np.sum(p) - 1.0)


def p2_over_p(amps):
    """sum p^2 / sum p over the amplitudes (p = |a|^2): (ideal-sample XEB + 1) / 2^n."""
    p = np.abs(np.asarray(amps).reshape(-1)) ** 2
    return float(np.sum(p * p) / np.sum(p))


def time_steps(torch, step, steps, stream):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        step()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end)


def time_each(torch, step, steps, stream):
    """CUDA-event time of each of ``steps`` calls (ms), recorded on ``stream`` around each."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        step()
        ev[i + 1].record(stream)
    ev[-1].synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]


def time_contract(torch, plan, amps, steps, stream):
    return time_steps(torch, lambda: plan.contract(amps, stream=stream), steps, stream)


def kernel_roofline(plan, step_index, before, slices_per_launch, tcc, peak, bound, unit,
                    traffic):
    after = plan.step_info(step_index)
    n = after["launches"] - before["launches"]
    t = after["time_ms"] - before["time_ms"]
    if n <= 0 or t <= 0:
        return None
    avg_s = t / n / 1e3
    achieved = tcc * slices_per_launch / avg_s / 1e12
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "kernel": after["kernel_name"],
            "avg_launch_ms": avg_s * 1e3, "launches": n,
            "flops_per_launch": tcc * slices_per_launch}


# ---------------------------------------------------------------------------------- arms
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2310_03978_gb300 import shard, tn, workload as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    wl = W.bench_workload()
    strong = args.scaling == "strong"
    net_w = wl.network if strong else shard.rank_network(wl, rank)
    s_begin, s_end = shard.slice_range(wl.num_slices, rank, world) if strong else (0, None)
    n_open = len(net_w.open_labels)
    pk = peaks()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        return shard.max_over_ranks(x, device=dev)

    def contract(plan, amps):
        # one step: this rank's slices (all of its own batch, or its range of the shared
        # batch followed by the FP64 sum-reduce of the amplitudes)
        plan.contract(amps, s_begin, s_end, stream=stream)
        if strong:
            shard.reduce_amplitudes(amps)

    net = tn.Network.from_workload(net_w)

    def measure(mode, steps, warmup, clocks=False, graph=False, topk=None, budget=None):
        topk = args.mixed_topk if topk is None else topk
        budget = args.eps_budget if budget is None else budget
        if graph:
            # headline: graph replays, no per-kernel events; the roofline comes from a profiled
            # pass of the same number of steps right after
            gplan = tn.Plan(net, wl.path, wl.sliced, mode=mode, use_graph=True,
                            autotune=bool(args.autotune), mixed_topk=topk, eps_budget=budget)
            amps = torch.zeros(1 << n_open, dtype=torch.complex128, device=dev)
            for _ in range(warmup):
                contract(gplan, amps)
            torch.cuda.synchronize()
            launches0 = gplan.info()["kernel_launches"]
            sampler = ClockSampler(local_rank) if clocks else None
            if sampler:
                sampler.start()
                time.sleep(0.5)
            barrier()
            torch.cuda.synchronize()
            each = time_each(torch, lambda: contract(gplan, amps), steps, stream)
            gms = sum(each)
            torch.cuda.synchronize()
            barrier()
            gclk = sampler.stop() if sampler else None
            glaunch = (gplan.info()["kernel_launches"] - launches0) // steps
            gplan.close()
            del amps
            res = measure(mode, steps, 1, clocks=False, graph=False, topk=topk, budget=budget)
            res["ms_profiled"] = res["ms"]
            res["ms"] = max_over_ranks(gms) / steps
            res["clocks"] = gclk
            res["launches"] = glaunch
            res["graph"] = True
            res["each_ms"] = each
            return res
        plan = tn.Plan(net, wl.path, wl.sliced, mode=mode, profile=True,
                       autotune=bool(args.autotune), mixed_topk=topk, eps_budget=budget)
        info = plan.info()
        amps = torch.zeros(1 << n_open, dtype=torch.complex128, device=dev)
        # correctness pass (not timed)
        contract(plan, amps)
        torch.cuda.synchronize()
        result = amps.cpu().numpy().copy()
        for _ in range(warmup):
            contract(plan, amps)
        torch.cuda.synchronize()
        kinds = [plan.step_info(i) for i in range(info["num_steps"])]
        variants = {i: k["tc_variant"] for i, k in enumerate(kinds) if k["tc_variant"] >= 0}
        dom = max((i for i in range(len(kinds)) if kinds[i]["kernel_name"] in
                   ("gemm_tc", "gemm_simt")), key=lambda i: kinds[i]["tcc"])
        before = plan.step_info(dom)
        launches0 = plan.info()["kernel_launches"]
        sampler = ClockSampler(local_rank) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.5)
        barrier()
        torch.cuda.synchronize()
        ms = time_steps(torch, lambda: contract(plan, amps), steps, stream)
        torch.cuda.synchronize()
        barrier()
        clk = sampler.stop() if sampler else None
        ms = max_over_ranks(ms)
        launches = plan.info()["kernel_launches"] - launches0
        flops = info["tcc_per_slice"] * info["num_slices"] + info["tcc_invariant"]
        kname = kinds[dom]["kernel_name"]
        if kname == "gemm_tc":
            peak, bound, unit = pk["bf16_tflops_sustained"], "tensor", "TFLOP/s"
        else:
            peak = NUM_SMS * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
            bound, unit = "alu", "TFLOP/s"
        roof = kernel_roofline(plan, dom, before, info["slices_in_flight"], kinds[dom]["tcc"],
                               peak, bound, unit, profile_traffic(kname))
        plan.close()
        return {"ms": ms / steps, "flops": flops, "info": info, "result": result,
                "roofline": roof, "launches": launches // steps, "clocks": clk, "steps": steps,
                "graph": False, "variants": variants}

    head = measure(args.mode, args.steps, args.warmup, clocks=True, graph=bool(args.graph))
    c64 = measure("c64", args.c64_steps, 1) if args.c64_steps > 0 else None
    split = measure("split_fp16", args.split_steps, 1) if args.split_steps > 0 else None
    bf16 = (measure("bf16_scaled", args.bf16_steps, 1, topk=0, budget=0.0)
            if args.bf16_steps > 0 and args.mode != "bf16_scaled" else None)

    # the same circuit along a path from the annealing optimiser (Sec. 3.2) with dynamic slicing
    # to the same 2^28 cap: the same amplitudes with a fraction of the work
    sa = None
    if world == 1 and args.sa_steps > 0:
        t0 = time.perf_counter()
        sa_path, sa_sliced, sa_info = tn.path_optimize(
            wl.network.labels, wl.network.open_labels, wl.path, seed=SA_SEED, sweeps=1000,
            sweeps_per_slice=40, sweeps_final=500, t_start=0.03, t_end=0.001,
            max_log2_size=28, chains=16, alpha=args.sa_alpha,
            greedy_trials=args.sa_greedy_trials)
        sa_opt_s = time.perf_counter() - t0
        # single-pass FP16 on every dense step of an annealed path can miss the 1e-3 ideal-XEB
        # bar (1.6e-3 on the greedy-started one): the error budget keeps the predicted amplitude
        # error at sa_budget, single-pass on the largest steps, the rest compensated
        sa_mode = args.mode
        sa_topk = args.mixed_topk
        splan = tn.Plan(net, sa_path, sa_sliced, mode=sa_mode, use_graph=True,
                        autotune=bool(args.autotune), mixed_topk=sa_topk,
                        eps_budget=args.sa_budget)
        amps = torch.zeros(1 << n_open, dtype=torch.complex128, device=dev)
        splan.contract(amps, stream=stream)
        torch.cuda.synchronize()
        sa_result = amps.cpu().numpy().copy()
        for _ in range(max(3, args.warmup)):
            splan.contract(amps, stream=stream)
        torch.cuda.synchronize()
        sms = time_steps(torch, lambda: splan.contract(amps, stream=stream), args.sa_steps,
                         stream) / args.sa_steps
        si = splan.info()
        splan.close()
        del amps
        sa = {"mode": sa_mode, "topk": sa_topk, "single_pass": si["num_single_pass"],
              "compensated": si["num_compensated"], "eps_predicted": si["eps_predicted"],
              "ms": sms, "flops": si["tcc_per_slice"] * si["num_slices"] + si["tcc_invariant"],
              "slices": si["num_slices"], "max_log2": si["max_log2_size"], "opt_s": sa_opt_s,
              "info": sa_info, "result": sa_result}

    # the 12-qubit circuit (3x4 grid, 8 cycles, 64 amplitudes) on the complex64 path: latency of
    # one small batch, checked against the state vector
    small = None
    if world == 1 and args.small_steps > 0:
        wl_s = W.small_workload()
        tnet_sm = tn.Network.from_workload(wl_s.network)
        splan = tn.Plan(tnet_sm, wl_s.path, wl_s.sliced, mode="c64", use_graph=True)
        amps = torch.zeros(1 << len(wl_s.network.open_labels), dtype=torch.complex128, device=dev)
        splan.contract(amps, stream=stream)
        torch.cuda.synchronize()
        sm_result = amps.cpu().numpy().copy()
        for _ in range(3):
            splan.contract(amps, stream=stream)
        torch.cuda.synchronize()
        sm_ms = time_steps(torch, lambda: splan.contract(amps, stream=stream), args.small_steps,
                           stream) / args.small_steps
        sm_launch = splan.info()["kernel_launches"]
        splan.close()
        tnet_sm.close()
        del amps
        sm_ref = golden_amps("sycamore_3x4_c8_open6")
        small = {"workload": "sycamore_3x4_c8_open6", "mode": "c64", "us_per_batch": sm_ms * 1e3,
                 "steps": args.small_steps,
                 "amp_rel_l2_vs_statevector": (rel_l2(sm_result, sm_ref)
                                               if sm_ref is not None else None)}

    # open-qubit amplitude batches in one launch: the same 12-qubit circuit with every qubit open
    # and six of them sliced, 64 batches of 64 amplitudes per call (graph replay)
    amp_batches = None
    if world == 1 and args.small_steps > 0:
        wl_s = W.small_workload()
        net_b = W.build_network(wl_s.circuit, list(range(wl_s.circuit.n_qubits)), {})
        path_b = W.greedy_path(net_b.labels, net_b.open_labels)
        tnet_b = tn.Network(net_b.tensors, net_b.labels, net_b.open_labels)
        bplan = tn.Plan(tnet_b, path_b, net_b.open_labels[:6], mode="c64", use_graph=True)
        amps = torch.zeros(1 << len(net_b.open_labels), dtype=torch.complex128, device=dev)
        bplan.contract(amps, stream=stream)
        torch.cuda.synchronize()
        b_result = amps.cpu().numpy().copy()
        for _ in range(3):
            bplan.contract(amps, stream=stream)
        torch.cuda.synchronize()
        b_ms = time_steps(torch, lambda: bplan.contract(amps, stream=stream), args.small_steps,
                          stream) / args.small_steps
        b_info = bplan.info()
        bplan.close()
        tnet_b.close()
        del amps
        b_ref = golden_amps("sycamore_3x4_c8_all_open")
        amp_batches = {"workload": "sycamore_3x4_c8_all_open: 12 qubits open, 6 sliced",
                   "mode": "c64", "batches": b_info["num_slices"], "amplitudes_per_batch": 64,
                   "slices_in_flight": b_info["slices_in_flight"], "us_per_call": b_ms * 1e3,
                   "us_per_64_amplitudes": b_ms * 1e3 / b_info["num_slices"],
                   "amp_rel_l2_vs_statevector": (rel_l2(b_result, b_ref)
                                                 if b_ref is not None else None)}

    # sparse-state contraction (Sec. 3.3): the amplitudes of 4096 sampled bitstrings of a
    # 24-qubit circuit with every qubit open, along an annealed path
    sparse = measure_sparse(args, dev, stream) if world == 1 and args.sparse_steps > 0 else None

    # the 53-qubit configurations (Sec. 5 / Table 5 shapes): 16 cycles, a few batches of slices
    # per mode; 20 cycles, a contiguous range of slices extrapolated to all of them
    c53 = {}
    if world == 1 and args.config4_batches > 0:
        c53["config4"] = measure_c53(args, 16, [m for m in args.config4_modes.split(",") if m],
                                     batches=args.config4_batches, compare=8,
                                     profile_mode=("fp16_scaled:0.001", "fp16_scaled"))
    if world == 1 and args.config5_slices > 0:
        modes5 = [m for m in args.config5_modes.split(",") if m]
        c53["config5"] = measure_c53(args, 20, modes5,
                                     slices={m: (0 if m.startswith("c64") else
                                                 args.config5_slices if i == 0 else
                                                 max(1, args.config5_slices // 4))
                                             for i, m in enumerate(modes5)},
                                     batches=1, compare=8)

    # end to end through the host-buffer entry points: set the network's numbers (H2D) and
    # contract into a host array (D2H), every step
    plan = tn.Plan(net, wl.path, wl.sliced, mode=args.mode, mixed_topk=args.mixed_topk,
                   eps_budget=args.eps_budget)
    host_out = np.zeros(1 << n_open, dtype=np.complex128)
    plan.contract_host(s_begin, s_end, out=host_out)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.e2e_steps)
    for _ in range(e2e_steps):
        net.set_data(net_w.tensors)
        plan.contract_host(s_begin, s_end, out=host_out, stream=stream)
        if strong:
            red = torch.from_numpy(host_out)
            if world > 1:
                red = red.to(dev)
                shard.reduce_amplitudes(red)
                host_out[:] = red.cpu().numpy()
    e2e_s = max_over_ranks(time.perf_counter() - t0) / e2e_steps
    plan.close()

    golden = read_golden() if rank == 0 else None
    acc = {}
    if golden is not None:
        for name, r in (("head", head), ("c64", c64), ("split_fp16", split),
                        ("bf16_scaled", bf16), ("annealed_path", sa)):
            if r is None:
                continue
            x_ref = xeb_ideal(golden, wl.circuit.n_qubits)
            x_got = xeb_ideal(r["result"], wl.circuit.n_qubits)
            acc[name] = {"amp_rel_l2": rel_l2(r["result"], golden),
                         "amp_max_rel": max_entry_err(r["result"], golden),
                         "eps_l2sq": eps_l2sq(r["result"], golden),
                         "xeb_ideal_rel_err": abs(x_got - x_ref) / abs(x_ref)}
            if "eps_predicted" in r.get("info", {}):
                acc[name]["eps_predicted"] = r["info"]["eps_predicted"]
                acc[name]["single_pass_steps"] = r["info"]["num_single_pass"]
                acc[name]["compensated_steps"] = r["info"]["num_compensated"]
    if rank != 0:
        return
    batches = 1 if strong else world
    tflops = batches * head["flops"] / (head["ms"] / 1e3) / 1e12
    line = {
        "metric": METRIC,
        "value": tflops,
        "unit": "TFLOPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms"],
        "ms_per_step_median": statistics.median(head["each_ms"]) if head.get("each_ms") else None,
        "ms_per_step_min_max": ([min(head["each_ms"]), max(head["each_ms"])]
                                if head.get("each_ms") else None),
        "s_per_batch": head["ms"] / 1e3,
        "higher_is_better": True,
        "scaling": args.scaling,
        "vs_baseline": None,
        "dtype": {"fp16_scaled": "f16", "bf16_scaled": "bf16", "c64": "f32"}.get(args.mode,
                                                                                  args.mode),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "qubits": wl.circuit.n_qubits, "cycles": 14,
                   "open_qubits": n_open, "slices": head["info"]["num_slices"],
                   "slices_in_flight": head["info"]["slices_in_flight"],
                   "max_intermediate_log2": head["info"]["max_log2_size"], "mode": args.mode,
                   **({"mixed_topk": max(1, args.mixed_topk)} if args.mode == "mixed" else {}),
                   "flops_per_batch": head["flops"],
                   "l2": "inputs larger than L2 (largest intermediate 2^28 x 8 B per slice)",
                   "cuda_graph": head["graph"],
                   "tc_variants_by_step": head.get("variants"),
                   "ms_per_step_without_graph": head.get("ms_profiled")},
        "roofline": head["roofline"],
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "e2e": {"value": batches * head["flops"] / e2e_s / 1e12, "unit": "TFLOPS",
                "s_per_batch": e2e_s, "h2d_bytes_per_step": net.data_bytes,
                "d2h_bytes_per_step": (1 << n_open) * 16},
        "accuracy": acc,
    }
    if c64 is not None:
        line["c64"] = {"value": batches * c64["flops"] / (c64["ms"] / 1e3) / 1e12,
                       "unit": "TFLOPS", "ms_per_step": c64["ms"], "steps": c64["steps"],
                       "roofline": c64["roofline"]}
        line["mixed_over_c64"] = c64["ms"] / head["ms"]
    if bf16 is not None:
        line["bf16_scaled"] = {"value": batches * bf16["flops"] / (bf16["ms"] / 1e3) / 1e12,
                               "unit": "TFLOPS", "ms_per_step": bf16["ms"],
                               "steps": bf16["steps"], "roofline": bf16["roofline"],
                               "single_pass_steps": bf16["info"]["num_single_pass"],
                               "compensated_steps": bf16["info"]["num_compensated"]}
    if split is not None:
        line["split_fp16"] = {"value": batches * split["flops"] / (split["ms"] / 1e3) / 1e12,
                              "unit": "TFLOPS", "ms_per_step": split["ms"],
                              "steps": split["steps"], "roofline": split["roofline"]}
    if sa is not None:
        line["annealed_path"] = {
            "s_per_batch": sa["ms"] / 1e3, "speedup_s_per_batch": head["ms"] / sa["ms"],
            "effective_tflops": sa["flops"] / (sa["ms"] / 1e3) / 1e12,
            "flops_per_batch": sa["flops"], "slices": sa["slices"],
            "max_intermediate_log2": sa["max_log2"], "steps": args.sa_steps,
            "mode": sa["mode"], "eps_budget": args.sa_budget,
            "single_pass_steps": sa["single_pass"], "compensated_steps": sa["compensated"],
            "eps_predicted": sa["eps_predicted"],
            "optimiser_s": sa["opt_s"], "optimiser": "tn_path_optimize seed %d, 16 chains, "
            "%d random greedy trees per chain, 1000 + 40 per slice + 500 sweeps, "
            "T 0.03 -> 0.001, alpha %g, beta 0, cap 2^28"
            % (SA_SEED, args.sa_greedy_trials, args.sa_alpha)}
    if small is not None:
        line["small_circuit"] = small
    if amp_batches is not None:
        if small is not None:
            amp_batches["speedup_over_one_batch_per_call"] = (
                small["us_per_batch"] / amp_batches["us_per_64_amplitudes"])
        line["amplitude_batches"] = amp_batches
    for key, cycles in (("config4", 16), ("config5", 20)):
        if key in c53:
            line[key] = {"workload": "sycamore53_6x9_c%d_open12" % cycles, "qubits": 53,
                         "cycles": cycles, "open_qubits": 12, **c53[key]}
    if sparse is not None:
        line["sparse_state"] = sparse_line(args, sparse)
    if world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(wl, args.cpu_seconds)
        one = oracle_child({"kind": "sample", "seconds": args.cpu_seconds / 2}, 1)
        sm_all = oracle_child({"kind": "small", "repeats": 5}, None)
        sm_one = oracle_child({"kind": "small", "repeats": 5}, 1)
        line["cpu_baseline"] = {
            "value": smp["rate"] / 1e12, "unit": "TFLOPS", "cores": smp["threads"],
            "kind": "oracle",
            "sample": "oracle einsum of the dominant step (%s) on %d output elements "
                      "(%d free labels fixed), %.1f s; s per batch extrapolated %.1f"
                      % (smp["shape"], smp["outputs"], smp["fixed_labels"], smp["seconds"],
                         head["flops"] / smp["rate"]),
            "one_core": ({"value": one["rate"] / 1e12, "unit": "TFLOPS", "cores": one["threads"],
                          "sample": "the same step on %d output elements, %.1f s"
                                    % (one["outputs"], one["seconds"]),
                          "s_per_batch_extrapolated": head["flops"] / one["rate"]}
                         if "rate" in one else one),
            "small_circuit": {
                "workload": "sycamore_3x4_c8_open6 (64 amplitudes), whole oracle contraction",
                "s_per_batch_median": sm_all.get("median_s"), "cores": sm_all.get("threads"),
                "s_per_batch_median_one_core": sm_one.get("median_s"), "repeats": 5,
                "gpu_us_per_batch": small["us_per_batch"] if small else None}}
    print(json.dumps(line))


from paper_2310_03978_gb300.slice_support import (slice_constraints, slice_supported,  # noqa: E402,F401
                                                    supported_slices)


def sycamore53_path(cycles=16, sweeps=None, retune=None):
    """The 53-qubit network (6x9 grid without site (5, 8), 12 open qubits) of ``cycles`` cycles
    and its path (``stored_path``)."""
    return stored_path("sycamore53_6x9_c%d_open12" % cycles, sweeps, retune)


def stored_path(name, sweeps=None, retune=None):
    """A named large workload's network and its path: the stored one (``paths/make_paths.py``)
    unless an annealing effort is given, else 100 random greedy trees per chain and ``sweeps``
    annealing sweeps (16 chains), then dynamic slicing to the size cap with ``retune``
    re-tuning sweeps per sliced bond.  Returns (network, path, sliced labels, description)."""
    from paper_2310_03978_gb300 import tn, workload as W
    from paper_2310_03978_gb300.paths import make_paths as MP
    _, cap, d_sweeps, d_retune = MP.SETTINGS[name]
    _, net = MP.network(name)
    rec = MP.load(name) if sweeps is None and retune is None else None
    if rec is not None:
        return net, [tuple(p) for p in rec["path"]], rec["sliced"], {
            "path": "stored (%s): %s" % (os.path.basename(MP.path_file(name)), rec["optimiser"]),
            "optimiser_s": rec["optimiser_s"]}
    sweeps = d_sweeps if sweeps is None else sweeps
    retune = d_retune if retune is None else retune
    t0 = time.perf_counter()
    g = W.greedy_path(net.labels, net.open_labels)
    path, _, _ = tn.path_optimize(net.labels, net.open_labels, g, seed=SA_SEED, sweeps=sweeps,
                                  sweeps_final=0, t_start=0.01, t_end=0.0005, chains=16,
                                  greedy_trials=100, beta=1.0)
    path, sliced, _ = tn.path_optimize(net.labels, net.open_labels, path, seed=SA_SEED + 1,
                                       sweeps=0, sweeps_per_slice=retune, sweeps_final=300,
                                       t_start=0.005, t_end=0.0005, chains=16,
                                       max_log2_size=cap)
    return net, path, sliced, {
        "path": "annealed here: 100 random greedy trees x 16 chains, %d sweeps, dynamic slicing "
                "to 2^%d with %d re-tuning sweeps per bond" % (sweeps, cap, retune),
        "optimiser_s": time.perf_counter() - t0}


def step_rows(plan, info, before, calls, mode):
    """Per-step roofline rows of a profile-mode plan after ``calls`` timed calls, slowest first:
    each step's CUDA-event time, its T_cc and algorithmic bytes (the storage formats the plan
    uses), the bound of its kernel class (tensor cores: the measured sustained BF16 peak, halved
    for TF32, on the executed products; CUDA cores: the FP32 ALU peak; both against the measured
    HBM copy bandwidth) and the fraction of that roofline reached."""
    pk = peaks()
    hbm = pk["hbm_gbs"] * 1e9
    tensor = pk["bf16_tflops_sustained"] * 1e12 * (0.5 if mode in ("tf32", "split_tf32")
                                                  else 1.0)
    alu = NUM_SMS * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6
    rows = []
    for i in range(info["num_steps"]):
        a = plan.step_info(i)
        b = before[i]
        n = a["launches"] - b["launches"]
        if n <= 0:
            continue
        ms = (a["time_ms"] - b["time_ms"] + a["prep_ms"] - b["prep_ms"]) / calls
        sl = info["slices_in_flight"] if a["slice_dependent"] else 1
        tcc, tmc = a["tcc"] * sl, a["tmc_bytes"] * sl
        form = a["gemm_form"]
        # executed tensor work: 4M = T_cc, 3M = 3/4 T_cc, compensated = 3 T_cc
        executed = tcc * {2: 0.75, 3: 3.0}.get(form, 1.0)
        compute = executed / tensor if a["kernel_name"] == "gemm_tc" else tcc / alu
        roof = max(compute, tmc / hbm)
        rows.append({"step": i, "kernel": a["kernel_name"], "variant": a["tc_variant"],
                     "log2_mnk": [a["log2_m"], a["log2_n"], a["log2_k"]],
                     "slices": sl, "ms": ms, "tflops": tcc / (ms / 1e3) / 1e12,
                     "gbs": tmc / (ms / 1e3) / 1e9,
                     "bound": "tensor" if compute >= tmc / hbm and a["kernel_name"] == "gemm_tc"
                     else ("alu" if compute >= tmc / hbm else "hbm"),
                     "roofline_ms": roof * 1e3, "frac": roof * 1e3 / ms,
                     "store_run_log2": a["store_run_log2"]})
    rows.sort(key=lambda r: -r["ms"])
    return rows, {"hbm_gbs": pk["hbm_gbs"], "tensor_tflops": tensor / 1e12,
                  "alu_tflops": alu / 1e12}


def measure_c53(args, cycles, modes, batches=0, slices=0, compare=8, profile_mode=None,
                ref_mode="c64"):
    """The 53-qubit Sycamore-shaped circuit of ``cycles`` cycles (2^12 amplitudes on 12 open
    qubits) along its stored path.  Per precision mode: a plan (CUDA-graph replay, autotuned on
    its first batch), a contiguous range of slices timed after two warm-up batches (``batches``
    batches of the slices in flight, or ``slices`` slices; a dict gives a count per mode), the
    time per slice extrapolated to all slices (the method of Sec. 5), and the amplitudes of up to
    ``compare`` contributing slices compared with ``ref_mode`` (complex64: within 1e-5 of FP64 on
    the circuits the oracle can check).  For the modes in ``profile_mode`` one more batch runs
    in profile mode for the per-step roofline."""
    import torch
    from paper_2310_03978_gb300 import tn
    net, path, sliced, pdesc = sycamore53_path(cycles)
    stream = torch.cuda.current_stream()
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    nout = 1 << len(net.open_labels)
    part = torch.zeros(nout, dtype=torch.complex128, device="cuda")

    def one_slice(plan, s):
        part.zero_()
        plan.contract(part, s, s + 1, stream=stream)
        torch.cuda.synchronize()
        return part.cpu().numpy()

    # reference amplitudes of contributing slices.  With fSim at theta = pi/2 and no final
    # single-qubit layer most slices vanish (a closed qubit's projector after its last swap-like
    # fSim fixes the partner's input bond); candidates that no tensor forces to zero come from a
    # seeded search, and the first ones whose reference result is nonzero are kept.
    picks, refs = [], []
    t0 = time.perf_counter()
    if compare > 0:
        cplan = tn.Plan(tnet, path, sliced, mode=ref_mode, max_slices_in_flight=1)
        for s in supported_slices(net, sliced, SA_SEED, 3 * compare):
            if len(picks) == compare:
                break
            r = one_slice(cplan, s)
            if np.linalg.norm(r) > 0:
                picks.append(s)
                refs.append(r)
        cplan.close()
    ref = np.sum(refs, axis=0) if refs else None
    out = {**pdesc, "sliced_bonds": len(sliced), "compared_slices": [int(s) for s in picks],
           "reference_mode": ref_mode, "reference_s": time.perf_counter() - t0, "modes": {}}
    for mode_spec in modes:
        # "mode" or "mode:budget" (the precision policy's error budget for that arm)
        mode, _, bud = mode_spec.partition(":")
        budget = float(bud) if bud else args.eps_budget
        plan = tn.Plan(tnet, path, sliced, mode=mode, use_graph=True, autotune=True,
                       eps_budget=budget, thin_tc=args.thin_tc)
        pi = plan.info()
        sb = pi["slices_in_flight"]
        amps = torch.zeros(nout, dtype=torch.complex128, device="cuda")
        for w in range(2):  # the first batch autotunes
            plan.contract(amps, w * sb, (w + 1) * sb, stream=stream)
        torch.cuda.synchronize()
        s0 = 2 * sb
        want = slices.get(mode_spec, 0) if isinstance(slices, dict) else slices
        nsl = min(want if want > 0 else max(1, batches) * sb, pi["num_slices"] - s0)
        ms = time_steps(torch, lambda: plan.contract(amps, s0, s0 + nsl, stream=stream), 1,
                        stream)
        per_slice_ms = ms / nsl
        flops_slice = pi["tcc_per_slice"]
        rec = {"slices_timed": nsl, "slice_range": [s0, s0 + nsl], "slices_in_flight": sb,
               "ms_per_slice": per_slice_ms,
               "s_per_batch_extrapolated": per_slice_ms / 1e3 * pi["num_slices"],
               "effective_tflops": flops_slice / (per_slice_ms / 1e3) / 1e12,
               "workspace_bytes": pi["workspace_bytes"],
               "single_pass_steps": pi["num_single_pass"],
               "compensated_steps": pi["num_compensated"],
               "eps_predicted": pi["eps_predicted"], "eps_budget": budget}
        if picks:
            tot = np.sum([one_slice(plan, s) for s in picks], axis=0)
            rec["amp_rel_l2_vs_ref"] = rel_l2(tot, ref)
            rec["amp_max_rel_vs_ref"] = max_entry_err(tot, ref)
            rec["eps_l2sq_vs_ref"] = eps_l2sq(tot, ref)
            # the ideal-sample XEB of the summed slices, 2^n sum p^2 / sum p - 1, is dominated
            # by the -1 while the slices hold a small part of each amplitude; its well-conditioned
            # part is sum p^2 / sum p (= (XEB + 1) / 2^n), compared relatively
            rec["xeb_ratio_rel_err_vs_ref"] = abs(p2_over_p(tot) / p2_over_p(ref) - 1.0)
        plan.close()
        if profile_mode and mode_spec in profile_mode:
            pplan = tn.Plan(tnet, path, sliced, mode=mode, profile=True, autotune=True,
                            eps_budget=budget, thin_tc=args.thin_tc)
            pinfo = pplan.info()
            psb = pinfo["slices_in_flight"]
            for w in range(2):
                pplan.contract(amps, w * psb, (w + 1) * psb, stream=stream)
            torch.cuda.synchronize()
            before = [pplan.step_info(i) for i in range(pinfo["num_steps"])]
            pplan.contract(amps, 2 * psb, 3 * psb, stream=stream)
            torch.cuda.synchronize()
            rows, pk_used = step_rows(pplan, pinfo, before, 1, mode)
            tot_ms = sum(r["ms"] for r in rows)
            roof_ms = sum(r["roofline_ms"] for r in rows)
            rec["step_roofline"] = {"frac": roof_ms / tot_ms, "sum_ms": tot_ms,
                                    "roofline_ms": roof_ms, "slices": psb,
                                    "top": [{k: r[k] for k in ("step", "kernel", "variant",
                                                               "log2_mnk", "ms", "bound",
                                                               "frac")} for r in rows[:6]],
                                    "peaks": pk_used}
            pplan.close()
        del amps
        out["modes"][mode_spec] = rec
        out.update({"slices": pi["num_slices"], "max_intermediate_log2": pi["max_log2_size"],
                    "flops_per_slice": flops_slice,
                    "flops_per_batch": flops_slice * pi["num_slices"] + pi["tcc_invariant"],
                    "steps": pi["num_steps"]})
    tnet.close()
    return out


def run_sycamore53(args):
    """--sycamore53 N: the 53-qubit circuit (--c53-cycles) on its stored path, N batches of
    slices per mode; one JSON record per mode."""
    modes = [m for m in (args.sycamore53_modes or args.mode).split(",") if m]
    res = measure_c53(args, args.c53_cycles, modes, batches=args.sycamore53,
                      compare=args.sycamore53_compare)
    for mode, rec in res["modes"].items():
        yield {"metric": "53-qubit sliced contraction: s per 2^12-amplitude batch (extrapolated)",
               "value": rec["s_per_batch_extrapolated"], "unit": "s", "higher_is_better": False,
               "mode": mode,
               "config": {"workload": "sycamore53_6x9_c%d_open12" % args.c53_cycles,
                          "qubits": 53, "cycles": args.c53_cycles, "open_qubits": 12,
                          **{k: v for k, v in res.items() if k != "modes"}},
               **rec}


def read_slice_golden(name):
    """Stored FP64 oracle amplitudes of a few slices of a stored-path workload
    (tests/golden/make_golden.py): (slice ids, amplitudes summed in increasing slice order)."""
    path = os.path.join(ROOT, "tests", "golden", name + ".slices.amps.txt")
    if not os.path.exists(path):
        return None, None
    slices = None
    for line in open(path):
        if line.startswith("# slices:"):
            slices = [int(x) for x in line.split(":", 1)[1].split()]
            break
    rows = np.loadtxt(path, comments="#")
    return slices, rows[:, 0] + 1j * rows[:, 1]


def run_table3(args):
    """The shape of the paper's Table 3 (Sec. 4.3) on the 45-qubit 14-cycle Sycamore-shaped
    circuit (5x9 grid, 12 open qubits, stored annealed path with 2^13 slices at the 2^26 cap):
    the k dense steps with the largest T_cc single-pass, the others compensated, for the paper's
    pair (TF32 / 3xTF32) and for FP16 / 3xFP16; per k the time of a contiguous range of slices
    (relative to all single-pass), the share of T_cc made single-pass, and the amplitude error
    of the stored slices against the FP64 oracle (eps_L2^2, Eq. l2_squared_error; rel. L2; per
    entry).  Then the error budget: the k the precision policy picks for a few budgets, with its
    prediction and the measured error.  One JSON line per row."""
    import torch
    from paper_2310_03978_gb300 import tn
    name = "sycamore45_5x9_c14_open12"
    net, path, sliced, pdesc = stored_path(name)
    gold_slices, gold = read_slice_golden(name)
    stream = torch.cuda.current_stream()
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    nout = 1 << len(net.open_labels)
    amps = torch.zeros(nout, dtype=torch.complex128, device="cuda")
    part = torch.zeros(nout, dtype=torch.complex128, device="cuda")

    def run(mode, topk=0, budget=0.0):
        plan = tn.Plan(tnet, path, sliced, mode=mode, use_graph=True, autotune=True,
                       mixed_topk=topk, eps_budget=budget)
        info = plan.info()
        sb = info["slices_in_flight"]
        for w in range(2):  # the first batch autotunes
            plan.contract(amps, w * sb, (w + 1) * sb, stream=stream)
        torch.cuda.synchronize()
        n = min(args.table3_slices, info["num_slices"] - 2 * sb)
        ms = time_steps(torch, lambda: plan.contract(amps, 2 * sb, 2 * sb + n, stream=stream),
                        1, stream)
        got = None
        if gold_slices:
            got = np.zeros(nout, dtype=np.complex128)
            for s in sorted(gold_slices):  # summed in increasing slice order, like the oracle
                part.zero_()
                plan.contract(part, s, s + 1, stream=stream)
                torch.cuda.synchronize()
                got += part.cpu().numpy()
        # T_cc of the single-pass dense steps over all T_cc (per slice)
        steps = [plan.step_info(i) for i in range(info["num_steps"])]
        single = sum(st["tcc"] for st in steps if st["kernel"] == 3 and st["gemm_form"] in (1, 2)
                     and st["slice_dependent"])
        plan.close()
        rec = {"mode": mode, "single_pass_steps": info["num_single_pass"],
               "compensated_steps": info["num_compensated"],
               "tcc_ratio_single_pass": single / info["tcc_per_slice"],
               "ms_per_slice": ms / n, "slices_timed": n, "eps_predicted": info["eps_predicted"]}
        if got is not None:
            rec.update({"eps_l2sq": eps_l2sq(got, gold), "amp_rel_l2": rel_l2(got, gold),
                        "amp_max_rel": max_entry_err(got, gold)})
        return rec, info

    base = {"metric": "Table 3 shape: time and eps_L2^2 against k single-pass dense steps",
            "workload": name, "qubits": 45, "cycles": 14, "open_qubits": 12,
            "slices": 1 << len(sliced), "reference": "FP64 oracle, slices %s" % gold_slices,
            **pdesc}
    for fast, slow in (("tf32", "split_tf32"), ("fp16_scaled", "split_fp16")):
        rows = []
        r0, info = run(slow)
        rows.append(dict(r0, k=0))
        ndense = r0["compensated_steps"]
        for k in [k for k in (1, 2, 4, 8, 16, 32, 64) if k < ndense] + [ndense]:
            r, _ = run(fast, topk=k, budget=1.0)  # a loose budget: k exactly
            rows.append(dict(r, k=k))
        t_all = rows[-1]["ms_per_slice"]
        for r in rows:
            r["relative_time"] = r["ms_per_slice"] / t_all
            print(json.dumps({**base, "pair": "%s / %s" % (fast, slow), "dense_steps": ndense,
                              "steps": info["num_steps"],
                              "flops_per_slice": info["tcc_per_slice"], **r}), flush=True)
    for mode in ("fp16_scaled", "bf16_scaled", "tf32"):
        for budget in (1e-4, 1e-3, 5e-3):
            r, _ = run(mode, budget=budget)
            print(json.dumps({**base, "budget": budget, **r}), flush=True)
    tnet.close()


def measure_sparse(args, dev, stream):
    """Sparse-state contraction of 4096 seeded bitstrings of the 24-qubit all-open circuit along
    an annealed path; time per batch and the error against the stored state-vector amplitudes."""
    import torch
    from paper_2310_03978_gb300 import tn, workload as W
    circ_s, net_s, smp = W.sparse_state_workload()
    g = W.greedy_path(net_s.labels, net_s.open_labels)
    sp_path, _, _ = tn.path_optimize(net_s.labels, net_s.open_labels, g, seed=SA_SEED,
                                     sweeps=500, sweeps_final=0, t_start=0.03, t_end=0.001,
                                     chains=8)
    tnet_s = tn.Network(net_s.tensors, net_s.labels, net_s.open_labels)
    splan = tn.SparsePlan(tnet_s, sp_path, smp, mode=args.mode)
    amps = torch.zeros(len(smp), dtype=torch.complex128, device=dev)
    splan.contract(amps, stream=stream)
    torch.cuda.synchronize()
    sp_result = amps.cpu().numpy().copy()
    for _ in range(2):
        splan.contract(amps, stream=stream)
    torch.cuda.synchronize()
    steps = max(1, args.sparse_steps)
    sp_ms = time_steps(torch, lambda: splan.contract(amps, stream=stream), steps, stream) / steps
    sp_info = splan.info()
    splan.close()
    tnet_s.close()
    del amps
    ref = golden_amps("sparse_state_sycamore_4x6_c12_all_open")
    return {"ms": sp_ms, "info": sp_info,
            "rel_l2": rel_l2(sp_result, ref) if ref is not None else None,
            "qubits": circ_s.n_qubits, "samples": len(smp)}


def sparse_line(args, sparse):
    si = sparse["info"]
    return {"workload": "sycamore_4x6_c12_all_open, %d seeded uniform bitstrings"
                        % sparse["samples"],
            "ms_per_batch": sparse["ms"], "samples": sparse["samples"],
            "distinct_samples": si["distinct_samples"], "flops_per_batch": si["tcc"],
            "effective_tflops": si["tcc"] / (sparse["ms"] / 1e3) / 1e12,
            "arena_bytes": si["arena_bytes"], "dense_subtrees": si["dense_subtrees"],
            "dense_subtree_steps": si["dense_subtree_steps"], "gemm_steps": si["gemm_steps"],
            "thin_steps": si["thin_steps"], "grouped_steps": si["grouped_steps"],
            "mode": args.mode,
            "amp_rel_l2_vs_statevector": sparse["rel_l2"]}


def run_step_bench(args):
    """Single-step microbench: C[M,N] = sum_K A[M,K] B[N,K] on random complex tensors with all
    dims 2 and seeded random label orders, timed through the C ABI.  `--mode` and `--gemm-form`
    may list several values (comma-separated); one JSON line per combination.  Each line splits
    the call into the GEMM kernel, the operand conversions (tensor-core steps) and the leaf
    binding (the permutation of both leaves into GEMM order, complex128 -> complex64), and gives
    the binding's bandwidth against the measured HBM copy peak and the GEMM's against its own."""
    import torch
    from paper_2310_03978_gb300 import tn
    lm, ln, lk = (int(x) for x in args.step.split(","))
    rng = np.random.default_rng(1000 + 37 * lm + 5 * ln + lk)
    M, N, K = list(range(lm)), list(range(100, 100 + ln)), list(range(200, 200 + lk))
    la = [int(x) for x in rng.permutation(M + K)]
    lb = [int(x) for x in rng.permutation(N + K)]
    out = [int(x) for x in rng.permutation(M + N)]
    ra, rb = lm + lk, ln + lk
    scale = 2.0 ** (-(ra + rb) / 4)  # amplitude-like magnitudes
    A = (rng.standard_normal((2,) * ra) + 1j * rng.standard_normal((2,) * ra)) * scale
    B = (rng.standard_normal((2,) * rb) + 1j * rng.standard_normal((2,) * rb)) * scale
    tensors, labels, path = [A, B], [la, lb], [(0, 1)]
    if args.feed_tc:
        # the measured step's result feeds a second tensor-core step (over all but two of its M
        # labels, with 7 new labels), so it is written directly as scaled planar 16-bit numbers
        if lm < 9:
            raise SystemExit("--feed-tc needs lm >= 9")
        P = list(range(300, 307))
        T = (rng.standard_normal((2,) * (lm - 2 + 7)) +
             1j * rng.standard_normal((2,) * (lm - 2 + 7))) * 2.0 ** -6
        tensors, labels = [A, B, T], [la, lb, M[2:] + P]
        out = M[:2] + N + P
        path = [(0, 1), (0, 2)]
    net = tn.Network(tensors, labels, out)
    ref = None
    if lm + ln + lk <= 22 and not args.feed_tc:  # numpy's complex128 einsum of the one pair
        ids = {l: i for i, l in enumerate(sorted(set(la + lb)))}
        ref = np.einsum(A, [ids[l] for l in la], B, [ids[l] for l in lb],
                        [ids[l] for l in out]).reshape(-1)
    pk = peaks()
    bind_bytes = 24.0 * ((1 << ra) + (1 << rb))  # complex128 read + complex64 written
    amps = torch.zeros(1 << len(out), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    for mode in args.mode.split(","):
        for form in args.gemm_form.split(","):
            plan = tn.Plan(net, path, (), mode=mode, profile=True, gemm_form=form,
                           tc_bk=args.tc_bk, tc_bn=args.tc_bn, autotune=bool(args.autotune),
                           thin_tc=args.thin_tc)
            for _ in range(args.warmup):
                plan.contract(amps, stream=stream)
            torch.cuda.synchronize()
            before, ib = plan.step_info(0), plan.info()
            ms = time_contract(torch, plan, amps, args.steps, stream) / args.steps
            si, ia = plan.step_info(0), plan.info()
            nl = max(1, si["launches"] - before["launches"])
            kern_ms = (si["time_ms"] - before["time_ms"]) / nl
            bind_ms = (ia["bind_ms"] - ib["bind_ms"]) / max(1, ia["bind_launches"] -
                                                             ib["bind_launches"])
            tcc = si["tcc"]
            check = None
            if ref is not None:
                amps.zero_()
                plan.contract(amps, stream=stream)
                check = rel_l2(amps.cpu().numpy(), ref)
            tc = si["kernel_name"] == "gemm_tc"
            kpeak = pk["bf16_tflops"] if tc else 80.54784
            print(json.dumps({
                "metric": "single-step effective TFLOPS", "value": tcc / (ms / 1e3) / 1e12,
                "unit": "TFLOPS", "kernel": si["kernel_name"], "tc_variant": si["tc_variant"],
                "ms_per_step": ms, "kernel_ms": kern_ms,
                "kernel_tflops": tcc / (kern_ms / 1e3) / 1e12,
                "kernel_frac": tcc / (kern_ms / 1e3) / 1e12 / kpeak,
                "kernel_peak": "bf16 burst (measured)" if tc else "FP32 ALU",
                "prep_ms": (si["prep_ms"] - before["prep_ms"]) / max(1, args.steps),
                "bind_ms": bind_ms, "bind_gbs": bind_bytes / (bind_ms / 1e3) / 1e9,
                "bind_frac_hbm": bind_bytes / (bind_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                "config": {"lm": lm, "ln": ln, "lk": lk, "rank_a": ra, "rank_b": rb,
                           "mode": mode, "gemm_form": form, "tc_bk": args.tc_bk,
                           "tc_bn": args.tc_bn, "autotune": args.autotune,
                           "feeds_tensor_cores": bool(args.feed_tc)},
                "rel_l2_vs_numpy_einsum": check}))
            plan.close()
    net.close()


def run_step_profile(args):
    """Per-step roofline of the bench workload (or, with --sycamore53, of one batch of slices of
    the 53-qubit path of --c53-cycles cycles): every step's CUDA-event time in profile mode
    (after the warm-up calls, averaged over --steps calls), its T_cc and algorithmic bytes (the
    storage formats the plan uses), the bound of its kernel class (tensor cores: the measured
    BF16 peak, halved for TF32; CUDA cores: the FP32 ALU peak; both against the measured HBM copy
    bandwidth) and the fraction of that roofline reached.  One JSON line per step, slowest
    first, then a summary line."""
    import torch
    from paper_2310_03978_gb300 import tn, workload as W
    if args.sycamore53:  # one batch of slices per call, consecutive batches
        wnet, path, sliced, _ = sycamore53_path(args.c53_cycles)
        workload = "sycamore53_6x9_c%d_open12" % args.c53_cycles
    else:  # every slice per call
        wl = W.bench_workload()
        wnet, path, sliced, workload = wl.network, wl.path, wl.sliced, WORKLOAD
    net = tn.Network(wnet.tensors, wnet.labels, wnet.open_labels)
    plan = tn.Plan(net, path, sliced, mode=args.mode, profile=True,
                   autotune=bool(args.autotune), mixed_topk=args.mixed_topk,
                   eps_budget=args.eps_budget, thin_tc=args.thin_tc)
    info = plan.info()
    nsteps = info["num_steps"]
    sb = info["slices_in_flight"]
    amps = torch.zeros(1 << len(wnet.open_labels), dtype=torch.complex128, device="cuda")
    calls = {"n": 0}

    def call():
        if args.sycamore53:
            plan.contract(amps, calls["n"] * sb, (calls["n"] + 1) * sb)
        else:
            plan.contract(amps)
        calls["n"] += 1

    for _ in range(max(1, args.warmup)):
        call()
    torch.cuda.synchronize()
    before = [plan.step_info(i) for i in range(nsteps)]
    for _ in range(args.steps):
        call()
    torch.cuda.synchronize()
    rows, pk_used = step_rows(plan, info, before, args.steps, args.mode)
    for r in rows[:args.step_profile]:
        print(json.dumps(r))
    total = sum(r["ms"] for r in rows)
    roof = sum(r["roofline_ms"] for r in rows)
    print(json.dumps({"summary": True, "workload": workload, "mode": args.mode,
                      "eps_budget": args.eps_budget, "single_pass_steps": info["num_single_pass"],
                      "compensated_steps": info["num_compensated"],
                      "slices_per_call": sb if args.sycamore53 else info["num_slices"],
                      "steps_timed": len(rows), "sum_ms": total, "roofline_ms": roof,
                      "frac": roof / total, "peaks": pk_used}))
    plan.close()
    net.close()


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, each step a bounded sample of the workload."""
    if rank != 0:
        return
    from paper_2310_03978_gb300 import workload as W
    wl = W.bench_workload()
    per = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(wl, per / 4)
    rates, secs = [], []
    smp = None
    for _ in range(args.steps):
        smp = oracle_sample(wl, per)
        rates.append(smp["rate"])
        secs.append(smp["seconds"])
    _, steps = dominant_step(wl)
    flops = sum(s.tcc for s in steps) * wl.num_slices
    rate = statistics.median(rates)
    line = {
        "metric": METRIC, "impl": "reference", "value": rate / 1e12, "unit": "TFLOPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(secs), "s_per_batch": flops / rate,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "oracle complex128"},
        "cpu_baseline": {"value": rate / 1e12, "unit": "TFLOPS", "cores": smp["threads"],
                         "kind": "oracle",
                         "sample": "dominant step (%s), %d output elements per step"
                                   % (smp["shape"], smp["outputs"])},
        "e2e": {"value": rate / 1e12, "unit": "TFLOPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.oracle_child:
        run_oracle_child(args.oracle_child)
        return
    if args.impl == "reference":
        from oracle import oracle as O
        O.build()
        run_reference(args, rank, world)
        return
    from paper_2310_03978_gb300 import tn
    if not os.path.exists(tn.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    from oracle import oracle as O
    O.build()  # the CPU-baseline leg times the oracle
    if args.step:
        run_step_bench(args)
        return
    if args.step_profile:
        run_step_profile(args)
        return
    if args.table3:
        import torch
        torch.cuda.set_device(local_rank)
        run_table3(args)
        return
    if args.sycamore53:
        import torch
        torch.cuda.set_device(local_rank)
        for rec in run_sycamore53(args):
            print(json.dumps(rec), flush=True)
        return
    if args.sparse_only:
        import torch
        torch.cuda.set_device(local_rank)
        r = measure_sparse(args, torch.device("cuda", local_rank), torch.cuda.current_stream())
        print(json.dumps({"metric": "sparse-state ms per batch", "value": r["ms"], "unit": "ms",
                          "higher_is_better": False, **sparse_line(args, r)}))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
