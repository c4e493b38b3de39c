#!/usr/bin/env python3
"""Benchmark: MSFV forward + misfit-gradient solves per second on GB300.

Workload: 3D, 128^3 cells, coarsening 8 (16^3 coarse cells, 7^3 interior dual-cell
problems with 8 right-hand sides), sigma = exp(m) with m a Gaussian random field
(std 1, correlation length 0.15) plus two +/-2 boxes, 16 dipoles and 512
receivers on the top layer.  One step = one forward solve (basis, coarse operator,
reduced solve, predicted data) plus the misfit gradient through dP/dm, all FP64,
inputs resident in HBM.  L2 is flushed (a 512 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the path has no
exchange step); value = solves of all ranks / max-over-ranks time.
``--impl reference`` times the CPU oracle on the host cores instead (rank 0 only).
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
sys.path.insert(0, ROOT)

from paper_1707_07598_gb300 import workloads as W  # noqa: E402
from paper_1707_07598_gb300 import replicas as R  # noqa: E402

METRIC = "batched/served MSFV fwd+grad solves/s vs plain at 1e-9 rel err; p50/p99 ms"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk x 2 flop x max SM clock
WORKLOAD = "3d_128^3_c8_16dipoles_512rec_fwd+grad"
# DRAM bytes (read + write) of one k_local_fwd<256,1> launch per fine cell, from the ncu
# capture of the current kernel at 64^3, c=8 (12.32 MB read + 13.16 MB write over 262144
# cells; profiles/k_local_fwd_interiors_3d_64cube_c8.md).  The kernel's traffic (factor and
# basis writes, conductivity reads) grows with the number of cells, so a launch on another
# mesh is scaled by its cell count.  Set to None whenever the kernel changes.
INTERIOR_DRAM_BYTES_PER_CELL = (12.322816e6 + 13.156096e6) / 64 ** 3


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=128, help="mesh size per axis (default 128)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--workload", default="plain",
                   choices=["plain", "batched", "served", "diff", "gn", "sources", "nodal"],
                   help="plain: the one-instance 128^3 step (default); batched: independent "
                        "instances in one CUDA graph vs one at a time; served: the Poisson "
                        "request stream; diff: 256^3, c=16 gradient, J v, J^T w; gn: 5 "
                        "Gauss-Newton-CG iterations on the 128^3 two-block model; sources: "
                        "the 128^3 step with source bases beside the plain one; nodal: "
                        "the paper's nodal Galerkin variant on the same survey shape")
    p.add_argument("--instances", type=int, default=64, help="batched: number of instances")
    p.add_argument("--rate", type=float, default=50.0, help="served: requests per second")
    p.add_argument("--duration", type=float, default=10.0,
                   help="served: seconds of the arrival stream that are replayed")
    p.add_argument("--fd-dirs", type=int, default=20, help="diff: finite-difference directions")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                   help="local problems of the top dimension: FP64 factor (default) or FP32 "
                        "factor with two FP64 refinement steps")
    p.add_argument("--policy", default="sjf", choices=["fifo", "sjf"],
                   help="served: admission order of the continuous-batching loop")
    return p.parse_args()


def dist_env():
    e = R.rank_env()
    return e.rank, e.world, e.local


# ---------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------------
SAMPLE_N = 64


def oracle_sample_time():
    """One oracle forward + gradient on the 64^3 sub-problem of the workload (same
    c = 8, 16 dipoles, 512 top receivers).  Returns (seconds, scale) where scale =
    cells(128^3) / cells(64^3) extrapolates the time to the full workload."""
    from oracle.msfv_oracle import Oracle
    prob, m = W.config_3d_128(n=SAMPLE_N)
    orc = Oracle(prob)
    t0 = time.perf_counter()
    st = orc.forward(m)
    d_obs = st['d'] * 1.01
    orc.misfit_gradient(st, d_obs)
    t1 = time.perf_counter()
    return t1 - t0, (128 / SAMPLE_N) ** 3


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample_time()
    times = []
    for _ in range(args.steps):
        t, scale = oracle_sample_time()
        times.append(t * scale)
    ms = 1000.0 * statistics.mean(times)
    val = 1000.0 / ms
    sample = (f"oracle fwd+grad on the {SAMPLE_N}^3 sub-problem of the workload (c=8, 16 dipoles, "
              f"512 top receivers) per step, time x{(128 // SAMPLE_N) ** 3} (cell ratio) for 128^3")
    out = {"metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": [128] * 3, "coarsen": 8, "n_src": 16,
                      "n_rec": 512},
           "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                        reasons.add(nm)
            except Exception:
                continue
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sm)}
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


def run_ours(args):
    import torch
    from paper_1707_07598_gb300 import build as B
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    B.build()
    from paper_1707_07598_gb300.msfv import Session

    seeds = R.replica_seeds(rank)
    prob, m_np = W.config_3d_128(seed=seeds.model, n=args.n)
    stream = torch.cuda.current_stream(dev)
    sess = Session(prob, stream=stream)
    m = torch.from_numpy(m_np).to(dev)
    # observed data: forward at an independent model plus 1% noise (outside the timing)
    m_true = torch.from_numpy(W.config_3d_128(seed=seeds.truth, n=args.n)[1]).to(dev)
    d_true = sess.forward(m_true).clone()
    noise = torch.from_numpy(W.noise_like(tuple(d_true.shape), 1.0, seeds.noise)).to(dev)
    d_obs = d_true + 0.01 * d_true.abs() * noise
    grad = torch.empty(prob.N, dtype=torch.float64, device=dev)
    d_pred = torch.empty((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        sess.forward(m, d_pred)
        sess.adjoint(d_obs, grad, want_phi=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sess.profile(True)
    sess.phase_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    time.sleep(0.3)
    R.barrier()
    torch.cuda.synchronize(dev)
    launches0 = sess.launch_count()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = sess.launch_count() - launches0
    R.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    phases = sess.phase_times(reset=True)
    sess.profile(False)
    info = sess.info()
    total_ms = R.max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = R.whole_job_rate(world, args.steps, total_ms / 1000.0)

    # roofline of the dominant kernel: the dual-cell interior basis solve
    int_ms, int_calls = phases.get("basis_interiors", (0.0, 0))
    int_avg_s = (int_ms / max(int_calls, 1)) / 1000.0
    flops = sess.interior_flops()
    achieved = flops / int_avg_s / 1e12 if int_avg_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_local_fwd<256,1> (3D dual-cell interiors)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "peak_source": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (recipe unit "
                           "counts and max clock); a DFMA probe measured 1.20 TFLOP/s at 1987 MHz",
            "flops_per_launch": flops, "avg_launch_ms": int_avg_s * 1000.0,
            "traffic": (INTERIOR_DRAM_BYTES_PER_CELL * prob.N
                        if INTERIOR_DRAM_BYTES_PER_CELL is not None else None),
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel at "
                              "64^3, scaled by the number of fine cells"}
    if args.precision == "mixed":
        roof.update(kernel="k_mix_fwd (3D dual-cell interiors: FP32 band factor, two FP64 "
                           "refinement steps)",
                    traffic=None,
                    note="the method's FP64 flop count (the same numerator as the FP64 kernel) "
                         "over the FP64 peak; most of the arithmetic runs in FP32")
    phase_ms = {k: v[0] / max(args.steps, 1) for k, v in phases.items() if v[1]}

    e2e = None
    if not args.no_e2e:
        m_h = torch.empty(prob.N, dtype=torch.float64).pin_memory()
        m_h.copy_(m.cpu())
        dobs_h = torch.empty(tuple(d_obs.shape), dtype=torch.float64).pin_memory()
        dobs_h.copy_(d_obs.cpu())
        dp_h = torch.empty(tuple(d_obs.shape), dtype=torch.float64).pin_memory()
        g_h = torch.empty(prob.N, dtype=torch.float64).pin_memory()
        mn, dn, dpn, gn = m_h.numpy(), dobs_h.numpy(), dp_h.numpy(), g_h.numpy()
        for _ in range(2):
            sess.solve_host(mn, dn, dpn, gn)
        times = []
        R.barrier()
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sess.solve_host(mn, dn, dpn, gn)
            times.append(time.perf_counter() - t0)
        R.barrier()
        tot = R.max_over_ranks(sum(times), dev)
        e2e = {"value": R.whole_job_rate(world, args.steps, tot), "unit": "solves/s",
               "h2d_bytes_per_step": 8 * prob.N + 8 * prob.n_src * prob.n_rec,
               "d2h_bytes_per_step": 8 * prob.N + 8 * prob.n_src * prob.n_rec + 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, scale = oracle_sample_time()
        cpu = {"value": 1.0 / (t * scale), "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"one oracle fwd+grad on the {SAMPLE_N}^3 sub-problem of the workload "
                         f"(c=8, 16 dipoles, 512 top receivers): {t:.2f} s, scaled x{scale:.0f} "
                         f"(cell ratio) to 128^3; numpy/scipy, single thread"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
               "p50_ms": float(np.percentile(step_ms, 50)),
               "p99_ms": float(np.percentile(step_ms, 99)),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD if args.n == 128 else f"3d_{args.n}^3_c8",
                          "n": [args.n] * 3, "coarsen": 8, "n_src": prob.n_src,
                          "n_rec": prob.n_rec, "parallelism": f"replicas x{world}",
                          "l2": "flushed before every timed step (512 MiB write)",
                          "factor_mode": "store", "precision": args.precision},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk, "phases_ms_per_step": phase_ms,
               "coarse": {"solver": "mg-gmres" if info["coarse_solver"] else "banded-lu",
                          "iters_fwd": info["coarse_iters"], "iters_adj": info["coarse_iters_T"]}}
        print(json.dumps(out))
    sess.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0



# ---------------------------------------------------------------------------------
# Extra workloads (not the default line): batched instances, served requests, and the
# 256^3 differentiation case.  Each prints its own JSON line.
# ---------------------------------------------------------------------------------
def _gpu_setup():
    import torch
    from paper_1707_07598_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    return torch, dev


def run_batched(args):
    """Independent 3D instances (sizes 64..192^3, c in {4, 8, 16}, 8-32 dipoles) as one
    CUDA graph per step, against the same instances run one at a time."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.msfv import Batch, Session
    specs = W.batch_instances(args.instances)
    sessions, ms, dobs = [], [], []
    per_instance_budget = 6 << 30     # larger stored factors switch to recompute
    for sp in specs:
        prob = sp.problem()
        st = torch.cuda.Stream(dev)
        sessions.append(Session(prob, stream=st, factor_mode=0,
                                hbm_budget_bytes=per_instance_budget))
        ms.append(W.gaussian_random_field_device(prob.n, sp.corr_len, sp.seed, dev))
        dobs.append(torch.zeros((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev))
    torch.cuda.synchronize()
    batch = Batch(sessions, ms, dobs)
    batch.run()
    batch.check()
    for k in range(len(specs)):                       # observed data: 97% of the prediction
        dobs[k].copy_(0.97 * batch.d_pred[k])
    for _ in range(max(args.warmup - 1, 0)):
        batch.run()
    batch.check()
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(stream)
        batch.run()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    batch.check()
    bt = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop()
    # the plain one-instance path: the same instances one after another, no graph
    plain_ms = []
    d_plain, g_plain = [], []
    for rep in range(max(1, min(args.steps, 2))):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k, s in enumerate(sessions):
            s.set_stream(stream)
            d = s.forward(ms[k])
            _, g = s.adjoint(dobs[k], want_phi=False)
            if rep == 0:
                d_plain.append(d)
                g_plain.append(g)
        t1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(t0.elapsed_time(t1))
    same = all(torch.equal(d_plain[k], batch.d_pred[k]) and torch.equal(g_plain[k], batch.grad[k])
               for k in range(len(specs)))
    K = len(specs)
    ms_step = float(np.mean(bt))
    value = K / (ms_step / 1000.0)
    plain_val = K / (float(np.mean(plain_ms)) / 1000.0)
    recompute = sum(int(s.info()["recompute"]) for s in sessions)
    mix = {}
    for sp in specs:
        key = f"{sp.n[0]}^3_c{sp.coarsen}"
        mix[key] = mix.get(key, 0) + 1
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "p50_ms": float(np.percentile(bt, 50)), "p99_ms": float(np.percentile(bt, 99)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"batched_{K}_instances_3d", "instances": K, "mix": mix,
                      "graph": "one CUDA graph per step, one branch per instance",
                      "recompute_instances": recompute,
                      "l2": "working set of every step far larger than L2"},
           "plain": {"value": plain_val, "unit": "solves/s",
                     "ms_per_step": float(np.mean(plain_ms)),
                     "path": "same sessions, forward + adjoint one instance at a time"},
           "speedup_vs_plain": value / plain_val,
           "parity": "batched == plain bit for bit on every instance" if same else "MISMATCH",
           "clocks": clk}
    print(json.dumps(out))
    batch.close()
    for s in sessions:
        s.close()
    return 0 if same else 1


def run_served(args):
    """The Poisson request stream (rate x duration), fine sizes 32..256^3, c in {4, 8, 16},
    1-64 dipoles, 150 GB budget: continuous batching against one request at a time."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.serve import GpuBackend, Server
    reqs = W.served_requests(rate=args.rate, duration=args.duration)
    budget = 150 * 10 ** 9
    # warm the kernels and the allocator pool on a small request
    warm = W.served_requests(rate=100.0, duration=0.05, seed=99, sizes=(32,))
    Server(GpuBackend(dev), budget, max_inflight=4).run(warm)
    res = {}
    clk = None
    for mode, inflight in (("served", 8), ("plain", 1)):
        clocks = ClockSampler(0)
        clocks.start()
        st = Server(GpuBackend(dev, use_graph=(inflight > 1)), budget, max_inflight=inflight,
                    policy=args.policy if inflight > 1 else "fifo").run(reqs)
        c = clocks.stop()
        if mode == "served":
            clk = c
        done = st.done()
        res[mode] = {"value": st.throughput, "unit": "solves/s", "completed": len(done),
                     "rejected": sum(r.status == "rejected" for r in st.records),
                     "p50_ms": 1000.0 * st.percentile(50), "p99_ms": 1000.0 * st.percentile(99),
                     "makespan_s": st.makespan, "sessions_opened": st.opened,
                     "evictions": st.evictions, "peak_session_bytes": st.peak_bytes}
    sv = res["served"]
    out = {"metric": METRIC, "value": sv["value"], "unit": "solves/s", "n_gpus": 1,
           "steps": len(reqs), "warmup": len(warm), "ms_per_step": 1000.0 / max(sv["value"], 1e-12),
           "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"served_poisson_{args.rate:g}_per_s_{args.duration:g}_s",
                      "requests": len(reqs), "sizes": [32, 64, 128, 256],
                      "coarsenings": [4, 8, 16], "sources": "1-64", "hbm_budget_bytes": budget,
                      "max_inflight": 8, "policy": args.policy},
           "served": sv, "plain": res["plain"],
           "speedup_vs_plain": sv["value"] / max(res["plain"]["value"], 1e-12), "clocks": clk}
    print(json.dumps(out))
    return 0


def run_diff(args):
    """256^3, c = 16, 64 dipoles, 4096 receivers: gradient, J v and J^T w through the
    torch.autograd bindings, with stored and with recomputed local factors; central
    differences (step 1e-6) along --fd-dirs random directions."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.autograd import misfit, predict
    from paper_1707_07598_gb300.msfv import Session
    import torch.autograd.forward_ad as fwAD
    n = args.n if args.n != 128 else 256
    prob = W.make_problem((n, n, n), 16, 64, 4096, seed=4, top_layer=True)
    m0 = W.gaussian_random_field_device(prob.n, 0.15, 4, dev)
    stream = torch.cuda.current_stream(dev)
    out_modes = {}
    for fm, name in ((1, "store"), (2, "recompute")):
        s = Session(prob, stream=stream, factor_mode=fm)
        d_obs = (s.forward(m0) * 1.02).contiguous()
        v = torch.randn(prob.N, dtype=torch.float64, device=dev,
                        generator=torch.Generator(device=dev).manual_seed(5))
        w = torch.randn((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev,
                        generator=torch.Generator(device=dev).manual_seed(6))

        def step():
            m = m0.clone().requires_grad_(True)
            phi = misfit(m, d_obs, s)
            phi.backward()
            with fwAD.dual_level():
                jv = fwAD.unpack_dual(predict(fwAD.make_dual(m0, v), s)).tangent
            m2 = m0.clone().requires_grad_(True)
            predict(m2, s).backward(w)
            return m.grad, jv, m2.grad
        for _ in range(max(args.warmup, 1)):
            g, jv, jtw = step()
        ts = []
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g, jv, jtw = step()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        # adjoint identity and central differences of the misfit
        dot = abs(float((w * jv).sum()) - float(jtw @ v)) / float(w.norm() * jv.norm())
        fd_err = 0.0
        gen = torch.Generator(device=dev).manual_seed(7)
        for k in range(args.fd_dirs):
            dirn = torch.randn(prob.N, dtype=torch.float64, device=dev, generator=gen)
            with torch.no_grad():
                fp = misfit(m0 + 1e-6 * dirn, d_obs, s).item()
                fm_ = misfit(m0 - 1e-6 * dirn, d_obs, s).item()
            an = float(g @ dirn)
            fd_err = max(fd_err, abs((fp - fm_) / 2e-6 - an) /
                         max(abs(an), 1e-3 * float(g.norm() * dirn.norm())))
        info = s.info()
        out_modes[name] = {"ms_per_step": float(np.mean(ts)), "p50_ms": float(np.percentile(ts, 50)),
                           "p99_ms": float(np.percentile(ts, 99)),
                           "factor_bytes": info["factor_bytes"],
                           "workspace_bytes": info["workspace_bytes"],
                           "fd_max_rel_err": fd_err, "fd_dirs": args.fd_dirs,
                           "adjoint_identity_rel_err": dot}
        s.close()
        torch.cuda.synchronize()
    st = out_modes["store"]
    out = {"metric": METRIC, "value": 1000.0 / st["ms_per_step"], "unit": "grad+Jv+JTw per s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": st["ms_per_step"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"diff_{n}^3_c16_64dipoles_4096rec", "n": [n] * 3,
                      "coarsen": 16, "n_src": 64, "n_rec": 4096,
                      "step": "misfit gradient + J v (forward-mode) + J^T w (reverse-mode)"},
           "modes": out_modes}
    print(json.dumps(out))
    return 0


def run_gn(args):
    """Five Gauss-Newton-CG iterations (10 CG iterations each) on the 128^3 / c = 8 /
    16-dipole / 512-receiver survey of the two-block model with 1% noise, from a
    homogeneous start; alpha = 1e-8 (Sec. 5)."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.msfv import Session
    n = args.n
    prob, _ = W.config_3d_128(n=n)
    s = Session(prob)
    m_true = torch.from_numpy(W.block_model(prob.n)).to(dev)
    d_true = s.forward(m_true).clone()
    noise = torch.from_numpy(W.noise_like(tuple(d_true.shape), 1.0, 9)).to(dev)
    d_obs = (d_true + 0.01 * d_true.abs() * noise).contiguous()
    m = torch.zeros(prob.N, dtype=torch.float64, device=dev)
    s.gn_step(m.clone(), d_obs, 1e-8, cg_iters=2)          # warm-up (kernels, workspace)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = []
    for _ in range(5):
        hist.append(s.gn_step(m, d_obs, 1e-8, cg_iters=10))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    fwd = sum(1 + h["backtracks"] + 1 for h in hist)
    out = {"metric": METRIC, "value": len(hist) / wall, "unit": "GN iterations/s", "n_gpus": 1,
           "steps": len(hist), "warmup": 1, "ms_per_step": 1000.0 * wall / len(hist),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"gn_{n}^3_c8_two_blocks", "alpha": 1e-8, "cg_iters": 10,
                      "noise": "1%", "start": "m = 0"},
           "misfit": [hist[0]["phi_d0"]] + [h["phi_d1"] for h in hist],
           "cg_iters": [h["cg_iters"] for h in hist], "steps_taken": [h["step"] for h in hist],
           "forwards": fwd,
           "misfit_reduction": hist[0]["phi_d0"] / max(hist[-1]["phi_d1"], 1e-300)}
    print(json.dumps(out))
    s.close()
    return 0

def run_sources(args):
    """The default workload (128^3, c = 8, 16 dipoles, 512 receivers) with source bases
    (Sec. 3.2): one forward + gradient per step, timed like the default line, beside the
    same steps without source bases on the same inputs."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.msfv import Session
    n = args.n
    prob, m_np = W.config_3d_128(n=n)
    stream = torch.cuda.current_stream(dev)
    m = torch.from_numpy(m_np).to(dev)
    m_true = torch.from_numpy(W.config_3d_128(seed=3, n=n)[1]).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for sb in (False, True):
        prob.source_bases = sb
        sess = Session(prob, stream=stream)
        d_true = sess.forward(m_true).clone()
        noise = torch.from_numpy(W.noise_like(tuple(d_true.shape), 1.0, 4)).to(dev)
        d_obs = d_true + 0.01 * d_true.abs() * noise
        grad = torch.empty(prob.N, dtype=torch.float64, device=dev)
        d_pred = torch.empty((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            sess.forward(m, d_pred)
            sess.adjoint(d_obs, grad, want_phi=False)
        torch.cuda.synchronize(dev)
        sess.profile(True)
        sess.phase_times(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.3)
        l0 = sess.launch_count()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            sess.forward(m, d_pred)
            sess.adjoint(d_obs, grad, want_phi=False)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        launches = sess.launch_count() - l0
        clk = clocks.stop()
        ms = [a.elapsed_time(b) for a, b in ev]
        ph = sess.phase_times(reset=True)
        info = sess.info()
        res[sb] = {"ms": sum(ms) / len(ms), "p50": float(np.percentile(ms, 50)),
                   "p99": float(np.percentile(ms, 99)), "launches": launches, "clocks": clk,
                   "phases": {k: v[0] / args.steps for k, v in ph.items() if v[1]},
                   "slots": info["source_slots"], "values": info["source_values"],
                   "iters": (info["coarse_iters"], info["coarse_iters_T"])}
        sess.close()
    r1, r0 = res[True], res[False]
    out = {"metric": METRIC, "value": 1000.0 / r1["ms"], "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r1["ms"],
           "p50_ms": r1["p50"], "p99_ms": r1["p99"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"3d_{n}^3_c8_16dipoles_512rec_fwd+grad_source_bases",
                      "source_bases": True, "l2": "flushed before every timed step (512 MiB write)",
                      "factor_mode": "store"},
           "gpu_launches": r1["launches"], "clocks": r1["clocks"],
           "source_slots": r1["slots"], "source_values": r1["values"],
           "plain": {"value": 1000.0 / r0["ms"], "ms_per_step": r0["ms"]},
           "overhead": r1["ms"] / r0["ms"] - 1.0,
           "phases_ms_per_step": r1["phases"],
           "coarse_iters": {"source_bases": r1["iters"], "plain": r0["iters"]}}
    print(json.dumps(out))
    return 0


def run_nodal(args):
    """The paper's own variant (nodal operator, Lagrange block data, Galerkin A_k) on the
    default survey shape: 128^3 cells (129^3 nodes), c = 8, 16 dipoles and 512
    receivers on the top surface; one forward + gradient per step, timed like the
    default line."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.msfv import Session
    n = args.n
    prob = W.make_problem((n, n, n), 8, 16, 512, seed=2, top_layer=True, nodal=True)
    m_np = W.config_3d_128(n=n)[1]
    stream = torch.cuda.current_stream(dev)
    sess = Session(prob, stream=stream)
    m = torch.from_numpy(m_np).to(dev)
    m_true = torch.from_numpy(W.config_3d_128(seed=3, n=n)[1]).to(dev)
    d_true = sess.forward(m_true).clone()
    noise = torch.from_numpy(W.noise_like(tuple(d_true.shape), 1.0, 4)).to(dev)
    d_obs = d_true + 0.01 * d_true.abs() * noise
    grad = torch.empty(prob.N, dtype=torch.float64, device=dev)
    d_pred = torch.empty((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        sess.forward(m, d_pred)
        sess.adjoint(d_obs, grad, want_phi=False)
    torch.cuda.synchronize(dev)
    sess.profile(True)
    sess.phase_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    l0 = sess.launch_count()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sess.forward(m, d_pred)
        sess.adjoint(d_obs, grad, want_phi=False)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = sess.launch_count() - l0
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    ph = sess.phase_times(reset=True)
    info = sess.info()
    mean = sum(ms) / len(ms)
    out = {"metric": METRIC, "value": 1000.0 / mean, "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean,
           "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"3d_{n}^3_c8_16dipoles_512rec_fwd+grad_nodal_galerkin",
                      "discretization": "nodal", "nodes": [n + 1] * 3,
                      "l2": "flushed before every timed step (512 MiB write)",
                      "factor_mode": "store"},
           "gpu_launches": launches, "clocks": clk,
           "phases_ms_per_step": {k: v[0] / args.steps for k, v in ph.items() if v[1]},
           "coarse": {"solver": "mg-gmres" if info["coarse_solver"] else "banded-lu",
                      "iters_fwd": info["coarse_iters"], "iters_adj": info["coarse_iters_T"]}}
    print(json.dumps(out))
    sess.close()
    return 0


def main():
    args = parse()
    if args.precision == "mixed":
        os.environ["MSFV_LOCAL_PRECISION"] = "mixed"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "diff":
        return run_diff(args)
    if args.workload == "gn":
        return run_gn(args)
    if args.workload == "sources":
        return run_sources(args)
    if args.workload == "nodal":
        return run_nodal(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
