#!/usr/bin/env python3
"""Benchmark: batched MSFV forward + misfit-gradient solves per second on GB300, against
the plain one-instance path on the same instances.

Default workload (the batching configuration): 64 independent 3D instances, fine size
drawn uniformly from {64, 96, 128, 192}^3, coarsening from {4, 8, 16} (uneven dual-cell
sizes), lognormal conductivity with correlation length U[0.05, 0.2], 8-32 dipoles and
256 receivers on the top layer, all FP64.  One step = one forward solve (basis, coarse
operator, reduced solve, predicted data) plus the misfit gradient through dP/dm of every
instance, replayed as one captured CUDA graph; inputs resident in HBM (the working set
of a step is tens of GB, far larger than L2).  Beside it, in the same run: the same
instances one at a time without a graph (the plain path), bit-for-bit equality of the
two, oracle parity on one instance, the end-to-end rate through host buffers, the plain
128^3 single-instance line with its roofline, and the CPU oracle on a sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batched|plain|served|diff|gn|sources|nodal|oversample]

Under torchrun (N > 1) every rank runs an independent replica (the path has no
exchange step); value = solves of all ranks / max-over-ranks time.
``--impl reference`` times the CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import os

if os.environ.get("MSFV_ORACLE_WORKER") == "1":
    # oracle worker processes: one thread each, so the core count is the worker count
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import argparse  # noqa: E402
import json  # noqa: E402
import platform  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1707_07598_gb300 import workloads as W  # noqa: E402
from paper_1707_07598_gb300 import replicas as R  # noqa: E402

METRIC = "batched/served MSFV fwd+grad solves/s vs plain at 1e-9 rel err; p50/p99 ms"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk x 2 flop x max SM clock
FP64_PEAK_SOURCE = ("FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (unit counts and "
                    "maximum SM clock of the profiling recipe); measured_tflops is the "
                    "library's DFMA probe (msfv_fp64_probe) in this run")
WORKLOAD = "3d_128^3_c8_16dipoles_512rec_fwd+grad"
COARSE_SOLVERS = {0: "banded-lu", 1: "mg-gmres", 2: "nested-dissection-lu"}
# DRAM bytes (read + write) of one k_local_fwd<256,1> launch on the 128^3, c = 8 workload,
# from an ncu capture of that launch (dram__bytes_read.sum + dram__bytes_write.sum).  Set
# to None whenever the kernel changes, until it is captured again.
INTERIOR_DRAM_BYTES_128 = 117296896.0 + 549022464.0
# DRAM bytes per algorithmic FP64 flop of the c = 16 interior kernel (global-memory window,
# panels of 8), from an ncu capture of one launch on the 192^3, c = 16 plain workload (2197
# interiors: 80.06 GB read + 118.99 GB written for 2.684e11 flops).  The kernel's traffic is
# its windows' passes through L2 and HBM, which grow with its flops, so a fused launch over
# c = 16 interiors is scaled by its flop count.  Set to None whenever the kernel changes.
C16_DRAM_BYTES_PER_FLOP = (80062537216.0 + 118986263296.0) / 268362314256.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=128, help="plain: mesh size per axis (default 128)")
    p.add_argument("--coarsen", type=int, default=8, help="plain: coarsening factor (default 8)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--workload", default="batched",
                   choices=["batched", "plain", "served", "diff", "gn", "sources", "nodal",
                            "oversample"],
                   help="batched: 64 uneven instances in one CUDA graph per step vs one at a "
                        "time (default); plain: the one-instance 128^3 step; served: the "
                        "Poisson request stream; diff: 256^3, c=16 gradient, J v, J^T w; gn: "
                        "5 Gauss-Newton-CG iterations on the 128^3 two-block model; sources: "
                        "the 128^3 step with source bases beside the plain one; nodal: "
                        "the paper's nodal Galerkin variant on the same survey shape")
    p.add_argument("--instances", type=int, default=64, help="batched: number of instances")
    p.add_argument("--instance-budget-gb", type=float, default=0.0,
                   help="batched: per-instance HBM budget (0 = store every local factor)")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip the autotuner (default: the batched line tunes each instance "
                        "class once, the plain lines their session)")
    p.add_argument("--plain-reps", type=int, default=2,
                   help="batched: timed passes of the one-at-a-time comparison")
    p.add_argument("--rate", type=float, default=50.0, help="served: requests per second")
    p.add_argument("--duration", type=float, default=10.0,
                   help="served: seconds of the arrival stream that are replayed")
    p.add_argument("--fd-dirs", type=int, default=20, help="diff: finite-difference directions")
    p.add_argument("--oversample", type=int, default=2,
                   help="oversampling width of the dual edge and face problems "
                        "(--workload oversample)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                   help="local problems of the top dimension: FP64 factor (default) or FP32 "
                        "factor with two FP64 refinement steps")
    p.add_argument("--policy", default="sjf", choices=["fifo", "sjf"],
                   help="served: admission order of the continuous-batching loop")
    return p.parse_args()


def dist_env():
    e = R.rank_env()
    return e.rank, e.world, e.local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------------
def _oracle_worker(conn, spec, send_arrays):
    """One oracle instance in its own process: build it once (the set-up, untimed), then
    one forward + misfit gradient per request, timed; d_obs = 0.97 x the oracle's own
    prediction, as the GPU arm does with its prediction."""
    try:
        from oracle.msfv_oracle import Oracle
        prob = spec.problem()
        m = W.gaussian_random_field(prob.n, spec.corr_len, spec.seed)
        t0 = time.perf_counter()
        orc = Oracle(prob)
        conn.send(("ready", time.perf_counter() - t0))
        while True:
            msg = conn.recv()
            if msg != "step":
                break
            t0 = time.perf_counter()
            st = orc.forward(m)
            phi, g = orc.misfit_gradient(st, 0.97 * st['d'])
            dt = time.perf_counter() - t0
            conn.send(("done", dt, (st['d'], g, phi) if send_arrays else None))
    except Exception as exc:   # report and stop; the parent raises
        conn.send(("error", repr(exc)))


class OraclePool:
    """One spawned single-threaded process per sampled instance.  Processes start before
    any CUDA call of the parent; a step runs one oracle forward + gradient on every
    instance at once and returns the wall time."""

    def __init__(self, specs, arrays_for=()):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.specs = list(specs)
        self.conns, self.procs = [], []
        os.environ["MSFV_ORACLE_WORKER"] = "1"
        try:
            for i, sp in enumerate(self.specs):
                a, b = ctx.Pipe()
                pr = ctx.Process(target=_oracle_worker, args=(b, sp, i in arrays_for),
                                 daemon=True)
                pr.start()
                self.conns.append(a)
                self.procs.append(pr)
        finally:
            del os.environ["MSFV_ORACLE_WORKER"]
        self.ready = False
        self.pending = False
        self.t_start = 0.0

    def _recv(self, c):
        msg = c.recv()
        if msg[0] == "error":
            raise RuntimeError("oracle worker failed: " + msg[1])
        return msg

    def wait_ready(self):
        if not self.ready:
            self.setup_s = [self._recv(c)[1] for c in self.conns]
            self.ready = True

    def start_step(self):
        self.wait_ready()
        self.t_start = time.perf_counter()
        for c in self.conns:
            c.send("step")
        self.pending = True

    def finish_step(self):
        out = [self._recv(c) for c in self.conns]
        wall = time.perf_counter() - self.t_start
        self.pending = False
        return wall, [o[1] for o in out], [o[2] for o in out]

    def step(self):
        self.start_step()
        return self.finish_step()

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)


def oracle_sample(specs):
    """The batch's instances the oracle solves in about 10-15 s each on one core: the
    64^3 ones with c = 8 or 16 (those with c = 4 take about three times longer, the larger
    meshes minutes)."""
    return [i for i, sp in enumerate(specs) if sp.n[0] == 64 and sp.coarsen in (8, 16)]


def sample_text(specs, idx, cores):
    kinds = {}
    for i in idx:
        key = f"{specs[i].n[0]}^3 c={specs[i].coarsen}"
        kinds[key] = kinds.get(key, 0) + 1
    mix = ", ".join(f"{v} x {k}" for k, v in sorted(kinds.items()))
    return (f"per step, one oracle forward + misfit gradient of each of the {len(idx)} "
            f"instances of the batch that the oracle finishes in seconds ({mix}; the larger "
            f"instances take minutes to hours each, so the rate on the whole mix is lower), "
            f"one single-threaded process per instance on {cores} host cores; value = "
            f"instances / wall time; oracle set-up (geometry) outside the timing")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "plain":
        return run_reference_plain(args)
    specs = W.batch_instances(args.instances)
    idx = oracle_sample(specs)
    pool = OraclePool([specs[i] for i in idx])
    pool.wait_ready()
    for _ in range(args.warmup):
        pool.step()
    walls = []
    for _ in range(args.steps):
        walls.append(pool.step()[0])
    pool.close()
    ms = 1000.0 * statistics.mean(walls)
    val = len(idx) * len(walls) / sum(walls)
    cores = len(idx)
    cfg = batched_config(specs, args)
    out = {"metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference", "config": cfg,
           "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": sample_text(specs, idx, cores),
                            "host_cores": host_cores(), "cpu_model": cpu_model()},
           "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_reference_plain(args):
    """The oracle on the full 128^3 plain workload, one forward + gradient per step."""
    from oracle.msfv_oracle import Oracle
    prob, m = W.config_3d_128(n=args.n)
    orc = Oracle(prob)

    def one():
        t0 = time.perf_counter()
        st = orc.forward(m)
        orc.misfit_gradient(st, st['d'] * 1.01)
        return time.perf_counter() - t0
    for _ in range(args.warmup):
        one()
    times = [one() for _ in range(args.steps)]
    ms = 1000.0 * statistics.mean(times)
    val = 1000.0 / ms
    out = {"metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": [args.n] * 3, "coarsen": 8, "n_src": 16,
                      "n_rec": 512},
           "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                            "sample": f"one oracle forward + gradient of the whole {args.n}^3 "
                                      "workload per step, one process, one thread",
                            "cpu_model": cpu_model()},
           "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def batched_config(specs, args):
    mix = {}
    for sp in specs:
        key = f"{sp.n[0]}^3_c{sp.coarsen}"
        mix[key] = mix.get(key, 0) + 1
    return {"workload": f"batched_{len(specs)}_instances_3d_sizes64-192_c4-16_8-32dipoles_256rec",
            "instances": len(specs), "mix": mix, "sizes": [64, 96, 128, 192],
            "coarsenings": [4, 8, 16], "dipoles": "8-32", "receivers": 256,
            "corr_len": "U[0.05, 0.2]", "parallelism": "replicas x1",
            "l2": "inputs and working set of a step (tens of GB) far larger than L2",
            "graph": "one CUDA graph per step: per-instance branches for the edges, faces, coarse problems and gradients, fused persistent launches for the dual-cell interiors of instances of one kernel shape"}


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


def plain_measure(args, dev, sess, prob, m, d_obs, world=1):
    """Time the plain one-instance step (msfv_forward + msfv_adjoint) of an open session:
    CUDA events on the session stream, L2 flushed before each step, phase timers for the
    roofline of the interior basis kernel, and the end-to-end rate through host buffers."""
    import torch
    stream = torch.cuda.current_stream(dev)
    grad = torch.empty(prob.N, dtype=torch.float64, device=dev)
    d_pred = torch.empty((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        sess.forward(m, d_pred)
        sess.adjoint(d_obs, grad, want_phi=False)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    sess.profile(True)
    sess.phase_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
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
    step_ms = [a.elapsed_time(b) for a, b in ev]
    phases = sess.phase_times(reset=True)
    sess.profile(False)
    info = sess.info()
    total_ms = R.max_over_ranks(sum(step_ms), dev)
    # roofline of the dominant kernel of this step: the dual-cell interior basis solve
    int_ms, int_calls = phases.get("basis_interiors", (0.0, 0))
    int_avg_s = (int_ms / max(int_calls, 1)) / 1000.0
    flops = sess.interior_flops()
    achieved = flops / int_avg_s / 1e12 if int_avg_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_local_fwd<256,1> (3D dual-cell interiors)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_SOURCE,
            "flops_per_launch": flops, "avg_launch_ms": int_avg_s * 1000.0,
            "traffic": INTERIOR_DRAM_BYTES_128
            if (args.n == 128 and getattr(args, "coarsen", 8) == 8 and args.precision == "fp64")
            else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of "
                              "this kernel on the 128^3 workload"}
    if args.precision == "mixed":
        roof.update(kernel="k_mix_fwd (3D dual-cell interiors: FP32 band factor, two FP64 "
                           "refinement steps)",
                    note="the method's FP64 flop count (the same numerator as the FP64 kernel) "
                         "over the FP64 peak; most of the arithmetic runs in FP32")
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
    return {"value": R.whole_job_rate(world, args.steps, total_ms / 1000.0), "unit": "solves/s",
            "ms_per_step": total_ms / args.steps,
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "roofline": roof, "e2e": e2e, "gpu_launches": launches,
            "phases_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in phases.items() if v[1]},
            "coarse": {"solver": COARSE_SOLVERS[info["coarse_solver"]],
                       "iters_fwd": info["coarse_iters"], "iters_adj": info["coarse_iters_T"]},
            "kernel_shapes": getattr(args, "tuned_shapes", None)}


def open_plain(args, dev, seed_model=2, seed_truth=3, seed_noise=4):
    """The 128^3 plain workload: session, model and observed data (forward at an
    independent model plus 1% noise, outside any timing)."""
    import torch
    from paper_1707_07598_gb300.msfv import Session
    c = getattr(args, "coarsen", 8)
    prob, m_np = W.config_3d_128(seed=seed_model, n=args.n, coarsen=c)
    sess = Session(prob, stream=torch.cuda.current_stream(dev))
    m = torch.from_numpy(m_np).to(dev)
    if not getattr(args, "no_autotune", False):
        # kernel shape per entity class (set-up, outside any timing)
        args.tuned_shapes = {k: v[0] for k, v in sess.autotune(m).items()}
    m_true = torch.from_numpy(W.config_3d_128(seed=seed_truth, n=args.n, coarsen=c)[1]).to(dev)
    d_true = sess.forward(m_true).clone()
    noise = torch.from_numpy(W.noise_like(tuple(d_true.shape), 1.0, seed_noise)).to(dev)
    d_obs = d_true + 0.01 * d_true.abs() * noise
    return sess, prob, m, d_obs


def run_plain(args):
    """The plain one-instance line: 128^3, c = 8, 16 dipoles, 512 receivers."""
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
    seeds = R.replica_seeds(rank)
    sess, prob, m, d_obs = open_plain(args, dev, seeds.model, seeds.truth, seeds.noise)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    time.sleep(0.3)
    res = plain_measure(args, dev, sess, prob, m, d_obs, world)
    clk = clocks.stop()
    if rank == 0:
        out = {"metric": METRIC, "value": res["value"], "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
               "p50_ms": res["p50_ms"], "p99_ms": res["p99_ms"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD if (args.n == 128 and args.coarsen == 8)
                          else f"3d_{args.n}^3_c{args.coarsen}",
                          "n": [args.n] * 3, "coarsen": args.coarsen, "n_src": prob.n_src,
                          "n_rec": prob.n_rec, "parallelism": f"replicas x{world}",
                          "l2": "flushed before every timed step (512 MiB write)",
                          "factor_mode": "store", "precision": args.precision,
                          "order": "first order in h at even c (coarse vertex half a cell off "
                                   "the coarse-cell centre)"},
               "roofline": res["roofline"], "cpu_baseline": None, "e2e": res["e2e"],
               "gpu_launches": res["gpu_launches"], "clocks": clk,
               "phases_ms_per_step": res["phases_ms_per_step"], "coarse": res["coarse"],
               "kernel_shapes": res["kernel_shapes"]}
        print(json.dumps(out))
    sess.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _gpu_setup():
    import torch
    from paper_1707_07598_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    return torch, dev


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r2 = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    ri = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
    return float(max(r2, ri))


def run_batched(args):
    """The default line: independent 3D instances (sizes 64..192^3, c in {4, 8, 16}, 8-32
    dipoles) as one CUDA graph per step, against the same instances one at a time."""
    import torch
    from paper_1707_07598_gb300 import build as B
    rank, world, local = dist_env()
    specs = W.batch_instances(args.instances, seed=3 + 1000 * rank)
    sample = oracle_sample(specs)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and sample:
        # before any CUDA call: the oracle processes start now and build their instances
        # while the GPU sessions are set up; their timed step runs after the GPU timings,
        # with the host otherwise idle
        pool = OraclePool([specs[i] for i in sample], arrays_for=(0,))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    B.build()
    from paper_1707_07598_gb300.msfv import Batch, Session, fp64_probe
    stream = torch.cuda.current_stream(dev)
    t_setup = time.perf_counter()
    budget = int(args.instance_budget_gb * (1 << 30))
    sessions, ms, dobs = [], [], []
    tuned = {}
    for k, sp in enumerate(specs):
        prob = sp.problem()
        sessions.append(Session(prob, stream=torch.cuda.Stream(dev), factor_mode=0,
                                hbm_budget_bytes=budget))
        if k in sample:    # the host generator: the oracle draws the same field
            ms.append(torch.from_numpy(W.gaussian_random_field(prob.n, sp.corr_len,
                                                               sp.seed)).to(dev))
        else:
            ms.append(W.gaussian_random_field_device(prob.n, sp.corr_len, sp.seed, dev))
        dobs.append(torch.zeros((prob.n_src, prob.n_rec), dtype=torch.float64, device=dev))
        key = (sp.n[0], sp.coarsen)
        if not args.no_autotune and key not in tuned:
            tuned[key] = sessions[-1].autotune(ms[-1])
    torch.cuda.synchronize()
    batch = Batch(sessions, ms, dobs, stream=stream)
    batch.run()
    batch.check()
    for k in range(len(specs)):                       # observed data: 97% of the prediction
        dobs[k].copy_(0.97 * batch.d_pred[k])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    cpu = None
    parity = None
    for _ in range(max(args.warmup - 1, 0)):
        batch.run()
    batch.check()
    fp64_tf, _ = fp64_probe(stream)
    # ---- timed: the batched step ----------------------------------------------------
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    R.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        ev[k][0].record(stream)
        batch.run()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    R.barrier()
    batch.check()
    clk = clocks.stop()
    bt = [a.elapsed_time(b) for a, b in ev]
    K = len(specs)
    # the same graph without fused interior launches (each instance its own branch)
    unfused = None
    if args.plain_reps > 0:
        os.environ["MSFV_BATCH_FUSE"] = "0"
        try:
            ub = Batch(sessions, ms, dobs, stream=stream)
        finally:
            del os.environ["MSFV_BATCH_FUSE"]
        ub.run()
        ub.check()
        ut = []
        for _ in range(max(1, args.plain_reps)):
            a = torch.cuda.Event(enable_timing=True)
            b2 = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ub.run()
            b2.record(stream)
            torch.cuda.synchronize(dev)
            ut.append(a.elapsed_time(b2))
        ub.check()
        ub.close()
        unfused = {"value": K / (float(np.mean(ut)) / 1000.0), "unit": "solves/s",
                   "ms_per_step": float(np.mean(ut)),
                   "path": "the same graph with every instance in its own branch (no fused "
                           "interior launches)"}
    total_ms = R.max_over_ranks(sum(bt), dev)
    value = R.whole_job_rate(world, K * args.steps, total_ms / 1000.0)
    d_b = [t.clone() for t in batch.d_pred]
    g_b = [t.clone() for t in batch.grad]
    # ---- the plain path: the same instances one at a time, no graph -------------------
    plain_ms, inst_ms = [], np.zeros(K)
    phase_tot = {}
    roof_cls = {}
    launches_step = 0
    same = True
    for s in sessions:
        s.set_stream(stream)
    for rep in range(max(1, args.plain_reps)):
        prof = rep == 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ie = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for k, s in enumerate(sessions):
            if prof:
                s.profile(True)
                s.phase_times(reset=True)
                l0 = s.launch_count()
            ie[k][0].record(stream)
            d = s.forward(ms[k])
            _, g = s.adjoint(dobs[k], want_phi=False)
            ie[k][1].record(stream)
            if prof:
                launches_step += s.launch_count() - l0
            if rep == 0:
                same = same and torch.equal(d, d_b[k]) and torch.equal(g, g_b[k])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms.append(e0.elapsed_time(e1))
        for k in range(K):
            inst_ms[k] += ie[k][0].elapsed_time(ie[k][1]) / max(1, args.plain_reps)
        if prof:
            for k, s in enumerate(sessions):
                ph = s.phase_times(reset=True)
                s.profile(False)
                for name, (t, c) in ph.items():
                    phase_tot[name] = phase_tot.get(name, 0.0) + t
                tms, tc = ph.get("basis_interiors", (0.0, 0))
                cls = f"c{specs[k].coarsen}"
                r = roof_cls.setdefault(cls, {"flops": 0.0, "ms": 0.0, "launches": 0})
                r["flops"] += s.interior_flops() * tc
                r["ms"] += tms
                r["launches"] += tc
    plain_val = R.whole_job_rate(world, K, R.max_over_ranks(float(np.mean(plain_ms)), dev) / 1000.0)
    # roofline of the dominant kernel: the fused launch of the dual-cell interiors of the
    # group that takes longest, timed with CUDA events on its stream in an eager replay of
    # the step (msfv_batch_run_timed; the launches inside the graph are the same kernels on
    # the same work lists).  Beside it, the interior kernels of the one-at-a-time pass per
    # coarsening class.
    groups = []
    for rep in range(2):
        if rep == 1:   # marks one eager step's launches for the profiler's launch list
            torch.cuda.nvtx.range_push("msfv_batched_step_eager")
        groups = batch.run_timed()
        if rep == 1:
            torch.cuda.nvtx.range_pop()
    roof = {"bound": "alu", "kernel": None, "achieved": 0.0, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": 0.0, "peak_source": FP64_PEAK_SOURCE,
            "measured_tflops": fp64_tf, "traffic": None}
    if groups:
        gtop = max(groups, key=lambda q: q["fwd_ms"])
        ach = gtop["flops"] / (gtop["fwd_ms"] / 1000.0) / 1e12 if gtop["fwd_ms"] > 0 else 0.0
        roof.update(kernel=f"k_local_fwd<256,1> fused over the batch: {gtop['entities']} dual-cell "
                           f"interiors of up to {gtop['nmax']} unknowns, half bandwidth "
                           f"{gtop['bmax']}",
                    achieved=ach, frac=ach / FP64_PEAK_TFLOPS,
                    frac_of_measured=ach / fp64_tf if fp64_tf else None,
                    flops_per_launch=gtop["flops"], avg_launch_ms=gtop["fwd_ms"],
                    traffic=C16_DRAM_BYTES_PER_FLOP * gtop["flops"]
                    if (C16_DRAM_BYTES_PER_FLOP and gtop["bmax"] == 225) else None,
                    traffic_source="ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                   "c = 16 interior kernel on one 192^3 instance (one launch, "
                                   "2197 interiors), per algorithmic flop, times this launch's "
                                   "flops",
                    fused_groups=[dict(q, achieved_tflops=q["flops"] / (q["fwd_ms"] / 1000.0) / 1e12
                                       if q["fwd_ms"] > 0 else 0.0) for q in groups])
    fl = sum(r["flops"] for r in roof_cls.values())
    tm = sum(r["ms"] for r in roof_cls.values())
    top = max(phase_tot.items(), key=lambda kv: kv[1])[0] if phase_tot else None
    roof["plain_pass_interiors"] = {
        "achieved": fl / (tm / 1000.0) / 1e12 if tm > 0 else 0.0, "ms_per_step": tm,
        "by_class": {c: {"achieved": r["flops"] / (r["ms"] / 1000.0) / 1e12 if r["ms"] else 0.0,
                         "ms_per_step": r["ms"], "launches": r["launches"]}
                     for c, r in sorted(roof_cls.items())},
        "largest_phase": top,
        "phase_share": {k2: v / max(sum(phase_tot.values()), 1e-12)
                        for k2, v in sorted(phase_tot.items(), key=lambda kv: -kv[1])[:6]}}
    # ---- end to end: host buffers through msfv_batch_run_host -------------------------
    e2e = None
    if not args.no_e2e:
        mh = [torch.empty(t.numel(), dtype=torch.float64).pin_memory() for t in ms]
        dh = [torch.empty(tuple(t.shape), dtype=torch.float64).pin_memory() for t in dobs]
        for k in range(K):
            mh[k].copy_(ms[k].cpu())
            dh[k].copy_(dobs[k].cpu())
        ph_ = [torch.empty(tuple(t.shape), dtype=torch.float64).pin_memory() for t in dobs]
        gh = [torch.empty(t.numel(), dtype=torch.float64).pin_memory() for t in ms]
        args_h = ([x.numpy() for x in mh], [x.numpy().reshape(-1) for x in dh],
                  [x.numpy().reshape(-1) for x in ph_], [x.numpy() for x in gh])
        batch.run_host(*args_h)
        n_e2e = max(1, min(args.steps, 3))
        R.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            batch.run_host(*args_h)
        tot = R.max_over_ranks(time.perf_counter() - t0, dev)
        same = same and all(np.array_equal(args_h[3][k], g_b[k].cpu().numpy()) for k in range(K))
        hb = sum(8 * t.numel() for t in ms) + sum(8 * t.numel() for t in dobs)
        db = sum(8 * t.numel() for t in ms) + sum(8 * t.numel() for t in dobs)
        e2e = {"value": R.whole_job_rate(world, K * n_e2e, tot), "unit": "solves/s",
               "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db, "steps": n_e2e,
               "api": "msfv_batch_run_host (pinned host buffers, copies inside the timing)"}
    # ---- the plain 128^3 single-instance line ---------------------------------------
    plain128 = None
    if world == 1:
        psess, pprob, pm, pdobs = open_plain(args, dev)
        pres = plain_measure(args, dev, psess, pprob, pm, pdobs, 1)
        psess.close()
        plain128 = dict(pres, workload=WORKLOAD,
                        note="the plain one-instance configuration: 128^3, c = 8, 16 "
                             "dipoles, 512 receivers; L2 flushed before each step; first "
                             "order in h at even c (coarse vertex half a cell off the "
                             "coarse-cell centre)")
    # ---- the CPU oracle on the sample (after the GPU timings: the host is idle), and
    # parity on the first sampled instance (same field, same survey) --------------------
    if pool is not None:
        wall, times, arrays = pool.step()
        pool.close()
        cpu = {"value": len(sample) / wall, "unit": "solves/s", "cores": len(sample),
               "kind": "oracle", "sample": sample_text(specs, sample, len(sample)),
               "wall_s": wall, "host_cores": host_cores(), "cpu_model": cpu_model(),
               "per_instance_s": times}
    if pool is not None and arrays[0] is not None:
        i0 = sample[0]
        d_o, g_o, phi_o = arrays[0]
        parity = {"instance": f"{specs[i0].n[0]}^3 c={specs[i0].coarsen} "
                              f"({specs[i0].n_src} dipoles)",
                  "rel_err_d": rel_err(d_b[i0].cpu().numpy(), d_o),
                  "rel_err_grad": rel_err(g_b[i0].cpu().numpy(), g_o),
                  "tol": 1e-9, "norm": "max of relative 2-norm and max-norm"}
        parity["ok"] = parity["rel_err_d"] < 1e-9 and parity["rel_err_grad"] < 1e-9
        gpu_same = sum(inst_ms[i] for i in sample) / 1000.0
        cpu["gpu_plain_same_sample"] = {"value": len(sample) / gpu_same, "unit": "solves/s",
                                        "note": "the same sampled instances on the GPU, one "
                                                "at a time"}
    recompute = sum(int(s.info()["recompute"]) for s in sessions)
    ws_gb = sum(int(s.info()["workspace_bytes"]) for s in sessions) / 1e9
    if rank == 0:
        cfg = batched_config(specs, args)
        cfg.update(recompute_instances=recompute, workspace_gb=ws_gb, fusion=batch.info(),
                   parallelism=f"replicas x{world}", autotuned_classes=len(tuned),
                   setup_s=setup_s)
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": total_ms / args.steps,
               "p50_ms": float(np.percentile(bt, 50)), "p99_ms": float(np.percentile(bt, 99)),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic", "config": cfg,
               "plain": {"value": plain_val, "unit": "solves/s",
                         "ms_per_step": float(np.mean(plain_ms)),
                         "path": "same sessions and inputs, msfv_forward + msfv_adjoint one "
                                 "instance at a time on one stream, no graph",
                         "per_instance_ms_p50": float(np.percentile(inst_ms, 50)),
                         "per_instance_ms_p99": float(np.percentile(inst_ms, 99))},
               "speedup_vs_plain": value / plain_val if plain_val else None,
               "graph_without_fusion": unfused,
               "bitwise_equal_to_plain": bool(same), "oracle_parity": parity,
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches_step * args.steps, "clocks": clk,
               "plain_128": plain128}
        print(json.dumps(out))
    batch.close()
    for s in sessions:
        s.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    ok = same and (parity is None or parity["ok"])
    return 0 if ok else 1


def run_served(args):
    """The Poisson request stream (rate x duration), fine sizes 32..256^3, c in {4, 8, 16},
    1-64 dipoles, 150 GB budget: continuous batching against one request at a time.
    Runs the checked build of the library (MSFV_CHECKED=1 unless set otherwise): its local
    and nested-dissection kernels validate every work descriptor before they touch its
    storage."""
    os.environ.setdefault("MSFV_CHECKED", "1")
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
           "build": "checked" if os.environ.get("MSFV_CHECKED", "0") not in ("", "0") else "default",
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


def run_oversample(args):
    """The default workload (128^3, c = 8, 16 dipoles, 512 receivers) with oversampled dual
    edge and face problems (width --oversample; Sec. 6 names oversampling, the
    construction is the library's reading): one forward + gradient per step, timed like
    the default line, beside the same steps without oversampling on the same inputs.  The
    roofline is that of the face boxes' basis kernel (k_over_fwd), FP64 flops over the
    phase timer of its launch."""
    torch, dev = _gpu_setup()
    from paper_1707_07598_gb300.msfv import Session
    n = args.n
    prob, m_np = W.config_3d_128(n=n)
    stream = torch.cuda.current_stream(dev)
    m = torch.from_numpy(m_np).to(dev)
    m_true = torch.from_numpy(W.config_3d_128(seed=3, n=n)[1]).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for w in (0, args.oversample):
        prob.oversample = w
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
        res[w] = {"ms": sum(ms) / len(ms), "p50": float(np.percentile(ms, 50)),
                  "p99": float(np.percentile(ms, 99)), "launches": launches, "clocks": clk,
                  "phases": {k: v[0] / args.steps for k, v in ph.items() if v[1]},
                  "phase_calls": {k: v[1] for k, v in ph.items() if v[1]},
                  "info": info, "d": d_pred.clone(), "g": grad.clone()}
        sess.close()
    r1, r0 = res[args.oversample], res[0]
    info = r1["info"]
    face_ms = r1["phases"].get("basis_faces", 0.0)
    face_calls = max(1, r1["phase_calls"].get("basis_faces", 1) // max(args.steps, 1))
    launch_s = face_ms / face_calls / 1000.0
    flops = float(info["oversampled_face_flops"])
    achieved = flops / launch_s / 1e12 if launch_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_over_fwd (oversampled dual-face boxes)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_SOURCE,
            "flops_per_launch": flops, "avg_launch_ms": launch_s * 1000.0, "traffic": None}
    dd = (r1["d"] - r0["d"]).norm().item() / max(r0["d"].norm().item(), 1e-300)
    out = {"metric": METRIC, "value": 1000.0 / r1["ms"], "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r1["ms"],
           "p50_ms": r1["p50"], "p99_ms": r1["p99"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"3d_{n}^3_c8_16dipoles_512rec_fwd+grad_oversample{args.oversample}",
                      "oversample": args.oversample,
                      "l2": "flushed before every timed step (512 MiB write)",
                      "factor_mode": "store"},
           "roofline": roof, "gpu_launches": r1["launches"], "clocks": r1["clocks"],
           "oversampled_boxes": info["oversampled_boxes"],
           "oversampled_face_kernel": {"smem_bytes": info["oversampled_smem_bytes"],
                                       "grid": info["oversampled_grid"]},
           "plain": {"value": 1000.0 / r0["ms"], "ms_per_step": r0["ms"]},
           "overhead": r1["ms"] / r0["ms"] - 1.0,
           "data_change_vs_plain": dd,
           "phases_ms_per_step": r1["phases"],
           "plain_phases_ms_per_step": r0["phases"]}
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
           "coarse": {"solver": COARSE_SOLVERS[info["coarse_solver"]],
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
    runners = {"batched": run_batched, "plain": run_plain, "served": run_served,
               "diff": run_diff, "gn": run_gn, "sources": run_sources, "nodal": run_nodal,
               "oversample": run_oversample}
    return runners[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())
