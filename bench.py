#!/usr/bin/env python
"""Throughput of design evaluations (solve + adjoint gradient) on GB300.

Workload: the continuous-shell configuration -- 64 x 64 MITC-4 quads
(4,225 nodes, 25,350 DOF) on a 20 m plan, z from a seeded smooth bump of
0..5 m, per-element thickness U[0.05, 0.2] m, E = 30 GPa, nu = 0.2, corners
pinned, self-weight 25 kN/m^3 x t.  A step evaluates a batch of B seeded
designs (different z and t on the same mesh): FP64 element matrices, bit-exact
assembly, block-Jacobi FP32 CG inside FP64 iterative refinement to a relative
FP64 residual of rtol, compliance, and the adjoint dC/dz, dC/dt (Eqs. 5-6).

Prints one JSON line (rank 0).  `value` is designs/s with the designs already
resident in HBM; `e2e` is the same through the C-ABI from host buffers
(design upload and result download inside the timed region).  `roofline`
reports the dominant kernel (CG kernel A: the FP32 BSR SpMV, or the FP64
residual SpMV in refinement passes), timed live with CUDA events on the
library's stream.  `--impl reference` times the FP64 CPU oracle on the same
workload instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402

METRIC = "design evals/sec (solve + adjoint grad) at <=1e-6 rel err vs FP64"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=128, help="designs per step")
    p.add_argument("--n-el", type=int, default=64)
    p.add_argument("--precision", default="fp32_ir", choices=["fp32_ir", "fp64"])
    p.add_argument("--precond", default="block_jacobi", choices=["block_jacobi", "jacobi"])
    p.add_argument("--rtol", type=float, default=1e-6)
    p.add_argument("--inner-rtol", type=float, default=1e-3)
    p.add_argument("--iters-per-launch", type=int, default=32)
    p.add_argument("--cpu-sample", type=int, default=3, help="oracle designs in cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def design_model(n_el, seed):
    return meshgen.shell(n_el=n_el, seed=seed)


def workload_name(a):
    n = a.n_el
    dof = 6 * (n + 1) ** 2
    return ("shell %dx%d quads (%d DOF), %d designs/step, %s %s CG + FP64 refinement to rtol %g, "
            "solve + adjoint dC/dz, dC/dt" % (n, n, dof, a.batch,
                                               "FP32" if a.precision == "fp32_ir" else "FP64",
                                               a.precond, a.rtol))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(kernel_file, key):
    """ncu DRAM bytes per launch of the dominant kernel, if the committed
    summary was taken on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[key]
        src = open(os.path.join(ROOT, "paper_2407_20026_gb300", "csrc", kernel_file), "rb").read()
        if rec.get("source_sha256") != hashlib.sha256(src).hexdigest():
            return None
        return rec
    except (OSError, KeyError, ValueError):
        return None


def cpu_oracle_sample(a, n_designs, gpu_results=None):
    """Times the oracle (FP64 band Cholesky + dual-number adjoint, 1 thread)
    on `n_designs` designs of the workload; compares with GPU results."""
    import oracle
    oracle.build()
    errs = []
    t0 = time.perf_counter()
    refs = []
    for i in range(n_designs):
        refs.append(oracle.gradient(design_model(a.n_el, i)))
    dt = time.perf_counter() - t0
    if gpu_results:
        for i, ref in enumerate(refs):
            if i in gpu_results:
                g = gpu_results[i]

                def rel(x, y):
                    return float(np.linalg.norm(x - y) / np.linalg.norm(y))
                errs.append({"u": rel(g["u"], ref["u"]),
                             "C": abs(g["C"] - ref["C"]) / abs(ref["C"]),
                             "dz": rel(g["dz"], ref["dz"]), "dt": rel(g["dt"], ref["dt"])})
    return n_designs / dt, dt, errs


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    for i in range(a.warmup):
        oracle.gradient(design_model(a.n_el, i))
    times = []
    for k in range(a.steps):
        t0 = time.perf_counter()
        oracle.gradient(design_model(a.n_el, k))
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = a.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000 * total / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a).replace("%d designs/step" % a.batch,
                                                        "1 design/step"),
                   "oracle": "FP64 band Cholesky + dual-number adjoint, single thread"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": "%d designs of the workload, one per step" % a.steps},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2407_20026_gb300 as sso
    from paper_2407_20026_gb300 import _build
    _build.build()

    B = a.batch
    seeds = [rank * B + i for i in range(B)]
    meshes = [design_model(a.n_el, s) for s in seeds]
    models = [sso.Model(m) for m in meshes]
    batch = sso.Batch(models)
    opts = sso.options(precision=a.precision, precond=a.precond, rtol=a.rtol,
                       inner_rtol=a.inner_rtol, iters_per_launch=a.iters_per_launch)
    z_dev = [torch.tensor(m["xyz"][:, 2], device=dev) for m in meshes]
    t_dev = [torch.tensor(m["quad_props"][:, 0], device=dev) for m in meshes]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step_device():
        for i, mdl in enumerate(models):
            mdl.set_design(z_dev[i], t_dev[i])
        st = batch.solve(opts)
        batch.gradient()
        return st

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up (also captures the CUDA graphs)
    for _ in range(a.warmup):
        stats = step_device()
    torch.cuda.synchronize()

    # timed region: device-resident designs
    peak_gbs, peak_kind = measured_peaks()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = sso.kernel_launches()
    batch.set_profiling(True)
    step_ms = []
    iters_total = 0
    sweeps_total = 0
    for k in range(a.steps):
        flush.fill_(float(k))  # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = step_device()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        bad = [s for s in stats if s["status"] != 0]
        if bad:
            raise RuntimeError("solve failed: %s" % bad[:3])
        iters_total += sum(s["iterations"] for s in stats)
        sweeps_total += sum(s["sweeps"] for s in stats)
    torch.cuda.synchronize()
    ms_a, ms_b, timed_pairs = batch.kernel_times()
    batch.set_profiling(False)
    launches = sso.kernel_launches() - launches0
    clk = clocks.stop()
    barrier()
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * B * a.steps / (total_ms / 1000.0)

    # algorithmic bytes of kernel A over the timed region
    n_nodes = models[0].n_nodes
    nblk = models[0].n_blocks
    fp32 = a.precision == "fp32_ir"
    wsz = 4 if fp32 else 8
    bytes_pcg = nblk * (36 * wsz + 4) + (n_nodes + 1) * 4 + 4 * (6 * n_nodes * wsz)
    bytes_resid = nblk * (36 * 8 + 4) + (n_nodes + 1) * 4 + 3 * (6 * n_nodes * 8)
    alg_bytes = iters_total * bytes_pcg + sweeps_total * bytes_resid
    achieved = alg_bytes / (ms_a / 1000.0) / 1e9 if ms_a > 0 else None
    a_launches = timed_pairs
    traffic = kernel_traffic("pcg.cu", "pcg_a_%s" % ("f32" if fp32 else "f64"))
    traffic_bytes = traffic["dram_bytes_per_design_launch"] * B if traffic else None

    # end to end: designs from pinned host memory, results back to host
    e2e = None
    if not a.no_e2e:
        z_host = [torch.tensor(m["xyz"][:, 2]).pin_memory() for m in meshes]
        t_host = [torch.tensor(m["quad_props"][:, 0]).pin_memory() for m in meshes]
        nq = models[0].n_quads
        out_u = [torch.empty(6 * n_nodes, dtype=torch.float64).pin_memory() for _ in models]
        out_dz = [torch.empty(n_nodes, dtype=torch.float64).pin_memory() for _ in models]
        out_dt = [torch.empty(nq, dtype=torch.float64).pin_memory() for _ in models]
        out_C = torch.empty(B, dtype=torch.float64).pin_memory()
        from paper_2407_20026_gb300 import _lib as L

        def step_e2e():
            for i, mdl in enumerate(models):
                mdl.set_design(z_host[i], t_host[i])
            st = batch.solve(opts)
            batch.gradient()
            for i, mdl in enumerate(models):
                L.check(L.load().sso_model_get(mdl.handle, out_u[i].data_ptr(),
                                               out_C.data_ptr() + 8 * i, out_dz[i].data_ptr(),
                                               out_dt[i].data_ptr(), None))
            return st

        step_e2e()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(a.steps):
            step_e2e()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = B * (n_nodes + nq) * 8
        d2h = B * (6 * n_nodes + n_nodes + nq + 1) * 8
        e2e = {"value": world * B * a.steps / e2e_s, "unit": "evals/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        gres = {}
        for i in range(min(a.cpu_sample, B)):
            r = models[i].result()
            gres[i] = r
        v, secs, errs = cpu_oracle_sample(a, min(a.cpu_sample, B), gres)
        cpu = {"value": v, "unit": "evals/s", "cores": 1, "kind": "oracle",
               "sample": "%d designs of the workload (seeds 0..%d), %.1f s" %
                         (min(a.cpu_sample, B), min(a.cpu_sample, B) - 1, secs)}
        if errs:
            accuracy = {k: max(e[k] for e in errs) for k in errs[0]}

    if rank == 0:
        lat = np.array(step_ms)
        n_free = 6 * n_nodes - int(meshes[0]["fixed"].sum())
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "designs_per_step": B,
                       "dof_per_design": 6 * n_nodes, "precision": a.precision,
                       "precond": a.precond, "rtol": a.rtol, "inner_rtol": a.inner_rtol,
                       "l2": "flushed between steps (256 MB write); working set > L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99))},
            "pcg_dof_per_s": n_free * iters_total / (total_ms / 1000.0) * world,
            "cg_iterations_per_design": iters_total / (B * a.steps),
            "roofline": {
                "bound": "hbm", "kernel": "pcg_a (BSR SpMV%s)" % (" FP32" if fp32 else " FP64"),
                "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs if achieved else None,
                "peak_kind": peak_kind,
                "traffic": traffic_bytes,
                "traffic_source": "profiles/traffic.json (ncu, scaled by designs)" if traffic else None,
                "alg_bytes_per_launch": alg_bytes / max(a_launches, 1),
                "alg_bytes_per_cg_launch": B * bytes_pcg,
                "launches_timed": a_launches, "kernel_ms_total": ms_a,
                "kernel_b_ms_total": ms_b,
            },
            "cpu_baseline": cpu, "accuracy_vs_oracle": accuracy,
            "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
