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
    p.add_argument("--batch", type=int, default=256, help="designs per step")
    p.add_argument("--n-el", type=int, default=64)
    p.add_argument("--precision", default="fp32_ir", choices=["fp32_ir", "fp64"])
    p.add_argument("--precond", default="block_jacobi",
                   choices=["block_jacobi", "jacobi", "two_level"])
    p.add_argument("--rtol", type=float, default=1e-6)
    p.add_argument("--inner-rtol", type=float, default=2e-3)
    p.add_argument("--iters-per-launch", type=int, default=32)
    p.add_argument("--parts", type=int, default=0,
                   help="shell: concurrent parts of the batch's CG (0: the library's choice)")
    p.add_argument("--cpu-sample", type=int, default=3, help="oracle designs in cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-two-level", action="store_true",
                   help="default line: skip the two-level preconditioner sub-record")
    p.add_argument("--workload", default="shell",
                   choices=["shell", "serving", "gridshell", "large", "training", "bridge"],
                   help="shell: batches of 64x64 shell designs (default line); serving: "
                        "continuous batching of a grid-shell request stream; gridshell: "
                        "latency of one 10x10 grid-shell evaluation; large: one 512x512 shell; "
                        "training: MLP through 64 batched 48x48 shell solves per step; "
                        "bridge: FEA and sensitivity time of the 100-span arch bridge vs DOF")
    p.add_argument("--el-per-span", default="2,6,10,20,30,80,1500,2500,4500,6500",
                   help="bridge workload: elements per span of the 100-span arch bridge")
    p.add_argument("--requests", type=int, default=512, help="serving: requests per run")
    p.add_argument("--rates", default="0.5,0.9",
                   help="serving: Poisson arrival rates as fractions of saturated throughput")
    p.add_argument("--hbm-budget-gb", type=float, default=64.0)
    p.add_argument("--max-systems", type=int, default=512)
    p.add_argument("--lanes", type=int, default=2,
                   help="serving: lanes of the server (stepped at once on their own threads)")
    p.add_argument("--alone-sample", type=int, default=16,
                   help="serving: requests timed one at a time on the FP64 path")
    p.add_argument("--repeats", type=int, default=1000, help="gridshell: timed evaluations")
    return p.parse_args()


def design_model(n_el, seed):
    return meshgen.shell(n_el=n_el, seed=seed)


def workload_name(a):
    """The workload both arms run (the same text on the oracle's line)."""
    n = a.n_el
    dof = 6 * (n + 1) ** 2
    return ("shell %dx%d quads (%d DOF), seeded designs (z bump, t ~ U[0.05, 0.2]), self-weight, "
            "corners pinned: solve + adjoint dC/dz, dC/dt at <=1e-6 rel err vs FP64"
            % (n, n, dof))


def solver_name(a):
    return ("%s %s CG%s to rtol %g, %d designs per batched step"
            % ("FP32" if a.precision == "fp32_ir" else "FP64", a.precond,
               " + FP64 refinement" if a.precision == "fp32_ir" else "", a.rtol, a.batch))


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


def host_cpu():
    """The host's CPU model and logical core count (the oracle's machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in ln:
                v = ln.split(":", 1)[1].strip()
                model = v if model is None else model + " " + v
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"cpu_model": model or platform.machine(), "nproc": os.cpu_count()}


def rel_errors(got, ref, keys=("u", "dz", "dt")):
    """Relative 2-norm errors of GPU results against the oracle's, and of C."""
    out = {}
    for k in keys:
        if k in got and k in ref and np.size(ref[k]):
            nr = np.linalg.norm(ref[k])
            out[k] = float(np.linalg.norm(np.asarray(got[k]) - ref[k]) / (nr if nr > 0 else 1.0))
    if "C" in got and "C" in ref:
        out["C"] = abs(float(got["C"]) - ref["C"]) / abs(ref["C"])
    return out


def max_errors(errs):
    """Per-quantity maximum over a list of rel_errors dicts."""
    keys = sorted({k for e in errs for k in e})
    return {k: max(e[k] for e in errs if k in e) for k in keys}


def oracle_gradients(meshes, w=1.0):
    """Oracle results of several models in threads (ctypes releases the GIL).
    Returns (results, seconds, threads)."""
    import concurrent.futures
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    n = max(1, min(len(meshes), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(n) as ex:
        res = list(ex.map(lambda m: oracle.gradient(m, w=w), meshes))
    return res, time.perf_counter() - t0, n


def rank_seeds(rank, world, batch):
    """Design seeds of one rank: ranks evaluate disjoint batches (weak scaling,
    no data-path collective)."""
    assert 0 <= rank < world
    return [rank * batch + i for i in range(batch)]


def slowest(seconds, world, dist=None, device=None):
    """The job's time: the maximum of every rank's time (one all-reduce)."""
    if world <= 1:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def assembly_bytes(mdl):
    """Algorithmic bytes of one model's assembly: its element blocks read once
    (in assembly order), cptr and the 2-byte support mask of every block, and
    K64 + K32 written."""
    nb = mdl.n_blocks
    return mdl.n_elem_blocks * 288 + (nb + 1) * 4 + nb * 2 + nb * (288 + 144)


def free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_replicas(cmd, n, stdout=None):
    """Runs `cmd` as n replica ranks on this node (rank r on GPU r), as
    torch.distributed.run would: RANK, LOCAL_RANK, WORLD_SIZE and a 127.0.0.1
    rendezvous in the environment.  Rank 0's stdout goes to `stdout` (default:
    this process's); the other ranks' stdout is discarded.  Returns the first
    non-zero exit code of any rank, else 0."""
    port = free_port()
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n),
                   LOCAL_WORLD_SIZE=str(n), GROUP_RANK="0", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        out = stdout if r == 0 else subprocess.DEVNULL
        procs.append(subprocess.Popen(cmd, env=env, stdout=out))
    codes = [p.wait() for p in procs]
    return next((c for c in codes if c != 0), 0)


def job_rate(world, batch, steps, seconds):
    """Whole-job throughput: the designs of all ranks over the slowest rank's time."""
    return world * batch * steps / seconds


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
                errs.append(rel_errors(gpu_results[i], ref))
    return n_designs / dt, dt, errs, refs


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
        "config": {"workload": workload_name(a),
                   "solver": "oracle: FP64 band Cholesky + dual-number adjoint (Eq. 6), "
                             "single thread, 1 design per step",
                   "host": host_cpu()},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": "%d designs of the workload (seeds 0..%d), one per step"
                                   % (a.steps, a.steps - 1), **host_cpu()},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Other workloads (one GPU each; one JSON line each)


def _pct(x, q):
    return float(np.percentile(np.asarray(x, float), q)) if len(x) else None


def _gpu_setup():
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import paper_2407_20026_gb300 as sso
    from paper_2407_20026_gb300 import _build
    _build.build()
    return torch, sso, local


def _mesh_bytes(m):
    n = m["xyz"].shape[0]
    nb = len(m["beam_conn"])
    nq = len(m["quad_conn"])
    return n * (3 * 8 + 6 + 6 * 8) + nb * (2 * 4 + 6 * 8) + nq * (4 * 4 + 5 * 8)


def stream_window(t_arrive, latency_ms):
    """Throughput of a request stream away from its ramp and drain: requests
    completed per second (and arrived per second) between the 10th and the
    90th percentile of the arrival times, the requests still queued or running
    at the last arrival, and how long after it the last one completed.
    t_arrive: sorted arrival times (s); latency_ms: per request, from arrival."""
    t = np.asarray(t_arrive, dtype=np.float64)
    done = np.sort(t + 1e-3 * np.asarray(latency_ms, dtype=np.float64))
    t1, t2 = float(t[len(t) // 10]), float(t[(9 * len(t)) // 10])
    span = max(t2 - t1, 1e-12)
    return {"achieved_steady_per_s": float(np.count_nonzero((done >= t1) & (done < t2))) / span,
            "offered_steady_per_s": float(np.count_nonzero((t >= t1) & (t < t2))) / span,
            "backlog_at_last_arrival": int(np.count_nonzero(done > t[-1])),
            "drain_s": float(done[-1] - t[-1])}


def run_serving(a):
    """Serving stream: grid-shell requests of n x n nodes, n ~ U{8..100}
    (seeded), plan and load as the 10 x 10 grid-shell; each request is solved
    and its adjoint dC/dz computed by the continuous-batching server.  Runs
    the stream saturated (every request queued at t = 0: throughput) and as
    Poisson arrivals at fractions of that throughput (latency from arrival),
    then times a sample of the same requests one at a time on the FP64
    single-model path."""
    torch, sso, local = _gpu_setup()
    from paper_2407_20026_gb300.serve import Server, run_stream
    spec = meshgen.serving_stream(a.requests, seed=0)
    meshes = [meshgen.gridshell(n_side=r["side"], seed=r["seed"]) for r in spec]
    dofs = [6 * m["xyz"].shape[0] for m in meshes]
    opts = sso.options(precision=a.precision, precond=a.precond, rtol=a.rtol,
                       inner_rtol=a.inner_rtol, iters_per_launch=a.iters_per_launch)
    srv = Server(opts, hbm_budget=int(a.hbm_budget_gb * (1 << 30)), max_systems=a.max_systems,
                 lanes=a.lanes)
    warm = [{"mesh": meshgen.gridshell(n_side=8 + 4 * k, seed=10 ** 6 + k), "t_arrive": 0.0}
            for k in range(max(a.warmup, 1))]
    run_stream(srv, warm)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    l0 = sso.kernel_launches()
    info0 = srv.info()
    res, elapsed = run_stream(srv, [{"mesh": m, "t_arrive": 0.0} for m in meshes],
                              time_limit_s=1800.0)
    info1 = srv.info()
    phases = {k: info1[k] - info0[k] for k in info1}
    launches = sso.kernel_launches() - l0
    clk = clocks.stop()
    failed = [i for i, r in enumerate(res) if r["stats"]["status"] != 0]
    sat = len(meshes) / elapsed
    accuracy = None
    if not a.no_cpu_baseline:
        # a seeded sample of 8 requests (sizes across the stream) against the oracle
        pick = sorted(np.random.default_rng(7).choice(len(meshes), min(8, len(meshes)),
                                                      replace=False).tolist())
        refs, o_s, o_threads = oracle_gradients([meshes[i] for i in pick])
        errs = [rel_errors(res[i], ref, keys=("u", "dz")) for i, ref in zip(pick, refs)]
        accuracy = {"requests": pick, "dof": [dofs[i] for i in pick], **max_errors(errs),
                    "oracle_seconds": o_s, "oracle_threads": o_threads}
    iters = [r["stats"]["iterations"] for r in res]
    lat_sat = [r["latency_ms"] for r in res]

    poisson = []
    for frac in [float(x) for x in a.rates.split(",") if x]:
        rate = frac * sat
        rng = np.random.default_rng(12345)
        gaps = rng.exponential(1.0 / rate, len(meshes))
        t = np.cumsum(gaps) - gaps[0]
        pinfo0 = srv.info()
        res2, el2 = run_stream(srv, [{"mesh": m, "t_arrive": float(tt)}
                                     for m, tt in zip(meshes, t)], time_limit_s=1800.0)
        pinfo1 = srv.info()
        lat = [r["latency_arrival_ms"] for r in res2]
        poisson.append({"rate_frac": frac, "offered_per_s": rate,
                        "achieved_per_s": len(meshes) / el2,
                        **stream_window(t, lat),
                        "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                        "failed": sum(r["stats"]["status"] != 0 for r in res2),
                        "server_host_phases": {k: pinfo1[k] - pinfo0[k] for k in pinfo1}})
    srv.close()

    # the plain path: one request at a time, FP64 CG, same rtol
    # (the two-level preconditioner is FP32-only: the plain path then uses block-Jacobi)
    o64 = sso.options(precision="fp64",
                      precond="block_jacobi" if a.precond == "two_level" else a.precond,
                      rtol=a.rtol, iters_per_launch=a.iters_per_launch)
    idx = list(range(min(a.alone_sample, len(meshes))))
    w = sso.Model(warm[0]["mesh"])
    w.solve(o64)
    w.gradient()
    w.result()
    w.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in idx:
        mdl = sso.Model(meshes[i])
        mdl.solve(o64)
        mdl.gradient()
        mdl.result()
        mdl.close()
    alone_s = time.perf_counter() - t0
    alone = len(idx) / alone_s

    line = {
        "metric": METRIC, "value": sat, "unit": "evals/s", "n_gpus": 1,
        "steps": len(meshes), "warmup": len(warm), "ms_per_step": 1000.0 / sat,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if a.precision == "fp32_ir" else "f64", "data": "synthetic",
        "config": {"workload": "serving stream: %d grid-shell requests, n x n nodes with n ~ "
                               "U{8..100} (seeded), 10 m plan, -1 kN per free node, solve + "
                               "adjoint dC/dz, %s %s CG to rtol %g; continuous batching"
                               % (len(meshes), "FP32+FP64 refinement" if a.precision ==
                                  "fp32_ir" else "FP64", a.precond, a.rtol),
                   "mean_dof": float(np.mean(dofs)), "max_dof": int(max(dofs)),
                   "hbm_budget_gb": a.hbm_budget_gb, "max_systems": a.max_systems,
                   "lanes": a.lanes,
                   "iters_per_launch": a.iters_per_launch,
                   "l2": "working set of the resident requests (GBs) > L2"},
        "saturated": {"evals_per_s": sat, "seconds": elapsed,
                      "latency_p50_ms": _pct(lat_sat, 50), "latency_p99_ms": _pct(lat_sat, 99),
                      "cg_iterations_mean": float(np.mean(iters)),
                      "cg_iterations_max": int(max(iters)), "failed": len(failed),
                      "pcg_dof_per_s": float(np.dot(iters, dofs)) / elapsed,
                      "server_host_phases": phases},
        "poisson": poisson,
        "accuracy_vs_oracle": accuracy,
        "one_at_a_time_fp64": {"evals_per_s": alone, "requests": len(idx),
                               "precond": "block_jacobi" if a.precond == "two_level"
                               else a.precond,
                               "mean_dof": float(np.mean([dofs[i] for i in idx])),
                               "speedup_of_serving": sat / alone},
        "roofline": None,
        "cpu_baseline": None,
        "clocks": clk, "gpu_launches": int(launches),
        "e2e": {"value": sat, "unit": "evals/s",
                "h2d_bytes_per_step": int(np.mean([_mesh_bytes(m) for m in meshes])),
                "d2h_bytes_per_step": int(np.mean([8 * (d + d // 6 + 1) for d in dofs])),
                "note": "the server takes meshes from host memory and returns results to host "
                        "memory, so value is already end to end"},
    }
    print(json.dumps(line), flush=True)


def run_gridshell(a):
    """Latency of one evaluation of the 10 x 10 grid-shell (261 beams, 600
    DOF) to the FP64 tolerance: set design, solve, adjoint dC/dz, results to
    host.  The value uses the one-CTA double-float CG (precision f32x2: the
    whole solve in one launch); the batched engine's FP64 CG on the same
    evaluation is timed beside it."""
    torch, sso, local = _gpu_setup()
    m = meshgen.gridshell(n_side=10, seed=0)
    z = np.ascontiguousarray(m["xyz"][:, 2])

    def evaluate(mdl, opts):
        mdl.set_design(z)
        st = mdl.solve(opts)
        mdl.gradient()
        return st, mdl.result()

    def timed(precision, repeats):
        mdl = sso.Model(m)
        opts = sso.options(precision=precision, precond=a.precond, rtol=1e-10,
                           iters_per_launch=a.iters_per_launch)
        for _ in range(max(a.warmup, 3)):
            evaluate(mdl, opts)
        torch.cuda.synchronize()
        lat = []
        l0 = sso.kernel_launches()
        t_all = time.perf_counter()
        for _ in range(repeats):
            t0 = time.perf_counter()
            st, r = evaluate(mdl, opts)
            lat.append(1e6 * (time.perf_counter() - t0))
        total = time.perf_counter() - t_all
        return st, r, lat, total, sso.kernel_launches() - l0

    clocks = ClockSampler(local)
    clocks.start()
    st, r, lat, total, launches = timed("f32x2", a.repeats)
    clk = clocks.stop()
    st64, r64, lat64, total64, launches64 = timed("fp64", max(20, a.repeats // 10))
    cpu = None
    err = err64 = None
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 5.0 or k < 3:
            ref = oracle.gradient(m)
            k += 1
        dt = time.perf_counter() - t0
        err = rel_errors(r, ref, keys=("u", "dz"))
        err64 = rel_errors(r64, ref, keys=("u", "dz"))
        cpu = {"value": k / dt, "unit": "evals/s", "cores": 1, "kind": "oracle",
               "sample": "%d evaluations of the same design, %.1f s" % (k, dt), **host_cpu()}
    line = {
        "metric": METRIC, "value": a.repeats / total, "unit": "evals/s", "n_gpus": 1,
        "steps": a.repeats, "warmup": max(a.warmup, 3), "ms_per_step": 1000 * total / a.repeats,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32x2",
        "data": "synthetic",
        "config": {"workload": "grid-shell 10x10 nodes, 261 beams, 600 DOF, one evaluation at a "
                               "time: set z, solve to rtol 1e-10, adjoint dC/dz, results to host",
                   "solver": "double-float %s CG, one CTA, one launch (f32x2)" % a.precond,
                   "l2": "problem fits L2 (latency workload)"},
        "latency_us": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "min": float(min(lat))},
        "cg_iterations": st["iterations"], "rel_residual": st["rel_residual"],
        "accuracy_vs_oracle": err,
        "fp64_cg": {"evals_per_s": len(lat64) / total64,
                    "latency_us": {"p50": _pct(lat64, 50), "p99": _pct(lat64, 99)},
                    "cg_iterations": st64["iterations"], "accuracy_vs_oracle": err64,
                    "launches_per_eval": launches64 / len(lat64)},
        "roofline": None, "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": int(launches), "launches_per_eval": launches / a.repeats,
        "e2e": {"value": a.repeats / total, "unit": "evals/s",
                "h2d_bytes_per_step": 8 * len(z), "d2h_bytes_per_step": 8 * (7 * len(z) + 1),
                "note": "every evaluation uploads z from host and reads u, C, dz back"},
    }
    print(json.dumps(line), flush=True)


def run_bridge(a):
    """The beam-path scaling structure: a 100-span bridge of 30 m x 10 m
    parabolic arches (Sec. 2.2.4), el_per_span elements per span (1,206 DOF at
    2 up to 3,900,006 DOF at 6,500).  For each size: FEA (set design, solve,
    C) and sensitivity analysis (FEA + adjoint dC/dz of every node), medians
    of 3 runs after a warm-up, with the direct block-tridiagonal solver
    (SSO_CHAIN, FP64) and, up to 60 k DOF, FP64 block-Jacobi CG to a relative
    residual of 1e-10.  The oracle's band Cholesky (1 thread) is timed at every
    size (its sensitivity analysis up to 60 k DOF) as the CPU baseline, and its
    residual shows the FP64 floor of each size: with 30 m spans cut into
    elements of a few mm, cond(K) nears 1/eps and no FP64 solve reaches a
    1e-10 residual (status 4 then reports the solve above rtol)."""
    torch, sso, local = _gpu_setup()
    sizes = [int(k) for k in a.el_per_span.split(",") if k]
    chain = sso.options(precision="fp64", precond="chain", rtol=1e-10, max_sweeps=3)
    cg = sso.options(precision="fp64", precond="block_jacobi", rtol=1e-10,
                     iters_per_launch=64, max_iter=4_000_000)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sso.kernel_launches()
    rows = []

    def timed(mdl, z, opts):
        mdl.set_design(z)
        mdl.solve(opts, raise_on_error=False)
        mdl.gradient()
        mdl.result()
        fea, sens = [], []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mdl.set_design(z)
            st = mdl.solve(opts, raise_on_error=False)
            C = mdl.result()["C"]
            fea.append(1000 * (time.perf_counter() - t0))
            t0 = time.perf_counter()
            mdl.set_design(z)
            mdl.solve(opts, raise_on_error=False)
            mdl.gradient()
            r = mdl.result()
            sens.append(1000 * (time.perf_counter() - t0))
        return st, r, float(np.median(fea)), float(np.median(sens))

    for k in sizes:
        m = meshgen.arch_bridge(el_per_span=k)
        z = np.ascontiguousarray(m["xyz"][:, 2])
        mdl = sso.Model(m)
        st, r, fea, sens = timed(mdl, z, chain)
        row = {"el_per_span": k, "dof": 6 * m["xyz"].shape[0],
               "direct": {"fea_ms": fea, "sensitivity_ms": sens,
                          "rel_residual": st["rel_residual"], "refinements": st["sweeps"],
                          "status": st["status"]},
               "C": float(r["C"])}
        if not a.no_cpu_baseline:
            # the oracle's FP64 band Cholesky: time and residual floor at every size
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            u_o, C_o = oracle.solve(m)
            row["oracle_fea_ms"] = 1000 * (time.perf_counter() - t0)
            f_o = oracle.load_vector(m)
            f_o[m["fixed"].ravel().astype(bool)] = 0.0
            row["oracle_rel_residual"] = float(np.linalg.norm(oracle.residual(m, u_o)) /
                                               np.linalg.norm(f_o))
            row["direct_rel_diff_C_vs_oracle"] = abs(row["C"] - C_o) / abs(C_o)
        if row["dof"] <= 60_000:
            st2, r2, fea2, sens2 = timed(mdl, z, cg)
            row["cg"] = {"fea_ms": fea2, "sensitivity_ms": sens2, "iterations": st2["iterations"],
                         "rel_residual": st2["rel_residual"],
                         "rel_diff_u_vs_direct": float(np.linalg.norm(r2["u"] - r["u"]) /
                                                       np.linalg.norm(r["u"]))}
            if not a.no_cpu_baseline:
                import oracle
                oracle.build()
                t0 = time.perf_counter()
                ref = oracle.gradient(m)
                row["oracle_sensitivity_ms"] = 1000 * (time.perf_counter() - t0)
                row["direct_rel_err_vs_oracle"] = {
                    "u": float(np.linalg.norm(r["u"] - ref["u"]) / np.linalg.norm(ref["u"])),
                    "dz": float(np.linalg.norm(r["dz"] - ref["dz"]) / np.linalg.norm(ref["dz"]))}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        del mdl
    launches = sso.kernel_launches() - l0
    clk = clocks.stop()
    big = rows[-1]
    line = {
        "metric": "sensitivity analyses/s of the 100-span arch bridge (FEA + adjoint dC/dz)",
        "value": 1000.0 / big["direct"]["sensitivity_ms"], "unit": "evals/s", "n_gpus": 1,
        "steps": 3 * len(rows), "warmup": 1, "ms_per_step": big["direct"]["sensitivity_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "100-span arch bridge, %s elements per span; direct "
                               "block-tridiagonal solve (FP64); value at the largest size"
                               % a.el_per_span},
        "sizes": rows, "roofline": None, "clocks": clk, "gpu_launches": int(launches),
        "e2e": {"value": 1000.0 / big["direct"]["sensitivity_ms"], "unit": "evals/s",
                "h2d_bytes_per_step": 8 * big["dof"] // 6,
                "d2h_bytes_per_step": 8 * (big["dof"] + big["dof"] // 6 + 1),
                "note": "every run uploads z from host and reads u, C, dz back"},
    }
    print(json.dumps(line), flush=True)


def run_large(a):
    """One large shell: 512 x 512 quads (263,169 nodes, 1,579,014 DOF), all
    edges clamped, 5 kPa pressure; FP32 Jacobi CG with FP64 refinement to a
    relative residual of 1e-8, then the adjoint dC/dz, dC/dt."""
    torch, sso, local = _gpu_setup()
    n_el = a.n_el if a.n_el != 64 else 512
    m = meshgen.shell(n_el=n_el, supports="clamped", load="pressure")
    mdl = sso.Model(m)
    batch = sso.Batch([mdl])
    opts = sso.options(precision=a.precision, precond=a.precond, rtol=1e-8,
                       inner_rtol=a.inner_rtol, iters_per_launch=a.iters_per_launch)
    warm = sso.options(precision=a.precision, precond=a.precond, rtol=1e-8,
                       inner_rtol=a.inner_rtol, iters_per_launch=a.iters_per_launch,
                       max_iter=4 * a.iters_per_launch)
    batch.solve(warm, raise_on_error=False)
    torch.cuda.synchronize()
    peak_gbs, peak_kind = measured_peaks()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sso.kernel_launches()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    stream = torch.cuda.current_stream()
    ev[0].record(stream)
    stats = batch.solve(opts)
    ev[1].record(stream)
    batch.gradient()
    ev[2].record(stream)
    ev[2].synchronize()
    launches = sso.kernel_launches() - l0
    clk = clocks.stop()
    # kernel and phase durations: the same solve again, untimed, with events
    # around every kernel (they serialise the kernels)
    batch.set_profiling(True)
    batch.solve(opts)
    batch.gradient()
    torch.cuda.synchronize()
    ms_a, ms_b, pairs = batch.kernel_times()
    su = batch.setup_times()
    batch.set_profiling(False)
    solve_ms = ev[0].elapsed_time(ev[1])
    grad_ms = ev[1].elapsed_time(ev[2])
    s0 = stats[0]
    n = mdl.n_nodes
    nb = mdl.n_blocks
    n_free = 6 * n - int(m["fixed"].sum())
    fp32 = a.precision == "fp32_ir"
    wsz = 4 if fp32 else 8
    bytes_pcg = nb * (36 * wsz + 4) + (n + 1) * 4 + 4 * (6 * n * wsz)
    bytes_resid = nb * (36 * 8 + 4) + (n + 1) * 4 + 3 * (6 * n * 8)
    alg = s0["iterations"] * bytes_pcg + s0["sweeps"] * bytes_resid
    ach = alg / (ms_a / 1e3) / 1e9 if ms_a > 0 else None
    accuracy = None
    if not a.no_cpu_baseline:
        # the oracle's element-by-element K applied to the GPU's u (FP64, host)
        import oracle
        oracle.build()
        res_u = mdl.result()
        fx = m["fixed"].ravel().astype(bool)
        f_o = oracle.load_vector(m)
        f_o[fx] = 0.0
        r_o = oracle.residual(m, res_u["u"])
        r_o[fx] = 0.0
        accuracy = {"oracle_rel_residual_of_gpu_u": float(np.linalg.norm(r_o) /
                                                          np.linalg.norm(f_o)),
                    "C_vs_oracle_f_dot_u_rel": abs(res_u["C"] - float(f_o @ res_u["u"])) /
                    abs(res_u["C"]),
                    "note": "no direct oracle solve at this size; the oracle's K bounds the "
                            "GPU solution's residual"}
    asm_bytes = assembly_bytes(mdl)
    asm_gbs = asm_bytes / (su["assembly"] / 1e3) / 1e9 if su["assembly"] > 0 else None
    line = {
        "metric": METRIC, "value": 1000.0 / (solve_ms + grad_ms), "unit": "evals/s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": solve_ms + grad_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
        "config": {"workload": "large shell %dx%d quads (%d DOF, %d free), clamped edges, 5 kPa, "
                               "%s %s CG to rtol 1e-8, solve + adjoint dC/dz, dC/dt"
                               % (n_el, n_el, 6 * n, n_free, "FP32+FP64 refinement" if fp32
                                  else "FP64", a.precond),
                   "l2": "K alone (%.0f MB FP32) exceeds L2" % (nb * 144 / 1e6)},
        "solve_ms": solve_ms, "gradient_ms": grad_ms, "cg_iterations": s0["iterations"],
        "refinement_sweeps": s0["sweeps"], "rel_residual": s0["rel_residual"],
        "pcg_dof_per_s": n_free * s0["iterations"] / (solve_ms / 1e3),
        "roofline": {"bound": "hbm", "kernel": "pcg_a (BSR SpMV)", "achieved": ach,
                     "peak": peak_gbs, "unit": "GB/s",
                     "frac": ach / peak_gbs if ach else None, "peak_kind": peak_kind,
                     "traffic": None, "alg_bytes_per_cg_launch": bytes_pcg,
                     "launches_timed": pairs, "kernel_ms_total": ms_a, "kernel_b_ms_total": ms_b},
        "assembly": {"ms": su["assembly"], "alg_bytes": asm_bytes, "achieved_gbs": asm_gbs,
                     "frac": asm_gbs / peak_gbs if asm_gbs else None},
        "elements_ms": su["elements"], "precond_loads_ms": su["precond"],
        "adjoint_contraction_ms": su["adjoint"], "accuracy_vs_oracle": accuracy,
        "cpu_baseline": None, "clocks": clk, "gpu_launches": int(launches),
        "e2e": None,
    }
    print(json.dumps(line), flush=True)


def run_training(a):
    """Physics-in-the-loop training: a 3-layer MLP (16 -> 128 -> 128 -> n_nodes,
    FP32) maps 64 seeded latent vectors to nodal z offsets (0.25 tanh, in m) of
    48 x 48-element shells (t = 0.1 m, corners pinned, self-weight) around the
    bump of the 64 x 64 shell workload; each step solves the 64
    shells in one batch, takes the adjoint through the autograd function and
    backpropagates loss = mean(C + 0.1 V) into the MLP (Adam).  Solves start
    from the previous step's displacements (warm start)."""
    torch, sso, local = _gpu_setup()
    from paper_2407_20026_gb300.autograd import BatchSSOFunction
    dev = torch.device("cuda", local)
    B, n_el = 64, 48
    base = meshgen.shell(n_el=n_el, seed=0, thickness=0.1)
    n = base["xyz"].shape[0]
    nq = base["quad_conn"].shape[0]
    batch = sso.Batch([sso.Model(base) for _ in range(B)])
    gen = torch.Generator().manual_seed(0)
    torch.manual_seed(0)
    mlp = torch.nn.Sequential(torch.nn.Linear(16, 128), torch.nn.ReLU(),
                              torch.nn.Linear(128, 128), torch.nn.ReLU(),
                              torch.nn.Linear(128, n)).to(dev)
    latents = torch.randn(B, 16, generator=gen).to(dev)
    optim = torch.optim.Adam(mlp.parameters(), lr=1e-3)
    z0 = torch.tensor(base["xyz"][:, 2], device=dev).expand(B, n)
    t = torch.full((B, nq), 0.1, dtype=torch.float64, device=dev)
    opts = sso.options(precision=a.precision, precond=a.precond, rtol=a.rtol,
                       inner_rtol=a.inner_rtol, iters_per_launch=a.iters_per_launch,
                       warm_start=1)

    def step():
        z = z0 + 0.25 * torch.tanh(mlp(latents)).double()
        u, C, V = BatchSSOFunction.apply(batch, z, t, opts)
        loss = (C + 0.1 * V).mean()
        optim.zero_grad()
        loss.backward()
        optim.step()
        return float(loss.detach())

    losses = [step() for _ in range(max(a.warmup, 3))]
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sso.kernel_launches()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        losses.append(step())
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    launches = sso.kernel_launches() - l0
    clk = clocks.stop()
    accuracy = None
    if not a.no_cpu_baseline:
        # the current MLP's designs: C and d(C + 0.1 V)/dz, dt of 4 of them vs the oracle
        zc = (z0 + 0.25 * torch.tanh(mlp(latents)).double()).detach().requires_grad_(True)
        tc = t.clone().requires_grad_(True)
        u, C, V = BatchSSOFunction.apply(batch, zc, tc, opts)
        (C + 0.1 * V).sum().backward()
        import oracle
        oracle.build()
        pick = [0, 21, 42, 63]
        models = []
        for i in pick:
            mi = dict(base)
            xyz = np.array(base["xyz"], copy=True)
            xyz[:, 2] = zc[i].detach().cpu().numpy()
            mi["xyz"] = xyz
            models.append(mi)
        refs, o_s, _ = oracle_gradients(models)
        errs = []
        for k, i in enumerate(pick):
            vol = oracle.volume(models[k])
            ref = {"C": refs[k]["C"], "dz": refs[k]["dz"] + 0.1 * vol["dz"],
                   "dt": refs[k]["dt"] + 0.1 * vol["dt"]}
            got = {"C": float(C[i].detach()), "dz": zc.grad[i].cpu().numpy(),
                   "dt": tc.grad[i].cpu().numpy()}
            errs.append(rel_errors(got, ref, keys=("dz", "dt")))
        accuracy = {"designs": pick, **max_errors(errs), "oracle_seconds": o_s,
                    "note": "gradients of C + 0.1 V after the timed steps"}
    line = {
        "metric": "training steps/sec (64 shell solves + adjoint per step)",
        "value": a.steps / el, "unit": "steps/s", "n_gpus": 1, "steps": a.steps,
        "warmup": max(a.warmup, 3), "ms_per_step": 1000 * el / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if a.precision == "fp32_ir" else "f64", "data": "synthetic",
        "config": {"workload": "training: MLP 16-128-128-%d (FP32), %d latents, %dx%d-element "
                               "shells (%d DOF), t = 0.1, loss = mean(C + 0.1 V), Adam 1e-3, "
                               "%s CG to rtol %g, warm start" % (n, B, n_el, n_el, 6 * n,
                                                                 a.precond, a.rtol),
                   "l2": "64 x K (%.0f MB) > L2" % (B * batch.models[0].n_blocks * 144 / 1e6)},
        "design_evals_per_s": B * a.steps / el,
        "loss_first": losses[0], "loss_last": losses[-1], "accuracy_vs_oracle": accuracy,
        "roofline": None, "cpu_baseline": None, "clocks": clk, "gpu_launches": int(launches),
        "e2e": None,
    }
    print(json.dumps(line), flush=True)


def run_workload(a):
    {"serving": run_serving, "gridshell": run_gridshell, "large": run_large,
     "training": run_training, "bridge": run_bridge}[a.workload](a)


def main():
    a = parse()
    if a.impl == "ours" and a.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one replica rank per GPU (the path shards by design; no data-path collective)
        sys.exit(launch_replicas([sys.executable, os.path.abspath(__file__), *sys.argv[1:]],
                                 a.gpus))
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload != "shell":
        run_workload(a)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        # the only collective is the max of the ranks' times
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2407_20026_gb300 as sso
    from paper_2407_20026_gb300 import _build
    _build.build()

    B = a.batch
    seeds = rank_seeds(rank, world, B)
    meshes = [design_model(a.n_el, s) for s in seeds]
    models = [sso.Model(m) for m in meshes]
    batch = sso.Batch(models)
    if a.parts > 0:
        batch.set_parts(a.parts)
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
    launches = sso.kernel_launches() - launches0
    clk = clocks.stop()
    barrier()
    # kernel durations: one more step, untimed, with CUDA events around every
    # CG kernel on the library's stream (the events serialise the kernels, so
    # they are kept out of the timed steps)
    batch.set_profiling(True)
    flush.fill_(-1.0)
    pstats = step_device()
    torch.cuda.synchronize()
    ms_a, ms_b, timed_pairs = batch.kernel_times()
    setup = batch.setup_times()
    batch.set_profiling(False)
    p_iters = sum(s["iterations"] for s in pstats)
    p_sweeps = sum(s["sweeps"] for s in pstats)
    total_ms = slowest(float(sum(step_ms)), world, dist, dev)
    value = job_rate(world, B, a.steps, total_ms / 1000.0)

    # algorithmic bytes of kernel A over the timed region
    n_nodes = models[0].n_nodes
    nblk = models[0].n_blocks
    fp32 = a.precision == "fp32_ir"
    wsz = 4 if fp32 else 8
    bytes_pcg = nblk * (36 * wsz + 4) + (n_nodes + 1) * 4 + 4 * (6 * n_nodes * wsz)
    bytes_resid = nblk * (36 * 8 + 4) + (n_nodes + 1) * 4 + 3 * (6 * n_nodes * 8)
    alg_bytes = p_iters * bytes_pcg + p_sweeps * bytes_resid
    step_bytes = (iters_total * (bytes_pcg + 264 * n_nodes) + sweeps_total * bytes_resid)
    step_gbs = step_bytes / (total_ms / 1000.0) / 1e9  # this GPU
    achieved = alg_bytes / (ms_a / 1000.0) / 1e9 if ms_a > 0 else None
    a_launches = timed_pairs
    traffic = kernel_traffic("pcg.cu", "pcg_a_%s" % ("f32" if fp32 else "f64"))
    traffic_bytes = traffic["dram_bytes_per_design_launch"] * B if traffic else None

    # kernel B over the same profiled step: 264 B per node per CG iteration
    # (packed M^-1 96, p and q 24 each, r and dx read and written 48 each, z 24)
    b_bytes = p_iters * 264 * n_nodes
    b_gbs = b_bytes / (ms_b / 1000.0) / 1e9 if ms_b > 0 else None
    roofline_b = {"bound": "hbm", "kernel": "pcg_b32 (update, z = M^-1 r, dots)",
                  "achieved": b_gbs, "peak": peak_gbs, "unit": "GB/s",
                  "frac": b_gbs / peak_gbs if b_gbs else None, "peak_kind": peak_kind,
                  "alg_bytes": b_bytes, "kernel_ms_total": ms_b} if fp32 else None

    # assembly: one launch for the whole batch, timed with events on the
    # library's stream in the profiled step
    asm_bytes = sum(assembly_bytes(m) for m in models)
    asm_ms = setup["assembly"]
    asm_gbs = asm_bytes / (asm_ms / 1e3) / 1e9 if asm_ms > 0 else None
    asm_traffic = kernel_traffic("assembly.cu", "assemble_bulk")
    roofline_assembly = {
        "bound": "hbm", "kernel": "assemble_bulk (one launch, %d designs)" % B,
        "achieved": asm_gbs, "peak": peak_gbs, "unit": "GB/s",
        "frac": asm_gbs / peak_gbs if asm_gbs else None, "peak_kind": peak_kind,
        "alg_bytes_per_launch": asm_bytes, "ms": asm_ms,
        "traffic": asm_traffic["dram_bytes_per_design"] * B if asm_traffic else None}

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
        e2e_s = slowest(time.perf_counter() - t0, world, dist, dev)
        h2d = B * (n_nodes + nq) * 8
        d2h = B * (6 * n_nodes + n_nodes + nq + 1) * 8
        e2e = {"value": job_rate(world, B, a.steps, e2e_s), "unit": "evals/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # results of the graded path for the oracle comparison (before any other solve)
    n_cmp = min(a.cpu_sample, B)
    gres = {i: models[i].result() for i in range(n_cmp)} if rank == 0 else {}

    # the two-level preconditioner on the same designs (not the graded value)
    two_level = None
    if a.precond == "block_jacobi" and a.precision == "fp32_ir" and not a.no_two_level:
        o2 = sso.options(precision=a.precision, precond="two_level", rtol=a.rtol,
                         inner_rtol=a.inner_rtol, iters_per_launch=a.iters_per_launch)

        def step_two_level():
            for i, mdl in enumerate(models):
                mdl.set_design(z_dev[i], t_dev[i])
            st = batch.solve(o2)
            batch.gradient()
            return st

        step_two_level()
        torch.cuda.synchronize()
        k2 = max(1, min(a.steps, 3))
        tl_ms, tl_iters = [], 0
        for k in range(k2):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st2 = step_two_level()
            e1.record(stream)
            e1.synchronize()
            tl_ms.append(e0.elapsed_time(e1))
            if any(s["status"] != 0 for s in st2):
                raise RuntimeError("two-level solve failed")
            tl_iters += sum(s["iterations"] for s in st2)
        tl_total = slowest(float(sum(tl_ms)), world, dist, dev)
        two_level = {"value": job_rate(world, B, k2, tl_total / 1000.0), "unit": "evals/s",
                     "steps": k2, "ms_per_step": tl_total / k2,
                     "cg_iterations_per_design": tl_iters / (B * k2),
                     "precond": "block-Jacobi + rigid-body coarse space of node aggregates"}
        if rank == 0:
            gres_tl = {i: models[i].result() for i in range(n_cmp)}

    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, secs, errs, refs = cpu_oracle_sample(a, n_cmp, gres)
        cpu = {"value": v, "unit": "evals/s", "cores": 1, "kind": "oracle",
               "sample": "%d designs of the workload (seeds 0..%d), %.1f s" %
                         (n_cmp, n_cmp - 1, secs), **host_cpu()}
        if errs:
            accuracy = max_errors(errs)
            accuracy["designs"] = n_cmp
        if two_level is not None:
            errs2 = [rel_errors(gres_tl[i], refs[i]) for i in range(n_cmp)]
            two_level["accuracy_vs_oracle"] = max_errors(errs2)

    if rank == 0:
        lat = np.array(step_ms)
        n_free = 6 * n_nodes - int(meshes[0]["fixed"].sum())
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "solver": solver_name(a),
                       "designs_per_step": B,
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
                "kernel_times_from": "profiled step: events around every CG launch, the "
                                     "batch run whole (the timed steps run it as two "
                                     "concurrent halves)" if B >= 32 else "profiled step",
                # the timed steps as a whole: the algorithmic bytes of both CG
                # kernels over the steps' elapsed time (everything else counted
                # as time), against the same peak
                "step_hbm": {
                    "achieved": step_gbs, "frac": step_gbs / peak_gbs,
                    "bytes": step_bytes, "note": "kernel A (SpMV, FP64 residual passes) and "
                                                 "kernel B (264 B per node) per CG iteration"},
            },
            # elapsed per phase of the profiled step; each set-up stage is
            # one launch for the whole batch
            "phase_ms_per_step": {"setup": setup["setup_wall"],
                                  "cg_kernel_a": ms_a, "cg_kernel_b_and_coarse": ms_b,
                                  "adjoint_contraction": setup["adjoint"],
                                  "setup_stages": {
                                      "element_matrices": setup["elements"],
                                      "assembly": setup["assembly"],
                                      "preconditioner_and_loads": setup["precond"]}},
            "roofline_b": roofline_b, "roofline_assembly": roofline_assembly,
            "cpu_baseline": cpu, "accuracy_vs_oracle": accuracy, "two_level": two_level,
            "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
