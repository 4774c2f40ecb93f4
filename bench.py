"""Benchmark of the RLB-MIE-FD Allen-Cahn stepper on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

One bench "step" is one pass of the hot path over the headline workload: the 3D
512^3 homogeneous-Neumann grid (h = 1/512, eps = 0.01, phi0 ~ U[-1, 1] from seed
1, FP32 state), set to phi0 and advanced 200 time steps with the discrete energy
E_h and the maximum norm computed every 50 steps (FP64 reductions).  Inputs are
resident in HBM when the timed region starts; each state buffer is 512 MiB, larger
than the 129 MB L2, so no L2 flush is needed between iterations.

value     lattice updates per second over all ranks (GLUPS), device-timed with CUDA
          events around K bench steps (barrier + synchronize on both sides, max over
          ranks).  With N > 1 every rank runs its own replica (the single problem is
          not sharded: weak scaling).
e2e       the same metric through the C ABI with host buffers: every step is one job
          that copies phi0 from pinned host memory, runs, and copies the state and the
          reductions back.  Reported: the pipelined runner (acs_pipe_submit / wait),
          whose copies overlap the neighbouring jobs' compute, timed over max(K, 10)
          jobs (`jobs`); serial_value: one context (acs_set_state_host, acs_run_logged,
          acs_get_state_host), K jobs (`serial_jobs`).
roofline  the step kernel's algorithmic bytes per launch (2 sizeof(T) per update, K
          fused steps per launch for temporal blocking) over its CUDA-event launch
          duration, against the measured HBM copy bandwidth.
cpu_baseline  the FP64 CPU oracle on the host cores, on a bounded sample of the
          same workload (rank 0, N = 1 only).

--impl reference times that oracle (the only other implementation of the method:
the paper ships no code) as the reference arm.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice-updates/s (GLUPS) and % of HBM roofline, FP32 & FP64; adjoint fwd+bwd time/step"
UNIT = "GLUPS"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running; the
    region starts once nvidia-smi has answered, and only samples taken inside it count."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.time() + 3.0
            while not self.lines and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if t < self.t0:
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_from_profile(kernel_tag: str):
    """Per-launch DRAM bytes of the step kernel from the committed ncu record, if the
    recorded digest of its sources still matches (else None: the kernel has changed)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if line.startswith("#") or len(parts) < 4 or parts[0] != kernel_tag:
                continue
            h = hashlib.sha256()
            for src in parts[1].split(","):
                fp = os.path.join(ROOT, "paper_2312_07010_gb300", "csrc", src)
                if not os.path.exists(fp):
                    return None
                h.update(open(fp, "rb").read())
            return float(parts[2]) if h.hexdigest()[:16] == parts[3] else None
    return None


def cpu_oracle_sample(budget_s: float = 12.0):
    """FP64 oracle on the 512^3 Neumann workload: as many whole time steps as fit the budget."""
    import numpy as np

    import oracle
    from workloads import cfg2
    w = cfg2("f64")
    phi = w.phi0()
    lam = oracle.lam(w.eps, w.dt, w.h)
    t0 = time.perf_counter()
    steps = 0
    while True:
        phi = oracle.step_fd(phi, w.eps, w.dt, w.h, w.bc)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 50:
            break
    del lam
    ups = w.numel * steps / el
    return {"value": ups / 1e9, "unit": UNIT, "cores": oracle.numthreads(), "kind": "oracle",
            "sample": f"{steps} time step(s) of the 512^3 Neumann workload, FP64 oracle "
                      f"(plain C, OpenMP over points), {el:.1f} s"}


def oracle_cpu_timing():
    """The FP64 oracle's FD step on the host cores, single-threaded and on all cores, for
    the 128^2 periodic (all 1000 steps), 4096^2 Dirichlet (2 steps) and 512^3 Neumann (1
    step) workloads: updates per second, with the CPU model and core count."""
    import oracle
    from workloads import cfg1, cfg2, cfg3
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    cores = oracle.numthreads()
    res = {"cpu_model": model, "nproc": os.cpu_count(), "threads_all": cores, "unit": "GLUPS"}
    for name, w, steps in (("cfg1_128sq_periodic_1000_steps", cfg1(), 1000),
                           ("cfg3_4096sq_dirichlet_2_steps", cfg3("f64"), 2),
                           ("cfg2_512cubed_neumann_1_step", cfg2("f64"), 1)):
        phi0 = w.phi0()
        row = {}
        for label, t in (("single_thread", 1), ("all_threads", cores)):
            oracle.set_threads(t)
            oracle.step_fd(phi0, w.eps, w.dt, w.h, w.bc)  # untimed: thread team and first touch
            p = phi0
            t0 = time.perf_counter()
            for _ in range(steps):  # one step per call, as the cpu_baseline sample
                p = oracle.step_fd(p, w.eps, w.dt, w.h, w.bc)
            row[label] = w.numel * steps / (time.perf_counter() - t0) / 1e9
        res[name] = row
    oracle.set_threads(cores)
    return res


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from workloads import cfg2
    w = cfg2("f64")
    phi0 = w.phi0()
    # each reference step: one time step of the workload on the whole 512^3 grid
    for _ in range(args.warmup):
        oracle.step_fd(phi0, w.eps, w.dt, w.h, w.bc)
    t0 = time.perf_counter()
    phi = phi0
    for _ in range(args.steps):
        phi = oracle.step_fd(phi, w.eps, w.dt, w.h, w.bc)
    el = time.perf_counter() - t0
    val = w.numel * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "cfg2_3d_neumann_512", "dims": 3, "n": 512, "bc": "neumann",
                   "eps": w.eps, "dt": w.dt, "h": w.h,
                   "sample": "one time step of the 512^3 grid per bench step (oracle)"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.numthreads(), "kind": "oracle",
                         "sample": f"{args.steps} x one time step of the 512^3 Neumann workload, FP64"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kernel", type=int, default=0, help="ACS_KERNEL_* (0 = auto)")
    ap.add_argument("--depth", type=int, default=1)
    ap.add_argument("--variant", type=int, default=-1, help="tile variant of the tiled kernel (-1 = tuned)")
    ap.add_argument("--chunk", type=int, default=0, help="planes per CTA with --variant (0 = automatic)")
    ap.add_argument("--profile", action="store_true",
                    help="only set up the 512^3 workload and run --steps time steps (for ncu captures)")
    ap.add_argument("--profile-lb", action="store_true",
                    help="only run --steps time steps of the collide-and-stream form on 256^3 Neumann FP32")
    ap.add_argument("--profile-lines", action="store_true",
                    help="only set up the 4096-line 1D workload and run --steps time steps")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="only run --steps forward+backward passes of the 1024^2 adjoint workload")
    ap.add_argument("--profile-batch", action="store_true",
                    help="only set up the 256-instance batched workload and run --steps time steps")
    ap.add_argument("--profile-2d", action="store_true",
                    help="only run --steps time steps of the 4096^2 Dirichlet workload (--dtype, --kernel, --depth)")
    ap.add_argument("--profile-energy", action="store_true",
                    help="only run --steps E_h / max-norm passes over the 512^3 FP32 state")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"],
                    help="state precision of --profile / --profile-2d")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch:
        return profile_batch(args)
    if args.profile_2d:
        return profile_2d(args)
    if args.profile_energy:
        return profile_energy(args)
    if args.profile_adjoint:
        return profile_adjoint(args)
    if args.profile_lines:
        return profile_lines(args)
    if args.profile_lb:
        return profile_lb(args)

    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    import paper_2312_07010_gb300 as P
    from workloads import cfg2
    P.lib()
    pdt = args.dtype if args.profile else "f32"
    w = cfg2(pdt)
    phi0_host = torch.from_numpy(w.phi0().astype(np.float32 if pdt == "f32" else np.float64)).pin_memory()
    phi0_dev = phi0_host.cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, pdt, stream=stream)
    if args.kernel:
        s.set_kernel(args.kernel, args.depth)
    if args.variant >= 0:
        P.check(P.lib().acs_set_variant(s.ctx, args.variant, args.chunk), "acs_set_variant")
    s.set_state(phi0_dev)
    s.step(2)  # the first step of an auto-kernel context runs the autotuner
    kernel, depth = s.get_kernel()
    vch = (ctypes.c_int(), ctypes.c_int())
    P.lib().acs_get_variant(s.ctx, ctypes.byref(vch[0]), ctypes.byref(vch[1]))
    variant, chunk = vch[0].value, vch[1].value
    if args.profile:
        s.set_state(phi0_dev)
        s.step(args.steps)
        s.sync()
        print(json.dumps({"profile": True, "kernel": kernel, "depth": depth, "time_steps": args.steps}))
        return 0
    log_every = 50
    n_logs = w.steps // log_every + 1

    def bench_step():
        s.set_state(phi0_dev)
        s.run_logged(w.steps, log_every)

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        bench_step()
    peak, peak_kind = _peaks()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            bench_step()
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    if pg is not None:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    updates = w.numel * w.steps * args.steps * ws
    value = updates / (ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers.  Serial: one context, each job
    # copies phi0 in, runs, copies the state out.  Pipelined (the reported number):
    # acs_pipe_*, three device states, so the copies of one job overlap its
    # neighbours' compute; each job still copies its own input in and result out.
    out_host = torch.empty(w.n, dtype=torch.float32).pin_memory()

    def e2e_serial_step():
        s.set_state_host(phi0_host)
        s.run_logged(w.steps, log_every)
        s.get_state_host(out_host)

    def timed_host(fn, k):
        barrier()
        t0 = time.perf_counter()
        fn(k)
        barrier()
        el = time.perf_counter() - t0
        if pg is not None:
            t = torch.tensor([el], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            el = float(t.item())
        return el

    e2e_serial_step()
    serial_s = timed_host(lambda k: [e2e_serial_step() for _ in range(k)], args.steps)

    with torch.cuda.stream(stream):
        pipe = P.Pipeline(w.n, w.eps, w.dt, w.h, w.bc, "f32", slots=3, stream=stream)
    for slot in range(pipe.slots):
        P.lib().acs_set_kernel(pipe.context(slot), kernel, depth)
        P.lib().acs_set_variant(pipe.context(slot), variant, chunk)
    outs = [pipe.host_buffer() for _ in range(pipe.slots)]
    logs = [pipe.log_buffer(w.steps, log_every) for _ in range(pipe.slots)]

    def e2e_jobs(k):
        for i in range(k):
            pipe.submit(phi0_host, outs[i % pipe.slots], w.steps, log_every, logs[i % pipe.slots])
        pipe.wait()

    e2e_jobs(pipe.slots)
    # at least 10 jobs, so that the first job's input copy and the last one's output copy
    # (which nothing overlaps) weigh as they do in a stream of jobs
    e2e_n = max(args.steps, 10)
    e2e_s = timed_host(e2e_jobs, e2e_n)
    e2e_val = w.numel * w.steps * e2e_n * ws / e2e_s / 1e9
    serial_val = updates / serial_s / 1e9
    pipe.close()
    state_bytes = w.numel * 4

    # the dominant kernel's launch duration: acs_step(2 K) is exactly two launches
    K = depth if kernel == P.ACS_KERNEL_TEMPORAL else 1
    s.set_state(phi0_dev)
    s.step(2 * K)
    reps = 20
    ea = torch.cuda.Event(enable_timing=True)
    eb = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ea.record(stream)
    for _ in range(reps):
        s.step(2 * K)
    eb.record(stream)
    torch.cuda.synchronize()
    launch_ms = ea.elapsed_time(eb) / (2 * reps)
    alg_bytes = 2 * 4 * w.numel * K
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    ktag = {P.ACS_KERNEL_NAIVE: "naive", P.ACS_KERNEL_TILED: f"tiled_v{variant}",
            P.ACS_KERNEL_TEMPORAL: f"temporal{K}_v{variant}"}[kernel]
    traffic = _traffic_from_profile(f"step3d_f32_neumann_512_{ktag}")

    # step launches, plus per logged state one reduction pass and its finishing launch;
    # on the streamed 3D kernel every logged state but the last is reduced by the first
    # step of its interval (fused), which leaves only the finishing launch
    fused_logs = n_logs - 1 if kernel == P.ACS_KERNEL_TILED else 0
    launches_per_step = (w.steps // K) + 2 * n_logs - fused_logs
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "cfg2_3d_neumann_512", "dims": 3, "n": 512, "bc": "neumann", "eps": w.eps,
                   "h": w.h, "dt": w.dt, "time_steps": w.steps, "log_every": log_every,
                   "kernel": ktag, "tile_variant": variant, "chunk": chunk,
                   "l2": "inputs larger than L2 (512 MiB per state buffer), no flush",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel_ms": launch_ms, "alg_bytes_per_launch": alg_bytes},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes + 16 * n_logs,
                "api": "acs_pipe_submit / acs_pipe_wait (pinned host buffers, three device states)",
                "jobs": e2e_n, "serial_value": serial_val, "serial_jobs": args.steps,
                "serial_api": "acs_set_state_host + acs_run_logged + acs_get_state_host"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "effective_hbm_frac": value / ws * 8 / peak,
    }
    if rank == 0 and ws == 1 and not args.no_extras:
        line["extra"] = extras(P, args)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample()
        if not args.no_extras:
            line.setdefault("extra", {})["oracle_cpu"] = oracle_cpu_timing()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def profile_2d(args):
    import numpy as np
    import torch

    import paper_2312_07010_gb300 as P
    from workloads import cfg3
    w = cfg3(args.dtype)
    s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, args.dtype)
    if args.kernel:
        s.set_kernel(args.kernel, args.depth)
    s.set_state(w.phi0().astype(np.float32 if args.dtype == "f32" else np.float64))
    s.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "cfg3_2d", "dtype": args.dtype, "kernel": s.get_kernel(), "time_steps": args.steps}))
    return 0


def profile_energy(args):
    import numpy as np
    import torch

    import paper_2312_07010_gb300 as P
    from workloads import cfg2
    w = cfg2("f32")
    s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    s.set_kernel(P.ACS_KERNEL_TILED)
    s.set_state(w.phi0().astype(np.float32))
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(args.steps):
        s.observe_async(out)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "energy_512", "passes": args.steps}))
    return 0


def profile_batch(args):
    import numpy as np
    import torch

    import paper_2312_07010_gb300 as P
    from workloads import batched_instances
    inst = batched_instances()
    b = P.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                [i.bc for i in inst], "f32")
    # largest instances first, as the autotuner picks for this workload
    b.set_temporal(max(1, args.depth), 0, 1 if args.depth > 1 else 0)
    b.set_states([i.phi0().astype(np.float32) for i in inst])
    b.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "batched", "instances": len(inst), "time_steps": args.steps,
                      "temporal_depth": b.get_temporal()[0]}))
    return 0


def profile_lb(args):
    import numpy as np
    import torch

    import paper_2312_07010_gb300 as P
    from workloads import dt_rule, uniform_field
    n, eps = 256, 0.01
    h = 1.0 / n
    s = P.AllenCahn((n, n, n), eps, dt_rule(3, eps, h), h, P.ACS_BC_NEUMANN, "f32")
    s.use_lb_form()
    s.set_state(uniform_field((n, n, n), -1, 1, 1).astype(np.float32))
    s.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "lb_form", "n": n, "time_steps": args.steps}))
    return 0


def profile_lines(args):
    import numpy as np
    import torch

    import paper_2312_07010_gb300 as P
    from workloads import line_instances
    lines = line_instances()
    L = P.Lines([i.n for i in lines], [i.eps for i in lines], [i.dt for i in lines], [i.h for i in lines],
                [i.bc for i in lines], "f32")
    L.set_states([i.phi0().astype(np.float32) for i in lines])
    L.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "lines", "lines": len(lines), "time_steps": args.steps}))
    return 0


def profile_adjoint(args):
    import numpy as np
    import torch

    import paper_2312_07010_gb300 as P
    from workloads import cfg5, tanh_disc
    w = cfg5()
    phi0 = torch.from_numpy(w.phi0().astype(np.float32)).cuda()
    target = torch.from_numpy(tanh_disc(w.n[0], w.h, w.eps).astype(np.float32)).cuda()
    s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    s.set_state(phi0)
    s.record_for_grad(w.steps, 50)
    for _ in range(args.steps):
        s.set_state(phi0)
        s.step(w.steps)
        s.grad(2 * (s.phi - target) / s.numel)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "adjoint", "time_steps": w.steps, "passes": args.steps}))
    return 0


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extras(P, args):
    """Secondary numbers: FP64 and 2D workloads, the adjoint, the batched form."""
    import numpy as np
    import torch

    from workloads import cfg1, cfg2, cfg3, cfg5, tanh_disc
    out = {}
    peak, _ = _peaks()
    # the E_h / max-norm pass on the 512^3 FP32 state: it reads the state once (4 B per
    # unknown) and forms every term exactly, so it is bound by FP32 issue, not HBM
    w2 = cfg2("f32")
    s = P.AllenCahn(w2.n, w2.eps, w2.dt, w2.h, w2.bc, "f32")
    s.set_state(torch.from_numpy(w2.phi0().astype(np.float32)).cuda())
    s.step(2)
    d2 = torch.empty(2, dtype=torch.float64, device="cuda")

    def observe():
        P.lib().acs_observe_async(s.ctx, ctypes.c_void_p(d2.data_ptr()))
    ms = _time(observe, 10)
    out["energy_pass_512cubed_f32"] = {"us": ms * 1e3, "alg_bytes": w2.numel * 4,
                                       "achieved_gbs": w2.numel * 4 / (ms * 1e-3) / 1e9,
                                       "hbm_frac": w2.numel * 4 / (ms * 1e-3) / 1e9 / peak,
                                       "bound": "FP32 issue (exact float-pair terms on packed lanes: about 42 "
                                                "packed operations per unknown)"}
    s.close()
    del s
    torch.cuda.empty_cache()
    # FP64 on the 512^3 workload (fewer steps)
    for name, w, nsteps in (("cfg2_fp64_512cubed", cfg2("f64"), 20), ("cfg3_fp32_4096sq", cfg3("f32"), 200),
                            ("cfg3_fp64_4096sq", cfg3("f64"), 50), ("cfg1_fp64_128sq", cfg1(), 1000)):
        s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, w.dtype)
        phi0 = torch.from_numpy(w.phi0().astype(np.float32 if w.dtype == "f32" else np.float64)).cuda()
        s.set_state(phi0)

        def go():
            s.step(nsteps)
        ms = _time(go, 3)
        glups = w.numel * nsteps / (ms * 1e-3) / 1e9
        esz = 4 if w.dtype == "f32" else 8
        k, d = s.get_kernel()
        rmode, rsplit = ctypes.c_int(), ctypes.c_int()
        P.check(P.lib().acs_get_root(s.ctx, ctypes.byref(rmode), ctypes.byref(rsplit)), "acs_get_root")
        out[name] = {"glups": glups, "ms_per_time_step": ms / nsteps, "hbm_frac_effective": glups * 2 * esz / peak,
                     "kernel": k, "depth": d, "root": {0: "newton", 1: "series", 2: "none"}[rmode.value],
                     "series_fp32_tail": bool(rsplit.value)}
        if name == "cfg1_fp64_128sq":
            # the configuration as stated: 1000 steps with E_h and max|phi| every 10
            def logged():
                s.run_logged(w.steps, w.log_every)
            ms = _time(logged, 3)
            out[name]["logged_every_10_glups"] = w.numel * w.steps / (ms * 1e-3) / 1e9
            out[name]["logged_every_10_ms"] = ms
        s.close()
        del s, phi0
        torch.cuda.empty_cache()
    # FP64 steps are bound by the FP64 pipe (ncu: 82-86 % busy), which retires 2 FP64
    # operations per cycle per SM; per update the step issues 17 of them in 2D (predictor:
    # 3 DADD, 2 DMUL, 2 DFMA; series root: 1 DMUL, 9 DFMA) and 19 in 3D (5 DADD), two fewer
    # where the series sums its last three terms in FP32 (acs_get_root)
    sm_mhz = _sm_max_mhz()
    for name, ops in (("cfg3_fp64_4096sq", 17), ("cfg2_fp64_512cubed", 19)):
        ops -= 2 if out[name]["series_fp32_tail"] else 0
        roof = 2.0 * 152 * sm_mhz * 1e6 / ops / 1e9
        out[name]["fp64_pipe_roof_glups"] = roof
        out[name]["fp64_ops_per_update"] = ops
        out[name]["fp64_pipe_roof_frac"] = out[name]["glups"] / roof
    # the 4096^2 Dirichlet FP32 workload by kernel: single steps, then K fused steps per pass
    w = cfg3("f32")
    phi0 = torch.from_numpy(w.phi0().astype(np.float32)).cuda()
    depths = {}
    for kernel, depth in ((P.ACS_KERNEL_TILED, 1), (P.ACS_KERNEL_TEMPORAL, 2), (P.ACS_KERNEL_TEMPORAL, 3),
                          (P.ACS_KERNEL_TEMPORAL, 4)):
        s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
        s.set_kernel(kernel, depth)
        s.set_state(phi0)
        ms = _time(lambda: s.step(96), 3)
        glups = w.numel * 96 / (ms * 1e-3) / 1e9
        depths[f"K{depth}"] = {"glups": glups, "us_per_time_step": 1e3 * ms / 96,
                               "hbm_frac_effective": glups * 8 / peak}
        s.close()
    out["cfg3_fp32_4096sq_by_depth"] = depths
    del phi0
    torch.cuda.empty_cache()
    # batched: 256 2D instances (seed 2), FP32, 500 steps in one persistent launch,
    # against the same instances stepped one after another as single problems
    from workloads import BATCH_STEPS, batched_instances
    inst = batched_instances()
    b = P.Batch([i.n for i in inst], [i.eps for i in inst], [i.dt for i in inst], [i.h for i in inst],
                [i.bc for i in inst], "f32")
    states = [i.phi0().astype(np.float32) for i in inst]
    b.set_states(states)
    b.set_config(0, 1, 0)  # all resident CTAs, one block per ticket, instance order
    b.set_temporal(1)      # single steps
    b.step(BATCH_STEPS)  # records the graph
    torch.cuda.synchronize()
    b.set_states(states)
    ms_default = _time(lambda: b.step(BATCH_STEPS), 1)
    us_tune = b.autotune()
    cfg_b = b.get_config()
    tcfg_b = b.get_temporal()
    b.set_states(states)
    b.step(BATCH_STEPS)
    torch.cuda.synchronize()
    b.set_states(states)
    ms_b = _time(lambda: b.step(BATCH_STEPS), 1)
    by_depth = {}
    for depth in (1, 2, 3, 4):
        # the tuned single-step configuration, or the tuned unit height and order at each depth
        b.set_temporal(depth, tcfg_b[1], tcfg_b[2])
        b.step(BATCH_STEPS)
        torch.cuda.synchronize()
        b.set_states(states)
        ms_d = _time(lambda: b.step(BATCH_STEPS), 1)
        by_depth[str(depth)] = {"glups": sum(i.n * i.n for i in inst) * BATCH_STEPS / (ms_d * 1e-3) / 1e9,
                                "ms": ms_d}
    b.set_temporal(*tcfg_b)
    units = sum(i.n * i.n for i in inst) * BATCH_STEPS
    E, M = b.observe()
    singles = []
    for k, i in enumerate(inst):
        s1 = P.AllenCahn((i.n, i.n), i.eps, i.dt, i.h, i.bc, "f32")
        s1.set_state(states[k])
        s1.step(BATCH_STEPS)
        singles.append(s1)
    torch.cuda.synchronize()

    def seq():
        for s1 in singles:
            s1.step(BATCH_STEPS)
    ms_s = _time(seq, 1)
    out["cfg4_batched_256"] = {"glups": units / (ms_b * 1e-3) / 1e9, "ms": ms_b, "instances": len(inst),
                               "unknowns": sum(i.n * i.n for i in inst), "steps": BATCH_STEPS,
                               "sequential_single_glups": units / (ms_s * 1e-3) / 1e9, "sequential_ms": ms_s,
                               "speedup_vs_sequential": ms_s / ms_b, "max_abs_phi": float(np.max(M)),
                               "hbm_frac_effective": units / (ms_b * 1e-3) * 8 / (peak * 1e9),
                               "autotuned_config": {"ctas_per_sm": cfg_b[0], "blocks_per_ticket": cfg_b[1],
                                                    "block_order": cfg_b[2], "temporal_depth": tcfg_b[0],
                                                    "rows_per_unit": tcfg_b[1], "unit_order": tcfg_b[2],
                                                    "tuning_us_per_step": us_tune},
                               "by_temporal_depth": by_depth,
                               "default_config_glups": units / (ms_default * 1e-3) / 1e9}
    del singles, b
    torch.cuda.empty_cache()
    # adjoint: 1024^2 periodic, FP32, 500 steps, checkpoints every 50
    w = cfg5()
    phi0 = torch.from_numpy(w.phi0().astype(np.float32)).cuda()
    target = torch.from_numpy(tanh_disc(w.n[0], w.h, w.eps).astype(np.float32)).cuda()
    s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    s.set_state(phi0)
    s.record_for_grad(w.steps, 50)

    def fwd_bwd():
        s.set_state(phi0)
        s.step(w.steps)
        g = 2 * (s.phi - target) / s.numel
        s.grad(g)

    def fwd_only():
        s.set_state(phi0)
        s.step(w.steps)
        torch.cuda.synchronize()
    # the plain single-instance forward on the same GPU (no checkpoint recording)
    sp = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")

    def plain_fwd():
        sp.set_state(phi0)
        sp.step(w.steps)
    ms_fb = _time(fwd_bwd, 3)
    ms_f = _time(fwd_only, 3)
    ms_p = _time(plain_fwd, 3)
    sp.close()
    s.close()
    del s
    torch.cuda.empty_cache()
    # the same with every state stored (501 x 4 MiB): the backward sweep recomputes nothing
    s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    s.set_state(phi0)
    s.record_for_grad(w.steps, 1)
    ms_fb1 = _time(fwd_bwd, 3)
    out["cfg5_adjoint_1024sq"] = {"fwd_bwd_ms_per_time_step": ms_fb / w.steps,
                                  "recording_fwd_ms_per_time_step": ms_f / w.steps,
                                  "plain_fwd_ms_per_time_step": ms_p / w.steps,
                                  "fwd_bwd_over_plain_fwd": ms_fb / ms_p,
                                  "checkpoint_every": 50,
                                  "store_every_state_fwd_bwd_ms_per_time_step": ms_fb1 / w.steps,
                                  "store_every_state_over_plain_fwd": ms_fb1 / ms_p}
    s.close()
    del s
    torch.cuda.empty_cache()
    # batched lines: 4096 1D problems (lengths log-uniform in [32, 4096], seed 4), FP32,
    # 2000 steps in one call, against single-line runs of a 64-line sample
    from workloads import LINE_STEPS, line_instances
    lines = line_instances()
    Lb = P.Lines([i.n for i in lines], [i.eps for i in lines], [i.dt for i in lines], [i.h for i in lines],
                 [i.bc for i in lines], "f32")
    lstates = [i.phi0().astype(np.float32) for i in lines]
    Lb.set_states(lstates)
    ms_l = _time(lambda: Lb.step(LINE_STEPS), 2)
    lunits = sum(i.n for i in lines) * LINE_STEPS
    sample = lines[:: len(lines) // 64][:64]
    singles = []
    for i in sample:
        s1 = P.AllenCahn((i.n,), i.eps, i.dt, i.h, i.bc, "f32")
        s1.set_state(i.phi0().astype(np.float32))
        singles.append(s1)

    def seq_lines():
        for s1 in singles:
            s1.step(LINE_STEPS)
    ms_s = _time(seq_lines, 1)
    sunits = sum(i.n for i in sample) * LINE_STEPS
    out["lines_4096_1d"] = {"glups": lunits / (ms_l * 1e-3) / 1e9, "ms": ms_l, "lines": len(lines),
                            "unknowns": sum(i.n for i in lines), "steps": LINE_STEPS,
                            "sequential_single_glups": sunits / (ms_s * 1e-3) / 1e9,
                            "sequential_sample": "64 lines, same lengths distribution"}
    del singles
    Lb.close()
    torch.cuda.empty_cache()
    # the collide-and-stream population form on the 512^3 workload, against the FD form:
    # per update it writes and reads 2d+1 populations (collide: 1 read + 7 writes; stream:
    # 7 + 1 reads + 1 write = 17 values), and keeps them resident
    w = cfg2("f32")
    s = P.AllenCahn(w.n, w.eps, w.dt, w.h, w.bc, "f32")
    s.use_lb_form()
    phi0 = torch.from_numpy(w.phi0().astype(np.float32)).cuda()
    s.set_state(phi0)
    nsteps = 20

    def go_lb():
        s.step(nsteps)
    ms = _time(go_lb, 2)
    glups = w.numel * nsteps / (ms * 1e-3) / 1e9
    vals = 2 * (2 * 3 + 1) + 3
    out["cfg2_fp32_lb_form"] = {"glups": glups, "ms_per_time_step": ms / nsteps,
                                "alg_bytes_per_update": vals * 4, "achieved_gbs": glups * vals * 4,
                                "hbm_frac": glups * vals * 4 / peak,
                                "resident_arrays_lb": 2 * 3 + 2, "resident_arrays_fd": 2}
    s.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
