#!/usr/bin/env python3
"""Throughput of the grid-refined KBC step on one GB300 (or N replicas).

Workload (default): the three-level turbulent-channel layout -- 256x64x128
coarse nodes, periodic x/z, half-way bounce-back walls in y, 2x bands
(y in [0,8], [55,63]) and 4x bands (y in [0,4], [59,63]), body force for
Re_tau = 180, laminar profile plus seeded +-5% perturbations, FP32.
A step is one coarse step: every level advances once per 2^-level of the
coarse time step (78,184,448 node updates).

Metric: fine-node-equivalent MLUPS = node updates per coarse step x steps /
time / 1e6.  The dominant kernel's HBM roofline fraction is reported next to
it, from CUDA events around each of its launches inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]
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

METRIC = "MLUPS (fine-node equiv) and % of HBM roofline; adjoint/forward time ratio"
UNIT = "MLUPS"
BYTES_PER_UPDATE = {"fp64": 432, "fp32": 216, "fp16s": 108, "bf16s": 108}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f32", "bf16s": "f32"}
L2_BYTES = 129e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", choices=["channel", "channel-half", "tgv", "sphere", "rbc"], default="channel")
    ap.add_argument("--storage", choices=sorted(BYTES_PER_UPDATE), default="fp32")
    ap.add_argument("--pr", type=float, default=0.7, help="Prandtl number of the rbc workload (Table I regime)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the full sphere and Rayleigh-Benard lines and the storage sweep")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the adjoint/forward timing of the 64^3 adjoint case (diagnostic line)")
    return ap.parse_args()


def workload(name, pr=0.7):
    from paper_1608_06915_gb300 import inputs as I
    if name in ("channel", "channel-half"):
        n = (256, 64, 128) if name == "channel" else (128, 64, 64)
        case = I.channel_case(n=n)

        def fields(info):
            return I.channel_fields(case, info["level"], info["org"], info["dim"])
        desc = "channel %dx%dx%d coarse, 3 levels (2x y in [0,8],[55,63]; 4x y in [0,4],[59,63]), Re_tau=180" % n
        return case, fields, desc
    if name == "sphere":
        case = I.sphere_case()

        def fields(info):
            x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
            return I.uniform_fields(x, (0.05, 0.0, 0.0))
        return case, fields, "sphere wake 384x192x192 coarse, 4 levels, D=64 finest nodes, Re=3700"
    if name == "rbc":
        case = I.rbc_case(pr=pr)

        def fields(info):
            return I.rbc_fields(case, info["level"], info["org"], info["dim"])
        return case, fields, ("Rayleigh-Benard 256x256x128 coarse, 3 levels (2x z in [0,12],[115,127]; 4x z in "
                              "[0,6],[121,127]), Ra=1e7, Pr=%g, thermal f+g" % pr)
    case = I.tgv_case()

    def fields(info):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        return I.tgv_fields(x, y, z)
    return case, fields, "Taylor-Green 32^3 with [8,24]^3 refined 2x"


def sample_case(name):
    """Bounded sample of the workload for the oracle: the same layout and
    parameters with the periodic extents reduced."""
    from paper_1608_06915_gb300 import inputs as I
    if name in ("channel", "channel-half"):
        case = I.channel_case(n=(16, 64, 8))

        def fields(info):
            return I.channel_fields(case, info["level"], info["org"], info["dim"])
        return case, fields, "channel 16x64x8 coarse (x/z extents of the 256x64x128 case reduced), same bands"
    if name == "rbc":
        case = I.rbc_small_case()

        def fields(info):
            return I.rbc_fields(case, info["level"], info["org"], info["dim"])
        return case, fields, "Rayleigh-Benard 8x8x32 coarse, same layering, Ra=1e5"
    if name == "sphere":
        case = I.sphere_case(scale=8)

        def fields(info):
            x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
            return I.uniform_fields(x, (0.05, 0.0, 0.0))
        return case, fields, "sphere 48x24x24 coarse, same nesting"
    case, fields, _ = workload(name)
    return case, fields, "Taylor-Green 32^3 with [8,24]^3 refined"


# ---------------------------------------------------------------------------
def oracle_run(name, seconds=None, steps=None, warmup=0):
    """Time the FP64 oracle on the bounded sample: either for about `seconds`
    of work, or exactly `steps` coarse steps after `warmup`."""
    from oracle import oracle as O
    O.build()
    case, fields, desc = sample_case(name)
    o = O.Oracle(case)
    for p, info in enumerate(o.patches):
        out = fields(info)
        o.init_equilibrium(p, *out)
    nup = o.node_updates_per_step()
    for _ in range(warmup):
        o.step(1)
    t0 = time.perf_counter()
    done = 0
    if steps is not None:
        o.step(steps)
        done = steps
    else:
        while True:
            o.step(1)
            done += 1
            if time.perf_counter() - t0 >= seconds:
                break
    dt = time.perf_counter() - t0
    return dict(value=nup * done / dt / 1e6, unit=UNIT, cores=O.max_threads(), kind="oracle",
                sample="%s; %d coarse step(s), %.0f node updates each, %.1f s" % (desc, done, nup, dt),
                seconds=dt, steps=done)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    r = oracle_run(args.workload, steps=args.steps, warmup=args.warmup)
    _, _, desc = workload(args.workload, args.pr)
    line = dict(impl="reference", metric=METRIC, value=r["value"], unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * r["seconds"] / r["steps"], higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=desc, storage="fp64 (oracle)", sample=r["sample"]),
                cpu_baseline=dict(value=r["value"], unit=UNIT, cores=r["cores"], kind="oracle", sample=r["sample"]),
                e2e=dict(value=r["value"], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9 or c[0] != self.gpu:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if c[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))


def source_hash():
    """Hash of the sources of the stream-collide kernels (profiles record it)."""
    h = hashlib.sha256()
    for f in ("device.cuh", "collide.cuh", "sc_tma.cuh", "sc_tma.cu", "sc_tma_fp32.cu"):
        with open(os.path.join(ROOT, "paper_1608_06915_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name, storage, nodes_per_launch):
    """DRAM bytes (read + write) per launch from the ncu summary in profiles/:
    the per-node traffic of the captured (smaller) case scaled by the nodes of
    one launch here; None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel_name, storage))
    if not os.path.exists(path):
        return None
    per_node, srch = None, None
    for line in open(path):
        if line.startswith("source_hash:"):
            srch = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_node:"):
            per_node = float(line.split(":", 1)[1].strip())
    if per_node is None or srch != source_hash():
        return None
    return per_node * nodes_per_launch


def end_to_end(args, g, L, host_fields, dfields, nup, world, barrier, dev):
    """The metric through the public API with host buffers: pinned H2D of the
    initial fields, init, K coarse steps, moments and D2H of rho and u."""
    import numpy as np
    import torch
    import torch.distributed as dist
    stream = g.stream
    h_in = [(torch.from_numpy(np.ascontiguousarray(r, dtype=np.float32)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).pin_memory()) for r, u in host_fields]
    h_out = [(torch.empty_like(a).pin_memory(), torch.empty_like(b).pin_memory()) for a, b in h_in]
    d_out = [(torch.empty_like(dr), torch.empty_like(du)) for dr, du in dfields]
    h2d = sum(a.numel() * 4 + b.numel() * 4 for a, b in h_in)
    d2h = h2d
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        f0.record(stream)
        for p, ((hr, hu), (dr, du)) in enumerate(zip(h_in, dfields)):
            dr.copy_(hr, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            g.init_equilibrium(p, dr, du)
        g.step(args.steps)
        for p, ((orr, ou), (hr, hu)) in enumerate(zip(d_out, h_out)):
            L.lib().lbm_moments(g.handle, p, L.Grid._ptr(orr), L.Grid._ptr(ou), None, None, 0)
            hr.copy_(orr, non_blocking=True)
            hu.copy_(ou, non_blocking=True)
        f1.record(stream)
    barrier()
    te = f0.elapsed_time(f1) / 1e3
    te_t = torch.tensor([te], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te_t, op=dist.ReduceOp.MAX)
    te = float(te_t.item())
    e2e = dict(value=nup * args.steps * world / te / 1e6, unit=UNIT, h2d_bytes_per_step=h2d / args.steps,
               d2h_bytes_per_step=d2h / args.steps,
               note="per job: H2D of initial rho,u (pinned), init, %d coarse steps, D2H of rho,u; grid layout "
                    "built and bound before timing" % args.steps)
    return e2e


def gamma_indicator(g, bpu, peak, block=8, reps=10):
    """Time of the refinement indicator (lbm_gamma_blocks) over the level-0
    patch: it reads the stored f of every fluid node once (half the bytes of
    an isothermal node update, bpu), CUDA events on the grid's stream after
    one warm call."""
    import torch
    fluid = float((g.mask(0) == 1).sum())
    g.gamma_blocks(0, block)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(g.stream)
    for _ in range(reps):
        g.gamma_blocks(0, block)
    e1.record(g.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = fluid * bpu / 2 / (ms / 1e3) / 1e9
    return dict(kernel="k_gamma_blocks, level 0, blocks of %d^3" % block, ms_per_call=ms, fluid_nodes=fluid,
                bytes_per_node=bpu / 2, achieved_gbs=gbs, frac=gbs / peak)


def adjoint_ratio(dev, storage="fp32", K=20, reps=3):
    """Time of the discrete adjoint of K coarse steps (lbm_adjoint_step: restore,
    recompute with snapshots, reverse) over the time of K forward steps, on the
    64^3 box with the [24,40]^3 box refined 2x (divergence-free random field):
    `reps` alternating timings of each, medians."""
    import statistics
    import torch
    from paper_1608_06915_gb300 import inputs as I
    from paper_1608_06915_gb300 import lbm as L
    case = I.adjoint_case()
    g = L.Grid(case, storage, device=dev)
    modes = I.divfree_modes(n=64, kmax=4.0, rms=0.03, seed=4)
    for p, info in enumerate(g.patches):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        rho, u = I.divfree_fields(x, y, z, modes)
        g.init_equilibrium(p, torch.from_numpy(rho).to(dev), torch.from_numpy(u).to(dev))
    tune = g.autotune(trials=4)  # the forward timed below is the tuned one
    ck = torch.empty(g.checkpoint_bytes(), dtype=torch.uint8, device=dev)
    lam, ws = g.adjoint_buffers(K)
    g.checkpoint(ck, save=True)
    g.step(K)
    # warm-up: the first call runs the reverse walk directly, the second
    # captures it as a CUDA graph, which later calls replay
    for _ in range(2):
        g.adjoint_seed(lam, ws)
        g.adjoint_step(ck, K, lam, ws)
    fwds, adjs = [], []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize(dev)
        e[0].record(g.stream)
        g.step(K)
        e[1].record(g.stream)
        g.adjoint_seed(lam, ws)
        e[2].record(g.stream)
        g.adjoint_step(ck, K, lam, ws)  # leaves the state at the segment start
        e[3].record(g.stream)
        torch.cuda.synchronize(dev)
        fwds.append(e[0].elapsed_time(e[1]) / K)
        adjs.append(e[2].elapsed_time(e[3]) / K)
    fwd, adj = statistics.median(fwds), statistics.median(adjs)
    return dict(workload="64^3 periodic, [24,40]^3 refined 2x, %s, segments of %d coarse steps" % (storage, K),
                forward_ms_per_step=fwd, adjoint_ms_per_step=adj, ratio=adj / fwd, autotune=tune,
                forward_ms_per_step_each=fwds, adjoint_ms_per_step_each=adjs,
                note="medians of %d alternating timings; adjoint time includes restoring the checkpoint and "
                     "recomputing the segment" % reps)


def measure_workload(name, storage, steps, warmup, dev, pr=0.7, peak=None, instrument=True):
    """One workload on one GPU: layout, equilibrium init, autotune, warm-up,
    `steps` coarse steps replayed as graphs (CUDA events on the grid's
    stream), then the same steps launched kernel by kernel between events for
    the per-class kernel table and the dominant kernel's roofline.  Returns
    a dict; frees the grid."""
    import numpy as np
    import torch
    from paper_1608_06915_gb300 import lbm as L
    case, fields, desc = workload(name, pr)
    g = L.Grid(case, storage, device=dev)
    for p, info in enumerate(g.patches):
        h = fields(info)
        t = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in h]
        g.init_equilibrium(p, t[0], t[1], t[2] if len(t) > 2 else None)
    nup = g.node_updates()
    tune = g.autotune(trials=2)
    g.step(warmup)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.step(steps)
    e1.record(g.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    out = dict(workload=desc, storage=storage, value=nup / (ms / 1e3) / 1e6, unit=UNIT, ms_per_step=ms,
               steps=steps, node_updates_per_coarse_step=nup, autotune=tune)
    if instrument:
        g.timing(True)
        g.step(steps)
        torch.cuda.synchronize(dev)
        report = g.timing_report()
        g.timing(False)
        top = max(report, key=lambda r: r["ms"])
        bpu = BYTES_PER_UPDATE[storage] * (2 if case.get("thermal") else 1)
        avg_ms = top["ms"] / top["launches"]
        alg = top["nodes"] / top["launches"] * bpu
        achieved = alg / (avg_ms / 1e3) / 1e9
        out["roofline"] = dict(bound="hbm", kernel="%s level %d" % (top["kind"], top["level"]), achieved=achieved,
                               peak=peak, unit="GB/s", frac=achieved / peak if peak else None,
                               bytes_per_node_update=bpu, avg_launch_ms=avg_ms)
        out["kernels"] = [dict(r, avg_us=1e3 * r["ms"] / r["launches"]) for r in report]
    d = g.diagnostics()
    out["diagnostics"] = dict(mass=d["mass"], min_rho=d["min_rho"], status=d["status"])
    del g
    torch.cuda.empty_cache()
    return out


def storage_error(name, storage, dev, steps):
    """Relative L2 error of the velocity of a storage against FP64 storage on
    the reduced case of the workload after `steps` coarse steps, both on the
    GPU (the FP64 path equals the FP64 oracle to 1e-12, which the parity tests
    check)."""
    import numpy as np
    import torch
    from paper_1608_06915_gb300 import lbm as L
    case, fields, desc = sample_case(name)
    res = {}
    for st in ("fp64", storage):
        g = L.Grid(case, st, device=dev)
        for p, info in enumerate(g.patches):
            h = fields(info)
            g.init_equilibrium(p, torch.from_numpy(np.ascontiguousarray(h[0])).to(dev),
                               torch.from_numpy(np.ascontiguousarray(h[1])).to(dev))
        g.step(steps)
        us = []
        for p in range(len(g.patches)):
            _, u, _, _ = g.moments(p)
            m = g.mask(p) == 1
            us.append(u.cpu().numpy()[:, m])
        res[st] = np.concatenate(us, axis=1)
        del g
    ref = res["fp64"]
    return float(np.sqrt(np.sum((res[storage] - ref) ** 2) / np.sum(ref ** 2)))


def cuda_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1608_06915_gb300 import lbm as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    case, fields, desc = workload(args.workload, args.pr)
    g = L.Grid(case, args.storage, device=dev)
    host_all = [fields(info) for info in g.patches]
    host_fields = [(h[0], h[1]) for h in host_all]
    dfields = []
    for p, h in enumerate(host_all):
        dr = torch.from_numpy(np.ascontiguousarray(h[0], dtype=np.float32)).to(dev)
        du = torch.from_numpy(np.ascontiguousarray(h[1], dtype=np.float32)).to(dev)
        dT = torch.from_numpy(np.ascontiguousarray(h[2], dtype=np.float32)).to(dev) if len(h) > 2 else None
        dfields.append((dr, du))
        g.init_equilibrium(p, dr, du, dT)
    nup = g.node_updates()
    stream = g.stream

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # setup: the autotuner times each variant (TMA kernel x sample schedule) over 4 coarse steps
    # (advancing the state) and keeps the fastest; then the warm-up
    tune = g.autotune(trials=4)
    g.step(args.warmup)
    barrier()
    # timed region: K coarse steps replayed as CUDA graphs, events on the grid's stream
    clocks = Clocks(local) if rank == 0 else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    barrier()
    # the same K steps again, every kernel launched directly between its own
    # pair of events: the per-kernel durations of the roofline
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.timing(True)
    e2.record(stream)
    g.step(args.steps)
    e3.record(stream)
    barrier()
    report = g.timing_report()
    g.timing(False)
    clk = clocks.stop() if clocks else None
    t = e0.elapsed_time(e1) / 1e3
    t_instr = e2.elapsed_time(e3) / 1e3
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t = float(tt.item())
    diag = g.diagnostics()
    value = nup * args.steps * world / t / 1e6
    # the refinement benefit: node updates a uniform finest-level grid would need
    nlev = 1 + max(info["level"] for info in g.patches)
    n_uniform = float(np.prod([float(v) * (1 << (nlev - 1)) for v in case["n"]])) * (1 << (nlev - 1))
    uniform_equiv = n_uniform * args.steps * world / t / 1e6

    # dominant kernel: the class with the largest device time
    top = max(report, key=lambda r: r["ms"])
    bpu = BYTES_PER_UPDATE[args.storage] * (2 if case.get("thermal") else 1)
    avg_ms = top["ms"] / top["launches"]
    nodes_per_launch = top["nodes"] / top["launches"]
    alg_bytes = nodes_per_launch * bpu
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = float(peaks["hbm_gbs"]) if peaks else 6800.0
    traffic = ncu_traffic("k_sc_tma_channel", args.storage, nodes_per_launch) if args.workload.startswith(
        "channel") else None
    roofline = dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak, traffic=traffic,
                    peak_source="measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                    kernel=("k_sc_tma, TMA tile pass batched over the patches of each instant"
                            if top["kind"] == "stream_collide_tma" else "%s level %d" % (top["kind"], top["level"])),
                    avg_launch_ms=avg_ms, alg_bytes_per_launch=alg_bytes, bytes_per_node_update=bpu,
                    frac_of_nominal_7900=achieved / 7900.0)
    kernels = [dict(r, avg_us=1e3 * r["ms"] / r["launches"]) for r in report]
    launches = sum(r["launches"] for r in report)

    indicator = gamma_indicator(g, BYTES_PER_UPDATE[args.storage], peak) if rank == 0 else None

    e2e = None
    if not args.no_e2e and not case.get("thermal"):
        e2e = end_to_end(args, g, L, host_fields, dfields, nup, world, barrier, dev)

    adj = None
    if rank == 0 and not args.no_adjoint and args.workload == "channel":
        adj = adjoint_ratio(dev)

    # the other workloads at full size, and the storage sweep (rank 0, after
    # the timed region; each grid is freed before the next)
    extras = {}
    ws = g.device_bytes
    if rank == 0 and args.workload == "channel" and not args.no_extras:
        del g
        torch.cuda.empty_cache()
        extras["sphere"] = measure_workload("sphere", "fp32", 10, 3, dev, peak=peak)
        extras["rbc"] = measure_workload("rbc", "fp32", 4, 2, dev, pr=args.pr, peak=peak)
        sweep = []
        for name in ("channel", "sphere"):
            for st in ("fp32", "fp16s", "bf16s"):
                if name == "channel" and st == args.storage:
                    r = dict(workload=desc, storage=st, value=value, ms_per_step=1e3 * t / args.steps,
                             roofline=dict(frac=roofline["frac"], bytes_per_node_update=bpu))
                elif name == "sphere" and st == "fp32":
                    r = extras["sphere"]
                else:
                    r = measure_workload(name, st, 10, 3, dev, peak=peak)
                err = storage_error(name, st, dev, 50 if name == "channel" else 20) if st != "fp64" else 0.0
                sweep.append(dict(workload=name, storage=st, mlups=r["value"], ms_per_step=r["ms_per_step"],
                                  roofline_frac=r["roofline"]["frac"],
                                  bytes_per_node_update=r["roofline"]["bytes_per_node_update"],
                                  u_rel_l2_vs_fp64=err))
        extras["storage_sweep"] = dict(
            rows=sweep, note="MLUPS and the dominant kernel's HBM fraction at the storage's bytes per node update; "
                             "u_rel_l2_vs_fp64: velocity error against FP64 storage on the reduced case (channel "
                             "16x64x8, 50 coarse steps; sphere 48x24x24, 20 coarse steps), both on the GPU")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r = oracle_run(args.workload, seconds=15.0)
        cpu = dict(value=r["value"], unit=UNIT, cores=r["cores"], kind="oracle", sample=r["sample"])

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=1e3 * t / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype=DTYPE[args.storage], data="synthetic",
                    config=dict(workload=desc, storage=args.storage, node_updates_per_coarse_step=nup,
                                parallelism="replicas" if world > 1 else "single GPU",
                                launch="one CUDA graph per coarse step",
                                autotune=tune,
                                direct_launch_ms_per_step=1e3 * t_instr / args.steps,
                                l2="no flush: working set %.2f GB > %.0f MB L2" % (ws / 1e9, L2_BYTES / 1e6)),
                    roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches, clocks=clk,
                    adjoint_forward_ratio=adj, gamma_indicator=indicator, **extras,
                    uniform_fine_equivalent=dict(
                        value=uniform_equiv, unit=UNIT,
                        note="node updates of a uniform grid at the finest spacing (%d levels) per coarse step, "
                             "%.4g, over the same time" % (nlev, n_uniform)),
                    kernels=kernels,
                    diagnostics=dict(mass=diag["mass"], min_rho=diag["min_rho"], status=diag["status"]))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.adjoint_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(dict(adjoint_forward_ratio=adjoint_ratio(torch.device("cuda", 0)))), flush=True)
        return 0
    return cuda_arm(args)


if __name__ == "__main__":
    sys.exit(main())
