#!/usr/bin/env python3
"""Throughput benchmark of the D3Q19 BGK hot path on GB300.

Default workload: fully periodic 384^3 lattice, FP32 storage of f_i - w_i,
tau = 0.8, initial shear wave u_x = 0.01 sin(2 pi z / N) at rho = 1 from
equilibrium. One benchmark step = one fused pull stream-and-collide update of
every node (one kernel launch). Metric: MLUPS (million lattice updates per
second, Sec. 1 footnote), plus the fraction of the measured HBM bandwidth
under the byte model of Sec. 4.1 (152 B per update in FP32).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica on its own GPU (the
lattice does not shard in this build); rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 384
# lattice updates per second; the HBM-roofline fraction is in "roofline" and
# the adjoint/forward time ratio with its accuracy in extras.adjoint
METRIC = "D3Q19 MLUPS"
TAU = 0.8
AMP = 0.01
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_DEFAULT, help="lattice edge (cube)")
    p.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    p.add_argument("--extras", default="all",
                   help="comma list of secondary workloads: storage,streaming,adjoint,batched,sweep,"
                        "tables (the paper's block-size x lattice-size experiment) (or all, the "
                        "default, for these six) and capacity (1024^3, opt-in)")
    p.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                   help="storage of the main timed workload (profiling runs)")
    p.add_argument("--geometry", default="periodic", choices=["periodic", "cavity"],
                   help="geometry of the main timed workload (profiling runs)")
    p.add_argument("--adj-n", type=int, default=128)
    p.add_argument("--adj-steps", type=int, default=500)
    p.add_argument("--batch-steps", type=int, default=2000)
    p.add_argument("--e2e-calls", type=int, default=5)
    p.add_argument("--cpu-sample-n", type=int, default=128)
    p.add_argument("--cpu-sample-steps", type=int, default=20,
                   help="oracle updates per call of the CPU baseline sample")
    p.add_argument("--cpu-sample-seconds", type=float, default=12.0,
                   help="the CPU baseline repeats its calls until this much work is timed")
    return p.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("paper_1309_1983_gb300/csrc/lbm_step_x2.cu", "paper_1309_1983_gb300/csrc/d3q19.cuh",
                  "paper_1309_1983_gb300/csrc/stream.cuh", "paper_1309_1983_gb300/csrc/internal.h",
                  "paper_1309_1983_gb300/csrc/pack.cuh", "paper_1309_1983_gb300/csrc/check.cuh")


def code_only(text):
    """C/C++ source without comments and blank lines (what the compiler sees
    of the kernel, as far as the hash below is concerned)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(read=None):
    """First 16 hex digits of the sha256 of the benchmark kernel's sources,
    comments and blank lines removed; `read(rel)` may supply the texts."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, rel)) as fh:
                text = fh.read()
        else:
            text = read(rel)
        h.update(code_only(text).encode())
    return h.hexdigest()[:16]


def ncu_traffic(summary_name):
    """DRAM bytes (read + write) per launch of the step kernel, measured by
    ncu at the benchmark's full size and recorded in a committed summary;
    None when the summary is missing or was taken on a different kernel
    source."""
    path = os.path.join(ROOT, "profiles", summary_name)
    try:
        kv = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.out = os.path.join("/tmp", f"lbm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.out):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    sm.append(float(parts[2]))
                    mx = float(parts[3])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[6:10]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.remove(self.out)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n, steps, min_seconds=0.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded
    sample: a periodic n^3 shear-wave lattice (the same workload, smaller),
    calls of ``steps`` updates repeated until at least ``min_seconds`` of
    work (at least one call). Returns MLUPS, the thread count, the seconds
    and the updates timed."""
    import oracle as O
    from paper_1309_1983_gb300 import workloads as W
    L = O.Lattice(n, n, n, TAU)
    f = O.to_aos(O.init_equilibrium(L, None, W.shear_wave(n, n, n, AMP)))
    f = O.run_aos(L, f, 1)  # warm the pages and the thread pool
    done = 0
    t0 = time.perf_counter()
    while True:
        f = O.run_aos(L, f, steps)
        done += steps
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    return n ** 3 * done / dt / 1e6, O.max_threads(), dt, done


def aggregate_replicas(ms, cells, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of ``world`` independent replicas: every rank
    updated ``cells`` nodes ``steps`` times; the job took as long as the
    slowest rank (max over ranks of the timed region, in ms). Returns
    (max ms, MLUPS over all ranks)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * cells * steps / (ms_max / 1e3) / 1e6


def workload_config(n):
    """The benchmarked workload, shared by both arms' JSON lines."""
    cells = n ** 3
    return {"workload": f"d3q19_bgk_periodic_{n}^3_fp32_shear_wave",
            "nx": n, "ny": n, "nz": n, "tau": TAU, "storage": "f32 (f_i - w_i)",
            "init": f"u_x = {AMP} sin(2 pi z / {n}), rho = 1, equilibrium",
            "l2": f"inputs larger than L2 ({2 * 19 * 4 * cells / 1e9:.2f} GB working set)",
            "bytes_per_update": 152}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    from paper_1309_1983_gb300 import workloads as W
    n = 64
    L = O.Lattice(n, n, n, TAU)
    f = O.to_aos(O.init_equilibrium(L, None, W.shear_wave(n, n, n, AMP)))
    f = O.run_aos(L, f, max(args.warmup, 1))
    t0 = time.perf_counter()
    O.run_aos(L, f, args.steps)  # all timed steps in one call of the oracle
    total = time.perf_counter() - t0
    mlups = n ** 3 * args.steps / total / 1e6
    sample = (f"FP64 oracle, one update of a periodic {n}^3 shear-wave lattice per step, "
              f"{args.steps} steps in one oracle call (bounded sample of the {args.n}^3 "
              f"workload; same per-node arithmetic)")
    # the config names the lattice actually timed, and the workload it samples
    config = dict(workload_config(n), sample_of=workload_config(args.n)["workload"])
    # the oracle keeps plain FP64 f in host memory (array of structures)
    config["storage"] = "f64 f_i (oracle, array of structures)"
    config["l2"] = (f"host run: {2 * 19 * 8 * n ** 3 / 1e9:.2f} GB of FP64 state in host memory "
                    "(no GPU cache involved)")
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": O.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def timed_steps(L, steps, torch):
    """Time ``steps`` single-update launches with CUDA events on the
    library's stream; returns (total ms, per-step ms list)."""
    s = L.stream
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(s)
    for k in range(steps):
        L.step(1)
        evs[k + 1].record(s)
    s.synchronize()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return evs[0].elapsed_time(evs[-1]), per


def extra_workloads(torch, n, steps=100, warmup=10):
    """Secondary workloads of the same hot path, each timed like the main
    one: the paper's lid-driven cavity (FP32 and 16-bit storage; halfway
    walls, and the on-site walls the paper used, at tau = 0.6 where they
    are stable), and the FP16 cavity on the tensor-copy staged kernel (a
    measured alternative to the default two-node kernel)."""
    from paper_1309_1983_gb300.lattice import Lattice
    from paper_1309_1983_gb300 import perfmodel as PM
    out = {}
    for name, storage, tau, onsite, kernel in (("cavity_f32", "f32", 0.55, False, None),
                                               ("cavity_f16", "f16", 0.55, False, None),
                                               ("cavity_bf16", "bf16", 0.55, False, None),
                                               ("cavity_onsite_f32", "f32", 0.6, True, None),
                                               ("cavity_onsite_f16", "f16", 0.6, True, None),
                                               ("cavity_f16_tma", "f16", 0.55, False, "tma")):
        L = Lattice(n, n, n, tau, walls=(True, True, True), lid=(0.05, 0.0, 0.0), storage=storage,
                    onsite=onsite)
        if kernel:
            L.set_kernel(kernel)
        L.init_equilibrium()
        L.step(warmup)
        ms, per = timed_steps(L, steps, torch)
        mlups = n ** 3 * steps / (ms / 1e3) / 1e6
        eb = 4 if storage == "f32" else 2
        out[name] = {"mlups": round(mlups, 1), "bytes_per_lu": PM.bytes_per_update(eb),
                     "gbs": round(PM.achieved_gbs(mlups, PM.bytes_per_update(eb)), 1),
                     "steps": steps, "kernel": kernel or "x2"}
        L.close()
        del L
        torch.cuda.empty_cache()
    return out


def paper_tables(torch, sizes=(64, 96, 128, 160, 192, 224, 256), steps=100):
    """The paper's throughput experiment (Sec. 6, Tables 1 and 2) on this
    GPU: the lid-driven cavity in FP32 (tau = 0.6, lid 0.05), 100 single
    launches per configuration, for cubic lattices of 64^3 to 256^3 and
    blocks of 32, 64, 128 and 256 threads along x with the one-node kernel
    (the paper's one node per thread), and the default two-node kernel;
    per-launch MLUPS as mean, standard deviation and best (the tables' style).
    The lattices up to 192^3 (0.8 GB per f copy and less) are partly
    resident in the 129 MB L2 only below 96^3."""
    import statistics
    from paper_1309_1983_gb300.lattice import Lattice
    out = {}
    for n in sizes:
        L = Lattice(n, n, n, 0.6, walls=(True, True, True), lid=(0.05, 0.0, 0.0))
        L.set_graph_steps(0)
        row = {}
        for name, kern, bx in (("node_32", "node", 32), ("node_64", "node", 64),
                               ("node_128", "node", 128), ("node_256", "node", 256),
                               ("x2", "x2", 0)):
            L.set_kernel(kern)
            if bx:
                L.set_block(bx, 1)
            L.init_equilibrium()
            L.step(5)
            _, per = timed_steps(L, steps, torch)
            m = [n ** 3 / (t / 1e3) / 1e6 for t in per]
            row[name] = {"mean": round(statistics.mean(m), 1), "sd": round(statistics.pstdev(m), 1),
                         "best": round(max(m), 1)}
        out[str(n)] = row
        L.close()
        del L
        torch.cuda.empty_cache()
    return out


def size_sweep(torch, sizes=(64, 128, 256), steps=1000):
    """The periodic shear-wave sweep: tau = 0.8, u_x = 0.01 sin(2 pi z/N)
    from equilibrium, FP32, `steps` single-update launches per size timed
    with CUDA events, then the same steps as one lbm_step call (CUDA-graph
    replay); the wave amplitude (projection of u_x on the initial
    sine) is sampled every steps/10 updates in an untimed second pass and
    its fitted decay rate compared with nu k^2 (Sec. 5 physics check at every
    size). 64^3 (20 MB per copy) stays resident in the 129 MB L2."""
    import numpy as np
    from paper_1309_1983_gb300.lattice import Lattice
    from paper_1309_1983_gb300 import workloads as W
    out = {}
    nu = (TAU - 0.5) / 3.0
    for n in sizes:
        L = Lattice(n, n, n, TAU)
        u0 = torch.from_numpy(W.shear_wave(n, n, n, AMP)).float().cuda()
        L.init_equilibrium(u=u0)
        L.step(10)
        ms, per = timed_steps(L, steps, torch)
        # the same steps as one call: replayed CUDA graphs of 32 launches
        L.step(64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(L.stream)
        L.step(steps)
        e1.record(L.stream)
        e1.synchronize()
        ms_call = e0.elapsed_time(e1)
        L.init_equilibrium(u=u0)
        sn = torch.sin(2 * np.pi * torch.arange(n, dtype=torch.float64) / n).cuda()
        t, A = [], []
        for k in range(11):
            _, u = L.moments()
            A.append(float((u[0].double().mean(dim=(1, 2)) * sn).sum() * 2 / n))
            t.append(k * (steps // 10))
            if k < 10:
                L.step(steps // 10)
        rate = -np.polyfit(np.array(t, dtype=np.float64), np.log(np.array(A)), 1)[0]
        kk = 2 * np.pi / n
        mlups = n ** 3 * steps / (ms / 1e3) / 1e6
        out[f"periodic_{n}"] = {
            "mlups": round(mlups, 1), "gbs": round(mlups * 152 / 1e3, 1),
            "one_call_graph_mlups": round(n ** 3 * steps / ms_call / 1e3, 1),
            "best_step_mlups": round(n ** 3 / (min(per) / 1e3) / 1e6, 1),
            "decay_rate_rel_err": float(rate / (nu * kk * kk) - 1.0),
            "l2_resident": 152 * n ** 3 < 129e6}
        L.close()
        del L, u0
        torch.cuda.empty_cache()
    return out


def capacity_workload(torch, n=1024, steps=20):
    """The largest cubic cavity the benchmark runs on one GPU: 1024^3 nodes,
    FP32, two f copies = 163 GB of the 288 GB HBM; `steps` single-update
    launches timed with CUDA events, and the FP64 mass before and after."""
    from paper_1309_1983_gb300.lattice import Lattice
    L = Lattice(n, n, n, 0.55, walls=(True, True, True), lid=(0.05, 0.0, 0.0))
    L.init_equilibrium()
    m0 = L.mass()
    L.step(3)
    ms, per = timed_steps(L, steps, torch)
    m1 = L.mass()
    mlups = n ** 3 * steps / (ms / 1e3) / 1e6
    out = {"config": f"cavity {n}^3 FP32 tau=0.55 lid 0.05", "f_bytes_total": 2 * L.layout.f_bytes,
           "mlups": round(mlups, 1), "gbs": round(mlups * 152 / 1e3, 1),
           "mass_rel_drift": abs(m1 - m0) / m0, "steps": steps}
    L.close()
    del L
    torch.cuda.empty_cache()
    return out


def streaming_ablation(torch, n, steps=50):
    """Sec. 4.3 redone on this GPU: streaming alone as an unshifted copy, a
    gather (misaligned reads; also with L2-only loads, no read-only cache)
    and a scatter (misaligned writes), and the full step in pull order
    (Alg. 3) and push order (Alg. 2); FP32, periodic."""
    from paper_1309_1983_gb300.lattice import Lattice
    L = Lattice(n, n, n, TAU)
    L.init_equilibrium()
    a, b = L.current_buffers()
    s = L.stream
    out = {}
    cases = (("copy", lambda x, y: L.streaming(x, y, "copy")),
             ("stream_gather", lambda x, y: L.streaming(x, y, "pull")),
             ("stream_gather_l2_only", lambda x, y: L.streaming(x, y, "pull_l2")),
             ("stream_scatter", lambda x, y: L.streaming(x, y, "push")),
             ("step_pull", lambda x, y: L.step_to(x, y)),
             ("step_push", lambda x, y: L.step_push(x, y)))
    for name, fn in cases:
        for _ in range(3):
            fn(a, b)
            a, b = b, a
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            fn(a, b)
            a, b = b, a
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"mlups": round(n ** 3 / ms / 1e3, 1),
                     "gbs": round(152 * n ** 3 / (ms / 1e3) / 1e9, 1)}
    L.close()
    del L
    torch.cuda.empty_cache()
    return out


def adjoint_workload(torch, n=128, T=500, K=50, tau=0.7):
    """Periodic 128^3, tau = 0.7, u0 and u_target random Fourier modes
    (|k| <= 4, amplitude 0.02, seeds 1 and 2), F = 0, T = 500, checkpoints
    every 50 steps: time of the forward (T steps) and of forward + backward,
    and the gradient's agreement with central differences of the loss."""
    from paper_1309_1983_gb300 import workloads as W
    from paper_1309_1983_gb300.adjoint import AdjointProblem
    P = AdjointProblem(n, n, n, tau, T=T, K=K)
    u0 = torch.from_numpy(W.fourier_modes(n, n, n, seed=1, amp=0.02)).float().cuda()
    ut = torch.from_numpy(W.fourier_modes(n, n, n, seed=2, amp=0.02)).float().cuda()
    F = torch.zeros((3, n, n, n), device="cuda")
    P.loss_and_grad(u0, F, ut)  # warm-up: allocates the checkpoint pool
    s = P.lat.stream
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(s)
    P.forward(u0, F)
    e[1].record(s)
    e[1].synchronize()
    e[2].record(s)
    loss, gu0, gF = P.loss_and_grad(u0, F, ut)
    e[3].record(s)
    e[3].synchronize()
    fwd = e[0].elapsed_time(e[1])
    both = e[2].elapsed_time(e[3])
    # accuracy at this size (untimed): directional derivatives of the GPU
    # gradient against central differences of the GPU forward loss, along a
    # third seeded Fourier field for u0 and for F
    d = torch.from_numpy(W.fourier_modes(n, n, n, seed=3, amp=0.02)).float().cuda()
    fd_err = {}
    for name, g, h, args in (("u0", gu0, 1e-2, lambda x: (u0 + x * d, F)),
                             ("F", gF, 1e-4, lambda x: (u0, F + x * d))):
        lp = P.loss(*args(h), ut).item()
        lm = P.loss(*args(-h), ut).item()
        fdv = (lp - lm) / (2 * h)
        adv = float((g.double() * d.double()).sum().item())
        fd_err[name] = abs(fdv - adv) / abs(fdv)
    cells = n ** 3
    out = {"config": f"periodic {n}^3 tau={tau} T={T} K={K}", "forward_ms": round(fwd, 2),
           "forward_backward_ms": round(both, 2), "ratio": round(both / fwd, 3),
           "forward_mlups": round(cells * T / (fwd / 1e3) / 1e6, 1),
           "reverse_step": "from stored collision moments" if P.moments else "re-gathering f^n",
           "loss": float(loss.item()),
           "grad_u0_norm": float(gu0.norm().item()), "grad_F_norm": float(gF.norm().item()),
           "directional_fd_rel_err": fd_err}
    del P
    torch.cuda.empty_cache()
    return out


def batch_workload(torch, steps=2000):
    """64 lid-driven cavities (seed 3: edges 16..96, tau in [0.55, 1], lid in
    [0.02, 0.08]), autotuned tiling, `steps` steps in one persistent
    graph-captured launch, against 64 separate single-lattice handles stepped
    one launch per domain and step."""
    from paper_1309_1983_gb300 import autotune, workloads as W
    from paper_1309_1983_gb300.batch import Batch
    from paper_1309_1983_gb300.lattice import Lattice
    G = W.batch_geometry(64, seed=3)
    B = Batch(G.dims, G.tau, G.lid_u)
    tiling = autotune.tune_batch(B, steps=50, cache_path=None)
    s = B.stream

    def dev_ms(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1)

    B.init_rest()
    B.step(steps)  # untimed: capture the graphs of a `steps`-step launch
    B.step(steps)  # from either buffer parity
    B.init_rest()
    ms = dev_ms(lambda: B.step(steps))  # replayed from a captured graph
    cells = int(G.dims.prod(axis=1).sum())
    info = B.info()
    # the same steps as one ordinary launch per step over the tile table
    B.step_launches(5)
    ms_launch = dev_ms(lambda: B.step_launches(200))
    B.close()
    lats = []
    for d in range(64):
        nx, ny, nz = (int(v) for v in G.dims[d])
        L = Lattice(nx, ny, nz, float(G.tau[d]), walls=(True, True, True),
                    lid=(float(G.lid_u[d]), 0.0, 0.0), stream=s)
        L.init_equilibrium()
        lats.append(L)
    sep_steps = 200
    for L in lats:
        L.step(2)

    def separate():
        for _ in range(sep_steps):
            for L in lats:
                L.step(1)
    ms_sep = dev_ms(separate)
    for L in lats:
        L.close()
    del lats
    torch.cuda.empty_cache()
    adj = batch_adjoint_workload(torch, G, steps, tiling=tiling[:2])
    return {"domains": 64, "cells": cells, "steps": steps, "forward_plus_adjoint": adj,
            "persistent_mlups": round(cells * steps / ms / 1e3, 1),
            "tile_launch_per_step_mlups": round(cells * 200 / ms_launch / 1e3, 1),
            "tuned_ms_per_step": round(tiling[2], 4),
            "separate_launches_mlups": round(cells * sep_steps / ms_sep / 1e3, 1),
            "tiling": {"threads": tiling[0], "blocks_per_sm": tiling[1]},
            "grid": info["grid"], "graph": info["graph"]}


def batch_adjoint_workload(torch, G, T, K=50, tiling=None):
    """Forward plus adjoint over the same 64 cavities: start at rest, T steps
    (checkpoints every K), loss against a seeded target velocity in every
    domain, gradients with respect to u0 and F (at F = 0). Every K-step
    forward segment, segment recompute and reverse sweep is one persistent
    launch (lbm_batch_run, lbm_batch_adjoint_run) with the forward's tiling."""
    from paper_1309_1983_gb300 import workloads as W
    from paper_1309_1983_gb300.adjoint import BatchAdjointProblem
    from paper_1309_1983_gb300.batch import Batch
    B = Batch(G.dims, G.tau, G.lid_u)
    if tiling:
        B.set_tiling(*tiling)
    P = BatchAdjointProblem(B, T, K)
    ut = B.pack_vectors([W.separable_modes(int(d[0]), int(d[1]), int(d[2]), seed=2 + k,
                                           amp=0.02)
                         for k, d in enumerate(G.dims)])
    u0 = torch.zeros_like(ut)
    F = torch.zeros_like(ut)
    P.loss_and_grad(u0, F, ut)  # warm-up: allocates checkpoints and segment buffers
    s = B.stream
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(s)
    P.forward(u0, F)
    e[1].record(s)
    e[1].synchronize()
    e[2].record(s)
    loss, gu0, gF = P.loss_and_grad(u0, F, ut)
    e[3].record(s)
    e[3].synchronize()
    fwd, both = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    cells = int(G.dims.prod(axis=1).sum())
    out = {"T": T, "K": K, "forward_ms": round(fwd, 1), "forward_backward_ms": round(both, 1),
           "ratio": round(both / fwd, 3), "forward_mlups": round(cells * T / (fwd / 1e3) / 1e6, 1),
           "loss": float(loss.item()), "grad_u0_norm": float(gu0.norm().item()),
           "grad_F_norm": float(gF.norm().item())}
    del P, B
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1309_1983_gb300 import build as B
    B.build()
    from paper_1309_1983_gb300 import capi, perfmodel as PM, workloads as W
    from paper_1309_1983_gb300.lattice import Lattice
    capi.load()

    n = args.n
    cells = n ** 3
    if args.geometry == "cavity":
        L = Lattice(n, n, n, 0.55, walls=(True, True, True), lid=(0.05, 0.0, 0.0),
                    storage=args.storage)
    else:
        L = Lattice(n, n, n, TAU, storage=args.storage)
    u0 = torch.from_numpy(W.shear_wave(n, n, n, AMP)).float().cuda()
    L.init_equilibrium(u=u0 if args.geometry == "periodic" else None)
    L.step(max(args.warmup, 3))
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    uuid = None
    try:
        uuid = "GPU-" + str(props.uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, per = timed_steps(L, args.steps, torch)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None

    ms_max, value = aggregate_replicas(ms, cells, args.steps, ws, dist, "cuda")
    per_rank_mlups = cells * args.steps / (ms / 1e3) / 1e6
    step_ms = ms / args.steps
    mlups_each = [cells / (p / 1e3) / 1e6 for p in per]

    # physics sanity on the benchmarked state: mass is conserved
    mass = L.mass()
    mass_rel = abs(mass / cells - 1.0)

    # roofline of the dominant (only) kernel
    bpl = PM.bytes_per_update(4 if args.storage == "f32" else 2)
    peak, peak_kind = measured_hbm()
    achieved = bpl * cells / (step_ms / 1e3) / 1e9
    default_run = n == 384 and args.storage == "f32" and args.geometry == "periodic"
    traffic = ncu_traffic("launches_bench_periodic_384.txt") if default_run else None

    # end to end through the C ABI on host buffers
    u0_h = torch.from_numpy(W.shear_wave(n, n, n, AMP)).float().pin_memory()
    rho_h = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    u_h = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    L.run_host(u0_h, 1, rho_h, u_h)  # warm
    e2e_t = []
    for _ in range(args.e2e_calls):
        t0 = time.perf_counter()
        L.run_host(u0_h, 1, rho_h, u_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e_mlups = cells / statistics.median(e2e_t) / 1e6

    extras = None
    if rank == 0 and not args.no_extras:
        L.close()
        del L, u0
        torch.cuda.empty_cache()
        want = set(args.extras.split(",")) if args.extras != "all" else {
            "storage", "streaming", "adjoint", "batched", "sweep", "tables"}
        extras = {}
        if "sweep" in want:
            extras["sweep"] = size_sweep(torch)
        if "capacity" in want:  # opt-in: 163 GB on the device
            extras["capacity"] = capacity_workload(torch)
        if "tables" in want:  # the paper's Tables 1-2 experiment
            extras["tables"] = paper_tables(torch)
        if "storage" in want:
            extras.update(extra_workloads(torch, n))
        if "streaming" in want:
            extras["streaming"] = streaming_ablation(torch, n)
        if "adjoint" in want:
            extras["adjoint"] = adjoint_workload(torch, n=args.adj_n, T=args.adj_steps)
        if "batched" in want:
            extras["batched"] = batch_workload(torch, steps=args.batch_steps)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    cpu = None
    if ws == 1:
        cm, cores, cdt, cdone = cpu_baseline(args.cpu_sample_n, args.cpu_sample_steps,
                                             args.cpu_sample_seconds)
        cpu = {"value": round(cm, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": (f"FP64 oracle, periodic {args.cpu_sample_n}^3 shear wave, "
                          f"{cdone} updates ({cdt:.1f} s), same per-node "
                          f"arithmetic as the {n}^3 workload")}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(n),
        "parallelism": "replicas" if ws > 1 else "single GPU",
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "kernel": "k_step_x2<f32, periodic> (two nodes per thread)",
                     "algorithmic_bytes_per_launch": bpl * cells},
        "e2e": {"value": round(e2e_mlups, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": 3 * 4 * cells, "d2h_bytes_per_step": 4 * 4 * cells,
                "call": "lbm_run_host(u0 host -> init -> 1 update -> rho,u host)"},
        "gpu_launches": args.steps,
        "per_step_mlups": {"mean": round(statistics.mean(mlups_each), 1),
                           "stdev": round(statistics.pstdev(mlups_each), 1),
                           "best": round(max(mlups_each), 1)},
        "step_time_spectrum": dict(zip(("peak_hz", "peak_amplitude_ms", "resolution_hz"),
                                       PM.step_time_spectrum(per))),
        "per_rank_mlups": round(per_rank_mlups, 1),
        "mass_rel_drift": mass_rel,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "extras": extras,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
