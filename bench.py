#!/usr/bin/env python
"""Benchmark: KKT solves/s to relative residual 1e-8 for the unsteady Stokes
control problem (Q2-Q1, 64x64 elements, n_t = 256 time blocks on T = 1,
beta in {1e-2, 1e-4, 1e-6}, seeded divergence-free desired state), with the
FP32 parallel-in-time preconditioner inside FP64 FGMRES(30); the plain FP64
preconditioner is timed beside it.

One step = the three problems (one per beta) solved concurrently to 1e-8
(right-hand sides resident, x0 = 0), one host thread and CUDA stream each,
their handles in one group (pint_group_*): each keeps its outer FGMRES, KKT
matvecs and time DFTs, and the frequency solves of their preconditioner
applies (Stokes transforms, batched inner GMRES with multigrid / Chebyshev
commutator preconditioning) run in shared launches over the frequencies of
all three.  value = solves / second over the timed steps; every result is bit
for bit the one of the problem solved alone (checked in the line), and the
line also reports the problems solved alone one after the other.  Inputs are
larger than L2 (the FP64 FGMRES bases alone are 28 GB), so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: replicas only (each rank solves its own problems; no collective
on the data path), launched by torch.distributed.run.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # configs: Stokes control, 64x64 Q2-Q1 grid, n_t = 256, T = 1
    "stokes64_nt256": dict(kind=0, level=6, K=256, T=1.0, betas=[1e-2, 1e-4, 1e-6], nu=1e-2, x0=0.0, x1=1.0,
                           wind=0),
    # same grid with n_t = 32: a shorter run of the same kernels, for profiling
    "stokes64_nt32": dict(kind=0, level=6, K=32, T=1.0, betas=[1e-4], nu=1e-2, x0=0.0, x1=1.0, wind=0),
    # small case the oracle solves in seconds (8x8 grid, n_t = 8)
    "stokes8_nt8": dict(kind=0, level=3, K=8, T=1.0, betas=[1e-2], nu=1e-2, x0=0.0, x1=1.0, wind=0),
    # Oseen control, 128x128 Q2-Q1 on [-1,1]^2, n_t = 128, nu = 1/100, recirculating wind,
    # time DFT as a 3xTF32 tensor-core contraction
    "oseen128_nt128": dict(kind=1, level=7, K=128, T=1.0, betas=[1e-4], nu=1e-2, x0=-1.0, x1=1.0, wind=1,
                           dft_mode=3, inner_maxit=40),
    # large Oseen control, 256x256, n_t = 128, nu = 1/500, beta = 1e-6, FGMRES(20)
    # (inner GMRES capped at 40 iterations: the Uzawa-preconditioned blocks need a few)
    "oseen256_nt128": dict(kind=1, level=8, K=128, T=1.0, betas=[1e-6], nu=2e-3, x0=-1.0, x1=1.0, wind=1,
                           restart=20, inner_maxit=40),
}
# FGMRES iterations per solve measured on the GB300 (FP64 and FP32 preconditioner
# agree) for the middle beta of each workload; used to extrapolate the oracle's
# per-block time to a whole solve in the reference arm.
OUTER_ITS_MEASURED = {"stokes64_nt256": 20, "stokes64_nt32": 21, "stokes8_nt8": 14}
METRIC = "KKT solves/s to rel-res 1e-8 (FP32 precond vs FP64 plain); p50/p99 latency"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stokes64_nt256", choices=list(WORKLOADS) + ["serve"],
                    help="'serve': the serving stream (pint_server_*), see --requests/--rate")
    ap.add_argument("--requests", type=int, default=16, help="serve: number of requests in the stream")
    ap.add_argument("--rate", type=float, default=1.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--slots", type=int, default=8, help="serve: worker slots of the server")
    ap.add_argument("--serve-prec", type=int, default=1, choices=[0, 1], help="serve: 1 = FP32 preconditioner")
    ap.add_argument("--share", type=int, default=1, choices=[0, 1],
                    help="serve: 1 = batch the frequency solves of the requests on the GPU in shared launches")
    ap.add_argument("--max-level", type=int, default=7, help="serve: largest grid level drawn (7 = 128x128)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp64-budget-s", type=float, default=120.0,
                    help="wall-clock budget for the FP64-plain comparison solves")
    ap.add_argument("--cpu-sample-s", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inner-maxit", type=int, default=100,
                    help="inner GMRES iteration cap (sizes the inner Krylov basis)")
    ap.add_argument("--only-timed", action="store_true",
                    help="run the warm-up and timed solves only (for profiler captures)")
    ap.add_argument("--beta", type=float, default=None,
                    help="solve for this one beta only (profiler captures: one handle on the device)")
    ap.add_argument("--outer-restart", type=int, default=None,
                    help="FGMRES restart length; smaller values shrink the device footprint for profiler "
                         "captures (the reported metric uses 30)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
class Clocks:
    """nvidia-smi sampler run during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def profiled_traffic(summary, source):
    """DRAM bytes per launch (dram__bytes_read + dram__bytes_write) from a
    committed ncu summary, or None once the kernel source has changed since
    the counters were taken.  The summary records the SHA-1 of the source
    file, or, with a `kernel_source_end:` line, of the file's text before that
    line (the part holding the kernel and everything it calls)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2405_18964_gb300", "csrc", source)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None
    keys = ("kernel_source_sha1:", "kernel_source_end:", "traffic_bytes")
    fields = dict(ln.rstrip("\n").split(":", 1) for ln in open(path) if ln.startswith(keys))
    sha = fields.get("kernel_source_sha1", "").split()[0:1]
    text = open(src, "rb").read()
    end = fields.get("kernel_source_end", "").strip()
    if end:
        i = text.find(end.encode())
        if i < 0:
            return None
        text = text[:i]
    if not sha or sha[0] != hashlib.sha1(text).hexdigest():
        return None
    return int(fields["traffic_bytes_per_launch"].strip())


def peaks_bf16():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops_sustained", 1700.0), "measured (sustained)"
    return 1700.0, "fallback (sustained)"


def dft_report(sizes, dft, bf16_peak, mode=0):
    """Time DFT of the FP32 preconditioner (tcgen05 for n_t <= 256:
    split-BF16 x6 by default, 3xTF32 with mode 3): algorithmic bytes (FP64
    time slices in, complex FP32 Hermitian half out, or the reverse) and
    tensor flops as issued (six, or three, 128 x npad x 32 MMA products per
    tile and reduction chunk).  The TF32 fraction is of half the BF16 peak
    (the dense TF32 rate is half the BF16 rate)."""
    K, J, nblk = sizes.n_t, sizes.J, sizes.n_blk
    npad = (K + 15) // 16 * 16
    tiles = (nblk + 127) // 128
    red = {"dft_fwd": (K + 31) // 32 * 32, "dft_inv": (2 * J + 31) // 32 * 32}
    nbytes = K * nblk * 8 + J * nblk * 8
    tf32 = mode == 3
    nprod = 3 if tf32 else 6
    peak = bf16_peak[0] / 2 if tf32 else bf16_peak[0]
    out = {"mode": ("tf32x3 tcgen05" if tf32 else "bf16x6 tcgen05") if K <= 256 else "simt",
           "bytes_per_launch": nbytes}
    for d, c in dft.items():
        if not c["timed"]:
            continue
        ms = c["ms"] / c["timed"]
        fl = nprod * 2 * 128 * npad * red[d] * tiles
        out[d] = {"avg_ms": round(ms, 4), "GBps": round(nbytes / (ms / 1e3) / 1e9, 1),
                  "tensor_tflops_issued": round(fl / (ms / 1e3) / 1e12, 1),
                  "tensor_frac_of_peak": round(fl / (ms / 1e3) / 1e12 / peak, 4)}
    out["peak_tflops"] = peak
    out["peak_source"] = bf16_peak[1] + (" BF16 rate / 2 for TF32" if tf32 else "")
    return out


def dist_init(backend="nccl"):
    """Replicas: one process per GPU under torch.distributed.run; the only
    collectives are the barrier around the timed region and the max over
    ranks of its duration (no collective on the data path)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    if backend == "nccl":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
    dist.init_process_group(backend, init_method="env://")
    return rank, ws, dist


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over all ranks (the job's timed duration)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank, count):
    """Data seeds of one replica's problems: distinct across ranks."""
    return [1000 * rank + i for i in range(count)]


def whole_job_rate(steps, world_size, max_ms):
    """Units all ranks processed divided by the slowest rank's time."""
    return steps * world_size / (max_ms / 1e3)


def workload_config(name, ws):
    """The `config` object of a bench line (both arms report the same one)."""
    W = WORKLOADS[name]
    N = 2 ** W["level"]
    m = W.get("restart", 30)
    basis = (2 * m + 1) * W["K"] * (4 * (2 * N + 1) ** 2 + 2 * (N + 1) ** 2) * 8
    l2 = (f"inputs larger than L2 (FP64 FGMRES basis {basis / 1e9:.1f} GB)" if basis > 129e6 else
          "inputs smaller than L2 (small parity case)")
    return {"workload": name, "kind": "oseen" if W["kind"] else "stokes", "grid": f"{N}x{N} Q2-Q1",
            "n_t": W["K"], "T": W["T"], "betas": W["betas"], "nu": W["nu"],
            "outer": f"FGMRES({m}), tol 1e-8", "inner_tol": 1e-2, "l2": l2, "parallelism": f"replicas x{ws}"}


def apply_roofline(cls, hbm, src):
    """Preconditioner applies against HBM: the algorithmic bytes of every
    kernel of the applies (the library's per-launch counts, pint.h
    pint_profile) over the event time of the shared frequency-solve batches
    (events on the group's stream around each batch; the pressure part's
    second stream joins inside it).  The time DFTs (0.5% of the launch time)
    run on the problems' own streams and count bytes but no time here."""
    from paper_2405_18964_gb300 import binding
    ap = cls["apply"]
    if not ap["timed"] or ap["ms"] <= 0:
        return None
    b = sum(cls[c]["bytes"] for c in binding.APPLY_CLASSES)
    gbs = b / (ap["ms"] / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "peak_source": src, "unit": "GB/s",
            "frac": round(gbs / hbm, 4), "applies": ap["timed"], "algorithmic_bytes": b,
            "event_ms": round(ap["ms"], 3),
            "bytes_by_class": {c: cls[c]["bytes"] for c in binding.APPLY_CLASSES if cls[c]["bytes"]}}


def algorithmic_bytes_mg_q2(sizes, nlaunch_jobs, cycles, bw):
    """Per-unit figure for one V-cycle on one complex Q2 field with 2+2
    sweeps: 24 n c b_w bytes (n nodes, c = 2, b_w bytes per word)."""
    return 24.0 * sizes.n_s * 2 * bw * cycles * nlaunch_jobs


# ------------------------------------------------------------- our arm
def run_ours(a):
    """One step = the workload's problems (one per beta) solved concurrently,
    one host thread and CUDA stream each, their handles in one group so that
    their frequency solves run in shared launches (pint_group_*)."""
    import threading

    import torch
    from paper_2405_18964_gb300 import binding, inputs

    rank, ws, dist = dist_init()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    W = WORKLOADS[a.workload]
    K, T = W["K"], W["T"]
    tau = T / (K + 1)
    N = 2 ** W["level"]

    def params(beta, prec):
        return binding.default_params(kind=W["kind"], level=W["level"], n_t=K, tau=tau, beta=beta, nu=W["nu"],
                                      x0=W["x0"], x1=W["x1"], wind=W["wind"], prec=prec,
                                      inner_maxit=W.get("inner_maxit", a.inner_maxit),
                                      outer_restart=a.outer_restart or W.get("restart", 30),
                                      dft_mode=W.get("dft_mode", 0) if prec else 0)

    betas = W["betas"] if a.beta is None else [a.beta]
    seeds = replica_seeds(rank, len(betas))
    vds = [inputs.desired_state(N, W["x0"], W["x1"], K, tau, T, sd) for sd in seeds]
    group = binding.Group()
    streams = [torch.cuda.Stream() for _ in betas]
    probs = []
    for b, vd, st in zip(betas, vds, streams):
        G = binding.Problem(params(b, 1), stream=st.cuda_stream, group=group)
        G.set_data(vd)
        probs.append(G)
    n = probs[0].kkt_len
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in probs]

    def concurrently(fn):
        """fn(k) for every problem, one host thread each; returns results and
        each call's wall time (ms)."""
        out, lat = [None] * len(probs), [0.0] * len(probs)

        def run(k):
            t0 = time.perf_counter()
            out[k] = fn(k)
            lat[k] = (time.perf_counter() - t0) * 1e3

        th = [threading.Thread(target=run, args=(k,)) for k in range(len(probs))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        return out, lat

    def solve_device(k):
        with torch.cuda.stream(streams[k]):
            xs[k].zero_()
        # profiler captures (--only-timed with a shrunken basis) may stop before 1e-8
        return probs[k].solve(xs[k], check=not a.only_timed)

    def step():
        return concurrently(solve_device)

    for i in range(a.warmup):
        step()
    torch.cuda.synchronize()
    # ---- timed region (device-resident inputs)
    group.profile_enable(["mg_q2", "apply"])
    for G in probs:
        G.profile_enable(["dft_fwd", "dft_inv"])
    clk = Clocks(dev)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s0 = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev[0].record(s0)
    infos, lat = [], []
    for i in range(a.steps):
        inf, lt = step()
        torch.cuda.synchronize()
        ev[i + 1].record(s0)
        infos += inf
        lat += lt
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, dist)
    gprof = group.profile_read()
    mprof = [G.profile_read() for G in probs]
    keys = ("launches", "timed", "ms", "bytes")
    cls = {c: {k: gprof[c][k] + sum(p[c][k] for p in mprof) for k in keys} for c in binding.PROF_CLASSES}
    cls["apply"] = gprof["apply"]  # whole batches of shared frequency solves
    mg = cls["mg_q2"]
    dft = {d: cls[d] for d in ("dft_fwd", "dft_inv")}
    launches = sum(c["launches"] for c in cls.values())
    solves = a.steps * len(probs)
    value = solves * ws / (total_ms / 1e3)
    gstats = group.stats()
    if a.only_timed:
        if rank == 0:
            hbm, src = peaks()
            mg_gbs = mg["bytes"] / (mg["ms"] / 1e3) / 1e9 if mg["ms"] > 0 else None
            print(json.dumps({"value": value, "unit": UNIT, "ms_per_step": total_ms / a.steps,
                              "outer_iterations": [inf.outer_iterations for inf in infos],
                              "gpu_launches": int(launches),
                              "mg_q2_avg_launch_ms": mg["ms"] / max(1, mg["timed"]),
                              "mg_q2_GBps": mg_gbs, "mg_q2_frac": mg_gbs / hbm if mg_gbs else None,
                              "apply": apply_roofline(cls, hbm, src), "shared": gstats,
                              "autotune": binding.autotune_report().strip().splitlines(),
                              "dft_avg_ms": {d: c["ms"] / max(1, c["timed"]) for d, c in dft.items()}}), flush=True)
        for G in probs:
            G.close()
        group.close()
        return

    # ---- per-class shares from one fully profiled step (outside the timed region)
    group.profile_enable(binding.PROF_CLASSES)
    for G in probs:
        G.profile_enable(binding.PROF_CLASSES)
    step()
    g2 = group.profile_read()
    m2 = [G.profile_read() for G in probs]
    share = {c: g2[c]["ms"] + sum(p[c]["ms"] for p in m2) for c in binding.PROF_CLASSES}
    share_launch = {c: g2[c]["launches"] + sum(p[c]["launches"] for p in m2) for c in binding.PROF_CLASSES}
    share_bytes = {c: g2[c]["bytes"] + sum(p[c]["bytes"] for p in m2) for c in binding.PROF_CLASSES}
    hbm_p, src_p = peaks()
    # per-class algorithmic bytes over the class's summed event time in this
    # profiled step (every launch timed)
    class_roofline = {}
    for c in ("mg_q2", "mg_q1", "cheb", "block_mv", "combo", "inner", "kkt_mv", "outer"):
        if share[c] > 0 and share_bytes[c] > 0:
            gbs = share_bytes[c] / (share[c] / 1e3) / 1e9
            class_roofline[c] = {"GBps": round(gbs, 1), "frac": round(gbs / hbm_p, 4), "launches": int(share_launch[c])}
    class_roofline["peak"] = hbm_p
    class_roofline["peak_source"] = src_p
    class_roofline["note"] = ("event times of launches that share the GPU with the other stream: the pressure part "
                              "(mg_q1, cheb) runs beside the velocity multigrid and its launches wait for SMs held "
                              "by it, so their fractions are lower bounds; serialised times are in profiles/")
    inner_loop = {"host_syncs_per_solve": round((g2["host_syncs"] + sum(p["host_syncs"] for p in m2)) / len(probs), 1),
                  "gpu_launches_per_solve": round(sum(share_launch.values()) / len(probs), 1),
                  "note": "one host synchronisation per inner GMRES step of a shared batch (the host reads how many "
                          "frequencies are still active), two per outer FGMRES step of each problem"}
    tot = sum(v for k, v in share.items() if k != "apply") or 1.0
    shares = {k: round(v / tot, 4) for k, v in share.items() if share_launch[k] and k != "apply"}
    shares["note"] = ("shares of the summed per-launch event times of one profiled step; the pressure part "
                      "runs on a second stream and the problems' outer steps on their own streams, so the "
                      "summed times exceed the wall time")
    group.profile_enable([])
    for G in probs:
        G.profile_enable([])

    # ---- e2e through the public API with host buffers (pinned): data upload,
    # solve from a host initial guess, solution download, all problems at once
    vd_pinned = [torch.from_numpy(vd).pin_memory() for vd in vds]
    xh = [torch.zeros(n, dtype=torch.float64).pin_memory() for _ in probs]

    def solve_host(k):
        probs[k].set_data(vd_pinned[k].numpy())
        xnp = xh[k].numpy()
        xnp[:] = 0.0
        return probs[k].solve_host(xnp)

    e2e_steps = min(a.steps, 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        concurrently(solve_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = int(sum(v.numel() for v in vd_pinned) * 8 + len(probs) * n * 8)
    d2h = int(len(probs) * n * 8)
    e2e = {"value": e2e_steps * len(probs) * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps}
    xg = [x.clone() for x in xs]  # the grouped FP32 solutions of the last timed step
    for G in probs:
        G.close()
    group.close()

    # ---- each problem alone (ordinary handle, sequential), FP32 and FP64 plain
    alone = {"fp32_ms": [], "fp32_outer_iterations": [], "bitwise_equal_to_grouped": []}
    fp64 = {"solves": 0, "ms": 0.0}
    errs, its64 = [], []
    t_start = time.perf_counter()
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    st0 = torch.cuda.current_stream()
    for k, b in enumerate(betas):
        for prec in (1, 0):
            if prec == 0 and (a.fp64_budget_s <= 0 or time.perf_counter() - t_start > a.fp64_budget_s):
                continue
            G = binding.Problem(params(b, prec), stream=st0.cuda_stream)
            G.set_data(vds[k])
            x1.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st0)
            inf = G.solve(x1)
            e1.record(st0)
            torch.cuda.synchronize()
            G.close()
            if prec:
                alone["fp32_ms"].append(round(e0.elapsed_time(e1), 1))
                alone["fp32_outer_iterations"].append(inf.outer_iterations)
                alone["bitwise_equal_to_grouped"].append(bool(torch.equal(x1, xg[k])))
            else:
                fp64["solves"] += 1
                fp64["ms"] += e0.elapsed_time(e1)
                its64.append(inf.outer_iterations)
                errs.append(float(torch.linalg.norm(xg[k] - x1) / torch.linalg.norm(x1)))
    fp64_value = fp64["solves"] / (fp64["ms"] / 1e3) if fp64["solves"] else None
    alone["value"] = round(len(alone["fp32_ms"]) / (sum(alone["fp32_ms"]) / 1e3), 4)
    alone["note"] = "each problem solved alone on an ordinary handle, one after the other"

    # ---- roofline of the dominant kernel (multigrid on the velocity fields):
    # the library's algorithmic bytes of every launch (only the fields of
    # frequencies still active are counted) over the launches' event time
    hbm, src = peaks()
    avg_ms = mg["ms"] / max(1, mg["timed"])
    alg = mg["bytes"] / max(1, mg["launches"])
    achieved = mg["bytes"] / (mg["ms"] / 1e3) / 1e9 if mg["timed"] == mg["launches"] and mg["ms"] > 0 else None
    apply_line = apply_roofline(cls, hbm, src)
    traffic = None
    if a.workload == "stokes64_nt256":
        full = profiled_traffic("mg_q2p_kernel_stokes64_nt256.md", "k_mgp.cu")
        if full:
            # captured on a full launch (every field active): scaled to the average launch by its fields
            sz = probs[0].sizes
            traffic = int(full * alg / algorithmic_bytes_mg_q2(sz, 4 * sz.J, 4, 4))
    dft_line = dft_report(probs[0].sizes, dft, peaks_bf16(), W.get("dft_mode", 0))

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(total_ms / a.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 preconditioner / f64 FGMRES",
        "data": "synthetic (seeded curl of 4 random sine modes)",
        "config": dict(workload_config(a.workload, ws),
                       step=f"the {len(probs)} problems (one per beta) solved concurrently, one host thread and "
                            "stream each, frequency solves shared in one group"),
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3)},
        "outer_iterations": [inf.outer_iterations for inf in infos],
        "relres": [inf.relres for inf in infos],
        "shared": gstats,
        "alone_fp32": alone,
        "fp64_plain": {"value": round(fp64_value, 5) if fp64_value else None, "unit": UNIT,
                       "solves": fp64["solves"], "outer_iterations": its64,
                       "speedup_fp32_over_fp64": round(value / fp64_value, 2) if fp64_value else None,
                       "speedup_fp32_alone_over_fp64": round(alone["value"] / fp64_value, 2) if fp64_value else None,
                       "betas": betas[:len(its64)], "fp32_outer_iterations": alone["fp32_outer_iterations"],
                       "fp32_vs_fp64_solution_relerr": errs},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "kernel_time_share": shares,
        "class_roofline": class_roofline,
        "inner_loop": inner_loop,
        "roofline": {"kernel": (f"mg_q2p_kernel<float, {N}> (multigrid W_j, 4 V-cycles, 4 fields x all active "
                                "frequencies of the batch)" if W["kind"] == 0 else
                                "mg_q2b_kernel<float, conv> (multigrids of Q_j and Q_j^H, 4 V-cycles, 2 fields each "
                                "x all active frequencies of the batch)"),
                     "bound": "hbm", "achieved": round(achieved, 1) if achieved else None,
                     "peak": hbm, "peak_source": src, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4) if achieved else None, "traffic": traffic,
                     "avg_launch_ms": round(avg_ms, 4), "timed_launches": mg["timed"],
                     "algorithmic_bytes_per_launch": round(alg), "algorithmic_bytes_total": mg["bytes"],
                     "event_ms_total": round(mg["ms"], 3), "apply": apply_line},
        "dft": dft_line,
        "autotune": binding.autotune_report().strip().splitlines(),
        "clocks": clocks,
    }
    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W, a.cpu_sample_s, [inf.outer_iterations for inf in infos])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------- serving stream
def serve_requests(seed, count, max_level):
    """The serving stream's requests, drawn from default_rng(seed) in this
    order per request: kind 50/50; N in {16, 32, 64, 128} (levels 4..7, capped
    at max_level); n_t in
    {16, 32, 64, 128, 256}; log10 beta ~ U[-6, -2]; nu in {1/50, 1/100} for
    Oseen (1e-2 for Stokes); a data seed.  Oseen requests with beta > 1e-4
    damp the SOR of their convection multigrids (sor_omega_conv = 0.5: with
    omega = 1 the multigrid of the convection-dominated low-frequency Q_j
    diverges there)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        oseen = bool(rng.integers(0, 2))
        level = int(rng.choice([4, 5, 6, 7]))
        K = int(rng.choice([16, 32, 64, 128, 256]))
        beta = float(10.0 ** rng.uniform(-6.0, -2.0))
        nu = float(rng.choice([1 / 50, 1 / 100])) if oseen else 1e-2
        dseed = int(rng.integers(0, 2 ** 31))
        omega_conv = 0.0
        if oseen:
            omega_conv = 0.5 if beta > 1e-4 else 0.0
        out.append(dict(oseen=oseen, level=min(level, max_level), K=K, beta=beta, nu=nu, seed=dseed,
                        omega_conv=omega_conv))
    return out


def run_serve(a):
    """Serving stream through pint_server_*: Poisson arrivals, continuous
    admission by device memory; throughput and latency percentiles."""
    import torch
    from paper_2405_18964_gb300 import binding, inputs
    reqs = serve_requests(a.seed, a.requests, a.max_level)
    arr = np.cumsum(np.random.default_rng(a.seed + 1).exponential(1.0 / a.rate, size=len(reqs)))
    built = []
    for r in reqs:
        x0, x1 = (-1.0, 1.0) if r["oseen"] else (0.0, 1.0)
        tau = 1.0 / (r["K"] + 1)
        p = binding.default_params(kind=int(r["oseen"]), level=r["level"], n_t=r["K"], tau=tau, beta=r["beta"],
                                   nu=r["nu"], x0=x0, x1=x1, wind=int(r["oseen"]), prec=a.serve_prec,
                                   sor_omega_conv=r["omega_conv"])
        vd = inputs.desired_state(2 ** r["level"], x0, x1, r["K"], tau, 1.0, seed=r["seed"])
        n = r["K"] * (4 * (2 ** (r["level"] + 1) + 1) ** 2 + 2 * (2 ** r["level"] + 1) ** 2)
        built.append((p, vd, n))
    torch.cuda.synchronize()
    srv = binding.Server(max_active=a.slots, share_solves=bool(a.share))
    clk = Clocks(0)
    clk.start()
    t0 = time.perf_counter()
    ids = []
    for (p, vd, _), ta in zip(built, arr):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(p, vd))
    lat, its, fails = [], [], 0
    for rid, (_, _, n) in zip(ids, built):
        _, info, ms, code = srv.wait(rid, n, check=False)
        lat.append(ms)
        its.append(info.outer_iterations)
        fails += code != 0
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    line = {"metric": "serving stream: solves/s and p50/p99 latency (FP32 precond)" if a.serve_prec else
            "serving stream: solves/s and p50/p99 latency (FP64 precond)",
            "value": round(len(ids) / wall, 4), "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 1),
                           "p99": round(float(np.percentile(lat, 99)), 1)},
            "requests": len(ids), "failed": fails, "arrival_rate": a.rate, "slots": a.slots,
            "shared_solves": {"on": bool(a.share), "batches": st["shared_batches"],
                              "member_applies": st["shared_member_solves"],
                              "frequencies": st["shared_frequencies"], "largest_batch": st["shared_max_members"]},
            "active_peak": st["active_peak"], "bytes_peak": st["bytes_peak"], "budget_bytes": st["budget_bytes"],
            "outer_iterations": its, "wall_s": round(wall, 2),
            "config": {"workload": "serve", "seed": a.seed, "max_level": a.max_level,
                       "requests": [{k: (round(v, 8) if isinstance(v, float) else v) for k, v in r.items()}
                                    for r in reqs]},
            "data": "synthetic (seeded)", "clocks": clocks}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- oracle timing
_ORACLE_CACHE = {}


def _oracle_block_task(task):
    """One frequency-block solve of the FP64 oracle (Algorithm 2: inner GMRES
    to 1e-2 with the multigrid / Chebyshev commutator preconditioner) in a
    pool worker.  The problem and block j's multigrid hierarchy are built
    before the clock starts; only the solve is timed."""
    (kind, level, K, tau, beta, nu, x0, x1, wind), j, seed = task
    from oracle import inexact, kkt
    key = (kind, level, K, tau, beta, nu, x0, x1, wind)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE.clear()
        P = kkt.Problem(kind, level, K, tau, beta, nu, x0, x1, wind)
        _ORACLE_CACHE[key] = (P, inexact.PinTPreconditioner(P))
    P, pc = _ORACLE_CACHE[key]
    nn = 2 * (2 * len(P.vi)) + 2 * len(P.pf)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(nn) + 1j * rng.standard_normal(nn)
    pc.block_prec(j)
    t0 = time.perf_counter()
    pc.solve_block(j, g)
    return j, time.perf_counter() - t0, int(pc.inner_its[j])


class OraclePool:
    """The oracle's frequency-block solves spread over the host cores by a
    process pool, one block per core at a time, as the paper distributes its
    frequency blocks over processes.  Started with `spawn` (this process has
    used the GPU); BLAS/OpenMP threads are pinned to one per worker."""

    def __init__(self, W):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.cores = len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        K, T = W["K"], W["T"]
        self.beta = W["betas"][len(W["betas"]) // 2]
        kind = "oseen" if W["kind"] else "stokes"
        wind = "recirc" if W["wind"] == 1 else None
        self.cfg = (kind, W["level"], K, T / (K + 1), self.beta, W["nu"], W["x0"], W["x1"], wind)
        self.K, self.J = K, K // 2 + 1

    def sample(self, r):
        """Round r's frequencies: one per core, evenly spread over 0..J-1
        (j = 0, the hardest block, in every round), shifted by r."""
        c = min(self.cores, self.J)
        return sorted({0} | {(round(i * (self.J - 1) / max(1, c - 1)) + r) % self.J for i in range(1, c)})

    def round(self, r):
        js = self.sample(r)
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_block_task, [(self.cfg, j, 1000 + j) for j in js], chunksize=1)
        return out, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()

    def estimate(self, results, outer_its):
        """Seconds per solve: the mean block time over the sample times the
        blocks each core solves in an apply (the K / 2 + 1 blocks of the
        half spectrum dealt out to the cores), times the outer iterations
        (one apply each)."""
        import math
        per_block = float(np.mean([t for _, t, _ in results]))
        apply_s = per_block * math.ceil(self.J / self.cores)
        return outer_its * apply_s, per_block, apply_s


def cpu_baseline(W, budget_s, outer_its):
    """The FP64 oracle's nested solver timed on the host cores on a bounded
    sample (rounds of one frequency-block solve per core), extrapolated to a
    whole solve."""
    op = OraclePool(W)
    try:
        op.round(0)  # warm-up: worker start, imports, first problem build
        res, t0, r = [], time.perf_counter(), 1
        while not res or time.perf_counter() - t0 < budget_s:
            out, _ = op.round(r)
            res += out
            r += 1
    finally:
        op.close()
    its = float(np.mean(outer_its)) if outer_its else 1.0
    solve_s, per_block, apply_s = op.estimate(res, its)
    js = sorted({j for j, _, _ in res})
    return {"value": round(1.0 / solve_s, 8), "unit": UNIT, "cores": op.cores, "kind": "oracle",
            "sample": f"{len(res)} frequency-block solves (Algorithm 2, inner GMRES to 1e-2, beta={op.beta}) at "
                      f"{2**W['level']}x{2**W['level']}, n_t={W['K']}, on a {op.cores}-process pool, "
                      f"j in {js[:6]}...{js[-3:]} (j = 0 in every round), hierarchies built before timing; "
                      f"{per_block:.2f} s/block x ceil({op.J} blocks / {op.cores} cores) = {apply_s:.1f} s/apply x "
                      f"{its:.1f} outer its (extrapolated)",
            "threads": "1 BLAS/OpenMP thread per process"}


def run_reference(a):
    """The oracle as it stands, on the host cores, same metric and workload;
    each step one round of frequency-block solves (one per core),
    extrapolated to a solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = WORKLOADS[a.workload]
    op = OraclePool(W)
    try:
        for i in range(a.warmup):
            op.round(i)
        res, per = [], []
        t0 = time.perf_counter()
        for i in range(a.steps):
            out, dt = op.round(a.warmup + i)
            res += out
            per.append(dt)
        dt = time.perf_counter() - t0
    finally:
        op.close()
    outer_its = OUTER_ITS_MEASURED.get(a.workload, 25)
    solve_s, per_block, apply_s = op.estimate(res, outer_its)
    v = 1.0 / solve_s
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 8), "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / a.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(a.workload, 1),
        "cpu_baseline": {"kind": "oracle", "cores": op.cores, "value": round(v, 8), "unit": UNIT,
                         "sample": f"each step one round of {len(op.sample(0))} frequency-block solves on a "
                                   f"{op.cores}-process pool ({per_block:.2f} s/block), x ceil({op.J} blocks / "
                                   f"{op.cores} cores) x {outer_its} outer its (extrapolated)"},
        "e2e": {"value": round(v, 8), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    a = parse()
    if not a.only_timed and (a.beta is not None or a.outer_restart is not None):
        sys.exit("--beta and --outer-restart change the workload: use them with --only-timed only")
    if a.impl == "reference":
        run_reference(a)
        return
    from paper_2405_18964_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    if a.workload == "serve":
        run_serve(a)
        return
    run_ours(a)


if __name__ == "__main__":
    main()
