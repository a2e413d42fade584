"""Benchmark of the RMS random-walker step on GB300.

One benchmark step = one whole simulation of the workload (walker
initialisation, every time step with face walk / membrane crossing / phase /
relaxation, the moment reductions and the signal read-out), with the label
volume and sequence tables already resident in HBM.  The default workload is
the 200 x 200 x 400 synthetic beaded-axon volume (0.1 um voxels, 200 axons,
kappa = 0.01 um/ms), 1e6 walkers x 1e5 steps of dt = 2e-4 ms, 30 directions
x 11 b-values.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own 1e6
walkers (distinct global walker ids): weak scaling, no collective on the data
path; the per-rank sums are combined after the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/s (FP64 plain vs FP32 form, |ΔS|≤1e-3); p50/p99 request latency"
UNIT = "walker-steps/s"
DEFAULT_WORKLOAD = "axons-200x200x400"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 6:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for n, v in zip(names, p[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(torch, buf):
    buf.add_(1.0)  # 256 MiB written: larger than the 129 MB L2


INTERACTIONS = {"ec": 0, "rs": 1, "erl": 2}  # elastic collision, rejection sampling, ERL


def workload_of(name, interaction="ec", rho=0.0):
    """The named workload with the given interaction and, when rho > 0, every
    membrane absorbing with surface relaxivity rho (um/ms, Sec. 2.1.3)."""
    import rms_inputs as ri
    wl = ri.workload(name).with_(interaction=INTERACTIONS[interaction])
    if rho > 0:
        R = np.full((wl.n_labels, wl.n_labels), float(rho))
        np.fill_diagonal(R, 0.0)
        wl = wl.with_(rho=R)
    return wl


def events_per_step(wl):
    """Expected face events per walker-step, 1.5 ds / l_p (exact for any
    lattice), averaged over labels by where the walkers are: the live
    volume, weighted by the spin concentration when there is one."""
    lab = wl.labels
    w = np.bincount(lab.ravel(), minlength=wl.n_labels).astype(np.float64)
    w *= np.asarray(wl.dead) == 0
    if wl.conc is not None:
        w *= np.asarray(wl.conc, np.float64)
    ds = np.sqrt(6.0 * wl.D * wl.dt)
    return float((w / w.sum() * 1.5 * ds / wl.voxel_um).sum())


def cpu_baseline(wl, seconds=12.0, threads=0):
    """The oracle as it stands on this host's cores, on a walker sample of the
    same workload (walkers are independent: the sample's rate is the run's)."""
    import oracle
    oracle.build()
    cores = threads or os.cpu_count() or 1
    probe = max(cores, 16)
    t0 = time.perf_counter()
    oracle.run(wl, 0, probe, n_threads=cores, hash_=False)
    dt = time.perf_counter() - t0
    rate = probe * wl.n_steps / dt
    W = max(cores, int(rate * seconds / wl.n_steps) // cores * cores)
    t0 = time.perf_counter()
    r = oracle.run(wl, 0, W, n_threads=cores, hash_=False)
    oracle.readout(r, wl)
    el = time.perf_counter() - t0
    return {"value": W * wl.n_steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"walkers 0..{W - 1} x all {wl.n_steps} steps of {wl.name} (+ read-out), {el:.1f} s"}


def run_reference(args):
    """The oracle timed as the reference arm (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload_of(args.workload, args.interaction, args.rho)
    import oracle
    oracle.build()
    cores = args.cpu_threads or os.cpu_count() or 1
    probe = max(cores, 16)
    t0 = time.perf_counter()
    oracle.run(wl, 0, probe, n_threads=cores, hash_=False)
    rate = probe * wl.n_steps / (time.perf_counter() - t0)
    W = max(cores, int(rate * 8.0 / wl.n_steps) // cores * cores)  # ~8 s per step
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.run(wl, it * W, (it + 1) * W, n_threads=cores, hash_=False)
        oracle.readout(r, wl)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    el = sum(times)
    value = args.steps * W * wl.n_steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "walkers_per_step": W, "steps_per_walker": wl.n_steps,
                       "interaction": args.interaction, "rho_um_per_ms": args.rho},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{W} walkers x {wl.n_steps} steps of {wl.name} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(args):
    """The small case the kernel profiles in profiles/ are captured on: the
    workload's first `--ncu-case` steps, all walkers, one walk launch per form."""
    import torch
    import paper_2012_06478_gb300 as rms
    wl = workload_of(args.workload, args.interaction, args.rho)
    n = args.ncu_case
    wl = wl.with_(n_steps=n, G=np.asarray(wl.G)[:, :n], rec_steps=wl.rec_steps[wl.rec_steps <= n])
    for prec in (rms.RMS_FP32, rms.RMS_FP64):
        r = rms.simulate(wl, prec, steps_per_launch=n)
        print(f"precision {prec}: {wl.n_walkers} walkers x {n} steps, walk {r['step_ms']:.2f} ms", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--interaction", default="ec", choices=sorted(INTERACTIONS),
                    help="particle-membrane interaction: elastic collision (the paper's method), rejection "
                         "sampling or ERL (App. A, B)")
    ap.add_argument("--rho", type=float, default=0.0,
                    help="surface relaxivity (um/ms) of every membrane: magnetization transfer (Sec. 2.1.3)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed FP64 plain-form steps")
    ap.add_argument("--fp64-warmup", type=int, default=1, help="untimed FP64 plain-form steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads for the oracle legs (cpu_baseline, --impl reference); 0: all cores")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=512)
    ap.add_argument("--serving-fp64", action="store_true", help="also serve the stream in the FP64 plain form")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ncu-case", type=int, default=0,
                    help="profiling case: one FP32 and one FP64 run of the workload with this many steps "
                         "(one walk launch each), no timing output")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return ncu_case(args)

    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2012_06478_gb300 as rms
    from paper_2012_06478_gb300 import shard
    wl = workload_of(args.workload, args.interaction, args.rho)
    W = wl.n_walkers
    w_begin, _ = shard.shard_range(rank, world, W, weak=True)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    sub = rms.rms_create_substrate(wl.labels, wl.voxel_um, wl.D, T2=wl.T2, T1=wl.T1, kappa=wl.kappa,
                                   dead=wl.dead, periodic=wl.periodic, stream=sp, rho=wl.rho, conc=wl.conc,
                                   lam=wl.lam, perm_model=wl.perm_model)
    seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps, mode=wl.mode)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed(precision, n_warm, n_timed):
        """Time n_timed runs after n_warm; the walkers of the last run are
        read after the timed region (for the FP32-vs-FP64 error bars)."""
        ev = []
        res = None
        walk_ms = []
        walkers = None
        for it in range(n_warm + n_timed):
            flush_l2(torch, flush)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run = rms.rms_run(seq, W, wl.seed, precision, 0, w_begin, 0, sp, wl.interaction)
            e1.record(stream)
            res = rms.rms_read_signal(run)
            if it >= n_warm:
                ev.append(e0.elapsed_time(e1))
                walk_ms.append(rms.rms_run_step_time_ms(run))
            if it == n_warm + n_timed - 1:
                walkers = rms.rms_read_walkers(run)
            run.close()
        barrier()
        return ev, walk_ms, res, walkers

    # FP32 form: the headline
    with Clocks(local) as clk:
        ms32, walk32, res32, wk32 = timed(rms.RMS_FP32, args.warmup, args.steps)
    # FP64 plain form, same workload
    if args.fp64_steps > 0:
        ms64, walk64, res64, wk64 = timed(rms.RMS_FP64, args.fp64_warmup, args.fp64_steps)
    else:
        ms64, walk64, res64, wk64 = [float("nan")], [], res32, wk32

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    t32 = max_over_ranks(sum(ms32))
    t64 = max_over_ranks(sum(ms64))
    ws = W * wl.n_steps
    value = world * ws * args.steps / (t32 * 1e-3)
    value64 = world * ws * args.fp64_steps / (t64 * 1e-3) if args.fp64_steps > 0 else None
    dS = float(np.abs(res32[0] - res64[0]).max())
    # FP32 form against the FP64 plain form on the same walkers: D and K along
    # x, y, z at every recording time (Sec. 2.3, narrow pulse)
    def _dk(M):
        t = wl.rec_steps * wl.dt
        a = M[:, 0]
        m2 = np.stack([M[:, 1], M[:, 4], M[:, 6]], 1) / a[:, None]
        m4 = np.stack([M[:, 7], M[:, 17], M[:, 21]], 1) / a[:, None]
        return m2 / (2 * t[:, None]), m4 / m2 ** 2 - 3
    D32, K32 = _dk(res32[1])
    D64, K64 = _dk(res64[1])
    sig = paired_sigma(torch, wl, rms.rms_sequence_bvalues(seq), wk64, wk32)
    fp32_err = {"max_abs_dS": dS, "max_rel_dD": float(np.max(np.abs(D32 - D64) / D64)),
                "max_abs_dK": float(np.max(np.abs(K32 - K64))),
                "paired_sigma_S_max": float(sig.max()),
                "dS_within_bar": bool(np.all(np.abs(res32[0] - res64[0]) <= 1e-3 + 4.5 * sig)),
                "bars": "|dS| <= 1e-3 (+ 4.5 standard errors of the paired per-walker differences, for walkers "
                        "that FP32 rounding drift has decorrelated), |dD|/D <= 1%, |dK| <= 0.01 max(|K|, 0.1)"}

    # the one exchange step: combine the per-rank sums (not timed)
    if world > 1:
        v = shard.allreduce_partials(shard.pack_partials(res32[0], res32[2], res32[1]))
        shard.unpack_partials(v, res32[0].shape, res32[1].shape)

    spl = max(64, min(2_000_000_000 // W, wl.n_steps))
    n_walk = math.ceil(wl.n_steps / spl)
    launches_per_step = 1 + n_walk + (1 if wl.rec_steps.size else 0) + 3
    walk_launch_ms = (sum(walk32) / len(walk32)) / n_walk
    eps = events_per_step(wl)
    alg_bytes = 2.0 * eps * W * spl  # label bytes per walk launch
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    achieved = alg_bytes / (walk_launch_ms * 1e-3) / 1e9
    sm_mhz = (clk.summary().get("sm_mhz") or pk.get("sm_max_mhz") or 2070.0)
    lane_peak = ISSUE_LANES_PER_CLOCK * sm_mhz * 1e6
    variant = args.interaction == "ec" and args.rho == 0
    kernel_name = f"walk_kernel<float,1,false,{INTERACTIONS[args.interaction]},{'true' if args.rho > 0 else 'false'}>"
    prof = PROFILED.get(wl.name if variant else f"{wl.name}/{args.interaction}/rho{args.rho:g}", {})
    lane_rate = (prof["inst_per_walker_step"] * (W * spl) / (walk_launch_ms * 1e-3)
                 if "inst_per_walker_step" in prof else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t32 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "walkers_per_gpu": W, "steps_per_walker": wl.n_steps, "dt_ms": wl.dt,
                   "grid_xyz": list(wl.shape_xyz), "voxel_um": wl.voxel_um, "labels": wl.n_labels,
                   "n_dirs": int(wl.dirs.shape[0]), "n_b": int(wl.b.size), "n_rec": int(wl.rec_steps.size),
                   "interaction": args.interaction, "rho_um_per_ms": args.rho,
                   "precision": "fp32 form (headline); fp64 plain form in fp64_plain",
                   "l2": "flushed between timed iterations (256 MiB write)", "parallelism": f"walker shards x{world}"},
        "fp64_plain": {"value": value64, "unit": UNIT, "dtype": "f64", "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                       "ms_per_step": t64 / args.fp64_steps if args.fp64_steps > 0 else None},
        "fp32_vs_fp64": fp32_err,
        "gpu_launches": launches_per_step * args.steps,
        # the binding roofline: the walk kernel is issue-bound (gathers and branches, no contraction)
        "roofline": {"bound": "alu", "achieved": lane_rate, "peak": lane_peak, "unit": "lane-instr/s",
                     "frac": lane_rate / lane_peak if lane_rate else None,
                     "traffic": prof.get("traffic_per_launch"), "kernel": kernel_name,
                     "inst_per_walker_step": prof.get("inst_per_walker_step"), "profile": prof.get("profile"),
                     "walker_steps_per_launch": W * spl, "launch_ms": walk_launch_ms,
                     "what": "issue slots: 152 SMs x 4 schedulers x 32 lanes x measured SM clock; work = "
                             "thread-instructions per walker-step (ncu) x walker-steps/s of the walk launches; "
                             "traffic = DRAM bytes per launch (ncu)"},
        # the label-lookup roofline: algorithmic label bytes against HBM copy bandwidth
        "roofline_label_lookup": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                  "frac": (achieved / hbm) if hbm else None, "kernel": kernel_name,
                                  "alg_bytes_per_walker_step": 2.0 * eps,
                                  "what": "label-lookup bytes (2 B per face event) against HBM copy bandwidth "
                                          "(of measured); the gathers are served by L2"},
        "clocks": clk.summary(),
    }
    if not args.no_e2e:
        line["e2e"] = e2e(rms, torch, wl, W, w_begin, sp, args, world, max_over_ranks)
    if not args.no_serving and world == 1 and variant:
        import rms_inputs as ri
        line["serving"] = serving(rms, ri, value, args.serving_requests, rms.RMS_FP32, sp)
        if args.serving_fp64 and value64:
            line["serving_fp64"] = serving(rms, ri, value64, args.serving_requests, rms.RMS_FP64, sp)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, threads=args.cpu_threads)
    seq.close()
    sub.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Per workload, from the ncu capture of one FP32 walk launch of its benchmark
# launch shape: thread-instructions per walker-step (smsp__inst_executed x
# thread_inst_executed_per_inst_executed / walker-steps) and DRAM bytes read +
# written per launch.  Workloads without a capture report null.
PROFILED = {
    "axons-200x200x400": {"inst_per_walker_step": 302.8, "traffic_per_launch": 152.4e6,
                          "profile": "profiles/walk_kernel_fp32_axons-200x200x400.md"},
}
ISSUE_LANES_PER_CLOCK = 152 * 4 * 32  # SMs x schedulers x lanes


def serving_pool(ri):
    """Resident substrates of the serving stream: each generator kind at
    32^3, 64^3, 128^3, 256^3 (0.1 um voxels, D = 2, kappa = 0.01)."""
    pool = {}
    for n in (32, 64, 128, 256):
        pool[("cylinder", n)] = ri.cylinder_labels(n, n / 3.2)
        pool[("axons", n)] = ri.axon_labels(n, n, n, 0.1, max(2, int(round(200 * (n / 200.0) ** 2))), seed=40 + n)
        pool[("voronoi", n)] = ri.voronoi_labels(n, max(8, int(1000 * (n / 512.0) ** 3)), seed=50 + n)
    return pool


def serving(rms, ri, capacity, n_requests, precision, sp):
    """A seeded stream of requests with Poisson arrivals at 80% of the
    measured capacity through the continuous-batching server; p50/p99 of
    submit-to-result latency."""
    import threading
    reqs = ri.serving_requests(n_requests, seed=4)
    pool = serving_pool(ri)
    dt = 2e-4
    subs, seqs = {}, []
    for key, lab in pool.items():
        L = int(lab.max()) + 1
        K = np.full((L, L), 0.01)
        np.fill_diagonal(K, 0.0)
        subs[key] = rms.rms_create_substrate(lab, 0.1, np.full(L, 2.0), kappa=K, stream=sp)
    for r in reqs:
        n = r["n_steps"]
        G = ri.pgse(0.25 * n * dt, 0.5 * n * dt, dt, n)[None, :]
        rec = np.unique(np.linspace(n / 10, n, 10).astype(np.int64))
        seqs.append(rms.rms_set_sequence(subs[(r["kind"], r["n"])], dt, G, ri.fibonacci_dirs(r["n_dirs"]),
                                         np.array([0.0, 1.0, 2.0]), rec))
    work = np.array([r["n_walkers"] * r["n_steps"] for r in reqs], dtype=np.float64)
    rate = 0.8 * capacity / work.mean()
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    srv = rms.Server(memory_budget_bytes=16 << 30, max_active=64, steps_per_tick=256)
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for k, r in enumerate(reqs):
            delay = arrivals[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(seqs[k], r["n_walkers"], r["seed"] % (2 ** 63), precision)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    for t in tickets:
        srv.wait(t)
    el = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    for q in seqs:
        q.close()
    for sb in subs.values():
        sb.close()
    return {"requests": len(reqs), "precision": "fp32" if precision == rms.RMS_FP32 else "fp64",
            "offered_load": 0.8, "arrival_rate_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "walker_steps_per_s": st["walker_steps_per_s"], "wall_s": el,
            "peak_in_flight": st["peak_in_flight"], "ticks": st["ticks"], "graph_updates": st["graph_updates"],
            "graph_instantiations": st["graph_instantiations"],
            "stream": "requests from 12 resident substrates (cylinder/axons/voronoi at 32^3..256^3), "
                      "walkers 1e4-1e6 and steps 1e3-5e4 log-uniform, 6-64 directions"}


def paired_sigma(torch, wl, b_s, w64, w32, dev="cuda"):
    """Per (shape, dir, b): the standard error of the mean of the paired
    per-walker differences alpha e^{-i phi} / <alpha> (FP32 form minus FP64
    form, same walkers).  Computed on the device in walker chunks."""
    f64 = torch.float64
    q = torch.tensor(np.sqrt(np.asarray(wl.b)[None, :] / np.asarray(b_s)[:, None]), dtype=f64, device=dev)
    dirs = torch.tensor(np.asarray(wl.dirs), dtype=f64, device=dev)
    a64 = torch.exp(-torch.tensor(w64["A"], dtype=f64, device=dev))
    a32 = torch.exp(-torch.tensor(w32["A"], dtype=f64, device=dev))
    m64, m32 = a64.mean(), a32.mean()
    W = a64.shape[0]
    chunk = max(1024, int(2e7) // (q.numel() * dirs.shape[0]))  # ~0.3 GB per complex term
    s1 = torch.zeros(q.shape[0], dirs.shape[0], q.shape[1], dtype=torch.complex128, device=dev)
    s2 = torch.zeros(s1.shape, dtype=f64, device=dev)
    for b in range(0, W, chunk):
        e = min(W, b + chunk)
        terms = []
        for wk, al, m in ((w32, a32, m32), (w64, a64, m64)):
            ph = torch.tensor(wk["phase"][b:e], dtype=f64, device=dev)        # (w, S, 3)
            phi = torch.einsum("wsa,da->wsd", ph, dirs)[..., None] * q[None, :, None, :]
            terms.append((al[b:e] / m)[:, None, None, None] * torch.exp(-1j * phi))
        d = terms[0] - terms[1]
        s1 += d.sum(0)
        s2 += (d.real ** 2 + d.imag ** 2).sum(0)
    var = s2 / W - (s1 / W).abs() ** 2
    return (var.clamp_min(0) / W).sqrt().cpu().numpy()


def e2e(rms, torch, wl, W, w_begin, sp, args, world, max_over_ranks):
    """The same metric through the C ABI from host buffers: upload of the
    label volume and tables, the run, the read-back of the signal and moments."""
    lab = np.ascontiguousarray(wl.labels, np.uint16)
    h2d = (lab.nbytes + wl.D.nbytes + wl.T2.nbytes + wl.T1.nbytes + wl.kappa.nbytes + wl.dead.nbytes +
           np.asarray(wl.G).nbytes + wl.dirs.nbytes + wl.b.nbytes + wl.rec_steps.nbytes)
    n_combo = np.asarray(wl.G).reshape(-1, wl.n_steps).shape[0] * wl.dirs.shape[0] * wl.b.size
    d2h = 16 * n_combo + 8 * 22 * wl.rec_steps.size + 8
    times = []
    for it in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sub = rms.rms_create_substrate(lab, wl.voxel_um, wl.D, T2=wl.T2, T1=wl.T1, kappa=wl.kappa, dead=wl.dead,
                                       periodic=wl.periodic, stream=sp, rho=wl.rho, conc=wl.conc, lam=wl.lam,
                                       perm_model=wl.perm_model)
        seq = rms.rms_set_sequence(sub, wl.dt, wl.G, wl.dirs, wl.b, wl.rec_steps, mode=wl.mode)
        run = rms.rms_run(seq, W, wl.seed, rms.RMS_FP32, 0, w_begin, 0, sp, wl.interaction)
        rms.rms_read_signal(run)
        el = time.perf_counter() - t0
        run.close()
        seq.close()
        sub.close()
        if it >= 1:
            times.append(el)
    t = max_over_ranks(sum(times))
    return {"value": world * W * wl.n_steps * args.steps / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


if __name__ == "__main__":
    main()
