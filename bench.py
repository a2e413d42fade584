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

Before the timed region the run measures the machine peaks its rooflines
divide by (random 2-byte gathers from a volume of the label volume's size,
FP64 adds and multiplies; include/rms_peaks.h).  After it: the FP32 form
against the plain FP64 form at every recording time, the same metric end to
end through the C ABI from host buffers, the serving stream under both tick
policies and in the FP64 form, and the oracle on a walker sample on the host.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
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
        r = rms.simulate(wl, prec, steps_per_launch=n, morton=args.morton)
        print(f"precision {prec}: {wl.n_walkers} walkers x {n} steps, walk {r['step_ms']:.2f} ms", flush=True)


def peaks_mode(args):
    """--peaks: the machine peaks the rooflines divide by, at the label
    volumes' sizes; one JSON line, and a markdown summary when --peaks-out
    names a file."""
    import torch
    import paper_2012_06478_gb300 as rms
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sp = torch.cuda.current_stream().cuda_stream
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        res = {"sm_count": rms.rms_device_sm_count(), "gather": {}, "gather_dep": {}}
        for lg in (16, 20, 24, 25, 26, 27, 28, 30):
            res["gather"][lg] = rms.rms_measure_peak(rms.RMS_PEAK_GATHER, 1 << lg, 20.0, 5, sp)[0]
            res["gather_dep"][lg] = rms.rms_measure_peak(rms.RMS_PEAK_GATHER_DEP, 1 << lg, 20.0, 5, sp)[0]
        for key, kind in (("fp64_add", rms.RMS_PEAK_FP64_ADD), ("fp64_mul", rms.RMS_PEAK_FP64_MUL),
                          ("fp64_fma", rms.RMS_PEAK_FP64_FMA)):
            res[key] = rms.rms_measure_peak(kind, 0, 20.0, 5, sp)[0]
    res["clocks"] = clk.summary()
    print(json.dumps(res), flush=True)
    if args.peaks_out:
        mhz = res["clocks"]["sm_mhz"] or 2070.0
        per_sm_clk = lambda r: r / (res["sm_count"] * mhz * 1e6)
        lines = [f"Measured with `python bench.py --peaks --peaks-out <file>` (best of 5 launches of ~20 ms, "
                 f"CUDA events); {res['sm_count']} SMs, median SM clock {mhz:.0f} MHz, "
                 f"throttle reasons: {res['clocks']['reasons'] or 'none'}.", "",
                 "| peak | rate | per SM per clock |", "|---|---|---|"]
        for key in ("fp64_add", "fp64_mul", "fp64_fma"):
            lines.append(f"| {key.replace('_', ' ')} (independent chains) | {res[key]:.4g} op/s | "
                         f"{per_sm_clk(res[key]):.3g} |")
        for lg in sorted(res["gather"]):
            mib = (2 << lg) / 2 ** 20
            lines.append(f"| random 2-byte gathers, {mib:g} MiB uint16 volume, 8 in flight per thread | "
                         f"{res['gather'][lg]:.4g} /s ({2 * res['gather'][lg] / 1e9:.0f} GB/s useful, "
                         f"{32 * res['gather'][lg] / 1e9:.0f} GB/s in 32-B sectors) | "
                         f"{per_sm_clk(res['gather'][lg]):.3g} |")
        for lg in sorted(res["gather_dep"]):
            mib = (2 << lg) / 2 ** 20
            lines.append(f"| dependent gathers (1 in flight per thread), {mib:g} MiB | "
                         f"{res['gather_dep'][lg]:.4g} /s | {per_sm_clk(res['gather_dep'][lg]):.3g} |")
        with open(args.peaks_out, "w") as f:
            f.write("\n".join(lines) + "\n")


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
    ap.add_argument("--serving-fp64-requests", type=int, default=64,
                    help="requests of the stream also served in the FP64 plain form (0: none)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--steps-per-launch", type=int, default=0,
                    help="steps per walk launch (0: the library's default, about 2e9 walker-steps per launch)")
    ap.add_argument("--morton", action="store_true",
                    help="re-bucket walkers in Morton order of their voxel before every launch (RMS_MORTON)")
    ap.add_argument("--ncu-case", type=int, default=0,
                    help="profiling case: one FP32 and one FP64 run of the workload with this many steps "
                         "(one walk launch each), no timing output")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the machine peaks behind the rooflines (FP64 add/mul, random-gather rates) and exit")
    ap.add_argument("--peaks-out", default="", help="with --peaks: write a markdown summary to this file")
    args = ap.parse_args()
    if args.peaks:
        return peaks_mode(args)
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
    run_flags = rms.RMS_MORTON if args.morton else 0

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
        res = num = None
        walk_ms = []
        walkers = None
        for it in range(n_warm + n_timed):
            flush_l2(torch, flush)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run = rms.rms_run(seq, W, wl.seed, precision, run_flags, w_begin, args.steps_per_launch, sp,
                              wl.interaction)
            e1.record(stream)
            res = rms.rms_read_signal(run)
            if it >= n_warm:
                ev.append(e0.elapsed_time(e1))
                walk_ms.append(rms.rms_run_step_time_ms(run))
            if it == n_warm + n_timed - 1:
                walkers = rms.rms_read_walkers(run)
                num = rms.rms_read_partials(run)[0]
            run.close()
        barrier()
        return ev, walk_ms, res, walkers, num

    # the peaks the rooflines divide by, measured on this GPU before the timed region
    pk = peaks()
    live = measure_peaks(rms, sp, wl.labels.size)
    # FP32 form: the headline
    with Clocks(local) as clk:
        ms32, walk32, res32, wk32, num32 = timed(rms.RMS_FP32, args.warmup, args.steps)
    # FP64 plain form, same workload
    if args.fp64_steps > 0:
        ms64, walk64, res64, wk64, _ = timed(rms.RMS_FP64, args.fp64_warmup, args.fp64_steps)
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
    fp32_err = fp32_vs_fp64(torch, wl, rms.rms_sequence_bvalues(seq), res32, res64, wk32, wk64)

    # the one exchange step: combine the per-rank sums (not timed)
    if world > 1:
        v = shard.allreduce_partials(shard.pack_partials(num32, res32[2], res32[1]))
        shard.unpack_partials(v, res32[0].shape, res32[1].shape)

    # the library's default launch size (about 8e9 walker-steps per launch with Morton re-bucketing)
    spl = args.steps_per_launch or max(64, min((8_000_000_000 if args.morton else 2_000_000_000) // W, wl.n_steps))
    n_walk = math.ceil(wl.n_steps / spl)
    # init, the walk launches, the two levels of the moment reduction, read-out, its reduction, normalisation
    launches_per_step = 1 + n_walk + (2 if wl.rec_steps.size else 0) + 3
    if args.morton:  # per walk launch: the key, 5 kernels per radix pass, the permutation
        launches_per_step += n_walk * (2 + 5 * morton_passes(wl.shape_xyz))
    sm_mhz = clk.summary().get("sm_mhz") or pk.get("sm_max_mhz") or 2070.0
    kernel = f"walk_kernel<{{}},1,false,{INTERACTIONS[args.interaction]},{'true' if args.rho > 0 else 'false'}>"
    variant = args.interaction == "ec" and args.rho == 0
    r32 = rooflines(wl, "fp32", W * spl, (sum(walk32) / len(walk32)) / n_walk, pk, live, sm_mhz,
                    kernel.format("float"), variant)
    r64 = (rooflines(wl, "fp64", W * spl, (sum(walk64) / len(walk64)) / n_walk, pk, live, sm_mhz,
                     kernel.format("double"), variant) if walk64 else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t32 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "walkers_per_gpu": W, "steps_per_walker": wl.n_steps, "dt_ms": wl.dt,
                   "grid_xyz": list(wl.shape_xyz), "voxel_um": wl.voxel_um, "labels": wl.n_labels,
                   "n_dirs": int(wl.dirs.shape[0]), "n_b": int(wl.b.size), "n_rec": int(wl.rec_steps.size),
                   "interaction": args.interaction, "rho_um_per_ms": args.rho,
                   "walker_order": "Morton order of the voxel, re-bucketed before every launch" if args.morton
                   else "walker id",
                   "precision": "fp32 form (headline); fp64 plain form in fp64_plain",
                   "l2": "flushed between timed iterations (256 MiB write)", "parallelism": f"walker shards x{world}"},
        "fp64_plain": {"value": value64, "unit": UNIT, "dtype": "f64", "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                       "ms_per_step": t64 / args.fp64_steps if args.fp64_steps > 0 else None,
                       "roofline": r64["roofline"] if r64 else None, "rooflines": r64["rooflines"] if r64 else None},
        "fp32_vs_fp64": fp32_err,
        "gpu_launches": launches_per_step * args.steps,
        "roofline": r32["roofline"],
        "rooflines": r32["rooflines"],
        "peaks": live,
        "clocks": clk.summary(),
    }
    line["config"]["steps_per_launch"] = spl
    if not args.no_e2e:
        line["e2e"] = e2e(rms, torch, wl, W, w_begin, sp, args, world, max_over_ranks)
    if not args.no_serving and world == 1 and variant:
        import rms_inputs as ri
        stream = serving_stream(rms, ri, args.serving_requests, sp)
        line["serving"] = serving(rms, stream, value, rms.RMS_FP32, rms.RMS_SERVE_FILL)
        line["serving_steps_policy"] = serving(rms, stream, value, rms.RMS_FP32, rms.RMS_SERVE_STEPS)
        if args.serving_fp64_requests > 0 and value64:
            line["serving_fp64"] = serving(rms, stream, value64, rms.RMS_FP64, rms.RMS_SERVE_FILL,
                                           args.serving_fp64_requests)
        for q in stream[2]:
            q.close()
        for sb in stream[1]:
            sb.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, threads=args.cpu_threads)
    seq.close()
    sub.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_peaks(rms, sp, n_voxels):
    """Machine peaks measured on this GPU (include/rms_peaks.h): random 2-byte
    gathers from a uint16 volume of the label volume's size (rounded up to a
    power of two), the same from a 512 MiB volume (past L2), one dependent
    gather in flight per thread, and independent FP64 adds and multiplies."""
    vol = 1 << max(10, int(math.ceil(math.log2(max(int(n_voxels), 1)))))
    out = {"sm_count": rms.rms_device_sm_count(), "gather_volume_elems": vol}
    for key, kind, elems in (("gather_per_s", rms.RMS_PEAK_GATHER, vol),
                             ("gather_dep_per_s", rms.RMS_PEAK_GATHER_DEP, vol),
                             ("gather_512MiB_per_s", rms.RMS_PEAK_GATHER, 1 << 28),
                             ("fp64_add_per_s", rms.RMS_PEAK_FP64_ADD, 0),
                             ("fp64_mul_per_s", rms.RMS_PEAK_FP64_MUL, 0),
                             ("fp64_fma_per_s", rms.RMS_PEAK_FP64_FMA, 0)):
        out[key] = rms.rms_measure_peak(kind, elems, 20.0, 3, sp)[0]
    return out


def _step_profile(wl):
    """Per-step quantities of the workload the operation counts depend on:
    face events per walker-step, the fraction of steps with a gradient (the
    phase update runs only then), the number of shapes, and whether any
    relaxation weight is accumulated."""
    G = np.asarray(wl.G, np.float64).reshape(-1, wl.n_steps) if wl.n_steps else np.zeros((1, 0))
    g_frac = float(np.any(G != 0.0, axis=0).mean()) if wl.n_steps else 0.0
    live = np.asarray(wl.dead) == 0
    relax = bool(np.any(np.isfinite(np.asarray(wl.T2)[live])) or np.any(np.isfinite(np.asarray(wl.T1)[live])))
    return events_per_step(wl), g_frac, G.shape[0], relax


def method_ops(wl):
    """Operations the method needs per walker-step in the FP32 form, counted
    from the method (not from any kernel): the issue floor.  One operation =
    one 32-bit ALU or FP32 instruction slot of one lane (a 32 x 32 -> 64-bit
    multiply, a three-input logical op, a fused multiply-add and a load each
    count one).
      Philox4x32-10 (one call per step): 10 rounds x (2 wide multiplies,
        2 three-input XORs); the round keys are constants of the run   40
      direction: z, r = sqrt((1-z)(1+z)), octant reduction, azimuth
        polynomials of degree 7/8, octant map, scaling                 28
      step vector d = n s_c                                            3
      face times (distance, |d|, reciprocal, product per axis)         12
      per face event: earliest axis, end test, neighbour index with
        wrap, label gather, label compare, voxel bookkeeping           13
      end of step: position and clamp per axis                         6
      phase, on steps with a gradient: displacement 4 per axis, Kahan
        add of dt G dx 5 per axis and shape                            12 + 15 S
      relaxation (a finite T1 or T2 somewhere): Kahan add               4
      step loop and flag load                                          3"""
    ev, g_frac, S, relax = _step_profile(wl)
    return 40 + 28 + 3 + 12 + 13 * ev + 6 + g_frac * (12 + 15 * S) + (4 if relax else 0) + 3


def fp64_ops(wl):
    """FP64 operations per walker-step of the plain form, counted from the
    method's arithmetic in the CPU reference's operation order (adds,
    multiplies, conversions; a division or a square root counts one):
      direction: sqrt 1; offset angle, its powers and the two polynomials
        11; angle addition 6; scaling by r 2                           20
      step vector                                                      3
      face times: 1 - o for axes moving up (half of them on average)
        and one division per axis                                      1.5 + 3
      per face event: segment time 1, the other two axes 4 (+2 with
        relaxation)                                                    5
      end of step: remaining fraction 1, positions 6 (+2 relaxation)    7
      phase, on steps with a gradient: displacement 4 per axis, dt G dx
        added 2 per axis and shape                                     12 + 6 S
    (z and (1 - z)(1 + z) are exact and built on the integer ALU: none.)"""
    ev, g_frac, S, relax = _step_profile(wl)
    return 20 + 3 + 4.5 + (5 + (2 if relax else 0)) * ev + 7 + (2 if relax else 0) + g_frac * (12 + 6 * S)


def kernel_source_sha(form):
    """A digest of the sources and build script that make the walk kernel of
    one form, to tell whether a profile summary still describes it."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2012_06478_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in ("walk_kernel.cuh", "rms_device.cuh", "soft_fp64.cuh", f"walk_{form}.cu")]
    files.append(os.path.join(ROOT, "paper_2012_06478_gb300", "build.py"))
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profile_counters(form, workload):
    """ncu figures of the walk kernel from profiles/walk_kernel_<form>_<workload>.md,
    only when the summary was taken of the current sources (its source-sha
    line equals kernel_source_sha(form)); otherwise None."""
    path = os.path.join(ROOT, "profiles", f"walk_kernel_{form}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for key, pat in (("sha", r"source-sha:\s*([0-9a-f]+)"),
                     ("inst_per_walker_step", r"thread-instructions per walker-step \|\s*([0-9.]+)"),
                     ("traffic_per_launch", r"dram bytes per launch \|\s*([0-9.eE+]+)"),
                     ("walker_steps_per_launch", r"walker-steps per launch \|\s*([0-9.eE+]+)")):
        m = re.search(pat, text)
        if m:
            vals[key] = m.group(1) if key == "sha" else float(m.group(1))
    if vals.get("sha") != kernel_source_sha(form):
        return None
    vals["profile"] = os.path.relpath(path, ROOT)
    return vals


def rooflines(wl, form, ws_per_launch, launch_ms, pk, live, sm_mhz, kernel, profiled=True):
    """The bounds of the walk kernel of one form, each as algorithmic work per
    launch over the measured launch time, against a measured peak:
      label_lookup_l2  2-byte label gathers (1.5 ds / l_p per walker-step)
                       against the measured random-gather rate of a volume
                       of the label volume's size (the level the gathers hit)
      label_lookup_hbm the same bytes against the HBM copy bandwidth
      issue_floor      the method's operation count (method_ops) against
                       the issue slots: SMs x 4 schedulers x 32 lanes x clock
      fp64_pipe        (plain form) the method's FP64 operations (fp64_ops)
                       against the measured FP64 add/multiply rate
    `roofline` is the bound with the highest fraction: the one that binds."""
    rate = ws_per_launch / (launch_ms * 1e-3)  # walker-steps/s of the walk launches
    ev = events_per_step(wl)
    gath = ev * rate
    hbm = pk.get("hbm_gbs")
    lanes = live["sm_count"] * 4 * 32 * sm_mhz * 1e6
    ops = method_ops(wl)
    out = {
        "label_lookup_l2": {"bound": "l2", "achieved": 2.0 * gath / 1e9, "peak": 2.0 * live["gather_per_s"] / 1e9,
                            "unit": "GB/s", "frac": gath / live["gather_per_s"],
                            "alg_bytes_per_walker_step": 2.0 * ev,
                            "what": "2 B per face event (1.5 ds/l_p events per walker-step) against random 2-byte "
                                    "gathers from a uint16 volume of the label volume's size, measured in this run"},
        "label_lookup_hbm": {"bound": "hbm", "achieved": 2.0 * gath / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": (2.0 * gath / 1e9 / hbm) if hbm else None,
                             "what": "the same label bytes against the HBM copy bandwidth (of measured)"},
        "issue_floor": {"bound": "alu", "achieved": ops * rate, "peak": lanes, "unit": "lane-op/s",
                        "frac": ops * rate / lanes, "ops_per_walker_step": ops,
                        "what": "method operations per walker-step (counted from the method) against "
                                f"{live['sm_count']} SMs x 4 x 32 lanes x {sm_mhz:.0f} MHz"},
    }
    if form == "fp64":
        f = fp64_ops(wl)
        peak64 = min(live["fp64_add_per_s"], live["fp64_mul_per_s"])
        out["fp64_pipe"] = {"bound": "fp64", "achieved": f * rate, "peak": peak64, "unit": "FP64 op/s",
                            "frac": f * rate / peak64, "ops_per_walker_step": f,
                            "what": "FP64 operations per walker-step of the plain form (a division or a square "
                                    "root counts one) against the measured FP64 add/multiply rate"}
        del out["issue_floor"]
    binding = max(out, key=lambda k: out[k]["frac"] or 0.0)
    prof = profile_counters(form, wl.name) if profiled else None
    head = dict(out[binding])
    head.update({"name": binding, "kernel": kernel, "launch_ms": launch_ms, "walker_steps_per_launch": ws_per_launch,
                 "traffic": prof["traffic_per_launch"] * ws_per_launch / prof["walker_steps_per_launch"]
                 if prof and "traffic_per_launch" in prof and "walker_steps_per_launch" in prof else None})
    if prof and "inst_per_walker_step" in prof:
        head["issue_utilisation"] = {"inst_per_walker_step": prof["inst_per_walker_step"],
                                     "frac": prof["inst_per_walker_step"] * rate / lanes,
                                     "profile": prof["profile"],
                                     "what": "thread-instructions the kernel executes per walker-step (ncu, from a "
                                             "capture of the current sources) x walker-steps/s, over the issue slots"}
    return {"roofline": head, "rooflines": out}


def fp32_vs_fp64(torch, wl, b_s, res32, res64, wk32, wk64, dev="cuda"):
    """The FP32 form against the plain FP64 form on the same walkers: S at
    every (shape, dir, b) and D, K along x, y, z at every recording time
    (Sec. 2.3, narrow pulse), each against its bar -- flat (|dS| <= 1e-3,
    |dD|/D <= 1 %, |dK| <= 1 % of |K|), and the stated readings (|dK| <=
    0.01 max(|K|, 0.1); |dS| <= 1e-3 + 4.5 standard errors of the paired
    per-walker differences, for walkers that FP32 rounding drift has
    decorrelated, whose number is given)."""
    dS = np.abs(res32[0] - res64[0])
    sig = paired_sigma(torch, wl, b_s, wk64, wk32, dev=dev)
    t = wl.rec_steps * wl.dt

    def _dk(M):
        a = M[:, 0]
        m2 = np.stack([M[:, 1], M[:, 4], M[:, 6]], 1) / a[:, None]
        m4 = np.stack([M[:, 7], M[:, 17], M[:, 21]], 1) / a[:, None]
        return m2 / (2 * t[:, None]), m4 / m2 ** 2 - 3
    out = {"max_abs_dS": float(dS.max()), "paired_sigma_S_max": float(sig.max()),
           "dS_within_flat_bar": bool(np.all(dS <= 1e-3)),
           "dS_within_bar": bool(np.all(dS <= 1e-3 + 4.5 * sig)),
           "decorrelated_walkers": int(np.any(wk32["i"] != wk64["i"], axis=1).sum()),
           "walkers": int(wk64["i"].shape[0])}
    if wl.rec_steps.size:
        D32, K32 = _dk(res32[1])
        D64, K64 = _dk(res64[1])
        rD = np.abs(D32 - D64) / D64
        aK = np.abs(K32 - K64)
        barK = 0.01 * np.maximum(np.abs(K64), 0.1)
        worst = np.unravel_index(np.argmax(aK / barK), aK.shape)
        out.update({
            "max_rel_dD": float(rD.max()), "max_abs_dK": float(aK.max()),
            "dD_within_bar": bool(np.all(rD <= 0.01)),
            "dK_within_bar": bool(np.all(aK <= barK)),
            "dK_within_flat_bar": bool(np.all(aK <= 0.01 * np.abs(K64))),
            "dK_worst": {"t_ms": float(t[worst[0]]), "axis": "xyz"[worst[1]], "K64": float(K64[worst]),
                         "K32": float(K32[worst]), "abs_dK": float(aK[worst]), "bar": float(barK[worst])},
            "per_time": {"t_ms": [round(float(x), 6) for x in t],
                         "max_rel_dD": [float(f"{x:.3g}") for x in rD.max(1)],
                         "dK_over_bar": [float(f"{x:.3g}") for x in (aK / barK).max(1)]},
        })
    out["bars"] = ("flat: |dS| <= 1e-3, |dD|/D <= 1%, |dK| <= 1% of |K|; stated (R14): |dK| <= 0.01 max(|K|, 0.1), "
                   "|dS| <= 1e-3 + 4.5 paired standard errors; every recording time and axis")
    return out


def serving_stream(rms, ri, n_requests, sp):
    """The seeded request stream of the serving benchmark, made resident:
    every request gets a substrate of its own -- a label volume from the
    generator pool (cylinder, axons or Voronoi at 32^3..256^3, 0.1 um voxels)
    with D, kappa and T1/T2 drawn for that request -- and a PGSE sequence
    (delta = TE/4, Delta = TE/2, b = 0, 1, 2 along its directions)."""
    reqs = ri.serving_requests(n_requests, seed=4)
    dt = 2e-4
    vols, subs, seqs = {}, [], []
    for r in reqs:
        key = (r["kind"], r["n"], r["geometry"])
        if key not in vols:
            vols[key] = ri.serving_geometry(*key)
        lab = vols[key]
        D, T2, T1, K = ri.serving_tables(r["kind"], int(lab.max()) + 1, r["seed"] % (2 ** 32))
        sub = rms.rms_create_substrate(lab, 0.1, D, T2=T2, T1=T1, kappa=K, stream=sp)
        n = r["n_steps"]
        G = ri.pgse(0.25 * n * dt, 0.5 * n * dt, dt, n)[None, :]
        rec = np.unique(np.linspace(n / 10, n, 10).astype(np.int64))
        subs.append(sub)
        seqs.append(rms.rms_set_sequence(sub, dt, G, ri.fibonacci_dirs(r["n_dirs"]), np.array([0.0, 1.0, 2.0]), rec))
    return reqs, subs, seqs


def serving(rms, stream, capacity, precision, policy, n_requests=None):
    """The stream through the continuous-batching server, Poisson arrivals at
    80 % of `capacity` (walker-steps/s of this precision); p50/p99 of
    submit-to-result latency, overall and by request size."""
    import threading
    reqs, subs, seqs = stream
    n = len(reqs) if n_requests is None else min(n_requests, len(reqs))
    reqs, seqs = reqs[:n], seqs[:n]
    work = np.array([r["n_walkers"] * r["n_steps"] for r in reqs], dtype=np.float64)
    rate = 0.8 * capacity / work.mean()
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    srv = rms.Server(memory_budget_bytes=16 << 30, max_active=64, steps_per_tick=256, policy=policy)
    tickets = [None] * n
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
    while not all(srv.poll(t) for t in tickets):
        time.sleep(0.01)
    el = time.perf_counter() - t0
    info = [srv.request_info(t) for t in tickets]
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    srv.close()
    lat = np.array([i["latency_ms"] for i in info])
    by_size = []
    edges = np.quantile(work, [0.0, 0.25, 0.5, 0.75, 1.0])
    for q in range(4):
        m = (work >= edges[q]) & ((work <= edges[q + 1]) if q == 3 else (work < edges[q + 1]))
        if m.any():
            by_size.append({"walker_steps": [float(f"{edges[q]:.3g}"), float(f"{edges[q + 1]:.3g}")],
                            "requests": int(m.sum()), "p50_ms": float(np.percentile(lat[m], 50)),
                            "p99_ms": float(np.percentile(lat[m], 99)),
                            "ms_per_1e9_walker_steps_p50": float(np.percentile(lat[m] / work[m] * 1e9, 50))})
    return {"requests": n, "precision": "fp32" if precision == rms.RMS_FP32 else "fp64",
            "policy": "fill" if policy == rms.RMS_SERVE_FILL else "steps",
            "offered_load": 0.8, "arrival_rate_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "walker_steps_per_s": st["walker_steps_per_s"], "wall_s": el,
            "peak_in_flight": st["peak_in_flight"], "ticks": st["ticks"], "graph_updates": st["graph_updates"],
            "graph_instantiations": st["graph_instantiations"],
            "queue_ms_max": float(max(i["queue_ms"] for i in info)), "by_size": by_size,
            "stream": "every request its own substrate: a cylinder/axon/Voronoi volume at 32^3..256^3 with its own "
                      "D, kappa, T1/T2; walkers 1e4-1e6 and steps 1e3-5e4 log-uniform, 6-64 directions"}


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


def morton_passes(shape_xyz):
    """Radix passes of RMS_MORTON's sort for a volume (8 key bits per pass;
    3 bits per coordinate bit, coordinates shifted to at most 8 bits)."""
    bits = int(max(shape_xyz) - 1).bit_length()
    return (3 * min(bits, 8) + 7) // 8


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
        run = rms.rms_run(seq, W, wl.seed, rms.RMS_FP32, rms.RMS_MORTON if args.morton else 0, w_begin,
                          args.steps_per_launch, sp, wl.interaction)
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
