"""Throughput of the digital-twin-brain step on GB300.

Workload: the 20,000,000-neuron / 2,000-voxel network with in-degree 500
(1e10 synapses, int16 weights at 2^-12, delays 1..80 steps, dt = 0.1 ms), run
at the 7, 15 and 30 Hz operating points.  A "step" is one simulation time step
of the whole path: neuron update, spike compaction, spike delivery, BOLD.

Prints ONE JSON line: synaptic events/s over the three rates (value), per-rate
events/s, biological seconds per wall second and HBM fraction, the dominant
kernel's roofline, the oracle's CPU baseline, an end-to-end figure through the
C ABI with host buffers, and SM clocks sampled while the steps run.

Each rate starts from a reset network that is first brought to its operating
point by SETTLE_STEPS untimed steps (more while its rate is off), whatever
--warmup is; then W warm-up steps, then K timed steps (dtb_step, CUDA graphs),
then K more steps of the same schedule with events around every kernel
(dtb_step_timed: the per-kernel times and the roofline), K more with the
kernels one after the other (dtb_profile_steps: each kernel's share, which
picks the dominant one, as a serialised launch list would), then K steps end
to end through host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs N independent replicas (one per rank, no communication): the step
has no data-parallel split on one node ("replicas only").
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

CONFIG = "c3_large_20m"
RATES = (7, 15, 30)
METRIC = "synaptic events/s (20M neurons, 7/15/30 Hz)"
UNIT = "synaptic events/s"
# untimed steps after each reset, whatever --warmup is: the network's
# transient (rates overshoot to 11 / 37 / 103 Hz in its first 300 steps) is
# over after about 2,500 steps at every rate
SETTLE_STEPS = 3000
SETTLE_PROBE = 500   # steps of each window that checks the rate afterwards
SETTLE_EXTRA = 4     # at most this many more windows while the rate is off
RATE_TOL = 0.10      # a rate within 10 % of its target counts as on the operating point
LOG_CAP = 1 << 25   # spike ids kept per call: 100 steps at 30 Hz of 20M neurons need 6M
E2E_CHUNK = 250     # steps per end-to-end call (25 ms of biological time)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def aggregate(ms: float, events: float, device="cpu"):
    """Whole-job figures of N independent replicas: the max time over ranks
    and the sum of events over ranks (no-op on one process)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    e = torch.tensor([events], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


class ClockSampler:
    """nvidia-smi samples (200 ms) while every rate's steps run: its settle,
    timed, per-kernel and end-to-end steps run the same kernels."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.file.flush()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.file.name).read().strip().splitlines() if r.strip()]
            os.unlink(self.file.name)
        except Exception:
            rows = []
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_bytes(cfg, n, nch, wbytes, spikes_per_step, events_per_step, delivery="queue"):
    """Algorithmic bytes per launch of each kernel of one step.  In bins mode
    the neuron update has no accumulator rows; it reads the step's binned
    arrival events instead (4 bytes each, 8 with int32 weights)."""
    if delivery == "bins":
        state = n * (4 + 16 + 1) * 2 + n / 8.0 + events_per_step * (8 if wbytes == 4 else 4)
    else:
        state = n * (4 + 16 + 1 + 4 * nch) * 2 + n / 8.0      # V, j, ref, ring slot read + write; spike bits
    compact = n / 8.0 + 4 * n / 1024 + 8 * spikes_per_step     # bits, block counts; ids (list + log)
    rows = spikes_per_step * 16 + events_per_step * (4 + wbytes)  # row pointers, word + weight per synapse
    acc = events_per_step * 8                                  # accumulator read-modify-write
    return {"neuron_update": state, "spike_compact": compact, "spike_delivery": rows + acc,
            "spike_deliver_rows": rows, "bold_step": 0.0}


UPDATE_END = b"// ==== end of the neuron update ===="


def update_source_sha256():
    """sha256 of the neuron update's source: step_kernels.cu up to its end
    marker, then dtb_device.cuh."""
    csrc = os.path.join(ROOT, "paper_2308_01241_gb300", "csrc")
    sk = open(os.path.join(csrc, "step_kernels.cu"), "rb").read()
    return hashlib.sha256(sk[:sk.index(UPDATE_END)] + open(os.path.join(csrc, "dtb_device.cuh"), "rb").read()).hexdigest()


def _traffic_record(kernel, delivery):
    """ncu DRAM bytes per launch recorded under profiles/, if the update's
    source is unchanged and the record is of the same delivery mode."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
        if rec.get("source_sha256") != update_source_sha256() or rec.get("delivery") != delivery:
            return None
        return rec.get("kernels", {}).get(kernel)
    except Exception:
        return None


SAMPLE_NEURONS, SAMPLE_VOXELS, SAMPLE_RATE = 100_000, 50, 15


def _oracle_sample():
    """The C oracle (single thread) on a bounded sample with the workload's
    per-neuron structure: 100,000 neurons in 50 voxels, in-degree 500 (half
    intra-voxel, half by the DTI-like matrix), delays 1..80, int16 weights, at
    the 15 Hz gain of the 20M-neuron config."""
    import oracle
    from paper_2308_01241_gb300 import netgen

    oracle.build()
    cfg = netgen.load_config(CONFIG)
    tb = netgen.make_tables(cfg, n_neurons=SAMPLE_NEURONS, n_vox=SAMPLE_VOXELS)
    d = netgen.oracle_inputs(tb, netgen.host_pull(tb), rate=SAMPLE_RATE)
    return oracle.OracleNet(d, "f32")


def _sample_text(steps, el, ev):
    return (f"{SAMPLE_NEURONS // 1000}k-neuron/{SAMPLE_VOXELS}-voxel network with the 20M config's per-neuron "
            f"structure (K=500, delays 1-80, int16, {SAMPLE_RATE} Hz gain): {steps} steps in {el:.1f} s, "
            f"{ev} events, single thread")


def _cpu_baseline(budget_s: float = 15.0):
    net = _oracle_sample()
    net.run(SETTLE_STEPS)  # transient, untimed
    ev0, steps, t0 = net.events(), 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        net.run(50)
        steps += 50
    el = time.perf_counter() - t0
    ev = net.events() - ev0
    return {"value": ev / el, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": _sample_text(steps, el, ev)}


def run_reference(args):
    """The oracle as it stands on the host cores: W untimed steps, then K timed
    steps of the bounded sample (rank 0 only)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    net = _oracle_sample()
    net.run(SETTLE_STEPS + args.warmup)  # the same untimed settle as the GPU arm, then the warm-up
    ev0 = net.events()
    t0 = time.perf_counter()
    net.run(args.steps)
    el = time.perf_counter() - t0
    ev = net.events() - ev0
    value = ev / el
    sample = _sample_text(args.steps, el, ev)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{CONFIG} sample on host cores", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def launches_per_call(k: int, delivery: str) -> int:
    """Kernels one dtb_step(k) call launches: the call's start, every step's
    update, compaction, delivery, BOLD (+ queue drain or binning), one
    step-counter advance per chunk of up to 32 steps (the first step is a
    chunk of its own), and the closing j-only update and spill-flag clear."""
    if k <= 0:
        return 1
    per_step = 4 if delivery == "ring" else 5
    return 1 + per_step * k + 1 + -(-(k - 1) // 32) + 2


def settle(net, n, dt_ms, target_hz, steps=SETTLE_STEPS, probe=SETTLE_PROBE, extra=SETTLE_EXTRA, tol=RATE_TOL):
    """Untimed steps that bring a freshly reset network to its operating
    point: `steps` steps (the transient of the 20M-neuron network lasts about
    2,500 steps at every rate), then up to `extra` more probe windows until the
    rate of the last one is within tol of the target.  Returns (steps run,
    rate of the last window)."""
    done = 0
    while done < steps:
        c = min(500, steps - done)
        net.step(c)
        done += c
    rate = None
    for _ in range(1 + extra):
        sp0 = net.counters()[1]
        net.step(probe)
        done += probe
        rate = (net.counters()[1] - sp0) / (n * probe * dt_ms * 1e-3)
        if abs(rate - target_hz) <= tol * target_hz:
            break
    return done, rate


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    from paper_2308_01241_gb300 import dtb, netgen

    cfg = netgen.load_config(args.config)
    tb = netgen.make_tables(cfg, n_neurons=args.neurons, n_vox=args.voxels, K=args.indegree)
    wfmt = args.wfmt or cfg["wfmt"]
    csr = netgen.device_csr(tb, wfmt, device=device)
    wbytes = {"int16": 2, "int32": 4, "bf16": 2, "int8": 1}[wfmt]
    net = dtb.from_tables(tb, csr, device=device, wfmt=wfmt, log_capacity=LOG_CAP, delivery=args.delivery)
    if args.shapes:
        net.set_shapes(*args.shapes)
    net.set_schedule(args.schedule)
    n, dt_ms = tb.n, float(cfg["dt"])
    nch = int(cfg["n_ch"])
    stream = net.stream
    peak, peak_kind = _peaks()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(device)

    per_rate = {}
    tot_ev, tot_ms, tot_steps = 0, 0.0, 0
    stages = {"neuron_update": ("neuron_update",), "spike_compact": ("spike_compact",),
              "spike_delivery": ("spike_deliver", "queue_drain"), "bold_step": ("bold_step",)}
    # per stage: summed launch ms, summed algorithmic bytes, launches (timed schedule, every rate),
    # summed ms with the kernels one after the other (the shares ncu's launch list shows)
    prof_acc = {k: [0.0, 0.0, 0, 0.0] for k in stages}
    launches = 0
    chunk = min(E2E_CHUNK, args.steps)
    # the end-to-end leg's host buffers live in pinned (page-locked) memory, as a
    # serving loop would keep them; numpy views of pinned torch tensors
    ids_buf = torch.empty(LOG_CAP, dtype=torch.int32, pin_memory=True).numpy()
    off_buf = torch.empty(chunk + 1, dtype=torch.int64, pin_memory=True).numpy()
    g_pin = torch.empty((tb.nv, 4), dtype=torch.float64, pin_memory=True).numpy()
    h2d = d2h = 0
    e2e_s = 0.0
    ev_e2e = 0
    settle_steps = {}
    clocks = ClockSampler(local)
    with clocks:
        for r in args.rates:
            gain = netgen.gain_for(cfg, r)
            g_host = np.ascontiguousarray(tb.vparams(gain)[:, 6:10])
            net.set_hyperparams(g_host)
            net.reset()
            settle_steps[str(r)], settle_rate = settle(net, n, dt_ms, r)
            net.step(args.warmup)
            ev0, sp0, _ = net.counters()
            barrier()
            # (1) the timed region: dtb_step (CUDA graphs), events on the library stream;
            # it is also the profiler range (cudaProfilerStart/Stop, no-ops unless a
            # profiler runs with profiling from the start off)
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            torch.cuda.profiler.start()
            start.record(stream)
            net.step(args.steps)
            end.record(stream)
            end.synchronize()
            torch.cuda.profiler.stop()
            ms = start.elapsed_time(end)
            barrier()
            ev1, sp1, _ = net.counters()
            ev = ev1 - ev0
            ms, ev_all = aggregate(ms, ev, device)
            launches += launches_per_call(args.steps, args.delivery)
            rate_hz = (sp1 - sp0) / (n * args.steps * dt_ms * 1e-3)
            # (2) per-kernel device time in the same schedule over the next K
            # steps (dtb_step_timed: events around every launch on its own
            # stream); the algorithmic bytes come from these steps' own counters
            ev2, sp2, _ = net.counters()
            kms_sum, kcnt = net.step_timed(args.steps)
            ev3, sp3, _ = net.counters()
            body = max(args.steps - 1, 1)
            kb = _kernel_bytes(cfg, n, nch, wbytes, (sp3 - sp2) / args.steps, (ev3 - ev2) / args.steps,
                               args.delivery)
            kms = {nm: (kms_sum[k] / kcnt[k] if kcnt[k] else 0.0) for k, nm in enumerate(dtb.KERNELS)}
            for st, parts in stages.items():
                cnt = int(kcnt[dtb.KERNELS.index(parts[0])])
                prof_acc[st][0] += sum(float(kms_sum[dtb.KERNELS.index(p)]) for p in parts)
                prof_acc[st][1] += kb[st] * cnt
                prof_acc[st][2] += cnt
            # (2b) the same kernels one after the other over K more steps: their shares of the
            # step (as in a serialised launch list) pick the dominant kernel
            iso = net.profile_steps(args.steps)
            kiso = {nm: iso[k] / args.steps for k, nm in enumerate(dtb.KERNELS)}
            for st, parts in stages.items():
                prof_acc[st][3] += sum(kiso[p] for p in parts)
            upd_ms = kms["neuron_update"]
            step_bytes = kb["neuron_update"] + kb["spike_deliver_rows"]
            deliver_ms = kms["spike_deliver"] + kms["queue_drain"]
            per_rate[str(r)] = {
                "gain": gain, "target_hz": r, "rate_hz": round(rate_hz, 3),
                "rate_ok": abs(rate_hz - r) <= RATE_TOL * r,
                "settle_steps": settle_steps[str(r)], "settle_rate_hz": round(settle_rate, 3),
                "ms_per_step": ms / args.steps,
                "synaptic_events_per_s": ev_all / (ms * 1e-3),
                "bio_s_per_wall_s": args.steps * dt_ms * 1e-3 / (ms * 1e-3),
                "wall_s_per_bio_s": (ms * 1e-3) / (args.steps * dt_ms * 1e-3),
                "hbm_frac_of_" + peak_kind: step_bytes / (ms * 1e-3 / args.steps) / (peak * 1e9),
                "kernel_ms": kms,
                "kernel_ms_source": f"dtb_step_timed over {args.steps} steps right after the timed region "
                                    f"({body} body launches per kernel)",
                "kernel_ms_isolated": kiso,
                "delivery_hbm_frac_isolated_of_" + peak_kind: (
                    kb["spike_delivery"] / ((kiso["spike_deliver"] + kiso["queue_drain"]) * 1e-3) / (peak * 1e9)),
                "neuron_update_gbs": kb["neuron_update"] / (upd_ms * 1e-3) / 1e9 if upd_ms else None,
                "delivery_hbm_frac_of_" + peak_kind: (kb["spike_delivery"] / (deliver_ms * 1e-3) / (peak * 1e9)
                                                      if deliver_ms else None),
            }
            # (3) end to end through the C ABI with host buffers, at the same
            # operating point: hyper-parameters in, raster and BOLD out, every
            # chunk of E2E_CHUNK steps
            ev0 = net.counters()[0]
            barrier()
            t0 = time.perf_counter()
            done = 0
            g_pin[:] = g_host
            while done < args.steps:
                c = min(chunk, args.steps - done)
                net.set_hyperparams(g_pin)
                h2d += g_pin.nbytes
                net.step(c)
                ids, off = net.get_spikes(c, ids_out=ids_buf, off_out=off_buf[: c + 1])
                y, _ = net.get_bold()
                d2h += ids.nbytes + off.nbytes + y.nbytes
                done += c
            barrier()
            dt_r, ev_r = aggregate(time.perf_counter() - t0, net.counters()[0] - ev0, device)
            e2e_s += dt_r
            ev_e2e += ev_r
            tot_ev += ev_all
            tot_ms += ms
            tot_steps += args.steps
            if rank == 0:
                print(f"[bench] {r} Hz: {json.dumps(per_rate[str(r)])}", file=sys.stderr, flush=True)

    # dominant kernel: the largest share of device time with the kernels one after the other (the
    # view of a serialised launch list); its achieved bandwidth from its launches in the timed,
    # pipelined schedule, over every rate
    dom = max(prof_acc, key=lambda k: prof_acc[k][3])
    iso_tot = sum(v[3] for v in prof_acc.values())
    dom_ms = prof_acc[dom][0] / max(prof_acc[dom][2], 1)
    dom_bytes = prof_acc[dom][1] / max(prof_acc[dom][2], 1)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = _traffic_record("+".join(stages[dom]), args.delivery)
    e2e_value = ev_e2e / e2e_s
    n_e2e_steps = args.steps * len(args.rates)
    ops_ok = all(v["rate_ok"] for v in per_rate.values())
    if rank == 0 and not ops_ok:
        print("[bench] WARNING: a rate missed its operating point by more than "
              f"{RATE_TOL:.0%}: " + ", ".join(f"{k} Hz -> {v['rate_hz']}" for k, v in per_rate.items()),
              file=sys.stderr, flush=True)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = _cpu_baseline()
        clk = clocks.summary()
        line = {
            "metric": METRIC, "value": tot_ev / (tot_ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / tot_steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded voxel network, device-generated)",
            "config": {"workload": f"{args.config}: {tb.n} neurons, {tb.nv} voxels, K={tb.K}, {tb.n * tb.K:.3g} "
                                   f"synapses, {wfmt} weights, delays 1-{tb.d_max}, dt {dt_ms} ms, rates "
                                   f"{list(args.rates)} Hz, {args.steps} steps each",
                       "delivery": args.delivery, "launch_shapes": args.shapes or "library default",
                       "schedule": "compaction beside the next update" if net.schedule_beside()
                       else "compaction after the update",
                       "settle_steps": settle_steps, "operating_points_ok": ops_ok,
                       "replicas": world, "l2": "inputs larger than L2 (60 GB CSR, 1.2 GB state per step)"},
            "per_rate": per_rate,
            "roofline": {"kernel": "+".join(stages[dom]), "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic, "algorithmic_bytes_per_launch": dom_bytes,
                         "avg_launch_ms": dom_ms, "launches": prof_acc[dom][2],
                         "share_serialised": prof_acc[dom][3] / iso_tot,
                         "source": "dominant by its share with the kernels one after the other "
                                   "(dtb_profile_steps); launch time from dtb_step_timed: CUDA events around "
                                   "every launch on its stream in the pipelined schedule of dtb_step, over every "
                                   "rate"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / n_e2e_steps,
                    "d2h_bytes_per_step": d2h / n_e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line))
    net.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=CONFIG)
    ap.add_argument("--rates", type=int, nargs="+", default=list(RATES))
    ap.add_argument("--wfmt", default=None)
    ap.add_argument("--delivery", default="bins", choices=["ring", "queue", "bins"])
    ap.add_argument("--schedule", type=int, default=-1, choices=[-1, 0, 1],
                    help="-1 by size, 0 compaction after the update, 1 beside the next update")
    ap.add_argument("--shapes", type=int, nargs=3, default=None, metavar=("STAGES", "UPD_PER_SM", "DEL_PER_SM"),
                    help="launch shapes (dtb_set_launch_shapes); default: the library's")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--neurons", type=int, default=None, help="scaled-down case (profiling only)")
    ap.add_argument("--voxels", type=int, default=None, help="scaled-down case (profiling only)")
    ap.add_argument("--indegree", type=int, default=None, help="scaled-down case (profiling only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
