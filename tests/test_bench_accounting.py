"""The algorithmic bytes bench.py divides by kernel time for its roofline
figures, checked against the per-unit definitions they follow (neuron state
read and written, spike bits, binned arrival events; synapse rows and the
accumulator read-modify-write per event; ids and work items per spike), the
traffic record's check of the kernel sources and delivery mode, the clocks
record taken from nvidia-smi samples, and the line the reference arm (the
oracle on the host cores) prints."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_neuron_update_bytes_per_mode():
    n, spikes, events = 20_000_000, 30_000.0, 15_000_000.0
    q = bench._kernel_bytes({}, n, 2, 2, spikes, events, "queue")
    b = bench._kernel_bytes({}, n, 2, 2, spikes, events, "bins")
    # V 4 + j 16 + ref 1 + two accumulator rows 8, read and written, + a spike bit
    assert q["neuron_update"] == n * 58 + n / 8
    # bins: no accumulator rows; every arrival event is read once (4 bytes)
    assert b["neuron_update"] == n * 42 + n / 8 + events * 4
    # int32 weights: two-word bin events
    assert bench._kernel_bytes({}, n, 2, 4, spikes, events, "bins")["neuron_update"] == n * 42 + n / 8 + events * 8
    # four channels widen only the accumulator rows of the queue and ring modes
    assert bench._kernel_bytes({}, n, 4, 2, spikes, events, "queue")["neuron_update"] == n * 74 + n / 8


def test_delivery_and_compaction_bytes():
    n, spikes, events = 1_000_000, 1_500.0, 750_000.0
    kb = bench._kernel_bytes({}, n, 2, 2, spikes, events, "bins")
    rows = spikes * 16 + events * (4 + 2)
    assert kb["spike_deliver_rows"] == rows
    assert kb["spike_delivery"] == rows + events * 8  # + accumulator read-modify-write per event
    assert kb["spike_compact"] == n / 8 + 4 * n / 1024 + 8 * spikes


def test_traffic_record_matches_sources_and_mode():
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    csrc = os.path.join(ROOT, "paper_2308_01241_gb300", "csrc")
    sk = open(os.path.join(csrc, "step_kernels.cu"), "rb").read()
    upd = sk[:sk.index(b"// ==== end of the neuron update ====")]
    assert b"neuron_update_kernel(DevNet g" in upd and b"spike_deliver_runs_kernel" not in upd
    src = upd + open(os.path.join(csrc, "dtb_device.cuh"), "rb").read()
    current = rec["source_sha256"] == hashlib.sha256(src).hexdigest()
    got = bench._traffic_record("neuron_update", rec["delivery"])
    assert got == (rec["kernels"]["neuron_update"] if current else None)
    other = "queue" if rec["delivery"] != "queue" else "bins"
    assert bench._traffic_record("neuron_update", other) is None


def test_traffic_record_follows_the_update_source_only(tmp_path, monkeypatch):
    """An edit after the end-of-update marker (delivery, binning) keeps the
    record; an edit of the update's part of the file drops it."""
    import shutil

    csrc = os.path.join(ROOT, "paper_2308_01241_gb300", "csrc")
    dst = tmp_path / "paper_2308_01241_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("step_kernels.cu", "dtb_device.cuh"):
        shutil.copy(os.path.join(csrc, f), dst / f)
    (tmp_path / "profiles").mkdir()
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec["source_sha256"] = bench.update_source_sha256()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    want = rec["kernels"]["neuron_update"]
    assert bench._traffic_record("neuron_update", rec["delivery"]) == want
    sk = (dst / "step_kernels.cu").read_text()
    (dst / "step_kernels.cu").write_text(sk + "\n// a change after the update\n")
    assert bench._traffic_record("neuron_update", rec["delivery"]) == want
    (dst / "step_kernels.cu").write_text("// a change before the update\n" + sk)
    assert bench._traffic_record("neuron_update", rec["delivery"]) is None


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the contract's keys, its own value repeated in cpu_baseline and e2e."""
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "8",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 8 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"]


def test_clock_summary_parses_samples_and_active_reasons(tmp_path):
    """The clocks record: median SM clock under load, the max clock, and the
    throttle reasons seen Active in any sample ("Not Active" is not one)."""
    rows = [
        "0, 1965, 2070, 900.1, 0x0000000000000004, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
    ]
    f = tmp_path / "clocks.csv"
    f.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)

    class _F:
        name = str(f)

    cs.file = _F()
    s = cs.summary()
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_launch_count_of_one_call():
    """Kernels of one dtb_step(k): the call's start, five per step (four in
    ring mode), one step-counter advance for the first step and one per chunk
    of up to 32 further steps, and the closing j-only update and flag clear."""
    assert bench.launches_per_call(1, "bins") == 1 + 5 + 1 + 2
    assert bench.launches_per_call(33, "bins") == 1 + 5 * 33 + 1 + 1 + 2
    assert bench.launches_per_call(34, "queue") == 1 + 5 * 34 + 1 + 2 + 2
    assert bench.launches_per_call(20, "ring") == 1 + 4 * 20 + 1 + 1 + 2
    assert bench.launches_per_call(0, "bins") == 1


class _FakeNet:
    """Spike counter of a network whose rate follows a given function of the
    step count (host logic of the settle only)."""

    def __init__(self, n, dt_ms, rate_of_step):
        self.n, self.dt_ms, self.rate_of_step = n, dt_ms, rate_of_step
        self.t = 0
        self.spikes = 0.0

    def step(self, k):
        for _ in range(k):
            self.spikes += self.rate_of_step(self.t) * self.n * self.dt_ms * 1e-3
            self.t += 1

    def counters(self):
        return 0, self.spikes, self.t


def test_settle_runs_its_steps_then_probes_until_the_rate_is_on_target():
    net = _FakeNet(1000, 0.1, lambda t: 50.0 if t < 4000 else 15.0)
    done, rate = bench.settle(net, 1000, 0.1, 15, steps=3000, probe=500, extra=4)
    assert (done, round(rate, 6)) == (4500, 15.0)  # two probes at 50 Hz, the third on target
    net = _FakeNet(1000, 0.1, lambda t: 7.2)
    assert bench.settle(net, 1000, 0.1, 7, steps=3000, probe=500, extra=4)[0] == 3500
    net = _FakeNet(1000, 0.1, lambda t: 40.0)  # never on target: gives up after the extra windows
    done, rate = bench.settle(net, 1000, 0.1, 30, steps=1000, probe=500, extra=2)
    assert done == 2500 and abs(rate - 40.0) < 1e-9
