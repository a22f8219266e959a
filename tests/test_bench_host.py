"""Host-side logic of bench.py, on the CPU: the algorithmic byte counts
against closed forms, the kernel-source hash that keys the committed ncu
traffic, the clock record's parsing, and the JSON line of the reference arm
(the FP64 oracle timed on the host cores)."""
import datetime
import json
import os
import shutil
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cell_counts_and_algorithmic_bytes():
    """301 x 901 interior + 40-cell CPML: padded 381 x 981; strips 2P x NZ and
    2P x NX; the 4-cell ring is (nz + 8)(nx + 8) - nz nx."""
    c = bench.counts(301, 901, 40)
    assert c["N_pad"] == 381 * 981 == 373761
    assert c["N_int"] == 301 * 901 == 271201
    assert c["N_x"] == 80 * 381 == 30480
    assert c["N_z"] == 80 * 981 == 78480
    assert c["N_ring"] == 309 * 909 - 301 * 901 == 9680
    # without a border the ring shrinks to the border width
    assert bench.counts(10, 12, 2)["N_ring"] == 14 * 16 - 10 * 12
    # per shot-step: forward 16 B per padded cell + 16 B per strip cell per
    # axis + 4 B per ring cell; backward adds 20 B per interior cell
    fwd, bwd = bench.alg_bytes_fwd(c), bench.alg_bytes_bwd(c)
    assert fwd == 16 * 373761 + 16 * (30480 + 78480) + 4 * 9680
    assert bwd - fwd == 20 * 271201
    assert 20 * bwd == 263725520  # the backward step of 20 shots


def test_interior_and_shared_k_figures():
    """Interior Gpts/s is the padded figure scaled by the interior share;
    with K counted once for the 20 shots the backward step of the workload
    reads 19 x 4 B fewer per padded cell."""
    c = bench.counts(301, 901, 40)
    assert bench.interior_gpts(373761.0, c) == pytest.approx(271201.0)
    assert bench.alg_bytes_k_once(bench.alg_bytes_bwd(c), c, 1) == bench.alg_bytes_bwd(c)
    assert bench.alg_bytes_k_once(bench.alg_bytes_bwd(c), c, 20) == 263725520 - 19 * 4 * 373761


def test_oracle_batch_sample_counts_padded_cell_steps():
    """The batch's CPU baseline times the oracle on the given problems with
    their records cut to nt_cap steps and counts padded cell-steps."""
    from paper_2604_14189_gb300 import inputs
    probs = inputs.workload_batch(count=2)
    for w in probs:  # keep it small: 12 x 14 interiors, 3-cell borders
        w.update(nz=12, nx=14, pml=3, model=w["model"][:12, :14],
                 src=w["src"][:1] % [12, 14], rec=w["rec"][:1, :14] % [12, 14])
    g, el, cores, sample = bench.oracle_batch_sample(probs, 7)
    assert el > 0 and cores >= 1
    # two problems of 18 x 20 padded cells, 7 steps, one shot each
    assert g == pytest.approx(2 * 18 * 20 * 7 * 1 / el / 1e9)
    assert "first 2 problems" in sample and "7 steps" in sample


def _scratch_root(tmp_name):
    d = os.path.join(ROOT, "_build", tmp_name)
    if os.path.exists(d):
        shutil.rmtree(d)
    src = os.path.join(ROOT, "paper_2604_14189_gb300", "csrc")
    dst = os.path.join(d, "paper_2604_14189_gb300", "csrc")
    shutil.copytree(src, dst, ignore=lambda p, names: [n for n in names
                                                       if n not in bench.KERNEL_SOURCES])
    return d, dst


def test_kernel_source_hash_ignores_comments_not_code(monkeypatch):
    base = bench.kernel_source_hash()
    root, csrc = _scratch_root("hash_check")
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.kernel_source_hash() == base
    path = os.path.join(csrc, "acoustic_cpml.cuh")
    src = open(path).read()
    with open(path, "w") as f:
        f.write("// a new comment\n/* and a block\n comment */\n" + src.replace("\n", "\n\n", 3))
    assert bench.kernel_source_hash() == base
    assert "constexpr int FT = 128;" in src
    with open(path, "w") as f:
        f.write(src.replace("constexpr int FT = 128;", "constexpr int FT = 64;"))
    assert bench.kernel_source_hash() != base


def test_traffic_read_only_for_the_profiled_sources(monkeypatch):
    kv = dict(l.split(":", 1) for l in open(bench.TRAFFIC_FILE) if ":" in l)
    stated = kv["kernel_source_hash"].strip()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: stated)
    t = bench.read_traffic()
    assert t == float(kv["dram_bytes_per_launch"]) and t > 0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.read_traffic() is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_summary(monkeypatch):
    """Samples outside the marked timed region are dropped; the median is
    taken over loaded samples; throttle reasons seen inside are listed."""
    os.makedirs(os.path.join(ROOT, "_build"), exist_ok=True)
    path = os.path.join(ROOT, "_build", "clock_record_test.csv")
    monkeypatch.setattr(bench.tempfile, "NamedTemporaryFile", lambda *a, **k: open(path, "w+"))
    s = bench.ClockSampler(0)
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    s.t0, s.t1 = t0, t0 + datetime.timedelta(seconds=2)

    def row(dt, sm, pcap="Not Active", hw="Not Active"):
        ts = (t0 + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {sm}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {pcap}\n"
    s.f.write(row(-3, 345, hw="Active"))   # before the region: dropped
    s.f.write(row(0.2, 2070))
    s.f.write(row(0.6, 2040, pcap="Active"))
    s.f.write(row(1.0, 345))               # idle sample: not a loaded one
    s.f.write(row(1.4, 2055))
    s.f.write(row(9.0, 300, hw="Active"))  # after the region: dropped
    s.f.flush()
    s.proc = _Done()
    out = s.stop()
    assert out["samples"] == 4
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2055.0
    assert out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(path)  # the record is removed once summarised


def test_reference_arm_json_line():
    """`bench.py --impl reference`: one JSON line, the oracle's throughput on
    the benchmark's workload, host-only (no device copies)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "Gpts/s fwd+adj" and d["unit"] == "Gpts/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert "301x901" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("rank", [1])
def test_reference_arm_other_ranks_exit_quietly(rank):
    """Under torchrun only rank 0 runs and prints the reference arm."""
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
