"""Host-side logic of bench.py, without a GPU: the flop count behind the
roofline, the source hash that keeps a stored DRAM capture tied to the code it
was taken on, the parsing of the clock samples, and the JSON line of the
reference (oracle) arm."""
import json
import subprocess
import sys
from types import SimpleNamespace

import pytest

import bench


def test_update_flops_counts_every_trailing_entry():
    """Each block step J updates the lower triangle of the rows below its
    panel, 2*nb flops per entry; counted entry by entry on small sizes."""
    for n, nb in ((1, 4), (4, 4), (5, 4), (13, 4), (300, 128), (257, 128)):
        want = 0
        for J in range(0, n, nb):
            lo = J + nb
            for i in range(lo, n):
                want += 2 * nb * (i - lo + 1)
        assert bench.update_flops(n, nb) == want, (n, nb)


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {\n  // add one\n  return x + 1; /* trailing\n block */\n}\n"
    b = "int f(int x) { return x + 1; }"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(b) != bench._code_only(c)


def test_stored_traffic_follows_the_source(monkeypatch):
    """The committed capture is scaled by the units of a launch while its
    source hash matches, and is dropped (None) once the kernel changed."""
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        ent = json.load(f)["k_split_gemm<update>"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files: ent["source_hash"])
    got = bench.stored_traffic("k_split_gemm<update>", ent["source_files"], 5456)
    assert got == pytest.approx(ent["bytes_per_tile"] * 5456)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files: "0" * 16)
    assert bench.stored_traffic("k_split_gemm<update>", ent["source_files"], 5456) is None
    assert bench.stored_traffic("no_such_kernel", ent["source_files"], 5456) is None


def test_kernel_source_hash_reads_the_named_files():
    h = bench.kernel_source_hash(["k_gemm.cu", "mixed_common.cuh"])
    assert len(h) == 16 and int(h, 16) >= 0
    assert h != bench.kernel_source_hash(["k_gemm.cu"])


def test_clock_samples_are_parsed(tmp_path):
    rows = [
        "0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1950, 2070, 1210.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbled line",
    ]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc, s.path = _Done(), str(p)
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 1965.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert not p.exists()


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_line(capsys):
    """The reference arm (the oracle on the host) prints one JSON line with
    the contract's keys, on a small case."""
    args = SimpleNamespace(n=96, T=8, steps=2, warmup=1, gpus=1, workload="hartman")
    assert bench.run_reference(args) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "evals/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "evals/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["n"] == 96 and line["config"]["T"] == 8


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = SimpleNamespace(n=96, T=8, steps=1, warmup=1, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_bench_help_runs_without_a_gpu():
    r = subprocess.run([sys.executable, bench.os.path.join(bench.ROOT, "bench.py"), "--help"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "--impl" in r.stdout


def test_variance_flops_counts_every_block_and_tile_row():
    """The variance solve's flop counts against an explicit sum: per point
    block and tile row J the update is 15 products of 128 x 128 x 128 J, the
    diagonal step 28 products of 128 x 128 x 128; the method's n^2 N."""
    import bench
    for n, N in ((1, 1), (128, 128), (300, 129), (4000, 1000)):
        nt, blocks = -(-n // 128), -(-N // 128)
        want = 0
        for _ in range(blocks):
            for J in range(nt):
                want += 15 * 2 * 128 * 128 * (128 * J) + 28 * 2 * 128 ** 3
        method, executed = bench.variance_flops(n, N)
        assert executed == want and method == float(n) * n * N
