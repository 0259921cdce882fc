"""Host-side contract of the bench's reference arm (the FP64 CPU oracle, no GPU): one JSON
line with the GPU arm's metric, unit, higher_is_better and workload config, plus the
reference keys (impl, cpu_baseline, e2e with zero copies)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_matches_the_gpu_arm_contract():
    import bench
    from paper_2604_25775_gb300 import inputs as I
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC
    assert line["unit"] == "E_loc/s" and line["higher_is_better"] is True
    # the same workload description the GPU arm prints for its default run
    assert line["config"] == bench.workload_config(I.workload("hubbard16x16"), "hubbard16x16", 8192, 1)
    assert line["value"] > 0 and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_workload_config_names_the_sizes():
    import bench
    from paper_2604_25775_gb300 import inputs as I
    c = bench.workload_config(I.workload("hubbard16x16"), "hubbard16x16", 8192, 2)
    assert c["workload"] == "hubbard16x16: 16x16 torus, U=8, 112+112, SCALE 1 conv 3x3 + 5 site-wise, h=32"
    assert c["walkers"] == 8192 and c["parallelism"] == "replicas x2"
    assert c["l2"] == "inputs larger than L2 (cached inverses 1.6 GB)"


def test_precision_modes_of_the_bench():
    """The bench's --precision names map onto the library's mixed modes, each with a dtype
    description naming its site-wise tensor-core products; without the option the workload's
    own mode runs (FP16x3 for the 16x16 workload)."""
    import bench
    from paper_2604_25775_gb300 import inputs as I
    assert bench.PRECISIONS == {"mixed": I.PREC_MIXED, "mixed_fp16": I.PREC_MIXED_FP16,
                                "mixed_bf16": I.PREC_MIXED_BF16}
    for name, mode in bench.PRECISIONS.items():
        word = {"mixed": "tf32", "mixed_fp16": "f16", "mixed_bf16": "bf16"}[name]
        assert f"3 {word} tensor-core products" in bench.DTYPES[mode]
    assert I.workload("hubbard16x16").precision == I.PREC_MIXED_FP16
