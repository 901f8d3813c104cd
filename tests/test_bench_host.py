"""Host logic of bench.py that needs no GPU: the kernel-source hash that keys
the recorded ncu traffic (comments and the SpMM and vector-reordering
sections do not change it, any other code does) and the traffic lookup."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KERNELS = os.path.join(ROOT, "paper_1103_2405_gb300", "csrc", "kernels.cu")


def _src():
    with open(KERNELS, encoding="utf-8") as fh:
        return fh.read()


def test_hash_ignores_comments_and_the_excluded_sections():
    text = _src()
    h = bench.kernel_source_sha(text)
    assert h == bench.kernel_source_sha()
    assert bench.kernel_source_sha(text.replace("// Solution 3", "// Solution three")) == h
    spmm = text.index("// " + "-" * 66 + " SpMM --")
    vec = text.index("// " + "-" * 61 + " vectors --")
    for at in (spmm, vec):
        i = text.index("\n__global__", at) + 1
        edited = text[:i] + "__device__ int spg_hash_probe;\n" + text[i:]
        assert bench.kernel_source_sha(edited) == h


def test_hash_changes_with_the_iteration_kernels():
    text = _src()
    h = bench.kernel_source_sha(text)
    i = text.index("k_part_staged(PartView pv")
    j = text.index("{", i) + 1
    edited = text[:j] + "\n    int spg_hash_probe = 0; (void)spg_hash_probe;" + text[j:]
    assert bench.kernel_source_sha(edited) != h


def test_traffic_is_reported_only_for_the_recorded_source():
    for w, (bytes_, sha) in bench.NCU_TRAFFIC.items():
        assert bytes_ > 0
        assert bench.ncu_traffic(w) == (bytes_ if sha == bench.kernel_source_sha() else None)
    assert bench.ncu_traffic("no such workload") is None


def test_reference_arm_prints_one_contract_line():
    # the reference arm (the FP64 oracle, timed on the host) on the small
    # R-MAT workload: one JSON line with the contract's keys
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "rmat14", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
