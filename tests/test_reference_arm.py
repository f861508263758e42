"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"].startswith("GN Hessian-vector products/s")
    assert d["unit"] == "Hv/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Hv/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_stored_stage_traffic_belongs_to_the_current_kernel_sources():
    """bench.py reports the ncu DRAM bytes of the stage kernels only for the
    kernel sources they were measured on; the stored entry must name the
    digest of the committed sources, or the line's roofline.traffic is null."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.TRAFFIC["digest"] == bench.kernel_digest()
    for k in ("tangent_stage_fused", "adjoint_stage_fused"):
        assert 1e8 < bench.TRAFFIC[k] < 1e9
