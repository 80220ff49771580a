"""bench.py without a GPU: the smoother's algorithmic-byte accounting and the
reference arm's JSON line (the CPU oracle on a tiny crop of the workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smooth_bytes_counts_the_correction_reads():
    sys.path.insert(0, ROOT)
    import bench
    from paper_0710_0736_gb300 import ac

    class Prof:
        pass

    p = Prof()
    p.launches = [0] * len(ac.PROF_CLASSES)
    p.launches[ac.PROF_CLASSES.index("smooth")] = 12
    p.smooth_bytes_per_launch = 1000.0
    p.smooth_corr_launches = 2
    p.smooth_corr_extra_bytes = 250.0
    # 12 launches of one colour each, two of which also read the other colour's correction
    assert bench.smooth_bytes(p) == 12 * 1000.0 + 2 * 250.0


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--crop", "24"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "steps/s"
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["nodes"] == 4097 * 4097


RANK_SCRIPT = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo", rank=rank, world_size=2)
rate, ms_max = bench.job_rate([100.0, 250.0][rank], [3, 5][rank], 2, "cpu")
dist.barrier()
dist.destroy_process_group()
print(f"RESULT {rank} {rate!r} {ms_max!r}", flush=True)
"""


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_rate_over_two_gloo_ranks():
    """The replicas' whole-job rate: units summed over the ranks, divided by the
    slowest rank's time (bench.py's aggregation, here over two gloo ranks)."""
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=300)
            assert p.returncode == 0, err[-2000:]
            outs.append(out)
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for out in outs:
        line = [l for l in out.splitlines() if l.startswith("RESULT")][0].split()
        rate, ms_max = float(line[2]), float(line[3])
        assert ms_max == 250.0
        assert rate == pytest.approx((3 + 5) / 0.25)  # 8 units in the slowest rank's 250 ms
