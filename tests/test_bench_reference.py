"""The bench's reference arm (the CPU oracle, bench.py --impl reference) on
the host: one JSON line with the contract's keys, run as the driver runs it
(no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_banded_lu_storage_matches_the_oracle_matrix_bandwidth():
    # The band storage the bench reports for the full-size workloads uses the
    # half-bandwidth nx*ny + nx + 1 of the 27-point operator in x-fastest
    # order; the oracle's assembled matrix on a small anisotropic grid has
    # exactly that bandwidth on both sides.
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import operator as O
    from oracle import weights as W
    nodes, T = W.fit_table()
    nz, ny, nx = 5, 4, 6
    v = np.full((nz, ny, nx), 2000.0, np.float32)
    prof = O.profiles_for(v.shape, 25.0, (1,) * 6, 2000.0, 1e-3)
    A = O.assemble_csr(v, 25.0, 6.0, prof, T, nodes).tocoo()
    kl = nx * ny + nx + 1
    assert int((A.row - A.col).max()) == kl and int((A.col - A.row).max()) == kl
    assert bench.banded_lu_bytes(nx, ny, nz) == (3 * kl + 1) * nx * ny * nz * 16
