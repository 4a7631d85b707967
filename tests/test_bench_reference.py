"""Host logic of bench.py: the reference arm times the oracle alone (no GPU,
no library of the package), and the window-to-grid face index map used to
compare the 3D column with the oracle's window solve."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_runs_the_oracle_only():
    code = r"""
import json, sys
sys.path.insert(0, %r)
import bench
bench.oracle_pcg_count = lambda n: (40, {"rows": {}, "header": []})
from argparse import Namespace
out = bench.run_reference(Namespace(workload="bumps1024", warmup=0, steps=1, ref_size=48,
                                   ref_complete_size=24))
loaded = sorted(m for m in sys.modules if m.startswith("paper_1010_2832_gb300"))
print(json.dumps({"out": out, "loaded": loaded, "torch": "torch" in sys.modules}))
""" % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["loaded"] == ["paper_1010_2832_gb300", "paper_1010_2832_gb300.workloads"]
    assert not d["torch"]
    out = d["out"]
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0
    for k in ("disk32_config1_all_cores", "bumps24_one_thread"):
        assert out["cpu_baseline"]["complete_solves"][k]["rel_residual"] <= 1e-8


def test_window_face_index_map():
    import bench
    n, win = 12, (3, 2, 4, 5, 6, 4)
    i0, j0, k0, ni, nj, nk = win
    wsh = [(nk, nj, ni + 1), (nk, nj + 1, ni), (nk + 1, nj, ni)]
    fsh = [(n, n, n + 1), (n, n + 1, n), (n + 1, n, n)]
    # a field whose value encodes the full-grid position of every face
    full = [np.fromfunction(lambda k, j, i, d=d: 1e6 * d + 1e4 * k + 1e2 * j + i, s) for d, s in enumerate(fsh)]
    win_vals = [f[k0:k0 + w[0], j0:j0 + w[1], i0:i0 + w[2]] for f, w in zip(full, wsh)]
    flat_full = np.concatenate([f.ravel() for f in full])
    flat_win = np.concatenate([f.ravel() for f in win_vals])
    idx = np.arange(flat_win.size)
    assert np.array_equal(flat_full[bench.window_face_to_full(idx, n, win)], flat_win)


def test_kernel_source_hash_follows_the_kernel_and_its_argument_types(tmp_path):
    """The stored ncu traffic of the local-solve kernel is reported only while
    the hash of its sources matches: the hash changes with the kernel's files
    and with the definitions of the types it takes (Layout, CgScalars), and
    not with other declarations of the shared header."""
    import shutil
    import bench
    src = os.path.join(ROOT, "paper_1010_2832_gb300", "csrc")
    for f in ("schwarz.cuh", "schwarz_plan.cuh", "internal.cuh"):
        shutil.copy(os.path.join(src, f), tmp_path / f)
    h0 = bench.kernel_source_hash("k_schwarz_gemv", str(tmp_path))
    assert h0 == bench.kernel_source_hash("k_schwarz_gemv")
    internal = (tmp_path / "internal.cuh").read_text()
    # another declaration of the header: same hash
    (tmp_path / "internal.cuh").write_text(internal.replace("struct ApplyArgs {", "struct ApplyArgs {\n    int unused_;"))
    assert bench.kernel_source_hash("k_schwarz_gemv", str(tmp_path)) == h0
    # a field of Layout: new hash
    (tmp_path / "internal.cuh").write_text(internal.replace("    int ntx, nty, ntz;", "    int ntx, nty, ntz, extra;"))
    assert bench.kernel_source_hash("k_schwarz_gemv", str(tmp_path)) != h0
    (tmp_path / "internal.cuh").write_text(internal)
    # the kernel's own file: new hash
    with open(tmp_path / "schwarz.cuh", "a") as f:
        f.write("\n// edit\n")
    assert bench.kernel_source_hash("k_schwarz_gemv", str(tmp_path)) != h0
