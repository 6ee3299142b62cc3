"""The kernels' index decomposition r = (k e1 + j) e0 + i (split3 in
csrc/awe_internal.cuh: unsigned 32-bit divisions while r fits in 32 bits,
64-bit ones beyond), compiled for the host from the same header and checked
against Python's integer divmod on both sides of 2^32 and at its edges."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2211_13295_gb300", "csrc")


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_split3_matches_divmod(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "index_probe")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "index_probe.cu"), "-o", exe],
                   check=True, capture_output=True)
    rng = np.random.default_rng(11)
    n = 100_000
    e0 = rng.integers(1, 4100, n).astype(np.int32)
    e1 = rng.integers(1, 4100, n).astype(np.int32)
    r = np.concatenate([rng.integers(0, 2 ** 32, n // 2), rng.integers(2 ** 32, 2 ** 40, n - n // 2)])
    edges = np.array([0, 1, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1, 2 ** 32, 2 ** 32 + 1, 2 ** 40])
    r[:edges.size] = edges
    e0[:edges.size] = 258
    e1[:edges.size] = 258
    r = r.astype(np.int64)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        f.write(np.int64(n).tobytes() + r.tobytes() + np.stack([e0, e1], axis=1).astype(np.int32).tobytes())
    subprocess.run([exe, fin, fout], check=True)
    got = np.frombuffer(open(fout, "rb").read(), dtype=np.int32).reshape(n, 3)
    t, i = np.divmod(r, e0.astype(np.int64))
    k, j = np.divmod(t, e1.astype(np.int64))
    assert np.array_equal(got[:, 0], i) and np.array_equal(got[:, 1], j)
    fits = k < 2 ** 31
    assert fits.sum() > n // 2
    assert np.array_equal(got[fits, 2], k[fits])
