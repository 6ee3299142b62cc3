"""The FP32 form's FP64 <-> FP32 conversions by bit operations
(csrc/fp_bits.cuh), compiled for the host from the same header the kernels
use and checked against numpy's IEEE conversions: narrowing equals rounding
toward zero (numpy's round-to-nearest result, stepped toward zero where it
rounded away) on every finite magnitude in [2^-126, 2^128), with the
documented ends (below 2^-126 a signed zero, at or above 2^128 and infinity
an infinity, NaN a NaN); widening of non-negative floats is exact for normal
values, 0 below 2^-126, and at least 2^128 for infinity and NaN; widening of
any float is exact for normal values and zeros, a signed zero for subnormal
values, and keeps infinities and NaN."""
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


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fpbits") / "fp_bits_probe")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "fp_bits_probe.cu"), "-o", exe],
                   check=True, capture_output=True)

    def run(x, b):
        x = np.ascontiguousarray(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float32)
        assert x.size == b.size
        d = tmp_path_factory.mktemp("io")
        fin, fout = str(d / "in.bin"), str(d / "out.bin")
        with open(fin, "wb") as f:
            f.write(np.int64(x.size).tobytes() + x.tobytes() + b.tobytes())
        subprocess.run([exe, fin, fout], check=True)
        raw = open(fout, "rb").read()
        y = np.frombuffer(raw[:4 * x.size], dtype=np.float32)
        w = np.frombuffer(raw[4 * x.size:12 * x.size], dtype=np.float64)
        g = np.frombuffer(raw[12 * x.size:], dtype=np.float64)
        return y, w, g
    return run


def _rz(x):
    with np.errstate(over="ignore"):
        y = x.astype(np.float32)
    away = np.abs(y.astype(np.float64)) > np.abs(x)
    y[away] = np.nextafter(y[away], np.float32(0))
    return y


def _inputs(seed):
    rng = np.random.default_rng(seed)
    n = 200_000
    mag = np.exp2(rng.uniform(-140.0, 140.0, n))
    x = mag * rng.choice([-1.0, 1.0], n)
    ends = np.array([0.0, -0.0, 2.0 ** -126, -(2.0 ** -126), np.nextafter(2.0 ** -126, 0),
                     2.0 ** -149, 5e-324, 2.0 ** 128, np.nextafter(2.0 ** 128, 0),
                     -np.nextafter(2.0 ** 128, 0), float(np.finfo(np.float32).max), 1e300, -1e300,
                     np.inf, -np.inf, np.nan, 1.0, -1.0, 1e-12, 1e-12 + 1e-30, 178.5, 1.0 + 2.0 ** -24,
                     1.0 + 2.0 ** -23 + 2.0 ** -24, 1.0 - 2.0 ** -25])
    # values on and next to FP32 grid points (exact, halfway, just off)
    f = rng.uniform(-1e4, 1e4, 2000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    grid = np.concatenate([f, f + 0.5 * ulp, f - 0.5 * ulp, np.nextafter(f, np.inf), np.nextafter(f, -np.inf)])
    x = np.concatenate([x, ends, grid])
    bm = np.exp2(rng.uniform(-150.0, 128.0, x.size)).astype(np.float32)
    bends = np.array([0.0, 2.0 ** -149, 2.0 ** -127, 2.0 ** -126, 1.0, float(np.finfo(np.float32).max),
                      np.inf, np.nan], dtype=np.float32)
    bm[:bends.size] = bends
    return x, bm


def test_narrowing_rounds_toward_zero(probe):
    x, b = _inputs(3)
    y, _, _ = probe(x, b)
    ax = np.abs(x)
    normal = (ax >= 2.0 ** -126) & (ax < 2.0 ** 128)
    assert normal.sum() > 150_000
    want = _rz(x[normal])
    assert np.array_equal(y[normal].view(np.uint32), want.view(np.uint32))
    small = ax < 2.0 ** -126
    assert np.all(y[small] == 0) and np.array_equal(np.signbit(y[small]), np.signbit(x[small]))
    big = (ax >= 2.0 ** 128) & ~np.isnan(x)
    assert np.all(np.isinf(y[big])) and np.array_equal(np.signbit(y[big]), np.signbit(x[big]))
    assert np.all(np.isnan(y[np.isnan(x)]))
    # against round-to-nearest: never farther than one FP32 step, never larger in magnitude
    with np.errstate(over="ignore"):
        yn = x[normal].astype(np.float32)
    assert np.all(np.abs(y[normal].astype(np.float64)) <= ax[normal])
    assert np.all(np.abs(y[normal].view(np.int32).astype(np.int64) - yn.view(np.int32).astype(np.int64)) <= 1)


def test_widening_is_exact_for_normal_values(probe):
    x, b = _inputs(5)
    _, w, _ = probe(x, b)
    normal = (b >= 2.0 ** -126) & np.isfinite(b)
    assert normal.sum() > 150_000
    assert np.array_equal(w[normal], b[normal].astype(np.float64))
    assert np.all(w[b < 2.0 ** -126] == 0.0)
    special = ~np.isfinite(b)
    assert special.sum() == 2 and np.all(w[special] >= 2.0 ** 128) and np.all(np.isfinite(w[special]))


def test_signed_widening(probe):
    x, b = _inputs(7)
    rng = np.random.default_rng(8)
    b = b * rng.choice(np.array([-1.0, 1.0], dtype=np.float32), b.size)
    b[:4] = np.array([-0.0, -np.inf, -(2.0 ** -140), -(2.0 ** -126)], dtype=np.float32)
    _, _, g = probe(x, b)
    a = np.abs(b)
    normal = (a >= 2.0 ** -126) & np.isfinite(b)
    assert normal.sum() > 150_000 and (b[normal] < 0).sum() > 50_000
    assert np.array_equal(g[normal], b[normal].astype(np.float64))
    sub = a < 2.0 ** -126
    assert np.all(g[sub] == 0.0) and np.array_equal(np.signbit(g[sub]), np.signbit(b[sub]))
    inf = np.isinf(b)
    assert np.array_equal(g[inf], b[inf].astype(np.float64))
    assert np.all(np.isnan(g[np.isnan(b)]))
