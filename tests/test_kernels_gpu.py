"""GPU checks of kernel building blocks through the C ABI (no oracle needed)."""
import os

import numpy as np
import pytest
from scipy import special

from paper_1807_02718_gb300 import fh as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1807_02718_gb300 import build
    build.build()
    F.load_library()


def test_bessel_routine_table(golden_dir):
    """The kernels' J0, Y0, J1, Y1 at the A&S Table 9.1 arguments."""
    rows = np.loadtxt(os.path.join(golden_dir, "bessel_table.txt"))
    out = F.fh_eval_bessel(rows[:, 0])
    # table columns are J0, J1, Y0, Y1; the routine returns J0, Y0, J1, Y1
    assert np.max(np.abs(out[:, [0, 2, 1, 3]] - rows[:, 1:5])) < 1e-15
    assert np.max(np.abs(out[:, 4:6] - rows[:, [1, 3]])) < 1e-15


def test_bessel_routine_dense_grid():
    """Against scipy over the argument range of the workloads (0 < x <= 2000),
    including both sides of the branch points x = 8 and x = 20."""
    x = np.concatenate([np.geomspace(1e-6, 8, 4000), np.linspace(7.99, 8.01, 101),
                        np.linspace(8, 40, 6000), np.linspace(19.99, 20.01, 101),
                        np.geomspace(40, 2000, 4000)])
    out = F.fh_eval_bessel(x)
    ref = np.stack([special.j0(x), special.y0(x), special.j1(x), special.y1(x)], 1)
    scale = np.maximum(1.0, np.abs(ref))
    err = np.abs(out[:, :4] - ref) / scale
    # scipy's own routines carry up to ~1e-15 absolute error in this range
    assert np.max(err) < 4e-15, np.max(err, axis=0)
    assert np.array_equal(out[:, 4:6], out[:, [0, 1]])
    # Wronskian J1 Y0 - J0 Y1 = 2/(pi x): an identity independent of scipy
    w = out[:, 2] * out[:, 1] - out[:, 0] * out[:, 3]
    assert np.max(np.abs(w * np.pi * x / 2 - 1)) < 5e-13


def test_double_float_hankel_form():
    """The double-float (FP32-pair) Hankel form of the mixed-precision kernels
    against the FP64 routine and scipy for 8 <= x <= 2000: ~1e-13 absolute,
    the budget that keeps the mixed path within 1e-10 of the oracle."""
    x = np.concatenate([np.linspace(8, 8.01, 101), np.linspace(8, 40, 8000),
                        np.linspace(9.99, 10.01, 51), np.linspace(59.99, 60.01, 51),
                        np.geomspace(40, 2000, 6000)])
    out = F.fh_eval_bessel_df(x)
    ref64 = F.fh_eval_bessel(x)[:, :4]
    ref = np.stack([special.j0(x), special.y0(x), special.j1(x), special.y1(x)], 1)
    assert np.max(np.abs(out - ref64)) < 2e-13, np.max(np.abs(out - ref64), axis=0)
    assert np.max(np.abs(out - ref)) < 2e-13
    w = out[:, 2] * out[:, 1] - out[:, 0] * out[:, 3]
    assert np.max(np.abs(w * np.pi * x / 2 - 1)) < 1e-11


def test_double_float_small_argument_series():
    """Below x = 8 the double-float path sums the same Chebyshev series as the
    FP64 routine (double-float head, binary32 tail) with a double-float
    logarithm: within ~1e-13 of the FP64 routine and scipy, relative to
    max(1, |value|) (Y0, Y1 grow like ln x and 1/x near 0)."""
    x = np.concatenate([np.geomspace(1e-3, 0.5, 400), np.linspace(0.5, 8.0, 4000, endpoint=False),
                        np.linspace(7.99, 8.0, 50, endpoint=False), [1.0, 2.0, 4.0, 1 / np.sqrt(2)]])
    out = F.fh_eval_bessel_df(x)
    ref64 = F.fh_eval_bessel(x)[:, :4]
    ref = np.stack([special.j0(x), special.y0(x), special.j1(x), special.y1(x)], 1)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.max(np.abs(out - ref64) / scale) < 2e-13, np.max(np.abs(out - ref64) / scale, axis=0)
    assert np.max(np.abs(out - ref) / scale) < 2e-13, np.max(np.abs(out - ref) / scale, axis=0)
    w = out[:, 2] * out[:, 1] - out[:, 0] * out[:, 3]     # Wronskian 2 / (pi x)
    assert np.max(np.abs(w * np.pi * x / 2 - 1)) < 1e-12


def test_fp64_peak_probe_runs():
    v = F.fh_probe_fma_peak(0, True, 256)
    assert v > 0.1


def _bf16(a):
    """Round float32 to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 512, 192)])
def test_tcgen05_gemm_bf16(M, N, K):
    """BF16 products are exact and accumulate in FP32: C = A B^T to FP32 rounding."""
    rng = np.random.default_rng(M + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C = F.fh_tc_gemm_test(1, A, B)
    ref = _bf16(A) @ _bf16(B).T
    assert np.max(np.abs(C - ref)) < 1e-5 * np.sqrt(K) * np.max(np.abs(ref))


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 128)])
def test_tcgen05_gemm_tf32(M, N, K):
    """TF32 operands (10-bit mantissa): C = A B^T to ~2^-11 relative per product."""
    rng = np.random.default_rng(7 * M + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C = F.fh_tc_gemm_test(2, A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    err = np.max(np.abs(C - ref)) / (np.sqrt(K) * np.max(np.abs(A)) * np.max(np.abs(B)))
    assert err < 2e-3
    # the result is not a plain FP32 GEMM in disguise of zeros or garbage
    assert np.corrcoef(C.ravel(), ref.ravel())[0, 1] > 0.999
