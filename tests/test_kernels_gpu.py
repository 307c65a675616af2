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


def test_fp64_peak_probe_runs():
    v = F.fh_probe_fma_peak(0, True, 256)
    assert v > 0.1
