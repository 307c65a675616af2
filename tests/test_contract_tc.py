"""The tensor-core contraction u = [Vr | Vi] [Gr ; Gm] (operands cut into exact
BF16 slices, exact FP32 sums per slice level): against the oracle's synthesis,
the double-float contraction and the FP64 path, on ragged tile counts, on rows
and columns with a wide dynamic range, at the largest size of one exact K
segment (2J = 512) and with two segments (2J = 514, 1024)."""
import numpy as np
import pytest

import fh_inputs as fi
import oracle as O
from paper_1807_02718_gb300 import fh as F

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1807_02718_gb300 import build
    build.build()
    F.load_library()


def problem(wl, precision, contract_tc=1):
    pr = F.Problem(0, precision)
    F.fh_set_tuning(pr.ctx, contract_tc=contract_tc)
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    return pr


def synth(wl, precision, V, T, contract_tc=1):
    pr = problem(wl, precision, contract_tc)   # kept alive: it owns the context
    u = F.fh_synthesize(pr.ctx, V, T)
    pr.close()
    return u


def fields(J, n_x, seed, spread=0.0):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n_x, J)) + 1j * rng.standard_normal((n_x, J))
    if spread:   # magnitudes over `spread` decades inside every row
        V *= 10.0 ** (-spread * rng.random((n_x, J)))
    V[:, 0] = 1.0
    return V


@pytest.mark.parametrize("n_x,n_t", [(300, 150), (128, 64), (1, 1), (129, 65)])
def test_matches_oracle_and_fp64(n_x, n_t):
    """Ragged and exact tile multiples (128 targets x 64 times per CTA)."""
    wl = fi.small_kite(J=40, W=12.0)
    T = (np.concatenate([np.linspace(0.0, 80.0, n_t - 3), [300.0, 2.5e3, 1e4]]) if n_t > 3
         else np.full(n_t, 20.0))   # a single time inside the signal, where u is not tiny
    V = fields(wl.J, n_x, 1)
    u_tc = synth(wl, F.FH_MIXED_TF32, V, T)
    u_df = synth(wl, F.FH_MIXED_TF32, V, T, contract_tc=0)
    u_64 = synth(wl, F.FH_FP64, V, T)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
    uo = O.synthesize(B, s, wl.omega, V, T)
    assert rel(u_64, uo) < 1e-12
    assert rel(u_tc, uo) < 1e-11, rel(u_tc, uo)
    assert rel(u_tc, u_df) < 1e-11
    assert rel(u_tc, u_64) < 1e-11


def test_wide_dynamic_range_within_rows():
    """Entries spread over six decades inside each row of V: every row is
    scaled by its largest entry, so the small ones keep fewer bits, but their
    contributions are as small; u still agrees with the FP64 path."""
    wl = fi.small_kite(J=64, W=12.0)
    V = fields(wl.J, 200, 2, spread=6.0)
    T = np.linspace(0.0, 120.0, 333)
    u_tc = synth(wl, F.FH_MIXED_TF32, V, T)
    u_64 = synth(wl, F.FH_FP64, V, T)
    assert rel(u_tc, u_64) < 1e-11, rel(u_tc, u_64)


def test_zero_rows_and_columns():
    """A zero target row (scale exponent 0) and times far past the signal give
    exact zeros / tiny values without NaN."""
    wl = fi.small_kite(J=24, W=10.0)
    V = fields(wl.J, 5, 3)
    V[2] = 0.0
    T = np.array([0.0, 20.0, 1e4, 1e6])
    u = synth(wl, F.FH_MIXED_TF32, V, T)
    assert np.all(np.isfinite(u))
    assert np.all(u[2] == 0.0)
    u_64 = synth(wl, F.FH_FP64, V, T)
    assert rel(u, u_64) < 1e-11


def test_largest_exact_size():
    """2J = 512 (the bench workload's K): eight levels of 512 terms still sum
    exactly, and u agrees with the double-float and FP64 contractions."""
    wl = fi.small_kite(J=256, W=30.0)
    wl.N = np.full(256, 64, dtype=np.int32)
    V = fields(wl.J, 150, 5)
    T = np.linspace(0.0, 60.0, 100)
    u_tc = synth(wl, F.FH_MIXED_TF32, V, T)
    u_df = synth(wl, F.FH_MIXED_TF32, V, T, contract_tc=0)
    u_64 = synth(wl, F.FH_FP64, V, T)
    assert rel(u_tc, u_64) < 1e-12, rel(u_tc, u_64)
    assert rel(u_df, u_64) < 1e-12


@pytest.mark.parametrize("J", [257, 512])
def test_k_segments(J):
    """2J = 514 and 1024 (the wide-band workload's K): the levels are exact
    integer sums over K segments of 512, combined in double-float; u agrees
    with the double-float and FP64 contractions."""
    wl = fi.small_kite(J=J, W=30.0)
    wl.N = np.full(J, 64, dtype=np.int32)
    V = fields(wl.J, 150, 4)
    T = np.linspace(0.0, 60.0, 100)
    u_tc = synth(wl, F.FH_MIXED_TF32, V, T)
    u_df = synth(wl, F.FH_MIXED_TF32, V, T, contract_tc=0)
    u_64 = synth(wl, F.FH_FP64, V, T)
    assert rel(u_tc, u_64) < 1e-12, rel(u_tc, u_64)
    assert rel(u_df, u_64) < 1e-12
