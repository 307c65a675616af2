"""Near-window sums of the synthesis (Sec. 4.1) from the sampled table: the
band-limited sums D_p(y) tabulated on the half-integer grid and interpolated
with the sinc x exponential-of-semicircle window (J <= 1025), against the
direct M-term sums that the allocation-free entry point and contexts with
J > 1025 use.  Times put windows at y = 0, near half-integers, next to the
near/far boundary |y| = 1.25 h, and J > 256 spans several column blocks."""
import math

import numpy as np
import pytest

import fh_inputs as fi
import oracle as O
from paper_1807_02718_gb300 import fh as F

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1807_02718_gb300 import build
    build.build()
    F.load_library()


def times(wl, h, W):
    """Times at window centres (y = 0), near half-integer y, just inside and
    outside the near range, and a spread over the signal."""
    s = 1.5 * wl.H * np.arange(4)
    edge = (1.25 * h - 1e-7) * math.pi / W
    T = [s[1], s[2], s[1] + 0.5 * math.pi / W, s[2] + 3.5 * math.pi / W,
         s[1] + edge, s[2] - edge, s[1] + edge + 2e-7 * math.pi / W]
    T += list(np.linspace(0.0, 60.0, 113))
    return np.asarray(T)


def both(J, W, n_x=24):
    import torch
    wl = fi.small_kite(J=J, W=W)
    wl.N = np.full(J, 64, dtype=np.int32)
    h = J - 1
    T = times(wl, h, W)
    pr = F.Problem()
    pr.discretize(wl.curve, wl.omega, wl.N)
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    s, B = F.fh_get_window_spectra(pr.ctx, wl.J)
    rng = np.random.default_rng(J)
    V = rng.standard_normal((n_x, J)) + 1j * rng.standard_normal((n_x, J))
    V[:, 0] = 1.0
    u_ctx = F.fh_synthesize(pr.ctx, V, T)
    pr.close()
    dev = torch.device("cuda", 0)
    d_s = torch.tensor(s, device=dev)
    d_B = torch.tensor(np.ascontiguousarray(B).view(np.float64).ravel(), device=dev)
    d_V = torch.tensor(np.ascontiguousarray(V.T).view(np.float64).ravel(), device=dev)
    d_T = torch.tensor(T, device=dev)
    d_u = torch.full((n_x * T.size,), float("nan"), device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream()
    F.fh_synthesize_static(J, float(wl.omega[-1]), d_s, d_B, d_V, d_T, d_u, stream.cuda_stream)
    stream.synchronize()
    return u_ctx, d_u.cpu().numpy().reshape(n_x, T.size)


@pytest.mark.parametrize("J,W", [(12, 6.0), (40, 12.0), (300, 30.0), (1025, 60.0)])
def test_sampled_near_sums_match_direct_sums(J, W):
    u_tab, u_dir = both(J, W)
    assert np.all(np.isfinite(u_tab))
    assert rel(u_tab, u_dir) < 1e-12, rel(u_tab, u_dir)


def test_direct_sums_above_the_table_bound():
    """J = 1026 has no table: the context path runs the direct sums, bit for
    bit those of the allocation-free entry point."""
    u_ctx, u_dir = both(1026, 60.0, n_x=8)
    assert np.array_equal(u_ctx, u_dir)


@pytest.mark.parametrize("J", [12, 1025])
def test_table_rows_against_oracle(J):
    """Every half-integer row of the near-sum table, negative rows included
    (those are derived from the positive ones by conjugation and an end-term
    correction), read through the synthesis: with a single window, a time at
    y = W (T - s_1) / pi = g/2 puts the 42-point interpolation exactly on
    sample g (weight 1 there, 0 on the others), so u at that time is the
    table row contracted with B and V.  Compared pointwise with the oracle's
    direct sum (1e-13 of the largest |u|), for every g with |g/2| < 1.25 h."""
    W = 6.0 if J == 12 else 60.0
    om = fi.frequency_mesh(J, W)
    t0, dt = -10.0, 0.01
    t = t0 + dt * np.arange(1500)                 # one window (K = 1, s_1 = 0)
    a = np.exp(-((t - 1.0) / 1.5) ** 2) * np.sin(2.0 * t)
    h = J - 1
    g_max = int(math.floor(2 * 1.25 * h - 1e-9))
    g = np.arange(-g_max, g_max + 1)
    if J > 100:                                   # all negative rows, a spread of positive ones
        g = np.concatenate([g[g < 0], g[g >= 0][::17]])
    T = (g / 2.0) * math.pi / W
    pr = F.Problem()
    pr.discretize(fi.circle(1.0), om, np.full(J, 16, dtype=np.int32))
    pr.window_spectra(a, t0, dt, 10.0)
    assert F.fh_get_num_windows(pr.ctx) == 1
    rng = np.random.default_rng(J + 1)
    V = rng.standard_normal((3, J)) + 1j * rng.standard_normal((3, J))
    V[:, 0] = 1.0
    u = F.fh_synthesize(pr.ctx, V, T)
    pr.close()
    s, B = O.window_spectra(a, t0, dt, 10.0, om)
    uo = O.synthesize(B, s, om, V, T)
    scale = np.max(np.abs(uo))
    neg = g < 0
    assert np.max(np.abs(u[:, neg] - uo[:, neg])) < 1e-13 * scale
    assert np.max(np.abs(u[:, ~neg] - uo[:, ~neg])) < 1e-13 * scale
