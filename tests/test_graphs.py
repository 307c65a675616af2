"""CUDA-graph replay of the solve and sample launch sequences: the same
kernels, bitwise the same results as direct launches, replays counted, and a
changed discretization takes a fresh sequence."""
import numpy as np
import pytest

import fh_inputs as fi
from oracle import fh_oracle as O
from paper_1807_02718_gb300 import fh as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1807_02718_gb300 import build
    build.build()


def cycle(pr, wl):
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x, wl.T)
    psi = np.concatenate([F.fh_get_density(pr.ctx, j, int(wl.N[j])) for j in range(1, wl.J)])
    return psi, u


@pytest.mark.parametrize("prec", [F.FH_FP64, F.FH_MIXED_TF32])
def test_graph_replay_equals_direct_launches(prec):
    wl = fi.small_kite()
    direct = F.Problem(0, prec)
    F.fh_set_graphs(direct.ctx, False)
    graphed = F.Problem(0, prec)
    F.fh_get_timings(direct.ctx, reset=True)
    F.fh_get_timings(graphed.ctx, reset=True)
    for rep in range(4):              # direct, capture, replay, replay
        pa, ua = cycle(direct, wl)
        pb, ub = cycle(graphed, wl)
        assert np.array_equal(pa, pb), rep
        assert np.array_equal(ua, ub), rep
    la = F.fh_get_timings(direct.ctx, reset=True)
    lb = F.fh_get_timings(graphed.ctx, reset=True)
    assert {k: v["launches"] for k, v in la.items()} == {k: v["launches"] for k, v in lb.items()}
    uo = O.run(wl)["u"]
    assert np.linalg.norm(ub - uo) / np.linalg.norm(uo) < 1e-10


def test_changed_discretization_after_replays():
    wl = fi.small_kite()
    pr = F.Problem(0, F.FH_MIXED_TF32)
    for _ in range(3):
        cycle(pr, wl)
    wl2 = fi.small_kite()
    wl2.N = (wl2.N + 2).astype(np.int32)
    psi, u = cycle(pr, wl2)
    fresh = F.Problem(0, F.FH_MIXED_TF32)
    psi2, u2 = cycle(fresh, wl2)
    assert np.array_equal(psi, psi2)
    assert np.array_equal(u, u2)
    _, u3 = cycle(pr, wl2)           # capture with the new shape
    _, u4 = cycle(pr, wl2)           # replay
    assert np.array_equal(u3, u2) and np.array_equal(u4, u2)


def test_sample_into_page_locked_buffer():
    """The host-pointer sample writing into a caller's page-locked buffer (the
    bench's end-to-end leg) gives bitwise the array it returns otherwise, on
    direct launches and on graph replays."""
    import torch
    wl = fi.small_kite()
    pr = F.Problem(0, F.FH_MIXED_TF32)
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    ref = F.fh_sample(pr.ctx, wl.x, wl.T)
    buf = torch.full((ref.size,), float("nan"), dtype=torch.float64).pin_memory().numpy()
    for _ in range(3):
        out = F.fh_sample(pr.ctx, wl.x, wl.T, out=buf)
        assert np.array_equal(out, ref) and np.shares_memory(out, buf)
    with pytest.raises(ValueError):
        F.fh_sample(pr.ctx, wl.x, wl.T, out=np.empty(ref.size + 1))
