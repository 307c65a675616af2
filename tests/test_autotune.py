"""Schedule parameters and the autotuner: every setting computes the same
discrete quantities (parity with the oracle at each setting), invalid settings
are rejected, and the tuner's choice reproduces, bit for bit, the results of
the same setting applied by hand."""
import numpy as np
import pytest

import fh_inputs as fi
import oracle as O
from paper_1807_02718_gb300 import fh as F

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1807_02718_gb300 import build
    build.build()
    F.load_library()


def runs_workload():
    """Equal-N runs of 5 frequencies (64, 96, 128 nodes), so that subgroups of
    2, 4 and 8 split them differently; a ragged last run."""
    wl = fi.small_kite(J=12, W=6.0)
    wl.N = np.asarray([0] + [64 + 32 * ((j - 1) // 5) for j in range(1, 12)], dtype=np.int32)
    return wl


def cycle(pr, wl):
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x, wl.T)
    psi = [F.fh_get_density(pr.ctx, j, int(wl.N[j])) for j in range(1, wl.J)]
    V = F.fh_get_target_field(pr.ctx, wl.n_x, wl.J)
    return psi, V, u


@pytest.fixture(scope="module")
def oracle_runs():
    wl = runs_workload()
    return wl, O.run(wl)


SETTINGS = [
    dict(assemble_group=1, field_group=1, field_chunk=16),
    dict(assemble_group=2, field_group=4, field_chunk=32),
    dict(assemble_group=4, field_group=2, field_chunk=64),
    dict(assemble_group=8, field_group=8, field_chunk=16),
    dict(assemble_group=3, field_group=5, field_chunk=32),
]


@pytest.mark.parametrize("prec", [F.FH_FP64, F.FH_MIXED_TF32])
@pytest.mark.parametrize("setting", range(len(SETTINGS)))
def test_every_setting_matches_the_oracle(prec, setting, oracle_runs):
    wl, ref = oracle_runs
    pr = F.Problem(0, prec)
    F.fh_set_tuning(pr.ctx, **SETTINGS[setting])
    psi, V, u = cycle(pr, wl)
    assert F.fh_get_tuning(pr.ctx)["field_chunk"] == SETTINGS[setting]["field_chunk"]
    for j in range(1, wl.J):
        assert rel(psi[j - 1], ref["psi"][j]) < TOL, j
    assert rel(V, ref["V"]) < TOL
    assert rel(u, ref["u"]) < TOL


@pytest.mark.parametrize("rows", [512, 256, 128])
def test_lu_rows_per_cta(rows):
    """rows 128 factors N = 160, 288, 520 with clusters of 2, 4 and 8 CTAs
    (CTAs without panel rows from the first panel on)."""
    wl = fi.small_kite(J=4, W=30.0)
    wl.N = np.asarray([0, 520, 288, 160], dtype=np.int32)
    pr = F.Problem(0, F.FH_MIXED_TF32)
    F.fh_set_tuning(pr.ctx, lu_rows_per_cta=rows)
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    st = pr.solve()
    assert st.residual_max < 1e-12
    psi_o = O.solve_all(wl)
    for j in (1, 2, 3):
        assert rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) < TOL


def test_invalid_settings_are_rejected():
    pr = F.Problem(0, F.FH_MIXED_TF32)
    before = F.fh_get_tuning(pr.ctx)
    assert before == {"assemble_group": 8, "field_group": 8, "field_chunk": 64,
                      "lu_rows_per_cta": 512, "lu_early": 0, "contract_tc": 1}
    for bad in (dict(assemble_group=0), dict(assemble_group=9), dict(field_group=0),
                dict(field_chunk=48), dict(field_chunk=128), dict(lu_rows_per_cta=1024),
                dict(lu_early=-1), dict(lu_early=51), dict(contract_tc=2)):
        with pytest.raises(F.FHError) as e:
            F.fh_set_tuning(pr.ctx, **bad)
        assert e.value.status == F.FH_EINVAL
        assert F.fh_get_tuning(pr.ctx) == before
    with pytest.raises(F.FHError) as e:
        F.fh_autotune(pr.ctx, None)
    assert e.value.status == F.FH_ESTATE       # no discretization yet


@pytest.mark.parametrize("prec", [F.FH_FP64, F.FH_MIXED_TF32])
def test_autotune_choice_equals_the_same_setting_by_hand(prec, oracle_runs):
    wl, ref = oracle_runs
    tuned = F.Problem(0, prec)
    tuned.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    F.fh_get_timings(tuned.ctx, reset=True)
    chosen, ms = F.fh_autotune(tuned.ctx, wl.x, reps=2)
    assert chosen == F.fh_get_tuning(tuned.ctx)
    assert chosen["assemble_group"] in (2, 4, 8) and chosen["field_group"] in (2, 4, 8)
    assert chosen["field_chunk"] in (16, 32, 64)
    assert ms["assemble"] > 0 and ms["field"] > 0
    if prec == F.FH_MIXED_TF32:
        assert chosen["lu_rows_per_cta"] in (128, 256, 512) and ms["factor"] > 0
        assert chosen["lu_early"] in (0, 10, 20, 35) and ms["assemble_factor"] > 0
    else:
        assert chosen["lu_rows_per_cta"] == 512 and ms["factor"] == 0
        assert chosen["lu_early"] == 0 and ms["assemble_factor"] == 0
    # tuning runs are not counted as launches of the path
    assert all(v["launches"] == 0 for v in F.fh_get_timings(tuned.ctx, reset=True).values())
    by_hand = F.Problem(0, prec)
    F.fh_set_tuning(by_hand.ctx, **chosen)
    a = cycle(tuned, wl)
    b = cycle(by_hand, wl)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert rel(a[2], ref["u"]) < TOL


def test_autotune_after_solve_keeps_the_solution(oracle_runs):
    """Tuning after a solve leaves the densities in place: sampling needs no
    new solve and still matches the oracle."""
    wl, ref = oracle_runs
    pr = F.Problem(0, F.FH_MIXED_TF32)
    psi0, _, _ = cycle(pr, wl)
    F.fh_autotune(pr.ctx, wl.x, reps=1)
    psi1 = [F.fh_get_density(pr.ctx, j, int(wl.N[j])) for j in range(1, wl.J)]
    for x, y in zip(psi0, psi1):
        assert np.array_equal(x, y)
    u = pr.sample(wl.x, wl.T)
    assert rel(u, ref["u"]) < TOL


@pytest.mark.parametrize("early", [10, 35, 50])
@pytest.mark.parametrize("graphs", [False, True])
def test_largest_systems_started_early(early, graphs, oracle_runs):
    """lu_early runs the largest systems' assembly and factorisation on a second
    stream: the same kernels on the same data, so bitwise the same densities,
    fields and u as the single sequence (direct launches and graph replay)."""
    wl, ref = oracle_runs
    one = F.Problem(0, F.FH_MIXED_TF32)
    two = F.Problem(0, F.FH_MIXED_TF32)
    F.fh_set_tuning(two.ctx, lu_early=early)
    F.fh_set_graphs(two.ctx, graphs)
    a = cycle(one, wl)
    for _ in range(3 if graphs else 1):     # direct, capture, replay
        b = cycle(two, wl)
        for x, y in zip(a[0], b[0]):
            assert np.array_equal(x, y)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert rel(b[2], ref["u"]) < TOL
