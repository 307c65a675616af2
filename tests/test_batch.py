"""Batches: several problems of uneven sizes solved in the same launches."""
import numpy as np
import pytest

import fh_inputs as fi
import oracle as O
from paper_1807_02718_gb300 import fh as F

TOL = 1e-10


def _problems(count=4, seed=21):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        cur = fi.random_star(rng)
        J = int(rng.integers(6, 14))
        W = float(rng.uniform(3.0, 9.0))
        om = fi.frequency_mesh(J, W)
        N = fi.boundary_sizes(cur, om, n_min=32, multiple=2)
        ang = float(rng.uniform(0, 2 * np.pi))
        out.append((cur, om, N, (np.cos(ang), np.sin(ang))))
    return out


def test_footprint_counts_matrices_and_tables():
    from paper_1807_02718_gb300 import build
    build.build()
    J = [3, 2]
    N = [np.array([0, 10, 20]), np.array([0, 8])]
    b64 = F.fh_footprint(J, N, F.FH_FP64)
    b32 = F.fh_footprint(J, N, F.FH_MIXED_FP32)
    n = np.array([10, 20, 8])
    assert b64 >= int(np.sum(n * n * 16))
    assert b32 - b64 == int(np.sum(n * n * 8 + n * 28))   # FP32 copy, rhs, perm, FP32 rhs


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [F.FH_FP64, F.FH_MIXED_FP32, F.FH_MIXED_TF32, F.FH_MIXED_BF16])
def test_batch_equals_each_problem_alone(precision):
    from paper_1807_02718_gb300 import build
    build.build()
    probs = _problems()
    sig = fi.pulse_train(5, n=3, span=30.0, fmin=1.0, fmax=4.0)
    t0, dt = -10.0, 0.02
    a = fi.sample_signal(sig, t0, dt, int(np.ceil((sig.t_end - t0) / dt)) + 1)
    x = fi.targets_on_circle(6, 2.5, center=(0.05, 0.1))
    T = np.concatenate([np.linspace(0, 50, 30), [400.0, 9000.0]])
    ctx = F.fh_create(0, precision)
    F.fh_discretize_batch(ctx, [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                          ps=[p[3] for p in probs])
    assert F.fh_num_problems(ctx) == len(probs)
    st = F.fh_solve_frequencies(ctx)
    assert st.n_solves == sum(len(p[1]) - 1 for p in probs)
    u_batch = []
    for q in range(len(probs)):
        F.fh_window_spectra_p(ctx, q, a, t0, dt)
        u_batch.append(F.fh_sample_p(ctx, q, x, T))
    for q, (cur, om, N, pdir) in enumerate(probs):
        alone = F.Problem(0, precision)
        alone.discretize(cur, om, N, 1.0, pdir)
        alone.solve()
        for j in range(1, len(om)):
            assert np.array_equal(F.fh_get_density_p(ctx, q, j, int(N[j])),
                                  F.fh_get_density(alone.ctx, j, int(N[j])))
        alone.window_spectra(a, t0, dt)
        assert np.array_equal(alone.sample(x, T), u_batch[q])
        alone.close()
    # and one problem of the batch against the oracle
    cur, om, N, pdir = probs[2]
    wl = fi.Workload("batch2", cur, om, N, 1.0, pdir, a, t0, dt, 10.0, x, T)
    ref = O.run(wl)["u"]
    assert np.linalg.norm(u_batch[2] - ref) / np.linalg.norm(ref) < TOL
    F.fh_destroy(ctx)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [F.FH_MIXED_TF32, F.FH_MIXED_BF16])
def test_batch_tensor_core_vs_oracle(precision):
    """Three star problems of uneven sizes (N up to ~300) in one batch on the
    tensor-core LU, with the largest systems split onto the second stream
    (lu_early) and the tensor-core contraction: every problem's densities and
    u(x, T) within 1e-10 of the oracle, each after graph replay."""
    from paper_1807_02718_gb300 import build
    build.build()
    rng = np.random.default_rng(8)
    probs = []
    for q in range(3):
        cur = fi.random_star(rng)
        J = int(rng.integers(20, 40))
        om = fi.frequency_mesh(J, float(rng.uniform(10.0, 30.0)))
        ang = float(rng.uniform(0, 2 * np.pi))
        probs.append((cur, om, fi.boundary_sizes(cur, om), (np.cos(ang), np.sin(ang))))
    sig = fi.pulse_train(9, n=6, span=60.0, fmin=4.0, fmax=12.0)
    t0, dt = -10.0, 0.01
    a = fi.sample_signal(sig, t0, dt, int(np.ceil((sig.t_end - t0) / dt)) + 1)
    x = fi.targets_on_circle(9, 2.6, center=(-0.1, 0.05))
    T = np.concatenate([np.linspace(0, 120, 97), [777.0, 1e4]])
    ctx = F.fh_create(0, precision)
    F.fh_set_tuning(ctx, lu_early=20, contract_tc=1)
    for _ in range(3):                      # direct launches, capture, replay
        F.fh_discretize_batch(ctx, [p[0] for p in probs], [p[1] for p in probs],
                              [p[2] for p in probs], ps=[p[3] for p in probs])
        st = F.fh_solve_frequencies(ctx)
        u_batch = []
        for q in range(3):
            F.fh_window_spectra_p(ctx, q, a, t0, dt)
            u_batch.append(F.fh_sample_p(ctx, q, x, T))
    assert st.residual_max < 1e-12
    for q, (cur, om, N, pdir) in enumerate(probs):
        wl = fi.Workload(f"batch{q}", cur, om, N, 1.0, pdir, a, t0, dt, 10.0, x, T)
        ref = O.run(wl)
        for j in range(1, len(om)):
            psi = F.fh_get_density_p(ctx, q, j, int(N[j]))
            assert np.linalg.norm(psi - ref["psi"][j]) / np.linalg.norm(ref["psi"][j]) < TOL
        assert np.linalg.norm(u_batch[q] - ref["u"]) / np.linalg.norm(ref["u"]) < TOL
    F.fh_destroy(ctx)
