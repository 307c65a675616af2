"""GPU parity: every step of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: the FP64 path must agree with the oracle within 1e-10 relative L2
per result (the required accuracy); the measured agreement is ~1e-13 or
better, limited by different Bessel implementations (scipy's and CUDA's carry
~1e-15 absolute error each) and rounding order.
"""
import math

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


def make(wl, precision=F.FH_FP64):
    pr = F.Problem(0, precision)
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    return pr


WORKLOADS = {
    "small_kite": lambda: fi.small_kite(),
    "circle": lambda: fi.circle_gauss(J=9, W=8.0, N=96, n_x=7, n_T=23),
    "star": lambda: _star_workload(),
}


def _star_workload():
    rng = np.random.default_rng(11)
    cur = fi.random_star(rng)
    wl = fi.small_kite(J=10, W=7.0)
    wl.curve = cur
    wl.N = np.asarray([0, 66, 64, 96, 130, 128, 160, 190, 200, 256], dtype=np.int32)
    return wl


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_geometry(name):
    wl = WORKLOADS[name]()
    pr = make(wl)
    for j in range(1, wl.J):
        n = int(wl.N[j])
        z, dz, ddz = F.fh_get_geometry(pr.ctx, j, n)
        _, zo, dzo, ddzo = O.discretize(wl.curve, n // 2)
        assert np.max(np.abs(z - (zo[0] + 1j * zo[1]))) < 1e-14
        assert np.max(np.abs(dz - (dzo[0] + 1j * dzo[1]))) < 1e-13
        assert np.max(np.abs(ddz - (ddzo[0] + 1j * ddzo[1]))) < 1e-12


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("prec", [F.FH_FP64, F.FH_MIXED_TF32])
def test_assembly(name, prec):
    """FP64 path: within 1e-13 of the oracle.  Mixed paths assemble the
    entries with kappa r >= 8 in double-float arithmetic: stated bound 2e-13
    relative L2, 1e-12 of the largest entry pointwise."""
    wl = WORKLOADS[name]()
    pr = make(wl, prec)
    tol = 1e-13 if prec == F.FH_FP64 else 2e-13
    for j in range(1, wl.J):
        n = int(wl.N[j])
        eta = 0.5 + wl.omega[j]
        A, g = F.fh_assemble_matrix(pr.ctx, j, eta, n)
        Ao = O.cfie_matrix(wl.curve, n // 2, wl.omega[j], wl.c, eta)
        go = O.cfie_rhs(wl.curve, n // 2, wl.omega[j], wl.c, wl.p, eta)
        assert rel(A, Ao) < tol, j
        assert np.max(np.abs(A - Ao)) < 1e-12 * np.max(np.abs(Ao))
        assert rel(g, go) < 1e-13


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_densities(name):
    wl = WORKLOADS[name]()
    pr = make(wl)
    st = pr.solve()
    assert st.n_solves == wl.J - 1
    psi_o = O.solve_all(wl)
    for j in range(1, wl.J):
        psi = F.fh_get_density(pr.ctx, j, int(wl.N[j]))
        assert rel(psi, psi_o[j]) < TOL, j


def test_densities_with_coupling():
    wl = fi.small_kite(J=6)
    eta = np.linspace(0.0, 3.0, wl.J) + 0.25
    wl.eta = eta
    pr = make(wl)
    pr.solve(eta)
    psi_o = O.solve_all(wl)
    for j in range(1, wl.J):
        assert rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) < TOL


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_window_spectra(name):
    wl = WORKLOADS[name]()
    pr = make(wl)
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    s, B = F.fh_get_window_spectra(pr.ctx, wl.J)
    so, Bo = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
    assert np.array_equal(s, so)
    assert rel(B, Bo) < 1e-13


def test_window_spectra_ragged_and_offset_grids():
    """Sample spans that end mid-window, start after t0, and one window only."""
    cur = fi.circle(1.0)
    om = fi.frequency_mesh(7, 9.0)
    for t0, n, dt in [(-10.0, 1, 0.01), (-3.0, 777, 0.01), (-10.0, 2345, 0.005), (2.5, 4000, 0.025)]:
        a = np.sin(np.arange(n) * 0.37) * np.exp(-((np.arange(n) - n / 2) / (n / 5 + 1)) ** 2)
        pr = F.Problem()
        pr.discretize(cur, om, np.full(7, 16, dtype=np.int32))
        pr.window_spectra(a, t0, dt, 10.0)
        s, B = F.fh_get_window_spectra(pr.ctx, 7)
        so, Bo = O.window_spectra(a, t0, dt, 10.0, om)
        assert np.array_equal(s, so)
        # rounding bound of a length-Q sum whose terms are |a w| dt: the test
        # signal is oscillatory, so B itself can be 1e4 times smaller than the sum
        bound = 1e-14 * dt * np.sum(np.abs(a)) * 4
        assert np.max(np.abs(B - Bo)) <= bound


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("prec", [F.FH_FP64, F.FH_MIXED_TF32])
def test_target_field_from_oracle_densities(name, prec):
    """Step F5 alone: the oracle's densities in, V(x, omega_j) out (the mixed
    paths evaluate H0 at kappa r >= 8 in double-float arithmetic)."""
    wl = WORKLOADS[name]()
    pr = make(wl, prec)
    psi_o = O.solve_all(wl)
    F.fh_set_densities(pr.ctx, np.concatenate([psi_o[j] for j in range(1, wl.J)]))
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    pr.sample(wl.x, wl.T[:3])
    V = F.fh_get_target_field(pr.ctx, wl.n_x, wl.J)
    Vo = O.target_fields(wl, psi_o)
    assert rel(V, Vo) < 1e-12
    assert np.all(V[:, 0] == 1.0)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_synthesis_from_oracle_fields(name):
    """Steps T0-T6 alone: oracle target fields in, u(x, T) out."""
    wl = WORKLOADS[name]()
    pr = make(wl)
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((4, wl.J)) + 1j * rng.standard_normal((4, wl.J))
    V[:, 0] = 1.0
    T = np.concatenate([wl.T, [-5.0, 0.0, 1e3, 5e4, 123456.789]])
    u = F.fh_synthesize(pr.ctx, V, T)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
    uo = O.synthesize(B, s, wl.omega, V, T)
    assert rel(u, uo) < 1e-12


def test_synthesis_e1_closed_form():
    """The Sec. 6.1 Gaussian through the GPU quadrature: with one window and
    a(t) = exp(-t^2)/sqrt(pi) sampled on [-5, 5), B^slow = exp(-w^2/4); the
    field V = e^{10 i w} shifts it, so u(t) = exp(-(t-10)^2)/sqrt(pi) at all t
    (no replica at t = 10 + 2 pi/dw)."""
    W, J = 12.0, 97
    om = np.linspace(0.0, W, J)
    pr = F.Problem()
    pr.discretize(fi.circle(1.0), om, np.full(J, 16, dtype=np.int32))
    t0, dt = -5.0, 0.01
    t = t0 + dt * np.arange(1000)
    a = np.exp(-t ** 2) / math.sqrt(math.pi)
    pr.window_spectra(a, t0, dt, 10.0)
    assert F.fh_get_num_windows(pr.ctx) == 1
    T = np.concatenate([np.linspace(-20, 40, 241), [10 + 2 * math.pi / (om[1] - om[0]), 1e4, 1e5]])
    V = np.exp(1j * 10 * om)[None, :]
    u = F.fh_synthesize(pr.ctx, V, T)[0]
    assert np.max(np.abs(u - np.exp(-(T - 10) ** 2) / math.sqrt(math.pi))) < 1e-10
    s, B = O.window_spectra(a, t0, dt, 10.0, om)
    assert rel(u, O.synthesize(B, s, om, V, T)[0]) < 1e-12


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_full_path(name):
    wl = WORKLOADS[name]()
    pr = make(wl)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x, wl.T)
    ref = O.run(wl)
    assert rel(u, ref["u"]) < TOL


def test_full_path_circle_gauss_config():
    """Circle, Gaussian-modulated sinusoid, 64 frequencies on [0,16], N=256,
    16 targets on r=3, 200 times on [0,20]."""
    wl = fi.circle_gauss()
    pr = make(wl)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x, wl.T)
    ref = O.run(wl)
    assert rel(u, ref["u"]) < TOL
    for j in (1, 17, 63):
        assert rel(F.fh_get_density(pr.ctx, j, 256), ref["psi"][j]) < TOL


def test_sample_reuses_state_and_is_repeatable():
    wl = fi.small_kite()
    pr = make(wl)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u1 = pr.sample(wl.x, wl.T)
    u2 = pr.sample(wl.x[:4], wl.T[::-1])
    u3 = pr.sample(wl.x, wl.T)
    assert np.array_equal(u1, u3)
    assert np.array_equal(u1[:2, ::-1], u2)


def test_device_pointer_variants_match_host():
    import torch
    wl = fi.small_kite()
    pr = make(wl)
    pr.solve()
    d_a = torch.tensor(wl.a, device="cuda", dtype=torch.float64)
    F.fh_window_spectra_dev(pr.ctx, d_a, wl.t0, wl.dt, wl.H)
    d_x = torch.tensor(wl.x, device="cuda", dtype=torch.float64)
    d_T = torch.tensor(wl.T, device="cuda", dtype=torch.float64)
    d_u = torch.empty(wl.n_x * wl.T.size, device="cuda", dtype=torch.float64)
    st = torch.cuda.current_stream()
    F.fh_set_stream(pr.ctx, st.cuda_stream)
    F.fh_sample_dev(pr.ctx, d_x, d_T, d_u)
    st.synchronize()
    u_host = pr.sample(wl.x, wl.T)
    assert np.array_equal(d_u.cpu().numpy().reshape(wl.n_x, -1), u_host)


def test_edge_cases_and_errors():
    wl = fi.small_kite(J=4)
    pr = make(wl)
    with pytest.raises(F.FHError) as e:
        pr.sample(wl.x, wl.T)
    assert e.value.status == F.FH_ESTATE
    pr.solve()
    with pytest.raises(F.FHError) as e:
        pr.sample(wl.x, wl.T)
    assert e.value.status == F.FH_ESTATE
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    assert pr.sample(wl.x, np.zeros(0)).shape == (wl.n_x, 0)
    assert pr.sample(np.zeros(0), wl.T).shape == (0, wl.T.size)
    with pytest.raises(F.FHError) as e:
        pr.window_spectra(wl.a, wl.t0, 0.013, wl.H)
    assert e.value.status == F.FH_EINVAL
    bad = F.Problem()
    with pytest.raises(F.FHError) as e:
        bad.discretize(wl.curve, np.array([0.0, 1.0, 2.5]), None)
    assert e.value.status == F.FH_EINVAL
    with pytest.raises(F.FHError) as e:
        bad.discretize(wl.curve, wl.omega, np.full(wl.J, 63, dtype=np.int32))
    assert e.value.status == F.FH_EINVAL
    with pytest.raises(F.FHError) as e:
        bad.discretize(wl.curve, wl.omega + 0.5, None)
    assert e.value.status == F.FH_EINVAL
    # state survives a failed call
    u = pr.sample(wl.x, wl.T)
    assert np.all(np.isfinite(u))


def test_minimal_sizes():
    """N = 8 nodes, J = 2 (one solve), one target, one time."""
    cur = fi.circle(1.0)
    om = np.array([0.0, 1.5])
    N = np.array([0, 8], dtype=np.int32)
    pr = F.Problem()
    pr.discretize(cur, om, N)
    pr.solve()
    t0, dt = -10.0, 0.01
    a = fi.sample_signal(lambda t: fi.gauss_sine(t, 1.0, 1.0, 3.0), t0, dt, 1600)
    pr.window_spectra(a, t0, dt, 10.0)
    u = pr.sample(np.array([2.0, 0.5]), np.array([4.0]))
    wl = fi.Workload("min", cur, om, N, 1.0, (1.0, 0.0), a, t0, dt, 10.0, np.array([2.0, 0.5]),
                     np.array([4.0]))
    assert rel(u, O.run(wl)["u"]) < TOL


def test_large_config_sampled():
    """Kite, 40-pulse train over [0, 400], 256 frequencies on [0, 40], N by 8
    points per wavelength (64..480), 1024 targets x 4096 times up to T = 1e4,
    in the launch configuration the benchmark times.  Every density is
    compared; the field is compared on a sample of 12 targets at all times."""
    wl = fi.kite_pulses()
    pr = make(wl)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x, wl.T)
    assert u.shape == (1024, 4096) and np.all(np.isfinite(u))
    psi_o = O.solve_all(wl)
    worst = max(rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) for j in range(1, wl.J))
    assert worst < TOL
    idx = np.array([0, 1, 77, 255, 256, 400, 511, 640, 777, 900, 1000, 1023])
    xs = wl.x.reshape(-1, 2)[idx].reshape(-1)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
    V = O.target_fields(wl, psi_o, xs)
    uo = O.synthesize(B, s, wl.omega, V, wl.T)
    assert rel(u[idx], uo) < TOL


# ------------------------------------------------------ mixed precision (FP32 LU + FP64 IR)

@pytest.mark.parametrize("name", list(WORKLOADS))
def test_densities_mixed_precision(name):
    """FP32 LU with FP64 refinement reaches the FP64 oracle within 1e-10."""
    wl = WORKLOADS[name]()
    pr = make(wl, F.FH_MIXED_FP32)
    st = pr.solve()
    assert 1 <= st.refine_iters_max <= 6
    assert st.residual_max < 1e-12
    psi_o = O.solve_all(wl)
    worst = max(rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) for j in range(1, wl.J))
    assert worst < TOL


def test_full_path_mixed_precision_circle_config():
    wl = fi.circle_gauss()
    pr = make(wl, F.FH_MIXED_FP32)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x, wl.T)
    assert rel(u, O.run(wl)["u"]) < TOL


def test_large_config_mixed_precision():
    """The benchmark workload solved in mixed precision: every density within
    1e-10 of the FP64 oracle, and the field equal to the FP64 GPU path's."""
    wl = fi.kite_pulses(n_near=256, n_far=64)
    pr = make(wl, F.FH_MIXED_FP32)
    st = pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u = pr.sample(wl.x[:64], wl.T)
    psi_o = O.solve_all(wl)
    worst = max(rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) for j in range(1, wl.J))
    assert worst < TOL, worst
    ref = make(wl)
    ref.solve()
    ref.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    u64 = ref.sample(wl.x[:64], wl.T)
    assert rel(u, u64) < TOL
    assert st.refine_iters_max <= 6


# ------------------------- tensor-core LU (tcgen05, 3xTF32 / 3xBF16) + FP64 IR

TC_PRECISIONS = {"tf32": F.FH_MIXED_TF32, "bf16": F.FH_MIXED_BF16}


@pytest.mark.parametrize("prec", list(TC_PRECISIONS))
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_densities_tensor_core_lu(name, prec):
    """Trailing updates on tcgen05 (TF32 or BF16 operands, split hi + lo):
    after FP64 refinement every density is within 1e-10 of the FP64 oracle."""
    wl = WORKLOADS[name]()
    pr = make(wl, TC_PRECISIONS[prec])
    st = pr.solve()
    assert 1 <= st.refine_iters_max <= 10
    assert st.residual_max < 1e-12
    psi_o = O.solve_all(wl)
    worst = max(rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) for j in range(1, wl.J))
    assert worst < TOL


@pytest.mark.parametrize("prec", list(TC_PRECISIONS))
def test_large_config_tensor_core_lu(prec):
    """The 256-frequency kite (N = 64..480, one CTA per system).  The LU is
    only a preconditioner, so a wrong entry in the FP32 copy it factors (written
    by the assembly) would show as extra sweeps rather than wrong densities: the
    sweep count is pinned at the 3 the split operands need (2^-16 BF16, 2^-21
    TF32, both contracting the error by more than 1e-4 per sweep)."""
    wl = fi.kite_pulses(n_near=256, n_far=64)
    pr = make(wl, TC_PRECISIONS[prec])
    st = pr.solve()
    psi_o = O.solve_all(wl)
    worst = max(rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) for j in range(1, wl.J))
    assert worst < TOL, worst
    assert st.refine_iters_max <= 3, st.refine_iters_max
    assert st.residual_max < 1e-12


@pytest.mark.parametrize("prec", list(TC_PRECISIONS))
def test_tensor_core_lu_clusters(prec):
    """Systems factored by clusters of 2, 4 and 8 CTAs (N = 520, 1536, 2600:
    ragged last row tiles, CTAs without panel rows, panels split over CTAs)."""
    wl = fi.small_kite(J=4, W=60.0)
    wl.N = np.asarray([0, 2600, 1536, 520], dtype=np.int32)
    pr = make(wl, TC_PRECISIONS[prec])
    st = pr.solve()
    assert st.residual_max < 1e-12
    psi_o = O.solve_all(wl)
    for j in (1, 2, 3):
        assert rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) < TOL


@pytest.mark.parametrize("prec", list(TC_PRECISIONS))
def test_tensor_core_lu_row_exchanges(prec):
    """The tensor-core LU keeps the diagonal pivots only where partial pivoting
    would (each panel checked; otherwise the panel is factored again with the
    per-column search).  With the CFIE coupling eta = omega no row is ever
    exchanged; with eta = 1000 omega the single layer dominates and the
    highest frequencies of the small kite (N 66..110) and the 520-point
    system of the cluster case need exchanges (checked on the oracle's
    matrices), while the 2600- and 1536-point systems (clusters of 6 and 3
    CTAs) keep the diagonal: every combination agrees with the oracle.  (The
    refinement stops on its correction tolerance; with the single layer scaled
    by 1000 the final relative residual is ~1e-12, so it is bounded at 1e-11.)"""
    for wl in (fi.small_kite(J=10, W=7.0), fi.small_kite(J=4, W=60.0)):
        if wl.J == 4:
            wl.N = np.asarray([0, 2600, 1536, 520], dtype=np.int32)
        wl.eta = 1e3 * wl.omega
        pr = make(wl, TC_PRECISIONS[prec])
        st = pr.solve(wl.eta)
        assert st.residual_max < 1e-11
        psi_o = O.solve_all(wl)
        for j in range(1, wl.J):
            assert rel(F.fh_get_density(pr.ctx, j, int(wl.N[j])), psi_o[j]) < TOL, (wl.J, j)


def test_resample_on_resident_target_fields():
    """fh_resample_p: new times on the target fields left by the last sample
    (no fresh step F5) equal a fresh fh_sample at those times bit for bit, and
    the oracle within 1e-10; fields stop being resident after a re-solve."""
    wl = fi.small_kite()
    pr = make(wl)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    with pytest.raises(F.FHError) as e:
        F.fh_resample_p(pr.ctx, 0, wl.T, wl.n_x)
    assert e.value.status == F.FH_ESTATE
    pr.sample(wl.x, wl.T[:5])
    T2 = np.concatenate([wl.T[::-1], [7.7e3]])
    u = F.fh_resample_p(pr.ctx, 0, T2, wl.n_x)
    assert np.array_equal(u, pr.sample(wl.x, T2))
    assert rel(u, O.run(wl, T=T2)["u"]) < TOL
    pr.solve()
    with pytest.raises(F.FHError) as e:
        F.fh_resample_p(pr.ctx, 0, T2, wl.n_x)
    assert e.value.status == F.FH_ESTATE
