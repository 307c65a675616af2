"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
solutions, printed parameters, exact quadrature identities, invariants, or a
brute-force evaluation.  A dropped term, sign or index anywhere in the oracle
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special

import fh_inputs as fi
import oracle as O


# ---------------------------------------------------------------- Bessel steps

def test_bessel_table(golden_dir):
    """Hankel kernels (Sec. 2.3) rest on J0, J1, Y0, Y1: A&S Table 9.1 values."""
    rows = np.loadtxt(os.path.join(golden_dir, "bessel_table.txt"))
    for x, j0, j1, y0, y1 in rows:
        got = [special.j0(x), special.j1(x), special.y0(x), special.y1(x)]
        # the library routines carry ~1e-15 absolute error near x = 5
        assert np.allclose(got, [j0, j1, y0, y1], rtol=0, atol=2e-15)


def test_bessel_wronskian():
    """J1(x) Y0(x) - J0(x) Y1(x) = 2 / (pi x) for all x > 0."""
    x = np.geomspace(1e-3, 600.0, 2001)
    w = special.j1(x) * special.y0(x) - special.j0(x) * special.y1(x)
    assert np.max(np.abs(w * math.pi * x / 2 - 1)) < 1e-12


# ------------------------------------------------------------- Kress weights

@pytest.mark.parametrize("n", [4, 16, 64])
def test_kress_weights_exact_on_trig_polynomials(n):
    """int_0^{2pi} ln(4 sin^2(tau/2)) cos(m tau) dtau = -2pi/m (m >= 1), 0 (m = 0);
    the weights R_d integrate cos(m tau) exactly for 0 <= m <= n."""
    R = O.kress_weights(n)
    t = math.pi * np.arange(2 * n) / n
    assert abs(R.sum()) < 1e-13
    for m in range(1, n + 1):
        assert abs(np.dot(R, np.cos(m * t)) + 2 * math.pi / m) < 1e-12
        assert abs(np.dot(R, np.sin(m * t))) < 1e-12


# --------------------------------------------------- Nystrom CFIE on a circle

def _circle_series(kappa, a, theta, r=None, nmax=80):
    """Exact circle solutions with data e^{i kappa x} (incidence +x):
    psi(theta) = -(2i/(pi a)) sum_n i^n e^{i n theta} / H_n(kappa a),
    U(r, theta) = sum_n i^n J_n(kappa a) H_n(kappa r) / H_n(kappa a) e^{i n theta}."""
    n = np.arange(-nmax, nmax + 1)
    Hn = special.hankel1(n, kappa * a)
    ph = np.exp(1j * np.outer(theta, n)) * (1j ** n)[None, :]
    if r is None:
        return -(2j / (math.pi * a)) * (ph / Hn[None, :]).sum(axis=1)
    return (ph * (special.jv(n, kappa * a) * special.hankel1(n, kappa * r) / Hn)[None, :]).sum(axis=1)


@pytest.mark.parametrize("kappa", [0.5, 4.0, 8.0, 16.0])
@pytest.mark.parametrize("a", [1.0, 0.7])
def test_cfie_circle_density_and_field(kappa, a):
    n = 128
    cur = fi.circle(a)
    psi = O.solve_density(cur, n, kappa)
    t = math.pi * np.arange(2 * n) / n
    ref = _circle_series(kappa, a, t)
    assert np.max(np.abs(psi - ref)) / np.max(np.abs(ref)) < 1e-13
    th = np.linspace(0.0, 2 * math.pi, 9, endpoint=False)
    x = np.stack([3 * np.cos(th), 3 * np.sin(th)], 1).reshape(-1)
    V = O.target_field(cur, n, kappa, psi, x)
    Vref = _circle_series(kappa, a, th, r=3.0)
    assert np.max(np.abs(V - Vref)) / np.max(np.abs(Vref)) < 1e-13


def test_cfie_oblique_incidence_circle():
    """Rotating the incidence direction rotates the circle solution."""
    n, kappa = 96, 6.0
    ang = 0.7
    p = (math.cos(ang), math.sin(ang))
    psi = O.solve_density(fi.circle(1.0), n, kappa, p=p)
    t = math.pi * np.arange(2 * n) / n
    ref = _circle_series(kappa, 1.0, t - ang)
    assert np.max(np.abs(psi - ref)) / np.max(np.abs(ref)) < 1e-13


# ------------------------------------------------- Nystrom CFIE on the kite

def _point_source_density(cur, n, kappa, y):
    """Density for Dirichlet data B = (i/4) H0(kappa |r - y|) (y outside the obstacle);
    the right side dB/dn - i kappa B is formed here from the Green's function."""
    _, z, dz, _ = O.discretize(cur, n)
    sp = np.hypot(dz[0], dz[1])
    nu = np.stack([dz[1] / sp, -dz[0] / sp])
    d = np.hypot(z[0] - y[0], z[1] - y[1])
    B = 0.25j * special.hankel1(0, kappa * d)
    dB = -0.25j * kappa * special.hankel1(1, kappa * d) * ((z[0] - y[0]) * nu[0] + (z[1] - y[1]) * nu[1]) / d
    A = O.cfie_matrix(cur, n, kappa)
    return np.linalg.solve(A, dB - 1j * kappa * B)


@pytest.mark.parametrize("kappa", [2.0, 9.0])
def test_cfie_kite_reciprocity(kappa):
    """Scattered fields of point sources are reciprocal: U_y(x) = U_x(y)."""
    cur = fi.kite()
    n = 160
    xa = np.array([2.6, 1.1])
    xb = np.array([-1.9, -2.4])
    Ua = O.target_field(cur, n, kappa, _point_source_density(cur, n, kappa, xa), xb)[0]
    Ub = O.target_field(cur, n, kappa, _point_source_density(cur, n, kappa, xb), xa)[0]
    assert abs(Ua - Ub) / abs(Ua) < 1e-11


@pytest.mark.parametrize("seed", [4, 19])
def test_star_geometry_matches_spectral_derivatives(seed):
    """Star branch of the node tables: z against the shape definition of the
    inputs module, z' and z'' against exact spectral differentiation of the
    sampled curve.  A star with five harmonics is a trigonometric polynomial
    of degree 6 in t, so differentiation by FFT on 2n >= 14 nodes is exact
    up to rounding; a wrong sign or factor in r', r'' fails this."""
    rng = np.random.default_rng(seed)
    cur = fi.random_star(rng, n_harm=5, amp_max=0.3)
    cur.center = (0.3, -0.2)
    for n in (16, 45):
        t, z, dz, ddz = O.discretize(cur, n)
        zp = cur.point(t)
        assert np.max(np.abs(z - zp)) < 1e-14
        k = np.fft.fftfreq(2 * n, 1.0 / (2 * n))
        k[n] = 0.0                        # Nyquist mode: zero for degree < n
        for c in range(2):
            Z = np.fft.fft(zp[c])
            d1 = np.real(np.fft.ifft(1j * k * Z))
            d2 = np.real(np.fft.ifft(-(k ** 2) * Z))
            assert np.max(np.abs(dz[c] - d1)) < 1e-12
            assert np.max(np.abs(ddz[c] - d2)) < 1e-11


@pytest.mark.parametrize("kappa", [3.0, 8.0])
def test_cfie_star_reciprocity(kappa):
    """Point-source reciprocity U_y(x) = U_x(y) on a star obstacle: the whole
    CFIE (including the curvature diagonal L2(t,t), which uses z'') through
    the star branch of the geometry."""
    rng = np.random.default_rng(23)
    cur = fi.random_star(rng, n_harm=5, amp_max=0.15)
    n = 128
    xa = np.array([2.2, 1.4])
    xb = np.array([-2.0, -1.7])
    Ua = O.target_field(cur, n, kappa, _point_source_density(cur, n, kappa, xa), xb)[0]
    Ub = O.target_field(cur, n, kappa, _point_source_density(cur, n, kappa, xb), xa)[0]
    assert abs(Ua - Ub) / abs(Ua) < 1e-11


def test_cfie_kite_spectral_convergence():
    """Far field from N = 192 and N = 384 agree to near machine precision."""
    cur = fi.kite()
    x = fi.targets_on_circle(6, 3.0)
    V = []
    for n in (96, 192):
        psi = O.solve_density(cur, n, 8.0, p=(0.8, 0.6))
        V.append(O.target_field(cur, n, 8.0, psi, x))
    assert np.max(np.abs(V[0] - V[1])) / np.max(np.abs(V[1])) < 1e-11


def test_cfie_kite_near_boundary_convergence():
    """Near Gamma (0.35 off the curve) two discretisations agree: the log-split
    quadrature resolves the near-singular source ring."""
    cur = fi.kite()
    n, kappa, p = 192, 5.0, (1.0, 0.0)
    psi = O.solve_density(cur, n, kappa, p=p)
    # points just outside the boundary, along the outward normal
    t = np.linspace(0.1, 6.2, 7)
    zz = cur.point(t)
    eps = 0.35
    dz = np.stack([-np.sin(t) - 1.3 * np.sin(2 * t), 1.5 * np.cos(t)])
    sp = np.hypot(dz[0], dz[1])
    xo = zz + eps * np.stack([dz[1] / sp, -dz[0] / sp])
    psi2 = O.solve_density(cur, 2 * n, kappa, p=p)
    V1 = O.target_field(cur, n, kappa, psi, xo.T.reshape(-1))
    V2 = O.target_field(cur, 2 * n, kappa, psi2, xo.T.reshape(-1))
    assert np.max(np.abs(V1 - V2)) < 1e-9


# ------------------------------------------------------------------ windows

def test_window_printed_parameters(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "window_params.json")))
    H = g["H"]
    assert abs(O.eta_w(0.5) - g["eta_half"]) < 1e-15
    s = O.window_centers(5, H)
    assert np.allclose(np.diff(s), 1.5 * H) and s[0] == 0.0
    t = np.linspace(-H / 2 + 1e-9, H / 2 - 1e-9, 101)
    assert np.all(O.window(t, H) == 1.0)
    assert np.all(O.window(np.array([-H - 1e-9, H + 1e-9, -30.0, 30.0]), H) == 0.0)
    # neighbouring windows overlap on [H/2, H] and sum to one there
    tt = np.linspace(H / 2, H, 501)
    assert np.max(np.abs(O.window(tt, H) + O.window(tt - 1.5 * H, H) - 1.0)) < 1e-15


def test_window_partition_of_unity():
    """sum_k w_k(t) = 1 on [0, T] (Sec. 3.1 item d)."""
    t = np.linspace(0.0, 420.0, 84001)
    s = O.window_centers(O.window_count(420.0))
    tot = sum(O.window(t - sk) for sk in s)
    assert np.max(np.abs(tot - 1.0)) < 1e-14


def test_window_smoothness():
    """w is C-infinity: its spectrum decays much faster than any low power."""
    dt = 0.005
    t = np.arange(-10.0, 10.0 + dt / 2, dt)
    w = O.window(t)
    F = np.abs(np.fft.rfft(w)) * dt
    f = np.fft.rfftfreq(t.size, dt) * 2 * math.pi
    assert F[np.argmin(np.abs(f - 20.0))] < 1e-6 * F[0]


# ---------------------------------------------------------- window spectra

def test_spectra_reassemble_closed_form():
    """sum_k e^{i w s_k} B_k^slow(w) = A(w) (eqs. Bk_def, Fk_sum) for the
    Gaussian-modulated sinusoid, whose transform is known in closed form."""
    wl = fi.circle_gauss()
    om = np.linspace(0.0, 40.0, 401)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, om)
    assert len(s) == 2
    tot = np.sum(np.exp(1j * np.outer(s, om)) * B, axis=0)
    A = fi.gauss_sine_spectrum(om)
    assert np.max(np.abs(tot - A)) < 5e-15 * 30


def test_spectra_converged_in_dt():
    """Halving dt leaves the spectra unchanged (the F1 temporal mesh is adequate)."""
    sig = fi.pulse_train(2, n=4, span=40.0, fmin=3.0, fmax=9.0)
    om = np.linspace(0, 16, 33)
    out = []
    for dt in (0.01, 0.005):
        t0 = -10.0
        n = int(math.ceil((sig.t_end - t0) / dt)) + 1
        out.append(O.window_spectra(fi.sample_signal(sig, t0, dt, n), t0, dt, 10.0, om)[1])
    assert np.max(np.abs(out[0] - out[1])) < 1e-13


def test_spectra_are_slow():
    """Recentred spectra B_k^slow are slowly varying: their inverse transform is
    confined to |t| <= H (eq. Fkslow_int)."""
    wl = fi.kite_pulses(J=8, n_x=1, n_near=1, n_far=0)
    om = np.linspace(-60, 60, 4801)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, om)
    dw = om[1] - om[0]
    for k in (3, 17):
        for t in (15.0, -15.0, 30.0):
            val = np.sum(B[k] * np.exp(-1j * om * t)) * dw / (2 * math.pi)
            assert abs(val) < 1e-8


# ---------------------------------------------------------------- synthesis

def test_e1_closed_form_no_aliasing(golden_dir):
    """Sec. 6.1: the sinc quadrature reproduces exp(-(t-10)^2)/sqrt(pi) at all t,
    including far beyond the trapezoidal aliasing period 2 pi / dw."""
    g = json.load(open(os.path.join(golden_dir, "paper_e1.json")))
    W, J = g["W"], 97
    om = np.linspace(0.0, W, J)
    F = np.exp(-om ** 2 / 4) * np.exp(1j * g["shift"] * om)
    dw = om[1] - om[0]
    T = np.concatenate([np.linspace(-20, 40, 241), [10 + 2 * math.pi / dw, 1e3, 1e4, 123456.7]])
    u = O.synthesize(F[None, :], np.array([0.0]), om, np.ones((1, J)), T)[0]
    assert np.max(np.abs(u - np.exp(-(T - 10) ** 2) / math.sqrt(math.pi))) < g["expected_max_error"]
    # the trapezoidal rule on the same nodes aliases (replica at 10 + 2pi/dw)
    _, M, wj, pj = O.full_band(om)
    Ff = np.where(pj >= 0, F[np.abs(pj)], np.conj(F[np.abs(pj)]))
    trap = np.real(np.sum(Ff * np.exp(-1j * wj * T[-4]))) * dw / (2 * math.pi)
    assert trap > 0.5


def test_e1_recentring():
    """A pulse at t = s + 10 synthesised from the recentred spectrum at centre s."""
    W, J = 12.0, 97
    om = np.linspace(0.0, W, J)
    F = np.exp(-om ** 2 / 4) * np.exp(1j * 10 * om)
    T = np.linspace(4990, 5030, 81)
    u = O.synthesize(F[None, :], np.array([5000.0]), om, np.ones((1, J)), T)[0]
    assert np.max(np.abs(u - np.exp(-(T - 5010) ** 2) / math.sqrt(math.pi))) < 1e-14


def test_synthesis_real_part_small():
    """u is real: the imaginary part dropped by Re[.] is bounded by |F(+-W)|."""
    wl = fi.circle_gauss()
    om = np.linspace(0, 32, 129)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, om)
    u = O.synthesize(B, s, om, np.ones((1, om.size)), np.linspace(0, 20, 101), return_complex=True)
    M = 2 * (om.size - 1)
    bound = np.sum(np.abs(B[:, -1])) * (om[-1] / math.pi) * (2 + math.log(M)) / M
    assert np.max(np.abs(u.imag)) < bound
    # with a spectrum that vanishes at +-W the result is real to rounding
    W, J = 12.0, 97
    om = np.linspace(0.0, W, J)
    F = np.exp(-om ** 2 / 4) * np.exp(1j * 10 * om)
    u = O.synthesize(F[None, :], np.array([0.0]), om, np.ones((1, J)), np.linspace(0, 30, 61),
                     return_complex=True)
    assert np.max(np.abs(u.imag)) < 1e-15


@pytest.mark.parametrize("W,J,tol", [(16.0, 64, 5e-5), (28.0, 113, 3e-8), (40.0, 161, 1e-9)])
def test_incident_field_reproduction(W, J, tol):
    """With V = 1 the windowed, recentred pieces sum back to a(t) (eqs. uk_def,
    bk_signal_def: sum_k b_k = b), up to the band-limit error that falls with W."""
    wl = fi.circle_gauss()
    om = np.linspace(0.0, W, J)
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, om)
    T = np.linspace(0.0, 20.0, 401)
    u = O.synthesize(B, s, om, np.ones((1, J)), T)[0]
    assert np.max(np.abs(u - fi.gauss_sine(T))) < tol


def test_incident_long_signal_many_windows():
    """Same reproduction across 29 windows and at times far past the signal."""
    sig = fi.pulse_train(1, n=12, span=380.0, fmin=4.0, fmax=8.0)
    t0, dt = -10.0, 0.01
    a = fi.sample_signal(sig, t0, dt, int(math.ceil((sig.t_end - t0) / dt)) + 1)
    om = np.linspace(0.0, 40.0, 201)
    s, B = O.window_spectra(a, t0, dt, 10.0, om)
    assert len(s) >= 20
    T = np.concatenate([np.linspace(0.0, 420.0, 841), [2000.0, 1e4]])
    u = O.synthesize(B, s, om, np.ones((1, om.size)), T)[0]
    assert np.max(np.abs(u - sig(T))) < 2e-9


def _circle_series_field(kappa, th, r=3.0):
    if kappa == 0.0:
        return np.ones_like(th, dtype=np.complex128)
    nmax = int(min(60, 10 + 6 * kappa))
    n = np.arange(-nmax, nmax + 1)
    c = (1j ** n) * special.jv(n, kappa) * special.hankel1(n, r * kappa) / special.hankel1(n, kappa)
    c = np.where(np.isfinite(c), c, 0.0)
    return np.sum(c[None, :] * np.exp(1j * np.outer(th, n)), axis=1)


def test_full_path_vs_brute_force_time_quadrature():
    """End-to-end circle: the oracle's u(x, t) against (1/pi) Re int_0^W A(w) U(x,w)
    e^{-iwt} dw with the exact series U and a graded composite Gauss-Legendre
    rule.  The tolerance is measured: it is set by the 2D log singularity at
    w = 0 (Sec. 4.2), which the plain Fourier quadrature resolves only slowly."""
    sig = lambda t: fi.gauss_sine(t, 8.0, 1.0, 7.0)
    spec = lambda w: fi.gauss_sine_spectrum(w, 8.0, 1.0, 7.0)
    cur = fi.circle(1.0)
    W, J = 20.0, 128
    om = np.linspace(0, W, J)
    t0, dt = -10.0, 0.01
    a = fi.sample_signal(sig, t0, dt, int(round(25 / dt)) + 1)
    th = np.array([0.3, 2.0, 4.0])
    x = np.stack([3 * np.cos(th), 3 * np.sin(th)], 1).reshape(-1)
    T = np.linspace(0, 30, 61)
    psi = [None] + [O.solve_density(cur, 64, w) for w in om[1:]]
    V = np.stack([O.target_field(cur, 64, w, psi[j], x) for j, w in enumerate(om)], 1)
    s, B = O.window_spectra(a, t0, dt, 10.0, om)
    u = O.synthesize(B, s, om, V, T)
    edges = np.concatenate([[0.0], W * np.geomspace(1e-8, 1, 60)])
    xg, wg = np.polynomial.legendre.leggauss(30)
    ws = np.concatenate([(b - a0) / 2 * xg + (a0 + b) / 2 for a0, b in zip(edges[:-1], edges[1:])])
    wt = np.concatenate([(b - a0) / 2 * wg for a0, b in zip(edges[:-1], edges[1:])])
    Ub = np.stack([_circle_series_field(w, th) for w in ws], 1)
    ub = np.real((Ub * spec(ws)[None, :] * wt[None, :]) @ np.exp(-1j * np.outer(ws, T))) / math.pi
    assert np.max(np.abs(ub)) > 0.3
    assert np.max(np.abs(u - ub)) < 3e-6


def test_causality_before_arrival():
    """Nothing scattered reaches r = 3 before the pulse does (zero initial data)."""
    wl = fi.circle_gauss(J=64, N=96, n_x=4, n_T=121, t_max=12.0)
    res = O.run(wl)
    # the pulse (delay 5, width 0.5) is at x = -1 at t ~ 1.5 at the earliest;
    # before that only the band-limit error at W = 16 (about 3e-5) remains
    early = res["u"][:, wl.T < 3.5]
    assert np.max(np.abs(early)) < 5e-5
    assert np.max(np.abs(res["u"])) > 0.1
