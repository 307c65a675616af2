"""Pins of the oracle's low-frequency quadrature, Fourier-continuation and
scaled-convolution steps (Sec. 4.1, Sec. 4.2) against closed forms, textbook
special cases, the paper's printed parameters and error table, and a
brute-force time-domain quadrature."""
import json
import math
import os

import numpy as np
import pytest
from scipy import special

import fh_inputs as fi
import oracle as O
from oracle import fh_sing as S


def poly_exp_integral(coef, a, b, t):
    """int_a^b p(w) e^{-iwt} dw exactly (p in monomial coefficients), by the
    antiderivative e^{sw} sum_j (-1)^j k!/(k-j)! w^{k-j} / s^{j+1}, s = -it,
    in 40-digit arithmetic (t = 0: the polynomial's own integral)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    if t == 0:
        return complex(mp.fsum(mp.mpf(c) * (mp.mpf(b) ** (k + 1) - mp.mpf(a) ** (k + 1)) / (k + 1)
                               for k, c in enumerate(coef)))
    s = mp.mpc(0, -t)

    def anti(w):
        w = mp.mpf(w)
        tot = mp.mpc(0)
        for k, c in enumerate(coef):
            tot += mp.mpf(c) * mp.fsum((-1) ** j * mp.factorial(k) / mp.factorial(k - j) * w ** (k - j)
                                       / s ** (j + 1) for j in range(k + 1))
        return mp.exp(s * w) * tot
    return complex(anti(b) - anti(a))


def test_graded_mesh_printed_parameters():
    """Sec. 4.2: M = 4, N = 8, q = 9.1, mu_j = w_c (j/4)^9.1; (M-1) N points."""
    mu = S.graded_mesh(2.0)
    assert np.allclose(mu, 2.0 * (np.arange(1, 5) / 4.0) ** 9.1, rtol=1e-15)
    assert mu[-1] == 2.0
    assert S.sing_frequencies(2.0).size == 3 * 8
    x = S.cc_nodes(8)
    assert x[0] == 1.0 and abs(x[-1] + 1.0) < 1e-15


def test_chebyshev_interpolant_at_nodes():
    rng = np.random.default_rng(1)
    f = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    a = S.cheb_interp_coeffs(f)
    assert np.allclose(np.polynomial.chebyshev.chebval(S.cc_nodes(8), a), f, atol=1e-14)
    # T_5 sampled at the nodes has the single coefficient a_5 = 1
    e = S.cheb_interp_coeffs(np.cos(5 * np.arccos(S.cc_nodes(8))))
    assert np.allclose(e, np.eye(8)[5], atol=1e-14)


@pytest.mark.parametrize("t", [0.0, 0.7, 13.0, 1.0e3, 1.0e4])
def test_fcc_exact_on_polynomials(t):
    """The FCC rule integrates (polynomial of degree < N) x e^{-iwt} exactly."""
    rng = np.random.default_rng(2)
    coef = rng.standard_normal(8)
    a, b = 0.3, 1.1
    w = 0.5 * (a + b) + 0.5 * (b - a) * S.cc_nodes(8)
    f = np.polynomial.polynomial.polyval(w, coef)
    got = S.fcc_interval(f, a, b, np.array([t]))[0]
    ref = poly_exp_integral(coef, a, b, t)
    assert abs(got - ref) < 1e-13 * max(1.0, abs(ref))


@pytest.mark.parametrize("t", [0.0, 1.0, 40.0])
def test_fcc_graded_rule_on_log_singular_integrand(t):
    """F(w) = w^0.3 log(w) e^{2iw} (singular derivative at 0) on (mu_1, w_c]:
    with the paper's M = 4, N = 8, q = 9.1 the composite rule is within the
    O(M^-(1+N)) = 4^-9 scale (5e-5) of the adaptive 30-digit quadrature of the
    same integral, and the error falls by more than 10x at M = 8 (q > N + 1,
    Sec. 4.2)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    wc = 1.5
    F = lambda w: w ** 0.3 * np.log(w) * np.exp(2j * w)
    g = lambda w: w ** mp.mpf(0.3) * mp.log(w) * mp.exp(mp.mpc(0, 2) * w - mp.mpc(0, t) * w)
    errs = []
    for M in (4, 8):
        mu = S.graded_mesh(wc, M)
        got = S.fcc_integral(F(S.sing_frequencies(wc, M)), wc, np.array([t]), M)[0]
        ref = complex(mp.quad(g, [mp.mpf(v) for v in mu]))
        errs.append(abs(got - ref))
    assert errs[0] < 5e-5 and errs[1] < errs[0] / 10


def test_fourier_series_transform_is_the_termwise_integral():
    """eq. approx: the sinc sum equals int_{-A}^{A} sum_m c_m e^{2 pi i m w/P}
    e^{-i(delta+w)t} dw, computed by a fine Gauss-Legendre rule."""
    rng = np.random.default_rng(3)
    c = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    A, P, delta = 2.5, 7.3, 4.0
    T = np.array([-3.0, 0.0, 0.4, 9.0, 250.0])
    got = S.fourier_series_transform(c, A, P, delta, T)
    xg, wg = np.polynomial.legendre.leggauss(4000)
    w = A * xg
    m = np.arange(-6, 6)
    Fs = np.exp(2j * math.pi * np.outer(w, m) / P) @ c
    ref = (A * wg * Fs) @ np.exp(-1j * np.outer(w + delta, T))
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_scaled_convolution_direct_is_the_transform_on_a_grid():
    """eq. discConv: at t_n = n dt the transform is e^{-i delta t_n} d_n with
    beta = alpha dt, gamma = 1 and b the sinc kernel."""
    rng = np.random.default_rng(4)
    c = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    A, P, delta, dt = 3.0, 8.0, 1.5, 0.37
    n = np.arange(-20, 41)
    beta = P / (2 * math.pi) * dt
    d = S.scaled_conv_direct(c, beta, 1.0, n, lambda q: S.sinc_kernel(q, A, P))
    ref = S.fourier_series_transform(c, A, P, delta, n * dt)
    assert np.max(np.abs(np.exp(-1j * delta * n * dt) * d - ref)) < 1e-12 * np.max(np.abs(ref))


def test_frft_with_integer_scaling_is_the_circular_convolution():
    """beta = gamma = 1: the fractional transforms are ordinary DFTs and eq.
    approx_conv_sum is the convolution theorem, exact (no wrap-around for
    L >= M + N) for any kernel sampled at the integers."""
    rng = np.random.default_rng(5)
    c = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    b = lambda q: np.exp(-0.1 * np.asarray(q, dtype=float) ** 2) * np.cos(np.asarray(q, dtype=float))
    L = 64
    n, d = S.scaled_conv_frft(c, 1.0, 1.0, 0, L, b)
    keep = np.abs(n) <= 20
    ref = S.scaled_conv_direct(c, 1.0, 1.0, n[keep], b)
    assert np.max(np.abs(d[keep] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_frft_error_on_the_paper_example(golden_dir):
    """Table tab:fast_conv_table's setting (F(w) = exp(-(w-10)^2/4) exp(-8iw) on
    [8, 15], time step 0.2; "the particular selection of the coefficients is
    immaterial"): coefficients of F on a period P = 1.3 (2A) > 2A, M = 100,
    N = 2000 times.  The FFT form with L = 2N and 4N differs from the direct
    sum by far less than the paper's eps^Fast for N <= 1e3 at M = 5000
    (6.2e-6): below 1e-8.  (With P = 2A, i.e. b sampled at the integers as
    2A delta_q, the same form is only O(q/L) accurate; the FC(Gram) pieces of
    Sec. 4.2 always have P > 2A.)"""
    table = json.load(open(os.path.join(golden_dir, "paper_fast_conv.json")))
    A, delta = 3.5, 11.5
    P = 1.3 * 2 * A
    M = 100
    w = delta + A * np.arange(-M // 2, M // 2) / (M // 2)
    F = np.exp(-(w - 10.0) ** 2 / 4.0) * np.exp(-8j * w)
    m = np.arange(-M // 2, M // 2)
    c = (np.exp(-2j * math.pi * np.outer(m, w - delta) / P) @ F) / M
    b = lambda q: S.sinc_kernel(q, A, P)
    beta = P / (2 * math.pi) * 0.2
    N = 2000
    errs = []
    for L in (2 * N, 4 * N):
        n, d = S.scaled_conv_frft(c, beta, 1.0, L // 2, L, b)
        keep = (n >= 0) & (n < N)
        ref = S.scaled_conv_direct(c, beta, 1.0, n[keep], b)
        errs.append(np.max(np.abs(d[keep] - ref)))
    assert max(errs) < 1e-8 < min(table["right"]["eps"][:3])


def test_fc_gram_basis_and_table():
    """Q is orthonormal on its d points and spans the polynomials of degree
    < d (projection reproduces them); the table rows are finite and the
    continuation of a constant blends it to zero (first value ~1, last ~0)."""
    A, Q = S.fc_gram_table()
    d = Q.shape[0]
    assert np.allclose(Q.T @ Q, np.eye(d), atol=1e-13)
    u = np.arange(d, dtype=float)
    for k in range(d):
        p = (u - 3.3) ** k
        assert np.allclose(Q @ (Q.T @ p), p, atol=1e-9 * max(1.0, np.max(np.abs(p))))
    e = A @ (Q.T @ np.ones(d))
    assert abs(e[0] - 1.0) < 0.5 and abs(e[-1]) < 1e-3


@pytest.mark.parametrize("f,a,b,bound", [(lambda x: np.exp(x) * np.cos(7 * x) + 1 / (2 + x), 0.0, 1.0, 1e-11),
                                         (lambda x: np.exp(3.1j * x) * np.exp(-0.05 * (x - 4) ** 2)
                                          / (1 + 0.1 * x), 1.3, 9.7, 1e-8)])
def test_fc_gram_converges_on_non_periodic_functions(f, a, b, bound):
    """The FC(Gram) Fourier series of a smooth non-periodic function matches
    it between the samples, with the algebraic order d = 6 of the table
    (Remark Fourier-FC: a user-prescribed negative power of the sample
    count): from 161 to 321 samples the relative error falls by more than 40x
    (2^6 = 64 nominally), to below 1e-11 for a slowly varying function and
    1e-8 for one with 4 radians per unit of its variable."""
    errs = []
    for n in (161, 321):
        w = np.linspace(a, b, n)
        c, A, P, delta = S.fc_coefficients(f(w), a, b)
        ws = np.linspace(a, b, 997)
        m = np.arange(-c.size // 2, c.size // 2)
        approx = np.exp(2j * math.pi * np.outer(ws - delta, m) / P) @ c
        errs.append(np.max(np.abs(approx - f(ws))) / np.max(np.abs(f(ws))))
    assert errs[1] < bound and errs[1] < errs[0] / 40


def _circle_series_field(kappa, th, r=3.0, nmax=60):
    n = np.arange(-nmax, nmax + 1)
    with np.errstate(invalid="ignore", over="ignore"):
        c = (1j ** n) * special.jv(n, kappa) * special.hankel1(n, r * kappa) / special.hankel1(n, kappa)
    c = np.where(np.isfinite(c), c, 0.0)
    return np.sum(c[None, :] * np.exp(1j * np.outer(th, n)), axis=1)


def test_sing_synthesis_tightens_the_brute_force_bound():
    """End-to-end circle (as the plain path's brute-force pin, on a finer
    mesh: 256 frequencies on [0, 20]): with the low-frequency split (FCC on
    (0, w_c], w_c = 5 dw, FC(Gram) on [w_c, W]) u agrees with the exact
    time-domain quadrature within 6e-9 (measured 4.8e-9), where the plain
    periodic synthesis on the same mesh is 2.6e-8 away (the 2D logarithmic
    singularity at w = 0, Sec. 4.2)."""
    sig = lambda t: fi.gauss_sine(t, 8.0, 1.0, 7.0)
    spec = lambda w: fi.gauss_sine_spectrum(w, 8.0, 1.0, 7.0)
    cur = fi.circle(1.0)
    W, J, j_c = 20.0, 256, 5
    om = np.linspace(0, W, J)
    t0, dt = -10.0, 0.01
    a = fi.sample_signal(sig, t0, dt, int(round(25 / dt)) + 1)
    th = np.array([0.3, 2.0, 4.0])
    x = np.stack([3 * np.cos(th), 3 * np.sin(th)], 1).reshape(-1)
    T = np.linspace(0, 30, 61)
    psi = [None] + [O.solve_density(cur, 64, w) for w in om[1:]]
    V = np.stack([O.target_field(cur, 64, w, psi[j], x) for j, w in enumerate(om)], 1)
    s, B = O.window_spectra(a, t0, dt, 10.0, om)
    osg = S.sing_frequencies(om[j_c])
    Vs = np.stack([O.target_field(cur, 64, w, O.solve_density(cur, 64, w), x) for w in osg], 1)
    _, Bs = O.window_spectra(a, t0, dt, 10.0, osg)
    u_sing = S.synthesize_sing(B, Bs, s, om, j_c, V, Vs, T)
    u_plain = O.synthesize(B, s, om, V, T)
    edges = np.concatenate([[0.0], W * np.geomspace(1e-8, 1, 60)])
    xg, wg = np.polynomial.legendre.leggauss(30)
    ws = np.concatenate([(b - a0) / 2 * xg + (a0 + b) / 2 for a0, b in zip(edges[:-1], edges[1:])])
    wt = np.concatenate([(b - a0) / 2 * wg for a0, b in zip(edges[:-1], edges[1:])])
    Ub = np.stack([_circle_series_field(w, th) for w in ws], 1)
    ub = np.real((Ub * spec(ws)[None, :] * wt[None, :]) @ np.exp(-1j * np.outer(ws, T))) / math.pi
    e_sing, e_plain = np.max(np.abs(u_sing - ub)), np.max(np.abs(u_plain - ub))
    assert np.max(np.abs(ub)) > 0.3
    assert e_sing < 6e-9 and e_sing < e_plain / 4
