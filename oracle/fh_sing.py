"""FP64 CPU oracle for the 2D low-frequency quadrature and the scaled
convolutions of the fast-hybrid synthesis (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Like fh_oracle, this module is a plain, slow,
readable statement of what the CUDA path computes; only the test-suite, the
smoke check and the benchmark's CPU legs may import it.  It shares no code
with the product path.

It follows Anderson, Bruno & Lyon (arXiv 1807.02718), Part I:

* Sec. 4.2, eqs. gradedmesh, gradedmeshIntRule: the modified
  Filon-Clenshaw-Curtis (FCC) rule for I_0^{w_c}[F](t) = int_0^{w_c} F(w)
  e^{-iwt} dw on the graded mesh mu_j = w_c (j/M)^q, j = 1..M, with an
  N-point Clenshaw-Curtis mesh on every subinterval [mu_{j-1}, mu_j],
  j = 2..M (the paper uses M = 4, N = 8, q = 9.1).  On each subinterval F is
  replaced by its polynomial interpolant at the Clenshaw-Curtis points and
  the product with the oscillatory kernel is integrated exactly.
* Sec. 4.1.1, eqs. approx, discConv: the term-wise integral of a Fourier
  series F(delta + w) = sum_m c_m e^{2 pi i m w / P} over [-A, A].
* Sec. 4.1.2, eqs. conv_sum, conv_sum_2, approx_conv_sum: the scaled
  convolution d_n = sum_m c_m b(beta n - gamma m) and its approximation by a
  gamma-fractional DFT, a DFT and an inverse beta-fractional DFT of length L.

Readings (where the paper is silent or garbled):

* The scaled-convolution index: eq. conv_sum prints b_{beta m - gamma n},
  eq. discConv b_{beta n - m}; eq. approx_conv_sum (C^{(gamma)} on the
  coefficients, e^{+2 pi i beta n p / L} on the output) is the convolution
  theorem for d_n = sum_m c_m b(beta n - gamma m), which is discConv at
  gamma = 1.  That form is taken.
* "Exact computation of the modified moments": the oracle integrates the
  interpolating polynomial times e^{-iwt} with a Gauss-Legendre rule of
  enough nodes to be exact to rounding for the polynomial degree and the
  oscillation (see fcc_interval).
* The interval [0, mu_1] is not integrated (the composite rule sums j = 2..M,
  eq. gradedmeshIntRule).
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Sec. 4.2: graded mesh and Filon-Clenshaw-Curtis quadrature
# ---------------------------------------------------------------------------

def graded_mesh(omega_c: float, M: int = 4, q: float = 9.1) -> np.ndarray:
    """mu_j = omega_c (j / M)^q, j = 1..M (eq. gradedmesh)."""
    j = np.arange(1, M + 1, dtype=np.float64)
    return omega_c * (j / M) ** q


def cc_nodes(Nq: int) -> np.ndarray:
    """Clenshaw-Curtis points x_k = cos(pi k / (Nq - 1)), k = 0..Nq-1, on [-1, 1]."""
    return np.cos(math.pi * np.arange(Nq) / (Nq - 1))


def sing_frequencies(omega_c: float, M: int = 4, Nq: int = 8, q: float = 9.1) -> np.ndarray:
    """The frequency set F^sing on (0, omega_c]: Nq Clenshaw-Curtis points on
    each subinterval [mu_{j-1}, mu_j], j = 2..M, interval by interval (shared
    end points appear twice), shape ((M-1) * Nq,)."""
    mu = graded_mesh(omega_c, M, q)
    x = cc_nodes(Nq)
    out = []
    for j in range(1, M):
        a, b = mu[j - 1], mu[j]
        out.append(0.5 * (a + b) + 0.5 * (b - a) * x)
    return np.concatenate(out)


def cheb_interp_coeffs(fvals: np.ndarray) -> np.ndarray:
    """Coefficients a_n (n < Nq) of the polynomial sum_n a_n T_n(x) that
    interpolates fvals at the Clenshaw-Curtis points x_k = cos(pi k/(Nq-1))
    (discrete cosine transform of type I, written out):
      a_n = (2 / (Nq-1)) sum_k'' f_k cos(pi n k / (Nq-1)),
    the double prime halving the k = 0 and k = Nq-1 terms, and a_0, a_{Nq-1}
    halved once more."""
    f = np.asarray(fvals)
    n1 = f.shape[0] - 1
    k = np.arange(n1 + 1)
    w = np.ones(n1 + 1)
    w[0] = w[-1] = 0.5
    C = np.cos(math.pi * np.outer(k, k) / n1)          # [n, k]
    a = (2.0 / n1) * (C * w[None, :]) @ f
    a[0] *= 0.5
    a[-1] *= 0.5
    return a


def fcc_interval(fvals: np.ndarray, a: float, b: float, t: np.ndarray) -> np.ndarray:
    """Filon-Clenshaw-Curtis approximation of int_a^b F(w) e^{-iwt} dw from F
    at the Nq Clenshaw-Curtis points of [a, b] (in cc_nodes order): the
    interpolating polynomial p(x) = sum_n a_n T_n(x), w = delta + h x
    (delta = (a+b)/2, h = (b-a)/2), is integrated against e^{-iwt} exactly:
      h e^{-i delta t} int_{-1}^{1} p(x) e^{-i h t x} dx,
    the last integral by composite 24-point Gauss-Legendre on 1 + h|t|/6
    equal panels (at most 12 radians of phase per panel: exact to rounding for
    the degree-(Nq-1) polynomial times the exponential)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    coef = cheb_interp_coeffs(np.asarray(fvals, dtype=np.complex128))
    delta, h = 0.5 * (a + b), 0.5 * (b - a)
    xg, wg = np.polynomial.legendre.leggauss(24)
    out = np.empty(t.size, dtype=np.complex128)
    for i, ti in enumerate(t):
        kap = h * ti
        edges = np.linspace(-1.0, 1.0, int(abs(kap) / 6.0) + 2)
        x = (0.5 * np.diff(edges)[:, None] * xg[None, :] + 0.5 * (edges[1:] + edges[:-1])[:, None]).ravel()
        w = (0.5 * np.diff(edges)[:, None] * wg[None, :]).ravel()
        p = np.polynomial.chebyshev.chebval(x, coef)
        out[i] = h * np.exp(-1j * delta * ti) * np.sum(w * p * np.exp(-1j * kap * x))
    return out


def fcc_integral(F_sing: np.ndarray, omega_c: float, t, M: int = 4, Nq: int = 8,
                 q: float = 9.1) -> np.ndarray:
    """I_0^{omega_c}[F](t) ~ sum_{j=2}^{M} FCC over [mu_{j-1}, mu_j]
    (eq. gradedmeshIntRule); F_sing holds F at sing_frequencies(...)."""
    mu = graded_mesh(omega_c, M, q)
    F = np.asarray(F_sing).reshape(M - 1, Nq)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros(t.size, dtype=np.complex128)
    for j in range(1, M):
        out += fcc_interval(F[j - 1], mu[j - 1], mu[j], t)
    return out


# ---------------------------------------------------------------------------
# Sec. 4.1: term-wise integral of a Fourier series, scaled convolutions
# ---------------------------------------------------------------------------

def sinc_kernel(q, A: float, P: float):
    """b_q = 2A sinc(2A q / P) with the normalised sinc sin(pi y)/(pi y)
    (eq. discConv)."""
    return 2.0 * A * np.sinc((2.0 * A / P) * np.asarray(q, dtype=np.float64))


def fourier_series_transform(c: np.ndarray, A: float, P: float, delta: float, t) -> np.ndarray:
    """I(t) = e^{-i delta t} sum_{m=-M/2}^{M/2-1} c_m (P / (pi (alpha t - m)))
    sin(pi (2A/P)(alpha t - m)), alpha = P / (2 pi) (eq. approx): the exact
    integral over [-A, A] of (sum_m c_m e^{2 pi i m w / P}) e^{-iwt}, shifted
    by delta."""
    c = np.asarray(c, dtype=np.complex128)
    M = c.size
    m = np.arange(-M // 2, M // 2, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    alpha = P / (2 * math.pi)
    S = sinc_kernel(alpha * t[:, None] - m[None, :], A, P)
    return np.exp(-1j * delta * t) * (S @ c)


def scaled_conv_direct(c: np.ndarray, beta: float, gamma: float, n: np.ndarray, b) -> np.ndarray:
    """d_n = sum_{m=-M/2}^{M/2-1} c_m b(beta n - gamma m) (eqs. conv_sum /
    discConv; b a function of its real index)."""
    c = np.asarray(c, dtype=np.complex128)
    M = c.size
    m = np.arange(-M // 2, M // 2, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    return b(beta * n[:, None] - gamma * m[None, :]) @ c


def scaled_conv_frft(c: np.ndarray, beta: float, gamma: float, n0: int, L: int, b) -> np.ndarray:
    """eq. approx_conv_sum for n = n0 - L/2 .. n0 + L/2 - 1:
      d_n ~ (1/L) sum_{p=-L/2}^{L/2-1} C_p^{(gamma)} B_p e^{2 pi i beta n p / L},
      C_p^{(gamma)} = sum_m c_m e^{-2 pi i gamma m p / L}  (c zero-padded to L),
      B_p = sum_{m=-L/2}^{L/2-1} b_m e^{-2 pi i m p / L},
    every sum evaluated directly (the fractional transforms by their
    definition).  Returns (n, d)."""
    c = np.asarray(c, dtype=np.complex128)
    M = c.size
    if L < M or L % 2:
        raise ValueError("L must be even and >= M")
    m = np.arange(-M // 2, M // 2, dtype=np.float64)
    p = np.arange(-L // 2, L // 2, dtype=np.float64)
    Cg = np.exp(-2j * math.pi * gamma * np.outer(p, m) / L) @ c
    mb = np.arange(-L // 2, L // 2, dtype=np.float64)
    Bp = np.exp(-2j * math.pi * np.outer(p, mb) / L) @ b(mb).astype(np.complex128)
    n = n0 + np.arange(-L // 2, L // 2)
    d = (np.exp(2j * math.pi * beta * np.outer(n.astype(np.float64), p) / L) @ (Cg * Bp)) / L
    return n, d


# ---------------------------------------------------------------------------
# Sec. 4.1 (Remark Fourier-FC): FC(Gram) Fourier continuation of a smooth,
# non-periodic F on [a, b]
# ---------------------------------------------------------------------------

_FC_TABLE = None


def fc_gram_table():
    """(A, Q): continuation table (C x d) and Gram basis (d x d) written by
    gen_fc_gram.py (d = 6, C = 31; the construction is stated there)."""
    global _FC_TABLE
    if _FC_TABLE is None:
        import json
        import os
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "fc_gram_d6_c31.json")) as fh:
            t = json.load(fh)
        _FC_TABLE = (np.asarray(t["A"], dtype=np.float64), np.asarray(t["Q"], dtype=np.float64))
    return _FC_TABLE


def fc_extend(f: np.ndarray) -> np.ndarray:
    """The FC(Gram) periodic extension of the samples f_0..f_{n-1}: the
    right end's d values projected on the Gram basis and blended to zero over
    the C continuation points, plus the left end's d values (read backwards)
    blended the same way and reversed; length n + C."""
    A, Q = fc_gram_table()
    d = Q.shape[0]
    f = np.asarray(f)
    a_r = Q.T @ f[-d:]
    a_l = Q.T @ f[:d][::-1]
    e = A @ a_r + (A @ a_l)[::-1]
    return np.concatenate([f, e])


def fc_coefficients(f: np.ndarray, a: float, b: float):
    """Coefficients of eq. fourier_approx for F on [a, b] from its n
    equispaced samples (both ends included; n + C must be even): the
    extended sequence g of length M = n + C has period P = M h (h = (b-a)/(n-1)),
    c_m = (1/M) sum_l g_l e^{-2 pi i m l / M}, m = -M/2 .. M/2-1, and F(delta + w)
    ~ sum_m c_m e^{2 pi i m (w + delta - a)/P}, so the coefficients about the
    centre delta = (a+b)/2 are c_m e^{2 pi i m (delta - a)/P}.
    Returns (c', A_half = (b-a)/2, P, delta)."""
    f = np.asarray(f, dtype=np.complex128)
    n = f.size
    g = fc_extend(f)
    M = g.size
    if M % 2:
        raise ValueError("n + C must be even")
    h = (b - a) / (n - 1)
    P = M * h
    m = np.arange(-M // 2, M // 2, dtype=np.float64)
    l = np.arange(M, dtype=np.float64)
    c = (np.exp(-2j * math.pi * np.outer(m, l) / M) @ g) / M
    delta = 0.5 * (a + b)
    return c * np.exp(2j * math.pi * m * (delta - a) / P), 0.5 * (b - a), P, delta


def smooth_transform(f: np.ndarray, a: float, b: float, t) -> np.ndarray:
    """I_a^b[F](t) = int_a^b F(w) e^{-iwt} dw from equispaced samples of F by
    FC(Gram) coefficients and the term-wise integral (eq. approx)."""
    c, A, P, delta = fc_coefficients(f, a, b)
    return fourier_series_transform(c, A, P, delta, t)


# ---------------------------------------------------------------------------
# Sec. 5, steps T1b - T2d, T5: the 2D synthesis with the low-frequency split
# ---------------------------------------------------------------------------

def synthesize_sing(B: np.ndarray, B_sing: np.ndarray, s: np.ndarray, omega: np.ndarray,
                    j_c: int, V: np.ndarray, V_sing: np.ndarray, T, M: int = 4, Nq: int = 8,
                    q: float = 9.1) -> np.ndarray:
    """u(x, t) = sum_k (1/pi) Re[ I_{w_c}^{W}[F_k](t - s_k) + I_0^{w_c}[F_k](t - s_k) ]
    with F_k(w) = B_k^slow(w) V(x, w) (eqs. ukW, Ukslow_repr, fourier_sing_decomp;
    the negative frequencies by F(-w) = conj F(w), so that
    (1/2pi) int_{-W}^{W} = (1/pi) Re int_0^W).  w_c = omega[j_c]; the smooth part
    uses the samples at omega[j_c .. J-1] (FC(Gram) + eq. approx), the singular
    part the samples at sing_frequencies(w_c, M, Nq, q) (FCC, eq.
    gradedmeshIntRule).
    B (K, J), B_sing (K, n_sing), V (n_x, J), V_sing (n_x, n_sing); u (n_x, n_T)."""
    omega = np.asarray(omega, dtype=np.float64)
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    wc, W = float(omega[j_c]), float(omega[-1])
    n_x = V.shape[0]
    u = np.zeros((n_x, T.size))
    for k in range(B.shape[0]):
        tk = T - s[k]
        for i in range(n_x):
            F = B[k, j_c:] * V[i, j_c:]
            Fs = B_sing[k] * V_sing[i]
            I = smooth_transform(F, wc, W, tk) + fcc_integral(Fs, wc, tk, M, Nq, q)
            u[i] += I.real / math.pi
    return u
