"""FP64 CPU oracle for the fast-hybrid 2D scattering path (test infrastructure).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, readable statement
of what the hot path computes.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path (the CUDA
library and its Python binding) never does, and shares no code with it.

Every function follows a passage of Anderson, Bruno & Lyon, "High-order,
dispersionless 'fast-hybrid' wave equation solver. Part I" (arXiv 1807.02718),
cited by section / equation label.  Where the paper defers to another source
or is silent, the reading taken is stated in the docstring:

* Nystrom discretisation of the CFIE (Sec. 2.3, eq. CFIE_direct): the paper
  cites Colton & Kress Sec. 3.5 without restating it; the logarithmic
  splitting with Kress's trigonometric weights is written out here.
* omega = 0 (Sec. 4.2): no integral equation is solvable there; the 2D
  low-frequency limit of the radiating solution with data e^{i kappa p.r}
  is the constant 1, so V(x, 0) := 1.
* Full-band mesh (Sec. 4.1, eqs. fourier_approx / approx): J non-negative
  nodes include 0 and W; M = 2(J-1) nodes on [-W, W) with F(-w) = conj F(w)
  for the real signals used.

Floating point is IEEE binary64 throughout (numpy float64 / complex128).
Library primitives used as single steps: scipy.special Bessel functions,
numpy.linalg.solve (LU with partial pivoting), matrix products.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

EULER_GAMMA = 0.57721566490153286061

# Curve kinds (same numbering as the inputs module; definitions restated here).
CURVE_CIRCLE, CURVE_KITE, CURVE_STAR = 0, 1, 2


# ---------------------------------------------------------------------------
# Step a1: boundary discretisation (Sec. 2.3; Nystrom nodes t_i = pi i / n)
# ---------------------------------------------------------------------------

def discretize(curve, n: int):
    """Nodes t_i = pi i / n (i < 2n) and z, z', z'' of the parametrised curve.

    Returns (t, z, dz, ddz) with z, dz, ddz of shape (2, 2n).
    """
    N = 2 * n
    t = math.pi * np.arange(N, dtype=np.float64) / n
    cx, cy = curve.center
    c1, s1 = np.cos(t), np.sin(t)
    if curve.kind == CURVE_KITE:
        c2, s2 = np.cos(2 * t), np.sin(2 * t)
        z = np.stack([cx + c1 + 0.65 * c2 - 0.65, cy + 1.5 * s1])
        dz = np.stack([-s1 - 1.3 * s2, 1.5 * c1])
        ddz = np.stack([-c1 - 2.6 * c2, -1.5 * s1])
        return t, z, dz, ddz
    r = np.full(N, float(curve.r0))
    dr = np.zeros(N)
    ddr = np.zeros(N)
    if curve.kind == CURVE_STAR:
        for k, (a, ph) in enumerate(zip(curve.amp, curve.phase), start=1):
            r += a * np.cos(k * t + ph)
            dr += -k * a * np.sin(k * t + ph)
            ddr += -k * k * a * np.cos(k * t + ph)
    z = np.stack([cx + r * c1, cy + r * s1])
    dz = np.stack([dr * c1 - r * s1, dr * s1 + r * c1])
    ddz = np.stack([ddr * c1 - 2 * dr * s1 - r * c1, ddr * s1 + 2 * dr * c1 - r * s1])
    return t, z, dz, ddz


# ---------------------------------------------------------------------------
# Step a2: Nystrom matrix of the direct CFIE (Sec. 2.3, eq. CFIE_direct)
# ---------------------------------------------------------------------------

def kress_weights(n: int) -> np.ndarray:
    """Kress quadrature weights R_d for the log kernel ln(4 sin^2((t-tau)/2)).

    R_d = -(2 pi / n) sum_{m=1}^{n-1} cos(m pi d / n) / m - (pi / n^2) cos(pi d),
    d = 0..2n-1; the weight for the pair (t_i, t_l) is R_{(i-l) mod 2n}.
    """
    N = 2 * n
    d = np.arange(N, dtype=np.float64)
    m = np.arange(1, n, dtype=np.float64)
    tab = np.cos(np.outer(d, m) * math.pi / n) / m[None, :]
    return -(2 * math.pi / n) * tab.sum(axis=1) - (math.pi / n ** 2) * np.cos(math.pi * d)


def cfie_matrix(curve, n: int, omega: float, c: float = 1.0, eta: float | None = None) -> np.ndarray:
    """Nystrom matrix A of  (1/2) psi + K* psi - i eta S psi  (eq. CFIE_direct).

    Rows are targets t_i, columns sources t_l.  With kappa = omega / c,
    r = |z(t_i) - z(t_l)|, speed s_l = |z'(t_l)| and
    N_il = z2'(t_i)(z1(t_l) - z1(t_i)) - z1'(t_i)(z2(t_l) - z2(t_i)):

      S kernel   M  = (i/4) H0(kappa r) s_l,      M1 = -(1/4pi) J0(kappa r) s_l
      K* kernel  L  = (i kappa/4) H1(kappa r)/r N_il s_l/s_i,
                 L1 = -(kappa/4pi) J1(kappa r)/r N_il s_l/s_i
      M2 = M - M1 ln(4 sin^2((t_i - t_l)/2)),  L2 = L - L1 ln(4 sin^2(...))
      diagonal: M1 = -s/4pi, M2 = [i/4 - C/2pi - ln(kappa s/2)/2pi] s,
                L1 = 0,      L2 = (z1'' z2' - z2'' z1') / (4 pi s^2)
      A = I/2 + R o (L1 - i eta M1) + (pi/n)(L2 - i eta M2).
    """
    if eta is None:
        eta = omega
    kappa = omega / c
    N = 2 * n
    t, z, dz, ddz = discretize(curve, n)
    speed = np.hypot(dz[0], dz[1])
    ii, ll = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    off = ii != ll
    d1 = z[0][ll] - z[0][ii]
    d2 = z[1][ll] - z[1][ii]
    r = np.hypot(d1, d2)
    r_safe = np.where(off, r, 1.0)
    x = kappa * r_safe
    J0, Y0 = special.j0(x), special.y0(x)
    J1, Y1 = special.j1(x), special.y1(x)
    H0 = J0 + 1j * Y0
    H1 = J1 + 1j * Y1
    Nil = dz[1][ii] * d1 - dz[0][ii] * d2
    sl = speed[ll]
    si = speed[ii]
    dt = np.where(off, t[ii] - t[ll], 1.0)
    logsin = np.where(off, np.log(4.0 * np.sin(dt / 2.0) ** 2), 0.0)

    M = 0.25j * H0 * sl
    M1 = -J0 * sl / (4 * math.pi)
    M2 = M - M1 * logsin
    L = 0.25j * kappa * H1 / r_safe * Nil * sl / si
    L1 = -(kappa / (4 * math.pi)) * J1 / r_safe * Nil * sl / si
    L2 = L - L1 * logsin

    diag = np.arange(N)
    M1[diag, diag] = -speed / (4 * math.pi)
    M2[diag, diag] = (0.25j - EULER_GAMMA / (2 * math.pi)
                      - np.log(kappa * speed / 2.0) / (2 * math.pi)) * speed
    L1[diag, diag] = 0.0
    L2[diag, diag] = (ddz[0] * dz[1] - ddz[1] * dz[0]) / (4 * math.pi * speed ** 2)

    R = kress_weights(n)[(ii - ll) % N]
    A = 0.5 * np.eye(N) + R * (L1 - 1j * eta * M1) + (math.pi / n) * (L2 - 1j * eta * M2)
    return A


def cfie_rhs(curve, n: int, omega: float, c: float = 1.0, p=(1.0, 0.0),
             eta: float | None = None) -> np.ndarray:
    """Right side dB/dn - i eta B of eq. CFIE_direct for B = e^{i kappa p.r}.

    The data are those of the fixed density set Psi (Sec. 3.2, eq. psikslow_repr):
    plane-wave incidence along p with unit spectrum.  n is the outward normal
    (z2', -z1')/|z'| of the counter-clockwise curve.
    """
    if eta is None:
        eta = omega
    kappa = omega / c
    _, z, dz, _ = discretize(curve, n)
    speed = np.hypot(dz[0], dz[1])
    nu1, nu2 = dz[1] / speed, -dz[0] / speed
    B = np.exp(1j * kappa * (p[0] * z[0] + p[1] * z[1]))
    return (1j * kappa * (p[0] * nu1 + p[1] * nu2) - 1j * eta) * B


def solve_density(curve, n: int, omega: float, c: float = 1.0, p=(1.0, 0.0),
                  eta: float | None = None) -> np.ndarray:
    """psi_p(., omega) at the 2n nodes (step F3): LU solve of A psi = g."""
    A = cfie_matrix(curve, n, omega, c, eta)
    g = cfie_rhs(curve, n, omega, c, p, eta)
    return np.linalg.solve(A, g)


# ---------------------------------------------------------------------------
# Step a5: target field V(x, omega) = int psi G dsigma (eqs. freq_domain_repr,
# Ukslow_repr), trapezoidal rule on the Nystrom nodes
# ---------------------------------------------------------------------------

def target_field(curve, n: int, omega: float, psi: np.ndarray, x: np.ndarray,
                 c: float = 1.0) -> np.ndarray:
    """V(x, omega) = (pi/n) sum_i (i/4) H0(kappa |x - z_i|) |z'_i| psi_i.

    x is interleaved (x0, y0, x1, y1, ...).  For omega = 0 the reading
    V := 1 is used (2D low-frequency limit, Sec. 4.2).
    """
    xy = np.asarray(x, dtype=np.float64).reshape(-1, 2)
    if omega == 0.0:
        return np.ones(xy.shape[0], dtype=np.complex128)
    kappa = omega / c
    _, z, dz, _ = discretize(curve, n)
    speed = np.hypot(dz[0], dz[1])
    r = np.hypot(xy[:, 0:1] - z[0][None, :], xy[:, 1:2] - z[1][None, :])
    G = 0.25j * (special.j0(kappa * r) + 1j * special.y0(kappa * r))
    return (math.pi / n) * (G * speed[None, :]) @ psi


# ---------------------------------------------------------------------------
# Step a4: windows and window spectra (Sec. 3.1 eq. window_func; Sec. 3.2
# eqs. ak_signal_def, Bkslow_eqn)
# ---------------------------------------------------------------------------

def eta_w(u):
    """Smooth cut-off eta(u) = exp(2 e^{-1/u} / (u - 1)) on (0,1); 1 for u<=0; 0 for u>=1."""
    u = np.asarray(u, dtype=np.float64)
    out = np.where(u <= 0.0, 1.0, 0.0)
    inside = (u > 0.0) & (u < 1.0)
    ui = np.where(inside, u, 0.5)
    val = np.exp(2.0 * np.exp(-1.0 / ui) / (ui - 1.0))
    return np.where(inside, val, out)


def window(t, H: float = 10.0):
    """Window w(t) of eq. window_func: 1 on |t| < H/2, 0 for |t| > H, smooth between."""
    t = np.asarray(t, dtype=np.float64)
    left = 1.0 - eta_w((t + H) / (H / 2))
    right = eta_w((t - H / 2) / (H / 2))
    return np.where(np.abs(t) > H, 0.0,
                    np.where(t <= -H / 2, left, np.where(t >= H / 2, right, 1.0)))


def window_centers(K: int, H: float = 10.0) -> np.ndarray:
    """s_k = 3 (k-1) H / 2, k = 1..K (Sec. 3.1, items a-d)."""
    return 1.5 * H * np.arange(K, dtype=np.float64)


def window_count(t_last: float, H: float = 10.0) -> int:
    """Number of windows k >= 1 whose support [s_k - H, s_k + H] starts before t_last."""
    K = 0
    while 1.5 * H * K - H < t_last:
        K += 1
    return max(K, 1)


def window_spectra(a: np.ndarray, t0: float, dt: float, H: float, omega: np.ndarray):
    """B_k^slow(omega_j) = int_{-H}^{H} w(tau) a(s_k + tau) e^{i omega tau} dtau (eq. Bkslow_eqn).

    a holds samples a(t0 + q dt); a vanishes outside the sampled span.  The
    integral is the trapezoidal rule on tau_q = -H + q dt (the integrand
    vanishes at both ends).  Returns (s, B) with B of shape (K, J).
    """
    a = np.asarray(a, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    Q = int(round(2 * H / dt))
    tau = -H + dt * np.arange(Q + 1)
    w = window(tau, H)
    K = window_count(t0 + (a.size - 1) * dt, H)
    s = window_centers(K, H)
    phase = np.exp(1j * np.outer(omega, tau))           # (J, Q+1)
    B = np.zeros((K, omega.size), dtype=np.complex128)
    for k in range(K):
        start = int(round((s[k] - H - t0) / dt))
        idx = start + np.arange(Q + 1)
        ok = (idx >= 0) & (idx < a.size)
        vals = np.where(ok, a[np.clip(idx, 0, a.size - 1)], 0.0)
        B[k] = dt * (phase @ (w * vals))
    return s, B


# ---------------------------------------------------------------------------
# Steps a6-a7: band-limited recentred synthesis (Sec. 3.2 eq. ukW; Sec. 4.1
# eqs. fourier_approx, approx; Sec. 5 steps T1-T5)
# ---------------------------------------------------------------------------

def full_band(omega: np.ndarray):
    """Full-band nodes w_j = -W + j dw, j < M = 2(J-1), and the map to the
    non-negative mesh: p_j >= 0 means F(w_j) = F(omega_{p_j}); p_j < 0 means
    F(w_j) = conj F(omega_{-p_j})."""
    J = omega.size
    W = float(omega[-1])
    M = 2 * (J - 1)
    dw = W / (J - 1)
    wj = -W + dw * np.arange(M)
    pj = np.arange(M) - (J - 1)
    return W, M, wj, pj


def synthesize(B: np.ndarray, s: np.ndarray, omega: np.ndarray, V: np.ndarray,
               T: np.ndarray, return_complex: bool = False, t_chunk: int = 512):
    """u(x, t) = sum_k Re[(1/2pi) sum_m c_m(x,k) 2W sinc(W (t - s_k)/pi - m)].

    F_k(w) = B_k^slow(w) V(x, w) (eq. Ukslow_repr) on the full band, c_m its
    DFT coefficients c_m = (1/M) sum_j F_k(w_j) e^{-i pi m w_j / W}
    (m = -M/2 .. M/2-1, eq. fourier_approx with P = 2A = 2W), and the term-wise
    exact integral of the trigonometric interpolant (eq. approx with delta = 0,
    alpha = W/pi); sinc is the normalised sin(pi y)/(pi y).  The sum over k is
    step T5 (eq. uk_def).
    V has shape (n_x, J), B (K, J); returns u of shape (n_x, n_T).
    """
    B = np.asarray(B, dtype=np.complex128)
    V = np.asarray(V, dtype=np.complex128)
    T = np.asarray(T, dtype=np.float64)
    W, M, wj, pj = full_band(np.asarray(omega, dtype=np.float64))
    m = np.arange(-M // 2, M // 2, dtype=np.float64)
    E = np.exp(-1j * math.pi * np.outer(m, wj) / W) / M        # (M, M): [m, j]
    pos = pj >= 0
    idx = np.abs(pj)
    n_x = V.shape[0]
    out = np.zeros((n_x, T.size), dtype=np.complex128)
    for k in range(B.shape[0]):
        Fk = B[k][None, idx] * V[:, idx]                         # (n_x, M)
        Fk = np.where(pos[None, :], Fk, np.conj(Fk))
        ck = Fk @ E.T                                            # (n_x, M): c_m
        for a0 in range(0, T.size, t_chunk):
            y = W * (T[a0:a0 + t_chunk] - s[k]) / math.pi
            S = 2 * W * np.sinc(y[:, None] - m[None, :])         # (nt, M)
            out[:, a0:a0 + t_chunk] += (ck @ S.T) / (2 * math.pi)
    return out if return_complex else out.real


# ---------------------------------------------------------------------------
# The whole path (Sec. 5, steps F1-F5 and T0-T6)
# ---------------------------------------------------------------------------

def solve_all(wl):
    """Densities psi_p(., omega_j) for every omega_j > 0 (step F3); None at omega = 0."""
    out = []
    for j, w in enumerate(wl.omega):
        if w == 0.0:
            out.append(None)
            continue
        eta = None if wl.eta is None else float(wl.eta[j])
        out.append(solve_density(wl.curve, int(wl.N[j]) // 2, float(w), wl.c, wl.p, eta))
    return out


def target_fields(wl, psi, x=None) -> np.ndarray:
    """V(x, omega_j) for all targets and frequencies (step F5 without the B factor)."""
    x = wl.x if x is None else x
    n_x = np.asarray(x).size // 2
    V = np.empty((n_x, wl.J), dtype=np.complex128)
    for j, w in enumerate(wl.omega):
        V[:, j] = target_field(wl.curve, int(wl.N[j]) // 2, float(w), psi[j], x, wl.c)
    return V


def run(wl, x=None, T=None):
    """Scattered field u(x, T) for a workload: F1-F5 then T0-T6."""
    psi = solve_all(wl)
    s, B = window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
    V = target_fields(wl, psi, x)
    u = synthesize(B, s, wl.omega, V, wl.T if T is None else T)
    return dict(psi=psi, s=s, B=B, V=V, u=u)
