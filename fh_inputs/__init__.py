"""Seeded synthetic inputs for the fast-hybrid scattering path.

This module builds the *inputs* only: obstacle descriptions, incident
signal samples, frequency meshes and per-frequency boundary sizes, target
points and sample times.  It holds none of the method's arithmetic (no
discretisation, quadrature, integral-equation or synthesis step); both the
CPU oracle and the CUDA path receive exactly these arrays.

Workload shapes follow the paper's 2D experiments: the kite of Sec. 6.2,
plane-wave incidence along a single direction (Remark 2.1), windows of
width H = 10 (Sec. 3.1), and Gaussian-type pulses and linear chirps as
incident signals (Secs. 6.2-6.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Obstacles
# ---------------------------------------------------------------------------

CURVE_CIRCLE = 0
CURVE_KITE = 1
CURVE_STAR = 2
MAX_HARMONICS = 16


@dataclass
class Curve:
    """A smooth closed curve, counter-clockwise in its parameter t in [0, 2pi).

    kind  CURVE_CIRCLE: z(t) = center + r0 (cos t, sin t)
          CURVE_KITE:   z(t) = center + (cos t + 0.65 cos 2t - 0.65, 1.5 sin t)
          CURVE_STAR:   z(t) = center + r(t) (cos t, sin t),
                        r(t) = r0 + sum_k amp[k-1] cos(k t + phase[k-1])
    """

    kind: int
    r0: float = 1.0
    amp: list = field(default_factory=list)
    phase: list = field(default_factory=list)
    center: tuple = (0.0, 0.0)

    def point(self, t):
        """Curve point z(t) (the shape definition itself, used only for sizing)."""
        t = np.asarray(t, dtype=np.float64)
        cx, cy = self.center
        if self.kind == CURVE_KITE:
            return np.stack([cx + np.cos(t) + 0.65 * np.cos(2 * t) - 0.65,
                             cy + 1.5 * np.sin(t)])
        r = np.full_like(t, self.r0)
        if self.kind == CURVE_STAR:
            for k, (a, ph) in enumerate(zip(self.amp, self.phase), start=1):
                r = r + a * np.cos(k * t + ph)
        return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)])


def circle(radius: float = 1.0) -> Curve:
    return Curve(CURVE_CIRCLE, r0=radius)


def kite() -> Curve:
    """The kite of Sec. 6.2 (also used for Fig. 6.3)."""
    return Curve(CURVE_KITE)


def random_star(rng: np.random.Generator, n_harm: int = 5, amp_max: float = 0.1) -> Curve:
    amp = rng.uniform(0.0, amp_max, n_harm).tolist()
    phase = rng.uniform(0.0, 2 * math.pi, n_harm).tolist()
    return Curve(CURVE_STAR, r0=1.0, amp=amp, phase=phase)


def perimeter(curve: Curve, n: int = 1 << 16) -> float:
    """Perimeter from a fine polygon (used only to size N by points per wavelength)."""
    t = np.linspace(0.0, 2 * math.pi, n + 1)
    z = curve.point(t)
    return float(np.sum(np.hypot(np.diff(z[0]), np.diff(z[1]))))


def max_radius(curve: Curve, n: int = 1 << 14) -> float:
    z = curve.point(np.linspace(0.0, 2 * math.pi, n, endpoint=False))
    return float(np.max(np.hypot(z[0] - curve.center[0], z[1] - curve.center[1])))


# ---------------------------------------------------------------------------
# Frequency mesh and boundary sizes
# ---------------------------------------------------------------------------

def frequency_mesh(J: int, W: float) -> np.ndarray:
    """J equispaced non-negative frequencies on [0, W], both ends included."""
    return np.linspace(0.0, W, J)


def boundary_sizes(curve: Curve, omega: np.ndarray, c: float = 1.0, ppw: float = 8.0,
                   n_min: int = 64, multiple: int = 32, n_max: int | None = None) -> np.ndarray:
    """N_j = max(n_min, ceil(ppw * kappa_j L / 2pi)) rounded up to `multiple` (even)."""
    L = perimeter(curve)
    out = []
    for w in omega:
        n = max(n_min, math.ceil(ppw * (w / c) * L / (2 * math.pi)))
        n = ((n + multiple - 1) // multiple) * multiple
        if n_max is not None:
            n = min(n, n_max)
        out.append(n)
    return np.asarray(out, dtype=np.int32)


# ---------------------------------------------------------------------------
# Incident signals a(t) (b = a(t - p.r/c), Remark 2.1)
# ---------------------------------------------------------------------------

def gauss_sine(t, f0: float = 8.0, sigma: float = 0.5, delay: float = 5.0):
    """Gaussian-modulated sinusoid sin(f0 (t-d)) exp(-(t-d)^2 / (2 sigma^2))."""
    s = np.asarray(t, dtype=np.float64) - delay
    return np.sin(f0 * s) * np.exp(-s * s / (2.0 * sigma * sigma))


def gauss_sine_spectrum(omega, f0: float = 8.0, sigma: float = 0.5, delay: float = 5.0):
    """Closed-form A(w) = int a(t) e^{i w t} dt of `gauss_sine` (exact)."""
    w = np.asarray(omega, dtype=np.float64)
    pref = sigma * math.sqrt(2 * math.pi) / 2j * np.exp(1j * w * delay)
    return pref * (np.exp(-sigma ** 2 * (w + f0) ** 2 / 2) - np.exp(-sigma ** 2 * (w - f0) ** 2 / 2))


@dataclass
class PulseTrain:
    delays: np.ndarray
    freqs: np.ndarray
    width: float = 1.0
    shift: float = 9.0

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        out = np.zeros_like(t)
        for d, f in zip(self.delays, self.freqs):
            s = t - self.shift - d
            out += np.sin(f * s) * np.exp(-s * s / (2 * self.width ** 2))
        return out

    @property
    def t_end(self) -> float:
        return float(self.shift + np.max(self.delays) + 9.0 * self.width)


def pulse_train(seed: int = 1, n: int = 40, span: float = 400.0, fmin: float = 5.0,
                fmax: float = 30.0, shift: float = 9.0) -> PulseTrain:
    """Sum of n unit Gaussian pulses, delays U[0,span], centre freqs U[fmin,fmax]."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.0, span, n)
    f = rng.uniform(fmin, fmax, n)
    return PulseTrain(d, f, 1.0, shift)


@dataclass
class Chirp:
    """Linear chirp sin(g + g^2/4000), g = 4t + 6cos(t/sqrt 12) (Sec. 6.3 form),
    under a smooth on/off envelope so the signal is compactly supported."""
    t_on: float = 0.0
    t_off: float = 100.0
    ramp: float = 5.0

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        g = 4 * t + 6 * np.cos(t / math.sqrt(12.0))
        env = _smooth_step((t - self.t_on) / self.ramp) * _smooth_step((self.t_off - t) / self.ramp)
        return env * np.sin(g + g * g / 4000.0)

    @property
    def t_end(self) -> float:
        return self.t_off


def _smooth_step(u):
    u = np.clip(u, 0.0, 1.0)
    out = np.zeros_like(u)
    inside = (u > 0) & (u < 1)
    a = np.exp(-1.0 / np.where(inside, u, 0.5))
    b = np.exp(-1.0 / np.where(inside, 1 - u, 0.5))
    out[inside] = (a / (a + b))[inside]
    out[u >= 1] = 1.0
    return out


def sample_signal(fn, t0: float, dt: float, n: int) -> np.ndarray:
    return np.ascontiguousarray(fn(t0 + dt * np.arange(n)), dtype=np.float64)


# ---------------------------------------------------------------------------
# Targets and times
# ---------------------------------------------------------------------------

def targets_on_circle(n: int, radius: float = 3.0, center=(0.0, 0.0)) -> np.ndarray:
    """n points on a circle, interleaved (x0, y0, x1, y1, ...)."""
    th = 2 * math.pi * np.arange(n) / n
    xy = np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th)], axis=1)
    return np.ascontiguousarray(xy.reshape(-1))


def long_time_grid(n_near: int = 3072, t_near: float = 480.0, n_far: int = 1024,
                   t_far: float = 1.0e4) -> np.ndarray:
    """n_near equispaced times on [0, t_near) then n_far equispaced on [t_near, t_far]."""
    a = t_near * np.arange(n_near) / n_near
    b = np.linspace(t_near, t_far, n_far)
    return np.concatenate([a, b])


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    curve: Curve
    omega: np.ndarray          # J non-negative frequencies, omega[0] = 0
    N: np.ndarray              # boundary points per frequency (even)
    c: float
    p: tuple                   # unit incidence direction
    a: np.ndarray              # signal samples a(t0 + q dt)
    t0: float
    dt: float
    H: float
    x: np.ndarray              # interleaved targets
    T: np.ndarray              # sample times
    eta: np.ndarray | None = None   # coupling per frequency (None: eta = omega)

    @property
    def n_x(self) -> int:
        return self.x.size // 2

    @property
    def J(self) -> int:
        return self.omega.size


def circle_gauss(J: int = 64, W: float = 16.0, N: int = 256, n_x: int = 16, n_T: int = 200,
                 radius_x: float = 3.0, t_max: float = 20.0, dt: float = 0.01) -> Workload:
    """Unit circle, incidence +x, Gaussian-modulated sinusoid (centre 8, width 0.5, delay 5)."""
    t0, t1 = -10.0, 12.0
    n = int(round((t1 - t0) / dt)) + 1
    return Workload(
        name=f"circle_gauss_J{J}_N{N}", curve=circle(1.0), omega=frequency_mesh(J, W),
        N=np.full(J, N, dtype=np.int32), c=1.0, p=(1.0, 0.0),
        a=sample_signal(gauss_sine, t0, dt, n), t0=t0, dt=dt, H=10.0,
        x=targets_on_circle(n_x, radius_x), T=np.linspace(0.0, t_max, n_T))


def kite_pulses(J: int = 256, W: float = 40.0, n_x: int = 1024, n_near: int = 3072,
                n_far: int = 1024, seed: int = 1, dt: float = 0.01, n_cap: int | None = None,
                ppw: float = 8.0) -> Workload:
    """Kite, incidence +x, 40-pulse train over [0,400] (+9 shift), N by 8 points/wavelength."""
    cur = kite()
    om = frequency_mesh(J, W)
    sig = pulse_train(seed)
    t0, t1 = -10.0, sig.t_end
    n = int(math.ceil((t1 - t0) / dt)) + 1
    T = long_time_grid(n_near, 480.0, n_far, 1.0e4) if n_near + n_far > 0 else np.zeros(0)
    return Workload(
        name=f"kite_pulses_J{J}", curve=cur, omega=om,
        N=boundary_sizes(cur, om, ppw=ppw, n_max=n_cap), c=1.0, p=(1.0, 0.0),
        a=sample_signal(sig, t0, dt, n), t0=t0, dt=dt, H=10.0,
        x=targets_on_circle(n_x, 3.0), T=T)


def kite_wide(J: int = 512, W: float = 160.0, n_x: int = 1024, n_near: int = 3072,
              n_far: int = 1024, seed: int = 1, dt: float = 0.005, n_cap: int | None = None,
              n_force: int | None = None) -> Workload:
    """Wide-band kite problem: J frequencies on [0, W] (8 points per wavelength,
    N up to ~1920 at W = 160; n_force scales N linearly with frequency up to
    n_force instead), the 40-pulse train with centre frequencies U[5, 30]."""
    wl = kite_pulses(J=J, W=W, n_x=n_x, n_near=n_near, n_far=n_far, seed=seed, dt=dt, n_cap=n_cap)
    if n_force is not None:
        N = np.ceil(n_force * wl.omega / W / 32.0).astype(np.int64) * 32
        wl.N = np.maximum(N, 64).astype(np.int32)
    wl.name = f"kite_wide_J{J}_W{int(W)}"
    return wl


def small_kite(J: int = 12, W: float = 6.0, n_x: int = 5, n_T: int = 37, seed: int = 3) -> Workload:
    """A tiny kite problem with ragged sizes for fast element-wise parity."""
    rng = np.random.default_rng(seed)
    cur = kite()
    om = frequency_mesh(J, W)
    N = np.asarray([64 + 2 * int(v) for v in rng.integers(0, 40, J)], dtype=np.int32)
    sig = pulse_train(seed, n=3, span=30.0, fmin=1.0, fmax=4.0, shift=9.0)
    t0, dt = -10.0, 0.02
    n = int(math.ceil((sig.t_end - t0) / dt)) + 1
    T = np.concatenate([np.linspace(0.0, 60.0, n_T - 3), [300.0, 2.5e3, 1.0e4]])
    return Workload(
        name="small_kite", curve=cur, omega=om, N=N, c=1.0, p=(0.8, 0.6),
        a=sample_signal(sig, t0, dt, n), t0=t0, dt=dt, H=10.0,
        x=targets_on_circle(n_x, 2.9, center=(0.1, -0.05)), T=T)


def star_batch(count: int = 32, J: int = 128, seed: int = 7, wmax_lo: float = 20.0,
               wmax_hi: float = 100.0, n_cap: int = 2048):
    """Random star obstacles, J frequencies each on [0, w_max], w_max ~ U(lo, hi)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        cur = random_star(rng)
        W = float(rng.uniform(wmax_lo, wmax_hi))
        om = frequency_mesh(J, W)
        out.append((cur, om, boundary_sizes(cur, om, n_max=n_cap)))
    return out
