"""Generate bessel_cheb.h: Chebyshev coefficients for J0, Y0, J1, Y1 in FP64.

The device routine (bessel.cuh) evaluates the four functions together:

  x < 8 (variable t = x^2/32 - 1 in [-1, 1]; all four series are entire in x^2):
      J0(x)            = A0(t)
      Y0(x)            = (2/pi) J0(x) ln(x/2) + A1(t)
      J1(x)            = x A2(t)
      Y1(x)            = (2/pi) J1(x) ln(x/2) - 2/(pi x) + x A3(t)
  x >= 8 (Hankel's asymptotic form, H_nu = sqrt(2/(pi x)) (P_nu + i Q_nu) e^{i chi_nu},
          chi_nu = x - (2 nu + 1) pi/4; variable u = (x0/x)^2 on each piece):
      P0 = B0(t), Q0 = (8/x) B1(t), P1 = B2(t), Q1 = (8/x) B3(t)
  on the pieces x in [8, 20] and [20, inf).

Each function is interpolated at Chebyshev points of the first kind with
mpmath at 40 digits and its Chebyshev series truncated once the remaining
coefficients fall below 1e-17 of the function scale.  This is Chebyshev
interpolation of the functions defined by their series and by the Hankel
asymptotic form (Abramowitz & Stegun 9.1.10-9.1.11 and 9.2.5-9.2.6); the
coefficients are this script's output, not taken from any library.

    python gen_bessel_cheb.py > bessel_cheb.h      (needs mpmath)
"""
import mpmath as mp

mp.mp.dps = 40
TWO_PI_INV = 2 / mp.pi
TOL = mp.mpf("1e-17")
NPTS = 48


def cheb(f, n=NPTS):
    xs = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n)]
    fs = [f(x) for x in xs]
    c = []
    for j in range(n):
        s = mp.fsum(fs[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / n) for k in range(n))
        c.append(2 * s / n if j else s / n)
    scale = max(abs(v) for v in c)
    last = max(j for j, v in enumerate(c) if abs(v) > TOL * max(scale, 1))
    return c[: last + 1]


def x_small(t):
    return mp.sqrt(32 * (t + 1))


def a0(t):
    return mp.besselj(0, x_small(t))


def a1(t):
    x = x_small(t)
    return mp.bessely(0, x) - TWO_PI_INV * mp.besselj(0, x) * mp.log(x / 2)


def a2(t):
    x = x_small(t)
    return mp.besselj(1, x) / x


def a3(t):
    x = x_small(t)
    return (mp.bessely(1, x) - TWO_PI_INV * mp.besselj(1, x) * mp.log(x / 2) + 2 / (mp.pi * x)) / x


def pq(nu, x):
    chi = x - (2 * nu + 1) * mp.pi / 4
    h = mp.hankel1(nu, x) * mp.exp(-1j * chi) * mp.sqrt(mp.pi * x / 2)
    return h.real, h.imag


def large(x0, x1):
    """Pieces on x in [x0, x1] (x1 = inf allowed) in u = (x0/x)^2, t = affine map of u."""
    u1 = mp.mpf(1)
    u0 = mp.mpf(0) if x1 == mp.inf else (x0 / x1) ** 2

    def x_of(t):
        u = u0 + (u1 - u0) * (t + 1) / 2
        return x0 / mp.sqrt(u)

    fs = [lambda t: pq(0, x_of(t))[0], lambda t: pq(0, x_of(t))[1] * x_of(t) / 8,
          lambda t: pq(1, x_of(t))[0], lambda t: pq(1, x_of(t))[1] * x_of(t) / 8]
    return [cheb(f) for f in fs], u0


PQ_BREAKS = [8, 10, 13, 18, 28, 60]   # x intervals [8,10), ..., [60, inf)
PQ_TERMS = 8


def cheb_to_monomial(c):
    """Monomial coefficients a_k of sum_j c_j T_j(t) (exact in mpmath)."""
    n = len(c)
    T = [[mp.mpf(1)] + [mp.mpf(0)] * (n - 1), [mp.mpf(0), mp.mpf(1)] + [mp.mpf(0)] * (n - 2)]
    for j in range(2, n):
        nxt = [mp.mpf(0)] * n
        for k in range(n):
            if k + 1 < n:
                nxt[k + 1] += 2 * T[j - 1][k]
            nxt[k] -= T[j - 2][k]
        T.append(nxt)
    a = [mp.mpf(0)] * n
    for j in range(n):
        for k in range(n):
            a[k] += c[j] * T[j][k]
    return a


def pq_table():
    """Horner tables for P0, q0, P1, q1 (Q = (8/x) q) on each x interval, in the
    variable t = (u - uc)/uh of u = (8/x)^2 mapped to [-1, 1]."""
    rows, ucs, uhs = [], [], []
    bounds = PQ_BREAKS + [mp.inf]
    for x0, x1 in zip(bounds[:-1], bounds[1:]):
        u_hi = (mp.mpf(8) / x0) ** 2
        u_lo = mp.mpf(0) if x1 == mp.inf else (mp.mpf(8) / x1) ** 2
        uc, uh = (u_hi + u_lo) / 2, (u_hi - u_lo) / 2

        def x_of(t, uc=uc, uh=uh):
            return 8 / mp.sqrt(uc + uh * t)

        fs = [lambda t: pq(0, x_of(t))[0], lambda t: pq(0, x_of(t))[1] * x_of(t) / 8,
              lambda t: pq(1, x_of(t))[0], lambda t: pq(1, x_of(t))[1] * x_of(t) / 8]
        for f in fs:
            c = cheb(f)
            if len(c) > PQ_TERMS:
                raise SystemExit(f"interval [{x0},{x1}) needs {len(c)} terms")
            c = c + [mp.mpf(0)] * (PQ_TERMS - len(c))
            rows.append(cheb_to_monomial(c))
        ucs.append(uc)
        uhs.append(uh)
    return rows, ucs, uhs


# Double-float evaluation (mixed-precision paths) writes each function as its
# first two Hankel terms, exact in binary32, plus a remainder u^2 G(u):
#   P0 = 1 - 9u/8192 + u^2 G0,   Q0 = (8/x) (-1/64 + 75u/524288 + u^2 G1),
#   P1 = 1 + 15u/8192 + u^2 G2,  Q1 = (8/x) (3/64 - 105u/524288 + u^2 G3),
# u = (8/x)^2 (A&S 9.2.9-9.2.10 with mu = 4 nu^2).  |u^2 G| <= 1e-4 on x >= 8;
# the constant term of each G piece is kept as a double-float pair and the
# rest (|.| <= 1e-6) in binary32, which leaves ~1e-14 absolute error.
LEAD = [(mp.mpf(1), mp.mpf(-9) / 8192), (mp.mpf(-1) / 64, mp.mpf(75) / 524288),
        (mp.mpf(1), mp.mpf(15) / 8192), (mp.mpf(3) / 64, mp.mpf(-105) / 524288)]
G_TERMS = 8   # table stride (two float4 per polynomial)
G_EVAL = 6    # nonzero terms the device sums


def g_table():
    """Horner tables (binary32) of G0..G3 per x interval, variable t as in pq_table."""
    rows = []
    bounds = PQ_BREAKS + [mp.inf]
    for x0, x1 in zip(bounds[:-1], bounds[1:]):
        u_hi = (mp.mpf(8) / x0) ** 2
        u_lo = mp.mpf(0) if x1 == mp.inf else (mp.mpf(8) / x1) ** 2
        uc, uh = (u_hi + u_lo) / 2, (u_hi - u_lo) / 2

        def u_of(t, uc=uc, uh=uh):
            return uc + uh * t

        def g(t, k, uc=uc, uh=uh):
            u = u_of(t)
            if u == 0:
                u = mp.mpf("1e-30")
            x = 8 / mp.sqrt(u)
            v = pq(k // 2, x)[k % 2]
            if k % 2:
                v = v * x / 8
            c0, c1 = LEAD[k]
            return (v - c0 - c1 * u) / (u * u)

        for k in range(4):
            c = cheb(lambda t, k=k: g(t, k))
            # binary32 needs ~1e-8 relative: drop the tail below that
            scale = max(abs(v) for v in c)
            c = [v for v in c]
            while len(c) > 1 and abs(c[-1]) < mp.mpf("1e-9") * scale:
                c.pop()
            if len(c) > G_EVAL:   # the device evaluates c0 .. c5 (g_poly in dfloat.cuh)
                raise SystemExit(f"G{k} on [{x0},{x1}) needs {len(c)} terms")
            c = c + [mp.mpf(0)] * (G_TERMS - len(c))
            rows.append(cheb_to_monomial(c))
    return rows


def emit_f(name, c):
    body = ",\n    ".join(repr(float(mp.mpf(v))) + "f" for v in c)
    return f"static __device__ __constant__ float {name}[{len(c)}] = {{\n    {body}}};\n"


def df_consts(name, vals):
    """Double-float (hi, lo) pairs of the given numbers."""
    import struct
    out = []
    for v in vals:
        hi = struct.unpack("f", struct.pack("f", float(v)))[0]
        lo = struct.unpack("f", struct.pack("f", float(v - mp.mpf(hi))))[0]
        out += [hi, lo]
    body = ",\n    ".join(repr(x) + "f" for x in out)
    return f"static __device__ __constant__ float {name}[{len(out)}] = {{\n    {body}}};\n"


def emit(name, c):
    body = ",\n    ".join(mp.nstr(v, 20, min_fixed=-1, max_fixed=-1) for v in c)
    return f"constexpr int {name}_N = {len(c)};\nstatic __device__ __constant__ double {name}[{len(c)}] = {{\n    {body}}};\n"


def main():
    out = ["// Generated by gen_bessel_cheb.py (Chebyshev interpolation with mpmath);",
           "// do not edit.  See that script and bessel.cuh for the definitions.",
           "#pragma once", ""]
    for name, f in (("kA0", a0), ("kA1", a1), ("kA2", a2), ("kA3", a3)):
        out.append(emit(name, cheb(f)))
    (b_lo, u0_lo) = large(mp.mpf(8), mp.mpf(20))
    (b_hi, u0_hi) = large(mp.mpf(20), mp.inf)
    out.append(f"constexpr double kBLoU0 = {mp.nstr(u0_lo, 20)};   // (8/20)^2")
    for k, c in enumerate(b_lo):
        out.append(emit(f"kBLo{k}", c))
    for k, c in enumerate(b_hi):
        out.append(emit(f"kBHi{k}", c))
    rows, ucs, uhs = pq_table()
    ni = len(ucs)
    out.append(f"constexpr int kPQ_NI = {ni};          // x intervals {PQ_BREAKS} .. inf")
    out.append(f"constexpr int kPQ_TERMS = {PQ_TERMS};")
    out.append("// Horner coefficients [interval][P0, q0, P1, q1][power of t], t = (u - uc)/uh, u = (8/x)^2")
    flat = [v for r in rows for v in r]
    out.append(emit("kPQ", flat))
    out.append(emit("kPQ_UC", ucs))
    out.append(emit("kPQ_UH", uhs))
    out.append("// binary32 remainder polynomials G0..G3 [interval][function][power of t] (double-float path)")
    out.append(f"constexpr int kG_TERMS = {G_TERMS};")
    g_rows = g_table()
    out.append(emit_f("kG", [v for r in g_rows for v in r]))
    out.append("// constant terms of G0..G3 as double-float pairs [interval][function][hi, lo]")
    out.append(df_consts("kG0DF", [r[0] for r in g_rows]))
    out.append(emit_f("kPQ_UCf", ucs))
    out.append(emit_f("kPQ_IUHf", [1 / v for v in uhs]))
    out.append("// (-1)^k / (2k+1)! and (-1)^k / (2k)! as double-float pairs, k = 0..8 (sine and cosine series)")
    out.append(df_consts("kSinDF", [(-1) ** k / mp.factorial(2 * k + 1) for k in range(9)]))
    out.append(df_consts("kCosDF", [(-1) ** k / mp.factorial(2 * k) for k in range(9)]))
    out.append("// A0..A3 (x < 8) as double-float pairs [hi, lo] for the double-float path")
    for name, f in (("kA0DF", a0), ("kA1DF", a1), ("kA2DF", a2), ("kA3DF", a3)):
        out.append(df_consts(name, cheb(f)))
    out.append("// 1 / (2k + 1), k = 0..10 (ln m = 2 s sum_k s^2k / (2k + 1), s = (m - 1)/(m + 1)),")
    out.append("// ln 2, 2 / pi and ln(1/2) as double-float pairs")
    out.append(df_consts("kAtanhDF", [mp.mpf(1) / (2 * k + 1) for k in range(11)]))
    out.append(df_consts("kLogConstDF", [mp.log(2), 2 / mp.pi, -mp.log(2)]))
    # Cody-Waite split of pi/2: C1 with 12 significant bits (k C1 exact in
    # binary32 for k < 2^12), C2 and C3 the next binary32 pieces
    c1 = mp.floor(mp.pi / 2 * 2 ** 11 + mp.mpf(1) / 2) / 2 ** 11
    import struct
    f32 = lambda v: mp.mpf(struct.unpack("f", struct.pack("f", float(v)))[0])
    c2 = f32(mp.pi / 2 - c1)
    c3 = f32(mp.pi / 2 - c1 - c2)
    out.append("// pi/2 = C1 + C2 + C3 (Cody-Waite, C1 with 12 significant bits) and pi/4 as a double-float pair")
    out.append(emit_f("kPio2CW", [c1, c2, c3]))
    out.append(df_consts("kPio4DF", [mp.pi / 4]))
    print("\n".join(out))


if __name__ == "__main__":
    main()
