"""Writes the FC(Gram) continuation table used by the oracle (test
infrastructure; run once, output committed: fc_gram_d6_c31.json).

FC(Gram) Fourier continuation (Sec. 4.1, Remark Fourier-FC, citing Bruno &
Lyon and Amlani & Bruno; the paper gives no tables).  The reading taken:

* d = 6 matching points, C = 31 continuation points, Z = 12 zero points,
  trigonometric degree 24 with period 96 (= 2 (d - 1 + C + Z)) in units of
  the grid spacing, oversampling 10 on the matching and zero intervals
  (d = 6 keeps the table entries below 6e4, so that rounding of O(1e-16)
  stays below 1e-11 of the result; larger d raises the order but the table
  entries grow to 1e6 .. 3e7);
* Gram basis: the polynomials q_0..q_{d-1} orthonormal for the discrete
  inner product on the d points u = 0..d-1 (Gram-Schmidt of 1, u, u^2, ...);
* for each q_k, g_k is the least-squares trigonometric polynomial
  g(u) = a_0 + sum_{l=1}^{24} (a_l cos(2 pi l u/96) + b_l sin(2 pi l u/96))
  with g = q_k on the oversampled matching interval [0, d-1] and g = 0 on the
  oversampled zero interval [d + C, d + C + Z - 1]; the least-squares matrix
  has full rank (smallest singular value 2.2e-24 of the largest), so
  g_k is unique;
* the continuation table is A[j, k] = g_k(d + j), j = 0..C-1 (the values
  that blend the right end's polynomial to zero); Q[i, k] = q_k(i).

Computed in 100-digit arithmetic (mpmath Householder least squares) and
rounded to binary64.

    python oracle/gen_fc_gram.py
"""
import json
import os

import mpmath as mp

D, C, Z, K, OVERSAMPLE = 6, 31, 12, 24, 10
PERIOD = 2 * (D - 1 + C + Z)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fc_gram_d6_c31.json")


def gram_basis(d):
    """Orthonormal polynomials on u = 0..d-1: values Q[i][k] and monomial coefficients."""
    u = [mp.mpf(i) for i in range(d)]
    qs = []
    for k in range(d):
        v = [x ** k for x in u]
        for q in qs:
            r = mp.fsum(a * b for a, b in zip(q, v))
            v = [a - r * b for a, b in zip(v, q)]
        nrm = mp.sqrt(mp.fsum(a * a for a in v))
        qs.append([a / nrm for a in v])
    V = mp.matrix([[x ** k for k in range(d)] for x in u])
    coefs = [mp.lu_solve(V, mp.matrix(q)) for q in qs]
    return qs, coefs


def trig_row(u):
    row = [mp.mpf(1)]
    for l in range(1, K + 1):
        a = 2 * mp.pi * l * u / PERIOD
        row += [mp.cos(a), mp.sin(a)]
    return row


def main():
    mp.mp.dps = 100
    qs, coefs = gram_basis(D)
    um = [mp.mpf(i) / OVERSAMPLE for i in range((D - 1) * OVERSAMPLE + 1)]
    z0 = D + C
    uz = [z0 + mp.mpf(i) / OVERSAMPLE for i in range((Z - 1) * OVERSAMPLE + 1)]
    Amat = mp.matrix([trig_row(u) for u in um + uz])
    table = []
    for k in range(D):
        rhs = mp.matrix([mp.fsum(coefs[k][i] * u ** i for i in range(D)) for u in um] + [0] * len(uz))
        x, _ = mp.qr_solve(Amat, rhs)
        table.append([mp.fsum(a * b for a, b in zip(trig_row(mp.mpf(D + j)), x)) for j in range(C)])
    out = {"d": D, "C": C, "Z": Z, "K": K, "period": PERIOD, "oversample": OVERSAMPLE,
           "A": [[float(table[k][j]) for k in range(D)] for j in range(C)],
           "Q": [[float(qs[k][i]) for k in range(D)] for i in range(D)]}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
