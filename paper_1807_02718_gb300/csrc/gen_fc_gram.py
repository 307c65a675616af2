"""Generates fc_gram_table.h: the FC(Gram) continuation table of the
low-frequency-split synthesis (k_sing.cu).

FC(Gram) Fourier continuation (Sec. 4.1, Remark Fourier-FC: a smooth,
non-periodic F on [a, b] is given a Fourier series of a period P > b - a).
The paper cites the method without tables; the construction used here:

* d = 6 matching points, C = 31 continuation points, a zero interval of
  Z = 12 points beyond them; functions of the grid coordinate u (unit spacing);
* Gram basis q_0..q_{d-1}: orthonormal for sum_{i<d} f(i) g(i), from 1, u, u^2, ...;
* blend-to-zero function of q_k: the trigonometric polynomial of degree 24
  and period 96 = 2 (d - 1 + C + Z) closest in least squares to q_k on the
  points i/10 of [0, d-1] and to 0 on the points d + C + i/10 of
  [d + C, d + C + Z - 1] (the least-squares matrix has full column rank);
* table A[j][k] = that function at u = d + j (j < C); Q[i][k] = q_k(i).

Solved here through the normal equations by Cholesky factorisation in
150-digit arithmetic (mpmath), rounded to binary64.

    python gen_fc_gram.py      # rewrites fc_gram_table.h beside this file
"""
import os

import mpmath as mp

D, C, Z, K, OS = 6, 31, 12, 24, 10
PERIOD = 2 * (D - 1 + C + Z)


def main():
    mp.mp.dps = 150
    pts = [mp.mpf(i) for i in range(D)]
    # Gram basis by modified Gram-Schmidt, kept as values and as monomial coefficients
    vals, mono = [], []
    for k in range(D):
        v = [p ** k for p in pts]
        c = [mp.mpf(0)] * D
        c[k] = mp.mpf(1)
        for qv, qc in zip(vals, mono):
            r = mp.fsum(a * b for a, b in zip(qv, v))
            v = [a - r * b for a, b in zip(v, qv)]
            c = [a - r * b for a, b in zip(c, qc)]
        s = mp.sqrt(mp.fsum(a * a for a in v))
        vals.append([a / s for a in v])
        mono.append([a / s for a in c])

    def basis(u):
        out = [mp.mpf(1)]
        for l in range(1, K + 1):
            th = 2 * mp.pi * l * u / PERIOD
            out.append(mp.cos(th))
            out.append(mp.sin(th))
        return out

    match = [mp.mpf(i) / OS for i in range((D - 1) * OS + 1)]
    zero = [D + C + mp.mpf(i) / OS for i in range((Z - 1) * OS + 1)]
    rows = [basis(u) for u in match + zero]
    nb = len(rows[0])
    G = mp.matrix(nb, nb)
    for r in rows:
        for i in range(nb):
            for j in range(nb):
                G[i, j] += r[i] * r[j]
    L = mp.cholesky(G)
    table = []
    for k in range(D):
        rhs = mp.matrix(nb, 1)
        for u, r in zip(match, rows):
            fu = mp.fsum(mono[k][i] * u ** i for i in range(D))
            for i in range(nb):
                rhs[i] += r[i] * fu
        y = mp.lu_solve(L, rhs)          # forward substitution (lower triangular)
        x = mp.lu_solve(L.T, y)          # back substitution
        table.append([mp.fsum(b * xx for b, xx in zip(basis(mp.mpf(D + j)), x)) for j in range(C)])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fc_gram_table.h")
    with open(out, "w") as f:
        f.write("// Generated by gen_fc_gram.py: FC(Gram) continuation table (d = %d, C = %d).\n" % (D, C))
        f.write("// kFcA[j][k]: blend-to-zero function of Gram polynomial k at continuation point j;\n")
        f.write("// kFcQ[i][k]: Gram polynomial k at matching point i.  Include from one translation unit.\n#pragma once\n\n")
        f.write("namespace fh {\nconstexpr int kFcD = %d, kFcC = %d;\n" % (D, C))
        f.write("__constant__ const double kFcA[kFcC][kFcD] = {\n")
        for j in range(C):
            f.write("    {" + ", ".join(mp.nstr(table[k][j], 17, min_fixed=0, max_fixed=0) for k in range(D)) + "},\n")
        f.write("};\n__constant__ const double kFcQ[kFcD][kFcD] = {\n")
        for i in range(D):
            f.write("    {" + ", ".join(mp.nstr(vals[k][i], 17, min_fixed=0, max_fixed=0) for k in range(D)) + "},\n")
        f.write("};\n}  // namespace fh\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
