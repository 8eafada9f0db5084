#!/usr/bin/env python3
"""Writes pred_pattern.h: which entries of the predictor matrices are exactly
zero, per (d, M).

P_e[k][l] = int_0^{tau_k} d theta_l / d xi_e (xi_k, s) ds (the closed form of
the Galerkin predictor, unknown node k, any node l), with theta_l the Lagrange
polynomial of space-time node l on the principal lattice of the
(d+1)-simplex.  Computed here in exact rational arithmetic, independently of
the floating-point tables the library builds at setup; the kernels skip the
terms this marks as zero.  Node order: time level outermost, then the
spatial lattice with the last coordinate outermost (as in refelem.cpp).

Run: python gen_pred_pattern.py > pred_pattern.h
"""
from fractions import Fraction as Fr
from math import comb

CONFIGS = [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3), (3, 4)]


def st_nodes(d, M):
    out = []
    for t in range(M + 1):
        K = M - t
        if d == 2:
            for j in range(K + 1):
                for i in range(K + 1 - j):
                    out.append((i, j, t))
        else:
            for k in range(K + 1):
                for j in range(K + 1 - k):
                    for i in range(K + 1 - j - k):
                        out.append((i, j, k, t))
    return out


# univariate polynomials in s as lists of Fractions (coefficient of s^p)
def pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def entry(d, M, node_k, node_l, e):
    """int_0^{tau_k} d theta_l / d xi_e at xi = xi_k, as an exact Fraction."""
    xi = [Fr(c, M) for c in node_k[:d]]
    tau_k = Fr(node_k[d], M)
    alpha = [M - sum(node_l)] + list(node_l)  # lambda_0, lambda_1..d (xi), lambda_{d+1} (tau)
    # barycentric coordinates along the line (xi_k, s): affine in s
    lam = [[1 - sum(xi), Fr(-1)]] + [[x, Fr(0)] for x in xi] + [[Fr(0), Fr(1)]]
    dlam = [-1] + [1 if a == e else 0 for a in range(d)] + [0]  # d lambda_c / d xi_e
    factors = []  # (polynomial in s, derivative wrt xi_e)
    for c, ac in enumerate(alpha):
        for j in range(ac):
            poly = [(M * lam[c][0] - j) / (j + 1), M * lam[c][1] / (j + 1)]
            factors.append((poly, Fr(M * dlam[c], j + 1)))
    deriv = [Fr(0)]
    for q, (_, dq) in enumerate(factors):
        if dq == 0:
            continue
        term = [dq]
        for r, (pr, _) in enumerate(factors):
            if r != q:
                term = pmul(term, pr)
        deriv = padd(deriv, term)
    return sum(c * tau_k ** (p + 1) / (p + 1) for p, c in enumerate(deriv))


def main():
    print("// Generated by gen_pred_pattern.py: nonzero pattern of the predictor")
    print("// matrices P_e[k][l] (exact rational arithmetic).  Do not edit.")
    print("#pragma once")
    print("namespace cw {")
    print("template <int D, int M>")
    print("struct PredPattern;")
    for d, M in CONFIGS:
        nodes = st_nodes(d, M)
        L = len(nodes)
        L0 = comb(M + d, d)
        L1 = L - L0
        bits = []
        for e in range(d):
            for k in range(L1):
                for l in range(L):
                    bits.append("1" if entry(d, M, nodes[L0 + k], nodes[l], e) != 0 else "0")
        nz = bits.count("1")
        print(f"template <>\nstruct PredPattern<{d}, {M}> {{  // {nz} of {d * L1 * L} nonzero")
        print(f"  // entry (e, k, l) at ((e * {L1}) + k) * {L} + l; constant indices fold at compile time")
        print("  __host__ __device__ static constexpr bool nz(int e, int k, int l) {")
        chunks = ["".join(bits[i:i + 100]) for i in range(0, len(bits), 100)]
        lit = "\n".join(f'        "{c}"' for c in chunks)
        print(f"    return (\n{lit})[(e * {L1} + k) * {L} + l] == '1';")
        print("  }")
        print("};")
    print("}  // namespace cw")


if __name__ == "__main__":
    main()
