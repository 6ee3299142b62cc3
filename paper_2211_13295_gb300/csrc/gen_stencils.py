"""Generate csrc/stencils.inc: WENO candidate-stencil coefficients, exact rationals.

For order r = N+1 the candidate k (k = 0..N) covers the zones k-N..k and is the
degree-N polynomial, in the scaled Legendre basis of the zone [-1/2,1/2]
(1, xi, xi^2 - 1/12, xi^3 - 3 xi/20), whose zone averages equal the data.  The
average of mode a over the zone at offset s is s, s^2, s^3 + s/10 (a = 1, 2, 3)
and 0 over the zone itself, so the modal coefficients solve an N x N linear
system in the differences u(s) - u(0); this script solves it in exact rational
arithmetic and writes each coefficient as a row of weights on the differences.
Run: python gen_stencils.py > stencils.inc
(the literal T(p.0 / q.0) is the rational p/q rounded once in the working precision T)
"""
from fractions import Fraction as Fr


def zone_avg(a, s):
    s = Fr(s)
    return [None, s, s * s, s ** 3 + s / 10][a]


def solve(A, b):
    n = len(A)
    M = [row[:] + [bb] for row, bb in zip(A, b)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[r][n] / M[r][r] for r in range(n)]


def stencils(N):
    """coef[k][a-1][j]: weight of d_j = u(j) - u(0) (j = -N..N) in mode a of candidate k"""
    out = []
    for k in range(N + 1):
        offs = [s for s in range(k - N, k + 1) if s != 0]
        A = [[zone_avg(a, s) for a in range(1, N + 1)] for s in offs]
        rows = []
        for a in range(N):
            w = {}
            for j, s in enumerate(offs):
                e = [Fr(int(i == j)) for i in range(N)]
                x = solve(A, e)
                w[s] = x[a]
            rows.append([w.get(s, Fr(0)) for s in range(-N, N + 1)])
        out.append(rows)
    return out


def term(v, j):
    """one term weight*d[j] with an exact rational literal"""
    lit = f"{v.numerator}.0" if v.denominator == 1 else f"({v.numerator}.0 / {v.denominator}.0)"
    return f"T({lit}) * d[{j}]"


def main():
    print("// generated by gen_stencils.py: exact rational WENO candidate stencils.")
    print("// d[j] = u(j-N) - u(0) for j = 0..2N; c[k][a] = mode a+1 of candidate k.")
    print("// Only the nonzero weights appear, so no FMA is spent on a zero.  Host-callable")
    print("// too: the library folds them with the linear weights into one stencil.")
    for N in (2, 3):
        S = stencils(N)
        print("template <typename T>")
        print(f"__host__ __device__ __forceinline__ void weno_candidates_n{N}(const T* d, T c[{N + 1}][{N}]) {{")
        for k in range(N + 1):
            for a in range(N):
                terms = [term(v, j) for j, v in enumerate(S[k][a]) if v != 0]
                print(f"  c[{k}][{a}] = " + " + ".join(terms) + ";")
        print("}")


if __name__ == "__main__":
    main()
