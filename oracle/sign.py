"""Composite minimax approximations of sign(x) (Section 5.4.2, Table 2: the
paper composes low-degree minimax polynomials after LLNK20 but prints no
coefficients).

TEST INFRASTRUCTURE (see oracle/__init__.py).

A stage is the odd polynomial p(x) = sum_{k<n} c_k x^(2k+1) of degree 2n-1
that minimises max |p(x) - 1| over x in [a, b] (and, being odd, |p(x) + 1| on
[-b, -a]), found by the Remez exchange: solve p(x_i) + (-1)^i E = 1 on n + 1
reference points, move the points to the alternating extrema of the error,
repeat until the extrema are level.  Stages compose: stage s maps [a_s, b_s]
into [1 - E_s, 1 + E_s], which is the next stage's interval (iterated
minimax; the first interval is [2^-alpha, 1]).  This is a reading: LLNK20's
jointly optimised composition is not printed, so Table 2's second row
(alpha 16, beta 20 with five degree-15 stages) needs a sixth stage here.
"""
from __future__ import annotations

import math

import mpmath as mp


def remez_odd(n_terms: int, a: float, b: float, iters: int = 100, grid: int = 4000, dps: int = 60):
    """Minimax odd polynomial with n_terms coefficients for 1 on [a, b].
    Returns (coefficients of x, x^3, ..., error E) with max |p - 1| = E."""
    with mp.workdps(dps):
        a, b = mp.mpf(a), mp.mpf(b)
        m = n_terms + 1
        xs = [(a + b) / 2 + (b - a) / 2 * mp.cos(mp.pi * (m - 1 - i) / (m - 1)) for i in range(m)]
        # the error is steepest near a: a grid quadratic in the distance from a
        pts = [a + (b - a) * (mp.mpf(j) / grid) ** 2 for j in range(grid + 1)]
        best = None
        for _ in range(iters):
            A = mp.matrix(m, m)
            rhs = mp.matrix(m, 1)
            for i, x in enumerate(xs):
                for k in range(n_terms):
                    A[i, k] = x ** (2 * k + 1)
                A[i, n_terms] = (-1) ** i
                rhs[i] = 1
            sol = mp.lu_solve(A, rhs)
            c = [sol[k] for k in range(n_terms)]
            lev = abs(sol[n_terms])
            e_of = lambda x: sum(ck * x ** (2 * k + 1) for k, ck in enumerate(c)) - 1
            err = [e_of(x) for x in pts]
            ext = [0] + [j for j in range(1, grid) if (err[j] - err[j - 1]) * (err[j + 1] - err[j]) <= 0] + [grid]
            # each interior extremum refined by a golden-section search of |e| between its grid neighbours
            cand = []
            for j in ext:
                if 0 < j < grid:
                    lo_, hi_ = pts[j - 1], pts[j + 1]
                    g = (mp.sqrt(5) - 1) / 2
                    for _ in range(60):
                        x1, x2 = hi_ - g * (hi_ - lo_), lo_ + g * (hi_ - lo_)
                        if abs(e_of(x1)) > abs(e_of(x2)):
                            hi_ = x2
                        else:
                            lo_ = x1
                    x = (lo_ + hi_) / 2
                    cand.append((x, e_of(x)))
                else:
                    cand.append((pts[j], err[j]))
            seq = []
            for x, e in cand:
                if seq and mp.sign(e) == mp.sign(seq[-1][1]):
                    if abs(e) > abs(seq[-1][1]):
                        seq[-1] = (x, e)
                else:
                    seq.append((x, e))
            while len(seq) > m:
                if abs(seq[0][1]) < abs(seq[-1][1]):
                    seq.pop(0)
                else:
                    seq.pop()
            emax = max(abs(e) for _, e in cand)
            best = ([float(ck) for ck in c], float(emax))
            if len(seq) < m or emax - lev <= mp.mpf(10) ** -25 * max(1, lev):
                break
            xs = [x for x, _ in seq]
        return best


def composite_minimax(alpha: float, degrees) -> tuple:
    """Iterated minimax stages for sign on [-1, -2^-alpha] u [2^-alpha, 1].
    Returns (list of per-stage coefficient lists, final error E): the composite
    is within E of sign(x) there, so step = (p + 1)/2 is within E/2 (beta =
    -log2(E/2) in Table 2's terms)."""
    lo, hi = 2.0 ** -alpha, 1.0
    stages, err = [], 1.0
    for d in degrees:
        if d % 2 == 0:
            raise ValueError("sign stages are odd polynomials")
        c, err = remez_odd((d + 1) // 2, lo, hi)
        stages.append(c)
        lo, hi = 1.0 - err, 1.0 + err
    return stages, err


def beta(err: float) -> float:
    return -math.log2(err / 2.0)
