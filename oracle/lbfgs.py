"""Lower-level solver: L-BFGS with backtracking (Section 5.1: history 10, backtracking), FP64.

Two-loop recursion with initial scaling gamma = s^T y / y^T y of the newest
pair (gamma = 1 before any pair exists).  Armijo backtracking on Phi with
c1 = 1e-4 and step halving, first trial step 1; `slack` > 0 adds slack * |Phi(x)|
to the sufficient-decrease bound (0, the plain rule, is the default).  A pair is stored only when
s^T y > 1e-12 ||s|| ||y||.  Stops when ||grad Phi|| <= gtol.
"""
from __future__ import annotations

import numpy as np


def lbfgs(fun, grad, x0, gtol, m=10, maxit=10000, c1=1e-4, max_backtrack=60, slack=0.0):
    x = x0.copy()
    f = fun(x)
    g = grad(x)
    S, Y = [], []
    it = 0
    evals = 1
    while np.linalg.norm(g) > gtol and it < maxit:
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(S), reversed(Y)):
            a = float(s @ q) / float(y @ s)
            alphas.append(a)
            q -= a * y
        gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) if S else 1.0
        d = gamma * q
        for (s, y), a in zip(zip(S, Y), reversed(alphas)):
            b = float(y @ d) / float(y @ s)
            d += (a - b) * s
        d = -d
        gd = float(g @ d)
        if gd >= 0:            # not a descent direction: restart from steepest descent
            S, Y = [], []
            d = -g
            gd = float(g @ d)
        t = 1.0
        for _ in range(max_backtrack):
            xn = x + t * d
            fn = fun(xn)
            evals += 1
            if fn <= f + c1 * t * gd + slack * abs(f):
                break
            t *= 0.5
        gn = grad(xn)
        s = xn - x
        y = gn - g
        if float(s @ y) > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, fn, gn
        it += 1
    return x, dict(iters=it, evals=evals, gnorm=float(np.linalg.norm(g)), f=f)
