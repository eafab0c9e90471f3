"""Brute-force pin of the oracle: the same definitions evaluated in 40-digit arithmetic
(mpmath) on small inputs.  Catches any FP64 instability in the oracle's route through
Eqs. 1, A1, 23 and 8, not only formula mistakes."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

import oracle as O
from paper_1303_4446_gb300 import workload as w

C = O.C_LIGHT


def _x2c_mp(m, c_val):
    two_c = "Wx" in m
    S, T, V, W = O.spinor_inputs(m)
    n = S.shape[0]
    c = mp.mpf(c_val)
    M = lambda A: mp.matrix(np.asarray(A).tolist())
    S, T, V, W = M(S), M(T), M(V), M(W)
    D = mp.zeros(2 * n, 2 * n)
    Mm = mp.zeros(2 * n, 2 * n)
    for i in range(n):
        for j in range(n):
            D[i, j] = V[i, j]
            D[i, n + j] = T[i, j]
            D[n + i, j] = T[i, j]
            D[n + i, n + j] = W[i, j] / (4 * c * c) - T[i, j]
            Mm[i, j] = S[i, j]
            Mm[n + i, n + j] = T[i, j] / (2 * c * c)
    L = mp.cholesky(Mm)
    Li = L**-1
    A = Li * D * Li.H
    E, Q = mp.eighe(A) if two_c else mp.eigsy(A)
    idx = sorted(range(2 * n), key=lambda i: mp.re(E[i]))
    Cv = Li.H * Q
    CL, CS = mp.zeros(n, n), mp.zeros(n, n)
    for jj, j in enumerate(idx[n:]):
        for i in range(n):
            CL[i, jj] = Cv[i, j]
            CS[i, jj] = Cv[n + i, j]
    X = CS * CL**-1
    St = S + X.H * T * X / (2 * c * c)

    def hpow(B, p):
        e, Qm = mp.eighe(B) if two_c else mp.eigsy(B)
        return Qm * mp.diag([mp.re(x) ** p for x in e]) * Qm.H

    Sm, Sp = hpow(S, -0.5), hpow(S, 0.5)
    UL = Sm * hpow(Sm * St * Sm, -0.5) * Sp
    US = X * UL
    Wp = W / (4 * c * c) - T
    h = UL.H * V * UL + UL.H * T * US + US.H * T * UL + US.H * Wp * US
    cv = (lambda x: complex(x)) if two_c else (lambda x: float(x))
    to = lambda B: np.array([[cv(B[i, j]) for j in range(B.cols)] for i in range(B.rows)])
    return to(h), to(UL), to(US)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("two_c", [False, True])
def test_oracle_matches_40_digit_arithmetic(two_c):
    mp.mp.dps = 40
    if two_c:
        # 10 functions keep the complex 40-digit eigensolve quick
        sub = np.r_[0:30:3]
        m = {k: v[np.ix_(sub, sub)] for k, v in w.atomic_inputs(47.0, "s30", True).items()}
    else:
        m = w.atomic_inputs(47.0, "s30", False)
    h, UL, US = _x2c_mp(m, C)
    r = O.x2c_full(m)
    assert _rel(r["h"], h) < 1e-13
    assert _rel(r["UL"], UL) < 1e-11
    assert _rel(r["US"], US) < 1e-11
