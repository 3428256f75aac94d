"""Optimal decoding of a general stabilizer code by brute force over Paulis (Sec. 2.1-2.3).

A Pauli (mod phase) is a pair (u, v) of bit strings (Sec. 2.1): u_i = 1 for X or Y on
qubit i, v_i = 1 for Z or Y.  Two Paulis anticommute iff u.v' + v.u' = 1 (mod 2), the
symplectic form.  The syndrome of an error e is its symplectic product with each
stabilizer generator; its logical class l = x^a z^b has a = <e, z_bar> and b = <e, x_bar>
(Sec. 2.2: lambda_i = <q, z_i>, mu_i = <q, x_i>).  The coset probability of class (a, b)
given syndrome m is the sum of P_E(e) over all e with that syndrome and class, which is
the sum over the stabilizer coset in Eq. (optimal_decoder).
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def pauli_to_uv(s: str):
    u = np.array([c in "XY" for c in s], dtype=np.int64)
    v = np.array([c in "ZY" for c in s], dtype=np.int64)
    return u, v


def coset_table(stabs, x_bar: str, z_bar: str, P_qubit):
    """Table T[m, a, b] = probability that the error has syndrome m (bit i = generator i)
    and logical class x^a z^b.  P_qubit[i] = (P(I), P(X), P(Y), P(Z)) for qubit i."""
    n = len(stabs[0])
    codes = np.arange(4 ** n, dtype=np.int64)
    digits = (codes[:, None] >> (2 * np.arange(n, dtype=np.int64))[None, :]) & 3   # 0 I,1 X,2 Y,3 Z
    u = ((digits == 1) | (digits == 2)).astype(np.int64)
    v = ((digits == 2) | (digits == 3)).astype(np.int64)

    def symp_with(s):
        su, sv = pauli_to_uv(s)
        return (u @ sv + v @ su) % 2

    m = np.zeros(len(codes), dtype=np.int64)
    for k, s in enumerate(stabs):
        m |= symp_with(s) << k
    a = symp_with(z_bar)
    b = symp_with(x_bar)
    P = np.asarray(P_qubit, dtype=np.float64)                      # [n, 4]
    prob = np.prod(P[np.arange(n)[None, :], digits], axis=1)
    T = np.zeros((1 << len(stabs), 2, 2))
    np.add.at(T, (m, a, b), prob)
    return T
