"""Host-side check of the generator-network planner (td_gen_rows_host, no device): the rows the
decoding calls sweep -- the representative r of each syndrome on the greedy column basis of H,
and r + xbar -- its class and the syndrome check, in the network's column order, bit for bit
against the oracle's representative (oracle/gen.py) and an independent column map."""
import ctypes as C
import os

import numpy as np
import pytest

from oracle import gen
from td_inputs import loop_sector_3d, sample_shots


@pytest.fixture(scope="module")
def lib():
    from paper_2310_10722_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def _td_gen(gp):
    from paper_2310_10722_gb300 import _lib
    qg = np.ascontiguousarray([list(e) + [-1] * (2 - len(e)) for e in gp.edges], dtype=np.int32).reshape(-1)
    p = np.ascontiguousarray(gp.p, dtype=np.float64)
    xyt = np.ascontiguousarray(gp.gen_xyt, dtype=np.int32).reshape(-1)
    hip, hix = gp.face_dem.H_csr()
    hip = np.ascontiguousarray(hip, dtype=np.int32)
    hix = np.ascontiguousarray(hix, dtype=np.int32)
    xb = np.ascontiguousarray(gp.xbar, dtype=np.int32)
    zb = np.ascontiguousarray(gp.zbar, dtype=np.int32)
    keep = [qg, p, xyt, hip, hix, xb, zb]
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    g = _lib.td_gen(len(xyt) // 3, len(qg) // 2, len(hip) - 1, P(qg, C.c_int32), P(p, C.c_double),
                    P(xyt, C.c_int32), P(hip, C.c_int32), P(hix, C.c_int32), len(xb), P(xb, C.c_int32),
                    len(zb), P(zb, C.c_int32))
    return g, keep


def _expected_columns(gp):
    """Column of every qubit by the documented rule, from the oracle's layering."""
    plan = gen.GenPlan(gp)
    S, T = plan.S, plan.T
    col = {}
    for t in range(T):
        for s in range(S):
            col[plan.below[t][s]] = t * S + s
    for s in range(S):
        col[plan.above[s]] = T * S + s
    k = S * (T + 1)
    for j in range(gp.n_qubits):
        if j not in col:
            col[j] = k
            k += 1
    return np.array([col[j] for j in range(gp.n_qubits)])


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_rows_match_oracle_representative(lib, d):
    gp = loop_sector_3d(d, 0.2)
    syn, _ = sample_shots(gp.face_dem, 12, seed=40 + d)
    syn = syn.copy()
    syn[5] = 0
    syn[5, 0] = 1                                    # a lone plaquette: no error has it
    g, keep = _td_gen(gp)
    B, nq = syn.shape[0], gp.n_qubits
    rows = np.zeros((2 * B, nq), np.uint8)
    cls = np.zeros(B, np.int32)
    col = np.zeros(nq, np.int32)
    s = np.ascontiguousarray(syn, dtype=np.uint8)
    st = lib.td_gen_rows_host(C.byref(g), s.ctypes.data_as(C.c_void_p), B, rows.ctypes.data_as(C.c_void_p),
                              cls.ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p))
    assert st == 0, lib.td_last_error()
    assert np.array_equal(col, _expected_columns(gp))
    xb = np.zeros(nq, np.uint8)
    xb[list(gp.xbar)] = 1
    for b in range(B):
        r = gen.representative(gp, syn[b])
        if r is None:
            assert cls[b] == -1
            continue
        assert cls[b] == gen.class_of(gp, r)
        assert np.array_equal(rows[2 * b][col], r)
        assert np.array_equal(rows[2 * b + 1][col], r ^ xb)
    assert (cls == -1).sum() == 1


def test_rows_host_rejects_bad_problem(lib):
    gp = loop_sector_3d(3, 0.1)
    g, keep = _td_gen(gp)
    g.n_zbar = 0                                     # zbar empty: commutes with xbar
    rows = np.zeros((2, gp.n_qubits), np.uint8)
    cls = np.zeros(1, np.int32)
    syn = np.zeros((1, gp.face_dem.n_det), np.uint8)
    st = lib.td_gen_rows_host(C.byref(g), syn.ctypes.data_as(C.c_void_p), 1, rows.ctypes.data_as(C.c_void_p),
                              cls.ctypes.data_as(C.c_void_p), None)
    assert st == 1 and b"odd" in lib.td_last_error()
