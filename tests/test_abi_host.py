"""Host-side checks of the C ABI: the library loads, exports every symbol of include/td.h,
and rejects invalid problems on the host (before any device work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from td_inputs import point_sector_3d, rotated_phenomenological

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_10722_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    src = open(os.path.join(ROOT, "include", "td.h")).read()
    names = set(re.findall(r"\b(td_[a-z_]+)\s*\(", src))
    assert names, "no declarations found"
    from paper_2310_10722_gb300 import _lib
    assert names == set(_lib.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_default_options(lib):
    from paper_2310_10722_gb300 import _lib
    o = _lib.td_options()
    lib.td_default_options(C.byref(o))
    assert (o.chi, o.chi_mps, o.precision) == (8, 16, 0)
    assert o.svd_cutoff == 1e-12 and o.mem_budget == 16 << 30


def _build(lib, dem, **kw):
    from paper_2310_10722_gb300 import _lib
    hip, hix = dem.H_csr()
    lip, lix = dem.L_csr()
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (hip, hix, lip, lix)]
    p = np.ascontiguousarray(kw.pop("p", dem.p), dtype=np.float64)
    xyt = np.ascontiguousarray(kw.pop("xyt", dem.det_xyt), dtype=np.int32).reshape(-1)
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    d = _lib.td_dem(len(hip) - 1, dem.n_mech, len(lip) - 1, P(arrs[0], C.c_int32), P(arrs[1], C.c_int32),
                    P(arrs[2], C.c_int32), P(arrs[3], C.c_int32), P(p, C.c_double))
    lay = _lib.td_layout(P(xyt, C.c_int32))
    o = _lib.td_options()
    lib.td_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p()
    st = lib.td_build_network(C.byref(d), C.byref(lay), C.byref(o), C.byref(h))
    if st == 0:
        lib.td_free_network(h)
    return st, lib.td_last_error().decode()


def test_rejects_rate_out_of_range(lib):
    dem = point_sector_3d(3, 0.05)
    p = dem.p.copy(); p[3] = 1.5
    st, msg = _build(lib, dem, p=p)
    assert st == 1 and "probability" in msg


def test_rejects_nonlocal_mechanism(lib):
    dem = point_sector_3d(3, 0.05)
    dem.mech_dets[5] = (0, 8)            # (0,0,0) and (2,2,0): not grid neighbours
    st, msg = _build(lib, dem)
    assert st == 2, msg


def test_rejects_two_observables(lib):
    dem = point_sector_3d(3, 0.05)
    dem.n_obs = 2
    dem.mech_obs[0] = (0, 1)
    st, msg = _build(lib, dem)
    assert st == 7, msg


def test_rejects_missing_detector(lib):
    dem = rotated_phenomenological(3, 1)
    xyt = dem.det_xyt.copy()
    xyt[0] = (7, 7, 0)                     # moves a detector off its site
    st, msg = _build(lib, dem, xyt=xyt)
    assert st in (2, 7), msg


def test_rejects_bad_chi(lib):
    dem = point_sector_3d(3, 0.05)
    assert _build(lib, dem, chi=0)[0] == 1
    assert _build(lib, dem, chi=64)[0] == 7


def test_null_network_calls(lib):
    assert lib.td_coset_logprob(None, None, 0, None, None) == 1
    assert lib.td_grad_logprob(None, None, 0, None, None, None, None) == 1
    lib.td_free_network(None)


def test_budget_below_one_shot_is_out_of_memory(lib):
    """A device-memory budget too small for one shot's workspace is refused with TD_ERR_OOM
    before any allocation (the host-side allocation failure of the build)."""
    dem = point_sector_3d(3, 0.05)
    st, msg = _build(lib, dem, mem_budget=1024)
    assert st == 3 and "mem_budget" in msg, (st, msg)


def test_unknown_precision_and_check_without_network(lib):
    dem = point_sector_3d(3, 0.05)
    assert _build(lib, dem, precision=3)[0] == 1
    assert lib.td_network_check(None, None) == 1


def _build_gen(lib, gp, **kw):
    """td_build_gen_network on a td_inputs.GenProblem; keyword overrides of the arrays."""
    from paper_2310_10722_gb300 import _lib
    qg = np.ascontiguousarray(kw.pop("qubit_gens", [list(e) + [-1] * (2 - len(e)) for e in gp.edges]),
                              dtype=np.int32).reshape(-1)
    p = np.ascontiguousarray(kw.pop("p", gp.p), dtype=np.float64)
    xyt = np.ascontiguousarray(kw.pop("gen_xyt", gp.gen_xyt), dtype=np.int32).reshape(-1)
    hip, hix = gp.face_dem.H_csr()
    hip = np.ascontiguousarray(hip, dtype=np.int32)
    hix = np.ascontiguousarray(hix, dtype=np.int32)
    xb = np.ascontiguousarray(kw.pop("xbar", gp.xbar), dtype=np.int32)
    zb = np.ascontiguousarray(kw.pop("zbar", gp.zbar), dtype=np.int32)
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    g = _lib.td_gen(len(xyt) // 3, len(qg) // 2, len(hip) - 1, P(qg, C.c_int32), P(p, C.c_double),
                    P(xyt, C.c_int32), P(hip, C.c_int32), P(hix, C.c_int32), len(xb), P(xb, C.c_int32),
                    len(zb), P(zb, C.c_int32))
    o = _lib.td_options()
    lib.td_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p()
    st = lib.td_build_gen_network(C.byref(g), C.byref(o), C.byref(h))
    if st == 0:
        lib.td_free_network(h)
    return st, lib.td_last_error().decode()


def test_generator_network_validation(lib):
    from td_inputs import loop_sector_3d
    gp = loop_sector_3d(3, 0.1)
    # a valid problem gets past validation (then needs a device: OOM / CUDA without a GPU)
    st, _ = _build_gen(lib, gp)
    assert st in (0, 3, 4)
    st, msg = _build_gen(lib, gp, p=np.full(gp.n_qubits, 1.5))
    assert st == 1 and "rate" in msg
    # xbar with a syndrome: drop one of its qubits
    st, msg = _build_gen(lib, gp, xbar=list(gp.xbar)[1:])
    assert st == 1 and "xbar" in msg
    # zbar that anticommutes with a generator: drop its top qubit
    st, msg = _build_gen(lib, gp, zbar=list(gp.zbar)[:-1])
    assert st == 1 and "zbar" in msg
    # xbar and zbar commuting: take zbar = xbar's complement overlap even (empty zbar)
    st, msg = _build_gen(lib, gp, zbar=[])
    assert st == 1 and "odd" in msg
    # a generator that anticommutes with a check: reroute one edge to a far generator
    qg = [list(e) + [-1] * (2 - len(e)) for e in gp.edges]
    j = next(k for k, e in enumerate(gp.edges) if len(e) == 2)
    qg[j] = [qg[j][0], gp.n_gen - 1 if qg[j][0] != gp.n_gen - 1 else 0]
    st, msg = _build_gen(lib, gp, qubit_gens=qg)
    assert st in (1, 2) and msg
    # bad generator index
    qg = [list(e) + [-1] * (2 - len(e)) for e in gp.edges]
    qg[0] = [gp.n_gen, -1]
    st, msg = _build_gen(lib, gp, qubit_gens=qg)
    assert st == 1 and "range" in msg
    st, msg = _build_gen(lib, gp, chi=33)
    assert st == 7


def test_generator_network_geometry_rules(lib):
    from td_inputs import loop_sector_3d
    gp = loop_sector_3d(3, 0.1)
    # move one generator to a layer of its own: a site without a generator in some layer
    xyt = np.array(gp.gen_xyt).copy()
    xyt[0, 2] = 5
    st, msg = _build_gen(lib, gp, gen_xyt=xyt)
    assert st in (1, 7) and msg


def test_generator_calls_on_detector_network_rejected_without_network(lib):
    assert lib.td_gen_coset_logprob(None, None, 0, None, None) == 1
    assert lib.td_gen_decode(None, None, 0, None, None, None) == 1
