"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/ddsg.h declares, and its host-side logic (argument and table
validation, regular grids of eq. 3.5, b coefficients of eq. 4.2) agrees with
the oracle. No compute call is made."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2202_06555_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            if not mt.group(0).lstrip().startswith(("typedef", "#", "return")):
                names.append(mt.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = G.load()
    names = _declared_functions()
    assert "hdmr_eval" in names and "hdmr_hierarchize" in names and len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly what the header declares
    assert set(names) <= set(G.SIGNATURES) | {"ddsg_version", "ddsg_last_error"}
    assert lib.ddsg_version().startswith(b"libddsg")


def test_create_validates_arguments():
    lib = G.load()
    h = C.c_void_p()
    z = np.zeros(3)
    o = np.ones(3)
    assert lib.hdmr_create(0, 1, 1, G._np_ptr(z), G._np_ptr(z), G._np_ptr(o), C.byref(h)) == -1
    assert lib.hdmr_create(3, 1, 9, G._np_ptr(z), G._np_ptr(z), G._np_ptr(o), C.byref(h)) == -1
    assert lib.hdmr_create(3, 1, 1, G._np_ptr(z), G._np_ptr(o), G._np_ptr(z), C.byref(h)) == -1
    assert b"lo" in lib.ddsg_last_error()
    assert lib.hdmr_create(3, 1, 1, G._np_ptr(z), G._np_ptr(z), G._np_ptr(o), C.byref(h)) == 0
    assert lib.hdmr_destroy(h) == 0


def test_add_component_validation():
    h = G.HDMR(3, 2, 2)
    h.add_component([])
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        h.add_component([])                              # duplicate component
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        h.add_component([2, 1], [[1, 1]], [[1, 1]])      # dims not ascending
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        h.add_component([0, 1, 2], [[1, 1, 1]], [[1, 1, 1]])  # k > order
    with pytest.raises(G.DDSGError, match="ERR_TABLE"):
        h.add_component([0], [[3]], [[2]])               # even index at level 3
    with pytest.raises(G.DDSGError, match="ERR_TABLE"):
        h.add_component([0], [[2]], [[1]])               # level 2 takes index 0 or 2
    with pytest.raises(G.DDSGError, match="ERR_TABLE"):
        h.add_component([0], [[1], [1]], [[1], [1]])     # duplicate point
    with pytest.raises(G.DDSGError, match="ERR_TABLE"):
        h.add_component([0], [[0]], [[1]])               # level 0
    assert h.add_component([0], [[1], [2], [2]], [[1], [0], [2]]) == 1
    h.close()


@pytest.mark.parametrize("k,level", [(0, 4), (1, 1), (1, 10), (2, 6), (3, 5), (4, 5)])
def test_regular_grid_matches_oracle(k, level):
    h = G.HDMR(max(k, 1), 1, max(k, 1))
    cid = h.add_regular(list(range(k)), level)
    dims, npts, first = h.component_info(cid)
    lv, ix = O.regular_grid(k, level)
    assert npts == lv.shape[0] and first == 0
    if k:
        glv, gix, xs = h.component_points(cid)
        assert np.array_equal(glv, lv[:, :k]) and np.array_equal(gix, ix[:, :k])
        ref = np.array([[O.node1d(l, i) for l, i in zip(a, b)] for a, b in zip(lv[:, :k], ix[:, :k])])
        assert np.array_equal(xs, ref)
    h.close()


def test_component_points_physical_coordinates():
    h = G.HDMR(2, 1, 1, lo=[0.8, -2.0], hi=[1.2, 2.0])
    h.add_component([])
    cid = h.add_regular([1], 3)
    _, _, xs = h.component_points(cid)
    assert np.array_equal(np.sort(xs[:, 0]), np.array([-2.0, -1.0, 0.0, 1.0, 2.0]))


def test_b_coefficients_match_oracle():
    d = 6
    comps = O.full_order_components(d, 2)
    comps = [u for u in comps if u not in [(0, 3), (2, 5)]]   # an eta-pruned set stays closed
    h = G.HDMR(d, 1, 2)
    E = O.OracleDDSG(d, 1)
    for u in comps:
        h.add_regular(list(u), 2)
        E.add_regular(u, 2)
    assert np.array_equal(h.b_coeffs(), E.b_coeffs())


def test_b_coefficients_non_closed_set_match_oracle():
    comps = [(), (0,), (0, 1), (0, 1, 2)]     # {1}, {2}, ... missing: eq. 4.2 over U as given
    h = G.HDMR(3, 1, 3)
    E = O.OracleDDSG(3, 1)
    for u in comps:
        h.add_regular(list(u), 2)
        E.add_regular(u, 2)
    assert np.array_equal(h.b_coeffs(), E.b_coeffs())


def test_table1_helper_matches_oracle():
    for N in (1, 3, 150):
        t = G.irbc_table1(N)
        I = O.IRBCOracle(N)
        assert abs(t["A"] - I.A) <= 1e-16 * I.A
        assert np.allclose(t["gamma"], I.gamma, rtol=0, atol=1e-15)
        assert np.allclose(t["tau"], I.tau, rtol=1e-14)


def test_irbc_create_table1_validates():
    """The Table 1 constructor refuses out-of-range calibrations before anything runs."""
    lib = G.load()
    h = C.c_void_p()
    ok = (3, 0.25, 0.99, 0.36, 0.01, 0.01, 0.95, 0.5)
    assert lib.irbc_create_table1(*ok, C.byref(h)) == 0
    assert lib.irbc_destroy(h) == 0
    for bad in ((0,) + ok[1:], (3, 0.0) + ok[2:], (3, 0.25, 1.0) + ok[3:], (3, 0.25, 0.99, 0.0) + ok[4:],
                (3, 0.25, 0.99, 0.36, 1.0) + ok[5:]):
        assert lib.irbc_create_table1(*bad, C.byref(h)) == -1, bad
    t = G.irbc_table1(1)
    assert t["gamma"].tolist() == [0.25] and abs(t["tau"][0] - t["A"] ** 4) <= 1e-15 * t["A"] ** 4


def test_irbc_create_validates():
    lib = G.load()
    h = C.c_void_p()
    prm = G.IrbcParams(0, 0.99, 0.36, 0.01, 0.01, 0.95, 0.5, 1.0)
    g = np.ones(1)
    assert lib.irbc_create(C.byref(prm), G._np_ptr(g), G._np_ptr(g), C.byref(h)) == -1
    prm.N = 1
    assert lib.irbc_create(C.byref(prm), G._np_ptr(g), G._np_ptr(g), C.byref(h)) == 0
    assert lib.irbc_destroy(h) == 0


def test_test_switches_validate_without_a_gpu():
    # allocation-failure switch: process-wide, no CUDA call
    with pytest.raises(G.DDSGError, match="ERR_ARG") as ei:
        G.inject_alloc_failure(-1, 1)
    assert ei.value.code == -1
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        G.inject_alloc_failure(0, -1)
    G.inject_alloc_failure(3, 2)
    G.inject_alloc_failure(0, 0)
    h = G.HDMR(3, 2, 1)
    h.add_regular([0], 2)
    assert G.load().hdmr_check(h._h, None) == 0   # nothing ran on a device: no status
    with pytest.raises(G.DDSGError, match="ERR_ARG"):
        h.set_fault_injection(-2)
    h.set_fault_injection(4)
    h.set_fault_injection(-1)
