"""Allocation failures and error statuses, made on the host (no GPU fault).

ddsg_inject_alloc_failure(skip, 1) lets `skip` device allocations of libddsg
succeed and fails the next one as an exhausted device would. For each entry point
that allocates, each of its allocation sites is failed in turn on a fresh object
(skip = 0, 1, 2, ...). The call must return DDSG_ERR_OOM, and the same call on the
same object must then succeed with the switch off, giving results identical to
those of an object that never saw a failure. Also here: hdmr_check turns a
wait timeout into DDSG_ERR_TIMEOUT, and hdmr_refine turns a non-finite surplus
into DDSG_ERR_NUMERIC.
"""
import numpy as np
import pytest

import oracle as O
import synth
from test_gpu_irbc import make_model, states_and_guess

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ERR_OOM, ERR_TIMEOUT, ERR_NUMERIC = -2, -6, -7


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def sweep(G, make, call, check, limit=200):
    """Fail allocation site 0, 1, 2, ... of call(make()); returns how many sites
    the call has (the first skip that fails nothing)."""
    for skip in range(limit):
        obj = make()
        G.inject_alloc_failure(skip, 1)
        try:
            call(obj)
            failed = False
        except G.DDSGError as e:
            assert e.code == ERR_OOM, e
            failed = True
        finally:
            G.inject_alloc_failure(0, 0)
        if not failed:
            check(obj)
            return skip
        call(obj)
        check(obj)
    raise AssertionError("the call kept allocating")


D, M_OUT = 4, 3
COMPS = O.full_order_components(D, 2)


def _values(h, c):
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    return np.concatenate([fn(u, h.component_points(i)[2]) for i, u in enumerate(COMPS)])


def _fresh(G):
    h = G.HDMR(D, M_OUT, 2)
    for u in COMPS:
        h.add_regular(list(u), 4)
    return h


def _eval(h, X, prec=0):
    x = torch.from_numpy(X).cuda()
    y = torch.zeros((X.shape[0], M_OUT), dtype=torch.float64, device="cuda")
    h.eval(x, y, prec, 1)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_hdmr_allocation_sites_fail_cleanly(G):
    c = synth.family_coeffs(synth.BASE_SEED + 91, M_OUT, D)
    X = synth.uniform_queries(92, 700, D)
    clean = _fresh(G)
    vals = torch.from_numpy(_values(clean, c)).cuda()
    clean.hierarchize(vals)
    want = _eval(clean, X)

    # first GPU use and table upload
    def check_h(h):
        assert np.array_equal(_eval(h, X), want)
    n = sweep(G, lambda: _fresh(G), lambda h: h.hierarchize(vals), check_h)
    assert n >= 5, n        # per-handle buffers, tables, surpluses

    # the evaluation workspace (a fresh handle per site, hierarchized cleanly)
    def ready():
        h = _fresh(G)
        h.hierarchize(vals)
        torch.cuda.synchronize()
        return h
    x = torch.from_numpy(X).cuda()
    y = torch.zeros((X.shape[0], M_OUT), dtype=torch.float64, device="cuda")

    def ev(h):
        h.eval(x, y, 0, 1)
        torch.cuda.synchronize()

    def check_ev(h):
        assert np.array_equal(y.cpu().numpy(), want)
    assert sweep(G, ready, ev, check_ev) >= 1

    # host buffers that are not page-locked go through a device staging buffer
    yh = np.zeros((X.shape[0], M_OUT))

    def evh(h):
        h.eval_host(np.ascontiguousarray(X), yh, 0, 1)

    def check_evh(h):
        assert np.array_equal(yh, want)
    assert sweep(G, ready, evh, check_evh) >= 1


def test_irbc_allocation_sites_fail_cleanly(G):
    N, ns = 4, 50
    I, E, h, M0, lam = make_model(G, N, level=3)
    S, g = states_and_guess(N, ns, lam, synth.BASE_SEED + 93)
    sd, gd = torch.from_numpy(S).cuda(), torch.from_numpy(g).cuda()

    def fresh():
        return G.IRBC(N, I.p["beta"], I.p["alpha"], I.p["delta"], I.p["sigma"], I.p["rho"],
                      I.p["phi"], I.A, I.gamma, I.tau)

    def resid(M):
        r = torch.zeros((ns, N + 1), dtype=torch.float64, device="cuda")
        J = torch.zeros((ns, N + 1, N + 1), dtype=torch.float64, device="cuda")
        M.residual(h, sd, gd, r, J, None, 0, 1)
        torch.cuda.synchronize()
        return r.cpu().numpy(), J.cpu().numpy()

    r_want, J_want = resid(M0)

    def check_r(M):
        r, J = resid(M)
        assert np.array_equal(r, r_want) and np.array_equal(J, J_want)
    assert sweep(G, fresh, resid, check_r) >= 2

    sol = torch.empty_like(gd)

    def newton(M):
        sol.copy_(gd)
        M.newton(h, sd, sol, 30, 1e-10, precision=0, form=1)
        torch.cuda.synchronize()
        return sol.cpu().numpy()
    s_want = newton(M0)

    def check_n(M):
        assert np.array_equal(newton(M), s_want)
    assert sweep(G, fresh, newton, check_n) >= 2


def test_mlp_allocation_sites_fail_cleanly(G):
    sizes = [6, 32, 32, 3]
    x = torch.from_numpy(synth.uniform_matrix(94, 300, sizes[0], 0.8, 1.2)).cuda()
    y = torch.zeros((300, sizes[-1]), dtype=torch.float64, device="cuda")

    def fresh():
        return G.MLP(sizes, seed=7)

    def infer(net):
        net.infer(x, y)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    want = infer(fresh())

    def check(net):
        assert np.array_equal(infer(net), want)
    assert sweep(G, fresh, infer, check) >= 10


def test_check_reports_wait_timeouts(G):
    c = synth.family_coeffs(synth.BASE_SEED + 95, M_OUT, D)
    h = _fresh(G)
    h.check()                                    # before any GPU use
    h.hierarchize(torch.from_numpy(_values(h, c)).cuda())
    X = synth.uniform_queries(96, 300, D)
    saved = h.eval_config(1, 1)
    h.set_eval_config(1, 1, 3, 8)
    want = _eval(h, X, 1)
    h.check()
    h.set_fault_injection(1)
    assert np.isnan(_eval(h, X, 1)).all()
    with pytest.raises(G.DDSGError, match="bounded wait") as ei:
        h.check()
    assert ei.value.code == ERR_TIMEOUT
    h.check()                                    # reported once, then cleared
    assert h.stats()["wait_timeouts"] == 0
    h.set_fault_injection(-1)
    assert np.array_equal(_eval(h, X, 1), want)
    h.check()
    h.set_eval_config(1, 1, *saved)


def test_refine_rejects_non_finite_surpluses(G):
    c = synth.family_coeffs(synth.BASE_SEED + 97, M_OUT, D)
    h = _fresh(G)
    v = _values(h, c)
    v[7, 1] = np.nan
    h.hierarchize(torch.from_numpy(v).cuda())
    with pytest.raises(G.DDSGError, match="not finite") as ei:
        h.refine(1e-3, 6)
    assert ei.value.code == ERR_NUMERIC
    assert h.sizes() == _fresh(G).sizes()        # nothing was added

    def fn(dims, X):
        out = synth.family_cut(c, dims, X)
        if len(dims) == 2:
            out[-1, 0] = np.inf
        return out
    h2 = G.HDMR(D, M_OUT, 2)
    for u in COMPS:
        h2.add_regular(list(u), 2)
    with pytest.raises(G.DDSGError, match="not finite"):
        G.build_adaptive(h2, fn, 1e-3, 6)
