"""GPU parity of the warm-start network (BF16 tensor-core kernels) against the
FP64 reference, and the network's gain as a Newton initial guess.

Bars (BF16 operands carry 8 significant bits, FP32 accumulation):
  forward: ||y_gpu - y_ref||_2 / ||y_ref - out_shift||_2 <= 2e-2 (normalized outputs);
  gradients: per tensor ||g_gpu - g_ref||_F / ||g_ref||_F <= 3e-2;
  loss curve over 10 Adam steps: |L_gpu - L_ref| / L_ref <= 5e-2 at every step."""
import numpy as np
import pytest

import synth
from oracle.mlp import OracleMLP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [40, 256, 256, 256, 21]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_06555_gb300 as G
    G.load()
    return G


def _params(sizes, seed):
    W, b, flat = [], [], []
    for l in range(len(sizes) - 1):
        bound = 1.0 / np.sqrt(sizes[l])
        w = synth.uniform_matrix(seed + l, sizes[l + 1], sizes[l], -bound, bound)
        bb = (synth.uniform(seed + 100 + l, sizes[l + 1]) - 0.5) * 0.1
        W.append(w)
        b.append(bb)
        flat += [w.ravel(), bb]
    return W, b, np.concatenate(flat).astype(np.float32)


def _norm(sizes):
    return (np.full(sizes[0], 1.0), np.full(sizes[0], 5.0),
            np.linspace(0.95, 1.05, sizes[-1]), np.full(sizes[-1], 10.0))


def _pair(G, seed=31):
    W, b, flat = _params(SIZES, seed)
    # oracle uses the BF16-representable FP32 weights the GPU starts from
    Wf = [w.astype(np.float32).astype(np.float64) for w in W]
    bf = [x.astype(np.float32).astype(np.float64) for x in b]
    nrm = _norm(SIZES)
    ref = OracleMLP(SIZES, *nrm, weights=(Wf, bf))
    net = G.MLP(SIZES, params=flat, in_shift=nrm[0], in_scale=nrm[1], out_shift=nrm[2], out_scale=nrm[3])
    return ref, net


def _data(n, seed):
    x = synth.uniform_matrix(seed, n, SIZES[0], 0.8, 1.2)
    A = synth.uniform_matrix(seed + 1, SIZES[0], SIZES[-1], -1, 1) / SIZES[0]
    y = 1.0 + 0.05 * np.sin(4 * (x - 1) @ A) + 0.02 * ((x - 1) ** 2) @ np.abs(A)
    return x, y


def test_forward_matches_reference(G):
    ref, net = _pair(G)
    x, _ = _data(1000, 41)
    y_ref = ref.predict(x)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros((x.shape[0], SIZES[-1]), dtype=torch.float64, device="cuda")
    net.infer(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref - ref.out_shift) <= 2e-2


def test_gradients_match_reference(G):
    ref, net = _pair(G)
    x, y = _data(512, 42)
    _, gW, gb = ref.loss_and_grads(x, y)
    net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 0.0)
    torch.cuda.synchronize()
    GW, Gb = net.grads()
    for l in range(len(gW)):
        assert np.linalg.norm(GW[l] - gW[l]) / np.linalg.norm(gW[l]) <= 3e-2, l
        assert np.linalg.norm(Gb[l] - gb[l]) / max(np.linalg.norm(gb[l]), 1e-30) <= 3e-2, l
    net.check()   # no tensor-core GEMM gave up a wait


@pytest.mark.parametrize("batch", [1, 127, 128, 129, 4096 + 65])
def test_ragged_batches_match_reference(G, batch):
    """Batches padded to the 128-row GEMM tile: ragged and tiny sizes (one row, one
    short of and one past a tile) through forward and backward."""
    ref, net = _pair(G)
    x, y = _data(batch, 45)
    _, gW, gb = ref.loss_and_grads(x, y)
    net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 0.0)
    GW, Gb = net.grads()
    for l in range(len(gW)):
        assert np.linalg.norm(GW[l] - gW[l]) / np.linalg.norm(gW[l]) <= 3e-2, (batch, l)
        assert np.linalg.norm(Gb[l] - gb[l]) / max(np.linalg.norm(gb[l]), 1e-30) <= 3e-2, (batch, l)
    yd = torch.zeros((batch, SIZES[-1]), dtype=torch.float64, device="cuda")
    net.infer(torch.from_numpy(x).cuda(), yd)
    y_ref = ref.predict(x)
    assert np.linalg.norm(yd.cpu().numpy() - y_ref) / np.linalg.norm(y_ref - ref.out_shift) <= 2e-2
    net.check()


def test_loss_curve_matches_reference(G):
    ref, net = _pair(G)
    x, y = _data(1024, 43)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for step in range(10):
        l_ref, gW, gb = ref.loss_and_grads(x, y)
        ref.adam_step(gW, gb, lr=1e-3)
        net.train_step(xd, yd, 1e-3, loss)
        torch.cuda.synchronize()
        assert abs(loss.item() - l_ref) / l_ref <= 5e-2, (step, loss.item(), l_ref)


def test_training_learns_a_smooth_map(G):
    _, net = _pair(G, seed=77)
    x, y = _data(8192, 44)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    first = None
    for step in range(300):
        lo = (step * 1024) % 8192
        net.train_step(xd[lo:lo + 1024], yd[lo:lo + 1024], 2e-3, loss)
        if step == 0:
            torch.cuda.synchronize()
            first = loss.item()
    torch.cuda.synchronize()
    assert loss.item() < 0.05 * first


def test_warm_start_reduces_newton_iterations(G):
    """IRBC N=5: solve the Euler equations at 6000 states from the previous
    policy's values, train the network on those (state, solution) pairs, then
    solve at 400 new states from (a) the previous policy and (b) the network:
    both converge to the same tolerance and the network needs fewer iterations."""
    from test_gpu_irbc import make_model
    N = 5
    I, E, h, M, lam = make_model(G, N)
    d, m = 2 * N, N + 1

    def solve(S, guess, tol=1e-10):
        sd = torch.from_numpy(S).cuda()
        z = torch.from_numpy(np.ascontiguousarray(guess)).cuda()
        it = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
        st = torch.zeros(S.shape[0], dtype=torch.int32, device="cuda")
        M.newton(h, sd, z, 30, tol, it, st, None, 0, 1)
        torch.cuda.synchronize()
        return z.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()

    def policy_guess(S):
        y = torch.zeros((S.shape[0], m), dtype=torch.float64, device="cuda")
        h.eval(torch.from_numpy(S).cuda(), y, 0, 1)
        torch.cuda.synchronize()
        return y.cpu().numpy()

    S = synth.irbc_states(synth.BASE_SEED + 500, 6000, N)
    sol, it0, st0 = solve(S, policy_guess(S))
    assert np.all(st0 == 0)
    sizes = [d, 64, 64, m]
    mu, sd_ = sol.mean(0), sol.std(0) + 1e-12
    net = G.MLP(sizes, seed=5, in_shift=np.full(d, 1.0), in_scale=np.full(d, 5.0), out_shift=mu,
                out_scale=1.0 / sd_)
    xd, yd = torch.from_numpy(S).cuda(), torch.from_numpy(sol).cuda()
    for ep in range(60):
        for lo in range(0, 6000, 500):
            net.train_step(xd[lo:lo + 500], yd[lo:lo + 500], 3e-3 if ep < 40 else 1e-3)
    T = synth.irbc_states(synth.BASE_SEED + 501, 400, N)
    g_nn = torch.zeros((400, m), dtype=torch.float64, device="cuda")
    net.infer(torch.from_numpy(T).cuda(), g_nn)
    torch.cuda.synchronize()
    z_p, it_p, st_p = solve(T, policy_guess(T))
    z_n, it_n, st_n = solve(T, g_nn.cpu().numpy())
    assert np.all(st_p == 0) and np.all(st_n == 0)
    assert np.allclose(z_p, z_n, atol=1e-8)
    assert it_n.mean() < it_p.mean()
