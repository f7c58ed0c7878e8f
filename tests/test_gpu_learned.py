"""The learned weights on the GPU: the MLP kernels against the FP64 oracle MLP,
the V-cycle loss gradient against the oracle's reverse mode, checkpointing,
the safety fallback, and what a trained network gains over the optimal
4th-kind weights on held-out problems."""
import numpy as np
import pytest

from oracle import mlp as omlp
from oracle.adjoint import error_reduction_loss
from oracle.amg import OracleAMG
from oracle.smoother import SmootherSpec
from paper_2407_09848_gb300 import problems as pr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_09848_gb300 import build
    build.build()
    return torch


def test_mlp_kernels_match_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2407_09848_gb300 import amgps
    rng = np.random.default_rng(0)
    th = (rng.standard_normal(4996) * 0.3).astype(np.float32)
    B = 37
    F = rng.standard_normal((B, 8)).astype(np.float32)
    ref = amgps.opt4_weights(4).astype(np.float32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    tp, Fd, rd = d(th), d(F), d(ref)
    beta = torch.empty(B * 4, dtype=torch.float32, device="cuda")
    acts = torch.empty(B * 132, dtype=torch.float32, device="cuda")
    amgps.mlp_forward(tp, Fd, rd, beta, acts)
    ob, cache = omlp.forward(th.astype(np.float64), F.astype(np.float64), ref.astype(np.float64))
    gb = beta.cpu().numpy().reshape(B, 4)
    assert np.max(np.abs(gb - ob)) <= 1e-5 * np.max(np.abs(ob))
    G = rng.standard_normal((B, 4)).astype(np.float32)
    grads = torch.empty(4996, dtype=torch.float32, device="cuda")
    work = torch.empty(B * 132, dtype=torch.float32, device="cuda")
    amgps.mlp_backward(tp, Fd, acts, beta, d(G), work, grads)
    og = omlp.backward(th.astype(np.float64), cache, G.astype(np.float64))
    gg = grads.cpu().numpy()
    assert np.linalg.norm(gg - og) <= 1e-5 * np.linalg.norm(og)
    m = torch.zeros(4996, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    amgps.mlp_adam(tp, grads, m, v, 1, 1e-3)
    onew, _, _ = omlp.adam(th.astype(np.float64), gg.astype(np.float64), np.zeros(4996),
                           np.zeros(4996), 1, 1e-3)
    assert np.max(np.abs(tp.cpu().numpy() - onew)) <= 1e-6


def test_loss_grad_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2407_09848_gb300.amgps import Solver
    H = pr.build_hierarchy(pr.varcoef(14, 1.2, 3.0, seed=3, ny=12, nz=10), coarse_max=30)
    S = Solver().load(H.A, H.P)
    rng = np.random.default_rng(4)
    specs = []
    for l in range(H.n_levels - 1):
        b = 1 + 0.2 * rng.uniform(-1, 1, 4)
        S.set_smoother(l, "weights", 4, weights=b)
        specs.append(SmootherSpec("weights", 4, beta=b))
    E0 = rng.standard_normal((5, H.A[0].shape[0]))
    loss, gw = S.loss_grad(torch.from_numpy(E0).cuda())
    oloss, og = error_reduction_loss(OracleAMG(H.A, H.P, specs), E0.T)
    assert abs(loss - oloss) <= 1e-11 * oloss
    for l in range(H.n_levels - 1):
        assert np.max(np.abs(gw[l, :4] - og[l])) <= 1e-10 * np.max(np.abs(og[l]))


def test_safety_fallback_and_checkpoint(torch_cuda, tmp_path):
    from paper_2407_09848_gb300 import amgps, learn
    assert learn.is_safe(amgps.opt4_weights(4))
    bad = np.array([3.0, 3.0, 3.0, 3.0])
    assert not learn.is_safe(bad)
    w, t = learn.make_safe(bad, amgps.opt4_weights(4))
    assert 0.0 < t < 1.0 and learn.is_safe(w)
    assert np.allclose(w, amgps.opt4_weights(4) + t * (bad - amgps.opt4_weights(4)))
    H = pr.build_hierarchy(pr.varcoef(12, 1.0, 3.0, seed=5), coarse_max=30)
    p = learn.Problem(H, nvec=4, seed=1, pre_cycles=0)
    ref = amgps.opt4_weights(4)
    nl = H.n_levels - 1
    l_ref, _ = p.loss_grad([ref] * nl)
    # unsafe weights are pulled back towards the optimal ones; the gradient
    # in the prediction is the installed weights' gradient times t
    l_bad, g_bad = p.loss_grad([bad] * nl)
    l_w, g_w = p.loss_grad([w] * nl)
    assert l_bad == l_w and np.allclose(g_bad, t * g_w, rtol=1e-12, atol=0)
    net = learn.WeightMLP(seed=1)
    probs = [p, learn.Problem(pr.build_hierarchy(pr.varcoef(12, 1.5, 4.0, seed=6), coarse_max=30),
                              nvec=4, seed=2)]
    learn.train(net, probs, 3, batch=2, lr=1e-3)
    net.save(tmp_path / "ckpt.npz")
    net2 = learn.WeightMLP(seed=99).load(tmp_path / "ckpt.npz")
    learn.train(net, probs, 1, batch=2, lr=1e-3, seed=5)
    learn.train(net2, probs, 1, batch=2, lr=1e-3, seed=5)
    assert np.array_equal(net.params.cpu().numpy(), net2.params.cpu().numpy())


def test_error_cycles_estimate_convergence_factor(torch_cuda):
    # after many cycles the one-cycle reduction approaches rho(E)^2, the
    # largest eigenvalue of E in the A inner product (dense check on 8^3)
    torch = torch_cuda
    from paper_2407_09848_gb300.amgps import Solver
    H = pr.build_hierarchy(pr.varcoef(8, 1.0, 3.0, seed=2), coarse_max=8)
    S = Solver().load(H.A, H.P)
    n = H.A[0].shape[0]
    ora = OracleAMG(H.A, H.P, SmootherSpec("cheb4_opt", 4))
    B = np.stack([ora.vcycle(e) for e in np.eye(n)], axis=1)
    Ad = H.A[0].toarray()
    L = np.linalg.cholesky(Ad)
    Et = L.T @ (np.eye(n) - B @ Ad) @ np.linalg.inv(L.T)   # E in the A-orthonormal basis
    rho = np.max(np.abs(np.linalg.eigvalsh(0.5 * (Et + Et.T))))
    E = torch.from_numpy(np.random.default_rng(0).standard_normal((3, n))).cuda()
    S.error_cycles(E, 60)
    loss, _ = S.loss_grad(E)
    # a Rayleigh quotient of E^2: approaches rho^2 from below
    assert 0.99 * rho ** 2 <= loss <= (1 + 1e-9) * rho ** 2


def test_trained_network_gain_over_optimal_weights(torch_cuda):
    # train on 12 log-normal 24^3 problems, evaluate on 6 held-out ones, with the
    # convergence-factor objective
    from paper_2407_09848_gb300 import learn
    train_set = learn.make_training_set(12, 24, seed0=0, nvec=8)
    test_set = learn.make_training_set(6, 24, seed0=5000, nvec=8)
    net = learn.WeightMLP(seed=0)
    before_learned, ref = learn.evaluate(net, test_set)
    assert abs(before_learned - ref) <= 1e-6 * ref   # untrained network = optimal weights
    hist = learn.train(net, train_set, 60, batch=12, lr=5e-3)
    after, _ = learn.evaluate(net, test_set)
    gain = 1.0 - after / ref
    print(f"held-out squared convergence factor: optimal weights {ref:.5f}, learned {after:.5f} "
          f"(gain {100 * gain:.2f}%); training loss {hist[0]:.5f} -> {hist[-1]:.5f}")
    assert hist[-1] < hist[0]
    assert after < ref


def test_optimal_weights_judge_the_network(torch_cuda):
    # set-up judge: the network's (safe) weights are kept exactly when PCG
    # with their V-cycle reduces the residual faster over the judge's
    # iterations than with the optimal weights; a smoother that barely
    # smooths (beta = 0.1) must lose
    from paper_2407_09848_gb300 import amgps, learn
    from paper_2407_09848_gb300.amgps import Solver
    H = pr.build_hierarchy(pr.varcoef(24, 1.5, 4.0, seed=9), coarse_max=100)
    S = Solver().load(H.A, H.P)
    nl = H.n_levels - 1
    ref = amgps.opt4_weights(4)
    b = torch_cuda.from_numpy(pr.vec_uniform(H.A[0].shape[0], seed=7)).cuda()
    fo = learn.pcg_factor(S, [ref] * nl, b)
    assert 0.0 < fo < 1.0
    for cand in (np.full(4, 0.1), np.full(4, 0.5), np.array([1.0, 1.1, 1.2, 1.6])):
        assert learn.is_safe(cand)
        used, fl, fo2, keep = learn.judge(S, [cand] * nl)
        assert fo2 == fo and keep == (fl < fo)
        assert all(np.array_equal(u, cand if keep else ref) for u in used)
        if cand[0] == 0.1:
            assert not keep and fl > fo
    used, fl, fo2, keep = learn.judge(S, [ref] * nl)  # equal factors: not kept
    assert fl == fo2 == fo and not keep
