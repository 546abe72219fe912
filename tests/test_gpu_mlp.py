"""GPU learned-eps network: features, forward, backward (against the float64
oracle's analytic gradients, themselves pinned by finite differences), and
what the trained network gains over the plain search at the same kappa_T."""
import numpy as np
import pytest
import torch

from oracle import mlp as om
from oracle import stencils as ost
from paper_1404_0812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def R():
    import paper_1404_0812_gb300 as R
    R._lib.load()
    return R


def test_features_match_oracle(R):
    ns = W.bumpy_sphere(5000)
    op = R.build_operator(T(ns.X), T(ns.normals), 50, kernel="imq", kappa_target=1e12)
    f, tgt = R.features(op, T(ns.X), T(ns.normals), 50)
    f = f.cpu().numpy()
    tgt = tgt.cpu().numpy()
    eps = R.get_stencil_info(op)["eps"].cpu().numpy()
    for k in range(0, ns.N, 211):
        idx = ost.stencil(ns.X, k, 50)
        fr, rs = om.features(ns.X[idx], ns.normals[idx[0]])
        assert np.abs(f[k] - fr).max() <= 2e-6
        assert abs(tgt[k] - np.log(eps[k] * rs)) <= 1e-5


def test_forward_and_gradients_match_oracle(R):
    n, B = 50, 300
    D = 3 * n
    p64 = W.mlp_init(D, seed=11)
    net = R.EpsNet(n, W.mlp_pack(p64).astype(np.float32))
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, (B, D))
    t = rng.normal(-1.0, 0.3, B)
    x32, t32 = x.astype(np.float32), t.astype(np.float32)
    pr = net.predict(T(x32, torch.float32)).cpu().numpy()
    y_ref, _ = om.forward(p64, x32.astype(np.float64))
    assert np.abs(pr - y_ref).max() <= 1e-5 * max(1.0, np.abs(y_ref).max())
    g, loss = net.loss_grad(T(x32, torch.float32), T(t32, torch.float32))
    l_ref, g_ref = om.loss_and_grads(p64, x32.astype(np.float64), t32.astype(np.float64))
    assert abs(loss - l_ref) <= 1e-5 * abs(l_ref)
    g = g.cpu().numpy()
    g_flat = W.mlp_pack(g_ref)
    assert np.abs(g - g_flat).max() <= 1e-4 * np.abs(g_flat).max()


def test_training_reduces_loss_and_warm_start_saves_evaluations(R):
    """Train on plain-search eps of a sphere and a torus (n = 50, IMQ,
    kappa_T = 1e12), then build a held-out bumpy sphere both ways: the
    learned start needs fewer kappa evaluations per stencil (the network is
    accepted outright for a third or more of the held-out stencils), every accepted
    prediction lies in the [0.5, 2] kappa_T band, and the rest still meet the
    search's tolerance."""
    n = 50
    feats, tg = [], []
    for ns in (W.fibonacci_sphere(100_000), W.torus_staggered(129)):   # 200k pairs
        op = R.build_operator(T(ns.X), T(ns.normals), n, kernel="imq", kappa_target=1e12)
        f, t = R.features(op, T(ns.X), T(ns.normals), n)
        feats.append(f)
        tg.append(t)
    F = torch.cat(feats).contiguous()
    Tt = torch.cat(tg).contiguous()
    net = R.EpsNet(n, W.mlp_pack(W.mlp_init(3 * n, seed=0)).astype(np.float32))
    losses = net.train(F, Tt, epochs=25, batch=1024, lr=1e-3, seed=0)
    assert losses[-1] < 0.2 * losses[0]
    test = W.bumpy_sphere(20000)
    X, Nn = T(test.X), T(test.normals)
    plain = R.build_operator(X, Nn, n, kernel="imq", kappa_target=1e12)
    learned = R.build_operator(X, Nn, n, kernel="imq", kappa_target=1e12, mlps=[net])
    ip = {k: v.cpu().numpy() for k, v in R.get_stencil_info(plain).items()}
    il = {k: v.cpu().numpy() for k, v in R.get_stencil_info(learned).items()}
    assert np.all(ip["status"] == 0)
    assert np.all((il["status"] == 0) | (il["status"] == 4))
    acc = il["status"] == 4
    print("accepted", acc.mean(), "evals learned", il["evals"].mean(), "plain", ip["evals"].mean())
    assert acc.mean() > 0.3
    assert np.all((il["kappa"][acc] >= 0.5e12) & (il["kappa"][acc] <= 2e12))
    assert np.all(np.abs(np.log(il["kappa"][~acc] / 1e12)) < 0.05)
    assert il["evals"].mean() < 0.6 * ip["evals"].mean()


def test_mlp_load_replaces_parameters(R):
    n = 31
    p1 = W.mlp_pack(W.mlp_init(3 * n, seed=1)).astype(np.float32)
    p2 = W.mlp_pack(W.mlp_init(3 * n, seed=2)).astype(np.float32)
    a = R.EpsNet(n, p1)
    a.load(p2)
    assert np.array_equal(a.params(), p2)
    b = R.EpsNet(n, p2)
    x = T(np.random.default_rng(5).uniform(-1, 1, (100, 3 * n)), torch.float32)
    assert torch.equal(a.predict(x), b.predict(x))
    with pytest.raises(ValueError):
        a.load(p2[:-1])


def _unpack_like(W, flat, p):
    return W.mlp_unpack(np.asarray(flat, dtype=np.float64), p["W1"].shape[0])



def test_adam_update_matches_oracle_exactly_given_the_gradient(R):
    """rbffd_mlp_train's optimiser step against oracle.mlp.adam_step (float64)
    at t = 1 and t = 2 (first and second moments, both bias corrections).
    Every sample is the same, so the shuffled full batch (epochs = 1, batch =
    count) sums exactly the tiles rbffd_mlp_loss_grad sums: the GPU gradient
    at each step is known bit for bit, and the oracle's Adam applied to it
    must give the GPU's new parameters up to float32 rounding."""
    n, B = 31, 256
    D = 3 * n
    p64 = W.mlp_init(D, seed=21)
    p32 = W.mlp_pack(p64).astype(np.float32)
    net = R.EpsNet(n, p32)
    rng = np.random.default_rng(22)
    x = np.repeat(rng.uniform(-1, 1, (1, D)), B, axis=0).astype(np.float32)
    t = np.full(B, -0.7, dtype=np.float32)
    X, Tt = T(x, torch.float32), T(t, torch.float32)
    ref = {k: v.astype(np.float32).astype(np.float64) for k, v in p64.items()}
    state = {}
    for step in (1, 2):
        g, _ = net.loss_grad(X, Tt)                      # gradient at the GPU's current params
        g = _unpack_like(W, g.cpu().numpy(), p64)
        net.train(X, Tt, epochs=1, batch=B, lr=1e-3, seed=step)
        om.adam_step(ref, g, state, lr=1e-3)
        got, want = net.params().astype(np.float64), W.mlp_pack(ref)
        err = np.abs(got - want)
        assert err.max() <= 1e-7 * max(1.0, np.abs(want).max()), (step, err.max())
        # the GPU continues from its own float32 parameters
        ref = {k: v.astype(np.float32).astype(np.float64) for k, v in
               W.mlp_unpack(got, D).items()}


def test_adam_full_batch_steps_match_float64_oracle(R):
    """Two full-batch rbffd_mlp_train steps (distinct samples) from known
    parameters against oracle.mlp.loss_and_grads + adam_step in float64.
    Parameters whose gradient is at least 1e-2 of the largest (the float32
    gradient is within 1e-4 of the largest, test above, so their direction
    is fixed) must move as the oracle moves them, to 2e-2 of the learning
    rate; the rest by at most the learning rate times Adam's bound."""
    n, B = 50, 512
    D = 3 * n
    p64 = W.mlp_init(D, seed=31)
    net = R.EpsNet(n, W.mlp_pack(p64).astype(np.float32))
    rng = np.random.default_rng(32)
    x = rng.uniform(-1, 1, (B, D)).astype(np.float32)
    t = rng.normal(-1.0, 0.3, B).astype(np.float32)
    X, Tt = T(x, torch.float32), T(t, torch.float32)
    ref = {k: v.astype(np.float32).astype(np.float64) for k, v in p64.items()}
    state = {}
    lr = 1e-3
    prev = W.mlp_pack(ref)
    for step in (1, 2):
        _, g = om.loss_and_grads(ref, x.astype(np.float64), t.astype(np.float64))
        om.adam_step(ref, g, state, lr=lr)
        net.train(X, Tt, epochs=1, batch=B, lr=lr, seed=step)
        got, want = net.params().astype(np.float64), W.mlp_pack(ref)
        gf = np.abs(W.mlp_pack(g))
        well = gf >= 1e-2 * gf.max()
        assert well.sum() > 50
        assert np.abs(got - want)[well].max() <= 2e-2 * lr, step
        # a bias-corrected Adam step moves a coordinate by at most ~lr at
        # t = 1 and 2 (Cauchy-Schwarz on m_hat / sqrt(v_hat): <= 1.0014 lr)
        assert np.abs(got - prev).max() <= 1.01 * lr * step
