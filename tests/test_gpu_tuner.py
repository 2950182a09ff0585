"""Tuner on the GPU: the MLP kernels against the FP64 oracle, the exhaustive sweep, and plan creation with
the sweep and with a learned model (including the fall-back to the sweep when the model's prediction
fails its sanity check)."""
import math

import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eh():
    import paper_2204_06666_gb300 as m
    torch.cuda.set_device(0)
    return m


def _data(seed, B=96):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 16))
    T = np.c_[np.tanh(X[:, :2].sum(1)), X[:, 2] * X[:, 3], np.abs(X[:, 4]), X[:, 5:8].mean(1)]
    theta = omlp.init(seed) + rng.uniform(-0.05, 0.05, omlp.NPARAM)
    return X, T, theta


def test_mlp_forward_matches_oracle(eh):
    X, T, theta = _data(1)
    net = eh.Mlp(torch.from_numpy(theta.astype(np.float32)))
    out = net.forward(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()
    ref, _ = omlp.forward(theta.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.allclose(out, ref, rtol=1e-4, atol=1e-5)


def test_mlp_gradients_match_oracle(eh):
    X, T, theta = _data(2)
    th32 = theta.astype(np.float32)
    net = eh.Mlp(torch.from_numpy(th32))
    loss, grad = net.loss_grad(torch.from_numpy(X.astype(np.float32)).cuda(),
                               torch.from_numpy(T.astype(np.float32)).cuda())
    L, g = omlp.grad(th32.astype(np.float64), X.astype(np.float32).astype(np.float64),
                     T.astype(np.float32).astype(np.float64))
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    gd = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gd - g) <= 1e-4 * np.linalg.norm(g)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.all(np.abs(gd[big] - g[big]) <= 1e-3 * np.abs(g[big]) + 1e-6)


def test_mlp_adam_step_matches_oracle(eh):
    X, T, theta = _data(3)
    th32 = theta.astype(np.float32)
    net = eh.Mlp(torch.from_numpy(th32))
    Xd, Td = torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda()
    th, m, v = th32.astype(np.float64), np.zeros(omlp.NPARAM), np.zeros(omlp.NPARAM)
    for t in range(1, 4):
        _, g = net.loss_grad(Xd, Td)
        net.adam(lr=1e-2)
        th, m, v = omlp.adam_step(th, m, v, g.cpu().numpy().astype(np.float64), t, lr=1e-2)
    assert np.allclose(net.params.cpu().numpy(), th, rtol=1e-5, atol=1e-6)


def test_mlp_training_on_gpu_reduces_loss(eh):
    X, T, theta = _data(4, B=512)
    net = eh.Mlp(torch.from_numpy(omlp.init(5).astype(np.float32)))
    Xd, Td = torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda()
    l0 = net.loss_grad(Xd, Td)[0].item()
    for _ in range(400):
        net.loss_grad(Xd, Td)
        net.adam(lr=3e-3)
    l1 = net.loss_grad(Xd, Td)[0].item()
    assert l1 < 0.25 * l0
    # the trained parameters evaluate to the same loss in the FP64 oracle
    L = omlp.loss(net.params.cpu().numpy().astype(np.float64), X.astype(np.float32), T.astype(np.float32))
    assert abs(L - l1) <= 1e-4 * L + 1e-7


def test_sweep_table_and_best(eh):
    A = gen.hex_lap3d(N=24)
    table, best = eh.tune_sweep(A, reps=5)
    assert len(table) == 112 and all(e["valid"] and e["ms"] > 0 for e in table)
    ms = [e["ms"] for e in table]
    assert best == int(np.argmin(ms))
    grid = eh.tune_grid(A)
    assert [(e["slice_rows"], e["ell_width_cap"], e["ell_tpr"]) for e in grid] == \
           [(e["slice_rows"], e["ell_width_cap"], e["ell_tpr"]) for e in table]


def _check_parity(eh, P, A, seed=3):
    x = gen.uniform(A.n, seed)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    P.spmv(xd, y)
    ref = oracle.spmv(A, x)
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-13 * np.linalg.norm(ref)


def test_plan_with_sweep(eh):
    A = gen.tet_lap3d(N=20, dirichlet=False)
    P = eh.Plan(A, tuner=2)
    info = P.info()
    assert info["tuner_path"] == 2
    _check_parity(eh, P, A)


def _constant_model(eh, slice_rows, log_ns):
    zeros = np.zeros(omlp.NPARAM, np.float32)   # the network outputs its (zero) last bias ...
    out_mean = np.array([math.log2(slice_rows), 0.0, 0.0, log_ns], np.float32)   # ... mapped to these
    eh.tuner_set_model(zeros, np.zeros(16), np.ones(16), out_mean, np.ones(4))


def test_learned_choice_kept_and_fallback(eh):
    A = gen.hex_elast3d(N=16)
    try:
        _constant_model(eh, 2048, math.log(1e6))     # a prediction that any plan meets
        assert eh.tuner_predict(A)[:3] == (2048, 0, 1)
        P = eh.Plan(A, tuner=1)
        info = P.info()
        assert info["tuner_path"] == 1 and info["slice_rows"] == 2048 and info["ell_tpr"] == 1
        _check_parity(eh, P, A)
        _constant_model(eh, 2048, math.log(1e-9))    # a prediction no plan meets: the sweep decides
        Q = eh.Plan(A, tuner=1)
        assert Q.info()["tuner_path"] == 3
        _check_parity(eh, Q, A)
    finally:
        eh.tuner_set_model(None, None, None, None, None)
    R = eh.Plan(A, tuner=1)                          # no model loaded: the sweep decides
    assert R.info()["tuner_path"] == 2


def test_trained_model_gains_over_eq1_default_on_heldout(eh):
    # the committed network (trained on the GPU by the library's MLP kernels on sweeps of matrices
    # 0..1999) against fresh sweeps of held-out matrices 5000..5011 (six FEM-like, six power-law)
    from paper_2204_06666_gb300 import tune
    tune.install()
    try:
        r_model, r_eq1 = [], []
        for i in range(5000, 5012):
            A = gen.tuner_matrix(i)
            table, best = eh.tune_sweep(A, reps=10)
            t = np.array([e["ms"] for e in table])
            sr, cap, tpr, _ = eh.tuner_predict(A)
            g = [(e["slice_rows"], e["ell_width_cap"], e["ell_tpr"]) for e in table].index((sr, cap, tpr))
            r_model.append(t[g] / t.min())
            r_eq1.append(t[0] / t.min())       # the method without the tuner: Eq. 1 VecSize, no cap, 1 lane
        gm_model = float(np.exp(np.mean(np.log(r_model))))
        gm_eq1 = float(np.exp(np.mean(np.log(r_eq1))))
        assert gm_model <= 1.10, r_model        # within 10% of the best swept configuration
        assert gm_eq1 / gm_model >= 1.3, (gm_eq1, gm_model)
        P = eh.Plan(gen.tuner_matrix(5001), tuner=1)    # plan creation through the model
        assert P.info()["tuner_path"] in (1, 3)
    finally:
        eh.tuner_set_model(None, None, None, None, None)
