"""The alpha/m MLP: CUDA forward/backward/Adam against the FP64 oracle, BF16 inference, and the
gain of the learned alpha over the fixed default on held-out instances."""
import time

import numpy as np
import pytest

from oracle import mlp_oracle as MO
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    return A


def rand_data(B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, 6)).astype(np.float32), rng.standard_normal((B, 2)).astype(np.float32)


def params(seed):
    th = MO.init_params(seed)
    th += 0.05 * np.random.default_rng(seed + 100).standard_normal(th.size)
    return th.astype(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("B", [1, 100, 128, 1000])
def test_forward_matches_oracle(aao, B):
    th = params(1)
    X, _ = rand_data(B, 2)
    h = aao.aao_mlp_create(th)
    Y = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    aao.aao_mlp_forward(h, dev(X), Y)
    ref, _ = MO.forward(th.astype(np.float64), X.astype(np.float64))
    assert np.abs(Y.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    aao.aao_mlp_forward(h, dev(X), Y, bf16=True)
    refb = MO.forward_bf16(th, X)
    got = Y.cpu().numpy()
    assert np.abs(got - refb).max() <= 2e-2 * max(1.0, np.abs(refb).max())
    assert np.abs(got - ref).max() <= 5e-2 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("B", [1, 127, 128, 129, 777])
def test_gradient_matches_oracle(aao, B):
    th = params(3)
    X, T = rand_data(B, 4)
    h = aao.aao_mlp_create(th)
    g, loss = aao.aao_mlp_grad(h, dev(X), dev(T))
    gr, lr_ = MO.grad(th.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr)
    assert abs(loss - lr_) <= 1e-5 * abs(lr_)
    g2, _ = aao.aao_mlp_grad(h, dev(X), dev(T))
    assert np.array_equal(g, g2)  # deterministic


def test_adam_matches_oracle(aao):
    th = params(5)
    X, T = rand_data(300, 6)
    h = aao.aao_mlp_create(th)
    ref = th.astype(np.float64)
    m = np.zeros_like(ref)
    v = np.zeros_like(ref)
    for t in range(1, 4):
        g, _ = aao.aao_mlp_grad(h, dev(X), dev(T))
        aao.aao_mlp_adam_step(h, dev(g), 1e-3)
        ref, m, v = MO.adam_step(ref, g.astype(np.float64), m, v, t, 1e-3)
    got = aao.aao_mlp_params(h)
    assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


def test_training_fits_a_teacher(aao):
    X, _ = rand_data(2048, 7)
    teacher = MO.init_params(8)
    T, _ = MO.forward(teacher, X.astype(np.float64))
    h = aao.aao_mlp_create(MO.init_params(9).astype(np.float32))
    Xd, Td = dev(X), dev(T.astype(np.float32))
    _, l0 = aao.aao_mlp_grad(h, Xd, Td)
    l1 = aao.aao_mlp_train(h, Xd, Td, 100, 256, 3e-3, seed=1)
    assert l1 < 0.05 * l0


def test_learned_alpha_and_m_against_the_default_on_held_out_instances(aao):
    """What the trained network gains over the fixed default (alpha 1e-3, m 20) on held-out
    instances of the batched distribution: every prediction converges (with the fallback), the
    iteration count is no worse on average, and the Krylov workspace, sum of m_i * n_i, is
    smaller. Labels come from the solver's own alpha sweep."""
    from paper_2401_16113_gb300 import alpha_mlp as AM
    train_ps = W.batch_instances(768, seed=101)
    test_ps = W.batch_instances(192, seed=202)
    t0 = time.time()
    h, loss, (a, m, n, its) = AM.train(train_ps, epochs=300, minibatch=256, lr=3e-3, seed=0, tol=1e-8, maxit=200)
    t1 = time.time()
    assert np.isfinite(loss)
    preds = [AM.predict(h, p) for p in test_ps]
    its_default = AM.sweep_iterations(test_ps, alphas=(AM.DEFAULT_ALPHA,), m=AM.DEFAULT_M)[:, 0]
    its_pred = np.full(len(test_ps), np.inf)
    for mv in sorted({m_ for _, m_ in preds}):
        ids = [i for i, (_, m_) in enumerate(preds) if m_ == mv]
        ps = [W.with_(test_ps[i], precision="mixed") for i in ids]
        bt = aao.aao_batch_create(ps, mv)
        bs = [torch.empty(k, dtype=torch.float64, device="cuda") for k in bt.sizes]
        xs = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in bt.sizes]
        aao.aao_batch_rhs(bt, bs)
        aao.aao_batch_set_alpha(bt, [preds[i][0] for i in ids])
        st = aao.batch_submit(bt, bs, xs, 1e-8, 200)
        for i, s in zip(ids, st):
            if s["status"] == 0:
                its_pred[i] = s["iterations"]
        bt.close()
    fallback = ~np.isfinite(its_pred)
    its_pred[fallback] = its_default[fallback]  # a failed prediction falls back to the default
    sizes = np.array([W.unknowns(p) for p in test_ps], dtype=np.float64)
    mem_pred = float(np.sum([m_ for _, m_ in preds] * sizes))
    mem_default = float(np.sum(AM.DEFAULT_M * sizes))
    print(f"sweep+train {t1 - t0:.1f}s; labels alpha {dict(zip(*np.unique(a, return_counts=True)))} "
          f"m {dict(zip(*np.unique(m, return_counts=True)))}; loss {loss:.4f}; held-out mean its: learned "
          f"{its_pred.mean():.3f} default {its_default.mean():.3f}; fallbacks {int(fallback.sum())}; "
          f"workspace learned/default {mem_pred / mem_default:.2f}")
    assert np.all(np.isfinite(its_default))
    assert its_pred.mean() <= its_default.mean() + 0.05
    assert mem_pred <= 0.5 * mem_default
