"""Batched persistent solver (one launch, one CTA per instance) against the FP64 oracle and
against single-instance solves; failure isolation between instances."""
import numpy as np
import pytest

from oracle import aao_oracle as O
from paper_2401_16113_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aao():
    from paper_2401_16113_gb300 import aao as A, build
    build.build()
    A.load()
    return A


def small_batch(n=24, seed=7):
    return W.batch_instances(n, seed=seed, nx_choices=(31, 63, 127), nt_choices=(16, 32, 64), m=20)


def vectors(bt, fill=0.0):
    return [torch.full((n,), fill, dtype=torch.float64, device="cuda") for n in bt.sizes]


def test_batch_matches_oracle_and_sequential_cn(aao):
    ps = small_batch()
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-10, 200)
    torch.cuda.synchronize()
    for i, p in enumerate(ps):
        assert st[i]["status"] == 0 and st[i]["rel_residual"] <= 1e-10, (i, st[i])
        b_ref = O.assemble_b(p)
        assert np.abs(bs[i].cpu().numpy() - b_ref).max() <= 1e-13 * np.abs(b_ref).max()
        x = xs[i].cpu().numpy()
        M = O.assemble_M(p)
        assert np.linalg.norm(b_ref - M @ x) <= 1.01e-10 * np.linalg.norm(b_ref)
        U = O.sequential_cn(p)
        assert np.abs(x - U.ravel()).max() <= 1e-7 * np.abs(U).max(), i
    bt.close()


def test_batch_agrees_with_single_instance_solves(aao):
    ps = small_batch(8, seed=11)
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-9, 200)
    for i, p in enumerate(ps):
        h = aao.aao_create(p)
        x1 = torch.zeros_like(xs[i])
        s1 = aao.fgmres_solve(h, bs[i], x1, 1e-9, 20, 200)
        assert abs(s1["iterations"] - st[i]["iterations"]) <= 1, (s1, st[i])
        torch.cuda.synchronize()
        a, b = xs[i].cpu().numpy(), x1.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()
        h.close()
    bt.close()


def test_batch_size_limits_agree_with_single_instance_solves(aao):
    """Instances at the batched solver's limits (nx = nt = 4096: 256 threads per tridiagonal bin,
    a one-column FFT tile; nx = 4095 with nt = 64; the smallest 2 x 2) in one launch, each against
    its single-instance solve and the true FP64 residual."""
    base = W.bs_put_255x256()
    ps = [W.with_(base, nx=4096, nt=4096, precision="mixed", alpha=1e-3, tol=1e-8, m=20, s_max=300.0),
          W.with_(base, nx=4095, nt=64, precision="mixed", payoff="call", alpha=1e-3, tol=1e-8, m=20),
          W.with_(base, nx=2, nt=2, precision="mixed", alpha=1e-3, tol=1e-8, m=20)]
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-8, 300)
    for i, p in enumerate(ps):
        assert st[i]["status"] == 0, (i, st[i])
        h = aao.aao_create(p)
        x1 = torch.zeros_like(xs[i])
        s1 = aao.fgmres_solve(h, bs[i], x1, 1e-8, 20, 300)
        assert s1["status"] == 0 and abs(s1["iterations"] - st[i]["iterations"]) <= 1, (s1, st[i])
        r = torch.empty_like(xs[i])
        aao.aao_matvec(h, xs[i], r)
        torch.cuda.synchronize()
        res = float(torch.linalg.norm(bs[i] - r) / torch.linalg.norm(bs[i]))
        assert res <= 1.01e-8, (i, res)
        a, b = xs[i].cpu().numpy(), x1.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), i
        h.close()
    bt.close()


def test_batch_failure_is_isolated_and_results_do_not_depend_on_neighbours(aao):
    ps = small_batch(12, seed=3)
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-10, 200)
    clean = [x.cpu().numpy().copy() for x in xs]
    bs[5][3] = float("nan")
    for x in xs:
        x.zero_()
    st2 = aao.batch_submit(bt, bs, xs, 1e-10, 200)
    assert st2[5]["status"] == aao.AAO_BREAKDOWN
    for i in range(len(ps)):
        if i == 5:
            continue
        assert st2[i]["status"] == 0
        assert st2[i]["iterations"] == st[i]["iterations"]
        assert np.array_equal(xs[i].cpu().numpy(), clean[i]), i
    bt.close()


def test_batch_maxit_and_replay(aao):
    ps = small_batch(6, seed=5)
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-14, 1)
    assert all(s["status"] == aao.AAO_NOT_CONVERGED and s["iterations"] == 1 for s in st)
    for x in xs:
        x.zero_()
    st_a = aao.batch_submit(bt, bs, xs, 1e-10, 200)
    first = [x.cpu().numpy().copy() for x in xs]
    for x in xs:
        x.zero_()
    st_b = aao.batch_submit(bt, bs, xs, 1e-10, 200)
    for i in range(len(ps)):
        assert st_a[i]["iterations"] == st_b[i]["iterations"]
        assert np.array_equal(first[i], xs[i].cpu().numpy())
    bt.close()


def test_batch_distribution_512_instances(aao):
    """The 512-instance distribution (Nx in {127..1023}, Nt in {64..1024}) to 1e-8; a sample
    of instances checked against the oracle."""
    ps = W.batch_instances(512, m=20)
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-8, 300)
    assert all(s["status"] == 0 and s["rel_residual"] <= 1e-8 for s in st)
    order = np.argsort([W.unknowns(p) for p in ps])
    for i in [int(order[0]), int(order[1]), int(order[len(order) // 2])]:
        p = ps[i]
        x = xs[i].cpu().numpy()
        b_ref = O.assemble_b(p)
        assert np.linalg.norm(b_ref - O.assemble_M(p) @ x) <= 1.01e-8 * np.linalg.norm(b_ref)
    bt.close()


def test_batch_mixed_radix_nt_matches_oracle_and_single_instance(aao):
    """Instances whose nt is not a power of two (prime factors 2, 3, 5, 7) take the mixed-radix FFT
    tiles inside the persistent kernel; mixed with power-of-two instances in one batch, each
    solution is the AaO solution (oracle residual, sequential CN) and agrees with the
    single-instance solver, which takes the stand-alone mixed-radix kernels."""
    ps = W.batch_instances(12, seed=23, nx_choices=(31, 63, 127), nt_choices=(12, 48, 96, 160, 210, 64), m=20)
    assert any(p["nt"] & (p["nt"] - 1) for p in ps)
    bt = aao.aao_batch_create(ps, 20)
    bs, xs = vectors(bt), vectors(bt)
    aao.aao_batch_rhs(bt, bs)
    st = aao.batch_submit(bt, bs, xs, 1e-10, 200)
    torch.cuda.synchronize()
    for i, p in enumerate(ps):
        assert st[i]["status"] == 0 and st[i]["rel_residual"] <= 1e-10, (i, p["nt"], st[i])
        b_ref = O.assemble_b(p)
        x = xs[i].cpu().numpy()
        M = O.assemble_M(p)
        assert np.linalg.norm(b_ref - M @ x) <= 1.01e-10 * np.linalg.norm(b_ref), (i, p["nt"])
        U = O.sequential_cn(p)
        assert np.abs(x - U.ravel()).max() <= 1e-7 * np.abs(U).max(), (i, p["nt"])
        h = aao.aao_create(p)
        x1 = torch.zeros_like(xs[i])
        s1 = aao.fgmres_solve(h, bs[i], x1, 1e-10, 20, 200)
        assert abs(s1["iterations"] - st[i]["iterations"]) <= 1, (p["nt"], s1, st[i])
        h.close()
    bt.close()


def test_batch_rejects_nt_with_a_prime_factor_above_7(aao):
    ps = W.batch_instances(3, seed=5, nx_choices=(31,), nt_choices=(16,), m=20)
    ps[1] = W.with_(ps[1], nt=22)
    with pytest.raises(aao.AaoError) as e:
        aao.aao_batch_create(ps, 20)
    assert e.value.code == aao.AAO_EINVAL
