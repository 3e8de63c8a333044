"""Learned right preconditioner on the GPU: the network, its loss and its gradient against the
oracle, training through the library's kernels, and the right-preconditioned mixed solve, whose
solution must reach a true FP64 residual below 1e-10 recomputed with the oracle's apply."""
import numpy as np
import pytest

import synth
from oracle import precond, wform
from tests.gpu_common import SMALL_CASES, CASE_IDS, to_dev, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")


def _weights(K, seed, scale=0.25):
    rng = np.random.default_rng(seed)
    A = scale * (rng.standard_normal((K, 9, 4, 4)) + 1j * rng.standard_normal((K, 9, 4, 4)))
    for l in range(K):
        A[l, 0] += np.eye(4)
    return A


def _f32(a):
    """The weights as the FP32 network holds them."""
    return (a.real.astype(np.float32) + 1j * a.imag.astype(np.float32)).astype(np.complex128)


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
def test_net_apply_matches_oracle(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 9000 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F32 | ok.W_LINKS)
    A = _weights(4, 9100 + sum(dims))
    net = ok.Net(4, A)
    assert np.array_equal(net.weights, _f32(A))
    psi = synth.gaussian_source(dims, 9200 + sum(dims)).astype(np.complex64)
    got = ok.net_apply(net, W, to_dev(psi)).cpu().numpy()
    exp = precond.apply(U, _f32(A), psi.astype(np.complex128), bc)
    assert rel_l2(got, exp) < 1e-5, rel_l2(got, exp)


@pytest.mark.parametrize("case", SMALL_CASES[:4], ids=CASE_IDS[:4])
def test_net_loss_and_gradient_match_oracle(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 9300 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F32 | ok.W_LINKS)
    A = _weights(3, 9400 + sum(dims), 0.2)
    net = ok.Net(3, A)
    b = synth.gaussian_source(dims, 9500 + sum(dims)).astype(np.complex64)
    x = synth.gaussian_source(dims, 9600 + sum(dims)).astype(np.complex64)
    loss, grad = ok.net_loss_grad(net, W, to_dev(b), to_dev(x))
    eloss, egrad = precond.loss_and_grad(U, _f32(A), b.astype(np.complex128), x.astype(np.complex128), bc)
    assert abs(loss - eloss) < 1e-5 * eloss
    assert rel_l2(grad, egrad) < 1e-4, rel_l2(grad, egrad)


def test_identity_network_leaves_the_solve_unchanged():
    dims, bc = (6, 5, 4, 8), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.3, 9701)
    c = synth.placeholder_coeffs(0.6)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32 | ok.W_LINKS)
    b = to_dev(synth.gaussian_source(dims, 9702))
    net = ok.Net(2)
    x1, i1 = ok.bicgstab_net(W, net, b, tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-2)
    x2, i2 = ok.bicgstab(W, b, tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-2)
    assert i1["iters"] == i2["iters"]
    assert rel_l2(x1.cpu().numpy(), x2.cpu().numpy()) < 1e-9
    r = np.linalg.norm(b.cpu().numpy() - wform.apply(U, c, x1.cpu().numpy(), bc)) / np.linalg.norm(b.cpu().numpy())
    assert r < 1e-10


def test_preconditioned_solve_is_independent_of_the_check_cadence():
    """The network's layers, like the other kernels of an iteration enqueued after the state
    halted, change nothing: the preconditioned solve is bit-identical for any check_every."""
    dims, bc = (6, 4, 4, 6), (1, 1, 1, 1)
    U = synth.random_links(dims, 0.3, 9721)
    c = synth.placeholder_coeffs(0.5)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32 | ok.W_LINKS)
    b = to_dev(synth.gaussian_source(dims, 9722))
    net = ok.Net(2, _weights(2, 9723, 0.05))
    runs = [ok.bicgstab_net(W, net, b, tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-2, check_every=ce) for ce in (1, 4, 7)]
    x0, i0 = runs[0]
    assert i0["status"] == 0
    r = np.linalg.norm(b.cpu().numpy() - wform.apply(U, c, x0.cpu().numpy(), bc)) / np.linalg.norm(b.cpu().numpy())
    assert r < 1e-10
    for x, i in runs[1:]:
        assert torch.equal(x, x0) and i["iters"] == i0["iters"]


def test_training_lowers_the_loss_and_the_trained_preconditioner_solves():
    """Train on pairs from our own solver over three synthetic fields, then solve a held-out field."""
    dims, bc = (8, 8, 8, 8), (1, 1, 1, 1)
    c = synth.placeholder_coeffs(0.5)
    fields = []
    for f in range(4):
        U = synth.random_links(dims, 0.1 + 0.1 * f / 3, 9800 + f)
        W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32 | ok.W_LINKS)
        fields.append((U, W))
    pairs = []
    for U, W in fields[:3]:
        bs = torch.stack([to_dev(synth.gaussian_source(dims, 9900 + 17 * len(pairs) + k)) for k in range(8)])
        xs, _ = ok.bicgstab_multi(W, bs, tol=1e-8, mode=ok.SOLVE_MIXED, delta=1e-2)
        pairs.append((W, bs.to(torch.complex64), xs.to(torch.complex64)))
    net = ok.Net(4)
    first = None
    for step in range(150):
        W, bs, xs = pairs[step % 3]
        loss = ok.net_train_step(net, W, bs, xs, lr=1e-2 if step < 100 else 3e-3)
        if first is None:
            first = loss
    losses = [ok.net_loss_grad(net, W, bs[k].contiguous(), xs[k].contiguous())[0] for W, bs, xs in pairs for k in range(2)]
    assert max(losses) < 0.5 * first, (first, losses)
    # held-out field
    U, W = fields[3]
    b = to_dev(synth.gaussian_source(dims, 9990))
    x, info = ok.bicgstab_net(W, net, b, tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-2)
    _, plain = ok.bicgstab(W, b, tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-2)
    r = np.linalg.norm(b.cpu().numpy() - wform.apply(U, c, x.cpu().numpy(), bc)) / np.linalg.norm(b.cpu().numpy())
    assert info["status"] == 0 and r < 1e-10, (info, r)
    assert info["iters"] < plain["iters"], (info["iters"], plain["iters"])


def test_net_argument_errors():
    dims = (4, 4, 4, 4)
    U = to_dev(synth.random_links(dims, 0.3, 9991))
    c = synth.placeholder_coeffs(0.5)
    W = ok.precompute_W(U, c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32)       # no links copy
    WL = ok.precompute_W(U, c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32 | ok.W_LINKS)
    net = ok.Net(2)
    psi = to_dev(synth.gaussian_source(dims, 9992).astype(np.complex64))
    with pytest.raises(ok.OKError):
        ok.net_apply(net, W, psi)
    b = to_dev(synth.gaussian_source(dims, 9993))
    with pytest.raises(ok.OKError):                 # the network runs in the FP32 iteration only
        ok.bicgstab_net(WL, net, b, mode=ok.SOLVE_F64)
    with pytest.raises(ValueError):
        ok.Net(2, np.zeros((3, 9, 4, 4)))
    bad = np.zeros((2, 9, 4, 4), dtype=np.complex128)
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(ok.OKError):
        net.weights = bad
    with pytest.raises(ok.OKError):
        ok.precompute_W(U, c, (1, 1, 1, 1), ok.W_LINKS)   # links alone: no W copy


def test_multi_rhs_solve_with_the_network():
    """The multi-RHS solve right-preconditioned by the network: the identity network changes
    nothing, a trained one cuts the iterations, and every system reaches 1e-10 (oracle apply)."""
    dims, bc = (8, 8, 8, 8), (1, 1, 1, 1)
    c = synth.placeholder_coeffs(0.5)
    U = synth.random_links(dims, 0.2, 9601)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32 | ok.W_F16 | ok.W_LINKS)
    V = int(np.prod(dims))
    b = torch.zeros((12, V, 12), dtype=torch.complex128, device="cuda")
    for k in range(12):
        b[k, 5, k] = 1.0
    b = b.reshape((12,) + synth.lattice_shape(dims) + (4, 3))
    x0, i0 = ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-2)
    x1, i1 = ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-2, net=ok.Net(2))
    assert [i["iters"] for i in i0] == [i["iters"] for i in i1]
    # a network trained on Gaussian pairs of two other fields
    net = ok.Net(4)
    pairs = []
    for f in range(2):
        Uf = synth.random_links(dims, 0.15 + 0.1 * f, 9610 + f)
        Wf = ok.precompute_W(to_dev(Uf), c, bc, ok.W_F64 | ok.W_F32 | ok.W_LINKS)
        bs = torch.stack([to_dev(synth.gaussian_source(dims, 9620 + 12 * f + k)) for k in range(12)])
        xs, _ = ok.bicgstab_multi(Wf, bs, tol=1e-8, mode=ok.SOLVE_MIXED, delta=1e-2)
        pairs.append((Wf, bs.to(torch.complex64), xs.to(torch.complex64)))
    for step in range(120):
        Wf, bs, xs = pairs[step % 2]
        j = 4 * ((step // 2) % 3)
        ok.net_train_step(net, Wf, bs[j:j + 4], xs[j:j + 4], lr=1e-2 if step < 80 else 3e-3)
    x2, i2 = ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-2, net=net)
    assert max(i["iters"] for i in i2) < min(i["iters"] for i in i0), ([i["iters"] for i in i2], [i["iters"] for i in i0])
    xs2, bs = x2.cpu().numpy(), b.cpu().numpy()
    for k in (0, 6, 11):
        r = np.linalg.norm(bs[k] - wform.apply(U, c, xs2[k], bc)) / np.linalg.norm(bs[k])
        assert i2[k]["true_relres"] < 1e-10 and r < 1e-10, (k, r)
    with pytest.raises(ok.OKError):            # the handle needs the links copy
        W2 = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F16)
        ok.bicgstab_multi(W2, b, mode=ok.SOLVE_MIXED16, net=net)
