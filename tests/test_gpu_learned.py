"""Learned level-0 smoother on the GPU (features, patch-inverse targets,
BF16/FP32 MLP forward and backward, Adam training, Lanczos damping) against
the FP64 oracle (oracle/learned.py).

Tolerances: features 1e-6 relative (FP64 arithmetic, FP32 output); targets
1e-10 (FP64); network outputs 2e-5 relative to their norm and 1e-4 element by element,
loss and gradient 2e-3 relative to their norm (gradient blocks also 1e-2
element by element) (FP32 accumulation; the oracle evaluates the same
BF16-rounded weights in FP64); V-cycle with the installed blocks 1e-10
element by element; the trained network must take fewer PCG iterations than
block-l1 Jacobi.
"""
import copy

import numpy as np
import pytest

from oracle import hierarchy, learned, solve
from workloads import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _amg():
    from paper_2011_13325_gb300 import amg
    return amg


_CASE = {}


def case():
    """A 9x8x7 box with per-element nu (3 levels), its oracle hierarchy and a
    context holding that hierarchy."""
    if not _CASE:
        p = make_problem((9, 8, 7), seed=41, nu_range=(0.3, 0.45))
        H = hierarchy.setup(p)
        _CASE.update(p=p, H=H, x=p.coords[p.free])
    return _CASE


def _ctx(prec=0):
    amg = _amg()
    c = case()
    ctx = amg.Context(0)
    ctx.upload_hierarchy(c["H"].A[0], c["H"].P, prec)
    return ctx


def _dev_features(ctx, x, n):
    X = torch.zeros((n, 13), dtype=torch.float32, device="cuda")
    tr = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.learned_features(x, X, tr)
    return X, tr


def test_features_match_oracle():
    c = case()
    ctx = _ctx()
    n = c["H"].A[0].n_rows
    X, tr = _dev_features(ctx, c["x"], n)
    Xo, tro = learned.features(c["H"].A[0], c["x"])
    assert np.abs(X.cpu().numpy() - Xo).max() <= 1e-6 * max(1.0, np.abs(Xo).max())
    assert np.allclose(tr.cpu().numpy(), tro, rtol=1e-14)


def test_patch_targets_match_oracle():
    c = case()
    ctx = _ctx()
    n = c["H"].A[0].n_rows
    T64 = torch.zeros((n, 9), dtype=torch.float64, device="cuda")
    T32 = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    ctx.learned_targets(T32, T64)
    To = learned.targets(c["H"].A[0]).reshape(n, 9)
    assert np.abs(T64.cpu().numpy() - To).max() <= 1e-10 * np.abs(To).max()
    assert np.allclose(T32.cpu().numpy(), To, rtol=1e-6, atol=1e-6 * np.abs(To).max())


def _data(ctx, c):
    n = c["H"].A[0].n_rows
    X, _ = _dev_features(ctx, c["x"], n)
    T = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    ctx.learned_targets(T32=T)
    return X, T


def test_forward_loss_and_gradient_match_oracle():
    amg = _amg()
    c = case()
    ctx = _ctx()
    X, T = _data(ctx, c)
    net = amg.Mlp(0, seed=3)
    w = net.params(working=True).astype(np.float64)
    # the BF16 working copy is the master rounded to nearest
    m = net.params()
    assert np.all(np.abs(w - m) <= 2.0 ** -8 * np.abs(m) + 1e-30)
    Xh = X.cpu().numpy().astype(np.float64)
    Th = T.cpu().numpy().astype(np.float64).reshape(-1, 3, 3)
    out = torch.zeros((X.shape[0], 6), dtype=torch.float32, device="cuda")
    net.infer(X, out)
    out_o, _ = learned.forward(w, Xh)
    oh = out.cpu().numpy()
    assert np.linalg.norm(oh - out_o) <= 2e-5 * np.linalg.norm(out_o)
    # element by element: every output within 1e-4 of the largest
    assert np.abs(oh - out_o).max() <= 1e-4 * np.abs(out_o).max()
    loss, g = net.loss_grad(X, T)
    loss_o, g_o = learned.loss_grad(w, Xh, Th)
    assert abs(loss - loss_o) <= 2e-3 * loss_o
    assert np.linalg.norm(g - g_o) <= 2e-3 * np.linalg.norm(g_o)
    # every parameter block, not only the large ones
    for name, sl in (("W1", slice(0, 832)), ("b1", slice(832, 896)), ("W2", slice(896, 4992)),
                     ("b2", slice(4992, 5056)), ("W3", slice(5056, 5440)), ("b3", slice(5440, 5446))):
        assert np.linalg.norm(g[sl] - g_o[sl]) <= 5e-3 * np.linalg.norm(g_o[sl]) + 1e-12, name
        assert np.abs(g[sl] - g_o[sl]).max() <= 1e-2 * np.abs(g_o[sl]).max() + 1e-12, name


def test_training_reduces_loss_deterministically():
    amg = _amg()
    c = case()
    ctx = _ctx()
    X, T = _data(ctx, c)
    nets = [amg.Mlp(0, seed=5) for _ in range(2)]
    l0, _ = nets[0].loss_grad(X, T)
    hists = [n.train(X, T, epochs=30, batch=128, lr=2e-3, seed=9) for n in nets]
    l1, _ = nets[0].loss_grad(X, T)
    assert l1 < 0.3 * l0, (l0, l1, hists[0])
    assert np.array_equal(hists[0], hists[1])
    assert np.array_equal(nets[0].params(), nets[1].params())


def test_learned_smoother_installs_damped_spd_blocks():
    amg = _amg()
    c = case()
    H = c["H"]
    ctx = _ctx()
    net = amg.Mlp(0, seed=11)
    lam, w = ctx.set_learned_smoother(net, c["x"])
    theta = net.params(working=True).astype(np.float64)
    Xo, tro = learned.features(H.A[0], c["x"])
    B = learned.smoother_blocks(theta, Xo, tro)
    lam_full = learned.lanczos_lambda_max(H.A[0], B, steps=300)
    assert lam <= lam_full * (1 + 1e-6) and lam >= 0.9 * lam_full
    assert abs(w - 4.0 / (3.0 * 1.05 * lam)) <= 1e-12 * w
    M = ctx.download_smoother(0)
    assert np.abs(M - w * B).max() <= 1e-4 * np.abs(w * B).max()
    # the V-cycle stays symmetric positive definite, PCG reaches 1e-8
    rng = np.random.default_rng(1)
    n = H.A[0].n_rows * 3
    a, b = rng.normal(size=(2, n))
    za = torch.zeros(n, dtype=torch.float64, device="cuda")
    zb = torch.zeros_like(za)
    ctx.vcycle(torch.from_numpy(a).cuda(), za)
    ctx.vcycle(torch.from_numpy(b).cuda(), zb)
    za, zb = za.cpu().numpy(), zb.cpu().numpy()
    assert abs(b @ za - a @ zb) <= 1e-10 * abs(a @ za) and a @ za > 0 and b @ zb > 0
    # the GPU V-cycle equals the oracle V-cycle with the installed blocks
    H2 = copy.copy(H)
    H2.Minv = list(H.Minv)
    H2.Minv[0] = M
    zo = solve.vcycle(H2, a)
    assert np.abs(za - zo).max() <= 1e-10 * np.abs(zo).max()
    f = c["p"].b[0]
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    s, its, rr = ctx.pcg_solve(torch.from_numpy(f).cuda(), u, rtol=1e-8, maxit=2000)
    uh = u.cpu().numpy()
    assert np.linalg.norm(f - solve.spmv(H.A[0], uh)) <= 1.5e-8 * np.linalg.norm(f)
    # back to block-l1 Jacobi
    ctx.reset_smoother()
    assert np.abs(ctx.download_smoother(0) - H.Minv[0]).max() <= 1e-10 * np.abs(H.Minv[0]).max()


def test_trained_smoother_gain_over_block_l1_jacobi():
    """Train on patch inverses of three 12^3 meshes (the library's own
    setup and kernels), apply to an unseen 14^3 mesh: the learned V-cycle
    stays SPD and convergent; its PCG iterations are compared with the
    method's block-l1 Jacobi on the same hierarchy, in FP64 and with the
    FP32 V-cycle."""
    amg = _amg()
    Xs, Ts = [], []
    for seed in (100, 101, 102):
        p = make_problem((12, 12, 12), seed=seed, nu_range=(0.3, 0.45))
        cx = amg.Context(0)
        cx.setup(p)
        n = cx.level_info(0)["n_rows"]
        X = torch.zeros((n, 13), dtype=torch.float32, device="cuda")
        T = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
        cx.learned_features(p.coords[p.free], X)
        cx.learned_targets(T32=T)
        Xs.append(X)
        Ts.append(T)
        cx.close()
    X, T = torch.cat(Xs), torch.cat(Ts)
    net = amg.Mlp(0, seed=1)
    l0, _ = net.loss_grad(X, T)
    hist = net.train(X, T, epochs=60, batch=256, lr=2e-3, seed=2)
    assert hist[-1] < 0.1 * l0
    p = make_problem((14, 14, 14), seed=7, nu_range=(0.3, 0.45))
    f = torch.from_numpy(p.b[0]).cuda()
    out = {}
    for prec in (0, 1):
        ctx = amg.Context(0)
        ctx.setup(p, prec)
        u = torch.zeros_like(f)
        _, it_l1, _ = ctx.pcg_solve(f, u, rtol=1e-8)
        lam, w = ctx.set_learned_smoother(net, p.coords[p.free])
        u.zero_()
        s, it_ln, rr = ctx.pcg_solve(f, u, rtol=1e-8)
        r = torch.empty_like(f)
        ctx.residual(0, f, u, r)
        assert float(torch.linalg.norm(r) / torch.linalg.norm(f)) <= 1.5e-8
        out[prec] = (it_l1[0], it_ln[0])
        ctx.close()
    print("iterations (block-l1 Jacobi, learned):", out)
    for prec, (a, b) in out.items():
        assert b < a, out     # a strict gain in both precisions
