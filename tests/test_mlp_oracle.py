"""Pins of the FP64 surrogate oracle (CPU): forward and gradient against
torch (float64 autograd, a library routine), the gradient against central
finite differences of the oracle's own forward, the bf16 rounding, and the
exact target P against the closed forms it reduces to."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as M
import sas_workloads as W

torch = pytest.importorskip("torch")


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(M.NPARAM, np.float32)
    p[M.OFF_W1:M.OFF_W2] = rng.uniform(-1, 1, M.OFF_W2 - M.OFF_W1) * np.sqrt(6 / 16) * scale
    p[M.OFF_W2:M.OFF_B1] = rng.uniform(-1, 1, M.OFF_B1 - M.OFF_W2) * np.sqrt(6 / 256) * scale
    p[M.OFF_B1 + 256:M.OFF_W5] = rng.normal(size=768) * 0.1
    p[M.OFF_W5:M.OFF_B5] = rng.uniform(-1, 1, 256) * 0.1
    p[M.OFF_B5] = -2.0
    return p


def _features(n, seed=1):
    box = W.surrogate_box()
    rng = np.random.default_rng(seed)
    q = box["q_max"] * np.sqrt(rng.random(n))
    ca = rng.random(n)
    raw = np.stack([q * ca, q * np.sqrt(1 - ca ** 2), rng.uniform(15, 25, n), rng.uniform(300, 500, n),
                    rng.uniform(box["sigma_orient_min"], box["sigma_orient_max"], n),
                    rng.uniform(0.05, 0.15, n)], 1)
    return box, raw, M.features(box, raw)


def _torch_net(p, X, rnd):
    W1, Ws, bs, w5, b5 = [torch.tensor(np.asarray(a, dtype=np.float64)) if not isinstance(a, list) else
                          [torch.tensor(np.asarray(x, dtype=np.float64)) for x in a] for a in M.unpack(p)]
    Wl = [W1] + Ws
    for t in Wl + bs + [w5]:
        t.requires_grad_(True)
    b5 = torch.tensor(float(b5), dtype=torch.float64, requires_grad=True)

    def r(x):   # straight-through rounding
        return x + (torch.tensor(rnd(x.detach().numpy())) - x).detach()

    a = r(torch.tensor(X))
    for l in range(4):
        a = r(torch.nn.functional.silu(torch.nn.functional.linear(a, r(Wl[l]), bs[l])))
    out = a @ w5 + b5
    return out, Wl, bs, w5, b5


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159265, 0.0, 65504.0, 1e-40], np.float32)
    got = M.bf16(x)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, ref)


def test_forward_matches_torch():
    p = _params()
    box, raw, X = _features(300)
    out = M.forward(p, X)
    t, *_ = _torch_net(p, X, M.bf16)
    assert np.max(np.abs(out - t.detach().numpy())) < 1e-10


def test_gradient_matches_torch_autograd():
    p = _params(3)
    box, raw, X = _features(200, 5)
    y = np.random.default_rng(7).normal(size=200) - 3.0
    loss, g = M.loss_and_grad(p, X, y)
    out, Wl, bs, w5, b5 = _torch_net(p, X, M.bf16)
    L = torch.mean((out - torch.tensor(y)) ** 2)
    L.backward()
    assert abs(loss - L.item()) < 1e-10
    offs = [M.OFF_W1, M.OFF_W2, M.OFF_W3, M.OFF_W4]
    for l in range(4):
        ref = Wl[l].grad.numpy().reshape(-1)
        assert np.max(np.abs(g[offs[l]:offs[l] + ref.size] - ref)) < 1e-10 * max(1, np.abs(ref).max())
        assert np.max(np.abs(g[M.OFF_B1 + 256 * l:M.OFF_B1 + 256 * (l + 1)] - bs[l].grad.numpy())) < 1e-10
    assert np.max(np.abs(g[M.OFF_W5:M.OFF_B5] - w5.grad.numpy())) < 1e-10
    assert abs(g[M.OFF_B5] - b5.grad.item()) < 1e-10


def test_gradient_matches_finite_differences():
    """Central differences of the oracle's forward (no rounding) at random
    parameters of every tensor."""
    p = _params(11).astype(np.float64)
    box, raw, X = _features(64, 13)
    y = np.random.default_rng(2).normal(size=64) - 2.0
    ident = M._ident
    _, g = M.loss_and_grad(p, X, y, rnd=ident)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.integers(M.OFF_W1, M.OFF_W2, 6), rng.integers(M.OFF_W2, M.OFF_B1, 12),
                          M.OFF_B1 + 256 + rng.integers(0, 768, 6), rng.integers(M.OFF_W5, M.OFF_B5, 4),
                          [M.OFF_B5]])
    X[:, 63] = 1.0
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, X, y, rnd=ident)[0] - M.loss_and_grad(pm, X, y, rnd=ident)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_features_definition():
    box = W.surrogate_box(n_fourier=2)
    raw = np.array([[0.1, 0.05, 20.0, 400.0, np.radians(15.0), 0.1]])
    F = M.features(box, raw)
    u, v, a = 0.1 * 200.0, 0.05 * 20.0, 10.0
    a_min, a_max = 0.5 * box["l_min"] / box["r_max"], 0.5 * box["l_max"] / box["r_min"]
    assert abs(F[0, 0] - (2 * u / (0.5 * box["q_max"] * box["l_max"]) - 1)) < 1e-15
    assert abs(F[0, 1] - (2 * v / (box["q_max"] * box["r_max"]) - 1)) < 1e-15
    assert abs(F[0, 2] - (2 * np.log(a / a_min) / np.log(a_max / a_min) - 1)) < 1e-12
    assert abs(F[0, 3]) < 1e-12 and abs(F[0, 4]) < 1e-12      # the box centre
    assert abs(F[0, 5] - (np.log(1 + u * u) / 4 - 1)) < 1e-15
    assert abs(F[0, 6] - (np.log(1 + v * v) / 4 - 1)) < 1e-15
    assert abs(F[0, 7] - (np.log(1 + (0.1 * 20.0) ** 2) / 4 - 1)) < 1e-15   # (u / a)^2 = (q_par R)^2
    # u pairs k = 1, 2 at columns 8..11, v pairs at 12..15
    assert abs(F[0, 8] - np.sin(u / 2)) < 1e-15 and abs(F[0, 9] - np.cos(u / 2)) < 1e-15
    assert abs(F[0, 10] - np.sin(u)) < 1e-15 and abs(F[0, 11] - np.cos(u)) < 1e-15
    assert abs(F[0, 12] - np.sin(v / 2)) < 1e-15 and abs(F[0, 15] - np.cos(v)) < 1e-15
    assert F[0, 63] == 1.0 and np.all(F[0, 16:63] == 0)


def test_exact_pbar_closed_forms():
    """The surrogate's target P reduces to closed forms: 1 at Q = 0 for both
    bodies; for a monodisperse ellipsoid with R_p = R (L = 2R), the sphere's
    (3 (sin x - x cos x) / x^3)^2 at x = |Q| R whatever the axis spread; for
    a monodisperse cylinder with an axis spread of 1e-5 rad, the aligned
    cylinder's (2 J1(q_perp R) / (q_perp R))^2 sinc(q_par L / 2)^2."""
    from scipy.special import j1
    oracle.build()
    R, L = 37.0, 150.0
    ebox = W.batched_ellipsoid_surrogate_box(n_fourier=4, n_buckets=8)
    ebox.update(n_poly=12, n_gamma=16, n_psi=16)
    raw = np.array([[0.0, 0.0, R, 2 * R, math.radians(10), 0.0, 0, 0],
                    [0.05, 0.03, R, 2 * R, math.radians(10), 0.0, 0, 0],
                    [0.01, 0.09, R, 2 * R, math.radians(25), 0.0, 0, 0]])
    x = np.hypot(raw[:, 0], raw[:, 1]) * R
    with np.errstate(all="ignore"):
        ref = np.where(x > 0, (3 * (np.sin(x) - x * np.cos(x)) / x ** 3) ** 2, 1.0)
    assert np.allclose(M.exact_pbar(ebox, raw), ref, rtol=1e-12, atol=0)
    cbox = W.batched_surrogate_box(n_fourier=4, n_buckets=8)
    cbox.update(n_poly=12, n_gamma=16, n_psi=16)
    raw = np.array([[0.0, 0.0, R, L, 1e-5, 0.0, 0, 0],
                    [0.0, 0.06, R, L, 1e-5, 0.0, 0, 0],
                    [0.02, 0.05, R, L, 1e-5, 0.0, 0, 0]])
    x, y = raw[:, 1] * R, raw[:, 0] * L / 2
    with np.errstate(all="ignore"):
        ref = (np.where(x > 0, 2 * j1(x) / x, 1.0) * np.where(y > 0, np.sin(y) / y, 1.0)) ** 2
    assert np.allclose(M.exact_pbar(cbox, raw), ref, rtol=1e-8, atol=0)
