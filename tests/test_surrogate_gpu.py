"""Learned surrogate on the tensor cores (GPU) against the FP64 oracle.

* forward (tcgen05 inference) vs the oracle network on the same weights,
  per element within a bound derived from the arithmetic (below);
* exact training targets vs the trace oracle's quadrature;
* gradients (tcgen05 backward + weight-gradient GEMMs + row sums) vs the
  oracle's backpropagation on the same BF16 weights, element by element:
  |g - g_oracle| <= 1e-2 |g_oracle| + 1e-3 m, m the element's L1 mass (the
  sum of the magnitudes of the per-sample terms it adds up), so that an
  element whose terms cancel is held to an absolute floor set by its terms;
* training lowers the loss; the trace uses the surrogate inside its box and
  the exact quadrature outside.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as M
import paper_2501_06054_gb300 as sas
import sas_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _small_box(n_fourier=4):
    b = W.surrogate_box(n_fourier=n_fourier, n_buckets=8)
    b.update(n_poly=12, n_gamma=16, n_psi=16)
    return b


def _raw(box, n, seed):
    rng = np.random.default_rng(seed)
    q = box["q_max"] * np.sqrt(rng.random(n))
    ca = rng.random(n)
    sp_b = np.array([box["poly_min"] + (box["poly_max"] - box["poly_min"]) * k / (box["n_buckets"] - 1)
                     for k in range(box["n_buckets"])], np.float32)
    bk = rng.integers(0, box["n_buckets"], n)
    raw = np.zeros((n, 8), np.float32)
    raw[:, 0] = q * ca
    raw[:, 1] = q * np.sqrt(1 - ca ** 2)
    raw[:, 2] = rng.uniform(box["r_min"], box["r_max"], n)
    raw[:, 3] = rng.uniform(box["l_min"], box["l_max"], n)
    raw[:, 4] = rng.uniform(box["sigma_orient_min"], box["sigma_orient_max"], n)
    raw[:, 5] = sp_b[bk]
    raw[:, 6] = bk
    return raw


# Forward tolerance. The kernel and the oracle multiply the same BF16
# weights; they differ in (a) the features (FP32 vs FP64 before rounding to
# BF16), (b) SiLU, which the kernel takes as z/2 (1 + tanh(z/2)) with the
# special-function unit's tanh.approx.f32 (relative error below 2^-11;
# 2^-10.5 is allowed here), (c) FP32 accumulation of the K = 256 products.
# Each layer rounds its activations to BF16 on both sides, so a deviation
# d << ulp of an activation either vanishes (both round alike) or becomes
# one BF16 ulp (a rounding flip), with probability E|d| / ulp. First-order
# propagation of these independent flips through the network (variances
# through W o W, SiLU' on the way) gives a per-sample standard deviation
# sigma of the output; the test requires |out - out_oracle| <= 6 sigma +
# 2e-6 (1 + |out|) for every sample, and a median of |out - out_oracle| /
# sigma below 1 (a numpy emulation of the kernel's roundings gives 0.4 with
# a largest ratio of 3).
TANH_REL = 2.0 ** -10.5


def _bf16_ulp(h):
    a = np.abs(h)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 2.0 ** -133)


def _flip_var(s, h):
    """Variance of bf16(h + d) - bf16(h) for a deviation d of std s."""
    u = _bf16_ulp(h)
    return np.minimum(1.0, math.sqrt(2.0 / math.pi) * s / u) * u * u + s * s


def _forward_sigma(box, p, raw):
    raw = np.asarray(raw, dtype=np.float64)
    X = M.features(box, raw)
    W1, Ws, bs, w5, _ = M.unpack(p)
    Wl = [M.bf16(W1)] + [M.bf16(W) for W in Ws]
    eps = 2.0 ** -24
    # (a) FP32 features: a few roundings of the scaled inputs; the Fourier
    # pair k carries the FP32 phase error of k u / 2 and its recurrence
    s0 = 4 * eps * (np.abs(X) + 1.0)
    s0[:, 2] = 2.0 ** -19                    # ln a by the special-function unit's log2
    s0[:, 5:8] = 2.0 ** -20                  # the three logarithmic envelopes
    u = 0.5 * raw[:, 0] * raw[:, 3]
    v = raw[:, 1] * raw[:, 2]
    n = box["n_fourier"]
    for t, x in enumerate((u, v)):
        for k in range(n):
            sk = (k + 1) * (0.5 * x * 4 * eps + 4 * eps)
            c = M.FOURIER0 + 2 * (t * n + k)
            s0[:, c] = sk
            s0[:, c + 1] = sk
    s0[:, 63] = 0.0
    a = M.bf16(X)
    vD = _flip_var(s0, X)
    for l in range(4):
        z = a @ Wl[l].T + bs[l]
        acc = 256 * eps * (np.abs(a) @ np.abs(Wl[l]).T)          # (c)
        vz = vD @ (Wl[l] ** 2).T + acc * acc / 3.0
        tau = 0.5 * np.abs(z) * TANH_REL * np.abs(np.tanh(0.5 * z))   # (b)
        h = M.silu(z)
        vh = M.dsilu(z) ** 2 * vz + tau * tau
        a = M.bf16(h)
        vD = _flip_var(np.sqrt(vh), h)
    acc = 256 * eps * (np.abs(a) @ np.abs(w5))
    return np.sqrt(vD @ (w5 ** 2) + acc * acc / 3.0)


def test_surrogate_forward_matches_oracle():
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=7, stream=torch.cuda.current_stream())
    n_params = sas.sas_surrogate_info(s)["n_params"]
    assert n_params == M.NPARAM
    p = sas.sas_surrogate_get_params(s, n_params)
    # give the output layer and biases some weight so the check is not trivial
    rng = np.random.default_rng(1)
    p[M.OFF_W5:M.OFF_B5] = rng.uniform(-1, 1, 256).astype(np.float32) * 0.3
    p[M.OFF_B1 + 256:M.OFF_W5] = rng.normal(size=768).astype(np.float32) * 0.1
    p[M.OFF_B5] = -1.5
    sas.sas_surrogate_set_params(s, p)
    n = 1000                                    # 7 full tiles and a ragged one
    raw = _raw(box, n, 3)
    rd = torch.tensor(raw, device="cuda")
    out = torch.empty(n, device="cuda")
    sas.sas_surrogate_eval(s, rd, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = M.forward(p, M.features(box, raw.astype(np.float64)))
    err = np.abs(got - ref)
    sig = _forward_sigma(box, p, raw)
    bound = 6.0 * sig + 2e-6 * (1.0 + np.abs(ref))
    assert np.all(err <= bound), (float(np.max(err / bound)), float(np.median(err)), float(np.median(sig)))
    # and the deviations are of the size the flip model predicts, not larger
    assert np.median(err / sig) < 1.0, float(np.median(err / sig))
    sas.sas_destroy_surrogate(s)


def test_exact_targets_match_oracle():
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=1, stream=torch.cuda.current_stream())
    raw = _raw(box, 97, 11)
    raw[0, :2] = 0.0                            # Q = 0
    rd = torch.tensor(raw, device="cuda")
    out = torch.empty(97, device="cuda")
    sas.sas_surrogate_exact(s, rd, 97, out)
    torch.cuda.synchronize()
    got = np.exp(out.cpu().numpy().astype(np.float64))
    ref = np.maximum(M.exact_pbar(box, raw), M.TARGET_FLOOR)
    assert abs(ref[0] - 1.0) < 1e-12
    assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-7), np.max(np.abs(got - ref) / ref)
    sas.sas_destroy_surrogate(s)


def test_exact_targets_full_grid():
    box = W.surrogate_box()
    s = sas.sas_create_surrogate(box, seed=1, stream=torch.cuda.current_stream())
    raw = _raw(box, 3, 5)
    rd = torch.tensor(raw, device="cuda")
    out = torch.empty(3, device="cuda")
    sas.sas_surrogate_exact(s, rd, 3, out)
    torch.cuda.synchronize()
    got = np.exp(out.cpu().numpy().astype(np.float64))
    ref = np.maximum(M.exact_pbar(box, raw), M.TARGET_FLOOR)
    assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-7)
    sas.sas_destroy_surrogate(s)


def test_generated_dataset_is_consistent():
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=1, stream=torch.cuda.current_stream())
    sas.sas_surrogate_generate(s, 4096, seed=9)
    rp, yp, n = sas.sas_surrogate_dataset(s)
    assert n == 4096
    torch.cuda.synchronize()
    raw = torch.as_tensor(_Dev(rp, (n, 8), "<f4"), device="cuda").cpu().numpy()
    y = torch.as_tensor(_Dev(yp, (n,), "<f4"), device="cuda").cpu().numpy()
    q = np.hypot(raw[:, 0], raw[:, 1])
    assert q.max() <= box["q_max"] * (1 + 1e-6)
    assert raw[:, 2].min() >= box["r_min"] and raw[:, 2].max() <= box["r_max"]
    assert np.all(np.isfinite(y)) and y.max() <= 1e-5
    idx = np.arange(0, n, 512)
    ref = np.maximum(M.exact_pbar(box, raw[idx]), M.TARGET_FLOOR)
    assert np.all(np.abs(np.exp(y[idx].astype(np.float64)) - ref) <= 1e-5 * ref + 1e-7)
    sas.sas_destroy_surrogate(s)


class _Dev:
    """Minimal __cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=shape, typestr=typestr, data=(ptr, False),
                                             version=3, strides=None)


def test_gradients_match_oracle():
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=5, stream=torch.cuda.current_stream())
    p = sas.sas_surrogate_get_params(s, M.NPARAM)
    rng = np.random.default_rng(2)
    p[M.OFF_W5:M.OFF_B5] = rng.uniform(-1, 1, 256).astype(np.float32) * 0.3
    p[M.OFF_B1 + 256:M.OFF_W5] = rng.normal(size=768).astype(np.float32) * 0.05
    sas.sas_surrogate_set_params(s, p)
    n = 512
    raw = _raw(box, n, 21)
    y = (np.random.default_rng(3).normal(size=n) - 3.0).astype(np.float32)
    rd = torch.tensor(raw, device="cuda")
    yd = torch.tensor(y, device="cuda")
    g = sas.sas_surrogate_grad(s, rd, yd, n, M.NPARAM).astype(np.float64)
    loss, go = M.loss_and_grad(p, M.features(box, raw.astype(np.float64)), y.astype(np.float64))
    go[M.OFF_B1:M.OFF_B1 + 256] = 0.0          # the layer-1 bias lives in W1[:, 63]
    segs = dict(W1=(M.OFF_W1, M.OFF_W2), W2=(M.OFF_W2, M.OFF_W3), W3=(M.OFF_W3, M.OFF_W4),
                W4=(M.OFF_W4, M.OFF_B1), b234=(M.OFF_B1 + 256, M.OFF_W5), w5=(M.OFF_W5, M.OFF_B5),
                b5=(M.OFF_B5, M.OFF_B5 + 1))
    mass = _grad_mass(p, M.features(box, raw.astype(np.float64)), y.astype(np.float64))
    for name, (a, b) in segs.items():
        tol = 1e-2 * np.abs(go[a:b]) + 1e-3 * mass[a:b]
        bad = np.abs(g[a:b] - go[a:b]) > tol
        assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(g[a:b] - go[a:b]) / (tol + 1e-300))))
    assert np.all(g[M.OFF_B1:M.OFF_B1 + 256] == 0.0)
    sas.sas_destroy_surrogate(s)


def _grad_mass(p, X, y):
    """L1 mass of every gradient element: the oracle's backpropagation with
    every factor replaced by its magnitude (sum over samples of |term|)."""
    out, zs, hs, Wl = M.forward(p, X, keep=True)
    n = X.shape[0]
    dout = np.abs(2.0 * (out - y) / n)
    mass = np.zeros(M.NPARAM)
    a4 = np.abs(M.bf16(hs[4]))
    mass[M.OFF_W5:M.OFF_B5] = a4.T @ dout
    mass[M.OFF_B5] = dout.sum()
    dh = np.outer(dout, np.abs(M.unpack(p)[3]))
    offs = [M.OFF_W1, M.OFF_W2, M.OFF_W3, M.OFF_W4]
    for l in range(3, -1, -1):
        dz = dh * np.abs(M.dsilu(zs[l]))
        gW = dz.T @ np.abs(M.bf16(hs[l]))
        mass[offs[l]: offs[l] + gW.size] = gW.reshape(-1)
        mass[M.OFF_B1 + l * M.H: M.OFF_B1 + (l + 1) * M.H] = dz.sum(axis=0)
        dh = dz @ np.abs(Wl[l])
    return mass


def _mse(s, raw_ptr, y_ptr, n):
    out = torch.empty(n, device="cuda")
    sas.sas_surrogate_eval(s, raw_ptr, n, out)
    y = torch.as_tensor(_Dev(y_ptr, (n,), "<f4"), device="cuda")
    torch.cuda.synchronize()
    return float(torch.mean((out - y) ** 2))


def test_training_reduces_loss():
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=3, stream=torch.cuda.current_stream())
    sas.sas_surrogate_generate(s, 1 << 17, seed=4)
    rp, yp, n = sas.sas_surrogate_dataset(s)
    before = _mse(s, rp, yp, n)
    sas.sas_surrogate_train(s, 400, 4096, 2e-3, 400)
    after = _mse(s, rp, yp, n)
    assert sas.sas_surrogate_info(s)["steps_done"] == 400
    assert after < 0.2 * before, (before, after)
    sas.sas_destroy_surrogate(s)


def test_surrogate_trace_falls_back_outside_the_box():
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=3, stream=torch.cuda.current_stream())
    inst = W.instrument(nx=64, ny=64, pixel_x=0.03, pixel_y=0.03)   # corners reach |Q| = 0.3 > q_max
    m = W.Model(kind=W.CYLINDER, radius=20.0, length=400.0, sld=2e-6, volume_fraction=0.01, poly=0.1,
                n_poly=12, sigma_orient=math.radians(15), n_gamma=16, n_psi=16)
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    sas.sas_attach_surrogate(e.h, s)
    n = 20000
    e.trace(n, seed=2)
    d = e.read()
    fb = sas.sas_surrogate_fallbacks(exp=e.h)
    ref = oracle.trace(inst, m, n, seed=2)
    assert np.array_equal(d["count"], ref["count"].astype(np.uint64))   # same histories
    assert 0 < fb < n
    # out-of-box model: exact path, identical to the plain trace
    m2 = W.Model(**{**m.as_dict(), "radius": 60.0})
    e.set_model(m2)
    e.trace(n, seed=2)
    d2 = e.read()
    ref2 = oracle.trace(inst, m2, n, seed=2)
    so = ref2["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d2["sum_w"] - so)[big] <= 1e-4 * so[big])
    e.close()
    sas.sas_destroy_surrogate(s)


def _axial_length(m):
    """The body's length along its axis, the surrogate's L: the cylinder's
    length, twice the ellipsoid's polar semi-axis."""
    return 2.0 * m.radius_polar if m.kind == W.ELLIPSOID else m.length


def _network_tally(box, p, inst, m, n, seed, first=0, exp_id=0):
    """Expected surrogate detector from the oracle alone: oracle geometry
    (pixel, Q, prefactor), the oracle network on the features of Q about the
    body's axis, and <V^2>/<V> from the oracle's Schulz nodes."""
    g = oracle.geometry_records(inst, n, seed, first=first, exp_id=exp_id)
    sc = g["pixel"] >= 0
    ax = np.array([math.sin(m.axis_theta) * math.cos(m.axis_phi),
                   math.sin(m.axis_theta) * math.sin(m.axis_phi), math.cos(m.axis_theta)])
    q = g["q"][sc]
    qp = q @ ax
    qt = np.sqrt(np.maximum(np.sum(q * q, axis=1) - qp * qp, 0.0))
    assert np.sqrt(np.sum(q * q, axis=1)).max() < box["q_max"]       # every history in the box
    raw = np.zeros((len(qp), 8))
    raw[:, 0], raw[:, 1] = np.abs(qp), qt
    raw[:, 2], raw[:, 3], raw[:, 4], raw[:, 5] = m.radius, _axial_length(m), m.sigma_orient, m.poly
    out = M.forward(p, M.features(box, raw))
    prep = oracle.Prepared(m)
    V = (4.0 / 3.0 * math.pi * prep.poly_r ** 2 * m.radius_polar if m.kind == W.ELLIPSOID
         else math.pi * prep.poly_r ** 2 * m.length)
    scale = m.volume_fraction * (m.sld - m.sld_solvent) ** 2 * float(np.dot(prep.poly_w, V * V)) / float(
        np.dot(prep.poly_w, V))
    w = g["pref"][sc] * scale * np.exp(out)
    npix = inst.nx * inst.ny
    return dict(sum_w=np.bincount(g["pixel"][sc], weights=w, minlength=npix),
                count=np.bincount(g["pixel"][sc], minlength=npix), trans=float(g["trans"].sum()))


@pytest.mark.parametrize("n, first", [(116813, 0), (700, 0), (40000, 123457)])
def test_surrogate_trace_tallies_the_network(n, first):
    """The warp-specialised trace (two tiles in flight, static pair
    schedule, reversed K order on the second tile) against the oracle
    geometry weighted by the oracle network on the same BF16 weights:
    identical histories per pixel, per-pixel sums within the BF16 operand
    tolerance of the network test, transmitted weight to FP32 rounding."""
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=7, stream=torch.cuda.current_stream())
    p = sas.sas_surrogate_get_params(s, M.NPARAM)
    rng = np.random.default_rng(4)
    p[M.OFF_W5:M.OFF_B5] = rng.uniform(-1, 1, 256).astype(np.float32) * 0.3
    p[M.OFF_B1 + 256:M.OFF_W5] = rng.normal(size=768).astype(np.float32) * 0.1
    p[M.OFF_B5] = -2.0
    sas.sas_surrogate_set_params(s, p)
    inst = W.instrument(nx=48, ny=40, pixel_x=0.008, pixel_y=0.008)
    m = W.Model(kind=W.CYLINDER, radius=19.0, length=420.0, sld=2e-6, volume_fraction=0.01, poly=0.1,
                n_poly=12, sigma_orient=math.radians(14), n_gamma=16, n_psi=16,
                axis_theta=math.radians(70), axis_phi=math.radians(20))
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    sas.sas_attach_surrogate(e.h, s)
    fb0 = sas.sas_surrogate_fallbacks(exp=e.h)
    sas.sas_reset_detector(e.h)
    e.trace_range(first, n, seed=5)
    d = e.read()
    assert sas.sas_surrogate_fallbacks(exp=e.h) == fb0                 # nothing left the box
    ref = _network_tally(box, p, inst, m, n, seed=5, first=first)
    assert np.array_equal(d["count"].ravel(), ref["count"].astype(np.uint64))
    got, exp_ = d["sum_w"].ravel(), ref["sum_w"]
    assert abs(got.sum() - exp_.sum()) <= 3e-3 * exp_.sum()
    # pixels with many histories average the per-history BF16 differences;
    # a short run has single-history pixels (bound of the network test)
    few = n < 20 * inst.nx * inst.ny
    hit = ref["count"] >= (1 if few else 20)
    assert hit.sum() > 100
    rel = np.abs(got - exp_)[hit] / exp_[hit]
    assert np.median(rel) < (5e-3 if few else 3e-3), np.median(rel)
    assert rel.max() < (8e-2 if few else 3e-2), rel.max()
    assert d["trans"] == pytest.approx(ref["trans"], rel=1e-5)
    e.close()
    sas.sas_destroy_surrogate(s)


def test_bounded_wait_gives_up_and_the_next_call_runs():
    """Failure detection without a GPU fault: the test hook makes the first
    CTA of the next evaluation wait on a barrier that nothing completes,
    before any copy or tensor-core operation is issued. The wait gives up
    after 20 ms, the call reports SAS_ERR_TIMEOUT, and the next evaluation
    (which allocates the tensor memory again in every CTA) returns the same
    values as the one before the failure."""
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=7, stream=torch.cuda.current_stream())
    n = 1000
    rd = torch.tensor(_raw(box, n, 3), device="cuda")
    out0 = torch.empty(n, device="cuda")
    sas.sas_surrogate_eval(s, rd, n, out0)
    out1 = torch.full((n,), -7.0, device="cuda")
    sas.sas_surrogate_test_stall(s, 20_000_000)
    with pytest.raises(sas.SasError) as e:
        sas.sas_surrogate_eval(s, rd, n, out1)
    assert e.value.status == sas.SAS_ERR_TIMEOUT
    assert torch.all(out1 == -7.0)                     # nothing was written
    out2 = torch.empty(n, device="cuda")
    sas.sas_surrogate_eval(s, rd, n, out2)             # the hook cleared itself
    torch.cuda.synchronize()
    assert torch.equal(out0, out2)
    with pytest.raises(sas.SasError):
        sas.sas_surrogate_test_stall(s, 2_000_000_000)
    sas.sas_destroy_surrogate(s)


def test_batch_surrogate_share_counts_covered_experiments():
    """sas_batch_surrogate_share reports the experiments (and their
    histories) whose model lies in the attached surrogate's box; the others
    run the exact quadrature and equal the oracle."""
    box = _small_box()
    s = sas.sas_create_surrogate(box, seed=3, stream=torch.cuda.current_stream())
    inst = W.instrument(nx=32, ny=32)
    cyl = dict(kind=W.CYLINDER, sld=2e-6, volume_fraction=0.01, n_poly=12, n_gamma=16, n_psi=16)
    models = [W.Model(radius=20.0, length=400.0, poly=0.1, sigma_orient=math.radians(15), **cyl),
              W.Model(radius=60.0, length=400.0, poly=0.1, sigma_orient=math.radians(15), **cyl),   # R out of box
              W.Model(kind=W.SPHERE, radius=30.0, poly=0.1, n_poly=8),
              W.Model(radius=18.0, length=320.0, poly=0.12, sigma_orient=math.radians(11), **cyl)]
    counts = np.array([3000, 2000, 5000, 1000], np.uint64)
    b = sas.sas_create_batch(inst, models, counts, stream=torch.cuda.current_stream())
    assert sas.sas_batch_surrogate_share(b) == (0, 0)          # nothing attached
    sas.sas_batch_attach_surrogate(b, s)
    assert sas.sas_batch_surrogate_share(b) == (2, 4000)
    sas.sas_trace_batch(b, seed=4)
    npix = inst.nx * inst.ny
    for e in (1, 2):                                               # exact path: the oracle's trace
        d = sas.sas_read_batch_detector(b, e, npix)
        ref = oracle.trace(inst, models[e], int(counts[e]), seed=4, exp_id=e)
        assert np.array_equal(d["count"], ref["count"].reshape(-1).astype(np.uint64))
        so = ref["sum_w"].reshape(-1)
        big = so > 1e-6 * so.max()
        assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
    sas.sas_batch_attach_surrogate(b, None)
    assert sas.sas_batch_surrogate_share(b) == (0, 0)
    sas.sas_destroy_batch(b)
    sas.sas_destroy_surrogate(s)


def test_exact_targets_batched_box():
    """The training targets over the batched box (R and L up to 200 A, |Q|
    up to 0.115, sigma_orient down to 1 deg, sigma_poly down to 0.01), where
    q_perp r reaches the large-argument forms of 2 J1(x)/x, against the
    oracle's quadrature; the corners of the box included."""
    box = W.batched_surrogate_box()
    s = sas.sas_create_surrogate(box, seed=1, stream=torch.cuda.current_stream())
    raw = _raw(box, 6, 13)
    corners = np.array([[0.113, 0.02, 200.0, 200.0, box["sigma_orient_min"], box["poly_min"]],
                        [0.02, 0.113, 200.0, 10.0, box["sigma_orient_max"], box["poly_max"]],
                        [0.08, 0.08, 10.0, 200.0, box["sigma_orient_min"], box["poly_max"]]], np.float32)
    nb = box["n_buckets"]
    for c in corners:
        bk = int(round((c[5] - box["poly_min"]) / (box["poly_max"] - box["poly_min"]) * (nb - 1)))
        row = np.zeros(8, np.float32)
        row[:6] = c
        row[5] = np.float32(box["poly_min"] + (box["poly_max"] - box["poly_min"]) * bk / (nb - 1))
        row[6] = bk
        raw = np.vstack([raw, row])
    n = len(raw)
    rd = torch.tensor(raw, device="cuda")
    out = torch.empty(n, device="cuda")
    sas.sas_surrogate_exact(s, rd, n, out)
    torch.cuda.synchronize()
    got = np.exp(out.cpu().numpy().astype(np.float64))
    ref = np.maximum(M.exact_pbar(box, raw), M.TARGET_FLOOR)
    assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-7), np.max(np.abs(got - ref) / ref)
    sas.sas_destroy_surrogate(s)


# ---- the ellipsoid of revolution (same network, L = 2 R_p) --------------

def _small_ell_box(n_fourier=4):
    b = W.batched_ellipsoid_surrogate_box(n_fourier=n_fourier, n_buckets=8)
    b.update(n_poly=12, n_gamma=16, n_psi=16)
    return b


def _set_test_params(s, seed):
    """Random but well-scaled output layer and biases, so that the network
    output spreads over a few units of log P."""
    p = sas.sas_surrogate_get_params(s, M.NPARAM)
    rng = np.random.default_rng(seed)
    p[M.OFF_W5:M.OFF_B5] = rng.uniform(-1, 1, 256).astype(np.float32) * 0.3
    p[M.OFF_B1 + 256:M.OFF_W5] = rng.normal(size=768).astype(np.float32) * 0.1
    p[M.OFF_B5] = -2.0
    sas.sas_surrogate_set_params(s, p)
    return p


def test_exact_targets_ellipsoid_match_oracle():
    """Training targets of the ellipsoid surrogate (polar semi-axis L / 2,
    Schulz-distributed equatorial semi-axis) against the oracle's
    quadrature: random rows of a small box, Q = 0, and the corners of the
    batched ellipsoid box (R and R_p up to 200 A at |Q| up to 0.115)."""
    for box, seed in ((_small_ell_box(), 21), (W.batched_ellipsoid_surrogate_box(), 22)):
        s = sas.sas_create_surrogate(box, seed=1, stream=torch.cuda.current_stream())
        raw = _raw(box, 24, seed)
        raw[0, :2] = 0.0
        nb = box["n_buckets"]
        corners = np.array([[0.113, 0.02, 200.0, 400.0, box["sigma_orient_min"], box["poly_min"]],
                            [0.02, 0.113, 200.0, 20.0, box["sigma_orient_max"], box["poly_max"]],
                            [0.08, 0.08, 10.0, 400.0, box["sigma_orient_min"], box["poly_max"]]], np.float32)
        for c in corners:
            bk = int(round((c[5] - box["poly_min"]) / (box["poly_max"] - box["poly_min"]) * (nb - 1)))
            row = np.zeros(8, np.float32)
            row[:6] = c
            row[5] = np.float32(box["poly_min"] + (box["poly_max"] - box["poly_min"]) * bk / (nb - 1))
            row[6] = bk
            raw = np.vstack([raw, row])
        n = len(raw)
        rd = torch.tensor(raw, device="cuda")
        out = torch.empty(n, device="cuda")
        sas.sas_surrogate_exact(s, rd, n, out)
        torch.cuda.synchronize()
        got = np.exp(out.cpu().numpy().astype(np.float64))
        ref = np.maximum(M.exact_pbar(box, raw), M.TARGET_FLOOR)
        assert abs(ref[0] - 1.0) < 1e-12
        assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-7), np.max(np.abs(got - ref) / ref)
        sas.sas_destroy_surrogate(s)


def test_ellipsoid_surrogate_trace_tallies_the_network():
    """The surrogate trace of an ellipsoid of revolution against the oracle
    geometry weighted by the oracle network (features with L = 2 R_p,
    <V^2>/<V> of the ellipsoid), as for the cylinder."""
    box = _small_ell_box()
    s = sas.sas_create_surrogate(box, seed=7, stream=torch.cuda.current_stream())
    p = _set_test_params(s, 5)
    inst = W.instrument(nx=48, ny=40, pixel_x=0.008, pixel_y=0.008)
    m = W.Model(kind=W.ELLIPSOID, radius=60.0, radius_polar=150.0, sld=2e-6, volume_fraction=0.01, poly=0.1,
                n_poly=12, sigma_orient=math.radians(14), n_gamma=16, n_psi=16,
                axis_theta=math.radians(70), axis_phi=math.radians(20))
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    sas.sas_attach_surrogate(e.h, s)
    fb0 = sas.sas_surrogate_fallbacks(exp=e.h)
    sas.sas_reset_detector(e.h)
    n, first = 60000, 123457
    e.trace_range(first, n, seed=5)
    d = e.read()
    assert sas.sas_surrogate_fallbacks(exp=e.h) == fb0
    ref = _network_tally(box, p, inst, m, n, seed=5, first=first)
    assert np.array_equal(d["count"].ravel(), ref["count"].astype(np.uint64))
    got, exp_ = d["sum_w"].ravel(), ref["sum_w"]
    assert abs(got.sum() - exp_.sum()) <= 3e-3 * exp_.sum()
    hit = ref["count"] >= 20
    assert hit.sum() > 100
    rel = np.abs(got - exp_)[hit] / exp_[hit]
    assert np.median(rel) < 3e-3, np.median(rel)
    assert rel.max() < 3e-2, rel.max()
    assert d["trans"] == pytest.approx(ref["trans"], rel=1e-5)
    e.close()
    sas.sas_destroy_surrogate(s)


def test_ellipsoid_surrogate_falls_back_outside_the_box():
    """Histories of an ellipsoid whose |Q| leaves the box take the exact
    ellipsoid quadrature: the same histories as the oracle's trace, some of
    them counted as fallbacks, and those pixels' sums equal the oracle's."""
    box = _small_ell_box()
    s = sas.sas_create_surrogate(box, seed=3, stream=torch.cuda.current_stream())
    inst = W.instrument(nx=64, ny=64, pixel_x=0.03, pixel_y=0.03)   # corners reach |Q| = 0.3 > q_max
    m = W.Model(kind=W.ELLIPSOID, radius=40.0, radius_polar=90.0, sld=2e-6, volume_fraction=0.01, poly=0.1,
                n_poly=12, sigma_orient=math.radians(15), n_gamma=16, n_psi=16, axis_theta=math.radians(50))
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    sas.sas_attach_surrogate(e.h, s)
    n = 20000
    e.trace(n, seed=2)
    d = e.read()
    fb = sas.sas_surrogate_fallbacks(exp=e.h)
    ref = oracle.trace(inst, m, n, seed=2)
    assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
    assert 0 < fb < n
    g = oracle.geometry_records(inst, n, 2)
    sc = g["pixel"] >= 0
    qn = np.sqrt(np.sum(g["q"][sc] ** 2, axis=1))
    npix = inst.nx * inst.ny
    # histories within rounding of the box edge count as inside (FP32 decides there)
    inside = np.bincount(g["pixel"][sc], weights=(qn <= box["q_max"] * (1 + 1e-5)).astype(float), minlength=npix)
    out_only = (inside == 0) & (ref["count"].reshape(-1) > 0)     # pixels reached by fallbacks alone
    assert out_only.sum() > 50
    so, got = ref["sum_w"].reshape(-1)[out_only], d["sum_w"].reshape(-1)[out_only]
    assert np.all(np.abs(got - so) <= 1e-4 * so + 1e-12 * so.max())
    e.close()
    sas.sas_destroy_surrogate(s)


def test_batch_holds_a_surrogate_per_kind():
    """A batch holds one cylinder and one ellipsoid surrogate: each serves
    the in-box experiments of its kind (their tallies are the oracle
    network's), the rest run the exact quadrature and equal the oracle;
    attaching a second surrogate of the same kind replaces the first, and
    NULL detaches both."""
    cbox, ebox = _small_box(), _small_ell_box()
    st = torch.cuda.current_stream()
    sc, se = sas.sas_create_surrogate(cbox, seed=3, stream=st), sas.sas_create_surrogate(ebox, seed=4, stream=st)
    pc, pe = _set_test_params(sc, 8), _set_test_params(se, 9)
    inst = W.instrument(nx=32, ny=32, pixel_x=0.008, pixel_y=0.008)
    com = dict(sld=2e-6, volume_fraction=0.01, n_poly=12, n_gamma=16, n_psi=16, poly=0.1,
               sigma_orient=math.radians(15), axis_theta=math.radians(60), axis_phi=math.radians(30))
    models = [W.Model(kind=W.CYLINDER, radius=20.0, length=400.0, **com),          # cylinder surrogate
              W.Model(kind=W.ELLIPSOID, radius=50.0, radius_polar=120.0, **com),   # ellipsoid surrogate
              W.Model(kind=W.ELLIPSOID, radius=50.0, radius_polar=250.0, **com),   # 2 R_p out of box
              W.Model(kind=W.SPHERE, radius=30.0, poly=0.1, n_poly=8)]
    counts = np.array([30000, 30000, 3000, 5000], np.uint64)
    b = sas.sas_create_batch(inst, models, counts, stream=st)
    sas.sas_batch_attach_surrogate(b, sc)
    assert sas.sas_batch_surrogate_share(b) == (1, 30000)
    sas.sas_batch_attach_surrogate(b, se)
    assert sas.sas_batch_surrogate_share(b) == (2, 60000)
    sas.sas_trace_batch(b, seed=4)
    npix = inst.nx * inst.ny
    for e_, box, p in ((0, cbox, pc), (1, ebox, pe)):
        d = sas.sas_read_batch_detector(b, e_, npix)
        ref = _network_tally(box, p, inst, models[e_], int(counts[e_]), seed=4, exp_id=e_)
        assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
        got, exp_ = d["sum_w"], ref["sum_w"]
        assert abs(got.sum() - exp_.sum()) <= 3e-3 * exp_.sum()
        hit = ref["count"] >= 20
        rel = np.abs(got - exp_)[hit] / exp_[hit]
        assert hit.sum() > 100 and np.median(rel) < 3e-3 and rel.max() < 3e-2, (e_, np.median(rel), rel.max())
    for e_ in (2, 3):
        d = sas.sas_read_batch_detector(b, e_, npix)
        ref = oracle.trace(inst, models[e_], int(counts[e_]), seed=4, exp_id=e_)
        assert np.array_equal(d["count"], ref["count"].reshape(-1).astype(np.uint64))
        so = ref["sum_w"].reshape(-1)
        big = so > 1e-6 * so.max()
        assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
    sc2 = sas.sas_create_surrogate(cbox, seed=5, stream=st)
    _set_test_params(sc2, 10)
    sas.sas_batch_attach_surrogate(b, sc2)                          # replaces sc, keeps se
    assert sas.sas_batch_surrogate_share(b) == (2, 60000)
    sas.sas_batch_attach_surrogate(b, None)
    assert sas.sas_batch_surrogate_share(b) == (0, 0)
    sas.sas_destroy_batch(b)
    for s in (sc, se, sc2):
        sas.sas_destroy_surrogate(s)
