"""FP64 oracle of the learned surrogate (TEST INFRASTRUCTURE ONLY).

Plain numpy definitions of what the surrogate computes:

* the feature map of an oriented polydisperse cylinder evaluation (see
  `features`): u = q_par L / 2, v = q_perp R, ln a with a = L / (2R),
  sigma_orient, sigma_poly, each scaled linearly to [-1, 1] over the
  training box, three logarithmic envelopes, n_fourier (sin, cos) pairs of
  k u / 2 and as many of k v / 2; the last of 64 columns is 1 (it carries
  the layer-1 bias through W1[:, 63]);
* the network log P = b5 + w5 . h4, h_l = SiLU(W_l h_{l-1} + b_l),
  SiLU(z) = z s(z), s(z) = 1/2 + tanh(z/2)/2, with BF16-rounded hidden
  weights and BF16-rounded inputs of every hidden matrix product (the
  tensor-core operands), FP64 arithmetic otherwise;
* the mean squared error of log P and its exact gradient (backpropagation);
* the exact target P = <|F|^2> / (drho^2 <V^2>) from the trace oracle, of
  a cylinder of length L or of an ellipsoid of revolution of polar
  semi-axis L / 2 (the same features serve both bodies).

Flat parameter layout (float32 master copy): W1 [256][64] | W2 | W3 | W4
[256][256] (out, in) | b1 (unused) | b2 | b3 | b4 | w5 [256] | b5.
"""
from __future__ import annotations

import math

import numpy as np

H, KIN = 256, 64
OFF_W1 = 0
OFF_W2 = OFF_W1 + H * KIN
OFF_W3 = OFF_W2 + H * H
OFF_W4 = OFF_W3 + H * H
OFF_B1 = OFF_W4 + H * H
OFF_W5 = OFF_B1 + 4 * H
OFF_B5 = OFF_W5 + H
NPARAM = OFF_B5 + 1
TARGET_FLOOR = 1e-6


def bf16(x):
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    W1 = p[OFF_W1:OFF_W2].reshape(H, KIN)
    Ws = [p[OFF_W2 + l * H * H: OFF_W2 + (l + 1) * H * H].reshape(H, H) for l in range(3)]
    bs = [p[OFF_B1 + l * H: OFF_B1 + (l + 1) * H] for l in range(4)]
    w5 = p[OFF_W5:OFF_B5]
    b5 = p[OFF_B5]
    return W1, Ws, bs, w5, b5


def sig(z):
    return 0.5 + 0.5 * np.tanh(0.5 * z)


def silu(z):
    return z * sig(z)


def dsilu(z):
    s = sig(z)
    return s * (1.0 + z * (1.0 - s))


def box_ranges(box):
    return dict(u_max=0.5 * box["q_max"] * box["l_max"], v_max=box["q_max"] * box["r_max"],
                la_min=math.log(0.5 * box["l_min"] / box["r_max"]),
                la_max=math.log(0.5 * box["l_max"] / box["r_min"]))


FOURIER0 = 8


def features(box, raw):
    """raw [n][>=6]: q_par, q_perp, R, L, sigma_orient, sigma_poly -> [n][64].

    u = q_par L / 2, v = q_perp R, a = L / (2R); columns 0..4: u, v, ln a,
    sigma_orient, sigma_poly scaled to [-1, 1] over the box; 5..7:
    ln(1 + u^2) / 4 - 1, ln(1 + v^2) / 4 - 1, ln(1 + (u / a)^2) / 4 - 1;
    from 8: n_fourier (sin, cos) pairs of k u / 2, then n_fourier pairs of
    k v / 2 (k = 1..n); 63: 1."""
    raw = np.asarray(raw, dtype=np.float64)
    rg = box_ranges(box)
    u = raw[:, 0] * 0.5 * raw[:, 3]
    v = raw[:, 1] * raw[:, 2]
    a = 0.5 * raw[:, 3] / raw[:, 2]
    la_max = rg["la_max"] if rg["la_max"] > rg["la_min"] else rg["la_min"] + 1.0
    F = np.zeros((raw.shape[0], KIN))
    F[:, 0] = 2 * u / rg["u_max"] - 1
    F[:, 1] = 2 * v / rg["v_max"] - 1
    F[:, 2] = 2 * (np.log(a) - rg["la_min"]) / (la_max - rg["la_min"]) - 1
    F[:, 3] = 2 * (raw[:, 4] - box["sigma_orient_min"]) / (box["sigma_orient_max"] - box["sigma_orient_min"]) - 1
    F[:, 4] = 2 * (raw[:, 5] - box["poly_min"]) / (box["poly_max"] - box["poly_min"]) - 1
    F[:, 5] = np.log1p(u * u) / 4 - 1
    F[:, 6] = np.log1p(v * v) / 4 - 1
    F[:, 7] = np.log1p((u / a) ** 2) / 4 - 1
    n = box["n_fourier"]
    for t, x in enumerate((u, v)):
        for k in range(n):
            c = FOURIER0 + 2 * (t * n + k)
            F[:, c] = np.sin((k + 1) * 0.5 * x)
            F[:, c + 1] = np.cos((k + 1) * 0.5 * x)
    F[:, 63] = 1.0
    return F


def _ident(x):
    return np.asarray(x, dtype=np.float64)


def forward(p, X, keep=False, rnd=bf16):
    """log P for features X [n][64]; with keep, also the pre-activations.
    rnd is the rounding of the tensor-core operands (bf16; identity for the
    finite-difference pin)."""
    W1, Ws, bs, w5, b5 = unpack(p)
    a = rnd(X)
    zs, hs = [], [a]
    Wl = [rnd(W1)] + [rnd(W) for W in Ws]
    for l in range(4):
        z = a @ Wl[l].T + bs[l]
        h = silu(z)
        zs.append(z)
        hs.append(h)
        a = rnd(h)
    out = b5 + a @ w5
    if keep:
        return out, zs, hs, Wl
    return out


def loss_and_grad(p, X, y, rnd=bf16):
    """Mean squared error of log P and its gradient (flat, FP64); the
    roundings pass gradients through unchanged."""
    out, zs, hs, Wl = forward(p, X, keep=True, rnd=rnd)
    n = X.shape[0]
    r = out - y
    loss = float(np.mean(r * r))
    g = np.zeros(NPARAM)
    dout = 2.0 * r / n
    a4 = rnd(hs[4])
    g[OFF_W5:OFF_B5] = a4.T @ dout
    g[OFF_B5] = dout.sum()
    dh = np.outer(dout, unpack(p)[3])
    offs = [OFF_W1, OFF_W2, OFF_W3, OFF_W4]
    for l in range(3, -1, -1):
        dz = dh * dsilu(zs[l])
        a_in = rnd(hs[l])
        gW = dz.T @ a_in
        g[offs[l]: offs[l] + gW.size] = gW.reshape(-1)
        g[OFF_B1 + l * H: OFF_B1 + (l + 1) * H] = dz.sum(axis=0)
        dh = dz @ Wl[l]
    return loss, g


def exact_pbar(box, raw):
    """Exact P at raw parameters [n][8] (bucket sigma_poly in column 5)
    with the trace oracle's quadrature about the z axis, for the box's body:
    the cylinder of length L, or (box model ELLIPSOID) the ellipsoid of
    revolution with polar semi-axis L / 2 and polydisperse equatorial
    semi-axis R. The training target is log max(P, TARGET_FLOOR)."""
    import oracle
    import sas_workloads as W
    ell = box.get("model", W.CYLINDER) == W.ELLIPSOID
    out = np.empty(len(raw))
    for i, r in enumerate(np.asarray(raw, dtype=np.float64)):
        qpar, qperp, R, L, so, sp = r[:6]
        shape = dict(kind=W.ELLIPSOID, radius_polar=0.5 * L) if ell else dict(kind=W.CYLINDER, length=L)
        m = W.Model(radius=R, sld=1.0, volume_fraction=1.0, poly=sp,
                    n_poly=box["n_poly"], sigma_orient=so, axis_theta=0.0, axis_phi=0.0,
                    n_gamma=box["n_gamma"], n_psi=box["n_psi"], **shape)
        prep = oracle.Prepared(m)
        V = (4.0 / 3.0 * math.pi * prep.poly_r ** 2 * 0.5 * L) if ell else math.pi * prep.poly_r ** 2 * L
        vm = float(np.dot(prep.poly_w, V))
        v2 = float(np.dot(prep.poly_w, V * V))
        ds = oracle.dsigma(prep, np.array([[qperp, 0.0, qpar]]))[0]
        out[i] = ds * vm / v2
    return out
