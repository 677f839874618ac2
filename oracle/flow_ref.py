"""FP64 reference of the learned importance sampler (TEST INFRASTRUCTURE ONLY:
used by tests/ to check the CUDA flow kernels; never imported by the product).

The sampler replaces the VEGAS map of the Monte Carlo integral (Sec. 2: importance
sampling) by an event-conditioned normalising flow on the unit cube:
  u ~ U(0,1)^d  ->  z0 = logit(u)  ->  K affine coupling layers  ->  y = sigmoid(z_K)
with coupling layer k:  z'[B] = z[B] * exp(s) + t,  z'[A] = z[A],
  (s_raw, t) = MLP_k([z[A], c]),  s = S_MAX tanh(s_raw / S_MAX),
MLP = Linear(|A|+C -> H), ReLU, Linear(H -> H), ReLU, Linear(H -> 2|B|).
A = indices with parity k % 2, B = the others; c = per-event conditioning vector.
The map's Jacobian is exact:
  log|dy/du| = sum_j log sigmoid'(z_K,j) + sum_k sum_B s_k - sum_j log sigmoid'(z0_j)
so f(y) |dy/du| is an unbiased weight for u uniform. Training minimises
  L = -sum_i w_i log q(y_i),  log q(y) = -log|dy/du| (evaluated by the inverse map)
on VEGAS-weighted samples (w normalised per item), i.e. the KL divergence from
the integrand's normalised density to q.
"""
from __future__ import annotations

import numpy as np

S_MAX = 2.0


def masks(d, k):
    A = np.array([j for j in range(d) if j % 2 == k % 2])
    B = np.array([j for j in range(d) if j % 2 != k % 2])
    return A, B


def init_params(d, n_layers, hidden, n_cond, seed, zero_last=True):
    rng = np.random.default_rng(seed)
    layers = []
    for k in range(n_layers):
        A, B = masks(d, k)
        fan1 = len(A) + n_cond
        L = {
            "W1a": rng.normal(0, 1 / np.sqrt(fan1), (len(A), hidden)),
            "W1c": rng.normal(0, 1 / np.sqrt(fan1), (n_cond, hidden)),
            "b1": np.zeros(hidden),
            "W2": rng.normal(0, 1 / np.sqrt(hidden), (hidden, hidden)),
            "b2": np.zeros(hidden),
            "W3": (np.zeros((hidden, 2 * len(B))) if zero_last
                   else rng.normal(0, 0.1 / np.sqrt(hidden), (hidden, 2 * len(B)))),
            "b3": np.zeros(2 * len(B)),
        }
        layers.append(L)
    return layers


PARAM_ORDER = ("W1a", "W1c", "b1", "W2", "b2", "W3", "b3")


def to_flat(layers):
    """The flat FP32 layout of the C ABI (per layer, PARAM_ORDER, row-major)."""
    return np.concatenate([layers[k][n].ravel() for k in range(len(layers)) for n in PARAM_ORDER])


def from_flat(flat, d, n_layers, hidden, n_cond):
    shapes = {}
    layers = []
    off = 0
    for k in range(n_layers):
        A, B = masks(d, k)
        shapes = {"W1a": (len(A), hidden), "W1c": (n_cond, hidden), "b1": (hidden,),
                  "W2": (hidden, hidden), "b2": (hidden,), "W3": (hidden, 2 * len(B)),
                  "b3": (2 * len(B),)}
        L = {}
        for n in PARAM_ORDER:
            size = int(np.prod(shapes[n]))
            L[n] = np.asarray(flat[off:off + size], dtype=np.float64).reshape(shapes[n])
            off += size
        layers.append(L)
    assert off == len(flat)
    return layers


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def _log_sig_prime(z):
    # log(sigmoid(z)(1 - sigmoid(z))) = -|z| - 2 log(1 + exp(-|z|))
    a = np.abs(z)
    return -a - 2.0 * np.log1p(np.exp(-a))


def _ident(a):
    return a


def _mlp(L, za, c, rnd=_ident):
    """za: (n, |A|), c: (n, C) -> s, t (n, |B|) and the hidden activations.
    rnd: rounding applied to the operands of the hidden and output products
    (the hidden activations and the weights W2, W3), identity by default."""
    a1 = za @ L["W1a"] + c @ L["W1c"] + L["b1"]
    h1 = rnd(np.maximum(a1, 0.0))
    a2 = h1 @ rnd(L["W2"]) + L["b2"]
    h2 = rnd(np.maximum(a2, 0.0))
    o = h2 @ rnd(L["W3"]) + L["b3"]
    nb = o.shape[1] // 2
    s_raw, t = o[:, :nb], o[:, nb:]
    s = S_MAX * np.tanh(s_raw / S_MAX)
    return s, t, (a1, h1, a2, h2, s_raw)


def forward(layers, u, c):
    """u (n, d) in (0,1), c (n, C) -> y (n, d), log|dy/du| (n,)."""
    d = u.shape[1]
    z = np.log(u) - np.log1p(-u)
    logj = -np.sum(_log_sig_prime(z), axis=1)
    for k, L in enumerate(layers):
        A, B = masks(d, k)
        s, t, _ = _mlp(L, z[:, A], c)
        z = z.copy()
        z[:, B] = z[:, B] * np.exp(s) + t
        logj += np.sum(s, axis=1)
    logj += np.sum(_log_sig_prime(z), axis=1)
    return _sig(z), logj


def inverse(layers, y, c, rnd=_ident):
    """y (n, d) -> u (n, d), log|dy/du| at that point (n,)."""
    d = y.shape[1]
    z = np.log(y) - np.log1p(-y)
    logj = np.sum(_log_sig_prime(z), axis=1)
    for k in reversed(range(len(layers))):
        A, B = masks(d, k)
        s, t, _ = _mlp(layers[k], z[:, A], c, rnd)
        z = z.copy()
        z[:, B] = (z[:, B] - t) * np.exp(-s)
        logj += np.sum(s, axis=1)
    logj -= np.sum(_log_sig_prime(z), axis=1)
    return _sig(z), logj


def loss(layers, y, w, c, rnd=_ident):
    """L = -sum_i w_i log q(y_i) = sum_i w_i log|dy/du|(y_i)."""
    _, logj = inverse(layers, y, c, rnd)
    return float(np.sum(w * logj))


def grad(layers, y, w, c, rnd=_ident):
    """Gradient of loss() with respect to every parameter, by hand-written
    reverse-mode differentiation through the inverse map. rnd: rounding of the
    operands of every product with the hidden layers (activations, weights,
    dL/d(out) and dL/da2), identity by default; with BF16 rounding it states the
    same computation as tensor-core kernels that take BF16 operands and
    accumulate in higher precision."""
    d = y.shape[1]
    n_layers = len(layers)
    z = np.log(y) - np.log1p(-y)
    zs = [None] * (n_layers + 1)
    zs[n_layers] = z
    caches = [None] * n_layers
    for k in reversed(range(n_layers)):
        A, B = masks(d, k)
        zk1 = zs[k + 1]
        s, t, cache = _mlp(layers[k], zk1[:, A], c, rnd)
        zk = zk1.copy()
        zk[:, B] = (zk1[:, B] - t) * np.exp(-s)
        zs[k] = zk
        caches[k] = (s, t, cache)
    # loss = sum w [ sum_k sum_B s_k - sum_j log sig'(z0_j) ] + const(y)
    z0 = zs[0]
    # d/dz log sig'(z) = 1 - 2 sigmoid(z)
    gz = -(w[:, None]) * (1.0 - 2.0 * _sig(z0))   # dL/dz0
    grads = [None] * n_layers
    for k in range(n_layers):
        A, B = masks(d, k)
        L = layers[k]
        zk1 = zs[k + 1]
        s, t, (a1, h1, a2, h2, s_raw) = caches[k]
        e = np.exp(-s)
        # z_k[B] = (z_{k+1}[B] - t) e^{-s};  z_k[A] = z_{k+1}[A]
        gzb = gz[:, B]
        g_zk1 = np.zeros_like(zk1)
        g_zk1[:, A] = gz[:, A]          # z_k[A] = z_{k+1}[A]
        g_zk1[:, B] = gzb * e
        g_t = -gzb * e
        g_s = -gzb * (zk1[:, B] - t) * e + w[:, None]          # + direct loss term
        g_sraw = g_s * (1.0 - np.tanh(s_raw / S_MAX) ** 2)
        g_o = rnd(np.concatenate([g_sraw, g_t], axis=1))
        G = {"W3": h2.T @ g_o, "b3": g_o.sum(0)}
        g_h2 = g_o @ rnd(L["W3"]).T
        g_a2 = rnd(g_h2 * (a2 > 0))
        G["W2"] = h1.T @ g_a2
        G["b2"] = g_a2.sum(0)
        g_h1 = g_a2 @ rnd(L["W2"]).T
        g_a1 = g_h1 * (a1 > 0)
        G["W1a"] = zk1[:, A].T @ g_a1
        G["W1c"] = c.T @ g_a1
        G["b1"] = g_a1.sum(0)
        g_zk1[:, A] += g_a1 @ L["W1a"].T
        gz = g_zk1
        grads[k] = G
    return grads


# ---------------------------------------------------------------------------
# Conditioning of the ttbar sampler: 16 measured-momentum features per item
# (event record, jet permutation), in units of 100 GeV, in the frame rotated
# about the beam axis so that the lepton has phi = 0. Massless objects:
# p = E (cos phi / cosh eta, sin phi / cosh eta, tanh eta).
# Order: lepton (px, pz); the jets assigned to b, bbar, d, ubar, each
# (px, py, pz); missing pT (x, y). Record layout: object o at [4o .. 4o+3] =
# (E, eta, phi, kind), lepton o = 0, jets o = 1..4, missing pT at [24], [25];
# permutation p (0..23) = the p-th lexicographic ordering of the 4 jets.
# ---------------------------------------------------------------------------
def _momentum(E, eta, phi):
    return E * np.array([np.cos(phi) / np.cosh(eta), np.sin(phi) / np.cosh(eta), np.tanh(eta)])


def features(rec, perm):
    import itertools
    rec = np.asarray(rec, dtype=np.float64)
    order = list(itertools.permutations(range(4)))[perm]
    phil = rec[2]
    R = np.array([[np.cos(phil), np.sin(phil), 0.0],      # rotation by -phi_l about z
                  [-np.sin(phil), np.cos(phil), 0.0],
                  [0.0, 0.0, 1.0]])
    pl = R @ _momentum(rec[0], rec[1], rec[2])
    out = [pl[0], pl[2]]
    for k in range(4):
        o = 1 + order[k]
        pj = R @ _momentum(rec[4 * o], rec[4 * o + 1], rec[4 * o + 2])
        out += list(pj)
    met = R @ np.array([rec[24], rec[25], 0.0])
    out += [met[0], met[1]]
    return np.array(out) / 100.0
