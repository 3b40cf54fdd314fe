"""CPU reference of the learned seed-set surrogate (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this network is the project's screening surrogate.
Definition (restated here, computed in float64):

  x_v   = [seed_v, beta, gamma, log(1+d_in(v)), log(1+d_out(v)), log(1+k_v), 0, 0]   (8)
          k_v = number of in-arcs of v whose source is a seed (arcs and seeds both
                counted with multiplicity: a seed listed twice counts twice)
  m_v   = mean over in-arcs u -> v of h_u (0 when d_in(v) = 0; arcs with multiplicity)
  h'_v  = ReLU(h_v Ws_l + m_v Wn_l + b_l),  l = 1, 2, 3, width 64
  p_v   = sigmoid(h3_v . w_o + b_o)
  loss  = mean_v (p_v - y_v)^2,  y_v = fraction of realizations in which v was infected

With `bf16=False` this is the plain float64 function, whose analytic gradients the tests
check against finite differences.  Evaluated on bfloat16-rounded weights and inputs (the
operands the network is given on the GPU), it is the reference the GPU's forward pass and
gradients are held to, within tolerances derived from the bfloat16 unit roundoff.

With `bf16=True` it additionally rounds the intermediate operands that the GPU rounds
before its tensor-core products (activations, aggregated means, and in the backward pass
the pre-activation gradients dz; round to nearest even).  That variant only serves as a
diagnostic: it separates accumulation-order differences from rounding differences.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
FIN = 8
LAYERS = 3

# flat parameter layout (float32 vector on the GPU side)
SHAPES = [("Ws1", (FIN, HIDDEN)), ("Wn1", (FIN, HIDDEN)), ("b1", (HIDDEN,)),
          ("Ws2", (HIDDEN, HIDDEN)), ("Wn2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("Ws3", (HIDDEN, HIDDEN)), ("Wn3", (HIDDEN, HIDDEN)), ("b3", (HIDDEN,)),
          ("wo", (HIDDEN,)), ("bo", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(row_ptr, col_idx, seeds, beta, gamma):
    n = len(row_ptr) - 1
    d_in = np.diff(np.asarray(row_ptr, dtype=np.int64))
    d_out = np.bincount(np.asarray(col_idx, dtype=np.int64), minlength=n)
    x = np.zeros((n, FIN), dtype=np.float64)
    x[np.asarray(seeds, dtype=np.int64), 0] = 1.0
    x[:, 1] = beta
    x[:, 2] = gamma
    x[:, 3] = np.log1p(d_in)
    x[:, 4] = np.log1p(d_out)
    times_seed = np.bincount(np.asarray(seeds, dtype=np.int64), minlength=n)
    dst = np.repeat(np.arange(n), d_in)
    k = np.bincount(dst, weights=times_seed[np.asarray(col_idx, dtype=np.int64)], minlength=n)
    x[:, 5] = np.log1p(k)
    return x


def _mean_agg(row_ptr, col_idx, h):
    n = len(row_ptr) - 1
    d = np.diff(np.asarray(row_ptr, dtype=np.int64))
    dst = np.repeat(np.arange(n), d)
    s = np.zeros((n, h.shape[1]))
    np.add.at(s, dst, h[np.asarray(col_idx, dtype=np.int64)])
    return s / np.maximum(d, 1)[:, None]


def _mean_agg_T(row_ptr, col_idx, g):
    """Adjoint of the mean aggregation: dh_u = sum over arcs u -> v of g_v / d_in(v)."""
    n = len(row_ptr) - 1
    d = np.diff(np.asarray(row_ptr, dtype=np.int64))
    dst = np.repeat(np.arange(n), d)
    w = g[dst] / np.maximum(d, 1)[dst][:, None]
    out = np.zeros_like(g)
    np.add.at(out, np.asarray(col_idx, dtype=np.int64), w)
    return out


def forward(theta, row_ptr, col_idx, x, bf16=True):
    """Returns p (n,) and the cache for backward."""
    P = unflatten(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = r(x)
    cache = []
    for l in (1, 2, 3):
        Ws, Wn, b = r(P[f"Ws{l}"]), r(P[f"Wn{l}"]), P[f"b{l}"]
        m = r(_mean_agg(row_ptr, col_idx, h))
        z = h @ Ws + m @ Wn + b
        hn = np.maximum(z, 0.0)
        cache.append((h, m, z))
        h = r(hn)
    wo = r(P["wo"])
    logit = h @ wo + P["bo"][0]
    p = 1.0 / (1.0 + np.exp(-logit))
    return p, (cache, h, wo)


def loss_and_grad(theta, row_ptr, col_idx, x, y, bf16=True):
    """MSE loss and its gradient w.r.t. the flat parameters (operands rounded as on the
    GPU when bf16=True; the gradient is that of the rounded forward with the rounding
    treated as identity, i.e. straight through, as the GPU computes it, with dz rounded
    where it enters a product)."""
    P = unflatten(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    n = len(row_ptr) - 1
    p, (cache, h3, wo) = forward(theta, row_ptr, col_idx, x, bf16)
    loss = float(np.mean((p - y) ** 2))
    G = {}
    dlogit = 2.0 * (p - y) / n * p * (1.0 - p)
    G["wo"] = h3.T @ dlogit
    G["bo"] = np.array([dlogit.sum()])
    dh = np.outer(dlogit, wo)
    for l in (3, 2, 1):
        h, m, z = cache[l - 1]
        Ws, Wn = r(P[f"Ws{l}"]), r(P[f"Wn{l}"])
        dz = dh * (z > 0)
        dzr = r(dz)
        G[f"Ws{l}"] = h.T @ dzr
        G[f"Wn{l}"] = m.T @ dzr
        G[f"b{l}"] = dz.sum(axis=0)
        dm = dzr @ Wn.T
        dh = dzr @ Ws.T + _mean_agg_T(row_ptr, col_idx, dm)
    return loss, flatten(G)


def init_params(seed=0, scale=None):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[0] * 2
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shp).ravel())
        elif name == "wo":
            parts.append(rng.normal(0.0, np.sqrt(1.0 / HIDDEN), size=shp).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    return np.concatenate(parts)


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; returns new arrays."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
