"""Masked-convolution autoregressive slice proposal (oracle side, FP64).

Test infrastructure only: the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

The paper has no learned proposal; it only suggests replacing frequent
contractions by cheaper cached knowledge of typical fields (Conclusions). This
network is that cheaper proposal. It is an independence proposal inside the
same exact Metropolis-Hastings step as the tensor network (Eq. (1)), so any
positive q_theta keeps the chain exact.

Architecture (PixelCNN-style masks, van den Oord et al. 2016), on the active
region of a slice with rows r = 1..m and columns x = 0..Lc-1 in the sampler's
raster order:
  inputs  spin one-hot [d, m, Lc] (masked stream, zero padding) and
          conditioning features [d + 4, m, Lc]: log phi(v) of the held field
          (max 0), beta*J of the right, left, lower and upper bonds
  layer 1 h1 = relu(maskA3x3(onehot) + conv3x3(cond) + b1)
  layer l h_l = h_{l-1} + relu(maskB3x3(h_{l-1}) + conv3x3(cond) + b_l), l = 2..L-1
  layer L logits = maskB3x3(h_{L-1}) + conv3x3(cond) + b_L      (d channels)
  log q(s) = sum over sites of log softmax(logits)[s]
Mask A keeps the taps of the row above and the left neighbour; mask B also
keeps the centre. Convolutions are cross-correlations with zero padding.
Loss = mean over slices of -log q(s) / (m Lc); Adam (Kingma & Ba 2015).
"""
from __future__ import annotations

from typing import Dict

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def mask(kind: str) -> np.ndarray:
    mk = np.zeros((3, 3))
    for dy, dx in TAPS:
        if dy < 0 or (dy == 0 and dx < 0) or (kind == "B" and dy == 0 and dx == 0):
            mk[dy + 1, dx + 1] = 1.0
    return mk


def n_cond(d: int) -> int:
    return d + 4


def init_params(d: int, channels: int = 64, layers: int = 6, seed: int = 0, scale: float = 1.0) -> Dict[str, np.ndarray]:
    """He-style random init. Spin kernels are stored unmasked; the mask is applied in every use."""
    rng = np.random.default_rng(seed)
    cc = n_cond(d)
    P = {}
    for l in range(1, layers + 1):
        cin = d if l == 1 else channels
        cout = d if l == layers else channels
        fan = (cin * 9 + cc * 9)
        P[f"ws{l}"] = rng.standard_normal((cout, cin, 3, 3)) * scale * np.sqrt(2.0 / fan)
        P[f"wc{l}"] = rng.standard_normal((cout, cc, 3, 3)) * scale * np.sqrt(2.0 / fan)
        P[f"b{l}"] = np.zeros(cout)
    return P


def n_layers(P) -> int:
    return sum(1 for k in P if k.startswith("ws"))


def cond_features(phi: np.ndarray, Jh: np.ndarray, Jv: np.ndarray, beta: float, ring: bool, j_scale: float) -> np.ndarray:
    """[d + 4, m, Lc] conditioning input from the slice's field factors and couplings."""
    m, Lc, d = phi.shape
    with np.errstate(divide="ignore"):
        lphi = np.log(phi)
    lphi = np.maximum(lphi, -30.0)
    bj_h = beta * j_scale * Jh.astype(np.float64)        # bond (r,x)->(r,x+1), wrap on rings
    bj_v = beta * j_scale * Jv.astype(np.float64)        # bond (r,x)->(r+1,x)
    right = bj_h.copy()
    left = np.zeros_like(bj_h)
    left[:, 1:] = bj_h[:, :-1]
    if ring:
        left[:, 0] = bj_h[:, Lc - 1]
    else:
        right[:, Lc - 1] = 0.0
    down = bj_v.copy()
    down[m - 1, :] = 0.0
    up = np.zeros_like(bj_v)
    up[1:, :] = bj_v[:-1, :]
    out = np.zeros((d + 4, m, Lc))
    out[:d] = np.transpose(lphi, (2, 0, 1))
    out[d], out[d + 1], out[d + 2], out[d + 3] = right, left, down, up
    return out


def conv(W: np.ndarray, x: np.ndarray, mk=None) -> np.ndarray:
    """out[o, r, c] = sum_{i, dy, dx} W[o, i, dy+1, dx+1] * x[i, r+dy, c+dx] (zero padding)."""
    if mk is not None:
        W = W * mk
    cin, m, L = x.shape
    xp = np.zeros((cin, m + 2, L + 2))
    xp[:, 1:m + 1, 1:L + 1] = x
    out = np.zeros((W.shape[0], m, L))
    for dy, dx in TAPS:
        out += np.einsum("oi,irc->orc", W[:, :, dy + 1, dx + 1], xp[:, 1 + dy:1 + dy + m, 1 + dx:1 + dx + L])
    return out


def conv_backward(W: np.ndarray, x: np.ndarray, gout: np.ndarray, mk=None):
    """Gradients of conv() with respect to W (masked) and x."""
    Wm = W if mk is None else W * mk
    cin, m, L = x.shape
    xp = np.zeros((cin, m + 2, L + 2))
    xp[:, 1:m + 1, 1:L + 1] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for dy, dx in TAPS:
        sl = xp[:, 1 + dy:1 + dy + m, 1 + dx:1 + dx + L]
        gW[:, :, dy + 1, dx + 1] = np.einsum("orc,irc->oi", gout, sl)
        gxp[:, 1 + dy:1 + dy + m, 1 + dx:1 + dx + L] += np.einsum("oi,orc->irc", Wm[:, :, dy + 1, dx + 1], gout)
    if mk is not None:
        gW = gW * mk
    return gW, gxp[:, 1:m + 1, 1:L + 1]


def onehot(s: np.ndarray, d: int) -> np.ndarray:
    return np.stack([(s == v).astype(np.float64) for v in range(d)])


def log_softmax(z: np.ndarray) -> np.ndarray:
    mx = z.max(axis=0, keepdims=True)
    return z - mx - np.log(np.exp(z - mx).sum(axis=0, keepdims=True))


def forward(P, cond: np.ndarray, s: np.ndarray):
    """Teacher-forced pass: logits [d, m, Lc] of every site given the spins before it, plus a cache."""
    nl = n_layers(P)
    d = P[f"ws{nl}"].shape[0]
    mA, mB = mask("A"), mask("B")
    h = onehot(s, d)
    cache = {"x0": h}
    for l in range(1, nl + 1):
        z = conv(P[f"ws{l}"], h, mA if l == 1 else mB) + conv(P[f"wc{l}"], cond) + P[f"b{l}"][:, None, None]
        cache[f"z{l}"] = z
        if l == nl:
            h = z
        elif l == 1:
            h = np.maximum(z, 0.0)
        else:
            h = h + np.maximum(z, 0.0)
        cache[f"x{l}"] = h
    return h, cache


def logq(P, cond, s) -> float:
    logits, _ = forward(P, cond, s)
    lp = log_softmax(logits)
    return float(np.sum(np.take_along_axis(lp, s[None].astype(np.int64), axis=0)))


def loss_and_grads(P, conds, spins):
    """Mean over the batch of -log q(s) / n_sites and its gradient for every parameter."""
    nl = n_layers(P)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    total = 0.0
    B = len(spins)
    mA, mB = mask("A"), mask("B")
    for cond, s in zip(conds, spins):
        s = s.astype(np.int64)
        logits, cache = forward(P, cond, s)
        n = s.size
        lp = log_softmax(logits)
        total += -float(np.sum(np.take_along_axis(lp, s[None], axis=0))) / n
        g = np.exp(lp)
        g -= onehot(s, logits.shape[0])
        g /= (n * B)                                   # d loss / d logits
        for l in range(nl, 0, -1):
            if l == nl:
                gz = g
            elif l == 1:
                gz = g * (cache[f"z{l}"] > 0)
            else:
                gz = g * (cache[f"z{l}"] > 0)
            hin = cache[f"x{l - 1}"]
            gWs, gh = conv_backward(P[f"ws{l}"], hin, gz, mA if l == 1 else mB)
            gWc, _ = conv_backward(P[f"wc{l}"], cond, gz)
            G[f"ws{l}"] += gWs
            G[f"wc{l}"] += gWc
            G[f"b{l}"] += gz.sum(axis=(1, 2))
            # residual: h_l = h_{l-1} + relu(z_l) for 2 <= l < nl
            g = gh + (g if 2 <= l < nl else 0.0)
    return total / B, G


def sample(P, cond, uniforms):
    """Ancestral draw in raster order; each conditional from a forward pass on the partial slice."""
    d = P[f"ws{n_layers(P)}"].shape[0]
    m, Lc = cond.shape[1:]
    s = np.zeros((m, Lc), dtype=np.int64)
    lq = 0.0
    for r in range(m):
        for x in range(Lc):
            logits, _ = forward(P, cond, s)
            p = np.exp(log_softmax(logits)[:, r, x])
            cdf, v = 0.0, d - 1
            for cand in range(d):
                cdf += p[cand]
                if uniforms[r, x] < cdf:
                    v = cand
                    break
            s[r, x] = v
            lq += float(np.log(p[v]))
    return s, lq


class Adam:
    """Adam of Kingma & Ba (2015) with bias correction."""

    def __init__(self, P, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in P.items()}
        self.v = {k: np.zeros_like(v) for k, v in P.items()}
        self.t = 0

    def step(self, P, G):
        self.t += 1
        for k in P:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * G[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * G[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            P[k] = P[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
