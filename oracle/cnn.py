"""FP64 CPU reference of the learned elimination proposal network.

TEST INFRASTRUCTURE.  Only the tests may import this module; the library never
does.  The network (an extension, not in the paper): five 3x3 convolutions with
zero padding (6 -> 32, then 32 -> 32 channels), GELU (exact, with erf) after
each, a 1x1 head (32 -> 1) and a sigmoid; loss = mean weighted binary
cross-entropy.  Parameters use the flat layout W1 b1 W2 b2 ... W5 b5 Wh bh.
Backward follows the chain rule written out per layer.
"""
import numpy as np
from scipy.special import erf

C = 32
CIN0 = 6
LAYERS = 5


def layout():
    """[(name, shape)] in flat order."""
    out = []
    cin = CIN0
    for l in range(LAYERS):
        out.append((f"W{l + 1}", (C, cin, 3, 3)))
        out.append((f"b{l + 1}", (C,)))
        cin = C
    out.append(("Wh", (C,)))
    out.append(("bh", (1,)))
    return out


def num_params():
    return sum(int(np.prod(s)) for _, s in layout())


def unflatten(p):
    p = np.asarray(p, dtype=np.float64)
    d, o = {}, 0
    for name, shape in layout():
        n = int(np.prod(shape))
        d[name] = p[o:o + n].reshape(shape)
        o += n
    return d


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in layout()])


def conv3x3(x, W, b=None):
    """out[b, o, y, x] = b[o] + sum_{c, ky, kx} W[o, c, ky, kx] xpad[b, c, y + ky, x + kx]."""
    B, Cin, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((B, W.shape[0], H, Wd))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + H, kx:kx + Wd]                  # (B, Cin, H, W)
            out += np.einsum("oc,bchw->bohw", W[:, :, ky, kx], patch)
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv3x3_weight_grad(x, dz):
    """dW[o, c, ky, kx] = sum_{b, y, x} dz[b, o, y, x] xpad[b, c, y + ky, x + kx]."""
    B, Cin, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dW = np.zeros((dz.shape[1], Cin, 3, 3))
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dz, xp[:, :, ky:ky + H, kx:kx + Wd])
    return dW


def conv3x3_input_grad(dz, W):
    """dx[b, c, y, x] = sum_{o, ky, kx} W[o, c, ky, kx] dz[b, o, y - ky + 1, x - kx + 1]."""
    B, O, H, Wd = dz.shape
    dzp = np.pad(dz, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dx = np.zeros((B, W.shape[1], H, Wd))
    for ky in range(3):
        for kx in range(3):
            # output pixel (y, x) saw input (y + ky - 1, x + kx - 1)
            patch = dzp[:, :, 2 - ky:2 - ky + H, 2 - kx:2 - kx + Wd]
            dx += np.einsum("oc,bohw->bchw", W[:, :, ky, kx], patch)
    return dx


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, x):
    """Returns (p, cache); x: (B, 6, H, W)."""
    P = unflatten(params)
    a = np.asarray(x, dtype=np.float64)
    cache = {"in": [], "pre": []}
    for l in range(LAYERS):
        cache["in"].append(a)
        z = conv3x3(a, P[f"W{l + 1}"], P[f"b{l + 1}"])
        cache["pre"].append(z)
        a = gelu(z)
    zh = np.einsum("c,bchw->bhw", P["Wh"], a) + P["bh"][0]
    cache["last"] = a
    cache["zh"] = zh
    return 1.0 / (1.0 + np.exp(-zh)), cache


def loss_and_grad(params, x, labels, pos_weight=1.0):
    """Mean weighted binary cross-entropy and its gradient (flat)."""
    P = unflatten(params)
    p, cache = forward(params, x)
    y = np.asarray(labels, dtype=np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    zh = cache["zh"]
    logp = -np.logaddexp(0.0, -zh)
    log1mp = -np.logaddexp(0.0, zh)
    n = y.size
    loss = float(-np.sum(w * (y * logp + (1.0 - y) * log1mp)) / n)
    dzh = w * (p - y) / n                                          # d loss / d zh
    g = {}
    a = cache["last"]
    g["Wh"] = np.einsum("bhw,bchw->c", dzh, a)
    g["bh"] = np.array([dzh.sum()])
    da = dzh[:, None, :, :] * P["Wh"][None, :, None, None]
    for l in reversed(range(LAYERS)):
        dz = da * gelu_grad(cache["pre"][l])
        g[f"W{l + 1}"] = conv3x3_weight_grad(cache["in"][l], dz)
        g[f"b{l + 1}"] = dz.sum(axis=(0, 2, 3))
        if l > 0:
            da = conv3x3_input_grad(dz, P[f"W{l + 1}"])
    return loss, flatten(g)
