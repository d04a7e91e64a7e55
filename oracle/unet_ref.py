"""FP64 CPU reference of the U-Net surrogate's forward and backward pass.

TEST INFRASTRUCTURE ONLY: the GPU network (built from the library's own
tensor-core kernels) is checked against this.  Plain numpy: a 3x3
convolution is the sum over the nine taps of shifted matrix products; the
backward pass is written out by hand (the transpose of each operation) and is
itself checked against central finite differences.  Layouts follow the
library: NHWC activations, weights [9][Cout][Cin] with tap = 3 * ky + kx,
input padded to 16 channels, parameters in the library's order.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b):
    """x [B,H,W,Ci], w [9,Co,Ci], b [Co] -> [B,H,W,Co] (zero padding)."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, W, w.shape[1]))
    for t in range(9):
        ky, kx = divmod(t, 3)
        y += xp[:, ky:ky + H, kx:kx + W, :] @ w[t].T
    return y + b


def conv3x3_bwd(x, w, gy):
    """Gradients of conv3x3 w.r.t. x, w, b for output gradient gy."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for t in range(9):
        ky, kx = divmod(t, 3)
        xs = xp[:, ky:ky + H, kx:kx + W, :]
        gw[t] = np.einsum("bhwo,bhwi->oi", gy, xs)
        gxp[:, ky:ky + H, kx:kx + W, :] += gy @ w[t]
    return gxp[:, 1:H + 1, 1:W + 1, :], gw, gy.sum(axis=(0, 1, 2))


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(g, shape):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


class UNetRef:
    """levels, base channels, in/out channels; params: list of arrays in the
    library's order.

    store: applied to every activation the network keeps (the packed input,
    each convolution output after bias and ReLU, each pooled map); identity
    by default.  A network that stores activations at reduced precision is
    compared with store = that rounding, so that both take every ReLU mask
    decision on the same stored values; gradients stay unrounded here."""

    def __init__(self, levels, base, in_ch, out_ch, store=None):
        self.L, self.base, self.in_ch, self.out_ch = levels, base, in_ch, out_ch
        self.q = store if store is not None else (lambda a: a)
        self.C = [base << l for l in range(levels)]
        shapes = []
        for l in range(levels):  # encoder conv a
            shapes.append(((9, self.C[l], 16 if l == 0 else self.C[l - 1]), (self.C[l],)))
        for l in range(levels):  # encoder conv b
            shapes.append(((9, self.C[l], self.C[l]), (self.C[l],)))
        for l in range(levels - 1):  # up conv
            shapes.append(((9, self.C[l], self.C[l + 1]), (self.C[l],)))
        for l in range(levels - 1):  # decoder conv a
            shapes.append(((9, self.C[l], 2 * self.C[l]), (self.C[l],)))
        for l in range(levels - 1):  # decoder conv b
            shapes.append(((9, self.C[l], self.C[l]), (self.C[l],)))
        self.shapes = [s for pair in shapes for s in pair] + [(out_ch, base), (out_ch,)]

    def unflatten(self, flat):
        out, o = [], 0
        for s in self.shapes:
            n = int(np.prod(s))
            out.append(flat[o:o + n].reshape(s))
            o += n
        return out

    def _split(self, params):
        L = self.L
        it = iter(range(0, len(params) - 2, 2))
        ea = [(params[i], params[i + 1]) for i in [next(it) for _ in range(L)]]
        eb = [(params[i], params[i + 1]) for i in [next(it) for _ in range(L)]]
        upc = [(params[i], params[i + 1]) for i in [next(it) for _ in range(L - 1)]]
        da = [(params[i], params[i + 1]) for i in [next(it) for _ in range(L - 1)]]
        db = [(params[i], params[i + 1]) for i in [next(it) for _ in range(L - 1)]]
        return ea, eb, upc, da, db, (params[-2], params[-1])

    def forward(self, x, params):
        """x [B,H,W,in_ch] -> (y [B,H,W,out_ch], cache)."""
        L = self.L
        ea, eb, upc, da, db, head = self._split(params)
        xin = np.zeros(x.shape[:3] + (16,))
        xin[..., :self.in_ch] = x
        q = self.q
        xin = q(xin)
        c = {"xin": xin, "ea": [], "eb": [], "pool": [None], "u": [None] * L,
             "up": [None] * L, "da": [None] * L, "db": [None] * L}
        h = xin
        for l in range(L):
            a = q(relu(conv3x3(h, *ea[l])))
            bb = q(relu(conv3x3(a, *eb[l])))
            c["ea"].append(a)
            c["eb"].append(bb)
            if l < L - 1:
                h = q(pool(bb))
                c["pool"].append(h)
        d = c["eb"][L - 1]
        for l in range(L - 2, -1, -1):
            u = up(d)
            uo = q(relu(conv3x3(u, *upc[l])))
            cat = np.concatenate([uo, c["eb"][l]], axis=-1)
            a = q(relu(conv3x3(cat, *da[l])))
            bb = q(relu(conv3x3(a, *db[l])))
            c["u"][l], c["up"][l], c["cat" + str(l)], c["da"][l], c["db"][l] = u, uo, cat, a, bb
            d = bb
        c["top"] = d
        y = d @ head[0].T + head[1]
        return y, c

    def loss_and_grads(self, x, t, params):
        L = self.L
        ea, eb, upc, da, db, head = self._split(params)
        y, c = self.forward(x, params)
        n = y.size
        loss = float(((y - t) ** 2).sum() / n)
        gy = 2.0 * (y - t) / n
        g_head_w = np.einsum("bhwo,bhwc->oc", gy, c["top"])
        g_head_b = gy.sum(axis=(0, 1, 2))
        g = (gy @ head[0]) * (c["top"] > 0)
        gr = {}
        g_skip = [None] * L
        for l in range(L - 1):  # decoder, top level downwards
            gx, gw, gb = conv3x3_bwd(c["da"][l], db[l][0], g)
            gr[("db", l)] = (gw, gb)
            g = gx * (c["da"][l] > 0)
            gx, gw, gb = conv3x3_bwd(c["cat" + str(l)], da[l][0], g)
            gr[("da", l)] = (gw, gb)
            C = self.C[l]
            g_up = gx[..., :C] * (c["up"][l] > 0)
            g_skip[l] = gx[..., C:]
            gx, gw, gb = conv3x3_bwd(c["u"][l], upc[l][0], g_up)
            gr[("up", l)] = (gw, gb)
            below = c["db"][l + 1] if l + 1 < L - 1 else c["eb"][L - 1]
            g = up_bwd(gx) * (below > 0)
        g_pool = None
        for l in range(L - 1, -1, -1):  # encoder, bottom upwards
            if l < L - 1:
                g = (g_skip[l] + pool_bwd(g_pool, None)) * (c["eb"][l] > 0)
            gx, gw, gb = conv3x3_bwd(c["ea"][l], eb[l][0], g)
            gr[("eb", l)] = (gw, gb)
            g = gx * (c["ea"][l] > 0)
            inp = c["xin"] if l == 0 else c["pool"][l]
            gx, gw, gb = conv3x3_bwd(inp, ea[l][0], g)
            gr[("ea", l)] = (gw, gb)
            g_pool = gx
        grads = []
        for key in ["ea", "eb", "up", "da", "db"]:
            for l in range(L if key in ("ea", "eb") else L - 1):
                grads.extend(gr[(key, l)])
        grads.extend([g_head_w, g_head_b])
        return loss, y, grads
