"""Oracle of the cut-order network: plain numpy in float64.

TEST INFRASTRUCTURE ONLY (see the package header).  It shares no code with
the CUDA kernels and imports nothing from the product package.

The paper leaves the choice of cutting decomposition open (Sec. "Discussion");
it prints no network, so this oracle is the definition of the network the
library documents for its learned cut order, written out layer by layer:

    H0      = relu(X W_in + b_in)
    M_l     = mean of H_l over each node's neighbours (0 for an isolated node)
    H_{l+1} = relu(H_l Ws_l + M_l Wn_l + b_l)          l = 0, 1, 2
    s       = H3 w_o + b_o

Weights are rounded to BF16 (round to nearest, ties to even) before use when
``bf16=True``; all arithmetic here is float64.  The loss is, per graph g
with the set L_g of labelled nodes (|L_g| >= 2),

    (1/G) sum_g (1/|L_g|) sum_{v in L_g} ((s_v - mean s) - (y_v - mean y))^2,

G the number of such graphs.  ``loss_grad`` returns the exact gradient of
that loss with respect to the (rounded) weights, by the chain rule applied
layer by layer; it is pinned to central differences of ``loss`` in the
tests.  Adam follows Kingma and Ba (2015), Algorithm 1.
"""
import numpy as np

F = 14
H = 64
LAYERS = 3
OFF_L = (F + 1) * H
LSZ = (2 * H + 1) * H
OFF_WO = OFF_L + LAYERS * LSZ
NPARAM = OFF_WO + H + 1


def bf16_round(a):
    """float32 values rounded to the nearest bfloat16 (ties to even), as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, bf16=True):
    """Split the flat parameter vector into named float64 arrays."""
    p = np.asarray(params)
    p = bf16_round(p) if bf16 else p.astype(np.float64)
    W = {"W_in": p[0:F * H].reshape(F, H), "b_in": p[F * H:OFF_L]}
    for l in range(LAYERS):
        o = OFF_L + l * LSZ
        W[f"Ws{l}"] = p[o:o + H * H].reshape(H, H)
        W[f"Wn{l}"] = p[o + H * H:o + 2 * H * H].reshape(H, H)
        W[f"b{l}"] = p[o + 2 * H * H:o + LSZ]
    W["w_o"] = p[OFF_WO:OFF_WO + H]
    W["b_o"] = p[OFF_WO + H]
    return W


def mean_neighbours(Hm, rowptr, col):
    """M[v] = mean of Hm[u] over the neighbours u of v, node by node."""
    n = len(rowptr) - 1
    M = np.zeros_like(Hm)
    for v in range(n):
        nb = col[rowptr[v]:rowptr[v + 1]]
        if len(nb):
            M[v] = Hm[nb].sum(axis=0) / len(nb)
    return M


def forward(params, x, rowptr, col, bf16=True, keep=False):
    W = unpack(params, bf16)
    x = np.asarray(x, dtype=np.float64).reshape(-1, F)
    Hs = [np.maximum(x @ W["W_in"] + W["b_in"], 0.0)]
    Ms = []
    for l in range(LAYERS):
        M = mean_neighbours(Hs[l], rowptr, col)
        Ms.append(M)
        Hs.append(np.maximum(Hs[l] @ W[f"Ws{l}"] + M @ W[f"Wn{l}"] + W[f"b{l}"], 0.0))
    s = Hs[-1] @ W["w_o"] + W["b_o"]
    return (s, W, x, Hs, Ms) if keep else s


def loss(params, x, rowptr, col, y, goff, bf16=True):
    s = forward(params, x, rowptr, col, bf16)
    return _loss_from_scores(s, y, goff)[0]


def _loss_from_scores(s, y, goff):
    y = np.asarray(y, dtype=np.float64)
    ds = np.zeros_like(s)
    per = []
    for g in range(len(goff) - 1):
        idx = np.arange(goff[g], goff[g + 1])
        idx = idx[~np.isnan(y[idx])]
        if len(idx) < 2:
            continue
        d = (s[idx] - s[idx].mean()) - (y[idx] - y[idx].mean())
        per.append((idx, d))
    G = len(per)
    total = 0.0
    for idx, d in per:
        total += (d * d).mean() / G
        # derivative of mean(d^2)/G; the centring terms cancel since sum(d) = 0
        ds[idx] = 2.0 * d / (len(idx) * G)
    return total, ds


def loss_grad(params, x, rowptr, col, y, goff, bf16=True):
    """(loss, gradient in the flat parameter layout), float64."""
    s, W, x, Hs, Ms = forward(params, x, rowptr, col, bf16, keep=True)
    L, ds = _loss_from_scores(s, y, goff)
    g = np.zeros(NPARAM)
    g[OFF_WO:OFF_WO + H] = Hs[-1].T @ ds
    g[OFF_WO + H] = ds.sum()
    dZ = np.outer(ds, W["w_o"]) * (Hs[-1] > 0)       # at the pre-activation of H3
    n = len(rowptr) - 1
    for l in reversed(range(LAYERS)):
        o = OFF_L + l * LSZ
        g[o:o + H * H] = (Hs[l].T @ dZ).ravel()
        g[o + H * H:o + 2 * H * H] = (Ms[l].T @ dZ).ravel()
        g[o + 2 * H * H:o + LSZ] = dZ.sum(axis=0)
        dH = dZ @ W[f"Ws{l}"].T
        dM = dZ @ W[f"Wn{l}"].T
        # M_l[v] = mean over N(v) of H_l[u]: H_l[u] receives dM[v] / deg(v)
        for v in range(n):
            nb = col[rowptr[v]:rowptr[v + 1]]
            if len(nb):
                dH[nb] += dM[v] / len(nb)
        dZ = dH * (Hs[l] > 0)
    g[0:F * H] = (x.T @ dZ).ravel()
    g[F * H:OFF_L] = dZ.sum(axis=0)
    return L, g


def adam_step(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) in float64."""
    p, g = np.asarray(params, np.float64), np.asarray(grad, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
