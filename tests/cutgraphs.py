"""Seeded synthetic graph batches for the cut-order network tests.

Holds no arithmetic of the network: node features shaped like the
compiler's (flags, a phase one-hot, log degree, fractions), random symmetric
adjacency without self loops, and labels like the compiler's (log2 of term
counts, NaN for unlabelled nodes).
"""
import numpy as np

F = 14


def random_batch(seed, n_graphs, n_min=1, n_max=40, deg=3, label_frac=0.5):
    rng = np.random.default_rng(seed)
    xs, rows, cols, ys, goff = [], [0], [], [], [0]
    base = 0
    for _ in range(n_graphs):
        n = int(rng.integers(n_min, n_max + 1))
        adj = [set() for _ in range(n)]
        for v in range(n):
            for _ in range(deg):
                u = int(rng.integers(0, n))
                if u != v:
                    adj[v].add(u)
                    adj[u].add(v)
        x = np.zeros((n, F), np.float32)
        lam = rng.integers(0, 8, n)
        x[:, 0] = lam & 1
        x[:, 1] = (lam % 4 == 0)
        x[:, 2] = (lam % 4 == 2)
        x[np.arange(n), 3 + lam] = 1.0
        x[:, 11] = np.log1p([len(a) for a in adj])
        x[:, 12] = rng.integers(0, 2, n)
        x[:, 13] = rng.random(n)
        y = np.where(rng.random(n) < label_frac, rng.integers(0, 12, n).astype(np.float32), np.nan)
        for v in range(n):
            nb = sorted(adj[v])
            cols.extend(u + base for u in nb)
            rows.append(len(cols))
        xs.append(x)
        ys.append(y.astype(np.float32))
        base += n
        goff.append(base)
    return (np.concatenate(xs), np.array(rows, np.int32), np.array(cols, np.int32),
            np.concatenate(ys), np.array(goff, np.int32))


def random_params(seed, n, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) * scale).astype(np.float32)
