"""Exact detector moments of a noisy circuit from the oracle's Pauli frames
(test helper).

The oracle's frames (oracle/frame.py) give which raw error bits flip which
detector (Sec. "Detectors"); the flips of a multi-bit outcome are the XOR of
its bits' flips, and the channels are independent, so a detector that is the
XOR of channel events has P(1) = (1 - prod_c (1 - 2 q_c)) / 2.  The same
formula on the XOR of two detectors gives P(d_a XOR d_b = 1) and so their
exact covariance.  The chi-square statistic weighs a vector of sampled rates
by that covariance.
"""
import numpy as np

from oracle import circuit as ocirc
from oracle import frame


def exact_moments(text):
    c = ocirc.parse(text)
    flips = frame.detector_flips(c)
    D = c.num_detectors
    F = np.array([fd for fd, _ in flips], dtype=np.int64).reshape(-1, D)  # raw bit -> detector flips
    # accumulate log(1 - 2 q) for single detectors and for XORs of pairs
    log1 = np.zeros(D)
    log2 = np.zeros((D, D))
    for ch in c.channels:
        pr = np.array([float(x) for x in ch.probs])
        outs = np.arange(len(pr))
        bits = ((outs[:, None] >> np.arange(ch.nbits)[None, :]) & 1)       # [outcome, bit]
        pat = (bits @ F[ch.first_bit:ch.first_bit + ch.nbits]) & 1          # [outcome, detector]
        q = pr @ pat                                                        # P(channel flips d)
        both = (pat * pr[:, None]).T @ pat                                  # P(flips a and b)
        qx = q[:, None] + q[None, :] - 2.0 * both                           # P(flips a XOR b)
        log1 += np.log1p(-2.0 * q)
        log2 += np.log1p(-2.0 * qx)
    p = (1.0 - np.exp(log1)) / 2.0
    pab = (1.0 - np.exp(log2)) / 2.0                                        # P(d_a XOR d_b = 1)
    joint = (p[:, None] + p[None, :] - pab) / 2.0                           # P(d_a = d_b = 1)
    cov = joint - np.outer(p, p)
    np.fill_diagonal(cov, p * (1 - p))
    return p, cov


def chi_square(mean, n, p, cov):
    """(statistic, degrees of freedom) of sampled detector means against the
    exact rates p and covariance cov of one shot, over n shots."""
    keep = np.diag(cov) > 0
    r = (mean - p)[keep]
    C = cov[np.ix_(keep, keep)] / n
    return float(r @ np.linalg.solve(C, r)), int(keep.sum())
