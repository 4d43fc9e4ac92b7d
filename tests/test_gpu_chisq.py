"""Chi-square agreement of sampled detector rates with their exact values.

The exact rate of every detector, and the covariance of every pair, follow
from the circuit alone through the oracle's Pauli frames (tests/rates.py).
10^6 GPU shots of the benchmark circuits, in both noise-sampling modes, are
compared through the covariance-weighted chi-square statistic of the rate
vector (p > 0.01).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_stats = pytest.importorskip("scipy.stats")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from tests.rates import chi_square, exact_moments

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", ["cfg1", "cfg2"])
@pytest.mark.parametrize("noise", [0, 1])
def test_detector_rates_chi_square(cfg, noise):
    text = Wk.config1_circuit(p=2e-3) if cfg == "cfg1" else Wk.config2_circuit(p=2e-3)
    prog = T.Program(text)
    prog.set_noise_sampling(noise)
    N = 1_000_000
    out = prog.sample_torch(N, 99 + noise, 0)
    T.tsim_sync()
    D = prog.info["num_detectors"]
    det = out["det"].cpu().numpy().view(np.uint8).reshape(N, -1)
    bits = np.unpackbits(det, axis=1, bitorder="little")[:, :D]
    mean = bits.mean(axis=0, dtype=np.float64)
    p, cov = exact_moments(text)
    stat, df = chi_square(mean, N, p, cov)
    pval = scipy_stats.chi2.sf(stat, df=df)
    assert pval > 0.01, (cfg, noise, stat, df)
