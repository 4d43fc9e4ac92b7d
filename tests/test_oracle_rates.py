"""The oracle's sampled detector rates against their exact values (CPU).

The exact moments come from the circuit through the oracle's Pauli frames
(tests/rates.py), independently of the compiled program; the samples come
from the oracle evaluator running the compiled program of the d=3 surface
code with an injected T, in both noise-sampling modes.  Agreement (chi-square
p > 0.01) ties the compiled channels, their reduction and the oracle's
sampling rules to the circuit's noise model.
"""
import numpy as np
import pytest

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram
from tests.rates import chi_square, exact_moments

scipy_stats = pytest.importorskip("scipy.stats")


@pytest.mark.parametrize("noise", [0, 1])
def test_oracle_detector_rates_chi_square(tmp_path, noise):
    text = Wk.config1_circuit(p=1e-2)
    prog = T.Program(text)
    prog.set_noise_sampling(noise)
    path = str(tmp_path / "c1.prog")
    prog.save(path)
    N = 30_000
    det = OracleProgram(path).sample(3 + noise, 0, N)["det"]
    D = prog.info["num_detectors"]
    bits = np.unpackbits(det.view(np.uint8).reshape(N, -1), axis=1, bitorder="little")[:, :D]
    p, cov = exact_moments(text)
    stat, df = chi_square(bits.mean(axis=0, dtype=np.float64), N, p, cov)
    assert scipy_stats.chi2.sf(stat, df=df) > 0.01, (noise, stat, df)
    # and a wrong noise strength is rejected by the same statistic
    p2, cov2 = exact_moments(Wk.config1_circuit(p=1.2e-2))
    stat2, _ = chi_square(bits.mean(axis=0, dtype=np.float64), N, p2, cov2)
    assert scipy_stats.chi2.sf(stat2, df=df) < 1e-6
