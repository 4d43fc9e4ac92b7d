"""Wide per-shot vectors: surface-code memories of distance 7, 9 and 11
need X of 6, 12 and 23 64-bit words (the kernels for 8, 16 and 32 words), and
their detectors form one run spanning many words of X and of the record.
Records must equal the oracle's bit for bit (ragged launch, global shot
index crossing 2^32), alone and in a batch with a narrow program."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from oracle.evaluator import OracleProgram

pytestmark = pytest.mark.gpu

WIDE = [(7, 7, 6), (9, 9, 12), (11, 12, 23)]


def _program(d, rounds):
    return T.Program(Wk.surface_code_t_injection(d=d, rounds=rounds, p=1e-3, rotation=Wk.t_rotation_sequence(4, 1)))


def _np(t):
    return None if t is None else t.cpu().numpy()


@pytest.mark.parametrize("d,rounds,words", WIDE)
def test_wide_surface_codes_bit_exact(tmp_path, d, rounds, words):
    prog = _program(d, rounds)
    i = prog.info
    assert i["x_words"] == words and prog.device_output_stats()[1:] == (1, i["num_detectors"])
    path = str(tmp_path / "w.prog")
    prog.save(path)
    shots, seed, offset = 1999, 5, (1 << 32) - 777
    out = prog.sample_torch(shots, seed, offset)
    T.tsim_sync()
    o = OracleProgram(path).sample(seed, offset, shots)
    np.testing.assert_array_equal(_np(out["det"]).view(np.uint64), o["det"])
    np.testing.assert_array_equal(_np(out["obs"]).view(np.uint64), o["obs"])
    np.testing.assert_array_equal(_np(out["accept"]), o["accept"])


def test_batch_mixing_widths():
    progs = [_program(11, 12), T.Program(Wk.config1_circuit()), _program(7, 7)]
    shots, seeds, offs = [3000, 5000, 1], [1, 2, 3], [0, 1 << 33, 7]
    want, got = [], []
    for p, n, sd, of in zip(progs, shots, seeds, offs):
        i = p.info
        mk = lambda: (torch.zeros((n, i["det_words"]), dtype=torch.int64, device="cuda"),  # noqa: E731
                      torch.zeros((n, i["obs_words"]), dtype=torch.int64, device="cuda"),
                      torch.zeros((n,), dtype=torch.uint8, device="cuda"))
        w = mk()
        T.tsim_sample(p.h, n, sd, of, None, *w)
        want.append(w)
        got.append(mk())
    T.tsim_sync()
    for autotune in (0, 2):
        batch = T.tsim_batch_create([p.h for p in progs], shots, seeds, offs, None, [g[0] for g in got],
                                    [g[1] for g in got], [g[2] for g in got], autotune=autotune)
        try:
            T.tsim_batch_launch(batch)
            T.tsim_sync()
            for w, g in zip(want, got):
                for a, b in zip(w, g):
                    assert torch.equal(a, b)
        finally:
            T.tsim_batch_free(batch)
