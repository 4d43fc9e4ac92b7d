"""GPU parity of the cut-order network kernels against the float64 oracle,
training behaviour, and exactness of learned-order programs.

Tolerances: the kernels apply the same BF16-rounded weights as the oracle and
accumulate every dot product (at most 128 + 1 terms per layer, four layers,
plus neighbour means) in FP32, so scores agree to about 1e-6 of the score
scale; 1e-4 leaves margin.  Gradients are compared per parameter block in
relative L2 norm (1e-4): an FP32 pre-activation that lands on the other side
of zero from the float64 one flips a single ReLU mask entry, which moves a
few gradient entries by a bounded amount but not a block's norm."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from oracle import cutnet as O
from oracle.evaluator import OracleProgram
from paper_2604_01059_gb300 import workloads as Wk
from tests.cutgraphs import random_batch, random_params

pytestmark = pytest.mark.gpu

BLOCKS = [("W_in", 0, O.F * O.H), ("b_in", O.F * O.H, O.OFF_L)] + [
    (f"{nm}{l}", O.OFF_L + l * O.LSZ + a, O.OFF_L + l * O.LSZ + b)
    for l in range(O.LAYERS)
    for nm, a, b in (("Ws", 0, O.H * O.H), ("Wn", O.H * O.H, 2 * O.H * O.H), ("b", 2 * O.H * O.H, O.LSZ))
] + [("w_o", O.OFF_WO, O.OFF_WO + O.H), ("b_o", O.OFF_WO + O.H, O.NPARAM)]


@pytest.mark.parametrize("seed,n_graphs,n_max", [(1, 40, 80), (2, 160, 150), (3, 1, 1)])
def test_forward_matches_oracle(seed, n_graphs, n_max):
    # (2, 160, 150): ~12k nodes, more node tiles than the dense kernels' grid
    x, rp, col, _, _ = random_batch(seed, n_graphs, n_max=n_max)
    p = random_params(seed + 10, O.NPARAM, scale=0.2)
    s = T.tsim_cut_forward(p, x, rp, col)
    want = O.forward(p, x, rp, col)
    scale = np.abs(want).max() + 1.0
    np.testing.assert_allclose(s, want, rtol=0, atol=1e-4 * scale)


def test_forward_empty_graph():
    s = T.tsim_cut_forward(np.zeros(O.NPARAM, np.float32), np.zeros((0, O.F), np.float32),
                           np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert s.shape == (0,)


@pytest.mark.parametrize("seed,n_graphs", [(4, 12), (5, 90)])
def test_loss_grad_matches_oracle(seed, n_graphs):
    x, rp, col, y, go = random_batch(seed, n_graphs, n_max=60)
    p = random_params(seed + 20, O.NPARAM, scale=0.2)
    L, g = T.tsim_cut_loss_grad(p, x, rp, col, y, go)
    Lo, go_ = O.loss_grad(p, x, rp, col, y, go)
    assert L == pytest.approx(Lo, rel=1e-4)
    # a block whose exact gradient is (near) zero is held to a floor scaled by
    # the whole gradient: the output bias b_o has gradient exactly 0, since the
    # per-graph centred loss does not change when every score shifts by b_o
    floor = 1e-6 * np.linalg.norm(go_)
    for name, a, b in BLOCKS:
        ref = go_[a:b]
        err = np.linalg.norm(g[a:b] - ref)
        assert err <= 1e-4 * np.linalg.norm(ref) + floor, name
    assert abs(go_[O.OFF_WO + O.H]) <= 1e-12 * np.linalg.norm(go_)
    assert abs(g[O.OFF_WO + O.H]) <= floor
    assert np.abs(g - go_).max() <= 1e-2 * np.abs(go_).max()


def test_adam_step_matches_oracle():
    n = O.NPARAM
    p, g = random_params(30, n), random_params(31, n)
    m, v = random_params(32, n, 0.01), np.abs(random_params(33, n, 0.01))
    p1, m1, v1 = T.tsim_cut_adam_step(p, g, m, v, 7, 1e-3)
    p2, m2, v2 = O.adam_step(p, g, m, v, 7, 1e-3)
    # float32 moments: the constants 0.9, 0.1, 0.999, 0.001 and each product
    # and sum round at 2^-24 relative to its summands, and the two summands
    # can cancel, so the bound scales with them rather than with the result
    eps = np.finfo(np.float32).eps
    g64, m64, v64 = (np.asarray(a, np.float64) for a in (g, m, v))
    assert (np.abs(m1 - m2) <= 4 * eps * (0.9 * np.abs(m64) + 0.1 * np.abs(g64)) + 1e-30).all()
    assert (np.abs(v1 - v2) <= 4 * eps * (0.999 * v64 + 0.001 * g64 * g64) + 1e-30).all()
    # the kernel returns float32 parameters: beyond the step's own relative
    # error, each updated value carries its rounding to float32, half an ulp
    err = np.abs(p1.astype(np.float64) - p2)
    assert (err <= 1e-4 * np.abs(p2 - p) + 0.5 * np.finfo(np.float32).eps * np.abs(p2) + 1e-30).all()


@pytest.fixture(scope="module")
def small_dataset(tmp_path_factory):
    path = tmp_path_factory.mktemp("cut") / "d.bin"
    T.tsim_cut_dataset(11, 96, 8, 16, 256, 8, path)
    return path


def test_training_lowers_loss_and_is_deterministic(small_dataset):
    p0 = T.tsim_cut_init_params(0)
    p1, h1 = T.tsim_cut_train(small_dataset, p0, epochs=30, batch_graphs=16, lr=1e-3, seed=1)
    p2, h2 = T.tsim_cut_train(small_dataset, p0, epochs=30, batch_graphs=16, lr=1e-3, seed=1)
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(h1, h2)
    assert np.isfinite(h1).all()
    assert h1[-5:].mean() < 0.8 * h1[:3].mean(), h1
    # the trained network's loss on the whole dataset, checked by the oracle
    x, rp, col, y, go = T.read_cut_dataset(str(small_dataset))
    L, _ = T.tsim_cut_loss_grad(p1, x, rp, col, y, go)
    assert L == pytest.approx(O.loss(p1, x, rp, col, y, go), rel=1e-4)
    assert L < O.loss(p0, x, rp, col, y, go)


def _records(prog, shots, seed, off):
    out = prog.sample_torch(shots, seed, off)
    T.tsim_sync()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("name", ["cfg1", "random"])
def test_learned_order_programs_sample_identical_records(tmp_path, small_dataset, name):
    # any cut order gives the same sum (exactness untouched): programs compiled
    # with the heuristic, single cuts and the learned order sample the same
    # records bit for bit, and the learned program matches the oracle
    p, _ = T.tsim_cut_train(small_dataset, T.tsim_cut_init_params(0), epochs=10, batch_graphs=16, seed=2)
    text = Wk.config1_circuit() if name == "cfg1" else Wk.random_clifford_t(3, n=12, depth=24, t_count=16)
    before = T.tsim_cut_policy_stats()
    T.tsim_cut_model_set(p)
    try:
        learned = T.Program(text, decomp=T.DECOMP_LEARNED)
    finally:
        T.tsim_cut_model_set(None)
    after = T.tsim_cut_policy_stats()
    assert after[1] - before[1] == after[0] - before[0] > 0          # the GPU scorer ran
    assert (after[2] - before[2]) + (after[3] - before[3]) == after[1] - before[1]
    heur = T.Program(text, decomp=T.DECOMP_HEURISTIC)
    single = T.Program(text, decomp=T.DECOMP_SINGLE_T, chi_budget=1 << 22)
    assert all(a <= b for a, b in zip(learned.table_terms(), heur.table_terms()))
    ref = _records(heur, 5000, 7, 1 << 20)
    for prog in (learned, single):
        got = _records(prog, 5000, 7, 1 << 20)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k])
    path = str(tmp_path / "l.prog")
    learned.save(path)
    o = OracleProgram(path).sample(7, 1 << 20, 600)
    for k in ("det", "obs", "accept"):
        if k in o and o[k] is not None and ref.get(k) is not None and ref[k].size:
            np.testing.assert_array_equal(ref[k][:600].view(o[k].dtype) if k != "accept" else ref[k][:600], o[k])
