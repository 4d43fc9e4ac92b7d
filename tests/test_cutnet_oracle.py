"""Pins of the cut-order network oracle and host-side checks of the
cut-order entry points (no GPU)."""
import math

import numpy as np
import pytest

import paper_2604_01059_gb300 as T
from oracle import cutnet as O
from tests.cutgraphs import random_batch, random_params


def test_parameter_layout_matches_library():
    assert T.tsim_cut_num_params() == O.NPARAM == 25793
    assert T.CUT_FEATURES == O.F


def test_bf16_rounding_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 20000),
                        # exact ties: halfway between two bf16 values, both parities of the kept bit
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0],
                                 np.float32)]).astype(np.float32)
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16_round(a), want)


def _hand_params():
    p = np.zeros(O.NPARAM, np.float32)
    p[0 * O.H + 0] = 1.0                       # W_in[0][0]
    for l in range(O.LAYERS):
        o = O.OFF_L + l * O.LSZ
        p[o + 0] = 2.0                         # Ws_l[0][0]
        p[o + O.H * O.H + 0] = 1.0             # Wn_l[0][0]
    p[O.OFF_WO + 0] = 1.0                      # w_o[0]
    p[O.OFF_WO + O.H] = 0.5                    # b_o
    return p


def _hand_graph():
    # nodes 0 - 1 joined, node 2 isolated; feature 0 = 1, 3, 2
    x = np.zeros((3, O.F), np.float32)
    x[:, 0] = [1, 3, 2]
    return x, np.array([0, 1, 2, 2], np.int32), np.array([1, 0], np.int32)


def test_hand_worked_example():
    # hidden unit 0 only: H0 = x0 = (1, 3, 2); each layer h' = 2h + mean of
    # neighbours: (5, 7, 4), (17, 19, 8), (53, 55, 16); s = h + 0.5
    s = O.forward(_hand_params(), *_hand_graph())
    np.testing.assert_array_equal(s, [53.5, 55.5, 16.5])


def test_zero_weights_give_output_bias():
    p = np.zeros(O.NPARAM, np.float32)
    p[-1] = 0.75
    x, rp, col, _, _ = random_batch(1, 3)
    np.testing.assert_array_equal(O.forward(p, x, rp, col), np.full(len(rp) - 1, 0.75))


def test_permutation_equivariance():
    x, rp, col, _, _ = random_batch(2, 1, n_min=25, n_max=25)
    p = random_params(3, O.NPARAM)
    n = len(rp) - 1
    perm = np.random.default_rng(4).permutation(n)        # new node i is old node perm[i]
    inv = np.argsort(perm)
    rows, cols = [0], []
    for i in range(n):
        old = perm[i]
        cols.extend(sorted(inv[col[rp[old]:rp[old + 1]]]))
        rows.append(len(cols))
    s0 = O.forward(p, x, rp, col)
    s1 = O.forward(p, x[perm], np.array(rows), np.array(cols))
    np.testing.assert_allclose(s1, s0[perm], rtol=1e-12, atol=1e-12)


def test_gradient_matches_central_differences():
    x, rp, col, y, go = random_batch(5, 3, n_min=4, n_max=9)
    p = random_params(6, O.NPARAM).astype(np.float64)
    L, g = O.loss_grad(p, x, rp, col, y, go, bf16=False)
    assert L == pytest.approx(O.loss(p, x, rp, col, y, go, bf16=False), rel=1e-12)
    rng = np.random.default_rng(7)
    # every block of the layout: W_in, b_in, each layer's Ws, Wn, b, w_o, b_o
    idx = list(rng.choice(O.F * O.H, 10, replace=False)) + list(O.F * O.H + rng.choice(O.H, 5, replace=False))
    for l in range(O.LAYERS):
        o = O.OFF_L + l * O.LSZ
        idx += list(o + rng.choice(2 * O.H * O.H + O.H, 20, replace=False))
    idx += list(O.OFF_WO + rng.choice(O.H, 5, replace=False)) + [O.NPARAM - 1]
    h = 1e-6
    for i in idx:
        q = p.copy(); q[i] += h
        lp = O.loss(q, x, rp, col, y, go, bf16=False)
        q[i] -= 2 * h
        lm = O.loss(q, x, rp, col, y, go, bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_loss_ignores_per_graph_offsets():
    # the loss compares centred scores: the output bias has zero gradient and
    # shifting every label of one graph by a constant changes nothing
    x, rp, col, y, go = random_batch(8, 4)
    p = random_params(9, O.NPARAM)
    L, g = O.loss_grad(p, x, rp, col, y, go)
    assert abs(g[-1]) < 1e-9 * max(1.0, np.abs(g).max())
    y2 = y.copy()
    y2[go[1]:go[2]] += 5.0
    assert O.loss(p, x, rp, col, y2, go) == pytest.approx(L, rel=1e-12)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = O.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    # step 1: m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)
    want = [-0.01 * 0.5 / (0.5 + 1e-8), 0.01 * 2.0 / (2.0 + 1e-8), -0.01 * 1e-3 / (1e-3 + 1e-8), 0.0]
    np.testing.assert_allclose(p, want, rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_init_params_are_seeded_he_uniform():
    a, b, c = T.tsim_cut_init_params(1), T.tsim_cut_init_params(1), T.tsim_cut_init_params(2)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    W = O.unpack(a, bf16=False)
    assert np.abs(W["W_in"]).max() <= math.sqrt(6 / O.F)
    assert np.abs(W["Ws0"]).max() <= math.sqrt(6 / (2 * O.H))
    assert W["b_in"].any() == False and W["b_o"] == 0.0
    # uniform(-b, b) has standard deviation b / sqrt(3)
    assert W["Ws1"].std() == pytest.approx(math.sqrt(6 / (2 * O.H)) / math.sqrt(3), rel=0.05)


def test_cut_entry_points_reject_bad_graphs():
    p = np.zeros(O.NPARAM, np.float32)
    x = np.zeros((2, O.F), np.float32)
    with pytest.raises(T.TsimError) as e:
        T.tsim_cut_forward(p, x, np.array([0, 2, 1], np.int32), np.array([1, 0], np.int32))
    assert e.value.code == 7                                   # rowptr not monotone
    with pytest.raises(T.TsimError) as e:
        T.tsim_cut_forward(p, x, np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32))
    assert e.value.code == 7                                   # neighbour out of range
    y = np.zeros(2, np.float32)
    with pytest.raises(T.TsimError) as e:                      # edge 0->1 without 1->0
        T.tsim_cut_loss_grad(p, x, np.array([0, 1, 1], np.int32), np.array([1], np.int32), y, [0, 2])
    assert e.value.code == 7
    with pytest.raises(T.TsimError) as e:                      # graph offsets do not end at n
        T.tsim_cut_loss_grad(p, x, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), y, [0, 1])
    assert e.value.code == 7


def test_dataset_file_structure(tmp_path):
    path = tmp_path / "d.bin"
    T.tsim_cut_dataset(3, 6, 4, 8, 64, 4, path)
    x, rp, col, y, go = T.read_cut_dataset(str(path))
    n = len(rp) - 1
    assert len(go) == 7 and go[-1] == n and x.shape == (n, O.F)
    # symmetric adjacency inside each graph, no self loops
    edges = {(v, int(u)) for v in range(n) for u in col[rp[v]:rp[v + 1]]}
    assert all((u, v) in edges and u != v for v, u in edges)
    g_of = np.searchsorted(go, np.arange(n), side="right") - 1
    assert all(g_of[v] == g_of[u] for v, u in edges)
    # features: flags agree with the phase one-hot; degree feature matches the adjacency
    lam = x[:, 3:11].argmax(axis=1)
    assert (x[:, 3:11].sum(axis=1) == 1).all()
    np.testing.assert_array_equal(x[:, 0], lam & 1)
    np.testing.assert_allclose(x[:, 11], np.log1p(np.diff(rp)), rtol=1e-6)
    # labels sit on non-Clifford spiders only, and are log2 of term counts <= 2 * budget
    lab = ~np.isnan(y)
    assert lab.any() and (x[lab, 0] == 1).all()
    counts = np.exp2(y[lab].astype(np.float64))
    np.testing.assert_allclose(counts, np.round(counts), rtol=1e-5)
    assert counts.min() >= 1 and counts.max() <= 128
    # the same seed writes the same file
    T.tsim_cut_dataset(3, 6, 4, 8, 64, 4, tmp_path / "e.bin")
    assert path.read_bytes() == (tmp_path / "e.bin").read_bytes()


def test_learned_without_model_compiles_heuristic_program(tmp_path):
    from paper_2604_01059_gb300 import workloads as Wk
    T.tsim_cut_model_set(None)
    text = Wk.config1_circuit()
    a = T.Program(text, decomp=T.DECOMP_HEURISTIC)
    b = T.Program(text, decomp=T.DECOMP_LEARNED)
    a.save(tmp_path / "a.prog")
    b.save(tmp_path / "b.prog")
    assert (tmp_path / "a.prog").read_bytes() == (tmp_path / "b.prog").read_bytes()
