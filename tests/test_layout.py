"""Device table layouts, checked on the host (packing needs no GPU): which
tables take the bit-sliced layout, how they split into segments and batches,
and that the layout can be changed and queried through the C ABI."""
import pytest

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from tests.test_compile_semantics import WORKED_EXAMPLE


@pytest.fixture(scope="module")
def color_code():
    return T.Program(Wk.config3_circuit())


def _layouts(prog):
    return [prog.device_table_layout(t) for t in range(prog.info["num_tables"])]


def test_color_code_default_layout(color_code):
    # marginals of 4 terms or more (no two with equal factor lists here) are
    # sliced; each segment's batches hold 32 terms but its last one, so a
    # table has at least ceil(n / 32) batches
    for (mode, nb, rows, ops, work, real), n in zip(_layouts(color_code), color_code.table_terms()):
        assert mode == (T.TABLE_SLICED if n >= 4 else T.TABLE_SCALAR)
        if mode == T.TABLE_SLICED:
            assert (n + 31) // 32 <= nb <= (n + 31) // 32 + n // 32
            assert rows % 4 == 0 or rows >= ops / 32
            assert rows * 32 >= ops and work > rows * 32 * 3
            # without padding: at least 3 lane-operations per real row,
            # never more than the padded count
            assert 3 * ops < real <= work
        else:
            assert nb == rows == ops == work == real == 0


@pytest.mark.parametrize("seg", [256, 1024, 2048, 16384])
def test_segment_sizes(color_code, seg):
    # smaller segments only add batches (a partial batch per segment) and
    # never change which tables are sliced or how many operations they hold
    color_code.set_table_layout(4, 0, seg)
    lay = _layouts(color_code)
    color_code.set_table_layout(4, 0, 16384)
    whole = _layouts(color_code)
    for a, b in zip(lay, whole):
        assert a[0] == b[0] and a[3] == b[3]
        assert a[1] >= b[1]


def test_layout_switches(color_code):
    color_code.set_table_layout(-1)
    assert T.TABLE_SLICED not in [m for m, *_ in _layouts(color_code)]
    color_code.set_table_layout(1)
    assert all(m == T.TABLE_SLICED for m, *_ in _layouts(color_code))
    color_code.set_table_layout(4)
    with pytest.raises(T.TsimError):
        color_code.device_table_layout(color_code.info["num_tables"])


def test_worked_example_forced_sliced():
    prog = T.Program(WORKED_EXAMPLE)
    prog.set_table_layout(1, 128, 16)
    for mode, nb, rows, ops, work, real in _layouts(prog):
        assert mode == T.TABLE_SLICED and nb >= 1


def test_detector_runs_of_the_surface_code():
    # d=5 memory: the 114 detectors are X bits in output order with no
    # constant, so they pack as one run; the observable stays an entry
    prog = T.Program(Wk.config2_circuit(p=1e-3))
    entries, runs, covered = prog.device_output_stats()
    assert (entries, runs, covered) == (2, 1, 114)
    assert prog.info["num_detectors"] == 114 and prog.info["num_outputs"] == 115


def test_measurement_mode_has_no_runs():
    # runs exist only for detector / observable records
    prog = T.Program(Wk.config1_circuit(p=2e-3), mode=T.MODE_MEASUREMENTS)
    entries, runs, covered = prog.device_output_stats()
    assert runs == 0 and covered == 0 and entries == prog.info["num_outputs"]


def test_output_entries_account_for_every_output():
    # every output is one entry or part of exactly one run
    for text in (WORKED_EXAMPLE, Wk.config1_circuit(), Wk.config3_circuit()):
        prog = T.Program(text)
        entries, runs, covered = prog.device_output_stats()
        i = prog.info
        assert covered <= i["num_outputs"] and entries + covered - runs == i["num_outputs"]


@pytest.mark.parametrize("seg", [16, 64, 1536])
def test_sliced_tables_match_exact_values_small_programs(seg):
    # a host emulation of the warp-cooperative kernel, reading the packed
    # segments, batches and rows, equals each table's exact value from its
    # term list on random per-shot vectors; tiny segments force many
    # segments and parity renumberings per table
    import random
    from tests.test_compile_semantics import PHASED_CHAIN, STEANE_CHECK, _random_circuit
    texts = [WORKED_EXAMPLE, STEANE_CHECK, PHASED_CHAIN, Wk.config1_circuit()]
    for k in range(4):
        texts.append(_random_circuit(random.Random(600 + k), 5, 30, tcount=8))
    for text in texts:
        for mode in (T.MODE_DETECTORS, T.MODE_MEASUREMENTS):
            try:
                prog = T.Program(text, mode=mode)
            except T.TsimError:
                continue
            prog.set_table_layout(1, 0, seg)
            T.tsim_selftest_sliced(prog.h, seed=seg, rounds=3)


def test_sliced_tables_match_exact_values_color_code(color_code):
    color_code.set_table_layout(4, 0, 1536)
    T.tsim_selftest_sliced(color_code.h, seed=7, rounds=1)
