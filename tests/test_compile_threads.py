"""The compiler decomposes a program's marginals on helper threads shared by
concurrent compilations.  Each marginal's terms must not depend on which
thread made them or on what else was compiling: the same circuit compiled
alone, twice, and from several Python threads at once gives byte-identical
program files; the program-wide term budget still rejects a program whose
marginals are individually within their own budget."""
from concurrent.futures import ThreadPoolExecutor

import pytest

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk


def _text(prog, path):
    prog.save(str(path))
    return open(str(path)).read()


def test_threaded_compile_is_deterministic(tmp_path):
    circuits = [Wk.config3_circuit(), Wk.config2_circuit(p=1e-3)] + \
        [txt for txt, _ in Wk.config5_pool(3, t_range=(20, 28))]
    alone = [_text(T.Program(c), tmp_path / f"a{k}.prog") for k, c in enumerate(circuits)]
    again = [_text(T.Program(c), tmp_path / f"b{k}.prog") for k, c in enumerate(circuits)]
    assert alone == again
    with ThreadPoolExecutor(max_workers=4) as ex:
        progs = list(ex.map(T.Program, circuits))
    together = [_text(p, tmp_path / f"c{k}.prog") for k, p in enumerate(progs)]
    assert together == alone


def test_program_budget_counts_all_marginals():
    # the colour-code check has 14 marginals; a program budget below their
    # sum but above any one's terms must still reject the program
    text = Wk.config3_circuit()
    whole = T.Program(text).info["total_terms"]
    per_table = max(T.Program(text).table_terms())
    assert per_table < whole - 1
    with pytest.raises(T.TsimError) as e:
        T.Program(text, total_budget=whole - 1)
    assert e.value.code == 3
    assert T.Program(text, total_budget=whole).info["total_terms"] == whole
