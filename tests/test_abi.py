"""The C-ABI library builds, loads and exports every entry point that
include/tsim.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import paper_2604_01059_gb300 as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tsim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsim_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = T.load_library()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/tsim.h but not exported"
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_status_codes_and_errors():
    with __import__("pytest").raises(T.TsimError) as e:
        T.tsim_compile("FOO 0\n")
    assert e.value.code == 2 and "FOO" in str(e.value)
    with __import__("pytest").raises(T.TsimError) as e:
        T.tsim_compile("H 0\nCX 0\n")
    assert e.value.code == 1
    with __import__("pytest").raises(T.TsimError) as e:
        T.tsim_compile("X_ERROR(1.5) 0\n")
    assert e.value.code == 1


def test_rewrite_rules_selftest():
    # every rewrite step and both decomposition policies preserve the
    # brute-force value of random small parameterised diagrams
    T.tsim_selftest_rules(seed=123, iterations=400)


def test_program_save_load_roundtrip(tmp_path):
    from paper_2604_01059_gb300 import workloads as Wk
    p = T.Program(Wk.config1_circuit())
    a = str(tmp_path / "a.prog")
    b = str(tmp_path / "b.prog")
    p.save(a)
    q = T.Program.load(a)
    q.save(b)
    assert open(a).read() == open(b).read()
    assert q.info == p.info


def test_chi_budget_is_enforced():
    from paper_2604_01059_gb300 import workloads as Wk
    with __import__("pytest").raises(T.TsimError) as e:
        T.tsim_compile(Wk.config2_circuit(), chi_budget=10)
    assert e.value.code == 3


def test_config4_generator_is_seeded_and_in_range():
    from oracle import circuit as oc
    from paper_2604_01059_gb300 import workloads as Wk
    a = Wk.config4_batch(n=8, seed=3)
    b = Wk.config4_batch(n=8, seed=3)
    assert a == b
    for txt, shots in a:
        c = oc.parse(txt)
        assert 20 <= c.num_qubits <= 60 and 1_000 <= shots <= 1_000_000
        assert 4 <= Wk.count_t(txt) <= 40
        assert c.num_detectors == c.num_qubits and c.num_observables == 1


def test_config5_generator_is_seeded_and_in_range():
    from oracle import circuit as oc
    from paper_2604_01059_gb300 import workloads as Wk
    a = Wk.config5_pool(6, t_range=(34, 46))
    assert a == Wk.config5_pool(6, t_range=(34, 46))
    for txt, shots in a:
        c = oc.parse(txt)
        assert 3 <= c.num_qubits <= 10 and shots == 100_000
        assert 34 <= Wk.count_t(txt) <= 46
        assert c.num_detectors == 0 and c.num_measurements == c.num_qubits
