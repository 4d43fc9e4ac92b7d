"""tsim_sample_noalloc -- sampling for callers that cannot allocate device
memory (code inside an allocator or memory pool it does not own, or a host
that carved up device memory in advance) -- must produce exactly the records
of tsim_sample, in both kernel variants (per-thread tables and bit-sliced
warp tables), and must refuse programs whose tables exceed its fixed array
without writing any output.

Kept in a file that pytest collects last, so that a run stopping at the first
failure has already run every other test.  It must pass on its own in a
fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2604_01059_gb300 as T
from paper_2604_01059_gb300 import workloads as Wk
from tests.test_compile_semantics import WORKED_EXAMPLE

pytestmark = pytest.mark.gpu


def _buffers(info, shots):
    meas = (torch.zeros((shots, info["meas_words"]), dtype=torch.int64, device="cuda")
            if info["mode"] == T.MODE_MEASUREMENTS and info["meas_words"] else None)
    det = torch.zeros((shots, info["det_words"]), dtype=torch.int64, device="cuda") if info["det_words"] else None
    obs = torch.zeros((shots, info["obs_words"]), dtype=torch.int64, device="cuda") if info["obs_words"] else None
    acc = torch.zeros((shots,), dtype=torch.uint8, device="cuda")
    return meas, det, obs, acc


def _call(fn_name, prog, shots, seed, offset, bufs):
    # straight through the C ABI: pointers and sizes only
    lib = T.load_library()
    fn = getattr(lib, fn_name)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = fn(ctypes.c_void_p(prog.h), ctypes.c_uint64(shots), ctypes.c_uint64(seed), ctypes.c_uint64(offset),
            *[ptr(t) for t in bufs], None)
    assert rc == 0, lib.tsim_last_error().decode()
    T.tsim_sync()
    return [None if t is None else t.cpu().numpy() for t in bufs]


def test_noalloc_matches_tsim_sample_on_consecutive_calls():
    # two calls in a row with different programs: the second overwrites the
    # shared scratch left by the first, and both must equal tsim_sample
    cases = [(T.Program(Wk.config1_circuit()), 5003, 17, 40),
             (T.Program(WORKED_EXAMPLE, mode=T.MODE_MEASUREMENTS), 4099, 3, 1 << 33)]
    want = []
    for prog, shots, seed, off in cases:
        want.append(_call("tsim_sample", prog, shots, seed, off, _buffers(prog.info, shots)))
    got = []
    for prog, shots, seed, off in cases:
        got.append(_call("tsim_sample_noalloc", prog, shots, seed, off, _buffers(prog.info, shots)))
    for w, g in zip(want, got):
        for a, b in zip(w, g):
            if a is None:
                assert b is None
            else:
                np.testing.assert_array_equal(a, b)
    # and again with the first program, after the second one used the array
    prog, shots, seed, off = cases[0]
    again = _call("tsim_sample_noalloc", prog, shots, seed, off, _buffers(prog.info, shots))
    for a, b in zip(want[0], again):
        if a is not None:
            np.testing.assert_array_equal(a, b)


def test_noalloc_sliced_tables_and_size_limit():
    # a small program forced into the bit-sliced warp layout (tables read with
    # 16-byte loads from the static array), twice in a row
    prog = T.Program(WORKED_EXAMPLE)
    prog.set_table_layout(0, 0, 16)
    assert any(prog.device_table_layout(t)[0] == 2 for t in range(prog.info["num_tables"]))
    shots, seed, off = 3001, 23, 1 << 32
    want = _call("tsim_sample", prog, shots, seed, off, _buffers(prog.info, shots))
    for _ in range(2):
        got = _call("tsim_sample_noalloc", prog, shots, seed, off, _buffers(prog.info, shots))
        for a, b in zip(want, got):
            if a is not None:
                np.testing.assert_array_equal(a, b)
    # the colour-code program: its packed tables (about 6.6 MB) exceed the
    # array, so the call is refused before any output is written
    big = T.Program(Wk.config3_circuit())
    assert big.device_bytes() > (4 << 20)
    bufs = _buffers(big.info, 64)
    for t in bufs:
        if t is not None:
            t.view(torch.uint8).fill_(0x5A)
    lib = T.load_library()
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = lib.tsim_sample_noalloc(ctypes.c_void_p(big.h), ctypes.c_uint64(64), ctypes.c_uint64(1),
                                 ctypes.c_uint64(0), *[ptr(t) for t in bufs], None)
    assert rc == 7, lib.tsim_last_error().decode()   # TSIM_ERR_ARG
    assert b"exceed" in lib.tsim_last_error()
    T.tsim_sync()
    for t in bufs:
        if t is not None:
            assert bool((t.view(torch.uint8) == 0x5A).all())
