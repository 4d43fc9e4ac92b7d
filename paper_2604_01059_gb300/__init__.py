"""GB300-native per-shot sampler for noisy Clifford+T circuits (Tsim's method).

Thin ctypes binding of the C ABI declared in ``include/tsim.h``: argument
marshalling only.  Every step of compilation runs in the native library and
every step of sampling runs in its sm_103a kernels; there is no Python or CPU
fallback -- if the native library is missing, importing the binding raises.
PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, build as _build

__all__ = [
    "TsimError", "Program", "tsim_compile", "tsim_program_info", "tsim_program_table_terms", "tsim_program_table_stats",
    "tsim_sample", "tsim_sample_host", "tsim_sample_noalloc", "tsim_sample_batch", "tsim_batch_create",
    "tsim_batch_launch", "tsim_batch_info", "tsim_batch_free", "tsim_sync", "tsim_eval_table",
    "tsim_raw_to_x", "tsim_program_save", "tsim_program_load", "tsim_program_free",
    "tsim_last_error", "tsim_selftest_rules", "tsim_measure_int_peak", "tsim_program_device_table_stats",
    "tsim_program_set_table_layout", "tsim_program_device_table_layout", "tsim_program_device_output_stats",
    "tsim_selftest_sliced", "tsim_cut_evaluate", "tsim_debug_sample", "tsim_program_set_noise_sampling", "tsim_program_noise_info",
    "tsim_program_device_bytes", "tsim_eval_table_float", "load_library",
    "MODE_DETECTORS", "MODE_MEASUREMENTS", "DECOMP_HEURISTIC", "DECOMP_LEARNED", "DECOMP_SINGLE_T", "DECOMP_PAIRS",
    "DECOMP_CAT5",
]

MODE_DETECTORS, MODE_MEASUREMENTS = 0, 1
DECOMP_HEURISTIC, DECOMP_LEARNED, DECOMP_SINGLE_T, DECOMP_PAIRS, DECOMP_CAT5 = 0, 1, 2, 3, 4

STATUS = {0: "TSIM_OK", 1: "TSIM_ERR_PARSE", 2: "TSIM_ERR_UNSUPPORTED_GATE", 3: "TSIM_ERR_CHI_BUDGET",
          4: "TSIM_ERR_OVERFLOW_BOUND", 5: "TSIM_ERR_CUDA", 6: "TSIM_ERR_OOM", 7: "TSIM_ERR_ARG",
          8: "TSIM_ERR_ZERO_PROB", 9: "TSIM_ERR_TIMEOUT", 10: "TSIM_ERR_INTERNAL"}


class TsimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class CompileOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("decomp", ctypes.c_int), ("chi_budget", ctypes.c_uint64),
                ("channel_reduction", ctypes.c_int), ("total_budget", ctypes.c_uint64)]


class ProgramInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "mode", "num_qubits", "num_measurements", "num_detectors", "num_observables",
        "num_error_bits", "num_channels", "num_f", "num_random", "num_outputs", "num_chains",
        "num_tables", "x_words")] + [
        ("total_terms", ctypes.c_uint64), ("max_terms", ctypes.c_uint64), ("max_factors", ctypes.c_int),
        ("meas_words", ctypes.c_int), ("det_words", ctypes.c_int), ("obs_words", ctypes.c_int),
        ("device_classes", ctypes.c_uint64), ("device_parities", ctypes.c_uint64), ("device_status", ctypes.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_lib_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load the native library (building it in-tree if it is absent or stale);
    safe to call from several threads at once."""
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is None:
            _lib = _load(path)
    return _lib


def _load(path):
    if path is None:
        path = _build() if not os.environ.get("TSIM_NO_BUILD") else LIB
    if not os.path.exists(path):
        raise ImportError(f"native library {path} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, u64, i32, i64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
    pp = ctypes.POINTER(vp)
    L.tsim_compile.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(CompileOpts), pp]
    L.tsim_program_info.argtypes = [vp, ctypes.POINTER(ProgramInfo)]
    L.tsim_program_table_terms.argtypes = [vp, i32, ctypes.POINTER(u64)]
    L.tsim_program_table_stats.argtypes = [vp, i32, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.tsim_sample.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp, vp]
    L.tsim_sample_host.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp, vp]
    L.tsim_sample_noalloc.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp, vp]
    L.tsim_sample_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                    ctypes.POINTER(u64), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.tsim_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                    ctypes.POINTER(u64), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), i32, pp]
    L.tsim_batch_launch.argtypes = [vp, vp]
    L.tsim_batch_info.argtypes = [vp, ctypes.POINTER(i64)]
    L.tsim_batch_free.argtypes = [vp]
    L.tsim_batch_free.restype = None
    L.tsim_sync.argtypes = [vp]
    L.tsim_eval_table.argtypes = [vp, i32, ctypes.POINTER(u64), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32)]
    L.tsim_raw_to_x.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(u64)]
    L.tsim_program_save.argtypes = [vp, ctypes.c_char_p]
    L.tsim_program_load.argtypes = [ctypes.c_char_p, pp]
    L.tsim_program_free.argtypes = [vp]
    L.tsim_program_free.restype = None
    L.tsim_last_error.restype = ctypes.c_char_p
    L.tsim_selftest_rules.argtypes = [u64, i32]
    L.tsim_measure_int_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
    L.tsim_program_device_table_stats.argtypes = [vp, i32, ctypes.POINTER(u64)]
    L.tsim_program_set_table_layout.argtypes = [vp, i64, i32, i32]
    L.tsim_program_device_table_layout.argtypes = [vp, i32, ctypes.POINTER(u64)]
    L.tsim_program_device_output_stats.argtypes = [vp, ctypes.POINTER(u64)]
    L.tsim_selftest_sliced.argtypes = [vp, u64, i32]
    L.tsim_debug_sample.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp, ctypes.POINTER(u64), i32,
                                    ctypes.POINTER(i64), vp]
    L.tsim_program_set_noise_sampling.argtypes = [vp, i32]
    L.tsim_program_noise_info.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.tsim_program_device_bytes.argtypes = [vp, ctypes.POINTER(u64)]
    L.tsim_eval_table_float.argtypes = [vp, i32, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double)]
    L.tsim_cut_num_params.argtypes = []
    L.tsim_cut_init_params.argtypes = [u64, vp]
    L.tsim_cut_dataset.argtypes = [u64, i32, i32, i32, u64, i32, ctypes.c_char_p]
    L.tsim_cut_forward.argtypes = [vp, i32, vp, vp, vp, vp]
    L.tsim_cut_loss_grad.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp, vp, vp]
    L.tsim_cut_adam_step.argtypes = [vp, vp, vp, vp, i32, ctypes.c_float]
    L.tsim_cut_train.argtypes = [ctypes.c_char_p, i32, i32, ctypes.c_float, u64, vp, vp]
    L.tsim_cut_model_set.argtypes = [vp]
    L.tsim_cut_policy_stats.argtypes = [vp]
    L.tsim_cut_evaluate.argtypes = [u64, i32, i32, i32, u64, vp]
    for n in ("tsim_compile", "tsim_program_info", "tsim_program_table_terms", "tsim_program_table_stats", "tsim_sample",
              "tsim_sample_host", "tsim_sample_noalloc", "tsim_sample_batch", "tsim_batch_create",
              "tsim_batch_launch", "tsim_batch_info", "tsim_sync", "tsim_eval_table", "tsim_raw_to_x",
              "tsim_program_save", "tsim_program_load", "tsim_selftest_rules", "tsim_measure_int_peak",
              "tsim_program_device_table_stats", "tsim_program_set_table_layout",
              "tsim_program_device_table_layout", "tsim_program_device_output_stats", "tsim_selftest_sliced",
              "tsim_debug_sample", "tsim_program_set_noise_sampling", "tsim_program_noise_info",
              "tsim_program_device_bytes", "tsim_eval_table_float",
              "tsim_cut_num_params",
              "tsim_cut_init_params",
              "tsim_cut_dataset", "tsim_cut_forward", "tsim_cut_loss_grad", "tsim_cut_adam_step", "tsim_cut_train",
              "tsim_cut_model_set", "tsim_cut_policy_stats", "tsim_cut_evaluate"):
        getattr(L, n).restype = ctypes.c_int
    return L


def _check(rc):
    if rc != 0:
        raise TsimError(rc, load_library().tsim_last_error().decode(errors="replace"))


def tsim_last_error() -> str:
    return load_library().tsim_last_error().decode(errors="replace")


def tsim_compile(text: str, mode=MODE_DETECTORS, decomp=DECOMP_HEURISTIC, chi_budget=0, channel_reduction=True,
                 total_budget=0):
    """Compile a Stim-format circuit; returns an opaque program handle (int)."""
    L = load_library()
    b = text.encode()
    opts = CompileOpts(mode, decomp, chi_budget, 1 if channel_reduction else 0, total_budget)
    h = ctypes.c_void_p()
    _check(L.tsim_compile(b, len(b), ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def tsim_program_info(h) -> dict:
    info = ProgramInfo()
    _check(load_library().tsim_program_info(h, ctypes.byref(info)))
    return info.as_dict()


def tsim_program_table_terms(h, t) -> int:
    n = ctypes.c_uint64()
    _check(load_library().tsim_program_table_terms(h, t, ctypes.byref(n)))
    return n.value


def tsim_program_table_stats(h, t):
    """(terms, total factors) of marginal table t."""
    n, f = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().tsim_program_table_stats(h, t, ctypes.byref(n), ctypes.byref(f)))
    return n.value, f.value


def _ptr(t):
    return None if t is None else t.data_ptr()


def tsim_sample(h, shots, seed, shot_offset=0, meas=None, det=None, obs=None, accept=None, stream=None):
    """Launch sampling into caller-owned device tensors (asynchronous on `stream`)."""
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    _check(load_library().tsim_sample(h, shots, seed, shot_offset, _ptr(meas), _ptr(det), _ptr(obs),
                                      _ptr(accept), s))


def tsim_sample_noalloc(h, shots, seed, shot_offset=0, meas=None, det=None, obs=None, accept=None, stream=None):
    """tsim_sample for callers that cannot allocate device memory (fixed 4 MiB table scratch)."""
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    _check(load_library().tsim_sample_noalloc(h, shots, seed, shot_offset, _ptr(meas), _ptr(det), _ptr(obs),
                                              _ptr(accept), s))


def tsim_debug_sample(h, shots, seed, shot_offset, dump_shots, meas=None, det=None, obs=None, accept=None,
                      stream=None):
    """tsim_sample plus an exact copy of every table evaluation of the shots
    dump_shots (indices within the launch).  Returns an int64 array
    [len(dump_shots)][num_chains + num_random][6 + x_words]: table, c0..c3,
    sqrt2 exponent, X words."""
    import numpy as np
    info = tsim_program_info(h)
    evals = info["num_chains"] + info["num_random"]
    n = len(dump_shots)
    out = np.zeros((n, evals, 6 + info["x_words"]), dtype=np.int64)
    ds = (ctypes.c_uint64 * max(n, 1))(*[int(v) for v in dump_shots])
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    _check(load_library().tsim_debug_sample(h, shots, seed, shot_offset, _ptr(meas), _ptr(det), _ptr(obs),
                                            _ptr(accept), ds, n,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), s))
    return out


def tsim_program_set_noise_sampling(h, mode):
    """0: one Philox word per channel; 1: geometric gaps; -1: the cheaper one."""
    _check(load_library().tsim_program_set_noise_sampling(h, int(mode)))


def tsim_program_noise_info(h):
    out = (ctypes.c_double * 4)()
    _check(load_library().tsim_program_noise_info(h, out))
    return {"mode": int(out[0]), "groups": int(out[1]), "words_per_channel_mode": out[2],
            "words_geometric_mode": out[3]}


def tsim_program_device_bytes(h):
    """Bytes of the program's packed device tables."""
    n = ctypes.c_uint64()
    _check(load_library().tsim_program_device_bytes(h, ctypes.byref(n)))
    return n.value


def tsim_sample_host(h, shots, seed, shot_offset=0, meas=None, det=None, obs=None, accept=None, stream=None):
    """Sample into host numpy arrays (copies inside, synchronous)."""
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    p = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    _check(load_library().tsim_sample_host(h, shots, seed, shot_offset, p(meas), p(det), p(obs), p(accept), s))


def tsim_sample_batch(hs, shots, seeds, shot_offsets=None, meas=None, det=None, obs=None, accept=None,
                      stream=None):
    n = len(hs)
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    arr = lambda xs, T: (T * n)(*xs)  # noqa: E731
    ptrs = lambda ts: None if ts is None else arr([_ptr(t) for t in ts], vp)  # noqa: E731
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    _check(load_library().tsim_sample_batch(arr(hs, vp), n, arr(shots, u64), arr(seeds, u64),
                                            arr(shot_offsets or [0] * n, u64), ptrs(meas), ptrs(det),
                                            ptrs(obs), ptrs(accept), s))


def _batch_arrays(hs, shots, seeds, shot_offsets, meas, det, obs, accept):
    n = len(hs)
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    arr = lambda xs, T: (T * n)(*xs)  # noqa: E731
    ptrs = lambda ts: None if ts is None else arr([_ptr(t) for t in ts], vp)  # noqa: E731
    return (arr(hs, vp), n, arr(shots, u64), arr(seeds, u64), arr(shot_offsets or [0] * n, u64),
            ptrs(meas), ptrs(det), ptrs(obs), ptrs(accept))


def tsim_batch_create(hs, shots, seeds, shot_offsets=None, meas=None, det=None, obs=None, accept=None,
                      autotune=True):
    """Reusable batched launch captured in a CUDA graph; autotune: 0 persistent
    kernel with defaults, 1 (True) autotuned shot blocks, residency and launch
    form, 2 one launch per program."""
    out = ctypes.c_void_p()
    _check(load_library().tsim_batch_create(*_batch_arrays(hs, shots, seeds, shot_offsets, meas, det, obs,
                                                           accept), int(autotune), ctypes.byref(out)))
    return out.value


def tsim_batch_launch(b, stream=None):
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    _check(load_library().tsim_batch_launch(b, s))


def tsim_batch_info(b):
    out = (ctypes.c_int64 * 7)()
    _check(load_library().tsim_batch_info(b, out))
    keys = ["shots_per_item", "blocks_per_sm", "work_items", "graph", "x_words", "tuned_us", "form"]
    return dict(zip(keys, list(out)))


def tsim_batch_free(b):
    load_library().tsim_batch_free(b)


def tsim_sync(stream=None):
    s = stream if isinstance(stream, (int, type(None))) else stream.cuda_stream
    _check(load_library().tsim_sync(s))


def tsim_eval_table(h, t, xwords):
    """Exact table value: ((c0, c1, c2, c3), k) meaning (sum c_i w^i) * sqrt2^k."""
    n = len(xwords)
    x = (ctypes.c_uint64 * n)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in xwords])
    out = (ctypes.c_int64 * 4)()
    k = ctypes.c_int32()
    _check(load_library().tsim_eval_table(h, t, x, out, ctypes.byref(k)))
    return tuple(out), k.value


def tsim_eval_table_float(h, t, xwords):
    """Value of any table at X in complex double (tables of arbitrary rotations included)."""
    n = len(xwords)
    x = (ctypes.c_uint64 * n)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in xwords])
    out = (ctypes.c_double * 2)()
    _check(load_library().tsim_eval_table_float(h, t, x, out))
    return complex(out[0], out[1])


def tsim_raw_to_x(h, e_bits, x_words):
    e = (ctypes.c_uint8 * max(1, len(e_bits)))(*e_bits)
    x = (ctypes.c_uint64 * x_words)()
    _check(load_library().tsim_raw_to_x(h, e, x))
    return list(x)


def tsim_program_save(h, path):
    _check(load_library().tsim_program_save(h, os.fsencode(path)))


def tsim_program_load(path):
    h = ctypes.c_void_p()
    _check(load_library().tsim_program_load(os.fsencode(path), ctypes.byref(h)))
    return h.value


def tsim_program_free(h):
    load_library().tsim_program_free(h)


def tsim_measure_int_peak(op):
    """Measured integer results per second of one instruction class on this GPU."""
    v = ctypes.c_double()
    _check(load_library().tsim_measure_int_peak(op, ctypes.byref(v)))
    return v.value


def tsim_program_device_table_stats(h, t):
    """(classes, class factors, distinct parities) of table t in the packed device tables."""
    out = (ctypes.c_uint64 * 3)()
    _check(load_library().tsim_program_device_table_stats(h, t, out))
    return tuple(out)


TABLE_SCALAR, TABLE_BASIS, TABLE_SLICED = 0, 1, 2


def tsim_program_set_table_layout(h, sliced_min_terms, stage_rows=-1, segment_parities=0):
    """Re-pack the device tables: tables with at least sliced_min_terms terms
    use the bit-sliced warp layout where they qualify (< 0: never); sliced
    batches of at most stage_rows rows are staged in shared memory (0: none,
    < 0: default); sliced tables are split into segments of at most
    segment_parities parity words (<= 0: default)."""
    _check(load_library().tsim_program_set_table_layout(h, int(sliced_min_terms), int(stage_rows),
                                                        int(segment_parities)))


def tsim_program_device_table_layout(h, t):
    """(layout, batches of 32 terms, padded operation rows, operations,
    integer lane-operations per 32 shots, the same without padding) of
    table t."""
    out = (ctypes.c_uint64 * 6)()
    _check(load_library().tsim_program_device_table_layout(h, t, out))
    return tuple(out)


def tsim_program_device_output_stats(h):
    """(output entries, runs, outputs covered by runs) of the packed program."""
    out = (ctypes.c_uint64 * 3)()
    _check(load_library().tsim_program_device_output_stats(h, out))
    return tuple(out)


def tsim_selftest_sliced(h, seed=0, rounds=2):
    """Host emulation of the program's bit-sliced tables against their exact values."""
    _check(load_library().tsim_selftest_sliced(h, seed, rounds))


def tsim_selftest_rules(seed=0, iterations=200):
    _check(load_library().tsim_selftest_rules(seed, iterations))


# ---- learned cut order (compile time)

CUT_FEATURES = 14


def _f32(a, n=None):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} floats, got {a.size}")
    return a


def _i32(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data


def tsim_cut_num_params() -> int:
    return load_library().tsim_cut_num_params()


def tsim_cut_init_params(seed=0):
    import numpy as np
    p = np.zeros(tsim_cut_num_params(), dtype=np.float32)
    _check(load_library().tsim_cut_init_params(seed, _p(p)))
    return p


def tsim_cut_dataset(seed, n_graphs, t_min, t_max, budget, max_candidates, path):
    _check(load_library().tsim_cut_dataset(seed, n_graphs, t_min, t_max, budget, max_candidates,
                                           str(path).encode()))


def tsim_cut_forward(params, x, rowptr, col):
    """Scores of every node (runs on the current CUDA device)."""
    import numpy as np
    params = _f32(params, tsim_cut_num_params())
    x, rowptr, col = _f32(x), _i32(rowptr), _i32(col)
    n = len(rowptr) - 1
    out = np.zeros(n, dtype=np.float32)
    _check(load_library().tsim_cut_forward(_p(params), n, _p(x), _p(rowptr), _p(col), _p(out)))
    return out


def tsim_cut_loss_grad(params, x, rowptr, col, y, graph_off):
    import numpy as np
    params = _f32(params, tsim_cut_num_params())
    x, rowptr, col, y, goff = _f32(x), _i32(rowptr), _i32(col), _f32(y), _i32(graph_off)
    n = len(rowptr) - 1
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros_like(params)
    _check(load_library().tsim_cut_loss_grad(_p(params), n, _p(x), _p(rowptr), _p(col), _p(y), len(goff) - 1,
                                             _p(goff), _p(loss), _p(grad)))
    return float(loss[0]), grad


def tsim_cut_adam_step(params, grad, m, v, step, lr):
    """One Adam step; returns new (params, m, v)."""
    n = tsim_cut_num_params()
    params, grad, m, v = (_f32(a, n).copy() for a in (params, grad, m, v))
    _check(load_library().tsim_cut_adam_step(_p(params), _p(grad), _p(m), _p(v), step, lr))
    return params, m, v


def tsim_cut_train(dataset_path, params, epochs=50, batch_graphs=32, lr=1e-3, seed=0):
    """Train on a dataset file; returns (trained params, loss per epoch)."""
    import numpy as np
    params = _f32(params, tsim_cut_num_params()).copy()
    hist = np.zeros(epochs, dtype=np.float32)
    _check(load_library().tsim_cut_train(str(dataset_path).encode(), epochs, batch_graphs, lr, seed, _p(params),
                                         _p(hist)))
    return params, hist


def tsim_cut_model_set(params):
    """Register the network for DECOMP_LEARNED (None removes it)."""
    if params is None:
        _check(load_library().tsim_cut_model_set(None))
        return
    params = _f32(params, tsim_cut_num_params())
    _check(load_library().tsim_cut_model_set(_p(params)))


def tsim_cut_policy_stats():
    out = (ctypes.c_uint64 * 4)()
    _check(load_library().tsim_cut_policy_stats(out))
    return tuple(out)


def tsim_cut_evaluate(seed, n_graphs, t_min, t_max, budget):
    """Held-out cut-order comparison: [graphs][5] = non-Clifford spiders,
    heuristic terms, learned-policy terms, random-first-cut terms (geometric
    mean), best-first-cut terms."""
    import numpy as np
    out = np.zeros((n_graphs, 5), dtype=np.float64)
    _check(load_library().tsim_cut_evaluate(seed, n_graphs, t_min, t_max, budget, out.ctypes.data))
    return out


def read_cut_dataset(path):
    """Parse a dataset file into (x, rowptr, col, y, graph_off) numpy arrays."""
    import numpy as np
    raw = open(path, "rb").read()
    if raw[:8] != b"TSIMCUTD":
        raise ValueError("not a cut-order dataset")
    ng, nf = np.frombuffer(raw, dtype=np.int32, count=2, offset=8)
    if nf != CUT_FEATURES:
        raise ValueError("feature count differs")
    off = 16
    xs, rps, cols, ys, goff = [], [], [], [], [0]
    n_tot = e_tot = 0
    for _ in range(int(ng)):
        n, nnz = (int(v) for v in np.frombuffer(raw, dtype=np.int32, count=2, offset=off))
        off += 8
        if n:
            xs.append(np.frombuffer(raw, dtype=np.float32, count=n * nf, offset=off).reshape(n, nf)); off += 4 * n * nf
            rp = np.frombuffer(raw, dtype=np.int32, count=n + 1, offset=off); off += 4 * (n + 1)
            c = np.frombuffer(raw, dtype=np.int32, count=nnz, offset=off); off += 4 * nnz
            ys.append(np.frombuffer(raw, dtype=np.float32, count=n, offset=off)); off += 4 * n
            rps.append(rp[1:] + e_tot)
            cols.append(c + n_tot)
            n_tot += n
            e_tot += nnz
        goff.append(n_tot)
    x = np.concatenate(xs) if xs else np.zeros((0, nf), np.float32)
    rowptr = np.concatenate([[0]] + rps).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    y = np.concatenate(ys) if ys else np.zeros(0, np.float32)
    return x, rowptr, col, y, np.array(goff, dtype=np.int32)


class Program:
    """Owning wrapper around a compiled program handle."""

    def __init__(self, text=None, *, handle=None, **opts):
        self.h = handle if handle is not None else tsim_compile(text, **opts)
        self.info = tsim_program_info(self.h)

    @classmethod
    def load(cls, path):
        return cls(handle=tsim_program_load(path))

    def save(self, path):
        tsim_program_save(self.h, path)

    def table_stats(self, t):
        return tsim_program_table_stats(self.h, t)

    def device_table_stats(self, t):
        return tsim_program_device_table_stats(self.h, t)

    def set_table_layout(self, sliced_min_terms, stage_rows=-1, segment_parities=0):
        tsim_program_set_table_layout(self.h, sliced_min_terms, stage_rows, segment_parities)
        self.info = tsim_program_info(self.h)

    def set_noise_sampling(self, mode):
        tsim_program_set_noise_sampling(self.h, mode)
        self.info = tsim_program_info(self.h)

    def noise_info(self):
        return tsim_program_noise_info(self.h)

    def device_bytes(self):
        return tsim_program_device_bytes(self.h)

    def device_table_layout(self, t):
        return tsim_program_device_table_layout(self.h, t)

    def device_output_stats(self):
        return tsim_program_device_output_stats(self.h)

    def table_terms(self):
        return [tsim_program_table_terms(self.h, t) for t in range(self.info["num_tables"])]

    def sample_torch(self, shots, seed, shot_offset=0, stream=None, device="cuda"):
        """Allocate torch output tensors on `device` and launch sampling."""
        import torch
        i = self.info
        meas = torch.empty((shots, i["meas_words"]), dtype=torch.int64, device=device) \
            if i["mode"] == MODE_MEASUREMENTS and i["meas_words"] else None
        det = torch.empty((shots, max(i["det_words"], 1)), dtype=torch.int64, device=device)
        obs = torch.empty((shots, max(i["obs_words"], 1)), dtype=torch.int64, device=device)
        acc = torch.empty((shots,), dtype=torch.uint8, device=device)
        tsim_sample(self.h, shots, seed, shot_offset, meas, det if i["det_words"] else None,
                    obs if i["obs_words"] else None, acc, stream)
        return {"meas": meas, "det": det[:, :i["det_words"]], "obs": obs[:, :i["obs_words"]], "accept": acc}

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            try:
                tsim_program_free(h)
            except Exception:
                pass
            self.h = None
