"""The multi-GPU path on the host: two gloo ranks (CPU) shard the shots of a
program the way bench.py does under torchrun, sample their shards with the
oracle, and gather them; the concatenation must equal one run over all shots,
and the timing reduction must take the slowest rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, path, shots, seed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle.evaluator import OracleProgram
        (off,) = bench.shard_offsets(rank, [shots])
        rec = OracleProgram(path).sample(seed, off, shots)
        det = torch.from_numpy(rec["det"].view(np.int64).copy())
        parts = [torch.empty_like(det) for _ in range(world)]
        dist.all_gather(parts, det)
        slowest = bench.max_over_ranks(float(rank + 1), dist)
        if rank == 0:
            np.save(out, torch.cat(parts).numpy())
            with open(out + ".t", "w") as f:
                f.write(repr(slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_concatenate_to_one_run(tmp_path, oracle_lib):
    import paper_2604_01059_gb300 as T
    from paper_2604_01059_gb300 import workloads as Wk
    from oracle.evaluator import OracleProgram
    prog = T.Program(Wk.config1_circuit(p=5e-3))
    path = str(tmp_path / "c1.prog")
    prog.save(path)
    shots, seed, world = 300, 77, 2
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_worker, args=(world, _free_port(), path, shots, seed, out), nprocs=world,
                       start_method="spawn")
    got = np.load(out)
    want = OracleProgram(path).sample(seed, 0, world * shots)["det"].view(np.int64)
    np.testing.assert_array_equal(got, want)
    assert float(open(out + ".t").read()) == world
