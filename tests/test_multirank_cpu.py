"""Multi-rank sharding on CPU (gloo, world_size 2): each rank filters its own
contiguous shard of the workload, as bench.py does under torchrun, and the
concatenated per-rank results equal a single-process run over the whole range.
The path has no data exchange; the only collectives are the timing barrier and
the max-over-ranks reduction, exercised here too."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

N_PER_RANK = 3000
E = 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_1809_07858_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reads, refs = synth.workload("sweep", N_PER_RANK, E=E, first=rank * N_PER_RANK)
    acc, cnt = oracle.shouji_batch(reads, refs, E)
    dist.barrier()
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    assert t.item() == float(world)
    gathered = [torch.zeros(N_PER_RANK, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(cnt.copy()))
    if rank == 0:
        np.save(os.path.join(out_dir, "counts.npy"), torch.cat(gathered).numpy())
    dist.destroy_process_group()


def test_two_rank_shards_concatenate_to_the_full_result(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_1809_07858_gb300 import synth
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    counts = np.load(tmp_path / "counts.npy")
    reads, refs = synth.workload("sweep", world * N_PER_RANK, E=E)
    _, full = oracle.shouji_batch(reads, refs, E)
    assert (counts == full).all()
