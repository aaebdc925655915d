"""The multi-GPU path of the benchmark (replicas, max-over-ranks timing, job
throughput), exercised with two gloo ranks on the CPU: each rank computes its
own cloud's barcode (with the CPU oracle standing in for its GPU), ranks see
different clouds, and every rank agrees on the slowest time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_2203_02527_gb300 import inputs
    from paper_2203_02527_gb300.replicas import job_throughput, max_over_ranks, replica_seed

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = inputs.uniform(64, 3, seed=replica_seed(inputs.DEFAULT_SEED, rank))
    bars, _, _ = oracle.barcodes(x)
    local_ms = 10.0 * (rank + 1)  # a slower second rank
    slowest = max_over_ranks(local_ms)
    m = 64 * 63 // 2
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([slowest, job_throughput(m, world, slowest), bars["death_sq"].sum()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0, r1 = (np.load(tmp_path / f"r{i}.npy") for i in range(2))
    assert r0[0] == r1[0] == 20.0                    # both ranks agree on the slowest step
    assert r0[1] == r1[1] == 2 * 2016 / 0.020        # all ranks' edges over the slowest time
    assert r0[2] != r1[2]                            # distinct replicas
