"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

Frames are independent, so ranks decode disjoint frame ranges with no exchange
of data; only the timing is reduced (maximum over ranks).  The reference
decoder stands in for the GPU here: each rank decodes its own shard, and the
union must equal a single-process decode of the same frame ids.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

FRAMES_PER_RANK = 24


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_1402_2773_gb300 import workload as wl
    r, w, _ = bench.env_rank()
    assert (r, w) == (rank, world)
    off, F = bench.shard(rank, world, FRAMES_PER_RANK)
    code = wl.peg_code(504, 252, 3, seed=1)
    y, _, sig = wl.frames(code, F, 3.0, seed=bench.DATA_SEED, frame_offset=off)
    op = oracle.make_params(**dict(bench.PARAMS, t_max=60))
    b, it, ps = oracle.load().decode_f32(code, y, sig, op, seed=bench.DECODER_SEED, frame_offset=off)
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), off=off, bits=b, iters=it, pas=ps)
    elapsed = 1.0 + rank                         # a stand-in timing per rank
    worst = bench.max_over_ranks(elapsed, "cpu")
    assert worst == float(world)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_without_exchange(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    import bench
    import oracle
    from paper_1402_2773_gb300 import workload as wl
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    offs = [int(p["off"]) for p in parts]
    assert offs == [0, FRAMES_PER_RANK]                         # disjoint, contiguous ranges
    code = wl.peg_code(504, 252, 3, seed=1)
    y, _, sig = wl.frames(code, 2 * FRAMES_PER_RANK, 3.0, seed=bench.DATA_SEED)
    op = oracle.make_params(**dict(bench.PARAMS, t_max=60))
    b, it, ps = oracle.load().decode_f32(code, y, sig, op, seed=bench.DECODER_SEED, frame_offset=0)
    got_b = np.concatenate([p["bits"] for p in parts])
    got_i = np.concatenate([p["iters"] for p in parts])
    assert (got_b == b).all() and (got_i == it).all()
