"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its own
replica, agree on the slowest rank's time and report the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    out[rank] = (ms, bench.replica_throughput(ms, world, 1000, 20))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 15.0
    assert value == pytest.approx(2 * 1000 * 20 / 15e-3)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(2.0, 1, 100, 10) == pytest.approx(100 * 10 / 2e-3)


def test_exact_draw_blocks_are_disjoint():
    """Each rank's 2^24 exact-solver interfaces come from its own block of
    draws, apart from every other rank's and from the training draws."""
    import bench
    n = 1 << 24
    blocks = [(bench.exact_offset(r, n), bench.exact_offset(r, n) + n) for r in range(16)]
    blocks.append((bench.TRAIN_OFFSET, bench.TRAIN_OFFSET + bench.TRAIN_ROWS))
    blocks.sort()
    assert all(a1 <= b0 for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]))
    assert bench.exact_offset(0, n) == 0


def test_block_shape():
    """Ranks of a decomposed-grid run form the most nearly square px x py
    (px >= py) unless a shape is given."""
    import bench
    assert [bench.block_shape(w) for w in (1, 2, 3, 4, 6, 8, 9, 12)] == \
        [(1, 1), (2, 1), (3, 1), (2, 2), (3, 2), (4, 2), (3, 3), (4, 3)]
    assert bench.block_shape(4, "4x1") == (4, 1)
    assert bench.block_shape(1, "2X1") == (2, 1)
