"""Host-side logic of the sharded pair histogram: the unit split, and two gloo ranks on the
CPU whose partial histograms (the oracle's, over each rank's row range) all-reduce to the
one-process histogram. The GPU kernels are not involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_08756_gb300 import shard, synth


@pytest.mark.parametrize("n", [0, 1, 2, 7, 64, 1001])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_range_partitions(n, world):
    ranges = [shard.shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [t1 - t0 for t0, t1 in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1 and sum(sizes) == n


def test_shard_range_rejects_bad_split():
    for args in [(5, 2, 2), (5, -1, 2), (5, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            shard.shard_range(*args)


def test_replica_seeds_distinct():
    assert len({shard.replica_seed(7, r) for r in range(64)}) == 64


class _RowUnits:
    """A stand-in handle whose units are the oracle's histogram rows i (pairs i < j)."""

    def __init__(self, system):
        import oracle
        self.ref = oracle.Box(system)
        self.n = system.n_atoms

    def epsr_partial_gr_tiles(self):
        return self.n

    def epsr_partial_gr_range(self, t0, t1, hist, stream=None):
        hist += torch.from_numpy(self.ref.histogram(t0, t1).reshape(-1).astype(np.int64))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = synth.water_box(90, seed=5, L_A=14.0)
        box = _RowUnits(s)
        H = torch.zeros(3 * s.n_bins, dtype=torch.int64)
        t0, t1 = shard.partial_gr_sharded(box, H)
        torch.save({"H": H, "range": (t0, t1)}, os.path.join(out, f"r{rank}.pt"))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_histogram_equals_full(tmp_path, world):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    import oracle
    s = synth.water_box(90, seed=5, L_A=14.0)
    full = oracle.Box(s).histogram().reshape(-1).astype(np.int64)
    res = [torch.load(os.path.join(tmp_path, f"r{r}.pt")) for r in range(world)]
    for r in res:
        assert np.array_equal(r["H"].numpy(), full)
    assert [r["range"] for r in res] == [shard.shard_range(s.n_atoms, r, world) for r in range(world)]
