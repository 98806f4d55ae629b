"""Host logic of the N > 1 benchmark path on CPU: two gloo ranks shard the
seeded event stream without overlap and take the max of their timings (the
only collective; the data path has none)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_0909_5257_gb300 import phasespace as ps
    first = bench.shard_first_event(rank, n)
    mom = ps.generate(ps.PhaseSpaceConfig(3, seed=ps.SEED_BASE + 1), n, first_event=first)
    np.save(os.path.join(out_dir, f"shard{rank}.npy"), mom)
    t = bench.max_over_ranks_value(float(rank + 1) * 0.5, dist, "cpu")
    np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing_reduction(tmp_path):
    world, n = 2, 257
    mp.spawn(_worker, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True)
    from paper_0909_5257_gb300 import phasespace as ps
    whole = ps.generate(ps.PhaseSpaceConfig(3, seed=ps.SEED_BASE + 1), world * n)
    shards = [np.load(tmp_path / f"shard{r}.npy") for r in range(world)]
    assert np.array_equal(np.concatenate(shards), whole)  # disjoint, covering, in order
    for r in range(world):
        assert np.load(tmp_path / f"max{r}.npy")[0] == 0.5 * world


def test_serving_request_stream_shards_without_overlap():
    """The serving workload's request stream (bench.serve_requests): each rank
    takes its own consecutive slice of one seeded stream, so two ranks see
    disjoint requests whose momenta ranges do not overlap, and rank 0's slice
    is the same whatever the world size."""
    import bench
    n = 17
    r0, r1 = bench.serve_requests(0, n), bench.serve_requests(1, n)
    both = bench.serve_requests(0, 2 * n)
    assert r0 + r1 == both
    seen = {}
    for kind, size, first in both:
        assert bench.SERVE_SIZES[0] <= size <= bench.SERVE_SIZES[1]
        for a, b in seen.get(kind, []):
            assert first >= b or first + size <= a
        seen.setdefault(kind, []).append((first, first + size))
    kinds = [k for k, _, _ in bench.serve_requests(0, 4000)]
    shares = np.bincount(kinds, minlength=3) / len(kinds)
    assert np.allclose(shares, [w for *_, w in bench.SERVE_MIX], atol=0.03)
