"""Multi-rank rendering on CPU (gloo, world size 2): ranks render disjoint sample
ranges of the same frame with the CPU oracle, the images are summed with an
all-reduce, and the result equals one process rendering all samples."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2506_11510_gb300 import sharding


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, spp, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2506_11510_gb300 import workloads as W
    from tests.conftest import scene_volume
    s = W.scene("tiny")
    g = O.Grid.for_scene(s, scene_volume("tiny"))
    off, n = sharding.sample_range(rank, world, spp)
    img, img2, _ = g.render(s.camera, s.medium, n, s.render_seed, sample_offset=off, nthreads=2)
    t = [torch.from_numpy(img), torch.from_numpy(img2)]
    sharding.reduce_images(t, lambda x: dist.all_reduce(x, op=dist.ReduceOp.SUM))
    if rank == 0:
        np.save(out_path, np.stack([t[0].numpy(), t[1].numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_equal_one_process(tmp_path):
    import oracle as O
    from paper_2506_11510_gb300 import workloads as W
    from tests.conftest import scene_volume
    O.build()
    spp = 2
    out = str(tmp_path / "img.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), spp, out), nprocs=2, start_method="spawn")
    got = np.load(out)
    s = W.scene("tiny")
    g = O.Grid.for_scene(s, scene_volume("tiny"))
    ref, ref2, _ = g.render(s.camera, s.medium, 2 * spp, s.render_seed, sample_offset=0, nthreads=2)
    # per-pixel sums of the same paths; only the summation order differs
    assert np.allclose(got[0], ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(got[1], ref2, rtol=1e-12, atol=1e-14)


def test_sample_ranges_are_disjoint_and_cover():
    spp, world = 5, 4
    seen = []
    for r in range(world):
        off, n = sharding.sample_range(r, world, spp)
        seen += list(range(off, off + n))
    assert sorted(seen) == list(range(world * spp))
    with pytest.raises(ValueError):
        sharding.sample_range(4, 4, 1)
