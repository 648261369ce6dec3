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


# ---- failure detection and recovery (host only: ranks are CPU processes) ----

def _resilient_main(rank, world, port, folder, spp, fail_after, out_path):
    import datetime
    import oracle as O
    from paper_2506_11510_gb300 import workloads as W
    from tests.conftest import scene_volume
    store = dist.TCPStore("127.0.0.1", port, None, False, datetime.timedelta(seconds=30))
    s = W.scene("tiny")
    g = O.Grid.for_scene(s, scene_volume("tiny"))
    rendered = []

    def render(off, n):
        rendered.append(off)
        img, img2, _ = g.render(s.camera, s.medium, n, s.render_seed, sample_offset=off, nthreads=1)
        return img, img2

    try:
        frame = sharding.render_resilient(rank, world, store, render, spp, 1, folder, timeout_s=1.0, poll_s=0.02,
                                          give_up_s=60.0, fail_after=fail_after)
    finally:
        np.save(out_path + ".rendered%d.npy" % rank, np.array(rendered, dtype=np.int64))
    np.save(out_path + ".frame%d.npy" % rank, np.stack(frame))


def _run_ranks(world, folder, spp, fail_after, out_path):
    import datetime
    import multiprocessing
    store = dist.TCPStore("127.0.0.1", 0, None, True, datetime.timedelta(seconds=30), wait_for_workers=False)
    ctx = multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_resilient_main, args=(r, world, store.port, folder, spp, fail_after.get(r), out_path))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    return codes


def _reference(spp):
    import oracle as O
    from paper_2506_11510_gb300 import workloads as W
    from tests.conftest import scene_volume
    s = W.scene("tiny")
    g = O.Grid.for_scene(s, scene_volume("tiny"))
    ref, ref2, _ = g.render(s.camera, s.medium, spp, s.render_seed, sample_offset=0, nthreads=2)
    return ref, ref2


def test_chunks_cover_the_frame(tmp_path):
    assert sharding.frame_chunks(10, 4) == [(0, 4), (4, 4), (8, 2)]
    assert sharding.frame_chunks(0, 3) == []
    with pytest.raises(ValueError):
        sharding.frame_chunks(4, 0)
    with pytest.raises(ValueError):
        sharding.render_resilient(0, 1, None, None, 0, 1, str(tmp_path))      # an empty frame
    with pytest.raises(ValueError):
        sharding.render_resilient(2, 2, None, None, 4, 1, str(tmp_path))      # rank out of range


def test_a_rank_that_dies_mid_frame_is_taken_over(tmp_path):
    """Three ranks; rank 2 raises after saving one of its three chunks.  The others
    see its heartbeat stop, claim its two unfinished chunks, and every surviving
    rank returns exactly the frame one process renders."""
    import oracle as O
    O.build()
    spp, out = 9, str(tmp_path / "out")
    codes = _run_ranks(3, str(tmp_path / "chunks"), spp, {2: 1}, out)
    assert codes[0] == 0 and codes[1] == 0 and codes[2] != 0, codes
    ref, ref2 = _reference(spp)
    for r in (0, 1):
        got = np.load(out + ".frame%d.npy" % r)
        assert np.allclose(got[0], ref, rtol=1e-12, atol=1e-14)
        assert np.allclose(got[1], ref2, rtol=1e-12, atol=1e-14)
    done = [np.load(out + ".rendered%d.npy" % r) for r in range(3)]
    assert sorted(np.concatenate(done).tolist()) == list(range(spp))   # every chunk rendered once
    assert done[2].tolist() == [2]


def test_a_restarted_job_resumes_from_its_saved_chunks(tmp_path):
    """Every rank fails after one chunk; the restarted job renders only the chunks
    that were not saved, and the frame equals one process rendering all of it."""
    import oracle as O
    O.build()
    spp, folder, out = 8, str(tmp_path / "chunks"), str(tmp_path / "out")
    codes = _run_ranks(2, folder, spp, {0: 1, 1: 1}, out + "a")
    assert all(c != 0 for c in codes), codes
    codes = _run_ranks(2, folder, spp, {}, out + "b")
    assert codes == [0, 0], codes
    again = np.concatenate([np.load(out + "b.rendered%d.npy" % r) for r in range(2)])
    assert sorted(again.tolist()) == [2, 3, 4, 5, 6, 7]                  # chunks 0 and 1 were kept
    ref, ref2 = _reference(spp)
    got = np.load(out + "b.frame0.npy")
    assert np.allclose(got[0], ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(got[1], ref2, rtol=1e-12, atol=1e-14)


def test_one_process_resumes_from_its_chunk_files(tmp_path):
    """World size 1 without a store: a run that fails after two chunks leaves them
    on disk; the next run renders only the other chunks and returns the frame."""
    import oracle as O
    from paper_2506_11510_gb300 import workloads as W
    from tests.conftest import scene_volume
    O.build()
    s = W.scene("tiny")
    g = O.Grid.for_scene(s, scene_volume("tiny"))
    done = []

    def render(off, n):
        done.append(off)
        img, img2, _ = g.render(s.camera, s.medium, n, s.render_seed, sample_offset=off, nthreads=2)
        return img, img2

    folder = str(tmp_path / "chunks")
    with pytest.raises(RuntimeError):
        sharding.render_resilient(0, 1, None, render, 5, 1, folder, fail_after=2)
    assert done == [0, 1]
    frame = sharding.render_resilient(0, 1, None, render, 5, 1, folder)
    assert done == [0, 1, 2, 3, 4]
    ref, ref2 = _reference(5)
    assert np.allclose(frame[0], ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(frame[1], ref2, rtol=1e-12, atol=1e-14)
    with pytest.raises(ValueError):
        sharding.render_resilient(0, 2, None, render, 5, 1, folder)           # two ranks need a store


def test_local_store_claims_once():
    st = sharding.LocalStore()
    assert st.compare_set("claim/0", "", "1") == b"1"
    assert st.compare_set("claim/0", "", "2") == b"1"                         # already claimed
    assert st.compare_set("claim/0", "1", "2") == b"2"                        # taken over from rank 1
    assert st.add("hb/0", 1) == 1 and st.add("hb/0", 0) == 1
    assert st.check(["claim/0"]) and not st.check(["claim/1"])
    assert st.compare_set("claim/1", "3", "4") == b"3" and not st.check(["claim/1"])


def test_a_reused_folder_of_another_frame_is_refused(tmp_path):
    """Chunk files carry their frame's key: a folder reused for a frame with another
    seed (tag) or another chunk size raises instead of summing the old chunks in,
    and the same frame still resumes from it."""
    calls = []

    def render(off, n):
        calls.append((off, n))
        v = np.full((3, 4), float(off + n), np.float32)
        return v, v * v

    folder = str(tmp_path / "chunks")
    a = sharding.render_resilient(0, 1, None, render, 4, 2, folder, frame_tag="seed=7")
    assert calls == [(0, 2), (2, 2)]
    with pytest.raises(ValueError, match="another frame"):
        sharding.render_resilient(0, 1, None, render, 4, 2, folder, frame_tag="seed=8")
    with pytest.raises(ValueError, match="another frame"):
        sharding.render_resilient(0, 1, None, render, 4, 1, folder, frame_tag="seed=7")
    calls.clear()
    b = sharding.render_resilient(0, 1, None, render, 4, 2, folder, frame_tag="seed=7")
    assert calls == [] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_chunks_of_different_image_shapes_are_refused(tmp_path):
    """Two chunks of one key but different image shapes (a corrupt or hand-edited
    folder) raise ValueError rather than broadcasting."""
    folder = str(tmp_path / "chunks")
    files = sharding.ChunkFiles(folder)
    files.save(0, np.zeros((2, 2)), np.zeros((2, 2)), sharding.chunk_key(0, 1, 1, 2, "t"))
    files.save(1, np.zeros((3, 2)), np.zeros((3, 2)), sharding.chunk_key(1, 1, 1, 2, "t"))
    with pytest.raises(ValueError, match="shape"):
        sharding.render_resilient(0, 1, None, None, 2, 1, folder, frame_tag="t")
