"""Host-side sharding of a frame across ranks.

Paths are independent and the grid is read-only, so N ranks render the same
frame with disjoint ranges of sample indices (each rank spp samples per pixel,
rank r starting at sample r * spp) and the per-pixel sums add up; with
counter-based Philox streams the union over ranks is exactly the frame a single
process would render with N * spp samples.  No data-path collective is needed;
a sum-reduce of the accumulation images is the only exchange, when the caller
wants one image.

render_resilient() is the fault-tolerant form: the frame is cut into chunks of
samples saved one file per chunk, ranks publish progress and heartbeats in a
key-value store, and the chunks of a rank that stops are claimed and rendered by
the others; a restarted job keeps the chunks already saved.
"""
from __future__ import annotations

import os
import time

import numpy as np


def sample_range(rank: int, world_size: int, spp: int) -> tuple[int, int]:
    """(sample_offset, spp) of `rank` when every rank renders spp samples per pixel."""
    if world_size < 1 or not 0 <= rank < world_size or spp < 0:
        raise ValueError("bad rank / world size / spp")
    return rank * spp, spp


def reduce_images(images, op_sum):
    """Sum-reduce accumulation images in place with op_sum (e.g. a
    torch.distributed all_reduce); returns the images."""
    for im in images:
        op_sum(im)
    return images


# ---------------------------------------------------------------------------
# Failure detection and recovery for multi-rank progressive rendering.
#
# A frame of spp samples per pixel is cut into chunks of consecutive sample
# indices.  A chunk's sums depend only on its sample range (counter-based random
# numbers), so the frame is the sum of its chunks whoever renders them, and a
# chunk written to disk is a checkpoint: a restarted job skips it.  Ranks share a
# key-value store (a torch.distributed TCPStore or any store with set / check /
# add / compare_set): a rank publishes each chunk it saved ("done/<c>") and bumps
# its heartbeat ("hb/<r>"); when a rank's heartbeat stops for longer than the
# timeout, the others claim its unfinished chunks one by one (an atomic
# compare-and-set on "claim/<c>") and render them.  Nothing waits on a collective,
# so a rank that raises, exits or never joins cannot stall the others.
# ---------------------------------------------------------------------------


def frame_chunks(spp: int, chunk_spp: int) -> list[tuple[int, int]]:
    """The (sample_offset, spp) ranges, in order, that make up a frame of spp samples."""
    if spp < 0 or chunk_spp < 1:
        raise ValueError("bad spp / chunk size")
    return [(o, min(chunk_spp, spp - o)) for o in range(0, spp, chunk_spp)]


class ChunkFiles:
    """One file per finished chunk: its per-pixel sums (the checkpoint) and the key
    of the frame it belongs to (its sample range, the frame's spp and chunk size,
    and a caller tag naming the seed, camera, grid and medium)."""

    def __init__(self, folder: str):
        self.folder = folder
        os.makedirs(folder, exist_ok=True)

    def path(self, c: int) -> str:
        return os.path.join(self.folder, "chunk%06d.npz" % c)

    def has(self, c: int) -> bool:
        return os.path.exists(self.path(c))

    def save(self, c: int, s, s2, key: str = "") -> None:
        tmp = self.path(c) + ".tmp%d" % os.getpid()
        with open(tmp, "wb") as fh:
            np.savez(fh, sum=_host(s), sumsq=_host(s2), key=np.array(key))
        os.replace(tmp, self.path(c))                # a chunk file is whole or absent

    def key(self, c: int) -> str:
        with np.load(self.path(c)) as z:
            return str(z["key"]) if "key" in z.files else ""

    def load(self, c: int):
        with np.load(self.path(c)) as z:
            return z["sum"], z["sumsq"]


def chunk_key(sample_offset: int, spp: int, chunk_spp: int, frame_spp: int, tag: str) -> str:
    """The frame key saved with a chunk: a chunk file is only reused by a frame
    whose key for that chunk is the same."""
    return "offset=%d spp=%d chunk_spp=%d frame_spp=%d tag=%s" % (sample_offset, spp, chunk_spp, frame_spp, tag)


def _host(t):
    if hasattr(t, "detach"):
        t = t.detach().cpu().numpy()
    return np.asarray(t)


class LocalStore:
    """The store operations render_resilient uses, in one process (world size 1)."""

    def __init__(self):
        self.kv = {}

    def set(self, key, value):
        self.kv[key] = value.encode() if isinstance(value, str) else bytes(value)

    def get(self, key):
        return self.kv[key]

    def check(self, keys):
        return all(k in self.kv for k in keys)

    def add(self, key, n):
        v = int(self.kv.get(key, b"0")) + int(n)
        self.kv[key] = str(v).encode()
        return v

    def compare_set(self, key, expected, desired):
        # as torch.distributed.TCPStore: set when the key holds `expected` (or is
        # absent and `expected` is empty); return the value now held, or `expected`
        # for an absent key that stays absent
        cur = self.kv.get(key)
        if (cur is None and expected == "") or (cur is not None and cur.decode() == expected):
            self.set(key, desired)
        return self.kv.get(key, expected.encode())


def render_resilient(rank: int, world_size: int, store, render, spp: int, chunk_spp: int, folder: str,
                     timeout_s: float = 30.0, poll_s: float = 0.05, give_up_s: float = 600.0, fail_after=None,
                     frame_tag: str = ""):
    """Render this rank's chunks of a frame and finish the chunks of ranks that stop.

    render(sample_offset, spp) -> (sum, sumsq) renders one chunk (per-pixel sums,
    numpy or torch).  With world_size 1 the store may be None: the chunk files
    alone then give checkpoint and resume.  Chunk c belongs to rank c % world_size until another rank
    claims it.  Returns the frame's (sum, sumsq) as float64 arrays (the chunks
    added in order) once every chunk is saved.  timeout_s must exceed one chunk's
    render time: a rank's heartbeat moves once per chunk and once per poll.
    fail_after=k makes this rank raise after saving k chunks (fault injection on
    the host, for tests).  Raises TimeoutError when no chunk completes for
    give_up_s.

    Every chunk file carries the frame's key for it (chunk_key: its sample range,
    spp, chunk_spp and frame_tag, which the caller sets to something naming the
    seed, camera, medium and grid).  A saved chunk is reused only when its key is
    this frame's; a folder holding chunks of another frame, or chunks of
    different image shapes, raises ValueError instead of being summed in."""
    chunks = frame_chunks(spp, chunk_spp)
    if not chunks or world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad spp / rank / world size")
    if store is None:
        if world_size != 1:
            raise ValueError("several ranks need a shared store")
        store = LocalStore()                         # one process: checkpoint and resume only
    files = ChunkFiles(folder)
    me = str(rank)
    saved = 0

    def beat():
        store.add("hb/%d" % rank, 1)

    def own_key(c):
        return chunk_key(chunks[c][0], chunks[c][1], chunk_spp, spp, frame_tag)

    def check_key(c):
        if files.key(c) != own_key(c):
            raise ValueError("chunk file %s belongs to another frame (%r, this frame wants %r)"
                             % (files.path(c), files.key(c), own_key(c)))

    def finish(c):
        nonlocal saved
        if files.has(c):                             # resuming: a saved chunk of this frame is kept
            check_key(c)
        else:
            if fail_after is not None and saved >= fail_after:
                raise RuntimeError("rank %d: injected failure" % rank)
            s, s2 = render(*chunks[c])
            files.save(c, s, s2, own_key(c))
            saved += 1
        store.set("done/%d" % c, me)
        beat()

    beat()
    for c in range(rank, len(chunks), world_size):
        finish(c)

    seen = {}                                        # rank -> (heartbeat, when it last moved)
    fewest, last_progress = len(chunks) + 1, time.monotonic()
    while True:
        missing = [c for c in range(len(chunks)) if not store.check(["done/%d" % c])]
        if not missing:
            break
        now = time.monotonic()
        if len(missing) < fewest:
            fewest, last_progress = len(missing), now
        elif now - last_progress > give_up_s:
            raise TimeoutError("rank %d: chunks %s did not finish" % (rank, missing[:8]))
        for c in missing:
            key = "claim/%d" % c
            holder = store.get(key).decode() if store.check([key]) else ""
            resp = int(holder) if holder else c % world_size    # the rank responsible for c
            hb = int(store.add("hb/%d" % resp, 0))
            h0, t0 = seen.get(resp, (None, now))
            if hb != h0:
                seen[resp] = (hb, now)
                continue
            if now - t0 < timeout_s:
                continue
            # its heartbeat has stopped: take the chunk over, unless another rank just did
            if store.compare_set(key, holder, me).decode() == me:
                finish(c)
        beat()
        time.sleep(poll_s)

    s = s2 = None
    for c in range(len(chunks)):
        check_key(c)                                 # a chunk another rank saved, too
        a, b = files.load(c)
        if s is not None and (a.shape != s.shape or b.shape != s2.shape):
            raise ValueError("chunk %d has image shape %s, chunk 0 has %s" % (c, a.shape, s.shape))
        s = a.astype(np.float64) if s is None else s + a
        s2 = b.astype(np.float64) if s2 is None else s2 + b
    return s, s2
