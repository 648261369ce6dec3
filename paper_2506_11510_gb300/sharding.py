"""Host-side sharding of a frame across ranks.

Paths are independent and the grid is read-only, so N ranks render the same
frame with disjoint ranges of sample indices (each rank spp samples per pixel,
rank r starting at sample r * spp) and the per-pixel sums add up; with
counter-based Philox streams the union over ranks is exactly the frame a single
process would render with N * spp samples.  No data-path collective is needed;
a sum-reduce of the accumulation images is the only exchange, when the caller
wants one image.
"""
from __future__ import annotations


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
