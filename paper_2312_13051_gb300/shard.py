"""Data-parallel split of Wilson-loop work over ranks (one process per GPU).

The method's units are independent of one another: every transverse row of a plane is
a loop of its own (Sec. II B, Eq. 3: one Wilson loop per transverse momentum), and
disorder realisations or supercells of different sizes are separate problems.  A job
therefore shards without any data-path collective: rank r takes a contiguous block of
units, computes it on its own GPU, and rank 0 gathers the blocks in unit order (the
only communication; NCCL between GPUs, gloo on the host).  The nested loop needs all
transverse rows of a plane at each base point, so it shards by planes or problems,
not by rows.

``compute`` callables keep this module free of device code: the GPU form is
``gpu_wilson_rows(precision)``, which calls the library through the binding.
"""
from __future__ import annotations

import numpy as np


def partition(n_units: int, world: int) -> list:
    """Balanced contiguous blocks [(start, stop)] of n_units over world ranks; the first
    n_units % world ranks take one unit more.  Ranks beyond n_units get empty blocks."""
    if n_units < 0 or world < 1:
        raise ValueError("need n_units >= 0 and world >= 1")
    q, r = divmod(n_units, world)
    out, s = [], 0
    for k in range(world):
        e = s + q + (1 if k < r else 0)
        out.append((s, e))
        s = e
    return out


def row_block(plane, i0: int, i1: int):
    """Transverse rows i0 .. i1-1 of a plane as a plane of their own:
    k(j, i) = origin + (i0 / N_t) trans_dir + (j / N) loop_dir + (i / (i1 - i0)) (i1 - i0) / N_t
    trans_dir, the same points as rows i0 .. i1-1 of the whole plane (up to rounding in
    the last bit of the coordinates)."""
    if not 0 <= i0 < i1 <= plane.N_t:
        raise ValueError(f"rows [{i0}, {i1}) outside [0, {plane.N_t})")
    o = np.asarray(plane.origin, np.float64) + (i0 / plane.N_t) * np.asarray(plane.trans_dir, np.float64)
    td = np.asarray(plane.trans_dir, np.float64) * ((i1 - i0) / plane.N_t)
    return type(plane)(plane.N, i1 - i0, origin=tuple(float(x) for x in o),
                       loop_dir=tuple(plane.loop_dir), trans_dir=tuple(float(x) for x in td))


def _dist():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist
    return None


def gather_to_rank0(local, rank: int, world: int):
    """Objects of every rank, in rank order, on rank 0 (None elsewhere)."""
    dist = _dist()
    if dist is None or world == 1:
        return [local]
    out = [None] * world if rank == 0 else None
    dist.gather_object(local, out, dst=0)
    return out


def rank_world():
    dist = _dist()
    if dist is None:
        return 0, 1
    return dist.get_rank(), dist.get_world_size()


def wilson_loop_rows(model, plane, p: int, compute, rank=None, world=None):
    """Hybrid Wannier centres of a plane with its transverse rows split over the ranks.
    compute(model, sub_plane, p) -> (phases[rows, p], min_gap[rows]) as numpy arrays.
    Returns (phases[N_t, p], min_gap[N_t]) on rank 0, None on the other ranks."""
    if rank is None or world is None:
        rank, world = rank_world()
    i0, i1 = partition(plane.N_t, world)[rank]
    if i1 > i0:
        ph, gap = compute(model, row_block(plane, i0, i1), p)
        local = (i0, np.asarray(ph), np.asarray(gap))
    else:
        local = (i0, np.empty((0, p)), np.empty((0,)))
    parts = gather_to_rank0(local, rank, world)
    if rank != 0:
        return None
    parts = sorted(parts, key=lambda t: t[0])
    return np.concatenate([t[1] for t in parts]), np.concatenate([t[2] for t in parts])


def map_problems(items, compute, rank=None, world=None):
    """Independent problems (e.g. disorder realisations) split over the ranks in
    contiguous blocks; compute(item) on each rank's block; the results on rank 0 in
    item order (None on the other ranks)."""
    if rank is None or world is None:
        rank, world = rank_world()
    items = list(items)
    s, e = partition(len(items), world)[rank]
    local = (s, [compute(it) for it in items[s:e]])
    parts = gather_to_rank0(local, rank, world)
    if rank != 0:
        return None
    out = []
    for _, res in sorted(parts, key=lambda t: t[0]):
        out.extend(res)
    return out


def gpu_wilson_rows(precision: str = "mixed", ctx=None):
    """compute(model, plane, p) for wilson_loop_rows on this rank's GPU (the library's
    Wilson loop through the binding; results copied to the host for the gather)."""
    from . import _lib

    def compute(model, plane, p):
        ph, gap = _lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
        return ph.cpu().numpy(), gap.cpu().numpy()
    return compute
