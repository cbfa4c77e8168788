"""Panel sharding of one permeable surface over ranks (Sec. III A, III B).

The paper partitions a surface's Faces (blocks of subfaces) over its MPI
ranks: the Faces are sorted by size and each goes to the rank with the
fewest subfaces so far.  Every rank needs the same observer time grid, so
the per-observer R_max and R_min of its own subfaces are reduced over the
ranks (maximum and minimum, the MPI_ALLREDUCE of Sec. III B "compute t");
after the forward pass the ranks' partial far-field signals are summed.

Here a rank is one process with one GPU and one FWH handle made on its
panels; the reductions are torch.distributed collectives (NCCL between GPUs,
gloo on CPU).  This module only partitions indices and calls collectives: the
arithmetic of the path runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def face_blocks(n_panels: int, face_size: int) -> list[tuple[int, int]]:
    """Contiguous panel ranges [lo, hi) of at most face_size panels: the Faces
    of a surface whose panels are stored face by face."""
    return [(lo, min(n_panels, lo + face_size)) for lo in range(0, n_panels, face_size)]


def partition_faces(face_sizes, n_ranks: int) -> list[list[int]]:
    """The paper's Face partition (Sec. III A): Faces in descending size, each
    to the least-loaded rank (ties to the lower rank).  Returns the face
    indices of every rank."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    sizes = np.asarray(face_sizes, dtype=np.int64)
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * n_ranks
    out: list[list[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(f) for f in out]


def rank_panels(faces: list[tuple[int, int]], mine: list[int]) -> np.ndarray:
    """Panel indices of the faces `mine` (in face order)."""
    idx = [np.arange(faces[f][0], faces[f][1]) for f in mine]
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def _comm_device(group=None):
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def shard_setup(engine, group=None) -> None:
    """Give every rank the common observer window: all-reduce the per-observer
    R_max (maximum) and R_min (minimum) of the ranks' panels and set them on
    this rank's surface.  Once per geometry and observer set."""
    import torch
    import torch.distributed as dist
    dev = _comm_device(group)
    mx, mn = engine.observer_extremes()
    tmx = torch.as_tensor(np.asarray(mx, dtype=np.float64), device=dev).clone()
    tmn = torch.as_tensor(np.asarray(mn, dtype=np.float64), device=dev).clone()
    dist.all_reduce(tmx, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(tmn, op=dist.ReduceOp.MIN, group=group)
    engine.set_observer_extremes(tmx.cpu().numpy(), tmn.cpu().numpy())


def sharded_forward(engine, fields, group=None, out=None):
    """This rank's forward pass on the common window, summed over the ranks:
    every rank returns the unsharded p_out [O][nt] (float64)."""
    import torch.distributed as dist
    dev = _comm_device(group)
    p = engine.forward(fields) if out is None else engine.forward(fields, out)
    pc = p if p.device == dev else p.to(dev)
    dist.all_reduce(pc, op=dist.ReduceOp.SUM, group=group)
    return pc
