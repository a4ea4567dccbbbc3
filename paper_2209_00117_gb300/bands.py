"""One map split into row bands across ranks (one GPU each).

A jump pass with step k (Table I, Section V-B) reads, for every pixel of row
y, rows y - k, y and y + k.  With the map's rows split into contiguous bands,
one per rank, a rank can compute its band's next map once it holds the rows
its band reads: [y0 - k, y1 - k) and [y0 + k, y1 + k) clipped to the map,
minus its own rows.  For small k these are k-row halos from the two
neighbouring bands; for JFA's first steps (k up to N / 2, Eq. 2) k exceeds
the band height and the rows come from bands further away, so the exchange is
planned per step.  dJFA's first step is bounded by Eq. 4, and with it the
halo depth of a dJFA frame.

Each rank keeps a map of the full size (only its band and the halo rows it
received are current; the rest is never read), so that the kernels address
rows by their global index; the computation and the map traffic split across
ranks, the memory does not.  The exchange is point-to-point (send/recv of
whole rows, which are contiguous in the row-major map) through
torch.distributed: NCCL between GPUs, gloo on the host.  The rows a rank
sends are read after its pass has completed on its stream and the rows it
receives land before its next pass, so nothing ever waits on a kernel of
another rank.

This module holds the plan (which rows go where) and the frame drivers; every
pass runs in the library's kernels (``VoronoiSim.pass_rows``).
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple

Rows = Tuple[int, int]  # [a, b)


def band_rows(h: int, world: int, rank: int) -> Rows:
    """Rows [y0, y1) of rank's band: the h rows split as evenly as possible,
    in rank order (a band may be empty when h < world)."""
    return rank * h // world, (rank + 1) * h // world


def _clip(a: int, b: int, h: int) -> Rows:
    return max(a, 0), min(b, h)


def _minus(r: Rows, cut: Rows) -> List[Rows]:
    """r with the rows of `cut` taken out (0, 1 or 2 ranges)."""
    a, b = r
    out = []
    if a < min(b, cut[0]):
        out.append((a, min(b, cut[0])))
    if max(a, cut[1]) < b:
        out.append((max(a, cut[1]), b))
    return out


def halo_rows(h: int, world: int, rank: int, k: int) -> List[Rows]:
    """The rows outside rank's band that its pass with step k reads, as
    disjoint increasing ranges."""
    y0, y1 = band_rows(h, world, rank)
    if y0 >= y1:
        return []
    need = []
    for r in (_clip(y0 - k, y1 - k, h), _clip(y0 + k, y1 + k, h)):
        if r[0] < r[1]:
            need.extend(_minus(r, (y0, y1)))
    need.sort()
    merged: List[Rows] = []
    for a, b in need:
        if merged and a <= merged[-1][1]:
            merged[-1] = (merged[-1][0], max(merged[-1][1], b))
        else:
            merged.append((a, b))
    return merged


def halo_plan(h: int, world: int, k: int) -> Dict[Tuple[int, int], List[Rows]]:
    """{(src, dst): row ranges src sends to dst} for a pass with step k: the
    halo rows of dst that lie in src's band."""
    plan: Dict[Tuple[int, int], List[Rows]] = {}
    for dst in range(world):
        for a, b in halo_rows(h, world, dst, k):
            for src in range(world):
                s0, s1 = band_rows(h, world, src)
                lo, hi = max(a, s0), min(b, s1)
                if lo < hi and src != dst:
                    plan.setdefault((src, dst), []).append((lo, hi))
    return plan


def exchange(dist, rows_view, plan, rank: int) -> int:
    """Sends this rank's rows of `plan` and receives the rows it needs, in
    place, with one batch of point-to-point operations (torch.distributed,
    any backend).  rows_view: this rank's map as an (h, pitch) tensor.
    Returns the number of rows received."""
    ops = []
    got = 0
    for (src, dst), ranges in sorted(plan.items()):
        for a, b in ranges:
            if src == rank:
                ops.append(dist.P2POp(dist.isend, rows_view[a:b].contiguous(), dst))
            elif dst == rank:
                ops.append(dist.P2POp(dist.irecv, rows_view[a:b], src))
                got += b - a
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return got


def run_passes(schedule: Sequence[Tuple[int, int]], h: int, world: int, rank: int,
               exchange_rows: Callable[[Dict[Tuple[int, int], List[Rows]]], None],
               band_pass: Callable[[int, int, int, int], None]) -> None:
    """The passes of one frame on rank's band: before each pass the halo rows
    its step needs arrive (exchange_rows(plan)), then the band's rows of the
    next map are computed (band_pass(k, nb, y0, y1))."""
    y0, y1 = band_rows(h, world, rank)
    for k, nb in schedule:
        exchange_rows(halo_plan(h, world, k))
        if y0 < y1:
            band_pass(k, nb, y0, y1)


class DeviceMap:
    """The current label map of a context as an (h, pitch) int32 CUDA tensor
    (borrowed: valid until the context's next pass flips its buffers)."""

    def __init__(self, sim):
        self.sim = sim

    def tensor(self):
        import torch

        ptr = self.sim.labels_device_ptr()
        h, pitch = self.sim.h, self.sim.pitch

        class _Iface:
            __cuda_array_interface__ = {"shape": (h, pitch), "typestr": "<i4", "data": (ptr, False),
                                        "version": 3, "strides": None}

        return torch.as_tensor(_Iface(), device=f"cuda:{torch.cuda.current_device()}")
