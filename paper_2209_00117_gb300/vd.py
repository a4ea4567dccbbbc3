"""Python binding of the C ABI: one :class:`VoronoiSim` per simulation.

Argument marshalling only -- every step runs in ``libvd.so``.  Arrays may be
numpy arrays (host) or torch tensors (host or CUDA); they must be contiguous
int32.  PyTorch supplies device memory and streams; it computes nothing here.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N

EUCLID, MANHATTAN = 0, 1
MOORE, VON_NEUMANN = 0, 1

OPT_FUSE_MAX_K = 1
OPT_BAND_ORDER_MIN_K = 2
OPT_USE_GRAPHS = 3
OPT_FUSE_TILE_X = 4
OPT_FUSE_TILE_Y = 5
OPT_PROFILE = 6
OPT_CLAMPED_KEYS = 7
OPT_PDL = 8
OPT_DEDUP_GATHERS = 9
OPT_BYTE_KEYS = 10
OPT_BLOCKED_PASS = 11
OPT_KEY_PACK = 12
OPT_BLOCKED_MIN_BLOCKS = 13
OPT_SPARSE_PASS = 14
OPT_JFA_POSITION_MAP = 15
OPT_PASS_TILE = 16
OPT_SMEM_TILE_MAX_K = 17
OPT_SMEM_TILE_ROWS = 18
OPT_PACKED_MAP = 19

KERNEL_KINDS = ("pass", "fused", "stamp", "move", "fill")

MAX_PASSES = 64


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _buf(a, n_elems: int | None = None, writable: bool = False):
    """(pointer, on_device) of a contiguous int32 numpy array or torch tensor."""
    if a is None:
        return None, 0
    if _is_torch(a):
        import torch

        if a.dtype != torch.int32 or not a.is_contiguous():
            raise TypeError("tensor must be contiguous int32")
        if n_elems is not None and a.numel() != n_elems:
            raise ValueError(f"expected {n_elems} elements, got {a.numel()}")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray) or a.dtype != np.int32 or not a.flags.c_contiguous:
        raise TypeError("array must be a C-contiguous int32 numpy array")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    if n_elems is not None and a.size != n_elems:
        raise ValueError(f"expected {n_elems} elements, got {a.size}")
    return a.ctypes.data, 0


def widen24(packed, h: int, w: int) -> np.ndarray:
    """int32 labels (h x w) from a 24-bit read-back (vd_get_labels24_async):
    three little-endian bytes a label, 0xFFFFFF the empty label -1."""
    b = np.asarray(packed, np.uint8).reshape(h * w, 3).astype(np.int32)
    v = b[:, 0] | (b[:, 1] << 8) | (b[:, 2] << 16)
    return np.where(v == 0xFFFFFF, -1, v).astype(np.int32).reshape(h, w)


def label_bits(n_seeds: int) -> int:
    """The fewest bits a packed read-back (vd_get_labels_packed_async) takes
    for n seeds: labels 0 .. n - 1 and the empty code 2^bits - 1 apart."""
    return max(1, int(n_seeds).bit_length())


def unpack_labels(packed, h: int, w: int, bits: int, rows_per_chunk: int = 1024) -> np.ndarray:
    """int32 labels (h x w) from a packed read-back: label j = y w + x at bits
    [j bits, (j + 1) bits) of the little-endian stream, 2^bits - 1 the empty
    label -1.  Unpacked a band of rows at a time."""
    buf = np.asarray(packed, np.uint8).reshape(-1)
    n = h * w
    if buf.size != (n * bits + 7) // 8:
        raise ValueError(f"expected {(n * bits + 7) // 8} bytes, got {buf.size}")
    pad = np.zeros(buf.size + 8, np.uint8)
    pad[:buf.size] = buf
    empty = (1 << bits) - 1
    out = np.empty(n, np.int32)
    step = max(1, rows_per_chunk) * w
    for j0 in range(0, n, step):
        j = np.arange(j0, min(n, j0 + step), dtype=np.int64) * bits
        byte = j >> 3
        v = np.zeros(j.size, np.uint64)
        for i in range(5):  # a label spans at most 5 bytes (7 + 32 bits)
            v |= pad[byte + i].astype(np.uint64) << np.uint64(8 * i)
        v = (v >> (j & 7).astype(np.uint64)) & np.uint64(empty)
        out[j0:j0 + j.size] = np.where(v == empty, -1, v.astype(np.int64))
    return out.reshape(h, w)


def _schedule(fn, *args):
    ks = np.zeros(MAX_PASSES, np.int32)
    nbs = np.zeros(MAX_PASSES, np.int32)
    n = N.check(fn(*args, ks.ctypes.data, nbs.ctypes.data, MAX_PASSES))
    return [(int(ks[i]), int(nbs[i])) for i in range(min(n, MAX_PASSES))]


def jfa_schedule(w: int, h: int, extra: int = 0):
    """[(k, neighbourhood)] of a JFA frame (Eq. 2)."""
    return _schedule(N.lib().vd_jfa_schedule, w, h, extra)


def djfa_schedule(w: int, h: int, n_seeds: int, d_max: int, vn_waves: int = 2, extra: int = 0):
    """[(k, neighbourhood)] of a dJFA frame (Eq. 3-4, Section V-B)."""
    return _schedule(N.lib().vd_djfa_schedule, w, h, n_seeds, d_max, vn_waves, extra)


def exact_noalloc(seeds_xy, w: int, h: int, labels_out=None, dist_out=None, metric: int = EUCLID,
                  stream=None):
    """The exact diagram from caller-owned CUDA tensors, allocating no device
    memory (the library's fixed scratch array is used instead): for callers
    that must not call cudaMalloc.  ``seeds_xy`` is an (n, 2) int32 CUDA
    tensor; the outputs are (h, w) int32 CUDA tensors (either may be None)."""
    n = seeds_xy.numel() // 2
    ps, ds = _buf(seeds_xy, 2 * n)
    pl, dl = _buf(labels_out, w * h, writable=True)
    pd, dd = _buf(dist_out, w * h, writable=True)
    if not ds or (labels_out is not None and not dl) or (dist_out is not None and not dd):
        raise ValueError("exact_noalloc takes CUDA tensors only")
    if stream is None:
        handle = _current_stream_handle()
    else:
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    N.check(N.lib().vd_exact_noalloc(ps, n, int(w), int(h), int(metric), pl, pd, ctypes.c_void_p(handle)))
    return labels_out, dist_out


def _current_stream_handle():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class VoronoiSim:
    """A w x h label map with n_seeds moving seeds resident on the GPU."""

    def __init__(self, w: int, h: int, n_seeds: int, stream=None):
        self._lib = N.lib()
        handle = self._lib.vd_create(int(w), int(h), int(n_seeds))
        if not handle:
            raise N.VDError(N.VD_EINVAL, N.last_error())
        self._h = ctypes.c_void_p(handle)
        self.w, self.h, self.n_seeds = int(w), int(h), int(n_seeds)
        p = ctypes.c_int32()
        N.check(self._lib.vd_get_shape(self._h, None, None, None, ctypes.byref(p)))
        self.pitch = p.value
        self.set_stream(stream)

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.vd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream=None):
        """Queue work on ``stream`` (a torch.cuda.Stream, a raw handle, or None =
        torch's current stream)."""
        if stream is None:
            handle = _current_stream_handle()
        elif hasattr(stream, "cuda_stream"):
            handle = stream.cuda_stream
        else:
            handle = int(stream)
        self.stream_handle = handle
        N.check(self._lib.vd_set_stream(self._h, ctypes.c_void_p(handle)))

    def synchronize(self):
        N.check(self._lib.vd_synchronize(self._h))

    def set_option(self, option: int, value: int):
        N.check(self._lib.vd_set_option(self._h, option, int(value)))

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        N.check(self._lib.vd_get_option(self._h, option, ctypes.byref(v)))
        return v.value

    def profile(self, reset: bool = False) -> dict:
        """Per kernel kind: {"ms": total GPU ms, "launches": n, "units": work units}
        over the launches bracketed since the last reset (needs OPT_PROFILE=1)."""
        k = len(KERNEL_KINDS)
        ms = np.zeros(k, np.float64)
        nl = np.zeros(k, np.int64)
        un = np.zeros(k, np.int64)
        N.check(self._lib.vd_profile_read(self._h, ms.ctypes.data, nl.ctypes.data, un.ctypes.data))
        out = {name: {"ms": float(ms[i]), "launches": int(nl[i]), "units": int(un[i])}
               for i, name in enumerate(KERNEL_KINDS)}
        if reset:
            N.check(self._lib.vd_profile_reset(self._h))
        return out

    def profile_reset(self):
        N.check(self._lib.vd_profile_reset(self._h))

    @property
    def launches(self) -> int:
        return int(self._lib.vd_launch_count(self._h))

    # -- seeds ----------------------------------------------------------
    def set_seeds(self, xy):
        ptr, dev = _buf(xy, 2 * self.n_seeds)
        N.check(self._lib.vd_set_seeds(self._h, ptr, dev))

    def get_seeds(self, out=None):
        if out is None:
            out = np.empty((self.n_seeds, 2), np.int32)
        ptr, dev = _buf(out, 2 * self.n_seeds, writable=True)
        N.check(self._lib.vd_get_seeds(self._h, ptr, dev))
        return out

    def move(self, dxy=None, max_disp: int = 0, rng_seed: int = 0, stream_id: int = 0, step: int = 0):
        """SimulateParticles: given displacements, or SplitMix64 draws in [-max_disp, max_disp]."""
        ptr, dev = _buf(dxy, 2 * self.n_seeds)
        N.check(self._lib.vd_move_seeds(self._h, ptr, dev, int(max_disp), int(rng_seed) & (2**64 - 1),
                                        int(stream_id) & (2**64 - 1), int(step)))

    def update_seeds(self, remove=None, add=None):
        """Removes the seeds with the given indices and appends new (x, y)
        seeds; survivors are renumbered in order and the map is relabelled
        (see vd_update_seeds).  Both host arrays or both CUDA int32 tensors."""
        rem = remove if remove is not None else np.zeros(0, np.int32)
        new = add if add is not None else np.zeros((0, 2), np.int32)
        if not _is_torch(rem):
            rem = np.ascontiguousarray(rem, dtype=np.int32).reshape(-1)
        if not _is_torch(new):
            new = np.ascontiguousarray(new, dtype=np.int32).reshape(-1)
        nr = int(rem.numel() if _is_torch(rem) else rem.size)
        na = int(new.numel() if _is_torch(new) else new.size) // 2
        pr, dr = _buf(rem) if nr else (None, None)
        pa, da = _buf(new) if na else (None, None)
        kinds = {d for d in (dr, da) if d is not None}
        if len(kinds) > 1:
            raise ValueError("removals and new seeds must both be host arrays or both CUDA tensors")
        on_device = kinds.pop() if kinds else 0
        N.check(self._lib.vd_update_seeds(self._h, pr, nr, pa, na, on_device))
        n = ctypes.c_int32()
        N.check(self._lib.vd_get_shape(self._h, None, None, ctypes.byref(n), None))
        self.n_seeds = n.value

    # -- frames ---------------------------------------------------------
    def jfa(self, extra: int = 0, metric: int = EUCLID):
        N.check(self._lib.vd_jfa(self._h, int(extra), int(metric)))

    def djfa_step(self, d_max: int, vn_waves: int = 2, extra: int = 0, metric: int = EUCLID):
        N.check(self._lib.vd_djfa_step(self._h, int(d_max), int(vn_waves), int(extra), int(metric)))

    def step(self, dxy=None, max_disp: int = 0, rng_seed: int = 0, stream_id: int = 0, step: int = 0,
             d_max: int = 1, vn_waves: int = 2, extra: int = 0, metric: int = EUCLID):
        """move() then djfa_step() as one call (one graph with OPT_USE_GRAPHS)."""
        ptr, dev = _buf(dxy, 2 * self.n_seeds)
        N.check(self._lib.vd_step(self._h, ptr, dev, int(max_disp), int(rng_seed) & (2**64 - 1),
                                  int(stream_id) & (2**64 - 1), int(step), int(d_max), int(vn_waves),
                                  int(extra), int(metric)))

    def stamp(self):
        N.check(self._lib.vd_stamp(self._h))

    def jump_pass(self, k: int, nb: int = MOORE, metric: int = EUCLID):
        N.check(self._lib.vd_pass(self._h, int(k), int(nb), int(metric)))

    def autotune(self, d_max: int, max_disp: int, vn_waves: int = 2, metric: int = EUCLID, rng_seed: int = 0,
                 steps: int = 5):
        """Times the pass launch shapes on this context's dJFA steps and keeps
        the fastest (state left as it was; see vd_autotune).  Returns
        ({option: value}, [ms per step of each candidate measured])."""
        chosen = np.zeros(9, np.int32)
        times = np.zeros(64, np.float64)
        n = self._lib.vd_autotune(self._h, int(d_max), int(max_disp), int(vn_waves), int(metric),
                                  int(rng_seed) & (2**64 - 1), int(steps),
                                  chosen.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), times.ctypes.data, 64)
        N.check(min(n, 0))
        names = ["pass_tile", "dedup_gathers", "sparse_pass", "blocked_pass", "blocked_min_blocks", "fuse_max_k",
                 "smem_tile_max_k", "smem_tile_rows", "packed_map"]
        return dict(zip(names, (int(v) for v in chosen))), [float(t) for t in times[:n]]

    def pass_rows(self, k: int, nb: int, y0: int, y1: int, metric: int = EUCLID, djfa_frame: bool = True):
        """One pass writing only rows [y0, y1) of the next map (one band of a
        split map; see vd_pass_rows)."""
        N.check(self._lib.vd_pass_rows(self._h, int(k), int(nb), int(metric), int(y0), int(y1),
                                       1 if djfa_frame else 0))

    def clear_labels(self):
        """Empties the current map (label -1 everywhere)."""
        N.check(self._lib.vd_clear_labels(self._h))

    # -- maps -----------------------------------------------------------
    def set_labels(self, labels):
        ptr, dev = _buf(labels, self.w * self.h)
        N.check(self._lib.vd_set_labels(self._h, ptr, dev))

    def labels(self, out=None):
        """The current label map as a dense (h, w) int32 array (or into ``out``)."""
        if out is None:
            out = np.empty((self.h, self.w), np.int32)
        ptr, dev = _buf(out, self.w * self.h, writable=True)
        N.check(self._lib.vd_get_labels(self._h, ptr, dev))
        return out

    def labels_async(self, out):
        """Queues a copy of the current map into host array/tensor ``out``
        (page-locked for overlap); complete after :meth:`wait_labels`."""
        ptr, dev = _buf(out, self.w * self.h, writable=True)
        if dev:
            raise ValueError("labels_async copies to host memory")
        N.check(self._lib.vd_get_labels_async(self._h, ptr))
        return out

    def labels16_async(self, out):
        """As :meth:`labels_async` into a contiguous host uint16 array or tensor
        of h * w elements (the empty label as 0xFFFF; at most 65535 seeds)."""
        if _is_torch(out):
            import torch

            if out.dtype not in (torch.uint16, torch.int16) or not out.is_contiguous() or out.is_cuda:
                raise TypeError("out must be a contiguous host uint16/int16 tensor")
            n, ptr = out.numel(), out.data_ptr()
        else:
            if not isinstance(out, np.ndarray) or out.dtype != np.uint16 or not out.flags.c_contiguous:
                raise TypeError("out must be a C-contiguous uint16 numpy array")
            if not out.flags.writeable:
                raise ValueError("output array is read-only")
            n, ptr = out.size, out.ctypes.data
        if n != self.w * self.h:
            raise ValueError(f"expected {self.w * self.h} elements, got {n}")
        N.check(self._lib.vd_get_labels16_async(self._h, ptr))
        return out

    def labels24_async(self, out):
        """As :meth:`labels_async` into a contiguous host uint8 array or tensor
        of 3 * h * w bytes: each label as three little-endian bytes, the empty
        label as 0xFFFFFF (at most 16777215 seeds); :func:`widen24` turns it
        back into int32 labels."""
        if _is_torch(out):
            if str(out.dtype) != "torch.uint8" or not out.is_contiguous() or out.is_cuda:
                raise TypeError("out must be a contiguous host uint8 tensor")
            n, ptr = out.numel(), out.data_ptr()
        else:
            if not isinstance(out, np.ndarray) or out.dtype != np.uint8 or not out.flags.c_contiguous:
                raise TypeError("out must be a C-contiguous uint8 numpy array")
            if not out.flags.writeable:
                raise ValueError("output array is read-only")
            n, ptr = out.size, out.ctypes.data
        if n != 3 * self.w * self.h:
            raise ValueError(f"expected {3 * self.w * self.h} bytes, got {n}")
        N.check(self._lib.vd_get_labels24_async(self._h, ptr))
        return out

    def labels_packed_async(self, out, bits: int):
        """As :meth:`labels_async` into a contiguous host uint8 array or tensor
        of ceil(h * w * bits / 8) bytes: a bit stream of `bits`-bit labels,
        the empty label as 2^bits - 1 (at most 2^bits - 1 seeds; see
        :func:`label_bits`); :func:`unpack_labels` turns it back into int32
        labels."""
        if _is_torch(out):
            if str(out.dtype) != "torch.uint8" or not out.is_contiguous() or out.is_cuda:
                raise TypeError("out must be a contiguous host uint8 tensor")
            n, ptr = out.numel(), out.data_ptr()
        else:
            if not isinstance(out, np.ndarray) or out.dtype != np.uint8 or not out.flags.c_contiguous:
                raise TypeError("out must be a C-contiguous uint8 numpy array")
            if not out.flags.writeable:
                raise ValueError("output array is read-only")
            n, ptr = out.size, out.ctypes.data
        want = (self.w * self.h * int(bits) + 7) // 8
        if n != want:
            raise ValueError(f"expected {want} bytes, got {n}")
        N.check(self._lib.vd_get_labels_packed_async(self._h, ptr, int(bits)))
        return out

    def wait_labels(self):
        N.check(self._lib.vd_wait_labels(self._h))

    def labels_device_ptr(self) -> int:
        p = ctypes.c_void_p()
        N.check(self._lib.vd_labels_device_ptr(self._h, ctypes.byref(p)))
        return int(p.value or 0)

    def similarity(self, exact_dist=None, ref_labels=None, metric: int = EUCLID):
        """(n_exact, n_match) counts of Section VI-A."""
        n = self.w * self.h
        pe, de = _buf(exact_dist, n)
        pr, dr = _buf(ref_labels, n)
        if exact_dist is not None and ref_labels is not None and de != dr:
            raise ValueError("both references must live on the same side")
        on_dev = de if exact_dist is not None else dr
        ne, nm = ctypes.c_uint64(), ctypes.c_uint64()
        N.check(self._lib.vd_similarity(self._h, pe, pr, on_dev, int(metric), ctypes.byref(ne), ctypes.byref(nm)))
        return int(ne.value), int(nm.value)

    def match_count(self, other: "VoronoiSim") -> int:
        """Pixels whose label equals ``other``'s current label (same grid)."""
        nm = ctypes.c_uint64()
        N.check(self._lib.vd_similarity_ctx(self._h, other._h, ctypes.byref(nm)))
        return int(nm.value)

    def exact(self, labels_out=None, dist_out=None, metric: int = EUCLID):
        """The exact diagram of Eq. 1 computed on the GPU: (labels, dist)."""
        if labels_out is None and dist_out is None:
            labels_out = np.empty((self.h, self.w), np.int32)
            dist_out = np.empty((self.h, self.w), np.int32)
        n = self.w * self.h
        pl, dl = _buf(labels_out, n, writable=True)
        pd, dd = _buf(dist_out, n, writable=True)
        if labels_out is not None and dist_out is not None and dl != dd:
            raise ValueError("both outputs must live on the same side")
        on_dev = dl if labels_out is not None else dd
        N.check(self._lib.vd_exact(self._h, pl, pd, on_dev, int(metric)))
        return labels_out, dist_out


BMODE_ROUNDS, BMODE_PERSISTENT = 0, 1
BOPT_MODE = 1
BOPT_ROWS_PER_THREAD = 2
BOPT_BLOCKS_PER_SM = 3
BOPT_USE_GRAPHS = 4
BOPT_BARRIER_TIMEOUT_US = 5
BOPT_TEST_SKIP_ARRIVE = 6
BOPT_CLAMPED_KEYS = 7
BOPT_PERSISTENT_BYTE_KEYS = 8
BOPT_PERSISTENT_MIN_BLOCKS = 9
BOPT_PACKED_MAP = 10


class VoronoiBatch:
    """Many independent simulations stepped together on the GPU (sim-major seeds)."""

    def __init__(self, shapes, stream=None):
        """``shapes``: iterable of (w, h, n_seeds)."""
        shapes = [tuple(int(v) for v in s) for s in shapes]
        w = np.array([s[0] for s in shapes], np.int32)
        h = np.array([s[1] for s in shapes], np.int32)
        n = np.array([s[2] for s in shapes], np.int32)
        self._lib = N.lib()
        handle = self._lib.vd_batch_create(len(shapes), w.ctypes.data, h.ctypes.data, n.ctypes.data)
        if not handle:
            raise N.VDError(N.VD_EINVAL, N.last_error())
        self._h = ctypes.c_void_p(handle)
        self.shapes = shapes
        self.seed_offsets = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
        self.total_seeds = int(n.sum())
        self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.vd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.shapes)

    def set_stream(self, stream=None):
        if stream is None:
            handle = _current_stream_handle()
        elif hasattr(stream, "cuda_stream"):
            handle = stream.cuda_stream
        else:
            handle = int(stream)
        N.check(self._lib.vd_batch_set_stream(self._h, ctypes.c_void_p(handle)))

    def synchronize(self):
        N.check(self._lib.vd_batch_synchronize(self._h))

    def set_option(self, option: int, value: int):
        N.check(self._lib.vd_batch_set_option(self._h, option, int(value)))

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        N.check(self._lib.vd_batch_get_option(self._h, option, ctypes.byref(v)))
        return v.value

    def set_seeds(self, xy_all):
        ptr, dev = _buf(xy_all, 2 * self.total_seeds)
        N.check(self._lib.vd_batch_set_seeds(self._h, ptr, dev))

    def get_seeds(self, sim: int, out=None):
        if out is None:
            out = np.empty((self.shapes[sim][2], 2), np.int32)
        ptr, dev = _buf(out, 2 * self.shapes[sim][2], writable=True)
        N.check(self._lib.vd_batch_get_seeds(self._h, int(sim), ptr, dev))
        return out

    def labels(self, sim: int, out=None):
        w, h, _ = self.shapes[sim]
        if out is None:
            out = np.empty((h, w), np.int32)
        ptr, dev = _buf(out, w * h, writable=True)
        N.check(self._lib.vd_batch_get_labels(self._h, int(sim), ptr, dev))
        return out

    def configure(self, d_max: int, vn_waves: int = 2, extra: int = 0, metric: int = EUCLID):
        N.check(self._lib.vd_batch_configure(self._h, int(d_max), int(vn_waves), int(extra), int(metric)))

    def jfa(self, metric: int = EUCLID):
        N.check(self._lib.vd_batch_jfa(self._h, int(metric)))

    def step(self, dxy_all=None, max_disp: int = 0, rng_seed: int = 0):
        ptr, dev = _buf(dxy_all, 2 * self.total_seeds)
        N.check(self._lib.vd_batch_step(self._h, ptr, dev, int(max_disp), int(rng_seed) & (2**64 - 1)))

    def step_subset(self, sims, max_disp: int, rng_seed: int = 0):
        a = np.ascontiguousarray(sims, np.int32)
        N.check(self._lib.vd_batch_step_subset(self._h, a.ctypes.data, len(a), int(max_disp),
                                               int(rng_seed) & (2**64 - 1)))

    def autotune(self, steps: int, max_disp: int, rng_seed: int = 0):
        """(best candidate index, ms per step of every candidate)."""
        best = ctypes.c_int32(-1)
        ms = np.zeros(32, np.float64)
        n = N.check(self._lib.vd_batch_autotune(self._h, int(steps), int(max_disp), int(rng_seed) & (2**64 - 1),
                                                ctypes.byref(best), ms.ctypes.data, 32))
        return best.value, ms[:n].tolist()

    def work(self):
        """(pixels, pixel-passes of one configured dJFA step, seeds)."""
        px, pp, sd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        N.check(self._lib.vd_batch_work(self._h, ctypes.byref(px), ctypes.byref(pp), ctypes.byref(sd)))
        return px.value, pp.value, sd.value

    @property
    def launches(self) -> int:
        return int(self._lib.vd_batch_launch_count(self._h))


class VoronoiServer:
    """Resident simulations served by step requests with continuous batching."""

    def __init__(self, max_sims: int, hbm_budget_bytes: int, d_max: int, max_disp: int, vn_waves: int = 2,
                 metric: int = EUCLID, rng_seed: int = 0):
        self._lib = N.lib()
        handle = self._lib.vd_server_create(int(max_sims), int(hbm_budget_bytes), int(d_max), int(vn_waves),
                                            int(metric), int(max_disp), int(rng_seed) & (2**64 - 1))
        if not handle:
            raise N.VDError(N.VD_EINVAL, N.last_error())
        self._h = ctypes.c_void_p(handle)
        self.shapes = {}

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.vd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_sim(self, w: int, h: int, xy) -> int:
        xy = np.ascontiguousarray(xy, np.int32).reshape(-1, 2)
        sim = N.check(self._lib.vd_server_add_sim(self._h, int(w), int(h), len(xy), xy.ctypes.data))
        self.shapes[sim] = (int(w), int(h), len(xy))
        return sim

    def remove_sim(self, sim: int):
        N.check(self._lib.vd_server_remove_sim(self._h, int(sim)))
        self.shapes.pop(sim, None)

    def submit(self, sim: int, t_arrive: float = -1.0) -> int:
        return N.check(self._lib.vd_server_submit(self._h, int(sim), float(t_arrive)))

    def progress(self) -> int:
        return N.check(self._lib.vd_server_progress(self._h))

    def drain(self):
        N.check(self._lib.vd_server_drain(self._h))

    def completions(self, cap: int = 65536):
        t = np.zeros(cap, np.int64)
        lat = np.zeros(cap, np.float64)
        sims = np.zeros(cap, np.int32)
        n = N.check(self._lib.vd_server_completions(self._h, t.ctypes.data, lat.ctypes.data, sims.ctypes.data, cap))
        return t[:n], lat[:n], sims[:n]

    def now(self) -> float:
        return float(self._lib.vd_server_now(self._h))

    def run_trace(self, arrival_s, sims):
        """Replays (arrival seconds, simulation) pairs; returns per-request latency (s)."""
        a = np.ascontiguousarray(arrival_s, np.float64)
        s = np.ascontiguousarray(sims, np.int32)
        lat = np.zeros(len(a), np.float64)
        N.check(self._lib.vd_server_run_trace(self._h, a.ctypes.data, s.ctypes.data, len(a), lat.ctypes.data))
        return lat

    def labels(self, sim: int, out=None):
        w, h, _ = self.shapes[sim]
        if out is None:
            out = np.empty((h, w), np.int32)
        ptr, dev = _buf(out, w * h, writable=True)
        N.check(self._lib.vd_server_get_labels(self._h, int(sim), ptr, dev))
        return out

    def stats(self) -> dict:
        u, b, p, sd, la = (ctypes.c_int64() for _ in range(5))
        live = ctypes.c_int32()
        N.check(self._lib.vd_server_stats(self._h, ctypes.byref(u), ctypes.byref(b), ctypes.byref(live),
                                          ctypes.byref(p), ctypes.byref(sd), ctypes.byref(la)))
        return {"used_bytes": u.value, "budget_bytes": b.value, "live_sims": live.value, "pending": p.value,
                "steps_done": sd.value, "launches": la.value}

    def set_max_batch(self, n: int):
        N.check(self._lib.vd_server_set_max_batch(self._h, int(n)))
