"""CPU oracle for discrete Voronoi diagrams, JFA and dJFA.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  It is the independent checker of the CUDA library: it shares no
code, header, table or helper with it, and the product path never calls it.

The arithmetic lives in ``vd_oracle.c`` (plain C, compiled by :func:`build`);
this module only marshals numpy arrays into it.  Each wrapper names the part of
the paper ("GPU Voronoi Diagrams for Random Moving Seeds") that it follows:

* Eq. 1 (Section II)   -- :func:`exact_brute`, :func:`exact_dist_edt`
* Eq. 2 (Section III)  -- :func:`jfa_first_step`, :func:`jfa_schedule`
* Table I (Section III)-- :func:`jump_pass` (Moore), Section V-B (Von Neumann)
* Eq. 3-4 (Section V-A) -- :func:`djfa_first_step`, :func:`djfa_schedule`
* Algorithm 1 (Section V-D) -- :func:`stamp`, :func:`jfa`, :func:`djfa_step`
* Section VI-A         -- :func:`similarity`

Parity status: pinned (see ``tests/test_oracle_pins.py``); no function here is
unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvd_oracle.so")

EUCLID = 0
MANHATTAN = 1
MOORE = 0
VON_NEUMANN = 1

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compiles ``vd_oracle.c`` with gcc (OpenMP) into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-Wno-unknown-pragmas", "-Wno-maybe-uninitialized", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32, i64, u64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        c_int = ctypes.c_int
        sig = {
            "orc_set_threads": (None, [c_int]),
            "orc_get_threads": (c_int, []),
            "orc_distance": (i64, [i32, i32, i32, i32, c_int]),
            "orc_jfa_first_step": (i32, [i32, i32]),
            "orc_djfa_first_step_uncapped": (i64, [i32, i32, i64, i32]),
            "orc_djfa_first_step": (i32, [i32, i32, i64, i32]),
            "orc_jfa_schedule": (c_int, [i32, i32, c_int, p, p, c_int]),
            "orc_djfa_schedule": (c_int, [i32, i32, i64, i32, c_int, c_int, p, p, c_int]),
            "orc_exact_brute": (None, [i32, i32, i64, p, c_int, p, p]),
            "orc_exact_dist_edt": (None, [i32, i32, i64, p, c_int, p]),
            "orc_move": (None, [i32, i32, i64, p, p]),
            "orc_splitmix64": (u64, [u64, u64]),
            "orc_rng_displacement": (i32, [u64, u64, u64, u64, c_int, i32]),
            "orc_move_rng": (None, [i32, i32, i64, p, i32, u64, u64, u64]),
            "orc_fill": (None, [i32, i32, p, i32]),
            "orc_stamp": (None, [i32, i32, i64, p, p]),
            "orc_pass": (None, [i32, i32, p, p, p, i32, c_int, c_int]),
            "orc_jfa": (None, [i32, i32, i64, p, c_int, c_int, p]),
            "orc_djfa_step": (None, [i32, i32, i64, p, i32, c_int, c_int, c_int, p]),
            "orc_similarity": (None, [i32, i32, p, p, p, p, c_int, p, p]),
            "orc_update_seeds": (i64, [i32, i32, i64, p, p, p, i64, p, i64, p]),
            "orc_repair_step": (None, [i32, i32, i64, p, c_int, c_int, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _seeds(xy) -> np.ndarray:
    a = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1, 2)
    return a


def _map(a, w, h) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int32)
    assert a.size == w * h, (a.shape, w, h)
    return a.reshape(h, w)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def distance(sx, sy, px, py, metric=EUCLID) -> int:
    """Section II distance d (squared Euclidean, or Manhattan of Section V-C)."""
    return int(_load().orc_distance(sx, sy, px, py, metric))


def jfa_first_step(w: int, h: int) -> int:
    """k_1 of Eq. 2 for a w x h grid (N = max(w, h)); 0 when N = 1."""
    return int(_load().orc_jfa_first_step(w, h))


def djfa_first_step(w: int, h: int, s: int, d_max: int, capped: bool = True) -> int:
    """delta_1 of Eq. 4 (exact integer form), capped at k_1 unless told not to."""
    lib = _load()
    if capped:
        return int(lib.orc_djfa_first_step(w, h, s, d_max))
    return int(lib.orc_djfa_first_step_uncapped(w, h, s, d_max))


def _schedule(fn, *args):
    ks = np.zeros(80, np.int32)
    nbs = np.zeros(80, np.int32)
    n = fn(*args, _ptr(ks), _ptr(nbs), 80)
    return [(int(ks[i]), int(nbs[i])) for i in range(n)]


def jfa_schedule(w: int, h: int, extra: int = 0):
    """[(k, neighbourhood), ...] of a JFA frame (Eq. 2, Table I, JFA+1/+2)."""
    return _schedule(_load().orc_jfa_schedule, w, h, extra)


def djfa_schedule(w: int, h: int, s: int, d_max: int, vn_waves: int = 2, extra: int = 0):
    """[(k, neighbourhood), ...] of a dJFA frame (Eq. 4, Section V-B)."""
    return _schedule(_load().orc_djfa_schedule, w, h, s, d_max, vn_waves, extra)


def exact_brute(w: int, h: int, xy, metric=EUCLID):
    """(label*, D*) of Eq. 1 by brute force; lowest index among equal distances."""
    xy = _seeds(xy)
    label = np.empty((h, w), np.int32)
    dist = np.empty((h, w), np.int32)
    _load().orc_exact_brute(w, h, len(xy), _ptr(xy), metric, _ptr(label), _ptr(dist))
    return label, dist


def exact_dist_edt(w: int, h: int, xy, metric=EUCLID):
    """D* of Eq. 1 by the separable exact distance transform (Felzenszwalb-Huttenlocher)."""
    xy = _seeds(xy)
    dist = np.empty((h, w), np.int32)
    _load().orc_exact_dist_edt(w, h, len(xy), _ptr(xy), metric, _ptr(dist))
    return dist


def move(w: int, h: int, xy, dxy) -> np.ndarray:
    """Seeds moved by integer displacements, clamped to the grid (returns a copy)."""
    out = _seeds(xy).copy()
    d = _seeds(dxy)
    assert d.shape == out.shape
    _load().orc_move(w, h, len(out), _ptr(out), _ptr(d))
    return out


def splitmix64(seed: int, n: int) -> int:
    """n-th output of SplitMix64 started at state ``seed``."""
    return int(_load().orc_splitmix64(seed, n))


def rng_displacement(rng_seed: int, stream: int, step: int, k: int, axis: int, max_disp: int) -> int:
    return int(_load().orc_rng_displacement(rng_seed, stream, step, k, axis, max_disp))


def move_rng(w: int, h: int, xy, max_disp: int, rng_seed: int, stream: int, step: int) -> np.ndarray:
    """Seeds moved by counter-based SplitMix64 displacements in [-max_disp, max_disp]."""
    out = _seeds(xy).copy()
    _load().orc_move_rng(w, h, len(out), _ptr(out), max_disp, rng_seed, stream, step)
    return out


def stamp(w: int, h: int, xy, label) -> np.ndarray:
    """Each seed pixel gets the lowest seed index standing on it (returns a copy)."""
    xy = _seeds(xy)
    out = _map(label, w, h).copy()
    _load().orc_stamp(w, h, len(xy), _ptr(xy), _ptr(out))
    return out


def jump_pass(w: int, h: int, xy, src, k: int, nb=MOORE, metric=EUCLID) -> np.ndarray:
    """One gather pass at step k (Table I / Section V-B); returns the new map."""
    xy = _seeds(xy)
    src = _map(src, w, h)
    dst = np.empty_like(src)
    _load().orc_pass(w, h, _ptr(xy), _ptr(src), _ptr(dst), k, nb, metric)
    return dst


def jfa(w: int, h: int, xy, extra: int = 0, metric=EUCLID) -> np.ndarray:
    """Full JFA frame from an empty map (Section III)."""
    xy = _seeds(xy)
    label = np.empty((h, w), np.int32)
    _load().orc_jfa(w, h, len(xy), _ptr(xy), extra, metric, _ptr(label))
    return label


def djfa_step(w: int, h: int, xy, prev_label, d_max: int, vn_waves: int = 2,
              extra: int = 0, metric=EUCLID) -> np.ndarray:
    """One dJFA frame on the previous map (Algorithm 1 after SimulateParticles)."""
    xy = _seeds(xy)
    label = _map(prev_label, w, h).copy()
    _load().orc_djfa_step(w, h, len(xy), _ptr(xy), d_max, vn_waves, extra, metric, _ptr(label))
    return label


def update_seeds(w: int, h: int, xy, label, remove=(), add=()):
    """Seed removal and insertion between frames (this library's rule; the
    paper leaves it to future work): survivors keep their order, new seeds are
    appended, the map is relabelled (a removed seed's pixels become -1).
    Returns (new seeds, new map), or None when the update is invalid."""
    xy = _seeds(xy)
    label = _map(label, w, h).copy()
    rem = np.ascontiguousarray(remove, dtype=np.int32).reshape(-1)
    add = np.ascontiguousarray(add, dtype=np.int32).reshape(-1, 2)
    out = np.empty((max(len(xy) + len(add), 1), 2), np.int32)
    n = _load().orc_update_seeds(w, h, len(xy), _ptr(xy), _ptr(label), _ptr(rem), len(rem),
                                 _ptr(add), len(add), _ptr(out))
    if n < 0:
        return None
    return out[:n].copy(), label


def repair_step(w: int, h: int, xy, label, extra: int = 0, metric=EUCLID) -> np.ndarray:
    """The frame after a removal: stamp, then the full JFA schedule on the map."""
    xy = _seeds(xy)
    out = _map(label, w, h).copy()
    _load().orc_repair_step(w, h, len(xy), _ptr(xy), extra, metric, _ptr(out))
    return out


def similarity(w: int, h: int, xy, label, exact_dist=None, ref_label=None, metric=EUCLID):
    """(n_exact, n_match) of Section VI-A: distance-correct and label-equal pixel counts."""
    xy = _seeds(xy)
    label = _map(label, w, h)
    ed = None if exact_dist is None else _map(exact_dist, w, h)
    rl = None if ref_label is None else _map(ref_label, w, h)
    ne = ctypes.c_uint64(0)
    nm = ctypes.c_uint64(0)
    _load().orc_similarity(w, h, _ptr(xy), _ptr(label), _ptr(ed), _ptr(rl), metric,
                           ctypes.byref(ne), ctypes.byref(nm))
    return int(ne.value), int(nm.value)
