"""Thin Python binding of the C ABI in ``include/pgg.h`` (ctypes, argument marshalling only).

Every computation runs in the CUDA library ``_lib/libpgg.so``; this module only
converts numpy arrays and Python numbers into the ABI's plain pointers and sizes.
If the library has not been built, loading raises instead of falling back to
anything else. PyTorch, when present, supplies the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpgg.so")
LIB_CHECKED_PATH = os.path.join(_PKG, "_lib", "libpgg_checked.so")

PGG_OK, PGG_ERR_ARG, PGG_ERR_CUDA, PGG_ERR_OOM, PGG_ERR_TIMEOUT, PGG_ERR_STATE = 0, -1, -2, -3, -4, -5
U8, BITPACK = 0, 1
KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_TILED, KERNEL_DIRECT, KERNEL_RESIDENT = 0, 1, 2, 3, 4
GAME_GROUP, GAME_PAIRWISE = 0, 1
GAMES = {"group": GAME_GROUP, "pairwise": GAME_PAIRWISE, GAME_GROUP: GAME_GROUP,
         GAME_PAIRWISE: GAME_PAIRWISE}
LAYOUTS = {"u8": U8, "bitpack": BITPACK, U8: U8, BITPACK: BITPACK}
KERNELS = {"auto": KERNEL_AUTO, "simple": KERNEL_SIMPLE, "tiled": KERNEL_TILED, "direct": KERNEL_DIRECT,
           "resident": KERNEL_RESIDENT}

_lib = None
_lib_checked = None

_vp = ctypes.c_void_p
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_ip = ctypes.POINTER(ctypes.c_int)


class PGGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def _declare(lib):
    sig = {
        "pgg_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, _vp]),
        "pgg_set_params": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
        "pgg_set_game": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "pgg_get_game": (ctypes.c_int, [_vp, _ip, ctypes.POINTER(ctypes.c_double)]),
        "pgg_seed": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double]),
        "pgg_step_mcs": (ctypes.c_int, [_vp, ctypes.c_int64, _vp]),
        "pgg_count_coop": (ctypes.c_int, [_vp, _u64p]),
        "pgg_get_lattice": (ctypes.c_int, [_vp, _u8p, _u64p]),
        "pgg_set_lattice": (ctypes.c_int, [_vp, _u8p, ctypes.c_uint64]),
        "pgg_get_state": (ctypes.c_int, [_vp, _u64p, _u64p]),
        "pgg_get_lattice_packed": (ctypes.c_int, [_vp, _u32p, _u64p]),
        "pgg_set_lattice_packed": (ctypes.c_int, [_vp, _u32p, ctypes.c_uint64]),
        "pgg_stage_lattice_packed": (ctypes.c_int, [_vp, _u32p, ctypes.c_uint64]),
        "pgg_set_kernel_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
        "pgg_threshold_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double), _u32p]),
        "pgg_kernel_time": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
        "pgg_set_schedule": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int]),
        "pgg_get_schedule": (ctypes.c_int, [_vp, _ip, _ip, _ip, _ip]),
        "pgg_set_spin_limit": (ctypes.c_int, [_vp, ctypes.c_uint]),
        "pgg_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _ip, _ip, _ip,
                                        ctypes.POINTER(ctypes.c_float)]),
        "pgg_get_threshold_table": (ctypes.c_int, [_vp, _u32p]),
        "pgg_lattice_device_ptr": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _u64p]),
        "pgg_step_mcs_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_int64, _vp, _vp]),
        "pgg_destroy": (None, [_vp]),
        "pgg_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _ip,
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), _u64p, _vp]),
        "pgg_batch_seed": (ctypes.c_int, [_vp, ctypes.c_double]),
        "pgg_batch_step_mcs": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
        "pgg_batch_set_team_warps": (ctypes.c_int, [_vp, _ip]),
        "pgg_batch_get_team_warps": (ctypes.c_int, [_vp, _ip]),
        "pgg_batch_set_cta_threads": (ctypes.c_int, [_vp, ctypes.c_int]),
        "pgg_batch_get_cta_threads": (ctypes.c_int, [_vp, _ip]),
        "pgg_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _ip, ctypes.POINTER(ctypes.c_float)]),
        "pgg_batch_use_graph": (ctypes.c_int, [_vp, ctypes.c_int]),
        "pgg_batch_get_lattice": (ctypes.c_int, [_vp, ctypes.c_int, _u8p, _u64p]),
        "pgg_batch_set_lattice": (ctypes.c_int, [_vp, ctypes.c_int, _u8p, ctypes.c_uint64]),
        "pgg_batch_size": (ctypes.c_int, [_vp, _ip]),
        "pgg_batch_destroy": (None, [_vp]),
        "pgg_mlp_info": (ctypes.c_int, [_ip, _ip, _ip, _ip]),
        "pgg_mlp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
        "pgg_mlp_set_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
        "pgg_mlp_get_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(ctypes.c_uint16)]),
        "pgg_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
        "pgg_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]),
        "pgg_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _vp]),
        "pgg_mlp_destroy": (None, [_vp]),
        "pgg_last_error": (ctypes.c_char_p, []),
        "pgg_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(checked: bool = False):
    """Load libpgg.so, or with checked=True the index-checking build libpgg_checked.so
    (raises if it was not built)."""
    global _lib, _lib_checked
    if (_lib_checked if checked else _lib) is None:
        path = LIB_CHECKED_PATH if checked else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing; "
                               "run paper_1704_08098_gb300.build.build()")
        try:  # let the library share PyTorch's CUDA runtime when torch is present
            import torch  # noqa: F401
        except Exception:
            pass
        lib = _declare(ctypes.CDLL(path))
        if checked:
            _lib_checked = lib
        else:
            _lib = lib
    return _lib_checked if checked else _lib


def last_error(lib=None) -> str:
    return (lib or load()).pgg_last_error().decode()


def check(status: int, where: str, lib=None) -> None:
    """Raise PGGError with the library's last message when status is not PGG_OK (lib: the
    library that made the call, the normal build by default)."""
    if status != PGG_OK:
        raise PGGError(status, where, last_error(lib))


def current_stream_handle() -> int:
    """The raw cudaStream_t of PyTorch's current stream (0 without torch)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class Lattice:
    """One L x L lattice context (``pgg_ctx``)."""

    def __init__(self, L: int, r: float, K: float, layout="u8", stream: int | None = None,
                 checked: bool = False):
        """checked=True runs on the index-checking build of the library (tests)."""
        self.lib = load(checked)
        self.L = int(L)
        self.layout = LAYOUTS[layout]
        self.stream = current_stream_handle() if stream is None else int(stream)
        h = _vp()
        self._check(self.lib.pgg_create(ctypes.byref(h), self.L, float(r), float(K), self.layout,
                                  _vp(self.stream)), "pgg_create")
        self._h = h

    def _check(self, status: int, where: str) -> None:
        check(status, where, self.lib)

    # -- lifetime ------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.pgg_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI calls -------------------------------------------------------------
    def set_params(self, r: float, K: float) -> None:
        self._check(self.lib.pgg_set_params(self._h, float(r), float(K)), "pgg_set_params")

    def set_game(self, game="group", payoff=None) -> None:
        """pgg_set_game: "group" (the default) or "pairwise" with payoff = (R, S, T, P)."""
        g = GAMES[game]
        if payoff is None:
            ptr = None
        else:
            pay = np.ascontiguousarray(np.asarray(payoff, dtype=np.float64))
            assert pay.shape == (4,)
            ptr = pay.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self.lib.pgg_set_game(self._h, g, ptr), "pgg_set_game")

    def game(self) -> tuple[str, tuple]:
        g = ctypes.c_int()
        pay = np.zeros(4, dtype=np.float64)
        self._check(self.lib.pgg_get_game(self._h, ctypes.byref(g),
                                    pay.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "pgg_get_game")
        return ("pairwise" if g.value == GAME_PAIRWISE else "group"), tuple(float(x) for x in pay)

    def seed(self, seed: int, p: float = 0.5) -> None:
        self._check(self.lib.pgg_seed(self._h, int(seed), float(p)), "pgg_seed")

    def step_mcs(self, n_mcs: int, counts: np.ndarray | int | None = None):
        """Advance n_mcs MCS. ``counts`` may be None (no counts), a host uint64 numpy
        array of length >= n_mcs (filled; the call synchronises), or an int device
        pointer (filled asynchronously). With counts=None a host array is returned."""
        if counts is None:
            out = np.zeros(max(int(n_mcs), 1), dtype=np.uint64)
            self._check(self.lib.pgg_step_mcs(self._h, int(n_mcs), out.ctypes.data), "pgg_step_mcs")
            return out[:n_mcs]
        if isinstance(counts, np.ndarray):
            assert counts.dtype == np.uint64 and counts.size >= n_mcs and counts.flags.c_contiguous
            self._check(self.lib.pgg_step_mcs(self._h, int(n_mcs), counts.ctypes.data), "pgg_step_mcs")
            return counts
        self._check(self.lib.pgg_step_mcs(self._h, int(n_mcs), _vp(int(counts))), "pgg_step_mcs")
        return None

    def advance(self, n_mcs: int) -> None:
        """Advance n_mcs MCS without reading counts (asynchronous)."""
        self._check(self.lib.pgg_step_mcs(self._h, int(n_mcs), None), "pgg_step_mcs")

    def count(self) -> int:
        v = ctypes.c_uint64()
        self._check(self.lib.pgg_count_coop(self._h, ctypes.byref(v)), "pgg_count_coop")
        return int(v.value)

    def get(self) -> tuple[np.ndarray, int]:
        out = np.empty((self.L, self.L), dtype=np.uint8)
        step = ctypes.c_uint64()
        self._check(self.lib.pgg_get_lattice(self._h, _ptr(out, _u8p), ctypes.byref(step)),
              "pgg_get_lattice")
        return out, int(step.value)

    def set(self, lattice: np.ndarray, step: int = 0) -> None:
        a = np.ascontiguousarray(lattice, dtype=np.uint8)
        assert a.shape == (self.L, self.L)
        self._check(self.lib.pgg_set_lattice(self._h, _ptr(a, _u8p), int(step)), "pgg_set_lattice")

    def set_from_pointer(self, host_ptr: int, step: int = 0) -> None:
        """pgg_set_lattice from a raw host pointer (e.g. pinned memory)."""
        self._check(self.lib.pgg_set_lattice(self._h, ctypes.cast(host_ptr, _u8p), int(step)),
              "pgg_set_lattice")

    def get_packed(self) -> tuple[np.ndarray, int]:
        """pgg_get_lattice_packed: (L, L/32) uint32 words, bit b of word w = column 32w + b."""
        out = np.empty((self.L, self.L // 32), dtype=np.uint32)
        step = ctypes.c_uint64()
        self._check(self.lib.pgg_get_lattice_packed(self._h, _ptr(out, _u32p), ctypes.byref(step)),
              "pgg_get_lattice_packed")
        return out, int(step.value)

    def set_packed(self, words: np.ndarray, step: int = 0) -> None:
        a = np.ascontiguousarray(words, dtype=np.uint32)
        assert a.shape == (self.L, self.L // 32)
        self._check(self.lib.pgg_set_lattice_packed(self._h, _ptr(a, _u32p), int(step)), "pgg_set_lattice_packed")

    def set_packed_from_pointer(self, host_ptr: int, step: int = 0) -> None:
        """pgg_set_lattice_packed from a raw host pointer (e.g. pinned memory)."""
        self._check(self.lib.pgg_set_lattice_packed(self._h, ctypes.cast(host_ptr, _u32p), int(step)),
              "pgg_set_lattice_packed")

    def stage_packed_from_pointer(self, host_ptr: int, step: int = 0) -> None:
        """pgg_stage_lattice_packed from a raw host pointer (pinned memory, for the copy to
        overlap the work already queued): the next step_mcs (or any call that reads the lattice)
        starts from it. The buffer must stay unchanged until that call's work has run."""
        self._check(self.lib.pgg_stage_lattice_packed(self._h, ctypes.cast(host_ptr, _u32p), int(step)),
                    "pgg_stage_lattice_packed")

    def state(self) -> tuple[int, int]:
        seed, step = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.pgg_get_state(self._h, ctypes.byref(seed), ctypes.byref(step)),
              "pgg_get_state")
        return int(seed.value), int(step.value)

    def set_schedule(self, kernel="auto", steps_per_launch: int = 1, tile_x: int = 0,
                     tile_y: int = 0) -> None:
        kern = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        self._check(self.lib.pgg_set_schedule(self._h, kern, int(steps_per_launch), int(tile_x),
                                        int(tile_y)), "pgg_set_schedule")

    def set_kernel_timing(self, enable: bool) -> None:
        """pgg_set_kernel_timing: CUDA events around every step-kernel launch from now on."""
        self._check(self.lib.pgg_set_kernel_timing(self._h, int(bool(enable))), "pgg_set_kernel_timing")

    def kernel_time(self) -> tuple[float, int]:
        """(summed milliseconds, launches) of the step-kernel launches recorded so far."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self.lib.pgg_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)), "pgg_kernel_time")
        return float(ms.value), int(n.value)

    def set_spin_limit(self, limit: int) -> None:
        self._check(self.lib.pgg_set_spin_limit(self._h, int(limit)), "pgg_set_spin_limit")

    def schedule(self) -> dict:
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self.lib.pgg_get_schedule(self._h, *[ctypes.byref(x) for x in v]),
              "pgg_get_schedule")
        names = {KERNEL_SIMPLE: "simple", KERNEL_TILED: "tiled", KERNEL_AUTO: "auto", KERNEL_DIRECT: "direct",
                 KERNEL_RESIDENT: "resident"}
        return dict(kernel=names[v[0].value], steps_per_launch=v[1].value, tile_x=v[2].value,
                    tile_y=v[3].value)

    def autotune(self, n_mcs: int = 3) -> dict:
        """pgg_autotune: pick the fastest schedule for this (device, L, layout)."""
        v = [ctypes.c_int() for _ in range(4)]
        ms = ctypes.c_float()
        self._check(self.lib.pgg_autotune(self._h, int(n_mcs), *[ctypes.byref(x) for x in v],
                                    ctypes.byref(ms)), "pgg_autotune")
        names = {KERNEL_SIMPLE: "simple", KERNEL_TILED: "tiled", KERNEL_DIRECT: "direct",
                 KERNEL_RESIDENT: "resident"}
        return dict(kernel=names[v[0].value], steps_per_launch=v[1].value, tile_x=v[2].value,
                    tile_y=v[3].value, ms_per_mcs=float(ms.value))

    def threshold_table(self) -> np.ndarray:
        out = np.zeros(2 * 26 * 26, dtype=np.uint32)
        self._check(self.lib.pgg_get_threshold_table(self._h, _ptr(out, _u32p)),
              "pgg_get_threshold_table")
        return out.reshape(2, 26, 26)

    def device_ptr(self) -> tuple[int, int]:
        p, n = _vp(), ctypes.c_uint64()
        self._check(self.lib.pgg_lattice_device_ptr(self._h, ctypes.byref(p), ctypes.byref(n)),
              "pgg_lattice_device_ptr")
        return int(p.value or 0), int(n.value)


def threshold_table(r: float, K: float, game: str = "group", payoff=None) -> np.ndarray:
    """pgg_threshold_table: the (2, 26, 26) uint32 adoption thresholds built on the host (no
    device needed); for the pairwise game the first 2*5*5 entries, indexed (s_x*5 + n_x)*5 + n_y."""
    lib = load()
    out = np.zeros((2, 26, 26), dtype=np.uint32)
    pay = None
    if payoff is not None:
        pay_arr = (ctypes.c_double * 4)(*[float(x) for x in payoff])
        pay = ctypes.cast(pay_arr, ctypes.POINTER(ctypes.c_double))
    check(lib.pgg_threshold_table(GAMES[game], float(r), float(K), pay,
                                  out.ctypes.data_as(_u32p)), "pgg_threshold_table")
    return out


def step_mcs_noalloc(lattice_in: int, lattice_out: int, L: int, layout, r: float, K: float,
                     seed: int, step0: int, n_mcs: int, counts_dev: int | None = None,
                     stream: int | None = None) -> None:
    """pgg_step_mcs_noalloc on raw device pointers (see include/pgg.h): for callers that
    cannot allocate device memory; the library's fixed scratch array is used instead."""
    lib = load()
    st = current_stream_handle() if stream is None else int(stream)
    check(lib.pgg_step_mcs_noalloc(_vp(int(lattice_in)), _vp(int(lattice_out)), int(L),
                                   LAYOUTS[layout], float(r), float(K), int(seed), int(step0),
                                   int(n_mcs), _vp(int(counts_dev)) if counts_dev else None,
                                   _vp(st)), "pgg_step_mcs_noalloc")


class Batch:
    """Many replicas advanced in one persistent launch (``pgg_batch``)."""

    def __init__(self, L, r, K, seeds, stream: int | None = None):
        self.lib = load()
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        n = self.L.size
        rr = np.ascontiguousarray(np.broadcast_to(np.asarray(r, dtype=np.float64), (n,)))
        KK = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.float64), (n,)))
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        assert rr.size == n and KK.size == n and sd.size == n
        self.n = n
        self.stream = current_stream_handle() if stream is None else int(stream)
        h = _vp()
        check(self.lib.pgg_batch_create(ctypes.byref(h), n, _ptr(self.L, _ip),
                                        _ptr(rr, ctypes.POINTER(ctypes.c_double)),
                                        _ptr(KK, ctypes.POINTER(ctypes.c_double)),
                                        _ptr(sd, _u64p), _vp(self.stream)), "pgg_batch_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.pgg_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def seed(self, p: float = 0.5) -> None:
        check(self.lib.pgg_batch_seed(self._h, float(p)), "pgg_batch_seed")

    def step_mcs(self, n_mcs: int, counts=True):
        """Advance all replicas; counts=True returns an (n, n_mcs) uint32 host array,
        counts=None skips them, an int is a device pointer filled asynchronously."""
        if counts is None or counts is False:
            check(self.lib.pgg_batch_step_mcs(self._h, int(n_mcs), None), "pgg_batch_step_mcs")
            return None
        if counts is True:
            out = np.zeros((self.n, max(int(n_mcs), 1)), dtype=np.uint32)
            check(self.lib.pgg_batch_step_mcs(self._h, int(n_mcs), out.ctypes.data),
                  "pgg_batch_step_mcs")
            return out[:, :n_mcs]
        check(self.lib.pgg_batch_step_mcs(self._h, int(n_mcs), _vp(int(counts))),
              "pgg_batch_step_mcs")
        return None

    def get(self, i: int) -> tuple[np.ndarray, int]:
        L = int(self.L[i])
        out = np.empty((L, L), dtype=np.uint8)
        step = ctypes.c_uint64()
        check(self.lib.pgg_batch_get_lattice(self._h, int(i), _ptr(out, _u8p), ctypes.byref(step)),
              "pgg_batch_get_lattice")
        return out, int(step.value)

    def set(self, i: int, lattice: np.ndarray, step: int = 0) -> None:
        a = np.ascontiguousarray(lattice, dtype=np.uint8)
        check(self.lib.pgg_batch_set_lattice(self._h, int(i), _ptr(a, _u8p), int(step)),
              "pgg_batch_set_lattice")

    def set_team_warps(self, warps) -> None:
        w = np.ascontiguousarray(warps, dtype=np.int32)
        check(self.lib.pgg_batch_set_team_warps(self._h, _ptr(w, _ip)), "pgg_batch_set_team_warps")

    def team_warps(self) -> list[int]:
        w = np.zeros(5, dtype=np.int32)
        check(self.lib.pgg_batch_get_team_warps(self._h, _ptr(w, _ip)), "pgg_batch_get_team_warps")
        return [int(x) for x in w]

    def set_cta_threads(self, threads: int) -> None:
        check(self.lib.pgg_batch_set_cta_threads(self._h, int(threads)), "pgg_batch_set_cta_threads")

    def cta_threads(self) -> int:
        v = ctypes.c_int()
        check(self.lib.pgg_batch_get_cta_threads(self._h, ctypes.byref(v)), "pgg_batch_get_cta_threads")
        return int(v.value)

    def use_graph(self, enable: bool) -> None:
        check(self.lib.pgg_batch_use_graph(self._h, int(bool(enable))), "pgg_batch_use_graph")

    def autotune(self, n_mcs: int = 20) -> dict:
        w = np.zeros(5, dtype=np.int32)
        ms = ctypes.c_float()
        check(self.lib.pgg_batch_autotune(self._h, int(n_mcs), _ptr(w, _ip), ctypes.byref(ms)),
              "pgg_batch_autotune")
        return dict(team_warps=[int(x) for x in w], cta_threads=self.cta_threads(),
                    ms=float(ms.value))


class MLP:
    """The surrogate network (``pgg_mlp``); X, Y and outputs are device pointers (int)."""

    def __init__(self, max_batch: int, stream: int | None = None):
        self.lib = load()
        v = [ctypes.c_int() for _ in range(4)]
        check(self.lib.pgg_mlp_info(*[ctypes.byref(x) for x in v]), "pgg_mlp_info")
        self.n_in, self.n_hidden, self.n_out, self.n_params = (x.value for x in v)
        self.max_batch = int(max_batch)
        self.stream = current_stream_handle() if stream is None else int(stream)
        h = _vp()
        check(self.lib.pgg_mlp_create(ctypes.byref(h), self.max_batch, _vp(self.stream)),
              "pgg_mlp_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.pgg_mlp_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, master: np.ndarray) -> None:
        a = np.ascontiguousarray(master, dtype=np.float32)
        assert a.size == self.n_params
        check(self.lib.pgg_mlp_set_params(self._h, _ptr(a, ctypes.POINTER(ctypes.c_float))),
              "pgg_mlp_set_params")

    def get_params(self) -> tuple[np.ndarray, np.ndarray]:
        """(FP32 master, BF16 image as float32 values)."""
        m = np.zeros(self.n_params, dtype=np.float32)
        q = np.zeros(self.n_params, dtype=np.uint16)
        check(self.lib.pgg_mlp_get_params(self._h, _ptr(m, ctypes.POINTER(ctypes.c_float)),
                                          _ptr(q, ctypes.POINTER(ctypes.c_uint16))),
              "pgg_mlp_get_params")
        return m, (q.astype(np.uint32) << 16).view(np.float32)

    def forward(self, X_dev: int, B: int, out_dev: int) -> None:
        check(self.lib.pgg_mlp_forward(self._h, _vp(X_dev), int(B), _vp(out_dev)), "pgg_mlp_forward")

    def loss_grad(self, X_dev: int, Y_dev: int, B: int, loss_dev: int | None,
                  grad_dev: int | None) -> None:
        check(self.lib.pgg_mlp_loss_grad(self._h, _vp(X_dev), _vp(Y_dev), int(B),
                                         _vp(loss_dev) if loss_dev else None,
                                         _vp(grad_dev) if grad_dev else None), "pgg_mlp_loss_grad")

    def train_step(self, X_dev: int, Y_dev: int, B: int, lr: float, loss_dev: int | None = None) -> None:
        check(self.lib.pgg_mlp_train_step(self._h, _vp(X_dev), _vp(Y_dev), int(B), float(lr),
                                          _vp(loss_dev) if loss_dev else None), "pgg_mlp_train_step")


def version() -> str:
    return load().pgg_version().decode()
