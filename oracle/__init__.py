"""CPU oracle for the spatial public goods game Monte Carlo (arXiv:1704.08098).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The GPU library never
loads it, and it never loads the GPU library.

The arithmetic lives in ``pgg_oracle.c`` (plain C, built with gcc by
:func:`build`); this module only marshals numpy arrays through ctypes. The C
header comment states what each function computes and which passage of the
paper it follows (Section III, Eq. (1)-(4); Section IV for the schedule).

Parity status of each function (what pins it; the tests live in ``tests/``):
  philox4x32_10        Random123 known-answer vectors (tests/golden).
  group / payoff       hand-worked lattices (tests/golden), brute-force group
                       membership on tiny tori, closed forms (all-C, all-D).
  fermi_threshold      W(D) + W(-D) = 1, tie = 2^31, K -> 0 and K -> inf limits.
  run / classic_run    absorbing states, order independence, statistical
                       agreement of the two schedules, rho_C = 0.5 at r = 3.98,
                       K = 0.5 (Section V, Fig. 5 caption), extinction below r_c.
  pair_*               the pairwise game of Section VI: hand-worked payoffs
                       (tests/golden), bond-by-bond brute force on tiny tori,
                       closed forms, the radius-2 read set of an update (Section
                       VI: one line less than the group game), a brute-force
                       replay of whole steps, equal payoffs = coin flips,
                       absorbing states, order independence, schedule agreement.
  offset / dir / u,    the stream layout is a convention (the paper names no
  init                 generator), so no outside value fixes it: the pins write the
                       documented counter layout out over the known-answer-pinned
                       Philox primitive and require these draws to follow it, then
                       replay whole group-game and pairwise steps from it with
                       brute-force payoffs; uniformity checks besides.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-fopenmp"]


def compile_source(src: str, out: str, extra: list[str] | None = None) -> str:
    """Compile a C oracle source file into a shared library with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", *CFLAGS, *(extra or []), "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Build ``oracle/_build/liboracle.so`` if missing or older than its source."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            compile_source(_SRC, _SO)
    return _SO


_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _declare(lib):
    lib.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_offset.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_offset.restype = ctypes.c_int
    lib.oracle_dir.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
    lib.oracle_dir.restype = ctypes.c_int
    lib.oracle_u.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
    lib.oracle_u.restype = ctypes.c_uint32
    lib.oracle_group_cooperators.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_group_cooperators.restype = ctypes.c_int
    lib.oracle_payoff_groups.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.oracle_payoff_groups.restype = ctypes.c_double
    lib.oracle_group_count_total.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_group_count_total.restype = ctypes.c_int
    lib.oracle_payoff_total.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.oracle_payoff_total.restype = ctypes.c_double
    lib.oracle_fermi_threshold.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.oracle_fermi_threshold.restype = ctypes.c_uint32
    lib.oracle_elementary_update.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_double]
    lib.oracle_elementary_update.restype = ctypes.c_int
    lib.oracle_init.argtypes = [_u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double]
    lib.oracle_init.restype = None
    lib.oracle_count.argtypes = [_u8p, ctypes.c_int]
    lib.oracle_count.restype = ctypes.c_uint64
    lib.oracle_sublattice_step.argtypes = [_u8p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_int]
    lib.oracle_sublattice_step.restype = ctypes.c_int64
    lib.oracle_run.argtypes = [_u8p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, _u64p,
                               ctypes.c_int, ctypes.c_int]
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_classic_run.argtypes = [_u8p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, _u64p]
    lib.oracle_classic_run.restype = ctypes.c_int
    _dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_pair_neighbour_cooperators.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_pair_neighbour_cooperators.restype = ctypes.c_int
    lib.oracle_pair_payoff_games.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    lib.oracle_pair_payoff_games.restype = ctypes.c_double
    lib.oracle_pair_payoff_total.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
    lib.oracle_pair_payoff_total.restype = ctypes.c_double
    lib.oracle_pair_update_threshold.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, _dp, ctypes.c_double]
    lib.oracle_pair_update_threshold.restype = ctypes.c_uint32
    lib.oracle_pair_elementary_update.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_uint32, _dp, ctypes.c_double]
    lib.oracle_pair_elementary_update.restype = ctypes.c_int
    lib.oracle_pair_sublattice_step.argtypes = [_u8p, ctypes.c_int, _dp, ctypes.c_double,
                                                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                                ctypes.c_int]
    lib.oracle_pair_sublattice_step.restype = ctypes.c_int64
    lib.oracle_pair_run.argtypes = [_u8p, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_int64, _u64p, ctypes.c_int, ctypes.c_int]
    lib.oracle_pair_run.restype = ctypes.c_int
    lib.oracle_pair_classic_run.argtypes = [_u8p, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_int64, _u64p]
    lib.oracle_pair_classic_run.restype = ctypes.c_int
    lib.oracle_error_count.argtypes = []
    lib.oracle_error_count.restype = ctypes.c_int
    lib.oracle_clear_errors.argtypes = []
    lib.oracle_clear_errors.restype = None
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads another build."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class Oracle:
    """numpy-facing wrapper around one loaded oracle library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    # --- random stream -------------------------------------------------------
    def philox(self, ctr, key) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
        k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
        out = np.zeros(4, dtype=np.uint32)
        self.lib.oracle_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
        return out

    def offset(self, seed: int, k: int) -> int:
        return self.lib.oracle_offset(seed, k)

    def dir(self, seed: int, k: int, a: int, b: int) -> int:
        return self.lib.oracle_dir(seed, k, a, b)

    def u(self, seed: int, k: int, a: int, b: int) -> int:
        return self.lib.oracle_u(seed, k, a, b)

    # --- the game ------------------------------------------------------------
    @staticmethod
    def _lat(lat) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(lat, dtype=np.uint8))
        assert a.ndim == 2 and a.shape[0] == a.shape[1]
        return a

    def group_cooperators(self, lat, ci: int, cj: int) -> int:
        a = self._lat(lat)
        return self.lib.oracle_group_cooperators(_ptr(a, _u8p), a.shape[0], ci, cj)

    def payoff_groups(self, lat, i: int, j: int, r: float) -> float:
        a = self._lat(lat)
        return self.lib.oracle_payoff_groups(_ptr(a, _u8p), a.shape[0], i, j, r)

    def group_count_total(self, lat, i: int, j: int) -> int:
        a = self._lat(lat)
        return self.lib.oracle_group_count_total(_ptr(a, _u8p), a.shape[0], i, j)

    def payoff_total(self, s: int, S: int, r: float) -> float:
        return self.lib.oracle_payoff_total(s, S, r)

    def threshold(self, pi_x: float, pi_y: float, K: float) -> int:
        return self.lib.oracle_fermi_threshold(pi_x, pi_y, K)

    def elementary_update(self, lat: np.ndarray, i: int, j: int, d: int, u: int, r: float,
                          K: float) -> int:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        return self.lib.oracle_elementary_update(_ptr(lat, _u8p), lat.shape[0], i, j, d, u, r, K)

    # --- dynamics --------------------------------------------------------------
    def init(self, L: int, seed: int, p: float = 0.5) -> np.ndarray:
        lat = np.zeros((L, L), dtype=np.uint8)
        self.lib.oracle_init(_ptr(lat, _u8p), L, seed, p)
        return lat

    def count(self, lat) -> int:
        a = self._lat(lat)
        return int(self.lib.oracle_count(_ptr(a, _u8p), a.shape[0]))

    def sublattice_step(self, lat: np.ndarray, r: float, K: float, seed: int, k: int,
                        reverse: bool = False, threads: int = 1) -> int:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        return int(self.lib.oracle_sublattice_step(_ptr(lat, _u8p), lat.shape[0], r, K, seed, k,
                                                   int(reverse), threads))

    def run(self, lat: np.ndarray, r: float, K: float, seed: int, k0: int, n_mcs: int,
            reverse: bool = False, threads: int = 1) -> np.ndarray:
        """Advance ``lat`` in place by ``n_mcs`` MCS from sublattice step ``k0``;
        returns the cooperator count after each MCS."""
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        counts = np.zeros(max(n_mcs, 1), dtype=np.uint64)
        rc = self.lib.oracle_run(_ptr(lat, _u8p), lat.shape[0], r, K, seed, k0, n_mcs,
                                 _ptr(counts, _u64p), int(reverse), threads)
        if rc != 0:
            raise ValueError(f"oracle_run rejected L={lat.shape[0]}")
        return counts[:n_mcs]

    def classic_run(self, lat: np.ndarray, r: float, K: float, seed: int, e0: int,
                    n_mcs: int) -> np.ndarray:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        counts = np.zeros(max(n_mcs, 1), dtype=np.uint64)
        rc = self.lib.oracle_classic_run(_ptr(lat, _u8p), lat.shape[0], r, K, seed, e0, n_mcs,
                                         _ptr(counts, _u64p))
        if rc != 0:
            raise ValueError("oracle_classic_run rejected the lattice")
        return counts[:n_mcs]

    # --- the pairwise game (Section VI); pay = (R, S, T, P) ------------------
    @staticmethod
    def _pay(pay) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(pay, dtype=np.float64))
        assert a.shape == (4,)
        return a

    def pair_neighbour_cooperators(self, lat, i: int, j: int) -> int:
        a = self._lat(lat)
        return self.lib.oracle_pair_neighbour_cooperators(_ptr(a, _u8p), a.shape[0], i, j)

    def pair_payoff_games(self, lat, i: int, j: int, pay) -> float:
        a, p = self._lat(lat), self._pay(pay)
        return self.lib.oracle_pair_payoff_games(_ptr(a, _u8p), a.shape[0], i, j,
                                                 _ptr(p, ctypes.POINTER(ctypes.c_double)))

    def pair_payoff_total(self, s: int, n: int, pay) -> float:
        p = self._pay(pay)
        return self.lib.oracle_pair_payoff_total(s, n, _ptr(p, ctypes.POINTER(ctypes.c_double)))

    def pair_update_threshold(self, lat, i: int, j: int, d: int, pay, K: float) -> int:
        a, p = self._lat(lat), self._pay(pay)
        return int(self.lib.oracle_pair_update_threshold(_ptr(a, _u8p), a.shape[0], i, j, d,
                                                         _ptr(p, ctypes.POINTER(ctypes.c_double)), K))

    def pair_elementary_update(self, lat: np.ndarray, i: int, j: int, d: int, u: int, pay,
                               K: float) -> int:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        p = self._pay(pay)
        return self.lib.oracle_pair_elementary_update(_ptr(lat, _u8p), lat.shape[0], i, j, d, u,
                                                      _ptr(p, ctypes.POINTER(ctypes.c_double)), K)

    def pair_sublattice_step(self, lat: np.ndarray, pay, K: float, seed: int, k: int,
                             reverse: bool = False, threads: int = 1) -> int:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        p = self._pay(pay)
        return int(self.lib.oracle_pair_sublattice_step(_ptr(lat, _u8p), lat.shape[0],
                                                        _ptr(p, ctypes.POINTER(ctypes.c_double)), K,
                                                        seed, k, int(reverse), threads))

    def pair_run(self, lat: np.ndarray, pay, K: float, seed: int, k0: int, n_mcs: int,
                 reverse: bool = False, threads: int = 1) -> np.ndarray:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        p = self._pay(pay)
        counts = np.zeros(max(n_mcs, 1), dtype=np.uint64)
        rc = self.lib.oracle_pair_run(_ptr(lat, _u8p), lat.shape[0],
                                      _ptr(p, ctypes.POINTER(ctypes.c_double)), K, seed, k0, n_mcs,
                                      _ptr(counts, _u64p), int(reverse), threads)
        if rc != 0:
            raise ValueError(f"oracle_pair_run rejected L={lat.shape[0]}")
        return counts[:n_mcs]

    def pair_classic_run(self, lat: np.ndarray, pay, K: float, seed: int, e0: int,
                         n_mcs: int) -> np.ndarray:
        assert lat.dtype == np.uint8 and lat.flags.c_contiguous
        p = self._pay(pay)
        counts = np.zeros(max(n_mcs, 1), dtype=np.uint64)
        rc = self.lib.oracle_pair_classic_run(_ptr(lat, _u8p), lat.shape[0],
                                              _ptr(p, ctypes.POINTER(ctypes.c_double)), K, seed, e0,
                                              n_mcs, _ptr(counts, _u64p))
        if rc != 0:
            raise ValueError("oracle_pair_classic_run rejected the lattice")
        return counts[:n_mcs]

    def errors(self) -> int:
        return self.lib.oracle_error_count()

    def clear_errors(self) -> None:
        self.lib.oracle_clear_errors()

    def max_threads(self) -> int:
        return self.lib.oracle_max_threads()
