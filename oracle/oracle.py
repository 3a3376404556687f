"""ctypes front end of the C oracle (test infrastructure, never on the product path).

The C side (``mp_oracle.c``) states the method step by step in FP64: the
Heisenberg energy of Eq. (1) with unit spins of Eq. (2), Metropolis single
spin-flip updates, lattice sweeps, and per-path outputs of Sec. 2.2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mp_oracle.c")
lib_path = os.path.join(HERE, "libmp_oracle.so")

SC, CHAIN, ISING = 0, 1, 2  # ISING: periodic L x L square lattice of +-1 spins (Appendix A)
INIT_SPHERE, INIT_ANGLES, INIT_ORDERED = 0, 1, 2
ORDER_CHECKER, ORDER_RANDOM = 0, 1
TWO_START = 0x100  # or-ed into init_mode by run(two_start=True)

# per-path record fields, in the order mp_oracle.c writes them
REC = dict(
    e=0, e2=1, m=2, m2=3, m4=4, mx=5, my=6, mz=7, mz2=8, amz=9,
    em=10, emz=11, mmz=12, fmx=13, fmy=14, fmz=15, fe=16, acc=17, norm=18,
)
NREC = 20


class _Sys(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("L", ctypes.c_int32),
        ("T", ctypes.c_double),
        ("J", ctypes.c_double),
        ("h", ctypes.c_double),
        ("n_paths", ctypes.c_int64),
        ("path_begin", ctypes.c_int64),
        ("path_count", ctypes.c_int64),
    ]


@dataclass
class System:
    """One (lattice, L, T, J, h) system with n_paths independent paths.

    ``path_begin``/``path_count`` select which path ids the oracle runs
    (default: all of them).  Path ids key the random streams, so a subset run
    reproduces exactly those paths of a full run.
    """

    L: int
    T: float
    J: float = 1.0
    h: float = 0.0
    n_paths: int = 1
    lattice: int = SC
    path_begin: int = 0
    path_count: int | None = None

    @property
    def N(self) -> int:
        if self.lattice == ISING:
            return self.L ** 2
        return self.L ** 3 if self.lattice == SC else self.L

    def count(self) -> int:
        return self.n_paths - self.path_begin if self.path_count is None else self.path_count


def build(force: bool = False) -> str:
    """Compile mp_oracle.c into libmp_oracle.so (FP contraction off)."""
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(SRC):
        tmp = lib_path + ".tmp"
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-pthread", "-o", tmp, SRC, "-lm",
        ])
        os.replace(tmp, lib_path)
    return lib_path


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(lib_path)
        u32, i64, dbl = ctypes.c_uint32, ctypes.c_int64, ctypes.c_double
        lib.oracle_philox.argtypes = [u32] * 6 + [ctypes.POINTER(u32)]
        lib.oracle_philox.restype = None
        lib.oracle_run.argtypes = [ctypes.POINTER(_Sys), ctypes.c_int, i64, i64, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_energy.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.POINTER(dbl)]
        lib.oracle_energy.restype = dbl
        lib.oracle_delta_e.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.POINTER(dbl),
                                       i64, ctypes.POINTER(dbl)]
        lib.oracle_delta_e.restype = dbl
        lib.oracle_trial.argtypes = [u32, u32, u32, u32, ctypes.c_uint64, ctypes.POINTER(dbl)]
        lib.oracle_trial.restype = None
        lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int, u32, u32, ctypes.c_uint64,
                                    ctypes.c_int, ctypes.POINTER(dbl)]
        lib.oracle_init.restype = ctypes.c_int
        lib.oracle_nrec.restype = ctypes.c_int
        assert lib.oracle_nrec() == NREC
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox(c0: int, c1: int, c2: int, c3: int, k0: int, k1: int) -> tuple[int, int, int, int]:
    """Philox4x32-10 of counter (c0..c3) under key (k0, k1)."""
    out = (ctypes.c_uint32 * 4)()
    _load().oracle_philox(c0, c1, c2, c3, k0, k1, out)
    return tuple(out)


def trial(site: int, sweep: int, path: int, sys_index: int, seed: int) -> np.ndarray:
    """The trial direction drawn for one update attempt."""
    out = np.zeros(3)
    _load().oracle_trial(site, sweep, path, sys_index, seed, _dptr(out))
    return out


def init(lattice: int, L: int, path: int, sys_index: int, seed: int,
         init_mode: int = INIT_SPHERE) -> np.ndarray:
    """Initial spins (N, 3) of one path."""
    N = L ** 3 if lattice == SC else L
    out = np.zeros((N, 3))
    if _load().oracle_init(lattice, L, path, sys_index, seed, init_mode, _dptr(out)) != 0:
        raise ValueError("oracle_init rejected its arguments")
    return out


def energy(lattice: int, L: int, J: float, h: float, spins: np.ndarray) -> float:
    """Total energy (Eq. 1 plus Zeeman term) of a spin array shaped (N, 3)."""
    s = np.ascontiguousarray(spins, dtype=np.float64)
    return _load().oracle_energy(lattice, L, J, h, _dptr(s))


def delta_e(lattice: int, L: int, J: float, h: float, spins: np.ndarray, i: int,
            t: np.ndarray) -> float:
    """Local-field energy change of replacing spin i by t."""
    s = np.ascontiguousarray(spins, dtype=np.float64)
    tt = np.ascontiguousarray(t, dtype=np.float64)
    return _load().oracle_delta_e(lattice, L, J, h, _dptr(s), i, _dptr(tt))


def run(systems: list[System], n_therm: int, n_meas: int, seed: int = 1,
        init_mode: int = INIT_SPHERE, order_mode: int = ORDER_CHECKER,
        threads: int | None = None, want_spins: bool = False, two_start: bool = False):
    """Run the requested paths of every system.

    With ``two_start`` (Sec. 4's convergence check) the first ceil(P/2) paths
    of each system start from ``init_mode`` and the rest from the ordered state.

    Returns a list (one entry per system) of per-path records shaped
    (path_count, NREC); with ``want_spins`` also the final spins of each path,
    shaped (path_count, N, 3).
    """
    lib = _load()
    arr = (_Sys * len(systems))()
    total, spin_total = 0, 0
    for k, s in enumerate(systems):
        c = s.count()
        arr[k] = _Sys(s.lattice, s.L, s.T, s.J, s.h, s.n_paths, s.path_begin, c)
        total += c
        spin_total += c * s.N * 3
    rec = np.zeros((max(total, 1), NREC))
    spins = np.zeros(max(spin_total, 1)) if want_spins else None
    if threads is None:
        threads = os.cpu_count() or 1
    mode = init_mode | (TWO_START if two_start else 0)
    rc = lib.oracle_run(arr, len(systems), n_therm, n_meas, seed, mode, order_mode,
                        threads, _dptr(rec), _dptr(spins) if want_spins else None)
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    out_rec, out_spins = [], []
    r0, s0 = 0, 0
    for s in systems:
        c = s.count()
        out_rec.append(rec[r0:r0 + c].copy())
        if want_spins:
            n = c * s.N * 3
            out_spins.append(spins[s0:s0 + n].reshape(c, s.N, 3).copy())
            s0 += n
        r0 += c
    return (out_rec, out_spins) if want_spins else out_rec
