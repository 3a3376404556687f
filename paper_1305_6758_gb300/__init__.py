"""GB300 multipath Metropolis simulation of the classical Heisenberg model.

Thin Python binding of the C ABI in ``include/mp.h`` (library ``libmp.so``
built in-tree by ``paper_1305_6758_gb300.build``).  Every step of the method
runs in the library's CUDA kernels; this module only marshals arguments,
hands the library device memory from PyTorch's caching allocator and the
current PyTorch stream, and converts results.  There is no CPU fallback:
importing the binding without the compiled library raises.

Method (Rakic et al., Sec. 2.2): many independent Metropolis paths of one
lattice at one temperature, each thermalised and measured; per-path outputs
averaged over paths into ensemble estimates with standard errors.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmp.so")

SC, CHAIN, ISING = 0, 1, 2  # ISING: periodic L x L square lattice of +-1 spins (Appendix A)
FP32, FP64 = 0, 1
INIT_SPHERE, INIT_ANGLES, INIT_ORDERED = 0, 1, 2
FLAG_GRAPH, FLAG_KEEP_SPINS, FLAG_STREAM, FLAG_AUTOTUNE, FLAG_TWO_START, FLAG_RANDOM_SITE = 1, 2, 4, 8, 16, 32
FLAG_TEST_STALL = 0x100
FLAG_DEVICE_UNITS = 0x200

MP_OK, MP_EINVAL, MP_ENOMEM, MP_ECUDA, MP_ESTATE, MP_ECANCELED, MP_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6

# per-path record fields (include/mp.h, MP_R_*)
REC = dict(
    e=0, e2=1, m=2, m2=3, m4=4, mx=5, my=6, mz=7, mz2=8, amz=9,
    em=10, emz=11, mmz=12, fmx=13, fmy=14, fmz=15, fe=16, acc=17, norm=18,
)
NREC = 20
NEST = 64
R_MAX_PATHS = 16384


class MPError(RuntimeError):
    """A non-zero status from the library, with its error text."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_STATUS = {0: "MP_OK", -1: "MP_EINVAL", -2: "MP_ENOMEM", -3: "MP_ECUDA", -4: "MP_ESTATE",
           -5: "MP_ECANCELED", -6: "MP_ETIMEOUT"}


class MPSystem(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("L", ctypes.c_int32), ("T", ctypes.c_double),
                ("J", ctypes.c_double), ("h", ctypes.c_double), ("n_paths", ctypes.c_int64),
                ("path_begin", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class MPConfig(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("init_mode", ctypes.c_int32),
        ("n_systems", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("systems", ctypes.POINTER(MPSystem)),
        ("n_therm", ctypes.c_int64), ("n_meas", ctypes.c_int64), ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("alloc_fn", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
        ("cta_threads", ctypes.c_int32), ("threads_per_path", ctypes.c_int32),
    ]


EST_FIELDS = [
    "n_paths", "N", "T", "n_meas",
    "e", "e_se", "e2", "e2_se",
    "m", "m_se", "m2", "m2_se", "m4", "m4_se",
    "mx", "mx_se", "my", "my_se", "mz", "mz_se",
    "mz2", "mz2_se", "amz", "amz_se",
    "acc", "acc_se",
    "chi", "chi_se", "cv", "cv_se", "binder", "binder_se",
    "de_dbeta", "de_dbeta_se", "dm_dbeta", "dm_dbeta_se", "dmz_dbeta", "dmz_dbeta_se",
    "de_dh", "de_dh_se", "dm_dh", "dm_dh_se", "dmz_dh", "dmz_dh_se",
    "cv_m",
    "r_e", "r_m", "r_mx", "r_my", "r_mz", "r_amz",
    "attempts", "norm_max",
    "e_a", "e_a_se", "e_b", "e_b_se", "m_a", "m_a_se", "m_b", "m_b_se", "start_z",
    "elapsed_s",
]


class MPEstimates(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in EST_FIELDS] + [("reserved", ctypes.c_double * 1)]


assert ctypes.sizeof(MPEstimates) == NEST * 8

# Every symbol include/mp.h declares.
EXPORTS = [
    "mp_create", "mp_create_ex", "mp_run", "mp_set_seed", "mp_estimates", "mp_paths",
    "mp_device_buffers", "mp_spins", "mp_backward", "mp_timing", "mp_plan", "mp_upload_bytes", "mp_system_plan",
    "mp_run_sweeps", "mp_progress", "mp_checkpoint", "mp_restore", "mp_cancel", "mp_philox",
    "mp_reduce", "mp_destroy", "mp_last_error", "mp_status_string",
]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmp.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    P = ctypes.POINTER
    i64, u64, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    lib.mp_create.argtypes = [ctypes.c_int, dbl, dbl, dbl, i64, i64, i64, u64, P(H)]
    lib.mp_create_ex.argtypes = [P(MPConfig), P(H)]
    lib.mp_run.argtypes = [H]
    lib.mp_set_seed.argtypes = [H, u64]
    lib.mp_estimates.argtypes = [H, ctypes.c_int, P(MPEstimates)]
    lib.mp_paths.argtypes = [H, ctypes.c_int, P(dbl), i64]
    lib.mp_device_buffers.argtypes = [H, P(ctypes.c_void_p), P(ctypes.c_void_p)]
    lib.mp_spins.argtypes = [H, ctypes.c_int, i64, P(dbl), i64]
    lib.mp_backward.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mp_timing.argtypes = [H, P(dbl), P(dbl)]
    lib.mp_plan.argtypes = [H] + [P(ctypes.c_int)] * 4
    lib.mp_upload_bytes.argtypes = [H, P(i64)]
    lib.mp_system_plan.argtypes = [H, ctypes.c_int] + [P(ctypes.c_int)] * 3
    lib.mp_run_sweeps.argtypes = [H, i64]
    lib.mp_progress.argtypes = [H, P(i64)]
    lib.mp_checkpoint.argtypes = [H, ctypes.c_void_p, P(ctypes.c_size_t)]
    lib.mp_restore.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
    lib.mp_cancel.argtypes = [H]
    lib.mp_philox.argtypes = [ctypes.c_void_p, i64, u64, ctypes.c_void_p, ctypes.c_void_p]
    lib.mp_reduce.argtypes = [P(MPSystem), ctypes.c_int, i64, i64, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p]
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_int
    lib.mp_destroy.argtypes = [H]
    lib.mp_destroy.restype = None
    lib.mp_last_error.argtypes = [H]
    lib.mp_last_error.restype = ctypes.c_char_p
    lib.mp_status_string.argtypes = [ctypes.c_int]
    lib.mp_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, handle=None):
    if status != MP_OK:
        msg = _lib.mp_last_error(handle)
        raise MPError(status, msg.decode() if msg else "")


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch

        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, ctx, nbytes):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except RuntimeError:
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ctx, ptr):
        self.live.pop(ptr, None)


@dataclass
class System:
    """One system of a batch: lattice kind, size, temperature, couplings, paths.

    ``path_begin`` is the path id of the first path: a process that runs part
    of one ensemble (paths path_begin .. path_begin + n_paths - 1, same seed)
    draws exactly those paths' random numbers.
    """

    L: int
    T: float
    J: float = 1.0
    h: float = 0.0
    n_paths: int = 1
    lattice: int = SC
    path_begin: int = 0

    @property
    def N(self) -> int:
        if self.lattice == ISING:
            return self.L ** 2
        return self.L ** 3 if self.lattice == SC else self.L


class Simulation:
    """A handle of the library: a batch of systems run together.

    Device memory comes from PyTorch's allocator on ``device`` (default
    ``cuda:0``); all work runs on ``self.stream``, a new ``torch.cuda.Stream``
    unless ``stream`` is given.
    """

    def __init__(self, systems: list[System], n_therm: int, n_meas: int, seed: int = 1,
                 precision: int = FP32, init_mode: int = INIT_SPHERE, graph: bool = True,
                 keep_spins: bool = False, cta_threads: int = 0, threads_per_path: int = 0,
                 device=None, stream=None, flags: int = 0):
        import torch

        lib = load_library()
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda:0")
        self.systems = list(systems)
        self._sys = (MPSystem * len(systems))(
            *[MPSystem(s.lattice, s.L, s.T, s.J, s.h, s.n_paths, s.path_begin) for s in systems])
        self._alloc = _TorchAllocator(self.device)
        # a stream of its own (PyTorch's default stream is the legacy NULL stream)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        cfg = MPConfig()
        cfg.precision = precision
        cfg.init_mode = init_mode
        cfg.n_systems = len(systems)
        cfg.flags = (FLAG_GRAPH if graph else 0) | (FLAG_KEEP_SPINS if keep_spins else 0) | flags
        cfg.systems = self._sys
        cfg.n_therm = n_therm
        cfg.n_meas = n_meas
        cfg.seed = seed
        cfg.stream = self.stream.cuda_stream
        cfg.alloc_fn = self._alloc.alloc_cb
        cfg.free_fn = self._alloc.free_cb
        cfg.cta_threads = cta_threads
        cfg.threads_per_path = threads_per_path
        self.n_therm, self.n_meas, self.precision = n_therm, n_meas, precision
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.mp_create_ex(ctypes.byref(cfg), ctypes.byref(self._h)))

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.mp_destroy(self._h)
            self._h = ctypes.c_void_p()

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

    # -- calls
    def run(self):
        """Queue one full run (all paths, all sweeps, reduction) on the stream."""
        with self.torch.cuda.device(self.device):
            _check(_lib.mp_run(self._h), self._h)
        return self

    def set_seed(self, seed: int):
        _check(_lib.mp_set_seed(self._h, seed), self._h)

    def estimates(self, system: int = 0) -> dict:
        out = MPEstimates()
        _check(_lib.mp_estimates(self._h, system, ctypes.byref(out)), self._h)
        return {f: getattr(out, f) for f in EST_FIELDS}

    def paths(self, system: int = 0) -> np.ndarray:
        """Per-path records of one system, shape (n_paths, NREC)."""
        n = self.systems[system].n_paths
        buf = np.empty((n, NREC))
        _check(_lib.mp_paths(self._h, system, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             buf.size), self._h)
        return buf

    def spins(self, system: int, path: int) -> np.ndarray:
        """Final spins (N, 3) of one path (needs keep_spins=True)."""
        N = self.systems[system].N
        buf = np.empty((N, 3))
        _check(_lib.mp_spins(self._h, system, path,
                             buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), buf.size), self._h)
        return buf

    def device_records(self):
        """The handle's per-path records as a (total_paths, NREC) float64 CUDA tensor view."""
        rec = ctypes.c_void_p()
        _check(_lib.mp_device_buffers(self._h, ctypes.byref(rec), None), self._h)
        total = sum(s.n_paths for s in self.systems)
        return _wrap_device(rec.value, (total, NREC), self.device)

    def backward(self, g_e, g_m):
        """Fluctuation-formula gradients (d/dbeta, d/dh) of g_e.<e> + g_m.<|m|> per system."""
        torch = self.torch
        n = len(self.systems)
        caller = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(caller)  # gradients the caller produced are ready
        with torch.cuda.stream(self.stream):
            ge = torch.as_tensor(g_e, dtype=torch.float64, device=self.device).reshape(n).contiguous()
            gm = torch.as_tensor(g_m, dtype=torch.float64, device=self.device).reshape(n).contiguous()
            gb = torch.empty(n, dtype=torch.float64, device=self.device)
            gh = torch.empty(n, dtype=torch.float64, device=self.device)
            _check(_lib.mp_backward(self._h, ge.data_ptr(), gm.data_ptr(), gb.data_ptr(), gh.data_ptr()),
                   self._h)
        caller.wait_stream(self.stream)  # results are ready on the caller's stream
        for t in (ge, gm, gb, gh):
            t.record_stream(self.stream)
        return gb, gh

    def timing(self) -> tuple[float, float]:
        """(sweep kernel ms, reduction kernel ms) of the last run."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(_lib.mp_timing(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    def plan(self) -> dict:
        v = [ctypes.c_int() for _ in range(4)]
        _check(_lib.mp_plan(self._h, *[ctypes.byref(x) for x in v]), self._h)
        return dict(cta_threads=v[0].value, grid=v[1].value, smem_bytes=v[2].value, n_items=v[3].value)

    def upload_bytes(self) -> int:
        """Bytes of plan tables the handle copied from host to device when it was created."""
        b = ctypes.c_int64()
        _check(_lib.mp_upload_bytes(self._h, ctypes.byref(b)), self._h)
        return b.value

    def run_sweeps(self, n: int):
        """Advance every path by n sweeps of its schedule from its saved state (synchronous)."""
        with self.torch.cuda.device(self.device):
            _check(_lib.mp_run_sweeps(self._h, n), self._h)
        return self

    def progress(self) -> int:
        v = ctypes.c_int64()
        _check(_lib.mp_progress(self._h, ctypes.byref(v)), self._h)
        return v.value

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(_lib.mp_checkpoint(self._h, None, ctypes.byref(n)), self._h)
        buf = ctypes.create_string_buffer(n.value)
        _check(_lib.mp_checkpoint(self._h, buf, ctypes.byref(n)), self._h)
        return buf.raw[: n.value]

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(_lib.mp_restore(self._h, buf, len(blob)), self._h)

    def cancel(self):
        _check(_lib.mp_cancel(self._h), self._h)

    def system_plan(self, system: int) -> dict:
        v = [ctypes.c_int() for _ in range(3)]
        _check(_lib.mp_system_plan(self._h, system, *[ctypes.byref(x) for x in v]), self._h)
        return dict(threads_per_path=v[0].value, paths_per_cta=v[1].value, streamed=v[2].value == 1,
                    cluster_pair=v[2].value == 2, in_place_hbm=v[2].value == 3)


def _wrap_device(ptr: int, shape, device):
    """Zero-copy float64 CUDA tensor over library-owned memory (valid while the handle lives)."""
    import torch

    n = int(np.prod(shape))

    class _Iface:
        __cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": "<f8", "data": (ptr, False), "version": 3,
            "strides": None,
        }

    t = torch.as_tensor(_Iface(), device=device)
    assert t.numel() == n
    return t


def philox(counters: np.ndarray, seed: int, device="cuda:0") -> np.ndarray:
    """Philox4x32-10 on the GPU of uint32 counters shaped (n, 4); returns (n, 4) uint32."""
    import torch

    lib = load_library()
    host = np.ascontiguousarray(np.asarray(counters, dtype=np.uint32).reshape(-1, 4))
    c = torch.from_numpy(host.view(np.int32)).to(device)
    out = torch.empty_like(c)
    st = torch.cuda.current_stream(c.device)
    _check(lib.mp_philox(c.data_ptr(), c.shape[0], seed, out.data_ptr(), st.cuda_stream))
    st.synchronize()
    return out.cpu().numpy().view(np.uint32)


def reduce_records(systems: list[System], n_therm: int, n_meas: int, records, device="cuda:0") -> list[dict]:
    """Estimates of per-path records (a float64 CUDA tensor of n_paths x NREC
    rows, systems one after another) through mp_reduce: for ranks that each
    ran part of one ensemble and gathered their records in path order."""
    import torch

    lib = load_library()
    rec = records.to(device=device, dtype=torch.float64).contiguous()
    n = len(systems)
    if rec.numel() != sum(s.n_paths for s in systems) * NREC:
        raise ValueError("records do not match the systems' path counts")
    arr = (MPSystem * n)(*[MPSystem(s.lattice, s.L, s.T, s.J, s.h, s.n_paths, s.path_begin) for s in systems])
    out = torch.empty(n * NEST, dtype=torch.float64, device=rec.device)
    st = torch.cuda.current_stream(rec.device)
    _check(lib.mp_reduce(arr, n, n_therm, n_meas, rec.data_ptr(), out.data_ptr(), st.cuda_stream))
    est = out.cpu().numpy().reshape(n, NEST)
    return [dict(zip(EST_FIELDS, row)) for row in est]


def simulate(L: int, T: float, J: float = 1.0, h: float = 0.0, n_paths: int = 256,
             n_therm: int = 1000, n_meas: int = 1000, seed: int = 1, **kw) -> dict:
    """One system end to end (create, run, estimates, destroy)."""
    with Simulation([System(L, T, J, h, n_paths)], n_therm, n_meas, seed, **kw) as sim:
        sim.run()
        return sim.estimates(0)
