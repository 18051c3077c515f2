"""GB300 local search for Ising spin glasses (García & Markov, arXiv:0912.3912).

A thin ctypes binding over the C ABI declared in include/ising.h.  It only
marshals arguments: every step of the search runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  Importing works without a GPU;
any call that needs the library raises if libising_gb300.so is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libising_gb300.so")

I8, F32, F64 = 0, 1, 2
_DT = {"i8": (I8, np.int8), "f32": (F32, np.float32), "f64": (F64, np.float64)}
SCHED_COLOUR, SCHED_SEQUENTIAL = 0, 1
KERNEL_AUTO, KERNEL_TILE, KERNEL_MSC, KERNEL_SWEEP, KERNEL_DENSE_TC, KERNEL_PLAIN = range(6)
DENSE_OWN, DENSE_LIBRARY = 0, 1
KERNEL_NAMES = {KERNEL_AUTO: "auto", KERNEL_TILE: "tile", KERNEL_MSC: "msc", KERNEL_SWEEP: "sweep",
                KERNEL_DENSE_TC: "dense_tc", KERNEL_PLAIN: "plain"}

STATUS = {0: "ok", 1: "invalid argument", 2: "asymmetric", 3: "self loop", 4: "bad hyper-edge",
          5: "bad colouring", 6: "unsupported", 7: "out of memory", 8: "CUDA error", 9: "timeout",
          10: "device check failed"}


class IsingError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class _Desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("J", C.c_void_p),
                ("J_dense", C.c_void_p), ("h", C.c_void_p), ("n_hyper", C.c_int32),
                ("hyper_ptr", C.c_void_p), ("hyper_members", C.c_void_p), ("hyper_J", C.c_void_p),
                ("colour", C.c_void_p), ("dtype", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("max_sweeps", C.c_int32), ("restarts", C.c_int32), ("sweep_budget", C.c_int32),
                ("refresh_every", C.c_int32), ("schedule", C.c_int32), ("kernel", C.c_int32),
                ("dense_variant", C.c_int32), ("dense_tensor_sweeps", C.c_int32), ("cluster_ctas", C.c_int32)]


class _FmParams(C.Structure):
    _fields_ = [("restarts", C.c_int32), ("max_passes", C.c_int32), ("starts", C.c_int32),
                ("reg_kernel", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("flip_evals", C.c_uint64), ("flips", C.c_uint64), ("minima", C.c_uint64),
                ("descents", C.c_uint64), ("sweeps", C.c_uint64), ("launches", C.c_uint64),
                ("evaluated", C.c_uint64)]


class _KTime(C.Structure):
    _fields_ = [("name", C.c_char_p), ("ms", C.c_double), ("launches", C.c_int32)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libising_gb300.so; raise if it was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_0912_3912_gb300.build.build() "
                                   "(or __graft_entry__.build()) first")
            L = C.CDLL(LIB_PATH)
            vp, i32 = C.c_void_p, C.c_int32
            L.ising_create.argtypes = [vp, i32, vp]
            L.ising_create.restype = i32
            L.ising_energy.argtypes = [vp, vp, i32, vp, vp, vp]
            L.ising_energy.restype = i32
            L.ising_local_search.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
            L.ising_local_search.restype = i32
            L.ising_plan_kernel.argtypes = [vp, i32, vp]
            L.ising_plan_kernel.restype = i32
            L.ising_autotune.argtypes = [vp, i32, vp, vp, vp]
            L.ising_autotune.restype = i32
            L.ising_destroy.argtypes = [vp]
            L.ising_destroy.restype = i32
            L.ising_energy_noalloc.argtypes = [i32, vp, vp, vp, vp, i32, vp, i32, vp, vp]
            L.ising_energy_noalloc.restype = i32
            L.ising_fm_search.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp]
            L.ising_fm_search.restype = i32
            L.ising_set_timing.argtypes = [vp, i32]
            L.ising_set_timing.restype = i32
            L.ising_kernel_times.argtypes = [vp, vp, i32]
            L.ising_kernel_times.restype = i32
            L.ising_logic_peak.argtypes = [vp]
            L.ising_logic_peak.restype = i32
            L.ising_logic_bits_rate.argtypes = [i32, vp]
            L.ising_logic_bits_rate.restype = i32
            L.ising_status_string.argtypes = [i32]
            L.ising_status_string.restype = C.c_char_p
            _lib = L
    return _lib


EXPORTED = ("ising_create", "ising_energy", "ising_local_search", "ising_plan_kernel",
            "ising_autotune", "ising_destroy", "ising_status_string", "ising_energy_noalloc",
            "ising_set_timing", "ising_kernel_times", "ising_fm_search", "ising_logic_peak",
            "ising_logic_bits_rate")


def _check(code: int, where: str):
    if code != 0:
        raise IsingError(code, where)


def _arr(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class SearchResult:
    spins: "object"        # torch int8 [instances * replicas, n] flattened per instance
    energy: "object"       # torch float64 [instances, replicas]
    energy_i32: "object"   # torch int32 or None
    minima: "object"       # torch int32 [instances, replicas]
    stats: Optional[dict]


class Handle:
    """Owns an ising_handle: instances uploaded once, searched many times."""

    def __init__(self, instances: Sequence, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        insts = list(instances)
        if not insts:
            raise ValueError("no instances")
        dts = {i.dtype for i in insts}
        if len(dts) != 1:
            raise ValueError("all instances of a handle share one dtype")
        self.dtype = dts.pop()
        self.ns = [int(i.n) for i in insts]
        self.n_inst = len(insts)
        keep = []
        descs = (_Desc * len(insts))()
        code, jdt = _DT[self.dtype]
        for k, inst in enumerate(insts):
            arrs = dict(
                row_ptr=_arr(inst.row_ptr, np.int64), col=_arr(inst.col, np.int32), J=_arr(inst.J, jdt),
                J_dense=_arr(getattr(inst, "J_dense", None), np.float32), h=_arr(inst.h, jdt),
                hyper_ptr=_arr(inst.hyper_ptr, np.int64), hyper_members=_arr(inst.hyper_members, np.int32),
                hyper_J=_arr(inst.hyper_J, jdt), colour=_arr(inst.colour, np.int32))
            keep.append(arrs)
            nh = 0 if arrs["hyper_ptr"] is None else len(arrs["hyper_ptr"]) - 1
            descs[k] = _Desc(int(inst.n), _ptr(arrs["row_ptr"]), _ptr(arrs["col"]), _ptr(arrs["J"]),
                             _ptr(arrs["J_dense"]), _ptr(arrs["h"]), nh, _ptr(arrs["hyper_ptr"]),
                             _ptr(arrs["hyper_members"]), _ptr(arrs["hyper_J"]), _ptr(arrs["colour"]),
                             code)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().ising_create(C.cast(descs, C.c_void_p), len(insts), C.byref(h)), "ising_create")
        self._h = h

    # ------------------------------------------------------------------ helpers
    def _stream(self, stream):
        s = stream if stream is not None else self._torch.cuda.current_stream(self.device)
        return C.c_void_p(s.cuda_stream)

    @staticmethod
    def params(max_sweeps=1000, restarts=1, sweep_budget=0, refresh_every=16,
               schedule=SCHED_COLOUR, kernel=KERNEL_AUTO, dense_variant=DENSE_OWN, dense_tensor_sweeps=0,
               cluster_ctas=0):
        return _Params(max_sweeps, restarts, sweep_budget, refresh_every, schedule, kernel, dense_variant,
                       dense_tensor_sweeps, cluster_ctas)

    @property
    def total_spins(self):
        return sum(self.ns)

    # ------------------------------------------------------------------ API
    def energy(self, spins, replicas: int, stream=None, want_i32=False):
        """Energies of device int8 spins [instance][replica][spin] -> float64 [instances, replicas]."""
        torch = self._torch
        assert spins.dtype == torch.int8 and spins.is_cuda and spins.is_contiguous()
        assert spins.numel() == replicas * self.total_spins
        E = torch.empty((self.n_inst, replicas), dtype=torch.float64, device=self.device)
        E32 = torch.empty((self.n_inst, replicas), dtype=torch.int32, device=self.device) if want_i32 else None
        _check(lib().ising_energy(self._h, C.c_void_p(spins.data_ptr()), replicas, C.c_void_p(E.data_ptr()),
                                  None if E32 is None else C.c_void_p(E32.data_ptr()), self._stream(stream)),
               "ising_energy")
        return (E, E32) if want_i32 else E

    def local_search(self, seeds, replicas: int, *, max_sweeps=1000, restarts=1, sweep_budget=0,
                     refresh_every=16, schedule=SCHED_COLOUR, kernel=KERNEL_AUTO, dense_variant=DENSE_OWN,
                     dense_tensor_sweeps=0, cluster_ctas=0, stream=None, stats=True, want_i32=False,
                     out=None) -> SearchResult:
        torch = self._torch
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(self.n_inst))
        p = self.params(max_sweeps, restarts, sweep_budget, refresh_every, schedule, kernel, dense_variant,
                        dense_tensor_sweeps, cluster_ctas)
        if out is None:
            spins = torch.empty(replicas * self.total_spins, dtype=torch.int8, device=self.device)
            E = torch.empty((self.n_inst, replicas), dtype=torch.float64, device=self.device)
            E32 = (torch.empty((self.n_inst, replicas), dtype=torch.int32, device=self.device)
                   if want_i32 else None)
            minima = torch.empty((self.n_inst, replicas), dtype=torch.int32, device=self.device)
        else:
            spins, E, E32, minima = out
        st = _Stats()
        _check(lib().ising_local_search(
            self._h, C.c_void_p(seeds.ctypes.data), replicas, C.byref(p), C.c_void_p(spins.data_ptr()),
            C.c_void_p(E.data_ptr()), None if E32 is None else C.c_void_p(E32.data_ptr()),
            None if minima is None else C.c_void_p(minima.data_ptr()),
            C.byref(st) if stats else None, self._stream(stream)), "ising_local_search")
        sd = None
        if stats:
            sd = {k: int(getattr(st, k)) for k, _ in _Stats._fields_}
        return SearchResult(spins, E, E32, minima, sd)

    def fm_search(self, seeds, replicas: int, *, restarts=1, max_passes=0, starts=0, reg_kernel=0, stream=None,
                  stats=True):
        """The paper's pass-based search with hill climbing (ising_fm_search).
        Returns (spins [total], energy [instances, replicas], passes, stats)."""
        torch = self._torch
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(self.n_inst))
        spins = torch.empty(replicas * self.total_spins, dtype=torch.int8, device=self.device)
        E = torch.empty((self.n_inst, replicas), dtype=torch.float64, device=self.device)
        passes = torch.empty((self.n_inst, replicas), dtype=torch.int32, device=self.device)
        st = _Stats()
        fp = _FmParams(restarts, max_passes, starts, reg_kernel)
        _check(lib().ising_fm_search(
            self._h, C.c_void_p(seeds.ctypes.data), replicas, C.byref(fp), C.c_void_p(spins.data_ptr()),
            C.c_void_p(E.data_ptr()), C.c_void_p(passes.data_ptr()), C.byref(st) if stats else None,
            self._stream(stream)), "ising_fm_search")
        sd = {k: int(getattr(st, k)) for k, _ in _Stats._fields_} if stats else None
        return spins, E, passes, sd

    def plan_kernel(self, replicas: int, **kw) -> int:
        p = self.params(**kw)
        k = lib().ising_plan_kernel(self._h, replicas, C.byref(p))
        if k < 0:
            raise IsingError(-k, "ising_plan_kernel")
        return k

    def autotune(self, replicas: int, stream=None, **kw) -> int:
        p = self.params(**kw)
        ch = C.c_int32(0)
        _check(lib().ising_autotune(self._h, replicas, C.byref(p), C.byref(ch), self._stream(stream)),
               "ising_autotune")
        return ch.value

    def set_timing(self, enable: bool) -> None:
        """Open (and clear) or close the device-timing window (ising_set_timing)."""
        _check(lib().ising_set_timing(self._h, 1 if enable else 0), "ising_set_timing")

    def kernel_times(self) -> dict:
        """{kernel name: (total ms, launches)} over the timing window."""
        buf = (_KTime * 16)()
        k = lib().ising_kernel_times(self._h, buf, 16)
        if k < 0:
            raise IsingError(-k, "ising_kernel_times")
        return {buf[i].name.decode(): (buf[i].ms, int(buf[i].launches)) for i in range(min(k, 16))}

    def spins_of(self, result_spins, b: int, replicas: int):
        """View of instance b's block as [replicas, n_b]."""
        off = replicas * sum(self.ns[:b])
        return result_spins[off: off + replicas * self.ns[b]].view(replicas, self.ns[b])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ising_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def energy_noalloc(row_ptr, col, J, h, spins, replicas: int, energy, stream=None) -> int:
    """ising_energy_noalloc on caller-owned device tensors (argument marshalling only).

    row_ptr int64 [n+1], col int32, J int8/float32, h (same dtype) or None,
    spins int8 [replicas, n], energy float64 [replicas] (written), all on one
    CUDA device, which is made current for the call.  Returns the status code
    (0 = ok).
    """
    import torch
    dev = spins.device
    for t in (row_ptr, col, J, h, energy):
        if t is not None and t.device != dev:
            raise ValueError(f"energy_noalloc: every tensor must be on {dev}, got one on {t.device}")
    n = row_ptr.numel() - 1
    dt = I8 if J.dtype == torch.int8 else F32
    with torch.cuda.device(dev):
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        return lib().ising_energy_noalloc(
            n, C.c_void_p(row_ptr.data_ptr()), C.c_void_p(col.data_ptr()), C.c_void_p(J.data_ptr()),
            None if h is None else C.c_void_p(h.data_ptr()), dt, C.c_void_p(spins.data_ptr()), replicas,
            C.c_void_p(energy.data_ptr()), C.c_void_p(s.cuda_stream))


def logic_peak() -> float:
    """Measured issue rate of 32-bit logic ops on the current CUDA device, in
    lane-ops/s (ising_logic_peak): the roofline of the multi-spin-coded kernels."""
    v = C.c_double(0.0)
    _check(lib().ising_logic_peak(C.byref(v)), "ising_logic_peak")
    return float(v.value)


def logic_bits_rate(word_bits: int) -> float:
    """Replica-bit logic operations per second on 32- or 64-bit words on the
    current CUDA device (ising_logic_bits_rate)."""
    v = C.c_double(0.0)
    _check(lib().ising_logic_bits_rate(int(word_bits), C.byref(v)), "ising_logic_bits_rate")
    return float(v.value)


def status_string(code: int) -> str:
    return lib().ising_status_string(code).decode()


def create_raw(descs_ptr, n: int):
    """ising_create on a prepared descriptor array (for tests of the argument checks)."""
    h = C.c_void_p()
    code = lib().ising_create(descs_ptr, n, C.byref(h))
    return code, h
