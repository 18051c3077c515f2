"""ctypes wrapper of the plain C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg.  It does not import the GPU package and the GPU
package does not import it.  Instances are accepted by duck typing (any object
with the attributes of ``workloads.Instance``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_INT, MODE_F64, MODE_F32 = 0, 1, 2
SCHED_COLOUR, SCHED_SEQUENTIAL = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so next to it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Inst(C.Structure):
    _fields_ = [("n", C.c_int32),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("J", C.c_void_p),
                ("J_dense", C.c_void_p), ("h", C.c_void_p),
                ("n_hyper", C.c_int32), ("hyper_ptr", C.c_void_p),
                ("hyper_members", C.c_void_p), ("hyper_J", C.c_void_p),
                ("colour", C.c_void_p), ("is_int", C.c_int32), ("is_f64", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("max_sweeps", C.c_int32), ("restarts", C.c_int32), ("sweep_budget", C.c_int32),
                ("refresh_every", C.c_int32), ("schedule", C.c_int32), ("mode", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.orc_energy.restype = C.c_double
            L.orc_energy_int.restype = C.c_int64
            L.orc_lower_bound.restype = C.c_double
            L.orc_fm_search.restype = C.c_double
            L.orc_bruteforce.restype = C.c_double
            L.orc_transfer_matrix.restype = C.c_double
            L.orc_greedy_colouring.restype = C.c_int32
            L.orc_colouring_valid.restype = C.c_int32
            L.orc_descent.restype = C.c_int32
            L.orc_bnb.restype = C.c_int32
            vp, i32, i64, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_random_start.argtypes = [i32, u64, u32, u32, u32, vp]
            L.orc_energy.argtypes = [vp, vp]
            L.orc_energy_int.argtypes = [vp, vp]
            L.orc_local_fields.argtypes = [vp, vp, vp]
            L.orc_lower_bound.argtypes = [vp]
            L.orc_greedy_colouring.argtypes = [vp, vp]
            L.orc_colouring_valid.argtypes = [vp, vp]
            L.orc_descent.argtypes = [vp, u64, u32, i32, vp, vp, vp, vp, vp]
            L.orc_descent_from.restype = C.c_int32
            L.orc_descent_from.argtypes = [vp, u64, u32, i32, i32, vp, vp, vp, vp, vp]
            L.orc_fm_search.argtypes = [vp, vp, vp]
            L.orc_bruteforce.argtypes = [vp, vp, vp]
            L.orc_bnb.argtypes = [vp, i64, vp, vp, vp]
            L.orc_transfer_matrix.argtypes = [vp, i32, i32, i32, i32, vp]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleInstance:
    """Keeps FP64 copies of an instance alive and exposes the C struct."""

    def __init__(self, inst, colour=None):
        self.n = int(inst.n)
        self.is_int = inst.dtype == "i8"
        self.is_f64 = inst.dtype == "f64"
        f64 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        self.row_ptr = None if inst.row_ptr is None else np.ascontiguousarray(inst.row_ptr, np.int64)
        self.col = None if inst.col is None else np.ascontiguousarray(inst.col, np.int32)
        self.J = f64(inst.J)
        self.J_dense = f64(inst.J_dense)
        self.h = f64(inst.h)
        self.hyper_ptr = None if inst.hyper_ptr is None else np.ascontiguousarray(inst.hyper_ptr, np.int64)
        self.hyper_members = None if inst.hyper_members is None else np.ascontiguousarray(
            inst.hyper_members, np.int32)
        self.hyper_J = f64(inst.hyper_J)
        col_src = colour if colour is not None else inst.colour
        self.colour = None if col_src is None else np.ascontiguousarray(col_src, np.int32)
        self.c = _Inst(self.n, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.J), _ptr(self.J_dense),
                       _ptr(self.h), 0 if self.hyper_ptr is None else len(self.hyper_ptr) - 1,
                       _ptr(self.hyper_ptr), _ptr(self.hyper_members), _ptr(self.hyper_J),
                       _ptr(self.colour), 1 if self.is_int else 0, 1 if self.is_f64 else 0)

    @property
    def ref(self):
        return C.byref(self.c)


def _oi(inst):
    return inst if isinstance(inst, OracleInstance) else OracleInstance(inst)


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return list(out)


def random_start(n, seed, b, r, k):
    s = np.empty(n, dtype=np.int8)
    lib().orc_random_start(C.c_int32(n), C.c_uint64(seed), C.c_uint32(b), C.c_uint32(r),
                           C.c_uint32(k), s.ctypes.data)
    return s


def energy(inst, s):
    oi = _oi(inst)
    s = np.ascontiguousarray(s, dtype=np.int8)
    if oi.is_int:
        return float(lib().orc_energy_int(oi.ref, s.ctypes.data))
    return float(lib().orc_energy(oi.ref, s.ctypes.data))


def energies(inst, spins):
    """Energy of each row of a [replicas, n] int8 array."""
    oi = _oi(inst)
    spins = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1, oi.n)
    return np.array([energy(oi, row) for row in spins])


def local_fields(inst, s):
    oi = _oi(inst)
    s = np.ascontiguousarray(s, dtype=np.int8)
    f = np.empty(oi.n, dtype=np.float64)
    lib().orc_local_fields(oi.ref, s.ctypes.data, f.ctypes.data)
    return f


def lower_bound(inst):
    return float(lib().orc_lower_bound(_oi(inst).ref))


def greedy_colouring(inst):
    oi = _oi(inst)
    col = np.empty(oi.n, dtype=np.int32)
    nc = lib().orc_greedy_colouring(oi.ref, col.ctypes.data)
    return col, int(nc)


def colouring_valid(inst, colour):
    oi = _oi(inst)
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    return bool(lib().orc_colouring_valid(oi.ref, colour.ctypes.data))


def descent(inst, seed, b, replicas, max_sweeps=1000, restarts=1, sweep_budget=0,
            refresh_every=0, schedule=SCHED_COLOUR, mode=None, colour=None, first_replica=0):
    """Run the oracle's descent with restarts for replicas first_replica ..
    first_replica + replicas - 1; returns (spins [R, n], E [R], minima [R], stats).
    The C call releases the GIL (ctypes), so host threads can run disjoint
    replica ranges at once; the oracle keeps no global state."""
    oi = inst if isinstance(inst, OracleInstance) else OracleInstance(inst, colour=colour)
    if mode is None:
        mode = MODE_INT if oi.is_int else (MODE_F64 if oi.is_f64 else MODE_F32)
    p = _Params(max_sweeps, restarts, sweep_budget, refresh_every, schedule, mode)
    spins = np.empty((replicas, oi.n), dtype=np.int8)
    E = np.empty(replicas, dtype=np.float64)
    minima = np.empty(replicas, dtype=np.int32)
    stats = np.zeros(5, dtype=np.uint64)
    rc = lib().orc_descent_from(oi.ref, C.c_uint64(seed), C.c_uint32(b), C.c_int32(first_replica),
                                C.c_int32(replicas), C.byref(p), spins.ctypes.data, E.ctypes.data,
                                minima.ctypes.data, stats.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc_descent failed with {rc}")
    keys = ("flip_evals", "flips", "minima", "descents", "sweeps")
    return spins, E, minima, dict(zip(keys, (int(x) for x in stats)))


def fm_search(inst, s0):
    oi = _oi(inst)
    s = np.array(s0, dtype=np.int8, copy=True)
    passes = C.c_int32(0)
    E = lib().orc_fm_search(oi.ref, s.ctypes.data, C.byref(passes))
    return s, float(E), int(passes.value)


def bruteforce(inst):
    oi = _oi(inst)
    arg = np.empty(oi.n, dtype=np.int8)
    ng = C.c_int64(0)
    E = lib().orc_bruteforce(oi.ref, arg.ctypes.data, C.byref(ng))
    return float(E), arg, int(ng.value)


def bnb(inst, node_limit=50_000_000):
    oi = _oi(inst)
    arg = np.empty(oi.n, dtype=np.int8)
    E = C.c_double(0)
    nodes = C.c_int64(0)
    done = lib().orc_bnb(oi.ref, C.c_int64(node_limit), C.byref(E), arg.ctypes.data, C.byref(nodes))
    return bool(done), float(E.value), arg, int(nodes.value)


def transfer_matrix(inst, rows, cols, periodic_rows, periodic_cols):
    oi = _oi(inst)
    ok = C.c_int32(0)
    E = lib().orc_transfer_matrix(oi.ref, rows, cols, int(periodic_rows), int(periodic_cols),
                                  C.byref(ok))
    if not ok.value:
        raise ValueError("instance is not a grid this routine accepts")
    return float(E)


def window_instance(inst, s, members):
    """The window check of Sec. V (branch and bound on a few dozen adjacent spins
    with the rest of a local-search result held fixed), as an instance over the
    spins `members` alone.  With every other spin fixed at `s`, Eq. 1 / Eq. 6
    split into terms inside the window, terms with one window spin (added to
    that spin's field: h_i plus J_ij s_j over fixed neighbours j, plus J_e times
    the fixed members' product for a hyper-edge with one window member), terms
    of hyper-edges with two or more window members (kept, coupling J_e times
    the fixed members' product) and a constant.  Returns (sub-instance, const)
    with E(state) = E_sub(state restricted to the window) + const.  Couplings
    and fields must be integers (int8 instances) so that the folded fields are
    exact."""
    import workloads as W  # the Instance container only
    if inst.dtype != "i8":
        raise ValueError("window_instance folds fields exactly for int8 instances only")
    members = [int(m) for m in members]
    pos = {m: k for k, m in enumerate(members)}
    s = np.asarray(s, dtype=np.int64)
    nw = len(members)
    h = np.zeros(nw, dtype=np.int64)
    if inst.h is not None:
        for m, k in pos.items():
            h[k] = int(inst.h[m])
    rows = [[] for _ in range(nw)]
    for m, k in pos.items():
        for q in range(int(inst.row_ptr[m]), int(inst.row_ptr[m + 1])):
            j = int(inst.col[q])
            Jv = int(inst.J[q])
            if j in pos:
                rows[k].append((pos[j], Jv))
            else:
                h[k] += Jv * s[j]
    hp, hm, hJ = [0], [], []
    if inst.hyper_ptr is not None:
        for e in range(len(inst.hyper_ptr) - 1):
            mem = [int(x) for x in inst.hyper_members[inst.hyper_ptr[e]:inst.hyper_ptr[e + 1]]]
            inside = [pos[x] for x in mem if x in pos]
            prod = 1
            for x in mem:
                if x not in pos:
                    prod *= int(s[x])
            Je = int(inst.hyper_J[e]) * prod
            if len(inside) == 1:
                h[inside[0]] += Je
            elif len(inside) >= 2:
                hm.extend(inside)
                hp.append(len(hm))
                hJ.append(Je)
    if np.abs(h).max(initial=0) > 127:
        raise ValueError("folded field outside int8")
    row_ptr = np.zeros(nw + 1, dtype=np.int64)
    col, J = [], []
    for k in range(nw):
        for j, Jv in sorted(rows[k]):
            col.append(j)
            J.append(Jv)
        row_ptr[k + 1] = len(col)
    sub = W.Instance(n=nw, row_ptr=row_ptr, col=np.array(col, dtype=np.int32), J=np.array(J, dtype=np.int8),
                     h=h.astype(np.int8),
                     hyper_ptr=np.array(hp, dtype=np.int64) if hJ else None,
                     hyper_members=np.array(hm, dtype=np.int32) if hJ else None,
                     hyper_J=np.array(hJ, dtype=np.int8) if hJ else None, dtype="i8")
    const = energy(inst, s.astype(np.int8)) - energy(sub, s[members].astype(np.int8))
    return sub, const
