"""Host-side checks of the C-ABI library that need no GPU.

The library must build for sm_103a, load, and export every function
include/ising.h declares; ising_create must reject malformed instances with
the documented status codes before it touches the device.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def isg():
    from paper_0912_3912_gb300 import build as B
    B.build()
    import paper_0912_3912_gb300 as m
    m.lib()
    return m


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "ising.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ising_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function(isg):
    names = _declared_functions()
    assert "ising_local_search" in names and len(names) >= 7
    L = C.CDLL(isg.LIB_PATH)
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(names) == set(isg.EXPORTED)


def test_product_path_fails_loudly_without_the_library():
    """No fallback: with the shared library absent, creating a handle raises."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_0912_3912_gb300 as m, workloads as W\n"
        "m.LIB_PATH = '/nonexistent/libising_gb300.so'\n"
        "m._lib = None\n"
        "try:\n"
        "    m.lib()\n"
        "except RuntimeError as e:\n"
        "    print('raised:', 'missing' in str(e))\n"
        "try:\n"
        "    m.Handle([W.lattice((4, 4), periodic=True, couplings='pm1', seed=1)])\n"
        "    print('handle created')\n"
        "except RuntimeError:\n"
        "    pass\n"
    ) % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised: True" in r.stdout and "handle created" not in r.stdout, (r.stdout, r.stderr)


def test_timing_entry_points_reject_a_null_handle(isg):
    L = isg.lib()
    assert L.ising_set_timing(None, 1) == 1          # ISING_ERR_INVALID_ARG
    assert L.ising_kernel_times(None, None, 0) == -1


def test_status_strings(isg):
    assert isg.status_string(0) == "ok"
    assert "symmetric" in isg.status_string(2)


def _desc(isg, inst, **over):
    code, jdt = isg._DT[inst.dtype]
    arrs = dict(row_ptr=np.ascontiguousarray(inst.row_ptr, np.int64),
                col=np.ascontiguousarray(inst.col, np.int32),
                J=np.ascontiguousarray(inst.J, jdt),
                h=None if inst.h is None else np.ascontiguousarray(inst.h, jdt),
                hyper_ptr=None if inst.hyper_ptr is None else np.ascontiguousarray(inst.hyper_ptr, np.int64),
                hyper_members=None if inst.hyper_members is None else np.ascontiguousarray(inst.hyper_members, np.int32),
                hyper_J=None if inst.hyper_J is None else np.ascontiguousarray(inst.hyper_J, jdt),
                colour=None if inst.colour is None else np.ascontiguousarray(inst.colour, np.int32))
    arrs.update(over)
    p = lambda a: None if a is None else a.ctypes.data
    nh = 0 if arrs["hyper_ptr"] is None else len(arrs["hyper_ptr"]) - 1
    d = isg._Desc(inst.n, p(arrs["row_ptr"]), p(arrs["col"]), p(arrs["J"]), None, p(arrs["h"]), nh,
                  p(arrs["hyper_ptr"]), p(arrs["hyper_members"]), p(arrs["hyper_J"]), p(arrs["colour"]),
                  code)
    return d, arrs


def _create_code(isg, d):
    arr = (isg._Desc * 1)(d)
    code, h = isg.create_raw(C.cast(arr, C.c_void_p), 1)
    assert not h.value or code == 0
    return code


def test_create_rejects_malformed_instances(isg):
    base = W.random_graph(40, 3.0, 1, dtype="f32", n_hyper=3, hyper_order=(3,))
    # asymmetric values
    J = base.J.copy()
    J[0] += 1.0
    d, keep = _desc(isg, base, J=J)
    assert _create_code(isg, d) == 2
    # self loop: point the first entry of row 0 at spin 0
    col = base.col.copy()
    col[base.row_ptr[0]] = 0
    d, keep = _desc(isg, base, col=col)
    assert _create_code(isg, d) == 3
    # out-of-range column
    col = base.col.copy()
    col[0] = 1000
    d, keep = _desc(isg, base, col=col)
    assert _create_code(isg, d) == 1
    # hyper-edge with a repeated member
    hm = base.hyper_members.copy()
    hm[1] = hm[0]
    d, keep = _desc(isg, base, hyper_members=hm)
    assert _create_code(isg, d) == 4
    # hyper-edge with one member
    hp = np.array([0, 1, 3, 6, 9], np.int64)
    hm = np.concatenate([[5], base.hyper_members]).astype(np.int32)
    hJ = np.concatenate([[1.0], base.hyper_J]).astype(np.float32)
    d, keep = _desc(isg, base, hyper_ptr=hp, hyper_members=hm, hyper_J=hJ)
    assert _create_code(isg, d) == 4
    # improper colouring: everybody colour 0
    d, keep = _desc(isg, base, colour=np.zeros(base.n, np.int32))
    assert _create_code(isg, d) == 5
    # decreasing row pointer
    rp = base.row_ptr.copy()
    rp[3] = rp[4] + 1
    d, keep = _desc(isg, base, row_ptr=rp)
    assert _create_code(isg, d) == 1


def test_create_rejects_bad_arguments(isg):
    code, h = isg.create_raw(None, 1)
    assert code == 1 and not h.value
    base = W.lattice((4, 4), couplings="pm1")
    d, keep = _desc(isg, base)
    d.n = 0
    assert _create_code(isg, d) == 1


def test_noalloc_rejects_null_pointers_before_any_device_work(isg):
    """ising_energy_noalloc checks its required pointers and sizes on the host
    and returns ISING_ERR_INVALID_ARG without touching a device."""
    L = isg.lib()
    fake = C.c_void_p(0x1000)  # never dereferenced: every call below fails its checks first
    args = dict(n=4, row_ptr=fake, col=fake, J=fake, h=None, dt=0, spins=fake, R=1, E=fake)
    cases = [dict(col=None), dict(J=None), dict(row_ptr=None), dict(spins=None), dict(E=None),
             dict(n=0), dict(R=0), dict(dt=7)]
    for c in cases:
        a = {**args, **c}
        code = L.ising_energy_noalloc(a["n"], a["row_ptr"], a["col"], a["J"], a["h"], a["dt"], a["spins"], a["R"],
                                      a["E"], None)
        assert code == 1, (c, code)


def test_create_checks_fp64_instances(isg):
    """FP64 instances (ISING_F64) get the same checks: non-finite values,
    asymmetric values, non-finite fields and hyper-edge strengths; a dense
    matrix is FP32 only."""
    import dataclasses
    base = W.random_graph(30, 3.0, 2, dtype="f32", n_hyper=2, hyper_order=(3,))
    base = dataclasses.replace(base, J=base.J.astype(np.float64), h=base.h.astype(np.float64),
                               hyper_J=base.hyper_J.astype(np.float64), dtype="f64")
    J = base.J.copy()
    J[0] = np.nan
    d, keep = _desc(isg, base, J=J)
    assert _create_code(isg, d) == 1
    J = base.J.copy()
    J[0] += 2.0 ** -40  # below FP32 resolution, a real asymmetry in FP64
    d, keep = _desc(isg, base, J=J)
    assert _create_code(isg, d) == 2
    hh = base.h.copy()
    hh[3] = np.inf
    d, keep = _desc(isg, base, h=hh)
    assert _create_code(isg, d) == 1
    hJ = base.hyper_J.copy()
    hJ[1] = np.nan
    d, keep = _desc(isg, base, hyper_J=hJ)
    assert _create_code(isg, d) == 1


def test_sk_eighths_fields_are_exact_in_bf16_and_fp32():
    """The premise of the dense path's exact-field parity cases: the
    generator's couplings are symmetric with a zero diagonal, round-trip
    through BF16 unchanged, and FP32 sums of a field's terms - in index order,
    reversed, and pairwise - equal the FP64 sums."""
    torch = pytest.importorskip("torch")
    n = 1024
    inst = W.sk_eighths(n, 5)
    J, h = inst.J_dense, inst.h
    assert np.array_equal(J, J.T) and not np.any(np.diag(J))
    assert np.array_equal(np.unique(J * 8), np.arange(-8, 9)) and np.array_equal(np.unique(h * 8), np.arange(-4, 5))
    assert np.array_equal(torch.from_numpy(J).to(torch.bfloat16).float().numpy(), J)
    rng = np.random.default_rng(1)
    s = rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(4, n))
    terms = J[None, :, :] * s[:, None, :]  # [replica, i, j] = J_ij s_j
    exact = terms.astype(np.float64).sum(axis=2) + h
    fwd = np.cumsum(terms, axis=2, dtype=np.float32)[:, :, -1] + h
    rev = np.cumsum(terms[:, :, ::-1], axis=2, dtype=np.float32)[:, :, -1] + h
    pair = terms.sum(axis=2, dtype=np.float32) + h
    for f in (fwd, rev, pair):
        assert f.dtype == np.float32 and np.array_equal(f.astype(np.float64), exact)
