"""GPU parity on degenerate and ragged inputs: single spins, isolated spins,
zero couplings, order-2 hyper-edges over an existing pair, uneven batches,
a single replica, a user-supplied colouring.  Bit-exact against the oracle
for integer couplings, spins bit-exact and energies within 1e-9 for FP32."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

isg = pytest.importorskip("paper_0912_3912_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0912_3912_gb300 import build as B
    B.build()
    oracle.build()


def _inst(n, edges, w, h, dtype, hyper=None, colour=None):
    u = np.array([e[0] for e in edges], dtype=np.int64)
    v = np.array([e[1] for e in edges], dtype=np.int64)
    npdt = np.int8 if dtype == "i8" else np.float32
    row_ptr, col, J = W.csr_from_edges(n, u, v, np.array(w, dtype=npdt), dtype)
    inst = W.Instance(n=n, row_ptr=row_ptr, col=col, J=J,
                      h=None if h is None else np.array(h, dtype=npdt), dtype=dtype,
                      colour=None if colour is None else np.asarray(colour, dtype=np.int32))
    if hyper:
        members, ptr, hj = [], [0], []
        for mem, val in hyper:
            members.extend(mem)
            ptr.append(len(members))
            hj.append(val)
        inst.hyper_ptr = np.array(ptr, dtype=np.int64)
        inst.hyper_members = np.array(members, dtype=np.int32)
        inst.hyper_J = np.array(hj, dtype=npdt)
    return inst


def _compare(insts, R, exact, **kw):
    seeds = [W.replica_seed(W.splitmix64(0xED6E + b)) for b in range(len(insts))]
    h = isg.Handle(insts)
    res = h.local_search(seeds, R, **kw)
    torch.cuda.synchronize()
    kw.pop("kernel", None)
    tot = dict(flip_evals=0, flips=0, minima=0, descents=0, sweeps=0)
    for b, inst in enumerate(insts):
        s, E, m, st = oracle.descent(inst, seeds[b], b, R, **kw)
        sp = h.spins_of(res.spins, b, R).cpu().numpy()
        assert np.array_equal(sp, s), f"spins differ for instance {b}"
        assert np.array_equal(res.minima[b].cpu().numpy(), m), f"minima differ for instance {b}"
        Eg = res.energy[b].cpu().numpy()
        if exact:
            assert np.array_equal(Eg, E), f"energies differ for instance {b}"
        else:
            np.testing.assert_allclose(Eg, E, rtol=1e-9, atol=1e-9)
        for k in tot:
            tot[k] += st[k]
    assert {k: res.stats[k] for k in tot} == tot
    h.close()


def _int_batch():
    return [
        _inst(1, [], [], [2], "i8"),                                   # one spin, field
        _inst(1, [], [], None, "i8"),                                  # one spin, nothing: never moves
        _inst(5, [], [], [-1, 0, 1, 2, -3], "i8"),                     # isolated spins
        _inst(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)], [0, 0, 0, 0, 0], [1, -1, 0, 0, 2, -2], "i8"),
        _inst(7, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6)], [3, -2, 1, -3, 2], [0, 1, 0, -1, 0, 0, 1], "i8",
              hyper=[((0, 1), -2), ((2, 4, 6), 3), ((3, 5), 1)]),      # order-2 edge over an existing pair
    ]


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_SWEEP, isg.KERNEL_PLAIN])
def test_degenerate_integer_batch(kernel):
    _compare(_int_batch(), 33, True, max_sweeps=50, restarts=3, kernel=kernel)


@pytest.mark.parametrize("kernel", [isg.KERNEL_MSC, isg.KERNEL_TILE, isg.KERNEL_SWEEP])
def test_degenerate_multi_spin_coded_batch(kernel):
    insts = [
        _inst(1, [], [], [1], "i8"),
        _inst(3, [], [], [-1, 0, 1], "i8"),
        _inst(4, [(0, 1), (1, 2), (2, 3), (0, 3)], [1, -1, 1, 1], None, "i8"),
    ]
    _compare(insts, 40, True, max_sweeps=50, restarts=2, kernel=kernel)


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_SWEEP, isg.KERNEL_PLAIN])
def test_degenerate_float_batch(kernel):
    insts = [
        _inst(1, [], [], [0.3], "f32"),
        _inst(4, [], [], [-0.5, 0.0, 1.25, -2.0], "f32"),
        _inst(5, [(0, 1), (1, 2), (3, 4)], [0.0, 0.0, 0.0], [0.1, -0.2, 0.0, 0.0, 0.7], "f32"),
        _inst(6, [(0, 1), (2, 3), (4, 5), (1, 2)], [0.5, -1.5, 2.0, 0.25], None, "f32",
              hyper=[((0, 3), 0.75), ((1, 4, 5), -1.0)]),
    ]
    _compare(insts, 5, False, max_sweeps=50, restarts=4, refresh_every=3, kernel=kernel)


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_MSC, isg.KERNEL_SWEEP, isg.KERNEL_PLAIN])
def test_single_replica(kernel):
    inst = W.lattice((8, 8), periodic=True, couplings="pm1", fields="pm1_0", seed=51)
    _compare([inst], 1, True, max_sweeps=100, restarts=5, kernel=kernel)


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_SWEEP])
def test_user_colouring_one_class_per_spin(kernel):
    """A valid colouring with one class per spin (the sequential order as classes)."""
    inst = W.random_graph(120, 4.0, 52, dtype="f32", n_hyper=10, hyper_order=(3,))
    inst.colour = np.arange(inst.n, dtype=np.int32)
    _compare([inst], 20, False, max_sweeps=200, restarts=2, kernel=kernel)
