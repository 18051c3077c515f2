"""The pass-based search with hill climbing (Sec. IV, Fig. 3) on the GPU
against the oracle's heap implementation (Fig. 4), move for move: the same
starts, the same passes, the same results.  Integer couplings: spins,
energies and pass counts exactly equal.  Float couplings: spins and pass
counts equal, energies within 1e-9 relative (the oracle sums energies with
compensation, the kernel in plain FP64; the improvement margin of a pass
absorbs that difference).  Instances whose fields and energies FP64 computes
exactly run in 64-bit integers on the GPU; one test mixes such an instance
with one whose couplings span too many binary orders for that (FP64 path);
another has two components at scales 2^30 apart, so its fields are exact
spin by spin but its energy is not one integer sum (per-spin integer path)."""
import dataclasses

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


def _oracle_fm(inst, seed, b, R, restarts):
    spins, energies, passes = [], [], []
    for r in range(R):
        best_E, best_s, tp = np.inf, None, 0
        for k in range(restarts):
            s, E, p = oracle.fm_search(inst, oracle.random_start(inst.n, seed, b, r, k))
            tp += p
            if E < best_E:
                best_E, best_s = E, s
        spins.append(best_s)
        energies.append(best_E)
        passes.append(tp)
    return np.array(spins), np.array(energies), np.array(passes)


def _compare(insts, R, restarts, exact):
    seeds = [W.replica_seed(W.splitmix64(0xF00 + b)) for b in range(len(insts))]
    h = isg.Handle(insts)
    sp, E, P, st = h.fm_search(seeds, R, restarts=restarts)
    torch.cuda.synchronize()
    total_passes = 0
    for b, inst in enumerate(insts):
        s_o, E_o, p_o = _oracle_fm(inst, seeds[b], b, R, restarts)
        s_g = h.spins_of(sp, b, R).cpu().numpy()
        assert np.array_equal(s_g, s_o), f"spins differ for instance {b}"
        assert np.array_equal(P[b].cpu().numpy(), p_o), f"pass counts differ for instance {b}"
        if exact:
            assert np.array_equal(E[b].cpu().numpy(), E_o)
        else:
            np.testing.assert_allclose(E[b].cpu().numpy(), E_o, rtol=1e-9, atol=1e-9)
        total_passes += int(p_o.sum())
    assert st["descents"] == len(insts) * R * restarts
    assert st["sweeps"] == total_passes
    h.close()


def test_fm_integer_graph_with_hyperedges():
    inst = W.random_graph(300, 4.0, 71, dtype="i8", n_hyper=25, hyper_order=(3, 4))
    _compare([inst], 16, 3, True)


def test_fm_pm_lattice_with_fields():
    inst = W.lattice((16, 16), periodic=True, couplings="pm1", fields="pm1_0", seed=72)
    _compare([inst], 32, 2, True)


def test_fm_float_graph_with_hyperedges():
    inst = W.random_graph(200, 5.0, 73, dtype="f32", n_hyper=20, hyper_order=(3,))
    _compare([inst], 16, 2, False)


def test_fm_uneven_integer_batch():
    insts = [W.random_graph(n, 3.0, 80 + n, dtype="i8", n_hyper=n // 20, hyper_order=(3,))
             for n in (1, 5, 100, 700)]
    _compare(insts, 8, 2, True)


def test_fm_chimera_2048_float():
    inst = W.chimera(16, seed=74)
    _compare([inst], 4, 1, False)


def test_fm_dense_sk():
    inst = W.sk(128, seed=75)
    _compare([inst], 8, 2, False)


def test_fm_reaches_lower_energies_than_greedy_descent():
    """Same starts: the passes with hill climbing end no higher than the first
    1-flip minimum (a pass only keeps a strictly better prefix), and lower on
    average."""
    inst = W.lattice((32, 32), periodic=True, couplings="gauss", seed=76)
    R, seed = 64, 77
    h = isg.Handle([inst])
    _, E_fm, _, _ = h.fm_search([seed], R, restarts=1)
    res = h.local_search([seed], R, max_sweeps=1000, restarts=1, refresh_every=1, schedule=isg.SCHED_SEQUENTIAL)
    torch.cuda.synchronize()
    e_fm, e_gd = E_fm[0].cpu().numpy(), res.energy[0].cpu().numpy()
    assert e_fm.mean() < e_gd.mean()
    h.close()


def test_fm_rejects_instances_beyond_its_size():
    inst = W.lattice((72, 72), periodic=True, couplings="pm1", seed=78)  # 5184 spins
    h = isg.Handle([inst])
    with pytest.raises(isg.IsingError) as ei:
        h.fm_search([1], 4)
    assert ei.value.code == 6  # ISING_ERR_UNSUPPORTED
    h.close()


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_fm_parallel_and_sequential_starts_agree(dtype):
    """Starts run one per warp (the best chosen by a second launch) or one
    after another in a warp: identical spins, energies and pass counts."""
    insts = [W.random_graph(n, 4.0, 90 + n, dtype=dtype, n_hyper=n // 25, hyper_order=(3,)) for n in (64, 333, 1500)]
    seeds = [11, 12, 13]
    out = {}
    for mode in ("0", "1"):
        h = isg.Handle(insts)
        sp, E, P, st = h.fm_search(seeds, 24, restarts=4, starts=1 if mode == "0" else 2)
        torch.cuda.synchronize()
        out[mode] = (sp.cpu().numpy(), E.cpu().numpy(), P.cpu().numpy(), st["descents"], st["sweeps"])
        h.close()
    for a, b in zip(out["0"], out["1"]):
        assert np.array_equal(a, b)
    assert out["0"][3] == 3 * 24 * 4


def _wide_spread(inst, scale=2.0 ** -60):
    """A copy with one coupling pair scaled far below the rest: the couplings
    then span more than 38 binary orders, so the integer form does not apply
    and the kernel keeps FP64."""
    J = inst.J.copy()
    i = int(np.nonzero(np.diff(inst.row_ptr) > 0)[0][0])
    k = int(inst.row_ptr[i])
    j = int(inst.col[k])
    J[k] = np.float32(J[k] * scale)
    lo, hi = int(inst.row_ptr[j]), int(inst.row_ptr[j + 1])
    kk = lo + int(np.nonzero(inst.col[lo:hi] == i)[0][0])
    J[kk] = J[k]
    return dataclasses.replace(inst, J=J)


def test_fm_float_exact_and_fp64_instances_in_one_batch():
    a = W.random_graph(300, 4.0, 91, dtype="f32", n_hyper=15, hyper_order=(3,))
    b = _wide_spread(W.random_graph(260, 4.0, 92, dtype="f32", n_hyper=12, hyper_order=(3, 4)))
    _compare([a, b], 12, 2, False)


def _two_scales(a, b, scale=2.0 ** -30):
    """Block-diagonal union of two FP32 instances, the second scaled by
    `scale`: each spin's terms stay within a narrow range of binary orders,
    the instance's as a whole do not."""
    n = a.n + b.n
    row_ptr = np.concatenate([a.row_ptr, a.row_ptr[-1] + b.row_ptr[1:]]).astype(np.int64)
    col = np.concatenate([a.col, b.col + a.n]).astype(np.int32)
    J = np.concatenate([a.J, (b.J * scale).astype(np.float32)])
    h = np.concatenate([a.h, (b.h * scale).astype(np.float32)])
    hp = np.concatenate([a.hyper_ptr, a.hyper_ptr[-1] + b.hyper_ptr[1:]]).astype(np.int64)
    hm = np.concatenate([a.hyper_members, b.hyper_members + a.n]).astype(np.int32)
    hJ = np.concatenate([a.hyper_J, (b.hyper_J * scale).astype(np.float32)])
    return W.Instance(n=n, row_ptr=row_ptr, col=col, J=J, h=h, hyper_ptr=hp, hyper_members=hm, hyper_J=hJ,
                      dtype="f32")


def test_fm_float_per_spin_exact_instance():
    a = W.random_graph(180, 4.0, 93, dtype="f32", n_hyper=10, hyper_order=(3,))
    b = W.random_graph(150, 4.0, 94, dtype="f32", n_hyper=8, hyper_order=(3, 4))
    c = W.random_graph(120, 4.0, 95, dtype="f32", n_hyper=6, hyper_order=(3,))
    _compare([_two_scales(a, b), c, _wide_spread(b)], 12, 2, False)


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_fm_denser_graph(dtype):
    """Degrees around 30-60: a move's changed fields span one or two rounds of
    the warp and, for the densest spins, more than the touched list holds (every
    block maximum is then recomputed)."""
    inst = W.random_graph(400, 46.0, 96, dtype=dtype, n_hyper=30, hyper_order=(3, 5))
    _compare([inst], 8, 2, dtype == "i8")


def test_two_handles_on_two_threads():
    """Calls on different handles from different host threads give the same
    results as the same calls made one after another."""
    import threading
    insts = [W.random_graph(500, 4.0, 97, dtype="f32", n_hyper=20, hyper_order=(3,)),
             W.lattice((24, 24), periodic=True, couplings="pm1", seed=98)]

    def run(inst, out, k):
        h = isg.Handle([inst])
        for _ in range(3):
            sp, E, P, _ = h.fm_search([7 + k], 64, restarts=2)
            res = h.local_search([7 + k], 64, max_sweeps=200, restarts=2)
        torch.cuda.synchronize()
        out[k] = (sp.cpu().numpy(), E.cpu().numpy(), res.spins.cpu().numpy(), res.energy.cpu().numpy())
        h.close()

    seq, par = {}, {}
    for k, inst in enumerate(insts):
        run(inst, seq, k)
    threads = [threading.Thread(target=run, args=(inst, par, k)) for k, inst in enumerate(insts)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for k in range(len(insts)):
        for a, b in zip(seq[k], par[k]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_fm_register_kernel_matches_shared_memory_kernel(dtype):
    """Instances of up to 512 spins in the one-unit integer form run on the
    register-resident kernel (8 or 16 spins per lane; reg_kernel=1 whatever
    the number of searches); reg_kernel=-1 keeps them on the shared-memory
    kernel.  Identical spins, energies and pass counts, including a dense
    instance (rows longer than a warp) and a hyper-edge with 40 members."""
    insts = [W.random_graph(n, 4.0, 110 + n, dtype=dtype, n_hyper=n // 20, hyper_order=(3, 4))
             for n in (7, 64, 200, 256, 257, 400, 512)]
    insts.append(W.random_graph(90, 50.0, 120, dtype=dtype))
    big = W.random_graph(120, 3.0, 121, dtype=dtype)
    hp = np.array([0, 40], dtype=np.int64)
    hm = np.arange(0, 80, 2, dtype=np.int32)
    hJ = np.array([1 if dtype == "i8" else 0.75], dtype=np.int8 if dtype == "i8" else np.float32)
    insts.append(dataclasses.replace(big, hyper_ptr=hp, hyper_members=hm, hyper_J=hJ))
    seeds = [31 + b for b in range(len(insts))]
    out = {}
    for mode in ("0", "1"):
        h = isg.Handle(insts)
        sp, E, P, st = h.fm_search(seeds, 12, restarts=3, reg_kernel=-1 if mode == "0" else 1)
        torch.cuda.synchronize()
        out[mode] = (sp.cpu().numpy(), E.cpu().numpy(), P.cpu().numpy(), st["sweeps"])
        h.close()
    for a, b in zip(out["0"], out["1"]):
        assert np.array_equal(a, b)
    last = len(insts) - 1
    _, E_o, p_o = _oracle_fm(insts[last], seeds[last], last, 12, 3)
    assert np.array_equal(out["1"][2][last], p_o)
    np.testing.assert_allclose(out["1"][1][last], E_o, rtol=1e-9, atol=1e-9)
