"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times (the same instances, seeds, replica counts, search parameters
and kernel planner):

* sampled outputs the oracle can compute one by one: the first replicas (or a
  few whole instances) are recomputed by the oracle and must match (spins bit
  for bit, energies exactly for integer couplings and within 1e-9 for FP32);
* properties that hold at any size, on every replica: the returned energy is
  the oracle's energy of the returned spins, and a replica with a converged
  descent returns a 1-flip local minimum (s_i f_i >= 0; for FP32 fields within
  the fields' rounding, 1e-4).
"""
import numpy as np
import pytest

import bench
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


def _search(name):
    insts, R, kw, _ = bench.make_workload(name)
    seeds = bench.seeds_for(name, len(insts), 0)
    h = isg.Handle(insts)
    res = h.local_search(seeds, R, kernel=isg.KERNEL_AUTO, **kw)
    torch.cuda.synchronize()
    return insts, R, kw, seeds, h, res


def _check_sample(inst, b, seed, R_sample, kw, sp, E, minima, exact):
    s, Eo, m, _ = oracle.descent(inst, seed, b, R_sample, **kw)
    assert np.array_equal(sp[:R_sample], s), f"spins differ (instance {b})"
    assert np.array_equal(minima[:R_sample], m), f"minima differ (instance {b})"
    if exact:
        assert np.array_equal(E[:R_sample], Eo)
    else:
        np.testing.assert_allclose(E[:R_sample], Eo, rtol=1e-9, atol=1e-9)


def _check_properties(inst, sp, E, minima, exact, tol=0.0):
    oi = oracle.OracleInstance(inst)
    Eo = oracle.energies(oi, sp)
    if exact:
        assert np.array_equal(E, Eo)
    else:
        np.testing.assert_allclose(E, Eo, rtol=1e-9, atol=1e-9)
    for r in np.nonzero(minima > 0)[0]:
        f = oracle.local_fields(oi, sp[r])
        assert np.all(sp[r] * f >= -tol), f"replica {r} is not a 1-flip minimum"


def test_fullsize_lattice_16x16():
    insts, R, kw, seeds, h, res = _search("c1")
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E, m = res.energy[0].cpu().numpy(), res.minima[0].cpu().numpy()
    _check_sample(insts[0], 0, seeds[0], R, kw, sp, E, m, True)
    h.close()


def test_fullsize_lattice_32cubed_1024_replicas():
    insts, R, kw, seeds, h, res = _search("c2")
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E, m = res.energy[0].cpu().numpy(), res.minima[0].cpu().numpy()
    _check_sample(insts[0], 0, seeds[0], 8, kw, sp, E, m, True)
    _check_properties(insts[0], sp, E, m, True)
    h.close()


def test_fullsize_chimera_batch_4096():
    insts, R, kw, seeds, h, res = _search("c3")
    for b in (0, 1, 2047, len(insts) - 1):
        sp = h.spins_of(res.spins, b, R).cpu().numpy()
        E, m = res.energy[b].cpu().numpy(), res.minima[b].cpu().numpy()
        _check_sample(insts[b], b, seeds[b], R, kw, sp, E, m, False)
    h.close()


def test_fullsize_dense_sk_4096():
    insts, R, kw, seeds, h, res = _search("c4")
    assert res.stats["minima"] == R and res.stats["descents"] == R
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E = res.energy[0].cpu().numpy()
    oi = oracle.OracleInstance(insts[0])
    pick = np.array([0, 1, 127, 128, 2048, R - 1])
    Eo = oracle.energies(oi, sp[pick])
    assert np.max(np.abs(E[pick] - Eo) / np.abs(Eo)) <= 1e-6
    for r in pick:
        f = oracle.local_fields(oi, sp[r])
        assert np.all(sp[r] * f >= -1e-4)
    h.close()


@pytest.mark.parametrize("name,exact,tol", [("c5", False, 1e-4), ("c5i", True, 0.0)])
def test_fullsize_lattice_100cubed(name, exact, tol):
    insts, R, kw, seeds, h, res = _search(name)
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E, m = res.energy[0].cpu().numpy(), res.minima[0].cpu().numpy()
    _check_sample(insts[0], 0, seeds[0], 1, kw, sp, E, m, exact)
    _check_properties(insts[0], sp, E, m, exact, tol)
    h.close()


# --------------------------------------------------------------------------- pass-based search
def _fm_full(name):
    insts, R, kw, _ = bench.make_workload(name)
    seeds = bench.seeds_for(name, len(insts), 0)
    restarts = int(kw.get("restarts", 1))
    h = isg.Handle(insts)
    sp, E, P, st = h.fm_search(seeds, R, restarts=restarts)
    torch.cuda.synchronize()
    return insts, R, restarts, seeds, h, sp, E.cpu().numpy(), P.cpu().numpy(), st


def _oracle_fm_best(inst, seed, b, r, restarts):
    best, total = None, 0
    for k in range(restarts):
        s, Ek, p = oracle.fm_search(inst, oracle.random_start(inst.n, seed, b, r, k))
        total += p
        if best is None or Ek < best[1]:
            best = (s, Ek)
    return best[0], best[1], total


def test_fm_c1_full_every_replica():
    """16x16 +/-J, 64 replicas x 10 starts (starts in parallel, then the
    best-start selection): every replica against the oracle."""
    insts, R, restarts, seeds, h, sp, E, P, st = _fm_full("c1")
    inst = insts[0]
    s_all = h.spins_of(sp, 0, R).cpu().numpy()
    for r in range(R):
        s_o, E_o, p_o = _oracle_fm_best(inst, seeds[0], 0, r, restarts)
        assert np.array_equal(s_all[r], s_o) and E[0, r] == E_o and P[0, r] == p_o, r
    assert st["descents"] == R * restarts
    h.close()


def test_fm_c3_full_sampled_and_energies():
    """4096 chimera instances x 32 replicas in one call: sampled searches
    (largest, middle and smallest instances) against the oracle; on every
    replica the returned energy is the oracle's energy of the returned spins."""
    insts, R, restarts, seeds, h, sp, E, P, st = _fm_full("c3")
    order = np.argsort([inst.n for inst in insts])
    for b in (int(order[-1]), int(order[-2]), int(order[len(order) // 2]), int(order[0])):
        s_all = h.spins_of(sp, b, R).cpu().numpy()
        for r in (0, R - 1):
            s_o, E_o, p_o = _oracle_fm_best(insts[b], seeds[b], b, r, restarts)
            assert np.array_equal(s_all[r], s_o), (b, r)
            assert P[b, r] == p_o
            np.testing.assert_allclose(E[b, r], E_o, rtol=1e-9, atol=1e-9)
    for b in range(0, len(insts), 97):
        s_all = h.spins_of(sp, b, R).cpu().numpy()
        Eo = oracle.energies(oracle.OracleInstance(insts[b]), s_all)
        np.testing.assert_allclose(E[b], Eo, rtol=1e-9, atol=1e-9)
    assert st["descents"] == len(insts) * R
    h.close()
