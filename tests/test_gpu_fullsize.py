"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times (the same instances, seeds, replica counts, search parameters
and kernel planner):

* sampled outputs the oracle can compute one by one: replica ranges spread
  over the replica words and groups (or a few whole instances) are recomputed
  by the oracle and must match (spins bit for bit, energies exactly for
  integer couplings and within 1e-9 for FP32);
* properties that hold at any size, on every replica: the returned energy is
  the oracle's energy of the returned spins, and a replica with a converged
  descent returns a 1-flip local minimum (s_i f_i >= 0; for FP32 fields within
  the fields' rounding, 1e-4).
"""
from concurrent.futures import ThreadPoolExecutor

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


def _check_sample(inst, b, seed, R_sample, kw, sp, E, minima, exact, first=0):
    """Replicas first .. first + R_sample - 1 against the oracle."""
    s, Eo, m, _ = oracle.descent(inst, seed, b, R_sample, first_replica=first, **kw)
    sl = slice(first, first + R_sample)
    assert np.array_equal(sp[sl], s), f"spins differ (instance {b}, replicas {first}..)"
    assert np.array_equal(minima[sl], m), f"minima differ (instance {b}, replicas {first}..)"
    if exact:
        assert np.array_equal(E[sl], Eo)
    else:
        np.testing.assert_allclose(E[sl], Eo, rtol=1e-9, atol=1e-9)


def _check_ranges(inst, seed, kw, sp, E, minima, exact, ranges):
    """Several replica ranges, each in its own host thread (the oracle's C
    calls release the GIL)."""
    with ThreadPoolExecutor(max_workers=len(ranges)) as ex:
        futs = [ex.submit(_check_sample, inst, 0, seed, cnt, kw, sp, E, minima, exact, first)
                for first, cnt in ranges]
        for f in futs:
            f.result()


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
    """Three whole 32-replica words (every bit position: the first, a middle
    and the last word of the multi-spin coding) against the oracle."""
    insts, R, kw, seeds, h, res = _search("c2")
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E, m = res.energy[0].cpu().numpy(), res.minima[0].cpu().numpy()
    _check_ranges(insts[0], seeds[0], kw, sp, E, m, True, [(0, 32), (496, 32), (992, 32)])
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
    """256 replicas, eight in each of the 32 tensor-core clusters of 128: the
    returned energy against the oracle's FP64 energy of the returned spins
    (1e-6 relative) and the 1-flip minimum property within the FP32 field
    rounding."""
    insts, R, kw, seeds, h, res = _search("c4")
    assert res.stats["minima"] == R and res.stats["descents"] == R
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E = res.energy[0].cpu().numpy()
    oi = oracle.OracleInstance(insts[0])
    pick = np.array(sorted({128 * k + 16 * j + (k % 16) for k in range(R // 128) for j in range(8)}))
    assert len(pick) == 256

    def one(r):
        Eo = oracle.energy(oi, sp[r])
        f = oracle.local_fields(oi, sp[r])
        return abs(E[r] - Eo) / abs(Eo), float(np.min(sp[r] * f))

    with ThreadPoolExecutor(max_workers=16) as ex:
        out = list(ex.map(one, pick))
    rel = max(o[0] for o in out)
    assert rel <= 1e-6, rel
    assert min(o[1] for o in out) >= -1e-4
    h.close()


def test_fullsize_dense_exact_fields_per_replica():
    """The dense launch configuration at full size (4096 spins, 4096 replicas,
    the benchmark's search parameters, seed and planner) on an instance whose
    couplings and fields are multiples of 1/8, so that no field carries a
    rounding: 32 replicas, one in each tensor-core cluster of 128 at a varying
    lane, each equal to the oracle's sequential FP64 descent from the same
    Philox start move for move (spins, energy, minima count)."""
    _, R, kw, _ = bench.make_workload("c4")
    seed = bench.seeds_for("c4", 1, 0)[0]
    inst = W.sk_eighths(4096, 4096)
    h = isg.Handle([inst])
    assert h.plan_kernel(R) == isg.KERNEL_DENSE_TC
    res = h.local_search([seed], R, kernel=isg.KERNEL_AUTO, **kw)
    torch.cuda.synchronize()
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E = res.energy[0].cpu().numpy()
    m = res.minima[0].cpu().numpy()
    assert res.stats["descents"] == R
    h.close()
    oi = oracle.OracleInstance(inst)
    pick = [128 * k + (37 * k + 5) % 128 for k in range(R // 128)]
    kw_o = dict(kw, mode=oracle.MODE_F64)

    def one(r):
        s, Eo, mo, _ = oracle.descent(oi, seed, 0, 1, first_replica=r, **kw_o)
        return r, s[0], Eo[0], mo[0]

    with ThreadPoolExecutor(max_workers=16) as ex:
        out = list(ex.map(one, pick))
    for r, s, Eo, mo in out:
        assert np.array_equal(sp[r], s), f"replica {r} differs from the sequential descent"
        assert E[r] == Eo and m[r] == mo, (r, E[r], Eo, m[r], mo)


@pytest.mark.parametrize("name,exact,tol", [("c5", False, 1e-4), ("c5i", True, 0.0)])
def test_fullsize_lattice_100cubed(name, exact, tol):
    """Four of the 16 replicas (first, two middle, last lane of the group)
    through their whole 1000-sweep budgets against the oracle, one host thread
    each; properties on all 16."""
    insts, R, kw, seeds, h, res = _search(name)
    sp = h.spins_of(res.spins, 0, R).cpu().numpy()
    E, m = res.energy[0].cpu().numpy(), res.minima[0].cpu().numpy()
    _check_ranges(insts[0], seeds[0], kw, sp, E, m, exact, [(0, 1), (5, 1), (10, 1), (R - 1, 1)])
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
