"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Integer couplings: spins, energies, per-replica minima counts and work counters
must match bit-exactly.  FP32 couplings: the library's documented FP32 field
semantics are mirrored by the oracle, so spins must match bit-exactly as well;
energies (FP64 on both sides, different summation order) within 1e-9 relative,
far inside the 1e-6 bar.
"""
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


def _run(insts, seeds, R, **kw):
    h = isg.Handle(insts)
    res = h.local_search(seeds, R, want_i32=insts[0].dtype == "i8", **kw)
    torch.cuda.synchronize()
    out = []
    for b, inst in enumerate(insts):
        sp = h.spins_of(res.spins, b, R).cpu().numpy()
        out.append((sp, res.energy[b].cpu().numpy(), res.minima[b].cpu().numpy()))
    e32 = None if res.energy_i32 is None else res.energy_i32.cpu().numpy()
    h.close()
    return out, res.stats, e32


def _oracle(insts, seeds, R, **kw):
    tot = dict(flip_evals=0, flips=0, minima=0, descents=0, sweeps=0)
    out = []
    for b, inst in enumerate(insts):
        kw2 = dict(kw)
        kw2.pop("kernel", None)
        s, E, m, st = oracle.descent(inst, seeds[b], b, R, **kw2)
        out.append((s, E, m))
        for k in tot:
            tot[k] += st[k]
    return out, tot


def _compare(insts, seeds, R, exact_energy, **kw):
    g, gst, e32 = _run(insts, seeds, R, **kw)
    o, ost = _oracle(insts, seeds, R, **kw)
    for b in range(len(insts)):
        assert np.array_equal(g[b][0], o[b][0]), f"spins differ for instance {b}"
        assert np.array_equal(g[b][2], o[b][2]), f"minima counts differ for instance {b}"
        if exact_energy:
            assert np.array_equal(g[b][1], o[b][1])
        else:
            np.testing.assert_allclose(g[b][1], o[b][1], rtol=1e-9, atol=1e-9)
    assert {k: gst[k] for k in ost} == ost
    assert gst["launches"] >= 1
    if e32 is not None:
        assert np.array_equal(e32.ravel(), np.concatenate([x[1] for x in o]).astype(np.int32))
    return g, o


# ----------------------------------------------------------- 16x16 +/-J lattice (64 replicas)
@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_MSC, isg.KERNEL_AUTO, isg.KERNEL_PLAIN])
def test_lattice_16x16_pmJ_bit_exact(kernel):
    inst = W.lattice((16, 16), periodic=True, couplings="pm1", seed=W.config_seed(0))
    seed = W.replica_seed(W.config_seed(0))
    _compare([inst], [seed], 64, True, max_sweeps=1000, restarts=10, kernel=kernel)


def test_lattice_4x4_reaches_bruteforce_ground_state():
    inst = W.lattice((4, 4), periodic=True, couplings="pm1", seed=3)
    Egs, _, _ = oracle.bruteforce(inst)
    g, o = _compare([inst], [11], 64, True, max_sweeps=100, restarts=10)
    E = g[0][1]
    assert np.all(E >= Egs) and np.any(E == Egs)


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_MSC])
def test_3d_pmJ_with_fields_ragged_replicas(kernel):
    inst = W.lattice((8, 8, 8), periodic=True, couplings="pm1", fields="pm1_0", seed=5)
    _compare([inst], [77], 37, True, max_sweeps=100, restarts=3, kernel=kernel)


@pytest.mark.parametrize("seed", [4, 5])
def test_msc_on_general_pm1_graph(seed):
    # +/-1 couplings, h in {-1,0,1}, irregular degrees: the generic multi-spin coded evaluator
    inst = W.random_graph(500, 4.0, seed, dtype="i8", int_range=1)
    assert set(np.unique(inst.J)) <= {-1, 1} and np.max(np.diff(inst.row_ptr)) <= 15
    _compare([inst], [seed], 70, True, max_sweeps=200, restarts=3, kernel=isg.KERNEL_MSC)


def test_msc_lattice_2d_and_3d_with_fields():
    for dims in [(14, 14), (10, 10, 10), (6, 8, 10)]:
        inst = W.lattice(dims, periodic=True, couplings="pm1", fields="pm1_0", seed=len(dims))
        _compare([inst], [len(dims)], 45, True, max_sweeps=300, restarts=4, kernel=isg.KERNEL_MSC)


@pytest.mark.parametrize("seed,kernel", [(1, isg.KERNEL_TILE), (2, isg.KERNEL_TILE), (3, isg.KERNEL_PLAIN)])
def test_random_integer_graph_with_hyperedges(seed, kernel):
    inst = W.random_graph(300, 5.0, seed, dtype="i8", n_hyper=40, hyper_order=(2, 3, 4))
    _compare([inst], [seed * 7], 40, True, max_sweeps=500, restarts=2, kernel=kernel)


@pytest.mark.parametrize("refresh,kernel", [(0, isg.KERNEL_TILE), (1, isg.KERNEL_TILE), (4, isg.KERNEL_TILE),
                                            (16, isg.KERNEL_TILE), (4, isg.KERNEL_PLAIN)])
def test_random_float_graph_fp32_mirror(refresh, kernel):
    inst = W.random_graph(333, 4.5, 9, dtype="f32", n_hyper=30, hyper_order=(3, 4))
    _compare([inst], [1234], 33, False, max_sweeps=500, restarts=2, refresh_every=refresh, kernel=kernel)


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_PLAIN])
def test_batched_uneven_chimera_fp32(kernel):
    insts = W.chimera_batch(9, 2, 7, seed=W.config_seed(2))
    seeds = [W.replica_seed(W.splitmix64(W.config_seed(2) + b)) for b in range(len(insts))]
    _compare(insts, seeds, 32, False, max_sweeps=1000, restarts=2, refresh_every=16, kernel=kernel)


@pytest.mark.parametrize("dtype,kernel", [("i8", isg.KERNEL_TILE), ("f32", isg.KERNEL_TILE),
                                          ("f32", isg.KERNEL_PLAIN)])
def test_sequential_schedule(dtype, kernel):
    if dtype == "i8":
        inst = W.random_graph(150, 4.0, 3, dtype="i8", n_hyper=10, hyper_order=(3,))
    else:
        inst = W.chimera(3, seed=4)
    _compare([inst], [5], 20, dtype == "i8", max_sweeps=300, restarts=2, refresh_every=8,
             schedule=isg.SCHED_SEQUENTIAL, kernel=kernel)


@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_MSC, isg.KERNEL_PLAIN])
def test_sweep_budget_and_cap(kernel):
    inst = W.lattice((12, 12, 12), periodic=True, couplings="pm1", fields="pm1_0", seed=6)
    _compare([inst], [3], 32, True, max_sweeps=5, restarts=1000, sweep_budget=23, kernel=kernel)


def test_local_minimum_property_and_energy_api():
    inst = W.chimera(6, seed=8)
    R = 64
    h = isg.Handle([inst])
    res = h.local_search([99], R, max_sweeps=2000, restarts=3)
    E_api = h.energy(res.spins, R)
    torch.cuda.synchronize()
    sp = res.spins.view(R, inst.n).cpu().numpy()
    E = res.energy.view(R).cpu().numpy()
    np.testing.assert_allclose(E_api.view(R).cpu().numpy(), E, rtol=1e-12, atol=1e-12)
    oi = oracle.OracleInstance(inst)
    for r in range(R):
        f = oracle.local_fields(oi, sp[r])
        assert np.all(sp[r] * f >= -1e-4)
        assert abs(oracle.energy(oi, sp[r]) - E[r]) <= 1e-9 * abs(E[r])
    h.close()


def test_energy_api_random_configurations():
    insts = [W.random_graph(n, 4.0, n, dtype="f32", n_hyper=5) for n in (50, 5000, 9000)]
    R = 3
    h = isg.Handle(insts)
    rng = np.random.default_rng(0)
    spins = (rng.integers(0, 2, size=R * h.total_spins) * 2 - 1).astype(np.int8)
    E = h.energy(torch.from_numpy(spins).cuda(), R).cpu().numpy()
    off = 0
    for b, inst in enumerate(insts):
        blk = spins[off: off + R * inst.n].reshape(R, inst.n)
        off += R * inst.n
        ref = oracle.energies(inst, blk)
        np.testing.assert_allclose(E[b], ref, rtol=1e-12, atol=1e-9)
    h.close()


def test_energy_api_dense_instances():
    """ising_energy on a batch of dense instances (Gaussian SK with fields, the
    1/8-multiple instance whose energies are exact in FP64, a size that is not
    a multiple of 256): random configurations against the oracle, and the
    energies a dense search returns against the energy call on its spins."""
    insts = [_sk_with_fields(300, 41), W.sk_eighths(512, 42), W.sk(1000, seed=43)]
    R = 5
    h = isg.Handle(insts)
    rng = np.random.default_rng(7)
    spins = (rng.integers(0, 2, size=R * h.total_spins) * 2 - 1).astype(np.int8)
    E = h.energy(torch.from_numpy(spins).cuda(), R).cpu().numpy()
    off = 0
    for b, inst in enumerate(insts):
        blk = spins[off: off + R * inst.n].reshape(R, inst.n)
        off += R * inst.n
        ref = oracle.energies(inst, blk)
        if b == 1:
            assert np.array_equal(E[b], ref)
        else:
            np.testing.assert_allclose(E[b], ref, rtol=1e-12, atol=1e-9)
    res = h.local_search([3, 4, 5], 64, max_sweeps=300, restarts=1, kernel=isg.KERNEL_DENSE_TC)
    E_api = h.energy(res.spins, 64).cpu().numpy()
    torch.cuda.synchronize()
    # the search's energies quantise J to 32-bit fixed point (at most pairs x max|J| x 2^-31
    # from the definition); the 1/8-multiple couplings are exact in it
    np.testing.assert_allclose(res.energy.cpu().numpy(), E_api, rtol=1e-7, atol=1e-9)
    assert np.array_equal(res.energy[1].cpu().numpy(), E_api[1])
    h.close()


def test_msc_rejected_for_float_and_large_fields():
    inst = W.chimera(2, seed=1)
    h = isg.Handle([inst])
    with pytest.raises(isg.IsingError) as ei:
        h.local_search([1], 32, kernel=isg.KERNEL_MSC)
    assert ei.value.code == 6
    h.close()
    inst = W.random_graph(64, 3.0, 2, dtype="i8", int_range=3)
    h = isg.Handle([inst])
    assert h.plan_kernel(32) == isg.KERNEL_TILE
    h.close()


# ----------------------------------------------------------- large-instance sweep family
@pytest.mark.parametrize("R", [64, 16, 5])
def test_sweep_family_pmJ_lattice_msc(R):
    inst = W.lattice((10, 10, 10), periodic=True, couplings="pm1", fields="pm1_0", seed=21)
    _compare([inst], [321], R, True, max_sweeps=100, restarts=3, kernel=isg.KERNEL_SWEEP)


def test_sweep_family_int_lattice_lanes():
    inst = W.lattice((12, 12), periodic=True, couplings="pm1", seed=22)
    inst.J = (inst.J * 2).astype(np.int8)  # |J| = 2: not multi-spin codable, integer lanes
    _compare([inst], [5], 40, True, max_sweeps=200, restarts=2, kernel=isg.KERNEL_SWEEP)


@pytest.mark.parametrize("R,refresh", [(16, 16), (32, 4), (8, 0)])
def test_sweep_family_gauss_lattice_fp32(R, refresh):
    inst = W.lattice((12, 12, 12), periodic=True, couplings="gauss", seed=23)
    _compare([inst], [77], R, False, max_sweeps=1000, restarts=1 << 20, sweep_budget=60,
             refresh_every=refresh, kernel=isg.KERNEL_SWEEP)


# Lattice energies are summed site by site from each site's +x, +y (+z) bonds:
# 2-D and 3-D, odd and even sides, integer and FP32 couplings, with fields.
@pytest.mark.parametrize("dims,R,couplings", [((15, 15), 8, "gauss"), ((20, 20), 16, "gauss"),
                                              ((9, 9, 9), 16, "gauss"), ((7, 7, 7), 12, "pm1"),
                                              ((8, 8, 8), 16, "pm2")])
def test_sweep_family_lattice_shapes(dims, R, couplings):
    inst = W.lattice(dims, periodic=True, couplings="pm1" if couplings == "pm2" else couplings,
                     fields="gauss" if couplings == "gauss" else "pm1_0", seed=len(dims) * 100 + dims[0])
    if couplings == "pm2":
        inst.J = (inst.J * 2).astype(np.int8)  # not multi-spin codable: integer lanes
    _compare([inst], [17], R, couplings != "gauss", max_sweeps=300, restarts=4, refresh_every=6,
             kernel=isg.KERNEL_SWEEP)


def test_sweep_family_csr_with_hyperedges():
    inst = W.random_graph(700, 4.0, 24, dtype="f32", n_hyper=50, hyper_order=(3, 4))
    _compare([inst], [9], 20, False, max_sweeps=500, restarts=3, refresh_every=8, kernel=isg.KERNEL_SWEEP)


def test_sweep_family_sequential_schedule():
    inst = W.random_graph(200, 4.0, 25, dtype="i8", n_hyper=10, hyper_order=(3,))
    _compare([inst], [3], 12, True, max_sweeps=300, restarts=2, schedule=isg.SCHED_SEQUENTIAL,
             kernel=isg.KERNEL_SWEEP)


# ----------------------------------------------------------- FP32 exponent ranges
def _exp_spread(inst, lo, hi):
    """Scale each coupling pair, field and hyper-edge by 2^e, e in [lo, hi),
    symmetric in the pair, so values span about hi - lo binades."""
    n = inst.n
    rows = np.repeat(np.arange(n), np.diff(inst.row_ptr))
    a = np.minimum(rows, inst.col.astype(np.int64))
    b = np.maximum(rows, inst.col.astype(np.int64))
    e = (a * 7919 + b * 104729) % (hi - lo) + lo
    inst.J = (inst.J.astype(np.float64) * np.exp2(e)).astype(np.float32)
    if inst.h is not None:
        eh = (np.arange(n) * 15485863) % (hi - lo) + lo
        inst.h = (inst.h.astype(np.float64) * np.exp2(eh)).astype(np.float32)
    if inst.hyper_J is not None:
        ee = (np.arange(inst.n_hyper) * 32452843) % (hi - lo) + lo
        inst.hyper_J = (inst.hyper_J.astype(np.float64) * np.exp2(ee)).astype(np.float32)
    return inst


# A refresh sums in fixed point when a spin's terms span few enough binades and
# in FP64 otherwise; energies likewise per instance.  Both sides of each switch:
@pytest.mark.parametrize("lo,hi", [(-12, 8), (-45, 25)])
@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_SWEEP])
def test_fp32_exponent_range_graph(lo, hi, kernel):
    inst = _exp_spread(W.random_graph(300, 5.0, 31, dtype="f32", n_hyper=25, hyper_order=(3,)), lo, hi)
    _compare([inst], [4321], 24, False, max_sweeps=400, restarts=3, refresh_every=3, kernel=kernel)


@pytest.mark.parametrize("lo,hi", [(-20, 4), (-50, 30)])
def test_fp32_exponent_range_lattice_sweep(lo, hi):
    inst = _exp_spread(W.lattice((10, 10, 10), periodic=True, couplings="gauss", fields="gauss", seed=32), lo, hi)
    _compare([inst], [99], 16, False, max_sweeps=1000, restarts=1 << 20, sweep_budget=40,
             refresh_every=5, kernel=isg.KERNEL_SWEEP)


# ----------------------------------------------------------- dense SK on tensor cores
def test_dense_sk_tensor_core_path():
    """BF16 hi+lo fields with FP32 accumulation: results are checked against the
    FP64 oracle on what is unique (energies of the returned states) and on the
    1-flip local-minimum property within the stated field error bound."""
    inst = W.sk(384, seed=5)
    R = 96
    h = isg.Handle([inst])
    assert h.plan_kernel(R) == isg.KERNEL_DENSE_TC
    res = h.local_search([17], R, max_sweeps=500, restarts=2, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    sp = res.spins.view(R, inst.n).cpu().numpy()
    E = res.energy.view(R).cpu().numpy()
    oi = oracle.OracleInstance(inst)
    Eo = oracle.energies(oi, sp)
    rel = np.abs(E - Eo) / np.abs(Eo)
    assert rel.max() <= 1e-6, rel.max()
    for r in range(R):
        f = oracle.local_fields(oi, sp[r])
        assert np.all(sp[r] * f >= -1e-4)
    # same schedule and seeds in FP64: energies reached agree on average
    _, Eo64, _, _ = oracle.descent(oi, 17, 0, R, max_sweeps=500, restarts=2, schedule=oracle.SCHED_SEQUENTIAL,
                                   mode=oracle.MODE_F64)
    assert abs(np.mean(E) - np.mean(Eo64)) <= 0.02 * abs(np.mean(Eo64))
    assert res.stats["minima"] == 2 * R
    h.close()


@pytest.mark.parametrize("n,R", [(512, 96), (768, 256)])
def test_dense_sk_tcgen05_kernel(n, R):
    """The hand-written tcgen05 kernel (n a multiple of 256): energies of the
    returned states within 1e-6 of the FP64 oracle, 1-flip minima within the
    field error bound, and the same results as the library-GEMM comparator on
    the large majority of replicas (fields differ only in FP32 rounding)."""
    inst = W.sk(n, seed=n)
    h = isg.Handle([inst])
    res = h.local_search([29], R, max_sweeps=500, restarts=2, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    sp = res.spins.view(R, n).cpu().numpy().copy()
    E = res.energy.view(R).cpu().numpy().copy()
    st = dict(res.stats)
    oi = oracle.OracleInstance(inst)
    Eo = oracle.energies(oi, sp)
    rel = np.abs(E - Eo) / np.abs(Eo)
    assert rel.max() <= 1e-6, rel.max()
    for r in range(R):
        f = oracle.local_fields(oi, sp[r])
        assert np.all(sp[r] * f >= -1e-4)
    assert st["minima"] == 2 * R and st["descents"] == 2 * R
    ref = h.local_search([29], R, max_sweeps=500, restarts=2, kernel=isg.KERNEL_DENSE_TC, dense_variant=isg.DENSE_LIBRARY)
    torch.cuda.synchronize()
    sp2 = ref.spins.view(R, n).cpu().numpy()
    same = np.mean(np.all(sp == sp2, axis=1))
    assert same >= 0.8, same
    assert abs(np.mean(E) - ref.energy.cpu().numpy().mean()) <= 1e-3 * abs(np.mean(E))
    h.close()


_EIGHTHS_ORACLE = {}


@pytest.mark.parametrize("n,R,restarts,variant,ts", [
    (256, 128, 3, isg.DENSE_OWN, 0),
    (384, 130, 3, isg.DENSE_OWN, 0),
    (384, 130, 3, isg.DENSE_OWN, -1),
    (384, 130, 3, isg.DENSE_OWN, 1000),
    (384, 130, 3, isg.DENSE_LIBRARY, 0),
    (768, 96, 2, isg.DENSE_OWN, 0),
    (5000, 4, 1, isg.DENSE_OWN, 0),
])
def test_dense_exact_fields_match_sequential_oracle_per_replica(n, R, restarts, variant, ts):
    """With couplings and fields in multiples of 1/8 the dense path's fields
    carry no rounding (BF16 holds each coupling exactly, every FP32 sum of
    such terms is exact), so every replica's search on the dense
    path is the oracle's sequential (index-order, Sec. IV) descent with
    restarts from the same Philox starts, move for move: spins, FP64
    energies, minima counts and the work counters all equal, for the
    tensor-core sweeps, the per-replica continuation, both mixed, the
    library-GEMM comparator, a zero-padded size, a partial 128-replica
    cluster, and a size above 4096."""
    inst = W.sk_eighths(n, 300 + n)
    key = (n, R, restarts)
    if key not in _EIGHTHS_ORACLE:
        _EIGHTHS_ORACLE[key] = oracle.descent(oracle.OracleInstance(inst), 23, 0, R, max_sweeps=500,
                                              restarts=restarts, schedule=oracle.SCHED_SEQUENTIAL,
                                              mode=oracle.MODE_F64)
    so, Eo, mo, sto = _EIGHTHS_ORACLE[key]
    h = isg.Handle([inst])
    res = h.local_search([23], R, max_sweeps=500, restarts=restarts, kernel=isg.KERNEL_DENSE_TC,
                         dense_variant=variant, dense_tensor_sweeps=ts)
    torch.cuda.synchronize()
    sp = res.spins.view(R, n).cpu().numpy()
    E = res.energy.view(R).cpu().numpy()
    m = res.minima.view(R).cpu().numpy()
    st = dict(res.stats)
    h.close()
    same = np.all(sp == so, axis=1)
    assert same.all(), f"replicas {np.nonzero(~same)[0][:8]} differ from the sequential descent"
    assert np.array_equal(E, Eo)
    assert np.array_equal(m, mo)
    assert {k: st[k] for k in sto} == sto


def _dense_checks(inst, res, R, tol=1e-4):
    sp = res.spins.view(R, inst.n).cpu().numpy().copy()
    E = res.energy.view(R).cpu().numpy().copy()
    oi = oracle.OracleInstance(inst)
    Eo = oracle.energies(oi, sp)
    rel = np.abs(E - Eo) / np.maximum(np.abs(Eo), 1.0)
    assert rel.max() <= 1e-6, rel.max()
    m = res.minima.view(R).cpu().numpy()
    for r in np.nonzero(m > 0)[0]:
        f = oracle.local_fields(oi, sp[r])
        assert np.all(sp[r] * f >= -tol), f"replica {r} is not a 1-flip minimum"
    return sp, E, m


def _sk_with_fields(n, seed, scale=0.3):
    inst = W.sk(n, seed=seed)
    inst.h = (np.random.default_rng(seed).standard_normal(n) * scale).astype(np.float32)
    return inst


@pytest.mark.parametrize("sweeps_a", ["0", "2", "1000"])
def test_dense_tc_phases_and_fields(sweeps_a):
    """The tensor-core path with its first-sweeps/continuation split moved
    (0: fields exported at once and every sweep continued per replica; 1000:
    every sweep on tensor cores), on an instance with fields h and a replica
    count that leaves a partial 128-replica cluster: energies of the returned
    states, 1-flip minima, work counters, and agreement with the comparator."""
    ts = int(sweeps_a) if int(sweeps_a) > 0 else -1
    inst = _sk_with_fields(512, 77)
    R = 160
    h = isg.Handle([inst])
    res = h.local_search([31], R, max_sweeps=500, restarts=3, kernel=isg.KERNEL_DENSE_TC, dense_tensor_sweeps=ts)
    torch.cuda.synchronize()
    sp, E, m = _dense_checks(inst, res, R)
    st = dict(res.stats)
    assert st["minima"] == 3 * R and st["descents"] == 3 * R and np.all(m == 3)
    assert st["flip_evals"] == st["sweeps"] * inst.n
    ref = h.local_search([31], R, max_sweeps=500, restarts=3, kernel=isg.KERNEL_DENSE_TC, dense_variant=isg.DENSE_LIBRARY)
    torch.cuda.synchronize()
    sp2 = ref.spins.view(R, inst.n).cpu().numpy()
    assert np.mean(np.all(sp == sp2, axis=1)) >= 0.8
    assert dict(ref.stats)["minima"] == 3 * R
    h.close()


@pytest.mark.parametrize("n", [1, 37, 300, 1000])
def test_dense_tc_padded_sizes(n):
    """Sizes that are not a multiple of 256 run zero-padded on the hand-written
    kernels: energies of the returned states, 1-flip minima, exact work
    counters (the instance's own spins), and agreement with the comparator."""
    inst = _sk_with_fields(n, 100 + n)
    R = 130
    h = isg.Handle([inst])
    assert h.plan_kernel(R) == isg.KERNEL_DENSE_TC
    res = h.local_search([11], R, max_sweeps=500, restarts=2, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    sp, E, m = _dense_checks(inst, res, R)
    st = dict(res.stats)
    assert st["minima"] == 2 * R and st["descents"] == 2 * R and np.all(m == 2)
    assert st["flip_evals"] == st["sweeps"] * n
    ref = h.local_search([11], R, max_sweeps=500, restarts=2, kernel=isg.KERNEL_DENSE_TC, dense_variant=isg.DENSE_LIBRARY)
    torch.cuda.synchronize()
    sp2 = ref.spins.view(R, n).cpu().numpy()
    assert np.mean(np.all(sp == sp2, axis=1)) >= 0.8
    h.close()


@pytest.mark.parametrize("n", [5000, 8192, 10000])
def test_dense_tc_sizes_above_4096(n):
    """4096 < n <= 16384 on the hand-written kernels (two-stage operand pipeline
    on tensor cores with the spin bits in shared memory up to 8192 spins and in
    global memory above; 256- and 512-thread continuation; 5000 and 10000
    zero-padded to 5120 and 10240): energies of the returned states against the
    oracle, 1-flip minima, work counters."""
    inst = _sk_with_fields(n, 200 + n)
    R = 130
    h = isg.Handle([inst])
    assert h.plan_kernel(R) == isg.KERNEL_DENSE_TC
    h.set_timing(True)
    res = h.local_search([13], R, max_sweeps=500, restarts=1, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    names = set(h.kernel_times())
    h.set_timing(False)
    assert "dense_tc_kernel" in names and "dense_push_kernel" in names, names
    sp, E, m = _dense_checks(inst, res, R)
    st = dict(res.stats)
    assert st["minima"] == R and st["descents"] == R and np.all(m == 1)
    assert st["flip_evals"] == st["sweeps"] * n
    h.close()


def test_dense_maximum_size_exact_per_replica():
    """The dense family's largest instance, 16384 spins (spin bits in global
    memory, 512-thread continuation, one partial 128-replica cluster), on the
    1/8-multiple couplings: both replicas equal the oracle's sequential FP64
    descent from the same starts move for move, and the returned energies are
    the oracle's energies of the returned spins exactly."""
    from concurrent.futures import ThreadPoolExecutor
    n, R = 16384, 2
    inst = W.sk_eighths(n, n)
    h = isg.Handle([inst])
    assert h.plan_kernel(R) == isg.KERNEL_DENSE_TC
    res = h.local_search([5], R, max_sweeps=1000, restarts=1, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    sp = res.spins.view(R, n).cpu().numpy()
    E = res.energy.view(R).cpu().numpy()
    m = res.minima.view(R).cpu().numpy()
    st = dict(res.stats)
    h.close()
    oi = oracle.OracleInstance(inst)

    def one(r):
        return oracle.descent(oi, 5, 0, 1, first_replica=r, max_sweeps=1000, restarts=1,
                              schedule=oracle.SCHED_SEQUENTIAL, mode=oracle.MODE_F64)

    with ThreadPoolExecutor(max_workers=R) as ex:
        out = list(ex.map(one, range(R)))
    for r, (s, Eo, mo, _) in enumerate(out):
        assert np.array_equal(sp[r], s[0]), f"replica {r} differs from the sequential descent"
        assert E[r] == Eo[0] == oracle.energy(oi, sp[r]) and m[r] == mo[0] == 1
    assert st["sweeps"] == sum(o[3]["sweeps"] for o in out)
    assert st["flips"] == sum(o[3]["flips"] for o in out)


def test_dense_batch_of_instances():
    """Several dense instances in one handle (sizes with and without padding,
    one with fields): each block of results checked on its own instance, and
    the same results when the batch is searched again."""
    insts = [_sk_with_fields(256, 120, scale=0.0), _sk_with_fields(384, 121), _sk_with_fields(1000, 122)]
    R = 64
    h = isg.Handle(insts)
    res = h.local_search([1, 2, 3], R, max_sweeps=400, restarts=2, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    first = res.spins.cpu().numpy().copy()
    st = dict(res.stats)
    assert st["minima"] == 2 * R * len(insts)
    for b, inst in enumerate(insts):
        sp = h.spins_of(res.spins, b, R).cpu().numpy()
        E = res.energy[b].cpu().numpy()
        oi = oracle.OracleInstance(inst)
        Eo = oracle.energies(oi, sp)
        assert np.max(np.abs(E - Eo) / np.maximum(np.abs(Eo), 1.0)) <= 1e-6
        for r in range(R):
            f = oracle.local_fields(oi, sp[r])
            assert np.all(sp[r] * f >= -1e-4)
    again = h.local_search([1, 2, 3], R, max_sweeps=400, restarts=2, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    assert np.array_equal(again.spins.cpu().numpy(), first)
    h.close()


@pytest.mark.parametrize("sweeps_a", ["0", "4"])
def test_dense_tc_sweep_cap_and_budget(sweeps_a):
    """Descents cut by the sweep cap (inside and after the tensor-core sweeps)
    return their final states, counted as no minimum; a sweep budget ends every
    replica after exactly that many sweeps over its restarts."""
    ts = int(sweeps_a) if int(sweeps_a) > 0 else -1
    inst = _sk_with_fields(256, 78, scale=0.1)
    R = 64
    h = isg.Handle([inst])
    for cap in (1, 3, 6):
        res = h.local_search([5], R, max_sweeps=cap, restarts=2, kernel=isg.KERNEL_DENSE_TC,
                             dense_tensor_sweeps=ts)
        torch.cuda.synchronize()
        sp, E, m = _dense_checks(inst, res, R)
        st = dict(res.stats)
        assert st["sweeps"] <= 2 * cap * R and st["descents"] == 2 * R
        if cap == 1:  # one sweep from a random start never ends at a minimum
            assert st["minima"] == 0 and np.all(m == 0) and st["sweeps"] == 2 * R
    res = h.local_search([6], R, max_sweeps=1000, restarts=1 << 20, sweep_budget=37, kernel=isg.KERNEL_DENSE_TC,
                             dense_tensor_sweeps=ts)
    torch.cuda.synchronize()
    _dense_checks(inst, res, R)
    st = dict(res.stats)
    assert st["sweeps"] == 37 * R and st["minima"] >= R
    h.close()


def test_dense_instance_with_hyper_edges_takes_the_csr_path():
    """Hyper-edges on a dense instance: the planner routes it to a CSR family,
    whose results match the oracle's FP32 mirror."""
    inst = _sk_with_fields(96, 79)
    inst.hyper_ptr = np.array([0, 3, 5], dtype=np.int64)
    inst.hyper_members = np.array([1, 7, 50, 3, 90], dtype=np.int32)
    inst.hyper_J = np.array([0.4, -0.25], dtype=np.float32)
    h = isg.Handle([inst])
    assert h.plan_kernel(32) != isg.KERNEL_DENSE_TC
    h.close()
    h2 = isg.Handle([inst])
    res = h2.local_search([3], 32, max_sweeps=200, restarts=2, refresh_every=16, schedule=1)
    torch.cuda.synchronize()
    s, Eo, mo, _ = oracle.descent(inst, 3, 0, 32, max_sweeps=200, restarts=2, refresh_every=16,
                                  schedule=oracle.SCHED_SEQUENTIAL)
    assert np.array_equal(h2.spins_of(res.spins, 0, 32).cpu().numpy(), s)
    np.testing.assert_allclose(res.energy[0].cpu().numpy(), Eo, rtol=1e-9, atol=1e-9)
    h2.close()


def test_autotuner_picks_an_eligible_family_and_results_do_not_depend_on_it(tmp_path, monkeypatch):
    monkeypatch.setenv("ISING_TUNE_CACHE", str(tmp_path / "tune.json"))
    inst = W.lattice((12, 12, 12), periodic=True, couplings="pm1", fields="pm1_0", seed=31)
    R = 64
    h = isg.Handle([inst])
    kw = dict(max_sweeps=100, restarts=3)
    fam = h.autotune(R, **kw)
    assert fam in (isg.KERNEL_MSC, isg.KERNEL_TILE, isg.KERNEL_SWEEP)
    assert h.plan_kernel(R, **kw) == fam
    assert (tmp_path / "tune.json").exists()
    outs = []
    for k in (isg.KERNEL_AUTO, isg.KERNEL_MSC, isg.KERNEL_TILE, isg.KERNEL_SWEEP):
        r = h.local_search([8], R, kernel=k, **kw)
        torch.cuda.synchronize()
        outs.append((r.spins.cpu().numpy().copy(), r.energy.cpu().numpy().copy(), r.stats))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
        assert {k: v for k, v in o[2].items() if k != "launches"} == {
            k: v for k, v in outs[0][2].items() if k != "launches"}
    h.close()
    # a fresh handle of the same class reads the decision from the cache file
    h2 = isg.Handle([inst])
    assert h2.autotune(R, **kw) == fam
    h2.close()


@pytest.mark.parametrize("dims,R", [((16, 16, 16), 70), ((64, 64), 40), ((32, 32, 32), 40), ((128, 128), 33)])
def test_msc_lattice_cluster_split(dims, R):
    """Lattices whose replica groups are few are split over a 4-CTA cluster
    (distributed shared memory for the slab-boundary neighbours)."""
    inst = W.lattice(dims, periodic=True, couplings="pm1", fields="pm1_0", seed=sum(dims))
    _compare([inst], [sum(dims)], R, True, max_sweeps=200, restarts=4, kernel=isg.KERNEL_MSC)
    _compare([inst], [sum(dims) + 1], R, True, max_sweeps=3, restarts=1000, sweep_budget=17,
             kernel=isg.KERNEL_MSC)


def test_msc_lattice_cluster_mixed_sizes():
    """Instances of different sides in one cluster launch (per-tile slab sizes)."""
    insts = [W.lattice((32, 32, 32), periodic=True, couplings="pm1", fields="pm1_0", seed=41),
             W.lattice((16, 16, 16), periodic=True, couplings="pm1", seed=42)]
    _compare(insts, [41, 42], 45, True, max_sweeps=200, restarts=3, kernel=isg.KERNEL_MSC)


def test_kernel_timing_window():
    """ising_set_timing / ising_kernel_times: names of the kernels a family ran,
    positive device times, one timed group per launch, nothing recorded once
    the window is closed, and results unchanged by the events."""
    inst = W.sk(512, seed=90)
    R = 128
    h = isg.Handle([inst])
    ref = h.local_search([4], R, max_sweeps=200, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    sp_ref = ref.spins.cpu().numpy().copy()
    h.set_timing(True)
    for _ in range(2):
        res = h.local_search([4], R, max_sweeps=200, kernel=isg.KERNEL_DENSE_TC)
    kt = h.kernel_times()
    h.set_timing(False)
    assert np.array_equal(res.spins.cpu().numpy(), sp_ref)
    assert set(kt) == {"dense_tc_kernel", "dense_push_kernel", "dense_energy_tc"}, kt
    for name, (ms, launches) in kt.items():
        assert ms > 0.0 and launches == 2, (name, ms, launches)
    h.local_search([4], R, max_sweeps=200, kernel=isg.KERNEL_DENSE_TC)
    assert h.kernel_times() == kt or all(h.kernel_times()[k][1] == 2 for k in kt)
    h.close()
    lat = W.lattice((12, 12, 12), periodic=True, couplings="pm1", seed=91)
    h2 = isg.Handle([lat])
    h2.set_timing(True)
    h2.local_search([5], 64, max_sweeps=100, restarts=2, kernel=isg.KERNEL_SWEEP)
    h2.local_search([5], 64, max_sweeps=100, restarts=2, kernel=isg.KERNEL_TILE)
    kt2 = h2.kernel_times()
    assert kt2["sweep_chunk"][1] >= 1 and kt2["tile_kernel"][1] == 1
    h2.close()


# ----------------------------------------------------------- evaluated visits and the logic-op peak
@pytest.mark.parametrize("kernel", [isg.KERNEL_TILE, isg.KERNEL_MSC, isg.KERNEL_SWEEP, isg.KERNEL_PLAIN])
def test_evaluated_visits_counter(kernel):
    """ising_stats.evaluated: at most the visits (flip_evals), every visit of the
    fresh first sweeps at least (a descent's first sweep evaluates everything),
    equal to the visits for the family that never skips, and independent of
    whether the counters were requested twice (the search itself is unchanged)."""
    inst = W.lattice((16, 16, 16), periodic=True, couplings="pm1", fields="pm1_0", seed=93)
    R, restarts = 32, 3
    h = isg.Handle([inst])
    a = h.local_search([8], R, max_sweeps=100, restarts=restarts, kernel=kernel, stats=True)
    b = h.local_search([8], R, max_sweeps=100, restarts=restarts, kernel=kernel, stats=True)
    torch.cuda.synchronize()
    sa, sb = dict(a.stats), dict(b.stats)
    assert sa == sb
    assert sa["evaluated"] <= sa["flip_evals"]
    assert sa["evaluated"] >= sa["descents"] * inst.n  # first sweeps visit every spin of every replica
    if kernel == isg.KERNEL_PLAIN:
        assert sa["evaluated"] == sa["flip_evals"]
    else:
        assert sa["evaluated"] < sa["flip_evals"]  # later sweeps skip stable spins
    assert np.array_equal(a.spins.cpu().numpy(), b.spins.cpu().numpy())
    h.close()


def test_logic_peak_measurement():
    """ising_logic_peak: a positive issue rate of 32-bit logic ops, below 128
    lanes per SM per clock at the highest SM clock any GB300 runs (2.1 GHz), and
    repeatable to within a few percent."""
    p1 = isg.logic_peak()
    p2 = isg.logic_peak()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < p1 <= sms * 128 * 2.1e9
    assert abs(p1 - p2) <= 0.05 * max(p1, p2)


def test_multi_spin_word_width():
    """ising_logic_bits_rate: replica-bit logic operations per second on 32- and
    64-bit words.  A 64-bit logic op issues as two 32-bit ones, so the wider word
    does not raise the rate at which replica bits are processed (the reason the
    multi-spin-coded kernels use 32-bit words).  A two-input XOR issues at least
    as fast as the three-input lop3 and at most twice as fast (measured 1.86x:
    the denominator of the logic rooflines is the three-input rate)."""
    r32 = isg.logic_bits_rate(32)
    r64 = isg.logic_bits_rate(64)
    lop = isg.logic_peak()
    print(f"replica-bit ops/s: 32-bit words {r32:.4g}, 64-bit words {r64:.4g}; lop3 lane-ops/s {lop:.4g}")
    assert r32 > 0 and r64 > 0
    assert r64 <= 1.1 * r32, (r32, r64)
    assert 0.8 * lop * 32 <= r32 <= 2.2 * lop * 32, (r32, lop)
    with pytest.raises(RuntimeError):
        isg.logic_bits_rate(16)
