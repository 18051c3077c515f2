"""Pins of the CPU oracle against facts the paper and mathematics fix.

Nothing here uses the GPU library.  Each test names what it pins:
  * Philox4x32-10 against its published known-answer vectors (SC'11);
  * the hyper-energy (Eq. 6) against the paper's printed N = 21 polynomial
    (Sec. VI, Fig. 7) and against (N - x y)^2 itself;
  * energies against exhaustive enumeration, the lower bound of Eq. 2, the
    closed-form ferromagnet ground state, gauge and global-flip invariance,
    and the move identity dE_i = 2 s_i f_i (Sec. IV gain);
  * descent results against the 1-flip local-minimum property, the even-step
    energy identity of integer couplings, a simultaneous-update restatement of
    the colour schedule, and the reduction of the colour schedule to the
    sequential one when every spin has its own colour;
  * FP32 field semantics against FP64 decisions (refresh every sweep makes them
    identical);
  * the FM-style passes (Fig. 3) against the local-minimum property and brute force;
  * branch and bound (Sec. III) and the transfer-matrix DP against brute force
    and against each other at sizes brute force cannot reach.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_spins(rng, n):
    return (rng.integers(0, 2, size=n) * 2 - 1).astype(np.int8)


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox(r[0:4], r[4:6]) == r[6:10]


def test_random_start_bits_and_independence():
    n = 1000
    s = oracle.random_start(n, 0x1234_5678_9ABC_DEF0, 3, 5, 7)
    assert set(np.unique(s)) <= {-1, 1}
    # bit mapping: spin i is bit (i mod 128) of the block-i//128 output
    out = oracle.philox([1, 5, 7, 3], [0x9ABCDEF0, 0x12345678])
    for t in range(128):
        assert s[128 + t] == (1 if (out[t // 32] >> (t % 32)) & 1 else -1)
    # different (r, k, b) give unrelated starts; balanced on average
    many = np.stack([oracle.random_start(4096, 99, b, r, k)
                     for b in range(2) for r in range(4) for k in range(4)])
    assert abs(many.mean()) < 0.02
    corr = np.corrcoef(many.astype(float))
    off = corr[~np.eye(len(corr), dtype=bool)]
    assert np.max(np.abs(off)) < 0.1


# --------------------------------------------------------------------------- energy
def _n21_instance(dtype):
    """N = 21 hyper-Ising instance read off Fig. 7: E = f - 210 with h_i = -c_i, J_e = -c_e."""
    terms = []
    with open(os.path.join(GOLDEN, "factoring_n21_fig7.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                vals = [int(x) for x in line.split()]
                terms.append((vals[0], tuple(vals[1:])))
    const = [c for c, m in terms if not m][0]
    h = np.zeros(3)
    edges = [(m, c) for c, m in terms if len(m) >= 2]
    for c, m in terms:
        if len(m) == 1:
            h[m[0]] = -c
    npdt = np.int8 if dtype == "i8" else np.float32
    ptr = np.cumsum([0] + [len(m) for m, _ in edges]).astype(np.int64)
    inst = W.Instance(n=3, row_ptr=np.zeros(4, np.int64), col=np.zeros(0, np.int32),
                      J=np.zeros(0, npdt), h=h.astype(npdt), hyper_ptr=ptr,
                      hyper_members=np.array([x for m, _ in edges for x in m], np.int32),
                      hyper_J=np.array([-c for _, c in edges], dtype=npdt), dtype=dtype)
    return inst, terms, const


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_energy_matches_fig7_factoring_polynomial(dtype):
    inst, terms, const = _n21_instance(dtype)
    found_factor = []
    for S in itertools.product([-1, 1], repeat=3):
        s = np.array(S, dtype=np.int8)
        f_printed = sum(c * np.prod([S[i] for i in m]) for c, m in terms)
        b = [(1 - x) // 2 for x in S]               # bit = (1 - S)/2, as Eq. 9 writes it
        x = 1 + 2 * b[0]
        y = 1 + 2 * b[2] + 4 * b[1]
        assert f_printed == (21 - x * y) ** 2       # the printed polynomial is Eq. 8
        assert oracle.energy(inst, s) == f_printed - const
        if f_printed == 0:
            found_factor.append((x, y))
    assert found_factor == [(3, 7)]
    E, arg, ng = oracle.bruteforce(inst)
    assert E == -const and list(arg) == [-1, -1, -1]
    done, Eb, _, _ = oracle.bnb(inst)
    assert done and Eb == -const


def test_energy_hand_example():
    # Triangle 0-1-2 with J01 = 2, J12 = -1, J02 = 3, h = (1, 0, -2), one 3-spin J_e = 1.
    u, v, w = np.array([0, 1, 0]), np.array([1, 2, 2]), np.array([2, -1, 3])
    rp, col, J = W.csr_from_edges(3, u, v, w, "i8")
    inst = W.Instance(n=3, row_ptr=rp, col=col, J=J, h=np.array([1, 0, -2], np.int8),
                      hyper_ptr=np.array([0, 3], np.int64),
                      hyper_members=np.array([0, 1, 2], np.int32),
                      hyper_J=np.array([1], np.int8), dtype="i8")
    # all +1: -(2 - 1 + 3) - 1 - (1 + 0 - 2) = -4 - 1 + 1 = -4
    assert oracle.energy(inst, np.array([1, 1, 1], np.int8)) == -4
    # (+1, -1, +1): bonds -(2*-1 + -1*-1 + 3*1) = -(-2 + 1 + 3) = -2; hyper -(1*-1) = 1;
    # fields -(1*1 + 0 + -2*1) = 1  -> total 0
    assert oracle.energy(inst, np.array([1, -1, 1], np.int8)) == 0


@pytest.mark.parametrize("dtype,seed", [("i8", 1), ("f32", 2), ("i8", 3), ("f32", 4)])
def test_energy_bruteforce_bound_and_flip_identity(dtype, seed):
    inst = W.random_graph(12, 3.0, seed, dtype=dtype, n_hyper=4, hyper_order=(2, 3, 4))
    rng = np.random.default_rng(seed)
    lb = oracle.lower_bound(inst)
    Es = []
    for bits in range(1 << inst.n):
        s = np.array([1 if (bits >> i) & 1 else -1 for i in range(inst.n)], np.int8)
        Es.append(oracle.energy(inst, s))
    Es = np.array(Es)
    assert Es.min() >= lb - 1e-9
    E, arg, ng = oracle.bruteforce(inst)
    assert abs(E - Es.min()) <= 1e-9 * (1 + abs(E))
    if dtype == "i8":
        assert ng == int(np.sum(Es == Es.min()))
    # dE_i = 2 s_i f_i for every spin of random configurations
    for _ in range(5):
        s = _rand_spins(rng, inst.n)
        f = oracle.local_fields(inst, s)
        E0 = oracle.energy(inst, s)
        for i in range(inst.n):
            t = s.copy()
            t[i] = -t[i]
            assert abs(oracle.energy(inst, t) - E0 - 2 * s[i] * f[i]) <= 1e-9 * (1 + abs(E0))


def test_ferromagnet_closed_form():
    inst = W.lattice((4, 4), periodic=True, couplings="ferro", seed=0)
    ones = np.ones(inst.n, np.int8)
    E_up = oracle.energy(inst, ones)
    assert E_up == -np.abs(inst.J.astype(float)).sum() / 2 == oracle.lower_bound(inst)
    assert oracle.energy(inst, -ones) == E_up
    E, arg, ng = oracle.bruteforce(inst)
    assert E == E_up and ng == 2
    assert oracle.transfer_matrix(inst, 4, 4, True, True) == E_up


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_gauge_and_global_flip_invariance(dtype):
    rng = np.random.default_rng(7)
    inst = W.random_graph(30, 4.0, 11, dtype=dtype, n_hyper=6, hyper_order=(2, 3, 4))
    tau = _rand_spins(rng, inst.n)
    # gauge transform: J'_ij = t_i t_j J_ij, h' = t h, J'_e = J_e prod t, s' = t s
    rows = np.repeat(np.arange(inst.n), np.diff(inst.row_ptr))
    Jg = (inst.J.astype(np.float64) * tau[rows] * tau[inst.col]).astype(inst.J.dtype)
    hg = (inst.h.astype(np.float64) * tau).astype(inst.h.dtype)
    hJg = inst.hyper_J.astype(np.float64).copy()
    for e in range(inst.n_hyper):
        hJg[e] *= np.prod(tau[inst.hyper_members[inst.hyper_ptr[e]:inst.hyper_ptr[e + 1]]])
    gauged = W.Instance(n=inst.n, row_ptr=inst.row_ptr, col=inst.col, J=Jg, h=hg,
                        hyper_ptr=inst.hyper_ptr, hyper_members=inst.hyper_members,
                        hyper_J=hJg.astype(inst.hyper_J.dtype), dtype=dtype)
    for _ in range(10):
        s = _rand_spins(rng, inst.n)
        a, b = oracle.energy(inst, s), oracle.energy(gauged, (tau * s).astype(np.int8))
        assert abs(a - b) <= 1e-9 * (1 + abs(a))
    # global flip: symmetric when h = 0 and all hyper-edges have even order
    even = W.random_graph(30, 4.0, 12, dtype=dtype, n_hyper=6, hyper_order=(2, 4), fields=False)
    odd = W.random_graph(30, 4.0, 13, dtype=dtype, n_hyper=6, hyper_order=(3,), fields=False)
    s = _rand_spins(rng, 30)
    assert abs(oracle.energy(even, s) - oracle.energy(even, -s)) <= 1e-9
    assert abs(oracle.energy(odd, s) - oracle.energy(odd, -s)) > 1e-6


# --------------------------------------------------------------------------- exact solvers
@pytest.mark.parametrize("dtype,seed", [("i8", 21), ("f32", 22), ("i8", 23), ("f32", 24)])
def test_bnb_equals_bruteforce(dtype, seed):
    inst = W.random_graph(18, 3.5, seed, dtype=dtype, n_hyper=5, hyper_order=(2, 3, 4))
    E, arg, _ = oracle.bruteforce(inst)
    done, Eb, argb, nodes = oracle.bnb(inst)
    assert done
    assert abs(Eb - E) <= 1e-9 * (1 + abs(E))
    assert abs(oracle.energy(inst, argb) - Eb) <= 1e-9 * (1 + abs(E))


@pytest.mark.parametrize("dims,periodic,coup", [((4, 5), False, "pm1"), ((4, 4), True, "gauss"),
                                               ((3, 6), True, "pm1"), ((5, 4), False, "gauss")])
def test_transfer_matrix_equals_bruteforce(dims, periodic, coup):
    inst = W.lattice(dims, periodic=periodic, couplings=coup, seed=5,
                     fields="pm1_0" if coup == "pm1" else "gauss")
    E, _, _ = oracle.bruteforce(inst)
    # spin index x + Lx*y: rows are y (dims[1]), columns x (dims[0])
    Etm = oracle.transfer_matrix(inst, dims[1], dims[0], periodic, periodic)
    assert abs(Etm - E) <= 1e-9 * (1 + abs(E))


@pytest.mark.parametrize("coup", ["pm1", "gauss"])
def test_bnb_equals_transfer_matrix_beyond_bruteforce(coup):
    # 6 x 6 open grid = 36 spins: out of reach for enumeration, exact by the DP
    inst = W.lattice((6, 6), periodic=False, couplings=coup, seed=9)
    Etm = oracle.transfer_matrix(inst, 6, 6, False, False)
    done, Eb, argb, nodes = oracle.bnb(inst, node_limit=200_000_000)
    assert done
    assert abs(Eb - Etm) <= 1e-9 * (1 + abs(Etm))


# --------------------------------------------------------------------------- descent
def _is_local_min(inst, s, tol=0.0):
    f = oracle.local_fields(inst, s)
    return bool(np.all(s.astype(float) * f >= -tol))


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_descent_returns_local_minima_and_stats(dtype):
    inst = W.random_graph(200, 4.0, 31, dtype=dtype, n_hyper=20, hyper_order=(3,))
    R, K = 6, 3
    spins, E, minima, st = oracle.descent(inst, 77, 0, R, max_sweeps=500, restarts=K,
                                          refresh_every=16)
    assert st["descents"] == R * K and st["minima"] == minima.sum() == R * K
    assert st["flip_evals"] == inst.n * st["sweeps"]
    for r in range(R):
        assert _is_local_min(inst, spins[r], tol=1e-4 if dtype == "f32" else 0.0)
        assert abs(oracle.energy(inst, spins[r]) - E[r]) <= 1e-9 * (1 + abs(E[r]))
        # keeping the best of K descents beats descent 0 alone
        s1, E1, _, _ = oracle.descent(inst, 77, 0, r + 1, max_sweeps=500, restarts=1,
                                      refresh_every=16)
        assert E[r] <= E1[r] + 1e-9


def test_descent_integer_energy_drops_by_even_steps():
    inst = W.lattice((8, 8, 8), periodic=True, couplings="pm1", fields="pm1_0", seed=3)
    R = 8
    spins, E, minima, st = oracle.descent(inst, 5, 0, R, max_sweeps=1000, restarts=1)
    E0 = np.array([oracle.energy(inst, oracle.random_start(inst.n, 5, 0, r, 0)) for r in range(R)])
    drop = E0 - E
    assert np.all(drop % 2 == 0)
    assert drop.sum() >= 2 * st["flips"]


def test_colour_schedule_equals_simultaneous_class_updates():
    inst = W.lattice((6, 6, 6), periodic=True, couplings="pm1", fields="pm1_0", seed=4)
    seed, R = 123, 3
    spins, E, _, st = oracle.descent(inst, seed, 2, R, max_sweeps=200, restarts=1)
    rows = np.repeat(np.arange(inst.n), np.diff(inst.row_ptr))
    Jm = np.zeros((inst.n, inst.n))
    Jm[rows, inst.col] = inst.J
    for r in range(R):
        s = oracle.random_start(inst.n, seed, 2, r, 0).astype(np.int64)
        for _ in range(200):
            flips = 0
            for c in (0, 1):
                f = Jm @ s + inst.h
                m = (inst.colour == c) & (s * f < 0)
                s[m] = -s[m]
                flips += int(m.sum())
            if flips == 0:
                break
        assert np.array_equal(s, spins[r])


def test_colour_schedule_reduces_to_sequential():
    inst = W.random_graph(60, 4.0, 41, dtype="f32", n_hyper=8, hyper_order=(3,))
    a = oracle.descent(inst, 9, 0, 4, max_sweeps=300, restarts=2, schedule=oracle.SCHED_SEQUENTIAL,
                       refresh_every=4)
    b = oracle.descent(inst, 9, 0, 4, max_sweeps=300, restarts=2, schedule=oracle.SCHED_COLOUR,
                       refresh_every=4, colour=np.arange(inst.n, dtype=np.int32))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[3] == b[3]


def test_fp32_fields_with_refresh_every_sweep_equal_fp64_decisions():
    inst = W.chimera(4, seed=3)
    a = oracle.descent(inst, 17, 0, 8, max_sweeps=500, restarts=2, refresh_every=1,
                       mode=oracle.MODE_F32)
    b = oracle.descent(inst, 17, 0, 8, max_sweeps=500, restarts=2, mode=oracle.MODE_F64)
    assert np.array_equal(a[0], b[0]) and a[3] == b[3]
    c = oracle.descent(inst, 17, 0, 8, max_sweeps=500, restarts=2, refresh_every=16,
                       mode=oracle.MODE_F32)
    assert np.mean(np.all(c[0] == b[0], axis=1)) >= 0.75
    assert np.allclose(c[1], b[1], rtol=0, atol=1e-2 * np.abs(b[1]).max())


def test_sweep_budget_and_cap():
    inst = W.lattice((8, 8), periodic=True, couplings="gauss", seed=8)
    spins, E, minima, st = oracle.descent(inst, 3, 0, 4, max_sweeps=3, restarts=1000,
                                          sweep_budget=40, refresh_every=16)
    assert st["sweeps"] == 4 * 40
    spins2, E2, minima2, st2 = oracle.descent(inst, 3, 0, 4, max_sweeps=1, restarts=1)
    assert st2["minima"] <= 4 and st2["sweeps"] == 4


def test_descent_reaches_ground_state_with_enough_restarts():
    inst = W.lattice((4, 4), periodic=True, couplings="pm1", seed=12)
    Egs, _, _ = oracle.bruteforce(inst)
    spins, E, minima, _ = oracle.descent(inst, 1, 0, 8, max_sweeps=100, restarts=64)
    assert np.all(E >= Egs)
    assert np.any(E == Egs)


# --------------------------------------------------------------------------- FM passes
@pytest.mark.parametrize("dtype,seed", [("i8", 51), ("f32", 52)])
def test_fm_passes_local_minimum_and_bruteforce(dtype, seed):
    inst = W.random_graph(16, 3.5, seed, dtype=dtype, n_hyper=3, hyper_order=(3,))
    Egs, _, _ = oracle.bruteforce(inst)
    hits = 0
    for k in range(40):
        s0 = oracle.random_start(inst.n, seed, 0, 0, k)
        s, E, passes = oracle.fm_search(inst, s0)
        assert passes >= 1
        assert E <= oracle.energy(inst, s0) + 1e-9
        assert E >= Egs - 1e-9
        assert _is_local_min(inst, s, tol=1e-6)
        hits += abs(E - Egs) <= 1e-9 * (1 + abs(Egs))
    assert hits >= 10


def _fm_bruteforce(inst, s0):
    """The passes of Fig. 3 with every gain taken as the difference of two full
    energies (Eq. 1 / Eq. 6): no gain heap, no incremental gain updates.  The
    largest gain among the unlocked spins moves (ties: lowest index), negative
    gains included; the pass keeps its earliest prefix strictly below every
    earlier energy (its start included); passes repeat while one improves."""
    n = inst.n
    s = np.array(s0, dtype=np.int8)
    E = oracle.energy(inst, s)
    passes = 0
    while True:
        passes += 1
        cur, Ecur = s.copy(), E
        locked = np.zeros(n, dtype=bool)
        best_E, best_s = E, s.copy()
        for _ in range(n):
            cand = []
            for i in range(n):
                if not locked[i]:
                    t = cur.copy()
                    t[i] = -t[i]
                    cand.append((-(Ecur - oracle.energy(inst, t)), i))
            _, i = min(cand)
            cur[i] = -cur[i]
            locked[i] = True
            Ecur = oracle.energy(inst, cur)
            if Ecur < best_E:
                best_E, best_s = Ecur, cur.copy()
        if best_E < E:
            s, E = best_s, best_E
            continue
        return s, E, passes


@pytest.mark.parametrize("seed", [61, 62, 63, 64])
def test_fm_passes_match_bruteforce_passes(seed):
    """Integer instances (exact gains): the oracle's heap and incremental
    updates make exactly the moves of the brute-force passes."""
    inst = W.random_graph(13, 3.5, seed, dtype="i8", n_hyper=4, hyper_order=(3, 4), int_range=2)
    for k in range(12):
        s0 = oracle.random_start(inst.n, seed, 0, 0, k)
        s_o, E_o, p_o = oracle.fm_search(inst, s0)
        s_b, E_b, p_b = _fm_bruteforce(inst, s0)
        assert np.array_equal(s_o, s_b) and E_o == E_b and p_o == p_b, (k, p_o, p_b, E_o, E_b)


def test_fm_passes_beat_greedy_descent_on_average():
    inst = W.lattice((16, 16), periodic=True, couplings="gauss", seed=2)
    R = 16
    _, Ed, _, _ = oracle.descent(inst, 4, 0, R, max_sweeps=1000, restarts=1, mode=oracle.MODE_F64)
    Efm = [oracle.fm_search(inst, oracle.random_start(inst.n, 4, 0, r, 0))[1] for r in range(R)]
    assert np.mean(Efm) < np.mean(Ed)


# --------------------------------------------------------------------------- colouring
def test_greedy_colouring():
    lat = W.lattice((6, 6), periodic=True, couplings="pm1", seed=0)
    col, nc = oracle.greedy_colouring(lat)
    assert nc == 2 and oracle.colouring_valid(lat, col)
    assert np.array_equal(col, lat.colour)
    ch = W.chimera(5, seed=1)
    col, nc = oracle.greedy_colouring(ch)
    assert oracle.colouring_valid(ch, col) and nc >= 3
    bad = col.copy()
    bad[ch.col[0]] = bad[0]
    assert not oracle.colouring_valid(ch, bad)


@pytest.mark.parametrize("seed,scale", [(3, 1), (11, 1), (29, 4096)])
def test_fp32_incremental_fields_exact_on_integer_couplings(seed, scale):
    """The FP32 path's incremental field updates (every flip adds +/-2 J to the
    neighbours' stored fields and hyper-edge terms, refreshed only at the start
    of a descent) against the exact integer path: with integer couplings and
    fields, scaled so that every sum stays below 2^24, FP32 arithmetic is exact,
    so both must take the same decisions move for move - same spins, energies,
    minima and work counters.  A dropped term, a wrong sign or a wrong index in
    the FP32 update would show here."""
    gi = W.random_graph(120, 4.0, seed, dtype="i8", n_hyper=12, hyper_order=(2, 3, 4))
    gf = W.Instance(n=gi.n, row_ptr=gi.row_ptr, col=gi.col, J=(gi.J.astype(np.float32) * scale),
                    h=None if gi.h is None else gi.h.astype(np.float32) * scale,
                    hyper_ptr=gi.hyper_ptr, hyper_members=gi.hyper_members,
                    hyper_J=None if gi.hyper_J is None else gi.hyper_J.astype(np.float32) * scale,
                    dtype="f32")
    a = oracle.descent(gi, 5 + seed, 0, 16, max_sweeps=300, restarts=3, mode=oracle.MODE_INT)
    b = oracle.descent(gf, 5 + seed, 0, 16, max_sweeps=300, restarts=3, refresh_every=0,
                       mode=oracle.MODE_F32)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[2], b[2]) and a[3] == b[3]
    assert np.array_equal(a[1] * scale, b[1])


@pytest.mark.parametrize("n,seed", [(24, 3), (37, 8)])
def test_sequential_descent_on_dense_instance_equals_plain_loop(n, seed):
    """The sequential (index-order) schedule on a dense instance, as the dense
    GPU path runs it, restated as a plain loop (Sec. IV): each restart starts
    from the pinned Philox start, visits spins 0..n-1 and flips a spin whose
    field points against it, until a sweep flips nothing; the best energy
    over the converged restarts is returned.  Couplings and fields are
    multiples of 1/8, so FP64 fields and energies are exact and the two must
    agree on spins, energies, minima counts and every work counter."""
    inst = W.sk_eighths(n, seed)
    J = inst.J_dense.astype(np.float64)
    h = inst.h.astype(np.float64)
    R, K, cap = 5, 3, 100
    so, Eo, mo, sto = oracle.descent(inst, 77, 0, R, max_sweeps=cap, restarts=K,
                                     schedule=oracle.SCHED_SEQUENTIAL, mode=oracle.MODE_F64)
    tot = dict(flip_evals=0, flips=0, minima=0, descents=0, sweeps=0)
    for r in range(R):
        best, bestE, minima, last = None, None, 0, None
        for k in range(K):
            s = oracle.random_start(n, 77, 0, r, k).astype(np.float64)
            tot["descents"] += 1
            converged = False
            for _ in range(cap):
                flips = 0
                for i in range(n):
                    f = J[i] @ s + h[i]
                    if s[i] * f < 0:
                        s[i] = -s[i]
                        flips += 1
                tot["sweeps"] += 1
                tot["flip_evals"] += n
                tot["flips"] += flips
                if flips == 0:
                    converged = True
                    break
            E = -(0.5 * s @ J @ s + h @ s)
            last = (s.copy(), E)
            if converged:
                minima += 1
                tot["minima"] += 1
                if bestE is None or E < bestE:
                    best, bestE = s.copy(), E
        sr, Er = (best, bestE) if minima else last
        assert np.array_equal(so[r], sr.astype(np.int8)) and Eo[r] == Er and mo[r] == minima
    assert sto == tot
