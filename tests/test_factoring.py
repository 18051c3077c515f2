"""Factoring instances (Sec. VI, Eqs. 7-9).

CPU: the generator reproduces Fig. 7's printed objective for N = 21, the
ground states of small instances (brute force) are exactly the factorisations,
and without the 3- and 4-spin terms N = 21 is still factored while 35 is not,
as the paper reports (the wrong products it prints for 35 and 91 come from
another encoding and are not reproduced).  The paper's numbers 612171 and
580003 have coefficients of up to 2^37 (sums below 2^44): FP64 instances,
exact, their brute-force ground states are the factorisations.  GPU: from
random starts the pass-based search (Fig. 3) reaches a factorisation at least
as often as greedy descent, with the oracle's states; on the paper's numbers
the FP64 search matches the oracle move for move, and the fraction of single
starts that factor is measured (the paper: 0.025 and 0.005)."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SMALL = [(21, 1, 2), (35, 2, 2), (143, 3, 3), (899, 4, 4), (3599, 5, 5)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _printed_fig7():
    terms = {}
    with open(os.path.join(GOLDEN, "factoring_n21_fig7.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                vals = [int(x) for x in line.split()]
                terms[tuple(vals[1:])] = vals[0]
    return terms


def test_generator_reproduces_fig7():
    inst = W.factoring(21, 1, 2)
    printed = _printed_fig7()
    got = {(): inst.meta["c0"]}
    for i in range(inst.n):
        if inst.h[i] != 0:
            got[(i,)] = -int(inst.h[i])
    for i in range(inst.n):
        for k in range(int(inst.row_ptr[i]), int(inst.row_ptr[i + 1])):
            j = int(inst.col[k])
            if j > i:
                got[(i, j)] = -int(inst.J[k])
    for e in range(len(inst.hyper_J)):
        mem = tuple(int(x) for x in inst.hyper_members[inst.hyper_ptr[e]:inst.hyper_ptr[e + 1]])
        got[mem] = -int(inst.hyper_J[e])
    assert got == printed


@pytest.mark.parametrize("N,nx,ny", SMALL)
def test_ground_states_are_the_factorisations(N, nx, ny):
    inst = W.factoring(N, nx, ny)
    E, arg, n_ground = oracle.bruteforce(inst)
    assert E == -inst.meta["c0"]
    x, y = W.factoring_decode(inst, arg)
    assert x * y == N and x > 1 and y > 1
    # every configuration's energy is (N - x y)^2 - c0
    rng = np.random.default_rng(N)
    for _ in range(32):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=inst.n)
        x, y = W.factoring_decode(inst, s)
        assert oracle.energy(inst, s) == (N - x * y) ** 2 - inst.meta["c0"]


def test_without_hyper_couplings():
    """Dropping the 3- and 4-spin terms: 21 is still factored, 35 is not."""
    for N, nx, ny, factored in ((21, 1, 2, True), (35, 2, 2, False)):
        inst = W.factoring(N, nx, ny, hyper=False)
        _, arg, _ = oracle.bruteforce(inst)
        x, y = W.factoring_decode(inst, arg)
        assert (x * y == N) == factored, (N, x, y)


def test_wide_coefficients_take_fp64():
    """Coefficients beyond FP32's exact integers: FP64 instances (exact below
    2^53), and an explicit FP32 request is refused."""
    with pytest.raises(ValueError):
        W.factoring(10403, 6, 6, dtype="f32")
    inst = W.factoring(10403, 6, 6)
    assert inst.dtype == "f64" and inst.meta["exact"]
    wide = W.factoring(10185081163, 16, 16)
    assert wide.dtype == "f64" and not wide.meta["exact"]


@pytest.mark.parametrize("N", [612171, 580003])
def test_paper_numbers_ground_states_and_energies(N):
    """The paper's 612171 and 580003 with 10-bit and 11-bit odd factors: the
    brute-force ground state decodes to a factorisation at energy -c0, and
    every configuration's FP64 energy is exactly (N - x y)^2 - c0."""
    inst = W.factoring(N, 9, 10)
    assert inst.dtype == "f64" and inst.meta["exact"] and inst.n == 19
    E, arg, _ = oracle.bruteforce(inst)
    assert E == -inst.meta["c0"]
    x, y = W.factoring_decode(inst, arg)
    assert x * y == N and x > 1 and y > 1
    rng = np.random.default_rng(N)
    for _ in range(64):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=inst.n)
        x, y = W.factoring_decode(inst, s)
        assert oracle.energy(inst, s) == (N - x * y) ** 2 - inst.meta["c0"]


@pytest.mark.gpu
def test_success_from_random_starts_on_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    isg = pytest.importorskip("paper_0912_3912_gb300")
    from paper_0912_3912_gb300 import build as B
    B.build()
    R, seed = 2048, 5
    for N, nx, ny in SMALL[2:]:
        inst = W.factoring(N, nx, ny)
        h = isg.Handle([inst])
        sp, E_fm, _, _ = h.fm_search([seed], R, restarts=1)
        res = h.local_search([seed], R, max_sweeps=1000, restarts=1, schedule=isg.SCHED_SEQUENTIAL)
        torch.cuda.synchronize()
        target = -inst.meta["c0"]
        fm = float(np.mean(E_fm[0].cpu().numpy() == target))
        gd = float(np.mean(res.energy[0].cpu().numpy() == target))
        s_fm = h.spins_of(sp, 0, R).cpu().numpy()
        h.close()
        for r in range(0, R, 256):  # the oracle's states, sampled
            s_o, _, _ = oracle.fm_search(inst, oracle.random_start(inst.n, seed, 0, r, 0))
            assert np.array_equal(s_fm[r], s_o)
        print(f"N={N}: pass-based search {fm:.4f}, greedy descent {gd:.4f} of {R} starts reach a factorisation")
        assert fm >= gd and fm > 0


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    isg = pytest.importorskip("paper_0912_3912_gb300")
    from paper_0912_3912_gb300 import build as B
    B.build()
    return torch, isg


def _successes(inst, spins):
    N = inst.meta["N"]
    hits = 0
    for s in spins:
        x, y = W.factoring_decode(inst, s)
        hits += x * y == N and x > 1 and y > 1
    return hits


@pytest.mark.gpu
@pytest.mark.parametrize("N", [612171, 580003])
def test_paper_numbers_on_gpu(N):
    """FP64 instances of the paper's numbers: the pass-based search matches the
    oracle move for move (spins, pass counts, energies; exact arithmetic) on
    sampled starts, plain descent (FP64 fields) matches the oracle's FP64
    descent, and the fraction of single random starts that factor N is
    measured over 8192 starts."""
    torch, isg = _gpu()
    inst = W.factoring(N, 9, 10)
    seed, R = 11, 8192
    h = isg.Handle([inst])
    sp, E, P, _ = h.fm_search([seed], R, restarts=1)
    res = h.local_search([seed], 256, max_sweeps=1000, restarts=1, kernel=isg.KERNEL_PLAIN)
    torch.cuda.synchronize()
    s_fm = h.spins_of(sp, 0, R).cpu().numpy()
    E_fm, P_fm = E[0].cpu().numpy(), P[0].cpu().numpy()
    for r in range(0, R, 512):
        s_o, E_o, p_o = oracle.fm_search(inst, oracle.random_start(inst.n, seed, 0, r, 0))
        assert np.array_equal(s_fm[r], s_o) and P_fm[r] == p_o and E_fm[r] == E_o
    s_d, E_d, _, _ = oracle.descent(inst, seed, 0, 256, max_sweeps=1000, restarts=1)
    assert np.array_equal(h.spins_of(res.spins, 0, 256).cpu().numpy(), s_d)
    assert np.array_equal(res.energy[0].cpu().numpy(), E_d)
    frac = _successes(inst, s_fm) / R
    frac_d = _successes(inst, h.spins_of(res.spins, 0, 256).cpu().numpy()) / 256
    h.close()
    print(f"N={N}: pass-based search factors from {frac:.4f} of {R} single starts "
          f"(greedy descent {frac_d:.4f} of 256)")
    assert frac > 0.0


@pytest.mark.gpu
def test_10185081163_with_15000_starts():
    """10185081163 = 100511 x 101333 with 17-bit odd factors: coefficients up
    to 2^65 do not fit FP64 exactly, so the instance is the FP64-rounded one
    (as in an FP64 program); both implementations take the same FP64 steps,
    so the GPU's states equal the oracle's on sampled starts.  15,000 single
    starts, as in the paper's run; the number that factor is reported."""
    torch, isg = _gpu()
    N = 10185081163
    inst = W.factoring(N, 16, 16)
    seed, R = 13, 15000
    h = isg.Handle([inst])
    sp, E, P, _ = h.fm_search([seed], R, restarts=1)
    torch.cuda.synchronize()
    s_fm = h.spins_of(sp, 0, R).cpu().numpy()
    E_fm = E[0].cpu().numpy()
    for r in (0, 1, 4999, 14999):
        s_o, E_o, _ = oracle.fm_search(inst, oracle.random_start(inst.n, seed, 0, r, 0))
        assert np.array_equal(s_fm[r], s_o) and E_fm[r] == E_o
    hits = _successes(inst, s_fm)
    h.close()
    print(f"N={N}: {hits} of {R} single starts reach 100511 x 101333")
