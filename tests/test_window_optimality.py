"""Window check of local-search results (Sec. V): branch and bound over a
window of adjacent spins with every other spin held at the result's value.
A result is window-optimal when no assignment of the window lowers the
energy.  The paper reports that its local search's results were never
improved this way on 25-49-spin windows; on these seeded ±J lattices the
pass-based search (Fig. 3) leaves few improvable windows and greedy descent
many, which the tests check, with the counts in the messages.

CPU tests use the oracle's searches; the GPU test runs the same statistic on
the library's searches, which return the oracle's states."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _window(L, x0, y0, w):
    return [((x0 + a) % L) + L * ((y0 + b) % L) for b in range(w) for a in range(w)]


def test_window_instance_folds_every_term():
    """E(state) = E_window(window spins) + const for every assignment of the
    window, the rest held fixed (brute force over a 12-spin window of a graph
    with 3- and 4-spin hyper-edges)."""
    inst = W.random_graph(40, 4.0, 301, dtype="i8", n_hyper=12, hyper_order=(3, 4), int_range=2)
    rng = np.random.default_rng(302)
    s = rng.choice(np.array([-1, 1], dtype=np.int8), size=inst.n)
    members = sorted(rng.choice(inst.n, size=12, replace=False).tolist())
    sub, const = oracle.window_instance(inst, s, members)
    for _ in range(64):
        w = rng.choice(np.array([-1, 1], dtype=np.int8), size=len(members))
        full = s.copy()
        full[members] = w
        assert oracle.energy(inst, full) == oracle.energy(sub, w) + const


def _improvable(inst, s, windows):
    count = 0
    for m in windows:
        sub, _ = oracle.window_instance(inst, s, m)
        done, E_opt, _, _ = oracle.bnb(sub)
        assert done
        if E_opt < oracle.energy(sub, s[m]):
            count += 1
    return count


L, WSIDE, STARTS, SEED = 16, 5, 6, 11


def _setup():
    inst = W.lattice((L, L), periodic=True, couplings="pm1", seed=7)
    windows = [_window(L, x0, y0, WSIDE) for x0 in range(0, L, WSIDE) for y0 in range(0, L, WSIDE)]
    return inst, windows


def test_pass_search_results_are_rarely_window_improvable():
    inst, windows = _setup()
    fm = gd = 0
    for r in range(STARTS):
        s_fm, _, _ = oracle.fm_search(inst, oracle.random_start(inst.n, SEED, 0, r, 0))
        fm += _improvable(inst, s_fm, windows)
    s_gd, _, _, _ = oracle.descent(inst, SEED, 0, STARTS, max_sweeps=1000, restarts=1,
                                   schedule=oracle.SCHED_SEQUENTIAL)
    for r in range(STARTS):
        gd += _improvable(inst, s_gd[r], windows)
    total = STARTS * len(windows)
    assert fm * 4 < gd, f"improvable windows: pass-based {fm}/{total}, greedy descent {gd}/{total}"
    assert fm <= total // 10, f"improvable windows: pass-based {fm}/{total}, greedy descent {gd}/{total}"


@pytest.mark.gpu
def test_window_statistic_on_gpu_results():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    isg = pytest.importorskip("paper_0912_3912_gb300")
    from paper_0912_3912_gb300 import build as B
    B.build()
    inst, windows = _setup()
    h = isg.Handle([inst])
    sp, _, _, _ = h.fm_search([SEED], STARTS, restarts=1)
    res = h.local_search([SEED], STARTS, max_sweeps=1000, restarts=1, schedule=isg.SCHED_SEQUENTIAL)
    torch.cuda.synchronize()
    s_fm = h.spins_of(sp, 0, STARTS).cpu().numpy()
    s_gd = h.spins_of(res.spins, 0, STARTS).cpu().numpy()
    h.close()
    fm = sum(_improvable(inst, s_fm[r], windows) for r in range(STARTS))
    gd = sum(_improvable(inst, s_gd[r], windows) for r in range(STARTS))
    fm_o = sum(_improvable(inst, oracle.fm_search(inst, oracle.random_start(inst.n, SEED, 0, r, 0))[0], windows)
               for r in range(STARTS))
    assert fm == fm_o
    assert fm * 4 < gd, (fm, gd)
