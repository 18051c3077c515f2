"""Failure paths, exercised without faulting the GPU.

* Host-injected faults (ISING_FAULT): an allocation that fails part-way
  through ising_create returns ISING_ERR_OOM and leaves no device memory
  behind; a failed launch returns ISING_ERR_CUDA and the handle stays usable.
* A device-side bounded wait that runs out: on the dense tensor-core path one
  CTA waits, with a 20 us limit, on a barrier that nothing completes; the call
  returns ISING_ERR_TIMEOUT, the context stays usable, and the next search on
  the same handle gives the same results as before.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

isg = pytest.importorskip("paper_0912_3912_gb300")

ERR_OOM, ERR_CUDA, ERR_TIMEOUT = 7, 8, 9


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0912_3912_gb300 import build as B
    B.build()


def test_injected_allocation_failures_leave_nothing_behind(monkeypatch):
    inst = W.random_graph(300, 4.0, 61, dtype="f32", n_hyper=20, hyper_order=(3,))
    h = isg.Handle([inst])
    h.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 3, 7, 12):
        monkeypatch.setenv("ISING_FAULT", f"alloc:{k}")
        with pytest.raises(isg.IsingError) as ei:
            isg.Handle([inst])
        assert ei.value.code == ERR_OOM
    monkeypatch.delenv("ISING_FAULT")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) <= 4 << 20, (free0, free1)
    h = isg.Handle([inst])
    res = h.local_search([7], 32, max_sweeps=200, restarts=2)
    torch.cuda.synchronize()
    assert res.minima.cpu().numpy().sum() > 0
    h.close()


def test_injected_launch_failure_leaves_the_handle_usable(monkeypatch):
    inst = W.lattice((8, 8), periodic=True, couplings="pm1", seed=62)
    h = isg.Handle([inst])
    ref = h.local_search([3], 32, max_sweeps=100, restarts=2)
    torch.cuda.synchronize()
    sp_ref = ref.spins.cpu().numpy().copy()
    monkeypatch.setenv("ISING_FAULT", "launch")
    with pytest.raises(isg.IsingError) as ei:
        h.local_search([3], 32, max_sweeps=100, restarts=2)
    assert ei.value.code == ERR_CUDA
    monkeypatch.delenv("ISING_FAULT")
    again = h.local_search([3], 32, max_sweeps=100, restarts=2)
    torch.cuda.synchronize()
    assert np.array_equal(again.spins.cpu().numpy(), sp_ref)
    h.close()


def test_device_wait_that_runs_out_returns_timeout(monkeypatch):
    inst = W.sk(512, seed=63)
    R = 256  # two 4-CTA clusters: the stalled one fails, the other completes
    h = isg.Handle([inst])
    ref = h.local_search([5], R, max_sweeps=300, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    sp_ref = ref.spins.cpu().numpy().copy()
    E_ref = ref.energy.cpu().numpy().copy()
    monkeypatch.setenv("ISING_FAULT", "device_timeout")
    with pytest.raises(isg.IsingError) as ei:
        h.local_search([5], R, max_sweeps=300, kernel=isg.KERNEL_DENSE_TC)
    assert ei.value.code == ERR_TIMEOUT
    monkeypatch.delenv("ISING_FAULT")
    assert torch.ones(1024, device="cuda").sum().item() == 1024.0  # the context still works
    again = h.local_search([5], R, max_sweeps=300, kernel=isg.KERNEL_DENSE_TC)
    torch.cuda.synchronize()
    assert np.array_equal(again.spins.cpu().numpy(), sp_ref)
    assert np.array_equal(again.energy.cpu().numpy(), E_ref)
    h.close()
