"""The allocation-free energy entry point against ising_energy and the oracle.

ising_energy_noalloc serves callers that cannot allocate device memory (their
pool allocator owns the device, or a cudaMalloc's implicit device-wide
synchronisation is not acceptable to them).  On two consecutive calls that
reuse its fixed scratch array it must return the energies the handle-based
ising_energy returns for the same configurations, and the CPU oracle's FP64
energies (bit-exact for int8 couplings, 1e-12 relative for FP32 ones); it must
refuse sizes beyond that array.  This file is collected last on purpose; it
also passes when run on its own.
"""
import numpy as np
import pytest

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
    import oracle
    oracle.build()


@pytest.mark.parametrize("kind", ["f32", "i8"])
def test_noalloc_energy_matches_handle_energy_twice(kind):
    if kind == "f32":
        inst = W.random_graph(9000, 5.0, 3, dtype="f32")
    else:
        inst = W.lattice((24, 24, 24), periodic=True, couplings="pm1", fields="pm1_0", seed=4)
    R = 6
    h = isg.Handle([inst])
    dev = torch.device("cuda", 0)
    npdt = torch.int8 if kind == "i8" else torch.float32
    row_ptr = torch.from_numpy(inst.row_ptr.astype(np.int64)).to(dev)
    col = torch.from_numpy(inst.col.astype(np.int32)).to(dev)
    J = torch.from_numpy(inst.J).to(dev)
    hh = torch.from_numpy(inst.h).to(dev)
    import oracle
    oi = oracle.OracleInstance(inst)
    rng = np.random.default_rng(0)
    for call in range(2):
        host_spins = (rng.integers(0, 2, size=(R, inst.n)) * 2 - 1).astype(np.int8)
        spins = torch.from_numpy(host_spins.reshape(-1)).to(dev)
        ref = h.energy(spins, R).view(R)
        out = torch.full((R,), float("nan"), dtype=torch.float64, device=dev)
        code = isg.energy_noalloc(row_ptr, col, J, hh, spins, R, out)
        assert code == 0, isg.status_string(code)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = oracle.energies(oi, host_spins)
        if kind == "i8":
            assert torch.equal(out, ref)
            assert np.array_equal(got, want)
        else:
            np.testing.assert_allclose(got, ref.cpu().numpy(), rtol=1e-12, atol=1e-9)
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    inst = W.lattice((16, 16), periodic=True, couplings="pm1", seed=1)
    dev = torch.device("cuda", 0)
    row_ptr = torch.from_numpy(inst.row_ptr).to(dev)
    col = torch.from_numpy(inst.col).to(dev)
    J = torch.from_numpy(inst.J).to(dev)
    R = 65537  # one chunk per replica: one more partial sum than the array holds
    spins = torch.ones(R * inst.n, dtype=torch.int8, device=dev)
    out = torch.empty(R, dtype=torch.float64, device=dev)
    assert isg.energy_noalloc(row_ptr, col, J, None, spins, R, out) == 6
