"""Host-side checks of the lattice index arithmetic the sweep kernels use.

The lazy FP32 visits on parity-coloured periodic lattices with an even side L
find the site of class position p without loading the class order: the two
classes hold the sites with even and odd coordinate sum in index order, so each
row of L sites holds L / 2 of either class and position p of class c is site
2 p + ((c + y + z) mod 2), y and z the coordinates of row 2 p / L.  Divisions by
L are done as (x m) >> k with k = 24 + ceil(log2 L) and m = ceil(2^k / L),
exact for x < 2^24.  These tests restate both in numpy and check them against
plain integer division and against the class order built from the colouring.
"""
import numpy as np
import pytest


def magic(L):
    lg = 0
    while (1 << lg) < L:  # ceil(log2 L)
        lg += 1
    k = 24 + lg
    return ((1 << k) + L - 1) // L, k


def div_magic(x, L):
    m, k = magic(L)
    return (x.astype(np.uint64) * np.uint64(m)) >> np.uint64(k)


@pytest.mark.parametrize("L", list(range(3, 130)) + [200, 255, 256, 300, 512, 1000, 1023, 1024, 4096])
def test_multiply_shift_division_is_exact(L):
    # every multiple of L below 2^24 and its two neighbours, plus the top of the range
    q = np.arange(0, (1 << 24) // L + 1, dtype=np.int64)
    x = np.concatenate([q * L - 1, q * L, q * L + L - 1, np.arange((1 << 24) - 4096, 1 << 24)])
    x = x[(x >= 0) & (x < (1 << 24))]
    assert np.array_equal(div_magic(x, L), (x // L).astype(np.uint64))


@pytest.mark.parametrize("dims", [(4, 4), (10, 10), (12, 12, 12), (100, 100), (16, 16, 16), (100, 100, 100)])
def test_parity_class_position_to_site(dims):
    L = dims[0]
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    colour = np.sum(np.stack(coords), axis=0) % 2
    for c in (0, 1):
        sites = idx[colour == c]  # class order: the class's sites in index order
        p = np.arange(len(sites), dtype=np.int64)
        p2 = 2 * p
        rho = div_magic(p2, L).astype(np.int64)
        z = div_magic(rho, L).astype(np.int64)
        y = rho - z * L
        j = p2 + ((c + y + z) & 1)
        assert np.array_equal(j, sites), (dims, c)
