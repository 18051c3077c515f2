"""Seeded synthetic spin-glass instances.

This module only builds inputs: coupling graphs in symmetric CSR form, fields,
hyper-edges and lattice checkerboard colourings, drawn from the distributions the
paper uses (Sec. II: Gaussian couplings N(0,1) or +/-1 bimodal; Sec. VI:
hyper-couplings).  It holds none of the method's arithmetic (no energies, fields,
gains or descents), so both the GPU library's tests and the CPU oracle can use
it without sharing any of the method with each other.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) for deriving seeds."""
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


@dataclasses.dataclass
class Instance:
    """One instance: symmetric CSR couplings (or a dense matrix), fields, hyper-edges."""

    n: int
    row_ptr: Optional[np.ndarray]          # int64 [n+1]
    col: Optional[np.ndarray]              # int32 [nnz]
    J: Optional[np.ndarray]                # int8, float32 or float64 [nnz]
    h: Optional[np.ndarray] = None         # same dtype as J [n]
    hyper_ptr: Optional[np.ndarray] = None     # int64 [n_hyper+1]
    hyper_members: Optional[np.ndarray] = None  # int32
    hyper_J: Optional[np.ndarray] = None       # same dtype as J [n_hyper]
    colour: Optional[np.ndarray] = None    # int32 [n]
    J_dense: Optional[np.ndarray] = None   # float32 [n, n]
    dtype: str = "f32"                     # "i8", "f32" or "f64"
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_hyper(self) -> int:
        return 0 if self.hyper_ptr is None else len(self.hyper_ptr) - 1

    @property
    def nnz(self) -> int:
        return 0 if self.row_ptr is None else int(self.row_ptr[-1])


def _np_dtype(dtype: str):
    return {"i8": np.int8, "f32": np.float32, "f64": np.float64}[dtype]


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray, dtype: str):
    """Symmetric CSR (rows sorted by column) from undirected edges u-v of weight w."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w)
    if np.any(u == v):
        raise ValueError("self loop")
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    vals = np.concatenate([w, w]).astype(_np_dtype(dtype))
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if len(rows) > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if np.any(dup):
            raise ValueError("repeated edge")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int64)
    return row_ptr, cols.astype(np.int32), vals


def _draw(rng: np.random.Generator, kind: str, size, scale: float = 1.0):
    if kind == "pm1":
        return (rng.integers(0, 2, size=size) * 2 - 1).astype(np.int8)
    if kind == "gauss":
        return (rng.standard_normal(size) * scale).astype(np.float32)
    if kind == "ferro":
        return np.ones(size, dtype=np.int8)
    raise ValueError(kind)


def lattice(dims: Sequence[int], periodic: bool = True, couplings: str = "pm1",
            fields: Optional[str] = None, seed: int = 0, field_scale: float = 1.0) -> Instance:
    """Hypercubic lattice, spin index = x0 + L0*(x1 + L1*(x2 ...)).

    couplings: "pm1" (+/-1 with probability 1/2 each, int8), "gauss" (N(0,1),
    float32) or "ferro" (all +1, int8).  fields: None, "pm1_0" (uniform in
    {-1, 0, +1}, int8) or "gauss" (N(0, field_scale), float32).  The colouring is
    the checkerboard (sum of coordinates mod 2) when it is proper.
    """
    dims = [int(d) for d in dims]
    if periodic and min(dims) < 3:
        raise ValueError("periodic lattices need every side >= 3")
    n = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    us, vs = [], []
    stride = 1
    for a, d in enumerate(dims):
        c = coords[a]
        if periodic:
            nb = idx + ((c + 1) % d - c) * stride
            us.append(idx)
            vs.append(nb)
        else:
            keep = c + 1 < d
            us.append(idx[keep])
            vs.append(idx[keep] + stride)
        stride *= d
    u = np.concatenate(us)
    v = np.concatenate(vs)
    dtype = "f32" if couplings == "gauss" or fields == "gauss" else "i8"
    w = _draw(rng, couplings, len(u))
    row_ptr, col, J = csr_from_edges(n, u, v, w, dtype)
    h = None
    if fields == "pm1_0":
        h = (rng.integers(0, 3, size=n) - 1).astype(np.int8)
    elif fields == "gauss":
        h = (rng.standard_normal(n) * field_scale).astype(np.float32)
    if h is not None:
        h = h.astype(_np_dtype(dtype))
    colour = None
    if not periodic or all(d % 2 == 0 for d in dims):
        colour = (np.sum(np.stack(coords), axis=0) % 2).astype(np.int32)
    return Instance(n=n, row_ptr=row_ptr, col=col, J=J, h=h, colour=colour, dtype=dtype,
                    meta={"kind": "lattice", "dims": dims, "periodic": periodic})


def chimera(side: int, seed: int = 0, h_scale: float = 0.1, k_scale: float = 0.5,
            triples: bool = True) -> Instance:
    """Grid of side x side K4,4 unit cells (open boundaries), 8*side^2 spins.

    Inside a cell, each of the 4 spins of side 0 couples to the 4 spins of side 1.
    Side-0 spin k couples to side-0 spin k of the cells above and below; side-1
    spin k to side-1 spin k of the cells left and right.  J ~ N(0,1),
    h ~ N(0, h_scale), and one 3-spin hyper-coupling K ~ N(0, k_scale) per cell on
    a uniformly drawn triple of the cell's 8 spins.  Float32.
    """
    rng = np.random.default_rng(seed)

    def sid(r, c, s, k):
        return ((r * side + c) * 2 + s) * 4 + k

    us, vs = [], []
    for r in range(side):
        for c in range(side):
            for a in range(4):
                for b in range(4):
                    us.append(sid(r, c, 0, a))
                    vs.append(sid(r, c, 1, b))
            for k in range(4):
                if r + 1 < side:
                    us.append(sid(r, c, 0, k))
                    vs.append(sid(r + 1, c, 0, k))
                if c + 1 < side:
                    us.append(sid(r, c, 1, k))
                    vs.append(sid(r, c + 1, 1, k))
    n = 8 * side * side
    u = np.array(us, dtype=np.int64)
    v = np.array(vs, dtype=np.int64)
    w = _draw(rng, "gauss", len(u))
    row_ptr, col, J = csr_from_edges(n, u, v, w, "f32")
    h = _draw(rng, "gauss", n, h_scale)
    hyper_ptr = hyper_members = hyper_J = None
    if triples:
        members = []
        for cell in range(side * side):
            trip = np.sort(rng.choice(8, size=3, replace=False)) + cell * 8
            members.append(trip)
        hyper_members = np.concatenate(members).astype(np.int32)
        hyper_ptr = np.arange(0, 3 * side * side + 1, 3, dtype=np.int64)
        hyper_J = _draw(rng, "gauss", side * side, k_scale)
    return Instance(n=n, row_ptr=row_ptr, col=col, J=J, h=h, hyper_ptr=hyper_ptr,
                    hyper_members=hyper_members, hyper_J=hyper_J, dtype="f32",
                    meta={"kind": "chimera", "side": side})


def chimera_batch(count: int, side_lo: int, side_hi: int, seed: int) -> list:
    """`count` chimera instances with cell-grid side uniform in [side_lo, side_hi]."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    return [chimera(int(s), seed=splitmix64(seed + b)) for b, s in enumerate(sides)]


def sk(n: int, seed: int = 0) -> Instance:
    """Sherrington-Kirkpatrick: J_ij ~ N(0,1)/sqrt(n), symmetric, zero diagonal, h = 0."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) / np.sqrt(n)
    upper = np.triu(a, 1)
    Jd = (upper + upper.T).astype(np.float32)
    return Instance(n=n, row_ptr=None, col=None, J=None, J_dense=Jd, dtype="f32",
                    meta={"kind": "sk"})


def sk_eighths(n: int, seed: int = 0) -> Instance:
    """A dense instance with couplings J_ij = k / 8, k uniform in [-8, 8]
    (symmetric, zero diagonal), and fields h_i = m / 8, m uniform in [-4, 4]:
    every coupling is exact in BF16, and every sum of at most 16384 such terms
    with +/-1 spins is exact in FP32, so a search over it carries no rounding."""
    rng = np.random.default_rng(seed)
    upper = np.triu(rng.integers(-8, 9, size=(n, n), dtype=np.int8), 1)
    Jd = (upper + upper.T).astype(np.float32)
    del upper
    Jd *= np.float32(0.125)
    h = (rng.integers(-4, 5, size=n).astype(np.float32) * np.float32(0.125))
    return Instance(n=n, row_ptr=None, col=None, J=None, J_dense=Jd, h=h, dtype="f32",
                    meta={"kind": "sk-eighths"})


def dense_to_csr(inst: Instance) -> Instance:
    """The same couplings as a CSR listing every off-diagonal pair."""
    n = inst.n
    iu, ju = np.triu_indices(n, 1)
    w = inst.J_dense[iu, ju]
    row_ptr, col, J = csr_from_edges(n, iu, ju, w, "f32")
    return Instance(n=n, row_ptr=row_ptr, col=col, J=J, h=inst.h, dtype="f32",
                    meta=dict(inst.meta, kind="sk-csr"))


def random_graph(n: int, avg_degree: float, seed: int, dtype: str = "f32",
                 n_hyper: int = 0, hyper_order: Sequence[int] = (3,),
                 fields: bool = True, int_range: int = 3) -> Instance:
    """Erdos-Renyi-style graph with optional hyper-edges, for parity cases.

    f32: Gaussian couplings and fields; i8: integers uniform in
    [-int_range, int_range] (zero allowed for fields only).
    """
    rng = np.random.default_rng(seed)
    m = int(round(avg_degree * n / 2))
    pairs = set()
    tries = 0
    while len(pairs) < m and tries < 50 * m + 100:
        a, b = rng.integers(0, n, size=2)
        tries += 1
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    pairs = sorted(pairs)
    u = np.array([p[0] for p in pairs], dtype=np.int64)
    v = np.array([p[1] for p in pairs], dtype=np.int64)
    if dtype == "f32":
        w = rng.standard_normal(len(u)).astype(np.float32)
        h = rng.standard_normal(n).astype(np.float32) if fields else None
    else:
        mag = rng.integers(1, int_range + 1, size=len(u))
        w = (mag * (rng.integers(0, 2, size=len(u)) * 2 - 1)).astype(np.int8)
        h = rng.integers(-int_range, int_range + 1, size=n).astype(np.int8) if fields else None
    row_ptr, col, J = csr_from_edges(n, u, v, w, dtype)
    hp = hm = hJ = None
    if n_hyper > 0:
        members, ptr = [], [0]
        for _ in range(n_hyper):
            k = int(rng.choice(list(hyper_order)))
            k = min(k, n)
            members.append(np.sort(rng.choice(n, size=k, replace=False)))
            ptr.append(ptr[-1] + k)
        hm = np.concatenate(members).astype(np.int32)
        hp = np.array(ptr, dtype=np.int64)
        if dtype == "f32":
            hJ = (rng.standard_normal(n_hyper) * 0.5).astype(np.float32)
        else:
            hJ = (rng.integers(1, int_range + 1, size=n_hyper)
                  * (rng.integers(0, 2, size=n_hyper) * 2 - 1)).astype(np.int8)
    return Instance(n=n, row_ptr=row_ptr, col=col, J=J, h=h, hyper_ptr=hp, hyper_members=hm,
                    hyper_J=hJ, dtype=dtype, meta={"kind": "random"})


def _poly_mul(a: dict, b: dict) -> dict:
    """Product of multilinear polynomials in +/-1 spins (S_i^2 = 1): monomials
    are frozensets of spin indices, multiplied by symmetric difference."""
    out = {}
    for ka, va in a.items():
        for kb, vb in b.items():
            k = ka ^ kb
            out[k] = out.get(k, 0) + va * vb
    return {k: v for k, v in out.items() if v}


def factoring(N: int, n_x: int, n_y: int, hyper: bool = True, dtype: Optional[str] = None) -> Instance:
    """Factoring N as a hyper-Ising instance (Sec. VI, Eqs. 7-9).

    x = 1 + sum_{i=1..n_x} 2^i b_i and y = 1 + sum_{j=1..n_y} 2^j c_j (odd
    factors; bit 0 is fixed), bits b = (1 - S) / 2.  Spins: x's bits 1..n_x
    first, then y's bits n_y..1 (the order of Fig. 7's N = 21 example).  The
    objective f = (N - x y)^2 expanded in the spins (integer coefficients, terms
    of up to four spins) becomes Eq. 6 with h_i = -c_i and J_e = -c_e, so that
    E = f - c_0 and the ground states (E = -c_0) are the factorisations.  Pair
    terms go to the CSR couplings, 3- and 4-spin terms to hyper-edges (left out
    with hyper=False, the reduced model whose ground states need not factor N).
    dtype None: "f32" when every coefficient is below 2^24 in magnitude (exact
    in FP32), else "f64" (exact while every coefficient is below 2^53; wider
    ones - N of more than about 26 bits - are rounded to FP64, and meta
    "exact" is False).  An explicit "f32" with wider coefficients raises
    ValueError.  meta holds N, n_x, n_y, c_0 and "exact"."""
    n = n_x + n_y
    x = {frozenset(): 1}
    y = {frozenset(): 1}
    for i in range(1, n_x + 1):  # 2^i b = 2^(i-1) (1 - S)
        x[frozenset()] += 2 ** (i - 1)
        x[frozenset([i - 1])] = -(2 ** (i - 1))
    for k, j in enumerate(range(n_y, 0, -1)):
        y[frozenset()] += 2 ** (j - 1)
        y[frozenset([n_x + k])] = -(2 ** (j - 1))
    g = {kk: -v for kk, v in _poly_mul(x, y).items()}
    g[frozenset()] = g.get(frozenset(), 0) + N
    f = _poly_mul({kk: v for kk, v in g.items() if v}, {kk: v for kk, v in g.items() if v})
    c0 = f.pop(frozenset(), 0)
    wide = any(abs(v) >= 1 << 24 for v in f.values())
    if dtype is None:
        dtype = "f64" if wide else "f32"
    if dtype == "f32" and wide:
        raise ValueError("coefficients beyond 2^24: not exact in FP32")
    if dtype not in ("f32", "f64"):
        raise ValueError(dtype)
    exact = all(abs(v) < 1 << 53 for v in f.values()) and sum(abs(v) for v in f.values()) < 1 << 53
    vt = np.float32 if dtype == "f32" else np.float64
    h = np.zeros(n, dtype=vt)
    u, v, w, hm, hp, hJ = [], [], [], [], [0], []
    for mono in sorted(f, key=lambda m: (len(m), sorted(m))):
        c = f[mono]
        idx = sorted(mono)
        if len(idx) == 1:
            h[idx[0]] = -c
        elif len(idx) == 2:
            u.append(idx[0])
            v.append(idx[1])
            w.append(-c)
        elif hyper:
            hm.extend(idx)
            hp.append(len(hm))
            hJ.append(-c)
    row_ptr, col, J = csr_from_edges(n, np.array(u, dtype=np.int64), np.array(v, dtype=np.int64),
                                     np.array([float(x) for x in w], dtype=vt), dtype)
    return Instance(n=n, row_ptr=row_ptr, col=col, J=J, h=h,
                    hyper_ptr=np.array(hp, dtype=np.int64) if hJ else None,
                    hyper_members=np.array(hm, dtype=np.int32) if hJ else None,
                    hyper_J=np.array([float(x) for x in hJ], dtype=vt) if hJ else None, dtype=dtype,
                    meta={"N": N, "n_x": n_x, "n_y": n_y, "c0": c0, "exact": exact})


def factoring_decode(inst: Instance, s) -> tuple:
    """(x, y) of a spin configuration of a factoring instance."""
    n_x, n_y = inst.meta["n_x"], inst.meta["n_y"]
    x = 1 + sum(2 ** i * (1 - int(s[i - 1])) // 2 for i in range(1, n_x + 1))
    y = 1 + sum(2 ** j * (1 - int(s[n_x + k])) // 2 for k, j in enumerate(range(n_y, 0, -1)))
    return x, y


def replica_seed(instance_seed: int) -> int:
    """Seed of the Philox random starts for an instance."""
    return splitmix64(instance_seed ^ 0xA5A5A5A5A5A5A5A5)


def config_seed(config_index: int) -> int:
    return 0x5EED0000 + config_index
