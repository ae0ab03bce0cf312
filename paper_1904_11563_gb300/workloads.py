"""Seeded synthetic workloads shaped like the paper's coded multiplications.

This module holds no arithmetic of the method: only random inputs, erasure
masks and the named workload shapes.  Both the CUDA path's tests/benchmarks
and the FP64 oracle's tests draw their inputs here, so the two sides see the
same numbers.

Named workloads (the paper has no dataset; every input is synthetic):

* ``table1_512``: Table I code (n=5, k=2, b=2, 4 sources), A 512 x 256 cut
  into h = 128-row blocks, B 256 x 128, entries iid U(-1,1), seed 0; every
  erasure pattern of at most 2 columns (and the 3-column ones).
* ``sysmoj_8192``: systematic Mojette array n = 11 (k = 8 data columns of an
  8 x 8 grid, e = 3 parities), h = 128, A and B 8192 x 8192 iid N(0,1);
  100 trials, each erasing 3 uniformly drawn columns (mask seed 2000 + t).
* ``table1_logu`` / ``table3_logu``: as table1_512 (Table III: h = 64, A
  576 x 256) with magnitudes log-uniform on [1e-3, 1e3] and random signs.
* ``mojA_16384``: Construction A n = 32, k = 24, b = 683 (16392 one-row
  sources), A 16384 x 16384, B 16384 x 8192, U(-1,1); 8 erased columns.
* ``sysmoj_8192_straggler`` / ``mojA_16384_straggler``: the same shapes with
  processor-level stragglers: cell task times sigma_c X_c, X_c ~ Exp(1) per
  step, decoded from the first decodable set of arrivals.
"""
from __future__ import annotations

import itertools

import numpy as np

WORKLOADS = {
    "table1_512": dict(code=("table1",), h=128, M=512, K=256, N=128, dist="uniform", seed=0, e=2),
    "sysmoj_8192": dict(code=("systematic", 8, 3, 8), h=128, M=8192, K=8192, N=8192,
                        dist="normal", seed=2, e=3, trials=100, mask_seed_base=2000),
    "table1_logu": dict(code=("table1",), h=128, M=512, K=256, N=128, dist="loguniform", seed=3, e=2),
    "table3_logu": dict(code=("table3",), h=64, M=576, K=256, N=128, dist="loguniform", seed=3, e=2),
    "mojA_16384": dict(code=("mojette_a", 32, 24, 683), h=1, M=16384, K=16384, N=8192,
                       dist="uniform", seed=4, e=8, mask_seed_base=4000),
    # the overhead-versus-conditioning sweep of Construction A n = 32, k = 24,
    # e = 8: grid heights b (S = 24 b one-row sources, A S x K), one seeded mask
    "mojA_bsweep": dict(code=("mojette_a", 32, 24, 0), bs=(16, 32, 64, 683), h=1, M=0, K=4096, N=1024,
                        dist="uniform", seed=4, e=8, mask_seed_base=4000, bsweep=True),
    # the benchmark workload with processor-level stragglers: every step draws
    # each cell's task time sigma_c X_c, X_c ~ Exp(mu = 1) (seed 5000 + step),
    # and decodes from the first decodable set of arrived products
    "sysmoj_8192_straggler": dict(code=("systematic", 8, 3, 8), h=128, M=8192, K=8192, N=8192,
                                  dist="normal", seed=2, e=0, trials=100, mask_seed_base=5000, mu=1.0,
                                  straggler=True),
    # Construction A (n = 32, k = 24, b = 683) with processor-level stragglers:
    # the same task-time model over its ~27.7k cells (seed 6000 + step)
    "mojA_16384_straggler": dict(code=("mojette_a", 32, 24, 683), h=1, M=16384, K=16384, N=8192,
                                 dist="uniform", seed=4, e=0, trials=100, mask_seed_base=6000, mu=1.0,
                                 straggler=True),
    # the benchmark code in the paper's two-dimensional scheme: 8 x 8 output
    # blocks of 1024 x 1024 (A in 8 row blocks, B in 8 column blocks)
    "sysmoj_8192_2d": dict(code=("systematic", 8, 3, 8), h=1024, M=8192, K=8192, N=8192,
                           dist="normal", seed=2, e=3, trials=100, mask_seed_base=2000, twod=True),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def erasure_mask(n: int, e: int, seed: int) -> np.ndarray:
    """uint8[n] with e distinct columns set, drawn uniformly (seeded)."""
    m = np.zeros(n, dtype=np.uint8)
    if e > 0:
        m[rng(seed).choice(n, size=e, replace=False)] = 1
    return m


def mask_from_columns(n: int, cols) -> np.ndarray:
    m = np.zeros(n, dtype=np.uint8)
    m[list(cols)] = 1
    return m


def all_masks(n: int, max_e: int):
    """Every erasure mask with at most max_e columns, by size then lexicographic."""
    for e in range(max_e + 1):
        for cols in itertools.combinations(range(n), e):
            yield mask_from_columns(n, cols)


def exponential_draws(n: int, mu: float, seed: int) -> np.ndarray:
    """n iid Exp(mu) draws (seeded): the unit-work task times of n processors
    before the straggler model scales them."""
    return rng(seed).exponential(1.0 / mu, size=n)


def matrix(shape, dist: str, seed: int) -> np.ndarray:
    """FP32 matrix with iid entries: 'uniform' U(-1,1), 'normal' N(0,1),
    'loguniform' |x| log-uniform on [1e-3, 1e3] with random signs,
    'int' integers in [-2, 2] (exact in every arithmetic used here),
    'ternary' sparse {-1, 0, 1} (half zeros)."""
    g = rng(seed)
    if dist == "uniform":
        return g.uniform(-1.0, 1.0, size=shape).astype(np.float32)
    if dist == "normal":
        return g.standard_normal(size=shape, dtype=np.float32)
    if dist == "loguniform":
        mag = np.exp(g.uniform(np.log(1e-3), np.log(1e3), size=shape))
        sgn = np.where(g.random(size=shape) < 0.5, -1.0, 1.0)
        return (mag * sgn).astype(np.float32)
    if dist == "int":
        return g.integers(-2, 3, size=shape).astype(np.float32)
    if dist == "ternary":
        v = g.integers(-1, 2, size=shape).astype(np.float32)
        v[g.random(size=shape) < 0.5] = 0.0
        return v
    raise ValueError(dist)


def inputs(M: int, K: int, N: int, dist: str, seed: int):
    """(A, B) for one workload: A from seed, B from seed + 1."""
    return matrix((M, K), dist, seed), matrix((K, N), dist, seed + 1)


def device_inputs(M: int, K: int, N: int, dist: str, seed: int, device="cuda"):
    """Large (A, B) drawn on the device with torch's seeded generator (for
    full-size runs); copy to the host for the oracle."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if dist == "normal":
        A = torch.randn((M, K), generator=g, device=device, dtype=torch.float32)
        B = torch.randn((K, N), generator=g, device=device, dtype=torch.float32)
    elif dist == "uniform":
        A = torch.rand((M, K), generator=g, device=device, dtype=torch.float32).mul_(2).sub_(1)
        B = torch.rand((K, N), generator=g, device=device, dtype=torch.float32).mul_(2).sub_(1)
    elif dist == "int":
        A = torch.randint(-2, 3, (M, K), generator=g, device=device).to(torch.float32)
        B = torch.randint(-2, 3, (K, N), generator=g, device=device).to(torch.float32)
    else:
        raise ValueError(dist)
    return A, B


def batch_specs(njobs: int, seed: int, lo: int = 256, hi: int = 4096):
    """Job descriptions of a batch of independent coded multiplications:
    M, N, K each 128 * round(x / 128) with x log-uniform on [lo, hi]; half
    array codes (Table I, Table III, systematic Mojette n in 6..32 with e in
    {2, 3}), half projection codes (Construction A, n in 6..32, e =
    floor(n / 4)); grid height b = max(1, M // k), the tallest grid the rows
    allow (a projection code's overhead falls as 1 / b); h = ceil(M / S);
    each job's erasure mask drawn from its own seed.  Returns dicts with
    code=(kind, *params), M, N, K, h, e, n, mask_seed."""
    out = []
    for i in range(njobs):
        g = rng(seed * 100003 + i)

        def dim():
            x = float(np.exp(g.uniform(np.log(lo), np.log(hi))))
            return max(128, 128 * int(round(x / 128)))

        M, N, K = dim(), dim(), dim()
        if g.random() < 0.5:
            pick = int(g.integers(0, 3))
            if pick == 0:
                code, S, n, e = ("table1",), 4, 5, 3
            elif pick == 1:
                code, S, n, e = ("table3",), 9, 5, 2
            else:
                n = int(g.integers(6, 33))
                e = int(g.integers(2, 4))
                k = n - e
                b = max(1, M // k)
                code, S = ("systematic", k, e, b), k * b
        else:
            n = int(g.integers(6, 33))
            e = n // 4
            k = n - e
            b = max(1, M // k)
            code, S = ("mojette_a", n, k, b), k * b
        h = -(-M // S)
        out.append(dict(code=code, M=M, N=N, K=K, h=h, e=e, n=n, mask_seed=seed * 100003 + i + 7))
    return out
