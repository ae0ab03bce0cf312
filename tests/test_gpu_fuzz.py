"""Randomised GPU parity (seeded): random codes of every family, ragged
shapes down to a single row or column group, random erasure patterns, tile
configurations and options, every precision and both schemes -- each case
against the oracle (schedule bit for bit; blocks within the precision's
tolerance times their propagation factor; exact slices and small-integer
inputs bit for bit)."""
import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "fp16x3": 1e-5, "bf16": 2e-2, "mxfp8": 6e-2}
CONFIGS = [0, 16041, 16042, 8041, 8042, 16045, 8046, 8085, 8086, 4081, 8080, 8089, 4080]


def _random_code(bpx, rng):
    kind = rng.integers(0, 5)
    if kind == 0:
        return bpx.Code.table1(), o.table1()
    if kind == 1:
        return bpx.Code.table3(), o.table3()
    if kind == 2:
        k, e, b = int(rng.integers(2, 7)), int(rng.integers(1, 4)), int(rng.integers(1, 6))
        return bpx.Code.systematic(k, e, b), o.systematic_mojette(k, e, b)
    if kind == 3:
        k = int(rng.integers(2, 6))
        n, b = k + int(rng.integers(0, 4)), int(rng.integers(1, 7))
        return bpx.Code.mojette_a(n, k, b), o.construction_a(n, k, b)
    k, q = int(rng.integers(2, 9)), int(rng.integers(1, 3))
    need = -(-k // 2 ** q)
    n, b = need + int(rng.integers(0, 3)), int(rng.integers(1, 5))
    return bpx.Code.mojette_b(n, k, b, q), o.construction_b(n, k, b, q)


def _nu(ref, A, B, h, sch):
    used = sorted(set(r for _s, r, _d in sch.order))
    P = o.coded_products(ref, A, B, h, used)
    nu = o.propagation(ref, sch, P, o.peel_decode(ref, P, sch, h, B.shape[1]))
    return {s: nu.get(s, 1.0) for s in range(ref.num_sources)}


PRECS = ["fp32", "bf16", "bf16x3", "mxfp8", "exact", "fp16x3"]


@pytest.mark.parametrize("seed", range(72))
def test_fuzz_one_dimensional(libbpx, seed):
    bpx = libbpx
    rng = np.random.default_rng(1000 + seed)
    code, ref = _random_code(bpx, rng)
    prec = PRECS[seed % len(PRECS)]
    h = int(rng.choice([1, 2, 3, 7, 16, 33, 64, 130]))
    M = max(1, ref.num_sources * h - int(rng.integers(0, h)))
    K = 128 * int(rng.integers(1, 4)) if prec == "mxfp8" else 8 * int(rng.integers(1, 70))
    N = 4 * int(rng.integers(1, 150))
    if prec == "mxfp8":
        # E4M3 rounds each operand with an RMS relative error near 2.5 %, so a
        # block's relative Frobenius error is a mean over its elements (about
        # 3.6e-2 in expectation); blocks of >= 1024 elements keep that mean
        # within a few percent of its expectation, below the 6e-2 tolerance
        N = max(N, 4 * -(-1024 // (4 * h)))
    dist = ["uniform", "normal", "int"][int(rng.integers(0, 3))]
    A, B = W.inputs(M, K, N, dist, 2000 + seed)
    e = int(rng.integers(0, ref.n - ref.k + 1)) if ref.n > ref.k else 0
    m = W.erasure_mask(ref.n, e, 3000 + seed)
    er = list(np.nonzero(m)[0])
    opts = bpx.default_opts(gemm_config=int(rng.choice(CONFIGS)), direct_write=int(rng.integers(0, 2)))
    if prec in ("bf16", "fp32") and rng.random() < 0.5:
        opts.compensate_depth = 2
    P = bpx.PRECISIONS[prec]
    ws = bpx.Workspace(code, M, N, K, h, P)
    C, info = bpx.coded_matmul(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h, P,
                               torch.from_numpy(m).cuda(), ws, opts=opts)
    torch.cuda.synchronize()
    C, info = C.cpu().numpy(), info.cpu().numpy()
    sch = o.wave_schedule(ref, o.surviving_cells(ref, er))
    assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE), (seed, prec)
    assert info[bpx.INFO_WAVES] == max([d for _s, _r, d in sch.order], default=0)
    if prec == "exact":
        R, _Q, _s = o.exact_slice_coded_matmul(ref, A, B, h, er)
        for s in range(ref.num_sources):
            lo, hi = s * h, min((s + 1) * h, M)
            if sch.depth[s] and lo < hi:
                assert np.array_equal(C[lo:hi].view(np.uint32), R[lo:hi].view(np.uint32)), (seed, s)
        return
    R, _s = o.coded_matmul(ref, A, B, h, er)
    if dist == "int" and prec in ("fp32", "bf16", "bf16x3", "fp16x3") and K * 4 * ref.sigma < 2 ** 20:
        for s in range(ref.num_sources):
            lo, hi = s * h, min((s + 1) * h, M)
            if sch.depth[s] and lo < hi:
                assert np.array_equal(C[lo:hi], R[lo:hi]), (seed, prec, s)
        return
    nu = _nu(ref, A, B, h, sch)
    for s in range(ref.num_sources):
        lo, hi = s * h, min((s + 1) * h, M)
        if not sch.depth[s] or lo >= hi:
            continue
        r = R[lo:hi]
        nr = np.linalg.norm(r)
        if nr == 0:
            continue
        err = np.linalg.norm(C[lo:hi] - r) / nr
        assert err <= TOL[prec] * max(1.0, nu[s]), (seed, prec, s, err, nu[s])


@pytest.mark.parametrize("seed", range(20))
def test_fuzz_two_dimensional(libbpx, seed):
    bpx = libbpx
    rng = np.random.default_rng(5000 + seed)
    code, ref = _random_code(bpx, rng)
    prec = ["bf16x3", "bf16"][seed % 2]
    h = int(rng.choice([1, 5, 16, 40, 129]))
    w = 4 * int(rng.integers(1, 40))
    M = max(1, ref.b * h - int(rng.integers(0, h)))
    K = 8 * int(rng.integers(1, 40))
    N = ref.k * w
    A = W.matrix((M, K), "int", 6000 + seed)
    B = W.matrix((K, N), "int", 7000 + seed)
    e = int(rng.integers(0, ref.n - ref.k + 1)) if ref.n > ref.k else 0
    m = W.erasure_mask(ref.n, e, 8000 + seed)
    er = list(np.nonzero(m)[0])
    opts = bpx.default_opts(gemm_config=int(rng.choice(CONFIGS)), direct_write=int(rng.integers(0, 2)))
    ws = bpx.Workspace2D(code, M, N, K, h, bpx.PRECISIONS[prec])
    C, info = bpx.coded_matmul_2d(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h,
                                  bpx.PRECISIONS[prec], torch.from_numpy(m).cuda(), ws, opts=opts)
    torch.cuda.synchronize()
    C, info = C.cpu().numpy(), info.cpu().numpy()
    R, sch = o.coded_matmul_2d(ref, A, B, h, w, er)
    assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
    for s in range(ref.num_sources):
        z, l = o.source_zl(ref, s)
        rows = max(0, min(h, M - z * h))
        if sch.depth[s] and rows:
            blk = (slice(z * h, z * h + rows), slice(l * w, (l + 1) * w))
            assert np.array_equal(C[blk], R[blk]), (seed, prec, s)
