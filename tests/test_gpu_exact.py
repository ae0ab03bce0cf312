"""GPU parity of the exact-slice path (BPX_EXACT) against the oracle.

The exact-slice decode is exact integer arithmetic from the fixed-point digit
planes to the peeled blocks, followed by one rounding to FP32, so the CUDA
path must match the oracle (oracle/bpx_oracle.py, exact_slice_*) bit for bit:
on every block, at every peel depth, for every erasure pattern.
"""
import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _pair(bpx, name):
    if name == "table1":
        return bpx.Code.table1(), o.table1()
    if name == "table3":
        return bpx.Code.table3(), o.table3()
    if name.startswith("sys"):
        k, e, b = (int(x) for x in name[3:].split("_"))
        return bpx.Code.systematic(k, e, b), o.systematic_mojette(k, e, b)
    if name.startswith("A"):
        n, k, b = (int(x) for x in name[1:].split("_"))
        return bpx.Code.mojette_a(n, k, b), o.construction_a(n, k, b)
    if name.startswith("B"):
        n, k, b, q = (int(x) for x in name[1:].split("_"))
        return bpx.Code.mojette_b(n, k, b, q), o.construction_b(n, k, b, q)
    raise ValueError(name)


def _run(bpx, code, A, B, h, mask, opts=None):
    M, K = A.shape
    N = B.shape[1]
    ws = bpx.Workspace(code, M, N, K, h, bpx.EXACT)
    C, info = bpx.coded_matmul(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h, bpx.EXACT,
                               torch.from_numpy(mask).cuda(), ws, opts=opts)
    torch.cuda.synchronize()
    return C.cpu().numpy(), info.cpu().numpy()


def _assert_bits(C, R, sch, h, M, what):
    """Recovered blocks bit-identical (rows < M; NaN marks unrecovered)."""
    for s in range(len(sch.depth)):
        if not sch.depth[s]:
            continue
        lo, hi = s * h, min((s + 1) * h, M)
        if lo >= hi:
            continue
        c, r = C[lo:hi], R[lo:hi]
        assert np.array_equal(c.view(np.uint32), r.view(np.uint32)), (what, s, sch.depth[s],
                                                                      np.abs(c - r).max())


def test_exact_table1_every_mask_bit_exact(libbpx):
    """Workload table1_512 (A 512 x 256, B 256 x 128, U(-1,1), h = 128):
    every pattern of <= 3 erased columns."""
    bpx = libbpx
    wl = W.WORKLOADS["table1_512"]
    code, ref = _pair(bpx, "table1")
    A, B = W.inputs(wl["M"], wl["K"], wl["N"], wl["dist"], wl["seed"])
    for m in W.all_masks(ref.n, 3):
        C, info = _run(bpx, code, A, B, wl["h"], m)
        R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, wl["h"], list(np.nonzero(m)[0]))
        assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
        _assert_bits(C, R, sch, wl["h"], wl["M"], tuple(m))


CASES = [
    # name, h, M, K, N, dist: ragged K (not a multiple of 64) and N, M short of S h
    ("table3", 64, 570, 200, 132, "loguniform"),
    ("sys8_3_8", 16, 64 * 16 - 5, 328, 264, "normal"),
    ("A7_4_10", 2, 79, 136, 36, "uniform"),
    ("B6_8_4_2", 3, 95, 96, 20, "normal"),
    ("sys6_5_5", 8, 240, 64, 268, "loguniform"),
]


@pytest.mark.parametrize("name,h,M,K,N,dist", CASES)
def test_exact_codes_ragged_bit_exact(libbpx, name, h, M, K, N, dist):
    """Several code families, ragged shapes and value distributions, a
    handful of masks with the most erasures the code tolerates."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    A, B = W.inputs(M, K, N, dist, 61)
    rng = np.random.default_rng(4)
    depths = set()
    for t in range(4):
        m = W.erasure_mask(code.n, code.e if t else 0, 500 + int(rng.integers(0, 10 ** 6)))
        C, info = _run(bpx, code, A, B, h, m)
        R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, list(np.nonzero(m)[0]))
        assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
        depths.update(d for _s, _r, d in sch.order)
        _assert_bits(C, R, sch, h, M, (name, tuple(m)))


@pytest.mark.parametrize("peel_ctas", [0, 4])
def test_exact_tall_code(libbpx, peel_ctas):
    """A tall code (Construction A n=12, k=9, b=120: 1080 sources, ~118
    waves) through the exact path on the default peel grid and on a 4-CTA
    grid (128 columns a CTA), M short of S h: bit for bit equal to the
    oracle's exact-slice decode."""
    bpx = libbpx
    code, ref = bpx.Code.mojette_a(12, 9, 120), o.construction_a(12, 9, 120)
    h, K, N = 2, 64, 1024
    M = ref.num_sources * h - 3
    A, B = W.inputs(M, K, N, "normal", 67)
    m = W.erasure_mask(12, 3, 5)
    C, info = _run(bpx, code, A, B, h, m, opts=bpx.default_opts(peel_ctas=peel_ctas))
    R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, list(np.nonzero(m)[0]))
    assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK and info[bpx.INFO_WAVES] > 50
    _assert_bits(C, R, sch, h, M, ("A12_9_120", peel_ctas))


@pytest.mark.parametrize("args,e", [((7, 6, 32), 1), ((24, 18, 40), 6)])
def test_exact_source_digit_form(libbpx, args, e):
    """Codes whose cells hold four or more sources on average cut each source
    row's digits once (int8, biased) and sum them per coded row in 16-bit
    lanes: Construction A [7, 6, 32] (sigma 6: 6-bit digits, S = 4) and
    [24, 18, 40] (sigma 18: 4-bit digits, S = 6), M short of S h, K with a
    padded tail: bit for bit equal to the oracle's exact-slice decode."""
    bpx = libbpx
    code, ref = bpx.Code.mojette_a(*args), o.construction_a(*args)
    assert len(code.cell_src) >= 4 * code.num_cells
    h, K, N = 2, 136, 68
    M = ref.num_sources * h - 3
    A, B = W.inputs(M, K, N, "normal", 71)
    m = W.erasure_mask(ref.n, e, 9)
    C, info = _run(bpx, code, A, B, h, m)
    R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, list(np.nonzero(m)[0]))
    assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
    _assert_bits(C, R, sch, h, M, args)


def test_exact_planes_then_peel(libbpx):
    """a3 alone: the S int32 diagonal planes of every surviving cell equal
    the oracle's exact digit products; then a4 alone from those planes."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 8, 512, 200, 68
    A, B = W.inputs(M, K, N, "normal", 71)
    ws = bpx.Workspace(code, M, N, K, h, bpx.EXACT)
    m = W.erasure_mask(code.n, 3, 91)
    bpx.schedule(code, torch.from_numpy(m).cuda(), ws)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    planes = bpx.exact_products(code, dA, dB, h, ws)
    pl = planes.cpu().numpy()
    S = bpx.exact_params(code, K)["S"]
    assert pl.shape[0] == S
    for c in o.surviving_cells(ref, list(np.nonzero(m)[0])):
        want = o.exact_coded_diagonals(ref, A, B, h, c)
        for d in range(S):
            assert np.array_equal(pl[d, c * h:(c + 1) * h].astype(np.int64), want[d]), (c, d)
    C = bpx.alloc_C(code, h, N)
    bpx.peel_decode_exact(code, planes, N, h, C, ws)
    R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, list(np.nonzero(m)[0]))
    _assert_bits(C.cpu().numpy(), R, sch, h, M, "separate")


def test_exact_segments_at_the_accumulation_bound(libbpx):
    """Adversarial digits: every entry of A and B is the same positive value
    whose balanced digits (w = 6) are (31, -32, -32, -32), the largest
    magnitudes the digits can take, so the coded digits of a degree-8 cell
    are 8 times that (|.| up to 256) and every digit product is about
    256 x 32: each 1024-wide segment sums to about 2^23, the bound the exact
    FP32 accumulation is sized for.  Bit-exact against the oracle."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    p = bpx.exact_params(code, 2048)
    assert (p["w"], p["S"], p["bits"], p["seg"]) == (6, 4, 23, 1024)
    xint = 31 * 2 ** 18 - 32 * (2 ** 12 + 2 ** 6 + 1)
    assert [int(d[0]) for d in o.balanced_digits(np.array([xint]), 6, 4)] == [31, -32, -32, -32]
    x = np.float32(xint * 2.0 ** -23)
    h, K, N = 4, 2048, 64
    M = ref.num_sources * h
    A = np.full((M, K), x, dtype=np.float32)
    B = np.full((K, N), x, dtype=np.float32)
    A[:, 1::7] = -x           # mixed signs elsewhere keep the digit magnitudes
    for mcols in [(), (8, 9, 10), (0, 3, 9)]:
        m = W.mask_from_columns(code.n, mcols)
        C, info = _run(bpx, code, A, B, h, m)
        R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, list(mcols))
        assert info[bpx.INFO_STATUS] == bpx.OK
        _assert_bits(C, R, sch, h, M, mcols)
    Bp = np.abs(B)
    Ap = np.abs(A)
    C, info = _run(bpx, code, Ap, Bp, h, W.mask_from_columns(code.n, ()))
    R, _Q, sch = o.exact_slice_coded_matmul(ref, Ap, Bp, h, [])
    _assert_bits(C, R, sch, h, M, "all positive")


@pytest.mark.parametrize("cfg", [0, 8085, 16085, 8086, 4086, 16081, 8042, 8080, 8089])
def test_exact_tile_configs_identical(libbpx, cfg):
    """Every tile configuration gives bit-identical results (the arithmetic
    is exact, so neither tile shape, CTA pairing, band nor segment choice can
    change a bit), equal to the oracle; 128-row tiles span several m-tiles
    with a ragged last one."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 24, 64 * 24, 264, 520
    A, B = W.inputs(M, K, N, "normal", 81)
    m = W.erasure_mask(code.n, 3, 17)
    C, info = _run(bpx, code, A, B, h, m, opts=bpx.default_opts(gemm_config=cfg))
    R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, list(np.nonzero(m)[0]))
    assert info[bpx.INFO_STATUS] == bpx.OK
    _assert_bits(C, R, sch, h, M, cfg)


def test_exact_undecodable_partial(libbpx):
    """Four erasures on Table I: status UNDECODABLE, the recovered blocks
    bit-exact, the others untouched."""
    bpx = libbpx
    code, ref = _pair(bpx, "table1")
    h, M, K, N = 16, 64, 96, 32
    A, B = W.inputs(M, K, N, "uniform", 5)
    m = W.mask_from_columns(5, (0, 1, 2, 3))
    ws = bpx.Workspace(code, M, N, K, h, bpx.EXACT)
    C = torch.full((code.num_sources * h, N), 7.0, device="cuda")
    C, info = bpx.coded_matmul(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h, bpx.EXACT,
                               torch.from_numpy(m).cuda(), ws, C=C)
    torch.cuda.synchronize()
    R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, [0, 1, 2, 3])
    assert not sch.ok and info.cpu().numpy()[bpx.INFO_STATUS] == bpx.ERR_UNDECODABLE
    Cn = C.cpu().numpy()
    _assert_bits(Cn, R, sch, h, M, "partial")
    for s in range(ref.num_sources):
        if not sch.depth[s]:
            assert np.all(Cn[s * h:(s + 1) * h] == 7.0)


def test_exact_host_entry_point(libbpx):
    """bpx_coded_matmul_host with BPX_EXACT (host buffers in and out)."""
    bpx = libbpx
    code, ref = _pair(bpx, "table3")
    h, M, K, N = 32, 288, 128, 64
    A, B = W.inputs(M, K, N, "normal", 13)
    m = W.mask_from_columns(5, (1, 4))
    ws = bpx.Workspace(code, M, N, K, h, bpx.EXACT)
    dA = torch.empty((M, K), device="cuda")
    dB = torch.empty((K, N), device="cuda")
    dm = torch.empty(5, dtype=torch.uint8, device="cuda")
    dC = bpx.alloc_C(code, h, N)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hm = torch.from_numpy(m).pin_memory()
    hC = torch.empty((M, N)).pin_memory()
    status, info = bpx.coded_matmul_host(code, hA, hB, h, bpx.EXACT, hm, hC, dA, dB, dm, dC, ws)
    assert status == bpx.OK
    R, _Q, sch = o.exact_slice_coded_matmul(ref, A, B, h, [1, 4])
    _assert_bits(hC.numpy(), R, sch, h, M, "host")


def test_exact_full_size_sysmoj_8192_sampled(libbpx):
    """The benchmark workload at full size (A, B 8192 x 8192 N(0,1), h = 128,
    3 erased columns) in the benchmark's launch configuration: the deepest
    sources and a direct one, on 48 sampled columns, bit-identical to the
    oracle's exact-slice product of the source (computed without the code --
    equal to the decode by the mask-independence pin)."""
    bpx = libbpx
    wl = W.WORKLOADS["sysmoj_8192"]
    code, ref = _pair(bpx, "sys8_3_8")
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    A, B = W.device_inputs(M, K, N, "normal", 2)
    m = W.erasure_mask(11, 3, wl["mask_seed_base"] + 7)
    ws = bpx.Workspace(code, M, N, K, h, bpx.EXACT)
    C, info = bpx.coded_matmul(code, A, B, h, bpx.EXACT, torch.from_numpy(m).cuda(), ws)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
    sch = o.wave_schedule(ref, o.surviving_cells(ref, list(np.nonzero(m)[0])))
    deep = sorted(range(64), key=lambda s: -sch.depth[s])[:2]
    direct = [s for s in range(64) if sch.depth[s] == 1][:1]
    cols = np.sort(np.random.default_rng(1).choice(N, 48, replace=False))
    Ah = A.cpu().numpy()
    Bh = B.cpu().numpy()
    eA = o.exact_row_exponents(Ah, h)
    for s in deep + direct:
        want, _q = o.exact_slice_block(Ah, Bh, s, h, ref.sigma, cols=cols, eA=eA)
        got = C[s * h:(s + 1) * h].cpu().numpy()[:, cols]
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (s, sch.depth[s])


def test_exact_construction_a_full_size_deep_rows(libbpx):
    """Workload mojA_16384 at full size (Construction A n=32, k=24, b=683,
    h=1, 8 erased columns, ~700 peel waves) with U(-1,1) inputs: rows at
    depth ~700 -- where every floating-point peel loses all accuracy -- are
    bit-identical to the oracle's exact-slice product of the row, and within
    2e-6 of FP64 A B relative to the row's largest entry."""
    bpx = libbpx
    wl = W.WORKLOADS["mojA_16384"]
    code = bpx.Code.mojette_a(32, 24, 683)
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    A, B = W.device_inputs(M, K, N, "uniform", 41)
    m = torch.from_numpy(W.erasure_mask(32, 8, wl["mask_seed_base"])).cuda()
    ws = bpx.Workspace(code, M, N, K, h, bpx.EXACT)
    C, info = bpx.coded_matmul(code, A, B, h, bpx.EXACT, m, ws)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[bpx.INFO_STATUS] == bpx.OK and inf[bpx.INFO_WAVES] > 100
    del ws
    order, _rec, _i = bpx.schedule(code, m, bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32))
    order = order.cpu().numpy()
    rows = [int(s) for s, _r, d in order[::-1][:4] if 0 <= s < M]
    rows += [int(s) for s, _r, d in order if d == 1][:2]
    cols = np.sort(np.random.default_rng(2).choice(N, 32, replace=False))
    Ah = A.cpu().numpy()
    Bh = B.cpu().numpy()
    eA = o.exact_row_exponents(Ah, h)
    for r in rows:
        want, _q = o.exact_slice_block(Ah, Bh, r, h, code.sigma, cols=cols, eA=eA)
        got = C[r:r + 1].cpu().numpy()[:, cols]
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), r
        ref = Ah[r:r + 1].astype(np.float64) @ Bh[:, cols].astype(np.float64)
        assert np.abs(got - ref).max() <= 2e-6 * K ** 0.5 * np.abs(Ah[r]).max() * np.abs(Bh).max()
