"""GPU parity of the two-dimensional scheme (Section III-A, Examples 1 and 2):
bpx_coded_matmul_2d against the oracle's coded_matmul_2d.

Blocks of C are A_z B_l; floating-point blocks must match the oracle's FP64
decode within the per-block tolerance times the block's propagation factor
(1e-5 split-BF16x3, 2e-2 BF16); small-integer inputs keep every
intermediate exact, so there the match is bit for bit.
"""
import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {"bf16x3": 1e-5, "bf16": 2e-2}


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
    raise ValueError(name)


def _run(bpx, code, A, B, h, prec, mask, opts=None):
    M, K = A.shape
    N = B.shape[1]
    ws = bpx.Workspace2D(code, M, N, K, h, prec)
    C, info = bpx.coded_matmul_2d(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h, prec,
                                  torch.from_numpy(mask).cuda(), ws, opts=opts)
    torch.cuda.synchronize()
    return C.cpu().numpy(), info.cpu().numpy()


def _blocks(C, code_o, h, w):
    return {s: C[z * h:(z + 1) * h, l * w:(l + 1) * w]
            for s in range(code_o.num_sources) for z, l in [o.source_zl(code_o, s)]}


def _nu_2d(ref, A, B, h, w, erased):
    sch = o.wave_schedule(ref, o.surviving_cells(ref, erased))
    used = sorted(set(r for _s, r, _d in sch.order))
    P = o.coded_products_2d(ref, A, B, h, w, used)
    Cd = o.peel_decode(ref, P, sch, h, w)
    nu = o.propagation(ref, sch, P, Cd)
    return {s: nu.get(s, 1.0) for s in range(ref.num_sources)}


def _check(C, R, ref, A, B, h, w, erased, prec, M):
    got = _blocks(C, ref, h, w)
    want = _blocks(R, ref, h, w)
    nu = _nu_2d(ref, A, B, h, w, erased)
    for s in range(ref.num_sources):
        z, _l = o.source_zl(ref, s)
        rows = max(0, min(h, M - z * h))
        if rows == 0:
            continue
        g, r = got[s][:rows], want[s][:rows]
        nr = np.linalg.norm(r)
        err = np.linalg.norm(g - r) / nr if nr > 0 else np.linalg.norm(g)
        assert err <= TOL[prec] * max(1.0, nu[s]), (prec, s, err, nu[s])


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_2d_table1_every_mask(libbpx, prec):
    """Example 1's code in the paper's own scheme: 2 x 2 blocks of C, every
    pattern of <= 3 erased columns."""
    bpx = libbpx
    code, ref = _pair(bpx, "table1")
    h, w, K = 96, 64, 256
    A, B = W.inputs(2 * h, K, 2 * w, "uniform", 3)
    for m in W.all_masks(5, 3):
        er = list(np.nonzero(m)[0])
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
        R, sch = o.coded_matmul_2d(ref, A, B, h, w, er)
        assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
        _check(C, R, ref, A, B, h, w, er, prec, 2 * h)


CASES = [
    # name, h, w, K, M (M < b h: zero-padded last row block), dist
    ("table3", 200, 132, 200, 590, "normal"),
    ("sys8_3_8", 48, 36, 136, 8 * 48 - 7, "uniform"),
    ("A7_4_10", 16, 20, 96, 160, "normal"),
    ("sys4_2_3", 130, 260, 72, 390, "uniform"),
]


@pytest.mark.parametrize("name,h,w,K,M,dist", CASES)
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_2d_codes_ragged(libbpx, name, h, w, K, M, dist, prec):
    """Ragged block shapes (h, w not multiples of the tile), several codes,
    masks with the most erasures the code tolerates."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    N = ref.k * w
    A, B = W.inputs(M, K, N, dist, 23)
    for t in range(3):
        m = W.erasure_mask(code.n, code.e if t else 0, 40 + t)
        er = list(np.nonzero(m)[0])
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
        R, sch = o.coded_matmul_2d(ref, A, B, h, w, er)
        assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
        _check(C, R, ref, A, B, h, w, er, prec, M)


@pytest.mark.parametrize("name,h,w", [("table1", 64, 32), ("table3", 40, 44), ("sys8_3_8", 32, 64),
                                      ("A7_4_10", 8, 24)])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_2d_integer_inputs_bit_exact(libbpx, name, h, w, prec):
    """Small-integer inputs: every block of C equals A B bit for bit."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    K = 128
    M, N = ref.b * h, ref.k * w
    A = W.matrix((M, K), "int", 31)
    B = W.matrix((K, N), "int", 32)
    exact = o.reference_product(A, B)
    for t in range(3):
        m = W.erasure_mask(code.n, code.e, 60 + t)
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
        assert info[bpx.INFO_STATUS] == bpx.OK
        assert np.array_equal(C, exact), (name, prec, t)


@pytest.mark.parametrize("cfg", [0, 16041, 16042, 8041, 8042, 16045, 8046, 8085, 8086, 8080, 8089])
def test_2d_tile_configs_bit_exact(libbpx, cfg):
    """Every tile configuration (widths, CTA pairs, 32 / 64-wide k-slices)
    on integer inputs with several m- and n-tiles per block."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, w, K = 264, 520, 192
    M, N = ref.b * h, ref.k * w
    A = W.matrix((M, K), "int", 41)
    B = W.matrix((K, N), "int", 42)
    m = W.erasure_mask(code.n, 3, 9)
    C, info = _run(bpx, code, A, B, h, bpx.BF16X3, m, opts=bpx.default_opts(gemm_config=cfg))
    assert info[bpx.INFO_STATUS] == bpx.OK
    assert np.array_equal(C, o.reference_product(A, B))


def test_2d_without_direct_writes(libbpx):
    """direct_write = 0: every block (depth 1 included) comes out of the peel."""
    bpx = libbpx
    code, ref = _pair(bpx, "table3")
    h, w, K = 32, 16, 64
    A = W.matrix((3 * h, K), "int", 51)
    B = W.matrix((K, 3 * w), "int", 52)
    m = W.mask_from_columns(5, (0, 2))
    C, info = _run(bpx, code, A, B, h, bpx.BF16X3, m, opts=bpx.default_opts(direct_write=0))
    assert info[bpx.INFO_STATUS] == bpx.OK
    assert np.array_equal(C, o.reference_product(A, B))


def test_2d_full_size_sysmoj_sampled(libbpx):
    """The benchmark code in the two-dimensional scheme at full size: A, B
    8192 x 8192 N(0,1), 8 x 8 blocks of 1024 x 1024, 3 erased columns;
    the deepest blocks and a direct one against FP64 A_z B_l."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    M = N = K = 8192
    h = w = 1024
    A, B = W.device_inputs(M, K, N, "normal", 12)
    m = W.erasure_mask(11, 3, 2007)
    ws = bpx.Workspace2D(code, M, N, K, h, bpx.BF16X3)
    C, info = bpx.coded_matmul_2d(code, A, B, h, bpx.BF16X3, torch.from_numpy(m).cuda(), ws)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
    er = list(np.nonzero(m)[0])
    sch = o.wave_schedule(ref, o.surviving_cells(ref, er))
    deep = sorted(range(64), key=lambda s: -sch.depth[s])[:2]
    direct = [s for s in range(64) if sch.depth[s] == 1][:1]
    Ah = A.cpu().numpy().astype(np.float64)
    Bh = B.cpu().numpy().astype(np.float64)
    # propagation factors from the leading 256 x 256 of every block: nu_s is
    # a ratio of Frobenius norms of blocks with iid entries, which a sample
    # of 65536 entries per block estimates to well under 1 %
    sub = 256
    A_sub = np.concatenate([Ah[z * h:z * h + sub] for z in range(ref.b)])
    B_sub = np.concatenate([Bh[:, l * w:l * w + sub] for l in range(ref.k)], axis=1)
    nu = _nu_2d(ref, A_sub, B_sub, sub, sub, er)
    for s in deep + direct:
        z, l = o.source_zl(ref, s)
        r = Ah[z * h:(z + 1) * h] @ Bh[:, l * w:(l + 1) * w]
        c = C[z * h:(z + 1) * h, l * w:(l + 1) * w].cpu().numpy()
        err = np.linalg.norm(c - r) / np.linalg.norm(r)
        assert err <= 1e-5 * max(1.0, nu[s]), (s, sch.depth[s], err, nu[s])
