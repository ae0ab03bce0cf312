"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer and index work (surviving cells, peel order, resolvers, depths,
recovered set) must match bit for bit; floating-point blocks of C must match
the oracle's FP64 decode within the relative Frobenius tolerance per block
(1e-5 for FP32, split-BF16x3 and split-FP16x3, 2e-2 for plain BF16) times
the block's propagation factor; split-FP16x3 also flat, without the factor,
on the full-size benchmark workload.  Small-integer inputs
keep every FP32 intermediate exact, so there the match is bit-exact too.
"""
import itertools

import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "fp16x3": 1e-5, "bf16": 2e-2}


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
    if name.startswith("xcode"):
        p = int(name[5:])
        return bpx.Code.xcode(p), o.xcode(p)
    raise ValueError(name)


def _masks(code_o, max_e, extra=()):
    ms = [m for m in W.all_masks(code_o.n, max_e)]
    for cols in extra:
        ms.append(W.mask_from_columns(code_o.n, cols))
    return ms


def _oracle_decode(code_o, A, B, h, mask):
    erased = list(np.nonzero(mask)[0])
    return o.coded_matmul(code_o, A, B, h, erased)


def _nu(ref, A, B, h, m):
    """Oracle propagation factor per source (1 for direct copies)."""
    cells = o.surviving_cells(ref, list(np.nonzero(m)[0]))
    sch = o.wave_schedule(ref, cells)
    used = sorted(set(r for _s, r, _d in sch.order))
    P = o.coded_products(ref, A, B, h, used)
    Cd = o.peel_decode(ref, P, sch, h, B.shape[1])
    nu = o.propagation(ref, sch, P, Cd)
    return np.array([nu.get(s, 1.0) for s in range(ref.num_sources)])


def _check_blocks(C, R, ref, A, B, h, m, prec):
    """Every block within TOL x nu_s: the stated per-block tolerance applies
    to each coded product and to each block copied from one; a block peeled
    out of several products inherits their errors, magnified by nu_s."""
    err = _rel_block_err(C, R, h, ref.num_sources)
    nu = _nu(ref, A, B, h, m)
    bound = TOL[prec] * np.maximum(1.0, nu)
    assert np.all(err <= bound), (prec, err.max(), (err / bound).max())
    return err, nu


def _rel_block_err(C, R, h, S):
    errs = []
    for s in range(S):
        r = R[s * h:(s + 1) * h]
        c = C[s * h:(s + 1) * h]
        nr = np.linalg.norm(r)
        errs.append(np.linalg.norm(c - r) / nr if nr > 0 else np.linalg.norm(c))
    return np.array(errs)


# ---------------------------------------------------------------- a1: schedule

SCHED_CODES = ["table1", "table3", "sys8_3_8", "sys6_5_5", "A7_4_10", "A11_8_12", "B6_8_4_2", "xcode7", "xcode13"]


@pytest.mark.parametrize("name", SCHED_CODES)
def test_schedule_bit_exact(libbpx, name):
    bpx = libbpx
    code, ref = _pair(bpx, name)
    ws = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32)
    rng = np.random.default_rng(1)
    masks = list(W.all_masks(code.n, min(code.e + 1, 3)))
    masks += [(rng.random(code.n) < 0.5).astype(np.uint8) for _ in range(10)]
    for m in masks:
        dm = torch.from_numpy(m).cuda()
        order, rec, info = bpx.schedule(code, dm, ws)
        torch.cuda.synchronize()
        sch = o.wave_schedule(ref, o.surviving_cells(ref, np.nonzero(m)[0]))
        exp = np.full((code.num_sources, 3), -1, dtype=np.int32)
        for i, (s, r, d) in enumerate(sch.order):
            exp[i] = (s, r, d)
        assert np.array_equal(order.cpu().numpy(), exp), m
        assert list(rec.cpu().numpy()) == sch.recovered
        inf = info.cpu().numpy()
        assert inf[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
        assert inf[bpx.INFO_RECOVERED] == sum(sch.recovered)
        assert inf[bpx.INFO_WAVES] == sch.num_waves
        assert inf[bpx.INFO_SURVIVING] == len(o.surviving_cells(ref, np.nonzero(m)[0]))


def test_schedule_large_construction_a(libbpx):
    """The full-size projection code (16392 sources, ~27.7k cells): bit-exact
    plan for seeded 8-column erasures."""
    bpx = libbpx
    code, ref = _pair(bpx, "A32_24_683")
    ws = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32)
    for t in range(2):
        m = W.erasure_mask(code.n, 8, 4000 + t)
        order, rec, info = bpx.schedule(code, torch.from_numpy(m).cuda(), ws)
        sch = o.wave_schedule(ref, o.surviving_cells(ref, np.nonzero(m)[0]))
        got = order.cpu().numpy()
        assert sch.ok
        assert np.array_equal(got, np.array(sch.order, dtype=np.int32))
        assert info.cpu().numpy()[bpx.INFO_WAVES] == sch.num_waves


def test_schedule_state_in_global_memory(libbpx):
    """A projection code too large for the plan's on-chip state (Construction
    A n = 16, k = 12, b = 2800: 33600 sources and ~45k cells, whose per-cell
    words and depths exceed the CTA's shared memory) plans with 64-bit cell
    words in global memory: bit-exact against the oracle, decodable and
    undecodable masks."""
    bpx = libbpx
    code, ref = _pair(bpx, "A16_12_2800")
    assert (code.num_cells + code.num_sources) * 4 > 224 * 1024
    ws = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32)
    for t, e in [(0, 4), (1, 4), (2, 5)]:
        m = W.erasure_mask(code.n, e, 4100 + t)
        order, rec, info = bpx.schedule(code, torch.from_numpy(m).cuda(), ws)
        sch = o.wave_schedule(ref, o.surviving_cells(ref, np.nonzero(m)[0]))
        exp = np.full((code.num_sources, 3), -1, dtype=np.int32)
        for i, (s_, r, d) in enumerate(sch.order):
            exp[i] = (s_, r, d)
        assert np.array_equal(order.cpu().numpy(), exp)
        assert list(rec.cpu().numpy()) == sch.recovered
        inf = info.cpu().numpy()
        assert inf[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE) and sch.ok == (e <= 4)
        assert inf[bpx.INFO_WAVES] == sch.num_waves


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_whole_path_with_plan_state_in_global_memory(libbpx, prec):
    """The whole path on a code whose plan state does not fit on chip
    (Construction A n = 16, k = 12, b = 2800: 33600 one-row sources, ~45k
    cells, ~2800 waves; the schedule keeps 64-bit cell words in global memory
    and, as for every code of more than 4096 sources, plans in two parts, the
    second beside the products): small-integer inputs decode to A B bit for
    bit on every row, with the plan equal to the oracle's."""
    bpx = libbpx
    code, ref = _pair(bpx, "A16_12_2800")
    h, K, N = 1, 64, 32
    M = ref.num_sources * h - 5
    A = W.matrix((M, K), "int", 51)
    B = W.matrix((K, N), "int", 52)
    exact = o.reference_product(A, B)
    m = W.erasure_mask(code.n, 4, 4200)
    C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
    assert info[bpx.INFO_STATUS] == bpx.OK and info[bpx.INFO_WAVES] > 1000
    assert np.array_equal(C[:M], exact)
    sch = o.wave_schedule(ref, o.surviving_cells(ref, np.nonzero(m)[0]))
    assert info[bpx.INFO_WAVES] == sch.num_waves and info[bpx.INFO_RECOVERED] == ref.num_sources


# ---------------------------------------------------------------- a2: encode

@pytest.mark.parametrize("name,h", [("table3", 3), ("sys8_3_8", 2), ("A7_4_10", 1)])
def test_encode_materialized(libbpx, name, h):
    bpx = libbpx
    code, ref = _pair(bpx, name)
    M, K = code.num_sources * h - 1, 40
    A = W.matrix((M, K), "uniform", 11)
    ws = bpx.Workspace(code, M, 8, K, h, bpx.FP32)
    m = W.erasure_mask(code.n, code.e, 5)
    bpx.schedule(code, torch.from_numpy(m).cuda(), ws)
    out = bpx.encode(code, torch.from_numpy(A).cuda(), h, ws).cpu().numpy()
    cells = o.surviving_cells(ref, np.nonzero(m)[0])
    for i, c in enumerate(cells):
        exp = o.encode(ref, A, h, c)
        np.testing.assert_allclose(out[i * h:(i + 1) * h], exp, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- whole path

def _run(bpx, code, A, B, h, prec, mask, opts=None):
    M, K = A.shape
    N = B.shape[1]
    ws = bpx.Workspace(code, M, N, K, h, prec)
    C, info = bpx.coded_matmul(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h, prec,
                               torch.from_numpy(mask).cuda(), ws, opts=opts)
    torch.cuda.synchronize()
    return C.cpu().numpy(), info.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "fp16x3"])
def test_table1_all_masks_vs_oracle(libbpx, prec):
    """Workload table1_512: every erasure pattern of <= 2 columns (and the
    3-column ones the code also tolerates), every block within tolerance."""
    bpx = libbpx
    wl = W.WORKLOADS["table1_512"]
    code, ref = _pair(bpx, "table1")
    A, B = W.inputs(wl["M"], wl["K"], wl["N"], wl["dist"], wl["seed"])
    P = bpx.PRECISIONS[prec]
    for m in _masks(ref, 3):
        C, info = _run(bpx, code, A, B, wl["h"], P, m)
        R, sch = _oracle_decode(ref, A, B, wl["h"], m)
        assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
        _check_blocks(C, R, ref, A, B, wl["h"], m, prec)


@pytest.mark.parametrize("name,h,M,K,N", [
    ("table3", 3, 26, 136, 200),       # ragged: M < S h, K and N not tile multiples
    ("sys8_3_8", 5, 320, 72, 36),
    ("A7_4_10", 1, 40, 264, 132),      # one-row sources, depth > 1
    ("B6_8_4_2", 2, 64, 32, 260),
    ("table1", 130, 520, 64, 8),       # blocks taller than a tile
])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "fp16x3"])
def test_integer_inputs_bit_exact(libbpx, name, h, M, K, N, prec):
    """Small-integer inputs: every intermediate is an exact integer < 2^24,
    so the decoded C equals the oracle (and A B) bit for bit."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    A = W.matrix((M, K), "int", 21)
    B = W.matrix((K, N), "int", 22)
    ref_C = o.reference_product(A, B)
    rng = np.random.default_rng(3)
    for t in range(6):
        m = W.erasure_mask(code.n, int(rng.integers(0, code.e + 1)), 100 + t)
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
        R, sch = _oracle_decode(ref, A, B, h, m)
        assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
        assert np.array_equal(C[:M], ref_C), (name, m)
        assert np.array_equal(C[:M], R[:M])


def test_products_and_peel_separately(libbpx):
    """a3 alone (no direct writes): every surviving cell's product within
    tolerance of the oracle; then a4 alone fed with those products."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 4, 256, 96, 64
    A, B = W.inputs(M, K, N, "normal", 31)
    ws = bpx.Workspace(code, M, N, K, h, bpx.FP32)
    m = W.erasure_mask(code.n, 3, 77)
    bpx.schedule(code, torch.from_numpy(m).cuda(), ws)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    P = bpx.coded_products(code, dA, dB, h, bpx.FP32, ws)
    Pn = P.cpu().numpy()
    cells = o.surviving_cells(ref, np.nonzero(m)[0])
    Po = o.coded_products(ref, A, B, h, cells)
    for c in cells:
        blk = Pn[c * h:(c + 1) * h]
        assert np.linalg.norm(blk - Po[c]) / np.linalg.norm(Po[c]) <= 1e-5
    C = bpx.alloc_C(code, h, N)
    bpx.peel_decode(code, P, N, h, C, ws, direct_written=False)
    R, sch = _oracle_decode(ref, A, B, h, m)
    err = _rel_block_err(C.cpu().numpy(), R, h, ref.num_sources)
    assert err.max() <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "exact"])
def test_peel_decode_takes_the_erasure_mask(libbpx, prec):
    """peel_decode(products, erasure_mask) -> C: given the mask, the peel
    plans itself -- over a workspace whose plan was overwritten by another
    mask's schedule it still decodes the products of its own mask, bit for
    bit as the whole path does; given no mask it peels along the plan in the
    workspace."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 4, 256, 96, 64
    A, B = W.inputs(M, K, N, "normal", 31)
    P_ = bpx.PRECISIONS[prec]
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    m = torch.from_numpy(W.erasure_mask(code.n, 3, 77)).cuda()
    other = torch.from_numpy(W.erasure_mask(code.n, 3, 78)).cuda()
    want, _info = bpx.coded_matmul(code, dA, dB, h, P_, m, bpx.Workspace(code, M, N, K, h, P_),
                                   opts=bpx.default_opts(direct_write=0))
    ws = bpx.Workspace(code, M, N, K, h, P_)
    bpx.schedule(code, m, ws)
    if prec == "exact":
        prods = bpx.exact_products(code, dA, dB, h, ws)
    else:
        prods = bpx.coded_products(code, dA, dB, h, P_, ws)
    bpx.schedule(code, other, ws)  # a stale plan for another mask
    C = bpx.alloc_C(code, h, N)
    info = torch.zeros(bpx.INFO_LEN, dtype=torch.int32, device="cuda")
    if prec == "exact":
        bpx.peel_decode_exact(code, prods, N, h, C, ws, mask=m, info=info)
    else:
        bpx.peel_decode(code, prods, N, h, C, ws, direct_written=False, mask=m, info=info)
    torch.cuda.synchronize()
    assert int(info[bpx.INFO_STATUS]) == bpx.OK
    assert torch.equal(C[:M], want[:M])
    C2 = bpx.alloc_C(code, h, N)
    if prec == "exact":
        bpx.peel_decode_exact(code, prods, N, h, C2, ws)
    else:
        bpx.peel_decode(code, prods, N, h, C2, ws, direct_written=False)
    torch.cuda.synchronize()
    assert torch.equal(C2[:M], want[:M])


def test_peel_without_a_plan_is_refused(libbpx):
    """A workspace no schedule has planned: the peel writes nothing and
    reports BPX_ERR_INVAL in the plan's info words."""
    bpx = libbpx
    code, _ref = _pair(bpx, "table1")
    h, N = 8, 16
    ws = bpx.Workspace(code, 32, N, 16, h, bpx.FP32)
    prods = torch.ones((code.num_cells * h, N), device="cuda")
    C = torch.full((code.num_sources * h, N), 7.0, device="cuda")
    bpx.peel_decode(code, prods, N, h, C, ws, direct_written=False)
    torch.cuda.synchronize()
    assert bool((C == 7.0).all())
    info = ws.info().cpu().numpy()
    assert info[bpx.INFO_STATUS] == bpx.ERR_INVAL and info[bpx.INFO_DEVICE_ERR] == bpx.ERR_INVAL


def test_undecodable_partial(libbpx):
    """Four erasures on Table I: status UNDECODABLE, recovered set as the
    oracle's, recovered blocks correct, the rest untouched."""
    bpx = libbpx
    code, ref = _pair(bpx, "table1")
    h, M, K, N = 8, 32, 16, 12
    A = W.matrix((M, K), "int", 41)
    B = W.matrix((K, N), "int", 42)
    for cols in itertools.combinations(range(5), 4):
        m = W.mask_from_columns(5, cols)
        C, info = _run(bpx, code, A, B, h, bpx.FP32, m)
        sch = o.wave_schedule(ref, o.surviving_cells(ref, cols))
        assert info[bpx.INFO_STATUS] == bpx.ERR_UNDECODABLE
        assert info[bpx.INFO_RECOVERED] == sum(sch.recovered)
        refC = o.reference_product(A, B)
        for s in range(4):
            blk = C[s * h:(s + 1) * h]
            if sch.depth[s] > 0:
                assert np.array_equal(blk, refC[s * h:(s + 1) * h])
            else:
                assert np.all(blk == 0)


def test_compensated_peel(libbpx):
    """compensate_depth = 0 forces the compensated subtraction on every
    wave; the result stays within tolerance and equals the plain path on
    integers."""
    bpx = libbpx
    code, ref = _pair(bpx, "table3")
    h, M, K, N = 6, 54, 48, 40
    A, B = W.inputs(M, K, N, "loguniform", 51)
    m = W.mask_from_columns(5, [0, 2])
    opts = bpx.default_opts(compensate_depth=0)
    C, info = _run(bpx, code, A, B, h, bpx.FP32, m, opts=opts)
    R, sch = _oracle_decode(ref, A, B, h, m)
    err = _rel_block_err(C, R, h, 9)
    kap = _kappas(ref, A, B, h, m)
    for s in range(9):
        assert err[s] <= 1e-5 * max(1.0, kap[s]), (s, err[s], kap[s])


def _kappas(ref, A, B, h, m):
    cells = o.surviving_cells(ref, np.nonzero(m)[0])
    sch = o.wave_schedule(ref, cells)
    P = o.coded_products(ref, A, B, h, cells)
    Cd = o.peel_decode(ref, P, sch, h, B.shape[1])
    return o.amplification(ref, sch, P, Cd)


def test_direct_write_off_matches_on(libbpx):
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 4, 256, 64, 48
    A = W.matrix((M, K), "int", 61)
    B = W.matrix((K, N), "int", 62)
    m = W.erasure_mask(11, 3, 9)
    C1, _ = _run(bpx, code, A, B, h, bpx.FP32, m)
    C2, _ = _run(bpx, code, A, B, h, bpx.FP32, m, opts=bpx.default_opts(direct_write=0))
    assert np.array_equal(C1, C2)


def test_host_entry_point_matches_device(libbpx):
    bpx = libbpx
    code, ref = _pair(bpx, "table1")
    h, M, K, N = 16, 64, 32, 24
    A, B = W.inputs(M, K, N, "uniform", 71)
    m = W.mask_from_columns(5, [1, 4])
    C_dev, _ = _run(bpx, code, A, B, h, bpx.FP32, m)
    ws = bpx.Workspace(code, M, N, K, h, bpx.FP32)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hm = torch.from_numpy(m).pin_memory()
    hC = torch.zeros((M, N), dtype=torch.float32).pin_memory()
    dA = torch.empty_like(hA, device="cuda")
    dB = torch.empty_like(hB, device="cuda")
    dm = torch.empty_like(hm, device="cuda")
    dC = bpx.alloc_C(code, h, N)
    rc, info = bpx.coded_matmul_host(code, hA, hB, h, bpx.FP32, hm, hC, dA, dB, dm, dC, ws)
    assert rc == bpx.OK and info[bpx.INFO_STATUS] == bpx.OK
    assert np.array_equal(hC.numpy(), C_dev[:M])


@pytest.mark.parametrize("prec", ["bf16x3", "exact"])
def test_async_host_calls_in_flight(libbpx, prec):
    """Three bpx_coded_matmul_host_async calls in flight on three streams
    (own buffers and workspaces, different masks), launched twice round:
    every result equals the synchronous call's, bit for bit."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 32, 64 * 32, 256, 512
    A, B = W.inputs(M, K, N, "normal", 73)
    P = bpx.PRECISIONS[prec]
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    masks = [torch.from_numpy(W.erasure_mask(code.n, 3, 300 + t)).pin_memory() for t in range(6)]
    want = []
    for t in range(6):
        C_dev, info = _run(bpx, code, A, B, h, P, masks[t].numpy())
        assert info[bpx.INFO_STATUS] == bpx.OK
        want.append(C_dev[:M])
    sets = []
    for j in range(3):
        sets.append(dict(dA=torch.empty((M, K), device="cuda"), dB=torch.empty((K, N), device="cuda"),
                         dm=torch.empty(code.n, dtype=torch.uint8, device="cuda"), dC=bpx.alloc_C(code, h, N),
                         ws=bpx.Workspace(code, M, N, K, h, P),
                         hC=torch.zeros((M, N), dtype=torch.float32).pin_memory(),
                         hinfo=torch.zeros(bpx.INFO_LEN, dtype=torch.int32).pin_memory(),
                         stream=torch.cuda.Stream()))
    for rnd in range(2):
        for j, S_ in enumerate(sets):
            t = 3 * rnd + j
            bpx.coded_matmul_host_async(code, hA, hB, h, P, masks[t], S_["hC"], S_["dA"], S_["dB"], S_["dm"],
                                        S_["dC"], S_["ws"], S_["hinfo"], stream=S_["stream"])
        for j, S_ in enumerate(sets):
            S_["stream"].synchronize()
            assert int(S_["hinfo"][bpx.INFO_STATUS]) == bpx.OK
            assert np.array_equal(S_["hC"].numpy(), want[3 * rnd + j])


@pytest.mark.parametrize("prec,cfg", [("bf16x3", 0), ("bf16", 0), ("fp32", 0), ("bf16x3", 16041), ("bf16x3", 8042),
                                      ("bf16", 16041), ("bf16x3", 16022), ("bf16x3", 16045), ("bf16x3", 8025),
                                      ("bf16x3", 16046), ("bf16", 16045), ("bf16", 8046), ("bf16x3", 8089),
                                      ("bf16", 16089), ("bf16x3", 8080), ("bf16", 4080), ("fp16x3", 0),
                                      ("fp16x3", 8080), ("fp16x3", 16021), ("fp16x3", 8049)])
def test_many_tiles_per_cta(libbpx, prec, cfg):
    """Bench-shaped code and block height at reduced N, K: ~600 output tiles
    of 128 x 256, so every persistent CTA runs several tiles and both TMEM
    accumulators and every barrier phase are exercised."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 128, 8192, 256, 2048
    A, B = W.inputs(M, K, N, "normal", 81)
    for t in range(2):
        m = W.erasure_mask(11, 3, 2000 + t)
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m, opts=bpx.default_opts(gemm_config=cfg))
        assert info[bpx.INFO_STATUS] == bpx.OK
        R, sch = _oracle_decode(ref, A, B, h, m)
        _check_blocks(C, R, ref, A, B, h, m, prec)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32", "bf16", "mxfp8", "fp16x3"])
def test_full_size_sysmoj_8192_sampled(libbpx, prec):
    """The benchmark workload at full size (A, B 8192 x 8192 N(0,1), h = 128,
    3 erased columns) in the benchmark's launch configuration; blocks of C
    checked against FP64 A_s B for the deepest sources and a direct one."""
    bpx = libbpx
    wl = W.WORKLOADS["sysmoj_8192"]
    code, ref = _pair(bpx, "sys8_3_8")
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    A, B = W.device_inputs(M, K, N, "normal", 2)
    m = W.erasure_mask(11, 3, wl["mask_seed_base"] + 7)
    ws = bpx.Workspace(code, M, N, K, h, bpx.PRECISIONS[prec])
    C, info = bpx.coded_matmul(code, A, B, h, bpx.PRECISIONS[prec], torch.from_numpy(m).cuda(), ws)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
    sch = o.wave_schedule(ref, o.surviving_cells(ref, list(np.nonzero(m)[0])))
    deep = sorted(range(64), key=lambda s: -sch.depth[s])[:2]
    direct = [s for s in range(64) if sch.depth[s] == 1][:1]
    Ah = A.cpu().numpy()
    Bf = B.cpu().numpy()
    Bh = Bf.astype(np.float64)
    nu = _nu(ref, Ah, Bf[:, :256], h, m)     # norms from a column slice
    for s in deep + direct:
        r = o.row_block(Ah, s, h) @ Bh
        c = C[s * h:(s + 1) * h].cpu().numpy()
        err = np.linalg.norm(c - r) / np.linalg.norm(r)
        assert err <= TOL[prec] * max(1.0, nu[s]), (prec, s, sch.depth[s], err, nu[s])


@pytest.mark.parametrize("trial", [21, 4])
def test_full_size_sysmoj_8192_flat_tolerance(libbpx, trial):
    """The accuracy target at full size: split-FP16x3 (the three tensor-core
    products of split-BF16x3 over fp16 halves) decodes the benchmark workload
    (A, B 8192 x 8192 N(0,1), h = 128, 3 erased columns, default launch
    configuration) with every checked block within a FLAT 1e-5 of FP64
    A_s B -- no propagation factor -- on the deepest sources and on
    directly copied ones.  Trials 21 and 4 of the benchmark's 100 masks
    reach depth 9; trial 21 (with 42) has the largest propagation factor
    of all 100 (32.6)."""
    bpx = libbpx
    wl = W.WORKLOADS["sysmoj_8192"]
    code, ref = _pair(bpx, "sys8_3_8")
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    A, B = W.device_inputs(M, K, N, "normal", 2)
    m = W.erasure_mask(11, 3, wl["mask_seed_base"] + trial)
    ws = bpx.Workspace(code, M, N, K, h, bpx.FP16X3)
    C, info = bpx.coded_matmul(code, A, B, h, bpx.FP16X3, torch.from_numpy(m).cuda(), ws)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
    sch = o.wave_schedule(ref, o.surviving_cells(ref, list(np.nonzero(m)[0])))
    deep = sorted(range(64), key=lambda s: -sch.depth[s])[:3]
    direct = [s for s in range(64) if sch.depth[s] == 1][:2]
    assert max(sch.depth) == 9
    Ah = A.cpu().numpy()
    Bh = B.cpu().numpy().astype(np.float64)
    for s in deep + direct:
        r = o.row_block(Ah, s, h) @ Bh
        c = C[s * h:(s + 1) * h].cpu().numpy()
        err = np.linalg.norm(c - r) / np.linalg.norm(r)
        assert err <= 1e-5, (s, sch.depth[s], err)


@pytest.mark.parametrize("name,h,M,K,N", [("table3", 8, 72, 200, 136), ("sys8_3_8", 4, 256, 520, 64)])
def test_fp16x3_wide_dynamic_range(libbpx, name, h, M, K, N):
    """Split-FP16x3 scales every coded row and every column of B by its own
    power of two: sources whose magnitudes differ by up to 2^80 and columns
    by up to 2^60 (far outside fp16's range unscaled) still decode within
    1e-5 times the propagation factor of the oracle's FP64 decode."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    rng = np.random.default_rng(7)
    A, B = W.inputs(M, K, N, "normal", 17)
    rows = np.repeat(2.0 ** rng.integers(-40, 41, size=(M + h - 1) // h), h)[:M]
    A = (A * rows[:, None]).astype(np.float32)
    B = (B * (2.0 ** rng.integers(-30, 31, size=N))[None, :]).astype(np.float32)
    for t in range(4):
        m = W.erasure_mask(code.n, t % (code.e + 1), 500 + t)
        C, info = _run(bpx, code, A, B, h, bpx.FP16X3, m)
        R, sch = _oracle_decode(ref, A, B, h, m)
        assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
        if sch.ok:
            _check_blocks(C, R, ref, A, B, h, m, "fp16x3")


@pytest.mark.parametrize("h,K,N", [(2, 264, 68), (1, 2056, 36), (3, 8, 4)])
def test_fp16x3_high_degree_code(libbpx, h, K, N):
    """A code whose cells hold 7.5 sources on average (Construction A
    [12, 9, 120]) takes the K-chunked split-FP16x3 encode -- unscaled sums
    staged, each row's exponent from a max over all its k-chunks, then the
    rescale in place -- with one ragged k-chunk (K = 264), with three
    (K = 2056), and with one 8-wide chunk per row (K = 8, 128 rows a CTA):
    small-integer inputs decode to A B bit for bit, normal inputs within 1e-5
    times the propagation factor of the oracle."""
    bpx = libbpx
    code, ref = bpx.Code.mojette_a(12, 9, 120), o.construction_a(12, 9, 120)
    assert len(code.cell_src) >= 4 * code.num_cells
    M = ref.num_sources * h - 1
    Ai, Bi = W.matrix((M, K), "int", 41), W.matrix((K, N), "int", 42)
    An, Bn = W.inputs(M, K, N, "normal", 43)
    exact = o.reference_product(Ai, Bi)
    for t in range(2):
        m = W.erasure_mask(12, 3, 70 + t)
        C, info = _run(bpx, code, Ai, Bi, h, bpx.FP16X3, m)
        assert info[bpx.INFO_STATUS] == bpx.OK
        assert np.array_equal(C[:M], exact), t
        C, info = _run(bpx, code, An, Bn, h, bpx.FP16X3, m)
        R, sch = _oracle_decode(ref, An, Bn, h, m)
        assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
        _check_blocks(C, R, ref, An, Bn, h, m, "fp16x3")


def test_fp16x3_zero_rows_columns_and_tiny_scales(libbpx):
    """Split-FP16x3's scale edge cases: a source block and a column of B that
    are all zero (exponent 0, products exactly zero), a row position scaled
    by 2^-100 in every source block (coded rows are sums of the same row
    position, so each keeps one scale) and a column of B by 2^100 (fp16
    holds neither unscaled): small-integer inputs under those scales stay
    exact, so C equals the oracle's FP64 decode bit for bit."""
    bpx = libbpx
    code, ref = _pair(bpx, "table3")
    h, K, N = 8, 64, 36
    M = ref.num_sources * h
    A = W.matrix((M, K), "int", 31).astype(np.float64)
    B = W.matrix((K, N), "int", 32).astype(np.float64)
    A[2 * h:3 * h] = 0.0            # a whole source block of zeros
    B[:, 5] = 0.0                   # a zero column
    A[3::h] *= 2.0 ** -100          # row position 3 of every block, near the bottom of FP32's range
    B[:, 7] *= 2.0 ** 100           # a column near the top
    A, B = A.astype(np.float32), B.astype(np.float32)
    for t in range(4):
        m = W.erasure_mask(code.n, t % (code.e + 1), 60 + t)
        C, info = _run(bpx, code, A, B, h, bpx.FP16X3, m)
        R, sch = _oracle_decode(ref, A, B, h, m)
        assert info[bpx.INFO_STATUS] == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
        for s in range(ref.num_sources):
            if sch.depth[s]:
                assert np.array_equal(C[s * h:(s + 1) * h], R[s * h:(s + 1) * h]), (t, s)


@pytest.mark.parametrize("prec", ["bf16x3", "mxfp8", "exact", "fp16x3"])
def test_steps_in_flight_on_two_streams(libbpx, prec):
    """The benchmark's launch configuration: steps in flight on two streams,
    each with its own workspace, C and info words, issued alternately with
    different masks -- every step's C equals the same step run alone on the
    default stream, bit for bit."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 32, 64 * 32, 512, 1024
    A, B = W.device_inputs(M, K, N, "normal", 81)
    P = bpx.PRECISIONS[prec]
    masks = [torch.from_numpy(W.erasure_mask(code.n, 3, 400 + t)).cuda() for t in range(6)]
    want = []
    ws0 = bpx.Workspace(code, M, N, K, h, P)
    for t in range(6):
        C, info = bpx.coded_matmul(code, A, B, h, P, masks[t], ws0)
        torch.cuda.synchronize()
        assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
        want.append(C.clone())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    wss = [bpx.Workspace(code, M, N, K, h, P) for _ in streams]
    got = [None] * 6
    torch.cuda.synchronize()
    for t in range(6):
        j = t % 2
        with torch.cuda.stream(streams[j]):
            got[t] = bpx.coded_matmul(code, A, B, h, P, masks[t], wss[j])
            if t >= 4:  # keep the last two in flight together
                continue
        if t % 2 == 1:
            for st in streams:
                st.synchronize()
    for st in streams:
        st.synchronize()
    for t in range(6):
        C, info = got[t]
        assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
        assert torch.equal(C, want[t]), (prec, t)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "fp32", "fp16x3"])
def test_construction_a_full_size_integer_bit_exact(libbpx, prec):
    """Workload mojA_16384 at full size (Construction A n=32, k=24, b=683,
    h=1: 16392 one-row sources, ~20.9k coded rows, A 16384 x 16384,
    B 16384 x 8192, 8 erased columns, hundreds of peel waves) with integer
    inputs in [-2, 2]: every product and every peeled row is an exact
    integer below 2^24, so the decoded rows must equal A B bit for bit --
    checked on the deepest rows, direct rows and random rows."""
    bpx = libbpx
    wl = W.WORKLOADS["mojA_16384"]
    code = bpx.Code.mojette_a(32, 24, 683)
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    A, B = W.device_inputs(M, K, N, "int", 40)
    m = torch.from_numpy(W.erasure_mask(32, 8, wl["mask_seed_base"])).cuda()
    ws = bpx.Workspace(code, M, N, K, h, bpx.PRECISIONS[prec])
    C, info = bpx.coded_matmul(code, A, B, h, bpx.PRECISIONS[prec], m, ws)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[bpx.INFO_STATUS] == bpx.OK
    assert inf[bpx.INFO_WAVES] > 100
    order, _rec, _i = bpx.schedule(code, m, bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32))
    order = order.cpu().numpy()
    rows = [int(s) for s, _r, d in order[::-1][:6] if s < M]          # deepest
    rows += [int(s) for s, _r, d in order if d == 1][:3]               # direct
    rows += list(np.random.default_rng(0).choice(M, 6, replace=False))
    Bh = B.cpu().numpy().astype(np.float64)
    Cn = C[rows].cpu().numpy()
    An = A[rows].cpu().numpy().astype(np.float64)
    ref = An @ Bh
    assert np.array_equal(Cn, ref), (prec, np.abs(Cn - ref).max())


@pytest.mark.parametrize("b", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3", "mxfp8", "exact"])
def test_construction_a_b_sweep(libbpx, b, prec):
    """Construction A n = 32, k = 24, e = 8 over the grid heights of the
    overhead-versus-conditioning sweep (b = 16: eps 14.4, depth 2; b = 32:
    depth 13; b = 64: depth 45, expansion coefficients up to ~8e4): every
    block within its tolerance times its propagation factor against the
    oracle's FP64 decode, exact slices bit for bit against the oracle's
    exact-slice decode."""
    bpx = libbpx
    code, ref = _pair(bpx, f"A32_24_{b}")
    h, K, N = 1, 512, 256
    M = ref.num_sources
    A, B = W.inputs(M, K, N, "uniform", 4)
    m = W.erasure_mask(32, 8, 4000)
    er = list(np.nonzero(m)[0])
    C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
    assert info[bpx.INFO_STATUS] == bpx.OK
    if prec == "exact":
        R, _Q, _s = o.exact_slice_coded_matmul(ref, A, B, h, er)
        assert np.array_equal(C[:M].view(np.uint32), R[:M].view(np.uint32))
        return
    R, sch = _oracle_decode(ref, A, B, h, m)
    TOLS = dict(TOL, mxfp8=6e-2)
    err = _rel_block_err(C, R, h, ref.num_sources)
    nu = _nu(ref, A, B, h, m)
    assert np.all(err <= TOLS[prec] * np.maximum(1.0, nu)), (prec, b, (err / (TOLS[prec] * np.maximum(1.0, nu))).max())


@pytest.mark.parametrize("wl_name,code_name", [("table1_logu", "table1"), ("table3_logu", "table3")])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp16x3"])
def test_precision_study_loguniform(libbpx, wl_name, code_name, prec):
    """Precision workload: magnitudes log-uniform on [1e-3, 1e3] with random
    signs (cancellation in the peel), every mask of <= 2 erased columns
    (Table I also its 3-column ones), compensated peel below depth 3;
    every block within its tolerance times its propagation factor."""
    bpx = libbpx
    wl = W.WORKLOADS[wl_name]
    code, ref = _pair(bpx, code_name)
    A, B = W.inputs(wl["M"], wl["K"], wl["N"], wl["dist"], wl["seed"])
    opts = bpx.default_opts(compensate_depth=3)
    for m in _masks(ref, 3 if code_name == "table1" else 2):
        C, info = _run(bpx, code, A, B, wl["h"], bpx.PRECISIONS[prec], m, opts=opts)
        R, sch = _oracle_decode(ref, A, B, wl["h"], m)
        assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
        _check_blocks(C, R, ref, A, B, wl["h"], m, prec)


TOL["mxfp8"] = 6e-2


@pytest.mark.parametrize("name,h,M,K,N", [
    ("table1", 16, 64, 256, 96),
    ("table3", 8, 70, 384, 200),
    ("table1", 130, 520, 128, 260),
])
@pytest.mark.parametrize("cfg", [0, 8001])
def test_mxfp8_exact_on_small_integers(libbpx, name, h, M, K, N, cfg):
    """MXFP8 (E4M3 with one UE8M0 scale per 32 K-elements): with degree-two
    codes and integers in [-2, 2] every coded 32-run scales onto E4M3 values
    exactly (|x| <= 4 becomes a multiple of 64 or 128 not above 448), so the
    decode is bit-exact -- with CTA-pair MMAs (0, the default) and 1-CTA MMAs (8001)."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    A = W.matrix((M, K), "int", 71)
    B = W.matrix((K, N), "int", 72)
    ref_C = o.reference_product(A, B)
    for t in range(5):
        m = W.erasure_mask(code.n, t % (code.e + 1), 300 + t)
        C, info = _run(bpx, code, A, B, h, bpx.MXFP8, m, opts=bpx.default_opts(gemm_config=cfg))
        assert info[bpx.INFO_STATUS] == bpx.OK
        assert np.array_equal(C[:M], ref_C), (name, m, cfg, np.abs(C[:M] - ref_C).max())


def test_mxfp8_table1_all_masks(libbpx):
    bpx = libbpx
    wl = W.WORKLOADS["table1_512"]
    code, ref = _pair(bpx, "table1")
    A, B = W.inputs(wl["M"], wl["K"], wl["N"], wl["dist"], wl["seed"])
    for m in _masks(ref, 3):
        C, info = _run(bpx, code, A, B, wl["h"], bpx.MXFP8, m)
        R, sch = _oracle_decode(ref, A, B, wl["h"], m)
        assert info[bpx.INFO_STATUS] == bpx.OK
        _check_blocks(C, R, ref, A, B, wl["h"], m, "mxfp8")


@pytest.mark.parametrize("cfg", [0, 8001])
def test_mxfp8_construction_a_tall_bit_exact(libbpx, cfg):
    """MXFP8 on a tall projection code: Construction A n = 12, k = 9, b = 120
    (1080 one-row sources, sigma = 9, so the peel takes its gathered form
    over many waves), three erased columns.  With ternary inputs every coded
    sum is an integer of magnitude <= 9, which a UE8M0-scaled E4M3 element
    holds exactly, and every product and peel step stays an exact FP32
    integer: the decode equals the oracle's, and A B, bit for bit."""
    bpx = libbpx
    code, ref = _pair(bpx, "A12_9_120")
    h, K, N = 1, 512, 256
    M = ref.num_sources * h
    A = W.matrix((M, K), "ternary", 61)
    B = W.matrix((K, N), "ternary", 62)
    ref_C = o.reference_product(A, B)
    for t in range(3):
        m = W.erasure_mask(code.n, 3, 700 + t)
        C, info = _run(bpx, code, A, B, h, bpx.MXFP8, m, opts=bpx.default_opts(gemm_config=cfg))
        R, sch = _oracle_decode(ref, A, B, h, m)
        assert sch.ok and info[bpx.INFO_STATUS] == bpx.OK
        assert max(sch.depth) > 5
        assert np.array_equal(C[:M], R[:M]), (t, np.abs(C[:M] - R[:M]).max())
        assert np.array_equal(C[:M], ref_C)


@pytest.mark.parametrize("cfg", [0, 8001, 4009])
def test_mxfp8_many_tiles(libbpx, cfg):
    """~600 tiles of 128 x 256 on the benchmark code: the single TMEM
    accumulator is drained and refilled on every tile of every CTA (1-CTA
    and CTA-pair forms)."""
    bpx = libbpx
    code, ref = _pair(bpx, "sys8_3_8")
    h, M, K, N = 128, 8192, 512, 2048
    A, B = W.inputs(M, K, N, "uniform", 91)
    m = W.erasure_mask(11, 3, 2001)
    C, info = _run(bpx, code, A, B, h, bpx.MXFP8, m, opts=bpx.default_opts(gemm_config=cfg))
    assert info[bpx.INFO_STATUS] == bpx.OK
    R, sch = _oracle_decode(ref, A, B, h, m)
    _check_blocks(C, R, ref, A, B, h, m, "mxfp8")


@pytest.mark.parametrize("name,h,M,K,N", [
    ("table3", 3, 26, 136, 200),       # ragged: M < S h, K and N not tile multiples, cells inside a tile
    ("sys8_3_8", 128, 8192, 512, 1024),  # the benchmark code: one cell per 128-row tile, many tiles per CTA
    ("A11_8_12", 1, 96, 264, 132),     # one-row sources of many cells in a tile, deep chains
    ("table1", 130, 520, 64, 8),       # blocks taller than a tile
    ("sys6_5_5", 40, 1200, 1000, 516),
])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_fused_encode_equals_materialized(libbpx, name, h, M, K, N, prec):
    """The encode fused into the GEMM's operand load forms the same coded
    sums (ascending sources, FP32 round-to-nearest) and the same bf16 split
    as the encode pass, so the decoded C is bit for bit the materialized
    path's -- for every tile shape the fused kernel takes."""
    bpx = libbpx
    code, ref = _pair(bpx, name)
    A, B = W.inputs(M, K, N, "normal", 23)
    for t, cfg in enumerate([0, 16080, 8020, 4040]):
        m = W.erasure_mask(code.n, min(code.e, t % 3), 900 + t)
        want, info0 = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m, opts=bpx.default_opts(gemm_config=cfg))
        got, info1 = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m,
                          opts=bpx.default_opts(gemm_config=cfg, fused_encode=1))
        assert info0[bpx.INFO_STATUS] == info1[bpx.INFO_STATUS]
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (name, prec, cfg)


def test_fused_encode_integer_bit_exact_and_refusals(libbpx):
    """Small-integer inputs through the fused encode: C equals A B bit for
    bit; a config other than the CTA-pair 64-wide tiles is refused
    (ERR_INVAL), and so is a precision the fused kernel does not build
    (ERR_UNSUPPORTED)."""
    bpx = libbpx
    code, ref = _pair(bpx, "B6_8_4_2")
    h, M, K, N = 2, 64, 32, 260
    A = W.matrix((M, K), "int", 21)
    B = W.matrix((K, N), "int", 22)
    for t in range(4):
        m = W.erasure_mask(code.n, t % (code.e + 1), 950 + t)
        C, info = _run(bpx, code, A, B, h, bpx.BF16X3, m, opts=bpx.default_opts(fused_encode=1))
        assert info[bpx.INFO_STATUS] == bpx.OK
        assert np.array_equal(C[:M], o.reference_product(A, B))
    m = W.erasure_mask(code.n, 1, 960)
    with pytest.raises(bpx.BpxError) as ei:
        _run(bpx, code, A, B, h, bpx.BF16X3, m, opts=bpx.default_opts(fused_encode=1, gemm_config=8081))
    assert ei.value.code == bpx.ERR_INVAL
    with pytest.raises(bpx.BpxError) as ei:
        _run(bpx, code, A, B, h, bpx.FP32, m, opts=bpx.default_opts(fused_encode=1))
    assert ei.value.code == bpx.ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "mxfp8", "exact"])
@pytest.mark.parametrize("cfg", [8083, 8084, 4087, 16088, -1])
def test_configs_without_a_tile_are_refused(libbpx, prec, cfg):
    """Tile codes 3, 4, 7, 8 (and negative configs) name no GEMM variant:
    the call fails with ERR_INVAL before anything is launched."""
    bpx = libbpx
    code, _ref = _pair(bpx, "table1")
    A, B = W.inputs(512, 256, 128, "uniform", 0)
    m = W.erasure_mask(5, 2, 1)
    with pytest.raises(bpx.BpxError) as ei:
        _run(bpx, code, A, B, 128, bpx.PRECISIONS[prec], m, opts=bpx.default_opts(gemm_config=cfg))
    assert ei.value.code == bpx.ERR_INVAL


@pytest.mark.parametrize("prec", ["bf16x3", "exact"])
def test_searched_code_on_the_gpu(libbpx, prec):
    """A code found by the library's search (a [5,3,2,4] array BP-XOR code
    with sigma = 2, meeting the straggler bound) runs through the whole GPU
    path: every pattern of two erased columns within tolerance of the
    oracle (bit-exact for exact slices)."""
    bpx = libbpx
    code, _ = bpx.Code.search(5, 3, 4, 2, iters=2000000, seed=5)
    assert code is not None
    ref = o.code_from_columns("found", 3, 4, code.columns())
    h, K, N = 24, 136, 68
    M = ref.num_sources * h
    A, B = W.inputs(M, K, N, "normal", 91)
    for m in _masks(ref, 2):
        er = list(np.nonzero(m)[0])
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
        assert info[bpx.INFO_STATUS] == bpx.OK
        if prec == "exact":
            R, _Q, _s = o.exact_slice_coded_matmul(ref, A, B, h, er)
            assert np.array_equal(C[:M].view(np.uint32), R[:M].view(np.uint32))
        else:
            R, _s = _oracle_decode(ref, A, B, h, m)
            _check_blocks(C, R, ref, A, B, h, m, prec)


# (n, k, b, sigma) -> (iters, seed, threads) of a library search that finds the code
_SEARCHED = {(6, 4, 4, 4): (1500000, 1, 4), (5, 3, 4, 6): (1500000, 1, 2), (6, 3, 4, 4): (6000000, 7, 8)}
_searched_cache = {}


def _searched(bpx, key):
    if key not in _searched_cache:
        iters, seed, threads = _SEARCHED[key]
        code, _ = bpx.Code.search(*key, iters=iters, seed=seed, threads=threads)
        assert code is not None and code.sigma == key[3]
        _searched_cache[key] = code
    return _searched_cache[key]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3", "exact"])
@pytest.mark.parametrize("which", ["xcode7", "xcode13", "search_6_4_4_4", "search_5_3_4_6", "search_6_3_4_4"])
def test_codes_of_degree_four_and_more_on_the_gpu(libbpx, prec, which):
    """Equal-height array BP-XOR codes with sigma >= 4 beyond Tables I / III --
    the X-code on 7 columns (sigma = 5, 35 sources) and on 13 (sigma = 11,
    143 sources), the [6, 4, 4] and [5, 3, 4] codes the search finds at
    sigma = 4 and 6, and the [6, 3, 4] code it finds at sigma = 4 that
    tolerates three erased columns -- through the whole GPU path under every
    pattern of n - k erased columns (a spread of 23 of the 78 pairs for the
    13-column X-code): within tolerance of the oracle per block (bit-exact
    for exact slices)."""
    bpx = libbpx
    if which.startswith("xcode"):
        p = int(which[5:])
        code, ref = bpx.Code.xcode(p), o.xcode(p)
    else:
        key = tuple(int(x) for x in which.split("_")[1:])
        code = _searched(bpx, key)
        ref = o.code_from_columns("found", key[1], key[2], code.columns())
    e = ref.n - ref.k
    h, K, N = (8, 136, 68) if ref.num_sources < 100 else (2, 72, 36)
    M = ref.num_sources * h - 3
    A, B = W.inputs(M, K, N, "normal", 93)
    pats = [m for m in _masks(ref, e) if m.sum() == e]
    if len(pats) > 24:  # the 13-column X-code: the first 12 pairs, then every sixth
        pats = pats[:12] + pats[12::6]
    for m in pats:
        er = list(np.nonzero(m)[0])
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m)
        assert info[bpx.INFO_STATUS] == bpx.OK
        if prec == "exact":
            R, _Q, _s = o.exact_slice_coded_matmul(ref, A, B, h, er)
            assert np.array_equal(C[:M].view(np.uint32), R[:M].view(np.uint32))
        else:
            R, _s = _oracle_decode(ref, A, B, h, m)
            _check_blocks(C, R, ref, A, B, h, m, prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("peel_ctas,comp", [(0, -1), (16, -1), (0, 0), (16, 0)])
def test_gathered_peel_waves(libbpx, prec, peel_ctas, comp):
    """A tall code (Construction A n=12, k=9, b=120: 1080 sources, ~118
    narrow waves), whose peel gathers each wave's blocks into shared memory.
    Integer inputs keep every product and every peeled row exact, so C must
    equal A B bit for bit: on the default grid (every wave in one round of
    the term buffer) and on a 16-CTA grid whose wide column slices (128
    float4 columns: 44 block rows per round) split the wider waves into
    several rounds, plain and with the compensated subtraction on every
    wave."""
    bpx = libbpx
    code, ref = bpx.Code.mojette_a(12, 9, 120), o.construction_a(12, 9, 120)
    h, K, N = 2, 64, 4096
    M = ref.num_sources * h - 3  # ragged: the last source block is partly padding
    A = W.matrix((M, K), "int", 91)
    B = W.matrix((K, N), "int", 92)
    exact = o.reference_product(A, B)
    opts = bpx.default_opts(peel_ctas=peel_ctas, compensate_depth=comp)
    for t in range(2):
        m = W.erasure_mask(12, 3, 5 + t)
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m, opts=opts)
        assert info[bpx.INFO_STATUS] == bpx.OK and info[bpx.INFO_WAVES] > 50
        assert np.array_equal(C[:M], exact), (prec, peel_ctas, comp, t)


def _ulps(a, b):
    """Distance in units in the last place between FP32 arrays (monotone
    integer map of the bit patterns)."""
    ai = a.view(np.int32).astype(np.int64)
    bi = b.view(np.int32).astype(np.int64)
    ai = np.where(ai < 0, -(ai & 0x7FFFFFFF), ai)
    bi = np.where(bi < 0, -(bi & 0x7FFFFFFF), bi)
    return np.abs(ai - bi)


@pytest.mark.parametrize("b", [120, 100])
def test_compensated_subtraction_rounds_once(libbpx, b):
    """The compensated peel (compensate_depth = 0) rounds each subtraction
    chain once: every decoded element equals the FP32 rounding of the exact
    value P_r - sum C_t of its own inputs (the products and the decoded
    blocks it subtracts), on a deep code with heavy cancellation (sources
    log-uniform in magnitude on [1e-3, 1e3], random signs; products rounded
    once from FP64 sums).  The plain peel, rounding after every subtraction,
    misses that rounding on most elements, so the check discriminates.
    Construction A n=12, k=9: b = 120 (1080 sources, gathered waves) and
    b = 100 (900 sources, register path)."""
    bpx = libbpx
    code, ref = bpx.Code.mojette_a(12, 9, b), o.construction_a(12, 9, b)
    h, N = 1, 256
    m = W.erasure_mask(12, 3, 5)
    sch = o.wave_schedule(ref, o.surviving_cells(ref, list(np.nonzero(m)[0])))
    assert sch.ok and sch.num_waves > 50
    rng = np.random.default_rng(7)
    S = ref.num_sources
    X = (np.exp(rng.uniform(np.log(1e-3), np.log(1e3), (S, N))) * rng.choice([-1, 1], (S, N))).astype(np.float32)
    P = np.zeros((len(ref.cells) * h, N), dtype=np.float32)
    for c in sorted(set(r for _s, r, _d in sch.order)):
        P[c] = np.sum(X[list(ref.cells[c])].astype(np.float64), axis=0).astype(np.float32)
    ws = bpx.Workspace(code, S * h, N, 8, h, bpx.FP32)
    bpx.schedule(code, torch.from_numpy(m).cuda(), ws)
    dP = torch.from_numpy(P).cuda()
    frac = {}
    for comp in (-1, 0):
        C = bpx.alloc_C(code, h, N)
        bpx.peel_decode(code, dP, N, h, C, ws, direct_written=False, opts=bpx.default_opts(compensate_depth=comp))
        Cn = C.cpu().numpy()
        worst, exact, total = 0, 0, 0
        for s, r, d in sch.order:
            v = P[r].astype(np.float64)
            for t in ref.cells[r]:
                if t != s:
                    v = v - Cn[t].astype(np.float64)
            u = _ulps(Cn[s], v.astype(np.float32))
            worst, exact, total = max(worst, int(u.max())), exact + int((u == 0).sum()), total + u.size
        frac[comp] = exact / total
        if comp == 0:
            assert worst <= 1 and frac[0] >= 0.999, (b, worst, frac[0])
    assert frac[-1] < 0.9, frac


@pytest.mark.parametrize("comp", [-1, 0])
def test_gathered_peel_with_register_waves(libbpx, comp):
    """Both peel forms in one launch: the tall code above extended by 306
    sources, each in one cell of a new column together with a source that
    the base code recovers at depth 6, so that wave 7 resolves more than 256
    positions (beyond the gather descriptors) and takes the register path
    while every other wave is gathered.  Integer inputs: C equals A B bit for
    bit, and the schedule equals the oracle's."""
    bpx = libbpx
    base = o.construction_a(12, 9, 120)
    er = list(np.nonzero(W.erasure_mask(12, 3, 5))[0])
    sch = o.wave_schedule(base, o.surviving_cells(base, er))
    d0 = 6
    at_d0 = [s for s in range(base.num_sources) if sch.depth[s] == d0]
    assert at_d0
    k, b = 9, 154                       # grid of 1386 source ids: 1080 base + 306 new
    extra = list(range(base.num_sources, b * k))
    columns = [[] for _ in range(13)]
    for c, cell in enumerate(base.cells):
        columns[base.col_of_cell[c]].append(tuple(cell))
    columns[12] = [(at_d0[i % len(at_d0)], s) for i, s in enumerate(extra)]
    code = bpx.Code.from_columns(13, k, b, columns, 3)
    ref = o.Code(name="mixed", n=13, k=k, b=b, num_sources=b * k,
                 cells=[tuple(sorted(c)) for col in columns for c in col],
                 col_of_cell=[j for j, col in enumerate(columns) for _ in col],
                 heights=[len(col) for col in columns], proj=[None] * 13, e=3)
    m = W.mask_from_columns(13, er)
    sch2 = o.wave_schedule(ref, o.surviving_cells(ref, er))
    assert sch2.ok and sum(1 for s in range(ref.num_sources) if sch2.depth[s] == d0 + 1) > 256
    h, K, N = 2, 64, 4096
    M = ref.num_sources * h - 3
    A = W.matrix((M, K), "int", 93)
    B = W.matrix((K, N), "int", 94)
    opts = bpx.default_opts(compensate_depth=comp)
    for prec in ("fp32", "bf16x3"):
        C, info = _run(bpx, code, A, B, h, bpx.PRECISIONS[prec], m, opts=opts)
        assert info[bpx.INFO_STATUS] == bpx.OK and info[bpx.INFO_WAVES] == sch2.num_waves
        assert np.array_equal(C[:M], o.reference_product(A, B)), (prec, comp)
    order, _rec, _i = bpx.schedule(code, torch.from_numpy(m).cuda(), bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32))
    assert [tuple(int(x) for x in r) for r in order.cpu().numpy()] == [tuple(x) for x in sch2.order]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "mxfp8", "exact", "fp16x3", "bf16x3-fused"])
def test_degenerate_shapes(libbpx, prec):
    """Edge cases of the path: M = 0 (every source block is zero padding, A
    empty: C must be zero), the smallest blocks (h = 1, N = 4, the smallest K
    the precision takes), and no erasure at all on a systematic code (the
    decode is a copy of the data cells' products) -- each bit for bit on
    small integers, with the plan's status OK."""
    bpx = libbpx
    fused = prec.endswith("-fused")   # the encode fused into the GEMM's operand load
    P = bpx.PRECISIONS[prec.replace("-fused", "")]
    kmin = 128 if prec == "mxfp8" else 8
    opts = bpx.default_opts(fused_encode=int(fused))
    # M = 0
    code = bpx.Code.table1()
    A = torch.empty((0, kmin), device="cuda")
    B = torch.from_numpy(W.matrix((kmin, 4), "int", 71)).cuda()
    ws = bpx.Workspace(code, 0, 4, kmin, 1, P)
    C, info = bpx.coded_matmul(code, A, B, 1, P, torch.from_numpy(W.erasure_mask(5, 3, 1)).cuda(), ws, opts=opts)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
    assert C.shape == (4, 4) and not C.abs().sum().item()
    # the smallest blocks: h = 1, N = 4
    An = W.matrix((4, kmin), "int", 72)
    Bn = W.matrix((kmin, 4), "int", 73)
    for t in range(3):
        m = W.erasure_mask(5, 3, 10 + t)
        Cn, inf = _run(bpx, code, An, Bn, 1, P, m, opts=opts)
        assert inf[bpx.INFO_STATUS] == bpx.OK
        assert np.array_equal(Cn, o.reference_product(An, Bn)), (prec, t)
    # no erasure on a systematic code
    code_s = bpx.Code.systematic(4, 2, 3)
    As = W.matrix((24, 2 * kmin), "int", 74)
    Bs = W.matrix((2 * kmin, 8), "int", 75)
    Cs, inf = _run(bpx, code_s, As, Bs, 2, P, np.zeros(6, dtype=np.uint8), opts=opts)
    assert inf[bpx.INFO_STATUS] == bpx.OK and inf[bpx.INFO_WAVES] == 1
    assert np.array_equal(Cs, o.reference_product(As, Bs))
