"""GPU path under processor-level stragglers (Section IV): cell-level erasure
masks and the straggler-time emulation against the oracle."""
import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _codes(bpx):
    return [(bpx.Code.table1(), o.table1(), 16), (bpx.Code.table3(), o.table3(), 8),
            (bpx.Code.systematic(8, 3, 8), o.systematic_mojette(8, 3, 8), 4),
            (bpx.Code.mojette_a(7, 4, 10), o.construction_a(7, 4, 10), 2)]


def test_cell_mask_schedule_bit_exact(libbpx):
    """Random cell subsets (decodable or not): peel order, resolvers, depths
    and the recovered set equal the oracle's wave schedule over the arrived
    cells."""
    bpx = libbpx
    rng = np.random.default_rng(6)
    for code, ref, _h in _codes(bpx):
        ws = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32)
        for _ in range(12):
            keep = rng.random(code.num_cells) < rng.uniform(0.5, 0.95)
            mask = torch.from_numpy((~keep).astype(np.uint8)).cuda()
            order, rec, info = bpx.schedule(code, mask, ws, cells=True)
            sch = o.wave_schedule(ref, [c for c in range(ref.num_cells) if keep[c]])
            got = [tuple(int(x) for x in r) for r in order.cpu().numpy() if r[0] >= 0]
            assert got == [tuple(t) for t in sch.order]
            assert list(rec.cpu().numpy().astype(bool)) == [bool(d) for d in sch.depth]
            assert int(info[bpx.INFO_STATUS]) == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_emulated_stragglers_decode(libbpx, prec):
    """The emulator's first decodable arrival set, run on the GPU with a
    cell-level mask: every block within tolerance of the oracle's decode
    over the same cells (1e-5 times the block's propagation factor)."""
    bpx = libbpx
    from paper_1904_11563_gb300 import straggler as st
    P = bpx.PRECISIONS[prec]
    for code, ref, h in _codes(bpx)[1:3]:
        M, K, N = ref.num_sources * h, 256, 128
        A, B = W.inputs(M, K, N, "normal", 5)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        for seed in range(4):
            X = W.exponential_draws(code.num_cells, 1.0, 100 + seed)
            r = st.emulate(code, dA, dB, h, P, X)
            torch.cuda.synchronize()
            assert r["first"] > 0 and int(r["info"][bpx.INFO_STATUS]) == bpx.OK
            arrived = [c for c in range(code.num_cells) if not r["cell_mask"][c]]
            R, sch = o.coded_matmul_cells(ref, A, B, h, arrived)
            assert sch.ok
            Cn = r["C"].cpu().numpy()
            used = sorted(set(rr for _s, rr, _d in sch.order))
            Pp = o.coded_products(ref, A, B, h, used)
            nu = o.propagation(ref, sch, Pp, o.peel_decode(ref, Pp, sch, h, N))
            for s in range(ref.num_sources):
                blk, want = Cn[s * h:(s + 1) * h], R[s * h:(s + 1) * h]
                err = np.linalg.norm(blk - want) / np.linalg.norm(want)
                assert err <= 1e-5 * max(1.0, nu[s]), (seed, s, err, nu[s])


def test_emulated_stragglers_exact(libbpx):
    """Exact slices under processor-level stragglers: every block
    bit-identical to the oracle's exact-slice product of the source, whatever
    set of processors arrived first."""
    bpx = libbpx
    from paper_1904_11563_gb300 import straggler as st
    code, ref = bpx.Code.systematic(8, 3, 8), o.systematic_mojette(8, 3, 8)
    h, K, N = 8, 136, 64
    M = ref.num_sources * h
    A, B = W.inputs(M, K, N, "normal", 9)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    direct = {s: o.exact_slice_block(A, B, s, h, ref.sigma)[0] for s in range(ref.num_sources)}
    for seed in range(3):
        X = W.exponential_draws(code.num_cells, 1.0, 300 + seed)
        r = st.emulate(code, dA, dB, h, bpx.EXACT, X)
        torch.cuda.synchronize()
        assert int(r["info"][bpx.INFO_STATUS]) == bpx.OK
        Cn = r["C"].cpu().numpy()
        for s in range(ref.num_sources):
            assert np.array_equal(Cn[s * h:(s + 1) * h].view(np.uint32), direct[s].view(np.uint32))


def test_host_entry_with_cell_mask(libbpx):
    """bpx_coded_matmul_host copies a num_cells-byte mask when mask_cells = 1."""
    bpx = libbpx
    code, ref = bpx.Code.table3(), o.table3()
    h, M, K, N = 16, 144, 64, 32
    A, B = W.inputs(M, K, N, "uniform", 3)
    keep = [c for c in range(ref.num_cells) if c not in (1, 4, 8, 12)]
    mask = np.ones(ref.num_cells, dtype=np.uint8)
    mask[keep] = 0
    ws = bpx.Workspace(code, M, N, K, h, bpx.FP32)
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    hm = torch.from_numpy(mask).pin_memory()
    hC = torch.zeros((M, N)).pin_memory()
    dA, dB = torch.empty((M, K), device="cuda"), torch.empty((K, N), device="cuda")
    dm = torch.empty(ref.num_cells, dtype=torch.uint8, device="cuda")
    dC = bpx.alloc_C(code, h, N)
    rc, info = bpx.coded_matmul_host(code, hA, hB, h, bpx.FP32, hm, hC, dA, dB, dm, dC, ws,
                                     opts=bpx.default_opts(mask_cells=1))
    R, sch = o.coded_matmul_cells(ref, A, B, h, keep)
    assert rc == (bpx.OK if sch.ok else bpx.ERR_UNDECODABLE)
    used = sorted(set(rr for _s, rr, _d in sch.order))
    Pp = o.coded_products(ref, A, B, h, used)
    nu = o.propagation(ref, sch, Pp, o.peel_decode(ref, Pp, sch, h, N))
    for s in range(ref.num_sources):
        if sch.depth[s]:
            want = R[s * h:(s + 1) * h]
            err = np.linalg.norm(hC.numpy()[s * h:(s + 1) * h] - want) / np.linalg.norm(want)
            assert err <= 1e-5 * max(1.0, nu.get(s, 1.0)), (s, err, nu.get(s, 1.0))


def test_online_recovery_matches_oracle(libbpx):
    """Sources recovered from each run of the decodable set's arrivals (the
    GPU schedule over each prefix of the arrival order) equal the oracle's
    wave schedule over the same prefixes, and sum to every source."""
    bpx = libbpx
    from paper_1904_11563_gb300 import straggler as st
    code, ref = bpx.Code.mojette_a(12, 9, 120), o.construction_a(12, 9, 120)
    ws = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32)
    for seed in (6001, 6003):
        T = st.task_times(code, W.exponential_draws(code.num_cells, 1.0, seed))
        order, first, _t, _rec = st.arrivals(code, T)
        got = st.online_recovery(code, order, first, ws, 8, device=torch.device("cuda"))
        want = []
        for j in range(8):
            n_j = (j + 1) * first // 8
            want.append(sum(o.wave_schedule(ref, sorted(int(c) for c in order[:n_j])).recovered))
        assert list(got) == list(np.diff([0] + want)) and int(got.sum()) == ref.num_sources
