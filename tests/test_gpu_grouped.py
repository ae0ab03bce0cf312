"""Grouped runs (bpx_grouped_run): many coded multiplications, each with its
own code, shapes and erasure mask, in one launch per stage -- checked job by
job against the FP64 oracle, replayed from a CUDA graph, and re-planned by
the tile autotuner."""
import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _codes(bpx, spec):
    kind, *args = spec["code"]
    if kind == "table1":
        return bpx.Code.table1(), o.table1()
    if kind == "table3":
        return bpx.Code.table3(), o.table3()
    if kind == "systematic":
        k, e, b = args
        return bpx.Code.systematic(k, e, b), o.systematic_mojette(k, e, b)
    n, k, b = args
    return bpx.Code.mojette_a(n, k, b), o.construction_a(n, k, b)


def _build(bpx, specs, dist, seed):
    jobs, refs = [], []
    for i, sp in enumerate(specs):
        code, ref = _codes(bpx, sp)
        A = W.matrix((sp["M"], sp["K"]), dist, seed + 2 * i)
        B = W.matrix((sp["K"], sp["N"]), dist, seed + 2 * i + 1)
        m = W.erasure_mask(code.n, sp["e"], sp["mask_seed"])
        jobs.append(dict(code=code, A=torch.from_numpy(A).cuda(), B=torch.from_numpy(B).cuda(),
                         C=bpx.alloc_C(code, sp["h"], sp["N"]), mask=torch.from_numpy(m).cuda(),
                         info=torch.zeros(16, dtype=torch.int32, device="cuda"), h=sp["h"]))
        refs.append((ref, A, B, m))
    return jobs, refs


def _check_exact(bpx, jobs, refs):
    for j, (ref, A, B, m) in zip(jobs, refs):
        assert j["info"].cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
        C = j["C"][:A.shape[0]].cpu().numpy()
        assert np.array_equal(C, o.reference_product(A, B))


SPECS = W.batch_specs(14, 5, lo=128, hi=640)


def test_specs_cover_every_family():
    kinds = {s["code"][0] for s in W.batch_specs(64, 5)}
    assert kinds == {"table1", "table3", "systematic", "mojette_a"}


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_grouped_integer_bit_exact(libbpx, prec):
    bpx = libbpx
    jobs, refs = _build(bpx, SPECS, "int", 100)
    G = bpx.Group(jobs, bpx.PRECISIONS[prec])
    G.run()
    torch.cuda.synchronize()
    _check_exact(bpx, jobs, refs)


def test_grouped_random_within_tolerance(libbpx):
    bpx = libbpx
    jobs, refs = _build(bpx, SPECS[:8], "normal", 200)
    G = bpx.Group(jobs, bpx.BF16X3)
    G.run()
    torch.cuda.synchronize()
    for j, (ref, A, B, m) in zip(jobs, refs):
        h = j["h"]
        cells = o.surviving_cells(ref, list(np.nonzero(m)[0]))
        sch = o.wave_schedule(ref, cells)
        used = sorted(set(r for _s, r, _d in sch.order))
        P = o.coded_products(ref, A, B, h, used)
        Cd = o.peel_decode(ref, P, sch, h, B.shape[1])
        nu = o.propagation(ref, sch, P, Cd)
        C = j["C"].cpu().numpy()
        for s, blk in Cd.items():
            err = np.linalg.norm(C[s * h:(s + 1) * h] - blk) / max(np.linalg.norm(blk), 1e-30)
            assert err <= 1e-5 * max(1.0, nu[s]), (ref.name, s, err, nu[s])


def test_graph_replay_and_new_masks(libbpx):
    """The captured graph reads the masks at every replay: changing them in
    place changes the decode, and each replay is exact."""
    bpx = libbpx
    jobs, refs = _build(bpx, SPECS, "int", 300)
    G = bpx.Group(jobs, bpx.BF16X3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G.graph_launch()
        stream.synchronize()
        _check_exact(bpx, jobs, refs)
        for j, r in zip(jobs, refs):
            j["C"].zero_()
            new = W.erasure_mask(j["code"].n, int(r[3].sum()), 999 + j["code"].n)
            j["mask"].copy_(torch.from_numpy(new))
        new_refs = [(ref, A, B, j["mask"].cpu().numpy()) for j, (ref, A, B, _m) in zip(jobs, refs)]
        G.graph_launch()
        stream.synchronize()
    _check_exact(bpx, jobs, new_refs)


def test_autotune_replans_and_stays_exact(libbpx):
    bpx = libbpx
    jobs, refs = _build(bpx, SPECS, "int", 400)
    G = bpx.Group(jobs, bpx.BF16X3)
    best, ms = G.autotune([16042, 16022, 8041, 16045, 8046])
    assert best in (16042, 16022, 8041, 16045, 8046) and ms > 0
    for j in jobs:
        j["C"].zero_()
    G.run()
    torch.cuda.synchronize()
    _check_exact(bpx, jobs, refs)
    # every other tile shape, re-planned, stays exact
    for cfg in (16041, 16042, 16045, 16046, 16049, 16040):
        G.set_config(cfg)
        for j in jobs:
            j["C"].zero_()
        G.run()
        torch.cuda.synchronize()
        _check_exact(bpx, jobs, refs)


def test_single_job_autotune_and_tile_configs(libbpx):
    bpx = libbpx
    code, ref = bpx.Code.systematic(8, 3, 8), o.systematic_mojette(8, 3, 8)
    h, M, K, N = 128, 8192, 256, 1000
    A = W.matrix((M, K), "int", 51)
    B = W.matrix((K, N), "int", 52)
    m = torch.from_numpy(W.erasure_mask(11, 3, 3)).cuda()
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ws = bpx.Workspace(code, M, N, K, h, bpx.BF16X3)
    best, ms = bpx.autotune(code, dA, dB, h, bpx.BF16X3, m, ws, configs=[16041, 16022, 4012, 32082, 16045, 8026])
    assert best in (16041, 16022, 4012, 32082, 16045, 8026)
    refC = o.reference_product(A, B)
    for cfg in (16041, 16022, 4012, 32082, 16045, 8026, 8089, 4019, best):
        C, info = bpx.coded_matmul(code, dA, dB, h, bpx.BF16X3, m, ws, opts=bpx.default_opts(gemm_config=cfg))
        torch.cuda.synchronize()
        assert np.array_equal(C[:M].cpu().numpy(), refC), cfg


def test_peel_autotune_replans_and_stays_exact(libbpx):
    """The grouped peel-schedule autotuner: the chosen plan (CTAs per job) is
    one of the candidates, and runs and graph replays under it -- and under
    every other candidate -- stay bit-exact."""
    bpx = libbpx
    jobs, refs = _build(bpx, SPECS, "int", 500)
    G = bpx.Group(jobs, bpx.BF16X3)
    cands = [19, 152, 608, 2432]
    best, ms = G.autotune_peel(cands)
    assert best in cands and ms > 0
    for j in jobs:
        j["C"].zero_()
    G.run()
    torch.cuda.synchronize()
    _check_exact(bpx, jobs, refs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for t in cands:
            G.autotune_peel([t])           # re-plan to this one target
            for j in jobs:
                j["C"].zero_()
            G.graph_launch()               # the graph is captured again for the new plan
            stream.synchronize()
            _check_exact(bpx, jobs, refs)


# Tall projection codes (more than 1024 sources: hundreds of peel waves),
# whose peels take the gathered form beside the register-path peels of the
# small jobs in the same grouped run.
TALL = [dict(code=("mojette_a", 12, 9, 120), M=2160, N=512, K=256, h=2, e=3, n=12, mask_seed=11),
        dict(code=("mojette_a", 16, 12, 100), M=1197, N=768, K=128, h=1, e=4, n=16, mask_seed=12)]


@pytest.mark.parametrize("comp", [-1, 0])
def test_grouped_tall_jobs_gathered_peel(libbpx, comp):
    """A batch mixing two tall Construction A jobs with six small jobs: the
    grouped peel runs the tall ones in its gathered form and the rest on the
    register path (two launches side by side), plain and compensated;
    bit-exact on integer inputs in a run, in graph replays, and under each
    peel plan the autotuner tries (wider column slices split waves into
    rounds)."""
    bpx = libbpx
    for sp in TALL:
        assert o.construction_a(*sp["code"][1:]).num_sources >= 1024
    jobs, refs = _build(bpx, TALL + SPECS[:6], "int", 600)
    G = bpx.Group(jobs, bpx.BF16X3)
    opts = bpx.default_opts(compensate_depth=comp)
    G.run(opts)
    torch.cuda.synchronize()
    _check_exact(bpx, jobs, refs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for t in (2, 19, 608):
            G.autotune_peel([t])
            for j in jobs:
                j["C"].zero_()
            G.graph_launch(opts)
            stream.synchronize()
            _check_exact(bpx, jobs, refs)


def test_single_job_peel_autotune(libbpx):
    """bpx_autotune_peel: the fastest peel CTA count among the candidates;
    the tuned run and the runs under each candidate stay bit-exact."""
    bpx = libbpx
    code = bpx.Code.systematic(8, 3, 8)
    h, M, K, N = 128, 8192, 256, 1000
    A = W.matrix((M, K), "int", 61)
    B = W.matrix((K, N), "int", 62)
    refC = o.reference_product(A, B)
    m = torch.from_numpy(W.erasure_mask(11, 3, 7)).cuda()
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for prec in (bpx.BF16X3, bpx.FP32):
        ws = bpx.Workspace(code, M, N, K, h, prec)
        C = bpx.alloc_C(code, h, N)
        cands = [8, 76, 152, 1216]
        best, ms = bpx.autotune_peel(code, dA, dB, h, prec, m, ws, C=C, ctas=cands)
        torch.cuda.synchronize()
        assert best in cands and ms > 0
        assert np.array_equal(C[:M].cpu().numpy(), refC)
        for c in cands + [best]:
            C2, info = bpx.coded_matmul(code, dA, dB, h, prec, m, ws, opts=bpx.default_opts(peel_ctas=c))
            torch.cuda.synchronize()
            assert info.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
            assert np.array_equal(C2[:M].cpu().numpy(), refC), (prec, c)
