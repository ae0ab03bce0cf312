"""Host-side checks of libbpx (no GPU needed): the library loads, exports
every entry point include/bpx.h declares, and builds code graphs identical
to the oracle's (bit-exact integer work)."""
import ctypes
import os
import re

import numpy as np

import pytest

from oracle import bpx_oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bpx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bpx_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(libbpx):
    names = _declared()
    assert len(names) >= 14
    L = ctypes.CDLL(libbpx.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


CASES = [
    ("table1", lambda b: b.Code.table1(), lambda: o.table1()),
    ("table3", lambda b: b.Code.table3(), lambda: o.table3()),
    ("sys8_3_8", lambda b: b.Code.systematic(8, 3, 8), lambda: o.systematic_mojette(8, 3, 8)),
    ("sys12_6_4", lambda b: b.Code.systematic(12, 4, 6), lambda: o.systematic_mojette(12, 4, 6)),
    ("sys6_5_5", lambda b: b.Code.systematic(6, 5, 5), lambda: o.systematic_mojette(6, 5, 5)),
    ("A5_3_4", lambda b: b.Code.mojette_a(5, 3, 4), lambda: o.construction_a(5, 3, 4)),
    ("A8_6_6", lambda b: b.Code.mojette_a(8, 6, 6), lambda: o.construction_a(8, 6, 6)),
    ("A11_8_12", lambda b: b.Code.mojette_a(11, 8, 12), lambda: o.construction_a(11, 8, 12)),
    ("A9_3_2", lambda b: b.Code.mojette_a(9, 3, 2), lambda: o.construction_a(9, 3, 2)),
    ("A32_24_683", lambda b: b.Code.mojette_a(32, 24, 683), lambda: o.construction_a(32, 24, 683)),
    ("B5_6_5_1", lambda b: b.Code.mojette_b(5, 6, 5, 1), lambda: o.construction_b(5, 6, 5, 1)),
    ("B6_8_4_2", lambda b: b.Code.mojette_b(6, 8, 4, 2), lambda: o.construction_b(6, 8, 4, 2)),
    ("B12_20_50_2", lambda b: b.Code.mojette_b(12, 20, 50, 2), lambda: o.construction_b(12, 20, 50, 2)),
]


@pytest.mark.parametrize("name,mk_lib,mk_orc", CASES, ids=[c[0] for c in CASES])
def test_code_graph_matches_oracle(libbpx, name, mk_lib, mk_orc):
    c = mk_lib(libbpx)
    r = mk_orc()
    assert (c.n, c.k, c.b, c.e) == (r.n, r.k, r.b, r.e)
    assert c.num_sources == r.num_sources
    assert c.num_cells == r.num_cells
    assert c.cells == [tuple(x) for x in r.cells]
    assert list(c.col_of_cell) == list(r.col_of_cell)
    assert list(c.heights) == list(r.heights)
    assert c.sigma == r.sigma
    assert c.eps == pytest.approx(r.eps(), rel=1e-12, abs=1e-15)
    for j, pq in enumerate(r.proj):
        if pq is not None:
            assert (c.proj_p[j], c.proj_q[j]) == pq


def test_invalid_parameters_raise(libbpx):
    with pytest.raises(libbpx.BpxError) as ei:
        libbpx.Code(libbpx.TABLE1, 5, 3, 2)
    assert ei.value.code == libbpx.ERR_INVAL and "Table I" in str(ei.value)
    with pytest.raises(libbpx.BpxError):
        libbpx.Code(libbpx.MOJETTE_A, 3, 4, 5)       # n < k
    with pytest.raises(libbpx.BpxError):
        libbpx.Code(libbpx.SYSTEMATIC, 8, 8, 4)       # no parity
    with pytest.raises(libbpx.BpxError):
        libbpx.Code(libbpx.MOJETTE_A, 5, 3, 4, e=1)   # wrong e
    with pytest.raises(libbpx.BpxError):
        libbpx.Code(99, 5, 3, 4)


def test_workspace_bytes_grow_with_shapes(libbpx):
    c = libbpx.Code.systematic(8, 3, 8)
    w0 = libbpx.workspace_bytes(c, 0, 0, 0, 1, libbpx.FP32)
    w1 = libbpx.workspace_bytes(c, 1024, 256, 256, 128, libbpx.FP32)
    w2 = libbpx.workspace_bytes(c, 1024, 256, 256, 128, libbpx.BF16X3)
    assert 0 < w0 < w1 < w2
    # products: num_cells * h * N floats
    assert w1 - w0 >= c.num_cells * 128 * 256 * 4


def test_build_info(libbpx):
    assert b"sm_103a" in libbpx.lib().bpx_build_info()


def test_exact_params_match_oracle(libbpx):
    """bpx_exact_params (host only) gives the digit width, plane count and
    fixed-point bits the oracle derives from sigma, and refuses codes or K
    where exactness could not be guaranteed."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    cases = [(bpx.Code.table1(), o.table1()), (bpx.Code.table3(), o.table3()),
             (bpx.Code.systematic(8, 3, 8), o.systematic_mojette(8, 3, 8)),
             (bpx.Code.mojette_a(32, 24, 683), None), (bpx.Code.mojette_a(7, 4, 10), o.construction_a(7, 4, 10)),
             (bpx.Code.mojette_b(6, 8, 4, 2), o.construction_b(6, 8, 4, 2))]
    for code, ref in cases:
        sigma = ref.sigma if ref is not None else code.sigma
        p = bpx.exact_params(code, 1000)
        assert (p["w"], p["S"], p["bits"]) == o.exact_slice_params(sigma)
        assert p["Kp"] == 1024 and p["seg"] % 64 == 0 and p["seg"] > 0
        # a segment's absolute sum stays below 2^23
        assert p["seg"] * sigma * 2 ** (2 * (p["w"] - 1)) <= 2 ** 23
    with pytest.raises(bpx.BpxError) as e:
        bpx.exact_params(bpx.Code.table1(), 65536)       # int32 diagonal sums could overflow
    assert e.value.code == bpx.ERR_UNSUPPORTED
    big = bpx.Code.systematic(80, 1, 2)                  # a parity of 80 sources: digits below 3 bits
    assert big.sigma > 64
    with pytest.raises(bpx.BpxError) as e:
        bpx.exact_params(big, 64)
    assert e.value.code == bpx.ERR_UNSUPPORTED
    with pytest.raises(bpx.BpxError):
        bpx.exact_params(bpx.Code.table1(), 12)          # K % 8 != 0
    # the workspace holds S int32 planes, the digit planes, scales and int64 blocks
    code = bpx.Code.systematic(8, 3, 8)
    need = bpx.workspace_bytes(code, 1024, 256, 512, 16, bpx.EXACT)
    S = 4
    assert need >= S * code.num_cells * 16 * 256 * 4 + (code.num_cells * 16 + 256) * S * 512 * 2 \
        + code.num_sources * 16 * 256 * 8


def test_terms_2d_match_oracle(libbpx):
    """The library's factoring of every cell for the two-dimensional scheme
    (an independent C++ implementation) gives the oracle's product count per
    cell, hence the paper's gray-cell counts for Tables I and III."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    cases = [(bpx.Code.table1(), o.table1()), (bpx.Code.table3(), o.table3()),
             (bpx.Code.systematic(8, 3, 8), o.systematic_mojette(8, 3, 8)),
             (bpx.Code.mojette_a(7, 4, 10), o.construction_a(7, 4, 10)),
             (bpx.Code.mojette_b(6, 8, 4, 2), o.construction_b(6, 8, 4, 2))]
    for code, ref in cases:
        per, summ = bpx.terms_2d(code)
        want = [len(o.terms_2d(ref, c)) for c in range(ref.num_cells)]
        assert list(per) == want
        assert summ["total"] == sum(want)
        assert summ["gray"] == len(o.gray_cells_2d(ref))
        A_ops = {Z for c in range(ref.num_cells) for Z, _L in o.terms_2d(ref, c)}
        B_ops = {L for c in range(ref.num_cells) for _Z, L in o.terms_2d(ref, c)}
        assert summ["a_operands"] == len(A_ops) and summ["b_operands"] == len(B_ops)
    assert bpx.terms_2d(bpx.Code.table1())[1]["gray"] == 2
    assert bpx.terms_2d(bpx.Code.table3())[1]["gray"] == 6
    code = bpx.Code.systematic(8, 3, 8)
    assert bpx.lib().bpx_workspace_bytes_2d(code.handle, 8192, 8192, 8192, 1024, bpx.BF16X3) > 0


def test_first_decodable_matches_oracle(libbpx):
    """The library's online peel over arriving cells (C++) gives the oracle's
    first decodable prefix and the same number of recovered sources after
    every arrival."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    cases = [(bpx.Code.table1(), o.table1()), (bpx.Code.table3(), o.table3()),
             (bpx.Code.systematic(6, 3, 4), o.systematic_mojette(6, 3, 4)),
             (bpx.Code.mojette_a(7, 4, 5), o.construction_a(7, 4, 5))]
    rng = np.random.default_rng(4)
    for code, ref in cases:
        for _ in range(10):
            order = rng.permutation(code.num_cells).astype(np.int32)
            first, rec = bpx.first_decodable(code, order)
            assert first == o.first_decodable(ref, list(order))
            for i in range(0, code.num_cells, max(1, code.num_cells // 7)):
                assert rec[i] == len(o.sequential_peel(ref, list(order[:i + 1])))
    with pytest.raises(bpx.BpxError):
        bpx.first_decodable(bpx.Code.table1(), np.array([0, 0], dtype=np.int32))


def test_straggler_arrivals_match_brute_force(libbpx):
    """T_par from the emulator (task times sigma_c X_c, first decodable
    arrival prefix) equals the oracle's brute-force min over decodable sets
    of the latest arrival, for the same draws."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    from paper_1904_11563_gb300 import straggler as st
    from paper_1904_11563_gb300 import workloads as W
    for code, ref in [(bpx.Code.table1(), o.table1()), (bpx.Code.table3(), o.table3())]:
        for seed in range(6):
            X = W.exponential_draws(code.num_cells, 1.5, seed)
            T = st.task_times(code, X)
            _order, first, t_par, _rec = st.arrivals(code, T)
            Tref = o.task_times(ref, 1.5, None, X=X)
            assert np.array_equal(T, Tref)
            assert t_par == o.parallel_task_time_brute(ref, Tref)


def test_overlap_bound_counts_and_the_peeling_cliff(libbpx):
    """The emulator's overlap bound -- per run of the decodable set's
    arrivals, the peel positions whose resolver and subtracted blocks have
    all arrived -- matches a count by closure (a position is ready after run
    j when every resolver in its dependency tree arrived by then), on the
    oracle's plan for Construction A [12, 9, 120] under the task-time model.
    And it shows why products and peel barely overlap on such codes: most
    non-direct positions need the last eighth of the arrivals, and even an
    arrival-ordered peel (resolvers among the cells in so far) recovers most
    sources only then (the peeling avalanche at the decodability threshold)."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    from paper_1904_11563_gb300 import straggler as st
    from paper_1904_11563_gb300 import workloads as W
    code, ref = bpx.Code.mojette_a(12, 9, 120), o.construction_a(12, 9, 120)
    nch = 8
    for seed in (6001, 6002):
        T = st.task_times(code, W.exponential_draws(code.num_cells, 1.0, seed))
        order, first, _t, _rec = st.arrivals(code, T)
        arrived = sorted(int(c) for c in order[:first])
        sch = o.wave_schedule(ref, arrived)
        assert sch.ok
        po = np.full((ref.num_sources, 3), -1, dtype=np.int32)
        for i, row in enumerate(sch.order):
            po[i] = row
        got = st.overlap_bound(code, order, first, po, nch)
        run = {int(c): i * nch // first for i, c in enumerate(order[:first])}
        res = {s_: r for s_, r, _d in sch.order}

        def tree(s_, seen):  # every source the block of s_ depends on
            if s_ in seen:
                return
            seen.add(s_)
            for t in ref.cells[res[s_]]:
                if t != s_:
                    tree(t, seen)

        want = np.zeros(nch, dtype=np.int64)
        for s_, _r, d in sch.order:
            if d > 1:
                seen = set()
                tree(s_, seen)
                want[max(run[res[t]] for t in seen)] += 1
        assert np.array_equal(got, want), (got, want)
        assert got[-1] >= 0.8 * got.sum()
        online = []
        for j in range(nch):
            n_j = (j + 1) * first // nch
            online.append(sum(o.wave_schedule(ref, sorted(int(c) for c in order[:n_j])).recovered))
        gain = np.diff([0] + online)
        assert gain[-1] >= 0.5 * ref.num_sources


def test_bounds_match_oracle(libbpx):
    """The library's bounds on n equal the oracle's, and Tables I / III meet
    them with equality."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    for k in range(2, 12):
        for b in (1, 2, 3, 8, 64):
            assert bpx.bound("k_equals_sigma", k, b) == o.bound_k_equals_sigma(k, b)
            for s in range(1, k):
                assert bpx.bound("paterson", k, b, s) == o.bound_paterson(k, b, s)
    assert bpx.bound("k_equals_sigma", 2, 2) == 5 == bpx.Code.table1().n
    assert bpx.bound("paterson", 3, 3, 2) == 5 == bpx.Code.table3().n


def test_code_from_columns_and_search(libbpx):
    """A code given by its cells builds the same graph as the literal table;
    the search finds array BP-XOR codes the oracle verifies by brute force
    for parameters the bounds allow (incl. ones meeting them), and none where
    the k = sigma bound rules them out."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    t1 = bpx.Code.table1()
    c = bpx.Code.from_columns(5, 2, 2, t1.columns(), e=3)
    assert c.cells == t1.cells and list(c.col_ptr) == list(t1.col_ptr) and c.sigma == 2
    for n, k, b, s in [(5, 2, 2, 2), (5, 3, 3, 2), (5, 3, 4, 2), (4, 2, 4, 2)]:
        code, used = bpx.Code.search(n, k, b, s, iters=2000000, seed=5)
        assert code is not None, (n, k, b, s, used)
        assert code.sigma <= s and code.e == n - k
        assert o.is_array_bpxor(o.code_from_columns("found", k, b, code.columns()))
    assert bpx.bound("k_equals_sigma", 2, 2) < 6
    code, used = bpx.Code.search(6, 2, 2, 2, iters=200000, seed=1)
    assert code is None and used == 200000
    with pytest.raises(bpx.BpxError):
        bpx.Code.from_columns(2, 1, 1, [[(0,)], [(1,)]], e=1)     # source 1 out of range


def test_search_finds_codes_of_degree_four_to_six(libbpx):
    """Equal-height array BP-XOR codes beyond Tables I / III at sigma >= 4:
    the multi-chain search finds [n, k, b] = [6, 4, 4] with sigma = 4 and
    [5, 3, 4] with sigma = 5 and 6 (n - k = 2 erased columns), each verified
    by the oracle's brute force over every erasure pattern."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    for n, k, b, s, th in [(6, 4, 4, 4, 4), (5, 3, 4, 5, 4), (5, 3, 4, 6, 2)]:
        code, used = bpx.Code.search(n, k, b, s, iters=1500000, seed=1, threads=th)
        assert code is not None, (n, k, b, s, used)
        assert code.sigma == s and code.e == n - k and all(h == b for h in code.heights)
        ref = o.code_from_columns("found", k, b, code.columns())
        assert ref.sigma == s and o.is_array_bpxor(ref)
        assert n <= o.bound_paterson(k, b, s) if s < k else n <= o.bound_k_equals_sigma(k, b)


def test_search_finds_a_three_erasure_code(libbpx):
    """An equal-height array BP-XOR code that tolerates three erased columns
    with more than two data columns: the search finds [n, k, b] = [6, 3, 4]
    at sigma = 4 (8 chains of 6 M moves; about half a minute on 8 host
    threads), and the oracle's brute force confirms that every set of three
    columns peels all 12 sources."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    code, used = bpx.Code.search(6, 3, 4, 4, iters=6000000, seed=7, threads=8)
    assert code is not None, used
    assert code.sigma == 4 and code.e == 3 and all(h == 4 for h in code.heights)
    ref = o.code_from_columns("found", 3, 4, code.columns())
    assert o.is_array_bpxor(ref) and ref.n - ref.k == 3


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13])
def test_xcode_graph_matches_oracle(libbpx, p):
    """The library's X-code (built column by column) has the oracle's cells
    (built from the data symbols' side), columns and parameters."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    c, ref = bpx.Code.xcode(p), o.xcode(p)
    assert (c.n, c.k, c.b, c.e, c.sigma, c.num_cells) == (ref.n, ref.k, ref.b, ref.e, ref.sigma, len(ref.cells))
    assert c.cells == ref.cells
    assert list(c.col_of_cell) == list(ref.col_of_cell) and list(c.heights) == [p] * p


def test_xcode_parameters_rejected(libbpx):
    bpx = libbpx
    for n, k, b in [(9, 7, 9), (7, 4, 7), (7, 5, 6), (2, 0, 2)]:
        with pytest.raises(bpx.BpxError):
            bpx.Code(bpx.XCODE, n, k, b)


def test_code_search_ex_threads_and_flags(libbpx):
    """The multi-chain search: a [7, 2] code with b = 3 (n meets the k = sigma
    bound 2 b + 1) is found and verified by brute force; the result does not
    depend on the threads' timing (same seed, same code twice); the
    systematic flag keeps the data columns' single-source cells; bad
    arguments are rejected."""
    bpx = libbpx
    from oracle import bpx_oracle as o
    assert bpx.bound("k_equals_sigma", 2, 3) == 7
    code, used = bpx.Code.search(7, 2, 3, 2, iters=2000000, seed=3, threads=1)
    assert code is not None, used
    assert code.sigma <= 2 and code.e == 5
    assert o.is_array_bpxor(o.code_from_columns("found", 2, 3, code.columns()))
    a, _ = bpx.Code.search(7, 2, 3, 2, iters=300000, seed=11, threads=4)
    b, _ = bpx.Code.search(7, 2, 3, 2, iters=300000, seed=11, threads=4)
    assert (a is None) == (b is None)
    if a is not None:
        assert a.cells == b.cells and list(a.col_ptr) == list(b.col_ptr)
    s, used = bpx.Code.search(5, 2, 2, 2, iters=20000, seed=0, systematic=True, threads=2)
    assert used <= 2 * 20000
    if s is not None:  # data columns: column l, cell z holds source z k + l alone
        cols = s.columns()
        assert cols[0] == [(0,), (2,)] and cols[1] == [(1,), (3,)]
    h = ctypes.c_void_p()
    used = ctypes.c_longlong()
    assert bpx.lib().bpx_code_search_ex(5, 2, 2, 2, 10, 0, 0, 0, ctypes.byref(h), ctypes.byref(used)) == bpx.ERR_INVAL
    assert bpx.lib().bpx_code_search_ex(5, 2, 2, 2, 10, 0, 4, 1, ctypes.byref(h), ctypes.byref(used)) == bpx.ERR_INVAL
