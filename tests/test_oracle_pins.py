"""Pins for the FP64 oracle: what the paper and the mathematics fix.

Each test checks the oracle against something other than itself -- a table
or number the paper prints (tests/golden/), a closed form, an independent
characterisation, or brute force on tiny inputs -- so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails here.
"""
import itertools
import os
import random

import numpy as np
import pytest

from oracle import bpx_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    cols = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            _node, cells = line.split(":", 1)
            col = []
            for cell in cells.split(";"):
                vs = [int(v.strip()[1:]) - 1 for v in cell.split("+")]
                col.append(tuple(sorted(vs)))
            cols.append(col)
    return cols


def _claims():
    out = {}
    with open(os.path.join(GOLDEN, "paper_claims.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = [int(x) for x in v.split(",")] if "," in v else int(v)
    return out


CLAIMS = _claims()


# ---------------------------------------------------------------- Table I / III

@pytest.mark.parametrize("fn,fixture", [(o.table1, "table1.txt"), (o.table3, "table3.txt")])
def test_literal_tables_match_transcription(fn, fixture):
    code = fn()
    cols = _read_table(fixture)
    assert code.n == len(cols)
    got = [[code.cells[c] for c in code.cells_of_column(j)] for j in range(code.n)]
    assert got == cols
    # column-major numbering
    assert code.col_of_cell == sorted(code.col_of_cell)


def test_table1_any_two_columns_decode():
    """Example 1: any two of the five nodes suffice; no single node does."""
    code = o.table1()
    m = CLAIMS["table1_min_columns"]
    for keep in itertools.combinations(range(5), m):
        erased = [j for j in range(5) if j not in keep]
        assert o.decodable(code, erased), keep
    for keep in itertools.combinations(range(5), m - 1):
        erased = [j for j in range(5) if j not in keep]
        assert not o.decodable(code, erased)


def test_table1_recovery_threshold_is_seven():
    """Example 1: every 7 of the 10 processor outputs decode; some 6 do not."""
    code = o.table1()
    thr = CLAIMS["table1_recovery_threshold"]
    for sub in itertools.combinations(range(code.num_cells), thr):
        assert o.wave_schedule(code, sub).ok
    assert any(not o.wave_schedule(code, sub).ok
               for sub in itertools.combinations(range(code.num_cells), thr - 1))


def test_table3_block_mds():
    """Example 2: [5,3,2,3] decodes from any 3 of its 5 columns."""
    code = o.table3()
    m = CLAIMS["table3_min_columns"]
    for keep in itertools.combinations(range(5), m):
        erased = [j for j in range(5) if j not in keep]
        assert o.decodable(code, erased), keep
    # and from no 2 columns (3 erasures exceed t = 2)
    for keep in itertools.combinations(range(5), m - 1):
        erased = [j for j in range(5) if j not in keep]
        assert not o.decodable(code, erased)


def test_literal_sigma():
    assert o.table1().sigma == CLAIMS["table1_sigma"]
    assert o.table3().sigma == CLAIMS["table3_sigma"]


# ---------------------------------------------------------------- Mojette

def test_fig2_heights():
    k, b = CLAIMS["fig2_k"], CLAIMS["fig2_b"]
    heights = []
    for p, q in [(-1, 1), (0, 1), (1, 1)]:
        bins = o.mojette_bins(k, b, p, q)
        # every label lies in [0, b_i) and the label range has b_i entries
        assert min(bins) == 0
        heights.append(max(bins) + 1)
        assert heights[-1] == o.mojette_height(k, b, p, q)
    assert heights == CLAIMS["fig2_heights"]


def _brute_lines(k, b, p, q):
    """Groups grid pixels by brute force: two pixels share a bin iff their
    difference is a multiple of the direction (p, -q) in (z, l).  Independent
    of the label formula of Eq. (moj1)."""
    pix = [(z, l) for z in range(b) for l in range(k)]
    parent = {x: x for x in pix}

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for (z, l) in pix:
        z2, l2 = z + p, l - q
        if 0 <= z2 < b and 0 <= l2 < k:
            parent[find((z2, l2))] = find((z, l))
    groups = {}
    for x in pix:
        groups.setdefault(find(x), []).append(x[0] * k + x[1])
    return sorted(tuple(sorted(g)) for g in groups.values())


@pytest.mark.parametrize("k,b", [(3, 4), (4, 3), (5, 7), (2, 6)])
@pytest.mark.parametrize("p,q", [(-1, 1), (0, 1), (1, 1), (2, 1), (-3, 1), (1, 2), (-1, 2), (3, 2), (5, 4), (1, 0)])
def test_bins_are_lines_of_direction(k, b, p, q):
    """Eq. (moj1) puts two pixels in one bin iff they lie on one discrete line
    of direction (p, q); a sign error in the label formula breaks this."""
    bins = o.mojette_bins(k, b, p, q)
    got = sorted(tuple(v) for v in bins.values())
    assert got == _brute_lines(k, b, p, q)
    h = o.mojette_height(k, b, p, q)
    assert all(0 <= lab < h for lab in bins)
    assert min(bins) == 0 and max(bins) == h - 1


@pytest.mark.parametrize("k,b", [(3, 4), (6, 5), (8, 8), (24, 40), (5, 17)])
@pytest.mark.parametrize("p,q", [(0, 1), (1, 1), (-1, 1), (2, 1), (-3, 1), (1, 2), (3, 4), (-5, 2)])
def test_sigma_formula_is_max_bin(k, b, p, q):
    """Theorem on sigma_i: the largest bin has min(ceil(b/|p|), ceil(k/|q|))
    pixels."""
    bins = o.mojette_bins(k, b, p, q)
    assert max(len(v) for v in bins.values()) == o.sigma_formula(k, b, p, q)


def test_lemma_a1_and_a002620():
    seq = CLAIMS["a002620_prefix"]
    for t in range(1, len(seq)):
        s = sum(abs(p) for p, _ in o.construction_a_slopes(t))
        assert s == seq[t] == o.lemma_a1_closed_form(t)
    for t in range(1, 60):
        assert sum(abs(p) for p, _ in o.construction_a_slopes(t)) == o.lemma_a1_closed_form(t)


def test_lemma_b1():
    for t in range(1, 60):
        ps = [p for p, _ in o.construction_b_slopes(t, 1)]
        assert all(p % 2 != 0 for p in ps) and len(set(ps)) == t
        assert ps == list(range(ps[0], ps[0] + 2 * t, 2))  # consecutive odds
        assert sum(abs(p) for p in ps) == o.lemma_b1_closed_form(t)


def test_construction_a_slope_set():
    # Construction A's set is n consecutive integers around zero, all coprime to q=1
    for n in range(1, 40):
        ps = [p for p, _ in o.construction_a_slopes(n)]
        assert ps == list(range(ps[0], ps[0] + n))
        assert -ps[0] == (n - 1) // 2 and ps[-1] == n // 2


@pytest.mark.parametrize("n,k,b", [(5, 3, 4), (6, 4, 5), (8, 6, 6), (7, 4, 10), (12, 9, 100),
                                   (32, 24, 683), (32, 24, 86), (9, 3, 7)])
def test_eps_construction_a_closed_form(n, k, b):
    """Appendix A: exact worst-case overhead of Construction A.  The oracle's
    eps comes from the column heights; for small n also brute-force every
    k-subset of columns."""
    code = o.construction_a(n, k, b)
    closed = o.eps_construction_a_closed_form(n, k, b)
    assert code.eps() == pytest.approx(closed, rel=1e-12, abs=1e-15)
    if n <= 12:
        worst = max(sum(code.heights[j] for j in sub)
                    for sub in itertools.combinations(range(n), k)) / (k * b) - 1
        assert worst == pytest.approx(closed, rel=1e-12, abs=1e-15)
    # Lemma A.1 bounds of Appendix A
    lo = (k - 1) / (4 * k * b) * (2 * k * n - k * k - 1)
    hi = (k - 1) / (4 * k * b) * (2 * k * n - k * k + 1)
    assert lo - 1e-12 <= closed <= hi + 1e-12


def test_heights_equal_label_ranges():
    for code in [o.construction_a(9, 5, 11), o.construction_b(7, 6, 9, 1), o.systematic_mojette(8, 3, 8)]:
        for j, pq in enumerate(code.proj):
            if pq is None:
                continue
            cells = [code.cells[c] for c in code.cells_of_column(j)]
            bins = o.mojette_bins(code.k, code.b, *pq)
            assert len(cells) == len(bins)
            assert max(bins) + 1 == code.heights[j]


# ---------------------------------------------------------------- Katz criterion

@pytest.mark.parametrize("k,b", [(3, 4), (4, 3), (4, 5), (5, 4), (3, 7)])
def test_katz_criterion_iff_peel(k, b):
    """Katz criterion: every projection subset satisfying it decodes by BP.
    The converse is tested, not assumed: a subset failing it leaves a ghost
    (the grid is not determined), so no decoder, BP included, can succeed."""
    directions = [(0, 1), (1, 1), (-1, 1), (2, 1), (-2, 1), (1, 2), (-1, 2), (3, 1), (1, 0)]
    for r in range(1, 5):
        for sub in itertools.combinations(directions, r):
            code = o._projection_code("katz", len(sub), k, b, list(sub))
            ok = o.wave_schedule(code, range(code.num_cells)).ok
            assert ok == o.katz_holds(k, b, sub), sub


def _ghost_free(k, b, sub):
    """Linear-algebra check (rank over the rationals) that the projections
    determine the grid -- independent of BP."""
    rows = []
    for p, q in sub:
        for v in o.mojette_bins(k, b, p, q).values():
            r = np.zeros(k * b)
            r[v] = 1
            rows.append(r)
    return np.linalg.matrix_rank(np.array(rows)) == k * b


@pytest.mark.parametrize("k,b", [(3, 4), (4, 4)])
def test_katz_matches_rank(k, b):
    directions = [(0, 1), (1, 1), (-1, 1), (2, 1), (1, 2), (1, 0)]
    for r in range(1, 4):
        for sub in itertools.combinations(directions, r):
            assert _ghost_free(k, b, sub) == o.katz_holds(k, b, sub), sub


# ---------------------------------------------------------------- decodability

@pytest.mark.parametrize("n,k,b", [(5, 3, 4), (6, 4, 5), (8, 6, 6), (7, 4, 10)])
def test_construction_a_any_k_projections(n, k, b):
    code = o.construction_a(n, k, b)
    for erased in itertools.combinations(range(n), n - k):
        assert o.decodable(code, erased)


@pytest.mark.parametrize("n,k,b,q_e", [(5, 6, 5, 1), (6, 8, 4, 2), (4, 7, 6, 1)])
def test_construction_b_ceil_k_over_q_projections(n, k, b, q_e):
    """Appendix B: ceil(k / 2^{q_e}) projections of Construction B decode."""
    code = o.construction_b(n, k, b, q_e)
    need = -(-k // 2 ** q_e)
    assert need <= n
    for keep in itertools.combinations(range(n), need):
        erased = [j for j in range(n) if j not in keep]
        assert o.decodable(code, erased), keep


@pytest.mark.parametrize("k,b,e", [(9, 6, 3), (8, 8, 3), (8, 4, 3), (12, 6, 4), (20, 4, 2), (6, 5, 5)])
def test_systematic_mojette_tolerates_e(k, b, e):
    code = o.systematic_mojette(k, e, b)
    for erased in itertools.combinations(range(k + e), e):
        assert o.decodable(code, erased)


# ---------------------------------------------------------------- peel contract

def _fixed_point_depth(code, cells):
    """Depth by value iteration: depth(s) = 1 + min over surviving cells c
    containing s of max_{t in c, t != s} depth(t) (max of nothing = 0);
    unrecoverable sources stay at infinity.  Independent of the round
    procedure."""
    INF = 10 ** 9
    S = code.num_sources
    d = [INF] * S
    changed = True
    while changed:
        changed = False
        for c in cells:
            cs = code.cells[c]
            for s in cs:
                m = max([d[t] for t in cs if t != s], default=0)
                if m < INF and m + 1 < d[s]:
                    d[s] = m + 1
                    changed = True
    return d


def _random_codes():
    rng = random.Random(7)
    yield o.table1()
    yield o.table3()
    yield o.systematic_mojette(8, 3, 8)
    yield o.construction_a(7, 4, 10)
    yield o.construction_b(6, 8, 4, 2)
    # random sparse codes
    for _ in range(6):
        S = rng.randint(3, 12)
        n = rng.randint(3, 7)
        cells, cols = [], []
        for j in range(n):
            for _ in range(rng.randint(1, 4)):
                deg = rng.randint(1, min(3, S))
                cells.append(tuple(sorted(rng.sample(range(S), deg))))
                cols.append(j)
        yield o.Code("rand", n, 1, 1, S, cells, cols, [1] * n, [None] * n, 1)


def test_wave_contract_fixed_point_and_resolver():
    rng = random.Random(3)
    for code in _random_codes():
        for _ in range(12):
            erased = [j for j in range(code.n) if rng.random() < 0.3]
            cells = o.surviving_cells(code, erased)
            sch = o.wave_schedule(code, cells)
            naive = o.wave_schedule_naive(code, cells)
            assert sch.depth == naive.depth and sch.resolver == naive.resolver
            assert sch.order == naive.order
            fp = _fixed_point_depth(code, cells)
            for s in range(code.num_sources):
                if sch.depth[s] == 0:
                    assert fp[s] >= 10 ** 9
                    continue
                assert sch.depth[s] == fp[s]
                # resolver: lowest surviving cell containing s whose other
                # members are all recovered in earlier rounds
                ok = [c for c in cells if s in code.cells[c]
                      and all(sch.depth[t] != 0 and sch.depth[t] < sch.depth[s]
                              for t in code.cells[c] if t != s)]
                assert sch.resolver[s] == min(ok)
            keys = [(d, s) for s, _r, d in sch.order]
            assert keys == sorted(keys)


def test_sequential_peel_same_stopping_set():
    """The final recovered set does not depend on the order in which
    degree-one nodes are taken (the peeling stopping set is unique)."""
    rng = random.Random(11)
    for code in _random_codes():
        for _ in range(10):
            erased = [j for j in range(code.n) if rng.random() < 0.4]
            cells = o.surviving_cells(code, erased)
            wave = {s for s in range(code.num_sources) if o.wave_schedule(code, cells).depth[s] > 0}
            for _ in range(3):
                seq = o.sequential_peel(code, cells, pick=lambda xs: rng.choice(xs))
                assert seq == wave


def test_undecodable_patterns_reported():
    code = o.table1()
    for erased in itertools.combinations(range(5), 4):
        sch = o.wave_schedule(code, o.surviving_cells(code, erased))
        assert not sch.ok
        assert 0 < sum(sch.recovered) < code.num_sources or sum(sch.recovered) == 0


# ---------------------------------------------------------------- numerics

def _int_inputs(rng, M, K, N, lim=3):
    A = rng.integers(-lim, lim + 1, size=(M, K)).astype(np.float32)
    B = rng.integers(-lim, lim + 1, size=(K, N)).astype(np.float32)
    return A, B


@pytest.mark.parametrize("maker,h", [(o.table1, 4), (o.table3, 3), (lambda: o.systematic_mojette(8, 3, 8), 2),
                                     (lambda: o.construction_a(7, 4, 10), 1)])
def test_integer_inputs_decode_exactly(maker, h):
    """Integer inputs keep every FP64 intermediate exact, so the decoded C
    must equal A B bit for bit, whatever the depth."""
    code = maker()
    rng = np.random.default_rng(5)
    M, K, N = code.num_sources * h, 24, 20
    A, B = _int_inputs(rng, M, K, N)
    ref = o.reference_product(A, B)
    for erased in list(o.all_erasure_patterns(code.n, code.e))[:40]:
        C, sch = o.coded_matmul(code, A, B, h, erased)
        assert sch.ok
        assert np.array_equal(C, ref)


def test_padded_rows_read_as_zero():
    code = o.table3()
    rng = np.random.default_rng(2)
    h = 4
    M = code.num_sources * h - 3   # last block ragged
    A, B = _int_inputs(rng, M, 16, 8)
    C, sch = o.coded_matmul(code, A, B, h, [1, 3])
    assert sch.ok
    assert np.array_equal(C[:M], o.reference_product(A, B))
    assert np.all(C[M:] == 0)


def test_random_inputs_error_within_amplification():
    """Random normal inputs: the decoded blocks match A B to within a small
    multiple of the FP64 unit roundoff times each source's amplification."""
    code = o.table3()
    rng = np.random.default_rng(9)
    h, K, N = 6, 40, 12
    A = rng.standard_normal((code.num_sources * h, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    ref = o.reference_product(A, B)
    for erased in o.all_erasure_patterns(code.n, 2):
        cells = o.surviving_cells(code, erased)
        sch = o.wave_schedule(code, cells)
        P = o.coded_products(code, A, B, h, cells)
        Cd = o.peel_decode(code, P, sch, h, N)
        kap = o.amplification(code, sch, P, Cd)
        for s, blk in Cd.items():
            r = ref[s * h:(s + 1) * h]
            err = np.linalg.norm(blk - r) / np.linalg.norm(r)
            assert err <= 1e-12 * max(1.0, kap[s])


def test_systematic_no_erasure_is_copy():
    """e = 0 on a systematic code: every source is resolved by its own
    degree-one data cell at depth 1, so decoding is a copy of P."""
    code = o.systematic_mojette(5, 2, 3)
    sch = o.wave_schedule(code, range(code.num_cells))
    assert sch.ok and sch.num_waves == 1
    for s, r, d in sch.order:
        assert code.cells[r] == (s,) and d == 1


def test_expansion_reproduces_products():
    """The integer expansion of C_s over the products, applied to the
    products, gives C_s back (exactly, on integer data)."""
    code = o.systematic_mojette(6, 3, 4)
    rng = np.random.default_rng(4)
    h = 2
    A, B = _int_inputs(rng, code.num_sources * h, 10, 6)
    erased = [0, 2, 4]
    cells = o.surviving_cells(code, erased)
    sch = o.wave_schedule(code, cells)
    P = o.coded_products(code, A, B, h, cells)
    Cd = o.peel_decode(code, P, sch, h, 6)
    for s, e in o.expansion(code, sch).items():
        tot = sum(v * P[c] for c, v in e.items())
        assert np.array_equal(tot, Cd[s])


@pytest.mark.parametrize("n,k,b,q_e", [(5, 6, 5, 1), (6, 8, 4, 2), (7, 6, 9, 1), (9, 10, 30, 1), (12, 20, 50, 2)])
def test_eps_construction_b_closed_form(n, k, b, q_e):
    """Construction B overhead: heights-based eps equals the Lemma B.1 closed
    form and brute force over every decoding set of columns."""
    code = o.construction_b(n, k, b, q_e)
    t = n - code.e
    assert t == -(-k // 2 ** q_e)
    closed = o.eps_construction_b_closed_form(n, k, b, q_e)
    brute = max(sum(code.heights[j] for j in sub)
                for sub in itertools.combinations(range(n), t)) / (k * b) - 1
    assert code.eps() == pytest.approx(closed, rel=1e-12)
    assert brute == pytest.approx(closed, rel=1e-12)


def test_planted_mistakes_are_caught(monkeypatch):
    """A sign error in the bin label of Eq. (moj1) or a dropped term in the
    peel subtraction must fail the pins above."""
    good_bins = o.mojette_bins

    def bad_bins(k, b, p, q):
        offset = (b - 1) * q * o._u(q) + (k - 1) * p * o._u(p)
        bins = {}
        for z in range(b):
            for l in range(k):
                bins.setdefault(offset - z * q + l * p, []).append(z * k + l)
        return {lab: sorted(v) for lab, v in bins.items()}

    monkeypatch.setattr(o, "mojette_bins", bad_bins)
    got = sorted(tuple(v) for v in o.mojette_bins(4, 3, 1, 1).values())
    assert got != _brute_lines(4, 3, 1, 1)
    monkeypatch.setattr(o, "mojette_bins", good_bins)

    def bad_peel(code, products, sched, h, N):
        C = {}
        for s, r, _d in sched.order:
            acc = products[r].copy()
            others = [t for t in code.cells[r] if t != s]
            for t in others[:-1]:          # drops the last term
                acc -= C[t]
            C[s] = acc
        return C

    code = o.table1()
    rng = np.random.default_rng(1)
    A, B = _int_inputs(rng, 8, 6, 5)
    cells = o.surviving_cells(code, [0, 1])
    sch = o.wave_schedule(code, cells)
    P = o.coded_products(code, A, B, 2, cells)
    Cd = bad_peel(code, P, sch, 2, 5)
    ref = o.reference_product(A, B)
    assert any(not np.array_equal(Cd[s], ref[2 * s:2 * s + 2]) for s in Cd)


def test_propagation_factors():
    """nu_s = 1 for sources copied from a degree-one cell; 1 <= nu_s <= kappa_s
    (Cauchy-Schwarz); and nu_s predicts the spread of injected product
    errors: perturbing every product by independent relative noise of size
    eps gives block errors of about eps nu_s."""
    code = o.systematic_mojette(8, 3, 8)
    rng = np.random.default_rng(12)
    h, K, N = 4, 64, 48
    A = rng.standard_normal((code.num_sources * h, K))
    B = rng.standard_normal((K, N))
    erased = [0, 3, 9]
    cells = o.surviving_cells(code, erased)
    sch = o.wave_schedule(code, cells)
    P = o.coded_products(code, A, B, h, cells)
    Cd = o.peel_decode(code, P, sch, h, N)
    nu = o.propagation(code, sch, P, Cd)
    kap = o.amplification(code, sch, P, Cd)
    for s, r, d in sch.order:
        if len(code.cells[r]) == 1:
            assert nu[s] == pytest.approx(1.0)
        assert 1.0 - 1e-12 <= nu[s] <= kap[s] + 1e-12
    eps = 1e-6
    ratios = []
    for trial in range(20):
        Pn = {c: p * (1 + eps * rng.standard_normal(p.shape)) for c, p in P.items()}
        Cn = o.peel_decode(code, Pn, sch, h, N)
        for s in Cd:
            err = np.linalg.norm(Cn[s] - Cd[s]) / np.linalg.norm(Cd[s])
            ratios.append(err / (eps * nu[s]))
    assert 0.7 < np.mean(ratios) < 1.3


# ---------------------------------------------------------------- exact-slice products

def _exact_bound(A, B, h, sigma):
    """Elementwise bound on |C_exact - A B| for the exact-slice path from the
    representation alone: rounding A and B to the fixed-point grid
    (half a unit each), the dropped digit pairs i + l >= S (each digit at
    most 2^(w-1)), and the final rounding to FP32."""
    w, S, bits = o.exact_slice_params(sigma)
    eA = o.exact_row_exponents(A, h).astype(float)
    eB = o.exact_col_exponents(B).astype(float)
    K = A.shape[1]
    M = A.shape[0]
    ea = eA[np.arange(M) % h][:, None]
    eb = eB[None, :]
    quant = K * (2.0 ** (ea - bits - 1) * 2.0 ** eb + 2.0 ** ea * (1 + 2.0 ** -bits) * 2.0 ** (eb - bits - 1))
    trunc_q = K * sum((2 * S - 1 - d) * 2.0 ** (w * (2 * S - 2 - d)) * 2.0 ** (2 * (w - 1))
                      for d in range(S, 2 * S - 1))
    trunc = trunc_q * 2.0 ** (ea + eb - 2 * bits)
    ref = A.astype(np.float64) @ B.astype(np.float64)
    return quant + trunc + 2.0 ** -24 * (np.abs(ref) + quant + trunc), ref


def test_exact_digits_recompose_and_stay_small():
    """x = sum_i 2^(w (S-1-i)) D_i exactly, |D_i| <= 2^(w-1), for every
    digit width the codes use, on random and extreme fixed-point values."""
    rng = np.random.default_rng(5)
    for sigma in (1, 2, 3, 5, 8, 12, 24, 40, 64):
        w, S, bits = o.exact_slice_params(sigma)
        assert sigma * 2 ** (w - 1) <= 256 and S * w >= bits + 1 and bits >= 23
        x = rng.integers(-(2 ** bits), 2 ** bits + 1, size=4000, dtype=np.int64)
        x[:4] = [2 ** bits, -(2 ** bits), 0, 2 ** bits - 1]
        D = o.balanced_digits(x, w, S)
        back = sum(D[i] << (w * (S - 1 - i)) for i in range(S))
        assert np.array_equal(back, x)
        for d in D:
            assert np.abs(d).max() <= 2 ** (w - 1)


def test_fixed_point_exponents_frexp_convention():
    A = np.array([[0.75, -3.0], [0.0, 0.0], [1.0, 0.5]], dtype=np.float32)
    assert list(o.exact_row_exponents(A, 3)) == [2, 0, 1]   # 3 < 2^2, 0 -> 0, 1 < 2^1
    assert list(o.exact_col_exponents(A)) == [1, 2]


@pytest.mark.parametrize("maker,h", [(o.table1, 4), (o.table3, 3),
                                     (lambda: o.systematic_mojette(4, 2, 3), 2),
                                     (lambda: o.construction_a(6, 4, 4), 1)])
def test_exact_slice_small_integers_give_the_exact_product(maker, h):
    """Small-integer inputs sit on the fixed-point grid with one nonzero
    digit, so the exact-slice path must return A B exactly (integer matmul),
    for every decodable erasure pattern."""
    code = maker()
    rng = np.random.default_rng(7)
    M, K, N = code.num_sources * h - 1, 24, 8
    A, B = _int_inputs(rng, M, K, N)
    exact = A.astype(np.int64) @ B.astype(np.int64)
    for er in o.all_erasure_patterns(code.n, code.n - code.k):
        if not o.decodable(code, er):
            continue
        C, _Q, sched = o.exact_slice_coded_matmul(code, A, B, h, er)
        assert sched.ok
        assert np.array_equal(C[:M], exact.astype(np.float32))


@pytest.mark.parametrize("maker,h,dist", [(o.table1, 16, "normal"), (o.table3, 8, "loguniform"),
                                          (lambda: o.systematic_mojette(4, 3, 4), 4, "uniform"),
                                          (lambda: o.construction_a(7, 4, 5), 2, "normal")])
def test_exact_slice_is_mask_and_depth_independent(maker, h, dist):
    """Every decodable pattern yields bit-identical C and identical exact
    integers Q_s, equal to the exact-slice product of the source computed
    directly without the code: the coded digit planes are linear in the
    sources and the peel is exact, so nothing depends on the resolver or the
    peel depth.  Also within the representation's error bound of A B."""
    code = maker()
    rng = np.random.default_rng(11)
    M, K, N = code.num_sources * h, 40, 12
    if dist == "normal":
        A = rng.standard_normal((M, K)).astype(np.float32)
        B = rng.standard_normal((K, N)).astype(np.float32)
    elif dist == "uniform":
        A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
        B = rng.uniform(-1, 1, (K, N)).astype(np.float32)
    else:
        A = (rng.choice([-1.0, 1.0], (M, K)) * 10.0 ** rng.uniform(-3, 3, (M, K))).astype(np.float32)
        B = (rng.choice([-1.0, 1.0], (K, N)) * 10.0 ** rng.uniform(-3, 3, (K, N))).astype(np.float32)
    direct = {}
    for s in range(code.num_sources):
        blk, q = o.exact_slice_block(A, B, s, h, code.sigma)
        direct[s] = (blk, q)
    bound, ref = _exact_bound(A, B, h, code.sigma)
    depths = set()
    patterns = list(o.all_erasure_patterns(code.n, code.n - code.k))
    for er in patterns[:: max(1, len(patterns) // 25)]:
        if not o.decodable(code, er):
            continue
        C, Q, sched = o.exact_slice_coded_matmul(code, A, B, h, er)
        depths.update(d for _s, _r, d in sched.order)
        for s in range(code.num_sources):
            assert np.array_equal(Q[s], direct[s][1])
            assert np.array_equal(C[s * h:(s + 1) * h], direct[s][0])
        assert np.all(np.abs(C.astype(np.float64) - ref) <= bound)
    assert max(depths) >= 2


def test_exact_slice_error_tracks_fp32_scale():
    """On N(0,1) data the exact-slice result is as close to A B as an FP32
    product (relative to max |A B|, below 1e-6) -- and no deeper source is
    worse than a direct one."""
    code = o.systematic_mojette(8, 3, 8)
    h = 4
    rng = np.random.default_rng(3)
    A = rng.standard_normal((code.num_sources * h, 256)).astype(np.float32)
    B = rng.standard_normal((256, 16)).astype(np.float32)
    C, _Q, sched = o.exact_slice_coded_matmul(code, A, B, h, (0, 3, 9))
    ref = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(C - ref).max() / np.abs(ref).max() < 1e-6
    assert max(d for _s, _r, d in sched.order) >= 3


def test_exact_slice_planted_mistakes_are_caught(monkeypatch):
    """Dropping the last kept diagonal, or forming coded digit planes with
    carries (digits of the coded sum instead of the sum of digits), must
    fail the bound or the mask-independence pin."""
    code = o.table1()
    h = 8
    rng = np.random.default_rng(2)
    A = rng.standard_normal((code.num_sources * h, 64)).astype(np.float32)
    B = rng.standard_normal((64, 8)).astype(np.float32)
    bound, ref = _exact_bound(A, B, h, code.sigma)
    good_q = o.exact_q

    def drop_last(Ad, Bd, w, S):
        q = np.zeros((Ad[0].shape[0], Bd[0].shape[1]), dtype=np.int64)
        for d in range(S - 1):
            q += sum(o.int_matmul(Ad[i], Bd[d - i]) for i in range(d + 1)) << (w * (S - 1 - d))
        return q

    monkeypatch.setattr(o, "exact_q", drop_last)
    C, _Q, _ = o.exact_slice_coded_matmul(code, A, B, h, (0, 1))
    assert not np.all(np.abs(C.astype(np.float64) - ref) <= bound)
    monkeypatch.setattr(o, "exact_q", good_q)

    w, S, bits = o.exact_slice_params(code.sigma)
    eA = o.exact_row_exponents(A, h)
    eB = o.exact_col_exponents(B)
    Bd = o.balanced_digits(o.fixed_point(B, eB[None, :], bits), w, S)
    sched = o.wave_schedule(code, o.surviving_cells(code, (0, 1)))
    Qc = {}
    for c in set(r for _s, r, _d in sched.order):
        tot = sum(o.fixed_point(o.row_block(A, s, h), eA[:, None], bits) for s in code.cells[c])
        Qc[c] = o.exact_q(o.balanced_digits(tot, w, S), Bd, w, S)   # carries: wrong
    CQ = {}
    for s, r, _d in sched.order:
        CQ[s] = Qc[r] - sum((CQ[t] for t in code.cells[r] if t != s), np.zeros_like(Qc[r]))
    direct = {s: o.exact_slice_block(A, B, s, h, code.sigma)[1] for s in range(code.num_sources)}
    assert any(not np.array_equal(CQ[s], direct[s]) for s in CQ)


def test_int_matmul_is_exact():
    """The FP64-matmul integer product equals Python's big-integer dot
    products, also near the 2^53 limit of its guard."""
    rng = np.random.default_rng(9)
    X = rng.integers(-256, 257, size=(5, 300), dtype=np.int64)
    Y = rng.integers(-(2 ** 20), 2 ** 20, size=(300, 4), dtype=np.int64)
    got = o.int_matmul(X, Y)
    for i in range(5):
        for j in range(4):
            assert got[i, j] == sum(int(a) * int(b) for a, b in zip(X[i], Y[:, j]))
    with pytest.raises(ValueError):
        o.int_matmul(np.full((1, 4), 2 ** 26, dtype=np.int64), np.full((4, 1), 2 ** 26, dtype=np.int64))


# ---------------------------------------------------------------- two-dimensional scheme

def test_gray_cells_match_paper():
    """Example 1 / Example 2: 2 of Table I's 10 cells and 6 of Table III's
    15 combine products sharing neither a block of A nor a block of B."""
    assert len(o.gray_cells_2d(o.table1())) == CLAIMS["table1_gray_cells"]
    assert o.table1().num_cells == CLAIMS["table1_cells"]
    assert len(o.gray_cells_2d(o.table3())) == CLAIMS["table3_gray_cells"]
    assert o.table3().num_cells == CLAIMS["table3_cells"]
    # for sigma = 2 "gray" is exactly: the two sources differ in both blocks
    for code in (o.table1(), o.table3()):
        for c in range(code.num_cells):
            zl = [o.source_zl(code, s) for s in code.cells[c]]
            neither = len(zl) == 2 and zl[0][0] != zl[1][0] and zl[0][1] != zl[1][1]
            assert (c in o.gray_cells_2d(code)) == neither


def test_terms_2d_partition_the_cell():
    """The factored products cover every source of the cell exactly once:
    the union of Z x L over the terms is the cell's set of (z, l), disjoint;
    a full rectangle of blocks is one product."""
    codes = [o.table1(), o.table3(), o.systematic_mojette(8, 3, 8), o.construction_a(7, 4, 5),
             o.construction_b(6, 8, 4, 2)]
    for code in codes:
        for c in range(code.num_cells):
            want = sorted(o.source_zl(code, s) for s in code.cells[c])
            got = sorted((z, l) for Z, L in o.terms_2d(code, c) for z in Z for l in L)
            assert got == want
            T = len(o.terms_2d(code, c))
            assert 1 <= T <= len(code.cells[c])
    full = o.Code(name="rect", n=1, k=3, b=3, num_sources=9, cells=[(0, 1, 3, 4)], col_of_cell=[0], heights=[1])
    assert o.terms_2d(full, 0) == [((0, 1), (0, 1))]


@pytest.mark.parametrize("maker,h,w", [(o.table1, 3, 4), (o.table3, 2, 4), (lambda: o.systematic_mojette(4, 2, 3), 2, 4),
                                       (lambda: o.construction_a(6, 4, 4), 1, 8)])
def test_2d_integer_inputs_decode_exactly(maker, h, w):
    """Integer inputs: every block of the two-dimensional decode equals the
    block of A B exactly, for every decodable erasure pattern; the factored
    products equal the definition."""
    code = maker()
    rng = np.random.default_rng(17)
    M, K, N = code.b * h - 1, 10, code.k * w
    A, B = _int_inputs(rng, M, K, N)
    ref = o.reference_product(A, B)
    for er in o.all_erasure_patterns(code.n, code.n - code.k):
        if not o.decodable(code, er):
            continue
        C, sched = o.coded_matmul_2d(code, A, B, h, w, er)
        assert sched.ok
        assert np.array_equal(C[:M], ref)
    P = o.coded_products_2d(code, A, B, h, w, range(code.num_cells))
    for c in range(code.num_cells):
        fac = sum((sum(o.row_block(A, z, h) for z in Z) @ sum(o.col_block(B, l, w) for l in L))
                  for Z, L in o.terms_2d(code, c))
        assert np.array_equal(fac, P[c])


def test_2d_example1_source_numbering():
    """Example 1: v1 = a1 b1, v2 = a1 b2, v3 = a2 b1, v4 = a2 b2, so the
    Table I cell v2 + v3 is A_0 B_1 + A_1 B_0."""
    code = o.table1()
    assert [o.source_zl(code, s) for s in range(4)] == [(0, 0), (0, 1), (1, 0), (1, 1)]
    c = code.cells.index((1, 2))
    assert o.terms_2d(code, c) == [((0,), (1,)), ((1,), (0,))]


# ---------------------------------------------------------------- straggler-time model

@pytest.mark.parametrize("maker", [o.table1, o.table3, lambda: o.systematic_mojette(3, 2, 2)])
def test_parallel_task_time_is_first_decodable_prefix(maker):
    """min over decodable sets of the latest arrival (Eq. (eqnTtotal), brute
    force over every subset) equals the arrival time of the first prefix of
    the arrival order that peels completely."""
    code = maker()
    rng = np.random.default_rng(8)
    for _ in range(15):
        T = o.task_times(code, 1.0, rng)
        order = list(np.argsort(T, kind="stable"))
        i = o.first_decodable(code, order)
        assert i > 0
        assert T[order[i - 1]] == o.parallel_task_time_brute(code, T)


def test_table1_first_decodable_at_most_seven():
    """Example 1: any 7 processor outputs suffice, so no arrival order needs
    more than 7 cells; some order needs exactly 7."""
    code = o.table1()
    rng = np.random.default_rng(1)
    worst = 0
    for _ in range(400):
        order = list(rng.permutation(code.num_cells))
        worst = max(worst, o.first_decodable(code, order))
    assert worst <= CLAIMS["table1_recovery_threshold"]
    # an order that starts with a non-decodable 6-set
    for S in itertools.combinations(range(10), 6):
        if not o.decodes(code, S):
            rest = [c for c in range(10) if c not in S]
            assert o.first_decodable(code, list(S) + rest) == 7
            break
    else:
        raise AssertionError("every 6-set decodes")


def test_task_time_scaling():
    """T_c = sigma_c X_c: mean of T_c / sigma_c is 1 / mu; the expected
    maximum of b rate-mu exponentials is H_b / mu (Section IV-A order
    statistics), checked by Monte Carlo on unscaled times."""
    code = o.table1()
    rng = np.random.default_rng(2)
    deg = np.array([len(c) for c in code.cells])
    Ts = np.stack([o.task_times(code, 2.0, rng) for _ in range(20000)])
    assert abs((Ts / deg).mean() - 0.5) < 0.01
    U = np.stack([o.task_times(code, 2.0, rng, scale_by_degree=False) for _ in range(20000)])
    H = sum(1.0 / j for j in range(1, 11))
    assert abs(U.max(axis=1).mean() - H / 2.0) < 0.03


# ---------------------------------------------------------------- bounds on n (Section III-B)

def test_paper_codes_meet_the_bounds():
    """Table I (k = sigma = 2, b = 2) meets n <= kb + 1 + max{k-3, 0} with
    equality; Table III (k = 3, b = 3, sigma = 2) meets the straggler count
    the simulations use with equality."""
    t1, t3 = o.table1(), o.table3()
    assert t1.k == t1.sigma and t1.n == CLAIMS["table1_n"] == o.bound_k_equals_sigma(t1.k, t1.b)
    assert t3.n - t3.k == CLAIMS["table3_n_minus_k"] == o.bound_paterson(t3.k, t3.b, t3.sigma) - t3.k


def test_array_bpxor_check_on_known_codes():
    assert o.is_array_bpxor(o.table1()) and o.is_array_bpxor(o.table3())
    bad = o.code_from_columns("rep", 2, 2, [[(0,), (1,)], [(2,), (3,)], [(0, 1), (2, 3)], [(0, 2), (1, 3)],
                                             [(0,), (3,)]])
    assert not o.is_array_bpxor(bad)


@pytest.mark.parametrize("p", [3, 5, 7, 11])
def test_xcode_is_an_mds_array_bpxor_code(p):
    """The X-code on p columns peels from every set of p - 2 columns (brute
    force over all pairs of erased columns: the MDS-by-peeling property Xu and
    Bruck prove, which is the Section III-A definition with t = 2), has equal
    column heights b = p, maximum degree sigma = p - 2 = k, and sits inside
    the k = sigma bound on n.  Parities taken along one diagonal twice, or at
    offset 0 or 3, break the property, so a wrong index or sign fails here."""
    c = o.xcode(p)
    assert (c.n, c.k, c.b, c.num_sources, c.e) == (p, p - 2, p, p * (p - 2), 2)
    assert all(h == p for h in c.heights) and c.sigma == p - 2
    assert o.is_array_bpxor(c)
    assert c.n <= o.bound_k_equals_sigma(c.k, c.b)
    # every source sits in its own column's degree-one cell and in exactly
    # two parity cells of two other columns (p = 3: the parities have degree
    # one as well)
    for s in range(c.num_sources if p >= 5 else 0):
        holders = [j for j, cell in enumerate(c.cells) if s in cell]
        cols = [c.col_of_cell[j] for j in holders]
        ones = [c.col_of_cell[j] for j in holders if len(c.cells[j]) == 1]
        assert len(holders) == 3 and len(set(cols)) == 3 and ones == [s // (p - 2)]
    if p >= 5:
        k = p - 2

        def mutated(off, sign):
            cols = []
            for i in range(p):
                col = [(i * k + r,) for r in range(k)]
                col.append(tuple(sorted(((i + r + 2) % p) * k + r for r in range(k))))
                col.append(tuple(sorted(((i + sign * (r + off)) % p) * k + r for r in range(k))))
                cols.append(col)
            return o.code_from_columns("mutated", k, p, cols)

        assert not o.is_array_bpxor(mutated(2, +1))
        assert not o.is_array_bpxor(mutated(0, -1))
        assert not o.is_array_bpxor(mutated(3, -1))
