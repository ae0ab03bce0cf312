"""FP64 CPU oracle for array BP-XOR coded matrix multiplication.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``.  The product path (the ``paper_1904_11563_gb300``
package and its CUDA library) never imports, links or executes anything here,
and this module imports nothing from the product.

What it computes (Arslan, "Array BP-XOR Codes for Hierarchically Distributed
Matrix Multiplication"):

* code graphs -- the literal array codes of Table I and Table III
  (Section III-A), the projection-geometry (Mojette) codes of Section III-C
  built bin by bin from Eq. (moj1) with Construction A (option1) and
  Construction B (option2), and a systematic Mojette array (k data columns
  plus projection parities);
* the belief-propagation (peeling) decoder of Section I-A, both as the
  sequential one-node-at-a-time procedure the paper describes and as the
  parallel "wave" reading used as the schedule contract (resolver = lowest
  cell id among the cells that have exactly one unknown source at the start
  of a round; sources of a round evaluated in ascending id);
* the numeric path over real matrices: encode A_c = sum of the row blocks in
  the support of cell c (XOR read as +), products P_c = A_c B, and the peel
  C_s = P_r - sum_{t in supp(r), t != s} C_t (XOR read as -), all in FP64;
* the uncoded reference C = A B and, per source, the integer expansion of
  C_s over the surviving products with its amplification factor;
* exact-slice coded products: A and B as fixed-point integers cut into
  balanced base-2^w digit planes, coded digit planes summed without carries
  (the worker-side encode applied plane by plane), digit-pair products
  grouped by diagonal, and the peel run on exact integers, so that the
  decoded C_s is the same number at every peel depth and under every
  decodable erasure pattern -- the exactness the paper's XOR over bits has
  (Section II) restored over the reals.  The digit representation is not in
  the paper; it is an Ozaki-style error-free splitting;
* the straggler-time model of Section IV: processor (cell) task times
  T_c = sigma_c X_c with X_c exponential of rate mu, and the parallel task
  time min over decodable sets S of max_{c in S} T_c of Eq. (eqnTtotal),
  both by brute force over subsets and as the first prefix of the arrival
  order that peels completely;
* the bounds on the number of columns n of Section III-B (the k = sigma
  bound and the general bound quoted from Paterson et al.), and a check that a code given by its cells is an
  array BP-XOR code (every k columns peel);
* the two-dimensional scheme of Section III-A (Examples 1 and 2): source
  (z, l) is the output block A_z B_l (row block z of A, column block l of
  B), a cell is the sum of its sources' block products, and the same peel
  rebuilds every block of C.  A cell factors into T products of summed
  operands (sum of A blocks) x (sum of B blocks); the cells with T > 1
  (for sigma = 2: the two products share neither a block of A nor one of B)
  are the ones whose encoding the paper says must happen on the worker.

Every function cites the passage it follows.  Nothing here is blocked, fused
or reordered beyond what the definition states; a library primitive (numpy's
FP64 matmul) serves as the product step.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Code graphs
# --------------------------------------------------------------------------


@dataclass
class Code:
    """A binary linear array code as a bipartite graph (Section I-A, III-A).

    ``cells[c]`` is the sorted tuple of source ids XORed (here: summed) into
    coded symbol ``c``; ``col_of_cell[c]`` is the code column (worker node)
    holding it.  Cells are numbered column-major: column ascending, then
    processor row / bin label ascending, empty bins dropped.
    """

    name: str
    n: int
    k: int
    b: int
    num_sources: int
    cells: list
    col_of_cell: list
    # Per column: nominal height (Mojette b_i of Section III-C; array codes: b)
    heights: list
    # Per column: projection (p, q), or None for a data / literal column
    proj: list = field(default_factory=list)
    e: int = 0

    @property
    def num_cells(self) -> int:
        return len(self.cells)

    def cells_of_column(self, j):
        return [c for c in range(self.num_cells) if self.col_of_cell[c] == j]

    @property
    def sigma(self) -> int:
        """Maximum coded-symbol degree (Section III-A)."""
        return max(len(c) for c in self.cells)

    def eps(self) -> float:
        """Worst-case coding overhead of Section III-B: over every set of
        columns large enough to decode (n - e of them: k for Construction A
        and the array codes, ceil(k / 2^{q_e}) for Construction B, as in
        Appendix B), (sum of their heights) / (k b) - 1.  The sum depends
        only on the chosen heights, so the worst case is the tallest ones."""
        hs = sorted(self.heights, reverse=True)[: self.n - self.e]
        return sum(hs) / (self.k * self.b) - 1.0


def _literal_code(name, n, k, b, columns):
    """Builds a code from columns of cells written with the paper's 1-based
    v indices; source s = v - 1."""
    cells, col_of_cell = [], []
    for j, col in enumerate(columns):
        for cell in col:
            cells.append(tuple(sorted(v - 1 for v in cell)))
            col_of_cell.append(j)
    return Code(name=name, n=n, k=k, b=b, num_sources=b * k, cells=cells,
                col_of_cell=col_of_cell, heights=[b] * n, proj=[None] * n,
                e=n - k)


def table1() -> Code:
    """Table I (Example 1, Section III-A): the [5,2,2,2] code, sigma = 2,
    four sources v1..v4 on n = 5 nodes with two processors each."""
    columns = [
        [(1,), (2, 3)],
        [(2,), (1, 4)],
        [(3,), (2, 4)],
        [(4,), (1, 3)],
        [(1, 2), (3, 4)],
    ]
    code = _literal_code("table1", 5, 2, 2, columns)
    # The label's third entry cannot be the erasure count: the code decodes
    # from any two of its five columns (Example 1), so t = n - k = 3.
    code.e = 3
    return code


def table3() -> Code:
    """Table III (Example 2, Section III-A): the [5,3,2,3] code, sigma = 2,
    nine sources v1..v9 on n = 5 nodes with three processors each."""
    columns = [
        [(1,), (3, 4), (6, 7)],
        [(1, 2), (4, 5), (7, 8)],
        [(2, 3), (5, 6), (8, 9)],
        [(7,), (9, 1), (4, 8)],
        [(3,), (2, 6), (9, 5)],
    ]
    return _literal_code("table3", 5, 3, 3, columns)


def _u(t: int) -> int:
    """Discrete unit function of Eq. (moj1): 1 for t > 0, else 0."""
    return 1 if t > 0 else 0


def mojette_height(k: int, b: int, p: int, q: int) -> int:
    """Projection length b_i = |p|(k-1) + |q|(b-1) + 1 (Section III-C)."""
    return abs(p) * (k - 1) + abs(q) * (b - 1) + 1


def mojette_bins(k: int, b: int, p: int, q: int):
    """Bins of projection (p, q) of the k x b grid, from Eq. (moj1).

    Pixel (z, l), z in [0, b), l in [0, k), is source s = z k + l.  The pixel
    lands in the bin with label
        (b-1) q u(q) + (k-1) p u(p) - z q - l p ,
    i.e. the bin index m + (b-1) q u(q) + (k-1) p u(p) of Eq. (moj1) with the
    Kronecker delta selecting m = -(z q + l p).  Returns a dict label -> sorted
    list of sources (empty labels absent).
    """
    offset = (b - 1) * q * _u(q) + (k - 1) * p * _u(p)
    bins: dict[int, list[int]] = {}
    for z in range(b):
        for l in range(k):
            label = offset - z * q - l * p
            bins.setdefault(label, []).append(z * k + l)
    return {lab: sorted(v) for lab, v in bins.items()}


def _projection_code(name, n, k, b, projections, data_columns=0, e=None):
    """Columns: ``data_columns`` systematic columns (column l holds sources
    z k + l, z ascending), then one column per projection with its bins in
    ascending label order (Section III-C: each projection is a code column,
    each bin a coded symbol)."""
    cells, col_of_cell, heights, proj = [], [], [], []
    j = 0
    for l in range(data_columns):
        for z in range(b):
            cells.append((z * k + l,))
            col_of_cell.append(j)
        heights.append(b)
        proj.append(None)
        j += 1
    for (p, q) in projections:
        bins = mojette_bins(k, b, p, q)
        for lab in sorted(bins):
            cells.append(tuple(bins[lab]))
            col_of_cell.append(j)
        heights.append(mojette_height(k, b, p, q))
        proj.append((p, q))
        j += 1
    assert j == n
    return Code(name=name, n=n, k=k, b=b, num_sources=k * b, cells=cells,
                col_of_cell=col_of_cell, heights=heights, proj=proj,
                e=(n - k) if e is None else e)


def construction_a_slopes(n: int):
    """Construction A (Cons33, option1): q_i = 1 and p_i running over the n
    consecutive integers -floor((n-1)/2) .. ceil((n-1)/2), ascending."""
    lo = -((n - 1) // 2)
    hi = -((-(n - 1)) // 2)  # ceil((n-1)/2)
    ps = list(range(lo, hi + 1))
    assert len(ps) == n
    return [(p, 1) for p in ps]


def construction_a(n: int, k: int, b: int) -> Code:
    """Mojette code of Construction A on a k x b grid: any k projections
    satisfy the Katz criterion through sum |q_i| = k, so t = n - k."""
    return _projection_code(f"mojA_n{n}_k{k}_b{b}", n, k, b,
                            construction_a_slopes(n), e=n - k)


def _ceil_odd(x: int) -> int:
    """Smallest odd integer >= x (the ceil_odd rounding of option2)."""
    return x if x % 2 != 0 else x + 1


def construction_b_slopes(n: int, q_e: int):
    """Construction B (cons35, option2): q_i = 2^{q_e} and p_i the n
    consecutive odd integers ceil_odd(-n+1), ..., ceil_odd(n-1)."""
    lo, hi = _ceil_odd(-n + 1), _ceil_odd(n - 1)
    ps = list(range(lo, hi + 1, 2))
    assert len(ps) == n, (n, ps)
    return [(p, 2 ** q_e) for p in ps]


def construction_b(n: int, k: int, b: int, q_e: int) -> Code:
    """Mojette code of Construction B: ceil(k / 2^{q_e}) projections satisfy
    the Katz criterion through sum |q_i| >= k (Appendix B)."""
    need = -(-k // (2 ** q_e))
    return _projection_code(f"mojB_n{n}_k{k}_b{b}_q{q_e}", n, k, b,
                            construction_b_slopes(n, q_e), e=n - need)


def systematic_slopes(e: int):
    """Parity slopes 0, +1, -1, +2, -2, ... with q = 1."""
    ps = [0]
    m = 1
    while len(ps) < e:
        ps.append(m)
        if len(ps) < e:
            ps.append(-m)
        m += 1
    return [(p, 1) for p in ps[:e]]


def systematic_mojette(k: int, e: int, b: int) -> Code:
    """Systematic Mojette array: the k x b data grid kept as k degree-one
    columns, plus e projection parities (q = 1, slopes 0, +1, -1, ...)."""
    return _projection_code(f"sysmoj_k{k}_e{e}_b{b}", k + e, k, b,
                            systematic_slopes(e), data_columns=k, e=e)


def xcode(p: int) -> Code:
    """X-code of Xu and Bruck (1999) on p columns, p prime: an equal-height
    MDS array code whose two-column erasure decoding is a peeling chain, so
    an array BP-XOR code in the sense of the Section III-A definition with
    n = p, k = p - 2, b = p, t = 2 and sigma = p - 2.  Column j stores its
    p - 2 data symbols (row r is source j (p - 2) + r) and two parity
    symbols; the data symbol of row r in column j enters the first parity
    of column j - r - 2 and the second parity of column j + r + 2 (mod p).
    Written here from the data symbols' side: each symbol is dropped into
    the two parities that contain it."""
    if p < 3 or any(p % d == 0 for d in range(2, int(p ** 0.5) + 1)):
        raise ValueError("X-code needs a prime p >= 3")
    k = p - 2
    first = [[] for _ in range(p)]
    second = [[] for _ in range(p)]
    for j in range(p):
        for r in range(k):
            s = j * k + r
            first[(j - r - 2) % p].append(s)
            second[(j + r + 2) % p].append(s)
    cells, col_of_cell = [], []
    for i in range(p):
        for r in range(k):
            cells.append((i * k + r,))
            col_of_cell.append(i)
        cells.append(tuple(sorted(first[i])))
        cells.append(tuple(sorted(second[i])))
        col_of_cell += [i, i]
    return Code(name=f"xcode_p{p}", n=p, k=k, b=p, num_sources=p * k, cells=cells, col_of_cell=col_of_cell,
                heights=[p] * p, proj=[None] * p, e=2)


def lemma_a1_closed_form(t: int) -> int:
    """Lemma A.1: sum of |p_i| over the t slopes of Construction A equals
    (t^2 - 1)/4 for odd t and t^2/4 for even t."""
    return (t * t - 1) // 4 if t % 2 else (t * t) // 4


def lemma_b1_closed_form(t: int) -> int:
    """Lemma B.1: sum of |p_i| over the t slopes of Construction B equals
    (t^2 + 1)/2 for odd t and t^2/2 for even t."""
    return (t * t + 1) // 2 if t % 2 else (t * t) // 2


def sigma_formula(k: int, b: int, p: int, q: int) -> int:
    """Theorem on the maximum projection degree (Section III-C):
    sigma_i = min(ceil(b/|p|), ceil(k/|q|)), an infinite term dropped."""
    terms = []
    if p != 0:
        terms.append(-(-b // abs(p)))
    if q != 0:
        terms.append(-(-k // abs(q)))
    return min(terms)


def katz_holds(k: int, b: int, projections) -> bool:
    """Katz criterion (Section III-C): sum |p_i| >= b or sum |q_i| >= k."""
    return (sum(abs(p) for p, _ in projections) >= b
            or sum(abs(q) for _, q in projections) >= k)


# --------------------------------------------------------------------------
# Belief-propagation (peeling) decoders
# --------------------------------------------------------------------------


def surviving_cells(code: Code, erased_cols) -> list:
    """Cells of the columns that did not straggle."""
    erased = set(int(j) for j in erased_cols)
    return [c for c in range(code.num_cells) if code.col_of_cell[c] not in erased]


def sequential_peel(code: Code, cell_subset, pick=None) -> set:
    """The BP decoder exactly as Section I-A describes it: start with every
    information node NULL; repeatedly take a coded node of degree one, copy
    it into its neighbour and remove that neighbour's edges from every coded
    node; stop when nothing is NULL (success) or no degree-one node is left
    (failure).  ``pick`` chooses among the current degree-one nodes (default:
    the first); returns the set of recovered sources."""
    residual = {c: set(code.cells[c]) for c in cell_subset}
    known: set = set()
    while len(known) < code.num_sources:
        ones = [c for c, r in residual.items() if len(r) == 1]
        if not ones:
            break
        c = ones[0] if pick is None else pick(ones)
        (s,) = residual[c]
        known.add(s)
        for r in residual.values():
            r.discard(s)
    return known


@dataclass
class Schedule:
    """Result of the wave peel: per source its depth (round, 0 = not
    recovered) and resolver cell (-1 = none); ``order`` lists (s, resolver,
    depth) sorted by (depth, s)."""

    ok: bool
    depth: list
    resolver: list
    order: list

    @property
    def num_waves(self) -> int:
        return max(self.depth) if self.depth else 0

    @property
    def recovered(self) -> list:
        return [1 if d > 0 else 0 for d in self.depth]


def wave_schedule_naive(code: Code, cell_subset) -> Schedule:
    """Parallel-round reading of the Section I-A decoder, written out plainly.

    Round r looks at every surviving cell with exactly one unknown source at
    the start of the round; each such source takes as resolver the lowest
    such cell id and gets depth r.  A round that recovers nothing ends the
    peel.  Cost O(rounds x edges): for small codes."""
    S = code.num_sources
    depth = [0] * S
    resolver = [-1] * S
    cells = sorted(cell_subset)
    r = 0
    while True:
        r += 1
        found: dict = {}
        for c in cells:
            unknown = [t for t in code.cells[c] if depth[t] == 0]
            if len(unknown) == 1:
                s = unknown[0]
                if s not in found or c < found[s]:
                    found[s] = c
        if not found:
            break
        for s, c in found.items():
            depth[s] = r
            resolver[s] = c
    order = sorted(((s, resolver[s], depth[s]) for s in range(S) if depth[s] > 0),
                   key=lambda x: (x[2], x[0]))
    return Schedule(ok=all(d > 0 for d in depth), depth=depth,
                    resolver=resolver, order=order)


def wave_schedule(code: Code, cell_subset) -> Schedule:
    """Same contract as ``wave_schedule_naive`` but each round only revisits
    the cells whose unknown count just dropped to one (the count of unknown
    sources per cell is kept up to date), so large codes finish in seconds.
    Tests pin the two against each other."""
    S = code.num_sources
    depth = [0] * S
    resolver = [-1] * S
    alive = sorted(cell_subset)
    cells_of_src: list = [[] for _ in range(S)]
    unknown_cnt = {}
    for c in alive:
        unknown_cnt[c] = len(code.cells[c])
        for t in code.cells[c]:
            cells_of_src[t].append(c)
    frontier = [c for c in alive if unknown_cnt[c] == 1]
    r = 0
    while frontier:
        r += 1
        found: dict = {}
        for c in frontier:
            if unknown_cnt[c] != 1:
                continue
            unknown = [t for t in code.cells[c] if depth[t] == 0]
            s = unknown[0]
            if s not in found or c < found[s]:
                found[s] = c
        if not found:
            break
        nxt = []
        for s, c in found.items():
            depth[s] = r
            resolver[s] = c
        for s in found:
            for c in cells_of_src[s]:
                unknown_cnt[c] -= 1
                if unknown_cnt[c] == 1:
                    nxt.append(c)
        frontier = nxt
    order = sorted(((s, resolver[s], depth[s]) for s in range(S) if depth[s] > 0),
                   key=lambda x: (x[2], x[0]))
    return Schedule(ok=all(d > 0 for d in depth), depth=depth,
                    resolver=resolver, order=order)


def decodable(code: Code, erased_cols) -> bool:
    return wave_schedule(code, surviving_cells(code, erased_cols)).ok


# --------------------------------------------------------------------------
# Numeric path over real matrices (XOR read as +, its inverse as -)
# --------------------------------------------------------------------------


def row_block(A: np.ndarray, s: int, h: int) -> np.ndarray:
    """Source s = rows [s h, (s+1) h) of A (Remark 2.1 partitioning); rows
    past the end of A read as zero (padding of the last blocks)."""
    M, K = A.shape
    out = np.zeros((h, K), dtype=np.float64)
    lo, hi = s * h, min((s + 1) * h, M)
    if lo < hi:
        out[: hi - lo] = A[lo:hi]
    return out


def encode(code: Code, A: np.ndarray, h: int, cell: int) -> np.ndarray:
    """Worker-side encoding (Section III-A, Example 1): the coded operand of
    a cell is the sum of its sources' row blocks, in ascending source id,
    in FP64 from the given inputs."""
    acc = np.zeros((h, A.shape[1]), dtype=np.float64)
    for s in code.cells[cell]:
        acc += row_block(A, s, h)
    return acc


def coded_products(code: Code, A: np.ndarray, B: np.ndarray, h: int, cells):
    """P_c = A_c B for every listed cell (the sigma dot products a processor
    executes, Section III-A), FP64.  Returns {cell: h x N array}."""
    B64 = np.asarray(B, dtype=np.float64)
    return {c: encode(code, A, h, c) @ B64 for c in cells}


def peel_decode(code: Code, products: dict, sched: Schedule, h: int, N: int):
    """Numeric BP peel along ``sched``: for each (s, r, d) in order,
    C_s = P_r - sum_{t in supp(r), t != s, ascending} C_t.  Returns
    {s: h x N FP64} for the recovered sources."""
    C: dict = {}
    for s, r, _d in sched.order:
        acc = products[r].copy()
        for t in code.cells[r]:
            if t != s:
                acc -= C[t]
        C[s] = acc
    return C


def reference_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The uncoded product A B in FP64."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


def coded_matmul(code: Code, A: np.ndarray, B: np.ndarray, h: int, erased_cols):
    """Whole path: schedule, encode, products of the surviving cells, peel.
    Returns (C as an (S h) x N FP64 array with unrecovered blocks NaN,
    schedule)."""
    cells = surviving_cells(code, erased_cols)
    sched = wave_schedule(code, cells)
    N = B.shape[1]
    used = sorted(set(r for _s, r, _d in sched.order))
    P = coded_products(code, A, B, h, used)
    Cd = peel_decode(code, P, sched, h, N)
    C = np.full((code.num_sources * h, N), np.nan)
    for s, blk in Cd.items():
        C[s * h:(s + 1) * h] = blk
    return C, sched


def expansion(code: Code, sched: Schedule) -> dict:
    """Integer expansion of every recovered C_s over the products: the map
    cell -> coefficient with C_s = sum_c coef_c P_c, following the peel."""
    coef: dict = {}
    for s, r, _d in sched.order:
        e = {r: 1}
        for t in code.cells[r]:
            if t != s:
                for c, v in coef[t].items():
                    e[c] = e.get(c, 0) - v
        coef[s] = {c: v for c, v in e.items() if v != 0}
    return coef


def amplification(code: Code, sched: Schedule, products: dict, C: dict) -> dict:
    """kappa_s = sum_c |coef_{s,c}| ||P_c||_F / ||C_s||_F: how much the
    rounding error of the products can be magnified on the way to C_s."""
    coef = expansion(code, sched)
    out = {}
    for s, e in coef.items():
        num = sum(abs(v) * np.linalg.norm(products[c]) for c, v in e.items())
        den = np.linalg.norm(C[s])
        out[s] = float(num / den) if den > 0 else float("inf")
    return out


def propagation(code: Code, sched: Schedule, products: dict, C: dict) -> dict:
    """nu_s = sqrt(sum_c coef_{s,c}^2 ||P_c||_F^2) / ||C_s||_F: the factor by
    which independent relative errors of size eps in every product grow, on
    average, on the way to C_s (eps nu_s is the expected relative error of
    C_s; kappa_s is its worst case).  nu_s = 1 for a source copied from a
    degree-one cell."""
    coef = expansion(code, sched)
    out = {}
    for s, e in coef.items():
        num = np.sqrt(sum(float(v) ** 2 * np.linalg.norm(products[c]) ** 2 for c, v in e.items()))
        den = np.linalg.norm(C[s])
        out[s] = float(num / den) if den > 0 else float("inf")
    return out


def all_erasure_patterns(n: int, max_e: int):
    """Every set of at most max_e erased columns."""
    for e in range(max_e + 1):
        yield from itertools.combinations(range(n), e)


def eps_construction_b_closed_form(n: int, k: int, b: int, q_e: int) -> float:
    """Exact worst-case overhead of Construction B: the t = ceil(k / 2^{q_e})
    tallest projections have heights |p|(k-1) + 2^{q_e}(b-1) + 1, and the
    sum of their |p| is the Lemma B.1 sum over n slopes minus the one over
    the n - t slopes nearest zero, so
    eps = ((k-1)(L(n) - L(n-t)) + t (2^{q_e}(b-1) + 1)) / (k b) - 1,
    L = Lemma B.1.  (Appendix B writes the |p| sums with Appendix A's phi;
    Lemma B.1 is the sum for this slope set.)"""
    t = -(-k // 2 ** q_e)
    L = lemma_b1_closed_form
    Lnt = L(n - t) if n - t > 0 else 0
    return ((k - 1) * (L(n) - Lnt) + t * (2 ** q_e * (b - 1) + 1)) / (k * b) - 1.0


def reference_block(A: np.ndarray, B: np.ndarray, s: int, h: int) -> np.ndarray:
    """C_s = A_s B in FP64 for one source (sampled checks at full size)."""
    return row_block(A, s, h) @ np.asarray(B, dtype=np.float64)


def eps_construction_a_closed_form(n: int, k: int, b: int) -> float:
    """Exact worst-case overhead of Construction A (Appendix A, before the
    bounds): (k-1)/(2 k b) (phi(n) + phi(n-1) - phi(n-k) - phi(n-k-1)),
    phi(x) = floor(x/2)(floor(x/2)+1)."""
    def phi(x):
        return (x // 2) * (x // 2 + 1) if x >= 0 else 0
    return (k - 1) / (2 * k * b) * (phi(n) + phi(n - 1) - phi(n - k) - phi(n - k - 1))



# --------------------------------------------------------------------------
# Exact-slice coded products (fixed-point digit planes, exact integer peel)
# --------------------------------------------------------------------------
#
# A (per row position j in [0, h), shared by every source block so that the
# rows summed into one coded row share a scale) and B (per column n) become
# integers x_int = rint(x 2^(bits - e)), with 2^(e-1) <= max|x| < 2^e.  Each
# integer is cut into S balanced digits of w bits (most significant first),
# x_int = sum_i 2^(w (S-1-i)) D_i with |D_i| <= 2^(w-1).  A coded digit plane
# is the plain sum of its sources' digit planes (no carry), so it stays
# linear in the sources; w is chosen from the code's largest degree sigma so
# that sigma 2^(w-1) <= 256 keeps every coded digit an integer that bf16
# holds exactly.  The digit pairs (i, l) with i + l <= S - 1 are kept and
# grouped by diagonal d = i + l:
#   Q_c = sum_d 2^(w (S-1-d)) sum_{i+l=d} D_i(A_c) D_l(B),
# an exact integer, linear in the sources; the peel subtracts these exactly
# and C_s = RN_fp32(Q_s 2^(w (S-1) - 2 bits + e_A[j] + e_B[n])).

EXACT_BITS = 24  # target fixed-point precision per operand (FP32 significand)


def exact_slice_params(sigma: int):
    """(w, S, bits): digit width, digit count and fixed-point bits for a
    code of largest degree sigma; w = min(8, 9 - ceil(log2 sigma)),
    S = ceil(24 / w), bits = min(24, w S - 1) (so the top balanced digit
    stays within 2^(w-1))."""
    if sigma < 1:
        raise ValueError("sigma >= 1")
    w = min(8, 9 - (sigma - 1).bit_length())
    if w < 1:
        raise ValueError("sigma too large for exact slices")
    S = -(-EXACT_BITS // w)
    bits = min(EXACT_BITS, w * S - 1)
    return w, S, bits


def exact_row_exponents(A: np.ndarray, h: int) -> np.ndarray:
    """e_A[j] for row position j: the binary exponent of the largest |A[r, k]|
    over the rows r = j (mod h) of A (frexp convention; 0 when all are 0)."""
    A64 = np.abs(np.asarray(A, dtype=np.float64))
    amax = np.zeros(h)
    if A64.size:
        rmax = A64.max(axis=1)
        for j in range(min(h, A64.shape[0])):
            amax[j] = rmax[j::h].max()
    return np.frexp(amax)[1].astype(np.int64)


def exact_col_exponents(B: np.ndarray) -> np.ndarray:
    """e_B[n]: the binary exponent of the largest |B[k, n]| over k."""
    B64 = np.abs(np.asarray(B, dtype=np.float64))
    amax = B64.max(axis=0) if B64.shape[0] else np.zeros(B64.shape[1])
    return np.frexp(amax)[1].astype(np.int64)


def fixed_point(X: np.ndarray, e, bits: int) -> np.ndarray:
    """rint(X 2^(bits - e)) as int64 (e broadcast against X)."""
    return np.rint(np.ldexp(np.asarray(X, dtype=np.float64), bits - np.asarray(e))).astype(np.int64)


def balanced_digits(X: np.ndarray, w: int, S: int) -> list:
    """The S balanced base-2^w digits of the integers X, most significant
    first: lower digits in [-2^(w-1), 2^(w-1)), the top digit takes the
    rest."""
    half, mask = 1 << (w - 1), (1 << w) - 1
    x = np.array(X, dtype=np.int64)
    digits = [None] * S
    for i in range(S - 1, 0, -1):
        d = ((x + half) & mask) - half
        digits[i] = d
        x = (x - d) >> w
    digits[0] = x
    return digits


def exact_source_digits(A: np.ndarray, eA: np.ndarray, s: int, h: int, w: int, S: int, bits: int):
    """Digit planes of source block s (rows past the end of A are zero)."""
    blk = row_block(A, s, h)
    return balanced_digits(fixed_point(blk, eA[:, None], bits), w, S)


def int_matmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Exact product of integer matrices through the FP64 matmul: every partial
    sum is an integer of magnitude at most K max|X| max|Y| < 2^53, so any
    summation order gives the exact result."""
    K = X.shape[1]
    bound = float(K) * float(np.abs(X).max(initial=0)) * float(np.abs(Y).max(initial=0))
    if bound >= 2.0 ** 53:
        raise ValueError("integer product not exact in FP64")
    return (X.astype(np.float64) @ Y.astype(np.float64)).astype(np.int64)


def exact_diagonals(Ad: list, Bd: list, S: int) -> list:
    """P^d = sum_{i+l=d} Ad[i] Bd[l] for d = 0 .. S-1 (exact int64)."""
    out = []
    for d in range(S):
        Pd = np.zeros((Ad[0].shape[0], Bd[0].shape[1]), dtype=np.int64)
        for i in range(d + 1):
            Pd += int_matmul(Ad[i], Bd[d - i])
        out.append(Pd)
    return out


def exact_q(Ad: list, Bd: list, w: int, S: int) -> np.ndarray:
    """Q = sum_{d <= S-1} 2^(w (S-1-d)) P^d, exact int64."""
    q = np.zeros((Ad[0].shape[0], Bd[0].shape[1]), dtype=np.int64)
    for d, Pd in enumerate(exact_diagonals(Ad, Bd, S)):
        q += Pd << (w * (S - 1 - d))
    return q


def exact_to_float(q: np.ndarray, eA: np.ndarray, eB: np.ndarray, w: int, S: int, bits: int) -> np.ndarray:
    """C = RN_fp32(q 2^(w (S-1) - 2 bits + e_A[j] + e_B[n])): exact to FP64
    (|q| < 2^53), exact power-of-two scaling, one rounding to FP32."""
    expo = w * (S - 1) - 2 * bits + eA[:, None] + eB[None, :]
    return np.ldexp(q.astype(np.float64), expo).astype(np.float32)


def exact_slice_coded_matmul(code: Code, A: np.ndarray, B: np.ndarray, h: int, erased_cols):
    """Whole exact-slice path: schedule (Section I-A waves), worker-side
    encode of every digit plane (Section III-A, sums without carry), the
    diagonal digit products Q_c of the resolvers, the peel on exact integers
    C_s = Q_r - sum_{t in supp(r), t != s} C_t, and one rounding to FP32.
    Returns (C as an (S_src h) x N float32 array with unrecovered blocks
    NaN, {s: exact int64 Q_s}, schedule)."""
    w, S, bits = exact_slice_params(code.sigma)
    N = B.shape[1]
    eA = exact_row_exponents(A, h)
    eB = exact_col_exponents(B)
    Bd = balanced_digits(fixed_point(B, eB[None, :], bits), w, S)
    cells = surviving_cells(code, erased_cols)
    sched = wave_schedule(code, cells)
    used = sorted(set(r for _s, r, _d in sched.order))
    src = {}
    Q = {}
    for c in used:
        Dc = [np.zeros((h, A.shape[1]), dtype=np.int64) for _ in range(S)]
        for s in code.cells[c]:
            if s not in src:
                src[s] = exact_source_digits(A, eA, s, h, w, S, bits)
            for i in range(S):
                Dc[i] += src[s][i]
        Q[c] = exact_q(Dc, Bd, w, S)
    CQ: dict = {}
    for s, r, _d in sched.order:
        acc = Q[r].copy()
        for t in code.cells[r]:
            if t != s:
                acc -= CQ[t]
        CQ[s] = acc
    C = np.full((code.num_sources * h, N), np.nan, dtype=np.float32)
    for s, q in CQ.items():
        C[s * h:(s + 1) * h] = exact_to_float(q, eA, eB, w, S, bits)
    return C, CQ, sched


def exact_coded_diagonals(code: Code, A: np.ndarray, B: np.ndarray, h: int, cell: int) -> list:
    """The S diagonal digit products P_c^d of one cell (what a worker's
    exact-slice product computes), from the carry-free coded digit planes."""
    w, S, bits = exact_slice_params(code.sigma)
    eA = exact_row_exponents(A, h)
    eB = exact_col_exponents(B)
    Bd = balanced_digits(fixed_point(B, eB[None, :], bits), w, S)
    Dc = [np.zeros((h, A.shape[1]), dtype=np.int64) for _ in range(S)]
    for s in code.cells[cell]:
        sd = exact_source_digits(A, eA, s, h, w, S, bits)
        for i in range(S):
            Dc[i] += sd[i]
    return exact_diagonals(Dc, Bd, S)


def exact_slice_block(A: np.ndarray, B: np.ndarray, s: int, h: int, sigma: int, cols=None, eA=None):
    """The exact-slice product of one source block computed directly (no
    code, no peel), optionally on a subset of B's columns: (float32 block,
    exact int64 Q_s).  e_A comes from all of A (pass it when sampling many
    blocks of a large A), e_B from the chosen columns (a column's exponent
    depends on that column only)."""
    w, S, bits = exact_slice_params(sigma)
    Bc = np.asarray(B)[:, cols] if cols is not None else np.asarray(B)
    if eA is None:
        eA = exact_row_exponents(A, h)
    eB = exact_col_exponents(Bc)
    Bd = balanced_digits(fixed_point(Bc, eB[None, :], bits), w, S)
    q = exact_q(exact_source_digits(A, eA, s, h, w, S, bits), Bd, w, S)
    return exact_to_float(q, eA, eB, w, S, bits), q


# --------------------------------------------------------------------------
# Two-dimensional scheme (Section III-A, Examples 1 and 2)
# --------------------------------------------------------------------------
#
# C = A B with A cut into b row blocks of h rows and B into k column blocks
# of w columns; source s = z k + l (the grid pixel of Section III-C) is the
# output block C_s = A_z B_l.  Table I's v_{(i-1)m+j} = a_i b_j is the
# b = k = m case with z = i - 1, l = j - 1.


def source_zl(code: Code, s: int):
    """(row block of A, column block of B) of source s: s = z k + l."""
    return divmod(s, code.k)


def terms_2d(code: Code, cell: int):
    """Factoring of a cell's sum of block products into products of summed
    operands: grouped by A block (each z with its set of l), blocks of A with
    the same set of l merged -- or the same by B block -- whichever needs
    fewer products (ties: by A block).  Returns a list of (Z, L) with
    sum_{s in cell} A_z(s) B_l(s) = sum_terms (sum_{z in Z} A_z)(sum_{l in L} B_l)."""
    zl = [source_zl(code, s) for s in code.cells[cell]]

    def factor(pairs):
        groups = {}
        for a, b_ in pairs:
            groups.setdefault(a, set()).add(b_)
        merged = {}
        for a, bs in groups.items():
            merged.setdefault(tuple(sorted(bs)), []).append(a)
        return [(tuple(sorted(as_)), bs) for bs, as_ in merged.items()]

    by_row = factor(zl)
    by_col = [(Z, L) for (L, Z) in factor([(l, z) for z, l in zl])]
    best = by_row if len(by_row) <= len(by_col) else by_col
    return sorted(best)


def gray_cells_2d(code: Code) -> list:
    """Cells that are not one product of a summed A operand and a summed B
    operand (T > 1): the encoding of these has to happen on the worker
    (Section III-A, the gray cells of Tables I and III)."""
    return [c for c in range(code.num_cells) if len(terms_2d(code, c)) > 1]


def col_block(B: np.ndarray, l: int, w: int) -> np.ndarray:
    """Column block l of B (columns past the end read as zero)."""
    K, N = B.shape
    out = np.zeros((K, w), dtype=np.float64)
    lo, hi = l * w, min((l + 1) * w, N)
    if lo < hi:
        out[:, : hi - lo] = B[:, lo:hi]
    return out


def coded_products_2d(code: Code, A: np.ndarray, B: np.ndarray, h: int, w: int, cells):
    """P_c = sum_{s in supp(c)} A_z(s) B_l(s), the definition (one block
    product per source, summed in ascending source id), FP64."""
    out = {}
    for c in cells:
        acc = np.zeros((h, w))
        for s in code.cells[c]:
            z, l = source_zl(code, s)
            acc += row_block(A, z, h) @ col_block(B, l, w)
        out[c] = acc
    return out


def coded_matmul_2d(code: Code, A: np.ndarray, B: np.ndarray, h: int, w: int, erased_cols):
    """Whole two-dimensional path: schedule, products of the resolvers, the
    peel (the same wave contract), C assembled from its b x k blocks.
    Returns (C as (b h) x (k w) FP64 with unrecovered blocks NaN, schedule)."""
    cells = surviving_cells(code, erased_cols)
    sched = wave_schedule(code, cells)
    used = sorted(set(r for _s, r, _d in sched.order))
    P = coded_products_2d(code, A, B, h, w, used)
    Cd = peel_decode(code, P, sched, h, w)
    C = np.full((code.b * h, code.k * w), np.nan)
    for s, blk in Cd.items():
        z, l = source_zl(code, s)
        C[z * h:(z + 1) * h, l * w:(l + 1) * w] = blk
    return C, sched


# --------------------------------------------------------------------------
# Straggler-time model (Section IV, Eq. (eqnTtotal))
# --------------------------------------------------------------------------


def task_times(code: Code, mu: float, rng: np.random.Generator, scale_by_degree: bool = True, X=None) -> np.ndarray:
    """T_c for every cell: a processor doing sigma_c long dot products has
    the exponential cdf of rate mu stretched by sigma_c (Section IV-A), i.e.
    T_c = sigma_c X_c with X_c ~ Exp(mu); sigma_c = 1 when not scaling.  X
    (the unscaled draws) may be given instead of drawn."""
    if X is None:
        X = rng.exponential(1.0 / mu, size=code.num_cells)
    deg = np.array([len(c) for c in code.cells], dtype=np.float64)
    return np.asarray(X, dtype=np.float64) * (deg if scale_by_degree else 1.0)


def coded_matmul_cells(code: Code, A: np.ndarray, B: np.ndarray, h: int, cells):
    """The whole path when exactly the given cells' products arrived (a
    processor-level erasure pattern).  Returns (C with unrecovered blocks
    NaN, schedule)."""
    sched = wave_schedule(code, sorted(cells))
    N = B.shape[1]
    used = sorted(set(r for _s, r, _d in sched.order))
    P = coded_products(code, A, B, h, used)
    Cd = peel_decode(code, P, sched, h, N)
    C = np.full((code.num_sources * h, N), np.nan)
    for s, blk in Cd.items():
        C[s * h:(s + 1) * h] = blk
    return C, sched


def decodes(code: Code, cell_subset) -> bool:
    """Peeling over the given cells recovers every source (Section I-A)."""
    return len(sequential_peel(code, list(cell_subset))) == code.num_sources


def parallel_task_time_brute(code: Code, T) -> float:
    """min over decodable cell sets S of max_{c in S} T_c, by enumerating
    every subset (tiny codes only)."""
    best = np.inf
    cells = range(code.num_cells)
    for r in range(1, code.num_cells + 1):
        for S in itertools.combinations(cells, r):
            t = max(T[c] for c in S)
            if t < best and decodes(code, S):
                best = t
    return float(best)


def first_decodable(code: Code, order) -> int:
    """Number of arrivals after which the cells received so far (in the
    given order) peel completely, or -1: the sink starts decoding as soon as
    a decodable set has arrived."""
    for i in range(1, len(order) + 1):
        if decodes(code, order[:i]):
            return i
    return -1


# --------------------------------------------------------------------------
# Bounds on the number of columns (Section III-B)
# --------------------------------------------------------------------------


def bound_k_equals_sigma(k: int, b: int) -> int:
    """n <= kb + 1 + max{k - 3, 0} when k = sigma (quoted from Paterson et
    al.)."""
    return k * b + 1 + max(k - 3, 0)


def bound_paterson(k: int, b: int, sigma: int) -> int:
    """n <= k + sigma - 1 + floor(sigma (sigma - 1)(b - 1) / ((k - sigma) b
    + sigma - 1)) for k > sigma: the form the Section V simulations use for
    the number of stragglers n - k."""
    return k + sigma - 1 + (sigma * (sigma - 1) * (b - 1)) // ((k - sigma) * b + sigma - 1)


def code_from_columns(name: str, k: int, b: int, columns) -> Code:
    """A code given by its columns, each a list of cells (source-id
    tuples, 0-based)."""
    cells, col_of_cell = [], []
    for j, col in enumerate(columns):
        for cell in col:
            cells.append(tuple(sorted(cell)))
            col_of_cell.append(j)
    n = len(columns)
    return Code(name=name, n=n, k=k, b=b, num_sources=b * k, cells=cells, col_of_cell=col_of_cell,
                heights=[len(c) for c in columns], proj=[None] * n, e=n - k)


def is_array_bpxor(code: Code) -> bool:
    """Every pattern of n - k erased columns peels completely (block MDS
    under BP decoding, Section III-A definition)."""
    return all(decodable(code, er) for er in itertools.combinations(range(code.n), code.n - code.k))
