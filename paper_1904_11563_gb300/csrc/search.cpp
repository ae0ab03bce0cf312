// Code-parameter tooling (Section III-B), host only:
//   - the bounds on the number of columns n,
//   - codes given by their cells (any array code a caller brings),
//   - a search for equal-height array BP-XOR codes: n columns of b cells,
//     every cell the XOR (here: sum) of at most sigma of the b k sources,
//     decodable by peeling from any k columns.
// The search is simulated annealing over the cells' supports with cost =
// the sources that the (n - k)-column erasure patterns leave unknown, summed
// over the patterns, plus a penalty for sources in fewer than n - k + 1
// columns (the appearance count Theorem 3.1 starts from).  Supports are bit
// masks (b k <= 64), so one peel is a few passes of mask operations.
// Optionally systematic (the first k columns fixed to single sources), and
// run as independent chains on host threads.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <random>
#include <thread>
#include <vector>

#include "bpx_internal.h"

namespace {

using Mask = uint64_t;

int popc(Mask m) { return __builtin_popcountll(m); }

struct Problem {
  int n, k, b, sigma, S;
  std::vector<uint32_t> patterns;  // every set of n - k erased columns
  Mask all;
};

}  // namespace

extern "C" int bpx_bound_k_equals_sigma(int k, int b, int* n_max) {
  bpx::clear_error();
  if (!n_max || k < 1 || b < 1) return bpx::fail(BPX_ERR_INVAL, "bpx_bound_k_equals_sigma: bad arguments");
  *n_max = k * b + 1 + std::max(k - 3, 0);
  return BPX_OK;
}

extern "C" int bpx_bound_paterson(int k, int b, int sigma, int* n_max) {
  bpx::clear_error();
  if (!n_max || k <= sigma || sigma < 1 || b < 1)
    return bpx::fail(BPX_ERR_INVAL, "bpx_bound_paterson: needs k > sigma >= 1, b >= 1");
  const long long num = static_cast<long long>(sigma) * (sigma - 1) * (b - 1);
  const long long den = static_cast<long long>(k - sigma) * b + sigma - 1;
  *n_max = static_cast<int>(k + sigma - 1 + num / den);
  return BPX_OK;
}

extern "C" int bpx_code_from_cells(int n, int k, int b, int num_cells, const int32_t* col_of_cell,
                                   const int32_t* cell_ptr, const int32_t* cell_src, int e, bpx_code** out) {
  bpx::clear_error();
  if (!out || !col_of_cell || !cell_ptr || !cell_src) return bpx::fail(BPX_ERR_INVAL, "bpx_code_from_cells: NULL");
  *out = nullptr;
  if (n < 1 || k < 1 || b < 1 || num_cells < 1 || e < 0 || e >= n)
    return bpx::fail(BPX_ERR_INVAL, "bpx_code_from_cells: bad n, k, b, cells or e");
  const int S = k * b;
  for (int c = 0; c < num_cells; ++c) {
    if (col_of_cell[c] < 0 || col_of_cell[c] >= n || (c > 0 && col_of_cell[c] < col_of_cell[c - 1]))
      return bpx::fail(BPX_ERR_INVAL, "bpx_code_from_cells: cells must be grouped by ascending column");
    if (cell_ptr[c + 1] <= cell_ptr[c]) return bpx::fail(BPX_ERR_INVAL, "bpx_code_from_cells: empty cell %d", c);
    for (int i = cell_ptr[c]; i < cell_ptr[c + 1]; ++i) {
      if (cell_src[i] < 0 || cell_src[i] >= S) return bpx::fail(BPX_ERR_INVAL, "bpx_code_from_cells: source out of range");
      if (i > cell_ptr[c] && cell_src[i] <= cell_src[i - 1])
        return bpx::fail(BPX_ERR_INVAL, "bpx_code_from_cells: supports must be ascending without repeats");
    }
  }
  bpx_code* code = new bpx_code();
  code->variant = BPX_LITERAL;
  code->n = n;
  code->k = k;
  code->b = b;
  code->S = S;
  code->e = e;
  std::vector<std::vector<int32_t>> cells(num_cells);
  for (int c = 0; c < num_cells; ++c) cells[c].assign(cell_src + cell_ptr[c], cell_src + cell_ptr[c + 1]);
  bpx::finish_code(code, cells, std::vector<int32_t>(col_of_cell, col_of_cell + num_cells));
  *out = code;
  return BPX_OK;
}

namespace {

// Sources left unknown after peeling the cells of the columns not in
// `erased`.
int unrecovered(const std::vector<Mask>& cells, const std::vector<int>& col, uint32_t erased, Mask all) {
  Mask known = 0;
  bool progress = true;
  while (progress && known != all) {
    progress = false;
    for (size_t c = 0; c < cells.size(); ++c) {
      if ((erased >> col[c]) & 1u) continue;
      const Mask u = cells[c] & ~known;
      if (u && !(u & (u - 1))) {
        known |= u;
        progress = true;
      }
    }
  }
  return popc(all & ~known);
}

// Annealing cost: the sources every erasure pattern leaves unknown (a
// smoother signal than the count of failing patterns), plus the shortfall of
// sources appearing in fewer than n - k + 1 columns.  Zero iff every pattern
// peels.
long long cost_smooth(const Problem& P, const std::vector<Mask>& cells, const std::vector<int>& col) {
  long long left = 0;
  for (uint32_t er : P.patterns) left += unrecovered(cells, col, er, P.all);
  long long short_by = 0;
  for (int s = 0; s < P.S; ++s) {
    uint32_t cols = 0;
    for (size_t c = 0; c < cells.size(); ++c)
      if ((cells[c] >> s) & 1u) cols |= 1u << col[c];
    const int have = __builtin_popcount(cols);
    if (have < P.n - P.k + 1) short_by += P.n - P.k + 1 - have;
  }
  return left + short_by;
}

struct Chain {
  bool found = false;
  long long moves = 0;
  std::vector<Mask> cells;
};

// One annealing chain from `seed`.  systematic: the first k columns are
// fixed single-source cells (column l, cell z = source z k + l) and only the
// parity columns' cells move.
Chain anneal(const Problem& P, int sigma, long long iters, unsigned long long seed, bool systematic) {
  Chain out;
  std::mt19937_64 rng(seed);
  const int n = P.n, k = P.k, b = P.b;
  std::vector<int> col(n * b);
  std::vector<Mask> cells(n * b);
  for (int c = 0; c < n * b; ++c) col[c] = c / b;
  const int first_free = systematic ? k * b : 0;
  if (systematic)
    for (int l = 0; l < k; ++l)
      for (int z = 0; z < b; ++z) cells[l * b + z] = Mask(1) << (z * k + l);
  auto rand_src = [&]() { return static_cast<int>(rng() % P.S); };
  auto restart = [&]() {  // every free cell a random support of 1 .. sigma sources
    for (int c = first_free; c < n * b; ++c) {
      Mask m = 0;
      const int d = 1 + static_cast<int>(rng() % sigma);
      while (popc(m) < d) m |= Mask(1) << rand_src();
      cells[c] = m;
    }
  };
  restart();
  long long cur = cost_smooth(P, cells, col);
  const long long epoch = std::max<long long>(20000, iters / 20);
  long long since = 0, best = cur;
  double T = 1.0;
  long long it = 0;
  const int nfree = n * b - first_free;
  for (; it < iters && cur > 0; ++it) {
    if (++since > epoch) {
      restart();
      cur = best = cost_smooth(P, cells, col);
      since = 0;
      T = 1.0;
    }
    const int c = first_free + static_cast<int>(rng() % nfree);
    const Mask old = cells[c];
    Mask m = old;
    const int r = static_cast<int>(rng() % 3);
    if (r == 0 && popc(m) < sigma) {
      m |= Mask(1) << rand_src();                       // add a source
    } else if (r == 1 && popc(m) > 1) {
      int drop = static_cast<int>(rng() % popc(m));      // remove one
      for (Mask t = m; t; t &= t - 1)
        if (drop-- == 0) m &= ~(t & (~t + 1));
    } else {
      int drop = static_cast<int>(rng() % popc(m));      // move one
      for (Mask t = m; t; t &= t - 1)
        if (drop-- == 0) m &= ~(t & (~t + 1));
      m |= Mask(1) << rand_src();
      if (m == 0) m = old;
    }
    if (m == old) continue;
    cells[c] = m;
    const long long nc = cost_smooth(P, cells, col);
    if (nc <= cur || std::exp((cur - nc) / T) > std::uniform_real_distribution<double>(0, 1)(rng)) {
      cur = nc;
      if (cur < best) {
        best = cur;
        since = 0;
      }
    } else {
      cells[c] = old;
    }
    T = std::max(0.02, T * (1.0 - 4.0 / epoch));
  }
  out.found = cur == 0;
  out.moves = it;
  out.cells = cells;
  return out;
}

}  // namespace

extern "C" int bpx_code_search_ex(int n, int k, int b, int sigma, long long iters, unsigned long long seed,
                                  int flags, int threads, bpx_code** out, long long* iters_used) {
  bpx::clear_error();
  if (!out) return bpx::fail(BPX_ERR_INVAL, "bpx_code_search: out is NULL");
  *out = nullptr;
  if (n < 2 || k < 1 || k >= n || b < 1 || sigma < 1 || k * b > 64 || n > 30 || iters < 1)
    return bpx::fail(BPX_ERR_INVAL, "bpx_code_search: needs 1 <= k < n <= 30, b k <= 64, sigma >= 1");
  if (threads < 1 || threads > 256) return bpx::fail(BPX_ERR_INVAL, "bpx_code_search: threads must be 1..256");
  if (flags & ~BPX_SEARCH_SYSTEMATIC) return bpx::fail(BPX_ERR_INVAL, "bpx_code_search: unknown flags %d", flags);
  Problem P{n, k, b, sigma, k * b, {}, 0};
  P.all = P.S == 64 ? ~Mask(0) : ((Mask(1) << P.S) - 1);
  const int e = n - k;
  for (uint32_t m = 0; m < (1u << n); ++m)
    if (__builtin_popcount(m) == e) P.patterns.push_back(m);
  const bool systematic = (flags & BPX_SEARCH_SYSTEMATIC) != 0;
  // Independent chains, chain t from seed + t; the result is the lowest t
  // that found a code, so it does not depend on the threads' timing.
  std::vector<Chain> chains(threads);
  {
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t)
      pool.emplace_back([&, t] { chains[t] = anneal(P, sigma, iters, seed + t, systematic); });
    chains[0] = anneal(P, sigma, iters, seed, systematic);
    for (auto& th : pool) th.join();
  }
  long long used = 0;
  int win = -1;
  for (int t = 0; t < threads; ++t) {
    used += chains[t].moves;
    if (win < 0 && chains[t].found) win = t;
  }
  if (iters_used) *iters_used = used;
  if (win < 0)
    return bpx::fail(BPX_ERR_UNSUPPORTED, "bpx_code_search: no code found in %lld moves", used);
  const std::vector<Mask>& cells = chains[win].cells;
  std::vector<int> col(n * b);
  for (int c = 0; c < n * b; ++c) col[c] = c / b;
  std::vector<std::vector<int32_t>> supp(cells.size());
  for (size_t c = 0; c < cells.size(); ++c)
    for (int s = 0; s < P.S; ++s)
      if ((cells[c] >> s) & 1u) supp[c].push_back(s);
  bpx_code* code = new bpx_code();
  code->variant = BPX_LITERAL;
  code->n = n;
  code->k = k;
  code->b = b;
  code->S = P.S;
  code->e = e;
  bpx::finish_code(code, supp, col);
  *out = code;
  return BPX_OK;
}

extern "C" int bpx_code_search(int n, int k, int b, int sigma, long long iters, unsigned long long seed,
                               bpx_code** out, long long* iters_used) {
  return bpx_code_search_ex(n, k, b, sigma, iters, seed, 0, 1, out, iters_used);
}
