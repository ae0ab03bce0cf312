// Two-dimensional scheme (Section III-A, Examples 1 and 2), host planning.
//
// Source s = z k + l is the output block A_z B_l (row block z of A, column
// block l of B); a cell's coded product is the sum of its sources' block
// products.  A cell is computed as few products of summed operands as its
// support allows: its sources grouped by A block (each z with the set of l it
// pairs with), A blocks with identical sets merged, giving terms
// (sum_{z in Z} A_z)(sum_{l in L} B_l); or the same grouped by B block --
// whichever gives fewer terms (ties: by A block).  A full rectangle of blocks
// is one product; a cell whose sources share neither an A block nor a B
// block (Tables I and III: the gray cells) needs one product per source,
// which is why its encoding has to happen on the worker.
#include <algorithm>
#include <map>
#include <vector>

#include "bpx_internal.h"

namespace bpx {
namespace {

using Set = std::vector<int32_t>;
using Term = std::pair<Set, Set>;  // (A blocks, B blocks)

// Groups (key, value) pairs by key, then merges keys with the same value set.
std::vector<std::pair<Set, Set>> factor(const std::vector<std::pair<int32_t, int32_t>>& kv) {
  std::map<int32_t, Set> by_key;
  for (auto& [a, b] : kv) by_key[a].push_back(b);
  std::map<Set, Set> by_values;
  for (auto& [a, bs] : by_key) {
    Set v = bs;
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    by_values[v].push_back(a);
  }
  std::vector<std::pair<Set, Set>> out;  // (keys, values)
  for (auto& [vals, keys] : by_values) {
    Set k = keys;
    std::sort(k.begin(), k.end());
    out.push_back({k, vals});
  }
  return out;
}

}  // namespace

void build_terms_2d(bpx_code* c) {
  c->t2_ptr.assign(1, 0);
  c->t2_a.clear();
  c->t2_b.clear();
  c->a2_ptr.assign(1, 0);
  c->a2_blk.clear();
  c->b2_ptr.assign(1, 0);
  c->b2_blk.clear();
  c->gray2 = 0;
  std::map<Set, int32_t> a_ops, b_ops;
  auto op_id = [](std::map<Set, int32_t>& ops, std::vector<int32_t>& ptr, std::vector<int32_t>& blk,
                  const Set& s) {
    auto it = ops.find(s);
    if (it != ops.end()) return it->second;
    const int32_t id = static_cast<int32_t>(ptr.size()) - 1;
    ops.emplace(s, id);
    blk.insert(blk.end(), s.begin(), s.end());
    ptr.push_back(static_cast<int32_t>(blk.size()));
    return id;
  };
  std::vector<int32_t> nterms(c->num_cells);
  for (int cell = 0; cell < c->num_cells; ++cell) {
    std::vector<std::pair<int32_t, int32_t>> zl, lz;
    for (int i = c->cell_ptr[cell]; i < c->cell_ptr[cell + 1]; ++i) {
      const int32_t s = c->cell_src[i];
      zl.push_back({s / c->k, s % c->k});
      lz.push_back({s % c->k, s / c->k});
    }
    std::vector<Term> rows, cols;
    for (auto& [Z, L] : factor(zl)) rows.push_back({Z, L});
    for (auto& [L, Z] : factor(lz)) cols.push_back({Z, L});
    std::vector<Term> terms = rows.size() <= cols.size() ? rows : cols;
    std::sort(terms.begin(), terms.end());
    for (auto& [Z, L] : terms) {
      c->t2_a.push_back(op_id(a_ops, c->a2_ptr, c->a2_blk, Z));
      c->t2_b.push_back(op_id(b_ops, c->b2_ptr, c->b2_blk, L));
    }
    c->t2_ptr.push_back(static_cast<int32_t>(c->t2_a.size()));
    nterms[cell] = static_cast<int32_t>(terms.size());
    if (terms.size() > 1) ++c->gray2;
  }
  c->t2_order.resize(c->num_cells);
  for (int i = 0; i < c->num_cells; ++i) c->t2_order[i] = i;
  std::stable_sort(c->t2_order.begin(), c->t2_order.end(),
                   [&](int32_t a, int32_t b) { return nterms[a] > nterms[b]; });
}

}  // namespace bpx
