// Straggler-time model (Section IV): the sink starts the peel as soon as the
// processor outputs received so far form a decodable set -- the time
// min over decodable S of max_{c in S} T_c of Eq. (eqnTtotal).  Given the
// order in which the cells' products arrive, this host routine peels online
// (Section I-A decoder): each arriving cell with exactly one unrecovered
// source recovers it, and every recovery lowers the unknown count of the
// other cells holding that source, which may make them resolvers in turn.
// Peeling reaches the same recovered set whatever order it takes, so the
// arrival after which every source is recovered is the first decodable
// prefix.
#include <vector>

#include "bpx_internal.h"

extern "C" int bpx_first_decodable(const bpx_code* c, const int32_t* order, int n, int32_t* recovered_after,
                                   int32_t* first) {
  bpx::clear_error();
  if (!c || !order || !first) return bpx::fail(BPX_ERR_INVAL, "bpx_first_decodable: NULL argument");
  if (n < 0 || n > c->num_cells) return bpx::fail(BPX_ERR_INVAL, "bpx_first_decodable: n = %d", n);
  std::vector<int32_t> unknown(c->num_cells);
  std::vector<char> arrived(c->num_cells, 0), known(c->S, 0);
  for (int cell = 0; cell < c->num_cells; ++cell) unknown[cell] = c->cell_ptr[cell + 1] - c->cell_ptr[cell];
  std::vector<int32_t> ready;
  int nrec = 0;
  *first = -1;
  for (int i = 0; i < n; ++i) {
    const int32_t cell = order[i];
    if (cell < 0 || cell >= c->num_cells || arrived[cell])
      return bpx::fail(BPX_ERR_INVAL, "bpx_first_decodable: order[%d] = %d is not a new cell", i, cell);
    arrived[cell] = 1;
    if (unknown[cell] == 1) ready.push_back(cell);
    while (!ready.empty()) {
      const int32_t r = ready.back();
      ready.pop_back();
      if (unknown[r] != 1) continue;  // its last source was recovered meanwhile
      int32_t s = -1;
      for (int e = c->cell_ptr[r]; e < c->cell_ptr[r + 1]; ++e)
        if (!known[c->cell_src[e]]) s = c->cell_src[e];
      known[s] = 1;
      ++nrec;
      for (int e = c->src_ptr[s]; e < c->src_ptr[s + 1]; ++e) {
        const int32_t other = c->src_cell[e];
        if (--unknown[other] == 1 && arrived[other]) ready.push_back(other);
      }
    }
    if (recovered_after) recovered_after[i] = nrec;
    if (nrec == c->S && *first < 0) *first = i + 1;
  }
  return BPX_OK;
}
