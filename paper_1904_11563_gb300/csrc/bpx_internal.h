// Internal declarations shared by the host code and the CUDA translation
// units of libbpx.  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "bpx.h"

// Host-side code graph (Section III): cells of each column, sources of each
// cell, and the transposed source -> cells adjacency the scheduler walks.
struct bpx_code {
  int variant = 0, n = 0, k = 0, e = 0, b = 0, q_e = 0;
  int S = 0, num_cells = 0, num_edges = 0, sigma = 0;
  double eps = 0.0;
  std::vector<int32_t> col_ptr, cell_ptr, cell_src, col_of_cell, heights, proj_p, proj_q;
  std::vector<int32_t> src_ptr, src_cell;  // source -> cells (ascending cell id)
  // Two-dimensional scheme (source s = z k + l is the block product A_z B_l):
  // every cell as a list of products of summed operands, term i of cell c at
  // [t2_ptr[c], t2_ptr[c+1]) = (A operand t2_a[i], B operand t2_b[i]); A
  // operand e sums the row blocks a2_blk[a2_ptr[e] ..], B operand f the
  // column blocks b2_blk[b2_ptr[f] ..]; t2_order lists the cells by
  // decreasing term count (ties by id); gray2 counts cells with > 1 term.
  std::vector<int32_t> t2_ptr, t2_a, t2_b, a2_ptr, a2_blk, b2_ptr, b2_blk, t2_order;
  int gray2 = 0;
};

namespace bpx {

// Thread-local error text; returns `code` for `return fail(...)`.
int fail(int code, const char* fmt, ...);
void clear_error();

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offsets of every array in the device workspace.  The graph section is
// filled once by bpx_workspace_init; the plan section by bpx_schedule; the
// product and staging sections by bpx_coded_products.
struct WsLayout {
  // graph (int32)
  size_t g_hdr, g_col_of_cell, g_cell_ptr, g_cell_src, g_src_ptr, g_src_cell;
  size_t g_t2_ptr, g_t2_a, g_t2_b, g_a2_ptr, g_a2_blk, g_b2_ptr, g_b2_blk, g_t2_order;
  // plan (int32)
  size_t p_info, p_ctr, p_cnt, p_surv, p_direct, p_front0, p_front1, p_word;
  size_t p_depth, p_resolver, p_order, p_wave_ptr, p_cursor;
  size_t p_pl_res, p_pl_ptr, p_pl_list;  // peel list: resolver and subtrahends per order entry
  size_t plan_end;
  // products (float, num_cells * h * N)
  size_t products;
  // staging for the tensor-core paths (bf16 / fp8 operands; exact-slice
  // digit planes in a_hi / b_hi)
  size_t a_hi, a_lo, b_hi, b_lo, a_scale, b_scale;
  // exact-slice: max |A| per row position (h words) then max |B| per column
  // (N words), as float bits; decoded sources as exact int64 (S h N)
  size_t ex_amax, ex_c64;
  // exact-slice, digits narrower than 8 bits: every source row's digit planes
  // as int8, computed once (0 = no such region)
  size_t ex_src;
  size_t total;
};

// Exact-slice representation of a code (see bpx_exact_params): digit width
// w, digit planes S (also the number of kept diagonals), fixed-point bits,
// K elements per exact FP32 accumulation segment, K padded to 64.
struct ExactParams {
  int w = 0, S = 0, bits = 0, seg = 0, Kp = 0;
};

// Fills *P for the code's sigma and K; BPX_ERR_UNSUPPORTED (with a message)
// when the digits or the exact integer sums would not fit.
int exact_params(const bpx_code* c, int K, ExactParams* P);

// twod: the two-dimensional scheme (products are h x (N / k) blocks, operand
// staging holds the summed A and B operands of the code's factored cells).
WsLayout ws_layout(const bpx_code* code, int M, int N, int K, int h, int precision, bool twod = false);

// Completes a code from its cells (supports ascending) and the column of
// each cell (grouped by ascending column): CSR views, source -> cells,
// sigma, the worst-case overhead, the two-dimensional factoring.  c->n, k,
// b, S and e must be set; col_ptr / heights / projections are derived when
// empty.
void finish_code(bpx_code* c, const std::vector<std::vector<int32_t>>& cells,
                 const std::vector<int32_t>& col_of_cell);

// Factors every cell for the two-dimensional scheme (fills the t2_* / a2_* /
// b2_* arrays of the code).
void build_terms_2d(bpx_code* c);

constexpr int32_t kWsMagic = 0x42505831;  // "BPX1"

// Graph header layout (int32 words at g_hdr)
enum { HDR_MAGIC = 0, HDR_N, HDR_S, HDR_CELLS, HDR_EDGES, HDR_SIGMA, HDR_LEN = 16 };

// Plan counters at p_ctr (int32 words)
enum {
  CTR_NSURV = 0,  // surviving cells
  CTR_NWAVES,     // rounds
  CTR_NREC,       // recovered sources
  CTR_NF,         // frontier size (scratch)
  CTR_NNEXT,      // next frontier size (scratch)
  CTR_NNEW,       // sources recovered this round (scratch)
  CTR_ERR,        // device error code raised by a kernel self-check
  CTR_PLAN,       // kPlanReady once a whole plan is in place (zeroed by bpx_workspace_init)
  CTR_LEN = 16
};
constexpr int32_t kPlanReady = 0x504C414E;  // "PLAN"

}  // namespace bpx
