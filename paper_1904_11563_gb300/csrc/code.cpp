// Code graphs of Section III, built on the host: the literal array codes of
// Table I and Table III, the systematic Mojette array, and the projection
// codes of Construction A (Cons33) and Construction B (cons35), each
// projection's bins placed by Eq. (moj1).  Also the workspace layout and
// the thread-local error text of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <new>

#include "bpx_internal.h"

namespace bpx {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

}  // namespace bpx

using bpx::fail;

namespace bpx {

void finish_code(bpx_code* c, const std::vector<std::vector<int32_t>>& cells,
                 const std::vector<int32_t>& col_of_cell) {
  c->col_of_cell = col_of_cell;
  if (c->col_ptr.empty()) {  // columns given only through col_of_cell
    c->col_ptr.assign(c->n + 1, 0);
    for (int32_t j : col_of_cell) ++c->col_ptr[j + 1];
    for (int j = 0; j < c->n; ++j) c->col_ptr[j + 1] += c->col_ptr[j];
  }
  if (c->heights.empty())
    for (int j = 0; j < c->n; ++j) c->heights.push_back(c->col_ptr[j + 1] - c->col_ptr[j]);
  if (c->proj_p.empty()) {
    c->proj_p.assign(c->n, 0);
    c->proj_q.assign(c->n, 0);
  }
  c->num_cells = static_cast<int>(cells.size());
  c->cell_ptr.assign(1, 0);
  c->cell_src.clear();
  c->sigma = 0;
  for (auto& s : cells) {
    c->cell_src.insert(c->cell_src.end(), s.begin(), s.end());
    c->cell_ptr.push_back(static_cast<int32_t>(c->cell_src.size()));
    c->sigma = std::max(c->sigma, static_cast<int>(s.size()));
  }
  c->num_edges = static_cast<int>(c->cell_src.size());
  // source -> cells, cells ascending
  std::vector<int32_t> deg(c->S + 1, 0);
  for (int32_t s : c->cell_src) ++deg[s + 1];
  c->src_ptr.assign(c->S + 1, 0);
  for (int s = 0; s < c->S; ++s) c->src_ptr[s + 1] = c->src_ptr[s] + deg[s + 1];
  c->src_cell.assign(c->num_edges, 0);
  std::vector<int32_t> fill(c->src_ptr.begin(), c->src_ptr.end() - 1);
  for (int cell = 0; cell < c->num_cells; ++cell)
    for (int i = c->cell_ptr[cell]; i < c->cell_ptr[cell + 1]; ++i)
      c->src_cell[fill[c->cell_src[i]]++] = cell;
  // Worst-case overhead (Section III-B): the tallest n - e columns, i.e.
  // the tallest set of columns that still has to decode.
  std::vector<int32_t> hs(c->heights);
  std::sort(hs.begin(), hs.end(), [](int a, int b) { return a > b; });
  long long tot = 0;
  for (int j = 0; j < c->n - c->e; ++j) tot += hs[j];
  c->eps = static_cast<double>(tot) / (static_cast<double>(c->k) * c->b) - 1.0;
  build_terms_2d(c);
}

}  // namespace bpx

namespace {

constexpr int kMaxSources = 1 << 24;

struct Builder {
  bpx_code* c;
  std::vector<std::vector<int32_t>> cells;  // support of each cell
  explicit Builder(bpx_code* code) : c(code) {}

  void begin_column(int height, int p, int q) {
    c->col_ptr.push_back(static_cast<int32_t>(cells.size()));
    c->heights.push_back(height);
    c->proj_p.push_back(p);
    c->proj_q.push_back(q);
  }

  void add_cell(std::vector<int32_t> supp) {
    std::sort(supp.begin(), supp.end());
    c->col_of_cell.push_back(static_cast<int32_t>(c->col_ptr.size()) - 1);
    cells.push_back(std::move(supp));
  }

  // One projection (p, q) of the k x b grid as a code column.  Pixel (z, l)
  // is source z k + l; its bin label is
  //   (b-1) q u(q) + (k-1) p u(p) - z q - l p,  u(t) = [t > 0],
  // which Eq. (moj1) keeps inside [0, b_i) with b_i = |p|(k-1) + |q|(b-1) + 1.
  // Bins are emitted in ascending label order; empty bins are skipped.
  void projection(int k, int b, int p, int q) {
    const long long height = static_cast<long long>(std::abs(p)) * (k - 1) +
                             static_cast<long long>(std::abs(q)) * (b - 1) + 1;
    const long long offset = static_cast<long long>(b - 1) * q * (q > 0 ? 1 : 0) +
                             static_cast<long long>(k - 1) * p * (p > 0 ? 1 : 0);
    begin_column(static_cast<int>(height), p, q);
    std::vector<std::vector<int32_t>> bins(static_cast<size_t>(height));
    for (int z = 0; z < b; ++z)
      for (int l = 0; l < k; ++l) {
        const long long label = offset - static_cast<long long>(z) * q - static_cast<long long>(l) * p;
        bins[static_cast<size_t>(label)].push_back(z * k + l);
      }
    for (auto& bin : bins)
      if (!bin.empty()) add_cell(std::move(bin));
  }

  // A systematic data column: column l of the grid, one degree-one cell per
  // pixel (z, l), z ascending.
  void data_column(int k, int b, int l) {
    begin_column(b, 0, 0);
    for (int z = 0; z < b; ++z) add_cell({z * k + l});
  }

  // A literal column, sources given as the paper's 1-based v indices.
  void literal_column(int height, std::initializer_list<std::initializer_list<int>> col) {
    begin_column(height, 0, 0);
    for (auto& cell : col) {
      std::vector<int32_t> s;
      for (int v : cell) s.push_back(v - 1);
      add_cell(std::move(s));
    }
  }

  // X-code column i of n = p columns (k = p - 2 rows of data): the k sources
  // of grid row i as degree-one cells, then the parities along the two
  // diagonals, data row r of column (i + r + 2) mod p and of (i - r - 2) mod p.
  void xcode_column(int p, int i) {
    const int k = p - 2;
    begin_column(p, 0, 0);
    for (int r = 0; r < k; ++r) add_cell({i * k + r});
    std::vector<int32_t> up, down;
    for (int r = 0; r < k; ++r) {
      up.push_back(((i + r + 2) % p) * k + r);
      down.push_back((((i - r - 2) % p + p) % p) * k + r);
    }
    add_cell(std::move(up));
    add_cell(std::move(down));
  }

  void finish() {
    c->col_ptr.push_back(static_cast<int32_t>(cells.size()));
    bpx::finish_code(c, cells, c->col_of_cell);
  }
};

int ceil_odd(int x) { return (x % 2 != 0) ? x : x + 1; }

}  // namespace

extern "C" int bpx_code_build(int variant, int n, int k, int e, int b, int q_e, bpx_code** out) {
  bpx::clear_error();
  if (!out) return fail(BPX_ERR_INVAL, "bpx_code_build: out is NULL");
  *out = nullptr;
  if (n < 1 || k < 1 || b < 1) return fail(BPX_ERR_INVAL, "bpx_code_build: n, k, b must be >= 1");
  if (static_cast<long long>(k) * b > kMaxSources)
    return fail(BPX_ERR_INVAL, "bpx_code_build: k*b = %lld sources exceeds 2^24", 1LL * k * b);
  bpx_code* c = new (std::nothrow) bpx_code();
  if (!c) return fail(BPX_ERR_NOMEM, "bpx_code_build: out of host memory");
  c->variant = variant;
  c->n = n;
  c->k = k;
  c->b = b;
  c->q_e = q_e;
  c->S = k * b;
  Builder B(c);
  int derived_e = -1;
  switch (variant) {
    case BPX_TABLE1:
      // Table I, [5,2,2,2], sigma = 2 (Example 1).  Decodes from any two of
      // its five columns, so it tolerates e = 3 column erasures.
      if (n != 5 || k != 2 || b != 2) {
        delete c;
        return fail(BPX_ERR_INVAL, "Table I code has (n,k,b) = (5,2,2)");
      }
      B.literal_column(2, {{1}, {2, 3}});
      B.literal_column(2, {{2}, {1, 4}});
      B.literal_column(2, {{3}, {2, 4}});
      B.literal_column(2, {{4}, {1, 3}});
      B.literal_column(2, {{1, 2}, {3, 4}});
      derived_e = 3;
      break;
    case BPX_TABLE3:
      // Table III, [5,3,2,3], sigma = 2 (Example 2): block MDS, e = 2.
      if (n != 5 || k != 3 || b != 3) {
        delete c;
        return fail(BPX_ERR_INVAL, "Table III code has (n,k,b) = (5,3,3)");
      }
      B.literal_column(3, {{1}, {3, 4}, {6, 7}});
      B.literal_column(3, {{1, 2}, {4, 5}, {7, 8}});
      B.literal_column(3, {{2, 3}, {5, 6}, {8, 9}});
      B.literal_column(3, {{7}, {9, 1}, {4, 8}});
      B.literal_column(3, {{3}, {2, 6}, {9, 5}});
      derived_e = 2;
      break;
    case BPX_SYSTEMATIC: {
      if (n <= k) {
        delete c;
        return fail(BPX_ERR_INVAL, "systematic code needs n > k (n = k + e)");
      }
      for (int l = 0; l < k; ++l) B.data_column(k, b, l);
      // parities q = 1, slopes 0, +1, -1, +2, -2, ...
      for (int i = 0; i < n - k; ++i) {
        const int m = (i + 1) / 2;
        const int p = (i == 0) ? 0 : ((i % 2 == 1) ? m : -m);
        B.projection(k, b, p, 1);
      }
      derived_e = n - k;
      break;
    }
    case BPX_MOJETTE_A: {
      // Construction A: q = 1, p = -floor((n-1)/2) .. ceil((n-1)/2).
      if (n < k) {
        delete c;
        return fail(BPX_ERR_INVAL, "Construction A needs n >= k");
      }
      const int lo = -((n - 1) / 2);
      for (int i = 0; i < n; ++i) B.projection(k, b, lo + i, 1);
      derived_e = n - k;
      break;
    }
    case BPX_MOJETTE_B: {
      // Construction B: q = 2^q_e, p = the n consecutive odd integers from
      // ceil_odd(1 - n) (the smallest odd integer >= 1 - n).
      if (q_e < 1 || q_e > 20) {
        delete c;
        return fail(BPX_ERR_INVAL, "Construction B needs 1 <= q_e <= 20");
      }
      const int q = 1 << q_e;
      const int need = (k + q - 1) / q;
      if (n < need) {
        delete c;
        return fail(BPX_ERR_INVAL, "Construction B needs n >= ceil(k / 2^q_e) = %d", need);
      }
      const int lo = ceil_odd(1 - n);
      for (int i = 0; i < n; ++i) B.projection(k, b, lo + 2 * i, q);
      derived_e = n - need;
      break;
    }
    case BPX_XCODE: {
      bool prime = n >= 3;
      for (int d = 2; prime && d * d <= n; ++d) prime = n % d != 0;
      if (!prime || k != n - 2 || b != n) {
        delete c;
        return fail(BPX_ERR_INVAL, "X-code needs n = p prime >= 3, k = p - 2, b = p");
      }
      for (int i = 0; i < n; ++i) B.xcode_column(n, i);
      derived_e = 2;
      break;
    }
    default:
      delete c;
      return fail(BPX_ERR_INVAL, "bpx_code_build: unknown variant %d", variant);
  }
  if (e >= 0 && e != derived_e) {
    delete c;
    return fail(BPX_ERR_INVAL, "bpx_code_build: e = %d but this code tolerates %d erasures", e, derived_e);
  }
  c->e = derived_e;
  B.finish();
  *out = c;
  return BPX_OK;
}

extern "C" int bpx_code_info_get(const bpx_code* c, bpx_code_info* out) {
  if (!c || !out) return fail(BPX_ERR_INVAL, "bpx_code_info_get: NULL argument");
  out->variant = c->variant;
  out->n = c->n;
  out->k = c->k;
  out->e = c->e;
  out->b = c->b;
  out->q_e = c->q_e;
  out->num_sources = c->S;
  out->num_cells = c->num_cells;
  out->num_edges = c->num_edges;
  out->sigma = c->sigma;
  out->eps = c->eps;
  out->col_ptr = c->col_ptr.data();
  out->cell_ptr = c->cell_ptr.data();
  out->cell_src = c->cell_src.data();
  out->col_of_cell = c->col_of_cell.data();
  out->heights = c->heights.data();
  out->proj_p = c->proj_p.data();
  out->proj_q = c->proj_q.data();
  return BPX_OK;
}

extern "C" void bpx_code_free(bpx_code* c) { delete c; }

extern "C" const char* bpx_last_error(void) { return bpx::g_last_error.c_str(); }

extern "C" bpx_opts bpx_default_opts(void) {
  bpx_opts o;
  o.direct_write = 1;
  o.compensate_depth = -1;
  o.peel_ctas = 0;
  o.gemm_config = 0;
  o.stage_events = nullptr;
  o.mask_cells = 0;
  o.fused_encode = 0;
  return o;
}

namespace bpx {

int exact_params(const bpx_code* c, int K, ExactParams* P) {
  if (!c || !P) return fail(BPX_ERR_INVAL, "exact_params: NULL argument");
  if (K <= 0 || K % 8 != 0) return fail(BPX_ERR_INVAL, "exact-slice: K = %d must be a positive multiple of 8", K);
  const int sigma = std::max(1, c->sigma);
  int lg = 0;
  while ((1 << lg) < sigma) ++lg;  // ceil(log2 sigma)
  const int w = std::min(8, 9 - lg);
  if (w < 3)
    return fail(BPX_ERR_UNSUPPORTED, "exact-slice: cell degree %d needs digits narrower than 3 bits (at most 64)",
                sigma);
  P->w = w;
  P->S = (24 + w - 1) / w;
  P->bits = std::min(24, w * P->S - 1);
  P->Kp = static_cast<int>(align_up(static_cast<size_t>(K), 64));
  // Largest |coded digit x B digit|; a segment keeps the sum of absolute
  // products below 2^23, so its FP32 accumulation is exact.
  const double maxprod = static_cast<double>(sigma) * std::ldexp(1.0, w - 1) * std::ldexp(1.0, w - 1);
  P->seg = static_cast<int>(std::floor(std::ldexp(1.0, 23) / maxprod / 64.0)) * 64;
  if (P->seg < 64) return fail(BPX_ERR_UNSUPPORTED, "exact-slice: segment below 64");
  // Per-diagonal int32 sums: S pairs x Kp elements at most.
  if (static_cast<double>(P->S) * P->Kp * maxprod >= std::ldexp(1.0, 31))
    return fail(BPX_ERR_UNSUPPORTED, "exact-slice: K = %d too large for exact int32 diagonal sums", K);
  // Q and the peel's partial differences stay exact in int64 and in FP64.
  double q = 0.0;
  for (int d = 0; d < P->S; ++d) q += std::ldexp(1.0, w * (P->S - 1 - d)) * (d + 1) * P->Kp * maxprod;
  if (2.0 * q >= std::ldexp(1.0, 52))
    return fail(BPX_ERR_UNSUPPORTED, "exact-slice: K = %d too large for exact decoded integers", K);
  return BPX_OK;
}

WsLayout ws_layout(const bpx_code* c, int M, int N, int K, int h, int precision, bool twod) {
  (void)M;
  WsLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  const size_t S = static_cast<size_t>(c->S), C = static_cast<size_t>(c->num_cells);
  const size_t E = static_cast<size_t>(c->num_edges);
  const size_t i32 = sizeof(int32_t);
  L.g_hdr = take(HDR_LEN * i32);
  L.g_col_of_cell = take(C * i32);
  L.g_cell_ptr = take((C + 1) * i32);
  L.g_cell_src = take(E * i32);
  L.g_src_ptr = take((S + 1) * i32);
  L.g_src_cell = take(E * i32);
  L.g_t2_ptr = take(c->t2_ptr.size() * i32);
  L.g_t2_a = take(c->t2_a.size() * i32);
  L.g_t2_b = take(c->t2_b.size() * i32);
  L.g_a2_ptr = take(c->a2_ptr.size() * i32);
  L.g_a2_blk = take(c->a2_blk.size() * i32);
  L.g_b2_ptr = take(c->b2_ptr.size() * i32);
  L.g_b2_blk = take(c->b2_blk.size() * i32);
  L.g_t2_order = take(c->t2_order.size() * i32);
  L.p_info = take(BPX_INFO_LEN * i32);
  L.p_ctr = take(CTR_LEN * i32);
  L.p_cnt = take(C * i32);
  L.p_surv = take(C * i32);
  L.p_direct = take(C * i32);
  L.p_front0 = take(C * i32);
  L.p_front1 = take(C * i32);
  L.p_word = take(C * sizeof(unsigned long long));
  L.p_depth = take(S * i32);
  L.p_resolver = take(S * i32);
  L.p_order = take(S * i32);
  L.p_wave_ptr = take((S + 2) * i32);
  L.p_cursor = take((S + 2) * i32);
  L.p_pl_res = take(S * i32);
  L.p_pl_ptr = take((S + 1) * i32);
  L.p_pl_list = take(E * i32);
  L.plan_end = off;
  const size_t hN = static_cast<size_t>(h > 0 ? h : 0) * static_cast<size_t>(N > 0 ? N : 0);
  if (twod) {
    // products: h x w per cell (w = N / k); staging: every A operand (h rows
    // each) and every B operand (w rows of B^T each), bf16 hi (+ lo)
    const size_t w = static_cast<size_t>(N > 0 ? N / c->k : 0), hh = static_cast<size_t>(h > 0 ? h : 0);
    const size_t Kq = static_cast<size_t>(K > 0 ? K : 0);
    const size_t EA = c->a2_ptr.size() - 1, EB = c->b2_ptr.size() - 1;
    L.products = take(C * hh * w * sizeof(float));
    L.a_hi = take(EA * hh * Kq * 2);
    L.b_hi = take(EB * w * Kq * 2);
    L.a_lo = L.b_lo = L.a_scale = L.b_scale = L.ex_amax = L.ex_c64 = off;
    if (precision == BPX_BF16X3) {
      L.a_lo = take(EA * hh * Kq * 2);
      L.b_lo = take(EB * w * Kq * 2);
    }
    L.total = off;
    return L;
  }
  if (precision == BPX_EXACT) {
    // Regions that depend on h and N only come first, so that the exact peel
    // (which does not know K) finds them at the same offsets.
    L.ex_amax = take((static_cast<size_t>(h > 0 ? h : 0) + static_cast<size_t>(N > 0 ? N : 0)) * sizeof(uint32_t));
    L.ex_c64 = take(S * hN * sizeof(int64_t));
  }
  L.products = take(C * hN * sizeof(float));
  const size_t rowsA = C * static_cast<size_t>(h > 0 ? h : 0);
  const size_t Kp = static_cast<size_t>(K > 0 ? K : 0), Np = static_cast<size_t>(N > 0 ? N : 0);
  L.a_hi = L.a_lo = L.b_hi = L.b_lo = L.a_scale = L.b_scale = off;
  if (precision == BPX_FP32) {
    L.a_hi = take(rowsA * Kp * 4);  // FP32 coded rows for the CUDA-core GEMM
  } else if (precision == BPX_BF16 || precision == BPX_BF16X3) {
    L.a_hi = take(rowsA * Kp * 2);
    L.b_hi = take(Np * Kp * 2);
    if (precision == BPX_BF16X3) {
      L.a_lo = take(rowsA * Kp * 2);
      L.b_lo = take(Np * Kp * 2);
    }
  } else if (precision == BPX_FP16X3) {
    // fp16 hi / lo operands, the exponent of every coded row's scale (int32),
    // and per column of B its max |B| (float bits) then its exponent
    L.a_hi = take(rowsA * Kp * 2);
    L.b_hi = take(Np * Kp * 2);
    L.a_lo = take(rowsA * Kp * 2);
    L.b_lo = take(Np * Kp * 2);
    L.a_scale = take(rowsA * sizeof(int32_t));
    L.b_scale = take(2 * Np * sizeof(int32_t));
  } else if (precision == BPX_EXACT) {
    ExactParams P;
    if (exact_params(c, K > 0 ? K : 8, &P) != BPX_OK) {
      clear_error();
      P.S = 1;
      P.Kp = static_cast<int>(align_up(Kp, 64));
    }
    const size_t planes = static_cast<size_t>(P.S), kp = static_cast<size_t>(P.Kp);
    take((planes - 1) * C * hN * sizeof(int32_t));  // products: S int32 planes from L.products on
    L.a_hi = take(rowsA * planes * kp * 2);
    L.b_hi = take(Np * planes * kp * 2);
    // digits of at most 7 bits (S >= 4) fit a byte: for codes whose cells hold
    // four or more sources on average each source row's planes are cut once,
    // then summed per coded row
    if (P.S >= 4 && c->num_edges >= 4LL * c->num_cells)
      L.ex_src = take(S * static_cast<size_t>(h > 0 ? h : 0) * planes * kp);
  } else if (precision == BPX_MXFP8) {
    // E4M3 operands (K-major rows) and UE8M0 scales, one per 32 K-elements,
    // stored per (tile, 128-wide K stage) in the order the GEMM copies them
    // to tensor memory: 512 B per 128-row A tile, 1 KB per 256-column B tile.
    const size_t ks = (Kp + 127) / 128;
    L.a_hi = take(rowsA * Kp);
    L.b_hi = take(Np * Kp);
    L.a_scale = take(((rowsA + 255) / 256) * 2 * ks * 512);  // an even tile count: CTA pairs read whole pairs
    L.b_scale = take(((Np + 255) / 256) * ks * 1024);
  }
  L.total = off;
  return L;
}

}  // namespace bpx

extern "C" int bpx_exact_params(const bpx_code* c, int K, int32_t* out) {
  bpx::clear_error();
  if (!out) return bpx::fail(BPX_ERR_INVAL, "bpx_exact_params: out is NULL");
  bpx::ExactParams P;
  if (int rc = bpx::exact_params(c, K, &P)) return rc;
  out[0] = P.w;
  out[1] = P.S;
  out[2] = P.bits;
  out[3] = P.seg;
  out[4] = P.Kp;
  return BPX_OK;
}

extern "C" size_t bpx_workspace_bytes(const bpx_code* c, int M, int N, int K, int h, int precision) {
  if (!c) return 0;
  return bpx::ws_layout(c, M, N, K, h, precision).total;
}
