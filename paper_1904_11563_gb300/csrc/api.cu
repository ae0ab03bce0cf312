// C-ABI entry points of libbpx: argument checks, workspace views and the
// launch sequence of the hot path.  Every step runs in the kernels of this
// library; the host only validates, binds pointers and launches.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "device_common.cuh"

using bpx::fail;

namespace bpx {

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

int& reserved_sms() {
  thread_local int r = 0;
  return r;
}

}  // namespace bpx

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  return fail(BPX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_ws(const bpx_code* c, const void* ws, size_t ws_bytes, const bpx::WsLayout& L) {
  if (!c) return fail(BPX_ERR_INVAL, "code is NULL");
  if (!ws) return fail(BPX_ERR_INVAL, "workspace is NULL");
  if (!aligned(ws, 256)) return fail(BPX_ERR_INVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < L.total)
    return fail(BPX_ERR_NOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
  return BPX_OK;
}

int check_shapes(const bpx_code* c, int M, int N, int K, int h) {
  if (M < 0 || N <= 0 || K <= 0 || h <= 0)
    return fail(BPX_ERR_INVAL, "need M >= 0 and N, K, h > 0 (M=%d N=%d K=%d h=%d)", M, N, K, h);
  if (N % 4 != 0) return fail(BPX_ERR_INVAL, "N = %d must be a multiple of 4", N);
  if (K % 8 != 0) return fail(BPX_ERR_INVAL, "K = %d must be a multiple of 8", K);
  if (static_cast<long long>(M) > static_cast<long long>(c->S) * h)
    return fail(BPX_ERR_INVAL, "M = %d exceeds S h = %lld rows", M, 1LL * c->S * h);
  if (static_cast<long long>(c->num_cells) * h > (1LL << 31) / 2)
    return fail(BPX_ERR_INVAL, "too many coded rows");
  return BPX_OK;
}

cudaStream_t S(bpx_stream s) { return static_cast<cudaStream_t>(s); }

// Records the caller's timing event for the start (end = 0) or end (end = 1)
// of a stage, when bpx_opts.stage_events asks for it.
void stage_mark(const bpx_opts* o, int stage, int end, cudaStream_t st) {
  if (!o || !o->stage_events) return;
  void* ev = o->stage_events[2 * stage + end];
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev), st);
}

}  // namespace

extern "C" size_t bpx_workspace_info_offset(const bpx_code* c) {
  if (!c) return 0;
  return bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32).p_info;
}

extern "C" int bpx_workspace_init(const bpx_code* c, void* ws, size_t ws_bytes, bpx_stream stream) {
  bpx::clear_error();
  const bpx::WsLayout L = bpx::ws_layout(c ? c : nullptr, 0, 0, 0, 1, BPX_FP32);
  if (!c) return fail(BPX_ERR_INVAL, "bpx_workspace_init: code is NULL");
  if (int rc = check_ws(c, ws, ws_bytes, L)) return rc;
  char* base = static_cast<char*>(ws);
  std::vector<int32_t> hdr(bpx::HDR_LEN, 0);
  hdr[bpx::HDR_MAGIC] = bpx::kWsMagic;
  hdr[bpx::HDR_N] = c->n;
  hdr[bpx::HDR_S] = c->S;
  hdr[bpx::HDR_CELLS] = c->num_cells;
  hdr[bpx::HDR_EDGES] = c->num_edges;
  hdr[bpx::HDR_SIGMA] = c->sigma;
  struct Part {
    size_t off;
    const void* src;
    size_t bytes;
  } parts[] = {
      {L.g_hdr, hdr.data(), hdr.size() * 4},
      {L.g_col_of_cell, c->col_of_cell.data(), c->col_of_cell.size() * 4},
      {L.g_cell_ptr, c->cell_ptr.data(), c->cell_ptr.size() * 4},
      {L.g_cell_src, c->cell_src.data(), c->cell_src.size() * 4},
      {L.g_src_ptr, c->src_ptr.data(), c->src_ptr.size() * 4},
      {L.g_src_cell, c->src_cell.data(), c->src_cell.size() * 4},
      {L.g_t2_ptr, c->t2_ptr.data(), c->t2_ptr.size() * 4},
      {L.g_t2_a, c->t2_a.data(), c->t2_a.size() * 4},
      {L.g_t2_b, c->t2_b.data(), c->t2_b.size() * 4},
      {L.g_a2_ptr, c->a2_ptr.data(), c->a2_ptr.size() * 4},
      {L.g_a2_blk, c->a2_blk.data(), c->a2_blk.size() * 4},
      {L.g_b2_ptr, c->b2_ptr.data(), c->b2_ptr.size() * 4},
      {L.g_b2_blk, c->b2_blk.data(), c->b2_blk.size() * 4},
      {L.g_t2_order, c->t2_order.data(), c->t2_order.size() * 4},
  };
  for (const Part& pt : parts) {
    if (pt.bytes == 0) continue;
    cudaError_t e = cudaMemcpyAsync(base + pt.off, pt.src, pt.bytes, cudaMemcpyHostToDevice, S(stream));
    if (e != cudaSuccess) return cuda_fail(e, "bpx_workspace_init: copy");
  }
  cudaError_t e = cudaMemsetAsync(base + L.p_info, 0, L.plan_end - L.p_info, S(stream));
  if (e != cudaSuccess) return cuda_fail(e, "bpx_workspace_init: memset");
  e = cudaStreamSynchronize(S(stream));
  if (e != cudaSuccess) return cuda_fail(e, "bpx_workspace_init: sync");
  return BPX_OK;
}

namespace {

int schedule_impl(const bpx_code* c, const uint8_t* d_mask, bool cell_mask, void* ws, size_t ws_bytes,
                  int32_t* d_peel_order, uint8_t* d_recovered, int32_t* d_info, cudaStream_t st, int part = 0) {
  if (!c) return fail(BPX_ERR_INVAL, "bpx_schedule: code is NULL");
  const bpx::WsLayout L = bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32);
  if (int rc = check_ws(c, ws, ws_bytes, L)) return rc;
  if (!d_mask) return fail(BPX_ERR_INVAL, "bpx_schedule: erasure mask is NULL");
  const bpx::DevGraph g = bpx::make_graph(c, ws, L);
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  cudaError_t e = bpx::launch_schedule(g, p, d_mask, d_peel_order, d_recovered, d_info, st, cell_mask, part);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_schedule: launch");
  return BPX_OK;
}

// Codes with this many sources plan in hundreds of dependent rounds: the
// rounds after the first then run on a second stream beside the products
// (which need only the survivors and the depth-1 map), and the GEMMs leave
// two SMs free for them.
constexpr int kOverlapSources = 4096;

// The second stream and the fork / join events of the calling thread.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int device = -1;
};

SideStream* side_stream() {
  thread_local SideStream ss;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (ss.s && ss.device == dev) return &ss;
  if (ss.s) {
    cudaStreamDestroy(ss.s);
    cudaEventDestroy(ss.fork);
    cudaEventDestroy(ss.join);
    ss.s = nullptr;
  }
  if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ss.s = nullptr;
    return nullptr;
  }
  ss.device = dev;
  return &ss;
}

struct ReserveGuard {
  explicit ReserveGuard(int n) { bpx::reserved_sms() = n; }
  ~ReserveGuard() { bpx::reserved_sms() = 0; }
};

}  // namespace

extern "C" int bpx_schedule(const bpx_code* c, const uint8_t* d_mask, void* ws, size_t ws_bytes,
                            int32_t* d_peel_order, uint8_t* d_recovered, int32_t* d_info,
                            bpx_stream stream) {
  bpx::clear_error();
  return schedule_impl(c, d_mask, false, ws, ws_bytes, d_peel_order, d_recovered, d_info, S(stream));
}

extern "C" int bpx_schedule_cells(const bpx_code* c, const uint8_t* d_cell_mask, void* ws, size_t ws_bytes,
                                  int32_t* d_peel_order, uint8_t* d_recovered, int32_t* d_info, bpx_stream stream) {
  bpx::clear_error();
  return schedule_impl(c, d_cell_mask, true, ws, ws_bytes, d_peel_order, d_recovered, d_info, S(stream));
}

extern "C" int bpx_encode(const bpx_code* c, const float* d_A, int M, int K, int h,
                          const void* ws, float* d_A_coded, bpx_stream stream) {
  bpx::clear_error();
  // (A may be NULL when M = 0: every source block is then zero padding)
  if (!c || (!d_A && M > 0) || !d_A_coded || !ws) return fail(BPX_ERR_INVAL, "bpx_encode: NULL argument");
  if (int rc = check_shapes(c, M, 4, K, h)) return rc;
  if (!aligned(d_A, 16) || !aligned(d_A_coded, 16))
    return fail(BPX_ERR_INVAL, "bpx_encode: buffers must be 16-byte aligned");
  const bpx::WsLayout L = bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32);
  const bpx::DevGraph g = bpx::make_graph(c, ws, L);
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  cudaError_t e = bpx::launch_encode_f32(g, p, d_A, M, K, h, d_A_coded, S(stream));
  if (e != cudaSuccess) return cuda_fail(e, "bpx_encode: launch");
  return BPX_OK;
}

namespace {

int products_impl(const bpx_code* c, const float* d_A, const float* d_B, int M, int N, int K,
                  int h, int precision, void* ws, size_t ws_bytes, float* d_products, float* d_C,
                  const bpx_opts* opts, int32_t* d_info, cudaStream_t st) {
  if (!c || (!d_A && M > 0) || !d_B || !ws || !d_products)  // A unused when M = 0
    return fail(BPX_ERR_INVAL, "bpx_coded_products: NULL argument");
  if (int rc = check_shapes(c, M, N, K, h)) return rc;
  if (!aligned(d_A, 16) || !aligned(d_B, 16) || !aligned(d_products, 16) ||
      (d_C && !aligned(d_C, 16)))
    return fail(BPX_ERR_INVAL, "bpx_coded_products: buffers must be 16-byte aligned");
  const bpx::WsLayout L = bpx::ws_layout(c, M, N, K, h, precision);
  if (int rc = check_ws(c, ws, ws_bytes, L)) return rc;
  const bpx::DevGraph g = bpx::make_graph(c, ws, L);
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  char* base = static_cast<char*>(ws);
  const int config = opts ? opts->gemm_config : 0;
  if (!bpx::gemm_config_ok(config)) return fail(BPX_ERR_INVAL, "bpx_coded_products: gemm_config %d names no tile", config);
  const bool fused = opts && opts->fused_encode;
  if (fused && precision != BPX_BF16 && precision != BPX_BF16X3)
    return fail(BPX_ERR_UNSUPPORTED, "bpx_coded_products: the fused encode is built for BPX_BF16 and BPX_BF16X3");
  if (fused && c->sigma > 8)
    return fail(BPX_ERR_UNSUPPORTED, "bpx_coded_products: the fused encode takes cells of at most 8 sources "
                "(sigma = %d)", c->sigma);
  if (fused && config != 0 && config % 10 != 0)
    return fail(BPX_ERR_INVAL, "bpx_coded_products: the fused encode needs gemm_config 0 or tile code 0 (got %d)",
                config);
  cudaError_t e = cudaSuccess;
  switch (precision) {
    case BPX_FP32: {
      float* a_coded = reinterpret_cast<float*>(base + L.a_hi);
      stage_mark(opts, BPX_STAGE_A_PREP, 0, st);
      e = bpx::launch_encode_f32(g, p, d_A, M, K, h, a_coded, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_GEMM, 0, st);
      if (e == cudaSuccess) e = bpx::launch_gemm_f32(g, p, a_coded, d_B, N, K, h, d_products, d_C, st);
      stage_mark(opts, BPX_STAGE_GEMM, 1, st);
      break;
    }
    case BPX_BF16:
    case BPX_BF16X3: {
      const bool split = precision == BPX_BF16X3;
      void* a_hi = base + L.a_hi;
      void* a_lo = split ? base + L.a_lo : nullptr;
      void* b_hi = base + L.b_hi;
      void* b_lo = split ? base + L.b_lo : nullptr;
      stage_mark(opts, BPX_STAGE_B_PREP, 0, st);
      e = bpx::launch_b_split(d_B, K, N, b_hi, b_lo, st);
      stage_mark(opts, BPX_STAGE_B_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 0, st);
      if (e == cudaSuccess && !fused) e = bpx::launch_encode_split(g, p, d_A, M, K, h, a_hi, a_lo, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_GEMM, 0, st);
      if (e == cudaSuccess && fused)
        e = bpx::launch_gemm_fused(g, p, d_A, M, b_hi, b_lo, c->num_cells, N, K, h, split, d_products, d_C, config,
                                   d_info, st);
      else if (e == cudaSuccess)
        e = bpx::launch_gemm_tc(g, p, a_hi, a_lo, b_hi, b_lo, c->num_cells, N, K, h, split,
                                d_products, d_C, config, d_info, st);
      stage_mark(opts, BPX_STAGE_GEMM, 1, st);
      if (e == cudaErrorNotSupported)
        return fail(BPX_ERR_UNSUPPORTED, "bf16 tensor-core path not available in this build");
      break;
    }
    case BPX_FP16X3: {
      void* a_hi = base + L.a_hi;
      void* a_lo = base + L.a_lo;
      void* b_hi = base + L.b_hi;
      void* b_lo = base + L.b_lo;
      int32_t* a_exp = reinterpret_cast<int32_t*>(base + L.a_scale);
      uint32_t* b_max = reinterpret_cast<uint32_t*>(base + L.b_scale);
      int32_t* b_exp = reinterpret_cast<int32_t*>(b_max + N);
      stage_mark(opts, BPX_STAGE_B_PREP, 0, st);
      e = bpx::launch_b_f16(d_B, K, N, b_hi, b_lo, b_max, b_exp, st);
      stage_mark(opts, BPX_STAGE_B_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 0, st);
      if (e == cudaSuccess) e = bpx::launch_encode_f16(g, p, d_A, M, K, h, a_hi, a_lo, a_exp, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_GEMM, 0, st);
      if (e == cudaSuccess)
        e = bpx::launch_gemm_tc(g, p, a_hi, a_lo, b_hi, b_lo, c->num_cells, N, K, h, true, d_products, d_C, config,
                                d_info, st, a_exp, b_exp);
      stage_mark(opts, BPX_STAGE_GEMM, 1, st);
      break;
    }
    case BPX_MXFP8: {
      if (K % 128 != 0) return fail(BPX_ERR_INVAL, "BPX_MXFP8 needs K %% 128 == 0 (K = %d)", K);
      void* a8 = base + L.a_hi;
      void* b8 = base + L.b_hi;
      void* sfa = base + L.a_scale;
      void* sfb = base + L.b_scale;
      stage_mark(opts, BPX_STAGE_B_PREP, 0, st);
      e = bpx::launch_b_mx(d_B, K, N, b8, sfb, st);
      stage_mark(opts, BPX_STAGE_B_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 0, st);
      if (e == cudaSuccess) e = bpx::launch_encode_mx(g, p, d_A, M, K, h, a8, sfa, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_GEMM, 0, st);
      if (e == cudaSuccess)
        e = bpx::launch_gemm_mx(p, a8, sfa, b8, sfb, c->num_cells, N, K, h, d_products, d_C, config, d_info, st);
      stage_mark(opts, BPX_STAGE_GEMM, 1, st);
      break;
    }
    case BPX_EXACT: {
      bpx::ExactParams P;
      if (int rc = bpx::exact_params(c, K, &P)) return rc;
      uint32_t* amax = reinterpret_cast<uint32_t*>(base + L.ex_amax);  // h words (A), then N (B)
      void* a_pl = base + L.a_hi;
      void* b_pl = base + L.b_hi;
      stage_mark(opts, BPX_STAGE_B_PREP, 0, st);
      e = bpx::launch_exact_b(d_B, K, N, P, amax + h, b_pl, st);
      stage_mark(opts, BPX_STAGE_B_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_A_PREP, 0, st);
      if (e == cudaSuccess)
        e = bpx::launch_exact_a(g, p, d_A, M, K, h, P, amax, a_pl, st, L.ex_src ? base + L.ex_src : nullptr);
      stage_mark(opts, BPX_STAGE_A_PREP, 1, st);
      stage_mark(opts, BPX_STAGE_GEMM, 0, st);
      if (e == cudaSuccess)
        e = bpx::launch_gemm_exact(p, a_pl, b_pl, c->num_cells, N, K, h, P, reinterpret_cast<int32_t*>(d_products),
                                   config, d_info, st);
      stage_mark(opts, BPX_STAGE_GEMM, 1, st);
      break;
    }
    default:
      return fail(BPX_ERR_UNSUPPORTED, "precision %d not supported", precision);
  }
  if (e != cudaSuccess) return cuda_fail(e, "bpx_coded_products: launch");
  return BPX_OK;
}

int peel_exact_impl(const bpx_code* c, const int32_t* d_planes, int N, int h, float* d_C, const bpx_opts* opts,
                    void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!c || !d_planes || !d_C || !ws) return fail(BPX_ERR_INVAL, "bpx_peel_decode_exact: NULL argument");
  if (N <= 0 || h <= 0 || N % 4 != 0) return fail(BPX_ERR_INVAL, "bpx_peel_decode_exact: bad N or h");
  if (!aligned(d_planes, 16) || !aligned(d_C, 16))
    return fail(BPX_ERR_INVAL, "bpx_peel_decode_exact: buffers must be 16-byte aligned");
  bpx::ExactParams P;
  if (int rc = bpx::exact_params(c, 8, &P)) return rc;  // w, S and bits depend on sigma only
  // The scales and the int64 blocks sit before every K-dependent region.
  const bpx::WsLayout L = bpx::ws_layout(c, 0, N, 8, h, BPX_EXACT);
  if (int rc = check_ws(c, ws, ws_bytes, L)) return rc;
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  char* base = static_cast<char*>(ws);
  const uint32_t* amax = reinterpret_cast<const uint32_t*>(base + L.ex_amax);
  long long* c64 = reinterpret_cast<long long*>(base + L.ex_c64);
  const int ctas = opts ? opts->peel_ctas : 0;
  stage_mark(opts, BPX_STAGE_PEEL, 0, st);
  cudaError_t e = bpx::launch_peel_exact(p, P, d_planes, static_cast<long long>(c->num_cells) * h * N, c64, d_C,
                                         amax, amax + h, N, h, ctas, st);
  stage_mark(opts, BPX_STAGE_PEEL, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_peel_decode_exact: launch");
  return BPX_OK;
}

int peel_impl(const bpx_code* c, const float* d_products, int N, int h, float* d_C,
              int direct_written, const bpx_opts* opts, const void* ws, cudaStream_t st) {
  if (!c || !d_products || !d_C || !ws) return fail(BPX_ERR_INVAL, "bpx_peel_decode: NULL argument");
  if (N <= 0 || h <= 0 || N % 4 != 0) return fail(BPX_ERR_INVAL, "bpx_peel_decode: bad N or h");
  if (!aligned(d_products, 16) || !aligned(d_C, 16))
    return fail(BPX_ERR_INVAL, "bpx_peel_decode: buffers must be 16-byte aligned");
  const bpx::WsLayout L = bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32);
  const bpx::DevGraph g = bpx::make_graph(c, ws, L);
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  const int comp = opts ? opts->compensate_depth : -1;
  const int ctas = opts ? opts->peel_ctas : 0;
  stage_mark(opts, BPX_STAGE_PEEL, 0, st);
  cudaError_t e = bpx::launch_peel(g, p, d_products, d_C, N, h, direct_written ? 2 : 1, comp, ctas, st);
  stage_mark(opts, BPX_STAGE_PEEL, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_peel_decode: launch");
  return BPX_OK;
}

}  // namespace

extern "C" int bpx_coded_products(const bpx_code* c, const float* d_A, const float* d_B, int M,
                                  int N, int K, int h, int precision, void* ws, size_t ws_bytes,
                                  float* d_products, float* d_C, const bpx_opts* opts,
                                  bpx_stream stream) {
  bpx::clear_error();
  return products_impl(c, d_A, d_B, M, N, K, h, precision, ws, ws_bytes, d_products, d_C, opts,
                       nullptr, S(stream));
}

extern "C" int bpx_peel_decode(const bpx_code* c, const float* d_products, const uint8_t* d_erasure_mask, int N,
                               int h, float* d_C, int direct_written, const bpx_opts* opts, void* ws,
                               size_t ws_bytes, int32_t* d_info, bpx_stream stream) {
  bpx::clear_error();
  if (!c || !ws) return fail(BPX_ERR_INVAL, "bpx_peel_decode: NULL argument");
  if (int rc = check_ws(c, ws, ws_bytes, bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32))) return rc;
  if (d_erasure_mask)  // plan the peel for this mask first
    if (int rc = schedule_impl(c, d_erasure_mask, opts && opts->mask_cells, ws, ws_bytes, nullptr, nullptr, d_info,
                               S(stream)))
      return rc;
  return peel_impl(c, d_products, N, h, d_C, direct_written, opts, ws, S(stream));
}

extern "C" int bpx_peel_decode_exact(const bpx_code* c, const int32_t* d_planes, const uint8_t* d_erasure_mask,
                                     int N, int h, float* d_C, const bpx_opts* opts, void* d_ws, size_t ws_bytes,
                                     int32_t* d_info, bpx_stream stream) {
  bpx::clear_error();
  if (!c || !d_ws) return fail(BPX_ERR_INVAL, "bpx_peel_decode_exact: NULL argument");
  if (int rc = check_ws(c, d_ws, ws_bytes, bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32))) return rc;
  if (d_erasure_mask)
    if (int rc = schedule_impl(c, d_erasure_mask, opts && opts->mask_cells, d_ws, ws_bytes, nullptr, nullptr,
                               d_info, S(stream)))
      return rc;
  return peel_exact_impl(c, d_planes, N, h, d_C, opts, d_ws, ws_bytes, S(stream));
}

// ---- two-dimensional scheme ------------------------------------------------

extern "C" int bpx_terms_2d(const bpx_code* c, int32_t* terms_per_cell, int32_t* summary) {
  bpx::clear_error();
  if (!c) return fail(BPX_ERR_INVAL, "bpx_terms_2d: code is NULL");
  if (terms_per_cell)
    for (int i = 0; i < c->num_cells; ++i) terms_per_cell[i] = c->t2_ptr[i + 1] - c->t2_ptr[i];
  if (summary) {
    summary[0] = static_cast<int32_t>(c->t2_a.size());
    summary[1] = c->gray2;
    summary[2] = static_cast<int32_t>(c->a2_ptr.size()) - 1;
    summary[3] = static_cast<int32_t>(c->b2_ptr.size()) - 1;
  }
  return BPX_OK;
}

extern "C" size_t bpx_workspace_bytes_2d(const bpx_code* c, int M, int N, int K, int h, int precision) {
  if (!c) return 0;
  return bpx::ws_layout(c, M, N, K, h, precision, true).total;
}

extern "C" int bpx_coded_matmul_2d(const bpx_code* c, const float* d_A, const float* d_B, int M, int N, int K, int h,
                                   int precision, const uint8_t* d_mask, float* d_C, const bpx_opts* opts, void* ws,
                                   size_t ws_bytes, int32_t* d_info, bpx_stream stream) {
  bpx::clear_error();
  if (!c || !d_A || !d_B || !d_mask || !d_C || !ws) return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: NULL argument");
  if (M < 0 || N <= 0 || K <= 0 || h <= 0) return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: bad shape");
  if (N % c->k != 0) return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: N = %d must be k w (k = %d)", N, c->k);
  const int w = N / c->k;
  if (w % 4 != 0) return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: block width w = N / k = %d must be a multiple of 4", w);
  if (K % 8 != 0) return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: K = %d must be a multiple of 8", K);
  if (static_cast<long long>(M) > static_cast<long long>(c->b) * h)
    return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: M = %d exceeds b h = %lld rows", M, 1LL * c->b * h);
  if (precision != BPX_BF16 && precision != BPX_BF16X3)
    return fail(BPX_ERR_UNSUPPORTED, "bpx_coded_matmul_2d: precision BPX_BF16 or BPX_BF16X3");
  if (!aligned(d_A, 16) || !aligned(d_B, 16) || !aligned(d_C, 16))
    return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: buffers must be 16-byte aligned");
  const bpx::WsLayout L = bpx::ws_layout(c, M, N, K, h, precision, true);
  if (int rc = check_ws(c, ws, ws_bytes, L)) return rc;
  const bpx_opts o = opts ? *opts : bpx_default_opts();
  if (!bpx::gemm_config_ok(o.gemm_config))
    return fail(BPX_ERR_INVAL, "bpx_coded_matmul_2d: gemm_config %d names no tile", o.gemm_config);
  cudaStream_t st = S(stream);
  stage_mark(&o, BPX_STAGE_SCHEDULE, 0, st);
  if (int rc = schedule_impl(c, d_mask, o.mask_cells != 0, ws, ws_bytes, nullptr, nullptr, d_info, st)) return rc;
  stage_mark(&o, BPX_STAGE_SCHEDULE, 1, st);
  const bpx::DevGraph g = bpx::make_graph(c, ws, L);
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  char* base = static_cast<char*>(ws);
  const bool split = precision == BPX_BF16X3;
  void* a_hi = base + L.a_hi;
  void* a_lo = split ? base + L.a_lo : nullptr;
  void* b_hi = base + L.b_hi;
  void* b_lo = split ? base + L.b_lo : nullptr;
  float* products = reinterpret_cast<float*>(base + L.products);
  stage_mark(&o, BPX_STAGE_A_PREP, 0, st);
  cudaError_t e = bpx::launch_stage_2d(g, d_A, d_B, M, N, K, h, w, a_hi, a_lo, b_hi, b_lo, st);
  stage_mark(&o, BPX_STAGE_A_PREP, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_coded_matmul_2d: staging");
  stage_mark(&o, BPX_STAGE_GEMM, 0, st);
  e = bpx::launch_gemm_2d(g, p, a_hi, a_lo, b_hi, b_lo, N, K, h, w, split, products, o.direct_write ? d_C : nullptr,
                          o.gemm_config, d_info, st);
  stage_mark(&o, BPX_STAGE_GEMM, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_coded_matmul_2d: GEMM");
  stage_mark(&o, BPX_STAGE_PEEL, 0, st);
  e = bpx::launch_peel_2d(g, p, products, d_C, N, h, w, o.direct_write ? 2 : 1, o.peel_ctas, st);
  stage_mark(&o, BPX_STAGE_PEEL, 1, st);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_coded_matmul_2d: peel");
  return BPX_OK;
}

extern "C" int bpx_coded_matmul(const bpx_code* c, const float* d_A, const float* d_B, int M, int N,
                                int K, int h, int precision, const uint8_t* d_mask, float* d_C,
                                const bpx_opts* opts, void* ws, size_t ws_bytes, int32_t* d_info,
                                bpx_stream stream) {
  bpx::clear_error();
  if (!c) return fail(BPX_ERR_INVAL, "bpx_coded_matmul: code is NULL");
  if (!d_C) return fail(BPX_ERR_INVAL, "bpx_coded_matmul: C is NULL");
  const bpx_opts o = opts ? *opts : bpx_default_opts();
  if (!bpx::gemm_config_ok(o.gemm_config))
    return fail(BPX_ERR_INVAL, "bpx_coded_matmul: gemm_config %d names no tile", o.gemm_config);
  const bpx::WsLayout L = bpx::ws_layout(c, M, N, K, h, precision);
  if (int rc = check_ws(c, ws, ws_bytes, L)) return rc;
  SideStream* side = c->S >= kOverlapSources ? side_stream() : nullptr;
  stage_mark(&o, BPX_STAGE_SCHEDULE, 0, S(stream));
  if (!side) {
    if (int rc = schedule_impl(c, d_mask, o.mask_cells != 0, ws, ws_bytes, nullptr, nullptr, d_info, S(stream)))
      return rc;
    stage_mark(&o, BPX_STAGE_SCHEDULE, 1, S(stream));
  } else {
    // survivors + depth-1 map now; the remaining rounds beside the products
    if (int rc = schedule_impl(c, d_mask, o.mask_cells != 0, ws, ws_bytes, nullptr, nullptr, d_info, S(stream), 1))
      return rc;
    cudaError_t e = cudaEventRecord(side->fork, S(stream));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side->s, side->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "bpx_coded_matmul: fork");
    if (int rc = schedule_impl(c, d_mask, o.mask_cells != 0, ws, ws_bytes, nullptr, nullptr, d_info, side->s, 2))
      return rc;
    stage_mark(&o, BPX_STAGE_SCHEDULE, 1, side->s);
    if ((e = cudaEventRecord(side->join, side->s)) != cudaSuccess) return cuda_fail(e, "bpx_coded_matmul: join");
  }
  float* products = reinterpret_cast<float*>(static_cast<char*>(ws) + L.products);
  ReserveGuard reserve(side ? 2 : 0);
  auto join = [&]() -> int {
    if (!side) return BPX_OK;
    const cudaError_t e = cudaStreamWaitEvent(S(stream), side->join, 0);
    return e == cudaSuccess ? BPX_OK : cuda_fail(e, "bpx_coded_matmul: join");
  };
  if (precision == BPX_EXACT) {
    if (int rc = products_impl(c, d_A, d_B, M, N, K, h, precision, ws, ws_bytes, products, nullptr, &o, d_info,
                               S(stream)))
      return rc;
    if (int rc = join()) return rc;
    return peel_exact_impl(c, reinterpret_cast<const int32_t*>(products), N, h, d_C, &o, ws, ws_bytes, S(stream));
  }
  if (int rc = products_impl(c, d_A, d_B, M, N, K, h, precision, ws, ws_bytes, products,
                             o.direct_write ? d_C : nullptr, &o, d_info, S(stream)))
    return rc;
  if (int rc = join()) return rc;
  return peel_impl(c, products, N, h, d_C, o.direct_write, &o, ws, S(stream));
}

namespace {

// Copies in, the whole path, copies out; synchronizes at the end when `sync`.
int host_impl(const bpx_code* c, const float* h_A, const float* h_B, int M, int N, int K, int h, int precision,
              const uint8_t* h_mask, float* h_C, float* d_A, float* d_B, uint8_t* d_mask, float* d_C,
              const bpx_opts* opts, void* ws, size_t ws_bytes, int32_t* h_info, cudaStream_t st, bool sync) {
  if (!c || !h_A || !h_B || !h_mask || !h_C || !d_A || !d_B || !d_mask || !d_C || !h_info)
    return fail(BPX_ERR_INVAL, "bpx_coded_matmul_host: NULL argument");
  if (int rc = check_shapes(c, M, N, K, h)) return rc;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_A, h_A, sizeof(float) * M * static_cast<size_t>(K),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "copy A");
  if ((e = cudaMemcpyAsync(d_B, h_B, sizeof(float) * K * static_cast<size_t>(N),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "copy B");
  const size_t mask_bytes = (opts && opts->mask_cells) ? static_cast<size_t>(c->num_cells) : static_cast<size_t>(c->n);
  if ((e = cudaMemcpyAsync(d_mask, h_mask, mask_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "copy mask");
  const bpx::WsLayout L = bpx::ws_layout(c, M, N, K, h, precision);
  int32_t* d_info = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + L.p_info);
  if (int rc = bpx_coded_matmul(c, d_A, d_B, M, N, K, h, precision, d_mask, d_C, opts, ws, ws_bytes,
                                nullptr, st))
    return rc;
  if ((e = cudaMemcpyAsync(h_C, d_C, sizeof(float) * M * static_cast<size_t>(N),
                           cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy C");
  if ((e = cudaMemcpyAsync(h_info, d_info, sizeof(int32_t) * BPX_INFO_LEN, cudaMemcpyDeviceToHost,
                           st)) != cudaSuccess)
    return cuda_fail(e, "copy info");
  if (!sync) return BPX_OK;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  if (h_info[BPX_INFO_DEVICE_ERR] != 0) return h_info[BPX_INFO_DEVICE_ERR];
  return h_info[BPX_INFO_STATUS];
}

}  // namespace

extern "C" int bpx_coded_matmul_host(const bpx_code* c, const float* h_A, const float* h_B, int M,
                                     int N, int K, int h, int precision, const uint8_t* h_mask,
                                     float* h_C, float* d_A, float* d_B, uint8_t* d_mask,
                                     float* d_C, const bpx_opts* opts, void* ws, size_t ws_bytes,
                                     int32_t* h_info, bpx_stream stream) {
  bpx::clear_error();
  return host_impl(c, h_A, h_B, M, N, K, h, precision, h_mask, h_C, d_A, d_B, d_mask, d_C, opts, ws, ws_bytes,
                   h_info, S(stream), true);
}

extern "C" int bpx_coded_matmul_host_async(const bpx_code* c, const float* h_A, const float* h_B, int M, int N,
                                           int K, int h, int precision, const uint8_t* h_mask, float* h_C,
                                           float* d_A, float* d_B, uint8_t* d_mask, float* d_C,
                                           const bpx_opts* opts, void* ws, size_t ws_bytes, int32_t* h_info,
                                           bpx_stream stream) {
  bpx::clear_error();
  return host_impl(c, h_A, h_B, M, N, K, h, precision, h_mask, h_C, d_A, d_B, d_mask, d_C, opts, ws, ws_bytes,
                   h_info, S(stream), false);
}

extern "C" const char* bpx_build_info(void) {
  return "libbpx 0.2 (sm_103a; tcgen05/TMA tensor-core paths incl. exact slices, FP32 SIMT path)";
}
