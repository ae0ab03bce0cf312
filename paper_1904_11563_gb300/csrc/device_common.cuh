// Device-side views of the workspace and helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bpx_internal.h"

namespace bpx {

// Code graph as uploaded into the workspace (CSR, int32).
struct DevGraph {
  const int32_t* col_of_cell;
  const int32_t* cell_ptr;
  const int32_t* cell_src;
  const int32_t* src_ptr;
  const int32_t* src_cell;
  // two-dimensional scheme: cell terms, operand block lists, cell order
  const int32_t* t2_ptr;
  const int32_t* t2_a;
  const int32_t* t2_b;
  const int32_t* a2_ptr;
  const int32_t* a2_blk;
  const int32_t* b2_ptr;
  const int32_t* b2_blk;
  const int32_t* t2_order;
  int n, S, num_cells, num_edges, sigma;
  int k, EA, EB;  // grid width (B blocks), A and B operand counts
};

// Peel plan written by the schedule kernel.
struct DevPlan {
  int32_t* info;      // BPX_INFO_LEN
  int32_t* ctr;       // CTR_LEN counters
  int32_t* cnt;       // sources per surviving cell (-1: erased column)
  int32_t* surv;      // surviving cells, ascending
  int32_t* direct;    // per cell: the source it resolves at depth 1, or -1
  int32_t* front0;    // frontier scratch
  int32_t* front1;
  unsigned long long* word;  // per cell: unknown count << 32 | XOR of unknown ids + 1 (large codes)
  int32_t* depth;     // per source: round of recovery (0 = not recovered)
  int32_t* resolver;  // per source: resolving cell (INT32_MAX = none)
  int32_t* order;     // recovered sources sorted by (depth, source)
  int32_t* wave_ptr;  // order[wave_ptr[d-1] .. wave_ptr[d]) = sources of depth d
  int32_t* cursor;    // placement cursors (scratch)
  // Peel list, one entry per position i of `order`: the resolver of order[i]
  // and, in pl_list[pl_ptr[i] .. pl_ptr[i+1]), the other sources of that
  // resolver in ascending id (the blocks subtracted from its product).
  int32_t* pl_res;
  int32_t* pl_ptr;
  int32_t* pl_list;
};

// The schedule's per-cell word holds the cell's unknown-source count above
// the XOR of its unknown sources' ids + 1 (values 1 .. S).  sched_id_bits:
// the bits of S; a 32-bit word (kept in shared memory) fits when the largest
// cell degree stays below the remaining 31 - bits (the top bit marks an
// erased cell), else the plan keeps 64-bit words in global memory.
inline __host__ __device__ int sched_id_bits(int S) {
  int b = 0;
  while (b < 31 && (S >> b) != 0) ++b;
  return b;
}
inline __host__ __device__ bool sched_packable32(int S, int sigma) {
  const int b = sched_id_bits(S);
  return b <= 30 && sigma < (1 << (31 - b));
}

inline DevGraph make_graph(const bpx_code* c, const void* ws, const WsLayout& L) {
  auto base = static_cast<const char*>(ws);
  DevGraph g;
  g.col_of_cell = reinterpret_cast<const int32_t*>(base + L.g_col_of_cell);
  g.cell_ptr = reinterpret_cast<const int32_t*>(base + L.g_cell_ptr);
  g.cell_src = reinterpret_cast<const int32_t*>(base + L.g_cell_src);
  g.src_ptr = reinterpret_cast<const int32_t*>(base + L.g_src_ptr);
  g.src_cell = reinterpret_cast<const int32_t*>(base + L.g_src_cell);
  g.t2_ptr = reinterpret_cast<const int32_t*>(base + L.g_t2_ptr);
  g.t2_a = reinterpret_cast<const int32_t*>(base + L.g_t2_a);
  g.t2_b = reinterpret_cast<const int32_t*>(base + L.g_t2_b);
  g.a2_ptr = reinterpret_cast<const int32_t*>(base + L.g_a2_ptr);
  g.a2_blk = reinterpret_cast<const int32_t*>(base + L.g_a2_blk);
  g.b2_ptr = reinterpret_cast<const int32_t*>(base + L.g_b2_ptr);
  g.b2_blk = reinterpret_cast<const int32_t*>(base + L.g_b2_blk);
  g.t2_order = reinterpret_cast<const int32_t*>(base + L.g_t2_order);
  g.k = c->k;
  g.EA = static_cast<int>(c->a2_ptr.size()) - 1;
  g.EB = static_cast<int>(c->b2_ptr.size()) - 1;
  g.n = c->n;
  g.S = c->S;
  g.num_cells = c->num_cells;
  g.num_edges = c->num_edges;
  g.sigma = c->sigma;
  return g;
}

inline DevPlan make_plan(const void* ws, const WsLayout& L) {
  char* base = const_cast<char*>(static_cast<const char*>(ws));
  auto at = [&](size_t off) { return reinterpret_cast<int32_t*>(base + off); };
  DevPlan p;
  p.info = at(L.p_info);
  p.ctr = at(L.p_ctr);
  p.cnt = at(L.p_cnt);
  p.surv = at(L.p_surv);
  p.direct = at(L.p_direct);
  p.front0 = at(L.p_front0);
  p.front1 = at(L.p_front1);
  p.word = reinterpret_cast<unsigned long long*>(base + L.p_word);
  p.depth = at(L.p_depth);
  p.resolver = at(L.p_resolver);
  p.order = at(L.p_order);
  p.wave_ptr = at(L.p_wave_ptr);
  p.cursor = at(L.p_cursor);
  p.pl_res = at(L.p_pl_res);
  p.pl_ptr = at(L.p_pl_ptr);
  p.pl_list = at(L.p_pl_list);
  return p;
}

// One job of a grouped launch (bpx_grouped_run): a whole coded
// multiplication with its own code, shapes, mask, workspace region and
// buffers.  *_base fields give the first CTA of the job in each multi-job
// kernel's grid (CTAs are looked up by binary search over these).
struct GJob {
  DevGraph g;
  DevPlan p;
  const float* A;
  const float* B;
  float* C;
  float* products;
  const uint8_t* mask;
  int32_t* info_out;
  void* a_hi;
  void* a_lo;
  void* b_hi;
  void* b_lo;
  int M, N, K, h;
  long long bsplit_base, enc_base, peel_base;
  int peel_chunk;
  int enc_sblocks;  // grouped encode: CTAs of the job (kEncGroupRows row blocks each, every k-chunk)
};

// Index of the last entry of the ascending array bases[0 .. n) that is <= x:
// the job of a grouped launch's CTA x.  The bases of one stage sit in a
// dense array (8 bytes a job, cached by every SM) rather than in the job
// records, so the search costs a few L1 hits per CTA.
__device__ __forceinline__ int find_base(const long long* __restrict__ bases, int n, long long x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(bases + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Encode grid geometry: 128 threads of 8 columns; a row takes
// min(128, next power of two >= K/8) threads, the CTA the rest in rows.
__host__ __device__ inline int enc_threads_per_row(int K) {
  int t = 1;
  while (t < 128 && t * 8 < K) t <<= 1;
  return t;
}
__host__ __device__ inline long long enc_row_blocks(long long rows, int K) {
  const int rpc = 128 / enc_threads_per_row(K);
  return (rows + rpc - 1) / rpc;
}
__host__ __device__ inline int enc_k_chunks(int K) {
  const int cols = enc_threads_per_row(K) * 8;
  return (K + cols - 1) / cols;
}

// Grid sizes of the multi-job kernels for one job.
inline long long bsplit_ctas(int N, int K) { return static_cast<long long>((N + 63) / 64) * ((K + 63) / 64); }
inline long long encode_ctas(long long rows, int K) { return enc_row_blocks(rows, K) * enc_k_chunks(K); }
// The grouped encode's CTA takes kEncGroupRows row blocks over every k-chunk,
// so that its job search and each row's lookups are shared by more elements.
constexpr int kEncGroupRows = 8;
inline long long enc_group_sblocks(long long rows, int K) {
  return (enc_row_blocks(rows, K) + kEncGroupRows - 1) / kEncGroupRows;
}
inline long long encode_group_ctas(long long rows, int K) { return enc_group_sblocks(rows, K); }
int peel_chunk_for(long long nv, int ctas_hint);

// Launchers (defined in the .cu files).  All return cudaError_t of the launch.
// max_state_bytes: the largest job's (cells + sources) x 4 bytes;
// max_want_bytes: the same with room for full ready lists (cells + 3 x
// sources); packable: every job passes sched_packable32 (else the plans'
// state stays in global memory).
cudaError_t launch_schedule_group(const GJob* d_jobs, int njobs, size_t max_state_bytes, size_t max_want_bytes,
                                  bool packable, cudaStream_t st);
// d_bases: the jobs' first CTA in the launch, ascending (job order).
cudaError_t launch_b_split_group(const GJob* d_jobs, const long long* d_bases, int njobs, long long total_ctas,
                                 cudaStream_t st);
cudaError_t launch_encode_split_group(const GJob* d_jobs, const long long* d_bases, int njobs,
                                      long long total_ctas, bool split, cudaStream_t st);
// Grouped peel: jobs d_order[0 .. ngather) in the gathered form (CTAs
// [0, gather_ctas)), the rest on the register path (CTAs [gather_ctas,
// total_ctas)), the latter on `side` between the events when both run;
// d_bases[i] = the first CTA of job d_order[i].
cudaError_t launch_peel_group(const GJob* d_jobs, const int32_t* d_order, const long long* d_bases, int njobs,
                              int ngather, long long gather_ctas, long long total_ctas, int first_wave,
                              int compensate_depth, int max_sigma, cudaStream_t st, cudaStream_t side,
                              cudaEvent_t fork, cudaEvent_t join);
// Whether a job's peel can take the gathered form in a grouped launch with this chunk.
bool peel_gather_ok(int S, int sigma, long long chunk);
// Split-fp16 scales (BPX_FP16X3).  The exponent e of a row of coded A or a
// column of B puts its largest magnitude amax at amax 2^e in [2^14, 2^15):
// both fp16 halves of every scaled element are then finite (the largest
// finite fp16 is 65504) and the hi half holds the top 11 bits of the largest
// one.  0 when amax is zero or not finite.
__host__ __device__ inline int f16_scale_exp(float amax) {
  if (!(amax > 0.f) || !(amax <= 3.402823466e38f)) return 0;
  int ex = 0;
  (void)frexpf(amax, &ex);  // amax = m 2^ex, m in [0.5, 1)
  return 15 - ex;           // amax 2^e = m 2^15
}
// 2^k as a float, for -126 <= k <= 127.
__host__ __device__ inline float pow2f(int k) {
  union { uint32_t u; float f; } v;
  v.u = static_cast<uint32_t>(k + 127) << 23;
  return v.f;
}
// x 2^e for the exponents f16_scale_exp returns (-113 <= e <= 163): two exact
// power-of-two multiplies (one rounding at most, when x 2^e is subnormal).
__host__ __device__ inline float scale_pow2(float x, int e) {
  const int e1 = e >> 1;
  return (x * pow2f(e1)) * pow2f(e - e1);
}
cudaError_t launch_encode_f16(const DevGraph& g, const DevPlan& p, const float* A, int M, int K, int h,
                              void* a_hi, void* a_lo, int32_t* a_exp, cudaStream_t st);
cudaError_t launch_b_f16(const float* B, int K, int N, void* b_hi, void* b_lo, uint32_t* b_max, int32_t* b_exp,
                         cudaStream_t st);
// gemm_config is a tile configuration the GEMM kernels have (tile codes 3,
// 4, 7 and 8 do not exist; negative values are invalid).
bool gemm_config_ok(int config);
cudaError_t launch_gemm_tc_grouped(const void* d_jobs, int njobs, long long total_tiles, bool split3,
                                   int config, cudaStream_t st);
size_t tc_job_bytes();

// Inputs of one job's entry in the grouped tensor-core GEMM table.
struct TcSpec {
  DevPlan p;
  const void* a_hi;
  const void* a_lo;
  const void* b_hi;
  const void* b_lo;
  int num_cells, N, K, h;
  float* products;
  float* C_direct;
  int32_t* info_out;
};
cudaError_t tc_build_table(const TcSpec* specs, int n, bool split3, int config, void* d_table,
                           long long* total_tiles, cudaStream_t st);
// cell_mask: the mask has one byte per cell instead of one per column.
// part: 0 = whole plan, 1 = survivors + depth-1 direct map, 2 = the rest.
cudaError_t launch_schedule(const DevGraph& g, const DevPlan& p, const uint8_t* mask,
                            int32_t* peel_order, uint8_t* recovered, int32_t* info_out,
                            cudaStream_t st, bool cell_mask = false, int part = 0);

// SMs the persistent GEMMs leave free (for a schedule running beside them);
// set by the entry points for the duration of a launch.
int& reserved_sms();
cudaError_t launch_peel(const DevGraph& g, const DevPlan& p, const float* P, float* C, int N, int h,
                        int first_wave, int compensate_depth, int ctas, cudaStream_t st);
cudaError_t launch_encode_f32(const DevGraph& g, const DevPlan& p, const float* A, int M, int K,
                              int h, float* out, cudaStream_t st);
cudaError_t launch_encode_split(const DevGraph& g, const DevPlan& p, const float* A, int M, int K,
                                int h, void* a_hi, void* a_lo, cudaStream_t st);
cudaError_t launch_b_split(const float* B, int K, int N, void* b_hi, void* b_lo, cudaStream_t st);
// MXFP8 staging (E4M3 data + UE8M0 scales in the GEMM's per-stage order) and GEMM.
cudaError_t launch_encode_mx(const DevGraph& g, const DevPlan& p, const float* A, int M, int K, int h,
                             void* out, void* sfa, cudaStream_t st);
cudaError_t launch_b_mx(const float* B, int K, int N, void* bt, void* sfb, cudaStream_t st);
cudaError_t launch_gemm_mx(const DevPlan& p, const void* a8, const void* sfa, const void* b8, const void* sfb,
                           int num_cells, int N, int K, int h, float* products, float* C_direct, int config,
                           int32_t* info_out, cudaStream_t st);
// Plain FP32 coded GEMM over the encode pass's FP32 coded rows.
cudaError_t launch_gemm_f32(const DevGraph& g, const DevPlan& p, const float* a_coded, const float* B, int N, int K,
                            int h, float* products, float* C_direct, cudaStream_t st);
// Tensor-core coded GEMM over the staged bf16 operands (split or plain).
// The encode fused into the GEMM's operand load (BPX_BF16 / BPX_BF16X3,
// CTA-pair 256 x 256 tiles): the coded rows are summed from A and split on
// chip; config 0 or a CTA-pair 64-wide config (tile code 0).
cudaError_t launch_gemm_fused(const DevGraph& g, const DevPlan& p, const float* A, int M, const void* b_hi,
                              const void* b_lo, int num_cells, int N, int K, int h, bool split3, float* products,
                              float* C_direct, int config, int32_t* info_out, cudaStream_t st);
// a_exp / b_exp non-null: the split-fp16 operands of BPX_FP16X3 (a_lo and
// b_lo required), unscaled by 2^-(a_exp[row] + b_exp[col]) in the epilogue.
cudaError_t launch_gemm_tc(const DevGraph& g, const DevPlan& p, const void* a_hi, const void* a_lo,
                           const void* b_hi, const void* b_lo, int num_cells, int N, int K, int h,
                           bool split3, float* products, float* C_direct, int config,
                           int32_t* info_out, cudaStream_t st, const int32_t* a_exp = nullptr,
                           const int32_t* b_exp = nullptr);

// Exact-slice staging (max |B| per column + B digit planes; max |A| per row
// position + coded A digit planes), digit-product GEMM and exact peel.
cudaError_t launch_exact_b(const float* B, int K, int N, const ExactParams& P, uint32_t* amax_b, void* bt,
                           cudaStream_t st);
// src_digits: the workspace's int8 source-digit region (ex_src) when the
// layout has one, else nullptr.
cudaError_t launch_exact_a(const DevGraph& g, const DevPlan& p, const float* A, int M, int K, int h,
                           const ExactParams& P, uint32_t* amax_a, void* a_planes, cudaStream_t st,
                           void* src_digits = nullptr);
cudaError_t launch_gemm_exact(const DevPlan& p, const void* a_planes, const void* b_planes, int num_cells, int N,
                              int K, int h, const ExactParams& P, int32_t* planes, int config, int32_t* info_out,
                              cudaStream_t st);
cudaError_t launch_peel_exact(const DevPlan& p, const ExactParams& P, const int32_t* planes, long long plane_stride,
                              long long* C64, float* C, const uint32_t* amax_a, const uint32_t* amax_b, int N,
                              int h, int ctas, cudaStream_t st);

// Two-dimensional scheme: operand staging (summed A blocks, summed B^T
// blocks, bf16 hi (+ lo)), products GEMM over each cell's terms, and the peel
// over strided h x w blocks of C.
cudaError_t launch_stage_2d(const DevGraph& g, const float* A, const float* B, int M, int N, int K, int h, int w,
                            void* a_hi, void* a_lo, void* b_hi, void* b_lo, cudaStream_t st);
cudaError_t launch_gemm_2d(const DevGraph& g, const DevPlan& p, const void* a_hi, const void* a_lo, const void* b_hi,
                           const void* b_lo, int N, int K, int h, int w, bool split3, float* products,
                           float* C_direct, int config, int32_t* info_out, cudaStream_t st);
cudaError_t launch_peel_2d(const DevGraph& g, const DevPlan& p, const float* P, float* C, int N, int h, int w,
                           int first_wave, int ctas, cudaStream_t st);

int num_sms();

}  // namespace bpx
