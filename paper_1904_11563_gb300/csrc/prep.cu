// a2 (materialized) and operand staging for the tensor-core paths.
//
//   encode_f32    A_coded row (i h + j) = sum_{s in supp(c_i)} A[s h + j]  (FP32)
//   encode_split  the same sum, then split into bf16 hi = RN(x) and
//                 lo = RN(x - hi) (or hi only for plain bf16), K-major rows
//                 ready for the TMA loads of the tcgen05 GEMM
//   b_split       B (K x N, FP32) -> B^T hi / lo (N x K, bf16, K-major)
//   encode_f16    the same sum per coded row, scaled by 2^e (e from the
//                 row's largest magnitude, f16_scale_exp), split into fp16
//                 hi = RN(x) and lo = RN(x - hi); e stored per coded row
//   b_colmax / b_split_f16
//                 max |B| per column, then B^T hi / lo in fp16 under the
//                 column's 2^e
//
// c_i is the i-th surviving cell of the plan.  Rows of A past M read as zero
// (the zero padding of the last source blocks).  All are HBM-bound streams.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int kEncThreads = 128;
constexpr int kEncVec = 8;  // consecutive K elements per thread (two float4 loads per source)

// A CTA covers `rows` coded rows x `cols` columns (cols = min(1024, K rounded
// up to a power of two), rows = 1024 / cols): short K still fills the CTA.
// blockIdx.x walks the coded rows fastest so that CTAs resident together read
// the same K-chunk of A (L2 reuse of a source block across the cells that
// contain it).
template <int kMode>  // 0: FP32 out, 1: bf16 hi only, 2: bf16 hi + lo
__device__ __forceinline__ void encode_body(const DevGraph& g, const DevPlan& p,
                                            const float* __restrict__ A, int M, int K, int h,
                                            float* out_f32, __nv_bfloat16* out_hi,
                                            __nv_bfloat16* out_lo, int rblock, int kchunk) {
  const int tpr = enc_threads_per_row(K);  // threads per row
  const int row = rblock * (kEncThreads / tpr) + threadIdx.x / tpr;  // coded row, compacted order
  const int nsurv = p.ctr[CTR_NSURV];
  if (row >= nsurv * h) return;
  const int ci = row / h, j = row - ci * h;
  const int cell = p.surv[ci];
  const int e0 = g.cell_ptr[cell], e1 = g.cell_ptr[cell + 1];
  const int k8 = (kchunk * tpr + threadIdx.x % tpr) * kEncVec;
  if (k8 >= K) return;
  const bool full = k8 + kEncVec <= K;  // K % 8 == 0, so a chunk is full or absent
  // the 8 sums as packed pairs (add.rn.f32x2: two FP32 adds an issue slot,
  // each rounded as a scalar add; the same ascending order per element)
  uint64_t acc2[kEncVec / 2] = {0, 0, 0, 0};
  if (full) {
    for (int e = e0; e < e1; ++e) {
      const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
      if (arow >= M) continue;
      const float* src = A + arow * K + k8;
      uint64_t x[kEncVec / 2];
      asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(x[0]), "=l"(x[1]) : "l"(src));
      asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(x[2]), "=l"(x[3]) : "l"(src + 4));
#pragma unroll
      for (int q = 0; q < kEncVec / 2; ++q) asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc2[q]) : "l"(x[q]));
    }
  }
  if (!full) return;
  float acc[kEncVec];
#pragma unroll
  for (int q = 0; q < kEncVec / 2; ++q) asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * q]), "=f"(acc[2 * q + 1]) : "l"(acc2[q]));
  const long long o = static_cast<long long>(row) * K + k8;
  if (kMode == 0) {
    float4* d = reinterpret_cast<float4*>(out_f32 + o);
    d[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    d[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  } else {
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(acc[2 * q], acc[2 * q + 1]);
      hv[q] = *reinterpret_cast<const uint32_t*>(&hh);
      if (kMode == 2) {
        const float2 f = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(acc[2 * q] - f.x, acc[2 * q + 1] - f.y);
        lv[q] = *reinterpret_cast<const uint32_t*>(&ll);
      }
    }
    *reinterpret_cast<uint4*>(out_hi + o) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    if (kMode == 2) *reinterpret_cast<uint4*>(out_lo + o) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
  }
}

template <int kMode>
__global__ void __launch_bounds__(kEncThreads)
encode_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, int M, int K, int h,
              float* out_f32, __nv_bfloat16* out_hi, __nv_bfloat16* out_lo) {
  encode_body<kMode>(g, p, A, M, K, h, out_f32, out_hi, out_lo, blockIdx.x, blockIdx.y);
}

// B (K x N row-major FP32) -> Bt (N x K row-major bf16) through a 64 x 64
// shared-memory tile: float4 reads along N, 16-byte bf16 writes along K.
constexpr int kTile = 64;
__device__ __forceinline__ void b_split_body(const float* __restrict__ B, int K, int N,
                                             __nv_bfloat16* bt_hi, __nv_bfloat16* bt_lo, int bx,
                                             int by) {
  __shared__ float tile[kTile][kTile + 1];
  const int n0 = bx * kTile, k0 = by * kTile;
  {
    // 64 rows (k) x 16 float4 (n): 4 float4 per thread
    const int c4 = threadIdx.x & 15, r0 = threadIdx.x >> 4;  // 16 x 16
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + 16 * i, k = k0 + r, n = n0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K && n < N) v = __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N + n));
      tile[r][4 * c4 + 0] = v.x;
      tile[r][4 * c4 + 1] = v.y;
      tile[r][4 * c4 + 2] = v.z;
      tile[r][4 * c4 + 3] = v.w;
    }
  }
  __syncthreads();
  // 64 n-rows x 8 chunks of 8 k: thread -> (n = t / 8, chunk = t % 8), two rounds
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int t = threadIdx.x + 256 * i;
    const int r = t >> 3, kc = t & 7;
    const int n = n0 + r, k = k0 + 8 * kc;
    if (n >= N || k >= K) continue;
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x0 = tile[8 * kc + 2 * q][r], x1 = tile[8 * kc + 2 * q + 1][r];
      const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
      hv[q] = *reinterpret_cast<const uint32_t*>(&hh);
      const float2 f = __bfloat1622float2(hh);
      const __nv_bfloat162 ll = __floats2bfloat162_rn(x0 - f.x, x1 - f.y);
      lv[q] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    const long long o = static_cast<long long>(n) * K + k;
    *reinterpret_cast<uint4*>(bt_hi + o) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    if (bt_lo) *reinterpret_cast<uint4*>(bt_lo + o) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
  }
}

__global__ void __launch_bounds__(256)
b_split_kernel(const float* __restrict__ B, int K, int N, __nv_bfloat16* bt_hi, __nv_bfloat16* bt_lo) {
  b_split_body(B, K, N, bt_hi, bt_lo, blockIdx.x, blockIdx.y);
}

// Grouped launches: a flat grid over every job's CTAs; each CTA finds its job
// and its local (x, y) block, x fastest as in the single-job grids.
__global__ void __launch_bounds__(256)
b_split_group_kernel(const GJob* __restrict__ jobs, const long long* __restrict__ bases, int njobs) {
  const long long b = blockIdx.x;
  const int j = find_base(bases, njobs, b);
  const GJob& J = jobs[j];
  const uint32_t local = static_cast<uint32_t>(b - __ldg(bases + j));  // < 2^31: one launch's CTAs
  const uint32_t gx = (J.N + kTile - 1) / kTile, by = local / gx;
  b_split_body(J.B, J.K, J.N, static_cast<__nv_bfloat16*>(J.b_hi), static_cast<__nv_bfloat16*>(J.b_lo),
               static_cast<int>(local - by * gx), static_cast<int>(by));
}

// One row block over every k-chunk (the grouped encode): the row's cell and
// source range are looked up once, then each of the thread's 8-element
// chunks along K sums the same sources in the same ascending order (the same
// bits as encode_body).
template <int kMode>
__device__ __forceinline__ void encode_rows_body(const DevGraph& g, const DevPlan& p, const float* __restrict__ A,
                                                 int M, int K, int h, __nv_bfloat16* out_hi, __nv_bfloat16* out_lo,
                                                 int rblock) {
  const int tpr = enc_threads_per_row(K);
  const int row = rblock * (kEncThreads / tpr) + threadIdx.x / tpr;
  if (row >= p.ctr[CTR_NSURV] * h) return;
  const int ci = row / h, j = row - ci * h;
  const int cell = p.surv[ci];
  const int e0 = g.cell_ptr[cell], e1 = g.cell_ptr[cell + 1];
  const long long obase = static_cast<long long>(row) * K;
  for (int k8 = (threadIdx.x % tpr) * kEncVec; k8 < K; k8 += tpr * kEncVec) {
    uint64_t acc2[kEncVec / 2] = {0, 0, 0, 0};
    for (int e = e0; e < e1; ++e) {
      const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
      if (arow >= M) continue;
      const float* src = A + arow * K + k8;
      uint64_t x[kEncVec / 2];
      asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(x[0]), "=l"(x[1]) : "l"(src));
      asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(x[2]), "=l"(x[3]) : "l"(src + 4));
#pragma unroll
      for (int q = 0; q < kEncVec / 2; ++q) asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc2[q]) : "l"(x[q]));
    }
    float acc[kEncVec];
#pragma unroll
    for (int q = 0; q < kEncVec / 2; ++q)
      asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * q]), "=f"(acc[2 * q + 1]) : "l"(acc2[q]));
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(acc[2 * q], acc[2 * q + 1]);
      hv[q] = *reinterpret_cast<const uint32_t*>(&hh);
      if (kMode == 2) {
        const float2 f = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(acc[2 * q] - f.x, acc[2 * q + 1] - f.y);
        lv[q] = *reinterpret_cast<const uint32_t*>(&ll);
      }
    }
    *reinterpret_cast<uint4*>(out_hi + obase + k8) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    if (kMode == 2) *reinterpret_cast<uint4*>(out_lo + obase + k8) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
  }
}

template <int kMode>
__global__ void __launch_bounds__(kEncThreads)
encode_group_kernel(const GJob* __restrict__ jobs, const long long* __restrict__ bases, int njobs) {
  const long long b = blockIdx.x;
  const int j = find_base(bases, njobs, b);
  const GJob& J = jobs[j];
  // kEncGroupRows row blocks, every k-chunk (row blocks past the job's rows
  // return at once: their coded rows are beyond the surviving cells')
  const int rb0 = static_cast<int>(b - __ldg(bases + j)) * kEncGroupRows;
#pragma unroll 1
  for (int i = 0; i < kEncGroupRows; ++i)
    encode_rows_body<kMode>(J.g, J.p, J.A, J.M, J.K, J.h, static_cast<__nv_bfloat16*>(J.a_hi),
                            static_cast<__nv_bfloat16*>(J.a_lo), rb0 + i);
}

// ---- split-fp16 staging (BPX_FP16X3) --------------------------------------
//
// One CTA per coded row: the threads sum 8 consecutive K-elements of every
// source of the row's cell at a time (ascending sources, RN FP32 adds, as the
// other encodes), take the row's largest magnitude with a block reduction,
// and write the scaled fp16 halves.  Up to kF16Keep chunks per thread stay in
// registers between the two steps: 256 threads hold rows of K <= 8192, 512
// threads K <= 16384; longer rows sum their later chunks a second time.
constexpr int kF16Keep = 4;
// Codes with at least this many sources per cell on average take the
// K-chunked form (below).
constexpr int kF16ChunkedDegree = 4;

__device__ __forceinline__ void coded_chunk(const DevGraph& g, const float* __restrict__ A, int M, int K, int h,
                                            int e0, int e1, int j, int k8, float (&acc)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll 4
  for (int e = e0; e < e1; ++e) {
    const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
    if (arow >= M) continue;
    const float4* src = reinterpret_cast<const float4*>(A + arow * K + k8);
    const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
    acc[0] += x0.x; acc[1] += x0.y; acc[2] += x0.z; acc[3] += x0.w;
    acc[4] += x1.x; acc[5] += x1.y; acc[6] += x1.z; acc[7] += x1.w;
  }
}

// 8 scaled values -> fp16 hi and lo (16 bytes each)
__device__ __forceinline__ void f16_split8(const float (&v)[8], int e, __half* hi, __half* lo) {
  uint32_t hv[4], lv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = scale_pow2(v[2 * q], e), x1 = scale_pow2(v[2 * q + 1], e);
    const __half2 hh = __floats2half2_rn(x0, x1);
    const float2 f = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(x0 - f.x, x1 - f.y);
    hv[q] = *reinterpret_cast<const uint32_t*>(&hh);
    lv[q] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  *reinterpret_cast<uint4*>(hi) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
  *reinterpret_cast<uint4*>(lo) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

template <int kF16Threads>
__global__ void __launch_bounds__(kF16Threads)
encode_f16_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, int M, int K, int h, __half* out_hi,
                  __half* out_lo, int32_t* a_exp) {
  __shared__ float red[kF16Threads / 32];
  const int row = blockIdx.x;  // coded row, compacted order
  if (row >= p.ctr[CTR_NSURV] * h) return;
  const int ci = row / h, j = row - ci * h;
  const int cell = p.surv[ci];
  const int e0 = g.cell_ptr[cell], e1 = g.cell_ptr[cell + 1];
  const int nchunks = K / 8;  // K % 8 == 0
  float keep[kF16Keep][8];
#pragma unroll
  for (int it = 0; it < kF16Keep; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) keep[it][i] = 0.f;
  // sources outermost: a thread's loads of one source are all in flight at once
  for (int e = e0; e < e1; ++e) {
    const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
    if (arow >= M) continue;
    const float* src = A + arow * K;
    float4 x[kF16Keep][2];
#pragma unroll
    for (int it = 0; it < kF16Keep; ++it) {
      const int c = it * kF16Threads + static_cast<int>(threadIdx.x);
      if (c < nchunks) {
        x[it][0] = __ldg(reinterpret_cast<const float4*>(src + 8 * c));
        x[it][1] = __ldg(reinterpret_cast<const float4*>(src + 8 * c) + 1);
      }
    }
#pragma unroll
    for (int it = 0; it < kF16Keep; ++it) {
      const int c = it * kF16Threads + static_cast<int>(threadIdx.x);
      if (c < nchunks) {
        float* a = keep[it];
        a[0] += x[it][0].x; a[1] += x[it][0].y; a[2] += x[it][0].z; a[3] += x[it][0].w;
        a[4] += x[it][1].x; a[5] += x[it][1].y; a[6] += x[it][1].z; a[7] += x[it][1].w;
      }
    }
  }
  float amax = 0.f;
#pragma unroll
  for (int it = 0; it < kF16Keep; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) amax = fmaxf(amax, fabsf(keep[it][i]));
  for (int c = kF16Keep * kF16Threads + static_cast<int>(threadIdx.x); c < nchunks; c += kF16Threads) {
    float v[8];
    coded_chunk(g, A, M, K, h, e0, e1, j, 8 * c, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) amax = fmaxf(amax, fabsf(v[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  amax = red[0];
#pragma unroll
  for (int w = 1; w < kF16Threads / 32; ++w) amax = fmaxf(amax, red[w]);
  const int e = f16_scale_exp(amax);
  if (threadIdx.x == 0) a_exp[row] = e;
  const long long base = static_cast<long long>(row) * K;
#pragma unroll
  for (int it = 0; it < kF16Keep; ++it) {
    const int c = it * kF16Threads + static_cast<int>(threadIdx.x);
    if (c < nchunks) f16_split8(keep[it], e, out_hi + base + 8 * c, out_lo + base + 8 * c);
  }
  for (int c = kF16Keep * kF16Threads + static_cast<int>(threadIdx.x); c < nchunks; c += kF16Threads) {
    float v[8];
    coded_chunk(g, A, M, K, h, e0, e1, j, 8 * c, v);
    f16_split8(v, e, out_hi + base + 8 * c, out_lo + base + 8 * c);
  }
}

// High-degree codes (sources in many cells) take a K-chunked form instead, in
// the encode grid (coded rows fastest, so that CTAs resident together read
// the same K-chunk of A and a source chunk read for one cell is still in L2
// for the next cells that contain it).  One CTA per coded row reads every
// source row of a cell from DRAM again for each later cell that contains
// it.  Three steps:
//   1. each thread's 8 coded sums, stored unscaled as their FP32 bit patterns
//      (upper halves in the hi buffer, lower halves in the lo buffer); their
//      largest magnitude, reduced over the row's lanes of a warp, folded into
//      the row's word by atomicMax on the float bits (non-negative floats
//      order like their bits);
//   2. per row, the word becomes the exponent e (f16_scale_exp);
//   3. per 8 elements, the sums read back, scaled by 2^e and split into fp16
//      hi / lo in place: the same bits as the one-CTA-per-row form.
__global__ void __launch_bounds__(kEncThreads)
encode_f16_sum_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, int M, int K, int h, uint16_t* out_hi,
                      uint16_t* out_lo, uint32_t* row_max) {
  const int tpr = enc_threads_per_row(K);
  const int row = blockIdx.x * (kEncThreads / tpr) + threadIdx.x / tpr;
  const bool live = row < p.ctr[CTR_NSURV] * h;
  const int k8 = (blockIdx.y * tpr + threadIdx.x % tpr) * kEncVec;
  float m = 0.f;
  if (live && k8 < K) {
    const int ci = row / h, j = row - ci * h;
    const int cell = p.surv[ci];
    float v[8];
    coded_chunk(g, A, M, K, h, g.cell_ptr[cell], g.cell_ptr[cell + 1], j, k8, v);
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t b0 = __float_as_uint(v[2 * q]), b1 = __float_as_uint(v[2 * q + 1]);
      hv[q] = (b0 >> 16) | (b1 & 0xffff0000u);
      lv[q] = (b0 & 0xffffu) | (b1 << 16);
      m = fmaxf(m, fmaxf(fabsf(v[2 * q]), fabsf(v[2 * q + 1])));
    }
    const long long o = static_cast<long long>(row) * K + k8;
    *reinterpret_cast<uint4*>(out_hi + o) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<uint4*>(out_lo + o) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
  }
  const int span = tpr < 32 ? tpr : 32;  // a row's lanes: an aligned power-of-two group
  for (int o = 1; o < span; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (live && threadIdx.x % span == 0 && m > 0.f) atomicMax(row_max + row, __float_as_uint(m));
}

__global__ void __launch_bounds__(256) encode_f16_exp_kernel(DevPlan p, int h, int32_t* a_exp) {
  const long long row = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x;
  if (row < static_cast<long long>(p.ctr[CTR_NSURV]) * h)
    a_exp[row] = f16_scale_exp(__uint_as_float(static_cast<uint32_t>(a_exp[row])));
}

__global__ void __launch_bounds__(256)
encode_f16_rescale_kernel(DevPlan p, int K, int h, __half* out_hi, __half* out_lo, const int32_t* __restrict__ a_exp) {
  const long long c = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x;  // 8-element chunk
  const int per_row = K / 8;
  const long long row = c / per_row;
  if (row >= static_cast<long long>(p.ctr[CTR_NSURV]) * h) return;
  const long long o = c * 8;
  const uint4 hv = *reinterpret_cast<const uint4*>(out_hi + o);
  const uint4 lv = *reinterpret_cast<const uint4*>(out_lo + o);
  const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
  float v[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[2 * q] = __uint_as_float((hw[q] << 16) | (lw[q] & 0xffffu));
    v[2 * q + 1] = __uint_as_float((hw[q] & 0xffff0000u) | (lw[q] >> 16));
  }
  f16_split8(v, a_exp[row], out_hi + o, out_lo + o);
}

// max |B| per column: a CTA takes 256 columns (64 float4) x a range of
// kColRows rows, four row phases; one atomicMax per column per CTA on the
// float bits (ordered like the values, all being non-negative).
constexpr int kColRows = 128;
__global__ void __launch_bounds__(256) b_colmax_kernel(const float* __restrict__ B, int K, int N, uint32_t* bmax) {
  __shared__ float4 red[4][64];
  const int c4 = threadIdx.x & 63, ph = threadIdx.x >> 6;
  const int n = blockIdx.x * 256 + 4 * c4;
  const int k0 = blockIdx.y * kColRows, k1 = min(K, k0 + kColRows);
  float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
  if (n < N) {
#pragma unroll 4
    for (int k = k0 + ph; k < k1; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N + n));
      m.x = fmaxf(m.x, fabsf(v.x));
      m.y = fmaxf(m.y, fabsf(v.y));
      m.z = fmaxf(m.z, fabsf(v.z));
      m.w = fmaxf(m.w, fabsf(v.w));
    }
  }
  red[ph][c4] = m;
  __syncthreads();
  if (ph == 0 && n < N) {
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      m.x = fmaxf(m.x, red[q][c4].x);
      m.y = fmaxf(m.y, red[q][c4].y);
      m.z = fmaxf(m.z, red[q][c4].z);
      m.w = fmaxf(m.w, red[q][c4].w);
    }
    atomicMax(bmax + n, __float_as_uint(m.x));
    atomicMax(bmax + n + 1, __float_as_uint(m.y));
    atomicMax(bmax + n + 2, __float_as_uint(m.z));
    atomicMax(bmax + n + 3, __float_as_uint(m.w));
  }
}

// B (K x N) -> B^T fp16 hi / lo (N x K) under each column's 2^e, through the
// same 64 x 64 shared-memory transpose as b_split; the first k-tile's CTAs
// also record each column's exponent for the GEMM epilogue.
__global__ void __launch_bounds__(256)
b_split_f16_kernel(const float* __restrict__ B, int K, int N, const uint32_t* __restrict__ bmax, __half* bt_hi,
                   __half* bt_lo, int32_t* b_exp) {
  __shared__ float tile[kTile][kTile + 1];
  const int n0 = blockIdx.x * kTile, k0 = blockIdx.y * kTile;
  {
    const int c4 = threadIdx.x & 15, r0 = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + 16 * i, k = k0 + r, n = n0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K && n < N) v = __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N + n));
      tile[r][4 * c4 + 0] = v.x;
      tile[r][4 * c4 + 1] = v.y;
      tile[r][4 * c4 + 2] = v.z;
      tile[r][4 * c4 + 3] = v.w;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int t = threadIdx.x + 256 * i;
    const int r = t >> 3, kc = t & 7;
    const int n = n0 + r, k = k0 + 8 * kc;
    if (n >= N || k >= K) continue;
    const int e = f16_scale_exp(__uint_as_float(__ldg(bmax + n)));
    if (blockIdx.y == 0 && kc == 0) b_exp[n] = e;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = tile[8 * kc + q][r];
    const long long o = static_cast<long long>(n) * K + k;
    f16_split8(v, e, bt_hi + o, bt_lo + o);
  }
}

// ---- MXFP8 staging -------------------------------------------------------
//
// Every run of 32 consecutive K-elements of a row gets one UE8M0 scale 2^e,
// e = the smallest integer with amax / 2^e <= 448 (the largest finite E4M3),
// and its elements become RN-satfinite E4M3 of x / 2^e.  The four threads
// that own a 32-run (8 elements each) agree on amax through shuffles.

__device__ __forceinline__ int ue8m0_of(float amax) {
  if (!(amax > 0.f)) return 0;
  const float y = amax / 448.f;
  const uint32_t bits = __float_as_uint(y);
  int e = static_cast<int>((bits >> 23) & 0xFF) - 127;
  if ((bits & 0x7FFFFF) != 0 || ((bits >> 23) & 0xFF) == 0) e += 1;  // ceil(log2 y)
  return max(0, min(254, e + 127));
}

__device__ __forceinline__ uint2 e4m3x8(const float (&v)[8], int sbyte) {
  const int e = sbyte - 127;
  uint32_t w[2] = {0u, 0u};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_fp8x2_storage_t q = __nv_cvt_float2_to_fp8x2(
        make_float2(ldexpf(v[2 * i], -e), ldexpf(v[2 * i + 1], -e)), __NV_SATFINITE, __NV_E4M3);
    w[i >> 1] |= static_cast<uint32_t>(q) << (16 * (i & 1));
  }
  return make_uint2(w[0], w[1]);
}

// Coded A -> E4M3 rows + A scale blocks (512 B per 128-row tile and 128-wide
// K stage: byte 16 l + 4 q + j holds row 32 q + l, K-run 4 s + j).
__device__ __forceinline__ void encode_mx_body(const DevGraph& g, const DevPlan& p,
                                               const float* __restrict__ A, int M, int K, int h,
                                               uint8_t* out, uint8_t* sfa, int rblock, int kchunk) {
  const int tpr = enc_threads_per_row(K);
  const int row = rblock * (kEncThreads / tpr) + threadIdx.x / tpr;
  const int nsurv = p.ctr[CTR_NSURV];
  const int k8 = (kchunk * tpr + threadIdx.x % tpr) * kEncVec;
  const bool valid = row < nsurv * h && k8 < K;
  float acc[kEncVec];
#pragma unroll
  for (int i = 0; i < kEncVec; ++i) acc[i] = 0.f;
  if (valid) {
    const int ci = row / h, j = row - ci * h;
    const int cell = p.surv[ci];
    for (int e = g.cell_ptr[cell]; e < g.cell_ptr[cell + 1]; ++e) {
      const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
      if (arow >= M) continue;
      const float4* src = reinterpret_cast<const float4*>(A + arow * K + k8);
      const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
      acc[0] += x0.x; acc[1] += x0.y; acc[2] += x0.z; acc[3] += x0.w;
      acc[4] += x1.x; acc[5] += x1.y; acc[6] += x1.z; acc[7] += x1.w;
    }
  }
  float am = 0.f;
#pragma unroll
  for (int i = 0; i < kEncVec; ++i) am = fmaxf(am, fabsf(acc[i]));
  am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 1));
  am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 2));
  if (!valid) return;
  const int sbyte = ue8m0_of(am);
  *reinterpret_cast<uint2*>(out + static_cast<long long>(row) * K + k8) = e4m3x8(acc, sbyte);
  if ((k8 & 31) == 0) {
    const int kblk = k8 >> 5, ks = kblk >> 2, kb = kblk & 3, KS = K / 128;
    const int mt = row >> 7, rr = row & 127;
    sfa[(static_cast<long long>(mt) * KS + ks) * 512 + 16 * (rr & 31) + 4 * (rr >> 5) + kb] =
        static_cast<uint8_t>(sbyte);
  }
}

__global__ void __launch_bounds__(kEncThreads)
encode_mx_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, int M, int K, int h, uint8_t* out,
                 uint8_t* sfa) {
  encode_mx_body(g, p, A, M, K, h, out, sfa, blockIdx.x, blockIdx.y);
}

// B (K x N FP32) -> B^T E4M3 (N x K) + B scale blocks (1 KB per 256-column
// tile and 128-wide K stage: byte 512 t + 16 l + 4 c + j holds column
// 128 t + 32 c + l, K-run 4 s + j).
__global__ void __launch_bounds__(256)
b_mx_kernel(const float* __restrict__ B, int K, int N, uint8_t* bt, uint8_t* sfb) {
  __shared__ float tile[kTile][kTile + 1];
  const int n0 = blockIdx.x * kTile, k0 = blockIdx.y * kTile;
  {
    const int c4 = threadIdx.x & 15, r0 = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + 16 * i, k = k0 + r, n = n0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K && n < N) v = __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N + n));
      tile[r][4 * c4 + 0] = v.x;
      tile[r][4 * c4 + 1] = v.y;
      tile[r][4 * c4 + 2] = v.z;
      tile[r][4 * c4 + 3] = v.w;
    }
  }
  __syncthreads();
  const int KS = K / 128;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int t = threadIdx.x + 256 * i;
    const int r = t >> 3, kc = t & 7;  // 8 consecutive lanes share a column; 4 lanes = one 32-run
    const int n = n0 + r, k = k0 + 8 * kc;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = tile[8 * kc + q][r];
    float am = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) am = fmaxf(am, fabsf(v[q]));
    am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 1));
    am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 2));
    if (n >= N || k >= K) continue;
    const int sbyte = ue8m0_of(am);
    *reinterpret_cast<uint2*>(bt + static_cast<long long>(n) * K + k) = e4m3x8(v, sbyte);
    if ((kc & 3) == 0) {
      const int kblk = k >> 5, ks = kblk >> 2, kb = kblk & 3;
      const int nt = n >> 8, nn = n & 255;
      sfb[(static_cast<long long>(nt) * KS + ks) * 1024 + 512 * (nn >> 7) + 16 * (nn & 31) +
          4 * ((nn & 127) >> 5) + kb] = static_cast<uint8_t>(sbyte);
    }
  }
}

}  // namespace

cudaError_t launch_encode_mx(const DevGraph& g, const DevPlan& p, const float* A, int M, int K, int h,
                             void* out, void* sfa, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || K == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(enc_row_blocks(rows, K)), static_cast<unsigned>(enc_k_chunks(K)));
  encode_mx_kernel<<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, static_cast<uint8_t*>(out),
                                                 static_cast<uint8_t*>(sfa));
  return cudaGetLastError();
}

cudaError_t launch_b_mx(const float* B, int K, int N, void* bt, void* sfb, cudaStream_t st) {
  if (K == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + kTile - 1) / kTile, (K + kTile - 1) / kTile);
  b_mx_kernel<<<grid, 256, 0, st>>>(B, K, N, static_cast<uint8_t*>(bt), static_cast<uint8_t*>(sfb));
  return cudaGetLastError();
}

cudaError_t launch_encode_f32(const DevGraph& g, const DevPlan& p, const float* A, int M, int K,
                              int h, float* out, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || K == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(enc_row_blocks(rows, K)), static_cast<unsigned>(enc_k_chunks(K)));
  encode_kernel<0><<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, out, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_encode_split(const DevGraph& g, const DevPlan& p, const float* A, int M, int K,
                                int h, void* a_hi, void* a_lo, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || K == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(enc_row_blocks(rows, K)), static_cast<unsigned>(enc_k_chunks(K)));
  auto hi = static_cast<__nv_bfloat16*>(a_hi);
  auto lo = static_cast<__nv_bfloat16*>(a_lo);
  if (lo)
    encode_kernel<2><<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, nullptr, hi, lo);
  else
    encode_kernel<1><<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, nullptr, hi, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_b_split_group(const GJob* d_jobs, const long long* d_bases, int njobs, long long total_ctas,
                                 cudaStream_t st) {
  if (total_ctas <= 0) return cudaSuccess;
  b_split_group_kernel<<<static_cast<unsigned>(total_ctas), 256, 0, st>>>(d_jobs, d_bases, njobs);
  return cudaGetLastError();
}

cudaError_t launch_encode_split_group(const GJob* d_jobs, const long long* d_bases, int njobs,
                                      long long total_ctas, bool split, cudaStream_t st) {
  if (total_ctas <= 0) return cudaSuccess;
  // plain bf16 jobs have no lo buffer: the hi-only variant never touches it
  if (split)
    encode_group_kernel<2><<<static_cast<unsigned>(total_ctas), kEncThreads, 0, st>>>(d_jobs, d_bases, njobs);
  else
    encode_group_kernel<1><<<static_cast<unsigned>(total_ctas), kEncThreads, 0, st>>>(d_jobs, d_bases, njobs);
  return cudaGetLastError();
}

cudaError_t launch_encode_f16(const DevGraph& g, const DevPlan& p, const float* A, int M, int K, int h,
                              void* a_hi, void* a_lo, int32_t* a_exp, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || K == 0) return cudaSuccess;
  if (rows > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (static_cast<long long>(g.num_edges) >= kF16ChunkedDegree * static_cast<long long>(g.num_cells)) {
    // high mean degree: the K-chunked form
    cudaError_t e = cudaMemsetAsync(a_exp, 0, sizeof(int32_t) * static_cast<size_t>(rows), st);
    if (e != cudaSuccess) return e;
    const dim3 grid(static_cast<unsigned>(enc_row_blocks(rows, K)), static_cast<unsigned>(enc_k_chunks(K)));
    encode_f16_sum_kernel<<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, static_cast<uint16_t*>(a_hi),
                                                         static_cast<uint16_t*>(a_lo), reinterpret_cast<uint32_t*>(a_exp));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    encode_f16_exp_kernel<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, st>>>(p, h, a_exp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long chunks = rows * (K / 8);
    if ((chunks + 255) / 256 > 0x7fffffffLL) return cudaErrorInvalidValue;
    encode_f16_rescale_kernel<<<static_cast<unsigned>((chunks + 255) / 256), 256, 0, st>>>(
        p, K, h, static_cast<__half*>(a_hi), static_cast<__half*>(a_lo), a_exp);
    return cudaGetLastError();
  }
  if (K <= 256 * 8 * kF16Keep)
    encode_f16_kernel<256><<<static_cast<unsigned>(rows), 256, 0, st>>>(
        g, p, A, M, K, h, static_cast<__half*>(a_hi), static_cast<__half*>(a_lo), a_exp);
  else
    encode_f16_kernel<512><<<static_cast<unsigned>(rows), 512, 0, st>>>(
        g, p, A, M, K, h, static_cast<__half*>(a_hi), static_cast<__half*>(a_lo), a_exp);
  return cudaGetLastError();
}

cudaError_t launch_b_f16(const float* B, int K, int N, void* b_hi, void* b_lo, uint32_t* b_max, int32_t* b_exp,
                         cudaStream_t st) {
  if (K == 0 || N == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(b_max, 0, sizeof(uint32_t) * static_cast<size_t>(N), st);
  if (e != cudaSuccess) return e;
  b_colmax_kernel<<<dim3((N + 255) / 256, (K + kColRows - 1) / kColRows), 256, 0, st>>>(B, K, N, b_max);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  b_split_f16_kernel<<<dim3((N + kTile - 1) / kTile, (K + kTile - 1) / kTile), 256, 0, st>>>(
      B, K, N, b_max, static_cast<__half*>(b_hi), static_cast<__half*>(b_lo), b_exp);
  return cudaGetLastError();
}

cudaError_t launch_b_split(const float* B, int K, int N, void* b_hi, void* b_lo, cudaStream_t st) {
  if (K == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + kTile - 1) / kTile, (K + kTile - 1) / kTile);
  b_split_kernel<<<grid, 256, 0, st>>>(B, K, N, static_cast<__nv_bfloat16*>(b_hi),
                                       static_cast<__nv_bfloat16*>(b_lo));
  return cudaGetLastError();
}

}  // namespace bpx
