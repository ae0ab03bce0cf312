// a2 (materialized) and operand staging for the tensor-core paths.
//
//   encode_f32    A_coded row (i h + j) = sum_{s in supp(c_i)} A[s h + j]  (FP32)
//   encode_split  the same sum, then split into bf16 hi = RN(x) and
//                 lo = RN(x - hi) (or hi only for plain bf16), K-major rows
//                 ready for the TMA loads of the tcgen05 GEMM
//   b_split       B (K x N, FP32) -> B^T hi / lo (N x K, bf16, K-major)
//
// c_i is the i-th surviving cell of the plan.  Rows of A past M read as zero
// (the zero padding of the last source blocks).  All are HBM-bound streams.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int kEncThreads = 256;

// One CTA per (coded row, 1024-column chunk); blockIdx.x walks the coded rows
// fastest so that CTAs resident together read the same K-chunk of A (L2 reuse
// of a source block across the cells that contain it).
template <int kMode>  // 0: FP32 out, 1: bf16 hi only, 2: bf16 hi + lo
__global__ void __launch_bounds__(kEncThreads)
encode_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, int M, int K, int h,
              float* out_f32, __nv_bfloat16* out_hi, __nv_bfloat16* out_lo) {
  const int nsurv = p.ctr[CTR_NSURV];
  const int row = blockIdx.x;  // coded row in the compacted order
  if (row >= nsurv * h) return;
  const int ci = row / h, j = row - ci * h;
  const int cell = p.surv[ci];
  const int e0 = g.cell_ptr[cell], e1 = g.cell_ptr[cell + 1];
  const int k4 = (blockIdx.y * kEncThreads + threadIdx.x) * 4;
  if (k4 >= K) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = e0; e < e1; ++e) {
    const long long arow = static_cast<long long>(g.cell_src[e]) * h + j;
    if (arow >= M) continue;
    const float4 x = __ldg(reinterpret_cast<const float4*>(A + arow * K + k4));
    acc.x += x.x;
    acc.y += x.y;
    acc.z += x.z;
    acc.w += x.w;
  }
  const long long o = static_cast<long long>(row) * K + k4;
  if (kMode == 0) {
    *reinterpret_cast<float4*>(out_f32 + o) = acc;
  } else {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(acc.x, acc.y);
    const __nv_bfloat162 h23 = __floats2bfloat162_rn(acc.z, acc.w);
    uint2 hv;
    hv.x = *reinterpret_cast<const uint32_t*>(&h01);
    hv.y = *reinterpret_cast<const uint32_t*>(&h23);
    *reinterpret_cast<uint2*>(out_hi + o) = hv;
    if (kMode == 2) {
      const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
      const __nv_bfloat162 l01 = __floats2bfloat162_rn(acc.x - f01.x, acc.y - f01.y);
      const __nv_bfloat162 l23 = __floats2bfloat162_rn(acc.z - f23.x, acc.w - f23.y);
      uint2 lv;
      lv.x = *reinterpret_cast<const uint32_t*>(&l01);
      lv.y = *reinterpret_cast<const uint32_t*>(&l23);
      *reinterpret_cast<uint2*>(out_lo + o) = lv;
    }
  }
}

// B (K x N row-major FP32) -> Bt (N x K row-major bf16) through a 64 x 64
// shared-memory tile: coalesced FP32 reads along N, bf16x2 writes along K.
constexpr int kTile = 64;
__global__ void __launch_bounds__(256)
b_split_kernel(const float* __restrict__ B, int K, int N, __nv_bfloat16* bt_hi,
               __nv_bfloat16* bt_lo) {
  __shared__ float tile[kTile][kTile + 1];
  const int n0 = blockIdx.x * kTile, k0 = blockIdx.y * kTile;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
  for (int r = ty; r < kTile; r += 4) {
    const int k = k0 + r, n = n0 + tx;
    tile[r][tx] = (k < K && n < N) ? __ldg(B + static_cast<long long>(k) * N + n) : 0.f;
  }
  __syncthreads();
  // write: thread handles (n = n0 + row, k = k0 + 2*c .. +1)
  const int c = threadIdx.x & 31, rr = threadIdx.x >> 5;  // 32 x 8
  for (int r = rr; r < kTile; r += 8) {
    const int n = n0 + r, k = k0 + 2 * c;
    if (n >= N || k >= K) continue;
    const float x0 = tile[2 * c][r], x1 = tile[2 * c + 1][r];
    const __nv_bfloat162 hv = __floats2bfloat162_rn(x0, x1);
    const long long o = static_cast<long long>(n) * K + k;
    *reinterpret_cast<__nv_bfloat162*>(bt_hi + o) = hv;
    if (bt_lo) {
      const float2 f = __bfloat1622float2(hv);
      *reinterpret_cast<__nv_bfloat162*>(bt_lo + o) = __floats2bfloat162_rn(x0 - f.x, x1 - f.y);
    }
  }
}

}  // namespace

cudaError_t launch_encode_f32(const DevGraph& g, const DevPlan& p, const float* A, int M, int K,
                              int h, float* out, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || K == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(rows), (K / 4 + kEncThreads - 1) / kEncThreads);
  encode_kernel<0><<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, out, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_encode_split(const DevGraph& g, const DevPlan& p, const float* A, int M, int K,
                                int h, void* a_hi, void* a_lo, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || K == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(rows), (K / 4 + kEncThreads - 1) / kEncThreads);
  auto hi = static_cast<__nv_bfloat16*>(a_hi);
  auto lo = static_cast<__nv_bfloat16*>(a_lo);
  if (lo)
    encode_kernel<2><<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, nullptr, hi, lo);
  else
    encode_kernel<1><<<grid, kEncThreads, 0, st>>>(g, p, A, M, K, h, nullptr, hi, nullptr);
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
