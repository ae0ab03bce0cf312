// Two-dimensional scheme (Section III-A, Examples 1 and 2): staging of the
// summed operands and the peel over h x w blocks of C.
//
// Source s = z k + l is the block C[z h .. , l w ..] = A_z B_l.  Every cell is
// a list of products (sum_{z in Z} A_z)(sum_{l in L} B_l) (host factoring);
// the distinct A operands (h rows each) and B operands (w rows of B^T each)
// are staged once per call as bf16 hi (+ lo) for the tensor-core GEMM:
//   a_ops_split  A operand e, row r = sum_{z in Z_e} A[z h + r, :]  (rows past
//                M read as zero), split hi = RN(x), lo = RN(x - hi)
//   b_ops_split  B operand f, row r of B^T = sum_{l in L_f} B[:, l w + r],
//                through a 64 x 64 shared-memory transpose
//   peel_2d      C_s = P_r - sum_{t in supp(r), t != s, ascending} C_t over
//                h x w blocks: products contiguous (row stride w), blocks of
//                C strided (row stride N)
// All three are HBM-bound streams.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int kThreads2 = 128;

__device__ __forceinline__ void split8(const float (&x)[8], __nv_bfloat16* hi, __nv_bfloat16* lo) {
  uint32_t hv[4], lv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    hv[q] = *reinterpret_cast<const uint32_t*>(&hh);
    const float2 f = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(x[2 * q] - f.x, x[2 * q + 1] - f.y);
    lv[q] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  *reinterpret_cast<uint4*>(hi) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
  if (lo) *reinterpret_cast<uint4*>(lo) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

// Thread = 8 consecutive k of one operand row (the encode geometry).
__global__ void __launch_bounds__(kThreads2)
a_ops_split_kernel(DevGraph g, const float* __restrict__ A, int M, int K, int h, __nv_bfloat16* a_hi,
                   __nv_bfloat16* a_lo) {
  const int tpr = enc_threads_per_row(K);
  const long long row = static_cast<long long>(blockIdx.x) * (kThreads2 / tpr) + threadIdx.x / tpr;
  if (row >= static_cast<long long>(g.EA) * h) return;
  const int e = static_cast<int>(row / h), r = static_cast<int>(row - static_cast<long long>(e) * h);
  const int k8 = (blockIdx.y * tpr + threadIdx.x % tpr) * 8;
  if (k8 >= K) return;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = g.a2_ptr[e]; i < g.a2_ptr[e + 1]; ++i) {
    const long long arow = static_cast<long long>(__ldg(g.a2_blk + i)) * h + r;
    if (arow >= M) continue;
    const float4* src = reinterpret_cast<const float4*>(A + arow * K + k8);
    const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
    acc[0] += x0.x; acc[1] += x0.y; acc[2] += x0.z; acc[3] += x0.w;
    acc[4] += x1.x; acc[5] += x1.y; acc[6] += x1.z; acc[7] += x1.w;
  }
  const long long o = row * K + k8;
  split8(acc, a_hi + o, a_lo ? a_lo + o : nullptr);
}

// blockIdx.x = (operand f, 64-column slice of its w columns), blockIdx.y =
// 64-row slice of K.
__global__ void __launch_bounds__(256)
b_ops_split_kernel(DevGraph g, const float* __restrict__ B, int K, int N, int w, __nv_bfloat16* bt_hi,
                   __nv_bfloat16* bt_lo) {
  __shared__ float tile[64][65];
  const int nslices = (w + 63) / 64;
  const int f = blockIdx.x / nslices;
  const int n0 = (blockIdx.x - f * nslices) * 64, k0 = blockIdx.y * 64;
  {
    const int c4 = threadIdx.x & 15, r0 = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + 16 * i, k = k0 + r, n = n0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K && n < w) {
        for (int j = g.b2_ptr[f]; j < g.b2_ptr[f + 1]; ++j) {
          const long long col = static_cast<long long>(__ldg(g.b2_blk + j)) * w + n;
          const float4 x = __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N + col));
          v.x += x.x;
          v.y += x.y;
          v.z += x.z;
          v.w += x.w;
        }
      }
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
    if (n >= w || k >= K) continue;
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = tile[8 * kc + q][r];
    const long long o = (static_cast<long long>(f) * w + n) * K + k;
    split8(x, bt_hi + o, bt_lo ? bt_lo + o : nullptr);
  }
}

__device__ __forceinline__ float4 ldg_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Peel over h x w blocks: each CTA owns a slice of the block's 4-element
// groups (v -> row v / (w/4), column 4 (v % (w/4))) and walks every wave;
// __syncthreads between waves is the only synchronisation.
template <int kB>
__global__ void __launch_bounds__(256)
peel_2d_kernel(DevPlan p, int kc, const float* __restrict__ P, float* C, int h, int w, long long ldc, long long nv,
               int chunk, int first_wave) {
  const int nwaves = p.ctr[CTR_NWAVES];
  const long long v0 = static_cast<long long>(blockIdx.x) * chunk;
  if (v0 >= nv) return;
  const int clen = static_cast<int>(min(static_cast<long long>(chunk), nv - v0));
  const int w4 = w / 4;
  const long long hw = static_cast<long long>(h) * w;
  for (int d = first_wave; d <= nwaves; ++d) {
    const int o0 = p.wave_ptr[d - 1], o1 = p.wave_ptr[d];
    const int items = (o1 - o0) * clen;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int jx = it / clen;
      const long long v = v0 + (it - jx * clen);
      const int i = o0 + jx;
      const int row = static_cast<int>(v / w4), col = static_cast<int>(v - static_cast<long long>(row) * w4) * 4;
      auto blk = [&](int s) {
        const int z = s / kc, l = s - z * kc;
        return C + (static_cast<long long>(z) * h + row) * ldc + static_cast<long long>(l) * w + col;
      };
      const int s = p.order[i], r = p.pl_res[i];
      float4 acc = ldg_stream(reinterpret_cast<const float4*>(P + static_cast<long long>(r) * hw +
                                                              static_cast<long long>(row) * w + col));
      for (int e = p.pl_ptr[i], e1 = p.pl_ptr[i + 1]; e < e1; e += kB) {
        int t[kB];
        float4 x[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q) t[q] = (e + q < e1) ? p.pl_list[e + q] : -1;
#pragma unroll
        for (int q = 0; q < kB; ++q)
          x[q] = t[q] >= 0 ? *reinterpret_cast<const float4*>(blk(t[q])) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kB; ++q)
          if (t[q] >= 0) {
            acc.x -= x[q].x;
            acc.y -= x[q].y;
            acc.z -= x[q].z;
            acc.w -= x[q].w;
          }
      }
      *reinterpret_cast<float4*>(blk(s)) = acc;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_stage_2d(const DevGraph& g, const float* A, const float* B, int M, int N, int K, int h, int w,
                            void* a_hi, void* a_lo, void* b_hi, void* b_lo, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.EA) * h;
  const dim3 ga(static_cast<unsigned>(enc_row_blocks(rows, K)), enc_k_chunks(K));
  a_ops_split_kernel<<<ga, kThreads2, 0, st>>>(g, A, M, K, h, static_cast<__nv_bfloat16*>(a_hi),
                                               static_cast<__nv_bfloat16*>(a_lo));
  const dim3 gb(static_cast<unsigned>(g.EB * ((w + 63) / 64)), (K + 63) / 64);
  b_ops_split_kernel<<<gb, 256, 0, st>>>(g, B, K, N, w, static_cast<__nv_bfloat16*>(b_hi),
                                         static_cast<__nv_bfloat16*>(b_lo));
  return cudaGetLastError();
}

cudaError_t launch_peel_2d(const DevGraph& g, const DevPlan& p, const float* P, float* C, int N, int h, int w,
                           int first_wave, int ctas, cudaStream_t st) {
  const long long nv = static_cast<long long>(h) * w / 4;
  if (nv <= 0) return cudaSuccess;
  const int chunk = peel_chunk_for(nv, ctas);
  const unsigned grid = static_cast<unsigned>((nv + chunk - 1) / chunk);
  if (g.sigma > 5)
    peel_2d_kernel<8><<<grid, 256, 0, st>>>(p, g.k, P, C, h, w, N, nv, chunk, first_wave);
  else
    peel_2d_kernel<4><<<grid, 256, 0, st>>>(p, g.k, P, C, h, w, N, nv, chunk, first_wave);
  return cudaGetLastError();
}

}  // namespace bpx
