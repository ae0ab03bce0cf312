// a2 + a3, plain FP32 path: coded products on the CUDA cores (FFMA) with the
// encode fused into the operand load.
//
// Rows of the stacked coded operand are the h rows of each surviving cell in
// ascending cell order.  While a CTA stages its 128 x 8 slice of coded A into
// shared memory, each loading thread sums the matching rows of the cell's
// source blocks (Section III-A: the worker forms the sum itself), so the
// coded operand never exists in global memory.  The product tile goes to the
// products buffer at the cell's slot, or -- for a cell that resolves a source
// at depth 1 -- straight into that source's block of C.
//
// Tiling: 128 x 128 output tile, k-step 8, 256 threads with an 8 x 8
// register tile each (two 4-row by two 4-column sub-blocks so that the
// shared-memory reads are conflict-free float4s), register-prefetched double
// buffer, one barrier per k-step.
#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, kThreads = 256, APAD = 4;

__global__ void __launch_bounds__(kThreads, 2)
gemm_f32_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, const float* __restrict__ B,
                int M, int N, int K, int h, float* products, float* C_direct) {
  const int nsurv = p.ctr[CTR_NSURV];
  const long long Mc = static_cast<long long>(nsurv) * h;
  const long long m0 = static_cast<long long>(blockIdx.y) * BM;
  if (m0 >= Mc) return;
  const int n0 = blockIdx.x * BN;

  __shared__ __align__(16) float As[2][BK][BM + APAD];
  __shared__ __align__(16) float Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  // A loader: one coded row, 4 consecutive k per thread.
  const int a_row = tid >> 1, a_k = (tid & 1) * 4;
  const long long r_glob = m0 + a_row;
  int a_e0 = 0, a_e1 = 0, a_j = 0;
  if (r_glob < Mc) {
    const int ci = static_cast<int>(r_glob / h);
    a_j = static_cast<int>(r_glob - static_cast<long long>(ci) * h);
    const int cell = p.surv[ci];
    a_e0 = g.cell_ptr[cell];
    a_e1 = g.cell_ptr[cell + 1];
  }
  // B loader: one k row, 4 consecutive columns per thread.
  const int b_k = tid >> 5, b_n = (tid & 31) * 4;

  auto load_a = [&](int k0) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int k = k0 + a_k;
    if (k < K) {
      for (int e = a_e0; e < a_e1; ++e) {
        const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + a_j;
        if (arow < M) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(A + arow * K + k));
          acc.x += x.x;
          acc.y += x.y;
          acc.z += x.z;
          acc.w += x.w;
        }
      }
    }
    return acc;
  };
  auto load_b = [&](int k0) {
    const int k = k0 + b_k, n = n0 + b_n;
    if (k < K && n < N) return __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N + n));
    return make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store_tiles = [&](int buf, float4 a, float4 b) {
    As[buf][a_k + 0][a_row] = a.x;
    As[buf][a_k + 1][a_row] = a.y;
    As[buf][a_k + 2][a_row] = a.z;
    As[buf][a_k + 3][a_row] = a.w;
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_n]) = b;
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int ktiles = (K + BK - 1) / BK;
  store_tiles(0, load_a(0), load_b(0));
  __syncthreads();

  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    float4 na, nb;
    const bool more = kt + 1 < ktiles;
    if (more) {
      na = load_a((kt + 1) * BK);
      nb = load_b((kt + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) store_tiles(buf ^ 1, na, nb);
    __syncthreads();
  }

  // Epilogue: rows ty*4+i and 64+ty*4+i, columns tx*4.. and 64+tx*4..
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= Mc) continue;
    const int ci = static_cast<int>(r / h);
    const int j = static_cast<int>(r - static_cast<long long>(ci) * h);
    const int cell = p.surv[ci];
    const int ds = C_direct ? p.direct[cell] : -1;
    float* dst = ds >= 0 ? C_direct + (static_cast<long long>(ds) * h + j) * N
                         : products + (static_cast<long long>(cell) * h + j) * N;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int n = n0 + half * 64 + tx * 4;
      if (n < N) {
        *reinterpret_cast<float4*>(dst + n) =
            make_float4(acc[i][half * 4 + 0], acc[i][half * 4 + 1], acc[i][half * 4 + 2],
                        acc[i][half * 4 + 3]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_gemm_f32(const DevGraph& g, const DevPlan& p, const float* A, const float* B,
                            int M, int N, int K, int h, float* products, float* C_direct,
                            cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, static_cast<unsigned>((rows + BM - 1) / BM));
  gemm_f32_kernel<<<grid, kThreads, 0, st>>>(g, p, A, B, M, N, K, h, products, C_direct);
  return cudaGetLastError();
}

}  // namespace bpx
