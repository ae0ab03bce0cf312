// a3, plain FP32 path: coded products on the CUDA cores (FFMA).
//
// The coded operand (rows of the surviving cells in ascending cell order,
// each the FP32 sum of its sources' rows) is formed by the encode pass first
// (an HBM-bound stream, well under 1 % of this GEMM's time), so that the GEMM
// streams both operands through asynchronous copies.  The product tile goes
// to the products buffer at the cell's slot, or -- for a cell that resolves a
// source at depth 1 -- straight into that source's block of C.
//
// Tiling: 128 x 256 output tile, 16-wide k-steps, 256 threads, each with an
// 8 x 16 register tile (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns
// tx*4 + {0..3} + {0, 64, 128, 192}, so that every shared-memory read is a
// conflict-free 16-byte load) held as packed pairs of adjacent columns and
// updated with fma.rn.f32x2.  B tiles arrive by cp.async (16-byte copies, zero-
// filled past K or N) into a ring of kStages buffers; A tiles go through
// registers so that they can be stored k-major (transposed), one k-step ahead.
// One barrier per 16-wide k-step.
#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int BM = 128, BN = 256, BK = 16, kThreads = 256, kStages = 3, APAD = 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  const int src_bytes = valid ? 16 : 0;  // 0: fill the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
gemm_f32_kernel(DevPlan p, const float* __restrict__ Ac, const float* __restrict__ B, int N, int K, int h,
                float* products, float* C_direct) {
  const int nsurv = p.ctr[CTR_NSURV];
  const long long Mc = static_cast<long long>(nsurv) * h;
  const long long m0 = static_cast<long long>(blockIdx.y) * BM;
  if (m0 >= Mc) return;
  const int n0 = blockIdx.x * BN;

  extern __shared__ __align__(16) float smem_f[];
  float (*As)[BK][BM + APAD] = reinterpret_cast<float (*)[BK][BM + APAD]>(smem_f);
  float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(smem_f + kStages * BK * (BM + APAD));

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  // A loader: row (tid % 128), k-half (tid / 128): two float4 along k
  const int a_row = tid & (BM - 1), a_kh = tid >> 7;
  const long long a_glob = m0 + a_row;
  const bool a_live = a_glob < Mc;
  const float* a_src = Ac + (a_live ? a_glob : 0) * static_cast<long long>(K);
  // B loader: k row (tid / 16), columns (tid % 16) * 4 + {0, 64, 128, 192}
  const int b_k = tid >> 4, b_n = (tid & 15) * 4;

  auto load_a = [&](int k0, float4& x0, float4& x1) {
    const int k = k0 + a_kh * 8;
    x0 = make_float4(0.f, 0.f, 0.f, 0.f);
    x1 = x0;
    if (a_live && k < K) x0 = __ldg(reinterpret_cast<const float4*>(a_src + k));
    if (a_live && k + 4 < K) x1 = __ldg(reinterpret_cast<const float4*>(a_src + k + 4));
  };
  auto store_a = [&](int buf, const float4& x0, const float4& x1) {
    const int k = a_kh * 8;
    As[buf][k + 0][a_row] = x0.x;
    As[buf][k + 1][a_row] = x0.y;
    As[buf][k + 2][a_row] = x0.z;
    As[buf][k + 3][a_row] = x0.w;
    As[buf][k + 4][a_row] = x1.x;
    As[buf][k + 5][a_row] = x1.y;
    As[buf][k + 6][a_row] = x1.z;
    As[buf][k + 7][a_row] = x1.w;
  };
  auto load_b = [&](int buf, int k0) {
    const int k = k0 + b_k;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + b_n + 64 * q;
      const bool v = k < K && n < N;
      const float* src = v ? B + static_cast<long long>(k) * N + n : B;
      cp_async16(&Bs[buf][b_k][b_n + 64 * q], src, v);
    }
  };

  // accumulators as packed pairs of adjacent columns (fma.rn.f32x2 does two
  // round-to-nearest FMAs per instruction, so the FMA stream takes half the
  // issue slots and the shared-memory reads fit beside it)
  uint64_t acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0ull;

  const int ktiles = (K + BK - 1) / BK;
  // prologue: B of the first kStages - 1 k-steps in flight, A of step 0 stored
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < ktiles) load_b(s, s * BK);
    cp_async_commit();
  }
  float4 ax0, ax1;
  load_a(0, ax0, ax1);
  store_a(0, ax0, ax1);
  if (ktiles > 1) load_a(BK, ax0, ax1);

  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt % kStages;
    cp_async_wait<kStages - 2>();  // B of step kt has landed
    __syncthreads();
    // refill: B of step kt + kStages - 1, A of step kt + 1 (held in
    // registers since the previous step), next A into registers
    if (kt + kStages - 1 < ktiles) load_b((kt + kStages - 1) % kStages, (kt + kStages - 1) * BK);
    cp_async_commit();
    if (kt + 1 < ktiles) {
      store_a((kt + 1) % kStages, ax0, ax1);
      if (kt + 2 < ktiles) load_a((kt + 2) * BK, ax0, ax1);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      uint64_t bv[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t addr = static_cast<uint32_t>(__cvta_generic_to_shared(&Bs[buf][kk][tx * 4 + 64 * q]));
        asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(bv[2 * q]), "=l"(bv[2 * q + 1]) : "r"(addr));
      }
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        uint64_t a2;
        asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(av[i]));
#pragma unroll
        for (int j = 0; j < 8; ++j) asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[i][j]) : "l"(a2), "l"(bv[j]));
      }
    }
  }
  cp_async_wait<0>();

  // Epilogue: rows ty*4+i (i < 4) and 64+ty*4+(i-4), columns tx*4 + 64 q.
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
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + tx * 4 + 64 * q;
      if (n < N) {
        const float2 lo = *reinterpret_cast<const float2*>(&acc[i][2 * q]);
        const float2 hi = *reinterpret_cast<const float2*>(&acc[i][2 * q + 1]);
        *reinterpret_cast<float4*>(dst + n) = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
    }
  }
}

}  // namespace

// a_coded: the FP32 coded rows of the surviving cells (encode pass output),
// num_cells h rows of K floats (only the surviving ones are read).
cudaError_t launch_gemm_f32(const DevGraph& g, const DevPlan& p, const float* a_coded, const float* B, int N, int K,
                            int h, float* products, float* C_direct, cudaStream_t st) {
  const long long rows = static_cast<long long>(g.num_cells) * h;
  if (rows == 0 || N == 0) return cudaSuccess;
  const size_t smem = sizeof(float) * kStages * BK * ((BM + APAD) + BN);
  cudaError_t e = cudaFuncSetAttribute(gemm_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dim3 grid((N + BN - 1) / BN, static_cast<unsigned>((rows + BM - 1) / BM));
  gemm_f32_kernel<<<grid, kThreads, smem, st>>>(p, a_coded, B, N, K, h, products, C_direct);
  return cudaGetLastError();
}

}  // namespace bpx
