// Exact-slice staging and peel (BPX_EXACT).
//
// A and B become fixed-point integers x_int = rint(x 2^(bits - e)), with
// 2^(e-1) <= max|x| < 2^e taken per row position j of A (rows r = j mod h,
// shared by every source block so that the rows summed into one coded row
// share a scale) and per column of B.  Each integer is cut into S balanced
// base-2^w digits, most significant first; a coded digit plane is the plain
// sum of its sources' planes (no carries: linear in the sources, as the
// worker-side encode of Section III-A needs), and sigma 2^(w-1) <= 256 keeps
// it exact in bf16.
//
//   amax_a / amax_b  max |A| per row position and max |B| per column, kept as
//                    float bits (atomicMax on the bit patterns of
//                    non-negative floats orders them like the floats)
//   b_digits         B (K x N FP32) -> S bf16 digit planes of B^T: N rows of
//                    S Kp elements, plane l at column l Kp, zero digits for
//                    k in [K, Kp)
//   a_digits         rows of the surviving cells (compacted order, as the
//                    GEMM reads them): plane i of coded row (c, j) =
//                    sum_{s in supp(c)} D_i(A_s[j, :]), same row layout
//   peel_exact       the peel (Section I-A decoder, XOR read as exact integer
//                    subtraction) over Q_c = sum_d 2^(w (S-1-d)) P_c^d built
//                    from the GEMM's int32 diagonal planes, int64 throughout,
//                    then one rounding of Q_s 2^(w (S-1) - 2 bits + e_A + e_B)
//                    to FP32.
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "rn_scaled.cuh"

namespace bpx {
namespace {

constexpr int kExThreads = 128;

__device__ __forceinline__ int exponent_of(uint32_t amax_bits) {
  const float m = __uint_as_float(amax_bits);
  if (!(m > 0.f)) return 0;
  int e;
  frexpf(m, &e);
  return e;
}

// rint(x 2^shift): exact power-of-two scaling (|result| <= 2^24), then round
// to nearest even.  The scale is two power-of-two factors computed once per
// row or column (each within the float exponent range for |shift| <= 252).
// A product can round only when it falls below the normal range; for the
// shifts this path makes (bits minus a float exponent: |shift| < 250) the
// final value is then far below 1/2 and rounds to 0 either way, so the
// result equals rint of the exact x 2^shift.
struct Pow2Pair {
  float a, b;
};
__device__ __forceinline__ Pow2Pair pow2_pair(int shift) {
  const int s1 = shift >> 1;
  return {pow2f(s1), pow2f(shift - s1)};
}
__device__ __forceinline__ int to_fixed(float x, const Pow2Pair& f) { return __float2int_rn((x * f.a) * f.b); }

// Balanced base-2^w digits of x, most significant first: d[1..S-1] in
// [-2^(w-1), 2^(w-1)), d[0] takes the rest.
template <int S>
__device__ __forceinline__ void balanced_digits(int x, int w, int (&d)[S]) {
  const int half = 1 << (w - 1), mask = (1 << w) - 1;
#pragma unroll
  for (int i = S - 1; i >= 1; --i) {
    const int r = ((x + half) & mask) - half;
    d[i] = r;
    x = (x - r) >> w;  // x - r is a multiple of 2^w
  }
  d[0] = x;
}

__device__ __forceinline__ uint32_t bf16x2_of(int a, int b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(static_cast<float>(a), static_cast<float>(b));
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float warp_max(float m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// One warp per row of A.
__global__ void __launch_bounds__(256) exact_amax_a_kernel(const float* __restrict__ A, int M, int K, int h,
                                                           uint32_t* amax) {
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= M) return;
  const float4* row = reinterpret_cast<const float4*>(A + static_cast<long long>(r) * K);
  float m = 0.f;
  for (int i = lane; i < K / 4; i += 32) {
    const float4 v = __ldg(row + i);
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  m = warp_max(m);
  if (lane == 0) atomicMax(amax + r % h, __float_as_uint(m));
}

// Thread = 4 columns of B over a 256-row slice of K.
__global__ void __launch_bounds__(256) exact_amax_b_kernel(const float* __restrict__ B, int K, int N,
                                                           uint32_t* amax) {
  const int c4 = blockIdx.x * 256 + threadIdx.x;
  if (c4 * 4 >= N) return;
  const int k0 = blockIdx.y * 256, k1 = min(K, k0 + 256);
  float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = k0; k < k1; ++k) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(B + static_cast<long long>(k) * N) + c4);
    m.x = fmaxf(m.x, fabsf(v.x));
    m.y = fmaxf(m.y, fabsf(v.y));
    m.z = fmaxf(m.z, fabsf(v.z));
    m.w = fmaxf(m.w, fabsf(v.w));
  }
  atomicMax(amax + 4 * c4 + 0, __float_as_uint(m.x));
  atomicMax(amax + 4 * c4 + 1, __float_as_uint(m.y));
  atomicMax(amax + 4 * c4 + 2, __float_as_uint(m.z));
  atomicMax(amax + 4 * c4 + 3, __float_as_uint(m.w));
}

// B (K x N) -> digit planes of B^T through a 64 x 64 shared-memory tile
// (float4 reads along N, 16-byte bf16 writes along K).  gridDim.y = Kp / 64.
template <int S>
__global__ void __launch_bounds__(256)
exact_b_digits_kernel(const float* __restrict__ B, int K, int N, const uint32_t* __restrict__ amax_b, int w,
                      int bits, int Kp, __nv_bfloat16* bt) {
  __shared__ float tile[64][65];
  const int n0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
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
  const long long row_len = static_cast<long long>(S) * Kp;
#pragma unroll 1
  for (int i = 0; i < 2; ++i) {
    const int t = threadIdx.x + 256 * i;
    const int r = t >> 3, kc = t & 7;
    const int n = n0 + r, k = k0 + 8 * kc;
    if (n >= N) continue;
    const Pow2Pair f = pow2_pair(bits - exponent_of(amax_b[n]));
    int dg[8][S];
#pragma unroll
    for (int q = 0; q < 8; ++q) balanced_digits<S>(to_fixed(tile[8 * kc + q][r], f), w, dg[q]);
    __nv_bfloat16* dst = bt + static_cast<long long>(n) * row_len + k;
#pragma unroll
    for (int l = 0; l < S; ++l)
      *reinterpret_cast<uint4*>(dst + static_cast<long long>(l) * Kp) =
          make_uint4(bf16x2_of(dg[0][l], dg[1][l]), bf16x2_of(dg[2][l], dg[3][l]), bf16x2_of(dg[4][l], dg[5][l]),
                     bf16x2_of(dg[6][l], dg[7][l]));
  }
}

// Coded digit planes: thread = 8 consecutive k of one coded row (the encode
// geometry of the other tensor-core paths, over Kp).
template <int S>
__global__ void __launch_bounds__(kExThreads)
exact_a_digits_kernel(DevGraph g, DevPlan p, const float* __restrict__ A, int M, int K, int h,
                      const uint32_t* __restrict__ amax_a, int w, int bits, int Kp, __nv_bfloat16* out) {
  const int tpr = enc_threads_per_row(Kp);
  const int row = blockIdx.x * (kExThreads / tpr) + threadIdx.x / tpr;
  const int nsurv = p.ctr[CTR_NSURV];
  if (row >= nsurv * h) return;
  const int ci = row / h, j = row - ci * h;
  const int cell = p.surv[ci];
  const int k8 = (blockIdx.y * tpr + threadIdx.x % tpr) * 8;
  if (k8 >= Kp) return;
  int acc[S][8];
#pragma unroll
  for (int l = 0; l < S; ++l)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[l][q] = 0;
  if (k8 < K) {  // K % 8 == 0: a chunk is inside K or in the padding
    const Pow2Pair f = pow2_pair(bits - exponent_of(amax_a[j]));
    const int e0 = g.cell_ptr[cell], e1 = g.cell_ptr[cell + 1];
    for (int e = e0; e < e1; ++e) {
      const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
      if (arow >= M) continue;
      const float4* src = reinterpret_cast<const float4*>(A + arow * K + k8);
      const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
      const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int dg[S];
        balanced_digits<S>(to_fixed(x[q], f), w, dg);
#pragma unroll
        for (int l = 0; l < S; ++l) acc[l][q] += dg[l];
      }
    }
  }
  __nv_bfloat16* dst = out + static_cast<long long>(row) * S * Kp + k8;
#pragma unroll
  for (int l = 0; l < S; ++l)
    *reinterpret_cast<uint4*>(dst + static_cast<long long>(l) * Kp) =
        make_uint4(bf16x2_of(acc[l][0], acc[l][1]), bf16x2_of(acc[l][2], acc[l][3]),
                   bf16x2_of(acc[l][4], acc[l][5]), bf16x2_of(acc[l][6], acc[l][7]));
}

// Digits narrower than 8 bits (S >= 4) of a code whose cells hold many
// sources: the balanced digits of every source row are cut once, stored as
// bytes biased by 2^(w-1) + 1 (a digit lies in [-2^(w-1) - 1, 2^(w-1) + 1],
// so the biased byte is in [0, 2^w + 2]), laid out per row and 8-column
// chunk as S planes of 8 bytes.  The coded rows then add their sources'
// biased bytes in 16-bit lanes of 32-bit words, two digits per add: a lane
// reaches at most sigma (2^w + 2) <= 512 + 128 (w <= 9 - ceil(log2 sigma),
// sigma <= 64), far below 2^16, so no lane carries into the next.  The bias
// comes off once per sum: the same integers, so the same planes, without
// cutting every source element again for each cell that holds it.
template <int S>
__global__ void __launch_bounds__(256)
exact_src_digits_kernel(const float* __restrict__ A, int M, int K, int h, const uint32_t* __restrict__ amax_a,
                        int w, int bits, int Kp, long long src_rows, uint8_t* out) {
  const long long c = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x;  // (row, 8-column chunk)
  const int per_row = Kp / 8;
  const long long r = c / per_row;
  if (r >= src_rows) return;
  const int k8 = static_cast<int>(c - r * per_row) * 8;
  float x[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (r < M && k8 < K) {  // K % 8 == 0: a chunk is inside K or in the padding
    const float4* src = reinterpret_cast<const float4*>(A + r * K + k8);
    const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
    x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
    x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
  }
  const Pow2Pair f = pow2_pair(bits - exponent_of(amax_a[r % h]));
  const int bias = (1 << (w - 1)) + 1;
  uint32_t lo[S], hi[S];
#pragma unroll
  for (int l = 0; l < S; ++l) lo[l] = hi[l] = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int dg[S];
    balanced_digits<S>(to_fixed(x[q], f), w, dg);
#pragma unroll
    for (int l = 0; l < S; ++l) {
      const uint32_t b = static_cast<uint32_t>(dg[l] + bias);  // in [0, 2^w + 2]
      if (q < 4)
        lo[l] |= b << (8 * q);
      else
        hi[l] |= b << (8 * (q - 4));
    }
  }
  uint2* dst = reinterpret_cast<uint2*>(out) + c * S;
#pragma unroll
  for (int l = 0; l < S; ++l) dst[l] = make_uint2(lo[l], hi[l]);
}

// The coded digit planes from the biased source-digit bytes (same grid as
// exact_a_digits_kernel).
template <int S>
__global__ void __launch_bounds__(kExThreads)
exact_a_digits_src_kernel(DevGraph g, DevPlan p, const uint8_t* __restrict__ src_digits, int M, int h, int Kp,
                          int K, int w, __nv_bfloat16* out) {
  const int tpr = enc_threads_per_row(Kp);
  const int row = blockIdx.x * (kExThreads / tpr) + threadIdx.x / tpr;
  const int nsurv = p.ctr[CTR_NSURV];
  if (row >= nsurv * h) return;
  const int ci = row / h, j = row - ci * h;
  const int cell = p.surv[ci];
  const int k8 = (blockIdx.y * tpr + threadIdx.x % tpr) * 8;
  if (k8 >= Kp) return;
  // per plane, four words of two 16-bit lanes: columns (0, 2), (1, 3), (4, 6), (5, 7)
  uint32_t acc[S][4];
#pragma unroll
  for (int l = 0; l < S; ++l)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[l][q] = 0u;
  int count = 0;
  if (k8 < K) {
    const int per_row = Kp / 8;
    const int e0 = g.cell_ptr[cell], e1 = g.cell_ptr[cell + 1];
    for (int e = e0; e < e1; ++e) {
      const long long arow = static_cast<long long>(__ldg(g.cell_src + e)) * h + j;
      if (arow >= M) continue;
      ++count;
      const uint2* src = reinterpret_cast<const uint2*>(src_digits) + (arow * per_row + k8 / 8) * S;
      uint2 v[S];
#pragma unroll
      for (int l = 0; l < S; ++l) v[l] = __ldg(src + l);
#pragma unroll
      for (int l = 0; l < S; ++l) {
        acc[l][0] += __byte_perm(v[l].x, 0u, 0x4240);  // bytes 0, 2 into the two lanes
        acc[l][1] += __byte_perm(v[l].x, 0u, 0x4341);  // bytes 1, 3
        acc[l][2] += __byte_perm(v[l].y, 0u, 0x4240);
        acc[l][3] += __byte_perm(v[l].y, 0u, 0x4341);
      }
    }
  }
  const int off = count * ((1 << (w - 1)) + 1);  // the bias of every summed digit
  __nv_bfloat16* dst = out + static_cast<long long>(row) * S * Kp + k8;
#pragma unroll
  for (int l = 0; l < S; ++l) {
    int d[8];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      d[4 * q + 0] = static_cast<int>(acc[l][2 * q] & 0xffffu) - off;
      d[4 * q + 2] = static_cast<int>(acc[l][2 * q] >> 16) - off;
      d[4 * q + 1] = static_cast<int>(acc[l][2 * q + 1] & 0xffffu) - off;
      d[4 * q + 3] = static_cast<int>(acc[l][2 * q + 1] >> 16) - off;
    }
    *reinterpret_cast<uint4*>(dst + static_cast<long long>(l) * Kp) =
        make_uint4(bf16x2_of(d[0], d[1]), bf16x2_of(d[2], d[3]), bf16x2_of(d[4], d[5]), bf16x2_of(d[6], d[7]));
  }
}

// Peel on exact integers.  As in the FP32 peel, each CTA owns one slice of
// the block's 4-element groups and walks every wave over it; __syncthreads
// between waves is the only synchronisation.
template <int S>
__global__ void __launch_bounds__(256)
exact_peel_kernel(DevPlan p, const int32_t* __restrict__ planes, long long plane_stride, long long* C64, float* C,
                  const uint32_t* __restrict__ amax_a, const uint32_t* __restrict__ amax_b, int N, int h, int w,
                  int bits, long long nv, int chunk) {
  if (p.ctr[CTR_PLAN] != kPlanReady) {  // no schedule has planned this workspace: refuse, write nothing
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicExch(&p.info[BPX_INFO_DEVICE_ERR], BPX_ERR_INVAL);
      atomicExch(&p.info[BPX_INFO_STATUS], BPX_ERR_INVAL);
    }
    return;
  }
  const int nwaves = p.ctr[CTR_NWAVES];
  const long long v0 = static_cast<long long>(blockIdx.x) * chunk;
  if (v0 >= nv) return;
  const int clen = static_cast<int>(min(static_cast<long long>(chunk), nv - v0));
  const long long hN = static_cast<long long>(h) * N;
  const int e_base = w * (S - 1) - 2 * bits;
  for (int d = 1; d <= nwaves; ++d) {
    const int o0 = p.wave_ptr[d - 1], o1 = p.wave_ptr[d];
    const int items = (o1 - o0) * clen;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int jx = it / clen;
      const long long v = v0 + (it - jx * clen);
      const int i = o0 + jx;
      const int s = p.order[i], r = p.pl_res[i];
      long long q[4] = {0, 0, 0, 0};
#pragma unroll
      for (int dd = 0; dd < S; ++dd) {
        const int4 pv =
            __ldg(reinterpret_cast<const int4*>(planes + dd * plane_stride + static_cast<long long>(r) * hN) + v);
        const long long sc = 1LL << (w * (S - 1 - dd));
        q[0] += pv.x * sc;
        q[1] += pv.y * sc;
        q[2] += pv.z * sc;
        q[3] += pv.w * sc;
      }
      // subtrahends four at a time: their loads in flight together (exact
      // integers, so the order of the subtractions does not matter)
      for (int e = p.pl_ptr[i], e1 = p.pl_ptr[i + 1]; e < e1; e += 4) {
        int t[4];
        longlong2 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = e + u < e1 ? p.pl_list[e + u] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = b[u] = make_longlong2(0, 0);
          if (t[u] >= 0) {
            const longlong2* src = reinterpret_cast<const longlong2*>(C64 + static_cast<long long>(t[u]) * hN) + 2 * v;
            a[u] = src[0];
            b[u] = src[1];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          q[0] -= a[u].x;
          q[1] -= a[u].y;
          q[2] -= b[u].x;
          q[3] -= b[u].y;
        }
      }
      longlong2* dst = reinterpret_cast<longlong2*>(C64 + static_cast<long long>(s) * hN) + 2 * v;
      dst[0] = make_longlong2(q[0], q[1]);
      dst[1] = make_longlong2(q[2], q[3]);
      const long long el = 4 * v;
      const int j = static_cast<int>(el / N), n = static_cast<int>(el - static_cast<long long>(j) * N);
      const int ej = e_base + exponent_of(amax_a[j]);
      float out[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        out[u] = rn_float_scaled(q[u], ej + exponent_of(amax_b[n + u]));
      *reinterpret_cast<float4*>(C + static_cast<long long>(s) * hN + el) = make_float4(out[0], out[1], out[2], out[3]);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_exact_b(const float* B, int K, int N, const ExactParams& P, uint32_t* amax_b, void* bt,
                           cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(amax_b, 0, sizeof(uint32_t) * N, st);
  if (e != cudaSuccess) return e;
  exact_amax_b_kernel<<<dim3((N / 4 + 255) / 256, (K + 255) / 256), 256, 0, st>>>(B, K, N, amax_b);
  const dim3 grid((N + 63) / 64, P.Kp / 64);
  auto* out = static_cast<__nv_bfloat16*>(bt);
  switch (P.S) {
    case 3: exact_b_digits_kernel<3><<<grid, 256, 0, st>>>(B, K, N, amax_b, P.w, P.bits, P.Kp, out); break;
    case 4: exact_b_digits_kernel<4><<<grid, 256, 0, st>>>(B, K, N, amax_b, P.w, P.bits, P.Kp, out); break;
    case 5: exact_b_digits_kernel<5><<<grid, 256, 0, st>>>(B, K, N, amax_b, P.w, P.bits, P.Kp, out); break;
    case 6: exact_b_digits_kernel<6><<<grid, 256, 0, st>>>(B, K, N, amax_b, P.w, P.bits, P.Kp, out); break;
    case 8: exact_b_digits_kernel<8><<<grid, 256, 0, st>>>(B, K, N, amax_b, P.w, P.bits, P.Kp, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_exact_a(const DevGraph& g, const DevPlan& p, const float* A, int M, int K, int h,
                           const ExactParams& P, uint32_t* amax_a, void* a_planes, cudaStream_t st,
                           void* src_digits) {
  cudaError_t e = cudaMemsetAsync(amax_a, 0, sizeof(uint32_t) * h, st);
  if (e != cudaSuccess) return e;
  if (M > 0) exact_amax_a_kernel<<<(M + 7) / 8, 256, 0, st>>>(A, M, K, h, amax_a);
  const long long rows = static_cast<long long>(g.num_cells) * h;
  const dim3 grid(static_cast<unsigned>(enc_row_blocks(rows, P.Kp)), enc_k_chunks(P.Kp));
  auto* out = static_cast<__nv_bfloat16*>(a_planes);
  // the source-digit form pays off when cells hold many sources (a source row
  // is cut once instead of once per cell that holds it)
  if (src_digits && P.S >= 4 && static_cast<long long>(g.num_edges) >= 4LL * g.num_cells) {
    const long long src_rows = static_cast<long long>(g.S) * h;
    const long long chunks = src_rows * (P.Kp / 8);
    if ((chunks + 255) / 256 > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned sg = static_cast<unsigned>((chunks + 255) / 256);
    auto* sd = static_cast<uint8_t*>(src_digits);
    switch (P.S) {
      case 4:
        exact_src_digits_kernel<4><<<sg, 256, 0, st>>>(A, M, K, h, amax_a, P.w, P.bits, P.Kp, src_rows, sd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        exact_a_digits_src_kernel<4><<<grid, kExThreads, 0, st>>>(g, p, sd, M, h, P.Kp, K, P.w, out);
        break;
      case 5:
        exact_src_digits_kernel<5><<<sg, 256, 0, st>>>(A, M, K, h, amax_a, P.w, P.bits, P.Kp, src_rows, sd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        exact_a_digits_src_kernel<5><<<grid, kExThreads, 0, st>>>(g, p, sd, M, h, P.Kp, K, P.w, out);
        break;
      case 6:
        exact_src_digits_kernel<6><<<sg, 256, 0, st>>>(A, M, K, h, amax_a, P.w, P.bits, P.Kp, src_rows, sd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        exact_a_digits_src_kernel<6><<<grid, kExThreads, 0, st>>>(g, p, sd, M, h, P.Kp, K, P.w, out);
        break;
      case 8:
        exact_src_digits_kernel<8><<<sg, 256, 0, st>>>(A, M, K, h, amax_a, P.w, P.bits, P.Kp, src_rows, sd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        exact_a_digits_src_kernel<8><<<grid, kExThreads, 0, st>>>(g, p, sd, M, h, P.Kp, K, P.w, out);
        break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (P.S) {
    case 3: exact_a_digits_kernel<3><<<grid, kExThreads, 0, st>>>(g, p, A, M, K, h, amax_a, P.w, P.bits, P.Kp, out); break;
    case 4: exact_a_digits_kernel<4><<<grid, kExThreads, 0, st>>>(g, p, A, M, K, h, amax_a, P.w, P.bits, P.Kp, out); break;
    case 5: exact_a_digits_kernel<5><<<grid, kExThreads, 0, st>>>(g, p, A, M, K, h, amax_a, P.w, P.bits, P.Kp, out); break;
    case 6: exact_a_digits_kernel<6><<<grid, kExThreads, 0, st>>>(g, p, A, M, K, h, amax_a, P.w, P.bits, P.Kp, out); break;
    case 8: exact_a_digits_kernel<8><<<grid, kExThreads, 0, st>>>(g, p, A, M, K, h, amax_a, P.w, P.bits, P.Kp, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_peel_exact(const DevPlan& p, const ExactParams& P, const int32_t* planes, long long plane_stride,
                              long long* C64, float* C, const uint32_t* amax_a, const uint32_t* amax_b, int N,
                              int h, int ctas, cudaStream_t st) {
  const long long nv = static_cast<long long>(h) * N / 4;
  if (nv <= 0) return cudaSuccess;
  const int chunk = peel_chunk_for(nv, ctas);
  const unsigned grid = static_cast<unsigned>((nv + chunk - 1) / chunk);
#define BPX_PEEL_EXACT(SV)                                                                                     \
  exact_peel_kernel<SV><<<grid, 256, 0, st>>>(p, planes, plane_stride, C64, C, amax_a, amax_b, N, h, P.w, P.bits, \
                                              nv, chunk)
  switch (P.S) {
    case 3: BPX_PEEL_EXACT(3); break;
    case 4: BPX_PEEL_EXACT(4); break;
    case 5: BPX_PEEL_EXACT(5); break;
    case 6: BPX_PEEL_EXACT(6); break;
    case 8: BPX_PEEL_EXACT(8); break;
    default: return cudaErrorInvalidValue;
  }
#undef BPX_PEEL_EXACT
  return cudaGetLastError();
}

}  // namespace bpx
