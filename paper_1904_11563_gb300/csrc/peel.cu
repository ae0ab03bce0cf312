// a4: numeric peel.  C_s = P_r - sum_{t in supp(r), t != s} C_t along the
// planned waves (Section I-A decoder, XOR read as subtraction).
//
// The subtraction is elementwise over the h x N block, so element i of C_s
// depends only on element i of the blocks it reads.  Each CTA therefore owns
// one contiguous slice of the block's float4 index range and walks the whole
// schedule over that slice: a __syncthreads between waves is the only
// synchronisation, with no grid barrier, flag or spin-wait.  Within a wave
// the (source, float4) items of the slice are spread over the CTA's threads,
// consecutive threads on consecutive float4s (128-bit coalesced accesses).
#include <algorithm>

#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int kPeelThreads = 256;

__device__ __forceinline__ float4 ldg_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ void sub4(float4& a, const float4& x) {
  a.x -= x.x;
  a.y -= x.y;
  a.z -= x.z;
  a.w -= x.w;
}

// One (source, float4) item: C_s[v] = P_r[v] - sum of the listed blocks,
// subtracted in ascending source id.
template <bool kF64, int kB>
__device__ __forceinline__ void peel_item(const DevPlan& p, const float4* P4, float4* C4, long long nv,
                                          int i, long long v) {
  const int s = p.order[i];
  const int r = p.pl_res[i];
  int e = p.pl_ptr[i];
  const int e1 = p.pl_ptr[i + 1];
  const float4 pr = ldg_stream(P4 + static_cast<long long>(r) * nv + v);
  if (!kF64) {
    // kB list entries, then kB independent block loads, then the ascending
    // subtractions: two round trips per kB subtrahends.  kB follows the
    // code's largest degree: wide batches hide latency on deep, sparse
    // waves; narrow ones keep registers low for the wide, bandwidth-bound
    // waves of tall blocks.
    float4 acc = pr;
    for (; e < e1; e += kB) {
      int t[kB];
      float4 x[kB];
#pragma unroll
      for (int q = 0; q < kB; ++q) t[q] = (e + q < e1) ? p.pl_list[e + q] : -1;
#pragma unroll
      for (int q = 0; q < kB; ++q)
        x[q] = t[q] >= 0 ? C4[static_cast<long long>(t[q]) * nv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < kB; ++q)
        if (t[q] >= 0) sub4(acc, x[q]);
    }
    C4[static_cast<long long>(s) * nv + v] = acc;
  } else {
    // Deep chains: subtract in FP64 and round once.
    double ax = pr.x, ay = pr.y, az = pr.z, aw = pr.w;
    for (; e < e1; ++e) {
      const float4 x = C4[p.pl_list[e] * nv + v];
      ax -= x.x;
      ay -= x.y;
      az -= x.z;
      aw -= x.w;
    }
    C4[static_cast<long long>(s) * nv + v] =
        make_float4(static_cast<float>(ax), static_cast<float>(ay), static_cast<float>(az),
                    static_cast<float>(aw));
  }
}

template <int kB>
__device__ __forceinline__ void peel_body(const DevPlan& p, const float* __restrict__ P, float* C,
                                          long long nv, int chunk, int first_wave,
                                          int compensate_depth, long long cta) {
  const int nwaves = p.ctr[CTR_NWAVES];
  const long long v0 = cta * chunk;
  if (v0 >= nv) return;
  const int clen = static_cast<int>(min(static_cast<long long>(chunk), nv - v0));
  const float4* P4 = reinterpret_cast<const float4*>(P);
  float4* C4 = reinterpret_cast<float4*>(C);

  for (int d = first_wave; d <= nwaves; ++d) {
    const int o0 = p.wave_ptr[d - 1], o1 = p.wave_ptr[d];
    const int items = (o1 - o0) * clen;
    const bool comp = compensate_depth >= 0 && d > compensate_depth;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int j = it / clen;
      const long long v = v0 + (it - j * clen);
      if (comp)
        peel_item<true, kB>(p, P4, C4, nv, o0 + j, v);
      else
        peel_item<false, kB>(p, P4, C4, nv, o0 + j, v);
    }
    __syncthreads();
  }
}

template <int kB>
__global__ void __launch_bounds__(kPeelThreads)
peel_kernel(DevPlan p, const float* __restrict__ P, float* C, long long nv, int chunk, int first_wave,
            int compensate_depth) {
  peel_body<kB>(p, P, C, nv, chunk, first_wave, compensate_depth, blockIdx.x);
}

template <int kB>
__global__ void __launch_bounds__(kPeelThreads)
peel_group_kernel(const GJob* __restrict__ jobs, int njobs, int first_wave, int compensate_depth) {
  const long long b = blockIdx.x;
  const int j = find_job(jobs, njobs, b, [](const GJob& J) { return J.peel_base; });
  const GJob& J = jobs[j];
  const long long nv = static_cast<long long>(J.h) * J.N / 4;
  peel_body<kB>(J.p, J.products, J.C, nv, J.peel_chunk, first_wave, compensate_depth, b - J.peel_base);
}

int batch_for(int sigma) { return sigma > 9 ? 16 : (sigma > 5 ? 8 : 4); }

}  // namespace

int peel_chunk_for(long long nv, int ctas_hint) {
  const int target = ctas_hint > 0 ? ctas_hint : 4 * num_sms();
  long long chunk = (nv + target - 1) / target;
  return static_cast<int>(std::max<long long>(8, (chunk + 7) / 8 * 8));
}

cudaError_t launch_peel_group(const GJob* d_jobs, int njobs, long long total_ctas, int first_wave,
                              int compensate_depth, int max_sigma, cudaStream_t st) {
  if (total_ctas <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>(total_ctas);
  switch (batch_for(max_sigma)) {
    case 4: peel_group_kernel<4><<<grid, kPeelThreads, 0, st>>>(d_jobs, njobs, first_wave, compensate_depth); break;
    case 8: peel_group_kernel<8><<<grid, kPeelThreads, 0, st>>>(d_jobs, njobs, first_wave, compensate_depth); break;
    default: peel_group_kernel<16><<<grid, kPeelThreads, 0, st>>>(d_jobs, njobs, first_wave, compensate_depth);
  }
  return cudaGetLastError();
}

cudaError_t launch_peel(const DevGraph& g, const DevPlan& p, const float* P, float* C, int N, int h,
                        int first_wave, int compensate_depth, int ctas, cudaStream_t st) {
  const long long nv = static_cast<long long>(h) * N / 4;
  if (nv <= 0) return cudaSuccess;
  // Every CTA walks every wave, so the grid never exceeds the CTAs that can
  // be resident at once (a CTA waiting for a slot would repeat the chain).
  auto launch = [&](auto kern) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPeelThreads, 0) != cudaSuccess || per_sm <= 0) {
      cudaGetLastError();
      per_sm = 1;
    }
    long long chunk = peel_chunk_for(nv, ctas);
    const long long slots = static_cast<long long>(per_sm) * num_sms();
    if ((nv + chunk - 1) / chunk > slots) chunk = (nv + slots - 1) / slots;
    const unsigned grid = static_cast<unsigned>((nv + chunk - 1) / chunk);
    kern<<<grid, kPeelThreads, 0, st>>>(p, P, C, nv, static_cast<int>(chunk), first_wave, compensate_depth);
  };
  switch (batch_for(g.sigma)) {
    case 4: launch(peel_kernel<4>); break;
    case 8: launch(peel_kernel<8>); break;
    default: launch(peel_kernel<16>);
  }
  return cudaGetLastError();
}

}  // namespace bpx
