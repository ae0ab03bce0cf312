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

// Gathered waves: when a wave's blocks over the CTA's columns fit in shared
// memory (the deep, narrow waves of tall codes with thin blocks), the CTA
// copies every block element the wave reads -- each position's product and
// all its subtrahends -- with cp.async into shared memory at once, so that
// the wave costs one global round trip instead of one per batch of kB
// subtrahends, with no registers held for the loads in flight.  The wave's
// descriptors (list offsets, resolvers, sources, subtrahend lists) were
// staged in shared memory while the previous wave's copies were in flight
// (two descriptor buffers), so they are off the chain from wave to wave.
// Thread t works on column t % clen of the CTA's slice for every position
// and list entry congruent to t / clen.  Wider waves take the register path.
constexpr int kTermCap = 3840;  // float4 block elements of one wave
constexpr int kListCap = 2048;  // subtrahend list entries of one wave
constexpr int kPosCap = 512;    // order positions of one wave
constexpr int kGatherMinSources = 1024;  // codes this tall peel in hundreds of waves
constexpr int kDescInts = kListCap + 3 * kPosCap + 1;  // one descriptor buffer
constexpr size_t kGatherSmem = static_cast<size_t>(kTermCap) * 16 + 2 * static_cast<size_t>(kDescInts) * 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

struct WaveDesc {
  int* list;  // subtrahend sources, relative to the wave's first entry
  int* ptr;   // per position: first list entry (np + 1 values)
  int* res;   // per position: resolving cell
  int* src;   // per position: recovered source
  __device__ WaveDesc(uint8_t* base) {
    list = reinterpret_cast<int*>(base);
    ptr = list + kListCap;
    res = ptr + kPosCap + 1;
    src = res + kPosCap;
  }
};

// Stages the descriptors of order positions [o0, o1) (list entries [l0, l1)).
__device__ __forceinline__ void stage_wave(const DevPlan& p, const WaveDesc& w, int o0, int o1, int l0, int l1) {
  const int np = o1 - o0, nl = l1 - l0;
  for (int t = threadIdx.x; t <= np; t += blockDim.x) w.ptr[t] = p.pl_ptr[o0 + t] - l0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    w.res[t] = p.pl_res[o0 + t];
    w.src[t] = p.order[o0 + t];
  }
  for (int t = threadIdx.x; t < nl; t += blockDim.x) w.list[t] = p.pl_list[l0 + t];
}

// kGather: the launch provides kGatherSmem bytes of dynamic shared memory.
template <int kB, bool kGather>
__device__ __forceinline__ void peel_body(const DevPlan& p, const float* __restrict__ P, float* C,
                                          long long nv, int chunk, int first_wave,
                                          int compensate_depth, long long cta) {
  extern __shared__ __align__(16) uint8_t peel_smem[];
  const int nwaves = p.ctr[CTR_NWAVES];
  const long long v0 = cta * chunk;
  if (v0 >= nv || first_wave > nwaves) return;
  const int clen = static_cast<int>(min(static_cast<long long>(chunk), nv - v0));
  const float4* P4 = reinterpret_cast<const float4*>(P);
  float4* C4 = reinterpret_cast<float4*>(C);
  if constexpr (!kGather) {  // register path only
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
    return;
  }
  float4* s_term = reinterpret_cast<float4*>(peel_smem);
  auto desc = [&](int b) { return WaveDesc(peel_smem + static_cast<size_t>(kTermCap) * 16 + b * (kDescInts * 4)); };
  // this thread's column and its first position / entry (stride G)
  const int col = threadIdx.x % clen, g0 = threadIdx.x / clen;
  const int G = static_cast<int>(blockDim.x) / clen;
  auto fits = [&](int np, int nl) {
    return kGather && clen <= static_cast<int>(blockDim.x) && np <= kPosCap && nl <= kListCap &&
           (np + nl) * clen <= kTermCap;
  };

  int o0 = p.wave_ptr[first_wave - 1], o1 = p.wave_ptr[first_wave];
  int l0 = p.pl_ptr[o0], l1 = p.pl_ptr[o1];
  bool fit = fits(o1 - o0, l1 - l0);
  int buf = 0;
  if (fit) stage_wave(p, desc(0), o0, o1, l0, l1);
  __syncthreads();

  for (int d = first_wave; d <= nwaves; ++d) {
    const bool comp = compensate_depth >= 0 && d > compensate_depth;
    const bool more = d < nwaves;
    const int o2 = more ? p.wave_ptr[d + 1] : o1;
    int l2 = l1;
    bool nfit = false;
    if (fit) {
      const WaveDesc w = desc(buf);
      const int np = o1 - o0, nl = l1 - l0, tp = np * clen;
      // terms [0, np clen): products; list entry e at tp + e clen + column
      if (g0 < G) {
        for (int j = g0; j < np; j += G)
          cp_async16(s_term + j * clen + col, P4 + static_cast<long long>(w.res[j]) * nv + v0 + col);
        for (int e = g0; e < nl; e += G)
          cp_async16(s_term + tp + e * clen + col, C4 + static_cast<long long>(w.list[e]) * nv + v0 + col);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (more) {  // the next wave's descriptors, while the copies fly
        l2 = p.pl_ptr[o2];
        nfit = fits(o2 - o1, l2 - l1);
        if (nfit) stage_wave(p, desc(buf ^ 1), o1, o2, l1, l2);
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
      if (g0 < G) {
        for (int j = g0; j < np; j += G) {
          const int e0 = w.ptr[j], e1 = w.ptr[j + 1];
          const float4* t = s_term + tp + col;
          float4 r;
          if (!comp) {
            r = s_term[j * clen + col];
            for (int e = e0; e < e1; ++e) sub4(r, t[e * clen]);
          } else {
            const float4 pr = s_term[j * clen + col];
            double ax = pr.x, ay = pr.y, az = pr.z, aw = pr.w;
            for (int e = e0; e < e1; ++e) {
              const float4 x = t[e * clen];
              ax -= x.x;
              ay -= x.y;
              az -= x.z;
              aw -= x.w;
            }
            r = make_float4(static_cast<float>(ax), static_cast<float>(ay), static_cast<float>(az),
                            static_cast<float>(aw));
          }
          C4[static_cast<long long>(w.src[j]) * nv + v0 + col] = r;
        }
      }
      __syncthreads();
    } else {
      const int items = (o1 - o0) * clen;
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / clen;
        const long long v = v0 + (it - j * clen);
        if (comp)
          peel_item<true, kB>(p, P4, C4, nv, o0 + j, v);
        else
          peel_item<false, kB>(p, P4, C4, nv, o0 + j, v);
      }
      if (more) {
        l2 = p.pl_ptr[o2];
        nfit = fits(o2 - o1, l2 - l1);
        if (nfit) stage_wave(p, desc(buf ^ 1), o1, o2, l1, l2);
      }
      __syncthreads();
    }
    o0 = o1;
    o1 = o2;
    l0 = l1;
    l1 = l2;
    fit = nfit;
    buf ^= 1;
  }
}

template <int kB, bool kGather>
__global__ void __launch_bounds__(kPeelThreads)
peel_kernel(DevPlan p, const float* __restrict__ P, float* C, long long nv, int chunk, int first_wave,
            int compensate_depth) {
  peel_body<kB, kGather>(p, P, C, nv, chunk, first_wave, compensate_depth, blockIdx.x);
}

template <int kB>
__global__ void __launch_bounds__(kPeelThreads)
peel_group_kernel(const GJob* __restrict__ jobs, int njobs, int first_wave, int compensate_depth) {
  const long long b = blockIdx.x;
  const int j = find_job(jobs, njobs, b, [](const GJob& J) { return J.peel_base; });
  const GJob& J = jobs[j];
  const long long nv = static_cast<long long>(J.h) * J.N / 4;
  peel_body<kB, false>(J.p, J.products, J.C, nv, J.peel_chunk, first_wave, compensate_depth, b - J.peel_base);
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
  // Register path only: a batch runs many short CTAs, and the gather
  // buffer's shared memory would cut how many fit on an SM (measured slower
  // on the 512-job batch: 14.0 vs 9.2 ms).
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
  const bool gather = g.S >= kGatherMinSources;
  const size_t smem = gather ? kGatherSmem : 0;
  auto launch = [&](auto kern) -> cudaError_t {  // kern: a peel_kernel<kB, gather>
    if (gather) {
      const cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPeelThreads, smem) != cudaSuccess ||
        per_sm <= 0) {
      cudaGetLastError();
      per_sm = 1;
    }
    long long chunk = peel_chunk_for(nv, ctas);
    const long long slots = static_cast<long long>(per_sm) * num_sms();
    if ((nv + chunk - 1) / chunk > slots) chunk = (nv + slots - 1) / slots;
    const unsigned grid = static_cast<unsigned>((nv + chunk - 1) / chunk);
    kern<<<grid, kPeelThreads, smem, st>>>(p, P, C, nv, static_cast<int>(chunk), first_wave, compensate_depth);
    return cudaGetLastError();
  };
  switch (batch_for(g.sigma)) {
    case 4: return gather ? launch(peel_kernel<4, true>) : launch(peel_kernel<4, false>);
    case 8: return gather ? launch(peel_kernel<8, true>) : launch(peel_kernel<8, false>);
    default: return gather ? launch(peel_kernel<16, true>) : launch(peel_kernel<16, false>);
  }
}

}  // namespace bpx
