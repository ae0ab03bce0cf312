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

// Compensated subtraction s - x (Knuth's TwoSum of s and -x): t = fl(s - x)
// and its exact rounding error, which is added to the running error term c
// (both FP32, no multiplies, so no contraction can change them).  A chain of
// these ends in one rounding fl(s + c): within about one FP32 rounding of the
// exact result plus a second-order term, on the FP32 pipes (GB300's FP64
// rate is a small fraction of its FP32 rate).
__device__ __forceinline__ void two_sub(float& s, float& c, float x) {
  const float t = s - x;
  const float bp = t - s;
  c += (s - (t - bp)) + (-x - bp);
  s = t;
}

__device__ __forceinline__ void two_sub4(float4& s, float4& c, const float4& x) {
  two_sub(s.x, c.x, x.x);
  two_sub(s.y, c.y, x.y);
  two_sub(s.z, c.z, x.z);
  two_sub(s.w, c.w, x.w);
}

__device__ __forceinline__ float4 two_sum_round(const float4& s, const float4& c) {
  return make_float4(s.x + c.x, s.y + c.y, s.z + c.z, s.w + c.w);
}

// One (source, float4) item: C_s[v] = P_r[v] - sum of the listed blocks,
// subtracted in ascending source id.
template <bool kComp, int kBatch>
__device__ __forceinline__ void peel_item(const DevPlan& p, const float4* P4, float4* C4, long long nv,
                                          int i, long long v) {
  // the compensated form holds a second float4 per item: narrower batches
  // keep the kernel's register count (shared with the plain form) unchanged
  constexpr int kB = kComp ? (kBatch < 4 ? kBatch : 4) : kBatch;
  const int s = p.order[i];
  const int r = p.pl_res[i];
  int e = p.pl_ptr[i];
  const int e1 = p.pl_ptr[i + 1];
  const float4 pr = ldg_stream(P4 + static_cast<long long>(r) * nv + v);
  // kB list entries, then kB independent block loads, then the ascending
  // subtractions: two round trips per kB subtrahends.  kB follows the code's
  // largest degree: wide batches hide latency on deep, sparse waves; narrow
  // ones keep registers low for the wide, bandwidth-bound waves of tall
  // blocks.  Deep chains (kComp) subtract with TwoSum compensation.
  float4 acc = pr, err = make_float4(0.f, 0.f, 0.f, 0.f);
  for (; e < e1; e += kB) {
    int t[kB];
    float4 x[kB];
#pragma unroll
    for (int q = 0; q < kB; ++q) t[q] = (e + q < e1) ? p.pl_list[e + q] : -1;
#pragma unroll
    for (int q = 0; q < kB; ++q)
      x[q] = t[q] >= 0 ? C4[static_cast<long long>(t[q]) * nv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kB; ++q) {
      if (t[q] < 0) continue;
      if (kComp)
        two_sub4(acc, err, x[q]);
      else
        sub4(acc, x[q]);
    }
  }
  C4[static_cast<long long>(s) * nv + v] = kComp ? two_sum_round(acc, err) : acc;
}

// Gathered waves (tall codes with thin blocks: hundreds of deep, narrow
// waves).  The CTA copies every block element a wave reads -- each
// position's product and all its subtrahends over the CTA's columns -- with
// cp.async into shared memory at once, so that the wave costs one global
// round trip instead of one per batch of kB subtrahends, with no registers
// held for the loads in flight.  A wave whose rows exceed the term buffer
// runs in rounds over runs of its positions (positions of one wave never
// read each other).  The descriptors of the next wave (list offsets,
// resolvers, sources, subtrahend lists) are copied into the second of two
// descriptor buffers with cp.async along with the current wave's first
// round, and the two scalars that bound them (its first order position and
// first list entry) are loaded one wave earlier still, so no dependent load
// sits on the chain from wave to wave.  Thread t works on column t % clen of
// the CTA's slice for every position and list entry congruent to t / clen.
// Waves with more positions or list entries than the descriptor buffers hold
// take the register path.
constexpr int kTermCap = 5632;       // float4 block elements of one round (88 KB): one job
constexpr int kTermCapGroup = 3200;  // grouped launches (50 KB): three CTAs per SM for the many chains
constexpr int kListCap = 2048;  // subtrahend list entries of one wave
constexpr int kPosCap = 256;    // order positions of one wave
constexpr int kGatherMinSources = 1024;  // codes this tall peel in hundreds of waves
constexpr int kDescInts = kListCap + 3 * kPosCap + 1;  // one descriptor buffer
// dynamic shared memory of the gathered form: 110 KB for one job (two CTAs
// per SM), 72 KB for grouped launches (three)
constexpr size_t gather_smem(int cap) { return static_cast<size_t>(cap) * 16 + 2 * static_cast<size_t>(kDescInts) * 4; }
constexpr size_t kGatherSmem = gather_smem(kTermCap);
constexpr size_t kGatherSmemGroup = gather_smem(kTermCapGroup);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}

struct WaveDesc {
  int* list;  // subtrahend sources, from the wave's first list entry on
  int* ptr;   // per position: first list entry, absolute (np + 1 values)
  int* res;   // per position: resolving cell
  int* src;   // per position: recovered source
  __device__ WaveDesc(uint8_t* base) {
    list = reinterpret_cast<int*>(base);
    ptr = list + kListCap;
    res = ptr + kPosCap + 1;
    src = res + kPosCap;
  }
};

// Starts the copies of the descriptors of order positions [o0, o1) (list
// entries [l0, l1)); they land with the caller's next cp.async.wait_all.
__device__ __forceinline__ void stage_wave(const DevPlan& p, const WaveDesc& w, int o0, int o1, int l0, int l1) {
  const int np = o1 - o0, nl = l1 - l0;
  for (int t = threadIdx.x; t <= np; t += blockDim.x) cp_async4(w.ptr + t, p.pl_ptr + o0 + t);
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    cp_async4(w.res + t, p.pl_res + o0 + t);
    cp_async4(w.src + t, p.order + o0 + t);
  }
  for (int t = threadIdx.x; t < nl; t += blockDim.x) cp_async4(w.list + t, p.pl_list + l0 + t);
}

// kGather: the launch provides gather_smem(kCap) bytes of dynamic shared
// memory, and sigma * chunk <= kCap (one position's rows fit a round).
template <int kB, bool kGather, int kCap = kTermCap>
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
  auto desc = [&](int b) { return WaveDesc(peel_smem + static_cast<size_t>(kCap) * 16 + b * (kDescInts * 4)); };
  // this thread's column and its first position / entry (stride G)
  const int col = threadIdx.x % clen, g0 = threadIdx.x / clen;
  const int G = static_cast<int>(blockDim.x) / clen;
  const int cap = kCap / clen;  // block rows of one round
  auto fits = [&](int np, int nl) {
    return clen <= static_cast<int>(blockDim.x) && np <= kPosCap && nl <= kListCap;
  };

  // wave d spans order positions [o0, o1) and list entries [l0, l1); wave
  // d + 1 ends at (o2, l2)
  int o0 = p.wave_ptr[first_wave - 1], o1 = p.wave_ptr[first_wave];
  int l0 = p.pl_ptr[o0], l1 = p.pl_ptr[o1];
  int o2 = first_wave < nwaves ? p.wave_ptr[first_wave + 1] : o1;
  int l2 = p.pl_ptr[o2];
  bool fit = fits(o1 - o0, l1 - l0);
  int buf = 0;
  if (fit) stage_wave(p, desc(0), o0, o1, l0, l1);
  asm volatile("cp.async.wait_all;" ::: "memory");  // commit + wait for every copy issued
  __syncthreads();

  for (int d = first_wave; d <= nwaves; ++d) {
    const bool comp = compensate_depth >= 0 && d > compensate_depth;
    const bool more = d < nwaves;
    const int o3 = d + 1 < nwaves ? p.wave_ptr[d + 2] : o2;  // wave d + 2, consumed after this wave
    const bool nfit = more && fits(o2 - o1, l2 - l1);
    if (fit) {
      const WaveDesc w = desc(buf);
      const int np = o1 - o0;
      // Rounds over runs of positions [j0, j1) whose product and subtrahend
      // rows fit the term buffer; one round when the whole wave fits.
      for (int j0 = 0, round = 0; round == 0 || j0 < np; ++round) {
        int j1 = min(j0 + 1, np);
        while (j1 < np && (j1 + 1 - j0) + (w.ptr[j1 + 1] - w.ptr[j0]) <= cap) ++j1;
        const int e0 = w.ptr[j0], e1 = w.ptr[j1], tp = (j1 - j0) * clen;
        // terms [0, tp): products; list entry e at tp + (e - e0) clen + column
        if (g0 < G) {
          for (int j = j0 + g0; j < j1; j += G)
            cp_async16(s_term + (j - j0) * clen + col, P4 + static_cast<long long>(w.res[j]) * nv + v0 + col);
          for (int e = e0 + g0; e < e1; e += G)
            cp_async16(s_term + tp + (e - e0) * clen + col,
                       C4 + static_cast<long long>(w.list[e - l0]) * nv + v0 + col);
        }
        if (round == 0 && nfit) stage_wave(p, desc(buf ^ 1), o1, o2, l1, l2);  // with the copies
        asm volatile("cp.async.wait_all;" ::: "memory");  // commit + wait for every copy issued
        __syncthreads();
        if (g0 < G) {
          const float4* t = s_term + tp + col;
          for (int j = j0 + g0; j < j1; j += G) {
            const int f0 = w.ptr[j] - e0, f1 = w.ptr[j + 1] - e0;
            float4 r;
            if (!comp) {
              r = s_term[(j - j0) * clen + col];
              for (int e = f0; e < f1; ++e) sub4(r, t[e * clen]);
            } else {
              float4 err = make_float4(0.f, 0.f, 0.f, 0.f);
              r = s_term[(j - j0) * clen + col];
              for (int e = f0; e < f1; ++e) two_sub4(r, err, t[e * clen]);
              r = two_sum_round(r, err);
            }
            C4[static_cast<long long>(w.src[j]) * nv + v0 + col] = r;
          }
        }
        __syncthreads();
        j0 = j1;
      }
    } else {
      if (nfit) stage_wave(p, desc(buf ^ 1), o1, o2, l1, l2);
      const int items = (o1 - o0) * clen;
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / clen;
        const long long v = v0 + (it - j * clen);
        if (comp)
          peel_item<true, kB>(p, P4, C4, nv, o0 + j, v);
        else
          peel_item<false, kB>(p, P4, C4, nv, o0 + j, v);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");  // commit + wait for every copy issued
      __syncthreads();
    }
    const int l3 = p.pl_ptr[o3];
    o0 = o1;
    o1 = o2;
    o2 = o3;
    l0 = l1;
    l1 = l2;
    l2 = l3;
    fit = nfit;
    buf ^= 1;
  }
}

template <int kB, bool kGather>
__global__ void __launch_bounds__(kPeelThreads)
peel_kernel(DevPlan p, const float* __restrict__ P, float* C, long long nv, int chunk, int first_wave,
            int compensate_depth) {
  if (p.ctr[CTR_PLAN] != kPlanReady) {  // no schedule has planned this workspace: refuse, write nothing
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicExch(&p.info[BPX_INFO_DEVICE_ERR], BPX_ERR_INVAL);
      atomicExch(&p.info[BPX_INFO_STATUS], BPX_ERR_INVAL);
    }
    return;
  }
  peel_body<kB, kGather>(p, P, C, nv, chunk, first_wave, compensate_depth, blockIdx.x);
}

// A grouped peel launch over the jobs order[0 .. n): their CTA ranges lie
// end to end from `base` on, job order[i] from bases[i].
template <int kB, bool kGather>
__global__ void __launch_bounds__(kPeelThreads)
peel_group_kernel(const GJob* __restrict__ jobs, const int32_t* __restrict__ order,
                  const long long* __restrict__ bases, int n, long long base, int first_wave,
                  int compensate_depth) {
  const long long b = base + blockIdx.x;
  const int i = find_base(bases, n, b);
  const GJob& J = jobs[order[i]];
  const long long nv = static_cast<long long>(J.h) * J.N / 4;
  peel_body<kB, kGather, kTermCapGroup>(J.p, J.products, J.C, nv, J.peel_chunk, first_wave, compensate_depth,
                                        b - __ldg(bases + i));
}

int batch_for(int sigma) { return sigma > 9 ? 16 : (sigma > 5 ? 8 : 4); }

}  // namespace

int peel_chunk_for(long long nv, int ctas_hint) {
  const int target = ctas_hint > 0 ? ctas_hint : 4 * num_sms();
  long long chunk = (nv + target - 1) / target;
  return static_cast<int>(std::max<long long>(8, (chunk + 7) / 8 * 8));
}

bool peel_gather_ok(int S, int sigma, long long chunk) {
  return S >= kGatherMinSources && chunk <= kPeelThreads &&
         static_cast<long long>(std::max(1, sigma)) * chunk <= kTermCapGroup;
}

cudaError_t launch_peel_group(const GJob* d_jobs, const int32_t* d_order, const long long* d_bases, int njobs,
                              int ngather, long long gather_ctas, long long total_ctas, int first_wave,
                              int compensate_depth, int max_sigma, cudaStream_t st, cudaStream_t side,
                              cudaEvent_t fork, cudaEvent_t join) {
  if (total_ctas <= 0) return cudaSuccess;
  const long long reg_ctas = total_ctas - gather_ctas;
  const bool both = gather_ctas > 0 && reg_ctas > 0;
  // The register launch goes to the side stream when both run, so that its
  // short CTAs fill the slots the gather CTAs' shared memory leaves free.
  cudaError_t e;
  if (both) {
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
  }
  auto go = [&](auto gather_kern, auto reg_kern) -> cudaError_t {
    if (gather_ctas > 0) {
      cudaError_t r = cudaFuncSetAttribute(gather_kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(kGatherSmemGroup));
      if (r != cudaSuccess) return r;
      gather_kern<<<static_cast<unsigned>(gather_ctas), kPeelThreads, kGatherSmemGroup, st>>>(
          d_jobs, d_order, d_bases, ngather, 0, first_wave, compensate_depth);
      if ((r = cudaGetLastError()) != cudaSuccess) return r;
    }
    if (reg_ctas > 0) {
      reg_kern<<<static_cast<unsigned>(reg_ctas), kPeelThreads, 0, both ? side : st>>>(
          d_jobs, d_order + ngather, d_bases + ngather, njobs - ngather, gather_ctas, first_wave,
          compensate_depth);
      return cudaGetLastError();
    }
    return cudaSuccess;
  };
  switch (batch_for(max_sigma)) {
    case 4: e = go(peel_group_kernel<4, true>, peel_group_kernel<4, false>); break;
    case 8: e = go(peel_group_kernel<8, true>, peel_group_kernel<8, false>); break;
    default: e = go(peel_group_kernel<16, true>, peel_group_kernel<16, false>);
  }
  if (e != cudaSuccess) return e;
  if (both) {
    if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_peel(const DevGraph& g, const DevPlan& p, const float* P, float* C, int N, int h,
                        int first_wave, int compensate_depth, int ctas, cudaStream_t st) {
  const long long nv = static_cast<long long>(h) * N / 4;
  if (nv <= 0) return cudaSuccess;
  // Every CTA walks every wave, so the grid never exceeds the CTAs that can
  // be resident at once (a CTA waiting for a slot would repeat the chain).
  // The CTA count: the hint's (default 4 per SM), capped at the CTAs that
  // can be resident at once for the kernel's shared memory.
  auto chunk_for = [&](auto kern, size_t smem, long long* chunk) -> cudaError_t {
    if (smem) {
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
    *chunk = peel_chunk_for(nv, ctas);
    const long long slots = static_cast<long long>(per_sm) * num_sms();
    if ((nv + *chunk - 1) / *chunk > slots) *chunk = (nv + slots - 1) / slots;
    return cudaSuccess;
  };
  auto run = [&](auto kern, size_t smem, long long chunk) -> cudaError_t {
    const unsigned grid = static_cast<unsigned>((nv + chunk - 1) / chunk);
    kern<<<grid, kPeelThreads, smem, st>>>(p, P, C, nv, static_cast<int>(chunk), first_wave, compensate_depth);
    return cudaGetLastError();
  };
  // The gathered form for tall codes, when one position's rows (at most
  // sigma) over the CTA's columns fit a round of the term buffer.
  auto go = [&](auto gather_kern, auto reg_kern) -> cudaError_t {
    long long chunk = 0;
    cudaError_t e;
    if (g.S >= kGatherMinSources) {
      if ((e = chunk_for(gather_kern, kGatherSmem, &chunk)) != cudaSuccess) return e;
      if (static_cast<long long>(std::max(1, g.sigma)) * chunk <= kTermCap) return run(gather_kern, kGatherSmem, chunk);
    }
    if ((e = chunk_for(reg_kern, 0, &chunk)) != cudaSuccess) return e;
    return run(reg_kern, 0, chunk);
  };
  switch (batch_for(g.sigma)) {
    case 4: return go(peel_kernel<4, true>, peel_kernel<4, false>);
    case 8: return go(peel_kernel<8, true>, peel_kernel<8, false>);
    default: return go(peel_kernel<16, true>, peel_kernel<16, false>);
  }
}

}  // namespace bpx
