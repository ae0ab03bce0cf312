// a3, MXFP8 path on the 5th-generation tensor cores: block-scaled
// tcgen05.mma kind::mxf8f6f4 over the E4M3 operands and UE8M0 scales written
// by the MXFP8 encode and B kernels.
#include <algorithm>

#include "tc_common.cuh"

namespace bpx {
namespace {

// ---- MXFP8 (E4M3 x E4M3, UE8M0 scale per 32 K-elements) --------------------
//
// Same warp roles as the bf16 kernel, 128 x 256 tiles, 128-wide K stages
// (one 128-byte swizzle row of fp8).  Each stage also carries the tile's
// scale blocks (512 B for A, 1 KB for B) fetched by a bulk copy; the MMA
// thread moves them into tensor memory with tcgen05.cp (32 lanes x 16 bytes,
// replicated to the four lane quarters), then issues four block-scaled MMAs
// (K = 32 each) whose scale-factor ids pick the byte of the stage's 32-run.
// Tensor memory: one 256-column accumulator + 12 scale columns per stage.
constexpr int kMxBK = 128;
constexpr int kMxStages = 4;
constexpr int kMxBN = 256;
constexpr uint32_t kMxA = BM * kMxBK;      // 16 KB
constexpr uint32_t kMxB = kMxBN * kMxBK;   // 32 KB
constexpr uint32_t kMxSfa = kMxA + kMxB;   // 512 B of A scales
constexpr uint32_t kMxSfb = kMxSfa + 512;  // 1 KB of B scales
constexpr uint32_t kMxStageBytes = 51200;  // 50 KB (data + scales, 1 KB aligned)
constexpr uint32_t kMxTx = kMxA + kMxB + 512 + 1024;
constexpr int kMxSfCol = 256;              // first TMEM column of the scale slots

struct MxParams {
  const uint8_t* sfa;
  const uint8_t* sfb;
  const int32_t* ctr;
  const int32_t* surv;
  const int32_t* direct;
  int32_t* info;
  int32_t* info_out;
  float* products;
  float* C_direct;
  int N, K, h, m_tiles_max, n_tiles, group;
};

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// No-swizzle descriptor of a 32-row x 16-byte tile (8-row groups 128 B apart).
__device__ __forceinline__ uint64_t sdesc_rows16(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFF) >> 4);
  d |= static_cast<uint64_t>(128 >> 4) << 16;
  d |= static_cast<uint64_t>(128 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

__device__ __forceinline__ void tmem_cp_32x128(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

// kind::mxf8f6f4 instruction descriptor: A = B = E4M3, UE8M0 scales, K-major,
// M = 128, N = 256, scale-factor ids a_id / b_id.
__device__ __forceinline__ uint32_t idesc_mx(uint32_t id) {
  return (id << 4) | (static_cast<uint32_t>(kMxBN >> 3) << 17) | (1u << 23) |
         (static_cast<uint32_t>(BM >> 4) << 24) | (id << 29);
}

__device__ __forceinline__ void umma_mx(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sfa,
                                        uint32_t sfb, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc));
}

// Streaming (.cs) output stores: written once, they should not push the
// operand tiles other CTAs still read out of L2.
__device__ __forceinline__ void st_cs4_mx(float* p, float a, float b, float c, float d) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void raise_mx(const MxParams& P, int code, volatile int* abort_flag) {
  *abort_flag = 1;
  atomicExch(&P.info[BPX_INFO_DEVICE_ERR], code);
  atomicExch(&P.info[BPX_INFO_STATUS], code);
  if (P.info_out) {
    atomicExch(&P.info_out[BPX_INFO_DEVICE_ERR], code);
    atomicExch(&P.info_out[BPX_INFO_STATUS], code);
  }
}

// One CTA per 128 x 256 tile.
__global__ void __launch_bounds__(kThreads, 1)
gemm_mx_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
               const __grid_constant__ MxParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kMxStages], empty_bar[kMxStages];
  __shared__ __align__(8) uint64_t dfull_bar, dempty_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Mc = P.ctr[CTR_NSURV] * P.h;
  const int m_tiles = (Mc + BM - 1) / BM;
  const int m_units = m_tiles;
  const int num_tiles = m_units * P.n_tiles;
  const int k_blocks = P.K / kMxBK;
  const int KS = k_blocks;
  const int cid = static_cast<int>(blockIdx.x);
  const int nclusters = static_cast<int>(gridDim.x);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kMxStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&dfull_bar), 1);
    mbar_init(smem_u32(&dempty_bar), 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  // (m, n) of tile t in bands of m-tiles
  auto tile_mn = [&](long long t, int& m, int& n) {
    const int band_tiles = P.group * P.n_tiles;
    const int band = static_cast<int>(t / band_tiles);
    const int r = static_cast<int>(t - static_cast<long long>(band) * band_tiles);
    const int rows_in_band = min(P.group, m_units - band * P.group);
    m = band * P.group + r % rows_in_band;
    n = r / rows_in_band;
  };

  if (warp == 0) {
    if (lane == 0) {
      int kb_all = 0;
      bool ok = true;
      for (long long j = 0; ok; ++j) {
        const long long t = snake(j, cid, nclusters);
        if (t >= num_tiles) break;
        int mt, nt;
        tile_mn(t, mt, nt);
        for (int kb = 0; kb < k_blocks; ++kb, ++kb_all) {
          const int s = kb_all % kMxStages;
          if (!mbar_wait(smem_u32(&empty_bar[s]), static_cast<uint32_t>((kb_all / kMxStages) & 1) ^ 1u,
                         &abort_flag)) {
            if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          const uint32_t base = smem_u32(smem + s * kMxStageBytes);
          const uint32_t fb = smem_u32(&full_bar[s]);
          mbar_expect_tx(fb, kMxTx);
          tma_load_2d(base, &map_a, fb, kb * kMxBK, mt * BM);
          tma_load_2d(base + kMxA, &map_b, fb, kb * kMxBK, nt * kMxBN);
          bulk_load(base + kMxSfa, P.sfa + (static_cast<long long>(mt) * KS + kb) * 512, 512, fb);
          bulk_load(base + kMxSfb, P.sfb + (static_cast<long long>(nt) * KS + kb) * 1024, 1024, fb);
        }
      }
      if (!ok || abort_flag) {
        for (int i = 0; i < kMxStages && i < kb_all; ++i) {
          const int kb = kb_all - 1 - i;
          mbar_wait(smem_u32(&full_bar[kb % kMxStages]), static_cast<uint32_t>((kb / kMxStages) & 1), nullptr);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int kb_all = 0, it = 0;
      bool ok = true;
      for (long long j = 0; ok; ++j, ++it) {
        const long long t = snake(j, cid, nclusters);
        if (t >= num_tiles) break;
        if (!mbar_wait(smem_u32(&dempty_bar), static_cast<uint32_t>(it & 1) ^ 1u, &abort_flag)) {
          if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
          break;
        }
        fence_after();
        for (int kb = 0; kb < k_blocks; ++kb, ++kb_all) {
          const int s = kb_all % kMxStages;
          if (!mbar_wait(smem_u32(&full_bar[s]), static_cast<uint32_t>((kb_all / kMxStages) & 1), &abort_flag)) {
            if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t base = smem_u32(smem + s * kMxStageBytes);
          const uint32_t sf = tmem_base + static_cast<uint32_t>(kMxSfCol + 12 * s);
          tmem_cp_32x128(sf, sdesc_rows16(base + kMxSfa));
          tmem_cp_32x128(sf + 4, sdesc_rows16(base + kMxSfb));
          tmem_cp_32x128(sf + 8, sdesc_rows16(base + kMxSfb + 512));
          const uint64_t ad = sdesc_sw128(base), bd = sdesc_sw128(base + kMxA);
#pragma unroll
          for (int kk = 0; kk < kMxBK / 32; ++kk) {
            const uint64_t adv = static_cast<uint64_t>(kk * 32) >> 4;  // 32 fp8 = 32 B
            umma_mx(tmem_base, ad + adv, bd + adv, idesc_mx(kk), sf, sf + 4, (kb == 0 && kk == 0) ? 0u : 1u);
          }
          umma_commit(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&dfull_bar));
      }
    }
  } else {
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int row = quarter * 32 + lane;
    int it = 0;
    for (long long j = 0;; ++j, ++it) {
      const long long t = snake(j, cid, nclusters);
      if (t >= num_tiles) break;
      if (!mbar_wait(smem_u32(&dfull_bar), static_cast<uint32_t>(it & 1), &abort_flag)) {
        if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
        break;
      }
      fence_after();
      // drain the single accumulator quickly (four loads, one wait): the
      // next tile's MMAs wait for it
      float accum[128];
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(half * 128);
      {
        uint32_t r[4][32];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld32_nowait(taddr + c * 32, r[c]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int i = 0; i < 32; ++i) accum[c * 32 + i] = __uint_as_float(r[c][i]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&dempty_bar));
      int mt, nt;
      tile_mn(t, mt, nt);
      const int r = mt * BM + row;
      if (r < Mc) {
        const int ci = r / P.h;
        const int j = r - ci * P.h;
        const int cell = P.surv[ci];
        const int ds = P.C_direct ? P.direct[cell] : -1;
        float* dst = ds >= 0 ? P.C_direct + (static_cast<long long>(ds) * P.h + j) * P.N
                             : P.products + (static_cast<long long>(cell) * P.h + j) * P.N;
        const int n0 = nt * kMxBN + half * 128;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int n = n0 + 4 * q;
          if (n < P.N)
            st_cs4_mx(dst + n, accum[4 * q], accum[4 * q + 1], accum[4 * q + 2], accum[4 * q + 3]);
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}

// 2-D K-major byte tensor map (E4M3 operands): rows x K bytes, box = box_rows
// x 128 with 128 B swizzle.
// ---- CTA-pair MXFP8 (cta_group::2) ---------------------------------------
//
// The two CTAs of a cluster compute one 256 x 256 tile: each stages its own
// 128 rows of A and half of the B tile (128 rows of B^T), its own 128 rows'
// A scales and the whole tile's B scales (every CTA's accumulator spans all
// 256 columns).  All of a stage's copies are TMA loads (the scale blocks
// through 2-D tensor maps of 32-bit words) that complete on the even CTA's
// stage barrier, armed there for both CTAs' bytes.  The even CTA's MMA thread
// copies each CTA's scale blocks into that CTA's tensor memory
// (tcgen05.cp.cta_group::2) and issues the M = 256 block-scaled MMAs for the
// pair; its commits arrive on both CTAs' barriers, and the odd CTA's
// epilogue warps arrive on the even CTA's accumulator-drained barrier.
// A CTA stages a third less operand data per MMA than in the 1-CTA kernel,
// and the pair shares each B tile's L2 reads.
constexpr int kMxpStages = 6;
constexpr uint32_t kMxpA = BM * kMxBK;                 // 16 KB
constexpr uint32_t kMxpB = (kMxBN / 2) * kMxBK;        // 16 KB: half of the B tile
constexpr uint32_t kMxpSfa = kMxpA + kMxpB;            // 512 B of A scales (own rows)
constexpr uint32_t kMxpSfb = kMxpSfa + 512;            // 1 KB of B scales (the whole tile)
constexpr uint32_t kMxpTx = kMxpSfb + 1024;            // bytes one CTA stages
constexpr uint32_t kMxpStageBytes = 34816;             // 34 KB, 1 KB aligned

__device__ __forceinline__ void tmem_cp_32x128_pair(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::2.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

// kind::mxf8f6f4, M = 256 (128 rows in each CTA of the pair), N = 256.
__device__ __forceinline__ uint32_t idesc_mx_pair(uint32_t id) {
  return (id << 4) | (static_cast<uint32_t>(kMxBN >> 3) << 17) | (1u << 23) |
         (static_cast<uint32_t>((2 * BM) >> 4) << 24) | (id << 29);
}

__device__ __forceinline__ void umma_mx_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t sfa,
                                             uint32_t sfb, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc));
}

__global__ void __launch_bounds__(kThreads, 1)
gemm_mx_pair_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                    const __grid_constant__ CUtensorMap map_sfa, const __grid_constant__ CUtensorMap map_sfb,
                    const __grid_constant__ MxParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kMxpStages], empty_bar[kMxpStages];
  __shared__ __align__(8) uint64_t dfull_bar, dempty_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Mc = P.ctr[CTR_NSURV] * P.h;
  const int m_tiles = (Mc + BM - 1) / BM;
  const int m_units = (m_tiles + 1) / 2;
  const int num_tiles = m_units * P.n_tiles;
  const int k_blocks = P.K / kMxBK;
  const int KS = k_blocks;
  const uint32_t rank = cluster_rank();
  const int cid = static_cast<int>(blockIdx.x >> 1);
  const int nclusters = static_cast<int>(gridDim.x >> 1);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kMxpStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&dfull_bar), 1);
    mbar_init(smem_u32(&dempty_bar), 16);  // both CTAs' epilogue warps
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {  // both CTAs of the pair allocate together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  cluster_sync();  // the peer's barriers exist before any copy or commit lands
  fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  // (pair unit, n) of tile t in bands of pair units; this CTA's m-tile
  auto tile_mn = [&](long long t, int& m, int& n) {
    const int band_tiles = P.group * P.n_tiles;
    const int band = static_cast<int>(t / band_tiles);
    const int r = static_cast<int>(t - static_cast<long long>(band) * band_tiles);
    const int rows_in_band = min(P.group, m_units - band * P.group);
    m = 2 * (band * P.group + r % rows_in_band) + static_cast<int>(rank);
    n = r / rows_in_band;
  };

  if (warp == 0) {
    if (lane == 0) {
      int kb_all = 0;
      bool ok = true;
      for (long long j = 0; ok; ++j) {
        const long long t = snake(j, cid, nclusters);
        if (t >= num_tiles) break;
        int mt, nt;
        tile_mn(t, mt, nt);
        for (int kb = 0; kb < k_blocks; ++kb, ++kb_all) {
          const int s = kb_all % kMxpStages;
          if (!mbar_wait(smem_u32(&empty_bar[s]), static_cast<uint32_t>((kb_all / kMxpStages) & 1) ^ 1u,
                         &abort_flag)) {
            if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          const uint32_t base = smem_u32(smem + s * kMxpStageBytes);
          const uint32_t fb = smem_u32(&full_bar[s]);
          const uint32_t fb0 = mapa_rank(fb, 0);
          if (rank == 0) mbar_expect_tx(fb, 2 * kMxpTx);
          tma_load_2d_pair(base, &map_a, fb0, kb * kMxBK, mt * BM);
          tma_load_2d_pair(base + kMxpA, &map_b, fb0, kb * kMxBK, nt * kMxBN + static_cast<int>(rank) * (kMxBN / 2));
          tma_load_2d_pair(base + kMxpSfa, &map_sfa, fb0, 0, mt * KS + kb);
          tma_load_2d_pair(base + kMxpSfb, &map_sfb, fb0, 0, nt * KS + kb);
        }
      }
      if ((!ok || abort_flag) && rank == 0) {
        // Stopping early: the copies in flight (both CTAs' count here) land
        // before shared memory goes away (bounded waits, abort ignored).
        for (int i = 0; i < kMxpStages && i < kb_all; ++i) {
          const int kb = kb_all - 1 - i;
          mbar_wait(smem_u32(&full_bar[kb % kMxpStages]), static_cast<uint32_t>((kb / kMxpStages) & 1), nullptr);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {  // the even CTA issues for the pair
      int kb_all = 0, it = 0;
      bool ok = true;
      for (long long j = 0; ok; ++j, ++it) {
        const long long t = snake(j, cid, nclusters);
        if (t >= num_tiles) break;
        if (!mbar_wait(smem_u32(&dempty_bar), static_cast<uint32_t>(it & 1) ^ 1u, &abort_flag)) {
          if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
          break;
        }
        fence_after();
        for (int kb = 0; kb < k_blocks; ++kb, ++kb_all) {
          const int s = kb_all % kMxpStages;
          if (!mbar_wait(smem_u32(&full_bar[s]), static_cast<uint32_t>((kb_all / kMxpStages) & 1), &abort_flag)) {
            if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t base = smem_u32(smem + s * kMxpStageBytes);
          const uint32_t sf = tmem_base + static_cast<uint32_t>(kMxSfCol + 12 * s);
          tmem_cp_32x128_pair(sf, sdesc_rows16(base + kMxpSfa));
          tmem_cp_32x128_pair(sf + 4, sdesc_rows16(base + kMxpSfb));
          tmem_cp_32x128_pair(sf + 8, sdesc_rows16(base + kMxpSfb + 512));
          const uint64_t ad = sdesc_sw128(base), bd = sdesc_sw128(base + kMxpA);
#pragma unroll
          for (int kk = 0; kk < kMxBK / 32; ++kk) {
            const uint64_t adv = static_cast<uint64_t>(kk * 32) >> 4;  // 32 fp8 = 32 B
            umma_mx_pair(tmem_base, ad + adv, bd + adv, idesc_mx_pair(kk), sf, sf + 4,
                         (kb == 0 && kk == 0) ? 0u : 1u);
          }
          umma_commit_pair(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        umma_commit_pair(smem_u32(&dfull_bar));
      }
    }
  } else {
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int row = quarter * 32 + lane;
    int it = 0;
    for (long long j = 0;; ++j, ++it) {
      const long long t = snake(j, cid, nclusters);
      if (t >= num_tiles) break;
      if (!mbar_wait(smem_u32(&dfull_bar), static_cast<uint32_t>(it & 1), &abort_flag)) {
        if (!abort_flag) raise_mx(P, BPX_ERR_TIMEOUT, &abort_flag);
        break;
      }
      fence_after();
      float accum[128];
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(half * 128);
      {
        uint32_t r[4][32];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld32_nowait(taddr + c * 32, r[c]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int i = 0; i < 32; ++i) accum[c * 32 + i] = __uint_as_float(r[c][i]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(mapa_rank(smem_u32(&dempty_bar), 0));
      int mt, nt;
      tile_mn(t, mt, nt);
      const int r = mt * BM + row;
      if (r < Mc) {
        const int ci = r / P.h;
        const int jj = r - ci * P.h;
        const int cell = P.surv[ci];
        const int ds = P.C_direct ? P.direct[cell] : -1;
        float* dst = ds >= 0 ? P.C_direct + (static_cast<long long>(ds) * P.h + jj) * P.N
                             : P.products + (static_cast<long long>(cell) * P.h + jj) * P.N;
        const int n0 = nt * kMxBN + half * 128;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int n = n0 + 4 * q;
          if (n < P.N)
            st_cs4_mx(dst + n, accum[4 * q], accum[4 * q + 1], accum[4 * q + 2], accum[4 * q + 3]);
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  cluster_sync();  // no CTA leaves while its peer may still read or write into it
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}

// 2-D map over scale blocks stored as rows of `words` 32-bit words (one
// block per row: (tile, 128-wide K stage) in the order the GEMM copies them).
bool make_map_words(CUtensorMap* map, const void* base, long long rows, int words) {
  auto enc = get_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(words), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(words) * 4};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(words), 1};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_map_u8(CUtensorMap* map, const void* base, long long rows, int K, int box_rows) {
  auto enc = get_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(K)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kMxBK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_gemm_mx(const DevPlan& p, const void* a8, const void* sfa, const void* b8, const void* sfb,
                           int num_cells, int N, int K, int h, float* products, float* C_direct, int config,
                           int32_t* info_out, cudaStream_t st) {
  if (K % kMxBK != 0) return cudaErrorInvalidValue;
  const long long rows = static_cast<long long>(num_cells) * h;
  CUtensorMap ma, mb;
  // config: band * 1000 + tile code; codes 9 and 0: 256 x 256 tiles of
  // CTA-pair MMAs (gemm_mx_pair_kernel; the default, config 0, is 16009, the
  // fastest measured: GEMM 0.501 ms on the benchmark against 0.533 ms for
  // 1-CTA MMAs); codes 1, 2, 5, 6: 128 x 256 tiles of 1-CTA MMAs
  if (!gemm_config_ok(config)) return cudaErrorInvalidValue;
  if (config == 0) config = 16009;
  const int tc = config % 10;
  const bool cta_pair = tc == 9 || tc == 0;
  if (!make_map_u8(&ma, a8, rows, K, BM) || !make_map_u8(&mb, b8, N, K, cta_pair ? kMxBN / 2 : kMxBN))
    return cudaErrorInvalidValue;
  MxParams P;
  P.sfa = static_cast<const uint8_t*>(sfa);
  P.sfb = static_cast<const uint8_t*>(sfb);
  P.ctr = p.ctr;
  P.surv = p.surv;
  P.direct = p.direct;
  P.info = p.info;
  P.info_out = info_out;
  P.products = products;
  P.C_direct = C_direct;
  P.N = N;
  P.K = K;
  P.h = h;
  P.m_tiles_max = static_cast<int>((rows + BM - 1) / BM);
  P.n_tiles = (N + kMxBN - 1) / kMxBN;
  P.group = config >= 1000 ? config / 1000 : 8;
  if (cta_pair) {
    // scale blocks as rows of 32-bit words: A 128 words per (m-tile, stage)
    // over an even number of m-tiles (the workspace pads to whole pairs), B
    // 256 words per (n-tile, stage)
    const int KS = K / kMxBK;
    CUtensorMap msa, msb;
    const long long a_tiles = (rows + 2 * BM - 1) / (2 * BM) * 2;
    if (!make_map_words(&msa, sfa, a_tiles * KS, 128) ||
        !make_map_words(&msb, sfb, static_cast<long long>(P.n_tiles) * KS, 256))
      return cudaErrorInvalidValue;
    const size_t smem2 = static_cast<size_t>(kMxpStages) * kMxpStageBytes + 1024;
    auto kern = gemm_mx_pair_kernel;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem2));
    if (e != cudaSuccess) return e;
    const long long pairs = ((P.m_tiles_max + 1) / 2) * static_cast<long long>(P.n_tiles);
    if (pairs <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem2;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * (num_sms() / 2));
    int resident = 0;
    if (cudaOccupancyMaxActiveClusters(&resident, kern, &cfg) != cudaSuccess || resident <= 0) {
      cudaGetLastError();
      resident = num_sms() / 2;
    }
    resident = std::max(1, resident - (reserved_sms() + 1) / 2);
    cfg.gridDim = dim3(2 * static_cast<int>(std::min<long long>(pairs, resident)));
    return cudaLaunchKernelEx(&cfg, kern, ma, mb, msa, msb, P);
  }
  const size_t smem = static_cast<size_t>(kMxStages) * kMxStageBytes + 1024;
  const long long tiles = static_cast<long long>(P.m_tiles_max) * P.n_tiles;
  cudaError_t e = cudaFuncSetAttribute(gemm_mx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int grid = static_cast<int>(std::min<long long>(tiles, std::max(1, num_sms() - reserved_sms())));
  if (grid <= 0) return cudaSuccess;
  gemm_mx_kernel<<<grid, kThreads, smem, st>>>(ma, mb, P);
  return cudaGetLastError();
}

}  // namespace bpx
