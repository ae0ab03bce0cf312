// a2 fused into a3: the worker-side encode (Section III-A, Example 1: each
// processor forms the sums of its cell's blocks itself) done inside the
// tensor-core GEMM's operand load instead of as a separate HBM pass.
//
// Same tile walk, CTA-pair MMAs (cta_group::2, 256 x 256 tiles, 64-wide
// k-slices), segmented TMEM accumulation and epilogue as the materialized
// path's default GEMM, but the A operand of every stage is produced on chip:
//   warp 0        TMA producer of the B^T halves (hi, lo) only
//   warp 1        TMEM owner + MMA issuer (even CTA of the pair)
//   warps 2-7     transform: once per tile, a shared-memory table of the A
//                 row of every source of each of the CTA's 128 coded rows
//                 (cells of at most 8 sources); then for each 8-element chunk
//                 of the rows x 64 k-slice, load the chunk of every source
//                 (FP32, 128-bit read-only loads, two chunks in flight), add them
//                 in ascending source order with round-to-nearest (the same
//                 sums, bit for bit, as the encode pass), split into bf16
//                 hi = RN(x) and lo = RN(x - hi), and store both into the
//                 stage in the 128-byte swizzled K-major layout the MMA reads
//   warps 8-15    epilogue (two warps per TMEM lane quarter)
// A stage is full when the even CTA's TMA bytes have landed and all twelve
// transform warps of the pair have arrived (after a proxy fence that makes
// their shared-memory stores visible to the tensor core).  The transform and
// producer warps run with 80 registers, the epilogue warps with 176
// (setmaxnreg; 2 x 128 x 80 + 2 x 128 x 176 = the launch's 512 x 128).
// Every wait is bounded as in the other GEMMs.
#include <cstring>
#include <algorithm>

#include <cuda_bf16.h>

#include "tc_common.cuh"

namespace bpx {
namespace {

constexpr int kFThreads = 512;
constexpr int kFTransformThreads = 192;  // warps 2-7
constexpr int kFBN = 256;                // a pair's tile width (each CTA stages 128 rows of B^T)
constexpr int kFBK = 64;
constexpr int kFMaxDeg = 8;              // codes with cells of at most 8 sources

struct FusedJob {
  CUtensorMap map_bhi, map_blo;
  const float* A;          // M x K FP32, row-major (the sources: rows s h .. s h + h - 1)
  const int32_t* cell_ptr;
  const int32_t* cell_src;
  const int32_t* ctr;
  const int32_t* surv;
  const int32_t* direct;
  int32_t* info;
  int32_t* info_out;
  float* products;
  float* C_direct;
  int M, N, K, h, n_tiles;
};

template <bool kSplit>
struct FStage {
  static constexpr uint32_t kA = BM * kFBK * 2;             // 16 KB
  static constexpr uint32_t kB = (kFBN / 2) * kFBK * 2;     // 16 KB: this CTA's half of B^T
  static constexpr uint32_t kAhi = 0;
  static constexpr uint32_t kAlo = kA;
  static constexpr uint32_t kBhi = kSplit ? 2 * kA : kA;
  static constexpr uint32_t kBlo = kBhi + kB;
  static constexpr uint32_t kBytes = kSplit ? 2 * (kA + kB) : (kA + kB);
  static constexpr uint32_t kTxB = kSplit ? 2 * kB : kB;    // TMA bytes of one CTA per stage
};

__device__ __forceinline__ void raise_f(const FusedJob& J, int code, volatile int* abort_flag) {
  *abort_flag = 1;
  atomicExch(&J.info[BPX_INFO_DEVICE_ERR], code);
  atomicExch(&J.info[BPX_INFO_STATUS], code);
  if (J.info_out) {
    atomicExch(&J.info_out[BPX_INFO_DEVICE_ERR], code);
    atomicExch(&J.info_out[BPX_INFO_STATUS], code);
  }
}

// (pair unit, n) of tile t in bands of `group` pair units
__device__ __forceinline__ void f_tile(long long t, int group, int m_units, int n_tiles, int& m, int& n) {
  const int band_tiles = group * n_tiles;
  const int band = static_cast<int>(t / band_tiles);
  const int r = static_cast<int>(t - static_cast<long long>(band) * band_tiles);
  const int rows_in_band = min(group, m_units - band * group);
  m = band * group + r % rows_in_band;
  n = r / rows_in_band;
}

// Splits 8 coded values into bf16 hi (and lo) and stores them at byte
// offset `off` of the stage's A hi (lo) tile.
template <bool kSplit, typename St>
__device__ __forceinline__ void f_store8(uint8_t* st_base, uint32_t off, const float (&v)[8]) {
  uint32_t hv[4], lv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    hv[i] = *reinterpret_cast<const uint32_t*>(&hh);
    if (kSplit) {
      const float2 f = __bfloat1622float2(hh);
      const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * i] - f.x, v[2 * i + 1] - f.y);
      lv[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
  }
  *reinterpret_cast<uint4*>(st_base + St::kAhi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
  if (kSplit) *reinterpret_cast<uint4*>(st_base + St::kAlo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

__device__ __forceinline__ void f_add8(float (&v)[8], const float4& x0, const float4& x1) {
  v[0] += x0.x; v[1] += x0.y; v[2] += x0.z; v[3] += x0.w;
  v[4] += x1.x; v[5] += x1.y; v[6] += x1.z; v[7] += x1.w;
}

template <bool kSplit, int kStages>
__global__ void __launch_bounds__(kFThreads, 1)
gemm_fused_kernel(const __grid_constant__ FusedJob J, int group, int seg_kb) {
  using St = FStage<kSplit>;
  constexpr int kTmemCols = 2 * kFBN;
  constexpr int kCols = kFBN / 2;  // columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
  __shared__ __align__(8) uint64_t sfull_bar[2], sempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  // the transform's table of the current tile: the A row of every source of
  // each coded row's cell (rows past M left out), and how many
  __shared__ int32_t f_src[BM][kFMaxDeg];
  __shared__ int32_t f_deg[BM];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Mc = J.ctr[CTR_NSURV] * J.h;
  const int m_units = ((Mc + BM - 1) / BM + 1) / 2;
  const long long total_tiles = static_cast<long long>(m_units) * J.n_tiles;
  const uint32_t rank = cluster_rank();
  const int cid = static_cast<int>(blockIdx.x >> 1);
  const int nclusters = static_cast<int>(gridDim.x >> 1);
  const int k_blocks = (J.K + kFBK - 1) / kFBK;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      // the even CTA's stage: its producer's armed arrive + 2 x 6 transform warps
      mbar_init(smem_u32(&full_bar[s]), 1 + 2 * (kFTransformThreads / 32));
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&sfull_bar[a]), 1);
      mbar_init(smem_u32(&sempty_bar[a]), 16);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  cluster_sync();
  fence_after();
  const uint32_t tmem_base = tmem_base_sh;
  if (warp < 8) {
    // producer, MMA and transform warpgroups give registers to the epilogue's
    asm volatile("setmaxnreg.dec.sync.aligned.u32 80;" ::: "memory");
    if (warp == 0) {
      if (lane == 0) {
        int kb_all = 0;
        bool ok = true;
        for (long long jt = 0; ok; ++jt) {
          const long long t = snake(jt, cid, nclusters);
          if (t >= total_tiles) break;
          int mu, nt;
          f_tile(t, group, m_units, J.n_tiles, mu, nt);
          if (2 * mu * BM >= Mc) continue;
          const int yh = nt * kFBN + static_cast<int>(rank) * (kFBN / 2);
          for (int kb = 0; kb < k_blocks; ++kb, ++kb_all) {
            const int s = kb_all % kStages;
            const uint32_t ph = static_cast<uint32_t>((kb_all / kStages) & 1) ^ 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph, &abort_flag)) {
              if (!abort_flag) raise_f(J, BPX_ERR_TIMEOUT, &abort_flag);
              ok = false;
              break;
            }
            const uint32_t base = smem_u32(smem + s * St::kBytes);
            const uint32_t fb = smem_u32(&full_bar[s]);
            const uint32_t fb0 = mapa_rank(fb, 0);
            if (rank == 0) mbar_expect_tx(fb, 2 * St::kTxB);
            tma_load_2d_pair(base + St::kBhi, &J.map_bhi, fb0, kb * kFBK, yh);
            if (kSplit) tma_load_2d_pair(base + St::kBlo, &J.map_blo, fb0, kb * kFBK, yh);
          }
        }
        if ((!ok || abort_flag) && rank == 0) {
          for (int i = 0; i < kStages && i < kb_all; ++i) {
            const int kb = kb_all - 1 - i;
            mbar_wait(smem_u32(&full_bar[kb % kStages]), static_cast<uint32_t>((kb / kStages) & 1), nullptr);
          }
        }
      }
    } else if (warp == 1) {
      if (lane == 0 && rank == 0) {
        int kb_all = 0, g = 0;
        bool ok = true;
        constexpr uint32_t idesc = idesc_bf16_pair<kFBN>();
        for (long long jt = 0; ok; ++jt) {
          const long long t = snake(jt, cid, nclusters);
          if (t >= total_tiles) break;
          int mu, nt;
          f_tile(t, group, m_units, J.n_tiles, mu, nt);
          if (2 * mu * BM >= Mc) continue;
          const int n_segs = (k_blocks + seg_kb - 1) / seg_kb;
          for (int sg = 0; sg < n_segs && ok; ++sg, ++g) {
            const int buf = g & 1;
            if (!mbar_wait(smem_u32(&sempty_bar[buf]), static_cast<uint32_t>((g >> 1) & 1) ^ 1u, &abort_flag)) {
              if (!abort_flag) raise_f(J, BPX_ERR_TIMEOUT, &abort_flag);
              ok = false;
              break;
            }
            fence_after();
            const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(buf * kFBN);
            const int kb0 = sg * seg_kb, kb1 = min(k_blocks, kb0 + seg_kb);
            for (int kb = kb0; kb < kb1; ++kb, ++kb_all) {
              const int s = kb_all % kStages;
              if (!mbar_wait(smem_u32(&full_bar[s]), static_cast<uint32_t>((kb_all / kStages) & 1), &abort_flag)) {
                if (!abort_flag) raise_f(J, BPX_ERR_TIMEOUT, &abort_flag);
                ok = false;
                break;
              }
              fence_after();
              const uint32_t base = smem_u32(smem + s * St::kBytes);
              const uint64_t ahi = sdesc_sw128(base + St::kAhi);
              const uint64_t bhi = sdesc_sw128(base + St::kBhi);
              const uint64_t alo = sdesc_sw128(base + St::kAlo);
              const uint64_t blo = sdesc_sw128(base + St::kBlo);
  #pragma unroll
              for (int kk = 0; kk < kFBK / 16; ++kk) {
                const uint64_t adv = static_cast<uint64_t>(kk * 32) >> 4;
                const uint32_t first = (kb == kb0 && kk == 0) ? 0u : 1u;
                umma_kf16_pair(d_tmem, ahi + adv, bhi + adv, idesc, first);
                if (kSplit) {
                  umma_kf16_pair(d_tmem, ahi + adv, blo + adv, idesc, 1u);
                  umma_kf16_pair(d_tmem, alo + adv, bhi + adv, idesc, 1u);
                }
              }
              umma_commit_pair(smem_u32(&empty_bar[s]));
            }
            if (!ok) break;
            umma_commit_pair(smem_u32(&sfull_bar[buf]));
          }
        }
      }
    } else {
      // transform: chunk q of the 128 x 64 tile = row q / 8, 16-byte column q % 8
      const int tt = static_cast<int>(threadIdx.x) - 64;
      int kb_all = 0;
      bool ok = true;
      for (long long jt = 0; ok; ++jt) {
        const long long t = snake(jt, cid, nclusters);
        if (t >= total_tiles) break;
        int mu, nt;
        f_tile(t, group, m_units, J.n_tiles, mu, nt);
        if (2 * mu * BM >= Mc) continue;
        const int row0 = (2 * mu + static_cast<int>(rank)) * BM;
        // The table rows this thread's chunks read (chunk q: row q / 8) belong
        // to its warp alone -- the 8 lanes of a row are lanes 8g .. 8g + 7 of
        // one warp -- so each row's first lane fills the row and a warp sync
        // publishes it (no barrier across warps).
        __syncwarp();
        if ((tt & 7) == 0) {
          for (int q = tt; q < BM * (kFBK / 8); q += kFTransformThreads) {
            const int r = q >> 3, R = row0 + r;
            int d = 0;
            if (R < Mc) {
              const int ci = R / J.h, j = R - ci * J.h;
              const int cell = __ldg(J.surv + ci);
              const int e1 = __ldg(J.cell_ptr + cell + 1);
              for (int e = __ldg(J.cell_ptr + cell); e < e1 && d < kFMaxDeg; ++e) {
                const long long arow = static_cast<long long>(__ldg(J.cell_src + e)) * J.h + j;
                if (arow < J.M) f_src[r][d++] = static_cast<int32_t>(arow);
              }
            }
            f_deg[r] = d;
          }
        }
        __syncwarp();
        for (int kb = 0; kb < k_blocks; ++kb, ++kb_all) {
          const int s = kb_all % kStages;
          const uint32_t ph = static_cast<uint32_t>((kb_all / kStages) & 1) ^ 1u;
          if (!mbar_wait(smem_u32(&empty_bar[s]), ph, &abort_flag)) {
            if (!abort_flag) raise_f(J, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          uint8_t* st_base = smem + s * St::kBytes;
          // each row's first lane prefetches into L2 the row segments (256 B:
          // two lines per source) of the k-slice two steps ahead
          if ((tt & 7) == 0 && kb + 2 < k_blocks) {
            for (int q = tt; q < BM * (kFBK / 8); q += kFTransformThreads) {
              const int r = q >> 3, d = f_deg[r];
              for (int i = 0; i < d; ++i) {
                const float* p = J.A + static_cast<long long>(f_src[r][i]) * J.K + (kb + 2) * kFBK;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
                if ((kb + 2) * kFBK + 32 < J.K) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 32));
              }
            }
          }
          // chunk q = row q / 8, 16-byte column q % 8; two chunks at a time,
          // their loads in flight together
          for (int q = tt; q < BM * (kFBK / 8); q += 2 * kFTransformThreads) {
            const int qb = q + kFTransformThreads;
            const int ra = q >> 3, ca = q & 7, rb = qb >> 3, cb = qb & 7;
            const bool hb = qb < BM * (kFBK / 8);
            const int ka = kb * kFBK + 8 * ca, kq = kb * kFBK + 8 * cb;
            const int da = ka < J.K ? f_deg[ra] : 0;
            const int db = (hb && kq < J.K) ? f_deg[rb] : 0;
            float va[8], vb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) va[i] = vb[i] = 0.f;
            for (int i = 0; i < max(da, db); ++i) {
              float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
              if (i < da) {
                const float4* p4 = reinterpret_cast<const float4*>(J.A + static_cast<long long>(f_src[ra][i]) * J.K + ka);
                a0 = __ldg(p4);
                a1 = __ldg(p4 + 1);
              }
              if (i < db) {
                const float4* p4 = reinterpret_cast<const float4*>(J.A + static_cast<long long>(f_src[rb][i]) * J.K + kq);
                b0 = __ldg(p4);
                b1 = __ldg(p4 + 1);
              }
              if (i < da) f_add8(va, a0, a1);
              if (i < db) f_add8(vb, b0, b1);
            }
            f_store8<kSplit, St>(st_base, static_cast<uint32_t>(ra * 128 + ((ca ^ (ra & 7)) << 4)), va);
            if (hb) f_store8<kSplit, St>(st_base, static_cast<uint32_t>(rb * 128 + ((cb ^ (rb & 7)) << 4)), vb);
          }
          // the stores become visible to the tensor core, then the warp arrives
          // on the even CTA's stage barrier
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                             mapa_rank(smem_u32(&full_bar[s]), 0))
                         : "memory");
        }
      }
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 176;" ::: "memory");
    // epilogue warps 8..15: TMEM lane quarter = warp % 4, column half by warp
    const int e = warp - 8;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int row = quarter * 32 + lane;
    int g = 0;
    bool ok = true;
    for (long long jt = 0; ok; ++jt) {
      const long long t = snake(jt, cid, nclusters);
      if (t >= total_tiles) break;
      int mu, nt;
      f_tile(t, group, m_units, J.n_tiles, mu, nt);
      if (2 * mu * BM >= Mc) continue;
      const int n_segs = (k_blocks + seg_kb - 1) / seg_kb;
      float accum[kCols];
#pragma unroll
      for (int i = 0; i < kCols; ++i) accum[i] = 0.f;
      for (int sg = 0; sg < n_segs; ++sg, ++g) {
        const int buf = g & 1;
        if (!mbar_wait(smem_u32(&sfull_bar[buf]), static_cast<uint32_t>((g >> 1) & 1), &abort_flag)) {
          if (!abort_flag) raise_f(J, BPX_ERR_TIMEOUT, &abort_flag);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                               static_cast<uint32_t>(buf * kFBN + half * kCols);
#pragma unroll
        for (int c = 0; c < kCols / 32; ++c) {
          float v[32];
          tmem_ld32(taddr + c * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) accum[c * 32 + i] = __fadd_rn(accum[c * 32 + i], v[i]);
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(mapa_rank(smem_u32(&sempty_bar[buf]), 0));
      }
      if (!ok) break;
      const int r = (2 * mu + static_cast<int>(rank)) * BM + row;
      if (r < Mc) {
        const int ci = r / J.h;
        const int j = r - ci * J.h;
        const int cell = J.surv[ci];
        const int ds = J.C_direct ? J.direct[cell] : -1;
        float* dst = ds >= 0 ? J.C_direct + (static_cast<long long>(ds) * J.h + j) * J.N
                             : J.products + (static_cast<long long>(cell) * J.h + j) * J.N;
        const int n0 = nt * kFBN + half * kCols;
#pragma unroll
        for (int q = 0; q < kCols / 4; ++q) {
          const int n = n0 + 4 * q;
          if (n < J.N)
            *reinterpret_cast<float4*>(dst + n) =
                make_float4(accum[4 * q], accum[4 * q + 1], accum[4 * q + 2], accum[4 * q + 3]);
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                 : "memory");
  }
}

bool f_make_map(CUtensorMap* map, const void* base, long long rows, int K, int box_rows) {
  auto enc = get_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(K) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kFBK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool kSplit, int kStages>
cudaError_t launch_fused_variant(const FusedJob& J, long long pairs, int group, int seg_kb, cudaStream_t st) {
  const size_t smem = static_cast<size_t>(kStages) * FStage<kSplit>::kBytes + 1024;
  auto kern = gemm_fused_kernel<kSplit, kStages>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (pairs <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kFThreads);
  cfg.dynamicSmemBytes = smem;
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
  return cudaLaunchKernelEx(&cfg, kern, J, group, seg_kb);
}

}  // namespace

cudaError_t launch_gemm_fused(const DevGraph& g, const DevPlan& p, const float* A, int M, const void* b_hi,
                              const void* b_lo, int num_cells, int N, int K, int h, bool split3, float* products,
                              float* C_direct, int config, int32_t* info_out, cudaStream_t st) {
  // the default CTA-pair tile config's band and segment (8080); config 0 or
  // any CTA-pair 64-wide config (tile code 0) may pick band and segment
  if (!gemm_config_ok(config) || (config != 0 && config % 10 != 0)) return cudaErrorInvalidValue;
  if (K % 8 != 0 || (!A && M > 0)) return cudaErrorInvalidValue;
  int group = 8, seg_kb = 8;
  if (config > 0) {
    if ((config / 10) % 100 > 0) seg_kb = (config / 10) % 100;
    if (config / 1000 > 0) group = config / 1000;
  }
  FusedJob J;
  memset(&J, 0, sizeof J);
  if (!f_make_map(&J.map_bhi, b_hi, N, K, kFBN / 2)) return cudaErrorInvalidValue;
  if (split3) {
    if (!f_make_map(&J.map_blo, b_lo, N, K, kFBN / 2)) return cudaErrorInvalidValue;
  } else {
    J.map_blo = J.map_bhi;
  }
  J.A = A;
  J.cell_ptr = g.cell_ptr;
  J.cell_src = g.cell_src;
  J.ctr = p.ctr;
  J.surv = p.surv;
  J.direct = p.direct;
  J.info = p.info;
  J.info_out = info_out;
  J.products = products;
  J.C_direct = C_direct;
  J.M = M;
  J.N = N;
  J.K = K;
  J.h = h;
  J.n_tiles = (N + kFBN - 1) / kFBN;
  const long long rows = static_cast<long long>(num_cells) * h;
  const long long pairs = ((rows + BM - 1) / BM + 1) / 2 * static_cast<long long>(J.n_tiles);
  return split3 ? launch_fused_variant<true, 3>(J, pairs, group, seg_kb, st)
                : launch_fused_variant<false, 6>(J, pairs, group, seg_kb, st);
}

}  // namespace bpx
