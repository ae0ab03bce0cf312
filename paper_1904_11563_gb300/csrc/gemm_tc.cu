// a3 on the 5th-generation tensor cores (tcgen05 + TMA + TMEM), sm_103a.
//
// Coded products P = A_coded * B over the staged bf16 operands:
//   A_coded (rows = h * surviving cells, K-major) written by the encode+split
//   kernel, B^T (N x K, K-major) written by the B split kernel.
// Split-BF16x3 accumulates hi*hi + hi*lo + lo*hi into one FP32 TMEM
// accumulator (the lo*lo term is below FP32 rounding); plain BF16 issues the
// hi*hi MMA only.  Split-FP16x3 (a job with exponent arrays) issues the same
// three MMAs over fp16 halves of row- and column-scaled operands, and the
// epilogue multiplies each output by 2^-(row exponent + column exponent).
//
// Persistent warp-specialised kernel, one 128 x 256 output tile per CTA at
// a time:
//   warp 0     TMA producer: 128B-swizzled 64-wide k-slices of A (hi, lo)
//              and B (hi, lo) into a ring of shared-memory stages
//   warp 1     TMEM owner + MMA issuer (one thread): tcgen05.mma kind::f16,
//              M=128 N=256 K=16, commit -> "stage empty" / "segment full"
//   warps 2-9  epilogue: two warps per TMEM lane quarter, 128 columns each.
// The default configuration runs the CTAs in clusters of two whose MMAs are
// CTA-pair MMAs (cta_group::2, M=256): each CTA stages its own 128 A rows and
// half of the B tile, and the even CTA's MMA thread issues for both.
//
// The tensor core adds each MMA's products into its FP32 accumulator with
// truncation, so the error of a long K sum grows with K.  The K range of a
// tile is therefore cut into segments of `seg_kb` k-blocks: the MMA warp
// accumulates a segment into one of two TMEM buffers (starting from zero),
// and the epilogue warps drain the finished buffer into FP32 registers with
// round-to-nearest adds while the next segment accumulates in the other
// buffer.  After a tile's last segment the registers are written out: rows
// scattered to the cell's product slot, or straight into the source block
// of C for depth-1 resolvers.
// Every mbarrier wait is bounded (clock64 budget); a wait that runs out
// raises BPX_ERR_TIMEOUT in the plan's info words, tells the other warps to
// stop, and the CTA still frees its TMEM and exits.
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "tc_common.cuh"

namespace bpx {
namespace {

// One coded GEMM: its tensor maps and where its plan and outputs live.
// A grouped launch keeps an array of these in global memory; a single launch
// passes one as a __grid_constant__ parameter.
struct __align__(64) TcJob {
  CUtensorMap map_ahi, map_alo, map_bhi, map_blo;
  const int32_t* ctr;     // plan counters (surviving-cell count)
  const int32_t* surv;    // surviving cells, ascending
  const int32_t* direct;  // per cell: the source it resolves at depth 1, or -1
  int32_t* info;          // plan info words (device error reporting)
  int32_t* info_out;      // caller's info words, or null
  float* products;
  float* C_direct;
  int N, K, h;
  int m_tiles_max, n_tiles;
  long long tile_base;    // first tile of this job in the launch's tile space
  // exact slices: int32 diagonal planes (plane d at planes + d plane_stride),
  // digit planes per operand row (= diagonals), K padded to 64
  int32_t* planes;
  long long plane_stride;
  int ex_S, ex_Kp;
  // two-dimensional scheme: every cell (in t2_order) is a list of terms (A
  // operand, B operand) over h-row A operands and w-row B^T operands; N is the
  // row stride of C; kc = the code's k (source s = z kc + l); cnt = -1 marks
  // the cells of erased columns
  const int32_t* t2_ptr;
  const int32_t* t2_a;
  const int32_t* t2_b;
  const int32_t* t2_order;
  const int32_t* cnt;
  int w2, kc, ncells;
  // split fp16 (rows mode): power-of-two exponent per coded row and per
  // column of B; null for bf16 operands
  const int32_t* a_exp;
  const int32_t* b_exp;
};

template <bool kSplit, int kBN, int kBK = BK>
struct Stage {
  static constexpr uint32_t kA = BM * kBK * 2;   // 16 or 8 KB
  static constexpr uint32_t kB = kBN * kBK * 2;  // 32, 16 or 8 KB
  static constexpr uint32_t kBytes = kSplit ? 2 * (kA + kB) : (kA + kB);
  static constexpr uint32_t kAhi = 0;
  static constexpr uint32_t kAlo = kA;
  static constexpr uint32_t kBhi = kSplit ? 2 * kA : kA;
  static constexpr uint32_t kBlo = kBhi + kB;
};

// Output stores of the epilogue: streaming (.cs), so that the products and
// C blocks written once per tile do not push the operand tiles other CTAs
// are still reading out of L2.
__device__ __forceinline__ void st_cs4(float* p, float a, float b, float c, float d) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void raise_error(const TcJob& J, int code, volatile int* abort_flag) {
  *abort_flag = 1;
  atomicExch(&J.info[BPX_INFO_DEVICE_ERR], code);
  atomicExch(&J.info[BPX_INFO_STATUS], code);
  if (J.info_out) {
    atomicExch(&J.info_out[BPX_INFO_DEVICE_ERR], code);
    atomicExch(&J.info_out[BPX_INFO_STATUS], code);
  }
}

// Where a tile of the launch's tile space lands: its job, its (m, n) tile of
// that job (bands of `group` m-tiles, n-major inside a band so that CTAs
// resident together share a few A row tiles and B column tiles in L2), and
// whether it covers surviving rows at all (tiles past the job's surviving
// rows are skipped by every role alike).
struct TileRef {
  const TcJob* J;
  int m, n, Mc, k_blocks;
  int d, k_steps;  // exact slices: diagonal, and k-slices over its digit pairs
  int cell, tp;    // two-dimensional scheme: the tile's cell and its first term
  bool live;
};

// Kernel modes: the coded GEMM of the one-dimensional scheme, its exact-slice
// digit products, and the two-dimensional scheme's per-cell term products.
enum { kModeRows = 0, kModeExact = 1, kMode2D = 2 };

// live_mc >= 0: a single job whose surviving row count is already known; its
// tile space then holds the live m-tiles only (no skipped tiles inside the
// rasterisation bands).  pair: the tile space counts pairs of vertically
// adjacent m-tiles (two CTAs of a cluster share the B tile); m is then the
// pair index and `live` tells whether the pair covers surviving rows.
// exact: a single job's tile space holds every tile once per diagonal d
// (innermost, so that a tile's diagonals run close together); the tile then
// walks the d + 1 digit pairs (i, d - i), all k-slices of one pair after the
// other.
__device__ __forceinline__ TileRef locate(const TcJob* jobs, int njobs, long long t, int group, int live_mc,
                                          bool pair, int bk, int mode = kModeRows) {
  const bool exact = mode == kModeExact;
  if (mode == kMode2D) {
    // one job; tile space = cells (most terms first) x m-units x n-tiles,
    // m fastest so that CTAs resident together share the B operand tile
    const TcJob& J = jobs[0];
    TileRef R;
    R.J = &J;
    const int m_units = pair ? (J.m_tiles_max + 1) / 2 : J.m_tiles_max;
    const int per_cell = m_units * J.n_tiles;
    const int ci = static_cast<int>(t / per_cell);
    const int r = static_cast<int>(t - static_cast<long long>(ci) * per_cell);
    R.cell = J.t2_order[ci];
    R.n = r / m_units;
    R.m = r - R.n * m_units;
    R.Mc = J.h;
    R.d = 0;
    R.tp = J.t2_ptr[R.cell];
    R.k_blocks = (J.K + bk - 1) / bk;
    R.k_steps = (J.t2_ptr[R.cell + 1] - R.tp) * R.k_blocks;
    R.live = J.cnt[R.cell] >= 0;
    return R;
  }
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {  // last job with tile_base <= t
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_base <= t) lo = mid;
    else hi = mid - 1;
  }
  TileRef R;
  R.J = &jobs[lo];
  const TcJob& J = *R.J;
  const int lt0 = static_cast<int>(t - J.tile_base);
  R.Mc = live_mc >= 0 ? live_mc : J.ctr[CTR_NSURV] * J.h;
  int m_units = live_mc >= 0 ? (live_mc + BM - 1) / BM : J.m_tiles_max;
  if (pair) m_units = (m_units + 1) / 2;
  int d = 0, lt = lt0;
  if (exact) {  // the diagonals of a tile are adjacent: they reuse its digit planes from L2
    d = lt % J.ex_S;
    lt /= J.ex_S;
  }
  const int band_tiles = group * J.n_tiles;
  const int band = lt / band_tiles;
  const int r = lt - band * band_tiles;
  const int rows_in_band = min(group, m_units - band * group);
  R.m = band * group + r % rows_in_band;
  R.n = r / rows_in_band;
  R.k_blocks = (J.K + bk - 1) / bk;
  R.d = d;
  R.cell = R.tp = 0;
  R.k_steps = exact ? (d + 1) * R.k_blocks : R.k_blocks;
  R.live = (pair ? 2 * R.m : R.m) * BM < R.Mc;
  return R;
}

// kPair == 2: launched in clusters of two CTAs that take the two m-tiles of
// a pair with the same B tile, computed by CTA-pair MMAs (cta_group::2,
// M = 256): each CTA loads only its own A rows and its half of the B tile,
// so a CTA's shared memory takes a third less traffic per MMA.  kPair == 0:
// one CTA per tile.  (No variant loads by TMA multicast.)
// kMode == kModeExact: exact-slice digit products (plain bf16 MMAs over the
// digit planes, k-slices of the diagonal's digit pairs in sequence; FP32
// segments exact by construction, promoted to int32 and stored to the
// diagonal's plane).  kMode == kMode2D: the two-dimensional scheme (k-slices
// of the cell's terms in sequence; h x w output blocks).
template <bool kSplit, int kStages, int kBN, int kPair, int kBK, int kMode = kModeRows>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ TcJob single, const TcJob* __restrict__ table, int njobs,
               long long total_tiles, int group, int seg_kb) {
  constexpr bool kExact = kMode == kModeExact;
  constexpr bool k2D = kMode == kMode2D;
  static_assert(kPair == 0 || kPair == 2, "tiles are 1-CTA or CTA-pair MMAs");
  constexpr bool k2Sm = kPair == 2;
  using St = Stage<kSplit, k2Sm ? kBN / 2 : kBN, kBK>;  // a CTA pair holds half the B tile each
  constexpr int kTmemCols = 2 * kBN;  // two FP32 segment accumulators
  constexpr int kCols = kBN / 2;      // columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
  __shared__ __align__(8) uint64_t sfull_bar[2], sempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const TcJob* jobs = table ? table : &single;
  const bool grouped = table != nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // A single job reads its surviving row count once and walks live tiles only.
  const int live_mc = grouped ? -1 : single.ctr[CTR_NSURV] * single.h;
  if (!grouped && !k2D) {
    int units = (live_mc + BM - 1) / BM;
    if (kPair) units = (units + 1) / 2;
    total_tiles = static_cast<long long>(units) * single.n_tiles * (kExact ? single.ex_S : 1);
  }
  const uint32_t rank = kPair ? cluster_rank() : 0u;
  const int cid = kPair ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int nclusters = kPair ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&sfull_bar[a]), 1);
      mbar_init(smem_u32(&sempty_bar[a]), k2Sm ? 16 : 8);  // CTA pair: both CTAs' epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (k2Sm) {  // both CTAs of the pair allocate together
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&tmem_base_sh)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&tmem_base_sh)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  fence_before();
  __syncthreads();
  if (kPair) cluster_sync();  // the peer's barriers exist before any of its copies or commits land
  fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      int kb_all = 0;
      bool ok = true;
      const TcJob* fenced = nullptr;
      for (long long j = 0; ok; ++j) {
        const long long t = snake(j, cid, nclusters);
        if (t >= total_tiles) break;
        const TileRef T = locate(jobs, njobs, t, group, live_mc, kPair, kBK, kMode);
        if (!T.live) continue;
        if (grouped && T.J != fenced) {
          tensormap_acquire(&T.J->map_ahi);
          tensormap_acquire(&T.J->map_bhi);
          if (kSplit) {
            tensormap_acquire(&T.J->map_alo);
            tensormap_acquire(&T.J->map_blo);
          }
          fenced = T.J;
        }
        const int m_cta = kPair ? 2 * T.m + static_cast<int>(rank) : T.m;
        int ya = m_cta * BM, yb = T.n * kBN, cur_term = -1;
        for (int q = 0; q < T.k_steps; ++q, ++kb_all) {
          const int s = kb_all % kStages;
          int xa = q * kBK, xb = q * kBK;
          if (kExact) {  // pair (pi, d - pi), k-slice kb
            const int pi = q / T.k_blocks, kb = q - pi * T.k_blocks;
            xa = pi * T.J->ex_Kp + kb * kBK;
            xb = (T.d - pi) * T.J->ex_Kp + kb * kBK;
          }
          if (k2D) {  // term ti of the cell, k-slice kb
            const int ti = q / T.k_blocks, kb = q - ti * T.k_blocks;
            if (ti != cur_term) {
              cur_term = ti;
              ya = T.J->t2_a[T.tp + ti] * T.J->h + m_cta * BM;
              yb = T.J->t2_b[T.tp + ti] * T.J->w2 + T.n * kBN;
            }
            xa = xb = kb * kBK;
          }
          const uint32_t ph = static_cast<uint32_t>((kb_all / kStages) & 1) ^ 1u;
          if (!mbar_wait(smem_u32(&empty_bar[s]), ph, &abort_flag)) {
            if (!abort_flag) raise_error(*T.J, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          const uint32_t base = smem_u32(smem + s * St::kBytes);
          const uint32_t fb = smem_u32(&full_bar[s]);
          if constexpr (k2Sm) {
            // both CTAs' copies count on the even CTA's barrier, armed there
            // for the two stages' bytes
            const uint32_t fb0 = mapa_rank(fb, 0);
            if (rank == 0) mbar_expect_tx(fb, 2 * St::kBytes);
            const int yh = yb + static_cast<int>(rank) * (kBN / 2);
            tma_load_2d_pair(base + St::kAhi, &T.J->map_ahi, fb0, xa, ya);
            if (kSplit) tma_load_2d_pair(base + St::kAlo, &T.J->map_alo, fb0, xa, ya);
            tma_load_2d_pair(base + St::kBhi, &T.J->map_bhi, fb0, xb, yh);
            if (kSplit) tma_load_2d_pair(base + St::kBlo, &T.J->map_blo, fb0, xb, yh);
            continue;
          }
          mbar_expect_tx(fb, St::kBytes);
          tma_load_2d(base + St::kAhi, &T.J->map_ahi, fb, xa, ya);
          if (kSplit) tma_load_2d(base + St::kAlo, &T.J->map_alo, fb, xa, ya);
          tma_load_2d(base + St::kBhi, &T.J->map_bhi, fb, xb, yb);
          if (kSplit) tma_load_2d(base + St::kBlo, &T.J->map_blo, fb, xb, yb);
        }
      }
      if ((!ok || abort_flag) && !(k2Sm && rank != 0)) {
        // Stopping early: let the copies this CTA still has in flight land
        // (bounded waits, abort ignored) before its shared memory goes away.
        // (A CTA pair's copies all complete on the even CTA's barriers.)
        for (int i = 0; i < kStages && i < kb_all; ++i) {
          const int kb = kb_all - 1 - i;
          mbar_wait(smem_u32(&full_bar[kb % kStages]), static_cast<uint32_t>((kb / kStages) & 1), nullptr);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && (!k2Sm || rank == 0)) {  // a CTA pair's MMAs issue from the even CTA
      int kb_all = 0, g = 0;
      bool ok = true;
      for (long long j = 0; ok; ++j) {
        const long long t = snake(j, cid, nclusters);
        if (t >= total_tiles) break;
        const TileRef T = locate(jobs, njobs, t, group, live_mc, kPair, kBK, kMode);
        if (!T.live) continue;
        const int n_segs = (T.k_steps + seg_kb - 1) / seg_kb;
        // operand format: fp16 for a split-fp16 job, else bf16
        const uint32_t idesc = (!kExact && !k2D && T.J->a_exp)
                                   ? (k2Sm ? idesc_f16_pair<kBN>() : idesc_f16<kBN>())
                                   : (k2Sm ? idesc_bf16_pair<kBN>() : idesc_bf16<kBN>());
        for (int sg = 0; sg < n_segs && ok; ++sg, ++g) {
          const int buf = g & 1;
          if (!mbar_wait(smem_u32(&sempty_bar[buf]), static_cast<uint32_t>((g >> 1) & 1) ^ 1u,
                         &abort_flag)) {
            if (!abort_flag) raise_error(*T.J, BPX_ERR_TIMEOUT, &abort_flag);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(buf * kBN);
          const int kb0 = sg * seg_kb, kb1 = min(T.k_steps, kb0 + seg_kb);
          for (int kb = kb0; kb < kb1; ++kb, ++kb_all) {
            const int s = kb_all % kStages;
            if (!mbar_wait(smem_u32(&full_bar[s]), static_cast<uint32_t>((kb_all / kStages) & 1),
                           &abort_flag)) {
              if (!abort_flag) raise_error(*T.J, BPX_ERR_TIMEOUT, &abort_flag);
              ok = false;
              break;
            }
            fence_after();
            const uint32_t base = smem_u32(smem + s * St::kBytes);
            const uint64_t ahi = sdesc_k<kBK>(base + St::kAhi);
            const uint64_t bhi = sdesc_k<kBK>(base + St::kBhi);
            const uint64_t alo = sdesc_k<kBK>(base + St::kAlo);
            const uint64_t blo = sdesc_k<kBK>(base + St::kBlo);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t adv = static_cast<uint64_t>(kk * 32) >> 4;  // 16 bf16 = 32 B
              const uint32_t first = (kb == kb0 && kk == 0) ? 0u : 1u;
              if constexpr (k2Sm) {
                umma_kf16_pair(d_tmem, ahi + adv, bhi + adv, idesc, first);
                if (kSplit) {
                  umma_kf16_pair(d_tmem, ahi + adv, blo + adv, idesc, 1u);
                  umma_kf16_pair(d_tmem, alo + adv, bhi + adv, idesc, 1u);
                }
              } else {
                umma_kf16(d_tmem, ahi + adv, bhi + adv, idesc, first);
                if (kSplit) {
                  umma_kf16(d_tmem, ahi + adv, blo + adv, idesc, 1u);
                  umma_kf16(d_tmem, alo + adv, bhi + adv, idesc, 1u);
                }
              }
            }
            if (k2Sm)
              umma_commit_pair(smem_u32(&empty_bar[s]));
            else
              umma_commit(smem_u32(&empty_bar[s]));
          }
          if (!ok) break;
          if (k2Sm)
            umma_commit_pair(smem_u32(&sfull_bar[buf]));
          else
            umma_commit(smem_u32(&sfull_bar[buf]));
        }
      }
    }
  } else {
    // epilogue warps 2..9: TMEM lane quarter = warp % 4, column half by warp
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int row = quarter * 32 + lane;
    int g = 0;
    bool ok = true;
    for (long long j = 0; ok; ++j) {
      const long long t = snake(j, cid, nclusters);
      if (t >= total_tiles) break;
      const TileRef T = locate(jobs, njobs, t, group, live_mc, kPair, kBK, kMode);
      if (!T.live) continue;
      const int n_segs = (T.k_steps + seg_kb - 1) / seg_kb;
      float accum[kCols];
      int iacc[kCols];
#pragma unroll
      for (int i = 0; i < kCols; ++i) {
        if constexpr (kExact) iacc[i] = 0;
        else accum[i] = 0.f;
      }
      for (int sg = 0; sg < n_segs; ++sg, ++g) {
        const int buf = g & 1;
        if (!mbar_wait(smem_u32(&sfull_bar[buf]), static_cast<uint32_t>((g >> 1) & 1), &abort_flag)) {
          if (!abort_flag) raise_error(*T.J, BPX_ERR_TIMEOUT, &abort_flag);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                               static_cast<uint32_t>(buf * kBN + half * kCols);
#pragma unroll
        for (int c = 0; c < kCols / 32; ++c) {
          float v[32];
          tmem_ld32(taddr + c * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if constexpr (kExact) iacc[c * 32 + i] += __float2int_rn(v[i]);  // an exact integer
            else accum[c * 32 + i] = __fadd_rn(accum[c * 32 + i], v[i]);
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) {
          if (k2Sm)  // the even CTA's MMA thread waits for both CTAs' drains
            mbar_arrive_cluster(mapa_rank(smem_u32(&sempty_bar[buf]), 0));
          else
            mbar_arrive(smem_u32(&sempty_bar[buf]));
        }
      }
      if (!ok) break;
      const TcJob& J = *T.J;
      const int r = (kPair ? 2 * T.m + static_cast<int>(rank) : T.m) * BM + row;
      if (k2D) {
        if (r < J.h) {  // row r of the cell's h x w block
          const int ds = J.C_direct ? J.direct[T.cell] : -1;
          float* dst;
          if (ds >= 0) {
            const int z = ds / J.kc, l = ds - z * J.kc;
            dst = J.C_direct + (static_cast<long long>(z) * J.h + r) * J.N + static_cast<long long>(l) * J.w2;
          } else {
            dst = J.products + (static_cast<long long>(T.cell) * J.h + r) * J.w2;
          }
          const int n0 = T.n * kBN + half * kCols;
#pragma unroll
          for (int q = 0; q < kCols / 4; ++q) {
            const int n = n0 + 4 * q;
            if (n < J.w2)
              st_cs4(dst + n, accum[4 * q], accum[4 * q + 1], accum[4 * q + 2], accum[4 * q + 3]);
          }
        }
      } else if (r < T.Mc) {
        const int ci = r / J.h;
        const int j = r - ci * J.h;
        const int cell = J.surv[ci];
        const int n0 = T.n * kBN + half * kCols;
        if constexpr (kExact) {
          int32_t* dst = J.planes + T.d * J.plane_stride + (static_cast<long long>(cell) * J.h + j) * J.N;
#pragma unroll
          for (int q = 0; q < kCols / 4; ++q) {
            const int n = n0 + 4 * q;
            if (n < J.N)
              *reinterpret_cast<int4*>(dst + n) = make_int4(iacc[4 * q], iacc[4 * q + 1], iacc[4 * q + 2], iacc[4 * q + 3]);
          }
        } else {
          const int ds = J.C_direct ? J.direct[cell] : -1;
          float* dst = ds >= 0 ? J.C_direct + (static_cast<long long>(ds) * J.h + j) * J.N
                               : J.products + (static_cast<long long>(cell) * J.h + j) * J.N;
          if (J.a_exp) {  // undo the operands' scales: exact unless the result is subnormal
            const int ea = J.a_exp[r];
#pragma unroll
            for (int q = 0; q < kCols / 4; ++q) {
              const int n = n0 + 4 * q;
              if (n < J.N) {
                const int4 eb = *reinterpret_cast<const int4*>(J.b_exp + n);
                accum[4 * q] = ldexpf(accum[4 * q], -(ea + eb.x));
                accum[4 * q + 1] = ldexpf(accum[4 * q + 1], -(ea + eb.y));
                accum[4 * q + 2] = ldexpf(accum[4 * q + 2], -(ea + eb.z));
                accum[4 * q + 3] = ldexpf(accum[4 * q + 3], -(ea + eb.w));
              }
            }
          }
#pragma unroll
          for (int q = 0; q < kCols / 4; ++q) {
            const int n = n0 + 4 * q;
            if (n < J.N)
              st_cs4(dst + n, accum[4 * q], accum[4 * q + 1], accum[4 * q + 2], accum[4 * q + 3]);
          }
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  if (kPair) cluster_sync();  // no CTA leaves while its peer may still write into it
  if (warp == 1) {
    fence_after();
    if constexpr (k2Sm)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(kTmemCols)
                   : "memory");
  }
}

// Failure-detection self-test: one thread waits on an mbarrier that nothing
// will ever arrive at, through the same bounded wait the GEMM uses, and
// reports BPX_ERR_TIMEOUT when the budget runs out.
__global__ void wait_timeout_kernel(long long budget, int32_t* info) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const long long t0 = clock64();
  const bool done = mbar_wait(smem_u32(&bar), 0u, nullptr, budget);
  info[BPX_INFO_STATUS] = done ? BPX_OK : BPX_ERR_TIMEOUT;
  info[BPX_INFO_DEVICE_ERR] = done ? 0 : BPX_ERR_TIMEOUT;
  info[6] = static_cast<int32_t>(min(clock64() - t0, static_cast<long long>(INT32_MAX)));
}

// 2-D K-major bf16 tensor map: rows x K, box = box_rows x bk (bk = 64: 128 B
// swizzle; bk = 32: 64 B swizzle), matching the UMMA descriptors.
bool make_map(CUtensorMap* map, const void* base, long long rows, int K, int box_rows, int bk = BK,
              bool fp16 = false) {
  auto enc = get_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(K) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(bk), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tile configurations the autotuner chooses among (gemm_config % 10):
// 1 = 128x256, 2 = 128x128, 5 / 6 = the same with 32-wide k-slices (64-byte
// swizzle, twice the stages of half the size); 9 / 0 = 256x256 tiles of
// CTA-pair MMAs (128x256 per CTA) with 32- / 64-wide k-slices.  Codes 3, 4,
// 7 and 8 are not tile configurations (rejected as invalid).
bool tile_valid(int config) {
  const int t = config % 10;
  return config >= 0 && t != 3 && t != 4 && t != 7 && t != 8;
}
int tile_bn(int config) {
  const int t = config % 10;
  return (t == 2 || t == 6) ? 128 : 256;
}
// 0: one CTA per tile; 2: CTA pairs computing one tile with cta_group::2 MMAs.
int tile_pair(int config) {
  const int t = config % 10;
  return (t == 9 || t == 0) ? 2 : 0;
}
int tile_bk(int config) { return (config % 10) >= 5 ? 32 : 64; }

// seg_kb: k-slices of kBK per TMEM accumulation segment.
template <bool kSplit, int kStages, int kBN, int kPair, int kBK, int kMode = kModeRows>
cudaError_t launch_variant(const TcJob& single, const TcJob* table, int njobs, long long total_tiles,
                           int group, int seg_kb, cudaStream_t st) {
  // 32-wide slices: 32 KB of slack after the stages, so that the descriptors
  // of the 64-byte swizzled layout can never reach past the allocation.
  // (a CTA of a cta_group::2 pair stages half the B tile)
  using St = Stage<kSplit, kPair == 2 ? kBN / 2 : kBN, kBK>;
  const size_t smem = static_cast<size_t>(kStages) * St::kBytes + 1024 + (kBK == 32 ? 32768 : 0);
  auto kern = gemm_tc_kernel<kSplit, kStages, kBN, kPair, kBK, kMode>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (total_tiles <= 0) return cudaSuccess;
  if (kPair == 0) {
    const int grid = static_cast<int>(std::min<long long>(total_tiles, std::max(1, num_sms() - reserved_sms())));
    kern<<<grid, kThreads, smem, st>>>(single, table, njobs, total_tiles, group, seg_kb);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // as many CTA pairs as can be resident at once (pairs must share a GPC)
  cfg.gridDim = dim3(2 * (num_sms() / 2));
  int resident = 0;
  if (cudaOccupancyMaxActiveClusters(&resident, kern, &cfg) != cudaSuccess || resident <= 0) {
    cudaGetLastError();
    resident = num_sms() / 2;
  }
  resident = std::max(1, resident - (reserved_sms() + 1) / 2);
  const int clusters = static_cast<int>(std::min<long long>(total_tiles, resident));
  cfg.gridDim = dim3(2 * clusters);
  return cudaLaunchKernelEx(&cfg, kern, single, table, njobs, total_tiles, group, seg_kb);
}

template <int kBK, int kMode = kModeRows>
cudaError_t dispatch_bk(bool split3, int bn, int pair, const TcJob& single, const TcJob* table, int njobs,
                        long long total_tiles, int group, int seg_kb, cudaStream_t st) {
  constexpr int m = BK / kBK;  // stages scale up as slices shrink
  seg_kb *= m;                 // configs count segments in 64-wide k-blocks
#define BPX_LV(SPLIT, STAGES, BN, PAIR) \
  launch_variant<SPLIT, STAGES, BN, PAIR, kBK, kMode>(single, table, njobs, total_tiles, group, seg_kb, st)
  // CTA-pair MMAs: a stage holds the CTA's A rows and half the B tile
  if (pair == 2) return split3 ? BPX_LV(true, 3 * m, 256, 2) : BPX_LV(false, 6 * m, 256, 2);
  if (split3) return bn == 128 ? BPX_LV(true, 3 * m, 128, 0) : BPX_LV(true, 2 * m, 256, 0);
  return bn == 128 ? BPX_LV(false, 6 * m, 128, 0) : BPX_LV(false, 4 * m, 256, 0);
#undef BPX_LV
}

// Exact slices: the tile's width, pairing and k-slice (the padded K is a
// multiple of 64, so a 64-wide slice never straddles two digit planes);
// seg in k-slices.
template <int kBK>
cudaError_t dispatch_exact_bk(int bn, int pair, const TcJob& J, long long total_tiles, int group, int seg,
                              cudaStream_t st) {
  constexpr int m = BK / kBK;
  if (pair == 2)
    return launch_variant<false, 6 * m, 256, 2, kBK, kModeExact>(J, nullptr, 1, total_tiles, group, seg, st);
  if (bn == 128) return launch_variant<false, 6 * m, 128, 0, kBK, kModeExact>(J, nullptr, 1, total_tiles, group, seg, st);
  return launch_variant<false, 4 * m, 256, 0, kBK, kModeExact>(J, nullptr, 1, total_tiles, group, seg, st);
}

cudaError_t dispatch_exact(int bn, int pair, int bk, const TcJob& J, long long total_tiles, int group, int seg,
                           cudaStream_t st) {
  if (bk == 64) return dispatch_exact_bk<64>(bn, pair, J, total_tiles, group, seg / 64, st);
  return dispatch_exact_bk<32>(bn, pair, J, total_tiles, group, seg / 32, st);
}

cudaError_t dispatch(bool split3, int bn, int pair, int bk, const TcJob& single, const TcJob* table, int njobs,
                     long long total_tiles, int group, int seg_kb, cudaStream_t st, bool twod = false) {
  if (twod) {
    if (bk == 32)
      return dispatch_bk<32, kMode2D>(split3, bn, pair, single, table, njobs, total_tiles, group, seg_kb, st);
    return dispatch_bk<64, kMode2D>(split3, bn, pair, single, table, njobs, total_tiles, group, seg_kb, st);
  }
  if (bk == 32) return dispatch_bk<32>(split3, bn, pair, single, table, njobs, total_tiles, group, seg_kb, st);
  return dispatch_bk<64>(split3, bn, pair, single, table, njobs, total_tiles, group, seg_kb, st);
}

// gemm_config: 0 = defaults (the fastest measured on the benchmark: 256x256
// tiles of CTA-pair MMAs, 64-wide k-slices, band 8, 512-wide K segments),
// else band * 1000 + seg_kb * 10 + tile (see tile_bn / tile_pair / tile_bk).
void decode_config(int config, int* group, int* seg_kb, int* bn, int* pair, int* bk) {
  *group = 8;
  *seg_kb = 8;
  *bn = 256;
  *pair = 2;
  *bk = 64;
  if (config > 0) {
    *group = 16;
    *seg_kb = 4;
    *bn = tile_bn(config);
    *pair = tile_pair(config);
    *bk = tile_bk(config);
    if ((config / 10) % 100 > 0) *seg_kb = (config / 10) % 100;
    if (config / 1000 > 0) *group = config / 1000;
  }
}

}  // namespace

namespace {

bool tc_fill_job(TcJob* J, const DevPlan& p, const void* a_hi, const void* a_lo, const void* b_hi,
                 const void* b_lo, int num_cells, int N, int K, int h, int bn, bool pair, int bk,
                 float* products, float* C_direct, int32_t* info_out, const int32_t* a_exp = nullptr,
                 const int32_t* b_exp = nullptr) {
  memset(J, 0, sizeof *J);
  const long long rows = static_cast<long long>(num_cells) * h;
  const int box_b = pair ? bn / 2 : bn;  // a paired CTA loads half of the B tile
  const bool f16 = a_exp != nullptr;
  if (!make_map(&J->map_ahi, a_hi, rows, K, BM, bk, f16) || !make_map(&J->map_bhi, b_hi, N, K, box_b, bk, f16))
    return false;
  J->a_exp = a_exp;
  J->b_exp = b_exp;
  if (a_lo) {
    if (!make_map(&J->map_alo, a_lo, rows, K, BM, bk, f16) || !make_map(&J->map_blo, b_lo, N, K, box_b, bk, f16))
      return false;
  } else {
    J->map_alo = J->map_ahi;
    J->map_blo = J->map_bhi;
  }
  J->ctr = p.ctr;
  J->surv = p.surv;
  J->direct = p.direct;
  J->info = p.info;
  J->info_out = info_out;
  J->products = products;
  J->C_direct = C_direct;
  J->N = N;
  J->K = K;
  J->h = h;
  J->m_tiles_max = static_cast<int>((rows + BM - 1) / BM);
  J->n_tiles = (N + bn - 1) / bn;
  J->tile_base = 0;
  return true;
}

}  // namespace

// Builds the device job table of a grouped GEMM for the given tile config:
// jobs ordered by decreasing K (longest tiles first, so the static striding
// of persistent CTAs over the tile space balances), tile_base prefix sums
// (in tiles, or in tile pairs for paired configs).  Copies the table to
// d_table (n * tc_job_bytes() bytes) and synchronises.
cudaError_t tc_build_table(const TcSpec* specs, int n, bool split3, int config, void* d_table,
                           long long* total_tiles, cudaStream_t st) {
  if (!tile_valid(config)) return cudaErrorInvalidValue;
  int group, seg_kb, bn, bk;
  int pair;
  decode_config(config, &group, &seg_kb, &bn, &pair, &bk);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return specs[a].K > specs[b].K; });
  std::vector<TcJob> tab(n);
  long long base = 0;
  for (int r = 0; r < n; ++r) {
    const TcSpec& S = specs[idx[r]];
    if (!tc_fill_job(&tab[r], S.p, S.a_hi, split3 ? S.a_lo : nullptr, S.b_hi, split3 ? S.b_lo : nullptr,
                     S.num_cells, S.N, S.K, S.h, bn, pair, bk, S.products, S.C_direct, S.info_out))
      return cudaErrorInvalidValue;
    tab[r].tile_base = base;
    const int units = pair ? (tab[r].m_tiles_max + 1) / 2 : tab[r].m_tiles_max;
    base += static_cast<long long>(units) * tab[r].n_tiles;
  }
  *total_tiles = base;
  cudaError_t e = cudaMemcpyAsync(d_table, tab.data(), sizeof(TcJob) * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

size_t tc_job_bytes() { return sizeof(TcJob); }

bool gemm_config_ok(int config) { return tile_valid(config); }

cudaError_t launch_gemm_tc(const DevGraph& g, const DevPlan& p, const void* a_hi, const void* a_lo,
                           const void* b_hi, const void* b_lo, int num_cells, int N, int K, int h,
                           bool split3, float* products, float* C_direct, int config,
                           int32_t* info_out, cudaStream_t st, const int32_t* a_exp, const int32_t* b_exp) {
  if (!tile_valid(config)) return cudaErrorInvalidValue;
  if ((a_exp != nullptr) != (b_exp != nullptr) || (a_exp && !split3)) return cudaErrorInvalidValue;
  (void)g;
  int group, seg_kb, bn, bk;
  int pair;
  decode_config(config, &group, &seg_kb, &bn, &pair, &bk);
  // split fp16: the default accumulates 128-wide K segments.  The truncating
  // TMEM adds would otherwise dominate its error: on the benchmark workload
  // 512-wide segments put 1.9e-6 on direct blocks, 256-wide 9.9e-7, 128-wide
  // 5.6e-7 (GEMM 2.05 / 2.10 / 2.27 ms), and on its worst peel chains
  // (propagation factor 32) 256-wide segments 9.2e-6, 128-wide 7.9e-6.
  if (a_exp && config == 0) seg_kb = 2;
  TcJob J;
  if (!tc_fill_job(&J, p, a_hi, split3 ? a_lo : nullptr, b_hi, split3 ? b_lo : nullptr, num_cells, N, K, h,
                   bn, pair, bk, products, C_direct, info_out, a_exp, b_exp))
    return cudaErrorInvalidValue;
  const int units = pair ? (J.m_tiles_max + 1) / 2 : J.m_tiles_max;
  const long long tiles = static_cast<long long>(units) * J.n_tiles;
  return dispatch(split3, bn, pair, bk, J, nullptr, 1, tiles, group, seg_kb, st);
}

// Exact-slice digit products: a_planes = coded rows x (S Kp) bf16, b_planes =
// N x (S Kp) bf16 (plane i of a row at column i Kp); diagonal d of cell c's
// product goes to planes + d * num_cells h N + c h N as int32.
cudaError_t launch_gemm_exact(const DevPlan& p, const void* a_planes, const void* b_planes, int num_cells, int N,
                              int K, int h, const ExactParams& P, int32_t* planes, int config, int32_t* info_out,
                              cudaStream_t st) {
  if (!tile_valid(config)) return cudaErrorInvalidValue;
  int group, seg_kb, bn, bk;
  int pair;
  // Default: 256x256 tiles of CTA-pair MMAs, 64-wide k-slices, bands of 8
  // (fastest measured; one MMA per k-slice and digit pair, so the wider
  // slice halves the stage hand-offs per MMA).
  decode_config(config > 0 ? config : 8080, &group, &seg_kb, &bn, &pair, &bk);
  TcJob J;
  if (!tc_fill_job(&J, p, a_planes, nullptr, b_planes, nullptr, num_cells, N, P.S * P.Kp, h, bn, pair, bk,
                   nullptr, nullptr, info_out))
    return cudaErrorInvalidValue;
  J.K = K;
  J.planes = planes;
  J.plane_stride = static_cast<long long>(num_cells) * h * N;
  J.ex_S = P.S;
  J.ex_Kp = P.Kp;
  const int units = pair ? (J.m_tiles_max + 1) / 2 : J.m_tiles_max;
  const long long tiles = static_cast<long long>(units) * J.n_tiles * P.S;
  return dispatch_exact(bn, pair, bk, J, tiles, group, P.seg, st);
}

// Two-dimensional scheme: A operands (EA x h rows) and B^T operands (EB x w
// rows) staged as bf16; every tile of every cell (erased cells' tiles are
// skipped) accumulates its cell's terms; h x w blocks go to products (cell c
// at c h w, row stride w) or, for depth-1 resolvers, to C (row stride N).
cudaError_t launch_gemm_2d(const DevGraph& g, const DevPlan& p, const void* a_hi, const void* a_lo, const void* b_hi,
                           const void* b_lo, int N, int K, int h, int w, bool split3, float* products,
                           float* C_direct, int config, int32_t* info_out, cudaStream_t st) {
  if (!tile_valid(config)) return cudaErrorInvalidValue;
  int group, seg_kb, bn, bk;
  int pair;
  decode_config(config, &group, &seg_kb, &bn, &pair, &bk);
  TcJob J;
  memset(&J, 0, sizeof J);
  const int box_b = pair ? bn / 2 : bn;
  const long long rows_a = static_cast<long long>(g.EA) * h, rows_b = static_cast<long long>(g.EB) * w;
  if (!make_map(&J.map_ahi, a_hi, rows_a, K, BM, bk) || !make_map(&J.map_bhi, b_hi, rows_b, K, box_b, bk))
    return cudaErrorInvalidValue;
  if (split3) {
    if (!make_map(&J.map_alo, a_lo, rows_a, K, BM, bk) || !make_map(&J.map_blo, b_lo, rows_b, K, box_b, bk))
      return cudaErrorInvalidValue;
  } else {
    J.map_alo = J.map_ahi;
    J.map_blo = J.map_bhi;
  }
  J.ctr = p.ctr;
  J.surv = p.surv;
  J.direct = p.direct;
  J.info = p.info;
  J.info_out = info_out;
  J.products = products;
  J.C_direct = C_direct;
  J.N = N;
  J.K = K;
  J.h = h;
  J.m_tiles_max = (h + BM - 1) / BM;
  J.n_tiles = (w + bn - 1) / bn;
  J.t2_ptr = g.t2_ptr;
  J.t2_a = g.t2_a;
  J.t2_b = g.t2_b;
  J.t2_order = g.t2_order;
  J.cnt = p.cnt;
  J.w2 = w;
  J.kc = g.k;
  J.ncells = g.num_cells;
  const int units = pair ? (J.m_tiles_max + 1) / 2 : J.m_tiles_max;
  const long long tiles = static_cast<long long>(units) * J.n_tiles * g.num_cells;
  return dispatch(split3, bn, pair, bk, J, nullptr, 1, tiles, group, seg_kb, st, true);
}

// Grouped launch over a device table of jobs (tile_base set, maps encoded).
cudaError_t launch_gemm_tc_grouped(const void* d_jobs, int njobs, long long total_tiles, bool split3,
                                   int config, cudaStream_t st) {
  if (!tile_valid(config)) return cudaErrorInvalidValue;
  int group, seg_kb, bn, bk;
  int pair;
  decode_config(config, &group, &seg_kb, &bn, &pair, &bk);
  TcJob dummy;
  memset(&dummy, 0, sizeof dummy);
  return dispatch(split3, bn, pair, bk, dummy, static_cast<const TcJob*>(d_jobs), njobs, total_tiles, group, seg_kb,
                  st);
}

}  // namespace bpx

extern "C" int bpx_selftest_wait_timeout(long long budget_cycles, int32_t* d_info, bpx_stream stream) {
  bpx::clear_error();
  if (!d_info || budget_cycles <= 0 || budget_cycles > bpx::kWaitBudget)
    return bpx::fail(BPX_ERR_INVAL, "bpx_selftest_wait_timeout: need d_info and 0 < budget <= %lld cycles",
                     bpx::kWaitBudget);
  bpx::wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(budget_cycles, d_info);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bpx::fail(BPX_ERR_CUDA, "bpx_selftest_wait_timeout: %s", cudaGetErrorString(e));
  return BPX_OK;
}
