// a1: symbolic peel.  One CTA turns an erasure mask into the peel plan:
// the surviving cells and, round by round, the sources that a surviving
// cell with exactly one unknown source resolves (Section I-A decoder read as
// parallel rounds).  Resolver = lowest such cell id; depth = the round; the
// recovered sources are then listed in (depth, source) order.
//
// Each cell keeps one word: its count of unknown sources above the XOR of
// its unknown sources' ids + 1.  A round walks only the sources recovered in
// the round before (one warp per source, lanes over its cells): each lane
// XORs the source out of the cell's word and then decrements the count; the
// lane that takes a count from two to one reads, in the word its decrement
// returned, the one source the cell still lacks -- unless a source of the
// same round is still on its way out, in which case the id found is that
// source's (already recovered, so no claim) or zero.  Every source recovered
// in a round already carries its depth when the round's decrements start, so
// the claim test (depth 0, or depth = next round when another cell got there
// first) is exact, and the claims for round r + 1 happen inside round r:
// one barrier per round, two dependent graph loads (the source's cell range
// and its cells).  The ready lists live in shared memory (overflow in the
// plan's frontier arrays).  The plan also carries a flat "peel list" (per
// recovered source: its resolver and the blocks to subtract) for the numeric
// peel.
#include <algorithm>
#include <climits>
#include <mutex>

#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int kThreads = 1024;
constexpr size_t kSmemMax = 224 * 1024;  // dynamic shared memory of a plan's CTA (state + ready lists)
constexpr size_t kSmemSmall = 16 * 1024;  // the same for the 256-thread CTA of small codes

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const int before = warp > 0 ? s_warp[warp - 1] : 0;
  *total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

// The per-cell word: 32 bits in shared memory (when the count fits above the
// id bits), 64 bits in the plan otherwise.
template <bool kSmem>
struct CellWord {
  using T = uint32_t;
};
template <>
struct CellWord<false> {
  using T = unsigned long long;
};

// kSmem: the per-cell words and per-source depths (the state every round
// reads and updates) live in shared memory, followed by the two ready lists
// (list_cap entries each); otherwise in the plan's global arrays.
// cell_mask: the mask has one byte per cell (a processor whose output is
// missing) instead of one per column (a node).
// part: 0 = the whole plan; 1 = what the products need (surviving cells,
// their count and the depth-1 direct map, from the first round alone);
// 2 = the rest of the plan after a part-1 launch, leaving the arrays part 1
// wrote untouched (so that it may run while the products read them).
template <bool kSmem>
__device__ __forceinline__ void schedule_body(const DevGraph& g, const DevPlan& p,
                                              const uint8_t* __restrict__ mask, int32_t* peel_order,
                                              uint8_t* recovered, int32_t* info_out, bool cell_mask, int part,
                                              int list_cap) {
  using W = typename CellWord<kSmem>::T;
  constexpr int kTop = static_cast<int>(sizeof(W)) * 8 - 1;  // set only in an erased cell's word
  extern __shared__ int32_t dyn_smem[];
  __shared__ int s_warp[32];
  __shared__ int s_cnt[3];  // ready-list lengths, round r at r % 3
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int shift = kSmem ? sched_id_bits(g.S) : 32;
  const W xmask = (W(1) << shift) - 1;
  const W erased = ~W(0);
  const W dec = W(0) - (W(1) << shift);
  W* word = kSmem ? reinterpret_cast<W*>(dyn_smem) : reinterpret_cast<W*>(p.word);
  int32_t* depth = kSmem ? dyn_smem + g.num_cells : p.depth;
  int32_t* lists = kSmem ? dyn_smem + g.num_cells + g.S : nullptr;
  if (!kSmem) list_cap = 0;
  // entry i of ready list q (round r's list is q = r & 1)
  auto list_at = [&](int q, int i) -> int32_t* {
    return i < list_cap ? lists + q * list_cap + i : (q ? p.front1 : p.front0) + i;
  };
  // cell c, with w its one unknown source, claims w for round r
  auto claim = [&](int c, int w, int r) {
    atomicMin(&p.resolver[w], c);
    if (atomicCAS(&depth[w], 0, r) == 0) *list_at(r & 1, atomicAdd(&s_cnt[r % 3], 1)) = w;
  };

  for (int c = tid; c < g.num_cells; c += nt) {
    const bool alive = (cell_mask ? mask[c] : mask[g.col_of_cell[c]]) == 0;
    const int e0 = g.cell_ptr[c], e1 = g.cell_ptr[c + 1];
    W v = erased;
    if (alive) {
      W x = 0;
      for (int e = e0; e < e1; ++e) x ^= static_cast<W>(g.cell_src[e] + 1);
      v = (static_cast<W>(e1 - e0) << shift) | x;
    }
    word[c] = v;
    p.cnt[c] = alive ? e1 - e0 : -1;  // the sign (erased column) is read by the two-dimensional GEMM
    if (part != 2) p.direct[c] = -1;
  }
  for (int s = tid; s < g.S; s += nt) {
    depth[s] = 0;
    p.resolver[s] = INT_MAX;
  }
  if (tid == 0) {
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    p.wave_ptr[0] = 0;
  }
  __syncthreads();

  // Surviving cells in ascending id; the degree-one ones claim their source
  // for round 1.
  int nsurv = 0;
  for (int base = 0; base < g.num_cells; base += nt) {
    const int c = base + tid;
    const W v = c < g.num_cells ? word[c] : erased;
    const int f = (v >> kTop) == 0 ? 1 : 0;
    int total;
    const int ex = block_exclusive_scan(f, s_warp, &total);
    if (f) {
      if (part != 2) p.surv[nsurv + ex] = c;
      if ((v >> shift) == 1) claim(c, static_cast<int>(v & xmask) - 1, 1);
    }
    nsurv += total;
  }
  __syncthreads();

  const int max_rounds = part == 1 ? 1 : INT_MAX;
  int round = 1, nrec = 0;
  for (;;) {
    const int nr = s_cnt[round % 3];
    if (nr == 0) {
      --round;
      break;
    }
    nrec += nr;
    if (tid == 0) {
      p.wave_ptr[round] = nrec;
      s_cnt[(round + 2) % 3] = 0;  // round - 1's length: every thread read it before the last barrier
    }
    if (round >= max_rounds) break;
    const int q = round & 1;
    for (int j = warp; j < nr; j += nwarps) {
      const int s = *list_at(q, j);
      const int e1 = g.src_ptr[s + 1];
      for (int e = g.src_ptr[s] + lane; e < e1; e += 32) {
        const int c = g.src_cell[e];
        if ((word[c] >> kTop) == 0) {  // a surviving cell (its top bit never changes)
          atomicXor(&word[c], static_cast<W>(s + 1));
          const W old = atomicAdd(&word[c], dec);
          if ((old >> shift) == 2) {
            const W x = old & xmask;
            if (x != 0 && x <= static_cast<W>(g.S)) {
              const int w = static_cast<int>(x) - 1;
              const int dw = *reinterpret_cast<volatile int32_t*>(&depth[w]);
              if (dw == 0 || dw == round + 1) claim(c, w, round + 1);
            }
          }
        }
      }
    }
    __syncthreads();
    ++round;
  }

  if (part == 1) {
    // what the products need: the depth-1 direct map and the survivor count
    __syncthreads();
    for (int s = tid; s < g.S; s += nt)
      if (depth[s] == 1) p.direct[p.resolver[s]] = s;
    if (tid == 0) {
      p.ctr[CTR_NSURV] = nsurv;
      p.ctr[CTR_PLAN] = 0;  // the rest of the plan follows (part 2)
      p.info[BPX_INFO_DEVICE_ERR] = 0;  // cleared before the products run
    }
    return;
  }

  // Place the recovered sources in (depth, source) order: one warp walks the
  // sources in ascending id; lanes of equal depth share one cursor bump.  The
  // cursors take the ready lists' shared memory when they fit.
  int32_t* cur = (kSmem && round + 1 <= 2 * list_cap) ? lists : p.cursor;
  for (int d = 1 + tid; d <= round; d += nt) cur[d] = p.wave_ptr[d - 1];
  __syncthreads();
  if (tid < 32) {
    for (int base = 0; base < g.S; base += 32) {
      const int s = base + lane;
      const int d = s < g.S ? depth[s] : 0;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int pos = 0;
      if (lane == leader && d > 0) {
        pos = cur[d];
        cur[d] = pos + __popc(peers);
      }
      pos = __shfl_sync(0xffffffffu, pos, leader);
      if (d > 0) p.order[pos + rank] = s;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int s = tid; s < g.S; s += nt) {
    const int d = depth[s];
    if (kSmem) p.depth[s] = d;
    if (d == 1 && part != 2) p.direct[p.resolver[s]] = s;
    if (recovered) recovered[s] = d > 0 ? 1 : 0;
  }
  // Peel list: for order position i, the resolver and the other sources of
  // its support (ascending), so the numeric peel reads flat descriptors.
  int lbase = 0;
  for (int base = 0; base < nrec; base += nt) {
    const int i = base + tid;
    int len = 0, r = 0, s = 0, e0 = 0, e1 = 0;
    if (i < nrec) {
      s = p.order[i];
      r = p.resolver[s];
      e0 = g.cell_ptr[r];
      e1 = g.cell_ptr[r + 1];
      len = e1 - e0 - 1;
    }
    int total;
    const int ex = block_exclusive_scan(len, s_warp, &total);
    if (i < nrec) {
      int o = lbase + ex;
      p.pl_res[i] = r;
      p.pl_ptr[i] = o;
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const int t = g.cell_src[e];
        if (t != s) p.pl_list[o++] = t;
      }
    }
    lbase += total;
  }
  if (tid == 0) p.pl_ptr[nrec] = lbase;
  if (peel_order) {
    for (int i = tid; i < g.S; i += nt) {
      if (i < nrec) {
        const int s = p.order[i];
        peel_order[3 * i + 0] = s;
        peel_order[3 * i + 1] = p.resolver[s];
        peel_order[3 * i + 2] = depth[s];
      } else {
        peel_order[3 * i + 0] = -1;
        peel_order[3 * i + 1] = -1;
        peel_order[3 * i + 2] = -1;
      }
    }
  }
  if (tid == 0) {
    p.ctr[CTR_NSURV] = nsurv;
    p.ctr[CTR_NWAVES] = round;
    p.ctr[CTR_NREC] = nrec;
    p.ctr[CTR_ERR] = 0;
    p.ctr[CTR_PLAN] = kPlanReady;
    int32_t inf[BPX_INFO_LEN];
    for (int i = 0; i < BPX_INFO_LEN; ++i) inf[i] = 0;
    // part 2 runs beside the products: keep a self-check error they raised
    const int32_t dev_err = part == 2 ? atomicAdd(&p.info[BPX_INFO_DEVICE_ERR], 0) : 0;
    inf[BPX_INFO_STATUS] = dev_err ? dev_err : ((nrec == g.S) ? BPX_OK : BPX_ERR_UNDECODABLE);
    inf[BPX_INFO_DEVICE_ERR] = dev_err;
    inf[BPX_INFO_RECOVERED] = nrec;
    inf[BPX_INFO_WAVES] = round;
    inf[BPX_INFO_SURVIVING] = nsurv;
    inf[BPX_INFO_DIRECT] = round >= 1 ? p.wave_ptr[1] : 0;
    for (int i = 0; i < BPX_INFO_LEN; ++i) {
      if (i == BPX_INFO_DEVICE_ERR || i == BPX_INFO_STATUS) {
        if (dev_err) continue;  // left as the products' atomic writes set them
      }
      p.info[i] = inf[i];
      if (info_out) info_out[i] = inf[i];
    }
  }
}

template <bool kSmem>
__global__ void __launch_bounds__(kThreads, 1)
schedule_kernel(DevGraph g, DevPlan p, const uint8_t* __restrict__ mask, int32_t* peel_order,
                uint8_t* recovered, int32_t* info_out, bool cell_mask, int part, int list_cap) {
  schedule_body<kSmem>(g, p, mask, peel_order, recovered, info_out, cell_mask, part, list_cap);
}

// Grouped launch: CTA j plans job j; smem_ints: the launch's dynamic shared
// memory in int32 words (each job's ready lists take what its state leaves).
template <bool kSmem>
__global__ void __launch_bounds__(kThreads, 1) schedule_group_kernel(const GJob* __restrict__ jobs, int smem_ints) {
  const GJob& J = jobs[blockIdx.x];
  int cap = 0;
  if (kSmem) cap = max(0, min(J.g.S, (smem_ints - J.g.num_cells - J.g.S) / 2));
  schedule_body<kSmem>(J.g, J.p, J.mask, nullptr, nullptr, J.info_out, false, 0, cap);
}

}  // namespace

cudaError_t launch_schedule_group(const GJob* d_jobs, int njobs, size_t max_state_bytes, size_t max_want_bytes,
                                  bool packable, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (packable && max_state_bytes <= kSmemMax) {
    const size_t smem = std::min(kSmemMax, std::max(max_state_bytes, max_want_bytes));
    cudaError_t e = cudaFuncSetAttribute(schedule_group_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemMax));
    if (e != cudaSuccess) return e;
    schedule_group_kernel<true><<<njobs, kThreads, smem, st>>>(d_jobs, static_cast<int>(smem / 4));
  } else {
    schedule_group_kernel<false><<<njobs, kThreads, 0, st>>>(d_jobs, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_schedule(const DevGraph& g, const DevPlan& p, const uint8_t* mask,
                            int32_t* peel_order, uint8_t* recovered, int32_t* info_out,
                            cudaStream_t st, bool cell_mask, int part) {
  const long long state = static_cast<long long>(g.num_cells) + g.S;  // int32 words
  // Small codes take a 256-thread block with at most 16 KB of shared memory:
  // it fits beside a resident GEMM CTA, so the schedule of one
  // multiplication can run while the GEMM of another still holds every SM.
  const bool small = state <= 4096;
  const int threads = small ? 256 : kThreads;
  const long long room = static_cast<long long>((small ? kSmemSmall : kSmemMax) / 4);
  if (sched_packable32(g.S, g.sigma) && state <= room) {
    const int cap = static_cast<int>(std::min<long long>(g.S, (room - state) / 2));
    const size_t smem = static_cast<size_t>(state + 2LL * cap) * sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(schedule_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemMax));
    if (e != cudaSuccess) return e;
    schedule_kernel<true><<<1, threads, smem, st>>>(g, p, mask, peel_order, recovered, info_out, cell_mask, part,
                                                    cap);
  } else {
    schedule_kernel<false><<<1, threads, 0, st>>>(g, p, mask, peel_order, recovered, info_out, cell_mask, part, 0);
  }
  return cudaGetLastError();
}

}  // namespace bpx

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot allocate device memory themselves: code that runs inside
// a host runtime which owns the whole device pool (a raw cudaMalloc would
// bypass its accounting or fail against its cap), or latency-critical callers
// that cannot afford the device-wide synchronisation cudaMalloc / cudaFree
// imply.  For them bpx_schedule_noalloc runs the same schedule kernel with its
// scratch (graph copy + peel plan) in the fixed array below instead of a
// caller workspace.  Every GPU that loads this library keeps the array until
// the process exits.
namespace bpx {
namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;  // 8 MiB
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocBytes / sizeof(int32_t)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

}  // namespace bpx

extern "C" int bpx_schedule_noalloc(const bpx_code* c, const uint8_t* d_mask, int32_t* d_peel_order,
                                    uint8_t* d_recovered, int32_t* d_info, bpx_stream stream) {
  using bpx::fail;
  bpx::clear_error();
  if (!c) return fail(BPX_ERR_INVAL, "bpx_schedule_noalloc: code is NULL");
  if (!d_mask) return fail(BPX_ERR_INVAL, "bpx_schedule_noalloc: erasure mask is NULL");
  const bpx::WsLayout L = bpx::ws_layout(c, 0, 0, 0, 1, BPX_FP32);
  if (L.total > bpx::kNoAllocBytes)
    return fail(BPX_ERR_INVAL,
                "bpx_schedule_noalloc: this code needs %zu bytes of scratch, more than the fixed "
                "%zu-byte array; use bpx_schedule with a workspace",
                L.total, bpx::kNoAllocBytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(BPX_ERR_CUDA, "bpx_schedule_noalloc: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= bpx::kMaxDevices) return fail(BPX_ERR_UNSUPPORTED, "device id %d too large", dev);
  void* base = nullptr;
  {
    // First call on a device: look up the array's device address with that
    // device current (the array's name is only a host-side stand-in).
    std::lock_guard<std::mutex> lk(bpx::g_noalloc_mu);
    if (!bpx::g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, bpx::g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(BPX_ERR_CUDA, "bpx_schedule_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      bpx::g_noalloc_ptr[dev] = p;
    }
    base = bpx::g_noalloc_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* b = static_cast<char*>(base);
  struct Part {
    size_t off;
    const void* src;
    size_t bytes;
  } parts[] = {
      {L.g_col_of_cell, c->col_of_cell.data(), c->col_of_cell.size() * 4},
      {L.g_cell_ptr, c->cell_ptr.data(), c->cell_ptr.size() * 4},
      {L.g_cell_src, c->cell_src.data(), c->cell_src.size() * 4},
      {L.g_src_ptr, c->src_ptr.data(), c->src_ptr.size() * 4},
      {L.g_src_cell, c->src_cell.data(), c->src_cell.size() * 4},
  };
  // The graph of this call's code replaces whatever the previous call left;
  // the kernel initialises every plan array it reads.
  for (const Part& pt : parts) {
    if (pt.bytes == 0) continue;
    e = cudaMemcpyAsync(b + pt.off, pt.src, pt.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(BPX_ERR_CUDA, "bpx_schedule_noalloc: copy: %s", cudaGetErrorString(e));
  }
  const bpx::DevGraph g = bpx::make_graph(c, base, L);
  const bpx::DevPlan p = bpx::make_plan(base, L);
  e = bpx::launch_schedule(g, p, d_mask, d_peel_order, d_recovered, d_info, st);
  if (e != cudaSuccess) return fail(BPX_ERR_CUDA, "bpx_schedule_noalloc: launch: %s", cudaGetErrorString(e));
  return BPX_OK;
}

