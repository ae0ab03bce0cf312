// a1: symbolic peel.  One CTA turns an erasure mask into the peel plan:
// the surviving cells and, round by round, the sources that a surviving
// cell with exactly one unknown source resolves (Section I-A decoder read as
// parallel rounds).  Resolver = lowest such cell id; depth = the round; the
// recovered sources are then listed in (depth, source) order.
//
// Each round only touches the cells whose unknown count just dropped to one
// (a warp-parallel ready queue: one warp per ready cell, one warp per newly
// recovered source), so the cost is linear in the graph edges plus one short
// barrier sequence per round.  The plan also carries a flat "peel list" (per
// recovered source: its resolver and the blocks to subtract) for the numeric
// peel.
#include <climits>
#include <mutex>

#include "device_common.cuh"

namespace bpx {
namespace {

constexpr int kThreads = 1024;
constexpr size_t kSmemStateMax = 200 * 1024;  // bytes of per-cell + per-source state kept on chip

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

// kSmem: the per-cell unknown counts and per-source depths (the state every
// round reads and updates) live in shared memory when they fit, else in the
// plan's global arrays.
// cell_mask: the mask has one byte per cell (a processor whose output is
// missing) instead of one per column (a node).
// part: 0 = the whole plan; 1 = what the products need (surviving cells,
// their count and the depth-1 direct map, from the first round alone);
// 2 = the rest of the plan after a part-1 launch, leaving the arrays part 1
// wrote untouched (so that it may run while the products read them).
template <bool kSmem>
__device__ __forceinline__ void schedule_body(const DevGraph& g, const DevPlan& p,
                                              const uint8_t* __restrict__ mask, int32_t* peel_order,
                                              uint8_t* recovered, int32_t* info_out, bool cell_mask = false,
                                              int part = 0) {
  extern __shared__ int32_t dyn_smem[];
  __shared__ int s_warp[32];
  __shared__ int s_nf, s_new[2], s_next[2];  // per-round counters, by round parity
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  int32_t* cnt = kSmem ? dyn_smem : p.cnt;
  int32_t* depth = kSmem ? dyn_smem + g.num_cells : p.depth;

  for (int c = tid; c < g.num_cells; c += nt) {
    const bool alive = (cell_mask ? mask[c] : mask[g.col_of_cell[c]]) == 0;
    const int v = alive ? (g.cell_ptr[c + 1] - g.cell_ptr[c]) : -1;
    cnt[c] = v;
    if (kSmem) p.cnt[c] = v;  // the sign (erased column) is read by the two-dimensional GEMM
    if (part != 2) p.direct[c] = -1;
  }
  for (int s = tid; s < g.S; s += nt) {
    depth[s] = 0;
    p.resolver[s] = INT_MAX;
  }
  if (tid == 0) {
    s_nf = 0;
    s_new[0] = s_new[1] = s_next[0] = s_next[1] = 0;
    p.wave_ptr[0] = 0;
  }
  __syncthreads();

  // Surviving cells in ascending id, and the first ready queue (degree one).
  int nsurv = 0;
  for (int base = 0; base < g.num_cells; base += nt) {
    const int c = base + tid;
    const int f = (c < g.num_cells && cnt[c] >= 0) ? 1 : 0;
    int total;
    const int ex = block_exclusive_scan(f, s_warp, &total);
    if (f) {
      if (part != 2) p.surv[nsurv + ex] = c;
      if (cnt[c] == 1) p.front0[atomicAdd(&s_nf, 1)] = c;
    }
    nsurv += total;
  }
  __syncthreads();

  int32_t* fr = p.front0;
  int32_t* nx = p.front1;
  int round = 0, nrec = 0;
  int nf = s_nf;
  // Two barriers per round.  Counters of round r live at parity r & 1 and the
  // other parity is cleared during round r, after every thread has read it.
  const int max_rounds = part == 1 ? 1 : INT_MAX;
  while (nf > 0 && round < max_rounds) {
    ++round;
    const int q = round & 1;
    // A: one warp per ready cell (exactly one unknown source at the start of
    // the round): the lanes scan its support together for that source -- one
    // with depth 0, or depth == round if another cell of this round has
    // already claimed it -- the lowest cell id becomes its resolver, and the
    // first claim records it as recovered in this round.
    for (int i = warp; i < nf; i += nwarps) {
      const int c = fr[i];
      int found = -1;
      if (cnt[c] == 1) {
        const int e0 = g.cell_ptr[c], e1 = g.cell_ptr[c + 1];
        for (int base = e0; base < e1; base += 32) {
          const int e = base + lane;
          const int t = e < e1 ? g.cell_src[e] : -1;
          int dt = 0;
          if (t >= 0) dt = depth[t];
          const unsigned m = __ballot_sync(0xffffffffu, t >= 0 && (dt == 0 || dt == round));
          if (m) {
            found = __shfl_sync(0xffffffffu, t, __ffs(m) - 1);
            break;
          }
        }
      }
      if (lane == 0 && found >= 0) {
        atomicMin(&p.resolver[found], c);
        if (atomicCAS(&depth[found], 0, round) == 0) p.newsrc[atomicAdd(&s_new[q], 1)] = found;
      }
    }
    __syncthreads();
    const int nnew = s_new[q];
    if (nnew == 0) {
      --round;
      break;
    }
    nrec += nnew;
    if (tid == 0) {
      p.wave_ptr[round] = nrec;
      s_new[q ^ 1] = 0;
      s_next[q ^ 1] = 0;
    }
    // B: one warp per recovered source drops it from its cells; a cell whose
    // unknown count reaches one joins the next ready queue.
    for (int j = warp; j < nnew; j += nwarps) {
      const int s = p.newsrc[j];
      const int e1 = g.src_ptr[s + 1];
      for (int e = g.src_ptr[s] + lane; e < e1; e += 32) {
        const int c = g.src_cell[e];
        if (cnt[c] >= 0) {
          const int old = atomicSub(&cnt[c], 1);
          if (old == 2) nx[atomicAdd(&s_next[q], 1)] = c;
        }
      }
    }
    __syncthreads();
    nf = s_next[q];
    int32_t* tmp = fr;
    fr = nx;
    nx = tmp;
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
  // sources in ascending id; lanes of equal depth share one cursor bump.
  for (int d = 1 + tid; d <= round; d += nt) p.cursor[d] = p.wave_ptr[d - 1];
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
        pos = p.cursor[d];
        p.cursor[d] = pos + __popc(peers);
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
    int len = 0, r = 0;
    if (i < nrec) {
      r = p.resolver[p.order[i]];
      len = g.cell_ptr[r + 1] - g.cell_ptr[r] - 1;
    }
    int total;
    const int ex = block_exclusive_scan(len, s_warp, &total);
    if (i < nrec) {
      p.pl_res[i] = r;
      p.pl_ptr[i] = lbase + ex;
    }
    lbase += total;
  }
  if (tid == 0) p.pl_ptr[nrec] = lbase;
  __syncthreads();
  for (int i = warp; i < nrec; i += nwarps) {
    const int s = p.order[i], r = p.pl_res[i], o = p.pl_ptr[i];
    const int e0 = g.cell_ptr[r], e1 = g.cell_ptr[r + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
      const int t = g.cell_src[e];
      if (t != s) p.pl_list[o + (e - e0) - (t > s ? 1 : 0)] = t;
    }
  }
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
                uint8_t* recovered, int32_t* info_out, bool cell_mask, int part) {
  schedule_body<kSmem>(g, p, mask, peel_order, recovered, info_out, cell_mask, part);
}

// Grouped launch: CTA j plans job j.
template <bool kSmem>
__global__ void __launch_bounds__(kThreads, 1) schedule_group_kernel(const GJob* __restrict__ jobs) {
  const GJob& J = jobs[blockIdx.x];
  schedule_body<kSmem>(J.g, J.p, J.mask, nullptr, nullptr, J.info_out);
}

}  // namespace

cudaError_t launch_schedule_group(const GJob* d_jobs, int njobs, size_t max_state_bytes, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (max_state_bytes <= kSmemStateMax) {
    cudaError_t e = cudaFuncSetAttribute(schedule_group_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemStateMax));
    if (e != cudaSuccess) return e;
    schedule_group_kernel<true><<<njobs, kThreads, max_state_bytes, st>>>(d_jobs);
  } else {
    schedule_group_kernel<false><<<njobs, kThreads, 0, st>>>(d_jobs);
  }
  return cudaGetLastError();
}

cudaError_t launch_schedule(const DevGraph& g, const DevPlan& p, const uint8_t* mask,
                            int32_t* peel_order, uint8_t* recovered, int32_t* info_out,
                            cudaStream_t st, bool cell_mask, int part) {
  const size_t smem = (static_cast<size_t>(g.num_cells) + g.S) * sizeof(int32_t);
  // Small codes take a 256-thread block: it fits beside a resident GEMM CTA
  // (registers), so the schedule of one multiplication can run while the
  // GEMM of another still holds every SM.
  const int threads = g.num_cells + g.S <= 4096 ? 256 : kThreads;
  if (smem <= kSmemStateMax) {
    cudaError_t e = cudaFuncSetAttribute(schedule_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemStateMax));
    if (e != cudaSuccess) return e;
    schedule_kernel<true><<<1, threads, smem, st>>>(g, p, mask, peel_order, recovered, info_out, cell_mask, part);
  } else {
    schedule_kernel<false><<<1, threads, 0, st>>>(g, p, mask, peel_order, recovered, info_out, cell_mask, part);
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

