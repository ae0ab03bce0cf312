// Batches: many independent coded multiplications -- each with its own code,
// shapes, erasure mask and buffers -- run as one launch per stage over all
// of them (symbolic peel, B split, encode + split, grouped tcgen05 GEMM,
// numeric peel).  A group is planned once on the host; the runs need no host
// synchronisation and no allocation, so they can be captured into a CUDA
// graph and replayed.  Also the tile autotuners (single job and group).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device_common.cuh"

using bpx::fail;

struct bpx_group {
  int precision = BPX_BF16X3;
  std::vector<bpx_job> jobs;
  std::vector<bpx::WsLayout> layouts;
  std::vector<size_t> offsets;
  size_t gjob_off = 0, tc_off = 0, total = 0;
  size_t max_state_bytes = 0, max_want_bytes = 0;
  int max_sigma = 1;
  bool sched_packable = true;  // every job's schedule state fits 32-bit cell words
  long long bsplit_total = 0, enc_total = 0, peel_total = 0, tiles_total = 0;
  void* ws = nullptr;
  int table_config = -1;  // tile config the device GEMM table was built for
  int tuned_config = 0;   // the autotuner's choice (0 = defaults)
  std::vector<bpx::TcSpec> specs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_key[5] = {0, 0, 0, 0, 0};
  int peel_target = 0;                // peel CTAs aimed at per job (0 = 4 x the SM count)
  std::vector<bpx::GJob> host_jobs;   // the device job table's host copy (re-planned peels)
  // peel launch order: the jobs in the gathered form first, then the rest
  size_t order_off = 0;
  // the grouped launches' first CTA per job: B split and encode (job order),
  // peel (peel order), three dense arrays of njobs
  size_t bases_off = 0;
  std::vector<int32_t> peel_order;
  int peel_ngather = 0;
  long long peel_gather_ctas = 0;
  cudaStream_t side = nullptr;        // the B split beside the schedule; the register-path peel beside the gathered one
  cudaEvent_t fork = nullptr, join = nullptr, fork_b = nullptr, join_b = nullptr;
};

namespace {

cudaStream_t S(bpx_stream s) { return static_cast<cudaStream_t>(s); }

int cuda_fail(cudaError_t e, const char* what) {
  return fail(BPX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void mark(const bpx_opts* o, int stage, int end, cudaStream_t st) {
  if (!o || !o->stage_events) return;
  void* ev = o->stage_events[2 * stage + end];
  if (ev) cudaEventRecord(static_cast<cudaEvent_t>(ev), st);
}

// The device GEMM table depends on the tile shape and pairing (gemm_config % 10).
int tile_of(int config) { return config % 10; }  // the default (0) is tile 0

// (Re)builds the device GEMM table when the tile width changes.
int ensure_table(bpx_group* G, int config, cudaStream_t st) {
  const int want = tile_of(config);
  if (G->table_config >= 0 && tile_of(G->table_config) == want) return BPX_OK;
  cudaError_t e = bpx::tc_build_table(G->specs.data(), static_cast<int>(G->specs.size()),
                                      G->precision == BPX_BF16X3, config,
                                      static_cast<char*>(G->ws) + G->tc_off, &G->tiles_total, st);
  if (e != cudaSuccess) return cuda_fail(e, "grouped GEMM table");
  G->table_config = config;
  return BPX_OK;
}

// The grouped peel's launch plan: each job's float4 columns cut into chunks
// so that the job gets about G->peel_target CTAs (0: 4 x the SM count); the
// jobs whose peel takes the gathered form (tall codes) first, then the rest,
// their CTA ranges laid end to end in that order.
void plan_peel(bpx_group* G) {
  const int njobs = static_cast<int>(G->host_jobs.size());
  std::vector<int32_t> gat, reg;
  for (int j = 0; j < njobs; ++j) {
    auto& g = G->host_jobs[j];
    const long long nv = static_cast<long long>(g.h) * g.N / 4;
    g.peel_chunk = bpx::peel_chunk_for(nv, G->peel_target);
    const bpx_code* c = G->jobs[j].code;
    (bpx::peel_gather_ok(c->S, c->sigma, g.peel_chunk) ? gat : reg).push_back(j);
  }
  long long pe = 0;
  auto lay = [&](const std::vector<int32_t>& js) {
    for (int j : js) {
      auto& g = G->host_jobs[j];
      const long long nv = static_cast<long long>(g.h) * g.N / 4;
      g.peel_base = pe;
      pe += (nv + g.peel_chunk - 1) / g.peel_chunk;
    }
  };
  lay(gat);
  G->peel_gather_ctas = pe;
  lay(reg);
  G->peel_total = pe;
  G->peel_ngather = static_cast<int>(gat.size());
  G->peel_order = gat;
  G->peel_order.insert(G->peel_order.end(), reg.begin(), reg.end());
}

const long long* bases(const bpx_group* G, int which) {  // 0: B split, 1: encode, 2: peel
  return reinterpret_cast<const long long*>(static_cast<char*>(G->ws) + G->bases_off) + which * G->jobs.size();
}

// Uploads the job table, the peel order and the base arrays (after plan_peel).
cudaError_t upload_jobs(bpx_group* G, cudaStream_t st) {
  const size_t njobs = G->host_jobs.size();
  std::vector<long long> b(3 * njobs);
  for (size_t j = 0; j < njobs; ++j) {
    b[j] = G->host_jobs[j].bsplit_base;
    b[njobs + j] = G->host_jobs[j].enc_base;
    b[2 * njobs + j] = G->host_jobs[G->peel_order[j]].peel_base;
  }
  cudaError_t e = cudaMemcpyAsync(static_cast<char*>(G->ws) + G->gjob_off, G->host_jobs.data(),
                                  sizeof(bpx::GJob) * njobs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<char*>(G->ws) + G->order_off, G->peel_order.data(), sizeof(int32_t) * njobs,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<char*>(G->ws) + G->bases_off, b.data(), sizeof(long long) * b.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
  return e;
}

cudaError_t launch_group_peel(bpx_group* G, int comp, cudaStream_t st) {
  const auto* gj = reinterpret_cast<const bpx::GJob*>(static_cast<char*>(G->ws) + G->gjob_off);
  const auto* order = reinterpret_cast<const int32_t*>(static_cast<char*>(G->ws) + G->order_off);
  return bpx::launch_peel_group(gj, order, bases(G, 2), static_cast<int>(G->jobs.size()), G->peel_ngather,
                                G->peel_gather_ctas, G->peel_total, 2, comp, G->max_sigma, st, G->side, G->fork,
                                G->join);
}

int run_group(bpx_group* G, const bpx_opts* o, int config, cudaStream_t st) {
  const int njobs = static_cast<int>(G->jobs.size());
  const auto* gj = reinterpret_cast<const bpx::GJob*>(static_cast<char*>(G->ws) + G->gjob_off);
  const bool split = G->precision == BPX_BF16X3;
  const int direct = o ? o->direct_write : 1;
  const int comp = o ? o->compensate_depth : -1;
  cudaError_t e;
  // The B split needs no plan: it runs on the side stream beside the
  // schedule (whose tallest jobs take hundreds of dependent rounds), issued
  // after it so that the schedule's CTAs are placed first.
  if ((e = cudaEventRecord(G->fork_b, st)) != cudaSuccess) return cuda_fail(e, "grouped B split fork");
  mark(o, BPX_STAGE_SCHEDULE, 0, st);
  if ((e = bpx::launch_schedule_group(gj, njobs, G->max_state_bytes, G->max_want_bytes, G->sched_packable, st)) != cudaSuccess)
    return cuda_fail(e, "grouped schedule");
  mark(o, BPX_STAGE_SCHEDULE, 1, st);
  if ((e = cudaStreamWaitEvent(G->side, G->fork_b, 0)) != cudaSuccess) return cuda_fail(e, "grouped B split fork");
  mark(o, BPX_STAGE_B_PREP, 0, G->side);
  if ((e = bpx::launch_b_split_group(gj, bases(G, 0), njobs, G->bsplit_total, G->side)) != cudaSuccess)
    return cuda_fail(e, "grouped B split");
  mark(o, BPX_STAGE_B_PREP, 1, G->side);
  if ((e = cudaEventRecord(G->join_b, G->side)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, G->join_b, 0)) != cudaSuccess)
    return cuda_fail(e, "grouped B split join");
  mark(o, BPX_STAGE_A_PREP, 0, st);
  if ((e = bpx::launch_encode_split_group(gj, bases(G, 1), njobs, G->enc_total, split, st)) != cudaSuccess)
    return cuda_fail(e, "grouped encode");
  mark(o, BPX_STAGE_A_PREP, 1, st);
  mark(o, BPX_STAGE_GEMM, 0, st);
  if ((e = bpx::launch_gemm_tc_grouped(static_cast<char*>(G->ws) + G->tc_off, njobs, G->tiles_total, split,
                                       config, st)) != cudaSuccess)
    return cuda_fail(e, "grouped GEMM");
  mark(o, BPX_STAGE_GEMM, 1, st);
  (void)direct;
  mark(o, BPX_STAGE_PEEL, 0, st);
  if ((e = launch_group_peel(G, comp, st)) != cudaSuccess) return cuda_fail(e, "grouped peel");
  mark(o, BPX_STAGE_PEEL, 1, st);
  return BPX_OK;
}

}  // namespace

extern "C" int bpx_group_create(const bpx_job* jobs, int njobs, int precision, bpx_group** out) {
  bpx::clear_error();
  if (!out) return fail(BPX_ERR_INVAL, "bpx_group_create: out is NULL");
  *out = nullptr;
  if (!jobs || njobs <= 0) return fail(BPX_ERR_INVAL, "bpx_group_create: no jobs");
  if (precision != BPX_BF16X3 && precision != BPX_BF16)
    return fail(BPX_ERR_UNSUPPORTED, "grouped runs support BPX_BF16 and BPX_BF16X3");
  auto* G = new bpx_group();
  G->precision = precision;
  G->jobs.assign(jobs, jobs + njobs);
  size_t off = 0;
  for (int j = 0; j < njobs; ++j) {
    const bpx_job& J = jobs[j];
    const bpx_code* c = J.code;
    if (!c || !J.A || !J.B || !J.C || !J.erasure_mask || J.M < 0 || J.N <= 0 || J.K <= 0 || J.h <= 0 ||
        J.N % 4 || J.K % 8 || static_cast<long long>(J.M) > static_cast<long long>(c->S) * J.h) {
      delete G;
      return fail(BPX_ERR_INVAL, "bpx_group_create: job %d has a bad argument", j);
    }
    const bpx::WsLayout L = bpx::ws_layout(c, J.M, J.N, J.K, J.h, precision);
    G->layouts.push_back(L);
    G->offsets.push_back(off);
    off = bpx::align_up(off + L.total, 256);
    G->max_state_bytes =
        std::max(G->max_state_bytes, (static_cast<size_t>(c->num_cells) + c->S) * sizeof(int32_t));
    G->max_want_bytes =
        std::max(G->max_want_bytes, (static_cast<size_t>(c->num_cells) + 3 * static_cast<size_t>(c->S)) * sizeof(int32_t));
    G->max_sigma = std::max(G->max_sigma, c->sigma);
    G->sched_packable = G->sched_packable && bpx::sched_packable32(c->S, c->sigma);
  }
  G->gjob_off = off;
  off = bpx::align_up(off + sizeof(bpx::GJob) * njobs, 256);
  G->order_off = off;
  off = bpx::align_up(off + sizeof(int32_t) * njobs, 256);
  G->bases_off = off;
  off = bpx::align_up(off + 3 * sizeof(long long) * njobs, 256);
  G->tc_off = off;
  off = bpx::align_up(off + bpx::tc_job_bytes() * njobs, 256);
  G->total = off;
  *out = G;
  return BPX_OK;
}

extern "C" size_t bpx_group_workspace_bytes(const bpx_group* G) { return G ? G->total : 0; }

extern "C" int bpx_group_init(bpx_group* G, void* ws, size_t ws_bytes, bpx_stream stream) {
  bpx::clear_error();
  if (!G || !ws) return fail(BPX_ERR_INVAL, "bpx_group_init: NULL argument");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(BPX_ERR_INVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < G->total) return fail(BPX_ERR_NOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, G->total);
  cudaStream_t st = S(stream);
  G->ws = ws;
  const int njobs = static_cast<int>(G->jobs.size());
  std::vector<bpx::GJob> gj(njobs);
  G->specs.assign(njobs, bpx::TcSpec{});
  long long bs = 0, en = 0;
  for (int j = 0; j < njobs; ++j) {
    const bpx_job& J = G->jobs[j];
    const bpx_code* c = J.code;
    void* base = static_cast<char*>(ws) + G->offsets[j];
    if (int rc = bpx_workspace_init(c, base, G->layouts[j].total, stream)) return rc;
    const bpx::WsLayout& L = G->layouts[j];
    bpx::GJob& g = gj[j];
    g.g = bpx::make_graph(c, base, L);
    g.p = bpx::make_plan(base, L);
    g.A = J.A;
    g.B = J.B;
    g.C = J.C;
    g.products = reinterpret_cast<float*>(static_cast<char*>(base) + L.products);
    g.mask = J.erasure_mask;
    g.info_out = J.info;
    g.a_hi = static_cast<char*>(base) + L.a_hi;
    g.a_lo = G->precision == BPX_BF16X3 ? static_cast<char*>(base) + L.a_lo : nullptr;
    g.b_hi = static_cast<char*>(base) + L.b_hi;
    g.b_lo = G->precision == BPX_BF16X3 ? static_cast<char*>(base) + L.b_lo : nullptr;
    g.M = J.M;
    g.N = J.N;
    g.K = J.K;
    g.h = J.h;
    g.bsplit_base = bs;
    bs += bpx::bsplit_ctas(J.N, J.K);
    g.enc_base = en;
    g.enc_sblocks = static_cast<int>(bpx::enc_group_sblocks(static_cast<long long>(c->num_cells) * J.h, J.K));
    en += bpx::encode_group_ctas(static_cast<long long>(c->num_cells) * J.h, J.K);
    bpx::TcSpec& sp = G->specs[j];
    sp.p = g.p;
    sp.a_hi = g.a_hi;
    sp.a_lo = g.a_lo;
    sp.b_hi = g.b_hi;
    sp.b_lo = g.b_lo;
    sp.num_cells = c->num_cells;
    sp.N = J.N;
    sp.K = J.K;
    sp.h = J.h;
    sp.products = g.products;
    sp.C_direct = J.C;
    sp.info_out = J.info;
  }
  G->bsplit_total = bs;
  G->enc_total = en;
  G->host_jobs = gj;
  plan_peel(G);
  cudaError_t e = cudaSuccess;
  if (!G->side) e = cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && !G->fork) e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !G->join) e = cudaEventCreateWithFlags(&G->join, cudaEventDisableTiming);
  if (e == cudaSuccess && !G->fork_b) e = cudaEventCreateWithFlags(&G->fork_b, cudaEventDisableTiming);
  if (e == cudaSuccess && !G->join_b) e = cudaEventCreateWithFlags(&G->join_b, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e, "bpx_group_init: side stream and events");
  if ((e = upload_jobs(G, st)) != cudaSuccess) return cuda_fail(e, "bpx_group_init: job table");
  G->table_config = -1;
  return ensure_table(G, G->tuned_config, st);
}

extern "C" int bpx_grouped_run(bpx_group* G, const bpx_opts* opts, bpx_stream stream) {
  bpx::clear_error();
  if (!G || !G->ws) return fail(BPX_ERR_INVAL, "bpx_grouped_run: group not initialised");
  const int config = (opts && opts->gemm_config) ? opts->gemm_config : G->tuned_config;
  if (!bpx::gemm_config_ok(config)) return fail(BPX_ERR_INVAL, "bpx_grouped_run: gemm_config %d names no tile", config);
  if (tile_of(config) != tile_of(G->table_config))
    return fail(BPX_ERR_INVAL, "bpx_grouped_run: tile shape %d differs from the planned one; "
                "call bpx_group_autotune or bpx_group_set_config first", tile_of(config));
  return run_group(G, opts, config, S(stream));
}

extern "C" int bpx_group_set_config(bpx_group* G, int config, bpx_stream stream) {
  bpx::clear_error();
  if (!G || !G->ws) return fail(BPX_ERR_INVAL, "bpx_group_set_config: group not initialised");
  if (!bpx::gemm_config_ok(config)) return fail(BPX_ERR_INVAL, "bpx_group_set_config: gemm_config %d names no tile", config);
  G->tuned_config = config;
  return ensure_table(G, config, S(stream));
}

extern "C" int bpx_group_graph_launch(bpx_group* G, const bpx_opts* opts, bpx_stream stream) {
  bpx::clear_error();
  if (!G || !G->ws) return fail(BPX_ERR_INVAL, "bpx_group_graph_launch: group not initialised");
  cudaStream_t st = S(stream);
  if (!st) return fail(BPX_ERR_INVAL, "bpx_group_graph_launch needs a non-default stream");
  const int config = (opts && opts->gemm_config) ? opts->gemm_config : G->tuned_config;
  if (!bpx::gemm_config_ok(config)) return fail(BPX_ERR_INVAL, "bpx_group_graph_launch: gemm_config %d names no tile", config);
  const int key[5] = {config, opts ? opts->direct_write : 1, opts ? opts->compensate_depth : -1, 1, G->peel_target};
  const bool same = G->exec && std::equal(key, key + 5, G->graph_key);
  if (!same) {
    if (int rc = ensure_table(G, config, st)) return rc;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    G->exec = nullptr;
    G->graph = nullptr;
    bpx_opts o = opts ? *opts : bpx_default_opts();
    o.stage_events = nullptr;  // events are not replayed per launch
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    const int rc = run_group(G, &o, config, st);
    e = cudaStreamEndCapture(st, &G->graph);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    if ((e = cudaGraphInstantiate(&G->exec, G->graph, 0)) != cudaSuccess) return cuda_fail(e, "instantiate");
    std::copy(key, key + 5, G->graph_key);
  }
  cudaError_t e = cudaGraphLaunch(G->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return BPX_OK;
}

namespace {

const int kDefaultConfigs[] = {8080, 16080, 4080, 8089, 16089, 8085, 16041, 8086, 16042};

// BPX_OK when every candidate GEMM config names a tile.
int check_configs(const int* configs, int n, const char* who) {
  for (int i = 0; configs && i < n; ++i)
    if (!bpx::gemm_config_ok(configs[i])) return fail(BPX_ERR_INVAL, "%s: gemm_config %d names no tile", who, configs[i]);
  return BPX_OK;
}

// Times `launch` on each candidate (one warm-up, then the best of three) and
// returns the fastest.
template <typename F>
int tune(const int* configs, int n, cudaStream_t st, F launch, int* best_config, float* best_ms) {
  if (!configs || n <= 0) {
    configs = kDefaultConfigs;
    n = static_cast<int>(sizeof(kDefaultConfigs) / sizeof(kDefaultConfigs[0]));
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  int arg = configs[0];
  for (int i = 0; i < n; ++i) {
    if (int rc = launch(configs[i])) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return rc;
    }
    float t_best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(a, st);
      if (int rc = launch(configs[i])) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return rc;
      }
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      t_best = std::min(t_best, ms);
    }
    if (t_best < best) {
      best = t_best;
      arg = configs[i];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (best_config) *best_config = arg;
  if (best_ms) *best_ms = best;
  return BPX_OK;
}

}  // namespace

extern "C" int bpx_group_autotune(bpx_group* G, const int* configs, int nconfigs, bpx_stream stream,
                                  int* best_config, float* best_ms) {
  bpx::clear_error();
  if (!G || !G->ws) return fail(BPX_ERR_INVAL, "bpx_group_autotune: group not initialised");
  if (int rc = check_configs(configs, nconfigs, "bpx_group_autotune")) return rc;
  cudaStream_t st = S(stream);
  // one full run so that every job's plan and staged operands exist
  if (int rc = run_group(G, nullptr, G->table_config > 0 ? G->table_config : 0, st)) return rc;
  int best = 0;
  const int split = G->precision == BPX_BF16X3;
  int rc = tune(configs, nconfigs, st,
                [&](int cfg) -> int {
                  if (int r = ensure_table(G, cfg, st)) return r;
                  cudaError_t e = bpx::launch_gemm_tc_grouped(static_cast<char*>(G->ws) + G->tc_off,
                                                              static_cast<int>(G->jobs.size()),
                                                              G->tiles_total, split, cfg, st);
                  return e == cudaSuccess ? BPX_OK : cuda_fail(e, "autotune launch");
                },
                &best, best_ms);
  if (rc) return rc;
  if (best_config) *best_config = best;
  G->tuned_config = best;
  return ensure_table(G, best, st);
}

extern "C" int bpx_autotune(const bpx_code* c, const float* d_A, const float* d_B, int M, int N, int K, int h,
                            int precision, const uint8_t* d_mask, float* d_C, void* ws, size_t ws_bytes,
                            const int* configs, int nconfigs, bpx_stream stream, int* best_config,
                            float* best_ms) {
  bpx::clear_error();
  if (precision != BPX_BF16 && precision != BPX_BF16X3 && precision != BPX_EXACT && precision != BPX_FP16X3)
    return fail(BPX_ERR_UNSUPPORTED,
                "bpx_autotune tunes the tensor-core GEMM (BPX_BF16 / BPX_BF16X3 / BPX_FP16X3 / BPX_EXACT)");
  if (int rc = check_configs(configs, nconfigs, "bpx_autotune")) return rc;
  // one full run: plan, staged operands
  if (int rc = bpx_coded_matmul(c, d_A, d_B, M, N, K, h, precision, d_mask, d_C, nullptr, ws, ws_bytes,
                                nullptr, stream))
    return rc;
  const bpx::WsLayout L = bpx::ws_layout(c, M, N, K, h, precision);
  const bpx::DevGraph g = bpx::make_graph(c, ws, L);
  const bpx::DevPlan p = bpx::make_plan(ws, L);
  char* base = static_cast<char*>(ws);
  const bool f16 = precision == BPX_FP16X3;
  const bool split = precision == BPX_BF16X3 || f16;
  const int32_t* a_exp = f16 ? reinterpret_cast<const int32_t*>(base + L.a_scale) : nullptr;
  const int32_t* b_exp = f16 ? reinterpret_cast<const int32_t*>(base + L.b_scale) + N : nullptr;
  float* products = reinterpret_cast<float*>(base + L.products);
  cudaStream_t st = S(stream);
  if (precision == BPX_EXACT) {
    bpx::ExactParams P;
    if (int rc = bpx::exact_params(c, K, &P)) return rc;
    static const int kExactConfigs[] = {8080, 16080, 4080, 8089, 8081, 8082, 8085};
    if (!configs || nconfigs <= 0) {
      configs = kExactConfigs;
      nconfigs = static_cast<int>(sizeof(kExactConfigs) / sizeof(kExactConfigs[0]));
    }
    return tune(configs, nconfigs, st,
                [&](int cfg) -> int {
                  cudaError_t e = bpx::launch_gemm_exact(p, base + L.a_hi, base + L.b_hi, c->num_cells, N, K, h, P,
                                                         reinterpret_cast<int32_t*>(products), cfg, nullptr, st);
                  return e == cudaSuccess ? BPX_OK : cuda_fail(e, "autotune launch");
                },
                best_config, best_ms);
  }
  return tune(configs, nconfigs, st,
              [&](int cfg) -> int {
                cudaError_t e = bpx::launch_gemm_tc(g, p, base + L.a_hi, split ? base + L.a_lo : nullptr,
                                                    base + L.b_hi, split ? base + L.b_lo : nullptr,
                                                    c->num_cells, N, K, h, split, products, d_C, cfg,
                                                    nullptr, st, a_exp, b_exp);
                return e == cudaSuccess ? BPX_OK : cuda_fail(e, "autotune launch");
              },
              best_config, best_ms);
}

extern "C" int bpx_group_autotune_peel(bpx_group* G, const int* targets, int ntargets, bpx_stream stream,
                                       int* best_target, float* best_ms) {
  bpx::clear_error();
  if (!G || !G->ws) return fail(BPX_ERR_INVAL, "bpx_group_autotune_peel: group not initialised");
  cudaStream_t st = S(stream);
  const int sms = bpx::num_sms();
  const int defaults[] = {std::max(1, sms / 8), std::max(1, sms / 4), std::max(1, sms / 2), sms, 2 * sms, 4 * sms,
                          8 * sms};
  if (!targets || ntargets <= 0) {
    targets = defaults;
    ntargets = static_cast<int>(sizeof(defaults) / sizeof(defaults[0]));
  }
  for (int i = 0; i < ntargets; ++i)
    if (targets[i] < 1) return fail(BPX_ERR_INVAL, "bpx_group_autotune_peel: targets must be >= 1");
  // one full run so that every job's plan, products and direct blocks exist;
  // re-running the peel alone then recomputes the same C
  if (int rc = run_group(G, nullptr, G->tuned_config, st)) return rc;
  auto upload = [&](int target) -> int {
    G->peel_target = target;
    plan_peel(G);
    const cudaError_t e = upload_jobs(G, st);
    return e == cudaSuccess ? BPX_OK : cuda_fail(e, "bpx_group_autotune_peel: job table");
  };
  int best = targets[0];
  int rc = tune(targets, ntargets, st,
                [&](int target) -> int {
                  if (G->peel_target != target || G->peel_total == 0)
                    if (int r = upload(target)) return r;
                  cudaError_t e = launch_group_peel(G, -1, st);
                  return e == cudaSuccess ? BPX_OK : cuda_fail(e, "autotune launch");
                },
                &best, best_ms);
  if (rc) return rc;
  if (best_target) *best_target = best;
  return upload(best);  // also retires a captured graph (the key holds the target)
}

extern "C" int bpx_autotune_peel(const bpx_code* c, const float* d_A, const float* d_B, int M, int N, int K, int h,
                                 int precision, const uint8_t* d_mask, float* d_C, void* ws, size_t ws_bytes,
                                 const int* ctas, int nctas, bpx_stream stream, int* best_ctas, float* best_ms) {
  bpx::clear_error();
  if (precision == BPX_EXACT)
    return fail(BPX_ERR_UNSUPPORTED, "bpx_autotune_peel tunes the floating-point peel (not BPX_EXACT)");
  const int sms = bpx::num_sms();
  const int defaults[] = {sms / 2, sms, 2 * sms, 3 * sms, 4 * sms, 8 * sms};
  if (!ctas || nctas <= 0) {
    ctas = defaults;
    nctas = static_cast<int>(sizeof(defaults) / sizeof(defaults[0]));
  }
  for (int i = 0; i < nctas; ++i)
    if (ctas[i] < 1) return fail(BPX_ERR_INVAL, "bpx_autotune_peel: CTA counts must be >= 1");
  // one full run: plan, products, direct blocks; the peel alone then
  // recomputes the same C from them
  if (int rc = bpx_coded_matmul(c, d_A, d_B, M, N, K, h, precision, d_mask, d_C, nullptr, ws, ws_bytes,
                                nullptr, stream))
    return rc;
  const bpx::WsLayout L = bpx::ws_layout(c, M, N, K, h, precision);
  const float* products = reinterpret_cast<const float*>(static_cast<char*>(ws) + L.products);
  bpx_opts o = bpx_default_opts();
  cudaStream_t st = S(stream);
  return tune(ctas, nctas, st,
              [&](int n_ctas) -> int {
                o.peel_ctas = n_ctas;
                return bpx_peel_decode(c, products, nullptr, N, h, d_C, 1, &o, ws, ws_bytes, nullptr, stream);
              },
              best_ctas, best_ms);
}

extern "C" void bpx_group_free(bpx_group* G) {
  if (!G) return;
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  if (G->fork) cudaEventDestroy(G->fork);
  if (G->join) cudaEventDestroy(G->join);
  if (G->fork_b) cudaEventDestroy(G->fork_b);
  if (G->join_b) cudaEventDestroy(G->join_b);
  if (G->side) cudaStreamDestroy(G->side);
  delete G;
}
