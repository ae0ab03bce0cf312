/*
 * bpx.h -- C ABI of libbpx: array BP-XOR coded matrix multiplication on one
 * GB300 GPU (sm_103a).
 *
 * The library computes C = A B for A (M x K) and B (K x N), FP32 row-major,
 * the way the coded scheme of Arslan, "Array BP-XOR Codes for Hierarchically
 * Distributed Matrix Multiplication", does it:
 *
 *   - A is cut into S = b k row blocks ("source symbols") of h rows each
 *     (Section II, Remark 2.1); block s is rows [s h, (s+1) h).  Rows past
 *     M read as zero.
 *   - Each coded symbol ("cell") c of an array code holds the XOR -- here the
 *     real sum -- of the blocks in its support (Section III-A, Definition of
 *     the [n,k,t,b] array BP-XOR code; Eq. (moj1) for projection codes).
 *     Cells are grouped into n code columns (worker nodes).
 *   - Every cell of a column that did not straggle yields its coded product
 *     P_c = (sum_{s in supp(c)} A_s) B (Section III-A, Example 1: a processor
 *     executes at most sigma dot products of summed operands).
 *   - The sink rebuilds every C_s = A_s B by belief-propagation peeling
 *     (Section I-A): a cell with one unknown source resolves it by
 *     subtraction, C_s = P_r - sum_{t in supp(r), t != s} C_t.
 *
 * Workers and stragglers are emulated: an erasure mask over the n columns
 * says which workers straggled.
 *
 * Conventions for every call
 *   - Pointers named d_* are device pointers (cudaMalloc'd or torch-owned,
 *     on the current device); h_* are host pointers.  The caller owns every
 *     buffer and the stream.  The library allocates no device memory: all
 *     per-call state lives in a caller-provided workspace (see
 *     bpx_workspace_bytes / bpx_workspace_init).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) unless stated otherwise.  The return value reports
 *     argument and launch errors only; the decode outcome lands in a device
 *     int32 info array (BPX_INFO_*), which synchronous calls also return.
 *   - Every return value is a bpx_status.  On failure bpx_last_error() gives
 *     a thread-local message.  No C++ exception crosses the ABI.
 *   - Alignment: all device buffers 16-byte aligned; the workspace 256-byte
 *     aligned.  N must be a multiple of 4 and K a multiple of 8.
 */
#ifndef BPX_H
#define BPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bpx_code bpx_code; /* opaque, host-side, library-owned */
typedef void* bpx_stream;         /* a cudaStream_t */

/* Code families (Section III). */
enum bpx_variant {
  BPX_TABLE1 = 0,     /* Table I, the [5,2,2,2] code: n=5, k=2, b=2, tolerates 3 erasures */
  BPX_TABLE3 = 1,     /* Table III, the [5,3,2,3] code: n=5, k=3, b=3, tolerates 2 */
  BPX_SYSTEMATIC = 2, /* systematic Mojette array: k data columns of the k x b grid + e
                         projection parities (q=1, slopes 0,+1,-1,+2,...), n = k + e */
  BPX_MOJETTE_A = 3,  /* Construction A (Cons33): n projections q=1,
                         p = -floor((n-1)/2)..ceil((n-1)/2) of the k x b grid; e = n - k */
  BPX_MOJETTE_B = 4,  /* Construction B (cons35): n projections q=2^q_e, p = n consecutive
                         odd integers from ceil_odd(1-n); e = n - ceil(k / 2^q_e) */
  BPX_LITERAL = 5,    /* a code given by its cells (bpx_code_from_cells, bpx_code_search) */
  BPX_XCODE = 6       /* X-code of Xu and Bruck (1999), an equal-height MDS array code whose
                         two-column erasure decoding is a peeling chain, so an array BP-XOR
                         code in the sense of Section III-A: n = p prime, b = p, k = p - 2,
                         e = 2, sigma = p - 2 */
};

/* Arithmetic of the coded products.  FP32 accumulation in every case. */
enum bpx_precision {
  BPX_FP32 = 0,   /* plain FP32 on the CUDA cores (FP32 encode pass, then an FFMA GEMM) */
  BPX_BF16 = 1,   /* coded A and B rounded to bf16, one tcgen05 MMA per k-step */
  BPX_BF16X3 = 2, /* split bf16: a = a_hi + a_lo; hi*hi + hi*lo + lo*hi on tcgen05 */
  BPX_MXFP8 = 3,  /* E4M3 with one UE8M0 scale per 32 K-elements (tcgen05 block-scaled) */
  BPX_EXACT = 4,  /* exact slices: the decode is exact at every peel depth (bpx_exact_params) */
  BPX_FP16X3 = 5  /* split fp16 under power-of-two scales: every coded row of A and every column
                     of B is scaled by 2^e so that its largest magnitude lies in [2^14, 2^15);
                     a = a_hi + a_lo in fp16 (22 significant bits against bf16's 16);
                     hi*hi + hi*lo + lo*hi on tcgen05 kind::f16 into FP32, the scales undone
                     exactly in the epilogue; 128-wide K accumulation segments by default */
};

enum bpx_status {
  BPX_OK = 0,
  BPX_ERR_INVAL = 1,       /* bad argument (size, alignment, null pointer, variant) */
  BPX_ERR_UNSUPPORTED = 2, /* valid request this build cannot run */
  BPX_ERR_UNDECODABLE = 3, /* peeling stopped before every source was recovered */
  BPX_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out; the kernel exited cleanly */
  BPX_ERR_CUDA = 5,        /* a CUDA runtime call failed (message in bpx_last_error) */
  BPX_ERR_NOMEM = 6        /* workspace smaller than bpx_workspace_bytes */
};

/* Device info array written by bpx_schedule / bpx_coded_matmul (int32[BPX_INFO_LEN]). */
enum bpx_info_index {
  BPX_INFO_STATUS = 0,      /* BPX_OK or BPX_ERR_UNDECODABLE (or BPX_ERR_TIMEOUT) */
  BPX_INFO_RECOVERED = 1,   /* number of recovered sources */
  BPX_INFO_WAVES = 2,       /* number of peel rounds (maximum depth) */
  BPX_INFO_SURVIVING = 3,   /* number of cells in non-erased columns */
  BPX_INFO_DIRECT = 4,      /* sources resolved at depth 1 (written by the GEMM epilogue) */
  BPX_INFO_DEVICE_ERR = 5,  /* 0, or the BPX_ERR_* a kernel's self-check raised */
  BPX_INFO_LEN = 16
};

typedef struct {
  int variant, n, k, e, b, q_e;
  int num_sources; /* S = b k */
  int num_cells;   /* coded symbols over all columns (empty Mojette bins dropped) */
  int num_edges;   /* sum of cell degrees */
  int sigma;       /* maximum cell degree (Section III-A; Section III-C theorem) */
  double eps;      /* worst-case coding overhead eps(b,n) of Section III-B: over all
                      choices of k columns, sum of their heights / (k b) - 1 */
  /* Host views owned by the code handle, valid until bpx_code_free. */
  const int32_t* col_ptr;     /* [n+1]: cells of column j are [col_ptr[j], col_ptr[j+1]) */
  const int32_t* cell_ptr;    /* [num_cells+1]: support of cell c is cell_src[cell_ptr[c] ..] */
  const int32_t* cell_src;    /* [num_edges]: source ids, ascending within a cell */
  const int32_t* col_of_cell; /* [num_cells] */
  const int32_t* heights;     /* [n]: column heights b_i = |p|(k-1) + |q|(b-1) + 1 (III-C) */
  const int32_t* proj_p;      /* [n]: projection p of each column (0 for data columns) */
  const int32_t* proj_q;      /* [n]: projection q of each column (0 for data columns) */
} bpx_code_info;

typedef struct {
  int direct_write;     /* 1 (default): the product epilogue writes each depth-1 resolver
                           straight into its C block, so the peel skips those sources */
  int compensate_depth; /* sources deeper than this are peeled with compensated subtraction
                           (TwoSum: each step's rounding error kept in a second FP32 term, one
                           final rounding); < 0 (default -1): never */
  int peel_ctas;        /* 0 = auto (a multiple of the SM count) */
  int gemm_config;      /* 0 = defaults; otherwise band * 1000 + seg_kb * 10 + tile (bpx_autotune).
                           BPX_MXFP8 reads band * 1000 + tile: tiles 9 / 0 = CTA-pair MMAs (the
                           default, 16009), 1 / 2 / 5 / 6 = 1-CTA MMAs.  Tile codes 3, 4, 7, 8
                           and negative values name no kernel: BPX_ERR_INVAL */
  void* const* stage_events; /* NULL, or cudaEvent_t[2 * BPX_NUM_STAGES] created by the caller:
                                events 2i / 2i+1 are recorded on the stream right before / after
                                stage i (enum bpx_stage).  Used to time kernels in place. */
  int mask_cells;       /* 0 (default): erasure masks have one byte per code column (a node
                           straggled); 1: one byte per cell (a single processor's output is
                           missing, the straggler model of Section IV) */
  int fused_encode;     /* 0 (default): the encode (a2) is its own HBM-bound pass writing the
                           coded bf16 operand before the GEMM; 1: BPX_BF16 / BPX_BF16X3 form
                           the coded rows inside the GEMM's operand load (transform warps sum
                           the FP32 source rows and split them on chip; the same bits); needs
                           gemm_config 0 or a CTA-pair 64-wide config (tile code 0), else
                           BPX_ERR_INVAL; other precisions and codes with sigma > 8:
                           BPX_ERR_UNSUPPORTED */
} bpx_opts;

/* Stages of the hot path, in launch order (for bpx_opts.stage_events). */
enum bpx_stage {
  BPX_STAGE_SCHEDULE = 0, /* a1 symbolic peel */
  BPX_STAGE_B_PREP = 1,   /* B split / quantize (tensor-core paths) */
  BPX_STAGE_A_PREP = 2,   /* encode (+ split / quantize / digit planes) of the coded operand */
  BPX_STAGE_GEMM = 3,     /* coded products */
  BPX_STAGE_PEEL = 4,     /* a4 numeric peel */
  BPX_NUM_STAGES = 5
};

/* ---------------------------------------------------------------- code graph */

/* Builds the code graph of a family of Section III (host only, no GPU needed).
 *   Table I / III: (n,k,b) must be (5,2,2) / (5,3,3); e may be -1.
 *   BPX_SYSTEMATIC: n = k + e data + parity columns on the k x b grid.
 *   BPX_MOJETTE_A / _B: n projections of the k x b grid; q_e >= 1 for _B.
 *   BPX_XCODE: n = p prime, k = p - 2, b = p.  Column i holds the sources of
 *     grid row i, s = i k + r (r < k), as degree-one cells, then the two
 *     diagonal parities {((i + r + 2) mod p) k + r} and {((i - r - 2) mod p) k + r}
 *     over r < k.
 * e = -1 derives the tolerated erasures; otherwise it must match.
 * Cell numbering: column ascending, then processor row / bin label ascending;
 * bins are placed by Eq. (moj1): pixel (z,l), z in [0,b), l in [0,k), is source
 * s = z k + l, label (b-1) q u(q) + (k-1) p u(p) - z q - l p.  Empty bins are
 * dropped.  *out receives a handle to release with bpx_code_free.
 * Errors: BPX_ERR_INVAL for inconsistent parameters or more than 2^24 sources. */
int bpx_code_build(int variant, int n, int k, int e, int b, int q_e, bpx_code** out);

/* Fills *out with sizes and host views of the graph (see bpx_code_info). */
int bpx_code_info_get(const bpx_code* code, bpx_code_info* out);

/* Releases the handle (NULL is a no-op). */
void bpx_code_free(bpx_code* code);

/* Thread-local text of the last error raised on this thread. */
const char* bpx_last_error(void);

/* ---------------------------------------------------------------- code-parameter tooling
 * Host only (no GPU needed). */

/* Bounds on the number of columns n of an array BP-XOR code with k data
 * columns, b rows and largest cell degree sigma (Section III-B):
 *   bpx_bound_k_equals_sigma: n <= kb + 1 + max{k - 3, 0} when k = sigma
 *     (quoted from Paterson et al.; Table I meets it with equality);
 *   bpx_bound_paterson (k > sigma): n <= k + sigma - 1 + floor(sigma
 *     (sigma - 1)(b - 1) / ((k - sigma) b + sigma - 1)) -- the straggler
 *     count n - k the paper's Section V simulations use (Table III meets it). */
int bpx_bound_k_equals_sigma(int k, int b, int* n_max);
int bpx_bound_paterson(int k, int b, int sigma, int* n_max);

/* A code given by its cells (variant BPX_LITERAL): num_cells cells grouped by
 * ascending column (col_of_cell[c] in [0, n)), cell c's support =
 * cell_src[cell_ptr[c] .. cell_ptr[c+1]) ascending, source ids in [0, b k)
 * (pixel (z, l) of the grid is z k + l).  e = the column erasures the code is
 * meant to tolerate (recorded, not checked).  The arrays are copied. */
int bpx_code_from_cells(int n, int k, int b, int num_cells, const int32_t* col_of_cell, const int32_t* cell_ptr,
                        const int32_t* cell_src, int e, bpx_code** out);

/* Searches for an equal-height array BP-XOR code: n columns of b cells, every
 * cell the sum of at most sigma of the b k sources, decodable by peeling from
 * every set of k columns (e = n - k).  Simulated annealing over the cells'
 * supports (cost: the sources left unknown, summed over the erasure patterns,
 * plus sources in fewer than n - k + 1 columns), at most `iters` moves from
 * `seed`.  b k <= 64, n <= 30.  *out receives the code (BPX_LITERAL) or NULL
 * with BPX_ERR_UNSUPPORTED when none was found; *iters_used (or NULL) the
 * moves taken.  Equivalent to bpx_code_search_ex with flags 0, threads 1. */
int bpx_code_search(int n, int k, int b, int sigma, long long iters, unsigned long long seed, bpx_code** out,
                    long long* iters_used);

/* Search flags. */
enum bpx_search_flags {
  BPX_SEARCH_SYSTEMATIC = 1 /* the first k columns hold the b k sources one per cell (column l,
                               cell z = source z k + l); only the parity columns are searched */
};

/* bpx_code_search with options: `threads` (1..256) independent annealing
 * chains run on host threads, chain t from seed + t with up to `iters` moves
 * each; the code returned is the one of the lowest t that found one, so the
 * result does not depend on the threads' timing.  *iters_used = the moves of
 * all chains.  flags: BPX_SEARCH_SYSTEMATIC or 0. */
int bpx_code_search_ex(int n, int k, int b, int sigma, long long iters, unsigned long long seed, int flags,
                       int threads, bpx_code** out, long long* iters_used);

/* ---------------------------------------------------------------- workspace */

/* Device bytes needed by the calls below for this code, shapes and precision
 * (graph copy + peel plan + operand staging for the tensor-core paths). */
size_t bpx_workspace_bytes(const bpx_code* code, int M, int N, int K, int h, int precision);

/* Binds a workspace to a code: uploads the graph (stream-ordered copies from
 * the handle's host arrays; the call synchronizes `stream` before returning so
 * the handle may be freed afterwards).  Once per workspace.  BPX_ERR_NOMEM if
 * ws_bytes is too small for bpx_workspace_bytes(code, 0, 0, 0, 1, BPX_FP32). */
int bpx_workspace_init(const bpx_code* code, void* d_ws, size_t ws_bytes, bpx_stream stream);

/* Byte offset in a workspace of this code of the plan's device info words
 * (int32[BPX_INFO_LEN], written by every schedule and by kernels' self-checks
 * and refusals); 0 when code is NULL.  Host only. */
size_t bpx_workspace_info_offset(const bpx_code* code);

/* ---------------------------------------------------------------- hot path */

/* a1. Symbolic peel (Section I-A decoder, parallel-round reading): from the
 * device erasure mask d_erasure_mask[n] (1 = column straggled) computes the
 * surviving cells and, round by round, every source whose surviving cell has
 * exactly one unknown source left: resolver = the lowest such cell id,
 * depth = the round.  Writes the plan into the workspace.  Optional outputs
 * (NULL to skip): d_peel_order int32[3 S] = (source, resolver, depth) sorted
 * by (depth, source), unused entries -1; d_recovered uint8[S]; d_info
 * int32[BPX_INFO_LEN].  Undecodable masks are not an error of the call: the
 * info array says BPX_ERR_UNDECODABLE and the partial plan stays usable. */
int bpx_schedule(const bpx_code* code, const uint8_t* d_erasure_mask, void* d_ws, size_t ws_bytes,
                 int32_t* d_peel_order, uint8_t* d_recovered, int32_t* d_info, bpx_stream stream);

/* a1 with a cell-level mask: d_cell_mask[num_cells], 1 = that processor's
 * output is missing (Section IV: processors straggle individually).
 * Otherwise as bpx_schedule. */
int bpx_schedule_cells(const bpx_code* code, const uint8_t* d_cell_mask, void* d_ws, size_t ws_bytes,
                       int32_t* d_peel_order, uint8_t* d_recovered, int32_t* d_info, bpx_stream stream);

/* Straggler-time model (Section IV, Eq. (eqnTtotal)), host only: the cells'
 * products arrive in order[0 .. n) (distinct cell ids); the sink peels online
 * as they arrive.  recovered_after[i] (or NULL) = sources recovered once
 * order[0..i] have arrived; *first = the number of arrivals after which every
 * source is recovered -- so T_{order[*first - 1]} = min over decodable sets S
 * of max_{c in S} T_c -- or -1 if the n arrivals never decode. */
int bpx_first_decodable(const bpx_code* code, const int32_t* order, int n, int32_t* recovered_after,
                        int32_t* first);

/* a2. Worker-side encode, materialized (Section III-A, Example 1: the nodes
 * form the sums themselves): for the i-th surviving cell c (ascending id, as
 * planned by bpx_schedule) writes rows [i h, (i+1) h) of d_A_coded (K columns,
 * FP32) = sum over s in supp(c), ascending, of A_s.  d_A_coded must hold
 * num_cells h rows; rows past the surviving count are left untouched. */
int bpx_encode(const bpx_code* code, const float* d_A, int M, int K, int h, const void* d_ws,
               float* d_A_coded, bpx_stream stream);

/* a3. Coded products (Section III-A): P_c = A_c B for every surviving cell,
 * in the given precision, the encode sums formed by a pass just before the GEMM.
 * P_c goes to d_products + c h N (d_products: num_cells h N floats, row-major
 * h x N per cell), except that with d_C non-NULL the product of each depth-1
 * resolver goes straight to its source block d_C + s h N.  Requires the plan
 * of bpx_schedule in d_ws.  BPX_EXACT: d_products is int32 storage for the S
 * diagonal planes (see bpx_peel_decode_exact), d_C is ignored, and the
 * scales of A and B are left in d_ws for the peel. */
int bpx_coded_products(const bpx_code* code, const float* d_A, const float* d_B, int M, int N,
                       int K, int h, int precision, void* d_ws, size_t ws_bytes,
                       float* d_products, float* d_C, const bpx_opts* opts, bpx_stream stream);

/* a4. Numeric peel (Section I-A, XOR read as subtraction; Section II: the
 * sink decodes from the products that arrived): for the erasure pattern
 * d_erasure_mask (as for bpx_schedule; one byte per cell when
 * opts->mask_cells), C_s = P_r - sum_{t in supp(r), t != s, ascending} C_t
 * for every recovered source, wave by wave.  The call first plans the peel
 * for that mask into d_ws (exactly as bpx_schedule, whose info words go to
 * d_info when non-NULL); the mask must be the one the products were computed
 * under.  d_erasure_mask = NULL peels along the plan already in d_ws (left by
 * bpx_schedule or bpx_coded_matmul); if no schedule has run on d_ws since
 * bpx_workspace_init, the peel writes nothing and sets BPX_ERR_INVAL in the
 * plan's info words (BPX_INFO_STATUS and BPX_INFO_DEVICE_ERR).  d_products:
 * P_c at d_products + c h N (bpx_coded_products).  d_C holds S h rows of N
 * floats (rows >= M are scratch for zero-padded blocks).  direct_written = 1
 * when bpx_coded_products already wrote the depth-1 sources into d_C.
 * Unrecovered blocks are left untouched. */
int bpx_peel_decode(const bpx_code* code, const float* d_products, const uint8_t* d_erasure_mask, int N, int h,
                    float* d_C, int direct_written, const bpx_opts* opts, void* d_ws, size_t ws_bytes,
                    int32_t* d_info, bpx_stream stream);

/* ---------------------------------------------------------------- exact slices
 *
 * BPX_EXACT restores over the reals the exactness the paper's XOR over bits
 * has (Section II: XOR coding and peeling are exact): the peel subtracts exact
 * integers, so a source decoded at depth 700 carries the same error as one
 * copied from a degree-1 cell, and the result does not depend on which
 * columns straggled.  The representation (an Ozaki-style error-free
 * splitting) is not in the paper:
 *   - A is scaled per row position j in [0, h) (shared by every source block,
 *     so that rows summed into one coded row share a scale) and B per column
 *     n, by 2^(bits - e) with 2^(e-1) <= max|x| < 2^e, and rounded to
 *     integers (round to nearest even);
 *   - each integer is cut into S balanced base-2^w digits (most significant
 *     first, |digit| <= 2^(w-1)), stored as bf16 digit planes;
 *   - a coded digit plane is the sum of its sources' planes (no carries), so
 *     it is linear in the sources; w is chosen from the code's largest degree
 *     sigma so that sigma 2^(w-1) <= 256 keeps coded digits exact in bf16;
 *   - the digit pairs (i, l) with i + l <= S - 1 are kept and grouped by
 *     diagonal d = i + l: the tensor core accumulates each diagonal over K in
 *     FP32 in segments whose absolute sums stay below 2^23 (exact), each
 *     segment is promoted to int32, and plane d of the products holds
 *     P_c^d = sum_{i+l=d} D_i(A_c) D_l(B) exactly;
 *   - the peel forms Q_c = sum_d 2^(w (S-1-d)) P_c^d in int64, subtracts
 *     exactly, and writes C_s = RN_fp32(Q_s 2^(w (S-1) - 2 bits + e_A[j] +
 *     e_B[n])): one rounding of the exact value, done in integer arithmetic
 *     (|Q_s| < 2^53, so the same bits as rounding the exact FP64 value).
 * The only errors are the fixed-point rounding of A and B and the dropped
 * pairs, both about 2^-24 relative to max|A row j| max|B column n| per K term.
 * Products cost S (S+1) / 2 bf16 MMAs per k-step (sigma 2: 6; sigma 8: 10;
 * sigma 24: 21) and the staged planes S times the bf16 operand bytes. */

/* out[5] = { w, S, bits, K elements per exact FP32 segment, K padded to 64 }
 * for this code and K (host only).  BPX_ERR_UNSUPPORTED when sigma > 64 (digits
 * below 3 bits) or K is so large that the int32 diagonal sums or the int64 /
 * FP64 decoded integers could lose exactness. */
int bpx_exact_params(const bpx_code* code, int K, int32_t* out);

/* a4 for BPX_EXACT: d_planes = the S int32 product planes written by
 * bpx_coded_products(..., BPX_EXACT, ...) (plane d at d_planes + d num_cells h N,
 * each num_cells h N, row-major h x N per cell); the scales and an int64 copy
 * of every decoded block live in d_ws, which must be the workspace that
 * bpx_coded_products used (sized for BPX_EXACT).  Every recovered source,
 * depth 1 included, is written to d_C.  d_erasure_mask / d_info: as for
 * bpx_peel_decode (NULL: the plan already in d_ws).  opts: only
 * stage_events, peel_ctas and mask_cells are read. */
int bpx_peel_decode_exact(const bpx_code* code, const int32_t* d_planes, const uint8_t* d_erasure_mask, int N,
                          int h, float* d_C, const bpx_opts* opts, void* d_ws, size_t ws_bytes, int32_t* d_info,
                          bpx_stream stream);

/* The whole path for one erasure pattern: schedule, encode + products, peel.
 * The products live in the workspace.  d_info as in bpx_schedule.  With
 * BPX_EXACT, direct_write and compensate_depth are ignored.  0 <= M <= S h:
 * rows M .. S h - 1 of the source blocks are zero padding (d_A may be NULL
 * when M = 0; C is then zero). */
int bpx_coded_matmul(const bpx_code* code, const float* d_A, const float* d_B, int M, int N, int K,
                     int h, int precision, const uint8_t* d_erasure_mask, float* d_C,
                     const bpx_opts* opts, void* d_ws, size_t ws_bytes, int32_t* d_info,
                     bpx_stream stream);

/* End-to-end from host memory: copies h_A, h_B and h_erasure_mask into the
 * caller's device buffers d_A, d_B, d_mask (M K, K N, n elements), runs
 * bpx_coded_matmul into d_C (S h x N), copies the first M rows of C into h_C
 * and the info array into h_info (int32[BPX_INFO_LEN]), then synchronizes the
 * stream.  Returns the decode status (BPX_OK / BPX_ERR_UNDECODABLE / ...).
 * Host buffers should be page-locked for full copy bandwidth. */
int bpx_coded_matmul_host(const bpx_code* code, const float* h_A, const float* h_B, int M, int N,
                          int K, int h, int precision, const uint8_t* h_erasure_mask, float* h_C,
                          float* d_A, float* d_B, uint8_t* d_mask, float* d_C, const bpx_opts* opts,
                          void* d_ws, size_t ws_bytes, int32_t* h_info, bpx_stream stream);

/* The same as bpx_coded_matmul_host without the final synchronization: the
 * copies in, the path and the copies out are enqueued on `stream` and the call
 * returns the launch status (BPX_OK or an argument / launch error).  h_C and
 * h_info (decode status in h_info[BPX_INFO_STATUS], kernel self-check in
 * [BPX_INFO_DEVICE_ERR]) are valid once `stream` has completed; until then
 * none of the call's buffers, nor its workspace, may be reused or freed.  A
 * caller streaming many multiplications keeps several calls in flight on
 * different streams, each with its own device buffers and workspace, so that
 * one call's host-to-device copies, another's kernels and a third's
 * device-to-host copies run at the same time (the two copy directions and the
 * SMs are separate resources).  Host buffers must be page-locked. */
int bpx_coded_matmul_host_async(const bpx_code* code, const float* h_A, const float* h_B, int M, int N,
                                int K, int h, int precision, const uint8_t* h_erasure_mask, float* h_C,
                                float* d_A, float* d_B, uint8_t* d_mask, float* d_C, const bpx_opts* opts,
                                void* d_ws, size_t ws_bytes, int32_t* h_info, bpx_stream stream);

/* ---------------------------------------------------------------- two-dimensional scheme
 *
 * The paper's own scheme (Section III-A, Examples 1 and 2): C = A B with A cut
 * into b row blocks of h rows and B into k column blocks of w = N / k columns;
 * source s = z k + l (the grid pixel of Section III-C; Table I's
 * v_{(i-1)m+j} = a_i b_j) is the output block C[z h .., l w ..] = A_z B_l, and
 * a cell's coded product is the sum of its sources' block products.  The
 * library computes a cell as few products of summed operands as its support
 * allows: its sources grouped by A block (each z with the set of l it pairs
 * with, A blocks with equal sets merged) or by B block, whichever gives
 * fewer products, each product (sum_{z in Z} A_z)(sum_{l in L} B_l).  A cell
 * with more than one product cannot be formed from one summed A operand and
 * one summed B operand (the gray cells of Tables I and III), so the worker
 * evaluates several block products (a K-concatenated product).  The peel is
 * the one-dimensional scheme's (same schedule), over h x w blocks. */

/* Host-only summary of the factoring: terms_per_cell[num_cells] (or NULL) and
 * summary[4] (or NULL) = { total products over all cells, cells with more
 * than one product, distinct summed A operands, distinct summed B operands }. */
int bpx_terms_2d(const bpx_code* code, int32_t* terms_per_cell, int32_t* summary);

/* Workspace for bpx_coded_matmul_2d: graph and plan (as bpx_workspace_bytes),
 * products (num_cells h w floats) and the staged operands (every summed A
 * operand as h bf16 rows of K, every summed B operand as w rows of B^T; hi and
 * lo for BPX_BF16X3).  The workspace is bound with bpx_workspace_init. */
size_t bpx_workspace_bytes_2d(const bpx_code* code, int M, int N, int K, int h, int precision);

/* Schedule (a1, shared with the one-dimensional scheme), staging of the summed
 * operands, the coded products of every surviving cell on the tensor cores
 * (one persistent launch over all cells' h x w tiles, most products first),
 * and the peel.  d_C: b h rows of N floats (row stride N; rows >= M are
 * scratch); block (z, l) at row z h, column l w.  N must be a multiple of k
 * with w = N / k a multiple of 4; K a multiple of 8; M <= b h.  precision:
 * BPX_BF16 or BPX_BF16X3.  opts: direct_write (depth-1 blocks written by the
 * GEMM), gemm_config (tile config as for bpx_autotune), peel_ctas,
 * stage_events (BPX_STAGE_A_PREP covers the staging of both operands). */
int bpx_coded_matmul_2d(const bpx_code* code, const float* d_A, const float* d_B, int M, int N, int K, int h,
                        int precision, const uint8_t* d_erasure_mask, float* d_C, const bpx_opts* opts, void* d_ws,
                        size_t ws_bytes, int32_t* d_info, bpx_stream stream);

/* ---------------------------------------------------------------- batches */

/* Many independent coded multiplications run together.  Each job is a whole
 * instance of the problem above (its own code, shapes, erasure mask and
 * buffers); the paper's scheme applies per job.  All device pointers are the
 * caller's and must stay valid while the group is used. */
typedef struct bpx_group bpx_group; /* opaque, host-side */

typedef struct {
  const bpx_code* code;        /* host handle; must outlive the group */
  const float* A;              /* device, M x K */
  const float* B;              /* device, K x N */
  float* C;                    /* device, S h x N (depth-1 blocks are written by the GEMM) */
  const uint8_t* erasure_mask; /* device, n bytes; read at every run */
  int32_t* info;               /* device int32[BPX_INFO_LEN] per job, or NULL */
  int M, N, K, h;
} bpx_job;

/* Plans a batch (host only): each job's workspace region, the per-stage grids
 * and the device job tables.  precision: BPX_BF16 or BPX_BF16X3. */
int bpx_group_create(const bpx_job* jobs, int njobs, int precision, bpx_group** out);

/* Device bytes the group needs (all jobs' workspaces + job tables). */
size_t bpx_group_workspace_bytes(const bpx_group* group);

/* Binds the workspace: uploads every job's code graph and the job tables,
 * encodes the TMA descriptors, creates the group's side stream and events;
 * synchronizes `stream`. */
int bpx_group_init(bpx_group* group, void* d_ws, size_t ws_bytes, bpx_stream stream);

/* Runs every job: one launch per stage over all jobs (a1 schedule, B split,
 * a2 encode + split, one persistent grouped tcgen05 GEMM over all jobs' tiles,
 * a4 peel).  The B split runs on the group's side stream beside the
 * schedule, and the register-path peel beside the gathered one (tall codes),
 * forked from and joined back to `stream` with events, so the call is still
 * ordered on `stream` as one unit.  No host synchronization or allocation
 * inside: the call can be captured in a CUDA graph.  Each job's outcome lands
 * in its info words.  Runs of one group must not overlap (they share the
 * workspace and the side stream).  opts->gemm_config must keep the planned
 * tile width (0 = the planned one). */
int bpx_grouped_run(bpx_group* group, const bpx_opts* opts, bpx_stream stream);

/* Captures bpx_grouped_run into a CUDA graph owned by the group on the first
 * call (or when the options change) and replays it; `stream` must not be the
 * legacy default stream. */
int bpx_group_graph_launch(bpx_group* group, const bpx_opts* opts, bpx_stream stream);

/* Selects the grouped GEMM's tile configuration (see bpx_autotune) and
 * re-plans the GEMM table if the tile width changes (synchronizes). */
int bpx_group_set_config(bpx_group* group, int gemm_config, bpx_stream stream);

/* Tile autotuner for the grouped GEMM: times each candidate configuration
 * (NULL / 0 = a built-in list) on the group's own jobs and keeps the fastest.
 * Synchronizes; not capturable. */
int bpx_group_autotune(bpx_group* group, const int* configs, int nconfigs, bpx_stream stream,
                       int* best_config, float* best_ms);

/* Tile autotuner for one coded multiplication on the tensor cores: runs the
 * whole path once, then times the GEMM under each candidate configuration.
 * gemm_config = band * 1000 + seg_kb * 10 + tile, tile 1 = 128x256 and
 * 2 = 128x128 output tiles, 5 / 6 = tiles 1 / 2 with 32-wide instead of
 * 64-wide k-slices, 0 / 9 = 256x256 tiles computed by CTA-pair MMAs
 * (cta_group::2; each CTA of the cluster holds 128 rows of A and half of
 * the B tile) with 64- / 32-wide k-slices; seg_kb = k-blocks of 64 per TMEM
 * accumulation segment, band = m-tiles (or m-tile pairs) per rasterisation
 * band.  gemm_config 0 = the default, 8080.  Precisions BPX_BF16,
 * BPX_BF16X3 and BPX_EXACT (which uses the tile shape, pairing, k-slice and
 * band, with its own exact segment length; its default is also 8080).
 * Tile codes 3, 4, 7 and 8 name no kernel (BPX_ERR_INVAL).  No kernel loads
 * by TMA multicast.  Synchronizes. */
int bpx_autotune(const bpx_code* code, const float* d_A, const float* d_B, int M, int N, int K, int h,
                 int precision, const uint8_t* d_erasure_mask, float* d_C, void* d_ws, size_t ws_bytes,
                 const int* configs, int nconfigs, bpx_stream stream, int* best_config, float* best_ms);

/* Peel-schedule autotuner of a group: times the grouped numeric peel (a4)
 * with each job's float4 columns cut so that the job gets about `targets[i]`
 * CTAs (NULL / 0 = a built-in list from 1/8 to 8 x the SM count; the default
 * plan aims at 4 x the SM count), on the group's own plans and products (one full
 * run first), keeps the fastest plan for later runs and graph launches, and
 * reports it.  Synchronizes; not capturable. */
int bpx_group_autotune_peel(bpx_group* group, const int* targets, int ntargets, bpx_stream stream,
                            int* best_target, float* best_ms);

/* Peel-schedule autotuner for one coded multiplication: runs the whole path
 * once, then times the numeric peel (a4, bpx_peel_decode over the staged
 * products) with opts->peel_ctas = each of `ctas` (NULL / 0 = a built-in list
 * from half to 8 x the SM count) and returns the fastest count (pass it as
 * bpx_opts.peel_ctas).  Precisions BPX_FP32, BPX_BF16, BPX_BF16X3, BPX_MXFP8.
 * d_C holds the decoded C afterwards.  Synchronizes. */
int bpx_autotune_peel(const bpx_code* code, const float* d_A, const float* d_B, int M, int N, int K, int h,
                      int precision, const uint8_t* d_erasure_mask, float* d_C, void* d_ws, size_t ws_bytes,
                      const int* ctas, int nctas, bpx_stream stream, int* best_ctas, float* best_ms);

void bpx_group_free(bpx_group* group);

/* a1 without any device allocation by the caller or the library (the paper has
 * no counterpart: this is a deployment convenience).  Same computation and
 * outputs as bpx_schedule, but the graph copy and the peel plan live in one
 * fixed 8 MiB array inside the library instead of a caller workspace.  Meant
 * for callers that cannot allocate device memory -- e.g. code embedded in a
 * runtime that owns the device pool, or latency-critical paths that cannot
 * take the synchronisation of cudaMalloc/cudaFree.  The caller still passes
 * the mask (input) and the outputs; NULL outputs are skipped.
 *   - The first call on each device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     The address is kept for the life of the process: after a device reset
 *     (cudaDeviceReset, or anything else that replaces the device's primary
 *     context) do not call this entry point again in that process.
 *   - Codes whose scratch exceeds 8 MiB are rejected with BPX_ERR_INVAL
 *     (roughly 3 num_edges + 9 num_cells + 8 num_sources int32 words, plus
 *     the code's two-dimensional term lists).
 *   - Every call uploads its code's graph into the shared array and reuses
 *     it, so calls that overlap on the GPU (other streams, other threads)
 *     race on it: serialise them.  The plan stays in the array until the next
 *     call; it is not usable by the workspace-based calls. */
int bpx_schedule_noalloc(const bpx_code* code, const uint8_t* d_erasure_mask,
                         int32_t* d_peel_order, uint8_t* d_recovered, int32_t* d_info,
                         bpx_stream stream);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * thread that waits, through the same bounded mbarrier wait the tensor-core
 * GEMM uses, on a barrier nothing ever arrives at.  After budget_cycles
 * (0 < budget <= the GEMM's own budget of 4e9 cycles) the wait gives up and the
 * kernel writes BPX_ERR_TIMEOUT into d_info[BPX_INFO_STATUS] and
 * [BPX_INFO_DEVICE_ERR] (cycles waited in d_info[6]) and returns normally, so
 * the context stays usable.  The GEMM handles an expired wait the same way
 * (after letting its in-flight copies land and freeing its TMEM). */
int bpx_selftest_wait_timeout(long long budget_cycles, int32_t* d_info, bpx_stream stream);

/* Default options (direct_write = 1, compensate_depth = -1, autos). */
bpx_opts bpx_default_opts(void);

/* Library version and the architecture it was compiled for ("sm_103a"). */
const char* bpx_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* BPX_H */
