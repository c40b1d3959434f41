// Batched T-products (qtp_batch_plan_*, qtp_forward_batched): thousands of
// independent products C_i = A_i * B_i of uneven (m, n, s, p), each by
// Algorithm 5.1, in grouped launches (the transforms one per tube length, the
// products one) replayed from a CUDA graph.
//
//   1. fft_fwd_grouped  - every tube of every A_i and B_i (Step 1): one
//                         launch per distinct tube length p
//   2. products         - all frequencies of all products (Step 2): one
//                         persistent tcgen05 launch, or one FP32 launch
//   3. fft_inv_grouped  - every tube of every C_i (Step 3), one launch per p
//
// The plan buckets the products by tube length p, then by size, so that CTAs
// working at the same time share a kernel specialisation and their
// products' spectra stay in L2; the pointer table keeps the caller's order.
// Tensor-core products can leave the grouped kernel (128 x 64 tiles, both
// output halves per tile) for the single-product kernel (128 x 256 or
// 128 x 128 tiles per output half, accumulator mode by K): a split-BF16
// product whose reduction (n per half) is longer than the grouped kernel's
// single accumulator keeps within 1e-5 (kTcSingleMaxK) always does, and with
// QTP_BATCH_AUTOTUNE every product with min(m, s) at or above a threshold the
// plan picks by timing (its wide MMAs cost less per column than the grouped
// kernel's narrow ones).  Those run one launch each after the grouped launch,
// spread over the plan's auxiliary streams, inside the same graph.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "qtp_internal.h"

using namespace qtp;

// The CTAs of one tube length in a grouped transform: one launch.
struct FftRange {
  int p;
  long long block0, nblocks;
  size_t smem;
};

struct qtp_batch_plan {
  int count = 0;
  int precision = 0;
  int fmt = 0;
  unsigned flags = 0;
  int device = 0;
  int num_sms = 0;
  std::vector<qtp_shape> shapes;
  size_t ws_bytes = 0;
  // device tables
  float2* d_tw = nullptr;
  FftGroupJob* d_fwd = nullptr;
  FftGroupJob* d_inv = nullptr;
  int* d_fwd_job = nullptr;   // job index of every CTA of the grouped FFTs
  int* d_inv_job = nullptr;
  int* d_prob_tile = nullptr; // product of every tile of the grouped FP32 products
  GroupProblem* d_probs = nullptr;
  void* d_tmaps = nullptr;  // 2 x 128 B per product (tensor-core path)
  const float2** d_ptrs = nullptr;
  int* d_err = nullptr;
  int n_fwd = 0, n_inv = 0, n_probs = 0;
  long long fwd_blocks = 0, inv_blocks = 0, total_tiles = 0;
  std::vector<FftRange> fwd_ranges, inv_ranges;
  // host copies needed to encode tensor maps
  std::vector<GroupProblem> h_probs;
  std::vector<int> prod_of_prob;  // product index of each GroupProblem
  // every product in walk order with its workspace offsets, and those that
  // take the single-product tensor-core kernel (long reductions, wide routing)
  struct LongProduct {
    int idx, m, n, s, p;
    size_t sa, sb, sc;  // workspace offsets of the spectra of A, B and C_hat
  };
  std::vector<LongProduct> prods;
  std::vector<LongProduct> long_probs;
  int route_min = 0x7fffffff;  // min(m, s) from which products take the single-product kernel
  static constexpr int kAux = 8;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kAux] = {};
  float tune_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // products time per candidate threshold (autotune)
  int tune_n = 0;
  void* h_tmaps = nullptr;        // pinned
  char* tmaps_for_ws = nullptr;   // workspace base the device tensor maps point into
  // per-call pointer staging (pinned, 2 slots) and stream plumbing
  const float2** h_ptrs[2] = {nullptr, nullptr};
  cudaEvent_t staged[2] = {nullptr, nullptr};
  int slot = 0;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;
  char* graph_ws = nullptr;
  int graph_tracing = 0;
  int tracing = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

#define BP_CUDA(call, what)                                                                              \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return set_error(QTP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_));      \
  } while (0)

void free_plan(qtp_batch_plan* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (int i = 0; i < 4; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  for (int i = 0; i < 2; ++i) {
    if (b->staged[i]) cudaEventDestroy(b->staged[i]);
    if (b->h_ptrs[i]) cudaFreeHost(b->h_ptrs[i]);
  }
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (int i = 0; i < qtp_batch_plan::kAux; ++i) {
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
    if (b->aux[i]) cudaStreamDestroy(b->aux[i]);
  }
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->h_tmaps) cudaFreeHost(b->h_tmaps);
  cudaFree(b->d_tw);
  cudaFree(b->d_fwd);
  cudaFree(b->d_inv);
  cudaFree(b->d_fwd_job);
  cudaFree(b->d_inv_job);
  cudaFree(b->d_prob_tile);
  cudaFree(b->d_probs);
  cudaFree(b->d_tmaps);
  cudaFree(b->d_ptrs);
  cudaFree(b->d_err);
  delete b;
}

// Trace event i on st.  While st is capturing a graph, the record must be an
// external event-record node, or the host could not wait on it later.
void trace(qtp_batch_plan* b, int i, cudaStream_t st, bool capturing) {
  if (!b->tracing) return;
  if (capturing) cudaEventRecordWithFlags(b->ev[i], st, cudaEventRecordExternal);
  else cudaEventRecord(b->ev[i], st);
}

// Step 2 on the tensor cores: the products that take the single-product
// kernel, dealt round-robin over the auxiliary streams, forked from st before
// the grouped launch and joined back after it, so that their CTAs fill the
// SMs that the persistent grouped kernel's tail frees (4096-product batch:
// products 31.4 -> 30.2 ms against a fork after the grouped kernel and four
// streams).
qtp_status enqueue_tc_products(qtp_batch_plan* b, char* ws, cudaStream_t st) {
  const int np = b->fmt == FMT_BF16X3 ? 4 : 2;
  const int na = (int)std::min<size_t>(qtp_batch_plan::kAux, b->long_probs.size());
  if (na > 0) {
    BP_CUDA(cudaEventRecord(b->ev_fork, st), "fork");
    for (int a = 0; a < na; ++a) BP_CUDA(cudaStreamWaitEvent(b->aux[a], b->ev_fork, 0), "fork");
  }
  BP_CUDA(launch_gemm_tc_grouped(b->d_probs, b->n_probs, b->total_tiles, np, ws, b->d_err, b->num_sms, st),
          "batched products (tensor cores)");
  for (size_t i = 0; i < b->long_probs.size(); ++i) {
    const auto& L = b->long_probs[i];
    const TcProblem pr = make_tc_fwd(L.m, L.n, L.s, L.p, np, TILE_AUTO, ws + L.sa, ws + L.sb, (float2*)(ws + L.sc));
    char msg[256] = "";
    cudaError_t e = launch_gemm_tc(pr, b->d_err, b->aux[i % na], msg, sizeof(msg));
    if (e != cudaSuccess)
      return set_error(QTP_ERR_CUDA, "batched products (single-product kernel): %s %s", cudaGetErrorString(e), msg);
  }
  for (int a = 0; a < na; ++a) {
    BP_CUDA(cudaEventRecord(b->ev_join[a], b->aux[a]), "join");
    BP_CUDA(cudaStreamWaitEvent(st, b->ev_join[a], 0), "join");
  }
  return QTP_OK;
}

// The grouped launches of one forward call, on stream st.
qtp_status enqueue(qtp_batch_plan* b, char* ws, cudaStream_t st, bool capturing) {
  trace(b, 0, st, capturing);
  for (const FftRange& r : b->fwd_ranges)
    BP_CUDA(launch_fft_fwd_grouped(b->d_fwd, b->d_fwd_job, r.block0, r.nblocks, r.p, b->fmt, b->d_ptrs, ws, b->d_tw,
                                   r.smem, st),
            "batched forward FFT");
  trace(b, 1, st, capturing);
  if (b->precision == QTP_PREC_FP32) {
    BP_CUDA(launch_gemm_simt_grouped(b->d_probs, b->d_prob_tile, b->total_tiles, ws, st), "batched products (fp32)");
  } else {
    qtp_status r = enqueue_tc_products(b, ws, st);
    if (r != QTP_OK) return r;
  }
  trace(b, 2, st, capturing);
  for (const FftRange& r : b->inv_ranges)
    BP_CUDA(launch_fft_inv_grouped(b->d_inv, b->d_inv_job, r.block0, r.nblocks, r.p, b->d_ptrs, ws, b->d_tw, r.smem,
                                   st),
            "batched inverse FFT");
  trace(b, 3, st, capturing);
  return QTP_OK;
}

// Tensor maps of every product's spectra for the workspace at ws (async upload on st).
qtp_status encode_tmaps(qtp_batch_plan* b, char* ws, cudaStream_t st) {
  const int np = b->fmt == FMT_BF16X3 ? 4 : 2;
  char msg[256];
  for (int i = 0; i < b->n_probs; ++i) {
    const GroupProblem& P = b->h_probs[i];
    char* tA = (char*)b->h_tmaps + (size_t)i * 256;
    if (!encode_group_map(tA, ws + P.sa_off, P.M, P.K, P.lda, P.p, np, false, !P.trans, msg, sizeof(msg)))
      return set_error(QTP_ERR_CUDA, "batched tensor map (A of product %d): %s", b->prod_of_prob[i], msg);
    if (!encode_group_map(tA + 128, ws + P.sb_off, P.K, P.N, P.ldb, P.p, np, true, false, msg, sizeof(msg)))
      return set_error(QTP_ERR_CUDA, "batched tensor map (B of product %d): %s", b->prod_of_prob[i], msg);
  }
  BP_CUDA(cudaMemcpyAsync(b->d_tmaps, b->h_tmaps, (size_t)b->n_probs * 256, cudaMemcpyHostToDevice, st),
          "upload tensor maps");
  b->tmaps_for_ws = ws;
  return QTP_OK;
}

// The products' tile space for a routing threshold: products with a long
// reduction (split-BF16) or with min(m, s) >= route_min take the
// single-product kernel (long_probs), the others get their grouped tiles.
void layout_products(qtp_batch_plan* b, int route_min) {
  const bool tc = b->precision != QTP_PREC_FP32;
  const int fmt = b->fmt;
  const int BMt = tc ? kGroupTcBM : kGroupSimtBM;
  const int BNt = tc ? kGroupTcBN : kGroupSimtBN;
  b->h_probs.clear();
  b->prod_of_prob.clear();
  b->long_probs.clear();
  long long tiles = 0;
  for (const auto& L : b->prods) {
    if (tc && ((fmt == FMT_BF16X3 && L.n > kTcSingleMaxK) || std::min(L.m, L.s) >= route_min)) {
      b->long_probs.push_back(L);
      continue;
    }
    GroupProblem P;
    memset(&P, 0, sizeof(P));
    P.tile_begin = tiles;
    P.sa_off = (long long)L.sa;
    P.sb_off = (long long)L.sb;
    P.out_off = (long long)L.sc;
    P.M = L.m;
    P.N = L.s;
    P.K = L.n;
    P.p = L.p;
    // Tensor cores: 128-row tiles, MMA width the tile's columns rounded up to
    // 16; computing C^T = B^T A^T instead when that pads less (the larger of
    // m and s then fills the 128 rows).
    P.bn = BNt;
    P.trans = 0;
    if (tc) {
      auto padded = [](long long rows, long long cols) {
        return (rows + 127) / 128 * 128 * ((cols + 15) / 16 * 16);
      };
      P.trans = padded(L.s, L.m) < padded(L.m, L.s) ? 1 : 0;
    }
    const int trows = P.trans ? L.s : L.m, tcols = P.trans ? L.m : L.s;
    P.tiles_m = (trows + BMt - 1) / BMt;
    P.tiles_n = (tcols + BNt - 1) / BNt;
    P.lda = (int)spec_ld_of(fmt, L.n);
    P.ldb = (int)spec_ld_of(fmt, L.s);
    // tensor cores: a tile computes both output halves; FP32: one tile per half
    tiles += (long long)P.tiles_m * P.tiles_n * (tc ? 1 : 2) * L.p;
    b->h_probs.push_back(P);
    b->prod_of_prob.push_back(L.idx);
  }
  b->n_probs = (int)b->h_probs.size();
  b->total_tiles = tiles;
  b->route_min = route_min;
  b->tmaps_for_ws = nullptr;  // the tensor maps follow the grouped products
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Tensor maps live in d_tmaps: grouped product i's pair at 256 i.
void set_tmap_slots(qtp_batch_plan* b) {
  if (b->precision == QTP_PREC_FP32) return;
  for (int i = 0; i < b->n_probs; ++i) {
    b->h_probs[i].tmA = (char*)b->d_tmaps + (size_t)i * 256;
    b->h_probs[i].tmB = (char*)b->d_tmaps + (size_t)i * 256 + 128;
  }
}

// Products time (ms, mean of reps after one warm-up) of the current layout on
// workspace ws, on the plan's stream.
qtp_status time_tc_products(qtp_batch_plan* b, char* ws, int reps, float* ms) {
  qtp_status r = encode_tmaps(b, ws, b->cap);
  if (r != QTP_OK) return r;
  BP_CUDA(cudaMemcpyAsync(b->d_probs, b->h_probs.data(), sizeof(GroupProblem) * std::max(b->n_probs, 1),
                          cudaMemcpyHostToDevice, b->cap),
          "upload products");
  if ((r = enqueue_tc_products(b, ws, b->cap)) != QTP_OK) return r;
  BP_CUDA(cudaEventRecord(b->ev[0], b->cap), "time products");
  for (int i = 0; i < reps; ++i)
    if ((r = enqueue_tc_products(b, ws, b->cap)) != QTP_OK) return r;
  BP_CUDA(cudaEventRecord(b->ev[1], b->cap), "time products");
  BP_CUDA(cudaEventSynchronize(b->ev[1]), "time products");
  BP_CUDA(cudaEventElapsedTime(ms, b->ev[0], b->ev[1]), "time products");
  *ms /= reps;
  return QTP_OK;
}

// Autotuner of the routing threshold (QTP_BATCH_AUTOTUNE): the products of
// this batch are timed, on a zeroed scratch workspace, for every candidate
// threshold (grouped kernel only, then min(m, s) >= 192, 128, 96, 64, 48 to
// the single-product kernel); the fastest is kept and cached per (device,
// precision, shapes) for the process.
std::mutex g_route_mu;
std::map<std::string, int> g_route_cache;

std::string route_key(const qtp_batch_plan* b) {
  unsigned long long h = 1469598103934665603ull;  // FNV-1a over the shapes
  for (const qtp_shape& q : b->shapes)
    for (int v : {q.m, q.n, q.s, q.p}) {
      h ^= (unsigned)v;
      h *= 1099511628211ull;
    }
  cudaDeviceProp prop;
  std::string dev = "dev";
  if (cudaGetDeviceProperties(&prop, b->device) == cudaSuccess) dev = prop.name;
  char buf[320];
  snprintf(buf, sizeof(buf), "%s:%d:%d:%016llx", dev.c_str(), b->precision, b->count, h);
  return buf;
}

qtp_status autotune_routing(qtp_batch_plan* b) {
  std::lock_guard<std::mutex> lock(g_route_mu);
  const std::string key = route_key(b);
  auto hit = g_route_cache.find(key);
  if (hit != g_route_cache.end()) {
    layout_products(b, hit->second);
    set_tmap_slots(b);
    BP_CUDA(cudaMemcpy(b->d_probs, b->h_probs.data(), sizeof(GroupProblem) * std::max(b->n_probs, 1),
                       cudaMemcpyHostToDevice),
            "upload products");
    return QTP_OK;
  }
  const int cands[] = {0x7fffffff, 192, 128, 96, 64, 48};
  char* ws = nullptr;
  cudaError_t e = cudaMalloc(&ws, std::max(b->ws_bytes, (size_t)256));
  if (e == cudaSuccess) e = cudaMemset(ws, 0, b->ws_bytes);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!b->ev[i]) e = cudaEventCreate(&b->ev[i]);
  if (e != cudaSuccess) {
    cudaFree(ws);
    return set_error(QTP_ERR_CUDA, "batch autotune scratch: %s", cudaGetErrorString(e));
  }
  int best = cands[0];
  float best_ms = 1e30f;
  qtp_status r = QTP_OK;
  b->tune_n = 0;
  for (int c : cands) {
    layout_products(b, c);
    set_tmap_slots(b);
    float ms = 0.f;
    r = time_tc_products(b, ws, 2, &ms);
    if (r != QTP_OK) break;
    b->tune_ms[b->tune_n++] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaStreamSynchronize(b->cap);
  cudaFree(ws);
  if (!b->tracing)  // the events were only borrowed for the timing
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(b->ev[i]);
      b->ev[i] = nullptr;
    }
  if (r != QTP_OK) return r;
  int v = 0;
  BP_CUDA(cudaMemcpy(&v, b->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (v != 0) {
    cudaMemset(b->d_err, 0, sizeof(int));
    return set_error(QTP_ERR_TIMEOUT, "batch autotune: a device-side wait gave up (code %d)", v);
  }
  layout_products(b, best);
  set_tmap_slots(b);
  BP_CUDA(cudaMemcpy(b->d_probs, b->h_probs.data(), sizeof(GroupProblem) * std::max(b->n_probs, 1),
                     cudaMemcpyHostToDevice),
          "upload products");
  g_route_cache[key] = best;
  return QTP_OK;
}

}  // namespace

extern "C" {

qtp_status qtp_batch_plan_route(const qtp_batch_plan* b, int* route_min, float* tuned_ms, int* tuned_count) {
  if (!b) return set_error(QTP_ERR_INVALID_ARG, "plan is NULL");
  if (route_min) *route_min = b->route_min;
  if (tuned_count) *tuned_count = b->tune_n;
  if (tuned_ms)
    for (int i = 0; i < b->tune_n; ++i) tuned_ms[i] = b->tune_ms[i];
  return QTP_OK;
}

qtp_status qtp_batch_plan_create(qtp_batch_plan** out, const qtp_shape* shapes, int count, int precision,
                                 unsigned flags) {
  clear_error();
  if (!out) return set_error(QTP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!shapes || count < 1) return set_error(QTP_ERR_INVALID_ARG, "need at least one shape");
  if (count > (1 << 20)) return set_error(QTP_ERR_INVALID_ARG, "at most 2^20 products per batch");
  if (precision != QTP_PREC_FP32 && precision != QTP_PREC_BF16X3 && precision != QTP_PREC_BF16)
    return set_error(QTP_ERR_INVALID_ARG, "unknown precision %d", precision);
  if (flags & ~(QTP_BATCH_NO_GRAPH | QTP_BATCH_AUTOTUNE)) return set_error(QTP_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  const long long lim = 1LL << 31;
  for (int i = 0; i < count; ++i) {
    const qtp_shape& q = shapes[i];
    if (q.m < 1 || q.n < 1 || q.s < 1 || q.p < 1)
      return set_error(QTP_ERR_INVALID_ARG, "product %d: dimensions must be >= 1", i);
    if (q.m > (1 << 20) || q.n > (1 << 20) || q.s > (1 << 20))
      return set_error(QTP_ERR_INVALID_ARG, "product %d: m, n, s must be <= 2^20", i);
    if (q.p > QTP_MAX_P) return set_error(QTP_ERR_UNSUPPORTED, "product %d: p=%d exceeds %d", i, q.p, QTP_MAX_P);
    if ((long long)q.m * q.n * q.p >= lim || (long long)q.n * q.s * q.p >= lim || (long long)q.m * q.s * q.p >= lim)
      return set_error(QTP_ERR_INVALID_ARG, "product %d: a tensor plane exceeds 2^31 entries", i);
  }
  if (precision != QTP_PREC_FP32 && !tc_supported())
    return set_error(QTP_ERR_UNSUPPORTED, "BF16 tensor-core products need an sm_103 device (tcgen05)");

  qtp_batch_plan* b = new qtp_batch_plan();
  b->count = count;
  b->precision = precision;
  b->fmt = spec_format_of(precision);
  b->flags = flags;
  b->shapes.assign(shapes, shapes + count);
  const int fmt = b->fmt;
  const bool tc = precision != QTP_PREC_FP32;

  // bucket by p, then by work (largest first)
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const qtp_shape& a = shapes[x];
    const qtp_shape& c = shapes[y];
    if (a.p != c.p) return a.p < c.p;
    return (long long)a.m * a.n * a.s > (long long)c.m * c.n * c.s;
  });

  // twiddle tables of the distinct tube lengths
  std::map<int, int> tw_off;
  int tw_total = 0;
  for (int i = 0; i < count; ++i)
    if (!tw_off.count(shapes[i].p)) {
      tw_off[shapes[i].p] = tw_total;
      tw_total += shapes[i].p;
    }

  // workspace layout, FFT jobs, product tiles
  std::vector<FftGroupJob> fwd, inv;
  size_t off = 0;
  long long fb = 0, ib = 0;
  for (int idx : order) {
    const qtp_shape& q = shapes[idx];
    const int Tf = fft_tubes_per_block(q.p, false), Ti = fft_tubes_per_block(q.p, true);
    const RadixPlan rp = make_radix_plan(q.p);
    const size_t sa = off;
    off += spec_bytes_of(fmt, q.p, q.m, q.n);
    const size_t sb = off;
    off += spec_bytes_of(fmt, q.p, q.n, q.s);
    const size_t sc = off;
    off += c32_bytes_of(q.p, q.m, q.s);
    auto job = [&](int which, int rows, int cols, size_t spec, long long& counter) {
      const int T = which == 2 ? Ti : Tf;
      FftGroupJob j;
      memset(&j, 0, sizeof(j));
      j.block_begin = counter;
      j.spec_off = (long long)spec;
      j.prod = idx;
      j.which = which;
      j.rows = rows;
      j.cols = cols;
      j.ld = which == 2 ? cols : (int)spec_ld_of(fmt, cols);
      j.p = q.p;
      j.T = T;
      j.tw_off = tw_off[q.p];
      j.rp = rp;
      const int run_cols = which == 2 ? cols : fft_fwd_run_cols(q.p, fmt, cols);
      counter += (2LL * rows * run_cols + T - 1) / T;
      return j;
    };
    fwd.push_back(job(0, q.m, q.n, sa, fb));
    fwd.push_back(job(1, q.n, q.s, sb, fb));
    inv.push_back(job(2, q.m, q.s, sc, ib));
    b->prods.push_back({idx, q.m, q.n, q.s, q.p, sa, sb, sc});
  }
  const char* route_env = getenv("QTP_BATCH_ROUTE_MIN");
  layout_products(b, route_env ? atoi(route_env) : 0x7fffffff);
  const long long tiles = b->total_tiles;
  if (fb > 0x7fffffffLL || ib > 0x7fffffffLL || (!tc && tiles > 0x7fffffffLL)) {
    free_plan(b);
    return set_error(QTP_ERR_UNSUPPORTED, "batch too large for one grouped launch");
  }
  b->ws_bytes = off;
  b->n_fwd = (int)fwd.size();
  b->n_inv = (int)inv.size();
  b->fwd_blocks = fb;
  b->inv_blocks = ib;
  // launch ranges: jobs are ordered by p, so each p's CTAs are contiguous
  auto ranges = [](const std::vector<FftGroupJob>& jobs, long long total, bool inv) {
    std::vector<FftRange> r;
    for (size_t j = 0; j < jobs.size(); ++j) {
      if (r.empty() || r.back().p != jobs[j].p) {
        if (!r.empty()) r.back().nblocks = jobs[j].block_begin - r.back().block0;
        r.push_back(FftRange{jobs[j].p, jobs[j].block_begin, 0, fft_smem_bytes_for(jobs[j].p, inv)});
      }
    }
    if (!r.empty()) r.back().nblocks = total - r.back().block0;
    return r;
  };
  b->fwd_ranges = ranges(fwd, fb, false);
  b->inv_ranges = ranges(inv, ib, true);

  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tw, sizeof(float2) * tw_total);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_fwd, sizeof(FftGroupJob) * fwd.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_inv, sizeof(FftGroupJob) * inv.size());
  // product tables sized for every product (the routing may change which are grouped)
  const size_t nprob_alloc = (size_t)count;
  if (e == cudaSuccess) e = cudaMalloc(&b->d_probs, sizeof(GroupProblem) * nprob_alloc);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ptrs, sizeof(float2*) * 3 * count);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e == cudaSuccess && tc) e = cudaMalloc(&b->d_tmaps, nprob_alloc * 256);
  if (e == cudaSuccess && tc) e = cudaMallocHost(&b->h_tmaps, nprob_alloc * 256);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMallocHost(&b->h_ptrs[i], sizeof(float2*) * 3 * count);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < qtp_batch_plan::kAux && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->aux[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_plan(b);
    return set_error(QTP_ERR_CUDA, "batch plan allocation: %s", cudaGetErrorString(e));
  }
  set_tmap_slots(b);
  for (auto& kv : tw_off) {
    e = launch_twiddles(b->d_tw + kv.second, kv.first, 0);
    if (e != cudaSuccess) break;
  }
  // direct lookup tables: CTA -> job, tile -> product
  std::vector<int> fwd_job((size_t)fb), inv_job((size_t)ib), prob_tile;
  for (size_t j = 0; j < fwd.size(); ++j) {
    const long long end = j + 1 < fwd.size() ? fwd[j + 1].block_begin : fb;
    for (long long k = fwd[j].block_begin; k < end; ++k) fwd_job[(size_t)k] = (int)j;
  }
  for (size_t j = 0; j < inv.size(); ++j) {
    const long long end = j + 1 < inv.size() ? inv[j + 1].block_begin : ib;
    for (long long k = inv[j].block_begin; k < end; ++k) inv_job[(size_t)k] = (int)j;
  }
  if (!tc) {
    prob_tile.resize((size_t)tiles);
    for (int g = 0; g < b->n_probs; ++g) {
      const long long end = g + 1 < b->n_probs ? b->h_probs[g + 1].tile_begin : tiles;
      for (long long k = b->h_probs[g].tile_begin; k < end; ++k) prob_tile[(size_t)k] = g;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_fwd_job, sizeof(int) * fwd_job.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_inv_job, sizeof(int) * inv_job.size());
  if (e == cudaSuccess && !tc) e = cudaMalloc(&b->d_prob_tile, sizeof(int) * std::max(prob_tile.size(), (size_t)1));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_fwd_job, fwd_job.data(), sizeof(int) * fwd_job.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_inv_job, inv_job.data(), sizeof(int) * inv_job.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tc)
    e = cudaMemcpy(b->d_prob_tile, prob_tile.data(), sizeof(int) * prob_tile.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_fwd, fwd.data(), sizeof(FftGroupJob) * fwd.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_inv, inv.data(), sizeof(FftGroupJob) * inv.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && b->n_probs > 0)
    e = cudaMemcpy(b->d_probs, b->h_probs.data(), sizeof(GroupProblem) * b->n_probs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_plan(b);
    return set_error(QTP_ERR_CUDA, "batch plan set-up: %s", cudaGetErrorString(e));
  }
  if (tc && (flags & QTP_BATCH_AUTOTUNE) && !route_env) {
    qtp_status r = autotune_routing(b);
    if (r != QTP_OK) {
      free_plan(b);
      return r;
    }
  }
  *out = b;
  return QTP_OK;
}

qtp_status qtp_batch_plan_destroy(qtp_batch_plan* b) {
  if (!b) return QTP_OK;
  if (b->cap) cudaStreamSynchronize(b->cap);
  free_plan(b);
  return QTP_OK;
}

qtp_status qtp_batch_workspace_size(const qtp_batch_plan* b, size_t* bytes) {
  if (!b) return set_error(QTP_ERR_INVALID_ARG, "plan is NULL");
  if (!bytes) return set_error(QTP_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = b->ws_bytes;
  return QTP_OK;
}

qtp_status qtp_forward_batched(qtp_batch_plan* b, const float* const* A, const float* const* B, float* const* C,
                               void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!b) return set_error(QTP_ERR_INVALID_ARG, "plan is NULL");
  if (!A || !B || !C) return set_error(QTP_ERR_INVALID_ARG, "pointer arrays must not be NULL");
  if (!workspace || ((uintptr_t)workspace & 255) != 0)
    return set_error(QTP_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < b->ws_bytes)
    return set_error(QTP_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, b->ws_bytes);
  for (int i = 0; i < b->count; ++i) {
    const void* ps[3] = {A[i], B[i], C[i]};
    for (int k = 0; k < 3; ++k)
      if (!ps[k] || ((uintptr_t)ps[k] & 15) != 0)
        return set_error(QTP_ERR_INVALID_ARG, "product %d: %c is NULL or not 16-byte aligned", i, "ABC"[k]);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = (char*)workspace;
  // stage this call's pointers (the slot's previous copy has finished once its event has)
  const int slot = b->slot;
  b->slot ^= 1;
  BP_CUDA(cudaEventSynchronize(b->staged[slot]), "wait for pointer staging");
  const float2** hp = b->h_ptrs[slot];
  for (int i = 0; i < b->count; ++i) {
    hp[3 * i] = reinterpret_cast<const float2*>(A[i]);
    hp[3 * i + 1] = reinterpret_cast<const float2*>(B[i]);
    hp[3 * i + 2] = reinterpret_cast<const float2*>(C[i]);
  }
  // the plan's stream follows the caller's stream
  BP_CUDA(cudaEventRecord(b->ev_in, st), "record entry event");
  BP_CUDA(cudaStreamWaitEvent(b->cap, b->ev_in, 0), "join plan stream");
  BP_CUDA(cudaMemcpyAsync(b->d_ptrs, hp, sizeof(float2*) * 3 * b->count, cudaMemcpyHostToDevice, b->cap),
          "upload pointer table");
  BP_CUDA(cudaEventRecord(b->staged[slot], b->cap), "record staging event");
  const bool tc = b->precision != QTP_PREC_FP32;
  if (tc && b->tmaps_for_ws != ws) {
    qtp_status r = encode_tmaps(b, ws, b->cap);
    if (r != QTP_OK) return r;
    // the next copy into h_tmaps must wait for this one: make it synchronous
    BP_CUDA(cudaStreamSynchronize(b->cap), "tensor-map upload");
  }
  if (b->flags & QTP_BATCH_NO_GRAPH) {
    qtp_status r = enqueue(b, ws, b->cap, false);
    if (r != QTP_OK) return r;
  } else {
    if (!b->graph || b->graph_ws != ws || b->graph_tracing != b->tracing) {
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      BP_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
      qtp_status r = enqueue(b, ws, b->cap, true);
      cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
      if (r != QTP_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (ce != cudaSuccess) return set_error(QTP_ERR_CUDA, "end capture: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return set_error(QTP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
      b->graph_ws = ws;
      b->graph_tracing = b->tracing;
    }
    BP_CUDA(cudaGraphLaunch(b->graph, b->cap), "graph launch");
  }
  BP_CUDA(cudaEventRecord(b->ev_out, b->cap), "record exit event");
  BP_CUDA(cudaStreamWaitEvent(st, b->ev_out, 0), "join caller stream");
  return QTP_OK;
}

qtp_status qtp_batch_plan_set_tracing(qtp_batch_plan* b, int enable) {
  if (!b) return set_error(QTP_ERR_INVALID_ARG, "plan is NULL");
  if (enable && !b->tracing) {
    for (int i = 0; i < 4; ++i) BP_CUDA(cudaEventCreate(&b->ev[i]), "create trace event");
    b->tracing = 1;
  } else if (!enable && b->tracing) {
    if (b->cap) cudaStreamSynchronize(b->cap);
    for (int i = 0; i < 4; ++i) {
      cudaEventDestroy(b->ev[i]);
      b->ev[i] = nullptr;
    }
    b->tracing = 0;
  }
  return QTP_OK;
}

qtp_status qtp_batch_stage_times(const qtp_batch_plan* b, float* ms3) {
  if (!b) return set_error(QTP_ERR_INVALID_ARG, "plan is NULL");
  if (!ms3) return set_error(QTP_ERR_INVALID_ARG, "ms3 is NULL");
  if (!b->tracing) return set_error(QTP_ERR_INVALID_ARG, "tracing is not enabled on this plan");
  BP_CUDA(cudaEventSynchronize(b->ev[3]), "wait for trace events");
  for (int i = 0; i < 3; ++i) BP_CUDA(cudaEventElapsedTime(&ms3[i], b->ev[i], b->ev[i + 1]), "stage time");
  return QTP_OK;
}

qtp_status qtp_batch_plan_sync(const qtp_batch_plan* b, void* stream) {
  if (!b) return set_error(QTP_ERR_INVALID_ARG, "plan is NULL");
  BP_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "stream synchronize");
  BP_CUDA(cudaStreamSynchronize(b->cap), "plan stream synchronize");
  int v = 0;
  BP_CUDA(cudaMemcpy(&v, b->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (v != 0) {
    cudaMemset(b->d_err, 0, sizeof(int));
    return set_error(QTP_ERR_TIMEOUT, "a device-side wait gave up (code %d)", v);
  }
  return QTP_OK;
}

}  // extern "C"
