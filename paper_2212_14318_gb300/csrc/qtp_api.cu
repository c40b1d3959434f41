// C ABI of libqtp: plans, argument validation, workspace layout and launch
// sequencing of Algorithm 5.1 (Steps 1-3) and of its backward pass.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qtp_internal.h"

using namespace qtp;

namespace {

thread_local char g_err[512] = "";

qtp_status fail(qtp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

qtp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(QTP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define QTP_CUDA(call, what)                 \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

int spec_format(int precision) {
  return precision == QTP_PREC_BF16X3 ? FMT_BF16X3 : (precision == QTP_PREC_BF16 ? FMT_BF16 : FMT_C32);
}

// Leading dimension of a spectra row: TMA needs 16-byte row strides.
long long spec_ld(int fmt, long long cols) { return fmt == FMT_C32 ? cols : round_up(cols, 8); }

size_t spec_bytes(int fmt, long long p, long long rows, long long cols) {
  return align256((size_t)2 * spec_parts(fmt) * p * rows * spec_ld(fmt, cols) * spec_elem_bytes(fmt));
}

size_t c32_bytes(long long p, long long rows, long long cols) {
  return align256((size_t)2 * p * rows * cols * sizeof(float2));
}

// Intermediate of the two-pass long-tube transforms: the largest set of
// tensors transformed in one launch (A with B, dC alone, C alone, dA with dB).
size_t split_scratch_bytes(const qtp_plan* pl) {
  if (pl->fft_split_fwd == FFT_ONE && pl->fft_split_inv == FFT_ONE) return 0;
  const size_t a = align256(fft_split_scratch_bytes(pl->p, pl->m, pl->n));
  const size_t b = align256(fft_split_scratch_bytes(pl->p, pl->n, pl->s));
  const size_t c = align256(fft_split_scratch_bytes(pl->p, pl->m, pl->s));
  return std::max(a + b, c);
}

struct FwdLayout {
  size_t sa, sb, sc, scr, total;
};

FwdLayout fwd_layout(const qtp_plan* pl) {
  const int fmt = spec_format(pl->precision);
  FwdLayout L;
  L.sa = 0;
  L.sb = L.sa + spec_bytes(fmt, pl->p, pl->m, pl->n);
  L.sc = L.sb + spec_bytes(fmt, pl->p, pl->n, pl->s);
  L.scr = L.sc + c32_bytes(pl->p, pl->m, pl->s);
  L.total = L.scr + split_scratch_bytes(pl);
  return L;
}

struct BwdLayout {
  size_t sa, sb, sg, sda, sdb, scr, total;
};

BwdLayout bwd_layout(const qtp_plan* pl) {
  const int fmt = spec_format(pl->precision);
  BwdLayout L;
  L.sa = 0;
  L.sb = L.sa + spec_bytes(fmt, pl->p, pl->m, pl->n);
  L.sg = L.sb + spec_bytes(fmt, pl->p, pl->n, pl->s);
  L.sda = L.sg + spec_bytes(fmt, pl->p, pl->m, pl->s);
  L.sdb = L.sda + c32_bytes(pl->p, pl->m, pl->n);
  L.scr = L.sdb + c32_bytes(pl->p, pl->n, pl->s);
  L.total = L.scr + split_scratch_bytes(pl);
  return L;
}

// Step 1 / Step 3 transforms of a plan: one kernel, or the two-pass form for
// long tubes (scratch: the layout's intermediate).
cudaError_t plan_fft_fwd(const qtp_plan* pl, const FftFwdJob* jobs, int njobs, int fmt, char* scratch,
                         cudaStream_t st) {
  if (pl->fft_split_fwd == FFT_LONG)
    return launch_fft_fwd_long(jobs, njobs, fmt, pl->p, pl->long_n2, pl->d_tw, (float2*)scratch, st);
  if (pl->fft_split_fwd == FFT_SPLIT)
    return launch_fft_fwd_split(jobs, njobs, fmt, pl->p, pl->d_tw, (float2*)scratch, st);
  return launch_fft_fwd(jobs, njobs, fmt, pl->rp, pl->d_tw, st);
}

cudaError_t plan_fft_inv(const qtp_plan* pl, const FftInvJob* jobs, int njobs, char* scratch, cudaStream_t st) {
  if (pl->fft_split_inv == FFT_LONG)
    return launch_fft_inv_long(jobs, njobs, pl->p, pl->long_n2, pl->d_tw, (float2*)scratch, st);
  if (pl->fft_split_inv == FFT_SPLIT) return launch_fft_inv_split(jobs, njobs, pl->p, pl->d_tw, (float2*)scratch, st);
  return launch_fft_inv(jobs, njobs, pl->rp, pl->d_tw, st);
}

// N2 of a plan's compile-time long form (0 when p has none).
int plan_long_n2(const qtp_plan* pl) {
  int n2 = 0;
  if (pl->p <= 128 || !fft_long_dims(pl->p, nullptr, &n2)) return 0;
  return pl->long_n2 ? pl->long_n2 : n2;
}

// Twiddle entries of a plan: w_p^e (e < p), followed, where p has a long
// form (any form may be chosen), by room for the largest N2 table (256).
int plan_twiddle_count(const qtp_plan* pl) {
  return plan_long_n2(pl) ? pl->p + 256 : pl->p;
}

// w_p^e, then w_N2^e (e < N2) of the plan's long form.
cudaError_t plan_twiddles(const qtp_plan* pl, cudaStream_t st) {
  cudaError_t e = launch_twiddles(pl->d_tw, pl->p, st);
  const int n2 = plan_long_n2(pl);
  if (e == cudaSuccess && n2) e = launch_twiddles(pl->d_tw + pl->p, n2, st);
  return e;
}

qtp_status check_plan(const qtp_plan* pl) {
  if (!pl) return fail(QTP_ERR_INVALID_ARG, "plan is NULL");
  return QTP_OK;
}

qtp_status check_dev_ptr(const void* ptr, const char* name, bool allow_null = false) {
  if (!ptr) {
    if (allow_null) return QTP_OK;
    return fail(QTP_ERR_INVALID_ARG, "%s is NULL", name);
  }
  if (((uintptr_t)ptr & 15) != 0) return fail(QTP_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QTP_ERR_INVALID_ARG, "%s: cudaPointerGetAttributes failed (%s)", name, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(QTP_ERR_INVALID_ARG, "%s is not device memory", name);
  return QTP_OK;
}

qtp_status check_host_ptr(const void* ptr, const char* name) {
  if (!ptr) return fail(QTP_ERR_INVALID_ARG, "%s is NULL", name);
  if (((uintptr_t)ptr & 15) != 0) return fail(QTP_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  return QTP_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int nblocks_for(long long rows, long long cols, int p, bool inv) {
  const long long T = fft_tubes_per_block(p, inv);
  return (int)((2 * rows * cols + T - 1) / T);
}

// Forward-transform runs of a rows x cols tensor written in format fmt.
int nblocks_fwd(long long rows, long long cols, int p, int fmt) {
  return nblocks_for(rows, fft_fwd_run_cols(p, fmt, (int)cols), p, false);
}

// Operand view helpers on complex FP32 spectra [plane][f][rows][cols].
CView view(const float2* spec, int plane, int p, long long rows, long long cols, bool row_is_first_index,
           int fneg, int conj) {
  CView v;
  v.base = spec + (long long)plane * p * rows * cols;
  v.fstride = rows * cols;
  // element (r, k) of the view: either (row, col) = (r, k) or (k, r)
  v.rstride = row_is_first_index ? cols : 1;
  v.kstride = row_is_first_index ? 1 : cols;
  v.fneg = fneg;
  v.conj = conj;
  return v;
}

TcView tcv(int tensor, int plane, int fneg, int conj) {
  TcView v;
  v.tensor = tensor;
  v.plane = plane;
  v.fneg = fneg;
  v.conj = conj;
  return v;
}

// Tensor-core problems of the three product kinds (forward, dA, dB) over
// bf16 spectra: which planes, frequencies, conjugations and signs feed each
// (output half, K half).  See run_products_fwd / run_products_bwd.
TcProblem tc_fwd(const qtp_plan* pl, const void* sa, const void* sb, float2* sc) {
  return make_tc_fwd(pl->m, pl->n, pl->s, pl->p, pl->precision == QTP_PREC_BF16X3 ? 4 : 2, pl->tile[0], sa, sb, sc);
}

}  // namespace

TcProblem qtp::make_tc_fwd(int m, int n, int s, int p, int nparts, int tile, const void* sa, const void* sb,
                           float2* sc) {
  TcProblem pr;
  memset(&pr, 0, sizeof(pr));
  pr.kind = TC_FWD;
  pr.tile = tile;
  pr.M = m; pr.N = s; pr.K = n; pr.p = p;
  pr.nparts = nparts;
  pr.a_base[0] = sa; pr.a_rows[0] = m; pr.a_cols[0] = n; pr.a_ld[0] = (int)spec_ld(FMT_BF16, n);
  pr.b_base[0] = sb; pr.b_rows[0] = n; pr.b_cols[0] = s; pr.b_ld[0] = (int)spec_ld(FMT_BF16, s);
  for (int h = 0; h < 2; ++h) {
    pr.a[h][0] = tcv(0, 0, 0, 0);
    pr.a[h][1] = tcv(0, 1, 0, 0);
  }
  pr.b[0][0] = tcv(0, 0, 0, 0); pr.sign[0][0] = 1.f;
  pr.b[0][1] = tcv(0, 1, 1, 1); pr.sign[0][1] = -1.f;
  pr.b[1][0] = tcv(0, 1, 0, 0); pr.sign[1][0] = 1.f;
  pr.b[1][1] = tcv(0, 0, 1, 1); pr.sign[1][1] = 1.f;
  pr.out = sc;
  pr.out_hstride = (long long)p * m * s;
  pr.out_fstride = (long long)m * s;
  pr.out_rstride = s;
  return pr;
}

namespace {

TcProblem tc_bwd_a(const qtp_plan* pl, const void* sb, const void* sg, float2* sda) {
  const int m = pl->m, n = pl->n, s = pl->s, p = pl->p;
  TcProblem pr;
  memset(&pr, 0, sizeof(pr));
  pr.kind = TC_BWD_A;
  pr.tile = pl->tile[1];
  pr.M = m; pr.N = n; pr.K = s; pr.p = p;
  pr.nparts = pl->precision == QTP_PREC_BF16X3 ? 4 : 2;
  pr.a_base[0] = sg; pr.a_rows[0] = m; pr.a_cols[0] = s; pr.a_ld[0] = (int)spec_ld(FMT_BF16, s);
  pr.b_base[0] = sb; pr.b_rows[0] = n; pr.b_cols[0] = s; pr.b_ld[0] = (int)spec_ld(FMT_BF16, s);
  for (int h = 0; h < 2; ++h) {
    pr.a[h][0] = tcv(0, 0, 0, 0);
    pr.a[h][1] = tcv(0, 1, 0, 0);
  }
  pr.b[0][0] = tcv(0, 0, 0, 1); pr.sign[0][0] = 1.f;
  pr.b[0][1] = tcv(0, 1, 0, 1); pr.sign[0][1] = 1.f;
  pr.b[1][0] = tcv(0, 1, 1, 0); pr.sign[1][0] = -1.f;
  pr.b[1][1] = tcv(0, 0, 1, 0); pr.sign[1][1] = 1.f;
  pr.out = sda;
  pr.out_hstride = (long long)p * m * n;
  pr.out_fstride = (long long)m * n;
  pr.out_rstride = n;
  return pr;
}

TcProblem tc_bwd_b(const qtp_plan* pl, const void* sa, const void* sg, float2* sdb) {
  const int m = pl->m, n = pl->n, s = pl->s, p = pl->p;
  TcProblem pr;
  memset(&pr, 0, sizeof(pr));
  pr.kind = TC_BWD_B;
  pr.tile = pl->tile[2];
  pr.M = n; pr.N = s; pr.K = m; pr.p = p;
  pr.nparts = pl->precision == QTP_PREC_BF16X3 ? 4 : 2;
  pr.a_base[0] = sa; pr.a_rows[0] = m; pr.a_cols[0] = n; pr.a_ld[0] = (int)spec_ld(FMT_BF16, n);
  pr.b_base[0] = sg; pr.b_rows[0] = m; pr.b_cols[0] = s; pr.b_ld[0] = (int)spec_ld(FMT_BF16, s);
  for (int h = 0; h < 2; ++h) {
    pr.a[h][0] = tcv(0, 0, 0, 1);
    pr.a[h][1] = tcv(0, 1, 1, 0);
  }
  pr.b[0][0] = tcv(0, 0, 0, 0); pr.sign[0][0] = 1.f;
  pr.b[0][1] = tcv(0, 1, 1, 1); pr.sign[0][1] = 1.f;
  pr.b[1][0] = tcv(0, 1, 0, 0); pr.sign[1][0] = 1.f;
  pr.b[1][1] = tcv(0, 0, 1, 1); pr.sign[1][1] = -1.f;
  pr.out = sdb;
  pr.out_hstride = (long long)p * n * s;
  pr.out_fstride = (long long)n * s;
  pr.out_rstride = s;
  return pr;
}

}  // namespace

// Forward products of small m and s at many frequencies (long tubes) through
// the persistent grouped kernel: one 128 x 64 tile per frequency holds both
// output halves, TMEM is double-buffered and the epilogue of one tile runs
// under the MMAs of the next, where the single-product kernel would start a
// CTA per tiny tile and pay its prologue and epilogue each time (64 x 64 x
// 4096: 402 us).  The problem record and the two tensor maps go to d_blob
// before every products launch by a one-block copy kernel (they travel as its
// parameter); the tensor maps are encoded again only when the spectra move.
struct SmallTiles {
  void* d_blob = nullptr;                        // device: tensor maps (A, B), then the problem record
  alignas(64) unsigned char h_blob[kPutBlobBytes];
  const void* sa = nullptr;                      // spectra the encoded maps describe
  const void* sb = nullptr;
  const void* sc = nullptr;
  int num_sms = 0;
};

namespace {

// The route: tensor-core precisions, a reduction short enough for single
// accumulators in split-BF16 (as in the batch), one grouped tile per
// frequency (max(m, s) <= 128, min(m, s) <= 64: the larger side on the 128
// rows) and enough frequencies for several tiles per SM.  QTP_SMALL_TILES = 0
// keeps the single-product kernel, 1 takes the route whenever the shape fits.
bool small_tiles_route(const qtp_plan* pl) {
  if (pl->precision == QTP_PREC_FP32) return false;
  if (pl->precision == QTP_PREC_BF16X3 && pl->n > kTcSingleMaxK) return false;
  if (fused_small_eligible(pl->m, pl->n, pl->s, pl->p)) return false;
  if (std::max(pl->m, pl->s) > kGroupTcBM || std::min(pl->m, pl->s) > kGroupTcBN) return false;
  int min_p = 256;
  if (const char* env = getenv("QTP_SMALL_TILES")) {
    if (!strcmp(env, "0")) return false;
    if (!strcmp(env, "1")) min_p = 1;
  }
  return pl->p >= min_p;
}

qtp_status run_products_small(const qtp_plan* pl, const void* sa, const void* sb, float2* sc, cudaStream_t st) {
  SmallTiles& S = *pl->small;
  const int fmt = pl->precision == QTP_PREC_BF16X3 ? FMT_BF16X3 : FMT_BF16;
  const int np = fmt == FMT_BF16X3 ? 4 : 2;
  const int m = pl->m, n = pl->n, s = pl->s, p = pl->p;
  GroupProblem P;
  static_assert(256 + sizeof(GroupProblem) <= (size_t)kPutBlobBytes, "blob size");
  if (S.sa != sa || S.sb != sb || S.sc != sc) {
    memset(&P, 0, sizeof(P));
    P.tile_begin = 0;
    P.sa_off = 0;  // offsets from the A spectra
    P.sb_off = (long long)((const char*)sb - (const char*)sa);
    P.out_off = (long long)((const char*)sc - (const char*)sa);
    P.M = m; P.N = s; P.K = n; P.p = p;
    P.bn = kGroupTcBN;
    auto padded = [](long long rows, long long cols) { return (rows + 127) / 128 * 128 * ((cols + 15) / 16 * 16); };
    P.trans = padded(s, m) < padded(m, s) ? 1 : 0;
    const int trows = P.trans ? s : m, tcols = P.trans ? m : s;
    P.tiles_m = (trows + kGroupTcBM - 1) / kGroupTcBM;
    P.tiles_n = (tcols + kGroupTcBN - 1) / kGroupTcBN;
    P.lda = (int)spec_ld(fmt, n);
    P.ldb = (int)spec_ld(fmt, s);
    P.tmA = S.d_blob;
    P.tmB = (const char*)S.d_blob + 128;
    char msg[256];
    if (!encode_group_map(S.h_blob, sa, m, n, P.lda, p, np, false, !P.trans, msg, sizeof(msg)) ||
        !encode_group_map(S.h_blob + 128, sb, n, s, P.ldb, p, np, true, false, msg, sizeof(msg)))
      return fail(QTP_ERR_CUDA, "products (grouped tiles): %s", msg);
    memcpy(S.h_blob + 256, &P, sizeof(P));
    S.sa = sa; S.sb = sb; S.sc = sc;
  } else {
    memcpy(&P, S.h_blob + 256, sizeof(P));
  }
  QTP_CUDA(launch_put_blob(S.h_blob, 256 + (int)sizeof(GroupProblem), S.d_blob, st), "products (grouped tiles)");
  const long long tiles = (long long)P.tiles_m * P.tiles_n * p;
  QTP_CUDA(launch_gemm_tc_grouped(reinterpret_cast<const GroupProblem*>((const char*)S.d_blob + 256), 1, tiles, np,
                                  (char*)const_cast<void*>(sa), pl->d_err, S.num_sms, st),
           "products (grouped tiles)");
  return QTP_OK;
}

// Step 2 of Alg. 5.1 for the forward product: out half 0 = C1, half 1 = C2.
//   C1_f = A1_f B1_f - A2_f conj(B2_{-f}),   C2_f = A1_f B2_f + A2_f conj(B1_{-f})
qtp_status run_products_fwd(const qtp_plan* pl, const void* sa, const void* sb, float2* sc, cudaStream_t st) {
  const int m = pl->m, n = pl->n, s = pl->s, p = pl->p;
  if (pl->small) return run_products_small(pl, sa, sb, sc, st);
  if (pl->precision == QTP_PREC_FP32) {
    GemmProblem pr;
    memset(&pr, 0, sizeof(pr));
    pr.M = m; pr.N = s; pr.K = n; pr.p = p;
    const float2* A = (const float2*)sa;
    const float2* B = (const float2*)sb;
    for (int h = 0; h < 2; ++h) {
      pr.a[h][0] = view(A, 0, p, m, n, true, 0, 0);
      pr.a[h][1] = view(A, 1, p, m, n, true, 0, 0);
    }
    // opB element (col c, k j) = B_hat[j][c]
    pr.b[0][0] = view(B, 0, p, n, s, false, 0, 0); pr.sign[0][0] = 1.f;
    pr.b[0][1] = view(B, 1, p, n, s, false, 1, 1); pr.sign[0][1] = -1.f;
    pr.b[1][0] = view(B, 1, p, n, s, false, 0, 0); pr.sign[1][0] = 1.f;
    pr.b[1][1] = view(B, 0, p, n, s, false, 1, 1); pr.sign[1][1] = 1.f;
    pr.out = sc;
    pr.out_hstride = (long long)p * m * s;
    pr.out_fstride = (long long)m * s;
    pr.out_rstride = s;
    QTP_CUDA(launch_gemm_simt(pr, st), "products (fp32)");
    return QTP_OK;
  }
  const TcProblem pr = tc_fwd(pl, sa, sb, sc);
  char msg[256] = "";
  cudaError_t e = launch_gemm_tc(pr, pl->d_err, st, msg, sizeof(msg));
  if (e != cudaSuccess) return fail(QTP_ERR_CUDA, "products (tensor cores): %s %s", cudaGetErrorString(e), msg);
  return QTP_OK;
}

// Backward products.  With G = F(dC) and the spectra of B^H and A^H
// ((B^H)_1,f = B1_f^*, (B^H)_2,f = -B2_{-f}^T), dA = dC * B^H and
// dB = A^H * dC by the same per-frequency rule:
//   dA1_f = G1_f B1_f^* + G2_f B2_f^*,        dA2_f = -G1_f B2_{-f}^T + G2_f B1_{-f}^T
//   dB1_f = A1_f^* G1_f + A2_{-f}^T conj(G2_{-f}),  dB2_f = A1_f^* G2_f - A2_{-f}^T conj(G1_{-f})
qtp_status run_products_bwd(const qtp_plan* pl, const void* sa, const void* sb, const void* sg, float2* sda,
                            float2* sdb, cudaStream_t st) {
  const int m = pl->m, n = pl->n, s = pl->s, p = pl->p;
  if (pl->precision == QTP_PREC_FP32) {
    const float2* A = (const float2*)sa;
    const float2* B = (const float2*)sb;
    const float2* G = (const float2*)sg;
    if (sda) {
      GemmProblem pr;
      memset(&pr, 0, sizeof(pr));
      pr.M = m; pr.N = n; pr.K = s; pr.p = p;
      for (int h = 0; h < 2; ++h) {
        pr.a[h][0] = view(G, 0, p, m, s, true, 0, 0);
        pr.a[h][1] = view(G, 1, p, m, s, true, 0, 0);
      }
      // opB element (col j, k c) = B_hat[j][c] -> row_is_first_index = true
      pr.b[0][0] = view(B, 0, p, n, s, true, 0, 1); pr.sign[0][0] = 1.f;
      pr.b[0][1] = view(B, 1, p, n, s, true, 0, 1); pr.sign[0][1] = 1.f;
      pr.b[1][0] = view(B, 1, p, n, s, true, 1, 0); pr.sign[1][0] = -1.f;
      pr.b[1][1] = view(B, 0, p, n, s, true, 1, 0); pr.sign[1][1] = 1.f;
      pr.out = sda;
      pr.out_hstride = (long long)p * m * n;
      pr.out_fstride = (long long)m * n;
      pr.out_rstride = n;
      QTP_CUDA(launch_gemm_simt(pr, st), "backward products dA (fp32)");
    }
    if (sdb) {
      GemmProblem pr;
      memset(&pr, 0, sizeof(pr));
      pr.M = n; pr.N = s; pr.K = m; pr.p = p;
      for (int h = 0; h < 2; ++h) {
        // opA element (row j, k i) = A_hat[i][j]
        pr.a[h][0] = view(A, 0, p, m, n, false, 0, 1);
        pr.a[h][1] = view(A, 1, p, m, n, false, 1, 0);
      }
      // opB element (col c, k i) = G_hat[i][c]
      pr.b[0][0] = view(G, 0, p, m, s, false, 0, 0); pr.sign[0][0] = 1.f;
      pr.b[0][1] = view(G, 1, p, m, s, false, 1, 1); pr.sign[0][1] = 1.f;
      pr.b[1][0] = view(G, 1, p, m, s, false, 0, 0); pr.sign[1][0] = 1.f;
      pr.b[1][1] = view(G, 0, p, m, s, false, 1, 1); pr.sign[1][1] = -1.f;
      pr.out = sdb;
      pr.out_hstride = (long long)p * n * s;
      pr.out_fstride = (long long)n * s;
      pr.out_rstride = s;
      QTP_CUDA(launch_gemm_simt(pr, st), "backward products dB (fp32)");
    }
    return QTP_OK;
  }
  char msg[256] = "";
  // dA and dB are independent: with both, the dB product runs alongside the
  // dA product (programmatic dependent launch, modes 1 and 2)
  const bool pair = sda && sdb;
  if (sda) {
    const TcProblem pr = tc_bwd_a(pl, sb, sg, sda);
    cudaError_t e = launch_gemm_tc(pr, pl->d_err, st, msg, sizeof(msg), pair ? 1 : 0);
    if (e != cudaSuccess) return fail(QTP_ERR_CUDA, "backward products dA: %s %s", cudaGetErrorString(e), msg);
  }
  if (sdb) {
    const TcProblem pr = tc_bwd_b(pl, sa, sg, sdb);
    cudaError_t e = launch_gemm_tc(pr, pl->d_err, st, msg, sizeof(msg), pair ? 2 : 0);
    if (e != cudaSuccess) return fail(QTP_ERR_CUDA, "backward products dB: %s %s", cudaGetErrorString(e), msg);
  }
  return QTP_OK;
}

// ----------------------------------------------------------------------------
// Autotuner (QTP_PLAN_AUTOTUNE): for each product kind, time the tensor-core
// tile candidates that keep the split-BF16 accuracy bound for that kind's
// reduction length K (128-wide with promoted accumulators always, with split
// accumulators for K <= kTcSplitMaxK, 256- and 128-wide single accumulators
// for K <= kTcSingleMaxK) on scratch spectra and keep the fastest.  Results are cached per (device, shape, precision) for the
// process and, when QTP_AUTOTUNE_CACHE names a file, across processes.
// ----------------------------------------------------------------------------
std::mutex g_tune_mu;
// per (device, shape, precision): tiles of the forward, dA, dB products, the
// forms of the forward and inverse tube transforms and the long form's N2
using TuneRecord = std::array<int, 6>;
std::map<std::string, TuneRecord> g_tune_cache;
bool g_tune_file_loaded = false;

std::string tune_key(const qtp_plan* pl) {
  cudaDeviceProp prop;
  std::string dev = "dev";
  if (cudaGetDeviceProperties(&prop, pl->device) == cudaSuccess) dev = prop.name;
  for (char& c : dev)
    if (c == ' ') c = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s:%d:%d:%d:%d:%d", dev.c_str(), pl->m, pl->n, pl->s, pl->p, pl->precision);
  return buf;
}

void tune_cache_load() {
  if (g_tune_file_loaded) return;
  g_tune_file_loaded = true;
  const char* path = getenv("QTP_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512], key[256];
  while (fgets(line, sizeof(line), f)) {
    TuneRecord r;
    if (sscanf(line, "%255s %d %d %d %d %d %d", key, &r[0], &r[1], &r[2], &r[3], &r[4], &r[5]) == 7)
      g_tune_cache[key] = r;
  }
  fclose(f);
}

void tune_cache_store(const std::string& key, const TuneRecord& t) {
  g_tune_cache[key] = t;
  const char* path = getenv("QTP_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d %d\n", key.c_str(), t[0], t[1], t[2], t[3], t[4], t[5]);
  fclose(f);
}

// Mean time (ms) of `reps` runs of fn on the legacy stream, after a warm-up.
template <class F>
float time_ms(F fn, cudaEvent_t e0, cudaEvent_t e1, int reps) {
  if (fn() != cudaSuccess) return 1e30f;
  cudaEventRecord(e0, 0);
  for (int i = 0; i < reps; ++i) fn();
  cudaEventRecord(e1, 0);
  if (cudaEventSynchronize(e1) != cudaSuccess) {
    cudaGetLastError();
    return 1e30f;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / reps;
}

// Tile of each product kind: the candidates that keep split-BF16 within 1e-5
// at that kind's reduction length, timed on scratch spectra.
cudaError_t tune_tiles(qtp_plan* pl, TuneRecord& best, cudaEvent_t e0, cudaEvent_t e1) {
  const int fmt = spec_format(pl->precision);
  const size_t bA = spec_bytes(fmt, pl->p, pl->m, pl->n), bB = spec_bytes(fmt, pl->p, pl->n, pl->s),
               bG = spec_bytes(fmt, pl->p, pl->m, pl->s);
  const size_t bOut = c32_bytes(pl->p, std::max(pl->m, pl->n), std::max(pl->s, pl->n));
  char* scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, bA + bB + bG + bOut);
  if (e == cudaSuccess) e = cudaMemset(scratch, 0, bA + bB + bG);
  if (e != cudaSuccess) {
    cudaFree(scratch);
    return e;
  }
  char* sa = scratch;
  char* sb = sa + bA;
  char* sg = sb + bB;
  float2* out = (float2*)(sg + bG);
  for (int kind = 0; kind < 3; ++kind) {
    TcProblem pr = kind == 0 ? tc_fwd(pl, sa, sb, out) : kind == 1 ? tc_bwd_a(pl, sb, sg, out) : tc_bwd_b(pl, sa, sg, out);
    std::vector<int> cands = {TILE_128_PROMOTE};
    if (pr.nparts == 2 || pr.K <= kTcSplitMaxK) cands.push_back(TILE_128_SPLIT);
    if (pr.nparts == 2 || pr.K <= kTcSingleMaxK) {
      cands.push_back(TILE_128);
      if (pr.N > 128) cands.push_back(TILE_256);
    }
    float best_ms = 1e30f;
    for (int c : cands) {
      pr.tile = c;
      char msg[256];
      const float ms = time_ms([&] { return launch_gemm_tc(pr, pl->d_err, 0, msg, sizeof(msg)); }, e0, e1, 3);
      if (ms < best_ms) {
        best_ms = ms;
        best[kind] = c;
      }
    }
  }
  e = cudaDeviceSynchronize();
  cudaFree(scratch);
  return e;
}

// Form of the forward and of the inverse tube transform (one kernel, runtime
// two-pass, compile-time long two-pass with each N2 p splits into), timed on
// scratch tensors of the plan's shapes: the forward transforms A and B, the
// inverse C.  Both directions share one N2 (one second twiddle table).
cudaError_t tune_forms(qtp_plan* pl, TuneRecord& best, cudaEvent_t e0, cudaEvent_t e1) {
  struct Cand {
    int form, n2;
  };
  std::vector<Cand> cands = {{FFT_ONE, 0}};
  if (fft_split_dims(pl->p, nullptr, nullptr)) cands.push_back({FFT_SPLIT, 0});
  int n2s[4];
  const int nl = fft_long_splits(pl->p, n2s);
  for (int i = 0; i < nl; ++i) cands.push_back({FFT_LONG, n2s[i]});
  best[3] = pl->fft_split_fwd;
  best[4] = pl->fft_split_inv;
  best[5] = pl->long_n2;
  if (cands.size() == 1) return cudaSuccess;
  const int fmt = spec_format(pl->precision);
  const size_t iA = c32_bytes(pl->p, pl->m, pl->n), iB = c32_bytes(pl->p, pl->n, pl->s),
               iC = c32_bytes(pl->p, pl->m, pl->s);
  const size_t sA = spec_bytes(fmt, pl->p, pl->m, pl->n), sB = spec_bytes(fmt, pl->p, pl->n, pl->s);
  const size_t zs = std::max(align256(fft_split_scratch_bytes(pl->p, pl->m, pl->n)) +
                                 align256(fft_split_scratch_bytes(pl->p, pl->n, pl->s)),
                             align256(fft_split_scratch_bytes(pl->p, pl->m, pl->s)));
  char* scratch = nullptr;
  const size_t total = iA + iB + 2 * iC + sA + sB + zs;
  cudaError_t e = cudaMalloc(&scratch, total);
  if (e == cudaSuccess) e = cudaMemset(scratch, 0, total);
  if (e != cudaSuccess) {
    cudaFree(scratch);
    return e;
  }
  char* A = scratch;
  char* B = A + iA;
  char* Chat = B + iB;
  char* C = Chat + iC;
  char* spA = C + iC;
  char* spB = spA + sA;
  char* z = spB + sB;
  FftFwdJob jobs[2];
  jobs[0].in = (const float2*)A;
  jobs[0].out = spA;
  jobs[0].rows = pl->m; jobs[0].cols = pl->n; jobs[0].ld = (int)spec_ld(fmt, pl->n);
  jobs[0].nblocks = nblocks_fwd(pl->m, pl->n, pl->p, fmt);
  jobs[1].in = (const float2*)B;
  jobs[1].out = spB;
  jobs[1].rows = pl->n; jobs[1].cols = pl->s; jobs[1].ld = (int)spec_ld(fmt, pl->s);
  jobs[1].nblocks = nblocks_fwd(pl->n, pl->s, pl->p, fmt);
  FftInvJob ij;
  ij.in = (const float2*)Chat;
  ij.out = (float2*)C;
  ij.rows = pl->m; ij.cols = pl->s;
  ij.nblocks = nblocks_for(pl->m, pl->s, pl->p, true);
  const int fwd0 = pl->fft_split_fwd, inv0 = pl->fft_split_inv, n20 = pl->long_n2;
  std::vector<float> tf(cands.size()), ti(cands.size());
  for (size_t c = 0; c < cands.size() && e == cudaSuccess; ++c) {
    pl->fft_split_fwd = pl->fft_split_inv = cands[c].form;
    if (cands[c].form == FFT_LONG) {
      pl->long_n2 = cands[c].n2;
      e = plan_twiddles(pl, 0);  // the N2 table of this split
    }
    tf[c] = time_ms([&] { return plan_fft_fwd(pl, jobs, 2, fmt, z, 0); }, e0, e1, 3);
    ti[c] = time_ms([&] { return plan_fft_inv(pl, &ij, 1, z, 0); }, e0, e1, 3);
  }
  // the fastest form per direction; when both are long forms, one N2 for both
  size_t bf = 0, bi = 0;
  for (size_t c = 1; c < cands.size(); ++c) {
    if (tf[c] < tf[bf]) bf = c;
    if (ti[c] < ti[bi]) bi = c;
  }
  int n2 = 0;
  if (cands[bf].form == FFT_LONG && cands[bi].form == FFT_LONG && cands[bf].n2 != cands[bi].n2) {
    size_t bb = bf;
    for (size_t c = 0; c < cands.size(); ++c)
      if (cands[c].form == FFT_LONG && tf[c] + ti[c] < tf[bb] + ti[bb]) bb = c;
    bf = bi = bb;
  }
  if (cands[bf].form == FFT_LONG) n2 = cands[bf].n2;
  else if (cands[bi].form == FFT_LONG) n2 = cands[bi].n2;
  best[3] = cands[bf].form;
  best[4] = cands[bi].form;
  best[5] = n2;
  pl->fft_split_fwd = fwd0;
  pl->fft_split_inv = inv0;
  pl->long_n2 = n20;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(scratch);
  return e;
}

qtp_status autotune(qtp_plan* pl) {
  const bool tiles = pl->precision != QTP_PREC_FP32;  // one FP32 products kernel: no tile to choose
  const bool forms = pl->p > 128;                     // one transform form below
  if (!tiles && !forms) return QTP_OK;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_cache_load();
  const std::string key = tune_key(pl);
  auto hit = g_tune_cache.find(key);
  if (hit != g_tune_cache.end()) {
    for (int k = 0; k < 3; ++k) pl->tile[k] = hit->second[k];
    pl->fft_split_fwd = hit->second[3];
    pl->fft_split_inv = hit->second[4];
    pl->long_n2 = hit->second[5];
    cudaError_t e = plan_twiddles(pl, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "autotune twiddles");
    return QTP_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  TuneRecord best = {TILE_AUTO, TILE_AUTO, TILE_AUTO, pl->fft_split_fwd, pl->fft_split_inv, pl->long_n2};
  if (e == cudaSuccess && tiles) e = tune_tiles(pl, best, e0, e1);
  if (e == cudaSuccess && forms) e = tune_forms(pl, best, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  int v = 0;
  cudaMemcpy(&v, pl->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (v != 0) {
    cudaMemset(pl->d_err, 0, sizeof(int));
    return fail(QTP_ERR_TIMEOUT, "autotune: a device-side wait gave up (code %d)", v);
  }
  for (int k = 0; k < 3; ++k) pl->tile[k] = best[k];
  pl->fft_split_fwd = best[3];
  pl->fft_split_inv = best[4];
  pl->long_n2 = best[5];
  e = plan_twiddles(pl, 0);  // the N2 table of the chosen split
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "autotune twiddles");
  tune_cache_store(key, best);
  return QTP_OK;
}

void trace(const qtp_plan* pl, int i, cudaStream_t st) {
  if (pl->tracing) cudaEventRecord(pl->ev[i], st);
}

qtp_status forward_impl(const qtp_plan* pl, const float* A, const float* B, float* C, char* ws,
                        cudaStream_t st, bool allow_fused = true) {
  if (allow_fused && fused_small_eligible(pl->m, pl->n, pl->s, pl->p)) {
    // all three steps in one CTA (qtp_fused_small.cu); traced as the products stage
    trace(pl, 0, st);
    trace(pl, 1, st);
    QTP_CUDA(launch_fused_small((const float2*)A, (const float2*)B, (float2*)C, pl->m, pl->n, pl->s, pl->p,
                                pl->d_tw, st),
             "fused small product");
    trace(pl, 2, st);
    trace(pl, 3, st);
    return QTP_OK;
  }
  const int fmt = spec_format(pl->precision);
  const FwdLayout L = fwd_layout(pl);
  FftFwdJob jobs[2];
  jobs[0].in = (const float2*)A;
  jobs[0].out = ws + L.sa;
  jobs[0].rows = pl->m; jobs[0].cols = pl->n; jobs[0].ld = (int)spec_ld(fmt, pl->n);
  jobs[0].nblocks = nblocks_fwd(pl->m, pl->n, pl->p, fmt);
  jobs[1].in = (const float2*)B;
  jobs[1].out = ws + L.sb;
  jobs[1].rows = pl->n; jobs[1].cols = pl->s; jobs[1].ld = (int)spec_ld(fmt, pl->s);
  jobs[1].nblocks = nblocks_fwd(pl->n, pl->s, pl->p, fmt);
  trace(pl, 0, st);
  QTP_CUDA(plan_fft_fwd(pl, jobs, 2, fmt, ws + L.scr, st), "forward tube FFT");
  trace(pl, 1, st);
  qtp_status r = run_products_fwd(pl, ws + L.sa, ws + L.sb, (float2*)(ws + L.sc), st);
  if (r != QTP_OK) return r;
  trace(pl, 2, st);
  FftInvJob ij;
  ij.in = (const float2*)(ws + L.sc);
  ij.out = (float2*)C;
  ij.rows = pl->m; ij.cols = pl->s;
  ij.nblocks = nblocks_for(pl->m, pl->s, pl->p, true);
  QTP_CUDA(plan_fft_inv(pl, &ij, 1, ws + L.scr, st), "inverse tube FFT");
  trace(pl, 3, st);
  return QTP_OK;
}

}  // namespace

namespace qtp {
qtp_status set_error(qtp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}
void clear_error() { g_err[0] = 0; }
int spec_format_of(int precision) { return spec_format(precision); }
long long spec_ld_of(int fmt, long long cols) { return spec_ld(fmt, cols); }
size_t spec_bytes_of(int fmt, long long p, long long rows, long long cols) { return spec_bytes(fmt, p, rows, cols); }
size_t c32_bytes_of(long long p, long long rows, long long cols) { return c32_bytes(p, rows, cols); }
}  // namespace qtp

extern "C" {

const char* qtp_last_error(void) { return g_err; }

int qtp_version(void) { return 100; }

qtp_status qtp_plan_create(qtp_plan** out, int m, int n, int s, int p, int precision, unsigned flags) {
  g_err[0] = 0;
  if (!out) return fail(QTP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || s < 1 || p < 1) return fail(QTP_ERR_INVALID_ARG, "dimensions must be >= 1 (m=%d n=%d s=%d p=%d)", m, n, s, p);
  if (m > (1 << 20) || n > (1 << 20) || s > (1 << 20))
    return fail(QTP_ERR_INVALID_ARG, "m, n, s must be <= 2^20");
  if (p > QTP_MAX_P) return fail(QTP_ERR_UNSUPPORTED, "p=%d exceeds the supported maximum %d", p, QTP_MAX_P);
  const long long lim = 1LL << 31;
  if ((long long)m * n * p >= lim || (long long)n * s * p >= lim || (long long)m * s * p >= lim)
    return fail(QTP_ERR_INVALID_ARG, "a tensor plane exceeds 2^31 complex entries");
  if (flags & ~QTP_PLAN_AUTOTUNE) return fail(QTP_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  if (precision != QTP_PREC_FP32 && precision != QTP_PREC_BF16X3 && precision != QTP_PREC_BF16)
    return fail(QTP_ERR_INVALID_ARG, "unknown precision %d", precision);
  if (precision != QTP_PREC_FP32 && !tc_supported())
    return fail(QTP_ERR_UNSUPPORTED, "BF16 tensor-core products need an sm_103 device (tcgen05)");
  qtp_plan* pl = new qtp_plan();
  pl->m = m; pl->n = n; pl->s = s; pl->p = p;
  pl->precision = precision;
  pl->rp = make_radix_plan(p);
  pl->fft_split_fwd = fft_form(p, false);
  pl->fft_split_inv = fft_form(p, true);
  if (const char* env = getenv("QTP_FFT_LONG_N2")) {  // the long form's N2, if p splits with it
    int n2s[4];
    const int k = fft_long_splits(p, n2s), want = atoi(env);
    for (int i = 0; i < k; ++i)
      if (n2s[i] == want) pl->long_n2 = want;
  }
  pl->d_tw = nullptr;
  pl->d_err = nullptr;
  pl->tracing = 0;
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_tw, sizeof(float2) * plan_twiddle_count(pl));
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(pl->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = plan_twiddles(pl, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    if (pl->d_tw) cudaFree(pl->d_tw);
    if (pl->d_err) cudaFree(pl->d_err);
    delete pl;
    return cuda_fail(e, "plan creation");
  }
  if (small_tiles_route(pl)) {
    pl->small = new SmallTiles();
    e = cudaMalloc(&pl->small->d_blob, kPutBlobBytes);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pl->small->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
    if (e != cudaSuccess) {
      cudaFree(pl->small->d_blob);
      delete pl->small;
      cudaFree(pl->d_tw);
      cudaFree(pl->d_err);
      delete pl;
      return cuda_fail(e, "plan creation");
    }
  }
  pl->flags = flags;
  if (flags & QTP_PLAN_AUTOTUNE) {
    qtp_status r = autotune(pl);
    if (r != QTP_OK) {
      if (pl->small) {
        cudaFree(pl->small->d_blob);
        delete pl->small;
      }
      cudaFree(pl->d_tw);
      cudaFree(pl->d_err);
      delete pl;
      return r;
    }
  }
  *out = pl;
  return QTP_OK;
}

qtp_status qtp_plan_get_tiles(const qtp_plan* pl, int* tiles3) {
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if (!tiles3) return fail(QTP_ERR_INVALID_ARG, "tiles3 is NULL");
  for (int k = 0; k < 3; ++k) tiles3[k] = pl->tile[k];
  return QTP_OK;
}

qtp_status qtp_plan_launch_count(const qtp_plan* pl, int* forward, int* backward) {
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if (!forward || !backward) return fail(QTP_ERR_INVALID_ARG, "output pointer is NULL");
  // each transform step takes two launches in its two-pass form
  const int sf = pl->fft_split_fwd != FFT_ONE, si = pl->fft_split_inv != FFT_ONE;
  *forward = fused_small_eligible(pl->m, pl->n, pl->s, pl->p) ? 1 : 3 + sf + si + (pl->small ? 1 : 0);
  *backward = 5 + 2 * sf + si;
  return QTP_OK;
}

// Copy streams and slot events of qtp_forward_host_many (one set per plan).
struct HostPipe {
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t entry = nullptr;
  cudaEvent_t in_ready[2] = {nullptr, nullptr};  // slot's A, B on the device
  cudaEvent_t computed[2] = {nullptr, nullptr};  // slot's C computed (its A, B consumed)
  cudaEvent_t out_done[2] = {nullptr, nullptr};  // slot's C copied out
};

static void destroy_pipe(HostPipe* P) {
  if (!P) return;
  if (P->h2d) cudaStreamDestroy(P->h2d);
  if (P->d2h) cudaStreamDestroy(P->d2h);
  cudaEvent_t* evs[] = {&P->entry, &P->in_ready[0], &P->in_ready[1], &P->computed[0], &P->computed[1],
                        &P->out_done[0], &P->out_done[1]};
  for (cudaEvent_t* e : evs)
    if (*e) cudaEventDestroy(*e);
  delete P;
}

qtp_status qtp_plan_destroy(qtp_plan* pl) {
  if (!pl) return QTP_OK;
  qtp_plan_set_tracing(pl, 0);
  destroy_pipe(pl->pipe);
  pl->pipe = nullptr;
  if (pl->small) {
    cudaFree(pl->small->d_blob);
    delete pl->small;
  }
  cudaFree(pl->d_tw);
  cudaFree(pl->d_err);
  delete pl;
  return QTP_OK;
}

qtp_status qtp_workspace_size(const qtp_plan* pl, size_t* bytes) {
  if (check_plan(pl) != QTP_OK) return QTP_ERR_INVALID_ARG;
  if (!bytes) return fail(QTP_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = fwd_layout(pl).total;
  return QTP_OK;
}

qtp_status qtp_backward_workspace_size(const qtp_plan* pl, size_t* bytes) {
  if (check_plan(pl) != QTP_OK) return QTP_ERR_INVALID_ARG;
  if (!bytes) return fail(QTP_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = bwd_layout(pl).total;
  return QTP_OK;
}

qtp_status qtp_forward(const qtp_plan* pl, const float* A, const float* B, float* C, void* workspace,
                       size_t workspace_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if ((r = check_dev_ptr(A, "A")) != QTP_OK) return r;
  if ((r = check_dev_ptr(B, "B")) != QTP_OK) return r;
  if ((r = check_dev_ptr(C, "C")) != QTP_OK) return r;
  if ((r = check_dev_ptr(workspace, "workspace")) != QTP_OK) return r;
  const size_t need = fwd_layout(pl).total;
  if (workspace_bytes < need)
    return fail(QTP_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, need);
  return forward_impl(pl, A, B, C, (char*)workspace, as_stream(stream));
}

qtp_status qtp_host_buffer_size(const qtp_plan* pl, size_t* bytes) {
  if (check_plan(pl) != QTP_OK) return QTP_ERR_INVALID_ARG;
  if (!bytes) return fail(QTP_ERR_INVALID_ARG, "bytes is NULL");
  // device copies of A, B, C (each exactly one tensor, 256-byte aligned) + workspace
  *bytes = c32_bytes(pl->p, pl->m, pl->n) + c32_bytes(pl->p, pl->n, pl->s) + c32_bytes(pl->p, pl->m, pl->s) +
           fwd_layout(pl).total;
  return QTP_OK;
}

qtp_status qtp_forward_host(const qtp_plan* pl, const float* A_host, const float* B_host, float* C_host,
                            void* dev_buffer, size_t dev_buffer_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if ((r = check_host_ptr(A_host, "A_host")) != QTP_OK) return r;
  if ((r = check_host_ptr(B_host, "B_host")) != QTP_OK) return r;
  if ((r = check_host_ptr(C_host, "C_host")) != QTP_OK) return r;
  if ((r = check_dev_ptr(dev_buffer, "dev_buffer")) != QTP_OK) return r;
  size_t need = 0;
  qtp_host_buffer_size(pl, &need);
  if (dev_buffer_bytes < need)
    return fail(QTP_ERR_WORKSPACE, "dev_buffer has %zu bytes, %zu needed", dev_buffer_bytes, need);
  const size_t bA = (size_t)2 * pl->m * pl->n * pl->p * sizeof(float2);
  const size_t bB = (size_t)2 * pl->n * pl->s * pl->p * sizeof(float2);
  const size_t bC = (size_t)2 * pl->m * pl->s * pl->p * sizeof(float2);
  char* base = (char*)dev_buffer;
  float* dA = (float*)base;
  float* dB = (float*)(base + c32_bytes(pl->p, pl->m, pl->n));
  float* dC = (float*)(base + c32_bytes(pl->p, pl->m, pl->n) + c32_bytes(pl->p, pl->n, pl->s));
  char* ws = base + c32_bytes(pl->p, pl->m, pl->n) + c32_bytes(pl->p, pl->n, pl->s) + c32_bytes(pl->p, pl->m, pl->s);
  cudaStream_t st = as_stream(stream);
  QTP_CUDA(cudaMemcpyAsync(dA, A_host, bA, cudaMemcpyHostToDevice, st), "copy A to device");
  QTP_CUDA(cudaMemcpyAsync(dB, B_host, bB, cudaMemcpyHostToDevice, st), "copy B to device");
  r = forward_impl(pl, dA, dB, dC, ws, st);
  if (r != QTP_OK) return r;
  QTP_CUDA(cudaMemcpyAsync(C_host, dC, bC, cudaMemcpyDeviceToHost, st), "copy C to host");
  return QTP_OK;
}

// Device slot of qtp_forward_host_many: A, B, C of one product.
static size_t host_slot_bytes(const qtp_plan* pl) {
  return c32_bytes(pl->p, pl->m, pl->n) + c32_bytes(pl->p, pl->n, pl->s) + c32_bytes(pl->p, pl->m, pl->s);
}

qtp_status qtp_host_many_buffer_size(const qtp_plan* pl, size_t* bytes) {
  if (check_plan(pl) != QTP_OK) return QTP_ERR_INVALID_ARG;
  if (!bytes) return fail(QTP_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 2 * host_slot_bytes(pl) + fwd_layout(pl).total;
  return QTP_OK;
}

static qtp_status ensure_pipe(const qtp_plan* pl) {
  if (pl->pipe) return QTP_OK;
  HostPipe* P = new HostPipe();
  cudaError_t e = cudaStreamCreateWithFlags(&P->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->d2h, cudaStreamNonBlocking);
  cudaEvent_t* evs[] = {&P->entry, &P->in_ready[0], &P->in_ready[1], &P->computed[0], &P->computed[1],
                        &P->out_done[0], &P->out_done[1]};
  for (cudaEvent_t* ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    destroy_pipe(P);
    return fail(QTP_ERR_CUDA, "host pipeline streams: %s", cudaGetErrorString(e));
  }
  const_cast<qtp_plan*>(pl)->pipe = P;  // plan-owned, created on first use
  return QTP_OK;
}

qtp_status qtp_forward_host_many(const qtp_plan* pl, int count, const float* const* A_host,
                                 const float* const* B_host, float* const* C_host, void* dev_buffer,
                                 size_t dev_buffer_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if (count < 0) return fail(QTP_ERR_INVALID_ARG, "count %d is negative", count);
  if (count == 0) return QTP_OK;
  if (!A_host || !B_host || !C_host) return fail(QTP_ERR_INVALID_ARG, "a host pointer array is NULL");
  for (int i = 0; i < count; ++i) {
    if ((r = check_host_ptr(A_host[i], "A_host[i]")) != QTP_OK) return r;
    if ((r = check_host_ptr(B_host[i], "B_host[i]")) != QTP_OK) return r;
    if ((r = check_host_ptr(C_host[i], "C_host[i]")) != QTP_OK) return r;
  }
  if ((r = check_dev_ptr(dev_buffer, "dev_buffer")) != QTP_OK) return r;
  size_t need = 0;
  qtp_host_many_buffer_size(pl, &need);
  if (dev_buffer_bytes < need)
    return fail(QTP_ERR_WORKSPACE, "dev_buffer has %zu bytes, %zu needed", dev_buffer_bytes, need);
  if ((r = ensure_pipe(pl)) != QTP_OK) return r;
  HostPipe& P = *pl->pipe;
  const size_t bA = (size_t)2 * pl->m * pl->n * pl->p * sizeof(float2);
  const size_t bB = (size_t)2 * pl->n * pl->s * pl->p * sizeof(float2);
  const size_t bC = (size_t)2 * pl->m * pl->s * pl->p * sizeof(float2);
  char* base = (char*)dev_buffer;
  const size_t slot = host_slot_bytes(pl);
  char* ws = base + 2 * slot;
  cudaStream_t st = as_stream(stream);
  // Everything enqueued on stream before this call precedes the first copy.
  QTP_CUDA(cudaEventRecord(P.entry, st), "host pipeline entry");
  QTP_CUDA(cudaStreamWaitEvent(P.h2d, P.entry, 0), "host pipeline entry");
  QTP_CUDA(cudaStreamWaitEvent(P.d2h, P.entry, 0), "host pipeline entry");
  for (int i = 0; i < count; ++i) {
    const int sl = i & 1;
    float* dA = (float*)(base + sl * slot);
    float* dB = (float*)(base + sl * slot + c32_bytes(pl->p, pl->m, pl->n));
    float* dC = (float*)(base + sl * slot + c32_bytes(pl->p, pl->m, pl->n) + c32_bytes(pl->p, pl->n, pl->s));
    // in: the slot's previous product (i - 2) has consumed its A and B
    if (i >= 2) QTP_CUDA(cudaStreamWaitEvent(P.h2d, P.computed[sl], 0), "host pipeline slot reuse");
    QTP_CUDA(cudaMemcpyAsync(dA, A_host[i], bA, cudaMemcpyHostToDevice, P.h2d), "copy A to device");
    QTP_CUDA(cudaMemcpyAsync(dB, B_host[i], bB, cudaMemcpyHostToDevice, P.h2d), "copy B to device");
    QTP_CUDA(cudaEventRecord(P.in_ready[sl], P.h2d), "host pipeline copy-in");
    // compute on stream: the slot's inputs are in and its previous C is out
    QTP_CUDA(cudaStreamWaitEvent(st, P.in_ready[sl], 0), "host pipeline copy-in");
    if (i >= 2) QTP_CUDA(cudaStreamWaitEvent(st, P.out_done[sl], 0), "host pipeline slot reuse");
    r = forward_impl(pl, dA, dB, dC, ws, st);
    if (r != QTP_OK) {
      // copies already queued still use the caller's buffers: make stream
      // cover them, so that synchronising it is enough before freeing those
      if (cudaEventRecord(P.in_ready[sl], P.h2d) == cudaSuccess) cudaStreamWaitEvent(st, P.in_ready[sl], 0);
      if (cudaEventRecord(P.out_done[sl], P.d2h) == cudaSuccess) cudaStreamWaitEvent(st, P.out_done[sl], 0);
      return r;
    }
    QTP_CUDA(cudaEventRecord(P.computed[sl], st), "host pipeline compute");
    // out
    QTP_CUDA(cudaStreamWaitEvent(P.d2h, P.computed[sl], 0), "host pipeline compute");
    QTP_CUDA(cudaMemcpyAsync(C_host[i], dC, bC, cudaMemcpyDeviceToHost, P.d2h), "copy C to host");
    QTP_CUDA(cudaEventRecord(P.out_done[sl], P.d2h), "host pipeline copy-out");
  }
  // The last copy-out follows every other copy of the call: join it to stream.
  QTP_CUDA(cudaStreamWaitEvent(st, P.out_done[(count - 1) & 1], 0), "host pipeline exit");
  return QTP_OK;
}

// ---------------------------------------------------------------------------
// T-SVD (qtp_tsvd.cu)
// ---------------------------------------------------------------------------

struct TsvdLayout {
  size_t tw, h, uh, vh, sh, scratch, status, total;
};

static TsvdLayout tsvd_layout(int m, int n, int p) {
  const int k = m < n ? m : n;
  TsvdLayout L;
  L.tw = 0;
  L.h = align256((size_t)p * sizeof(float2));
  L.uh = L.h + c32_bytes(p, m, n);
  L.vh = L.uh + c32_bytes(p, m, k);
  L.sh = L.vh + c32_bytes(p, n, k);
  L.scratch = L.sh + c32_bytes(p, k, k);
  L.status = L.scratch + align256(tsvd_scratch_bytes(m, n, p));
  L.total = L.status + 256;
  return L;
}

static qtp_status check_tsvd_shape(int m, int n, int p) {
  if (m < 1 || n < 1 || p < 1) return fail(QTP_ERR_INVALID_ARG, "T-SVD shape %d x %d x %d", m, n, p);
  if (p > QTP_MAX_P) return fail(QTP_ERR_UNSUPPORTED, "p=%d exceeds the supported maximum %d", p, QTP_MAX_P);
  if ((m < n ? m : n) > QTP_TSVD_MAX_K)
    return fail(QTP_ERR_UNSUPPORTED, "min(m, n) = %d exceeds the T-SVD maximum %d", m < n ? m : n, QTP_TSVD_MAX_K);
  if ((m > n ? m : n) > QTP_TSVD_MAX_MN)
    return fail(QTP_ERR_UNSUPPORTED, "max(m, n) = %d exceeds the T-SVD maximum %d", m > n ? m : n, QTP_TSVD_MAX_MN);
  return QTP_OK;
}

qtp_status qtp_tsvd_workspace_size(int m, int n, int p, size_t* bytes) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_tsvd_shape(m, n, p)) != QTP_OK) return r;
  if (!bytes) return fail(QTP_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = tsvd_layout(m, n, p).total;
  return QTP_OK;
}

qtp_status qtp_tsvd(int m, int n, int p, const float* A, float* U, float* S, float* V, float* sigma, void* workspace,
                    size_t workspace_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_tsvd_shape(m, n, p)) != QTP_OK) return r;
  if ((r = check_dev_ptr(A, "A")) != QTP_OK) return r;
  if ((r = check_dev_ptr(U, "U")) != QTP_OK) return r;
  if ((r = check_dev_ptr(S, "S")) != QTP_OK) return r;
  if ((r = check_dev_ptr(V, "V")) != QTP_OK) return r;
  if ((r = check_dev_ptr(sigma, "sigma")) != QTP_OK) return r;
  if ((r = check_dev_ptr(workspace, "workspace")) != QTP_OK) return r;
  const TsvdLayout L = tsvd_layout(m, n, p);
  if (workspace_bytes < L.total)
    return fail(QTP_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
  const int k = m < n ? m : n;
  cudaStream_t st = as_stream(stream);
  char* ws = (char*)workspace;
  float2* tw = (float2*)(ws + L.tw);
  float2* H = (float2*)(ws + L.h);
  float2* Uh = (float2*)(ws + L.uh);
  float2* Vh = (float2*)(ws + L.vh);
  float2* Sh = (float2*)(ws + L.sh);
  float2* scratch = tsvd_scratch_bytes(m, n, p) ? (float2*)(ws + L.scratch) : nullptr;
  const RadixPlan rp = make_radix_plan(p);
  QTP_CUDA(launch_twiddles(tw, p, st), "T-SVD twiddles");
  // spectra of A (plain transforms of both Cayley-Dickson halves)
  FftFwdJob fj;
  fj.in = (const float2*)A;
  fj.out = H;
  fj.rows = m;
  fj.cols = n;
  fj.ld = n;
  fj.nblocks = nblocks_fwd(m, n, p, FMT_C32);
  QTP_CUDA(launch_fft_fwd(&fj, 1, FMT_C32, rp, tw, st), "T-SVD forward FFT");
  QTP_CUDA(cudaMemsetAsync(Sh, 0, c32_bytes(p, k, k), st), "T-SVD clear S");
  int* status = (int*)(ws + L.status);
  QTP_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st), "T-SVD clear status");
  QTP_CUDA(launch_tsvd_pairs(H, m, n, p, Uh, Vh, Sh, sigma, scratch, status, st), "T-SVD per-frequency SVDs");
  FftInvJob ij[2];
  ij[0].in = Uh;
  ij[0].out = (float2*)U;
  ij[0].rows = m;
  ij[0].cols = k;
  ij[0].nblocks = nblocks_for(m, k, p, true);
  ij[1].in = Vh;
  ij[1].out = (float2*)V;
  ij[1].rows = n;
  ij[1].cols = k;
  ij[1].nblocks = nblocks_for(n, k, p, true);
  QTP_CUDA(launch_fft_inv(ij, 2, rp, tw, st), "T-SVD inverse FFT of U, V");
  FftInvJob sj;
  sj.in = Sh;
  sj.out = (float2*)S;
  sj.rows = k;
  sj.cols = k;
  sj.nblocks = nblocks_for(k, k, p, true);
  QTP_CUDA(launch_fft_inv(&sj, 1, rp, tw, st), "T-SVD inverse FFT of S");
  return QTP_OK;
}

qtp_status qtp_tsvd_sync(int m, int n, int p, const void* workspace, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_tsvd_shape(m, n, p)) != QTP_OK) return r;
  if ((r = check_dev_ptr(workspace, "workspace")) != QTP_OK) return r;
  QTP_CUDA(cudaStreamSynchronize(as_stream(stream)), "stream synchronize");
  int v = 0;
  QTP_CUDA(cudaMemcpy(&v, (const char*)workspace + tsvd_layout(m, n, p).status, sizeof(int), cudaMemcpyDeviceToHost),
           "read T-SVD status");
  if (v != 0) return fail(QTP_ERR_NOT_CONVERGED, "T-SVD: Jacobi sweeps reached their limit still rotating");
  return QTP_OK;
}

// Backward steps (validated arguments).  saved: the workspace of a
// qtp_forward_saving call whose spectra of A and B are reused (then A and B
// are not read); null: A and B are transformed here.
static qtp_status bwd_impl(const qtp_plan* pl, const float* dC, const float* A, const float* B, const char* saved,
                           float* dA, float* dB, char* ws, cudaStream_t st) {
  qtp_status r;
  const BwdLayout L = bwd_layout(pl);
  const int fmt = spec_format(pl->precision);
  const char* sa = saved ? saved + fwd_layout(pl).sa : ws + L.sa;
  const char* sb = saved ? saved + fwd_layout(pl).sb : ws + L.sb;
  // Step 1 on dC (and A, B unless their spectra are saved).
  trace(pl, 0, st);
  if (!saved) {
  FftFwdJob jobs[2];
  jobs[0].in = (const float2*)A;
  jobs[0].out = ws + L.sa;
  jobs[0].rows = pl->m; jobs[0].cols = pl->n; jobs[0].ld = (int)spec_ld(fmt, pl->n);
  jobs[0].nblocks = nblocks_fwd(pl->m, pl->n, pl->p, fmt);
  jobs[1].in = (const float2*)B;
  jobs[1].out = ws + L.sb;
  jobs[1].rows = pl->n; jobs[1].cols = pl->s; jobs[1].ld = (int)spec_ld(fmt, pl->s);
  jobs[1].nblocks = nblocks_fwd(pl->n, pl->s, pl->p, fmt);
  QTP_CUDA(plan_fft_fwd(pl, jobs, 2, fmt, ws + L.scr, st), "backward FFT of A, B");
  }
  FftFwdJob gj;
  gj.in = (const float2*)dC;
  gj.out = ws + L.sg;
  gj.rows = pl->m; gj.cols = pl->s; gj.ld = (int)spec_ld(fmt, pl->s);
  gj.nblocks = nblocks_fwd(pl->m, pl->s, pl->p, fmt);
  QTP_CUDA(plan_fft_fwd(pl, &gj, 1, fmt, ws + L.scr, st), "backward FFT of dC");
  trace(pl, 1, st);
  // Step 2.
  r = run_products_bwd(pl, sa, sb, ws + L.sg, dA ? (float2*)(ws + L.sda) : nullptr,
                       dB ? (float2*)(ws + L.sdb) : nullptr, st);
  if (r != QTP_OK) return r;
  trace(pl, 2, st);
  // Step 3 on dA and dB.
  FftInvJob ij[2];
  int nj = 0;
  if (dA) {
    ij[nj].in = (const float2*)(ws + L.sda);
    ij[nj].out = (float2*)dA;
    ij[nj].rows = pl->m; ij[nj].cols = pl->n;
    ij[nj].nblocks = nblocks_for(pl->m, pl->n, pl->p, true);
    ++nj;
  }
  if (dB) {
    ij[nj].in = (const float2*)(ws + L.sdb);
    ij[nj].out = (float2*)dB;
    ij[nj].rows = pl->n; ij[nj].cols = pl->s;
    ij[nj].nblocks = nblocks_for(pl->n, pl->s, pl->p, true);
    ++nj;
  }
  QTP_CUDA(plan_fft_inv(pl, ij, nj, ws + L.scr, st), "backward inverse FFT");
  trace(pl, 3, st);
  return QTP_OK;
}

qtp_status qtp_backward(const qtp_plan* pl, const float* dC, const float* A, const float* B, float* dA,
                        float* dB, void* workspace, size_t workspace_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if ((r = check_dev_ptr(dC, "dC")) != QTP_OK) return r;
  if ((r = check_dev_ptr(A, "A")) != QTP_OK) return r;
  if ((r = check_dev_ptr(B, "B")) != QTP_OK) return r;
  if ((r = check_dev_ptr(dA, "dA", true)) != QTP_OK) return r;
  if ((r = check_dev_ptr(dB, "dB", true)) != QTP_OK) return r;
  if ((r = check_dev_ptr(workspace, "workspace")) != QTP_OK) return r;
  if (!dA && !dB) return QTP_OK;
  const BwdLayout L = bwd_layout(pl);
  if (workspace_bytes < L.total)
    return fail(QTP_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
  return bwd_impl(pl, dC, A, B, nullptr, dA, dB, (char*)workspace, as_stream(stream));
}

qtp_status qtp_forward_saving(const qtp_plan* pl, const float* A, const float* B, float* C, void* saved,
                              size_t saved_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if ((r = check_dev_ptr(A, "A")) != QTP_OK) return r;
  if ((r = check_dev_ptr(B, "B")) != QTP_OK) return r;
  if ((r = check_dev_ptr(C, "C")) != QTP_OK) return r;
  if ((r = check_dev_ptr(saved, "saved")) != QTP_OK) return r;
  const size_t need = fwd_layout(pl).total;
  if (saved_bytes < need) return fail(QTP_ERR_WORKSPACE, "saved has %zu bytes, %zu needed", saved_bytes, need);
  return forward_impl(pl, A, B, C, (char*)saved, as_stream(stream), false);
}

qtp_status qtp_backward_saved(const qtp_plan* pl, const float* dC, const void* saved, size_t saved_bytes, float* dA,
                              float* dB, void* workspace, size_t workspace_bytes, void* stream) {
  g_err[0] = 0;
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if ((r = check_dev_ptr(dC, "dC")) != QTP_OK) return r;
  if ((r = check_dev_ptr(saved, "saved")) != QTP_OK) return r;
  if ((r = check_dev_ptr(dA, "dA", true)) != QTP_OK) return r;
  if ((r = check_dev_ptr(dB, "dB", true)) != QTP_OK) return r;
  if ((r = check_dev_ptr(workspace, "workspace")) != QTP_OK) return r;
  if (saved_bytes < fwd_layout(pl).total)
    return fail(QTP_ERR_WORKSPACE, "saved has %zu bytes, %zu needed", saved_bytes, fwd_layout(pl).total);
  if (!dA && !dB) return QTP_OK;
  const BwdLayout L = bwd_layout(pl);
  if (workspace_bytes < L.total)
    return fail(QTP_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
  return bwd_impl(pl, dC, nullptr, nullptr, (const char*)saved, dA, dB, (char*)workspace, as_stream(stream));
}

qtp_status qtp_plan_set_tracing(qtp_plan* pl, int enable) {
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if (enable && !pl->tracing) {
    for (int i = 0; i < 4; ++i) QTP_CUDA(cudaEventCreate(&pl->ev[i]), "create trace event");
    pl->tracing = 1;
  } else if (!enable && pl->tracing) {
    for (int i = 0; i < 4; ++i) cudaEventDestroy(pl->ev[i]);
    pl->tracing = 0;
  }
  return QTP_OK;
}

qtp_status qtp_plan_stage_times(const qtp_plan* pl, float* ms3) {
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  if (!ms3) return fail(QTP_ERR_INVALID_ARG, "ms3 is NULL");
  if (!pl->tracing) return fail(QTP_ERR_INVALID_ARG, "tracing is not enabled on this plan");
  QTP_CUDA(cudaEventSynchronize(pl->ev[3]), "wait for trace events");
  for (int i = 0; i < 3; ++i) QTP_CUDA(cudaEventElapsedTime(&ms3[i], pl->ev[i], pl->ev[i + 1]), "stage time");
  return QTP_OK;
}

qtp_status qtp_plan_sync(const qtp_plan* pl, void* stream) {
  qtp_status r;
  if ((r = check_plan(pl)) != QTP_OK) return r;
  QTP_CUDA(cudaStreamSynchronize(as_stream(stream)), "stream synchronize");
  int v = 0;
  QTP_CUDA(cudaMemcpy(&v, pl->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (v != 0) {
    cudaMemset(pl->d_err, 0, sizeof(int));
    return fail(QTP_ERR_TIMEOUT, "a device-side wait gave up (code %d)", v);
  }
  return QTP_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// qtp_forward_noalloc: the forward product without any allocation.
//
// Some callers may not allocate device memory: a host program whose device
// memory is owned entirely by another allocator (a framework's caching pool or
// a fixed memory budget) must not call cudaMalloc behind that allocator's back,
// and latency-bound code cannot afford cudaMalloc's implicit synchronisation.
// Plan creation allocates (twiddles, error word) and qtp_forward needs a
// caller-provided workspace, so this entry point takes neither: its twiddle
// table, error word and spectra live in one file-scope device array of
// QTP_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library holds
// until the process exits.
// ----------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[QTP_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the static array in the current device's context.  In
// host code the array's name only stands for it; cudaGetSymbolAddress (which
// allocates nothing) gives the address, looked up on every call so that it
// stays valid after a device reset or a new primary context.
qtp_status noalloc_scratch(void** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch array");
  *out = ptr;
  return QTP_OK;
}

}  // namespace

extern "C" qtp_status qtp_forward_noalloc(int m, int n, int s, int p, int precision, const float* A,
                                          const float* B, float* C, void* stream) {
  g_err[0] = 0;
  if (m < 1 || n < 1 || s < 1 || p < 1)
    return fail(QTP_ERR_INVALID_ARG, "dimensions must be >= 1 (m=%d n=%d s=%d p=%d)", m, n, s, p);
  if (m > (1 << 20) || n > (1 << 20) || s > (1 << 20))
    return fail(QTP_ERR_INVALID_ARG, "m, n, s must be <= 2^20");
  if (p > QTP_MAX_P) return fail(QTP_ERR_UNSUPPORTED, "p=%d exceeds the supported maximum %d", p, QTP_MAX_P);
  if (precision != QTP_PREC_FP32 && precision != QTP_PREC_BF16X3 && precision != QTP_PREC_BF16)
    return fail(QTP_ERR_INVALID_ARG, "unknown precision %d", precision);
  qtp_plan pl;
  memset(&pl, 0, sizeof(pl));
  pl.m = m; pl.n = n; pl.s = s; pl.p = p;
  pl.precision = precision;
  pl.rp = make_radix_plan(p);
  pl.fft_split_fwd = fft_form(p, false);
  pl.fft_split_inv = fft_form(p, true);
  // static scratch: [twiddles][error word][forward workspace]
  const size_t tw_bytes = align256((size_t)plan_twiddle_count(&pl) * sizeof(float2));
  const size_t ws_off = tw_bytes + 256;
  const size_t need = ws_off + fwd_layout(&pl).total;
  if (need > (size_t)QTP_NOALLOC_SCRATCH_BYTES)
    return fail(QTP_ERR_WORKSPACE,
                "this product needs %zu bytes of scratch; qtp_forward_noalloc's static array holds %d bytes",
                need, QTP_NOALLOC_SCRATCH_BYTES);
  qtp_status r;
  if ((r = check_dev_ptr(A, "A")) != QTP_OK) return r;
  if ((r = check_dev_ptr(B, "B")) != QTP_OK) return r;
  if ((r = check_dev_ptr(C, "C")) != QTP_OK) return r;
  if (precision != QTP_PREC_FP32 && !tc_supported())
    return fail(QTP_ERR_UNSUPPORTED, "BF16 tensor-core products need an sm_103 device (tcgen05)");
  void* scratch = nullptr;
  if ((r = noalloc_scratch(&scratch)) != QTP_OK) return r;
  QTP_CUDA(cudaGetDevice(&pl.device), "cudaGetDevice");
  char* base = (char*)scratch;
  pl.d_tw = (float2*)base;
  pl.d_err = (int*)(base + tw_bytes);
  cudaStream_t st = as_stream(stream);
  // The array keeps the previous call's contents: the error word must start at
  // zero and the twiddles may belong to another p, so both are rewritten here.
  QTP_CUDA(cudaMemsetAsync(pl.d_err, 0, sizeof(int), st), "clear the error word");
  QTP_CUDA(plan_twiddles(&pl, st), "twiddles");
  return forward_impl(&pl, A, B, C, base + ws_off, st);
}
