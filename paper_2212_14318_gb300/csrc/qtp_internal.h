// Internal declarations of libqtp (CUDA sources only; not part of the ABI).
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "../../include/qtp.h"

#define QTP_MAX_P 4096
#define QTP_MAX_RADIX_STAGES 16

// Error codes written to a plan's device error word by bounded waits.
#define QTP_DEVERR_TIMEOUT_FULL 1   // consumer gave up waiting for a TMA stage
#define QTP_DEVERR_TIMEOUT_EMPTY 2  // producer gave up waiting for a free stage
#define QTP_DEVERR_TIMEOUT_ACC 3    // epilogue gave up waiting for the accumulator

namespace qtp {

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per device for one
// kernel: `mask` (a static of the kernel's launcher) holds a bit per device
// already set.  Setting it before every launch cost host time that small
// products see inside their step.
template <class K>
inline cudaError_t ensure_smem_attr(std::atomic<unsigned long long>& mask, K kernel, size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((mask.load(std::memory_order_acquire) >> dev) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev < 64) mask.fetch_or(1ull << dev, std::memory_order_acq_rel);
  return e;
}

// Whole small products in one CTA (qtp_fused_small.cu): all three spectra of
// the product in shared memory, FP32 arithmetic.
constexpr int kFusedMaxP = 64;
constexpr size_t kFusedSmemMax = 96 * 1024;
size_t fused_small_smem(int m, int n, int s, int p);
bool fused_small_eligible(int m, int n, int s, int p);  // false when QTP_NO_FUSED is set
cudaError_t launch_fused_small(const float2* A, const float2* B, float2* C, int m, int n, int s, int p,
                               const float2* tw, cudaStream_t st);

// Programmatic dependent launch: a kernel launched with
// cudaLaunchAttributeProgrammaticStreamSerialization may start while the
// previous kernel on its stream drains; every thread that reads that kernel's
// output first executes grid_dep_wait() (griddepcontrol.wait: returns once the
// prerequisite grid has completed and its writes are visible).  A kernel
// calls grid_dep_launch() (griddepcontrol.launch_dependents) to let such a
// successor be scheduled before it finishes.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Output formats of the forward tube FFT (Alg. 5.1 Step 1).
enum SpecFormat : int {
  FMT_C32 = 0,     // complex FP32, [plane][f][row][ld]
  FMT_BF16X3 = 1,  // 4 bf16 parts (re_hi, re_lo, im_hi, im_lo), [plane][part][f][row][ld]
  FMT_BF16 = 2,    // 2 bf16 parts (re, im), [plane][part][f][row][ld]
};

inline int spec_parts(int fmt) { return fmt == FMT_BF16X3 ? 4 : (fmt == FMT_BF16 ? 2 : 1); }
inline int spec_elem_bytes(int fmt) { return fmt == FMT_C32 ? 8 : 2; }

// Radix plan of a length-p transform: p = prod(radix[i]).
struct RadixPlan {
  int p;
  int nstages;
  int radix[QTP_MAX_RADIX_STAGES];
};

RadixPlan make_radix_plan(int p);

// One tensor transformed by the forward FFT: tubes in[plane][row][col][0..p).
struct FftFwdJob {
  const float2* in;
  void* out;         // spectra, format given by the launch
  int rows, cols;    // tensor is (rows x cols x p) per plane
  int ld;            // row stride (elements) of the spectra, >= cols
  int nblocks;       // CTAs assigned to this job
};

// Inverse transform: spectra in[plane][f][row][col] (complex FP32, ld = cols)
// back to tubes out[plane][row][col][0..p), scaled by 1/p.
struct FftInvJob {
  const float2* in;
  float2* out;
  int rows, cols;
  int nblocks;
};

int fft_tubes_per_block(int p, bool inv);  // tubes per CTA of the forward / inverse transform
// Columns of the forward transform's run space for a tensor of `cols`
// columns written in format fmt: cols + 1 when the two-pass body pads odd
// rows for bf16 spectra (the phantom tube's stores land in the row padding),
// else cols.  Runs = ceil(2 rows fft_fwd_run_cols / tubes per CTA).
int fft_fwd_run_cols(int p, int fmt, int cols);
size_t fft_smem_bytes_for(int p, bool inv);  // dynamic shared memory of one such CTA

// Grouped (batched) tube FFTs: one job per tensor of each product.
struct FftGroupJob {
  long long block_begin;  // first global CTA of this job
  long long spec_off;     // byte offset of this tensor's spectra in the workspace
  int prod;               // product index into the per-call pointer table
  int which;              // 0 = A, 1 = B (forward input), 2 = C (inverse output)
  int rows, cols, ld, p;
  int T;                  // tubes per CTA for this p
  int tw_off;             // first entry of this p's twiddle table
  RadixPlan rp;           // for tube lengths without a compile-time kernel
};

// One launch over global CTAs [block0, block0 + nblocks), all of whose jobs
// have tube length p (any p without a compile-time kernel may share a range,
// with smem the largest of theirs).
cudaError_t launch_fft_fwd_grouped(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0,
                                   long long nblocks, int p, int fmt, const float2* const* d_ptrs, char* ws,
                                   const float2* d_tw, size_t smem, cudaStream_t st);
cudaError_t launch_fft_inv_grouped(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0,
                                   long long nblocks, int p, const float2* const* d_ptrs, char* ws,
                                   const float2* d_tw, size_t smem, cudaStream_t st);
size_t fft_fixed_smem(int p, bool inv);

// Compile-time specialisations (qtp_fft_fixed.cu) for the common tube lengths:
// tubes per CTA, or 0 when p has none; the launches return
// cudaErrorNotSupported for other p.
int fft_fixed_tubes(int p, bool inv);
cudaError_t launch_fft_fwd_fixed(const FftFwdJob* jobs, int njobs, int fmt, int p, const float2* tw,
                                 cudaStream_t st);
cudaError_t launch_fft_inv_fixed(const FftInvJob* jobs, int njobs, int p, const float2* tw, cudaStream_t st);

// Long tubes (qtp_fft_split.cu): the two-pass ("four-step") transforms
// through an FP32 intermediate, p = N1 N2.  fft_split_dims picks N2, the
// largest divisor <= sqrt(p), and returns false when it is below 4 (p prime
// or twice a prime, ...).  fft_split_eligible: whether the forward (inv =
// false) or inverse transform of length p takes the two-pass form by default
// (forward from p = 2048 up without a compile-time transform, where it
// measured faster); environment QTP_FFT_SPLIT=0: never, =1: both directions
// for every splittable length above 128.  Scratch: fft_split_scratch_bytes
// per tensor transformed in the same launch (the first tensor's intermediate
// first).
bool fft_split_dims(int p, int* n1, int* n2);
bool fft_split_eligible(int p, bool inv);
// Compile-time long form: p = N1 N2 with N2 in {128, 256, 100, 64} (a tuned
// two-pass length) and N1 <= 32 (registers).  fft_long_splits writes every
// such N2 of p (at most 4, in that order of preference) and returns their
// count; fft_long_dims gives the default (the first).  The launches take the
// N2 to use (0: the default); their twiddles are the length-p table followed
// by the length-N2 one.
int fft_long_splits(int p, int* n2s);
bool fft_long_dims(int p, int* n1, int* n2);
cudaError_t launch_fft_fwd_long(const FftFwdJob* jobs, int njobs, int fmt, int p, int n2, const float2* tw,
                                float2* scratch, cudaStream_t st);
cudaError_t launch_fft_inv_long(const FftInvJob* jobs, int njobs, int p, int n2, const float2* tw, float2* scratch,
                                cudaStream_t st);
// Transform form of a tube length, per direction: one kernel, the two-pass
// form with runtime-radix sub-DFTs, or the compile-time long form.  Default:
// the long form where fft_long_dims splits p (above 128, no one-kernel
// compile-time transform), else the runtime two-pass forward from p = 2048,
// else one kernel.  Environment QTP_FFT_SPLIT: 0 one kernel, 1 runtime
// two-pass, 2 long form (where p splits), for every length above 128.
enum FftForm : int { FFT_ONE = 0, FFT_SPLIT = 1, FFT_LONG = 2 };
int fft_form(int p, bool inv);
size_t fft_split_scratch_bytes(int p, long long rows, long long cols);
cudaError_t launch_fft_fwd_split(const FftFwdJob* jobs, int njobs, int fmt, int p, const float2* tw, float2* scratch,
                                 cudaStream_t st);
cudaError_t launch_fft_inv_split(const FftInvJob* jobs, int njobs, int p, const float2* tw, float2* scratch,
                                 cudaStream_t st);

cudaError_t launch_twiddles(float2* tw, int p, cudaStream_t st);
cudaError_t launch_fft_fwd(const FftFwdJob* jobs, int njobs, int fmt, const RadixPlan& rp,
                           const float2* tw, cudaStream_t st);
cudaError_t launch_fft_inv(const FftInvJob* jobs, int njobs, const RadixPlan& rp,
                           const float2* tw, cudaStream_t st);

// T-SVD (qtp_tsvd.cu): one CTA per frequency pair {f, -f} factors M_f of A's
// spectra H ([plane][f][m][n], complex FP32) and writes the spectra of U
// ([plane][f][m][k]), V ([plane][f][n][k]) and S ([plane][f][k][k], zeroed by
// the caller) and sigma ([f][k]); k = min(m, n) <= 64.  scratch: global
// buffers of tsvd_scratch_bytes(m, n, p) bytes when one pair's matrices do not
// fit in shared memory (0 bytes otherwise); *status is set to 1 (never
// cleared) when a pair's Jacobi sweeps stop at their limit still rotating.
size_t tsvd_scratch_bytes(int m, int n, int p);
cudaError_t launch_tsvd_pairs(const float2* H, int m, int n, int p, float2* Uh, float2* Vh, float2* Sh,
                              float* sigma, float2* scratch, int* status, cudaStream_t st);

// ----------------------------------------------------------------------------
// Per-frequency complex products (Alg. 5.1 Step 2), generic operand views.
//
// Output half h in {0,1} of frequency f is
//   Out_h(f) = sum_{kh in {0,1}} sign[h][kh] * opA[h][kh](f) . opB[h][kh](f)
// where opA is M x K and opB is K x N complex.  Element (r, k) of an operand
// view at frequency f reads base[g*fstride + r*rstride + k*kstride] with
// g = fneg ? (p - f) % p : f, conjugated when conj != 0.
// ----------------------------------------------------------------------------
struct CView {
  const float2* base;
  long long fstride, rstride, kstride;
  int fneg, conj;
};

struct GemmProblem {
  int M, N, K, p;
  CView a[2][2];  // [h][kh], rows = M index
  CView b[2][2];  // [h][kh], "rows" = N index (element (n, k) = opB(k, n))
  float sign[2][2];
  float2* out;    // out[h][f][row][col]
  long long out_hstride, out_fstride, out_rstride;
};

cudaError_t launch_gemm_simt(const GemmProblem& pr, cudaStream_t st);

// Tensor-core variant: operands are bf16 part planes written by the forward
// FFT in FMT_BF16X3 / FMT_BF16.  A plane view is (tensor, plane, fneg, conj),
// with the major-ness of each operand fixed per problem kind.
struct TcView {
  int tensor;     // index into TcProblem::tmap_* (0 or 1)
  int plane;      // Cayley-Dickson half, 0 or 1
  int fneg;       // read frequency (p - f) % p
  int conj;       // negate the imaginary part
};

enum TcKind : int {
  TC_FWD = 0,     // A K-major (A[f][i][j]),  B MN-major (B[f][j][c])
  TC_BWD_A = 1,   // A K-major (G[f][i][c]),  B K-major  (B[f][j][c], k = c)
  TC_BWD_B = 2,   // A MN-major (A[f][i][j], m = j, k = i), B MN-major (G[f][i][c])
};

// Tensor-core tile choice: 0 = heuristic (256 wide for N > 160; split
// accumulators for K > kTcSingleMaxK, promoted ones for K > kTcSplitMaxK),
// else one of these.
enum TcTile : int { TILE_AUTO = 0, TILE_256 = 1, TILE_128 = 2, TILE_128_SPLIT = 3, TILE_128_PROMOTE = 4 };

// Reduction lengths (K per half of the m x 2n x 2s complex product) up to which
// each split-BF16 accumulator mode keeps the relative error within 1e-5 on
// N(0,1) data, and the segment length of the promoted mode (K steps of 16).
constexpr int kTcSingleMaxK = 384;   // one accumulator pair (5.6e-6 at 256)
constexpr int kTcSplitMaxK = 1024;   // split accumulators (6.2e-6 at 1024, 1.0e-5 at 2048)
constexpr int kTcPromoteSteps = 32;  // promoted: at most 32 K steps per TMEM accumulation

// Failure-path testing: the environment variables QTP_INJECT_WITHHOLD (a K
// step index) and QTP_INJECT_WAIT_NS (nanoseconds) make the next tensor-core
// launches never load that K step's operands and bound every wait by that
// many nanoseconds, so the bounded waits expire and the kernels unwind
// (recording QTP_DEVERR_* in the error word) without touching any memory
// outside their buffers.  Unset: *withhold = -1, *wait_ns = the default bound.
void fault_injection(int* withhold, unsigned long long* wait_ns);

struct TcProblem {
  int kind;
  int tile;            // TcTile
  int M, N, K, p;
  int nparts;          // 4 (bf16x3) or 2 (bf16)
  TcView a[2][2];
  TcView b[2][2];
  float sign[2][2];
  float2* out;
  long long out_hstride, out_fstride, out_rstride;
  // Spectra tensors (bf16 parts): base, rows, cols, ld (elements).
  const void* a_base[2]; int a_rows[2], a_cols[2], a_ld[2];
  const void* b_base[2]; int b_rows[2], b_cols[2], b_ld[2];
};

// Grouped (batched) per-frequency products, forward only: product g reads its
// spectra at workspace offsets and writes C_hat at out_off.  Tiles of all
// products form one index space; product g owns tiles [tile_begin, tile_begin
// + tiles_m * tiles_n * p) ordered (f, mt, nt) on the tensor cores (a tile
// computes both output halves), and [tile_begin, tile_begin + tiles_m *
// tiles_n * 2 * p) ordered (f, h, mt, nt) in FP32; nt fastest.
struct GroupProblem {
  long long tile_begin;
  long long sa_off, sb_off, out_off;  // byte offsets in the workspace
  const void* tmA;                    // tensor maps (device memory), tensor-core path only
  const void* tmB;
  int M, N, K, p;
  int tiles_m, tiles_n;
  int lda, ldb;                       // spectra row strides (elements)
  int bn;                             // tile width (complex columns)
  int trans;                          // tensor-core path: tiles of C^T = B^T A^T (rows over s, columns over m)
};

cudaError_t launch_gemm_tc_grouped(const GroupProblem* d_probs, int nprobs, long long total_tiles, int nparts,
                                   char* ws, int* d_err, int num_ctas, cudaStream_t st);
cudaError_t launch_gemm_simt_grouped(const GroupProblem* d_probs, const int* d_prob_of_tile, long long total_tiles,
                                     char* ws, cudaStream_t st);
// Copy nbytes (<= kPutBlobBytes) of host data to device memory at dst with
// one stream-ordered one-block kernel (the bytes travel as its parameter, so
// the host buffer may change as soon as the call returns).
constexpr int kPutBlobBytes = 512;
cudaError_t launch_put_blob(const void* host, int nbytes, void* dst, cudaStream_t st);
// Tile shapes of the grouped kernels (rows x complex columns).
constexpr int kGroupTcBM = 128, kGroupTcBN = 64;
constexpr int kGroupSimtBM = 64, kGroupSimtBN = 128;
// Tensor map of a spectra tensor for the grouped tensor-core kernel (K-major A
// or MN-major B), written to host memory at *tm (128 bytes).
bool encode_group_map(void* tm, const void* base, int rows, int cols, int ld, int p, int nparts, bool mn_major,
                      bool all_parts, char* msg, size_t msglen);

bool tc_supported();

// Shared host helpers (qtp_api.cu): thread-local error message, spectra layout.
qtp_status set_error(qtp_status st, const char* fmt, ...);
void clear_error();
int spec_format_of(int precision);
long long spec_ld_of(int fmt, long long cols);
size_t spec_bytes_of(int fmt, long long p, long long rows, long long cols);
size_t c32_bytes_of(long long p, long long rows, long long cols);

cudaError_t launch_gemm_tc(const TcProblem& pr, int* d_err, cudaStream_t st, char* msg, size_t msglen,
                           int dep_mode = 0);
// The forward product's tensor-core problem (Thm 5.1 in the plain-transform
// form) over bf16 spectra sa (A, [plane][part][f][m][ld]), sb (B) written by
// the forward FFT, output C_hat sc ([plane][f][m][s], complex FP32).
TcProblem make_tc_fwd(int m, int n, int s, int p, int nparts, int tile, const void* sa, const void* sb, float2* sc);

}  // namespace qtp

struct qtp_plan {
  int m, n, s, p;
  int precision;
  unsigned flags;
  int tile[3];       // TcTile per product kind (forward, dA, dB); TILE_AUTO unless tuned
  int device;
  float2* d_tw;      // w^e = exp(-2 pi i e / p), e in [0, p)
  int* d_err;        // device error word written by bounded waits
  qtp::RadixPlan rp;
  int fft_split_fwd;  // FftForm of the forward / inverse tube transforms (two-pass
  int fft_split_inv;  // forms go through a workspace intermediate)
  int long_n2;        // N2 of the compile-time long form (0: its default split)
  int tracing;
  cudaEvent_t ev[4];  // stage boundaries of the last traced call
  // streams and events of qtp_forward_host_many, created on its first call
  struct HostPipe* pipe;
  // forward products of small m and s at many frequencies through the grouped
  // kernel (null: the single-product kernel)
  struct SmallTiles* small;
};
