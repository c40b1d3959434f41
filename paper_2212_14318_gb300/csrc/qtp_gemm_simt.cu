// Per-frequency complex products of Algorithm 5.1 Step 2 in plain FP32 FMA
// on the CUDA cores (the "plain FP32 GPU path").
//
// For frequency f and output half h the kernel forms
//   Out_h(f) = sum_kh sign[h][kh] * opA[h][kh](f) . opB[h][kh](f)
// from operand views of the frequency-major spectra (see GemmProblem).  In the
// forward product (Thm 5.1, eqs. TC/TC2 in the plain-transform form) this is
//   C1_f = A1_f B1_f - A2_f conj(B2_{-f}),  C2_f = A1_f B2_f + A2_f conj(B1_{-f}),
// i.e. 4p complex m x n x s products (Thm 5.2).  Conjugation and sign are
// applied while a tile is staged to shared memory, so the inner loop is a
// plain complex multiply-add.
//
// Tiling: 64 x 128 complex outputs per CTA, 256 threads, each thread owns a
// 4 x 8 register tile (columns strided by 16 so that stores coalesce);
// K is staged 8 complex at a time.
#include "qtp_internal.h"

namespace qtp {

namespace {

constexpr int BM = 64;
constexpr int BN = 128;
constexpr int BK = 8;
constexpr int kThreads = 256;

// One BM x BN complex output tile (frequency f, output half h, origin m0, n0).
__device__ __forceinline__ void simt_tile(const GemmProblem& pr, int f, int h, int m0, int n0) {
  __shared__ __align__(16) float2 As[BK][BM];
  __shared__ __align__(16) float2 Bs[BK][BN];
  const int tx = threadIdx.x & 15;
  const int ty = threadIdx.x >> 4;
  const int p = pr.p;

  float2 acc[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = make_float2(0.f, 0.f);

  for (int kh = 0; kh < 2; ++kh) {
    const CView va = pr.a[h][kh];
    const CView vb = pr.b[h][kh];
    const float sg = pr.sign[h][kh];
    if (va.base == nullptr || vb.base == nullptr) continue;
    const int ga = va.fneg ? (p - f) % p : f;
    const int gb = vb.fneg ? (p - f) % p : f;
    const float2* abase = va.base + (long long)ga * va.fstride;
    const float2* bbase = vb.base + (long long)gb * vb.fstride;
    const float aim = va.conj ? -sg : sg;  // sign of imag(A) after conj and sign
    const float bim = vb.conj ? -1.f : 1.f;
    const bool a_kcontig = (va.kstride == 1);
    const bool b_kcontig = (vb.kstride == 1);
    for (int k0 = 0; k0 < pr.K; k0 += BK) {
      // A tile: BM x BK, 2 entries per thread.
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int idx = threadIdx.x + e * kThreads;
        int row, k;
        if (a_kcontig) { k = idx % BK; row = idx / BK; } else { row = idx % BM; k = idx / BM; }
        float2 v = make_float2(0.f, 0.f);
        if (m0 + row < pr.M && k0 + k < pr.K) {
          v = __ldg(abase + (long long)(m0 + row) * va.rstride + (long long)(k0 + k) * va.kstride);
          v.x *= sg;
          v.y *= aim;
        }
        As[k][row] = v;
      }
      // B tile: BK x BN, 4 entries per thread.
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = threadIdx.x + e * kThreads;
        int col, k;
        if (b_kcontig) { k = idx % BK; col = idx / BK; } else { col = idx % BN; k = idx / BN; }
        float2 v = make_float2(0.f, 0.f);
        if (n0 + col < pr.N && k0 + k < pr.K) {
          v = __ldg(bbase + (long long)(n0 + col) * vb.rstride + (long long)(k0 + k) * vb.kstride);
          v.y *= bim;
        }
        Bs[k][col] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a01 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 a23 = *reinterpret_cast<const float4*>(&As[kk][ty * 4 + 2]);
        const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                             make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
        float2 b[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            acc[r][c].x = fmaf(a[r].x, b[c].x, acc[r][c].x);
            acc[r][c].x = fmaf(-a[r].y, b[c].y, acc[r][c].x);
            acc[r][c].y = fmaf(a[r].x, b[c].y, acc[r][c].y);
            acc[r][c].y = fmaf(a[r].y, b[c].x, acc[r][c].y);
          }
      }
      __syncthreads();
    }
  }

  float2* out = pr.out + (long long)h * pr.out_hstride + (long long)f * pr.out_fstride;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int row = m0 + ty * 4 + r;
    if (row >= pr.M) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = n0 + tx + 16 * c;
      if (col < pr.N) out[(long long)row * pr.out_rstride + col] = acc[r][c];
    }
  }
}

__global__ void __launch_bounds__(kThreads) gemm_simt_kernel(GemmProblem pr) {
  simt_tile(pr, blockIdx.z >> 1, blockIdx.z & 1, blockIdx.y * BM, blockIdx.x * BN);
}

// Batched forward products: one CTA per tile of the global tile space (see
// GroupProblem); the CTA rebuilds its product's operand views from the
// workspace offsets: C1 = A1 B1 - A2 conj(B2(-f)), C2 = A1 B2 + A2 conj(B1(-f)).
__global__ void __launch_bounds__(kThreads) gemm_simt_grouped_kernel(const GroupProblem* __restrict__ probs,
                                                                     const int* __restrict__ prob_of_tile, char* ws) {
  const long long t = blockIdx.x;
  const GroupProblem& P = probs[__ldg(prob_of_tile + t)];
  long long local = t - P.tile_begin;
  const int nt = (int)(local % P.tiles_n);
  local /= P.tiles_n;
  const int mt = (int)(local % P.tiles_m);
  local /= P.tiles_m;
  const int h = (int)(local & 1);
  const int f = (int)(local >> 1);
  const long long m = P.M, n = P.K, s = P.N, p = P.p;
  const float2* A = reinterpret_cast<const float2*>(ws + P.sa_off);
  const float2* B = reinterpret_cast<const float2*>(ws + P.sb_off);
  GemmProblem pr;
  pr.M = P.M; pr.N = P.N; pr.K = P.K; pr.p = P.p;
  for (int hh = 0; hh < 2; ++hh)
    for (int kh = 0; kh < 2; ++kh) {
      CView a;
      a.base = A + kh * p * m * n;
      a.fstride = m * n; a.rstride = n; a.kstride = 1; a.fneg = 0; a.conj = 0;
      pr.a[hh][kh] = a;
      CView b;
      const int plane = (hh == kh) ? 0 : 1;  // h0: B1, B2(-f); h1: B2, B1(-f)
      b.base = B + plane * p * n * s;
      b.fstride = n * s; b.rstride = 1; b.kstride = s; b.fneg = kh; b.conj = kh;
      pr.b[hh][kh] = b;
      pr.sign[hh][kh] = (hh == 0 && kh == 1) ? -1.f : 1.f;
    }
  pr.out = reinterpret_cast<float2*>(ws + P.out_off);
  pr.out_hstride = p * m * s;
  pr.out_fstride = m * s;
  pr.out_rstride = s;
  simt_tile(pr, f, h, mt * BM, nt * BN);
}

}  // namespace

cudaError_t launch_gemm_simt_grouped(const GroupProblem* d_probs, const int* d_prob_of_tile, long long total_tiles,
                                     char* ws, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  if (total_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  gemm_simt_grouped_kernel<<<(unsigned)total_tiles, kThreads, 0, st>>>(d_probs, d_prob_of_tile, ws);
  return cudaGetLastError();
}

cudaError_t launch_gemm_simt(const GemmProblem& pr, cudaStream_t st) {
  if (pr.M <= 0 || pr.N <= 0 || pr.p <= 0) return cudaSuccess;
  dim3 grid((pr.N + BN - 1) / BN, (pr.M + BM - 1) / BM, 2 * pr.p);
  gemm_simt_kernel<<<grid, kThreads, 0, st>>>(pr);
  return cudaGetLastError();
}

}  // namespace qtp
