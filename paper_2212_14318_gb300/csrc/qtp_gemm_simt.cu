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

__global__ void __launch_bounds__(kThreads) gemm_simt_kernel(GemmProblem pr) {
  __shared__ __align__(16) float2 As[BK][BM];
  __shared__ __align__(16) float2 Bs[BK][BN];
  const int f = blockIdx.z >> 1;
  const int h = blockIdx.z & 1;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
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

}  // namespace

cudaError_t launch_gemm_simt(const GemmProblem& pr, cudaStream_t st) {
  if (pr.M <= 0 || pr.N <= 0 || pr.p <= 0) return cudaSuccess;
  dim3 grid((pr.N + BN - 1) / BN, (pr.M + BM - 1) / BM, 2 * pr.p);
  gemm_simt_kernel<<<grid, kThreads, 0, st>>>(pr);
  return cudaGetLastError();
}

}  // namespace qtp
