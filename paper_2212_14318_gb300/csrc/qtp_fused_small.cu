// The whole of Algorithm 5.1 for one small product in one CTA: the DFT of
// every tube of A and B (Step 1), the per-frequency products (Step 2, Thm 5.1
// in the plain-transform form)
//   C1(f) = A1(f) B1(f) - A2(f) conj(B2(-f)),  C2(f) = A1(f) B2(f) + A2(f) conj(B1(-f)),
// and the inverse DFT with the 1/p scale (Step 3), with the inputs and all
// three spectra in shared memory and one launch instead of three.  For the products this path
// takes (spectra within kFusedSmemMax bytes, p <= kFusedMaxP) a launch costs
// more than the arithmetic: the tube transforms are the register DFTs for the
// compile-time lengths up to 32 (direct sums X(f) = sum_k x(k) w^(f k) over
// the plan's table of w^e otherwise), and the products run in FP32 on the CUDA
// cores, whatever precision the plan names.
#include "qtp_fft_common.cuh"
#include "qtp_internal.h"

namespace qtp {

namespace {

constexpr int kFusedThreads = 1024;

__device__ __forceinline__ float2 cmac(float2 acc, float2 x, float2 y) {
  acc.x = fmaf(x.x, y.x, fmaf(-x.y, y.y, acc.x));
  acc.y = fmaf(x.x, y.y, fmaf(x.y, y.x, acc.y));
  return acc;
}

// Shared memory, FP32 complex, every tube a row of pitch PP = p | 1 (odd, so
// that a thread per tube and a lane per sample are both free of bank
// conflicts): the raw tubes of A and B (copied in first, coalesced), the
// spectra Ah[plane][i][j][f], Bh[plane][j][t][f], Ch[half][i][t][f], and the
// twiddle table.  P > 0: steps 1 and 3 are the register DFTs of length P, one
// thread per tube; P = 0: direct sums over the table for any p.
template <int P>
__global__ void __launch_bounds__(kFusedThreads) fused_small_kernel(const float2* __restrict__ A,
                                                                    const float2* __restrict__ B,
                                                                    float2* __restrict__ C, int m, int n, int s, int p,
                                                                    const float2* __restrict__ tw) {
  using namespace fftdev;
  extern __shared__ float2 fused_sm[];
  const int PP = p | 1;
  const int mn = m * n, ns = n * s, ms = m * s;
  const int ta = 2 * mn, tb = 2 * ns, tc = 2 * ms;  // tubes
  float2* Ar = fused_sm;
  float2* Br = Ar + ta * PP;
  float2* Ah = Br + tb * PP;
  float2* Bh = Ah + ta * PP;
  float2* Ch = Bh + tb * PP;
  float2* w = Ch + tc * PP;  // w^e, e < p

  for (int idx = threadIdx.x; idx < ta * p; idx += blockDim.x) Ar[(idx / p) * PP + idx % p] = __ldg(A + idx);
  for (int idx = threadIdx.x; idx < tb * p; idx += blockDim.x) Br[(idx / p) * PP + idx % p] = __ldg(B + idx);
  for (int idx = threadIdx.x; idx < p; idx += blockDim.x) w[idx] = __ldg(tw + idx);
  __syncthreads();

  // Step 1: X(f) = sum_k x(k) w^(f k) for every tube of A and B
  if constexpr (P > 0) {
    for (int tube = threadIdx.x; tube < ta + tb; tube += blockDim.x) {
      const float2* x = tube < ta ? Ar + tube * PP : Br + (tube - ta) * PP;
      float2* y = tube < ta ? Ah + tube * PP : Bh + (tube - ta) * PP;
      float2 v[P];
#pragma unroll
      for (int k = 0; k < P; ++k) v[k] = x[k];
      Dft<P, false>::run(v);
#pragma unroll
      for (int f = 0; f < P; ++f) y[f] = v[f];
    }
  } else {
    for (int idx = threadIdx.x; idx < (ta + tb) * p; idx += blockDim.x) {
      const int tube = idx / p, f = idx - tube * p;
      const float2* x = tube < ta ? Ar + tube * PP : Br + (tube - ta) * PP;
      float2 acc = make_float2(0.f, 0.f);
      int ex = 0;  // (f k) mod p
      for (int k = 0; k < p; ++k) {
        acc = cmac(acc, x[k], w[ex]);
        ex += f;
        if (ex >= p) ex -= p;
      }
      (tube < ta ? Ah + tube * PP : Bh + (tube - ta) * PP)[f] = acc;
    }
  }
  __syncthreads();

  // Step 2: output (half h, row i, column t, frequency f); half h multiplies by
  // B's plane h at f and by B's other plane, conjugated, at -f
  for (int idx = threadIdx.x; idx < tc * p; idx += blockDim.x) {
    const int f = idx % p;
    int r = idx / p;
    const int t = r % s;
    r /= s;
    const int i = r % m;
    const int h = r / m;
    const int g = f == 0 ? 0 : p - f;
    const float2* a1 = Ah + i * n * PP + f;
    const float2* a2 = Ah + (mn + i * n) * PP + f;
    const float2* b1 = Bh + (h * ns + t) * PP + f;
    const float2* b2 = Bh + ((1 - h) * ns + t) * PP + g;
    const float sg = h == 0 ? -1.f : 1.f;
    float2 acc = make_float2(0.f, 0.f);
    float2 cor = make_float2(0.f, 0.f);  // sum_j A2(f) conj(b2)
    for (int j = 0; j < n; ++j) {
      acc = cmac(acc, a1[j * PP], b1[j * s * PP]);
      const float2 u = a2[j * PP], v = b2[j * s * PP];
      cor.x = fmaf(u.x, v.x, fmaf(u.y, v.y, cor.x));
      cor.y = fmaf(u.y, v.x, fmaf(-u.x, v.y, cor.y));
    }
    Ch[(idx / p) * PP + f] = make_float2(fmaf(sg, cor.x, acc.x), fmaf(sg, cor.y, acc.y));
  }
  __syncthreads();

  // Step 3: x(k) = 1/p sum_f X(f) conj(w^(f k)) for every tube of C, in place
  // for P > 0 (then copied out, coalesced), straight to C for P = 0
  const float scale = 1.f / (float)p;
  if constexpr (P > 0) {
    for (int tube = threadIdx.x; tube < tc; tube += blockDim.x) {
      float2* y = Ch + tube * PP;
      float2 v[P];
#pragma unroll
      for (int f = 0; f < P; ++f) v[f] = y[f];
      Dft<P, true>::run(v);
#pragma unroll
      for (int k = 0; k < P; ++k) y[k] = make_float2(v[k].x * scale, v[k].y * scale);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < tc * p; idx += blockDim.x) C[idx] = Ch[(idx / p) * PP + idx % p];
  } else {
    for (int idx = threadIdx.x; idx < tc * p; idx += blockDim.x) {
      const int tube = idx / p, k = idx - tube * p;
      const float2* x = Ch + tube * PP;
      float2 acc = make_float2(0.f, 0.f);
      int ex = 0;  // (f k) mod p
      for (int f = 0; f < p; ++f) {
        const float2 v = x[f], c = w[ex];  // v * conj(c)
        acc.x = fmaf(v.x, c.x, fmaf(v.y, c.y, acc.x));
        acc.y = fmaf(v.y, c.x, fmaf(-v.x, c.y, acc.y));
        ex += k;
        if (ex >= p) ex -= p;
      }
      C[idx] = make_float2(acc.x * scale, acc.y * scale);
    }
  }
}

template <int P>
cudaError_t fused_launch(const float2* A, const float2* B, float2* C, int m, int n, int s, int p, const float2* tw,
                         size_t smem, cudaStream_t st) {
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = ensure_smem_attr(attr_set, fused_small_kernel<P>, kFusedSmemMax);
  if (e != cudaSuccess) return e;
  fused_small_kernel<P><<<1, kFusedThreads, smem, st>>>(A, B, C, m, n, s, p, tw);
  return cudaGetLastError();
}

}  // namespace

size_t fused_small_smem(int m, int n, int s, int p) {
  const size_t tubes = 2 * (2 * (size_t)m * n + 2 * (size_t)n * s) + 2 * (size_t)m * s;
  return sizeof(float2) * (tubes * (size_t)(p | 1) + (size_t)p);
}

bool fused_small_eligible(int m, int n, int s, int p) {
  if (getenv("QTP_NO_FUSED")) return false;
  return p <= kFusedMaxP && fused_small_smem(m, n, s, p) <= kFusedSmemMax;
}

cudaError_t launch_fused_small(const float2* A, const float2* B, float2* C, int m, int n, int s, int p,
                               const float2* tw, cudaStream_t st) {
  const size_t smem = fused_small_smem(m, n, s, p);
  switch (p) {
    case 8: return fused_launch<8>(A, B, C, m, n, s, p, tw, smem, st);
    case 12: return fused_launch<12>(A, B, C, m, n, s, p, tw, smem, st);
    case 16: return fused_launch<16>(A, B, C, m, n, s, p, tw, smem, st);
    case 31: return fused_launch<31>(A, B, C, m, n, s, p, tw, smem, st);
    case 32: return fused_launch<32>(A, B, C, m, n, s, p, tw, smem, st);
    default: return fused_launch<0>(A, B, C, m, n, s, p, tw, smem, st);
  }
}

}  // namespace qtp
