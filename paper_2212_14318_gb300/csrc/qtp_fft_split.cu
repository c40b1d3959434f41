// Tube FFTs of Algorithm 5.1 (Steps 1 and 3) for long tubes, in two passes
// through an FP32 intermediate in the workspace ("four-step" transform).
//
// The forward transform of Step 1 writes its spectra frequency-major: for a
// frequency f, consecutive tubes land at consecutive addresses, so a store is
// coalesced only over as many tubes as one CTA holds.  A one-kernel transform
// keeps whole tubes in shared memory, and for p in the thousands that is one
// to four tubes: 2- to 8-byte store runs, a few percent of the HBM rate.  Here
// the tube length factors as p = N1 N2 with t = N2 n1 + n2 and
// f = k1 + N1 k2, so that (Cooley-Tukey)
//     X[k1 + N1 k2] = sum_n2 w_N2^(n2 k2) [w_p^(n2 k1) sum_n1 x[N2 n1 + n2] w_N1^(n1 k1)]
// and the two sums run in different kernels:
//   pass 1: a CTA loads whole tubes (contiguous), runs the N2 length-N1 DFTs
//           of each, applies w_p^(n2 k1) and writes Z[k1][tube][n2];
//   pass 2: a CTA takes one k1 and T2 ~ 64 tubes, reads their Z rows
//           (contiguous), runs the length-N2 DFTs and stores the spectra
//           frequency-major in runs of T2 tubes.
// The inverse (Step 3, scale 1/p) mirrors it: pass 1 gathers X[k1 + N1 k2]
// for one k1 over T2 tubes, inverse DFT over k2, twiddle w_p^(-n2 k1), writes
// Z[k1][tube][n2]; pass 2 loads all of a tube's Z, inverse DFT over k1 and
// stores the tube contiguously.  Each pass reads and writes every entry once
// (twice the one-kernel transform's bytes), all in long coalesced runs.  The
// sub-DFTs are the Stockham stages of the one-kernel transforms, reading the
// length-p twiddle table with stride N2 (w_N1^e = w_p^(e N2)) or N1.
//
// Compile-time form ("long" transforms, fft_long_*): when p = N1 N2 with N2 a
// length that has a tuned two-pass transform (64, 100, 128, 256) and N1 <= 32,
// the N1-point DFTs run in registers and the N2-point ones are that two-pass
// transform (qtp_fft_twopass.cuh) with its frequencies remapped:
//   forward pass 1: thread (tube, n2 or n2 pair) loads x[N2 n1 + n2] for all
//                   n1 (16-byte loads, coalesced across n2), DFT-N1 in
//                   registers, twiddle w_p^(n2 k1), stores Z[k1][tube][n2];
//   forward pass 2: for each k1, the two-pass N2 transform of the Z rows
//                   (tubes of length N2), storing frequency k1 + N1 k2;
//   inverse pass 1: for each k1, the inverse two-pass N2 transform gathering
//                   frequencies k1 + N1 k2, its output sample n2 multiplied by
//                   w_p^(-k1 n2), stored Z[k1][tube][n2];
//   inverse pass 2: thread (tube, n2 pair) loads Z[k1][tube][n2] for all k1,
//                   inverse DFT-N1, stores x[N2 n1 + n2] / N1.
// The N2 table w_N2^e sits after the length-p table (plan twiddles p + N2).
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>

#include "qtp_fft_common.cuh"
#include "qtp_fft_twopass.cuh"
#include "qtp_internal.h"

namespace qtp {

namespace {

using namespace fftdev;

constexpr int kSplitThreads = 256;
constexpr int kSplitElems = 4096;  // complex entries per ping-pong buffer (32 KB)

struct SplitArgs {
  int p, n1, n2;
  int T1;  // tubes per CTA in the whole-tube pass
  int T2;  // tubes per CTA in the per-k1 pass
  RadixPlan rp1, rp2;
};

__host__ __device__ inline long long ntubes_of(int rows, int cols) { return 2LL * rows * cols; }
__host__ __device__ inline long long div_up(long long a, long long b) { return (a + b - 1) / b; }

// Forward pass 1 for tubes [g0, g0 + Tb) of one tensor: Z[k1][g][n2].
__device__ void split_fwd1_body(const FftFwdJob& job, long long b, const SplitArgs& a, const float2* __restrict__ tw,
                                float2* __restrict__ z, float2* smem) {
  const int p = a.p, n1 = a.n1, n2 = a.n2, P1 = n1 | 1;
  const long long nt = ntubes_of(job.rows, job.cols);
  const long long g0 = b * a.T1;
  if (g0 >= nt) return;
  const int Tb = (int)min((long long)a.T1, nt - g0);
  float2* buf0 = smem;
  float2* buf1 = smem + a.T1 * n2 * P1;
  // sample t = N2 n1 + n2 of tube i -> virtual tube (i, n2), position n1
  const float2* src = job.in + g0 * p;
  const int n = Tb * p;
  if ((p & 1) == 0) {
    const float4* src4 = reinterpret_cast<const float4*>(src);
    for (int e2 = threadIdx.x; e2 < n / 2; e2 += blockDim.x) {
      const float4 v = __ldg(src4 + e2);
      const int e = 2 * e2;
      const int i = e / p, t = e - i * p;  // t even, t + 1 in the same tube
      const int q = t / n2, r = t - q * n2;
      buf0[(i * n2 + r) * P1 + q] = make_float2(v.x, v.y);
      const int q1 = (t + 1) / n2, r1 = (t + 1) - q1 * n2;
      buf0[(i * n2 + r1) * P1 + q1] = make_float2(v.z, v.w);
    }
  } else {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int i = e / p, t = e - i * p;
      const int q = t / n2, r = t - q * n2;
      buf0[(i * n2 + r) * P1 + q] = __ldg(src + e);
    }
  }
  __syncthreads();
  const float2* Y = run_stages<false>(buf0, buf1, Tb * n2, P1, a.rp1, tw, n2);
  // Z[k1][g0 + i][n2]: for each k1 a contiguous run of Tb * N2 entries
  const int run = Tb * n2;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int k1 = e / run, r = e - k1 * run;
    const int m2 = r % n2;
    float2 v = Y[r * P1 + k1];
    const int ex = m2 * k1;  // < p
    if (ex) v = cmul(v, twid<false>(tw, ex));
    z[(long long)k1 * nt * n2 + g0 * n2 + r] = v;
  }
}

// Forward pass 2 for one k1 and tubes [g0, g0 + Tb): spectra, frequency-major.
template <int FMT>
__device__ void split_fwd2_body(const FftFwdJob& job, long long b, const SplitArgs& a, const float2* __restrict__ tw,
                                const float2* __restrict__ z, float2* smem) {
  const int p = a.p, n1 = a.n1, n2 = a.n2, P2 = n2 | 1;
  const long long nt = ntubes_of(job.rows, job.cols);
  const long long nbat = div_up(nt, a.T2);
  const int k1 = (int)(b / nbat);
  const long long g0 = (b - k1 * nbat) * a.T2;
  const int Tb = (int)min((long long)a.T2, nt - g0);
  float2* buf0 = smem;
  float2* buf1 = smem + a.T2 * P2;
  long long* tube_off = reinterpret_cast<long long*>(smem + 2 * a.T2 * P2);
  const float2* src = z + (long long)k1 * nt * n2 + g0 * n2;
  const int n = Tb * n2;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e / n2, k = e - i * n2;
    buf0[i * P2 + k] = src[e];
  }
  constexpr int NPARTS = FMT == FMT_BF16X3 ? 4 : (FMT == FMT_BF16 ? 2 : 1);
  const long long per_plane = (long long)job.rows * job.cols;
  const long long ld = job.ld;
  const long long plane_f_stride = (long long)job.rows * ld;
  for (int i = threadIdx.x; i < Tb; i += blockDim.x) {
    const long long t = g0 + i;
    const long long plane = t / per_plane;
    const long long rem = t - plane * per_plane;
    const long long row = rem / job.cols;
    const long long col = rem - row * job.cols;
    tube_off[i] = plane * NPARTS * p * plane_f_stride + row * ld + col;
  }
  __syncthreads();
  const float2* X = run_stages<false>(buf0, buf1, Tb, P2, a.rp2, tw, n1);
  const long long part = (long long)p * plane_f_stride;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int k2 = e / Tb, i = e - k2 * Tb;
    const float2 v = X[i * P2 + k2];
    const long long o = tube_off[i] + (long long)(k1 + n1 * k2) * plane_f_stride;
    if (FMT == FMT_C32) {
      reinterpret_cast<float2*>(job.out)[o] = v;
    } else if (FMT == FMT_BF16X3) {
      __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(job.out);
      __nv_bfloat16 rh, rl, ih, il;
      split_bf16(v.x, rh, rl);
      split_bf16(v.y, ih, il);
      out[o] = rh;
      out[o + part] = rl;
      out[o + 2 * part] = ih;
      out[o + 3 * part] = il;
    } else {
      __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(job.out);
      out[o] = __float2bfloat16_rn(v.x);
      out[o + part] = __float2bfloat16_rn(v.y);
    }
  }
}

// Inverse pass 1 for one k1 and tubes [g0, g0 + Tb): Z[k1][g][n2].
__device__ void split_inv1_body(const FftInvJob& job, long long b, const SplitArgs& a, const float2* __restrict__ tw,
                                float2* __restrict__ z, float2* smem) {
  const int p = a.p, n1 = a.n1, n2 = a.n2, P2 = n2 | 1;
  const long long nt = ntubes_of(job.rows, job.cols);
  const long long nbat = div_up(nt, a.T2);
  const int k1 = (int)(b / nbat);
  const long long g0 = (b - k1 * nbat) * a.T2;
  const int Tb = (int)min((long long)a.T2, nt - g0);
  float2* buf0 = smem;
  float2* buf1 = smem + a.T2 * P2;
  long long* tube_off = reinterpret_cast<long long*>(smem + 2 * a.T2 * P2);
  const long long per_plane = (long long)job.rows * job.cols;
  for (int i = threadIdx.x; i < Tb; i += blockDim.x) {
    const long long t = g0 + i;
    const long long plane = t / per_plane;
    tube_off[i] = plane * p * per_plane + (t - plane * per_plane) + (long long)k1 * per_plane;
  }
  __syncthreads();
  const int n = Tb * n2;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int k2 = e / Tb, i = e - k2 * Tb;
    buf0[i * P2 + k2] = __ldg(job.in + tube_off[i] + (long long)n1 * k2 * per_plane);
  }
  __syncthreads();
  const float2* Y = run_stages<true>(buf0, buf1, Tb, P2, a.rp2, tw, n1);
  float2* dst = z + (long long)k1 * nt * n2 + g0 * n2;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e / n2, m2 = e - i * n2;
    float2 v = Y[i * P2 + m2];
    const int ex = m2 * k1;  // < p
    if (ex) v = cmul(v, twid<true>(tw, ex));
    dst[e] = v;
  }
}

// Inverse pass 2 for tubes [g0, g0 + Tb): the tubes, contiguous, scaled by 1/p.
__device__ void split_inv2_body(const FftInvJob& job, long long b, const SplitArgs& a, const float2* __restrict__ tw,
                                const float2* __restrict__ z, float2* smem) {
  const int p = a.p, n1 = a.n1, n2 = a.n2, P1 = n1 | 1;
  const long long nt = ntubes_of(job.rows, job.cols);
  const long long g0 = b * a.T1;
  if (g0 >= nt) return;
  const int Tb = (int)min((long long)a.T1, nt - g0);
  float2* buf0 = smem;
  float2* buf1 = smem + a.T1 * n2 * P1;
  const int run = Tb * n2;
  const int n = Tb * p;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int k1 = e / run, r = e - k1 * run;
    buf0[r * P1 + k1] = z[(long long)k1 * nt * n2 + g0 * n2 + r];
  }
  __syncthreads();
  const float2* X = run_stages<true>(buf0, buf1, Tb * n2, P1, a.rp1, tw, n2);
  const float scale = 1.0f / (float)p;
  float2* dst = job.out + g0 * p;
  if ((p & 1) == 0) {
    float4* dst4 = reinterpret_cast<float4*>(dst);
    for (int e2 = threadIdx.x; e2 < n / 2; e2 += blockDim.x) {
      const int e = 2 * e2;
      const int i = e / p, t = e - i * p;
      const int q = t / n2, r = t - q * n2;
      const int q1 = (t + 1) / n2, r1 = (t + 1) - q1 * n2;
      const float2 u = X[(i * n2 + r) * P1 + q];
      const float2 w = X[(i * n2 + r1) * P1 + q1];
      dst4[e2] = make_float4(u.x * scale, u.y * scale, w.x * scale, w.y * scale);
    }
  } else {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int i = e / p, t = e - i * p;
      const int q = t / n2, r = t - q * n2;
      const float2 u = X[(i * n2 + r) * P1 + q];
      dst[e] = make_float2(u.x * scale, u.y * scale);
    }
  }
}

// Kernels over up to two tensors (A and B, or dA and dB): blocks [0, nb0)
// belong to the first, the rest to the second; z0 / z1 their intermediates.
__global__ void __launch_bounds__(kSplitThreads) fft_split_fwd1(FftFwdJob j0, FftFwdJob j1, long long nb0,
                                                                SplitArgs a, const float2* __restrict__ tw,
                                                                float2* z0, float2* z1) {
  extern __shared__ float4 smem_f4[];
  const long long b = blockIdx.x;
  const bool second = b >= nb0;
  split_fwd1_body(second ? j1 : j0, second ? b - nb0 : b, a, tw, second ? z1 : z0, reinterpret_cast<float2*>(smem_f4));
}

template <int FMT>
__global__ void __launch_bounds__(kSplitThreads) fft_split_fwd2(FftFwdJob j0, FftFwdJob j1, long long nb0,
                                                                SplitArgs a, const float2* __restrict__ tw,
                                                                const float2* z0, const float2* z1) {
  extern __shared__ float4 smem_f4[];
  const long long b = blockIdx.x;
  const bool second = b >= nb0;
  split_fwd2_body<FMT>(second ? j1 : j0, second ? b - nb0 : b, a, tw, second ? z1 : z0,
                       reinterpret_cast<float2*>(smem_f4));
}

__global__ void __launch_bounds__(kSplitThreads) fft_split_inv1(FftInvJob j0, FftInvJob j1, long long nb0,
                                                                SplitArgs a, const float2* __restrict__ tw,
                                                                float2* z0, float2* z1) {
  extern __shared__ float4 smem_f4[];
  const long long b = blockIdx.x;
  const bool second = b >= nb0;
  split_inv1_body(second ? j1 : j0, second ? b - nb0 : b, a, tw, second ? z1 : z0, reinterpret_cast<float2*>(smem_f4));
}

__global__ void __launch_bounds__(kSplitThreads) fft_split_inv2(FftInvJob j0, FftInvJob j1, long long nb0,
                                                                SplitArgs a, const float2* __restrict__ tw,
                                                                const float2* z0, const float2* z1) {
  extern __shared__ float4 smem_f4[];
  const long long b = blockIdx.x;
  const bool second = b >= nb0;
  split_inv2_body(second ? j1 : j0, second ? b - nb0 : b, a, tw, second ? z1 : z0, reinterpret_cast<float2*>(smem_f4));
}

SplitArgs split_args(int p) {
  SplitArgs a;
  fft_split_dims(p, &a.n1, &a.n2);
  a.p = p;
  a.T1 = kSplitElems / (a.n2 * (a.n1 | 1));
  if (a.T1 < 1) a.T1 = 1;
  a.T2 = kSplitElems / (a.n2 | 1);
  if (a.T2 > 256) a.T2 = 256;
  a.rp1 = make_radix_plan(a.n1);
  a.rp2 = make_radix_plan(a.n2);
  return a;
}

size_t smem_pass1(const SplitArgs& a) { return (size_t)2 * a.T1 * a.n2 * (a.n1 | 1) * sizeof(float2); }
size_t smem_pass2(const SplitArgs& a) {
  return (size_t)2 * a.T2 * (a.n2 | 1) * sizeof(float2) + (size_t)a.T2 * sizeof(long long);
}

template <class K>
cudaError_t set_smem(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int FMT>
cudaError_t launch_fwd2(const FftFwdJob* jobs, int njobs, const SplitArgs& a, const float2* tw, const float2* z0,
                        const float2* z1, cudaStream_t st) {
  const size_t smem = smem_pass2(a);
  cudaError_t e = set_smem(fft_split_fwd2<FMT>, smem);
  if (e != cudaSuccess) return e;
  const long long nb0 = (long long)a.n1 * div_up(ntubes_of(jobs[0].rows, jobs[0].cols), a.T2);
  const long long nb1 = njobs > 1 ? (long long)a.n1 * div_up(ntubes_of(jobs[1].rows, jobs[1].cols), a.T2) : 0;
  if (nb0 + nb1 > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  fft_split_fwd2<FMT><<<(unsigned)(nb0 + nb1), kSplitThreads, smem, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], nb0,
                                                                          a, tw, z0, z1);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- long form

constexpr int kLongThreads = 256;
// In order of preference: at p = 4096, N2 = 128 measured 354 / 173 us forward /
// inverse on 64x64 tensors against 369 / 194 for 256 and 370 / 194 for 64.
constexpr int kLongN2[] = {128, 256, 100, 64};

// Register pass of the forward transform (PAIR: two neighbouring n2 per
// thread, 16-byte accesses).  Items over [job 0 tubes x N2 / W][job 1 ...].
template <int N1, bool PAIR>
__global__ void __launch_bounds__(kLongThreads) fft_long_fwd1(const float2* __restrict__ x0,
                                                              const float2* __restrict__ x1, long long items0,
                                                              long long items, long long nt0, long long nt1, int n2,
                                                              int p, const float2* __restrict__ tw, float2* z0,
                                                              float2* z1) {
  constexpr int W = PAIR ? 2 : 1;
  const long long it = (long long)blockIdx.x * kLongThreads + threadIdx.x;
  if (it >= items) return;
  const bool second = it >= items0;
  const long long li = second ? it - items0 : it;
  const float2* __restrict__ x = second ? x1 : x0;
  float2* z = second ? z1 : z0;
  const long long nt = second ? nt1 : nt0;
  const int per = n2 / W;
  const long long g = li / per;
  const int m2 = (int)(li - g * per) * W;
  const float2* src = x + g * p + m2;
  float2 a[N1], c[N1];
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    if (PAIR) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src + (long long)k * n2));
      a[k] = make_float2(v.x, v.y);
      c[k] = make_float2(v.z, v.w);
    } else {
      a[k] = __ldg(src + (long long)k * n2);
    }
  }
  Dft<N1, false>::run(a);
  if (PAIR) Dft<N1, false>::run(c);
  float2* dst = z + g * n2 + m2;
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    float2 u = a[k1];
    if (k1 > 0 && m2 > 0) u = cmul(u, twid<false>(tw, m2 * k1));
    float2* o = dst + (long long)k1 * nt * n2;
    if (PAIR) {
      float2 w = c[k1];
      if (k1 > 0) w = cmul(w, twid<false>(tw, (m2 + 1) * k1));
      *reinterpret_cast<float4*>(o) = make_float4(u.x, u.y, w.x, w.y);
    } else {
      *o = u;
    }
  }
}

// Register pass of the inverse transform: x[N2 n1 + n2] = 1/N1 sum_k1 Z[k1][g][n2] w_N1^(-k1 n1).
template <int N1, bool PAIR>
__global__ void __launch_bounds__(kLongThreads) fft_long_inv2(const float2* __restrict__ z0,
                                                              const float2* __restrict__ z1, long long items0,
                                                              long long items, long long nt0, long long nt1, int n2,
                                                              int p, float2* x0, float2* x1) {
  constexpr int W = PAIR ? 2 : 1;
  const long long it = (long long)blockIdx.x * kLongThreads + threadIdx.x;
  if (it >= items) return;
  const bool second = it >= items0;
  const long long li = second ? it - items0 : it;
  const float2* __restrict__ z = second ? z1 : z0;
  float2* x = second ? x1 : x0;
  const long long nt = second ? nt1 : nt0;
  const int per = n2 / W;
  const long long g = li / per;
  const int m2 = (int)(li - g * per) * W;
  const float2* src = z + g * n2 + m2;
  float2 a[N1], c[N1];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    if (PAIR) {
      const float4 v = *reinterpret_cast<const float4*>(src + (long long)k1 * nt * n2);
      a[k1] = make_float2(v.x, v.y);
      c[k1] = make_float2(v.z, v.w);
    } else {
      a[k1] = src[(long long)k1 * nt * n2];
    }
  }
  Dft<N1, true>::run(a);
  if (PAIR) Dft<N1, true>::run(c);
  const float sc = 1.0f / (float)N1;
  float2* dst = x + g * p + m2;
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    float2* o = dst + (long long)n1 * n2;
    if (PAIR) *reinterpret_cast<float4*>(o) = make_float4(a[n1].x * sc, a[n1].y * sc, c[n1].x * sc, c[n1].y * sc);
    else *o = make_float2(a[n1].x * sc, a[n1].y * sc);
  }
}

// Two-pass pass of the forward transform for every k1: blocks [0, n1 nbk0)
// belong to the first tensor (k1 = b / nbk0), the rest to the second.
template <int N2, int FMT>
__global__ void __launch_bounds__(kThreads, min_blocks<N2, false>()) fft_long_fwd2(FftFwdJob j0, FftFwdJob j1,
                                                                               long long nbk0, long long nbk1, int n1,
                                                                               int p, const float2* __restrict__ tw_n2,
                                                                               const float2* z0, const float2* z1) {
  extern __shared__ float4 smem_f4[];
  long long b = blockIdx.x;
  const bool second = b >= (long long)n1 * nbk0;
  if (second) b -= (long long)n1 * nbk0;
  const long long nbk = second ? nbk1 : nbk0;
  const int k1 = (int)(b / nbk);
  FftFwdJob job = second ? j1 : j0;
  job.in = (second ? z1 : z0) + (long long)k1 * ntubes_of(job.rows, job.cols) * N2;
  const LongMap L{n1, k1, p, nullptr};
  fs_fwd_body<N2, FMT, true>(job, b - k1 * nbk, tw_n2, reinterpret_cast<float2*>(smem_f4), L);
}

template <int N2>
__global__ void __launch_bounds__(kThreads, min_blocks<N2, true>()) fft_long_inv1(FftInvJob j0, FftInvJob j1,
                                                                              long long nbk0, long long nbk1, int n1,
                                                                              int p, const float2* __restrict__ tw_n2,
                                                                              const float2* __restrict__ tw_p,
                                                                              float2* z0, float2* z1) {
  extern __shared__ float4 smem_f4[];
  long long b = blockIdx.x;
  const bool second = b >= (long long)n1 * nbk0;
  if (second) b -= (long long)n1 * nbk0;
  const long long nbk = second ? nbk1 : nbk0;
  const int k1 = (int)(b / nbk);
  FftInvJob job = second ? j1 : j0;
  job.out = (second ? z1 : z0) + (long long)k1 * ntubes_of(job.rows, job.cols) * N2;
  const LongMap L{n1, k1, p, tw_p};
  fs_inv_body<N2, true>(job, b - k1 * nbk, tw_n2, reinterpret_cast<float2*>(smem_f4), L);
}

template <int N2, bool INV>
constexpr size_t long_smem() {
  return (size_t)N2 * fs_pitch(N2, INV, true) * sizeof(float2);
}

// Runs of the two-pass N2 transform over one k1's rows: the padded run space
// of the bf16 forward (odd rows get a phantom tube) or the plain one.
long long long_runs(int rows, int cols, int n2, bool inv, int fmt) {
  const int cp = (!inv && fmt != FMT_C32 && (cols & 1)) ? cols + 1 : cols;
  return div_up(2LL * rows * cp, tubes_for(n2, inv, true));
}

template <int N1>
cudaError_t launch_reg(bool inv, const float2* a0, const float2* a1, long long nt0, long long nt1, int n2, int p,
                       const float2* tw, float2* b0, float2* b1, cudaStream_t st) {
  constexpr bool PAIR = N1 <= 16;  // two n2 per thread while the registers allow
  const long long items0 = nt0 * n2 / (PAIR ? 2 : 1), items = items0 + nt1 * n2 / (PAIR ? 2 : 1);
  if (items == 0) return cudaSuccess;
  const long long blocks = div_up(items, kLongThreads);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (!inv)
    fft_long_fwd1<N1, PAIR><<<(unsigned)blocks, kLongThreads, 0, st>>>(a0, a1, items0, items, nt0, nt1, n2, p, tw, b0,
                                                                      b1);
  else
    fft_long_inv2<N1, PAIR><<<(unsigned)blocks, kLongThreads, 0, st>>>(a0, a1, items0, items, nt0, nt1, n2, p, b0, b1);
  return cudaGetLastError();
}

cudaError_t launch_reg_n1(int n1, bool inv, const float2* a0, const float2* a1, long long nt0, long long nt1, int n2,
                          int p, const float2* tw, float2* b0, float2* b1, cudaStream_t st) {
#define QTP_LONG_N1(N) \
  case N: return launch_reg<N>(inv, a0, a1, nt0, nt1, n2, p, tw, b0, b1, st);
  switch (n1) {
    QTP_LONG_N1(2) QTP_LONG_N1(3) QTP_LONG_N1(4) QTP_LONG_N1(5) QTP_LONG_N1(6) QTP_LONG_N1(8) QTP_LONG_N1(10)
    QTP_LONG_N1(12) QTP_LONG_N1(16) QTP_LONG_N1(20) QTP_LONG_N1(24) QTP_LONG_N1(25) QTP_LONG_N1(30) QTP_LONG_N1(32)
    default: return cudaErrorInvalidValue;
  }
#undef QTP_LONG_N1
}

template <int N2, int FMT>
cudaError_t launch_fwd2_long(const FftFwdJob* jobs, int njobs, int n1, int p, const float2* tw_n2, const float2* z0,
                             const float2* z1, cudaStream_t st) {
  constexpr size_t smem = long_smem<N2, false>();
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = ensure_smem_attr(attr_set, fft_long_fwd2<N2, FMT>, smem);
  if (e != cudaSuccess) return e;
  const long long nbk0 = long_runs(jobs[0].rows, jobs[0].cols, N2, false, FMT);
  const long long nbk1 = njobs > 1 ? long_runs(jobs[1].rows, jobs[1].cols, N2, false, FMT) : 0;
  const long long blocks = (long long)n1 * (nbk0 + nbk1);
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  fft_long_fwd2<N2, FMT><<<(unsigned)blocks, kThreads, smem, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], nbk0, nbk1,
                                                                    n1, p, tw_n2, z0, z1);
  return cudaGetLastError();
}

template <int N2>
cudaError_t launch_fwd2_fmt(const FftFwdJob* jobs, int njobs, int fmt, int n1, int p, const float2* tw_n2,
                            const float2* z0, const float2* z1, cudaStream_t st) {
  switch (fmt) {
    case FMT_C32: return launch_fwd2_long<N2, FMT_C32>(jobs, njobs, n1, p, tw_n2, z0, z1, st);
    case FMT_BF16X3: return launch_fwd2_long<N2, FMT_BF16X3>(jobs, njobs, n1, p, tw_n2, z0, z1, st);
    case FMT_BF16: return launch_fwd2_long<N2, FMT_BF16>(jobs, njobs, n1, p, tw_n2, z0, z1, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N2>
cudaError_t launch_inv1_long(const FftInvJob* jobs, int njobs, int n1, int p, const float2* tw_n2, const float2* tw_p,
                             float2* z0, float2* z1, cudaStream_t st) {
  constexpr size_t smem = long_smem<N2, true>();
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = ensure_smem_attr(attr_set, fft_long_inv1<N2>, smem);
  if (e != cudaSuccess) return e;
  const long long nbk0 = long_runs(jobs[0].rows, jobs[0].cols, N2, true, FMT_C32);
  const long long nbk1 = njobs > 1 ? long_runs(jobs[1].rows, jobs[1].cols, N2, true, FMT_C32) : 0;
  const long long blocks = (long long)n1 * (nbk0 + nbk1);
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  fft_long_inv1<N2><<<(unsigned)blocks, kThreads, smem, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], nbk0, nbk1, n1,
                                                              p, tw_n2, tw_p, z0, z1);
  return cudaGetLastError();
}

}  // namespace

static bool long_n1_ok(int n1) {
  static const int n1s[] = {2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 25, 30, 32};
  for (int c : n1s)
    if (c == n1) return true;
  return false;
}

int fft_long_splits(int p, int* n2s) {
  int k = 0;
  for (int N2 : kLongN2)
    if (p % N2 == 0 && long_n1_ok(p / N2)) n2s[k++] = N2;
  return k;
}

bool fft_long_dims(int p, int* n1, int* n2) {
  int c[4];
  if (fft_long_splits(p, c) == 0) return false;
  if (n1) *n1 = p / c[0];
  if (n2) *n2 = c[0];
  return true;
}

// n2 = 0: the default split (fft_long_dims); else that N2 (a fft_long_splits entry)
static bool long_split_of(int p, int n2_req, int* n1, int* n2) {
  if (n2_req == 0) return fft_long_dims(p, n1, n2);
  int c[4];
  const int k = fft_long_splits(p, c);
  for (int i = 0; i < k; ++i)
    if (c[i] == n2_req) {
      *n1 = p / n2_req;
      *n2 = n2_req;
      return true;
    }
  return false;
}

cudaError_t launch_fft_fwd_long(const FftFwdJob* jobs, int njobs, int fmt, int p, int n2_req, const float2* tw,
                                float2* scratch, cudaStream_t st) {
  int n1 = 0, n2 = 0;
  if (njobs < 1 || njobs > 2 || !long_split_of(p, n2_req, &n1, &n2)) return cudaErrorInvalidValue;
  const long long nt0 = ntubes_of(jobs[0].rows, jobs[0].cols);
  const long long nt1 = njobs > 1 ? ntubes_of(jobs[1].rows, jobs[1].cols) : 0;
  float2* z0 = scratch;
  float2* z1 = scratch + nt0 * p;
  cudaError_t e = launch_reg_n1(n1, false, jobs[0].in, njobs > 1 ? jobs[1].in : jobs[0].in, nt0, nt1, n2, p, tw, z0,
                                z1, st);
  if (e != cudaSuccess) return e;
  const float2* tw_n2 = tw + p;
  switch (n2) {
    case 256: return launch_fwd2_fmt<256>(jobs, njobs, fmt, n1, p, tw_n2, z0, z1, st);
    case 128: return launch_fwd2_fmt<128>(jobs, njobs, fmt, n1, p, tw_n2, z0, z1, st);
    case 100: return launch_fwd2_fmt<100>(jobs, njobs, fmt, n1, p, tw_n2, z0, z1, st);
    case 64: return launch_fwd2_fmt<64>(jobs, njobs, fmt, n1, p, tw_n2, z0, z1, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fft_inv_long(const FftInvJob* jobs, int njobs, int p, int n2_req, const float2* tw,
                                float2* scratch, cudaStream_t st) {
  int n1 = 0, n2 = 0;
  if (njobs < 1 || njobs > 2 || !long_split_of(p, n2_req, &n1, &n2)) return cudaErrorInvalidValue;
  const long long nt0 = ntubes_of(jobs[0].rows, jobs[0].cols);
  const long long nt1 = njobs > 1 ? ntubes_of(jobs[1].rows, jobs[1].cols) : 0;
  float2* z0 = scratch;
  float2* z1 = scratch + nt0 * p;
  const float2* tw_n2 = tw + p;
  cudaError_t e;
  switch (n2) {
    case 256: e = launch_inv1_long<256>(jobs, njobs, n1, p, tw_n2, tw, z0, z1, st); break;
    case 128: e = launch_inv1_long<128>(jobs, njobs, n1, p, tw_n2, tw, z0, z1, st); break;
    case 100: e = launch_inv1_long<100>(jobs, njobs, n1, p, tw_n2, tw, z0, z1, st); break;
    case 64: e = launch_inv1_long<64>(jobs, njobs, n1, p, tw_n2, tw, z0, z1, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return launch_reg_n1(n1, true, z0, z1, nt0, nt1, n2, p, nullptr, jobs[0].out, njobs > 1 ? jobs[1].out : jobs[0].out,
                       st);
}

bool fft_split_dims(int p, int* n1, int* n2) {
  // the largest divisor N2 <= sqrt(p), and N1 = p / N2 >= N2
  int best = 1;
  for (int d = 2; (long long)d * d <= p; ++d)
    if (p % d == 0) best = d;
  if (n1) *n1 = p / best;
  if (n2) *n2 = best;
  return best >= 4;
}

bool fft_split_eligible(int p, bool inv) {
  if (!fft_split_dims(p, nullptr, nullptr)) return false;
  if (const char* env = getenv("QTP_FFT_SPLIT")) {
    if (env[0] == '0') return false;
    if (env[0] == '1') return p > 128;  // both directions, also lengths with a one-kernel transform
  }
  // Measured (64 x 64 tensors): the forward two-pass form beats the one-kernel
  // transform from the lengths where a CTA holds a single tube (p = 4096:
  // 1.14 against 2.65 ms), not at p = 1000 (0.30 against 0.23 ms); the
  // inverse two-pass form is slower at both (0.65 against 0.51 ms at 4096).
  return !inv && p >= 2048 && fft_fixed_tubes(p, false) == 0;
}

int fft_form(int p, bool inv) {
  if (const char* env = getenv("QTP_FFT_SPLIT")) {
    if (p <= 128 || env[0] == '0') return FFT_ONE;
    if (env[0] == '2' && fft_long_dims(p, nullptr, nullptr)) return FFT_LONG;
    if (env[0] == '1' || env[0] == '2') return fft_split_dims(p, nullptr, nullptr) ? FFT_SPLIT : FFT_ONE;
  }
  if (p > 128 && fft_fixed_tubes(p, false) == 0 && fft_long_dims(p, nullptr, nullptr)) return FFT_LONG;
  return fft_split_eligible(p, inv) ? FFT_SPLIT : FFT_ONE;
}

size_t fft_split_scratch_bytes(int p, long long rows, long long cols) {
  return (size_t)ntubes_of((int)rows, (int)cols) * p * sizeof(float2);
}

cudaError_t launch_fft_fwd_split(const FftFwdJob* jobs, int njobs, int fmt, int p, const float2* tw, float2* scratch,
                                 cudaStream_t st) {
  if (njobs < 1 || njobs > 2) return cudaErrorInvalidValue;
  const SplitArgs a = split_args(p);
  float2* z0 = scratch;
  float2* z1 = scratch + ntubes_of(jobs[0].rows, jobs[0].cols) * p;
  const long long nb0 = div_up(ntubes_of(jobs[0].rows, jobs[0].cols), a.T1);
  const long long nb1 = njobs > 1 ? div_up(ntubes_of(jobs[1].rows, jobs[1].cols), a.T1) : 0;
  if (nb0 + nb1 == 0) return cudaSuccess;
  if (nb0 + nb1 > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const size_t s1 = smem_pass1(a);
  cudaError_t e = set_smem(fft_split_fwd1, s1);
  if (e != cudaSuccess) return e;
  fft_split_fwd1<<<(unsigned)(nb0 + nb1), kSplitThreads, s1, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], nb0, a, tw,
                                                                    z0, z1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (fmt) {
    case FMT_C32: return launch_fwd2<FMT_C32>(jobs, njobs, a, tw, z0, z1, st);
    case FMT_BF16X3: return launch_fwd2<FMT_BF16X3>(jobs, njobs, a, tw, z0, z1, st);
    case FMT_BF16: return launch_fwd2<FMT_BF16>(jobs, njobs, a, tw, z0, z1, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fft_inv_split(const FftInvJob* jobs, int njobs, int p, const float2* tw, float2* scratch,
                                 cudaStream_t st) {
  if (njobs < 1 || njobs > 2) return cudaErrorInvalidValue;
  const SplitArgs a = split_args(p);
  float2* z0 = scratch;
  float2* z1 = scratch + ntubes_of(jobs[0].rows, jobs[0].cols) * p;
  const long long t0 = ntubes_of(jobs[0].rows, jobs[0].cols);
  const long long t1 = njobs > 1 ? ntubes_of(jobs[1].rows, jobs[1].cols) : 0;
  const long long nb0 = (long long)a.n1 * div_up(t0, a.T2), nb1 = (long long)a.n1 * div_up(t1, a.T2);
  if (nb0 + nb1 == 0) return cudaSuccess;
  if (nb0 + nb1 > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const size_t s2 = smem_pass2(a);
  cudaError_t e = set_smem(fft_split_inv1, s2);
  if (e != cudaSuccess) return e;
  const FftInvJob& j1 = njobs > 1 ? jobs[1] : jobs[0];
  fft_split_inv1<<<(unsigned)(nb0 + nb1), kSplitThreads, s2, st>>>(jobs[0], j1, nb0, a, tw, z0, z1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long mb0 = div_up(t0, a.T1), mb1 = div_up(t1, a.T1);
  const size_t s1 = smem_pass1(a);
  e = set_smem(fft_split_inv2, s1);
  if (e != cudaSuccess) return e;
  fft_split_inv2<<<(unsigned)(mb0 + mb1), kSplitThreads, s1, st>>>(jobs[0], j1, mb0, a, tw, z0, z1);
  return cudaGetLastError();
}

}  // namespace qtp
