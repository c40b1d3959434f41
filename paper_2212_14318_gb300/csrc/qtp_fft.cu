// Tube FFTs of Algorithm 5.1 (Steps 1 and 3).
//
// Step 1 (Thm 4.4, eq. fft-Q) transforms every tube X(r, k, :) of both
// Cayley-Dickson halves along the third mode with the unnormalised DFT,
// omega = exp(-2 pi i / p) (eq. DFT, Prop. 2.1).  Step 3 (eq. ifft-C) is the
// inverse transform with scale 1/p.
//
// Kernel design (GB300): a CTA owns T consecutive tubes.  The forward kernel
// reads them as one contiguous run (tube-contiguous layout, 16-byte loads),
// runs a self-sorting mixed-radix Stockham FFT in shared memory (radices 8,
// 4, 2 and 3, 5, 7 unrolled in registers; any other prime as a direct DFT),
// and writes the spectrum frequency-major, X_hat[plane][f][row][col], so that
// for a fixed frequency consecutive tubes land at consecutive addresses: the
// transpose into the per-frequency GEMM operand layout is fused into the
// store.  In the BF16 formats the store also splits each FP32 value x into
// hi = bf16(x), lo = bf16(x - hi).  The inverse kernel does the mirror image:
// frequency-major gather, Stockham with conjugate twiddles, contiguous store.
// Tubes sit at an odd stride (p | 1) in shared memory and consecutive threads
// take consecutive tubes, so the stages, gathers and scatters are free of bank
// conflicts.
#include <cuda_bf16.h>

#include "qtp_fft_common.cuh"
#include "qtp_internal.h"

namespace qtp {

namespace {

using namespace fftdev;

constexpr int kFftThreads = 256;
constexpr int kFftElemsPerBuf = 4096;  // complex entries per ping-pong buffer
constexpr int kFftMaxTubes = 512;

// One radix-R Stockham stage for butterfly j of one tube: the inputs sit at
// stride p/R, are twiddled by w_{Ns R}^(r (j mod Ns)), transformed, and written
// to (j / Ns) Ns R + (j mod Ns) + r Ns.  Ns is the length already transformed.
template <int R, bool INV>
__device__ __forceinline__ void butterfly(const float2* __restrict__ in, float2* __restrict__ out, int j,
                                          int Ns, int p, const float2* __restrict__ tw) {
  const int stride = p / R;
  const int k = j % Ns;
  const int twstep = p / (Ns * R);
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v[r] = in[j + r * stride];
    if (r > 0 && k > 0) v[r] = cmul(v[r], twid<INV>(tw, r * k * twstep));
  }
  Dft<R, INV>::run(v, tw, p);
  const int base = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
}

// Radix that is a prime > 8: direct DFT of length R straight from shared memory.
template <bool INV>
__device__ __forceinline__ void butterfly_generic(const float2* __restrict__ in, float2* __restrict__ out,
                                                  int j, int Ns, int R, int p,
                                                  const float2* __restrict__ tw) {
  const int stride = p / R;
  const int k = j % Ns;
  const int twstep = p / (Ns * R);
  const int base = (j / Ns) * Ns * R + k;
  for (int u = 0; u < R; ++u) {
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < R; ++r) {
      float2 x = in[j + r * stride];
      if (r > 0 && k > 0) x = cmul(x, twid<INV>(tw, r * k * twstep));
      const int e = ((r * u) % R) * stride;
      acc = cadd(acc, e ? cmul(x, twid<INV>(tw, e)) : x);
    }
    out[base + u * Ns] = acc;
  }
}

// All stages over T tubes held at tube stride P in buf0.  Returns the buffer
// that holds the result (natural order).
template <bool INV>
__device__ float2* run_stages(float2* buf0, float2* buf1, int T, int P, const RadixPlan& rp,
                              const float2* __restrict__ tw) {
  const int p = rp.p;
  float2* in = buf0;
  float2* out = buf1;
  int Ns = 1;
  for (int st = 0; st < rp.nstages; ++st) {
    const int R = rp.radix[st];
    const int nb = p / R;  // butterflies per tube
    const int total = T * nb;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      // tube-fastest: with an odd tube stride P consecutive threads hit
      // distinct banks for every radix and stage
      const int j = idx / T;
      const int tube = idx - j * T;
      const float2* ti = in + tube * P;
      float2* to = out + tube * P;
      switch (R) {
        case 2: butterfly<2, INV>(ti, to, j, Ns, p, tw); break;
        case 3: butterfly<3, INV>(ti, to, j, Ns, p, tw); break;
        case 4: butterfly<4, INV>(ti, to, j, Ns, p, tw); break;
        case 5: butterfly<5, INV>(ti, to, j, Ns, p, tw); break;
        case 7: butterfly<7, INV>(ti, to, j, Ns, p, tw); break;
        case 8: butterfly<8, INV>(ti, to, j, Ns, p, tw); break;
        default: butterfly_generic<INV>(ti, to, j, Ns, R, p, tw); break;
      }
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    Ns *= R;
  }
  return in;
}

template <int FMT>
__global__ void __launch_bounds__(kFftThreads) fft_fwd_kernel(FftFwdJob job0, FftFwdJob job1, int njobs,
                                                              RadixPlan rp, int T,
                                                              const float2* __restrict__ tw) {
  extern __shared__ float4 smem_f4[];
  float2* smem = reinterpret_cast<float2*>(smem_f4);
  const int p = rp.p;
  const int P = p | 1;
  int b = blockIdx.x;
  const FftFwdJob& job = (njobs > 1 && b >= job0.nblocks) ? job1 : job0;
  if (njobs > 1 && b >= job0.nblocks) b -= job0.nblocks;
  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = (long long)b * T;
  if (t0 >= ntubes) return;
  const int Tb = (int)min((long long)T, ntubes - t0);
  float2* buf0 = smem;
  float2* buf1 = smem + T * P;
  long long* tube_off = reinterpret_cast<long long*>(smem + 2 * T * P);

  // Contiguous load of Tb tubes (Tb * p complex) into padded rows.
  const float2* src = job.in + t0 * p;
  const int n = Tb * p;
  if ((p & 1) == 0) {
    const float4* src4 = reinterpret_cast<const float4*>(src);
    for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
      const float4 v = __ldg(src4 + i);
      const int e = 2 * i;
      const int tube = e / p;
      const int k = e - tube * p;
      buf0[tube * P + k] = make_float2(v.x, v.y);
      buf0[tube * P + k + 1] = make_float2(v.z, v.w);
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int tube = i / p;
      const int k = i - tube * p;
      buf0[tube * P + k] = __ldg(src + i);
    }
  }
  // Output offset of frequency 0 of every tube (one 64-bit division per tube).
  const long long ld = job.ld;
  const long long plane_f_stride = (long long)job.rows * ld;  // one (plane, part, f) slab
  constexpr int NPARTS = FMT == FMT_BF16X3 ? 4 : (FMT == FMT_BF16 ? 2 : 1);
  for (int tube = threadIdx.x; tube < Tb; tube += blockDim.x) {
    const long long t = t0 + tube;
    const long long plane = t / per_plane;
    const long long rem = t - plane * per_plane;
    const long long row = rem / job.cols;
    const long long col = rem - row * job.cols;
    tube_off[tube] = plane * NPARTS * p * plane_f_stride + row * ld + col;
  }
  __syncthreads();
  const float2* X = run_stages<false>(buf0, buf1, Tb, P, rp, tw);

  // Frequency-major store: for a fixed f, consecutive tubes are consecutive columns.
  const long long part = (long long)p * plane_f_stride;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int f = i / Tb;
    const int tube = i - f * Tb;
    const float2 v = X[tube * P + f];
    const long long o = tube_off[tube] + (long long)f * plane_f_stride;
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

__global__ void __launch_bounds__(kFftThreads) fft_inv_kernel(FftInvJob job0, FftInvJob job1, int njobs,
                                                              RadixPlan rp, int T,
                                                              const float2* __restrict__ tw) {
  extern __shared__ float4 smem_f4[];
  float2* smem = reinterpret_cast<float2*>(smem_f4);
  const int p = rp.p;
  const int P = p | 1;
  int b = blockIdx.x;
  const FftInvJob& job = (njobs > 1 && b >= job0.nblocks) ? job1 : job0;
  if (njobs > 1 && b >= job0.nblocks) b -= job0.nblocks;
  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = (long long)b * T;
  if (t0 >= ntubes) return;
  const int Tb = (int)min((long long)T, ntubes - t0);
  float2* buf0 = smem;
  float2* buf1 = smem + T * P;
  const int n = Tb * p;

  // Frequency-major gather: spectra in[plane][f][row][col].
  long long* tube_off = reinterpret_cast<long long*>(smem + 2 * T * P);
  for (int tube = threadIdx.x; tube < Tb; tube += blockDim.x) {
    const long long t = t0 + tube;
    const long long plane = t / per_plane;
    tube_off[tube] = plane * p * per_plane + (t - plane * per_plane);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int f = i / Tb;
    const int tube = i - f * Tb;
    buf0[tube * P + f] = __ldg(job.in + tube_off[tube] + (long long)f * per_plane);
  }
  __syncthreads();
  const float2* X = run_stages<true>(buf0, buf1, Tb, P, rp, tw);

  const float scale = 1.0f / (float)p;
  float2* dst = job.out + t0 * p;
  if ((p & 1) == 0) {
    float4* dst4 = reinterpret_cast<float4*>(dst);
    for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
      const int e = 2 * i;
      const int tube = e / p;
      const int k = e - tube * p;
      const float2 a = X[tube * P + k];
      const float2 c = X[tube * P + k + 1];
      dst4[i] = make_float4(a.x * scale, a.y * scale, c.x * scale, c.y * scale);
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int tube = i / p;
      const int k = i - tube * p;
      const float2 a = X[tube * P + k];
      dst[i] = make_float2(a.x * scale, a.y * scale);
    }
  }
}

__global__ void twiddle_kernel(float2* tw, int p) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p) return;
  double s, c;
  sincospi(2.0 * (double)e / (double)p, &s, &c);
  tw[e] = make_float2((float)c, (float)(-s));
}

size_t fft_smem_bytes(int p, int T) { return (size_t)2 * T * (p | 1) * sizeof(float2) + (size_t)T * sizeof(long long); }

}  // namespace

RadixPlan make_radix_plan(int p) {
  RadixPlan rp;
  rp.p = p;
  rp.nstages = 0;
  int q = p;
  auto push = [&](int r) {
    rp.radix[rp.nstages++] = r;
    q /= r;
  };
  while (q % 8 == 0) push(8);
  if (q % 4 == 0) push(4);
  if (q % 2 == 0) push(2);
  for (int r : {3, 5, 7})
    while (q % r == 0) push(r);
  for (int r = 11; q > 1 && r * r <= q; r += 2)
    while (q % r == 0) push(r);
  if (q > 1) push(q);
  return rp;
}

int fft_tubes_per_block(int p) {
  const int fixed = fft_fixed_tubes(p);
  if (fixed) return fixed;
  int T = kFftElemsPerBuf / (p | 1);
  if (T > kFftMaxTubes) T = kFftMaxTubes;
  return T < 1 ? 1 : T;
}

cudaError_t launch_twiddles(float2* tw, int p, cudaStream_t st) {
  twiddle_kernel<<<(p + 255) / 256, 256, 0, st>>>(tw, p);
  return cudaGetLastError();
}

template <int FMT>
static cudaError_t launch_fwd_fmt(const FftFwdJob* jobs, int njobs, const RadixPlan& rp, const float2* tw,
                                  cudaStream_t st) {
  const int T = fft_tubes_per_block(rp.p);
  const size_t smem = fft_smem_bytes(rp.p, T);
  cudaError_t e = cudaFuncSetAttribute(fft_fwd_kernel<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  for (int i = 0; i < njobs; ++i) nb += jobs[i].nblocks;
  if (nb == 0) return cudaSuccess;
  fft_fwd_kernel<FMT><<<nb, kFftThreads, smem, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], njobs, rp, T, tw);
  return cudaGetLastError();
}

cudaError_t launch_fft_fwd(const FftFwdJob* jobs, int njobs, int fmt, const RadixPlan& rp, const float2* tw,
                           cudaStream_t st) {
  if (fft_fixed_tubes(rp.p)) return launch_fft_fwd_fixed(jobs, njobs, fmt, rp.p, tw, st);
  switch (fmt) {
    case FMT_C32: return launch_fwd_fmt<FMT_C32>(jobs, njobs, rp, tw, st);
    case FMT_BF16X3: return launch_fwd_fmt<FMT_BF16X3>(jobs, njobs, rp, tw, st);
    case FMT_BF16: return launch_fwd_fmt<FMT_BF16>(jobs, njobs, rp, tw, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fft_inv(const FftInvJob* jobs, int njobs, const RadixPlan& rp, const float2* tw,
                           cudaStream_t st) {
  if (fft_fixed_tubes(rp.p)) return launch_fft_inv_fixed(jobs, njobs, rp.p, tw, st);
  const int T = fft_tubes_per_block(rp.p);
  const size_t smem = fft_smem_bytes(rp.p, T);
  cudaError_t e = cudaFuncSetAttribute(fft_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  for (int i = 0; i < njobs; ++i) nb += jobs[i].nblocks;
  if (nb == 0) return cudaSuccess;
  fft_inv_kernel<<<nb, kFftThreads, smem, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], njobs, rp, T, tw);
  return cudaGetLastError();
}

}  // namespace qtp
