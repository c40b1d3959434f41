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

template <int FMT>
__global__ void __launch_bounds__(kFftThreads) fft_fwd_kernel(FftFwdJob job0, FftFwdJob job1, int njobs,
                                                              RadixPlan rp, int T,
                                                              const float2* __restrict__ tw) {
  extern __shared__ float4 smem_f4[];
  int b = blockIdx.x;
  const bool second = njobs > 1 && b >= job0.nblocks;
  if (second) b -= job0.nblocks;
  generic_fwd_body<FMT>(second ? job1 : job0, b, rp, T, tw, reinterpret_cast<float2*>(smem_f4));
}

__global__ void __launch_bounds__(kFftThreads) fft_inv_kernel(FftInvJob job0, FftInvJob job1, int njobs,
                                                              RadixPlan rp, int T,
                                                              const float2* __restrict__ tw) {
  extern __shared__ float4 smem_f4[];
  int b = blockIdx.x;
  const bool second = njobs > 1 && b >= job0.nblocks;
  if (second) b -= job0.nblocks;
  generic_inv_body(second ? job1 : job0, b, rp, T, tw, reinterpret_cast<float2*>(smem_f4));
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

size_t fft_smem_bytes_for(int p, bool inv) {
  const size_t fixed = fft_fixed_smem(p, inv);
  if (fixed) return fixed;
  return fft_smem_bytes(p, fft_tubes_per_block(p, inv));
}

int fft_tubes_per_block(int p, bool inv) {
  const int fixed = fft_fixed_tubes(p, inv);
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
  const int T = fft_tubes_per_block(rp.p, false);
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
  if (fft_fixed_tubes(rp.p, false)) return launch_fft_fwd_fixed(jobs, njobs, fmt, rp.p, tw, st);
  switch (fmt) {
    case FMT_C32: return launch_fwd_fmt<FMT_C32>(jobs, njobs, rp, tw, st);
    case FMT_BF16X3: return launch_fwd_fmt<FMT_BF16X3>(jobs, njobs, rp, tw, st);
    case FMT_BF16: return launch_fwd_fmt<FMT_BF16>(jobs, njobs, rp, tw, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fft_inv(const FftInvJob* jobs, int njobs, const RadixPlan& rp, const float2* tw,
                           cudaStream_t st) {
  if (fft_fixed_tubes(rp.p, true)) return launch_fft_inv_fixed(jobs, njobs, rp.p, tw, st);
  const int T = fft_tubes_per_block(rp.p, true);
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
