// Tube FFTs of Algorithm 5.1 (Steps 1 and 3) specialised for a compile-time
// tube length P (the workloads' lengths 8, 12, 16, 31, 32, 64, 100, 128, and
// 256, 512, 1024 for long tubes), with every index computation known to the
// compiler.  Lengths with a split P = R1 R2 run the two-pass transform (one
// register DFT per pass, one shared-memory exchange; see fs_fwd_body); P = 31
// runs Stockham stages in shared memory at an odd tube stride.  Both store the
// forward spectra frequency-major with the bf16 hi/lo split fused in and, when
// the tensor has an even number of columns, two neighbouring tubes together
// (16-byte complex pairs or 4-byte bf16 pairs; gathered the same way by the
// inverse).  Grouped variants serve the batched path, one launch per length.
#include "qtp_fft_common.cuh"
#include "qtp_fft_twopass.cuh"
#include "qtp_internal.h"

namespace qtp {

namespace {

using namespace fftdev;

struct Radices {
  int n;
  int r[12];
};

// Greedy factorisation of P: radix 8 first, then 4, 2, then odd primes.
__host__ __device__ constexpr Radices radices_of(int p) {
  Radices rl{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
  int q = p;
  while (q % 8 == 0) { rl.r[rl.n++] = 8; q /= 8; }
  if (q % 4 == 0) { rl.r[rl.n++] = 4; q /= 4; }
  if (q % 2 == 0) { rl.r[rl.n++] = 2; q /= 2; }
  for (int f = 3; q > 1; f += 2)
    while (q % f == 0) { rl.r[rl.n++] = f; q /= f; }
  return rl;
}

template <int P, bool INV>
constexpr size_t smem_for() {
  if constexpr (split_of(P, INV).r1 != 0) return (size_t)P * fs_pitch(P, INV) * sizeof(float2);
  return (size_t)2 * tubes_for(P, INV) * (P | 1) * sizeof(float2);
}

// Radix-R Stockham butterfly j of one tube, Ns = length already transformed.
// Element k of the tube is read at in[k * IES] and written at out[k * OES]:
// stride 1 in the tube-major layout (tube t at t * (P | 1)) and stride T in
// the frequency-major layout (tube t at t, element k at k * T + t).
template <int R, int NS, int P, bool INV, int IES, int OES>
__device__ __forceinline__ void bfly(const float2* __restrict__ in, float2* __restrict__ out, int j,
                                     const float2* __restrict__ tw) {
  constexpr int stride = P / R;
  constexpr int twstep = P / (NS * R);
  const int k = j % NS;
  const int base = (j / NS) * NS * R + k;
  if constexpr (R <= 8) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = in[(j + r * stride) * IES];
      if (NS > 1 && r > 0) v[r] = cmul(v[r], twid<INV>(tw, r * k * twstep));
    }
    Dft<R, INV>::run(v, tw, P);
#pragma unroll
    for (int r = 0; r < R; ++r) out[(base + r * NS) * OES] = v[r];
  } else {
    static_assert(R < 0, "radices above 8 go through bfly_odd");
  }
}

// Odd radix R > 8, output pairs (u, R - u) for u in group G (4 pairs per
// group): one thread per (tube, butterfly, group) keeps the register count of
// the radix-R DFT low and spreads its work over all threads of the CTA.  Same
// symmetric form as Dft<R> (x_r +- x_{R-r} against compile-time cos / sin).
constexpr int kOddPairsPerThread = 4;
template <int R>
__host__ __device__ constexpr int odd_groups() {
  return ((R - 1) / 2 + kOddPairsPerThread - 1) / kOddPairsPerThread;
}

template <int R, int NS, int P, bool INV, int IES, int OES, int G>
__device__ __forceinline__ void bfly_odd(const float2* __restrict__ in, float2* __restrict__ out, int j,
                                         const float2* __restrict__ tw) {
  constexpr int H = (R - 1) / 2;
  constexpr int stride = P / R;
  constexpr int twstep = P / (NS * R);
  constexpr int u0 = 1 + G * kOddPairsPerThread;
  constexpr int u1 = u0 + kOddPairsPerThread - 1 < H ? u0 + kOddPairsPerThread - 1 : H;
  const int k = j % NS;
  const int base = (j / NS) * NS * R + k;
  const float2 x0 = in[j * IES];
  float2 sp[H], dm[H];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    float2 a = in[(j + r * stride) * IES];
    float2 c = in[(j + (R - r) * stride) * IES];
    if (NS > 1) {
      a = cmul(a, twid<INV>(tw, r * k * twstep));
      c = cmul(c, twid<INV>(tw, (R - r) * k * twstep));
    }
    sp[r - 1] = cadd(a, c);
    dm[r - 1] = csub(a, c);
  }
  if constexpr (G == 0) {
    float2 dc = x0;
#pragma unroll
    for (int r = 0; r < H; ++r) dc = cadd(dc, sp[r]);
    out[base * OES] = dc;
  }
  static_for<u0, u1 + 1>([&](auto uc) {
    constexpr int u = decltype(uc)::value;
    float2 a = x0, bsum = make_float2(0.f, 0.f);
    static_for<1, H + 1>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      constexpr float c = (float)cos_turn(r * u, R);
      constexpr float sn = (float)sin_turn(r * u, R);
      a.x = fmaf(sp[r - 1].x, c, a.x);
      a.y = fmaf(sp[r - 1].y, c, a.y);
      bsum.x = fmaf(dm[r - 1].x, sn, bsum.x);
      bsum.y = fmaf(dm[r - 1].y, sn, bsum.y);
    });
    const float2 mib = make_float2(bsum.y, -bsum.x);  // -i B
    out[(base + u * NS) * OES] = INV ? csub(a, mib) : cadd(a, mib);
    out[(base + (R - u) * NS) * OES] = INV ? cadd(a, mib) : csub(a, mib);
  });
}

template <int R, int NS, int P, bool INV, int IES, int OES, int G = 0>
__device__ __forceinline__ void bfly_odd_group(const float2* __restrict__ in, float2* __restrict__ out, int j, int g,
                                               const float2* __restrict__ tw) {
  if constexpr (G < odd_groups<R>()) {
    if (g == G) bfly_odd<R, NS, P, INV, IES, OES, G>(in, out, j, tw);
    else bfly_odd_group<R, NS, P, INV, IES, OES, G + 1>(in, out, j, g, tw);
  }
}

// Stages ST.. of the plan over the CTA's tubes; returns the buffer holding the
// result.  The first stage reads the frequency-major layout when IN_FM, the
// last stage writes it when OUT_FM; all other accesses are tube-major.
template <int P, int ST, int NS, bool INV, bool IN_FM, bool OUT_FM>
__device__ __forceinline__ float2* stages(float2* in, float2* out, int Tb, const float2* __restrict__ tw) {
  constexpr Radices RL = radices_of(P);
  if constexpr (ST == RL.n) {
    return in;
  } else {
    constexpr int R = RL.r[ST];
    constexpr int NB = P / R;
    constexpr int T = tubes_for(P, INV);
    constexpr int PP = P | 1;
    constexpr bool FMI = IN_FM && ST == 0;
    constexpr bool FMO = OUT_FM && ST == RL.n - 1;
    // tube-fastest: consecutive threads take consecutive tubes, so both layouts
    // are free of bank conflicts (odd stride PP, or unit stride)
    constexpr int NG = R > 8 ? odd_groups<R>() : 1;
    for (int idx = threadIdx.x; idx < T * NB * NG; idx += kThreads) {
      const int g = idx / (T * NB);
      const int rest = idx - g * (T * NB);
      const int j = rest / T;
      const int tube = rest - j * T;
      if (tube < Tb) {
        const float2* ti = in + (FMI ? tube : tube * PP);
        float2* to = out + (FMO ? tube : tube * PP);
        if constexpr (R > 8) bfly_odd_group<R, NS, P, INV, FMI ? T : 1, FMO ? T : 1>(ti, to, j, g, tw);
        else bfly<R, NS, P, INV, FMI ? T : 1, FMO ? T : 1>(ti, to, j, tw);
      }
    }
    __syncthreads();
    return stages<P, ST + 1, NS * R, INV, IN_FM, OUT_FM>(out, in, Tb, tw);
  }
}

// Forward transform of the b-th run of T = tubes_for(P) tubes of one tensor.
template <int P, int FMT>
__device__ __forceinline__ void fixed_fwd_body(const FftFwdJob& job, long long b, const float2* __restrict__ tw,
                                               float2* smem) {
  if constexpr (split_of(P, false).r1 != 0) {
    fs_fwd_body<P, FMT>(job, b, tw, smem);
    return;
  }
  constexpr int T = tubes_for(P, false);
  constexpr int PP = P | 1;
  constexpr int NPARTS = FMT == FMT_BF16X3 ? 4 : (FMT == FMT_BF16 ? 2 : 1);
  static_assert(kThreads % T == 0, "a thread keeps one tube in the store loops");
  float2* buf0 = smem;
  float2* buf1 = buf0 + T * PP;

  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = b * T;
  if (t0 >= ntubes) return;
  const int Tb = (int)min((long long)T, ntubes - t0);

  // contiguous load of the CTA's tubes; consecutive lanes write consecutive
  // elements of a tube (conflict-free with the odd tube stride PP)
  const float2* src = job.in + t0 * P;
  for (int i = threadIdx.x; i < Tb * P; i += kThreads) {
    const int tube = i / P;
    buf0[tube * PP + (i - tube * P)] = __ldg(src + i);
  }
  __syncthreads();
  const float2* X = stages<P, 0, 1, false, false, true>(buf0, buf1, Tb, tw);  // frequency-major result

  const long long ld = job.ld;
  const long long slab = (long long)job.rows * ld;  // one (plane, part, f) slab
  const long long part = (long long)P * slab;
  // spectra offset of tube t: [plane][part 0][f 0][row][col]
  auto spec_off = [&](long long t) {
    const long long plane = t / per_plane;
    const long long rem = t - plane * per_plane;
    const long long row = rem / job.cols;
    return plane * NPARTS * P * slab + row * ld + (rem - row * job.cols);
  };
  if ((job.cols & 1) == 0) {
    // pairs of neighbouring tubes share a row: 16-byte / 4-byte stores
    constexpr int TH = T / 2;
    const int tube = 2 * (threadIdx.x % TH);
    if (tube >= Tb) return;
    const long long o0 = spec_off(t0 + tube);
    for (int f = threadIdx.x / TH; f < P; f += kThreads / TH) {
      const float4 v01 = *reinterpret_cast<const float4*>(X + f * T + tube);
      const float2 v0 = make_float2(v01.x, v01.y);
      const float2 v1 = make_float2(v01.z, v01.w);
      const long long o = o0 + (long long)f * slab;
      if constexpr (FMT == FMT_C32) {
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(job.out) + o) = make_float4(v0.x, v0.y, v1.x, v1.y);
      } else if constexpr (FMT == FMT_BF16X3) {
        __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(job.out);
        __nv_bfloat16 rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
        split_bf16(v0.x, rh0, rl0);
        split_bf16(v0.y, ih0, il0);
        split_bf16(v1.x, rh1, rl1);
        split_bf16(v1.y, ih1, il1);
        *reinterpret_cast<__nv_bfloat162*>(out + o) = __halves2bfloat162(rh0, rh1);
        *reinterpret_cast<__nv_bfloat162*>(out + o + part) = __halves2bfloat162(rl0, rl1);
        *reinterpret_cast<__nv_bfloat162*>(out + o + 2 * part) = __halves2bfloat162(ih0, ih1);
        *reinterpret_cast<__nv_bfloat162*>(out + o + 3 * part) = __halves2bfloat162(il0, il1);
      } else {
        __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(job.out);
        *reinterpret_cast<__nv_bfloat162*>(out + o) =
            __halves2bfloat162(__float2bfloat16_rn(v0.x), __float2bfloat16_rn(v1.x));
        *reinterpret_cast<__nv_bfloat162*>(out + o + part) =
            __halves2bfloat162(__float2bfloat16_rn(v0.y), __float2bfloat16_rn(v1.y));
      }
    }
  } else {
    const int tube = threadIdx.x % T;
    if (tube >= Tb) return;
    const long long o0 = spec_off(t0 + tube);
    for (int f = threadIdx.x / T; f < P; f += kThreads / T) {
      const float2 v = X[f * T + tube];
      const long long o = o0 + (long long)f * slab;
      if constexpr (FMT == FMT_C32) {
        reinterpret_cast<float2*>(job.out)[o] = v;
      } else if constexpr (FMT == FMT_BF16X3) {
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
}

// Inverse transform (scale 1/P) of the b-th run of T = tubes_for(P) tubes.
template <int P>
__device__ __forceinline__ void fixed_inv_body(const FftInvJob& job, long long b, const float2* __restrict__ tw,
                                               float2* smem) {
  if constexpr (split_of(P, true).r1 != 0) {
    fs_inv_body<P>(job, b, tw, smem);
    return;
  }
  constexpr int T = tubes_for(P, true);
  constexpr int PP = P | 1;
  static_assert(kThreads % T == 0, "a thread keeps one tube in the gather loops");
  float2* buf0 = smem;
  float2* buf1 = buf0 + T * PP;

  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = b * T;
  if (t0 >= ntubes) return;
  const int Tb = (int)min((long long)T, ntubes - t0);

  // frequency-major gather of C_hat[plane][f][row][col]
  auto spec_off = [&](long long t) {
    const long long plane = t / per_plane;
    return plane * P * per_plane + (t - plane * per_plane);
  };
  if ((job.cols & 1) == 0) {
    constexpr int TH = T / 2;
    const int tube = 2 * (threadIdx.x % TH);
    if (tube < Tb) {
      const float2* in = job.in + spec_off(t0 + tube);
      for (int f = threadIdx.x / TH; f < P; f += kThreads / TH)
        *reinterpret_cast<float4*>(buf0 + f * T + tube) =
            __ldg(reinterpret_cast<const float4*>(in + (long long)f * per_plane));
    }
  } else {
    const int tube = threadIdx.x % T;
    if (tube < Tb) {
      const float2* in = job.in + spec_off(t0 + tube);
      for (int f = threadIdx.x / T; f < P; f += kThreads / T) buf0[f * T + tube] = __ldg(in + (long long)f * per_plane);
    }
  }
  __syncthreads();
  const float2* X = stages<P, 0, 1, true, true, false>(buf0, buf1, Tb, tw);  // frequency-major input

  // contiguous store; consecutive lanes read consecutive elements of a tube
  const float scale = 1.0f / (float)P;
  float2* dst = job.out + t0 * P;
  for (int i = threadIdx.x; i < Tb * P; i += kThreads) {
    const int tube = i / P;
    const float2 a = X[tube * PP + (i - tube * P)];
    dst[i] = make_float2(a.x * scale, a.y * scale);
  }
}

template <int P, int FMT>
__global__ void __launch_bounds__(kThreads, min_blocks<P, false>()) fft_fwd_fixed(FftFwdJob job0, FftFwdJob job1, int njobs,
                                                          const float2* __restrict__ tw) {
  extern __shared__ float4 smem_f4[];
  if (threadIdx.x == 0) grid_dep_launch();  // the products may be scheduled once every CTA got here
  int b = blockIdx.x;
  const bool second = njobs > 1 && b >= job0.nblocks;
  if (second) b -= job0.nblocks;
  fixed_fwd_body<P, FMT>(second ? job1 : job0, b, tw, reinterpret_cast<float2*>(smem_f4));
}

template <int P>
__global__ void __launch_bounds__(kThreads, min_blocks<P, true>()) fft_inv_fixed(FftInvJob job0, FftInvJob job1, int njobs,
                                                          const float2* __restrict__ tw) {
  extern __shared__ float4 smem_f4[];
  grid_dep_wait();  // C's spectra come from the previous kernel (launched with PDL)
  int b = blockIdx.x;
  const bool second = njobs > 1 && b >= job0.nblocks;
  if (second) b -= job0.nblocks;
  fixed_inv_body<P>(second ? job1 : job0, b, tw, reinterpret_cast<float2*>(smem_f4));
}

// ---------------------------------------------------------------------------
// Grouped transforms for batches of products with mixed (rows, cols, p).  The
// plan orders the jobs by tube length, so the CTAs of one p form a contiguous
// range of the global block space; each range is one launch of the body
// specialised for that p (P = 0: the runtime-radix body), which keeps each
// launch at its own register count and occupancy.  A CTA finds its job with
// one table load (job_of_block).  Tensor pointers come from a per-call device
// table ptrs[3 * product + {0: A, 1: B, 2: C}].
// ---------------------------------------------------------------------------

template <int P, int FMT>
__global__ void __launch_bounds__(kThreads, min_blocks<P, false>()) fft_fwd_grouped(const FftGroupJob* __restrict__ jobs,
                                                            const int* __restrict__ job_of_block, long long block0,
                                                            const float2* const* __restrict__ ptrs, char* ws,
                                                            const float2* __restrict__ tw_all) {
  extern __shared__ float4 smem_f4[];
  float2* smem = reinterpret_cast<float2*>(smem_f4);
  const long long b = block0 + blockIdx.x;
  const FftGroupJob& J = jobs[__ldg(job_of_block + b)];
  FftFwdJob job;
  job.in = ptrs[3 * J.prod + J.which];
  job.out = ws + J.spec_off;
  job.rows = J.rows;
  job.cols = J.cols;
  job.ld = J.ld;
  job.nblocks = 0;
  const long long lb = b - J.block_begin;
  const float2* tw = tw_all + J.tw_off;
  if constexpr (P == 0) generic_fwd_body<FMT>(job, lb, J.rp, J.T, tw, smem);
  else fixed_fwd_body<P, FMT>(job, lb, tw, smem);
}

template <int P>
__global__ void __launch_bounds__(kThreads, min_blocks<P, true>()) fft_inv_grouped(const FftGroupJob* __restrict__ jobs,
                                                            const int* __restrict__ job_of_block, long long block0,
                                                            const float2* const* __restrict__ ptrs, char* ws,
                                                            const float2* __restrict__ tw_all) {
  extern __shared__ float4 smem_f4[];
  float2* smem = reinterpret_cast<float2*>(smem_f4);
  const long long b = block0 + blockIdx.x;
  const FftGroupJob& J = jobs[__ldg(job_of_block + b)];
  FftInvJob job;
  job.in = reinterpret_cast<const float2*>(ws + J.spec_off);
  job.out = const_cast<float2*>(ptrs[3 * J.prod + J.which]);
  job.rows = J.rows;
  job.cols = J.cols;
  job.nblocks = 0;
  const long long lb = b - J.block_begin;
  const float2* tw = tw_all + J.tw_off;
  if constexpr (P == 0) generic_inv_body(job, lb, J.rp, J.T, tw, smem);
  else fixed_inv_body<P>(job, lb, tw, smem);
}

template <int P, int FMT>
cudaError_t fwd_grouped_launch(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0,
                               long long nblocks, const float2* const* d_ptrs, char* ws, const float2* d_tw,
                               size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(fft_fwd_grouped<P, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fft_fwd_grouped<P, FMT><<<(unsigned)nblocks, kThreads, smem, st>>>(d_jobs, d_job_of_block, block0, d_ptrs, ws, d_tw);
  return cudaGetLastError();
}

template <int P>
cudaError_t fwd_grouped_fmt(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0, long long nblocks,
                            int fmt, const float2* const* d_ptrs, char* ws, const float2* d_tw, size_t smem,
                            cudaStream_t st) {
  switch (fmt) {
    case FMT_C32: return fwd_grouped_launch<P, FMT_C32>(d_jobs, d_job_of_block, block0, nblocks, d_ptrs, ws, d_tw, smem, st);
    case FMT_BF16X3: return fwd_grouped_launch<P, FMT_BF16X3>(d_jobs, d_job_of_block, block0, nblocks, d_ptrs, ws, d_tw, smem, st);
    case FMT_BF16: return fwd_grouped_launch<P, FMT_BF16>(d_jobs, d_job_of_block, block0, nblocks, d_ptrs, ws, d_tw, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int P>
cudaError_t inv_grouped_launch(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0,
                               long long nblocks, const float2* const* d_ptrs, char* ws, const float2* d_tw,
                               size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(fft_inv_grouped<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fft_inv_grouped<P><<<(unsigned)nblocks, kThreads, smem, st>>>(d_jobs, d_job_of_block, block0, d_ptrs, ws, d_tw);
  return cudaGetLastError();
}

template <int P, int FMT>
cudaError_t fwd_launch(const FftFwdJob* jobs, int njobs, const float2* tw, cudaStream_t st) {
  constexpr size_t smem = smem_for<P, false>();
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = ensure_smem_attr(attr_set, fft_fwd_fixed<P, FMT>, smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  for (int i = 0; i < njobs; ++i) nb += jobs[i].nblocks;
  if (nb == 0) return cudaSuccess;
  fft_fwd_fixed<P, FMT><<<nb, kThreads, smem, st>>>(jobs[0], njobs > 1 ? jobs[1] : jobs[0], njobs, tw);
  return cudaGetLastError();
}

template <int P>
cudaError_t fwd_fmt(const FftFwdJob* jobs, int njobs, int fmt, const float2* tw, cudaStream_t st) {
  switch (fmt) {
    case FMT_C32: return fwd_launch<P, FMT_C32>(jobs, njobs, tw, st);
    case FMT_BF16X3: return fwd_launch<P, FMT_BF16X3>(jobs, njobs, tw, st);
    case FMT_BF16: return fwd_launch<P, FMT_BF16>(jobs, njobs, tw, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int P>
cudaError_t inv_launch(const FftInvJob* jobs, int njobs, const float2* tw, cudaStream_t st) {
  constexpr size_t smem = smem_for<P, true>();
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = ensure_smem_attr(attr_set, fft_inv_fixed<P>, smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  for (int i = 0; i < njobs; ++i) nb += jobs[i].nblocks;
  if (nb == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, fft_inv_fixed<P>, jobs[0], njobs > 1 ? jobs[1] : jobs[0], njobs, tw);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

size_t fft_fixed_smem(int p, bool inv) {
#define QTP_SMEM_CASE(P) \
  case P: return inv ? smem_for<P, true>() : smem_for<P, false>();
  switch (p) {
    QTP_SMEM_CASE(8) QTP_SMEM_CASE(12) QTP_SMEM_CASE(16) QTP_SMEM_CASE(31)
    QTP_SMEM_CASE(32) QTP_SMEM_CASE(64) QTP_SMEM_CASE(100) QTP_SMEM_CASE(128)
    QTP_SMEM_CASE(256) QTP_SMEM_CASE(512) QTP_SMEM_CASE(1024)
    default: return 0;
  }
#undef QTP_SMEM_CASE
}

cudaError_t launch_fft_fwd_grouped(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0,
                                   long long nblocks, int p, int fmt, const float2* const* d_ptrs, char* ws,
                                   const float2* d_tw, size_t smem, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
#define QTP_FWD_GROUPED_CASE(P) \
  case P: return fwd_grouped_fmt<P>(d_jobs, d_job_of_block, block0, nblocks, fmt, d_ptrs, ws, d_tw, smem, st);
  switch (p) {
    QTP_FWD_GROUPED_CASE(8) QTP_FWD_GROUPED_CASE(12) QTP_FWD_GROUPED_CASE(16) QTP_FWD_GROUPED_CASE(31)
    QTP_FWD_GROUPED_CASE(32) QTP_FWD_GROUPED_CASE(64) QTP_FWD_GROUPED_CASE(100) QTP_FWD_GROUPED_CASE(128)
    QTP_FWD_GROUPED_CASE(256) QTP_FWD_GROUPED_CASE(512) QTP_FWD_GROUPED_CASE(1024)
    default: return fwd_grouped_fmt<0>(d_jobs, d_job_of_block, block0, nblocks, fmt, d_ptrs, ws, d_tw, smem, st);
  }
#undef QTP_FWD_GROUPED_CASE
}

cudaError_t launch_fft_inv_grouped(const FftGroupJob* d_jobs, const int* d_job_of_block, long long block0,
                                   long long nblocks, int p, const float2* const* d_ptrs, char* ws,
                                   const float2* d_tw, size_t smem, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
#define QTP_INV_GROUPED_CASE(P) \
  case P: return inv_grouped_launch<P>(d_jobs, d_job_of_block, block0, nblocks, d_ptrs, ws, d_tw, smem, st);
  switch (p) {
    QTP_INV_GROUPED_CASE(8) QTP_INV_GROUPED_CASE(12) QTP_INV_GROUPED_CASE(16) QTP_INV_GROUPED_CASE(31)
    QTP_INV_GROUPED_CASE(32) QTP_INV_GROUPED_CASE(64) QTP_INV_GROUPED_CASE(100) QTP_INV_GROUPED_CASE(128)
    QTP_INV_GROUPED_CASE(256) QTP_INV_GROUPED_CASE(512) QTP_INV_GROUPED_CASE(1024)
    default: return inv_grouped_launch<0>(d_jobs, d_job_of_block, block0, nblocks, d_ptrs, ws, d_tw, smem, st);
  }
#undef QTP_INV_GROUPED_CASE
}

int fft_fwd_run_cols(int p, int fmt, int cols) {
  const bool two_pass = fft_fixed_tubes(p, false) != 0 && split_of(p, false).r1 != 0;
  return two_pass && fmt != FMT_C32 && (cols & 1) ? cols + 1 : cols;
}

int fft_fixed_tubes(int p, bool inv) {
  switch (p) {
    case 8: case 12: case 16: case 31: case 32: case 64: case 100: case 128: case 256: case 512: case 1024:
      return tubes_for(p, inv);
    default: return 0;
  }
}

cudaError_t launch_fft_fwd_fixed(const FftFwdJob* jobs, int njobs, int fmt, int p, const float2* tw,
                                 cudaStream_t st) {
  switch (p) {
    case 8: return fwd_fmt<8>(jobs, njobs, fmt, tw, st);
    case 12: return fwd_fmt<12>(jobs, njobs, fmt, tw, st);
    case 16: return fwd_fmt<16>(jobs, njobs, fmt, tw, st);
    case 31: return fwd_fmt<31>(jobs, njobs, fmt, tw, st);
    case 32: return fwd_fmt<32>(jobs, njobs, fmt, tw, st);
    case 64: return fwd_fmt<64>(jobs, njobs, fmt, tw, st);
    case 100: return fwd_fmt<100>(jobs, njobs, fmt, tw, st);
    case 128: return fwd_fmt<128>(jobs, njobs, fmt, tw, st);
    case 256: return fwd_fmt<256>(jobs, njobs, fmt, tw, st);
    case 512: return fwd_fmt<512>(jobs, njobs, fmt, tw, st);
    case 1024: return fwd_fmt<1024>(jobs, njobs, fmt, tw, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_fft_inv_fixed(const FftInvJob* jobs, int njobs, int p, const float2* tw, cudaStream_t st) {
  switch (p) {
    case 8: return inv_launch<8>(jobs, njobs, tw, st);
    case 12: return inv_launch<12>(jobs, njobs, tw, st);
    case 16: return inv_launch<16>(jobs, njobs, tw, st);
    case 31: return inv_launch<31>(jobs, njobs, tw, st);
    case 32: return inv_launch<32>(jobs, njobs, tw, st);
    case 64: return inv_launch<64>(jobs, njobs, tw, st);
    case 100: return inv_launch<100>(jobs, njobs, tw, st);
    case 128: return inv_launch<128>(jobs, njobs, tw, st);
    case 256: return inv_launch<256>(jobs, njobs, tw, st);
    case 512: return inv_launch<512>(jobs, njobs, tw, st);
    case 1024: return inv_launch<1024>(jobs, njobs, tw, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace qtp
