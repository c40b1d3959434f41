// Two-pass (one shared-memory exchange) tube transforms of a compile-time
// length P = R1 R2, shared by the one-kernel transforms (qtp_fft_fixed.cu)
// and the long-tube transforms (qtp_fft_split.cu), which run them as the
// inner pass of a length N1 P transform (LONG = true, see LongMap).
// Internal to libqtp.
#pragma once

#include <cuda_bf16.h>

#include "qtp_fft_common.cuh"
#include "qtp_internal.h"

namespace qtp {
namespace {

using namespace fftdev;

constexpr int kThreads = 256;

// Two-pass transforms (see fs_fwd_body) take p = R1 R2 with both factors in
// registers; p without such a split runs the Stockham stages below.  The
// forward p = 100 takes 20 x 5 (fewer pass-2 registers; measured 7.9 ms on
// the batch's p = 100 products against 9.0 ms for the stages, 9.8 for 10 x 10).
struct Split {
  int r1, r2;
};
__host__ __device__ constexpr Split split_of(int p, bool inv) {
  switch (p) {
    case 8: return Split{4, 2};
    case 12: return Split{4, 3};
    case 16: return Split{4, 4};
    case 32: return Split{8, 4};
    case 64: return Split{8, 8};
    case 100: return inv ? Split{10, 10} : Split{20, 5};
    case 128: return Split{16, 8};
    case 256: return Split{16, 16};
    case 512: return Split{32, 16};
    case 1024: return Split{32, 32};
    default: return Split{0, 0};
  }
}

// Tubes per CTA: a power of two, at most kThreads, so that in the strided
// loops over (frequency, tube) every thread keeps one tube (or tube pair) and
// computes its address once.
//   Two-pass: about QTP_FS_ELEMS = 4096 complex per CTA (32 KB of exchange
//   buffer), at least 32 tubes (the frequency-major stores write runs of T
//   tubes) as long as the buffer stays within 64 KB (p = 256, 512, 1024:
//   32, 16, 8 tubes).  The forward one-kernel form takes about
//   QTP_FS_ELEMS_FWD = 6400, which changes p = 100 alone (64 tubes, 50 KB:
//   the batch's p = 100 forward transforms 1026 -> 927 us on 512 products;
//   the inverse and the long form's inner p = 100 measured slower with 64).
//   Stockham: about QTP_FFT_ELEMS complex per buffer (2304: ~34 KB per CTA,
//   up to six resident CTAs per SM; measured faster than 4608); the forward
//   transform keeps at least 32 tubes, the inverse, whose stores are
//   contiguous tubes, takes the smaller count for occupancy.
#ifndef QTP_FFT_ELEMS
#define QTP_FFT_ELEMS 2304
#endif
#ifndef QTP_FS_ELEMS
#define QTP_FS_ELEMS 4096
#endif
#ifndef QTP_FS_ELEMS_FWD
#define QTP_FS_ELEMS_FWD 6400
#endif
// Resident CTAs per SM the transform kernels are compiled for (caps their
// registers at 65536 / (kThreads * resident CTAs)): the two-pass transforms
// are latency-bound.  Forward: three (85 registers; video forward 80 -> 66 us
// against the spill-free count; four measured slower).  Inverse: four (64
// registers; the batch's inverse transforms 9.4 -> 8.7 ms).
#ifndef QTP_FFT_MINB
#define QTP_FFT_MINB 3
#endif
#ifndef QTP_FFT_MINB_INV
#define QTP_FFT_MINB_INV 4
#endif
// Tube lengths of 256 and up (64 KB CTAs, DFTs of 16 or 32 per thread) take
// two CTAs per SM: 128 registers, no spills.
template <int P, bool INV>
__host__ __device__ constexpr int min_blocks() {
  return P >= 256 ? 2 : (INV ? QTP_FFT_MINB_INV : QTP_FFT_MINB);
}

// lng: the inner pass of a long transform (qtp_fft_split.cu).
__host__ __device__ constexpr int tubes_for(int p, bool inv, bool lng = false) {
  int lim = 0;
  if (split_of(p, inv).r1 != 0) {
    // at least 32 tubes while the buffer stays within 64 KB (8 192 complex)
    lim = (inv || lng ? QTP_FS_ELEMS : QTP_FS_ELEMS_FWD) / p;
    const int cap = 8192 / p < 32 ? 8192 / p : 32;
    if (lim < cap) lim = cap;
  } else {
    lim = QTP_FFT_ELEMS / (p | 1);
    if (!inv && lim < 32 && p <= 128) lim = 32;
  }
  if (lim > 256) lim = 256;
  int t = 2;
  while (2 * t <= lim) t *= 2;
  return t;
}

// Row pitch (complex) of the two-pass exchange buffer: T plus the even pad
// that minimises shared-memory bank conflicts of its scalar accesses, thread
// idx touching row (idx % A) + const at column idx / A (A = R2: forward
// pass-1 writes, inverse pass-2 reads).  Cost: per half warp, the largest
// number of 8-byte accesses on one bank pair.
__host__ __device__ constexpr int fs_conflicts(int A, int S, int tp) {
  int total = 0;
  for (int w = 0; w < 8; ++w)
    for (int h = 0; h < 2; ++h) {
      int cnt[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      int mx = 0;
      for (int l = 0; l < 16; ++l) {
        const int idx = 32 * w + 16 * h + l;
        const int b = ((idx % A) * S * tp + idx / A) % 16;
        ++cnt[b];
        if (cnt[b] > mx) mx = cnt[b];
      }
      total += mx;
    }
  return total;
}
__host__ __device__ constexpr int fs_pitch(int p, bool inv, bool lng = false) {
  const Split sp = split_of(p, inv);
  const int T = tubes_for(p, inv, lng);
  const int A = sp.r2, S = 1;
  int best = T, cost = fs_conflicts(A, S, T);
  for (int pad = 2; pad < 32; pad += 2) {
    const int c = fs_conflicts(A, S, T + pad);
    if (c < cost) {
      cost = c;
      best = T + pad;
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// Two-pass transforms for p = R1 R2 (Cooley-Tukey with a single exchange).
// Forward, tube sample n = R2 n1 + n2, frequency f = k1 + R1 k2, w = w_p:
//   X[k1 + R1 k2] = sum_n2 w_R2^(n2 k2) w^(n2 k1) sum_n1 x[R2 n1 + n2] w_R1^(n1 k1)
//   pass 1: thread (tube, n2) loads its R1 samples from HBM, DFT-R1, twiddle
//           w^(n2 k1), writes Y[k1][n2][tube] to shared memory;
//   pass 2: thread (tube pair, k1) reads Y[k1][.][tube pair], DFT-R2, stores
//           frequencies k1 + R1 k2 to the frequency-major spectra.
// Inverse, f = f1 + F1 f2, n = n1 + F2 n2 (F1 = R1, F2 = R2), conjugate roots:
//   x[n1 + F2 n2] = 1/p sum_f1 w_F1^(n2 f1) w^(n1 f1) sum_f2 X[f1 + F1 f2] w_F2^(n1 f2)
//   pass 1: thread (tube pair, f1) gathers X[f1 + F1 f2], DFT-F2, twiddle,
//           writes Z[f1][n1][tube pair];
//   pass 2: thread (tube, n1) reads Z[.][n1][tube], DFT-F1, stores the
//           samples n1 + F2 n2.
// Every sample crosses shared memory once; both HBM sides are coalesced
// (pass-1 loads / pass-2 stores of runs of R2 samples per tube; frequency-
// major runs of T / 2 tube pairs).
// ---------------------------------------------------------------------------

// The transform of length P as the inner pass of a long one of length
// p_total = N1 P (qtp_fft_split.cu): the forward writes its frequency f' at
// the long spectrum's f_add + f_mul f' (f_mul = N1, f_add = k1) with planes
// and parts p_total frequencies apart; the inverse gathers those frequencies
// and multiplies its output sample t by w_p^(-f_add t) (tw_p: the length-p
// table).  Unused when LONG is false.
struct LongMap {
  int f_mul, f_add, p_total;
  const float2* tw_p;
};

template <int P, int FMT, bool LONG = false>
__device__ __forceinline__ void fs_fwd_body(const FftFwdJob& job, long long b, const float2* __restrict__ tw,
                                            float2* smem, const LongMap& L = LongMap{1, 0, P, nullptr}) {
  constexpr int R1 = split_of(P, false).r1, R2 = split_of(P, false).r2;
  constexpr int T = tubes_for(P, false, LONG);
  constexpr int TP = fs_pitch(P, false, LONG);
  constexpr int NPARTS = FMT == FMT_BF16X3 ? 4 : (FMT == FMT_BF16 ? 2 : 1);
  static_assert(R1 * R2 == P && kThreads % T == 0, "two-pass split");

  // Run space: the tubes row by row, each row padded to an even count for the
  // bf16 spectra (a phantom tube after an odd row: zero input, and its stores
  // land in the spectra's row padding, ld >= cols + 1), so that pass 2 always
  // stores tube pairs.  fft_fwd_run_cols gives the host the same count.
  const int cp = (FMT != FMT_C32 && (job.cols & 1)) ? job.cols + 1 : job.cols;
  const long long per_plane = (long long)job.rows * cp;
  const long long ntubes = 2 * per_plane;
  const long long t0 = b * T;
  if (t0 >= ntubes) return;
  const int Tb = (int)min((long long)T, ntubes - t0);

  // pass 1: every load of the thread's NI items is issued before the first
  // DFT, to keep more bytes in flight
  constexpr int NI = (T * R2 + kThreads - 1) / kThreads;
  float2 v[NI][R1];
  if (cp == job.cols) {
    // no phantom tubes: the run space is the tensor's, tubes contiguous
    const float2* src = job.in + t0 * P;
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      const int idx = threadIdx.x + it * kThreads;
      const int tube = idx / R2;
      if (idx < T * R2 && tube < Tb) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[it][n1] = __ldg(src + tube * P + R2 * n1 + idx % R2);
      }
    }
  } else {
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      const int idx = threadIdx.x + it * kThreads;
      const int tube = idx / R2;
      bool real = idx < T * R2 && tube < Tb;
      const float2* src = job.in;
      if (real) {
        const long long t = t0 + tube;
        const int plane = t >= per_plane;
        const long long rem = t - (plane ? per_plane : 0);
        long long row;
        int col;
        if (per_plane <= 0x7fffffffLL) {
          const unsigned r32 = (unsigned)rem, row32 = r32 / (unsigned)cp;
          row = row32;
          col = (int)(r32 - row32 * (unsigned)cp);
        } else {
          row = rem / cp;
          col = (int)(rem - row * cp);
        }
        real = col < job.cols;  // a phantom tube reads nothing and transforms zeros
        src = job.in + (((long long)plane * job.rows + row) * job.cols + col) * P;
      }
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[it][n1] = real ? __ldg(src + R2 * n1 + idx % R2) : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    const int idx = threadIdx.x + it * kThreads;
    const int n2 = idx % R2;
    const int tube = idx / R2;
    if (idx >= T * R2 || tube >= Tb) continue;
    Dft<R1, false>::run(v[it]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 y = (k1 == 0 || n2 == 0) ? v[it][k1] : cmul(v[it][k1], twid<false>(tw, n2 * k1));
      smem[(k1 * R2 + n2) * TP + tube] = y;
    }
  }
  __syncthreads();

  // pass 2
  const long long ld = job.ld;
  const long long slab = (long long)job.rows * ld;  // one (plane, part, f) slab
  const long long nfreq = LONG ? L.p_total : P;     // frequencies of the spectrum written
  const long long part = nfreq * slab;
  auto spec_off = [&](long long t) {  // [plane][part 0][f 0][row][col] of run tube t
    const long long plane = t / per_plane;
    const long long rem = t - plane * per_plane;
    const long long row = rem / cp;
    return plane * NPARTS * nfreq * slab + row * ld + (rem - row * cp);
  };
  auto freq = [&](int f) { return LONG ? L.f_add + L.f_mul * f : f; };
  // Tube pairs (4-byte bf16 pair stores) when the run rows are even and two
  // tubes' R2 values fit in registers.
  constexpr bool kPairs = R2 <= 10;
  if (kPairs && (cp & 1) == 0) {
    // tube pairs share a row: 16-byte / 4-byte stores
    constexpr int TH = T / 2;
    const int tube = 2 * (threadIdx.x % TH);
    if (tube >= Tb) return;
    const long long o0 = spec_off(t0 + tube);
    for (int k1 = threadIdx.x / TH; k1 < R1; k1 += kThreads / TH) {
      float2 a[R2], c[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) {
        const float4 y = *reinterpret_cast<const float4*>(smem + (k1 * R2 + n2) * TP + tube);
        a[n2] = make_float2(y.x, y.y);
        c[n2] = make_float2(y.z, y.w);
      }
      Dft<R2, false>::run(a);
      Dft<R2, false>::run(c);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const long long o = o0 + (long long)freq(k1 + R1 * k2) * slab;
        const float2 v0 = a[k2], v1 = c[k2];
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
    }
  } else {
    const int tube = threadIdx.x % T;
    if (tube >= Tb) return;
    const long long o0 = spec_off(t0 + tube);
    for (int k1 = threadIdx.x / T; k1 < R1; k1 += kThreads / T) {
      float2 a[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) a[n2] = smem[(k1 * R2 + n2) * TP + tube];
      Dft<R2, false>::run(a);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const long long o = o0 + (long long)freq(k1 + R1 * k2) * slab;
        const float2 v = a[k2];
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
}

template <int P, bool LONG = false>
__device__ __forceinline__ void fs_inv_body(const FftInvJob& job, long long b, const float2* __restrict__ tw,
                                            float2* smem, const LongMap& L = LongMap{1, 0, P, nullptr}) {
  constexpr int F1 = split_of(P, true).r1, F2 = split_of(P, true).r2;
  constexpr int T = tubes_for(P, true, LONG);
  constexpr int TP = fs_pitch(P, true, LONG);
  static_assert(F1 * F2 == P && kThreads % T == 0, "two-pass split");

  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = b * T;
  if (t0 >= ntubes) return;
  const int Tb = (int)min((long long)T, ntubes - t0);
  const long long nfreq = LONG ? L.p_total : P;  // frequencies of the spectrum read
  auto spec_off = [&](long long t) {  // [plane][f 0][row][col] of tube t
    const long long plane = t / per_plane;
    return plane * nfreq * per_plane + (t - plane * per_plane);
  };
  auto freq = [&](int f) { return LONG ? L.f_add + L.f_mul * f : f; };

  // pass 1 (tube pairs: 16-byte loads, when two tubes' F2 values fit in registers)
  constexpr bool kPairs = F2 <= 10;
  if (kPairs && (job.cols & 1) == 0) {
    constexpr int TH = T / 2;
    const int tube = 2 * (threadIdx.x % TH);
    if (tube < Tb) {
      const float2* in = job.in + spec_off(t0 + tube);
      for (int f1 = threadIdx.x / TH; f1 < F1; f1 += kThreads / TH) {
        float2 a[F2], c[F2];
#pragma unroll
        for (int f2 = 0; f2 < F2; ++f2) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(in + (long long)freq(f1 + F1 * f2) * per_plane));
          a[f2] = make_float2(x.x, x.y);
          c[f2] = make_float2(x.z, x.w);
        }
        Dft<F2, true>::run(a);
        Dft<F2, true>::run(c);
#pragma unroll
        for (int n1 = 0; n1 < F2; ++n1) {
          float2 za = a[n1], zc = c[n1];
          if (n1 > 0 && f1 > 0) {
            const float2 w = twid<true>(tw, n1 * f1);
            za = cmul(za, w);
            zc = cmul(zc, w);
          }
          *reinterpret_cast<float4*>(smem + (f1 * F2 + n1) * TP + tube) = make_float4(za.x, za.y, zc.x, zc.y);
        }
      }
    }
  } else {
    const int tube = threadIdx.x % T;
    if (tube < Tb) {
      const float2* in = job.in + spec_off(t0 + tube);
      for (int f1 = threadIdx.x / T; f1 < F1; f1 += kThreads / T) {
        float2 a[F2];
#pragma unroll
        for (int f2 = 0; f2 < F2; ++f2) a[f2] = __ldg(in + (long long)freq(f1 + F1 * f2) * per_plane);
        Dft<F2, true>::run(a);
#pragma unroll
        for (int n1 = 0; n1 < F2; ++n1)
          smem[(f1 * F2 + n1) * TP + tube] = (n1 > 0 && f1 > 0) ? cmul(a[n1], twid<true>(tw, n1 * f1)) : a[n1];
      }
    }
  }
  __syncthreads();

  // pass 2
  const float scale = 1.0f / (float)P;
  float2* dst = job.out + t0 * P;
  for (int idx = threadIdx.x; idx < T * F2; idx += kThreads) {
    const int n1 = idx % F2;
    const int tube = idx / F2;
    if (tube >= Tb) continue;
    float2 v[F1];
#pragma unroll
    for (int f1 = 0; f1 < F1; ++f1) v[f1] = smem[(f1 * F2 + n1) * TP + tube];
    Dft<F1, true>::run(v);
#pragma unroll
    for (int n2 = 0; n2 < F1; ++n2) {
      float2 x = v[n2];
      if (LONG && L.f_add > 0) x = cmul(x, twid<true>(L.tw_p, L.f_add * (n1 + F2 * n2)));
      dst[tube * P + n1 + F2 * n2] = make_float2(x.x * scale, x.y * scale);
    }
  }
}

}  // namespace
}  // namespace qtp
