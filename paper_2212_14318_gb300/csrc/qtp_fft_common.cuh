// Device helpers shared by the tube-FFT kernels (internal to libqtp).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "qtp_internal.h"

namespace qtp {
namespace fftdev {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// w^e for the forward (INV = false) or inverse (conjugate) transform.
template <bool INV>
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int e) {
  float2 w = __ldg(tw + e);
  if (INV) w.y = -w.y;
  return w;
}

// Multiply by the fourth root of unity omega_4 = -i (forward) or +i (inverse).
template <bool INV>
__device__ __forceinline__ float2 mul_w4(float2 v) {
  return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 a0 = cadd(v0, v2), a1 = csub(v0, v2);
  float2 b0 = cadd(v1, v3), b1 = mul_w4<INV>(csub(v1, v3));
  v0 = cadd(a0, b0);
  v2 = csub(a0, b0);
  v1 = cadd(a1, b1);
  v3 = csub(a1, b1);
}

// cos and sin of 2 pi k / n in double, usable as compile-time constants: the
// angle is reduced to [-pi, pi] and summed by its Taylor series up to x^61
// (within 1e-13 of the exact value, far below the float rounding the kernels
// apply to it).
constexpr double kTwoPi = 6.283185307179586476925286766559;
__host__ __device__ constexpr double turn_angle(int k, int n) {
  k %= n;
  if (2 * k > n) k -= n;
  return kTwoPi * (double)k / (double)n;
}
__host__ __device__ constexpr double cos_turn(int k, int n) {
  const double x = turn_angle(k, n);
  double t = 1.0, sum = 1.0;
  for (int i = 1; i <= 30; ++i) {
    t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += t;
  }
  return sum;
}
__host__ __device__ constexpr double sin_turn(int k, int n) {
  const double x = turn_angle(k, n);
  double t = x, sum = x;
  for (int i = 1; i <= 30; ++i) {
    t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += t;
  }
  return sum;
}

// Calls f(integral_constant<int, I>) for I = B .. E-1, so that f's body sees
// I as a constant expression.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Length-R DFT in registers: X[u] = sum_r x_r w^(r u), w = e^(-2 pi i/R)
// (conjugate for the inverse), with every root of unity a compile-time
// constant.  R = 2, 4, 8 have their own specialisations below.
//
// R odd: pairing r with R - r,
//   X[u]     = A_u - i B_u,   X[R - u] = A_u + i B_u   (forward; signs of B
//   swap for the inverse), A_u = x_0 + sum_r (x_r + x_{R-r}) cos(2 pi r u / R),
//   B_u = sum_r (x_r - x_{R-r}) sin(2 pi r u / R),  r = 1 .. (R-1)/2,
// a quarter of the multiplies of the plain sum.
// R even: even/odd split, X[u] = E[u] + w^u O[u], X[u + R/2] = E[u] - w^u O[u]
// with E, O the length-R/2 DFTs of the even and odd samples.
template <int R, bool INV>
struct Dft {
  static_assert(R >= 3, "radix");
  __device__ __forceinline__ static void run(float2 (&v)[R], const float2* tw = nullptr, int p = 0) {
    if constexpr (R % 2 == 1) {
      constexpr int H = (R - 1) / 2;
      float2 sp[H], dm[H];
      const float2 x0 = v[0];
      float2 dc = x0;
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        sp[r - 1] = cadd(v[r], v[R - r]);
        dm[r - 1] = csub(v[r], v[R - r]);
        dc = cadd(dc, sp[r - 1]);
      }
      v[0] = dc;
      static_for<1, H + 1>([&](auto uc) {
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
        // -i B = (B.y, -B.x)
        const float2 mib = make_float2(bsum.y, -bsum.x);
        v[u] = INV ? csub(a, mib) : cadd(a, mib);
        v[R - u] = INV ? cadd(a, mib) : csub(a, mib);
      });
    } else {
      constexpr int Q = R / 2;
      float2 e[Q], o[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
      }
      Dft<Q, INV>::run(e);
      Dft<Q, INV>::run(o);
      static_for<0, Q>([&](auto uc) {
        constexpr int u = decltype(uc)::value;
        constexpr float c = (float)cos_turn(u, R);
        constexpr float sn = (float)sin_turn(u, R);
        const float2 w = make_float2(c, INV ? sn : -sn);
        const float2 t = u == 0 ? o[u] : cmul(o[u], w);
        v[u] = cadd(e[u], t);
        v[u + Q] = csub(e[u], t);
      });
    }
  }
};

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[2], const float2* = nullptr, int = 0) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[4], const float2* = nullptr, int = 0) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  }
};

template <bool INV>
struct Dft<8, INV> {
  // Even/odd split: X[u] = E[u] + omega_8^u O[u], X[u+4] = E[u] - omega_8^u O[u].
  __device__ __forceinline__ static void run(float2 (&v)[8], const float2* = nullptr, int = 0) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    constexpr float h = (float)cos_turn(1, 8);  // sqrt(1/2)
    const float2 w1 = make_float2(h, INV ? h : -h);
    const float2 w3 = make_float2(-h, INV ? h : -h);
    o1 = cmul(o1, w1);
    o2 = mul_w4<INV>(o2);
    o3 = cmul(o3, w3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  }
};

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}


// One radix-R Stockham stage for butterfly j of one tube: the inputs sit at
// stride p/R, are twiddled by w_{Ns R}^(r (j mod Ns)), transformed, and written
// to (j / Ns) Ns R + (j mod Ns) + r Ns.  Ns is the length already transformed.
// tw holds w_p^e at entry e * tws (tws > 1: a sub-length p of a longer
// transform whose table is read with stride tws).
template <int R, bool INV>
__device__ __forceinline__ void butterfly(const float2* __restrict__ in, float2* __restrict__ out, int j,
                                          int Ns, int p, const float2* __restrict__ tw, int tws = 1) {
  const int stride = p / R;
  const int k = j % Ns;
  const int twstep = p / (Ns * R) * tws;
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
                                                  const float2* __restrict__ tw, int tws = 1) {
  const int stride = p / R;
  const int k = j % Ns;
  const int twstep = p / (Ns * R) * tws;
  const int base = (j / Ns) * Ns * R + k;
  for (int u = 0; u < R; ++u) {
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < R; ++r) {
      float2 x = in[j + r * stride];
      if (r > 0 && k > 0) x = cmul(x, twid<INV>(tw, r * k * twstep));
      const int e = ((r * u) % R) * stride * tws;
      acc = cadd(acc, e ? cmul(x, twid<INV>(tw, e)) : x);
    }
    out[base + u * Ns] = acc;
  }
}

// All stages over T tubes held at tube stride P in buf0.  Returns the buffer
// that holds the result (natural order).  tws: stride of the twiddle table
// (see butterfly).
template <bool INV>
__device__ inline float2* run_stages(float2* buf0, float2* buf1, int T, int P, const RadixPlan& rp,
                              const float2* __restrict__ tw, int tws = 1) {
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
        case 2: butterfly<2, INV>(ti, to, j, Ns, p, tw, tws); break;
        case 3: butterfly<3, INV>(ti, to, j, Ns, p, tw, tws); break;
        case 4: butterfly<4, INV>(ti, to, j, Ns, p, tw, tws); break;
        case 5: butterfly<5, INV>(ti, to, j, Ns, p, tw, tws); break;
        case 7: butterfly<7, INV>(ti, to, j, Ns, p, tw, tws); break;
        case 8: butterfly<8, INV>(ti, to, j, Ns, p, tw, tws); break;
        default: butterfly_generic<INV>(ti, to, j, Ns, R, p, tw, tws); break;
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

// Forward transform of the b-th run of T tubes of one tensor (runtime radix plan).
template <int FMT>
__device__ void generic_fwd_body(const FftFwdJob& job, long long b, const RadixPlan& rp, int T,
                                 const float2* __restrict__ tw, float2* smem) {
  const int p = rp.p;
  const int P = p | 1;
  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = b * T;
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

// Inverse transform (scale 1/p) of the b-th run of T tubes of one tensor.
__device__ inline void generic_inv_body(const FftInvJob& job, long long b, const RadixPlan& rp, int T,
                                        const float2* __restrict__ tw, float2* smem) {
  const int p = rp.p;
  const int P = p | 1;
  const long long per_plane = (long long)job.rows * job.cols;
  const long long ntubes = 2 * per_plane;
  const long long t0 = b * T;
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

}  // namespace fftdev
}  // namespace qtp
