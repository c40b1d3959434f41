// Device helpers shared by the tube-FFT kernels (internal to libqtp).
#pragma once

#include <cuda_bf16.h>

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

// Length-R DFT in registers.  Generic version: direct sum with roots of unity
// read from the length-p table (omega_R^e = w^(e p / R)).
template <int R, bool INV>
struct Dft {
  __device__ __forceinline__ static void run(float2 (&v)[R], const float2* __restrict__ tw, int p) {
    float2 w[R];
    const int step = p / R;
#pragma unroll
    for (int e = 0; e < R; ++e) w[e] = twid<INV>(tw, e * step);
    float2 o[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      float2 acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 t = cmul(v[r], w[(r * u) % R]);
        acc = cadd(acc, t);
      }
      o[u] = acc;
    }
#pragma unroll
    for (int u = 0; u < R; ++u) v[u] = o[u];
  }
};

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[2], const float2*, int) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[4], const float2*, int) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  }
};

template <bool INV>
struct Dft<8, INV> {
  // Even/odd split: X[u] = E[u] + omega_8^u O[u], X[u+4] = E[u] - omega_8^u O[u].
  __device__ __forceinline__ static void run(float2 (&v)[8], const float2* __restrict__ tw, int p) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    const float2 w1 = twid<INV>(tw, p / 8);
    const float2 w3 = twid<INV>(tw, 3 * p / 8);
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

}  // namespace fftdev
}  // namespace qtp
