// T-SVD of a quaternion tensor under the T-product (a method the paper names
// in Sec. 6 as enabled by its fast T-product; the decomposition is not in the
// paper).  The per-frequency structure of Thm 5.1 in its plain-transform form
// carries it: with A1_hat = fft(A1), A2_hat = fft(A2) along mode 3 and
// g = (-f) mod p, the 2m x 2n complex matrix
//     M_f(A) = [[A1_hat(f), A2_hat(f)], [-conj A2_hat(g), conj A1_hat(g)]]
// turns T-products into matrix products and ^H into ^H, and
// M_g = Q conj(M_f) Q^T (Q = [[0, I], [-I, 0]]).  One SVD per frequency pair
// {f, g} therefore gives A = U * S * V^H with U, V unitary tensors and S
// f-diagonal:
//   f != g: the left / right singular vectors of odd rank (1st, 3rd, ...)
//           are U's, V's spectra at f, those of even rank (through the
//           conjugate block pattern) at g; S's spectra at f and g are the
//           odd- and even-ranked singular values;
//   f == g: M_f is a quaternion matrix's complex adjoint, its singular
//           values come in equal pairs, and the factors keep the pattern
//           (second half = Q^T conj(first half)).
//
// Kernel: each frequency pair runs a one-sided (Hestenes) Jacobi SVD of M_f,
// or of M_f^H when m < n (the columns are the 2 min(m, n) side): cyclic
// sweeps in round-robin order (disjoint column pairs per round, one warp per
// pair), each 2x2 step a phase that makes the off-diagonal real followed by
// the symmetric Jacobi rotation.  Then the columns' norms are sorted, null
// columns completed by Gram-Schmidt, and the factors written to the spectra
// of U, V and S (frequency-major, for the inverse transform).  When a pair's
// buffers fit in shared memory one CTA does all of it there; otherwise they
// sit in a per-pair global scratch (resident in L2) and a cluster of up to
// four CTAs shares the sweeps, the round's column pairs dealt over all its
// warps with a cluster barrier between rounds, and the cluster's first CTA
// finishes alone.  When 2 max(m, n) <= 256 the columns stay in registers for
// a whole phase and pass between neighbouring warps (ring_sweeps) instead of
// going through L2 every round; those clusters take up to eight CTAs, as
// many as keep all pairs in one wave.  The rotations and their order are the same
// in every variant.
#include <cooperative_groups.h>

#include <mutex>
#include <utility>
#include <vector>

#include "qtp_internal.h"

namespace qtp {

namespace {

constexpr int kTsvdThreads = 512;
constexpr int kTsvdWarps = kTsvdThreads / 32;
constexpr int kTsvdMaxCols = 128;   // 2 min(m, n)
constexpr int kTsvdMaxSweeps = 40;
// A phase ends after a sweep in which every pair was orthogonal to within this
// relative off-diagonal |x^H y| / (|x| |y|) when it was visited: cyclic
// Jacobi converges quadratically there, so the next sweep would meet
// off-diagonals of order 1e-8, far under the rotation threshold, and is
// skipped (a sweep without rotations also meets the bound).
constexpr float kTsvdStopRatio = 1e-4f;
// Phase 0 (before the Newton-Schulz step) may stop earlier: the sweep after
// the step rotates every pair still above the rotation threshold (measured:
// a sweep at 2.6e-4 is followed by one at 2.0e-6).
constexpr float kTsvdStopRatio0 = 1e-3f;
constexpr size_t kTsvdSmemMax = 200 * 1024;  // dynamic shared memory of the in-smem variant
constexpr int kTsvdClusterMax = 8;            // CTAs per pair of the global-scratch variant (portable)

namespace cg = cooperative_groups;

// Loads and stores of the working buffers.  In the global-scratch variant
// several CTAs (SMs) of a cluster write and read the same columns, so those
// go through L2 only (.cg), and no SM keeps a stale copy in its L1.
template <bool G>
__device__ __forceinline__ float2 ldw(const float2* p) {
  if constexpr (G) return __ldcg(p);
  else return *p;
}
template <bool G>
__device__ __forceinline__ void stw(float2* p, float2 v) {
  if constexpr (G) __stcg(p, v);
  else *p = v;
}
// Barrier over the CTAs that share a pair (release / acquire at cluster scope).
template <bool G>
__device__ __forceinline__ void pair_sync() {
  if constexpr (G) cg::this_cluster().sync();
  else __syncthreads();
}

// One 32 x 32 complex output tile out(i, j) = sum_l a(i, l) b(l, j) (CONJA:
// conj(a(i, l))) by one CTA (512 threads, two outputs each), the operands
// staged through shared memory kTileK entries of l at a time (sm: kTileSmem
// bytes) and read once per tile.  fa(i, l), fb(l, j) return the entries
// (0 <= i < ni, 0 <= j < nj, 0 <= l < K); IFAST stages a with i fastest (a
// column-major over rows i), else l fastest (columns over l), so that the
// loads are coalesced either way; b is staged l fastest.  put(i, j, value)
// receives the result.
constexpr int kTileP = 33;   // padded pitch of a's staging
constexpr int kTileK = 128;  // inner entries staged at a time
constexpr size_t kTileSmem = (size_t)(kTileP + 32) * kTileK * sizeof(float2);

template <bool IFAST, bool CONJA, class FA, class FB, class Put>
__device__ void tile_mm(FA fa, FB fb, int K, int ni, int nj, float2* sm, Put put) {
  float2* As = sm;                   // [l][i], pitch kTileP
  float2* Bs = sm + kTileP * kTileK;  // [j][l], pitch kTileK
  const int i = threadIdx.x & 31, j0 = threadIdx.x >> 5;
  float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTileK) {
    const int kc = min(kTileK, K - k0);
    // every load of the chunk in flight at once (a thread's share is at most
    // 32 kTileK / 512 = 8 entries of each operand), then the shared stores
    constexpr int U = 32 * kTileK / kTsvdThreads;
    float2 va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = threadIdx.x + u * kTsvdThreads;
      va[u] = vb[u] = make_float2(0.f, 0.f);
      if (idx < 32 * kc) {
        const int ii = IFAST ? (idx & 31) : idx / kc, ll = IFAST ? (idx >> 5) : idx - (idx / kc) * kc;
        if (ii < ni) va[u] = fa(ii, k0 + ll);
        const int jj = idx / kc, lb = idx - jj * kc;
        if (jj < nj) vb[u] = fb(k0 + lb, jj);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = threadIdx.x + u * kTsvdThreads;
      if (idx < 32 * kc) {
        const int ii = IFAST ? (idx & 31) : idx / kc, ll = IFAST ? (idx >> 5) : idx - (idx / kc) * kc;
        As[ll * kTileP + ii] = va[u];
        const int jj = idx / kc, lb = idx - jj * kc;
        Bs[jj * kTileK + lb] = vb[u];
      }
    }
    __syncthreads();
    for (int l = 0; l < kc; ++l) {
      float2 a = As[l * kTileP + i];
      if (CONJA) a.y = -a.y;
      const float2 b0 = Bs[j0 * kTileK + l], b1 = Bs[(j0 + 16) * kTileK + l];
      re0 = fmaf(a.x, b0.x, fmaf(-a.y, b0.y, re0));
      im0 = fmaf(a.x, b0.y, fmaf(a.y, b0.x, im0));
      re1 = fmaf(a.x, b1.x, fmaf(-a.y, b1.y, re1));
      im1 = fmaf(a.x, b1.y, fmaf(a.y, b1.x, im1));
    }
    __syncthreads();
  }
  if (i < ni && j0 < nj) put(i, j0, make_float2(re0, im0));
  if (i < ni && j0 + 16 < nj) put(i, j0 + 16, make_float2(re1, im1));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x^H y over n entries, by one warp (every lane gets the sum).
__device__ float2 warp_dot(const float2* __restrict__ x, const float2* __restrict__ y, int n, int lane) {
  float re = 0.f, im = 0.f;
  for (int r = lane; r < n; r += 32) {
    const float2 a = x[r], b = y[r];
    re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
    im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
  }
  return make_float2(warp_sum(re), warp_sum(im));
}

// y -= c x, by one warp.
__device__ void warp_axpy(float2* __restrict__ y, const float2* __restrict__ x, float2 c, int n, int lane) {
  for (int r = lane; r < n; r += 32) {
    const float2 v = cmul(c, x[r]);
    y[r].x -= v.x;
    y[r].y -= v.y;
  }
  __syncwarp();
}

// The quaternion partner of a column of 2h entries: [-conj(w[h:]); conj(w[:h])].
__device__ __forceinline__ float2 partner_at(const float2* w, int h, int r) {
  return r < h ? make_float2(-w[h + r].x, w[h + r].y) : make_float2(w[r - h].x, -w[r - h].y);
}

// (partner of x)^H y, by one warp.
__device__ float2 warp_dot_partner(const float2* __restrict__ x, const float2* __restrict__ y, int h, int lane) {
  float re = 0.f, im = 0.f;
  for (int r = lane; r < 2 * h; r += 32) {
    const float2 a = partner_at(x, h, r), b = y[r];
    re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
    im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
  }
  return make_float2(warp_sum(re), warp_sum(im));
}

// One warp: project column w (2h entries) off the nb columns of B (stride
// ldb) and, when with_partners, off their partners too (two passes); return
// its norm after projection (w is not normalised).
__device__ float warp_project(float2* w, const float2* B, int nb, long long ldb, int h, bool with_partners,
                              int lane) {
  const int n = 2 * h;
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < nb; ++j) {
      const float2* b = B + (long long)j * ldb;
      warp_axpy(w, b, warp_dot(b, w, n, lane), n, lane);
      if (with_partners) {
        const float2 c = warp_dot_partner(b, w, h, lane);
        for (int r = lane; r < n; r += 32) {
          const float2 v = cmul(c, partner_at(b, h, r));
          w[r].x -= v.x;
          w[r].y -= v.y;
        }
        __syncwarp();
      }
    }
  }
  const float2 d = warp_dot(w, w, n, lane);
  return sqrtf(fmaxf(d.x, 0.f));
}

// One warp: w (2h entries) := a unit vector orthogonal to the nb columns of B
// (and their partners when with_partners), tried from the basis vectors.
__device__ void warp_complete(float2* w, const float2* B, int nb, long long ldb, int h, bool with_partners,
                              int lane) {
  const int n = 2 * h;
  for (int t = 0; t < n; ++t) {
    for (int r = lane; r < n; r += 32) w[r] = make_float2(r == t ? 1.f : 0.f, 0.f);
    __syncwarp();
    const float nw = warp_project(w, B, nb, ldb, h, with_partners, lane);
    if (nw > 0.5f) {
      for (int r = lane; r < n; r += 32) w[r] = cscale(w[r], 1.f / nw);
      __syncwarp();
      return;
    }
  }
}

// Whole block: project w (2h entries) off the nb columns of B (stride ldb)
// and their partners, by two passes of classical Gram-Schmidt (all the
// coefficients of a pass at once, one warp per column, then one subtraction
// with the threads over the entries); returns |w| after projection (the same
// value in every thread).  coef: 2 nb entries of shared memory.
__device__ float block_project_partners(float2* w, const float2* B, int nb, long long ldb, int h, float2* coef,
                                        float* nrm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = 2 * h;
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = warp; j < nb; j += kTsvdWarps) {
      const float2* b = B + (long long)j * ldb;
      const float2 c0 = warp_dot(b, w, n, lane);
      const float2 c1 = warp_dot_partner(b, w, h, lane);
      if (lane == 0) {
        coef[2 * j] = c0;
        coef[2 * j + 1] = c1;
      }
    }
    __syncthreads();
    for (int r = tid; r < n; r += kTsvdThreads) {
      float2 acc = make_float2(0.f, 0.f);
      for (int j = 0; j < nb; ++j) {
        const float2* b = B + (long long)j * ldb;
        const float2 u = cmul(coef[2 * j], b[r]), v = cmul(coef[2 * j + 1], partner_at(b, h, r));
        acc.x += u.x + v.x;
        acc.y += u.y + v.y;
      }
      w[r].x -= acc.x;
      w[r].y -= acc.y;
    }
    __syncthreads();
  }
  if (warp == 0) {
    const float2 d = warp_dot(w, w, n, lane);
    if (lane == 0) *nrm = sqrtf(fmaxf(d.x, 0.f));
  }
  __syncthreads();
  const float v = *nrm;
  __syncthreads();
  return v;
}

template <bool G>
__device__ __forceinline__ float4 ldw4(const float4* p) {
  if constexpr (G) return __ldcg(p);
  else return *p;
}
template <bool G>
__device__ __forceinline__ void stw4(float4* p, float4 v) {
  if constexpr (G) __stcg(p, v);
  else *p = v;
}

// One Jacobi step on a column pair held in registers by one warp: columns x,
// y of X (R rows) and vx, vy of V (C rows), in 16-byte pairs of entries
// (R, C even), pair r = lane + 32 i of a column in element i (NX pairs of an
// X column, R <= 64 NX; NV of a V column, C <= 64 NV; the pairs past the
// column are zero and stay zero).  Rotates in place; returns whether it did.
template <int NX, int NV>
__device__ __forceinline__ bool rotate_regs(float4 (&xr)[NX], float4 (&yr)[NX], float4 (&vxr)[NV],
                                            float4 (&vyr)[NV], float tol, float& ratio) {
  float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    const float4 u = xr[i], v = yr[i];
    al = fmaf(u.x, u.x, fmaf(u.y, u.y, fmaf(u.z, u.z, fmaf(u.w, u.w, al))));
    be = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, be))));
    gr = fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, fmaf(u.w, v.w, gr))));
    gi = fmaf(u.x, v.y, fmaf(-u.y, v.x, fmaf(u.z, v.w, fmaf(-u.w, v.z, gi))));
  }
  al = warp_sum(al);
  be = warp_sum(be);
  gr = warp_sum(gr);
  gi = warp_sum(gi);
  const float gabs = hypotf(gr, gi);
  const float nrm = sqrtf(al * be);
  ratio = nrm > 0.f ? gabs / nrm : 0.f;
  if (!(gabs > tol * nrm && gabs > 1e-30f)) return false;
  const float zeta = (be - al) / (2.f * gabs);
  const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float cs = 1.f / sqrtf(1.f + tt * tt), sn = cs * tt;
  const float2 ce = make_float2(gr / gabs, -gi / gabs);
  // [x, y] <- [x, conj(e) y] [[c, s], [-s, c]] on both entries of a pair
  auto rot = [&](float4& u, float4& w) {
    const float2 v0 = cmul(ce, make_float2(w.x, w.y)), v1 = cmul(ce, make_float2(w.z, w.w));
    const float4 xo =
        make_float4(cs * u.x - sn * v0.x, cs * u.y - sn * v0.y, cs * u.z - sn * v1.x, cs * u.w - sn * v1.y);
    w = make_float4(sn * u.x + cs * v0.x, sn * u.y + cs * v0.y, sn * u.z + cs * v1.x, sn * u.w + cs * v1.y);
    u = xo;
  };
#pragma unroll
  for (int i = 0; i < NX; ++i) rot(xr[i], yr[i]);
#pragma unroll
  for (int i = 0; i < NV; ++i) rot(vxr[i], vyr[i]);
  return true;
}

// A column (n2 16-byte pairs) into / out of the register layout of rotate_regs.
template <bool G, int N>
__device__ __forceinline__ void load_col(float4 (&r)[N], const float4* src, int n2, int lane) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int e = lane + 32 * i;
    r[i] = e < n2 ? ldw4<G>(src + e) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}
template <bool G, int N>
__device__ __forceinline__ void store_col(const float4 (&r)[N], float4* dst, int n2, int lane) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int e = lane + 32 * i;
    if (e < n2) stw4<G>(dst + e, r[i]);
  }
}

// One Jacobi step on columns x, y of X and vx, vy of V in memory, by one
// warp: every entry a lane touches loaded at once into registers (one round
// trip to memory per pair), rotated there and stored once.  Columns 16-byte
// aligned.  Returns whether it rotated.
template <bool G, int NX, int NV>
__device__ __forceinline__ bool jacobi_pair_reg(float2* __restrict__ x, float2* __restrict__ y,
                                                float2* __restrict__ vx, float2* __restrict__ vy, int R, int C,
                                                float tol, int lane, float& ratio) {
  const int R2 = R >> 1, C2 = C >> 1;
  float4 xr[NX], yr[NX], vxr[NV], vyr[NV];
  load_col<G>(xr, reinterpret_cast<const float4*>(x), R2, lane);
  load_col<G>(yr, reinterpret_cast<const float4*>(y), R2, lane);
  load_col<G>(vxr, reinterpret_cast<const float4*>(vx), C2, lane);
  load_col<G>(vyr, reinterpret_cast<const float4*>(vy), C2, lane);
  if (!rotate_regs(xr, yr, vxr, vyr, tol, ratio)) return false;
  store_col<G>(xr, reinterpret_cast<float4*>(x), R2, lane);
  store_col<G>(yr, reinterpret_cast<float4*>(y), R2, lane);
  store_col<G>(vxr, reinterpret_cast<float4*>(vx), C2, lane);
  store_col<G>(vyr, reinterpret_cast<float4*>(vy), C2, lane);
  return true;
}

struct TsvdArgs {
  const float2* H;   // spectra of A: [plane][f][m][n] (complex FP32)
  float2* Uh;        // [plane][f][m][k]
  float2* Vh;        // [plane][f][n][k]
  float2* Sh;        // [plane][f][k][k], zeroed by the host
  float* sigma;      // [f][k]
  float2* scratch;   // per-pair buffers when shared memory is too small (G variant; else null)
  long long scratch_stride;
  int m, n, p, k;
  int R, C;          // rows and columns of the matrix the Jacobi sweeps work on
  int tall;          // 1: the sweeps work on M_f (m >= n); 0: on M_f^H
  int* status;       // set to 1 when a phase's sweeps end at kTsvdMaxSweeps still rotating
};

// Round-robin schedule: pair t of round rr over C (even) columns; column 0
// stays, the others rotate, so every pair meets once per sweep of C - 1 rounds.
__device__ __forceinline__ void rr_pair(int C, int rr, int t, int& a, int& b) {
  a = t == 0 ? 0 : 1 + (rr + t - 1) % (C - 1);
  b = 1 + (rr + C - 2 - t) % (C - 1);
}

// Jacobi sweeps with the columns in registers (the cluster variant when
// R <= 256).  Pair slot t (one per warp of the first wpc warps of each of the
// cluster's CTAs) keeps its two columns of X and V in registers for a whole
// phase; between rounds every slot hands
// one column to each neighbour through shared memory (distributed shared
// memory between the cluster's CTAs), which is the round-robin order of
// rr_pair run as a ring (T = C/2 - 1):
//   slot 0 keeps column 0 and takes slot 1's first column as its second;
//   slot t, 0 < t < T, takes slot t+1's first column and slot t-1's second;
//   slot T moves its second column to first and takes slot T-1's second.
// At a sweep boundary slot t holds rr_pair(C, 0, t) again.  The hand-over
// buffers alternate between two sets, so the one cluster barrier per round
// orders both the hand-over and the reuse of a set two rounds later.  The
// rotations and their order are those of the sweeps from memory.
// Returns whether the stop test (largest relative off-diagonal of a sweep
// under stop) ended the loop (cluster-uniform).
__device__ __forceinline__ bool ring_sweeps(float2* X, float2* V, int R, int C, float tol, float stop, int nc,
                                            int rank, int warp, int lane, int tid, int* maxoff, float4* slots) {
  cg::cluster_group cl = cg::this_cluster();
  const int R2 = R >> 1, C2 = C >> 1, L = R2 + C2;
  const int T = C / 2 - 1;
  const int wpc = (T + nc) / nc;  // slots per CTA, ceil((T + 1) / nc) <= kTsvdWarps
  const int t = rank * wpc + warp;
  const bool active = warp < wpc && t <= T;
  float4 xa[4], xb[4], va[2], vb[2];
  int ca = 0, cb = 0;
  if (active) {
    rr_pair(C, 0, t, ca, cb);
    load_col<true>(xa, reinterpret_cast<const float4*>(X + (long long)ca * R), R2, lane);
    load_col<true>(xb, reinterpret_cast<const float4*>(X + (long long)cb * R), R2, lane);
    load_col<true>(va, reinterpret_cast<const float4*>(V + (long long)ca * C), C2, lane);
    load_col<true>(vb, reinterpret_cast<const float4*>(V + (long long)cb * C), C2, lane);
  }
  // hand-over buffer of slot u: set s, kind 0 (its first column) or 1 (its second)
  auto local_slot = [&](int s, int kind, int w) { return slots + ((s * 2 + kind) * kTsvdWarps + w) * L; };
  auto slot_of = [&](int s, int kind, int u) -> const float4* {
    return cl.map_shared_rank(local_slot(s, kind, u % wpc), u / wpc);
  };
  int set = 0;
  bool converged = false;
  for (int sweep = 0; sweep < kTsvdMaxSweeps; ++sweep) {
    if (tid == 0) *maxoff = 0;
    cl.sync();
    for (int rr = 0; rr < C - 1; ++rr) {
      if (active) {
        float ratio;
        rotate_regs(xa, xb, va, vb, tol, ratio);
        if (lane == 0) atomicMax(maxoff, __float_as_int(ratio));  // ratio >= 0: ordered as an int
      }
      if (T == 0) continue;  // one pair: nothing moves
      if (active && t >= 1) {
        float4* s = local_slot(set, 0, warp);
        store_col<false>(xa, s, R2, lane);
        store_col<false>(va, s + R2, C2, lane);
      }
      if (active && t < T) {
        float4* s = local_slot(set, 1, warp);
        store_col<false>(xb, s, R2, lane);
        store_col<false>(vb, s + R2, C2, lane);
      }
      cl.sync();
      if (active) {
        if (t == 0) {
          const float4* s = slot_of(set, 0, 1);
          load_col<false>(xb, s, R2, lane);
          load_col<false>(vb, s + R2, C2, lane);
        } else {
          if (t < T) {
            const float4* s = slot_of(set, 0, t + 1);
            load_col<false>(xa, s, R2, lane);
            load_col<false>(va, s + R2, C2, lane);
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) xa[i] = xb[i];
#pragma unroll
            for (int i = 0; i < 2; ++i) va[i] = vb[i];
          }
          const float4* s = slot_of(set, 1, t - 1);
          load_col<false>(xb, s, R2, lane);
          load_col<false>(vb, s + R2, C2, lane);
        }
      }
      set ^= 1;
    }
    // every CTA takes the same maximum, after the last round's updates and
    // before the next sweep clears them
    cl.sync();
    int worst = 0;
    for (int j = 0; j < nc; ++j) worst = max(worst, *cl.map_shared_rank(maxoff, j));
    const bool done = __int_as_float(worst) < stop;
    cl.sync();
    if (done) {
      converged = true;
      break;
    }
  }
  if (active) {
    rr_pair(C, 0, t, ca, cb);
    store_col<true>(xa, reinterpret_cast<float4*>(X + (long long)ca * R), R2, lane);
    store_col<true>(xb, reinterpret_cast<float4*>(X + (long long)cb * R), R2, lane);
    store_col<true>(va, reinterpret_cast<float4*>(V + (long long)ca * C), C2, lane);
    store_col<true>(vb, reinterpret_cast<float4*>(V + (long long)cb * C), C2, lane);
  }
  cl.sync();
  return converged;
}

// G = false: one CTA per pair, buffers in dynamic shared memory.  G = true:
// a cluster of nc CTAs per pair (blockIdx.x = pair * nc + rank), buffers in
// the global scratch, the sweeps from memory or (RING) in registers; every
// CTA of the cluster takes the same barriers in the same order (the loop
// bounds and the convergence test are cluster-uniform).  The sweep variants
// are separate kernels so that neither's registers constrain the other's.
template <bool G, bool RING = false>
__global__ void __launch_bounds__(kTsvdThreads) tsvd_pair_kernel(TsvdArgs a) {
  extern __shared__ float4 tsvd_smem[];
  __shared__ float sig[kTsvdMaxCols];
  __shared__ int perm[kTsvdMaxCols];
  __shared__ int maxoff;  // largest relative off-diagonal of the sweep (float bits)
  int nc = 1, rank = 0;
  if constexpr (G) {
    nc = (int)cg::this_cluster().num_blocks();
    rank = (int)cg::this_cluster().block_rank();
  }
  const int q = blockIdx.x / nc;
  const int p = a.p, m = a.m, n = a.n, k = a.k, R = a.R, C = a.C;
  const int f = q, g = (p - q) % p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // thread and warp indices over the CTAs that share the pair
  const int gtid = rank * kTsvdThreads + tid, gthreads = nc * kTsvdThreads;
  const int gwarp = rank * kTsvdWarps + warp, gwarps = nc * kTsvdWarps;
  float2* X = G ? a.scratch + (long long)q * a.scratch_stride : reinterpret_cast<float2*>(tsvd_smem);
  float2* V = X + (long long)R * C;           // C x C
  float2* Tm = V + (long long)C * C;          // C x C: the Newton-Schulz factor
  float2* Tmp = Tm + (long long)C * C;        // C x C: products
  float2* Wa = Tmp + (long long)C * C;        // 2m x k (self-paired frequencies)
  float2* Za = Wa + (long long)2 * m * k;     // 2n x k

  // 1. X = M_f (tall) or M_f^H, column-major; V = I
  const long long slab = (long long)m * n;
  const float2* H1f = a.H + (long long)f * slab;
  const float2* H2f = a.H + ((long long)p + f) * slab;
  const float2* H1g = a.H + (long long)g * slab;
  const float2* H2g = a.H + ((long long)p + g) * slab;
  auto Mval = [&](int r, int c) -> float2 {  // M_f[r][c], r < 2m, c < 2n
    if (r < m) return c < n ? H1f[(long long)r * n + c] : H2f[(long long)r * n + (c - n)];
    const int rr = r - m;
    if (c < n) {
      const float2 v = H2g[(long long)rr * n + c];
      return make_float2(-v.x, v.y);
    }
    return cconj(H1g[(long long)rr * n + (c - n)]);
  };
  for (long long idx = gtid; idx < (long long)R * C; idx += gthreads) {
    const int c = (int)(idx / R), r = (int)(idx - (long long)c * R);
    stw<G>(X + idx, a.tall ? Mval(r, c) : cconj(Mval(c, r)));
  }
  for (int idx = gtid; idx < C * C; idx += gthreads)
    stw<G>(V + idx, make_float2(idx % (C + 1) == 0 ? 1.f : 0.f, 0.f));
  pair_sync<G>();

  // 2. cyclic one-sided Jacobi sweeps; X = M V throughout.
  // A rotation is skipped once |x^H y| <= tol |x| |y|; FP32 dot products over
  // R entries carry about sqrt(R / 32) eps of rounding, so the bound grows
  // past 256 rows.  Phase 0 sweeps until a sweep's pairs were all orthogonal
  // to kTsvdStopRatio0 when visited (1e-3; the sweep after the step below
  // finishes the job), phase 1 until kTsvdStopRatio (1e-4: quadratic
  // convergence leaves the next sweep nothing to rotate).  V then has
  // drifted from unitary by the rounding of its rotations (about
  // sqrt(rotations per column) eps: 1e-5 for 128 columns, which would show in
  // A = U S V^H), so one Newton-Schulz step T = (3 I - V^H V) / 2 is applied
  // to V and to X (keeping X = M V), and phase 1 sweeps again (one sweep
  // restores the columns' orthogonality, the step having moved them by ~1e-5).
  const float tol = 2e-6f * fmaxf(1.f, sqrtf((float)R / 256.f));
  const bool reg_path = R <= 512 && C <= 128;  // jacobi_pair_reg's register capacity
  for (int phase = 0; phase < 2; ++phase) {
  if (phase == 1 && G) {
    // Newton-Schulz step with 32 x 32 tiles staged in shared memory, the
    // tiles dealt over the cluster's CTAs: Tm = (3 I - V^H V) / 2, then
    // V <- V Tm and X <- X Tm in blocks of C rows, through Tmp.
    float2* sm = reinterpret_cast<float2*>(tsvd_smem);
    const int nt = (C + 31) / 32;
    for (int t = rank; t < nt * nt; t += nc) {
      const int i0 = (t / nt) * 32, c0 = (t % nt) * 32;
      tile_mm<false, true>([&](int i, int l) { return ldw<G>(V + (long long)(i0 + i) * C + l); },
                           [&](int l, int j) { return ldw<G>(V + (long long)(c0 + j) * C + l); }, C,
                           min(32, C - i0), min(32, C - c0), sm, [&](int i, int j, float2 g) {
                             stw<G>(Tm + (long long)(c0 + j) * C + i0 + i,
                                    make_float2(0.5f * ((i0 + i == c0 + j ? 3.f : 0.f) - g.x), -0.5f * g.y));
                           });
    }
    pair_sync<G>();
    for (int blk = -1; blk < (R + C - 1) / C; ++blk) {
      float2* src = blk < 0 ? V : X;
      const long long lds = blk < 0 ? C : R;
      const int r0 = blk < 0 ? 0 : blk * C;
      const int rows = blk < 0 ? C : min(C, R - r0);
      const int ntr = (rows + 31) / 32;
      for (int t = rank; t < ntr * nt; t += nc) {
        const int rb = (t / nt) * 32, c0 = (t % nt) * 32;
        tile_mm<true, false>([&](int i, int l) { return ldw<G>(src + (long long)l * lds + r0 + rb + i); },
                             [&](int l, int j) { return ldw<G>(Tm + (long long)(c0 + j) * C + l); }, C,
                             min(32, rows - rb), min(32, C - c0), sm,
                             [&](int i, int j, float2 v) { stw<G>(Tmp + (long long)(c0 + j) * rows + rb + i, v); });
      }
      pair_sync<G>();
      for (int idx = gtid; idx < rows * C; idx += gthreads) {
        const int j = idx / rows, r = idx - j * rows;
        stw<G>(src + (long long)j * lds + r0 + r, ldw<G>(Tmp + idx));
      }
      pair_sync<G>();
    }
  } else if (phase == 1) {
    // Tm = (3 I - V^H V) / 2, column-major
    for (int idx = gtid; idx < C * C; idx += gthreads) {
      const int j = idx / C, i = idx - j * C;
      const float2* vi = V + (long long)i * C;
      const float2* vj = V + (long long)j * C;
      float re = 0.f, im = 0.f;
      for (int r = 0; r < C; ++r) {
        const float2 x = ldw<G>(vi + r), y = ldw<G>(vj + r);
        re = fmaf(x.x, y.x, fmaf(x.y, y.y, re));
        im = fmaf(x.x, y.y, fmaf(-x.y, y.x, im));
      }
      stw<G>(Tm + idx, make_float2(0.5f * ((i == j ? 3.f : 0.f) - re), -0.5f * im));
    }
    pair_sync<G>();
    // V <- V Tm, then X <- X Tm in blocks of C rows, through Tmp
    for (int blk = -1; blk < (R + C - 1) / C; ++blk) {
      float2* src = blk < 0 ? V : X;
      const long long lds = blk < 0 ? C : R;
      const int r0 = blk < 0 ? 0 : blk * C;
      const int rows = blk < 0 ? C : min(C, R - r0);
      for (int idx = gtid; idx < rows * C; idx += gthreads) {
        const int j = idx / rows, r = idx - j * rows;
        float re = 0.f, im = 0.f;
        for (int l = 0; l < C; ++l) {
          const float2 x = ldw<G>(src + (long long)l * lds + r0 + r), t = ldw<G>(Tm + (long long)j * C + l);
          re = fmaf(x.x, t.x, fmaf(-x.y, t.y, re));
          im = fmaf(x.x, t.y, fmaf(x.y, t.x, im));
        }
        stw<G>(Tmp + (long long)j * rows + r, make_float2(re, im));
      }
      pair_sync<G>();
      for (int idx = gtid; idx < rows * C; idx += gthreads) {
        const int j = idx / rows, r = idx - j * rows;
        stw<G>(src + (long long)j * lds + r0 + r, ldw<G>(Tmp + idx));
      }
      pair_sync<G>();
    }
  }
  if constexpr (RING) {
    if (!ring_sweeps(X, V, R, C, tol, phase == 0 ? kTsvdStopRatio0 : kTsvdStopRatio, nc, rank, warp, lane, tid,
                     &maxoff, reinterpret_cast<float4*>(tsvd_smem)) &&
        rank == 0 && tid == 0)
      atomicExch(a.status, 1);
    continue;
  }
  bool converged = false;
  for (int sweep = 0; sweep < kTsvdMaxSweeps; ++sweep) {
    if (tid == 0) maxoff = 0;
    pair_sync<G>();
    for (int rr = 0; rr < C - 1; ++rr) {
      for (int t = gwarp; t < C / 2; t += gwarps) {
        int ca, cb;
        rr_pair(C, rr, t, ca, cb);
        float2* x = X + (long long)ca * R;
        float2* y = X + (long long)cb * R;
        if (reg_path) {
          float2* vx = V + (long long)ca * C;
          float2* vy = V + (long long)cb * C;
          float ratio;
          if (R <= 256) jacobi_pair_reg<G, 4, 2>(x, y, vx, vy, R, C, tol, lane, ratio);
          else jacobi_pair_reg<G, 8, 2>(x, y, vx, vy, R, C, tol, lane, ratio);
          if (lane == 0) atomicMax(&maxoff, __float_as_int(ratio));
          continue;
        }
        float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
        for (int r = lane; r < R; r += 32) {
          const float2 u = ldw<G>(x + r), v = ldw<G>(y + r);
          al = fmaf(u.x, u.x, fmaf(u.y, u.y, al));
          be = fmaf(v.x, v.x, fmaf(v.y, v.y, be));
          gr = fmaf(u.x, v.x, fmaf(u.y, v.y, gr));
          gi = fmaf(u.x, v.y, fmaf(-u.y, v.x, gi));
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const float gabs = hypotf(gr, gi);
        const float nrm = sqrtf(al * be);
        if (lane == 0) atomicMax(&maxoff, __float_as_int(nrm > 0.f ? gabs / nrm : 0.f));
        if (gabs > tol * nrm && gabs > 1e-30f) {
          // [x, y] <- [x, conj(e) y] [[c, s], [-s, c]], e = gamma / |gamma|
          const float zeta = (be - al) / (2.f * gabs);
          const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float cs = 1.f / sqrtf(1.f + tt * tt), sn = cs * tt;
          const float2 ce = make_float2(gr / gabs, -gi / gabs);
          for (int r = lane; r < R; r += 32) {
            const float2 u = ldw<G>(x + r), v = cmul(ce, ldw<G>(y + r));
            stw<G>(x + r, make_float2(cs * u.x - sn * v.x, cs * u.y - sn * v.y));
            stw<G>(y + r, make_float2(sn * u.x + cs * v.x, sn * u.y + cs * v.y));
          }
          float2* vx = V + (long long)ca * C;
          float2* vy = V + (long long)cb * C;
          for (int r = lane; r < C; r += 32) {
            const float2 u = ldw<G>(vx + r), v = cmul(ce, ldw<G>(vy + r));
            stw<G>(vx + r, make_float2(cs * u.x - sn * v.x, cs * u.y - sn * v.y));
            stw<G>(vy + r, make_float2(sn * u.x + cs * v.x, sn * u.y + cs * v.y));
          }
        }
      }
      pair_sync<G>();
    }
    // every CTA of the pair takes the same maximum, after the round's barrier
    // and before the next sweep clears it (the barrier below)
    int worst = maxoff;
    if constexpr (G) {
      worst = 0;
      for (int j = 0; j < nc; ++j) worst = max(worst, *cg::this_cluster().map_shared_rank(&maxoff, j));
    }
    const bool done = __int_as_float(worst) < (phase == 0 ? kTsvdStopRatio0 : kTsvdStopRatio);
    pair_sync<G>();
    if (done) {
      converged = true;
      break;
    }
  }
  if (!converged && rank == 0 && tid == 0) atomicExch(a.status, 1);
  }
  // the rest (sorting, completion, scatter) is the first CTA's alone, but for
  // the structured completion at a self-paired frequency, which every CTA of
  // the cluster shares; the others leave after their last barrier, with no
  // access to their shared memory pending
  const bool share = G && f == g;  // uniform in the cluster
  if (rank != 0 && !share) return;

  // 3. singular values (column norms), sorted decreasing (ties by index)
  for (int c = warp; c < C && rank == 0; c += kTsvdWarps) {
    const float2 d = warp_dot(X + (long long)c * R, X + (long long)c * R, R, lane);
    if (lane == 0) sig[c] = sqrtf(fmaxf(d.x, 0.f));
  }
  __syncthreads();
  if (tid < C && rank == 0) {
    const float s = sig[tid];
    int rk = 0;
    for (int j = 0; j < C; ++j) rk += (sig[j] > s) || (sig[j] == s && j < tid);
    perm[rk] = tid;
  }
  __syncthreads();
  if (share) {
    // the other CTAs take the norms and the order from the first
    pair_sync<G>();
    if (rank != 0)
      for (int c = tid; c < C; c += kTsvdThreads) {
        sig[c] = *cg::this_cluster().map_shared_rank(&sig[c], 0);
        perm[c] = *cg::this_cluster().map_shared_rank(&perm[c], 0);
      }
    pair_sync<G>();  // the copies are done before the first CTA may leave
  }
  const float smax = sig[perm[0]];
  const float null_tol = 1e-6f * smax;

  // 4. normalise the X columns (the left vectors when tall, else the right
  //    ones); the other side is V, unitary already
  for (long long idx = tid; idx < (long long)R * C && rank == 0; idx += kTsvdThreads) {
    const int c = (int)(idx / R);
    const float s = sig[c];
    X[idx] = s > null_tol && s > 0.f ? cscale(X[idx], 1.f / s) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // left vectors W (2m rows), right vectors Z (2n rows), column c
  float2* W = a.tall ? X : V;
  float2* Z = a.tall ? V : X;
  const long long ldw = a.tall ? R : C, ldz = a.tall ? C : R;

  if (f != g) {
    // null columns on the X side: complete against the other X columns, in
    // rank order, by warp 0
    if (warp == 0) {
      for (int i = 0; i < C; ++i) {
        const int c = perm[i];
        if (sig[c] > null_tol && sig[c] > 0.f) continue;
        // the columns of rank < i are final (live ones rank first): project a
        // basis vector off each of them
        float2* w = X + (long long)c * R;
        for (int t = 0; t < R; ++t) {
          for (int r = lane; r < R; r += 32) w[r] = make_float2(r == t ? 1.f : 0.f, 0.f);
          __syncwarp();
          for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < i; ++j) {
              const float2* b = X + (long long)perm[j] * R;
              warp_axpy(w, b, warp_dot(b, w, R, lane), R, lane);
            }
          const float nw = sqrtf(fmaxf(warp_dot(w, w, R, lane).x, 0.f));
          if (nw > 0.5f) {
            for (int r = lane; r < R; r += 32) w[r] = cscale(w[r], 1.f / nw);
            __syncwarp();
            break;
          }
        }
      }
    }
    __syncthreads();
    // scatter: rank 2i -> frequency f, rank 2i + 1 -> frequency g
    const long long sU = (long long)m * k, sV = (long long)n * k, sS = (long long)k * k;
    for (int idx = tid; idx < m * k; idx += kTsvdThreads) {
      const int r = idx / k, i = idx - r * k;
      const float2* wa = W + (long long)perm[2 * i] * ldw;
      const float2* wb = W + (long long)perm[2 * i + 1] * ldw;
      a.Uh[(long long)f * sU + idx] = wa[r];
      a.Uh[((long long)p + f) * sU + idx] = wb[r];
      a.Uh[((long long)p + g) * sU + idx] = make_float2(-wa[m + r].x, wa[m + r].y);
      a.Uh[(long long)g * sU + idx] = cconj(wb[m + r]);
    }
    for (int idx = tid; idx < n * k; idx += kTsvdThreads) {
      const int r = idx / k, i = idx - r * k;
      const float2* za = Z + (long long)perm[2 * i] * ldz;
      const float2* zb = Z + (long long)perm[2 * i + 1] * ldz;
      a.Vh[(long long)f * sV + idx] = za[r];
      a.Vh[((long long)p + f) * sV + idx] = zb[r];
      a.Vh[((long long)p + g) * sV + idx] = make_float2(-za[n + r].x, za[n + r].y);
      a.Vh[(long long)g * sV + idx] = cconj(zb[n + r]);
    }
    for (int i = tid; i < k; i += kTsvdThreads) {
      const float sa = sig[perm[2 * i]], sb = sig[perm[2 * i + 1]];
      a.sigma[(long long)f * k + i] = sa;
      a.sigma[(long long)g * k + i] = sb;
      a.Sh[(long long)f * sS + (long long)i * k + i] = make_float2(sa, 0.f);
      a.Sh[(long long)g * sS + (long long)i * k + i] = make_float2(sb, 0.f);
    }
    return;
  }

  // f == g: one vector per equal pair, the partners complete the factors.
  // Column by column in rank order, the whole block takes the candidate of
  // rank 2i and projects it off the chosen columns and their partners (two
  // passes of classical Gram-Schmidt); a null or dependent candidate is
  // completed from basis vectors by warp 0.
  __shared__ float2 coef[2 * kTsvdMaxCols];
  __shared__ float nrm;
  bool structured = false;
  if constexpr (G) {
    // When every candidate is live, one Newton-Schulz step on each side's
    // structured set S = [w_0 .. w_{k-1} | partner(w_0) .. partner(w_{k-1})]
    // does the orthogonalisation at once: the candidates are orthonormal, and
    // orthogonal to the other candidates' partners, to the sweeps' accuracy
    // (a doubled singular value's subspace holds its vectors' partners), so
    // S^H S = I + E with small E and S (3 I - S^H S) / 2 is orthonormal to
    // O(|E|^2).  The new w_i are the first k columns.  The tiles are dealt over
    // the cluster's CTAs.  Otherwise (a null or nearly dependent candidate:
    // |E| > 0.1) the first CTA runs the sequential completion below.
    bool all_live = true;
    for (int i = 0; i < k; ++i) {
      const float sv = sig[perm[2 * i]];
      if (!(sv > null_tol && sv > 0.f)) all_live = false;
    }
    if (all_live) {  // the same in every CTA
      float2* sm = reinterpret_cast<float2*>(tsvd_smem);
      pair_sync<G>();  // the first CTA's normalisation of X is complete
      for (int idx = gtid; idx < 2 * m * k; idx += gthreads) {
        const int i = idx / (2 * m), r = idx - i * 2 * m;
        __stcg(Wa + idx, __ldcg(W + (long long)perm[2 * i] * ldw + r));
      }
      for (int idx = gtid; idx < 2 * n * k; idx += gthreads) {
        const int i = idx / (2 * n), r = idx - i * 2 * n;
        __stcg(Za + idx, __ldcg(Z + (long long)perm[2 * i] * ldz + r));
      }
      if (tid == 0) maxoff = 0;
      pair_sync<G>();
      const int nt = (C + 31) / 32;
      float mydev = 0.f;  // this thread's largest |S^H S - I| entry
      for (int t = rank; t < 2 * nt * nt; t += nc) {
        const int side = t / (nt * nt), tt = t - side * nt * nt;
        const float2* B = side == 0 ? Wa : Za;
        const int h = side == 0 ? m : n;
        float2* T = side == 0 ? Tm : Tmp;
        auto col = [&](int c, int l) -> float2 {
          if (c < k) return __ldcg(B + (long long)c * 2 * h + l);
          const float2* w = B + (long long)(c - k) * 2 * h;  // partner_at, read through L2
          return l < h ? make_float2(-__ldcg(w + h + l).x, __ldcg(w + h + l).y)
                       : make_float2(__ldcg(w + l - h).x, -__ldcg(w + l - h).y);
        };
        const int i0 = (tt / nt) * 32, c0 = (tt % nt) * 32;
        tile_mm<false, true>([&](int i, int l) { return col(i0 + i, l); }, [&](int l, int j) { return col(c0 + j, l); },
                             2 * h, min(32, C - i0), min(32, C - c0), sm, [&](int i, int j, float2 g) {
                               const bool d = i0 + i == c0 + j;
                               mydev = fmaxf(mydev, fabsf(g.x - (d ? 1.f : 0.f)) + fabsf(g.y));
                               __stcg(T + (long long)(c0 + j) * C + i0 + i,
                                      make_float2(0.5f * ((d ? 3.f : 0.f) - g.x), -0.5f * g.y));
                             });
      }
      {
        const int wdev = __reduce_max_sync(0xffffffffu, __float_as_int(mydev));  // deviations >= 0
        if (lane == 0) atomicMax(&maxoff, wdev);
      }
      pair_sync<G>();
      int worst = 0;
      for (int j = 0; j < nc; ++j) worst = max(worst, *cg::this_cluster().map_shared_rank(&maxoff, j));
      if (__int_as_float(worst) <= 0.1f) {  // the same in every CTA
        // X is free (its columns were copied into Wa or Za): the new W at
        // X (2m x k), the new Z after it (2n x k)
        const int ntw = ((2 * m + 31) / 32) * ((k + 31) / 32), ntz = ((2 * n + 31) / 32) * ((k + 31) / 32);
        for (int t = rank; t < ntw + ntz; t += nc) {
          const int side = t < ntw ? 0 : 1, tt = side == 0 ? t : t - ntw;
          const float2* B = side == 0 ? Wa : Za;
          const int h = side == 0 ? m : n;
          const float2* T = side == 0 ? Tm : Tmp;
          float2* out = side == 0 ? X : X + (long long)2 * m * k;
          const int ntc = (k + 31) / 32;
          const int r0 = (tt / ntc) * 32, c0 = (tt % ntc) * 32;
          tile_mm<true, false>(
              [&](int i, int l) {
                if (l < k) return __ldcg(B + (long long)l * 2 * h + r0 + i);
                const float2* w = B + (long long)(l - k) * 2 * h;
                const int r = r0 + i;
                return r < h ? make_float2(-__ldcg(w + h + r).x, __ldcg(w + h + r).y)
                             : make_float2(__ldcg(w + r - h).x, -__ldcg(w + r - h).y);
              },
              [&](int l, int j) { return __ldcg(T + (long long)(c0 + j) * C + l); }, C, min(32, 2 * h - r0),
              min(32, k - c0), sm, [&](int i, int j, float2 v) { __stcg(out + (long long)(c0 + j) * 2 * h + r0 + i, v); });
        }
        pair_sync<G>();
        for (int idx = gtid; idx < 2 * m * k; idx += gthreads) __stcg(Wa + idx, __ldcg(X + idx));
        for (int idx = gtid; idx < 2 * n * k; idx += gthreads) __stcg(Za + idx, __ldcg(X + (long long)2 * m * k + idx));
        pair_sync<G>();
        structured = true;
      }
    }
  }
  // the sequential completion and the scatter are the first CTA's
  if (rank != 0) return;
  for (int i = 0; i < k && !structured; ++i) {
    const int c = perm[2 * i];
    const bool live = sig[c] > null_tol && sig[c] > 0.f;
    float2* wa = Wa + (long long)i * 2 * m;
    float2* za = Za + (long long)i * 2 * n;
    const float2* wc = W + (long long)c * ldw;
    const float2* zc = Z + (long long)c * ldz;
    for (int r = tid; r < 2 * m; r += kTsvdThreads) wa[r] = wc[r];
    for (int r = tid; r < 2 * n; r += kTsvdThreads) za[r] = zc[r];
    __syncthreads();
    const float nw = block_project_partners(wa, Wa, i, 2 * m, m, coef, &nrm);
    const float nz = block_project_partners(za, Za, i, 2 * n, n, coef, &nrm);
    const bool keep_w = live && nw > 0.5f, keep_z = live && nz > 0.5f;
    for (int r = tid; r < 2 * m; r += kTsvdThreads)
      if (keep_w) wa[r] = cscale(wa[r], 1.f / nw);
    for (int r = tid; r < 2 * n; r += kTsvdThreads)
      if (keep_z) za[r] = cscale(za[r], 1.f / nz);
    __syncthreads();
    if (warp == 0) {
      if (!keep_w) warp_complete(wa, Wa, i, 2 * m, m, true, lane);
      if (!keep_z) warp_complete(za, Za, i, 2 * n, n, true, lane);
    }
    __syncthreads();
  }
  const long long sU = (long long)m * k, sV = (long long)n * k, sS = (long long)k * k;
  for (int idx = tid; idx < m * k; idx += kTsvdThreads) {
    const int r = idx / k, i = idx - r * k;
    const float2* wa = Wa + (long long)i * 2 * m;
    a.Uh[(long long)f * sU + idx] = wa[r];
    a.Uh[((long long)p + f) * sU + idx] = make_float2(-wa[m + r].x, wa[m + r].y);
  }
  for (int idx = tid; idx < n * k; idx += kTsvdThreads) {
    const int r = idx / k, i = idx - r * k;
    const float2* za = Za + (long long)i * 2 * n;
    a.Vh[(long long)f * sV + idx] = za[r];
    a.Vh[((long long)p + f) * sV + idx] = make_float2(-za[n + r].x, za[n + r].y);
  }
  for (int i = tid; i < k; i += kTsvdThreads) {
    const float s = sig[perm[2 * i]];
    const bool live = s > null_tol && s > 0.f;
    a.sigma[(long long)f * k + i] = live ? s : 0.f;
    a.Sh[(long long)f * sS + (long long)i * k + i] = make_float2(live ? s : 0.f, 0.f);
  }
}

// Complex entries of one pair's buffers: the working matrix (R x C), V, the
// Newton-Schulz factor and a product buffer (C x C each) and the self-paired
// halves Wa (2m x k), Za (2n x k).
long long tsvd_pair_elems(int m, int n) {
  const int k = m < n ? m : n;
  const long long R = 2LL * (m > n ? m : n), C = 2LL * k;
  return R * C + 3 * C * C + 2LL * m * k + 2LL * n * k;
}

}  // namespace

size_t tsvd_scratch_bytes(int m, int n, int p) {
  const size_t bytes = sizeof(float2) * (size_t)tsvd_pair_elems(m, n);
  if (bytes <= kTsvdSmemMax) return 0;
  return bytes * (size_t)(p / 2 + 1);
}

cudaError_t launch_tsvd_pairs(const float2* H, int m, int n, int p, float2* Uh, float2* Vh, float2* Sh,
                              float* sigma, float2* scratch, int* status, cudaStream_t st) {
  const int k = m < n ? m : n;
  if (2 * k > kTsvdMaxCols) return cudaErrorInvalidValue;
  TsvdArgs a;
  a.status = status;
  a.H = H;
  a.Uh = Uh;
  a.Vh = Vh;
  a.Sh = Sh;
  a.sigma = sigma;
  a.m = m;
  a.n = n;
  a.p = p;
  a.k = k;
  a.tall = m >= n ? 1 : 0;
  a.R = 2 * (m > n ? m : n);
  a.C = 2 * k;
  const long long elems = tsvd_pair_elems(m, n);
  const size_t bytes = sizeof(float2) * (size_t)elems;
  if (bytes <= kTsvdSmemMax) {
    a.scratch = nullptr;
    a.scratch_stride = 0;
    static std::atomic<unsigned long long> attr_set{0};
    cudaError_t e = ensure_smem_attr(attr_set, tsvd_pair_kernel<false>, kTsvdSmemMax);
    if (e != cudaSuccess) return e;
    tsvd_pair_kernel<false><<<p / 2 + 1, kTsvdThreads, bytes, st>>>(a);
    return cudaGetLastError();
  }
  if (!scratch) return cudaErrorInvalidValue;
  a.scratch = scratch;
  a.scratch_stride = elems;
  // columns in registers when a lane's share fits rotate_regs<4, 2> (R <= 256,
  // C <= 128); the hand-over buffers: 2 sets x 2 columns x 16 slots per CTA
  const bool ring = a.R <= 256;
  size_t ring_smem = ring ? (size_t)4 * kTsvdWarps * (a.R / 2 + a.C / 2) * sizeof(float4) : 0;
  if (ring_smem > kTsvdSmemMax) return cudaErrorInvalidValue;
  if (ring_smem < kTileSmem) ring_smem = kTileSmem;  // the Newton-Schulz tiles
  auto kfn = ring ? tsvd_pair_kernel<true, true> : tsvd_pair_kernel<true, false>;
  static std::atomic<unsigned long long> attr_set_ring{0}, attr_set_l2{0};
  {
    cudaError_t e = ring ? ensure_smem_attr(attr_set_ring, tsvd_pair_kernel<true, true>, kTsvdSmemMax)
                         : ensure_smem_attr(attr_set_l2, tsvd_pair_kernel<true, false>, kTsvdSmemMax);
    if (e != cudaSuccess) return e;
  }
  // enough CTAs that every column pair of a round has its own warp (C / 2
  // pairs); the sweeps from L2 deal the pairs over the warps in order, so
  // they take no more
  const int npairs = p / 2 + 1;
  const int nc_min = (a.C / 2 + kTsvdWarps - 1) / kTsvdWarps < 1 ? 1 : (a.C / 2 + kTsvdWarps - 1) / kTsvdWarps;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kTsvdThreads);
  cfg.dynamicSmemBytes = ring_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto set_nc = [&](int c) {
    cfg.gridDim = dim3((unsigned)(npairs * c));
    attr[0].val.clusterDim.x = (unsigned)c;
  };
  int nc = nc_min;
  if (ring) {
    // The ring's rounds are bound by each SM's issue of its slots' steps, so
    // the slots are spread over more CTAs while the clusters still run in
    // one wave (128x64x32, 17 pairs: 4, 5, 6 CTAs 2.95, 2.68, 2.37 ms; 8 CTAs
    // 1.96 ms a wave, but only 16 clusters of 8 fit at once).  The count
    // with the fewest waves x (slots per CTA + 8), the waves from the
    // occupancy query, cached per (device, C, pairs).
    int dev = 0;
    cudaGetDevice(&dev);
    const long long key = ((long long)dev << 40) | ((long long)a.C << 20) | npairs;
    static std::mutex mu;
    static std::vector<std::pair<long long, int>> chosen;
    int found = 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (const auto& kv : chosen)
        if (kv.first == key) found = kv.second;
    }
    if (found == 0) {
      found = nc_min;
      double best = 1e30;
      for (int c = nc_min; c <= kTsvdClusterMax; ++c) {
        set_nc(c);
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, kfn, &cfg) != cudaSuccess || active < 1) {
          (void)cudaGetLastError();
          continue;
        }
        const int wpc = (a.C / 2 + c - 1) / c;
        const double cost = (double)((npairs + active - 1) / active) * (wpc + 8);
        if (cost < best) {
          best = cost;
          found = c;
        }
      }
      std::lock_guard<std::mutex> lk(mu);
      chosen.emplace_back(key, found);
    }
    nc = found;
    if (const char* ev = getenv("QTP_TSVD_CLUSTER")) {  // a fixed count, for measurement
      const int want = atoi(ev);
      if (want >= nc_min && want <= kTsvdClusterMax) nc = want;
    }
  }
  set_nc(nc);
  cudaError_t e = cudaLaunchKernelEx(&cfg, kfn, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace qtp
