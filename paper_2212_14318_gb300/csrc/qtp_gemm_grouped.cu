// Per-frequency products of Algorithm 5.1 Step 2 for a batch of products with
// uneven (m, n, s, p): one persistent tcgen05 launch (split-BF16, forward).
//
// A tile is (frequency f, 128-row tile, 64-column tile) of one product and
// computes both output halves,
//   C1(f) = A1(f) B1(f) - A2(f) conj(B2(-f)),  C2(f) = A1(f) B2(f) + A2(f) conj(B1(-f)),
// so each K step loads the A tile (plane kh at f) once for both halves and
// one B tile per half (B's two planes at f for kh = 0, at -f for kh = 1).  The
// MMA width is the tile's valid columns rounded up to 16.  On these small
// products the time goes to issuing the many narrow (N <= 64) MMAs, about 80
// cycles each against 37 of tensor work (per-role timestamps), not to operand
// fetch or the epilogue.  A product with trans set is computed
// as C^T = B^T A^T, rows over s and columns over m (the larger of m and s fills
// the MMA's 128 rows): B's MN-major spectra are then the A operands (one per
// half) and A's K-major spectra the shared B operand, and the epilogue writes
// C^T's rows, which are C's contiguous columns.
//
// All tiles of all products form one index space; product g owns
// [tile_begin_g, tile_begin_g + tiles_m * tiles_n * p_g), ordered (frequency,
// row tile, column tile).  CTA i (one per SM) takes tiles i, i + grid, ...
// Warp 0 issues TMA, warp 1 tcgen05.mma, warps 2-5 drain TMEM; the 4-stage
// ring runs on across tiles, and TMEM holds two sets of the four accumulators
// (C1 and C2, real and imaginary, 64 columns each), so the epilogue of one
// tile overlaps the MMAs of the next.  In the plain orientation both halves
// add A1(f) B(f) with the same signs over the first K half, so there one
// 128-wide MMA per part and term covers C1 and C2 (the B descriptor's
// leading byte offset steps from half 0's slot to half 1's; the accumulators
// sit C1 re, C2 re, C1 im, C2 im): grouped products 35.3 -> 34.3 ms on the
// 4096-product workload.  Each product has its own two tensor
// maps in device memory, acquired for the async proxy before use.  All waits
// are bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include "qtp_internal.h"
#include "qtp_tc_common.cuh"

namespace qtp {

namespace {

using namespace tcdev;

constexpr int GBM = kGroupTcBM;          // 128 rows
constexpr int GBN = kGroupTcBN;          // 64 complex columns
constexpr int GBK = 16;                  // K per stage
constexpr int GSTAGES = 4;
constexpr int G_SLOT = 128 * GBK * 2;    // 4 KB: one bf16 part of a 128 x 16 (or 16 x 128) operand tile
constexpr int kGThreads = 192;
constexpr uint32_t G_TMEM_COLS = 512;    // 2 buffers x (C1 re, C2 re, C1 im, C2 im) x 64 columns
static_assert(4 * GBN * 2 <= (int)G_TMEM_COLS, "TMEM budget");

// Operand roles of the forward product per (output half h, K half kh): A and B
// planes, whether B is read at frequency -f, and which of the four real
// MMA products (a_re.b_re, a_im.b_im, a_re.b_im, a_im.b_re, with a and b the
// MMA's operands) is subtracted, for the plain (negmask) and the transposed
// (negmask_t) orientation.  Filled on the host; entry e = 2 h + kh sits in bit
// e (planes, fneg) or bits 4e..4e+3 (masks), so the kernel reads registers,
// not an indexed copy in local memory.
struct GViews {
  uint32_t a_plane, b_plane, b_fneg, negmask, negmask_t;
};
__device__ __forceinline__ uint32_t gv_bit(uint32_t bits, int h, int kh) { return (bits >> (2 * h + kh)) & 1u; }

struct GTile {
  int g, f, mt, nt;
};

// Tile t of the global index space.  A CTA visits increasing t, so its
// product cursor g only moves forward (a step or two per tile at most).
__device__ __forceinline__ GTile decode_tile(const GroupProblem* __restrict__ probs, int nprobs, long long t, int& g) {
  while (g + 1 < nprobs && probs[g + 1].tile_begin <= t) ++g;
  const GroupProblem& P = probs[g];
  long long local = t - P.tile_begin;
  GTile r;
  r.g = g;
  r.nt = (int)(local % P.tiles_n);
  local /= P.tiles_n;
  r.mt = (int)(local % P.tiles_m);
  r.f = (int)(local / P.tiles_m);
  return r;
}

// Stage s holds, per bf16 part q, three 4 KB slots: [shared operand (A's
// spectra)][operand of half 0][operand of half 1], each role's NP parts
// consecutive, so a role's part q sits at role_base + q * G_SLOT.
template <int NP>
__global__ void __launch_bounds__(kGThreads, 1)
    gemm_tc_grouped_kernel(const GroupProblem* __restrict__ probs, int nprobs, long long total_tiles, char* ws,
                           int* err, const GViews V, int merge0, long long withhold, unsigned long long wait_ns) {
  constexpr int STAGE = 3 * NP * G_SLOT;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint32_t tmem_base_slot;
  __shared__ int abort_flag;

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bars = base + GSTAGES * STAGE;
  const uint32_t full = bars, empty = bars + 8 * GSTAGES;
  const uint32_t acc_full = bars + 16 * GSTAGES;      // 2 barriers
  const uint32_t acc_empty = acc_full + 16;           // 2 barriers
  const uint32_t mma_done = acc_empty + 16;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(full + 8 * s, 1);
      mbar_init(empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + 8 * b, 1);
      mbar_init(acc_empty + 8 * b, 4);  // one arrival per epilogue warp
    }
    mbar_init(mma_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"(G_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_slot;
  long long it = 0;  // producer: stages issued (or withheld) so far

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int cur = 0, prev = -1;
      bool ok = true;
      for (long long t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
        const GTile T = decode_tile(probs, nprobs, t, cur);
        const GroupProblem& P = probs[T.g];
        const CUtensorMap* tmA = reinterpret_cast<const CUtensorMap*>(P.tmA);
        const CUtensorMap* tmB = reinterpret_cast<const CUtensorMap*>(P.tmB);
        if (T.g != prev) {  // first tile of this product on this CTA
          tensormap_acquire(tmA);
          tensormap_acquire(tmB);
          prev = T.g;
        }
        {  // warm the descriptor cache for the next tile's product
          const long long tn = t + gridDim.x;
          if (tn < total_tiles) {
            int gn = T.g;
            while (gn + 1 < nprobs && probs[gn + 1].tile_begin <= tn) ++gn;
            if (gn != T.g) {
              asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(probs[gn].tmA)) : "memory");
              asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(probs[gn].tmB)) : "memory");
            }
          }
        }
        const int nkb = (P.K + GBK - 1) / GBK;
        // plain: A tile 128 rows of all parts (one box), B tiles one 64-column box;
        // transposed: B tiles 128 rows of s (two 64-column boxes), A tile 64 rows
        const uint32_t tx_bytes = (uint32_t)(NP * (P.trans ? 2 * G_SLOT + G_SLOT / 2 : G_SLOT + G_SLOT));
        for (int kk = 0; kk < 2 * nkb; ++kk, ++it) {
          const int kh = kk / nkb;
          const int k0 = (kk - kh * nkb) * GBK;
          const int s = (int)(it % GSTAGES);
          const uint32_t ph = (uint32_t)(it / GSTAGES) & 1u;
          if (!mbar_wait(empty + 8 * s, ph ^ 1u, wait_ns)) {
            atomicExch(err, QTP_DEVERR_TIMEOUT_EMPTY);
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          if (*(volatile int*)&abort_flag) {
            ok = false;
            break;
          }
          if (it == withhold) continue;  // failure-path test: this stage never arrives
          mbar_expect_tx(full + 8 * s, tx_bytes);
          // A plane kh at f (both halves); B planes b_plane[h][kh] at f or -f
          const int gb = gv_bit(V.b_fneg, 0, kh) ? (P.p - T.f) % P.p : T.f;
          const int pa = (int)gv_bit(V.a_plane, 0, kh) * NP;
          const int pb0 = (int)gv_bit(V.b_plane, 0, kh) * NP, pb1 = (int)gv_bit(V.b_plane, 1, kh) * NP;
          const uint32_t st0 = base + (uint32_t)s * STAGE;
          // plain: the 128-row A tile of all NP parts in one copy (its tensor
          // map's box spans the parts)
          if (!P.trans) tma_load_4d(st0, tmA, full + 8 * s, k0, T.mt * GBM, T.f, pa);
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const uint32_t sh = st0 + (uint32_t)q * G_SLOT;
            const uint32_t h0 = sh + NP * G_SLOT, h1 = h0 + NP * G_SLOT;
            if (P.trans) {
              const int c = T.mt * GBM;  // 128 columns of s
              tma_load_4d(h0, tmB, full + 8 * s, c, k0, gb, pb0 + q);
              tma_load_4d(h0 + 128u * GBK, tmB, full + 8 * s, c + 64, k0, gb, pb0 + q);
              tma_load_4d(h1, tmB, full + 8 * s, c, k0, gb, pb1 + q);
              tma_load_4d(h1 + 128u * GBK, tmB, full + 8 * s, c + 64, k0, gb, pb1 + q);
              tma_load_4d(sh, tmA, full + 8 * s, k0, T.nt * GBN, T.f, pa + q);
            } else {
              tma_load_4d(h0, tmB, full + 8 * s, T.nt * GBN, k0, gb, pb0 + q);
              tma_load_4d(h1, tmB, full + 8 * s, T.nt * GBN, k0, gb, pb1 + q);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // The issuing thread is this kernel's critical path (narrow MMAs): stage,
    // phase and descriptor words are counters, one asm statement per half.
    if (lane == 0) {
      // descriptor words of the three slots of stage 0, K-major and MN-major
      const uint64_t dsh_k = part_desc<false, GBK>(base, 0);
      const uint64_t dh0_mn = part_desc<true, GBK>(base + NP * G_SLOT, 0);
      const uint32_t k_hi = (uint32_t)(dsh_k >> 32), mn_hi = (uint32_t)(dh0_mn >> 32);
      const uint32_t sh0 = (uint32_t)dsh_k, h00 = (uint32_t)dh0_mn;
      // Both halves' B tiles of a part as one 128-column MN-major operand: the
      // second 64-column block is half 1's slot, NP slots on (the leading byte
      // offset of the descriptor), so one MMA of N = 128 serves C1 and C2.
      const uint32_t h00m =
          (uint32_t)smem_desc(base + NP * G_SLOT, (uint32_t)(NP * G_SLOT), 1024u, kLayoutSw128);
      const uint32_t idesc_m = make_idesc(false, true, 2 * GBN);
      constexpr uint32_t PART = (uint32_t)(G_SLOT >> 4);    // part-to-part step
      constexpr uint32_t HALF = (uint32_t)(NP * G_SLOT) >> 4; // half 0 -> half 1 slot
      constexpr uint32_t STG = (uint32_t)STAGE >> 4;         // stage-to-stage step
      uint32_t so = 0;  // stage offset (descriptor units)
      int s = 0;
      uint32_t ph = 0;
      int lt = 0, cur = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < total_tiles && ok; t += gridDim.x, ++lt) {
        const GTile T = decode_tile(probs, nprobs, t, cur);
        const GroupProblem& P = probs[T.g];
        const bool tr = P.trans != 0;
        const int ncols = tr ? P.M : P.N;
        const int nw = (min(GBN, ncols - T.nt * GBN) + 15) & ~15;
        const uint32_t idesc = make_idesc(tr, !tr, nw);
        const uint32_t nmask = tr ? V.negmask_t : V.negmask;
        const int nkb = (P.K + GBK - 1) / GBK;
        const int buf = lt & 1;
        const uint32_t uph = (uint32_t)(lt >> 1) & 1u;
        if (!mbar_wait(acc_empty + 8 * buf, uph ^ 1u, wait_ns)) {
          atomicExch(err, QTP_DEVERR_TIMEOUT_ACC);
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        fence_after();
        // accumulators of this buffer: C1 re, C2 re, C1 im, C2 im (64 columns each)
        const uint32_t d0 = tmem + (uint32_t)(buf * 4 * GBN);
        uint32_t acc = 0;
        for (int kh = 0; kh < 2 && ok; ++kh) {
          uint32_t p0, p1, p2, p3, q0, q1, q2, q3;
          const bool merged = !tr && kh == 0 && merge0;
          signed_idescs(merged ? idesc_m : idesc, nmask >> (4 * kh), p0, p1, p2, p3);
          signed_idescs(idesc, nmask >> (4 * (2 + kh)), q0, q1, q2, q3);
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(full + 8 * s, ph, wait_ns)) {
              atomicExch(err, QTP_DEVERR_TIMEOUT_FULL);
              atomicExch(&abort_flag, 1);
              ok = false;
              break;
            }
            fence_after();
            if (merged) {  // one 128-wide product per part and term for both halves
              complex_kstep_issue<NP, false>(sh0 + so, k_hi, h00m + so, mn_hi, PART, PART, p0, p1, p2, p3, d0,
                                             d0 + 2 * GBN, d0, d0 + 2 * GBN, acc);
            } else if (tr) {  // A operands: B's spectra per half (MN-major); B operand: A's spectra (K-major, shared)
              complex_kstep_issue<NP, false>(h00 + so, mn_hi, sh0 + so, k_hi, PART, PART, p0, p1, p2, p3, d0,
                                             d0 + 2 * GBN, d0, d0 + 2 * GBN, acc);
              complex_kstep_issue<NP, false>(h00 + HALF + so, mn_hi, sh0 + so, k_hi, PART, PART, q0, q1, q2, q3,
                                             d0 + GBN, d0 + 3 * GBN, d0 + GBN, d0 + 3 * GBN, acc);
            } else {   // A operand: A's spectra (K-major, shared); B operands: B's spectra per half (MN-major)
              complex_kstep_issue<NP, false>(sh0 + so, k_hi, h00 + so, mn_hi, PART, PART, p0, p1, p2, p3, d0,
                                             d0 + 2 * GBN, d0, d0 + 2 * GBN, acc);
              complex_kstep_issue<NP, false>(sh0 + so, k_hi, h00 + HALF + so, mn_hi, PART, PART, q0, q1, q2, q3,
                                             d0 + GBN, d0 + 3 * GBN, d0 + GBN, d0 + 3 * GBN, acc);
            }
            acc = 1u;
            mma_commit(empty + 8 * s);
            if (++s == GSTAGES) {
              s = 0;
              ph ^= 1u;
              so = 0;
            } else {
              so += STG;
            }
          }
        }
        if (!ok) break;
        mma_commit(acc_full + 8 * buf);
      }
      if (!ok) {
        mma_commit(mma_done);
        mbar_wait(mma_done, 0, wait_ns);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    int lt = 0, cur = 0;
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x, ++lt) {
      const GTile T = decode_tile(probs, nprobs, t, cur);
      const GroupProblem& P = probs[T.g];
      const int buf = lt & 1;
      const uint32_t uph = (uint32_t)(lt >> 1) & 1u;
      if (!mbar_wait(acc_full + 8 * buf, uph, wait_ns)) {
        if (lane == 0) {
          atomicExch(err, QTP_DEVERR_TIMEOUT_ACC);
          atomicExch(&abort_flag, 1);
        }
        break;
      }
      fence_after();
      const int row0 = T.mt * GBM + q * 32;  // this warp's first accumulator row
      const int ncols = P.trans ? P.M : P.N;
      const int nw = min(GBN, ncols - T.nt * GBN);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        float2* out = reinterpret_cast<float2*>(ws + P.out_off) + (long long)h * P.p * P.M * P.N +
                      (long long)T.f * P.M * P.N;
        const uint32_t tb = tmem + (uint32_t)(buf * 4 * GBN + h * GBN) + lane_off;  // re; im 2 GBN on
        const bool vec = ((reinterpret_cast<uintptr_t>(out) | (uintptr_t)(P.N & 1) * 8u) & 15u) == 0;
#pragma unroll 1
        for (int c0 = 0; c0 < nw; c0 += 32) {
          const int col0 = T.nt * GBN + c0;
          if (!P.trans) {
            store_chunk<false>(tb + (uint32_t)c0, 2 * GBN, 0, out + (long long)row0 * P.N + col0, P.N, P.M - row0,
                               P.N - col0, lane, vec);
          } else {
            uint32_t re[32], im[32];
            tmem_ld32x2(tb + (uint32_t)c0, tb + (uint32_t)(2 * GBN + c0), re, im);
            // accumulator row = column of C (index into s), column = row of C
            // (index into m): lane-consecutive stores along C's rows
            const int cs = row0 + lane;
            if (cs < P.N) {
              const int nj = min(32, P.M - col0);
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < nj) out[(long long)(col0 + j) * P.N + cs] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + 8 * buf);
      if (*(volatile int*)&abort_flag) break;
    }
    fence_before();
  }
  __syncthreads();
  // Never leave with copies in flight: after an abort (final here) the
  // producer waits (bounded) for the last GSTAGES stages it issued, which
  // hold every stage the MMA warp did not consume.
  if (warp == 0 && lane == 0 && *(volatile int*)&abort_flag) {
    const long long first = it - GSTAGES < 0 ? 0 : it - GSTAGES;
    for (long long j = first; j < it; ++j)
      if (j != withhold) mbar_wait(full + 8 * (int)(j % GSTAGES), (uint32_t)(j / GSTAGES) & 1u, wait_ns);
  }
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_TMEM_COLS) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

// Spectra tensor [plane][part][f][rows][ld] (bf16) as a 4-D tensor map for
// the grouped kernel: box (16, 64) with the 32-byte swizzle for A's K-major
// spectra, (64, 16) with the 128-byte swizzle for B's MN-major spectra.
bool encode_group_map(void* tm, const void* base, int rows, int cols, int ld, int p, int nparts, bool mn_major,
                      bool all_parts, char* msg, size_t msglen) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    snprintf(msg, msglen, "cuTensorMapEncodeTiled unavailable");
    return false;
  }
  cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)p, (cuuint64_t)(2 * nparts)};
  cuuint64_t strides[3] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * rows, (cuuint64_t)ld * 2 * rows * p};
  // all_parts (K-major only): one box is a whole 128-row A tile in all nparts
  // bf16 parts of one plane, landing part after part 4 KB apart
  cuuint32_t box[4] = {mn_major ? 64u : (cuuint32_t)GBK, mn_major ? (cuuint32_t)GBK : (all_parts ? (cuuint32_t)GBM : 64u),
                       1, all_parts ? (cuuint32_t)nparts : 1u};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(tm), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base),
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   mn_major ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(msg, msglen, "cuTensorMapEncodeTiled failed (%d) rows=%d cols=%d ld=%d", (int)r, rows, cols, ld);
    return false;
  }
  return true;
}

namespace {
// Bytes handed to a kernel by value and copied to device memory by one block.
struct Blob {
  alignas(64) unsigned char b[kPutBlobBytes];
};
__global__ void put_blob_kernel(const __grid_constant__ Blob src, int nbytes, unsigned char* dst) {
  for (int i = threadIdx.x; i < nbytes; i += blockDim.x) dst[i] = src.b[i];
}
}  // namespace

cudaError_t launch_put_blob(const void* host, int nbytes, void* dst, cudaStream_t st) {
  if (nbytes <= 0 || nbytes > kPutBlobBytes) return cudaErrorInvalidValue;
  Blob b;
  memcpy(b.b, host, (size_t)nbytes);
  put_blob_kernel<<<1, 128, 0, st>>>(b, nbytes, reinterpret_cast<unsigned char*>(dst));
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc_grouped(const GroupProblem* d_probs, int nprobs, long long total_tiles, int nparts,
                                   char* ws, int* d_err, int num_ctas, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  const int np = nparts == 4 ? 4 : 2;
  const size_t smem = (size_t)GSTAGES * 3 * np * G_SLOT + 1024 + 256;
  const int grid = (int)(total_tiles < num_ctas ? total_tiles : num_ctas);
  // Forward product (Thm 5.1): C1 = A1 B1 - A2 conj(B2(-f)), C2 = A1 B2 + A2 conj(B1(-f)).
  // (tau ar + i tau ai)(br + i sb bi): re += tau ar.br - tau sb ai.bi, im += tau sb ar.bi + tau ai.br
  GViews V = {0u, 0u, 0u, 0u, 0u};
  const int a_plane[2][2] = {{0, 1}, {0, 1}};
  const int b_plane[2][2] = {{0, 1}, {1, 0}};
  const int b_conj[2][2] = {{0, 1}, {0, 1}};
  const float sign[2][2] = {{1.f, -1.f}, {1.f, 1.f}};
  for (int h = 0; h < 2; ++h)
    for (int kh = 0; kh < 2; ++kh) {
      const int e = 2 * h + kh;
      V.a_plane |= (uint32_t)a_plane[h][kh] << e;
      V.b_plane |= (uint32_t)b_plane[h][kh] << e;
      V.b_fneg |= (uint32_t)b_conj[h][kh] << e;  // the conjugated B operand is the one read at -f
      const float tau = sign[h][kh];
      const float sb = b_conj[h][kh] ? -1.f : 1.f;
      // MMA products (a_re b_re, a_im b_im, a_re b_im, a_im b_re).  Plain: a = A,
      // b = B (conjugate when sb = -1).  Transposed: a = B, b = A; the complex
      // product commutes, so only the cross terms swap their signs.
      const float c[4] = {tau, -tau * sb, tau * sb, tau};
      const float ct[4] = {tau, -tau * sb, tau, tau * sb};
      uint32_t mask = 0, mask_t = 0;
      for (int q = 0; q < 4; ++q) {
        if (c[q] < 0) mask |= 1u << q;
        if (ct[q] < 0) mask_t |= 1u << q;
      }
      V.negmask |= mask << (4 * e);
      V.negmask_t |= mask_t << (4 * e);
    }
  // the kernel loads one A tile for both halves and reads B at one frequency per K half
  for (int kh = 0; kh < 2; ++kh)
    if (a_plane[0][kh] != a_plane[1][kh] || b_conj[0][kh] != b_conj[1][kh]) return cudaErrorInvalidValue;
  // The first K half of the plain orientation may run both halves as one
  // 128-wide MMA when their signs agree (C1 and C2 both add A1 B at f).
  int merge0 = ((V.negmask >> 0) & 15u) == ((V.negmask >> 8) & 15u);
  if (const char* env = getenv("QTP_GROUPED_MERGE"))  // 0: two 64-wide MMAs per half (comparison runs)
    if (!strcmp(env, "0")) merge0 = 0;
  int withhold = -1;
  unsigned long long wait_ns = 0;
  fault_injection(&withhold, &wait_ns);
  cudaError_t e;
  if (np == 4) {
    e = cudaFuncSetAttribute(gemm_tc_grouped_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tc_grouped_kernel<4><<<grid, kGThreads, smem, st>>>(d_probs, nprobs, total_tiles, ws, d_err, V, merge0,
                                                             withhold, wait_ns);
  } else {
    e = cudaFuncSetAttribute(gemm_tc_grouped_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tc_grouped_kernel<2><<<grid, kGThreads, smem, st>>>(d_probs, nprobs, total_tiles, ws, d_err, V, merge0,
                                                             withhold, wait_ns);
  }
  return cudaGetLastError();
}

}  // namespace qtp
