// tcgen05 / TMA / mbarrier device helpers shared by the tensor-core kernels
// (internal to libqtp).  Every wait is bounded by kWaitNs of %globaltimer.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace qtp {
namespace tcdev {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false after limit_ns
// nanoseconds of %globaltimer (kWaitNs unless a launch asks for less).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023u) == 0 && globaltimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
          "r"(dst),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), version 1 at bit 46, swizzle at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}

constexpr uint32_t kLayoutSw128 = 2;
constexpr uint32_t kLayoutSw64 = 4;
constexpr uint32_t kLayoutSw32 = 6;

// Descriptor of one bf16 part tile for the MMA at K offset 16 * k16.
//   K-major: rows of BK bf16 (2 BK bytes, swizzled over the row: 64-byte
//            pattern for BK = 32, 32-byte for BK = 16); 8-row groups 16 BK
//            bytes apart; the k16 step moves 32 B along the row.
//   MN-major: K rows of 64 bf16 (128 B, 128-byte swizzle); consecutive 64-wide
//             blocks of M/N are 128 BK bytes apart, 8-row K groups 1024 B apart.
template <bool MN_MAJOR, int BK>
__device__ __forceinline__ uint64_t part_desc(uint32_t tile, int k16) {
  if (MN_MAJOR) return smem_desc(tile + (uint32_t)k16 * 2048u, 128u * BK, 1024u, kLayoutSw128);
  return smem_desc(tile + (uint32_t)k16 * 32u, 16u, 16u * BK, BK == 32 ? kLayoutSw64 : kLayoutSw32);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 32 consecutive TMEM columns of this thread's lane.  The wait sits in the same
// asm statement, so the outputs are complete when the compiler sees them.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Two (four) loads of 32 consecutive TMEM columns each, completed by one
// tcgen05.wait::ld: the loads' latencies overlap instead of adding up.
__device__ __forceinline__ void tmem_ld32x2(uint32_t a0, uint32_t a1, uint32_t (&r)[32], uint32_t (&s)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15]),
        "=r"(s[16]), "=r"(s[17]), "=r"(s[18]), "=r"(s[19]), "=r"(s[20]), "=r"(s[21]), "=r"(s[22]), "=r"(s[23]),
        "=r"(s[24]), "=r"(s[25]), "=r"(s[26]), "=r"(s[27]), "=r"(s[28]), "=r"(s[29]), "=r"(s[30]), "=r"(s[31])
      : "r"(a0), "r"(a1)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t (&r)[32],
                                            uint32_t (&s)[32], uint32_t (&t)[32], uint32_t (&u)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%128];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%129];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%64, %65, %66, %67, %68, %69, %70, %71, %72, %73, %74, %75, %76, %77, %78, %79, %80, %81, %82, %83, %84, %85, %86, %87, %88, %89, %90, %91, %92, %93, %94, %95}, [%130];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%96, %97, %98, %99, %100, %101, %102, %103, %104, %105, %106, %107, %108, %109, %110, %111, %112, %113, %114, %115, %116, %117, %118, %119, %120, %121, %122, %123, %124, %125, %126, %127}, [%131];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15]),
        "=r"(s[16]), "=r"(s[17]), "=r"(s[18]), "=r"(s[19]), "=r"(s[20]), "=r"(s[21]), "=r"(s[22]), "=r"(s[23]),
        "=r"(s[24]), "=r"(s[25]), "=r"(s[26]), "=r"(s[27]), "=r"(s[28]), "=r"(s[29]), "=r"(s[30]), "=r"(s[31]),
        "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]),
        "=r"(t[8]), "=r"(t[9]), "=r"(t[10]), "=r"(t[11]), "=r"(t[12]), "=r"(t[13]), "=r"(t[14]), "=r"(t[15]),
        "=r"(t[16]), "=r"(t[17]), "=r"(t[18]), "=r"(t[19]), "=r"(t[20]), "=r"(t[21]), "=r"(t[22]), "=r"(t[23]),
        "=r"(t[24]), "=r"(t[25]), "=r"(t[26]), "=r"(t[27]), "=r"(t[28]), "=r"(t[29]), "=r"(t[30]), "=r"(t[31]),
        "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
        "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
}

// tcgen05.ld 16x256b: at TMEM address (lane L, column C), repetition j of .x4
// hands thread t the words (lane L + t/4, columns C + 8j + 2(t%4) and +1) in
// registers 4j, 4j+1 and (lane L + 8 + t/4, the same columns) in 4j+2, 4j+3
// (checked on the GPU against words written in the 32x32b layout).  Two (four)
// loads of 32 columns each behind one tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld16x256x2(uint32_t a0, uint32_t a1, uint32_t (&r)[16], uint32_t (&s)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      :
        "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15])
      : "r"(a0), "r"(a1)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16x256x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t (&r)[16],
                                                uint32_t (&s)[16], uint32_t (&t)[16], uint32_t (&u)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%65];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%66];\n\t"
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%67];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      :
        "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15]),
        "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]),
        "=r"(t[8]), "=r"(t[9]), "=r"(t[10]), "=r"(t[11]), "=r"(t[12]), "=r"(t[13]), "=r"(t[14]), "=r"(t[15]),
        "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
}

// Write 32 consecutive TMEM columns of this thread's lane (the inverse of
// tmem_ld32); tmem_st_wait() makes the stores complete before a thread
// signals that the columns may be overwritten.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), negate A / B at bits 13 / 14, A/B major at bits 15/16,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(bool a_mn, bool b_mn, int bn, int bm = 128) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(bm >> 4) << 24);
}
constexpr uint32_t kNegA = 1u << 13;
constexpr uint32_t kNegB = 1u << 14;

// A-operand collector use of one tcgen05.mma: read A from shared memory and
// keep it (FILL), or take the kept A a last time and release it (LASTUSE).
// Used on pairs of consecutive MMAs with the same A descriptor and the same
// instruction descriptor (different B and accumulator), which then read A from
// shared memory once.  (Chains with .collector::a::use between them, across
// MMAs whose instruction descriptors differ in a negate bit, gave wrong
// results on the GB300 and are not used.)
enum : int { kCollFill = 1, kCollLastUse = 3 };

template <int COLL>
__device__ __forceinline__ void mma_bf16_c(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  if constexpr (COLL == kCollFill) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    static_assert(COLL == kCollLastUse, "collector use");
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// The MMAs of one K step of a complex product in split-BF16 (NP = 4 parts per
// operand: re_hi, re_lo, im_hi, im_lo) or plain BF16 (NP = 2: re, im):
//   re += s0 ar.br + s1 ai.bi,   im += s2 ar.bi + s3 ai.br,
// each real product x.y as x_hi.y_hi (into the main accumulator) plus
// x_hi.y_lo + x_lo.y_hi (into the correction accumulator, which is the main
// one unless the kernel splits them).  Bit q of neg makes s_q = -1, applied by
// negating B.  In split-BF16 the two MMAs x_hi.y_hi and x_hi.y_lo share A and
// sign and run as a collector pair, so a K step reads each A_hi part twice
// from shared memory instead of four times.  da, db: the descriptors of part 0
// of the A and B tiles; a_step, b_step: descriptor increments from one part to
// the next.  acc_*: accumulate flags (0 until the accumulator's first MMA).
template <int NP, bool SPLIT>
__device__ __forceinline__ void complex_kstep(uint64_t da, uint64_t db, uint32_t a_step, uint32_t b_step,
                                              uint32_t idesc, uint32_t neg, uint32_t d_re, uint32_t d_im,
                                              uint32_t c_re, uint32_t c_im, uint32_t& acc_re, uint32_t& acc_im,
                                              uint32_t& acc_cre, uint32_t& acc_cim) {
  const uint32_t s0 = (neg & 1u) ? idesc | kNegB : idesc;
  const uint32_t s1 = (neg & 2u) ? idesc | kNegB : idesc;
  const uint32_t s2 = (neg & 4u) ? idesc | kNegB : idesc;
  const uint32_t s3 = (neg & 8u) ? idesc | kNegB : idesc;
  if constexpr (NP == 4) {
    const uint64_t ar_hi = da, ar_lo = da + a_step, ai_hi = da + 2 * a_step, ai_lo = da + 3 * a_step;
    const uint64_t br_hi = db, br_lo = db + b_step, bi_hi = db + 2 * b_step, bi_lo = db + 3 * b_step;
    const uint32_t f_cre = SPLIT ? acc_cre : 1u, f_cim = SPLIT ? acc_cim : 1u;
    mma_bf16_c<kCollFill>(d_re, ar_hi, br_hi, s0, acc_re);
    mma_bf16_c<kCollLastUse>(c_re, ar_hi, br_lo, s0, f_cre);
    mma_bf16_c<kCollFill>(d_im, ar_hi, bi_hi, s2, acc_im);
    mma_bf16_c<kCollLastUse>(c_im, ar_hi, bi_lo, s2, f_cim);
    mma_bf16(c_re, ar_lo, br_hi, s0, 1u);
    mma_bf16(c_im, ar_lo, bi_hi, s2, 1u);
    mma_bf16_c<kCollFill>(d_re, ai_hi, bi_hi, s1, 1u);
    mma_bf16_c<kCollLastUse>(c_re, ai_hi, bi_lo, s1, 1u);
    mma_bf16_c<kCollFill>(d_im, ai_hi, br_hi, s3, 1u);
    mma_bf16_c<kCollLastUse>(c_im, ai_hi, br_lo, s3, 1u);
    mma_bf16(c_re, ai_lo, bi_hi, s1, 1u);
    mma_bf16(c_im, ai_lo, br_hi, s3, 1u);
    acc_cre = 1u;
    acc_cim = 1u;
  } else {
    const uint64_t ar = da, ai = da + a_step, br = db, bi = db + b_step;
    mma_bf16(d_re, ar, br, s0, acc_re);
    mma_bf16(d_im, ar, bi, s2, acc_im);
    mma_bf16(d_re, ai, bi, s1, 1u);
    mma_bf16(d_im, ai, br, s3, 1u);
  }
  acc_re = 1u;
  acc_im = 1u;
}

// The same K step with every MMA issued from one asm statement.  The MMA
// warp's single issuing thread is the critical path for 128-wide and
// narrower tiles (a 16-deep step of 12 MMAs takes ~1100 cycles at N = 128,
// and every dependent instruction of the issue loop adds to it), so the
// descriptors travel as 32-bit low words (start address >> 4 and the leading
// byte offset: a part or stage offset never carries out of the 14-bit
// address field, shared memory being < 256 KB) with one shared high word per
// operand, are packed with mov.b64 inside the asm, and the accumulate
// predicates are set once.  a_lo / b_lo: low words of part 0 of the A / B
// tiles; a_step / b_step: part-to-part increments; i0..i3: instruction
// descriptors of the four real products (negate-B bit per sign, see
// complex_kstep); acc: 0 for the first K step into the accumulators.
template <int NP, bool SPLIT>
__device__ __forceinline__ void complex_kstep_issue(uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi,
                                                    uint32_t a_step, uint32_t b_step, uint32_t i0, uint32_t i1,
                                                    uint32_t i2, uint32_t i3, uint32_t d_re, uint32_t d_im,
                                                    uint32_t c_re, uint32_t c_im, uint32_t acc) {
  if constexpr (NP == 4) {
    asm volatile(
        "{\n\t"
        ".reg .pred pa, pc, pt;\n\t"
        ".reg .b32 t1, t2, t3;\n\t"
        ".reg .b64 arh, arl, aih, ail, brh, brl, bih, bil;\n\t"
        "setp.ne.b32 pa, %14, 0;\n\t"
        "setp.eq.b32 pt, %14, %14;\n\t"
        "setp.ne.b32 pc, %15, 0;\n\t"
        "add.u32 t1, %0, %4;\n\t"
        "add.u32 t2, t1, %4;\n\t"
        "add.u32 t3, t2, %4;\n\t"
        "mov.b64 arh, {%0, %1};\n\t"
        "mov.b64 arl, {t1, %1};\n\t"
        "mov.b64 aih, {t2, %1};\n\t"
        "mov.b64 ail, {t3, %1};\n\t"
        "add.u32 t1, %2, %5;\n\t"
        "add.u32 t2, t1, %5;\n\t"
        "add.u32 t3, t2, %5;\n\t"
        "mov.b64 brh, {%2, %3};\n\t"
        "mov.b64 brl, {t1, %3};\n\t"
        "mov.b64 bih, {t2, %3};\n\t"
        "mov.b64 bil, {t3, %3};\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%10], arh, brh, %6, pa;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%12], arh, brl, %6, pc;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%11], arh, bih, %8, pa;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%13], arh, bil, %8, pc;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%12], arl, brh, %6, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%13], arl, bih, %8, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%10], aih, bih, %7, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%12], aih, bil, %7, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%11], aih, brh, %9, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%13], aih, brl, %9, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%12], ail, bih, %7, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%13], ail, brh, %9, pt;\n\t"
        "}" ::"r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(a_step), "r"(b_step), "r"(i0), "r"(i1), "r"(i2),
        "r"(i3), "r"(d_re), "r"(d_im), "r"(c_re), "r"(c_im), "r"(acc), "r"(SPLIT ? acc : 1u)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred pa, pt;\n\t"
        ".reg .b32 t1;\n\t"
        ".reg .b64 ar, ai, br, bi;\n\t"
        "setp.ne.b32 pa, %10, 0;\n\t"
        "setp.eq.b32 pt, %10, %10;\n\t"
        "add.u32 t1, %0, %4;\n\t"
        "mov.b64 ar, {%0, %1};\n\t"
        "mov.b64 ai, {t1, %1};\n\t"
        "add.u32 t1, %2, %5;\n\t"
        "mov.b64 br, {%2, %3};\n\t"
        "mov.b64 bi, {t1, %3};\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%11], ar, br, %6, pa;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%12], ar, bi, %8, pa;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%11], ai, bi, %7, pt;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%12], ai, br, %9, pt;\n\t"
        "}" ::"r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(a_step), "r"(b_step), "r"(i0), "r"(i1), "r"(i2),
        "r"(i3), "r"(acc), "r"(d_re), "r"(d_im)
        : "memory");
  }
}

// Instruction descriptors of the four real products of a complex product:
// bit q of neg subtracts product q (ar.br, ai.bi, ar.bi, ai.br).
__device__ __forceinline__ void signed_idescs(uint32_t idesc, uint32_t neg, uint32_t& i0, uint32_t& i1,
                                              uint32_t& i2, uint32_t& i3) {
  i0 = (neg & 1u) ? idesc | kNegB : idesc;
  i1 = (neg & 2u) ? idesc | kNegB : idesc;
  i2 = (neg & 4u) ? idesc | kNegB : idesc;
  i3 = (neg & 8u) ? idesc | kNegB : idesc;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Acquire a tensor map that lives in global memory for the async proxy.
__device__ __forceinline__ void tensormap_acquire(const void* tm) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<unsigned long long>(tm))
               : "memory");
}

// Epilogue store of one warp's 32 x 32 complex chunk of an accumulator tile,
// straight from the 16x256b register layout: a thread holds two neighbouring
// columns of two rows of the real and of the imaginary accumulator, so it
// writes 16 contiguous bytes (two complex values) and four neighbouring
// threads fill 64 contiguous bytes of a row (whole 32-byte sectors), with no
// shared-memory transpose.  t: TMEM address of the warp's first lane and the
// chunk's first column of the real accumulator; the imaginary one at
// t + im_off; CORR adds the pair at t + corr_off (split correction or promoted
// running sum).  out points at (row0, col0) of a row-major matrix with row
// stride ld (float2); rows_valid / cols_valid clip the chunk at the matrix
// edge; vec: out and ld allow 16-byte stores (out 16-byte aligned, ld even).
template <bool CORR>
__device__ __forceinline__ void store_chunk(uint32_t t, uint32_t im_off, uint32_t corr_off, float2* out, long long ld,
                                            int rows_valid, int cols_valid, int lane, bool vec) {
  const int rq = lane >> 2, cq = 2 * (lane & 3);
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const uint32_t th = t + ((uint32_t)(16 * hh) << 16);
    uint32_t re[16], im[16];
    if constexpr (CORR) {
      uint32_t cre[16], cim[16];
      tmem_ld16x256x4(th, th + im_off, th + corr_off, th + corr_off + im_off, re, im, cre, cim);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        re[i] = __float_as_uint(__uint_as_float(re[i]) + __uint_as_float(cre[i]));
        im[i] = __float_as_uint(__uint_as_float(im[i]) + __uint_as_float(cim[i]));
      }
    } else {
      tmem_ld16x256x2(th, th + im_off, re, im);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int r = 16 * hh + 8 * g + rq, c = 8 * j + cq, k = 4 * j + 2 * g;
        if (r < rows_valid) {
          float2* o = out + (long long)r * ld + c;
          const float r0 = __uint_as_float(re[k]), i0 = __uint_as_float(im[k]);
          const float r1 = __uint_as_float(re[k + 1]), i1 = __uint_as_float(im[k + 1]);
          if (vec && c + 1 < cols_valid) {
            *reinterpret_cast<float4*>(o) = make_float4(r0, i0, r1, i1);
          } else {
            if (c < cols_valid) o[0] = make_float2(r0, i0);
            if (c + 1 < cols_valid) o[1] = make_float2(r1, i1);
          }
        }
      }
    }
  }
}

}  // namespace tcdev
}  // namespace qtp
