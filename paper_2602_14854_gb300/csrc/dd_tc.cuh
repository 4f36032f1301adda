// Blackwell (sm_103a) tensor-core building blocks: TMA tile loads, mbarriers, tensor
// memory (TMEM) and tcgen05.mma, as inline PTX.
//
// Operand layout in shared memory (no swizzle, K-major, the canonical "interleaved"
// layout of tcgen05): a core matrix is 8 rows x 16 bytes stored contiguously (128 B);
// core matrices adjacent along K are LBO bytes apart, 8-row groups SBO bytes apart.
// Here an operand of R rows and a K extent of KB bytes is stored as R/8 groups, each
// holding its KB/16 core matrices back to back: LBO = 128, SBO = 8 * KB, and the
// element (row, kbyte) sits at (row / 8) * SBO + (kbyte / 16) * 128 + (row % 8) * 16 +
// kbyte % 16.  One MMA consumes 32 bytes of K (8 TF32 or 16 BF16 values): its
// descriptors start at base + 256 s for K-slab s.
//
// D (M = 128 rows, FP32) lives in TMEM: row i in lane i, column j in column j.  Warp w
// of the CTA reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace dd {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier --------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// plain arrive (one of the barrier's expected arrivals)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// arrive on the barrier and add `bytes` to its expected transaction count
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity: false after `limit` polls (the caller
// records the failure and skips the work that depended on it).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---- TMA ---------------------------------------------------------------------------
// 2D tiled load of the box at (x = column, y = row) of the tensor map into shared memory,
// completing on bar (transaction bytes counted there).  x * element size must be a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// ---- proxy and tcgen05 fences ---------------------------------------------------------
// generic-proxy shared-memory writes made visible to the async proxy (the MMA's reads)
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- tensor memory ----------------------------------------------------------------
// Warp-wide (all 32 lanes): allocate ncols (a power of two >= 32) columns; the base
// address is written to *holder (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(holder)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 lanes (lane = row)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- descriptors ------------------------------------------------------------------
// shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor: FP32 accumulator, both operands K-major, M x N
// (a_fmt = b_fmt: 1 = BF16 under kind::f16, 2 = TF32 under kind::tf32)
__host__ __device__ __forceinline__ uint32_t idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
enum { FMT_BF16 = 1, FMT_TF32 = 2 };

// D (+)= A B^T, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
// arrive on bar when every MMA this thread issued so far has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// ---- FP64 <-> FP32 by integer operations ----------------------------------------------
// On this GPU FP64 instructions (conversions included) issue at 1/64 of the FP32 rate, so
// the operand conversions below touch only integer and FP32 units.
// x rounded to FP32 (half-way cases away from zero); magnitudes below FP32's normal range
// become a signed zero, above it infinity (non-finite inputs: infinity).
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) + (1ull << 28);
  const unsigned w = (unsigned)(u >> 32);
  const int E = (int)((w >> 20) & 0x7ff) - 896;
  unsigned b = (unsigned)(__double_as_longlong(x) >> 32) & 0x80000000u;
  if (E >= 255) b |= 0x7f800000u;
  else if (E > 0) b |= ((unsigned)E << 23) | ((unsigned)(u >> 29) & 0x7fffffu);
  return __uint_as_float(b);
}
// exact FP64 value of an FP32 (subnormals as zero)
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  unsigned hw = b & 0x80000000u, lw = 0u;
  if (e == 255u) hw |= 0x7ff00000u | ((b & 0x7fffffu) ? 0x80000u : 0u);
  else if (e) { hw |= ((e + 896u) << 20) | ((b >> 3) & 0xfffffu); lw = b << 29; }
  return __hiloint2double((int)hw, (int)lw);
}

// ---- operand splitting ------------------------------------------------------------
// f = hi + lo + O(2^-22 |f|) with hi, lo TF32 (round to nearest, ties away: cvt.rna);
// f - hi is exact in FP32
__device__ __forceinline__ void split_tf32(float f, uint32_t* hi, uint32_t* lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
  const float r = f - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
  *hi = h;
  *lo = l;
}
// f = hi + lo + O(2^-17 |f|) with hi, lo BF16 (round to nearest even)
__device__ __forceinline__ void split_bf16(float f, uint16_t* hi, uint16_t* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  const __nv_bfloat16 l = __float2bfloat16_rn(f - __bfloat162float(h));
  *hi = __bfloat16_as_ushort(h);
  *lo = __bfloat16_as_ushort(l);
}

// byte offset of element (row, kbyte) in the operand layout above, K extent KB bytes
__host__ __device__ __forceinline__ uint32_t op_off(int row, int kbyte, int KB) {
  return (uint32_t)((row >> 3) * (8 * KB) + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15));
}

}  // namespace tc
}  // namespace dd
