// PTX helpers for the tcgen05 / TMEM / bulk-copy / mbarrier machinery of sm_100-family GPUs,
// used by the tensor-core contraction (contract_tc.cu).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

namespace ssht {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// A-operand tiles of the contraction: 128 rows x 32 K values.  In shared memory two split parts of
// 16 KB each; in global memory one part of FP32 values for the 3xTF32 form (the contraction splits
// them on arrival) and both parts for the split-BF16 form.
constexpr int kTileRows = 128, kTileK = 32;
constexpr int kAPart = kTileRows * kTileK * 4;
constexpr int kATile = 2 * kAPart;

// Byte offset of element (row, kbyte) in a K-major tile with 128-byte rows in the SWIZZLE_128B
// layout: 8-row x 128-byte atoms stacked along rows, the 16-byte chunk c of row r stored at
// chunk c ^ (r mod 8).  Tiles start on 1024-byte boundaries.
__host__ __device__ __forceinline__ uint32_t sw128(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ row) & 7) << 4) + (kbyte & 15));
}

// Shared-memory matrix descriptor: start address, stride between 8-row groups (1024 bytes),
// descriptor version 1, SWIZZLE_128B.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N.
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Instruction descriptor: D = F32, A = B = BF16 (kind::f16), both K-major, shape M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Orders this thread's shared-memory writes (generic proxy) before later reads of the tensor core
// (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase of the given parity: false once limit_ns of device time has passed
// (checked after every poll) or, if abort is not null, once *abort is set (every 256 polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, long long limit_ns) {
  const uint32_t b = smem_u32(bar);
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned i = 1;; ++i) {
    if (mbar_test(b, parity)) return true;
    if ((i & 255u) == 0u && abort && *abort) return false;
    if ((long long)(globaltimer() - t0) > limit_ns) return false;
  }
}

// Waits for work this CTA has already issued (bulk copies, tensor-core operations) before it
// leaves: not cut short by the abort flag, bounded by two seconds.
constexpr long long kDrainNs = 2000000000ll;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared, completion counted in bytes on an mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::tf32, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 with BF16 operands (K = 16 per instruction).
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// Arrive on an mbarrier once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// x = hi + lo with hi rounded to TF32 (10 explicit mantissa bits, round to nearest) and lo the
// remainder rounded the same way: the pair carries about 22 significant bits of x.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split_tf32(float x, float* hi, float* lo) {
  *hi = tf32_round(x);
  *lo = tf32_round(x - *hi);
}

// x = h + m + l with each part rounded to BF16 (8 significant bits, round to nearest): the three
// parts carry about 24 significant bits of x; each remainder is exact in FP32.
__device__ __forceinline__ void split_bf16x3(float x, uint16_t* h, uint16_t* m, uint16_t* l) {
  const __nv_bfloat16 a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  const __nv_bfloat16 c = __float2bfloat16_rn(r2);
  *h = __bfloat16_as_ushort(a);
  *m = __bfloat16_as_ushort(b);
  *l = __bfloat16_as_ushort(c);
}

// Writes element (row, k), k < 32, of a K-chunk operand tile as it is stored in global memory
// (128-byte swizzled rows).  TF32 form: one part, the FP32 value itself (split into hi + lo by
// the contraction when the tile arrives in shared memory).  BF16 split: part 0 = [h | m] (2-byte
// elements, k at byte 2k and 64 + 2k), part 1 = [l | 0], each part part_bytes long.
template <bool BF>
__device__ __forceinline__ void put_split(uint8_t* tile, int part_bytes, int row, int k, float x) {
  if constexpr (BF) {
    uint16_t h, m, l;
    split_bf16x3(x, &h, &m, &l);
    *(uint16_t*)(tile + sw128(row, 2 * k)) = h;
    *(uint16_t*)(tile + sw128(row, 64 + 2 * k)) = m;
    *(uint16_t*)(tile + part_bytes + sw128(row, 2 * k)) = l;
    *(uint16_t*)(tile + part_bytes + sw128(row, 64 + 2 * k)) = 0;
  } else {
    (void)part_bytes;
    *(float*)(tile + sw128(row, 4 * k)) = x;
  }
}

// Global parts of an operand tile: 1 for the TF32 form, 2 for split-BF16.
template <bool BF> constexpr int kParts = BF ? 2 : 1;

// Splits, in shared memory, the FP32 values of an arrived 3xTF32 operand region into hi (in place)
// and lo (lo_offset bytes further on), 16 bytes a step; the layout's swizzle permutes whole
// 16-byte chunks, so the split goes position by position.  Threads t of nt take steps t, t + nt, ...
__device__ __forceinline__ void split_region_tf32(uint8_t* region, int bytes, int lo_offset, int t, int nt) {
  for (int o = 16 * t; o < bytes; o += 16 * nt) {
    float4 x = *(const float4*)(region + o), h, l;
    split_tf32(x.x, &h.x, &l.x);
    split_tf32(x.y, &h.y, &l.y);
    split_tf32(x.z, &h.z, &l.z);
    split_tf32(x.w, &h.w, &l.w);
    *(float4*)(region + o) = h;
    *(float4*)(region + lo_offset + o) = l;
  }
}

}  // namespace tc
}  // namespace ssht
