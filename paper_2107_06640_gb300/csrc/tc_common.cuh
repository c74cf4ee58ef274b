// tcgen05 helpers (sm_103a): shared-memory and instruction descriptors for
// kind::tf32 with K-major, non-swizzled operands, TMEM allocation, MMA issue,
// commit to an mbarrier and bounded waits.
//
// Operand layout in shared memory ("canonical K-major, no swizzle"): an R x K
// fp32 matrix is stored as core matrices of 8 rows x 4 values (16 bytes per
// row, 128 bytes per core matrix); element (r, k) sits at float offset
//   ((k/4) * (R/8) + r/8) * 32 + (r%8) * 4 + (k%4),
// so core matrices adjacent along M/N are 128 B apart (stride byte offset) and
// adjacent along K are (R/8)*128 B apart (leading byte offset).  One
// kind::tf32 MMA consumes K = 8 (two core matrices along K).
// Accumulator layout in TMEM: M = 128 puts row r in lane r; M = 64 puts rows
// 16w..16w+15 in lanes 32w..32w+15 (w = 0..3); column j of D is TMEM column j.
#pragma once
#include <cstdint>

namespace adg {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__host__ __device__ __forceinline__ int canon(int r, int k, int R) {
  return ((k >> 2) * (R >> 3) + (r >> 3)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;
}

// instruction descriptor: D f32, A and B tf32, both K-major, dense
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// round-toward-zero to tf32 (keep sign, exponent and 10 mantissa bits)
__host__ __device__ __forceinline__ float tf32_trunc(float x) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
#else
  uint32_t u;
  __builtin_memcpy(&u, &x, 4);
  u &= 0xFFFFE000u;
  __builtin_memcpy(&x, &u, 4);
  return x;
#endif
}

// MMA with the A operand in TMEM (lane = row, one tf32 per column)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(db), "r"(idesc), "r"(acc));
}

// 3xTF32 product chain into d (M = 128): A in TMEM (hi at column ah, lo at
// al) times B^T, B canonical K-major N x K in shared memory (hi at byte
// address bh, lo at bl); K / 8 steps of A_hi B_hi + A_hi B_lo + A_lo B_hi.
// The descriptors are built once; a step advances their start address.
// K0 (a multiple of 8) starts the chain part-way through K.
template <int N, int K, int K0 = 0>
__device__ __forceinline__ void mma3_ts(uint32_t d, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                        bool acc_first) {
  constexpr uint32_t idesc = idesc_tf32(128, N);
  constexpr uint32_t lbo = (N / 8) * 128;
  const uint64_t dh0 = sdesc(bh, lbo, 128), dl0 = sdesc(bl, lbo, 128);
#pragma unroll
  for (int kk = K0 / 8; kk < K / 8; ++kk) {
    const uint64_t step = (uint64_t)((kk * 2 * lbo) >> 4);
    mma_ts(d, ah + 8 * kk, dh0 + step, idesc, (kk > K0 / 8 || acc_first) ? 1u : 0u);
    mma_ts(d, ah + 8 * kk, dl0 + step, idesc, 1u);
    mma_ts(d, al + 8 * kk, dh0 + step, idesc, 1u);
  }
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

// one thread's arrival on the mbarrier, announcing `bytes` of asynchronous copies
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// bulk copy (TMA engine, non-tensor) global -> this CTA's shared memory, both
// 16-byte aligned, bytes a multiple of 16; completes on the mbarrier
__device__ __forceinline__ void bulk_load(void* sm, const void* g, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(sm)),
               "l"(g), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}
// thread 0 of the CTA: `bytes` from global to shared memory in bulk copies of
// at most 32 KB, all completing on `mbar` (initialised, phase 0)
__device__ __forceinline__ void bulk_load_all(void* sm, const void* g, uint32_t bytes, uint64_t* mbar) {
  mbar_expect_tx(mbar, bytes);
  for (uint32_t o = 0; o < bytes; o += 32768u)
    bulk_load(static_cast<char*>(sm) + o, static_cast<const char*>(g) + o, bytes - o < 32768u ? bytes - o : 32768u,
              mbar);
}

// wait for phase `parity` of the mbarrier; false if the bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int max_iter) {
  for (int it = 0; it < max_iter; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (ok) return true;
  }
  return false;
}

// bring [p, p + bytes) into L2 ahead of use (16-byte aligned, bytes a multiple
// of 16), in pieces of at most 8 KB
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (uint32_t o = 0; o < bytes; o += 8192u) {
    const uint32_t n = bytes - o < 8192u ? bytes - o : 8192u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + o), "r"(n) : "memory");
  }
}

// asynchronous 4-byte copy global -> shared (cp.async; committed and waited
// for with cp.async.commit_group / cp.async.wait_group)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory"); }

// the same for any span: only its 16-byte aligned interior (a hint; the
// bytes at either end that share a 16-byte unit with the span's neighbours
// are left out)
__device__ __forceinline__ void prefetch_l2_inner(const void* p, uint32_t bytes) {
  const uintptr_t a0 = ((uintptr_t)p + 15) & ~(uintptr_t)15, a1 = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (a1 > a0) prefetch_l2(reinterpret_cast<const void*>(a0), (uint32_t)(a1 - a0));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
// bulk copy shared -> global (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_store(void* g, const void* sm, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g), "r"(smem_u32(sm)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source of every committed bulk copy has been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk copy is complete
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "n"(NCOLS));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOLS));
}

// three groups of 8 consecutive fp32 columns of this warp's lanes (one wait)
__device__ __forceinline__ void ld3x8(uint32_t t0, uint32_t t1, uint32_t t2, float o[24]) {
  uint32_t r[24];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
      : "r"(t0), "r"(t1), "r"(t2));
#pragma unroll
  for (int j = 0; j < 24; ++j) o[j] = __uint_as_float(r[j]);
}

// 8 consecutive fp32 columns of this warp's lanes
__device__ __forceinline__ void ld8(uint32_t t, float o[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(t));
#pragma unroll
  for (int j = 0; j < 8; ++j) o[j] = __uint_as_float(r[j]);
}

// 8 values of this lane's row -> tf32 hi at column th, lo (the remainder) at column tl
__device__ __forceinline__ void st_split8(uint32_t th, uint32_t tl, const float x[8]) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float hh = tf32_trunc(x[j]);
    h[j] = __float_as_uint(hh);
    l[j] = __float_as_uint(x[j] - hh);
  }
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(th), "r"(h[0]),
               "r"(h[1]), "r"(h[2]), "r"(h[3]), "r"(h[4]), "r"(h[5]), "r"(h[6]), "r"(h[7]));
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(tl), "r"(l[0]),
               "r"(l[1]), "r"(l[2]), "r"(l[3]), "r"(l[4]), "r"(l[5]), "r"(l[6]), "r"(l[7]));
}


}  // namespace tc
}  // namespace adg
