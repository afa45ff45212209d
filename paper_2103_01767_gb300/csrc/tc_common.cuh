// tc_common.cuh -- inline-PTX building blocks of the tensor-core convolutions: mbarriers with
// bounded waits, TMA tiled and bulk loads (cp.async.bulk[.tensor]), tcgen05 shared-memory and
// instruction descriptors, tcgen05.mma / commit, TMEM allocation and loads.
//
// Operand layouts are the canonical no-swizzle ones of tcgen05:
//   K-major:  core matrix = 8 rows (M or N) x 16 bytes of K; LBO = byte stride between core
//             matrices adjacent in K, SBO = byte stride between 8-row groups.
//   MN-major: core matrix = 8 rows of K x 16 bytes of M (or N); LBO = byte stride between
//             8-row groups of K, SBO = byte stride between 16-byte groups of M (or N).
// Both were checked element by element on the device (small-integer GEMMs, exact results).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ptylm {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after `limit` polls
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t i = 0; i < limit; ++i) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 4D tiled load: the box at coordinates (c0, c1, c2, c3) (innermost first) of the map into
// shared memory, completing on `bar`; out-of-range elements read as zero
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// contiguous copy of `bytes` (multiple of 16, both addresses 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// shared-memory matrix descriptor (no swizzle, version 1); the start address occupies the
// low 14 bits (address >> 4), so adding (byte offset >> 4) moves the start.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::f16: D F32, A and B BF16, M x N, majors (0 K, 1 MN)
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate `cols` TMEM columns (power of two >= 32), base address to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
// whole warp: 16 consecutive FP32 columns of the warp's 32 lanes (lane i of the warp reads
// TMEM lane 32 (warp % 4) + i)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
          "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
        : "r"(taddr)
        : "memory");
}

// x = hi + lo with hi = bf16(x), lo = bf16(x - hi): |x - hi - lo| <= 2^-18 |x|
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Feature-map pairs (hi, lo), channel-chunk major: [N][C/8][H][W][8] ("plain", par = 0) or
// split by pixel parity, [N][C/8][2][2][H/2][W/2][8] (par = 1).
// element offset of 8-channel chunk q at pixel (y, x) of image n
__device__ __forceinline__ size_t chunk_at(int par, int C8, int H, int W, int n, int y, int x, int q) {
    if (!par) return ((((size_t)n * C8 + q) * H + y) * W + x) * 8;
    return (((((size_t)n * C8 + q) * 4 + ((y & 1) << 1) + (x & 1)) * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1)) * 8;
}

__device__ __forceinline__ void store_pair8(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t o, const float* v) {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split_bf16(v[j], h[j], l[j]);
    *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(l);
}

// v[j] = hi + lo of the 8 channels of one chunk
__device__ __forceinline__ void load_pair8(const __nv_bfloat16* hi, const __nv_bfloat16* lo, size_t o, float* v) {
    __align__(16) __nv_bfloat16 h[8], l[8];
    *reinterpret_cast<uint4*>(h) = __ldg(reinterpret_cast<const uint4*>(hi + o));
    *reinterpret_cast<uint4*>(l) = __ldg(reinterpret_cast<const uint4*>(lo + o));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __bfloat162float(h[j]) + __bfloat162float(l[j]);
}

// m[j] = (hi + lo > 0) of 8 channels
__device__ __forceinline__ void load_mask8(const __nv_bfloat16* hi, const __nv_bfloat16* lo, size_t o, bool* m) {
    float v[8];
    load_pair8(hi, lo, o, v);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] = v[j] > 0.0f;
}

}  // namespace tc
}  // namespace ptylm
