// Blackwell (sm_100a / sm_103a) tensor-core helpers: TMEM allocation,
// shared-memory matrix descriptors, tcgen05.mma (kind::f16, bf16 inputs,
// float32 accumulation in TMEM), commit to an mbarrier with a bounded wait,
// and TMEM -> register loads.  Inline PTX only.
//
// Operand layout used throughout (K-major, no swizzle): an R x K bf16 tile
// is made of 8 x 8 "core matrices" (8 rows, 16 contiguous bytes of K each,
// 128 bytes per core matrix).  Element (r, k) lives at byte
//     (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2
// with LBO = 128 (K-adjacent core matrices contiguous) and SBO = 16 * K
// (one 8-row group holds all K / 8 core matrices of its rows).
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace tc {

CR_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major no-swizzle tile with K columns
CR_HD uint32_t kmajor_offset(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (16 * K) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// 64-bit shared-memory matrix descriptor (sm_100 layout): start address,
// leading-dimension byte offset (K direction) and stride byte offset (8-row
// groups), all in 16-byte units; version 1; no swizzle.
CR_D uint64_t make_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, LBO mode 0, swizzle none
}

// 32-bit instruction descriptor of tcgen05.mma kind::f16: D float32, A and
// B bf16, both K-major, M x N tile.
CR_HD uint32_t make_idesc_bf16(int M, int N) {
    uint32_t d = 0;
    d |= 1u << 4;                       // D format: float32
    d |= 1u << 7;                       // A format: bf16
    d |= 1u << 10;                      // B format: bf16
    d |= (uint32_t)(N >> 3) << 17;      // N / 8
    d |= (uint32_t)(M >> 4) << 24;      // M / 16
    return d;
}

// TMEM allocation by one full warp; the address lands in *slot (shared).
CR_D void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
CR_D void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
CR_D void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
CR_D void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
CR_D void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
CR_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// D[tmem] (+)= A * B, issued by one thread.
CR_D void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accum) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accum)
        : "memory");
}

// Make mbar track completion of this thread's earlier tcgen05 operations.
CR_D void commit(uint64_t* mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(mbar))
        : "memory");
}

CR_D void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count)
                 : "memory");
}
// Arm mbar for one arrival (this thread) plus `bytes` of asynchronous copies.
CR_D void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile(
        "{\n"
        ".reg .b64 st;\n"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n"
        "}\n" ::"r"(smem_u32(mbar)),
        "r"(bytes)
        : "memory");
}

// Bulk (non-tensor) copy global -> shared, completion counted on mbar in
// bytes.  Both addresses 16-byte aligned, size a multiple of 16.
CR_D void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

CR_D void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Wait for the phase with the given parity to complete, giving up after
// max_iter polls.  Returns false on timeout (the caller records an error and
// still releases its TMEM).
CR_D bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_iter) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < max_iter; ++it) {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.b32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 lanes x 32 bits, 16 consecutive columns per thread: warp w of a
// warpgroup reads TMEM lanes [32 (w % 4), +32); thread lane l gets row
// 32 (w % 4) + l, columns col .. col + 15.
CR_D void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
