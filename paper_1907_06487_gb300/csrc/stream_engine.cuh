// Bulk-copy streaming of CRS row blocks into shared memory (sm_100+ / sm_103a).
//
// A row block is a run of consecutive rows whose nonzeros (at most kChunk)
// and row pointers fit one pipeline stage.  One elected thread of the block
// issues cp.async.bulk copies (the TMA engine's 1-D form, no tensor map) of
// the block's val, col and row_ptr slices into a stage and arms the stage's
// mbarrier with the byte count; the other threads wait on the mbarrier's
// phase parity.  Copies start at 16-byte boundaries: slices are widened to
// multiples of 4 elements at both ends, and every streamed array is padded
// by kPad elements on the device so the widened tail stays in bounds.
//
// Every wait is bounded: after kSpinLimit polls the kernel records
// RACE_ERR_TIMEOUT in a device status word and leaves its loop.
#pragma once
#include <cstdint>

namespace race_dev {

constexpr int kChunk = 1024;       // max nonzeros per row block
constexpr int kRowsMax = 256;      // max rows per row block
constexpr int kPad = 8;            // device padding (elements) of streamed arrays
constexpr int kStages = 3;         // pipeline depth
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Returns false if the wait gave up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Returns false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One pipeline stage: widened slices of val, col and row_ptr.
template <typename VT>
struct Stage {
    VT val[kChunk + 8];
    int32_t col[kChunk + 8];
    int32_t rp[kRowsMax + 8];
};

// Geometry of one row block.
struct BlockGeom {
    int32_t r0, r1;    // rows [r0, r1)
    int32_t s, e;      // nonzeros [s, e)
    int32_t s_al;      // s rounded down to a multiple of 4
    int32_t r0_al;     // r0 rounded down to a multiple of 4
    uint32_t n_el;     // widened nonzero count (multiple of 4)
    uint32_t n_rp;     // widened row-pointer count (multiple of 4)
};

__device__ __forceinline__ BlockGeom block_geom(const int32_t* __restrict__ blk_row, const int32_t* __restrict__ rp,
                                                int64_t blk) {
    BlockGeom g;
    g.r0 = __ldg(blk_row + blk);
    g.r1 = __ldg(blk_row + blk + 1);
    g.s = __ldg(rp + g.r0);
    g.e = __ldg(rp + g.r1);
    g.s_al = g.s & ~3;
    g.r0_al = g.r0 & ~3;
    g.n_el = static_cast<uint32_t>(((g.e - g.s_al) + 3) & ~3);
    g.n_rp = static_cast<uint32_t>(((g.r1 + 1 - g.r0_al) + 3) & ~3);
    return g;
}

// Issue the copies of one block into a stage (one thread).
template <typename VT>
__device__ __forceinline__ void issue_block(Stage<VT>* st, uint64_t* bar, const BlockGeom& g, const VT* val,
                                            const int32_t* col, const int32_t* rp) {
    const uint32_t bytes = g.n_el * (sizeof(VT) + sizeof(int32_t)) + g.n_rp * sizeof(int32_t);
    mbar_expect_tx(bar, bytes);
    if (g.n_el) {
        bulk_g2s(st->val, val + g.s_al, g.n_el * sizeof(VT), bar);
        bulk_g2s(st->col, col + g.s_al, g.n_el * sizeof(int32_t), bar);
    }
    bulk_g2s(st->rp, rp + g.r0_al, g.n_rp * sizeof(int32_t), bar);
}

}  // namespace race_dev
