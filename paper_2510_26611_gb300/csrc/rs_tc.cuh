// 5th-generation tensor core (tcgen05) building blocks for the W-form contraction,
// in inline PTX for sm_100-family GPUs: shared-memory matrix descriptors, the
// instruction descriptor of a BF16 x BF16 -> FP32 MMA, Tensor Memory (TMEM)
// allocation, MMA issue with completion tracked by an mbarrier, TMEM loads, and the
// exact BF16 slicing that lets FP32-accumulating MMAs reach float-pair accuracy.
//
// Slicing (the splitting idea of Ozaki et al., "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012): a row x (float pairs) is scaled by a
// power of two 2^(5-E) so that |x| < 32, then written as kSlices = 5 integers
// d_0 + d_1 2^-8 + d_2 2^-16 + d_3 2^-24 + d_4 2^-32 (|d_0| <= 32, |d_j| <= 128, each
// exact in BF16, stored with its weight 2^-8j).  A product of two rows is the sum of
// the slice products (i, j); those with i + j <= 4 are formed, in two FP32
// accumulators of TMEM:
//   diagonals 0 and 1: multiples of 2^-8 whose K-sums stay below 2^15 -> exact;
//   diagonals 2 to 4:  terms ~2^-14 below the top, rounded in FP32.
// The two are combined with an error-free sum into a float pair.  The result
// carries ~2^-33 of K times the row and column maxima (the second accumulator's
// rounding and the dropped products with i + j >= 5, measured on an FP32-accumulated
// CPU emulation of the scheme); the CUDA-core pair arithmetic carries ~2^-47.  Two
// accumulators keep a tile within 128 TMEM columns, so four CTAs share an SM.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "rs_common.cuh"

namespace rs {
namespace tc {

constexpr int kSlices = 5;          // BF16 slices per operand
constexpr int kTopBits = 5;         // |top slice| <= 2^kTopBits
constexpr int kTileRows = 128;      // MMA M: atoms per tile
constexpr uint32_t kLBO = 128;      // bytes between core matrices adjacent in K

__host__ __device__ constexpr int kp_of(int RP) { return (RP + 15) / 16 * 16; }
__host__ __device__ constexpr int np_of(int RP) { return (2 * RP + 15) / 16 * 16; }

// Tile geometry of the W-form MMA for padded Tucker rank RP.  B holds, for one
// axis-3 cell, W row a at column 2a and D row a at column 2a + 1 (K = the axis-2
// index b), so one 16-column TMEM load returns eight (W, D) column pairs.
template <int RP>
struct Shape {
    static constexpr int KP = kp_of(RP);                    // K padded to the MMA K step
    static constexpr int NP = np_of(RP);                    // N (multiple of 16 for M = 128)
    static constexpr uint32_t SBO = KP * 16;                // bytes between 8-row groups
    static constexpr uint32_t A_SLICE = kTileRows * KP * 2; // one slice of a 128-row A tile
    static constexpr uint32_t B_SLICE = NP * KP * 2;
    static constexpr uint32_t B_BYTES = kSlices * B_SLICE;  // B image of one cell
};

// Byte offset of element (row, k) in the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes stored contiguously, K-adjacent core matrices kLBO
// bytes apart, 8-row groups sbo bytes apart.
__host__ __device__ constexpr uint32_t kmajor_offset(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * kLBO + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), no negation, both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor: start address >> 4 in bits 0-13, leading-dimension
// byte offset >> 4 in 16-29, stride-dimension byte offset >> 4 in 32-45, descriptor
// version 1 in bits 46-47, base offset 0, layout type 0 (no swizzle) in bits 61-63.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp; the base
// address is written to *slot in shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy writes to shared memory made visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

// Waits for phase `parity` of the barrier to complete, giving up after ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it >= 64) __nanosleep(128);
    }
    return false;
}

// Bulk copy (TMA, no tensor map) of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// One arrival on the barrier (release: this thread's earlier writes are visible to a
// thread that then waits on the phase).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One arrival on the barrier that also announces `bytes` of bulk-copy transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// D[tmem] (+)= A * B^T for one 128 x N x 16 step; accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the barrier once every MMA this thread has issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Power-of-two scale of a row: returns s = 2^(kTopBits-E) with max |x_h| < 2^E (so
// |x s| < 32) and its inverse; a row whose maximum is 0 or below 2^-119 gets s = 0
// (all slices 0).
__device__ __forceinline__ void row_scale(float m, float& s, float& inv) {
    const int be = (__float_as_int(m) >> 23) & 0xFF;  // m = 1.f * 2^(be-127) < 2^(be-126)
    if (m == 0.f || be < 8) {
        s = 0.f;
        inv = 0.f;
        return;
    }
    s = __int_as_float((127 + 126 + kTopBits - be) << 23);  // 2^(kTopBits - E), E = be - 126
    inv = __int_as_float((be - 126 - kTopBits + 127) << 23);  // 2^(E - kTopBits)
}

// The weighted slices of one scaled pair value y (|y| < 32): d_0 + d_1 2^-8 + ... +
// d_4 2^-32 with every d_j an integer.  Each remainder step is exact; the low word
// enters at slice 2 (one rounding at ~2^-33 of y's unit).
__device__ __forceinline__ void slice5(dev::F2 y, float (&o)[kSlices]) {
    const float d0 = rintf(y.h);
    float t = __fmul_rn(__fsub_rn(y.h, d0), 256.f);
    const float d1 = rintf(t);
    t = __fmaf_rn(__fsub_rn(t, d1), 256.f, __fmul_rn(y.l, 65536.f));
    const float d2 = rintf(t);
    t = __fmul_rn(__fsub_rn(t, d2), 256.f);
    const float d3 = rintf(t);
    t = __fmul_rn(__fsub_rn(t, d3), 256.f);
    const float d4 = rintf(t);
    o[0] = d0;
    o[1] = __fmul_rn(d1, 0x1p-8f);
    o[2] = __fmul_rn(d2, 0x1p-16f);
    o[3] = __fmul_rn(d3, 0x1p-24f);
    o[4] = __fmul_rn(d4, 0x1p-32f);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Writes row `row` of an A tile (kSlices slices of kTileRows x KP BF16, K-major) from
// RP pair values x (entries RP..KP-1 are zero).  Returns the row's inverse scale.
template <int RP>
__device__ __forceinline__ float write_row(const dev::F2 (&x)[RP], uint8_t* tile, int row) {
    using S = Shape<RP>;
    float m = 0.f;
#pragma unroll
    for (int b = 0; b < RP; ++b) m = fmaxf(m, fabsf(x[b].h));
    float s, inv;
    row_scale(m, s, inv);
#pragma unroll
    for (int kk = 0; kk < S::KP / 8; ++kk) {
        uint32_t w[kSlices][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float lo[kSlices], hi[kSlices];
            const int b0 = kk * 8 + e, b1 = b0 + 1;
            if (b0 < RP) {
                slice5(dev::F2{__fmul_rn(x[b0 < RP ? b0 : 0].h, s), __fmul_rn(x[b0 < RP ? b0 : 0].l, s)}, lo);
            } else {
#pragma unroll
                for (int j = 0; j < kSlices; ++j) lo[j] = 0.f;
            }
            if (b1 < RP) {
                slice5(dev::F2{__fmul_rn(x[b1 < RP ? b1 : 0].h, s), __fmul_rn(x[b1 < RP ? b1 : 0].l, s)}, hi);
            } else {
#pragma unroll
                for (int j = 0; j < kSlices; ++j) hi[j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < kSlices; ++j) w[j][e / 2] = pack_bf16x2(lo[j], hi[j]);
        }
#pragma unroll
        for (int j = 0; j < kSlices; ++j)
            *reinterpret_cast<uint4*>(tile + j * S::A_SLICE + kmajor_offset(row, kk * 8, S::SBO)) =
                make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
    }
    return inv;
}

// Zero row of an A tile.
template <int RP>
__device__ __forceinline__ void zero_row(uint8_t* tile, int row) {
    using S = Shape<RP>;
#pragma unroll
    for (int kk = 0; kk < S::KP / 8; ++kk)
#pragma unroll
        for (int j = 0; j < kSlices; ++j)
            *reinterpret_cast<uint4*>(tile + j * S::A_SLICE + kmajor_offset(row, kk * 8, S::SBO)) =
                make_uint4(0u, 0u, 0u, 0u);
}

// Accumulators of one contraction in TMEM: columns [0, NP) diagonals 0-1 (exact),
// [NP, 2NP) diagonals 2-4.
constexpr int kAccs = 2;

// The fifteen slice products (i, j) with i + j <= 4, in a fixed order, each into the
// accumulator of its diagonal (the first product of an accumulator overwrites it).
template <int RP>
__device__ __forceinline__ void issue_products(uint32_t tmem_d, uint32_t a_saddr, uint32_t b_saddr) {
    using S = Shape<RP>;
    constexpr uint32_t idesc = idesc_bf16_f32(kTileRows, S::NP);
    constexpr int kI[15] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};
    constexpr int kJ[15] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0};
#pragma unroll
    for (int p = 0; p < 15; ++p) {
        const int acc = p < 3 ? 0 : 1;
        const bool first = p == 0 || p == 3;
        const uint32_t d = tmem_d + (uint32_t)(acc * S::NP);
#pragma unroll
        for (int ks = 0; ks < S::KP / 16; ++ks) {
            const uint64_t ad = smem_desc(a_saddr + kI[p] * S::A_SLICE + ks * 2 * kLBO, kLBO, S::SBO);
            const uint64_t bd = smem_desc(b_saddr + kJ[p] * S::B_SLICE + ks * 2 * kLBO, kLBO, S::SBO);
            mma_bf16(d, ad, bd, idesc, (first && ks == 0) ? 0u : 1u);
        }
    }
}

// Pair value of one output column: (acc0 + acc1) * scale, the sum taken error-free
// (scale is a power of two).
__device__ __forceinline__ dev::F2 combine(float acc0, float acc1, float scale) {
    float s, e;
    dev::two_sum(acc0, acc1, s, e);
    return dev::F2{__fmul_rn(s, scale), __fmul_rn(e, scale)};
}

// Two 16-column TMEM loads (32 lanes x 32 bits: thread t reads lane base + t, one load
// per accumulator) and the wait for them, in one statement so no use of the values
// precedes the wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float (&a)[16], float (&b)[16]) {
    uint32_t x[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
        "[%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]),
          "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]), "=r"(x[15]),
          "=r"(x[16]), "=r"(x[17]), "=r"(x[18]), "=r"(x[19]), "=r"(x[20]), "=r"(x[21]), "=r"(x[22]),
          "=r"(x[23]), "=r"(x[24]), "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]), "=r"(x[29]),
          "=r"(x[30]), "=r"(x[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        a[i] = __uint_as_float(x[i]);
        b[i] = __uint_as_float(x[16 + i]);
    }
}

#endif  // __CUDACC__

}  // namespace tc
}  // namespace rs
