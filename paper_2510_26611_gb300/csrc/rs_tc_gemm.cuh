// Float-pair-accurate GEMM on the 5th-generation tensor cores, for the GEMM-shaped
// steps of the Tucker build (RHOSVD, Sec. 1 and Algorithm TEP step 4): the block
// products Y = G Q of the subspace iteration on the per-axis Gram matrices.
//
// Exact slicing (the error-free splitting of Ozaki et al., Numer. Algorithms 59,
// 2012, with six slices): every operand value is scaled by a power of two so that
// |y| < 32 and written as y = sum_u d_u 2^(-8u), u = 0..5, with integers |d_0| <= 32,
// |d_1|, |d_2| <= 128 and |d_3|, |d_4|, |d_5| <= 256 (exact in BF16); the scale is
// taken per (row, 64-wide K chunk) of A and per (column, K chunk) of B.  The product
// of two values is the sum of the slice products d_u e_v 2^(-8(u+v)); the 21 with
// u + v <= 5 are formed by tcgen05 MMAs (BF16 x BF16 -> FP32), one TMEM accumulator
// per diagonal u + v.  Over a 64-wide K chunk a diagonal's sum is an integer of
// magnitude at most 64 * 147456 < 2^24 (diagonal 5, the largest), so the FP32
// accumulation is exact; the six diagonals are combined error-free into a float
// pair, scaled back and written per K chunk.  The dropped products u + v >= 6 and
// the last slice's remainder leave ~2^-45 of the chunk's row and column maxima:
// float-pair accuracy.  Everything runs on the FP32 pipes and the tensor cores: GB300
// executes FP64 at 1/64 of its FP32 rate, so the slicing takes float pairs apart with
// exact FP32 steps rather than doubles.
#pragma once

#include <cstdint>

#include "rs_common.cuh"
#include "rs_tc.cuh"

namespace rs {
namespace tcg {

constexpr int kS = 6;                 // slices per operand
constexpr int kM = 128;               // rows per tile (MMA M)
constexpr int kK = 64;                // K chunk (columns of A / rows of B per MMA group)
constexpr uint32_t kSBO = kK * 16;    // bytes between 8-row groups (K-major, no swizzle)
constexpr uint32_t kSliceA = kM * kK * 2;  // one slice of an A tile (16 KB)

template <int NP>
struct GemmShape {
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "N of the sliced GEMM");
    static constexpr uint32_t SLICE_B = NP * kK * 2;
    static constexpr uint32_t A_BYTES = kS * kSliceA;
    static constexpr uint32_t B_BYTES = kS * SLICE_B;
    static constexpr uint32_t BAR_OFF = A_BYTES + B_BYTES;    // [0] loads, [1] MMAs
    static constexpr uint32_t SLOT_OFF = BAR_OFF + 16;
    static constexpr uint32_t BINV_OFF = SLOT_OFF + 16;        // the chunk's column scales
    static constexpr uint32_t SMEM = BINV_OFF + NP * 4;
    static constexpr uint32_t COLS = kS * NP;  // one accumulator per diagonal
    static constexpr uint32_t NCOL = COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
};

// Six slices of a float pair (h, l) already scaled to |h + l| < 32, with exact FP32
// steps: the high word is cut into d_0 ... d_5 (each step subtracts an integer from
// an exact remainder and multiplies by 256), the low word, which lies below 2^-19 of
// the scale, from slice 3 on in the same way, and the two streams add slice by slice
// (|d_3| <= 128 + 16, |d_4|, |d_5| <= 256).
__device__ __forceinline__ void slice6(float h, float l, float (&d)[kS]) {
    float r = h;
#pragma unroll
    for (int u = 0; u < kS; ++u) {
        const float q = rintf(r);
        d[u] = q;
        r = __fmul_rn(__fsub_rn(r, q), 256.f);
    }
    r = __fmul_rn(l, 16777216.f);  // l in units of slice 3 (2^-24)
#pragma unroll
    for (int u = 3; u < kS; ++u) {
        const float q = rintf(r);
        d[u] = __fadd_rn(d[u], q);
        r = __fmul_rn(__fsub_rn(r, q), 256.f);
    }
}

// sum_d x_d 2^(-8d) of the six diagonal sums (exact integers in FP32), smallest term
// first, into a float pair; every weight is a power of two, so each product is exact.
__device__ __forceinline__ dev::F2 combine6(float x0, float x1, float x2, float x3, float x4, float x5) {
    dev::F2 s{__fmul_rn(x5, 0x1p-40f), 0.f};
    s = dev::df_add(s, dev::F2{__fmul_rn(x4, 0x1p-32f), 0.f});
    s = dev::df_add(s, dev::F2{__fmul_rn(x3, 0x1p-24f), 0.f});
    s = dev::df_add(s, dev::F2{__fmul_rn(x2, 0x1p-16f), 0.f});
    s = dev::df_add(s, dev::F2{__fmul_rn(x1, 0x1p-8f), 0.f});
    return dev::df_add(s, dev::F2{x0, 0.f});
}

// Three 8-column TMEM loads (32 lanes x 32 bits: thread t reads lane base + t) at
// t, t + stride, t + 2 stride and the wait for them, in one statement so no use of the
// values precedes the wait.
__device__ __forceinline__ void tmem_ld8x3(uint32_t t, uint32_t stride, float (&a)[8], float (&b)[8],
                                           float (&c)[8]) {
    uint32_t x[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]),
          "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]), "=r"(x[15]),
          "=r"(x[16]), "=r"(x[17]), "=r"(x[18]), "=r"(x[19]), "=r"(x[20]), "=r"(x[21]), "=r"(x[22]),
          "=r"(x[23])
        : "r"(t), "r"(t + stride), "r"(t + 2 * stride)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = __uint_as_float(x[i]);
        b[i] = __uint_as_float(x[8 + i]);
        c[i] = __uint_as_float(x[16 + i]);
    }
}

// Power-of-two scale for a chunk whose largest magnitude is m: s with m s < 32, and
// 1/s; zero chunks (or m below 2^-119) get s = inv = 0.
__device__ __forceinline__ void chunk_scale(float m, float& s, float& inv) { tc::row_scale(m, s, inv); }

// A operand: the n x n matrices G[ax] (float pairs, row-major), cut into tiles of
// kM rows x kK columns; tile (ax, mt, kc) holds its kS slices contiguously
// (slice u at u * kSliceA, each in the canonical K-major layout) at
//   out + ((ax * MT + mt) * KC + kc) * kS * kSliceA;
// ainv[(ax * KC + kc) * (MT * kM) + row] = 1 / scale of (row, chunk).  Rows and
// columns beyond n are zero.  CTA: kM threads (one row each) of tile (mt, kc, ax).
__global__ void __launch_bounds__(kM) k_slice_rows(int n, int MT, int KC, const float2* __restrict__ G,
                                                    uint8_t* __restrict__ out, float* __restrict__ ainv) {
    const int mt = blockIdx.x, kc = blockIdx.y, ax = blockIdx.z;
    const int row = threadIdx.x, i = mt * kM + row;
    const int k0 = kc * kK;
    const float2* Gr = G + ((size_t)ax * n + (size_t)min(i, n - 1)) * n;
    float m = 0.f;
    if (i < n)
        for (int k = k0; k < min(n, k0 + kK); ++k) m = fmaxf(m, fabsf(Gr[k].x));
    float s, inv;
    chunk_scale(m, s, inv);
    ainv[((size_t)ax * KC + kc) * ((size_t)MT * kM) + i] = inv;
    uint8_t* tile = out + (((size_t)ax * MT + mt) * KC + kc) * (size_t)kS * kSliceA;
#pragma unroll 1
    for (int g = 0; g < kK / 8; ++g) {
        uint32_t w[kS][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float lo[kS], hi[kS];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k0 + g * 8 + e + h;
                const float2 v = (i < n && k < n) ? Gr[k] : make_float2(0.f, 0.f);
                slice6(__fmul_rn(v.x, s), __fmul_rn(v.y, s), h ? hi : lo);
            }
#pragma unroll
            for (int u = 0; u < kS; ++u) w[u][e / 2] = tc::pack_bf16x2(lo[u], hi[u]);
        }
#pragma unroll
        for (int u = 0; u < kS; ++u)
            *reinterpret_cast<uint4*>(tile + u * kSliceA + tc::kmajor_offset(row, g * 8, kSBO)) =
                make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
    }
}

// B operand: the n x NP matrices Q[ax] (float pairs, row-major: K = the row index), cut
// into K chunks; chunk (ax, kc) holds its kS slices (N = NP rows of the canonical
// K-major layout, slice v at v * SLICE_B) at out + (ax * KC + kc) * B_BYTES;
// binv[(ax * KC + kc) * NP + j] = 1 / scale of (column j, chunk).  Rows beyond n are
// zero.  CTA: NP threads (one column each) of chunk (kc, ax).
template <int NP>
__global__ void __launch_bounds__(NP) k_slice_cols(int n, int KC, const float2* __restrict__ Q,
                                                    uint8_t* __restrict__ out, float* __restrict__ binv) {
    using Sh = GemmShape<NP>;
    const int kc = blockIdx.x, ax = blockIdx.y, j = threadIdx.x;
    const int k0 = kc * kK;
    const float2* Qa = Q + (size_t)ax * n * NP;
    float m = 0.f;
    for (int k = k0; k < min(n, k0 + kK); ++k) m = fmaxf(m, fabsf(Qa[(size_t)k * NP + j].x));
    float s, inv;
    chunk_scale(m, s, inv);
    binv[((size_t)ax * KC + kc) * NP + j] = inv;
    uint8_t* tile = out + ((size_t)ax * KC + kc) * Sh::B_BYTES;
#pragma unroll 1
    for (int g = 0; g < kK / 8; ++g) {
        uint32_t w[kS][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float lo[kS], hi[kS];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k0 + g * 8 + e + h;
                const float2 v = k < n ? Qa[(size_t)k * NP + j] : make_float2(0.f, 0.f);
                slice6(__fmul_rn(v.x, s), __fmul_rn(v.y, s), h ? hi : lo);
            }
#pragma unroll
            for (int v = 0; v < kS; ++v) w[v][e / 2] = tc::pack_bf16x2(lo[v], hi[v]);
        }
#pragma unroll
        for (int v = 0; v < kS; ++v)
            *reinterpret_cast<uint4*>(tile + v * Sh::SLICE_B + tc::kmajor_offset(j, g * 8, kSBO)) =
                make_uint4(w[v][0], w[v][1], w[v][2], w[v][3]);
    }
}

// Y partial of one (row tile, K chunk, axis): Yp[kc][ax][i][j] = sum over the chunk's
// k of A[i][k] B[k][j], as a float pair (rows i < n).  CTA: kGemmThreads threads; thread
// 0 loads the operands by bulk copies and issues the MMAs; then warps w and w + 4 read
// TMEM lanes 32 (w mod 4) .. + 31 (thread = row) and finish alternate 16-column blocks
// of the row (two warps per scheduler for the epilogue, where six diagonals are
// combined per column).  On a load or MMA that does not complete
// within the bounded wait the tile's outputs are NaN and *err is set.
constexpr int kGemmThreads = 2 * kM;

template <int NP>
__global__ void __launch_bounds__(kGemmThreads, 1) k_tc_gemm(int n, int MT, int KC, const uint8_t* __restrict__ As,
                                                    const float* __restrict__ ainv, const uint8_t* __restrict__ Bs,
                                                    const float* __restrict__ binv, float2* __restrict__ Yp,
                                                    int* __restrict__ err) {
    using Sh = GemmShape<NP>;
    extern __shared__ __align__(16) uint8_t smem_g[];
    const int mt = blockIdx.x, kc = blockIdx.y, ax = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_g + Sh::BAR_OFF);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem_g + Sh::SLOT_OFF);
    if (warp == 0) tc::tmem_alloc(slot, Sh::NCOL);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(bar + 1, 1);
        // the tile's A slices and the chunk's B slices (contiguous in global memory)
        // by bulk copies, one per slice
        const uint8_t* ga = As + (((size_t)ax * MT + mt) * KC + kc) * Sh::A_BYTES;
        const uint8_t* gb = Bs + ((size_t)ax * KC + kc) * Sh::B_BYTES;
        tc::mbar_arrive_expect_tx(bar, Sh::A_BYTES + Sh::B_BYTES);
#pragma unroll
        for (int u = 0; u < kS; ++u) {
            tc::bulk_g2s(smem_g + u * kSliceA, ga + u * kSliceA, kSliceA, bar);
            tc::bulk_g2s(smem_g + Sh::A_BYTES + u * Sh::SLICE_B, gb + u * Sh::SLICE_B, Sh::SLICE_B, bar);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    // scales for the epilogue, loaded while the copies and MMAs run
    float* sbinv = reinterpret_cast<float*>(smem_g + Sh::BINV_OFF);
    const int row = (warp & 3) * 32 + (tid & 31), half = warp >> 2;
    const int i = mt * kM + row;
    const float ai = ainv[((size_t)ax * KC + kc) * ((size_t)MT * kM) + i];
    if (tid < NP) sbinv[tid] = binv[((size_t)ax * KC + kc) * NP + tid];
    const bool loaded = tc::mbar_wait_bounded(bar, 0);
    if (tid == 0 && loaded) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kM, NP);
        const uint32_t a0 = tc::smem_u32(smem_g), b0 = a0 + Sh::A_BYTES;
#pragma unroll
        for (int d = 0; d < kS; ++d)
#pragma unroll
            for (int u = 0; u <= d; ++u) {
                const int v = d - u;
#pragma unroll
                for (int ks = 0; ks < kK / 16; ++ks) {
                    const uint64_t ad = tc::smem_desc(a0 + u * kSliceA + ks * 2 * tc::kLBO, tc::kLBO, kSBO);
                    const uint64_t bd = tc::smem_desc(b0 + v * Sh::SLICE_B + ks * 2 * tc::kLBO, tc::kLBO, kSBO);
                    tc::mma_bf16(tmem + (uint32_t)(d * NP), ad, bd, idesc, (u == 0 && ks == 0) ? 0u : 1u);
                }
            }
        tc::mma_commit(bar + 1);
    }
    const bool ok = loaded && tc::mbar_wait_bounded(bar + 1, 0);
    const bool failed = __syncthreads_or(!ok);
    tc::fence_after_sync();
    float2* out = Yp + (((size_t)kc * 3 + ax) * n + (size_t)i) * NP;
    if (failed) {
        if (i < n)
            for (int j = 0; j < NP; ++j)
                if (((j >> 4) & 1) == half) out[j] = make_float2(__int_as_float(-1), 0.f);
        if (tid == 0) atomicExch(err, 1);
    } else {
        const float* bi = sbinv;
        const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
        for (int c0 = 16 * half; c0 < NP; c0 += 32) {
            float acc[kS][16];
#pragma unroll
            for (int d = 0; d < kS; d += 2)
                tc::tmem_ld16x2(tl + d * NP + c0, tl + (d + 1) * NP + c0, acc[d], acc[d + 1]);
            if (i < n) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const dev::F2 s = combine6(acc[0][c], acc[1][c], acc[2][c], acc[3][c], acc[4][c], acc[5][c]);
                    const float sc = __fmul_rn(ai, bi[c0 + c]);
                    out[c0 + c] = make_float2(__fmul_rn(s.h, sc), __fmul_rn(s.l, sc));
                }
            }
        }
    }
    // a load that timed out may still be landing in shared memory: wait for it once
    // more (bounded) before the CTA exits
    if (!loaded && tid == 0) tc::mbar_wait_bounded(bar, 0);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::NCOL);
}

}  // namespace tcg
}  // namespace rs
