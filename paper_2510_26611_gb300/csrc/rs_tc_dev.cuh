// Tensor-core evaluation of the W form over cell-sorted pose-atoms (the long range
// of Sec. 3's Tucker potential at every atom, Eq. lerp-Tucker): for the atoms of one
// axis-3 cell i, with v2 the interpolated axis-2 factor row of each atom,
//   X = v2 W[i]^T  and  X' = v2 D[i]^T         (one 128 x 2r x r MMA per slice pair)
// so that  phi = sum_a v1[a] (X[a] + f3 X'[a])  and, for the gradient,
//   d phi / d x1 = sum_a dv1[a] (X[a] + f3 X'[a]),  d phi / d x3 = sum_a v1[a] X'[a],
//   d phi / d x2 = sum_a v1[a] (Z[a] + f3 Z'[a])  with Z, Z' the products of dv2.
// The per-atom CUDA-core work drops from O(r^2) pair operations to O(r); the
// products run on tcgen05 MMAs with BF16 slices (rs_tc.cuh) at ~2^-31 relative
// accuracy, accumulated in TMEM and read back once per tile.
//
// One CTA of 128 threads walks a contiguous run of sorted records; a tile is up to
// 128 consecutive records of one key (one cell of one protein).  Per tile: each
// thread slices its atom's v2 into the A tile in shared memory, thread 0 issues the
// MMAs and commits them to an mbarrier, then every thread reads its own TMEM lane
// (row = atom) and finishes its atom; for gradients a second round does the same
// with dv2 in the same A tile and TMEM columns (so both passes fit 256 columns and
// two CTAs per SM).  The B image of the cell (built with the protein) is copied to
// shared memory when the key changes.
#pragma once

#include <climits>

#include "rs_common.cuh"
#include "rs_pose_dev.cuh"
#include "rs_sorted_dev.cuh"
#include "rs_tc.cuh"

namespace rs {
namespace {

// A tile holds up to 128 records of one cell, and its cost barely depends on how
// many rows are filled.  A launch whose cells hold fewer atoms than this on average
// (pose-atoms / grid cells along axis 3) takes the float-pair W form instead, which
// walks the records 32 at a time per warp (measured on GB300: 0.27 ns per pose-atom
// for full tensor-core tiles, 0.46 ns for the float-pair kernel at any fill).
constexpr double kTcMinAtomsPerCell = 96.0;

template <int RP, bool GRAD>
struct TcLayout {
    using S = tc::Shape<RP>;
    static constexpr uint32_t A_SET = tc::kSlices * S::A_SLICE;   // one A tile (all slices)
    static constexpr uint32_t B_OFF = A_SET;
    static constexpr uint32_t CS_OFF = B_OFF + S::B_BYTES;
    static constexpr uint32_t BAR_OFF = (CS_OFF + S::NP * 4 + 15) / 16 * 16;
    static constexpr uint32_t SLOT_OFF = BAR_OFF + 8;
    static constexpr uint32_t BYTES = SLOT_OFF + 8;
    static constexpr uint32_t COLS_USED = tc::kAccs * S::NP;
    static constexpr uint32_t NCOL = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                                   : COLS_USED <= 256 ? 256 : 512;
    static_assert(COLS_USED <= 512, "TMEM columns");
};

// Record sources.  Single pair: the key is the axis-3 cell.  Grouped pairs: the key is
// the segment's first key + the cell, the segment index is in bits 8.. of r.bits.
struct TcSingle {
    const ProteinView* P;
    const LigandView* lig;
    __device__ __forceinline__ int seg(const AtomRec&) const { return 0; }
    __device__ __forceinline__ const ProteinView& prot(int) const { return *P; }
    __device__ __forceinline__ const LigandView& ligand(int) const { return *lig; }
    __device__ __forceinline__ int cell(const AtomRec& r, int) const { return r.i3; }
    __device__ __forceinline__ int atom(const AtomRec& r, int) const { return r.slot % lig->L; }
};

// The interpolated axis-2 row v2 = V2[i2] + f2 dV2[i2] (slope = false) or its slope
// dV2[i2] (slope = true), as float pairs.
template <int RP>
__device__ __forceinline__ void tc_axis2_row(const ProteinView& P, const AtomRec& r, bool slope,
                                             dev::F2 (&v2)[RP]) {
    const size_t o = (size_t)r.i2 * RP;
    const float4* vh = (const float4*)(P.Vt[1][0] + o);
    const float4* vl = (const float4*)(P.Vt[1][1] + o);
    const float4* dh = (const float4*)(P.Vt[1][2] + o);
    const float4* dl = (const float4*)(P.Vt[1][3] + o);
#pragma unroll
    for (int c4 = 0; c4 < RP / 4; ++c4) {
        const float4 c = __ldg(dh + c4), d = __ldg(dl + c4);
        const float cv[4] = {c.x, c.y, c.z, c.w}, dv[4] = {d.x, d.y, d.z, d.w};
        if (slope) {
#pragma unroll
            for (int u = 0; u < 4; ++u) v2[4 * c4 + u] = dev::F2{cv[u], dv[u]};
        } else {
            const float4 a = __ldg(vh + c4), b = __ldg(vl + c4);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v2[4 * c4 + u] = dev::df_lerp(dev::F2{av[u], bv[u]}, dev::F2{cv[u], dv[u]}, r.f2);
        }
    }
}

// One contraction round of a tile, in two halves so that independent work can run
// between them.  tc_issue: every thread writes its row (or a zero row), thread 0
// issues the MMAs and commits them to the barrier.  tc_wait: loads the next tile's
// record (rn) while the MMAs run, then waits (bounded); returns false on a timed-out
// wait (then uniformly in the CTA).
template <int RP>
__device__ __forceinline__ void tc_issue(uint8_t* sA, uint32_t a_saddr, uint32_t b_saddr, uint32_t tmem,
                                         uint64_t* bar, bool write, const dev::F2 (&x)[RP], float& inv) {
    const int tid = threadIdx.x;
    if (write) inv = tc::write_row<RP>(x, sA, tid);
    else tc::zero_row<RP>(sA, tid);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        tc::issue_products<RP>(tmem, a_saddr, b_saddr);
        tc::mma_commit(bar);
    }
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t& phase, const AtomRec* __restrict__ srt,
                                        const int* __restrict__ off, int ksub, long long t1, long long s1,
                                        AtomRec& rn, AtomRec& hn, int& endn) {
    const int tid = threadIdx.x;
    if (t1 + tid < s1) rn = srt[t1 + tid];
    if (t1 < s1) {  // the next tile's first record and the end of its cell
        hn = srt[t1];
        endn = off[(hn.i3 + 1) * ksub];
    }
    const bool ok = tc::mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    const bool failed = __syncthreads_or(!ok);
    tc::fence_after_sync();
    return !failed;
}

// Walks the sorted records [s0, s1) (cell keys ascending, off[(key + 1) ksub] = end of
// the cell's records) with the whole CTA (128 threads) and writes each atom's contributions.
// smem: TcLayout<RP, GRAD>::BYTES bytes, 16-byte aligned.  On an MMA that does not
// complete within the bounded wait the tile's contributions are set to NaN, *err is
// set and the CTA stops.
template <int RP, bool GRAD, class Src>
__device__ __forceinline__ void tc_wform_range(const Src& src, const AtomRec* __restrict__ srt,
                                               const int* __restrict__ off, int ksub, long long s0, long long s1,
                                               const float2* __restrict__ shortv, float2* __restrict__ contrib,
                                               uint8_t* smem, int* __restrict__ err) {
    using S = tc::Shape<RP>;
    using Lay = TcLayout<RP, GRAD>;
    using dev::F2;
    constexpr int NC = GRAD ? 7 : 1;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t* sA = smem;
    uint8_t* sB = smem + Lay::B_OFF;
    float* sCs = reinterpret_cast<float*>(smem + Lay::CS_OFF);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFF);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + Lay::SLOT_OFF);
    if (warp == 0) tc::tmem_alloc(slot, Lay::NCOL);
    if (tid == 0) tc::mbar_init(bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lane quarter
    const uint32_t a_saddr = tc::smem_u32(sA), b_saddr = tc::smem_u32(sB);
    int cur = -1;
    uint32_t phase = 0;
    // software pipeline: the next tile's record is loaded during this tile's MMAs, and
    // every global load a tile needs is issued before its MMA wait
    AtomRec rn, hn;
    int endn = 0;
    if (s0 + tid < s1) rn = srt[s0 + tid];
    if (s0 < s1) {
        hn = srt[s0];
        endn = off[(hn.i3 + 1) * ksub];
    }
    for (long long t0 = s0; t0 < s1;) {
        const AtomRec r0 = hn;
        const int key = r0.i3;
        const long long t1 = min(s1, min(t0 + tc::kTileRows, (long long)endn));
        const int sg = src.seg(r0);
        const ProteinView& P = src.prot(sg);
        if (key != cur) {
            const size_t cell = (size_t)src.cell(r0, sg);
            const uint4* gB = reinterpret_cast<const uint4*>(P.Wtc) + cell * (S::B_BYTES / 16);
            uint4* dB = reinterpret_cast<uint4*>(sB);
            for (int e = tid; e < (int)(S::B_BYTES / 16); e += tc::kTileRows) dB[e] = __ldg(gB + e);
            for (int e = tid; e < S::NP; e += tc::kTileRows) sCs[e] = __ldg(P.Wsc + cell * S::NP + e);
            cur = key;
        }
        const bool act = t0 + tid < t1;
        const AtomRec r = act ? rn : r0;
        const bool in1 = r.bits & 1, in2 = r.bits & 2, in3 = r.bits & 4;
        (void)in1;
        (void)in2;
        (void)in3;
        const float f3 = r.f3;
        // short-range value (DRAM) and the axis-1 rows (L2), issued now
        F2 phs{0.f, 0.f}, gs[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (act) short_value<GRAD>(shortv, r.slot, phs, gs);
        F2 va[RP];
        F2 dva[GRAD ? RP : 1];
        F2 phi{0.f, 0.f}, g1{0.f, 0.f}, g2{0.f, 0.f}, g3{0.f, 0.f};
        bool ok;
        // round 1: X = v2 W^T, X' = v2 D^T
        {
            float inv = 0.f;
            {
                F2 v2[RP];
                tc_axis2_row<RP>(P, r, false, v2);
                tc_issue<RP>(sA, a_saddr, b_saddr, tmem, bar, act, v2, inv);
            }
            // axis-1 rows (L2), loaded and interpolated while the MMAs run
            {
                const size_t o1 = (size_t)r.i1 * RP;
                const float4* v1h = (const float4*)(P.Vt[0][0] + o1);
                const float4* v1l = (const float4*)(P.Vt[0][1] + o1);
                const float4* v1dh = (const float4*)(P.Vt[0][2] + o1);
                const float4* v1dl = (const float4*)(P.Vt[0][3] + o1);
#pragma unroll
                for (int c4 = 0; c4 < RP / 4; ++c4) {
                    const float4 a = __ldg(v1h + c4), b = __ldg(v1l + c4), c = __ldg(v1dh + c4),
                                 d = __ldg(v1dl + c4);
                    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
                    const float cv[4] = {c.x, c.y, c.z, c.w}, dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const F2 dv1{cv[u], dv[u]};
                        va[4 * c4 + u] = dev::df_lerp(F2{av[u], bv[u]}, dv1, r.f1);
                        if constexpr (GRAD) dva[4 * c4 + u] = in1 ? dv1 : F2{0.f, 0.f};
                    }
                }
            }
            ok = tc_wait(bar, phase, srt, off, ksub, t1, s1, rn, hn, endn);
            if (ok) {
#pragma unroll
                for (int ch = 0; ch < S::NP / 16; ++ch) {
                    float x0[16], x1[16];
                    tc::tmem_ld16x2(tl + ch * 16, tl + S::NP + ch * 16, x0, x1);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int a = ch * 8 + q;
                        if (a < RP) {
                            const F2 X = tc::combine(x0[2 * q], x1[2 * q], __fmul_rn(inv, sCs[2 * a]));
                            const F2 Xd = tc::combine(x0[2 * q + 1], x1[2 * q + 1], __fmul_rn(inv, sCs[2 * a + 1]));
                            const F2 u = dev::df_lerp(X, Xd, f3);
                            dev::df_fma_acc(phi, va[a], u);
                            if constexpr (GRAD) {
                                dev::df_fma_acc(g1, dva[a], u);
                                if (in3) dev::df_fma_acc(g3, va[a], Xd);
                            }
                        }
                    }
                }
            }
        }
        // round 2 (gradient): Z = dv2 W^T, Z' = dv2 D^T into the same TMEM columns and A tile
        if constexpr (GRAD) {
            if (ok) {
                tc::fence_before_sync();
                __syncthreads();
                float inv = 0.f;
                {
                    F2 dv2[RP];
                    tc_axis2_row<RP>(P, r, true, dv2);
                    tc_issue<RP>(sA, a_saddr, b_saddr, tmem, bar, act && in2, dv2, inv);
                }
                ok = tc_wait(bar, phase, srt, off, ksub, t1, s1, rn, hn, endn);
                if (ok) {
#pragma unroll
                    for (int ch = 0; ch < S::NP / 16; ++ch) {
                        float x0[16], x1[16];
                        tc::tmem_ld16x2(tl + ch * 16, tl + S::NP + ch * 16, x0, x1);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int a = ch * 8 + q;
                            if (a < RP) {
                                const F2 Z = tc::combine(x0[2 * q], x1[2 * q], __fmul_rn(inv, sCs[2 * a]));
                                const F2 Zd = tc::combine(x0[2 * q + 1], x1[2 * q + 1], __fmul_rn(inv, sCs[2 * a + 1]));
                                dev::df_fma_acc(g2, va[a], dev::df_lerp(Z, Zd, f3));
                            }
                        }
                    }
                }
            }
        }
        if (!ok) {
            if (act)
                for (int c = 0; c < NC; ++c)
                    contrib[(size_t)r.slot * kContribStride<GRAD> + c] = make_float2(__int_as_float(-1), 0.f);
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        if (act) {
            const int j = src.atom(r, sg);
            const float ry[3] = {r.ry0, r.ry1, r.ry2};
            store_contrib<GRAD>(P, phi, g1, g2, g3, phs, gs, src.ligand(sg).q64[j], ry, contrib, r.slot);
        }
        tc::fence_before_sync();
        __syncthreads();
        t0 = t1;
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Lay::NCOL);
}

// Dynamic shared memory and CTAs per SM for a tensor-core W-form kernel.  No more
// CTAs may fit on an SM than its TMEM holds (512 columns / ncol): an allocation
// beyond that would wait for a resident CTA to finish.  The count comes from the
// device's shared-memory and register limits (the runtime's occupancy query
// reports one CTA per SM for kernels that allocate TMEM); smem is padded until the
// shared-memory limit alone caps the residency at the TMEM share.
template <class K>
rs_status tc_occupancy(K kern, uint32_t ncol, size_t& smem, int& per_sm) {
    const int cap = 512 / (int)ncol;
    int dev = 0, sm_smem = 0, reserved = 0, sm_regs = 0, sm_threads = 0;
    RS_TRY_CUDA(cudaGetDevice(&dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    cudaFuncAttributes fa{};
    RS_TRY_CUDA(cudaFuncGetAttributes(&fa, kern));
    const size_t per_cta = (size_t)fa.sharedSizeBytes + (size_t)reserved;
    auto by_smem = [&](size_t dyn) { return (int)((size_t)sm_smem / (dyn + per_cta)); };
    while (by_smem(smem) > cap) smem += 1024;
    const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = sm_regs / (regs_per_warp * (tc::kTileRows / 32));
    per_sm = std::min(std::min(by_smem(smem), by_regs), sm_threads / tc::kTileRows);
    if (per_sm < 1 || smem > 227 * 1024) {
        set_error("tensor-core W form: no residency (smem %zu, regs %d)", smem, fa.numRegs);
        return RS_ERR_UNSUPPORTED;
    }
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the whole unified L1/shared array as shared memory, so per_sm CTAs fit
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    return RS_OK;
}

// FP32 pipe operations per atom of the tensor-core W form (the MMAs excluded), per
// column of the rank r: energy: the axis-2 pair lerp (14), its five slices (~20),
// two column combinations (2 x 8), the axis-1 and axis-3 pair lerps (2 x 14) and one
// Dot2 step (13); gradient: the same round plus two more Dot2 steps, then the slope
// row's slices, two combinations, one lerp and one Dot2 step; ~60 / ~100 per atom for
// the rest (record, contributions).  Both match the kernels' FP32 instruction
// counters within 1 % on the protein workload.
inline double tc_ops_per_atom(int RP, bool grad) {
    double r = RP;
    return grad ? 178.0 * r + 100.0 : 89.0 * r + 60.0;
}

}  // namespace
}  // namespace rs
