// Device pieces of the cell-grouped Tucker pose path shared by the single-pair
// launch (rs_sorted.cu) and the grouped multi-pair launch (rs_group.cu): the atom
// record, the per-cell scan and scatter, and the long range of one sorted atom.
#pragma once

#include <climits>

#include "rs_common.cuh"
#include "rs_pose_dev.cuh"

namespace rs {
namespace {

struct __align__(16) AtomRec {
    int i1, i2, i3;       // interpolation cells (i3 = n - 1: pose skipped)
    float f1, f2, f3;     // fractions in the cells
    int slot;             // pl * L + j within the chunk
    int bits;             // bits 0-2: coordinate a inside [-b, b]; 3-7: sub-bucket; 8-: segment
    float ry0, ry1, ry2;  // R y (FP32), the torque arm
    int rank;             // position among the atoms of its sort key
};
static_assert(sizeof(AtomRec) == 48, "AtomRec layout");

// Sort keys: each axis-3 cell is split into kSub sub-buckets by the axis-2 row, so
// the atoms of a cell come out grouped by i2 and neighbouring atoms of a tile read
// the same axis-2 factor rows (L1 hits instead of L2 round trips).  key = cell key *
// kSub + sub-bucket; a cell's records are [off[c kSub], off[(c + 1) kSub]).
// The single-pair path uses kSub; the grouped path fewer when its chunks hold many
// cells (a power of two ksub <= kSub, the same for the whole chunk).
constexpr int kSub = 32;
__device__ __forceinline__ int sub_bucket(int i2, int n, int ksub) {
    return min(ksub - 1, (int)(((long long)i2 * ksub) / max(n - 1, 1)));
}
__device__ __forceinline__ int rec_key(const AtomRec& r, int ksub) {
    return r.i3 * ksub + ((r.bits >> 3) & (ksub - 1));
}


// Exclusive scan of count[0..m) into off[0..m] over the whole GPU: blocks of
// kScanT threads x kScanE keys reduce their segments (k_scan_blocks), one block
// scans the segment sums (k_scan_sums), and every block rescans its segment from its
// base (k_scan_apply).  Fixed order, so the offsets do not depend on scheduling.
constexpr int kScanT = 512, kScanE = 16, kScanSeg = kScanT * kScanE;

__device__ __forceinline__ int block_exclusive(int v, int* sm_warp, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int x = lane < nw ? sm_warp[lane] : 0, xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < nw) sm_warp[lane] = xi - x;  // exclusive prefix of the warp totals
        if (lane == nw - 1) sm_warp[32] = xi;
    }
    __syncthreads();
    total = sm_warp[32];
    const int r = sm_warp[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanT) k_scan_blocks(int m, const int* __restrict__ count, int* __restrict__ bsum) {
    __shared__ int smw[33];
    const long long base = (long long)blockIdx.x * kScanSeg + (long long)threadIdx.x * kScanE;
    int s = 0;
#pragma unroll
    for (int e = 0; e < kScanE; ++e)
        if (base + e < m) s += count[base + e];
    int total;
    block_exclusive(s, smw, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// In place: bsum[0..nb) -> exclusive prefix, bsum[nb] = total; one block.
__global__ void __launch_bounds__(1024) k_scan_sums(int nb, int* __restrict__ bsum) {
    __shared__ int smw[33];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int total;
        const int ex = block_exclusive(v, smw, total);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanT) k_scan_apply(int m, int nb, const int* __restrict__ count,
                                                       const int* __restrict__ bsum, int* __restrict__ off) {
    __shared__ int smw[33];
    const long long base = (long long)blockIdx.x * kScanSeg + (long long)threadIdx.x * kScanE;
    int v[kScanE], s = 0;
#pragma unroll
    for (int e = 0; e < kScanE; ++e) {
        v[e] = base + e < m ? count[base + e] : 0;
        s += v[e];
    }
    int total;
    int run = bsum[blockIdx.x] + block_exclusive(s, smw, total);
#pragma unroll
    for (int e = 0; e < kScanE; ++e) {
        if (base + e < m) off[base + e] = run;
        run += v[e];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[m] = bsum[nb];
}

// Scratch ints of the scan for m keys, and the launch (three kernels).
inline size_t key_scan_ints(long long m) { return (size_t)((m + kScanSeg - 1) / kScanSeg) + 1; }
inline void launch_key_scan(int m, const int* count, int* bsum, int* off, cudaStream_t st) {
    const int nb = (int)((m + kScanSeg - 1) / kScanSeg);
    if (nb > 0) k_scan_blocks<<<nb, kScanT, 0, st>>>(m, count, bsum);
    k_scan_sums<<<1, 1024, 0, st>>>(nb, bsum);
    if (nb > 0) k_scan_apply<<<nb, kScanT, 0, st>>>(m, nb, count, bsum, off);
    else k_scan_apply<<<1, kScanT, 0, st>>>(m, 0, count, bsum, off);
}

__global__ void k_sorted_scatter(long long M, int ksub, const AtomRec* __restrict__ rec,
                                 const int* __restrict__ off, AtomRec* __restrict__ srt) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M) return;
    AtomRec r = rec[g];
    srt[off[rec_key(r, ksub)] + r.rank] = r;
}


// Short-range value of a pose-atom (float pairs): phi_s (energies) or phi_s and its
// gradient (4 pairs) at index slot.
template <bool GRAD>
__device__ __forceinline__ void short_value(const float2* __restrict__ shortv, long long slot, dev::F2& phs,
                                            dev::F2 gs[3]) {
    if constexpr (GRAD) {
        const float4 a = reinterpret_cast<const float4*>(shortv)[2 * slot];
        const float4 b = reinterpret_cast<const float4*>(shortv)[2 * slot + 1];
        phs = dev::F2{a.x, a.y};
        gs[0] = dev::F2{a.z, a.w};
        gs[1] = dev::F2{b.x, b.y};
        gs[2] = dev::F2{b.z, b.w};
    } else {
        const float2 v = shortv[slot];
        phs = dev::F2{v.x, v.y};
    }
}

template <bool GRAD>
__device__ __forceinline__ void store_short_value(float2* __restrict__ shortv, long long slot, dev::F2 phs,
                                                  const dev::F2 gs[3]) {
    if constexpr (GRAD) {
        reinterpret_cast<float4*>(shortv)[2 * slot] = make_float4(phs.h, phs.l, gs[0].h, gs[0].l);
        reinterpret_cast<float4*>(shortv)[2 * slot + 1] = make_float4(gs[1].h, gs[1].l, gs[2].h, gs[2].l);
    } else {
        shortv[slot] = make_float2(phs.h, phs.l);
    }
}

// Per-atom contributions of the cell-grouped paths in global memory: NC = 7 float
// pairs per atom for gradients, stored 8 apart (64 bytes, a whole number of 32-byte
// sectors, so the scattered per-atom writes never leave a sector partly written, which
// would make the L2 fetch the rest of it from DRAM); 1 for energies.
template <bool GRAD>
constexpr int kContribStride = GRAD ? 8 : 1;

// Contributions of one atom (atom_contrib) at their slot of the cell-grouped layout.
template <bool GRAD>
__device__ __forceinline__ void store_contrib(const ProteinView& P, dev::F2 phi, dev::F2 g1, dev::F2 g2, dev::F2 g3,
                                              dev::F2 phs, const dev::F2 gs[3], double qd, const float ry[3],
                                              float2* __restrict__ contrib, long long slot) {
    float2* cj = contrib + (size_t)slot * kContribStride<GRAD>;
    atom_contrib<GRAD>(P, phi, g1, g2, g3, phs, gs, qd, ry, cj);
    if constexpr (GRAD) cj[7] = make_float2(0.f, 0.f);
}

// Long range of one atom from its record (ligand atom j), with the axis-3 slab of
// its cell in shared memory (planes Wh, Wl, Dh, Dl of RP x RP floats); writes its
// contributions at slot r.slot.
template <int RP, bool GRAD>
__device__ __forceinline__ void sorted_atom(const ProteinView& P, const LigandView& lig, const AtomRec& r, int j,
                                            const float* __restrict__ slab, const float2* __restrict__ shortv,
                                            float2* __restrict__ contrib) {
    using dev::F2;
    const bool in1 = r.bits & 1, in2 = r.bits & 2, in3 = r.bits & 4;
    F2 v2[RP];
    F2 dv2[GRAD ? RP : 1];
    {
        size_t o = (size_t)r.i2 * RP;
        const float4* vh = (const float4*)(P.Vt[1][0] + o);
        const float4* vl = (const float4*)(P.Vt[1][1] + o);
        const float4* dh = (const float4*)(P.Vt[1][2] + o);
        const float4* dl = (const float4*)(P.Vt[1][3] + o);
#pragma unroll
        for (int c4 = 0; c4 < RP / 4; ++c4) {
            float4 a = __ldg(vh + c4), b = __ldg(vl + c4), c = __ldg(dh + c4), d = __ldg(dl + c4);
            float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
            float cv[4] = {c.x, c.y, c.z, c.w}, dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v2[4 * c4 + u] = dev::df_lerp(F2{av[u], bv[u]}, F2{cv[u], dv[u]}, r.f2);
                if constexpr (GRAD) dv2[4 * c4 + u] = in2 ? F2{cv[u], dv[u]} : F2{0.f, 0.f};
            }
        }
    }
    const size_t o1 = (size_t)r.i1 * RP;
    const float* V1h = P.Vt[0][0] + o1;
    const float* V1l = P.Vt[0][1] + o1;
    const float* V1dh = P.Vt[0][2] + o1;
    const float* V1dl = P.Vt[0][3] + o1;
    const float* Wh = slab;
    const float* Wl = slab + RP * RP;
    const float* Dh = slab + 2 * RP * RP;
    const float* Dl = slab + 3 * RP * RP;
    const float f3 = r.f3;
    F2 phi{0.f, 0.f}, g1{0.f, 0.f}, g2{0.f, 0.f}, g3{0.f, 0.f};
    for (int a = 0; a < RP; ++a) {
        const float ch = __ldg(V1dh + a), cl = __ldg(V1dl + a);
        const F2 va = dev::df_lerp(F2{__ldg(V1h + a), __ldg(V1l + a)}, F2{ch, cl}, r.f1);
        F2 u{0.f, 0.f}, u2{0.f, 0.f}, u3{0.f, 0.f};
        const float4* wh = (const float4*)(Wh + a * RP);
        const float4* wl = (const float4*)(Wl + a * RP);
        const float4* dh = (const float4*)(Dh + a * RP);
        const float4* dl = (const float4*)(Dl + a * RP);
#pragma unroll
        for (int b4 = 0; b4 < RP / 4; ++b4) {
            float4 xa = wh[b4], xb = wl[b4], xc = dh[b4], xd = dl[b4];
            float av[4] = {xa.x, xa.y, xa.z, xa.w}, bv[4] = {xb.x, xb.y, xb.z, xb.w};
            float cv[4] = {xc.x, xc.y, xc.z, xc.w}, dv[4] = {xd.x, xd.y, xd.z, xd.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                F2 t = dev::df_lerp(F2{av[k], bv[k]}, F2{cv[k], dv[k]}, f3);
                dev::df_fma_acc(u, v2[4 * b4 + k], t);
                if constexpr (GRAD) {
                    dev::df_fma_acc(u2, dv2[4 * b4 + k], t);
                    if (in3) dev::df_fma_acc(u3, v2[4 * b4 + k], F2{cv[k], dv[k]});
                }
            }
        }
        dev::df_fma_acc(phi, va, u);
        if constexpr (GRAD) {
            const F2 dva = in1 ? F2{ch, cl} : F2{0.f, 0.f};
            dev::df_fma_acc(g1, dva, u);
            dev::df_fma_acc(g2, va, u2);
            dev::df_fma_acc(g3, va, u3);
        }
    }
    F2 phs, gs[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    short_value<GRAD>(shortv, r.slot, phs, gs);
    const float ry[3] = {r.ry0, r.ry1, r.ry2};
    store_contrib<GRAD>(P, phi, g1, g2, g3, phs, gs, lig.q64[j], ry, contrib, r.slot);
}

}  // namespace
}  // namespace rs
