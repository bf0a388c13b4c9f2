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
constexpr int kSub = 32;
__device__ __forceinline__ int sub_bucket(int i2, int n) {
    return min(kSub - 1, (int)(((long long)i2 * kSub) / max(n - 1, 1)));
}
__device__ __forceinline__ int rec_key(const AtomRec& r) { return r.i3 * kSub + ((r.bits >> 3) & (kSub - 1)); }


// Exclusive scan of count[0..m) into off[0..m]; one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_cell_scan(int m, const int* __restrict__ count, int* __restrict__ off) {
    __shared__ int part[1024];
    const int per = (m + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(m, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int base = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        off[i] = base;
        base += count[i];
    }
    if (threadIdx.x == 1023) off[m] = part[1023];
}

__global__ void k_sorted_scatter(long long M, const AtomRec* __restrict__ rec, const int* __restrict__ off,
                                 AtomRec* __restrict__ srt) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M) return;
    AtomRec r = rec[g];
    srt[off[rec_key(r)] + r.rank] = r;
}


// Long range of one atom from its record (ligand atom j), with the axis-3 slab of
// its cell in shared memory (planes Wh, Wl, Dh, Dl of RP x RP floats); writes its
// contributions at slot r.slot.
template <int RP, bool GRAD>
__device__ __forceinline__ void sorted_atom(const ProteinView& P, const LigandView& lig, const AtomRec& r, int j,
                                            const float* __restrict__ slab, const double* __restrict__ shortv,
                                            double* __restrict__ contrib) {
    using dev::F2;
    constexpr int NC = GRAD ? 7 : 1;
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
    double phs, gs[3] = {0.0, 0.0, 0.0};
    if constexpr (GRAD) {
        double4 v = reinterpret_cast<const double4*>(shortv)[r.slot];
        phs = v.x;
        gs[0] = v.y;
        gs[1] = v.z;
        gs[2] = v.w;
    } else {
        phs = shortv[r.slot];
    }
    const float ry[3] = {r.ry0, r.ry1, r.ry2};
    atom_contrib<GRAD>(P, phi, g1, g2, g3, phs, gs, lig.q64[j], ry, contrib + (size_t)r.slot * NC);
}

}  // namespace
}  // namespace rs
