// Algorithm PLIE (Sec. 3.4) for many protein-ligand pairs of one padded Tucker
// rank at once, with the ligand atoms of all their poses grouped by (pair, axis-3
// cell): the multi-pair form of the cell-grouped path (rs_sorted.cu), used by the
// batched launch and the serving loop.
//
// The pairs' poses are laid end to end and cut into chunks of at most
// `max_atoms` pose-atoms; a chunk is a list of segments (one pair's consecutive
// poses each).  Per chunk:
//   k_group_poses    pose setups
//   k_group_atoms    per pose-atom: position, cells, short range and vdW, record
//                    keyed by the segment's first cell + the axis-3 cell
//   key scan         exclusive scan of the per-key counts (three kernels)
//   k_sorted_scatter records in key order
//   k_group_wform    per warp: a run of sorted atoms, the slab of the current
//                    (pair, cell) in shared memory, long range + contributions
//   k_group_reduce   per pose: sums over its atoms, outputs to the pair's arrays
// Per-atom and per-pose arithmetic is that of the single-pair path, in the same
// order, so every pair's results equal rs_energy_poses bit for bit.
#include <algorithm>
#include <atomic>
#include <climits>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"
#include "rs_pose_dev.cuh"
#include "rs_sorted_dev.cuh"
#include "rs_batch_dev.cuh"
#include "rs_group.cuh"
#include "rs_tc_dev.cuh"

namespace rs {
namespace {

// Segment of the chunk holding chunk pose q (pose_off ascending).
__device__ __forceinline__ int seg_of_pose(const GroupSeg* __restrict__ segs, int nseg, int q) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].pose_off <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int seg_of_atom(const GroupSeg* __restrict__ segs, int nseg, long long g) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].atom_off <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_group_poses(const PairDesc* __restrict__ pairs, const GroupSeg* __restrict__ segs, int nseg,
                              int npose, PoseSetup* __restrict__ ps, int* __restrict__ pflag) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npose) return;
    const GroupSeg sg = segs[seg_of_pose(segs, nseg, q)];
    const PairDesc& pd = pairs[sg.pair];
    pflag[q] = 0;
    setup_pose(pd.prot, pd.rot, pd.trans, sg.p0 + (q - sg.pose_off), false, ps[q]);
}

template <int WPB>
__global__ void __launch_bounds__(32 * WPB)
    k_group_atoms(const PairDesc* __restrict__ pairs, const GroupSeg* __restrict__ segs, int nseg, long long natom,
                  int ksub, const PoseSetup* __restrict__ ps, int* __restrict__ pflag,
                  AtomRec* __restrict__ rec, float2* __restrict__ shortv, int* __restrict__ count,
                  unsigned long long* __restrict__ cursor) {
    __shared__ NearQueue<false> queues[WPB];
    __shared__ int lane_pair[WPB][32];
    // persistent warps taking 32-atom chunks from a launch-wide cursor
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long nchunk = (natom + 31) / 32;
    for (;;) {
        unsigned long long cu = 0;
        if (lane == 0) cu = atomicAdd(cursor, 1ULL);
        const long long c = (long long)__shfl_sync(0xffffffffu, cu, 0);
        if (c >= nchunk) break;
        const long long g = c * 32 + lane;
        const bool in_range = g < natom;
        int s = 0, q = 0, j = 0;
        if (in_range) {
            s = seg_of_atom(segs, nseg, g);
            const int L = pairs[segs[s].pair].lig.L;
            const long long local = g - segs[s].atom_off;
            q = segs[s].pose_off + (int)(local / L);
            j = (int)(local % L);
        }
        const GroupSeg sg = segs[s];
        const PairDesc& pd = pairs[sg.pair];
        float ry[3] = {0.f, 0.f, 0.f};
        F2 x[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int ci[3] = {0, 0, 0};
        float cf[3] = {0.f, 0.f, 0.f};
        bool ins[3] = {true, true, true};
        if (in_range) atom_geometry(pd.prot, pd.lig, ps[q], j, ry, x, ci, cf, ins);
        F2 php{0.f, 0.f}, gp[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int clash = 0;
        // the lanes of a warp may belong to different pairs: each near pair is evaluated
        // against its owner's protein
        int* lp = lane_pair[wib];
        __syncwarp();
        lp[lane] = sg.pair;
        __syncwarp();
        short_coop_with<false>([&](int l) -> const ProteinView& { return pairs[lp[l]].prot; }, in_range, x,
                               AtomRef{&ps[q], pd.lig.y64 + 3 * j},
                               queues[wib], php, gp, clash);
        if (!in_range) continue;
        AtomRec r;
        r.slot = (int)g;
        int fl = clash ? RS_FLAG_CLASH : 0;
        if (!(ins[0] && ins[1] && ins[2])) fl |= RS_FLAG_OUT_OF_GRID;
        if (fl) atomicOr(&pflag[q], fl);
        shortv[g] = make_float2(php.h, php.l);
        r.i1 = ci[0];
        r.i2 = ci[1];
        r.i3 = sg.cell_base + ci[2];
        r.f1 = cf[0];
        r.f2 = cf[1];
        r.f3 = cf[2];
        r.bits = (ins[0] ? 1 : 0) | (ins[1] ? 2 : 0) | (ins[2] ? 4 : 0) | (sub_bucket(ci[1], pd.prot.n, ksub) << 3) |
                 (s << 8);
        r.ry0 = ry[0];
        r.ry1 = ry[1];
        r.ry2 = ry[2];
        r.rank = atomicAdd(&count[rec_key(r, ksub)], 1);
        rec[g] = r;
    }
}

template <int RP, int WPB>
__global__ void __launch_bounds__(32 * WPB, 20 / WPB)
    k_group_wform(const PairDesc* __restrict__ pairs, const GroupSeg* __restrict__ segs,
                  const AtomRec* __restrict__ srt, long long natom, const float2* __restrict__ shortv,
                  float2* __restrict__ contrib) {
    extern __shared__ float4 sm4[];
    constexpr int SLAB4 = RP * RP / 4;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4* slab4 = sm4 + (size_t)wib * 4 * SLAB4;
    const long long nw = (long long)gridDim.x * WPB;
    const long long w = (long long)blockIdx.x * WPB + wib;
    const long long per = ((natom + nw - 1) / nw + 31) / 32 * 32;
    const long long s0 = w * per, s1 = std::min<long long>(natom, s0 + per);
    int cur = -1;
    for (long long base = s0; base < s1; base += 32) {
        const long long idx = base + lane;
        AtomRec r;
        int c = INT_MAX;
        if (idx < s1) {
            r = srt[idx];
            c = r.i3;
        }
        for (;;) {
            const int cm = __reduce_min_sync(0xffffffffu, c);
            if (cm == INT_MAX) break;
            if (cm != cur) {
                // every lane holding key cm has the same segment; broadcast it
                const unsigned holders = __ballot_sync(0xffffffffu, c == cm);
                const int src = __ffs(holders) - 1;
                const int sgi = __shfl_sync(0xffffffffu, c == cm ? (r.bits >> 8) : 0, src);
                const GroupSeg sg = segs[sgi];
                const ProteinView& P = pairs[sg.pair].prot;
                __syncwarp();
                const size_t o = (size_t)(cm - sg.cell_base) * RP * RP;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4* src4 = (const float4*)(P.Wt[k] + o);
                    for (int e = lane; e < SLAB4; e += 32) slab4[k * SLAB4 + e] = __ldg(src4 + e);
                }
                __syncwarp();
                cur = cm;
            }
            if (c == cm) {
                const GroupSeg sg = segs[r.bits >> 8];
                const PairDesc& pd = pairs[sg.pair];
                const int j = (int)((r.slot - sg.atom_off) % pd.lig.L);
                AtomRec rr = r;
                rr.bits &= 7;
                sorted_atom<RP, false>(pd.prot, pd.lig, rr, j, (const float*)slab4, shortv, contrib);
                c = INT_MAX;
            }
        }
    }
}

// Records of a grouped chunk for the tensor-core W form: segment in bits 8.. of
// r.bits, key = the segment's first key + the axis-3 cell.
struct TcGroup {
    const PairDesc* pairs;
    const GroupSeg* segs;
    __device__ __forceinline__ int seg(const AtomRec& r) const { return r.bits >> 8; }
    __device__ __forceinline__ const ProteinView& prot(int sg) const { return pairs[segs[sg].pair].prot; }
    __device__ __forceinline__ const LigandView& ligand(int sg) const { return pairs[segs[sg].pair].lig; }
    __device__ __forceinline__ int cell(const AtomRec& r, int sg) const { return r.i3 - segs[sg].cell_base; }
    __device__ __forceinline__ int atom(const AtomRec& r, int sg) const {
        return (int)((r.slot - segs[sg].atom_off) % pairs[segs[sg].pair].lig.L);
    }
};

template <int RP>
__global__ void __launch_bounds__(tc::kTileRows, 4)
    k_group_tc(const PairDesc* __restrict__ pairs, const GroupSeg* __restrict__ segs, const AtomRec* __restrict__ srt,
               const int* __restrict__ off, int ksub, long long natom, const float2* __restrict__ shortv,
               float2* __restrict__ contrib, int* __restrict__ err) {
    extern __shared__ __align__(16) uint8_t smem_tc[];
    const long long per = (natom + gridDim.x - 1) / gridDim.x;
    const long long s0 = (long long)blockIdx.x * per, s1 = std::min<long long>(natom, s0 + per);
    const TcGroup src{pairs, segs};
    tc_wform_range<RP, false>(src, srt, off, ksub, s0, s1, shortv, contrib, smem_tc, err);
}

__global__ void k_group_reduce(const PairDesc* __restrict__ pairs, const GroupSeg* __restrict__ segs, int nseg,
                               int npose, const PoseSetup* __restrict__ ps, const float2* __restrict__ contrib,
                               const int* __restrict__ pflag) {
    const int lane = threadIdx.x & 31;
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= npose) return;
    const GroupSeg sg = segs[seg_of_pose(segs, nseg, (int)q)];
    const PairDesc& pd = pairs[sg.pair];
    const int L = pd.lig.L;
    double s[1];
    pose_sums<1>(contrib + sg.atom_off + (size_t)(q - sg.pose_off) * L, L, lane, s);
    if (lane == 0) write_pose<1>(ps[q], s, pflag[q], sg.p0 + (q - sg.pose_off), pd.E, pd.flags, nullptr, nullptr);
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

struct GroupScratch {
    PoseSetup* ps;
    int* pflag;
    AtomRec* rec;
    AtomRec* srt;
    float2* shortv;
    float2* contrib;
    int* count;
    int* off;
    int* bsum;
    unsigned long long* cursor;  // work cursor of the atoms kernel
};

// nkey counts cells; the sort uses nkey * ksub sub-bucket keys.
size_t chunk_scratch(int npose, long long natom, int nkey, int ksub) {
    nkey *= ksub;
    return align256((size_t)npose * sizeof(PoseSetup)) + align256((size_t)npose * 4) +
           2 * align256((size_t)natom * sizeof(AtomRec)) + 2 * align256((size_t)natom * 8) +
           align256((size_t)nkey * 4) + align256((size_t)(nkey + 1) * 4) + align256(key_scan_ints(nkey) * 4) + 256;
}

GroupScratch carve_group(void* base, int npose, long long natom, int nkey, int ksub) {
    nkey *= ksub;
    char* p = (char*)base;
    auto take = [&](size_t b) {
        char* q = p;
        p += align256(b);
        return q;
    };
    GroupScratch s;
    s.ps = (PoseSetup*)take((size_t)npose * sizeof(PoseSetup));
    s.pflag = (int*)take((size_t)npose * 4);
    s.rec = (AtomRec*)take((size_t)natom * sizeof(AtomRec));
    s.srt = (AtomRec*)take((size_t)natom * sizeof(AtomRec));
    s.shortv = (float2*)take((size_t)natom * 8);
    s.contrib = (float2*)take((size_t)natom * 8);
    s.count = (int*)take((size_t)nkey * 4);
    s.off = (int*)take((size_t)(nkey + 1) * 4);
    s.bsum = (int*)take(key_scan_ints(nkey) * 4);
    s.cursor = (unsigned long long*)take(8);
    return s;
}

template <int RP, int WPB>
rs_status launch_group_wform(const PairDesc* d_pairs, const GroupSeg* d_segs, const GroupScratch& s,
                             long long natom, cudaStream_t st, bool events) {
    auto kern = k_group_wform<RP, WPB>;
    const size_t smem = (size_t)WPB * 4 * RP * RP * sizeof(float);
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, sms = 0, dev = 0;
    RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPB, smem));
    RS_TRY_CUDA(cudaGetDevice(&dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long want = (natom + 32 * WPB - 1) / (32 * WPB);
    long long grid = std::max<long long>(1, std::min<long long>(want, (long long)std::max(per_sm, 1) * sms));
    {
        ::rs::KernelTimer kt__("k_group_wform", st, (double)natom * wform_ops_per_atom(RP, false), true, events);
        kern<<<(unsigned)grid, 32 * WPB, smem, st>>>(d_pairs, d_segs, s.srt, natom, s.shortv, s.contrib);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

template <int RP>
rs_status launch_group_tc(const PairDesc* d_pairs, const GroupSeg* d_segs, const GroupScratch& s, int ksub, long long natom,
                          cudaStream_t st, bool events) {
    auto kern = k_group_tc<RP>;
    size_t smem = TcLayout<RP, false>::BYTES;
    int per_sm = 0, sms = 0, dev = 0;
    RS_TRY(tc_occupancy(kern, TcLayout<RP, false>::NCOL, smem, per_sm));
    RS_TRY_CUDA(cudaGetDevice(&dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int* err = tc_error_flag(dev);
    if (!err) {
        set_error("tensor-core W form: no error flag on device %d", dev);
        return RS_ERR_CUDA;
    }
    const long long want = (natom + tc::kTileRows - 1) / tc::kTileRows;
    const long long grid = std::max<long long>(1, std::min<long long>(want, (long long)per_sm * sms));
    note_tc_launch(grid, smem, per_sm);
    {
        ::rs::KernelTimer kt__("k_group_tc", st, (double)natom * tc_ops_per_atom(RP, false), true, events);
        kern<<<(unsigned)grid, tc::kTileRows, smem, st>>>(d_pairs, d_segs, s.srt, s.off, ksub, natom, s.shortv, s.contrib,
                                                          err);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

template <int WPB>
rs_status dispatch_group_wform(int RP, const PairDesc* d_pairs, const GroupSeg* d_segs, const GroupScratch& s,
                               int ksub, int ncell, long long natom, cudaStream_t st, bool events) {
    const bool tcore = wform_kernel_mode() == 1 && (double)natom >= kTcMinAtomsPerCell * (double)ncell;
    switch (RP) {
#define RS_CASE(R)                                                                   \
    case R:                                                                          \
        return tcore ? launch_group_tc<R>(d_pairs, d_segs, s, ksub, natom, st, events) \
                     : launch_group_wform<R, WPB>(d_pairs, d_segs, s, natom, st, events);
        RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        default:
            set_error("unsupported padded Tucker rank %d", RP);
            return RS_ERR_UNSUPPORTED;
    }
}

}  // namespace

rs_status group_plan(const std::vector<PairDesc>& pairs, const std::vector<int>& members, long long max_atoms,
                     GroupPlan* out) {
    GroupPlan& G = *out;
    G = GroupPlan();
    if (members.empty()) return RS_OK;
    G.RP = pairs[members[0]].prot.R;
    GroupChunk ch{0, 0, 0, 0, 0};
    auto close_chunk = [&]() {
        if (ch.seg_end > ch.seg_begin) {
            // sub-buckets per cell: as many as keep the chunk's keys near 2^20
            ch.ksub = kSub;
            while (ch.ksub > 1 && (long long)ch.nkey * ch.ksub > (1LL << 20)) ch.ksub >>= 1;
            G.scratch = std::max(G.scratch, chunk_scratch(ch.npose, ch.natom, ch.nkey, ch.ksub));
            G.chunks.push_back(ch);
        }
        ch = GroupChunk{(int)G.segs.size(), (int)G.segs.size(), 0, 0, 0, kSub};
    };
    for (int m : members) {
        const PairDesc& pd = pairs[m];
        if (pd.prot.R != G.RP || pd.prot.kind != 1) {
            set_error("group_plan: pair %d is not Tucker-reduced with padded rank %d", m, G.RP);
            return RS_ERR_INVALID;
        }
        const int L = pd.lig.L;
        long long p = 0;
        while (p < pd.P) {
            long long room = (max_atoms - ch.natom) / L;
            if (room < 1) {
                close_chunk();
                room = std::max<long long>(1, max_atoms / L);
            }
            const long long take = std::min<long long>(room, pd.P - p);
            GroupSeg sg;
            sg.pair = m;
            sg.pc = (int)take;
            sg.p0 = p;
            sg.pose_off = ch.npose;
            sg.cell_base = ch.nkey;
            sg.atom_off = ch.natom;
            G.segs.push_back(sg);
            ch.seg_end = (int)G.segs.size();
            ch.npose += (int)take;
            ch.natom += take * L;
            ch.nkey += pd.prot.n - 1;
            p += take;
        }
    }
    close_chunk();
    return RS_OK;
}

rs_status group_launch(const GroupPlan& G, const PairDesc* d_pairs, const GroupSeg* d_segs, void* ws,
                       size_t ws_bytes, int wpb, cudaStream_t st, bool events) {
    if (ws_bytes < G.scratch) {
        set_error("group_launch: scratch of %zu bytes, %zu needed", ws_bytes, G.scratch);
        return RS_ERR_INVALID;
    }
    for (const GroupChunk& ch : G.chunks) {
        const GroupSeg* segs = d_segs + ch.seg_begin;
        const int nseg = ch.seg_end - ch.seg_begin;
        GroupScratch s = carve_group(ws, ch.npose, ch.natom, ch.nkey, ch.ksub);
        RS_TRY_CUDA(cudaMemsetAsync(s.count, 0, (size_t)ch.nkey * ch.ksub * 4, st));
        RS_TRY_CUDA(cudaMemsetAsync(s.cursor, 0, 8, st));
        {
            ::rs::KernelTimer kt__("k_group_poses", st, 0.0, false, events);
            k_group_poses<<<(ch.npose + 127) / 128, 128, 0, st>>>(d_pairs, segs, nseg, ch.npose, s.ps, s.pflag);
        }
        {
            static std::atomic<int> resident{0};  // CTAs that fit on the device at once
            int res = resident.load(std::memory_order_relaxed);
            if (res == 0) {
                int per_sm = 0, sms = 0, dev = 0;
                RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group_atoms<4>, 128, 0));
                RS_TRY_CUDA(cudaGetDevice(&dev));
                RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                res = std::max(per_sm, 1) * sms;
                resident.store(res, std::memory_order_relaxed);
            }
            const long long grid = std::max<long long>(1, std::min<long long>((ch.natom + 127) / 128, res));
            ::rs::KernelTimer kt__("k_group_atoms", st, 0.0, true, events);
            k_group_atoms<4><<<(unsigned)grid, 128, 0, st>>>(d_pairs, segs, nseg, ch.natom, ch.ksub, s.ps, s.pflag, s.rec,
                                                            s.shortv, s.count, s.cursor);
        }
        {
            ::rs::KernelTimer kt__("k_key_scan", st, 0.0, false, events);
            launch_key_scan(ch.nkey * ch.ksub, s.count, s.bsum, s.off, st);
            note_launch(2);  // three kernels under one timer
        }
        {
            ::rs::KernelTimer kt__("k_sorted_scatter", st, 0.0, false, events);
            k_sorted_scatter<<<(unsigned)((ch.natom + 255) / 256), 256, 0, st>>>(ch.natom, ch.ksub, s.rec, s.off,
                                                                                   s.srt);
        }
        RS_TRY_CUDA(cudaGetLastError());
        if (wpb == 8) RS_TRY(dispatch_group_wform<8>(G.RP, d_pairs, segs, s, ch.ksub, ch.nkey, ch.natom, st, events));
        else RS_TRY(dispatch_group_wform<4>(G.RP, d_pairs, segs, s, ch.ksub, ch.nkey, ch.natom, st, events));
        {
            ::rs::KernelTimer kt__("k_group_reduce", st, 0.0, false, events);
            k_group_reduce<<<(unsigned)((ch.npose * 32LL + 255) / 256), 256, 0, st>>>(d_pairs, segs, nseg, ch.npose,
                                                                                   s.ps, s.contrib, s.pflag);
        }
        RS_TRY_CUDA(cudaGetLastError());
    }
    return RS_OK;
}

}  // namespace rs
