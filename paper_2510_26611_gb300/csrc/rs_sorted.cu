// Algorithm PLIE (Sec. 3.4) for a Tucker-reduced protein with the ligand atoms of
// all poses grouped by their interpolation cell along axis 3.
//
// The W-form evaluation of one atom reads the whole slab W[i3], D[i3] (4 RP^2
// floats) of its axis-3 cell.  Taken atom by atom in pose order those reads are
// scattered over the table and the L1 cache cannot hold them; grouped by cell, a
// warp stages a slab in shared memory once and every atom of that cell reads it
// there as a broadcast.  The launch sequence per chunk of poses is
//   k_sorted_poses   pose setups (rotation, Jacobian) of the chunk
//   k_sorted_keys    per atom: its sort key and its rank in a per-key count
//   key scan         exclusive scan of the per-key counts (three kernels)
//   k_sorted_atoms   per atom: position, cells, fractions, short range and vdW
//                    (flags), and a 48-byte record written at its sorted position
//   k_sorted_wform   per warp: a contiguous run of sorted atoms; slab of the current
//                    cell in shared memory; long range + contributions per atom
//   k_sorted_reduce  per pose: sums over its atoms (one warp per pose)
// Every per-atom value is computed by the same helpers, in the same order, as the
// one-block-per-pose-batch path (wform_block), and the pose sums are taken in the
// same order, so both paths give the same bits; the order of atoms within a cell
// (set by atomics) never enters any arithmetic.
#include <algorithm>
#include <atomic>
#include <climits>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"
#include "rs_pose_dev.cuh"
#include "rs_sorted_dev.cuh"
#include "rs_tc_dev.cuh"

namespace rs {
namespace {

constexpr int kWarpsPerBlock = 4;

__global__ void k_sorted_poses(ProteinView P, const double* __restrict__ rot,
                               const double* __restrict__ trans, long long p0, int PC, bool rotvec,
                               const uint8_t* __restrict__ skip, PoseSetup* __restrict__ ps,
                               int* __restrict__ pflag) {
    int pl = blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= PC) return;
    long long p = p0 + pl;
    pflag[pl] = 0;
    if (!(skip && skip[p])) setup_pose(P, rot, trans, p, rotvec, ps[pl]);
    else ps[pl].valid = 0;
}

// Sort key and rank of every pose-atom of the chunk, kr[g] = (key, rank) (key
// (n - 1) kSub: a skipped pose).  The key comes from the same position and cell
// arithmetic as the atom's record in k_sorted_atoms, which places the record at
// off[key] + rank: the (key, rank) pairs are distinct, so the positions are a
// permutation of the chunk's atoms.
__global__ void k_sorted_keys(ProteinView P, LigandView lig, const PoseSetup* __restrict__ ps, int PC,
                              int* __restrict__ count, int2* __restrict__ kr) {
    const long long M = (long long)PC * lig.L;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M) return;
    const int pl = (int)(g / lig.L), j = (int)(g - (long long)pl * lig.L);
    int key = (P.n - 1) * kSub;
    if (ps[pl].valid) {
        F2 x[3];
        atom_position(ps[pl], lig.yd + 3 * j, x);
        int i2, i3;
        float f;
        bool in;
        dev::axis_cell(x[1], F2{P.b_h, P.b_l}, F2{P.inv_h_h, P.inv_h_l}, P.n, i2, f, in);
        dev::axis_cell(x[2], F2{P.b_h, P.b_l}, F2{P.inv_h_h, P.inv_h_l}, P.n, i3, f, in);
        key = i3 * kSub + sub_bucket(i2, P.n, kSub);
    }
    kr[g] = make_int2(key, atomicAdd(&count[key], 1));
}

// One thread per pose-atom; the short range of a warp's 32 atoms is taken
// together (short_coop), so the pair work of near pairs keeps all lanes busy.  Warps
// are persistent and take 32-atom chunks from a launch-wide cursor, so a warp whose
// atoms had few neighbours moves on at once, and the chunks with many near pairs
// spread over all warps instead of over the ones a fixed stride assigns them to.
template <bool GRAD>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, GRAD ? 6 : 8)
    k_sorted_atoms(ProteinView P, LigandView lig, const PoseSetup* __restrict__ ps, int PC,
                   int* __restrict__ pflag, const int2* __restrict__ kr, const int* __restrict__ off,
                   AtomRec* __restrict__ srt, float2* __restrict__ shortv, unsigned long long* __restrict__ counters,
                   unsigned long long* __restrict__ cursor) {
    __shared__ NearQueue<GRAD> queues[kWarpsPerBlock];
    const int L = lig.L;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    ShortCounts sc;
    long long natoms = 0;
    const long long M = (long long)PC * L;
    const long long nchunk = (M + 31) / 32;
    for (;;) {
        unsigned long long cu = 0;
        if (lane == 0) cu = atomicAdd(cursor, 1ULL);
        const long long c = (long long)__shfl_sync(0xffffffffu, cu, 0);
        if (c >= nchunk) break;
        const long long g = c * 32 + lane;
        const bool in_range = g < M;
        const int pl = in_range ? (int)(g / L) : 0;
        const int j = in_range ? (int)(g - (long long)pl * L) : 0;
        const bool valid = in_range && ps[pl].valid;
        float ry[3] = {0.f, 0.f, 0.f};
        F2 x[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int ci[3] = {0, 0, 0};
        float cf[3] = {0.f, 0.f, 0.f};
        bool ins[3] = {true, true, true};
        if (valid) atom_geometry(P, lig, ps[pl], j, ry, x, ci, cf, ins);
        F2 php{0.f, 0.f}, gp[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int clash = 0;
        short_coop<GRAD>(P, valid, x, AtomRef{&ps[pl], lig.y64 + 3 * j}, queues[wib], php, gp, clash, &sc);
        natoms += __popc(__ballot_sync(0xffffffffu, valid));
        if (!in_range) continue;
        AtomRec r;
        r.slot = (int)g;
        const int2 kg = kr[g];
        r.rank = kg.y;
        AtomRec* dst = srt + off[kg.x] + kg.y;
        if (!valid) {
            r.i3 = P.n - 1;
            r.bits = 0;
            *dst = r;
            continue;
        }
        int fl = clash ? RS_FLAG_CLASH : 0;
        if (!(ins[0] && ins[1] && ins[2])) fl |= RS_FLAG_OUT_OF_GRID;
        if (fl) atomicOr(&pflag[pl], fl);
        store_short_value<GRAD>(shortv, g, php, gp);
        r.i1 = ci[0];
        r.i2 = ci[1];
        r.i3 = ci[2];
        r.f1 = cf[0];
        r.f2 = cf[1];
        r.f3 = cf[2];
        r.bits = (ins[0] ? 1 : 0) | (ins[1] ? 2 : 0) | (ins[2] ? 4 : 0) | (sub_bucket(ci[1], P.n, kSub) << 3);
        r.ry0 = ry[0];
        r.ry1 = ry[1];
        r.ry2 = ry[2];
        *dst = r;
    }
    if (lane == 0 && natoms > 0) {  // work counters of the launch (diagnostics)
        atomicAdd(&counters[0], (unsigned long long)natoms);
        atomicAdd(&counters[1], (unsigned long long)sc.cand);
        atomicAdd(&counters[2], (unsigned long long)sc.near);
    }
}

template <int RP, bool GRAD>
// Energy: 5 CTAs (20 warps) per SM caps registers at 96 (measured 17 % faster than
// the unconstrained 107); gradient: 3 CTAs per SM, its natural occupancy at ~168
// registers (a 128 cap spills and measured 7 % slower; no cap let the compiler take
// more registers and measured 14 % slower).
__global__ void __launch_bounds__(32 * kWarpsPerBlock, GRAD ? 3 : 5)
    k_sorted_wform(ProteinView P, LigandView lig, const AtomRec* __restrict__ srt, const int* __restrict__ off,
                   const float2* __restrict__ shortv, float2* __restrict__ contrib) {
    extern __shared__ float4 sm4[];
    constexpr int SLAB4 = RP * RP / 4;  // float4 per plane
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4* slab4 = sm4 + (size_t)wib * 4 * SLAB4;
    const int Mv = off[(P.n - 1) * kSub];  // atoms of evaluated poses
    const long long nw = (long long)gridDim.x * kWarpsPerBlock;
    const long long w = (long long)blockIdx.x * kWarpsPerBlock + wib;
    const long long per = ((Mv + nw - 1) / nw + 31) / 32 * 32;
    const long long s0 = w * per, s1 = std::min<long long>(Mv, s0 + per);
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
                __syncwarp();
                const size_t o = (size_t)cm * RP * RP;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4* src = (const float4*)(P.Wt[k] + o);
                    for (int e = lane; e < SLAB4; e += 32) slab4[k * SLAB4 + e] = __ldg(src + e);
                }
                __syncwarp();
                cur = cm;
            }
            if (c == cm) {
                sorted_atom<RP, GRAD>(P, lig, r, r.slot % lig.L, (const float*)slab4, shortv, contrib);
                c = INT_MAX;
            }
        }
    }
}

// Tensor-core W form (rs_tc_dev.cuh): CTA b walks a contiguous run of the sorted
// records of evaluated poses.
template <int RP, bool GRAD>
__global__ void __launch_bounds__(tc::kTileRows, 4)
    k_sorted_tc(const __grid_constant__ ProteinView P, const __grid_constant__ LigandView lig,
                const AtomRec* __restrict__ srt, const int* __restrict__ off, const float2* __restrict__ shortv,
                float2* __restrict__ contrib, int* __restrict__ err) {
    extern __shared__ __align__(16) uint8_t smem_tc[];
    const long long Mv = off[(P.n - 1) * kSub];
    const long long per = (Mv + gridDim.x - 1) / gridDim.x;
    const long long s0 = (long long)blockIdx.x * per, s1 = std::min<long long>(Mv, s0 + per);
    const TcSingle src{&P, &lig};
    tc_wform_range<RP, GRAD>(src, srt, off, kSub, s0, s1, shortv, contrib, smem_tc, err);
}

template <int NC>
__global__ void k_sorted_reduce(const PoseSetup* __restrict__ ps, int PC, int L, long long p0,
                                const float2* __restrict__ contrib, const int* __restrict__ pflag,
                                double* __restrict__ E, uint8_t* __restrict__ flags, double* __restrict__ gt,
                                double* __restrict__ gw) {
    const int lane = threadIdx.x & 31;
    const long long pl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pl >= PC || !ps[pl].valid) return;
    constexpr int CS = kContribStride<NC == 7>;
    double s[NC];
    pose_sums<NC, CS>(contrib + (size_t)pl * L * CS, L, lane, s);
    if (lane == 0) write_pose<NC>(ps[pl], s, pflag[pl], p0 + pl, E, flags, gt, gw);
}

// Scratch of one chunk of PC poses (M = PC L atoms), carved in this order.
struct SortedScratch {
    PoseSetup* ps;
    int* pflag;
    int2* kr;     // sort key of each atom and its rank among the atoms of that key
    AtomRec* srt;
    float2* shortv;
    float2* contrib;
    int* count;
    int* off;
    int* bsum;  // segment sums of the key scan
    unsigned long long* cursor;  // work cursor of the atoms kernel
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t chunk_bytes(long long PC, int L, int n, bool grad) {
    const long long M = PC * L;
    const int CS = grad ? kContribStride<true> : kContribStride<false>;
    return align256(PC * sizeof(PoseSetup)) + align256(PC * 4) + align256(M * 8) + align256(M * sizeof(AtomRec)) +
           align256(M * 8 * (grad ? 4 : 1)) + align256(M * 8 * CS) + align256((size_t)n * kSub * 4) +
           align256(((size_t)n * kSub + 1) * 4) + align256(key_scan_ints((long long)n * kSub) * 4) + 256;
}

SortedScratch carve(void* base, long long PC, int L, int n, bool grad) {
    const long long M = PC * L;
    const int CS = grad ? kContribStride<true> : kContribStride<false>;
    char* p = (char*)base;
    SortedScratch s;
    auto take = [&](size_t b) {
        char* q = p;
        p += align256(b);
        return q;
    };
    s.ps = (PoseSetup*)take(PC * sizeof(PoseSetup));
    s.pflag = (int*)take(PC * 4);
    s.kr = (int2*)take(M * 8);
    s.srt = (AtomRec*)take(M * sizeof(AtomRec));
    s.shortv = (float2*)take(M * 8 * (grad ? 4 : 1));
    s.contrib = (float2*)take(M * 8 * CS);
    s.count = (int*)take((size_t)n * kSub * 4);
    s.off = (int*)take(((size_t)n * kSub + 1) * 4);
    s.bsum = (int*)take(key_scan_ints((long long)n * kSub) * 4);
    s.cursor = (unsigned long long*)take(8);
    return s;
}

template <int RP, bool GRAD>
rs_status launch_sorted_wform(const EvalLaunch& a, const SortedScratch& s, long long M, cudaStream_t st) {
    auto kern = k_sorted_wform<RP, GRAD>;
    const size_t smem = (size_t)kWarpsPerBlock * 4 * RP * RP * sizeof(float);
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, sms = 0, dev = 0;
    RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kWarpsPerBlock, smem));
    RS_TRY_CUDA(cudaGetDevice(&dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long want = (M + 32 * kWarpsPerBlock - 1) / (32 * kWarpsPerBlock);
    long long grid = std::max<long long>(1, std::min<long long>(want, (long long)std::max(per_sm, 1) * sms));
    double work = (double)M * wform_ops_per_atom(RP, GRAD);
    {
        ::rs::KernelTimer kt__(GRAD ? "k_sorted_wform_grad" : "k_sorted_wform", st, work, true, a.events);
        kern<<<(unsigned)grid, 32 * kWarpsPerBlock, smem, st>>>(a.prot, a.lig, s.srt, s.off, s.shortv, s.contrib);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

template <int RP, bool GRAD>
rs_status launch_sorted_tc(const EvalLaunch& a, const SortedScratch& s, long long M, cudaStream_t st) {
    auto kern = k_sorted_tc<RP, GRAD>;
    size_t smem = TcLayout<RP, GRAD>::BYTES;
    int per_sm = 0, sms = 0, dev = 0;
    RS_TRY(tc_occupancy(kern, TcLayout<RP, GRAD>::NCOL, smem, per_sm));
    RS_TRY_CUDA(cudaGetDevice(&dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int* err = tc_error_flag(dev);
    if (!err) {
        set_error("tensor-core W form: no error flag on device %d", dev);
        return RS_ERR_CUDA;
    }
    const long long want = (M + tc::kTileRows - 1) / tc::kTileRows;
    const long long grid = std::max<long long>(1, std::min<long long>(want, (long long)per_sm * sms));
    note_tc_launch(grid, smem, per_sm);
    const double work = (double)M * tc_ops_per_atom(RP, GRAD);
    {
        ::rs::KernelTimer kt__(GRAD ? "k_sorted_tc_grad" : "k_sorted_tc", st, work, true, a.events);
        kern<<<(unsigned)grid, tc::kTileRows, smem, st>>>(a.prot, a.lig, s.srt, s.off, s.shortv, s.contrib, err);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

// The W-form kernel of a chunk of M atoms: the tensor-core form when the call's full
// chunks (M_call atoms each) fill its tiles, else the float-pair form.  Every chunk of
// a call takes the same form, so a pose's result does not depend on which chunk (or
// which position in the batch) holds it.
template <bool GRAD>
rs_status dispatch_sorted_wform(const EvalLaunch& a, const SortedScratch& s, long long M, long long M_call,
                                cudaStream_t st) {
    const bool tcore = wform_kernel_mode() == 1 && a.prot.Wtc != nullptr &&
                       (double)M_call >= kTcMinAtomsPerCell * (double)(a.prot.n - 1);
    switch (a.prot.R) {
#define RS_CASE(R)                                                                          \
    case R:                                                                                 \
        return tcore ? launch_sorted_tc<R, GRAD>(a, s, M, st) : launch_sorted_wform<R, GRAD>(a, s, M, st);
        RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        default:
            set_error("unsupported padded Tucker rank %d", a.prot.R);
            return RS_ERR_UNSUPPORTED;
    }
}

// CTAs of the persistent atoms kernel: as many as fit on the device at once (at most
// one per 32-atom chunk of warps).
template <bool GRAD>
unsigned atoms_grid(long long M) {
    static std::atomic<int> cached{0};  // CTAs per SM x SMs, computed once per instance
    int resident = cached.load(std::memory_order_relaxed);
    if (resident == 0) {
        int per_sm = 0, sms = 0, dev = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sorted_atoms<GRAD>, 32 * kWarpsPerBlock, 0) !=
                cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 4;
            sms = 152;
        }
        resident = std::max(per_sm, 1) * std::max(sms, 1);
        cached.store(resident, std::memory_order_relaxed);
    }
    const long long need = (M + 32 * kWarpsPerBlock - 1) / (32 * kWarpsPerBlock);
    return (unsigned)std::max<long long>(1, std::min<long long>(need, resident));
}

// Per-atom contributions of the pc poses whose setups are in s.ps: sort keys, key
// scan, short range and vdW with the records at their sorted positions, and the W
// form (into s.contrib and s.pflag).
template <bool GRAD>
rs_status sorted_chunk_contrib(const EvalLaunch& a, const SortedScratch& s, int pc, long long pc_call,
                               cudaStream_t st) {
    const int L = a.lig.L, n = a.prot.n;
    const long long M = (long long)pc * L;
    RS_TRY_CUDA(cudaMemsetAsync(s.count, 0, (size_t)n * kSub * 4, st));
    RS_TRY_CUDA(cudaMemsetAsync(s.cursor, 0, 8, st));
    {
        ::rs::KernelTimer kt__("k_sorted_keys", st, 0.0, false, a.events);
        k_sorted_keys<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(a.prot, a.lig, s.ps, pc, s.count, s.kr);
    }
    {
        ::rs::KernelTimer kt__("k_key_scan", st, 0.0, false, a.events);
        launch_key_scan(n * kSub, s.count, s.bsum, s.off, st);
        note_launch(2);  // three kernels under one timer
    }
    {
        const unsigned grid = atoms_grid<GRAD>(M);
        int dev = 0;
        RS_TRY_CUDA(cudaGetDevice(&dev));
        unsigned long long* ctr = short_counters(dev, GRAD);
        if (!ctr) {
            set_error("sorted pose path: no counters on device %d", dev);
            return RS_ERR_CUDA;
        }
        ::rs::KernelTimer kt__(GRAD ? "k_sorted_atoms_grad" : "k_sorted_atoms", st, 0.0, true, a.events);
        k_sorted_atoms<GRAD><<<grid, 32 * kWarpsPerBlock, 0, st>>>(a.prot, a.lig, s.ps, pc, s.pflag, s.kr, s.off,
                                                                    s.srt, s.shortv, ctr, s.cursor);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return dispatch_sorted_wform<GRAD>(a, s, M, pc_call * L, st);
}

template <bool GRAD>
rs_status run_sorted(const EvalLaunch& a, cudaStream_t st) {
    const int L = a.lig.L, n = a.prot.n;
    const long long PC = sorted_chunk_poses(a.ws_bytes, L, n, GRAD);
    if (PC < 1) {
        set_error("sorted pose path: scratch of %zu bytes too small", a.ws_bytes);
        return RS_ERR_INVALID;
    }
    constexpr int NC = GRAD ? 7 : 1;
    for (long long p0 = 0; p0 < a.P; p0 += PC) {
        const int pc = (int)std::min<long long>(PC, a.P - p0);
        SortedScratch s = carve(a.ws, pc, L, n, GRAD);
        {
            ::rs::KernelTimer kt__("k_sorted_poses", st, 0.0, false, a.events);
            k_sorted_poses<<<(pc + 127) / 128, 128, 0, st>>>(a.prot, a.rot, a.trans, p0, pc, GRAD, a.skip, s.ps,
                                                              s.pflag);
        }
        RS_TRY(sorted_chunk_contrib<GRAD>(a, s, pc, std::min<long long>(PC, a.P), st));
        {
            ::rs::KernelTimer kt__("k_sorted_reduce", st, 0.0, false, a.events);
            k_sorted_reduce<NC><<<(unsigned)((pc * 32LL + 255) / 256), 256, 0, st>>>(
                s.ps, pc, L, p0, s.contrib, s.pflag, a.E, a.flags, a.gt, a.gw);
        }
        RS_TRY_CUDA(cudaGetLastError());
    }
    return RS_OK;
}

// ------------------------------------------------------------------ FD forces
// The backward differences of Eq. differ_ligand need the potential at x_l and at
// x_l - h e_i (i = 1..3) for every atom l.  Those points are the atoms of the same
// rigid ligand under four translations of the pose, so each pose becomes four
// evaluation poses (k = 0: the pose; k = i: translation t - h e_i) and the chunk
// pipeline above gives the charge-weighted potentials q_l phi at all of them.

// Evaluation poses v = 4 (p - p0) + k of the chunk's poses p0 .. p0 + pc - 1.
__global__ void k_fd_expand(const double* __restrict__ rot, const double* __restrict__ trans, long long p0, int pc,
                            double h, double* __restrict__ vrot, double* __restrict__ vtrans) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= 4 * pc) return;
    const long long p = p0 + (v >> 2);
    const int k = v & 3;
    for (int a = 0; a < 3; ++a) {
        vrot[3 * v + a] = rot[3 * p + a];
        vtrans[3 * v + a] = k == a + 1 ? trans[3 * p + a] - h : trans[3 * p + a];
    }
}

// r0 of Eq. Field_phi: the given radius, or (r0 = 0) the RMS distance of the
// ligand atoms from their centre.  One warp.
__global__ void k_fd_radius(LigandView lig, double r0, double* __restrict__ out) {
    double s = 0.0;
    for (int j = threadIdx.x; j < lig.L; j += 32) {
        const double* y = lig.y64 + 3 * (size_t)j;
        s = fma(y[2], y[2], fma(y[1], y[1], y[0] * y[0])) + s;
    }
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = r0 > 0.0 ? r0 : sqrt(s / lig.L);
}

// One warp per pose: per atom F_l = (c_0 - c_i) / h from the contributions
// c = q_l phi of its four evaluation poses (Eq. differ_ligand), the split of F_l
// along v_l = r_l / |r_l| (r_l = R y_l), and the pose sums
//   E, Fsum = sum F_l, F0 = sum of the radial parts (Eq. Field_Xcenter),
//   Fphi = sum (|r_l| / r0) x tangential part (Eq. Field_phi), M = sum r_l x F_l.
// The differences c_0 - c_i cancel most of their operands' digits and are taken in
// float-pair arithmetic (E is summed exactly as the pose sums of the other paths);
// the quotients keep ~2^-24 of F_l in FP32, and the split and the vector sums run
// in FP32 (FP64 throughput is a small fraction of FP32's here).
__global__ void k_fd_reduce(const PoseSetup* __restrict__ ps, int pc, LigandView lig, long long p0,
                            const float2* __restrict__ contrib, const int* __restrict__ pflag, double inv_h,
                            const double* __restrict__ r0p, FdOut o) {
    const int lane = threadIdx.x & 31;
    const long long pl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pl >= pc) return;
    const int L = lig.L;
    const PoseSetup& q = ps[4 * pl];
    const double r0 = *r0p;
    const float inv_r0 = r0 > 0.0 ? (float)(1.0 / r0) : 0.f;
    const float2* c0 = contrib + (size_t)(4 * pl) * L;
    const float ih = (float)inv_h;
    float s[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) s[c] = 0.f;
    for (int j = lane; j < L; j += 32) {
        const F2 e0{c0[j].x, c0[j].y};
        float F[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float2 ci = c0[(size_t)(i + 1) * L + j];
            const F2 d = dev::df_sub(e0, F2{ci.x, ci.y});
            F[i] = __fmul_rn(__fadd_rn(d.h, d.l), ih);
        }
        const float4 y = lig.y[j];
        float r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) r[a] = fmaf(q.Rf[3 * a + 2], y.z, fmaf(q.Rf[3 * a + 1], y.y, q.Rf[3 * a] * y.x));
        const float rn = sqrtf(fmaf(r[2], r[2], fmaf(r[1], r[1], r[0] * r[0])));
        float Fr[3];
        if (rn > 0.f) {
            const float ir = 1.f / rn;
            const float v0 = r[0] * ir, v1 = r[1] * ir, v2 = r[2] * ir;
            const float d = fmaf(F[2], v2, fmaf(F[1], v1, F[0] * v0));
            Fr[0] = d * v0;
            Fr[1] = d * v1;
            Fr[2] = d * v2;
        } else {
            Fr[0] = F[0];
            Fr[1] = F[1];
            Fr[2] = F[2];
        }
        const float sc = rn * inv_r0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s[a] += F[a];
            s[3 + a] += Fr[a];
            s[6 + a] = fmaf(sc, F[a] - Fr[a], s[6 + a]);
        }
        s[9] += r[1] * F[2] - r[2] * F[1];
        s[10] += r[2] * F[0] - r[0] * F[2];
        s[11] += r[0] * F[1] - r[1] * F[0];
    }
    double E1[1];
    pose_sums<1>(c0, L, lane, E1);
    const double E = E1[0];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], off);
    if (lane == 0) {
        const long long p = p0 + pl;
        o.E[p] = E;
        if (o.flags) o.flags[p] = (uint8_t)pflag[4 * pl];
        for (int a = 0; a < 3; ++a) {
            o.F[3 * p + a] = s[a];
            o.F0[3 * p + a] = s[3 + a];
            o.Fphi[3 * p + a] = s[6 + a];
            o.M[3 * p + a] = s[9 + a];
        }
    }
}

}  // namespace

long long sorted_chunk_poses(size_t ws_bytes, int L, int n, bool grad) {
    // upper bound: an atom takes at least its 48-byte record
    long long lo = 0, hi = std::max<long long>(1, (long long)(ws_bytes / ((size_t)L * sizeof(AtomRec))) + 1);
    // largest PC whose carve fits (chunk_bytes is increasing in PC)
    while (lo < hi) {
        long long mid = (lo + hi + 1) / 2;
        if (chunk_bytes(mid, L, n, grad) <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

size_t sorted_scratch_bytes(long long P, int L, int n, bool grad) {
    const long long max_atoms = 1LL << 23;  // a chunk holds at most ~8.4M atoms
    long long PC = std::max<long long>(1, std::min<long long>(P, max_atoms / std::max(L, 1)));
    return chunk_bytes(PC, L, n, grad);
}

rs_status launch_sorted(const EvalLaunch& a, bool grad, cudaStream_t st) {
    if (a.P <= 0) return RS_OK;
    return grad ? run_sorted<true>(a, st) : run_sorted<false>(a, st);
}

long long sorted_fd_chunk_poses(size_t ws_bytes, int L, int n) { return sorted_chunk_poses(ws_bytes, L, n, false) / 4; }

size_t sorted_fd_scratch_bytes(long long P, int L, int n) {
    return sorted_scratch_bytes(4 * std::max<long long>(P, 1), L, n, false);
}

size_t fd_pose_bytes(long long PC) { return (size_t)PC * 4 * 3 * 8 * 2 + 256; }

rs_status launch_sorted_fd(const EvalLaunch& a, double h, double r0, void* vbuf, const FdOut& o, cudaStream_t st) {
    if (a.P <= 0) return RS_OK;
    const int L = a.lig.L, n = a.prot.n;
    const long long PC = sorted_fd_chunk_poses(a.ws_bytes, L, n);
    if (PC < 1) {
        set_error("finite-difference forces: scratch of %zu bytes too small", a.ws_bytes);
        return RS_ERR_INVALID;
    }
    double* vrot = (double*)vbuf;
    double* vtrans = vrot + PC * 12;
    double* r0d = vtrans + PC * 12;
    {
        ::rs::KernelTimer kt__("k_fd_radius", st, 0.0, false, a.events);
        k_fd_radius<<<1, 32, 0, st>>>(a.lig, r0, r0d);
    }
    for (long long p0 = 0; p0 < a.P; p0 += PC) {
        const int pc = (int)std::min<long long>(PC, a.P - p0);
        const int pv = 4 * pc;
        SortedScratch s = carve(a.ws, pv, L, n, false);
        {
            ::rs::KernelTimer kt__("k_fd_expand", st, 0.0, false, a.events);
            k_fd_expand<<<(pv + 127) / 128, 128, 0, st>>>(a.rot, a.trans, p0, pc, h, vrot, vtrans);
        }
        {
            ::rs::KernelTimer kt__("k_sorted_poses", st, 0.0, false, a.events);
            k_sorted_poses<<<(pv + 127) / 128, 128, 0, st>>>(a.prot, vrot, vtrans, 0, pv, true, nullptr, s.ps,
                                                              s.pflag);
        }
        RS_TRY(sorted_chunk_contrib<false>(a, s, pv, 4 * std::min<long long>(PC, a.P), st));
        {
            ::rs::KernelTimer kt__("k_fd_reduce", st, 0.0, false, a.events);
            k_fd_reduce<<<(unsigned)((pc * 32LL + 255) / 256), 256, 0, st>>>(s.ps, pc, a.lig, p0, s.contrib,
                                                                              s.pflag, 1.0 / h, r0d, o);
        }
        RS_TRY_CUDA(cudaGetLastError());
    }
    return RS_OK;
}

}  // namespace rs
