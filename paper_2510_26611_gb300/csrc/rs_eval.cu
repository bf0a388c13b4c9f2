// Pose kernels: Algorithm PLIE (Sec. 3.4) over a batch of rigid poses, the
// short-range part and vdW check through the cell list, and the exact adjoint
// with respect to (translation, rotation vector).
//
// Per ligand atom j of pose p:  x_j = R_p y_j + t_p
//   phi_long(x) = trilinear interpolation of the long-range tensor, done per
//                 1D factor (Sec. 2 entry evaluation; Lemma 3.3)
//   phi_short   = sum over protein atoms closer than r_c (Def. 2.1)
//   E_p = sum_j q_j (phi_long + phi_short)(x_j)             (Eq. EnergySum_ligand)
// FP32 evaluation; per-atom sums carried as float pairs; per-pose sums FP64.
#include <algorithm>
#include <cmath>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"
#include "rs_pose_dev.cuh"

namespace rs {
namespace {

template <int RP, bool GRAD, int NT>
__global__ void __launch_bounds__(NT) k_eval_wform(ProteinView P, LigandView lig,
                                                   const double* __restrict__ rot,
                                                   const double* __restrict__ trans,
                                                   long long Ptot, int PB,
                                                   double* __restrict__ E,
                                                   uint8_t* __restrict__ flags,
                                                   double* __restrict__ gt,
                                                   double* __restrict__ gw,
                                                   const uint8_t* __restrict__ skip) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long nblocks = (Ptot + PB - 1) / PB;
    for (long long pb = blockIdx.x; pb < nblocks; pb += gridDim.x)
        wform_block<RP, GRAD, NT>(P, lig, rot, trans, Ptot, PB, pb * PB, E, flags, gt, gw, smem, skip);
}

// --------------------------------------------------------------- canonical path
// Warp per atom; lanes stride over the rank in float4 columns, so each of the
// six factor rows an atom needs is read as contiguous 512-byte segments.
template <bool GRAD>
__global__ void __launch_bounds__(256) k_eval_canon(ProteinView P, LigandView lig,
                                                    const double* __restrict__ rot,
                                                    const double* __restrict__ trans,
                                                    long long Ptot, int PB,
                                                    double* __restrict__ E,
                                                    uint8_t* __restrict__ flags,
                                                    double* __restrict__ gt,
                                                    double* __restrict__ gw,
                                                    const uint8_t* __restrict__ skip) {
    constexpr int NC = GRAD ? 7 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    PoseSetup* ps = (PoseSetup*)smem;
    float2* contrib = (float2*)(ps + PB);
    int* pflag = (int*)(contrib + (size_t)PB * lig.L * NC);
    const int L = lig.L;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    const long long nblocks = (Ptot + PB - 1) / PB;
    const int ld4 = P.ld / 4;
    const float4* Fa0 = (const float4*)P.F[0];
    const float4* Fa1 = (const float4*)P.F[1];
    const float4* Fa2 = (const float4*)P.F[2];
    for (long long pb = blockIdx.x; pb < nblocks; pb += gridDim.x) {
        long long p0 = pb * PB;
        __syncthreads();
        for (int pl = threadIdx.x; pl < PB; pl += blockDim.x) {
            long long p = p0 + pl;
            pflag[pl] = 0;
            if (p < Ptot && !(skip && skip[p])) setup_pose(P, rot, trans, p, GRAD, ps[pl]);
            else ps[pl].valid = 0;
        }
        __syncthreads();
        for (int g = warp; g < PB * L; g += nw) {
            int pl = g / L, j = g - pl * L;
            float2* cj = contrib + (size_t)g * NC;
            const PoseSetup& q = ps[pl];
            if (!q.valid) {
                if (lane < NC) cj[lane] = make_float2(0.f, 0.f);
                continue;
            }
            float ry[3];
            int ci[3];
            float cf[3];
            bool ins[3];
            F2 x[3];
            atom_geometry(P, lig, q, j, ry, x, ci, cf, ins);
            const float4* a0 = Fa0 + (size_t)ci[0] * ld4;
            const float4* a1 = Fa1 + (size_t)ci[1] * ld4;
            const float4* a2 = Fa2 + (size_t)ci[2] * ld4;
            FAcc acc, acc1, acc2, acc3;
            for (int r4 = lane; r4 < ld4; r4 += 32) {
                float4 x0 = __ldg(a0 + r4), x0n = __ldg(a0 + ld4 + r4);
                float4 x1 = __ldg(a1 + r4), x1n = __ldg(a1 + ld4 + r4);
                float4 x2 = __ldg(a2 + r4), x2n = __ldg(a2 + ld4 + r4);
                float u0[4] = {x0.x, x0.y, x0.z, x0.w}, w0[4] = {x0n.x, x0n.y, x0n.z, x0n.w};
                float u1[4] = {x1.x, x1.y, x1.z, x1.w}, w1[4] = {x1n.x, x1n.y, x1n.z, x1n.w};
                float u2[4] = {x2.x, x2.y, x2.z, x2.w}, w2[4] = {x2n.x, x2n.y, x2n.z, x2n.w};
                float s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float d0 = w0[u] - u0[u], d1 = w1[u] - u1[u], d2 = w2[u] - u2[u];
                    float l0 = fmaf(cf[0], d0, u0[u]);
                    float l1 = fmaf(cf[1], d1, u1[u]);
                    float l2 = fmaf(cf[2], d2, u2[u]);
                    // the term l0 l1 l2 with both product roundings recovered by FMA,
                    // each term summed into the pair: the rank terms cancel strongly at
                    // close range, where FP32 partial sums lost ~1e-5 of the energy
                    float l12 = l1 * l2;
                    const float e12 = fmaf(l1, l2, -l12);
                    const float t = l0 * l12;
                    const float et = fmaf(l0, l12, -t);
                    acc.add(t);
                    acc.lo += fmaf(l0, e12, et);
                    if constexpr (GRAD) {
                        s1 = fmaf(d0, l12, s1);
                        s2 = fmaf(l0 * d1, l2, s2);
                        s3 = fmaf(l0 * l1, d2, s3);
                    }
                }
                if constexpr (GRAD) {
                    acc1.add(s1);
                    acc2.add(s2);
                    acc3.add(s3);
                }
            }
            double phi = warp_sum(acc.value());
            double gl[3] = {0.0, 0.0, 0.0};
            if constexpr (GRAD) {
                gl[0] = ins[0] ? warp_sum(acc1.value()) * P.inv_h : 0.0;
                gl[1] = ins[1] ? warp_sum(acc2.value()) * P.inv_h : 0.0;
                gl[2] = ins[2] ? warp_sum(acc3.value()) * P.inv_h : 0.0;
            }
            // short range split over lanes
            F2 phs{0.f, 0.f}, gs[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            int clash = 0;
            short_vdw<GRAD>(P, x, AtomRef{&q, lig.y64 + 3 * j}, lane, 32, phs, gs, clash);
            phi += warp_sum(dev::df_to(phs));
            if constexpr (GRAD)
                for (int a = 0; a < 3; ++a) gl[a] += warp_sum(dev::df_to(gs[a]));
            clash = __any_sync(0xffffffffu, clash);
            if (lane == 0) {
                int fl = clash ? RS_FLAG_CLASH : 0;
                if (!(ins[0] && ins[1] && ins[2])) fl |= RS_FLAG_OUT_OF_GRID;
                if (fl) atomicOr(&pflag[pl], fl);
                // the canonical path sums its rank terms in FP64; its contributions
                // are stored as float pairs like every other path's
                auto put = [&](int c, double v) {
                    const dev::F2 p = dev::df_from(v);
                    cj[c] = make_float2(p.h, p.l);
                };
                double qj = lig.q64[j];
                put(0, qj * phi);
                if constexpr (GRAD) {
                    double g0 = qj * gl[0], g1 = qj * gl[1], g2 = qj * gl[2];
                    put(1, g0);
                    put(2, g1);
                    put(3, g2);
                    double r0 = ry[0], r1 = ry[1], r2 = ry[2];
                    put(4, r1 * g2 - r2 * g1);
                    put(5, r2 * g0 - r0 * g2);
                    put(6, r0 * g1 - r1 * g0);
                }
            }
        }
        __syncthreads();
        reduce_poses<NC>(P, PB, L, p0, Ptot, ps, contrib, pflag, E, flags, gt, gw);
    }
}

// Ligand about its geometric centre (FP64 mean in a fixed order); one CTA.
__global__ void k_prep_ligand(int L, const double* __restrict__ xyz, const double* __restrict__ q,
                              float4* __restrict__ y, float2* __restrict__ yd, double* __restrict__ y64,
                              double* __restrict__ q64) {
    __shared__ double sm[3][256];
    double s[3] = {0, 0, 0};
    for (int j = threadIdx.x; j < L; j += blockDim.x)
        for (int a = 0; a < 3; ++a) s[a] += xyz[3 * (size_t)j + a];
    for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] = s[a];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int a = 0; a < 3; ++a) sm[a][threadIdx.x] += sm[a][threadIdx.x + o];
        __syncthreads();
    }
    double c0 = sm[0][0] / L, c1 = sm[1][0] / L, c2 = sm[2][0] / L;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        double a = xyz[3 * (size_t)j] - c0, b = xyz[3 * (size_t)j + 1] - c1,
               c = xyz[3 * (size_t)j + 2] - c2;
        const dev::F2 pa = dev::df_from(a), pb = dev::df_from(b), pc = dev::df_from(c);
        yd[3 * (size_t)j] = make_float2(pa.h, pa.l);
        yd[3 * (size_t)j + 1] = make_float2(pb.h, pb.l);
        yd[3 * (size_t)j + 2] = make_float2(pc.h, pc.l);
        y64[3 * (size_t)j] = a;
        y64[3 * (size_t)j + 1] = b;
        y64[3 * (size_t)j + 2] = c;
        q64[j] = q[j];
        y[j] = make_float4((float)a, (float)b, (float)c, (float)q[j]);
    }
}

template <bool GRAD>
size_t canon_smem(int PB, int L) {
    size_t s = (size_t)PB * sizeof(PoseSetup) + (size_t)PB * L * (GRAD ? 7 : 1) * 8 + (size_t)PB * 4;
    return (s + 15) / 16 * 16;
}

int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

template <int RP, bool GRAD>
rs_status launch_tucker(const EvalLaunch& a, cudaStream_t st) {
    int PB = a.PB > 0 ? a.PB : std::min(128, std::max(1, 256 / a.lig.L));  // ~256 pose-atoms per block
    size_t sm = wform_smem<RP, GRAD>(PB, a.lig.L);
    while (sm > 160 * 1024 && PB > 1) {
        PB = std::max(1, PB / 2);
        sm = wform_smem<RP, GRAD>(PB, a.lig.L);
    }
    if (sm > 220 * 1024) {
        set_error("ligand too large for the pose kernel (L=%d)", a.lig.L);
        return RS_ERR_UNSUPPORTED;
    }
    auto kern = k_eval_wform<RP, GRAD, 128>;
    const char* kname = GRAD ? "k_eval_wform_grad" : "k_eval_wform";
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, sm));
    long long nblocks = (a.P + PB - 1) / PB;
    long long grid = std::min<long long>(nblocks, (long long)std::max(per_sm, 1) * num_sms());
    if (a.grid > 0) grid = std::min<long long>(nblocks, a.grid);
    if (grid < 1) return RS_OK;
    double work = (double)a.P * a.lig.L * wform_ops_per_atom(RP, GRAD);
    {
        ::rs::KernelTimer kt__(kname, st, work, true, a.events);
        kern<<<(unsigned)grid, 128, sm, st>>>(a.prot, a.lig, a.rot, a.trans, a.P, PB, a.E, a.flags,
                                              a.gt, a.gw, a.skip);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

template <bool GRAD>
rs_status launch_canon(const EvalLaunch& a, cudaStream_t st) {
    int PB = a.PB > 0 ? a.PB : std::min(64, std::max(1, 256 / a.lig.L));
    size_t sm = canon_smem<GRAD>(PB, a.lig.L);
    while (sm > 160 * 1024 && PB > 1) {
        PB = std::max(1, PB / 2);
        sm = canon_smem<GRAD>(PB, a.lig.L);
    }
    if (sm > 220 * 1024) {
        set_error("ligand too large for the pose kernel (L=%d)", a.lig.L);
        return RS_ERR_UNSUPPORTED;
    }
    auto kern = k_eval_canon<GRAD>;
    const char* kname = GRAD ? "k_eval_canon_grad" : "k_eval_canon";
    // FP32 operations per (atom, rank term): 3 differences, 3 lerp FMAs, 2 products,
    // 1 accumulate (energy); the gradient adds 5 products/accumulates
    double work = (double)a.P * a.lig.L * (double)a.prot.R * (GRAD ? 14.0 : 9.0);
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm));
    long long nblocks = (a.P + PB - 1) / PB;
    long long grid = std::min<long long>(nblocks, (long long)std::max(per_sm, 1) * num_sms());
    if (a.grid > 0) grid = std::min<long long>(nblocks, a.grid);
    if (grid < 1) return RS_OK;
    {
        ::rs::KernelTimer kt__(kname, st, work, true, a.events);
        kern<<<(unsigned)grid, 256, sm, st>>>(a.prot, a.lig, a.rot, a.trans, a.P, PB, a.E, a.flags,
                                              a.gt, a.gw, a.skip);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

}  // namespace

rs_status launch_prep_ligand(int L, const double* xyz, const double* q, float4* y, float2* yd, double* y64,
                             double* q64, cudaStream_t st, bool events) {
    {
        ::rs::KernelTimer kt__("k_prep_ligand", st, 0.0, false, events);
        k_prep_ligand<<<1, 256, 0, st>>>(L, xyz, q, y, yd, y64, q64);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

namespace {
// One thread per pose: the atoms' cells by the pose kernels' own geometry helpers, so
// the decision is the one their interpolation took.
__global__ void k_box_flags(ProteinView P, LigandView lig, const double* __restrict__ rot,
                            const double* __restrict__ trans, long long Ptot, bool rotvec,
                            const uint8_t* __restrict__ skip, uint8_t* __restrict__ flags) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Ptot || (skip && skip[p])) return;
    PoseSetup q;
    setup_pose(P, rot, trans, p, rotvec, q);
    bool out = false;
    for (int j = 0; j < lig.L && !out; ++j) {
        dev::F2 x[3];
        atom_position(q, lig.yd + 3 * j, x);
        for (int a = 0; a < 3; ++a) {
            int ci;
            float cf;
            bool ins;
            dev::axis_cell(x[a], dev::F2{P.b_h, P.b_l}, dev::F2{P.inv_h_h, P.inv_h_l}, P.n, ci, cf, ins);
            out = out || ci < P.cell_lo[a] || ci > P.cell_hi[a];
        }
    }
    if (out) flags[p] |= RS_FLAG_OUT_OF_GRID;
}
}  // namespace

rs_status launch_box_flags(const ProteinView& P, const LigandView& lig, const double* rot, const double* trans,
                           long long Ptot, bool rotvec, const uint8_t* skip, uint8_t* flags, cudaStream_t st) {
    if (!P.box || !flags || Ptot <= 0) return RS_OK;
    {
        ::rs::KernelTimer kt__("k_box_flags", st, 0.0, false);
        k_box_flags<<<(unsigned)((Ptot + 127) / 128), 128, 0, st>>>(P, lig, rot, trans, Ptot, rotvec, skip, flags);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

rs_status launch_eval_paths(const EvalLaunch& a, bool grad, cudaStream_t st);

rs_status launch_eval(const EvalLaunch& a, bool grad, cudaStream_t st) {
    RS_TRY(launch_eval_paths(a, grad, st));
    return launch_box_flags(a.prot, a.lig, a.rot, a.trans, a.P, grad, a.skip, a.flags, st);
}

rs_status launch_eval_paths(const EvalLaunch& a, bool grad, cudaStream_t st) {
    if (a.P <= 0) return RS_OK;
    // the cell-grouped path pays six launches and a sort per chunk and one slab load
    // per (warp, cell): it is taken for batches of at least 2^17 pose-atoms that
    // average at least 64 per axis-3 grid cell, without a skip mask (the masked
    // trial passes of rs_pgd_run evaluate few poses; the per-block kernel skips them)
    const long long atoms = a.P * a.lig.L;
    if (a.prot.kind == 1 && a.ws && a.PB == 0 && a.grid == 0 && !a.skip && atoms >= (1LL << 17) &&
        atoms >= 64LL * a.prot.n)
        return launch_sorted(a, grad, st);
    if (a.prot.kind == 0) return grad ? launch_canon<true>(a, st) : launch_canon<false>(a, st);
    switch (a.prot.R) {
#define RS_CASE(R) \
    case R: return grad ? launch_tucker<R, true>(a, st) : launch_tucker<R, false>(a, st);
        RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        default:
            set_error("unsupported padded Tucker rank %d", a.prot.R);
            return RS_ERR_UNSUPPORTED;
    }
}

// Layout of the per-call ligand scratch inside the context buffer.
size_t ligand_scratch_bytes(int L) {
    return ((size_t)L * sizeof(float4) + 2 * (size_t)L * 3 * 8 + (size_t)L * 8 + 256 * 4);
}

LigandView carve_ligand(void* base, int L) {
    char* p = (char*)base;
    LigandView v;
    v.L = L;
    v.y = (const float4*)p;
    p += ((size_t)L * sizeof(float4) + 255) / 256 * 256;
    v.yd = (const float2*)p;
    p += ((size_t)L * 24 + 255) / 256 * 256;
    v.y64 = (const double*)p;
    p += ((size_t)L * 24 + 255) / 256 * 256;
    v.q64 = (const double*)p;
    return v;
}

}  // namespace rs

// ------------------------------------------------------------------ C ABI
namespace {

using namespace rs;

rs_status run_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L, const double* lig_xyz,
                    const double* lig_q, int64_t P, const double* rot, const double* trans,
                    double* E_out, double* dE_dt, double* dE_dw, uint8_t* flags_out,
                    int mem_flags, void* stream, bool grad) {
    clear_error();
    RS_CHECK_ARG(ctx && prot, "NULL context or protein");
    RS_CHECK_ARG(L >= 1 && L <= 4096, "L=%d out of range [1, 4096]", L);
    RS_CHECK_ARG(P >= 0 && P <= 0x7fffffffLL, "P=%lld out of range", (long long)P);
    RS_CHECK_ARG(mem_flags == RS_MEM_HOST || mem_flags == RS_MEM_DEVICE, "bad mem_flags %d", mem_flags);
    RS_CHECK_ARG(prot->device == ctx->device, "protein built on device %d, context on %d",
                 prot->device, ctx->device);
    if (P == 0) return RS_OK;
    RS_CHECK_ARG(lig_xyz && lig_q && rot && trans && E_out, "NULL input or output pointer");
    if (grad) RS_CHECK_ARG(dE_dt && dE_dw, "NULL gradient output");
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;  // NULL: the CUDA default stream
    const int rdim = grad ? 3 : 4;
    // ligand scratch
    RS_TRY(ensure_buffer(&ctx->lig_buf, &ctx->lig_bytes, ligand_scratch_bytes(L) + 1024));
    LigandView lig = carve_ligand(ctx->lig_buf, L);
    const double *d_xyz = lig_xyz, *d_q = lig_q, *d_rot = rot, *d_trans = trans;
    double *d_E = E_out, *d_gt = dE_dt, *d_gw = dE_dw;
    uint8_t* d_flags = flags_out;
    if (mem_flags == RS_MEM_HOST) {
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t o = off;
            off += (bytes + 255) / 256 * 256;
            return o;
        };
        size_t o_xyz = take((size_t)L * 24), o_q = take((size_t)L * 8);
        size_t o_rot = take((size_t)P * rdim * 8), o_tr = take((size_t)P * 24);
        size_t o_E = take((size_t)P * 8), o_f = take((size_t)P);
        size_t o_gt = grad ? take((size_t)P * 24) : 0, o_gw = grad ? take((size_t)P * 24) : 0;
        RS_TRY(ensure_buffer(&ctx->io_buf, &ctx->io_bytes, off));
        char* b = (char*)ctx->io_buf;
        d_xyz = (const double*)(b + o_xyz);
        d_q = (const double*)(b + o_q);
        d_rot = (const double*)(b + o_rot);
        d_trans = (const double*)(b + o_tr);
        d_E = (double*)(b + o_E);
        d_flags = (uint8_t*)(b + o_f);
        if (grad) {
            d_gt = (double*)(b + o_gt);
            d_gw = (double*)(b + o_gw);
        }
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_xyz, lig_xyz, (size_t)L * 24, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_q, lig_q, (size_t)L * 8, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_rot, rot, (size_t)P * rdim * 8, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_trans, trans, (size_t)P * 24, cudaMemcpyHostToDevice, st));
    }
    RS_TRY(launch_prep_ligand(L, d_xyz, d_q, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64, (double*)lig.q64, st));
    EvalLaunch a;
    a.prot = prot->view;
    a.lig = lig;
    a.rot = d_rot;
    a.trans = d_trans;
    a.P = P;
    a.E = d_E;
    a.flags = (mem_flags == RS_MEM_HOST || flags_out) ? d_flags : nullptr;
    a.gt = d_gt;
    a.gw = d_gw;
    if (prot->view.kind == 1) {
        RS_TRY(ensure_buffer(&ctx->eval_buf, &ctx->eval_bytes, sorted_scratch_bytes(P, L, prot->n, grad)));
        a.ws = ctx->eval_buf;
        a.ws_bytes = ctx->eval_bytes;
    }
    RS_TRY(launch_eval(a, grad, st));
    if (mem_flags == RS_MEM_HOST) {
        RS_TRY_CUDA(cudaMemcpyAsync(E_out, d_E, (size_t)P * 8, cudaMemcpyDeviceToHost, st));
        if (flags_out) RS_TRY_CUDA(cudaMemcpyAsync(flags_out, d_flags, (size_t)P, cudaMemcpyDeviceToHost, st));
        if (grad) {
            RS_TRY_CUDA(cudaMemcpyAsync(dE_dt, d_gt, (size_t)P * 24, cudaMemcpyDeviceToHost, st));
            RS_TRY_CUDA(cudaMemcpyAsync(dE_dw, d_gw, (size_t)P * 24, cudaMemcpyDeviceToHost, st));
        }
        RS_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return RS_OK;
}

}  // namespace

extern "C" rs_status rs_energy_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L,
                                     const double* lig_xyz, const double* lig_q, int64_t P,
                                     const double* quat, const double* trans, double* E_out,
                                     uint8_t* flags_out, int mem_flags, void* stream) {
    return run_poses(ctx, prot, L, lig_xyz, lig_q, P, quat, trans, E_out, nullptr, nullptr,
                     flags_out, mem_flags, stream, false);
}

extern "C" rs_status rs_energy_grad_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L,
                                          const double* lig_xyz, const double* lig_q, int64_t P,
                                          const double* rotvec, const double* trans,
                                          double* E_out, double* dE_dt, double* dE_dw,
                                          uint8_t* flags_out, int mem_flags, void* stream) {
    return run_poses(ctx, prot, L, lig_xyz, lig_q, P, rotvec, trans, E_out, dE_dt, dE_dw,
                     flags_out, mem_flags, stream, true);
}

// Finite-difference forces of Eq. differ_ligand and the rigid-cluster resultants of
// Eq. Field_Xcenter / Eq. Field_phi (Tucker-reduced proteins, cell-grouped path).
extern "C" rs_status rs_fd_forces_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L, const double* lig_xyz,
                                        const double* lig_q, int64_t P, const double* rotvec,
                                        const double* trans, double h, double r0, double* E_out, double* F_out,
                                        double* F0_out, double* Fphi_out, double* M_out, uint8_t* flags_out,
                                        int mem_flags, void* stream) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && prot, "NULL context or protein");
    RS_CHECK_ARG(L >= 1 && L <= 4096, "L=%d out of range [1, 4096]", L);
    RS_CHECK_ARG(P >= 0 && P <= (1LL << 29), "P=%lld out of range", (long long)P);
    RS_CHECK_ARG(mem_flags == RS_MEM_HOST || mem_flags == RS_MEM_DEVICE, "bad mem_flags %d", mem_flags);
    RS_CHECK_ARG(prot->device == ctx->device, "protein built on device %d, context on %d", prot->device,
                 ctx->device);
    RS_CHECK_ARG(std::isfinite(h) && h >= 0.0, "finite-difference step h=%g must be finite and >= 0", h);
    RS_CHECK_ARG(std::isfinite(r0) && r0 >= 0.0, "reference radius r0=%g must be finite and >= 0", r0);
    if (prot->view.kind != 1) {
        set_error("finite-difference forces need a Tucker-reduced protein (tucker_cap > 0)");
        return RS_ERR_UNSUPPORTED;
    }
    if (P == 0) return RS_OK;
    RS_CHECK_ARG(lig_xyz && lig_q && rotvec && trans && E_out && F_out && F0_out && Fphi_out && M_out,
                 "NULL input or output pointer");
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const double hs = h > 0.0 ? h : prot->view.h;
    RS_TRY(ensure_buffer(&ctx->lig_buf, &ctx->lig_bytes, ligand_scratch_bytes(L) + 1024));
    LigandView lig = carve_ligand(ctx->lig_buf, L);
    const double *d_xyz = lig_xyz, *d_q = lig_q, *d_rot = rotvec, *d_trans = trans;
    FdOut o{E_out, flags_out, F_out, F0_out, Fphi_out, M_out};
    if (mem_flags == RS_MEM_HOST) {
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t at = off;
            off += (bytes + 255) / 256 * 256;
            return at;
        };
        const size_t o_xyz = take((size_t)L * 24), o_q = take((size_t)L * 8), o_rot = take((size_t)P * 24),
                     o_tr = take((size_t)P * 24), o_E = take((size_t)P * 8), o_f = take((size_t)P),
                     o_F = take((size_t)P * 96);
        RS_TRY(ensure_buffer(&ctx->io_buf, &ctx->io_bytes, off));
        char* b = (char*)ctx->io_buf;
        d_xyz = (const double*)(b + o_xyz);
        d_q = (const double*)(b + o_q);
        d_rot = (const double*)(b + o_rot);
        d_trans = (const double*)(b + o_tr);
        double* F = (double*)(b + o_F);
        o = FdOut{(double*)(b + o_E), (uint8_t*)(b + o_f), F, F + 3 * P, F + 6 * P, F + 9 * P};
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_xyz, lig_xyz, (size_t)L * 24, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_q, lig_q, (size_t)L * 8, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_rot, rotvec, (size_t)P * 24, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_trans, trans, (size_t)P * 24, cudaMemcpyHostToDevice, st));
    }
    RS_TRY(launch_prep_ligand(L, d_xyz, d_q, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64, (double*)lig.q64, st));
    EvalLaunch a;
    a.prot = prot->view;
    a.lig = lig;
    a.rot = d_rot;
    a.trans = d_trans;
    a.P = P;
    RS_TRY(ensure_buffer(&ctx->eval_buf, &ctx->eval_bytes, sorted_fd_scratch_bytes(P, L, prot->n)));
    a.ws = ctx->eval_buf;
    a.ws_bytes = ctx->eval_bytes;
    const long long PC = sorted_fd_chunk_poses(a.ws_bytes, L, prot->n);
    RS_TRY(ensure_buffer(&ctx->fd_buf, &ctx->fd_bytes, fd_pose_bytes(std::max<long long>(PC, 1))));
    RS_TRY(launch_sorted_fd(a, hs, r0, ctx->fd_buf, o, st));
    RS_TRY(launch_box_flags(a.prot, a.lig, a.rot, a.trans, P, true, nullptr, o.flags, st));
    if (mem_flags == RS_MEM_HOST) {
        RS_TRY_CUDA(cudaMemcpyAsync(E_out, o.E, (size_t)P * 8, cudaMemcpyDeviceToHost, st));
        if (flags_out) RS_TRY_CUDA(cudaMemcpyAsync(flags_out, o.flags, (size_t)P, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(F_out, o.F, (size_t)P * 24, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(F0_out, o.F0, (size_t)P * 24, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(Fphi_out, o.Fphi, (size_t)P * 24, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(M_out, o.M, (size_t)P * 24, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return RS_OK;
}

namespace rs {
namespace {
// E += E_p, flags |= flags_p (one molecule's contribution to the complex).
__global__ void k_complex_acc(long long P, const double* __restrict__ Ep, const uint8_t* __restrict__ fp,
                              double* __restrict__ E, uint8_t* __restrict__ F, int first) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    E[i] = first ? Ep[i] : E[i] + Ep[i];
    F[i] = first ? fp[i] : (uint8_t)(F[i] | fp[i]);
}
}  // namespace
}  // namespace rs

// A molecular complex against a ligand molecule (Sec. 5.1, Eq. EnergySum_Mcomplex):
// the pose path per molecule, summed on the device in molecule order.
extern "C" rs_status rs_energy_poses_complex(rs_ctx* ctx, int32_t nmol, const rs_protein* const* mols, int32_t L,
                                             const double* lig_xyz, const double* lig_q, int64_t P,
                                             const double* quat, const double* trans, double* E_out,
                                             uint8_t* flags_out, int mem_flags, void* stream) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && mols && nmol >= 1 && nmol <= 64, "NULL context or molecule list, or nmol=%d not in [1, 64]",
                 nmol);
    for (int i = 0; i < nmol; ++i) {
        RS_CHECK_ARG(mols[i], "molecule %d is NULL", i);
        RS_CHECK_ARG(mols[i]->device == ctx->device, "molecule %d on device %d, context on %d", i, mols[i]->device,
                     ctx->device);
    }
    RS_CHECK_ARG(L >= 1 && L <= 4096, "L=%d out of range [1, 4096]", L);
    RS_CHECK_ARG(P >= 0 && P <= 0x7fffffffLL, "P=%lld out of range", (long long)P);
    RS_CHECK_ARG(mem_flags == RS_MEM_HOST || mem_flags == RS_MEM_DEVICE, "bad mem_flags %d", mem_flags);
    if (P == 0) return RS_OK;
    RS_CHECK_ARG(lig_xyz && lig_q && quat && trans && E_out, "NULL input or output pointer");
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    RS_TRY(ensure_buffer(&ctx->lig_buf, &ctx->lig_bytes, ligand_scratch_bytes(L) + 1024));
    LigandView lig = carve_ligand(ctx->lig_buf, L);
    // staging: inputs (host calls), the sums, one molecule's energies and flags
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_xyz = take((size_t)L * 24), o_q = take((size_t)L * 8), o_rot = take((size_t)P * 32),
                 o_tr = take((size_t)P * 24), o_E = take((size_t)P * 8), o_F = take((size_t)P),
                 o_Ep = take((size_t)P * 8), o_Fp = take((size_t)P);
    RS_TRY(ensure_buffer(&ctx->fd_buf, &ctx->fd_bytes, off));
    char* b = (char*)ctx->fd_buf;
    const double *d_xyz = lig_xyz, *d_q = lig_q, *d_rot = quat, *d_trans = trans;
    double* d_E = E_out;
    uint8_t* d_F = (uint8_t*)(b + o_F);
    if (mem_flags == RS_MEM_DEVICE && flags_out) d_F = flags_out;
    if (mem_flags == RS_MEM_HOST) {
        d_xyz = (const double*)(b + o_xyz);
        d_q = (const double*)(b + o_q);
        d_rot = (const double*)(b + o_rot);
        d_trans = (const double*)(b + o_tr);
        d_E = (double*)(b + o_E);
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_xyz, lig_xyz, (size_t)L * 24, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_q, lig_q, (size_t)L * 8, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_rot, quat, (size_t)P * 32, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_trans, trans, (size_t)P * 24, cudaMemcpyHostToDevice, st));
    }
    RS_TRY(launch_prep_ligand(L, d_xyz, d_q, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64, (double*)lig.q64, st));
    double* Ep = (double*)(b + o_Ep);
    uint8_t* Fp = (uint8_t*)(b + o_Fp);
    for (int i = 0; i < nmol; ++i) {
        const rs_protein* prot = mols[i];
        EvalLaunch a;
        a.prot = prot->view;
        a.lig = lig;
        a.rot = d_rot;
        a.trans = d_trans;
        a.P = P;
        a.E = Ep;
        a.flags = Fp;
        if (prot->view.kind == 1) {
            RS_TRY(ensure_buffer(&ctx->eval_buf, &ctx->eval_bytes, sorted_scratch_bytes(P, L, prot->n, false)));
            a.ws = ctx->eval_buf;
            a.ws_bytes = ctx->eval_bytes;
        }
        RS_TRY(launch_eval(a, false, st));
        {
            ::rs::KernelTimer kt__("k_complex_acc", st, 0.0, false);
            k_complex_acc<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(P, Ep, Fp, d_E, d_F, i == 0);
        }
        RS_TRY_CUDA(cudaGetLastError());
    }
    if (mem_flags == RS_MEM_HOST) {
        RS_TRY_CUDA(cudaMemcpyAsync(E_out, d_E, (size_t)P * 8, cudaMemcpyDeviceToHost, st));
        if (flags_out) RS_TRY_CUDA(cudaMemcpyAsync(flags_out, d_F, (size_t)P, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return RS_OK;
}
