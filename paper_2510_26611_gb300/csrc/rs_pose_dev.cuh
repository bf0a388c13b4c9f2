// Device code of the pose kernels shared by the plain and batched launches:
// pose setup, short-range/vdW walk, per-pose reduction, and one block of the
// W-form (Tucker) evaluation.  Included by rs_eval.cu and rs_batch.cu.
#pragma once

#include "rs_common.cuh"

namespace rs {
namespace {

using dev::FAcc;

struct PoseSetup {
    double R[9];
    double t[3];
    double s[3];      // (t + b) / h
    double J[9];      // left Jacobian (gradient kernels)
    float Rf[9];
    int valid;
};

__device__ __forceinline__ void setup_pose(const ProteinView& P, const double* __restrict__ rot,
                                           const double* __restrict__ trans, long long p,
                                           bool rotvec, PoseSetup& ps) {
    if (rotvec) {
        double wx = rot[3 * p], wy = rot[3 * p + 1], wz = rot[3 * p + 2];
        dev::rotvec_to_rot(wx, wy, wz, ps.R);
        dev::left_jacobian(wx, wy, wz, ps.J);
    } else {
        dev::quat_to_rot(rot[4 * p], rot[4 * p + 1], rot[4 * p + 2], rot[4 * p + 3], ps.R);
    }
    for (int a = 0; a < 9; ++a) ps.Rf[a] = (float)ps.R[a];
    for (int a = 0; a < 3; ++a) {
        ps.t[a] = trans[3 * p + a];
        ps.s[a] = (ps.t[a] + P.b) * P.inv_h;
    }
    ps.valid = 1;
}

// Short-range part and vdW decision for one atom; candidates split over
// `nl` cooperating lanes starting at `lane`.  Distances are screened in FP32;
// pairs inside the cutoff, and vdW decisions within 1e-4 relative of sigma^2,
// are taken in FP64 from x = t + R y evaluated in FP64.
template <bool GRAD>
__device__ __forceinline__ void short_vdw(const ProteinView& P, const float xf[3],
                                          const double x64[3], int lane, int nl, double& phi,
                                          double g[3], int& clash) {
    float u0 = (xf[0] - P.co0) * P.inv_cell, u1 = (xf[1] - P.co1) * P.inv_cell,
          u2 = (xf[2] - P.co2) * P.inv_cell;
    u0 = fminf(fmaxf(u0, -4.f), (float)P.nc0 + 4.f);
    u1 = fminf(fmaxf(u1, -4.f), (float)P.nc1 + 4.f);
    u2 = fminf(fmaxf(u2, -4.f), (float)P.nc2 + 4.f);
    int c0 = (int)floorf(u0), c1 = (int)floorf(u1), c2 = (int)floorf(u2);
    for (int dz = -1; dz <= 1; ++dz) {
        int cz = c2 + dz;
        if (cz < 0 || cz >= P.nc2) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int cy = c1 + dy;
            if (cy < 0 || cy >= P.nc1) continue;
            int x_lo = max(c0 - 1, 0), x_hi = min(c0 + 1, P.nc0 - 1);
            if (x_lo > x_hi) continue;
            int base = (cz * P.nc1 + cy) * P.nc0;
            int s = P.cell_start[base + x_lo], e = P.cell_start[base + x_hi + 1];
            for (int k = s + lane; k < e; k += nl) {
                float4 a = P.atoms[k];
                float e0 = xf[0] - a.x, e1 = xf[1] - a.y, e2 = xf[2] - a.z;
                float d2 = e0 * e0 + e1 * e1 + e2 * e2;
                bool near_sig = d2 < P.sig2_hi;
                bool near_rc = d2 < P.rc2_hi;
                if (!(near_sig || near_rc)) continue;
                D4 a64 = P.atoms64[k];
                double f0 = x64[0] - a64.x, f1 = x64[1] - a64.y, f2 = x64[2] - a64.z;
                double d2d = f0 * f0 + f1 * f1 + f2 * f2;
                if (near_sig && (d2 < P.sig2_lo || d2d < P.sig2)) clash = 1;
                if (near_rc && d2d < P.rc2) {
                    // cubic Hermite interpolation of the tabulated radial function (FP64)
                    double xs = d2d * P.stab_inv_h;
                    int j = min((int)xs, P.stab_n - 2);
                    double u = xs - j;
                    double2 A = P.stab[j], B = P.stab[j + 1];
                    double u2 = u * u, u3 = u2 * u;
                    double fv = (2.0 * u3 - 3.0 * u2 + 1.0) * A.x + (u3 - 2.0 * u2 + u) * A.y +
                                (3.0 * u2 - 2.0 * u3) * B.x + (u3 - u2) * B.y;
                    phi += a64.w * fv;
                    if constexpr (GRAD) {
                        double dp = (6.0 * u2 - 6.0 * u) * (A.x - B.x) + (3.0 * u2 - 4.0 * u + 1.0) * A.y +
                                    (3.0 * u2 - 2.0 * u) * B.y;
                        double fgr = 2.0 * a64.w * dp * P.stab_inv_h;  // grad_x f(|x-x_m|^2)
                        g[0] += fgr * f0;
                        g[1] += fgr * f1;
                        g[2] += fgr * f2;
                    }
                }
            }
        }
    }
}

// FP64 atom position x = R y + t (the interpolation coordinates and the
// short-range distances use it; FP32 rotation alone misplaces atoms by ~1e-6 A).
__device__ __forceinline__ void atom_position(const PoseSetup& q, const double* __restrict__ y64,
                                              double x64[3]) {
    double y0 = y64[0], y1 = y64[1], y2 = y64[2];
    for (int r = 0; r < 3; ++r)
        x64[r] = q.t[r] + (q.R[3 * r] * y0 + q.R[3 * r + 1] * y1 + q.R[3 * r + 2] * y2);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduction of per-atom contributions to per-pose outputs (one warp per pose).
template <int NC>
__device__ void reduce_poses(const ProteinView& P, int PB, int L, long long p0, long long Ptot,
                             const PoseSetup* ps, const double* contrib, const int* pflag,
                             double* __restrict__ E, uint8_t* __restrict__ flags,
                             double* __restrict__ gt, double* __restrict__ gw) {
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    for (int pl = warp; pl < PB; pl += nw) {
        long long p = p0 + pl;
        if (p >= Ptot) break;
        if (!ps[pl].valid) continue;  // skipped pose: outputs untouched
        double s[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = 0.0;
        for (int j = lane; j < L; j += 32) {
            const double* cj = contrib + ((size_t)pl * L + j) * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) s[c] += cj[c];
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = warp_sum(s[c]);
        if (lane == 0) {
            E[p] = s[0];
            if (flags) flags[p] = (uint8_t)pflag[pl];
            if (NC == 7) {
                const PoseSetup& q = ps[pl];
                for (int a = 0; a < 3; ++a) gt[3 * p + a] = s[1 + a];
                // dE/dw = J_l^T tau
                for (int a = 0; a < 3; ++a)
                    gw[3 * p + a] = q.J[a] * s[4] + q.J[3 + a] * s[5] + q.J[6 + a] * s[6];
            }
        }
    }
}

// ------------------------------------------------------------------ Tucker path
// Thread per atom.  The Tucker form phi = sum_abc core[a][b][c] v1_a v2_b v3_c is
// evaluated through its exact rewrite W[i][a][b] = sum_c V3'[i][c] core[a][b][c]:
//   t_ab = W[i3][a][b] + f3 D[i3][a][b]            (interpolation along axis 3)
//   phi  = sum_a v1_a sum_b v2_b t_ab               (v_l = lerp of V'^(l) rows)
// with every factor stored as a float pair and sums carried as pairs (Dot2), so the
// per-atom value keeps ~2^-44 relative accuracy even where the terms cancel.
// One block of PB poses starting at p0 (PB <= 128): pose setup, per-atom
// evaluation, per-pose reduction.  NT threads; `smem` laid out by wform_smem.
template <int RP, bool GRAD, int NT>
__device__ __forceinline__ void wform_block(const ProteinView& P, const LigandView& lig,
                                            const double* __restrict__ rot,
                                            const double* __restrict__ trans, long long Ptot,
                                            int PB, long long p0, double* __restrict__ E,
                                            uint8_t* __restrict__ flags, double* __restrict__ gt,
                                            double* __restrict__ gw, unsigned char* smem,
                                            const uint8_t* __restrict__ skip = nullptr) {
    using dev::F2;
    constexpr int NC = GRAD ? 7 : 1;
    constexpr int NV = GRAD ? 4 : 2;  // per-thread smem planes: v1h, v1l (, dv1h, dv1l)
    float* v1s = (float*)smem;                                   // [NV][RP][NT]
    PoseSetup* ps = (PoseSetup*)(v1s + NV * RP * NT);
    double* contrib = (double*)(ps + PB);
    int* pflag = (int*)(contrib + (size_t)PB * lig.L * NC);
    const int L = lig.L;
    const int tid = threadIdx.x;
    __syncthreads();
    for (int pl = tid; pl < PB; pl += blockDim.x) {
        long long p = p0 + pl;
        pflag[pl] = 0;
        if (p < Ptot && !(skip && skip[p])) setup_pose(P, rot, trans, p, GRAD, ps[pl]);
        else ps[pl].valid = 0;
    }
    __syncthreads();
    for (int g = tid; g < PB * L; g += NT) {
        int pl = g / L, j = g - pl * L;
        double* cj = contrib + (size_t)g * NC;
        const PoseSetup& q = ps[pl];
        if (!q.valid) {
#pragma unroll
            for (int c = 0; c < NC; ++c) cj[c] = 0.0;
            continue;
        }
        float4 yq = lig.y[j];
        float ry[3];
        for (int r = 0; r < 3; ++r)
            ry[r] = q.Rf[3 * r] * yq.x + q.Rf[3 * r + 1] * yq.y + q.Rf[3 * r + 2] * yq.z;
        int ci[3];
        float cf[3];
        bool ins[3];
        double x64[3];
        atom_position(q, lig.y64 + 3 * j, x64);
        for (int a = 0; a < 3; ++a) dev::axis_cell(x64[a], P.b, P.inv_h, P.n, ci[a], cf[a], ins[a]);
        // v1 (axis 1) into this thread's shared-memory column; v2 (axis 2) in registers
        {
            size_t o = (size_t)ci[0] * RP;
            const float4* vh = (const float4*)(P.Vt[0][0] + o);
            const float4* vl = (const float4*)(P.Vt[0][1] + o);
            const float4* dh = (const float4*)(P.Vt[0][2] + o);
            const float4* dl = (const float4*)(P.Vt[0][3] + o);
#pragma unroll
            for (int c4 = 0; c4 < RP / 4; ++c4) {
                float4 a = __ldg(vh + c4), b = __ldg(vl + c4), c = __ldg(dh + c4), d = __ldg(dl + c4);
                float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
                float cv[4] = {c.x, c.y, c.z, c.w}, dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    F2 v = dev::df_lerp(F2{av[u], bv[u]}, F2{cv[u], dv[u]}, cf[0]);
                    int col = 4 * c4 + u;
                    v1s[(0 * RP + col) * NT + tid] = v.h;
                    v1s[(1 * RP + col) * NT + tid] = v.l;
                    if constexpr (GRAD) {
                        v1s[(2 * RP + col) * NT + tid] = ins[0] ? cv[u] : 0.f;
                        v1s[(3 * RP + col) * NT + tid] = ins[0] ? dv[u] : 0.f;
                    }
                }
            }
        }
        F2 v2[RP];
        F2 dv2[GRAD ? RP : 1];
        {
            size_t o = (size_t)ci[1] * RP;
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
                    v2[4 * c4 + u] = dev::df_lerp(F2{av[u], bv[u]}, F2{cv[u], dv[u]}, cf[1]);
                    if constexpr (GRAD) dv2[4 * c4 + u] = ins[1] ? F2{cv[u], dv[u]} : F2{0.f, 0.f};
                }
            }
        }
        const size_t wrow = (size_t)ci[2] * RP * RP;
        const float* Wh = P.Wt[0] + wrow;
        const float* Wl = P.Wt[1] + wrow;
        const float* Dh = P.Wt[2] + wrow;
        const float* Dl = P.Wt[3] + wrow;
        const float f3 = cf[2];
        const bool in3 = ins[2];
        F2 phi{0.f, 0.f}, g1{0.f, 0.f}, g2{0.f, 0.f}, g3{0.f, 0.f};
        for (int a = 0; a < RP; ++a) {
            F2 u{0.f, 0.f}, u2{0.f, 0.f}, u3{0.f, 0.f};
            const float4* wh = (const float4*)(Wh + a * RP);
            const float4* wl = (const float4*)(Wl + a * RP);
            const float4* dh = (const float4*)(Dh + a * RP);
            const float4* dl = (const float4*)(Dl + a * RP);
#pragma unroll
            for (int b4 = 0; b4 < RP / 4; ++b4) {
                float4 xa = __ldg(wh + b4), xb = __ldg(wl + b4), xc = __ldg(dh + b4), xd = __ldg(dl + b4);
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
            F2 va{v1s[(0 * RP + a) * NT + tid], v1s[(1 * RP + a) * NT + tid]};
            dev::df_fma_acc(phi, va, u);
            if constexpr (GRAD) {
                F2 dva{v1s[(2 * RP + a) * NT + tid], v1s[(3 * RP + a) * NT + tid]};
                dev::df_fma_acc(g1, dva, u);
                dev::df_fma_acc(g2, va, u2);
                dev::df_fma_acc(g3, va, u3);
            }
        }
        double ph = (double)phi.h + (double)phi.l;
        double gl[3] = {0.0, 0.0, 0.0};
        if constexpr (GRAD) {
            gl[0] = ((double)g1.h + (double)g1.l) * P.inv_h;
            gl[1] = ((double)g2.h + (double)g2.l) * P.inv_h;
            gl[2] = ((double)g3.h + (double)g3.l) * P.inv_h;
        }
        // short range and vdW
        float xf[3];
        for (int a = 0; a < 3; ++a) xf[a] = (float)x64[a];
        int clash = 0;
        short_vdw<GRAD>(P, xf, x64, 0, 1, ph, gl, clash);
        int fl = clash ? RS_FLAG_CLASH : 0;
        if (!(ins[0] && ins[1] && ins[2])) fl |= RS_FLAG_OUT_OF_GRID;
        if (fl) atomicOr(&pflag[pl], fl);
        double qj = lig.q64[j];
        cj[0] = qj * ph;
        if constexpr (GRAD) {
            double g0 = qj * gl[0], g1d = qj * gl[1], g2d = qj * gl[2];
            cj[1] = g0;
            cj[2] = g1d;
            cj[3] = g2d;
            double r0 = ry[0], r1 = ry[1], r2 = ry[2];
            cj[4] = r1 * g2d - r2 * g1d;
            cj[5] = r2 * g0 - r0 * g2d;
            cj[6] = r0 * g1d - r1 * g0;
        }
    }
    __syncthreads();
    reduce_poses<NC>(P, PB, L, p0, Ptot, ps, contrib, pflag, E, flags, gt, gw);
}

template <int RP, bool GRAD, int NT = 128>
size_t wform_smem(int PB, int L) {
    size_t s = (size_t)(GRAD ? 4 : 2) * RP * NT * 4;
    s += (size_t)PB * sizeof(PoseSetup);
    s += (size_t)PB * L * (GRAD ? 7 : 1) * 8;
    s += (size_t)PB * 4;
    return (s + 15) / 16 * 16;
}

// FP32 flops (FMA = 2) per atom of the W-form evaluation: per (a, b) one pair
// lerp (16) and one (energy) or three (gradient) Dot2 steps (15 each); per a one
// or four Dot2 steps; one pair lerp (16) per column of v1 and v2; pose transform,
// cell index and reduction ~60 (energy) / ~80 (gradient).
inline double wform_flops_per_atom(int RP, bool grad) {
    double r = RP;
    return grad ? 61.0 * r * r + 92.0 * r + 80.0 : 31.0 * r * r + 47.0 * r + 60.0;
}

}  // namespace
}  // namespace rs
