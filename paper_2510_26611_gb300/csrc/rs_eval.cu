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
                                          const PoseSetup& ps, const double* __restrict__ y64,
                                          int lane, int nl, double& phi, double g[3],
                                          int& clash) {
    float u0 = (xf[0] - P.co0) * P.inv_cell, u1 = (xf[1] - P.co1) * P.inv_cell,
          u2 = (xf[2] - P.co2) * P.inv_cell;
    u0 = fminf(fmaxf(u0, -4.f), (float)P.nc0 + 4.f);
    u1 = fminf(fmaxf(u1, -4.f), (float)P.nc1 + 4.f);
    u2 = fminf(fmaxf(u2, -4.f), (float)P.nc2 + 4.f);
    int c0 = (int)floorf(u0), c1 = (int)floorf(u1), c2 = (int)floorf(u2);
    bool have64 = false;
    double x64[3];
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
                if (!have64) {
                    for (int r = 0; r < 3; ++r)
                        x64[r] = ps.t[r] + (ps.R[3 * r] * y64[0] + ps.R[3 * r + 1] * y64[1] +
                                            ps.R[3 * r + 2] * y64[2]);
                    have64 = true;
                }
                D4 a64 = P.atoms64[k];
                double f0 = x64[0] - a64.x, f1 = x64[1] - a64.y, f2 = x64[2] - a64.z;
                double d2d = f0 * f0 + f1 * f1 + f2 * f2;
                if (near_sig && (d2 < P.sig2_lo || d2d < P.sig2)) clash = 1;
                if (near_rc && d2d < P.rc2) {
                    float d2f = (float)d2d;
                    float sv = 0.f, sd = 0.f;
                    for (int q = 0; q < P.Ks; ++q) {
                        float ev = P.as[q] * expf(-P.ts2[q] * d2f);
                        sv += ev;
                        if constexpr (GRAD) sd += P.ts2[q] * ev;
                    }
                    phi += a64.w * (double)sv;
                    if constexpr (GRAD) {
                        double fgr = -2.0 * a64.w * (double)sd;
                        g[0] += fgr * f0;
                        g[1] += fgr * f1;
                        g[2] += fgr * f2;
                    }
                }
            }
        }
    }
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
template <int RP, bool GRAD>
__global__ void __launch_bounds__(128) k_eval_wform(ProteinView P, LigandView lig,
                                                    const double* __restrict__ rot,
                                                    const double* __restrict__ trans,
                                                    long long Ptot, int PB,
                                                    double* __restrict__ E,
                                                    uint8_t* __restrict__ flags,
                                                    double* __restrict__ gt,
                                                    double* __restrict__ gw) {
    using dev::F2;
    constexpr int NC = GRAD ? 7 : 1;
    constexpr int NT = 128;
    constexpr int NV = GRAD ? 4 : 2;  // per-thread smem planes: v1h, v1l (, dv1h, dv1l)
    extern __shared__ __align__(16) unsigned char smem[];
    float* v1s = (float*)smem;                                   // [NV][RP][NT]
    PoseSetup* ps = (PoseSetup*)(v1s + NV * RP * NT);
    double* contrib = (double*)(ps + PB);
    int* pflag = (int*)(contrib + (size_t)PB * lig.L * NC);

    const int L = lig.L;
    const long long nblocks = (Ptot + PB - 1) / PB;
    const float inv_h = (float)P.inv_h;
    const int tid = threadIdx.x;
    for (long long pb = blockIdx.x; pb < nblocks; pb += gridDim.x) {
        long long p0 = pb * PB;
        __syncthreads();
        for (int pl = tid; pl < PB; pl += blockDim.x) {
            long long p = p0 + pl;
            pflag[pl] = 0;
            if (p < Ptot) setup_pose(P, rot, trans, p, GRAD, ps[pl]);
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
            for (int a = 0; a < 3; ++a) dev::axis_cell(q.s[a], ry[a] * inv_h, P.n, ci[a], cf[a], ins[a]);
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
            for (int a = 0; a < 3; ++a) xf[a] = (float)(q.t[a] + (double)ry[a]);
            int clash = 0;
            short_vdw<GRAD>(P, xf, q, lig.y64 + 3 * j, 0, 1, ph, gl, clash);
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
                                                    double* __restrict__ gw) {
    constexpr int NC = GRAD ? 7 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    PoseSetup* ps = (PoseSetup*)smem;
    double* contrib = (double*)(ps + PB);
    int* pflag = (int*)(contrib + (size_t)PB * lig.L * NC);
    const int L = lig.L;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    const long long nblocks = (Ptot + PB - 1) / PB;
    const float inv_h = (float)P.inv_h;
    const int ld4 = P.ld / 4;
    const float4* F0 = (const float4*)P.F[0];
    const float4* F1 = (const float4*)P.F[1];
    const float4* F2 = (const float4*)P.F[2];
    for (long long pb = blockIdx.x; pb < nblocks; pb += gridDim.x) {
        long long p0 = pb * PB;
        __syncthreads();
        for (int pl = threadIdx.x; pl < PB; pl += blockDim.x) {
            long long p = p0 + pl;
            pflag[pl] = 0;
            if (p < Ptot) setup_pose(P, rot, trans, p, GRAD, ps[pl]);
            else ps[pl].valid = 0;
        }
        __syncthreads();
        for (int g = warp; g < PB * L; g += nw) {
            int pl = g / L, j = g - pl * L;
            double* cj = contrib + (size_t)g * NC;
            const PoseSetup& q = ps[pl];
            if (!q.valid) {
                if (lane < NC) cj[lane] = 0.0;
                continue;
            }
            float4 yq = lig.y[j];
            float ry[3];
            for (int r = 0; r < 3; ++r)
                ry[r] = q.Rf[3 * r] * yq.x + q.Rf[3 * r + 1] * yq.y + q.Rf[3 * r + 2] * yq.z;
            int ci[3];
            float cf[3];
            bool ins[3];
            for (int a = 0; a < 3; ++a) dev::axis_cell(q.s[a], ry[a] * inv_h, P.n, ci[a], cf[a], ins[a]);
            const float4* a0 = F0 + (size_t)ci[0] * ld4;
            const float4* a1 = F1 + (size_t)ci[1] * ld4;
            const float4* a2 = F2 + (size_t)ci[2] * ld4;
            FAcc acc, acc1, acc2, acc3;
            for (int r4 = lane; r4 < ld4; r4 += 32) {
                float4 x0 = __ldg(a0 + r4), x0n = __ldg(a0 + ld4 + r4);
                float4 x1 = __ldg(a1 + r4), x1n = __ldg(a1 + ld4 + r4);
                float4 x2 = __ldg(a2 + r4), x2n = __ldg(a2 + ld4 + r4);
                float u0[4] = {x0.x, x0.y, x0.z, x0.w}, w0[4] = {x0n.x, x0n.y, x0n.z, x0n.w};
                float u1[4] = {x1.x, x1.y, x1.z, x1.w}, w1[4] = {x1n.x, x1n.y, x1n.z, x1n.w};
                float u2[4] = {x2.x, x2.y, x2.z, x2.w}, w2[4] = {x2n.x, x2n.y, x2n.z, x2n.w};
                float s = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float d0 = w0[u] - u0[u], d1 = w1[u] - u1[u], d2 = w2[u] - u2[u];
                    float l0 = fmaf(cf[0], d0, u0[u]);
                    float l1 = fmaf(cf[1], d1, u1[u]);
                    float l2 = fmaf(cf[2], d2, u2[u]);
                    float l12 = l1 * l2;
                    s = fmaf(l0, l12, s);
                    if constexpr (GRAD) {
                        s1 = fmaf(d0, l12, s1);
                        s2 = fmaf(l0 * d1, l2, s2);
                        s3 = fmaf(l0 * l1, d2, s3);
                    }
                }
                acc.add(s);
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
            float xf[3];
            for (int a = 0; a < 3; ++a) xf[a] = (float)(q.t[a] + (double)ry[a]);
            double phs = 0.0, gs[3] = {0.0, 0.0, 0.0};
            int clash = 0;
            short_vdw<GRAD>(P, xf, q, lig.y64 + 3 * j, lane, 32, phs, gs, clash);
            phi += warp_sum(phs);
            if constexpr (GRAD)
                for (int a = 0; a < 3; ++a) gl[a] += warp_sum(gs[a]);
            clash = __any_sync(0xffffffffu, clash);
            if (lane == 0) {
                int fl = clash ? RS_FLAG_CLASH : 0;
                if (!(ins[0] && ins[1] && ins[2])) fl |= RS_FLAG_OUT_OF_GRID;
                if (fl) atomicOr(&pflag[pl], fl);
                double qj = lig.q64[j];
                cj[0] = qj * phi;
                if constexpr (GRAD) {
                    double g0 = qj * gl[0], g1 = qj * gl[1], g2 = qj * gl[2];
                    cj[1] = g0;
                    cj[2] = g1;
                    cj[3] = g2;
                    double r0 = ry[0], r1 = ry[1], r2 = ry[2];
                    cj[4] = r1 * g2 - r2 * g1;
                    cj[5] = r2 * g0 - r0 * g2;
                    cj[6] = r0 * g1 - r1 * g0;
                }
            }
        }
        __syncthreads();
        reduce_poses<NC>(P, PB, L, p0, Ptot, ps, contrib, pflag, E, flags, gt, gw);
    }
}

// Ligand about its geometric centre (FP64 mean in a fixed order); one CTA.
__global__ void k_prep_ligand(int L, const double* __restrict__ xyz, const double* __restrict__ q,
                              float4* __restrict__ y, double* __restrict__ y64,
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
        y64[3 * (size_t)j] = a;
        y64[3 * (size_t)j + 1] = b;
        y64[3 * (size_t)j + 2] = c;
        q64[j] = q[j];
        y[j] = make_float4((float)a, (float)b, (float)c, (float)q[j]);
    }
}

template <int RP, bool GRAD>
size_t wform_smem(int PB, int L) {
    size_t s = (size_t)(GRAD ? 4 : 2) * RP * 128 * 4;
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
    int PB = a.PB > 0 ? a.PB : std::min(128, std::max(1, 512 / a.lig.L));
    size_t sm = wform_smem<RP, GRAD>(PB, a.lig.L);
    while (sm > 160 * 1024 && PB > 1) {
        PB = std::max(1, PB / 2);
        sm = wform_smem<RP, GRAD>(PB, a.lig.L);
    }
    if (sm > 220 * 1024) {
        set_error("ligand too large for the pose kernel (L=%d)", a.lig.L);
        return RS_ERR_UNSUPPORTED;
    }
    auto kern = k_eval_wform<RP, GRAD>;
    const char* kname = GRAD ? "k_eval_wform_grad" : "k_eval_wform";
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, sm));
    long long nblocks = (a.P + PB - 1) / PB;
    long long grid = std::min<long long>(nblocks, (long long)std::max(per_sm, 1) * num_sms());
    if (a.grid > 0) grid = std::min<long long>(nblocks, a.grid);
    if (grid < 1) return RS_OK;
    double work = (double)a.P * a.lig.L * wform_flops_per_atom(RP, GRAD);
    {
        ::rs::KernelTimer kt__(kname, st, work, true, a.events);
        kern<<<(unsigned)grid, 128, sm, st>>>(a.prot, a.lig, a.rot, a.trans, a.P, PB, a.E, a.flags,
                                              a.gt, a.gw);
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
                                              a.gt, a.gw);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

}  // namespace

rs_status launch_prep_ligand(int L, const double* xyz, const double* q, float4* y, double* y64,
                             double* q64, cudaStream_t st, bool events) {
    {
        ::rs::KernelTimer kt__("k_prep_ligand", st, 0.0, false, events);
        k_prep_ligand<<<1, 256, 0, st>>>(L, xyz, q, y, y64, q64);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

rs_status launch_eval(const EvalLaunch& a, bool grad, cudaStream_t st) {
    if (a.P <= 0) return RS_OK;
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
    return ((size_t)L * sizeof(float4) + (size_t)L * 3 * 8 + (size_t)L * 8 + 256 * 3);
}

LigandView carve_ligand(void* base, int L) {
    char* p = (char*)base;
    LigandView v;
    v.L = L;
    v.y = (const float4*)p;
    p += ((size_t)L * sizeof(float4) + 255) / 256 * 256;
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
    RS_TRY(launch_prep_ligand(L, d_xyz, d_q, (float4*)lig.y, (double*)lig.y64, (double*)lig.q64, st));
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
