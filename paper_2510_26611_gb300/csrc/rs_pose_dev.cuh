// Device code of the pose kernels shared by the plain and batched launches:
// pose setup, short-range/vdW walk, per-pose reduction, and one block of the
// W-form (Tucker) evaluation.  Included by rs_eval.cu and rs_batch.cu.
#pragma once

#include "rs_common.cuh"

namespace rs {
namespace {

using dev::FAcc;

using dev::F2;

struct PoseSetup {
    double R[9];
    double t[3];
    double J[9];      // left Jacobian (gradient kernels)
    F2 Rd[9];         // R and t as float pairs (atom positions)
    F2 td[3];
    float Rf[9];      // R in FP32 (torque arm)
    int valid;
};

// FP64 position x = t + R y (12 FP64 operations; used only for vdW decisions
// inside the sigma band, where the FP64 oracle's decision must be reproduced).
__device__ __forceinline__ void atom_position64(const PoseSetup& q, const double* __restrict__ y64,
                                                double x64[3]) {
    const double y0 = y64[0], y1 = y64[1], y2 = y64[2];
    for (int r = 0; r < 3; ++r)
        x64[r] = __dadd_rn(q.t[r], fma(q.R[3 * r + 2], y2, fma(q.R[3 * r + 1], y1, __dmul_rn(q.R[3 * r], y0))));
}

// Where an atom's FP64 position comes from: its pose's FP64 setup and its FP64
// ligand coordinates.  The position is formed only for the rare pair that falls
// inside the +-1e-4 sigma^2 band (GB300 runs FP64 at 1/64 of its FP32 rate, and
// every other decision is taken in FP32 or pair arithmetic).
struct AtomRef {
    const PoseSetup* q;
    const double* y64;
    __device__ __forceinline__ void pos64(double x64[3]) const { atom_position64(*q, y64, x64); }
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
    for (int a = 0; a < 9; ++a) {
        ps.Rf[a] = (float)ps.R[a];
        ps.Rd[a] = dev::df_from(ps.R[a]);
    }
    for (int a = 0; a < 3; ++a) {
        ps.t[a] = trans[3 * p + a];
        ps.td[a] = dev::df_from(ps.t[a]);
    }
    ps.valid = 1;
}

// Candidate list [s, e) of the fine cell holding an FP32 position (empty outside the
// fine grid: no protein atom lies within the neighbour radius there).
__device__ __forceinline__ void short_list(const ProteinView& P, const float xf[3], int& s, int& e) {
    const float u0 = __fmul_rn(__fsub_rn(xf[0], P.fo0), P.inv_fine);
    const float u1 = __fmul_rn(__fsub_rn(xf[1], P.fo1), P.inv_fine);
    const float u2 = __fmul_rn(__fsub_rn(xf[2], P.fo2), P.inv_fine);
    s = e = 0;
    if (!(u0 >= 0.f && u1 >= 0.f && u2 >= 0.f && u0 < (float)P.nf0 && u1 < (float)P.nf1 && u2 < (float)P.nf2))
        return;
    const int c = ((int)u2 * P.nf1 + (int)u1) * P.nf0 + (int)u0;
    s = P.nb_start[c];
    e = P.nb_start[c + 1];
}

// FP32 screen of one candidate: squared distance and its band bits
// (1: within the vdW band, 2: within the cutoff band, 4: surely closer than sigma).
__device__ __forceinline__ int short_screen(const ProteinView& P, const float xf[3], float4 a) {
    float e0 = __fsub_rn(xf[0], a.x), e1 = __fsub_rn(xf[1], a.y), e2 = __fsub_rn(xf[2], a.z);
    float d2 = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
    return (d2 < P.sig2_hi ? 1 : 0) | (d2 < P.rc2_hi ? 2 : 0) | (d2 < P.sig2_lo ? 4 : 0);
}

// Decision and term of a screened pair in float-pair arithmetic (about 2^-47
// relative): f = x - x_m, d2 = |f|^2; bit 1 = clash, bit 2 = inside the cutoff with
// w = z_m, the radial function value fv = f(d2) and (gradients) fgr = 2 w f'(d2),
// so the pair adds w fv to phi and fgr f to grad phi.
template <bool GRAD>
__device__ __forceinline__ int short_pair(const ProteinView& P, const F2 x[3], const AtomRef& ref, int k,
                                          int bits, F2 f[3], F2& w, F2& fv, F2& fgr) {
    const float4 ah = P.atoms[k], al = P.atoms_lo[k];
    f[0] = dev::df_sub(x[0], F2{ah.x, al.x});
    f[1] = dev::df_sub(x[1], F2{ah.y, al.y});
    f[2] = dev::df_sub(x[2], F2{ah.z, al.z});
    F2 d2{0.f, 0.f};
    dev::df_fma_acc(d2, f[0], f[0]);
    dev::df_fma_acc(d2, f[1], f[1]);
    dev::df_fma_acc(d2, f[2], f[2]);
    d2 = dev::df_norm(d2);
    w = F2{ah.w, al.w};
    int out = 0;
    if (bits & 1) {
        if (bits & 4) {
            out = 1;
        } else {
            // inside the +-1e-4 sigma^2 band: the decision is taken in FP64 from the
            // FP64 position and atom record
            double x64[3];
            ref.pos64(x64);
            const double4 a64 = P.atoms64[k];
            const double e0 = __dsub_rn(x64[0], a64.x), e1 = __dsub_rn(x64[1], a64.y),
                         e2 = __dsub_rn(x64[2], a64.z);
            const double d2d = fma(e2, e2, fma(e1, e1, __dmul_rn(e0, e0)));
            out = d2d < P.sig2 ? 1 : 0;
        }
    }
    if ((bits & 2) && dev::df_lt(d2, F2{P.rc2_ph, P.rc2_pl})) {
        out |= 2;
        // local variable of the interval: u = d2/hs - j in [0, 1]
        const F2 xs = dev::df_mul(d2, F2{P.stab_ih_h, P.stab_ih_l});
        float jf = floorf(xs.h);
        if (jf == xs.h && xs.l < 0.f) jf = __fsub_rn(jf, 1.f);
        const int j = max(0, min((int)jf, P.stab_n - 2));
        const F2 u = dev::df_norm(F2{__fsub_rn(xs.h, (float)j), xs.l});
        const float4 c01 = P.stab2[2 * j], c23 = P.stab2[2 * j + 1];
        const F2 c0{c01.x, c01.y}, c1{c01.z, c01.w}, c2{c23.x, c23.y}, c3{c23.z, c23.w};
        // Horner: fv = ((c3 u + c2) u + c1) u + c0
        F2 v = dev::df_add(dev::df_mul(c3, u), c2);
        v = dev::df_add(dev::df_mul(v, u), c1);
        fv = dev::df_add(dev::df_mul(v, u), c0);
        if constexpr (GRAD) {
            // dp/du = (3 c3 u + 2 c2) u + c1 = hs f'(d2); grad_x f(|x - x_m|^2) = 2 f' (x - x_m)
            F2 dv = dev::df_add(dev::df_mul(dev::df_mul(c3, F2{3.f, 0.f}), u), dev::df_mul(c2, F2{2.f, 0.f}));
            dv = dev::df_add(dev::df_mul(dv, u), c1);
            fgr = dev::df_mul(dev::df_mul(w, dv), F2{2.f * P.stab_ih_h, 2.f * P.stab_ih_l});
        }
    }
    return out;
}

// The term of one pair inside the cutoff: e = w fv (the potential) and, for
// gradients, ge = fgr f (its gradient), each a pair product (~2^-47).
template <bool GRAD>
struct PairTerm {
    F2 e;
    F2 ge[GRAD ? 3 : 1];
};
template <bool GRAD>
__device__ __forceinline__ PairTerm<GRAD> short_term(F2 w, F2 fv, F2 fgr, const F2 f[3]) {
    PairTerm<GRAD> t;
    t.e = dev::df_mul(w, fv);
    if constexpr (GRAD)
        for (int a = 0; a < 3; ++a) t.ge[a] = dev::df_mul(fgr, f[a]);
    return t;
}

// Accumulation of one pair's term into an atom's sums (pair sums), in candidate order.
template <bool GRAD>
__device__ __forceinline__ void short_accumulate(const PairTerm<GRAD>& t, F2& phi, F2 g[3]) {
    dev::df_acc(phi, t.e);
    if constexpr (GRAD)
        for (int a = 0; a < 3; ++a) dev::df_acc(g[a], t.ge[a]);
}

// Short-range part and vdW decision for one atom; candidates split over
// `nl` cooperating lanes starting at `lane`.  Distances are screened in FP32;
// pairs inside the cutoff, and vdW decisions within 1e-4 relative of sigma^2,
// are taken in pair arithmetic from the pair position x.  phi and g are added to
// (callers pass zeros) in candidate order; with nl = 1 the sums equal those of
// short_coop for the same atom bit for bit.
template <bool GRAD>
__device__ __noinline__ void short_vdw(const ProteinView& P, const F2 x[3], const AtomRef ref, int lane,
                                       int nl, F2& phi, F2 g[3], int& clash) {
    const float xf[3] = {x[0].h, x[1].h, x[2].h};
    int s, e;
    short_list(P, xf, s, e);
    for (int j = s + lane; j < e; j += nl) {
        const int bits = short_screen(P, xf, P.nb_atoms[j]);
        if (!(bits & 3)) continue;
        F2 f[3], w, fv{0.f, 0.f}, fgr{0.f, 0.f};
        const int out = short_pair<GRAD>(P, x, ref, P.nb_idx[j], bits, f, w, fv, fgr);
        if (out & 1) clash = 1;
        if (out & 2) short_accumulate<GRAD>(short_term<GRAD>(w, fv, fgr, f), phi, g);
    }
}

// Per-warp queue of screened near pairs (short_coop): up to kNearCap pairs in the
// order of the warp's candidate list, with their terms once evaluated.
constexpr int kNearCap = 96;
template <bool GRAD>
struct NearQueue {
    int owner[kNearCap];   // lane whose atom the pair belongs to
    int k[kNearCap];       // protein atom (cell-sorted index)
    int bits[kNearCap];    // screen bits, then the pair's outcome bits
    float2 term[GRAD ? 4 : 1][kNearCap];  // the pair's term: e, then (gradients) ge[0..2]
    float2 x[3][32]; // pair positions of the warp's atoms
    float2 acc[GRAD ? 4 : 1][GRAD ? 32 : 1];  // (gradients) the atoms' sums during a flush
    int clash[GRAD ? 32 : 1];
    const PoseSetup* rq[32];  // where the atoms' FP64 positions come from (decisions
    const double* ry64[32];   // inside the sigma band)
    int ls[32];         // first entry of each lane's candidate list
    int lstart[32];     // prefix of the lanes' list lengths over the warp
    int seg0[32], seg1[32];  // per owner lane: its entries [seg0, seg1) of the queue
};

// Short range and vdW decision for the 32 atoms of a warp (one per lane).  The
// candidate lists of all 32 atoms form one list (lane by lane, each lane's in its own
// candidate order) that the lanes screen in FP32 32 at a time; the near pairs queue
// up in list order and are evaluated in pair arithmetic one pair per lane, 32 at a
// time, so atoms with very different numbers of candidates or near pairs still keep
// every lane busy.  When the queue is full (and at the end) each lane adds the terms
// of its own atom's pairs, which sit contiguously in the queue, in list order: one
// pass over the longest run instead of one per 32 pairs.  Every lane of the warp
// must call it; lanes with active = false contribute no atom.  prot_of(l) is the
// protein of lane l's atom (lanes may belong to different proteins).  Each atom's
// sums are accumulated in its own candidate order, so they equal short_vdw's (nl = 1)
// bit for bit.
// Candidates screened and near pairs evaluated by a warp (warp-uniform counts).
struct ShortCounts {
    long long cand = 0, near = 0;
};

template <bool GRAD, class ProtOf>
__device__ void short_coop_with(ProtOf prot_of, bool active, const F2 x[3], const AtomRef& ref,
                                NearQueue<GRAD>& Q, F2& phi, F2 g[3], int& clash, ShortCounts* cnt = nullptr) {
    const int lane = threadIdx.x & 31;
    const ProteinView& P = prot_of(lane);
    const unsigned full = 0xffffffffu;
    int total = 0;
    int ls = 0;
    if (active) {
        float xf[3];
        for (int a = 0; a < 3; ++a) {
            xf[a] = x[a].h;
            Q.x[a][lane] = make_float2(x[a].h, x[a].l);
        }
        Q.rq[lane] = ref.q;
        Q.ry64[lane] = ref.y64;
        int le;
        short_list(P, xf, ls, le);
        total = le - ls;
    }
    Q.ls[lane] = ls;
    // warp prefix of the totals: lane l's candidates are list entries [lstart, lstart + total)
    int incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
    }
    Q.lstart[lane] = incl - total;
    const int grand = __shfl_sync(full, incl, 31);
    if (cnt) cnt->cand += grand;
    __syncwarp();
    int qn = 0;     // entries in the queue (the same in every lane)
    int pdone = 0;  // entries whose terms are evaluated
    // terms of entries [pdone, pdone + m), one per lane
    auto process = [&](int m) {
        if (lane < m) {
            const int e = pdone + lane;
            const int o = Q.owner[e];
            const F2 xo[3] = {F2{Q.x[0][o].x, Q.x[0][o].y}, F2{Q.x[1][o].x, Q.x[1][o].y},
                              F2{Q.x[2][o].x, Q.x[2][o].y}};
            const AtomRef ro{Q.rq[o], Q.ry64[o]};
            F2 f[3], w, fv{0.f, 0.f}, fgr{0.f, 0.f};
            const int out = short_pair<GRAD>(prot_of(o), xo, ro, Q.k[e], Q.bits[e], f, w, fv, fgr);
            Q.bits[e] = out;
            if (out & 2) {
                const PairTerm<GRAD> t = short_term<GRAD>(w, fv, fgr, f);
                Q.term[0][e] = make_float2(t.e.h, t.e.l);
                if constexpr (GRAD)
                    for (int a = 0; a < 3; ++a) Q.term[1 + a][e] = make_float2(t.ge[a].h, t.ge[a].l);
            }
        }
        pdone += m;
    };
    // every queued pair's term into its owner's sums (in queue order), then empty the queue
    auto flush = [&]() {
        if (pdone < qn) process(qn - pdone);
        Q.seg0[lane] = 0;
        Q.seg1[lane] = 0;
        __syncwarp();
        for (int e = lane; e < qn; e += 32) {
            const int o = Q.owner[e];
            if (e == 0 || Q.owner[e - 1] != o) Q.seg0[o] = e;
            if (e == qn - 1 || Q.owner[e + 1] != o) Q.seg1[o] = e + 1;
        }
        __syncwarp();
        if constexpr (!GRAD) {
            if (active)
                for (int e = Q.seg0[lane], e1 = Q.seg1[lane]; e < e1; ++e) {
                    const int out = Q.bits[e];
                    if (out & 1) clash = 1;
                    if (out & 2) dev::df_acc(phi, F2{Q.term[0][e].x, Q.term[0][e].y});
                }
        } else {
            // four sums per atom (phi, g): one lane per (atom, sum), eight atoms at a time,
            // each sum still taken over the atom's pairs in queue order
            Q.acc[0][lane] = make_float2(phi.h, phi.l);
            for (int a = 0; a < 3; ++a) Q.acc[1 + a][lane] = make_float2(g[a].h, g[a].l);
            Q.clash[lane] = 0;
            __syncwarp();
            const int c = lane & 3;
            for (int pass = 0; pass < 4; ++pass) {
                const int o = pass * 8 + (lane >> 2);
                F2 sum{Q.acc[c][o].x, Q.acc[c][o].y};
                int cl = 0;
                for (int e = Q.seg0[o], e1 = Q.seg1[o]; e < e1; ++e) {
                    const int out = Q.bits[e];
                    cl |= out & 1;
                    if (out & 2) dev::df_acc(sum, F2{Q.term[c][e].x, Q.term[c][e].y});
                }
                Q.acc[c][o] = make_float2(sum.h, sum.l);
                if (c == 0 && cl) Q.clash[o] = 1;
            }
            __syncwarp();
            phi = F2{Q.acc[0][lane].x, Q.acc[0][lane].y};
            for (int a = 0; a < 3; ++a) g[a] = F2{Q.acc[1 + a][lane].x, Q.acc[1 + a][lane].y};
            if (active && Q.clash[lane]) clash = 1;
        }
        __syncwarp();
        qn = 0;
        pdone = 0;
    };
    for (int base = 0; base < grand; base += 32) {
        if (qn > kNearCap - 32) flush();  // room for a whole screened batch
        const int e = base + lane;
        int bits = 0, k = 0, o = 0;
        if (e < grand) {
            // owner: the last lane whose list starts at or before e
            int lo = 0, hi = 31;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (Q.lstart[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            o = lo;
            const int j = Q.ls[o] + (e - Q.lstart[o]);
            const float xo[3] = {Q.x[0][o].x, Q.x[1][o].x, Q.x[2][o].x};
            const ProteinView& Po = prot_of(o);
            bits = short_screen(Po, xo, Po.nb_atoms[j]);
            if (bits & 3) k = Po.nb_idx[j];
        }
        const bool near = (bits & 3) != 0;
        const unsigned m = __ballot_sync(full, near);
        if (near) {
            const int slot = qn + __popc(m & ((1u << lane) - 1u));
            Q.owner[slot] = o;
            Q.k[slot] = k;
            Q.bits[slot] = bits;
        }
        qn += __popc(m);
        if (cnt) cnt->near += __popc(m);
        __syncwarp();
        if (qn - pdone >= 32) {
            process(32);
            __syncwarp();
        }
    }
    if (qn > 0) flush();
}

// The same for a warp whose atoms all belong to protein P.
template <bool GRAD>
__device__ __forceinline__ void short_coop(const ProteinView& P, bool active, const F2 x[3], const AtomRef& ref,
                                           NearQueue<GRAD>& Q, F2& phi, F2 g[3], int& clash,
                                           ShortCounts* cnt = nullptr) {
    short_coop_with<GRAD>([&](int) -> const ProteinView& { return P; }, active, x, ref, Q, phi, g, clash, cnt);
}

// Atom position x = R y + t in float-pair arithmetic (Dot2 of the pair rows of R
// with the pair coordinates; FP32 rotation alone misplaces atoms by ~1e-6 A).
__device__ __forceinline__ void atom_position(const PoseSetup& q, const float2* __restrict__ yd, F2 x[3]) {
    const F2 y[3] = {F2{yd[0].x, yd[0].y}, F2{yd[1].x, yd[1].y}, F2{yd[2].x, yd[2].y}};
    for (int r = 0; r < 3; ++r) {
        F2 acc = q.td[r];
        dev::df_fma_acc(acc, q.Rd[3 * r], y[0]);
        dev::df_fma_acc(acc, q.Rd[3 * r + 1], y[1]);
        dev::df_fma_acc(acc, q.Rd[3 * r + 2], y[2]);
        x[r] = dev::df_norm(acc);
    }
}

// Geometry of ligand atom j in pose q: rotated offset R y in FP32 (torque arm of
// the gradient), pair position, and per axis the interpolation cell, fraction and
// whether the coordinate lies inside [-b, b].
__device__ __forceinline__ void atom_geometry(const ProteinView& P, const LigandView& lig,
                                              const PoseSetup& q, int j, float ry[3],
                                              F2 x[3], int ci[3], float cf[3], bool ins[3]) {
    float4 yq = lig.y[j];
    for (int r = 0; r < 3; ++r)
        ry[r] = __fmaf_rn(q.Rf[3 * r + 2], yq.z, __fmaf_rn(q.Rf[3 * r + 1], yq.y, __fmul_rn(q.Rf[3 * r], yq.x)));
    atom_position(q, lig.yd + 3 * j, x);
    for (int a = 0; a < 3; ++a)
        dev::axis_cell(x[a], F2{P.b_h, P.b_l}, F2{P.inv_h_h, P.inv_h_l}, P.n, ci[a], cf[a], ins[a]);
}

// Per-atom contributions to the pose sums (float pairs) from the long-range value
// (pair sums phi, g1..g3 of the W-form loop) and the short-range sums: q_j phi_j
// and, for gradients, q_j grad phi_j and the torque arm (R y_j) x q_j grad phi_j.
template <bool GRAD>
__device__ __forceinline__ void atom_contrib(const ProteinView& P, dev::F2 phi, dev::F2 g1, dev::F2 g2,
                                             dev::F2 g3, dev::F2 phs, const dev::F2 gs[3], double qd,
                                             const float ry[3], float2* cj) {
    // float-pair arithmetic throughout (~2^-47): GB300 runs FP64 at 1/64 of its FP32
    // rate, and these few operations per atom were a large share of the FP64 pipe
    const F2 qj = dev::df_from(qd);
    const F2 e = dev::df_mul(qj, dev::df_add(phi, phs));
    cj[0] = make_float2(e.h, e.l);
    if constexpr (GRAD) {
        const F2 ih{P.inv_h_h, P.inv_h_l};
        const F2 g[3] = {g1, g2, g3};
        F2 gq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gq[a] = dev::df_mul(qj, dev::df_add(dev::df_mul(g[a], ih), gs[a]));
            cj[1 + a] = make_float2(gq[a].h, gq[a].l);
        }
        const F2 r0{ry[0], 0.f}, r1{ry[1], 0.f}, r2{ry[2], 0.f};
        const F2 t0 = dev::df_sub(dev::df_mul(r1, gq[2]), dev::df_mul(r2, gq[1]));
        const F2 t1 = dev::df_sub(dev::df_mul(r2, gq[0]), dev::df_mul(r0, gq[2]));
        const F2 t2 = dev::df_sub(dev::df_mul(r0, gq[1]), dev::df_mul(r1, gq[0]));
        cj[4] = make_float2(t0.h, t0.l);
        cj[5] = make_float2(t1.h, t1.l);
        cj[6] = make_float2(t2.h, t2.l);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Butterfly sum of float pairs over a warp (every lane ends with the same pair:
// the pair sum is commutative).
__device__ __forceinline__ F2 warp_sum_pair(F2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = dev::df_add(v, F2{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
    return v;
}

// Sum over the atoms of one pose of its per-atom contributions [L][CS] (NC float
// pairs per atom, CS >= NC apart), by one warp: lane-strided pair sums, then a
// butterfly; every lane ends with s (FP64).
template <int NC, int CS = NC>
__device__ __forceinline__ void pose_sums(const float2* __restrict__ cpose, int L, int lane, double s[NC]) {
    F2 acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = F2{0.f, 0.f};
    for (int j = lane; j < L; j += 32) {
        const float2* cj = cpose + (size_t)j * CS;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = dev::df_add(acc[c], F2{cj[c].x, cj[c].y});
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = dev::df_to(warp_sum_pair(acc[c]));
}

// Outputs of one pose from its sums: E, flags and, for gradients, dE/dt and
// dE/dw = J_l(w)^T tau.
template <int NC>
__device__ __forceinline__ void write_pose(const PoseSetup& q, const double s[NC], int pflag, long long p,
                                           double* __restrict__ E, uint8_t* __restrict__ flags,
                                           double* __restrict__ gt, double* __restrict__ gw) {
    E[p] = s[0];
    if (flags) flags[p] = (uint8_t)pflag;
    if constexpr (NC == 7) {
        for (int a = 0; a < 3; ++a) gt[3 * p + a] = s[1 + a];
        for (int a = 0; a < 3; ++a)
            gw[3 * p + a] = fma(q.J[6 + a], s[6], fma(q.J[3 + a], s[5], __dmul_rn(q.J[a], s[4])));
    }
}

// Reduction of per-atom contributions to per-pose outputs (one warp per pose).
template <int NC>
__device__ void reduce_poses(const ProteinView& P, int PB, int L, long long p0, long long Ptot,
                             const PoseSetup* ps, const float2* contrib, const int* pflag,
                             double* __restrict__ E, uint8_t* __restrict__ flags,
                             double* __restrict__ gt, double* __restrict__ gw) {
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    for (int pl = warp; pl < PB; pl += nw) {
        long long p = p0 + pl;
        if (p >= Ptot) break;
        if (!ps[pl].valid) continue;  // skipped pose: outputs untouched
        double s[NC];
        pose_sums<NC>(contrib + (size_t)pl * L * NC, L, lane, s);
        if (lane == 0) write_pose<NC>(ps[pl], s, pflag[pl], p, E, flags, gt, gw);
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
    float2* contrib = (float2*)(ps + PB);
    int* pflag = (int*)(contrib + (size_t)PB * lig.L * NC);
    NearQueue<GRAD>* queues = (NearQueue<GRAD>*)((((uintptr_t)(pflag + PB)) + 15) / 16 * 16);
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
    // every lane of a warp runs the same number of iterations (short_coop needs all 32)
    for (int base = 0; base < PB * L; base += NT) {
        const int g = base + tid;
        const bool in_range = g < PB * L;
        const int pl = in_range ? g / L : 0, j = in_range ? g - pl * L : 0;
        float2* cj = contrib + (size_t)g * NC;
        const bool valid = in_range && ps[pl].valid;
        if (in_range && !valid) {
#pragma unroll
            for (int c = 0; c < NC; ++c) cj[c] = make_float2(0.f, 0.f);
        }
        float ry[3] = {0.f, 0.f, 0.f};
        int ci[3] = {0, 0, 0};
        float cf[3] = {0.f, 0.f, 0.f};
        bool ins[3] = {true, true, true};
        F2 x[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (valid) atom_geometry(P, lig, ps[pl], j, ry, x, ci, cf, ins);
        // short range and vdW of the warp's atoms
        F2 phs{0.f, 0.f}, gs[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int clash = 0;
        short_coop<GRAD>(P, valid, x, AtomRef{&ps[pl], lig.y64 + 3 * j}, queues[tid >> 5], phs, gs, clash);
        if (!valid) continue;
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
        int fl = clash ? RS_FLAG_CLASH : 0;
        if (!(ins[0] && ins[1] && ins[2])) fl |= RS_FLAG_OUT_OF_GRID;
        if (fl) atomicOr(&pflag[pl], fl);
        atom_contrib<GRAD>(P, phi, g1, g2, g3, phs, gs, lig.q64[j], ry, cj);
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
    s = (s + 15) / 16 * 16 + (size_t)(NT / 32) * sizeof(NearQueue<GRAD>);
    return (s + 15) / 16 * 16;
}

// FP32 pipe operations (FADD, FMUL and FFMA each count 1) per atom of the W-form
// evaluation: per (a, b) one pair lerp (14) and one (energy) or three (gradient)
// Dot2 steps (13 each); per a one or four Dot2 steps; one pair lerp per column of
// v1 and v2; pose transform, cell index and reduction ~60 (energy) / ~80 (gradient).
// The counts match the FP32 instruction counters of the kernels within 1%.
inline double wform_ops_per_atom(int RP, bool grad) {
    double r = RP;
    return grad ? 53.0 * r * r + 80.0 * r + 80.0 : 27.0 * r * r + 41.0 * r + 60.0;
}

}  // namespace
}  // namespace rs
