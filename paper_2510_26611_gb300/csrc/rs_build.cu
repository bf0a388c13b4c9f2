// Algorithm TEP (Sec. 3.4): the RS potential of a protein on the device.
//
//   cell list  : protein atoms binned into cubes of side >= max(r_c, sigma)
//   canonical  : U^(l)[i, (m,k)] = exp(-t_k^2 (x_i - x_m^l)^2), axis 3 times
//                xi_(m,k) = z_m a_k  (Eq. Long-Range_Sum, TEP step 3)
//   Tucker     : RHOSVD of the same tensor (TEP step 4):
//                 1. Gram G = Z Z^T of Z = U diag(|xi|^(1/3)) by the Gaussian
//                    product identity (exact, O(n N R_l) instead of O(n^2 N R_l))
//                 2. block subspace iteration on G (pair GEMM, FP64 CholQR2) and
//                    Rayleigh-Ritz (p x p eigenproblems on the host, FP64)
//                 3. interpolative ("skeleton") rows S of V: V' = V V[S,:]^{-1};
//                    the Tucker tensor is rewritten exactly in this basis
//                 4. C' = (V V[S,:]^T)^T U and core beta' = sum_r xi_r C'1 o C'2 o C'3
// The Gram, the subspace iteration and the skeleton are FP64; the projections and
// the core run in float-pair arithmetic on the FP32 pipes (about 2^-47 relative per
// operation); factors are stored as float pairs for evaluation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_tc_gemm.cuh"

namespace rs {
namespace {

constexpr int kBlock = 256;

// Temporary device buffers of one build.  They are carved from the context's
// workspace (a grow-only device buffer); what does not fit is allocated and freed
// at the end, and the workspace is grown to the high-water mark for the next build.
struct Scratch {
    rs_ctx* ctx = nullptr;
    size_t used = 0;
    std::vector<void*> extra;
    explicit Scratch(rs_ctx* c) : ctx(c) {}
    ~Scratch() {
        for (void* p : extra) cudaFree(p);
        if (ctx && used > ctx->ws_bytes) {
            if (ctx->ws_buf) cudaFree(ctx->ws_buf);
            ctx->ws_buf = nullptr;
            ctx->ws_bytes = 0;
            if (cudaMalloc(&ctx->ws_buf, used) == cudaSuccess) ctx->ws_bytes = used;
            else cudaGetLastError();
        }
    }
    template <class T>
    rs_status get(T** p, size_t count) {
        size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
        if (bytes == 0) bytes = 256;
        size_t off = used;
        used += bytes;
        if (ctx && ctx->ws_buf && used <= ctx->ws_bytes) {
            *p = (T*)((char*)ctx->ws_buf + off);
            return RS_OK;
        }
        void* v = nullptr;
        if (cudaMalloc(&v, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("build scratch: cudaMalloc of %zu bytes failed", bytes);
            return RS_ERR_OOM;
        }
        extra.push_back(v);
        *p = (T*)v;
        return RS_OK;
    }
};

// Several arrays of one protein in one device allocation (256-byte aligned parts):
// add() records a pointer and its element count, alloc() makes the allocation (owned
// by the protein) and sets the pointers.
struct DeviceArena {
    std::vector<std::pair<void**, size_t>> parts;  // (pointer, bytes)
    template <class T>
    void add(T** p, size_t count) {
        parts.emplace_back(reinterpret_cast<void**>(p), (count * sizeof(T) + 255) / 256 * 256);
    }
    rs_status alloc(rs_protein* P) {
        size_t total = 0;
        for (auto& pr : parts) total += pr.second;
        void* base = nullptr;
        RS_TRY(device_alloc(P, &base, total));
        char* c = static_cast<char*>(base);
        for (auto& pr : parts) {
            *pr.first = c;
            c += pr.second;
        }
        return RS_OK;
    }
};

}  // namespace
bool symeig_host(int n, const double* A, double* lam, double* W);
void gs_qr_host(int n, int k, double* A, double* R);
namespace {

inline unsigned blocks_for(size_t n, int bs = kBlock) { return (unsigned)((n + bs - 1) / bs); }

// Float pair (hi, lo) of a double on the host: hi the nearest float, lo the nearest
// float to the remainder.
inline void split_host(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// ------------------------------------------------------------------ cell list
__global__ void k_cell_count(int N, const double* __restrict__ xyz, double co0, double co1,
                             double co2, double inv_cell, int nc0, int nc1, int nc2,
                             int* __restrict__ cell_of, int* __restrict__ count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c0 = (int)floor((xyz[3 * (size_t)i + 0] - co0) * inv_cell);
    int c1 = (int)floor((xyz[3 * (size_t)i + 1] - co1) * inv_cell);
    int c2 = (int)floor((xyz[3 * (size_t)i + 2] - co2) * inv_cell);
    c0 = min(max(c0, 0), nc0 - 1);
    c1 = min(max(c1, 0), nc1 - 1);
    c2 = min(max(c2, 0), nc2 - 1);
    int id = (c2 * nc1 + c1) * nc0 + c0;
    cell_of[i] = id;
    atomicAdd(&count[id], 1);
}

// Exclusive prefix sum of n ints into out[0..n] (one CTA; the cell grids are small).
__global__ void k_scan(int n, const int* __restrict__ in, int* __restrict__ out) {
    __shared__ int sm[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < n ? in[i] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int t = threadIdx.x >= off ? sm[threadIdx.x - off] : 0;
            __syncthreads();
            sm[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) out[i + 1] = carry + sm[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += sm[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0;
}

__global__ void k_cell_fill(int N, const int* __restrict__ cell_of, const int* __restrict__ start,
                            int* __restrict__ cursor, int* __restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c = cell_of[i];
    int slot = start[c] + atomicAdd(&cursor[c], 1);
    perm[slot] = i;
}

// Sorts each cell's atoms by original index (so the layout does not depend on
// atomic ordering) and writes the atom records as float pairs: atoms holds the
// floats nearest (x, y, z, q), atoms_lo the remainders; atoms64 the FP64 record.
__global__ void k_cell_sort(int ncell, const int* __restrict__ start, int* __restrict__ perm,
                            const double* __restrict__ xyz, const double* __restrict__ q,
                            float4* __restrict__ atoms, float4* __restrict__ atoms_lo,
                            double4* __restrict__ atoms64) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int s = start[c], e = start[c + 1];
    for (int a = s + 1; a < e; ++a) {
        int v = perm[a];
        int b = a - 1;
        while (b >= s && perm[b] > v) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = v;
    }
    for (int a = s; a < e; ++a) {
        int i = perm[a];
        const dev::F2 x = dev::df_from(xyz[3 * (size_t)i]), y = dev::df_from(xyz[3 * (size_t)i + 1]),
                      z = dev::df_from(xyz[3 * (size_t)i + 2]), w = dev::df_from(q[i]);
        atoms[a] = make_float4(x.h, y.h, z.h, w.h);
        atoms_lo[a] = make_float4(x.l, y.l, z.l, w.l);
        atoms64[a] = make_double4(xyz[3 * (size_t)i], xyz[3 * (size_t)i + 1], xyz[3 * (size_t)i + 2], q[i]);
    }
}

// The FP64 atom records (x, y, z, q) of a built protein back to flat coordinates
// [N][3] and charges [N] (the inputs of the cell build), for the union of molecules.
__global__ void k_split_atoms64(int N, const double4* __restrict__ atoms64, double* __restrict__ xyz,
                                double* __restrict__ q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double4 r = atoms64[i];
    xyz[3 * (size_t)i] = r.x;
    xyz[3 * (size_t)i + 1] = r.y;
    xyz[3 * (size_t)i + 2] = r.z;
    q[i] = r.w;
}

// Short-range candidate lists.  Fine cell c (box [lo, lo + f] per axis) lists every
// atom whose distance to the box is at most R, visiting the coarse cells (side >= R)
// that can hold such atoms in increasing id order, so each list is in cell-sorted
// atom order.  One warp per fine cell: the lanes test a coarse row's atoms 32 at a
// time (FP32 distance against R + 1e-3 A, a superset of the FP64 test) and a ballot
// keeps their order.  pass 0 counts, pass 1 writes at start[c].
__global__ void k_nb_lists(int pass, int nf0, int nf1, int nf2, double fo0, double fo1, double fo2, double f,
                           int nc0, int nc1, int nc2, double co0, double co1, double co2, double cell, double R,
                           const int* __restrict__ cell_start, const float4* __restrict__ atoms,
                           int* __restrict__ count, const int* __restrict__ start, float4* __restrict__ nb_atoms,
                           int* __restrict__ nb_idx) {
    const long long id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (id >= (long long)nf0 * nf1 * nf2) return;  // warp-uniform
    const int cx = (int)(id % nf0), cy = (int)((id / nf0) % nf1), cz = (int)(id / ((long long)nf0 * nf1));
    const double lo[3] = {fo0 + cx * f, fo1 + cy * f, fo2 + cz * f};
    const double co[3] = {co0, co1, co2};
    const int nc[3] = {nc0, nc1, nc2};
    int c_lo[3], c_hi[3];
    for (int a = 0; a < 3; ++a) {
        c_lo[a] = max(0, (int)floor((lo[a] - R - co[a]) / cell));
        c_hi[a] = min(nc[a] - 1, (int)floor((lo[a] + f + R - co[a]) / cell));
    }
    const float blo[3] = {(float)lo[0], (float)lo[1], (float)lo[2]};
    const float bhi[3] = {(float)(lo[0] + f), (float)(lo[1] + f), (float)(lo[2] + f)};
    const float Rf = (float)(R + 1e-3);
    const float R2 = Rf * Rf;
    int n = 0;
    const int out = pass ? start[id] : 0;
    for (int z = c_lo[2]; z <= c_hi[2]; ++z)
        for (int y = c_lo[1]; y <= c_hi[1]; ++y) {
            if (c_lo[0] > c_hi[0]) continue;
            const int row = (z * nc1 + y) * nc0;
            const int s = cell_start[row + c_lo[0]], e = cell_start[row + c_hi[0] + 1];
            for (int k0 = s; k0 < e; k0 += 32) {
                const int k = k0 + lane;
                bool in = false;
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < e) {
                    a = atoms[k];
                    const float p[3] = {a.x, a.y, a.z};
                    float d2 = 0.f;
                    for (int q = 0; q < 3; ++q) {
                        const float d = fmaxf(fmaxf(blo[q] - p[q], p[q] - bhi[q]), 0.f);
                        d2 = fmaf(d, d, d2);
                    }
                    in = d2 <= R2;
                }
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (pass && in) {
                    const int o = out + n + __popc(m & ((1u << lane) - 1u));
                    nb_atoms[o] = a;
                    nb_idx[o] = k;
                }
                n += __popc(m);
            }
        }
    if (!pass && lane == 0) count[id] = n;
}

// ---------------------------------------------------- unreduced canonical factors
// Collocation: the Gaussian's value at the node.  Galerkin (Sec. 2, Eq. galten, read as
// the average over the node's cell): (1/h) int_{x_i-h/2}^{x_i+h/2} exp(-t^2 (x - x_m)^2) dx
// = sqrt(pi) / (2 t h) (erf(t (d + h/2)) - erf(t (d - h/2))), d = x_i - x_m; 1 for t = 0.
__device__ __forceinline__ double factor_entry(double t, double d, double h, int galerkin) {
    if (!galerkin) return exp(-t * t * d * d);
    if (t == 0.0) return 1.0;
    const double th = t * h;
    if (th < 1e-3) {
        // the cell is narrow against the Gaussian: midpoint value times the average of
        // exp(-t^2 (2 d s + s^2)) over s in [-h/2, h/2], to second order in t h
        const double g = exp(-t * t * d * d);
        return g * (1.0 + th * th * (2.0 * t * t * d * d - 1.0) / 12.0);
    }
    // erf(B) - erf(A) without cancellation in the tails (erfc when the signs agree)
    const double A = t * (d - 0.5 * h), B = t * (d + 0.5 * h);
    const double diff = A >= 0.0 ? erfc(A) - erfc(B) : (B <= 0.0 ? erfc(-B) - erfc(-A) : erf(B) - erf(A));
    return 0.886226925452758014 / th * diff;
}

__global__ void k_canon_factors(int n, double b, double h, int N, int Rl,
                                const double* __restrict__ xyz, const double* __restrict__ q,
                                const double* __restrict__ tl, const double* __restrict__ al,
                                int ld, float* __restrict__ F0, float* __restrict__ F1,
                                float* __restrict__ F2, int galerkin) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (r >= ld) return;
    size_t o = (size_t)i * ld + r;
    if (r >= N * Rl) {
        F0[o] = 0.f;
        F1[o] = 0.f;
        F2[o] = 0.f;
        return;
    }
    int m = r / Rl, k = r - m * Rl;
    double xi = -b + i * h;
    const double t = tl[k];
    double d0 = xi - xyz[3 * (size_t)m], d1 = xi - xyz[3 * (size_t)m + 1], d2 = xi - xyz[3 * (size_t)m + 2];
    F0[o] = (float)factor_entry(t, d0, h, galerkin);
    F1[o] = (float)factor_entry(t, d1, h, galerkin);
    F2[o] = (float)(factor_entry(t, d2, h, galerkin) * q[m] * al[k]);
}

// ------------------------------------------------------------- pair exponential
// exp(x) for a float pair x, |x| <= 80, on the FP32 pipes, by the table-driven method
// of P. T. P. Tang ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15, 1989): x = (256 n + j) ln2/256 + r with
// |r| <= ln2/512, exp(x) = 2^n 2^(j/256) exp(r); ln2/256 is split into C1 (8
// significant bits, so m C1 is exact for |m| < 2^16), C2 and C3; the 256 table values
// 2^(j/256) are float pairs of FP64 values; exp(r) is its Taylor polynomial to degree 4
// (the omitted r^5/120 is below 2^-54).  Relative error ~2^-46.
__global__ void k_exp2_table(float2* __restrict__ tab) {
    const int j = threadIdx.x;
    const double v = exp2(j / 256.0);
    const dev::F2 p = dev::df_from(v);
    tab[j] = make_float2(p.h, p.l);
}

__device__ __forceinline__ dev::F2 df_exp(dev::F2 x, const float2* __restrict__ tab) {
    using dev::F2;
    const float m = rintf(__fmul_rn(x.h, 0x1.715476p+8f));  // x 256 / ln2
    F2 r = dev::df_add(x, F2{-__fmul_rn(m, 0x1.62p-9f), 0.f});  // m C1 exact
    const float p2 = __fmul_rn(m, 0x1.c85fep-18f);
    const float e2 = __fmaf_rn(m, 0x1.c85fep-18f, -p2);          // m C2 = p2 + e2 exactly
    r = dev::df_add(r, F2{-p2, -e2});
    r = dev::df_add(r, F2{__fmul_rn(m, 0x1.71844p-43f), 0.f});    // - m C3 (C3 < 0)
    const int mi = (int)m;
    const int j = mi & 255, n = mi >> 8;
    F2 t = dev::df_add(F2{0x1.555556p-3f, -0x1.555556p-28f}, dev::df_mul(r, F2{0x1.555556p-5f, -0x1.555556p-30f}));
    t = dev::df_add(F2{0.5f, 0.f}, dev::df_mul(r, t));
    t = dev::df_add(F2{1.f, 0.f}, dev::df_mul(r, t));
    t = dev::df_add(F2{1.f, 0.f}, dev::df_mul(r, t));
    const float2 tj = tab[j];
    const F2 v = dev::df_mul(F2{tj.x, tj.y}, t);
    const float sc = __int_as_float((n + 127) << 23);
    return F2{__fmul_rn(v.h, sc), __fmul_rn(v.l, sc)};
}

__global__ void k_diag_pair_exp(int n, const double* __restrict__ x, const float2* __restrict__ tab,
                                double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = dev::df_to(df_exp(dev::df_from(x[i]), tab));
}

// a / b for float pairs (one Newton correction of the FP32 quotient).
__device__ __forceinline__ dev::F2 df_div(dev::F2 a, dev::F2 b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const dev::F2 rem = dev::df_sub(a, dev::df_mul(b, dev::F2{q1, 0.f}));
    const float q2 = __fdiv_rn(rem.h, b.h);
    return dev::fast_two_sum(q1, q2);
}

// ------------------------------------------------------------- Gram by Gaussian products
// G[i,i'] = sum_(m,k) |xi|^(2/3) e^{-t^2 (x_i-x_m)^2} e^{-t^2 (x_i'-x_m)^2}
//         = sum_k |a_k|^(2/3) e^{-t^2 (x_i-x_i')^2 / 2} D_k(y_{i+i'}),
// D_k(y) = sum_m |z_m|^(2/3) e^{-2 t^2 (y - x_m)^2},  y_s = -b + s h/2 (half grid).
// One thread: SC half-grid points, one (axis, k), MC atoms.  Each Gaussian is
// walked forwards through the chunk from its first point within reach (e^-50 of the
// peak: the whole chunk for an atom to its left, the rising side for one to its right)
// with the exact ratio recurrence g_{s+1} = g_s rho_s, rho_{s+1} = rho_s c, all in float
// pairs on the FP32 pipes: the atom records are float pairs (k_dsum_atoms), the two
// seeds per (atom, chunk) are pair exponentials (df_exp), so the loop runs no FP64
// instruction (GB300's FP64 rate is 1/64 of FP32); about 2^-46 relative per seed and
// 2^-47 per step, at most 31 steps from a seed.  The walk starts at a value at least
// e^-50 of the peak and only grows towards it, so no seed underflows; values below
// that on the rising side are left out (the float-pair sums carry ~e^-32 of the peak).
constexpr int kSC = 32;
constexpr int kMC = 128;

// Atom records of the Gaussian sums: per axis (x_a as a pair, |z|^(2/3) as a pair).
__global__ void k_dsum_atoms(int N, const double* __restrict__ xyz, const double* __restrict__ cz,
                             float4* __restrict__ pk) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int ax = blockIdx.y;
    if (m >= N) return;
    const dev::F2 x = dev::df_from(xyz[3 * (size_t)m + ax]), c = dev::df_from(cz[m]);
    pk[(size_t)ax * N + m] = make_float4(x.h, x.l, c.h, c.l);
}

__global__ void __launch_bounds__(128) k_gauss_dsum(int n, double b, double h, int N, int Rl,
                                                     const float4* __restrict__ pk,
                                                     const double* __restrict__ tl,
                                                     const float2* __restrict__ etab, int nsc, int nmc,
                                                     double* __restrict__ Dp) {
    using dev::F2;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)nsc * Rl * 3 * nmc;
    if (idx >= total) return;
    int sc = (int)(idx % nsc);
    long long rest = idx / nsc;
    int k = (int)(rest % Rl);
    rest /= Rl;
    int ax = (int)(rest % 3);
    int mc = (int)(rest / 3);
    const int S = 2 * n - 1;
    const double delta = 0.5 * h;
    const int s0 = sc * kSC;
    const double t2 = 2.0 * tl[k] * tl[k];
    // per-thread constants (FP64 once, then pairs)
    const F2 y0 = dev::df_from(-b + s0 * delta), dl = dev::df_from(delta), t2p = dev::df_from(t2);
    const F2 t2d = dev::df_from(t2 * delta), cqp = dev::df_from(exp(-2.0 * t2 * delta * delta));
    const float inv_delta = (float)(1.0 / delta);
    // reach: the Gaussian is below e^-50 of its peak where |y - x_m| > R
    const float R = t2 > 0.0 ? (float)sqrt(50.0 / t2) : INFINITY;
    F2 acc[kSC];
#pragma unroll
    for (int s = 0; s < kSC; ++s) acc[s] = F2{0.f, 0.f};
    const float4* pa = pk + (size_t)ax * N;
    int m_end = min(N, (mc + 1) * kMC);
    for (int m = mc * kMC; m < m_end; ++m) {
        const float4 a = pa[m];
        // the chunk's points within reach of x_m, in units of delta from y0
        const float plo = __fmul_rn(__fsub_rn(__fsub_rn(a.x, R), y0.h), inv_delta);
        const float phi = __fmul_rn(__fsub_rn(__fadd_rn(a.x, R), y0.h), inv_delta);
        if (plo > (float)(kSC - 1) || phi < 0.f) continue;  // the whole chunk is out of reach
        const int ss = plo > 0.f ? (int)ceilf(plo) : 0;
        // dp = y0 + ss delta - x_m; g_ss = z e^{-t2 dp^2}; rho_ss = e^{-t2 delta (2 dp + delta)}
        const F2 dp = dev::df_sub(dev::df_add(y0, dev::df_mul(F2{(float)ss, 0.f}, dl)), F2{a.x, a.y});
        const F2 arg = dev::df_mul(t2p, dev::df_mul(dp, dp));
        const F2 a1 = dev::df_mul(t2d, dev::df_add(F2{2.f * dp.h, 2.f * dp.l}, dl));
        F2 r = df_exp(F2{-a1.h, -a1.l}, etab);
        F2 g = dev::df_mul(F2{a.z, a.w}, df_exp(F2{-arg.h, -arg.l}, etab));
#pragma unroll
        for (int s = 0; s < kSC; ++s) {
            if (s >= ss) {
                dev::df_acc(acc[s], g);
                g = dev::df_mul(g, r);
                r = dev::df_mul(r, cqp);
            }
        }
    }
    double* out = Dp + (((size_t)mc * 3 + ax) * Rl + k) * S;
#pragma unroll
    for (int s = 0; s < kSC; ++s)
        if (s0 + s < S) out[s0 + s] = dev::df_to(acc[s]);
}

// out[i] = sum over the chunks of in[c][i] (FP64, four interleaved partial sums in a
// fixed order: the dependent FP64 add chain is GB300's cost here); out2 (if not null)
// gets the sums as float pairs.
__global__ void k_sum_chunks(size_t len, int nchunk, const double* __restrict__ in,
                             double* __restrict__ out, float2* __restrict__ out2) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    int c = 0;
    for (; c + 4 <= nchunk; c += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] += in[(size_t)(c + u) * len + i];
    for (; c < nchunk; ++c) s[c & 3] += in[(size_t)c * len + i];
    const double v = (s[0] + s[1]) + (s[2] + s[3]);
    out[i] = v;
    if (out2) {
        const dev::F2 p = dev::df_from(v);
        out2[i] = make_float2(p.h, p.l);
    }
}

// WE[k][d] = |a_k|^{2/3} exp(-t_k^2 (d h)^2 / 2) as float pairs (the distance factor
// of the product identity with its weight).
__global__ void k_exp_table(int n, double h, int Rl, const double* __restrict__ tl,
                            const double* __restrict__ w2, float2* __restrict__ WE) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (d >= n) return;
    double x = d * h;
    const dev::F2 p = dev::df_from(w2[k] * exp(-0.5 * tl[k] * tl[k] * x * x));
    WE[(size_t)k * n + d] = make_float2(p.h, p.l);
}

// G[i, j] = sum_k WE[k][|i - j|] D[k][i + j] in float-pair arithmetic: every term is
// positive, so the pair sum keeps ~2^-47 of G (GB300's FP64 rate made the FP64
// version of this 3 n^2 R_l-term sum throughput-bound).
__global__ void k_gram(int n, int Rl, const float2* __restrict__ WE, const float2* __restrict__ D2,
                       float2* __restrict__ G) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    int ax = blockIdx.z;
    if (j >= n) return;
    const int S = 2 * n - 1;
    int d = abs(i - j);
    const float2* Dax = D2 + (size_t)ax * Rl * S;
    dev::F2 s{0.f, 0.f};
    for (int k = 0; k < Rl; ++k) {
        const float2 a = WE[(size_t)k * n + d], b = Dax[(size_t)k * S + i + j];
        dev::df_fma_acc(s, dev::F2{a.x, a.y}, dev::F2{b.x, b.y});
    }
    const dev::F2 g = dev::df_norm(s);
    G[((size_t)ax * n + i) * n + j] = make_float2(g.h, g.l);
}

__global__ void k_trace(int n, const float2* __restrict__ G, double* __restrict__ tr) {
    __shared__ double sm[kBlock];
    int ax = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 g = G[((size_t)ax * n + i) * n + i];
        s += dev::df_to(dev::F2{g.x, g.y});
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tr[ax] = sm[0];
}

// --------------------------------------------------------- subspace iteration (FP64)
// Deterministic start block: a hash of (axis, row, column) mapped to [-1, 1) on a grid
// of 2^-23, so each value is a float: Q (FP64) and Q2 (float pairs, the GEMM's operand)
// hold the same numbers.  The block is not orthonormalised: the first subspace step's
// CholQR of G Q spans the same columns either way.
__global__ void k_init_block(int n, int p, double* __restrict__ Q, float2* __restrict__ Q2) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)3 * n * p;
    if (idx >= total) return;
    unsigned long long x = idx * 0x9E3779B97F4A7C15ull + 0x1234567ull;
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    const double v = (double)(x >> 40) * (1.0 / 8388608.0) - 1.0;
    Q[idx] = v;
    Q2[idx] = make_float2((float)v, 0.f);
}

// Y[ax] = G[ax] Q[ax] (G n x n, Q n x p, p <= 48, both float pairs), split over K:
// CTA (row block of 64, K slice ks, axis) writes the partial product of its K slice
// to Yp[ks][ax] (FP64).  Thread tile 4 rows x 3 columns: twelve independent Dot2
// accumulators per thread; KS slices give enough CTAs to fill the GPU for n ~ 1000.
constexpr int kGemmKS = 8;
constexpr int kGemmRows = 64;
// Largest grid of the tensor-core G Q (its slices take 12 bytes per Gram entry).
constexpr int kTcGemmMaxN = 4097;

__global__ void __launch_bounds__(256) k_gemm_gq(int n, int p, const float2* __restrict__ G,
                                                  const float2* __restrict__ Q, double* __restrict__ Yp) {
    using dev::F2;
    __shared__ float2 Gs[kGemmRows][33];
    __shared__ float2 Qs[32][48];
    const int ax = blockIdx.z, ks = blockIdx.y;
    const int i0 = blockIdx.x * kGemmRows;
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    const int kchunk = ((n + kGemmKS - 1) / kGemmKS + 31) / 32 * 32;
    const int kbeg = ks * kchunk, kend = min(n, kbeg + kchunk);
    const float2* Ga = G + (size_t)ax * n * n;
    const float2* Qa = Q + (size_t)ax * n * p;
    F2 acc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 3; ++u) acc[a][u] = F2{0.f, 0.f};
    const float2 z = make_float2(0.f, 0.f);
    for (int k0 = kbeg; k0 < kend; k0 += 32) {
        for (int e = threadIdx.x; e < kGemmRows * 32; e += 256) {
            const int rr = e >> 5, kk = e & 31;
            const int gi = i0 + rr, gk = k0 + kk;
            Gs[rr][kk] = (gi < n && gk < kend) ? Ga[(size_t)gi * n + gk] : z;
        }
        for (int e = threadIdx.x; e < 32 * p; e += 256) {
            const int kk = e / p, c = e % p;
            const int gk = k0 + kk;
            Qs[kk][c] = gk < kend ? Qa[(size_t)gk * p + c] : z;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
            F2 g[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) g[a] = F2{Gs[4 * tr + a][kk].x, Gs[4 * tr + a][kk].y};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int c = tc + 16 * u;
                if (c < p) {
                    const F2 q{Qs[kk][c].x, Qs[kk][c].y};
#pragma unroll
                    for (int a = 0; a < 4; ++a) dev::df_fma_acc(acc[a][u], g[a], q);
                }
            }
        }
        __syncthreads();
    }
    double* out = Yp + ((size_t)ks * 3 + ax) * n * p;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int gi = i0 + 4 * tr + a;
        if (gi >= n) continue;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int c = tc + 16 * u;
            if (c < p) out[(size_t)gi * p + c] = dev::df_to(acc[a][u]);
        }
    }
}

// Y = sum over the nks K slices of Yp (FP64) or Yp2 (float pairs) in a fixed order, and
// with Sp != nullptr the partial
// Gram of each 16-row block, Sp[ax][blk] = Y_blk^T Y_blk (p x p, FP64), so CholQR
// needs no separate pass over Y.  CTA: 16 rows of one axis.
__global__ void __launch_bounds__(256) k_gemm_reduce(int n, int p, int nks, const double* __restrict__ Yp,
                                                      const float2* __restrict__ Yp2, double* __restrict__ Y,
                                                      double* __restrict__ Sp) {
    __shared__ double Ys[16][49];
    const int ax = blockIdx.y;
    const int i0 = blockIdx.x * 16;
    for (int e = threadIdx.x; e < 16 * p; e += 256) {
        const int r = e / p, c = e % p;
        const int gi = i0 + r;
        double v = 0.0;
        if (gi < n) {
            if (Yp2) {  // float-pair partials (tensor-core GEMM), summed in pair arithmetic
                dev::F2 acc{0.f, 0.f};
                for (int ks = 0; ks < nks; ++ks) {
                    const float2 t = Yp2[(((size_t)ks * 3 + ax) * n + gi) * p + c];
                    acc = dev::df_add(acc, dev::F2{t.x, t.y});
                }
                v = dev::df_to(acc);
            } else {
                for (int ks = 0; ks < nks; ++ks) v += Yp[(((size_t)ks * 3 + ax) * n + gi) * p + c];
            }
            Y[((size_t)ax * n + gi) * p + c] = v;
        }
        Ys[r][c] = v;
    }
    if (Sp == nullptr) return;
    __syncthreads();
    double* out = Sp + ((size_t)ax * gridDim.x + blockIdx.x) * p * p;
    for (int e = threadIdx.x; e < p * p; e += 256) {
        int a = e / p, c = e % p;
        double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) s[rr & 3] = fma(Ys[rr][a], Ys[rr][c], s[rr & 3]);
        out[e] = (s[0] + s[1]) + (s[2] + s[3]);
    }
}

// S[ax] = sum over blocks of Sp[ax][blk] in a fixed order.  CTA: 32 consecutive entries
// (one per lane, coalesced) of one axis; warp w adds blocks w, w + 8, ... (two
// interleaved partial sums, so a warp has several loads in flight), then the eight
// warps' sums are added in warp order.
constexpr int kSumGramWarps = 8;
__global__ void __launch_bounds__(32 * kSumGramWarps) k_sum_gram(int nblk, int p, const double* __restrict__ Sp,
                                                                 double* __restrict__ S) {
    __shared__ double part[kSumGramWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    const int ax = blockIdx.y;
    double s0 = 0.0, s1 = 0.0;
    if (e < p * p) {
        const double* src = Sp + (size_t)ax * nblk * p * p + e;
        const size_t stride = (size_t)kSumGramWarps * p * p;
        int b = w;
#pragma unroll 4
        for (; b + kSumGramWarps < nblk; b += 2 * kSumGramWarps) {
            s0 += src[(size_t)b * p * p];
            s1 += src[(size_t)b * p * p + stride];
        }
        if (b < nblk) s0 += src[(size_t)b * p * p];
    }
    part[w][lane] = s0 + s1;
    __syncthreads();
    if (w == 0 && e < p * p) {
        double t = part[0][lane];
#pragma unroll
        for (int q = 1; q < kSumGramWarps; ++q) t += part[q][lane];
        S[(size_t)ax * p * p + e] = t;
    }
}

// Partial products Sp[ax][blk] = A_blk^T B_blk (p x p) of 16-row blocks of A and
// B (n x p); k_sum_gram adds the blocks in a fixed order.  CTA: one block of one axis.
__global__ void __launch_bounds__(256) k_atb(int n, int p, const double* __restrict__ A,
                                              const double* __restrict__ B, double* __restrict__ Sp) {
    __shared__ double As[16][49], Bs[16][49];
    const int ax = blockIdx.y, i0 = blockIdx.x * 16;
    const double* Aa = A + (size_t)ax * n * p;
    const double* Ba = B + (size_t)ax * n * p;
    for (int e = threadIdx.x; e < 16 * p; e += 256) {
        const int r = e / p, c = e % p, gi = i0 + r;
        As[r][c] = gi < n ? Aa[(size_t)gi * p + c] : 0.0;
        Bs[r][c] = gi < n ? Ba[(size_t)gi * p + c] : 0.0;
    }
    __syncthreads();
    double* out = Sp + ((size_t)ax * gridDim.x + blockIdx.x) * p * p;
    for (int e = threadIdx.x; e < p * p; e += 256) {
        const int a = e / p, c = e % p;
        double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int r = 0; r < 16; ++r) s[r & 3] = fma(As[r][a], Bs[r][c], s[r & 3]);
        out[e] = (s[0] + s[1]) + (s[2] + s[3]);
    }
}

// Cholesky S + shift*I = R^T R (R upper) and Rinv = R^{-1} (p <= 48) in float-pair
// arithmetic: one CTA per axis, 256 threads over a 16 x 16 tile, one barrier per step.
//   Cholesky, right-looking: step k takes rk = 1/sqrt(A[k][k]) (in every thread) and
//   updates the trailing upper triangle by A[k][i] A[k][j] rk^2; row k of R is
//   A[k][j] rk, formed where it is used.
//   Inverse, by rows from the bottom: X[k][k] = rk, X[k][j] = -rk acc[k][j], and
//   acc[i][j] += R[i][k] X[k][j] for i < k <= j.
// S is a Gram matrix: a pivot at or below 1e-14 of its trace belongs to a direction
// the block does not span (a rank-deficient block, e.g. a protein with fewer Gaussian
// terms than the block size); its column of Q becomes 0 (R[k][k] = 0, rk = 0) instead
// of amplifying rounding noise, and only a NaN pivot is a failure.  GB300 takes ~40 cycles per dependent FP64 FMA and ~450 for an
// FP64 reciprocal square root against ~4 per FP32 operation, and each step's chain
// (pivot -> row scale -> trailing update) sets the time, so the chain runs on the
// FP32 pipes: the pivot's reciprocal square root is an FP32 seed refined by one Newton
// step in pairs (~2^-45).  Pair accuracy suffices: Q = Y R^-1 spans Y's columns for any
// nonsingular R as long as the product itself is taken accurately (k_apply_rinv,
// FP64), and R only has to orthonormalise to ~1e-13 (the condition of S times 2^-47).
__device__ __forceinline__ dev::F2 pair_rsqrt(dev::F2 d) {
    using dev::F2;
    const float y = rsqrtf(d.h);
    const F2 e = dev::df_sub(F2{1.f, 0.f}, dev::df_mul(d, dev::df_mul(F2{y, 0.f}, F2{y, 0.f})));
    return dev::df_add(F2{y, 0.f}, dev::df_mul(F2{0.5f * y, 0.f}, e));  // y + y (1 - d y^2) / 2
}

__global__ void __launch_bounds__(256) k_chol_pair(int p, const double* __restrict__ S, double rel_shift,
                                                   double* __restrict__ Rinv, int* __restrict__ fail) {
    using dev::F2;
    __shared__ float2 A[48][49];   // factorised in place; R[k][j] = A[k][j] rk[k] (j > k)
    __shared__ float2 X[48][49];   // accumulators, then R^{-1}
    __shared__ float2 rk[48];      // 1 / R[k][k]
    __shared__ double red[2];
    const int ax = blockIdx.x;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const double* Sa = S + (size_t)ax * p * p;
    for (int i = ty; i < p; i += 16)
        for (int j = tx; j < p; j += 16) {
            const F2 v = dev::df_from(Sa[i * p + j]);
            A[i][j] = make_float2(v.h, v.l);
            X[i][j] = make_float2(0.f, 0.f);
        }
    if (threadIdx.x < 32) {  // shift = rel_shift * trace; null pivots at or below 1e-14 of it
        double t = 0.0;
        for (int i = threadIdx.x; i < p; i += 32) t += Sa[(size_t)i * p + i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) {
            red[0] = rel_shift * t;
            red[1] = 1e-14 * t;
        }
    }
    __syncthreads();
    const F2 shift = dev::df_from(red[0]);
    const float thresh = (float)red[1];
    if (threadIdx.x < p) {
        const F2 d = dev::df_add(F2{A[threadIdx.x][threadIdx.x].x, A[threadIdx.x][threadIdx.x].y}, shift);
        A[threadIdx.x][threadIdx.x] = make_float2(d.h, d.l);
    }
    __syncthreads();
    for (int k = 0; k < p; ++k) {
        // every thread takes the pivot's reciprocal square root itself (the same value),
        // so the step needs one barrier; row k stays unscaled (R[k][j] = A[k][j] rk)
        const F2 d{A[k][k].x, A[k][k].y};
        const F2 r = d.h > thresh ? pair_rsqrt(d) : F2{0.f, 0.f};
        if (threadIdx.x == 0) {
            if (d.h != d.h) fail[ax] = 1;
            rk[k] = make_float2(r.h, r.l);
        }
        const F2 r2 = dev::df_mul(r, r);
        for (int i = k + 1 + ty; i < p; i += 16) {
            const F2 aki = dev::df_mul(F2{A[k][i].x, A[k][i].y}, r2);
            for (int j = k + 1 + tx; j < p; j += 16)
                if (j >= i) {
                    const F2 v = dev::df_sub(F2{A[i][j].x, A[i][j].y}, dev::df_mul(aki, F2{A[k][j].x, A[k][j].y}));
                    A[i][j] = make_float2(v.h, v.l);
                }
        }
        __syncthreads();
    }
    // R^{-1}, rows from the bottom: step k adds row k's part to the rows above (X[k][.]
    // taken from its sums, complete once every row below k has been added) and makes
    // row k + 1 final, which no thread reads in this step: one barrier per step
    auto final_x = [&](int k, int j) {
        const F2 rr{rk[k].x, rk[k].y};
        const F2 v = j == k ? rr : dev::df_mul(F2{-rr.h, -rr.l}, F2{X[k][j].x, X[k][j].y});
        X[k][j] = make_float2(v.h, v.l);
    };
    for (int k = p - 1; k >= 0; --k) {
        const F2 r{rk[k].x, rk[k].y};
        for (int i = ty; i < k; i += 16) {
            const F2 rik = dev::df_mul(F2{A[i][k].x, A[i][k].y}, F2{rk[i].x, rk[i].y});  // R[i][k]
            for (int j = k + tx; j < p; j += 16) {
                const F2 xkj = j == k ? r : dev::df_mul(F2{-r.h, -r.l}, F2{X[k][j].x, X[k][j].y});
                const F2 v = dev::df_add(F2{X[i][j].x, X[i][j].y}, dev::df_mul(rik, xkj));
                X[i][j] = make_float2(v.h, v.l);
            }
        }
        if (k + 1 < p && threadIdx.x > k && threadIdx.x < p) final_x(k + 1, threadIdx.x);
        __syncthreads();
    }
    if (threadIdx.x < p) final_x(0, threadIdx.x);
    __syncthreads();
    double* Ra = Rinv + (size_t)ax * p * p;
    for (int i = ty; i < p; i += 16)
        for (int j = tx; j < p; j += 16) Ra[i * p + j] = j >= i ? dev::df_to(F2{X[i][j].x, X[i][j].y}) : 0.0;
}

// Shifted Cholesky and inverse of the three p x p Grams of a CholQR pass.
void launch_chol(int p, const double* S, double rel_shift, double* Rinv, int* fail, cudaStream_t st) {
    k_chol_pair<<<3, 256, 0, st>>>(p, S, rel_shift, Rinv, fail);  // p <= 48
}

// Q = Y Rinv (Rinv upper triangular), n x p; Q2 (if not null) gets Q as float pairs.
__global__ void k_apply_rinv(int n, int p, const double* __restrict__ Y,
                             const double* __restrict__ Rinv, double* __restrict__ Q,
                             float2* __restrict__ Q2) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ax = blockIdx.y;
    if (idx >= (size_t)n * p) return;
    int i = (int)(idx / p), c = (int)(idx % p);
    const double* Ya = Y + ((size_t)ax * n + i) * p;
    const double* Ra = Rinv + (size_t)ax * p * p;
    double t[4] = {0.0, 0.0, 0.0, 0.0};  // four interleaved partial sums, fixed order
    for (int k = 0; k <= c; ++k) t[k & 3] = fma(Ya[k], Ra[(size_t)k * p + c], t[k & 3]);
    const double s = (t[0] + t[1]) + (t[2] + t[3]);
    Q[((size_t)ax * n + i) * p + c] = s;
    if (Q2) {
        const dev::F2 q = dev::df_from(s);
        Q2[((size_t)ax * n + i) * p + c] = make_float2(q.h, q.l);
    }
}

// V[ax][:, 0:RP] = Q[ax] W[ax][:, 0:r_ax] (zero columns r_ax..RP-1); n x RP.
__global__ void k_ritz_vectors(int n, int p, int RP, const int* __restrict__ r_ax,
                               const double* __restrict__ Q, const double* __restrict__ W,
                               double* __restrict__ V) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ax = blockIdx.y;
    if (idx >= (size_t)n * RP) return;
    int i = (int)(idx / RP), c = (int)(idx % RP);
    double s = 0.0;
    if (c < r_ax[ax]) {
        const double* Qa = Q + ((size_t)ax * n + i) * p;
        const double* Wa = W + (size_t)ax * p * p;
        for (int k = 0; k < p; ++k) s += Qa[k] * Wa[(size_t)k * p + c];
    }
    V[((size_t)ax * n + i) * RP + c] = s;
}

// ------------------------------------------------------------------ skeleton basis
// Pivoted Gram-Schmidt on the rows of V (n x r) picks r rows S (largest residual
// norm first; ties to the lower index); A = V[S,:] sorted by row index; then
// Vs = V A^{-1} (cardinal basis: Vs[S_a, b] = delta_ab) and Wp = V A^T.
__global__ void __launch_bounds__(512) k_skeleton(int n, int RP, const int* __restrict__ r_ax,
                                                   const double* __restrict__ V,
                                                   double* __restrict__ M,
                                                   int* __restrict__ Sidx,
                                                   double* __restrict__ Ainv,
                                                   int* __restrict__ fail, bool use_smem) {
    __shared__ float red_v[512];
    __shared__ int red_i[512];
    __shared__ float piv[RS_MAX_TUCKER];
    __shared__ int sel[RS_MAX_TUCKER];
    __shared__ double A[RS_MAX_TUCKER][2 * RS_MAX_TUCKER + 1];
    extern __shared__ float rows_sm[];  // the residual rows when they fit (n RP floats)
    int ax = blockIdx.x;
    int r = r_ax[ax];
    const double* Va = V + (size_t)ax * n * RP;
    // The selection runs in FP32: it only has to pick well-conditioned rows (the
    // basis change V V[S,:]^-1 and the core transform use the exact FP64 rows), and
    // GB300's FP64 rate made the FP64 version the build's slowest serial kernel.  The
    // residual rows live in shared memory when the launch provides it (every step
    // reads and rewrites all of them).
    float* Ma = use_smem ? rows_sm : reinterpret_cast<float*>(M) + (size_t)ax * n * RP;
    for (size_t e = threadIdx.x; e < (size_t)n * RP; e += blockDim.x) Ma[e] = (float)Va[e];
    __syncthreads();
    for (int step = 0; step < r; ++step) {
        float best = -1.f;
        int bi = n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float s = 0.f;
            for (int c = 0; c < r; ++c) s = fmaf(Ma[(size_t)i * RP + c], Ma[(size_t)i * RP + c], s);
            if (s > best || (s == best && i < bi)) {
                best = s;
                bi = i;
            }
        }
        red_v[threadIdx.x] = best;
        red_i[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                float v2 = red_v[threadIdx.x + o];
                int i2 = red_i[threadIdx.x + o];
                if (v2 > red_v[threadIdx.x] || (v2 == red_v[threadIdx.x] && i2 < red_i[threadIdx.x])) {
                    red_v[threadIdx.x] = v2;
                    red_i[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        int pi = red_i[0];
        float nrm = sqrtf(red_v[0]);
        if (threadIdx.x == 0) {
            sel[step] = pi;
            if (!(nrm > 0.f)) fail[ax] = 2;
        }
        if (threadIdx.x < r) piv[threadIdx.x] = nrm > 0.f ? Ma[(size_t)pi * RP + threadIdx.x] / nrm : 0.f;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float d = 0.f;
            for (int c = 0; c < r; ++c) d = fmaf(Ma[(size_t)i * RP + c], piv[c], d);
            for (int c = 0; c < r; ++c) Ma[(size_t)i * RP + c] = fmaf(-d, piv[c], Ma[(size_t)i * RP + c]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {  // sort selected rows ascending
        for (int i = 1; i < r; ++i) {
            int v = sel[i];
            int j = i - 1;
            while (j >= 0 && sel[j] > v) {
                sel[j + 1] = sel[j];
                --j;
            }
            sel[j + 1] = v;
        }
    }
    __syncthreads();
    // [A | I] -> [I | A^{-1}] by Gauss-Jordan with partial pivoting
    for (int e = threadIdx.x; e < r * 2 * r; e += blockDim.x) {
        int i = e / (2 * r), j = e % (2 * r);
        A[i][j] = (j < r) ? Va[(size_t)sel[i] * RP + j] : ((j - r) == i ? 1.0 : 0.0);
    }
    __syncthreads();
    __shared__ int pivrow;
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x < 32) {  // partial pivoting: warp argmax of |A[i][k]|, i >= k (lowest i on ties)
            const int i = k + (int)threadIdx.x;
            double v = i < r ? fabs(A[i][k]) : -1.0;
            int bi = i;
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (v2 > v || (v2 == v && i2 < bi)) {
                    v = v2;
                    bi = i2;
                }
            }
            if (threadIdx.x == 0) {
                pivrow = bi;
                if (!(v > 0.0)) fail[ax] = 3;
            }
        }
        __syncthreads();
        const int best = pivrow;
        if (best != k)
            for (int j = threadIdx.x; j < 2 * r; j += blockDim.x) {
                const double t = A[k][j];
                A[k][j] = A[best][j];
                A[best][j] = t;
            }
        __syncthreads();
        double d = A[k][k];
        __syncthreads();
        for (int j = threadIdx.x; j < 2 * r; j += blockDim.x) A[k][j] /= d;
        __syncthreads();
        for (int e = threadIdx.x; e < r * 2 * r; e += blockDim.x) {
            int i = e / (2 * r), j = e % (2 * r);
            if (i != k) {
                double f = A[i][k];
                if (j != k) A[i][j] -= f * A[k][j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < r; i += blockDim.x)
            if (i != k) A[i][k] = 0.0;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
        int i = e / RP, j = e % RP;
        Ainv[((size_t)ax * RP + i) * RP + j] = (i < r && j < r) ? A[i][r + j] : 0.0;
    }
    for (int i = threadIdx.x; i < RP; i += blockDim.x) Sidx[ax * RS_MAX_TUCKER + i] = i < r ? sel[i] : -1;
}

// Vs = V Ainv (the cardinal evaluation basis, FP64) and Wp = V V[S,:]^T (float pairs).
__global__ void k_skeleton_apply(int n, int RP, const int* __restrict__ r_ax,
                                 const double* __restrict__ V, const double* __restrict__ Ainv,
                                 const int* __restrict__ Sidx, double* __restrict__ Vs,
                                 float2* __restrict__ Wp2) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ax = blockIdx.y;
    if (idx >= (size_t)n * RP) return;
    int i = (int)(idx / RP), c = (int)(idx % RP);
    int r = r_ax[ax];
    const double* Vr = V + ((size_t)ax * n + i) * RP;
    double s = 0.0, w = 0.0;
    if (c < r) {
        const double* Ai = Ainv + (size_t)ax * RP * RP;
        for (int k = 0; k < r; ++k) s += Vr[k] * Ai[(size_t)k * RP + c];
        int srow = Sidx[ax * RS_MAX_TUCKER + c];
        const double* Vsr = V + ((size_t)ax * n + srow) * RP;
        for (int k = 0; k < r; ++k) w += Vr[k] * Vsr[k];
    }
    Vs[((size_t)ax * n + i) * RP + c] = s;
    const dev::F2 wp = dev::df_from(w);
    Wp2[((size_t)ax * n + i) * RP + c] = make_float2(wp.h, wp.l);
}

__device__ __forceinline__ void split_pair(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// Float-pair rows of the axis-1 and axis-2 cardinal factors and their row
// differences: Vh + Vl = V'[i][c], VDh + VDl = V'[i+1][c] - V'[i][c].
__global__ void k_pair_rows(int n, int RP, const double* __restrict__ Vs, float* __restrict__ out0,
                            float* __restrict__ out1) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ax = blockIdx.y;
    if (idx >= (size_t)n * RP) return;
    int i = (int)(idx / RP), c = (int)(idx % RP);
    const double* Va = Vs + (size_t)ax * n * RP;
    double v = Va[(size_t)i * RP + c];
    double d = i + 1 < n ? Va[(size_t)(i + 1) * RP + c] - v : 0.0;
    float* o = ax == 0 ? out0 : out1;
    size_t plane = (size_t)n * RP;
    split_pair(v, o[idx], o[plane + idx]);
    split_pair(d, o[2 * plane + idx], o[3 * plane + idx]);
}

// W[i][a][b] = sum_c V3'[i][c] core[a][b][c] and D[i] = W[i+1] - W[i] (FP64), split
// into float pairs: out = [Wh | Wl | Dh | Dl], each [n][RP][RP].
__global__ void k_wtable(int n, int RP, const double* __restrict__ Vs3,
                         const double* __restrict__ B, float* __restrict__ out) {
    int ab = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (ab >= RP * RP) return;
    const double* row0 = Vs3 + (size_t)i * RP;
    const double* row1 = Vs3 + (size_t)min(i + 1, n - 1) * RP;
    const double* bc = B + (size_t)ab * RP;
    double w0 = 0.0, w1 = 0.0;
    for (int c = 0; c < RP; ++c) {
        w0 += row0[c] * bc[c];
        w1 += row1[c] * bc[c];
    }
    double d = i + 1 < n ? w1 - w0 : 0.0;
    size_t plane = (size_t)n * RP * RP;
    size_t o = (size_t)i * RP * RP + ab;
    split_pair(w0, out[o], out[plane + o]);
    split_pair(d, out[2 * plane + o], out[3 * plane + o]);
}

// C'[ax][a][(m,k)] = sum_i Wp[ax][i][a] exp(-t_k^2 (x_i - x_m^ax)^2), in float-pair
// arithmetic on the FP32 pipes (GB300's FP64 rate is 1/64 of its FP32 rate).
// CTA: 128 atoms, one (k, axis).  The CTA walks the union of the atoms' windows
// (rows where the exponent is <= 46, i.e. the Gaussian is >= 1e-20 of its peak);
// each thread runs its Gaussian by the ratio recurrence g <- g rho, rho <- rho q
// (q = exp(-2 t^2 h^2)) in pairs, re-seeded from FP64 exponentials every 256 rows
// so the recurrence error stays ~1e-12; Gaussians narrower than the grid
// (t^2 h^2 > 8) are evaluated directly at every row.
constexpr int kProjReseed = 256;

// Atoms of each axis in order of their grid row (a counting sort): k_project gives a
// CTA 128 consecutive atoms of this order, so their Gaussian windows nearly coincide
// and the CTA walks few rows outside its atoms' windows.  The order within a row
// (atomic slots) decides only which thread computes a column, not its value.
__global__ void k_axis_count(int N, const double* __restrict__ xyz, double b, double h, int n,
                             int* __restrict__ cnt, int* __restrict__ row_of) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x, ax = blockIdx.y;
    if (m >= N) return;
    const int i = min(max((int)floor((xyz[3 * (size_t)m + ax] + b) / h), 0), n - 1);
    row_of[(size_t)ax * N + m] = i;
    atomicAdd(&cnt[(size_t)ax * n + i], 1);
}

__global__ void k_axis_fill(int N, int n, const int* __restrict__ row_of, const int* __restrict__ start,
                            int* __restrict__ cursor, int* __restrict__ perm) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x, ax = blockIdx.y;
    if (m >= N) return;
    const int i = row_of[(size_t)ax * N + m];
    perm[(size_t)ax * N + start[(size_t)ax * (n + 1) + i] + atomicAdd(&cursor[(size_t)ax * n + i], 1)] = m;
}

template <int RP>
__global__ void __launch_bounds__(128) k_project(int n, double b, double h, int N, int Rl,
                                                  const double* __restrict__ xyz,
                                                  const double* __restrict__ tl,
                                                  const int* __restrict__ perm,
                                                  const float2* __restrict__ Wp2,
                                                  float2* __restrict__ Cp2) {
    using dev::F2;
    __shared__ float2 Ws[32][RP];
    __shared__ int wlo[128], whi[128];
    int k = blockIdx.y, ax = blockIdx.z;
    const int mo = blockIdx.x * 128 + threadIdx.x;
    bool valid = mo < N;
    const int m = valid ? perm[(size_t)ax * N + mo] : 0;  // atoms in grid-row order
    double t2 = tl[k] * tl[k];
    double xm = valid ? xyz[3 * (size_t)m + ax] : 0.0;
    int lo = n, hi = -1;
    const bool direct = t2 * h * h > 8.0;
    if (valid) {
        if (t2 == 0.0) {
            lo = 0;
            hi = n - 1;
        } else {
            double hw = sqrt(46.0 / t2);
            double l = ceil((xm - hw + b) / h), u = floor((xm + hw + b) / h);
            l = fmax(l, 0.0);
            u = fmin(u, (double)(n - 1));
            if (l <= u) {
                lo = (int)l;
                hi = (int)u;
            }
        }
    }
    wlo[threadIdx.x] = lo;
    whi[threadIdx.x] = hi;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            wlo[threadIdx.x] = min(wlo[threadIdx.x], wlo[threadIdx.x + o]);
            whi[threadIdx.x] = max(whi[threadIdx.x], whi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    int ulo = wlo[0], uhi = whi[0];
    __syncthreads();
    F2 acc[RP];
#pragma unroll
    for (int a = 0; a < RP; ++a) acc[a] = F2{0.f, 0.f};
    const F2 cq = dev::df_from(direct ? 0.0 : exp(-2.0 * t2 * h * h));
    F2 g{0.f, 0.f}, rho{0.f, 0.f};
    int since = 0;
    const float2* Wa = Wp2 + (size_t)ax * n * RP;
    for (int i0 = ulo; i0 <= uhi; i0 += 32) {
        for (int e = threadIdx.x; e < 32 * RP; e += 128) {
            int ii = e / RP, c = e % RP;
            int gi = i0 + ii;
            Ws[ii][c] = gi <= uhi ? Wa[(size_t)gi * RP + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        int iend = min(32, uhi - i0 + 1);
        for (int ii = 0; ii < iend; ++ii) {
            int i = i0 + ii;
            if (i < lo || i > hi) continue;
            if (i == lo || direct || since == kProjReseed) {
                double d = (-b + i * h) - xm;
                g = dev::df_from(exp(-t2 * d * d));
                rho = dev::df_from(exp(-t2 * (2.0 * d * h + h * h)));
                since = 0;
            } else {
                g = dev::df_mul(g, rho);
                rho = dev::df_mul(rho, cq);
            }
            ++since;
#pragma unroll
            for (int a = 0; a < RP; ++a) dev::df_fma_acc(acc[a], F2{Ws[ii][a].x, Ws[ii][a].y}, g);
        }
        __syncthreads();
    }
    if (valid) {
        size_t Rp = (size_t)N * Rl;
        size_t col = (size_t)m * Rl + k;
#pragma unroll
        for (int a = 0; a < RP; ++a) {
            float sh, sl;
            dev::two_sum(acc[a].h, acc[a].l, sh, sl);
            Cp2[((size_t)ax * RP + a) * Rp + col] = make_float2(sh, sl);
        }
    }
}

// Partial cores over column chunks: Bp[chunk][a][b][c] = sum_r xi_r C'1[a,r] C'2[b,r] C'3[c,r],
// in float-pair arithmetic; CTA: RP*RP threads, thread = (a, b), CH columns per CTA.
template <int RP>
__global__ void __launch_bounds__(RP * RP, 1) k_core(int Rtot, int Rl, int CH,
                                               const double* __restrict__ q,
                                               const double* __restrict__ al,
                                               const float2* __restrict__ Cp2,
                                               double* __restrict__ Bp) {
    using dev::F2;
    __shared__ float2 C1s[32][RP], C2s[32][RP], C3s[32][RP], xis[32];
    int chunk = blockIdx.x;
    int a = threadIdx.x / RP, bb = threadIdx.x % RP;
    F2 acc[RP];
#pragma unroll
    for (int c = 0; c < RP; ++c) acc[c] = F2{0.f, 0.f};
    int r0 = chunk * CH, r1 = min(Rtot, r0 + CH);
    for (int t0 = r0; t0 < r1; t0 += 32) {
        for (int e = threadIdx.x; e < 32 * RP; e += blockDim.x) {
            int j = e / RP, c = e % RP;
            int col = t0 + j;
            bool ok = col < r1;
            float2 z = make_float2(0.f, 0.f);
            C1s[j][c] = ok ? Cp2[((size_t)0 * RP + c) * Rtot + col] : z;
            C2s[j][c] = ok ? Cp2[((size_t)1 * RP + c) * Rtot + col] : z;
            C3s[j][c] = ok ? Cp2[((size_t)2 * RP + c) * Rtot + col] : z;
        }
        for (int j = threadIdx.x; j < 32; j += blockDim.x) {
            int col = t0 + j;
            F2 x = dev::df_from(col < r1 ? q[col / Rl] * al[col % Rl] : 0.0);
            xis[j] = make_float2(x.h, x.l);
        }
        __syncthreads();
        int jend = min(32, r1 - t0);
        for (int j = 0; j < jend; ++j) {
            F2 u = dev::df_mul(dev::df_mul(F2{xis[j].x, xis[j].y}, F2{C1s[j][a].x, C1s[j][a].y}),
                               F2{C2s[j][bb].x, C2s[j][bb].y});
#pragma unroll
            for (int c = 0; c < RP; ++c) dev::df_fma_acc(acc[c], u, F2{C3s[j][c].x, C3s[j][c].y});
        }
        __syncthreads();
    }
    double* out = Bp + (size_t)chunk * RP * RP * RP + ((size_t)a * RP + bb) * RP;
#pragma unroll
    for (int c = 0; c < RP; ++c) out[c] = dev::df_to(acc[c]);
}

// ------------------------------------------------------------- tensor-core projection
// k_project on tcgen05: for one axis, one long-range term k and 128 atoms m (in grid-row
// order), C'[a, (m, k)] = sum_i Wp[i, a] g_k(x_i - x_m) is the GEMM (atoms x grid rows) x
// (grid rows x a) with K = the grid rows of the CTA's window, cut into 16-row chunks.
// The Gaussians are generated per chunk in float pairs (seeds by the pair exponential
// every 32 rows, then the ratio recurrence g_{i+1} = g_i rho_i, rho_{i+1} = rho_i
// e^{-2 t^2 h^2}) and cut into six exact BF16 slices straight into the A tile; Wp's
// slices per (column, chunk) are made once per build (k_slice_wp).  The 21 slice
// products go to six TMEM accumulators, one per diagonal.  Six consecutive chunks (a
// 96-row group) share one scale per atom (from the largest Gaussian value of the group
// in the atom's window) and one per column of Wp, so the accumulators run over the
// whole group: a diagonal's integer K-sum stays below 96 * 122880 < 2^24 (diagonal 5,
// |d_0| <= 32, |d_1|, |d_2| <= 128, |d_3| <= 160, |d_4|, |d_5| <= 256: exact), and the
// six diagonals are combined error-free into a float pair once per group and summed
// over the groups in pair arithmetic.  Rows outside an atom's own window (where its
// Gaussian is below e^-46 of the peak) are zero, as in the float-pair kernel.
//
// Warp roles: warps 0-3 own one atom per thread (the A rows), warp 4 copies Wp's
// slices and issues the MMAs.  The chunks run through a ring of kPS stages of A and B
// tiles with mbarriers instead of CTA-wide barriers: a row warp announces its rows of
// a stage (full), the issuer waits for all four and for the B copy, issues and commits
// (mma); a row warp reuses a stage once its MMAs have completed and reads TMEM at the
// end of a group, after which it announces that the accumulators may be overwritten
// (drained).  So each warp runs ahead to the next chunk as soon as its own rows are
// written, and the MMAs of one chunk overlap the rows of the next ones.
constexpr int kPK = 16;                        // grid rows per K chunk (one MMA K step)
constexpr int kPG = 6;                         // chunks per scale group (96 rows)
constexpr int kPS = 3;                         // stages of the ring
constexpr uint32_t kPSBO = kPK * 16;           // bytes between 8-row groups of a tile
constexpr uint32_t kPSliceA = 128 * kPK * 2;   // one slice of an A tile (4 KB)

template <int NP>
struct ProjShape {
    static constexpr uint32_t SLICE_B = NP * kPK * 2;
    static constexpr uint32_t A_BYTES = tcg::kS * kPSliceA;  // one A stage
    static constexpr uint32_t B_BYTES = tcg::kS * SLICE_B;   // one B stage (one chunk)
    static constexpr uint32_t B_OFF = kPS * A_BYTES;
    // barriers: full[kPS], ld[kPS], mma[kPS], drained
    static constexpr uint32_t BAR_OFF = B_OFF + kPS * B_BYTES;
    static constexpr uint32_t SLOT_OFF = BAR_OFF + (3 * kPS + 1) * 8;
    static constexpr uint32_t ABORT_OFF = SLOT_OFF + 4;
    static constexpr uint32_t WIN_OFF = SLOT_OFF + 16;  // window bounds, 2 x 128 ints
    static constexpr uint32_t SMEM = WIN_OFF + 2 * 128 * 4;
    static constexpr uint32_t COLS = tcg::kS * NP;
    static constexpr uint32_t NCOL = COLS <= 128 ? 128 : 256;
};

// B slices of Wp (n x RP float pairs per axis), K = the grid row: chunk kc of axis ax at
// out + (ax KC + kc) B_BYTES (rows a >= RP zero); the scale of column a is shared by the
// chunk's 96-row group g = kc / kPG: binv[(ax KG + g) NP + a] = 1 / scale.
template <int NP>
__global__ void __launch_bounds__(NP) k_slice_wp(int n, int RP, int KC, int KG, const float2* __restrict__ Wp,
                                                  uint8_t* __restrict__ out, float* __restrict__ binv) {
    using Sh = ProjShape<NP>;
    const int kc = blockIdx.x, ax = blockIdx.y, a = threadIdx.x;
    const int i0 = kc * kPK, grp = kc / kPG, g0 = grp * kPG * kPK;
    const float2* Wa = Wp + (size_t)ax * n * RP;
    float m = 0.f;
    if (a < RP)
        for (int i = g0; i < min(n, g0 + kPG * kPK); ++i) m = fmaxf(m, fabsf(Wa[(size_t)i * RP + a].x));
    float sc, inv;
    tc::row_scale(m, sc, inv);
    if (kc % kPG == 0) binv[((size_t)ax * KG + grp) * NP + a] = inv;
    uint8_t* tile = out + ((size_t)ax * KC + kc) * Sh::B_BYTES;
#pragma unroll 1
    for (int g = 0; g < kPK / 8; ++g) {
        uint32_t w[tcg::kS][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float lo[tcg::kS], hi[tcg::kS];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int i = i0 + g * 8 + e + hh;
                const float2 v = (a < RP && i < n) ? Wa[(size_t)i * RP + a] : make_float2(0.f, 0.f);
                tcg::slice6(__fmul_rn(v.x, sc), __fmul_rn(v.y, sc), hh ? hi : lo);
            }
#pragma unroll
            for (int u = 0; u < tcg::kS; ++u) w[u][e / 2] = tc::pack_bf16x2(lo[u], hi[u]);
        }
#pragma unroll
        for (int u = 0; u < tcg::kS; ++u)
            *reinterpret_cast<uint4*>(tile + u * Sh::SLICE_B + tc::kmajor_offset(a, g * 8, kPSBO)) =
                make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
    }
}

// The Gaussian of one atom on a chunk's rows ia..ib (others zero) as six slices into
// row `row` of an A stage.  DIRECT: every value by the pair exponential; else the ratio
// recurrence (g, rho) continues from the previous row.
struct ProjGauss {
    dev::F2 nt2, hp, base, cq;
    const float2* etab;
    __device__ __forceinline__ dev::F2 offset(int i) const {
        return dev::df_add(base, dev::df_mul(hp, dev::F2{(float)i, 0.f}));
    }
    __device__ __forceinline__ dev::F2 gauss(dev::F2 d) const {
        return df_exp(dev::df_mul(nt2, dev::df_mul(d, d)), etab);
    }
};

template <bool DIRECT>
__device__ __forceinline__ void proj_row(const ProjGauss& G, uint8_t* sA, int row, int i0, int ia, int ib, float sc,
                                         dev::F2& g, dev::F2& rho) {
    using dev::F2;
#pragma unroll 1
    for (int gq = 0; gq < kPK / 8; ++gq) {
        uint32_t w[tcg::kS][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float slo[tcg::kS], shi[tcg::kS];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int i = i0 + gq * 8 + e + hh;
                F2 val{0.f, 0.f};
                if (i >= ia && i <= ib) {
                    if (DIRECT) {
                        val = G.gauss(G.offset(i));
                    } else {
                        val = g;
                        g = dev::df_mul(g, rho);
                        rho = dev::df_mul(rho, G.cq);
                    }
                }
                tcg::slice6(__fmul_rn(val.h, sc), __fmul_rn(val.l, sc), hh ? shi : slo);
            }
#pragma unroll
            for (int u = 0; u < tcg::kS; ++u) w[u][e / 2] = tc::pack_bf16x2(slo[u], shi[u]);
        }
#pragma unroll
        for (int u = 0; u < tcg::kS; ++u)
            *reinterpret_cast<uint4*>(sA + u * kPSliceA + tc::kmajor_offset(row, gq * 8, kPSBO)) =
                make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]);
    }
}

template <int RP, int NP>
__global__ void __launch_bounds__(160, 2) k_project_tc(int n, double b, double h, int N, int Rl, int KC, int KG,
                                                     const double* __restrict__ xyz,
                                                     const double* __restrict__ tl,
                                                     const int* __restrict__ perm,
                                                     const float2* __restrict__ etab,
                                                     const uint8_t* __restrict__ Bs,
                                                     const float* __restrict__ binv,
                                                     float2* __restrict__ Cp2, int* __restrict__ err) {
    using dev::F2;
    using Sh = ProjShape<NP>;
    extern __shared__ __align__(16) uint8_t smem_p[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_p + Sh::BAR_OFF);  // rows written (4 arrivals)
    uint64_t* ldb = full + kPS;                                          // B copy landed
    uint64_t* mmb = ldb + kPS;                                           // MMAs complete
    uint64_t* drained = mmb + kPS;                                       // TMEM read (4 arrivals)
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem_p + Sh::SLOT_OFF);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem_p + Sh::ABORT_OFF);
    int* wlo = reinterpret_cast<int*>(smem_p + Sh::WIN_OFF);
    int* whi = wlo + 128;
    const int k = blockIdx.y, ax = blockIdx.z, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool rows = warp < 4;  // warps 0-3: one atom per thread; warp 4: copies and MMAs
    const int mo = blockIdx.x * 128 + tid;
    const bool valid = rows && mo < N;
    const int m = valid ? perm[(size_t)ax * N + mo] : 0;  // atoms in grid-row order
    const double t2 = tl[k] * tl[k];
    const double xm = valid ? xyz[3 * (size_t)m + ax] : 0.0;
    int lo = n, hi = -1;
    if (valid) {
        if (t2 == 0.0) {
            lo = 0;
            hi = n - 1;
        } else {
            const double hw = sqrt(46.0 / t2);
            const double l = fmax(ceil((xm - hw + b) / h), 0.0), u = fmin(floor((xm + hw + b) / h), (double)(n - 1));
            if (l <= u) {
                lo = (int)l;
                hi = (int)u;
            }
        }
    }
    if (rows) {
        wlo[tid] = lo;
        whi[tid] = hi;
    }
    if (warp == 0) tc::tmem_alloc(slot, Sh::NCOL);
    if (tid == 0) {
        for (int q = 0; q < kPS; ++q) {
            tc::mbar_init(full + q, 4);
            tc::mbar_init(ldb + q, 1);
            tc::mbar_init(mmb + q, 1);
        }
        tc::mbar_init(drained, 4);
        *abort_flag = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    for (int o = 64; o > 0; o >>= 1) {
        if (tid < o) {
            wlo[tid] = min(wlo[tid], wlo[tid + o]);
            whi[tid] = max(whi[tid], whi[tid + o]);
        }
        __syncthreads();
    }
    const int ulo = wlo[0], uhi = whi[0];
    const uint32_t tmem = *slot;
    const int c0 = ulo <= uhi ? ulo / kPK : 0, nch = ulo <= uhi ? uhi / kPK - c0 + 1 : 0;
    F2 acc[RP];
#pragma unroll
    for (int a = 0; a < RP; ++a) acc[a] = F2{0.f, 0.f};
    if (!rows) {
        // ---- issuer: lane 0 of warp 4
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NP);
            int last_ld = -1, last_mma = -1, grp = -1;
            bool ok = true;
            for (int j = 0; j < nch && ok; ++j) {
                const int s = j % kPS, c = c0 + j;
                const uint32_t ph = (uint32_t)(j / kPS) & 1u;
                const bool gfirst = j == 0 || c % kPG == 0;
                uint8_t* sA = smem_p + s * Sh::A_BYTES;
                uint8_t* sB = smem_p + Sh::B_OFF + s * Sh::B_BYTES;
                // stage s was last read by the MMAs of chunk j - kPS
                if (j >= kPS) ok = tc::mbar_wait_bounded(mmb + s, ph ^ 1u);
                if (!ok || *abort_flag) break;
                tc::mbar_arrive_expect_tx(ldb + s, Sh::B_BYTES);
                tc::bulk_g2s(sB, Bs + ((size_t)ax * KC + c) * Sh::B_BYTES, Sh::B_BYTES, ldb + s);
                last_ld = j;
                ok = tc::mbar_wait_bounded(full + s, ph) && tc::mbar_wait_bounded(ldb + s, ph);
                // a new group overwrites the accumulators: the row warps have read them
                if (ok && gfirst && grp >= 0) ok = tc::mbar_wait_bounded(drained, (uint32_t)grp & 1u);
                if (!ok || *abort_flag) break;
                if (gfirst) ++grp;
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
                for (int d = 0; d < tcg::kS; ++d)
#pragma unroll
                    for (int u = 0; u <= d; ++u) {
                        const uint64_t ad = tc::smem_desc(a0 + u * kPSliceA, tc::kLBO, kPSBO);
                        const uint64_t bd = tc::smem_desc(b0 + (d - u) * Sh::SLICE_B, tc::kLBO, kPSBO);
                        tc::mma_bf16(tmem + (uint32_t)(d * NP), ad, bd, idesc, (gfirst && u == 0) ? 0u : 1u);
                    }
                tc::mma_commit(mmb + s);
                last_mma = j;
            }
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                atomicExch(err, 1);
                // a copy or MMAs may still be in flight: wait for them (bounded)
                if (last_ld >= 0) tc::mbar_wait_bounded(ldb + last_ld % kPS, (uint32_t)(last_ld / kPS) & 1u);
                if (last_mma >= 0) tc::mbar_wait_bounded(mmb + last_mma % kPS, (uint32_t)(last_mma / kPS) & 1u);
            }
        }
    } else {
        // ---- row warps: one atom per thread
        ProjGauss G;
        G.nt2 = dev::df_from(-t2);
        G.hp = dev::df_from(h);
        G.base = dev::df_from(-b - xm);
        G.etab = etab;
        const bool direct = t2 * h * h > 8.0;
        G.cq = direct ? F2{0.f, 0.f} : df_exp(dev::df_from(-2.0 * t2 * h * h), etab);
        const int ipeak = valid ? (int)rint((xm + b) / h) : 0;  // grid row nearest the atom
        const uint32_t tl_lane = tmem + ((uint32_t)(warp * 32) << 16);
        float sc = 0.f, ainv = 0.f;     // the atom's scale in the current group
        F2 g{0.f, 0.f}, rho{0.f, 0.f};  // the recurrence, carried from chunk to chunk
        bool ok = true;
        for (int j = 0; j < nch; ++j) {
            const int s = j % kPS, c = c0 + j, i0 = c * kPK;
            const uint32_t ph = (uint32_t)(j / kPS) & 1u;
            const bool gfirst = j == 0 || c % kPG == 0;
            const bool glast = j == nch - 1 || c % kPG == kPG - 1;
            uint8_t* sA = smem_p + s * Sh::A_BYTES;
            if (j >= kPS) ok = tc::mbar_wait_bounded(mmb + s, ph ^ 1u);  // stage s free
            if (__any_sync(0xffffffffu, !ok || *abort_flag != 0)) {  // one decision per warp
                ok = false;
                break;
            }
            if (gfirst) {  // the atom's scale over the group's rows of its window
                const int g0 = (c / kPG) * kPG * kPK;
                const int ga = max(lo, g0), gb = min(hi, g0 + kPG * kPK - 1);
                sc = 0.f;
                ainv = 0.f;
                if (ga <= gb) {
                    const int ip = min(max(ipeak, ga), gb);  // the group's row nearest the peak
                    const F2 gmax = G.gauss(G.offset(ip));
                    tc::row_scale(__fmul_rn(gmax.h, 1.00000095367431640625f), sc, ainv);
                }
            }
            const int ia = max(lo, i0), ib = min(hi, i0 + kPK - 1);
            if (direct) {
                proj_row<true>(G, sA, tid, i0, ia, ib, sc, g, rho);
            } else {
                // seed at the window's first row and every 32 rows; else continue the walk
                if (ia <= ib && (ia == lo || (c & 1) == 0)) {
                    const F2 d0 = G.offset(ia);
                    g = G.gauss(d0);
                    // rho_i = e^{-t^2 (2 d_i h + h^2)}
                    const F2 arg = dev::df_add(dev::df_mul(F2{2.f, 0.f}, dev::df_mul(d0, G.hp)), dev::df_mul(G.hp, G.hp));
                    rho = df_exp(dev::df_mul(G.nt2, arg), etab);
                }
                proj_row<false>(G, sA, tid, i0, ia, ib, sc, g, rho);
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full + s);
            if (glast) {
                ok = tc::mbar_wait_bounded(mmb + s, ph);  // every MMA of the group
                if (__any_sync(0xffffffffu, !ok)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const float* bi = binv + ((size_t)ax * KG + c / kPG) * NP;
#pragma unroll
                for (int cb = 0; cb < NP; cb += 8) {
                    if (cb < RP) {
                        float x[tcg::kS][8];
                        tcg::tmem_ld8x3(tl_lane + cb, NP, x[0], x[1], x[2]);
                        tcg::tmem_ld8x3(tl_lane + 3 * NP + cb, NP, x[3], x[4], x[5]);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (cb + q < RP) {
                                const F2 sum = tcg::combine6(x[0][q], x[1][q], x[2][q], x[3][q], x[4][q], x[5][q]);
                                const float scl = __fmul_rn(ainv, __ldg(bi + cb + q));
                                acc[cb + q] =
                                    dev::df_add(acc[cb + q], F2{__fmul_rn(sum.h, scl), __fmul_rn(sum.l, scl)});
                            }
                        }
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(drained);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            if (tid == 0) atomicExch(err, 1);
#pragma unroll
            for (int a = 0; a < RP; ++a) acc[a] = F2{__int_as_float(-1), 0.f};
        }
        if (valid) {
            const size_t Rp = (size_t)N * Rl, col = (size_t)m * Rl + k;
#pragma unroll
            for (int a = 0; a < RP; ++a) {
                float sh, sl;
                dev::two_sum(acc[a].h, acc[a].l, sh, sl);
                Cp2[((size_t)ax * RP + a) * Rp + col] = make_float2(sh, sl);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::NCOL);
}

// Piecewise-cubic table of the short-range radial function f(s) = sum_short a_k
// exp(-t_k^2 s): on [j hs, (j+1) hs] the Hermite cubic of f and hs f' at both ends,
// in u = s/hs - j, as Horner coefficients (FP64, stored as float pairs):
//   c0 = f_j, c1 = hs f'_j, c2 = 3(f_{j+1} - f_j) - 2 hs f'_j - hs f'_{j+1},
//   c3 = 2(f_j - f_{j+1}) + hs f'_j + hs f'_{j+1}.
__device__ __forceinline__ void short_f(const ProteinView& v, double sv, double hs, double& f, double& fp) {
    f = 0.0;
    fp = 0.0;
    for (int q = 0; q < v.Ks; ++q) {
        double e = v.as[q] * exp(-v.ts2[q] * sv);
        f += e;
        fp -= v.ts2[q] * e;
    }
    fp *= hs;
}

__global__ void k_short_table(ProteinView v, int M, double hs, float4* __restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M - 1) return;
    double fa, da, fb, db;
    short_f(v, j * hs, hs, fa, da);
    short_f(v, (j + 1) * hs, hs, fb, db);
    const dev::F2 c0 = dev::df_from(fa), c1 = dev::df_from(da);
    const dev::F2 c2 = dev::df_from(3.0 * (fb - fa) - 2.0 * da - db);
    const dev::F2 c3 = dev::df_from(2.0 * (fa - fb) + da + db);
    out[2 * (size_t)j] = make_float4(c0.h, c0.l, c1.h, c1.l);
    out[2 * (size_t)j + 1] = make_float4(c2.h, c2.l, c3.h, c3.l);
}

__global__ void k_to_float(size_t len, const double* __restrict__ in, float* __restrict__ out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = (float)in[i];
}

// Inputs of the tensor-core projection (use = false: the float-pair kernel).
struct ProjTc {
    bool use = false;
    const float2* etab = nullptr;  // the pair exponential's table
    uint8_t* Bs = nullptr;         // slices of Wp, 3 x KC x ProjShape<32>::B_BYTES (16-row chunks)
    float* binv = nullptr;         // their scales, 3 x KG x 32 (96-row groups)
    int* err = nullptr;
};

template <int RP>
rs_status launch_project_core(cudaStream_t st, int n, double b, double h, int N, int Rl,
                              const double* xyz, const double* q, const double* tl,
                              const double* al, const int* perm, const float2* Wp2, float2* Cp2, double* Bp,
                              int nchunk, int CH, double proj_points, const ProjTc& tcp) {
    dim3 gp((N + 127) / 128, Rl, 3);
    if (tcp.use) {
        constexpr int NP = RP <= 16 ? 16 : 32;
        const int KC = (n + kPK - 1) / kPK, KG = (KC + kPG - 1) / kPG;
        {
            ::rs::KernelTimer kt__("k_slice_wp", st, 0.0, false);
            k_slice_wp<NP><<<dim3(KC, 3), NP, 0, st>>>(n, RP, KC, KG, Wp2, tcp.Bs, tcp.binv);
        }
        auto kern = k_project_tc<RP, NP>;
        RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ProjShape<NP>::SMEM));
        // the projection's algorithmic flops: one product and one sum per (row, column, a)
        ::rs::KernelTimer kt__("k_project_tc", st, 2.0 * RP * proj_points, true);
        kern<<<gp, 160, ProjShape<NP>::SMEM, st>>>(n, b, h, N, Rl, KC, KG, xyz, tl, perm, tcp.etab, tcp.Bs,
                                                  tcp.binv, Cp2, tcp.err);
    } else {
        // FP32 pipe ops per active (row, atom, term): two pair products (9 each) and RP
        // Dot2 steps (13 each)
        const double work = proj_points * (18.0 + 13.0 * RP);
        ::rs::KernelTimer kt__("k_project", st, work, true);
        k_project<RP><<<gp, 128, 0, st>>>(n, b, h, N, Rl, xyz, tl, perm, Wp2, Cp2);
    }
    double work;
    // FP32 pipe ops per column and (a, b): two pair products (9 each) and RP Dot2 steps
    work = (double)N * Rl * RP * RP * (18.0 + 13.0 * RP);
    RS_TRY_CUDA(cudaGetLastError());
    {
        ::rs::KernelTimer kt__("k_core", st, work, true);
        k_core<RP><<<nchunk, RP * RP, 0, st>>>(N * Rl, Rl, CH, q, al, Cp2, Bp);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

rs_status dispatch_project_core(int RP, cudaStream_t st, int n, double b, double h, int N, int Rl,
                                const double* xyz, const double* q, const double* tl,
                                const double* al, const int* perm, const float2* Wp2, float2* Cp2, double* Bp,
                                int nchunk, int CH, double proj_points, const ProjTc& tcp) {
    switch (RP) {
#define RS_CASE(R)                                                                                       \
    case R:                                                                                              \
        return launch_project_core<R>(st, n, b, h, N, Rl, xyz, q, tl, al, perm, Wp2, Cp2, Bp, nchunk, CH, \
                                      proj_points, tcp);
        RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        default:
            set_error("unsupported padded Tucker rank %d", RP);
            return RS_ERR_UNSUPPORTED;
    }
}

}  // namespace

// ------------------------------------------------------------------ build steps
static rs_status build_cells(rs_protein* P, cudaStream_t st, const double* d_xyz,
                             const double* d_q, const std::vector<double>& hxyz, Scratch& S) {
    const int N = P->N;
    // bounding box of the charges (min and max are exact: the same on host and device)
    double bb[6] = {hxyz[0], hxyz[1], hxyz[2], hxyz[0], hxyz[1], hxyz[2]};
    for (int i = 1; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            bb[a] = std::min(bb[a], hxyz[3 * (size_t)i + a]);
            bb[3 + a] = std::max(bb[3 + a], hxyz[3 * (size_t)i + a]);
        }
    double cell = std::max(P->table.r_c, P->sigma) * (1.0 + 1e-4) + 1e-4;
    int nc[3];
    double co[3];
    size_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        co[a] = bb[a] - cell;
        nc[a] = (int)std::floor((bb[3 + a] - co[a]) / cell) + 2;
        ncell *= (size_t)nc[a];
    }
    if (ncell > (size_t)1 << 26) {
        set_error("protein extent needs %zu cells (max 2^26)", ncell);
        return RS_ERR_UNSUPPORTED;
    }
    int *d_cell_of, *d_count, *d_cursor, *d_perm, *d_start;
    RS_TRY(S.get(&d_cell_of, N));
    RS_TRY(S.get(&d_count, ncell));
    RS_TRY(S.get(&d_cursor, ncell));
    RS_TRY(S.get(&d_perm, N));
    RS_TRY(S.get(&d_start, ncell + 1));
    float4 *d_atoms, *d_atoms_lo;
    double4* d_atoms64;
    {
        DeviceArena ar;
        ar.add(&d_atoms, N);
        ar.add(&d_atoms_lo, N);
        ar.add(&d_atoms64, N);
        RS_TRY(ar.alloc(P));
    }
    RS_TRY_CUDA(cudaMemsetAsync(d_count, 0, ncell * sizeof(int), st));
    RS_TRY_CUDA(cudaMemsetAsync(d_cursor, 0, ncell * sizeof(int), st));
    {
        ::rs::KernelTimer kt__("k_cell_count", st, 0.0, false);
        k_cell_count<<<blocks_for(N), kBlock, 0, st>>>(N, d_xyz, co[0], co[1], co[2], 1.0 / cell, nc[0],
                                                       nc[1], nc[2], d_cell_of, d_count);
    }
    {
        ::rs::KernelTimer kt__("k_scan", st, 0.0, false);
        k_scan<<<1, 1024, 0, st>>>((int)ncell, d_count, d_start);
    }
    {
        ::rs::KernelTimer kt__("k_cell_fill", st, 0.0, false);
        k_cell_fill<<<blocks_for(N), kBlock, 0, st>>>(N, d_cell_of, d_start, d_cursor, d_perm);
    }
    {
        ::rs::KernelTimer kt__("k_cell_sort", st, 0.0, false);
        k_cell_sort<<<blocks_for(ncell), kBlock, 0, st>>>((int)ncell, d_start, d_perm, d_xyz, d_q,
                                                          d_atoms, d_atoms_lo, d_atoms64);
    }
    RS_TRY_CUDA(cudaGetLastError());
    // candidate lists on fine cells of side R/2 over the box grown by R (the radius
    // with a margin for the FP32 cell lookup of a query and the screen's bands)
    const double R = std::max(P->table.r_c, P->sigma) * (1.0 + 1e-4) + 1e-3;
    const double f = 0.5 * R;
    int nf[3];
    double fo[3];
    size_t nfine = 1;
    for (int a = 0; a < 3; ++a) {
        fo[a] = bb[a] - R;
        nf[a] = (int)std::floor((bb[3 + a] + R - fo[a]) / f) + 1;
        nfine *= (size_t)nf[a];
    }
    if (nfine > (size_t)1 << 26) {
        set_error("protein extent needs %zu candidate-list cells (max 2^26)", nfine);
        return RS_ERR_UNSUPPORTED;
    }
    int *d_nb_count, *d_nb_start;
    RS_TRY(S.get(&d_nb_count, nfine));
    RS_TRY(device_alloc(P, (void**)&d_nb_start, (nfine + 1) * sizeof(int)));
    {
        ::rs::KernelTimer kt__("k_nb_lists", st, 0.0, false);
        k_nb_lists<<<blocks_for(nfine * 32), kBlock, 0, st>>>(0, nf[0], nf[1], nf[2], fo[0], fo[1], fo[2], f,
                                                             nc[0], nc[1], nc[2], co[0], co[1], co[2], cell, R,
                                                             d_start, d_atoms, d_nb_count, nullptr, nullptr,
                                                             nullptr);
    }
    {
        ::rs::KernelTimer kt__("k_scan", st, 0.0, false);
        k_scan<<<1, 1024, 0, st>>>((int)nfine, d_nb_count, d_nb_start);
    }
    int total = 0;
    RS_TRY_CUDA(cudaMemcpyAsync(&total, d_nb_start + nfine, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_TRY_CUDA(cudaStreamSynchronize(st));
    float4* d_nb_atoms;
    int* d_nb_idx;
    {
        DeviceArena ar;
        ar.add(&d_nb_atoms, std::max(total, 1));
        ar.add(&d_nb_idx, std::max(total, 1));
        RS_TRY(ar.alloc(P));
    }
    {
        ::rs::KernelTimer kt__("k_nb_lists", st, 0.0, false);
        k_nb_lists<<<blocks_for(nfine * 32), kBlock, 0, st>>>(1, nf[0], nf[1], nf[2], fo[0], fo[1], fo[2], f,
                                                             nc[0], nc[1], nc[2], co[0], co[1], co[2], cell, R,
                                                             d_start, d_atoms, nullptr, d_nb_start, d_nb_atoms,
                                                             d_nb_idx);
    }
    RS_TRY_CUDA(cudaGetLastError());
    ProteinView& v = P->view;
    v.atoms = d_atoms;
    v.atoms_lo = d_atoms_lo;
    v.atoms64 = d_atoms64;
    v.nb_start = d_nb_start;
    v.nb_atoms = d_nb_atoms;
    v.nb_idx = d_nb_idx;
    v.nf0 = nf[0];
    v.nf1 = nf[1];
    v.nf2 = nf[2];
    v.fo0 = (float)fo[0];
    v.fo1 = (float)fo[1];
    v.fo2 = (float)fo[2];
    v.inv_fine = (float)(1.0 / f);
    return RS_OK;
}

static rs_status build_canonical(rs_protein* P, cudaStream_t st, const double* d_xyz,
                                 const double* d_q, const double* d_tl, const double* d_al, int galerkin) {
    const int N = P->N, Rl = P->R_l, n = P->n;
    size_t R = (size_t)N * Rl;
    size_t ld = (R + 127) / 128 * 128;
    if (ld > (size_t)1 << 30 || (double)ld * n * 12.0 > 64e9) {
        set_error("unreduced canonical factors need %.1f GB; use tucker_cap", ld * n * 12.0 / 1e9);
        return RS_ERR_UNSUPPORTED;
    }
    float* F[3];
    for (int a = 0; a < 3; ++a) RS_TRY(device_alloc(P, (void**)&F[a], (size_t)n * ld * sizeof(float)));
    dim3 g(blocks_for(ld), n);
    double work = (double)n * ld * 3 * sizeof(float);  // bytes written
    {
        ::rs::KernelTimer kt__("k_canon_factors", st, work, true);
        k_canon_factors<<<g, kBlock, 0, st>>>(n, P->b, P->h, N, Rl, d_xyz, d_q, d_tl, d_al, (int)ld,
                                             F[0], F[1], F[2], galerkin);
    }
    RS_TRY_CUDA(cudaGetLastError());
    ProteinView& v = P->view;
    v.kind = 0;
    v.ld = (int)ld;
    v.R = (int)ld;
    for (int a = 0; a < 3; ++a) v.F[a] = F[a];
    v.core = nullptr;
    P->kind = 0;
    for (int a = 0; a < 3; ++a) P->rank[a] = (int)R;
    return RS_OK;
}

// The short-range terms of the protein's sinc table, the tabulated short-range sum
// (cubic Hermite) and the decision bands of the vdW check, into P->view.
static rs_status finish_short_range(rs_protein* P, cudaStream_t st) {
    ProteinView& v = P->view;
    v.n = P->n;
    v.b = P->b;
    v.h = P->h;
    v.inv_h = 1.0 / P->h;
    v.Ks = 0;
    for (int k = 0; k < P->K; ++k)
        if (!P->table.is_long[k]) {
            v.ts2[v.Ks] = P->table.t[k] * P->table.t[k];
            v.as[v.Ks] = P->table.a[k];
            ++v.Ks;
        }
    double rc = P->table.r_c;
    v.rc2 = rc * rc;
    v.rc2_hi = (float)(rc * rc * (1.0 + 1e-4));
    v.stab2 = nullptr;
    v.stab_n = 0;
    v.stab_inv_h = 0.0;
    if (v.Ks > 0 && rc > 0) {
        // spacing from the cubic Hermite bound |f - p| <= hs^4/384 max|f''''| with
        // max|f''''| <= sum a_k t_k^8 (at s = 0), for 1e-10 relative to f(0)
        double f0 = 0.0, f4 = 0.0;
        for (int q = 0; q < v.Ks; ++q) {
            f0 += v.as[q];
            f4 += v.as[q] * std::pow(v.ts2[q], 4.0);
        }
        double hs = std::pow(384.0 * 1e-10 * f0 / std::max(f4, 1e-300), 0.25);
        double smax = (double)v.rc2_hi * (1.0 + 1e-6);
        int M = (int)std::ceil(smax / hs) + 2;
        if (M > (1 << 22)) {
            set_error("short-range table of %d entries is too large", M);
            return RS_ERR_UNSUPPORTED;
        }
        float4* tab = nullptr;
        RS_TRY(device_alloc(P, (void**)&tab, (size_t)2 * (M - 1) * sizeof(float4)));
        {
            ::rs::KernelTimer kt__("k_short_table", st, 0.0, false);
            k_short_table<<<blocks_for((size_t)M), kBlock, 0, st>>>(v, M, hs, tab);
        }
        RS_TRY_CUDA(cudaGetLastError());
        v.stab2 = tab;
        v.stab_n = M;
        v.stab_inv_h = 1.0 / hs;
        split_host(v.stab_inv_h, v.stab_ih_h, v.stab_ih_l);
    }
    v.sig2 = P->sigma * P->sigma;
    v.sig2_lo = (float)(v.sig2 * (1.0 - 1e-4));
    v.sig2_hi = (float)(v.sig2 * (1.0 + 1e-4));
    split_host(v.sig2, v.sig2_ph, v.sig2_pl);
    split_host(v.rc2, v.rc2_ph, v.rc2_pl);
    split_host(v.b, v.b_h, v.b_l);
    split_host(v.inv_h, v.inv_h_h, v.inv_h_l);
    return RS_OK;
}

// Cardinal (skeleton) basis of the Tucker factors V (3 x n x RP, FP64, columns >= r_ax
// zero): pivoted Gram-Schmidt picks r rows S per axis (k_skeleton), Vs = V V[S,:]^-1
// and Wp = V V[S,:]^T (k_skeleton_apply).  d_M, d_Ainv, d_S, d_Wp: scratch of
// 3 n RP, 3 RP^2, 3 RS_MAX_TUCKER and 3 n RP; *d_Vs is taken from S.
static rs_status skeleton_basis(cudaStream_t st, int n, int RP, const int* d_rax, const double* d_V, double* d_M,
                                double* d_Ainv, int* d_S, float2* d_Wp, int* d_fail, Scratch& S, double** d_Vs) {
    {
        // the residual rows in shared memory when they fit beside the kernel's static arrays
        const size_t rows_bytes = (size_t)n * RP * sizeof(float);
        const bool rows_smem = rows_bytes <= 192 * 1024;
        if (rows_smem)
            RS_TRY_CUDA(cudaFuncSetAttribute(k_skeleton, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_bytes));
        ::rs::KernelTimer kt__("k_skeleton", st, 0.0, false);
        k_skeleton<<<3, 512, rows_smem ? rows_bytes : 0, st>>>(n, RP, d_rax, d_V, d_M, d_S, d_Ainv, d_fail,
                                                               rows_smem);
    }
    RS_TRY(S.get(d_Vs, (size_t)3 * n * RP));
    {
        ::rs::KernelTimer kt__("k_skeleton_apply", st, 0.0, false);
        k_skeleton_apply<<<dim3(blocks_for((size_t)n * RP), 3), kBlock, 0, st>>>(
            n, RP, d_rax, d_V, d_Ainv, d_S, *d_Vs, d_Wp);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

// The evaluation tables of a Tucker handle from its cardinal factors Vs (3 x n x RP)
// and core beta' (RP^3), both FP64 on the device: float-pair rows of V1', V2', the
// W form W = V3' beta'_(3)^T with its tensor-core B image, the core in FP32, and FP64
// copies of Vs and beta' kept with the handle (for add-and-compress).  Checks the
// skeleton's failure flags (one stream synchronisation) and sets P->view.
static rs_status tucker_tables(rs_protein* P, cudaStream_t st, int n, int RP, const double* d_Vs, const double* d_B,
                               const int* d_fail) {
    const size_t blen = (size_t)RP * RP * RP;
    float *core, *vt0, *vt1, *wt, *wsc;
    uint16_t* wtc;
    double *fac64, *core64;
    size_t vplane = (size_t)n * RP, wplane = (size_t)n * RP * RP;
    {
        DeviceArena ar;
        ar.add(&core, blen);
        ar.add(&vt0, 4 * vplane);
        ar.add(&vt1, 4 * vplane);
        ar.add(&wt, 4 * wplane);
        ar.add(&wtc, tc_bimage_bytes(n, RP) / sizeof(uint16_t));
        ar.add(&wsc, tc_bscale_bytes(n, RP) / sizeof(float));
        ar.add(&fac64, 3 * vplane);
        ar.add(&core64, blen);
        RS_TRY(ar.alloc(P));
    }
    {
        ::rs::KernelTimer kt__("k_to_float", st, 0.0, false);
        k_to_float<<<blocks_for(blen), kBlock, 0, st>>>(blen, d_B, core);
    }
    RS_TRY_CUDA(cudaGetLastError());
    RS_TRY_CUDA(cudaMemcpyAsync(fac64, d_Vs, 3 * vplane * sizeof(double), cudaMemcpyDeviceToDevice, st));
    RS_TRY_CUDA(cudaMemcpyAsync(core64, d_B, blen * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int fail[3];
    RS_TRY_CUDA(cudaMemcpyAsync(fail, d_fail, sizeof(fail), cudaMemcpyDeviceToHost, st));
    RS_TRY_CUDA(cudaStreamSynchronize(st));
    if (fail[0] || fail[1] || fail[2]) {
        set_error("skeleton selection failed (rank-deficient factor basis)");
        return RS_ERR_CUDA;
    }
    // evaluation tables: float-pair rows of V1', V2' and of W = V3' core_(3)^T
    {
        ::rs::KernelTimer kt__("k_pair_rows", st, 0.0, false);
        k_pair_rows<<<dim3(blocks_for(vplane), 2), kBlock, 0, st>>>(n, RP, d_Vs, vt0, vt1);
    }
    {
        ::rs::KernelTimer kt__("k_wtable", st, 0.0, false);
        k_wtable<<<dim3(blocks_for((size_t)RP * RP), n), kBlock, 0, st>>>(n, RP, d_Vs + 2 * vplane, d_B, wt);
    }
    RS_TRY_CUDA(cudaGetLastError());
    RS_TRY(tc_build_bimage(n, RP, wt, wtc, wsc, st));
    RS_TRY_CUDA(cudaStreamSynchronize(st));
    ProteinView& v = P->view;
    v.kind = 1;
    v.Wtc = wtc;
    v.Wsc = wsc;
    v.ld = RP;
    v.R = RP;
    for (int a = 0; a < 3; ++a) v.F[a] = nullptr;
    for (int k = 0; k < 4; ++k) {
        v.Wt[k] = wt + k * wplane;
        v.Vt[0][k] = vt0 + k * vplane;
        v.Vt[1][k] = vt1 + k * vplane;
    }
    v.core = core;
    P->fac64 = fac64;
    P->core64 = core64;
    P->kind = 1;
    return RS_OK;
}

static rs_status build_tucker(rs_protein* P, cudaStream_t st, const double* d_xyz,
                              const double* d_q, const double* d_tl, const double* d_al,
                              const std::vector<double>& tl_host, const std::vector<double>& al_host,
                              const std::vector<double>& q_host_abs23,
                              const std::vector<double>& xyz_host, int cap, double eps_r,
                              Scratch& S) {
    const int N = P->N, Rl = P->R_l, n = P->n;
    const double b = P->b, h = P->h;
    if (cap > RS_MAX_TUCKER) {
        set_error("tucker_cap %d exceeds %d", cap, RS_MAX_TUCKER);
        return RS_ERR_INVALID;
    }
    const int Sh = 2 * n - 1;
    // 1. Gram matrices
    double *d_cz, *d_w2, *d_Dp, *d_D, *d_tr;
    float2 *d_WE, *d_D2;
    float2* d_G;
    RS_TRY(S.get(&d_cz, N));
    RS_TRY(S.get(&d_w2, Rl));
    RS_TRY_CUDA(cudaMemcpyAsync(d_cz, q_host_abs23.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
    std::vector<double> w2(Rl);
    for (int k = 0; k < Rl; ++k) w2[k] = std::pow(std::fabs(al_host[k]), 2.0 / 3.0);
    RS_TRY_CUDA(cudaMemcpyAsync(d_w2, w2.data(), Rl * sizeof(double), cudaMemcpyHostToDevice, st));
    int nsc = (Sh + kSC - 1) / kSC;
    int nmc = (N + kMC - 1) / kMC;
    RS_TRY(S.get(&d_Dp, (size_t)nmc * 3 * Rl * Sh));
    RS_TRY(S.get(&d_D, (size_t)3 * Rl * Sh));
    RS_TRY(S.get(&d_WE, (size_t)Rl * n));
    RS_TRY(S.get(&d_D2, (size_t)3 * Rl * Sh));
    RS_TRY(S.get(&d_G, (size_t)3 * n * n));
    RS_TRY(S.get(&d_tr, 3));
    long long threads = (long long)nsc * Rl * 3 * nmc;
    double work = 0.0;
    float4* d_pk;
    float2* d_etab;
    RS_TRY(S.get(&d_pk, (size_t)3 * N));
    RS_TRY(S.get(&d_etab, 256));
    {
        ::rs::KernelTimer kt__("k_dsum_atoms", st, 0.0, false);
        k_dsum_atoms<<<dim3(blocks_for(N), 3), kBlock, 0, st>>>(N, d_xyz, d_cz, d_pk);
        k_exp2_table<<<1, 256, 0, st>>>(d_etab);
        note_launch(1);
    }
    {
        ::rs::KernelTimer kt__("k_gauss_dsum", st, 0.0, true);
        k_gauss_dsum<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(n, b, h, N, Rl, d_pk, d_tl, d_etab,
                                                                         nsc, nmc, d_Dp);
        // FP32 pipe ops: 26 per half-grid point of the pair walk (two pair products,
        // one pair sum) plus ~200 for the seeds (two pair exponentials, the offsets)
        // of every chunk within e^-50 of a Gaussian's peak (closed form per term;
        // only when timed).
        if (kt__.active()) {
            const double delta = 0.5 * h;
            double w = 0.0;
            for (int k = 0; k < Rl; ++k) {
                double t2 = 2.0 * tl_host[k] * tl_host[k];
                double reach = t2 > 0 ? std::sqrt(50.0 / t2) : 1e300;
                for (size_t e = 0; e < xyz_host.size(); ++e) {
                    double lo = std::max(0.0, std::floor((xyz_host[e] - reach + b) / delta / kSC));
                    double hi = std::min((double)(nsc - 1), std::floor((xyz_host[e] + reach + b) / delta / kSC));
                    if (hi >= lo) w += (hi - lo + 1) * (kSC * 26.0 + 200.0);
                }
            }
            kt__.set_work(w);
        }
    }
    RS_TRY_CUDA(cudaGetLastError());
    size_t dlen = (size_t)3 * Rl * Sh;
    {
        ::rs::KernelTimer kt__("k_sum_chunks", st, 0.0, false);
        k_sum_chunks<<<blocks_for(dlen), kBlock, 0, st>>>(dlen, nmc, d_Dp, d_D, d_D2);
    }
    {
        ::rs::KernelTimer kt__("k_exp_table", st, 0.0, false);
        k_exp_table<<<dim3(blocks_for(n), Rl), kBlock, 0, st>>>(n, h, Rl, d_tl, d_w2, d_WE);
    }
    work = 3.0 * n * (double)n * Rl * 8.0;  // FP32 pipe ops (one Dot2 step per term)
    {
        ::rs::KernelTimer kt__("k_gram", st, work, true);
        k_gram<<<dim3(blocks_for(n), n, 3), kBlock, 0, st>>>(n, Rl, d_WE, d_D2, d_G);
    }
    {
        ::rs::KernelTimer kt__("k_trace", st, 0.0, false);
        k_trace<<<3, kBlock, 0, st>>>(n, d_G, d_tr);
    }
    RS_TRY_CUDA(cudaGetLastError());

    // 2. block subspace iteration with CholQR2 and Rayleigh-Ritz
    int p = std::min(n, cap + 12);
    p = std::min(48, (p + 1) / 2 * 2);
    if (p > n) p = n - (n % 2);
    if (p < cap) {
        set_error("grid too small for tucker_cap %d (n=%d)", cap, n);
        return RS_ERR_UNSUPPORTED;
    }
    // G Q on the tensor cores for block sizes that are multiples of 16 (the MMA's N)
    const int p16 = (p + 15) / 16 * 16;
    const bool use_tc = build_gemm_mode() == 1 && n <= kTcGemmMaxN && p16 <= std::min(48, n);
    if (use_tc) p = p16;
    const int MT = (n + tcg::kM - 1) / tcg::kM, KC = (n + tcg::kK - 1) / tcg::kK;
    uint8_t *d_As = nullptr, *d_Bs = nullptr;
    float *d_ainv = nullptr, *d_binv = nullptr;
    int* d_tcerr = nullptr;
    if (use_tc) {
        int dev = 0;
        RS_TRY_CUDA(cudaGetDevice(&dev));
        d_tcerr = tc_error_flag(dev);
        if (!d_tcerr) {
            set_error("tensor-core build GEMM: no error flag on device %d", dev);
            return RS_ERR_CUDA;
        }
        RS_TRY(S.get(&d_As, (size_t)3 * MT * KC * tcg::kS * tcg::kSliceA));
        RS_TRY(S.get(&d_ainv, (size_t)3 * KC * MT * tcg::kM));
        RS_TRY(S.get(&d_Bs, (size_t)3 * KC * tcg::kS * p * tcg::kK * 2));
        RS_TRY(S.get(&d_binv, (size_t)3 * KC * p));
        {
            ::rs::KernelTimer kt__("k_slice_rows", st, 0.0, false);
            tcg::k_slice_rows<<<dim3(MT, KC, 3), tcg::kM, 0, st>>>(n, MT, KC, d_G, d_As, d_ainv);
        }
        RS_TRY_CUDA(cudaGetLastError());
    }
    const int nks = use_tc ? KC : kGemmKS;
    double *d_Q, *d_Y, *d_Sm, *d_Ri, *d_W;
    int* d_fail;
    RS_TRY(S.get(&d_Q, (size_t)3 * n * p));
    RS_TRY(S.get(&d_Y, (size_t)3 * n * p));
    RS_TRY(S.get(&d_Sm, (size_t)3 * p * p));
    RS_TRY(S.get(&d_Ri, (size_t)3 * p * p));
    RS_TRY(S.get(&d_W, (size_t)3 * p * p));
    float2* d_Q2;  // Q as float pairs, the operand of the pair GEMM
    RS_TRY(S.get(&d_Q2, (size_t)3 * n * p));
    RS_TRY(S.get(&d_fail, 3));
    RS_TRY_CUDA(cudaMemsetAsync(d_fail, 0, 3 * sizeof(int), st));
    {
        ::rs::KernelTimer kt__("k_init_block", st, 0.0, false);
        k_init_block<<<blocks_for((size_t)3 * n * p), kBlock, 0, st>>>(n, p, d_Q, d_Q2);
    }
    dim3 gq((n + kGemmRows - 1) / kGemmRows, kGemmKS, 3);
    const int nblk = (n + 15) / 16;
    double *d_Sp, *d_Yp = nullptr;
    float2* d_Yp2 = nullptr;
    RS_TRY(S.get(&d_Sp, (size_t)3 * nblk * p * p));
    if (use_tc) RS_TRY(S.get(&d_Yp2, (size_t)nks * 3 * n * p));
    else RS_TRY(S.get(&d_Yp, (size_t)nks * 3 * n * p));
    // CholQR2 of Yin (d_Q or d_Y): shifted CholQR then plain CholQR; every pass reads
    // one buffer and writes the other, and the result ends in d_Q.
    auto cholqr_pass = [&](const double* src, double* dst, double shift) -> rs_status {
        {
            ::rs::KernelTimer kt__("k_atb", st, 0.0, false);
            k_atb<<<dim3(nblk, 3), 256, 0, st>>>(n, p, src, src, d_Sp);
        }
        {
            ::rs::KernelTimer kt__("k_sum_gram", st, 0.0, false);
            k_sum_gram<<<dim3((p * p + 31) / 32, 3), 32 * kSumGramWarps, 0, st>>>(nblk, p, d_Sp, d_Sm);
        }
        {
            ::rs::KernelTimer kt__("k_chol", st, 0.0, false);
            launch_chol(p, d_Sm, shift, d_Ri, d_fail, st);
        }
        {
            ::rs::KernelTimer kt__("k_apply_rinv", st, 0.0, false);
            k_apply_rinv<<<dim3(blocks_for((size_t)n * p), 3), kBlock, 0, st>>>(
                n, p, src, d_Ri, dst, dst == d_Q ? d_Q2 : nullptr);
        }
        RS_TRY_CUDA(cudaGetLastError());
        return RS_OK;
    };
    auto orthonormalize = [&](double* Yin) -> rs_status {
        double* other = (Yin == d_Q) ? d_Y : d_Q;
        RS_TRY(cholqr_pass(Yin, other, 1e-13));
        RS_TRY(cholqr_pass(other, Yin, 0.0));
        if (Yin != d_Q)
            RS_TRY_CUDA(cudaMemcpyAsync(d_Q, Yin, (size_t)3 * n * p * sizeof(double),
                                        cudaMemcpyDeviceToDevice, st));
        return RS_OK;
    };
    work = 3.0 * 13.0 * n * (double)n * p;  // FP32 pipe ops per G Q (one Dot2 step per product)
    // Y partials of G Q per K slice into d_Yp: float-pair GEMM, or slices of Q and the
    // tensor-core GEMM
    auto gemm_gq = [&]() -> rs_status {
        if (!use_tc) {
            ::rs::KernelTimer kt__("k_gemm_gq", st, work, true);
            k_gemm_gq<<<gq, 256, 0, st>>>(n, p, d_G, d_Q2, d_Yp);
        } else {
            // BF16 MMA flops of the 21 slice products
            const double tflops = 2.0 * 21.0 * 3.0 * (double)MT * tcg::kM * (double)KC * tcg::kK * p;
            switch (p) {
#define RS_GQ_CASE(NP)                                                                                    \
    case NP: {                                                                                            \
        {                                                                                                 \
            ::rs::KernelTimer kt__("k_slice_cols", st, 0.0, false);                                       \
            tcg::k_slice_cols<NP><<<dim3(KC, 3), NP, 0, st>>>(n, KC, d_Q2, d_Bs, d_binv);                 \
        }                                                                                                 \
        RS_TRY_CUDA(cudaFuncSetAttribute(tcg::k_tc_gemm<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)tcg::GemmShape<NP>::SMEM));                                 \
        ::rs::KernelTimer kt__("k_tc_gemm", st, tflops, true);                                            \
        tcg::k_tc_gemm<NP><<<dim3(MT, KC, 3), tcg::kGemmThreads, tcg::GemmShape<NP>::SMEM, st>>>(         \
            n, MT, KC, d_As, d_ainv, d_Bs, d_binv, d_Yp2, d_tcerr);                                       \
        break;                                                                                            \
    }
                RS_GQ_CASE(16) RS_GQ_CASE(32) RS_GQ_CASE(48)
#undef RS_GQ_CASE
                default:
                    set_error("tensor-core build GEMM: block size %d", p);
                    return RS_ERR_UNSUPPORTED;
            }
        }
        RS_TRY_CUDA(cudaGetLastError());
        return RS_OK;
    };
    // one subspace step: Y = G Q with partial Grams, S = Y^T Y, shifted Cholesky, Q = Y R^-1
    auto step = [&]() -> rs_status {
        RS_TRY(gemm_gq());
        {
            ::rs::KernelTimer kt__("k_gemm_reduce", st, 0.0, false);
            k_gemm_reduce<<<dim3(nblk, 3), 256, 0, st>>>(n, p, nks, d_Yp, d_Yp2, d_Y, d_Sp);
        }
        {
            ::rs::KernelTimer kt__("k_sum_gram", st, 0.0, false);
            k_sum_gram<<<dim3((p * p + 31) / 32, 3), 32 * kSumGramWarps, 0, st>>>(nblk, p, d_Sp, d_Sm);
        }
        {
            ::rs::KernelTimer kt__("k_chol", st, 0.0, false);
            launch_chol(p, d_Sm, 1e-13, d_Ri, d_fail, st);
        }
        {
            ::rs::KernelTimer kt__("k_apply_rinv", st, 0.0, false);
            k_apply_rinv<<<dim3(blocks_for((size_t)n * p), 3), kBlock, 0, st>>>(n, p, d_Y, d_Ri, d_Q, d_Q2);
        }
        RS_TRY_CUDA(cudaGetLastError());
        return RS_OK;
    };
    // host copies of the Rayleigh-Ritz matrices and eigenvectors (alive for the whole
    // build, so the copy of the eigenvectors needs no wait)
    std::vector<double> H((size_t)3 * p * p), Wh((size_t)3 * p * p);
    // one Rayleigh-Ritz step; fail_out (if not null) gets the orthonormalisation flags
    // and tr_out the Gram traces in the same device round trip
    auto ritz = [&](std::vector<double>& lam_out, int* fail_out, double* tr_out) -> rs_status {
        RS_TRY(orthonormalize(d_Q));
        RS_TRY(gemm_gq());
        {
            ::rs::KernelTimer kt__("k_gemm_reduce", st, 0.0, false);
            k_gemm_reduce<<<dim3(nblk, 3), 256, 0, st>>>(n, p, nks, d_Yp, d_Yp2, d_Y, nullptr);
        }
        {
            ::rs::KernelTimer kt__("k_atb", st, 0.0, false);
            k_atb<<<dim3(nblk, 3), 256, 0, st>>>(n, p, d_Q, d_Y, d_Sp);
        }
        {
            ::rs::KernelTimer kt__("k_sum_gram", st, 0.0, false);
            k_sum_gram<<<dim3((p * p + 31) / 32, 3), 32 * kSumGramWarps, 0, st>>>(nblk, p, d_Sp, d_Sm);
        }
        RS_TRY_CUDA(cudaGetLastError());
        // p x p eigenproblems on the host (FP64): a few microseconds each
        RS_TRY_CUDA(cudaMemcpyAsync(H.data(), d_Sm, H.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (fail_out) RS_TRY_CUDA(cudaMemcpyAsync(fail_out, d_fail, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (tr_out) RS_TRY_CUDA(cudaMemcpyAsync(tr_out, d_tr, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaStreamSynchronize(st));
        lam_out.resize((size_t)3 * p);
        for (int a = 0; a < 3; ++a)
            if (!symeig_host(p, H.data() + (size_t)a * p * p, lam_out.data() + (size_t)a * p,
                             Wh.data() + (size_t)a * p * p)) {
                set_error("Rayleigh-Ritz eigen-decomposition did not converge");
                return RS_ERR_CUDA;
            }
        RS_TRY_CUDA(cudaMemcpyAsync(d_W, Wh.data(), Wh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        return RS_OK;
    };
    // Subspace iteration converges like (lambda_{p+1} / lambda_r)^T.  After a few
    // steps the Ritz values estimate that ratio (lambda_p / lambda_r as a safe
    // proxy); the remaining steps bring the subspace error below 1e-12 (the energies
    // carry it amplified by the Tucker sum's cancellation, ~1e3: far below 1e-5).
    const int warm = 6;
    for (int it = 0; it < warm; ++it) RS_TRY(step());
    std::vector<double> lam_est;
    RS_TRY(ritz(lam_est, nullptr, nullptr));
    int more = 0;
    for (int a = 0; a < 3; ++a) {
        const double* la = lam_est.data() + (size_t)a * p;
        int r = std::min(cap, p - 1);
        double ratio = (la[r - 1] > 0 && la[p - 1] > 0) ? la[p - 1] / la[r - 1] : 0.5;
        ratio = std::min(std::max(ratio, 1e-8), 0.95);
        int need = (int)std::ceil(std::log(1e-12) / std::log(ratio)) - warm + 2;
        more = std::max(more, need);
    }
    more = std::min(std::max(more, 2), 60);
    for (int it = 0; it < more; ++it) RS_TRY(step());
    P->subspace_steps = warm + more;
    std::vector<double> lam, tr(3);
    int fail[3];
    RS_TRY(ritz(lam, fail, tr.data()));
    if (fail[0] || fail[1] || fail[2]) {
        set_error("orthonormalisation failed in the subspace iteration");
        return RS_ERR_CUDA;
    }
    int r_ax[3];
    int rmax = 0;
    for (int a = 0; a < 3; ++a) {
        const double* la = lam.data() + (size_t)a * p;
        double s1 = std::sqrt(std::max(la[0], 0.0));
        int r = 0;
        for (int i = 0; i < p; ++i)
            if (std::sqrt(std::max(la[i], 0.0)) > eps_r * s1) ++r;
        r = std::min(r, cap);
        r = std::max(r, 1);
        r_ax[a] = r;
        rmax = std::max(rmax, r);
        double head = 0.0;
        for (int i = 0; i < r; ++i) head += la[i];
        P->sv_tail[a] = std::sqrt(std::max(tr[a] - head, 0.0) / std::max(la[0], 1e-300));
        P->sv_gap[a] = (r < p && la[r] > 0) ? std::sqrt(la[r - 1] / la[r]) : 0.0;
        P->rank[a] = r;
    }
    const int RP = (rmax + 3) / 4 * 4;
    int* d_rax;
    double *d_V, *d_M, *d_Ainv;
    float2* d_Wp;
    int* d_S;
    RS_TRY(S.get(&d_rax, 3));
    RS_TRY_CUDA(cudaMemcpyAsync(d_rax, r_ax, sizeof(r_ax), cudaMemcpyHostToDevice, st));
    RS_TRY(S.get(&d_V, (size_t)3 * n * RP));
    RS_TRY(S.get(&d_M, (size_t)3 * n * RP));
    RS_TRY(S.get(&d_Ainv, (size_t)3 * RP * RP));
    RS_TRY(S.get(&d_Wp, (size_t)3 * n * RP));
    RS_TRY(S.get(&d_S, (size_t)3 * RS_MAX_TUCKER));
    {
        ::rs::KernelTimer kt__("k_ritz_vectors", st, 0.0, false);
        k_ritz_vectors<<<dim3(blocks_for((size_t)n * RP), 3), kBlock, 0, st>>>(n, p, RP, d_rax, d_Q, d_W, d_V);
    }
    // 3. skeleton basis
    double* d_Vs;
    RS_TRY(skeleton_basis(st, n, RP, d_rax, d_V, d_M, d_Ainv, d_S, d_Wp, d_fail, S, &d_Vs));
    // 4. projections and core
    const int Rtot = N * Rl;
    // columns per k_core CTA: about 152 CTAs (one wave of one CTA per SM on GB300; the
    // accumulators of a thread stay in registers), a multiple of the 32-column tile;
    // a function of the problem only, so the partial cores' order is fixed
    const int CH = ((Rtot + 151) / 152 + 31) / 32 * 32;
    const int nchunk = (Rtot + CH - 1) / CH;
    double *d_Bp, *d_B;
    float2* d_Cp;
    RS_TRY(S.get(&d_Cp, (size_t)3 * RP * Rtot));
    RS_TRY(S.get(&d_Bp, (size_t)nchunk * RP * RP * RP));
    RS_TRY(S.get(&d_B, (size_t)RP * RP * RP));
    double proj_points = 0.0;
    if (timing_mode() > 0) {
        for (int k = 0; k < Rl; ++k) {
            double t2 = tl_host[k] * tl_host[k];
            double hw = t2 > 0 ? std::sqrt(46.0 / t2) : 1e300;
            for (size_t e = 0; e < xyz_host.size(); ++e) {
                double lo = std::max(0.0, std::ceil((xyz_host[e] - hw + b) / h));
                double hi = std::min((double)(n - 1), std::floor((xyz_host[e] + hw + b) / h));
                if (hi >= lo) proj_points += hi - lo + 1;
            }
        }
    }
    int *d_row_of, *d_acnt, *d_astart, *d_acur, *d_perm;
    RS_TRY(S.get(&d_row_of, (size_t)3 * N));
    RS_TRY(S.get(&d_acnt, (size_t)3 * n));
    RS_TRY(S.get(&d_astart, (size_t)3 * (n + 1)));
    RS_TRY(S.get(&d_acur, (size_t)3 * n));
    RS_TRY(S.get(&d_perm, (size_t)3 * N));
    RS_TRY_CUDA(cudaMemsetAsync(d_acnt, 0, (size_t)3 * n * sizeof(int), st));
    RS_TRY_CUDA(cudaMemsetAsync(d_acur, 0, (size_t)3 * n * sizeof(int), st));
    {
        ::rs::KernelTimer kt__("k_axis_sort", st, 0.0, false);
        k_axis_count<<<dim3(blocks_for(N), 3), kBlock, 0, st>>>(N, d_xyz, b, h, n, d_acnt, d_row_of);
        for (int a = 0; a < 3; ++a)
            k_scan<<<1, 1024, 0, st>>>(n, d_acnt + (size_t)a * n, d_astart + (size_t)a * (n + 1));
        k_axis_fill<<<dim3(blocks_for(N), 3), kBlock, 0, st>>>(N, n, d_row_of, d_astart, d_acur, d_perm);
        note_launch(4);  // the timer counts one of the five launches
    }
    RS_TRY_CUDA(cudaGetLastError());
    ProjTc tcp;
    if (build_gemm_mode() == 1) {
        const int KCp = (n + kPK - 1) / kPK;
        int dev = 0;
        RS_TRY_CUDA(cudaGetDevice(&dev));
        tcp.use = true;
        tcp.etab = d_etab;
        tcp.err = tc_error_flag(dev);
        if (!tcp.err) {
            set_error("tensor-core projection: no error flag on device %d", dev);
            return RS_ERR_CUDA;
        }
        RS_TRY(S.get(&tcp.Bs, (size_t)3 * KCp * ProjShape<32>::B_BYTES));
        RS_TRY(S.get(&tcp.binv, (size_t)3 * ((KCp + kPG - 1) / kPG) * 32));
    }
    RS_TRY(dispatch_project_core(RP, st, n, b, h, N, Rl, d_xyz, d_q, d_tl, d_al, d_perm, d_Wp, d_Cp, d_Bp,
                                 nchunk, CH, proj_points, tcp));
    size_t blen = (size_t)RP * RP * RP;
    {
        ::rs::KernelTimer kt__("k_sum_chunks", st, 0.0, false);
        k_sum_chunks<<<blocks_for(blen), kBlock, 0, st>>>(blen, nchunk, d_Bp, d_B, nullptr);
    }
    return tucker_tables(P, st, n, RP, d_Vs, d_B, d_fail);
}

}  // namespace rs

extern "C" rs_status rs_diag_pair_exp(int32_t n, const double* x, double* out) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(x && out && n >= 1 && n <= (1 << 24), "rs_diag_pair_exp: bad argument");
    for (int i = 0; i < n; ++i)
        RS_CHECK_ARG(std::fabs(x[i]) <= 80.0, "rs_diag_pair_exp: |x| = %g exceeds 80", std::fabs(x[i]));
    char* buf = nullptr;
    const size_t vb = (size_t)n * sizeof(double);
    RS_TRY_CUDA(cudaMalloc(&buf, 2 * vb + 256 * sizeof(float2) + 512));
    double* d_x = (double*)buf;
    double* d_o = (double*)(buf + vb);
    float2* d_t = (float2*)(buf + 2 * vb + 256);
    rs_status st = RS_OK;
    if (cudaMemcpy(d_x, x, vb, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("rs_diag_pair_exp: copy failed");
        st = RS_ERR_CUDA;
    } else {
        k_exp2_table<<<1, 256>>>(d_t);
        k_diag_pair_exp<<<(n + 255) / 256, 256>>>(n, d_x, d_t, d_o);
        note_launch(2);
        if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(out, d_o, vb, cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("rs_diag_pair_exp: %s", cudaGetErrorString(cudaGetLastError()));
            st = RS_ERR_CUDA;
        }
    }
    cudaFree(buf);
    return st;
}

extern "C" rs_status rs_build_protein(rs_ctx* ctx, int32_t N, const double* xyz, const double* q,
                                      const rs_params* prm, int mem_flags, void* stream,
                                      rs_protein** out) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && xyz && q && prm && out, "rs_build_protein: NULL argument");
    *out = nullptr;
    RS_CHECK_ARG(N >= 1 && N <= (1 << 22), "rs_build_protein: N=%d out of range [1, 2^22]", N);
    RS_CHECK_ARG(prm->n >= 3 && prm->n <= 16385, "rs_build_protein: n=%d out of range [3, 16385]", prm->n);
    RS_CHECK_ARG(prm->b > 0 && prm->sigma > 0, "rs_build_protein: b and sigma must be > 0");
    RS_CHECK_ARG(prm->tucker_cap >= 0, "rs_build_protein: tucker_cap must be >= 0");
    RS_CHECK_ARG(prm->galerkin == 0 || prm->galerkin == 1, "rs_build_protein: galerkin=%d not 0 or 1", prm->galerkin);
    if (prm->galerkin && prm->tucker_cap > 0) {
        set_error("rs_build_protein: Galerkin factors are built for the canonical form only (tucker_cap = 0)");
        return RS_ERR_UNSUPPORTED;
    }
    RS_CHECK_ARG(mem_flags == RS_MEM_HOST || mem_flags == RS_MEM_DEVICE,
                 "rs_build_protein: bad mem_flags %d", mem_flags);
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;  // NULL: the CUDA default stream

    rs_protein* P = new rs_protein();
    P->device = ctx->device;
    P->N = N;
    P->n = prm->n;
    P->b = prm->b;
    P->h = 2.0 * prm->b / (prm->n - 1);
    P->sigma = prm->sigma;
    P->R_l = prm->R_l;
    auto fail_out = [&](rs_status s) {
        rs_protein_free(P);
        return s;
    };
    rs_status s = make_sinc_table(prm->b, prm->sigma, prm->R_l, prm->r_min, prm->tau,
                                  prm->short_tol, &P->table);
    if (s != RS_OK) return fail_out(s);
    P->K = (int)P->table.t.size();

    Scratch S(ctx);
    // inputs on the device and on the host (the small host-side parts: bounding box,
    // charge weights, work estimates); host inputs need no device round trip
    std::vector<double> hq(N), hxyz((size_t)3 * N);
    double *d_xyz = nullptr, *d_q = nullptr;
    if ((s = S.get(&d_xyz, (size_t)3 * N)) != RS_OK) return fail_out(s);
    if ((s = S.get(&d_q, (size_t)N)) != RS_OK) return fail_out(s);
    bool copied;
    if (mem_flags == RS_MEM_HOST) {
        std::memcpy(hxyz.data(), xyz, hxyz.size() * sizeof(double));
        std::memcpy(hq.data(), q, hq.size() * sizeof(double));
        copied = cudaMemcpyAsync(d_xyz, hxyz.data(), hxyz.size() * sizeof(double), cudaMemcpyHostToDevice, st) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(d_q, hq.data(), hq.size() * sizeof(double), cudaMemcpyHostToDevice, st) ==
                     cudaSuccess;
    } else {
        copied = cudaMemcpyAsync(d_xyz, xyz, hxyz.size() * sizeof(double), cudaMemcpyDeviceToDevice, st) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(d_q, q, hq.size() * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(hxyz.data(), xyz, hxyz.size() * sizeof(double), cudaMemcpyDeviceToHost, st) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(hq.data(), q, hq.size() * sizeof(double), cudaMemcpyDeviceToHost, st) ==
                     cudaSuccess &&
                 cudaStreamSynchronize(st) == cudaSuccess;
    }
    if (!copied) {
        set_error("rs_build_protein: input copy failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail_out(RS_ERR_CUDA);
    }
    for (int i = 0; i < N; ++i)
        if (!std::isfinite(hq[i])) {
            set_error("rs_build_protein: charge %d is not finite", i);
            return fail_out(RS_ERR_INVALID);
        }

    // sinc terms on the device
    const int Rl = P->R_l;
    std::vector<double> tl(Rl), al(Rl);
    for (int k = 0; k < Rl; ++k) {
        tl[k] = P->table.t[k];
        al[k] = P->table.a[k];
    }
    double *d_tl, *d_al;
    if ((s = S.get(&d_tl, Rl)) != RS_OK) return fail_out(s);
    if ((s = S.get(&d_al, Rl)) != RS_OK) return fail_out(s);
    cudaMemcpyAsync(d_tl, tl.data(), Rl * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_al, al.data(), Rl * sizeof(double), cudaMemcpyHostToDevice, st);

    if ((s = build_cells(P, st, d_xyz, d_q, hxyz, S)) != RS_OK) return fail_out(s);
    if (prm->tucker_cap == 0) {
        s = build_canonical(P, st, d_xyz, d_q, d_tl, d_al, prm->galerkin);
    } else {
        std::vector<double> cz(N);
        for (int i = 0; i < N; ++i) cz[i] = std::pow(std::fabs(hq[i]), 2.0 / 3.0);
        s = build_tucker(P, st, d_xyz, d_q, d_tl, d_al, tl, al, cz, hxyz, prm->tucker_cap,
                         prm->eps_r > 0 ? prm->eps_r : 0.0, S);
    }
    if (s != RS_OK) return fail_out(s);

    if ((s = finish_short_range(P, st)) != RS_OK) return fail_out(s);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("rs_build_protein: %s", cudaGetErrorString(cudaGetLastError()));
        return fail_out(RS_ERR_CUDA);
    }
    *out = P;
    return RS_OK;
}

namespace {

// Mode product of a d0 x d1 x d2 tensor T (row-major) with M (m x d_ax, row stride
// ldm) along axis ax: out has d_ax replaced by m, out[.., i, ..] = sum_a M[i][a] T[.., a, ..].
std::vector<double> mode_product(const std::vector<double>& T, const int d[3], int ax, const double* M, int m,
                                 int ldm, int dout[3]) {
    for (int a = 0; a < 3; ++a) dout[a] = d[a];
    dout[ax] = m;
    std::vector<double> out((size_t)dout[0] * dout[1] * dout[2], 0.0);
    for (int x = 0; x < d[0]; ++x)
        for (int y = 0; y < d[1]; ++y)
            for (int z = 0; z < d[2]; ++z) {
                const double v = T[((size_t)x * d[1] + y) * d[2] + z];
                if (v == 0.0) continue;
                const int a = ax == 0 ? x : ax == 1 ? y : z;
                for (int i = 0; i < m; ++i) {
                    const int ox = ax == 0 ? i : x, oy = ax == 1 ? i : y, oz = ax == 2 ? i : z;
                    out[((size_t)ox * dout[1] + oy) * dout[2] + oz] += M[(size_t)i * ldm + a] * v;
                }
            }
    return out;
}

}  // namespace

extern "C" rs_status rs_protein_add_compress(rs_ctx* ctx, const rs_protein* const* parts, int32_t count,
                                             int32_t tucker_cap, double eps_r, void* stream, rs_protein** out) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && parts && out, "rs_protein_add_compress: NULL argument");
    *out = nullptr;
    RS_CHECK_ARG(count >= 1 && count <= 16, "rs_protein_add_compress: count=%d out of range [1, 16]", count);
    RS_CHECK_ARG(tucker_cap >= 1 && tucker_cap <= RS_MAX_TUCKER,
                 "rs_protein_add_compress: tucker_cap=%d out of range [1, %d]", tucker_cap, RS_MAX_TUCKER);
    RS_CHECK_ARG(std::isfinite(eps_r) && eps_r >= 0.0 && eps_r < 1.0,
                 "rs_protein_add_compress: eps_r=%g not in [0, 1)", eps_r);
    const rs_protein* p0 = parts[0];
    int ksum[3] = {0, 0, 0};
    long long Ntot = 0;
    for (int p = 0; p < count; ++p) {
        const rs_protein* M = parts[p];
        RS_CHECK_ARG(M, "rs_protein_add_compress: parts[%d] is NULL", p);
        RS_CHECK_ARG(M->kind == 1 && M->view.kind == 1 && M->fac64 && M->core64 && !M->view.box,
                     "rs_protein_add_compress: parts[%d] is not a Tucker-reduced protein", p);
        RS_CHECK_ARG(M->device == ctx->device, "rs_protein_add_compress: parts[%d] is on another device", p);
        RS_CHECK_ARG(M->n == p0->n && M->b == p0->b && M->sigma == p0->sigma && M->R_l == p0->R_l &&
                         M->table.t == p0->table.t && M->table.a == p0->table.a &&
                         M->table.is_long == p0->table.is_long && M->table.r_c == p0->table.r_c,
                     "rs_protein_add_compress: parts[%d] has another grid or sinc table than parts[0]", p);
        for (int a = 0; a < 3; ++a) ksum[a] += M->rank[a];
        Ntot += M->N;
    }
    for (int a = 0; a < 3; ++a)
        RS_CHECK_ARG(ksum[a] <= 128, "rs_protein_add_compress: the parts' ranks on axis %d sum to %d (at most 128)",
                     a, ksum[a]);
    RS_CHECK_ARG(Ntot <= (1 << 22), "rs_protein_add_compress: %lld atoms in the union (at most 2^22)", Ntot);
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p0->n;
    const int N = (int)Ntot;

    rs_protein* P = new rs_protein();
    P->device = ctx->device;
    P->N = N;
    P->n = n;
    P->b = p0->b;
    P->h = p0->h;
    P->sigma = p0->sigma;
    P->R_l = p0->R_l;
    P->table = p0->table;
    P->K = p0->K;
    auto fail_out = [&](rs_status s) {
        rs_protein_free(P);
        return s;
    };
    Scratch S(ctx);
    rs_status s;

    // the parts' FP64 factors and cores on the host
    std::vector<std::vector<double>> fac(count), core(count);
    for (int p = 0; p < count; ++p) {
        const int R = parts[p]->view.R;
        fac[p].resize((size_t)3 * n * R);
        core[p].resize((size_t)R * R * R);
        if (cudaMemcpyAsync(fac[p].data(), parts[p]->fac64, fac[p].size() * sizeof(double), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaMemcpyAsync(core[p].data(), parts[p]->core64, core[p].size() * sizeof(double),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            set_error("rs_protein_add_compress: factor download failed");
            return fail_out(RS_ERR_CUDA);
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("rs_protein_add_compress: %s", cudaGetErrorString(cudaGetLastError()));
        return fail_out(RS_ERR_CUDA);
    }

    // 1. per axis, [V^(1) ... V^(count)] = Q R (thin QR)
    std::vector<double> Q[3], Rf[3];
    for (int a = 0; a < 3; ++a) {
        const int k = ksum[a];
        Q[a].assign((size_t)k * n, 0.0);
        Rf[a].resize((size_t)k * k);
        int col = 0;
        for (int p = 0; p < count; ++p) {
            const int R = parts[p]->view.R;
            const double* Va = fac[p].data() + (size_t)a * n * R;
            for (int c = 0; c < parts[p]->rank[a]; ++c, ++col)
                for (int i = 0; i < n; ++i) Q[a][(size_t)col * n + i] = Va[(size_t)i * R + c];
        }
        rs::gs_qr_host(n, k, Q[a].data(), Rf[a].data());
    }
    // 2. the core in the orthonormal bases: C = sum_p beta_p x_l R_l[:, columns of p]
    std::vector<double> C((size_t)ksum[0] * ksum[1] * ksum[2], 0.0);
    {
        int off[3] = {0, 0, 0};
        for (int p = 0; p < count; ++p) {
            const int R = parts[p]->view.R;
            int d[3] = {parts[p]->rank[0], parts[p]->rank[1], parts[p]->rank[2]};
            std::vector<double> T((size_t)d[0] * d[1] * d[2]);
            for (int x = 0; x < d[0]; ++x)
                for (int y = 0; y < d[1]; ++y)
                    for (int z = 0; z < d[2]; ++z)
                        T[((size_t)x * d[1] + y) * d[2] + z] = core[p][((size_t)x * R + y) * R + z];
            for (int a = 0; a < 3; ++a) {
                int dn[3];
                T = mode_product(T, d, a, Rf[a].data() + off[a], ksum[a], ksum[a], dn);
                for (int e = 0; e < 3; ++e) d[e] = dn[e];
            }
            for (size_t e = 0; e < C.size(); ++e) C[e] += T[e];
            for (int a = 0; a < 3; ++a) off[a] += parts[p]->rank[a];
        }
    }
    // 3. HOSVD of C: the leading eigenvectors of each mode unfolding's Gram matrix
    std::vector<double> U[3];
    int r_ax[3], rmax = 0;
    for (int a = 0; a < 3; ++a) {
        const int k = ksum[a];
        std::vector<double> G((size_t)k * k, 0.0), lam(k), W((size_t)k * k);
        const int d1 = a == 0 ? ksum[1] : ksum[0], d2 = a == 2 ? ksum[1] : ksum[2];
        auto at = [&](int i, int u, int v) -> double {
            // element of C with index i on axis a and (u, v) on the other two axes
            if (a == 0) return C[((size_t)i * ksum[1] + u) * ksum[2] + v];
            if (a == 1) return C[((size_t)u * ksum[1] + i) * ksum[2] + v];
            return C[((size_t)u * ksum[1] + v) * ksum[2] + i];
        };
        std::vector<double> rows((size_t)k * d1 * d2);
        for (int i = 0; i < k; ++i)
            for (int u = 0; u < d1; ++u)
                for (int v = 0; v < d2; ++v) rows[((size_t)i * d1 + u) * d2 + v] = at(i, u, v);
        const size_t len = (size_t)d1 * d2;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j <= i; ++j) {
                double g = 0.0;
                const double* ri = rows.data() + (size_t)i * len;
                const double* rj = rows.data() + (size_t)j * len;
                for (size_t e = 0; e < len; ++e) g += ri[e] * rj[e];
                G[(size_t)i * k + j] = G[(size_t)j * k + i] = g;
            }
        if (!symeig_host(k, G.data(), lam.data(), W.data())) {
            set_error("rs_protein_add_compress: eigen-decomposition of the axis-%d Gram did not converge", a);
            return fail_out(RS_ERR_CUDA);
        }
        const double s1 = std::sqrt(std::max(lam[0], 0.0));
        int r = 0;
        for (int i = 0; i < k; ++i)
            if (std::sqrt(std::max(lam[i], 0.0)) > eps_r * s1) ++r;
        r = std::max(1, std::min(r, (int)tucker_cap));
        double tail = 0.0;
        for (int i = r; i < k; ++i) tail += std::max(lam[i], 0.0);
        P->sv_tail[a] = std::sqrt(tail / std::max(lam[0], 1e-300));
        P->sv_gap[a] = (r < k && lam[r] > 0) ? std::sqrt(lam[r - 1] / lam[r]) : 0.0;
        P->rank[a] = r_ax[a] = r;
        rmax = std::max(rmax, r);
        // U^T (r x k, row-major) for the core's mode products
        U[a].resize((size_t)r * k);
        for (int c = 0; c < r; ++c)
            for (int i = 0; i < k; ++i) U[a][(size_t)c * k + i] = W[(size_t)i * k + c];
    }
    // core = C x_l U_l^T, V_l = Q_l U_l (rows padded to RP columns)
    std::vector<double> B0 = C;
    {
        int d[3] = {ksum[0], ksum[1], ksum[2]};
        for (int a = 0; a < 3; ++a) {
            int dn[3];
            B0 = mode_product(B0, d, a, U[a].data(), r_ax[a], ksum[a], dn);
            for (int e = 0; e < 3; ++e) d[e] = dn[e];
        }
    }
    const int RP = (rmax + 3) / 4 * 4;
    std::vector<double> hV((size_t)3 * n * RP, 0.0);
    for (int a = 0; a < 3; ++a) {
        const int k = ksum[a];
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < r_ax[a]; ++c) {
                double v = 0.0;
                for (int j = 0; j < k; ++j) v += Q[a][(size_t)j * n + i] * U[a][(size_t)c * k + j];
                hV[((size_t)a * n + i) * RP + c] = v;
            }
    }

    // 4. cardinal basis of the compressed factors on the device, and the core in it:
    //    V = Vs V[S,:], so beta' = core x_l V_l[S_l,:]
    int* d_rax;
    double *d_V, *d_M, *d_Ainv, *d_B;
    float2* d_Wp;
    int *d_S, *d_fail;
    if ((s = S.get(&d_rax, 3)) != RS_OK || (s = S.get(&d_V, (size_t)3 * n * RP)) != RS_OK ||
        (s = S.get(&d_M, (size_t)3 * n * RP)) != RS_OK || (s = S.get(&d_Ainv, (size_t)3 * RP * RP)) != RS_OK ||
        (s = S.get(&d_Wp, (size_t)3 * n * RP)) != RS_OK || (s = S.get(&d_S, (size_t)3 * RS_MAX_TUCKER)) != RS_OK ||
        (s = S.get(&d_fail, 3)) != RS_OK || (s = S.get(&d_B, (size_t)RP * RP * RP)) != RS_OK)
        return fail_out(s);
    if (cudaMemcpyAsync(d_rax, r_ax, sizeof(r_ax), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_V, hV.data(), hV.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d_fail, 0, 3 * sizeof(int), st) != cudaSuccess) {
        set_error("rs_protein_add_compress: factor upload failed");
        return fail_out(RS_ERR_CUDA);
    }
    double* d_Vs;
    if ((s = skeleton_basis(st, n, RP, d_rax, d_V, d_M, d_Ainv, d_S, d_Wp, d_fail, S, &d_Vs)) != RS_OK)
        return fail_out(s);
    int hS[3 * RS_MAX_TUCKER];
    if (cudaMemcpyAsync(hS, d_S, sizeof(hS), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("rs_protein_add_compress: %s", cudaGetErrorString(cudaGetLastError()));
        return fail_out(RS_ERR_CUDA);
    }
    {
        int d[3] = {r_ax[0], r_ax[1], r_ax[2]};
        for (int a = 0; a < 3; ++a) {
            const int r = r_ax[a];
            std::vector<double> A((size_t)r * r);
            for (int i = 0; i < r; ++i) {
                const int row = hS[a * RS_MAX_TUCKER + i];
                if (row < 0 || row >= n) {
                    set_error("skeleton selection failed (rank-deficient factor basis)");
                    return fail_out(RS_ERR_CUDA);
                }
                for (int c = 0; c < r; ++c) A[(size_t)i * r + c] = hV[((size_t)a * n + row) * RP + c];
            }
            int dn[3];
            B0 = mode_product(B0, d, a, A.data(), r, r, dn);
            for (int e = 0; e < 3; ++e) d[e] = dn[e];
        }
    }
    std::vector<double> hB((size_t)RP * RP * RP, 0.0);
    for (int x = 0; x < r_ax[0]; ++x)
        for (int y = 0; y < r_ax[1]; ++y)
            for (int z = 0; z < r_ax[2]; ++z)
                hB[((size_t)x * RP + y) * RP + z] = B0[((size_t)x * r_ax[1] + y) * r_ax[2] + z];
    if (cudaMemcpyAsync(d_B, hB.data(), hB.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_error("rs_protein_add_compress: core upload failed");
        return fail_out(RS_ERR_CUDA);
    }
    if ((s = tucker_tables(P, st, n, RP, d_Vs, d_B, d_fail)) != RS_OK) return fail_out(s);

    // 5. the short range of the union of the molecules' atoms
    double *d_xyz, *d_q;
    if ((s = S.get(&d_xyz, (size_t)3 * N)) != RS_OK || (s = S.get(&d_q, (size_t)N)) != RS_OK) return fail_out(s);
    {
        size_t off = 0;
        for (int p = 0; p < count; ++p) {
            const int Np = parts[p]->N;
            ::rs::KernelTimer kt__("k_split_atoms64", st, 0.0, false);
            k_split_atoms64<<<blocks_for(Np), kBlock, 0, st>>>(Np, parts[p]->view.atoms64, d_xyz + 3 * off,
                                                               d_q + off);
            off += (size_t)Np;
        }
    }
    std::vector<double> hxyz((size_t)3 * N);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hxyz.data(), d_xyz, hxyz.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("rs_protein_add_compress: %s", cudaGetErrorString(cudaGetLastError()));
        return fail_out(RS_ERR_CUDA);
    }
    if ((s = build_cells(P, st, d_xyz, d_q, hxyz, S)) != RS_OK) return fail_out(s);
    if ((s = finish_short_range(P, st)) != RS_OK) return fail_out(s);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("rs_protein_add_compress: %s", cudaGetErrorString(cudaGetLastError()));
        return fail_out(RS_ERR_CUDA);
    }
    *out = P;
    return RS_OK;
}
