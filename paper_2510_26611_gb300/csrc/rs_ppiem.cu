// Pose scan of Algorithm PPIEM (Sec. 3.4, steps A0-A7) on the GPU.
//
// For every orbit direction u_d (A5) and self-rotation q_r (A4) the ligand approaches
// the protein centre x_P along x_P + s u_d from far outside (A3); the first contact is
//   s*_dr = max over atom pairs (j, m) with q < sigma^2 of  c + sqrt(sigma^2 - q),
//   w = x_m - x_P - R_r y_j,  c = u_d . w,  q = |w|^2 - c^2,
// and the pose (q_r, x_P + (s*_dr + margin sigma) u_d) is evaluated by the library's
// pose path (A4).  A6: per direction the lowest feasible energy over the rotations,
// then the directions whose lowest energy is a local minimum on the direction grid.
//
// Launch sequence:
//   k_scan_setup     x_P (protein centre unless given), ligand radius, directions,
//                    rotation matrices
//   k_scan_filter    per direction: the protein atoms within (ligand radius + sigma)
//                    of the axis x_P + s u_d (no other atom can meet a ligand line)
//   k_scan_bin       per direction (one CTA): the filtered atoms binned into square
//                    cells of side >= sigma in the plane across u_d and sorted, in each
//                    cell, by descending axial coordinate u_d . (x_m - x_P)
//   k_scan_contact   thread per ligand line (r, j): the 3 x 3 cells around the line's
//                    foot (every atom within sigma of the line is there), each walked
//                    from its front atom until c + sigma falls below the line's best
//                    (no later atom can do better); FP32 screen, FP64 value for the
//                    pairs whose FP32 candidate comes within its error bound of the
//                    best; the line's FP64 maximum goes to its pose by an ordered
//                    64-bit atomic max
//   k_scan_poses     contact poses (quaternion, translation) for the pose path
//   pose path        energies and flags of all D x n_rot poses (launch_eval)
//   k_scan_best      per direction: lowest feasible energy and its rotation
//   k_scan_minima    per direction: local minimum over its grid neighbours
#include <cmath>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"

namespace rs {
namespace {

constexpr int kLines = 256;      // ligand lines (rotation, atom) per contact CTA
constexpr int kBinCap = 8192;    // filtered atoms a direction's binning CTA sorts in shared memory
constexpr int kCellsMax = 32;    // cells per side of a direction's plane grid (at most)
constexpr double kNoContact = -INFINITY;

// Order-preserving map of doubles to signed 64-bit integers (for atomicMax).
__device__ __forceinline__ long long dkey(double x) {
    long long i = __double_as_longlong(x);
    return i >= 0 ? i : i ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double dkey_inv(long long k) {
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffLL);
}

struct ScanView {
    int D, n_theta, n_phi, n_rot, L, N;
    double sigma, sig2, margin;
    const double* y64;      // [L][3] ligand about its centre
    double* xP;             // [3]
    float* rlig;            // [1] max |y_j|
    double* dirs;           // [D][3]
    double* rots;           // [n_rot][9]
    float4* flist;          // [D][N] filtered atoms (x, y, z, index as float bits)
    int* fcount;            // [D]
    long long* keys;        // [D n_rot] ordered max of the contact offset
    double* basis;          // [D][6] e1, e2: orthonormal, across u_d
    float4* fsort;          // [D][N] the filtered atoms by (cell, descending axial)
    int* cbeg;              // [D][kCellsMax^2] cell ranges in fsort
    int* cend;
    float* grid;            // [3] plane grid: half width G, cell side cs, cells per side nc
    double* lp64;           // [n_rot L][3] line points x_P + R_r y_j (FP64)
    float4* lp32;           // [n_rot L] the same in FP32, and R_r y_j in FP32 (.w unused)
    float4* lo32;
};

struct PlaneGrid {
    float G, cs;
    int nc;
    __device__ __forceinline__ explicit PlaneGrid(const float* g) : G(g[0]), cs(g[1]), nc((int)g[2]) {}
    __device__ __forceinline__ int idx(float a) const {
        return min(max((int)floorf((a + G) / cs), 0), nc - 1);
    }
};

// One CTA: x_P (FP64 mean of the protein's atoms when not given), ligand radius;
// then every thread: directions and rotation matrices.
__global__ void k_scan_setup(ProteinView P, ScanView v, const double* __restrict__ xP_in,
                             const double* __restrict__ quats) {
    __shared__ double sm[3][256];
    __shared__ float rmax[256];
    const int t = threadIdx.x;
    double s[3] = {0.0, 0.0, 0.0};
    for (int m = t; m < v.N; m += blockDim.x) {
        const double4 a = P.atoms64[m];
        s[0] += a.x;
        s[1] += a.y;
        s[2] += a.z;
    }
    for (int a = 0; a < 3; ++a) sm[a][t] = s[a];
    float r = 0.f;
    for (int j = t; j < v.L; j += blockDim.x) {
        const double* y = v.y64 + 3 * (size_t)j;
        r = fmaxf(r, (float)sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]));
    }
    rmax[t] = r;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            for (int a = 0; a < 3; ++a) sm[a][t] += sm[a][t + o];
            rmax[t] = fmaxf(rmax[t], rmax[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        for (int a = 0; a < 3; ++a) v.xP[a] = xP_in ? xP_in[a] : sm[a][0] / v.N;
        const float rl = rmax[0] * (1.f + 1e-5f) + 1e-5f;
        v.rlig[0] = rl;
        // plane grid around the axis: the filtered atoms lie within rl + sigma of it;
        // cells of side >= sigma (plus a margin for FP32 rounding), so the 3 x 3 cells
        // around a line's foot hold every atom within sigma of the line
        const float G = rl + (float)v.sigma + 1e-2f;
        const float cs = fmaxf((float)v.sigma * (1.f + 1e-3f) + 1e-3f, 2.f * G / kCellsMax);
        v.grid[0] = G;
        v.grid[1] = cs;
        v.grid[2] = (float)min(kCellsMax, (int)ceilf(2.f * G / cs));
    }
    for (int d = t; d < v.D; d += blockDim.x) {
        const int a = d / v.n_phi, b = d - a * v.n_phi;
        const double th = (a + 0.5) * M_PI / v.n_theta, ph = b * 2.0 * M_PI / v.n_phi;
        const double u0 = sin(th) * cos(ph), u1 = sin(th) * sin(ph), u2 = cos(th);
        v.dirs[3 * d] = u0;
        v.dirs[3 * d + 1] = u1;
        v.dirs[3 * d + 2] = u2;
        // e1 = u x a / |u x a| with a = e_z (e_x near the poles), e2 = u x e1
        const double ax = fabs(u2) < 0.9 ? 0.0 : 1.0, az = 1.0 - ax;
        double e0 = u1 * az, e1 = u2 * ax - u0 * az, e2 = -u1 * ax;
        const double nrm = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        e0 /= nrm;
        e1 /= nrm;
        e2 /= nrm;
        double* B = v.basis + 6 * d;
        B[0] = e0;
        B[1] = e1;
        B[2] = e2;
        B[3] = u1 * e2 - u2 * e1;
        B[4] = u2 * e0 - u0 * e2;
        B[5] = u0 * e1 - u1 * e0;
    }
    for (int r2 = t; r2 < v.n_rot; r2 += blockDim.x)
        dev::quat_to_rot(quats[4 * r2], quats[4 * r2 + 1], quats[4 * r2 + 2], quats[4 * r2 + 3], v.rots + 9 * r2);
}

// One warp per direction: protein atoms whose squared distance from the axis is at
// most (ligand radius + sigma)^2 (FP32, with a margin), compacted in atom order.
__global__ void k_scan_filter(ProteinView P, ScanView v) {
    const int lane = threadIdx.x & 31;
    const int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (d >= v.D) return;
    const float u0 = (float)v.dirs[3 * d], u1 = (float)v.dirs[3 * d + 1], u2 = (float)v.dirs[3 * d + 2];
    const float x0 = (float)v.xP[0], x1 = (float)v.xP[1], x2 = (float)v.xP[2];
    const float lim = v.rlig[0] + (float)v.sigma;
    const float lim2 = lim * lim * (1.f + 1e-3f) + 1e-3f;
    float4* out = v.flist + (size_t)d * v.N;
    int n = 0;
    for (int base = 0; base < v.N; base += 32) {
        const int m = base + lane;
        bool keep = false;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < v.N) {
            a = P.atoms[m];
            const float w0 = a.x - x0, w1 = a.y - x1, w2 = a.z - x2;
            const float c = fmaf(u2, w2, fmaf(u1, w1, u0 * w0));
            const float q = fmaf(w2, w2, fmaf(w1, w1, w0 * w0)) - c * c;
            keep = q <= lim2;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) out[n + __popc(bal & ((1u << lane) - 1u))] = make_float4(a.x, a.y, a.z, __int_as_float(m));
        n += __popc(bal);
    }
    if (lane == 0) v.fcount[d] = n;
}

// Order key of a float (ascending floats give ascending keys).
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// One CTA per direction: key = (cell, descending axial coordinate), bitonic sort of
// (key, position) pairs in shared memory, then the atoms in key order and the cell
// ranges.  A direction with more than kBinCap filtered atoms keeps no cells
// (cbeg[0] = -1) and its lines scan the whole list.
__global__ void __launch_bounds__(512) k_scan_bin(ScanView v) {
    extern __shared__ __align__(16) unsigned char smb[];
    unsigned long long* key = (unsigned long long*)smb;
    int* pos = (int*)(key + kBinCap);
    const int d = blockIdx.x;
    const int cnt = v.fcount[d];
    const PlaneGrid pg(v.grid);
    int* cb = v.cbeg + (size_t)d * kCellsMax * kCellsMax;
    int* ce = v.cend + (size_t)d * kCellsMax * kCellsMax;
    for (int c = threadIdx.x; c < pg.nc * pg.nc; c += blockDim.x) {
        cb[c] = 0;
        ce[c] = 0;
    }
    if (cnt > kBinCap) {
        if (threadIdx.x == 0) cb[0] = -1;
        return;
    }
    const float4* in = v.flist + (size_t)d * v.N;
    const double* B = v.basis + 6 * d;
    const float b0 = (float)B[0], b1 = (float)B[1], b2 = (float)B[2];
    const float c0 = (float)B[3], c1 = (float)B[4], c2 = (float)B[5];
    const float u0 = (float)v.dirs[3 * d], u1 = (float)v.dirs[3 * d + 1], u2 = (float)v.dirs[3 * d + 2];
    const float x0 = (float)v.xP[0], x1 = (float)v.xP[1], x2 = (float)v.xP[2];
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (i < cnt) {
            const float4 a = in[i];
            const float w0 = a.x - x0, w1 = a.y - x1, w2 = a.z - x2;
            const float a1 = fmaf(b2, w2, fmaf(b1, w1, b0 * w0));
            const float a2 = fmaf(c2, w2, fmaf(c1, w1, c0 * w0));
            const float ax = fmaf(u2, w2, fmaf(u1, w1, u0 * w0));
            const int cell = pg.idx(a2) * pg.nc + pg.idx(a1);
            key[i] = ((unsigned long long)cell << 32) | (unsigned long long)(~fkey(ax));
        } else {
            key[i] = ~0ULL;
        }
        pos[i] = i;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long ki = key[i], kl = key[l];
                    if ((ki > kl) == up) {
                        key[i] = kl;
                        key[l] = ki;
                        const int t = pos[i];
                        pos[i] = pos[l];
                        pos[l] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    float4* out = v.fsort + (size_t)d * v.N;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        out[i] = in[pos[i]];
        const int c = (int)(key[i] >> 32);
        if (i == 0 || (int)(key[i - 1] >> 32) != c) cb[c] = i;
        if (i == cnt - 1 || (int)(key[i + 1] >> 32) != c) ce[c] = i + 1;
    }
}

// Line points of every (rotation, ligand atom): they do not depend on the direction.
__global__ void k_scan_lines(ScanView v) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)v.n_rot * v.L) return;
    const int r = (int)(g / v.L), j = (int)(g - (long long)r * v.L);
    const double* R = v.rots + 9 * r;
    const double* y = v.y64 + 3 * (size_t)j;
    double o[3], p[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = fma(R[3 * a + 2], y[2], fma(R[3 * a + 1], y[1], R[3 * a] * y[0]));
        p[a] = v.xP[a] + o[a];
        v.lp64[3 * g + a] = p[a];
    }
    v.lp32[g] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
    v.lo32[g] = make_float4((float)o[0], (float)o[1], (float)o[2], 0.f);
}

// One protein atom against line p.  Every candidate is <= c + sigma, and the FP32 c
// is within 1e-3 A of the FP64 one, so a front-to-back walk of a cell stops (returns
// false) once c + sigma + 1e-3 falls below lb, a lower bound of the line's answer.
// The FP32 q errs by at most band (a few ulps of |w|^2 + c^2 plus the coordinates'
// rounding), hence the FP32 candidate by at most tol = sqrt(band) + 2e-3 A.
//   PASS 0 (FP32 only): pairs with q < sigma^2 - band block in FP64 too, so their
//                       candidate - tol is a lower bound: lb = max of those.
//   PASS 1: the pairs that may block (q < sigma^2 + band) and may reach lb
//           (candidate + tol >= lb) get the FP64 value of the definition.
template <int PASS>
__device__ __forceinline__ bool contact_pair(const ProteinView& P, const ScanView& v, float4 a, const float pf[3],
                                             const float uf[3], const double* __restrict__ p, const double* u,
                                             float s2, float sigf, float& lb, double& best) {
    const float w0 = a.x - pf[0], w1 = a.y - pf[1], w2 = a.z - pf[2];
    const float c = fmaf(uf[2], w2, fmaf(uf[1], w1, uf[0] * w0));
    if (c + sigf + 1e-3f < lb) return false;
    const float wsq = fmaf(w2, w2, fmaf(w1, w1, w0 * w0));
    const float q = fmaf(-c, c, wsq);
    const float band = 1e-6f * (wsq + c * c) + 1e-4f;
    if (q < s2 + band) {
        const float tol = sqrtf(band) + 2e-3f;
        const float cand = c + sqrtf(fmaxf(s2 - q, 0.f));
        if (PASS == 0) {
            if (q < s2 - band) lb = fmaxf(lb, cand - tol);
        } else if (cand + tol >= lb) {
            const double4 b = P.atoms64[__float_as_int(a.w)];
            const double x0 = b.x - p[0], x1 = b.y - p[1], x2 = b.z - p[2];
            const double cc = u[0] * x0 + u[1] * x1 + u[2] * x2;
            const double qq = (x0 * x0 + x1 * x1 + x2 * x2) - cc * cc;
            if (qq < v.sig2) best = fmax(best, cc + sqrt(v.sig2 - qq));
        }
    }
    return true;
}

// Contact offsets: CTA (line block, direction); thread = ligand line (r, j).
__global__ void __launch_bounds__(kLines) k_scan_contact(ProteinView P, ScanView v) {
    const int d = blockIdx.y;
    const long long g = (long long)blockIdx.x * kLines + threadIdx.x;
    const long long lines = (long long)v.n_rot * v.L;
    if (g >= lines) return;
    const int r = (int)(g / v.L), j = (int)(g - (long long)r * v.L);
    (void)j;
    const double* u = v.dirs + 3 * d;
    // line point p = x_P + R_r y_j: FP64 (read only for the FP64 pairs) and FP32
    const double* p = v.lp64 + 3 * g;
    const float4 pl = v.lp32[g], ol = v.lo32[g];
    const float pf[3] = {pl.x, pl.y, pl.z};
    const float uf[3] = {(float)u[0], (float)u[1], (float)u[2]};
    const float s2 = (float)v.sig2, sigf = (float)v.sigma;
    // the pose's offset is the maximum over its lines: a candidate below a lower bound
    // of another line's answer cannot matter, so the lines of a pose share their
    // lower bounds through the pose's key (an FP64 maximum at the end, which is never
    // below a lower bound)
    long long* kp = v.keys + (size_t)d * v.n_rot + r;
    float lb = __double2float_rd(dkey_inv(*(volatile long long*)kp));
    double best = kNoContact;
    const int* cb = v.cbeg + (size_t)d * kCellsMax * kCellsMax;
    const int* ce = v.cend + (size_t)d * kCellsMax * kCellsMax;
    if (cb[0] < 0) {
        const float4* list = v.flist + (size_t)d * v.N;
        const int cnt = v.fcount[d];
        for (int e = 0; e < cnt; ++e) contact_pair<0>(P, v, list[e], pf, uf, p, u, s2, sigf, lb, best);
        for (int e = 0; e < cnt; ++e) contact_pair<1>(P, v, list[e], pf, uf, p, u, s2, sigf, lb, best);
    } else {
        // the line's foot in the plane grid (FP32: the cells carry a 1e-3 A margin)
        const double* B = v.basis + 6 * d;
        const float a1 = fmaf((float)B[2], ol.z, fmaf((float)B[1], ol.y, (float)B[0] * ol.x));
        const float a2 = fmaf((float)B[5], ol.z, fmaf((float)B[4], ol.y, (float)B[3] * ol.x));
        const PlaneGrid pg(v.grid);
        const int i1 = pg.idx(a1), i2 = pg.idx(a2);
        const float4* list = v.fsort + (size_t)d * v.N;
        // the line's own cell first (it usually holds the contact), then its 8 neighbours
        for (int pass = 0; pass < 2; ++pass) {
            for (int k = 0; k < 9; ++k) {
                const int dd = k == 0 ? 4 : (k <= 4 ? k - 1 : k);
                const int c1 = i1 + dd % 3 - 1, c2 = i2 + dd / 3 - 1;
                if (c1 < 0 || c2 < 0 || c1 >= pg.nc || c2 >= pg.nc) continue;
                const int c = c2 * pg.nc + c1;
                if (pass == 0) {
                    for (int e = cb[c]; e < ce[c]; ++e)
                        if (!contact_pair<0>(P, v, list[e], pf, uf, p, u, s2, sigf, lb, best)) break;
                    if (k == 0 && lb > -INFINITY)
                        lb = fmaxf(lb, __double2float_rd(dkey_inv(atomicMax(kp, dkey((double)lb)))));
                } else {
                    for (int e = cb[c]; e < ce[c]; ++e)
                        if (!contact_pair<1>(P, v, list[e], pf, uf, p, u, s2, sigf, lb, best)) break;
                }
            }
            if (pass == 0 && lb > -INFINITY)
                lb = fmaxf(lb, __double2float_rd(dkey_inv(atomicMax(kp, dkey((double)lb)))));
        }
    }
    if (best > kNoContact) atomicMax(kp, dkey(best));
}

__global__ void k_scan_init_keys(long long* keys, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = dkey(kNoContact);
}

// Contact poses for the pose path; s_out (optional) gets s*.
__global__ void k_scan_poses(ScanView v, const double* __restrict__ quats, double* __restrict__ pq,
                             double* __restrict__ pt, double* __restrict__ s_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)v.D * v.n_rot) return;
    const int d = (int)(i / v.n_rot), r = (int)(i - (long long)d * v.n_rot);
    const double s = dkey_inv(v.keys[i]);
    if (s_out) s_out[i] = s;
    for (int a = 0; a < 4; ++a) pq[4 * i + a] = quats[4 * r + a];
    const double off = s > kNoContact ? s + v.margin * v.sigma : 0.0;
    for (int a = 0; a < 3; ++a) pt[3 * i + a] = v.xP[a] + off * v.dirs[3 * d + a];
}

// One warp per direction: no-contact poses get E = +inf and flag 4; then the lowest
// feasible energy (lowest rotation index among equal energies).
__global__ void k_scan_best(ScanView v, double* __restrict__ E, uint8_t* __restrict__ F,
                            const double* __restrict__ pt, double* __restrict__ E_best,
                            int* __restrict__ rot_best, double* __restrict__ t_best) {
    const int lane = threadIdx.x & 31;
    const int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (d >= v.D) return;
    double bE = INFINITY;
    int br = -1;
    for (int r = lane; r < v.n_rot; r += 32) {
        const long long i = (long long)d * v.n_rot + r;
        if (!(dkey_inv(v.keys[i]) > kNoContact)) {
            E[i] = INFINITY;
            F[i] = 4;
            continue;
        }
        if (F[i] == 0 && (E[i] < bE || (E[i] == bE && (br < 0 || r < br)))) {
            bE = E[i];
            br = r;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double oE = __shfl_xor_sync(0xffffffffu, bE, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (orr >= 0 && (oE < bE || (oE == bE && (br < 0 || orr < br)))) {
            bE = oE;
            br = orr;
        }
    }
    if (lane == 0) {
        E_best[d] = bE;
        rot_best[d] = br;
        for (int a = 0; a < 3; ++a) t_best[3 * d + a] = br >= 0 ? pt[3 * ((long long)d * v.n_rot + br) + a] : NAN;
    }
}

// Local minima of E_best on the (theta, phi) grid: neighbours a +- 1 (no wrap) and
// b +- 1 (wrapping); ties go to the lower direction index.
__global__ void k_scan_minima(ScanView v, const double* __restrict__ E_best, uint8_t* __restrict__ is_min) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= v.D) return;
    const double e = E_best[d];
    bool m = e < INFINITY;
    const int a = d / v.n_phi, b = d - a * v.n_phi;
    int nb[4];
    int k = 0;
    if (a > 0) nb[k++] = d - v.n_phi;
    if (a + 1 < v.n_theta) nb[k++] = d + v.n_phi;
    nb[k++] = a * v.n_phi + (b + v.n_phi - 1) % v.n_phi;
    nb[k++] = a * v.n_phi + (b + 1) % v.n_phi;
    for (int i = 0; i < k && m; ++i) {
        const int o = nb[i];
        if (o == d) continue;
        const double f = E_best[o];
        m = e < f || (e == f && d < o);
    }
    is_min[d] = m ? 1 : 0;
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace rs

extern "C" rs_status rs_ppiem_scan(rs_ctx* ctx, const rs_protein* prot, int32_t L, const double* lig_xyz,
                                   const double* lig_q, int32_t n_theta, int32_t n_phi, int32_t n_rot,
                                   const double* quats, const double* x_P, double margin, double* s_out,
                                   double* E_out, uint8_t* flags_out, double* E_best, int32_t* rot_best,
                                   double* t_best, uint8_t* is_min, int mem_flags, void* stream) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && prot, "NULL context or protein");
    RS_CHECK_ARG(L >= 1 && L <= 4096, "L=%d out of range [1, 4096]", L);
    RS_CHECK_ARG(n_theta >= 1 && n_phi >= 1 && (long long)n_theta * n_phi <= 65535,
                 "direction grid %d x %d out of range", n_theta, n_phi);
    RS_CHECK_ARG(n_rot >= 1, "n_rot=%d must be >= 1", n_rot);
    const long long D = (long long)n_theta * n_phi, PT = D * n_rot;
    RS_CHECK_ARG(PT <= (1LL << 26), "%lld poses exceed 2^26", PT);
    RS_CHECK_ARG(std::isfinite(margin) && margin >= 0.0, "margin=%g must be finite and >= 0", margin);
    RS_CHECK_ARG(mem_flags == RS_MEM_HOST || mem_flags == RS_MEM_DEVICE, "bad mem_flags %d", mem_flags);
    RS_CHECK_ARG(prot->device == ctx->device, "protein built on device %d, context on %d", prot->device,
                 ctx->device);
    RS_CHECK_ARG(lig_xyz && lig_q && quats && E_best && rot_best && t_best && is_min, "NULL input or output pointer");
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int N = prot->N;
    const double mg = margin > 0.0 ? margin : 1e-6;
    // scratch: inputs (host calls), scan state, pose arrays, per-pose outputs
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += al256(b);
        return o;
    };
    const size_t o_lx = take((size_t)L * 24), o_lq = take((size_t)L * 8), o_qu = take((size_t)n_rot * 32),
                 o_xp = take(24), o_xin = take(24), o_rl = take(4), o_dir = take((size_t)D * 24),
                 o_rot = take((size_t)n_rot * 72), o_fl = take((size_t)D * N * 16), o_fc = take((size_t)D * 4),
                 o_key = take((size_t)PT * 8), o_pq = take((size_t)PT * 32), o_pt = take((size_t)PT * 24),
                 o_E = take((size_t)PT * 8), o_F = take((size_t)PT), o_s = take((size_t)PT * 8),
                 o_Eb = take((size_t)D * 8), o_rb = take((size_t)D * 4), o_tb = take((size_t)D * 24),
                 o_im = take((size_t)D), o_bas = take((size_t)D * 48), o_fs = take((size_t)D * N * 16),
                 o_cb = take((size_t)D * kCellsMax * kCellsMax * 4), o_ce = take((size_t)D * kCellsMax * kCellsMax * 4),
                 o_grid = take(16), o_lp64 = take((size_t)n_rot * L * 24), o_lp32 = take((size_t)n_rot * L * 16),
                 o_lo32 = take((size_t)n_rot * L * 16);
    RS_TRY(ensure_buffer(&ctx->fd_buf, &ctx->fd_bytes, off));
    char* B = (char*)ctx->fd_buf;
    const double *d_lx = lig_xyz, *d_lq = lig_q, *d_qu = quats, *d_xin = x_P;
    double *d_E = E_out ? E_out : (double*)(B + o_E), *d_s = s_out;
    uint8_t* d_F = flags_out ? flags_out : (uint8_t*)(B + o_F);
    double *d_Eb = E_best, *d_tb = t_best;
    int* d_rb = rot_best;
    uint8_t* d_im = is_min;
    if (mem_flags == RS_MEM_HOST) {
        d_lx = (const double*)(B + o_lx);
        d_lq = (const double*)(B + o_lq);
        d_qu = (const double*)(B + o_qu);
        d_xin = x_P ? (const double*)(B + o_xin) : nullptr;
        d_E = (double*)(B + o_E);
        d_F = (uint8_t*)(B + o_F);
        d_s = s_out ? (double*)(B + o_s) : nullptr;
        d_Eb = (double*)(B + o_Eb);
        d_rb = (int*)(B + o_rb);
        d_tb = (double*)(B + o_tb);
        d_im = (uint8_t*)(B + o_im);
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_lx, lig_xyz, (size_t)L * 24, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_lq, lig_q, (size_t)L * 8, cudaMemcpyHostToDevice, st));
        RS_TRY_CUDA(cudaMemcpyAsync((void*)d_qu, quats, (size_t)n_rot * 32, cudaMemcpyHostToDevice, st));
        if (x_P) RS_TRY_CUDA(cudaMemcpyAsync((void*)d_xin, x_P, 24, cudaMemcpyHostToDevice, st));
    }
    RS_TRY(ensure_buffer(&ctx->lig_buf, &ctx->lig_bytes, ligand_scratch_bytes(L) + 1024));
    LigandView lig = carve_ligand(ctx->lig_buf, L);
    RS_TRY(launch_prep_ligand(L, d_lx, d_lq, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64, (double*)lig.q64, st));
    ScanView v;
    v.D = (int)D;
    v.n_theta = n_theta;
    v.n_phi = n_phi;
    v.n_rot = n_rot;
    v.L = L;
    v.N = N;
    v.sigma = prot->sigma;
    v.sig2 = prot->view.sig2;
    v.margin = mg;
    v.y64 = lig.y64;
    v.xP = (double*)(B + o_xp);
    v.rlig = (float*)(B + o_rl);
    v.dirs = (double*)(B + o_dir);
    v.rots = (double*)(B + o_rot);
    v.flist = (float4*)(B + o_fl);
    v.fcount = (int*)(B + o_fc);
    v.keys = (long long*)(B + o_key);
    v.basis = (double*)(B + o_bas);
    v.fsort = (float4*)(B + o_fs);
    v.cbeg = (int*)(B + o_cb);
    v.cend = (int*)(B + o_ce);
    v.grid = (float*)(B + o_grid);
    v.lp64 = (double*)(B + o_lp64);
    v.lp32 = (float4*)(B + o_lp32);
    v.lo32 = (float4*)(B + o_lo32);
    double* pq = (double*)(B + o_pq);
    double* pt = (double*)(B + o_pt);
    {
        ::rs::KernelTimer kt__("k_scan_setup", st, 0.0, false);
        k_scan_setup<<<1, 256, 0, st>>>(prot->view, v, d_xin, d_qu);
    }
    {
        ::rs::KernelTimer kt__("k_scan_filter", st, 0.0, false);
        k_scan_filter<<<(unsigned)((D * 32 + 255) / 256), 256, 0, st>>>(prot->view, v);
    }
    {
        const long long lines = (long long)n_rot * L;
        ::rs::KernelTimer kt__("k_scan_lines", st, 0.0, false);
        k_scan_lines<<<(unsigned)((lines + 255) / 256), 256, 0, st>>>(v);
    }
    {
        const size_t smem = (size_t)kBinCap * 12;
        RS_TRY_CUDA(cudaFuncSetAttribute(k_scan_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ::rs::KernelTimer kt__("k_scan_bin", st, 0.0, false);
        k_scan_bin<<<(unsigned)D, 512, smem, st>>>(v);
    }
    {
        ::rs::KernelTimer kt__("k_scan_init_keys", st, 0.0, false);
        k_scan_init_keys<<<(unsigned)((PT + 255) / 256), 256, 0, st>>>(v.keys, PT);
    }
    {
        const long long lines = (long long)n_rot * L;
        dim3 grid((unsigned)((lines + kLines - 1) / kLines), (unsigned)D);
        ::rs::KernelTimer kt__("k_scan_contact", st, 0.0, false);
        k_scan_contact<<<grid, kLines, 0, st>>>(prot->view, v);
    }
    {
        ::rs::KernelTimer kt__("k_scan_poses", st, 0.0, false);
        k_scan_poses<<<(unsigned)((PT + 255) / 256), 256, 0, st>>>(v, d_qu, pq, pt, d_s);
    }
    RS_TRY_CUDA(cudaGetLastError());
    EvalLaunch a;
    a.prot = prot->view;
    a.lig = lig;
    a.rot = pq;
    a.trans = pt;
    a.P = PT;
    a.E = d_E;
    a.flags = d_F;
    if (prot->view.kind == 1) {
        RS_TRY(ensure_buffer(&ctx->eval_buf, &ctx->eval_bytes, sorted_scratch_bytes(PT, L, prot->n, false)));
        a.ws = ctx->eval_buf;
        a.ws_bytes = ctx->eval_bytes;
    }
    RS_TRY(launch_eval(a, false, st));
    {
        ::rs::KernelTimer kt__("k_scan_best", st, 0.0, false);
        k_scan_best<<<(unsigned)((D * 32 + 255) / 256), 256, 0, st>>>(v, d_E, d_F, pt, d_Eb, d_rb, d_tb);
    }
    {
        ::rs::KernelTimer kt__("k_scan_minima", st, 0.0, false);
        k_scan_minima<<<(unsigned)((D + 255) / 256), 256, 0, st>>>(v, d_Eb, d_im);
    }
    RS_TRY_CUDA(cudaGetLastError());
    if (mem_flags == RS_MEM_HOST) {
        if (s_out) RS_TRY_CUDA(cudaMemcpyAsync(s_out, d_s, (size_t)PT * 8, cudaMemcpyDeviceToHost, st));
        if (E_out) RS_TRY_CUDA(cudaMemcpyAsync(E_out, d_E, (size_t)PT * 8, cudaMemcpyDeviceToHost, st));
        if (flags_out) RS_TRY_CUDA(cudaMemcpyAsync(flags_out, d_F, (size_t)PT, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(E_best, d_Eb, (size_t)D * 8, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(rot_best, d_rb, (size_t)D * 4, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(t_best, d_tb, (size_t)D * 24, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaMemcpyAsync(is_min, d_im, (size_t)D, cudaMemcpyDeviceToHost, st));
        RS_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return RS_OK;
}
