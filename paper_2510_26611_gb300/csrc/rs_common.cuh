// Internal definitions shared by the librs translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/rs.h"

#define RS_MAX_SHORT 24      // short-range sinc terms handled on the device
#define RS_MAX_TUCKER 32     // largest Tucker rank per axis

namespace rs {

void set_error(const char* fmt, ...);
void clear_error();

#define RS_TRY_CUDA(expr)                                                              \
    do {                                                                               \
        cudaError_t e__ = (expr);                                                      \
        if (e__ != cudaSuccess) {                                                      \
            ::rs::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e__),   \
                            __FILE__, __LINE__);                                       \
            return RS_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

#define RS_TRY(expr)                           \
    do {                                       \
        rs_status s__ = (expr);                \
        if (s__ != RS_OK) return s__;          \
    } while (0)

#define RS_CHECK_ARG(cond, ...)                \
    do {                                       \
        if (!(cond)) {                         \
            ::rs::set_error(__VA_ARGS__);      \
            return RS_ERR_INVALID;             \
        }                                      \
    } while (0)

// Host copy of the sinc quadrature (Sec. 2, Eq. sinc) and its range split.
struct SincTable {
    std::vector<double> t, a;
    std::vector<uint8_t> is_long;
    double h_s = 0, box_len = 0, r_c = 0, quad_err = -1, r_min = 0;
    int R_l = 0;
};
double sinc_quad_error(const SincTable& T);
rs_status make_sinc_table(double b, double sigma, int R_l, double r_min, double tau,
                          double short_tol, SincTable* out);

// Everything a pose kernel needs about one protein, passed by value.
struct ProteinView {
    int n;
    double b, h, inv_h;
    int kind;            // 0: canonical factors, 1: Tucker (skeleton basis, W form)
    int ld;              // floats per factor row
    int R;               // canonical: padded rank (multiple of 128); Tucker: padded rank RP
    const float* F[3];   // canonical: factor rows [n][ld]; axis 3 carries the weights xi
    // Tucker, evaluated through W[i][a][b] = sum_c V3'[i][c] core[a][b][c] (an exact
    // rewrite of the Tucker form) and the row differences D[i] = W[i+1] - W[i],
    // each stored as a float pair hi + lo:
    const float* Wt[4];      // Wh, Wl, Dh, Dl   [n][RP][RP]
    const float* Vt[2][4];   // axes 1, 2: Vh, Vl, VDh, VDl  [n][RP]
    // the same W form as BF16-sliced MMA operands (rs_tc.cuh): per axis-3 cell the
    // B image (4 slices of NP x KP, canonical K-major layout) and NP inverse scales
    const uint16_t* Wtc;
    const float* Wsc;
    const float* core;   // Tucker core [RP][RP][RP] (FP32, diagnostics)
    int Ks;              // short-range terms: t_k^2 and a_k (FP64)
    double ts2[RS_MAX_SHORT];
    double as[RS_MAX_SHORT];
    // short-range radial function f(s) = sum_short a_k exp(-t_k^2 s), s = d^2, as
    // piecewise cubics on s in [j hs, (j+1) hs], j = 0..stab_n-2: the Hermite cubic
    // of f and hs f' at both ends in the local variable u = s/hs - j, stored as
    // Horner coefficients c0..c3 in float pairs, two float4 per interval:
    // stab2[2j] = (c0.h, c0.l, c1.h, c1.l), stab2[2j+1] = (c2.h, c2.l, c3.h, c3.l)
    const float4* stab2;
    int stab_n;
    double stab_inv_h;
    float stab_ih_h, stab_ih_l;  // 1/hs as a float pair
    double rc2;          // r_c^2
    float rc2_hi;        // r_c^2 (1 + 1e-4): FP32 pre-filter
    float rc2_ph, rc2_pl;    // r_c^2 as a float pair
    double sig2;         // sigma^2
    float sig2_lo, sig2_hi;  // sigma^2 (1 -/+ 1e-4): FP32 decision band
    float sig2_ph, sig2_pl;  // sigma^2 as a float pair
    float b_h, b_l, inv_h_h, inv_h_l;  // b and 1/h as float pairs
    const float4* atoms;     // cell-sorted protein atoms (x, y, z, q), FP32 nearest
    const float4* atoms_lo;  // remainders: atoms + atoms_lo = the record to ~2^-48
    const double4* atoms64;  // the FP64 record (vdW decisions inside the sigma band)
    // Short-range candidate lists: fine cells of side f over the protein's box grown by
    // the neighbour radius R; cell c lists, in cell-sorted atom order, every atom within
    // R (plus a margin) of its box, so a query reads one contiguous list.
    const int* nb_start;     // [nf0 nf1 nf2 + 1]
    const float4* nb_atoms;  // the listed atoms' FP32 records (list order)
    const int* nb_idx;       // their indices into atoms / atoms_lo / atoms64
    int nf0, nf1, nf2;
    float fo0, fo1, fo2;     // fine-grid origin
    float inv_fine;          // 1 / f
    // a local-box handle (scheme C): its tables cover the interpolation cells
    // [cell_lo, cell_hi] per axis only; a pose with an atom outside them is flagged out
    // of grid by a pass after the evaluation (launch_box_flags), which keeps the test
    // out of the pose kernels' per-atom geometry
    int box;
    int cell_lo[3], cell_hi[3];
};

// A prepared ligand on the device: coordinates about the geometric centre.
struct LigandView {
    int L;
    const float4* y;     // (y_x, y_y, y_z, q) FP32
    const float2* yd;    // [L][3] coordinates as float pairs (hi, lo)
    const double* y64;   // [L][3] FP64 (vdW decisions inside the sigma band)
    const double* q64;   // [L]
};

// One protein-ligand pair of a batched launch: views, pose inputs (quaternions) and
// outputs, all device memory.
struct PairDesc {
    ProteinView prot;
    LigandView lig;
    const double* rot;
    const double* trans;
    long long P;
    double* E;
    uint8_t* flags;
};

}  // namespace rs

struct rs_protein {
    int device = 0;
    int n = 0, N = 0, R_l = 0, K = 0;
    double b = 0, h = 0, sigma = 0;
    rs::SincTable table;
    int kind = 0;
    int rank[3] = {0, 0, 0};
    double sv_gap[3] = {0, 0, 0};
    double sv_tail[3] = {0, 0, 0};
    rs::ProteinView view{};
    std::vector<void*> allocations;   // device buffers owned by the handle
    size_t device_bytes = 0;
    int subspace_steps = 0;           // Tucker build: subspace-iteration steps taken
    // Tucker handles: FP64 cardinal factors (3 x n x R, R = view.R) and core (R^3) on
    // the device, kept for add-and-compress
    double* fac64 = nullptr;
    double* core64 = nullptr;
    // local-box handles share their parent's short-range data: the parent is freed
    // only when it and all of its local handles have been freed
    rs_protein* parent = nullptr;
    int children = 0;
    bool released = false;            // rs_protein_free called while children lived
};

struct rs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // Scratch owned by the context: prepared ligand and staging for host calls.
    void* lig_buf = nullptr;
    size_t lig_bytes = 0;
    void* io_buf = nullptr;
    size_t io_bytes = 0;
    // Projected-gradient workspace (per-pose state of rs_pgd_run).
    void* pgd_buf = nullptr;
    size_t pgd_bytes = 0;
    // Per-atom arrays of the cell-grouped pose path.
    void* eval_buf = nullptr;
    size_t eval_bytes = 0;
    // Scratch of the finite-difference forces (evaluation poses), the pose scan and
    // the molecular-complex call (staging and per-molecule results).
    void* fd_buf = nullptr;
    size_t fd_bytes = 0;
    // Build workspace, grown to the largest build seen (one build at a time).
    void* ws_buf = nullptr;
    size_t ws_bytes = 0;
};

namespace rs {
rs_status ensure_buffer(void** buf, size_t* cap, size_t need);
// Device int counting tensor-core tiles whose MMA did not complete in the bounded
// wait (allocated once per device, on first use from a context's creation).
int* tc_error_flag(int device);
// W-form kernel of the cell-grouped pose paths: 1 tensor cores, 0 float pairs.
int wform_kernel_mode();
int build_gemm_mode();
// Work counters of the sorted atoms kernels on a device (atoms, candidates, near
// pairs; one triple for energies, one for gradients), in the same device buffer.
unsigned long long* short_counters(int device, bool grad);
// FP32 pipe operations (FADD, FMUL, FFMA one each) of the atoms kernel's algorithmic
// work: per pose-atom the pair position (nine Dot2 steps, three renormalisations),
// three grid-cell lookups and the list cell (~230); per screened candidate the FP32
// squared distance (6); per near pair the pair-arithmetic offset, distance and
// cubic and its accumulation (121 for energies, 179 with the gradient terms).  The
// totals match the kernels' FP32 instruction counters on the protein workload.
double short_work_ops(bool grad, double atoms, double cand, double near);
// Launch shape of the latest tensor-core W-form launch (diagnostics).
void note_tc_launch(long long grid, size_t smem, int per_sm);
// B images of the W form for the tensor-core path (rs_tc.cu): sizes for n cells of
// padded rank RP, and the build from the W-form planes wt ([Wh|Wl|Dh|Dl][n][RP][RP]).
size_t tc_bimage_bytes(int n, int RP);
size_t tc_bscale_bytes(int n, int RP);
rs_status tc_build_bimage(int n, int RP, const float* wt, uint16_t* img, float* csc, cudaStream_t st);
rs_status device_alloc(rs_protein* p, void** ptr, size_t bytes);
}  // namespace rs

// ---------------------------------------------------------------- device helpers
namespace rs {
namespace dev {

// The pair arithmetic below is written with explicit round-to-nearest intrinsics:
// the compiler may not fuse a product into a following sum there, which keeps the
// error-free transformations exact and makes every kernel that uses them compute
// the same bits from the same inputs.

// Error-free sum of two floats (Knuth TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Unevaluated float pair hi + lo (about 48 significant bits).
struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// Pair value a + f*d with a, d pairs and f a float in [0, 1].
__device__ __forceinline__ F2 df_lerp(F2 a, F2 d, float f) {
    float p = __fmul_rn(f, d.h);
    float ep = __fmaf_rn(f, d.h, -p);
    float s, e;
    two_sum(a.h, p, s, e);
    float lo = __fadd_rn(__fadd_rn(e, ep), __fmaf_rn(f, d.l, a.l));
    return fast_two_sum(s, lo);
}

// acc += x * y for pairs x, y, in the manner of the compensated dot product
// Dot2 (Ogita, Rump, Oishi 2005): the rounding errors of the leading product and
// sum are carried in acc.l (the lo*lo term is dropped).
__device__ __forceinline__ void df_fma_acc(F2& acc, F2 x, F2 y) {
    float p = __fmul_rn(x.h, y.h);
    float ep = __fmaf_rn(x.h, y.h, -p);
    float s, e;
    two_sum(acc.h, p, s, e);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(__fadd_rn(e, ep), __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.h))));
}

// Pair product a*b (the lo*lo term dropped; about 2^-47 relative).
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

// acc += x for pairs (the rounding error of the leading sum is carried in acc.l).
__device__ __forceinline__ void df_acc(F2& acc, F2 x) {
    float s, e;
    two_sum(acc.h, x.h, s, e);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(e, x.l));
}

// Renormalised pair (hi = the float nearest hi + lo) of an accumulator.
__device__ __forceinline__ F2 df_norm(F2 a) {
    float s, e;
    two_sum(a.h, a.l, s, e);
    return {s, e};
}

// a + b and a - b for pairs (results renormalised).
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return fast_two_sum(s, e);
}
__device__ __forceinline__ F2 df_sub(F2 a, F2 b) { return df_add(a, F2{-b.h, -b.l}); }

// a < b for renormalised pairs.
__device__ __forceinline__ bool df_lt(F2 a, F2 b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }

// Pair nearest a double (hi = the float nearest v, lo = the float nearest v - hi),
// and back.  Values must stay inside the float range.
__device__ __forceinline__ F2 df_from(double v) {
    float h = __double2float_rn(v);
    return {h, __double2float_rn(__dsub_rn(v, (double)h))};
}
__device__ __forceinline__ double df_to(F2 a) { return __dadd_rn((double)a.h, (double)a.l); }

// Accumulator of float values carried as an unevaluated pair hi + lo.
struct FAcc {
    float hi, lo;
    __device__ __forceinline__ FAcc() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ void add(float x) {
        float s, e;
        two_sum(hi, x, s, e);
        lo += e;
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Rotation matrix of a (not necessarily unit) quaternion (w, x, y, z), FP64.
__device__ __forceinline__ void quat_to_rot(double w, double x, double y, double z, double* R) {
    double nrm = sqrt(w * w + x * x + y * y + z * z);
    double s = nrm > 0.0 ? 1.0 / nrm : 0.0;
    w *= s; x *= s; y *= s; z *= s;
    if (nrm == 0.0) w = 1.0;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// R = exp([w]x) by Rodrigues' formula; series coefficients for small angles.
__device__ __forceinline__ void rotvec_to_rot(double wx, double wy, double wz, double* R) {
    double th2 = wx * wx + wy * wy + wz * wz;
    double th = sqrt(th2);
    double A, B;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    // K = [w]x ; K^2 = w w^T - th2 I
    R[0] = 1 + B * (wx * wx - th2); R[1] = -A * wz + B * wx * wy; R[2] = A * wy + B * wx * wz;
    R[3] = A * wz + B * wx * wy; R[4] = 1 + B * (wy * wy - th2); R[5] = -A * wx + B * wy * wz;
    R[6] = -A * wy + B * wx * wz; R[7] = A * wx + B * wy * wz; R[8] = 1 + B * (wz * wz - th2);
}

// SO(3) left Jacobian J_l(w) = I + (1-cos t)/t^2 [w]x + (t - sin t)/t^3 [w]x^2.
__device__ __forceinline__ void left_jacobian(double wx, double wy, double wz, double* J) {
    double th2 = wx * wx + wy * wy + wz * wz;
    double th = sqrt(th2);
    double B, C;
    if (th < 1e-4) {
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    J[0] = 1 + C * (wx * wx - th2); J[1] = -B * wz + C * wx * wy; J[2] = B * wy + C * wx * wz;
    J[3] = B * wz + C * wx * wy; J[4] = 1 + C * (wy * wy - th2); J[5] = -B * wx + C * wy * wz;
    J[6] = -B * wy + C * wx * wz; J[7] = B * wx + C * wy * wz; J[8] = 1 + C * (wz * wz - th2);
}

// Cell index and fraction along one axis from a coordinate x given as a float pair:
// s = (x + b)/h (pair arithmetic); i = clamp(floor(s), 0, n-2), f = clamp(s - i, 0, 1);
// inside = 0 <= s <= n-1, decided on the pair.
__device__ __forceinline__ void axis_cell(F2 x, F2 b, F2 inv_h, int n, int& i, float& f, bool& inside) {
    const F2 s = df_mul(df_add(x, b), inv_h);
    const float top = (float)(n - 1);
    inside = (s.h > 0.f || (s.h == 0.f && s.l >= 0.f)) && (s.h < top || (s.h == top && s.l <= 0.f));
    float fl = floorf(s.h);
    if (fl == s.h && s.l < 0.f) fl = __fsub_rn(fl, 1.f);
    fl = fminf(fmaxf(fl, 0.f), (float)(n - 2));
    i = (int)fl;
    const float fr = __fadd_rn(__fsub_rn(s.h, fl), s.l);
    f = fminf(fmaxf(fr, 0.f), 1.f);
}

}  // namespace dev
}  // namespace rs
