// B images of the W form for the tensor-core evaluation, and a diagnostic entry that
// runs the contraction of one tile alone.
#include <cmath>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_tc.cuh"

namespace rs {
namespace {

// For every axis-3 cell i and column nn = 2a + t of B (t = 0: row a of W[i], t = 1:
// row a of D[i]; K = the axis-2 index b): the BF16 slices of the row (float pairs)
// relative to its power-of-two scale, cut exactly in FP32 by slice5 (the same
// slicing as the A rows of the pose kernels), written in the canonical K-major layout
// the MMA reads, eight K values per 16-byte store; csc = the inverse scale.
__global__ void k_tc_bimage(int n, int RP, const float* __restrict__ wt, uint16_t* __restrict__ img,
                            float* __restrict__ csc) {
    const int KP = tc::kp_of(RP), NP = tc::np_of(RP);
    const int nn = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (nn >= NP) return;
    const size_t plane = (size_t)n * RP * RP;
    const int a = nn >> 1, t = nn & 1;
    const float* wh = wt + 2 * t * plane + ((size_t)i * RP + a) * RP;
    const float* wl = wt + (2 * t + 1) * plane + ((size_t)i * RP + a) * RP;
    const bool row = a < RP;
    float m = 0.f;
    if (row)
        for (int b = 0; b < RP; ++b) m = fmaxf(m, fabsf(wh[b]));
    float s, inv;
    tc::row_scale(m, s, inv);
    const size_t slice = (size_t)NP * KP;
    uint16_t* base = img + (size_t)i * tc::kSlices * slice;
    const uint32_t sbo = (uint32_t)KP * 16;
    for (int k8 = 0; k8 < KP; k8 += 8) {
        uint32_t w[tc::kSlices][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float lo[tc::kSlices], hi[tc::kSlices];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int b = k8 + e + hh;
                const dev::F2 x = (row && b < RP) ? dev::F2{__fmul_rn(wh[b], s), __fmul_rn(wl[b], s)}
                                                  : dev::F2{0.f, 0.f};
                tc::slice5(x, hh ? hi : lo);
            }
#pragma unroll
            for (int j = 0; j < tc::kSlices; ++j) w[j][e / 2] = tc::pack_bf16x2(lo[j], hi[j]);
        }
#pragma unroll
        for (int j = 0; j < tc::kSlices; ++j)
            *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(base + j * slice) +
                                      tc::kmajor_offset(nn, k8, sbo)) = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
    }
    csc[(size_t)i * NP + nn] = inv;
}

// One tile of the contraction: rows v (pairs from FP64), B image of cell 0.
template <int RP>
__global__ void __launch_bounds__(tc::kTileRows)
    k_diag_tc(int rows, const double* __restrict__ v, const uint16_t* __restrict__ img,
              const float* __restrict__ csc, double* __restrict__ X, double* __restrict__ Xd,
              int* __restrict__ err) {
    using S = tc::Shape<RP>;
    extern __shared__ __align__(16) uint8_t smem_d[];
    uint8_t* sA = smem_d;
    uint8_t* sB = sA + tc::kSlices * S::A_SLICE;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + S::B_BYTES);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr uint32_t USED = tc::kAccs * S::NP;
    constexpr uint32_t NCOL = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : 256;
    if (warp == 0) tc::tmem_alloc(slot, NCOL);
    if (tid == 0) tc::mbar_init(bar, 1);
    for (int e = tid; e < (int)(S::B_BYTES / 16); e += tc::kTileRows)
        reinterpret_cast<uint4*>(sB)[e] = reinterpret_cast<const uint4*>(img)[e];
    float inv = 0.f;
    if (tid < rows) {
        dev::F2 x[RP];
        for (int b = 0; b < RP; ++b) x[b] = dev::df_from(v[(size_t)tid * RP + b]);
        inv = tc::write_row<RP>(x, sA, tid);
    } else {
        tc::zero_row<RP>(sA, tid);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    if (tid == 0) {
        tc::issue_products<RP>(tmem, tc::smem_u32(sA), tc::smem_u32(sB));
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        tc::fence_after_sync();
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int ch = 0; ch < S::NP / 16; ++ch) {
            float x0[16], x1[16];
            tc::tmem_ld16x2(tl + ch * 16, tl + S::NP + ch * 16, x0, x1);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int a = ch * 8 + q;
                if (a < RP && tid < rows) {
                    const dev::F2 w = tc::combine(x0[2 * q], x1[2 * q], __fmul_rn(inv, csc[2 * a]));
                    const dev::F2 d = tc::combine(x0[2 * q + 1], x1[2 * q + 1], __fmul_rn(inv, csc[2 * a + 1]));
                    X[(size_t)tid * RP + a] = dev::df_to(w);
                    Xd[(size_t)tid * RP + a] = dev::df_to(d);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
}

template <int RP>
rs_status run_diag_tc(int rows, const double* dv, const uint16_t* img, const float* csc, double* dX, double* dXd,
                      int* derr, cudaStream_t st) {
    using S = tc::Shape<RP>;
    const size_t smem = tc::kSlices * S::A_SLICE + S::B_BYTES + 16;
    auto kern = k_diag_tc<RP>;
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        ::rs::KernelTimer kt__("k_diag_tc", st, 0.0, false);
        kern<<<1, tc::kTileRows, smem, st>>>(rows, dv, img, csc, dX, dXd, derr);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

}  // namespace

size_t tc_bimage_bytes(int n, int RP) {
    return (size_t)n * tc::kSlices * tc::np_of(RP) * tc::kp_of(RP) * sizeof(uint16_t);
}

size_t tc_bscale_bytes(int n, int RP) { return (size_t)n * tc::np_of(RP) * sizeof(float); }

rs_status tc_build_bimage(int n, int RP, const float* wt, uint16_t* img, float* csc, cudaStream_t st) {
    const int NP = tc::np_of(RP);
    {
        ::rs::KernelTimer kt__("k_tc_bimage", st, 0.0, false);
        k_tc_bimage<<<dim3((NP + 63) / 64, n), 64, 0, st>>>(n, RP, wt, img, csc);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

}  // namespace rs

extern "C" rs_status rs_diag_tc_contract(int32_t RP, int32_t rows, const double* v, const double* W,
                                         const double* D, double* X, double* Xd) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(v && W && D && X && Xd, "rs_diag_tc_contract: NULL argument");
    RS_CHECK_ARG(RP >= 4 && RP <= 32 && RP % 4 == 0, "rs_diag_tc_contract: RP=%d not in {4, 8, ..., 32}", RP);
    RS_CHECK_ARG(rows >= 1 && rows <= tc::kTileRows, "rs_diag_tc_contract: rows=%d out of [1, 128]", rows);
    // W-form planes of one cell (n = 1): Wh, Wl, Dh, Dl as float pairs of W and D
    std::vector<float> wt(4 * (size_t)RP * RP);
    for (size_t e = 0; e < (size_t)RP * RP; ++e) {
        const double w = W[e], d = D[e];
        const float wh = (float)w, dh = (float)d;
        wt[e] = wh;
        wt[(size_t)RP * RP + e] = (float)(w - (double)wh);
        wt[2 * (size_t)RP * RP + e] = dh;
        wt[3 * (size_t)RP * RP + e] = (float)(d - (double)dh);
    }
    const size_t img_b = tc_bimage_bytes(1, RP), csc_b = tc_bscale_bytes(1, RP);
    const size_t vb = (size_t)rows * RP * sizeof(double);
    char* buf = nullptr;
    const size_t total = wt.size() * 4 + img_b + csc_b + vb * 3 + 256 * 8;
    RS_TRY_CUDA(cudaMalloc(&buf, total));
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char* p = buf;
    float* d_wt = (float*)p;
    p += al(wt.size() * 4);
    uint16_t* d_img = (uint16_t*)p;
    p += al(img_b);
    float* d_csc = (float*)p;
    p += al(csc_b);
    double* d_v = (double*)p;
    p += al(vb);
    double* d_X = (double*)p;
    p += al(vb);
    double* d_Xd = (double*)p;
    p += al(vb);
    int* d_err = (int*)p;
    rs_status st = RS_OK;
    cudaStream_t s = nullptr;
    int herr = 0;
    do {
        if (cudaMemcpy(d_wt, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_v, v, vb, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) {
            set_error("rs_diag_tc_contract: copy failed");
            st = RS_ERR_CUDA;
            break;
        }
        st = tc_build_bimage(1, RP, d_wt, d_img, d_csc, s);
        if (st != RS_OK) break;
        switch (RP) {
#define RS_CASE(R) \
    case R: st = run_diag_tc<R>(rows, d_v, d_img, d_csc, d_X, d_Xd, d_err, s); break;
            RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        }
        if (st != RS_OK) break;
        if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(X, d_X, vb, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(Xd, d_Xd, vb, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("rs_diag_tc_contract: %s", cudaGetErrorString(cudaGetLastError()));
            st = RS_ERR_CUDA;
            break;
        }
        if (herr) {
            set_error("rs_diag_tc_contract: MMA did not complete");
            st = RS_ERR_CUDA;
        }
    } while (0);
    cudaFree(buf);
    return st;
}
