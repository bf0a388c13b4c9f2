// Local-box handles: scheme (C) of Sec. 3.2 (Table 1).  The global Tucker potential is
// restricted to the grid nodes of a box Pi and re-truncated there by an HOSVD of the
// restricted node tensor, which has lower multilinear ranks than the whole box's
// (the potential of the protein seen from a small region outside it is smoother).
//
// The restricted tensor is read from the handle's own evaluation tables (the float
// pairs the pose kernels evaluate), in the W form
//   T[i1, i2, i3] = sum_ab A1[i1, a] A2[i2, b] W[i3, a, b],
// and reduced on the host in FP64 (matrices of at most 32 columns and 512 rows):
//   A_l = Q_l R_l             (orthonormal Q_l from the Gram A_l^T A_l, l = 1, 2)
//   C[i3, a', b'] = sum_ab R1[a', a] R2[b', b] W[i3, a, b]
//   mode Grams of C -> left singular vectors U_1, U_2, U_3 and singular values,
//   ranks r_l = #{s_i > eps s_1}
//   A_l'' = Q_l U_l[:, :r_l],  W''[i3] = P_3 (U_1^T C U_2)[i3],  P_3 = U_3 U_3^T (r_3 columns)
// The new tables are laid out like a build's (rows outside the box zero) and the
// handle shares its parent's short-range data.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_tc.cuh"

namespace rs {
namespace {

constexpr int kMaxBoxRows = 512;

// Eigen-decomposition of a symmetric m x m matrix (descending), via the library's
// host solver.
rs_status eig(int m, const std::vector<double>& A, std::vector<double>& lam, std::vector<double>& V) {
    lam.assign(m, 0.0);
    V.assign((size_t)m * m, 0.0);
    return rs_symeig_host(m, A.data(), lam.data(), V.data());
}

// Rank from eigenvalues of a Gram (squared singular values), relative threshold eps.
int rank_of(const std::vector<double>& lam, double eps, int cap) {
    const double s1 = lam.empty() ? 0.0 : std::sqrt(std::max(lam[0], 0.0));
    int r = 0;
    for (double l : lam)
        if (std::sqrt(std::max(l, 0.0)) > eps * s1) ++r;
    return std::max(1, std::min(r, cap));
}

void split(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

}  // namespace
}  // namespace rs

extern "C" rs_status rs_protein_local_box(rs_ctx* ctx, rs_protein* parent, const double* lo, const double* hi,
                                          double eps, rs_protein** out) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && parent && lo && hi && out, "rs_protein_local_box: NULL argument");
    *out = nullptr;
    RS_CHECK_ARG(parent->kind == 1 && parent->view.kind == 1, "rs_protein_local_box: the protein is not Tucker-reduced");
    RS_CHECK_ARG(!parent->view.box, "rs_protein_local_box: the protein is already a local-box handle");
    RS_CHECK_ARG(std::isfinite(eps) && eps >= 0.0 && eps < 1.0, "rs_protein_local_box: eps=%g not in [0, 1)", eps);
    RS_CHECK_ARG(parent->device == ctx->device, "protein built on device %d, context on %d", parent->device,
                 ctx->device);
    const int n = parent->n, RP = parent->view.R;
    const double b = parent->b, h = parent->h;
    int c0[3], c1[3], m[3];
    for (int a = 0; a < 3; ++a) {
        RS_CHECK_ARG(std::isfinite(lo[a]) && std::isfinite(hi[a]) && lo[a] < hi[a],
                     "rs_protein_local_box: box axis %d is empty or not finite", a);
        c0[a] = (int)std::min(std::max(std::floor((lo[a] + b) / h), 0.0), (double)(n - 2));
        c1[a] = (int)std::min(std::max(std::ceil((hi[a] + b) / h) - 1.0, (double)c0[a]), (double)(n - 2));
        m[a] = c1[a] - c0[a] + 2;  // the cells' nodes
        RS_CHECK_ARG(m[a] <= kMaxBoxRows, "rs_protein_local_box: the box spans %d grid rows on axis %d (at most %d)",
                     m[a], a, kMaxBoxRows);
    }
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    RS_TRY_CUDA(cudaDeviceSynchronize());
    // 1. the parent's tables on the box rows, as FP64
    const size_t vplane = (size_t)n * RP, wplane = (size_t)n * RP * RP;
    std::vector<double> A[2], Wr((size_t)m[2] * RP * RP);
    for (int a = 0; a < 2; ++a) {
        std::vector<float> hb((size_t)m[a] * RP), lb((size_t)m[a] * RP);
        RS_TRY_CUDA(cudaMemcpy(hb.data(), parent->view.Vt[a][0] + (size_t)c0[a] * RP, hb.size() * 4,
                               cudaMemcpyDeviceToHost));
        RS_TRY_CUDA(cudaMemcpy(lb.data(), parent->view.Vt[a][1] + (size_t)c0[a] * RP, lb.size() * 4,
                               cudaMemcpyDeviceToHost));
        A[a].resize(hb.size());
        for (size_t e = 0; e < hb.size(); ++e) A[a][e] = (double)hb[e] + (double)lb[e];
    }
    {
        std::vector<float> hb(Wr.size()), lb(Wr.size());
        RS_TRY_CUDA(cudaMemcpy(hb.data(), parent->view.Wt[0] + (size_t)c0[2] * RP * RP, hb.size() * 4,
                               cudaMemcpyDeviceToHost));
        RS_TRY_CUDA(cudaMemcpy(lb.data(), parent->view.Wt[1] + (size_t)c0[2] * RP * RP, lb.size() * 4,
                               cudaMemcpyDeviceToHost));
        for (size_t e = 0; e < Wr.size(); ++e) Wr[e] = (double)hb[e] + (double)lb[e];
    }
    // 2. A_l = Q_l R_l through the Gram's eigenvectors
    std::vector<double> Q[2], R[2];
    int k[2];
    for (int a = 0; a < 2; ++a) {
        std::vector<double> G((size_t)RP * RP, 0.0), lam, E;
        for (int i = 0; i < m[a]; ++i)
            for (int p = 0; p < RP; ++p)
                for (int q = 0; q < RP; ++q) G[(size_t)p * RP + q] += A[a][(size_t)i * RP + p] * A[a][(size_t)i * RP + q];
        RS_TRY(eig(RP, G, lam, E));
        int kk = 0;
        while (kk < RP && lam[kk] > 1e-26 * std::max(lam[0], 1e-300)) ++kk;
        kk = std::max(kk, 1);
        k[a] = kk;
        Q[a].assign((size_t)m[a] * kk, 0.0);
        R[a].assign((size_t)kk * RP, 0.0);
        for (int c = 0; c < kk; ++c) {
            const double s = std::sqrt(std::max(lam[c], 1e-300));
            for (int q = 0; q < RP; ++q) R[a][(size_t)c * RP + q] = s * E[(size_t)q * RP + c];
            for (int i = 0; i < m[a]; ++i) {
                double acc = 0.0;
                for (int q = 0; q < RP; ++q) acc += A[a][(size_t)i * RP + q] * E[(size_t)q * RP + c];
                Q[a][(size_t)i * kk + c] = acc / s;
            }
        }
    }
    const int k1 = k[0], k2 = k[1], m3 = m[2];
    // 3. C[i3][a'][b'] = sum_ab R1[a'][a] R2[b'][b] W[i3][a][b]
    std::vector<double> C((size_t)m3 * k1 * k2, 0.0);
    {
        std::vector<double> tmp((size_t)k1 * RP);
        for (int i = 0; i < m3; ++i) {
            const double* w = Wr.data() + (size_t)i * RP * RP;
            std::fill(tmp.begin(), tmp.end(), 0.0);
            for (int p = 0; p < k1; ++p)
                for (int a = 0; a < RP; ++a) {
                    const double r = R[0][(size_t)p * RP + a];
                    for (int bb = 0; bb < RP; ++bb) tmp[(size_t)p * RP + bb] += r * w[(size_t)a * RP + bb];
                }
            double* c = C.data() + (size_t)i * k1 * k2;
            for (int p = 0; p < k1; ++p)
                for (int q = 0; q < k2; ++q) {
                    double acc = 0.0;
                    for (int bb = 0; bb < RP; ++bb) acc += tmp[(size_t)p * RP + bb] * R[1][(size_t)q * RP + bb];
                    c[(size_t)p * k2 + q] = acc;
                }
        }
    }
    // 4. mode Grams, left singular vectors, ranks
    std::vector<double> M1((size_t)k1 * k1, 0.0), M2((size_t)k2 * k2, 0.0), M3((size_t)m3 * m3, 0.0);
    for (int i = 0; i < m3; ++i) {
        const double* c = C.data() + (size_t)i * k1 * k2;
        for (int p = 0; p < k1; ++p)
            for (int p2 = 0; p2 < k1; ++p2) {
                double acc = 0.0;
                for (int q = 0; q < k2; ++q) acc += c[(size_t)p * k2 + q] * c[(size_t)p2 * k2 + q];
                M1[(size_t)p * k1 + p2] += acc;
            }
        for (int q = 0; q < k2; ++q)
            for (int q2 = 0; q2 < k2; ++q2) {
                double acc = 0.0;
                for (int p = 0; p < k1; ++p) acc += c[(size_t)p * k2 + q] * c[(size_t)p * k2 + q2];
                M2[(size_t)q * k2 + q2] += acc;
            }
    }
    for (int i = 0; i < m3; ++i)
        for (int j = 0; j <= i; ++j) {
            double acc = 0.0;
            const double *ci = C.data() + (size_t)i * k1 * k2, *cj = C.data() + (size_t)j * k1 * k2;
            for (int e = 0; e < k1 * k2; ++e) acc += ci[e] * cj[e];
            M3[(size_t)i * m3 + j] = M3[(size_t)j * m3 + i] = acc;
        }
    std::vector<double> lam1, U1, lam2, U2, lam3, U3;
    RS_TRY(eig(k1, M1, lam1, U1));
    RS_TRY(eig(k2, M2, lam2, U2));
    RS_TRY(eig(m3, M3, lam3, U3));
    const int r1 = rank_of(lam1, eps, 32), r2 = rank_of(lam2, eps, 32), r3 = rank_of(lam3, eps, m3);
    const int RN = (std::max(r1, r2) + 3) / 4 * 4;
    // 5. new factors and W'' = P3 (U1^T C U2)
    std::vector<double> F[2];
    const int rr[2] = {r1, r2};
    const std::vector<double>* Us[2] = {&U1, &U2};
    for (int a = 0; a < 2; ++a) {
        F[a].assign((size_t)m[a] * RN, 0.0);
        const int kk = k[a];
        for (int i = 0; i < m[a]; ++i)
            for (int c = 0; c < rr[a]; ++c) {
                double acc = 0.0;
                for (int p = 0; p < kk; ++p) acc += Q[a][(size_t)i * kk + p] * (*Us[a])[(size_t)p * kk + c];
                F[a][(size_t)i * RN + c] = acc;
            }
    }
    std::vector<double> Wp((size_t)m3 * RN * RN, 0.0), Wn((size_t)m3 * RN * RN, 0.0);
    for (int i = 0; i < m3; ++i) {
        const double* c = C.data() + (size_t)i * k1 * k2;
        for (int x = 0; x < r1; ++x)
            for (int y = 0; y < r2; ++y) {
                double acc = 0.0;
                for (int p = 0; p < k1; ++p) {
                    double t = 0.0;
                    for (int q = 0; q < k2; ++q) t += c[(size_t)p * k2 + q] * U2[(size_t)q * k2 + y];
                    acc += U1[(size_t)p * k1 + x] * t;
                }
                Wp[((size_t)i * RN + x) * RN + y] = acc;
            }
    }
    {
        // P3 = U3r U3r^T applied along i3
        std::vector<double> proj((size_t)r3 * RN * RN, 0.0);
        for (int c = 0; c < r3; ++c)
            for (int i = 0; i < m3; ++i) {
                const double u = U3[(size_t)i * m3 + c];
                const double* w = Wp.data() + (size_t)i * RN * RN;
                double* o = proj.data() + (size_t)c * RN * RN;
                for (int e = 0; e < RN * RN; ++e) o[e] += u * w[e];
            }
        for (int i = 0; i < m3; ++i)
            for (int c = 0; c < r3; ++c) {
                const double u = U3[(size_t)i * m3 + c];
                const double* pr = proj.data() + (size_t)c * RN * RN;
                double* o = Wn.data() + (size_t)i * RN * RN;
                for (int e = 0; e < RN * RN; ++e) o[e] += u * pr[e];
            }
    }
    // 6. tables in the build's layout, rows outside the box zero
    const size_t vpn = (size_t)n * RN, wpn = (size_t)n * RN * RN;
    std::vector<float> vt[2] = {std::vector<float>(4 * vpn, 0.f), std::vector<float>(4 * vpn, 0.f)};
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < m[a]; ++i)
            for (int c = 0; c < RN; ++c) {
                const size_t o = (size_t)(c0[a] + i) * RN + c;
                const double v = F[a][(size_t)i * RN + c];
                const double vn = i + 1 < m[a] ? F[a][(size_t)(i + 1) * RN + c] : 0.0;
                split(v, vt[a][o], vt[a][vpn + o]);
                split(vn - v, vt[a][2 * vpn + o], vt[a][3 * vpn + o]);
            }
    std::vector<float> wt(4 * wpn, 0.f);
    for (int i = 0; i < m3; ++i)
        for (int e = 0; e < RN * RN; ++e) {
            const size_t o = (size_t)(c0[2] + i) * RN * RN + e;
            const double w = Wn[(size_t)i * RN * RN + e];
            const double wn = i + 1 < m3 ? Wn[(size_t)(i + 1) * RN * RN + e] : 0.0;
            split(w, wt[o], wt[wpn + o]);
            split(wn - w, wt[2 * wpn + o], wt[3 * wpn + o]);
        }
    rs_protein* P = new rs_protein();
    P->device = parent->device;
    P->n = n;
    P->N = parent->N;
    P->R_l = parent->R_l;
    P->K = parent->K;
    P->b = b;
    P->h = h;
    P->sigma = parent->sigma;
    P->table = parent->table;
    P->kind = 1;
    P->rank[0] = r1;
    P->rank[1] = r2;
    P->rank[2] = r3;
    const std::vector<double>* lams[3] = {&lam1, &lam2, &lam3};
    const int rk[3] = {r1, r2, r3};
    for (int a = 0; a < 3; ++a) {
        const auto& L = *lams[a];
        double tail = 0.0;
        for (size_t i = rk[a]; i < L.size(); ++i) tail += std::max(L[i], 0.0);
        const double s1 = std::sqrt(std::max(L[0], 1e-300));
        P->sv_tail[a] = std::sqrt(tail) / s1;
        P->sv_gap[a] = (size_t)rk[a] < L.size() && L[rk[a]] > 0 ? std::sqrt(L[rk[a] - 1] / L[rk[a]]) : 0.0;
    }
    P->view = parent->view;
    ProteinView& v = P->view;
    auto alloc = [&](void** p, size_t bytes) -> rs_status {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("rs_protein_local_box: device allocation of %zu bytes failed", bytes);
            return RS_ERR_OOM;
        }
        P->allocations.push_back(*p);
        P->device_bytes += bytes;
        return RS_OK;
    };
    float *d_vt0 = nullptr, *d_vt1 = nullptr, *d_wt = nullptr, *d_wsc = nullptr;
    uint16_t* d_wtc = nullptr;
    rs_status st = RS_OK;
    do {
        if ((st = alloc((void**)&d_vt0, 4 * vpn * 4)) != RS_OK || (st = alloc((void**)&d_vt1, 4 * vpn * 4)) != RS_OK ||
            (st = alloc((void**)&d_wt, 4 * wpn * 4)) != RS_OK ||
            (st = alloc((void**)&d_wtc, tc_bimage_bytes(n, RN))) != RS_OK ||
            (st = alloc((void**)&d_wsc, tc_bscale_bytes(n, RN))) != RS_OK)
            break;
        if (cudaMemcpy(d_vt0, vt[0].data(), 4 * vpn * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_vt1, vt[1].data(), 4 * vpn * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_wt, wt.data(), 4 * wpn * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("rs_protein_local_box: upload failed");
            st = RS_ERR_CUDA;
            break;
        }
        if ((st = tc_build_bimage(n, RN, d_wt, d_wtc, d_wsc, nullptr)) != RS_OK) break;
        if (cudaDeviceSynchronize() != cudaSuccess) {
            set_error("rs_protein_local_box: %s", cudaGetErrorString(cudaGetLastError()));
            st = RS_ERR_CUDA;
        }
    } while (0);
    if (st != RS_OK) {
        for (void* p : P->allocations) cudaFree(p);
        delete P;
        return st;
    }
    v.R = RN;
    v.ld = RN;
    v.core = nullptr;
    v.Wtc = d_wtc;
    v.Wsc = d_wsc;
    for (int q = 0; q < 4; ++q) {
        v.Wt[q] = d_wt + q * wpn;
        v.Vt[0][q] = d_vt0 + q * vpn;
        v.Vt[1][q] = d_vt1 + q * vpn;
    }
    v.box = 1;
    for (int a = 0; a < 3; ++a) {
        v.cell_lo[a] = c0[a];
        v.cell_hi[a] = c1[a];
    }
    P->parent = parent;
    parent->children++;
    *out = P;
    return RS_OK;
}
