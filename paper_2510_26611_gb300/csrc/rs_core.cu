// Context, errors, parameters and the sinc table (host FP64) of librs.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "rs_common.cuh"

namespace rs {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_tc_mu;
int* g_tc_flag[kMaxDevices] = {};
std::atomic<int> g_wform_mode{1};
std::atomic<int> g_build_gemm_mode{1};
}  // namespace

int* tc_error_flag(int device) {
    if (device < 0 || device >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (!g_tc_flag[device]) {
        int* p = nullptr;
        if (cudaMalloc(&p, 256) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaMemset(p, 0, 256) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p);
            return nullptr;
        }
        g_tc_flag[device] = p;
    }
    return g_tc_flag[device];
}

int wform_kernel_mode() { return g_wform_mode.load(std::memory_order_relaxed); }
int build_gemm_mode() { return g_build_gemm_mode.load(std::memory_order_relaxed); }

double short_work_ops(bool grad, double atoms, double cand, double near) {
    return 230.0 * atoms + 6.0 * cand + (grad ? 179.0 : 121.0) * near;
}

unsigned long long* short_counters(int device, bool grad) {
    int* base = tc_error_flag(device);  // 256 bytes: the error count, then the counters
    if (!base) return nullptr;
    return reinterpret_cast<unsigned long long*>(base) + 8 + (grad ? 3 : 0);
}

namespace {
std::atomic<long long> g_tc_grid{0};
std::atomic<long long> g_tc_smem{0};
std::atomic<int> g_tc_per_sm{0};
}  // namespace

void note_tc_launch(long long grid, size_t smem, int per_sm) {
    g_tc_grid.store(grid, std::memory_order_relaxed);
    g_tc_smem.store((long long)smem, std::memory_order_relaxed);
    g_tc_per_sm.store(per_sm, std::memory_order_relaxed);
}

rs_status ensure_buffer(void** buf, size_t* cap, size_t need) {
    if (*cap >= need && *buf) return RS_OK;
    if (*buf) {
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    size_t sz = need < 4096 ? 4096 : need;
    if (cudaMalloc(buf, sz) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        set_error("cudaMalloc of %zu bytes failed", sz);
        return RS_ERR_OOM;
    }
    *cap = sz;
    return RS_OK;
}

rs_status device_alloc(rs_protein* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 256;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed", bytes);
        return RS_ERR_OOM;
    }
    p->allocations.push_back(*ptr);
    p->device_bytes += bytes;
    return RS_OK;
}

// Sum of Gaussians for 1/r (Sec. 2, Eq. sinc).  The substitution t = sinh(u)/B
// (B = 2 sqrt(3) b, the box diagonal) turns 1/r = (2/sqrt(pi)) int_0^inf
// exp(-r^2 t^2) dt into (1/B)(1/sqrt(pi)) int_R cosh(u) exp(-(r/B)^2 sinh(u)^2) du;
// the trapezoid rule with step h_s, with the +k and -k nodes merged, gives
// t_k = sinh(k h_s)/B and a_k = 2 h_s cosh(k h_s)/(sqrt(pi) B) (a_0 = h_s/(sqrt(pi) B)).
// The R_l widest terms are the long-range part (Eq. Split_Tens); h_s puts the
// narrowest of them at t = tau/sigma (TEP step 2).
rs_status make_sinc_table(double b, double sigma, int R_l, double r_min, double tau,
                          double short_tol, SincTable* out) {
    if (!(b > 0) || !(sigma > 0) || R_l < 2 || R_l > 64 || !(r_min > 0) || !(tau > 0) ||
        !(short_tol > 0)) {
        set_error("invalid sinc parameters (b=%g sigma=%g R_l=%d r_min=%g tau=%g tol=%g)", b,
                  sigma, R_l, r_min, tau, short_tol);
        return RS_ERR_INVALID;
    }
    const double sqrt_pi = std::sqrt(M_PI);
    SincTable T;
    T.R_l = R_l;
    T.box_len = 2.0 * std::sqrt(3.0) * b;
    T.h_s = std::asinh(tau * T.box_len / sigma) / (double)(R_l - 1);
    int K = (int)std::ceil(std::asinh(tau * T.box_len / r_min) / T.h_s);
    if (K < R_l - 1) K = R_l - 1;
    if (K + 1 - R_l > RS_MAX_SHORT) {
        set_error("sinc table needs %d short-range terms (max %d); raise r_min", K + 1 - R_l,
                  RS_MAX_SHORT);
        return RS_ERR_UNSUPPORTED;
    }
    for (int k = 0; k <= K; ++k) {
        double u = k * T.h_s;
        T.t.push_back(std::sinh(u) / T.box_len);
        double w = (k == 0 ? 1.0 : 2.0) * T.h_s * std::cosh(u) / sqrt_pi;
        T.a.push_back(w / T.box_len);
        T.is_long.push_back(k < R_l ? 1 : 0);
    }
    auto shortf = [&](double r) {
        double s = 0;
        for (size_t k = 0; k < T.t.size(); ++k)
            if (!T.is_long[k]) s += T.a[k] * std::exp(-T.t[k] * T.t[k] * r * r);
        return r * s;
    };
    T.quad_err = -1.0;  // measured on first request (sinc_quad_error)
    T.r_min = r_min;
    // short-range cutoff: beyond the peak of the widest short-range term every
    // short-range Gaussian decreases, so r*sum is decreasing there; bisect.
    double r_c = 0.0;
    if (K + 1 > R_l) {
        double tmin = T.t[R_l];
        double lo = 1.0 / (std::sqrt(2.0) * tmin), hi = T.box_len;
        if (shortf(hi) > short_tol) {
            r_c = hi;
        } else if (shortf(lo) <= short_tol) {
            // the sum is already below tolerance at the peak of the widest term;
            // walk down to the last point above it
            double r = lo;
            while (r > 1e-6 && shortf(r) <= short_tol) r *= 0.5;
            lo = r;
            hi = r * 2.0;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (shortf(mid) > short_tol) lo = mid; else hi = mid;
            }
            r_c = hi;
        } else {
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (shortf(mid) > short_tol) lo = mid; else hi = mid;
            }
            r_c = hi;
        }
    }
    T.r_c = r_c;
    *out = std::move(T);
    return RS_OK;
}

// Max relative error of sum_k a_k exp(-t_k^2 r^2) against 1/r on [r_min, B]
// (20001 geometrically spaced points): a diagnostic, computed once per table.
double sinc_quad_error(const SincTable& T) {
    const int M = 20001;
    double err = 0;
    for (int i = 0; i < M; ++i) {
        double r = T.r_min * std::pow(T.box_len / T.r_min, (double)i / (M - 1));
        double s = 0;
        for (size_t k = 0; k < T.t.size(); ++k) s += T.a[k] * std::exp(-T.t[k] * T.t[k] * r * r);
        double e = std::fabs(r * s - 1.0);
        if (e > err) err = e;
    }
    return err;
}

}  // namespace rs

extern "C" {

const char* rs_last_error(void) { return rs::g_last_error.c_str(); }

const char* rs_version(void) { return "librs 0.1 (sm_103a)"; }

void rs_params_default(rs_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->n = 257;
    p->b = 32.0;
    p->sigma = 3.0;
    p->R_l = 20;
    p->r_min = 0.5;
    p->tau = 4.0;
    p->short_tol = 1e-9;
    p->tucker_cap = 0;
    p->eps_r = 1e-7;
    p->galerkin = 0;
}

rs_status rs_ctx_create(int device, rs_ctx** out) {
    rs::clear_error();
    if (!out) {
        rs::set_error("rs_ctx_create: out is NULL");
        return RS_ERR_INVALID;
    }
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        rs::set_error("rs_ctx_create: no CUDA device available");
        return RS_ERR_CUDA;
    }
    if (device < 0 || device >= count) {
        rs::set_error("rs_ctx_create: device %d out of range [0, %d)", device, count);
        return RS_ERR_INVALID;
    }
    RS_TRY_CUDA(cudaSetDevice(device));
    if (!rs::tc_error_flag(device)) {
        rs::set_error("rs_ctx_create: device allocation failed");
        return RS_ERR_OOM;
    }
    rs_ctx* c = new rs_ctx();
    c->device = device;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        rs::set_error("rs_ctx_create: cudaStreamCreate failed");
        return RS_ERR_CUDA;
    }
    *out = c;
    return RS_OK;
}

void rs_ctx_destroy(rs_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->lig_buf) cudaFree(c->lig_buf);
    if (c->io_buf) cudaFree(c->io_buf);
    if (c->ws_buf) cudaFree(c->ws_buf);
    if (c->pgd_buf) cudaFree(c->pgd_buf);
    if (c->eval_buf) cudaFree(c->eval_buf);
    if (c->fd_buf) cudaFree(c->fd_buf);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

void rs_protein_free(rs_protein* p) {
    if (!p) return;
    if (p->children > 0) {  // local-box handles still read its short-range data
        p->released = true;
        return;
    }
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    for (void* a : p->allocations) cudaFree(a);
    rs_protein* parent = p->parent;
    delete p;
    if (parent && --parent->children == 0 && parent->released) {
        parent->released = false;
        rs_protein_free(parent);
    }
}

rs_status rs_protein_get_info(const rs_protein* p, rs_protein_info* o) {
    rs::clear_error();
    if (!p || !o) {
        rs::set_error("rs_protein_get_info: NULL argument");
        return RS_ERR_INVALID;
    }
    memset(o, 0, sizeof(*o));
    o->n = p->n;
    o->N = p->N;
    o->R_l = p->R_l;
    o->K = p->K;
    o->b = p->b;
    o->h = p->h;
    o->sigma = p->sigma;
    o->r_c = p->table.r_c;
    o->h_s = p->table.h_s;
    if (p->table.quad_err < 0) const_cast<rs_protein*>(p)->table.quad_err = rs::sinc_quad_error(p->table);
    o->quad_err = p->table.quad_err;
    o->kind = p->kind;
    for (int a = 0; a < 3; ++a) {
        o->rank[a] = p->rank[a];
        o->sv_gap[a] = p->sv_gap[a];
        o->sv_tail[a] = p->sv_tail[a];
    }
    o->device_bytes = p->device_bytes;
    return RS_OK;
}

int rs_set_wform_kernel(int mode) {
    return rs::g_wform_mode.exchange(mode ? 1 : 0);
}

int rs_set_build_gemm_kernel(int mode) {
    return rs::g_build_gemm_mode.exchange(mode ? 1 : 0);
}

rs_status rs_tc_error_count(int device, int32_t* out) {
    rs::clear_error();
    if (!out) {
        rs::set_error("rs_tc_error_count: out is NULL");
        return RS_ERR_INVALID;
    }
    *out = 0;
    RS_TRY_CUDA(cudaSetDevice(device));
    int* p = rs::tc_error_flag(device);
    if (!p) {
        rs::set_error("rs_tc_error_count: device %d unavailable", device);
        return RS_ERR_INVALID;
    }
    RS_TRY_CUDA(cudaMemcpy(out, p, sizeof(int), cudaMemcpyDeviceToHost));
    return RS_OK;
}

rs_status rs_diag_short_counts(int device, int grad, uint64_t* counts, double* fp32_ops, int reset) {
    rs::clear_error();
    if (!counts || !fp32_ops) {
        rs::set_error("rs_diag_short_counts: NULL argument");
        return RS_ERR_INVALID;
    }
    RS_TRY_CUDA(cudaSetDevice(device));
    unsigned long long* p = rs::short_counters(device, grad != 0);
    if (!p) {
        rs::set_error("rs_diag_short_counts: device %d unavailable", device);
        return RS_ERR_INVALID;
    }
    RS_TRY_CUDA(cudaDeviceSynchronize());
    unsigned long long h[3];
    RS_TRY_CUDA(cudaMemcpy(h, p, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 3; ++i) counts[i] = h[i];
    *fp32_ops = rs::short_work_ops(grad != 0, (double)h[0], (double)h[1], (double)h[2]);
    if (reset) RS_TRY_CUDA(cudaMemset(p, 0, sizeof(h)));
    return RS_OK;
}

rs_status rs_diag_tc_launch(int64_t* grid, int64_t* smem, int32_t* per_sm) {
    rs::clear_error();
    if (!grid || !smem || !per_sm) {
        rs::set_error("rs_diag_tc_launch: NULL argument");
        return RS_ERR_INVALID;
    }
    *grid = rs::g_tc_grid.load();
    *smem = rs::g_tc_smem.load();
    *per_sm = rs::g_tc_per_sm.load();
    return RS_OK;
}

rs_status rs_protein_get_table(const rs_protein* p, double* t, double* a, uint8_t* is_long) {
    rs::clear_error();
    if (!p || !t || !a || !is_long) {
        rs::set_error("rs_protein_get_table: NULL argument");
        return RS_ERR_INVALID;
    }
    for (int k = 0; k < p->K; ++k) {
        t[k] = p->table.t[k];
        a[k] = p->table.a[k];
        is_long[k] = p->table.is_long[k];
    }
    return RS_OK;
}

}  // extern "C"
