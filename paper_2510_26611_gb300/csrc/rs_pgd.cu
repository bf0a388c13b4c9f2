// Constrained energy minimisation of rigid poses (Sec. 3.4, Eq. Energy_Min):
// arg min E(t, w) subject to dist(M, F(L)) >= sigma, by projected gradient descent
// on (translation, rotation vector) with backtracking:
//   step 0: dt = -eta_t g_t / |g_t|,  dw = -eta_r g_w / |g_w|   (g from the adjoint)
//   trial s = 0..max_halvings: (t + dt/2^s, w + dw/2^s); accept the first trial that
//   is feasible (flags == 0) and does not raise E; otherwise keep the pose.
// One step = a gradient pass and up to max_halvings+1 trial/energy/accept passes;
// it is captured once as a CUDA graph and replayed for every step.
#include <algorithm>
#include <cmath>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"

namespace rs {
namespace {

__global__ void k_pgd_init(long long P, uint8_t* __restrict__ done, int* __restrict__ accepted) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    done[p] = 0;
    accepted[p] = -1;
}

// Trial pose of halving level `level` for every pose not yet accepted.
__global__ void k_pgd_trial(long long P, int level, double eta_t, double eta_r,
                            const double* __restrict__ rv, const double* __restrict__ tr,
                            const double* __restrict__ gt, const double* __restrict__ gw,
                            const uint8_t* __restrict__ done, double* __restrict__ trv,
                            double* __restrict__ ttr, double* __restrict__ tq) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || done[p]) return;
    double sc = ldexp(1.0, -level);
    double g0 = gt[3 * p], g1 = gt[3 * p + 1], g2 = gt[3 * p + 2];
    double n = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    double ft = n > 0.0 ? -eta_t * sc / n : 0.0;
    double w0 = gw[3 * p], w1 = gw[3 * p + 1], w2 = gw[3 * p + 2];
    double m = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
    double fw = m > 0.0 ? -eta_r * sc / m : 0.0;
    double t[3] = {tr[3 * p] + ft * g0, tr[3 * p + 1] + ft * g1, tr[3 * p + 2] + ft * g2};
    double w[3] = {rv[3 * p] + fw * w0, rv[3 * p + 1] + fw * w1, rv[3 * p + 2] + fw * w2};
    for (int a = 0; a < 3; ++a) {
        ttr[3 * p + a] = t[a];
        trv[3 * p + a] = w[a];
    }
    // unit quaternion of exp([w]x): (cos(th/2), sin(th/2) w/th)
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double s = th < 1e-8 ? 0.5 - th * th / 48.0 : sin(0.5 * th) / th;
    tq[4 * p] = cos(0.5 * th);
    tq[4 * p + 1] = s * w[0];
    tq[4 * p + 2] = s * w[1];
    tq[4 * p + 3] = s * w[2];
}

__global__ void k_pgd_accept(long long P, int level, const double* __restrict__ E_cur,
                             const double* __restrict__ E_trial, const uint8_t* __restrict__ f_trial,
                             const double* __restrict__ trv, const double* __restrict__ ttr,
                             uint8_t* __restrict__ done, int* __restrict__ accepted,
                             double* __restrict__ rv, double* __restrict__ tr,
                             double* __restrict__ E_new, uint8_t* __restrict__ f_new) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || done[p]) return;
    if (f_trial[p] == 0 && E_trial[p] <= E_cur[p]) {
        for (int a = 0; a < 3; ++a) {
            rv[3 * p + a] = trv[3 * p + a];
            tr[3 * p + a] = ttr[3 * p + a];
        }
        E_new[p] = E_trial[p];
        f_new[p] = 0;
        accepted[p] = level;
        done[p] = 1;
    }
}

// Poses kept at this step report the energy and flags of the gradient pass.
__global__ void k_pgd_keep(long long P, const uint8_t* __restrict__ done,
                           const double* __restrict__ E_cur, const uint8_t* __restrict__ f_cur,
                           double* __restrict__ E_new, uint8_t* __restrict__ f_new) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || done[p]) return;
    E_new[p] = E_cur[p];
    f_new[p] = f_cur[p];
}

inline unsigned nblk(long long P) { return (unsigned)((P + 255) / 256); }

}  // namespace
}  // namespace rs

extern "C" rs_status rs_pgd_run(rs_ctx* ctx, const rs_protein* prot, int32_t L, const double* lig_xyz,
                                const double* lig_q, int64_t P, double* rotvec, double* trans,
                                int32_t nsteps, double eta_t, double eta_r, int32_t max_halvings,
                                double* E_out, uint8_t* flags_out, int32_t* accepted_out,
                                void* stream) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && prot, "rs_pgd_run: NULL context or protein");
    RS_CHECK_ARG(L >= 1 && L <= 4096, "rs_pgd_run: L=%d out of range", L);
    RS_CHECK_ARG(P >= 0 && P <= 0x7fffffffLL, "rs_pgd_run: P out of range");
    RS_CHECK_ARG(nsteps >= 0 && nsteps <= 1000000, "rs_pgd_run: nsteps=%d out of range", nsteps);
    RS_CHECK_ARG(max_halvings >= 0 && max_halvings <= 30, "rs_pgd_run: max_halvings out of range");
    RS_CHECK_ARG(eta_t >= 0 && eta_r >= 0, "rs_pgd_run: step lengths must be >= 0");
    if (P == 0 || nsteps == 0) return RS_OK;
    RS_CHECK_ARG(lig_xyz && lig_q && rotvec && trans && E_out && flags_out && accepted_out,
                 "rs_pgd_run: NULL pointer");
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t st = ctx->stream;  // capturable stream owned by the context
    // workspace: prepared ligand + per-pose state
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    size_t o_lig = take(ligand_scratch_bytes(L) + 1024);
    size_t o_Ec = take(P * 8), o_gt = take(P * 24), o_gw = take(P * 24), o_fc = take(P);
    size_t o_trv = take(P * 24), o_ttr = take(P * 24), o_tq = take(P * 32);
    size_t o_Et = take(P * 8), o_ft = take(P), o_done = take(P);
    RS_TRY(ensure_buffer(&ctx->pgd_buf, &ctx->pgd_bytes, off));
    char* b = (char*)ctx->pgd_buf;
    LigandView lig = carve_ligand(b + o_lig, L);
    double *Ec = (double*)(b + o_Ec), *gt = (double*)(b + o_gt), *gw = (double*)(b + o_gw);
    uint8_t* fc = (uint8_t*)(b + o_fc);
    double *trv = (double*)(b + o_trv), *ttr = (double*)(b + o_ttr), *tq = (double*)(b + o_tq);
    double* Et = (double*)(b + o_Et);
    uint8_t *ft = (uint8_t*)(b + o_ft), *done = (uint8_t*)(b + o_done);

    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    RS_TRY_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    RS_TRY_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
    auto cleanup = [&]() {
        cudaEventDestroy(ev_in);
        cudaEventDestroy(ev_out);
    };
    // order after the caller's stream
    if (cudaEventRecord(ev_in, user) != cudaSuccess || cudaStreamWaitEvent(st, ev_in, 0) != cudaSuccess) {
        cleanup();
        set_error("rs_pgd_run: stream ordering failed");
        return RS_ERR_CUDA;
    }
    rs_status s = launch_prep_ligand(L, lig_xyz, lig_q, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64, (double*)lig.q64, st);
    if (s != RS_OK) {
        cleanup();
        return s;
    }
    // make sure the pose kernels' attributes are set outside the capture
    EvalLaunch g;
    g.prot = prot->view;
    g.lig = lig;
    g.rot = rotvec;
    g.trans = trans;
    g.P = P;
    g.E = Ec;
    g.flags = fc;
    g.gt = gt;
    g.gw = gw;
    g.events = false;
    if (prot->view.kind == 1) {  // scratch of the cell-grouped path, shared by both passes
        s = ensure_buffer(&ctx->eval_buf, &ctx->eval_bytes, sorted_scratch_bytes(P, L, prot->n, true));
        if (s != RS_OK) {
            cleanup();
            return s;
        }
        g.ws = ctx->eval_buf;
        g.ws_bytes = ctx->eval_bytes;
    }
    EvalLaunch e = g;
    e.rot = tq;
    e.trans = ttr;
    e.E = Et;
    e.flags = ft;
    e.gt = e.gw = nullptr;
    e.skip = done;
    int nk = 0;
    auto one_step = [&]() -> rs_status {
        nk = 0;
        RS_TRY(launch_eval(g, true, st));
        ++nk;
        {
            ::rs::KernelTimer kt__("k_pgd_init", st, 0.0, false, false);
            k_pgd_init<<<nblk(P), 256, 0, st>>>(P, done, accepted_out);
        }
        ++nk;
        for (int lv = 0; lv <= max_halvings; ++lv) {
            {
                ::rs::KernelTimer kt__("k_pgd_trial", st, 0.0, false, false);
                k_pgd_trial<<<nblk(P), 256, 0, st>>>(P, lv, eta_t, eta_r, rotvec, trans, gt, gw, done,
                                                     trv, ttr, tq);
            }
            RS_TRY(launch_eval(e, false, st));
            {
                ::rs::KernelTimer kt__("k_pgd_accept", st, 0.0, false, false);
                k_pgd_accept<<<nblk(P), 256, 0, st>>>(P, lv, Ec, Et, ft, trv, ttr, done, accepted_out,
                                                      rotvec, trans, E_out, flags_out);
            }
            nk += 3;
        }
        {
            ::rs::KernelTimer kt__("k_pgd_keep", st, 0.0, false, false);
            k_pgd_keep<<<nblk(P), 256, 0, st>>>(P, done, Ec, fc, E_out, flags_out);
        }
        ++nk;
        RS_TRY_CUDA(cudaGetLastError());
        return RS_OK;
    };
    // first step runs eagerly (sets kernel attributes); the rest replay its graph
    s = one_step();
    if (s != RS_OK) {
        cleanup();
        return s;
    }
    if (nsteps > 1) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cleanup();
            set_error("rs_pgd_run: stream capture failed to start");
            return RS_ERR_CUDA;
        }
        s = one_step();
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (s != RS_OK || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            cleanup();
            if (s == RS_OK) set_error("rs_pgd_run: graph capture failed");
            return s == RS_OK ? RS_ERR_CUDA : s;
        }
        for (int it = 1; it < nsteps; ++it) {
            if (cudaGraphLaunch(exec, st) != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                cleanup();
                set_error("rs_pgd_run: graph launch failed");
                return RS_ERR_CUDA;
            }
        }
        // the capture counted one step's launches; the replays add the rest
        note_launch((unsigned)(nk * (nsteps - 2) > 0 ? nk * (nsteps - 2) : 0));
        cudaStreamSynchronize(st);  // the executable graph is released only after its replays
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
    }
    if (cudaEventRecord(ev_out, st) != cudaSuccess || cudaStreamWaitEvent(user, ev_out, 0) != cudaSuccess) {
        cleanup();
        set_error("rs_pgd_run: stream ordering failed");
        return RS_ERR_CUDA;
    }
    cleanup();
    return RS_OK;
}
