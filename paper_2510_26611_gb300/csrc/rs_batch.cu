// Batched pose evaluation: many protein-ligand pairs of uneven sizes, captured
// once in a CUDA graph and replayed.  Pairs are grouped by padded Tucker rank; for
// each group an autotuner times the candidates on all of the group's poses and
// keeps the fastest:
//   * the cell-grouped multi-pair pipeline (rs_group.cu): the pose-atoms of all
//     pairs sorted by (pair, axis-3 cell), the long range of each cell's atoms on
//     the tensor cores (or in float pairs where cells hold few atoms); candidates
//     differ in chunk size;
//   * one persistent per-block launch: each pair's poses cut into items of PB poses
//     (PB ~ atoms-per-item / L), largest first, taken from a device counter;
//     candidates differ in threads per CTA and atoms per item.
// Every path computes each pose's energy to the same tolerance (flags identical);
// the per-block and float-pair kernels agree with rs_energy_poses bit for bit where
// it takes the same kernel, and the results do not depend on the mix or on which
// CTA ran them.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"
#include "rs_pose_dev.cuh"
#include "rs_batch_dev.cuh"
#include "rs_group.cuh"

namespace rs {
namespace {

// mode 0: per-block launch with `shape`; mode 1: cell-grouped pipeline with `wpb`
// warps per W-form CTA and chunks of at most `chunk` pose-atoms; mode 2: each pair on
// its own through the single-pair dispatch (what a plain call of the pair runs: the
// cell-grouped path when it is large, else the per-block kernel), one pair after the
// other; mode 3: the same single-pair dispatch with the
// pairs spread over `streams` concurrent streams (parallel branches of the graph), so
// that one pair's serial small kernels (key scan, pose setup, reduction) and tails
// overlap another pair's work.
struct Choice {
    int mode;
    Shape shape;
    int wpb;
    long long chunk;
    int streams = 1;
};

constexpr int kMaxStreams = 4;

const Choice kCandidates[] = {
    {1, {128, 512}, 4, 1LL << 23}, {1, {128, 512}, 4, 1LL << 21}, {0, {128, 256}, 0, 0},
    {0, {128, 512}, 0, 0},         {0, {256, 512}, 0, 0},          {2, {128, 256}, 0, 0},
    {3, {128, 256}, 0, 0, 2},      {3, {128, 256}, 0, 0, kMaxStreams}};

std::mutex g_tune_mu;
std::map<int, Choice> g_tuned;  // padded rank -> best choice (process-wide cache)

struct Group {
    int RP;
    std::vector<int> pairs;  // indices into the batch's pair list
    Choice choice{1, {128, 512}, 4, 1LL << 23};
    Shape shape{128, 512};
    int nitems = 0;
    int grid = 0;
    size_t smem = 0;
    BatchItem* d_items = nullptr;
    int* d_counter = nullptr;
    GroupPlan plan;
    GroupSeg* d_segs = nullptr;
};

}  // namespace
}  // namespace rs

struct rs_batch {
    int device = 0;
    std::vector<rs::PairDesc> pairs;
    std::vector<int> Ls;
    rs::PairDesc* d_pairs = nullptr;
    void* d_lig = nullptr;
    void* d_ws = nullptr;  // scratch of the cell-grouped pipeline (largest group chunk)
    size_t ws_bytes = 0;
    std::vector<rs::Group> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    // concurrent pairs (mode 3): side streams, fork/join events, one scratch region
    // of ws_side_bytes per stream
    cudaStream_t side[rs::kMaxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[rs::kMaxStreams] = {};
    void* d_ws_side = nullptr;
    size_t ws_side_bytes = 0;
    int ws_side_count = 0;
    double tune_ms = 0.0;
    std::vector<void*> allocs;
};

namespace rs {
namespace {

template <int RP, int NT>
rs_status launch_group(rs_batch* B, Group& g, cudaStream_t st, bool set_attr) {
    auto kern = k_eval_batch<RP, NT>;
    size_t sm = batch_smem<RP, NT>(B->Ls, g.shape.atoms);
    if (sm > 200 * 1024) {
        set_error("batch: shared memory %zu exceeds the limit", sm);
        return RS_ERR_UNSUPPORTED;
    }
    if (set_attr) {
        RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int per_sm = 0;
        RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm));
        int sms = 0;
        RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device));
        g.grid = std::max(1, std::min(g.nitems, std::max(per_sm, 1) * sms));
        g.smem = sm;
    }
    RS_TRY_CUDA(cudaMemsetAsync(g.d_counter, 0, sizeof(int), st));
    {
        ::rs::KernelTimer kt__("k_eval_batch", st, 0.0, true, false);
        kern<<<g.grid, NT, g.smem, st>>>(B->d_pairs, g.d_items, g.nitems, g.d_counter);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

template <int RP>
rs_status launch_group_nt(rs_batch* B, Group& g, cudaStream_t st, bool set_attr) {
    return g.shape.nt == 256 ? launch_group<RP, 256>(B, g, st, set_attr)
                             : launch_group<RP, 128>(B, g, st, set_attr);
}

rs_status dispatch_block(rs_batch* B, Group& g, cudaStream_t st, bool set_attr) {
    switch (g.RP) {
#define RS_CASE(R) \
    case R: return launch_group_nt<R>(B, g, st, set_attr);
        RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        default:
            set_error("batch: unsupported padded rank %d", g.RP);
            return RS_ERR_UNSUPPORTED;
    }
}

rs_status dispatch_pairs(rs_batch* B, Group& g, cudaStream_t st) {
    for (int pi : g.pairs) {
        const PairDesc& d = B->pairs[pi];
        if (d.P <= 0) continue;
        EvalLaunch a;
        a.prot = d.prot;
        a.lig = d.lig;
        a.rot = d.rot;
        a.trans = d.trans;
        a.P = d.P;
        a.E = d.E;
        a.flags = d.flags;
        a.events = false;
        a.ws = B->d_ws;
        a.ws_bytes = B->ws_bytes;
        RS_TRY(launch_eval_paths(a, false, st));
    }
    return RS_OK;
}

// Pairs with poses, longest (P L) first, each onto the stream with the least work so
// far (ties to the lower stream): a fixed assignment, so the graph and the results do
// not depend on timing.
std::vector<std::vector<int>> assign_streams(const rs_batch* B, const Group& g, int S) {
    std::vector<int> order;
    for (int pi : g.pairs)
        if (B->pairs[pi].P > 0) order.push_back(pi);
    auto work = [&](int pi) { return (double)B->pairs[pi].P * B->pairs[pi].lig.L; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    std::vector<std::vector<int>> lists(S);
    std::vector<double> load(S, 0.0);
    for (int pi : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[k].push_back(pi);
        load[k] += work(pi);
    }
    return lists;
}

// Mode 3: fork the group's pairs from st onto the side streams and join them back.
// The join is recorded even when a launch fails, so that a capture ends cleanly.
rs_status dispatch_streams(rs_batch* B, Group& g, cudaStream_t st) {
    const int S = g.choice.streams;
    const auto lists = assign_streams(B, g, S);
    RS_TRY_CUDA(cudaEventRecord(B->fork_ev, st));
    for (int k = 0; k < S; ++k) RS_TRY_CUDA(cudaStreamWaitEvent(B->side[k], B->fork_ev, 0));
    rs_status first = RS_OK;
    for (int k = 0; k < S && first == RS_OK; ++k)
        for (int pi : lists[k]) {
            const PairDesc& d = B->pairs[pi];
            EvalLaunch a;
            a.prot = d.prot;
            a.lig = d.lig;
            a.rot = d.rot;
            a.trans = d.trans;
            a.P = d.P;
            a.E = d.E;
            a.flags = d.flags;
            a.events = false;
            a.ws = (char*)B->d_ws_side + (size_t)k * B->ws_side_bytes;
            a.ws_bytes = B->ws_side_bytes;
            if ((first = launch_eval_paths(a, false, B->side[k])) != RS_OK) break;
        }
    for (int k = 0; k < S; ++k) {
        RS_TRY_CUDA(cudaEventRecord(B->join_ev[k], B->side[k]));
        RS_TRY_CUDA(cudaStreamWaitEvent(st, B->join_ev[k], 0));
    }
    return first;
}

rs_status dispatch_group(rs_batch* B, Group& g, cudaStream_t st, bool set_attr) {
    if (g.choice.mode == 0) return dispatch_block(B, g, st, set_attr);
    if (g.choice.mode == 2) return dispatch_pairs(B, g, st);
    if (g.choice.mode == 3) return dispatch_streams(B, g, st);
    return group_launch(g.plan, B->d_pairs, g.d_segs, B->d_ws, B->ws_bytes, g.choice.wpb, st, false);
}

// Plan of the cell-grouped pipeline over a fraction of each pair's poses, with its
// segments on the device and the batch scratch grown to fit.
rs_status build_plan(rs_batch* B, Group& g, double pose_fraction) {
    std::vector<PairDesc> pairs = B->pairs;
    if (pose_fraction < 1.0)
        for (int pi : g.pairs) pairs[pi].P = std::max<long long>(1, (long long)(pairs[pi].P * pose_fraction));
    RS_TRY(group_plan(pairs, g.pairs, g.choice.chunk, &g.plan));
    if (g.d_segs) {
        cudaFree(g.d_segs);
        B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), (void*)g.d_segs), B->allocs.end());
        g.d_segs = nullptr;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(1, g.plan.segs.size()) * sizeof(GroupSeg)) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch: segment table allocation failed");
        return RS_ERR_OOM;
    }
    B->allocs.push_back(p);
    g.d_segs = (GroupSeg*)p;
    RS_TRY_CUDA(cudaMemcpy(g.d_segs, g.plan.segs.data(), g.plan.segs.size() * sizeof(GroupSeg),
                           cudaMemcpyHostToDevice));
    if (g.plan.scratch > B->ws_bytes) {
        if (B->d_ws) {
            cudaFree(B->d_ws);
            B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), B->d_ws), B->allocs.end());
            B->d_ws = nullptr;
            B->ws_bytes = 0;
        }
        if (cudaMalloc(&B->d_ws, g.plan.scratch) != cudaSuccess) {
            cudaGetLastError();
            set_error("batch: scratch allocation of %zu bytes failed", g.plan.scratch);
            return RS_ERR_OOM;
        }
        B->allocs.push_back(B->d_ws);
        B->ws_bytes = g.plan.scratch;
    }
    return RS_OK;
}

// Work items of a group for a shape: per pair, blocks of PB poses; largest
// items first so the tail of the persistent launch is short.
rs_status build_items(rs_batch* B, Group& g, double pose_fraction) {
    std::vector<BatchItem> items;
    std::vector<double> cost;
    for (int pi : g.pairs) {
        const PairDesc& d = B->pairs[pi];
        int PB = pb_for(d.lig.L, g.shape.atoms);
        long long P = std::max<long long>(1, (long long)(d.P * pose_fraction));
        if (pose_fraction >= 1.0) P = d.P;
        for (long long p0 = 0; p0 < P; p0 += PB) {
            items.push_back({pi, PB, p0});
            long long np = std::min<long long>(PB, d.P - p0);
            cost.push_back((double)np * d.lig.L);
        }
    }
    std::vector<size_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<BatchItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    g.nitems = (int)sorted.size();
    if (g.d_items) {
        cudaFree(g.d_items);
        B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), (void*)g.d_items), B->allocs.end());
        g.d_items = nullptr;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(1, sorted.size()) * sizeof(BatchItem)) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch: item list allocation failed");
        return RS_ERR_OOM;
    }
    B->allocs.push_back(p);
    g.d_items = (BatchItem*)p;
    RS_TRY_CUDA(cudaMemcpy(g.d_items, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    return RS_OK;
}

// Scratch of the single-pair path for the group's largest pair.
rs_status size_pairs(rs_batch* B, Group& g) {
    size_t need = 0;
    for (int pi : g.pairs) {
        const PairDesc& d = B->pairs[pi];
        if (d.P > 0) need = std::max(need, sorted_scratch_bytes(d.P, d.lig.L, d.prot.n, false));
    }
    if (need > B->ws_bytes) {
        if (B->d_ws) {
            cudaFree(B->d_ws);
            B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), B->d_ws), B->allocs.end());
            B->d_ws = nullptr;
            B->ws_bytes = 0;
        }
        if (cudaMalloc(&B->d_ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("batch: scratch allocation of %zu bytes failed", need);
            return RS_ERR_OOM;
        }
        B->allocs.push_back(B->d_ws);
        B->ws_bytes = need;
    }
    return RS_OK;
}

// Side streams, events and per-stream scratch of mode 3 (created on first use; the
// scratch grows to the largest pair of any group and to the most streams asked).
rs_status size_streams(rs_batch* B, Group& g) {
    if (!B->fork_ev) {
        for (int k = 0; k < kMaxStreams; ++k) {
            if (cudaStreamCreateWithFlags(&B->side[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->join_ev[k], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                set_error("batch: stream or event creation failed");
                return RS_ERR_CUDA;
            }
        }
        if (cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            set_error("batch: event creation failed");
            return RS_ERR_CUDA;
        }
    }
    size_t need = 0;
    for (int pi : g.pairs) {
        const PairDesc& d = B->pairs[pi];
        if (d.P > 0) need = std::max(need, sorted_scratch_bytes(d.P, d.lig.L, d.prot.n, false));
    }
    need = (need + 255) / 256 * 256;
    const int S = g.choice.streams;
    if (need > B->ws_side_bytes || S > B->ws_side_count) {
        const size_t per = std::max(need, B->ws_side_bytes);
        const int count = std::max(S, B->ws_side_count);
        if (B->d_ws_side) {
            cudaFree(B->d_ws_side);
            B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), B->d_ws_side), B->allocs.end());
            B->d_ws_side = nullptr;
            B->ws_side_bytes = 0;
            B->ws_side_count = 0;
        }
        if (cudaMalloc(&B->d_ws_side, per * count) != cudaSuccess) {
            cudaGetLastError();
            set_error("batch: scratch allocation of %zu bytes failed", per * count);
            return RS_ERR_OOM;
        }
        B->allocs.push_back(B->d_ws_side);
        B->ws_side_bytes = per;
        B->ws_side_count = count;
    }
    return RS_OK;
}

rs_status prepare(rs_batch* B, Group& g, double pose_fraction) {
    g.shape = g.choice.shape;
    if (g.choice.mode == 2) return size_pairs(B, g);
    if (g.choice.mode == 3) return size_streams(B, g);
    return g.choice.mode == 0 ? build_items(B, g, pose_fraction) : build_plan(B, g, pose_fraction);
}

// Times every candidate on all of the group's poses (results are written to the real
// outputs and overwritten by the real run) and keeps the best.  A sample of the poses
// would thin out the cells and favour the per-block path unfairly.
rs_status tune_group(rs_batch* B, Group& g, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(g.RP);
        if (it != g_tuned.end()) {
            g.choice = it->second;
            return RS_OK;
        }
    }
    cudaEvent_t a, b;
    RS_TRY_CUDA(cudaEventCreate(&a));
    RS_TRY_CUDA(cudaEventCreate(&b));
    float best = 1e30f;
    Choice best_choice = g.choice;
    for (const Choice& c : kCandidates) {
        g.choice = c;
        RS_TRY(prepare(B, g, 1.0));
        RS_TRY(dispatch_group(B, g, st, true));  // warm-up
        float total = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            RS_TRY_CUDA(cudaEventRecord(a, st));
            RS_TRY(dispatch_group(B, g, st, false));
            RS_TRY_CUDA(cudaEventRecord(b, st));
            RS_TRY_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            RS_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
            total += ms;
        }
        B->tune_ms += total;
        if (total < best) {
            best = total;
            best_choice = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    g.choice = best_choice;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[g.RP] = best_choice;
    return RS_OK;
}

void batch_destroy(rs_batch* B) {
    if (!B) return;
    cudaSetDevice(B->device);
    cudaDeviceSynchronize();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    for (int k = 0; k < kMaxStreams; ++k) {
        if (B->side[k]) cudaStreamDestroy(B->side[k]);
        if (B->join_ev[k]) cudaEventDestroy(B->join_ev[k]);
    }
    if (B->fork_ev) cudaEventDestroy(B->fork_ev);
    for (void* p : B->allocs) cudaFree(p);
    delete B;
}

}  // namespace

void batch_shape_for(int RP, int* nt, int* atoms) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(RP);
    const bool tuned = it != g_tuned.end() && it->second.mode == 0;
    // untuned: 256 pose-atoms per work item (measured 2x faster than 512 on a serving
    // launch of 73 requests x 2048 poses; smaller items fit more CTAs per SM)
    *nt = tuned ? it->second.shape.nt : 128;
    *atoms = tuned ? it->second.shape.atoms : 256;
}

}  // namespace rs

extern "C" {

rs_status rs_batch_create(rs_ctx* ctx, int32_t npairs, const rs_pair* pairs, int32_t autotune,
                          rs_batch** out) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(ctx && pairs && out, "rs_batch_create: NULL argument");
    RS_CHECK_ARG(npairs >= 1 && npairs <= (1 << 20), "rs_batch_create: npairs=%d out of range", npairs);
    RS_CHECK_ARG(autotune >= 0 && autotune <= 4, "rs_batch_create: autotune=%d not in {0, 1, 2, 3, 4}", autotune);
    *out = nullptr;
    for (int i = 0; i < npairs; ++i) {
        const rs_pair& p = pairs[i];
        RS_CHECK_ARG(p.prot, "rs_batch_create: pair %d has no protein", i);
        RS_CHECK_ARG(p.prot->device == ctx->device, "rs_batch_create: pair %d on another device", i);
        if (p.prot->view.box) {
            set_error("rs_batch_create: pair %d uses a local-box handle (not batched; use rs_energy_poses)", i);
            return RS_ERR_UNSUPPORTED;
        }
        RS_CHECK_ARG(p.L >= 1 && p.L <= 4096, "rs_batch_create: pair %d L=%d out of range", i, p.L);
        RS_CHECK_ARG(p.P >= 0 && p.P <= 0x7fffffffLL, "rs_batch_create: pair %d P out of range", i);
        RS_CHECK_ARG(p.lig_xyz && p.lig_q && (p.P == 0 || (p.quat && p.trans && p.E_out)),
                     "rs_batch_create: pair %d has a NULL pointer", i);
        if (p.prot->kind != 1) {
            set_error("rs_batch_create: pair %d: batching takes Tucker-reduced proteins", i);
            return RS_ERR_UNSUPPORTED;
        }
    }
    RS_TRY_CUDA(cudaSetDevice(ctx->device));
    rs_batch* B = new rs_batch();
    B->device = ctx->device;
    auto fail = [&](rs_status s) {
        batch_destroy(B);
        return s;
    };
    if (cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("rs_batch_create: stream creation failed");
        return fail(RS_ERR_CUDA);
    }
    cudaStream_t st = B->cap_stream;
    // prepared ligands, one region per pair
    std::vector<size_t> off(npairs);
    size_t total = 0;
    for (int i = 0; i < npairs; ++i) {
        off[i] = total;
        total += (ligand_scratch_bytes(pairs[i].L) + 1023) / 256 * 256;
    }
    if (cudaMalloc(&B->d_lig, total) != cudaSuccess) {
        cudaGetLastError();
        set_error("rs_batch_create: ligand scratch allocation failed");
        return fail(RS_ERR_OOM);
    }
    B->allocs.push_back(B->d_lig);
    for (int i = 0; i < npairs; ++i) {
        const rs_pair& p = pairs[i];
        LigandView lig = carve_ligand((char*)B->d_lig + off[i], p.L);
        rs_status s = launch_prep_ligand(p.L, p.lig_xyz, p.lig_q, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64,
                                         (double*)lig.q64, st, false);
        if (s != RS_OK) return fail(s);
        PairDesc d;
        d.prot = p.prot->view;
        d.lig = lig;
        d.rot = p.quat;
        d.trans = p.trans;
        d.P = p.P;
        d.E = p.E_out;
        d.flags = p.flags_out;
        B->pairs.push_back(d);
        B->Ls.push_back(p.L);
    }
    if (cudaMalloc((void**)&B->d_pairs, npairs * sizeof(PairDesc)) != cudaSuccess) {
        cudaGetLastError();
        set_error("rs_batch_create: descriptor allocation failed");
        return fail(RS_ERR_OOM);
    }
    B->allocs.push_back(B->d_pairs);
    if (cudaMemcpy(B->d_pairs, B->pairs.data(), npairs * sizeof(PairDesc), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("rs_batch_create: descriptor copy failed");
        return fail(RS_ERR_CUDA);
    }
    // groups by padded rank
    std::map<int, std::vector<int>> by_rp;
    for (int i = 0; i < npairs; ++i)
        if (pairs[i].P > 0) by_rp[pairs[i].prot->view.R].push_back(i);
    for (auto& kv : by_rp) {
        Group g;
        g.RP = kv.first;
        g.pairs = kv.second;
        void* c = nullptr;
        if (cudaMalloc(&c, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("rs_batch_create: counter allocation failed");
            return fail(RS_ERR_OOM);
        }
        B->allocs.push_back(c);
        g.d_counter = (int*)c;
        B->groups.push_back(g);
    }
    rs_status s;
    for (Group& g : B->groups) {
        if (autotune == 2) g.choice = Choice{0, {128, 256}, 0, 0};  // per-block path, default shape
        if (autotune == 3) g.choice = Choice{2, {128, 256}, 0, 0};  // pair by pair, single-pair path
        if (autotune == 4) g.choice = Choice{3, {128, 256}, 0, 0, kMaxStreams};  // pairs on concurrent streams
        if (autotune == 1 && (s = tune_group(B, g, st)) != RS_OK) return fail(s);
        if ((s = prepare(B, g, 1.0)) != RS_OK) return fail(s);
        if ((s = dispatch_group(B, g, st, true)) != RS_OK) return fail(s);  // sets attributes, grid
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("rs_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(RS_ERR_CUDA);
    }
    // capture the whole batch once
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("rs_batch_create: stream capture failed to start");
        return fail(RS_ERR_CUDA);
    }
    for (Group& g : B->groups) {
        s = dispatch_group(B, g, st, false);
        if (s != RS_OK) {
            cudaGraph_t dummy;
            cudaStreamEndCapture(st, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
            return fail(s);
        }
    }
    if (cudaStreamEndCapture(st, &B->graph) != cudaSuccess ||
        cudaGraphInstantiate(&B->exec, B->graph, 0) != cudaSuccess) {
        set_error("rs_batch_create: graph capture failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(RS_ERR_CUDA);
    }
    *out = B;
    return RS_OK;
}

rs_status rs_batch_run(rs_batch* B, void* stream) {
    rs::clear_error();
    RS_CHECK_ARG(B && B->exec, "rs_batch_run: NULL batch");
    RS_TRY_CUDA(cudaSetDevice(B->device));
    RS_TRY_CUDA(cudaGraphLaunch(B->exec, (cudaStream_t)stream));
    rs::note_launch((unsigned)B->groups.size());
    return RS_OK;
}

void rs_batch_free(rs_batch* B) { rs::batch_destroy(B); }

rs_status rs_batch_get_info(const rs_batch* B, rs_batch_info* o) {
    rs::clear_error();
    RS_CHECK_ARG(B && o, "rs_batch_get_info: NULL argument");
    memset(o, 0, sizeof(*o));
    o->npairs = (int32_t)B->pairs.size();
    o->ngroups = (int32_t)B->groups.size();
    for (const rs::Group& g : B->groups) {
        if (g.choice.mode == 0) {
            o->nitems += g.nitems;
            o->grid += g.grid;
        } else if (g.choice.mode == 1) {
            o->nchunks += (int32_t)g.plan.chunks.size();
        }
    }
    if (!B->groups.empty()) {
        const rs::Group& g = B->groups[0];
        o->mode = g.choice.mode;
        o->threads = g.choice.mode == 0 ? g.shape.nt : 0;
        o->atoms_per_item = g.choice.mode == 0 ? g.shape.atoms : 0;
        o->warps_per_cta = g.choice.mode == 1 ? g.choice.wpb : 0;
        o->chunk_atoms = g.choice.mode == 1 ? g.choice.chunk : 0;
        o->streams = g.choice.mode == 3 ? g.choice.streams : 1;
    }
    o->tune_ms = B->tune_ms;
    return RS_OK;
}

}  // extern "C"
