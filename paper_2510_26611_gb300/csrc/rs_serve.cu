// Serving: a request loop with continuous batching around Algorithm PLIE (Sec. 3.4).
//
// Requests (protein + ligand + poses, host memory) are queued by rs_serve_submit.
// A builder thread builds missing proteins on its own context; the scheduler thread
// owns another context and loops:
//   1. retire: launches whose completion event fired hand their results (already
//      staged in pinned host memory by the launch's stream) to the callers'
//      buffers and give their device blocks back to the pool;
//   2. admit: queued requests, in arrival order, while the device-memory budget
//      allows.  A protein's RS factors come from a resident cache keyed by the
//      caller's protein id (built on a miss; idle proteins are evicted least
//      recently used first under memory pressure).  Per-request buffers come from a
//      size-class pool that keeps its slabs while serving, so no cudaFree stalls the
//      device between launches;
//   3. launch: every request admitted in this pass goes into one batched pose launch
//      per padded Tucker rank (the cell-grouped multi-pair pipeline for requests
//      with many pose-atoms per grid cell, one persistent per-block kernel for the
//      rest; both compute every pose as rs_energy_poses does) on the next free stream.  Up to
//      max_inflight_launches launches run at once, so work that arrives while the
//      GPU is busy is admitted into the next launch and overlaps with the running one.
// All host waits are bounded (condition-variable timeouts, event queries); no device
// code waits on anything.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rs_common.cuh"
#include "rs_diag.cuh"
#include "rs_eval.cuh"
#include "rs_batch_dev.cuh"
#include "rs_group.cuh"

namespace rs {
namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

enum PoolResult { POOL_OK = 0, POOL_OVER_BUDGET = 1, POOL_FAILED = 2 };

// Device (or pinned host) blocks in power-of-two size classes.  Slabs stay
// allocated while serving; trim() frees the idle ones.
struct Pool {
    bool host = false;
    std::map<size_t, std::vector<void*>> free;
    std::unordered_map<void*, size_t> size_of;
    size_t reserved = 0;
    int* inject = nullptr;  // test hook: fail this many further slab allocations
    static size_t cls(size_t b) {
        size_t c = 4096;
        while (c < b) c <<= 1;
        return c;
    }
    PoolResult get(size_t bytes, size_t budget_left, void** out) {
        *out = nullptr;
        size_t c = cls(bytes);
        auto& fl = free[c];
        if (!fl.empty()) {
            *out = fl.back();
            fl.pop_back();
            return POOL_OK;
        }
        if (c > budget_left) return POOL_OVER_BUDGET;
        if (inject && *inject > 0) {
            --*inject;
            return POOL_FAILED;
        }
        void* p = nullptr;
        cudaError_t e = host ? cudaHostAlloc(&p, c, cudaHostAllocDefault) : cudaMalloc(&p, c);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return POOL_FAILED;
        }
        size_of[p] = c;
        reserved += c;
        *out = p;
        return POOL_OK;
    }
    void put(void* p) {
        if (!p) return;
        auto it = size_of.find(p);
        if (it != size_of.end()) free[it->second].push_back(p);
    }
    void release(void* p) {
        if (host) cudaFreeHost(p);
        else cudaFree(p);
    }
    void trim() {
        for (auto& kv : free)
            for (void* p : kv.second) {
                reserved -= size_of[p];
                size_of.erase(p);
                release(p);
            }
        free.clear();
    }
    void clear() {
        for (auto& kv : size_of) release(kv.first);
        size_of.clear();
        free.clear();
        reserved = 0;
    }
};

enum EntryState { BUILDING = 0, READY = 1, FAILED = 2 };

struct ProteinEntry {
    EntryState state = BUILDING;
    rs_protein* prot = nullptr;
    size_t reserve = 0;      // bytes held for a protein being built
    bool anonymous = false;  // built for one request: freed when it retires
    int inflight = 0;
    int64_t last_use = 0;
    rs_status status = RS_OK;  // of a failed build
    char message[160] = {0};
};

// A protein build handed to the builder thread (it owns a second context, so a
// build never stalls the scheduler loop or the launches in flight).
struct BuildJob {
    uint64_t key = 0;
    int32_t N = 0;
    std::vector<double> xyz, q;  // copied, so a cancelled request's arrays are not read later
    rs_params params{};
};

struct BuildDone {
    uint64_t key;
    rs_protein* prot;
    rs_status status;
    char message[160];
};

enum State { QUEUED = 0, ADMITTED = 1, LAUNCHED = 2, DONE = 3, CANCELLED = 4 };

struct Request {
    uint64_t id = 0;
    rs_request req{};
    double* E_host = nullptr;
    uint8_t* flags_host = nullptr;
    State state = QUEUED;
    rs_status status = RS_OK;
    char message[160] = {0};
    int64_t t_submit = 0, t_admit = 0, t_start = 0, t_end = 0;
    uint64_t cache_key = 0;
    bool started_build = false;  // its protein was not resident on arrival
    ProteinEntry* pe = nullptr;
    void* d_in = nullptr;   // ligand, poses, prepared ligand
    void* d_out = nullptr;  // E [P] then flags [P]
    void* h_out = nullptr;  // pinned staging of d_out
    void fail(rs_status s, const char* msg) {
        status = s;
        snprintf(message, sizeof(message), "%s", msg ? msg : "");
    }
};

struct Launch {
    cudaEvent_t done = nullptr;
    int stream = 0;
    std::vector<Request*> reqs;
    std::vector<void*> blocks;  // descriptors and work items
};

size_t in_bytes_for(const rs_request& r) {
    return round256((size_t)r.L * 24) + round256((size_t)r.L * 8) + round256((size_t)r.P * 32) +
           round256((size_t)r.P * 24) + round256(ligand_scratch_bytes(r.L) + 1024);
}

size_t out_bytes_for(const rs_request& r) { return round256((size_t)r.P * 8) + round256((size_t)r.P); }

// Device bytes of a protein before it is built (Tucker: node coordinates of the
// cell list plus the W-form tables; canonical: three n x (N R_l) factor tables).
size_t protein_estimate(const rs_request& r) {
    size_t n = (size_t)r.params.n;
    size_t atoms = (size_t)r.N * 64;
    if (r.params.tucker_cap > 0) {
        size_t rp = (size_t)(r.params.tucker_cap + 3) / 4 * 4;
        return atoms + 2 * n * rp * rp * 8 + 4 * n * rp * 8 + ((size_t)4 << 20);
    }
    return atoms + 3 * n * (size_t)r.N * (size_t)r.params.R_l * 4 + ((size_t)4 << 20);
}

}  // namespace
}  // namespace rs

struct rs_server {
    rs_ctx* ctx = nullptr;   // scheduler thread: uploads and pose launches
    rs_ctx* bctx = nullptr;  // builder thread: protein builds
    rs_serve_params prm{};
    std::thread worker, builder;
    std::mutex mu;  // guards queue, reqs, request states and the statistics
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<rs::Request*> queue;
    std::unordered_map<uint64_t, rs::Request*> reqs;
    // builder hand-off (under bmu)
    std::mutex bmu;
    std::condition_variable bcv;
    std::deque<rs::BuildJob> bjobs;
    std::vector<rs::BuildDone> bdone;
    bool bstop = false;
    bool bhold = false;  // test hook: builds wait until released
    // scheduler-thread state
    std::map<uint64_t, rs::ProteinEntry> cache;
    rs::Pool dev, pinned;
    int inject_left = 0;
    size_t budget = 0;
    std::vector<cudaStream_t> streams;  // one per in-flight launch, then the build stream
    std::vector<bool> stream_busy;
    std::vector<rs::Launch> launches;
    std::vector<rs::Request*> graveyard;  // cancelled requests, freed by the scheduler
    uint64_t anon_seq = 0;
    // statistics (under mu)
    rs_serve_stats st{};
    double reqs_launched = 0.0;
};

namespace rs {
namespace {

size_t used_bytes(rs_server* S) {
    size_t u = S->dev.reserved;
    for (auto& kv : S->cache) u += kv.second.prot ? kv.second.prot->device_bytes : kv.second.reserve;
    return u;
}

size_t left_bytes(rs_server* S) {
    size_t u = used_bytes(S);
    return S->budget > u ? S->budget - u : 0;
}

// Frees idle resident proteins, least recently used first, until `need` bytes fit.
void evict_for(rs_server* S, size_t need) {
    while (left_bytes(S) < need) {
        auto victim = S->cache.end();
        for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
            if (it->second.state == READY && it->second.inflight == 0 &&
                (victim == S->cache.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == S->cache.end()) return;
        rs_protein_free(victim->second.prot);
        S->cache.erase(victim);
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.evictions++;
    }
}

// Tries to make room for `need` bytes: evict idle proteins; with nothing running,
// also free the pool's idle slabs.  Returns true if the bytes fit now.
bool make_room(rs_server* S, size_t need) {
    evict_for(S, need);
    if (left_bytes(S) >= need) return true;
    if (S->launches.empty()) {
        S->dev.trim();
        evict_for(S, need);
    }
    return left_bytes(S) >= need;
}

void finish(rs_server* S, Request* r) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.cached_proteins = S->cache.size();  // the cache is only changed by this thread
    S->st.used_bytes = used_bytes(S);
    r->t_end = now_ns();
    r->state = DONE;
    if (r->status == RS_OK) S->st.done++;
    else S->st.failed++;
    S->cv_done.notify_all();
}

// Removes a request that fails before admission from the queue and finishes it.
void fail_queued(rs_server* S, Request* r, rs_status s, const char* msg) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (r->state != QUEUED) return;  // cancelled meanwhile
        auto q = std::find(S->queue.begin(), S->queue.end(), r);
        if (q != S->queue.end()) S->queue.erase(q);
        r->fail(s, msg);
        r->t_admit = now_ns();
    }
    finish(S, r);
}

void builder_main(rs_server* S) {
    cudaSetDevice(S->bctx->device);
    cudaStream_t st = S->streams.back();
    for (;;) {
        BuildJob job;
        {
            std::unique_lock<std::mutex> lk(S->bmu);
            while ((S->bjobs.empty() || S->bhold) && !S->bstop)
                S->bcv.wait_for(lk, std::chrono::milliseconds(50));
            if (S->bstop) return;
            job = S->bjobs.front();
            S->bjobs.pop_front();
        }
        BuildDone d{job.key, nullptr, RS_OK, {0}};
        d.status = rs_build_protein(S->bctx, job.N, job.xyz.data(), job.q.data(), &job.params, RS_MEM_HOST,
                                    st, &d.prot);
        if (d.status == RS_OK && cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            rs_protein_free(d.prot);
            d.prot = nullptr;
            d.status = RS_ERR_CUDA;
            snprintf(d.message, sizeof(d.message), "protein build failed on the device");
        } else if (d.status != RS_OK) {
            snprintf(d.message, sizeof(d.message), "%s", rs_last_error());
        }
        {
            std::lock_guard<std::mutex> lk(S->bmu);
            S->bdone.push_back(d);
        }
        S->cv_work.notify_one();
    }
}

// Moves finished builds into the cache.
void collect_builds(rs_server* S) {
    std::vector<BuildDone> done;
    {
        std::lock_guard<std::mutex> lk(S->bmu);
        done.swap(S->bdone);
    }
    for (BuildDone& d : done) {
        auto it = S->cache.find(d.key);
        if (it == S->cache.end()) {  // nobody waits for it any more
            rs_protein_free(d.prot);
            continue;
        }
        ProteinEntry& e = it->second;
        e.reserve = 0;
        if (d.status == RS_OK) {
            e.prot = d.prot;
            e.state = READY;
            e.last_use = now_ns();
        } else {
            e.state = FAILED;
            e.status = d.status;
            snprintf(e.message, sizeof(e.message), "%s", d.message);
        }
    }
}

// Admits queued requests whose protein is resident, in arrival order, and starts
// builds for the ones whose protein is missing.  Stops admitting at the first request
// that must wait for buffer memory held by running launches.  With can_launch false
// (every stream busy) it only starts builds.
void admit(rs_server* S, std::vector<Request*>& ready, bool can_launch) {
    collect_builds(S);
    std::vector<Request*> snap;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request* g : S->graveyard) delete g;  // no snapshot refers to them any more
        S->graveyard.clear();
        snap.assign(S->queue.begin(), S->queue.end());
    }
    bool builds_blocked = false;
    for (Request* r : snap) {
        const rs_request& q = r->req;
        size_t ib = in_bytes_for(q), ob = out_bytes_for(q);
        size_t bufs = Pool::cls(ib) + Pool::cls(ob);
        uint64_t key = q.protein_id ? q.protein_id : r->cache_key;
        auto it = key ? S->cache.find(key) : S->cache.end();
        if (it == S->cache.end()) {
            if (builds_blocked) continue;
            size_t need = protein_estimate(q);
            if (need + bufs > S->budget) {
                fail_queued(S, r, RS_ERR_OOM, "protein and request buffers exceed the memory budget");
                continue;
            }
            if (!make_room(S, need + bufs)) {
                builds_blocked = true;  // later requests of resident proteins may still go
                continue;
            }
            BuildJob job;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                if (r->state != QUEUED) continue;  // cancelled: its arrays may be gone
                job.xyz.assign(q.prot_xyz, q.prot_xyz + 3 * (size_t)q.N);
                job.q.assign(q.prot_q, q.prot_q + (size_t)q.N);
                S->st.builds++;
            }
            if (!key) key = 0x8000000000000000ull | ++S->anon_seq;
            r->cache_key = key;
            r->started_build = true;
            ProteinEntry& e = S->cache[key];
            e.state = BUILDING;
            e.reserve = need;
            e.anonymous = q.protein_id == 0;
            job.key = key;
            job.N = q.N;
            job.params = q.params;
            {
                std::lock_guard<std::mutex> lk(S->bmu);
                S->bjobs.push_back(std::move(job));
            }
            S->bcv.notify_one();
            continue;
        }
        ProteinEntry& e = it->second;
        r->cache_key = key;
        if (e.state == BUILDING || (e.state == READY && !can_launch)) continue;
        if (e.state == FAILED) {
            rs_status s = e.status;
            char msg[160];
            snprintf(msg, sizeof(msg), "%s", e.message);
            bool waiting = false;  // other queued requests of the same key fail the same way
            for (Request* o : snap)
                if (o != r && o->state == QUEUED && (o->req.protein_id ? o->req.protein_id : o->cache_key) == key)
                    waiting = true;
            if (!waiting) S->cache.erase(it);
            fail_queued(S, r, s, msg);
            continue;
        }
        e.inflight++;  // pins the protein while its buffers are found
        e.last_use = now_ns();
        if (!make_room(S, bufs)) {
            e.inflight--;
            return;  // wait for running launches to give memory back
        }
        PoolResult a = S->dev.get(ib, left_bytes(S), &r->d_in);
        PoolResult b = a == POOL_OK ? S->dev.get(ob, left_bytes(S), &r->d_out) : POOL_OK;
        PoolResult c = (a == POOL_OK && b == POOL_OK) ? S->pinned.get(ob, (size_t)-1, &r->h_out) : POOL_OK;
        if (a != POOL_OK || b != POOL_OK || c != POOL_OK) {
            S->dev.put(r->d_in);
            S->dev.put(r->d_out);
            S->pinned.put(r->h_out);
            r->d_in = r->d_out = r->h_out = nullptr;
            e.inflight--;
            if (a == POOL_OVER_BUDGET || b == POOL_OVER_BUDGET) return;  // wait
            if (e.anonymous && e.inflight == 0) {
                rs_protein_free(e.prot);
                S->cache.erase(key);
            }
            fail_queued(S, r, RS_ERR_OOM, "request buffer allocation failed");
            continue;
        }
        bool admitted = false;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (r->state == QUEUED) {
                auto qi = std::find(S->queue.begin(), S->queue.end(), r);
                if (qi != S->queue.end()) S->queue.erase(qi);
                r->t_admit = now_ns();
                r->state = ADMITTED;
                if (!r->started_build) S->st.cache_hits++;
                admitted = true;
            }
        }
        if (!admitted) {  // cancelled while its buffers were found
            S->dev.put(r->d_in);
            S->dev.put(r->d_out);
            S->pinned.put(r->h_out);
            r->d_in = r->d_out = r->h_out = nullptr;
            e.inflight--;
            continue;
        }
        r->pe = &e;
        ready.push_back(r);
    }
}

// Pose-atoms per chunk of a serving launch (bounds its scratch to ~230 MB).
constexpr long long kServeChunkAtoms = 1LL << 21;

// A request takes the cell-grouped path when it has at least 2^20 pose-atoms and
// they average at least 64 per grid cell along axis 3 (each staged W slab then
// serves many atoms and the pipeline's launches are amortised); other requests take
// the per-block kernel (measured faster for 2048-pose requests).
constexpr double kDenseAtomsPerCell = 64.0;
constexpr long long kDenseMinAtoms = 1LL << 20;

template <int RP, int NT>
rs_status launch_group(const PairDesc* d_desc, const BatchItem* d_items, int nitems, int* d_counter,
                       size_t smem, cudaStream_t st) {
    auto kern = k_eval_batch<RP, NT>;
    RS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, sms = 0, dev = 0;
    RS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    RS_TRY_CUDA(cudaGetDevice(&dev));
    RS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int grid = std::max(1, std::min(nitems, std::max(per_sm, 1) * sms));
    RS_TRY_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(int), st));
    {
        ::rs::KernelTimer kt__("k_eval_batch", st, 0.0, true);
        kern<<<grid, NT, smem, st>>>(d_desc, d_items, nitems, d_counter);
    }
    RS_TRY_CUDA(cudaGetLastError());
    return RS_OK;
}

rs_status dispatch(int RP, int NT, const PairDesc* d_desc, const BatchItem* d_items, int nitems,
                   int* d_counter, const std::vector<int>& Ls, int atoms, cudaStream_t st) {
    switch (RP) {
#define RS_CASE(R)                                                                               \
    case R:                                                                                      \
        return NT == 256 ? launch_group<R, 256>(d_desc, d_items, nitems, d_counter,              \
                                                batch_smem<R, 256>(Ls, atoms), st)               \
                         : launch_group<R, 128>(d_desc, d_items, nitems, d_counter,              \
                                                batch_smem<R, 128>(Ls, atoms), st);
        RS_CASE(4) RS_CASE(8) RS_CASE(12) RS_CASE(16) RS_CASE(20) RS_CASE(24) RS_CASE(28) RS_CASE(32)
#undef RS_CASE
        default:
            set_error("serve: unsupported padded Tucker rank %d", RP);
            return RS_ERR_UNSUPPORTED;
    }
}


// Uploads the inputs of the requests admitted in this pass and launches them
// together on stream `si`; results are staged to pinned memory on the same stream.
void launch(rs_server* S, std::vector<Request*>& ready, int si) {
    cudaStream_t st = S->streams[si];
    Launch Lh;
    Lh.stream = si;
    std::vector<PairDesc> desc;
    std::vector<Request*> ok;
    for (Request* r : ready) {
        const rs_request& q = r->req;
        char* p = (char*)r->d_in;
        double* lx = (double*)p;
        p += round256((size_t)q.L * 24);
        double* lq = (double*)p;
        p += round256((size_t)q.L * 8);
        double* qu = (double*)p;
        p += round256((size_t)q.P * 32);
        double* tr = (double*)p;
        p += round256((size_t)q.P * 24);
        LigandView lig = carve_ligand(p, q.L);
        bool good = cudaMemcpyAsync(lx, q.lig_xyz, (size_t)q.L * 24, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                    cudaMemcpyAsync(lq, q.lig_q, (size_t)q.L * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
        if (good && q.P > 0)
            good = cudaMemcpyAsync(qu, q.quat, (size_t)q.P * 32, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                   cudaMemcpyAsync(tr, q.trans, (size_t)q.P * 24, cudaMemcpyHostToDevice, st) == cudaSuccess;
        if (good)
            good = launch_prep_ligand(q.L, lx, lq, (float4*)lig.y, (float2*)lig.yd, (double*)lig.y64, (double*)lig.q64, st) == RS_OK;
        if (!good) {
            cudaGetLastError();
            r->fail(RS_ERR_CUDA, "input upload failed");
            continue;
        }
        PairDesc d;
        d.prot = r->pe->prot->view;
        d.lig = lig;
        d.rot = qu;
        d.trans = tr;
        d.P = q.P;
        d.E = (double*)r->d_out;
        d.flags = (uint8_t*)r->d_out + round256((size_t)q.P * 8);
        desc.push_back(d);
        ok.push_back(r);
    }
    // group the Tucker requests by padded rank; canonical ones launch one by one
    std::map<int, std::vector<int>> groups;
    std::vector<int> canon;
    for (size_t i = 0; i < ok.size(); ++i) {
        if (desc[i].P == 0) continue;
        if (desc[i].prot.kind == 1) groups[desc[i].prot.R].push_back((int)i);
        else canon.push_back((int)i);
    }
    rs_status status = RS_OK;
    const char* why = "";
    void* d_desc = nullptr;
    if (!groups.empty()) {
        size_t db = desc.size() * sizeof(PairDesc);
        // descriptors and work items are small; they are not held to the budget
        if (S->dev.get(db, (size_t)-1, &d_desc) != POOL_OK) {
            status = RS_ERR_OOM;
            why = "descriptor allocation failed";
        } else {
            Lh.blocks.push_back(d_desc);
            if (cudaMemcpyAsync(d_desc, desc.data(), db, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                status = RS_ERR_CUDA;
                why = "descriptor upload failed";
            }
        }
    }
    int64_t t_start = now_ns();
    for (auto& g : groups) {
        if (status != RS_OK) break;
        std::vector<int> dense, sparse;
        for (int i : g.second)
            ((double)desc[i].P * desc[i].lig.L >=
                     std::max((double)S->prm.group_min_atoms, S->prm.group_atoms_per_cell * desc[i].prot.n)
                 ? dense
                 : sparse)
                .push_back(i);
        if (!dense.empty()) {
            // the cell-grouped multi-pair pipeline over the dense requests
            GroupPlan plan;
            status = group_plan(desc, dense, kServeChunkAtoms, &plan);
            if (status != RS_OK) {
                why = "launch plan failed";
                break;
            }
            void* segs = nullptr;
            void* ws = nullptr;
            const size_t sb = plan.segs.size() * sizeof(GroupSeg);
            if (S->dev.get(sb, (size_t)-1, &segs) != POOL_OK || S->dev.get(plan.scratch, (size_t)-1, &ws) != POOL_OK) {
                S->dev.put(segs);
                status = RS_ERR_OOM;
                why = "launch scratch allocation failed";
                break;
            }
            Lh.blocks.push_back(segs);
            Lh.blocks.push_back(ws);
            if (cudaMemcpyAsync(segs, plan.segs.data(), sb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                status = RS_ERR_CUDA;
                why = "segment upload failed";
                break;
            }
            status = group_launch(plan, (const PairDesc*)d_desc, (const GroupSeg*)segs, ws, Pool::cls(plan.scratch),
                                  4, st, true);
            if (status != RS_OK) {
                why = "batched launch failed";
                break;
            }
        }
        if (!sparse.empty()) {
            // one persistent per-block launch over the sparse requests' pose blocks
            int nt = 128, atoms = 512;
            batch_shape_for(g.first, &nt, &atoms);
            std::vector<BatchItem> items;
            std::vector<int> Ls;
            for (int i : sparse) {
                int PB = pb_for(desc[i].lig.L, atoms);
                Ls.push_back(desc[i].lig.L);
                for (long long p0 = 0; p0 < desc[i].P; p0 += PB) items.push_back({i, PB, p0});
            }
            size_t ib = round256(items.size() * sizeof(BatchItem)) + 256;
            void* blk = nullptr;
            if (S->dev.get(ib, (size_t)-1, &blk) != POOL_OK) {
                status = RS_ERR_OOM;
                why = "work-list allocation failed";
                break;
            }
            Lh.blocks.push_back(blk);
            int* counter = (int*)((char*)blk + round256(items.size() * sizeof(BatchItem)));
            if (cudaMemcpyAsync(blk, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
                status = RS_ERR_CUDA;
                why = "work-list upload failed";
                break;
            }
            status = dispatch(g.first, nt, (const PairDesc*)d_desc, (const BatchItem*)blk, (int)items.size(),
                              counter, Ls, atoms, st);
            if (status != RS_OK) {
                why = "batched launch failed";
                break;
            }
        }
    }
    for (int i : canon) {
        if (status != RS_OK) break;
        EvalLaunch a;
        a.prot = desc[i].prot;
        a.lig = desc[i].lig;
        a.rot = desc[i].rot;
        a.trans = desc[i].trans;
        a.P = desc[i].P;
        a.E = desc[i].E;
        a.flags = desc[i].flags;
        status = launch_eval(a, false, st);
        if (status != RS_OK) why = "canonical launch failed";
    }
    for (Request* r : ok) {
        if (status != RS_OK || r->req.P == 0) continue;
        if (cudaMemcpyAsync(r->h_out, r->d_out, out_bytes_for(r->req), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            status = RS_ERR_CUDA;
            why = "result download failed";
        }
    }
    if (cudaEventCreateWithFlags(&Lh.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(Lh.done, st) != cudaSuccess) {
        cudaGetLastError();
        // without an event the launch is waited for here
        cudaStreamSynchronize(st);
        if (Lh.done) cudaEventDestroy(Lh.done);
        Lh.done = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.launches++;
        S->reqs_launched += (double)ready.size();
        for (Request* r : ready) {
            if (r->status == RS_OK && status != RS_OK) r->fail(status, why);
            r->state = LAUNCHED;
            r->t_start = t_start;
        }
    }
    Lh.reqs = ready;
    S->stream_busy[si] = true;
    S->launches.push_back(Lh);
}

void release_request(rs_server* S, Request* r) {
    S->dev.put(r->d_in);
    S->dev.put(r->d_out);
    S->pinned.put(r->h_out);
    r->d_in = r->d_out = r->h_out = nullptr;
    if (r->pe) {
        r->pe->inflight--;
        r->pe->last_use = now_ns();
        if (r->pe->anonymous && r->pe->inflight == 0) {
            rs_protein_free(r->pe->prot);
            S->cache.erase(r->cache_key);
        }
        r->pe = nullptr;
    }
}

// Retires launches whose completion event fired (all of them if `wait`).
void retire(rs_server* S, bool wait) {
    std::vector<Launch> keep;
    for (auto& Lh : S->launches) {
        cudaError_t q = cudaSuccess;
        if (Lh.done) q = wait ? cudaEventSynchronize(Lh.done) : cudaEventQuery(Lh.done);
        if (q == cudaErrorNotReady) {
            keep.push_back(Lh);
            continue;
        }
        if (q != cudaSuccess) cudaGetLastError();
        for (Request* r : Lh.reqs) {
            const rs_request& rq = r->req;
            if (q != cudaSuccess && r->status == RS_OK) r->fail(RS_ERR_CUDA, "launch failed on the device");
            if (r->status == RS_OK && rq.P > 0) {
                memcpy(r->E_host, r->h_out, (size_t)rq.P * 8);
                if (r->flags_host)
                    memcpy(r->flags_host, (char*)r->h_out + round256((size_t)rq.P * 8), (size_t)rq.P);
            }
            release_request(S, r);
            finish(S, r);
        }
        for (void* b : Lh.blocks) S->dev.put(b);
        if (Lh.done) cudaEventDestroy(Lh.done);
        S->stream_busy[Lh.stream] = false;
    }
    S->launches.swap(keep);
}

int free_stream(rs_server* S) {
    int inflight = (int)S->launches.size();
    if (inflight >= S->prm.max_inflight_launches) return -1;
    for (int i = 0; i < (int)S->stream_busy.size(); ++i)
        if (!S->stream_busy[i]) return i;
    return -1;
}

void worker_main(rs_server* S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            if (S->queue.empty() && S->launches.empty())
                S->cv_work.wait_for(lk, std::chrono::milliseconds(std::max(1, S->prm.idle_wait_ms)));
            if (S->stop) break;
        }
        retire(S, false);
        int si = free_stream(S);
        std::vector<Request*> ready;
        admit(S, ready, si >= 0);
        if (!ready.empty()) launch(S, ready, si);
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->st.cached_proteins = S->cache.size();
            S->st.used_bytes = used_bytes(S);
            // nothing launched: sleep until a submission or a finished build (bounded)
            if (ready.empty() && !S->stop)
                S->cv_work.wait_for(lk, std::chrono::microseconds(S->launches.empty() ? 1000 : 20));
        }
    }
    retire(S, true);
}

}  // namespace
}  // namespace rs

extern "C" {

rs_status rs_request_validate(const rs_request* r) {
    rs::clear_error();
    RS_CHECK_ARG(r, "request is NULL");
    RS_CHECK_ARG(r->L >= 1 && r->L <= 4096, "request: L=%d out of range [1, 4096]", r->L);
    RS_CHECK_ARG(r->P >= 0 && r->P <= ((int64_t)1 << 26), "request: P=%lld out of range", (long long)r->P);
    RS_CHECK_ARG(r->lig_xyz && r->lig_q, "request: ligand pointers are NULL");
    RS_CHECK_ARG(r->P == 0 || (r->quat && r->trans), "request: pose pointers are NULL");
    RS_CHECK_ARG(r->N >= 1 && r->N <= (1 << 22), "request: N=%d out of range", r->N);
    RS_CHECK_ARG(r->prot_xyz && r->prot_q, "request: protein pointers are NULL");
    RS_CHECK_ARG(r->params.n >= 3 && r->params.n <= 16385, "request: n=%d out of range", r->params.n);
    RS_CHECK_ARG(r->params.b > 0 && r->params.sigma > 0, "request: b and sigma must be > 0");
    RS_CHECK_ARG(r->params.R_l >= 2 && r->params.R_l <= 64, "request: R_l=%d out of range", r->params.R_l);
    RS_CHECK_ARG(r->params.tucker_cap >= 0 && r->params.tucker_cap <= RS_MAX_TUCKER,
                 "request: tucker_cap=%d out of range", r->params.tucker_cap);
    return RS_OK;
}

void rs_serve_params_default(rs_serve_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->mem_budget_bytes = 0;
    p->max_queue = 1 << 16;
    p->max_inflight_launches = 2;
    p->idle_wait_ms = 2;
    p->inject_alloc_failures = 0;
    p->group_min_atoms = rs::kDenseMinAtoms;
    p->group_atoms_per_cell = rs::kDenseAtomsPerCell;
}

rs_status rs_serve_create(int device, const rs_serve_params* prm, rs_server** out) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(out, "rs_serve_create: out is NULL");
    *out = nullptr;
    rs_serve_params p;
    if (prm) p = *prm;
    else rs_serve_params_default(&p);
    RS_CHECK_ARG(p.max_queue >= 1, "rs_serve_create: max_queue must be >= 1");
    RS_CHECK_ARG(p.max_inflight_launches >= 1 && p.max_inflight_launches <= 8,
                 "rs_serve_create: max_inflight_launches must be in [1, 8]");
    RS_CHECK_ARG(p.inject_alloc_failures >= 0, "rs_serve_create: inject_alloc_failures < 0");
    RS_CHECK_ARG(p.group_min_atoms >= 0 && p.group_atoms_per_cell >= 0.0,
                 "rs_serve_create: negative grouping threshold");
    rs_ctx* ctx = nullptr;
    rs_ctx* bctx = nullptr;
    RS_TRY(rs_ctx_create(device, &ctx));
    if (rs_ctx_create(device, &bctx) != RS_OK) {
        rs_ctx_destroy(ctx);
        return RS_ERR_CUDA;
    }
    rs_server* S = new rs_server();
    S->ctx = ctx;
    S->bctx = bctx;
    S->prm = p;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
    }
    S->budget = p.mem_budget_bytes ? (size_t)p.mem_budget_bytes : fr / 2;
    S->inject_left = p.inject_alloc_failures;
    S->dev.inject = &S->inject_left;
    S->bhold = p.hold_builds != 0;
    S->pinned.host = true;
    // one stream per in-flight launch plus one for protein builds
    for (int i = 0; i <= p.max_inflight_launches; ++i) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            rs_ctx_destroy(ctx);
            rs_ctx_destroy(bctx);
            delete S;
            set_error("rs_serve_create: stream creation failed");
            return RS_ERR_CUDA;
        }
        S->streams.push_back(s);
    }
    S->stream_busy.assign(p.max_inflight_launches, false);
    S->st.budget_bytes = S->budget;
    S->worker = std::thread(worker_main, S);
    S->builder = std::thread(builder_main, S);
    *out = S;
    return RS_OK;
}

rs_status rs_serve_release_builds(rs_server* S) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(S, "rs_serve_release_builds: NULL server");
    {
        std::lock_guard<std::mutex> lk(S->bmu);
        S->bhold = false;
    }
    S->bcv.notify_all();
    return RS_OK;
}

rs_status rs_serve_submit(rs_server* S, const rs_request* r, double* E_out, uint8_t* flags_out,
                          uint64_t* req_id) {
    using namespace rs;
    clear_error();
    RS_CHECK_ARG(S && req_id, "rs_serve_submit: NULL argument");
    RS_TRY(rs_request_validate(r));
    RS_CHECK_ARG(r->P == 0 || E_out, "rs_serve_submit: E_out is NULL");
    Request* q = new Request();
    q->req = *r;
    q->E_host = E_out;
    q->flags_host = flags_out;
    q->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete q;
            set_error("rs_serve_submit: server is shutting down");
            return RS_ERR_BUSY;
        }
        if ((int)S->queue.size() >= S->prm.max_queue) {
            delete q;
            set_error("rs_serve_submit: queue full (%d)", S->prm.max_queue);
            return RS_ERR_BUSY;
        }
        q->id = S->next_id++;
        S->queue.push_back(q);
        S->reqs[q->id] = q;
    }
    S->cv_work.notify_one();
    *req_id = q->id;
    return RS_OK;
}

// Under S->mu.
static rs_status take_result(rs_server* S, uint64_t id, rs_result* out) {
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) {
        rs::set_error("unknown request id %llu", (unsigned long long)id);
        return RS_ERR_INVALID;
    }
    rs::Request* r = it->second;
    if (r->state != rs::DONE) return RS_ERR_NOT_READY;
    if (out) {
        out->status = r->status;
        out->t_submit_ns = r->t_submit;
        out->t_admit_ns = r->t_admit;
        out->t_start_ns = r->t_start;
        out->t_end_ns = r->t_end;
        snprintf(out->message, sizeof(out->message), "%s", r->message);
    }
    delete r;
    S->reqs.erase(it);
    return RS_OK;
}

rs_status rs_serve_poll(rs_server* S, uint64_t id, rs_result* out) {
    rs::clear_error();
    RS_CHECK_ARG(S, "rs_serve_poll: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    return take_result(S, id, out);
}

rs_status rs_serve_wait(rs_server* S, uint64_t id, int32_t timeout_ms, rs_result* out) {
    rs::clear_error();
    RS_CHECK_ARG(S, "rs_serve_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    for (;;) {
        rs_status s = take_result(S, id, out);
        if (s != RS_ERR_NOT_READY) return s;
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            s = take_result(S, id, out);
            if (s != RS_ERR_NOT_READY) return s;
            rs::set_error("request %llu still pending after %d ms", (unsigned long long)id, timeout_ms);
            return RS_ERR_TIMEOUT;
        }
    }
}

rs_status rs_serve_cancel(rs_server* S, uint64_t id) {
    rs::clear_error();
    RS_CHECK_ARG(S, "rs_serve_cancel: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) {
        rs::set_error("rs_serve_cancel: unknown request id %llu", (unsigned long long)id);
        return RS_ERR_INVALID;
    }
    rs::Request* r = it->second;
    if (r->state != rs::QUEUED) {
        rs::set_error("rs_serve_cancel: request %llu already admitted", (unsigned long long)id);
        return RS_ERR_BUSY;
    }
    auto q = std::find(S->queue.begin(), S->queue.end(), r);
    if (q != S->queue.end()) S->queue.erase(q);
    r->state = rs::CANCELLED;
    S->graveyard.push_back(r);  // the scheduler may still hold it in a snapshot
    S->reqs.erase(it);
    return RS_OK;
}

rs_status rs_serve_get_stats(rs_server* S, rs_serve_stats* out) {
    rs::clear_error();
    RS_CHECK_ARG(S && out, "rs_serve_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->queued = S->queue.size();
    out->mean_requests_per_launch = S->st.launches ? S->reqs_launched / (double)S->st.launches : 0.0;
    return RS_OK;
}

void rs_serve_destroy(rs_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    {
        std::lock_guard<std::mutex> lk(S->bmu);
        S->bstop = true;
    }
    S->cv_work.notify_all();
    S->bcv.notify_all();
    if (S->worker.joinable()) S->worker.join();  // retires every launch before it exits
    if (S->builder.joinable()) S->builder.join();  // finishes the build it is in
    cudaSetDevice(S->ctx->device);
    for (cudaStream_t s : S->streams) cudaStreamSynchronize(s);
    for (auto& d : S->bdone) rs_protein_free(d.prot);
    for (auto& kv : S->cache) rs_protein_free(kv.second.prot);
    S->cache.clear();
    for (auto& kv : S->reqs) delete kv.second;
    for (rs::Request* g : S->graveyard) delete g;
    S->reqs.clear();
    S->dev.clear();
    S->pinned.clear();
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    rs_ctx_destroy(S->ctx);
    rs_ctx_destroy(S->bctx);
    delete S;
}

}  // extern "C"
