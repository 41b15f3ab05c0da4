// C ABI of the batched step (elbm_batch_*, declared in include/elbm.h):
// membership, the device member table, the block-size autotuner and the CUDA
// graphs of launch sequences.
//
// A batch has one of two forms, fixed by the kernel form of its members.
//  * Two-pass members (form 1): the batched kernels read the member table from
//    constant memory (one table per storage mode, refreshed before each launch
//    sequence), so a live batch owns the table of its (lattice, storage) kind:
//    one live batch of this form per kind and device.  A launch sequence of n
//    steps is captured once as a CUDA graph; when membership changes the block
//    total, the graph is re-captured and the executable graph updated in place.
//  * Single-pass members (form 3, two population arrays each): every member's
//    n-step sequence of single-pass launches is captured once as a graph of
//    its own and replayed on a pool of private streams, so the members' blocks
//    run side by side; a member's result is bit-identical to stepping it alone
//    because it is the same sequence of launches.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

#include "elbm_internal.h"

struct elbm_batch {
    std::vector<elbm_solver*> members;
    std::vector<elbm::BatchMember> table;
    int lattice = 0, storage = 0, D = 0, device = 0;
    int blocks[2] = {0, 0};            // current block totals (128, 256 threads)
    cudaStream_t stream = nullptr;      // the members' stream
    cudaStream_t exec_stream = nullptr; // private stream that captures and replays graphs
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int block_size = 0;                // chosen by the autotuner
    float tuned_ms[2] = {0, 0};
    struct Seq {
        cudaGraphExec_t exec = nullptr;
        int grid = 0;                  // block total it was captured for
    };
    std::map<int, Seq> graphs;         // launch sequences by step count
    long long launches = 0;
    int form = 1;                      // 1 two-pass members, 3 single-pass members
    struct MemberGraph {               // form 3: one member's n-step sequence
        long long uid = 0;             // the member's solver (uid, never reused)
        int nsteps = 0;
        const void* f = nullptr;       // its current array when captured
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;
    };
    std::vector<MemberGraph> member_graphs;
    struct Retired {                   // graphs of departed members, destroyed once `done` has passed
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<Retired> retired;
    std::vector<cudaStream_t> pool;    // form 3: private streams the member graphs run on
    std::vector<cudaEvent_t> pool_done;
};

namespace {

int bfail(int code, const char* msg) { return elbm::set_error(code, msg); }

int bcuda(cudaError_t e, const char* what)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return elbm::set_error(e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA, buf);
}

// Block size chosen by the autotuner, per (lattice, storage), shared by every
// batch of the process: the first batch of a kind pays the two tuning steps.
std::mutex g_tune_lock;
std::map<std::pair<int, int>, int> g_tuned;
// Kinds (device, lattice, storage) with a live batch: each owns a constant table.
std::set<std::tuple<int, int, int>> g_live;

void drop_graphs(elbm_batch* b)
{
    for (auto& kv : b->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    b->graphs.clear();
}

// ------------------------------------------------------------ form 3 helpers
constexpr int kPoolStreams = 16;     // private streams of a single-pass batch
constexpr int kGraphsPerMember = 4;  // cached step counts per member

int member_form(const elbm_solver* s) { return elbm::effective_kernel(s) == 3 ? 3 : 1; }

// Hand the cached graphs of solver uid over for destruction once the work
// enqueued so far on the batch's stream (which every member launch joins) is done.
cudaError_t retire_graphs(elbm_batch* b, long long uid, int keep_newest)
{
    std::vector<size_t> idx;
    for (size_t k = 0; k < b->member_graphs.size(); ++k)
        if (b->member_graphs[k].uid == uid) idx.push_back(k);
    if ((int)idx.size() <= keep_newest) return cudaSuccess;
    const size_t drop = idx.size() - (size_t)keep_newest;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
    if (e != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        return e;
    }
    bool first = true;
    for (size_t j = drop; j-- > 0;) {
        elbm_batch::Retired r;
        r.exec = b->member_graphs[idx[j]].exec;
        r.done = first ? ev : nullptr;  // one event covers the whole group (kept with its first entry)
        first = false;
        b->retired.push_back(r);
        b->member_graphs.erase(b->member_graphs.begin() + (long)idx[j]);
    }
    return cudaSuccess;
}

// Destroy retired graphs whose last launches have completed (all of them when wait).
void reap(elbm_batch* b, bool wait)
{
    std::vector<elbm_batch::Retired> keep;
    bool passed = true;  // whether the group of the entries that follow has passed its event
    for (auto& r : b->retired) {
        if (r.done) passed = wait ? cudaEventSynchronize(r.done) == cudaSuccess : cudaEventQuery(r.done) == cudaSuccess;
        if (passed) {
            if (r.exec) cudaGraphExecDestroy(r.exec);
            if (r.done) cudaEventDestroy(r.done);
        } else {
            keep.push_back(r);
        }
    }
    (void)cudaGetLastError();  // a query that found pending work is not an error
    b->retired.swap(keep);
}

// The executable graph of nsteps single-pass steps of member s from its
// current array (captured on stream ps the first time).
cudaError_t member_graph(elbm_batch* b, elbm_solver* s, int nsteps, cudaStream_t ps, cudaGraphExec_t* exec,
                         long long* launches)
{
    for (const auto& g : b->member_graphs)
        if (g.uid == s->uid && g.nsteps == nsteps && g.f == s->f) {
            *exec = g.exec;
            *launches = g.launches;
            return cudaSuccess;
        }
    cudaError_t e = retire_graphs(b, s->uid, kGraphsPerMember - 1);
    if (e != cudaSuccess) return e;
    elbm::Solver seq = *s;  // the member as the capture sees it: its own arrays, the pool stream
    seq.stream = ps;
    elbm_batch::MemberGraph g;
    g.uid = s->uid;
    g.nsteps = nsteps;
    g.f = s->f;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e1 = cudaSuccess;
    for (int k = 0; k < nsteps && e1 == cudaSuccess; ++k) {
        e1 = elbm::step_single_impl<3>(seq, seq.f2, &g.launches);
        std::swap(seq.f, seq.f2);
    }
    e = cudaStreamEndCapture(ps, &graph);
    if (e == cudaSuccess) e = e1;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    b->member_graphs.push_back(g);
    *exec = g.exec;
    *launches = g.launches;
    return cudaSuccess;
}

cudaError_t ensure_pool(elbm_batch* b, int n)
{
    while ((int)b->pool.size() < n) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (st) cudaStreamDestroy(st);
            return e;
        }
        b->pool.push_back(st);
        b->pool_done.push_back(ev);
    }
    return cudaSuccess;
}

// nsteps single-pass steps of every member: fork the pool streams from the
// batch's stream, launch each member's graph on one of them, join them back.
int step_single_form(elbm_batch* b, int nsteps)
{
    for (const auto* s : b->members)
        if (member_form(s) != 3 || s->parity != 0 || !s->f2)
            return bfail(ELBM_ERR_STATE, "a member of a single-pass batch no longer steps in the single-pass form");
    reap(b, false);
    const int n = (int)b->members.size(), P = std::min(n, kPoolStreams);
    cudaError_t e = ensure_pool(b, P);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in, b->stream);
    for (int k = 0; k < P && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->pool[k], b->ev_in, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        elbm_solver* s = b->members[k];
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;
        e = member_graph(b, s, nsteps, b->pool[k % P], &exec, &launches);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->pool[k % P]);
        if (e == cudaSuccess) {
            b->launches += launches;
            s->launches += launches;
        }
    }
    for (int k = 0; k < P && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->pool_done[k], b->pool[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->pool_done[k], 0);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return bcuda(e, "elbm_batch_step");
    }
    for (auto* s : b->members) {
        if (nsteps & 1) std::swap(s->f, s->f2);
        s->steps_done += nsteps;
    }
    return ELBM_OK;
}

cudaError_t join_in(elbm_batch* b)
{
    cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
    return e == cudaSuccess ? cudaStreamWaitEvent(b->exec_stream, b->ev_in, 0) : e;
}
cudaError_t join_out(elbm_batch* b)
{
    cudaError_t e = cudaEventRecord(b->ev_out, b->exec_stream);
    return e == cudaSuccess ? cudaStreamWaitEvent(b->stream, b->ev_out, 0) : e;
}

// Recompute the block layout, refresh every member's parameter block and
// parity, and upload the table to the constant memory of the batch's kind (on
// the private stream, ordered before the next launch sequence; copies from
// pageable memory return once the source has been read).
cudaError_t upload(elbm_batch* b)
{
    const size_t n = b->members.size();
    long long begin128 = 0, begin256 = 0;
    b->table.resize(n);
    for (size_t k = 0; k < n; ++k) {
        elbm_solver* s = b->members[k];
        elbm::fill_params(*s, b->table[k].p);
        b->table[k].parity = s->parity;
        b->table[k].block_begin[0] = (int)begin128;
        b->table[k].block_begin[1] = (int)begin256;
        begin128 += (s->N + 127) / 128;
        begin256 += (s->N + 255) / 256;
    }
    b->blocks[0] = (int)begin128;
    b->blocks[1] = (int)begin256;
    return (b->D == 2) ? elbm::batch_upload_impl<2>(b->storage, b->table.data(), (int)n, b->exec_stream)
                       : elbm::batch_upload_impl<3>(b->storage, b->table.data(), (int)n, b->exec_stream);
}

cudaError_t enqueue(elbm_batch* b, int block_size, int grid, int nsteps)
{
    return (b->D == 2) ? elbm::batch_enqueue_impl<2>(b->storage, block_size, grid, nsteps, b->exec_stream, &b->launches)
                       : elbm::batch_enqueue_impl<3>(b->storage, block_size, grid, nsteps, b->exec_stream, &b->launches);
}

void advance_members(elbm_batch* b, int nsteps)
{
    for (auto* s : b->members) {
        s->parity = (s->parity + nsteps) & 1;
        s->steps_done += nsteps;
    }
}

// One real step per candidate block size, timed with events; the faster wins.
// Every candidate computes the same bits, so the tuning steps are ordinary steps.
int autotune(elbm_batch* b, int* steps_left)
{
    const int candidates[2] = {256, 128};
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    int rc = ELBM_OK;
    for (int c = 0; c < 2 && *steps_left > 0; ++c) {
        const int bs = candidates[c], idx = bs == 128 ? 0 : 1;
        cudaError_t e = join_in(b);
        if (e == cudaSuccess) e = upload(b);
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->exec_stream);
        if (e == cudaSuccess) e = enqueue(b, bs, b->blocks[idx], 1);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->exec_stream);
        if (e == cudaSuccess) e = join_out(b);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e != cudaSuccess) {
            rc = bcuda(e, "elbm_batch_step (tuning)");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        b->tuned_ms[idx] = ms;
        advance_members(b, 1);
        --*steps_left;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc == ELBM_OK && b->tuned_ms[0] > 0.f && b->tuned_ms[1] > 0.f) {
        b->block_size = (b->tuned_ms[0] < b->tuned_ms[1]) ? 128 : 256;
        std::lock_guard<std::mutex> lock(g_tune_lock);
        g_tuned[{b->lattice, b->storage}] = b->block_size;
    }
    return rc;
}

int check_member(const elbm_batch* b, const elbm_solver* s)
{
    if (!s) return bfail(ELBM_ERR_ARG, "NULL solver in batch");
    if (!s->initialised) return bfail(ELBM_ERR_STATE, "batch member not initialised");
    if (s->lattice != b->lattice || s->storage != b->storage)
        return bfail(ELBM_ERR_ARG, "batch members must share lattice and storage mode");
    if (s->stream != b->stream) return bfail(ELBM_ERR_ARG, "batch members must share one stream");
    if (member_form(s) != b->form)
        return bfail(ELBM_ERR_ARG, "batch members must share the kernel form (single pass or two-pass)");
    if (b->form == 1 && (s->eq_mode == 2 || s->walls_y || s->g[0] != 0.0 || s->g[1] != 0.0 || s->g[2] != 0.0))
        return bfail(ELBM_ERR_ARG, "the batched step takes periodic, unforced solvers with the extended or "
                                   "product-form equilibrium");
    if (b->form == 3 && (s->parity != 0 || !s->f2))
        return bfail(ELBM_ERR_STATE, "single-pass batch member not in the own-location layout");
    if (std::find(b->members.begin(), b->members.end(), s) != b->members.end())
        return bfail(ELBM_ERR_ARG, "solver listed twice in batch");
    if ((int)b->members.size() >= elbm::kBatchMax) return bfail(ELBM_ERR_ARG, "a batch holds at most 40 solvers");
    return ELBM_OK;
}

}  // namespace

extern "C" {

void elbm_batch_destroy(elbm_batch* b);

int elbm_batch_create(elbm_solver* const* solvers, int n, elbm_batch** out)
{
    if (!out) return bfail(ELBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!solvers || n < 1 || !solvers[0]) return bfail(ELBM_ERR_ARG, "a batch needs at least one solver");
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    elbm_batch* b = new elbm_batch();
    b->lattice = solvers[0]->lattice;
    b->storage = solvers[0]->storage;
    b->D = solvers[0]->D;
    b->stream = solvers[0]->stream;
    b->device = solvers[0]->device;
    b->form = member_form(solvers[0]);
    for (int k = 0; k < n; ++k) {
        const int rc = check_member(b, solvers[k]);
        if (rc != ELBM_OK) {
            delete b;
            return rc;
        }
        b->members.push_back(solvers[k]);
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_lock);
        if (b->form == 1 && !g_live.insert({b->device, b->lattice, b->storage}).second) {
            delete b;
            return bfail(ELBM_ERR_STATE, "a batch of this lattice and storage mode is already live on this device");
        }
        auto it = g_tuned.find({b->lattice, b->storage});
        if (b->form == 1 && it != g_tuned.end()) b->block_size = it->second;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->exec_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        elbm_batch_destroy(b);
        return bcuda(e, "elbm_batch_create");
    }
    *out = b;
    return ELBM_OK;
}

int elbm_batch_add(elbm_batch* b, elbm_solver* s)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    const int rc = check_member(b, s);
    if (rc != ELBM_OK) return rc;
    b->members.push_back(s);
    return ELBM_OK;
}

int elbm_batch_remove(elbm_batch* b, elbm_solver* s)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    auto it = std::find(b->members.begin(), b->members.end(), s);
    if (it == b->members.end()) return bfail(ELBM_ERR_ARG, "solver is not in the batch");
    if (b->form == 3) {
        const cudaError_t e = retire_graphs(b, s->uid, 0);
        if (e != cudaSuccess) return bcuda(e, "elbm_batch_remove");
    }
    b->members.erase(it);
    return ELBM_OK;
}

int elbm_batch_size(const elbm_batch* b) { return b ? (int)b->members.size() : 0; }

int elbm_batch_step(elbm_batch* b, int nsteps)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(ELBM_ERR_ARG, "nsteps must be >= 0");
    if (b->members.empty() || nsteps == 0) return ELBM_OK;
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (b->form == 3) return step_single_form(b, nsteps);
    int left = nsteps;
    if (b->block_size == 0) {
        const int rc = autotune(b, &left);
        if (rc != ELBM_OK) return rc;
    }
    if (left == 0) return ELBM_OK;
    const int bs = b->block_size ? b->block_size : 256, idx = bs == 128 ? 0 : 1;
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    cudaError_t e = join_in(b);
    if (e == cudaSuccess) e = upload(b);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) {
        elbm_batch::Seq& seq = b->graphs[left];
        if (!seq.exec || seq.grid != b->blocks[idx]) {
            // capture the launch sequence for the current block total; update
            // the executable graph in place when it exists
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->exec_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = enqueue(b, bs, b->blocks[idx], left);
                e = cudaStreamEndCapture(b->exec_stream, &g);
                if (e == cudaSuccess) e = e1;
            }
            if (e == cudaSuccess && seq.exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(seq.exec, g, &info) != cudaSuccess) {
                    (void)cudaGetLastError();
                    cudaGraphExecDestroy(seq.exec);
                    seq.exec = nullptr;
                }
            }
            if (e == cudaSuccess && !seq.exec) e = cudaGraphInstantiate(&seq.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) seq.grid = b->blocks[idx];
        }
        exec = seq.exec;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->exec_stream);
    if (e == cudaSuccess) e = join_out(b);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return bcuda(e, "elbm_batch_step");
    }
    advance_members(b, left);
    return ELBM_OK;
}

int elbm_batch_info(const elbm_batch* b, int* block_size, double* tuned_ms, long long* launches)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    if (block_size) *block_size = b->form == 1 ? b->block_size : 0;
    if (tuned_ms) {
        tuned_ms[0] = b->tuned_ms[0];
        tuned_ms[1] = b->tuned_ms[1];
    }
    if (launches) *launches = b->launches;
    return ELBM_OK;
}

void elbm_batch_destroy(elbm_batch* b)
{
    if (!b) return;
    if (b->exec_stream) cudaStreamSynchronize(b->exec_stream);
    for (auto st : b->pool) cudaStreamSynchronize(st);
    drop_graphs(b);
    for (auto& g : b->member_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    b->member_graphs.clear();
    reap(b, true);
    for (size_t k = 0; k < b->pool.size(); ++k) {
        cudaEventDestroy(b->pool_done[k]);
        cudaStreamDestroy(b->pool[k]);
    }
    if (b->form == 1) {
        std::lock_guard<std::mutex> lock(g_tune_lock);
        g_live.erase({b->device, b->lattice, b->storage});
    }
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->exec_stream) cudaStreamDestroy(b->exec_stream);
    delete b;
}

}  // extern "C"
