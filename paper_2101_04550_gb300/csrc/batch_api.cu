// C ABI of the batched step (elbm_batch_*, declared in include/elbm.h):
// membership, the device member table, the block-size autotuner and the CUDA
// graphs of launch sequences.
//
// A batch has one of two forms, fixed by the kernel form of its members.
//  * Two-pass members (form 1): the batched kernels read the member table from
//    device memory of the batch, refreshed before each launch sequence.  A
//    launch sequence of n steps is captured once as a CUDA graph; when
//    membership changes the block total, the graph is re-captured and the
//    executable graph updated in place.
//  * Single-pass members (form 3, two population arrays each).  Members whose
//    grids the TMEM single pass takes advance together in one launch per step
//    of the flattened batch kernel (batch_single.cuh) over a work list of
//    (member, tile column, z range) items; the n launches of a call are
//    captured once as a CUDA graph and replayed.  The work list's segment
//    depth and order come from an autotuner written here, which times two
//    real steps of every candidate -- segments of 32, 16 or 8 planes, members
//    one after another or interleaved, and per-member graphs -- and keeps the
//    fastest per (storage, walls/force, size class of the batch) for the
//    process.  Other single-pass members (32 x 8 TMA or cp.async kernels), and
//    every member when the tuner picks it, run as per-member graphs: each
//    member's n-step sequence of solo launches captured once and replayed on
//    a pool of private streams, so the members' blocks run side by side.
//    Either way a member's result is bit-identical to stepping it alone.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
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
    // form 3, flattened launch: member records (host copy and device table),
    // the work list on the device and the graphs of n launches
    struct SpCached {                  // a member's record, arrays in the order first seen
        long long uid = 0;
        const void* a0 = nullptr;
        const void* a1 = nullptr;
        std::vector<unsigned char> rec;
    };
    std::vector<SpCached> sp_cache;
    std::vector<unsigned char> sp_table;
    void* sp_table_dev = nullptr;
    size_t sp_table_cap = 0;
    void* sp_work_dev = nullptr;
    size_t sp_work_cap = 0;
    int sp_nwork = 0;
    std::vector<long long> sp_work_sig;   // what the uploaded work list was built from
    struct SpGraph {
        cudaGraphExec_t exec = nullptr;
        int nwork = 0;
        bool bc = false;
        bool fx = false;
        int rows = 16;
    };
    std::map<int, SpGraph> sp_graphs;  // by step count
    struct Staging {                   // pinned host buffer of an asynchronous upload
        void* host = nullptr;
        size_t cap = 0;
        cudaEvent_t done = nullptr;    // recorded after the copy out of it
    };
    Staging sp_stage[3][2];            // [single-pass table, work list, two-pass table][alternate buffers]
    int sp_stage_next[3] = {0, 0, 0};
    void* tp_table_dev = nullptr;      // two-pass member table (kBatchMax records)
    int sp_pinned = -1;                // configuration set by elbm_batch_set_config (-1: the autotuner's)
    int sp_config = -1;                // configuration of the last flattened call
    long long sp_key = -1;             // its tuning key
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

// Autotuner candidates of the single-pass batch: configurations 0..11 are
// the flattened launch -- TMEM kernel on 32 x 16 tile columns (c < 6) or TMA
// kernel on 32 x 8 (6 <= c < 12), segments of kSegCand[c % 3] planes, members
// one after another or interleaved item by item ((c % 6) >= 3) -- over the
// members that kernel takes, the other members as per-member graphs;
// configuration 12 is per-member graphs for every member.
constexpr int kSpCandidates = ELBM_BATCH_CONFIGS;
constexpr int kSpGraphs = ELBM_BATCH_CONFIGS - 1;
constexpr int kSegCand[3] = {32, 16, 8};
int cfg_tile_rows(int c) { return c < 6 ? 16 : 8; }
bool cfg_interleaved(int c) { return (c % 6) >= 3; }
struct SpTuning {
    double ms[kSpCandidates] = {};
    int next = 0;        // next candidate to time
    int chosen = -1;
};
// Shared by every batch of the process, by (storage, walls/force, size class).
std::map<long long, SpTuning> g_sp_tuning;

bool bounded_member(const elbm_solver* s)
{
    return s->walls_y || s->g[0] != 0.0 || s->g[1] != 0.0 || s->g[2] != 0.0;
}

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
        e1 = (seq.D == 2) ? elbm::step_single_impl<2>(seq, seq.f2, &g.launches)
                          : elbm::step_single_impl<3>(seq, seq.f2, &g.launches);
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

// nsteps single-pass steps of the given members as per-member graphs: fork
// the pool streams from the batch's stream, launch each member's graph on one
// of them, join them back.  The members' arrays are not swapped here.
cudaError_t run_member_graphs(elbm_batch* b, const std::vector<elbm_solver*>& ms, int nsteps)
{
    if (ms.empty() || nsteps == 0) return cudaSuccess;
    const int n = (int)ms.size(), P = std::min(n, kPoolStreams);
    cudaError_t e = ensure_pool(b, P);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in, b->stream);
    for (int k = 0; k < P && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->pool[k], b->ev_in, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        elbm_solver* s = ms[k];
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
    return e;
}

cudaError_t join_in(elbm_batch* b);
cudaError_t join_out(elbm_batch* b);

// Members the flattened launch of configuration c takes (the others run as
// per-member graphs).
std::vector<elbm_solver*> flat_of(const elbm_batch* b, int c, std::vector<elbm_solver*>* rest)
{
    std::vector<elbm_solver*> flat;
    for (auto* s : b->members) {
        const bool takes = c < 6 ? elbm::single_pass_variant(*s) == 1 : c < kSpGraphs && elbm::sp_tma_member(*s);
        (takes ? flat : *rest).push_back(s);
    }
    return flat;
}

// Tuning key of a batch: storage, walls/force, floor(log2(total nodes)).
long long sp_key(const elbm_batch* b, const std::vector<elbm_solver*>& members)
{
    long long nodes = 0;
    bool bc = false;
    for (const auto* s : members) {
        nodes += s->N;
        bc = bc || bounded_member(s);
    }
    int cls = 0;
    while ((2ll << cls) <= nodes) ++cls;
    return ((long long)b->storage * 2 + (bc ? 1 : 0)) * 64 + cls;
}

// Enqueue the copy of `bytes` from src to dev on the batch's private stream
// through pinned staging buffer pair `which` (0 single-pass table, 1 work
// list, 2 two-pass table), so that
// the copy does not make the host wait for the stream; a buffer is reused
// once the copy out of it two uploads ago has run.
cudaError_t staged_upload(elbm_batch* b, int which, void* dev, const void* src, size_t bytes)
{
    elbm_batch::Staging& st = b->sp_stage[which][b->sp_stage_next[which]];
    b->sp_stage_next[which] ^= 1;
    cudaError_t e = cudaSuccess;
    if (st.done) e = cudaEventSynchronize(st.done);
    if (e == cudaSuccess && bytes > st.cap) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.cap = 0;
        e = cudaHostAlloc(&st.host, 2 * bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) st.cap = 2 * bytes;
    }
    if (e == cudaSuccess && !st.done) e = cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    std::memcpy(st.host, src, bytes);
    e = cudaMemcpyAsync(dev, st.host, bytes, cudaMemcpyHostToDevice, b->exec_stream);
    if (e == cudaSuccess) e = cudaEventRecord(st.done, b->exec_stream);
    return e;
}

// Member records of the flattened members into the device table, each with
// the phase of its current array.
cudaError_t sp_upload_table(elbm_batch* b, const std::vector<elbm_solver*>& flat)
{
    const size_t rb = elbm::sp_member_bytes();
    b->sp_table.resize(rb * flat.size());
    for (size_t k = 0; k < flat.size(); ++k) {
        elbm_solver* s = flat[k];
        elbm_batch::SpCached* c = nullptr;
        for (auto& x : b->sp_cache)
            if (x.uid == s->uid) c = &x;
        const bool same = c && ((c->a0 == s->f && c->a1 == s->f2) || (c->a0 == s->f2 && c->a1 == s->f));
        if (!c) {
            b->sp_cache.push_back({});
            c = &b->sp_cache.back();
        }
        elbm::Solver fixed = *s;  // arrays in the record's order
        if (same) {
            fixed.f = const_cast<void*>(c->a0);
            fixed.f2 = const_cast<void*>(c->a1);
        } else {
            c->uid = s->uid;
            c->a0 = s->f;
            c->a1 = s->f2;
            c->rec.assign(rb, 0);
        }
        const cudaError_t e = elbm::sp_member_fill(fixed, c->rec.data(), !same);
        if (e != cudaSuccess) return e;
        unsigned char* rec = b->sp_table.data() + k * rb;
        std::memcpy(rec, c->rec.data(), rb);
        elbm::sp_member_set_phase(rec, s->f == c->a0 ? 0 : 1);
    }
    const size_t bytes = b->sp_table.size();
    if (bytes > b->sp_table_cap) {
        cudaError_t e = cudaStreamSynchronize(b->exec_stream);  // nothing may still read the old table
        if (b->sp_table_dev) cudaFree(b->sp_table_dev);
        b->sp_table_dev = nullptr;
        b->sp_table_cap = 0;
        for (auto& kv : b->sp_graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        b->sp_graphs.clear();
        if (e == cudaSuccess) e = cudaMalloc(&b->sp_table_dev, 2 * bytes);
        if (e != cudaSuccess) return e;
        b->sp_table_cap = 2 * bytes;
    }
    return staged_upload(b, 0, b->sp_table_dev, b->sp_table.data(), bytes);
}

// Work list of configuration c over the flattened members (rebuilt and
// uploaded only when the members or the configuration change).
cudaError_t sp_upload_work(elbm_batch* b, const std::vector<elbm_solver*>& flat, int c)
{
    std::vector<long long> sig{c};
    for (const auto* s : flat) sig.insert(sig.end(), {s->uid, s->nx, s->ny, s->nz});
    if (sig == b->sp_work_sig && b->sp_work_dev) return cudaSuccess;
    const int seg = kSegCand[c % 3], rows = cfg_tile_rows(c);
    std::vector<std::vector<int4>> per(flat.size());
    for (size_t m = 0; m < flat.size(); ++m) {
        const elbm_solver* s = flat[m];
        for (int z0 = 0; z0 < s->nz; z0 += seg)
            for (int y0 = 0; y0 < s->ny; y0 += rows)
                for (int x0 = 0; x0 < s->nx; x0 += 32)
                    per[m].push_back(make_int4((int)m, x0, y0, z0 | (std::min(s->nz, z0 + seg) << 16)));
    }
    std::vector<int4> work;
    if (!cfg_interleaved(c)) {
        for (auto& v : per) work.insert(work.end(), v.begin(), v.end());
    } else {
        for (size_t k = 0;; ++k) {
            bool any = false;
            for (auto& v : per)
                if (k < v.size()) {
                    work.push_back(v[k]);
                    any = true;
                }
            if (!any) break;
        }
    }
    const size_t bytes = work.size() * sizeof(int4);
    if (bytes > b->sp_work_cap) {
        cudaError_t e = cudaStreamSynchronize(b->exec_stream);
        if (b->sp_work_dev) cudaFree(b->sp_work_dev);
        b->sp_work_dev = nullptr;
        b->sp_work_cap = 0;
        for (auto& kv : b->sp_graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        b->sp_graphs.clear();
        if (e == cudaSuccess) e = cudaMalloc(&b->sp_work_dev, 2 * bytes);
        if (e != cudaSuccess) return e;
        b->sp_work_cap = 2 * bytes;
    }
    b->sp_nwork = (int)work.size();
    b->sp_work_sig = sig;
    return staged_upload(b, 1, b->sp_work_dev, work.data(), bytes);
}

// nsteps steps of the flattened members in configuration c (0..11), as one
// CUDA graph of nsteps launches (graph = true) or as direct launches.
cudaError_t run_flat(elbm_batch* b, const std::vector<elbm_solver*>& flat, int c, int nsteps, bool graph)
{
    if (flat.empty() || nsteps == 0) return cudaSuccess;
    const int rows = cfg_tile_rows(c);
    bool bc = false, fx = true;
    for (const auto* s : flat) {
        bc = bc || bounded_member(s);
        fx = fx && s->g[1] == 0.0 && s->g[2] == 0.0;
    }
    cudaError_t e = join_in(b);
    if (e == cudaSuccess) e = sp_upload_table(b, flat);
    if (e == cudaSuccess) e = sp_upload_work(b, flat, c);
    if (e != cudaSuccess) return e;
    if (!graph) {
        e = elbm::sp_batch_enqueue(b->storage, rows, bc, fx, b->sp_table_dev, b->sp_work_dev, b->sp_nwork, nsteps,
                                   b->exec_stream, &b->launches);
    } else {
        elbm_batch::SpGraph& g = b->sp_graphs[nsteps];
        if (!g.exec || g.nwork != b->sp_nwork || g.bc != bc || g.fx != fx || g.rows != rows) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            cudaGraph_t graph_ = nullptr;
            long long dummy = 0;
            e = cudaStreamBeginCapture(b->exec_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = elbm::sp_batch_enqueue(b->storage, rows, bc, fx, b->sp_table_dev,
                                                              b->sp_work_dev, b->sp_nwork, nsteps, b->exec_stream,
                                                              &dummy);
                e = cudaStreamEndCapture(b->exec_stream, &graph_);
                if (e == cudaSuccess) e = e1;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph_, 0);
            if (graph_) cudaGraphDestroy(graph_);
            if (e != cudaSuccess) return e;
            g.nwork = b->sp_nwork;
            g.bc = bc;
            g.fx = fx;
            g.rows = rows;
        }
        e = cudaGraphLaunch(g.exec, b->exec_stream);
        if (e == cudaSuccess) b->launches += nsteps;
    }
    for (auto* s : flat) s->launches += nsteps;
    if (e == cudaSuccess) e = join_out(b);
    return e;
}

// Time two real steps of the whole batch in every candidate not yet timed
// for this tuning key (as many as *steps_left allows); once all are timed the
// fastest is chosen.  Host-side preparation (the uploads of a flattened
// configuration, the captures of member graphs) stays outside the timed
// interval.
cudaError_t sp_tune(elbm_batch* b, SpTuning& t, int* steps_left)
{
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    while (e == cudaSuccess && t.next < kSpCandidates && *steps_left >= 2) {
        const int c = t.next;
        std::vector<elbm_solver*> rest;
        const std::vector<elbm_solver*> flat = flat_of(b, c, &rest);
        if (!flat.empty()) {
            e = join_in(b);
            if (e == cudaSuccess) e = sp_upload_table(b, flat);
            if (e == cudaSuccess) e = sp_upload_work(b, flat, c);
            if (e == cudaSuccess) e = join_out(b);
        }
        if (e == cudaSuccess && !rest.empty()) e = ensure_pool(b, std::min((int)rest.size(), kPoolStreams));
        for (size_t k = 0; k < rest.size() && e == cudaSuccess; ++k) {
            cudaGraphExec_t exec = nullptr;
            long long launches = 0;
            e = member_graph(b, rest[k], 2, b->pool[k % b->pool.size()], &exec, &launches);
        }
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = run_flat(b, flat, c, 2, false);
        if (e == cudaSuccess) e = run_member_graphs(b, rest, 2);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) break;
        t.ms[c] = ms;
        ++t.next;
        *steps_left -= 2;  // two steps: every member's state is back in the array it started in
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e == cudaSuccess && t.next == kSpCandidates && t.chosen < 0) {
        t.chosen = 0;
        for (int c = 1; c < kSpCandidates; ++c)
            if (t.ms[c] < t.ms[t.chosen]) t.chosen = c;
    }
    return e;
}

// nsteps single-pass steps of every member.
int step_single_form(elbm_batch* b, int nsteps)
{
    for (const auto* s : b->members)
        if (member_form(s) != 3 || s->parity != 0 || !s->f2)
            return bfail(ELBM_ERR_STATE, "a member of a single-pass batch no longer steps in the single-pass form");
    reap(b, false);
    bool any_flat = false;  // does some member take a flattened kernel at all
    for (const auto* s : b->members)
        any_flat = any_flat || elbm::single_pass_variant(*s) == 1 || elbm::sp_tma_member(*s);
    cudaError_t e = cudaSuccess;
    int left = nsteps;
    int c = kSpGraphs;
    if (any_flat) {
        const long long key = sp_key(b, b->members);
        SpTuning* t = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_tune_lock);
            t = &g_sp_tuning[key];  // map nodes stay where they are
        }
        // the tuning steps are real steps of every member (an even number, so
        // each state ends in the array it started in)
        if (t->chosen < 0 && b->sp_pinned < 0) e = sp_tune(b, *t, &left);
        // while still tuning: TMEM tiles, 32-plane segments, member-major
        c = b->sp_pinned >= 0 ? b->sp_pinned : t->chosen >= 0 ? t->chosen : 0;
        b->sp_key = key;
    }
    b->sp_config = c;
    if (e == cudaSuccess && left > 0) {
        std::vector<elbm_solver*> rest;
        const std::vector<elbm_solver*> flat = flat_of(b, c, &rest);
        e = run_flat(b, flat, c, left, true);
        if (e == cudaSuccess) e = run_member_graphs(b, rest, left);
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
    return staged_upload(b, 2, b->tp_table_dev, b->table.data(), n * sizeof(elbm::BatchMember));
}

cudaError_t enqueue(elbm_batch* b, int block_size, int grid, int nsteps)
{
    const int n = (int)b->members.size();
    return (b->D == 2) ? elbm::batch_enqueue_impl<2>(b->storage, block_size, grid, nsteps, b->tp_table_dev, n,
                                                     b->exec_stream, &b->launches)
                       : elbm::batch_enqueue_impl<3>(b->storage, block_size, grid, nsteps, b->tp_table_dev, n,
                                                     b->exec_stream, &b->launches);
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
        auto it = g_tuned.find({b->lattice, b->storage});
        if (b->form == 1 && it != g_tuned.end()) b->block_size = it->second;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->exec_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && b->form == 1)
        e = cudaMalloc(&b->tp_table_dev, sizeof(elbm::BatchMember) * elbm::kBatchMax);
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
        // its flattened-launch record (the next upload rebuilds the table without it)
        b->sp_cache.erase(std::remove_if(b->sp_cache.begin(), b->sp_cache.end(),
                                         [&](const elbm_batch::SpCached& c) { return c.uid == s->uid; }),
                          b->sp_cache.end());
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

int elbm_batch_set_config(elbm_batch* b, int config)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    if (config < -1 || config >= kSpCandidates) return bfail(ELBM_ERR_ARG, "config must be -1 or 0..12");
    if (b->form != 3) return bfail(ELBM_ERR_STATE, "only single-pass batches have a configuration");
    b->sp_pinned = config;
    return ELBM_OK;
}

int elbm_batch_tuning(const elbm_batch* b, int* config, int* tile_rows, int* seg_planes, int* interleaved, double* ms)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    if (b->form != 3 || b->sp_config < 0) return bfail(ELBM_ERR_STATE, "no single-pass batch step has run");
    SpTuning t;
    {
        std::lock_guard<std::mutex> lock(g_tune_lock);
        auto it = g_sp_tuning.find(b->sp_key);
        if (it != g_sp_tuning.end()) t = it->second;
    }
    const int c = b->sp_config;
    if (config) *config = c;
    if (tile_rows) *tile_rows = c < kSpGraphs ? cfg_tile_rows(c) : 0;
    if (seg_planes) *seg_planes = c < kSpGraphs ? kSegCand[c % 3] : 0;
    if (interleaved) *interleaved = c < kSpGraphs && cfg_interleaved(c) ? 1 : 0;
    if (ms)
        for (int k = 0; k < kSpCandidates; ++k) ms[k] = k < t.next ? t.ms[k] : -1.0;
    // no member takes a flattened kernel: nothing to tune, per-member graphs
    if (b->sp_key < 0) return ELBM_OK;
    return t.chosen >= 0 || b->sp_pinned >= 0 ? ELBM_OK : 1;
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
    for (auto& kv : b->sp_graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    b->sp_graphs.clear();
    if (b->sp_table_dev) cudaFree(b->sp_table_dev);
    if (b->sp_work_dev) cudaFree(b->sp_work_dev);
    for (auto& pair : b->sp_stage)
        for (auto& st : pair) {
            if (st.done) cudaEventSynchronize(st.done);
            if (st.host) cudaFreeHost(st.host);
            if (st.done) cudaEventDestroy(st.done);
        }
    reap(b, true);
    for (size_t k = 0; k < b->pool.size(); ++k) {
        cudaEventDestroy(b->pool_done[k]);
        cudaStreamDestroy(b->pool[k]);
    }
    if (b->tp_table_dev) cudaFree(b->tp_table_dev);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->exec_stream) cudaStreamDestroy(b->exec_stream);
    delete b;
}

}  // extern "C"
