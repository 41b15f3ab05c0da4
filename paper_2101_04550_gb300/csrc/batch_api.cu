// C ABI of the batched step (elbm_batch_*, declared in include/elbm.h):
// membership checks, the device member table, the block-size autotuner and
// the CUDA graph of a launch sequence.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "elbm_internal.h"

struct elbm_batch {
    std::vector<elbm_solver*> members;
    std::vector<elbm::BatchMember> table;
    elbm::BatchMember* d_table = nullptr;
    int lattice = 0, storage = 0, D = 0;
    int blocks[2] = {0, 0};        // total blocks for 128- and 256-thread launches
    cudaStream_t stream = nullptr;
    int block_size = 0;            // 0 until the autotuner has chosen 128 or 256
    float tuned_ms[2] = {0, 0};    // time of one tuning step per block size
    cudaGraphExec_t exec = nullptr;
    int exec_steps = 0;
    long long launches = 0;
};

namespace {

int bfail(int code, const char* msg) { return elbm::set_error(code, msg); }

int bcuda(cudaError_t e, const char* what)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return elbm::set_error(e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA, buf);
}

// Refresh every member's parameter block and parity and upload the table.
cudaError_t upload_table(elbm_batch* b)
{
    for (size_t k = 0; k < b->members.size(); ++k) {
        elbm::fill_params(*b->members[k], b->table[k].p);
        b->table[k].parity = b->members[k]->parity;
    }
    return cudaMemcpyAsync(b->d_table, b->table.data(), b->table.size() * sizeof(elbm::BatchMember),
                           cudaMemcpyHostToDevice, b->stream);
}

cudaError_t enqueue(elbm_batch* b, int block_size, int nsteps)
{
    const int blocks = b->blocks[block_size == 128 ? 0 : 1];
    return (b->D == 2) ? elbm::batch_enqueue_impl<2>(b->storage, block_size, b->d_table, (int)b->members.size(),
                                                     blocks, nsteps, b->stream, &b->launches)
                       : elbm::batch_enqueue_impl<3>(b->storage, block_size, b->d_table, (int)b->members.size(),
                                                     blocks, nsteps, b->stream, &b->launches);
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
    for (int c = 0; c < 2 && *steps_left > 0; ++c) {
        cudaError_t e = upload_table(b);
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = enqueue(b, candidates[c], 1);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e != cudaSuccess) {
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            return bcuda(e, "elbm_batch_step (tuning)");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        b->tuned_ms[candidates[c] == 128 ? 0 : 1] = ms;
        advance_members(b, 1);
        --*steps_left;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (b->tuned_ms[0] > 0.f && b->tuned_ms[1] > 0.f)
        b->block_size = (b->tuned_ms[0] < b->tuned_ms[1]) ? 128 : 256;
    return ELBM_OK;
}

}  // namespace

extern "C" {

int elbm_batch_create(elbm_solver* const* solvers, int n, elbm_batch** out)
{
    if (!out) return bfail(ELBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!solvers || n < 1) return bfail(ELBM_ERR_ARG, "a batch needs at least one solver");
    elbm_batch* b = new elbm_batch();
    long long begin128 = 0, begin256 = 0;
    for (int k = 0; k < n; ++k) {
        elbm_solver* s = solvers[k];
        if (!s) { delete b; return bfail(ELBM_ERR_ARG, "NULL solver in batch"); }
        if (!s->initialised) { delete b; return bfail(ELBM_ERR_STATE, "batch member not initialised"); }
        if (k == 0) {
            b->lattice = s->lattice;
            b->storage = s->storage;
            b->D = s->D;
            b->stream = s->stream;
        } else if (s->lattice != b->lattice || s->storage != b->storage) {
            delete b;
            return bfail(ELBM_ERR_ARG, "batch members must share lattice and storage mode");
        } else if (s->stream != b->stream) {
            delete b;
            return bfail(ELBM_ERR_ARG, "batch members must share one stream");
        }
        for (int j = 0; j < k; ++j)
            if (solvers[j] == s) { delete b; return bfail(ELBM_ERR_ARG, "solver listed twice in batch"); }
        b->members.push_back(s);
        elbm::BatchMember m{};
        m.block_begin[0] = (int)begin128;
        m.block_begin[1] = (int)begin256;
        begin128 += (s->N + 127) / 128;
        begin256 += (s->N + 255) / 256;
        b->table.push_back(m);
    }
    if (begin128 >= (1ll << 31)) { delete b; return bfail(ELBM_ERR_ARG, "batch too large"); }
    b->blocks[0] = (int)begin128;
    b->blocks[1] = (int)begin256;
    cudaError_t e = cudaMalloc((void**)&b->d_table, b->table.size() * sizeof(elbm::BatchMember));
    if (e != cudaSuccess) {
        delete b;
        return bcuda(e, "elbm_batch_create");
    }
    *out = b;
    return ELBM_OK;
}

int elbm_batch_step(elbm_batch* b, int nsteps)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(ELBM_ERR_ARG, "nsteps must be >= 0");
    int left = nsteps;
    if (b->block_size == 0) {
        const int rc = autotune(b, &left);
        if (rc != ELBM_OK) return rc;
    }
    if (left == 0) return ELBM_OK;
    const int bs = b->block_size ? b->block_size : 256;
    cudaError_t e = upload_table(b);
    if (e == cudaSuccess && (!b->exec || b->exec_steps != left)) {
        // capture the launch sequence of `left` steps once and replay it
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = enqueue(b, bs, left);
            e = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        b->exec_steps = (e == cudaSuccess) ? left : 0;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return bcuda(e, "elbm_batch_step");
    advance_members(b, left);
    return ELBM_OK;
}

int elbm_batch_info(const elbm_batch* b, int* block_size, double* tuned_ms, long long* launches)
{
    if (!b) return bfail(ELBM_ERR_ARG, "batch is NULL");
    if (block_size) *block_size = b->block_size;
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
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->d_table);
    delete b;
}

}  // extern "C"
