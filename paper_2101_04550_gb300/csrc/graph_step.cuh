// Graph-scheduled pipelined form of the in-place (AA) extended LBGK step.
//
// The correction term needs the anomaly Q~_aaa of the neighbours at the same
// time level (Eq. Paastar1), which the in-place form gets from an anomaly
// pass A over the grid before the collide pass C.  Run over the whole grid,
// the two passes read the populations twice from HBM.  Here the grid is cut
// along its slowest axis (z for D3Q27, y for D2Q9) into K chunks of a few
// layers, and one step is a CUDA graph of 2K kernels A(c), C(c) with the
// edges
//   C(c) <- A(c-1), A(c), A(c+1)     (q of chunks c-1..c+1 complete; A(c) has
//                                     read the slot set of c before C(c)
//                                     rewrites it; slot sets are disjoint)
//   A(c) <- A(c-1)                   (anomaly chunks in order: A(K-1), A(0), A(1), ...)
//   A(c) <- C(c-L)                   (the anomaly pass runs at most L chunks
//                                     ahead, so the populations it reads are
//                                     still in L2 when C re-reads them)
// The graph scheduler runs the A chain and the C kernels concurrently; no
// kernel waits on another from the device, and the graph boundary orders
// consecutive steps.
#pragma once
#include <vector>

#include "step_kernels.cuh"

// Chunks the anomaly kernels may run ahead of the collide kernels, and
// whether consecutive anomaly kernels are also ordered among themselves.
#ifndef ELBM_GRAPH_LOOKAHEAD
#define ELBM_GRAPH_LOOKAHEAD 3
#endif
#ifndef ELBM_GRAPH_CHAIN
#define ELBM_GRAPH_CHAIN 0
#endif

namespace elbm {

template <int D, int ST, int PAR>
__global__ void __launch_bounds__(kBlock) k_anomaly_range(StepParams p, int begin, int end)
{
    const int cell = begin + blockIdx.x * kBlock + threadIdx.x;
    if (cell >= end) return;
    const Node n = make_node<D>(p, cell);
    float g[Lat<D>::Q];
    gather<D, ST, PAR>(p, n, g);
    float drho, j[3];
    moments<D>(p, g, drho, j);
    const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
    for (int a = 0; a < D; ++a) p.q[a * p.N + cell] = anomaly(p, a, j[a], j[a] * inv_rho);
}

template <int D, int ST, int PAR>
__global__ void __launch_bounds__(kBlock, ELBM_COLLIDE_MIN_BLOCKS) k_collide_range(StepParams p, int begin, int end)
{
    __shared__ unsigned stage[Lat<D>::Q * kBlock];
    const int cell = begin + blockIdx.x * kBlock + threadIdx.x;
    if (cell >= end) return;
    collide_staged<D, ST, PAR>(p, cell, stage + threadIdx.x);
}

// Chunking of the graph-scheduled step: chunks of about 2^18 nodes (a few
// z planes of a large grid, so that L + 1 chunks of populations fit L2), at
// least 3 chunks.
struct GraphGeom {
    int layer, nlayers, chunk_layers, nchunks, lookahead;
};

template <int D>
GraphGeom graph_geometry(const Solver& s)
{
    GraphGeom g{};
    g.layer = (D == 3) ? s.nx * s.ny : s.nx;
    g.nlayers = (D == 3) ? s.nz : s.ny;
    g.chunk_layers = std::max(1, std::min(g.nlayers, (262144 + g.layer - 1) / g.layer));
    g.nchunks = (g.nlayers + g.chunk_layers - 1) / g.chunk_layers;
    g.lookahead = ELBM_GRAPH_LOOKAHEAD;
    return g;
}

template <int D, int ST, int PAR>
cudaError_t build_graph_typed(const Solver& s, cudaGraphExec_t* out, int* nodes)
{
    const GraphGeom g = graph_geometry<D>(s);
    const int K = g.nchunks, chunk_cells = g.chunk_layers * g.layer;
    StepParams p;
    fill_params(s, p);
    p.parity = PAR;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> A(K, nullptr), C(K, nullptr);
    std::vector<int> begin(K), end(K);
    for (int c = 0; c < K; ++c) {
        begin[c] = c * chunk_cells;
        end[c] = std::min((int)s.N, begin[c] + chunk_cells);
    }
    auto add = [&](const void* fn, int c, std::vector<cudaGraphNode_t>& deps, cudaGraphNode_t* node) {
        void* args[] = {&p, &begin[c], &end[c]};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(fn);
        kp.gridDim = dim3((unsigned)((end[c] - begin[c] + kBlock - 1) / kBlock));
        kp.blockDim = dim3(kBlock);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        return cudaGraphAddKernelNode(node, graph, deps.data(), deps.size(), &kp);
    };
    const void* fa = (const void*)k_anomaly_range<D, ST, PAR>;
    const void* fc = (const void*)k_collide_range<D, ST, PAR>;
    // anomaly chain A(K-1), A(0), ..., A(K-2); C(j) as soon as its anomalies exist;
    // A(c) also waits for C(c - L)
    std::vector<int> a_order;
    a_order.push_back(K - 1);
    for (int c = 0; c < K - 1; ++c) a_order.push_back(c);
    std::vector<char> a_done(K, 0), c_done(K, 0);
    cudaGraphNode_t prev_a = nullptr;
    auto try_collides = [&]() -> cudaError_t {
        for (int c = 0; c < K; ++c) {
            if (c_done[c]) continue;
            const int cm = (c + K - 1) % K, cp = (c + 1) % K;
            if (!(a_done[cm] && a_done[c] && a_done[cp])) continue;
            std::vector<cudaGraphNode_t> deps{A[c]};
            if (cm != c) deps.push_back(A[cm]);
            if (cp != c && cp != cm) deps.push_back(A[cp]);
            cudaError_t r = add(fc, c, deps, &C[c]);
            if (r != cudaSuccess) return r;
            c_done[c] = 1;
        }
        return cudaSuccess;
    };
    for (size_t k = 0; k < a_order.size() && e == cudaSuccess; ++k) {
        const int c = a_order[k];
        std::vector<cudaGraphNode_t> deps;
        if (prev_a && ELBM_GRAPH_CHAIN) deps.push_back(prev_a);
        const int lag = c - g.lookahead;
        if (c != K - 1 && lag >= 0 && c_done[lag]) deps.push_back(C[lag]);
        e = add(fa, c, deps, &A[c]);
        if (e != cudaSuccess) break;
        a_done[c] = 1;
        prev_a = A[c];
        e = try_collides();
    }
    if (e == cudaSuccess) e = try_collides();
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    *nodes = 2 * K;
    return e;
}

template <int D>
cudaError_t build_step_graph_impl(const Solver& s, int parity, cudaGraphExec_t* out, int* nodes)
{
    ELBM_DISPATCH_STORAGE(s.storage, {
        return parity == 0 ? build_graph_typed<D, ST, 0>(s, out, nodes) : build_graph_typed<D, ST, 1>(s, out, nodes);
    });
    return cudaErrorInvalidValue;
}

}  // namespace elbm
