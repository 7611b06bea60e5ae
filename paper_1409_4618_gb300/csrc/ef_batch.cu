// Batched assembly: many independent meshes, each to its own CSR, in one
// persistent kernel launch.
//
// Work is a queue of tiles: first every (mesh, element tile) in the batch's
// tile order, then every (mesh, sum tile) in the same mesh order. A CTA takes
// the next tile (dynamic schedule: an integer ticket; static schedule: tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...).
//   - element tile: one thread per element computes its signed local K and M
//     (ef_element.cuh) and writes them to the mesh's contribution list; the
//     CTA then counts the tile done for its mesh (fence + integer atomic).
//   - sum tile: one thread per upper nonzero adds the mesh's contributions in
//     ascending element order (same order and bits as ef_assemble) and writes
//     (r,c) and (c,r) of K and M. Before reading, the CTA waits until its
//     mesh's element tiles are all done. With the dynamic schedule every
//     element tile has been handed to a running CTA before any sum tile is
//     handed out, so the wait ends; it is bounded all the same (poll limit,
//     then a timeout status and the tile is skipped).
// The last CTA to leave resets the ticket and the counters, so the launch
// needs no separate reset and can be replayed from a CUDA graph.
//
// Autotuner (ef_batch_tune): times every candidate schedule (elements per
// tile, uppers per sum tile, CTAs per SM, dynamic or static schedule, mesh
// order as given or largest first) on the bound buffers with CUDA events and
// keeps the fastest.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ef_assemble.cuh"
#include "ef_internal.cuh"

struct ef_batch_mesh {           // device-side descriptor of one mesh
    const int32_t* elems;
    const uint32_t* inv;
    const uint32_t* wseg;        // work-ordered list ranges, CSR positions (see ef_assemble.cu)
    const uint32_t* wpos_up;
    const uint32_t* wpos_lo;
    double* list;                // 2 * np * T contribution values
    const double* nodes;         // bound by ef_batch_bind
    const double* coeff;
    double* K;
    double* M;
    int64_t T, U;
    int64_t etiles;              // element tiles of this mesh
};

struct ef_batch {
    int kind, dim, variant, n;
    std::vector<ef_plan*> plans;
    std::vector<ef_batch_mesh> host_desc;
    ef_batch_mesh* d_desc;
    int64_t* d_eoff;             // n + 1: first element tile of each mesh (in tile order)
    int64_t* d_soff;             // n + 1: first sum tile of each mesh
    int32_t* d_order;            // n: mesh at tile-order position
    uint32_t* d_ctrl;            // [0] ticket, [1] exited, [2..2+n) done counters
    int* d_status;
    int bound;
    ef_batch_config_t cfg;
    int64_t NE, NS;              // tiles of the current configuration
    int sms;
};

namespace ef {
namespace {

constexpr unsigned kPollLimit = 20000000u;   // ~1-2 s of polling with back-off

__device__ __forceinline__ int find_mesh(const int64_t* off, int n, int64_t k)
{
    int lo = 0, hi = n - 1;   // largest i with off[i] <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int VAR, int BE>
__global__ void __launch_bounds__(BE) k_batch(const ef_batch_mesh* __restrict__ md, const int32_t* __restrict__ order,
                                              int n, const int64_t* __restrict__ eoff,
                                              const int64_t* __restrict__ soff, int64_t NE, int64_t NS, int BU,
                                              int dynamic, uint32_t* ctrl, int* status)
{
    using E = ElemTraits<VAR>;
    __shared__ int64_t s_tile;
    uint32_t* ticket = ctrl;
    uint32_t* exited = ctrl + 1;
    uint32_t* done = ctrl + 2;
    int64_t next = blockIdx.x;
    for (;;) {
        if (threadIdx.x == 0) s_tile = dynamic ? (int64_t)atomicAdd(ticket, 1u) : next;
        __syncthreads();
        const int64_t k = s_tile;
        __syncthreads();
        next += gridDim.x;
        if (k >= NE + NS) break;
        if (k < NE) {
            const int pos = find_mesh(eoff, n, k);
            const int m = order[pos];
            const ef_batch_mesh d = md[m];
            const int64_t e = (k - eoff[pos]) * BE + threadIdx.x;
            if (e < d.T) {
                double Kq[E::NP], Mq[E::NP];
                const double sigma = d.coeff ? __ldg(d.coeff + e) : 1.0;
                if (compute_element<VAR>(d.elems, d.nodes, sigma, e, Kq, Mq)) atomicOr(status, ST_DEGENERATE);
                const int64_t nK = (int64_t)E::NP * d.T;
#pragma unroll
                for (int q = 0; q < E::NP; q++) {
                    const uint32_t p = __ldg(d.inv + (int64_t)q * d.T + e);
                    d.list[p] = Kq[q];
                    d.list[nK + p] = Mq[q];
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&done[m], 1u);
            }
        } else {
            const int64_t ks = k - NE;
            const int pos = find_mesh(soff, n, ks);
            const int m = order[pos];
            const ef_batch_mesh d = md[m];
            __shared__ int s_ok;
            if (threadIdx.x == 0) {
                int ok = 1;
                unsigned polls = 0;
                while (atomicAdd(&done[m], 0u) < (uint32_t)d.etiles) {
                    if (++polls > kPollLimit) {
                        ok = 0;
                        atomicOr(status, ST_TIMEOUT);
                        break;
                    }
                    __nanosleep(128);
                }
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) {
                const int64_t u0 = (ks - soff[pos]) * BU;
                const int64_t u1 = u0 + BU < d.U ? u0 + BU : d.U;
                const double* lK = d.list;
                const double* lM = d.list + (int64_t)E::NP * d.T;
                for (int64_t i = u0 + threadIdx.x; i < u1; i += BE) {
                    const uint32_t s0 = d.wseg[i], s1 = d.wseg[i + 1];
                    const uint32_t pu = d.wpos_up[i], pl = d.wpos_lo[i];
                    double kv = __ldcg(lK + s0), mv = __ldcg(lM + s0);
                    for (uint32_t s = s0 + 1; s < s1; s++) {
                        kv += __ldcg(lK + s);
                        mv += __ldcg(lM + s);
                    }
                    d.K[pu] = kv;
                    d.M[pu] = mv;
                    if (pl != 0xffffffffu) {
                        d.K[pl] = kv;
                        d.M[pl] = mv;
                    }
                }
            }
            __syncthreads();
        }
    }
    // the last CTA out resets the queue for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(exited, 1u) == gridDim.x - 1) {
            for (int i = 0; i < n; i++) done[i] = 0;
            *ticket = 0;
            __threadfence();
            *exited = 0;
        }
    }
}

template <int VAR, int BE>
int launch_t(const ef_batch* b, cudaStream_t s)
{
    const int grid = b->cfg.ctas_per_sm * b->sms;
    k_batch<VAR, BE><<<grid, BE, 0, s>>>(b->d_desc, b->d_order, b->n, b->d_eoff, b->d_soff, b->NE, b->NS,
                                          b->cfg.sum_tile, b->cfg.dynamic, b->d_ctrl, b->d_status);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

template <int BE>
int launch_be(const ef_batch* b, cudaStream_t s)
{
    switch (b->variant) {
        case RT2: return launch_t<RT2, BE>(b, s);
        case NED2: return launch_t<NED2, BE>(b, s);
        case RT3: return launch_t<RT3, BE>(b, s);
        default: return launch_t<NED3, BE>(b, s);
    }
}

int max_ctas_per_sm(const ef_batch* b, int BE)
{
    int nb = 0;
    cudaError_t e = cudaSuccess;
    switch (b->variant * 2 + (BE == 256)) {
        case RT2 * 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<RT2, 128>, 128, 0); break;
        case RT2 * 2 + 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<RT2, 256>, 256, 0); break;
        case RT3 * 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<RT3, 128>, 128, 0); break;
        case RT3 * 2 + 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<RT3, 256>, 256, 0); break;
        case NED2 * 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<NED2, 128>, 128, 0); break;
        case NED2 * 2 + 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<NED2, 256>, 256, 0); break;
        case NED3 * 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<NED3, 128>, 128, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<NED3, 256>, 256, 0); break;
    }
    return e == cudaSuccess ? nb : 0;
}

// Tile offsets for the current configuration (tile order and tile sizes).
int apply_config(ef_batch* b, cudaStream_t s)
{
    const int n = b->n, BE = b->cfg.elems_per_tile, BU = b->cfg.sum_tile;
    std::vector<int32_t> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    if (b->cfg.largest_first) {
        // stable: larger meshes first, ties by index
        std::vector<int32_t> tmp(order);
        for (int i = 1; i < n; i++)
            for (int j = i; j > 0 && b->host_desc[order[j]].T > b->host_desc[order[j - 1]].T; j--) {
                int32_t t = order[j];
                order[j] = order[j - 1];
                order[j - 1] = t;
            }
    }
    std::vector<int64_t> eoff(n + 1), soff(n + 1);
    eoff[0] = soff[0] = 0;
    for (int i = 0; i < n; i++) {
        ef_batch_mesh& d = b->host_desc[order[i]];
        d.etiles = (d.T + BE - 1) / BE;
        eoff[i + 1] = eoff[i] + d.etiles;
        soff[i + 1] = soff[i] + (d.U + BU - 1) / BU;
    }
    b->NE = eoff[n];
    b->NS = soff[n];
    if (b->NE + b->NS >= ((int64_t)1 << 32)) return EF_ERR_SIZE;
    EF_CUDA(cudaMemcpyAsync(b->d_desc, b->host_desc.data(), sizeof(ef_batch_mesh) * n, cudaMemcpyHostToDevice, s));
    EF_CUDA(cudaMemcpyAsync(b->d_order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    EF_CUDA(cudaMemcpyAsync(b->d_eoff, eoff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    EF_CUDA(cudaMemcpyAsync(b->d_soff, soff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    EF_CUDA(cudaStreamSynchronize(s));
    return EF_OK;
}

int launch(const ef_batch* b, cudaStream_t s)
{
    if (b->NE + b->NS == 0) return EF_OK;
    return b->cfg.elems_per_tile == 128 ? launch_be<128>(b, s) : launch_be<256>(b, s);
}

void destroy(ef_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    for (ef_plan* p : b->plans)
        if (p) ef_plan_destroy(p);
    void* ptrs[] = {b->d_desc, b->d_eoff, b->d_soff, b->d_order, b->d_ctrl, b->d_status};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete b;
}

}  // namespace
}  // namespace ef

using namespace ef;

extern "C" {

int ef_batch_create(int kind, int dim, int n_meshes, const int64_t* n_nodes, const int64_t* n_elems,
                    const int32_t* const* d_elems, void* stream, ef_batch** out)
{
    if (!out) return EF_ERR_ARG;
    *out = nullptr;
    if (n_meshes <= 0 || !n_nodes || !n_elems || !d_elems) return EF_ERR_ARG;
    if ((kind != EF_RT0 && kind != EF_NED1) || (dim != 2 && dim != 3)) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ef_batch* b = new ef_batch();
    b->kind = kind;
    b->dim = dim;
    b->variant = variant_of(kind, dim);
    b->n = n_meshes;
    b->plans.assign(n_meshes, nullptr);
    b->host_desc.assign(n_meshes, ef_batch_mesh());
    int st = EF_OK;
    for (int m = 0; m < n_meshes && st == EF_OK; m++) {
        st = plan_create_internal(kind, dim, n_nodes[m], n_elems[m], d_elems[m], s,
                                  EF_PLAN_NO_PIPELINE | EF_PLAN_NO_ADJOINT, &b->plans[m]);
        if (st != EF_OK) break;
        const ef_plan* p = b->plans[m];
        ef_batch_mesh& d = b->host_desc[m];
        memset(&d, 0, sizeof(d));
        d.elems = p->d_elems;
        d.inv = p->d_inv;
        d.wseg = p->d_wseg;
        d.wpos_up = p->d_wpos_up;
        d.wpos_lo = p->d_wpos_lo;
        d.list = p->d_local;
        d.T = p->T;
        d.U = p->U;
    }
    if (st == EF_OK) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
        auto ok = [](cudaError_t e) { return e == cudaSuccess; };
        if (!ok(cudaMalloc((void**)&b->d_desc, sizeof(ef_batch_mesh) * n_meshes)) ||
            !ok(cudaMalloc((void**)&b->d_eoff, sizeof(int64_t) * (n_meshes + 1))) ||
            !ok(cudaMalloc((void**)&b->d_soff, sizeof(int64_t) * (n_meshes + 1))) ||
            !ok(cudaMalloc((void**)&b->d_order, sizeof(int32_t) * n_meshes)) ||
            !ok(cudaMalloc((void**)&b->d_ctrl, sizeof(uint32_t) * (n_meshes + 2))) ||
            !ok(cudaMalloc((void**)&b->d_status, sizeof(int))))
            st = EF_ERR_OOM;
    }
    if (st == EF_OK) {
        cudaMemsetAsync(b->d_ctrl, 0, sizeof(uint32_t) * (n_meshes + 2), s);
        cudaMemsetAsync(b->d_status, 0, sizeof(int), s);
        b->cfg.elems_per_tile = 128;
        b->cfg.sum_tile = 1024;
        b->cfg.dynamic = 1;
        b->cfg.largest_first = 0;
        b->cfg.ctas_per_sm = max_ctas_per_sm(b, 128);
        if (b->cfg.ctas_per_sm < 1) st = EF_ERR_CUDA;
    }
    if (st == EF_OK) st = apply_config(b, s);
    if (st != EF_OK) {
        destroy(b);
        return st;
    }
    *out = b;
    return EF_OK;
}

int ef_batch_sizes(const ef_batch* b, int64_t* n_dofs, int64_t* nnz)
{
    if (!b) return EF_ERR_ARG;
    for (int m = 0; m < b->n; m++) {
        if (n_dofs) n_dofs[m] = b->plans[m]->N;
        if (nnz) nnz[m] = b->plans[m]->nnz;
    }
    return EF_OK;
}

int ef_batch_pattern(const ef_batch* b, int mesh, int64_t* d_rowptr, int32_t* d_colidx, void* stream)
{
    if (!b || mesh < 0 || mesh >= b->n) return EF_ERR_ARG;
    return ef_plan_pattern(b->plans[mesh], d_rowptr, d_colidx, stream);
}

int ef_batch_bind(ef_batch* b, const double* const* d_nodes, const double* const* d_coeff, double* const* d_K,
                  double* const* d_M, void* stream)
{
    if (!b || !d_nodes || !d_K || !d_M) return EF_ERR_ARG;
    for (int m = 0; m < b->n; m++) {
        if (b->host_desc[m].T > 0 && (!d_nodes[m] || !d_K[m] || !d_M[m])) return EF_ERR_ARG;
        b->host_desc[m].nodes = d_nodes[m];
        b->host_desc[m].coeff = d_coeff ? d_coeff[m] : nullptr;
        b->host_desc[m].K = d_K[m];
        b->host_desc[m].M = d_M[m];
    }
    EF_TRY(apply_config(b, (cudaStream_t)stream));
    b->bound = 1;
    return EF_OK;
}

int ef_batch_assemble(const ef_batch* b, void* stream)
{
    if (!b || !b->bound) return EF_ERR_ARG;
    return launch(b, (cudaStream_t)stream);
}

int ef_batch_get_config(const ef_batch* b, ef_batch_config_t* cfg)
{
    if (!b || !cfg) return EF_ERR_ARG;
    *cfg = b->cfg;
    return EF_OK;
}

int ef_batch_set_config(ef_batch* b, const ef_batch_config_t* cfg, void* stream)
{
    if (!b || !cfg) return EF_ERR_ARG;
    if (cfg->elems_per_tile != 128 && cfg->elems_per_tile != 256) return EF_ERR_ARG;
    if (cfg->sum_tile < cfg->elems_per_tile || cfg->sum_tile > (1 << 20)) return EF_ERR_ARG;
    const int maxc = max_ctas_per_sm(b, cfg->elems_per_tile);
    if (cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > maxc) return EF_ERR_ARG;
    b->cfg = *cfg;
    return apply_config(b, (cudaStream_t)stream);
}

int ef_batch_tune(ef_batch* b, int reps, ef_batch_config_t* best_out, void* stream)
{
    if (!b || !b->bound) return EF_ERR_ARG;
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    EF_CUDA(cudaEventCreate(&e0));
    EF_CUDA(cudaEventCreate(&e1));
    ef_batch_config_t best = b->cfg;
    float best_ms = 1e30f;
    const int tiles[2] = {128, 256};
    const int sums[3] = {512, 2048, 8192};
    int st = EF_OK;
    for (int ti = 0; ti < 2 && st == EF_OK; ti++) {
        const int maxc = max_ctas_per_sm(b, tiles[ti]);
        for (int su = 0; su < 3 && st == EF_OK; su++)
            for (int dyn = 0; dyn < 2 && st == EF_OK; dyn++)
                for (int lf = 0; lf < 2 && st == EF_OK; lf++)
                    for (int occ = 0; occ < 2 && st == EF_OK; occ++) {
                        ef_batch_config_t c;
                        c.elems_per_tile = tiles[ti];
                        c.sum_tile = sums[su] < tiles[ti] ? tiles[ti] : sums[su];
                        c.dynamic = dyn;
                        c.largest_first = lf;
                        c.ctas_per_sm = occ == 0 ? maxc : (maxc + 1) / 2;
                        if (c.ctas_per_sm < 1) continue;
                        b->cfg = c;
                        if ((st = apply_config(b, s)) != EF_OK) break;
                        if ((st = launch(b, s)) != EF_OK) break;   // warm-up
                        cudaEventRecord(e0, s);
                        for (int r = 0; r < reps && st == EF_OK; r++) st = launch(b, s);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) {
                            st = EF_ERR_CUDA;
                            break;
                        }
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        ms /= reps;
                        if (ms < best_ms) {
                            best_ms = ms;
                            best = c;
                        }
                    }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != EF_OK) return st;
    b->cfg = best;
    EF_TRY(apply_config(b, s));
    if (best_out) *best_out = best;
    return ef_batch_check(b, stream);
}

int ef_batch_check(ef_batch* b, void* stream)
{
    if (!b) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    EF_CUDA(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    if (st) EF_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int), s));
    if (st & ST_TIMEOUT) return EF_ERR_TIMEOUT;
    if (st & ST_DEGENERATE) return EF_ERR_DEGENERATE;
    return EF_OK;
}

void ef_batch_destroy(ef_batch* b) { destroy(b); }

}  // extern "C"
