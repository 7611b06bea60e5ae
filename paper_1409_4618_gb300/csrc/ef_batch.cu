// Batched assembly: many independent meshes, each to its own CSR, in one
// persistent kernel launch: the interleaved queue of ef_queue.cu over all
// meshes (element tiles of mesh m+1 run while the sums of mesh m are formed).
// Values are those of ef_assemble on each mesh, bit for bit.
//
// Autotuner (ef_batch_tune): times every candidate schedule (elements per
// tile, nonzeros per sum tile, one interleaved queue or element/sum role
// split, dynamic or static schedule, mesh order as given or largest first) on
// the bound buffers with CUDA events and keeps the fastest.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ef_internal.cuh"
#include "ef_queue.cuh"

struct ef_batch {
    int kind, dim, variant, n;
    std::vector<ef_plan*> plans;
    ef::Queue queue;
    int bound;
};

namespace ef {
namespace {

void destroy(ef_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    for (ef_plan* p : b->plans)
        if (p) ef_plan_destroy(p);
    queue_free(&b->queue);
    delete b;
}

// Per-call buffers of ef_batch_assemble: the four pointer tables of up to
// BIND_CHUNK meshes travel as one kernel's parameters (2 KiB, inside the
// classic 4 KiB limit) and are written into the device descriptors on the
// call's stream, so the call needs no host synchronisation, no allocation
// and no copy from host memory, and a captured call keeps the tables it was
// captured with.
constexpr int BIND_CHUNK = 64;
struct BindChunk {
    int first, count;
    const double* nodes[BIND_CHUNK];
    const double* coeff[BIND_CHUNK];
    double* K[BIND_CHUNK];
    double* M[BIND_CHUNK];
};

__global__ void k_bind_tables(QueueMesh* __restrict__ md, const BindChunk c)
{
    const int i = threadIdx.x;
    if (i >= c.count) return;
    QueueMesh& d = md[c.first + i];
    d.nodes = c.nodes[i];
    d.coeff = c.coeff[i];
    d.K = c.K[i];
    d.M = c.M[i];
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
    b->bound = 0;
    b->plans.assign(n_meshes, nullptr);
    int st = EF_OK;
    for (int m = 0; m < n_meshes && st == EF_OK; m++)
        st = plan_create_internal(kind, dim, n_nodes[m], n_elems[m], d_elems[m], s,
                                  EF_PLAN_NO_PIPELINE | EF_PLAN_NO_ADJOINT, &b->plans[m]);
    if (st == EF_OK) st = queue_init(&b->queue, b->variant, nullptr);
    if (st == EF_OK) {
        b->queue.cfg.elems_per_tile = 128;
        b->queue.cfg.sum_tile = 2048;
        b->queue.cfg.elem_ctas = 0;
        b->queue.cfg.two_launch = 1;
        b->queue.cfg.ctas_per_sm = queue_max_ctas_per_sm(b->variant, 128);
        if (b->queue.cfg.ctas_per_sm < 1) st = EF_ERR_CUDA;
    }
    if (st == EF_OK) st = queue_set_meshes(&b->queue, b->plans, s);
    if (st == EF_OK) st = queue_build(&b->queue, b->plans, s);
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
    for (int m = 0; m < b->n; m++)
        if (b->plans[m]->T > 0 && (!d_nodes[m] || !d_K[m] || !d_M[m])) return EF_ERR_ARG;
    for (int m = 0; m < b->n; m++) {
        QueueMesh& d = b->queue.host_mesh[m];
        d.nodes = d_nodes[m];
        d.coeff = d_coeff ? d_coeff[m] : nullptr;
        d.K = d_K[m];
        d.M = d_M[m];
    }
    EF_TRY(queue_set_meshes(&b->queue, b->plans, (cudaStream_t)stream));
    b->bound = 1;
    return EF_OK;
}

int ef_batch_assemble_bound(const ef_batch* b, void* stream)
{
    if (!b || !b->bound) return EF_ERR_ARG;
    return queue_launch(&b->queue, QueueArgs(), (cudaStream_t)stream);
}

int ef_batch_plan_create(int kind, int dim, int n_meshes, const int64_t* n_nodes, const int64_t* n_elems,
                         const int32_t* const* d_elems, void* stream, ef_batch_plan** out)
{
    return ef_batch_create(kind, dim, n_meshes, n_nodes, n_elems, d_elems, stream, out);
}

int ef_batch_assemble(const ef_batch_plan* b, const double* const* d_nodes, const double* const* d_coeff,
                      double* const* d_Kval, double* const* d_Mval, void* stream)
{
    if (!b || !d_nodes || !d_Kval || !d_Mval) return EF_ERR_ARG;
    for (int m = 0; m < b->n; m++)
        if (b->plans[m]->T > 0 && (!d_nodes[m] || !d_Kval[m] || !d_Mval[m])) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int m0 = 0; m0 < b->n; m0 += BIND_CHUNK) {
        BindChunk c;
        memset(&c, 0, sizeof(c));
        c.first = m0;
        c.count = b->n - m0 < BIND_CHUNK ? b->n - m0 : BIND_CHUNK;
        for (int i = 0; i < c.count; i++) {
            c.nodes[i] = d_nodes[m0 + i];
            c.coeff[i] = d_coeff ? d_coeff[m0 + i] : nullptr;
            c.K[i] = d_Kval[m0 + i];
            c.M[i] = d_Mval[m0 + i];
        }
        k_bind_tables<<<1, BIND_CHUNK, 0, s>>>(b->queue.d_mesh, c);
    }
    EF_CUDA(cudaGetLastError());
    return queue_launch(&b->queue, QueueArgs(), s);
}

void ef_batch_plan_destroy(ef_batch_plan* b) { destroy(b); }

int ef_batch_get_config(const ef_batch* b, ef_batch_config_t* cfg)
{
    if (!b || !cfg) return EF_ERR_ARG;
    *cfg = b->queue.cfg;
    return EF_OK;
}

int ef_batch_set_config(ef_batch* b, const ef_batch_config_t* cfg, void* stream)
{
    if (!b || !cfg) return EF_ERR_ARG;
    if (cfg->elems_per_tile != 128 && cfg->elems_per_tile != 256) return EF_ERR_ARG;
    if (cfg->elem_ctas < 0 || cfg->elem_ctas > 3) return EF_ERR_ARG;
    if (cfg->two_launch != 0 && cfg->two_launch != 1) return EF_ERR_ARG;
    if (cfg->sum_tile < cfg->elems_per_tile || cfg->sum_tile > (1 << 20)) return EF_ERR_ARG;
    const int maxc = queue_max_ctas_per_sm(b->variant, cfg->elems_per_tile);
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > maxc) return EF_ERR_ARG;
    b->queue.cfg = *cfg;
    if (cfg->ctas_per_sm == 0) b->queue.cfg.ctas_per_sm = maxc;   // 0: as many as fit
    return queue_build(&b->queue, b->plans, (cudaStream_t)stream);
}

int ef_batch_tune(ef_batch* b, int reps, ef_batch_config_t* best_out, void* stream)
{
    if (!b || !b->bound) return EF_ERR_ARG;
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    EF_CUDA(cudaEventCreate(&e0));
    EF_CUDA(cudaEventCreate(&e1));
    ef_batch_config_t best = b->queue.cfg;
    float best_ms = 1e30f;
    const int tiles[2] = {128, 256};
    const int sums[2] = {512, 2048};
    int st = EF_OK;
    auto time_config = [&](const ef_batch_config_t& c) {
        b->queue.cfg = c;
        if ((st = queue_build(&b->queue, b->plans, s)) != EF_OK) return;
        if ((st = queue_launch(&b->queue, QueueArgs(), s)) != EF_OK) return;   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == EF_OK; r++) st = queue_launch(&b->queue, QueueArgs(), s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = EF_ERR_CUDA;
            return;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    {
        ef_batch_config_t c = b->queue.cfg;
        c.two_launch = 1;
        time_config(c);
    }
    for (int ti = 0; ti < 2 && st == EF_OK; ti++) {
        const int maxc = queue_max_ctas_per_sm(b->variant, tiles[ti]);
        for (int su = 0; su < 2 && st == EF_OK; su++)
            for (int ec = 0; ec < 3 && st == EF_OK; ec++)
                for (int lf = 0; lf < 2 && st == EF_OK; lf++)
                    for (int dyn = (ec ? 1 : 0); dyn < 2 && st == EF_OK; dyn++) {
                        ef_batch_config_t c;
                        c.elems_per_tile = tiles[ti];
                        c.sum_tile = sums[su] < tiles[ti] ? tiles[ti] : sums[su];
                        c.dynamic = dyn;
                        c.largest_first = lf;
                        c.elem_ctas = ec;
                        c.two_launch = 0;
                        c.ctas_per_sm = maxc;
                        if (c.ctas_per_sm < 1) continue;
                        time_config(c);
                    }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != EF_OK) return st;
    b->queue.cfg = best;
    EF_TRY(queue_build(&b->queue, b->plans, s));
    if (best_out) *best_out = best;
    return ef_batch_check(b, stream);
}

int ef_batch_check(ef_batch* b, void* stream)
{
    if (!b) return EF_ERR_ARG;
    return queue_check(&b->queue, (cudaStream_t)stream);
}

void ef_batch_destroy(ef_batch* b) { destroy(b); }

}  // extern "C"
