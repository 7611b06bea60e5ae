// C ABI entry points of libedgefem (declared in include/edgefem.h).
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ef_internal.cuh"
#include "ef_queue.cuh"

using namespace ef;

namespace {

void free_plan_memory(ef_plan* p)
{
    release_fused(p);
    void* ptrs[] = {p->d_elems,     p->d_elem2dof,   p->d_signbits,  p->d_dof2nodes,   p->d_rowptr,
                    p->d_colidx,    p->d_seg,        p->d_perm,      p->d_pos_up,      p->d_pos_lo,
                    p->d_local,     p->d_status,
                    p->d_stage_nodes, p->d_stage_coeff, p->d_stage_K, p->d_stage_M,
                    p->d_node_off,  p->d_node_inc,   p->d_adj_part,  p->d_adj_jpart, p->d_l2_part,
                    p->d_dof_off,   p->d_dof_inc,    p->d_load_local};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (cudaEvent_t e : p->copy_ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
}

int plan_args(int kind, int dim, int64_t n_nodes, int64_t n_elems, const void* d_elems)
{
    if ((kind != EF_RT0 && kind != EF_NED1) || (dim != 2 && dim != 3)) return EF_ERR_ARG;
    if (n_nodes < 0 || n_elems < 0 || (n_elems > 0 && !d_elems)) return EF_ERR_ARG;
    if (n_nodes > (int64_t)INT32_MAX) return EF_ERR_SIZE;
    const int v = variant_of(kind, dim);
    const int64_t lim = (int64_t)1 << 32;
    if (n_elems >= lim / npair_of(v)) return EF_ERR_SIZE;
    if (v == RT3 && n_nodes > 2642245) return EF_ERR_KEY_OVERFLOW;  // 2642245^3 < 2^64
    return EF_OK;
}

int create(int kind, int dim, int64_t n_nodes, int64_t n_elems, const int32_t* d_elems, cudaStream_t s, int flags,
           ef_plan** out)
{
    ef_plan* p = (ef_plan*)calloc(1, sizeof(ef_plan));
    if (!p) return EF_ERR_OOM;
    p->flags = flags;
    p->kind = kind;
    p->dim = dim;
    p->variant = variant_of(kind, dim);
    p->nv = dim + 1;
    p->nl = nloc_of(p->variant);
    p->np = npair_of(p->variant);
    p->ent = ent_nodes_of(p->variant);
    p->V = n_nodes;
    p->T = n_elems;
    int st = EF_OK;
    do {
        cudaError_t e = cudaMalloc((void**)&p->d_status, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_elems, (size_t)(n_elems > 0 ? n_elems : 1) * p->nv * 4);
        if (e != cudaSuccess) {
            set_last_error("cudaMalloc", e);
            st = e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
            break;
        }
        e = cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
        if (e == cudaSuccess && n_elems > 0)
            e = cudaMemcpyAsync(p->d_elems, d_elems, (size_t)n_elems * p->nv * 4, cudaMemcpyDefault, s);
        if (e != cudaSuccess) {
            set_last_error("cudaMemcpyAsync(elems)", e);
            st = EF_ERR_CUDA;
            break;
        }
        if ((st = validate_elems(p, s)) != EF_OK) break;
        if ((st = build_topology(p, s)) != EF_OK) break;
        if ((st = build_pattern(p, s)) != EF_OK) break;
        e = cudaMalloc((void**)&p->d_local, (size_t)(p->T > 0 ? p->T : 1) * p->np * 2 * sizeof(double));
        if (e != cudaSuccess) {
            set_last_error("cudaMalloc(local)", e);
            st = EF_ERR_OOM;
            break;
        }
        if ((st = build_work_order(p, default_pipeline_chunks(p), s)) != EF_OK) break;
        if (!(flags & EF_PLAN_NO_PIPELINE) && (st = plan_queue_rebuild(p, s)) != EF_OK) break;
        if (!(flags & EF_PLAN_NO_ADJOINT) && (st = build_adjoint(p, s)) != EF_OK) break;
        p->use_two_pass = 1;   // the fastest schedule until ef_plan_tune / ef_plan_set_pipeline picks another
    } while (0);
    if (st != EF_OK) {
        cudaStreamSynchronize(s);
        plan_queue_free(p);
        release_work_order(p);
        free_plan_memory(p);
        free(p);
        return st;
    }
    *out = p;
    return EF_OK;
}

int assemble_checks(const ef_plan* plan, const double* nodes, double* K, double* M)
{
    if (!plan) return EF_ERR_ARG;
    if (plan->T > 0 && (!nodes || !K || !M)) return EF_ERR_ARG;
    return EF_OK;
}

int one_shot(int kind, int dim, const double* d_nodes, int64_t n_nodes, const int32_t* d_elems, int64_t n_elems,
             const double* d_coeff, ef_csr* out, void* stream)
{
    if (!out) return EF_ERR_ARG;
    memset(out, 0, sizeof(*out));
    if (n_elems > 0 && !d_nodes) return EF_ERR_ARG;
    ef_plan* p = nullptr;
    int st = plan_args(kind, dim, n_nodes, n_elems, d_elems);
    if (st == EF_OK)
        st = create(kind, dim, n_nodes, n_elems, d_elems, (cudaStream_t)stream,
                    EF_PLAN_NO_PIPELINE | EF_PLAN_NO_ADJOINT, &p);
    if (st != EF_OK) return st;
    ef_csr c;
    memset(&c, 0, sizeof(c));
    c.n_dofs = p->N;
    c.nnz = p->nnz;
    cudaError_t e = cudaMalloc((void**)&c.d_rowptr, (size_t)(p->N + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.d_colidx, (size_t)(p->nnz > 0 ? p->nnz : 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.d_K, (size_t)(p->nnz > 0 ? p->nnz : 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.d_M, (size_t)(p->nnz > 0 ? p->nnz : 1) * 8);
    if (e != cudaSuccess) {
        set_last_error("cudaMalloc(csr)", e);
        st = EF_ERR_OOM;
    }
    if (st == EF_OK) st = ef_plan_pattern(p, c.d_rowptr, c.d_colidx, stream);
    if (st == EF_OK) st = ef_assemble(p, d_nodes, d_coeff, c.d_K, c.d_M, stream);
    if (st == EF_OK) st = ef_plan_check(p, stream);
    ef_plan_destroy(p);
    if (st != EF_OK) {
        ef_csr_free(&c);
        return st;
    }
    *out = c;
    return EF_OK;
}

}  // namespace

namespace ef {

// CUDA events of ef_plan_profile: three per recorded ef_assemble call.
struct Profile {
    std::vector<cudaEvent_t> ev;
    std::vector<char> two;   // per call: a second kernel ran between the middle and last events
    int cap = 0, calls = 0;
    bool mid = false;
};

void profile_begin(const ef_plan* p, cudaStream_t s)
{
    Profile* pr = p->prof;
    if (!pr || pr->calls >= pr->cap) return;
    cudaEventRecord(pr->ev[(size_t)3 * pr->calls], s);
    pr->mid = false;
}

void profile_mid(const ef_plan* p, cudaStream_t s)
{
    Profile* pr = p->prof;
    if (!pr || pr->calls >= pr->cap) return;
    cudaEventRecord(pr->ev[(size_t)3 * pr->calls + 1], s);
    pr->mid = true;
}

void profile_end(const ef_plan* p, cudaStream_t s)
{
    Profile* pr = p->prof;
    if (!pr || pr->calls >= pr->cap) return;
    cudaEvent_t* e = &pr->ev[(size_t)3 * pr->calls];
    if (!pr->mid) cudaEventRecord(e[1], s);   // one-kernel paths: all time is the first kernel's
    cudaEventRecord(e[2], s);
    pr->two[pr->calls] = pr->mid ? 1 : 0;
    pr->calls++;
}

void profile_free(ef_plan* p)
{
    if (!p->prof) return;
    for (cudaEvent_t e : p->prof->ev)
        if (e) cudaEventDestroy(e);
    delete p->prof;
    p->prof = nullptr;
}

int plan_create_internal(int kind, int dim, int64_t n_nodes, int64_t n_elems, const int32_t* d_elems, cudaStream_t s,
                         int flags, ef_plan** out)
{
    if (!out) return EF_ERR_ARG;
    *out = nullptr;
    int st = plan_args(kind, dim, n_nodes, n_elems, d_elems);
    if (st != EF_OK) return st;
    return create(kind, dim, n_nodes, n_elems, d_elems, s, flags, out);
}
}  // namespace ef

extern "C" {

int ef_plan_create(int kind, int dim, int64_t n_nodes, int64_t n_elems, const int32_t* d_elems, void* stream,
                   ef_plan** out)
{
    if (!out) return EF_ERR_ARG;
    *out = nullptr;
    int st = plan_args(kind, dim, n_nodes, n_elems, d_elems);
    if (st != EF_OK) return st;
    return create(kind, dim, n_nodes, n_elems, d_elems, (cudaStream_t)stream, 0, out);
}

int ef_plan_sizes(const ef_plan* plan, int64_t* n_dofs, int64_t* nnz)
{
    if (!plan) return EF_ERR_ARG;
    if (n_dofs) *n_dofs = plan->N;
    if (nnz) *nnz = plan->nnz;
    return EF_OK;
}

int ef_plan_info(const ef_plan* plan, ef_plan_info_t* info)
{
    if (!plan || !info) return EF_ERR_ARG;
    memset(info, 0, sizeof(*info));
    info->n_dofs = plan->N;
    info->nnz = plan->nnz;
    info->n_upper = plan->U;
    info->n_contrib = plan->T * plan->np;
    if (plan->T == 0)
        info->assemble_launches = 0;
    else if (plan->use_blocked && plan->fb_nblocks > 0)
        info->assemble_launches = 1;
    else
        info->assemble_launches = (plan->queue && !plan->use_two_pass) ? 1 : 2;
    info->fused_block = plan->use_blocked ? plan->fb_block : 0;
    info->pipeline_chunks = plan->pc_chunks;
    info->fused_blocks = plan->fb_nblocks;
    info->fused_partial = plan->n_partial;
    info->fused_sfc = plan->use_blocked ? plan->fb_sfc : 0;
    return EF_OK;
}

int ef_plan_set_block(ef_plan* plan, int block, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    if (block == 0) {
        plan->use_blocked = 0;
        return EF_OK;
    }
    if (!fused_block_supported(block)) return EF_ERR_ARG;
    EF_TRY(build_fused_block(plan, block, nullptr, (cudaStream_t)stream));
    plan->use_blocked = 1;
    plan->use_two_pass = 0;
    return EF_OK;
}

int ef_plan_set_fused(ef_plan* plan, const double* d_nodes, int block, void* stream)
{
    if (!plan || (plan->T > 0 && !d_nodes)) return EF_ERR_ARG;
    if (block == 0) {
        plan->use_blocked = 0;
        return EF_OK;
    }
    if (!fused_block_supported(block)) return EF_ERR_ARG;
    EF_TRY(build_fused_block(plan, block, d_nodes, (cudaStream_t)stream));
    plan->use_blocked = 1;
    plan->use_two_pass = 0;
    return EF_OK;
}

int ef_plan_set_pipeline(ef_plan* plan, int chunks, void* stream)
{
    if (!plan || chunks < 1 || chunks > EF_MAX_CHUNKS) return EF_ERR_ARG;
    if (plan->flags & EF_PLAN_NO_PIPELINE) return EF_ERR_ARG;
    EF_TRY(build_work_order(plan, chunks, (cudaStream_t)stream));
    EF_TRY(plan_queue_rebuild(plan, (cudaStream_t)stream));
    plan->use_blocked = 0;
    plan->use_two_pass = 0;
    return EF_OK;
}

int ef_plan_inject_stall(ef_plan* plan, int on, void* stream)
{
    if (!plan || !plan->queue) return EF_ERR_ARG;
    if (on && (plan->use_two_pass || plan->use_blocked)) return EF_ERR_ARG;
    return queue_inject_stall(plan->queue, on, (cudaStream_t)stream);
}

int ef_plan_tune(ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval, double* d_Mval,
                 int reps, int* chosen, void* stream)
{
    EF_TRY(assemble_checks(plan, d_nodes, d_Kval, d_Mval));
    if (plan->flags & EF_PLAN_NO_PIPELINE) return EF_ERR_ARG;
    if (reps < 1) reps = 5;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    EF_CUDA(cudaEventCreate(&e0));
    EF_CUDA(cudaEventCreate(&e1));
    struct Cand {
        int chunks, block, two_pass;   // block > 0: element-block path; two_pass: plain kernels
        int sfc;                       // element-block path along the Morton order of the centroids
        ef_batch_config_t q;
    };
    std::vector<Cand> cands;
    {
        Cand k{};
        k.two_pass = 1;
        k.chunks = default_pipeline_chunks(plan);
        cands.push_back(k);
    }
    const int chunk_opts[] = {4, 8, 16};
    for (int c : chunk_opts) {
        if (c > 1 && plan->T / c < 8192) continue;
        for (int be : {128, 256})
            for (int bu : {1024, 4096})
                for (int ec : {0, 1, 2}) {
                    Cand k{};
                    k.chunks = c;
                    k.q.elems_per_tile = be;
                    k.q.sum_tile = bu;
                    k.q.dynamic = 1;
                    k.q.largest_first = 0;
                    k.q.elem_ctas = ec;
                    k.q.ctas_per_sm = queue_max_ctas_per_sm(plan->variant, be);
                    if (k.q.ctas_per_sm >= 1) cands.push_back(k);
                }
    }
    for (int sfc : {0, 1})
        for (int b : {128, 256}) {
            Cand k{};
            k.block = b;
            k.sfc = sfc;
            cands.push_back(k);
        }
    int st = EF_OK, best = -1;
    float best_ms = 1e30f;
    for (size_t i = 0; i < cands.size() && st == EF_OK; i++) {
        const Cand& c = cands[i];
        if (c.block > 0)
            st = c.sfc ? ef_plan_set_fused(plan, d_nodes, c.block, stream) : ef_plan_set_block(plan, c.block, stream);
        else if (c.two_pass) {
            // the two-pass kernels do not depend on the chunking; keep the
            // default one, which ef_assemble_host overlaps with its copies
            if (plan->pc_chunks != c.chunks) st = ef_plan_set_pipeline(plan, c.chunks, stream);
            plan->use_blocked = 0;
            plan->use_two_pass = 1;
        } else {
            if (plan->pc_chunks != c.chunks) st = ef_plan_set_pipeline(plan, c.chunks, stream);
            plan->use_blocked = 0;
            plan->use_two_pass = 0;
            if (st == EF_OK) st = plan_queue_config(plan, c.q, s);
        }
        if (st == EF_ERR_OOM || st == EF_ERR_SIZE) {   // a schedule that does not fit: skip it
            cudaGetLastError();
            st = EF_OK;
            continue;
        }
        if (st != EF_OK) break;
        if ((st = ef_assemble(plan, d_nodes, d_coeff, d_Kval, d_Mval, stream)) != EF_OK) break;
        // one timed call sets how many to time: at least `reps`, and enough for
        // about 2 ms, so that calls of a few microseconds are not timed by noise
        cudaEventRecord(e0, s);
        st = ef_assemble(plan, d_nodes, d_coeff, d_Kval, d_Mval, stream);
        cudaEventRecord(e1, s);
        float one = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&one, e0, e1) != cudaSuccess) {
            st = EF_ERR_CUDA;
            break;
        }
        int n = reps;
        if (one > 0 && one * n < 2.0f) n = (int)(2.0f / one) + 1;
        if (n > 1000) n = 1000;
        cudaEventRecord(e0, s);
        for (int r = 0; r < n && st == EF_OK; r++) st = ef_assemble(plan, d_nodes, d_coeff, d_Kval, d_Mval, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = EF_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= n;
        if (ms < best_ms) {
            best_ms = ms;
            best = (int)i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != EF_OK || best < 0) return st != EF_OK ? st : EF_ERR_ARG;
    const Cand& c = cands[best];
    if (c.block > 0) {
        st = c.sfc ? ef_plan_set_fused(plan, d_nodes, c.block, stream) : ef_plan_set_block(plan, c.block, stream);
        if (chosen) *chosen = c.sfc ? -(c.block + 1) : -c.block;
    } else if (c.two_pass) {
        st = ef_plan_set_pipeline(plan, c.chunks, stream);
        plan->use_two_pass = 1;
        if (chosen) *chosen = 0;
    } else {
        st = ef_plan_set_pipeline(plan, c.chunks, stream);
        plan->use_blocked = 0;
        if (st == EF_OK) st = plan_queue_config(plan, c.q, s);
        if (chosen) *chosen = c.chunks * 100 + c.q.elem_ctas * 10 + (c.q.elems_per_tile == 256);
    }
    return st == EF_OK ? ef_plan_check(plan, stream) : st;
}

int ef_plan_pattern(const ef_plan* plan, int64_t* d_rowptr, int32_t* d_colidx, void* stream)
{
    if (!plan || !d_rowptr || (plan->nnz > 0 && !d_colidx)) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    EF_CUDA(cudaMemcpyAsync(d_rowptr, plan->d_rowptr, (size_t)(plan->N + 1) * 8, cudaMemcpyDeviceToDevice, s));
    if (plan->nnz > 0)
        EF_CUDA(cudaMemcpyAsync(d_colidx, plan->d_colidx, (size_t)plan->nnz * 4, cudaMemcpyDeviceToDevice, s));
    return EF_OK;
}

int ef_plan_topology(const ef_plan* plan, int32_t* d_elem2dof, uint8_t* d_signbits, int32_t* d_dof2nodes,
                     void* stream)
{
    if (!plan) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_elem2dof && plan->T > 0)
        EF_CUDA(cudaMemcpyAsync(d_elem2dof, plan->d_elem2dof, (size_t)plan->T * plan->nl * 4, cudaMemcpyDeviceToDevice, s));
    if (d_signbits && plan->T > 0)
        EF_CUDA(cudaMemcpyAsync(d_signbits, plan->d_signbits, (size_t)plan->T, cudaMemcpyDeviceToDevice, s));
    if (d_dof2nodes && plan->N > 0)
        EF_CUDA(cudaMemcpyAsync(d_dof2nodes, plan->d_dof2nodes, (size_t)plan->N * plan->ent * 4,
                                cudaMemcpyDeviceToDevice, s));
    return EF_OK;
}

int ef_assemble_two_pass(const ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval,
                         double* d_Mval, void* stream)
{
    EF_TRY(assemble_checks(plan, d_nodes, d_Kval, d_Mval));
    return launch_two_pass(plan, d_nodes, d_coeff, d_Kval, d_Mval, (cudaStream_t)stream);
}

int ef_assemble(const ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval, double* d_Mval,
                void* stream)
{
    EF_TRY(assemble_checks(plan, d_nodes, d_Kval, d_Mval));
    if (plan->T == 0) return EF_OK;   // no elements: no nonzeros either
    cudaStream_t s = (cudaStream_t)stream;
    profile_begin(plan, s);
    int st;
    if (plan->use_blocked && plan->fb_nblocks > 0)
        st = launch_fused(plan, d_nodes, d_coeff, d_Kval, d_Mval, s);
    else if (!plan->queue || plan->use_two_pass)
        st = launch_two_pass(plan, d_nodes, d_coeff, d_Kval, d_Mval, s);
    else
        st = launch_queue(plan, d_nodes, d_coeff, d_Kval, d_Mval, s);
    profile_end(plan, s);
    return st;
}

int ef_assemble2(const ef_plan* plan, const double* d_nodes, const double* d_coeff_K, const double* d_coeff_M,
                 double* d_Kval, double* d_Mval, void* stream)
{
    EF_TRY(assemble_checks(plan, d_nodes, d_Kval, d_Mval));
    cudaStream_t s = (cudaStream_t)stream;
    profile_begin(plan, s);
    const int st = launch_two_pass2(plan, d_nodes, d_coeff_K, d_coeff_M, d_Kval, d_Mval, s);
    profile_end(plan, s);
    return st;
}

int ef_plan_profile(ef_plan* plan, int max_calls)
{
    if (!plan || max_calls < 0) return EF_ERR_ARG;
    profile_free(plan);
    if (max_calls == 0) return EF_OK;
    Profile* pr = new Profile();
    pr->cap = max_calls;
    pr->ev.assign((size_t)3 * max_calls, nullptr);
    pr->two.assign((size_t)max_calls, 0);
    for (cudaEvent_t& e : pr->ev) {
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) {
            set_last_error("cudaEventCreate", r);
            plan->prof = pr;
            profile_free(plan);
            return EF_ERR_CUDA;
        }
    }
    plan->prof = pr;
    return EF_OK;
}

int ef_plan_profile_read(const ef_plan* plan, double* ms_first, double* ms_second, int* calls)
{
    if (!plan) return EF_ERR_ARG;
    double a = 0, b = 0;
    int n = 0;
    if (plan->prof) {
        Profile* pr = plan->prof;
        n = pr->calls;
        for (int c = 0; c < n; c++) {
            cudaEvent_t* e = &pr->ev[(size_t)3 * c];
            EF_CUDA(cudaEventSynchronize(e[2]));
            float x = 0, y = 0;
            EF_CUDA(cudaEventElapsedTime(&x, e[0], e[1]));
            if (pr->two[c]) EF_CUDA(cudaEventElapsedTime(&y, e[1], e[2]));
            a += x;
            b += y;
        }
    }
    if (ms_first) *ms_first = a;
    if (ms_second) *ms_second = b;
    if (calls) *calls = n;
    return EF_OK;
}

int ef_assemble_host(ef_plan* plan, const double* h_nodes, const double* h_coeff, double* h_Kval, double* h_Mval,
                     void* stream)
{
    if (!plan) return EF_ERR_ARG;
    if (plan->T > 0 && (!h_nodes || !h_Kval || !h_Mval)) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)(plan->V > 0 ? plan->V : 1) * plan->dim * 8;
    const size_t cb = (size_t)(plan->T > 0 ? plan->T : 1) * 8;
    const size_t vb = (size_t)(plan->nnz > 0 ? plan->nnz : 1) * 8;
    if (!plan->d_stage_nodes) {
        EF_CUDA(cudaMalloc((void**)&plan->d_stage_nodes, nb));
        EF_CUDA(cudaMalloc((void**)&plan->d_stage_coeff, cb));
        EF_CUDA(cudaMalloc((void**)&plan->d_stage_K, vb));
        EF_CUDA(cudaMalloc((void**)&plan->d_stage_M, vb));
    }
    if (plan->V > 0 && h_nodes)
        EF_CUDA(cudaMemcpyAsync(plan->d_stage_nodes, h_nodes, (size_t)plan->V * plan->dim * 8, cudaMemcpyHostToDevice, s));
    if (h_coeff && plan->T > 0)
        EF_CUDA(cudaMemcpyAsync(plan->d_stage_coeff, h_coeff, (size_t)plan->T * 8, cudaMemcpyHostToDevice, s));
    const double* dn = plan->d_stage_nodes;
    const double* dc = h_coeff ? plan->d_stage_coeff : nullptr;
    double *dK = plan->d_stage_K, *dM = plan->d_stage_M;
    const bool chunked = plan->T > 0 && plan->pc_chunks > 1 && !(plan->use_blocked && plan->fb_nblocks > 0);
    if (!chunked) {
        EF_TRY(ef_assemble(plan, dn, dc, dK, dM, stream));
        if (plan->nnz > 0) {
            EF_CUDA(cudaMemcpyAsync(h_Kval, dK, (size_t)plan->nnz * 8, cudaMemcpyDeviceToHost, s));
            EF_CUDA(cudaMemcpyAsync(h_Mval, dM, (size_t)plan->nnz * 8, cudaMemcpyDeviceToHost, s));
        }
        return ef_plan_check(plan, stream);
    }
    // Chunked: element chunk c and the sums it completes run on `stream`;
    // the CSR entries that are final after chunk c go back to the host on
    // the plan's copy stream while the next chunks compute.
    if (!plan->copy_stream) EF_CUDA(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : plan->copy_ev)
        if (!e) EF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaStream_t cs = plan->copy_stream;
    int64_t sent = 0;
    for (int c = 0; c < plan->pc_chunks; c++) {
        EF_TRY(launch_two_pass_chunk(plan, c, dn, dc, dK, dM, s));
        const int64_t done = plan->pc_csr_done[c + 1];
        if (done > sent) {
            EF_CUDA(cudaEventRecord(plan->copy_ev[c], s));
            EF_CUDA(cudaStreamWaitEvent(cs, plan->copy_ev[c], 0));
            EF_CUDA(cudaMemcpyAsync(h_Kval + sent, dK + sent, (size_t)(done - sent) * 8, cudaMemcpyDeviceToHost, cs));
            EF_CUDA(cudaMemcpyAsync(h_Mval + sent, dM + sent, (size_t)(done - sent) * 8, cudaMemcpyDeviceToHost, cs));
            sent = done;
        }
    }
    EF_CUDA(cudaEventRecord(plan->copy_ev[EF_MAX_CHUNKS], cs));
    EF_CUDA(cudaStreamWaitEvent(s, plan->copy_ev[EF_MAX_CHUNKS], 0));
    return ef_plan_check(plan, stream);
}

int ef_adjoint(const ef_plan* plan, const double* d_nodes, const double* d_coeff, const double* d_u,
               const double* d_v, double* d_J, double* d_grad_nodes, double* d_grad_coeff, void* stream)
{
    if (!plan || plan->variant != NED3) return EF_ERR_ARG;
    if (plan->T > 0 && (!d_nodes || !d_u || !d_v)) return EF_ERR_ARG;
    return launch_adjoint(plan, d_nodes, d_coeff, d_u, d_v, d_J, d_grad_nodes, d_grad_coeff, (cudaStream_t)stream);
}

int ef_plan_check(ef_plan* plan, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    EF_CUDA(cudaMemcpyAsync(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    if (st) EF_CUDA(cudaMemsetAsync(plan->d_status, 0, sizeof(int), s));
    if (st & ST_TIMEOUT) return EF_ERR_TIMEOUT;
    if (st & ST_DEGENERATE) return EF_ERR_DEGENERATE;
    return EF_OK;
}

void ef_plan_destroy(ef_plan* plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    profile_free(plan);
    plan_queue_free(plan);
    release_work_order(plan);
    free_plan_memory(plan);
    free(plan);
}

int rt0_assemble(int dim, const double* d_nodes, int64_t n_nodes, const int32_t* d_elems, int64_t n_elems,
                 const double* d_coeff, ef_csr* out, void* stream)
{
    return one_shot(EF_RT0, dim, d_nodes, n_nodes, d_elems, n_elems, d_coeff, out, stream);
}

int ned_assemble(int dim, const double* d_nodes, int64_t n_nodes, const int32_t* d_elems, int64_t n_elems,
                 const double* d_coeff, ef_csr* out, void* stream)
{
    return one_shot(EF_NED1, dim, d_nodes, n_nodes, d_elems, n_elems, d_coeff, out, stream);
}

void ef_csr_free(ef_csr* csr)
{
    if (!csr) return;
    cudaDeviceSynchronize();
    if (csr->d_rowptr) cudaFree(csr->d_rowptr);
    if (csr->d_colidx) cudaFree(csr->d_colidx);
    if (csr->d_K) cudaFree(csr->d_K);
    if (csr->d_M) cudaFree(csr->d_M);
    memset(csr, 0, sizeof(*csr));
}

const char* ef_status_string(int status)
{
    switch (status) {
        case EF_OK: return "ok";
        case EF_ERR_ARG: return "invalid argument";
        case EF_ERR_RANGE: return "node id out of range";
        case EF_ERR_DEGENERATE: return "degenerate element (det B_K = 0)";
        case EF_ERR_KEY_OVERFLOW: return "face key overflow (n_nodes^3 >= 2^64)";
        case EF_ERR_OOM: return "device out of memory";
        case EF_ERR_CUDA: return "CUDA error";
        case EF_ERR_TIMEOUT: return "bounded device wait timed out";
        case EF_ERR_SIZE: return "size beyond a limit of the call (32-bit indices or a fixed scratch array)";
        default: return "unknown status";
    }
}

const char* ef_last_error(void) { return last_error_text(); }

}  // extern "C"
