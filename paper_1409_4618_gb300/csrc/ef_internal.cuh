// Internal declarations of libedgefem (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/edgefem.h"

namespace ef {

// Element kinds handled by one plan.
enum Variant { RT2 = 0, RT3 = 1, NED2 = 2, NED3 = 3 };

inline int variant_of(int kind, int dim)
{
    if (kind == EF_RT0) return dim == 2 ? RT2 : RT3;
    return dim == 2 ? NED2 : NED3;
}
// local DOFs per element: edges (3 or 6) or faces (4)
inline int nloc_of(int v) { return v == RT3 ? 4 : (v == NED3 ? 6 : 3); }
// nodes of the mesh entity carrying a DOF: 2 (edge) or 3 (face)
inline int ent_nodes_of(int v) { return v == RT3 ? 3 : 2; }
// upper-triangle pairs (k <= l) of a local matrix
inline int npair_of(int v)
{
    int n = nloc_of(v);
    return n * (n + 1) / 2;
}

// Device status bits (plan->d_status).
enum : int { ST_DEGENERATE = 1, ST_RANGE = 2, ST_REPEAT = 4, ST_TIMEOUT = 8 };

// Error helpers ------------------------------------------------------------
void set_last_error(const char* where, cudaError_t err);
// printf-style text for ef_last_error (argument and size refusals)
void set_last_message(const char* fmt, ...);
#define EF_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            ::ef::set_last_error(#call, e_);             \
            return e_ == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA; \
        }                                                \
    } while (0)
#define EF_TRY(expr)          \
    do {                      \
        int s_ = (expr);      \
        if (s_ != EF_OK) return s_; \
    } while (0)

// Exclusive prefix sums -------------------------------------------------------
// out[i] = sum_{j<i} in[j] for i < n; out[n] = total when write_total.
// tmp: scan_tmp_bytes(n) bytes of device scratch.
size_t scan_tmp_bytes(int64_t n);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, bool write_total, void* tmp, cudaStream_t s);
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, bool write_total, void* tmp, cudaStream_t s);

// Stable LSD radix sort of (uint64 key, uint32 value) pairs on the low `bits`
// bits of the keys. Result ends in keys/vals. Scratch: radix_tmp_bytes(n).
size_t radix_tmp_bytes(int64_t n);
int radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, void* tmp, cudaStream_t s);

inline int bits_for(uint64_t max_value)
{
    int b = 0;
    while (b < 64 && (max_value >> b) != 0) b++;
    return b;
}

}  // namespace ef

#define EF_MAX_CHUNKS 16

namespace ef {
struct Queue;
struct Profile;
}
#define EF_PLAN_NO_PIPELINE 1   // members of a batch: one chunk, no plan streams
#define EF_PLAN_NO_ADJOINT 2    // no adjoint incidence / scratch

// The plan object behind the opaque C handle.
struct ef_plan {
    int flags;                // EF_PLAN_* bits
    int kind, dim, variant;
    int nv;     // nodes per element
    int nl;     // local DOFs
    int np;     // upper pairs per element
    int ent;    // nodes per DOF entity
    int64_t V, T, N, nnz, U;  // nodes, elements, DOFs, CSR nonzeros, upper nonzeros

    int32_t* d_elems;     // T x nv (plan copy)
    int32_t* d_elem2dof;  // T x nl
    uint8_t* d_signbits;  // T
    int32_t* d_dof2nodes; // N x ent
    int64_t* d_rowptr;    // N + 1
    int32_t* d_colidx;    // nnz
    uint32_t* d_seg;      // U + 1: contribution range of each upper nonzero
    uint32_t* d_perm;     // T * np: local-matrix index (pair * T + elem) of each contribution, segment order
    uint32_t* d_inv;      // T * np: position of (pair * T + elem) in the work-ordered contribution list
    uint32_t* d_pos_up;   // U: CSR position of (r, c), r <= c
    uint32_t* d_pos_lo;   // U: CSR position of (c, r), or 0xffffffff on the diagonal
    uint32_t* d_wseg;     // U + 1: list range of each work item of the sum (work order: completing
                          //   chunk, then descending contribution count inside 256-windows of u)
    uint32_t* d_wpos_up;  // U: CSR position of (r, c) of each work item
    uint32_t* d_wpos_lo;  // U: CSR position of (c, r), or 0xffffffff
    void* d_wst_up;       // U: per block of sum items (ef_assemble.cu), the items in ascending (r, c) position
    void* d_wst_lo;       // U: per block of sum items, the items in ascending (c, r) position
    double* d_local;      // 2 * np * T: contribution list of the two-pass paths, (K, M) pairs in work order
    int* d_status;        // device status word

    // fused path (one kernel over blocks of fb_block elements along an element order): see ef_fused.cu
    int fb_block;             // elements per block (0: no fused schedule)
    int fb_sfc;               // 1: blocks along the Morton order of the element centroids; 0: mesh order
    int fb_qcap;              // most partial slots of one block (its ticket queue in shared memory)
    int64_t fb_nblocks;
    int64_t fb_nslots;
    uint32_t* d_fb_order;     // T: the elements in block order (NULL: mesh order)
    uint32_t* d_fb_slot_off;  // nblocks + 1: slot range of each block
    uint32_t* d_fb_part_off;  // nblocks: first partial slot of each block
    uint32_t* d_fb_sinfo;     // per slot: start | count << 16
    uint32_t* d_fb_posA;      // per slot: CSR position of (r,c), or the split index if partial
    uint32_t* d_fb_posB;      // per slot: CSR position of (c,r), or 0xffffffff
    uint16_t* d_fb_sidx;      // per block [pair][element in block]: the value's place in the block's slot order
    uint32_t* d_fb_gpos;      // per contribution, block-major: its position in the global list
    uint32_t* d_px_uid;       // upper nonzeros split across blocks
    uint32_t* d_px_nb;        // per split nonzero: blocks contributing to it
    uint32_t* d_px_cnt;       // per split nonzero: tickets drawn in the current call
    int64_t n_px;
    int64_t n_partial;        // contributions of the split nonzeros

    // adjoint (3D Nedelec): node -> (element, vertex) incidence in element order, scratch
    uint32_t* d_node_off;    // V + 1
    uint32_t* d_node_inc;    // T * 4: element * 4 + vertex, grouped by node
    double* d_adj_part;      // T * 4 * 3: per (element, vertex) gradient
    double* d_adj_jpart;     // per-CTA partial energies

    // chunking of the work order, interleaved by the persistent queue (ef_queue.cu)
    int pc_chunks;                       // number of element chunks
    int64_t pc_chunk;                    // elements per chunk
    uint32_t pc_woff[EF_MAX_CHUNKS + 1]; // work-list range of the sums each chunk completes
    int64_t pc_csr_done[EF_MAX_CHUNKS + 1]; // CSR entries [0, pc_csr_done[c+1]) are final after chunks 0..c
    struct ef::Queue* queue;             // the single-launch schedule of ef_assemble
    int use_blocked;                     // ef_assemble runs the element-block kernel (ef_plan_set_block)
    int use_two_pass;                    // ef_assemble runs the plain two-pass kernels (chosen by ef_plan_tune)

    // host staging for ef_assemble_host, and its copy stream and chunk events
    double *d_stage_nodes, *d_stage_coeff, *d_stage_K, *d_stage_M;
    cudaStream_t copy_stream;
    cudaEvent_t copy_ev[EF_MAX_CHUNKS + 1];

    // per-kernel CUDA events of ef_assemble calls (ef_plan_profile)
    struct ef::Profile* prof;

    // per-CTA partial norms of ef_norm_l2 (allocated on first use)
    double* d_l2_part;
    // ef_load_vector (allocated on first use): DOF -> (element * nl + k)
    // incidence in ascending element order, and the local load vectors
    uint32_t* d_dof_off;
    uint32_t* d_dof_inc;
    double* d_load_local;
};

namespace ef {
const char* last_error_text();
int plan_create_internal(int kind, int dim, int64_t n_nodes, int64_t n_elems, const int32_t* d_elems, cudaStream_t s,
                         int flags, ef_plan** out);
int validate_elems(ef_plan* p, cudaStream_t s);
int build_topology(ef_plan* p, cudaStream_t s);
int build_pattern(ef_plan* p, cudaStream_t s);
int build_work_order(ef_plan* p, int nchunks, cudaStream_t s);
int default_pipeline_chunks(const ef_plan* p);
void release_work_order(ef_plan* p);
// Order a list of upper nonzeros by descending contribution count (stable), in place.
int order_by_count(const uint32_t* seg, uint32_t* list, int64_t n, uint64_t* keys, uint32_t* vals, void* tmp,
                   cudaStream_t s);
// nodes == NULL: blocks in mesh order; else along the Morton order of the centroids under nodes
int build_fused_block(ef_plan* p, int BE, const double* nodes, cudaStream_t s);
void release_fused(ef_plan* p);
bool fused_block_supported(int BE);
int build_adjoint(ef_plan* p, cudaStream_t s);
int launch_two_pass(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s);
// Two-pass kernels with K weighted by coeffK and M by coeffM (NULL: 1).
int launch_two_pass2(const ef_plan* p, const double* nodes, const double* coeffK, const double* coeffM, double* K,
                     double* M, cudaStream_t s);
// Element chunk c of the work order and the sums it completes.
int launch_two_pass_chunk(const ef_plan* p, int c, const double* nodes, const double* coeff, double* K, double* M,
                          cudaStream_t s);
int plan_queue_rebuild(ef_plan* p, cudaStream_t s);
int plan_queue_config(ef_plan* p, const ef_batch_config_t& cfg, cudaStream_t s);
int queue_max_ctas_per_sm(int variant, int BE);
void plan_queue_free(ef_plan* p);
int launch_queue(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s);
int launch_fused(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s);
// Events of ef_plan_profile: recorded before the call's first kernel, between
// its first and second kernel, and after its last kernel.
void profile_begin(const ef_plan* p, cudaStream_t s);
void profile_mid(const ef_plan* p, cudaStream_t s);
void profile_end(const ef_plan* p, cudaStream_t s);
void profile_free(ef_plan* p);
int launch_adjoint(const ef_plan* p, const double* nodes, const double* coeff, const double* u, const double* v,
                   double* J, double* gx, double* gs, cudaStream_t s);
}  // namespace ef
