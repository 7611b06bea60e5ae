// Assembly of K and M values: element kernel + fixed-order segmented sum.
//
// Element kernel: one thread per element computes its signed local K and M
// upper triangles (Sec. 2.4 integrals in closed form, ef_element.cuh) into
// pair-major scratch, coalesced per pair. This is the FP64-bound part.
//
// Sum: one thread per upper nonzero adds its contributions in ascending
// element order (the order fixed by the plan's stable sort) and writes the
// value to (r, c) and (c, r). No floating-point atomics.
//
// Work order of the sum: the upper nonzeros are grouped by the element chunk
// that completes them (the chunk of their last contribution) and, inside
// windows of 256 consecutive nonzeros, by descending contribution count, so
// that the lanes of a warp run loops of equal length (on this GPU an FP64
// warp instruction holds the FP64 pipe for its full duration even when lanes
// are idle) while memory accesses stay local.
//
// Layout: the contribution list is in the sum's work order (each item's
// contributions contiguous, ascending element order inside, items one after
// the other), and the element kernel writes each contribution straight to its
// slot through the plan's inverse map; a warp of the sum then reads one
// contiguous run and its per-item data (list start, CSR positions) coalesced.
//
// The chunking of the work order (the chunk that completes each nonzero) is
// what the persistent queue of ef_queue.cu interleaves; the kernels here are
// the plain two-pass form (ef_assemble_two_pass).
#include "ef_assemble.cuh"
#include "ef_internal.cuh"
#include "ef_queue.cuh"

namespace ef {
namespace {

constexpr int TPB = 256;
constexpr int EPB = 128;   // threads (elements) per CTA of the element kernels

// Writes each contribution to its slot in the nonzero-ordered contribution
// list: inv[q * T + e] = position of (element e, pair q). K values occupy
// list[0, np T), M values list[np T, 2 np T).
template <int VAR>
__device__ __forceinline__ void element_body(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                             const double* __restrict__ coeffK, const double* __restrict__ coeffM,
                                             const uint32_t* __restrict__ inv, int64_t e, int64_t T,
                                             double2* __restrict__ list, int* status)
{
    using E = ElemTraits<VAR>;
    double Kq[E::NP], Mq[E::NP];
    if (compute_element<VAR>(elems, nodes, coeffK, coeffM, e, Kq, Mq)) atomicOr(status, ST_DEGENERATE);
#pragma unroll
    for (int q = 0; q < E::NP; q++) {
        const uint32_t pos = __ldg(inv + (int64_t)q * T + e);
        list[pos] = make_double2(Kq[q], Mq[q]);
    }
}

// CTAs of EPB threads per SM the register budget is sized for: 96 registers
// for the 3D routines with products on the integer pipes (0.4 % faster than
// 80 at 64^3), at most 80 for the 2D ones
template <int VAR>
constexpr int elem_min_blocks()
{
    return (VAR == NED3 || VAR == RT3) ? 5 : 6;
}

template <int VAR>
__global__ void __launch_bounds__(EPB, elem_min_blocks<VAR>()) k_element_local(const int32_t* __restrict__ elems,
                                                       const double* __restrict__ nodes,
                                                       const double* __restrict__ coeffK,
                                                       const double* __restrict__ coeffM,
                                                       const uint32_t* __restrict__ inv, int64_t e0, int64_t e1,
                                                       int64_t T, double2* __restrict__ list, int* status)
{
    const int64_t e = e0 + (int64_t)blockIdx.x * EPB + threadIdx.x;
    if (e >= e1) return;
    element_body<VAR>(elems, nodes, coeffK, coeffM, inv, e, T, list, status);
}

// Mesh descriptor of CTA b of a batch launch into shared memory: blk_mesh[b]
// is the CTA's mesh, blk_off[m] the first CTA of mesh m; the descriptor's
// words are loaded by the first threads in parallel.
__device__ __forceinline__ int64_t load_block_mesh(const QueueMesh* __restrict__ md,
                                                   const uint32_t* __restrict__ blk_mesh,
                                                   const int64_t* __restrict__ blk_off, QueueMesh& d, int64_t* first)
{
    constexpr int W = (int)(sizeof(QueueMesh) / 8);
    static_assert(sizeof(QueueMesh) % 8 == 0, "descriptor of 8-byte words");
    const uint32_t m = __ldg(blk_mesh + blockIdx.x);
    if (threadIdx.x < W)
        reinterpret_cast<uint64_t*>(&d)[threadIdx.x] = __ldg(reinterpret_cast<const uint64_t*>(md + m) + threadIdx.x);
    if (threadIdx.x == W) *first = __ldg(blk_off + m);
    __syncthreads();
    return blockIdx.x - *first;
}

// The element kernel over every mesh of a batch: CTA b takes TPB elements of
// mesh m, blocks of meshes one after the other (blk_off: prefix of blocks).
template <int VAR>
__global__ void __launch_bounds__(EPB, elem_min_blocks<VAR>()) k_batch_element(const QueueMesh* __restrict__ md,
                                                       const uint32_t* __restrict__ blk_mesh,
                                                       const int64_t* __restrict__ blk_off, int* status)
{
    __shared__ QueueMesh d;
    __shared__ int64_t first;
    const int64_t e = load_block_mesh(md, blk_mesh, blk_off, d, &first) * EPB + threadIdx.x;
    if (e >= d.T) return;
    element_body<VAR>(d.elems, d.nodes, d.coeff, d.coeff, d.inv, e, d.T, d.list, status);
}

__global__ void k_work_keys(const uint32_t* seg, const uint32_t* perm, int64_t U, int64_t T, int64_t chunk,
                            uint64_t* keys, uint32_t* vals, uint32_t* chunk_count)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    const uint32_t s0 = seg[u], s1 = seg[u + 1];
    const uint32_t cnt = s1 - s0;
    const uint64_t rc = (uint64_t)((perm[s1 - 1] % T) / chunk);
    keys[u] = (rc << 32) | ((uint64_t)(u >> 8) << 8) | (uint64_t)(255u - (cnt < 255u ? cnt : 255u));
    vals[u] = (uint32_t)u;
    atomicAdd(&chunk_count[rc], 1u);
}

__global__ void k_work_items(const uint32_t* order, int64_t U, const uint32_t* seg, const uint32_t* pos_up,
                             const uint32_t* pos_lo, uint32_t* wcnt, uint32_t* wpos_up, uint32_t* wpos_lo)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= U) return;
    const uint32_t u = order[i];
    wcnt[i] = seg[u + 1] - seg[u];
    wpos_up[i] = pos_up[u];
    wpos_lo[i] = pos_lo[u];
}

// inv[pair * T + element] = position of that contribution in the work-ordered list
__global__ void k_work_inv(const uint32_t* order, int64_t U, const uint32_t* seg, const uint32_t* perm,
                           const uint32_t* wseg, uint32_t* inv)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= U) return;
    const uint32_t u = order[i];
    const uint32_t s0 = seg[u], s1 = seg[u + 1], w0 = wseg[i];
    for (uint32_t s = s0; s < s1; s++) inv[perm[s]] = w0 + (s - s0);
}

// The sum kernels: one CTA of SB threads per aligned block of SB work items
// (sum_block of ef_assemble.cuh).
__global__ void __launch_bounds__(SB) k_scatter(int64_t w0, int64_t w1, int64_t U, const uint32_t* __restrict__ wseg,
                                                const uint32_t* __restrict__ wpos_up,
                                                const uint32_t* __restrict__ wpos_lo,
                                                const StoreIdx* __restrict__ st_up, const StoreIdx* __restrict__ st_lo,
                                                const double2* __restrict__ list, double* __restrict__ K,
                                                double* __restrict__ M)
{
    sum_block((w0 / SB + blockIdx.x) * SB, w0, w1, U, wseg, wpos_up, wpos_lo, st_up, st_lo, list, K, M);
}

// The sum over every mesh of a batch: CTA b takes the SB-block of work items
// b - blk_off[m] of mesh m.
template <int NP>
__global__ void __launch_bounds__(SB, 8) k_batch_scatter(const QueueMesh* __restrict__ md,
                                                      const uint32_t* __restrict__ blk_mesh,
                                                      const int64_t* __restrict__ blk_off)
{
    // the CTA's mesh descriptor in shared memory: read there where it is used
    // instead of held in registers
    __shared__ QueueMesh d;
    __shared__ int64_t first;
    const int64_t base = load_block_mesh(md, blk_mesh, blk_off, d, &first) * SB;
    sum_block(base, 0, d.U, d.U, d.wseg, d.wpos_up, d.wpos_lo, (const StoreIdx*)d.wst_up,
                  (const StoreIdx*)d.wst_lo, d.list, d.K, d.M);
}

// Store-order keys: block of the work item, then its CSR position.
__global__ void k_store_keys(const uint32_t* __restrict__ wpos, int64_t U, uint64_t* keys, uint32_t* vals)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= U) return;
    keys[i] = ((uint64_t)(i / SB) << 32) | wpos[i];
    vals[i] = (uint32_t)(i % SB);
}

__global__ void k_store_index(const uint32_t* __restrict__ vals, int64_t U, StoreIdx* out)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < U) out[i] = (StoreIdx)vals[i];
}

// Latest completing chunk of every CSR row: row r is final once every upper
// nonzero in row r or column r is summed.
__global__ void k_row_last_chunk(const uint32_t* seg, const uint32_t* perm, const uint32_t* pos_up,
                                 const uint32_t* pos_lo, const int32_t* colidx, int64_t U, int64_t T, int64_t chunk,
                                 uint32_t* row_last)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    const uint32_t rc = (uint32_t)((perm[seg[u + 1] - 1] % T) / chunk);
    const uint32_t j = (uint32_t)colidx[pos_up[u]];
    if (rc) atomicMax(row_last + j, rc);
    const uint32_t pl = pos_lo[u];
    if (pl != 0xffffffffu && rc) atomicMax(row_last + colidx[pl], rc);
}

// first_row[c] = smallest row whose last chunk is > c (rows before it are
// final after chunks 0..c); a CTA reduces in shared memory first.
__global__ void k_first_open_row(const uint32_t* row_last, int64_t N, int nc, uint32_t* first_row)
{
    __shared__ uint32_t s_min[EF_MAX_CHUNKS];
    if (threadIdx.x < EF_MAX_CHUNKS) s_min[threadIdx.x] = 0xffffffffu;
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (r < N)
        for (uint32_t c = 0; c < row_last[r]; c++) atomicMin(&s_min[c], (uint32_t)r);
    __syncthreads();
    if (threadIdx.x < nc && s_min[threadIdx.x] != 0xffffffffu) atomicMin(first_row + threadIdx.x, s_min[threadIdx.x]);
}

__global__ void k_rows_to_positions(const uint32_t* first_row, const int64_t* rowptr, int64_t N, int nc,
                                    int64_t* pos)
{
    const int c = threadIdx.x;
    if (c >= nc) return;
    const uint32_t r = first_row[c];
    pos[c] = rowptr[r < N ? r : N];
}

__global__ void k_count_keys(const uint32_t* seg, const uint32_t* list, int64_t n, uint64_t* keys, uint32_t* vals)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    const uint32_t u = list[i];
    const uint32_t cnt = seg[u + 1] - seg[u];
    keys[i] = ((uint64_t)(i >> 8) << 8) | (uint64_t)(255u - (cnt < 255u ? cnt : 255u));
    vals[i] = u;
}

int element_range(const ef_plan* p, const double* nodes, const double* cK, const double* cM, int64_t e0, int64_t e1,
                  cudaStream_t s)
{
    if (e1 <= e0) return EF_OK;
    const unsigned grid = (unsigned)((e1 - e0 + EPB - 1) / EPB);
    switch (p->variant) {
        case RT2: k_element_local<RT2><<<grid, EPB, 0, s>>>(p->d_elems, nodes, cK, cM, p->d_inv, e0, e1, p->T, (double2*)p->d_local, p->d_status); break;
        case NED2: k_element_local<NED2><<<grid, EPB, 0, s>>>(p->d_elems, nodes, cK, cM, p->d_inv, e0, e1, p->T, (double2*)p->d_local, p->d_status); break;
        case RT3: k_element_local<RT3><<<grid, EPB, 0, s>>>(p->d_elems, nodes, cK, cM, p->d_inv, e0, e1, p->T, (double2*)p->d_local, p->d_status); break;
        default: k_element_local<NED3><<<grid, EPB, 0, s>>>(p->d_elems, nodes, cK, cM, p->d_inv, e0, e1, p->T, (double2*)p->d_local, p->d_status); break;
    }
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int scatter_range(const ef_plan* p, int64_t w0, int64_t w1, double* K, double* M, cudaStream_t s)
{
    if (w1 <= w0) return EF_OK;
    const unsigned grid = (unsigned)((w1 - 1) / SB - w0 / SB + 1);
    k_scatter<<<grid, SB, 0, s>>>(w0, w1, p->U, p->d_wseg, p->d_wpos_up, p->d_wpos_lo, (const StoreIdx*)p->d_wst_up,
                                  (const StoreIdx*)p->d_wst_lo, (const double2*)p->d_local, K, M);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

void free_work_order(ef_plan* p)
{
    void* ptrs[] = {p->d_wseg, p->d_wpos_up, p->d_wpos_lo, p->d_inv, p->d_wst_up, p->d_wst_lo};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    p->d_wseg = p->d_wpos_up = p->d_wpos_lo = p->d_inv = nullptr;
    p->d_wst_up = p->d_wst_lo = nullptr;
}

}  // namespace

// Reorder `list` (upper nonzero ids) inside windows of 256 entries by
// descending contribution count (stable). keys / vals: n entries of scratch.
int order_by_count(const uint32_t* seg, uint32_t* list, int64_t n, uint64_t* keys, uint32_t* vals, void* tmp,
                   cudaStream_t s)
{
    if (n <= 1) return EF_OK;
    k_count_keys<<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, s>>>(seg, list, n, keys, vals);
    EF_CUDA(cudaGetLastError());
    EF_TRY(radix_sort_pairs(keys, vals, n, bits_for(((uint64_t)(n >> 8) << 8) | 255u), tmp, s));
    EF_CUDA(cudaMemcpyAsync(list, vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    return EF_OK;
}

// Work order and contribution-list layout for `nchunks` element chunks
// (1 = plain two-pass): the order of the sums, their list ranges, CSR
// positions, the element kernel's write positions, and the plan streams.
int build_work_order(ef_plan* p, int nchunks, cudaStream_t s)
{
    p->pc_chunks = 0;
    free_work_order(p);
    if (p->U == 0) return EF_OK;
    if (nchunks < 1 || nchunks > EF_MAX_CHUNKS) return EF_ERR_ARG;
    const int64_t U = p->U, T = p->T, n = T * p->np;
    int64_t chunk = (T + nchunks - 1) / nchunks;
    chunk = (chunk + TPB - 1) / TPB * TPB;
    const int nc = (int)((T + chunk - 1) / chunk);
    uint64_t* keys = nullptr;
    uint32_t *order = nullptr, *cnt = nullptr, *wcnt = nullptr;
    void* tmp = nullptr;
    size_t tb = radix_tmp_bytes(U);
    if (scan_tmp_bytes(U + 1) > tb) tb = scan_tmp_bytes(U + 1);
    int st = EF_OK;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMalloc((void**)&p->d_inv, n * 4)) || !ok(cudaMalloc((void**)&p->d_wseg, (U + 1) * 4)) ||
        !ok(cudaMalloc((void**)&p->d_wpos_up, U * 4)) || !ok(cudaMalloc((void**)&p->d_wpos_lo, U * 4)) ||
        !ok(cudaMalloc(&p->d_wst_up, U * sizeof(StoreIdx))) || !ok(cudaMalloc(&p->d_wst_lo, U * sizeof(StoreIdx))) ||
        !ok(cudaMalloc((void**)&order, U * 4)) || !ok(cudaMalloc((void**)&keys, U * 8)) ||
        !ok(cudaMalloc((void**)&wcnt, U * 4)) || !ok(cudaMalloc((void**)&cnt, EF_MAX_CHUNKS * 4)) ||
        !ok(cudaMalloc(&tmp, tb)))
        st = EF_ERR_OOM;
    uint32_t hc[EF_MAX_CHUNKS] = {0};
    const unsigned gu = (unsigned)((U + TPB - 1) / TPB);
    if (st == EF_OK) {
        cudaMemsetAsync(cnt, 0, EF_MAX_CHUNKS * 4, s);
        k_work_keys<<<gu, TPB, 0, s>>>(p->d_seg, p->d_perm, U, T, chunk, keys, order, cnt);
        st = radix_sort_pairs(keys, order, U, bits_for(((uint64_t)(nc - 1) << 32) | 0xffffffffull), tmp, s);
    }
    if (st == EF_OK) {
        k_work_items<<<gu, TPB, 0, s>>>(order, U, p->d_seg, p->d_pos_up, p->d_pos_lo, wcnt, p->d_wpos_up,
                                        p->d_wpos_lo);
        st = exclusive_scan_u32(wcnt, p->d_wseg, U, true, tmp, s);
    }
    int64_t hpos[EF_MAX_CHUNKS] = {0};
    if (st == EF_OK) {
        k_work_inv<<<gu, TPB, 0, s>>>(order, U, p->d_seg, p->d_perm, p->d_wseg, p->d_inv);
        // store orders of the sum (keys and wcnt are free scratch now)
        const uint64_t kmax = ((uint64_t)((U - 1) / SB) << 32) | 0xffffffffull;
        k_store_keys<<<gu, TPB, 0, s>>>(p->d_wpos_up, U, keys, wcnt);
        st = radix_sort_pairs(keys, wcnt, U, bits_for(kmax), tmp, s);
        if (st == EF_OK) {
            k_store_index<<<gu, TPB, 0, s>>>(wcnt, U, (StoreIdx*)p->d_wst_up);
            k_store_keys<<<gu, TPB, 0, s>>>(p->d_wpos_lo, U, keys, wcnt);
            st = radix_sort_pairs(keys, wcnt, U, bits_for(kmax), tmp, s);
        }
        if (st == EF_OK) k_store_index<<<gu, TPB, 0, s>>>(wcnt, U, (StoreIdx*)p->d_wst_lo);
    }
    if (st == EF_OK) {
        cudaMemcpyAsync(hc, cnt, EF_MAX_CHUNKS * 4, cudaMemcpyDeviceToHost, s);
        // CSR prefix that is final after each chunk (the scratch `order` and
        // `keys` are free again): rows' last chunks, first open row, position
        uint32_t* row_last = (uint32_t*)keys;                       // N entries (N <= 2 U)
        uint32_t* first_row = cnt;
        int64_t* pos = (int64_t*)order;
        if ((int64_t)p->N * 4 > U * 8) {
            st = EF_ERR_ARG;   // cannot happen: every row holds a diagonal upper nonzero
        } else {
            cudaMemsetAsync(row_last, 0, (size_t)p->N * 4, s);
            k_row_last_chunk<<<gu, TPB, 0, s>>>(p->d_seg, p->d_perm, p->d_pos_up, p->d_pos_lo, p->d_colidx, U, T,
                                                 chunk, row_last);
            cudaMemsetAsync(first_row, 0xff, EF_MAX_CHUNKS * 4, s);
            k_first_open_row<<<(unsigned)((p->N + TPB - 1) / TPB), TPB, 0, s>>>(row_last, p->N, nc, first_row);
            k_rows_to_positions<<<1, 32, 0, s>>>(first_row, p->d_rowptr, p->N, nc, pos);
            cudaMemcpyAsync(hpos, pos, sizeof(int64_t) * nc, cudaMemcpyDeviceToHost, s);
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_last_error("build_work_order", e);
            st = EF_ERR_CUDA;
        }
    }
    cudaFree(keys);
    cudaFree(order);
    cudaFree(wcnt);
    cudaFree(cnt);
    cudaFree(tmp);
    if (st != EF_OK) {
        free_work_order(p);
        return st;
    }
    p->pc_chunks = nc;
    p->pc_chunk = chunk;
    p->pc_woff[0] = 0;
    for (int c = 0; c < nc; c++) p->pc_woff[c + 1] = p->pc_woff[c] + hc[c];
    p->pc_csr_done[0] = 0;
    for (int c = 0; c < nc; c++) p->pc_csr_done[c + 1] = hpos[c] > p->pc_csr_done[c] ? hpos[c] : p->pc_csr_done[c];
    p->pc_csr_done[nc] = p->nnz;
    return EF_OK;
}

int default_pipeline_chunks(const ef_plan* p)
{
    if (p->flags & EF_PLAN_NO_PIPELINE) return 1;
    // chunks of at least 32K elements, at most 16 of them
    int64_t c = p->T / 32768;
    if (c < 1) c = 1;
    if (c > EF_MAX_CHUNKS) c = EF_MAX_CHUNKS;
    return (int)c;
}

void release_work_order(ef_plan* p) { free_work_order(p); }

// Batch in two launches: every mesh's element kernel, then every mesh's sums.
int launch_batch_two_pass(int variant, const QueueMesh* d_mesh, const uint32_t* d_emesh, const int64_t* d_eblk,
                          int64_t n_eblk, const uint32_t* d_smesh, const int64_t* d_sblk, int64_t n_sblk, int* status,
                          cudaStream_t s)
{
    if (n_eblk > 0) {
        const unsigned g = (unsigned)n_eblk;
        switch (variant) {
            case RT2: k_batch_element<RT2><<<g, EPB, 0, s>>>(d_mesh, d_emesh, d_eblk, status); break;
            case NED2: k_batch_element<NED2><<<g, EPB, 0, s>>>(d_mesh, d_emesh, d_eblk, status); break;
            case RT3: k_batch_element<RT3><<<g, EPB, 0, s>>>(d_mesh, d_emesh, d_eblk, status); break;
            default: k_batch_element<NED3><<<g, EPB, 0, s>>>(d_mesh, d_emesh, d_eblk, status); break;
        }
    }
    if (n_sblk > 0) {
        const unsigned g = (unsigned)n_sblk;
        switch (variant) {
            case RT2:
            case NED2: k_batch_scatter<ElemTraits<RT2>::NP><<<g, SB, 0, s>>>(d_mesh, d_smesh, d_sblk); break;
            case RT3: k_batch_scatter<ElemTraits<RT3>::NP><<<g, SB, 0, s>>>(d_mesh, d_smesh, d_sblk); break;
            default: k_batch_scatter<ElemTraits<NED3>::NP><<<g, SB, 0, s>>>(d_mesh, d_smesh, d_sblk); break;
        }
    }
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int64_t element_blocks(int64_t T) { return (T + EPB - 1) / EPB; }
int64_t sum_blocks(int64_t U) { return (U + SB - 1) / SB; }

int launch_two_pass_chunk(const ef_plan* p, int c, const double* nodes, const double* coeff, double* K, double* M,
                          cudaStream_t s)
{
    if (c < 0 || c >= p->pc_chunks) return EF_ERR_ARG;
    const int64_t e0 = (int64_t)c * p->pc_chunk;
    const int64_t e1 = e0 + p->pc_chunk < p->T ? e0 + p->pc_chunk : p->T;
    EF_TRY(element_range(p, nodes, coeff, coeff, e0, e1, s));
    return scatter_range(p, p->pc_woff[c], p->pc_woff[c + 1], K, M, s);
}

int launch_two_pass2(const ef_plan* p, const double* nodes, const double* coeffK, const double* coeffM, double* K,
                     double* M, cudaStream_t s)
{
    if (p->T == 0) return EF_OK;
    EF_TRY(element_range(p, nodes, coeffK, coeffM, 0, p->T, s));
    profile_mid(p, s);
    return scatter_range(p, 0, p->U, K, M, s);
}

int launch_two_pass(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M,
                    cudaStream_t s)
{
    return launch_two_pass2(p, nodes, coeff, coeff, K, M, s);
}

}  // namespace ef
