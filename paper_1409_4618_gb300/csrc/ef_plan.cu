// Plan construction: mesh topology (Sec. 3: elems2edges / elems2faces,
// edges2nodes / faces2nodes, signs_e / signs_f) and the CSR pattern with the
// contribution -> nonzero map used by the deterministic sum.
//
// Topology: every (element, local DOF) slot gets the key of its entity's
// sorted global node ids (edge: a*V + b; face: (a*V + b)*V + c), the slots
// are radix-sorted by key, and the DOF id is the rank of the key among the
// distinct keys, i.e. the lexicographic order of the node tuples.
//
// Pattern: every upper pair (k <= l) of every element gives the key
// min(i,j)*N + max(i,j) of its DOFs; a stable sort groups the contributions
// of each upper nonzero in ascending element order. The CSR row r holds first
// its columns below the diagonal (from the transposed upper list, sorted by a
// second radix sort), then the diagonal and the columns above it.
#include <stdio.h>
#include <stdlib.h>

#include "ef_element.cuh"
#include "ef_internal.cuh"

namespace ef {
namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

struct DevBuf {
    void* p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { reset(); }
    void reset()
    {
        if (p) cudaFree(p);
        p = nullptr;
    }
    int alloc(size_t bytes)
    {
        if (p) cudaFree(p);
        p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
        if (e != cudaSuccess) {
            set_last_error("cudaMalloc", e);
            p = nullptr;
            return EF_ERR_OOM;
        }
        return EF_OK;
    }
    template <typename T>
    T* as() const
    {
        return (T*)p;
    }
};

__global__ void k_validate(const int32_t* elems, int64_t T, int nv, int64_t V, int* status)
{
    int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (e >= T) return;
    int32_t g[4];
    int bad = 0;
    for (int a = 0; a < nv; a++) {
        g[a] = elems[e * nv + a];
        if (g[a] < 0 || (int64_t)g[a] >= V) bad |= ST_RANGE;
        for (int b = 0; b < a; b++)
            if (g[b] == g[a]) bad |= ST_REPEAT;
    }
    if (bad) atomicOr(status, bad);
}

__device__ __forceinline__ void sort2(int32_t& a, int32_t& b)
{
    int32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

template <int VAR>
__global__ void k_entity_keys(const int32_t* elems, int64_t T, uint64_t V, uint64_t* keys, uint32_t* vals)
{
    constexpr int NV = (VAR == RT2 || VAR == NED2) ? 3 : 4;
    constexpr int NL = (VAR == RT3) ? 4 : ((VAR == NED3) ? 6 : 3);
    int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (e >= T) return;
    int32_t g[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) g[a] = elems[e * NV + a];
#pragma unroll
    for (int k = 0; k < NL; k++) {
        uint64_t key;
        if (VAR == RT3) {
            int32_t a = g[kFace3[k][0]], b = g[kFace3[k][1]], c = g[kFace3[k][2]];
            sort2(a, b);
            sort2(b, c);
            sort2(a, b);
            key = ((uint64_t)a * V + (uint64_t)b) * V + (uint64_t)c;
        } else if (VAR == NED3) {
            int32_t a = g[kEdge3[k][0]], b = g[kEdge3[k][1]];
            sort2(a, b);
            key = (uint64_t)a * V + (uint64_t)b;
        } else {
            int32_t a = g[kEdge2[k][0]], b = g[kEdge2[k][1]];
            sort2(a, b);
            key = (uint64_t)a * V + (uint64_t)b;
        }
        keys[e * NL + k] = key;
        vals[e * NL + k] = (uint32_t)(e * NL + k);
    }
}

__global__ void k_heads(const uint64_t* keys, int64_t n, uint32_t* flag)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_assign_dofs(const uint64_t* keys, const uint32_t* vals, const uint32_t* flag, const uint32_t* ex,
                              int64_t n, uint64_t V, int ent, int32_t* elem2dof, int32_t* dof2nodes)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    uint32_t id = ex[i] + flag[i] - 1u;
    elem2dof[vals[i]] = (int32_t)id;
    if (flag[i]) {
        uint64_t k = keys[i];
        if (ent == 2) {
            dof2nodes[(int64_t)id * 2 + 0] = (int32_t)(k / V);
            dof2nodes[(int64_t)id * 2 + 1] = (int32_t)(k % V);
        } else {
            uint64_t c = k % V, ab = k / V;
            dof2nodes[(int64_t)id * 3 + 0] = (int32_t)(ab / V);
            dof2nodes[(int64_t)id * 3 + 1] = (int32_t)(ab % V);
            dof2nodes[(int64_t)id * 3 + 2] = (int32_t)c;
        }
    }
}

template <int VAR>
__global__ void k_signbits(const int32_t* elems, int64_t T, uint8_t* bits)
{
    constexpr int NV = (VAR == RT2 || VAR == NED2) ? 3 : 4;
    int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (e >= T) return;
    int32_t g[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) g[a] = elems[e * NV + a];
    bits[e] = (uint8_t)sign_bits<VAR>(g);
}

// upper pair q -> (k, l), row-major over k <= l
__device__ __forceinline__ void pair_of(int q, int nl, int& k, int& l)
{
    k = 0;
    int row = nl;
    while (q >= row) {
        q -= row;
        k++;
        row--;
    }
    l = k + q;
}

__global__ void k_contrib_keys(const int32_t* e2d, int64_t T, int nl, int np, uint64_t N, uint64_t* keys,
                               uint32_t* vals)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= T * np) return;
    int64_t e = i / np;
    int q = (int)(i - e * np), k, l;
    pair_of(q, nl, k, l);
    uint64_t a = (uint64_t)e2d[e * nl + k], b = (uint64_t)e2d[e * nl + l];
    uint64_t r = a < b ? a : b, c = a < b ? b : a;
    keys[i] = r * N + c;
    vals[i] = (uint32_t)((int64_t)q * T + e);  // index into the pair-major local-matrix array
}

__global__ void k_upper(const uint64_t* keys, const uint32_t* flag, const uint32_t* ex, int64_t n, uint64_t N,
                        uint32_t* seg, int32_t* urow, int32_t* ucol, uint32_t* upper_cnt, uint32_t* lower_cnt)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n || !flag[i]) return;
    uint32_t u = ex[i];
    uint64_t k = keys[i];
    int32_t r = (int32_t)(k / N), c = (int32_t)(k % N);
    seg[u] = (uint32_t)i;
    urow[u] = r;
    ucol[u] = c;
    atomicAdd(&upper_cnt[r], 1u);
    if (r < c) atomicAdd(&lower_cnt[c], 1u);
}

__global__ void k_row_len(const uint32_t* upper_cnt, const uint32_t* lower_cnt, int64_t N, int64_t* len)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < N) len[i] = (int64_t)upper_cnt[i] + lower_cnt[i];
}

__global__ void k_row_first(const int32_t* urow, int64_t U, uint32_t* row_first)
{
    int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    if (u == 0 || urow[u] != urow[u - 1]) row_first[urow[u]] = (uint32_t)u;
}

__global__ void k_pos_up(const int32_t* urow, const int32_t* ucol, int64_t U, uint64_t N, const int64_t* rowptr,
                         const uint32_t* lower_cnt, const uint32_t* row_first, uint32_t* pos_up, uint32_t* pos_lo,
                         int32_t* colidx, uint64_t* key2, uint32_t* val2)
{
    int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    int32_t r = urow[u], c = ucol[u];
    int64_t p = rowptr[r] + lower_cnt[r] + (u - row_first[r]);
    pos_up[u] = (uint32_t)p;
    colidx[p] = c;
    if (r < c) {
        int64_t j = u - (int64_t)r - 1;   // the diagonal of rows 0..r precede u
        key2[j] = (uint64_t)c * N + (uint64_t)r;
        val2[j] = (uint32_t)u;
    } else {
        pos_lo[u] = 0xffffffffu;
    }
}

__global__ void k_group_first(const uint64_t* key2, int64_t n, uint64_t N, uint32_t* gfirst)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    uint64_t c = key2[i] / N;
    if (i == 0 || key2[i - 1] / N != c) gfirst[c] = (uint32_t)i;
}

__global__ void k_pos_lo(const uint64_t* key2, const uint32_t* val2, int64_t n, uint64_t N, const int64_t* rowptr,
                         const uint32_t* gfirst, uint32_t* pos_lo, int32_t* colidx)
{
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key2[i];
    uint64_t c = k / N, r = k % N;
    int64_t p = rowptr[c] + (i - gfirst[c]);
    pos_lo[val2[i]] = (uint32_t)p;
    colidx[p] = (int32_t)r;
}

template <typename T>
int dalloc(T** p, int64_t n)
{
    cudaError_t e = cudaMalloc((void**)p, (size_t)(n > 0 ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_last_error("cudaMalloc", e);
        return EF_ERR_OOM;
    }
    return EF_OK;
}

}  // namespace

int build_topology(ef_plan* p, cudaStream_t s)
{
    const int64_t T = p->T, n = T * p->nl;
    const uint64_t V = (uint64_t)p->V;
    EF_TRY(dalloc(&p->d_elem2dof, n));
    EF_TRY(dalloc(&p->d_signbits, T));
    if (T == 0) {
        p->N = 0;
        EF_TRY(dalloc(&p->d_dof2nodes, 1));
        return EF_OK;
    }
    DevBuf keys, vals, flag, ex, tmp;
    EF_TRY(keys.alloc((size_t)n * 8));
    EF_TRY(vals.alloc((size_t)n * 4));
    EF_TRY(flag.alloc((size_t)n * 4));
    EF_TRY(ex.alloc((size_t)n * 4 + 4));
    size_t tb = radix_tmp_bytes(n);
    if (scan_tmp_bytes(n) > tb) tb = scan_tmp_bytes(n);
    EF_TRY(tmp.alloc(tb));

    switch (p->variant) {
        case RT2: k_entity_keys<RT2><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, V, keys.as<uint64_t>(), vals.as<uint32_t>()); break;
        case NED2: k_entity_keys<NED2><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, V, keys.as<uint64_t>(), vals.as<uint32_t>()); break;
        case RT3: k_entity_keys<RT3><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, V, keys.as<uint64_t>(), vals.as<uint32_t>()); break;
        default: k_entity_keys<NED3><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, V, keys.as<uint64_t>(), vals.as<uint32_t>()); break;
    }
    EF_CUDA(cudaGetLastError());
    uint64_t maxkey = p->variant == RT3 ? (V * V * V - 1) : (V * V - 1);
    EF_TRY(radix_sort_pairs(keys.as<uint64_t>(), vals.as<uint32_t>(), n, bits_for(maxkey), tmp.p, s));
    k_heads<<<grid_for(n), TPB, 0, s>>>(keys.as<uint64_t>(), n, flag.as<uint32_t>());
    EF_TRY(exclusive_scan_u32(flag.as<uint32_t>(), ex.as<uint32_t>(), n, true, tmp.p, s));
    uint32_t Nh = 0;
    EF_CUDA(cudaMemcpyAsync(&Nh, ex.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    p->N = Nh;
    EF_TRY(dalloc(&p->d_dof2nodes, p->N * p->ent));
    k_assign_dofs<<<grid_for(n), TPB, 0, s>>>(keys.as<uint64_t>(), vals.as<uint32_t>(), flag.as<uint32_t>(),
                                              ex.as<uint32_t>(), n, V, p->ent, p->d_elem2dof, p->d_dof2nodes);
    switch (p->variant) {
        case RT2: k_signbits<RT2><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, p->d_signbits); break;
        case NED2: k_signbits<NED2><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, p->d_signbits); break;
        case RT3: k_signbits<RT3><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, p->d_signbits); break;
        default: k_signbits<NED3><<<grid_for(T), TPB, 0, s>>>(p->d_elems, T, p->d_signbits); break;
    }
    EF_CUDA(cudaGetLastError());
    EF_CUDA(cudaStreamSynchronize(s));
    return EF_OK;
}

int build_pattern(ef_plan* p, cudaStream_t s)
{
    const int64_t T = p->T, N = p->N, n = T * p->np;
    EF_TRY(dalloc(&p->d_rowptr, N + 1));
    if (T == 0) {
        p->nnz = 0;
        p->U = 0;
        EF_CUDA(cudaMemsetAsync(p->d_rowptr, 0, 8, s));
        EF_TRY(dalloc(&p->d_colidx, 1));
        EF_TRY(dalloc(&p->d_seg, 1));
        EF_TRY(dalloc(&p->d_perm, 1));
        EF_TRY(dalloc(&p->d_pos_up, 1));
        EF_TRY(dalloc(&p->d_pos_lo, 1));
        EF_CUDA(cudaStreamSynchronize(s));
        return EF_OK;
    }
    const uint64_t Nu = (uint64_t)N;
    DevBuf keys, flag, ex, tmp;
    EF_TRY(keys.alloc((size_t)n * 8));
    EF_TRY(dalloc(&p->d_perm, n));
    EF_TRY(flag.alloc((size_t)n * 4));
    EF_TRY(ex.alloc((size_t)n * 4 + 4));
    size_t tb = radix_tmp_bytes(n);
    if (scan_tmp_bytes(n) > tb) tb = scan_tmp_bytes(n);
    EF_TRY(tmp.alloc(tb));

    k_contrib_keys<<<grid_for(n), TPB, 0, s>>>(p->d_elem2dof, T, p->nl, p->np, Nu, keys.as<uint64_t>(), p->d_perm);
    EF_CUDA(cudaGetLastError());
    EF_TRY(radix_sort_pairs(keys.as<uint64_t>(), p->d_perm, n, bits_for(Nu * Nu - 1), tmp.p, s));
    k_heads<<<grid_for(n), TPB, 0, s>>>(keys.as<uint64_t>(), n, flag.as<uint32_t>());
    EF_TRY(exclusive_scan_u32(flag.as<uint32_t>(), ex.as<uint32_t>(), n, true, tmp.p, s));
    uint32_t Uh = 0;
    EF_CUDA(cudaMemcpyAsync(&Uh, ex.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    const int64_t U = Uh;
    p->U = U;
    p->nnz = 2 * U - N;   // every row holds its diagonal once; off-diagonal uppers appear twice
    if (p->nnz >= ((int64_t)1 << 32) - 1) return EF_ERR_SIZE;

    DevBuf urow, ucol, ucnt, lcnt, rfirst, rowlen, key2, val2, gfirst;
    EF_TRY(dalloc(&p->d_seg, U + 1));
    EF_TRY(urow.alloc((size_t)U * 4));
    EF_TRY(ucol.alloc((size_t)U * 4));
    EF_TRY(ucnt.alloc((size_t)N * 4));
    EF_TRY(lcnt.alloc((size_t)N * 4));
    EF_CUDA(cudaMemsetAsync(ucnt.p, 0, (size_t)N * 4, s));
    EF_CUDA(cudaMemsetAsync(lcnt.p, 0, (size_t)N * 4, s));
    k_upper<<<grid_for(n), TPB, 0, s>>>(keys.as<uint64_t>(), flag.as<uint32_t>(), ex.as<uint32_t>(), n, Nu, p->d_seg,
                                        urow.as<int32_t>(), ucol.as<int32_t>(), ucnt.as<uint32_t>(),
                                        lcnt.as<uint32_t>());
    {
        uint32_t nn = (uint32_t)n;
        EF_CUDA(cudaMemcpyAsync(p->d_seg + U, &nn, 4, cudaMemcpyHostToDevice, s));
        EF_CUDA(cudaStreamSynchronize(s));
    }
    keys.reset();  // release the big buffers before the next stage
    flag.reset();
    ex.reset();

    EF_TRY(rowlen.alloc((size_t)N * 8));
    k_row_len<<<grid_for(N), TPB, 0, s>>>(ucnt.as<uint32_t>(), lcnt.as<uint32_t>(), N, rowlen.as<int64_t>());
    EF_TRY(exclusive_scan_i64(rowlen.as<int64_t>(), p->d_rowptr, N, true, tmp.p, s));
    EF_TRY(rfirst.alloc((size_t)N * 4));
    k_row_first<<<grid_for(U), TPB, 0, s>>>(urow.as<int32_t>(), U, rfirst.as<uint32_t>());
    const int64_t n2 = U - N;
    EF_TRY(dalloc(&p->d_colidx, p->nnz));
    EF_TRY(dalloc(&p->d_pos_up, U));
    EF_TRY(dalloc(&p->d_pos_lo, U));
    EF_TRY(key2.alloc((size_t)(n2 > 0 ? n2 : 1) * 8));
    EF_TRY(val2.alloc((size_t)(n2 > 0 ? n2 : 1) * 4));
    k_pos_up<<<grid_for(U), TPB, 0, s>>>(urow.as<int32_t>(), ucol.as<int32_t>(), U, Nu, p->d_rowptr,
                                         lcnt.as<uint32_t>(), rfirst.as<uint32_t>(), p->d_pos_up, p->d_pos_lo,
                                         p->d_colidx, key2.as<uint64_t>(), val2.as<uint32_t>());
    EF_CUDA(cudaGetLastError());
    if (n2 > 0) {
        EF_TRY(radix_sort_pairs(key2.as<uint64_t>(), val2.as<uint32_t>(), n2, bits_for(Nu * Nu - 1), tmp.p, s));
        EF_TRY(gfirst.alloc((size_t)N * 4));
        k_group_first<<<grid_for(n2), TPB, 0, s>>>(key2.as<uint64_t>(), n2, Nu, gfirst.as<uint32_t>());
        k_pos_lo<<<grid_for(n2), TPB, 0, s>>>(key2.as<uint64_t>(), val2.as<uint32_t>(), n2, Nu, p->d_rowptr,
                                              gfirst.as<uint32_t>(), p->d_pos_lo, p->d_colidx);
        EF_CUDA(cudaGetLastError());
    }
    EF_CUDA(cudaStreamSynchronize(s));
    return EF_OK;
}

int validate_elems(ef_plan* p, cudaStream_t s)
{
    if (p->T == 0) return EF_OK;
    EF_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    k_validate<<<grid_for(p->T), TPB, 0, s>>>(p->d_elems, p->T, p->nv, p->V, p->d_status);
    EF_CUDA(cudaGetLastError());
    int st = 0;
    EF_CUDA(cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    EF_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    if (st & ST_RANGE) return EF_ERR_RANGE;
    if (st & ST_REPEAT) return EF_ERR_ARG;
    return EF_OK;
}

}  // namespace ef
