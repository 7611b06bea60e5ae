// Fused assembly: one kernel, one CTA per block of BE elements; the blocks
// follow an element order -- the mesh's own order (ef_plan_set_block) or a
// Morton curve of the element centroids (ef_plan_set_fused), which keeps a
// block compact in space so that most nonzeros are completed inside it.
//
// Phase 1: thread t computes the signed local K and M of the block's t-th
//   element (closed forms of ef_element.cuh) and puts each value into shared
//   memory at its place in the block's slot order (a plan-time map), so that
//   the contributions of every slot lie contiguous there.
// Phase 2: the CTA walks the block's "slots", the upper nonzeros its elements
//   touch, each with the block's contributions to it listed in the order of
//   the plan's global contribution list (ascending element id within a
//   nonzero):
//   - complete slot (every contribution of the nonzero lies in this block):
//     summed in that order and written to (r, c) and (c, r) of K and M;
//   - partial slot (the nonzero is split across blocks): the raw
//     contributions are written to their positions in the global list.
// Phase 3: for every split nonzero the CTA has contributed to, it takes an
//   integer ticket; the CTA that draws the last one (the nonzero's count of
//   contributing blocks) sums the nonzero's whole list in order and writes
//   it. Nothing waits: a CTA that is not last simply moves on. Writers fence
//   their list entries before taking the ticket, the last CTA fences after
//   it and reads the list through L2 (the pattern of a last-block
//   reduction). The finisher resets the ticket for the next call.
// Every nonzero is therefore the same left-to-right sum as in the two-pass
// path, bit for bit, whatever the order and block size. No floating-point
// atomics; only the split nonzeros' contributions reach global memory.
//
// Schedule (built once per plan and order on the GPU): the contribution list
// is stably re-sorted by (block, split flag), slot heads are where the
// nonzero changes, and each slot stores (start | count << 16) plus two words:
// the CSR positions of (r,c) and (c,r) for a complete slot, the split index
// for a partial one. Within a block the complete slots come first, in
// ascending (r, c), then the partial ones.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ef_assemble.cuh"
#include "ef_internal.cuh"

namespace ef {
namespace {

constexpr int TPB = 256;
constexpr uint32_t NONE = 0xffffffffu;
constexpr size_t SMEM_LIMIT = 227 * 1024;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

// ---- element order: Morton curve of the centroids ---------------------------

// Order-preserving map of a double to uint64 (for atomic min / max).
__device__ __forceinline__ unsigned long long ordered_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

inline double from_ordered(unsigned long long o)
{
    const unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// Bounding box of the nodes: lohi[c] = min, lohi[dim + c] = max (ordered bits).
__global__ void k_bbox(const double* __restrict__ nodes, int64_t V, int dim, unsigned long long* lohi)
{
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < dim; c++) {
            const double x = nodes[v * dim + c];
            lo[c] = fmin(lo[c], x);
            hi[c] = fmax(hi[c], x);
        }
    for (int c = 0; c < dim; c++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(lohi + c, ordered_bits(lo[c]));
            atomicMax(lohi + dim + c, ordered_bits(hi[c]));
        }
    }
}

// 21 bits spread to every third bit (3D), 31 bits to every other bit (2D).
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint64_t spread2(uint32_t v)
{
    uint64_t x = v & 0x7fffffffu;
    x = (x | x << 16) & 0x0000ffff0000ffffull;
    x = (x | x << 8) & 0x00ff00ff00ff00ffull;
    x = (x | x << 4) & 0x0f0f0f0f0f0f0f0full;
    x = (x | x << 2) & 0x3333333333333333ull;
    x = (x | x << 1) & 0x5555555555555555ull;
    return x;
}

// Morton key of each element's centroid, quantised to 21 (3D) or 31 (2D)
// bits per coordinate over the bounding box.
__global__ void k_morton_keys(const int32_t* __restrict__ elems, const double* __restrict__ nodes, int64_t T, int dim,
                              double lo0, double lo1, double lo2, double sc0, double sc1, double sc2, uint64_t* keys,
                              uint32_t* vals)
{
    const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (e >= T) return;
    const int nv = dim + 1;
    const double lo[3] = {lo0, lo1, lo2}, sc[3] = {sc0, sc1, sc2};
    const uint32_t qmax = dim == 3 ? 0x1fffffu : 0x7fffffffu;
    uint64_t key = 0;
    for (int c = 0; c < dim; c++) {
        double x = 0;
        for (int a = 0; a < nv; a++) x += nodes[(int64_t)elems[e * nv + a] * dim + c];
        double q = floor((x / nv - lo[c]) * sc[c]);
        q = q < 0 ? 0 : (q > qmax ? qmax : q);
        key |= (dim == 3 ? spread3((uint32_t)q) : spread2((uint32_t)q)) << c;
    }
    keys[e] = key;
    vals[e] = (uint32_t)e;
}

__global__ void k_rank(const uint32_t* __restrict__ order, int64_t T, uint32_t* rank)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < T) rank[order[i]] = (uint32_t)i;
}

// ---- schedule ------------------------------------------------------------------

__device__ __forceinline__ uint32_t block_of(uint32_t v, int64_t T, int BE, const uint32_t* rank)
{
    const uint32_t e = (uint32_t)(v % T);
    return (rank ? rank[e] : e) / (uint32_t)BE;
}

// Per upper nonzero: its contributions' owner (uos), whether they all lie in
// one block, and how many distinct blocks they come from.
__global__ void k_nonzero_blocks(const uint32_t* seg, const uint32_t* perm, int64_t U, int64_t T, int BE,
                                 const uint32_t* rank, uint32_t* uos, uint8_t* complete, uint32_t* nblk)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    const uint32_t s0 = seg[u], s1 = seg[u + 1];
    uint32_t distinct = 0;
    for (uint32_t s = s0; s < s1; s++) {
        uos[s] = (uint32_t)u;
        const uint32_t b = block_of(perm[s], T, BE, rank);
        bool seen = false;
        for (uint32_t r = s0; r < s && !seen; r++) seen = block_of(perm[r], T, BE, rank) == b;
        distinct += seen ? 0u : 1u;
    }
    complete[u] = distinct == 1;
    nblk[u] = distinct;
}

__global__ void k_block_keys(const uint32_t* perm, const uint32_t* uos, const uint8_t* complete, int64_t n,
                             int64_t T, int BE, const uint32_t* rank, uint64_t* keys, uint32_t* vals)
{
    const int64_t s = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (s >= n) return;
    keys[s] = ((uint64_t)block_of(perm[s], T, BE, rank) << 1) | (complete[uos[s]] ? 0u : 1u);
    vals[s] = (uint32_t)s;
}

__global__ void k_slot_heads(const uint64_t* keys, const uint32_t* bsorted, const uint32_t* uos, int64_t n,
                             uint32_t* flag)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || keys[i] != keys[i - 1] || uos[bsorted[i]] != uos[bsorted[i - 1]]) ? 1u : 0u;
}

__global__ void k_slot_start(const uint32_t* flag, const uint32_t* ex, int64_t n, uint32_t* sstart)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < n && flag[i]) sstart[ex[i]] = (uint32_t)i;
}

__global__ void k_split_flags(const uint8_t* complete, int64_t U, uint32_t* flag)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u < U) flag[u] = complete[u] ? 0u : 1u;
}

__global__ void k_split_list(const uint32_t* flag, const uint32_t* ex, const uint32_t* nblk, int64_t U, uint32_t* px,
                             uint32_t* px_nb)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u < U && flag[u]) {
        px[ex[u]] = (uint32_t)u;
        px_nb[ex[u]] = nblk[u];
    }
}

__global__ void k_slots(const uint64_t* keys, const uint32_t* bsorted, const uint32_t* uos, const uint32_t* sstart,
                        int64_t nslots, int64_t n, int64_t per_block, const uint32_t* pos_up, const uint32_t* pos_lo,
                        const uint32_t* xidx, uint32_t* sinfo, uint32_t* posA, uint32_t* posB, uint32_t* slot_off,
                        uint32_t* part_off)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= nslots) return;
    const int64_t i = sstart[j];
    const int64_t next = (j + 1 < nslots) ? (int64_t)sstart[j + 1] : n;
    const uint64_t key = keys[i];
    const int64_t b = (int64_t)(key >> 1);
    const uint32_t partial = (uint32_t)(key & 1u);
    const uint32_t u = uos[bsorted[i]];
    sinfo[j] = (uint32_t)(i - b * per_block) | ((uint32_t)(next - i) << 16);
    posA[j] = partial ? xidx[u] : pos_up[u];
    posB[j] = partial ? NONE : pos_lo[u];
    if (i == b * per_block) slot_off[b] = (uint32_t)j;
    if (partial && (i == b * per_block || keys[i - 1] != key)) part_off[b] = (uint32_t)j;
}

// Blocks without partial slots: their partial range starts at the next block.
__global__ void k_part_fix(const uint32_t* slot_off, int64_t nblocks, uint32_t* part_off)
{
    const int64_t b = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (b < nblocks && part_off[b] == NONE) part_off[b] = slot_off[b + 1];
}

// Per contribution i of the block-sorted list (block b, slot order): its
// pair q and element r of the block give sidx[b][q][r] = i - b per_block, the
// place where the element's thread puts that value in shared memory, so that
// every slot's contributions lie contiguous and in list order there.
__global__ void k_slot_places(const uint64_t* keys, const uint32_t* bsorted, const uint32_t* perm, int64_t n, int64_t T,
                       int BE, int64_t per_block, const uint32_t* rank, uint16_t* sidx, uint32_t* gpos,
                       unsigned long long* n_partial)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool part = i < n && (keys[i] & 1u);
    const unsigned m = __ballot_sync(0xffffffffu, part);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(n_partial, (unsigned long long)__popc(m));
    if (i >= n) return;
    const uint32_t s = bsorted[i];
    const uint32_t v = perm[s];
    const int64_t q = v / T, e = v % T;
    const int64_t b = i / per_block;
    const int64_t r = rank ? (int64_t)rank[e] : e;
    sidx[b * per_block + q * BE + (r - b * BE)] = (uint16_t)(i - b * per_block);
    gpos[i] = s;
}

// ---- assembly ---------------------------------------------------------------------

// CTAs per SM that shared memory allows (local matrices of the block plus its
// ticket queue): the register budget the compiler is held to
template <int VAR, int BE>
constexpr int fused_min_blocks()
{
    return VAR == NED3 ? (BE == 128 ? 4 : 2) : (VAR == RT3 ? (BE == 128 ? 8 : 5) : (BE == 128 ? 12 : 6));
}

// Products on the integer pipes, except for 3D RT0, where the registers they
// need cost this kernel more occupancy than they save FP64 work (measured at
// 128^3: 2.62 against 2.59 ms per call)
template <int VAR>
constexpr bool fused_int_mul()
{
    return VAR != RT3;
}

// Additions as FMAs with per-thread constants (full FP64 rate) in the 3D
// kernels; the 2D ones, held to 40 registers, keep plain additions (the
// per-thread constants cost them spills: level-11 L-shape 2.19 / 2.26 ms
// against 2.18 / 2.23 ms)
template <int VAR>
constexpr bool fused_reg_const()
{
    return VAR == NED3 || VAR == RT3;
}

template <int VAR, int BE>
__global__ void __launch_bounds__(BE, (fused_min_blocks<VAR, BE>())) k_fused(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                              const double* __restrict__ coeff, int64_t T,
                                              const uint32_t* __restrict__ order, const uint16_t* __restrict__ sidx,
                                              const uint32_t* __restrict__ gpos,
                                              const uint32_t* __restrict__ slot_off,
                                              const uint32_t* __restrict__ part_off,
                                              const uint32_t* __restrict__ sinfo, const uint32_t* __restrict__ posA,
                                              const uint32_t* __restrict__ posB, const uint32_t* __restrict__ seg,
                                              const uint32_t* __restrict__ pos_up,
                                              const uint32_t* __restrict__ pos_lo, const uint32_t* __restrict__ px,
                                              const uint32_t* __restrict__ px_nb, uint32_t* __restrict__ px_cnt,
                                              double* __restrict__ K, double* __restrict__ M, double* partK,
                                              double* partM, int* status)
{
    using E = ElemTraits<VAR>;
    extern __shared__ double sm[];
    double* smK = sm;
    double* smM = sm + E::NP * BE;
    uint32_t* s_queue = reinterpret_cast<uint32_t*>(sm + 2 * E::NP * BE);
    __shared__ uint32_t s_qn;
    const int t = threadIdx.x;
    const int64_t b = blockIdx.x;
    if (t == 0) s_qn = 0;
    // the block's slot ranges and this thread's first complete slot, loaded
    // before the FP64 work so that they arrive while it runs
    const uint32_t j0 = __ldg(slot_off + b), jp = __ldg(part_off + b), j1 = __ldg(slot_off + b + 1);
    uint32_t j = j0 + t, info_n = 0, pa_n = 0, pb_n = 0;
    if (j < jp) {
        info_n = __ldg(sinfo + j);
        pa_n = __ldg(posA + j);
        pb_n = __ldg(posB + j);
    }
    const int64_t i = b * BE + t;
    if (i < T) {
        const int64_t e = order ? (int64_t)__ldg(order + i) : i;
        // where each of this element's contributions goes (slot order),
        // loaded before the FP64 work (coalesced over the block's threads)
        const uint16_t* si = sidx + b * (int64_t)(BE * E::NP) + t;
        uint16_t pos[E::NP];
#pragma unroll
        for (int q = 0; q < E::NP; q++) pos[q] = __ldg(si + q * BE);
        double Kq[E::NP], Mq[E::NP];
        if (compute_element<VAR, fused_int_mul<VAR>(), fused_reg_const<VAR>()>(elems, nodes, coeff, coeff, e, Kq, Mq))
            atomicOr(status, ST_DEGENERATE);
#pragma unroll
        for (int q = 0; q < E::NP; q++) {
            smK[pos[q]] = Kq[q];
            smM[pos[q]] = Mq[q];
        }
    }
    __syncthreads();
    const uint32_t* g = gpos + b * (int64_t)(BE * E::NP);
    // complete slots: sum in list order, store both triangles; the next
    // slot's metadata is loaded one iteration ahead
    for (; j < jp; j += BE) {
        const uint32_t info = info_n, pa = pa_n, pb = pb_n;
        if (j + BE < jp) {
            info_n = __ldg(sinfo + j + BE);
            pa_n = __ldg(posA + j + BE);
            pb_n = __ldg(posB + j + BE);
        }
        const uint32_t start = info & 0xffffu, cnt = info >> 16;
        double k = smK[start], m = smM[start];
        for (uint32_t r = 1; r < cnt; r++) {
            k += smK[start + r];
            m += smM[start + r];
        }
        K[pa] = k;
        M[pa] = m;
        if (pb != NONE) {
            K[pb] = k;
            M[pb] = m;
        }
    }
    // partial slots: raw contributions to their places in the global list
    for (uint32_t j = jp + t; j < j1; j += BE) {
        const uint32_t info = __ldg(sinfo + j);
        const uint32_t start = info & 0xffffu, cnt = info >> 16;
        for (uint32_t r = 0; r < cnt; r++) {
            const uint32_t s = __ldg(g + start + r);
            partK[s] = smK[start + r];
            partM[s] = smM[start + r];
        }
    }
    __threadfence();
    __syncthreads();
    // tickets: the block that completes a split nonzero's contributions sums it
    for (uint32_t j = jp + t; j < j1; j += BE) {
        const uint32_t x = __ldg(posA + j);
        if (atomicAdd(px_cnt + x, 1u) + 1u == __ldg(px_nb + x)) s_queue[atomicAdd(&s_qn, 1u)] = x;
    }
    __threadfence();
    __syncthreads();
    const uint32_t nq = s_qn;
    for (uint32_t k2 = t; k2 < nq; k2 += BE) {
        const uint32_t x = s_queue[k2];
        px_cnt[x] = 0;   // every ticket of this call is drawn: ready for the next call
        const uint32_t u = __ldg(px + x);
        const uint32_t s0 = __ldg(seg + u), s1 = __ldg(seg + u + 1);
        double k = __ldcg(partK + s0), m = __ldcg(partM + s0);
        for (uint32_t s = s0 + 1; s < s1; s++) {
            k += __ldcg(partK + s);
            m += __ldcg(partM + s);
        }
        uint32_t p = __ldg(pos_up + u);
        K[p] = k;
        M[p] = m;
        p = __ldg(pos_lo + u);
        if (p != NONE) {
            K[p] = k;
            M[p] = m;
        }
    }
}

template <int VAR, int BE>
size_t smem_bytes(const ef_plan* p)
{
    return (size_t)2 * ElemTraits<VAR>::NP * BE * sizeof(double) + (size_t)p->fb_qcap * 4;
}

template <int VAR, int BE>
int launch_fused_t(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s)
{
    const size_t smem = smem_bytes<VAR, BE>(p);
    static size_t configured = 0;   // per instance: the dynamic shared memory limit raised so far
    if (smem > configured) {
        EF_CUDA(cudaFuncSetAttribute(k_fused<VAR, BE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = smem;
    }
    double* partK = p->d_local;
    double* partM = p->d_local + (int64_t)p->np * p->T;
    k_fused<VAR, BE><<<(unsigned)p->fb_nblocks, BE, smem, s>>>(
        p->d_elems, nodes, coeff, p->T, p->d_fb_order, p->d_fb_sidx, p->d_fb_gpos, p->d_fb_slot_off,
        p->d_fb_part_off, p->d_fb_sinfo, p->d_fb_posA, p->d_fb_posB, p->d_seg, p->d_pos_up, p->d_pos_lo, p->d_px_uid,
        p->d_px_nb, p->d_px_cnt, K, M, partK, partM, p->d_status);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

template <int BE>
int launch_variant(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s)
{
    switch (p->variant) {
        case RT2: return launch_fused_t<RT2, BE>(p, nodes, coeff, K, M, s);
        case NED2: return launch_fused_t<NED2, BE>(p, nodes, coeff, K, M, s);
        case RT3: return launch_fused_t<RT3, BE>(p, nodes, coeff, K, M, s);
        default: return launch_fused_t<NED3, BE>(p, nodes, coeff, K, M, s);
    }
}

size_t smem_needed(const ef_plan* p, int BE)
{
    return (size_t)2 * p->np * BE * sizeof(double) + (size_t)p->fb_qcap * 4;
}

void free_fused(ef_plan* p)
{
    void* ptrs[] = {p->d_fb_slot_off, p->d_fb_part_off, p->d_fb_sinfo, p->d_fb_sidx, p->d_fb_gpos,
                    p->d_fb_posA,     p->d_fb_posB,     p->d_px_uid,   p->d_px_nb,   p->d_px_cnt,
                    p->d_fb_order};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    p->d_fb_slot_off = p->d_fb_part_off = p->d_fb_sinfo = p->d_fb_posA = p->d_fb_posB = nullptr;
    p->d_px_uid = p->d_px_nb = p->d_px_cnt = p->d_fb_gpos = p->d_fb_order = nullptr;
    p->d_fb_sidx = nullptr;
    p->fb_block = 0;
    p->fb_nblocks = 0;
    p->fb_nslots = 0;
    p->fb_qcap = 0;
    p->fb_sfc = 0;
    p->n_px = 0;
    p->n_partial = 0;
}

// Element order along the Morton curve of the centroids of the elements
// under coordinates `nodes`: order[i] = the i-th element (device, T entries).
int morton_order(const ef_plan* p, const double* nodes, uint32_t* order, cudaStream_t s)
{
    const int64_t T = p->T;
    const int dim = p->dim;
    unsigned long long* lohi = nullptr;
    uint64_t* keys = nullptr;
    void* tmp = nullptr;
    int st = EF_OK;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMalloc((void**)&lohi, 6 * 8)) || !ok(cudaMalloc((void**)&keys, (size_t)T * 8)) ||
        !ok(cudaMalloc(&tmp, radix_tmp_bytes(T))))
        st = EF_ERR_OOM;
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    if (st == EF_OK) {
        unsigned long long init[6];
        for (int c = 0; c < dim; c++) {
            init[c] = ~0ull;
            init[dim + c] = 0ull;
        }
        if (!ok(cudaMemcpyAsync(lohi, init, sizeof(unsigned long long) * 2 * dim, cudaMemcpyHostToDevice, s)))
            st = EF_ERR_CUDA;
        if (st == EF_OK && p->V > 0) {
            const int64_t gb = (p->V + TPB - 1) / TPB;
            k_bbox<<<(unsigned)(gb < 4096 ? gb : 4096), TPB, 0, s>>>(nodes, p->V, dim, lohi);
        }
        if (st == EF_OK && (!ok(cudaMemcpyAsync(h, lohi, sizeof(unsigned long long) * 2 * dim, cudaMemcpyDeviceToHost,
                                                s)) ||
                            !ok(cudaStreamSynchronize(s))))
            st = EF_ERR_CUDA;
    }
    if (st == EF_OK) {
        double lo[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
        const double qn = dim == 3 ? 2097152.0 : 2147483648.0;   // 2^21, 2^31
        for (int c = 0; c < dim; c++) {
            lo[c] = from_ordered(h[c]);
            const double ext = from_ordered(h[dim + c]) - lo[c];
            sc[c] = ext > 0 ? qn / ext : 0.0;
        }
        k_morton_keys<<<grid_for(T), TPB, 0, s>>>(p->d_elems, nodes, T, dim, lo[0], lo[1], lo[2], sc[0], sc[1], sc[2],
                                                  keys, order);
        st = radix_sort_pairs(keys, order, T, dim == 3 ? 63 : 62, tmp, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == EF_OK && e == cudaSuccess) e = cudaGetLastError();
    if (st == EF_OK && e != cudaSuccess) {
        set_last_error("morton_order", e);
        st = EF_ERR_CUDA;
    }
    cudaFree(lohi);
    cudaFree(keys);
    cudaFree(tmp);
    return st;
}

}  // namespace

bool fused_block_supported(int BE) { return BE == 128 || BE == 256; }

// Build the fused schedule for blocks of BE elements along the mesh's own
// order (nodes == NULL) or the Morton order of the centroids under `nodes`.
int build_fused_block(ef_plan* p, int BE, const double* nodes, cudaStream_t s)
{
    free_fused(p);
    if (p->T == 0) return EF_OK;
    if (!fused_block_supported(BE)) return EF_ERR_ARG;
    const int64_t T = p->T, n = T * p->np, U = p->U, per_block = (int64_t)BE * p->np;
    const int64_t nblocks = (T + BE - 1) / BE;
    if (per_block > 65535) return EF_ERR_ARG;

    int st = EF_OK;
    uint32_t *uos = nullptr, *flag = nullptr, *ex = nullptr, *bsorted = nullptr, *sstart = nullptr, *nblk = nullptr;
    uint32_t* rank = nullptr;
    uint8_t* complete = nullptr;
    uint64_t* keys = nullptr;
    unsigned long long* npart = nullptr;
    void* tmp = nullptr;
    size_t tb = radix_tmp_bytes(n);
    if (scan_tmp_bytes(n) > tb) tb = scan_tmp_bytes(n);
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMalloc((void**)&uos, n * 4)) || !ok(cudaMalloc((void**)&complete, U > 0 ? U : 1)) ||
        !ok(cudaMalloc((void**)&nblk, (U > 0 ? U : 1) * 4)) || !ok(cudaMalloc((void**)&keys, n * 8)) ||
        !ok(cudaMalloc((void**)&bsorted, n * 4)) || !ok(cudaMalloc((void**)&flag, n * 4)) ||
        !ok(cudaMalloc((void**)&ex, n * 4 + 4)) || !ok(cudaMalloc(&tmp, tb)) ||
        !ok(cudaMalloc((void**)&npart, 8)))
        st = EF_ERR_OOM;
    do {
        if (st) break;
        if (nodes) {
            if (!ok(cudaMalloc((void**)&p->d_fb_order, T * 4)) || !ok(cudaMalloc((void**)&rank, T * 4))) {
                st = EF_ERR_OOM;
                break;
            }
            if ((st = morton_order(p, nodes, p->d_fb_order, s))) break;
            k_rank<<<grid_for(T), TPB, 0, s>>>(p->d_fb_order, T, rank);
        }
        k_nonzero_blocks<<<grid_for(U), TPB, 0, s>>>(p->d_seg, p->d_perm, U, T, BE, rank, uos, complete, nblk);
        k_block_keys<<<grid_for(n), TPB, 0, s>>>(p->d_perm, uos, complete, n, T, BE, rank, keys, bsorted);
        if ((st = radix_sort_pairs(keys, bsorted, n, bits_for(((uint64_t)(nblocks - 1) << 1) | 1u), tmp, s))) break;
        k_slot_heads<<<grid_for(n), TPB, 0, s>>>(keys, bsorted, uos, n, flag);
        if ((st = exclusive_scan_u32(flag, ex, n, true, tmp, s))) break;
        uint32_t nslots = 0;
        if (!ok(cudaMemcpyAsync(&nslots, ex + n, 4, cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s))) {
            st = EF_ERR_CUDA;
            break;
        }
        if (!ok(cudaMalloc((void**)&sstart, (size_t)nslots * 4)) ||
            !ok(cudaMalloc((void**)&p->d_fb_sinfo, (size_t)nslots * 4)) ||
            !ok(cudaMalloc((void**)&p->d_fb_posA, (size_t)nslots * 4)) ||
            !ok(cudaMalloc((void**)&p->d_fb_posB, (size_t)nslots * 4)) ||
            !ok(cudaMalloc((void**)&p->d_fb_slot_off, (size_t)(nblocks + 1) * 4)) ||
            !ok(cudaMalloc((void**)&p->d_fb_part_off, (size_t)nblocks * 4)) ||
            !ok(cudaMalloc((void**)&p->d_fb_sidx, (size_t)nblocks * per_block * 2)) ||   // [block][pair][element]
            !ok(cudaMalloc((void**)&p->d_fb_gpos, (size_t)n * 4))) {
            st = EF_ERR_OOM;
            break;
        }
        k_slot_start<<<grid_for(n), TPB, 0, s>>>(flag, ex, n, sstart);
        // split nonzeros: compact index, their contributing-block counts, tickets
        k_split_flags<<<grid_for(U), TPB, 0, s>>>(complete, U, flag);
        if ((st = exclusive_scan_u32(flag, ex, U, true, tmp, s))) break;
        uint32_t npx = 0;
        if (!ok(cudaMemcpyAsync(&npx, ex + U, 4, cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s))) {
            st = EF_ERR_CUDA;
            break;
        }
        const size_t pxn = (size_t)(npx > 0 ? npx : 1);
        if (!ok(cudaMalloc((void**)&p->d_px_uid, pxn * 4)) || !ok(cudaMalloc((void**)&p->d_px_nb, pxn * 4)) ||
            !ok(cudaMalloc((void**)&p->d_px_cnt, pxn * 4))) {
            st = EF_ERR_OOM;
            break;
        }
        k_split_list<<<grid_for(U), TPB, 0, s>>>(flag, ex, nblk, U, p->d_px_uid, p->d_px_nb);
        cudaMemsetAsync(p->d_px_cnt, 0, pxn * 4, s);
        cudaMemsetAsync(p->d_fb_part_off, 0xff, (size_t)nblocks * 4, s);
        k_slots<<<grid_for(nslots), TPB, 0, s>>>(keys, bsorted, uos, sstart, nslots, n, per_block, p->d_pos_up,
                                                 p->d_pos_lo, ex, p->d_fb_sinfo, p->d_fb_posA, p->d_fb_posB,
                                                 p->d_fb_slot_off, p->d_fb_part_off);
        if (!ok(cudaMemcpyAsync(p->d_fb_slot_off + nblocks, &nslots, 4, cudaMemcpyHostToDevice, s))) {
            st = EF_ERR_CUDA;
            break;
        }
        k_part_fix<<<grid_for(nblocks), TPB, 0, s>>>(p->d_fb_slot_off, nblocks, p->d_fb_part_off);
        cudaMemsetAsync(npart, 0, 8, s);
        k_slot_places<<<grid_for(n), TPB, 0, s>>>(keys, bsorted, p->d_perm, n, T, BE, per_block, rank, p->d_fb_sidx,
                                           p->d_fb_gpos, npart);
        // the largest number of partial slots of a block bounds its ticket queue
        std::vector<uint32_t> so((size_t)nblocks + 1), po((size_t)nblocks);
        unsigned long long hpart = 0;
        if (!ok(cudaMemcpyAsync(so.data(), p->d_fb_slot_off, so.size() * 4, cudaMemcpyDeviceToHost, s)) ||
            !ok(cudaMemcpyAsync(po.data(), p->d_fb_part_off, po.size() * 4, cudaMemcpyDeviceToHost, s)) ||
            !ok(cudaMemcpyAsync(&hpart, npart, 8, cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s))) {
            st = EF_ERR_CUDA;
            break;
        }
        uint32_t qcap = 1;
        for (int64_t b = 0; b < nblocks; b++)
            if (so[b + 1] - po[b] > qcap) qcap = so[b + 1] - po[b];
        p->fb_block = BE;
        p->fb_nblocks = nblocks;
        p->fb_nslots = nslots;
        p->fb_qcap = (int)qcap;
        p->fb_sfc = nodes ? 1 : 0;
        p->n_px = npx;
        p->n_partial = (int64_t)hpart;
        if (smem_needed(p, BE) > SMEM_LIMIT) st = EF_ERR_SIZE;
    } while (0);
    cudaError_t e = cudaGetLastError();
    if (st == EF_OK && e != cudaSuccess) {
        set_last_error("build_fused", e);
        st = EF_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    cudaFree(uos);
    cudaFree(complete);
    cudaFree(nblk);
    cudaFree(keys);
    cudaFree(bsorted);
    cudaFree(flag);
    cudaFree(ex);
    cudaFree(sstart);
    cudaFree(rank);
    cudaFree(npart);
    cudaFree(tmp);
    if (st != EF_OK) free_fused(p);
    return st;
}

void release_fused(ef_plan* p) { free_fused(p); }

int launch_fused(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s)
{
    if (p->T == 0) return EF_OK;
    if (p->fb_block == 128) return launch_variant<128>(p, nodes, coeff, K, M, s);
    return launch_variant<256>(p, nodes, coeff, K, M, s);
}

}  // namespace ef
