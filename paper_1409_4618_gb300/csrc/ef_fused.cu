// Fused assembly: one CTA per block of BE consecutive elements.
//
// Phase 1: thread t computes the signed local K and M of element b*BE + t
// (closed forms of ef_element.cuh) into shared memory, pair-major.
// Phase 2: the CTA walks the block's "slots": the upper nonzeros its elements
// touch, each with the block's contributions to it in the order of the
// plan's global contribution list (ascending element id within a nonzero).
//   - complete slot (every contribution of the nonzero lies in this block):
//     summed in that order and written to (r, c) and (c, r) of K and M;
//   - partial slot: the raw contributions are written to their global
//     positions in the plan scratch, and a fix-up kernel sums each split
//     nonzero over its whole contribution list in the same order.
// Every nonzero is therefore the same left-to-right sum as in the two-pass
// path, bit for bit, whatever the block size. Local matrices never reach
// HBM except for split nonzeros. No floating-point atomics.
//
// Schedule (built once per plan on the GPU): the global contribution list is
// stably re-sorted by block, slot heads are where the nonzero changes, and
// each slot stores (start | count << 16 | partial << 31) plus two output
// positions (CSR positions of (r,c) and (c,r), or the global list position of
// its first contribution when partial).
#include "ef_assemble.cuh"
#include "ef_internal.cuh"

namespace ef {
namespace {

constexpr int TPB = 256;
constexpr uint32_t NONE = 0xffffffffu;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

// ---- schedule construction ----------------------------------------------------

__global__ void k_u_of_s(const uint32_t* seg, const uint32_t* perm, int64_t U, int64_t T, int BE, uint32_t* uos,
                         uint8_t* complete)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    const uint32_t s0 = seg[u], s1 = seg[u + 1];
    for (uint32_t s = s0; s < s1; s++) uos[s] = (uint32_t)u;
    const int64_t e0 = perm[s0] % T, e1 = perm[s1 - 1] % T;
    complete[u] = (e0 / BE) == (e1 / BE);
}

__global__ void k_block_keys(const uint32_t* perm, int64_t n, int64_t T, int BE, uint64_t* keys, uint32_t* vals)
{
    const int64_t s = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (s >= n) return;
    keys[s] = (uint64_t)((perm[s] % T) / BE);
    vals[s] = (uint32_t)s;
}

__global__ void k_slot_heads(const uint32_t* bsorted, const uint32_t* uos, int64_t n, int64_t per_block,
                             uint32_t* flag)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i % per_block == 0 || uos[bsorted[i]] != uos[bsorted[i - 1]]) ? 1u : 0u;
}

__global__ void k_slot_start(const uint32_t* flag, const uint32_t* ex, int64_t n, uint32_t* sstart)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < n && flag[i]) sstart[ex[i]] = (uint32_t)i;
}

__global__ void k_slots(const uint32_t* bsorted, const uint32_t* uos, const uint8_t* complete, const uint32_t* sstart,
                        int64_t nslots, int64_t n, int64_t per_block, const uint32_t* pos_up, const uint32_t* pos_lo,
                        uint32_t* sinfo, uint32_t* posA, uint32_t* posB, uint32_t* slot_off)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= nslots) return;
    const int64_t i = sstart[j];
    const int64_t next = (j + 1 < nslots) ? (int64_t)sstart[j + 1] : n;
    const int64_t b = i / per_block;
    const uint32_t start = (uint32_t)(i - b * per_block);
    const uint32_t count = (uint32_t)(next - i);
    const uint32_t s = bsorted[i];
    const uint32_t u = uos[s];
    const uint32_t partial = complete[u] ? 0u : 1u;
    sinfo[j] = start | (count << 16) | (partial << 31);
    posA[j] = partial ? s : pos_up[u];
    posB[j] = partial ? NONE : pos_lo[u];
    if (i % per_block == 0) slot_off[b] = (uint32_t)j;
}

__global__ void k_cidx(const uint32_t* bsorted, const uint32_t* perm, int64_t n, int64_t T, int BE, int64_t per_block,
                       uint16_t* cidx)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = perm[bsorted[i]];
    const int64_t q = v / T, e = v % T;
    const int64_t b = i / per_block;
    cidx[i] = (uint16_t)(q * BE + (e - b * BE));
}

__global__ void k_px_flags(const uint8_t* complete, int64_t U, uint32_t* flag)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u < U) flag[u] = complete[u] ? 0u : 1u;
}

__global__ void k_px_list(const uint32_t* flag, const uint32_t* ex, int64_t U, uint32_t* px)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u < U && flag[u]) px[ex[u]] = (uint32_t)u;
}

// ---- assembly -------------------------------------------------------------------


__global__ void k_slot_order_keys(const uint32_t* sstart, const uint32_t* sinfo, int64_t nslots, int64_t per_block,
                                  uint64_t* keys, uint32_t* vals)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= nslots) return;
    const uint64_t b = (uint64_t)(sstart[j] / per_block);
    const uint32_t cnt = (sinfo[j] >> 16) & 0x7fffu;
    keys[j] = (b << 15) | (uint64_t)(0x7fffu - cnt);
    vals[j] = (uint32_t)j;
}

__global__ void k_gather3(const uint32_t* order, int64_t n, const uint32_t* a, const uint32_t* b, const uint32_t* c,
                          uint32_t* ao, uint32_t* bo, uint32_t* co)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= n) return;
    const uint32_t o = order[j];
    ao[j] = a[o];
    bo[j] = b[o];
    co[j] = c[o];
}

// keys / vals / tmp: scratch of at least nslots entries (radix_tmp_bytes(nslots) for tmp).
int order_slots_by_count(ef_plan* p, int64_t nslots, int64_t nblocks, int64_t per_block, uint64_t* keys,
                         uint32_t* vals, void* tmp, cudaStream_t s, const uint32_t* sstart)
{
    if (nslots <= 1) return EF_OK;
    k_slot_order_keys<<<grid_for(nslots), TPB, 0, s>>>(sstart, p->d_fb_sinfo, nslots, per_block, keys, vals);
    EF_TRY(radix_sort_pairs(keys, vals, nslots, bits_for(((uint64_t)nblocks << 15) | 0x7fffu), tmp, s));
    uint32_t *a = nullptr, *b = nullptr, *c = nullptr;
    if (cudaMalloc((void**)&a, nslots * 4) != cudaSuccess || cudaMalloc((void**)&b, nslots * 4) != cudaSuccess ||
        cudaMalloc((void**)&c, nslots * 4) != cudaSuccess) {
        cudaFree(a);
        cudaFree(b);
        return EF_ERR_OOM;
    }
    k_gather3<<<grid_for(nslots), TPB, 0, s>>>(vals, nslots, p->d_fb_sinfo, p->d_fb_posA, p->d_fb_posB, a, b, c);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(p->d_fb_sinfo);
    cudaFree(p->d_fb_posA);
    cudaFree(p->d_fb_posB);
    p->d_fb_sinfo = a;
    p->d_fb_posA = b;
    p->d_fb_posB = c;
    if (e != cudaSuccess) {
        set_last_error("order_slots_by_count", e);
        return EF_ERR_CUDA;
    }
    return EF_OK;
}

template <int VAR, int BE>
__global__ void __launch_bounds__(BE) k_fused(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                              const double* __restrict__ coeff, int64_t T,
                                              const uint16_t* __restrict__ cidx, const uint32_t* __restrict__ slot_off,
                                              const uint32_t* __restrict__ sinfo, const uint32_t* __restrict__ posA,
                                              const uint32_t* __restrict__ posB, double* __restrict__ K,
                                              double* __restrict__ M, double* __restrict__ partK,
                                              double* __restrict__ partM, int* status)
{
    using E = ElemTraits<VAR>;
    extern __shared__ double sm[];
    double* smK = sm;
    double* smM = sm + E::NP * BE;
    const int64_t b = blockIdx.x;
    const int64_t e = b * BE + threadIdx.x;
    if (e < T) {
        double Kq[E::NP], Mq[E::NP];
        const double sigma = coeff ? __ldg(coeff + e) : 1.0;
        if (compute_element<VAR>(elems, nodes, sigma, sigma, e, Kq, Mq)) atomicOr(status, ST_DEGENERATE);
#pragma unroll
        for (int q = 0; q < E::NP; q++) {
            smK[q * BE + threadIdx.x] = Kq[q];
            smM[q * BE + threadIdx.x] = Mq[q];
        }
    }
    __syncthreads();
    const uint16_t* c = cidx + b * (int64_t)(BE * E::NP);
    const uint32_t j1 = slot_off[b + 1];
    for (uint32_t j = slot_off[b] + threadIdx.x; j < j1; j += BE) {
        const uint32_t info = __ldg(sinfo + j);
        const uint32_t start = info & 0xffffu, cnt = (info >> 16) & 0x7fffu;
        const uint32_t pa = __ldg(posA + j);
        if (!(info >> 31)) {
            uint32_t idx = c[start];
            double k = smK[idx], m = smM[idx];
            for (uint32_t t = 1; t < cnt; t++) {
                idx = c[start + t];
                k += smK[idx];
                m += smM[idx];
            }
            K[pa] = k;
            M[pa] = m;
            const uint32_t pb = __ldg(posB + j);
            if (pb != NONE) {
                K[pb] = k;
                M[pb] = m;
            }
        } else {
            for (uint32_t t = 0; t < cnt; t++) {
                const uint32_t idx = c[start + t];
                partK[pa + t] = smK[idx];
                partM[pa + t] = smM[idx];
            }
        }
    }
}

__global__ void __launch_bounds__(TPB) k_fixup(const uint32_t* __restrict__ px, int64_t npx,
                                               const uint32_t* __restrict__ seg, const uint32_t* __restrict__ pos_up,
                                               const uint32_t* __restrict__ pos_lo, const double* __restrict__ partK,
                                               const double* __restrict__ partM, double* __restrict__ K,
                                               double* __restrict__ M)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= npx) return;
    const uint32_t u = px[i];
    const uint32_t s0 = seg[u], s1 = seg[u + 1];
    double k = partK[s0], m = partM[s0];
    for (uint32_t s = s0 + 1; s < s1; s++) {
        k += partK[s];
        m += partM[s];
    }
    uint32_t p = pos_up[u];
    K[p] = k;
    M[p] = m;
    p = pos_lo[u];
    if (p != NONE) {
        K[p] = k;
        M[p] = m;
    }
}

template <int VAR, int BE>
int launch_fused_t(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s)
{
    using E = ElemTraits<VAR>;
    const size_t smem = (size_t)2 * E::NP * BE * sizeof(double);
    static bool configured = false;   // per template instance: raise the dynamic shared memory limit once
    if (!configured) {
        EF_CUDA(cudaFuncSetAttribute(k_fused<VAR, BE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    double* partK = p->d_local;
    double* partM = p->d_local + (int64_t)p->np * p->T;
    k_fused<VAR, BE><<<(unsigned)p->fb_nblocks, BE, smem, s>>>(p->d_elems, nodes, coeff, p->T, p->d_fb_cidx,
                                                                p->d_fb_slot_off, p->d_fb_sinfo, p->d_fb_posA,
                                                                p->d_fb_posB, K, M, partK, partM, p->d_status);
    profile_mid(p, s);
    if (p->n_px > 0)
        k_fixup<<<grid_for(p->n_px), TPB, 0, s>>>(p->d_px_uid, p->n_px, p->d_seg, p->d_pos_up, p->d_pos_lo, partK,
                                                  partM, K, M);
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

void free_fused(ef_plan* p)
{
    void* ptrs[] = {p->d_fb_slot_off, p->d_fb_sinfo, p->d_fb_cidx, p->d_fb_posA, p->d_fb_posB, p->d_px_uid};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    p->d_fb_slot_off = p->d_fb_sinfo = p->d_fb_posA = p->d_fb_posB = p->d_px_uid = nullptr;
    p->d_fb_cidx = nullptr;
    p->fb_block = 0;
    p->fb_nblocks = 0;
    p->fb_nslots = 0;
    p->n_px = 0;
    p->n_partial = 0;
}

}  // namespace

bool fused_block_supported(int BE) { return BE == 128 || BE == 256; }

int default_fused_block(int variant) { return variant == NED3 ? 128 : 256; }

int build_fused_block(ef_plan* p, int BE, cudaStream_t s)
{
    free_fused(p);
    if (p->T == 0) return EF_OK;
    if (!fused_block_supported(BE)) return EF_ERR_ARG;
    const int64_t T = p->T, n = T * p->np, U = p->U, per_block = (int64_t)BE * p->np;
    const int64_t nblocks = (T + BE - 1) / BE;
    if (per_block > 65535) return EF_ERR_ARG;

    int st = EF_OK;
    uint32_t *uos = nullptr, *flag = nullptr, *ex = nullptr, *bsorted = nullptr, *sstart = nullptr;
    uint8_t* complete = nullptr;
    uint64_t* keys = nullptr;
    void* tmp = nullptr;
    size_t tb = radix_tmp_bytes(n);
    if (scan_tmp_bytes(n) > tb) tb = scan_tmp_bytes(n);
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMalloc((void**)&uos, n * 4)) || !ok(cudaMalloc((void**)&complete, U > 0 ? U : 1)) ||
        !ok(cudaMalloc((void**)&keys, n * 8)) || !ok(cudaMalloc((void**)&bsorted, n * 4)) ||
        !ok(cudaMalloc((void**)&flag, n * 4)) || !ok(cudaMalloc((void**)&ex, n * 4 + 4)) || !ok(cudaMalloc(&tmp, tb)))
        st = EF_ERR_OOM;
    do {
        if (st) break;
        k_u_of_s<<<grid_for(U), TPB, 0, s>>>(p->d_seg, p->d_perm, U, T, BE, uos, complete);
        k_block_keys<<<grid_for(n), TPB, 0, s>>>(p->d_perm, n, T, BE, keys, bsorted);
        if ((st = radix_sort_pairs(keys, bsorted, n, bits_for((uint64_t)(nblocks - 1)), tmp, s))) break;
        k_slot_heads<<<grid_for(n), TPB, 0, s>>>(bsorted, uos, n, per_block, flag);
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
            !ok(cudaMalloc((void**)&p->d_fb_cidx, (size_t)n * 2))) {
            st = EF_ERR_OOM;
            break;
        }
        k_slot_start<<<grid_for(n), TPB, 0, s>>>(flag, ex, n, sstart);
        k_slots<<<grid_for(nslots), TPB, 0, s>>>(bsorted, uos, complete, sstart, nslots, n, per_block, p->d_pos_up,
                                                 p->d_pos_lo, p->d_fb_sinfo, p->d_fb_posA, p->d_fb_posB,
                                                 p->d_fb_slot_off);
        if (!ok(cudaMemcpyAsync(p->d_fb_slot_off + nblocks, &nslots, 4, cudaMemcpyHostToDevice, s))) {
            st = EF_ERR_CUDA;
            break;
        }
        // Within each block, order the slots by descending contribution count so
        // that the lanes of a warp run loops of equal length (the FP64 pipe
        // spends a warp instruction's full time even for idle lanes).
        if ((st = order_slots_by_count(p, nslots, nblocks, per_block, keys, uos, tmp, s, sstart))) break;
        k_cidx<<<grid_for(n), TPB, 0, s>>>(bsorted, p->d_perm, n, T, BE, per_block, p->d_fb_cidx);
        // split nonzeros for the fix-up
        k_px_flags<<<grid_for(U), TPB, 0, s>>>(complete, U, flag);
        if ((st = exclusive_scan_u32(flag, ex, U, true, tmp, s))) break;
        uint32_t npx = 0;
        if (!ok(cudaMemcpyAsync(&npx, ex + U, 4, cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s))) {
            st = EF_ERR_CUDA;
            break;
        }
        if (!ok(cudaMalloc((void**)&p->d_px_uid, (size_t)(npx > 0 ? npx : 1) * 4))) {
            st = EF_ERR_OOM;
            break;
        }
        k_px_list<<<grid_for(U), TPB, 0, s>>>(flag, ex, U, p->d_px_uid);
        if ((st = order_by_count(p->d_seg, p->d_px_uid, npx, keys, uos, tmp, s))) break;
        // raw contributions of split nonzeros = their segment lengths
        int64_t npart = 0;
        {
            // count on the host from the segment lengths of the split nonzeros
            uint32_t* hpx = (uint32_t*)malloc((size_t)(npx > 0 ? npx : 1) * 4);
            uint32_t* hseg = (uint32_t*)malloc((size_t)(U + 1) * 4);
            if (!hpx || !hseg) {
                free(hpx);
                free(hseg);
                st = EF_ERR_OOM;
                break;
            }
            cudaMemcpyAsync(hpx, p->d_px_uid, (size_t)npx * 4, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(hseg, p->d_seg, (size_t)(U + 1) * 4, cudaMemcpyDeviceToHost, s);
            if (!ok(cudaStreamSynchronize(s))) st = EF_ERR_CUDA;
            for (uint32_t i = 0; i < npx; i++) npart += hseg[hpx[i] + 1] - hseg[hpx[i]];
            free(hpx);
            free(hseg);
            if (st) break;
        }
        p->fb_block = BE;
        p->fb_nblocks = nblocks;
        p->fb_nslots = nslots;
        p->n_px = npx;
        p->n_partial = npart;
    } while (0);
    cudaError_t e = cudaGetLastError();
    if (st == EF_OK && e != cudaSuccess) {
        set_last_error("build_fused", e);
        st = EF_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    cudaFree(uos);
    cudaFree(complete);
    cudaFree(keys);
    cudaFree(bsorted);
    cudaFree(flag);
    cudaFree(ex);
    cudaFree(sstart);
    cudaFree(tmp);
    if (st != EF_OK) free_fused(p);
    return st;
}

int build_fused(ef_plan* p, cudaStream_t s) { return build_fused_block(p, default_fused_block(p->variant), s); }

void release_fused(ef_plan* p) { free_fused(p); }

int launch_fused(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s)
{
    if (p->T == 0) return EF_OK;
    if (p->fb_block == 128) return launch_variant<128>(p, nodes, coeff, K, M, s);
    return launch_variant<256>(p, nodes, coeff, K, M, s);
}

}  // namespace ef
