// Persistent interleaved work queue: element tiles and sum tiles of one or
// many meshes in a single kernel launch.
//
// Every mesh's elements are cut into chunks; the sum's work order groups the
// upper nonzeros by the chunk that completes them (ef_assemble.cu). The
// queue is a sequence of segments over all (mesh, chunk) pairs X_0 .. X_{N-1}:
//   E(X_0), E(X_1), S(X_0), E(X_2), S(X_1), ..., E(X_{N-1}), S(X_{N-2}), S(X_{N-1})
// where E(X) are the element tiles of chunk X and S(X) the sum tiles of the
// nonzeros X completes. A CTA takes tiles in queue order (integer ticket, or
// the static stride blockIdx.x + k gridDim.x). Alternatively (role split) in
// every group of four CTAs some take only element tiles, in chunk order, from
// one ticket, and the others only sum tiles, in chunk order, from a second
// ticket, so that FP64-bound and memory-bound work share every SM. An element tile writes its
// contributions into the mesh's work-ordered list and then counts itself
// done for its chunk (fence + integer atomic). A sum tile first waits until
// every element chunk of its mesh up to its own is done. In the single queue
// those tiles were all handed out earlier, so they are held by running CTAs;
// with the role split, element CTAs never wait, so every element tile is
// finished by a running CTA. Either way the wait ends; it is bounded
// regardless (poll limit, then a timeout status, and the tile is skipped). Because sums lag one
// chunk behind, FP64-bound element tiles and memory-bound sum tiles are in
// flight on the SMs at the same time.
//
// The last CTA to leave resets the ticket and the counters, so one launch is
// the whole assembly: no memset, no host synchronisation, capturable in a
// CUDA graph. Sums are the same left-to-right sums as in every other path.
#include <string.h>

#include <vector>

#include "ef_assemble.cuh"
#include "ef_queue.cuh"

namespace ef {
namespace {

// A sum tile gives up waiting after kWaitNs of wall time (the GPU's global
// nanosecond timer) or kPollLimit polls, whichever comes first, sets the
// timeout status and skips its work; once any tile has given up, the others
// see the status within 64 polls and give up too. Legitimate waits last at
// most the element work of a few chunks (milliseconds).
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr unsigned kPollLimit = 50000000u;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// CTAs per SM the kernel is compiled for: 80 registers per thread (6 CTAs
// of 128 threads), with the element tiles' products on the integer pipes and
// their additions as full-rate DFMAs (the 3D Nedelec tiles spill about 150
// bytes). Measured on the 256-mesh batch: 21.9 ms, against 23.4 ms with FP64
// products at 64 registers (8 CTAs, the sum tiles' 32 warps per SM), 24.1 ms
// with plain FP64 additions there as well, and 22.6 ms with integer products
// at 96 registers (5 CTAs).
constexpr int queue_min_blocks(int BE) { return BE == 128 ? 6 : 3; }

__device__ __forceinline__ int find_segment(const QueueSegment* __restrict__ seg, int nseg, int64_t k)
{
    int lo = 0, hi = nseg - 1;   // last segment with tile_off <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg[mid].tile_off <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int VAR, int BE, int MINB>
__global__ void __launch_bounds__(BE, MINB) k_queue(const QueueMesh* __restrict__ md,
                                                    const QueueSegment* __restrict__ sg, int nseg,
                                                    const uint32_t* __restrict__ need, int64_t ntiles,
                                                    int64_t n_elem_tiles, int BU, int dynamic, int elem_ctas,
                                                    uint32_t* ctrl, int nctr,
                                                    const double* __restrict__ nodes0,
                                                    const double* __restrict__ coeff0, double* __restrict__ K0,
                                                    double* __restrict__ M0, int* status)
{
    using E = ElemTraits<VAR>;
    __shared__ int64_t s_tile;
    __shared__ int s_ok;
    uint32_t* ticket = ctrl;
    uint32_t* exited = ctrl + 1;
    uint32_t* ticket2 = ctrl + 2;
    uint32_t* done = ctrl + 3;
    // role split (elem_ctas = k > 0): in each group of 4 CTAs the first k take
    // element tiles [0, n_elem_tiles) from `ticket`, the others sum tiles
    // [n_elem_tiles, ntiles) from `ticket2`; element CTAs never wait.
    const bool split = elem_ctas > 0;
    const bool elem_role = (int)(blockIdx.x & 3u) < elem_ctas;
    uint32_t* my_ticket = (split && !elem_role) ? ticket2 : ticket;
    const int64_t lo = split ? (elem_role ? 0 : n_elem_tiles) : 0;
    const int64_t hi = split ? (elem_role ? n_elem_tiles : ntiles) : ntiles;
    int64_t next = blockIdx.x;
    for (;;) {
        if (threadIdx.x == 0) s_tile = lo + (int64_t)atomicAdd(my_ticket, 1u);
        __syncthreads();
        const int64_t k = dynamic || split ? s_tile : next;
        __syncthreads();
        next += gridDim.x;
        if (k >= hi) break;
        const int si = find_segment(sg, nseg, k);
        const QueueSegment g = sg[si];
        const QueueMesh& d = md[g.mesh];
        const double* nodes = nodes0 ? nodes0 : d.nodes;
        const int64_t t = k - g.tile_off;
        if (g.type == 0) {
            const int64_t e = g.lo + t * BE + threadIdx.x;
            if (e < g.hi) {
                const double* coeff = nodes0 ? coeff0 : d.coeff;
                double Kq[E::NP], Mq[E::NP];
                if (compute_element<VAR, true, true>(d.elems, nodes, coeff, coeff, e, Kq, Mq))
                    atomicOr(status, ST_DEGENERATE);
#pragma unroll
                for (int q = 0; q < E::NP; q++) {
                    const uint32_t p = __ldg(d.inv + (int64_t)q * d.T + e);
                    d.list[p] = make_double2(Kq[q], Mq[q]);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&done[g.chunk], 1u);
            }
        } else {
            if (threadIdx.x == 0) {
                int ok = 1;
                unsigned polls = 0;
                uint64_t t0 = 0;
                for (int j = g.dep_first; j < g.dep_first + g.dep_count && ok; j++) {
                    while (atomicAdd(&done[j], 0u) < need[j]) {
                        if (polls == 0) t0 = global_ns();
                        ++polls;
                        if ((polls & 63u) == 0 && (*(volatile int*)status & ST_TIMEOUT)) {
                            ok = 0;
                            break;
                        }
                        if (polls > kPollLimit || global_ns() - t0 > kWaitNs) {
                            ok = 0;
                            atomicOr(status, ST_TIMEOUT);
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) {
                // one thread per work item, stored where it lies (ordering the
                // stores per block of 256 items as the two-launch sum kernel
                // does made this schedule slower: 26.9 against 25.0 ms for the
                // 256-mesh batch)
                double* K = nodes0 ? K0 : d.K;
                double* M = nodes0 ? M0 : d.M;
                const double2* l = d.list;
                const int64_t i0 = g.lo + t * BU;
                const int64_t i1 = i0 + BU < g.hi ? i0 + BU : g.hi;
                for (int64_t i = i0 + threadIdx.x; i < i1; i += BE) {
                    const uint32_t s0 = d.wseg[i], s1 = d.wseg[i + 1];
                    const uint32_t pu = d.wpos_up[i], pl = d.wpos_lo[i];
                    double2 v = __ldcg(l + s0);
                    double kv = v.x, mv = v.y;
                    for (uint32_t s = s0 + 1; s < s1; s++) {
                        v = __ldcg(l + s);
                        kv += v.x;
                        mv += v.y;
                    }
                    K[pu] = kv;
                    M[pu] = mv;
                    if (pl != 0xffffffffu) {
                        K[pl] = kv;
                        M[pl] = mv;
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
            for (int i = 0; i < nctr; i++) done[i] = 0;
            *ticket = 0;
            *ticket2 = 0;
            __threadfence();
            *exited = 0;
        }
    }
}

template <int VAR, int BE>
int launch_t(const Queue* q, const QueueArgs& a, cudaStream_t s)
{
    constexpr int MINB = queue_min_blocks(BE);
    const int grid = q->cfg.ctas_per_sm * q->sms;
    k_queue<VAR, BE, MINB><<<grid, BE, 0, s>>>(q->d_mesh, q->d_seg, q->nseg, q->d_need, q->ntiles, q->n_elem_tiles,
                                               q->cfg.sum_tile, q->cfg.dynamic, q->cfg.elem_ctas, q->d_ctrl,
                                               q->nctr, a.nodes, a.coeff, a.K, a.M, q->d_status);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

template <int BE>
int launch_be(const Queue* q, const QueueArgs& a, cudaStream_t s)
{
    switch (q->variant) {
        case RT2: return launch_t<RT2, BE>(q, a, s);
        case NED2: return launch_t<NED2, BE>(q, a, s);
        case RT3: return launch_t<RT3, BE>(q, a, s);
        default: return launch_t<NED3, BE>(q, a, s);
    }
}

template <int VAR>
int occupancy_t(int BE)
{
    int nb = 0;
    cudaError_t e = BE == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &nb, k_queue<VAR, 128, queue_min_blocks(128)>, 128, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &nb, k_queue<VAR, 256, queue_min_blocks(256)>, 256, 0);
    return e == cudaSuccess ? nb : 0;
}

}  // namespace

int queue_max_ctas_per_sm(int variant, int BE)
{
    switch (variant) {
        case RT2: return occupancy_t<RT2>(BE);
        case NED2: return occupancy_t<NED2>(BE);
        case RT3: return occupancy_t<RT3>(BE);
        default: return occupancy_t<NED3>(BE);
    }
}

// Segment table for the meshes' current chunking (each plan's pc_chunks /
// pc_chunk / pc_woff) and the configuration's tile sizes and mesh order:
// element chunks X_0 .. X_{N-1} (mesh by mesh, chunk by chunk), emitted as
// E(X_0), E(X_1), S(X_0), E(X_2), S(X_1), ..., S(X_{N-1}).
int queue_build(Queue* q, const std::vector<ef_plan*>& plans, cudaStream_t s)
{
    const int n = (int)plans.size(), BE = q->cfg.elems_per_tile, BU = q->cfg.sum_tile;
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    if (q->cfg.largest_first)
        for (int i = 1; i < n; i++)
            for (int j = i; j > 0 && plans[order[j]]->T > plans[order[j - 1]]->T; j--) {
                int t = order[j];
                order[j] = order[j - 1];
                order[j - 1] = t;
            }
    struct X { int mesh, chunk; };
    std::vector<X> xs;
    for (int oi = 0; oi < n; oi++) {
        const int m = order[oi];
        if (plans[m]->T == 0) continue;
        const int nc = plans[m]->pc_chunks > 0 ? plans[m]->pc_chunks : 1;
        for (int c = 0; c < nc; c++) xs.push_back({m, c});
    }
    const int N = (int)xs.size();
    std::vector<QueueSegment> segs;
    std::vector<uint32_t> need(N > 0 ? N : 1, 0);
    segs.reserve(2 * N);
    int64_t off = 0;
    auto add_e = [&](int xi) {
        const ef_plan* p = plans[xs[xi].mesh];
        QueueSegment g;
        memset(&g, 0, sizeof(g));
        g.type = 0;
        g.mesh = xs[xi].mesh;
        g.chunk = xi;
        g.lo = (int64_t)xs[xi].chunk * p->pc_chunk;
        g.hi = g.lo + p->pc_chunk < p->T ? g.lo + p->pc_chunk : p->T;
        g.ntiles = (g.hi - g.lo + BE - 1) / BE;
        g.tile_off = off;
        need[xi] = (uint32_t)g.ntiles;
        off += g.ntiles;
        segs.push_back(g);
    };
    auto add_s = [&](int xi) {
        const ef_plan* p = plans[xs[xi].mesh];
        const int c = xs[xi].chunk;
        QueueSegment g;
        memset(&g, 0, sizeof(g));
        g.type = 1;
        g.mesh = xs[xi].mesh;
        g.chunk = xi;
        g.lo = p->pc_woff[c];
        g.hi = p->pc_woff[c + 1];
        g.ntiles = (g.hi - g.lo + BU - 1) / BU;
        g.dep_first = xi - c;          // chunks 0..c of the same mesh are consecutive in xs
        g.dep_count = c + 1;
        g.tile_off = off;
        off += g.ntiles;
        if (g.ntiles > 0) segs.push_back(g);
    };
    if (q->cfg.elem_ctas > 0) {
        // two queues: every element chunk in order, then every sum chunk in order
        for (int xi = 0; xi < N; xi++) add_e(xi);
        q->n_elem_tiles = off;
        for (int xi = 0; xi < N; xi++) add_s(xi);
    } else {
        for (int xi = 0; xi < N; xi++) {
            add_e(xi);
            if (xi > 0) add_s(xi - 1);
        }
        if (N > 0) add_s(N - 1);
        q->n_elem_tiles = 0;
    }
    q->nseg = (int)segs.size();
    q->ntiles = off;
    q->nctr = N;
    // two-launch schedule: element and sum blocks of the meshes, in mesh order
    {
        std::vector<int64_t> eb(n + 1, 0), sb(n + 1, 0);
        for (int m = 0; m < n; m++) {
            eb[m + 1] = eb[m] + element_blocks(plans[m]->T);
            sb[m + 1] = sb[m] + sum_blocks(plans[m]->U);
        }
        if (q->nmesh < n || !q->d_eblk) {
            if (q->d_eblk) cudaFree(q->d_eblk);
            if (q->d_sblk) cudaFree(q->d_sblk);
            q->d_eblk = q->d_sblk = nullptr;
            EF_CUDA(cudaMalloc((void**)&q->d_eblk, sizeof(int64_t) * (n + 1)));
            EF_CUDA(cudaMalloc((void**)&q->d_sblk, sizeof(int64_t) * (n + 1)));
        }
        q->nmesh = n;
        q->n_eblk = eb[n];
        q->n_sblk = sb[n];
        std::vector<uint32_t> em((size_t)(eb[n] > 0 ? eb[n] : 1)), sm((size_t)(sb[n] > 0 ? sb[n] : 1));
        for (int m = 0; m < n; m++) {
            for (int64_t b = eb[m]; b < eb[m + 1]; b++) em[b] = (uint32_t)m;
            for (int64_t b = sb[m]; b < sb[m + 1]; b++) sm[b] = (uint32_t)m;
        }
        if (q->cap_eblk < (int64_t)em.size() || q->cap_sblk < (int64_t)sm.size()) {
            if (q->d_emesh) cudaFree(q->d_emesh);
            if (q->d_smesh) cudaFree(q->d_smesh);
            q->d_emesh = q->d_smesh = nullptr;
            q->cap_eblk = q->cap_sblk = 0;
            EF_CUDA(cudaMalloc((void**)&q->d_emesh, sizeof(uint32_t) * em.size()));
            EF_CUDA(cudaMalloc((void**)&q->d_smesh, sizeof(uint32_t) * sm.size()));
            q->cap_eblk = (int64_t)em.size();
            q->cap_sblk = (int64_t)sm.size();
        }
        EF_CUDA(cudaMemcpyAsync(q->d_eblk, eb.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
        EF_CUDA(cudaMemcpyAsync(q->d_sblk, sb.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
        EF_CUDA(cudaMemcpyAsync(q->d_emesh, em.data(), sizeof(uint32_t) * em.size(), cudaMemcpyHostToDevice, s));
        EF_CUDA(cudaMemcpyAsync(q->d_smesh, sm.data(), sizeof(uint32_t) * sm.size(), cudaMemcpyHostToDevice, s));
        EF_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
    }
    if (off >= ((int64_t)1 << 32)) return EF_ERR_SIZE;
    if (q->cap_seg < q->nseg || q->cap_ctr < N + 3) {
        if (q->d_seg) cudaFree(q->d_seg);
        if (q->d_need) cudaFree(q->d_need);
        if (q->d_ctrl) cudaFree(q->d_ctrl);
        q->d_seg = nullptr;
        q->d_need = nullptr;
        q->d_ctrl = nullptr;
        const int cs = q->nseg > 0 ? q->nseg : 1;
        EF_CUDA(cudaMalloc((void**)&q->d_seg, sizeof(QueueSegment) * cs));
        EF_CUDA(cudaMalloc((void**)&q->d_need, sizeof(uint32_t) * (N > 0 ? N : 1)));
        EF_CUDA(cudaMalloc((void**)&q->d_ctrl, sizeof(uint32_t) * (N + 3)));
        q->cap_seg = cs;
        q->cap_ctr = N + 3;
    }
    if (q->nseg > 0)
        EF_CUDA(cudaMemcpyAsync(q->d_seg, segs.data(), sizeof(QueueSegment) * q->nseg, cudaMemcpyHostToDevice, s));
    if (N > 0) EF_CUDA(cudaMemcpyAsync(q->d_need, need.data(), sizeof(uint32_t) * N, cudaMemcpyHostToDevice, s));
    q->stall = 0;
    EF_CUDA(cudaMemsetAsync(q->d_ctrl, 0, sizeof(uint32_t) * (N + 3), s));
    EF_CUDA(cudaStreamSynchronize(s));
    return EF_OK;
}

int queue_set_meshes(Queue* q, const std::vector<ef_plan*>& plans, cudaStream_t s)
{
    const int n = (int)plans.size();
    q->host_mesh.resize(n);
    for (int m = 0; m < n; m++) {
        const ef_plan* p = plans[m];
        QueueMesh& d = q->host_mesh[m];
        const double* keep_nodes = d.nodes;
        const double* keep_coeff = d.coeff;
        double *keep_K = d.K, *keep_M = d.M;
        memset(&d, 0, sizeof(d));
        d.elems = p->d_elems;
        d.inv = p->d_inv;
        d.wseg = p->d_wseg;
        d.wpos_up = p->d_wpos_up;
        d.wpos_lo = p->d_wpos_lo;
        d.wst_up = p->d_wst_up;
        d.wst_lo = p->d_wst_lo;
        d.list = (double2*)p->d_local;
        d.T = p->T;
        d.U = p->U;
        d.nodes = keep_nodes;
        d.coeff = keep_coeff;
        d.K = keep_K;
        d.M = keep_M;
    }
    if (q->cap_mesh < n) {
        if (q->d_mesh) cudaFree(q->d_mesh);
        q->d_mesh = nullptr;
        EF_CUDA(cudaMalloc((void**)&q->d_mesh, sizeof(QueueMesh) * (n > 0 ? n : 1)));
        q->cap_mesh = n;
    }
    if (n > 0)
        EF_CUDA(cudaMemcpyAsync(q->d_mesh, q->host_mesh.data(), sizeof(QueueMesh) * n, cudaMemcpyHostToDevice, s));
    EF_CUDA(cudaStreamSynchronize(s));
    return EF_OK;
}

int queue_init(Queue* q, int variant, int* shared_status)
{
    q->variant = variant;
    int dev = 0;
    EF_CUDA(cudaGetDevice(&dev));
    EF_CUDA(cudaDeviceGetAttribute(&q->sms, cudaDevAttrMultiProcessorCount, dev));
    if (shared_status) {
        q->d_status = shared_status;
        q->own_status = false;
    } else {
        EF_CUDA(cudaMalloc((void**)&q->d_status, sizeof(int)));
        EF_CUDA(cudaMemset(q->d_status, 0, sizeof(int)));
        q->own_status = true;
    }
    q->cfg.elems_per_tile = 256;
    q->cfg.sum_tile = 2048;
    q->cfg.dynamic = 1;
    q->cfg.largest_first = 0;
    q->cfg.elem_ctas = 0;
    q->cfg.two_launch = 0;
    q->cfg.ctas_per_sm = queue_max_ctas_per_sm(variant, 256);
    if (q->cfg.ctas_per_sm < 1) return EF_ERR_CUDA;
    return EF_OK;
}

void queue_free(Queue* q)
{
    void* ptrs[] = {q->d_mesh, q->d_seg, q->d_need, q->d_ctrl, q->own_status ? q->d_status : nullptr, q->d_eblk,
                    q->d_sblk, q->d_emesh, q->d_smesh};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    q->d_eblk = q->d_sblk = nullptr;
    q->d_emesh = q->d_smesh = nullptr;
    q->cap_eblk = q->cap_sblk = 0;
    q->nmesh = 0;
    q->d_mesh = nullptr;
    q->d_seg = nullptr;
    q->d_need = nullptr;
    q->d_ctrl = nullptr;
    q->d_status = nullptr;
    q->cap_mesh = q->cap_seg = q->cap_ctr = 0;
}

int queue_launch(const Queue* q, const QueueArgs& a, cudaStream_t s)
{
    if (q->cfg.two_launch && !a.nodes)
        return launch_batch_two_pass(q->variant, q->d_mesh, q->d_emesh, q->d_eblk, q->n_eblk, q->d_smesh, q->d_sblk,
                                     q->n_sblk, q->d_status, s);
    if (q->ntiles == 0) return EF_OK;
    return q->cfg.elems_per_tile == 128 ? launch_be<128>(q, a, s) : launch_be<256>(q, a, s);
}

int queue_check(const Queue* q, cudaStream_t s)
{
    int st = 0;
    EF_CUDA(cudaMemcpyAsync(&st, q->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    if (st) EF_CUDA(cudaMemsetAsync(q->d_status, 0, sizeof(int), s));
    if (st & ST_TIMEOUT) return EF_ERR_TIMEOUT;
    if (st & ST_DEGENERATE) return EF_ERR_DEGENERATE;
    return EF_OK;
}

// Fault injection: raise (on) or restore (!on) the number of element tiles
// that the first element chunk must report done. Raised, the sums that
// depend on that chunk wait for a tile that never comes, give up after the
// wait limit, and the launch ends with the timeout status.
int queue_inject_stall(Queue* q, int on, cudaStream_t s)
{
    if (!q->d_need || q->nctr < 1) return EF_ERR_ARG;
    const uint32_t want = on ? 1u : 0u;
    if (want == q->stall) return EF_OK;
    uint32_t n0 = 0;
    EF_CUDA(cudaMemcpyAsync(&n0, q->d_need, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    EF_CUDA(cudaStreamSynchronize(s));
    n0 = n0 - q->stall + want;
    EF_CUDA(cudaMemcpyAsync(q->d_need, &n0, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    EF_CUDA(cudaStreamSynchronize(s));
    q->stall = want;
    return EF_OK;
}

}  // namespace ef

// ---- the single-mesh plan's queue -------------------------------------------------

namespace ef {

void plan_queue_free(ef_plan* p)
{
    if (p->queue) {
        queue_free(p->queue);
        delete p->queue;
        p->queue = nullptr;
    }
}

// (Re)build the plan's one-launch schedule for its current work order.
int plan_queue_rebuild(ef_plan* p, cudaStream_t s)
{
    if (!p->queue) {
        p->queue = new Queue();
        int st = queue_init(p->queue, p->variant, p->d_status);
        if (st != EF_OK) {
            plan_queue_free(p);
            return st;
        }
    }
    std::vector<ef_plan*> one(1, p);
    EF_TRY(queue_set_meshes(p->queue, one, s));
    return queue_build(p->queue, one, s);
}

int plan_queue_config(ef_plan* p, const ef_batch_config_t& cfg, cudaStream_t s)
{
    if (!p->queue) EF_TRY(plan_queue_rebuild(p, s));
    p->queue->cfg = cfg;
    std::vector<ef_plan*> one(1, p);
    return queue_build(p->queue, one, s);
}

int launch_queue(const ef_plan* p, const double* nodes, const double* coeff, double* K, double* M, cudaStream_t s)
{
    if (p->T == 0) return EF_OK;
    if (!p->queue) return EF_ERR_ARG;
    QueueArgs a;
    a.nodes = nodes;
    a.coeff = coeff;
    a.K = K;
    a.M = M;
    return queue_launch(p->queue, a, s);
}

}  // namespace ef
