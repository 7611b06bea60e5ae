// Device primitives used at plan time: exclusive prefix sums and a stable
// LSD radix sort of (uint64 key, uint32 value) pairs.
//
// Both are reduce-then-scan designs with no inter-CTA waiting: each pass is
// a sequence of ordinary launches on one stream, so no launch can wait on
// another CTA.
#include <stdarg.h>
#include <stdio.h>

#include "ef_internal.cuh"

namespace ef {

static thread_local char g_last_error[256] = "";

void set_last_error(const char* where, cudaError_t err)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(err));
}

void set_last_message(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

const char* last_error_text() { return g_last_error; }

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int NWARP = SCAN_THREADS / 32;

// Exclusive scan of one value per thread across the CTA; *total gets the CTA sum.
template <typename T>
__device__ __forceinline__ T cta_exclusive_scan(T v, T* warp_tot, T* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NWARP ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NWARP) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    T before = warp > 0 ? warp_tot[warp - 1] : T(0);
    *total = warp_tot[NWARP - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const T* in, int64_t n, T* sums)
{
    __shared__ T wt[NWARP];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T acc = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += in[i];
    }
    T tot;
    cta_exclusive_scan(acc, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the tile sums in place (exclusive), chunk by chunk with a carry.
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(T* sums, int64_t m, T* total_out)
{
    __shared__ T wt[NWARP];
    T carry = 0;
    for (int64_t base = 0; base < m; base += SCAN_TILE) {
        T v[SCAN_ITEMS];
        T tsum = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + j;
            v[j] = i < m ? sums[i] : T(0);
            tsum += v[j];
        }
        T tot;
        T run = carry + cta_exclusive_scan(tsum, wt, &tot);
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + j;
            if (i < m) sums[i] = run;
            run += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const T* in, int64_t n, const T* offs, T* out)
{
    __shared__ T wt[NWARP];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T v[SCAN_ITEMS];
    T tsum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + j;
        v[j] = i < n ? in[i] : T(0);
        tsum += v[j];
    }
    T tot;
    T run = offs[blockIdx.x] + cta_exclusive_scan(tsum, wt, &tot);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
}

template <typename T>
int exclusive_scan(const T* in, T* out, int64_t n, bool write_total, void* tmp, cudaStream_t s)
{
    if (n <= 0) {
        if (write_total) EF_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
        return EF_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    T* sums = (T*)tmp;
    k_tile_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums);
    k_scan_sums<T><<<1, SCAN_THREADS, 0, s>>>(sums, tiles, write_total ? out + n : nullptr);
    k_scan_tiles<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums, out);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

// ---- radix sort --------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* keys, int64_t n, int shift, uint32_t* hist,
                                                        int64_t ntiles)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: items of a tile are visited in index order, 256 per round;
// a key's rank among equal digits = earlier rounds + earlier warps + earlier lanes.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                                                           uint32_t* vout, int64_t n, int shift,
                                                           const uint32_t* hist_scan, int64_t ntiles)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[RS_WARPS][257];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = hist_scan[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) wc[w][tid] = 0;
    if (tid < RS_WARPS) wc[tid][256] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = tile0 + (int64_t)r * RS_THREADS + tid;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        uint32_t val = valid ? vin[i] : 0u;
        unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt_mask);
        if (rank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = base[d] + rank;
            for (int w = 0; w < warp; w++) off += wc[w][d];
            kout[off] = key;
            vout[off] = val;
        }
        __syncthreads();
        {
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; w++) {
                sum += wc[w][tid];
                wc[w][tid] = 0;
            }
            base[tid] += sum;
            if (tid < RS_WARPS) wc[tid][256] = 0;
        }
        __syncthreads();
    }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n)
{
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(tiles > 0 ? tiles : 1) * 8 + 256;
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, bool write_total, void* tmp, cudaStream_t s)
{
    return exclusive_scan<uint32_t>(in, out, n, write_total, tmp, s);
}

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, bool write_total, void* tmp, cudaStream_t s)
{
    return exclusive_scan<int64_t>(in, out, n, write_total, tmp, s);
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t radix_tmp_bytes(int64_t n)
{
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    if (ntiles < 1) ntiles = 1;
    size_t hist = (size_t)ntiles * 256;
    return align256((size_t)n * 8) + align256((size_t)n * 4) + align256(hist * 4) + align256(scan_tmp_bytes((int64_t)hist));
}

int radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, void* tmp, cudaStream_t s)
{
    if (n <= 1 || bits <= 0) return EF_OK;
    if (n >= (int64_t)1 << 32) return EF_ERR_SIZE;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    size_t hist_n = (size_t)ntiles * 256;
    char* t = (char*)tmp;
    uint64_t* k_alt = (uint64_t*)t;
    t += align256((size_t)n * 8);
    uint32_t* v_alt = (uint32_t*)t;
    t += align256((size_t)n * 4);
    uint32_t* hist = (uint32_t*)t;
    t += align256(hist_n * 4);
    void* scan_tmp = t;
    uint64_t *ka = keys, *kb = k_alt;
    uint32_t *va = vals, *vb = v_alt;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, hist, ntiles);
        EF_TRY(exclusive_scan_u32(hist, hist, (int64_t)hist_n, false, scan_tmp, s));
        k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist, ntiles);
        EF_CUDA(cudaGetLastError());
        uint64_t* tk = ka;
        ka = kb;
        kb = tk;
        uint32_t* tv = va;
        va = vb;
        vb = tv;
        passes++;
    }
    if (passes & 1) {
        EF_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        EF_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return EF_OK;
}

}  // namespace ef
