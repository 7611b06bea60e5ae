// ef_fp64_probe: throughput of this GPU's FP64 pipe (not part of the paper's
// method; it measures the denominator of the element kernels' roofline), and
// of the integer-pipe multiply (ef_intmul.cuh) alone and beside the FP64 pipe.
//
// Every thread runs CHAINS independent dependency chains of one operation
// (DFMA, DADD, DMUL, the integer-pipe multiply, DFMA in half of the chains
// and the integer-pipe multiply in the other half, DFMA with literal
// operands, or an addition as a DFMA with a per-thread 1.0), `iters` each
// (rounded up to a multiple of UNROLL); with CHAINS chains per thread and 32
// warps per SM the latency is hidden, so the time is set by the issue rate.
// The result is lane operations per second (a DFMA counts as one operation,
// as in the element kernels' op counts). The operands other than the chain
// value are per-thread registers (ef_fp64.cuh): a literal or warp-uniform
// operand would hold a DFMA to 84 % of the pipe's rate, the rate DADD and
// DMUL run at in any form.
//
// ef_int_mul_check compares the integer-pipe multiply with the FP64 multiply
// instruction bit for bit on generated operands.
#include "ef_fp64.cuh"
#include "ef_internal.cuh"
#include "ef_intmul.cuh"

namespace ef {
namespace {

constexpr int PROBE_TPB = 256;
constexpr int PROBE_CTAS_PER_SM = 4;
constexpr int CHAINS = 8;
constexpr int UNROLL = 8;

template <int OP>
__global__ void __launch_bounds__(PROBE_TPB) k_fp64_probe(int rounds, double seed, double* sink)
{
    double a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; i++) a[i] = seed + 1e-3 * threadIdx.x + i;
    const double m = per_thread(1.0 + 1e-12), c = per_thread(1e-15), one = per_thread(1.0);
    IntMul im;
    // UNROLL rounds per loop trip, so that the loop's own integer work is small
    for (int it = 0; it < rounds; it++) {
#pragma unroll
        for (int u = 0; u < UNROLL; u++)
#pragma unroll
            for (int i = 0; i < CHAINS; i++) {
                if (OP == 0) a[i] = fma(a[i], m, c);
                if (OP == 1) a[i] = a[i] + c;
                if (OP == 2) a[i] = a[i] * m;
                if (OP == 3) a[i] = im(a[i], m);
                if (OP == 4) a[i] = i < CHAINS / 2 ? fma(a[i], m, c) : im(a[i], m);
                if (OP == 5) a[i] = fma(a[i], 1.0 + 1e-12, 1e-15);   // literal operands
                if (OP == 6) a[i] = fma(a[i], one, c);               // a + c at the full rate
            }
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; i++) s += a[i];
    // never true for the seeds used; keeps the chains live
    if (s == -1.0 || im.off == 12345u) sink[0] = s;
}

__device__ __forceinline__ uint64_t splitmix(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Operand pairs i = 0 .. n-1 from SplitMix64(seed, i): random significands
// and signs; exponents over the whole range (one pair in 8), near the bias
// (where products stay normal), or with many trailing zero bits in the
// significands (ties), or a special value (zero, subnormal, infinity, NaN,
// the largest and smallest normals) in one operand.
__global__ void __launch_bounds__(256) k_int_mul_check(int64_t n, uint64_t seed,
                                                       unsigned long long* __restrict__ counts)
{
    unsigned long long flagged = 0, mismatched = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r1 = splitmix(seed ^ (3 * (uint64_t)i)), r2 = splitmix(seed ^ (3 * (uint64_t)i + 1)),
                       r3 = splitmix(seed ^ (3 * (uint64_t)i + 2));
        const int mode = (int)(r3 & 7);
        uint64_t ea = 1023 + (r3 >> 8) % 1200 - 600, eb = 1023 + (r3 >> 24) % 1200 - 600;
        if (mode == 1) {
            ea = (r3 >> 8) % 2048;
            eb = (r3 >> 24) % 2048;
        }
        uint64_t fa = r1 & 0xfffffffffffffull, fb = r2 & 0xfffffffffffffull;
        if (mode == 2) {
            fa |= 0xfffffff000000ull;
            fb |= 0xffffff0000000ull;
        }
        if (mode == 6) {
            fa &= 0xfff0000000000ull;
            fb &= 0xffff000000000ull;
        }
        uint64_t ua = (r1 & 0x8000000000000000ull) | ((ea & 0x7ff) << 52) | fa;
        uint64_t ub = (r2 & 0x8000000000000000ull) | ((eb & 0x7ff) << 52) | fb;
        const uint64_t specials[8] = {0ull, 1ull, 0x000fffffffffffffull, 0x0010000000000000ull,
                                      0x7fefffffffffffffull, 0x7ff0000000000000ull, 0x7ff8000000000000ull,
                                      0x3ff0000000000000ull};
        if (mode == 4) ua = specials[(r3 >> 40) & 7] | (r1 & 0x8000000000000000ull);
        if (mode == 5) ub = specials[(r3 >> 44) & 7] | (r2 & 0x8000000000000000ull);
        const double a = __longlong_as_double((long long)ua), b = __longlong_as_double((long long)ub);
        IntMul im;
        const double p = im(a, b);
        if (im.off)
            flagged++;
        else if (__double_as_longlong(p) != __double_as_longlong(__dmul_rn(a, b)))
            mismatched++;
    }
    atomicAdd(counts + 0, flagged);
    atomicAdd(counts + 1, mismatched);
}

}  // namespace
}  // namespace ef

using namespace ef;

extern "C" int ef_fp64_probe(int op, int64_t iters, double* d_sink, double* ops_per_s, double* ms, void* stream)
{
    if (op < 0 || op > 6 || iters < 1 || !d_sink || !ops_per_s) return EF_ERR_ARG;
    int dev = 0, sms = 0;
    EF_CUDA(cudaGetDevice(&dev));
    EF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t rounds64 = (iters + UNROLL - 1) / UNROLL;
    if (rounds64 > INT32_MAX) return EF_ERR_ARG;
    const int rounds = (int)rounds64;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    EF_CUDA(cudaEventCreate(&e0));
    EF_CUDA(cudaEventCreate(&e1));
    const unsigned grid = (unsigned)(sms * PROBE_CTAS_PER_SM);
    auto launch = [&](int n) {
        if (op == 0) k_fp64_probe<0><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
        if (op == 1) k_fp64_probe<1><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
        if (op == 2) k_fp64_probe<2><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
        if (op == 3) k_fp64_probe<3><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
        if (op == 4) k_fp64_probe<4><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
        if (op == 5) k_fp64_probe<5><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
        if (op == 6) k_fp64_probe<6><<<grid, PROBE_TPB, 0, s>>>(n, 1.0, d_sink);
    };
    launch(rounds < 8 ? rounds : 8);   // warm-up
    cudaEventRecord(e0, s);
    launch(rounds);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float t = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        set_last_error("ef_fp64_probe", err);
        return EF_ERR_CUDA;
    }
    const double ops = (double)grid * PROBE_TPB * CHAINS * UNROLL * (double)rounds;
    *ops_per_s = ops / (t * 1e-3);
    if (ms) *ms = t;
    return EF_OK;
}

extern "C" int ef_int_mul_check(int64_t n, uint64_t seed, unsigned long long* d_counts, void* stream)
{
    if (n < 0 || !d_counts) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    EF_CUDA(cudaMemsetAsync(d_counts, 0, 2 * sizeof(unsigned long long), s));
    if (n > 0) {
        int dev = 0, sms = 0;
        EF_CUDA(cudaGetDevice(&dev));
        EF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int64_t blocks = (n + 255) / 256;
        const unsigned grid = (unsigned)(blocks < 8 * (int64_t)sms ? blocks : 8 * (int64_t)sms);
        k_int_mul_check<<<grid, 256, 0, s>>>(n, seed, d_counts);
        EF_CUDA(cudaGetLastError());
    }
    return EF_OK;
}
