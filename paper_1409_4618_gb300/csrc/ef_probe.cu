// ef_fp64_probe: throughput of this GPU's FP64 pipe (not part of the paper's
// method; it measures the denominator of the element kernels' roofline).
//
// Every thread runs CHAINS independent dependency chains of one FP64
// operation (DFMA, DADD or DMUL), `iters` operations each (rounded up to a
// multiple of UNROLL); with CHAINS chains per
// thread and 32 warps per SM the pipe's latency is hidden, so the time is
// set by its issue rate. The result is lane operations per second (a DFMA
// counts as one operation, as in the element kernels' op counts).
#include "ef_internal.cuh"

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
    const double m = 1.0 + 1e-12, c = 1e-15;
    // UNROLL rounds per loop trip, so that the loop's own integer work is small
    for (int it = 0; it < rounds; it++) {
#pragma unroll
        for (int u = 0; u < UNROLL; u++)
#pragma unroll
            for (int i = 0; i < CHAINS; i++) {
                if (OP == 0) a[i] = fma(a[i], m, c);
                if (OP == 1) a[i] = a[i] + c;
                if (OP == 2) a[i] = a[i] * m;
            }
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; i++) s += a[i];
    if (s == -1.0) sink[0] = s;   // never true for the seeds used; keeps the chains live
}

}  // namespace
}  // namespace ef

using namespace ef;

extern "C" int ef_fp64_probe(int op, int64_t iters, double* d_sink, double* ops_per_s, double* ms, void* stream)
{
    if (op < 0 || op > 2 || iters < 1 || !d_sink || !ops_per_s) return EF_ERR_ARG;
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
