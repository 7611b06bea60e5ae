// ef_assemble_noalloc: the two-pass assembly with its scratch in a static
// device array, for callers that must not allocate device memory.
//
// Who needs it: code that runs while a CUDA stream capture is open in global
// mode (any cudaMalloc in the process would invalidate that capture), loops
// with a latency budget that cannot absorb the device-wide synchronisation a
// cudaMalloc or cudaFree may imply, and applications whose device memory is
// owned by another allocator with a fixed budget. This entry point calls no
// allocating routine: the element matrices go to the file-scope array
// g_scratch below, which every GPU that loads this library holds until the
// process exits.
//
// The array's name in host code is a host-side stand-in, not a device
// address, so the host looks up the real address once per device with
// cudaGetSymbolAddress (with that device current) and passes it to the
// kernels; device code could name the array directly.
#include <mutex>

#include "ef_assemble.cuh"
#include "ef_internal.cuh"

namespace ef {
namespace {

constexpr int TPB = 256;
constexpr size_t kScratchBytes = (size_t)64 << 20;   // EF_NOALLOC_SCRATCH_BYTES in edgefem.h
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchBytes / sizeof(double)];

std::mutex g_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(double** out)
{
    int dev = 0;
    EF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return EF_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) {
            set_last_error("cudaGetSymbolAddress(g_scratch)", e);
            return EF_ERR_CUDA;
        }
        g_addr[dev] = (double*)ptr;
    }
    *out = g_addr[dev];
    return EF_OK;
}

template <int VAR>
__global__ void __launch_bounds__(TPB) k_element_static(const int32_t* __restrict__ elems,
                                                        const double* __restrict__ nodes,
                                                        const double* __restrict__ coeff, int64_t T,
                                                        double* __restrict__ local, int* status)
{
    using E = ElemTraits<VAR>;
    const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (e >= T) return;
    double Kq[E::NP], Mq[E::NP];
    if (compute_element<VAR>(elems, nodes, coeff, coeff, e, Kq, Mq)) atomicOr(status, ST_DEGENERATE);
#pragma unroll
    for (int q = 0; q < E::NP; q++) {
        local[(int64_t)q * T + e] = Kq[q];
        local[(int64_t)(E::NP + q) * T + e] = Mq[q];
    }
}

__global__ void __launch_bounds__(TPB) k_sum_static(const uint32_t* __restrict__ seg, const uint32_t* __restrict__ perm,
                                                    const uint32_t* __restrict__ pos_up,
                                                    const uint32_t* __restrict__ pos_lo,
                                                    const double* __restrict__ localK,
                                                    const double* __restrict__ localM, int64_t U,
                                                    double* __restrict__ K, double* __restrict__ M)
{
    const int64_t u = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (u >= U) return;
    const uint32_t s0 = seg[u], s1 = seg[u + 1];
    uint32_t idx = perm[s0];
    double k = localK[idx], m = localM[idx];
    for (uint32_t s = s0 + 1; s < s1; s++) {
        idx = perm[s];
        k += localK[idx];
        m += localM[idx];
    }
    uint32_t p = pos_up[u];
    K[p] = k;
    M[p] = m;
    p = pos_lo[u];
    if (p != 0xffffffffu) {
        K[p] = k;
        M[p] = m;
    }
}

}  // namespace
}  // namespace ef

using namespace ef;

extern "C" int ef_assemble_noalloc(const ef_plan* plan, const double* d_nodes, const double* d_coeff,
                                   double* d_Kval, double* d_Mval, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    if (plan->T > 0 && (!d_nodes || !d_Kval || !d_Mval)) return EF_ERR_ARG;
    const size_t need = (size_t)plan->T * plan->np * 2 * sizeof(double);
    if (need > kScratchBytes) {
        set_last_message("ef_assemble_noalloc: this plan needs %zu bytes of scratch, more than the "
                         "EF_NOALLOC_SCRATCH_BYTES = %zu of the static array",
                         need, kScratchBytes);
        return EF_ERR_SIZE;
    }
    if (plan->T == 0) return EF_OK;
    double* local = nullptr;
    EF_TRY(scratch_address(&local));
    // Nothing in the scratch has to start at zero: the element kernel writes
    // every entry the sum kernel reads, so leftovers of an earlier call are
    // never used.
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned ge = (unsigned)((plan->T + TPB - 1) / TPB);
    switch (plan->variant) {
        case RT2: k_element_static<RT2><<<ge, TPB, 0, s>>>(plan->d_elems, d_nodes, d_coeff, plan->T, local, plan->d_status); break;
        case NED2: k_element_static<NED2><<<ge, TPB, 0, s>>>(plan->d_elems, d_nodes, d_coeff, plan->T, local, plan->d_status); break;
        case RT3: k_element_static<RT3><<<ge, TPB, 0, s>>>(plan->d_elems, d_nodes, d_coeff, plan->T, local, plan->d_status); break;
        default: k_element_static<NED3><<<ge, TPB, 0, s>>>(plan->d_elems, d_nodes, d_coeff, plan->T, local, plan->d_status); break;
    }
    const unsigned gu = (unsigned)((plan->U + TPB - 1) / TPB);
    k_sum_static<<<gu, TPB, 0, s>>>(plan->d_seg, plan->d_perm, plan->d_pos_up, plan->d_pos_lo, local,
                                    local + (int64_t)plan->np * plan->T, plan->U, d_Kval, d_Mval);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}
