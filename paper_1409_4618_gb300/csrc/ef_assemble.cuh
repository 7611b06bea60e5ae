// Loading one element (node ids, coordinates, signs) and evaluating its
// local matrices; shared by every kernel that computes element matrices.
#pragma once

#include "ef_element.cuh"
#include "ef_internal.cuh"

namespace ef {

template <int VAR>
struct ElemTraits {
    static constexpr int DIM = (VAR == RT2 || VAR == NED2) ? 2 : 3;
    static constexpr int NV = DIM + 1;
    static constexpr int NL = VAR == RT3 ? 4 : (VAR == NED3 ? 6 : 3);
    static constexpr int NP = NL * (NL + 1) / 2;
};

template <int VAR>
__device__ __forceinline__ void load_ids(const int32_t* __restrict__ elems, int64_t e, int32_t (&g)[ElemTraits<VAR>::NV])
{
    if (ElemTraits<VAR>::DIM == 3) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(elems) + e);  // plan copy is 16-byte aligned
        g[0] = v.x;
        g[1] = v.y;
        g[2] = v.z;
        g[ElemTraits<VAR>::NV - 1] = v.w;
    } else {
#pragma unroll
        for (int a = 0; a < ElemTraits<VAR>::NV; a++) g[a] = __ldg(elems + e * ElemTraits<VAR>::NV + a);
    }
}

// Signed local K, M upper triangles of element e, K times sigmaK and M times
// sigmaM; true if degenerate.
template <int VAR>
__device__ __forceinline__ bool compute_element(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                                double sigmaK, double sigmaM, int64_t e,
                                                double (&Kq)[ElemTraits<VAR>::NP], double (&Mq)[ElemTraits<VAR>::NP])
{
    using E = ElemTraits<VAR>;
    int32_t g[E::NV];
    load_ids<VAR>(elems, e, g);
    const uint32_t neg = sign_bits<VAR>(g);
    if constexpr (E::DIM == 3) {
        double p[4][3];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) p[a][c] = __ldg(nodes + (int64_t)g[a] * 3 + c);
        if constexpr (VAR == NED3)
            return ned3_local(p, sigmaK, sigmaM, neg, Kq, Mq);
        else
            return rt3_local(p, sigmaK, sigmaM, neg, Kq, Mq);
    } else {
        double p[3][2];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c < 2; c++) p[a][c] = __ldg(nodes + (int64_t)g[a] * 2 + c);
        return tri_local<VAR == NED2 ? 2 : 0>(p, sigmaK, sigmaM, neg, Kq, Mq);
    }
}

// ---- the fixed-order sum of one aligned block of work items ------------------
//
// Work item i sums list[wseg[i] .. wseg[i+1]): the contributions of one upper
// nonzero, contiguous and in ascending element order. A block owns the
// aligned range of SB work items [base, base + SB) (only those in [w0, w1)
// are summed here), keeps the sums in shared memory, and then stores them in
// ascending (r, c) and in ascending (c, r) CSR position (the plan's per-block
// store orders st_up, st_lo: the t-th entry is the block-local item stored
// t-th), so that the stores of a warp fall on few adjacent sectors; scattered
// 8-byte stores are bound by the L2's transaction rate.
constexpr int SB = 256;
using StoreIdx = uint8_t;

__device__ __forceinline__ void sum_block(int64_t base, int64_t w0, int64_t w1, int64_t U,
                                          const uint32_t* __restrict__ wseg, const uint32_t* __restrict__ wpos_up,
                                          const uint32_t* __restrict__ wpos_lo, const StoreIdx* __restrict__ st_up,
                                          const StoreIdx* __restrict__ st_lo, const double2* __restrict__ list,
                                          double* __restrict__ K, double* __restrict__ M)
{
    __shared__ double sk[SB], sm[SB];
    __shared__ uint32_t su[SB], sl[SB];
    const int t = threadIdx.x;
    {
        const int64_t i = base + t;
        if (i >= w0 && i < w1) {
            const uint32_t s0 = wseg[i], s1 = wseg[i + 1];
            su[t] = wpos_up[i];
            sl[t] = wpos_lo[i];
            double2 v = list[s0];
            double k = v.x, m = v.y;
            for (uint32_t s = s0 + 1; s < s1; s++) {
                v = list[s];
                k += v.x;
                m += v.y;
            }
            sk[t] = k;
            sm[t] = m;
        }
    }
    __syncthreads();
    {
        if (base + t < U) {
            int q = st_up[base + t];
            if (base + q >= w0 && base + q < w1) {
                const uint32_t p = su[q];
                K[p] = sk[q];
                M[p] = sm[q];
            }
            q = st_lo[base + t];
            if (base + q >= w0 && base + q < w1) {
                const uint32_t p = sl[q];
                if (p != 0xffffffffu) {
                    K[p] = sk[q];
                    M[p] = sm[q];
                }
            }
        }
    }
}

}  // namespace ef
