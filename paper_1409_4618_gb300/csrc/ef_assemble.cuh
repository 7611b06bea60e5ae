// Loading one element (node ids, coordinates, signs) and evaluating its
// local matrices; shared by every kernel that computes element matrices.
#pragma once

#include <type_traits>

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

template <int VAR>
__device__ __forceinline__ void load_coords(const double* __restrict__ nodes, const int32_t (&g)[ElemTraits<VAR>::NV],
                                            double (&p)[ElemTraits<VAR>::NV][ElemTraits<VAR>::DIM])
{
    using E = ElemTraits<VAR>;
#pragma unroll
    for (int a = 0; a < E::NV; a++)
#pragma unroll
        for (int c = 0; c < E::DIM; c++) p[a][c] = __ldg(nodes + (int64_t)g[a] * E::DIM + c);
}

template <int VAR>
__device__ __forceinline__ void load_element(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                             const double* __restrict__ coeffK, const double* __restrict__ coeffM,
                                             int64_t e, int32_t (&g)[ElemTraits<VAR>::NV],
                                             double (&p)[ElemTraits<VAR>::NV][ElemTraits<VAR>::DIM], double& sigmaK,
                                             double& sigmaM)
{
    load_ids<VAR>(elems, e, g);
    load_coords<VAR>(nodes, g, p);
    sigmaK = coeffK ? __ldg(coeffK + e) : 1.0;
    sigmaM = coeffM == coeffK ? sigmaK : (coeffM ? __ldg(coeffM + e) : 1.0);
}

// Numbers carried from an element routine's first part (all its products) to
// its second (additions and FMAs).
template <int VAR>
struct ScaledTraits {
    static constexpr int N = (VAR == NED3 || VAR == RT3) ? 12 : TriScaled<VAR == NED2 ? 2 : 0>::N;
};

template <int VAR, class MUL, class FK>
__device__ __forceinline__ bool element_scaled(MUL& mul, const FK& f,
                                               const double (&p)[ElemTraits<VAR>::NV][ElemTraits<VAR>::DIM],
                                               double sigmaK, double sigmaM, double (&s)[ScaledTraits<VAR>::N])
{
    if constexpr (VAR == NED3)
        return ned3_scaled(mul, f, p, sigmaK, sigmaM, s);
    else if constexpr (VAR == RT3)
        return rt3_scaled(mul, f, p, sigmaK, sigmaM, s);
    else
        return tri_scaled<VAR == NED2 ? 2 : 0>(mul, f, p, sigmaK, sigmaM, s);
}

// Signed local K, M upper triangles of element e, K times its coefficient in
// coeffK and M times its coefficient in coeffM (NULL: 1); true if degenerate.
// With INT_MUL the products run on the integer pipes (IntMul). An element in
// which an operand or a product leaves the normal numbers and zero
// (subnormal, infinite, NaN, overflowing: IntMul sets off) is repeated with
// the FP64 multiply from its data loaded again (so that none of it has to
// stay in registers meanwhile). Either way the entries are those of the
// routine with FP64 products, bit for bit, so a kernel may take whichever
// form runs faster in it (the integer form needs more registers). Likewise
// REG_CONST: additions as FMAs with per-thread constants (FpK, the FP64
// pipe's full rate) or plain (FpLit, three registers fewer); same bits.
template <int VAR, bool INT_MUL = true, bool REG_CONST = true>
__device__ __forceinline__ bool compute_element(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                                const double* __restrict__ coeffK, const double* __restrict__ coeffM,
                                                int64_t e, double (&Kq)[ElemTraits<VAR>::NP],
                                                double (&Mq)[ElemTraits<VAR>::NP])
{
    using E = ElemTraits<VAR>;
    const std::conditional_t<REG_CONST, FpK, FpLit> f;
    double s[ScaledTraits<VAR>::N];
    uint32_t neg;
    bool bad;
    {
        int32_t g[E::NV];
        double p[E::NV][E::DIM], sigmaK, sigmaM;
        load_element<VAR>(elems, nodes, coeffK, coeffM, e, g, p, sigmaK, sigmaM);
        neg = sign_bits<VAR>(g);
        if constexpr (!INT_MUL) {
            FpMul fm;
            bad = element_scaled<VAR>(fm, f, p, sigmaK, sigmaM, s);
        } else {
            IntMul im;
            bad = element_scaled<VAR>(im, f, p, sigmaK, sigmaM, s);
            if (im.off) {
                // the index through an opaque move: the loads are not merged with the ones above
                int64_t e2 = e;
                asm volatile("" : "+l"(e2));
                load_element<VAR>(elems, nodes, coeffK, coeffM, e2, g, p, sigmaK, sigmaM);
                FpMul fm;
                bad = element_scaled<VAR>(fm, f, p, sigmaK, sigmaM, s);
            }
        }
    }
    if constexpr (VAR == NED3)
        ned3_entries(f, s, neg, Kq, Mq);
    else if constexpr (VAR == RT3)
        rt3_entries(f, s, neg, Kq, Mq);
    else
        tri_entries<VAR == NED2 ? 2 : 0>(f, s, neg, Kq, Mq);
    return bad;
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
