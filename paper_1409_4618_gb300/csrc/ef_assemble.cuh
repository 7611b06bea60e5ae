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

}  // namespace ef
