// Per-element local matrices in closed form (FP64), shared by the element
// kernels of the two-pass and fused paths.
//
// Each function returns the upper triangle (k <= l, row-major) of the
// signed local K and M of one element, K times the element's coefficient
// sigmaK and M times sigmaM (the same sigma in the paper's assembly; the
// eddy-current problem of Sec. 4.2 weights K by 1/mu and M by kappa). Below,
// sigma stands for the coefficient of the matrix in question:
//
//   RT0 (Eq. RT0local2 with Piola map RT0piola): with eta_k = x - p_opp(k)
//   (Sec. 2.1, the opposite vertex of DOF k), B eta_k(xhat) = x - P_a, so
//     M_kl = s_k s_l sigma / det^2 * int_K (x - P_a).(x - P_b) dx,
//     K_kl = s_k s_l sigma (div eta)^2 |Khat| / |det|
//   and int_K lambda_i lambda_j = |K| (1 + delta_ij) / ((d+1)(d+2)) gives,
//   with y_i = P_i - P_0, S = sum_i y_i, H = Gram(y_1..y_d):
//     int_K (x-P_a).(x-P_b) = |K|/((d+1)(d+2)) [S.S + tr H - (d+2) S.(y_a+y_b) + (d+1)(d+2) y_a.y_b].
//   Nedelec (Sec. 2.4, Ned0piola1-3): B^-T eta_k is the Whitney form
//   lambda_t grad lambda_h - lambda_h grad lambda_t of its edge (t -> h), so
//     M_(ab)(cd) = sigma |K|/((d+1)(d+2)) [(1+d_ac)G_bd - (1+d_ad)G_bc - (1+d_bc)G_ad + (1+d_bd)G_ac],
//   G_ij = grad lambda_i . grad lambda_j = adj(H)_ij / det^2 (rows 1..d of
//   B^-1 scaled by det), grad lambda_0 = -sum_i grad lambda_i. In 3D,
//   B curl eta_k = 2 w_k with w = (e3-e2, e1-e3, e2-e1, e3, e1, e2), e_i the
//   columns of B, so K_kl = (2 sigma / (3 |det|)) w_k . w_l, a combination of
//   the entries of H = B^T B. In 2D every curl is 2/det, K_kl = 2 sigma/|det|.
//
// Signs are applied by flipping the IEEE sign bit (integer XOR), so they cost
// no floating-point work. |det B| enters only through r = 1/|det B|, with det B
// from the triple product (accurate to cond(B) eps, also on nearly flat
// elements) and r by Newton-Raphson steps (recip_positive).
//
// Each routine has a first part holding all of its products (the MUL policy:
// IntMul on the integer pipes or FpMul, ef_intmul.cuh) and a second part of
// additions and FMAs (the FK policy: FpK with full-rate DFMA forms or FpLit,
// ef_fp64.cuh). Every combination gives the same bits; the kernels pick the
// fastest for their register budget.
#pragma once

#include <stdint.h>

#include "ef_fp64.cuh"
#include "ef_intmul.cuh"

namespace ef {

// local DOF entities (Fig. 1), 0-based
__device__ __constant__ const int8_t kEdge2[3][2] = {{1, 2}, {2, 0}, {0, 1}};
__device__ __constant__ const int8_t kEdge3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {2, 3}, {3, 1}};
__device__ __constant__ const int8_t kFace3[4][4] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 3, 1}, {1, 2, 3, 0}};

// Sign flips and absolute values as 32-bit integer operations on the high
// word: written on the 64-bit pattern, the compiler turned some of them into
// FP64 additions (measured: 9 FP64 instructions per 3D Nedelec element), and
// the FP64 pipe bounds the element kernels.
__device__ __forceinline__ double flip_if(double x, uint32_t f)
{
    return __hiloint2double(__double2hiint(x) ^ (int)((f & 1u) << 31), __double2loint(x));
}

__device__ __forceinline__ double abs_bits(double x)
{
    return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}

// Orientation sign bits (bit k set iff s_k = -1), from global node ids only.
// Edges: s = +1 iff id(tail) > id(head). Faces: s = -parity of the
// permutation (face nodes by ascending id, opposite node).
template <int VAR>
__device__ __forceinline__ uint32_t sign_bits(const int32_t* g)
{
    uint32_t bits = 0;
    if (VAR == 1) {  // RT3: faces
#pragma unroll
        for (int k = 0; k < 4; k++) {
            int a = kFace3[k][0], b = kFace3[k][1], c = kFace3[k][2];
            // inversions among the three face nodes when sorted by id, relative to (a,b,c)
            int inv = (g[a] > g[b]) + (g[a] > g[c]) + (g[b] > g[c]);
            // positions: sorted face nodes keep the relative order of (a,b,c) up to `inv`
            // inversions; the opposite node 3-k comes last. Inversions of the full
            // permutation = inv + (number of face positions greater than the opposite one).
            int opp = 3 - k;
            int tail = (a > opp) + (b > opp) + (c > opp);
            int parity_even = ((inv + tail) & 1) == 0;
            bits |= (uint32_t)parity_even << k;   // s = -1 for even permutations
        }
    } else if (VAR == 3) {
#pragma unroll
        for (int k = 0; k < 6; k++) bits |= (uint32_t)(g[kEdge3[k][0]] < g[kEdge3[k][1]]) << k;
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) bits |= (uint32_t)(g[kEdge2[k][0]] < g[kEdge2[k][1]]) << k;
    }
    return bits;
}

// 2x exactly, as x + x gives it, on the integer pipe only: for normal x whose
// double stays finite, add one to the exponent field; zero and subnormal x
// shift their magnitude left (a carry into the exponent field is exact);
// 2x above the largest double is infinity; infinity stays, NaN is made quiet.
__device__ __forceinline__ double twice(double x)
{
    const uint64_t b = bits_of(x);
    const uint64_t s = b & 0x8000000000000000ull, m = b & 0x7fffffffffffffffull;
    const unsigned ex = (unsigned)(m >> 52);
    uint64_t r;
    if (ex - 1u < 0x7fdu)
        r = b + (1ull << 52);
    else if (ex == 0u)
        r = s | (m << 1);
    else if (ex == 0x7feu)
        r = s | 0x7ff0000000000000ull;
    else
        r = b | (m > 0x7ff0000000000000ull ? 0x0008000000000000ull : 0ull);
    return double_of(r);
}

// |det B| that is not a positive normal number (zero, below 2^-1022, or not
// finite) marks a degenerate element; tested on the bit pattern.
__device__ __forceinline__ bool not_positive(double x)
{
    const long long b = (long long)bits_of(x);
    return b < 0x0010000000000000ll || (b & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;
}

// 1/x for a positive normal x by Newton-Raphson iteration for the reciprocal,
// y <- y + y (1 - x y) (quadratic convergence: a relative error e becomes e^2
// plus one rounding), started from the hardware's approximate reciprocal (PTX
// rcp.approx.ftz.f64, relative error below 2^-22): two steps reach double
// precision to about one ulp. Four DFMA on the FP64 pipe, which bounds the
// element kernels, against the longer sequence of the IEEE division. Callers
// flag x outside the positive normals as degenerate (not_positive); one = 1
// from a per-thread register keeps the FMAs at the pipe's full rate (FpK).
__device__ __forceinline__ double recip_positive(double x, double one = 1.0)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, one), y);
    return fma(y, fma(-x, y, one), y);
}

// ---- 3D Nedelec: 21 + 21 upper entries ---------------------------------------
// Every product of the routine is in its first part, which reduces the element
// to twelve numbers: s[0..5] = h = (2 sigma_K / (3|det|)) H and s[6..11] = g =
// (sigma_M / (120|det|)) adj(H) (upper triangles, order 11, 22, 33, 12, 13, 23).
// MUL forms the products (IntMul on the integer pipes, or FpMul); true if
// degenerate.
template <class MUL, class FK>
__device__ __forceinline__ bool ned3_scaled(MUL& mul, const FK& f, const double (&p)[4][3], double sigmaK,
                                            double sigmaM, double (&s)[12])
{
    const double e1x = f.sub(p[1][0], p[0][0]), e1y = f.sub(p[1][1], p[0][1]), e1z = f.sub(p[1][2], p[0][2]);
    const double e2x = f.sub(p[2][0], p[0][0]), e2y = f.sub(p[2][1], p[0][1]), e2z = f.sub(p[2][2], p[0][2]);
    const double e3x = f.sub(p[3][0], p[0][0]), e3y = f.sub(p[3][1], p[0][1]), e3z = f.sub(p[3][2], p[0][2]);
    const double H11 = fma(e1z, e1z, fma(e1y, e1y, mul(e1x, e1x)));
    const double H22 = fma(e2z, e2z, fma(e2y, e2y, mul(e2x, e2x)));
    const double H33 = fma(e3z, e3z, fma(e3y, e3y, mul(e3x, e3x)));
    const double H12 = fma(e1z, e2z, fma(e1y, e2y, mul(e1x, e2x)));
    const double H13 = fma(e1z, e3z, fma(e1y, e3y, mul(e1x, e3x)));
    const double H23 = fma(e2z, e3z, fma(e2y, e3y, mul(e2x, e3x)));
    // adj(H) = det(B)^2 * Gram(grad lambda_1..3)
    const double A11 = fma(H22, H33, -mul(H23, H23));
    const double A22 = fma(H11, H33, -mul(H13, H13));
    const double A33 = fma(H11, H22, -mul(H12, H12));
    const double A12 = fma(H13, H23, -mul(H12, H33));
    const double A13 = fma(H12, H23, -mul(H13, H22));
    const double A23 = fma(H12, H13, -mul(H11, H23));
    // det B by the triple product e1 . (e2 x e3): its error grows like cond(B),
    // where det(H) = det(B)^2 from the Gram matrix would grow like cond(B)^2
    const double cx = fma(e2y, e3z, -mul(e2z, e3y)), cy = fma(e2z, e3x, -mul(e2x, e3z)), cz = fma(e2x, e3y, -mul(e2y, e3x));
    const double adet = abs_bits(fma(e1z, cz, fma(e1y, cy, mul(e1x, cx))));
    const bool bad = not_positive(adet);
    const double r = recip_positive(adet, f.one);
    const double srK = mul(sigmaK, r), srM = mul(sigmaM, r);

    // K_kl = (2 sigma / (3|det|)) w_k . w_l
    const double cK = mul(srK, 2.0 / 3.0);
    s[0] = mul(cK, H11); s[1] = mul(cK, H22); s[2] = mul(cK, H33);
    s[3] = mul(cK, H12); s[4] = mul(cK, H13); s[5] = mul(cK, H23);
    const double cM = mul(srM, 1.0 / 120.0);
    s[6] = mul(cM, A11); s[7] = mul(cM, A22); s[8] = mul(cM, A33);
    s[9] = mul(cM, A12); s[10] = mul(cM, A13); s[11] = mul(cM, A23);
    return bad;
}

// The 21 + 21 signed entries from h and g: additions and FMAs only.
template <class FK>
__device__ __forceinline__ void ned3_entries(const FK& f, const double (&s)[12], uint32_t neg, double (&Kq)[21],
                                             double (&Mq)[21])
{
    const double h11 = s[0], h22 = s[1], h33 = s[2], h12 = s[3], h13 = s[4], h23 = s[5];
    const double k03 = f.sub(h33, h23), k04 = f.sub(h13, h12), k05 = f.sub(h23, h22);
    const double k13 = f.sub(h13, h33), k14 = f.sub(h11, h13), k15 = f.sub(h12, h23);
    const double k23 = f.sub(h23, h13), k24 = f.sub(h12, h11), k25 = f.sub(h22, h12);
    const double k00 = f.sub(k03, k05), k11 = f.sub(k14, k13), k22 = f.sub(k25, k24);
    const double k01 = f.sub(k04, k03), k02 = f.sub(k05, k04), k12 = f.sub(k15, k14);
    // M: Whitney-form combinations of g = sigma/(120|det|) adj(H) (the
    // scaled Gram matrix of grad lambda_1..3). With p_ab = -G_ab for the six
    // node pairs (the row of node 0 from the zero row sums), S_a = G_aa, and
    // o = p_e + p_e' over the three pairs of opposite edges (e, e'), the
    // Whitney mass entries |K|/20 int (lambda_a grad lambda_b - ...) . (...)
    // reduce to: diagonal 2 (S_a + S_b + p_ab) = 2 (o_i + o_j + 3 p_e) (o_i,
    // o_j the two other pairs); edges sharing node s with other ends u, v:
    // +-(2 S_s - (p_uv + o(uv))); disjoint edges (a,b), (c,d): p_ad + p_bc -
    // p_ac - p_bd, a difference of two o's. 41 operations after the scaling.
    const double g11 = s[6], g22 = s[7], g33 = s[8], g12 = s[9], g13 = s[10], g23 = s[11];
    const double p01 = f.add(f.add(g11, g12), g13), p02 = f.add(f.add(g12, g22), g23),
                 p03 = f.add(f.add(g13, g23), g33);   // p12 = -g12, ...
    const double S0 = f.add(f.add(p01, p02), p03);
    const double oA = f.sub(p01, g23), oB = f.sub(p02, g13), oC = f.sub(p03, g12);   // {01,23}, {02,13}, {03,12}
    const double QA = f.add(oB, oC), QB = f.add(oA, oC), QC = f.add(oA, oB);
    const double r01 = f.add(oA, p01), r02 = f.add(oB, p02), r03 = f.add(oC, p03);
    const double r12 = f.sub(oC, g12), r13 = f.sub(oB, g13), r23 = f.sub(oA, g23);

    // order: (0,0)..(0,5), (1,1)..(1,5), (2,2)..(2,5), (3,3)..(3,5), (4,4),(4,5), (5,5)
    Kq[0] = k00; Kq[1] = k01; Kq[2] = k02; Kq[3] = k03; Kq[4] = k04; Kq[5] = k05;
    Kq[6] = k11; Kq[7] = k12; Kq[8] = k13; Kq[9] = k14; Kq[10] = k15;
    Kq[11] = k22; Kq[12] = k23; Kq[13] = k24; Kq[14] = k25;
    Kq[15] = h33; Kq[16] = h13; Kq[17] = h23;
    Kq[18] = h11; Kq[19] = h12;
    Kq[20] = h22;

    // local edges 0..5 = (0,1), (0,2), (0,3), (1,2), (2,3), (3,1)
    const double two = f.two, three = f.three;
    Mq[0] = twice(fma(three, p01, QA));
    Mq[1] = fma(two, S0, -r12);
    Mq[2] = fma(two, S0, -r13);
    Mq[3] = fma(-two, g11, r02);
    Mq[4] = f.sub(oC, oB);
    Mq[5] = fma(two, g11, -r03);
    Mq[6] = twice(fma(three, p02, QB));
    Mq[7] = fma(two, S0, -r23);
    Mq[8] = fma(two, g22, -r01);
    Mq[9] = fma(-two, g22, r03);
    Mq[10] = f.sub(oA, oC);
    Mq[11] = twice(fma(three, p03, QC));
    Mq[12] = f.sub(oB, oA);
    Mq[13] = fma(two, g33, -r02);
    Mq[14] = fma(-two, g33, r01);
    Mq[15] = twice(fma(-three, g12, QC));
    Mq[16] = fma(-two, g22, r13);
    Mq[17] = fma(-two, g11, r23);
    Mq[18] = twice(fma(-three, g23, QA));
    Mq[19] = fma(-two, g33, r12);
    Mq[20] = twice(fma(-three, g13, QB));

    // signs s_k s_l on the off-diagonal pairs
    int q = 0;
#pragma unroll
    for (int k = 0; k < 6; k++)
#pragma unroll
        for (int l = k; l < 6; l++, q++) {
            uint32_t f = (neg >> k) ^ (neg >> l);
            Kq[q] = flip_if(Kq[q], f);
            Mq[q] = flip_if(Mq[q], f);
        }
}

// ---- 3D RT0: 10 + 10 upper entries (DOF k <-> opposite vertex 3-k) ---------
// First part (every product): s = (H11, H22, H33, H12, H13, H23, m20, c0s, q1,
// q2, q3, kv) in the notation below.
template <class MUL, class FK>
__device__ __forceinline__ bool rt3_scaled(MUL& mul, const FK& f, const double (&p)[4][3], double sigmaK,
                                           double sigmaM, double (&s)[12])
{
    const double e1x = f.sub(p[1][0], p[0][0]), e1y = f.sub(p[1][1], p[0][1]), e1z = f.sub(p[1][2], p[0][2]);
    const double e2x = f.sub(p[2][0], p[0][0]), e2y = f.sub(p[2][1], p[0][1]), e2z = f.sub(p[2][2], p[0][2]);
    const double e3x = f.sub(p[3][0], p[0][0]), e3y = f.sub(p[3][1], p[0][1]), e3z = f.sub(p[3][2], p[0][2]);
    const double H11 = fma(e1z, e1z, fma(e1y, e1y, mul(e1x, e1x)));
    const double H22 = fma(e2z, e2z, fma(e2y, e2y, mul(e2x, e2x)));
    const double H33 = fma(e3z, e3z, fma(e3y, e3y, mul(e3x, e3x)));
    const double H12 = fma(e1z, e2z, fma(e1y, e2y, mul(e1x, e2x)));
    const double H13 = fma(e1z, e3z, fma(e1y, e3y, mul(e1x, e3x)));
    const double H23 = fma(e2z, e3z, fma(e2y, e3y, mul(e2x, e3x)));
    const double cx = fma(e2y, e3z, -mul(e2z, e3y)), cy = fma(e2z, e3x, -mul(e2x, e3z)), cz = fma(e2x, e3y, -mul(e2y, e3x));
    const double adet = abs_bits(fma(e1z, cz, fma(e1y, cy, mul(e1x, cx))));
    const bool bad = not_positive(adet);
    const double r = recip_positive(adet, f.one);
    const double srK = mul(sigmaK, r), srM = mul(sigmaM, r);
    // M: sigma/(120|det|) [c0 - 5 (S.y_a + S.y_b) + 20 y_a.y_b]
    const double r1 = f.add(f.add(H11, H12), H13), r2 = f.add(f.add(H12, H22), H23), r3 = f.add(f.add(H13, H23), H33);
    const double c0 = f.add(f.add(f.add(r1, r2), r3), f.add(f.add(H11, H22), H33));
    const double cM = mul(srM, 1.0 / 120.0);
    const double m5 = mul(-5.0, cM);
    s[0] = H11; s[1] = H22; s[2] = H33; s[3] = H12; s[4] = H13; s[5] = H23;
    s[6] = mul(20.0, cM);
    s[7] = mul(c0, cM);
    s[8] = mul(r1, m5); s[9] = mul(r2, m5); s[10] = mul(r3, m5);
    s[11] = mul(srK, 1.5);   // (div eta)^2 |Khat| = 9/6
    return bad;
}

template <class FK>
__device__ __forceinline__ void rt3_entries(const FK& f, const double (&s)[12], uint32_t neg, double (&Kq)[10],
                                            double (&Mq)[10])
{
    const double H11 = s[0], H22 = s[1], H33 = s[2], H12 = s[3], H13 = s[4], H23 = s[5];
    const double m20 = s[6], c0s = s[7], q1 = s[8], q2 = s[9], q3 = s[10], kv = s[11];
    const double t1 = f.add(c0s, q1), t2 = f.add(c0s, q2), t3 = f.add(c0s, q3);
    // DOF k <-> opposite vertex a = 3 - k; vertex 0 has y_0 = 0
    // (0,0):a=3  (0,1):3,2  (0,2):3,1  (0,3):3,0  (1,1):2  (1,2):2,1  (1,3):2,0  (2,2):1  (2,3):1,0  (3,3):0
    Mq[0] = fma(m20, H33, f.add(t3, q3));
    Mq[1] = fma(m20, H23, f.add(t3, q2));
    Mq[2] = fma(m20, H13, f.add(t3, q1));
    Mq[3] = t3;
    Mq[4] = fma(m20, H22, f.add(t2, q2));
    Mq[5] = fma(m20, H12, f.add(t2, q1));
    Mq[6] = t2;
    Mq[7] = fma(m20, H11, f.add(t1, q1));
    Mq[8] = t1;
    Mq[9] = c0s;
    int q = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int l = k; l < 4; l++, q++) {
            uint32_t f = (neg >> k) ^ (neg >> l);
            Kq[q] = flip_if(kv, f);
            Mq[q] = flip_if(Mq[q], f);
        }
}

// ---- 2D RT0 (VAR 0) and 2D Nedelec (VAR 2): 6 + 6 upper entries ------------
// First part (every product): RT0 s = (H11, H12, H22, m12, c0s, q1, q2, kv),
// Nedelec s = (g11, g22, g12, kv) in the notation below.
template <int VAR>
struct TriScaled {
    static constexpr int N = VAR == 0 ? 8 : 4;
};

template <int VAR, class MUL, class FK>
__device__ __forceinline__ bool tri_scaled(MUL& mul, const FK& f, const double (&p)[3][2], double sigmaK,
                                           double sigmaM, double (&s)[TriScaled<VAR>::N])
{
    const double e1x = f.sub(p[1][0], p[0][0]), e1y = f.sub(p[1][1], p[0][1]);
    const double e2x = f.sub(p[2][0], p[0][0]), e2y = f.sub(p[2][1], p[0][1]);
    const double H11 = fma(e1y, e1y, mul(e1x, e1x)), H22 = fma(e2y, e2y, mul(e2x, e2x)),
                 H12 = fma(e1y, e2y, mul(e1x, e2x));
    const double adet = abs_bits(fma(e1x, e2y, -mul(e1y, e2x)));
    const bool bad = not_positive(adet);
    const double r = recip_positive(adet, f.one);
    const double srK = mul(sigmaK, r), srM = mul(sigmaM, r);
    const double cM = mul(srM, 1.0 / 24.0);
    const double kv = twice(srK);   // (div eta)^2 |Khat| = 4/2 (RT); curl^2 |Khat| = 4/2 (Ned)
    if constexpr (VAR == 0) {
        // RT0: sigma/(24|det|) [c0 - 4 (S.y_a + S.y_b) + 12 y_a.y_b], DOF k <-> vertex k
        const double r1 = f.add(H11, H12), r2 = f.add(H12, H22);
        const double c0 = f.add(f.add(r1, r2), f.add(H11, H22));
        const double m4 = mul(-4.0, cM);
        s[0] = H11; s[1] = H12; s[2] = H22;
        s[3] = mul(12.0, cM);
        s[4] = mul(c0, cM);
        s[5] = mul(r1, m4); s[6] = mul(r2, m4);
        s[7] = kv;
    } else {
        // Nedelec: Whitney forms on edges (1,2), (2,0), (0,1); g = sigma/(24|det|) adj(H)
        s[0] = mul(cM, H22); s[1] = mul(cM, H11); s[2] = -mul(cM, H12);
        s[3] = kv;
    }
    return bad;
}

template <int VAR, class FK>
__device__ __forceinline__ void tri_entries(const FK& f, const double (&s)[TriScaled<VAR>::N], uint32_t neg,
                                            double (&Kq)[6], double (&Mq)[6])
{
    double kv;
    if constexpr (VAR == 0) {
        const double H11 = s[0], H12 = s[1], H22 = s[2], m12 = s[3], c0s = s[4], q1 = s[5], q2 = s[6];
        kv = s[7];
        const double t1 = f.add(c0s, q1), t2 = f.add(c0s, q2);
        Mq[0] = c0s;                              // (0,0)
        Mq[1] = t1;                               // (0,1)
        Mq[2] = t2;                               // (0,2)
        Mq[3] = fma(m12, H11, f.add(t1, q1));     // (1,1)
        Mq[4] = fma(m12, H12, f.add(t1, q2));     // (1,2)
        Mq[5] = fma(m12, H22, f.add(t2, q2));     // (2,2)
    } else {
        const double g11 = s[0], g22 = s[1], g12 = s[2];
        kv = s[3];
        const double g01 = -f.add(g11, g12), g02 = -f.add(g12, g22);
        const double g00 = -f.add(g01, g02);
        const double two = f.two;
        Mq[0] = twice(f.sub(f.add(g11, g22), g12));
        Mq[1] = fma(-two, g01, f.add(f.sub(g02, g22), g12));
        Mq[2] = fma(-two, g02, f.add(f.sub(g12, g11), g01));
        Mq[3] = twice(f.sub(f.add(g22, g00), g02));
        Mq[4] = fma(-two, g12, f.add(f.sub(g01, g00), g02));
        Mq[5] = twice(f.sub(f.add(g00, g11), g01));
    }
    int q = 0;
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int l = k; l < 3; l++, q++) {
            uint32_t f = (neg >> k) ^ (neg >> l);
            Kq[q] = flip_if(kv, f);
            Mq[q] = flip_if(Mq[q], f);
        }
}

}  // namespace ef
