// Vectorised integration over the mesh (Sec. 3.1): the squared L2 norm of a
// function, sum over elements K and quadrature points q of
// w_q |det B_K| |f(F_K(xhat_q))|^2, with the loop over quadrature points and
// every element at once, as in the paper's norm_L2.
//
// GB300 form. The caller evaluates its function at the physical quadrature
// points (ef_quad_points), stored point-major, [q][element][component], so
// that for each point the elements are contiguous (the paper's F_K_ip) and
// every load and store of the kernels below is coalesced. ef_fe_values
// evaluates the finite-element function of a DOF vector (Piola-mapped,
// signed basis, Sec. 2.1-2.3) at the same points; ef_norm_l2 forms the
// per-element and total norms of f, or of f minus that FE function, in one
// kernel. Totals are fixed-order sums (per-CTA tree, then one CTA over the
// partials): the same bits on every run.
//
// The rule: collapsed Gauss-Legendre product rule with n points per
// direction, triangle xhat = (u, v (1 - u)), weight J = 1 - u; tetrahedron
// xhat = (u, v (1 - u), s (1 - u)(1 - v)), J = (1 - u)^2 (1 - v). It is exact
// for polynomials of total degree 2n - dim (n = 1 .. EF_QUAD_MAX_N).
#include <math.h>
#include <string.h>

#include "ef_assemble.cuh"
#include "ef_internal.cuh"

namespace ef {
namespace {

constexpr int ITPB = 256;

struct Rule1D {
    double t[EF_QUAD_MAX_N];   // Gauss-Legendre nodes on [0, 1]
    double w[EF_QUAD_MAX_N];   // weights, summing to 1
    int n;
};

// Gauss-Legendre nodes and weights on [0, 1]: roots of P_n by Newton's method
// from the asymptotic guess cos(pi (4i + 3) / (4n + 2)), weight
// 2 / ((1 - x^2) P_n'(x)^2) on [-1, 1], halved for [0, 1].
void legendre_rule(int n, Rule1D* r)
{
    r->n = n;
    for (int i = 0; i < n; i++) {
        double x = cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double dpn = 1.0;
        for (int it = 0; it < 64; it++) {
            // P_n(x) and P_n'(x) by the three-term recurrence
            double pm1 = 0.0, p = 1.0;
            for (int k = 0; k < n; k++) {
                const double pk1 = ((2.0 * k + 1.0) * x * p - k * pm1) / (k + 1.0);
                pm1 = p;
                p = pk1;
            }
            dpn = n * (pm1 - x * p) / (1.0 - x * x);
            const double dx = p / dpn;
            x -= dx;
            if (fabs(dx) <= 1e-16 * fabs(x) + 1e-300) break;
        }
        // weight from the derivative at the converged root
        double pm1 = 0.0, p = 1.0;
        for (int k = 0; k < n; k++) {
            const double pk1 = ((2.0 * k + 1.0) * x * p - k * pm1) / (k + 1.0);
            pm1 = p;
            p = pk1;
        }
        dpn = n * (pm1 - x * p) / (1.0 - x * x);
        r->t[n - 1 - i] = 0.5 * (1.0 + x);   // ascending on [0, 1]
        r->w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dpn * dpn);
    }
}

// Reference point and weight of point q (q = (i n + j) n + k in 3D, i n + j in 2D).
template <int DIM>
__device__ __forceinline__ double quad_point(const Rule1D& r, int q, double (&xh)[3])
{
    const int n = r.n;
    if (DIM == 3) {
        const int i = q / (n * n), j = (q / n) % n, k = q % n;
        const double u = r.t[i], v = r.t[j], s = r.t[k];
        const double ou = 1.0 - u, ov = 1.0 - v;
        xh[0] = u;
        xh[1] = v * ou;
        xh[2] = s * ou * ov;
        return r.w[i] * r.w[j] * r.w[k] * ou * ou * ov;
    } else {
        const int i = q / n, j = q % n;
        const double u = r.t[i], v = r.t[j];
        xh[0] = u;
        xh[1] = v * (1.0 - u);
        xh[2] = 0.0;
        return r.w[i] * r.w[j] * (1.0 - u);
    }
}

template <int DIM>
__device__ __forceinline__ void load_vertices(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                              int64_t e, double (&p)[4][3])
{
    constexpr int VAR = DIM == 3 ? NED3 : NED2;   // vertex ids do not depend on the element kind
    int32_t g[ElemTraits<VAR>::NV];
    load_ids<VAR>(elems, e, g);
#pragma unroll
    for (int a = 0; a < DIM + 1; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) p[a][c] = c < DIM ? __ldg(nodes + (int64_t)g[a] * DIM + c) : 0.0;
}

// Columns of B (e_i = P_i - P_0) and det B.
template <int DIM>
__device__ __forceinline__ double edge_frame(const double (&p)[4][3], double (&B)[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) B[c][i] = (i < DIM) ? p[i + 1][c] - p[0][c] : 0.0;
    if (DIM == 2) return fma(B[0][0], B[1][1], -(B[1][0] * B[0][1]));
    const double cx = fma(B[1][1], B[2][2], -(B[2][1] * B[1][2]));
    const double cy = fma(B[2][1], B[0][2], -(B[0][1] * B[2][2]));
    const double cz = fma(B[0][1], B[1][2], -(B[1][1] * B[0][2]));
    return fma(B[2][0], cz, fma(B[1][0], cy, B[0][0] * cx));
}

// The FE function v_h = sum_k s_k v[dof_k] phi_k on one element is affine in
// xhat, v_h = V0 + sum_i xhat_i V_i, formed once per element:
// Nedelec (Whitney forms, B^-T eta_k = l_t grad l_h - l_h grad l_t):
//   v_h = sum_ij l_i C_ij grad l_j, C antisymmetric with C_th = s_k v_k for
//   local edge k = (t -> h); with l_0 = 1 - sum_i xhat_i:
//   V0 = sum_j C_0j grad l_j, V_i = sum_j (C_ij - C_0j) grad l_j;
// RT0 (B eta_k = x - P_a, phi_k = B eta_k / det B), x = P_0 + B xhat:
//   v_h = (S x - sum_k c_k P_a(k)) / det B, c_k = s_k v_k, S = sum_k c_k:
//   V0 = (S P_0 - sum_k c_k P_a(k)) / det B, V_i = S B e_i / det B.
template <int VAR>
struct FeAffine {
    static constexpr int DIM = ElemTraits<VAR>::DIM;
    static constexpr bool NED = (VAR == NED2 || VAR == NED3);
    double V0[3], V[3][3];   // V[i] = coefficient of xhat_i

    __device__ __forceinline__ void setup(const double (&p)[4][3], const double (&B)[3][3], double det,
                                          const int32_t* __restrict__ e2d, uint32_t neg,
                                          const double* __restrict__ v, int64_t e)
    {
        constexpr int NL = ElemTraits<VAR>::NL;
        double c[6];
#pragma unroll
        for (int k = 0; k < NL; k++) {
            const double x = __ldg(v + __ldg(e2d + e * NL + k));
            c[k] = ((neg >> k) & 1u) ? -x : x;
        }
        const double rdet = 1.0 / det;
        if (NED) {
            double G[4][3];   // grad lambda_0 .. lambda_DIM: rows of B^-1 = cofactor columns / det
            if (DIM == 3) {
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const int a = (i + 1) % 3, b = (i + 2) % 3;
                    G[i + 1][0] = fma(B[1][a], B[2][b], -(B[2][a] * B[1][b])) * rdet;
                    G[i + 1][1] = fma(B[2][a], B[0][b], -(B[0][a] * B[2][b])) * rdet;
                    G[i + 1][2] = fma(B[0][a], B[1][b], -(B[1][a] * B[0][b])) * rdet;
                }
            } else {
                G[1][0] = B[1][1] * rdet;
                G[1][1] = -B[0][1] * rdet;
                G[2][0] = -B[1][0] * rdet;
                G[2][1] = B[0][0] * rdet;
                G[1][2] = G[2][2] = G[3][0] = G[3][1] = G[3][2] = 0.0;
            }
#pragma unroll
            for (int r = 0; r < 3; r++) G[0][r] = -(G[1][r] + G[2][r] + G[3][r]);
            double C[4][4];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) C[i][j] = 0.0;
#pragma unroll
            for (int k = 0; k < NL; k++) {
                const int t = DIM == 3 ? kEdge3[k][0] : kEdge2[k][0];
                const int h = DIM == 3 ? kEdge3[k][1] : kEdge2[k][1];
                C[t][h] = c[k];
                C[h][t] = -c[k];
            }
#pragma unroll
            for (int r = 0; r < 3; r++) {
                double s0 = 0.0;
#pragma unroll
                for (int j = 1; j < DIM + 1; j++) s0 = fma(C[0][j], G[j][r], s0);
                V0[r] = s0;
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    double si = 0.0;
                    if (i < DIM)
#pragma unroll
                        for (int j = 0; j < DIM + 1; j++) si = fma(C[i + 1][j] - C[0][j], G[j][r], si);
                    V[i][r] = si;
                }
            }
        } else {
            double S = 0.0, Q[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < NL; k++) {
                const int a = DIM == 3 ? 3 - k : k;   // vertex opposite DOF k
                S += c[k];
#pragma unroll
                for (int r = 0; r < 3; r++) Q[r] = fma(c[k], p[a][r], Q[r]);
            }
            const double Sr = S * rdet;
#pragma unroll
            for (int r = 0; r < 3; r++) {
                V0[r] = fma(S, p[0][r], -Q[r]) * rdet;
#pragma unroll
                for (int i = 0; i < 3; i++) V[i][r] = i < DIM ? Sr * B[r][i] : 0.0;
            }
        }
    }

};

// The rule's points and weights in shared memory, filled by the CTA:
// table[q] = (xhat_0, xhat_1, xhat_2, w_q).
template <int DIM>
__device__ __forceinline__ int fill_rule_table(const Rule1D& r, double (*table)[4])
{
    const int nq = DIM == 3 ? r.n * r.n * r.n : r.n * r.n;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double xh[3];
        const double w = quad_point<DIM>(r, q, xh);
        table[q][0] = xh[0];
        table[q][1] = xh[1];
        table[q][2] = xh[2];
        table[q][3] = w;
    }
    __syncthreads();
    return nq;
}

constexpr int QMAX = EF_QUAD_MAX_N * EF_QUAD_MAX_N * EF_QUAD_MAX_N;

template <int DIM>
__global__ void __launch_bounds__(ITPB) k_quad_points(const int32_t* __restrict__ elems,
                                                      const double* __restrict__ nodes, int64_t T, Rule1D r,
                                                      double* __restrict__ x)
{
    __shared__ double table[QMAX][4];
    const int nq = fill_rule_table<DIM>(r, table);
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (e >= T) return;
    double p[4][3], B[3][3];
    load_vertices<DIM>(elems, nodes, e, p);
    edge_frame<DIM>(p, B);
    for (int q = 0; q < nq; q++) {
#pragma unroll
        for (int c = 0; c < DIM; c++) {
            double v = p[0][c];
#pragma unroll
            for (int i = 0; i < DIM; i++) v = fma(B[c][i], table[q][i], v);
            x[((int64_t)q * T + e) * DIM + c] = v;
        }
    }
}

template <int VAR>
__global__ void __launch_bounds__(ITPB) k_fe_values(const int32_t* __restrict__ elems,
                                                    const double* __restrict__ nodes,
                                                    const int32_t* __restrict__ e2d,
                                                    const uint8_t* __restrict__ signbits,
                                                    const double* __restrict__ v, int64_t T, Rule1D r,
                                                    double* __restrict__ out, int* status)
{
    constexpr int DIM = ElemTraits<VAR>::DIM;
    __shared__ double table[QMAX][4];
    const int nq = fill_rule_table<DIM>(r, table);
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (e >= T) return;
    double p[4][3], B[3][3];
    FeAffine<VAR> fe;
    load_vertices<DIM>(elems, nodes, e, p);
    const double det = edge_frame<DIM>(p, B);
    if (not_positive(abs_bits(det))) atomicOr(status, ST_DEGENERATE);
    fe.setup(p, B, det, e2d, __ldg(signbits + e), v, e);
    // runs of n points along the innermost collapsed coordinate, as in k_norm_l2
    const int n = r.n;
    for (int q0 = 0; q0 < nq; q0 += n) {
        double A[3];
#pragma unroll
        for (int c = 0; c < DIM; c++) {
            double a = fe.V0[c];
#pragma unroll
            for (int i = 0; i < DIM - 1; i++) a = fma(fe.V[i][c], table[q0][i], a);
            A[c] = a;
        }
        for (int q = q0; q < q0 + n; q++) {
            const double xl = table[q][DIM - 1];
#pragma unroll
            for (int c = 0; c < DIM; c++) out[((int64_t)q * T + e) * DIM + c] = fma(fe.V[DIM - 1][c], xl, A[c]);
        }
    }
}

// Per element: |det B| sum_q w_q |f_q - v_h(x_q)|^2 (v_h omitted when v is
// NULL); f: [q][element][ncomp]. CTA sums in a fixed tree.
template <int VAR>
__global__ void __launch_bounds__(ITPB) k_norm_l2(const int32_t* __restrict__ elems,
                                                  const double* __restrict__ nodes,
                                                  const int32_t* __restrict__ e2d,
                                                  const uint8_t* __restrict__ signbits,
                                                  const double* __restrict__ v, const double* __restrict__ f,
                                                  int ncomp, int64_t T, Rule1D r, double* __restrict__ elem_out,
                                                  double* __restrict__ part, int* status)
{
    constexpr int DIM = ElemTraits<VAR>::DIM;
    __shared__ double table[QMAX][4];
    __shared__ double red[ITPB];
    const int nq = fill_rule_table<DIM>(r, table);
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    double acc = 0.0;
    if (e < T) {
        double p[4][3], B[3][3];
        load_vertices<DIM>(elems, nodes, e, p);
        const double det = edge_frame<DIM>(p, B);
        if (not_positive(abs_bits(det))) atomicOr(status, ST_DEGENERATE);
        double s = 0.0;
        if (v) {
            const FpK fk;   // the subtractions as full-rate DFMAs (same bits)
            FeAffine<VAR> fe;
            fe.setup(p, B, det, e2d, __ldg(signbits + e), v, e);
            // The points come in runs of n along the innermost collapsed
            // coordinate (point q = (i n + j) n + k in 3D, i n + j in 2D):
            // within a run only xhat_{dim-1} changes, so v_h = A + xhat_{dim-1}
            // V_{dim-1} with A = V0 + sum_{i < dim-1} xhat_i V_i formed once
            // per run (DIM FMAs per point instead of DIM^2).
            const int n = r.n;
            for (int q0 = 0; q0 < nq; q0 += n) {
                double A[3];
#pragma unroll
                for (int c = 0; c < DIM; c++) {
                    double a = fe.V0[c];
#pragma unroll
                    for (int i = 0; i < DIM - 1; i++) a = fma(fe.V[i][c], table[q0][i], a);
                    A[c] = a;
                }
                for (int q = q0; q < q0 + n; q++) {
                    const double xl = table[q][DIM - 1];
                    const double* fq = f + ((int64_t)q * T + e) * DIM;
                    double d2 = 0.0;
#pragma unroll
                    for (int c = 0; c < DIM; c++) {
                        const double d = fk.sub(__ldg(fq + c), fma(fe.V[DIM - 1][c], xl, A[c]));
                        d2 = fma(d, d, d2);
                    }
                    s = fma(table[q][3], d2, s);
                }
            }
        } else {
            for (int q = 0; q < nq; q++) {
                const double* fq = f + ((int64_t)q * T + e) * ncomp;
                double d2 = 0.0;
                for (int c = 0; c < ncomp; c++) {
                    const double d = __ldg(fq + c);
                    d2 = fma(d, d, d2);
                }
                s = fma(table[q][3], d2, s);
            }
        }
        acc = abs_bits(det) * s;
        if (elem_out) elem_out[e] = acc;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = ITPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// grad lambda_0 .. lambda_DIM: rows of B^-1 (cofactor columns / det).
template <int DIM>
__device__ __forceinline__ void barycentric_gradients(const double (&B)[3][3], double rdet, double (&G)[4][3])
{
    if (DIM == 3) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int a = (i + 1) % 3, b = (i + 2) % 3;
            G[i + 1][0] = fma(B[1][a], B[2][b], -(B[2][a] * B[1][b])) * rdet;
            G[i + 1][1] = fma(B[2][a], B[0][b], -(B[0][a] * B[2][b])) * rdet;
            G[i + 1][2] = fma(B[0][a], B[1][b], -(B[1][a] * B[0][b])) * rdet;
        }
    } else {
        G[1][0] = B[1][1] * rdet;
        G[1][1] = -B[0][1] * rdet;
        G[2][0] = -B[1][0] * rdet;
        G[2][1] = B[0][0] * rdet;
        G[1][2] = G[2][2] = G[3][0] = G[3][1] = G[3][2] = 0.0;
    }
#pragma unroll
    for (int r = 0; r < 3; r++) G[0][r] = -(G[1][r] + G[2][r] + G[3][r]);
}

// The rule with each weight times the barycentric coordinates of its point:
// table[q][a] = w_q lambda_a(xhat_q), a = 0..DIM.
template <int DIM>
__device__ __forceinline__ int fill_lambda_table(const Rule1D& r, double (*table)[4])
{
    const int nq = DIM == 3 ? r.n * r.n * r.n : r.n * r.n;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double xh[3];
        const double w = quad_point<DIM>(r, q, xh);
        table[q][0] = w * (1.0 - xh[0] - xh[1] - xh[2]);
        table[q][1] = w * xh[0];
        table[q][2] = w * xh[1];
        table[q][3] = w * xh[2];
    }
    __syncthreads();
    return nq;
}

// Local load vectors l_k = s_k |det B| sum_q w_q F(x_q) . phi_k(x_q), F:
// [q][element][dim]. Every lowest-order basis function is affine, a
// combination of the barycentric coordinates, so the rule is applied once
// to the moments m_a = sum_q w_q lambda_a(x_q) F(x_q) (a = 0..dim; dim + 1
// FMAs per point and component) and each l_k follows from them:
//   Nedelec, edge t -> h: phi = lambda_t grad lambda_h - lambda_h grad lambda_t,
//     sum_q w_q F . phi = grad lambda_h . m_t - grad lambda_t . m_h;
//   RT0, opposite vertex a: phi = (x - P_a) / det B = sum_b lambda_b (P_b - P_a) / det B,
//     sum_q w_q F . phi = sum_b (P_b - P_a) . m_b / det B.
template <int VAR>
__global__ void __launch_bounds__(ITPB) k_load_local(const int32_t* __restrict__ elems,
                                                     const double* __restrict__ nodes,
                                                     const uint8_t* __restrict__ signbits,
                                                     const double* __restrict__ F, int64_t T, Rule1D r,
                                                     double* __restrict__ local, int* status)
{
    constexpr int DIM = ElemTraits<VAR>::DIM;
    constexpr int NL = ElemTraits<VAR>::NL;
    __shared__ double table[QMAX][4];
    const int nq = fill_lambda_table<DIM>(r, table);
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (e >= T) return;
    double p[4][3], B[3][3];
    load_vertices<DIM>(elems, nodes, e, p);
    const double det = edge_frame<DIM>(p, B);
    if (not_positive(abs_bits(det))) atomicOr(status, ST_DEGENERATE);
    const double rdet = 1.0 / det;
    double m[DIM + 1][DIM];
#pragma unroll
    for (int a = 0; a <= DIM; a++)
#pragma unroll
        for (int c = 0; c < DIM; c++) m[a][c] = 0.0;
    for (int q = 0; q < nq; q++) {
        const double* fq = F + ((int64_t)q * T + e) * DIM;
        double f[DIM];
#pragma unroll
        for (int c = 0; c < DIM; c++) f[c] = __ldg(fq + c);
#pragma unroll
        for (int a = 0; a <= DIM; a++)
#pragma unroll
            for (int c = 0; c < DIM; c++) m[a][c] = fma(table[q][a], f[c], m[a][c]);
    }
    double l[NL];
    if (VAR == NED2 || VAR == NED3) {
        double G[4][3];
        barycentric_gradients<DIM>(B, rdet, G);
#pragma unroll
        for (int k = 0; k < NL; k++) {
            const int t = DIM == 3 ? kEdge3[k][0] : kEdge2[k][0];
            const int h = DIM == 3 ? kEdge3[k][1] : kEdge2[k][1];
            double d = 0.0;
#pragma unroll
            for (int c = 0; c < DIM; c++) d = fma(G[h][c], m[t][c], fma(-G[t][c], m[h][c], d));
            l[k] = d;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NL; k++) {
            const int a = DIM == 3 ? 3 - k : k;
            double d = 0.0;
#pragma unroll
            for (int b = 0; b <= DIM; b++)
                if (b != a)
#pragma unroll
                    for (int c = 0; c < DIM; c++) d = fma(p[b][c] - p[a][c], m[b][c], d);
            l[k] = d * rdet;
        }
    }
    const uint32_t neg = __ldg(signbits + e);
    const double adet = abs_bits(det);
#pragma unroll
    for (int k = 0; k < NL; k++) {
        const double v = adet * l[k];
        local[e * NL + k] = ((neg >> k) & 1u) ? -v : v;
    }
}

// Local derivative load vectors l_k = s_k (|det B| sum_q w_q g(x_q)) . D phi_k
// with D phi_k constant on the element (as in k_fe_curl): RT0 div phi_k =
// dim / det B; 2D Nedelec curl phi_k = 2 / det B; 3D Nedelec curl phi_k =
// 2 w_k / det B. g: [q][element][nc], nc = 3 for 3D Nedelec, else 1.
template <int VAR>
__global__ void __launch_bounds__(ITPB) k_load_deriv_local(const int32_t* __restrict__ elems,
                                                           const double* __restrict__ nodes,
                                                           const uint8_t* __restrict__ signbits,
                                                           const double* __restrict__ gf, int64_t T, Rule1D r,
                                                           double* __restrict__ local, int* status)
{
    constexpr int DIM = ElemTraits<VAR>::DIM;
    constexpr int NL = ElemTraits<VAR>::NL;
    constexpr int NC = VAR == NED3 ? 3 : 1;
    __shared__ double table[QMAX][4];
    const int nq = fill_rule_table<DIM>(r, table);
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (e >= T) return;
    double p[4][3], B[3][3];
    load_vertices<DIM>(elems, nodes, e, p);
    const double det = edge_frame<DIM>(p, B);
    if (not_positive(abs_bits(det))) atomicOr(status, ST_DEGENERATE);
    double gi[3] = {0.0, 0.0, 0.0};   // sum_q w_q g(x_q)
    for (int q = 0; q < nq; q++) {
        const double* gq = gf + ((int64_t)q * T + e) * NC;
#pragma unroll
        for (int c = 0; c < NC; c++) gi[c] = fma(table[q][3], __ldg(gq + c), gi[c]);
    }
    // |det B| / det B = sign(det B): the integral times the derivative's 1 / det B
    const double f = (det < 0.0 ? -1.0 : 1.0) * (VAR == RT3 ? 3.0 : 2.0);
    const uint32_t neg = __ldg(signbits + e);
    double l[6];
    if (VAR == NED3) {
#pragma unroll
        for (int k = 0; k < 6; k++) l[k] = 0.0;
#pragma unroll
        for (int r2 = 0; r2 < 3; r2++) {
            const double w[6] = {B[r2][2] - B[r2][1], B[r2][0] - B[r2][2], B[r2][1] - B[r2][0], B[r2][2], B[r2][0],
                                 B[r2][1]};
#pragma unroll
            for (int k = 0; k < 6; k++) l[k] = fma(gi[r2], w[k], l[k]);
        }
#pragma unroll
        for (int k = 0; k < 6; k++) l[k] *= f;
    } else {
#pragma unroll
        for (int k = 0; k < NL; k++) l[k] = f * gi[0];
    }
#pragma unroll
    for (int k = 0; k < NL; k++) local[e * NL + k] = ((neg >> k) & 1u) ? -l[k] : l[k];
}

// b[dof] = sum of its local entries in ascending element order (the DOF's
// incidence segment: element * nl + k, sorted by DOF, stable in element).
__global__ void __launch_bounds__(ITPB) k_load_sum(const uint32_t* __restrict__ off, const uint32_t* __restrict__ inc,
                                                   const double* __restrict__ local, int64_t N,
                                                   double* __restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (i >= N) return;
    const uint32_t s0 = off[i], s1 = off[i + 1];
    double v = s1 > s0 ? local[inc[s0]] : 0.0;
    for (uint32_t s = s0 + 1; s < s1; s++) v += local[inc[s]];
    b[i] = v;
}

__global__ void k_dof_keys(const int32_t* __restrict__ e2d, int64_t n, uint64_t* keys, uint32_t* vals,
                           uint32_t* cnt)
{
    const int64_t i = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (i >= n) return;
    const int32_t d = e2d[i];
    keys[i] = (uint64_t)d;
    vals[i] = (uint32_t)i;   // element * nl + k
    atomicAdd(&cnt[d], 1u);
}

// The constant curl of the Nedelec function of v on an element, with
// c_k = s_k v[dof_k] (Ned0piola3, curl phi_k = B curl eta_k / det B):
//   2D: 2 / det B * sum_k c_k (every reference curl is 2);
//   3D: 2 / det B * sum_k c_k w_k, w = (e3 - e2, e1 - e3, e2 - e1, e3, e1, e2)
//   (B curl eta_k = 2 w_k, e_i the columns of B);
// or the constant divergence of the RT0 function, dim / det B * sum_k c_k.
// out[0] (2D, RT0) or out[0..2] (3D Nedelec).
template <int VAR>
__device__ __forceinline__ void fe_derivative(const double (&B)[3][3], double rdet, const int32_t* __restrict__ e2d,
                                              uint32_t neg, const double* __restrict__ v, int64_t e,
                                              double (&out)[3])
{
    constexpr int NL = ElemTraits<VAR>::NL;
    double c[6];
#pragma unroll
    for (int k = 0; k < NL; k++) {
        const double x = __ldg(v + __ldg(e2d + e * NL + k));
        c[k] = ((neg >> k) & 1u) ? -x : x;
    }
    if (VAR == NED3) {
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const double w[6] = {B[r][2] - B[r][1], B[r][0] - B[r][2], B[r][1] - B[r][0], B[r][2], B[r][0], B[r][1]};
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 6; k++) s = fma(c[k], w[k], s);
            out[r] = 2.0 * s * rdet;
        }
    } else {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < NL; k++) sum += c[k];
        out[0] = (VAR == RT3 ? 3.0 : 2.0) * sum * rdet;
        out[1] = out[2] = 0.0;
    }
}

// Per element, the constant curl or divergence of the FE function of v.
template <int VAR>
__global__ void __launch_bounds__(ITPB) k_fe_curl(const int32_t* __restrict__ elems,
                                                  const double* __restrict__ nodes,
                                                  const int32_t* __restrict__ e2d,
                                                  const uint8_t* __restrict__ signbits,
                                                  const double* __restrict__ v, int64_t T,
                                                  double* __restrict__ out, int* status)
{
    constexpr int DIM = ElemTraits<VAR>::DIM;
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    if (e >= T) return;
    double p[4][3], B[3][3];
    load_vertices<DIM>(elems, nodes, e, p);
    const double det = edge_frame<DIM>(p, B);
    if (not_positive(abs_bits(det))) atomicOr(status, ST_DEGENERATE);
    double d[3];
    fe_derivative<VAR>(B, 1.0 / det, e2d, __ldg(signbits + e), v, e, d);
    if (VAR == NED3) {
#pragma unroll
        for (int r = 0; r < 3; r++) out[e * 3 + r] = d[r];
    } else {
        out[e] = d[0];
    }
}

// Per element: |det B| sum_q w_q |g_q - D v_h|^2, D v_h the constant curl or
// divergence of the FE function of v (omitted when v is NULL); g:
// [q][element][nc], nc = 3 for 3D Nedelec, else 1. CTA sums in a fixed tree.
template <int VAR>
__global__ void __launch_bounds__(ITPB) k_norm_l2_deriv(const int32_t* __restrict__ elems,
                                                        const double* __restrict__ nodes,
                                                        const int32_t* __restrict__ e2d,
                                                        const uint8_t* __restrict__ signbits,
                                                        const double* __restrict__ v, const double* __restrict__ g,
                                                        int64_t T, Rule1D r, double* __restrict__ elem_out,
                                                        double* __restrict__ part, int* status)
{
    constexpr int DIM = ElemTraits<VAR>::DIM;
    constexpr int NC = VAR == NED3 ? 3 : 1;
    __shared__ double table[QMAX][4];
    __shared__ double red[ITPB];
    const int nq = fill_rule_table<DIM>(r, table);
    const int64_t e = (int64_t)blockIdx.x * ITPB + threadIdx.x;
    double acc = 0.0;
    if (e < T) {
        double p[4][3], B[3][3];
        load_vertices<DIM>(elems, nodes, e, p);
        const double det = edge_frame<DIM>(p, B);
        if (not_positive(abs_bits(det))) atomicOr(status, ST_DEGENERATE);
        double d[3] = {0.0, 0.0, 0.0};
        if (v) fe_derivative<VAR>(B, 1.0 / det, e2d, __ldg(signbits + e), v, e, d);
        double s = 0.0;
        const FpK fk;   // the subtractions as full-rate DFMAs (same bits)
        for (int q = 0; q < nq; q++) {
            const double* gq = g + ((int64_t)q * T + e) * NC;
            double d2 = 0.0;
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const double x = fk.sub(__ldg(gq + c), d[c]);
                d2 = fma(x, x, d2);
            }
            s = fma(table[q][3], d2, s);
        }
        acc = abs_bits(det) * s;
        if (elem_out) elem_out[e] = acc;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = ITPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// The partial sums in one fixed order: thread t adds t, t + 1024, ..., then a tree.
__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ part, int64_t n, double* out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

int make_rule(int dim, int n, Rule1D* r, int* nq)
{
    if (n < 1 || n > EF_QUAD_MAX_N || (dim != 2 && dim != 3)) return EF_ERR_ARG;
    legendre_rule(n, r);
    *nq = dim == 3 ? n * n * n : n * n;
    return EF_OK;
}

}  // namespace
}  // namespace ef

using namespace ef;

namespace {

// DOF -> (element, local DOF) incidence, ascending element order inside a
// DOF, and the per-(element, local DOF) scratch of the load vectors; built on
// first use (allocates, synchronises `s`).
int ensure_load_incidence(ef_plan* plan, cudaStream_t s)
{
    if (plan->d_dof_inc) return EF_OK;
    const int64_t nl = plan->nl, n_inc = plan->T * nl;
    uint64_t* keys = nullptr;
    uint32_t* cnt = nullptr;
    void* tmp = nullptr;
    size_t tb = radix_tmp_bytes(n_inc);
    if (scan_tmp_bytes(plan->N) > tb) tb = scan_tmp_bytes(plan->N);
    int st = EF_OK;
    if (cudaMalloc((void**)&plan->d_dof_inc, n_inc * 4) != cudaSuccess ||
        cudaMalloc((void**)&plan->d_dof_off, (plan->N + 1) * 4) != cudaSuccess ||
        cudaMalloc((void**)&plan->d_load_local, n_inc * 8) != cudaSuccess ||
        cudaMalloc((void**)&keys, n_inc * 8) != cudaSuccess || cudaMalloc((void**)&cnt, plan->N * 4) != cudaSuccess ||
        cudaMalloc(&tmp, tb) != cudaSuccess) {
        set_last_error("cudaMalloc(load vector)", cudaErrorMemoryAllocation);
        st = EF_ERR_OOM;
    }
    if (st == EF_OK) {
        cudaMemsetAsync(cnt, 0, plan->N * 4, s);
        k_dof_keys<<<(unsigned)((n_inc + ITPB - 1) / ITPB), ITPB, 0, s>>>(plan->d_elem2dof, n_inc, keys,
                                                                          plan->d_dof_inc, cnt);
        st = radix_sort_pairs(keys, plan->d_dof_inc, n_inc, bits_for((uint64_t)plan->N), tmp, s);
        if (st == EF_OK) st = exclusive_scan_u32(cnt, plan->d_dof_off, plan->N, true, tmp, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (st == EF_OK && e != cudaSuccess) {
            set_last_error("load vector incidence", e);
            st = EF_ERR_CUDA;
        }
    }
    cudaFree(keys);
    cudaFree(cnt);
    cudaFree(tmp);
    if (st != EF_OK) {
        cudaFree(plan->d_dof_inc);
        cudaFree(plan->d_dof_off);
        cudaFree(plan->d_load_local);
        plan->d_dof_inc = plan->d_dof_off = nullptr;
        plan->d_load_local = nullptr;
    }
    return st;
}

// Shared argument checks of the load vectors; *done if there is nothing to
// integrate (b zeroed).
int load_checks(ef_plan* plan, const double* d_nodes, int n, const double* d_in, double* d_b, Rule1D* r,
                cudaStream_t s, bool* done)
{
    *done = false;
    if (!plan) return EF_ERR_ARG;
    int nq = 0;
    EF_TRY(make_rule(plan->dim, n, r, &nq));
    if (plan->N > 0 && !d_b) return EF_ERR_ARG;
    if (plan->T == 0) {
        if (plan->N > 0) EF_CUDA(cudaMemsetAsync(d_b, 0, (size_t)plan->N * sizeof(double), s));
        *done = true;
        return EF_OK;
    }
    if (!d_nodes || !d_in) return EF_ERR_ARG;
    return ensure_load_incidence(plan, s);
}

}  // namespace

extern "C" {

int ef_quad_rule(int dim, int n, double* h_xhat, double* h_w, int cap, int* nq)
{
    Rule1D r;
    int m = 0;
    EF_TRY(make_rule(dim, n, &r, &m));
    if (nq) *nq = m;
    if (!h_xhat && !h_w) return EF_OK;
    if (cap < m) return EF_ERR_SIZE;
    for (int q = 0; q < m; q++) {
        double xh[3], w;
        if (dim == 3) {
            const int i = q / (n * n), j = (q / n) % n, k = q % n;
            const double u = r.t[i], v = r.t[j], s = r.t[k];
            xh[0] = u;
            xh[1] = v * (1.0 - u);
            xh[2] = s * (1.0 - u) * (1.0 - v);
            w = r.w[i] * r.w[j] * r.w[k] * (1.0 - u) * (1.0 - u) * (1.0 - v);
        } else {
            const int i = q / n, j = q % n;
            const double u = r.t[i], v = r.t[j];
            xh[0] = u;
            xh[1] = v * (1.0 - u);
            w = r.w[i] * r.w[j] * (1.0 - u);
        }
        if (h_xhat)
            for (int c = 0; c < dim; c++) h_xhat[q * dim + c] = xh[c];
        if (h_w) h_w[q] = w;
    }
    return EF_OK;
}

int ef_quad_points(const ef_plan* plan, const double* d_nodes, int n, double* d_x, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    Rule1D r;
    int nq = 0;
    EF_TRY(make_rule(plan->dim, n, &r, &nq));
    if (plan->T == 0) return EF_OK;
    if (!d_nodes || !d_x) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = (unsigned)((plan->T + ITPB - 1) / ITPB);
    if (plan->dim == 3) k_quad_points<3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, plan->T, r, d_x);
    else k_quad_points<2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, plan->T, r, d_x);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int ef_fe_values(const ef_plan* plan, const double* d_nodes, const double* d_v, int n, double* d_vals, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    Rule1D r;
    int nq = 0;
    EF_TRY(make_rule(plan->dim, n, &r, &nq));
    if (plan->T == 0) return EF_OK;
    if (!d_nodes || !d_v || !d_vals) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = (unsigned)((plan->T + ITPB - 1) / ITPB);
    const int32_t* e2d = plan->d_elem2dof;
    const uint8_t* sb = plan->d_signbits;
    switch (plan->variant) {
        case RT2: k_fe_values<RT2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, r, d_vals, plan->d_status); break;
        case NED2: k_fe_values<NED2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, r, d_vals, plan->d_status); break;
        case RT3: k_fe_values<RT3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, r, d_vals, plan->d_status); break;
        default: k_fe_values<NED3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, r, d_vals, plan->d_status); break;
    }
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int ef_fe_curl(const ef_plan* plan, const double* d_nodes, const double* d_v, double* d_out, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    if (plan->T == 0) return EF_OK;
    if (!d_nodes || !d_v || !d_out) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = (unsigned)((plan->T + ITPB - 1) / ITPB);
    const int32_t* e2d = plan->d_elem2dof;
    const uint8_t* sb = plan->d_signbits;
    switch (plan->variant) {
        case RT2: k_fe_curl<RT2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, d_out, plan->d_status); break;
        case NED2: k_fe_curl<NED2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, d_out, plan->d_status); break;
        case RT3: k_fe_curl<RT3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, d_out, plan->d_status); break;
        default: k_fe_curl<NED3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, plan->T, d_out, plan->d_status); break;
    }
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}


int ef_load_vector(ef_plan* plan, const double* d_nodes, int n, const double* d_F, double* d_b, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    Rule1D r;
    bool done = false;
    EF_TRY(load_checks(plan, d_nodes, n, d_F, d_b, &r, s, &done));
    if (done) return EF_OK;
    const unsigned g = (unsigned)((plan->T + ITPB - 1) / ITPB);
    const uint8_t* sb = plan->d_signbits;
    double* loc = plan->d_load_local;
    switch (plan->variant) {
        case RT2: k_load_local<RT2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_F, plan->T, r, loc, plan->d_status); break;
        case NED2: k_load_local<NED2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_F, plan->T, r, loc, plan->d_status); break;
        case RT3: k_load_local<RT3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_F, plan->T, r, loc, plan->d_status); break;
        default: k_load_local<NED3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_F, plan->T, r, loc, plan->d_status); break;
    }
    k_load_sum<<<(unsigned)((plan->N + ITPB - 1) / ITPB), ITPB, 0, s>>>(plan->d_dof_off, plan->d_dof_inc, loc, plan->N,
                                                                         d_b);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int ef_load_derivative(ef_plan* plan, const double* d_nodes, int n, const double* d_g, double* d_b, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    Rule1D r;
    bool done = false;
    EF_TRY(load_checks(plan, d_nodes, n, d_g, d_b, &r, s, &done));
    if (done) return EF_OK;
    const unsigned g = (unsigned)((plan->T + ITPB - 1) / ITPB);
    const uint8_t* sb = plan->d_signbits;
    double* loc = plan->d_load_local;
    switch (plan->variant) {
        case RT2: k_load_deriv_local<RT2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_g, plan->T, r, loc, plan->d_status); break;
        case NED2: k_load_deriv_local<NED2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_g, plan->T, r, loc, plan->d_status); break;
        case RT3: k_load_deriv_local<RT3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_g, plan->T, r, loc, plan->d_status); break;
        default: k_load_deriv_local<NED3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, sb, d_g, plan->T, r, loc, plan->d_status); break;
    }
    k_load_sum<<<(unsigned)((plan->N + ITPB - 1) / ITPB), ITPB, 0, s>>>(plan->d_dof_off, plan->d_dof_inc, loc, plan->N,
                                                                         d_b);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int ef_norm_l2(ef_plan* plan, const double* d_nodes, int n, int ncomp, const double* d_f, const double* d_v,
               double* d_elem, double* d_total, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    Rule1D r;
    int nq = 0;
    EF_TRY(make_rule(plan->dim, n, &r, &nq));
    if (ncomp < 1 || ncomp > 3 || (d_v && ncomp != plan->dim)) return EF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->T == 0) {
        if (d_total) EF_CUDA(cudaMemsetAsync(d_total, 0, sizeof(double), s));
        return EF_OK;
    }
    if (!d_nodes || !d_f) return EF_ERR_ARG;
    const int64_t nb = (plan->T + ITPB - 1) / ITPB;
    if (!plan->d_l2_part) {
        cudaError_t e = cudaMalloc((void**)&plan->d_l2_part, (size_t)nb * sizeof(double));
        if (e != cudaSuccess) {
            set_last_error("cudaMalloc(l2 partials)", e);
            return EF_ERR_OOM;
        }
    }
    const unsigned g = (unsigned)nb;
    const int32_t* e2d = plan->d_elem2dof;
    const uint8_t* sb = plan->d_signbits;
    double* part = plan->d_l2_part;
    switch (plan->variant) {
        case RT2: k_norm_l2<RT2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_f, ncomp, plan->T, r, d_elem, part, plan->d_status); break;
        case NED2: k_norm_l2<NED2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_f, ncomp, plan->T, r, d_elem, part, plan->d_status); break;
        case RT3: k_norm_l2<RT3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_f, ncomp, plan->T, r, d_elem, part, plan->d_status); break;
        default: k_norm_l2<NED3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_f, ncomp, plan->T, r, d_elem, part, plan->d_status); break;
    }
    if (d_total) k_sum_partials<<<1, 1024, 0, s>>>(part, nb, d_total);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

int ef_norm_l2_derivative(ef_plan* plan, const double* d_nodes, int n, const double* d_g, const double* d_v,
                          double* d_elem, double* d_total, void* stream)
{
    if (!plan) return EF_ERR_ARG;
    Rule1D r;
    int nq = 0;
    EF_TRY(make_rule(plan->dim, n, &r, &nq));
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->T == 0) {
        if (d_total) EF_CUDA(cudaMemsetAsync(d_total, 0, sizeof(double), s));
        return EF_OK;
    }
    if (!d_nodes || !d_g) return EF_ERR_ARG;
    const int64_t nb = (plan->T + ITPB - 1) / ITPB;
    if (!plan->d_l2_part) {
        cudaError_t e = cudaMalloc((void**)&plan->d_l2_part, (size_t)nb * sizeof(double));
        if (e != cudaSuccess) {
            set_last_error("cudaMalloc(l2 partials)", e);
            return EF_ERR_OOM;
        }
    }
    const unsigned g = (unsigned)nb;
    const int32_t* e2d = plan->d_elem2dof;
    const uint8_t* sb = plan->d_signbits;
    double* part = plan->d_l2_part;
    switch (plan->variant) {
        case RT2: k_norm_l2_deriv<RT2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_g, plan->T, r, d_elem, part, plan->d_status); break;
        case NED2: k_norm_l2_deriv<NED2><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_g, plan->T, r, d_elem, part, plan->d_status); break;
        case RT3: k_norm_l2_deriv<RT3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_g, plan->T, r, d_elem, part, plan->d_status); break;
        default: k_norm_l2_deriv<NED3><<<g, ITPB, 0, s>>>(plan->d_elems, d_nodes, e2d, sb, d_v, d_g, plan->T, r, d_elem, part, plan->d_status); break;
    }
    if (d_total) k_sum_partials<<<1, 1024, 0, s>>>(part, nb, d_total);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

}  // extern "C"
