// Adjoint of J(x, sigma) = u^T K u + v^T M v for 3D Nedelec elements.
//
// Per element (Sec. 2.4 matrices, closed forms of ef_element.cuh), with
// u~_k = s_k u[dof_k], v~_k = s_k v[dof_k], e_i the columns of B,
// H = B^T B, A = adj(H), r = 1/|det B| = det(H)^(-1/2) (det B taken by the
// triple product):
//   K part: sum_k u~_k (B curl eta_k)/2 = B a, a = (u1-u2+u4, -u0+u2+u5, u0-u1+u3),
//           J_K = sigma (2/3) r a^T H a;
//   M part: with the Whitney forms, psi = sum_k v~_k (l_t grad l_h - l_h grad l_t)
//           = sum_ij C_ij l_i grad l_j (C antisymmetric, C_th = v~_k), and
//           int_K l_i l_k = |K| (1 + d_ik)/20, so
//           int_K |psi|^2 = r/120 <P, A>,  P = S^T (c c^T + C^T C) S,
//           c = column sums of C, S = [-1 -1 -1; I] (grad l_0 = -sum grad l_i);
//           J_M = sigma r/120 <P, A>.
// Derivatives through H: d r = -r^3/2 <A, dH>, d<P, A> = r^2 <P,A> <A, dH>
// - r^2 <A P A, dH>, so with Gamma = dJ/dH / sigma
//   Gamma = (2/3)(r a a^T - r^3/2 (a^T H a) A) + r^3/120 (<P,A>/2 A - A P A),
// dJ/dB = 2 sigma B Gamma; node i >= 1 gets column i-1, node 0 minus their sum.
// dJ/dsigma_K = J_K / sigma. Geometry is recomputed here, not stored by the
// forward pass. The per-(element, vertex) gradients go to plan scratch and are
// summed per node in ascending element order; J is summed per CTA in a fixed
// tree and the CTA sums in a fixed strided order and tree. No floating-point
// atomics.
#include "ef_assemble.cuh"
#include "ef_internal.cuh"

namespace ef {
namespace {

// 128 threads per CTA, 4 CTAs of 128 registers per SM (1.889 ms at 96^3,
// against 1.907 ms with 2 CTAs of 256; at 96 registers the kernel spills)
constexpr int ADJ_TPB = 128;

// One element: J1 = u~^T K^ u~ + v~^T M^ v~ with the coefficient left out (the
// element's energy is sigma J1) and 2 sigma (B Gamma) column by column into
// gcol (node i+1 gets column i). MUL forms every product (IntMul on the
// integer pipes, or FpMul): no product is contracted into an FMA, so both give
// the same bits.
template <class MUL>
__device__ __forceinline__ void adjoint_element(MUL& mul, const FpK& f, const double (&p)[4][3], double sigma,
                                                const double (&ut)[6], const double (&vt)[6], bool& degenerate,
                                                double& J1, double (&gcol)[3][3])
{
    double B[3][3];   // B[row][col], col i = e_{i+1}
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) B[c][i] = f.sub(p[i + 1][c], p[0][c]);
    double H[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            H[i][j] = fma(B[2][i], B[2][j], fma(B[1][i], B[1][j], mul(B[0][i], B[0][j])));
            H[j][i] = H[i][j];
        }
    double A[3][3];
    A[0][0] = fma(H[1][1], H[2][2], -mul(H[1][2], H[1][2]));
    A[1][1] = fma(H[0][0], H[2][2], -mul(H[0][2], H[0][2]));
    A[2][2] = fma(H[0][0], H[1][1], -mul(H[0][1], H[0][1]));
    A[0][1] = A[1][0] = fma(H[0][2], H[1][2], -mul(H[0][1], H[2][2]));
    A[0][2] = A[2][0] = fma(H[0][1], H[1][2], -mul(H[0][2], H[1][1]));
    A[1][2] = A[2][1] = fma(H[0][1], H[0][2], -mul(H[0][0], H[1][2]));
    // det B by the triple product (error ~ cond(B) eps)
    const double cx = fma(B[1][1], B[2][2], -mul(B[2][1], B[1][2]));
    const double cy = fma(B[2][1], B[0][2], -mul(B[0][1], B[2][2]));
    const double cz = fma(B[0][1], B[1][2], -mul(B[1][1], B[0][2]));
    const double adet = abs_bits(fma(B[2][0], cz, fma(B[1][0], cy, mul(B[0][0], cx))));
    degenerate = not_positive(adet);
    const double r = recip_positive(adet, f.one);
    const double r3 = mul(mul(r, r), r);

    // K part: aHa = a^T H a over the symmetric H
    const double av[3] = {f.add(f.sub(ut[1], ut[2]), ut[4]), f.add(f.sub(ut[2], ut[0]), ut[5]),
                          f.add(f.sub(ut[0], ut[1]), ut[3])};
    const double aHa = fma(av[0], fma(H[0][0], av[0], twice(fma(H[0][1], av[1], mul(H[0][2], av[2])))),
                           fma(av[1], fma(H[1][1], av[1], twice(mul(H[1][2], av[2]))), mul(av[2], mul(H[2][2], av[2]))));

    // M part: C antisymmetric over the 4 nodes, edges (0,1),(0,2),(0,3),(1,2),(2,3),(3,1)
    const double c0 = -f.add(f.add(vt[0], vt[1]), vt[2]);
    const double c1 = f.add(f.sub(vt[0], vt[3]), vt[5]);
    const double c2 = f.sub(f.add(vt[1], vt[3]), vt[4]);
    const double c3 = f.sub(f.add(vt[2], vt[4]), vt[5]);
    const double beta[3] = {f.sub(c1, c0), f.sub(c2, c0), f.sub(c3, c0)};
    // D = C S: row k, column j (node j+1): C_k,j+1 - C_k,0
    const double D[4][3] = {{vt[0], vt[1], vt[2]},
                            {vt[0], f.add(vt[3], vt[0]), f.sub(vt[0], vt[5])},
                            {f.sub(vt[1], vt[3]), vt[1], f.add(vt[4], vt[1])},
                            {f.add(vt[5], vt[2]), f.sub(vt[2], vt[4]), vt[2]}};
    double P[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            double s = mul(beta[i], beta[j]);
#pragma unroll
            for (int k = 0; k < 4; k++) s = fma(D[k][i], D[k][j], s);
            P[i][j] = s;
            P[j][i] = s;
        }
    // <P, A> over the symmetric pair
    const double PA = fma(P[0][0], A[0][0], fma(P[1][1], A[1][1], fma(P[2][2], A[2][2],
                          twice(fma(P[0][1], A[0][1], fma(P[0][2], A[0][2], mul(P[1][2], A[1][2])))))));

    // J1 = (2/3) r aHa + (r/120) PA
    J1 = fma(mul(r, 2.0 / 3.0), aHa, mul(mul(r, 1.0 / 120.0), PA));

    // 2 sigma Gamma, Gamma = (2/3)(r a a^T - r^3/2 aHa A) + r^3/120 (PA/2 A - A P A),
    // symmetric: six entries; A P A from the full A P and the upper half of (A P) A
    double AP[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) AP[i][j] = fma(A[i][2], P[2][j], fma(A[i][1], P[1][j], mul(A[i][0], P[0][j])));
    const double s2 = twice(sigma);
    const double kA = mul(s2, fma(mul(r3, -1.0 / 3.0), aHa, mul(mul(r3, 1.0 / 240.0), PA)));
    const double kAPA = mul(s2, mul(r3, -1.0 / 120.0));
    const double kaa = mul(s2, mul(r, 2.0 / 3.0));
    const double ka[3] = {mul(kaa, av[0]), mul(kaa, av[1]), mul(kaa, av[2])};
    double Gm[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) {
            const double apa = fma(AP[i][2], A[2][j], fma(AP[i][1], A[1][j], mul(AP[i][0], A[0][j])));
            Gm[i][j] = fma(kAPA, apa, fma(kA, A[i][j], mul(ka[i], av[j])));
            Gm[j][i] = Gm[i][j];
        }
    // dJ/de_i = 2 sigma (B Gamma)[:, i]
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) gcol[i][c] = fma(B[c][2], Gm[2][i], fma(B[c][1], Gm[1][i], mul(B[c][0], Gm[0][i])));
}

__device__ __forceinline__ void adjoint_load(const int32_t* __restrict__ elems, const double* __restrict__ nodes,
                                             const double* __restrict__ coeff, const int32_t* __restrict__ e2d,
                                             const double* __restrict__ u, const double* __restrict__ v, int64_t e,
                                             double (&p)[4][3], double& sigma, double (&ut)[6], double (&vt)[6])
{
    int32_t g[4];
    load_ids<NED3>(elems, e, g);
    const uint32_t neg = sign_bits<NED3>(g);
    load_coords<NED3>(nodes, g, p);
    sigma = coeff ? __ldg(coeff + e) : 1.0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int32_t d = __ldg(e2d + e * 6 + k);
        ut[k] = flip_if(__ldg(u + d), neg >> k);
        vt[k] = flip_if(__ldg(v + d), neg >> k);
    }
}

// The products on the integer pipes (IntMul); an element in which an operand
// or a product leaves the normal numbers and zero is repeated with the FP64
// multiply from its data loaded again, which gives the same bits.
__global__ void __launch_bounds__(ADJ_TPB, 4) k_adjoint_ned3(const int32_t* __restrict__ elems,
                                                          const double* __restrict__ nodes,
                                                          const double* __restrict__ coeff,
                                                          const int32_t* __restrict__ e2d,
                                                          const double* __restrict__ u, const double* __restrict__ v,
                                                          int64_t T, double* __restrict__ gpart,
                                                          double* __restrict__ gcoeff, double* __restrict__ jpart,
                                                          int* status)
{
    __shared__ double red[ADJ_TPB];
    const int64_t e = (int64_t)blockIdx.x * ADJ_TPB + threadIdx.x;
    double Jloc = 0.0;
    if (e < T) {
        const FpK f;
        double J1, gcol[3][3], sigma;
        bool degenerate;
        {
            double p[4][3], ut[6], vt[6];
            adjoint_load(elems, nodes, coeff, e2d, u, v, e, p, sigma, ut, vt);
            IntMul im;
            adjoint_element(im, f, p, sigma, ut, vt, degenerate, J1, gcol);
            if (im.off) {
                // the index through an opaque move: the loads are not merged with the ones above
                int64_t e2 = e;
                asm volatile("" : "+l"(e2));
                adjoint_load(elems, nodes, coeff, e2d, u, v, e2, p, sigma, ut, vt);
                FpMul fm;
                adjoint_element(fm, f, p, sigma, ut, vt, degenerate, J1, gcol);
            }
        }
        if (degenerate) atomicOr(status, ST_DEGENERATE);
        if (gcoeff) gcoeff[e] = J1;
        Jloc = __dmul_rn(sigma, J1);
        // node 0 gets minus the sum of the other three
        double g0[3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                gpart[(e * 4 + i + 1) * 3 + c] = gcol[i][c];
                g0[c] = i == 0 ? -gcol[i][c] : f.sub(g0[c], gcol[i][c]);
            }
#pragma unroll
        for (int c = 0; c < 3; c++) gpart[(e * 4) * 3 + c] = g0[c];
    }
    // fixed-order tree sum of the CTA's element energies
    red[threadIdx.x] = Jloc;
    __syncthreads();
    for (int w = ADJ_TPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) jpart[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_node_reduce(const uint32_t* __restrict__ off, const uint32_t* __restrict__ inc,
                                                     const double* __restrict__ gpart, int64_t V,
                                                     double* __restrict__ grad)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= V) return;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (uint32_t s = off[i]; s < off[i + 1]; s++) {
        const int64_t q = inc[s];
        gx += gpart[q * 3 + 0];
        gy += gpart[q * 3 + 1];
        gz += gpart[q * 3 + 2];
    }
    grad[i * 3 + 0] = gx;
    grad[i * 3 + 1] = gy;
    grad[i * 3 + 2] = gz;
}

// Sum of the per-CTA energies in one fixed order: thread t adds parts t,
// t + SUM_TPB, ... in turn, then a fixed shared-memory tree.
constexpr int SUM_TPB = 1024;

__global__ void __launch_bounds__(SUM_TPB) k_sum_parts(const double* __restrict__ part, int64_t n, double* out)
{
    __shared__ double red[SUM_TPB];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += SUM_TPB) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = SUM_TPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_node_keys(const int32_t* elems, int64_t T, uint64_t* keys, uint32_t* vals, uint32_t* cnt)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= T * 4) return;
    const int32_t g = elems[i];
    keys[i] = (uint64_t)g;
    vals[i] = (uint32_t)i;  // element * 4 + local vertex
    atomicAdd(&cnt[g], 1u);
}

}  // namespace

int build_adjoint(ef_plan* p, cudaStream_t s)
{
    if (p->variant != NED3 || p->T == 0) return EF_OK;
    const int64_t n = p->T * 4, V = p->V;
    uint64_t* keys = nullptr;
    uint32_t* cnt = nullptr;
    void* tmp = nullptr;
    int st = EF_OK;
    size_t tb = radix_tmp_bytes(n);
    if (scan_tmp_bytes(V) > tb) tb = scan_tmp_bytes(V);
    if (cudaMalloc((void**)&p->d_node_inc, n * 4) != cudaSuccess || cudaMalloc((void**)&p->d_node_off, (V + 1) * 4) != cudaSuccess ||
        cudaMalloc((void**)&p->d_adj_part, n * 3 * 8) != cudaSuccess ||
        cudaMalloc((void**)&p->d_adj_jpart, ((p->T + ADJ_TPB - 1) / ADJ_TPB) * 8) != cudaSuccess ||
        cudaMalloc((void**)&keys, n * 8) != cudaSuccess || cudaMalloc((void**)&cnt, (V > 0 ? V : 1) * 4) != cudaSuccess ||
        cudaMalloc(&tmp, tb) != cudaSuccess) {
        set_last_error("cudaMalloc(adjoint)", cudaErrorMemoryAllocation);
        st = EF_ERR_OOM;
    }
    if (st == EF_OK) {
        cudaMemsetAsync(cnt, 0, (V > 0 ? V : 1) * 4, s);
        k_node_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->d_elems, p->T, keys, p->d_node_inc, cnt);
        st = radix_sort_pairs(keys, p->d_node_inc, n, bits_for((uint64_t)V), tmp, s);
        if (st == EF_OK) st = exclusive_scan_u32(cnt, p->d_node_off, V, true, tmp, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (st == EF_OK && e != cudaSuccess) {
            set_last_error("build_adjoint", e);
            st = EF_ERR_CUDA;
        }
    }
    if (keys) cudaFree(keys);
    if (cnt) cudaFree(cnt);
    if (tmp) cudaFree(tmp);
    return st;
}

int launch_adjoint(const ef_plan* p, const double* nodes, const double* coeff, const double* u, const double* v,
                   double* J, double* gx, double* gs, cudaStream_t s)
{
    if (p->variant != NED3) return EF_ERR_ARG;
    if (p->T == 0) {
        if (J) EF_CUDA(cudaMemsetAsync(J, 0, 8, s));
        if (gx && p->V > 0) EF_CUDA(cudaMemsetAsync(gx, 0, (size_t)p->V * 24, s));
        return EF_OK;
    }
    const int64_t nb = (p->T + ADJ_TPB - 1) / ADJ_TPB;
    k_adjoint_ned3<<<(unsigned)nb, ADJ_TPB, 0, s>>>(p->d_elems, nodes, coeff, p->d_elem2dof, u, v, p->T, p->d_adj_part,
                                                    gs, p->d_adj_jpart, p->d_status);
    if (gx) k_node_reduce<<<(unsigned)((p->V + 255) / 256), 256, 0, s>>>(p->d_node_off, p->d_node_inc, p->d_adj_part, p->V, gx);
    if (J) k_sum_parts<<<1, SUM_TPB, 0, s>>>(p->d_adj_jpart, nb, J);
    EF_CUDA(cudaGetLastError());
    return EF_OK;
}

}  // namespace ef
