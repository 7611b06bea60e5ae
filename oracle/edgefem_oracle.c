/*
 * edgefem_oracle.c -- CPU FP64 oracle for the assembly of lowest-order
 * Raviart-Thomas (H(div)) and Nedelec first-kind (H(curl)) mass and
 * div/curl stiffness matrices on triangles and tetrahedra
 * (I. Anjam, J. Valdman, "Fast MATLAB assembly of FEM matrices in 2D and 3D:
 * Edge elements", arXiv 1409.4618).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the reference the CUDA path is
 * checked against. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code with the CUDA library.
 *
 * Plain and slow on purpose. What it computes, in the paper's terms:
 *   - reference elements, DOFs and basis functions (Sec. 2.1, 2.2, Fig. 1);
 *   - Piola maps (Eqs. RT0piola, Ned0piola1-3);
 *   - orientation signs (Sec. 2.3, Eq. RT0piola2), decided GEOMETRICALLY here:
 *     a global direction is fixed for every edge / face from its sorted global
 *     node ids, and each element's sign says whether its mapped local DOF
 *     agrees with it;
 *   - global DOF numbering = rows of edges2nodes / faces2nodes (Sec. 3), taken
 *     as the lexicographic order of the sorted node tuples;
 *   - local matrices by explicit quadrature on the reference element
 *     (Sec. 2.4, Eq. RT0local2), multiplied by the element coefficient;
 *   - global matrices K_ij = sum over elements of local entries whose local
 *     DOFs map to (i, j), accumulated element by element in ascending element
 *     order into a CSR pattern holding every DOF pair that shares an element.
 * The adjoint (gradient of sum_K sigma_K (u_K^T Khat_K u_K + v_K^T Mhat_K v_K)
 * with respect to node coordinates and sigma) runs the same local-matrix code
 * on forward-mode dual numbers. The vectorised integration of Sec. 3.1
 * (norm_L2: squared L2 norms by quadrature, loop over points, all elements
 * at once) evaluates the same Piola-mapped, signed basis at quadrature points.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_RT0 1
#define ORA_NED1 2

#define ORA_OK 0
#define ORA_ERR_ARG (-1)
#define ORA_ERR_RANGE (-2)
#define ORA_ERR_DEGENERATE (-3)
#define ORA_ERR_OOM (-5)

/* ------------------------------------------------------------------------ */
/* Reference elements (Sec. 2, Fig. 1)                                       */
/* ------------------------------------------------------------------------ */

/* A reference basis function is affine: eta(x) = a + A x, A[r][c] = d eta_r / d x_c. */
typedef struct {
    double a[3];
    double A[3][3];
} affine_field;

/* Sec. 2.1, 2D RT: eta1 = (x1, x2), eta2 = (x1-1, x2), eta3 = (x1, x2-1) */
static const affine_field RT2[3] = {
    {{0, 0, 0}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 0}}},
    {{-1, 0, 0}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 0}}},
    {{0, -1, 0}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 0}}},
};
/* Sec. 2.1, 3D RT: eta1 = (x1, x2, x3-1), eta2 = (x1, x2-1, x3), eta3 = (x1-1, x2, x3), eta4 = (x1, x2, x3) */
static const affine_field RT3[4] = {
    {{0, 0, -1}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}},
    {{0, -1, 0}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}},
    {{-1, 0, 0}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}},
    {{0, 0, 0}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}},
};
/* Sec. 2.2, 2D Ned: eta1 = (-x2, x1), eta2 = (-x2, x1-1), eta3 = (1-x2, x1) */
static const affine_field NED2[3] = {
    {{0, 0, 0}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 0}}},
    {{0, -1, 0}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 0}}},
    {{1, 0, 0}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 0}}},
};
/* Sec. 2.2, 3D Ned:
 *   eta1 = (1-x3-x2, x1, x1), eta2 = (x2, 1-x3-x1, x2), eta3 = (x3, x3, 1-x2-x1),
 *   eta4 = (-x2, x1, 0),      eta5 = (0, -x3, x2),      eta6 = (x3, 0, -x1)     */
static const affine_field NED3[6] = {
    {{1, 0, 0}, {{0, -1, -1}, {1, 0, 0}, {1, 0, 0}}},
    {{0, 1, 0}, {{0, 1, 0}, {-1, 0, -1}, {0, 1, 0}}},
    {{0, 0, 1}, {{0, 0, 1}, {0, 0, 1}, {-1, -1, 0}}},
    {{0, 0, 0}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 0}}},
    {{0, 0, 0}, {{0, 0, 0}, {0, 0, -1}, {0, 1, 0}}},
    {{0, 0, 0}, {{0, 0, 1}, {0, 0, 0}, {-1, 0, 0}}},
};

/* Local DOF entities (Fig. 1). 2D edge k lies opposite local node k and runs
 * tail -> head as the reference tangent t_k; 3D edges as drawn; 3D face k is
 * listed by its three nodes followed by the opposite node. 0-based. */
static const int EDGE2[3][2] = {{1, 2}, {2, 0}, {0, 1}};
static const int EDGE3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {2, 3}, {3, 1}};
static const int FACE3[4][4] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 3, 1}, {1, 2, 3, 0}};

static int valid_kind(int kind, int dim)
{
    return (kind == ORA_RT0 || kind == ORA_NED1) && (dim == 2 || dim == 3);
}

static int nloc_of(int kind, int dim)
{
    if (dim == 2) return 3;
    return kind == ORA_RT0 ? 4 : 6;
}

/* number of nodes of the mesh entity a DOF sits on: 2 (edge) or 3 (face) */
static int ent_nodes(int kind, int dim)
{
    return (kind == ORA_RT0 && dim == 3) ? 3 : 2;
}

static const affine_field* ref_basis(int kind, int dim)
{
    if (kind == ORA_RT0) return dim == 2 ? RT2 : RT3;
    return dim == 2 ? NED2 : NED3;
}

/* local node indices of the entity of local DOF k (sorted by nothing) */
static void local_entity(int kind, int dim, int k, int* nodes, int* opp)
{
    if (kind == ORA_RT0 && dim == 3) {
        nodes[0] = FACE3[k][0]; nodes[1] = FACE3[k][1]; nodes[2] = FACE3[k][2];
        *opp = FACE3[k][3];
    } else if (dim == 2) {
        nodes[0] = EDGE2[k][0]; nodes[1] = EDGE2[k][1];
        *opp = k;
    } else {
        nodes[0] = EDGE3[k][0]; nodes[1] = EDGE3[k][1];
        *opp = -1;
    }
}

/* ------------------------------------------------------------------------ */
/* Quadrature                                                                */
/* ------------------------------------------------------------------------ */

#define QMAX 4096
typedef struct {
    int n;
    double x[3 * QMAX];
    double w[QMAX];
} qrule;

/* Symmetric degree-2 rules: 3 points on the triangle (barycentric 2/3, 1/6,
 * 1/6), 4 points on the tetrahedron (barycentric a, b, b, b with
 * a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20); equal weights summing to the
 * reference measure. Exact for the degree-2 integrands of the mass matrices;
 * stiffness integrands are constants (Sec. 3.2 uses order 1 for them). */
static void rule_degree2(int dim, qrule* q)
{
    memset(q, 0, sizeof(*q));
    if (dim == 2) {
        static const double p[3][2] = {{1.0 / 6, 1.0 / 6}, {2.0 / 3, 1.0 / 6}, {1.0 / 6, 2.0 / 3}};
        q->n = 3;
        for (int i = 0; i < 3; i++) {
            q->x[3 * i] = p[i][0];
            q->x[3 * i + 1] = p[i][1];
            q->w[i] = 1.0 / 6.0;
        }
    } else {
        double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
        double p[4][3] = {{b, b, b}, {a, b, b}, {b, a, b}, {b, b, a}};
        q->n = 4;
        for (int i = 0; i < 4; i++) {
            for (int c = 0; c < 3; c++) q->x[3 * i + c] = p[i][c];
            q->w[i] = 1.0 / 24.0;
        }
    }
}

/* Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n. */
static void gauss_legendre01(int n, double* t, double* w)
{
    for (int i = 0; i < n; i++) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < n; k++) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < n; k++) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        t[i] = 0.5 * (x + 1.0);
        w[i] = 1.0 / ((1.0 - x * x) * dp * dp);  /* = (2 / ((1-x^2) P'^2)) / 2 */
    }
}

/* Collapsed (Duffy) product Gauss-Legendre rule with n points per direction:
 * triangle x = (u, v(1-u)), J = 1-u; tetrahedron x = (u, v(1-u), w(1-u)(1-v)),
 * J = (1-u)^2 (1-v). Exact for total degree <= 2n - 1 - (dim - 1). */
static int rule_collapsed(int dim, int n, qrule* q)
{
    double t[64], w[64];
    if (n < 1 || n > 16) return ORA_ERR_ARG;
    memset(q, 0, sizeof(*q));
    gauss_legendre01(n, t, w);
    int m = 0;
    if (dim == 2) {
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                double u = t[i], v = t[j];
                q->x[3 * m] = u;
                q->x[3 * m + 1] = v * (1.0 - u);
                q->w[m] = w[i] * w[j] * (1.0 - u);
                m++;
            }
    } else {
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                for (int k = 0; k < n; k++) {
                    double u = t[i], v = t[j], s = t[k];
                    q->x[3 * m] = u;
                    q->x[3 * m + 1] = v * (1.0 - u);
                    q->x[3 * m + 2] = s * (1.0 - u) * (1.0 - v);
                    q->w[m] = w[i] * w[j] * w[k] * (1.0 - u) * (1.0 - u) * (1.0 - v);
                    m++;
                }
    }
    q->n = m;
    return ORA_OK;
}

static int make_rule(int dim, int rule, int n, qrule* q)
{
    if (rule == 0) {
        rule_degree2(dim, q);
        return ORA_OK;
    }
    return rule_collapsed(dim, n, q);
}

/* ------------------------------------------------------------------------ */
/* Local matrices: plain doubles                                             */
/* ------------------------------------------------------------------------ */

#define SC double
#define FN(name) name##_d
#define SC_C(x) ((double)(x))
#define SC_ADD(a, b) ((a) + (b))
#define SC_SUB(a, b) ((a) - (b))
#define SC_MUL(a, b) ((a) * (b))
#define SC_DIV(a, b) ((a) / (b))
#define SC_NEG(a) (-(a))
#define SC_SCL(a, s) ((a) * (s))
#define SC_V(a) (a)
#include "local_body.inc"
#undef SC
#undef FN
#undef SC_C
#undef SC_ADD
#undef SC_SUB
#undef SC_MUL
#undef SC_DIV
#undef SC_NEG
#undef SC_SCL
#undef SC_V

/* ------------------------------------------------------------------------ */
/* Local matrices: forward-mode dual numbers (12 coordinates + sigma)        */
/* ------------------------------------------------------------------------ */

#define ND 13
typedef struct {
    double v;
    double d[ND];
} dual;

static dual du_c(double x)
{
    dual r;
    memset(&r, 0, sizeof(r));
    r.v = x;
    return r;
}
static dual du_add(dual a, dual b)
{
    for (int i = 0; i < ND; i++) a.d[i] += b.d[i];
    a.v += b.v;
    return a;
}
static dual du_sub(dual a, dual b)
{
    for (int i = 0; i < ND; i++) a.d[i] -= b.d[i];
    a.v -= b.v;
    return a;
}
static dual du_mul(dual a, dual b)
{
    dual r;
    r.v = a.v * b.v;
    for (int i = 0; i < ND; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static dual du_div(dual a, dual b)
{
    dual r;
    r.v = a.v / b.v;
    for (int i = 0; i < ND; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}
static dual du_neg(dual a)
{
    for (int i = 0; i < ND; i++) a.d[i] = -a.d[i];
    a.v = -a.v;
    return a;
}
static dual du_scl(dual a, double s)
{
    for (int i = 0; i < ND; i++) a.d[i] *= s;
    a.v *= s;
    return a;
}

#define SC dual
#define FN(name) name##_dual
#define SC_C(x) du_c(x)
#define SC_ADD(a, b) du_add((a), (b))
#define SC_SUB(a, b) du_sub((a), (b))
#define SC_MUL(a, b) du_mul((a), (b))
#define SC_DIV(a, b) du_div((a), (b))
#define SC_NEG(a) du_neg(a)
#define SC_SCL(a, s) du_scl((a), (s))
#define SC_V(a) ((a).v)
#include "local_body.inc"

/* ------------------------------------------------------------------------ */
/* Topology: edges / faces and their global numbering (Sec. 3)               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n[3];   /* sorted global node ids of the entity (n[2] = -1 for edges) */
    int64_t slot;   /* element * nloc + local DOF */
} ent_rec;

static int cmp_ent(const void* pa, const void* pb)
{
    const ent_rec* a = (const ent_rec*)pa;
    const ent_rec* b = (const ent_rec*)pb;
    for (int i = 0; i < 3; i++) {
        if (a->n[i] < b->n[i]) return -1;
        if (a->n[i] > b->n[i]) return 1;
    }
    if (a->slot < b->slot) return -1;
    if (a->slot > b->slot) return 1;
    return 0;
}

static void sort3(int32_t* v, int m)
{
    for (int i = 1; i < m; i++)
        for (int j = i; j > 0 && v[j - 1] > v[j]; j--) {
            int32_t t = v[j];
            v[j] = v[j - 1];
            v[j - 1] = t;
        }
}

static int check_elems(int dim, int64_t V, int64_t T, const int32_t* elems)
{
    int nv = dim + 1;
    for (int64_t e = 0; e < T; e++)
        for (int a = 0; a < nv; a++) {
            int32_t g = elems[e * nv + a];
            if (g < 0 || (int64_t)g >= V) return ORA_ERR_RANGE;
            for (int b = 0; b < a; b++)
                if (elems[e * nv + b] == g) return ORA_ERR_ARG;
        }
    return ORA_OK;
}

/* elem2dof[T*nl], dof2nodes[N*ne] (malloc'd), N */
static int build_topology(int kind, int dim, int64_t T, const int32_t* elems,
                          int32_t** elem2dof_out, int32_t** dof2nodes_out, int64_t* n_dofs)
{
    int nl = nloc_of(kind, dim), ne = ent_nodes(kind, dim), nv = dim + 1;
    int64_t n = T * nl;
    ent_rec* rec = (ent_rec*)malloc((size_t)(n > 0 ? n : 1) * sizeof(ent_rec));
    int32_t* e2d = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!rec || !e2d) {
        free(rec);
        free(e2d);
        return ORA_ERR_OOM;
    }
    for (int64_t e = 0; e < T; e++)
        for (int k = 0; k < nl; k++) {
            int ln[3], opp;
            ent_rec* r = &rec[e * nl + k];
            local_entity(kind, dim, k, ln, &opp);
            r->n[2] = -1;
            for (int i = 0; i < ne; i++) r->n[i] = elems[e * nv + ln[i]];
            sort3(r->n, ne);
            r->slot = e * nl + k;
        }
    qsort(rec, (size_t)n, sizeof(ent_rec), cmp_ent);
    int64_t N = 0;
    for (int64_t i = 0; i < n; i++) {
        if (i > 0 && memcmp(rec[i].n, rec[i - 1].n, sizeof(rec[i].n)) != 0) N++;
        e2d[rec[i].slot] = (int32_t)(n > 0 ? N : 0);
    }
    if (n > 0) N++;
    int32_t* d2n = (int32_t*)malloc((size_t)(N > 0 ? N : 1) * ne * sizeof(int32_t));
    if (!d2n) {
        free(rec);
        free(e2d);
        return ORA_ERR_OOM;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t d = e2d[rec[i].slot];
        for (int j = 0; j < ne; j++) d2n[d * ne + j] = rec[i].n[j];
    }
    free(rec);
    *elem2dof_out = e2d;
    *dof2nodes_out = d2n;
    *n_dofs = N;
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Orientation signs, decided from geometry (Sec. 2.3)                       */
/* ------------------------------------------------------------------------ */

static void gather_points(int dim, const double* nodes, const int32_t* el, double P[4][3])
{
    for (int a = 0; a < 4; a++)
        for (int c = 0; c < 3; c++) P[a][c] = 0.0;
    for (int a = 0; a <= dim; a++)
        for (int c = 0; c < dim; c++) P[a][c] = nodes[(int64_t)el[a] * dim + c];
}

static double det_of(int dim, double P[4][3])
{
    double B[3][3];
    for (int r = 0; r < dim; r++)
        for (int c = 0; c < dim; c++) B[r][c] = P[c + 1][r] - P[0][r];
    if (dim == 2) return B[0][0] * B[1][1] - B[0][1] * B[1][0];
    return B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
           B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
}

/*
 * Global directions: an edge {a < b} (global ids) is directed from b to a,
 * tangent X_a - X_b; a 2D RT edge carries the normal R_cw (X_a - X_b) with
 * R_cw (x, y) = (y, -x); a face {a < b < c} carries N = (X_b - X_a) x (X_c - X_a).
 *
 * Ned (covariant Piola): the mapped local tangent is B t_k, parallel to
 *   X_head - X_tail, so s_k = sign((X_head - X_tail) . (X_a - X_b)).
 * RT (contravariant Piola): the flux of (1/det B) B eta_k through the
 *   physical edge/face in its OUTWARD direction is sign(det B) times the
 *   reference flux (Sec. 2.3: it depends on whether F_K keeps orientation), so
 *   s_k = sign(det B) * sign(n_out . N). The outward side is found from the
 *   opposite vertex: n_out . N has the sign of N . (X_on_entity - X_opposite).
 */
static int element_signs(int kind, int dim, const double* nodes, const int32_t* el, double* sgn)
{
    double P[4][3];
    int nl = nloc_of(kind, dim), ne = ent_nodes(kind, dim);
    gather_points(dim, nodes, el, P);
    double det = det_of(dim, P);
    if (det == 0.0) return ORA_ERR_DEGENERATE;
    for (int k = 0; k < nl; k++) {
        int ln[3], opp;
        local_entity(kind, dim, k, ln, &opp);
        /* global ids and positions of the entity nodes, sorted by global id */
        int idx[3] = {ln[0], ln[1], ne == 3 ? ln[2] : -1};
        for (int i = 1; i < ne; i++)
            for (int j = i; j > 0 && el[idx[j - 1]] > el[idx[j]]; j--) {
                int t = idx[j];
                idx[j] = idx[j - 1];
                idx[j - 1] = t;
            }
        double s;
        if (kind == ORA_NED1) {
            double dot = 0.0;
            for (int c = 0; c < dim; c++) dot += (P[ln[1]][c] - P[ln[0]][c]) * (P[idx[0]][c] - P[idx[1]][c]);
            if (dot == 0.0) return ORA_ERR_DEGENERATE;
            s = dot > 0 ? 1.0 : -1.0;
        } else if (dim == 2) {
            double tx = P[idx[0]][0] - P[idx[1]][0], ty = P[idx[0]][1] - P[idx[1]][1];
            double Nx = ty, Ny = -tx;
            double side = Nx * (P[ln[0]][0] - P[opp][0]) + Ny * (P[ln[0]][1] - P[opp][1]);
            if (side == 0.0) return ORA_ERR_DEGENERATE;
            s = ((det > 0) == (side > 0)) ? 1.0 : -1.0;
        } else {
            double u[3], v[3], N[3], side = 0.0;
            for (int c = 0; c < 3; c++) {
                u[c] = P[idx[1]][c] - P[idx[0]][c];
                v[c] = P[idx[2]][c] - P[idx[0]][c];
            }
            N[0] = u[1] * v[2] - u[2] * v[1];
            N[1] = u[2] * v[0] - u[0] * v[2];
            N[2] = u[0] * v[1] - u[1] * v[0];
            for (int c = 0; c < 3; c++) side += N[c] * (P[idx[0]][c] - P[opp][c]);
            if (side == 0.0) return ORA_ERR_DEGENERATE;
            s = ((det > 0) == (side > 0)) ? 1.0 : -1.0;
        }
        sgn[k] = s;
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* CSR pattern: every pair of DOFs that share an element                     */
/* ------------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static int build_pattern(int nl, int64_t T, int64_t N, const int32_t* e2d, int64_t** rowptr_out,
                         int32_t** colidx_out, int64_t* nnz_out)
{
    int64_t* cnt = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    int64_t* inc = (int64_t*)malloc((size_t)(T * nl > 0 ? T * nl : 1) * sizeof(int64_t));
    int64_t* rowptr = (int64_t*)malloc(((size_t)N + 1) * sizeof(int64_t));
    if (!cnt || !inc || !rowptr) goto oom;
    /* DOF -> incident elements, ascending */
    for (int64_t i = 0; i < T * nl; i++) cnt[e2d[i] + 1]++;
    for (int64_t d = 0; d < N; d++) cnt[d + 1] += cnt[d];
    {
        int64_t* fill = (int64_t*)malloc(((size_t)N + 1) * sizeof(int64_t));
        if (!fill) goto oom;
        memcpy(fill, cnt, ((size_t)N + 1) * sizeof(int64_t));
        for (int64_t e = 0; e < T; e++)
            for (int k = 0; k < nl; k++) inc[fill[e2d[e * nl + k]]++] = e;
        free(fill);
    }
    /* row lengths, then the column lists */
    int32_t* buf = NULL;
    int64_t bufcap = 0, nnz = 0;
    rowptr[0] = 0;
    for (int pass = 0; pass < 2; pass++) {
        int32_t* colidx = NULL;
        if (pass == 1) {
            colidx = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
            if (!colidx) {
                free(buf);
                goto oom;
            }
        }
        for (int64_t d = 0; d < N; d++) {
            int64_t m = (cnt[d + 1] - cnt[d]) * nl;
            if (m > bufcap) {
                bufcap = 2 * m;
                buf = (int32_t*)realloc(buf, (size_t)bufcap * sizeof(int32_t));
                if (!buf) goto oom;
            }
            int64_t w = 0;
            for (int64_t j = cnt[d]; j < cnt[d + 1]; j++)
                for (int k = 0; k < nl; k++) buf[w++] = e2d[inc[j] * nl + k];
            qsort(buf, (size_t)w, sizeof(int32_t), cmp_i32);
            int64_t u = 0;
            for (int64_t j = 0; j < w; j++)
                if (j == 0 || buf[j] != buf[j - 1]) buf[u++] = buf[j];
            if (pass == 0)
                rowptr[d + 1] = rowptr[d] + u;
            else
                memcpy(colidx + rowptr[d], buf, (size_t)u * sizeof(int32_t));
        }
        if (pass == 0) nnz = rowptr[N];
        else *colidx_out = colidx;
    }
    free(buf);
    free(cnt);
    free(inc);
    *rowptr_out = rowptr;
    *nnz_out = nnz;
    return ORA_OK;
oom:
    free(cnt);
    free(inc);
    free(rowptr);
    return ORA_ERR_OOM;
}

static int64_t find_col(const int64_t* rowptr, const int32_t* colidx, int64_t row, int32_t col)
{
    int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (colidx[mid] == col) return mid;
        if (colidx[mid] < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Exported API                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n_elems, n_dofs, nnz;
    int32_t nloc, ent_nodes;
    int32_t* elem2dof;   /* n_elems x nloc                      */
    int8_t* sign;        /* n_elems x nloc, +1 / -1            */
    int32_t* dof2nodes;  /* n_dofs x ent_nodes, ascending ids  */
    int64_t* rowptr;     /* n_dofs + 1                          */
    int32_t* colidx;     /* nnz, ascending within a row         */
    double* K;           /* nnz */
    double* M;           /* nnz */
    double* Kabs;        /* nnz: sum of |local contributions|   */
    double* Mabs;        /* nnz                                 */
} ora_result;

void ora_free(ora_result* r)
{
    if (!r) return;
    free(r->elem2dof);
    free(r->sign);
    free(r->dof2nodes);
    free(r->rowptr);
    free(r->colidx);
    free(r->K);
    free(r->M);
    free(r->Kabs);
    free(r->Mabs);
    memset(r, 0, sizeof(*r));
}

int ora_nloc(int kind, int dim)
{
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    return nloc_of(kind, dim);
}

/* Quadrature rule: rule 0 = symmetric degree-2 rule, rule 1 = collapsed
 * Gauss-Legendre with n points per direction. Writes up to cap points
 * (x as 3 doubles each) and returns the number of points. */
int ora_quadrature(int dim, int rule, int n, double* x, double* w, int cap)
{
    static qrule q;
    if (dim != 2 && dim != 3) return ORA_ERR_ARG;
    int st = make_rule(dim, rule, n, &q);
    if (st) return st;
    if (q.n > cap) return ORA_ERR_ARG;
    memcpy(x, q.x, sizeof(double) * 3 * q.n);
    memcpy(w, q.w, sizeof(double) * q.n);
    return q.n;
}

/* Reference basis values (nloc x dim) and divergence/curl (nloc x 1, or
 * nloc x 3 for the 3D curl) at one reference point. */
int ora_ref_basis(int kind, int dim, const double* xh, double* val, double* dval)
{
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    const affine_field* b = ref_basis(kind, dim);
    int nl = nloc_of(kind, dim);
    int nd = (kind == ORA_NED1 && dim == 3) ? 3 : 1;
    for (int k = 0; k < nl; k++) {
        for (int r = 0; r < dim; r++) {
            double v = b[k].a[r];
            for (int c = 0; c < dim; c++) v += b[k].A[r][c] * xh[c];
            val[k * dim + r] = v;
        }
        if (kind == ORA_RT0) {
            double d = 0;
            for (int r = 0; r < dim; r++) d += b[k].A[r][r];
            dval[k] = d;
        } else if (dim == 2) {
            dval[k] = b[k].A[1][0] - b[k].A[0][1];
        } else {
            dval[k * nd + 0] = b[k].A[2][1] - b[k].A[1][2];
            dval[k * nd + 1] = b[k].A[0][2] - b[k].A[2][0];
            dval[k * nd + 2] = b[k].A[1][0] - b[k].A[0][1];
        }
    }
    return nl;
}

/* Local K and M of one element with vertices P ((dim+1) x dim) and the given
 * signs, by quadrature rule (rule, n). Output nloc x nloc each, row-major. */
int ora_local(int kind, int dim, const double* P, const double* sgn, double coeff, int rule, int n,
              double* Kout, double* Mout)
{
    static qrule q;
    double Pl[4][3] = {{0}}, Kl[6][6], Ml[6][6];
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    int st = make_rule(dim, rule, n, &q);
    if (st) return st;
    for (int a = 0; a <= dim; a++)
        for (int c = 0; c < dim; c++) Pl[a][c] = P[a * dim + c];
    st = local_matrices_d(kind, dim, Pl, sgn, coeff, &q, Kl, Ml);
    if (st) return st;
    int nl = nloc_of(kind, dim);
    for (int k = 0; k < nl; k++)
        for (int l = 0; l < nl; l++) {
            Kout[k * nl + l] = Kl[k][l];
            Mout[k * nl + l] = Ml[k][l];
        }
    return ORA_OK;
}

/* Topology and signs only (no pattern, no values). */
int ora_topology(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems,
                 ora_result* out)
{
    memset(out, 0, sizeof(*out));
    if (!valid_kind(kind, dim) || V < 0 || T < 0 || !elems || !nodes) return ORA_ERR_ARG;
    int st = check_elems(dim, V, T, elems);
    if (st) return st;
    int nl = nloc_of(kind, dim);
    out->n_elems = T;
    out->nloc = nl;
    out->ent_nodes = ent_nodes(kind, dim);
    st = build_topology(kind, dim, T, elems, &out->elem2dof, &out->dof2nodes, &out->n_dofs);
    if (st) {
        ora_free(out);
        return st;
    }
    out->sign = (int8_t*)malloc((size_t)(T * nl > 0 ? T * nl : 1));
    if (!out->sign) {
        ora_free(out);
        return ORA_ERR_OOM;
    }
    for (int64_t e = 0; e < T; e++) {
        double s[6];
        st = element_signs(kind, dim, nodes, elems + e * (dim + 1), s);
        if (st) {
            ora_free(out);
            return st;
        }
        for (int k = 0; k < nl; k++) out->sign[e * nl + k] = (int8_t)(s[k] > 0 ? 1 : -1);
    }
    return ORA_OK;
}

/* Full assembly: topology, signs, pattern, and K / M values by quadrature
 * rule (rule, n), K scaled by coeff_K and M by coeff_M (either may be NULL:
 * unit coefficient). With two different arrays the local matrices are
 * evaluated once per coefficient and K taken from the first, M from the
 * second (the matrices are linear in the coefficient). */
int ora_assemble2(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems,
                  const double* coeff_K, const double* coeff_M, int rule, int n, ora_result* out)
{
    static qrule q;
    int st = ora_topology(kind, dim, V, nodes, T, elems, out);
    if (st) return st;
    st = make_rule(dim, rule, n, &q);
    if (st) {
        ora_free(out);
        return st;
    }
    int nl = out->nloc, nv = dim + 1;
    st = build_pattern(nl, T, out->n_dofs, out->elem2dof, &out->rowptr, &out->colidx, &out->nnz);
    if (st) {
        ora_free(out);
        return st;
    }
    size_t nz = (size_t)(out->nnz > 0 ? out->nnz : 1);
    out->K = (double*)calloc(nz, sizeof(double));
    out->M = (double*)calloc(nz, sizeof(double));
    out->Kabs = (double*)calloc(nz, sizeof(double));
    out->Mabs = (double*)calloc(nz, sizeof(double));
    if (!out->K || !out->M || !out->Kabs || !out->Mabs) {
        ora_free(out);
        return ORA_ERR_OOM;
    }
    for (int64_t e = 0; e < T; e++) {
        double P[4][3], s[6], Kl[6][6], Ml[6][6];
        gather_points(dim, nodes, elems + e * nv, P);
        for (int k = 0; k < nl; k++) s[k] = out->sign[e * nl + k];
        st = local_matrices_d(kind, dim, P, s, coeff_K ? coeff_K[e] : 1.0, &q, Kl, Ml);
        if (!st && coeff_M != coeff_K) {
            double K2[6][6];
            st = local_matrices_d(kind, dim, P, s, coeff_M ? coeff_M[e] : 1.0, &q, K2, Ml);
        }
        if (st) {
            ora_free(out);
            return st;
        }
        for (int k = 0; k < nl; k++)
            for (int l = 0; l < nl; l++) {
                int64_t p = find_col(out->rowptr, out->colidx, out->elem2dof[e * nl + k], out->elem2dof[e * nl + l]);
                if (p < 0) {
                    ora_free(out);
                    return ORA_ERR_ARG;
                }
                out->K[p] += Kl[k][l];
                out->M[p] += Ml[k][l];
                out->Kabs[p] += fabs(Kl[k][l]);
                out->Mabs[p] += fabs(Ml[k][l]);
            }
    }
    return ORA_OK;
}

/* One coefficient for both matrices. */
int ora_assemble(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems,
                 const double* coeff, int rule, int n, ora_result* out)
{
    return ora_assemble2(kind, dim, V, nodes, T, elems, coeff, coeff, rule, n, out);
}

/*
 * Adjoint of J = sum_K sigma_K (u_K^T Khat_K u_K + v_K^T Mhat_K v_K), where
 * Khat_K, Mhat_K are the signed local matrices with unit coefficient and
 * u_K = u[elem2dof(K, :)]. Forward mode: the 12 vertex coordinates of an
 * element and sigma_K are seeded as 13 dual directions, the local matrices
 * are evaluated by the same quadrature code as the assembly, and the element's
 * derivatives are added to the node gradient in ascending element order.
 * grad_nodes: V x dim, grad_coeff: T. coeff may be NULL (unit).
 */
int ora_adjoint(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems,
                const double* coeff, const double* u, const double* v, int rule, int n, double* J,
                double* grad_nodes, double* grad_coeff)
{
    static qrule q;
    ora_result topo;
    int st = ora_topology(kind, dim, V, nodes, T, elems, &topo);
    if (st) return st;
    st = make_rule(dim, rule, n, &q);
    if (st) {
        ora_free(&topo);
        return st;
    }
    int nl = topo.nloc, nv = dim + 1;
    double Jsum = 0.0;
    memset(grad_nodes, 0, sizeof(double) * (size_t)V * dim);
    for (int64_t e = 0; e < T; e++) {
        dual P[4][3], Kl[6][6], Ml[6][6];
        double s[6];
        const int32_t* el = elems + e * nv;
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) P[a][c] = du_c(0.0);
        for (int a = 0; a < nv; a++)
            for (int c = 0; c < dim; c++) {
                P[a][c] = du_c(nodes[(int64_t)el[a] * dim + c]);
                P[a][c].d[a * 3 + c] = 1.0;
            }
        dual sig = du_c(coeff ? coeff[e] : 1.0);
        sig.d[12] = 1.0;
        for (int k = 0; k < nl; k++) s[k] = topo.sign[e * nl + k];
        st = local_matrices_dual(kind, dim, P, s, sig, &q, Kl, Ml);
        if (st) {
            ora_free(&topo);
            return st;
        }
        dual Je = du_c(0.0);
        for (int k = 0; k < nl; k++)
            for (int l = 0; l < nl; l++) {
                double uk = u[topo.elem2dof[e * nl + k]], ul = u[topo.elem2dof[e * nl + l]];
                double vk = v[topo.elem2dof[e * nl + k]], vl = v[topo.elem2dof[e * nl + l]];
                Je = du_add(Je, du_scl(Kl[k][l], uk * ul));
                Je = du_add(Je, du_scl(Ml[k][l], vk * vl));
            }
        Jsum += Je.v;
        for (int a = 0; a < nv; a++)
            for (int c = 0; c < dim; c++) grad_nodes[(int64_t)el[a] * dim + c] += Je.d[a * 3 + c];
        grad_coeff[e] = Je.d[12];
    }
    *J = Jsum;
    ora_free(&topo);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Vectorised integration (Sec. 3.1, norm_L2)                                 */
/* ------------------------------------------------------------------------ */

/* Physical quadrature points x = B xhat_q + P_0 of every element for the
 * collapsed Gauss-Legendre rule with n points per direction (rule 1),
 * point-major: x[(q * T + e) * dim + c]. Returns the number of points. */
int ora_quad_points(int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems, int n, double* x)
{
    static qrule q;
    if ((dim != 2 && dim != 3) || V < 0 || T < 0) return ORA_ERR_ARG;
    int st = make_rule(dim, 1, n, &q);
    if (st) return st;
    for (int64_t e = 0; e < T; e++) {
        double P[4][3];
        gather_points(dim, nodes, elems + e * (dim + 1), P);
        for (int i = 0; i < q.n; i++)
            for (int r = 0; r < dim; r++) {
                double xr = P[0][r];
                for (int c = 0; c < dim; c++) xr += (P[c + 1][r] - P[0][r]) * q.x[3 * i + c];
                x[((int64_t)i * T + e) * dim + r] = xr;
            }
    }
    return q.n;
}

/* Squared L2 norm, element by element, of f - v_h over the mesh by the same
 * rule: elem_out[e] = |det B_K| sum_q w_q |f_q - v_h(x_q)|^2 (the paper's
 * fnorm), *total = their sum in element order. f: [q][element][ncomp] at the
 * points of ora_quad_points; v: DOF vector (n_dofs) or NULL (v_h = 0), with
 * v_h = sum_k s_k v[dof_k] phi_k, phi_k = (1/det B) B eta_k (RT0, Eq.
 * RT0piola) or B^-T eta_k (Nedelec, Ned0piola1) at xhat_q, s_k the geometric
 * signs. elem_out may be NULL. */
int ora_norm_l2(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems, int n, int ncomp,
                const double* f, const double* v, double* elem_out, double* total)
{
    static qrule q;
    ora_result topo;
    memset(&topo, 0, sizeof(topo));
    if (!valid_kind(kind, dim) || ncomp < 1 || ncomp > 3 || (v && ncomp != dim)) return ORA_ERR_ARG;
    int st = make_rule(dim, 1, n, &q);
    if (st) return st;
    if (v) {
        st = ora_topology(kind, dim, V, nodes, T, elems, &topo);
        if (st) return st;
    }
    const affine_field* basis = ref_basis(kind, dim);
    int nl = nloc_of(kind, dim);
    double sum = 0.0;
    for (int64_t e = 0; e < T; e++) {
        double P[4][3], B[3][3], Bi[3][3];
        gather_points(dim, nodes, elems + e * (dim + 1), P);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) B[r][c] = (r < dim && c < dim) ? P[c + 1][r] - P[0][r] : (r == c ? 1.0 : 0.0);
        double det = det_of(dim, P);
        if (det == 0.0) {
            ora_free(&topo);
            return ORA_ERR_DEGENERATE;
        }
        /* B^-1 = adj(B) / det (cofactors; the 2D case has B[2][2] = 1) */
        Bi[0][0] = (B[1][1] * B[2][2] - B[1][2] * B[2][1]) / det;
        Bi[0][1] = (B[0][2] * B[2][1] - B[0][1] * B[2][2]) / det;
        Bi[0][2] = (B[0][1] * B[1][2] - B[0][2] * B[1][1]) / det;
        Bi[1][0] = (B[1][2] * B[2][0] - B[1][0] * B[2][2]) / det;
        Bi[1][1] = (B[0][0] * B[2][2] - B[0][2] * B[2][0]) / det;
        Bi[1][2] = (B[0][2] * B[1][0] - B[0][0] * B[1][2]) / det;
        Bi[2][0] = (B[1][0] * B[2][1] - B[1][1] * B[2][0]) / det;
        Bi[2][1] = (B[0][1] * B[2][0] - B[0][0] * B[2][1]) / det;
        Bi[2][2] = (B[0][0] * B[1][1] - B[0][1] * B[1][0]) / det;
        double acc = 0.0;
        for (int i = 0; i < q.n; i++) {
            const double* xh = q.x + 3 * i;
            double vh[3] = {0.0, 0.0, 0.0};
            if (v) {
                for (int k = 0; k < nl; k++) {
                    double eta[3] = {0.0, 0.0, 0.0}, phi[3] = {0.0, 0.0, 0.0};
                    for (int r = 0; r < dim; r++) {
                        eta[r] = basis[k].a[r];
                        for (int c = 0; c < dim; c++) eta[r] += basis[k].A[r][c] * xh[c];
                    }
                    for (int r = 0; r < dim; r++)
                        for (int c = 0; c < dim; c++)
                            phi[r] += (kind == ORA_RT0) ? B[r][c] * eta[c] / det : Bi[c][r] * eta[c];
                    double coef = topo.sign[e * nl + k] * v[topo.elem2dof[e * nl + k]];
                    for (int r = 0; r < dim; r++) vh[r] += coef * phi[r];
                }
            }
            double d2 = 0.0;
            for (int c = 0; c < ncomp; c++) {
                double d = f[((int64_t)i * T + e) * ncomp + c] - vh[c];
                d2 += d * d;
            }
            acc += q.w[i] * d2;
        }
        double ne = fabs(det) * acc;
        if (elem_out) elem_out[e] = ne;
        sum += ne;
    }
    if (total) *total = sum;
    ora_free(&topo);
    return ORA_OK;
}

/* Shared by the functions below: B (dim x dim, identity-padded), B^-1, det. */
static int element_frame(int dim, const double* nodes, const int32_t* el, double P[4][3], double B[3][3],
                         double Bi[3][3], double* det)
{
    gather_points(dim, nodes, el, P);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) B[r][c] = (r < dim && c < dim) ? P[c + 1][r] - P[0][r] : (r == c ? 1.0 : 0.0);
    *det = det_of(dim, P);
    if (*det == 0.0) return ORA_ERR_DEGENERATE;
    double d = *det;
    Bi[0][0] = (B[1][1] * B[2][2] - B[1][2] * B[2][1]) / d;
    Bi[0][1] = (B[0][2] * B[2][1] - B[0][1] * B[2][2]) / d;
    Bi[0][2] = (B[0][1] * B[1][2] - B[0][2] * B[1][1]) / d;
    Bi[1][0] = (B[1][2] * B[2][0] - B[1][0] * B[2][2]) / d;
    Bi[1][1] = (B[0][0] * B[2][2] - B[0][2] * B[2][0]) / d;
    Bi[1][2] = (B[0][2] * B[1][0] - B[0][0] * B[1][2]) / d;
    Bi[2][0] = (B[1][0] * B[2][1] - B[1][1] * B[2][0]) / d;
    Bi[2][1] = (B[0][1] * B[2][0] - B[0][0] * B[2][1]) / d;
    Bi[2][2] = (B[0][0] * B[1][1] - B[0][1] * B[1][0]) / d;
    return ORA_OK;
}

/* Mapped reference basis function k at xhat (unsigned): (1/det B) B eta_k
 * (RT0, Eq. RT0piola) or B^-T eta_k (Nedelec, Ned0piola1). */
static void mapped_basis(int kind, int dim, int k, const double* xh, double B[3][3], double Bi[3][3], double det,
                         double phi[3])
{
    const affine_field* f = &ref_basis(kind, dim)[k];
    double eta[3] = {0.0, 0.0, 0.0};
    for (int r = 0; r < dim; r++) {
        eta[r] = f->a[r];
        for (int c = 0; c < dim; c++) eta[r] += f->A[r][c] * xh[c];
    }
    for (int r = 0; r < 3; r++) phi[r] = 0.0;
    for (int r = 0; r < dim; r++)
        for (int c = 0; c < dim; c++) phi[r] += (kind == ORA_RT0) ? B[r][c] * eta[c] / det : Bi[c][r] * eta[c];
}

/* Load vector b_i = int F . eta_i by the collapsed Gauss-Legendre rule (n per
 * direction): element by element in ascending order, b[dof_k] += s_k |det B|
 * sum_q w_q F_q . phi_k(xhat_q). F: [q][element][dim] at ora_quad_points. */
int ora_load_vector(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems, int n,
                    const double* F, double* b)
{
    static qrule q;
    ora_result topo;
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    int st = make_rule(dim, 1, n, &q);
    if (st) return st;
    st = ora_topology(kind, dim, V, nodes, T, elems, &topo);
    if (st) return st;
    int nl = nloc_of(kind, dim);
    for (int64_t i = 0; i < topo.n_dofs; i++) b[i] = 0.0;
    for (int64_t e = 0; e < T; e++) {
        double P[4][3], B[3][3], Bi[3][3], det;
        st = element_frame(dim, nodes, elems + e * (dim + 1), P, B, Bi, &det);
        if (st) {
            ora_free(&topo);
            return st;
        }
        for (int k = 0; k < nl; k++) {
            double acc = 0.0;
            for (int i = 0; i < q.n; i++) {
                double phi[3];
                mapped_basis(kind, dim, k, q.x + 3 * i, B, Bi, det, phi);
                double d = 0.0;
                for (int c = 0; c < dim; c++) d += F[((int64_t)i * T + e) * dim + c] * phi[c];
                acc += q.w[i] * d;
            }
            b[topo.elem2dof[e * nl + k]] += topo.sign[e * nl + k] * fabs(det) * acc;
        }
    }
    ora_free(&topo);
    return ORA_OK;
}

/* Derivative load vector b_i = int g . D eta_i with D = div (RT0) or curl
 * (Nedelec), by the collapsed Gauss-Legendre rule (n per direction). The
 * derivative of a mapped basis function is constant on an element and comes
 * from the reference basis's derivatives: div eta_k / det B (Eq. RT0piola),
 * curl eta_k / det B (2D) and B curl eta_k / det B (3D) (Ned0piola2/3).
 * g: [q][element][ncomp] at ora_quad_points, ncomp = 3 for 3D Nedelec, 1
 * otherwise. Element by element in ascending order: b[dof_k] += s_k |det B|
 * sum_q w_q g_q . D eta_k. */
int ora_load_derivative(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems, int n,
                        const double* g, double* b)
{
    static qrule q;
    ora_result topo;
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    int st = make_rule(dim, 1, n, &q);
    if (st) return st;
    st = ora_topology(kind, dim, V, nodes, T, elems, &topo);
    if (st) return st;
    const affine_field* basis = ref_basis(kind, dim);
    int nl = nloc_of(kind, dim);
    int nc = (kind == ORA_NED1 && dim == 3) ? 3 : 1;
    for (int64_t i = 0; i < topo.n_dofs; i++) b[i] = 0.0;
    for (int64_t e = 0; e < T; e++) {
        double P[4][3], B[3][3], Bi[3][3], det;
        st = element_frame(dim, nodes, elems + e * (dim + 1), P, B, Bi, &det);
        if (st) {
            ora_free(&topo);
            return st;
        }
        for (int k = 0; k < nl; k++) {
            const affine_field* f = &basis[k];
            double D[3] = {0.0, 0.0, 0.0};
            if (kind == ORA_RT0) {
                for (int r = 0; r < dim; r++) D[0] += f->A[r][r];
                D[0] /= det;
            } else if (dim == 2) {
                D[0] = (f->A[1][0] - f->A[0][1]) / det;
            } else {
                double cr[3] = {f->A[2][1] - f->A[1][2], f->A[0][2] - f->A[2][0], f->A[1][0] - f->A[0][1]};
                for (int r = 0; r < 3; r++)
                    for (int c = 0; c < 3; c++) D[r] += B[r][c] * cr[c] / det;
            }
            double acc = 0.0;
            for (int i = 0; i < q.n; i++) {
                double d = 0.0;
                for (int c = 0; c < nc; c++) d += g[((int64_t)i * T + e) * nc + c] * D[c];
                acc += q.w[i] * d;
            }
            b[topo.elem2dof[e * nl + k]] += topo.sign[e * nl + k] * fabs(det) * acc;
        }
    }
    ora_free(&topo);
    return ORA_OK;
}

/* Values at the points of ora_quad_points of v_h = sum_k s_k v[dof_k] phi_k:
 * out [q][element][dim]. */
int ora_fe_values(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems, int n,
                  const double* v, double* out)
{
    static qrule q;
    ora_result topo;
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    int st = make_rule(dim, 1, n, &q);
    if (st) return st;
    st = ora_topology(kind, dim, V, nodes, T, elems, &topo);
    if (st) return st;
    int nl = nloc_of(kind, dim);
    for (int64_t e = 0; e < T; e++) {
        double P[4][3], B[3][3], Bi[3][3], det;
        st = element_frame(dim, nodes, elems + e * (dim + 1), P, B, Bi, &det);
        if (st) {
            ora_free(&topo);
            return st;
        }
        for (int i = 0; i < q.n; i++) {
            double vh[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < nl; k++) {
                double phi[3];
                mapped_basis(kind, dim, k, q.x + 3 * i, B, Bi, det, phi);
                double coef = topo.sign[e * nl + k] * v[topo.elem2dof[e * nl + k]];
                for (int r = 0; r < dim; r++) vh[r] += coef * phi[r];
            }
            for (int r = 0; r < dim; r++) out[((int64_t)i * T + e) * dim + r] = vh[r];
        }
    }
    ora_free(&topo);
    return ORA_OK;
}

/* Per element: curl (Nedelec; Ned0piola2/3: curl eta / det B in 2D, B curl
 * eta / det B in 3D) or divergence (RT0: div eta / det B) of v_h, from the
 * derivatives of the reference basis. out: [T] or [T][3] (3D Nedelec). */
int ora_fe_curl(int kind, int dim, int64_t V, const double* nodes, int64_t T, const int32_t* elems, const double* v,
                double* out)
{
    ora_result topo;
    if (!valid_kind(kind, dim)) return ORA_ERR_ARG;
    int st = ora_topology(kind, dim, V, nodes, T, elems, &topo);
    if (st) return st;
    const affine_field* basis = ref_basis(kind, dim);
    int nl = nloc_of(kind, dim);
    for (int64_t e = 0; e < T; e++) {
        double P[4][3], B[3][3], Bi[3][3], det;
        st = element_frame(dim, nodes, elems + e * (dim + 1), P, B, Bi, &det);
        if (st) {
            ora_free(&topo);
            return st;
        }
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nl; k++) {
            const affine_field* f = &basis[k];
            double coef = topo.sign[e * nl + k] * v[topo.elem2dof[e * nl + k]];
            if (kind == ORA_RT0) {
                double dv = 0.0;
                for (int r = 0; r < dim; r++) dv += f->A[r][r];
                acc[0] += coef * dv / det;
            } else if (dim == 2) {
                acc[0] += coef * (f->A[1][0] - f->A[0][1]) / det;
            } else {
                double cr[3] = {f->A[2][1] - f->A[1][2], f->A[0][2] - f->A[2][0], f->A[1][0] - f->A[0][1]};
                for (int r = 0; r < 3; r++)
                    for (int c = 0; c < 3; c++) acc[r] += coef * B[r][c] * cr[c] / det;
            }
        }
        if (kind == ORA_NED1 && dim == 3)
            for (int r = 0; r < 3; r++) out[e * 3 + r] = acc[r];
        else
            out[e] = acc[0];
    }
    ora_free(&topo);
    return ORA_OK;
}
