/*
 * edgefem.h -- C ABI of libedgefem.so: GPU assembly of lowest-order
 * Raviart-Thomas (H(div)) and Nedelec first-kind (H(curl)) mass and
 * div/curl stiffness matrices on triangle and tetrahedron meshes into
 * global CSR matrices, after I. Anjam and J. Valdman, "Fast MATLAB assembly
 * of FEM matrices in 2D and 3D: Edge elements" (arXiv 1409.4618).
 *
 * The matrices (Sec. 2.4):
 *   M_ij = int_Omega sigma eta_i . eta_j,
 *   K_ij = int_Omega sigma div eta_i div eta_j        (RT0),
 *   K_ij = int_Omega sigma curl eta_i . curl eta_j    (Nedelec, curl scalar in 2D),
 * where eta_i are the global basis functions built from the reference bases
 * of Sec. 2.1-2.2 with the Piola maps of Eqs. RT0piola and Ned0piola1-3 and
 * the orientation signs of Sec. 2.3, and sigma is a per-element coefficient
 * (1 if none is given) that scales both K and M. The 3D RT0 basis is used
 * exactly as printed in Sec. 2.1 (its face fluxes are 1/2).
 *
 * Conventions shared by every entry point:
 *   - Meshes: nodes are V x dim doubles, row-major (x, y[, z] per node);
 *     elements are T x (dim+1) int32 node ids, row-major, 0-based. Any
 *     orientation (det B_K of either sign) is allowed (Sec. 2.3).
 *   - Global DOF numbering (Sec. 3, "row indices of edges2nodes /
 *     faces2nodes"): the DOFs are the distinct edges (faces for 3D RT0) ranked
 *     lexicographically by their sorted global node ids.
 *   - Local DOF order and directions (Fig. 1): 2D edge k lies opposite local
 *     node k and runs (1,2), (2,0), (0,1); 3D edges run (0,1), (0,2), (0,3),
 *     (1,2), (2,3), (3,1); 3D face k is opposite local node 3-k.
 *   - Orientation signs (Sec. 2.3): an edge DOF gets +1 iff the global id of
 *     its tail exceeds that of its head (the rule Sec. 3 states for 2D,
 *     applied to every edge); a face DOF gets -parity of the permutation that
 *     lists its three nodes by ascending global id followed by the opposite
 *     node. Sign bit k of an element is set iff its sign is -1.
 *   - CSR: 0-based, both triangles stored, columns ascending within a row,
 *     int64 row pointers, int32 column indices. The pattern holds every pair
 *     of DOFs that share an element; entries that happen to be zero are kept.
 *     K and M share one pattern.
 *   - Pointers named d_* are CUDA device pointers, h_* host pointers. The
 *     caller owns every buffer it passes; the library owns plan internals.
 *     `stream` is a cudaStream_t (NULL = the legacy default stream); all
 *     device work of a call is ordered on it.
 *   - Every call returns EF_OK (0) or a negative status; nothing is written
 *     to caller buffers when an argument check fails. There is no CPU
 *     fallback: without a CUDA device every compute call returns EF_ERR_CUDA.
 *   - All floating-point arithmetic is IEEE FP64. Sums of element
 *     contributions are formed in a fixed order (ascending element id within
 *     a nonzero), without floating-point atomics: results are bitwise
 *     reproducible from run to run.
 */
#ifndef EDGEFEM_H
#define EDGEFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EF_OK 0
#define EF_ERR_ARG (-1)          /* bad pointer, size, kind or dim; repeated node in an element */
#define EF_ERR_RANGE (-2)        /* node id outside [0, n_nodes) */
#define EF_ERR_DEGENERATE (-3)   /* an element has det B_K = 0 (|det B_K| below 2^-1022, or not finite) */
#define EF_ERR_KEY_OVERFLOW (-4) /* 3D RT0 face keys need n_nodes^3 < 2^64 (n_nodes <= 2642245) */
#define EF_ERR_OOM (-5)          /* device allocation failed */
#define EF_ERR_CUDA (-6)         /* a CUDA runtime call failed (see ef_last_error) */
#define EF_ERR_TIMEOUT (-7)      /* a bounded device-side wait gave up */
#define EF_ERR_SIZE (-8)         /* size beyond a limit stated per call (32-bit indices, fixed scratch) */

typedef enum { EF_RT0 = 1, EF_NED1 = 2 } ef_kind;

typedef struct ef_plan ef_plan;

/*
 * Build the per-mesh plan: topology (edges / faces, their global numbering
 * and the per-element orientation signs; Sec. 3 "get_edges / get_faces /
 * signs_edges / signs_faces") and the CSR pattern with the map from every
 * element contribution to its nonzero. Depends on the connectivity only,
 * never on coordinates or coefficients; reused by every ef_assemble.
 *   kind: EF_RT0 or EF_NED1; dim: 2 or 3.
 *   d_elems: n_elems x (dim+1) int32, device; copied, may be freed after.
 * Synchronises `stream` (the sizes of the plan depend on the data).
 * Errors: EF_ERR_ARG, EF_ERR_RANGE, EF_ERR_KEY_OVERFLOW, EF_ERR_OOM,
 *   EF_ERR_CUDA, EF_ERR_SIZE (n_elems * nloc(nloc+1)/2 >= 2^32 or nnz >= 2^32).
 * On success *out owns device memory until ef_plan_destroy.
 */
int ef_plan_create(int kind, int dim, int64_t n_nodes, int64_t n_elems, const int32_t* d_elems, void* stream,
                   ef_plan** out);

/* Number of global DOFs (rows) and CSR nonzeros of the plan. Host only. */
int ef_plan_sizes(const ef_plan* plan, int64_t* n_dofs, int64_t* nnz);

/* Plan facts for diagnostics and benchmarks (host only): counts and how
 * ef_assemble runs. Not part of the paper's method. */
typedef struct {
    int64_t n_dofs, nnz;
    int64_t n_upper;              /* nonzeros with row <= column */
    int64_t n_contrib;            /* element contributions: n_elems * nloc (nloc+1) / 2 */
    int32_t assemble_launches;    /* kernel launches made by one ef_assemble */
    int32_t fused_block;          /* elements per CTA of the element-block path if selected, else 0 */
    int64_t fused_blocks;
    int64_t fused_partial;        /* element-block path: contributions of nonzeros split across blocks */
    int32_t pipeline_chunks;      /* element chunks of the work order (the persistent queue's chunks) */
    int32_t fused_sfc;            /* element-block path along the Morton order of the centroids (1) or not */
} ef_plan_info_t;
int ef_plan_info(const ef_plan* plan, ef_plan_info_t* info);

/* Select how ef_assemble runs. block = 0: leave the element-block path
 * (back to the two-pass kernels or the queue selected before). block = 128
 * or 256: the element-block path, ONE kernel with one CTA per block of
 * `block` consecutive elements of the mesh's order: the CTA keeps its
 * elements' local matrices in shared memory and completes the nonzeros lying
 * wholly in the block; the contributions of nonzeros split across blocks go
 * to the plan's scratch, and the CTA that contributes last to such a nonzero
 * (an integer ticket per nonzero; nothing waits) sums it. Results are
 * identical bit for bit (every nonzero is summed in ascending element order);
 * only speed differs. Synchronises `stream` and allocates when building the
 * block schedule. Errors: EF_ERR_ARG, EF_ERR_OOM, EF_ERR_SIZE (a block's
 * schedule does not fit in shared memory). */
int ef_plan_set_block(ef_plan* plan, int block, void* stream);

/* The element-block path of ef_plan_set_block with the blocks taken along a
 * space-filling (Morton, Z-order) curve through the element centroids under
 * the coordinates d_nodes (n_nodes x dim, device), so that a block is a
 * compact piece of the mesh and fewer nonzeros are split across blocks. The
 * coordinates only choose the grouping: later ef_assemble calls may pass
 * any coordinates, and the values are those of ef_assemble_two_pass bit for
 * bit (each nonzero is still summed in ascending element id). block = 0
 * leaves the element-block path. Synchronises `stream`; allocates.
 * Errors as ef_plan_set_block. */
int ef_plan_set_fused(ef_plan* plan, const double* d_nodes, int block, void* stream);

/* Select the one-launch persistent queue with `chunks` element chunks (1 to
 * 16; sums of a chunk may start once the chunks they depend on are done).
 * Results do not depend on it. Synchronises `stream`; reallocates the plan's
 * work-order arrays. */
int ef_plan_set_pipeline(ef_plan* plan, int chunks, void* stream);

/* Fault injection for tests of the bounded waits (the paper has no such
 * step). With on != 0, the next calls of ef_assemble on the one-launch queue
 * selected by ef_plan_set_pipeline wait for an element tile that never
 * completes: each waiting sum tile gives up after at most about one second
 * of wall time (a CTA stops waiting as soon as another has given up), skips
 * its sums, and ef_plan_check returns EF_ERR_TIMEOUT. The GPU stays usable;
 * K and M of such a call are incomplete. on = 0 restores the schedule, as
 * does any later ef_plan_set_pipeline or ef_plan_tune. Synchronises
 * `stream`. Errors: EF_ERR_ARG if the plan has no queue schedule, or (on !=
 * 0) if another schedule is selected. */
int ef_plan_inject_stall(ef_plan* plan, int on, void* stream);

/* Autotuner for ef_assemble on this plan: times at least `reps` calls of each
 * candidate (and enough calls for about 2 ms) on the given buffers and keeps
 * the fastest: the plain two-pass
 * kernels (*chosen = 0); the one-launch persistent queue with 4, 8 or 16
 * element chunks, 128 or 256 elements per tile, 1024 or 4096 nonzeros per
 * sum tile and 0, 1 or 2 element-only CTAs per four (*chosen = chunks*100 +
 * elem_ctas*10 + (tile == 256)); the element-block path in mesh order
 * (*chosen = -block) and along the Morton curve of the centroids under
 * d_nodes (*chosen = -(block + 1)).
 * A candidate whose schedule cannot be built (EF_ERR_OOM, EF_ERR_SIZE) is
 * skipped. Overwrites d_Kval / d_Mval. Synchronises `stream`. */
int ef_plan_tune(ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval, double* d_Mval,
                 int reps, int* chosen, void* stream);

/* Device time per kernel of ef_assemble. ef_plan_profile(plan, n) creates
 * 3n CUDA events and records them, on each call's stream, around the kernels
 * of the next n ef_assemble calls on this plan: before the first kernel,
 * between the first and the second, after the last (n = 0 stops recording
 * and frees the events). ef_plan_profile_read waits for the recorded events
 * and returns the summed milliseconds of the first kernel (the element kernel
 * of the two-pass schedule, the fused kernel of the element-block one, the
 * whole launch of the persistent queue or of the element-block kernel) and of
 * the second (the sum, or 0), and the number of calls recorded. Either output may be NULL.
 * Errors: EF_ERR_ARG, EF_ERR_CUDA. */
int ef_plan_profile(ef_plan* plan, int max_calls);
int ef_plan_profile_read(const ef_plan* plan, double* ms_first, double* ms_second, int* calls);

/* Copy the CSR pattern into caller buffers: d_rowptr [n_dofs+1] int64,
 * d_colidx [nnz] int32 (device). Asynchronous on `stream`. */
int ef_plan_pattern(const ef_plan* plan, int64_t* d_rowptr, int32_t* d_colidx, void* stream);

/* Copy the topology into caller buffers (any pointer may be NULL to skip):
 * d_elem2dof [n_elems x nloc] int32 (elems2edges / elems2faces of Sec. 3),
 * d_signbits [n_elems] uint8 (bit k set iff local DOF k has sign -1),
 * d_dof2nodes [n_dofs x 2] (edges) or [n_dofs x 3] (faces) int32, ascending
 * node ids (edges2nodes / faces2nodes). Asynchronous on `stream`. */
int ef_plan_topology(const ef_plan* plan, int32_t* d_elem2dof, uint8_t* d_signbits, int32_t* d_dof2nodes,
                     void* stream);

/*
 * Assemble K and M values into caller-owned CSR value arrays (pattern of
 * ef_plan_pattern): local matrices by the closed forms of the Sec. 2.4
 * integrals on every element, then the fixed-order sum into each nonzero.
 * By default two kernels (those of ef_assemble_two_pass); ef_plan_tune,
 * ef_plan_set_pipeline and ef_plan_set_block select another schedule (one
 * persistent launch, or the element-block kernels) with the same values.
 *   d_nodes: n_nodes x dim doubles; d_coeff: n_elems doubles or NULL (= 1);
 *   d_Kval, d_Mval: nnz doubles each (overwritten).
 * Asynchronous; allocates nothing; no host synchronisation (capturable in a
 * CUDA graph). A degenerate element (det B_K = 0) is reported by the next
 * ef_plan_check, not by this call; its contributions are then non-finite.
 * Calls on one plan that overlap on the GPU race on the plan's scratch.
 */
int ef_assemble(const ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval, double* d_Mval,
                void* stream);

/* Assembly with separate element coefficients for the two matrices: K_K
 * weighted by d_coeff_K[e] and M_K by d_coeff_M[e] (n_elems doubles each, or
 * NULL = 1), e.g. 1/mu and kappa of the eddy-current problem (Sec. 4.2,
 * curl 1/mu curl E + kappa E). Runs the two-pass kernels of
 * ef_assemble_two_pass whatever schedule the plan has selected; with equal
 * coefficient arrays the values are those of ef_assemble bit for bit.
 * Asynchronous; allocates nothing; capturable. */
int ef_assemble2(const ef_plan* plan, const double* d_nodes, const double* d_coeff_K, const double* d_coeff_M,
                 double* d_Kval, double* d_Mval, void* stream);

/* Same sums as ef_assemble, in two separate kernels: an element kernel writes
 * every local matrix to plan scratch, then one thread per upper nonzero sums
 * its contributions. Same values bit for bit (same summation order). */
int ef_assemble_two_pass(const ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval,
                         double* d_Mval, void* stream);

/*
 * End-to-end form for host data: copies h_nodes (n_nodes x dim) and h_coeff
 * (n_elems, or NULL) to plan-owned device staging buffers, assembles, and
 * copies K and M values back into h_Kval / h_Mval (nnz doubles each). Host
 * buffers should be pinned for asynchronous copies. When the plan's work
 * order has several element chunks (the default from 65,536 elements on),
 * the two-pass kernels run chunk by chunk and the CSR rows that a chunk
 * leaves final are copied back on a plan-owned stream while the next chunks
 * compute; values are the same bits as ef_assemble's. Synchronises `stream`
 * before returning and reports degenerate elements (EF_ERR_DEGENERATE).
 * The first call allocates the staging buffers, the copy stream and events.
 */
int ef_assemble_host(ef_plan* plan, const double* h_nodes, const double* h_coeff, double* h_Kval, double* h_Mval,
                     void* stream);

/*
 * ef_assemble_noalloc -- the paper has no counterpart to this call; it is
 * for callers that must not allocate device memory while they assemble:
 * code running while a CUDA stream capture is open in global mode (any
 * cudaMalloc in the process would break that capture), loops with a latency
 * budget that cannot absorb the device-wide synchronisation a cudaMalloc or
 * cudaFree may cause, and applications whose device memory belongs to
 * another allocator with a fixed budget.
 *
 * Same result as ef_assemble_two_pass (the same sums in the same order, so
 * the same bits), computed by two kernels with the element matrices kept in
 * one library-wide static device array of EF_NOALLOC_SCRATCH_BYTES instead
 * of the plan's own scratch. No cudaMalloc, cudaFree or other allocating
 * routine is called. The array exists on every GPU that loads the library
 * and stays there until the process exits.
 *   Limit: n_elems * nloc (nloc+1)/2 * 16 bytes must fit in the array
 *   (3D Nedelec: 199,728 elements; 3D RT0: 419,430; 2D: 699,050); larger
 *   plans get EF_ERR_SIZE (ef_last_error names the bytes needed) and nothing
 *   is launched.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and keeps it for the
 *   life of the process; make that first call before any stream capture.
 *   The kept address belongs to the device's primary context: after
 *   cudaDeviceReset (or any other teardown of that context) this entry point
 *   must not be called again in the process.
 *   Every call uses the same array and leaves its contents there; nothing in
 *   it has to start at zero, because each call overwrites every entry it
 *   reads. Calls whose work overlaps on the GPU (on different streams, or on
 *   plans of different threads) race on the array.
 * Asynchronous on `stream`. Other errors: EF_ERR_ARG, EF_ERR_CUDA.
 */
#define EF_NOALLOC_SCRATCH_BYTES (64ull << 20)
int ef_assemble_noalloc(const ef_plan* plan, const double* d_nodes, const double* d_coeff, double* d_Kval,
                        double* d_Mval, void* stream);

/* Synchronise `stream`, then read and clear the plan's device status word:
 * EF_ERR_DEGENERATE if an element with det B_K = 0 was met since the last
 * check, EF_ERR_TIMEOUT if a bounded wait gave up, else EF_OK. */
int ef_plan_check(ef_plan* plan, void* stream);

/* Free the plan (device memory included). Synchronises the device. NULL is a no-op. */
void ef_plan_destroy(ef_plan* plan);

/*
 * Adjoint of the quadratic form
 *   J(x, sigma) = u^T K(x, sigma) u + v^T M(x, sigma) v
 *              = sum_K sigma_K (u_K^T Khat_K u_K + v_K^T Mhat_K v_K),
 * u_K = u[elem2dof(K,:)], Khat_K / Mhat_K the signed unit-coefficient local
 * matrices (Sec. 2.4). Writes d_J (1 double), d_grad_nodes (n_nodes x dim,
 * dJ/dx) and d_grad_coeff (n_elems, dJ/dsigma); any output may be NULL to
 * skip it. Element geometry is recomputed, nothing is stored per element.
 * Nedelec 3D only (other kinds return EF_ERR_ARG). d_u, d_v: n_dofs doubles.
 * Asynchronous; no allocation; fixed summation order.
 */
int ef_adjoint(const ef_plan* plan, const double* d_nodes, const double* d_coeff, const double* d_u,
               const double* d_v, double* d_J, double* d_grad_nodes, double* d_grad_coeff, void* stream);

/* ---- vectorised integration (Sec. 3.1, norm_L2) ------------------------------ */

/* Quadrature: collapsed Gauss-Legendre product rule with n points per
 * direction (1 <= n <= EF_QUAD_MAX_N): n^2 points on the triangle, n^3 on the
 * tetrahedron, exact for polynomials of total degree 2n - dim. Triangle:
 * xhat = (u, v(1-u)), weight w_u w_v (1-u); tetrahedron: xhat = (u, v(1-u),
 * s(1-u)(1-v)), weight w_u w_v w_s (1-u)^2 (1-v), with (u, v, s) Gauss-Legendre
 * nodes on [0, 1]; point q = (i n + j) n + k (3D), i n + j (2D). Weights sum
 * to the reference measure (1/2, 1/6). */
#define EF_QUAD_MAX_N 8

/* The reference rule into host arrays h_xhat [nq x dim], h_w [nq] (cap
 * entries; both may be NULL to query *nq). Host only, no GPU needed.
 * Errors: EF_ERR_ARG (dim, n), EF_ERR_SIZE (cap < nq). */
int ef_quad_rule(int dim, int n, double* h_xhat, double* h_w, int cap, int* nq);

/* Physical quadrature points x = B_K xhat_q + P_K,0 of every element:
 * d_x [nq][n_elems][dim] (point-major: for each point, all elements
 * contiguous). Asynchronous. */
int ef_quad_points(const ef_plan* plan, const double* d_nodes, int n, double* d_x, void* stream);

/* Values at the same points of the finite-element function with DOF vector
 * d_v [n_dofs]: v_h = sum_k s_k v[dof_k] phi_k, phi_k the Piola-mapped
 * reference basis (RT0: B eta_k / det B = (x - P_opp(k)) / det B; Nedelec:
 * B^-T eta_k, the Whitney form of edge k), s_k the orientation signs of
 * ef_plan_topology. d_vals [nq][n_elems][dim]. Asynchronous. */
int ef_fe_values(const ef_plan* plan, const double* d_nodes, const double* d_v, int n, double* d_vals,
                 void* stream);

/* Squared L2 norm of f - v_h (v_h omitted if d_v is NULL), f given by its
 * values at the points of ef_quad_points: d_f [nq][n_elems][ncomp] (ncomp 1
 * to 3; with d_v, ncomp = dim). Per element (d_elem [n_elems], may be NULL)
 * |det B_K| sum_q w_q |f_q - v_h(x_q)|^2; total (d_total [1], may be NULL)
 * summed in a fixed order. The first call allocates per-CTA scratch in the
 * plan. Asynchronous. Errors: EF_ERR_ARG, EF_ERR_OOM. */
int ef_norm_l2(ef_plan* plan, const double* d_nodes, int n, int ncomp, const double* d_f, const double* d_v,
               double* d_elem, double* d_total, void* stream);

/* Squared L2 norm of g - D v_h, D v_h the per-element curl (Nedelec) or
 * divergence (RT0) of the FE function of d_v (omitted if d_v is NULL), as in
 * ||div y + f|| of the majorant (Sec. 4.1) or the curl part of the H(curl)
 * energy error (Sec. 4.2); g given at the points of ef_quad_points: d_g
 * [nq][n_elems][nc], nc = 3 for 3D Nedelec, 1 otherwise. Per element
 * (d_elem, may be NULL) and total (d_total, may be NULL; fixed order), as
 * ef_norm_l2, whose scratch it shares. Errors: EF_ERR_ARG, EF_ERR_OOM. */
int ef_norm_l2_derivative(ef_plan* plan, const double* d_nodes, int n, const double* d_g, const double* d_v,
                          double* d_elem, double* d_total, void* stream);

/* Per-element curl (Nedelec) or divergence (RT0) of the FE function with DOF
 * vector d_v, constant on each element: d_out [n_elems] (2D Nedelec, RT0) or
 * [n_elems x 3] (3D Nedelec). Asynchronous. */
int ef_fe_curl(const ef_plan* plan, const double* d_nodes, const double* d_v, double* d_out, void* stream);

/* Load vector b_i = int_Omega F . eta_i by the rule with n points per
 * direction, F given at the points of ef_quad_points: d_F [nq][n_elems][dim];
 * d_b [n_dofs]. Each b_i is the sum of its elements' contributions in
 * ascending element order (bitwise reproducible). The first call builds a
 * DOF-to-element incidence and scratch in the plan (allocates,
 * synchronises `stream`). Asynchronous afterwards. */
int ef_load_vector(ef_plan* plan, const double* d_nodes, int n, const double* d_F, double* d_b, void* stream);

/* Derivative load vector b_i = int_Omega g . D eta_i with D = div (RT0) or
 * curl (Nedelec), as in the right-hand sides of the majorant minimisation
 * (Sec. 4.1, int f div phi) and of curl-type sources; D eta_i is constant on
 * an element (the values of ef_fe_curl's basis), so each element contributes
 * s_i (|det B_K| sum_q w_q g(x_q)) . D phi_i. g given at the points of
 * ef_quad_points: d_g [nq][n_elems][nc], nc = 3 for 3D Nedelec, 1 otherwise.
 * Summed per DOF in ascending element order (bitwise reproducible), with the
 * incidence and scratch of ef_load_vector (built on first use of either).
 * Errors: EF_ERR_ARG, EF_ERR_OOM. */
int ef_load_derivative(ef_plan* plan, const double* d_nodes, int n, const double* d_g, double* d_b, void* stream);

/* ---- batched assembly of many meshes ---------------------------------------- */

/*
 * A batch holds independent meshes of one kind and dimension, each with its
 * own plan and its own CSR. ef_batch_assemble (buffers passed per call) and
 * ef_batch_assemble_bound (buffers bound once) assemble all of them either in
 * ONE persistent kernel launch over (mesh, element tile) and (mesh, sum tile)
 * work, where a sum tile starts once the element tiles it depends on are done
 * (a bounded wait; EF_ERR_TIMEOUT from ef_batch_check if a wait gave up), or
 * in two launches over all meshes (element kernel, then sum kernel), as the
 * configuration says. Values are those of ef_assemble on each mesh, bit for
 * bit.
 */
typedef struct ef_batch ef_batch;

/* Schedule of the persistent launch (chosen by ef_batch_tune). */
typedef struct {
    int32_t elems_per_tile;  /* elements per element tile = threads per CTA: 128 or 256 */
    int32_t sum_tile;        /* upper nonzeros per sum tile */
    int32_t ctas_per_sm;     /* persistent grid = ctas_per_sm x number of SMs (0 in ef_batch_set_config:
                                as many as fit) */
    int32_t dynamic;         /* 1: tiles by an integer ticket; 0: static stride blockIdx + k gridDim */
    int32_t largest_first;   /* 1: meshes in order of decreasing size; 0: as given */
    int32_t elem_ctas;       /* 0: every CTA takes tiles of both kinds from one interleaved queue;
                                k in 1..3: in each group of 4 CTAs, k take only element tiles and
                                4-k only sum tiles (two queues) */
    int32_t two_launch;      /* 1: instead of the persistent launch, two launches over all meshes:
                                the element kernel, then the sum kernel (the other fields unused) */
} ef_batch_config_t;

/* Build the per-mesh plans (as ef_plan_create for each). n_nodes, n_elems:
 * host arrays [n_meshes]; d_elems: host array of n_meshes device pointers.
 * Synchronises `stream`. Errors as ef_plan_create. */
int ef_batch_create(int kind, int dim, int n_meshes, const int64_t* n_nodes, const int64_t* n_elems,
                    const int32_t* const* d_elems, void* stream, ef_batch** out);
/* Per-mesh sizes into host arrays [n_meshes] (either may be NULL). */
int ef_batch_sizes(const ef_batch* batch, int64_t* n_dofs, int64_t* nnz);
/* CSR pattern of one mesh (as ef_plan_pattern). */
int ef_batch_pattern(const ef_batch* batch, int mesh, int64_t* d_rowptr, int32_t* d_colidx, void* stream);
/* Bind the per-mesh device buffers used by ef_batch_assemble_bound and the
 * tuner: host arrays
 * [n_meshes] of device pointers to nodes (n_nodes x dim), coefficients
 * (n_elems, or a NULL array / NULL entries for 1) and K, M values (nnz).
 * Copies the pointer tables to the device and synchronises `stream`. */
int ef_batch_bind(ef_batch* batch, const double* const* d_nodes, const double* const* d_coeff, double* const* d_K,
                  double* const* d_M, void* stream);
/* Assemble every mesh into its bound buffers: one persistent launch, or two
 * launches with two_launch set. Asynchronous, no allocation, no host
 * synchronisation; capturable in a CUDA graph. Calls that overlap on the GPU
 * race. EF_ERR_ARG if nothing is bound. */
int ef_batch_assemble_bound(const ef_batch* batch, void* stream);
/* Autotuner: times each candidate schedule `reps` times on the bound buffers
 * (the two-launch form; the persistent launch with 128/256 elements per tile,
 * 512/2048 nonzeros per sum tile, 0-2 element-only CTAs per four, dynamic or
 * static tickets, given or largest-first mesh order) and keeps the fastest;
 * writes it to *best (may be NULL). Overwrites the bound K, M. */
int ef_batch_tune(ef_batch* batch, int reps, ef_batch_config_t* best, void* stream);
int ef_batch_get_config(const ef_batch* batch, ef_batch_config_t* cfg);
int ef_batch_set_config(ef_batch* batch, const ef_batch_config_t* cfg, void* stream);
/* Synchronise `stream`; EF_ERR_DEGENERATE / EF_ERR_TIMEOUT if met since the last check. */
int ef_batch_check(ef_batch* batch, void* stream);
void ef_batch_destroy(ef_batch* batch);

/*
 * The batched calls with the buffers passed per call (the batch plan is the
 * same object as ef_batch; every ef_batch_* call above accepts it):
 *   ef_batch_plan_create: as ef_batch_create (per-mesh plans: the topology
 *     and CSR pattern of Sec. 3 for each mesh). Synchronises `stream`.
 *   ef_batch_assemble: assembles every mesh m into d_Kval[m], d_Mval[m]
 *     (nnz_m doubles each) from d_nodes[m] (n_nodes_m x dim) and d_coeff[m]
 *     (n_elems_m, or NULL; d_coeff itself may be NULL for all ones). The four
 *     arguments are HOST arrays [n_meshes] of device pointers; they are read
 *     during the call and need not outlive it. The call writes them into the
 *     plan's device descriptors by kernels on `stream` (one per 64 meshes),
 *     then runs the schedule the plan has selected (ef_batch_set_config /
 *     ef_batch_tune): same values as ef_plan-wise ef_assemble, bit for bit.
 *     Asynchronous; no allocation, no host synchronisation, no host-to-device
 *     copy: capturable in a CUDA graph, a replay reusing the pointers given
 *     at capture. Calls that overlap on the GPU race on the descriptors.
 *     Errors: EF_ERR_ARG (NULL table, or NULL entry for a non-empty mesh).
 *   ef_batch_plan_destroy: as ef_batch_destroy.
 */
typedef struct ef_batch ef_batch_plan;
int ef_batch_plan_create(int kind, int dim, int n_meshes, const int64_t* n_nodes, const int64_t* n_elems,
                         const int32_t* const* d_elems, void* stream, ef_batch_plan** out);
int ef_batch_assemble(const ef_batch_plan* batch, const double* const* d_nodes, const double* const* d_coeff,
                      double* const* d_Kval, double* const* d_Mval, void* stream);
void ef_batch_plan_destroy(ef_batch_plan* batch);

/* ---- one-shot convenience calls ------------------------------------------ */

typedef struct {
    int64_t n_dofs;
    int64_t nnz;
    int64_t* d_rowptr; /* n_dofs + 1, device, library-allocated */
    int32_t* d_colidx; /* nnz, device */
    double* d_K;       /* nnz, device */
    double* d_M;       /* nnz, device */
} ef_csr;

/* Plan + assemble + check in one call for RT0 (rt0_) or Nedelec (ned_)
 * elements; dim 2 or 3. The CSR arrays in *out are allocated by the library
 * and released with ef_csr_free. Synchronises `stream`. Errors as
 * ef_plan_create, plus EF_ERR_DEGENERATE. */
int rt0_assemble(int dim, const double* d_nodes, int64_t n_nodes, const int32_t* d_elems, int64_t n_elems,
                 const double* d_coeff, ef_csr* out, void* stream);
int ned_assemble(int dim, const double* d_nodes, int64_t n_nodes, const int32_t* d_elems, int64_t n_elems,
                 const double* d_coeff, ef_csr* out, void* stream);
void ef_csr_free(ef_csr* csr);

/* ---- measurement -------------------------------------------------------------- */

/*
 * ef_fp64_probe -- not part of the paper's method: measures the throughput of
 * this GPU's FP64 pipe, the bound of the element kernels (their work is a
 * stream of FP64 additions, multiplications and fused multiply-adds, see
 * Sec. 2.4's local matrices). op = 0: DFMA, 1: DADD, 2: DMUL, 3: the
 * integer-pipe multiply of the element kernels (bit for bit DMUL), 4: DFMA in
 * half of the chains and the integer-pipe multiply in the other half (both
 * pipes at once), 5: DFMA with literal constant operands, 6: an addition as a
 * DFMA with 1.0 in a per-thread register (bit for bit DADD). The operands
 * other than the chain value are per-thread registers except in op 5; on
 * GB300 only DFMA with all-register operands runs at the pipe's full rate.
 * Every thread
 * of a grid of 4 CTAs of 256 threads per SM runs 8 independent chains of
 * `iters` operations (rounded up to a multiple of 8); *ops_per_s receives the lane operations per second
 * (one per DFMA), *ms (may be NULL) the timed launch's duration. d_sink: one
 * device double the kernel may write (it never does for these inputs).
 * Launches a short warm-up and the timed kernel on `stream`, synchronises it.
 * Errors: EF_ERR_ARG, EF_ERR_CUDA.
 */
int ef_fp64_probe(int op, int64_t iters, double* d_sink, double* ops_per_s, double* ms, void* stream);

/*
 * ef_int_mul_check -- not part of the paper's method: checks the integer-pipe
 * FP64 multiply that the element and adjoint kernels use for their products
 * against the FP64 multiply instruction. Generates n operand pairs from
 * SplitMix64(seed, index) (random significands and signs; exponents over the
 * whole range, near the bias, and significands with many trailing zeros;
 * special values: zero, subnormals, infinity, NaN, the extreme normals),
 * multiplies each both ways and counts into the caller's device buffer
 * d_counts[2] (unsigned 64-bit): [0] pairs the integer form hands back to the
 * FP64 instruction (an operand or the product outside the normal numbers and
 * zero), [1] the other pairs whose bits differ (0 when correct). Clears
 * d_counts and launches on `stream`; does not synchronise. Errors: EF_ERR_ARG
 * (n < 0, NULL d_counts), EF_ERR_CUDA.
 */
int ef_int_mul_check(int64_t n, uint64_t seed, unsigned long long* d_counts, void* stream);

/* ---- diagnostics ------------------------------------------------------------ */

/* Static text for a status code. */
const char* ef_status_string(int status);
/* Text of the last CUDA error seen by this thread inside the library ("" if none). */
const char* ef_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EDGEFEM_H */
