/* hdg.h - C ABI of the GB300 HDG static-condensation library (libhdg.so).
 *
 * The library implements the data-parallel hot path of the hybridized DG method of
 * Fernandez, Christophe, Terrana, Nguyen and Peraire, "Hybridized discontinuous Galerkin
 * methods for wave propagation" (arXiv 1807.00086), on affine triangles (d = 2) and
 * tetrahedra (d = 3), for first-order acoustics (1/(rho c^2)) p_t + div v = s,
 * rho v_t + grad p = 0, and for linear elastodynamics (Sec. 4.1) in the velocity /
 * symmetric-stress form C^{-1} sigma_t = eps(v), rho v_t = div sigma, flux
 * sigma_hat n = sigma n - s (v - v_hat), s = 2 rho c_s (Eq. eq:stab_matrix_lin):
 *
 *   Sec. 2.2 (Eqs. e:spaces1, e:spaces2)  discontinuous P_k fields, P_k face traces (HDG);
 *   Sec. 2.3 (Eqs. ch5appendx1:eq8-eq10)  the semi-discrete DAE, BDF steps and DIRK stages;
 *   Sec. 2.4 (Eq. LS)                      static condensation K = D - C A^{-1} B,
 *                                          r = g - C A^{-1} h, element-local recovery.
 *
 * Conventions (fixed here; every array below follows them):
 *   - element vertices are used in ascending global id; local face j is opposite local
 *     vertex j; a face is parametrised from its vertices in ascending global id;
 *   - faces are numbered 0..n_faces-1 in lexicographic order of their sorted vertex ids;
 *   - element fields: [n_elem][ncomp][Np] FP64, coefficients in the orthonormal Dubiner basis
 *     of the unit reference simplex (mass = |det J| I); acoustic components (p, v_1, .., v_d),
 *     ncomp = d + 1; elastic components (v_1, .., v_d, sigma_11, sigma_22, [sigma_33,
 *     sigma_23, sigma_13,] sigma_12), ncomp = d + d(d+1)/2;
 *   - face traces: [n_faces][Nf] FP64 in the orthonormal basis of the reference face
 *     (face mass = J_F I, J_F = edge length (d = 2) or twice the face area (d = 3));
 *     acoustic: p_hat, Nf = C(k+d-1, d-1); elastic: v_hat component-major, Nf = d C(k+d-1, d-1);
 *   - Np = C(k+d, d), n = ncomp Np, m = (d+1) Nf;
 *   - boundary faces carry Dirichlet data for the trace (elastic: clamped, v_hat = 0); only
 *     interior faces are unknowns.
 *
 * Memory: pointers named *_dev are device pointers owned by the caller, used on the
 * context's stream and borrowed for the duration of the call (the call returns after
 * the work is enqueued or, where stated, completed). Pointers named *_host are host
 * memory, borrowed for the call. The context owns every other buffer.
 *
 * Errors: every call returns an hdg_status; on failure hdg_last_error(ctx) gives a
 * message owned by ctx (valid until the next call on ctx). Nothing is printed, nothing
 * exits, and no kernel traps: device-side failures surface as status codes.
 */
#ifndef HDG_H
#define HDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_ctx hdg_ctx;

typedef enum {
  HDG_OK = 0,
  HDG_EINVAL = -1,   /* bad argument or mesh                                   */
  HDG_ENOMEM = -2,   /* device allocation failed                               */
  HDG_ECUDA = -3,    /* a CUDA runtime call failed                             */
  HDG_ENOCONV = -4,  /* Krylov solve hit maxit before rtol                     */
  HDG_ETIMEOUT = -5, /* reserved: no kernel of the library spins on a flag; every device  */
                     /* loop ends by its own iteration bound (maxit, max_sweeps)          */
  HDG_ESTATE = -6    /* call out of order (e.g. solve before condense)         */
} hdg_status;

typedef enum { HDG_BE = 1, HDG_BDF2 = 2, HDG_DIRK3 = 3 } hdg_scheme;
typedef enum { HDG_ACOUSTIC = 0, HDG_ELASTIC = 1, HDG_SVK = 2 } hdg_physics;
typedef enum { HDG_FP64 = 0, HDG_MIXED = 1, HDG_MIXED16 = 2 } hdg_precision;

typedef struct {
  int32_t dim;              /* 2 or 3                                                */
  int64_t n_vert, n_elem;
  const double* vert;       /* _host [n_vert][dim]                                   */
  const int32_t* elem_vert; /* _host [n_elem][dim+1], any vertex order               */
  const int32_t* elem_k;    /* _host [n_elem] per-element degree in 1..4, or NULL for */
                            /* the uniform degree k of hdg_setup. 3D elastic only:    */
                            /* v_h, sigma_h in P_{k_K}(K), the trace on a face in     */
                            /* P_{k_F}, k_F = max over the face's elements. Fields    */
                            /* and traces are then flat (sizes field_entries /        */
                            /* trace_entries of hdg_sizes): element K holds its       */
                            /* 9 N_p(k_K) coefficients [comp][mode] in element order, */
                            /* face F its 3 N_f(k_F) trace values [comp][mode] in     */
                            /* face order. Boundary faces are clamped (v_hat = 0)     */
} hdg_mesh;

typedef struct {
  hdg_physics phys;         /* HDG_ACOUSTIC (uses rho, c), HDG_ELASTIC (rho, lam, mu) or  */
                            /* HDG_SVK (rho, lam, mu: nonlinear elastodynamics below)   */
  const double* rho;        /* _host [n_elem] density, > 0                           */
  const double* c;          /* _host [n_elem] sound speed, > 0 (acoustic)            */
  const double* lam;        /* _host [n_elem] Lame lambda (elastic), d lam + 2 mu > 0 */
  const double* mu;         /* _host [n_elem] Lame mu (elastic), > 0                 */
} hdg_material;

typedef struct {
  hdg_precision prec;       /* HDG_FP64: everything FP64. HDG_MIXED: the Krylov       */
                            /* iterations apply an FP32 copy of S_K inside FP64        */
                            /* iterative refinement of the trace system.               */
                            /* HDG_MIXED16: as MIXED with an FP16 copy of S_K (one     */
                            /* FP32 scale per element) in the Krylov iterations; a     */
                            /* sweep that gains less than 10x switches the rest of     */
                            /* that solve to the FP32 copy. Acoustic, nrhs = 1; other  */
                            /* configurations run as HDG_MIXED                         */
  double rtol;              /* relative residual target of the trace solve (FP64)     */
  int32_t maxit;            /* Krylov iteration cap per solve (per sweep if MIXED)    */
  int32_t check_every;      /* host polls the device convergence flag this often      */
  double inner_rtol;        /* MIXED: relative residual target of each FP32 solve     */
  int32_t max_sweeps;       /* MIXED: refinement sweep cap                            */
  int32_t nrhs;             /* R independent right-hand sides (power of two, 1..256)  */
                            /* solved together: every field and trace array below     */
                            /* gains an innermost column index [..][R]; one read of    */
                            /* each S_K serves all R columns                           */
  int32_t use_graphs;       /* nrhs > 1: replay captured CUDA graphs of Krylov        */
                            /* iteration chunks (fewer host launches; small problems)  */
  int32_t guess_history;    /* hdg_step: number q of earlier stage solutions per column */
                            /* (0..8) whose span gives the initial guess of each trace */
                            /* solve: lam0 = sum c_i lam_i minimising |b - K lam0|     */
                            /* (K lam_i = b_i at convergence, so only the stored right- */
                            /* hand sides enter; damped normal equations, Sec. 2.4's   */
                            /* least-squares guess over earlier solutions); with R     */
                            /* columns each column has its own fit; hdg_reset_column  */
                            /* drops a column's pairs. 0: the polynomial extrapolation */
                            /* of the last traces (BDF only)                           */
  int32_t device_loops;     /* each trace solve (any nrhs) is one CUDA-graph launch whose */
                            /* Krylov iterations and refinement sweeps are WHILE loops   */
                            /* with conditions set on the device (no host polling; the   */
                            /* graphs are built at the first solve per buffer pair and   */
                            /* kept). 0: host-driven loops polled every check_every      */
                            /* iterations. Statistics (hdg_enable_stats) use the host-   */
                            /* driven loops, which time each apply with CUDA events      */
  int32_t trace_space;      /* Sec. 2.2, Eq. e:spaces2: HDG_TRACE_HDG (default) traces   */
                            /* discontinuous across face edges; HDG_TRACE_IEDG traces    */
                            /* continuous on the interior faces (unknowns: the degree-k  */
                            /* equispaced face nodes shared between interior faces;      */
                            /* boundary faces keep the L2-projected Dirichlet data);     */
                            /* HDG_TRACE_EDG continuous on all faces (nodes on the       */
                            /* boundary fixed; homogeneous Dirichlet data only). The     */
                            /* trace system is then R^T K R mu = R^T r, lam_F = V^{-1}   */
                            /* mu(nodes of F). Acoustic, uniform k, nrhs = 1,            */
                            /* device_loops = 1                                          */
  int32_t solver;           /* HDG_SOLVER_CG (default): preconditioned CG on sgn K (SPD).  */
                            /* HDG_SOLVER_GMRES: restarted GMRES(gmres_restart) with      */
                            /* iterated classical Gram-Schmidt (two passes) and right      */
                            /* Jacobi preconditioning, the paper's Krylov method (Sec.     */
                            /* 2.4); FP64, HDG traces, nrhs = 1, host-driven iterations    */
  int32_t gmres_restart;    /* Krylov basis size before a restart (2..64)                */
  double newton_tol;        /* HDG_SVK: a stage's Newton iteration stops when the largest */
                            /* increment (fields and traces) is <= newton_tol *         */
                            /* max(1, max |u|)                                          */
  int32_t newton_maxit;     /* HDG_SVK: Newton iteration cap per stage (HDG_ENOCONV)     */
  int32_t precond;          /* HDG_SOLVER_GMRES right preconditioner: HDG_PRECOND_JACOBI */
                            /* (default, the inverse diagonal) or HDG_PRECOND_BILU0: block */
                            /* ILU(0) of the assembled trace system (Sec. 2.4), one N_f x  */
                            /* N_f block per pair of faces sharing an element, rows in     */
                            /* face order; factored after every condensation, applied by   */
                            /* level-scheduled block substitutions (N_f <= 32)             */
} hdg_options;

enum { HDG_PRECOND_JACOBI = 0, HDG_PRECOND_BILU0 = 1 };

enum { HDG_SOLVER_CG = 0, HDG_SOLVER_GMRES = 1 };

enum { HDG_TRACE_HDG = 0, HDG_TRACE_IEDG = 1, HDG_TRACE_EDG = 2 };

typedef struct {
  int32_t dim, k, Np, Nf, n_local, n_trace_local;  /* n_local = n, n_trace_local = m */
  int64_t n_elem, n_faces, n_bnd_faces;
  int32_t nq_vol, nq_face;  /* projection quadrature points per element / face       */
  int64_t device_bytes;     /* device memory held by the context                     */
  int64_t field_entries;    /* entries of one field column: n_elem x n_local, or the */
                            /* sum of the elements' own sizes (per-element degrees)   */
  int64_t trace_entries;    /* entries of one trace column: n_faces x the trace DOFs */
                            /* of a face (N_f, or 3 N_f elastic); with per-element    */
                            /* degrees the sum of the faces' own sizes                */
  int64_t schur_entries;    /* stored S_K entries summed over the elements (m^2 each) */
  int64_t slot_entries;     /* element trace entries summed over the elements (m each) */
  int64_t trace_unknowns;   /* unknowns of the global trace system: interior trace      */
                            /* entries (HDG) or free shared face nodes (IEDG / EDG)     */
} hdg_sizes;

typedef struct {
  int32_t iterations;       /* Krylov iterations of the last solve (sum over sweeps)  */
  int32_t sweeps;           /* refinement sweeps (mixed precision), else 1            */
  double rel_residual;      /* final ||r|| / ||b|| of the trace system (FP64)         */
} hdg_solve_info;

/* Defaults: FP64, rtol 1e-13, maxit 2000, check_every 16, inner_rtol 1e-4, max_sweeps 20, nrhs 1,
 * use_graphs 0, guess_history 8, device_loops 1, trace_space HDG_TRACE_HDG, solver HDG_SOLVER_CG,
 * gmres_restart 40, newton_tol 1e-11, newton_maxit 25, precond HDG_PRECOND_JACOBI. */
void hdg_default_options(hdg_options* opt);

/* Sec. 2.1 mesh and skeleton + Sec. 2.2 spaces. Validates the mesh, builds the face
 * table and affine geometry on the host, uploads them and the reference tables of
 * degree k (1 <= k <= 4), and binds the context to `cuda_stream` (a cudaStream_t, may
 * be NULL for the legacy stream). tau > 0 is the stabilisation of the numerical flux
 * v_hat.n = v.n + tau (p - p_hat). Returns HDG_EINVAL for a degenerate element, a face
 * shared by more than two elements, or sizes out of range. */
hdg_status hdg_setup(const hdg_mesh* mesh, int32_t k, double tau, const hdg_material* mat,
                     const hdg_options* opt, void* cuda_stream, hdg_ctx** out);
void hdg_destroy(hdg_ctx* ctx);
const char* hdg_last_error(const hdg_ctx* ctx);
hdg_status hdg_get_sizes(const hdg_ctx* ctx, hdg_sizes* out);

/* Sec. 2.4, Eq. LS: forms, for the mass shift alpha > 0 (A_K = alpha M_K + df/du), the
 * factor of each A_K and the Schur block S_K = D_K - C_K A_K^{-1} B_K of every element,
 * and the Jacobi preconditioner of the trace system. Enqueued on the context stream. */
hdg_status hdg_condense(hdg_ctx* ctx, double alpha);

/* Copies S_K of the last hdg_condense into S_dev [n_elem][m][m] (row-major). */
hdg_status hdg_get_schur(hdg_ctx* ctx, double* S_dev);

/* Matrix-free trace apply (Sec. 2.4): y = K x = sum_K P_K^T S_K P_K x on interior faces.
 * x_dev, y_dev: [n_faces][Nf]; boundary entries of x are ignored (treated as zero) and
 * boundary entries of y are set to zero. */
hdg_status hdg_trace_apply(hdg_ctx* ctx, const double* x_dev, double* y_dev);

/* Condensed right-hand side (Eq. LS): r = -sum_K P_K^T C_K A_K^{-1} (F_K - B_K lamD_K)
 * on interior faces (zero on boundary faces). F_dev: element right-hand sides
 * [n_elem][n] of A_K u_K + B_K lam_K = F_K; lamD_dev: [n_faces][Nf] whose boundary
 * entries hold the Dirichlet trace (may be NULL for zero data); r_dev: [n_faces][Nf]. */
hdg_status hdg_condensed_rhs(hdg_ctx* ctx, const double* F_dev, const double* lamD_dev, double* r_dev);

/* Krylov solve of K lam = r on interior faces (preconditioned CG on -K, which is SPD).
 * r_dev, lam_dev: [n_faces][Nf]; lam_dev on entry is the initial guess (interior
 * entries), on exit the solution; its boundary entries are left unchanged. Completes
 * before returning; fills info (may be NULL). HDG_ENOCONV if maxit was reached.
 * IEDG / EDG contexts solve R^T K R mu = R^T r from mu = 0 and return lam = R mu on the
 * interior faces (the entry values of lam_dev are not used as a guess). */
hdg_status hdg_trace_solve(hdg_ctx* ctx, const double* r_dev, double* lam_dev, hdg_solve_info* info);

/* Local recovery: u_K = A_K^{-1} (F_K - B_K lam_K) for every element, lam_dev over all
 * faces (boundary entries = Dirichlet trace). F_dev, u_dev: [n_elem][n]. */
hdg_status hdg_recover(hdg_ctx* ctx, const double* F_dev, const double* lam_dev, double* u_dev);

/* Element-local post-processing of the acoustic pressure into P_{k+1} (the local,
 * superconvergent post-processing step of HDG methods, Sec. 1; the paper writes no formula
 * for this scheme, so this is the standard one with the method's own discrete gradient).
 * For every element K, p* in P_{k+1}(K) solves
 *   (grad p*, grad w)_K = (q_h, grad w)_K  for all w in P_{k+1}(K),  (p*, 1)_K = (p_h, 1)_K,
 * where q_h in [P_k(K)]^d is given by the local momentum equation,
 *   (q_h, r)_K = -(p_h, div r)_K + <p_hat_h, r.n>_dK  for all r in [P_k(K)]^d.
 * u_dev: fields [n_elem][n] (pressure block first); lam_dev: traces [n_faces][Nf] with the
 * Dirichlet values on boundary faces (as hdg_get_state returns them); pstar_dev:
 * [n_elem][Np(k+1)] coefficients of p* in the orthonormal degree-(k+1) basis (same
 * construction and mode order as the degree-k basis). All device memory, caller-owned,
 * stream-ordered on the context's stream. Acoustic contexts with nrhs = 1 only
 * (HDG_EINVAL otherwise). The first call builds and uploads small reference tables
 * (one allocation, then a stream synchronisation). */
hdg_status hdg_postprocess(hdg_ctx* ctx, const double* u_dev, const double* lam_dev, double* pstar_dev);

/* Host-only views of what hdg_setup builds on the host, for tests and tools: no context, no
 * CUDA call, all pointers host memory owned by the caller. HDG_EINVAL (nothing written
 * beyond what was already copied) for invalid arguments.
 * hdg_host_skeleton: the skeleton E_h and the affine geometry of a simplex mesh (Sec. 2.1),
 * vert [n_vert][dim] and elem [n_elem][dim+1] as in hdg_mesh. Outputs:
 *   n_faces                        number of faces (lexicographic order of sorted vertex ids)
 *   elem_face [n_elem][dim+1]      face of local face j (opposite the j-th vertex, ascending ids)
 *   face_slot [(dim+1) n_elem][2]  slots e*(dim+1)+j of each face, lower first, -1 if none
 *                                  (the first 2 n_faces entries are written)
 *   face_bnd  [(dim+1) n_elem]     boundary index or -1 (the first n_faces entries are written)
 *   geo       [n_elem][32]         |det J|, J^{-1} row-major (d xi_r / d x_j), face Jacobians,
 *                                  outward unit normals (face-major)
 * hdg_host_tables: reference tables of degree k (1..4) in dimension dim (2, 3), orthonormal
 * Dubiner bases phi (degree k), mu (faces, degree k), psi (degree k + 1); any pointer may be NULL:
 *   Dr [dim][Np][Np]        Dr[r][i][l] = int d_r phi_l phi_i
 *   Ff [dim+1][Np][Nf]      Ff[f][i][m] = int over reference face f of phi_i mu_m
 *   K1 [dim][dim][Np1][Np1] K1[r][s][i][l] = int d_r psi_i d_s psi_l
 *   E1 [dim][Np1][Np]       E1[r][i][l] = int d_r psi_i phi_l                              */
hdg_status hdg_host_skeleton(int32_t dim, int64_t n_vert, int64_t n_elem, const double* vert, const int32_t* elem,
                             int64_t* n_faces, int32_t* elem_face, int32_t* face_slot, int32_t* face_bnd,
                             double* geo);
hdg_status hdg_host_tables(int32_t dim, int32_t k, double* Dr, double* Ff, double* K1, double* E1);
/* hdg_host_trace_nodes: the continuous trace spaces of Sec. 2.2 on the mesh of
 * hdg_host_skeleton, all faces continuous (all_faces = 1: EDG) or the interior faces
 * (all_faces = 0: IEDG). The unknowns are the degree-k equispaced face nodes, shared between
 * faces; EDG fixes those on the boundary. Outputs:
 *   n_free                       number of free nodes
 *   face_node [(dim+1) n_elem][Nf] free node of each face node (the first n_faces * Nf entries
 *                                are written; -1 for a fixed node or a face outside the set),
 *                                face nodes in lexicographic order of their integer barycentric
 *                                weights on the face's vertices (ascending global ids)
 *   Vinv [Nf][Nf]                nodal values -> coefficients of the orthonormal face basis    */
hdg_status hdg_host_trace_nodes(int32_t dim, int64_t n_vert, int64_t n_elem, const double* vert, const int32_t* elem,
                                int32_t k, int32_t all_faces, int64_t* n_free, int32_t* face_node, double* Vinv);

/* Data of the time-dependent problem. Point sources in the pressure equation at
 * positions pos_host [nsrc][dim], source i with amplitude amp_host[i] and the Ricker
 * wavelet r(t - d_i), r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), delayed
 * by d_i = delay_host[i] (NULL: 0); each is attached to the lowest-id element containing
 * it and acts on right-hand-side column col_host[i] (NULL: column 0). nsrc = 0 removes
 * all sources. */
hdg_status hdg_set_sources(hdg_ctx* ctx, int32_t nsrc, const double* pos_host, const double* amp_host,
                           const int32_t* col_host, const double* delay_host, double f0, double t0);

/* A dedicated non-blocking CUDA stream (cudaStream_t) for one context, e.g. for several
 * contexts stepping concurrently from different threads; destroy it after the context. */
hdg_status hdg_stream_create(void** stream_out);
hdg_status hdg_stream_destroy(void* stream);

/* z = M^{-1} r with the right preconditioner of the GMRES trace solve (Jacobi or block
 * ILU(0), Sec. 2.4) for sgn K, on face vectors r_dev, z_dev [n_faces][Nf] (boundary entries
 * of r ignored, of z zero). Solver HDG_SOLVER_GMRES after hdg_condense; returns after the
 * work completes. */
hdg_status hdg_precond_apply(hdg_ctx* ctx, const double* r_dev, double* z_dev);

/* Rebinds the context to another caller-owned stream (cudaStream_t, may be NULL for the
 * legacy stream). The call first waits for all work enqueued on the previous stream; every
 * later call enqueues on the new one. The context's cached CUDA graphs do not depend on
 * the stream they are launched on and stay valid. The library never creates or destroys
 * the bound stream. HDG_ECUDA if the wait fails (the binding is then left unchanged). */
hdg_status hdg_set_stream(hdg_ctx* ctx, void* cuda_stream);

/* Zeroes column j of the fields, the previous level and the traces (a column restarted
 * from rest; used to recycle a finished request's slot). Enqueued on the stream. */
hdg_status hdg_reset_column(hdg_ctx* ctx, int32_t j);

/* Physical coordinates of the projection quadrature points: which = 0 volume
 * ([n_elem][nq_vol][dim]), which = 1 boundary faces in face order ([n_bnd][nq_face][dim]).
 * With per-element degrees (which = 0 only): element K has its own rule of (k_K + 2)^dim
 * points and the elements' points are concatenated in element order. */
hdg_status hdg_quadrature_points(hdg_ctx* ctx, int32_t which, double* xyz_host);

/* Element-wise L2 projection of point values vals_host [n_elem][nq_vol][ncomp] at the
 * volume quadrature points into u_dev [n_elem][n] (ncomp = d + 1 acoustic (p, v), d + d(d+1)/2
 * elastic (v, sigma)); with per-element degrees vals_host is [total points][ncomp] in the order
 * of hdg_quadrature_points and u_dev the flat field array. */
hdg_status hdg_project_volume(hdg_ctx* ctx, const double* vals_host, double* u_dev);

/* Dirichlet trace p_hat = g(x) cos(omega t + phase) on all boundary faces; vals_host
 * [n_bnd][nq_face] holds g at the boundary quadrature points (NULL: zero data). */
hdg_status hdg_set_dirichlet(hdg_ctx* ctx, const double* vals_host, double omega, double phase);

/* Time state (checkpoint/resume). hdg_set_state sets the fields u at time t (u_dev
 * [n_elem][n]), the previous level used by BDF2 (uprev_dev, same layout; NULL: equal
 * to u, i.e. a start from rest or a steady state) and the traces (lam_dev
 * [n_faces][Nf]; NULL: zero), which the next trace solve takes as its initial guess unless
 * the least-squares guess replaces it: its stored (right-hand side, solution) pairs satisfy
 * K lam_i = b_i for the current operator whatever the state, so they are kept (hdg_condense
 * and a new mass shift drop them).
 * hdg_get_state copies the current
 * fields, the previous level and the traces (lam_dev [n_faces][Nf], boundary entries =
 * Dirichlet values); any output pointer may be NULL. Both complete before returning. The
 * buffers of both calls may also be page-locked host memory (cudaHostAlloc /
 * cudaHostRegister): the copies then run host <-> device on the context stream. */
hdg_status hdg_set_state(hdg_ctx* ctx, const double* u_dev, const double* uprev_dev, const double* lam_dev,
                         double t);
hdg_status hdg_get_state(hdg_ctx* ctx, double* u_dev, double* uprev_dev, double* lam_dev, double* t);

/* Complete solver checkpoint for a bitwise resume: the time, the fields and the previous level,
 * the traces and their history, the stored stage solutions of the least-squares initial guess
 * (and its Gram matrices), the nodal unknowns of IEDG / EDG contexts, and the mass shift of the
 * last condensation. A context with the same mesh, degree, material and options that loads the
 * checkpoint (condensing first if its operators are for another alpha) continues exactly as the
 * saved one would (given the same sources and boundary data): the same steps give the same
 * bits. hdg_checkpoint_size gives the bytes of
 * host memory the caller provides; hdg_save_checkpoint writes them (completes before returning),
 * hdg_load_checkpoint reads them (HDG_EINVAL if the checkpoint was written by a context of
 * other sizes or options). */
hdg_status hdg_checkpoint_size(const hdg_ctx* ctx, int64_t* bytes);
hdg_status hdg_save_checkpoint(hdg_ctx* ctx, void* host_buf);
hdg_status hdg_load_checkpoint(hdg_ctx* ctx, const void* host_buf);

/* Advances nsteps implicit steps of size dt with BE or BDF2 (Eq. ch5appendx1:eq9b) or
 * Alexander's DIRK(3,3) in the stage form of Eq. ch5appendx1:eq10_1 with the update of
 * Eq. 10_2. Each step (stage) forms the element right-hand sides, the condensed
 * right-hand side, solves the trace system and recovers the fields; the operators are
 * re-condensed when alpha = a_s/(b_s dt) or 1/(gamma dt) changes. Completes before
 * returning; info (may be NULL) accumulates over the steps. */
hdg_status hdg_step(hdg_ctx* ctx, double dt, hdg_scheme scheme, int32_t nsteps, hdg_solve_info* info);

/* Allocation-free trace apply. The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc at the moment they need y = K x, for instance code
 * that must not stall the device with an allocation's implicit synchronisation inside a
 * latency-bound loop, code confined to memory it was handed at start-up, or plug-ins
 * that may not touch the process's allocator. It computes the same y = K x as
 * hdg_trace_apply, with every input and output owned by the caller and no context:
 *   S_dev          [n_elem][m][m]   element Schur blocks, row-major (e.g. copied by
 *                                   hdg_get_schur); y gathers S_K x_K, so S_K need not be
 *                                   symmetric
 *   elem_face_dev  [n_elem][dim+1]  face id of local face j, where the element's vertices are
 *                                   taken in ascending global id and local face j is the face
 *                                   opposite the j-th of them (faces numbered in the library's
 *                                   lexicographic order of sorted vertex ids; a face's trace
 *                                   modes are parametrised from its vertices in ascending
 *                                   global id, as hdg_setup does; tables built from unsorted
 *                                   connectivity give a wrong y without an error)
 *   face_slot_dev  [n_faces][2]     slots e*(dim+1)+j of the face's elements, lower element
 *                                   first, -1 for the missing side of a boundary face
 *   face_bnd_dev   [n_faces]        >= 0 on boundary faces, -1 on interior faces
 *   x_dev, y_dev   [n_faces][Nf]    as in hdg_trace_apply (boundary entries of y set to 0)
 * all device memory, used on cuda_stream. The only scratch, n_elem * m doubles of
 * per-element products, lives in one fixed 8 MiB device array inside the library (held
 * by every GPU that loads it until the process exits), so n_elem * m may not exceed
 * 1,048,576 (26,214 tetrahedra at k = 3); larger sizes return HDG_EINVAL with a message
 * in err (err_len bytes, may be NULL). Each call looks up the array's device address with
 * the current device (no allocation); the first call on each device must come before any
 * stream capture (HDG_ESTATE otherwise). The call enqueues work and returns; it allocates
 * and frees nothing. Every call shares the one array and leaves its products there; each
 * call writes every entry it reads before reading it, so nothing has to be cleared, but
 * calls whose work overlaps on the GPU (e.g. on two streams at once) race on the array. */
hdg_status hdg_trace_apply_noalloc(int32_t dim, int32_t k, int64_t n_elem, int64_t n_faces, const double* S_dev,
                                   const int32_t* elem_face_dev, const int32_t* face_slot_dev,
                                   const int32_t* face_bnd_dev, const double* x_dev, double* y_dev,
                                   void* cuda_stream, char* err, int32_t err_len);

/* Tiles of the per-element-degree (elastic, elem_k) kernels, chosen by the library's
 * autotuner on the context's own data: at the first hdg_condense it times each candidate tile
 * of the matrix-free apply (warps per block in {4, 8} x columns in flight in {4, 8, 16}) on
 * the condensed operator: apply64 is the FP64-accurate apply (the FP64 kernel, or with mixed
 * precision the double-float refinement-residual kernel), apply32 the FP32 inner apply
 * (mixed precision). At the first local solve of
 * each kind it times the block size of the one-launch element-local solve (64, 128 or 256
 * threads per element). tuned = 0 before the first condensation; local_threads are 0 until
 * the first condensed right-hand side (index 0) / recovery (index 1). HDG_EINVAL for a
 * context without per-element degrees. */
typedef struct {
  int32_t tuned;
  int32_t apply32_warps, apply32_unroll;
  int32_t apply64_warps, apply64_unroll;
  int32_t local_threads[2];
} hdg_tuning;
hdg_status hdg_get_tuning(const hdg_ctx* ctx, hdg_tuning* out);

/* ---- Nonlinear elastodynamics (Sec. 4.4, Eqs. UNEL, eq:HDG_nelas1-5): HDG_SVK contexts.
 * Saint Venant-Kirchhoff material, P = F S(F), S = lam tr(E) I + 2 mu E, E = (F^T F - I) / 2,
 * in the velocity / deformation-gradient / stress form
 *   (alpha rho (v - h_v), w) + (P, grad w) - <P n - s (v - v_hat), w> = (f, w)
 *   (alpha (H - h_H), G) + (v, div G) - <v_hat, G n> = 0,   H = F - I
 *   (P, Q) - (F S(F), Q) = 0
 * with s = 2 sqrt(rho mu) per element and conservation of P n - s (v - v_hat) on the faces.
 * 3D tetrahedra, uniform k in 1..3, nrhs = 1, HDG traces, CG, FP64. Fields [n_elem][21][Np]:
 * v_1..3, H_iJ (row-major (i, J)), P_iJ; traces [n_faces][3 Nf] (v_hat, component-major).
 * Boundary faces are clamped (v_hat = 0) unless marked as traction faces. The volume rule of
 * hdg_quadrature_points / hdg_project_volume has (2k + 2)^3 points (nq_vol of hdg_get_sizes).
 * Every implicit stage is solved by Newton's method: each iteration forms, per element, the
 * residual and its Jacobian at quadrature points, condenses it (Eq. LS: H and P eliminated
 * through their diagonal mass blocks, then the velocity block by Cholesky), solves the trace
 * system (CG to rtol; 1e-10 is enough, Newton corrects the rest) and recovers the element
 * increments. hdg_step runs HDG_DIRK3 (the stages start Newton from the previous stage);
 * info->sweeps returns the Newton iterations, info->iterations the CG iterations.
 * hdg_condense / hdg_condensed_rhs / hdg_recover / hdg_postprocess / hdg_set_dirichlet with
 * data return HDG_EINVAL; HDG_EINVAL also when an element's velocity block is not positive
 * definite (the tangent lost ellipticity). */

/* Marks boundary faces as traction faces (mask_host [n_bnd] in the order of
 * hdg_quadrature_points(which = 1), 1 = traction; NULL clears): their traces become
 * unknowns, loaded by the traction data of the forcing callback. */
hdg_status hdg_svk_set_traction_faces(hdg_ctx* ctx, const uint8_t* mask_host);

/* Forcing of the stage equations, called by hdg_step on the host before each stage with the
 * stage time t: fill f_host [n_elem][nq_vol][3] with the body force f at the volume points and
 * g_host [n_bnd][nq_face][3] with the traction P n at the boundary-face points (only traction
 * faces are read). Both arrive zero-filled; return 0 on success (otherwise hdg_step fails with
 * HDG_EINVAL). NULL fn: no forcing. */
typedef int32_t (*hdg_svk_forcing)(void* user, double t, double* f_host, double* g_host);
hdg_status hdg_svk_set_forcing(hdg_ctx* ctx, hdg_svk_forcing fn, void* user);

/* Newton iterations of each stage of the last hdg_step (count = 3 x steps); writes at most
 * cap entries into out_host (may be NULL to query the count). */
hdg_status hdg_svk_newton_counts(const hdg_ctx* ctx, int32_t* out_host, int32_t cap, int32_t* count);

/* Instrumentation (not part of the method). When enabled, the context counts its kernel
 * launches and times every launch of the matrix-free trace apply with CUDA events on the
 * context stream; hdg_get_stats returns the totals since the last reset. */
typedef struct {
  int64_t kernel_launches;  /* all kernels launched by the context                     */
  int64_t apply_launches;   /* launches of the FP64 trace-apply kernel                 */
  double apply_ms;          /* summed device time of those launches (CUDA events)      */
  int64_t apply32_launches; /* launches of the FP32 (mixed precision) trace apply      */
  double apply32_ms;        /* summed device time of those launches                    */
  int64_t applydf_launches; /* launches of the double-float refinement-residual apply   */
  double applydf_ms;        /* summed device time of those launches                    */
  int64_t apply16_launches; /* launches of the FP16 apply (HDG_MIXED16 Krylov iterations) */
  double apply16_ms;        /* summed device time of those launches                    */
  /* Device-side timing of the single-column FP32 and FP16 applies, taken by the kernels
   * themselves from %globaltimer (first CTA start to the end of the last CTA) and therefore
   * also inside the CUDA graphs of the device-driven loops. It runs whether or not stats are
   * enabled; launches that return at once (solve already converged) are not counted. The
   * timer ticks at about 1 us on some parts, so use the mean over many launches. */
  int64_t dev_apply32_launches;
  double dev_apply32_ms;
  int64_t dev_apply16_launches;
  double dev_apply16_ms;
  int64_t svk_condense_launches; /* HDG_SVK: per-Newton-iteration condensation kernel   */
  double svk_condense_ms;        /* (CUDA events while stats are enabled)               */
  int64_t svk_recover_launches;  /* HDG_SVK: per-Newton-iteration recovery kernel       */
  double svk_recover_ms;
} hdg_stats;
hdg_status hdg_enable_stats(hdg_ctx* ctx, int32_t enable);
hdg_status hdg_get_stats(hdg_ctx* ctx, hdg_stats* out, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* HDG_H */
