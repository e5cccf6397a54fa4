/*
 * dd.h -- C ABI of the GB300 MFETI-DP1 Maxwell field-solve library (libdd.so).
 *
 * The library advances the implicit Newmark-beta (gamma = 1/2, beta = 1/4)
 * time march of the Whitney edge-element wave equation on a tetrahedral mesh
 * (Sec. II-B, Eq. maxnmb, edge-only reading) and solves every time step with
 * the MFETI-DP1 domain decomposition (Sec. III-A: tearing into subdomains,
 * local eliminations Eq. rF1, interface system Eq. F1lr, corner system
 * Eq. F1uc, Schur-complement interface system Eq. f1schur) on one GPU.
 *
 * Per step, with A = T + (dt^2/4) S and B = 2T - (dt^2/2) S,
 *     A e^{n+1} = B e^n - A e^{n-1} - (g^{n+1} - 2 g^n + g^{n-1}),
 * where e are the interior (non-PEC) edge unknowns, T the mass and S the
 * curl-curl matrix, and g_i(t) = <W_i, G(t)> the tested integrated current
 * G = int_0^t J (Sec. II-A).
 *
 * Conventions for every entry point:
 *   - The return value is a status code (DD_OK = 0 or one of DD_ERR_*).  No
 *     C++ exception or abort crosses this boundary; dd_last_error() returns a
 *     readable message for the last failure on a handle.
 *   - "host" pointers are CPU memory, read during the call and not retained.
 *     "device" pointers are GPU global memory owned by the caller (for
 *     instance torch tensors); the library never frees them.
 *   - All device memory the library uses (matrices, maps, vectors) lives in
 *     one caller-allocated workspace bound with dd_bind_workspace().  The
 *     handle itself owns only host metadata.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered; a call that returns statistics to
 *     the host synchronises that stream.
 *   - Unknown numbering: mesh edges are the distinct node pairs (lo, hi),
 *     lo < hi, sorted lexicographically and oriented lo -> hi.  Edges lying in
 *     a boundary triangle are removed (PEC wall).  The remaining "dofs" keep
 *     the global edge order.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define DD_OK 0
#define DD_ERR_ARG 1             /* bad argument (NULL, size, range)               */
#define DD_ERR_MESH 2            /* degenerate or inverted tetrahedron             */
#define DD_ERR_PARTITION 3       /* empty subdomain or subdomain without r dofs   */
#define DD_ERR_NOT_SPD 4         /* non-positive pivot while factoring            */
#define DD_ERR_NO_CONVERGENCE 5  /* interface CG did not reach tol in max_it      */
#define DD_ERR_NONFINITE 6       /* NaN/Inf in a residual                          */
#define DD_ERR_TIMEOUT 7         /* a bounded device wait expired                  */
#define DD_ERR_CUDA 8            /* a CUDA runtime call failed                     */
#define DD_ERR_STATE 9           /* call out of order (e.g. step before factor)   */

/* ---- precision modes ------------------------------------------------- */
#define DD_FP64 0   /* every per-step operation in FP64                                   */
#define DD_MIXED 1  /* FP32 local/interface/coarse application, FP64 residual refinement  */

/* Interface solvers (dd_params.solver). */
#define DD_SOLVER_SCHUR_CG 0       /* Eq. f1schur (symmetric positive definite) by Jacobi CG       */
#define DD_SOLVER_COUPLED_GMRES 1  /* Eqs. F1lr + F1uc together by restarted GMRES (Sec. III-A end,
                                      Sec. IV, Fig. fetiIter)                                      */
#define DD_MAX_RESTART 32          /* largest GMRES restart length                                */

/* Factorisation paths (dd_params.factor_mode). */
#define DD_FACTOR_FP64 0    /* trailing updates on the FP64 CUDA cores                      */
#define DD_FACTOR_TENSOR 1  /* trailing updates from BF16 slices on the tensor cores, FP64-accurate */

/* Domain-decomposition schemes (dd_params.scheme). */
#define DD_SCHEME_DP1 0  /* MFETI-DP1 (Sec. III-A): one multiplier per interface edge         */
#define DD_SCHEME_DP2 1  /* MFETI-DP2 (Sec. III-B), edge-only reading: Robin term alpha*M_T on
                            every local interface, one multiplier per interface edge and side */

typedef struct dd_handle dd_handle;

/* Tetrahedral mesh (host arrays, copied during dd_setup).
 * xyz  [n_nodes*3] node coordinates, x fastest.
 * tets [n_tets*4]  node ids of each tet; any vertex order (orientation is
 *                  taken from the sign of the volume, which must be non-zero).
 * eps  [n_tets]    relative permittivity per tet, or NULL for 1.
 * mu               relative permeability (uniform). */
typedef struct {
    int64_t n_nodes;
    int64_t n_tets;
    const double* xyz;
    const int32_t* tets;
    const double* eps;
    double mu;
} dd_mesh;

/* Solver parameters.
 * tol        relative residual of the interface solve: stop when
 *            ||r_k||_2 <= tol * ||rhs||_2 (CG: Eq. f1schur; GMRES: the
 *            coupled system, r = [d_r; f~_c] - M [lambda; x_c]).
 * max_it     iteration cap per solve (CG iterations / GMRES Arnoldi steps).
 * precond    0 = none, 1 = Jacobi (diagonal of F_rr; the paper's diagonal
 *            preconditioner of Sec. III-C; for the coupled GMRES the diagonal
 *            of the coupled matrix, diag(F_rr) and diag(K~cc)).
 * warm_start 1 = start each interface solve from the previous multipliers;
 *            2 = start the first solve of a step from the linear extrapolation
 *            2 lambda^{n-1} - lambda^{n-2} of the previous steps' multipliers
 *            (the coupled GMRES: of [lambda; x_c], DP2 [lambda^(1); lambda^(2);
 *            x_c]) once two steps of history exist; the adjoint march uses 1.
 * refine_tol DD_MIXED only: stop refining a step when the FP64 residual of the
 *            step's linear system satisfies ||r||_2 <= refine_tol * ||b||_2.
 * max_refine DD_MIXED only: cap on FP32 correction solves per step.
 * chunk      CG iterations issued between two convergence checks (host
 *            polls in eager mode; iterations per WHILE-body launch in graph mode).
 * use_graph  1 = dd_step runs as a CUDA graph captured once per time-level
 *            phase (rebuilt after dd_factor / dd_set_params): the CG loop is a
 *            conditional WHILE node whose condition the CG kernels set, and
 *            every further mixed-precision refinement pass is a conditional IF
 *            node, so a step needs no host round trip unless stats are
 *            requested.  The step's source is copied into the workspace before
 *            each launch.  0 = eager launches with host convergence polling.
 * solver     DD_SOLVER_SCHUR_CG (default) or DD_SOLVER_COUPLED_GMRES: the
 *            coupled equations F1lr and F1uc,
 *                [ F_rr     F_rc ] [lambda]   [d_r ]
 *                [ -F_rc^T  K~cc ] [x_c   ] = [f~_c],
 *            solved by GMRES(restart) with right preconditioning (the
 *            residual tested is the unpreconditioned one), classical
 *            Gram-Schmidt applied twice, Givens rotations; warm start from
 *            the previous solve's [lambda; x_c] (warm_start 2: extrapolated).
 *            DD_FP64 or DD_MIXED (FP32 Krylov vectors inside the FP64
 *            refinement).  K~cc^-1 is not used by this solver.
 * restart    GMRES restart length m, 1..DD_MAX_RESTART (the paper: 20).
 * scheme     DD_SCHEME_DP1 (default) or DD_SCHEME_DP2.  DP2 (Sec. III-B, read for
 *            the edge-only step system A = T + dt^2/4 S): every local matrix
 *            gets the Robin term R = robin_alpha * M_T on its interface edges
 *            (M_T: tangential Whitney mass of the interface faces, restricted
 *            to the multiplier edges); each interface edge carries one
 *            multiplier per side, (A^(s) + R^(s)) x^(s) = b^(s) + lambda^(s), with
 *            the transmission conditions lambda^(1) + lambda^(2) =
 *            2 alpha M_T x^(2) = 2 alpha M_T x^(1) (Eq. f2imp1); corners stay
 *            primal.  Solved as the coupled system for [lambda^(1); lambda^(2);
 *            x_c] by GMRES (DD_SOLVER_COUPLED_GMRES required, DD_ERR_ARG
 *            otherwise) with the diagonal preconditioner [1; 1; diag(K~cc)].
 *            The scheme and alpha are fixed by dd_factor: a step with another
 *            scheme than the factorisation returns DD_ERR_STATE.
 * robin_alpha DP2 Robin coefficient; <= 0 selects dt / 2 (the admittance of
 *            vacuum, eta = 1, times Newmark's dt/2).
 * sym_fp32   DD_MIXED: 1 = the FP32 GEMVs over symmetric blocks (local solve,
 *            interface rows, coupled operator) read the packed lower triangle
 *            of the symmetric matrix S = J M (the swept local matrix M is J
 *            times a symmetric matrix, J = diag(I_r, -I_c)) in FP32 tiles cut
 *            to the index groups' own sizes (no padding of the groups;
 *            diagonal tiles as triangles), about half of the dense bytes;
 *            0 = the dense FP32 copy.  Results differ by FP32 rounding only.
 * members    Ensemble size R, 1..64 (fixed by dd_setup; dd_set_params must keep
 *            it).  R > 1 marches R independent field problems on the same mesh,
 *            materials and dt at once (multi-RHS batching): member r is copy r
 *            of the mesh -- node ids offset by r * n_nodes, subdomain ids by
 *            r * n_sub -- so its dofs, multipliers and corners follow those of
 *            member r - 1, and every vector (source, fields, multipliers) holds
 *            the R members one after the other.  The factored local operators
 *            are computed and stored once and read by every member: the GEMVs
 *            visit the R copies of a subdomain together, so that one read from
 *            HBM serves them through L2.  The members' interface systems are
 *            solved as one block-diagonal system: one Krylov iteration serves
 *            all members and the stopping tests use the norms of the stacked
 *            vectors (members of very different magnitude are solved to the
 *            same absolute, not relative, accuracy).  R > 1 needs
 *            DD_SOLVER_COUPLED_GMRES (the Schur CG would need the dense inverse
 *            of the stacked coarse problem; DD_ERR_ARG otherwise); probes, the
 *            PIC cycle, the adjoint and dd_schur_apply return DD_ERR_STATE.
 * factor_mode DD_FACTOR_FP64 (0): the elimination's trailing updates (rank-32
 *            GEMMs, Sec. III-C's one inverse per subdomain) on the FP64 CUDA
 *            cores; DD_FACTOR_TENSOR (1, the default): the same updates on the tensor cores,
 *            FP64-accurate: every row of the column panel and every column of
 *            the row panel is scaled by a power of two and cut into seven 8-bit
 *            BF16 slices, the slice products of each weight class are summed
 *            exactly in FP32 tensor memory (tcgen05 MMAs) and the classes are
 *            combined in FP64 (an Ozaki splitting).  Results agree with the FP64
 *            path to FP64 rounding.  Read by dd_factor. */
typedef struct {
    int precision;
    double tol;
    int max_it;
    int precond;
    int warm_start;
    double refine_tol;
    int max_refine;
    int chunk;
    int use_graph;
    int solver;
    int restart;
    int sym_fp32;
    int scheme;
    double robin_alpha;
    int members;
    int factor_mode;
} dd_params;

/* Sizes of a set-up problem. */
typedef struct {
    int64_t n_edges;        /* mesh edges                                     */
    int64_t n_dof;          /* interior (non-PEC) edges = unknowns            */
    int32_t n_sub;          /* subdomains N_v                                 */
    int64_t n_lambda;       /* Lagrange multipliers (edges shared by 2 subdomains) */
    int64_t n_corner;       /* corner unknowns (edges shared by >= 3 subdomains)   */
    int64_t n_local;        /* sum over subdomains of local unknowns          */
    int64_t nnz_local;      /* nonzeros of the subassembled local matrices    */
    int32_t max_nr;         /* largest local r block                          */
    int32_t max_ns;         /* largest local system (r + c)                   */
    size_t workspace_bytes; /* bytes dd_bind_workspace needs                  */
    int64_t dense_bytes_fp64; /* bytes of the per-subdomain dense operators (stored once for all members) */
    int32_t members;        /* ensemble size R: n_dof, n_sub, n_lambda, ... count all members */
} dd_sizes;

/* Tearing maps, written to caller-allocated host arrays (any may be NULL).
 * Lengths follow dd_sizes.  Local order inside subdomain s is
 * [interior (m=1), interface r (m=2), corner (m>=3)], each sorted by dof id.
 *   edges      [n_edges*2] int64  (lo, hi) node ids
 *   dof_edge   [n_dof]     int64  mesh edge id of each dof
 *   sub_ptr    [n_sub+1]   int64  offsets of each subdomain in local_dof
 *   local_dof  [n_local]   int64  dof id of each local unknown
 *   n_int, n_gam, n_cor [n_sub] int32  sizes of the three local groups
 *   mult_dof   [n_lambda]  int64  dof of each multiplier (global edge order)
 *   mult_sub   [n_lambda*2] int32 (s1, s2), s1 < s2; B_r is +1 in s1, -1 in s2
 *   mult_loc   [n_lambda*2] int32 local index of the dof in s1 and in s2
 *   corner_dof [n_corner]  int64  dof of each corner (global edge order)
 *   owner      [n_dof]     int32  lowest subdomain containing the dof */
typedef struct {
    int64_t* edges;
    int64_t* dof_edge;
    int64_t* sub_ptr;
    int64_t* local_dof;
    int32_t* n_int;
    int32_t* n_gam;
    int32_t* n_cor;
    int64_t* mult_dof;
    int32_t* mult_sub;
    int32_t* mult_loc;
    int64_t* corner_dof;
    int32_t* owner;
} dd_maps;

/* Per-call statistics (host struct).  iters = interface CG iterations (GMRES:
 * Arnoldi steps) summed over the solves of the call; refinements = FP32
 * correction solves (DD_MIXED); resid = final relative residual (interface
 * solve for DD_FP64 -- for GMRES the Givens residual estimate --, step system
 * for DD_MIXED); status = DD_OK or the error the call returned. */
typedef struct {
    int iters;
    int refinements;
    double resid;
    int status;
} dd_stats;

/* Build the tearing (Sec. III-A) on the host: edges, PEC removal, element
 * matrices, multiplicities, local numbering, B_r / B_c, local CSR matrices.
 * part [n_tets] (host) gives the subdomain 0..n_sub-1 of every tet.
 * params may be NULL (defaults: FP64, tol 1e-12, max_it 500, Jacobi, warm
 * start, refine_tol 1e-12, max_refine 4, chunk 8, eager launches, tensor-core
 * trailing updates).  On success *out owns a new
 * handle (free with dd_destroy).  Errors: DD_ERR_ARG, DD_ERR_MESH,
 * DD_ERR_PARTITION.  No GPU work is done. */
int dd_setup(const dd_mesh* mesh, const int32_t* part, int32_t n_sub, const dd_params* params,
             dd_handle** out);

/* Change solver parameters of an existing handle (precision needs a
 * workspace large enough for it: the workspace is always sized for both). */
int dd_set_params(dd_handle* h, const dd_params* params);

int dd_get_sizes(const dd_handle* h, dd_sizes* out);
int dd_get_maps(const dd_handle* h, dd_maps* out);

/* Probe points (host [n_probe*3]); replaces any previous set.  A point is
 * located in the lowest-id tet whose barycentric coordinates are all
 * >= -1e-12.  Errors: DD_ERR_ARG if a point lies outside the mesh. */
int dd_set_probes(dd_handle* h, int32_t n_probe, const double* xyz);

/* Bind the caller-allocated device workspace (>= workspace_bytes, 256-byte
 * aligned) and upload the maps into it.  Synchronises `stream`.  The
 * workspace must stay allocated until dd_destroy. */
int dd_bind_workspace(dd_handle* h, void* dev_ptr, size_t bytes, void* stream);

/* Factor for time step dt (Sec. III-C: one inverse per subdomain kept in
 * memory): assemble the dense local A^(s) = T^(s) + dt^2/4 S^(s), eliminate
 * its r block in FP64 to obtain A_rr^-1, A_rr^-1 A_rc and the local corner
 * Schur complements, assemble and invert K~cc, build the Jacobi diagonal, and
 * (always) FP32 copies for DD_MIXED.  Resets the time level to n = 0 with
 * e^0 = e^{-1} = 0.  Synchronises `stream`.  Errors: DD_ERR_STATE (no
 * workspace), DD_ERR_NOT_SPD, DD_ERR_CUDA. */
int dd_factor(dd_handle* h, double dt, void* stream);

/* One time step: e^{n+1} from (e^n, e^{n-1}) and the source.
 * d2g  device [n_dof] second difference g^{n+1} - 2 g^n + g^{n-1} of the tested
 *      integrated current, or NULL for no source.
 * e_out device [n_dof] receives e^{n+1}, or NULL.
 * stats host, or NULL.  With stats == NULL and DD_FP64 the call only
 *      synchronises to poll CG convergence between chunks of iterations.
 * Errors: DD_ERR_STATE (not factored), DD_ERR_NO_CONVERGENCE (fields are
 * still advanced with the last iterate), DD_ERR_NONFINITE, DD_ERR_CUDA. */
int dd_step(dd_handle* h, const double* d2g, double* e_out, dd_stats* stats, void* stream);

/* dd_step with the source scaled on the device: d2g is taken as scale * d2g
 * (a fixed spatial pattern, e.g. the tested current of a line source, times a
 * time function's second difference), so that a caller marching a separable
 * source J(x, t) = p(x) I(t) passes the pattern once and a host scalar per
 * step.  scale must be finite (DD_ERR_ARG).  Otherwise as dd_step; with
 * scale = 1 the result is bitwise that of dd_step. */
int dd_step_scaled(dd_handle* h, const double* d2g, double scale, double* e_out, dd_stats* stats, void* stream);

/* ---- discrete adjoint (gradients of a probe objective) ----------------
 * Not in the paper; derived from the recurrence above.  For the objective
 * J = sum_k sum_p |E(r_p; e^k)|^2 and the forward residuals
 * R^k = A e^{k+1} - B e^k + A e^{k-1} + a d2g^k, the adjoint march runs backward,
 *     A mu^k = B mu^{k+1} - A mu^{k+2} + dJ/de^k,   mu^{N+1} = mu^{N+2} = 0,
 * with the same factors (A and B are symmetric), and
 *     dJ/deps_K = -sum_k mu^k^T T_K (e^k - 2 e^{k-1} + e^{k-2}),
 *     dJ/da     = -sum_k mu^k . d2g^{k-1}   (T_K: unit-eps element mass matrix of tet K).
 * The adjoint keeps its own time levels and interface multipliers in the workspace. */

/* mu^{k+1} = mu^{k+2} = 0: start of a backward sweep. */
int dd_adjoint_reset(dd_handle* h, void* stream);

/* One backward level: mu^k from (mu^{k+1}, mu^{k+2}) and seed = dJ/de^k
 * (device [n_dof]), then, if grad_eps (device [n_tets]) is given,
 * grad_eps[K] -= mu^k^T T_K (e_k - 2 e_km1 + e_km2) with the forward fields
 * e_k = e^k, e_km1 = e^{k-1}, e_km2 = e^{k-2} (device [n_dof]); if grad_amp
 * (device scalar) and d2g_hat (device [n_dof], unit-amplitude source second
 * difference of forward step k-1) are given, *grad_amp -= mu^k . d2g_hat.
 * mu_out (device [n_dof] or NULL) receives mu^k.  Uses the handle's precision
 * and tolerances.  Errors as dd_step. */
int dd_adjoint_step(dd_handle* h, const double* seed, const double* e_k, const double* e_km1, const double* e_km2,
                    const double* d2g_hat, double* grad_eps, double* grad_amp, double* mu_out, dd_stats* stats,
                    void* stream);

/* dd_adjoint_step with d2g_hat taken as d2g_scale * d2g_hat (the separable
 * source of dd_step_scaled): *grad_amp -= d2g_scale * (mu^k . d2g_hat).  With
 * d2g_scale = 1 it is dd_adjoint_step.  d2g_scale must be finite (DD_ERR_ARG). */
int dd_adjoint_step_scaled(dd_handle* h, const double* seed, const double* e_k, const double* e_km1,
                           const double* e_km2, const double* d2g_hat, double d2g_scale, double* grad_eps,
                           double* grad_amp, double* mu_out, dd_stats* stats, void* stream);

/* seed = 2 * weight * P^T P e: dJ/de of weight * sum_p |E(r_p; e)|^2 over the
 * probe set (device [n_dof] e and seed; seed is overwritten). */
int dd_probe_seed(dd_handle* h, const double* e, double weight, double* seed, void* stream);

/* The probe objective on the device: *J += weight * sum_p |E(r_p; e)|^2 over
 * the probe set (Sec. II's field interpolation E = sum_i e_i W_i at each
 * point), summed in a fixed order (probes, then x, y, z).  e: device [n_dof],
 * or NULL for the current e^n; J: device scalar, accumulated.  Errors:
 * DD_ERR_ARG, DD_ERR_STATE (no workspace, or an ensemble). */
int dd_probe_objective(dd_handle* h, const double* e, double weight, double* J, void* stream);

/* New relative permittivity per tet, on the device (eps: device [n_tets],
 * read during the call): re-assembles the subassembled local mass matrices
 * T^(s) = sum_K eps_K T_K (Sec. II-B's mass matrix, torn as in Sec. III-A) from
 * the unit-eps element matrices kept in the workspace -- in the host
 * assembly's order, so the values equal those dd_setup would build from the
 * same eps bitwise -- and marks the handle unfactored: call dd_factor next
 * (which rebuilds A = T + dt^2/4 S, the local eliminations and the coarse
 * problem).  The mesh, the tearing and mu are unchanged; eps must be positive
 * (not checked on the device).  The first call uploads the element-to-entry
 * map (synchronous).  Errors: DD_ERR_ARG, DD_ERR_STATE (no workspace, or an
 * ensemble), DD_ERR_CUDA.  Synchronises `stream`. */
int dd_set_eps(dd_handle* h, const double* eps, void* stream);

/* ---- particle-in-cell coupling (Sec. II PIC cycle) --------------------
 * Macro-particles enter through the mesh boundary at given times and move on
 * straight segments within a step.  Per step (dd_pic_step):
 *  1. push: Boris with E(x^n) from the edge field e^n (Whitney 1-forms) and
 *     B(x^n) from the face fluxes b^n (Whitney 2-forms); a particle injected
 *     during the step moves without a push from its injection time;
 *  2. deposit: q * int W_e . dl along the path, cut at every face crossed
 *     (exact; conserves charge per particle), into dep^{n+1/2}; a path that
 *     reaches a wall stops there;
 *  3. field step: dd_step with d2g = dep^{n+1/2} - dep^{n-1/2} (the second
 *     difference of the integrated current g);
 *  4. Faraday: b^{n+1} = b^n - dt/2 * C (e^{n+1} + e^n), C the discrete curl.
 * Deposition uses FP64 atomic adds (summation order is not fixed). */
typedef struct {
    int64_t n_particles;
    const double* x_inj;   /* host [n*3] injection points (on the mesh boundary) */
    const double* v_inj;   /* host [n*3] velocity from injection on */
    const double* t_inj;   /* host [n] injection times (t >= 0) */
    double q;              /* macro-particle charge */
    double qm;             /* charge / mass */
} dd_beam;

/* Host set-up of the particle data: faces, tet adjacency, the boundary tet of
 * every injection point.  Call after dd_setup and before dd_bind_workspace
 * (the workspace size grows with the particles).  Errors: DD_ERR_ARG when an
 * injection point is not on the mesh boundary. */
int dd_set_beam(dd_handle* h, const dd_beam* beam);

/* One PIC cycle at t_n = step * dt (see above).  stats as dd_step; a particle
 * crossing more than 64 tets in one step sets DD_ERR_ARG. */
int dd_pic_step(dd_handle* h, dd_stats* stats, void* stream);

/* Particle state and integrated current (device outputs, any may be NULL):
 * x [n*3] positions, status [n] (0 waiting, 1 in flight, 2 stopped at a wall),
 * G [n_dof] integrated current g^n, b [n_faces] face fluxes.  Sizes: n_faces
 * is returned in *n_faces (host, may be NULL). */
int dd_pic_state(const dd_handle* h, double* x, int32_t* status, double* G, double* b, int64_t* n_faces,
                 void* stream);

/* Apply the Schur-complement interface operator of Eq. f1schur,
 * out = (F_rr + F_rc K~cc^-1 F_rc^T) lam, in FP64 with the factors of the last
 * dd_factor.  lam, out: device [n_lambda]. */
int dd_schur_apply(dd_handle* h, const double* lam, double* out, void* stream);

/* Apply the coupled operator of Eqs. F1lr + F1uc in FP64 with the factors of
 * the last dd_factor:
 *   out[0:n_lambda]          = F_rr u_l + F_rc u_c
 *   out[n_lambda:+n_corner]  = -F_rc^T u_l + K~cc u_c
 * with u_l = u[0:n_lambda], u_c = u[n_lambda:n_lambda+n_corner].
 * u, out: device [n_lambda + n_corner], not overlapping.  Uses the handle's
 * workspace (not reentrant on one handle).  Errors: DD_ERR_ARG, DD_ERR_STATE
 * (not factored), DD_ERR_CUDA. */
int dd_coupled_apply(dd_handle* h, const double* u, double* out, void* stream);

/* With the DP2 factorisation (scheme DD_SCHEME_DP2 at dd_factor) the coupled
 * operator of Eqs. f2imp1 + F2un instead, u = [l1; l2; x_c] (device
 * [2 n_lambda + n_corner]):
 *   out[0:nl]        = l1 + l2 - 2 alpha M_T t2(u)
 *   out[nl:2nl]      = l1 + l2 - 2 alpha M_T t1(u)
 *   out[2nl:]        = K~cc x_c + sum_s B_c A_cr (A+R)_rr^-1 lambda^(s)
 * with t_side(u) the interface traces (A+R)_rr^-1 (lambda^(s) - A_rc x_c) of
 * the multiplier edges in the subdomain of that side.  Errors as
 * dd_coupled_apply (DD_ERR_STATE if the factorisation is DP1). */
int dd_dp2_apply(dd_handle* h, const double* u, double* out, void* stream);

/* Interface tangential mass M_T on the multiplier edges (host CSR, n_lambda
 * rows; column = multiplier index).  *nnz (host) receives the number of
 * entries; ptr [n_lambda+1], col [nnz], val [nnz] may each be NULL. */
int dd_get_interface_mass(const dd_handle* h, int64_t* nnz, int64_t* ptr, int32_t* col, double* val);

/* Same result as dd_schur_apply, for callers that must not allocate device
 * memory (for example code running inside a fixed memory pool, a callback
 * that may only use buffers it was handed, or a latency-critical loop where an
 * allocation would synchronise the device).  The paper has no counterpart: this
 * is a library convenience.  The call allocates nothing: its scratch vectors
 * live in a file-scope device array of 2^20 doubles (8 MiB) that every GPU
 * loading the library keeps until the process exits.  The caller passes lam and
 * out (device [n_lambda]) and must have bound a workspace and factored.
 * Limit: (n_local rounded up to 32) + 2 x (n_corner rounded up to 32) <= 2^20,
 * else DD_ERR_ARG with a message.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  The address is cached per device
 * ordinal, so calls must run in the device's primary context (the one the CUDA
 * runtime and torch use), not in another driver-API context on that device.
 * All calls on a device share the array: calls whose kernels overlap on the GPU
 * race on it. */
int dd_schur_apply_static(dd_handle* h, const double* lam, double* out, void* stream);

/* Evaluate E = sum_i e_i W_i at the probe points for the current e^n.
 * out: device [n_probe*3] (x, y, z per probe). */
int dd_probe(dd_handle* h, double* out, void* stream);

/* Read / write the time levels (e^n, e^{n-1}), device [n_dof] each, and the
 * step counter (checkpoint / resume).  dd_set_state also clears the CG warm
 * start. */
int dd_get_state(const dd_handle* h, double* e_n, double* e_nm1, int64_t* step, void* stream);
int dd_set_state(dd_handle* h, const double* e_n, const double* e_nm1, int64_t step, void* stream);

/* Per-stage timing of the library's own kernels (CUDA events recorded on the
 * launch stream around every launch while enabled).
 * Stages: 0 right-hand side SpMV, 1 local solve GEMV (A_rr^-1 b_r),
 * 2 interface-row GEMV of the Eq. f1schur operator (F_rr and F_rc pieces),
 * 3 coarse K~cc^-1 GEMV, 4 corner-row GEMVs (F_rc^T pieces, and the F_rc
 * pieces of the interface right-hand side), 5 recovery GEMV (Eq. rF1),
 * 6 interface/corner vector kernels (jumps, gathers, CG updates),
 * 7 FP64 refinement residual, 8 factorisation kernels.
 * launches   kernels launched (including ones that exit early after convergence)
 * work       launches that did their full work
 * ms         summed event time of all launches of the stage
 * bytes      algorithmic bytes of the launches that did full work (matrix
 *            elements read at the stage's precision + vectors read and written)
 * total_launches  every kernel launched by the library since the last reset. */
#define DD_N_STAGES 9
typedef struct {
    int64_t launches[DD_N_STAGES];
    int64_t work[DD_N_STAGES];
    double ms[DD_N_STAGES];
    double bytes[DD_N_STAGES];
    int64_t total_launches;
} dd_profile_stats;

/* enable: 1 = reset counters and start recording events, 0 = stop recording,
 * -1 = leave as is.  out (host, may be NULL) receives the accumulated numbers
 * (synchronises `stream`).  Launch counting is always on; event timing only
 * while enabled. */
int dd_profile(dd_handle* h, int enable, dd_profile_stats* out, void* stream);

/* Tile autotuner for the batched subdomain GEMVs (the per-step hot kernels).
 * For each GEMV kind (local solve, corner rows, corner coupling, recovery,
 * coarse, interface rows) and each precision it times every candidate tile --
 * lanes per matrix row in {8, 16, 32} x rows per CTA in {8, 16, 32, 64, 128} --
 * on the factored operators with CUDA events (1 warm-up + 3 timed launches)
 * and keeps the fastest.  For the kinds read from packed symmetric tiles
 * (DD_MIXED, sym_fp32) it also times the kernel form, CTAs per subdomain and
 * ring depth, then the number of subdomains kept in L2 (1 warm-up + 8 timed
 * launches each; see dd_get_sym_config).  cache_path (host string, may be
 * NULL): a text file of "key precision kind lanes rows" lines (and "key 2 kind
 * cl st keep form" for the packed kinds) keyed by device name and problem
 * sizes; a complete entry is reused without timing, new results are appended.
 * Requires dd_factor; results are bitwise unaffected only up to the order of
 * floating-point sums inside a row (lanes per row changes it).  seconds (host,
 * may be NULL) receives the wall time.  Synchronises `stream`. */
int dd_autotune(dd_handle* h, const char* cache_path, double* seconds, void* stream);

/* Current tiles: lpr[p*7 + k], rows[p*7 + k] for precision p (0 FP64, 1 FP32)
 * and GEMV kind k (0 local, 1 corner rows, 2 corner coupling, 3 recovery,
 * 4 coarse, 5 interface rows, 6 coupled operator) of the dense kernel; host
 * int32[14] each.  Kinds 0, 3, 5 and 6
 * run in DD_MIXED on the packed symmetric tiles when sym_fp32 = 1: cl[k] CTAs (one cluster) per subdomain, a TMA ring
 * of st[k] tiles, and the tiles of subdomains 0 .. keep[k]-1 copied with an
 * L2 evict_last policy (the rest evict_first) so that they stay in L2 across
 * the launches of a Krylov solve; ws[k] is the kernel form: 0 the
 * CTA-synchronous kernel, 1 the warp-specialised one (a producer warp refills
 * the ring as the four consumer warps release slots, each consumer warp keeping
 * its own partial y), 2 (ensembles) one CTA applying every tile it loads to the
 * x of 2 or 4 ensemble copies of its subdomain, 3 (ensembles) the same for
 * pairs of copies, 4 (ensembles; local solve, recovery and coupled operator)
 * the tensor-core form: one CTA applies the kind's operator rectangle, stored
 * as 128 x 64 panels of three BF16 pieces (their sum is the FP64 value to about
 * 24 bits), to the x of 16 ensemble copies by tcgen05 MMAs accumulating in FP32
 * in tensor memory, six piece products per panel (results agree with the FP32
 * forms to FP32 rounding; cl, st and keep do not apply), 5 (single problems)
 * the persistent form: as many CTAs as the SMs hold, each streaming the
 * tiles of a queue of whole subdomains through one ring of st[k] (2..10)
 * tiles, the queues filled largest subdomain first to the least-loaded CTA,
 * cl[k] (1, 2 or 4) groups of four consumer warps taking alternate tiles,
 * helper warps staging x of the next subdomain and storing y of the last
 * (with one group bitwise the results of form 1 with cl = 1) (host int32[7]
 * each, 0 for the other kinds; any pointer may be NULL). */
int dd_get_tiles(const dd_handle* h, int32_t* lpr, int32_t* rows);

/* Bytes of one full launch of GEMV kind `kind` (numbering of dd_get_tiles) at
 * `precision` (DD_FP64 or DD_MIXED) with the current storage choice (host
 * doubles, either may be NULL).  algorithmic: the matrix elements the product
 * needs at the launch's precision -- for the packed symmetric FP32 operator its
 * distinct elements (a symmetric group block's triangle counted once) -- plus
 * the vectors read and written once; these are the bytes dd_profile reports.
 * streamed: what the kernel reads from memory by construction (for the packed
 * kinds the whole 64 x 64 tiles, padding and full diagonal tiles included;
 * otherwise equal to algorithmic).  Errors: DD_ERR_ARG. */
int dd_get_gemv_bytes(const dd_handle* h, int32_t kind, int32_t precision, double* algorithmic, double* streamed);
int dd_get_sym_config(const dd_handle* h, int32_t* cl, int32_t* st, int32_t* keep, int32_t* ws);

/* Sets the packed-tile launch of GEMV kind `kind` (0, 3, 5 or 6) to cl CTAs per subdomain (1, 2, 4 or 8), a ring of st tiles (2..4),
 * keep stored subdomains in L2 (0..n_sub) and kernel form ws (0..5 as in
 * dd_get_sym_config; 4 only for an ensemble's kinds 0, 3 and 6; 5 only for a
 * single problem, with cl = consumer groups (1, 2 or 4) and st up to 10 a
 * multiple of cl), as
 * dd_autotune would (its next run may change it again).
 * Results differ from another setting only in the order of FP32 sums.
 * DD_ERR_ARG for other kinds or values (or form 2 when its shared memory exceeds
 * a CTA's, or form 5 when cl of its CTAs do not fit one SM's shared memory; the
 * setting is then unchanged), DD_ERR_STATE before dd_bind_workspace or during a capture.
 * Synchronises `stream`; drops captured step graphs. */
int dd_set_sym_config(dd_handle* h, int32_t kind, int32_t cl, int32_t st, int32_t keep, int32_t ws, void* stream);

/* Failure-path testing aid for the bounded device waits.  With
 * first_wait_polls > 0, the first wait of every CTA of the packed-tile GEMVs
 * (DD_MIXED with sym_fp32) polls an mbarrier that nothing completes that many
 * times and gives up, as a wait on a lost copy would: the CTA records the
 * failure in the device status word, waits (bounded) for the copies it has in
 * flight and exits.  The step then returns DD_ERR_TIMEOUT -- in eager mode at
 * once, in graph mode from the first call that reads stats -- and is not
 * taken: e^n, e^{n-1} and the step counter stay where they were and the next
 * solve starts cold.  0 restores the normal waits (2^20 polls).  Synchronises
 * `stream`.  Errors: DD_ERR_ARG (negative), DD_ERR_STATE (no workspace). */
int dd_set_wait_limit(dd_handle* h, int32_t first_wait_polls, void* stream);

/* FP64 FMA throughput of the current device in TFLOP/s (2 flops per FMA):
 * eight independent FMA chains per thread, 8 CTAs of 256 threads per SM, best
 * of three CUDA-event-timed launches after one warm-up.  The roofline of the
 * FP64 path (its GEMVs are FP64-ALU bound on GB300) is stated against it.
 * Synchronises `stream`.  Errors: DD_ERR_ARG, DD_ERR_CUDA. */
int dd_measure_fp64_rate(double* tflops, void* stream);

/* Self-check of the fifth-generation tensor-core path the library builds on
 * (tcgen05 MMA, BF16 operands in shared memory, FP32 accumulator in tensor
 * memory): one 128 x 16 x 64 product per operand layout on integer-valued
 * inputs, compared element by element with the same sums on the CUDA cores.
 * *passed_mask (host) receives bit v set for each layout that matched exactly:
 * v = 0 A K-major; v = 1, 2 A stored M-major (the transposed operand) with the
 * two assignments of the descriptor's leading and stride offsets.  The paper
 * has no counterpart (a hardware check).  Synchronises `stream`.  Errors:
 * DD_ERR_ARG, DD_ERR_CUDA. */
int dd_tc_selftest(int32_t* passed_mask, void* stream);

void dd_destroy(dd_handle* h);
const char* dd_last_error(const dd_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
