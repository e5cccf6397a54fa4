// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dd.h"

// Dense per-subdomain operator: row-major ns x ld block at element offset moff of
// the dense buffer.  After dd_factor the block holds the partially swept local
// matrix [[A_rr^-1, -A_rr^-1 A_rc], [A_cr A_rr^-1, A_cc - A_cr A_rr^-1 A_rc]].
struct MatDesc {
    int64_t moff;   // element offset of row 0 in the dense buffer
    int64_t voff;   // offset of the subdomain's first local slot in flat local vectors
    int32_t ld;     // row stride (elements), multiple of 4
    int32_t nI;     // interior (m = 1) unknowns
    int32_t nr;     // r block = interior + interface
    int32_t ns;     // r + corner
};

#ifdef __CUDACC__
#define DD_HD __host__ __device__
#else
#define DD_HD
#endif

// Packed symmetric FP32 storage of the swept local matrices (DD_MIXED GEMVs).
// M_s = J S_s with S_s symmetric and J = diag(I_r, -I_c) (A_rr^-1 and the
// corner Schur complement are symmetric, M_s[c][r] = -M_s[r][c]^T); the
// lower triangle of S_s is stored and y = M x is formed as J (S x).  The local
// order [I | Gamma | c] is cut into two runs of tile rows of height kSymT, the
// interior I (tile rows 0 .. tI-1) and G = [Gamma | c] (tile rows tI .. nt-1),
// the last row of each run as short as the run leaves it.  Tile (a, b), b <= a,
// is h(a) x h(b): stored row-major with its width rounded up to 4 floats
// (zeros after the last column), or, on the diagonal (a == b), as its lower
// triangle with row r padded to 4 * ceil((r+1)/4) floats and the diagonal
// entries halved (the tile then serves as a lower and as an upper triangle
// alike).  Per subdomain the tiles follow each other without gaps: the lower
// triangle of the G x G block (row order; everything the interface rows and the
// coupled operator read is one run), the G x I rectangle, the lower triangle of
// the I block.  Every tile starts on a 16-byte boundary and its size is a
// multiple of 16 bytes (one bulk copy each).
constexpr int kSymT = 64;
constexpr int kSymTile = kSymT * kSymT;   // floats of the largest tile (a ring slot)
constexpr int kSymCLMax = 8;       // most CTAs per subdomain (one thread-block cluster)
constexpr int kSymStages = 4;      // deepest TMA ring (tiles in flight per CTA)
constexpr int kSymStagesPs = 10;   // deepest ring of the persistent packed form (one or two CTAs per SM)

struct SymDesc {
    int64_t toff;     // float offset of the subdomain's first tile in the packed buffer
    int64_t voff;     // first slot of the subdomain
    int32_t n[3];     // nI, nGamma, nc
    int32_t tI;       // tile rows of I
    int32_t nt;       // tile rows in all (I, then G)
};

// Height of tile row a.
DD_HD inline int sym_h(const SymDesc& sd, int a) {
    const int left = a < sd.tI ? sd.n[0] - kSymT * a : sd.n[1] + sd.n[2] - kSymT * (a - sd.tI);
    return left < kSymT ? left : kSymT;
}
// Element groups (bit 0 I, bit 1 Gamma, bit 2 c) present in tile row a.
DD_HD inline int sym_gmask(const SymDesc& sd, int a) {
    if (a < sd.tI) return 1;
    const int g0 = kSymT * (a - sd.tI), g1 = g0 + sym_h(sd, a);
    return (g0 < sd.n[1] ? 2 : 0) | (g1 > sd.n[1] ? 4 : 0);
}
// Local index of padded position p = kSymT * a + q (-1 beyond the run's end).
DD_HD inline int sym_local(const SymDesc& sd, int p) {
    const int a = p / kSymT, q = p - kSymT * a;
    if (a < sd.tI) return kSymT * a + q < sd.n[0] ? kSymT * a + q : -1;
    const int g = kSymT * (a - sd.tI) + q;
    return g < sd.n[1] + sd.n[2] ? sd.n[0] + g : -1;
}
DD_HD inline int sym_lgroup(const SymDesc& sd, int l) { return l < sd.n[0] ? 0 : (l < sd.n[0] + sd.n[1] ? 1 : 2); }
// Diagonal tiles: padded length and start of row r (floats).
DD_HD inline int sym_rowlen(int r) { return ((r + 4) >> 2) << 2; }
DD_HD inline int sym_trioff(int r) {
    const int k = r >> 2, m = r & 3;
    return 8 * k * (k + 1) + 4 * m * (k + 1);
}
// Floats of a stored tile of h rows and w columns (diag: the padded triangle).
DD_HD inline int sym_tile_floats(int h, int w, bool diag) { return diag ? sym_trioff(h) : h * ((w + 3) & ~3); }

// Row and column groups (bit 0 I, bit 1 Gamma, bit 2 c) of the GEMV modes that
// use the packed storage; false for the others.
DD_HD inline bool sym_masks(int mode, int* rmask, int* cmask) {
    switch (mode) {
        case 0: *rmask = 7; *cmask = 3; return true;   // GEMV_LOCAL:   rows all, cols r
        case 3: *rmask = 3; *cmask = 6; return true;   // GEMV_RECOVER: rows r, cols Gamma c (ensembles only)
        case 5: *rmask = 2; *cmask = 6; return true;   // GEMV_SCHUR_G: rows Gamma, cols Gamma c
        case 6: *rmask = 6; *cmask = 6; return true;   // GEMV_COUPLED: rows Gamma c, cols Gamma c
        default: return false;
    }
}

// What stored tile (a, b), b <= a, contributes to y[R] = M[R, C] x[C]:
// bit 0 direct (rows of a, columns of b), bit 1 mirrored (rows of b, columns
// of a: the transposed tile), bit 2 a diagonal tile (both roles of its stored
// triangle).  Element-level masks (x staged as 0 outside C, rows outside R not
// stored) make a tile that only partly overlaps R or C exact.
DD_HD inline int sym_tile_flags(const SymDesc& sd, int a, int b, int rmask, int cmask) {
    const int ga = sym_gmask(sd, a), gb = sym_gmask(sd, b);
    if (a == b) return ((ga & rmask) && (ga & cmask)) ? 7 : 0;
    int f = 0;
    if ((ga & rmask) && (gb & cmask)) f |= 1;
    if ((gb & rmask) && (ga & cmask)) f |= 2;
    return f;
}

// Tensor-core operator storage of the ensemble GEMVs (members > 1; kernel form 4
// of the packed kinds local solve, recovery and coupled operator): the mode's
// rectangle M_s[r0:r1, c0:c1] of the swept matrix cut into panels of 128 rows x
// 64 columns, each stored as three BF16 matrices whose sum is the FP64 value to
// about 24 bits (A1 = bf16(m), A2 = bf16(m - A1), A3 = bf16(m - A1 - A2)), in the
// K-major core-matrix layout of the tcgen05 operands (zeros past r1 / c1).
// Panels follow each other column block by column block (block q, then panel p).
constexpr int kTcP = 128;                 // panel rows (MMA M)
constexpr int kTcK = 64;                  // panel columns
constexpr int kTcN = 16;                  // ensemble members per CTA (MMA N)
constexpr int kTcPieceElems = kTcP * kTcK;      // BF16 elements of one piece
constexpr int kTcBlockElems = 3 * kTcPieceElems; // of one panel block (three pieces)
struct TcDesc {
    int64_t off;        // BF16 element offset of block (p = 0, q = 0)
    int32_t r0, r1;     // local row range of the mode
    int32_t c0, c1;     // local column range
    int32_t P, Q;       // panels and column blocks
};
// The tensor-core kinds and their index in the per-kind tables.
DD_HD inline int tc_kind_index(int mode) { return mode == 0 ? 0 : (mode == 3 ? 1 : (mode == 6 ? 2 : -1)); }
constexpr int kTcKinds = 3;

// One CTA of a batched GEMV: rows [row0, row1) of matrix `mat`.
struct GemvTask {
    int32_t mat;
    int32_t row0;
    int32_t row1;
    int32_t pad;
};

// Column/row ranges of the batched dense GEMV, all relative to one MatDesc.
enum GemvMode : int {
    GEMV_LOCAL = 0,    // rows [0,ns)  cols [0,nr):  [y; A_cr y] from b_r                  (Eq. rF1 / F1uc)
    GEMV_SCHUR_C = 1,  // rows [nr,ns) cols [nI,nr): A_cr A_rr^-1 B_r^T z, the F_rc^T pieces (Eq. f1schur)
    GEMV_CORNER = 2,   // rows [nI,nr) cols [nr,ns): A_rr^-1 A_rc v, the F_rc pieces       (Eq. f1schur)
    GEMV_RECOVER = 3,  // rows [0,nr)  cols [nI,ns): x_r from y, lambda, x_c               (Eq. rF1)
    GEMV_COARSE = 4,   // the dense K~cc^-1 (single matrix)
    GEMV_SCHUR_G = 5,  // rows [nI,nr) cols [nI,ns): F_rr and F_rc pieces in one pass       (Eq. f1schur)
    GEMV_COUPLED = 6,  // rows [nI,ns) cols [nI,ns): F_rr, F_rc, F_rc^T and K~cc pieces   (Eqs. F1lr, F1uc)
    GEMV_NMODES = 7
};

// Source of the x vector of a batched GEMV (staged in shared memory per CTA).
// kind (X_*): X_FLAT x_j = v[slot]; X_LAMBDA x_j = (B_r^T v)_j; X_PCG x_j =
// (B_r^T (z + beta p))_j with z = v, p = v2; X_CORNER x_j = v[corner(slot)];
// X_RECOVER interface slot -(B_r^T v)_j, corner slot v2[corner(slot)];
// X_COARSE x_j = v[j]; X_PCG_CV / X_LAMBDA_CV: interface slots as X_PCG /
// X_LAMBDA, corner slots -v3[corner(slot)]; X_SIDE_CP (MFETI-DP2) interface
// slots v[m] in the first subdomain of multiplier m and v2[m] in the second
// (unsigned), corner slots +v3[corner(slot)].  k_gemv<double> reads v/v2, k_gemv<float> reads the
// FP32 shadows vf/v2f so that it executes no FP64 instruction.
struct XSrc {
    int kind;
    const double* v;
    const double* v2;
    const double* v3;
    const float* vf;
    const float* v2f;
    const float* v3f;
    const int32_t* slot_mult;
    const int32_t* slot_corner;
    const struct PcgScalars* sc;
};

// Output of a batched GEMV: out[voff+row] = base + alpha * (M x)_row, written in
// FP64 (out/base) and/or FP32 (out32/base32; FP32 arithmetic).  pos (may be
// null; then base is null too): the row of slot o is written at out[pos[o]].
struct GemvOut {
    double* out;
    const double* base;
    float* out32;
    const float* base32;
    double alpha;
    const int32_t* pos = nullptr;
};

// Tile shape of a batched GEMV launch: lanes cooperating on one row and rows
// handled by one CTA.  Defaults below; dd_autotune replaces them by measurement.
struct TileCfg {
    int32_t lpr;
    int32_t rows;
};

// Device scalars of the interface CG (one struct in the workspace).
struct PcgScalars {
    double rz;        // r . z
    double rz_new;
    double pq;        // p . q
    double alpha, beta;
    double rr;        // ||r||^2
    double gg;        // ||rhs||^2
    double tol2;      // tol^2 * gg
    int32_t it;       // iterations done
    int32_t done;     // 1 when converged (kernels become no-ops)
    int32_t status;   // DD_OK / DD_ERR_NONFINITE
    int32_t wait_err; // nonzero once a bounded TMA wait of the packed-tile GEMV gave up
    double norm_b2;   // mixed mode: ||b||^2 of the step system
    double norm_r2;   // mixed mode: ||r||^2 of the current FP64 residual
    int32_t lam_levels;   // warm_start 2: multiplier history levels available (0, 1, 2)
    int32_t wait_first;   // > 0: the first mbarrier wait of every packed-GEMV CTA polls an mbarrier
                          // nothing completes, this many times, and gives up (failure-path test; 0 = off)
    int32_t it_total;     // graph mode: CG iterations of the whole step
    int32_t refinements;  // graph mode: solves of the whole step
    int32_t step_status;  // graph mode: DD status of the whole step
    int32_t cycles;       // graph mode: GMRES restart cycles of the whole step
    uint32_t counter[8];  // last-block counters of the grid reductions
};

constexpr int kMaxRestart = DD_MAX_RESTART;
constexpr int kMaxMembers = 64;   // ensemble size limit
constexpr int kSymRng = 5;        // ints per CTA in a packed GEMV work table
constexpr int kTlW = 2;           // u32 words per tile-list entry (a << 16 | b << 3 | flags, float offset)
#ifndef DD_GM_ELEMS
#define DD_GM_ELEMS 4
#endif
constexpr int kGmElems = DD_GM_ELEMS;                // vector elements per thread in the GMRES kernels
constexpr int kGmChunk = kGmElems * 256;             // elements per block

// Device state of the restarted GMRES of the coupled system (one struct in the
// workspace).  The control words come first: eager mode reads them back.
struct GmresScalars {
    int32_t j;          // Arnoldi column being built in the current cycle
    int32_t it;         // Arnoldi steps of this solve
    int32_t k;          // columns of the cycle that just ended (update x with y[0..k))
    int32_t cycle_end;  // the current cycle has ended (inner loop stops)
    int32_t final;      // the solve ends after the pending update (converged, budget spent or non-finite)
    int32_t converged;
    int32_t status;     // DD_OK / DD_ERR_NONFINITE
    int32_t skip;       // cycle_end: per-step kernels exit at once
    double bnorm;       // ||b||
    double tol;         // relative tolerance of the solve
    double thr;         // tol * ||b||
    double beta;        // ||r_0|| of the cycle
    double hnext;       // norm of the vector to normalise next (beta, then H[j+1][j])
    double resid;       // |g_{j+1}| after the last step
    int32_t max_it, m, cycles;
    int32_t nh2;        // terms of the second projection k_gm_normalize applies (0 at a cycle start)
    uint32_t counter[4];
    double g[kMaxRestart + 1];
    double cs[kMaxRestart], sn[kMaxRestart];
    double y[kMaxRestart];
    double h1[kMaxRestart + 1];   // first Gram-Schmidt projection of the current column
    double h2[kMaxRestart + 1];   // second projection
    double H[kMaxRestart * (kMaxRestart + 1)];   // column j at H[j * (kMaxRestart + 1)], rotated in place
};
constexpr size_t kGmCtrlBytes = offsetof(GmresScalars, max_it);

// The unknown of a coupled solve in three blocks, u = [u1 (n1); u2 (n2); uc (nc)]:
// MFETI-DP1 u1 = lambda, n2 = 0; MFETI-DP2 u1, u2 = the multipliers of the first
// and of the second subdomain of every interface edge.  Also what turns the
// output w (per slot) of the [Gamma|c]-row GEMV into (M u).
struct UView {
    int64_t n1 = 0, n2 = 0, nc = 0;
    const double* b1 = nullptr;   // right-hand side blocks
    const double* b2 = nullptr;
    const double* bc = nullptr;
    double* x1 = nullptr;         // iterate blocks
    double* x2 = nullptr;
    double* xc = nullptr;
    float* x1f = nullptr;         // their FP32 shadows (DD_MIXED) or null
    float* x2f = nullptr;
    float* xcf = nullptr;
    const double* d1 = nullptr;   // inverse diagonal of block 1 (null: 1); block 2 has 1
    const double* dc = nullptr;   // inverse diagonal of the corner block (null: 1)
    const int64_t* ms = nullptr;  // mult_slot, corner_ptr, corner_slot
    const int64_t* cp = nullptr;
    const int64_t* cs = nullptr;
    const int64_t* mtp = nullptr; // MFETI-DP2: interface tangential mass (CSR over multipliers); null for DP1
    const int32_t* mtc = nullptr;
    const double* mtv = nullptr;
    double two_alpha = 0.0;
};

struct DevPtrs {
    // maps (slot = flat local index over all subdomains)
    MatDesc* mats = nullptr;
    MatDesc* coarse_desc = nullptr;  // single descriptor of K~cc (ld = ldc)
    int32_t* slot_sub = nullptr;     // subdomain of each slot
    int64_t* copy_ptr = nullptr;     // [n_dof+1] copies of each dof, by subdomain
    int64_t* copy_slot = nullptr;    // [n_local]
    int32_t* slot_mult = nullptr;    // +(m+1) in s1, -(m+1) in s2, 0 if not an interface slot
    int32_t* slot_corner = nullptr;  // corner id of a corner slot, else -1
    int32_t* slot_dof = nullptr;     // dof of each slot
    uint8_t* slot_own = nullptr;     // 1 if this slot's subdomain owns the dof
    int64_t* mult_slot = nullptr;    // [n_lambda*2] slots of s1 and s2
    int64_t* corner_ptr = nullptr;   // [n_corner+1]
    int64_t* corner_slot = nullptr;  // copies of every corner, by subdomain
    int32_t* slot_upos = nullptr;    // [n_local] where the coupled operator writes a slot's row: 2 m + side for
                                     // multiplier m, 2 n_lambda + k for corner copy k, -1 for interior slots
    int64_t* owner_slot = nullptr;   // [n_dof] slot in the owner subdomain
    int64_t* row_ptr = nullptr;      // local CSR over slots [n_local+1]
    int32_t* col_loc = nullptr;      // local column index
    int32_t* col_dof = nullptr;      // global dof of the column
    double* Tval = nullptr;
    double* Sval = nullptr;
    double* Aval = nullptr;          // T + dt^2/4 S (filled by dd_factor)
    GemvTask* tasks[2][GEMV_NMODES] = {};   // [0] FP64 tiles, [1] FP32 tiles
    int32_t* probe_dof = nullptr;
    double* probe_w = nullptr;
    // dense operators
    double* M64 = nullptr;           // per-subdomain swept matrices
    float* M32 = nullptr;            // FP32 copy
    float* Msym = nullptr;           // packed symmetric FP32 tiles (see SymDesc)
    SymDesc* symd = nullptr;         // [n_sub]
    int32_t* sym_dir = nullptr;      // [tiles * 4] (stored subdomain, a, b, float offset) of every stored tile
    uint16_t* Mtc = nullptr;         // tensor-core operator storage of the ensemble GEMVs (BF16 bits, see TcDesc)
    TcDesc* tcd[kTcKinds] = {};      // [n_sub_real] per tensor-core kind
    int32_t* tc_dir = nullptr;       // [blocks * 4] (kind, stored subdomain, p, q) of every stored panel block
    int32_t* sym_rng[GEMV_NMODES] = {};   // [n_sub * kSymCLMax * kSymRng] (list offset, tile count, end tile row,
                                          // subdomain, ensemble members served) per CTA
    uint32_t* sym_tl[GEMV_NMODES] = {};   // tiles of each packed mode, every subdomain in row order
    double* K64 = nullptr;           // K~cc^-1, n_corner x ldc
    float* K32 = nullptr;
    double* Pinv = nullptr;          // [n_sub+1][NB*NB] pivot-block inverses while factoring
    uint16_t* oz_slices = nullptr;   // DD_FACTOR_TENSOR: BF16 slices of one pivot block's panels
    int32_t* oz_exps = nullptr;      // and their row / column exponents
    double* dinv = nullptr;          // [n_lambda] inverse Jacobi diagonal
    // particles (dd_set_beam): state, per-tet geometry and faces
    double* px = nullptr;            // [n_p*3] positions
    double* pv = nullptr;            // [n_p*3] velocities
    double* pt = nullptr;            // [n_p] injection times
    int32_t* ptet = nullptr;         // [n_p] current tet
    int32_t* pstat = nullptr;        // [n_p] 0 waiting, 1 in flight, 2 stopped at a wall
    int32_t* tets_dev = nullptr;     // [n_tets*4] node ids
    double* tgrad = nullptr;         // [n_tets*12] barycentric gradients
    double* tx0 = nullptr;           // [n_tets*3] coordinates of local vertex 0
    int32_t* tface = nullptr;        // [n_tets*4] face opposite each local vertex
    int32_t* tnbr = nullptr;         // [n_tets*4] neighbour across that face, -1 on the wall
    int32_t* face_nodes = nullptr;   // [n_faces*3] sorted node triple
    int32_t* face_edge = nullptr;    // [n_faces*3] dofs of edges (a,b), (b,c), (a,c); -1 on the wall
    double* bflux = nullptr;         // [n_faces] magnetic flux (Whitney 2-form dofs)
    double* dep[2] = {nullptr, nullptr};  // [n_dof] deposited integrated current of this / the previous step
    double* Gcum = nullptr;          // [n_dof] integrated current g^n (sum of deposits)
    double* d2g_pic = nullptr;       // [n_dof] source second difference of the PIC step
    int32_t* pic_err = nullptr;      // traversal overflow flag

    // time levels (ring of 3) of the forward and the adjoint march
    double* e[3] = {nullptr, nullptr, nullptr};
    double* mu[3] = {nullptr, nullptr, nullptr};
    double* lam_adj = nullptr;       // adjoint multipliers (warm start), swapped with lam
    double* lam2 = nullptr;          // MFETI-DP2: multipliers of the second subdomain of each interface edge
    float* lam2f = nullptr;
    double* lam2_adj = nullptr;
    float* lam2f_adj = nullptr;
    double* lam2_scratch = nullptr;  // first refinement pass's second block (next step's warm start)
    float* lam2f_scratch = nullptr;
    double* g2 = nullptr;            // MFETI-DP2: right-hand side of the second multiplier block
    int64_t* mt_ptr = nullptr;       // MFETI-DP2: interface tangential mass, CSR over multipliers
    int32_t* mt_col = nullptr;
    double* mt_val = nullptr;
    double* lam_prev = nullptr;      // multipliers of the step before (warm_start 2 extrapolation)
    double* lam_prev_adj = nullptr;
    double* xC_prev = nullptr;       // corner solution and DP2 second-side multipliers of the step
    double* xC_prev_adj = nullptr;   // before (warm_start 2 with the coupled GMRES)
    double* lam2_prev = nullptr;
    double* lam2_prev_adj = nullptr;
    float* lamf_adj = nullptr;
    int64_t* eps_ptr = nullptr;      // [nnz_local+1] dd_set_eps: contributions of each local mass entry
    int32_t* eps_idx = nullptr;      // element-matrix entries 36 t + 6 p + q, in the host assembly's order
    int32_t* tet_dof = nullptr;      // [n_tets*6] dof of each tet edge, -1 on the PEC wall
    double* That = nullptr;          // [n_tets*36] unit-eps oriented element mass matrices
    // flat local vectors (n_local)
    double* b = nullptr;             // local right-hand side
    double* y = nullptr;             // GEMV outputs / local solutions
    double* w = nullptr;             // interface operator output per slot
    double* x = nullptr;             // recovered local solution
    float* bf = nullptr;             // FP32 shadows for DD_MIXED (inputs/outputs of k_gemv<float>)
    float* wf = nullptr;
    // interface vectors (n_lambda)
    double* lam = nullptr;
    double* g = nullptr;
    double* r = nullptr;
    double* p = nullptr;
    double* q = nullptr;
    double* z = nullptr;
    double* lam_scratch = nullptr;
    // corner vectors (n_corner)
    double* fC = nullptr;
    double* uC = nullptr;
    double* vC = nullptr;
    double* xC = nullptr;
    double* xC_adj = nullptr;        // adjoint march's corner solution (coupled GMRES warm start)
    float* xCf_adj = nullptr;
    double* dinvC = nullptr;         // [n_corner] inverse diagonal of K~cc
    // coupled GMRES vectors (n_u = n_lambda + n_corner, leading dimension gm_ldv)
    double* Vk = nullptr;            // [(kMaxRestart+1) * gm_ldv] Krylov basis
    double* tu = nullptr;            // [n_u] Arnoldi work vector
    double* zu = nullptr;            // [n_u] D^-1 v_j, the operator's input
    float* zuf = nullptr;            // [n_u] FP32 shadow of zu (DD_MIXED)
    double* xC_scratch = nullptr;    // [n_corner] first-pass corner solution kept across refinement passes
    float* xCf_scratch = nullptr;
    GmresScalars* gs = nullptr;
    double* gpart = nullptr;         // [(kMaxRestart+1) * gm_blocks] block partials
    float* fCf = nullptr;
    float* uCf = nullptr;
    float* vCf = nullptr;
    float* xCf = nullptr;
    float* zf = nullptr;             // [n_lambda] shadows
    float* pf = nullptr;
    float* lamf = nullptr;
    float* lamf_scratch = nullptr;
    // global vectors (n_dof)
    double* delta = nullptr;         // assembled correction of the step
    double* delta_k = nullptr;       // assembled correction of one refinement
    double* src_in = nullptr;        // graph mode: the step's source, copied in before each launch
    double* res = nullptr;           // assembled FP64 residual
    // scalars
    PcgScalars* sc = nullptr;
    double* partials = nullptr;      // [kMaxPartials] block partial sums
    int32_t* status = nullptr;       // factor status word
};

struct dd_handle {
    dd_params prm{};
    std::string err;

    // mesh
    int64_t n_nodes = 0, n_tets = 0;
    std::vector<double> xyz;
    std::vector<int32_t> tets;
    std::vector<double> eps;
    double mu = 1.0;

    // edges and elements
    int64_t n_edges = 0, n_dof = 0;
    std::vector<int64_t> edges;      // 2 per edge
    std::vector<int64_t> dof_edge;   // n_dof
    std::vector<int64_t> tet_dof;    // 6 per tet, -1 on the PEC wall
    std::vector<double> That, Shat;  // 36 per tet, oriented, unit coefficients
    std::vector<double> grad;        // 12 per tet: barycentric gradients
    std::vector<double> vol;

    // tearing
    int32_t n_sub = 0;
    std::vector<int32_t> part;
    std::vector<int64_t> sub_ptr;
    std::vector<int64_t> local_dof;
    std::vector<int32_t> nI, nG, nC;
    std::vector<int32_t> owner;
    std::vector<int64_t> mult_dof;
    std::vector<int32_t> mult_sub, mult_loc;
    std::vector<int64_t> corner_dof;
    std::vector<int32_t> slot_mult, slot_corner, slot_dof;
    std::vector<uint8_t> slot_own;
    std::vector<int64_t> mult_slot, corner_ptr, corner_slot, owner_slot;
    std::vector<int32_t> slot_upos;
    int32_t members = 0;           // ensemble size R (set by dd_setup)
    int32_t n_sub_real = 0;        // subdomains of one member: the ones whose operators are stored (0 .. n_sub_real-1)
    std::vector<int32_t> slot_sub;
    std::vector<int64_t> copy_ptr, copy_slot;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col_loc, col_dof;
    std::vector<double> Tval, Sval;
    int64_t eps_contrib = 0;         // element-matrix entries that land in the local mass (dd_set_eps map size)
    bool eps_map_up = false;         // the dd_set_eps map is in the workspace
    std::vector<int64_t> mt_ptr;     // MFETI-DP2: interface tangential mass, CSR over multipliers
    std::vector<int32_t> mt_col;
    std::vector<double> mt_val;
    std::vector<MatDesc> mats;
    int64_t dense_elems = 0;
    int32_t ldc = 0;                 // leading dimension of K~cc
    int32_t max_nr = 0, max_ns = 0;
    std::vector<GemvTask> tasks[2][GEMV_NMODES];   // per precision (tile shapes may differ)
    std::vector<SymDesc> sym;                      // packed symmetric storage per subdomain
    std::vector<int32_t> sym_dir;                  // (stored subdomain, a, b, float offset) of every stored tile
    std::vector<TcDesc> tcd[kTcKinds];             // tensor-core storage per kind and stored subdomain (ensembles)
    std::vector<int32_t> tc_dir;                   // (kind, stored subdomain, p, q) of every panel block
    int64_t tc_elems = 0;                          // BF16 elements of the tensor-core storage
    int64_t sym_elems = 0;
    int32_t sym_np_max = 0;                        // largest padded side (floats)
    std::vector<int32_t> sym_rng[GEMV_NMODES];
    std::vector<uint32_t> sym_tl[GEMV_NMODES];     // tile list of each packed mode: pairs (a << 16 | b << 3 | flags,
                                                   // float offset of the tile in its subdomain)
    std::vector<int64_t> sym_tl_off[GEMV_NMODES];  // start of each subdomain's run in sym_tl (n_sub + 1)
    int32_t sym_cl[GEMV_NMODES] = {4, 1, 1, 1, 1, 2, 2};   // CTAs per subdomain of each packed mode
    int32_t sym_st[GEMV_NMODES] = {4, 4, 4, 4, 4, 4, 4};   // TMA ring depth of each packed mode
    int32_t sym_nl[GEMV_NMODES] = {};                      // longest tile list of one CTA (shared memory)
    int32_t sym_keep[GEMV_NMODES] = {};                    // subdomains whose tiles are kept in L2 (evict_last)
    int32_t sym_ws[GEMV_NMODES] = {};                      // packed kernel form: 0 CTA-synchronous, 1 warp-specialised,
                                                           // 2 ensemble copies of a subdomain in one CTA (up to 4),
                                                           // 3 ensemble copies in pairs, 4 tensor cores (ensembles),
                                                           // 5 persistent queues of subdomains (sym_cl = CTAs per SM)
    int32_t sym_grid[GEMV_NMODES] = {};                    // CTAs of the launch (sym_ranges)
    int32_t n_sm = 0;                                      // multiprocessors of the bound device
    int32_t sym_max_tiles = 0;                     // largest tile count of one subdomain
    int64_t sym_ntiles = 0;                        // stored tiles in all (entries of sym_dir / 4)
    bool sym_ok = false;                           // the packed GEMV's shared memory fits one CTA
    size_t task_cap[GEMV_NMODES] = {};             // device capacity: tasks at the smallest row count
    TileCfg tile[2][GEMV_NMODES];                  // lanes per row and rows per CTA, per precision and mode
    bool tuned = false;

    // particles (dd_set_beam)
    int64_t n_particles = 0;
    double pq = 0.0, pqm = 0.0;
    std::vector<double> p_x, p_v, p_t;
    std::vector<int32_t> p_tet;
    int64_t n_faces = 0;
    std::vector<int32_t> face_nodes, face_edge, tet_face, tet_nbr;
    int dep_cur = 0;

    // probes
    int32_t n_probe = 0;
    std::vector<int32_t> probe_dof;  // 6 per probe
    std::vector<double> probe_w;     // 18 per probe

    // device state
    char* ws = nullptr;
    size_t ws_bytes = 0;
    DevPtrs d;
    bool bound = false;
    bool factored = false;
    double dt = 0.0;
    int64_t step = 0;
    int cur = 0;                     // e[cur] = e^n, e[(cur+2)%3] = e^{n-1}
    int cur_adj = 0;                 // mu[cur_adj] = mu^{k+1}, mu[(cur_adj+2)%3] = mu^{k+2}
    bool lam_valid = false;
    bool lam_adj_valid = false;
    int factored_scheme = DD_SCHEME_DP1;   // scheme of the last dd_factor
    double factored_alpha = 0.0;           // its Robin coefficient (DP2)

    // CUDA-graph mode (dd_params.use_graph): one executable graph per time-level phase
    void* gexec[3] = {nullptr, nullptr, nullptr};   // cudaGraphExec_t
    void* gstream[16] = {};                         // private capture streams, one per nesting depth
    bool capturing = false;
    int64_t g_kernels_main = 0;      // kernels outside conditional bodies
    int64_t g_kernels_iter = 0;      // kernels per CG iteration (WHILE body)
    int64_t g_kernels_pass = 0;      // kernels per extra refinement pass outside its WHILE body
    int64_t g_kernels_cycle = 0;     // kernels per GMRES restart cycle outside its inner WHILE body
    int64_t gm_ldv = 0;              // leading dimension of the GMRES basis
    int32_t gm_blocks = 1;           // blocks of the GMRES vector kernels

    // profiling (dd_profile)
    bool prof_on = false;
    std::vector<void*> ev_pool;            // cudaEvent_t
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_recs;   // (stage, index of start event)
    int64_t launches[DD_N_STAGES] = {};
    int64_t work[DD_N_STAGES] = {};
    double work_bytes[DD_N_STAGES] = {};
    int64_t total_launches = 0;
    double bytes_per_launch[DD_N_STAGES] = {};  // algorithmic bytes of one full launch (RHS, refinement)
    double mode_bytes[GEMV_NMODES] = {};        // algorithmic bytes of one GEMV launch, FP64 matrices
    double mode_bytes32[GEMV_NMODES] = {};      // same with FP32 matrices
    double mode_bytes_sym[GEMV_NMODES] = {};    // same for the packed symmetric FP32 operator: its distinct elements
    double mode_tile_bytes_sym[GEMV_NMODES] = {};   // bytes the packed kernel streams (whole tiles, padding included)

    int fail(int code, const std::string& msg) {
        err = msg;
        return code;
    }
};

constexpr int kNB = 32;              // pivot block of the dense elimination
// default tile shapes per mode (LOCAL, SCHUR_C, CORNER, RECOVER, COARSE, SCHUR_G, COUPLED):
// rows per CTA, and lanes per row for FP32 and FP64 (8 lanes for FP64 keeps the
// FP64 reduction adds off GB300's narrow FP64 pipe)
constexpr int kRowsPerMode[GEMV_NMODES] = {32, 32, 64, 32, 8, 64, 64};
constexpr int kLprF32[GEMV_NMODES] = {32, 16, 8, 16, 32, 16, 16};
constexpr int kLprF64[GEMV_NMODES] = {8, 8, 8, 8, 32, 8, 8};
constexpr int kMinRowsPerTask = 8;    // smallest rows per CTA of any default or candidate tile (sets task capacity)
constexpr int kMaxPartials = 4096;   // block partials of the grid reductions

// setup.cpp
int dd_build_host(dd_handle* h, const dd_mesh* mesh, const int32_t* part, int32_t n_sub);
int dd_locate_probes(dd_handle* h, int32_t n, const double* xyz);
void build_tasks(const dd_handle* h, int mode, int rows, std::vector<GemvTask>& out);
int dd_build_beam(dd_handle* h, const dd_beam* beam);
size_t dd_workspace_layout(dd_handle* h, bool assign);

// kernels.cu launchers (return a cudaError_t value; 0 = success)
int launch_csr_combine(const dd_handle* h, double ca, void* stream);
int launch_dense_assemble(const dd_handle* h, void* stream);
int launch_sweep(const dd_handle* h, bool coarse, int k0, void* stream);
int launch_coarse_assemble(const dd_handle* h, void* stream);
int launch_factor_finish(const dd_handle* h, void* stream);
int launch_rhs(const dd_handle* h, const double* e_n, const double* src, double src_sign, double dt, void* stream);
int launch_grad_eps(const dd_handle* h, const double* mu, const double* e_k, const double* e_km1, const double* e_km2,
                    double* grad_eps, void* stream);
int launch_dot_sub(const dd_handle* h, const double* a, const double* b, double scale, double* acc, void* stream);
int launch_probe_objective(const dd_handle* h, const double* e, double weight, double* J, void* stream);
int launch_scale_copy(const dd_handle* h, double* dst, const double* src, double scale, void* stream);
int launch_assemble_mass(const dd_handle* h, const double* eps, void* stream);
void build_eps_map(const dd_handle* h, std::vector<int64_t>& ptr, std::vector<int32_t>& idx);
int launch_probe_seed(const dd_handle* h, const double* e, double weight, double* seed, void* stream);
int launch_residual_local(const dd_handle* h, void* stream);
int launch_assembled_norm(const dd_handle* h, int set_b, float* bf, void* stream);
int launch_gemv(const dd_handle* h, int mode, int prec, XSrc xs, GemvOut go, bool check_done, void* stream,
                const int32_t* skip_flag = nullptr);
int launch_iface_rhs(const dd_handle* h, float* fCf, void* stream);
int launch_corner_gather(const dd_handle* h, const double* w, const float* wf, const double* add, double* uC, float* uCf,
                         bool check_done, void* stream);
int launch_jump(const dd_handle* h, const double* w, const float* wf, const double* base, double sign, double* out,
                void* stream);
int launch_pcg_init(const dd_handle* h, int have_q, double tol, const float* wf, float* zf, float* pf,
                    unsigned long long cond, int adaptive, void* stream);
int launch_step_begin(const dd_handle* h, void* stream);
int launch_extrapolate(const dd_handle* h, bool f32, void* stream);
int launch_solve_end(const dd_handle* h, void* stream);
int launch_refine_cond(const dd_handle* h, unsigned long long cond, void* stream);
int launch_pcg_alpha(const dd_handle* h, const float* wf, float* pf, void* stream);
int launch_pcg_update(const dd_handle* h, float* zf, float* lamf, unsigned long long cond, void* stream);
int launch_writeback(const dd_handle* h, const double* e_n, const double* e_nm1, double* delta_k, double* delta_acc,
                     int first, double* e_np1, void* stream);
int launch_advance(const dd_handle* h, const double* e_n, const double* e_nm1, const double* delta, double* e_np1,
                   void* stream);
int launch_probe(const dd_handle* h, const double* e, double* out, void* stream);
int launch_pic_move(const dd_handle* h, double t_n, double dt, const double* e_n, double* dep, void* stream);
int launch_pic_source(const dd_handle* h, const double* dep_new, const double* dep_old, void* stream);
int launch_faraday(const dd_handle* h, const double* e_np1, const double* e_n, double dt, void* stream);

// symgemv.cu: packed symmetric FP32 storage and its GEMV
void build_sym(dd_handle* h);
void sym_ranges(dd_handle* h, int mode, int cl);
int launch_sym_pack(const dd_handle* h, void* stream);
int launch_symgemv(const dd_handle* h, int mode, XSrc xs, GemvOut go, const int32_t* skip, void* stream);
size_t sym_smem_bytes(const dd_handle* h);
// Packed kinds in use: the recovery reads the packed tiles only for an ensemble (its I x [Gamma|c]
// rectangle has no symmetric twin, so one problem gains almost nothing; an ensemble shares the reads).
bool sym_active(const dd_handle* h, int mode);
// ozaki.cu
size_t oz_slice_elems(int nm, int nmax);
int launch_oz_update(const MatDesc* mats, double* M, int nm, int nmax, int k0, uint16_t* slices, int32_t* exps,
                     int32_t* err, void* stream);
// tensor.cu
void build_tc(dd_handle* h);
int launch_tc_pack(const dd_handle* h, void* stream);
int launch_tc_gemv(const dd_handle* h, int mode, XSrc xs, GemvOut go, const int32_t* skip, void* stream);
bool tc_available(const dd_handle* h, int mode);
size_t sym_smem_bytes_nr(const dd_handle* h, int nr);
int sym_members_per_cta(const dd_handle* h, int mode);

// gmres.cu: coupled-system GMRES (u = [lambda; x_c])
int launch_corner_diag(const dd_handle* h, void* stream);
// wf: FP32 GEMV output (DD_MIXED) or null; zuf: FP32 operator input to write (DD_MIXED) or null
int launch_gm_init(const dd_handle* h, double tol, int max_it, int m, int adaptive, unsigned long long cond_outer,
                   void* stream);
int launch_gm_start(const dd_handle* h, const UView& U, int have_q, const float* wf, unsigned long long cond_inner,
                    void* stream);
int launch_gm_normalize(const dd_handle* h, const UView& U, float* zuf, void* stream);
int launch_gm_pass(const dd_handle* h, const UView& U, int phase, const float* wf, const float* zuf,
                   unsigned long long cond_inner, void* stream);
int launch_gm_update(const dd_handle* h, const UView& U, unsigned long long cond_outer, void* stream);
int launch_gm_combine(const dd_handle* h, const UView& U, const double* in, double* out, void* stream);
int launch_dp2_rhs(const dd_handle* h, const UView& U, void* stream);
int launch_robin_add(const dd_handle* h, double alpha, void* stream);

// GEMV x-source kinds (see kernels.cu)
enum : int { X_FLAT = 0, X_LAMBDA = 1, X_PCG = 2, X_CORNER = 3, X_RECOVER = 4, X_COARSE = 5, X_PCG_CV = 6,
             X_LAMBDA_CV = 7, X_SIDE_CP = 8 };

constexpr int kMaxProbes = 256;
