// C ABI entry points (include/dd.h): handle lifecycle, workspace layout, the
// factorisation sequence and the per-step MFETI-DP1 solve (Sec. III-A).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <chrono>
#include <fstream>
#include <map>
#include <new>
#include <sstream>

#include "dd_internal.h"

namespace {

int cuda_fail(dd_handle* h, int code, const char* what) {
    h->err = std::string(what) + ": " + cudaGetErrorString((cudaError_t)code);
    return DD_ERR_CUDA;
}

void drop_graphs(dd_handle* h) {
    for (int k = 0; k < 3; ++k)
        if (h->gexec[k]) {
            cudaGraphExecDestroy((cudaGraphExec_t)h->gexec[k]);
            h->gexec[k] = nullptr;
        }
}

#define CK(h, expr, what)                                     \
    do {                                                      \
        int rc_ = (expr);                                     \
        if (rc_ != 0) return cuda_fail((h), rc_, (what));     \
    } while (0)

dd_params default_params() {
    dd_params p;
    p.precision = DD_FP64;
    p.tol = 1e-12;
    p.max_it = 500;
    p.precond = 1;
    p.warm_start = 1;
    p.refine_tol = 1e-12;
    p.max_refine = 4;
    p.chunk = 8;
    p.use_graph = 0;
    p.solver = DD_SOLVER_SCHUR_CG;
    p.restart = 20;
    p.sym_fp32 = 1;
    p.scheme = DD_SCHEME_DP1;
    p.robin_alpha = 0.0;
    p.members = 1;
    p.factor_mode = DD_FACTOR_TENSOR;
    return p;
}

int check_params(dd_handle* h, const dd_params& p) {
    if (p.precision != DD_FP64 && p.precision != DD_MIXED) return h->fail(DD_ERR_ARG, "precision must be DD_FP64 or DD_MIXED");
    if (!(p.tol > 0.0) || p.max_it < 1 || p.chunk < 1 || p.max_refine < 1 || !(p.refine_tol > 0.0))
        return h->fail(DD_ERR_ARG, "tol, refine_tol must be > 0 and max_it, chunk, max_refine >= 1");
    if (p.sym_fp32 != 0 && p.sym_fp32 != 1) return h->fail(DD_ERR_ARG, "sym_fp32 must be 0 or 1");
    if (p.warm_start < 0 || p.warm_start > 2) return h->fail(DD_ERR_ARG, "warm_start must be 0, 1 or 2");
    if (p.scheme != DD_SCHEME_DP1 && p.scheme != DD_SCHEME_DP2)
        return h->fail(DD_ERR_ARG, "scheme must be DD_SCHEME_DP1 or DD_SCHEME_DP2");
    if (p.scheme == DD_SCHEME_DP2 && p.solver != DD_SOLVER_COUPLED_GMRES)
        return h->fail(DD_ERR_ARG, "MFETI-DP2 is solved by the coupled GMRES (its system is not symmetric)");
    if (!std::isfinite(p.robin_alpha)) return h->fail(DD_ERR_ARG, "robin_alpha must be finite");
    if (p.solver != DD_SOLVER_SCHUR_CG && p.solver != DD_SOLVER_COUPLED_GMRES)
        return h->fail(DD_ERR_ARG, "solver must be DD_SOLVER_SCHUR_CG or DD_SOLVER_COUPLED_GMRES");
    if (p.solver == DD_SOLVER_COUPLED_GMRES) {
        if (p.restart < 1 || p.restart > kMaxRestart) return h->fail(DD_ERR_ARG, "restart must be in 1..DD_MAX_RESTART");
    }
    if (p.factor_mode != DD_FACTOR_FP64 && p.factor_mode != DD_FACTOR_TENSOR)
        return h->fail(DD_ERR_ARG, "factor_mode must be DD_FACTOR_FP64 or DD_FACTOR_TENSOR");
    if (p.members < 1 || p.members > kMaxMembers) return h->fail(DD_ERR_ARG, "members must be in 1..64");
    if (p.members > 1 && p.solver != DD_SOLVER_COUPLED_GMRES)
        return h->fail(DD_ERR_ARG, "an ensemble (members > 1) is solved by the coupled GMRES");
    if (h->members > 0 && p.members != h->members)
        return h->fail(DD_ERR_ARG, "members is fixed by dd_setup");
    return DD_OK;
}

// ---- profiling: events around every launch while enabled --------------------
enum Stage { ST_RHS = 0, ST_LOCAL = 1, ST_SCHUR = 2, ST_COARSE = 3, ST_CORNER = 4, ST_RECOVER = 5, ST_VEC = 6,
             ST_REFINE = 7, ST_FACTOR = 8 };

cudaEvent_t grab_event(dd_handle* h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back((void*)e);
    }
    return (cudaEvent_t)h->ev_pool[h->ev_used++];
}

// Counts `nk` kernel launches of `stage`; a positive `bytes` marks them as one
// full-work launch with that many algorithmic bytes.
struct Prof {
    dd_handle* h;
    int stage;
    cudaStream_t s;
    size_t i0 = 0;
    bool on;
    Prof(dd_handle* h_, int stage_, cudaStream_t s_, int nk = 1, double bytes = 0.0)
        : h(h_), stage(stage_), s(s_), on(h_->prof_on) {
        h->launches[stage] += nk;
        h->total_launches += nk;
        if (bytes > 0.0) {
            h->work[stage] += 1;
            h->work_bytes[stage] += bytes;
        }
        if (on) {
            i0 = h->ev_used;
            cudaEvent_t a = grab_event(h);
            grab_event(h);
            if (a) cudaEventRecord(a, s);
        }
    }
    ~Prof() {
        if (on && i0 + 1 < h->ev_used) {
            cudaEventRecord((cudaEvent_t)h->ev_pool[i0 + 1], s);
            h->prof_recs.push_back({stage, i0});
        }
    }
};

// algorithmic bytes of one full GEMV launch of `mode` at precision `prec`
double mb(const dd_handle* h, int mode, int prec) {
    if (prec != DD_MIXED) return h->mode_bytes[mode];
    if (h->prm.sym_fp32 && h->sym_ok && sym_active(h, mode) && h->mode_bytes_sym[mode] > 0.0) return h->mode_bytes_sym[mode];
    return h->mode_bytes32[mode];
}

// Algorithmic bytes of one full launch: matrix elements read at the launch's
// precision plus the vectors read and written once.
void compute_stage_bytes(dd_handle* h) {
    const double nl = (double)h->sub_ptr.back(), nd = (double)h->n_dof, nnz = (double)h->row_ptr.back();
    const double nc = (double)h->corner_dof.size();
    for (int k = 0; k < DD_N_STAGES; ++k) h->bytes_per_launch[k] = 0.0;
    // RHS: S values + column ids, row pointers, e^n, source, b
    h->bytes_per_launch[ST_RHS] = nnz * 12.0 + nl * (8.0 + 8.0 + 5.0) + 2.0 * nd * 8.0;
    for (int mode = 0; mode < GEMV_NMODES; ++mode) {
        double elems = 0.0, vec = 0.0;
        if (mode == GEMV_COARSE) {
            elems = nc * nc;
            vec = 2.0 * nc * 8.0;
        } else {
            for (const MatDesc& md : h->mats) {
                int r0, r1, c0, c1;
                switch (mode) {
                    case GEMV_LOCAL: r0 = 0; r1 = md.ns; c0 = 0; c1 = md.nr; break;
                    case GEMV_SCHUR_C: r0 = md.nr; r1 = md.ns; c0 = md.nI; c1 = md.nr; break;
                    case GEMV_CORNER: r0 = md.nI; r1 = md.nr; c0 = md.nr; c1 = md.ns; break;
                    case GEMV_SCHUR_G: r0 = md.nI; r1 = md.nr; c0 = md.nI; c1 = md.ns; break;
                    case GEMV_COUPLED: r0 = md.nI; r1 = md.ns; c0 = md.nI; c1 = md.ns; break;
                    default: r0 = 0; r1 = md.nr; c0 = md.nI; c1 = md.ns; break;
                }
                elems += (double)(r1 - r0) * (double)(c1 - c0);
                const bool acc = mode == GEMV_RECOVER;
                vec += (double)(c1 - c0) * 8.0 + (double)(r1 - r0) * 8.0 * (acc ? 2.0 : 1.0);
            }
        }
        h->mode_bytes[mode] = elems * 8.0 + vec;
        h->mode_bytes32[mode] = elems * 4.0 + vec;
    }
    // FP64 residual b -= A delta (A values + ids + b) and the assembled norm
    h->bytes_per_launch[ST_REFINE] = nnz * 12.0 + nl * 24.0 + nd * 8.0;
}

struct Layout {
    size_t off = 0;
    char* base = nullptr;
    template <typename T>
    void take(T*& ptr, size_t count) {
        off = (off + 255) / 256 * 256;
        ptr = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += sizeof(T) * std::max<size_t>(count, 1);
    }
};

// Task lists must fit the capacity reserved in the workspace layout.
int upload_tasks(dd_handle* h, int p, int m, cudaStream_t s) {
    if (h->tasks[p][m].size() > h->task_cap[m]) return h->fail(DD_ERR_STATE, "GEMV task list exceeds its capacity");
    if (h->tasks[p][m].empty()) return DD_OK;
    const int rc = (int)cudaMemcpyAsync(h->d.tasks[p][m], h->tasks[p][m].data(), sizeof(GemvTask) * h->tasks[p][m].size(),
                                        cudaMemcpyHostToDevice, s);
    return rc ? DD_ERR_CUDA : DD_OK;
}

template <typename T>
int upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (src.empty()) return 0;
    return (int)cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s);
}

}  // namespace

size_t dd_workspace_layout(dd_handle* h, bool assign) {
    Layout L;
    L.base = assign ? h->ws : nullptr;
    DevPtrs d;
    const size_t nl = (size_t)h->sub_ptr.back(), nd = (size_t)h->n_dof, nm = h->mult_dof.size(),
                 nc = h->corner_dof.size(), nnz = (size_t)h->row_ptr.back();
    L.take(d.mats, h->mats.size());
    L.take(d.coarse_desc, 1);
    L.take(d.slot_mult, nl);
    L.take(d.slot_corner, nl);
    L.take(d.slot_dof, nl);
    L.take(d.slot_sub, nl);
    L.take(d.slot_own, nl);
    L.take(d.mult_slot, 2 * nm);
    L.take(d.corner_ptr, nc + 1);
    L.take(d.corner_slot, h->corner_slot.size());
    L.take(d.slot_upos, h->slot_upos.size());
    L.take(d.owner_slot, nd);
    L.take(d.copy_ptr, nd + 1);
    L.take(d.copy_slot, nl);
    L.take(d.row_ptr, nl + 1);
    L.take(d.col_loc, nnz);
    L.take(d.col_dof, nnz);
    L.take(d.Tval, nnz);
    L.take(d.Sval, nnz);
    L.take(d.Aval, nnz);
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < GEMV_NMODES; ++m) L.take(d.tasks[p][m], h->task_cap[m]);
    L.take(d.probe_dof, 6 * kMaxProbes);
    L.take(d.probe_w, 18 * kMaxProbes);
    L.take(d.M64, (size_t)h->dense_elems);
    L.take(d.M32, (size_t)h->dense_elems);
    L.take(d.Msym, (size_t)h->sym_elems);
    L.take(d.symd, (size_t)h->n_sub);
    L.take(d.sym_dir, h->sym_dir.size());
    L.take(d.Mtc, (size_t)h->tc_elems);
    for (int k = 0; k < kTcKinds; ++k) L.take(d.tcd[k], h->tcd[k].size());
    L.take(d.tc_dir, h->tc_dir.size());
    for (int m = 0; m < GEMV_NMODES; ++m) {
        int rm, cm;
        if (sym_masks(m, &rm, &cm)) {
            L.take(d.sym_rng[m], (size_t)h->n_sub * kSymCLMax * kSymRng);
            L.take(d.sym_tl[m], std::max<size_t>(1, h->sym_tl[m].size()));
        }
    }
    L.take(d.K64, nc * (size_t)h->ldc);
    L.take(d.K32, nc * (size_t)h->ldc);
    L.take(d.Pinv, (size_t)(h->n_sub + 1) * kNB * kNB);
    {   // slices and exponents of one pivot block for the tensor-core trailing update (local or coarse)
        const int nloc = std::max(1, h->n_sub_real), ncor = (int)nc;
        L.take(d.oz_slices, std::max(oz_slice_elems(nloc, h->max_ns), oz_slice_elems(1, ncor)));
        L.take(d.oz_exps, 2 * std::max((size_t)nloc * h->max_ns, (size_t)ncor));
    }
    L.take(d.dinv, nm);
    for (int k = 0; k < 3; ++k) L.take(d.e[k], nd);
    for (int k = 0; k < 3; ++k) L.take(d.mu[k], nd);
    L.take(d.lam_adj, nm);
    L.take(d.lam2, nm);
    L.take(d.lam2f, nm);
    L.take(d.lam2_adj, nm);
    L.take(d.lam2f_adj, nm);
    L.take(d.lam2_scratch, nm);
    L.take(d.lam2f_scratch, nm);
    L.take(d.g2, nm);
    L.take(d.mt_ptr, nm + 1);
    L.take(d.mt_col, h->mt_col.size());
    L.take(d.mt_val, h->mt_val.size());
    L.take(d.lamf_adj, nm);
    L.take(d.lam_prev, nm);
    L.take(d.lam_prev_adj, nm);
    L.take(d.xC_prev, nc);
    L.take(d.xC_prev_adj, nc);
    L.take(d.lam2_prev, nm);
    L.take(d.lam2_prev_adj, nm);
    if (h->members <= 1) {   // dd_set_eps map (filled on its first call)
        L.take(d.eps_ptr, nnz + 1);
        L.take(d.eps_idx, (size_t)h->eps_contrib);
    }
    L.take(d.tet_dof, 6 * (size_t)h->n_tets);
    L.take(d.That, 36 * (size_t)h->n_tets);
    {
        const size_t np = (size_t)h->n_particles, nt = h->n_particles ? (size_t)h->n_tets : 0,
                     nfc = h->n_particles ? (size_t)h->n_faces : 0, ndp = h->n_particles ? nd : 0;
        L.take(d.px, 3 * np);
        L.take(d.pv, 3 * np);
        L.take(d.pt, np);
        L.take(d.ptet, np);
        L.take(d.pstat, np);
        L.take(d.tets_dev, 4 * nt);
        L.take(d.tgrad, 12 * nt);
        L.take(d.tx0, 3 * nt);
        L.take(d.tface, 4 * nt);
        L.take(d.tnbr, 4 * nt);
        L.take(d.face_nodes, 3 * nfc);
        L.take(d.face_edge, 3 * nfc);
        L.take(d.bflux, nfc);
        L.take(d.dep[0], ndp);
        L.take(d.dep[1], ndp);
        L.take(d.Gcum, ndp);
        L.take(d.d2g_pic, ndp);
        L.take(d.pic_err, 4);
    }
    L.take(d.b, nl);
    L.take(d.y, nl);
    L.take(d.w, nl);
    L.take(d.x, nl);
    L.take(d.bf, nl);
    L.take(d.wf, nl);
    L.take(d.zf, nm);
    L.take(d.pf, nm);
    L.take(d.lamf, nm);
    L.take(d.lamf_scratch, nm);
    L.take(d.fCf, nc);
    L.take(d.uCf, nc);
    L.take(d.vCf, nc);
    L.take(d.xCf, nc);
    L.take(d.lam, nm);
    L.take(d.g, nm);
    L.take(d.r, nm);
    L.take(d.p, nm);
    L.take(d.q, nm);
    L.take(d.z, nm);
    L.take(d.lam_scratch, nm);
    L.take(d.fC, nc);
    L.take(d.uC, nc);
    L.take(d.vC, nc);
    L.take(d.xC, nc);
    L.take(d.xC_adj, nc);
    L.take(d.xCf_adj, nc);
    L.take(d.xC_scratch, nc);
    L.take(d.xCf_scratch, nc);
    L.take(d.dinvC, nc);
    {
        const int64_t nu = (int64_t)(2 * nm + nc);   // MFETI-DP2 has two multiplier blocks
        h->gm_ldv = (nu + 31) / 32 * 32;
        h->gm_blocks = (int32_t)std::max<int64_t>(1, (nu + kGmChunk - 1) / kGmChunk);
        L.take(d.Vk, (size_t)(kMaxRestart + 1) * (size_t)h->gm_ldv);
        L.take(d.tu, (size_t)nu);
        L.take(d.zu, (size_t)nu);
        L.take(d.zuf, (size_t)nu);
        L.take(d.gs, 1);
        L.take(d.gpart, (size_t)(kMaxRestart + 1) * (size_t)h->gm_blocks);
    }
    L.take(d.delta, nd);
    L.take(d.delta_k, nd);
    L.take(d.src_in, nd);
    L.take(d.sc, 1);
    L.take(d.partials, 3 * kMaxPartials);
    L.take(d.status, 4);
    if (assign) h->d = d;
    return (L.off + 255) / 256 * 256;
}

namespace {

// True when a bounded device wait gave up since the word was last cleared (synchronises).
bool wait_err_set(dd_handle* h, cudaStream_t s) {
    int32_t v = 0;
    if (cudaMemcpyAsync(&v, &h->d.sc->wait_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    return v != 0;
}

// Read the CG scalars back (synchronises the stream).
int read_scalars(dd_handle* h, PcgScalars* out, cudaStream_t s) {
    int rc = (int)cudaMemcpyAsync(out, h->d.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s);
    if (rc) return rc;
    return (int)cudaStreamSynchronize(s);
}

// w <- interface operator pieces for x-source (kind, v, v2):
// rows Gamma: S_Gamma z + Psi_Gamma K~cc^-1 Psi^T z ; then the caller jumps w.
// Vector set of one precision: DD_MIXED GEMVs read/write FP32 shadows.
struct Vecs {
    bool f32;
    float* wf;      // interface-operator output (FP32) or null (FP64 path uses d.w)
    float* zf;
    float* pf;
    float* lamf;
    float* fCf;
    float* uCf;
    float* vCf;
    float* xCf;
    float* bf;
};

Vecs vecs(dd_handle* h, int prec) {
    if (prec != DD_MIXED) return Vecs{false, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const DevPtrs& d = h->d;
    return Vecs{true, d.wf, d.zf, d.pf, d.lamf, d.fCf, d.uCf, d.vCf, d.xCf, d.bf};
}

XSrc xsrc(int kind, const double* v, const double* v2, const float* vf, const float* v2f,
          const double* v3 = nullptr, const float* v3f = nullptr) {
    XSrc x{};
    x.kind = kind;
    x.v = v;
    x.v2 = v2;
    x.v3 = v3;
    x.vf = vf;
    x.v2f = v2f;
    x.v3f = v3f;
    return x;
}

// FP64 path writes the double output; the FP32 path writes the FP32 output
// (out32) and, where a double consumer exists, the double output too.
GemvOut gout(double* out, const double* base, float* out32, const float* base32, double alpha) {
    return GemvOut{out, base, out32, base32, alpha};
}

// Output of the coupled operator's GEMV, in the order the GMRES combine reads:
// both sides of every multiplier, then the corner copies.
GemvOut gout_coupled(const dd_handle* h, double* out, float* out32) {
    GemvOut go = gout(out, nullptr, out32, nullptr, 1.0);
    go.pos = h->d.slot_upos;
    return go;
}

// w <- interface operator pieces for x-source (kind, v, v2) of Eq. f1schur:
// rows Gamma: S_Gamma z + Psi_Gamma K~cc^-1 Psi^T z (the caller jumps w).
// Inside the CG loop (check_done) launches after convergence exit early; their
// full-work count is added by dd_solve once the iteration count is known.
int apply_schur_w(dd_handle* h, int prec, int kind, const double* v, const double* v2, const float* vf,
                  const float* v2f, bool check_done, cudaStream_t s) {
    const Vecs V = vecs(h, prec);
    const double full = check_done ? 0.0 : 1.0;   // CG-loop launches are counted by count_cg_work
    int rc;
    const int kind_cv = kind == X_PCG ? X_PCG_CV : X_LAMBDA_CV;
    if (!h->corner_dof.empty()) {
        // u_s = A_cr A_rr^-1 B_r^T z (corner rows), K~cc^-1 sum_s B_c^T u_s
        {
            Prof P(h, ST_CORNER, s, 1, full * mb(h, GEMV_SCHUR_C, prec));
            rc = launch_gemv(h, GEMV_SCHUR_C, prec, xsrc(kind, v, v2, vf, v2f),
                             V.f32 ? gout(nullptr, nullptr, V.wf, nullptr, 1.0) : gout(h->d.w, nullptr, nullptr, nullptr, 1.0),
                             check_done, s);
        }
        if (rc) return rc;
        {
            Prof P(h, ST_VEC, s, 1);
            rc = launch_corner_gather(h, h->d.w, V.wf, nullptr, h->d.uC, V.uCf, check_done, s);
        }
        if (rc) return rc;
        {
            Prof P(h, ST_COARSE, s, 1, full * mb(h, GEMV_COARSE, prec));
            rc = launch_gemv(h, GEMV_COARSE, prec, xsrc(X_FLAT, h->d.uC, nullptr, V.uCf, nullptr),
                             V.f32 ? gout(nullptr, nullptr, V.vCf, nullptr, 1.0) : gout(h->d.vC, nullptr, nullptr, nullptr, 1.0),
                             check_done, s);
        }
        if (rc) return rc;
    }
    // interface rows over [Gamma | c] columns with x = [B_r^T z ; -v]:
    // A_rr^-1 B_r^T z + A_rr^-1 A_rc B_c K~cc^-1 (...) in one pass (M[Gamma, c] = -A_rr^-1 A_rc)
    Prof P(h, ST_SCHUR, s, 1, full * mb(h, GEMV_SCHUR_G, prec));
    return launch_gemv(h, GEMV_SCHUR_G, prec, xsrc(kind_cv, v, v2, vf, v2f, h->d.vC, V.vCf),
                       V.f32 ? gout(nullptr, nullptr, V.wf, nullptr, 1.0) : gout(h->d.w, nullptr, nullptr, nullptr, 1.0),
                       check_done, s);
}

// Adds n full-work CG iterations to the stage counters once the count is known.
void count_cg_work(dd_handle* h, int prec, int n) {
    const bool c = !h->corner_dof.empty();
    h->work[ST_SCHUR] += n;
    h->work_bytes[ST_SCHUR] += n * mb(h, GEMV_SCHUR_G, prec);
    if (c) {
        h->work[ST_CORNER] += n;
        h->work_bytes[ST_CORNER] += n * mb(h, GEMV_SCHUR_C, prec);
        h->work[ST_COARSE] += n;
        h->work_bytes[ST_COARSE] += n * mb(h, GEMV_COARSE, prec);
    }
}

// Solve the torn system A x = b for the local right-hand sides in d.b
// (subassembled; DD_MIXED also needs the FP32 shadow d.bf), leaving x in d.x
// (r slots) and x_c in d.xC.  Returns a DD status; iteration count and the
// final relative interface residual in *it_out / *res_out.
// Graph capture helpers: add a conditional node at the current end of stream s's
// capture and return its body graph; later work captured on s depends on it.
int add_conditional(dd_handle* h, cudaStream_t s, cudaGraphConditionalHandle hc, cudaGraphConditionalNodeType type,
                    cudaGraph_t* body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(h, (int)cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd), "capture info");
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(h, (int)cudaGraphAddNode(&node, g, deps, nullptr, nd, &p), "add conditional node");
    *body = p.conditional.phGraph_out[0];
    CK(h, (int)cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies), "deps");
    return DD_OK;
}

int create_handle(dd_handle* h, cudaStream_t s, cudaGraphConditionalHandle* hc) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    CK(h, (int)cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
    CK(h, (int)cudaGraphConditionalHandleCreate(hc, g, 0, cudaGraphCondAssignDefault), "conditional handle");
    return DD_OK;
}

cudaStream_t capture_stream(dd_handle* h, int depth) {
    if (depth < 0 || depth >= (int)(sizeof(h->gstream) / sizeof(h->gstream[0]))) return nullptr;
    if (!h->gstream[depth]) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        h->gstream[depth] = (void*)cs;
    }
    return (cudaStream_t)h->gstream[depth];
}

// Read the control words of the coupled GMRES back (synchronises the stream).
int read_gm(dd_handle* h, GmresScalars* out, cudaStream_t s) {
    int rc = (int)cudaMemcpyAsync(out, h->d.gs, kGmCtrlBytes, cudaMemcpyDeviceToHost, s);
    if (rc) return rc;
    return (int)cudaStreamSynchronize(s);
}

// Coupled solve of Eqs. F1lr + F1uc by restarted GMRES with right diagonal
// preconditioning: u = [lambda; x_c] from b = [d_r; f~_c] (in d.g, d.fC), left
// in d.lam and d.xC (DD_MIXED: FP32 GEMVs on FP32 shadows, FP64 Krylov vectors
// and least-squares problem).  Eager mode polls the control words after every
// cycle start and every `chunk` Arnoldi steps; graph mode captures the restart
// cycles as a conditional WHILE node whose body holds the cycle start, a nested
// WHILE node over the Arnoldi steps and the update of u.
// The coupled solve's unknown in blocks (DP1: [lambda; x_c]; DP2: [lambda^(s1);
// lambda^(s2); x_c]), right-hand side [g; (g2;) fC], diagonal preconditioner.
UView uview(const dd_handle* h, int prec) {
    const DevPtrs& d = h->d;
    const bool f32 = prec == DD_MIXED;
    const bool dp2 = h->factored_scheme == DD_SCHEME_DP2;
    const bool pc = h->prm.precond != 0;
    UView U;
    U.n1 = (int64_t)h->mult_dof.size();
    U.n2 = dp2 ? U.n1 : 0;
    U.nc = (int64_t)h->corner_dof.size();
    U.b1 = d.g;
    U.b2 = dp2 ? d.g2 : nullptr;
    U.bc = d.fC;
    U.x1 = d.lam;
    U.x2 = dp2 ? d.lam2 : nullptr;
    U.xc = d.xC;
    U.x1f = f32 ? d.lamf : nullptr;
    U.x2f = (f32 && dp2) ? d.lam2f : nullptr;
    U.xcf = f32 ? d.xCf : nullptr;
    U.d1 = (pc && !dp2) ? d.dinv : nullptr;   // DP2: the multiplier blocks have unit diagonal
    U.dc = pc ? d.dinvC : nullptr;
    U.ms = d.mult_slot;
    U.cp = d.corner_ptr;
    U.cs = d.corner_slot;
    if (dp2) {
        U.mtp = d.mt_ptr;
        U.mtc = d.mt_col;
        U.mtv = d.mt_val;
        U.two_alpha = 2.0 * h->factored_alpha;
    }
    return U;
}

int gmres_solve(dd_handle* h, int prec, double tol, bool warm, int* it_out, double* res_out, cudaStream_t s,
                int depth, int adaptive) {
    const size_t nm = h->mult_dof.size(), nc = h->corner_dof.size();
    *it_out = 0;
    *res_out = 0.0;
    if (nm + nc == 0) return DD_OK;
    const Vecs V = vecs(h, prec);
    const UView U = uview(h, prec);
    const bool dp2 = U.n2 > 0;
    const bool use_warm = warm && (h->lam_valid || h->capturing);
    if (!use_warm) {
        if (nm) CK(h, (int)cudaMemsetAsync(h->d.lam, 0, sizeof(double) * nm, s), "memset");
        if (nc) CK(h, (int)cudaMemsetAsync(h->d.xC, 0, sizeof(double) * nc, s), "memset");
        if (V.f32 && nm) CK(h, (int)cudaMemsetAsync(V.lamf, 0, sizeof(float) * nm, s), "memset");
        if (V.f32 && nc) CK(h, (int)cudaMemsetAsync(V.xCf, 0, sizeof(float) * nc, s), "memset");
        if (dp2) CK(h, (int)cudaMemsetAsync(h->d.lam2, 0, sizeof(double) * nm, s), "memset");
        if (dp2 && V.f32) CK(h, (int)cudaMemsetAsync(h->d.lam2f, 0, sizeof(float) * nm, s), "memset");
    }
    float* zuf = V.f32 ? h->d.zuf : nullptr;
    // DP1: x = [B_r^T u_l ; -u_c] over the [Gamma | c] columns of every local matrix;
    // DP2: x = [lambda^(s) (the subdomain's own side) ; +u_c]
    const int64_t o2 = (int64_t)(dp2 ? 2 * nm : nm);   // offset of the corner block in u
    const XSrc xs_x = dp2 ? xsrc(X_SIDE_CP, h->d.lam, h->d.lam2, V.lamf, V.f32 ? h->d.lam2f : nullptr, h->d.xC, V.xCf)
                          : xsrc(X_LAMBDA_CV, h->d.lam, nullptr, V.lamf, nullptr, h->d.xC, V.xCf);
    const XSrc xs_z = dp2 ? xsrc(X_SIDE_CP, h->d.zu, h->d.zu + nm, zuf, zuf ? zuf + nm : nullptr, h->d.zu + o2,
                                 zuf ? zuf + o2 : nullptr)
                          : xsrc(X_LAMBDA_CV, h->d.zu, nullptr, zuf, nullptr, h->d.zu + nm, zuf ? zuf + nm : nullptr);
    const GemvOut go = V.f32 ? gout_coupled(h, nullptr, V.wf) : gout_coupled(h, h->d.w, nullptr);
    const double mbc = mb(h, GEMV_COUPLED, prec);
    const int32_t* skip = &h->d.gs->skip;
    auto cycle_start = [&](cudaStream_t st, int have_q, unsigned long long cond_inner) -> int {
        if (have_q) {
            Prof P(h, ST_SCHUR, st, 1, mbc);
            CK(h, launch_gemv(h, GEMV_COUPLED, prec, xs_x, go, false, st), "coupled operator on x");
        }
        Prof P(h, ST_VEC, st, 2);
        CK(h, launch_gm_start(h, U, have_q, V.wf, cond_inner, st), "gmres start");
        CK(h, launch_gm_normalize(h, U, zuf, st), "gmres normalize");
        return DD_OK;
    };
    // one Arnoldi step; its full-work count is added once the step count is known
    auto arnoldi = [&](cudaStream_t st, unsigned long long cond_inner) -> int {
        {
            Prof P(h, ST_SCHUR, st, 1);
            CK(h, launch_gemv(h, GEMV_COUPLED, prec, xs_z, go, false, st, skip), "coupled operator");
        }
        Prof P(h, ST_VEC, st, 3);
        CK(h, launch_gm_pass(h, U, 0, V.wf, zuf, 0ull, st), "gmres pass 0");
        CK(h, launch_gm_pass(h, U, 1, V.wf, zuf, cond_inner, st), "gmres pass 1");
        CK(h, launch_gm_normalize(h, U, zuf, st), "gmres normalize");
        return DD_OK;
    };
    if (h->capturing) {
        cudaGraphConditionalHandle ho;
        int rc = create_handle(h, s, &ho);
        if (rc) return rc;
        {
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_gm_init(h, tol, h->prm.max_it, h->prm.restart, adaptive, (unsigned long long)ho, s),
               "gmres init");
        }
        cudaGraph_t body;
        rc = add_conditional(h, s, ho, cudaGraphCondTypeWhile, &body);
        if (rc) return rc;
        cudaStream_t bo = capture_stream(h, depth + 1);
        if (!bo) return h->fail(DD_ERR_CUDA, "capture stream");
        CK(h, (int)cudaStreamBeginCaptureToGraph(bo, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
           "capture cycle");
        const int64_t l0 = h->total_launches;
        cudaGraphConditionalHandle hi;
        int brc = create_handle(h, bo, &hi);
        if (!brc) brc = cycle_start(bo, 1, (unsigned long long)hi);
        cudaGraph_t ibody;
        if (!brc) brc = add_conditional(h, bo, hi, cudaGraphCondTypeWhile, &ibody);
        if (!brc) {
            cudaStream_t bi = capture_stream(h, depth + 2);
            if (!bi) {
                brc = h->fail(DD_ERR_CUDA, "capture stream");
            } else {
                const int crc = (int)cudaStreamBeginCaptureToGraph(bi, ibody, nullptr, nullptr, 0,
                                                                   cudaStreamCaptureModeRelaxed);
                if (crc) {
                    brc = cuda_fail(h, crc, "capture arnoldi");
                } else {
                    const int64_t l1 = h->total_launches;
                    for (int k = 0; k < h->prm.chunk && !brc; ++k) brc = arnoldi(bi, (unsigned long long)hi);
                    cudaGraph_t out;
                    const int erc = (int)cudaStreamEndCapture(bi, &out);
                    if (!brc && erc) brc = cuda_fail(h, erc, "end arnoldi capture");
                    h->g_kernels_iter = (h->total_launches - l1) / std::max(1, h->prm.chunk);
                    h->total_launches = l1;
                }
            }
        }
        if (!brc) {
            Prof P(h, ST_VEC, bo, 1);
            const int urc = launch_gm_update(h, U, (unsigned long long)ho, bo);
            if (urc) brc = cuda_fail(h, urc, "gmres update");
        }
        cudaGraph_t out_body;
        const int erc = (int)cudaStreamEndCapture(bo, &out_body);
        if (brc) return brc;
        CK(h, erc, "end cycle capture");
        h->g_kernels_cycle = h->total_launches - l0;
        h->total_launches = l0;
        {
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_solve_end(h, s), "solve end");
        }
        h->lam_valid = true;
        return DD_OK;
    }
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_gm_init(h, tol, h->prm.max_it, h->prm.restart, 0, 0ull, s), "gmres init");
    }
    GmresScalars c;
    bool first = true;
    for (;;) {
        const int have_q = (!first || use_warm) ? 1 : 0;
        first = false;
        int rc = cycle_start(s, have_q, 0ull);
        if (rc) return rc;
        CK(h, read_gm(h, &c, s), "gmres scalars");
        while (!c.cycle_end) {
            const int it0 = c.it;
            for (int k = 0; k < h->prm.chunk; ++k) {
                rc = arnoldi(s, 0ull);
                if (rc) return rc;
            }
            CK(h, read_gm(h, &c, s), "gmres scalars");
            h->work[ST_SCHUR] += c.it - it0;
            h->work_bytes[ST_SCHUR] += (c.it - it0) * mbc;
        }
        {
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_gm_update(h, U, 0ull, s), "gmres update");
        }
        if (c.final) break;
    }
    h->lam_valid = true;
    *it_out = c.it;
    *res_out = c.bnorm > 0 ? c.resid / c.bnorm : 0.0;
    if (c.status != DD_OK) {
        h->err = "non-finite GMRES residual";
        return c.status;
    }
    if (!c.converged) {
        h->err = "coupled GMRES did not converge";
        return DD_ERR_NO_CONVERGENCE;
    }
    return DD_OK;
}

int dd_solve(dd_handle* h, int prec, double tol, bool warm, int* it_out, double* res_out, cudaStream_t s,
             int adaptive = 0, int depth = 0) {
    if (h->prm.scheme != h->factored_scheme)
        return h->fail(DD_ERR_STATE, "the scheme changed since dd_factor: factor again");
    const bool has_c = !h->corner_dof.empty();
    const bool has_l = !h->mult_dof.empty();
    const Vecs V = vecs(h, prec);
    const size_t nlb = sizeof(double) * h->mult_dof.size();
    // y = A_rr^-1 b_r (r rows) and A_cr y (corner rows)          Eq. rF1 / F1uc
    {
        Prof P(h, ST_LOCAL, s, 1, mb(h, GEMV_LOCAL, prec));
        CK(h, launch_gemv(h, GEMV_LOCAL, prec, xsrc(X_FLAT, h->d.b, nullptr, V.bf, nullptr),
                          gout(h->d.y, nullptr, nullptr, nullptr, 1.0), false, s), "gemv local");
    }
    // g = d_r ; f~_c
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_iface_rhs(h, V.fCf, s), "iface rhs");
    }
    if (h->prm.solver == DD_SOLVER_COUPLED_GMRES) {
        const bool dp2 = h->factored_scheme == DD_SCHEME_DP2;
        if (dp2) {   // b1 = 2 alpha M_T t2(y), b2 = 2 alpha M_T t1(y)            Eqs. f2imp1
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_dp2_rhs(h, uview(h, prec), s), "dp2 rhs");
        }
        // [lambda; x_c] from the coupled Eqs. F1lr + F1uc (DP2: f2imp1 + F2un), then x_r   Eq. rF1 / IF2
        const int status = gmres_solve(h, prec, tol, warm, it_out, res_out, s, depth, adaptive);
        if (status != DD_OK && status != DD_ERR_NO_CONVERGENCE) return status;
        const std::string msg = h->err;
        {
            Prof P(h, ST_RECOVER, s, 1, mb(h, GEMV_RECOVER, prec));
            const XSrc xr = dp2 ? xsrc(X_SIDE_CP, h->d.lam, h->d.lam2, V.lamf, V.f32 ? h->d.lam2f : nullptr, h->d.xC,
                                       V.xCf)
                                : xsrc(X_RECOVER, h->d.lam, h->d.xC, V.lamf, V.xCf);
            CK(h, launch_gemv(h, GEMV_RECOVER, prec, xr, gout(h->d.x, h->d.y, nullptr, nullptr, 1.0), false, s),
               "recover");
        }
        h->err = msg;
        return status;
    }
    if (has_c && has_l) {
        // g = d_r - F_rc K~cc^-1 f~_c                                Eq. f1schur
        {
            Prof P(h, ST_COARSE, s, 1, mb(h, GEMV_COARSE, prec));
            CK(h, launch_gemv(h, GEMV_COARSE, prec, xsrc(X_FLAT, h->d.fC, nullptr, V.fCf, nullptr),
                              V.f32 ? gout(nullptr, nullptr, V.vCf, nullptr, 1.0) : gout(h->d.vC, nullptr, nullptr, nullptr, 1.0),
                              false, s), "coarse");
        }
        {
            Prof P(h, ST_CORNER, s, 1, mb(h, GEMV_CORNER, prec));
            CK(h, launch_gemv(h, GEMV_CORNER, prec, xsrc(X_CORNER, h->d.vC, nullptr, V.vCf, nullptr),
                              V.f32 ? gout(nullptr, nullptr, V.wf, nullptr, -1.0) : gout(h->d.w, nullptr, nullptr, nullptr, -1.0),
                              false, s), "corner");
        }
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_jump(h, h->d.w, V.wf, h->d.g, -1.0, h->d.g, s), "jump");
    }
    int status = DD_OK;
    int iters = 0;
    double res = 0.0;
    if (has_l) {
        // a captured graph always takes the warm start; dd_step zeroes lambda before
        // launching it when the multipliers are not valid (same values as a cold start)
        const bool use_warm = warm && (h->lam_valid || h->capturing);
        if (use_warm) {
            CK(h, apply_schur_w(h, prec, X_LAMBDA, h->d.lam, nullptr, V.lamf, nullptr, false, s), "apply lambda0");
        } else {
            CK(h, (int)cudaMemsetAsync(h->d.lam, 0, nlb, s), "memset");
            CK(h, (int)cudaMemsetAsync(h->d.lamf, 0, sizeof(float) * h->mult_dof.size(), s), "memset");
        }
        if (h->capturing) {
            // CG loop as a conditional WHILE node; the CG kernels set its condition
            cudaGraphConditionalHandle hc;
            int rc = create_handle(h, s, &hc);
            if (rc) return rc;
            {
                Prof P(h, ST_VEC, s, 1);
                CK(h, launch_pcg_init(h, use_warm ? 1 : 0, tol, V.wf, V.zf, V.pf, (unsigned long long)hc, adaptive, s),
                   "pcg init");
            }
            cudaGraph_t body;
            rc = add_conditional(h, s, hc, cudaGraphCondTypeWhile, &body);
            if (rc) return rc;
            cudaStream_t bs = capture_stream(h, depth + 1);
            if (!bs) return h->fail(DD_ERR_CUDA, "capture stream");
            CK(h, (int)cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
               "capture body");
            const int64_t l0 = h->total_launches;
            int brc = DD_OK;
            for (int k = 0; k < h->prm.chunk && brc == DD_OK; ++k) {
                brc = apply_schur_w(h, prec, X_PCG, h->d.z, h->d.p, V.zf, V.pf, true, bs);
                if (brc) break;
                Prof P(h, ST_VEC, bs, 2);
                brc = launch_pcg_alpha(h, V.wf, V.pf, bs);
                if (!brc) brc = launch_pcg_update(h, V.zf, V.lamf, (unsigned long long)hc, bs);
            }
            cudaGraph_t out_body;
            const int erc = (int)cudaStreamEndCapture(bs, &out_body);
            if (brc) return brc > 0 && brc < 100 ? brc : cuda_fail(h, brc, "capture body");
            CK(h, erc, "end body capture");
            h->g_kernels_iter = (h->total_launches - l0) / std::max(1, h->prm.chunk);
            h->total_launches = l0;
            {
                Prof P(h, ST_VEC, s, 1);
                CK(h, launch_solve_end(h, s), "solve end");
            }
            h->lam_valid = true;
        } else {
        {
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_pcg_init(h, use_warm ? 1 : 0, tol, V.wf, V.zf, V.pf, 0ull, 0, s), "pcg init");
        }
        PcgScalars hs;
        CK(h, read_scalars(h, &hs, s), "pcg scalars");
        while (!hs.done && hs.it < h->prm.max_it) {
            const int n = std::min(h->prm.chunk, h->prm.max_it - hs.it);
            for (int k = 0; k < n; ++k) {
                CK(h, apply_schur_w(h, prec, X_PCG, h->d.z, h->d.p, V.zf, V.pf, true, s), "apply");
                Prof P(h, ST_VEC, s, 2);
                CK(h, launch_pcg_alpha(h, V.wf, V.pf, s), "pcg alpha");
                CK(h, launch_pcg_update(h, V.zf, V.lamf, 0ull, s), "pcg update");
            }
            CK(h, read_scalars(h, &hs, s), "pcg scalars");
        }
        iters = hs.it;
        count_cg_work(h, prec, hs.it);
        res = hs.gg > 0 ? std::sqrt(hs.rr / hs.gg) : 0.0;
        if (hs.status != DD_OK) status = hs.status;
        else if (!hs.done) status = DD_ERR_NO_CONVERGENCE;
        h->lam_valid = true;
        }
    }
    // x_c = K~cc^-1 (f~_c + F_rc^T lambda)                           Eq. F1uc
    if (has_c) {
        if (has_l) {
            {
                Prof P(h, ST_CORNER, s, 1, mb(h, GEMV_SCHUR_C, prec));
                CK(h, launch_gemv(h, GEMV_SCHUR_C, prec, xsrc(X_LAMBDA, h->d.lam, nullptr, V.lamf, nullptr),
                                  V.f32 ? gout(nullptr, nullptr, V.wf, nullptr, 1.0) : gout(h->d.w, nullptr, nullptr, nullptr, 1.0),
                                  false, s), "Frc^T");
            }
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_corner_gather(h, h->d.w, V.wf, h->d.fC, h->d.uC, V.uCf, false, s), "corner gather");
        }
        Prof P(h, ST_COARSE, s, 1, mb(h, GEMV_COARSE, prec));
        const double* src64 = has_l ? h->d.uC : h->d.fC;
        const float* src32 = has_l ? V.uCf : V.fCf;
        CK(h, launch_gemv(h, GEMV_COARSE, prec, xsrc(X_FLAT, src64, nullptr, src32, nullptr),
                          gout(h->d.xC, nullptr, V.xCf, nullptr, 1.0), false, s), "xc");
    }
    // x_r = y + A_rr^-1 (-B_r^T lambda) - A_rr^-1 A_rc x_c                  Eq. rF1
    {
        Prof P(h, ST_RECOVER, s, 1, mb(h, GEMV_RECOVER, prec));
        CK(h, launch_gemv(h, GEMV_RECOVER, prec, xsrc(X_RECOVER, h->d.lam, h->d.xC, V.lamf, V.xCf),
                          gout(h->d.x, h->d.y, nullptr, nullptr, 1.0), false, s), "recover");
    }
    if (it_out) *it_out = iters;
    if (res_out) *res_out = res;
    if (status != DD_OK) h->err = status == DD_ERR_NO_CONVERGENCE ? "interface CG did not converge" : "non-finite CG residual";
    return status;
}

}  // namespace

extern "C" {

namespace {
int reset_particles(dd_handle* h, cudaStream_t s);
int upload_pic_mesh(dd_handle* h, cudaStream_t s);
}  // namespace

int dd_setup(const dd_mesh* mesh, const int32_t* part, int32_t n_sub, const dd_params* params, dd_handle** out) {
    if (!out) return DD_ERR_ARG;
    *out = nullptr;
    if (!mesh || !part || n_sub < 1 || !mesh->xyz || !mesh->tets || mesh->n_nodes < 4 || mesh->n_tets < 1)
        return DD_ERR_ARG;
    dd_handle* h = new (std::nothrow) dd_handle();
    if (!h) return DD_ERR_ARG;
    h->prm = params ? *params : default_params();
    int rc = check_params(h, h->prm);
    if (rc == DD_OK) {
        try {
            const int R = h->prm.members;
            h->members = R;
            h->n_sub_real = n_sub;
            if (R == 1) {
                rc = dd_build_host(h, mesh, part, n_sub);
            } else {
                // member r = copy r of the mesh: node ids + r N, subdomain ids + r n_sub
                const int64_t N = mesh->n_nodes, T = mesh->n_tets;
                std::vector<double> xyz((size_t)(R * 3 * N)), eps;
                std::vector<int32_t> tets((size_t)(R * 4 * T)), prt((size_t)(R * T));
                if (mesh->eps) eps.resize((size_t)(R * T));
                for (int r = 0; r < R; ++r) {
                    std::copy(mesh->xyz, mesh->xyz + 3 * N, xyz.begin() + r * 3 * N);
                    for (int64_t k = 0; k < 4 * T; ++k) tets[r * 4 * T + k] = mesh->tets[k] + (int32_t)(r * N);
                    for (int64_t t = 0; t < T; ++t) prt[r * T + t] = part[t] + r * n_sub;
                    if (mesh->eps) std::copy(mesh->eps, mesh->eps + T, eps.begin() + r * T);
                }
                if ((int64_t)R * N > INT32_MAX) rc = h->fail(DD_ERR_ARG, "ensemble mesh too large");
                dd_mesh rep{R * N, R * T, xyz.data(), tets.data(), mesh->eps ? eps.data() : nullptr, mesh->mu};
                if (rc == DD_OK) rc = dd_build_host(h, &rep, prt.data(), R * n_sub);
            }
        } catch (const std::exception& ex) {
            rc = h->fail(DD_ERR_ARG, std::string("setup failed: ") + ex.what());
        }
    }
    *out = h;  // returned even on failure so that dd_last_error can be read; caller destroys
    return rc;
}

int dd_set_params(dd_handle* h, const dd_params* params) {
    if (!h || !params) return DD_ERR_ARG;
    int rc = check_params(h, *params);
    if (rc) return rc;
    if (h->capturing) return h->fail(DD_ERR_STATE, "dd_set_params during capture");
    h->prm = *params;
    drop_graphs(h);
    return DD_OK;
}

int dd_get_sizes(const dd_handle* h, dd_sizes* o) {
    if (!h || !o) return DD_ERR_ARG;
    o->n_edges = h->n_edges;
    o->n_dof = h->n_dof;
    o->n_sub = h->n_sub;
    o->n_lambda = (int64_t)h->mult_dof.size();
    o->n_corner = (int64_t)h->corner_dof.size();
    o->n_local = h->sub_ptr.empty() ? 0 : h->sub_ptr.back();
    o->nnz_local = h->row_ptr.empty() ? 0 : h->row_ptr.back();
    o->max_nr = h->max_nr;
    o->max_ns = h->max_ns;
    o->workspace_bytes = h->sub_ptr.empty() ? 0 : dd_workspace_layout(const_cast<dd_handle*>(h), false);
    o->dense_bytes_fp64 = h->dense_elems * 8;
    o->members = h->members;
    return DD_OK;
}

int dd_get_maps(const dd_handle* h, dd_maps* m) {
    if (!h || !m || h->sub_ptr.empty()) return DD_ERR_ARG;
    auto cp = [](auto* dst, const auto& v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(v[0]) * v.size());
    };
    cp(m->edges, h->edges);
    cp(m->dof_edge, h->dof_edge);
    cp(m->sub_ptr, h->sub_ptr);
    cp(m->local_dof, h->local_dof);
    cp(m->n_int, h->nI);
    cp(m->n_gam, h->nG);
    cp(m->n_cor, h->nC);
    cp(m->mult_dof, h->mult_dof);
    cp(m->mult_sub, h->mult_sub);
    cp(m->mult_loc, h->mult_loc);
    cp(m->corner_dof, h->corner_dof);
    cp(m->owner, h->owner);
    return DD_OK;
}

int dd_set_probes(dd_handle* h, int32_t n, const double* xyz) {
    if (!h || n < 0 || n > kMaxProbes || (n > 0 && !xyz)) return h ? h->fail(DD_ERR_ARG, "bad probe list") : DD_ERR_ARG;
    if (n > 0 && h->members > 1) return h->fail(DD_ERR_STATE, "probes are not available for an ensemble (members > 1)");
    int rc = dd_locate_probes(h, n, xyz);
    if (rc) return rc;
    if (h->bound && n > 0) {
        CK(h, upload(h->d.probe_dof, h->probe_dof, 0), "upload probes");
        CK(h, upload(h->d.probe_w, h->probe_w, 0), "upload probes");
        CK(h, (int)cudaStreamSynchronize(0), "sync");
    }
    return DD_OK;
}

int dd_bind_workspace(dd_handle* h, void* dev, size_t bytes, void* stream) {
    if (!h || !dev || h->sub_ptr.empty()) return DD_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(dev) & 255) != 0) return h->fail(DD_ERR_ARG, "workspace must be 256-byte aligned");
    const size_t need = dd_workspace_layout(h, false);
    if (bytes < need) return h->fail(DD_ERR_ARG, "workspace too small: need " + std::to_string(need) + " bytes");
    drop_graphs(h);
    {
        int dev_id = 0;
        CK(h, (int)cudaGetDevice(&dev_id), "device");
        CK(h, (int)cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev_id), "device attribute");
    }
    h->ws = static_cast<char*>(dev);
    h->ws_bytes = bytes;
    dd_workspace_layout(h, true);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nd = (size_t)h->n_dof;
    MatDesc cd{0, 0, h->ldc, 0, (int32_t)h->corner_dof.size(), (int32_t)h->corner_dof.size()};
    CK(h, (int)cudaMemcpyAsync(h->d.mats, h->mats.data(), sizeof(MatDesc) * h->mats.size(), cudaMemcpyHostToDevice, s), "upload");
    CK(h, (int)cudaMemcpyAsync(h->d.coarse_desc, &cd, sizeof(MatDesc), cudaMemcpyHostToDevice, s), "upload");
    CK(h, upload(h->d.slot_mult, h->slot_mult, s), "upload");
    CK(h, upload(h->d.slot_corner, h->slot_corner, s), "upload");
    CK(h, upload(h->d.slot_dof, h->slot_dof, s), "upload");
    CK(h, upload(h->d.slot_sub, h->slot_sub, s), "upload");
    CK(h, upload(h->d.slot_own, h->slot_own, s), "upload");
    CK(h, upload(h->d.mult_slot, h->mult_slot, s), "upload");
    CK(h, upload(h->d.slot_upos, h->slot_upos, s), "upload");
    CK(h, upload(h->d.corner_ptr, h->corner_ptr, s), "upload");
    CK(h, upload(h->d.corner_slot, h->corner_slot, s), "upload");
    CK(h, upload(h->d.owner_slot, h->owner_slot, s), "upload");
    CK(h, upload(h->d.copy_ptr, h->copy_ptr, s), "upload");
    CK(h, upload(h->d.copy_slot, h->copy_slot, s), "upload");
    CK(h, upload(h->d.row_ptr, h->row_ptr, s), "upload");
    CK(h, upload(h->d.col_loc, h->col_loc, s), "upload");
    CK(h, upload(h->d.col_dof, h->col_dof, s), "upload");
    CK(h, upload(h->d.Tval, h->Tval, s), "upload");
    CK(h, upload(h->d.symd, h->sym, s), "upload");
    if (!h->sym_dir.empty()) CK(h, upload(h->d.sym_dir, h->sym_dir, s), "upload");
    for (int k = 0; k < kTcKinds; ++k)
        if (!h->tcd[k].empty()) CK(h, upload(h->d.tcd[k], h->tcd[k], s), "upload");
    if (!h->tc_dir.empty()) CK(h, upload(h->d.tc_dir, h->tc_dir, s), "upload");
    CK(h, upload(h->d.mt_ptr, h->mt_ptr, s), "upload");
    CK(h, upload(h->d.mt_col, h->mt_col, s), "upload");
    CK(h, upload(h->d.mt_val, h->mt_val, s), "upload");
    for (int m = 0; m < GEMV_NMODES; ++m) {
        if (!h->sym_rng[m].empty()) CK(h, upload(h->d.sym_rng[m], h->sym_rng[m], s), "upload");
        if (!h->sym_tl[m].empty()) CK(h, upload(h->d.sym_tl[m], h->sym_tl[m], s), "upload");
    }
    CK(h, upload(h->d.Sval, h->Sval, s), "upload");
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < GEMV_NMODES; ++m) {
            const int urc = upload_tasks(h, p, m, s);
            if (urc) return urc == DD_ERR_CUDA ? h->fail(DD_ERR_CUDA, "upload tasks") : urc;
        }
    {
        std::vector<int32_t> td(h->tet_dof.size());
        for (size_t i = 0; i < td.size(); ++i) td[i] = (int32_t)h->tet_dof[i];
        CK(h, upload(h->d.tet_dof, td, s), "upload");
        CK(h, (int)cudaStreamSynchronize(s), "sync");   // td is a local
    }
    CK(h, upload(h->d.That, h->That, s), "upload");
    {
        const int prc = upload_pic_mesh(h, s);
        if (prc) return prc;
    }
    if (h->n_probe) {
        CK(h, upload(h->d.probe_dof, h->probe_dof, s), "upload");
        CK(h, upload(h->d.probe_w, h->probe_w, s), "upload");
    }
    for (int k = 0; k < 3; ++k) CK(h, (int)cudaMemsetAsync(h->d.e[k], 0, sizeof(double) * nd, s), "memset");
    for (int k = 0; k < 3; ++k) CK(h, (int)cudaMemsetAsync(h->d.mu[k], 0, sizeof(double) * nd, s), "memset");
    CK(h, (int)cudaMemsetAsync(h->d.sc, 0, sizeof(PcgScalars), s), "memset");
    CK(h, (int)cudaMemsetAsync(h->d.gs, 0, sizeof(GmresScalars), s), "memset");
    CK(h, (int)cudaMemsetAsync(h->d.status, 0, 16, s), "memset");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    h->bound = true;
    h->factored = false;
    h->eps_map_up = false;
    compute_stage_bytes(h);
    return DD_OK;
}

int dd_factor(dd_handle* h, double dt, void* stream) {
    if (!h) return DD_ERR_ARG;
    if (!h->bound) return h->fail(DD_ERR_STATE, "dd_factor before dd_bind_workspace");
    if (!(dt > 0.0) || !std::isfinite(dt)) return h->fail(DD_ERR_ARG, "dt must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    h->factored = false;
    drop_graphs(h);
    CK(h, (int)cudaMemsetAsync(h->d.status, 0, 4, s), "memset");
    {
        Prof P(h, ST_FACTOR, s, 2);
        CK(h, launch_csr_combine(h, dt * dt / 4.0, s), "A = T + dt^2/4 S");
        CK(h, launch_dense_assemble(h, s), "dense assemble");
    }
    const double alpha = h->prm.robin_alpha > 0.0 ? h->prm.robin_alpha : 0.5 * dt;
    if (h->prm.scheme == DD_SCHEME_DP2) {
        Prof P(h, ST_FACTOR, s, 1);
        CK(h, launch_robin_add(h, alpha, s), "Robin term");
    }
    for (int k0 = 0; k0 < h->max_nr; k0 += kNB) {
        Prof P(h, ST_FACTOR, s, 3);
        CK(h, launch_sweep(h, false, k0, s), "local elimination");
    }
    const int nc = (int)h->corner_dof.size();
    if (nc && h->ldc) {
        {
            Prof P(h, ST_FACTOR, s, 1);
            CK(h, launch_coarse_assemble(h, s), "coarse assemble");
        }
        for (int k0 = 0; k0 < nc; k0 += kNB) {
            Prof P(h, ST_FACTOR, s, 3);
            CK(h, launch_sweep(h, true, k0, s), "coarse inverse");
        }
    }
    {
        Prof P(h, ST_FACTOR, s, 3);
        CK(h, launch_factor_finish(h, s), "factor finish");
        CK(h, launch_corner_diag(h, s), "coarse diagonal");
    }
    {
        Prof P(h, ST_FACTOR, s, 1);
        CK(h, launch_sym_pack(h, s), "packed symmetric tiles");
        CK(h, launch_tc_pack(h, s), "tensor-core panels");
    }
    int32_t st = 0;
    CK(h, (int)cudaMemcpyAsync(&st, h->d.status, 4, cudaMemcpyDeviceToHost, s), "status");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    if (st != 0) return h->fail(DD_ERR_NOT_SPD, "non-positive pivot in the local or coarse elimination");
    if (wait_err_set(h, s)) {   // a bounded wait of the tensor-core update gave up: the factors are void
        CK(h, (int)cudaMemsetAsync(&h->d.sc->wait_err, 0, sizeof(int32_t), s), "clear wait error");
        CK(h, (int)cudaStreamSynchronize(s), "sync");
        return h->fail(DD_ERR_TIMEOUT, "a bounded device wait of the tensor-core elimination gave up");
    }
    const size_t nd = (size_t)h->n_dof;
    for (int k = 0; k < 3; ++k) CK(h, (int)cudaMemsetAsync(h->d.e[k], 0, sizeof(double) * nd, s), "memset");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    for (int k = 0; k < 3; ++k) CK(h, (int)cudaMemsetAsync(h->d.mu[k], 0, sizeof(double) * nd, s), "memset");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    {
        const int prc = reset_particles(h, s);
        if (prc) return prc;
    }
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    CK(h, (int)cudaMemsetAsync(&h->d.sc->lam_levels, 0, sizeof(int32_t), s), "memset");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    h->dt = dt;
    h->step = 0;
    h->cur = 0;
    h->cur_adj = 0;
    h->lam_valid = false;
    h->lam_adj_valid = false;
    h->factored_scheme = h->prm.scheme;
    h->factored_alpha = alpha;
    h->factored = true;
    return DD_OK;
}

namespace {

// warm_start 2: before the first solve of a step, lambda_0 = 2 lambda^{n-1} -
// lambda^{n-2} once two levels of history exist (a device counter), so that
// eager and graph launches extrapolate on the same steps.
int extrapolate_lambda(dd_handle* h, int prec, cudaStream_t s) {
    if (h->prm.warm_start != 2 || h->mult_dof.empty()) return DD_OK;
    const size_t nm = h->mult_dof.size(), nc = h->corner_dof.size();
    const bool gm = h->prm.solver == DD_SOLVER_COUPLED_GMRES, dp2 = h->factored_scheme == DD_SCHEME_DP2;
    if (!h->lam_valid && !h->capturing) {
        CK(h, (int)cudaMemsetAsync(h->d.lam, 0, sizeof(double) * nm, s), "memset");
        CK(h, (int)cudaMemsetAsync(h->d.lamf, 0, sizeof(float) * nm, s), "memset");
        if (gm && nc) {
            CK(h, (int)cudaMemsetAsync(h->d.xC, 0, sizeof(double) * nc, s), "memset");
            CK(h, (int)cudaMemsetAsync(h->d.xCf, 0, sizeof(float) * nc, s), "memset");
        }
        if (dp2) {
            CK(h, (int)cudaMemsetAsync(h->d.lam2, 0, sizeof(double) * nm, s), "memset");
            CK(h, (int)cudaMemsetAsync(h->d.lam2f, 0, sizeof(float) * nm, s), "memset");
        }
    }
    Prof P(h, ST_VEC, s, 2 + (gm && nc ? 1 : 0) + (dp2 ? 1 : 0));
    CK(h, launch_extrapolate(h, prec == DD_MIXED, s), "extrapolate");
    return DD_OK;
}

// Mixed refinement: the first pass's interface solution (lambda and, for the
// coupled GMRES, x_c) is the next step's warm start; the later passes solve for
// corrections.  save: copy it aside after the first pass; !save: put it back.
int keep_first_pass(dd_handle* h, bool save, cudaStream_t s) {
    const size_t nm = h->mult_dof.size(), nc = h->corner_dof.size();
    auto cp = [&](void* a, void* b, size_t n) -> int {
        if (!n) return DD_OK;
        CK(h, (int)cudaMemcpyAsync(save ? b : a, save ? a : b, n, cudaMemcpyDeviceToDevice, s), "warm-start copy");
        return DD_OK;
    };
    int rc = cp(h->d.lam, h->d.lam_scratch, sizeof(double) * nm);
    if (!rc) rc = cp(h->d.lamf, h->d.lamf_scratch, sizeof(float) * nm);
    if (!rc && h->prm.solver == DD_SOLVER_COUPLED_GMRES) {
        rc = cp(h->d.xC, h->d.xC_scratch, sizeof(double) * nc);
        if (!rc) rc = cp(h->d.xCf, h->d.xCf_scratch, sizeof(float) * nc);
    }
    if (!rc && h->factored_scheme == DD_SCHEME_DP2) {
        rc = cp(h->d.lam2, h->d.lam2_scratch, sizeof(double) * nm);
        if (!rc) rc = cp(h->d.lam2f, h->d.lam2f_scratch, sizeof(float) * nm);
    }
    return rc;
}

// One level of the Newmark recurrence from (u_n, u_nm1) into u_np1:
// A delta = -dt^2 S u_n + src_sign * src (subassembled, source on the owner),
// u_np1 = 2 u_n - u_nm1 + delta.  Used by the forward step (src = d2g, sign -1)
// and by the adjoint step (src = seed, sign +1).
// A bounded device wait gave up during the step (PcgScalars::wait_err): the step
// is void.  Clears the sticky word, drops the multiplier warm start (the last
// solve's iterate may be garbage) and returns DD_ERR_TIMEOUT; the caller keeps
// the time levels where they were.
int report_timeout(dd_handle* h, cudaStream_t s) {
    CK(h, (int)cudaMemsetAsync(&h->d.sc->wait_err, 0, sizeof(int32_t), s), "clear wait error");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    h->lam_valid = false;
    h->err = "a bounded device wait of the packed-tile GEMV gave up; the step was not taken";
    return DD_ERR_TIMEOUT;
}


int advance(dd_handle* h, const double* u_n, const double* u_nm1, double* u_np1, const double* src, double src_sign,
            int* iters_out, int* refs_out, double* resid_out, cudaStream_t s) {
    int status = DD_OK, iters = 0, refinements = 0;
    double resid = 0.0;
    {
        Prof P(h, ST_RHS, s, 1, h->bytes_per_launch[ST_RHS]);
        CK(h, launch_rhs(h, u_n, src, src_sign, h->dt, s), "rhs");
    }
    {
        const int xrc = extrapolate_lambda(h, h->prm.precision, s);
        if (xrc) return xrc;
    }
    if (h->prm.precision == DD_FP64) {
        status = dd_solve(h, DD_FP64, h->prm.tol, h->prm.warm_start != 0, &iters, &resid, s);
        if (status != DD_OK && status != DD_ERR_NO_CONVERGENCE) return status;
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_writeback(h, u_n, u_nm1, nullptr, nullptr, 1, u_np1, s), "writeback");
    } else {
        // FP64 iterative refinement of the step system with FP32 DD correction solves
        {
            Prof P(h, ST_REFINE, s, 1);
            CK(h, launch_assembled_norm(h, 1, h->d.bf, s), "norm b");
        }
        PcgScalars hs;
        for (int k = 0; k < h->prm.max_refine; ++k) {
            const bool warm = (k == 0) && h->prm.warm_start != 0;
            if (k == 1) {
                const int xrc = keep_first_pass(h, true, s);
                if (xrc) return xrc;
            }
            int it = 0;
            double r = 0.0;
            // the first pass solves to tol; a later pass only has to cut the current
            // residual (resid, relative to ||b||) down to refine_tol, with a 3x margin
            double tol_k = h->prm.tol;
            if (k > 0 && resid > 0.0) tol_k = std::min(0.1, std::max(h->prm.tol, 0.3 * h->prm.refine_tol / resid));
            int st = dd_solve(h, DD_MIXED, tol_k, warm, &it, &r, s);
            iters += it;
            ++refinements;
            if (st != DD_OK && st != DD_ERR_NO_CONVERGENCE) {   // a void operator can end the solve early
                if (st != DD_ERR_CUDA && wait_err_set(h, s)) return report_timeout(h, s);
                return st;
            }
            {
                Prof P(h, ST_VEC, s, 1);
                CK(h, launch_writeback(h, u_n, u_nm1, h->d.delta_k, h->d.delta, k == 0 ? 1 : 0, nullptr, s), "writeback");
            }
            {
                Prof P(h, ST_REFINE, s, 2, h->bytes_per_launch[ST_REFINE]);
                CK(h, launch_residual_local(h, s), "residual");
                CK(h, launch_assembled_norm(h, 0, h->d.bf, s), "norm r");
            }
            CK(h, read_scalars(h, &hs, s), "scalars");
            if (hs.wait_err) {   // a bounded wait of the packed GEMV gave up: this pass's result is void
                status = DD_ERR_TIMEOUT;
                break;
            }
            resid = hs.norm_b2 > 0 ? std::sqrt(hs.norm_r2 / hs.norm_b2) : 0.0;
            if (!std::isfinite(resid)) {
                status = DD_ERR_NONFINITE;
                break;
            }
            if (resid <= h->prm.refine_tol) break;
            if (k + 1 == h->prm.max_refine) status = DD_ERR_NO_CONVERGENCE;
        }
        if (refinements > 1) {
            const int xrc = keep_first_pass(h, false, s);
            if (xrc) return xrc;
        }
        if (status == DD_ERR_NONFINITE) return status;
        if (status == DD_ERR_TIMEOUT) return report_timeout(h, s);
        {
            Prof P(h, ST_VEC, s, 1);
            CK(h, launch_advance(h, u_n, u_nm1, h->d.delta, u_np1, s), "advance");
        }
        if (status == DD_ERR_NO_CONVERGENCE) h->err = "refinement did not reach refine_tol";
    }
    *iters_out = iters;
    *refs_out = refinements;
    *resid_out = resid;
    return status;
}

// ---- graph mode ---------------------------------------------------------------

// Mixed-precision refinement passes k >= 2 as nested conditional IF nodes:
// the condition of each pass is set by the residual kernel at the end of the
// previous pass (it defaults to 0 at every launch).
int refine_chain(dd_handle* h, int k, int depth, cudaStream_t s, const double* u_n, const double* u_nm1) {
    cudaGraphConditionalHandle hc;
    int rc = create_handle(h, s, &hc);
    if (rc) return rc;
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_refine_cond(h, (unsigned long long)hc, s), "refine cond");
    }
    cudaGraph_t body;
    rc = add_conditional(h, s, hc, cudaGraphCondTypeIf, &body);
    if (rc) return rc;
    cudaStream_t bs = capture_stream(h, depth + 1);
    if (!bs) return h->fail(DD_ERR_CUDA, "capture stream");
    CK(h, (int)cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture if");
    const int64_t l0 = h->total_launches;
    int brc = DD_OK;
    {
        const size_t nm = h->mult_dof.size();
        if (nm) {  // later passes start cold, as in eager mode
            brc = (int)cudaMemsetAsync(h->d.lam, 0, sizeof(double) * nm, bs);
            if (!brc) brc = (int)cudaMemsetAsync(h->d.lamf, 0, sizeof(float) * nm, bs);
            if (brc) brc = cuda_fail(h, brc, "memset");
        }
        int it = 0;
        double r = 0.0;
        if (!brc) brc = dd_solve(h, DD_MIXED, h->prm.tol, false, &it, &r, bs, 1, depth + 1);
        if (!brc) {
            Prof P(h, ST_VEC, bs, 1);
            brc = launch_writeback(h, u_n, u_nm1, h->d.delta_k, h->d.delta, 0, nullptr, bs);
            if (brc) brc = cuda_fail(h, brc, "writeback");
        }
        if (!brc) {
            Prof P(h, ST_REFINE, bs, 2, h->bytes_per_launch[ST_REFINE]);
            brc = launch_residual_local(h, bs);
            if (!brc) brc = launch_assembled_norm(h, 0, h->d.bf, bs);
            if (brc) brc = cuda_fail(h, brc, "residual");
        }
        if (!brc && k + 1 < h->prm.max_refine) brc = refine_chain(h, k + 1, depth + 1, bs, u_n, u_nm1);
    }
    cudaGraph_t out_body;
    const int erc = (int)cudaStreamEndCapture(bs, &out_body);
    if (brc) return brc;
    CK(h, erc, "end if capture");
    if (k == 1) h->g_kernels_pass = h->total_launches - l0;
    h->total_launches = l0;
    return DD_OK;
}

// The whole step from (u_n, u_nm1) into u_np1, captured on stream s; the source is d.src_in.
int step_body_graph(dd_handle* h, const double* u_n, const double* u_nm1, double* u_np1, cudaStream_t s) {
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_step_begin(h, s), "step begin");
    }
    {
        Prof P(h, ST_RHS, s, 1, h->bytes_per_launch[ST_RHS]);
        CK(h, launch_rhs(h, u_n, h->d.src_in, -1.0, h->dt, s), "rhs");
    }
    int it = 0;
    double r = 0.0;
    {
        const int xrc = extrapolate_lambda(h, h->prm.precision, s);
        if (xrc) return xrc;
    }
    if (h->prm.precision == DD_FP64) {
        int rc = dd_solve(h, DD_FP64, h->prm.tol, h->prm.warm_start != 0, &it, &r, s, 0, 0);
        if (rc) return rc;
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_writeback(h, u_n, u_nm1, nullptr, nullptr, 1, u_np1, s), "writeback");
        return DD_OK;
    }
    {
        Prof P(h, ST_REFINE, s, 1);
        CK(h, launch_assembled_norm(h, 1, h->d.bf, s), "norm b");
    }
    int rc = dd_solve(h, DD_MIXED, h->prm.tol, h->prm.warm_start != 0, &it, &r, s, 0, 0);
    if (rc) return rc;
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_writeback(h, u_n, u_nm1, h->d.delta_k, h->d.delta, 1, nullptr, s), "writeback");
    }
    {
        Prof P(h, ST_REFINE, s, 2, h->bytes_per_launch[ST_REFINE]);
        CK(h, launch_residual_local(h, s), "residual");
        CK(h, launch_assembled_norm(h, 0, h->d.bf, s), "norm r");
    }
    rc = keep_first_pass(h, true, s);   // the first pass's solution is the next step's warm start
    if (rc) return rc;
    if (h->prm.max_refine > 1) {
        rc = refine_chain(h, 1, 0, s, u_n, u_nm1);
        if (rc) return rc;
    }
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_refine_cond(h, 0ull, s), "refine final");
    }
    rc = keep_first_pass(h, false, s);
    if (rc) return rc;
    Prof P(h, ST_VEC, s, 1);
    CK(h, launch_advance(h, u_n, u_nm1, h->d.delta, u_np1, s), "advance");
    return DD_OK;
}

// Capture the step of time-level phase `phase` (e[phase] = e^n) into h->gexec[phase].
int capture_step(dd_handle* h, int phase) {
    cudaStream_t cs = capture_stream(h, 0);
    if (!cs) return h->fail(DD_ERR_CUDA, "capture stream");
    const bool prof_saved = h->prof_on;
    const int64_t l0 = h->total_launches;
    int64_t lk[DD_N_STAGES], wk[DD_N_STAGES];
    double bk[DD_N_STAGES];
    for (int k = 0; k < DD_N_STAGES; ++k) {
        lk[k] = h->launches[k];
        wk[k] = h->work[k];
        bk[k] = h->work_bytes[k];
    }
    h->prof_on = false;
    h->capturing = true;
    const bool lam_valid = h->lam_valid;
    int rc = (int)cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (rc) {
        h->capturing = false;
        h->prof_on = prof_saved;
        return cuda_fail(h, rc, "begin capture");
    }
    rc = step_body_graph(h, h->d.e[phase], h->d.e[(phase + 2) % 3], h->d.e[(phase + 1) % 3], cs);
    cudaGraph_t g = nullptr;
    const int erc = (int)cudaStreamEndCapture(cs, &g);
    h->capturing = false;
    h->prof_on = prof_saved;
    h->lam_valid = lam_valid;
    h->g_kernels_main = h->total_launches - l0;
    h->total_launches = l0;
    for (int k = 0; k < DD_N_STAGES; ++k) {  // capture is not execution
        h->launches[k] = lk[k];
        h->work[k] = wk[k];
        h->work_bytes[k] = bk[k];
    }
    if (rc || erc) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : cuda_fail(h, erc, "end capture");
    }
    cudaGraphExec_t ex;
    rc = (int)cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (rc) return cuda_fail(h, rc, "graph instantiate");
    h->gexec[phase] = (void*)ex;
    return DD_OK;
}

int dd_step_graph(dd_handle* h, const double* d2g, double scale, double* e_out, dd_stats* stats, cudaStream_t s) {
    const int phase = h->cur;
    if (!h->gexec[phase]) {
        int rc = capture_step(h, phase);
        if (rc) return rc;
    }
    const size_t nb = sizeof(double) * h->n_dof;
    if (d2g && scale == 1.0) CK(h, (int)cudaMemcpyAsync(h->d.src_in, d2g, nb, cudaMemcpyDeviceToDevice, s), "source copy");
    else if (d2g) CK(h, launch_scale_copy(h, h->d.src_in, d2g, scale, s), "source copy");
    else CK(h, (int)cudaMemsetAsync(h->d.src_in, 0, nb, s), "source clear");
    if (!h->lam_valid && !h->mult_dof.empty()) {
        CK(h, (int)cudaMemsetAsync(h->d.lam, 0, sizeof(double) * h->mult_dof.size(), s), "memset");
        CK(h, (int)cudaMemsetAsync(h->d.lamf, 0, sizeof(float) * h->mult_dof.size(), s), "memset");
    }
    if (!h->lam_valid && h->prm.solver == DD_SOLVER_COUPLED_GMRES && !h->corner_dof.empty()) {
        CK(h, (int)cudaMemsetAsync(h->d.xC, 0, sizeof(double) * h->corner_dof.size(), s), "memset");
        CK(h, (int)cudaMemsetAsync(h->d.xCf, 0, sizeof(float) * h->corner_dof.size(), s), "memset");
    }
    if (!h->lam_valid && h->factored_scheme == DD_SCHEME_DP2 && !h->mult_dof.empty()) {
        CK(h, (int)cudaMemsetAsync(h->d.lam2, 0, sizeof(double) * h->mult_dof.size(), s), "memset");
        CK(h, (int)cudaMemsetAsync(h->d.lam2f, 0, sizeof(float) * h->mult_dof.size(), s), "memset");
    }
    CK(h, (int)cudaGraphLaunch((cudaGraphExec_t)h->gexec[phase], s), "graph launch");
    h->lam_valid = true;
    double* e_np1 = h->d.e[(phase + 1) % 3];
    h->cur = (phase + 1) % 3;
    h->step += 1;
    if (e_out) CK(h, (int)cudaMemcpyAsync(e_out, e_np1, nb, cudaMemcpyDeviceToDevice, s), "e_out");
    int status = DD_OK;
    if (stats) {
        PcgScalars hs;
        CK(h, read_scalars(h, &hs, s), "scalars");
        stats->iters = hs.it_total;
        stats->refinements = h->prm.precision == DD_MIXED ? hs.refinements : 0;
        stats->resid = h->prm.precision == DD_MIXED ? (hs.norm_b2 > 0 ? std::sqrt(hs.norm_r2 / hs.norm_b2) : 0.0)
                                                     : (hs.gg > 0 ? std::sqrt(hs.rr / hs.gg) : 0.0);
        status = hs.step_status;
        if (hs.wait_err || status == DD_ERR_TIMEOUT) {   // void step: keep e^n, e^{n-1} and the step counter
            h->cur = phase;
            h->step -= 1;
            status = report_timeout(h, s);
        }
        stats->status = status;
        h->total_launches += h->g_kernels_main + h->g_kernels_iter * (int64_t)hs.it_total +
                             h->g_kernels_pass * (int64_t)std::max(0, hs.refinements - 1) +
                             h->g_kernels_cycle * (int64_t)hs.cycles;
        if (status == DD_ERR_NO_CONVERGENCE) h->err = "interface CG or refinement did not converge";
        if (status == DD_ERR_NONFINITE) h->err = "non-finite residual";
    }
    return status;
}

// Swap the interface multipliers (warm start) between the forward and the
// adjoint march, which share the factors but not their CG history.
void swap_lambda(dd_handle* h) {
    std::swap(h->d.lam, h->d.lam_adj);
    std::swap(h->d.lamf, h->d.lamf_adj);
    std::swap(h->d.lam_prev, h->d.lam_prev_adj);
    std::swap(h->d.xC_prev, h->d.xC_prev_adj);
    std::swap(h->d.lam2_prev, h->d.lam2_prev_adj);
    std::swap(h->d.xC, h->d.xC_adj);
    std::swap(h->d.xCf, h->d.xCf_adj);
    std::swap(h->d.lam2, h->d.lam2_adj);
    std::swap(h->d.lam2f, h->d.lam2f_adj);
    std::swap(h->lam_valid, h->lam_adj_valid);
}

}  // namespace

int dd_step(dd_handle* h, const double* d2g, double* e_out, dd_stats* stats, void* stream) {
    return dd_step_scaled(h, d2g, 1.0, e_out, stats, stream);
}

int dd_step_scaled(dd_handle* h, const double* d2g, double scale, double* e_out, dd_stats* stats, void* stream) {
    if (!h) return DD_ERR_ARG;
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_step before dd_factor");
    if (!std::isfinite(scale)) return h->fail(DD_ERR_ARG, "source scale must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->prm.use_graph) return dd_step_graph(h, d2g, scale, e_out, stats, s);
    const double* e_n = h->d.e[h->cur];
    const double* e_nm1 = h->d.e[(h->cur + 2) % 3];
    double* e_np1 = h->d.e[(h->cur + 1) % 3];
    int iters = 0, refinements = 0;
    double resid = 0.0;
    // b = -dt^2 S e^n - d2g (subassembled): A delta = b, e^{n+1} = 2e^n - e^{n-1} + delta
    const int status = advance(h, e_n, e_nm1, e_np1, d2g, -scale, &iters, &refinements, &resid, s);
    if (status != DD_OK && status != DD_ERR_NO_CONVERGENCE) return status;
    h->cur = (h->cur + 1) % 3;
    h->step += 1;
    if (e_out) CK(h, (int)cudaMemcpyAsync(e_out, e_np1, sizeof(double) * h->n_dof, cudaMemcpyDeviceToDevice, s), "e_out");
    if (stats) {
        stats->iters = iters;
        stats->refinements = refinements;
        stats->resid = resid;
        stats->status = status;
    }
    return status;
}

int dd_adjoint_reset(dd_handle* h, void* stream) {
    if (!h) return DD_ERR_ARG;
    if (h->members > 1) return h->fail(DD_ERR_STATE, "the adjoint is not available for an ensemble (members > 1)");
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < 3; ++k) CK(h, (int)cudaMemsetAsync(h->d.mu[k], 0, sizeof(double) * h->n_dof, s), "memset");
    h->cur_adj = 0;
    h->lam_adj_valid = false;
    return DD_OK;
}

int dd_adjoint_step(dd_handle* h, const double* seed, const double* e_k, const double* e_km1, const double* e_km2,
                    const double* d2g_hat, double* grad_eps, double* grad_amp, double* mu_out, dd_stats* stats,
                    void* stream) {
    return dd_adjoint_step_scaled(h, seed, e_k, e_km1, e_km2, d2g_hat, 1.0, grad_eps, grad_amp, mu_out, stats, stream);
}

int dd_adjoint_step_scaled(dd_handle* h, const double* seed, const double* e_k, const double* e_km1,
                           const double* e_km2, const double* d2g_hat, double d2g_scale, double* grad_eps,
                           double* grad_amp, double* mu_out, dd_stats* stats, void* stream) {
    if (!h || !seed) return DD_ERR_ARG;
    if (!std::isfinite(d2g_scale)) return h->fail(DD_ERR_ARG, "source scale must be finite");
    if (h->members > 1) return h->fail(DD_ERR_STATE, "the adjoint is not available for an ensemble (members > 1)");
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_adjoint_step before dd_factor");
    if (grad_eps && (!e_k || !e_km1 || !e_km2)) return h->fail(DD_ERR_ARG, "grad_eps needs e_k, e_km1, e_km2");
    cudaStream_t s = (cudaStream_t)stream;
    const double* mu_k1 = h->d.mu[h->cur_adj];
    const double* mu_k2 = h->d.mu[(h->cur_adj + 2) % 3];
    double* mu_k = h->d.mu[(h->cur_adj + 1) % 3];
    int iters = 0, refinements = 0;
    double resid = 0.0;
    // A mu^k = B mu^{k+1} - A mu^{k+2} + seed   (A, B symmetric: same factors as the forward march)
    swap_lambda(h);
    const int ws = h->prm.warm_start;
    h->prm.warm_start = std::min(ws, 1);   // the extrapolation history belongs to the forward march
    const int status = advance(h, mu_k1, mu_k2, mu_k, seed, +1.0, &iters, &refinements, &resid, s);
    h->prm.warm_start = ws;
    swap_lambda(h);
    if (status != DD_OK && status != DD_ERR_NO_CONVERGENCE) return status;
    h->cur_adj = (h->cur_adj + 1) % 3;
    if (grad_eps) {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_grad_eps(h, mu_k, e_k, e_km1, e_km2, grad_eps, s), "grad eps");
    }
    if (grad_amp && d2g_hat) {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_dot_sub(h, mu_k, d2g_hat, d2g_scale, grad_amp, s), "grad amp");
    }
    if (mu_out) CK(h, (int)cudaMemcpyAsync(mu_out, mu_k, sizeof(double) * h->n_dof, cudaMemcpyDeviceToDevice, s), "mu_out");
    if (stats) {
        stats->iters = iters;
        stats->refinements = refinements;
        stats->resid = resid;
        stats->status = status;
    }
    return status;
}

int dd_probe_seed(dd_handle* h, const double* e, double weight, double* seed, void* stream) {
    if (!h || !e || !seed) return DD_ERR_ARG;
    if (h->members > 1) return h->fail(DD_ERR_STATE, "dd_probe_seed is not available for an ensemble (members > 1)");
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    CK(h, (int)cudaMemsetAsync(seed, 0, sizeof(double) * h->n_dof, s), "memset");
    Prof P(h, ST_VEC, s, 1);
    CK(h, launch_probe_seed(h, e, weight, seed, s), "probe seed");
    return DD_OK;
}

int dd_probe_objective(dd_handle* h, const double* e, double weight, double* J, void* stream) {
    if (!h || !J) return DD_ERR_ARG;
    if (h->members > 1) return h->fail(DD_ERR_STATE, "dd_probe_objective is not available for an ensemble (members > 1)");
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    Prof P(h, ST_VEC, s, 1);
    CK(h, launch_probe_objective(h, e ? e : h->d.e[h->cur], weight, J, s), "probe objective");
    return DD_OK;
}

int dd_set_eps(dd_handle* h, const double* eps, void* stream) {
    if (!h || !eps) return DD_ERR_ARG;
    if (h->members > 1) return h->fail(DD_ERR_STATE, "dd_set_eps is not available for an ensemble (members > 1)");
    if (!h->bound) return h->fail(DD_ERR_STATE, "dd_set_eps before dd_bind_workspace");
    if (h->n_tets * 36 >= (int64_t)INT32_MAX) return h->fail(DD_ERR_ARG, "dd_set_eps: mesh too large (36 n_tets >= 2^31)");
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->eps_map_up) {
        std::vector<int64_t> ptr;
        std::vector<int32_t> idx;
        build_eps_map(h, ptr, idx);
        if ((int64_t)idx.size() != h->eps_contrib || ptr.size() != (size_t)h->row_ptr.back() + 1)
            return h->fail(DD_ERR_STATE, "dd_set_eps: mass map does not match the local matrices");
        CK(h, upload(h->d.eps_ptr, ptr, s), "upload");
        CK(h, upload(h->d.eps_idx, idx, s), "upload");
        CK(h, (int)cudaStreamSynchronize(s), "sync");   // ptr, idx are locals
        h->eps_map_up = true;
    }
    drop_graphs(h);
    CK(h, launch_assemble_mass(h, eps, s), "mass assembly");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    h->factored = false;
    return DD_OK;
}

int dd_set_wait_limit(dd_handle* h, int32_t first_wait_polls, void* stream) {
    if (!h || first_wait_polls < 0) return DD_ERR_ARG;
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    CK(h, (int)cudaMemcpyAsync(&h->d.sc->wait_first, &first_wait_polls, sizeof(int32_t), cudaMemcpyHostToDevice, s),
       "wait limit");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    return DD_OK;
}

int dd_schur_apply(dd_handle* h, const double* lam, double* out, void* stream) {
    if (!h || !lam || !out) return DD_ERR_ARG;
    if (h->members > 1) return h->fail(DD_ERR_STATE, "dd_schur_apply is not available for an ensemble (members > 1)");
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_schur_apply before dd_factor");
    if (h->factored_scheme != DD_SCHEME_DP1) return h->fail(DD_ERR_STATE, "dd_schur_apply needs the DP1 factorisation");
    if (h->mult_dof.empty()) return DD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(h, apply_schur_w(h, DD_FP64, X_LAMBDA, lam, nullptr, nullptr, nullptr, false, s), "apply");
    Prof P(h, ST_VEC, s, 1);
    CK(h, launch_jump(h, h->d.w, nullptr, nullptr, 1.0, out, s), "jump");
    return DD_OK;
}

int dd_coupled_apply(dd_handle* h, const double* u, double* out, void* stream) {
    if (!h || !u || !out) return DD_ERR_ARG;
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_coupled_apply before dd_factor");
    if (h->factored_scheme != DD_SCHEME_DP1) return h->fail(DD_ERR_STATE, "dd_coupled_apply needs the DP1 factorisation");
    const size_t nm = h->mult_dof.size(), nc = h->corner_dof.size();
    if (nm + nc == 0) return DD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    {
        Prof P(h, ST_SCHUR, s, 1, mb(h, GEMV_COUPLED, DD_FP64));
        CK(h, launch_gemv(h, GEMV_COUPLED, DD_FP64, xsrc(X_LAMBDA_CV, u, nullptr, nullptr, nullptr, u + nm, nullptr),
                          gout_coupled(h, h->d.w, nullptr), false, s), "coupled operator");
    }
    Prof P(h, ST_VEC, s, 1);
    CK(h, launch_gm_combine(h, uview(h, DD_FP64), u, out, s), "combine");
    return DD_OK;
}

int dd_dp2_apply(dd_handle* h, const double* u, double* out, void* stream) {
    if (!h || !u || !out) return DD_ERR_ARG;
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_dp2_apply before dd_factor");
    if (h->factored_scheme != DD_SCHEME_DP2) return h->fail(DD_ERR_STATE, "dd_dp2_apply needs the DP2 factorisation");
    const size_t nm = h->mult_dof.size(), nc = h->corner_dof.size();
    if (nm + nc == 0) return DD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    {
        Prof P(h, ST_SCHUR, s, 1, mb(h, GEMV_COUPLED, DD_FP64));
        CK(h, launch_gemv(h, GEMV_COUPLED, DD_FP64,
                          xsrc(X_SIDE_CP, u, u + nm, nullptr, nullptr, u + 2 * nm, nullptr),
                          gout_coupled(h, h->d.w, nullptr), false, s), "DP2 operator");
    }
    Prof P(h, ST_VEC, s, 1);
    CK(h, launch_gm_combine(h, uview(h, DD_FP64), u, out, s), "combine");
    return DD_OK;
}

int dd_get_interface_mass(const dd_handle* h, int64_t* nnz, int64_t* ptr, int32_t* col, double* val) {
    if (!h || !nnz) return DD_ERR_ARG;
    *nnz = (int64_t)h->mt_col.size();
    if (ptr && !h->mt_ptr.empty()) std::memcpy(ptr, h->mt_ptr.data(), sizeof(int64_t) * h->mt_ptr.size());
    if (col && !h->mt_col.empty()) std::memcpy(col, h->mt_col.data(), sizeof(int32_t) * h->mt_col.size());
    if (val && !h->mt_val.empty()) std::memcpy(val, h->mt_val.data(), sizeof(double) * h->mt_val.size());
    return DD_OK;
}

int dd_probe(dd_handle* h, double* out, void* stream) {
    if (!h || !out) return DD_ERR_ARG;
    if (!h->bound) return h->fail(DD_ERR_STATE, "dd_probe before dd_bind_workspace");
    Prof P(h, ST_VEC, (cudaStream_t)stream, 1);
    CK(h, launch_probe(h, h->d.e[h->cur], out, (cudaStream_t)stream), "probe");
    return DD_OK;
}

int dd_get_state(const dd_handle* hc, double* e_n, double* e_nm1, int64_t* step, void* stream) {
    dd_handle* h = const_cast<dd_handle*>(hc);
    if (!h) return DD_ERR_ARG;
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = sizeof(double) * h->n_dof;
    if (e_n) CK(h, (int)cudaMemcpyAsync(e_n, h->d.e[h->cur], nb, cudaMemcpyDeviceToDevice, s), "copy");
    if (e_nm1) CK(h, (int)cudaMemcpyAsync(e_nm1, h->d.e[(h->cur + 2) % 3], nb, cudaMemcpyDeviceToDevice, s), "copy");
    if (step) *step = h->step;
    return DD_OK;
}

int dd_set_state(dd_handle* h, const double* e_n, const double* e_nm1, int64_t step, void* stream) {
    if (!h || !e_n || !e_nm1 || step < 0) return DD_ERR_ARG;
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = sizeof(double) * h->n_dof;
    h->cur = 0;
    CK(h, (int)cudaMemcpyAsync(h->d.e[0], e_n, nb, cudaMemcpyDeviceToDevice, s), "copy");
    CK(h, (int)cudaMemcpyAsync(h->d.e[2], e_nm1, nb, cudaMemcpyDeviceToDevice, s), "copy");
    CK(h, (int)cudaMemsetAsync(&h->d.sc->lam_levels, 0, sizeof(int32_t), s), "memset");
    h->step = step;
    h->lam_valid = false;
    return DD_OK;
}

namespace {

// Particles back at their injection data, fields of the PIC coupling zeroed.
int reset_particles(dd_handle* h, cudaStream_t s) {
    if (!h->n_particles) return DD_OK;
    const size_t np = (size_t)h->n_particles, nd = (size_t)h->n_dof;
    CK(h, upload(h->d.px, h->p_x, s), "upload");
    CK(h, upload(h->d.pv, h->p_v, s), "upload");
    CK(h, upload(h->d.pt, h->p_t, s), "upload");
    CK(h, upload(h->d.ptet, h->p_tet, s), "upload");
    CK(h, (int)cudaMemsetAsync(h->d.pstat, 0, sizeof(int32_t) * np, s), "memset");
    CK(h, (int)cudaMemsetAsync(h->d.bflux, 0, sizeof(double) * (size_t)h->n_faces, s), "memset");
    for (int k = 0; k < 2; ++k) CK(h, (int)cudaMemsetAsync(h->d.dep[k], 0, sizeof(double) * nd, s), "memset");
    CK(h, (int)cudaMemsetAsync(h->d.Gcum, 0, sizeof(double) * nd, s), "memset");
    CK(h, (int)cudaMemsetAsync(h->d.pic_err, 0, 4, s), "memset");
    h->dep_cur = 0;
    return DD_OK;
}

int upload_pic_mesh(dd_handle* h, cudaStream_t s) {
    if (!h->n_particles) return DD_OK;
    std::vector<double> x0(3 * (size_t)h->n_tets);
    for (int64_t t = 0; t < h->n_tets; ++t)
        for (int c = 0; c < 3; ++c) x0[3 * t + c] = h->xyz[3 * (int64_t)h->tets[4 * t] + c];
    CK(h, upload(h->d.tets_dev, h->tets, s), "upload");
    CK(h, upload(h->d.tgrad, h->grad, s), "upload");
    CK(h, upload(h->d.tx0, x0, s), "upload");
    CK(h, upload(h->d.tface, h->tet_face, s), "upload");
    CK(h, upload(h->d.tnbr, h->tet_nbr, s), "upload");
    CK(h, upload(h->d.face_nodes, h->face_nodes, s), "upload");
    CK(h, upload(h->d.face_edge, h->face_edge, s), "upload");
    CK(h, (int)cudaStreamSynchronize(s), "sync");   // x0 is a local
    return reset_particles(h, s);
}

}  // namespace

int dd_set_beam(dd_handle* h, const dd_beam* beam) {
    if (!h || !beam || beam->n_particles < 0 || (beam->n_particles > 0 && (!beam->x_inj || !beam->v_inj || !beam->t_inj)))
        return h ? h->fail(DD_ERR_ARG, "bad beam") : DD_ERR_ARG;
    if (h->bound) return h->fail(DD_ERR_STATE, "dd_set_beam after dd_bind_workspace");
    if (h->members > 1) return h->fail(DD_ERR_STATE, "the PIC cycle is not available for an ensemble (members > 1)");
    return dd_build_beam(h, beam);
}

int dd_pic_step(dd_handle* h, dd_stats* stats, void* stream) {
    if (!h) return DD_ERR_ARG;
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_pic_step before dd_factor");
    if (!h->n_particles) return h->fail(DD_ERR_STATE, "dd_pic_step without dd_set_beam");
    cudaStream_t s = (cudaStream_t)stream;
    const double t_n = (double)h->step * h->dt;
    double* dn = h->d.dep[h->dep_cur];
    const double* dold = h->d.dep[1 - h->dep_cur];
    const double* e_n = h->d.e[h->cur];
    CK(h, (int)cudaMemsetAsync(dn, 0, sizeof(double) * (size_t)h->n_dof, s), "memset");
    {
        Prof P(h, ST_VEC, s, 2);
        CK(h, launch_pic_move(h, t_n, h->dt, e_n, dn, s), "pic move");
        CK(h, launch_pic_source(h, dn, dold, s), "pic source");
    }
    const int rc = dd_step(h, h->d.d2g_pic, nullptr, stats, stream);
    if (rc != DD_OK && rc != DD_ERR_NO_CONVERGENCE) return rc;
    {
        Prof P(h, ST_VEC, s, 1);
        CK(h, launch_faraday(h, h->d.e[h->cur], e_n, h->dt, s), "faraday");
    }
    h->dep_cur = 1 - h->dep_cur;
    if (stats) {
        int32_t err = 0;
        CK(h, (int)cudaMemcpyAsync(&err, h->d.pic_err, 4, cudaMemcpyDeviceToHost, s), "pic err");
        CK(h, (int)cudaStreamSynchronize(s), "sync");
        if (err) return h->fail(DD_ERR_ARG, "a particle crossed more than 64 tets in one step");
    }
    return rc;
}

int dd_pic_state(const dd_handle* hc, double* x, int32_t* status, double* G, double* b, int64_t* n_faces, void* stream) {
    dd_handle* h = const_cast<dd_handle*>(hc);
    if (!h) return DD_ERR_ARG;
    if (n_faces) *n_faces = h->n_faces;
    if (!h->n_particles) return (x || status || G || b) ? h->fail(DD_ERR_STATE, "no beam") : DD_OK;
    if (!h->bound) return h->fail(DD_ERR_STATE, "no workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)h->n_particles;
    if (x) CK(h, (int)cudaMemcpyAsync(x, h->d.px, 3 * np * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    if (status) CK(h, (int)cudaMemcpyAsync(status, h->d.pstat, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, s), "copy");
    if (G) CK(h, (int)cudaMemcpyAsync(G, h->d.Gcum, (size_t)h->n_dof * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    if (b) CK(h, (int)cudaMemcpyAsync(b, h->d.bflux, (size_t)h->n_faces * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    return DD_OK;
}

int dd_autotune(dd_handle* h, const char* cache_path, double* seconds, void* stream) {
    if (!h) return DD_ERR_ARG;
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_autotune before dd_factor");
    if (h->capturing) return h->fail(DD_ERR_STATE, "dd_autotune during capture");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    CK(h, (int)cudaGetDevice(&dev), "device");
    cudaDeviceProp prop;
    CK(h, (int)cudaGetDeviceProperties(&prop, dev), "device properties");
    std::string key = std::string(prop.name) + "|" + std::to_string(h->n_sub) + "|" + std::to_string(h->n_dof) + "|" +
                      std::to_string(h->sub_ptr.back()) + "|" + std::to_string(h->corner_dof.size()) + "|" +
                      std::to_string(h->max_ns);
    for (char& c : key)
        if (c == ' ' || c == '\t') c = '_';
    std::map<std::pair<int, int>, TileCfg> found;
    struct SymCfg {
        int cl, st, keep, ws;
    };
    std::map<int, SymCfg> found_cl;   // packed symmetric modes: CTAs per subdomain, ring depth, subdomains kept
                                      // in L2, kernel form; cache lines "key 2 mode cl st keep ws"
    int n_sym = 0;
    for (int m = 0; m < GEMV_NMODES; ++m) {
        if (sym_active(h, m)) ++n_sym;
    }
    if (cache_path && *cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream is(line);
            std::string k;
            int p, m, lpr, rows;
            if (!(is >> k >> p >> m >> lpr >> rows) || k != key || m < 0 || m >= GEMV_NMODES) continue;
            if (p >= 0 && p < 2 && (lpr == 8 || lpr == 16 || lpr == 32) && rows >= kMinRowsPerTask)
                found[{p, m}] = TileCfg{lpr, rows};
            int keep = 0, ws = 0;
            if (p == 2 && sym_active(h, m) && rows >= 2 && (is >> keep >> ws) && keep >= 0 && keep <= h->n_sub &&
                ((ws <= 3 && (lpr == 1 || lpr == 2 || lpr == 4 || lpr == 8) && rows <= kSymStages) ||
                 (ws == 4 && tc_available(h, m) && lpr == 1 && rows <= kSymStages) ||
                 (ws == 5 && h->members <= 1 && (lpr == 1 || lpr == 2 || lpr == 4) && rows % lpr == 0 &&
                  rows <= kSymStagesPs)))
                found_cl[m] = SymCfg{lpr, rows, keep, ws};
        }
    }
    const bool cached = found.size() == (size_t)(2 * GEMV_NMODES) && found_cl.size() == (size_t)n_sym;
    cudaEvent_t e0, e1;
    CK(h, (int)cudaEventCreate(&e0), "event");
    CK(h, (int)cudaEventCreate(&e1), "event");
    const auto t_start = std::chrono::steady_clock::now();
    int rc = DD_OK;
    const size_t nl = (size_t)h->sub_ptr.back(), nc = h->corner_dof.size();
    if (!cached) {
        // time every candidate tile on the real operators (inputs zero: timing only)
        rc = (int)cudaMemsetAsync(h->d.b, 0, sizeof(double) * nl, s);
        if (!rc) rc = (int)cudaMemsetAsync(h->d.bf, 0, sizeof(float) * nl, s);
        if (!rc && nc) rc = (int)cudaMemsetAsync(h->d.uC, 0, sizeof(double) * nc, s);
        if (!rc && nc) rc = (int)cudaMemsetAsync(h->d.uCf, 0, sizeof(float) * nc, s);
        const int lprs[3] = {8, 16, 32};
        const int rowss[5] = {8, 16, 32, 64, 128};
        for (int p = 0; p < 2 && !rc; ++p) {
            const int prec = p == 0 ? DD_FP64 : DD_MIXED;
            for (int m = 0; m < GEMV_NMODES && !rc; ++m) {
                const bool sym_saved = h->prm.sym_fp32 != 0;
                if (p == 1 && h->sym_ok && sym_active(h, m)) {
                    // packed symmetric tiles: time both kernel forms with 1, 2, 4 and 8 CTAs per subdomain and
                    // rings of 2, 3 and 4 tiles
                    h->prm.sym_fp32 = 1;
                    XSrc xs{};
                    xs.kind = X_FLAT;
                    xs.v = h->d.b;
                    xs.vf = h->d.bf;
                    const GemvOut go{nullptr, nullptr, h->d.wf, nullptr, 1.0};
                    // then, for the kinds a Krylov solve repeats, how many subdomains' tiles to keep in
                    // L2 (evict_last) across launches: 0, 32, 64 or 96 MB worth
                    float best = 1e30f;
                    SymCfg bcl{h->sym_cl[m], h->sym_st[m], 0, 0};
                    const bool repeated = m != GEMV_LOCAL;
                    const double per_sub = h->mode_bytes_sym[m] / std::max(1, h->n_sub);
                    // kernel forms: CTA-synchronous, warp-specialised and, for an ensemble whose
                    // shared memory allows it, the copies of a subdomain in one CTA
                    const bool form2 = h->members > 1 && sym_smem_bytes_nr(h, h->members <= 2 ? 2 : 4) <= 227 * 1024;
                    const bool form3 = h->members > 2 && sym_smem_bytes_nr(h, 2) <= 227 * 1024;
                    const int nsweep = 12 * (form3 ? 4 : (form2 ? 3 : 2));
                    const int ntc = tc_available(h, m) ? 1 : 0;   // the tensor-core form (one configuration)
                    // the persistent form (single problems): 1, 2 or 4 consumer groups, rings of 2 to 10 tiles
                    const int nps = h->members <= 1 ? 15 : 0;
                    for (int cand = 0; cand < nsweep + ntc + nps + (repeated ? 3 : 0) && !rc; ++cand) {
                        int cl, st, keep = 0, ws;
                        if (cand < nsweep) {
                            ws = cand / 12;
                            cl = 1 << ((cand % 12) / 3);
                            st = 2 + cand % 3;
                        } else if (cand < nsweep + ntc) {
                            ws = 4;
                            cl = 1;
                            st = 2;
                        } else if (cand < nsweep + ntc + nps) {
                            const int q = cand - nsweep - ntc;
                            ws = 5;
                            cl = 1 << (q / 5);
                            st = 2 + 2 * (q % 5);
                        } else if (bcl.ws == 4) {
                            break;   // no L2-kept subset for the tensor-core form
                        } else {
                            cl = bcl.cl;
                            st = bcl.st;
                            ws = bcl.ws;
                            keep = std::min(h->n_sub, (int)((cand - nsweep - ntc - nps + 1) * 32.0e6 / std::max(1.0, per_sub)));
                        }
                        h->sym_st[m] = st;
                        h->sym_keep[m] = keep;
                        h->sym_ws[m] = ws;
                        sym_ranges(h, m, cl);
                        if (ws == 5 && h->sym_grid[m] < 1) continue;   // no room, or fewer slots than groups
                        rc = upload(h->d.sym_rng[m], h->sym_rng[m], s);
                        // one warm-up and eight timed launches: the forms are often within a few per cent
                        for (int it = 0; it < 9 && !rc; ++it) {
                            if (it == 1) rc = (int)cudaEventRecord(e0, s);
                            if (!rc) rc = launch_gemv(h, m, DD_MIXED, xs, go, false, s);
                        }
                        if (!rc) rc = (int)cudaEventRecord(e1, s);
                        if (!rc) rc = (int)cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (!rc) rc = (int)cudaEventElapsedTime(&ms, e0, e1);
                        h->launches[ST_FACTOR] += 9;
                        h->total_launches += 9;
                        if (rc) break;
                        if (wait_err_set(h, s)) {   // a bounded wait gave up: not a candidate
                            rc = (int)cudaMemsetAsync(&h->d.sc->wait_err, 0, sizeof(int32_t), s);
                            if (rc) break;
                            continue;
                        }
                        if (ms < best) {
                            best = ms;
                            bcl = SymCfg{cl, st, keep, ws};
                        }
                    }
                    found_cl[m] = bcl;
                    if (rc) {
                        h->prm.sym_fp32 = sym_saved ? 1 : 0;
                        break;
                    }
                }
                h->prm.sym_fp32 = 0;   // the dense tiles below time the dense kernel
                if (h->tasks[p][m].empty()) {
                    found[{p, m}] = h->tile[p][m];
                    h->prm.sym_fp32 = sym_saved ? 1 : 0;
                    continue;
                }
                const bool co = m == GEMV_COARSE;
                XSrc xs{};
                xs.kind = X_FLAT;
                xs.v = co ? h->d.uC : h->d.b;
                xs.vf = co ? h->d.uCf : h->d.bf;
                GemvOut go = p == 0 ? GemvOut{co ? h->d.vC : h->d.x, nullptr, nullptr, nullptr, 1.0}
                                    : GemvOut{nullptr, nullptr, co ? h->d.vCf : h->d.wf, nullptr, 1.0};
                float best = 1e30f;
                TileCfg bt = h->tile[p][m];
                for (int li = 0; li < 3 && !rc; ++li)
                    for (int ri = 0; ri < 5 && !rc; ++ri) {
                        h->tile[p][m] = TileCfg{lprs[li], rowss[ri]};
                        build_tasks(h, m, rowss[ri], h->tasks[p][m]);
                        const int urc = upload_tasks(h, p, m, s);
                        if (urc) {
                            cudaEventDestroy(e0);
                            cudaEventDestroy(e1);
                            return urc == DD_ERR_CUDA ? h->fail(DD_ERR_CUDA, "upload tasks") : urc;
                        }
                        for (int it = 0; it < 4 && !rc; ++it) {
                            if (it == 1) rc = (int)cudaEventRecord(e0, s);
                            if (!rc) rc = launch_gemv(h, m, prec, xs, go, false, s);
                        }
                        if (!rc) rc = (int)cudaEventRecord(e1, s);
                        if (!rc) rc = (int)cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (!rc) rc = (int)cudaEventElapsedTime(&ms, e0, e1);
                        h->launches[ST_FACTOR] += 4;
                        h->total_launches += 4;
                        if (!rc && ms < best) {
                            best = ms;
                            bt = h->tile[p][m];
                        }
                    }
                found[{p, m}] = bt;
                h->prm.sym_fp32 = sym_saved ? 1 : 0;
            }
        }
        if (!rc && cache_path && *cache_path) {
            std::ofstream f(cache_path, std::ios::app);
            for (const auto& kv : found)
                f << key << "\t" << kv.first.first << "\t" << kv.first.second << "\t" << kv.second.lpr << "\t"
                  << kv.second.rows << "\n";
            for (const auto& kv : found_cl)
                f << key << "\t2\t" << kv.first << "\t" << kv.second.cl << "\t" << kv.second.st << "\t"
                  << kv.second.keep << "\t" << kv.second.ws << "\n";
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return cuda_fail(h, rc, "autotune");
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < GEMV_NMODES; ++m) {
            h->tile[p][m] = found[{p, m}];
            build_tasks(h, m, h->tile[p][m].rows, h->tasks[p][m]);
            const int urc = upload_tasks(h, p, m, s);
            if (urc) return urc == DD_ERR_CUDA ? h->fail(DD_ERR_CUDA, "upload tasks") : urc;
        }
    for (const auto& kv : found_cl) {
        h->sym_st[kv.first] = kv.second.st;
        h->sym_keep[kv.first] = kv.second.keep;
        h->sym_ws[kv.first] = kv.second.ws;
        sym_ranges(h, kv.first, kv.second.cl);
        CK(h, upload(h->d.sym_rng[kv.first], h->sym_rng[kv.first], s), "upload ranges");
    }
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    drop_graphs(h);
    h->tuned = true;
    if (seconds)
        *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return DD_OK;
}

int dd_get_gemv_bytes(const dd_handle* h, int32_t kind, int32_t precision, double* algorithmic, double* streamed) {
    if (!h || kind < 0 || kind >= GEMV_NMODES || (precision != DD_FP64 && precision != DD_MIXED)) return DD_ERR_ARG;
    const double alg = mb(h, kind, precision);
    double str = alg;
    if (precision == DD_MIXED && h->prm.sym_fp32 && h->sym_ok && sym_active(h, kind) && h->mode_tile_bytes_sym[kind] > 0.0)
        str = h->mode_tile_bytes_sym[kind];
    if (algorithmic) *algorithmic = alg;
    if (streamed) *streamed = str;
    return DD_OK;
}

int dd_get_tiles(const dd_handle* h, int32_t* lpr, int32_t* rows) {
    if (!h || !lpr || !rows) return DD_ERR_ARG;
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < GEMV_NMODES; ++m) {
            lpr[p * GEMV_NMODES + m] = h->tile[p][m].lpr;
            rows[p * GEMV_NMODES + m] = h->tile[p][m].rows;
        }
    return DD_OK;
}

int dd_get_sym_config(const dd_handle* h, int32_t* cl, int32_t* st, int32_t* keep, int32_t* ws) {
    if (!h) return DD_ERR_ARG;
    for (int m = 0; m < GEMV_NMODES; ++m) {
        const bool on = sym_active(h, m);
        if (cl) cl[m] = on ? h->sym_cl[m] : 0;
        if (st) st[m] = on ? h->sym_st[m] : 0;
        if (keep) keep[m] = on ? h->sym_keep[m] : 0;
        if (ws) ws[m] = on ? h->sym_ws[m] : 0;
    }
    return DD_OK;
}

int dd_set_sym_config(dd_handle* h, int32_t kind, int32_t cl, int32_t st, int32_t keep, int32_t ws, void* stream) {
    if (!h) return DD_ERR_ARG;
    if (kind < 0 || kind >= GEMV_NMODES || !sym_active(h, kind))
        return h->fail(DD_ERR_ARG, "dd_set_sym_config: not a packed GEMV kind");
    if (ws == 5) {
        if (!(cl == 1 || cl == 2 || cl == 4) || st < 2 || st % cl != 0 || st > kSymStagesPs || keep < 0 ||
            keep > h->n_sub)
            return h->fail(DD_ERR_ARG, "dd_set_sym_config: the persistent form takes cl (consumer groups) in {1,2,4}, "
                                       "2 <= st <= 10 a multiple of cl, 0 <= keep <= n_sub");
        if (h->members > 1) return h->fail(DD_ERR_ARG, "dd_set_sym_config: the persistent form serves single problems");
    } else if (!(cl == 1 || cl == 2 || cl == 4 || cl == 8) || st < 2 || st > kSymStages || keep < 0 ||
               keep > h->n_sub || ws < 0 || ws > 4) {
        return h->fail(DD_ERR_ARG, "dd_set_sym_config: cl in {1,2,4,8}, 2 <= st <= 4, 0 <= keep <= n_sub, ws in {0..5}");
    }
    if (ws == 4 && !tc_available(h, kind))
        return h->fail(DD_ERR_ARG, "dd_set_sym_config: the tensor-core form needs an ensemble and a local solve, "
                                   "recovery or coupled kind");
    if ((ws == 2 && sym_smem_bytes_nr(h, h->members <= 2 ? 2 : 4) > 227 * 1024) ||
        (ws == 3 && sym_smem_bytes_nr(h, 2) > 227 * 1024))
        return h->fail(DD_ERR_ARG, "dd_set_sym_config: the ensemble form needs more shared memory than a CTA has");
    if (!h->bound) return h->fail(DD_ERR_STATE, "dd_set_sym_config before dd_bind_workspace");
    if (h->capturing) return h->fail(DD_ERR_STATE, "dd_set_sym_config during capture");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t old_st = h->sym_st[kind], old_keep = h->sym_keep[kind], old_ws = h->sym_ws[kind], old_cl = h->sym_cl[kind];
    h->sym_st[kind] = st;
    h->sym_keep[kind] = keep;
    h->sym_ws[kind] = ws;
    sym_ranges(h, kind, cl);
    if (ws == 5 && h->sym_grid[kind] < 1) {
        h->sym_st[kind] = old_st;
        h->sym_keep[kind] = old_keep;
        h->sym_ws[kind] = old_ws;
        sym_ranges(h, kind, old_cl);
        return h->fail(DD_ERR_ARG, "dd_set_sym_config: the persistent form's ring and buffers need more shared "
                                   "memory than one CTA can have");
    }
    CK(h, upload(h->d.sym_rng[kind], h->sym_rng[kind], s), "upload ranges");
    CK(h, (int)cudaStreamSynchronize(s), "sync");
    drop_graphs(h);
    return DD_OK;
}

int dd_profile(dd_handle* h, int enable, dd_profile_stats* out, void* stream) {
    if (!h) return DD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (out) {
        CK(h, (int)cudaStreamSynchronize(s), "sync");
        std::memset(out, 0, sizeof(*out));
        for (int k = 0; k < DD_N_STAGES; ++k) {
            out->launches[k] = h->launches[k];
            out->work[k] = h->work[k];
            out->bytes[k] = h->work_bytes[k];
        }
        for (const auto& rec : h->prof_recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, (cudaEvent_t)h->ev_pool[rec.second], (cudaEvent_t)h->ev_pool[rec.second + 1]) ==
                cudaSuccess)
                out->ms[rec.first] += ms;
        }
        out->total_launches = h->total_launches;
    }
    if (enable == 1 || enable == 0) {
        CK(h, (int)cudaStreamSynchronize(s), "sync");
        h->prof_recs.clear();
        h->ev_used = 0;
        if (enable == 1) {
            for (int k = 0; k < DD_N_STAGES; ++k) {
                h->launches[k] = h->work[k] = 0;
                h->work_bytes[k] = 0.0;
            }
            h->total_launches = 0;
        }
        h->prof_on = enable == 1;
    }
    return DD_OK;
}

void dd_destroy(dd_handle* h) {
    if (!h) return;
    drop_graphs(h);
    for (void* st : h->gstream)
        if (st) cudaStreamDestroy((cudaStream_t)st);
    for (void* e : h->ev_pool) cudaEventDestroy((cudaEvent_t)e);
    delete h;
}

const char* dd_last_error(const dd_handle* h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
