// Restarted GMRES on the coupled MFETI-DP1 system of Eqs. F1lr + F1uc (sm_103a).
//
// Unknown u = [lambda; x_c] (n_u = n_lambda + n_corner), right-hand side
// b = [d_r; f~_c], operator
//     M u = [ F_rr u_l + F_rc u_c ; -F_rc^T u_l + K~cc u_c ].
// One application of M is one batched GEMV over the rows and columns
// [Gamma | c] of every swept local matrix (GEMV_COUPLED, x = [B_r^T u_l; -u_c])
// followed by the jump over the multipliers and the negated corner assembly,
// which the first Gram-Schmidt kernel below performs while it reads the
// output.  Preconditioning is on the right with D = diag(M) (the paper's
// diagonal preconditioner): the basis vectors v_j are scaled by D^-1 before
// they enter the GEMV, and x += D^-1 V y at the end of a cycle, so the
// residual tested is the unpreconditioned b - M x.
//
// In DD_MIXED the Krylov vectors (basis, work vector) are FP32, the
// least-squares problem and the iterate FP64.
//
// One Arnoldi step = GEMV + two Gram-Schmidt kernels + one normalisation
// (classical Gram-Schmidt applied twice):
//   pass 0: t = M D^-1 v_j (combine),        h1 = V^T t
//   pass 1: t1 = t - V h1, h2 = V^T t1, ||t1||^2; H[j+1][j] = ||t1 - V h2|| =
//           sqrt(||t1||^2 - ||h2||^2); the last block applies the stored Givens
//           rotations to column j, makes the new one, updates the
//           least-squares residual |g_{j+1}| and decides the end of the cycle
//           (converged, m steps, budget spent, breakdown); at the end it
//           back-substitutes y = R^-1 g.
//   normalise: v_{j+1} = (t1 - V h2) / H[j+1][j], z = D^-1 v_{j+1}.
// Multi-dot products are block partials reduced in fixed block order by the
// last block to finish (atomic ticket, no spinning): results do not depend on
// scheduling.
#include <cuda_runtime.h>

#include "dd_internal.h"

namespace {

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

constexpr int kT = 256;
constexpr int kWarps = kT / 32;
constexpr int kM1 = kMaxRestart + 1;
constexpr int kE = kGmElems;       // vector elements per thread
constexpr int kKB = 8;             // basis vectors loaded per batch
static_assert(kGmChunk == kE * kT, "block chunk of the Krylov vector kernels");

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double wv(const double* __restrict__ w, const float* __restrict__ wf, int64_t slot) {
    return wf ? (double)wf[slot] : w[slot];
}

// Input of the operator in its two multiplier blocks (DP2 needs u1 + u2): FP32
// (DD_MIXED operator input) or FP64.
struct UIn {
    const double* d1;
    const double* d2;
    const float* f1;
    const float* f2;
    __device__ __forceinline__ double sum(int64_t k) const {
        return f1 ? (double)f1[k] + (double)f2[k] : d1[k] + d2[k];
    }
};

// (M u)_i from the coupled operator's GEMV output w (or its FP32 form wf),
// stored as both sides of every multiplier (w[2 m + side]) followed by the
// copies of every corner (w[2 n1 + k], k in [cp[c], cp[c+1])).
// MFETI-DP1: jump over multiplier i; minus the assembly over the copies of a corner.
// MFETI-DP2: u1_k + u2_k - 2 alpha (M_T t)_k with t the interface traces of the
// other side (side 2 for block 1, side 1 for block 2); plus the assembly over
// the copies of a corner (the multipliers enter the local problems with +).
__device__ __forceinline__ double combine(int64_t i, const UView& U, const double* __restrict__ w,
                                          const float* __restrict__ wf, const UIn& in) {
    const int64_t wc = 2 * U.n1;   // first corner copy
    if (!U.mtp) {
        if (i < U.n1) return wv(w, wf, 2 * i) - wv(w, wf, 2 * i + 1);
        const int64_t c = i - U.n1;
        double s = 0.0;
        for (int64_t k = U.cp[c]; k < U.cp[c + 1]; ++k) s += wv(w, wf, wc + k);
        return -s;
    }
    if (i < U.n1 + U.n2) {
        const bool first = i < U.n1;
        const int64_t k = first ? i : i - U.n1;
        const int other = first ? 1 : 0;
        double acc = 0.0;
        for (int64_t p = U.mtp[k]; p < U.mtp[k + 1]; ++p) acc += U.mtv[p] * wv(w, wf, 2 * (int64_t)U.mtc[p] + other);
        return in.sum(k) - U.two_alpha * acc;
    }
    const int64_t c = i - U.n1 - U.n2;
    double s = 0.0;
    for (int64_t k = U.cp[c]; k < U.cp[c + 1]; ++k) s += wv(w, wf, wc + k);
    return s;
}

// combine() of MFETI-DP1 for the E elements i0 + e stride of one thread: the
// multiplier pairs are adjacent in w; a corner's copies are contiguous and
// loaded four at a time.  Same sums in the same order as combine().
template <int E, typename VT>
__device__ __forceinline__ void combine_dp1(int64_t i0, int stride, const UView& U, const double* __restrict__ w,
                                            const float* __restrict__ wf, VT* t) {
    const int64_t nu = U.n1 + U.nc, wc = 2 * U.n1;
    double va[E], vb[E];
    int64_t k0[E], k1[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t i = i0 + (int64_t)e * stride;
        const bool mult = i < U.n1, corner = !mult && i < nu;
        va[e] = mult ? wv(w, wf, 2 * i) : 0.0;
        vb[e] = mult ? wv(w, wf, 2 * i + 1) : 0.0;
        k0[e] = corner ? U.cp[i - U.n1] : 0;
        k1[e] = corner ? U.cp[i - U.n1 + 1] : 0;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t i = i0 + (int64_t)e * stride;
        if (i < U.n1) {
            t[e] = (VT)(va[e] - vb[e]);
        } else if (i < nu) {
            double sum = 0.0;
            for (int64_t k = k0[e]; k < k1[e]; k += 4) {
                double v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = k + q < k1[e] ? wv(w, wf, wc + k + q) : 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (k + q < k1[e]) sum += v[q];
            }
            t[e] = (VT)(-sum);
        } else {
            t[e] = (VT)0;
        }
    }
}

__device__ __forceinline__ double dinv_at(int64_t i, const UView& U) {
    if (i < U.n1) return U.d1 ? U.d1[i] : 1.0;
    if (i < U.n1 + U.n2) return 1.0;
    return U.dc ? U.dc[i - U.n1 - U.n2] : 1.0;
}

__device__ __forceinline__ double b_at(int64_t i, const UView& U) {
    if (i < U.n1) return U.b1[i];
    if (i < U.n1 + U.n2) return U.b2[i - U.n1];
    return U.bc[i - U.n1 - U.n2];
}

// Ticket of a multi-block reduction: every writer thread has fenced its partials
// before the barrier; true in every thread of the last block.
__device__ bool last_block(uint32_t* counter) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// tot[k] = sum over b of partials[k * nb + b] for k < nsum, by the whole block:
// 8 threads per k (b = segment mod 8, up to 8 loads in flight per thread), the
// segments combined by a fixed shuffle tree; fixed order for a given nb.  L2
// loads: the partials were written by other blocks of this launch.
__device__ __forceinline__ void reduce_partials_all(const double* partials, int nsum, int nb, double* tot) {
    const int seg = threadIdx.x & 7;
    for (int k = threadIdx.x >> 3; k - (int)(threadIdx.x >> 3) < nsum; k += kT / 8) {
        const bool own = k < nsum;
        const double* p = partials + (int64_t)(own ? k : 0) * nb;
        double s = 0.0;
        for (int b0 = seg; b0 < nb; b0 += 64) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (own && b0 + 8 * u < nb) ? __ldcg(p + b0 + 8 * u) : 0.0;
            s += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (own && seg == 0) tot[k] = s;
    }
}

// Block sum of one value (all threads call); result in thread 0.
__device__ double block_sum1(double v) {
    __shared__ double red[kWarps];
    v = wsum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kWarps; ++w) s += red[w];
    return s;
}

// K~cc diagonal: sum over the copies of each corner of the local Schur
// complement's diagonal (the corner block of the swept M_s), inverted.
__global__ void k_corner_diag(int64_t nc, const int64_t* __restrict__ cp, const int64_t* __restrict__ cs,
                              const int32_t* __restrict__ slot_sub, const MatDesc* __restrict__ mats,
                              const double* __restrict__ M, double* __restrict__ dinvC) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t k = cp[c]; k < cp[c + 1]; ++k) {
            const int64_t slot = cs[k];
            const MatDesc md = mats[slot_sub[slot]];
            const int64_t row = slot - md.voff;
            s += M[md.moff + row * md.ld + row];
        }
        dinvC[c] = 1.0 / s;
    }
}

// adaptive: a later mixed-precision refinement pass only has to cut the current
// step residual (relative to ||b||) to refine_tol, with a 3x margin.
__global__ void k_gm_init(GmresScalars* gs, const PcgScalars* sc, double tol, double refine_tol, int adaptive,
                          int max_it, int m, unsigned long long cond) {
    if (adaptive) {
        const double resid = sc->norm_b2 > 0.0 ? sqrt(sc->norm_r2 / sc->norm_b2) : 0.0;
        if (resid > 0.0) tol = fmin(0.1, fmax(tol, 0.3 * refine_tol / resid));
    }
    gs->it = 0;
    gs->final = 0;
    gs->converged = 0;
    gs->status = DD_OK;
    gs->cycle_end = 0;
    gs->skip = 0;
    gs->k = 0;
    gs->j = 0;
    gs->tol = tol;
    gs->max_it = max_it;
    gs->m = m;
    gs->cycles = 0;
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 1u);
}

// Start of a cycle: t = b - M x (have_q: w holds the GEMV of x), beta = ||t||,
// ||b||; decides whether the solve is already over.  VT: type of the Krylov
// vectors (double; float for the FP32 inner solves of DD_MIXED, whose tolerance
// is far above FP32 rounding -- GB300's FP64 rate would otherwise make the
// Gram-Schmidt arithmetic a sizeable part of the step).
template <typename VT>
__global__ void __launch_bounds__(kT) k_gm_start(UView U, const double* __restrict__ w, const float* __restrict__ wf,
                                                 int have_q, VT* __restrict__ tu, GmresScalars* gs, PcgScalars* sc,
                                                 double* __restrict__ partials, unsigned long long cond) {
    const int64_t nu = U.n1 + U.n2 + U.nc;
    const UIn in{U.x1, U.n2 ? U.x2 : U.x1, nullptr, nullptr};
    double rr = 0.0, bb = 0.0;
#pragma unroll
    for (int e = 0; e < kGmElems; ++e) {
        const int64_t i = (int64_t)blockIdx.x * kGmChunk + e * kT + threadIdx.x;
        if (i < nu) {
            const double b = b_at(i, U);
            const VT r = (VT)(b - (have_q ? combine(i, U, w, wf, in) : 0.0));
            tu[i] = r;
            rr += (double)r * (double)r;
            bb += b * b;
        }
    }
    rr = block_sum1(rr);
    bb = block_sum1(bb);
    const int nb = gridDim.x;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = rr;
        partials[nb + blockIdx.x] = bb;
    }
    if (!last_block(&gs->counter[0])) return;
    __shared__ double tot[2];
    reduce_partials_all(partials, 2, nb, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        gs->counter[0] = 0u;
        const double beta = sqrt(tot[0]);
        gs->bnorm = sqrt(tot[1]);
        gs->thr = gs->tol * gs->bnorm;
        gs->beta = beta;
        gs->hnext = beta;
        gs->resid = beta;
        gs->g[0] = beta;
        gs->j = 0;
        gs->k = 0;
        gs->nh2 = 0;
        gs->cycles += 1;
        sc->cycles += 1;
        int end = 0;
        if (!isfinite(beta) || !isfinite(gs->bnorm)) {
            gs->status = DD_ERR_NONFINITE;
            end = 1;
        } else if (beta <= gs->thr) {
            gs->converged = 1;
            end = 1;
        } else if (gs->it >= gs->max_it) {
            end = 1;
        }
        gs->final = end;
        gs->cycle_end = end;
        gs->skip = end;
        if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, end ? 0u : 1u);
    }
}

// v_j = (t - sum_k h2_k v_k) / hnext (the second Gram-Schmidt projection of the
// previous column, nh2 terms, none at a cycle start), z = D^-1 v_j: FP64 z for
// the FP64 GEMV, FP32 z for the FP32 one.  The basis entries of a thread's
// elements are loaded kKB vectors at a time, all in flight before any is used.
template <typename VT>
__global__ void __launch_bounds__(kT) k_gm_normalize(UView U, VT* __restrict__ V, int64_t ldv, const VT* __restrict__ tu,
                                                     double* __restrict__ zu, float* __restrict__ zuf,
                                                     const GmresScalars* gs) {
    if (gs->skip) return;
    __shared__ VT coef[kM1];
    const int nh2 = gs->nh2;
    if (threadIdx.x < nh2) coef[threadIdx.x] = (VT)gs->h2[threadIdx.x];
    const int64_t nu = U.n1 + U.n2 + U.nc;
    const int64_t i0 = (int64_t)blockIdx.x * kGmChunk + threadIdx.x;
    VT t[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) t[e] = i0 + e * kT < nu ? tu[i0 + e * kT] : (VT)0;
    __syncthreads();
    for (int k0 = 0; k0 < nh2; k0 += kKB) {
        VT vv[kKB][kE];
#pragma unroll
        for (int q = 0; q < kKB; ++q)
#pragma unroll
            for (int e = 0; e < kE; ++e)
                vv[q][e] = (k0 + q < nh2 && i0 + e * kT < nu) ? V[(int64_t)(k0 + q) * ldv + i0 + e * kT] : (VT)0;
#pragma unroll
        for (int q = 0; q < kKB; ++q)
            if (k0 + q < nh2)
#pragma unroll
                for (int e = 0; e < kE; ++e) t[e] -= coef[k0 + q] * vv[q][e];
    }
    const VT inv = (VT)(1.0 / gs->hnext);
    VT* vj = V + (int64_t)gs->j * ldv;
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        const int64_t i = i0 + e * kT;
        if (i >= nu) continue;
        const VT v = t[e] * inv;
        const VT z = (VT)dinv_at(i, U) * v;
        vj[i] = v;
        if (zu) zu[i] = (double)z;
        if (zuf) zuf[i] = (float)z;
    }
}

// Gram-Schmidt passes of Arnoldi column j (see the file comment).
//   PHASE 0: t = combine(w), h1 = V^T t.
//   PHASE 1: t1 = t - V h1, h2 = V^T t1 and ||t1||^2; the last block takes
//            H[:, j] = h1 + h2 and H[j+1][j] = ||t1 - V h2|| = sqrt(||t1||^2 -
//            ||h2||^2) (V orthonormal; h2 is the small reorthogonalisation
//            correction, applied to the vector by k_gm_normalize), then the
//            Givens rotations and the end-of-cycle logic.
template <int PHASE, typename VT>
__global__ void __launch_bounds__(kT) k_gm_pass(UView U, const double* __restrict__ w, const float* __restrict__ wf,
                                                UIn in, const VT* __restrict__ V, int64_t ldv,
                                                VT* __restrict__ tu, GmresScalars* gs,
                                                PcgScalars* sc, double* __restrict__ partials,
                                                unsigned long long cond) {
    if (gs->skip) return;
    __shared__ VT coef[kM1];
    __shared__ double red[kM1 + 1][kWarps];
    __shared__ double tot[kM1 + 1];
    const int64_t nu = U.n1 + U.n2 + U.nc;
    const int j = gs->j;
    const int nv = j + 1;
    const int nsum = PHASE == 0 ? nv : nv + 1;   // PHASE 1 adds ||t1||^2 as sum nv
    const int nb = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (PHASE == 1 && threadIdx.x < nv) coef[threadIdx.x] = (VT)gs->h1[threadIdx.x];
    const int64_t i0 = (int64_t)blockIdx.x * kGmChunk + threadIdx.x;
    VT t[kE];
    if (PHASE == 0 && !U.mtp) {
        combine_dp1<kE, VT>(i0, kT, U, w, wf, t);
    } else {
#pragma unroll
        for (int e = 0; e < kE; ++e) {
            const int64_t i = i0 + e * kT;
            t[e] = (VT)0;
            if (i < nu) t[e] = PHASE == 0 ? (VT)combine(i, U, w, wf, in) : tu[i];
        }
    }
    __syncthreads();   // coef
    if (PHASE == 1) {   // t1 = t - V h1, kKB basis vectors per batch of loads
        for (int k0 = 0; k0 < nv; k0 += kKB) {
            VT vv[kKB][kE];
#pragma unroll
            for (int q = 0; q < kKB; ++q)
#pragma unroll
                for (int e = 0; e < kE; ++e)
                    vv[q][e] = (k0 + q < nv && i0 + e * kT < nu) ? V[(int64_t)(k0 + q) * ldv + i0 + e * kT] : (VT)0;
#pragma unroll
            for (int q = 0; q < kKB; ++q)
                if (k0 + q < nv)
#pragma unroll
                    for (int e = 0; e < kE; ++e) t[e] -= coef[k0 + q] * vv[q][e];
        }
    }
#pragma unroll
    for (int e = 0; e < kE; ++e)
        if (i0 + e * kT < nu) tu[i0 + e * kT] = t[e];
    // partial dots with v_0 .. v_j (and ||t||^2 in PHASE 1)
    for (int k0 = 0; k0 < nv; k0 += kKB) {
        VT vv[kKB][kE];
#pragma unroll
        for (int q = 0; q < kKB; ++q)
#pragma unroll
            for (int e = 0; e < kE; ++e)
                vv[q][e] = (k0 + q < nv && i0 + e * kT < nu) ? V[(int64_t)(k0 + q) * ldv + i0 + e * kT] : (VT)0;
#pragma unroll
        for (int q = 0; q < kKB; ++q) {
            if (k0 + q < nv) {
                VT p = (VT)0;
#pragma unroll
                for (int e = 0; e < kE; ++e) p += t[e] * vv[q][e];
                p = wsum(p);
                if (lane == 0) red[k0 + q][warp] = (double)p;
            }
        }
    }
    if (PHASE == 1) {
        VT p = (VT)0;
#pragma unroll
        for (int e = 0; e < kE; ++e) p += t[e] * t[e];
        p = wsum(p);
        if (lane == 0) red[nv][warp] = (double)p;
    }
    __syncthreads();
    if (threadIdx.x < nsum) {
        double s = 0.0;
        for (int q = 0; q < kWarps; ++q) s += red[threadIdx.x][q];
        partials[(int64_t)threadIdx.x * nb + blockIdx.x] = s;
        __threadfence();
    }
    if (!last_block(&gs->counter[1 + PHASE])) return;
    reduce_partials_all(partials, nsum, nb, tot);
    __syncthreads();
    if (PHASE == 0) {
        if (threadIdx.x < nv) gs->h1[threadIdx.x] = tot[threadIdx.x];
        if (threadIdx.x == 0) gs->counter[1] = 0u;
        return;
    }
    // Column j of H, its Givens rotations and, at a cycle end, y = R^-1 g: on
    // shared-memory copies of H, the rotations and g that the whole block loads
    // at once (one thread working through global memory would wait for every
    // load in turn).  Same arithmetic in the same order as the sequential
    // definition.
    __shared__ double sH[kMaxRestart * kM1];   // columns 0 .. j
    __shared__ double scs[kMaxRestart], ssn[kMaxRestart], sg[kM1], sy[kMaxRestart];
    __shared__ int s_end, s_k;
    const int tid = threadIdx.x;
    for (int p = tid; p < j * kM1; p += kT) sH[p] = gs->H[p];
    if (tid < j) {
        scs[tid] = gs->cs[tid];
        ssn[tid] = gs->sn[tid];
    }
    if (tid <= j) sg[tid] = gs->g[tid];
    if (tid < nv) {
        gs->h2[tid] = tot[tid];
        sH[j * kM1 + tid] = gs->h1[tid] + tot[tid];
    }
    const int it = gs->it + 1, max_it = gs->max_it, m = gs->m;
    const double thr = gs->thr;
    __syncthreads();
    double* col = sH + j * kM1;
    if (tid == 0) {
        double h2sq = 0.0;
        for (int k = 0; k < nv; ++k) h2sq += tot[k] * tot[k];
        const double hsub = sqrt(fmax(tot[nv] - h2sq, 0.0));
        col[j + 1] = hsub;
        for (int i = 0; i < j; ++i) {
            const double a = col[i], b = col[i + 1];
            col[i] = scs[i] * a + ssn[i] * b;
            col[i + 1] = -ssn[i] * a + scs[i] * b;
        }
        double c = 1.0, s = 0.0;
        {
            const double a = col[j], b = col[j + 1];
            const double r = hypot(a, b);
            if (r != 0.0) {
                c = a / r;
                s = b / r;
            }
        }
        col[j] = c * col[j] + s * col[j + 1];
        col[j + 1] = 0.0;
        gs->cs[j] = c;
        gs->sn[j] = s;
        sg[j + 1] = -s * sg[j];
        sg[j] = c * sg[j];
        gs->g[j + 1] = sg[j + 1];
        gs->g[j] = sg[j];
        gs->it = it;
        sc->it_total += 1;
        const double resid = fabs(sg[j + 1]);
        gs->resid = resid;
        const bool finite = isfinite(resid) && isfinite(hsub) && isfinite(col[j]);
        const bool conv = finite && resid <= thr;
        const bool out_of_budget = it >= max_it;
        const bool end = !finite || conv || out_of_budget || j + 1 == m || hsub == 0.0;
        if (!finite) gs->status = DD_ERR_NONFINITE;
        gs->counter[2] = 0u;
        s_end = end ? 1 : 0;
        s_k = finite ? j + 1 : 0;
        if (end) {
            const int k = s_k;
            for (int i = k - 1; i >= 0; --i) {
                double v = sg[i];
                for (int l = i + 1; l < k; ++l) v -= sH[l * kM1 + i] * sy[l];
                sy[i] = v / sH[i * kM1 + i];
            }
            gs->k = k;
            gs->converged = conv ? 1 : 0;
            gs->final = (!finite || conv || out_of_budget) ? 1 : 0;
            gs->cycle_end = 1;
            gs->skip = 1;
        } else {
            gs->nh2 = nv;
            gs->j = j + 1;
            gs->hnext = hsub;
        }
        if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, end ? 0u : 1u);
    }
    __syncthreads();
    if (tid <= j + 1) gs->H[(int64_t)j * kM1 + tid] = col[tid];
    if (s_end && tid < s_k) gs->y[tid] = sy[tid];
}

// End of a cycle: x += D^-1 V y (x = [lambda; x_c] in place); at the end of the
// solve, publish its outcome in the CG scalars (step statistics, solve end).
template <typename VT>
__global__ void __launch_bounds__(kT) k_gm_update(UView U, const VT* __restrict__ V, int64_t ldv,
                                                  const GmresScalars* gs, PcgScalars* sc, unsigned long long cond) {
    __shared__ VT y[kMaxRestart];
    const int k = gs->k;
    if (threadIdx.x < k) y[threadIdx.x] = (VT)gs->y[threadIdx.x];
    __syncthreads();
    const int64_t nu = U.n1 + U.n2 + U.nc;
    const int64_t i0 = (int64_t)blockIdx.x * kGmChunk + threadIdx.x;
    VT vs[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) vs[e] = (VT)0;
    for (int q0 = 0; q0 < k; q0 += kKB) {
        VT vv[kKB][kE];
#pragma unroll
        for (int q = 0; q < kKB; ++q)
#pragma unroll
            for (int e = 0; e < kE; ++e)
                vv[q][e] = (q0 + q < k && i0 + e * kT < nu) ? V[(int64_t)(q0 + q) * ldv + i0 + e * kT] : (VT)0;
#pragma unroll
        for (int q = 0; q < kKB; ++q)
            if (q0 + q < k)
#pragma unroll
                for (int e = 0; e < kE; ++e) vs[e] += y[q0 + q] * vv[q][e];
    }
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        const int64_t i = i0 + e * kT;
        if (k == 0 || i >= nu) continue;
        const double v = (double)vs[e] * dinv_at(i, U);
        double* x;
        float* xf;
        int64_t o;
        if (i < U.n1) {
            x = U.x1;
            xf = U.x1f;
            o = i;
        } else if (i < U.n1 + U.n2) {
            x = U.x2;
            xf = U.x2f;
            o = i - U.n1;
        } else {
            x = U.xc;
            xf = U.xcf;
            o = i - U.n1 - U.n2;
        }
        const double nx = x[o] + v;
        x[o] = nx;
        if (xf) xf[o] = (float)nx;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (gs->final) {
            sc->status = gs->status;
            sc->done = gs->converged;
            sc->it = gs->it;
            sc->rr = gs->resid * gs->resid;
            sc->gg = gs->bnorm * gs->bnorm;
        }
        if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, gs->final ? 0u : 1u);
    }
}

__global__ void k_gm_combine(UView U, const double* __restrict__ w, const double* __restrict__ in,
                             double* __restrict__ out) {
    const UIn ui{in, U.n2 ? in + U.n1 : in, nullptr, nullptr};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < U.n1 + U.n2 + U.nc;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = combine(i, U, w, nullptr, ui);
}

// MFETI-DP2 right-hand side of the multiplier blocks from y = (A+R)_rr^-1 b_r (per
// slot): b1_k = 2 alpha (M_T t2)_k, b2_k = 2 alpha (M_T t1)_k (traces of the other side).
__global__ void k_dp2_rhs(UView U, const double* __restrict__ y, double* __restrict__ b1, double* __restrict__ b2) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < U.n1; k += (int64_t)gridDim.x * blockDim.x) {
        double a1 = 0.0, a2 = 0.0;
        for (int64_t p = U.mtp[k]; p < U.mtp[k + 1]; ++p) {
            const int64_t l = U.mtc[p];
            a1 += U.mtv[p] * y[U.ms[2 * l + 1]];
            a2 += U.mtv[p] * y[U.ms[2 * l]];
        }
        b1[k] = U.two_alpha * a1;
        b2[k] = U.two_alpha * a2;
    }
}

// MFETI-DP2 Robin term: M_s[i][j] += alpha (M_T)_kl at the slots of multipliers k, l
// in each of their two subdomains (before the local elimination).  Every (k, l)
// entry is distinct, so no two threads write the same matrix element.
__global__ void k_robin_add(int64_t nl, const int64_t* __restrict__ mtp, const int32_t* __restrict__ mtc,
                            const double* __restrict__ mtv, const int64_t* __restrict__ ms,
                            const int32_t* __restrict__ slot_sub, const MatDesc* __restrict__ mats, double alpha,
                            double* __restrict__ M) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nl; k += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = mtp[k]; p < mtp[k + 1]; ++p) {
            const int64_t l = mtc[p];
            for (int side = 0; side < 2; ++side) {
                const int64_t sk = ms[2 * k + side], sl = ms[2 * l + side];
                const MatDesc md = mats[slot_sub[sk]];
                M[md.moff + (sk - md.voff) * md.ld + (sl - md.voff)] += alpha * mtv[p];
            }
        }
}

int vec_blocks(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    if (b > 2 * 152) b = 2 * 152;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int launch_corner_diag(const dd_handle* h, void* stream) {
    const int64_t nc = (int64_t)h->corner_dof.size();
    if (nc == 0) return 0;
    k_corner_diag<<<vec_blocks(nc), kT, 0, S(stream)>>>(nc, h->d.corner_ptr, h->d.corner_slot, h->d.slot_sub, h->d.mats,
                                                       h->d.M64, h->d.dinvC);
    return (int)cudaGetLastError();
}

int launch_gm_init(const dd_handle* h, double tol, int max_it, int m, int adaptive, unsigned long long cond_outer,
                   void* stream) {
    k_gm_init<<<1, 1, 0, S(stream)>>>(h->d.gs, h->d.sc, tol, h->prm.refine_tol, adaptive, max_it, m, cond_outer);
    return (int)cudaGetLastError();
}

int launch_gm_start(const dd_handle* h, const UView& U, int have_q, const float* wf, unsigned long long cond_inner,
                    void* stream) {
    if (wf)
        k_gm_start<float><<<h->gm_blocks, kT, 0, S(stream)>>>(U, h->d.w, wf, have_q, reinterpret_cast<float*>(h->d.tu),
                                                              h->d.gs, h->d.sc, h->d.gpart, cond_inner);
    else
        k_gm_start<double><<<h->gm_blocks, kT, 0, S(stream)>>>(U, h->d.w, nullptr, have_q, h->d.tu, h->d.gs, h->d.sc,
                                                               h->d.gpart, cond_inner);
    return (int)cudaGetLastError();
}

int launch_gm_normalize(const dd_handle* h, const UView& U, float* zuf, void* stream) {
    if (zuf)
        k_gm_normalize<float><<<h->gm_blocks, kT, 0, S(stream)>>>(U, reinterpret_cast<float*>(h->d.Vk), h->gm_ldv,
                                                                   reinterpret_cast<const float*>(h->d.tu), nullptr,
                                                                   zuf, h->d.gs);
    else
        k_gm_normalize<double><<<h->gm_blocks, kT, 0, S(stream)>>>(U, h->d.Vk, h->gm_ldv, h->d.tu, h->d.zu, nullptr,
                                                                    h->d.gs);
    return (int)cudaGetLastError();
}

template <int PHASE, typename VT>
void run_pass(const dd_handle* h, const UView& U, const float* wf, const float* zuf, unsigned long long cond,
              cudaStream_t st) {
    const DevPtrs& d = h->d;
    const UIn in{d.zu, U.n2 ? d.zu + U.n1 : d.zu, zuf, (zuf && U.n2) ? zuf + U.n1 : zuf};
    k_gm_pass<PHASE, VT><<<h->gm_blocks, kT, 0, st>>>(U, d.w, wf, in, reinterpret_cast<const VT*>(d.Vk), h->gm_ldv,
                                                      reinterpret_cast<VT*>(d.tu), d.gs, d.sc, d.gpart, cond);
}

int launch_gm_pass(const dd_handle* h, const UView& U, int phase, const float* wf, const float* zuf,
                   unsigned long long cond_inner, void* stream) {
    const cudaStream_t st = S(stream);
    if (wf) {
        if (phase == 0) run_pass<0, float>(h, U, wf, zuf, 0ull, st);
        else run_pass<1, float>(h, U, wf, zuf, cond_inner, st);
    } else {
        if (phase == 0) run_pass<0, double>(h, U, nullptr, nullptr, 0ull, st);
        else run_pass<1, double>(h, U, nullptr, nullptr, cond_inner, st);
    }
    return (int)cudaGetLastError();
}

int launch_gm_update(const dd_handle* h, const UView& U, unsigned long long cond_outer, void* stream) {
    if (U.x1f || U.xcf)
        k_gm_update<float><<<h->gm_blocks, kT, 0, S(stream)>>>(U, reinterpret_cast<const float*>(h->d.Vk), h->gm_ldv,
                                                                h->d.gs, h->d.sc, cond_outer);
    else
        k_gm_update<double><<<h->gm_blocks, kT, 0, S(stream)>>>(U, h->d.Vk, h->gm_ldv, h->d.gs, h->d.sc, cond_outer);
    return (int)cudaGetLastError();
}

int launch_gm_combine(const dd_handle* h, const UView& U, const double* in, double* out, void* stream) {
    const int64_t nu = U.n1 + U.n2 + U.nc;
    if (nu == 0) return 0;
    k_gm_combine<<<vec_blocks(nu), kT, 0, S(stream)>>>(U, h->d.w, in, out);
    return (int)cudaGetLastError();
}

int launch_dp2_rhs(const dd_handle* h, const UView& U, void* stream) {
    if (U.n1 == 0) return 0;
    k_dp2_rhs<<<vec_blocks(U.n1), kT, 0, S(stream)>>>(U, h->d.y, h->d.g, h->d.g2);
    return (int)cudaGetLastError();
}

int launch_robin_add(const dd_handle* h, double alpha, void* stream) {
    // member 0's multipliers (the first 1/R of them) touch every stored matrix once
    const int64_t nl = (int64_t)h->mult_dof.size() / std::max(1, h->members);
    if (nl == 0) return 0;
    k_robin_add<<<vec_blocks(nl), kT, 0, S(stream)>>>(nl, h->d.mt_ptr, h->d.mt_col, h->d.mt_val, h->d.mult_slot,
                                                     h->d.slot_sub, h->d.mats, alpha, h->d.M64);
    return (int)cudaGetLastError();
}
