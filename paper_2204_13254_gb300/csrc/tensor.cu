// Tensor-core (tcgen05) GEMV of the ensembles and its self-check.
//
// Ensemble GEMV (kernel form 4 of the local solve, the recovery and the coupled
// operator when members > 1): one CTA applies a subdomain's operator rectangle
// to the x of up to 16 ensemble copies at once as a sequence of MMAs
// D[128 x 16] += A[128 x 64] X[64 x 16], A a panel of the operator (TcDesc), X
// the members' x over the panel's 64 columns, D the members' y over the panel's
// 128 rows, accumulated in tensor memory over the column blocks.  Precision:
// the operator is stored as three BF16 pieces A1 + A2 + A3 and every x as three
// pieces X1 + X2 + X3 (each piece the BF16 rounding of what the previous ones
// leave), and the six products A1X1, A1X2, A1X3, A2X1, A2X2, A3X1 -- every term
// down to 2^-16 relative -- are accumulated in FP32, which reproduces an FP32
// GEMV to its own rounding level.  Roles (warp-specialised, 128 threads):
// warp 0 streams the 48 KB panel blocks into a two-deep ring with bulk copies,
// warp 1 issues the MMAs (one thread) and frees ring slots and x buffers with
// tcgen05.commit, warps 2-3 split the next column block's x into BF16 pieces
// (double-buffered); then all four warps read the accumulators (32 lanes each)
// and store y.  Every wait is bounded; a wait that gives up sets the error word,
// stops its role, and the CTA still drains its copies and frees its tensor
// memory.
//
// dd_tc_selftest runs one 128 x 16 x 64 BF16 MMA with an FP32 accumulator in
// tensor memory, for the operand layouts the library uses, on integer-valued
// inputs whose exact products and sums the FP32 accumulator holds, and compares
// every element with the same sums formed by the CUDA cores.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "dd_internal.h"
#include "tcgen05.cuh"
#include "xsrc.cuh"

namespace {

constexpr int kM = 128, kN = 16, kK = 64;
constexpr unsigned kPolls = 1u << 20;

__device__ int g_tc_result;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (unsigned k = 0; k < kPolls; ++k) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(tc::smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ float a_val(int r, int k) { return (float)((r * 3 + k * 5) % 7 - 3); }
__device__ __forceinline__ float b_val(int n, int k) { return (float)((n * 7 + k) % 5 - 2); }

// variant 0: A K-major; variants 1, 2: A stored M-major (transposed operand),
// core matrix (m / 8, k / 8) at ((k / 8) * 16 + m / 8) * 128 bytes with 16
// contiguous bytes along M, described with (LBO, SBO) = (K step, M step) or
// (M step, K step).  B is K-major throughout.
__global__ void __launch_bounds__(128) k_tc_selftest(int variant) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(sm);              // 64 KB region (16 KB used)
    __nv_bfloat16* B = reinterpret_cast<__nv_bfloat16*>(sm + 65536);      // 2 KB
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 65536 + 2048);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 65536 + 2048 + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 65536 / 2; i += 128) A[i] = __float2bfloat16(0.0f);
    __syncthreads();
    for (int i = tid; i < kM * kK; i += 128) {
        const int r = i / kK, k = i % kK;
        uint32_t off;
        if (variant == 0) off = tc::kmajor_off(r, k, kK);
        else off = (uint32_t)(((k >> 3) * (kM >> 3) + (r >> 3)) * 128 + (k & 7) * 16 + (r & 7) * 2);
        A[off / 2] = __float2bfloat16(a_val(r, k));
    }
    for (int i = tid; i < kN * kK; i += 128) {
        const int n = i / kK, k = i % kK;
        B[tc::kmajor_off(n, k, kK) / 2] = __float2bfloat16(b_val(n, k));
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(tslot, 32);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(kM, kN, variant != 0, false);
        for (int s = 0; s < kK / 16; ++s) {
            uint64_t ad;
            if (variant == 0) ad = tc::smem_desc(tc::smem_addr(A) + s * 256, 128, (kK / 8) * 128);
            else if (variant == 1) ad = tc::smem_desc(tc::smem_addr(A) + s * 2 * (kM / 8) * 128, (kM / 8) * 128, 128);
            else ad = tc::smem_desc(tc::smem_addr(A) + s * 2 * (kM / 8) * 128, 128, (kM / 8) * 128);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(B) + s * 256, 128, (kK / 8) * 128);
            tc::mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
    }
    const bool done = mbar_wait_bounded(bar, 0);
    tc::fence_after_sync();
    int bad = done ? 0 : 1;
    if (done) {
        float d[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), d);
        const int r = 32 * warp + lane;
        for (int n = 0; n < kN; ++n) {
            float ref = 0.0f;
            for (int k = 0; k < kK; ++k) ref += a_val(r, k) * b_val(n, k);
            if (d[n] != ref) ++bad;
        }
    }
    bad = __syncthreads_count(bad != 0);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tmem, 32);
    if (tid == 0) g_tc_result = bad;
}

// ---- ensemble GEMV ------------------------------------------------------------

constexpr int kTcST = 2;                                   // ring depth (panel blocks)
constexpr uint32_t kTcPieceBytes = kTcPieceElems * 2;      // 16 KB
constexpr uint32_t kTcBlockBytes = kTcBlockElems * 2;      // 48 KB
constexpr uint32_t kTcXPiece = kTcN * kTcK * 2;            // 2 KB: one BF16 piece of x over a column block
constexpr uint32_t kTcXBuf = 3 * kTcXPiece;                // its three pieces
constexpr size_t kTcSmem = kTcST * kTcBlockBytes + 2 * kTcXBuf + 16 * sizeof(uint64_t) + 16;
constexpr unsigned kTcPolls = 1u << 22;

__device__ __forceinline__ bool tc_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc::smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    for (unsigned k = 0; k < kTcPolls; ++k) {
        if (tc_test(bar, parity)) return true;
        if ((k & 255u) == 255u && *abort) return false;
    }
    return false;
}
__device__ __forceinline__ void tc_bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tc_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

// BF16 bits of round-to-nearest v and the remainder v - that.
__device__ __forceinline__ uint16_t bf16_split(float& v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    v -= __bfloat162float(b);
    return __bfloat16_as_ushort(b);
}

// One CTA: stored subdomain `sub` (blockIdx.x % n_real) and the ensemble copies
// m0 .. m0 + nmem - 1 (group blockIdx.x / n_real).
__global__ void __launch_bounds__(128) k_tc_gemv(const TcDesc* __restrict__ tcd, const SymDesc* __restrict__ descs,
                                                 const uint16_t* __restrict__ Mtc, int n_real, int members, XSrc xs,
                                                 GemvOut go, const int32_t* __restrict__ skip, int32_t* __restrict__ err) {
    if (skip && *skip) return;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    unsigned char* xbuf = smem + kTcST * kTcBlockBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(xbuf + 2 * kTcXBuf);
    uint64_t* full = bars;              // [kTcST] block landed
    uint64_t* empty = bars + kTcST;     // [kTcST] its MMAs done
    uint64_t* xfull = bars + 2 * kTcST; // [2] x pieces written
    uint64_t* xfree = xfull + 2;        // [2] their MMAs done
    uint64_t* done = xfree + 2;         // every MMA done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sub = blockIdx.x % n_real, m0 = (blockIdx.x / n_real) * kTcN;
    const int nmem = min(kTcN, members - m0);
    const TcDesc td = tcd[sub];
    const int P = td.P, Q = td.Q, nblk = P * Q;
    const uint32_t ncols = P * kTcN <= 32 ? 32 : (P * kTcN <= 64 ? 64 : (P * kTcN <= 128 ? 128 : 256));
    if (tid == 0) {
        for (int i = 0; i < kTcST; ++i) {
            tc_bar_init(&full[i], 1);
            tc_bar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc_bar_init(&xfull[i], 64);
            tc_bar_init(&xfree[i], 1);
        }
        tc_bar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint16_t* blocks = Mtc + td.off;
    int issued = 0;   // producer lane

    if (warp == 0) {
        if (lane == 0) {   // producer: panel blocks in (q, p) order
            for (int b = 0; b < nblk; ++b) {
                const int slot = b % kTcST;
                if (b >= kTcST && !tc_wait(&empty[slot], (uint32_t)((b / kTcST) - 1) & 1u, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                tc_load(ring + slot * kTcBlockBytes, blocks + (int64_t)b * kTcBlockElems, kTcBlockBytes, &full[slot]);
                ++issued;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = tc::idesc_bf16_f32(kTcP, kTcN);
            const int pa[6] = {0, 0, 0, 1, 1, 2}, px[6] = {0, 1, 2, 0, 1, 0};
            bool ok = true;
            for (int q = 0; q < Q && ok; ++q) {
                ok = tc_wait(&xfull[q & 1], (uint32_t)(q >> 1) & 1u, &abort_flag);
                if (!ok) break;
                const uint32_t xb = tc::smem_addr(xbuf + (q & 1) * kTcXBuf);
                for (int p = 0; p < P; ++p) {
                    const int b = q * P + p, slot = b % kTcST;
                    ok = tc_wait(&full[slot], (uint32_t)(b / kTcST) & 1u, &abort_flag);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t ab = tc::smem_addr(ring + slot * kTcBlockBytes);
                    for (int c = 0; c < 6; ++c)
                        for (int s = 0; s < kTcK / 16; ++s) {
                            const uint64_t ad = tc::smem_desc(ab + pa[c] * kTcPieceBytes + s * 256, 128, (kTcK / 8) * 128);
                            const uint64_t bd = tc::smem_desc(xb + px[c] * kTcXPiece + s * 256, 128, (kTcK / 8) * 128);
                            tc::mma_bf16(tmem + p * kTcN, ad, bd, idesc, (q > 0 || c > 0 || s > 0) ? 1u : 0u);
                        }
                    tc::mma_commit(&empty[slot]);
                }
                if (!ok) break;
                tc::mma_commit(&xfree[q & 1]);
            }
            if (!ok) abort_flag = 1;
            tc::mma_commit(done);   // arrives once every MMA issued so far has completed
        }
    } else {   // warps 2-3: x of column block q split into three BF16 pieces, members as MMA N
        const int t = tid - 64;
        const float beta = (xs.kind == X_PCG || xs.kind == X_PCG_CV) ? (float)xs.sc->beta : 0.0f;
        for (int q = 0; q < Q; ++q) {
            if (q >= 2 && !tc_wait(&xfree[q & 1], (uint32_t)((q >> 1) - 1) & 1u, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            unsigned char* xq = xbuf + (q & 1) * kTcXBuf;
            for (int i0 = t; i0 < kTcN * kTcK; i0 += 64 * 8) {
                int sl[8], mm[8], cc[8], jj[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 64 * u;
                    const int n = i / kTcK, k = i % kTcK, lj = td.c0 + q * kTcK + k;
                    const bool need = i < kTcN * kTcK && n < nmem && lj < td.c1;
                    const int64_t slot = need ? descs[sub + (m0 + n) * n_real].voff + lj : 0;
                    sl[u] = (int)slot;
                    jj[u] = need ? lj : -1;
                    mm[u] = need ? xs.slot_mult[slot] : 0;
                    cc[u] = need ? xs.slot_corner[slot] : -1;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 64 * u;
                    if (i >= kTcN * kTcK) continue;
                    float v = jj[u] >= 0 ? xref_value(xsrc_ref_f(xs, mm[u], cc[u], sl[u], jj[u]), beta) : 0.0f;
                    const uint32_t o = tc::kmajor_off(i / kTcK, i % kTcK, kTcK);
#pragma unroll
                    for (int piece = 0; piece < 3; ++piece)
                        *reinterpret_cast<uint16_t*>(xq + piece * kTcXPiece + o) = bf16_split(v);
                }
            }
            tc::fence_proxy_async();
            tc_arrive(&xfull[q & 1]);
        }
    }
    // epilogue: y of the panel rows for the members of this CTA
    const bool all_done = tc_wait(done, 0u, &abort_flag);
    tc::fence_after_sync();
    const bool good = __all_sync(0xffffffffu, all_done) && !abort_flag;
    __syncwarp();
    if (!good) {
        if (lane == 0) atomicExch(err, 1);
    } else {
        for (int p = 0; p < P; ++p) {
            float d[kTcN];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + p * kTcN, d);
            const int li = td.r0 + p * kTcP + 32 * warp + lane;
            if (li >= td.r1) continue;
            for (int n = 0; n < nmem; ++n) {
                const int64_t o = descs[sub + (m0 + n) * n_real].voff + li;
                const int64_t oo = go.pos ? (int64_t)go.pos[o] : o;
                const float v = d[n];
                if (go.out32) {
                    float w = (float)go.alpha * v;
                    if (go.base32) w += go.base32[o];
                    go.out32[oo] = w;
                }
                if (go.out) {
                    double w = (double)v;
                    if (go.alpha != 1.0) w *= go.alpha;
                    if (go.base) w += go.base[o];
                    go.out[oo] = w;
                }
            }
        }
    }
    // copies still in flight land before the CTA ends (bounded), then tensor memory is freed
    if (warp == 0 && lane == 0 && abort_flag) {
        for (int b = max(0, issued - kTcST); b < issued; ++b) {
            for (unsigned k = 0; k < kTcPolls; ++k)
                if (tc_test(&full[b % kTcST], (uint32_t)(b / kTcST) & 1u)) break;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tmem, ncols);
}

// Pack: one CTA per panel block (directory entry): the three BF16 pieces of the
// FP64 swept matrix over the block's 128 x 64 elements, zeros outside the mode's rectangle.
struct TcTabs {
    const TcDesc* t[kTcKinds];
};

__global__ void __launch_bounds__(256) k_tc_pack(TcTabs tabs, const MatDesc* __restrict__ mats,
                                                 const int32_t* __restrict__ dir, const double* __restrict__ M,
                                                 uint16_t* __restrict__ Mtc) {
    const int32_t* dr = dir + 4 * (int64_t)blockIdx.x;
    const int kind = dr[0], s = dr[1], p = dr[2], q = dr[3];
    const TcDesc td = tabs.t[kind][s];
    const MatDesc md = mats[s];
    uint16_t* out = Mtc + td.off + (int64_t)(q * td.P + p) * kTcBlockElems;
    for (int e = threadIdx.x; e < kTcPieceElems; e += blockDim.x) {
        const int r = e / kTcK, k = e % kTcK;
        const int li = td.r0 + p * kTcP + r, lj = td.c0 + q * kTcK + k;
        double m = (li < td.r1 && lj < td.c1) ? M[md.moff + (int64_t)li * md.ld + lj] : 0.0;
        const uint32_t o = tc::kmajor_off(r, k, kTcK) / 2;
#pragma unroll
        for (int piece = 0; piece < 3; ++piece) {
            const __nv_bfloat16 b = __double2bfloat16(m);
            m -= (double)__bfloat162float(b);
            out[piece * kTcPieceElems + o] = __bfloat16_as_ushort(b);
        }
    }
}

}  // namespace

// Host: per tensor-core kind and stored subdomain, the rectangle, its panels and
// their place in the BF16 storage; the directory of panel blocks for packing.
void build_tc(dd_handle* h) {
    h->tc_dir.clear();
    h->tc_elems = 0;
    for (int k = 0; k < kTcKinds; ++k) h->tcd[k].clear();
    if (h->members <= 1) return;
    const int modes[kTcKinds] = {GEMV_LOCAL, GEMV_RECOVER, GEMV_COUPLED};
    for (int k = 0; k < kTcKinds; ++k) {
        h->tcd[k].resize(h->n_sub_real);
        for (int s = 0; s < h->n_sub_real; ++s) {
            const MatDesc& md = h->mats[s];
            TcDesc td{};
            switch (modes[k]) {
                case GEMV_LOCAL: td.r0 = 0; td.r1 = md.ns; td.c0 = 0; td.c1 = md.nr; break;
                case GEMV_RECOVER: td.r0 = 0; td.r1 = md.nr; td.c0 = md.nI; td.c1 = md.ns; break;
                default: td.r0 = md.nI; td.r1 = md.ns; td.c0 = md.nI; td.c1 = md.ns; break;
            }
            td.P = (td.r1 - td.r0 + kTcP - 1) / kTcP;
            td.Q = (td.c1 - td.c0 + kTcK - 1) / kTcK;
            td.off = h->tc_elems;
            h->tc_elems += (int64_t)td.P * td.Q * kTcBlockElems;
            for (int q = 0; q < td.Q; ++q)
                for (int p = 0; p < td.P; ++p) h->tc_dir.insert(h->tc_dir.end(), {k, s, p, q});
            h->tcd[k][s] = td;
        }
    }
}

bool tc_available(const dd_handle* h, int mode) {
    const int k = tc_kind_index(mode);
    if (k < 0 || h->members <= 1 || h->tcd[k].empty()) return false;
    for (const TcDesc& td : h->tcd[k])
        if (td.P * kTcN > 256) return false;   // accumulators beyond one CTA's tensor-memory share
    return true;
}

int launch_tc_pack(const dd_handle* h, void* stream) {
    if (h->tc_dir.empty()) return 0;
    TcTabs tabs{{h->d.tcd[0], h->d.tcd[1], h->d.tcd[2]}};
    k_tc_pack<<<(unsigned)(h->tc_dir.size() / 4), 256, 0, (cudaStream_t)stream>>>(tabs, h->d.mats, h->d.tc_dir,
                                                                                  h->d.M64, h->d.Mtc);
    return (int)cudaGetLastError();
}

int launch_tc_gemv(const dd_handle* h, int mode, XSrc xs, GemvOut go, const int32_t* skip, void* stream) {
    const int k = tc_kind_index(mode);
    if (k < 0 || !tc_available(h, mode)) return (int)cudaErrorInvalidValue;
    xs.slot_mult = h->d.slot_mult;
    xs.slot_corner = h->d.slot_corner;
    xs.sc = h->d.sc;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return (int)e;
    const int groups = (h->members + kTcN - 1) / kTcN;
    k_tc_gemv<<<(unsigned)(h->n_sub_real * groups), 128, kTcSmem, (cudaStream_t)stream>>>(
        h->d.tcd[k], h->d.symd, h->d.Mtc, h->n_sub_real, h->members, xs, go, skip, &h->d.sc->wait_err);
    return (int)cudaGetLastError();
}

extern "C" int dd_tc_selftest(int32_t* passed_mask, void* stream) {
    if (!passed_mask) return DD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int smem = 65536 + 2048 + 16;
    if (cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return DD_ERR_CUDA;
    int mask = 0;
    for (int v = 0; v < 3; ++v) {
        const int minus1 = -1;
        if (cudaMemcpyToSymbolAsync(g_tc_result, &minus1, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return DD_ERR_CUDA;
        k_tc_selftest<<<1, 128, smem, s>>>(v);
        int r = -1;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyFromSymbolAsync(&r, g_tc_result, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return DD_ERR_CUDA;
        if (r == 0) mask |= 1 << v;
    }
    *passed_mask = mask;
    return DD_OK;
}
