// Batched GEMV on packed symmetric FP32 tiles (sm_103a): TMA bulk copies,
// mbarrier ring, one thread-block cluster per subdomain, DSMEM reduction.
//
// The swept local matrix is M_s = J S_s with S_s symmetric, J = diag(I_r, -I_c)
// (A_rr^-1 and the corner Schur complement are symmetric and
// M_s[c][r] = -M_s[r][c]^T), so only the lower triangle of S_s is stored
// (SymDesc: two runs of tile rows, I and [Gamma|c], short last rows, diagonal
// tiles as padded triangles with halved diagonals) and y[R] = J_R (S[R, C] x[C]).
// A stored tile (a, b) acts directly (rows of a, columns of b) and/or
// transposed (rows of b, columns of a): every needed tile is read from HBM once
// for both roles, and no padding of the index groups is streamed.
//
// Work split: the cl CTAs of a cluster (1..kSymCLMax; per mode, like the ring
// depth st <= kSymStages, chosen by dd_autotune) share one subdomain by ranges of
// tile rows (balanced on the host by bytes).  The tiles a mode needs are
// listed once on the host (row order, per subdomain, with their storage
// offsets); a CTA copies its run of that list to shared memory (or reads it
// from global memory where the copy would cost a CTA per SM) and stages only
// the x entries its tile rows read, issuing the index loads of eight entries
// before their value loads.  It streams its tiles through an st-deep ring of
// shared-memory slots filled by cp.async.bulk (one copy per tile, completion on
// an mbarrier) issued by one thread, and accumulates its partial S x over the
// subdomain's padded index range in shared memory:
//  * 128 threads; thread (rg, cq) = (tid / 16, tid % 16) reads rows
//    8 rg .. 8 rg + 7, columns 4 cq .. 4 cq + 3 of the tile with 16-byte
//    loads (a half-warp reads one row's contiguous chunks: no bank conflicts);
//    a full 64 x 64 tile takes an unpredicated path, a short, narrow or
//    diagonal tile a predicated one;
//  * direct role: per-thread row partials stay in registers across the tile
//    row and are reduced over the half-warp (fixed shuffle tree) when the
//    tile row ends;
//  * transposed role: the 8-row column partials of the eight row groups are
//    added in fixed order once per tile.
// The cluster then sums the cl partial vectors through distributed shared
// memory in rank order and applies J.  All sums have a fixed order: results
// are deterministic.  Every mbarrier wait is bounded: a wait that gives up sets
// an error word, the CTA drains its outstanding copies (bounded again) and
// still takes part in both cluster barriers, so no wait can hang the GPU.
//
// Forms (dd_autotune picks one per mode): the CTA-synchronous kernel above, a
// warp-specialised one (producer warp, four consumer warps with their own
// partial y), the ensemble forms (one CTA applying each tile to the x of 2 or 4
// members), and persistent queues (whole subdomains balanced over the SMs'
// CTAs, one ring per queue, helper warps staging x and storing y).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dd_internal.h"
#include "xsrc.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kT = 128;             // threads per CTA: 8 row groups x 16 column quads of a tile
constexpr uint32_t kTileBytes = kSymTile * sizeof(float);
constexpr unsigned kWaitLimit = 1u << 20;   // polls of one mbarrier wait before it gives up (well under a second)

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// L2 policies for the tile copies: evict_last keeps a subset of the operator
// resident in L2 across the launches of one Krylov solve, evict_first streams
// the rest past it.
__device__ __forceinline__ uint64_t l2_policy(bool keep) {
    uint64_t pol;
    if (keep) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// One tile (bytes: a multiple of 16, at most kTileBytes) global -> shared,
// completing on `bar` (which expects the bytes).
__device__ __forceinline__ void load_tile(float* dst, const float* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned limit = kWaitLimit) {
    for (unsigned k = 0; k < limit; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Failure-path test (PcgScalars::wait_first > 0): the CTA's first wait polls
// `never`, an mbarrier no thread or copy ever completes, wait_first times and
// gives up, exercising the give-up / drain / report path with every copy issued.
__device__ __forceinline__ bool first_wait_test(const XSrc& xs, uint64_t* never) {
    const int n = xs.sc ? xs.sc->wait_first : 0;
    return n > 0 ? mbar_wait(never, 0u, (unsigned)n) : true;
}

// Shape of a listed tile: rows, padded width (floats per row of a rectangle),
// diagonal (padded triangle), bytes.
struct TileShape {
    int h, wp;
    bool diag, full;
    uint32_t bytes;
};

// Shape of the tile of list entry word e0, from the subdomain's descriptor.
__device__ __forceinline__ TileShape tile_shape(const SymDesc& sd, uint32_t e) {
    const int a = (int)(e >> 16), b = (int)((e >> 3) & 0x1fff);
    const bool diag = (e & 4) != 0;
    TileShape t;
    t.h = sym_h(sd, a);
    const int w = sym_h(sd, b);
    t.wp = (w + 3) & ~3;
    t.diag = diag;
    t.full = !diag && t.h == kSymT && w == kSymT;
    t.bytes = 4u * (uint32_t)sym_tile_floats(t.h, w, diag);
    return t;
}

// First word of list entry k (the tile's rows, columns and roles): from the
// CTA's copy in shared memory (LSM) or, read-only, from the mode's list in
// global memory.
template <bool LSM>
__device__ __forceinline__ uint32_t tl_word(const uint32_t* tl, int k) {
    return LSM ? tl[kTlW * k] : __ldg(tl + kTlW * k);
}

// Issue the bulk copy of list entry k.
template <bool LSM = false>
__device__ __forceinline__ void issue_tile(const uint32_t* tl, int k, const SymDesc& sd, const float* tiles, float* dst,
                                           uint64_t* bar, uint64_t pol) {
    const uint32_t e0 = tl_word<LSM>(tl, k), e1 = LSM ? tl[kTlW * k + 1] : __ldg(tl + kTlW * k + 1);
    load_tile(dst, tiles + e1, tile_shape(sd, e0).bytes, bar, pol);
}

// Row `row` (0..63), column chunk cq (0..15) of a tile in a ring slot: the four
// floats as a float4, zero outside the stored tile.
__device__ __forceinline__ float4 tile_chunk(const float* slot, const TileShape& t, int row, int cq) {
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (row >= t.h) return z;
    if (t.diag) return 4 * cq < sym_rowlen(row) ? *reinterpret_cast<const float4*>(slot + sym_trioff(row) + 4 * cq) : z;
    return 4 * cq < t.wp ? *reinterpret_cast<const float4*>(slot + row * t.wp + 4 * cq) : z;
}

// Shared-memory layouts (floats unless noted), span = the padded index range
// the mode touches (from its first group on), st = ring depth, nl = longest
// tile list of one CTA:
//   k_symgemv<NR>: ring [st][kSymTile] | x [NR][span] | y [NR][span] | red [2][NR][8][64] |
//                  bars (u64) [kSymStages + 1] | tile list (u32 pairs) [nl] (when LSM)
//   k_symgemv_ws: ring [st][kSymTile] | x [span] | y [4][span] | full, empty (u64) [kSymStages], never (u64) |
//                 tile list (u32 pairs) [nl] (when LSM)
// The CTA copies its run of the tile list to shared memory (LSM) when that
// leaves the CTAs one SM holds unchanged; otherwise it reads the list from
// global memory.
// (the last barrier of each form is the one no copy completes, see first_wait_test)
__host__ __device__ inline size_t sym_smem(int span, int st, int nr = 1, int nl = 0) {
    size_t f = (size_t)st * kSymTile + 2 * (size_t)nr * span + 2 * (size_t)nr * 8 * 64;
    return f * sizeof(float) + (kSymStages + 1) * sizeof(uint64_t) + kTlW * sizeof(uint32_t) * (size_t)nl;
}
__host__ __device__ inline size_t sym_smem_ws(int span, int st, int nl = 0) {
    size_t f = (size_t)st * kSymTile + 5 * (size_t)span;
    return f * sizeof(float) + (2 * kSymStages + 1) * sizeof(uint64_t) + kTlW * sizeof(uint32_t) * (size_t)nl;
}
//   k_symgemv_ps<NG>: ring [st][kSymTile] | x [2][span] | y [2][4 NG][span] | full, empty (u64) [kSymStagesPs],
//                     xfull, ydone (u64) [2], never (u64)
__host__ __device__ inline size_t sym_smem_ps(int span, int st, int ng) {
    size_t f = (size_t)st * kSymTile + 2 * (1 + 4 * (size_t)ng) * span;
    return f * sizeof(float) + (2 * kSymStagesPs + 5) * sizeof(uint64_t);
}

// tile list entry: a << 16 | b << 3 | flags (a, b < 8192), then the tile's float offset
__host__ __device__ __forceinline__ uint32_t tile_entry(int a, int b, int f) { return ((uint32_t)a << 16) | ((uint32_t)b << 3) | f; }

// First padded position a mode touches (the I run only when I is in the mask).
__host__ __device__ inline int mask_lo(const SymDesc& sd, int mask) { return (mask & 1) ? 0 : kSymT * sd.tI; }

// x over the column groups of tile rows < a_end (the only ones the CTA reads),
// eight entries per thread per pass: their index loads, then their value loads;
// 0 outside the column groups and past a run's end.
__device__ __forceinline__ void stage_x(const XSrc& xs, const SymDesc& sd, int cmask, int p_lo, int p_end, float* xsh,
                                        int tid, int nthr) {
    const float beta = (xs.kind == X_PCG || xs.kind == X_PCG_CV) ? (float)xs.sc->beta : 0.0f;
    constexpr int kStage = 8;
    for (int p0 = p_lo + tid; p0 < p_end; p0 += nthr * kStage) {
        int mm[kStage], cc[kStage], ll[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int p = p0 + u * nthr;
            const int l = p < p_end ? sym_local(sd, p) : -1;
            const bool need = l >= 0 && ((cmask >> sym_lgroup(sd, l)) & 1);
            ll[u] = need ? l : -1;
            mm[u] = need ? xs.slot_mult[sd.voff + l] : 0;
            cc[u] = need ? xs.slot_corner[sd.voff + l] : -1;
        }
        float vv[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const XRef r = ll[u] >= 0 ? xsrc_ref_f(xs, mm[u], cc[u], sd.voff + ll[u], ll[u])
                                      : XRef{nullptr, nullptr, 0, 1.0f};
            vv[u] = xref_value(r, beta);
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int p = p0 + u * nthr;
            if (p < p_end) xsh[p - p_lo] = vv[u];
        }
    }
}

// Row l (group g) of y = J S x: v negated on the corner rows (J), then
// alpha v (+ base) stored at l's output position in FP32 and/or FP64.
__device__ __forceinline__ void store_y(const GemvOut& go, const SymDesc& sd, int l, int g, float v) {
    if (g == 2) v = -v;   // J: the corner rows of M = J S
    const int64_t o = sd.voff + l;
    const int64_t oo = go.pos ? (int64_t)go.pos[o] : o;
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

// y[R] = J_R (sum over the cluster's partial vectors ysh, rank order); this CTA
// stores every cl-th chunk of rows.  Both cluster barriers are taken by every CTA.
__device__ __forceinline__ void cluster_store(cg::cluster_group& cluster, const float* ysh, const SymDesc& sd,
                                              int rmask, int r_lo, int p_lo, int np, int cl, const GemvOut& go,
                                              int tid, int nthr) {
    cluster.sync();
    const int rank = (int)cluster.block_rank();
    for (int p = r_lo + rank * nthr + tid; p < np; p += cl * nthr) {
        const int l = sym_local(sd, p);
        if (l < 0) continue;
        const int g = sym_lgroup(sd, l);
        if (!((rmask >> g) & 1)) continue;
        float part[kSymCLMax];
#pragma unroll
        for (int c = 0; c < kSymCLMax; ++c)
            part[c] = c < cl ? cluster.map_shared_rank(const_cast<float*>(ysh), c)[p - p_lo] : 0.0f;
        float v = 0.0f;
#pragma unroll
        for (int c = 0; c < kSymCLMax; ++c)
            if (c < cl) v += part[c];
        store_y(go, sd, l, g, v);
    }
    cluster.sync();   // no CTA leaves while another reads its shared memory
}

// CTA-synchronous form: 128 threads consume every tile together, one barrier per
// tile.  NR > 1 (ensembles): the CTA serves the nmem <= NR ensemble copies sub,
// sub + n_real, ... of one stored subdomain, applying every tile it loads to each
// member's x (one TMA copy and one pass over shared memory per tile for all of them).
template <int NR, bool LSM>
__global__ void __launch_bounds__(kT) k_symgemv(const SymDesc* __restrict__ descs, const int32_t* __restrict__ ranges,
                                                const uint32_t* __restrict__ tlist, const float* __restrict__ Msym,
                                                int span_max, int cl, int st, int rmask, int cmask, int keep, int n_real,
                                                XSrc xs, GemvOut go, const int32_t* __restrict__ skip,
                                                int32_t* __restrict__ err) {
    if (skip && *skip) return;   // the same word for every CTA of the grid
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* xsh = ring + st * kSymTile;   // [NR][span_max], index p - p_lo
    float* ysh = xsh + NR * span_max;    // [NR][span_max]
    float* red = ysh + NR * span_max;    // [2][NR][8][64] transposed-role partials, double-buffered
    uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * NR * 8 * 64);
    uint64_t* never = bars + kSymStages;

    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int32_t* rg5 = ranges + kSymRng * blockIdx.x;
    const int sub = rg5[3], nmem = rg5[4];
    const SymDesc sd = descs[sub];
    const int np = sd.nt * kSymT;
    // this CTA's run of the mode's tile list and the end of its tile rows
    const uint32_t* lst_g = tlist + kTlW * (int64_t)rg5[0];
    const int nt_cta = rg5[1];
    const int a_end = rg5[2];
    const float* tiles = Msym + sd.toff;
    const int p_lo = mask_lo(sd, rmask | cmask);
    const int r_lo = mask_lo(sd, rmask);

    // thread 0: barriers and the first st tiles (in flight while the CTA stages x)
    int issued = 0;
    const uint64_t pol = l2_policy(sub % n_real < keep);   // stored subdomains below `keep` stay in L2
    if (tid == 0) {
        for (int s = 0; s < st; ++s) mbar_init(&bars[s], 1);
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < st && s < nt_cta; ++s, ++issued) issue_tile<false>(lst_g, s, sd, tiles, ring + s * kSymTile, &bars[s], pol);
    }
    uint32_t* tsm = reinterpret_cast<uint32_t*>(never + 1);
    if (LSM)
        for (int k = tid; k < kTlW * nt_cta; k += kT) tsm[k] = __ldg(lst_g + k);
    const uint32_t* lst = LSM ? tsm : lst_g;
    const int p_end = min(np, a_end * kSymT);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        for (int p = p_lo + tid; p < np; p += kT) ysh[q * span_max + p - p_lo] = 0.0f;
        if (q < nmem) {
            stage_x(xs, descs[sub + q * n_real], cmask, p_lo, p_end, xsh + q * span_max, tid, kT);
        } else {   // an empty member slot of the group reads zeros
            for (int p = p_lo + tid; p < p_end; p += kT) xsh[q * span_max + p - p_lo] = 0.0f;
        }
    }
    __syncthreads();

    // thread (rg, cq): rows 8 rg .. 8 rg + 7 and columns 4 cq .. 4 cq + 3 of a tile
    // (16-byte shared loads; a half-warp covers one row group)
    const int rg = tid >> 4, cq = tid & 15;
    float acc[NR][8], xa[NR][8];
    int cur = -1, k = 0, slot = 0;
    uint32_t phase = 0;
    bool bad = false;
    // direct-role row partials of tile row `row` -> y: sum over the 16 column
    // quads (one half-warp, fixed shuffle tree), lane cq == r adds row r.  No
    // barrier: only this half-warp writes these rows before the next tile's barrier.
    auto flush = [&](int row) {
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                float v = acc[q][r];
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (cq == r) ysh[q * span_max + row * kSymT + rg * 8 + r - p_lo] += v;
            }
    };
    for (; k < nt_cta; ++k) {
        const uint32_t e = tl_word<LSM>(lst, k);
        const int ca = (int)(e >> 16), cb = (int)((e >> 3) & 0x1fff), cf = (int)(e & 7);
        const TileShape ts = tile_shape(sd, e);
        if (ca != cur) {
            if (cur >= 0) flush(cur);
            cur = ca;
#pragma unroll
            for (int q = 0; q < NR; ++q)
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    acc[q][r] = 0.0f;
                    xa[q][r] = xsh[q * span_max + ca * kSymT + rg * 8 + r - p_lo];
                }
        }
        const bool ok = (k > 0 || first_wait_test(xs, never)) && mbar_wait(&bars[slot], phase);
        const float* Ts = ring + slot * kSymTile;
        float4 xb[NR], col[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            xb[q] = (cf & 1) ? *reinterpret_cast<const float4*>(xsh + q * span_max + cb * kSymT + 4 * cq - p_lo)
                             : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            col[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        if (ok) {
            float4 mm[8];
            if (ts.full) {   // (uniform over the CTA)
                const float* base = Ts + rg * 8 * kSymT + 4 * cq;
#pragma unroll
                for (int r = 0; r < 8; ++r) mm[r] = *reinterpret_cast<const float4*>(base + r * kSymT);
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r) mm[r] = tile_chunk(Ts, ts, rg * 8 + r, cq);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float4 m = mm[r];
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    acc[q][r] = fmaf(m.x, xb[q].x, fmaf(m.y, xb[q].y, fmaf(m.z, xb[q].z, fmaf(m.w, xb[q].w, acc[q][r]))));
                    col[q].x = fmaf(m.x, xa[q][r], col[q].x);
                    col[q].y = fmaf(m.y, xa[q][r], col[q].y);
                    col[q].z = fmaf(m.z, xa[q][r], col[q].z);
                    col[q].w = fmaf(m.w, xa[q][r], col[q].w);
                }
            }
        }
        // A diagonal tile ends its tile row, and its transposed role adds to that row's
        // y after the barrier below: the row's direct-role partials go first.
        if (cf & 4) {   // (uniform over the CTA: every thread reads the same entry)
            flush(cur);
            cur = -1;
        }
        float* rd = red + (k & 1) * NR * 8 * 64;
#pragma unroll
        for (int q = 0; q < NR; ++q) *reinterpret_cast<float4*>(rd + q * 512 + rg * 64 + 4 * cq) = col[q];
        bad = __syncthreads_or(!ok) != 0;   // also: every thread is done with ring slot `slot`
        if (bad) break;
        if (tid == 0 && k + st < nt_cta) {
            issue_tile<LSM>(lst, k + st, sd, tiles, ring + slot * kSymTile, &bars[slot], pol);
            ++issued;
        }
        if (cf & 2) {   // transposed role: column c of the tile for member q, 8 row groups in order
            for (int t = tid; t < 64 * NR; t += kT) {
                const int q = t >> 6, c = t & 63;
                float sum = rd[q * 512 + c];
#pragma unroll
                for (int g = 1; g < 8; ++g) sum += rd[q * 512 + g * 64 + c];
                ysh[q * span_max + cb * kSymT + c - p_lo] += sum;
            }
        }
        if (++slot == st) {
            slot = 0;
            phase ^= 1u;
        }
    }
    if (!bad && cur >= 0) flush(cur);
    if (bad && tid == 0) {
        for (int q = k; q < issued; ++q) mbar_wait(&bars[q % st], (uint32_t)(q / st) & 1u);   // k: the tile that failed
        atomicExch(err, 1);
    }

    for (int q = 0; q < nmem; ++q)
        cluster_store(cluster, ysh + q * span_max, descs[sub + q * n_real], rmask, r_lo, p_lo, np, cl, go, tid, kT);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, const volatile int* abort) {
    for (unsigned k = 0; k < kWaitLimit; ++k) {
        if (mbar_test(bar, parity)) return true;
        if ((k & 255u) == 255u && *abort) return false;
    }
    return false;
}

// Consumer warps of the warp-specialised forms.  Thread (rg, cq) of the warp
// (rg = tid / 16 over the CTA's 128 consumer threads, cq = tid % 16).
// ws_flush: the direct-role row partials of tile row `row`, reduced over the
// half-warp (fixed shuffle tree), added to the warp's copy yc of the partial y.
__device__ __forceinline__ void ws_flush(float* yc, int row, int p_lo, const float (&acc)[8], int rg, int cq) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        float v = acc[r];
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (cq == r) yc[row * kSymT + rg * 8 + r - p_lo] += v;
    }
    __syncwarp();
}

// ws_tile: one listed tile in ring slot Ts: the direct role (row partials acc
// with the x of the tile's columns) and the transposed role (column partials
// with the x of the tile's rows xa), then the slot is released (one `empty`
// arrival per warp, after the arithmetic: releasing it before would expose the
// shared-memory load latency, which the FMAs hide otherwise), then the warp's two
// row groups' column partials are combined by one shuffle and added to yc.
__device__ __forceinline__ void ws_tile(const float* Ts, const TileShape& ts, int cf, int cb, const float* xsh,
                                        int p_lo, float* yc, float (&acc)[8], const float (&xa)[8],
                                        uint64_t* empty_slot, int rg, int cq, int lane) {
    float4 m[8];
    if (ts.full) {   // (uniform over the warp)
        const float* base = Ts + rg * 8 * kSymT + 4 * cq;
#pragma unroll
        for (int r = 0; r < 8; ++r) m[r] = *reinterpret_cast<const float4*>(base + r * kSymT);
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) m[r] = tile_chunk(Ts, ts, rg * 8 + r, cq);
    }
    const float4 xb = (cf & 1) ? *reinterpret_cast<const float4*>(xsh + cb * kSymT + 4 * cq - p_lo)
                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 col = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        acc[r] = fmaf(m[r].x, xb.x, fmaf(m[r].y, xb.y, fmaf(m[r].z, xb.z, fmaf(m[r].w, xb.w, acc[r]))));
        col.x = fmaf(m[r].x, xa[r], col.x);
        col.y = fmaf(m[r].y, xa[r], col.y);
        col.z = fmaf(m[r].z, xa[r], col.z);
        col.w = fmaf(m[r].w, xa[r], col.w);
    }
    __syncwarp();   // every lane is done with the slot
    if (lane == 0) mbar_arrive(empty_slot);
    if (cf & 2) {   // transposed role: the warp's 16 rows of column 4 cq .. 4 cq + 3, row group order
        col.x += __shfl_xor_sync(0xffffffffu, col.x, 16);
        col.y += __shfl_xor_sync(0xffffffffu, col.y, 16);
        col.z += __shfl_xor_sync(0xffffffffu, col.z, 16);
        col.w += __shfl_xor_sync(0xffffffffu, col.w, 16);
        if (lane < 16) {
            float4* yp = reinterpret_cast<float4*>(yc + cb * kSymT + 4 * cq - p_lo);
            float4 yv = *yp;
            yv.x += col.x;
            yv.y += col.y;
            yv.z += col.z;
            yv.w += col.w;
            *yp = yv;
        }
        __syncwarp();
    }
}

// Warp-specialised form: warp 4 (one elected lane) refills the ring as soon as
// the four consumer warps have released a slot (an `empty` mbarrier per slot,
// four arrivals); each consumer warp reads rows 16 w .. 16 w + 15 of every tile
// (the same thread layout as k_symgemv) and keeps its own copy of the partial
// y, so no barrier spans the CTA between tiles: the direct-role row sums are
// warp-local as before, and the transposed-role column sums of the warp's two
// row groups combine with one shuffle.  The four copies are added in warp order
// at the end (deterministic).
constexpr int kTW = kT + 32;

template <bool LSM>
__global__ void __launch_bounds__(kTW) k_symgemv_ws(const SymDesc* __restrict__ descs,
                                                    const int32_t* __restrict__ ranges,
                                                    const uint32_t* __restrict__ tlist, const float* __restrict__ Msym,
                                                    int span_max, int cl, int st, int rmask, int cmask, int keep,
                                                    int n_real, XSrc xs, GemvOut go, const int32_t* __restrict__ skip,
                                                    int32_t* __restrict__ err) {
    if (skip && *skip) return;   // the same word for every CTA of the grid
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* xsh = ring + st * kSymTile;   // index p - p_lo
    float* yw = xsh + span_max;          // [4][span_max]: one partial y per consumer warp
    uint64_t* full = reinterpret_cast<uint64_t*>(yw + 4 * span_max);
    uint64_t* empty = full + kSymStages;
    uint64_t* never = empty + kSymStages;
    __shared__ int abort_flag;

    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int sub = ranges[kSymRng * blockIdx.x + 3];
    const SymDesc sd = descs[sub];
    const int np = sd.nt * kSymT;
    const uint32_t* lst_g = tlist + kTlW * (int64_t)ranges[kSymRng * blockIdx.x];
    const int nt_cta = ranges[kSymRng * blockIdx.x + 1];
    const int a_end = ranges[kSymRng * blockIdx.x + 2];
    const float* tiles = Msym + sd.toff;
    const int p_lo = mask_lo(sd, rmask | cmask);
    const int r_lo = mask_lo(sd, rmask);
    const int span = np - p_lo;

    int issued = 0;   // producer lane only
    const uint64_t pol = l2_policy(sub % n_real < keep);
    if (tid == kT) {
        for (int s = 0; s < st; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 4);
        }
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
        for (int s = 0; s < st && s < nt_cta; ++s, ++issued) issue_tile<false>(lst_g, s, sd, tiles, ring + s * kSymTile, &full[s], pol);
    }
    uint32_t* tsm = reinterpret_cast<uint32_t*>(never + 1);
    if (LSM)
        for (int k = tid; k < kTlW * nt_cta; k += kTW) tsm[k] = __ldg(lst_g + k);
    const uint32_t* lst = LSM ? tsm : lst_g;
    for (int p = tid; p < 4 * span; p += kTW) yw[(p / span) * span_max + p % span] = 0.0f;
    stage_x(xs, sd, cmask, p_lo, min(np, a_end * kSymT), xsh, tid, kTW);
    __syncthreads();

    if (warp == 4) {
        if (lane == 0) {
            for (int k = st; k < nt_cta; ++k) {
                const int s = k % st;
                const uint32_t use = (uint32_t)(k / st);   // >= 1: the slot's previous tile was k - st
                if (!mbar_wait_or_abort(&empty[s], (use - 1u) & 1u, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                issue_tile<LSM>(lst, k, sd, tiles, ring + s * kSymTile, &full[s], pol);
                ++issued;
            }
        }
    } else {
        const int rg = tid >> 4, cq = tid & 15;
        float* yc = yw + warp * span_max;   // this warp's copy (index p - p_lo)
        float acc[8], xa[8];
        int cur = -1, slot = 0;
        uint32_t phase = 0;
        bool bad = false;
        for (int k = 0; k < nt_cta; ++k) {
            const uint32_t e = tl_word<LSM>(lst, k);
            const int ca = (int)(e >> 16), cb = (int)((e >> 3) & 0x1fff), cf = (int)(e & 7);
            const TileShape ts = tile_shape(sd, e);
            if (ca != cur) {
                if (cur >= 0) ws_flush(yc, cur, p_lo, acc, rg, cq);
                cur = ca;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    acc[r] = 0.0f;
                    xa[r] = xsh[ca * kSymT + rg * 8 + r - p_lo];
                }
            }
            const bool ok = __all_sync(0xffffffffu, (k > 0 || first_wait_test(xs, never)) &&
                                                        mbar_wait_or_abort(&full[slot], phase, &abort_flag));
            if (!ok) {
                if (lane == 0) abort_flag = 1;
                bad = true;
                break;
            }
            ws_tile(ring + slot * kSymTile, ts, cf, cb, xsh, p_lo, yc, acc, xa, &empty[slot], rg, cq, lane);
            if (++slot == st) {
                slot = 0;
                phase ^= 1u;
            }
        }
        if (!bad && cur >= 0) ws_flush(yc, cur, p_lo, acc, rg, cq);
    }
    __syncthreads();
    if (abort_flag) {   // drain the copies still in flight (the last one of each slot), then report
        if (tid == kT) {
            for (int q = issued > st ? issued - st : 0; q < issued; ++q)
                mbar_wait(&full[q % st], (uint32_t)(q / st) & 1u);
            atomicExch(err, 1);
        }
        __syncthreads();
    }
    // the four warp copies, added in warp order into copy 0
    for (int p = tid; p < span; p += kTW)
        yw[p] = ((yw[p] + yw[span_max + p]) + yw[2 * span_max + p]) + yw[3 * span_max + p];
    cluster_store(cluster, yw, sd, rmask, r_lo, p_lo, np, cl, go, tid, kTW);
}

// Persistent form (single problems): as many CTAs as the SMs hold walk queues of
// whole subdomains that the host balanced by bytes (largest first, each to the
// least-loaded CTA), and one ring of up to kSymStagesPs tiles runs through each
// queue, so the copies never pause between subdomains and no SM idles while
// another finishes a large subdomain.  Warp roles:
//  * NG groups of 4 consumer warps: group q takes the queue's tiles g = q, q + NG,
//    q + 2 NG, ... (g counts the tiles of the whole queue; the ring depth st is
//    a multiple of NG, so each slot serves one group and a group's waits on a
//    slot come in phase order) with the tile
//    arithmetic of the warp-specialised form (ws_tile, ws_flush), every warp
//    into its own copy of the partial y, each subdomain into one of two buffer
//    sets b = j % 2 (NG groups keep NG tiles in work at once: the per-tile
//    chain of one warp is latency-bound);
//  * one producer warp: one lane issues the bulk copies of the queue's tiles in
//    order as slots are released;
//  * 4 stager warps: for queue entry j, store y of entry j - 2 once its
//    consumers are done (the 4 NG copies added in warp order, J), then zero the
//    copies and stage x of entry j into the same buffer set.  Every stager
//    thread reads, zeroes and stages only indices i = its id mod 128, so these
//    steps need no barrier among the stagers.
// The tile list is read from global memory (each consumer loads its next
// entry word while it works on the current tile).  mbarriers: full / empty per ring
// slot (4 arrivals: the consuming group), xfull[b] (128 stager arrivals) and
// ydone[b] (128 NG consumer arrivals).  Every wait is bounded and gives up once
// any role has aborted; the producer then drains its copies and the error word
// is set.
template <int NG>
constexpr int ps_threads() { return 128 * NG + 32 + 128; }

template <int NG>
__global__ void __launch_bounds__(ps_threads<NG>(), 1) k_symgemv_ps(const SymDesc* __restrict__ descs,
                                                                 const int32_t* __restrict__ ranges,
                                                                 const uint32_t* __restrict__ tlist,
                                                                 const float* __restrict__ Msym, int span_max, int st,
                                                                 int rmask, int cmask, int keep, int n_real, XSrc xs,
                                                                 GemvOut go, const int32_t* __restrict__ skip,
                                                                 int32_t* __restrict__ err) {
    constexpr int kCons = 128 * NG, kCopies = 4 * NG;
    if (skip && *skip) return;   // the same word for every CTA of the grid
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* xbuf = ring + st * kSymTile;   // [2][span_max]
    float* ybuf = xbuf + 2 * span_max;    // [2][kCopies][span_max]
    uint64_t* full = reinterpret_cast<uint64_t*>(ybuf + 2 * kCopies * span_max);
    uint64_t* empty = full + kSymStagesPs;
    uint64_t* xfull = empty + kSymStagesPs;
    uint64_t* ydone = xfull + 2;
    uint64_t* never = ydone + 2;
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nit = ranges[2 * blockIdx.x + 1];
    const int32_t* items = ranges + 2 * (int64_t)gridDim.x + kSymRng * (int64_t)ranges[2 * blockIdx.x];
    int issued = 0;   // producer lane only
    if (tid == kCons) {
        for (int s = 0; s < st; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 4);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&xfull[b], 128);
            mbar_init(&ydone[b], kCons);
        }
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();

    if (warp == 4 * NG) {
        if (lane == 0) {
            int g = 0;
            bool stop = false;
            for (int j = 0; j < nit && !stop; ++j) {
                const int sub = items[kSymRng * j + 3], n = items[kSymRng * j + 1];
                const SymDesc sd = descs[sub];
                const uint32_t* lst = tlist + kTlW * (int64_t)items[kSymRng * j];
                const uint64_t pol = l2_policy(sub % n_real < keep);
                for (int k = 0; k < n; ++k, ++g) {
                    const int s = g % st;
                    const uint32_t use = (uint32_t)(g / st);   // >= 1: the slot's previous tile was g - st
                    if (use > 0 && !mbar_wait_or_abort(&empty[s], (use - 1u) & 1u, &abort_flag)) {
                        abort_flag = 1;
                        stop = true;
                        break;
                    }
                    issue_tile(lst, k, sd, Msym + sd.toff, ring + s * kSymTile, &full[s], pol);
                    ++issued;
                }
            }
        }
    } else if (warp < 4 * NG) {
        const int grp = warp >> 2;
        const int rg = (tid & 127) >> 4, cq = tid & 15;
        int gbase = 0, slot = grp % st;
        uint32_t phase = (uint32_t)(grp / st) & 1u;
        bool bad = false;
        for (int j = 0; j < nit && !bad; ++j) {
            const int b = j & 1;
            const int n = items[kSymRng * j + 1];
            const SymDesc sd = descs[items[kSymRng * j + 3]];
            const uint32_t* lst = tlist + kTlW * (int64_t)items[kSymRng * j];
            const int p_lo = mask_lo(sd, rmask | cmask);
            const float* xsh = xbuf + b * span_max;
            float* yc = ybuf + (b * kCopies + warp) * span_max;
            const int k0 = ((grp - gbase) % NG + NG) % NG;   // this group's first tile of the entry
            if (!__all_sync(0xffffffffu, mbar_wait_or_abort(&xfull[b], (uint32_t)(j >> 1) & 1u, &abort_flag))) {
                if (lane == 0) abort_flag = 1;
                bad = true;
                break;
            }
            float acc[8], xa[8];
            int cur = -1;
            uint32_t e = k0 < n ? tl_word<false>(lst, k0) : 0u;
            for (int k = k0; k < n; k += NG) {
                const uint32_t nxt = k + NG < n ? tl_word<false>(lst, k + NG) : 0u;   // the next entry, early
                const int ca = (int)(e >> 16), cb = (int)((e >> 3) & 0x1fff), cf = (int)(e & 7);
                const TileShape ts = tile_shape(sd, e);
                if (ca != cur) {
                    if (cur >= 0) ws_flush(yc, cur, p_lo, acc, rg, cq);
                    cur = ca;
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        acc[r] = 0.0f;
                        xa[r] = xsh[ca * kSymT + rg * 8 + r - p_lo];
                    }
                }
                const bool ok = __all_sync(0xffffffffu, (gbase + k > 0 || first_wait_test(xs, never)) &&
                                                            mbar_wait_or_abort(&full[slot], phase, &abort_flag));
                if (!ok) {
                    if (lane == 0) abort_flag = 1;
                    bad = true;
                    break;
                }
                ws_tile(ring + slot * kSymTile, ts, cf, cb, xsh, p_lo, yc, acc, xa, &empty[slot], rg, cq, lane);
                slot += NG;   // st is a multiple of NG: the group's own slots, at most one wrap
                if (slot >= st) {
                    slot -= st;
                    phase ^= 1u;
                }
                e = nxt;
            }
            if (bad) break;
            if (cur >= 0) ws_flush(yc, cur, p_lo, acc, rg, cq);
            gbase += n;
            mbar_arrive(&ydone[b]);   // every consumer thread, after its own writes to yc
        }
    } else {
        const int sid = tid - kCons - 32;   // 0 .. 127
        for (int j = 0; j < nit + 2; ++j) {
            const int b = j & 1;
            float* y0 = ybuf + b * kCopies * span_max;
            if (j >= 2) {   // y of entry q = j - 2 (buffer set b)
                const int q = j - 2;
                if (!mbar_wait_or_abort(&ydone[b], (uint32_t)(q >> 1) & 1u, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                const SymDesc sd = descs[items[kSymRng * q + 3]];
                const int p_lo = mask_lo(sd, rmask | cmask), r_lo = mask_lo(sd, rmask);
                const int span = sd.nt * kSymT - p_lo;
                for (int i = sid; i < span; i += 128) {
                    const int p = p_lo + i;
                    if (p < r_lo) continue;
                    const int l = sym_local(sd, p);
                    if (l < 0) continue;
                    const int g = sym_lgroup(sd, l);
                    if (!((rmask >> g) & 1)) continue;
                    float v = y0[i];
#pragma unroll
                    for (int c = 1; c < kCopies; ++c) v += y0[c * span_max + i];
                    store_y(go, sd, l, g, v);
                }
            }
            if (j < nit) {   // zero the copies of set b, stage x of entry j
                const SymDesc sd = descs[items[kSymRng * j + 3]];
                const int np = sd.nt * kSymT, p_lo = mask_lo(sd, rmask | cmask);
                const int a_end = items[kSymRng * j + 2];
                for (int i = sid; i < np - p_lo; i += 128)
#pragma unroll
                    for (int c = 0; c < kCopies; ++c) y0[c * span_max + i] = 0.0f;
                stage_x(xs, sd, cmask, p_lo, min(np, a_end * kSymT), xbuf + b * span_max, sid, 128);
                mbar_arrive(&xfull[b]);
            }
        }
    }
    __syncthreads();
    if (abort_flag && tid == kCons) {   // drain the copies still in flight (the last one of each slot), then report
        for (int q = issued > st ? issued - st : 0; q < issued; ++q) mbar_wait(&full[q % st], (uint32_t)(q / st) & 1u);
        atomicExch(err, 1);
    }
}

// Pack: one CTA per stored tile (directory entry blockIdx.x) from the swept FP64
// matrix: S = J M rounded to FP32 (corner rows negated), the diagonal halved on
// diagonal tiles, zeros in the padding.
__global__ void k_sym_pack(const SymDesc* __restrict__ descs, const MatDesc* __restrict__ mats,
                           const int32_t* __restrict__ dir, const double* __restrict__ M, float* __restrict__ Msym) {
    const int32_t* dr = dir + 4 * (int64_t)blockIdx.x;
    const int s = dr[0], a = dr[1], b = dr[2];
    const SymDesc sd = descs[s];
    const MatDesc md = mats[s];
    const bool diag = a == b;
    const int h = sym_h(sd, a), w = sym_h(sd, b), wp = (w + 3) & ~3;
    const int nfl = sym_tile_floats(h, w, diag);
    const int la0 = a < sd.tI ? kSymT * a : sd.n[0] + kSymT * (a - sd.tI);
    const int lb0 = b < sd.tI ? kSymT * b : sd.n[0] + kSymT * (b - sd.tI);
    float* out = Msym + sd.toff + dr[3];
    for (int e = threadIdx.x; e < nfl; e += blockDim.x) {
        int r, j;
        if (diag) {
            r = 0;
            while (r + 1 < h && sym_trioff(r + 1) <= e) ++r;
            j = e - sym_trioff(r);
        } else {
            r = e / wp;
            j = e - r * wp;
        }
        double v = 0.0;
        if (j < w && (!diag || j <= r)) {
            const int li = la0 + r, lj = lb0 + j;
            v = M[md.moff + (int64_t)li * md.ld + lj];
            if (li >= sd.n[0] + sd.n[1]) v = -v;   // S = J M
            if (diag && j == r) v *= 0.5;
        }
        out[e] = (float)v;
    }
}

}  // namespace

bool sym_active(const dd_handle* h, int mode) {
    int rm, cm;
    (void)h;
    return sym_masks(mode, &rm, &cm);
}

// Ensemble copies of a subdomain served by one CTA: 1 for the single-member
// forms; form 2: 4 (2 for a two-member ensemble); form 3: pairs (half the
// shared memory of form 2, so more CTAs share an SM, at two tile reads per
// four members).
int sym_members_per_cta(const dd_handle* h, int mode) {
    if (h->sym_ws[mode] == 4) return 1;   // the tensor-core form has its own grid (sym_ranges unused)
    if (h->sym_ws[mode] == 5) return 1;   // the persistent form: single problems
    if (h->sym_ws[mode] == 3) return 2;
    if (h->sym_ws[mode] != 2) return 1;
    return h->members <= 2 ? 2 : 4;
}

// Shared memory of the ensemble form with nr members per CTA at the deepest ring.
size_t sym_smem_bytes_nr(const dd_handle* h, int nr) { return sym_smem(h->sym_np_max, kSymStages, nr); }

size_t sym_smem_bytes(const dd_handle* h) {
    return std::max(sym_smem(h->sym_np_max, kSymStages), sym_smem_ws(h->sym_np_max, kSymStages));
}

// Padded index range a mode touches in the largest subdomain (from its first group on).
int sym_span(const dd_handle* h, int mode) {
    int rmask, cmask, span = 0;
    if (!sym_masks(mode, &rmask, &cmask)) return 0;
    for (const SymDesc& sd : h->sym) span = std::max(span, sd.nt * kSymT - mask_lo(sd, rmask | cmask));
    return span;
}

// Shared memory of one CTA of the persistent form in its current queue layout.
// The persistent form's kernel for ng consumer groups (1, 2 or 4), its threads.
static void (*ps_kernel(int ng, int* threads))(const SymDesc*, const int32_t*, const uint32_t*, const float*, int, int,
                                               int, int, int, int, XSrc, GemvOut, const int32_t*, int32_t*) {
    switch (ng) {
        case 1: *threads = ps_threads<1>(); return k_symgemv_ps<1>;
        case 2: *threads = ps_threads<2>(); return k_symgemv_ps<2>;
        case 4: *threads = ps_threads<4>(); return k_symgemv_ps<4>;
        default: *threads = 0; return nullptr;
    }
}

// CTAs of the persistent form one SM holds at once for mode's shared memory
// (0 if none fits or the query fails).
static int ps_ctas_per_sm(const dd_handle* h, int mode, int ng, int st) {
    int threads = 0;
    auto kern = ps_kernel(ng, &threads);
    const size_t smem = sym_smem_ps(sym_span(h, mode), st, ng);
    if (!kern || smem > 227 * 1024) return 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess) return 0;
    return nb;
}

// Host side: tile descriptors, the tile directory, the algorithmic and
// streamed bytes and the tile list of every packed mode.
void build_sym(dd_handle* h) {
    h->sym.assign(h->n_sub, SymDesc{});
    h->sym_dir.clear();
    int64_t toff = 0;
    h->sym_np_max = 0;
    h->sym_max_tiles = 0;
    std::vector<std::vector<int32_t>> offs(h->n_sub_real);   // float offset of tile (a, b) at a * nt + b
    auto tile_fl = [](const SymDesc& sd, int a, int b) { return sym_tile_floats(sym_h(sd, a), sym_h(sd, b), a == b); };
    for (int s = 0; s < h->n_sub; ++s) {
        SymDesc& sd = h->sym[s];
        sd.voff = h->mats[s].voff;
        sd.n[0] = h->nI[s];
        sd.n[1] = h->nG[s];
        sd.n[2] = h->nC[s];
        sd.tI = (sd.n[0] + kSymT - 1) / kSymT;
        sd.nt = sd.tI + (sd.n[1] + sd.n[2] + kSymT - 1) / kSymT;
        if (s >= h->n_sub_real) {   // ensemble copy: member 0's tiles
            sd.toff = h->sym[s % h->n_sub_real].toff;
            continue;
        }
        const int nt = sd.nt, tI = sd.tI;
        std::vector<int32_t>& off = offs[s];
        off.assign((size_t)nt * nt, -1);
        int64_t cur = 0;
        auto put = [&](int a, int b) {
            off[(size_t)a * nt + b] = (int32_t)cur;
            h->sym_dir.insert(h->sym_dir.end(), {s, a, b, (int32_t)cur});
            cur += tile_fl(sd, a, b);
        };
        for (int a = tI; a < nt; ++a)
            for (int b = tI; b <= a; ++b) put(a, b);
        for (int a = tI; a < nt; ++a)
            for (int b = 0; b < tI; ++b) put(a, b);
        for (int a = 0; a < tI; ++a)
            for (int b = 0; b <= a; ++b) put(a, b);
        sd.toff = toff;
        toff += cur;
        h->sym_np_max = std::max(h->sym_np_max, nt * kSymT);
        h->sym_max_tiles = std::max<int32_t>(h->sym_max_tiles, (int32_t)((int64_t)nt * (nt + 1) / 2));
    }
    h->sym_elems = toff;
    h->sym_ntiles = (int64_t)h->sym_dir.size() / 4;
    for (int mode = 0; mode < GEMV_NMODES; ++mode) {
        h->mode_bytes_sym[mode] = 0.0;
        h->mode_tile_bytes_sym[mode] = 0.0;
        int rmask, cmask;
        if (!sym_masks(mode, &rmask, &cmask)) continue;
        // algorithmic bytes: the distinct elements of the symmetric operator that
        // y[R] = M[R, C] x[C] needs (a diagonal group block counts its triangle
        // once, an off-diagonal pair of groups its rectangle once), 4 bytes each,
        // plus the vectors; streamed bytes: the stored tiles read.
        double bytes = 0.0, tile_bytes = 0.0;
        for (int s = 0; s < h->n_sub; ++s) {
            const SymDesc& sd = h->sym[s];
            double elems = 0.0;
            for (int ga = 0; ga < 3; ++ga)
                for (int gb = 0; gb <= ga; ++gb) {
                    const bool need = (((rmask >> ga) & 1) && ((cmask >> gb) & 1)) ||
                                      (((rmask >> gb) & 1) && ((cmask >> ga) & 1));
                    if (!need) continue;
                    const double na = sd.n[ga], nb = sd.n[gb];
                    elems += ga == gb ? na * (na + 1.0) / 2.0 : na * nb;
                }
            double vec = 0.0;
            for (int g = 0; g < 3; ++g) {   // x and y vectors of the groups read and written
                if ((cmask >> g) & 1) vec += 4.0 * sd.n[g];
                if ((rmask >> g) & 1) vec += 4.0 * sd.n[g];
            }
            bytes += 4.0 * elems + vec;
            for (int a = 0; a < sd.nt; ++a)
                for (int b = 0; b <= a; ++b)
                    if (sym_tile_flags(sd, a, b, rmask, cmask)) tile_bytes += 4.0 * tile_fl(sd, a, b);
            tile_bytes += vec;
        }
        h->mode_bytes_sym[mode] = bytes;
        h->mode_tile_bytes_sym[mode] = tile_bytes;
        // the mode's tiles of every stored subdomain in row order, with their offsets
        // (what the kernel streams; ensemble copies share member 0's list)
        std::vector<uint32_t>& tl = h->sym_tl[mode];
        std::vector<int64_t>& off = h->sym_tl_off[mode];
        tl.clear();
        off.assign(1, 0);
        for (int s = 0; s < h->n_sub_real; ++s) {
            const SymDesc& sd = h->sym[s];
            for (int a = 0; a < sd.nt; ++a)
                for (int b = 0; b <= a; ++b) {
                    const int f = sym_tile_flags(sd, a, b, rmask, cmask);
                    if (!f) continue;
                    tl.push_back(tile_entry(a, b, f));
                    tl.push_back((uint32_t)offs[s][(size_t)a * sd.nt + b]);
                }
            off.push_back((int64_t)tl.size() / kTlW);
        }
        sym_ranges(h, mode, h->sym_cl[mode]);
    }
}

// Queues of the persistent form (single problems; ng consumer groups): P =
// min(SMs x the CTAs one SM holds, subdomains) CTAs; the subdomains, largest first (bytes of the tiles the mode
// streams; ties by index), each go to the CTA with the smallest load so far
// (lowest index among equals).  Layout of the ranges: P pairs (first queue
// entry, entries), then the entries in CTA order, kSymRng ints each (list
// offset, tile count, end tile row, subdomain, 1).
static void sym_queue(dd_handle* h, int mode, int ng, int rmask, int cmask) {
    const int per_sm = ps_ctas_per_sm(h, mode, ng, h->sym_st[mode]);
    // st a multiple of ng: each ring slot then serves one consumer group only.  (A slot shared by two
    // groups could see a group that runs ahead wait for the slot's next phase while the current one is
    // still open, and an mbarrier parity wait cannot tell those phases apart.)
    if (per_sm < 1 || h->sym_st[mode] % ng != 0) return;   // sym_grid stays 0: the launch is refused
    const int n = h->n_sub_real;
    std::vector<int64_t> bytes(n, 0), tiles(n, 0);
    for (int s = 0; s < n; ++s) {
        const SymDesc& sd = h->sym[s];
        for (int a = 0; a < sd.nt; ++a)
            for (int b = 0; b <= a; ++b)
                if (sym_tile_flags(sd, a, b, rmask, cmask)) {
                    bytes[s] += 4 * (int64_t)sym_tile_floats(sym_h(sd, a), sym_h(sd, b), a == b);
                    ++tiles[s];
                }
    }
    const int P = std::max(1, std::min(std::max(1, h->n_sm) * per_sm, n));   // CTAs of one wave
    std::vector<int> order(n);
    for (int s = 0; s < n; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return bytes[x] > bytes[y]; });
    std::vector<std::vector<int>> q(P);
    std::vector<int64_t> load(P, 0);
    for (int s : order) {
        int c = 0;
        for (int k = 1; k < P; ++k)
            if (load[k] < load[c]) c = k;
        q[c].push_back(s);
        load[c] += bytes[s];
    }
    std::vector<int32_t>& rng = h->sym_rng[mode];
    rng.assign(2 * (size_t)P, 0);
    int32_t first_item = 0;
    for (int c = 0; c < P; ++c) {
        rng[2 * c] = first_item;
        rng[2 * c + 1] = (int32_t)q[c].size();
        first_item += (int32_t)q[c].size();
        for (int s : q[c]) {
            rng.push_back((int32_t)h->sym_tl_off[mode][s]);
            rng.push_back((int32_t)tiles[s]);
            rng.push_back(tiles[s] ? h->sym[s].nt : 0);
            rng.push_back(s);
            rng.push_back(1);
        }
    }
    h->sym_grid[mode] = P;
}

// Work of each of the cl CTAs of every subdomain for `mode`: contiguous tile-row
// ranges, CTA c ending where the running byte count comes closest to (c + 1) / cl
// of the subdomain's total; stored as (first entry in the mode's tile list, tile
// count, end tile row, subdomain, members served).  Ensemble copies of a
// subdomain follow each other (they stream the same tiles, which L2 then serves).
void sym_ranges(dd_handle* h, int mode, int cl) {
    int rmask, cmask;
    h->sym_rng[mode].clear();
    h->sym_cl[mode] = cl;
    h->sym_nl[mode] = 0;
    h->sym_grid[mode] = 0;
    if (!sym_masks(mode, &rmask, &cmask)) return;
    if (h->sym_ws[mode] == 5) {
        sym_queue(h, mode, cl, rmask, cmask);
        return;
    }
    const int R = std::max(1, h->members);
    const int per = sym_members_per_cta(h, mode);   // ensemble copies served by one CTA
    for (int s0 = 0; s0 < h->n_sub_real; ++s0) {
        const SymDesc& sd = h->sym[s0];
        const int nt = sd.nt;
        std::vector<int64_t> per_row(nt, 0), cnt_row(nt, 0);   // needed floats / tiles of each tile row
        int64_t total = 0;
        for (int a = 0; a < nt; ++a) {
            for (int b = 0; b <= a; ++b)
                if (sym_tile_flags(sd, a, b, rmask, cmask)) {
                    per_row[a] += sym_tile_floats(sym_h(sd, a), sym_h(sd, b), a == b);
                    ++cnt_row[a];
                }
            total += per_row[a];
        }
        for (int m0 = 0; m0 < R; m0 += per) {
            const int nmem = std::min(per, R - m0), sub = m0 * h->n_sub_real + s0;
            int a = 0;
            int64_t run = 0, first = h->sym_tl_off[mode][s0];
            for (int c = 0; c < cl; ++c) {
                const int begin = a;
                if (c == cl - 1) {
                    a = nt;
                } else {
                    const int64_t target = total * (c + 1) / cl;
                    while (a < nt && run + per_row[a] <= target) run += per_row[a++];
                    if (a < nt && target - run > run + per_row[a] - target) run += per_row[a++];
                }
                int64_t n = 0;
                for (int q = begin; q < a; ++q) n += cnt_row[q];
                h->sym_rng[mode].push_back((int32_t)first);
                h->sym_rng[mode].push_back((int32_t)n);
                h->sym_rng[mode].push_back(n ? a : 0);
                h->sym_rng[mode].push_back(sub);
                h->sym_rng[mode].push_back(nmem);
                first += n;
                h->sym_nl[mode] = std::max<int32_t>(h->sym_nl[mode], (int32_t)n);
            }
        }
    }
    // Largest clusters first (longest CTA tile list, stable): when the grid is larger than
    // one wave, the short clusters fill the slots the long ones leave at the end.
    std::vector<int32_t>& rng = h->sym_rng[mode];
    const size_t per_cluster = (size_t)cl * kSymRng, ncl = rng.size() / per_cluster;
    std::vector<int32_t> longest(ncl, 0);
    std::vector<size_t> order(ncl);
    for (size_t q = 0; q < ncl; ++q) {
        order[q] = q;
        for (int c = 0; c < cl; ++c) longest[q] = std::max(longest[q], rng[q * per_cluster + c * kSymRng + 1]);
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return longest[x] > longest[y]; });
    std::vector<int32_t> sorted;
    sorted.reserve(rng.size());
    for (size_t q : order) sorted.insert(sorted.end(), rng.begin() + q * per_cluster, rng.begin() + (q + 1) * per_cluster);
    rng.swap(sorted);
    h->sym_grid[mode] = (int32_t)(rng.size() / kSymRng);
}

int launch_sym_pack(const dd_handle* h, void* stream) {
    if (h->n_sub == 0 || h->sym_ntiles == 0) return 0;
    k_sym_pack<<<(unsigned)h->sym_ntiles, kT, 0, S(stream)>>>(h->d.symd, h->d.mats, h->d.sym_dir, h->d.M64, h->d.Msym);
    return (int)cudaGetLastError();
}

int launch_symgemv(const dd_handle* h, int mode, XSrc xs, GemvOut go, const int32_t* skip, void* stream) {
    int rmask, cmask;
    if (!sym_masks(mode, &rmask, &cmask)) return (int)cudaErrorInvalidValue;
    if (h->sym_ws[mode] == 4) return launch_tc_gemv(h, mode, xs, go, skip, stream);
    xs.slot_mult = h->d.slot_mult;
    xs.slot_corner = h->d.slot_corner;
    xs.sc = h->d.sc;
    const int span = sym_span(h, mode);
    const int st = h->sym_st[mode];
    const int form = h->sym_ws[mode];
    if (form == 5) {
        const int ng = h->sym_cl[mode];
        int threads = 0;
        auto kern = ps_kernel(ng, &threads);
        const size_t smem = sym_smem_ps(span, st, ng);
        if (!kern || smem > 227 * 1024 || st > kSymStagesPs || st % ng != 0 || h->sym_grid[mode] < 1)
            return (int)cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        kern<<<(unsigned)h->sym_grid[mode], (unsigned)threads, smem, S(stream)>>>(
            (const SymDesc*)h->d.symd, (const int32_t*)h->d.sym_rng[mode], (const uint32_t*)h->d.sym_tl[mode],
            (const float*)h->d.Msym, span, st, rmask, cmask, h->sym_keep[mode], std::max(1, h->n_sub_real), xs, go,
            skip, &h->d.sc->wait_err);
        return (int)cudaGetLastError();
    }
    const int nr = sym_members_per_cta(h, mode);
    const bool ws = form == 1;
    // the tile list in shared memory when the CTAs an SM holds (by shared memory) stay the same
    const int nl = h->sym_nl[mode];
    const size_t base = ws ? sym_smem_ws(span, st) : sym_smem(span, st, nr);
    const size_t with = ws ? sym_smem_ws(span, st, nl) : sym_smem(span, st, nr, nl);
    auto per_sm = [](size_t b) { return (int)(233472 / (b + 1024)); };   // 228 KB, 1 KB reserved per CTA
    const int lsm = with <= 227 * 1024 && per_sm(with) == per_sm(base) ? 1 : 0;
    const size_t smem = lsm ? with : base;
    auto kern = lsm ? (ws ? k_symgemv_ws<true>
                          : (nr == 4 ? k_symgemv<4, true> : (nr == 2 ? k_symgemv<2, true> : k_symgemv<1, true>)))
                    : (ws ? k_symgemv_ws<false>
                          : (nr == 4 ? k_symgemv<4, false> : (nr == 2 ? k_symgemv<2, false> : k_symgemv<1, false>)));
    if (smem > 227 * 1024) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    const int cl = h->sym_cl[mode];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(h->sym_rng[mode].size() / kSymRng));
    cfg.blockDim = dim3(ws ? kTW : kT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = S(stream);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, kern, (const SymDesc*)h->d.symd, (const int32_t*)h->d.sym_rng[mode],
                                   (const uint32_t*)h->d.sym_tl[mode], (const float*)h->d.Msym, span, cl, st, rmask,
                                   cmask, h->sym_keep[mode], std::max(1, h->n_sub_real), xs, go, skip,
                                   &h->d.sc->wait_err);
}
