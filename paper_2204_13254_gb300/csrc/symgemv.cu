// Batched GEMV on packed symmetric FP32 tiles (sm_103a): TMA bulk copies,
// mbarrier ring, one thread-block cluster per subdomain, DSMEM reduction.
//
// The swept local matrix is M_s = J S_s with S_s symmetric, J = diag(I_r, -I_c)
// (A_rr^-1 and the corner Schur complement are symmetric and
// M_s[c][r] = -M_s[r][c]^T), so only the lower triangle of 64x64 tiles is
// stored (SymDesc).  For y[R] = M[R, C] x[C] (R, C unions of the groups I,
// Gamma, c) a stored tile (a, b) acts directly (rows of a, columns of b)
// and/or transposed (rows of b, columns of a, sign J_a J_b): every needed
// tile is read from HBM once for both roles, about 60 % of the dense bytes of
// the local solve, the interface rows and the coupled operator.
//
// Work split: the cl CTAs of a cluster (1..kSymCLMax; per mode, like the ring
// depth st <= kSymStages, chosen by dd_autotune) share one subdomain by ranges of
// tile rows (balanced on the host by tile count).  Each CTA streams its tiles
// through an st-deep ring of shared-memory buffers filled by
// cp.async.bulk (one 16 KB copy per tile, completion on an mbarrier) issued by
// one thread, and accumulates its partial y over the subdomain's whole padded
// index range in shared memory:
//  * 128 threads; thread (rg, cq) = (tid / 16, tid % 16) reads rows
//    8 rg .. 8 rg + 7, columns 4 cq .. 4 cq + 3 of the tile with 16-byte
//    loads (a half-warp reads 256 contiguous bytes of one row: no bank
//    conflicts);
//  * direct role: per-thread row partials stay in registers across the tile
//    row and are reduced over the half-warp (fixed shuffle tree) when the
//    tile row ends;
//  * transposed role: the 8-row column partials of the eight row groups are
//    added in fixed order once per tile.
// The cluster then sums the cl partial vectors through distributed shared
// memory in rank order.  All sums have a fixed order: results are
// deterministic.  Every mbarrier wait is bounded: a wait that gives up sets an
// error word, the CTA drains its outstanding copies (bounded again) and still
// takes part in both cluster barriers, so no wait can hang the GPU.
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

// One 16 KB tile global -> shared, completing on `bar` (which expects the bytes).
__device__ __forceinline__ void load_tile(float* dst, const float* src, uint64_t* bar, uint64_t pol) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(kTileBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(kTileBytes), "r"(smem_u32(bar)), "l"(pol)
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (unsigned k = 0; k < kWaitLimit; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Tile groups of one subdomain as scalars (no dynamically indexed arrays:
// those would live in local memory).
struct Groups {
    int t1, t2, nt;   // first tile of Gamma, first tile of c, tiles per side
    int n0, n1, n2;   // group sizes
    __device__ __forceinline__ int of(int a) const { return (a >= t1) + (a >= t2); }
    __device__ __forceinline__ int first(int g) const { return g == 0 ? 0 : (g == 1 ? t1 : t2); }
    __device__ __forceinline__ int end(int g) const { return g == 0 ? t1 : (g == 1 ? t2 : nt); }
    __device__ __forceinline__ int size(int g) const { return g == 0 ? n0 : (g == 1 ? n1 : n2); }
    __device__ __forceinline__ int start(int g) const { return g == 0 ? 0 : (g == 1 ? n0 : n0 + n1); }
    // flags of tile (a, b) as sym_tile_flags
    __device__ __forceinline__ int flags(int a, int b, int rmask, int cmask) const {
        const int ga = of(a), gb = of(b);
        int f = 0;
        if (((rmask >> ga) & 1) && ((cmask >> gb) & 1)) f |= 1;
        if (a != b && ((rmask >> gb) & 1) && ((cmask >> ga) & 1)) f |= 2;
        if ((ga == 2) != (gb == 2)) f |= 4;
        return f;
    }
    // Next tile (a, b) at or after the iterator position, in row order over tile
    // rows [.., a1), that contributes to the mode; flags in f.  Flags depend
    // only on the groups of a and b (and on a == b), so a group that
    // contributes nothing is skipped whole.
    __device__ __forceinline__ bool next(int rmask, int cmask, int a1, int& a, int& b, int& f) const {
        for (; a < a1; ++a, b = 0) {
            while (b <= a) {
                f = flags(a, b, rmask, cmask);
                if (f & 3) return true;
                int nb = end(of(b));
                if (nb > a) nb = a;   // the diagonal tile has flags of its own
                b = nb > b ? nb : b + 1;
            }
        }
        return false;
    }
};

// Shared-memory layout of k_symgemv (floats unless noted), span = the padded
// index range the mode touches (from its first group on), st = ring depth,
// nl = longest tile list of one CTA:
//   ring [st][kSymTile] | x [span] | y [span] | red [2][8][64] | bars (u64) [kSymStages] | tile list (u32) [nl]
__host__ __device__ inline size_t sym_smem(int span, int st, int nl) {
    size_t f = (size_t)st * kSymTile + 2 * (size_t)span + 2 * 8 * 64;
    return f * sizeof(float) + kSymStages * sizeof(uint64_t) + (size_t)nl * sizeof(uint32_t);
}

// tile list entry: a << 16 | b << 3 | flags (a, b < 8192)
__device__ __forceinline__ uint32_t tile_entry(int a, int b, int f) { return ((uint32_t)a << 16) | ((uint32_t)b << 3) | f; }

__host__ __device__ inline int lowest_group(int mask) { return (mask & 1) ? 0 : ((mask & 2) ? 1 : 2); }

__global__ void __launch_bounds__(kT) k_symgemv(const SymDesc* __restrict__ descs, const int32_t* __restrict__ ranges,
                                                const float* __restrict__ Msym, int span_max, int cl, int st,
                                                int rmask, int cmask, int keep, XSrc xs, GemvOut go,
                                                const int32_t* __restrict__ skip, int32_t* __restrict__ err) {
    // (ranges/list capacity: the host sizes the list region for the longest range of this mode)
    if (skip && *skip) return;   // the same word for every CTA of the grid
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* xsh = ring + st * kSymTile;   // index p - p_lo
    float* ysh = xsh + span_max;
    float* red = ysh + span_max;        // [2][8][64] transposed-role partials, double-buffered
    uint64_t* bars = reinterpret_cast<uint64_t*>(red + 2 * 8 * 64);
    uint32_t* tl = reinterpret_cast<uint32_t*>(bars + kSymStages);

    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int sub = blockIdx.x / cl;
    const SymDesc sd = descs[sub];
    const Groups G{sd.t0[1], sd.t0[2], sd.t0[3], sd.n[0], sd.n[1], sd.n[2]};
    const int np = G.nt * kSymT;
    const int a0 = ranges[2 * blockIdx.x], a1 = ranges[2 * blockIdx.x + 1];
    const float* tiles = Msym + sd.toff;
    const int p_lo = G.first(lowest_group(rmask | cmask)) * kSymT;
    const int r_lo = G.first(lowest_group(rmask)) * kSymT;

    // thread 0: barriers, the first st tiles (in flight while the CTA stages x),
    // then the CTA's whole tile list
    __shared__ int n_tiles;
    int issued = 0;
    const uint64_t pol = l2_policy(sub < keep);   // subdomains below `keep` stay in L2
    if (tid == 0) {
        for (int s = 0; s < st; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        int pa = a0, pb = 0, pf = 0;
        for (int s = 0; s < st && G.next(rmask, cmask, a1, pa, pb, pf); ++s, ++pb, ++issued)
            load_tile(ring + s * kSymTile, tiles + sym_tile_index(pa, pb, G.t1, G.nt) * kSymTile, &bars[s], pol);
        int n = 0;
        pa = a0;
        pb = 0;
        while (G.next(rmask, cmask, a1, pa, pb, pf)) tl[n++] = tile_entry(pa, pb++, pf);
        n_tiles = n;
    }
    // x over the column groups (padded index space from p_lo), y = 0
    const float beta = (xs.kind == X_PCG || xs.kind == X_PCG_CV) ? (float)xs.sc->beta : 0.0f;
    for (int p = p_lo + tid; p < np; p += kT) {
        const int g = G.of(p / kSymT);
        const int q = p - G.first(g) * kSymT;
        float v = 0.0f;
        if (((cmask >> g) & 1) && q < G.size(g)) {
            const int l = G.start(g) + q;
            v = xsrc_value_f(xs, sd.voff + l, l, beta);
        }
        xsh[p - p_lo] = v;
        ysh[p - p_lo] = 0.0f;
    }
    __syncthreads();

    // thread (rg, cq): rows 8 rg .. 8 rg + 7 and columns 4 cq .. 4 cq + 3 of a tile
    // (16-byte shared loads; a half-warp covers one row group)
    const int rg = tid >> 4, cq = tid & 15;
    const int nt_cta = n_tiles;
    float acc[8], xa[8];
    int cur = -1, k = 0, slot = 0;
    uint32_t phase = 0;
    bool bad = false;
    // direct-role row partials of tile row `row` -> y: sum over the 16 column
    // quads (one half-warp, fixed shuffle tree), lane cq == r adds row r.  No
    // barrier: only this half-warp writes these rows before the next tile's barrier.
    auto flush = [&](int row) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float v = acc[r];
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (cq == r) ysh[row * kSymT + rg * 8 + r - p_lo] += v;
        }
    };
    for (; k < nt_cta; ++k) {
        const uint32_t e = tl[k];
        const int ca = (int)(e >> 16), cb = (int)((e >> 3) & 0x1fff), cf = (int)(e & 7);
        if (ca != cur) {
            if (cur >= 0) flush(cur);
            cur = ca;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                acc[r] = 0.0f;
                xa[r] = xsh[ca * kSymT + rg * 8 + r - p_lo];
            }
        }
        const bool ok = mbar_wait(&bars[slot], phase);
        const float4* T = reinterpret_cast<const float4*>(ring + slot * kSymTile) + rg * 8 * (kSymT / 4) + cq;
        const float4 xb = (cf & 1) ? *reinterpret_cast<const float4*>(xsh + cb * kSymT + 4 * cq - p_lo)
                                   : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float4 col = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (ok) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float4 m = T[r * (kSymT / 4)];
                acc[r] = fmaf(m.x, xb.x, fmaf(m.y, xb.y, fmaf(m.z, xb.z, fmaf(m.w, xb.w, acc[r]))));
                col.x = fmaf(m.x, xa[r], col.x);
                col.y = fmaf(m.y, xa[r], col.y);
                col.z = fmaf(m.z, xa[r], col.z);
                col.w = fmaf(m.w, xa[r], col.w);
            }
        }
        float* rd = red + (k & 1) * 8 * 64;
        *reinterpret_cast<float4*>(rd + rg * 64 + 4 * cq) = col;
        bad = __syncthreads_or(!ok) != 0;   // also: every thread is done with ring slot `slot`
        if (bad) break;
        if (tid == 0 && k + st < nt_cta) {
            const uint32_t en = tl[k + st];
            const int na = (int)(en >> 16), nb = (int)((en >> 3) & 0x1fff);
            load_tile(ring + slot * kSymTile, tiles + sym_tile_index(na, nb, G.t1, G.nt) * kSymTile, &bars[slot], pol);
            ++issued;
        }
        if ((cf & 2) && tid < 64) {   // transposed role: column tid of the tile, 8 row groups in order
            float sum = rd[tid];
#pragma unroll
            for (int q = 1; q < 8; ++q) sum += rd[q * 64 + tid];
            ysh[cb * kSymT + tid - p_lo] += (cf & 4) ? -sum : sum;
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

    // y[R] = sum over the cluster's partial vectors, rank order; this CTA stores every cl-th row
    cluster.sync();
    const int rank = (int)cluster.block_rank();
    for (int p = r_lo + rank * kT + tid; p < np; p += cl * kT) {
        const int g = G.of(p / kSymT);
        const int q = p - G.first(g) * kSymT;
        if (!((rmask >> g) & 1) || q >= G.size(g)) continue;
        float v = 0.0f;
        for (int c = 0; c < cl; ++c) v += cluster.map_shared_rank(ysh, c)[p - p_lo];
        const int64_t o = sd.voff + G.start(g) + q;
        if (go.out32) {
            float w = (float)go.alpha * v;
            if (go.base32) w += go.base32[o];
            go.out32[o] = w;
        }
        if (go.out) {
            double w = (double)v;
            if (go.alpha != 1.0) w *= go.alpha;
            if (go.base) w += go.base[o];
            go.out[o] = w;
        }
    }
    cluster.sync();   // no CTA leaves while another reads its shared memory
}

// Pack: tile (a, b) of subdomain blockIdx.y from the swept FP64 matrix.
__global__ void k_sym_pack(const SymDesc* __restrict__ descs, const MatDesc* __restrict__ mats,
                           const double* __restrict__ M, float* __restrict__ Msym) {
    const SymDesc sd = descs[blockIdx.y];
    const int nt = sd.t0[3];
    const int64_t kt = blockIdx.x;
    if (kt >= (int64_t)nt * (nt + 1) / 2) return;
    int a = (int)((sqrt(8.0 * (double)kt + 1.0) - 1.0) * 0.5);
    while ((int64_t)a * (a + 1) / 2 > kt) --a;
    while ((int64_t)(a + 1) * (a + 2) / 2 <= kt) ++a;
    const int b = (int)(kt - (int64_t)a * (a + 1) / 2);
    const MatDesc md = mats[blockIdx.y];
    const int gstart[3] = {0, sd.n[0], sd.n[0] + sd.n[1]};
    const int ga = sym_group(sd.t0, a), gb = sym_group(sd.t0, b);
    float* out = Msym + sd.toff + sym_tile_index(a, b, sd.t0[1], nt) * kSymTile;
    for (int e = threadIdx.x; e < kSymTile; e += blockDim.x) {
        const int qi = (a - sd.t0[ga]) * kSymT + e / kSymT;
        const int qj = (b - sd.t0[gb]) * kSymT + e % kSymT;
        float v = 0.0f;
        if (qi < sd.n[ga] && qj < sd.n[gb])
            v = (float)M[md.moff + (int64_t)(gstart[ga] + qi) * md.ld + gstart[gb] + qj];
        out[e] = v;
    }
}

}  // namespace

size_t sym_smem_bytes(const dd_handle* h) { return sym_smem(h->sym_np_max, kSymStages, h->sym_max_tiles); }

// Padded index range a mode touches in the largest subdomain (from its first group on).
int sym_span(const dd_handle* h, int mode) {
    int rmask, cmask, span = 0;
    if (!sym_masks(mode, &rmask, &cmask)) return 0;
    const int gl = lowest_group(rmask | cmask);
    for (const SymDesc& sd : h->sym) span = std::max(span, (sd.t0[3] - sd.t0[gl]) * kSymT);
    return span;
}

// Host side: tile descriptors and the algorithmic bytes of every packed mode.
void build_sym(dd_handle* h) {
    h->sym.assign(h->n_sub, SymDesc{});
    int64_t toff = 0;
    h->sym_np_max = 0;
    h->sym_max_tiles = 0;
    for (int s = 0; s < h->n_sub; ++s) {
        SymDesc& sd = h->sym[s];
        sd.toff = toff;
        sd.voff = h->mats[s].voff;
        sd.n[0] = h->nI[s];
        sd.n[1] = h->nG[s];
        sd.n[2] = h->nC[s];
        sd.t0[0] = 0;
        for (int g = 0; g < 3; ++g) sd.t0[g + 1] = sd.t0[g] + (sd.n[g] + kSymT - 1) / kSymT;
        const int nt = sd.t0[3];
        const int64_t ntl = (int64_t)nt * (nt + 1) / 2;
        toff += ntl * kSymTile;
        h->sym_np_max = std::max(h->sym_np_max, nt * kSymT);
        h->sym_max_tiles = std::max<int32_t>(h->sym_max_tiles, (int32_t)ntl);
    }
    h->sym_elems = toff;
    for (int mode = 0; mode < GEMV_NMODES; ++mode) {
        h->mode_bytes_sym[mode] = 0.0;
        int rmask, cmask;
        if (!sym_masks(mode, &rmask, &cmask)) continue;
        double bytes = 0.0;
        for (const SymDesc& sd : h->sym) {
            for (int a = 0; a < sd.t0[3]; ++a)
                for (int b = 0; b <= a; ++b)
                    if (sym_tile_flags(sd.t0, a, b, rmask, cmask) & 3) bytes += kTileBytes;
            for (int g = 0; g < 3; ++g) {   // x and y vectors of the groups read and written
                if ((cmask >> g) & 1) bytes += 4.0 * sd.n[g];
                if ((rmask >> g) & 1) bytes += 4.0 * sd.n[g];
            }
        }
        h->mode_bytes_sym[mode] = bytes;
        sym_ranges(h, mode, h->sym_cl[mode]);
    }
}

// Tile-row range of each of the cl CTAs of every subdomain for `mode`:
// contiguous ranges, CTA c ending where the running tile count comes closest
// to (c + 1) / cl of the subdomain's total.
void sym_ranges(dd_handle* h, int mode, int cl) {
    int rmask, cmask;
    h->sym_rng[mode].clear();
    h->sym_cl[mode] = cl;
    h->sym_nl[mode] = 0;
    if (!sym_masks(mode, &rmask, &cmask)) return;
    for (const SymDesc& sd : h->sym) {
        const int nt = sd.t0[3];
        std::vector<int64_t> per_row(nt, 0);
        int64_t total = 0;
        for (int a = 0; a < nt; ++a) {
            for (int b = 0; b <= a; ++b)
                if (sym_tile_flags(sd.t0, a, b, rmask, cmask) & 3) ++per_row[a];
            total += per_row[a];
        }
        int a = 0;
        int64_t run = 0;
        for (int c = 0; c < cl; ++c) {
            const int begin = a;
            if (c == cl - 1) {
                a = nt;
            } else {
                const int64_t target = total * (c + 1) / cl;
                while (a < nt && run + per_row[a] <= target) run += per_row[a++];
                if (a < nt && target - run > run + per_row[a] - target) run += per_row[a++];
            }
            h->sym_rng[mode].push_back(begin);
            h->sym_rng[mode].push_back(a);
            int64_t n = 0;
            for (int q = begin; q < a; ++q) n += per_row[q];
            h->sym_nl[mode] = std::max<int32_t>(h->sym_nl[mode], (int32_t)n);
        }
    }
}

int launch_sym_pack(const dd_handle* h, void* stream) {
    if (h->n_sub == 0 || h->sym_max_tiles == 0) return 0;
    k_sym_pack<<<dim3((unsigned)h->sym_max_tiles, (unsigned)h->n_sub), kT, 0, S(stream)>>>(h->d.symd, h->d.mats,
                                                                                           h->d.M64, h->d.Msym);
    return (int)cudaGetLastError();
}

int launch_symgemv(const dd_handle* h, int mode, XSrc xs, GemvOut go, const int32_t* skip, void* stream) {
    int rmask, cmask;
    if (!sym_masks(mode, &rmask, &cmask)) return (int)cudaErrorInvalidValue;
    xs.slot_mult = h->d.slot_mult;
    xs.slot_corner = h->d.slot_corner;
    xs.sc = h->d.sc;
    const int span = sym_span(h, mode);
    const int st = h->sym_st[mode];
    const size_t smem = sym_smem(span, st, h->sym_nl[mode]);
    cudaError_t e = cudaFuncSetAttribute(k_symgemv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sym_smem_bytes(h));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_symgemv, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    const int cl = h->sym_cl[mode];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(h->n_sub * cl));
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = S(stream);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_symgemv, (const SymDesc*)h->d.symd, (const int32_t*)h->d.sym_rng[mode],
                                   (const float*)h->d.Msym, span, cl, st, rmask, cmask, h->sym_keep[mode], xs, go, skip,
                                   &h->d.sc->wait_err);
}
