// FP64-accurate trailing update of the elimination on the tensor cores (sm_103a).
//
// The exchange sweep's trailing update C[i][j] += A[i][:] B[:][j] (A the pivot
// block's column panel, B its row panel already multiplied by -P^-1, K = 32) is
// formed from BF16 slices on tcgen05 instead of FP64 FMAs (the Ozaki splitting
// of a product into exact low-precision products):
//  * each row i of A is scaled by a power of two 2^-e_i so that |A_ik| 2^-e_i < 1,
//    each column j of B by 2^-f_j likewise;
//  * the scaled values are cut into seven slices of 8 bits: r_0 = A 2^-e, then
//    a_p = rint(r_p 2^8), r_{p+1} = r_p 2^8 - a_p, so that
//    A 2^-e = sum_p 2^-8(p+1) a_p with integer slices |a_0| <= 256, |a_p| <= 128
//    (exact in BF16), and the same for B;
//  * for every weight class d = p + q <= 6 the products a_p b_q are summed over
//    K = 32 and over the (d + 1) slice pairs of the class in one FP32
//    accumulator in tensor memory: every partial sum is an integer below 2^24,
//    so the accumulation is exact;
//  * the classes are combined exactly in 64-bit integers (two partial sums, each
//    exact as a double, joined by one FMA) and scaled back with one FP64 FMA:
//    C_ij += 2^(e_i + f_j - 16) sum_d 2^-8d D_d[i][j].
// Dropping the classes d >= 7 leaves an error below 2^-55 of |A_i||B_j| per
// term, i.e. FP64 accuracy.  The FP64 work per matrix element and pivot block
// falls from 32 FMAs to two conversions and two FMAs; the tensor cores do 28 x 2 MMAs
// (M = 128 rows, N = 32 columns, K = 16) per 128 x 32 tile.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "dd_internal.h"
#include "tcgen05.cuh"

namespace {

constexpr int kOzS = 7;                      // slices per operand (8 bits each)
constexpr int kOzRows = 128;                 // rows of a tile (MMA M)
constexpr int kOzCols = 32;                  // columns of a tile (MMA N)
constexpr int kOzK = kNB;                    // pivot block width (MMA K = 2 x 16)
constexpr uint32_t kOzAPiece = kOzRows * kOzK * 2;   // 8 KB: one slice of a 128-row block
constexpr uint32_t kOzBPiece = kOzCols * kOzK * 2;   // 2 KB: one slice of a 32-column block
constexpr uint32_t kOzABytes = kOzS * kOzAPiece;     // 56 KB
constexpr uint32_t kOzBBytes = kOzS * kOzBPiece;     // 14 KB
constexpr unsigned kOzPolls = 1u << 22;
static_assert(kOzK == 32, "the slice layout assumes a 32-wide pivot block");

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

// Exponent e with |x| < 2^e for the largest |x| (0 for an all-zero vector).
__device__ __forceinline__ int scale_exp(double maxabs) {
    if (!(maxabs > 0.0)) return 0;
    int e;
    frexp(maxabs, &e);   // maxabs = f 2^e, f in [0.5, 1)
    return e;
}

// The seven 8-bit slices of r = x 2^-e (|r| < 1) as BF16 bits.
__device__ __forceinline__ void cut(double x, int e, uint16_t* out) {
    double r = ldexp(x, -e);
#pragma unroll
    for (int p = 0; p < kOzS; ++p) {
        const double t = r * 256.0;
        const double a = rint(t);
        r = t - a;
        out[p] = __bfloat16_as_ushort(__double2bfloat16(a));
    }
}

// Column panel A = M[i][k0 .. k0+nb) of every matrix: one CTA per (128-row block,
// matrix), one thread per row.  Slices in the K-major core-matrix layout of the
// MMA's A operand (K = 32), row exponents e_i.
__global__ void __launch_bounds__(kOzRows) k_oz_split_a(const MatDesc* __restrict__ mats, const double* __restrict__ M,
                                                        int k0, int nblk, uint16_t* __restrict__ As,
                                                        int32_t* __restrict__ ea, int nmax) {
    const int m = blockIdx.y, rb = blockIdx.x;
    const MatDesc md = mats[m];
    if (k0 >= md.nr || rb * kOzRows >= md.ns) return;
    const int nb = min(kOzK, md.nr - k0);
    const int r = threadIdx.x, i = rb * kOzRows + r;
    double v[kOzK];
    double mx = 0.0;
#pragma unroll
    for (int k = 0; k < kOzK; ++k) {
        v[k] = (i < md.ns && k < nb) ? M[md.moff + (int64_t)i * md.ld + k0 + k] : 0.0;
        mx = fmax(mx, fabs(v[k]));
    }
    const int e = scale_exp(mx);
    if (i < md.ns) ea[(int64_t)m * nmax + i] = e;
    uint16_t* out = As + ((int64_t)m * nblk + rb) * (kOzABytes / 2);
#pragma unroll
    for (int k = 0; k < kOzK; ++k) {
        uint16_t s[kOzS];
        cut(v[k], e, s);
        const uint32_t o = tc::kmajor_off(r, k, kOzK) / 2;
#pragma unroll
        for (int p = 0; p < kOzS; ++p) out[p * (kOzAPiece / 2) + o] = s[p];
    }
}

// Row panel B = M[k0 .. k0+nb)[j] (already -P^-1 times the pivot rows): one CTA
// per (32-column block, matrix), one thread per column; slices in the K-major
// layout of the MMA's B operand (N = 32 columns, K = 32), column exponents f_j.
__global__ void __launch_bounds__(kOzCols) k_oz_split_b(const MatDesc* __restrict__ mats, const double* __restrict__ M,
                                                        int k0, int nblk, uint16_t* __restrict__ Bs,
                                                        int32_t* __restrict__ fb, int nmax) {
    const int m = blockIdx.y, cb = blockIdx.x;
    const MatDesc md = mats[m];
    if (k0 >= md.nr || cb * kOzCols >= md.ns) return;
    const int nb = min(kOzK, md.nr - k0);
    const int c = threadIdx.x, j = cb * kOzCols + c;
    double v[kOzK];
    double mx = 0.0;
#pragma unroll
    for (int k = 0; k < kOzK; ++k) {
        v[k] = (j < md.ns && k < nb) ? M[md.moff + (int64_t)(k0 + k) * md.ld + j] : 0.0;
        mx = fmax(mx, fabs(v[k]));
    }
    const int f = scale_exp(mx);
    if (j < md.ns) fb[(int64_t)m * nmax + j] = f;
    uint16_t* out = Bs + ((int64_t)m * nblk + cb) * (kOzBBytes / 2);
#pragma unroll
    for (int k = 0; k < kOzK; ++k) {
        uint16_t s[kOzS];
        cut(v[k], f, s);
        const uint32_t o = tc::kmajor_off(c, k, kOzK) / 2;
#pragma unroll
        for (int p = 0; p < kOzS; ++p) out[p * (kOzBPiece / 2) + o] = s[p];
    }
}

__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity) {
    for (unsigned k = 0; k < kOzPolls; ++k) {
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

// One CTA per (128-row block, run of kOzCb 32-column blocks, matrix) of the
// trailing update: the row block's A slices are copied once and serve every
// column block of the run; the B slices come through two buffers, the next
// column block's copy in flight while the current one is combined.  Per column
// block one thread issues the 28 slice products x 2 K-steps into the seven
// class accumulators (224 tensor-memory columns), then the 256 threads combine
// them: warp w reads rows 32 (w mod 4) .. + 31 (its tensor-memory lane
// quarter) and columns 16 (w / 4) .. + 15, and adds the exact FP64 update to C
// (the pivot rows and columns are left alone).  Every wait is bounded; a CTA
// whose wait gives up sets the error word, lets its copies land and frees its
// tensor memory.
constexpr int kOzCb = 8;   // column blocks per CTA
constexpr int kOzThreads = 256;
constexpr size_t kOzSmem = kOzABytes + 2 * kOzBBytes + 8 * sizeof(uint64_t) + 16;

__device__ __forceinline__ void oz_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

__global__ void __launch_bounds__(kOzThreads, 2) k_oz_update(const MatDesc* __restrict__ mats, double* __restrict__ M,
                                                          int k0, int nrb, int ncb, const uint16_t* __restrict__ As,
                                                          const uint16_t* __restrict__ Bs,
                                                          const int32_t* __restrict__ ea,
                                                          const int32_t* __restrict__ fb, int nmax,
                                                          int32_t* __restrict__ err) {
    const int m = blockIdx.z, rb = blockIdx.y, cb0 = blockIdx.x * kOzCb;
    const MatDesc md = mats[m];
    const int ncb_m = (md.ns + kOzCols - 1) / kOzCols;
    if (k0 >= md.nr || rb * kOzRows >= md.ns || cb0 >= ncb_m) return;
    const int nc = min(kOzCb, ncb_m - cb0);   // column blocks of this CTA
    const int nb = min(kOzK, md.nr - k0);
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* sA = sm;
    unsigned char* sB = sm + kOzABytes;   // [2][kOzBBytes]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 2 * kOzBBytes);   // [0] A, [1..2] B buffers, [3] MMAs
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint16_t* gb = Bs + ((int64_t)m * ncb + cb0) * (kOzBBytes / 2);
    if (tid == 0) {
        for (int q = 0; q < 4; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_addr(&bars[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        oz_copy(sA, As + ((int64_t)m * nrb + rb) * (kOzABytes / 2), kOzABytes, &bars[0]);
        oz_copy(sB, gb, kOzBBytes, &bars[1]);
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(kOzRows, kOzCols);
    const int r = 32 * (warp & 3) + lane, hcol = 16 * (warp >> 2);
    const int i = rb * kOzRows + r;
    const bool row_ok = i < md.ns && (i < k0 || i >= k0 + nb);
    const int e = row_ok ? ea[(int64_t)m * nmax + i] : 0;
    double* crow = M + md.moff + (int64_t)i * md.ld;
    int issued_b = 1;   // B copies issued (thread 0)
    bool good = true;
    for (int c = 0; c < nc && good; ++c) {
        const int buf = c & 1;
        bool ok = true;   // thread 0: the copies of this column block arrived
        if (tid == 0) {
            ok = (c > 0 || oz_wait(&bars[0], 0u)) && oz_wait(&bars[1 + buf], (uint32_t)(c >> 1) & 1u);
            if (ok) {
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB + buf * kOzBBytes);
                for (int d = 0; d < kOzS; ++d) {
                    bool first = true;
                    for (int p = 0; p <= d; ++p) {
                        const int q = d - p;
                        for (int ks = 0; ks < kOzK / 16; ++ks) {
                            const uint64_t ad = tc::smem_desc(a0 + p * kOzAPiece + ks * 256, 128, (kOzK / 8) * 128);
                            const uint64_t bd = tc::smem_desc(b0 + q * kOzBPiece + ks * 256, 128, (kOzK / 8) * 128);
                            tc::mma_bf16(tmem + d * kOzCols, ad, bd, idesc, first ? 0u : 1u);
                            first = false;
                        }
                    }
                }
            }
            tc::mma_commit(&bars[3]);   // arrives once the MMAs issued above (if any) have completed
            // the other buffer's products (column block c - 1) completed before its combination
            if (ok && c + 1 < nc) {
                oz_copy(sB + (buf ^ 1) * kOzBBytes, gb + (int64_t)(c + 1) * (kOzBBytes / 2), kOzBBytes,
                        &bars[1 + (buf ^ 1)]);
                ++issued_b;
            }
        }
        const bool done = oz_wait(&bars[3], (uint32_t)c & 1u);
        tc::fence_after_sync();
        good = __syncthreads_and(done && ok) != 0;
        if (!good) break;
        const int cb = cb0 + c;
#pragma unroll
        for (int half = 0; half < 2; ++half) {   // eight columns at a time (registers)
            float D[kOzS][8];
#pragma unroll
            for (int d = 0; d < kOzS; ++d)
                tc::tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + d * kOzCols + hcol + 8 * half, D[d]);
            if (!row_ok) continue;
            const int jb = cb * kOzCols + hcol + 8 * half;
            bool on[8];
            double cv[8];
            int fe[8];
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {   // C and the column exponents first, all loads in flight
                const int j = jb + cc;
                on[cc] = j < md.ns && (j < k0 || j >= k0 + nb);
                cv[cc] = on[cc] ? crow[j] : 0.0;
                fe[cc] = on[cc] ? fb[(int64_t)m * nmax + j] : 0;
            }
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                if (!on[cc]) continue;
                // The class sums are exact integers below 2^22: combine them in 64-bit
                // integer arithmetic, H = D0 2^16 + D1 2^8 + D2 and L = D3 2^24 + D4 2^16 +
                // D5 2^8 + D6, both exact as doubles, so that
                // 2^16 sum_d D_d 2^-8d = H + L 2^-32 with one rounding.
                const long long H = ((long long)__float2int_rn(D[0][cc]) << 16) +
                                    ((long long)__float2int_rn(D[1][cc]) << 8) + (long long)__float2int_rn(D[2][cc]);
                const long long L = ((long long)__float2int_rn(D[3][cc]) << 24) +
                                    ((long long)__float2int_rn(D[4][cc]) << 16) +
                                    ((long long)__float2int_rn(D[5][cc]) << 8) + (long long)__float2int_rn(D[6][cc]);
                const double v = fma((double)L, 0x1p-32, (double)H);
                // times 2^(e + f - 32) from its exponent bits when that is a normal double
                const int x = e + fe[cc] - 32;
                const int j = jb + cc;
                if (x > -1023 && x < 1024) crow[j] = fma(v, __longlong_as_double((long long)(x + 1023) << 52), cv[cc]);
                else crow[j] = cv[cc] + ldexp(v, x);
            }
        }
        // every thread's tensor-memory reads complete before the next products overwrite the accumulators
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!good && tid == 0) {
        atomicExch(err, 1);
        // the copies issued land before the CTA ends (bounded): A, and the last one of each B buffer
        oz_wait(&bars[0], 0u);
        for (int q = issued_b > 2 ? issued_b - 2 : 0; q < issued_b; ++q) oz_wait(&bars[1 + (q & 1)], (uint32_t)(q >> 1) & 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tmem, 256);
}

}  // namespace

// Workspace of the tensor-core update: slices and exponents of one pivot block.
size_t oz_slice_elems(int nm, int nmax) {
    const size_t nrb = (size_t)(nmax + kOzRows - 1) / kOzRows, ncb = (size_t)(nmax + kOzCols - 1) / kOzCols;
    return (size_t)nm * (nrb * (kOzABytes / 2) + ncb * (kOzBBytes / 2));
}

int launch_oz_update(const MatDesc* mats, double* M, int nm, int nmax, int k0, uint16_t* slices, int32_t* exps,
                     int32_t* err, void* stream) {
    const int nrb = (nmax + kOzRows - 1) / kOzRows, ncb = (nmax + kOzCols - 1) / kOzCols;
    uint16_t* As = slices;
    uint16_t* Bs = slices + (size_t)nm * nrb * (kOzABytes / 2);
    int32_t* ea = exps;
    int32_t* fb = exps + (size_t)nm * nmax;
    k_oz_split_a<<<dim3((unsigned)nrb, (unsigned)nm), kOzRows, 0, S(stream)>>>(mats, M, k0, nrb, As, ea, nmax);
    k_oz_split_b<<<dim3((unsigned)ncb, (unsigned)nm), kOzCols, 0, S(stream)>>>(mats, M, k0, ncb, Bs, fb, nmax);
    // (84 KB of shared memory: at most two CTAs per SM, whose two 256-column tensor-memory allocations
    // fill its 512 columns)
    static_assert(3 * (kOzSmem + 1024) > 228 * 1024 && 2 * (kOzSmem + 1024) <= 228 * 1024, "two CTAs per SM");
    cudaError_t e = cudaFuncSetAttribute(k_oz_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e != cudaSuccess) return (int)e;
    const int nchunk = (ncb + kOzCb - 1) / kOzCb;
    k_oz_update<<<dim3((unsigned)nchunk, (unsigned)nrb, (unsigned)nm), kOzThreads, kOzSmem, S(stream)>>>(
        mats, M, k0, nrb, ncb, As, Bs, ea, fb, nmax, err);
    return (int)cudaGetLastError();
}
