// x-vector staging of the batched GEMVs: the value of local column j (flat
// slot `slot`) for each XSrc kind (included by the GEMV translation units).
#pragma once

#include "dd_internal.h"

namespace {

__device__ __forceinline__ double xsrc_value(const XSrc& xs, int64_t slot, int64_t j, double beta) {
    switch (xs.kind) {
        case X_FLAT: return xs.v[slot];
        case X_LAMBDA: {
            const int m = xs.slot_mult[slot];
            return m > 0 ? xs.v[m - 1] : (m < 0 ? -xs.v[-m - 1] : 0.0);
        }
        case X_PCG: {
            const int m = xs.slot_mult[slot];
            if (m == 0) return 0.0;
            const int mi = (m > 0 ? m : -m) - 1;
            const double pv = xs.v[mi] + beta * xs.v2[mi];
            return m > 0 ? pv : -pv;
        }
        case X_CORNER: return xs.v[xs.slot_corner[slot]];
        case X_RECOVER: {
            const int m = xs.slot_mult[slot];
            if (m != 0) return m > 0 ? -xs.v[m - 1] : xs.v[-m - 1];
            const int c = xs.slot_corner[slot];
            return c >= 0 ? xs.v2[c] : 0.0;
        }
        case X_PCG_CV: {
            const int m = xs.slot_mult[slot];
            if (m == 0) {
                const int c = xs.slot_corner[slot];
                return c >= 0 ? -xs.v3[c] : 0.0;
            }
            const int mi = (m > 0 ? m : -m) - 1;
            const double pv = xs.v[mi] + beta * xs.v2[mi];
            return m > 0 ? pv : -pv;
        }
        case X_LAMBDA_CV: {
            const int m = xs.slot_mult[slot];
            if (m == 0) {
                const int c = xs.slot_corner[slot];
                return c >= 0 ? -xs.v3[c] : 0.0;
            }
            return m > 0 ? xs.v[m - 1] : -xs.v[-m - 1];
        }
        case X_SIDE_CP: {
            const int m = xs.slot_mult[slot];
            if (m == 0) {
                const int c = xs.slot_corner[slot];
                return c >= 0 ? xs.v3[c] : 0.0;
            }
            return m > 0 ? xs.v[m - 1] : xs.v2[-m - 1];
        }
        default: return xs.v[j];
    }
}

// FP32 staging: only FP32 loads and FP32 arithmetic (GB300's FP64 pipe is
// ~1/64 of FP32 and would otherwise dominate short-row GEMVs).
__device__ __forceinline__ float xsrc_value_f(const XSrc& xs, int64_t slot, int64_t j, float beta) {
    switch (xs.kind) {
        case X_FLAT: return xs.vf[slot];
        case X_LAMBDA: {
            const int m = xs.slot_mult[slot];
            return m > 0 ? xs.vf[m - 1] : (m < 0 ? -xs.vf[-m - 1] : 0.0f);
        }
        case X_PCG: {
            const int m = xs.slot_mult[slot];
            if (m == 0) return 0.0f;
            const int mi = (m > 0 ? m : -m) - 1;
            const float pv = fmaf(beta, xs.v2f[mi], xs.vf[mi]);
            return m > 0 ? pv : -pv;
        }
        case X_CORNER: return xs.vf[xs.slot_corner[slot]];
        case X_RECOVER: {
            const int m = xs.slot_mult[slot];
            if (m != 0) return m > 0 ? -xs.vf[m - 1] : xs.vf[-m - 1];
            const int c = xs.slot_corner[slot];
            return c >= 0 ? xs.v2f[c] : 0.0f;
        }
        case X_PCG_CV: {
            const int m = xs.slot_mult[slot];
            if (m == 0) {
                const int c = xs.slot_corner[slot];
                return c >= 0 ? -xs.v3f[c] : 0.0f;
            }
            const int mi = (m > 0 ? m : -m) - 1;
            const float pv = fmaf(beta, xs.v2f[mi], xs.vf[mi]);
            return m > 0 ? pv : -pv;
        }
        case X_LAMBDA_CV: {
            const int m = xs.slot_mult[slot];
            if (m == 0) {
                const int c = xs.slot_corner[slot];
                return c >= 0 ? -xs.v3f[c] : 0.0f;
            }
            return m > 0 ? xs.vf[m - 1] : -xs.vf[-m - 1];
        }
        case X_SIDE_CP: {
            const int m = xs.slot_mult[slot];
            if (m == 0) {
                const int c = xs.slot_corner[slot];
                return c >= 0 ? xs.v3f[c] : 0.0f;
            }
            return m > 0 ? xs.vf[m - 1] : xs.v2f[-m - 1];
        }
        default: return xs.vf[j];
    }
}

// Where the FP32 value of one slot comes from, from its pre-loaded slot_mult (m)
// and slot_corner (c) entries: value = sgn * (a[i] + beta * b[i]) (b may be
// null), 0 when a is null.  Lets a caller issue the index loads of several
// slots, then their value loads, without a dependent chain per slot; the
// values equal xsrc_value_f's bit for bit (the sign is a multiplication by +-1).
struct XRef {
    const float* a;
    const float* b;
    int64_t i;
    float sgn;
};

__device__ __forceinline__ XRef xsrc_ref_f(const XSrc& xs, int m, int c, int64_t slot, int64_t j) {
    const XRef none{nullptr, nullptr, 0, 1.0f};
    const int mi = (m > 0 ? m : -m) - 1;
    const float ms = m > 0 ? 1.0f : -1.0f;
    switch (xs.kind) {
        case X_FLAT: return {xs.vf, nullptr, slot, 1.0f};
        case X_LAMBDA: return m != 0 ? XRef{xs.vf, nullptr, mi, ms} : none;
        case X_PCG: return m != 0 ? XRef{xs.vf, xs.v2f, mi, ms} : none;
        case X_CORNER: return c >= 0 ? XRef{xs.vf, nullptr, c, 1.0f} : none;
        case X_RECOVER:
            if (m != 0) return {xs.vf, nullptr, mi, -ms};
            return c >= 0 ? XRef{xs.v2f, nullptr, c, 1.0f} : none;
        case X_PCG_CV:
            if (m != 0) return {xs.vf, xs.v2f, mi, ms};
            return c >= 0 ? XRef{xs.v3f, nullptr, c, -1.0f} : none;
        case X_LAMBDA_CV:
            if (m != 0) return {xs.vf, nullptr, mi, ms};
            return c >= 0 ? XRef{xs.v3f, nullptr, c, -1.0f} : none;
        case X_SIDE_CP:
            if (m != 0) return m > 0 ? XRef{xs.vf, nullptr, mi, 1.0f} : XRef{xs.v2f, nullptr, mi, 1.0f};
            return c >= 0 ? XRef{xs.v3f, nullptr, c, 1.0f} : none;
        default: return {xs.vf, nullptr, j, 1.0f};
    }
}

__device__ __forceinline__ float xref_value(const XRef& r, float beta) {
    if (!r.a) return 0.0f;
    const float v = r.b ? fmaf(beta, r.b[r.i], r.a[r.i]) : r.a[r.i];
    return r.sgn * v;
}

}  // namespace
