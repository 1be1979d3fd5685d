// CSR-3 SpMV / SpMM kernels for sm_103a.
//
// Mapping (Sec. 3's GPU view of CSR-3, re-designed for GB300):
//   * one super-super-row (SSR) at a time per thread block; the blocks are persistent
//     and walk the SSRs blockIdx.x, blockIdx.x + gridDim.x, ...
//   * the block's consumer warps share the stream of super-rows (SR) of those SSRs:
//     warp w takes every W-th SR, so an SR is handled by one warp (the paper's y level);
//   * inside an SR, `LPR` lanes cooperate on one row (LPR = 1 is GPU-SpMV-3's row per
//     thread, LPR > 1 is GPU-SpMV-3.5's lanes across a row, reduced with warp shuffles
//     instead of a shared-memory tree);
//   * SpMM: `G` lanes share a row and split its right-hand-side columns.
// Because an SSR's rows are contiguous, its sr_ptr, rowptr, colidx and vals slices are
// four contiguous byte ranges.  In the TMA kernel a producer warp copies them into a
// ring of shared-memory stages with cp.async.bulk (completion counted by an mbarrier,
// L2 evict-first hint so that x stays resident in L2), S-1 SSRs ahead of the consumers.
// The column slice is int32, or (MODE 3) delta-coded 16-bit steps rebuilt by the lanes.
// x is gathered through the read-only path; y is written once per row, through the
// permutation when the unpermute is fused.  Rows split off as long rows are not in any
// SSR (long_rows.cu computes them).
//
// GB300 note: FP64 FMA runs at about 2 per clock per SM here, so the FP64 path spends
// exactly one FP64 instruction per nonzero: narrow values are widened with integer
// instructions (a float->double conversion would also occupy the FP64 pipe) and the
// row-per-lane mapping needs no FP64 shuffle reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "csrk_internal.h"


namespace csrk {
namespace dev {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete, giving up after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > timeout_ns) return false;
    }
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 1-D bulk copy global -> shared, completion reported to `bar` in bytes.  dst, src and
// bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// ------------------------------------------------------------------ value widening
// FP32 bit pattern -> FP64 with integer instructions only (exact for every input).
__device__ __forceinline__ double f32bits_to_f64(uint32_t u) {
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t m = u & 0x7FFFFFu;
    uint64_t bits;
    if (e - 1u < 254u) {   // normal
        bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
    } else if (e == 0xFFu) {   // Inf / NaN
        bits = sign | 0x7FF0000000000000ull | ((uint64_t)m << 29);
    } else if (m == 0) {   // zero
        bits = sign;
    } else {   // FP32 subnormal: m * 2^-149, normalise
        const int top = 31 - __clz(m);   // 0..22
        const uint64_t frac = (uint64_t)(m ^ (1u << top)) << (52 - top);
        bits = sign | ((uint64_t)(top + 874) << 52) | frac;
    }
    return __longlong_as_double((long long)bits);
}

template <typename VT> struct Val;
template <> struct Val<double> {
    static constexpr int bytes = 8;
    __device__ __forceinline__ static double f64(double v) { return v; }
    __device__ __forceinline__ static float f32(double v) { return (float)v; }
};
template <> struct Val<float> {
    static constexpr int bytes = 4;
    __device__ __forceinline__ static double f64(float v) { return f32bits_to_f64(__float_as_uint(v)); }
    __device__ __forceinline__ static float f32(float v) { return v; }
};
// BF16 values travel as their 16-bit pattern.
struct bf16_t { uint16_t bits; };
template <> struct Val<bf16_t> {
    static constexpr int bytes = 2;
    __device__ __forceinline__ static double f64(bf16_t v) { return f32bits_to_f64((uint32_t)v.bits << 16); }
    __device__ __forceinline__ static float f32(bf16_t v) { return __uint_as_float((uint32_t)v.bits << 16); }
};

__device__ __forceinline__ double x_f64(double x) { return x; }
__device__ __forceinline__ double x_f64(float x) { return f32bits_to_f64(__float_as_uint(x)); }

template <typename AT> struct Acc;
template <> struct Acc<double> {
    template <typename VT, typename XT>
    __device__ __forceinline__ static double fma(VT v, XT x, double s) {
        return ::fma(Val<VT>::f64(v), x_f64(x), s);
    }
};
template <> struct Acc<float> {
    template <typename VT, typename XT>
    __device__ __forceinline__ static float fma(VT v, XT x, float s) {
        return fmaf(Val<VT>::f32(v), (float)x, s);
    }
};

// ------------------------------------------------------------------ FP64 on FP32 pipes
// A stored FP64 value a as an (hi, lo) pair of FP32 values with hi = RN(a) and
// lo = RN(a - hi): 48 significant bits, |a - hi - lo| <= 2^-48 |a|.  Built on the host.
struct ds_t { float hi, lo; };
template <> struct Val<ds_t> { static constexpr int bytes = 8; };

// The FP64 value of a stored pair (exact: the two halves do not overlap).
__device__ __forceinline__ double ds_value(const ds_t a) { return x_f64(a.hi) + x_f64(a.lo); }

// An FP64 x value as an (hi, lo) FP32 pair: hi its top 24 significant bits, lo the next
// 24 (rounded), |x - hi - lo| <= 2^-48 |x|.  Built once per SpMV by split_pairs_kernel,
// which also flags any x outside [2^-39, 2^60] (non-zero) or non-finite.
struct xpair { float hi, lo; };

// Split one FP64 value with integer instructions.  Returns false when x is outside the
// pair range (x = 0 splits to (0, 0) and is in range).
__device__ __forceinline__ bool split_x(double x, xpair& out) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e - 984u <= 99u) {   // biased exponent 984..1083: 2^-39 <= |x| < 2^61
        const uint32_t sgn = hi & 0x80000000u;
        out.hi = __uint_as_float(sgn | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
        // the remaining 29 bits, exactly as an integer-valued float via the 2^23 trick on
        // their top 23 bits, then scaled by a power of two
        const float m = __fsub_rn(__uint_as_float(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)), 8388608.0f);
        out.lo = __fmul_rn(m, __uint_as_float(sgn | ((e - 942u) << 23)));
        return true;
    }
    out.hi = 0.f;
    out.lo = 0.f;
    return ((hi & 0x7FFFFFFFu) | lo) == 0;
}

// s += a * x for one nonzero with the row sum held as an unevaluated pair (sh + sl) of FP32
// values: a*x = p + ep + (a.hi*x.lo + a.lo*x.hi) up to 2^-45 |a x| (p = RN(a.hi*x.hi), ep its
// exact error by FMA, a.lo*x.lo dropped); p enters by TwoSum, the small terms go to sl, and
// (sh, sl) is renormalised by Fast2Sum so |sl| <= ulp(sh) / 2.  Over a row of m <= 48
// entries the error stays below 1e-12 of sum |a x|.  Explicit round-to-nearest intrinsics
// keep the compiler from contracting or reassociating the error-free transforms.
__device__ __forceinline__ void ds_accum(const ds_t a, const xpair x, float& sh, float& sl) {
    const float p = __fmul_rn(a.hi, x.hi);
    const float ep = __fmaf_rn(a.hi, x.hi, -p);
    const float t = __fmaf_rn(a.hi, x.lo, __fmaf_rn(a.lo, x.hi, ep));
    const float s = __fadd_rn(sh, p);
    const float bp = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    const float l = __fadd_rn(sl, __fadd_rn(err, t));
    const float s2 = __fadd_rn(s, l);
    sl = __fsub_rn(l, __fsub_rn(s2, s));
    sh = s2;
}

template <typename T>
__device__ __forceinline__ T ldg_x(const T* p) { return __ldg(p); }

__device__ __forceinline__ void report(int32_t* status, int32_t bit) {
    if (status) atomicOr(status, bit);
}

// Epilogue selector, uniform over a launch and decided on the host, so that no per-row
// FP64 compare or multiply is issued when alpha == 1 or beta == 0.
enum : int { EPI_SCALE = 1, EPI_ACCUM = 2 };   // alpha != 1, beta != 0

// y = alpha*acc + beta*y in the accumulation precision; beta == 0 never reads y.
template <typename XT, typename AT>
__device__ __forceinline__ void store_y(XT* y, int64_t idx, AT acc, double alpha, double beta,
                                        int epi) {
    if constexpr (sizeof(AT) == 8) {
        double r = (epi & EPI_SCALE) ? alpha * acc : acc;
        if (epi & EPI_ACCUM) r = fma(beta, x_f64(y[idx]), r);
        y[idx] = (XT)r;
    } else {
        float r = (epi & EPI_SCALE) ? (float)alpha * acc : acc;
        if (epi & EPI_ACCUM) r = fmaf((float)beta, (float)y[idx], r);
        y[idx] = (XT)r;
    }
}

// ------------------------------------------------------------------ row compute
// One pass of a warp over up to 32/LPR rows [rb + lane/LPR ...] of a super-row.
// col_s / val_s are indexable by absolute nonzero index (already offset).  Each lane walks
// its row's nonzeros sub, sub+LPR, ... in chunks of U: it first issues the U independent
// x gathers of a chunk (the long-latency loads, all in flight together), then runs the
// chunk's U FMAs in stored order.  Full chunks carry no predicates; the last fewer-than-U
// entries go in predicated chunks of 4, so a row issues at most 3 idle FP64 slots (wider
// tail chunks measured slower on the 27-point stencil, where FP64 issue binds).
// CT is the stored column type: int32_t, or delta-coded uint16_t (one row per lane only):
// a row's first entry is its column minus the SSR's cbase (folded into x by the caller),
// every further entry the step from the previous column, so the lane rebuilds the column
// with one integer add per nonzero.
// LOCAL (kernel 5): CT = uint16_t codes are offsets into the SSR's x window, which x
// points to in shared memory (one row per lane).  With 16-bit codes (kernels 4 and 5)
// yperm, when set, is the SSR's staged slice of the permutation, in shared memory.
template <typename VT, typename XT, typename AT, int LPR, int U, typename CT = int32_t, bool LOCAL = false>
__device__ __forceinline__ void spmv_rows(int rb, int re, const int32_t* __restrict__ rp,
                                          const CT* __restrict__ col_s,
                                          const VT* __restrict__ val_s,
                                          const XT* __restrict__ x, XT* __restrict__ y,
                                          double alpha, double beta, int epi, int lane,
                                          const int32_t* __restrict__ yperm = nullptr,
                                          const uint16_t* __restrict__ ord = nullptr, int r0 = 0) {
    constexpr int RPP = 32 / LPR;   // rows per pass
    constexpr int T = U < 4 ? U : 4;
    const int sub = lane % LPR;
    for (int base = rb; base < re; base += RPP) {
        int r = base + lane / LPR;
        AT acc = 0;
        if constexpr (LOCAL) {
            // LOCAL with ord: position r of the SSR's length-ordered rows is row r0 + ord[r]
            const bool live = r < re;
            if (ord && live) r = r0 + ord[r];
            static_assert(LPR == 1 && sizeof(CT) == 2, "window codes take one row per lane");
            if (live) {
                const int pe = rp[r + 1];
                int c = rp[r];
                for (; c + (U - 1) < pe; c += U) {
                    XT xv[U];
#pragma unroll
                    for (int t = 0; t < U; ++t) xv[t] = x[col_s[c + t]];
#pragma unroll
                    for (int t = 0; t < U; ++t) acc = Acc<AT>::fma(val_s[c + t], xv[t], acc);
                }
                // the last fewer-than-U entries in chunks of 4, 2 and 1: a warp issues an
                // FP64 instruction only for a product some lane needs (x comes from shared
                // memory, so the smaller chunks cost no extra memory round trips)
                if constexpr (U > 4) {
                    for (; c + 3 < pe; c += 4) {
                        XT xv[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) xv[t] = x[col_s[c + t]];
#pragma unroll
                        for (int t = 0; t < 4; ++t) acc = Acc<AT>::fma(val_s[c + t], xv[t], acc);
                    }
                }
                if (c + 1 < pe) {
                    const XT x0 = x[col_s[c]], x1 = x[col_s[c + 1]];
                    acc = Acc<AT>::fma(val_s[c], x0, acc);
                    acc = Acc<AT>::fma(val_s[c + 1], x1, acc);
                    c += 2;
                }
                if (c < pe) acc = Acc<AT>::fma(val_s[c], x[col_s[c]], acc);
            }
        } else if constexpr (sizeof(CT) == 2) {
            static_assert(LPR == 1, "delta-coded columns take one row per lane");
            if (r < re) {
                const int pe = rp[r + 1];
                int c = rp[r];
                int col = 0;
                for (; c + (U - 1) < pe; c += U) {
                    XT xv[U];
#pragma unroll
                    for (int t = 0; t < U; ++t) {
                        col += col_s[c + t];
                        xv[t] = ldg_x(&x[col]);
                    }
#pragma unroll
                    for (int t = 0; t < U; ++t) acc = Acc<AT>::fma(val_s[c + t], xv[t], acc);
                }
                for (; c < pe; c += T) {
                    XT xv[T];
#pragma unroll
                    for (int t = 0; t < T; ++t)
                        if (c + t < pe) {
                            col += col_s[c + t];
                            xv[t] = ldg_x(&x[col]);
                        }
#pragma unroll
                    for (int t = 0; t < T; ++t)
                        if (c + t < pe) acc = Acc<AT>::fma(val_s[c + t], xv[t], acc);
                }
            }
        } else if (r < re) {
            const int pe = rp[r + 1];
            int c = rp[r] + sub;
            for (; c + (U - 1) * LPR < pe; c += U * LPR) {
                XT xv[U];
#pragma unroll
                for (int t = 0; t < U; ++t) xv[t] = ldg_x(&x[col_s[c + t * LPR]]);
#pragma unroll
                for (int t = 0; t < U; ++t) acc = Acc<AT>::fma(val_s[c + t * LPR], xv[t], acc);
            }
            for (; c < pe; c += T * LPR) {
                XT xv[T];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const int p = c + t * LPR;
                    if (p < pe) xv[t] = ldg_x(&x[col_s[p]]);
                }
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const int p = c + t * LPR;
                    if (p < pe) acc = Acc<AT>::fma(val_s[p], xv[t], acc);
                }
            }
        }
        if constexpr (LPR > 1) {
#pragma unroll
            for (int off = LPR / 2; off > 0; off >>= 1)
                acc += __shfl_xor_sync(0xffffffffu, acc, off);
        }
        if constexpr (sizeof(CT) == 2) {   // kernels 4, 5: the permutation slice is staged in shared memory
            if (base + lane < re) store_y<XT, AT>(y, yperm ? yperm[r] : r, acc, alpha, beta, epi);
        } else {
            if (r < re && sub == 0) store_y<XT, AT>(y, yperm ? __ldg(&yperm[r]) : r, acc, alpha, beta, epi);
        }
    }
}

// spmv_rows for FP64 values stored as (hi, lo) FP32 pairs: one row per lane.  Fast path
// (x2 = x split into pairs, every element in range): the row sum in FP32 pairs (ds_accum),
// chunks of U pair gathers issued before their accumulations.  When the split pass flagged
// an element (`slow`), the launch multiplies in FP64 from the pairs' exact FP64 values and
// the FP64 x instead.
template <int U>
__device__ __forceinline__ void spmv_rows_ds(int rb, int re, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ col_s,
                                             const ds_t* __restrict__ val_s,
                                             const xpair* __restrict__ x2,
                                             const double* __restrict__ x64, bool slow,
                                             double* __restrict__ y, double alpha, double beta,
                                             int epi, int lane, const int32_t* __restrict__ yperm) {
    for (int base = rb; base < re; base += 32) {
        const int r = base + lane;
        if (r >= re) continue;
        const int pe = rp[r + 1];
        int c = rp[r];
        double acc;
        if (!slow) {
            float sh = 0.f, sl = 0.f;
            for (; c + U <= pe; c += U) {
                xpair xv[U];
#pragma unroll
                for (int t = 0; t < U; ++t) {
                    const float2 v = __ldg(reinterpret_cast<const float2*>(x2) + col_s[c + t]);
                    xv[t] = xpair{v.x, v.y};
                }
#pragma unroll
                for (int t = 0; t < U; ++t) ds_accum(val_s[c + t], xv[t], sh, sl);
            }
            for (; c < pe; c += 4) {
                xpair xv[4];
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (c + t < pe) {
                        const float2 v = __ldg(reinterpret_cast<const float2*>(x2) + col_s[c + t]);
                        xv[t] = xpair{v.x, v.y};
                    }
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (c + t < pe) ds_accum(val_s[c + t], xv[t], sh, sl);
            }
            acc = x_f64(sh) + x_f64(sl);
        } else {
            acc = 0.0;
            for (; c < pe; ++c) acc = fma(ds_value(val_s[c]), __ldg(&x64[col_s[c]]), acc);
        }
        store_y<double, double>(y, yperm ? __ldg(&yperm[r]) : r, acc, alpha, beta, epi);
    }
}

// spmv_rows_ds over a staged x window (kernel 6): col_s are 16-bit window offsets, xs the
// window in shared memory -- FP32 pairs of x in the fast path, FP64 x when the split pass
// flagged an element (`slow`, uniform over the launch) -- and yperm, when set, the SSR's
// staged slice of the permutation; ord, when set, the SSR's length order of its rows (as in
// spmv_rows).
template <int U>
__device__ __forceinline__ void spmv_rows_ds_win(int rb, int re, const int32_t* __restrict__ rp,
                                                 const uint16_t* __restrict__ col_s,
                                                 const ds_t* __restrict__ val_s, const void* xs, bool slow,
                                                 double* __restrict__ y, double alpha, double beta, int epi,
                                                 int lane, const int32_t* __restrict__ yperm,
                                                 const uint16_t* __restrict__ ord, int r0) {
    for (int base = rb; base < re; base += 32) {
        int r = base + lane;
        if (r >= re) continue;
        if (ord) r = r0 + ord[r];   // position -> row of the length order
        const int pe = rp[r + 1];
        int c = rp[r];
        double acc;
        if (!slow) {
            const float2* __restrict__ x2 = static_cast<const float2*>(xs);
            float sh = 0.f, sl = 0.f;
            for (; c + U <= pe; c += U) {
                xpair xv[U];
#pragma unroll
                for (int t = 0; t < U; ++t) {
                    const float2 v = x2[col_s[c + t]];
                    xv[t] = xpair{v.x, v.y};
                }
#pragma unroll
                for (int t = 0; t < U; ++t) ds_accum(val_s[c + t], xv[t], sh, sl);
            }
            for (; c < pe; c += 4) {
                xpair xv[4];
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (c + t < pe) {
                        const float2 v = x2[col_s[c + t]];
                        xv[t] = xpair{v.x, v.y};
                    }
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (c + t < pe) ds_accum(val_s[c + t], xv[t], sh, sl);
            }
            acc = x_f64(sh) + x_f64(sl);
        } else {
            const double* __restrict__ x64 = static_cast<const double*>(xs);
            acc = 0.0;
            for (; c < pe; ++c) acc = fma(ds_value(val_s[c]), x64[col_s[c]], acc);
        }
        store_y<double, double>(y, yperm ? yperm[r] : r, acc, alpha, beta, epi);
    }
}

// SpMM pass: G lanes per row, lane c0 = lane % G owns columns c0, c0+G, ... (< k, CPL of
// them).  X, Y row-major with leading dimensions ldx, ldy.  As in spmv_rows, the X gathers
// of a chunk of 8 nonzeros are issued before their FMAs (a predicated 4-wide tail ends the
// row), so each lane keeps several loads in flight.
template <typename VT, typename XT, typename AT, int G, int CPL>
__device__ __forceinline__ void spmm_rows(int rb, int re, const int32_t* __restrict__ rp,
                                          const int32_t* __restrict__ col_s,
                                          const VT* __restrict__ val_s,
                                          const XT* __restrict__ X, int64_t ldx,
                                          XT* __restrict__ Y, int64_t ldy, int k,
                                          double alpha, double beta, int epi, int lane) {
    constexpr int RPP = 32 / G;
    constexpr int U = CPL == 1 ? 8 : 4;
    const int c0 = lane % G;
    bool on[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) on[j] = c0 + j * G < k;
    for (int base = rb; base < re; base += RPP) {
        const int r = base + lane / G;
        if (r >= re) continue;
        AT acc[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) acc[j] = 0;
        const int pe = rp[r + 1];
        int p = rp[r];
        for (; p + U <= pe; p += U) {
            XT xv[U][CPL];
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const XT* xr = X + (int64_t)col_s[p + t] * ldx + c0;
#pragma unroll
                for (int j = 0; j < CPL; ++j) xv[t][j] = on[j] ? ldg_x(xr + j * G) : XT(0);
            }
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const VT v = val_s[p + t];
#pragma unroll
                for (int j = 0; j < CPL; ++j) acc[j] = Acc<AT>::fma(v, xv[t][j], acc[j]);
            }
        }
        for (; p < pe; p += 4) {
            XT xv[4][CPL];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (p + t < pe) {
                    const XT* xr = X + (int64_t)col_s[p + t] * ldx + c0;
#pragma unroll
                    for (int j = 0; j < CPL; ++j) xv[t][j] = on[j] ? ldg_x(xr + j * G) : XT(0);
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (p + t < pe) {
                    const VT v = val_s[p + t];
#pragma unroll
                    for (int j = 0; j < CPL; ++j) acc[j] = Acc<AT>::fma(v, xv[t][j], acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < CPL; ++j)
            if (on[j]) store_y<XT, AT>(Y + (int64_t)r * ldy, c0 + j * G, acc[j], alpha, beta, epi);
    }
}

// ------------------------------------------------------------------ TMA kernel
struct TmaParams {
    const SsrDesc* desc;
    const int32_t* sr_ptr;
    const int32_t* rowptr;
    const void* colidx;    // int32 columns; MODE 3: uint16 offsets from each SSR's cbase
    const void* vals;
    const void* x;
    void* y;
    int64_t ldx, ldy;
    int32_t k;
    int32_t nssr;
    double alpha, beta;
    int32_t epi;   // EPI_SCALE | EPI_ACCUM
    const int32_t* skip;   // optional: non-zero on the device means "do nothing"
    const double* x64;     // MODE 2: FP64 x (P.x then holds its FP32-pair split)
    const int32_t* yperm;  // SpMV: when set, row r's result goes to y[yperm[r]] (fused unpermute)
    const int32_t* xflag;  // MODE 2: non-zero when the split found an out-of-range element
    int32_t* status;
    const int2* win;       // MODES 4, 5: x-window runs (start, offset), SSR by SSR
    const int32_t* wptr;   // MODES 4, 5: first run of each SSR in win
    const uint16_t* rord;  // MODES 4, 5 (optional): each SSR's rows in length order, as offsets
                           // from its first row; staged at off_ord
    // extents, read by the bounds checks of a CSRK_CHECKS build only
    int32_t n;             // rows (and entries of x and y)
    int32_t nsr;           // super-rows
    int64_t nnz;           // stored entries
    uint32_t off_srp, off_rp, off_col, off_val, off_x, off_perm, off_ord, stage_bytes, header_bytes;
    int32_t stages;
    unsigned long long timeout_ns;
};

#ifdef CSRK_CHECKS
// Bounds checks of a CSRK_CHECKS build (a debugging build standing in for a memory
// checker): before a warp computes a super-row, every index it is about to follow is
// checked -- the super-row's row range inside its SSR's, each row's nonzero range inside
// the SSR's, every column (int32: inside [0, n); CM 1, delta codes: the rebuilt column
// inside [0, n); CM 2, window offsets: inside the staged window) and every target of the
// fused unpermute.  A super-row with a bad index is skipped and bit 1 (value 2) of the
// status word is set; nothing out of bounds is read or written.  The regular build
// compiles none of this.
template <int CM, typename CT>
__device__ bool sr_in_bounds(int rb, int re, int r_lo, int r_hi, int64_t p_lo, int64_t p_hi,
                             const int32_t* rp, const CT* col, int64_t cbase, int64_t limit,
                             const int32_t* yperm, int32_t n, int lane, int32_t* status,
                             const uint16_t* ord = nullptr) {
    bool bad = rb < r_lo || re > r_hi || rb > re;
    for (int pos = rb + lane; !bad && pos < re; pos += 32) {
        const int r = ord ? r_lo + ord[pos] : pos;   // the row at position pos of a length order
        if (r < r_lo || r >= r_hi) {
            bad = true;
            break;
        }
        const int64_t p = rp[r], q = rp[r + 1];
        if (p < p_lo || q > p_hi || p > q) {
            bad = true;
            break;
        }
        int64_t c = 0;
        for (int64_t k = p; k < q; ++k) {
            if constexpr (CM == 1) c += (int64_t)col[k];
            else c = (int64_t)col[k];
            const int64_t abs = CM == 1 ? cbase + c : c;
            if (abs < 0 || abs >= limit) {
                bad = true;
                break;
            }
        }
        if (!bad && yperm && (yperm[r] < 0 || yperm[r] >= n)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) report(status, 2);
        return false;
    }
    return true;
}

// An SSR descriptor whose ranges leave the arrays is not staged (checks build).
__device__ __forceinline__ bool desc_in_bounds(const SsrDesc& d, int32_t nsr, int32_t n, int64_t nnz) {
    return 0 <= d.s0 && d.s0 <= d.s1 && d.s1 <= nsr && 0 <= d.r0 && d.r0 <= d.r1 && d.r1 <= n && 0 <= d.p0 &&
           d.p0 <= d.p1 && d.p1 <= nnz;
}
#endif

// Byte range [b, e) of an element slice rounded out to 16-byte boundaries.
template <int ESZ>
__device__ __forceinline__ void slice16(int64_t first, int64_t last_excl, int64_t& a0, uint32_t& bytes) {
    constexpr int64_t per = 16 / ESZ;
    a0 = first & ~(per - 1);
    const int64_t a1 = (last_excl + per - 1) & ~(per - 1);
    bytes = (uint32_t)((a1 - a0) * ESZ);
}

// MODE 0: SpMV with LPR lanes per row and gather chunks of U.  MODE 1: SpMM with G = LPR
// lanes per row and U columns per lane.  MODE 2: SpMV with FP64 values as FP32 pairs
// (VT = ds_t, one row per lane, FP64 accuracy on the FP32 pipes).  MODE 3: MODE 0 with
// delta-coded 16-bit columns (2 bytes per nonzero instead of 4; see spmv_rows), one row
// per lane, the consumers indexing x + cbase.  MODE 4 (kernel 5): the stage also holds
// the SSR's x window -- the runs of x its columns fall in, copied by the producer warp
// (one lane per run) -- and the 16-bit column codes are offsets into that window, so the
// consumers read x from shared memory instead of gathering it from L2.  MODE 5 (kernel
// 6): MODE 4 with FP64 values stored as FP32 pairs and row sums kept as FP32 pairs
// (spmv_rows_ds_win); the window holds the split x (FP32 pairs), or FP64 x when the
// split flagged an out-of-range element.
// At most 60 registers per thread, so two blocks of 16 consumer warps + 1 producer warp
// fit on one SM (65,536 registers).
template <typename VT, typename XT, typename AT, int LPR, int MODE, int U>
__global__ void __launch_bounds__(544, 2) csr3_tma_kernel(const TmaParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (P.skip && *P.skip) return;   // uniform over the grid: every thread leaves together
    const int S = P.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    SsrDesc* dsc = reinterpret_cast<SsrDesc*>(smem + 16 * S);   // one per stage
    unsigned char* stage0 = smem + P.header_bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = (blockDim.x >> 5) - 1;   // consumer warps; the last warp produces
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == W) {
        constexpr int CSZ = (MODE == 3 || MODE == 4 || MODE == 5) ? 2 : 4;   // bytes per stored column
        if constexpr (MODE == 4 || MODE == 5) {
            // ---------------- producer warp: lane 0 copies the slices, lane j the j-th x run
            // of the window (32 runs per round).  The metadata is loaded ahead in a short
            // pipeline -- the next SSR's descriptor and runs, the one after's run pointers --
            // so that no load waits on another while this SSR's stage is being refilled.
            const uint64_t pol = policy_evict_first();
            const uint64_t polx = policy_evict_normal();   // x runs: read again by nearby SSRs
            // MODE 5 stages the FP32-pair split of x (8 bytes an element, as FP64), or the
            // FP64 x itself when the split flagged an element
            const XT* __restrict__ xg = static_cast<const XT*>(MODE == 5 && *P.xflag ? (const void*)P.x64 : P.x);
            const int32_t* __restrict__ WP = P.wptr;
            const int2* __restrict__ W = P.win;
            const int g = gridDim.x;
            int t = blockIdx.x;
            SsrDesc d{};
            int2 run = make_int2(0, 0);
            int wcur = 0, wnext = 0, wnext_e = 0;   // runs of t start at wcur; of t + g at wnext
            if (t < P.nssr) {
                d = P.desc[t];
                wcur = WP[t];
                if (lane < WP[t + 1] - wcur) run = W[wcur + lane];
            }
            if (t + g < P.nssr) {
                wnext = WP[t + g];
                wnext_e = WP[t + g + 1];
            }
            for (int i = 0; t < P.nssr; t += g, ++i) {
                const int s = i % S;
                const int tn = t + g, tnn = t + 2 * g;
                SsrDesc dn{};
                int2 run_n = make_int2(0, 0);
                int w2 = 0, w2e = 0;
                if (tn < P.nssr) {
                    dn = P.desc[tn];
                    if (lane < wnext_e - wnext) run_n = W[wnext + lane];
                }
                if (tnn < P.nssr) {
                    w2 = WP[tnn];
                    w2e = WP[tnn + 1];
                }
                bool ok = true;
                if (lane == 0 && i >= S && !mbar_wait_bounded(&empty[s], ((i / S) - 1) & 1, P.timeout_ns)) {
                    report(P.status, 1);
                    ok = false;
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                unsigned char* st = stage0 + (size_t)s * P.stage_bytes;
                XT* xs = reinterpret_cast<XT*>(st + P.off_x);
#ifdef CSRK_CHECKS
                {   // a descriptor or a run outside its array: stage nothing, consumers skip the SSR
                    const int k = lane;
                    bool bad = !desc_in_bounds(d, P.nsr, P.n, P.nnz) || d.aux < 0 ||
                               (int64_t)d.cbase * (int64_t)sizeof(XT) > (int64_t)(P.off_perm - P.off_x);
                    if (!bad && k < d.aux) {
                        const int end = k + 1 == d.aux ? d.cbase : W[wcur + k + 1].y;
                        bad = run.x < 0 || run.y < 0 || end < run.y || (int64_t)run.x + (end - run.y) > P.n;
                    }
                    if (__any_sync(0xffffffffu, bad)) {
                        if (lane == 0) {
                            report(P.status, 2);
                            SsrDesc e = d;
                            e.s1 = e.s0;   // no super-rows
                            dsc[s] = e;
                            mbar_arrive_expect_tx(&full[s], 0);
                        }
                        __syncwarp();
                        d = dn;
                        run = run_n;
                        wcur = wnext;
                        wnext = w2;
                        wnext_e = w2e;
                        continue;
                    }
                }
#endif
                const int nrun = d.aux;                 // runs of this SSR's window
                const uint32_t xexact = (uint32_t)d.cbase * (uint32_t)sizeof(XT);   // elements covered
                const uint32_t xbulk = xexact & ~15u;
                if (lane == 0) {
                    dsc[s] = d;
                    // the window's last run may end at n off a 16-byte boundary: its last
                    // (at most 3) elements are copied with plain loads, before the arrive
                    if (xbulk != xexact) {
                        const int2 lr = W[wcur + nrun - 1];
                        const int len = d.cbase - lr.y;
                        for (int e = len - (int)((xexact - xbulk) / sizeof(XT)); e < len; ++e)
                            xs[lr.y + e] = xg[lr.x + e];
                    }
                    uint32_t b_srp, b_rp, b_col, b_val, b_pm = 0;
                    int64_t o_srp, o_rp, o_col, o_val, o_pm = 0;
                    slice16<4>(d.s0, (int64_t)d.s1 + 1, o_srp, b_srp);
                    slice16<4>(d.r0, (int64_t)d.r1 + 1, o_rp, b_rp);
                    slice16<CSZ>(d.p0, d.p1, o_col, b_col);
                    slice16<sizeof(VT)>(d.p0, d.p1, o_val, b_val);
                    if (P.yperm) slice16<4>(d.r0, d.r1, o_pm, b_pm);   // the fused unpermute's targets
                    uint32_t b_ord = 0;
                    int64_t o_ord = 0;
                    if (P.rord) slice16<2>(d.r0, d.r1, o_ord, b_ord);  // the rows' length order
                    mbar_arrive_expect_tx(&full[s], b_srp + b_rp + b_col + b_val + xbulk + b_pm + b_ord);
                    if (b_pm) bulk_g2s(st + P.off_perm, P.yperm + o_pm, b_pm, &full[s], pol);
                    if (b_ord) bulk_g2s(st + P.off_ord, P.rord + o_ord, b_ord, &full[s], pol);
                    bulk_g2s(st + P.off_srp, P.sr_ptr + o_srp, b_srp, &full[s], pol);
                    bulk_g2s(st + P.off_rp, P.rowptr + o_rp, b_rp, &full[s], pol);
                    if (b_col)
                        bulk_g2s(st + P.off_col, static_cast<const unsigned char*>(P.colidx) + o_col * CSZ,
                                 b_col, &full[s], pol);
                    if (b_val)
                        bulk_g2s(st + P.off_val, static_cast<const VT*>(P.vals) + o_val, b_val, &full[s], pol);
                }
                __syncwarp();
                // the runs, 32 per round (after the arrive, so the expected bytes come first);
                // a run ends where the next begins in the window, the last at the SSR's count
                for (int k0 = 0; k0 < nrun; k0 += 32) {
                    const int k = k0 + lane;
                    const int2 r = k0 == 0 ? run : (k < nrun ? W[wcur + k] : make_int2(0, 0));
                    const int next_base = __shfl_down_sync(0xffffffffu, r.y, 1);
                    if (k < nrun) {
                        const int end = k + 1 == nrun ? d.cbase : (lane == 31 ? W[wcur + k + 1].y : next_base);
                        const uint32_t b = ((uint32_t)(end - r.y) * (uint32_t)sizeof(XT)) & ~15u;
                        if (b) bulk_g2s(xs + r.y, xg + r.x, b, &full[s], polx);
                    }
                }
                d = dn;
                run = run_n;
                wcur = wnext;
                wnext = w2;
                wnext_e = w2e;
            }
        } else if (lane == 0) {
            // ---------------- producer: one elected lane issues the bulk copies
            const uint64_t pol = policy_evict_first();
            int i = 0;
            SsrDesc dn{};   // the next SSR's descriptor, loaded ahead of the wait for its stage
            if ((int)blockIdx.x < P.nssr) dn = P.desc[blockIdx.x];
            for (int t = blockIdx.x; t < P.nssr; t += gridDim.x, ++i) {
                const int s = i % S;
                const SsrDesc d = dn;
                if (t + (int)gridDim.x < P.nssr) dn = P.desc[t + gridDim.x];
                if (i >= S && !mbar_wait_bounded(&empty[s], ((i / S) - 1) & 1, P.timeout_ns)) {
                    report(P.status, 1);
                    break;
                }
#ifdef CSRK_CHECKS
                if (!desc_in_bounds(d, P.nsr, P.n, P.nnz)) {   // stage nothing, consumers skip it
                    report(P.status, 2);
                    SsrDesc e = d;
                    e.s1 = e.s0;
                    dsc[s] = e;
                    mbar_arrive_expect_tx(&full[s], 0);
                    continue;
                }
#endif
                dsc[s] = d;
                unsigned char* st = stage0 + (size_t)s * P.stage_bytes;
                uint32_t b_srp, b_rp, b_col, b_val;
                int64_t o_srp, o_rp, o_col, o_val;
                slice16<4>(d.s0, (int64_t)d.s1 + 1, o_srp, b_srp);
                slice16<4>(d.r0, (int64_t)d.r1 + 1, o_rp, b_rp);
                slice16<CSZ>(d.p0, d.p1, o_col, b_col);
                slice16<sizeof(VT)>(d.p0, d.p1, o_val, b_val);
                uint32_t b_pm = 0;
                int64_t o_pm = 0;
                if (MODE == 3 && P.yperm) slice16<4>(d.r0, d.r1, o_pm, b_pm);   // the fused unpermute's targets
                mbar_arrive_expect_tx(&full[s], b_srp + b_rp + b_col + b_val + b_pm);
                if (b_pm) bulk_g2s(st + P.off_perm, P.yperm + o_pm, b_pm, &full[s], pol);
                bulk_g2s(st + P.off_srp, P.sr_ptr + o_srp, b_srp, &full[s], pol);
                bulk_g2s(st + P.off_rp, P.rowptr + o_rp, b_rp, &full[s], pol);
                if (b_col)
                    bulk_g2s(st + P.off_col, static_cast<const unsigned char*>(P.colidx) + o_col * CSZ, b_col,
                             &full[s], pol);
                if (b_val)
                    bulk_g2s(st + P.off_val, static_cast<const VT*>(P.vals) + o_val, b_val,
                             &full[s], pol);
            }
        }
        return;
    }

    // ---------------- consumers
    const XT* __restrict__ x = static_cast<const XT*>(P.x);
    const bool slow = (MODE == 2 || MODE == 5) && P.xflag && *P.xflag;
    (void)slow;
    XT* __restrict__ y = static_cast<XT*>(P.y);
    int i = 0;
    int sr_seq = 0;   // index of the next super-row in this block's stream
    for (int t = blockIdx.x; t < P.nssr; t += gridDim.x, ++i) {
        const int s = i % S;
        if (!mbar_wait_bounded(&full[s], (i / S) & 1, P.timeout_ns)) {
            report(P.status, 1);
            // wait once more, bounded, for the copies of this stage to land before leaving
            mbar_wait_bounded(&full[s], (i / S) & 1, P.timeout_ns);
            return;
        }
        const SsrDesc d = dsc[s];
        const unsigned char* st = stage0 + (size_t)s * P.stage_bytes;
        const int32_t* srp = reinterpret_cast<const int32_t*>(st + P.off_srp) - (d.s0 & ~3);
        const int32_t* rp = reinterpret_cast<const int32_t*>(st + P.off_rp) - (d.r0 & ~3);
        const int32_t* col = reinterpret_cast<const int32_t*>(st + P.off_col) - (d.p0 & ~3);
        const uint16_t* col16 = reinterpret_cast<const uint16_t*>(st + P.off_col) - (d.p0 & ~7);
        (void)col16;
        constexpr int VPER = 16 / (int)sizeof(VT);
        const VT* val = reinterpret_cast<const VT*>(st + P.off_val) - (d.p0 & ~(VPER - 1));
        const int nsr = d.s1 - d.s0;
        // super-rows of this SSR that fall to this warp in the block-wide stream
        int first = (warp - sr_seq % W + W) % W;
        for (int j = first; j < nsr; j += W) {
            const int sr = d.s0 + j;
            const int rb = srp[sr], re = srp[sr + 1];
#ifdef CSRK_CHECKS
            {
                const int32_t* yp = (MODE == 3 || MODE == 4 || MODE == 5) && P.yperm
                                        ? reinterpret_cast<const int32_t*>(st + P.off_perm) - (d.r0 & ~3)
                                        : P.yperm;
                bool ok;
                if constexpr (MODE == 3)
                    ok = sr_in_bounds<1>(rb, re, d.r0, d.r1, d.p0, d.p1, rp, col16, d.cbase, P.n, yp, P.n, lane,
                                         P.status);
                else if constexpr (MODE == 4 || MODE == 5)
                    ok = sr_in_bounds<2>(rb, re, d.r0, d.r1, d.p0, d.p1, rp, col16, 0, d.cbase, yp, P.n, lane,
                                         P.status,
                                         P.rord ? reinterpret_cast<const uint16_t*>(st + P.off_ord) - (d.r0 & ~7)
                                                : nullptr);
                else
                    ok = sr_in_bounds<0>(rb, re, d.r0, d.r1, d.p0, d.p1, rp, col, 0, P.n, yp, P.n, lane, P.status);
                if (!ok) continue;
            }
#endif
            if constexpr (MODE == 2)
                spmv_rows_ds<U>(rb, re, rp, col, val, reinterpret_cast<const xpair*>(P.x), P.x64,
                                slow, y, P.alpha, P.beta, P.epi, lane, P.yperm);
            else if constexpr (MODE == 0)
                spmv_rows<VT, XT, AT, LPR, U>(rb, re, rp, col, val, x, y, P.alpha, P.beta, P.epi,
                                              lane, P.yperm);
            else if constexpr (MODE == 3)
                spmv_rows<VT, XT, AT, LPR, U, uint16_t>(
                    rb, re, rp, col16, val, x + d.cbase, y, P.alpha, P.beta, P.epi, lane,
                    P.yperm ? reinterpret_cast<const int32_t*>(st + P.off_perm) - (d.r0 & ~3) : nullptr);
            else if constexpr (MODE == 5)
                spmv_rows_ds_win<U>(rb, re, rp, col16, val, st + P.off_x, slow, y, P.alpha, P.beta, P.epi, lane,
                                    P.yperm ? reinterpret_cast<const int32_t*>(st + P.off_perm) - (d.r0 & ~3)
                                            : nullptr,
                                    P.rord ? reinterpret_cast<const uint16_t*>(st + P.off_ord) - (d.r0 & ~7)
                                           : nullptr,
                                    d.r0);
            else if constexpr (MODE == 4)
                spmv_rows<VT, XT, AT, 1, U, uint16_t, true>(
                    rb, re, rp, col16, val, reinterpret_cast<const XT*>(st + P.off_x), y, P.alpha, P.beta,
                    P.epi, lane,
                    P.yperm ? reinterpret_cast<const int32_t*>(st + P.off_perm) - (d.r0 & ~3) : nullptr,
                    P.rord ? reinterpret_cast<const uint16_t*>(st + P.off_ord) - (d.r0 & ~7) : nullptr, d.r0);
            else
                spmm_rows<VT, XT, AT, LPR, U>(rb, re, rp, col, val, x, P.ldx, y, P.ldy, P.k,
                                               P.alpha, P.beta, P.epi, lane);
        }
        sr_seq += nsr;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------------ direct kernel
// One block per SSR (the paper's 1-D grid), consumer warps stride the SSR's super-rows,
// operands read straight from global memory.  Used when an SSR does not fit a stage and
// as an autotuner alternative.
template <typename VT, typename XT, typename AT, int LPR, int MODE, int U>
__global__ void __launch_bounds__(512, 1) csr3_direct_kernel(const TmaParams P) {
    if (P.skip && *P.skip) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const XT* __restrict__ x = static_cast<const XT*>(P.x);
    const bool slow = MODE == 2 && P.xflag && *P.xflag;
    (void)slow;
    XT* __restrict__ y = static_cast<XT*>(P.y);
    const VT* __restrict__ vals = static_cast<const VT*>(P.vals);
    for (int t = blockIdx.x; t < P.nssr; t += gridDim.x) {
        const SsrDesc d = P.desc[t];
#ifdef CSRK_CHECKS
        if (!desc_in_bounds(d, P.nsr, P.n, P.nnz)) {
            if (threadIdx.x == 0) report(P.status, 2);
            continue;
        }
#endif
        for (int sr = d.s0 + warp; sr < d.s1; sr += W) {
            const int rb = __ldg(&P.sr_ptr[sr]), re = __ldg(&P.sr_ptr[sr + 1]);
            const int32_t* cols = static_cast<const int32_t*>(P.colidx);
#ifdef CSRK_CHECKS
            if (!sr_in_bounds<0>(rb, re, d.r0, d.r1, d.p0, d.p1, P.rowptr, cols, 0, P.n, P.yperm, P.n, lane,
                                 P.status))
                continue;
#endif
            if constexpr (MODE == 2)
                spmv_rows_ds<U>(rb, re, P.rowptr, cols, vals, reinterpret_cast<const xpair*>(P.x),
                                P.x64, slow, y, P.alpha, P.beta, P.epi, lane, P.yperm);
            else if constexpr (MODE == 0)
                spmv_rows<VT, XT, AT, LPR, U>(rb, re, P.rowptr, cols, vals, x, y, P.alpha,
                                              P.beta, P.epi, lane, P.yperm);
            else
                spmm_rows<VT, XT, AT, LPR, U>(rb, re, P.rowptr, cols, vals, x, P.ldx, y,
                                               P.ldy, P.k, P.alpha, P.beta, P.epi, lane);
        }
    }
}

}  // namespace dev
}  // namespace csrk
