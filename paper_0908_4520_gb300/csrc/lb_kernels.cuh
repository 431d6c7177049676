// Fused collide-stream kernels for sm_103a (templates; instantiated per
// velocity set in k_<set>.cu).
//
// One launch advances every cell by one time level of Eq. 2order:
//   pull-stream   f~_a(x) = S_a[f*_a](x)        exact shift by e_a (on-lattice) or
//                                               tensor-product Lax-Wendroff (off-lattice;
//                                               second-order upwind as an option)
//   moments       rho, rho u, 2 rho T (Sec. 2.2, D = 2)
//   equilibrium   f^eq_a = w_a rho sum_{kx+ky<=N} c_kx(u_x) c_ky(u_y) He_kx He_ky / (kx! ky!)
//                 (Sec. 2.1: the Hermite coefficients of the Maxwellian factorise per
//                 axis, c_k(u, T) = E[He_k(X)], X ~ Normal(u, T), from the recurrence
//                 c_{k+1} = u c_k + k (T - 1) c_{k-1})
//   relax         f*_a = f~_a + omega (f^eq_a - f~_a), omega = dt / (tau + dt/2)
//                 (dt / tau for the first-order scheme of Eq. slb)
//   store         f*_a (the next launch streams it)
//   diagnostics   FP64 grid sums of the observables of f~ (mass, momentum, the
//                 sin/cos Fourier amplitudes of u_y and sigma_xy, H norm)
// The stored variable is the deviation d = f - w rho0 (16-bit: d / (w S)), so
// moments and equilibrium are formed without the O(1) background and keep
// FP32 precision relative to the O(U0) signal.
//
// Work decomposition: a tile is ROWS lattice rows x 32 V columns; warp w of a
// block owns row y0 + w and each lane V consecutive cells, so every
// population-plane access of a warp is one contiguous row segment (coalesced,
// vectorised when V = 2).  The last tile of a row is shifted left to end at
// nx (its overlap with the previous tile is recomputed but neither stored nor
// counted), so every warp of a row wider than a tile is full.  The grid is
// persistent (a multiple of the SM count) and walks tiles row-major (the
// TMA-staged kernel: column-major in bands of tile rows for the exact-shift
// sets), so the halo rows a tile re-reads were fetched moments earlier by its
// neighbours and sit in L2.  Populations carry a rim of periodic images (ghost columns and
// rows), rewritten by every store, so no read ever wraps.
//
// Two step kernels share the collision code and give bitwise-identical results:
//  * lb_tma_step_kernel (the hot path): one producer warp streams, per group of
//    velocities, the tile's source box (with its halo) from HBM into a ring of
//    shared-memory stages with cp.async.bulk.tensor, completion tracked by
//    mbarriers; the consumer warps read their row from shared memory, so the
//    next tile's loads overlap this tile's collision.  Every wait is bounded:
//    on expiry the kernel flags LB_ERR_TIMEOUT in the status word and returns.
//  * lb_fused_kernel: plain coalesced loads from global memory (moments read-back,
//    the first level, FP64 storage and grids too small for the TMA tiles).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lb_device.h"

namespace lbk {

// ---------------------------------------------------------------- storage I/O
template <class S>
struct Is16 : std::false_type {};
template <>
struct Is16<__nv_bfloat16> : std::true_type {};
template <>
struct Is16<__half> : std::true_type {};

template <class S, class R>
__device__ __forceinline__ R ld1(const S* p, R scale) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        return __bfloat162float(__ldg(p)) * scale;
    } else if constexpr (std::is_same<S, __half>::value) {
        return __half2float(__ldg(p)) * scale;
    } else {
        (void)scale;
        return __ldg(p);
    }
}

// shared-memory loads (plain, no read-only path)
template <class S, class R>
__device__ __forceinline__ R sld1(const S* p, R scale) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        return __bfloat162float(*p) * scale;
    } else if constexpr (std::is_same<S, __half>::value) {
        return __half2float(*p) * scale;
    } else {
        (void)scale;
        return *p;
    }
}

template <class S, class R>
__device__ __forceinline__ void sld2(const S* p, R scale, R& v0, R& v1) {
    if constexpr (std::is_same<S, float>::value) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v0 = t.x;
        v1 = t.y;
    } else if constexpr (std::is_same<S, double>::value) {
        const double2 t = *reinterpret_cast<const double2*>(p);
        v0 = t.x;
        v1 = t.y;
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        v0 = t.x * scale;
        v1 = t.y * scale;
    } else {
        const float2 t = __half22float2(*reinterpret_cast<const __half2*>(p));
        v0 = t.x * scale;
        v1 = t.y * scale;
    }
    (void)scale;
}

// aligned pair p[0], p[1]
template <class S, class R>
__device__ __forceinline__ void ld2(const S* p, R scale, R& v0, R& v1) {
    if constexpr (std::is_same<S, float>::value) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(p));
        v0 = t.x;
        v1 = t.y;
    } else if constexpr (std::is_same<S, double>::value) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p));
        v0 = t.x;
        v1 = t.y;
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        const float2 t = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
        v0 = t.x * scale;
        v1 = t.y * scale;
    } else {
        const float2 t = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        v0 = t.x * scale;
        v1 = t.y * scale;
    }
    (void)scale;
}

template <class S, class R>
__device__ __forceinline__ void st1(S* p, R v, R scinv) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        *p = __float2bfloat16_rn(v * scinv);
    } else if constexpr (std::is_same<S, __half>::value) {
        *p = __float2half_rn(v * scinv);
    } else {
        (void)scinv;
        *p = v;
    }
}

template <class S, class R>
__device__ __forceinline__ void st2(S* p, R v0, R v1, R scinv) {
    if constexpr (std::is_same<S, float>::value) {
        __stcs(reinterpret_cast<float2*>(p), make_float2(v0, v1));
    } else if constexpr (std::is_same<S, double>::value) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(v0, v1));
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        __stcs(reinterpret_cast<__nv_bfloat162*>(p), __floats2bfloat162_rn(v0 * scinv, v1 * scinv));
    } else {
        __stcs(reinterpret_cast<__half2*>(p), __floats2half2_rn(v0 * scinv, v1 * scinv));
    }
    (void)scinv;
}

template <class S, class R>
__device__ __forceinline__ R load_scale(const Tab<R>& t, int a) {
    if constexpr (Is16<S>::value) return t.sc[a];
    (void)t;
    (void)a;
    return R(1);
}

template <class S, class R>
__device__ __forceinline__ R store_scale(const Tab<R>& t, int a) {
    if constexpr (Is16<S>::value) return t.scinv[a];
    (void)t;
    (void)a;
    return R(1);
}

// ---------------------------------------------------------------- stochastic rounding
// 16-bit stores of the step kernels round stochastically (unbiased: the stored
// value equals the FP32 value in expectation), so per-step changes smaller than
// half a 16-bit ulp are not rounded away (the decay would stagnate).  The random
// bits come from a counter-based generator: MurmurHash3's 32-bit finalizer of
// (cell, level) seeds one 32-bit linear congruential stream per cell (multiplier
// 1664525, increment 1013904223), advanced once per velocity; its high bits are
// the rounding bits.  The result does not depend on the launch geometry.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint32_t sr_next(uint32_t x) { return x * 1664525u + 1013904223u; }
__device__ __forceinline__ uint32_t sr_seed(long long level, long long cell) {
    return fmix32((uint32_t)cell ^ fmix32((uint32_t)level * 0x9e3779b9u + 0x7f4a7c15u));
}
// random bits below the 16-bit mantissa of an FP32 value: 13 for FP16, 16 for BF16
template <class S>
__device__ __forceinline__ uint32_t sr_bits(uint32_t r) {
    return std::is_same<S, __half>::value ? (r >> 19) : (r >> 16);
}

// storage value of a deviation (16-bit: stochastic rounding with the random bits of r)
template <class S, class R>
__device__ __forceinline__ S to_storage(R v, R scinv, uint32_t r) {
    if constexpr (std::is_same<S, __half>::value) {
        return __float2half_rz(__uint_as_float(__float_as_uint(v * scinv) + sr_bits<S>(r)));
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        return __float2bfloat16_rz(__uint_as_float(__float_as_uint(v * scinv) + sr_bits<S>(r)));
    } else {
        (void)scinv;
        (void)r;
        return v;
    }
}

// Two scaled values (already multiplied by the storage scale) rounded stochastically
// into one 16-bit pair word, the first in the low half (one conversion instruction).
template <class S>
__device__ __forceinline__ uint32_t to_storage16x2(float h0, float h1, uint32_t r0, uint32_t r1) {
    const float a = __uint_as_float(__float_as_uint(h0) + sr_bits<S>(r0));
    const float b = __uint_as_float(__float_as_uint(h1) + sr_bits<S>(r1));
    uint32_t d;
    if constexpr (std::is_same<S, __half>::value) {
        asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    } else {
        asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    }
    return d;
}

template <class S>
__device__ __forceinline__ void store_raw(S* p, S a) {
    *p = a;
}
template <class S>
__device__ __forceinline__ void store_raw2(S* p, S a, S b) {
    if constexpr (std::is_same<S, float>::value) {
        __stcs(reinterpret_cast<float2*>(p), make_float2(a, b));
    } else if constexpr (std::is_same<S, double>::value) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(a, b));
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        __nv_bfloat162 t;
        t.x = a;
        t.y = b;
        __stcs(reinterpret_cast<__nv_bfloat162*>(p), t);
    } else {
        __half2 t;
        t.x = a;
        t.y = b;
        __stcs(reinterpret_cast<__half2*>(p), t);
    }
}

// compile-time loop: f(integral_constant<int, a>) for a in [A_, Q)
template <int A_, int Q, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (A_ < Q) {
        f(std::integral_constant<int, A_>{});
        static_for<A_ + 1, Q>(f);
    }
}

// ------------------------------------------------------------ packed lanes
// Two cells of a thread travel as one packed pair (f2) through the paired FP32
// instructions of sm_100-class GPUs (add/sub/mul/fma .f32x2).  Each half of a
// pair rounds exactly as the scalar instruction would, so a pair gives the
// results of two scalar evaluations bit for bit.
struct __align__(8) f2 {
    float x, y;
};

__device__ __forceinline__ unsigned long long f2_bits(f2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ f2 f2_from(unsigned long long r) {
    f2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from(d);
}
__device__ __forceinline__ f2 vadd(f2 a, f2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}
__device__ __forceinline__ f2 vsub(f2 a, f2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}
__device__ __forceinline__ f2 vmul(f2 a, f2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}
__device__ __forceinline__ f2 vrcp(f2 a) { return f2{1.0f / a.x, 1.0f / a.y}; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vrcp(float a) { return 1.0f / a; }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vrcp(double a) { return 1.0 / a; }

template <class T>
struct LaneScalar {
    using type = T;
};
template <>
struct LaneScalar<f2> {
    using type = float;
};

template <class T>
__device__ __forceinline__ T vsplat(typename LaneScalar<T>::type c) {
    if constexpr (std::is_same<T, f2>::value) {
        return f2{c, c};
    } else {
        return c;
    }
}

// lane K of a packed value, and packing of V lane values
template <int K>
__device__ __forceinline__ float lane_get(const f2& v) {
    if constexpr (K == 0) {
        return v.x;
    } else {
        return v.y;
    }
}
template <int K>
__device__ __forceinline__ float lane_get(const float& v) {
    return v;
}
template <int K>
__device__ __forceinline__ double lane_get(const double& v) {
    return v;
}
template <class T, class R>
__device__ __forceinline__ T pack_lanes(R v0, R v1) {
    if constexpr (std::is_same<T, f2>::value) {
        return f2{v0, v1};
    } else {
        (void)v1;
        return v0;
    }
}

template <class R, int V>
struct Pack {
    using T = R;
};
template <>
struct Pack<float, 2> {
    using T = f2;
};

// ------------------------------------------------------------ configuration
// Launch shapes, from sweeps at 4096^2 (FP32, N = 3) and 2048^2 (D2Q64, N = 4):
//  * Lax-Wendroff (Gauss-Hermite product) sets: one cell per lane and many warps
//    (19 consumer rows, or 15 for q = 64), 6 velocities per TMA stage (12 for q = 64);
//  * exact-shift sets: two cells per lane (packed f32x2), 11 consumer rows (13 for
//    q <= 25), 18 velocities per stage.
// The plain-load kernel takes the same cells per lane as the TMA-staged one, so the
// two give the same bits.  Each value is overridable at build time (0 = the choice above).
#ifndef LB_CFG_V
#define LB_CFG_V 0
#endif
#ifndef LB_TMA_V
#define LB_TMA_V 0
#endif
#ifndef LB_CFG_ROWS
#define LB_CFG_ROWS 8
#endif
#ifndef LB_CFG_MINB
#define LB_CFG_MINB 0
#endif
#ifndef LB_TMA_ROWS
#define LB_TMA_ROWS 0
#endif
#ifndef LB_TMA_K
#define LB_TMA_K 0
#endif
#ifndef LB_TMA_TILE_SYNC
#define LB_TMA_TILE_SYNC -1  // -1: per set and storage (see TmaCfg), 0: never, 1: always
#endif
#ifndef LB_TMA_EVICT_LAST
#define LB_TMA_EVICT_LAST 1  // TMA loads keep their lines in L2 for the neighbouring tiles (-3 % DRAM reads)
#endif
#ifndef LB_PAIR_COLLISION
#define LB_PAIR_COLLISION 1  // one cell per lane: collide velocity pairs as packed f32x2 values
#endif
#ifndef LB_TMA_HALO
#define LB_TMA_HALO -1  // -1: per set and storage (see TmaCfg), 0: never, 1: always
#endif
#ifndef LB_TMA_NS_TILES
#define LB_TMA_NS_TILES 2  // ring depth cap, in tiles of stages
#endif
#ifndef LB_TMA_SMEM
#define LB_TMA_SMEM (200 * 1024)
#endif
#ifndef LB_TMA_MINB
#define LB_TMA_MINB 1
#endif
#ifndef LB_TMA_BAND
// TMA kernel tile order: -1 per set, 0 row-major, B > 0 column-major in bands of B tile rows.
// Measured at 4096^2 FP32 (same box; row-major / bands of 4, 8, 16): D2Q37 12.6 / 18.2 / 16.7 /
// 14.6 GLUPS, D2Q36-GH 14.8 / 7.7 / 7.6 / 7.4, D2Q16-GH 38.5 / 35.3 / 32.4 / 31.2, D2Q36-GH FP16
// 16.8 / 15.6 / 11.8 / 14.8: bands for the exact-shift sets, row-major for Lax-Wendroff
#define LB_TMA_BAND -1
#endif
#ifndef LB_TMA_BAND_SHIFT
#define LB_TMA_BAND_SHIFT 4  // band height of the exact-shift sets under LB_TMA_BAND = -1
#endif
#ifndef LB_TMA_WIDE_WARPS
#define LB_TMA_WIDE_WARPS 0  // consumer warps of the store-staged kernel (two per tile row); 0: 18, q = 64: 14
#endif
#ifndef LB_TMA_WIDE_SMEM
// ring + output tile of the store-staged kernel.  D2Q36-GH FP32 at 4096^2 (GLUPS): 224 KB
// (8 stages) 17.2, 192 KB (6 stages: one tile ahead) 17.5; 9 velocities per stage instead of 6:
// +0.2 %; 16 / 20 consumer warps instead of 18: 15.0 / 15.9
#define LB_TMA_WIDE_SMEM (192 * 1024)
#endif
#ifndef LB_DIAG_PREFETCH
// load sin/cos of the diagnostics before the collision: -1 per set and kernel (measured at
// 4096^2 FP32, same box: TMA kernel with plain stores D2Q16-GH 35.7 -> 38.5 GLUPS, D2Q37
// 12.6 -> 12.6, D2Q36-GH 14.8 -> 11.8; store-staged kernel D2Q36-GH 17.44 -> 17.91; so
// D2Q16-GH and the store-staged kernel), 0 never, 1 always
#define LB_DIAG_PREFETCH -1
#endif

// cells per lane along x (FP64 storage: always 1)
template <class VS, class S, int OVERRIDE>
constexpr int cells_per_lane() {
    return sizeof(S) == 8 ? 1 : (OVERRIDE > 0 ? OVERRIDE : (VS::kOnLattice ? 2 : 1));
}

template <class VS, class S>
struct Cfg {
    static constexpr int V = cells_per_lane<VS, S, (LB_CFG_V > 0 ? LB_CFG_V : LB_TMA_V)>();
    static constexpr int ROWS = LB_CFG_ROWS;
    static constexpr int THREADS = 32 * ROWS;
    // one cell per lane needs under 128 registers: two blocks (16 warps) per SM
    static constexpr int MINB = LB_CFG_MINB > 0 ? LB_CFG_MINB : (V == 1 && sizeof(S) != 8 ? 2 : 1);
};

// UPW: second-order upwind streaming of a Lax-Wendroff set (one cell per lane): lanes
// 0, 1 and 30, 31 compute the y pass of the two columns on either side of the 28 cells
// that lanes 2..29 own, and the box carries two extra rows above and below.
// WIDE: the store-staged variant of the Lax-Wendroff kernel (one cell per lane, halo
// lanes): two warps share a tile row (FP32: 30 cells each, 60 per row, 240 bytes; 16-bit:
// 28 cells each - lanes 30, 31 idle - 56 per row, 112 bytes: whole 16-byte TMA granules),
// the consumer warps write the relaxed populations of the tile (16-bit: stochastically
// rounded) into a shared-memory output tile, and the producer warp writes it to HBM with
// one TMA tensor store per tile (cp.async.bulk.tensor, shared -> global), so no thread
// issues per-velocity global stores and every DRAM sector of the tile is written whole.
template <class VS, class S, bool UPW = false, bool WIDE = false>
struct TmaCfg {
    static constexpr bool LW = !VS::kOnLattice;
    static constexpr int V = cells_per_lane<VS, S, LB_TMA_V>();
    static_assert(!UPW || (LW && V == 1), "upwind TMA staging: Lax-Wendroff sets, one cell per lane");
    static_assert(!WIDE || (LW && V == 1 && !UPW && sizeof(S) <= 4), "store staging: 32/16-bit Lax-Wendroff sets");
    // consumer warps (+ one producer warp); the register cap follows from the count
    // (exact shift at 4096^2 FP32, 11 / 13 rows, GLUPS: D2Q37 18.3 / 16.8, D2Q25 21.3 / 22.3,
    // D2Q21 25.4 / 27.7, D2Q17 41.6 / 42.1, D2Q16 44.7 / 45.1, D2Q9 68.6 / 72.6)
    static constexpr int CW = WIDE ? (LB_TMA_WIDE_WARPS > 0 ? LB_TMA_WIDE_WARPS : (VS::Q > 40 ? 14 : 18))
                                   : (LB_TMA_ROWS > 0 ? LB_TMA_ROWS : (LW ? (VS::Q > 40 ? 15 : 19) : (VS::Q > 30 ? 11 : 13)));
    static constexpr int WPR = WIDE ? 2 : 1;            // consumer warps per tile row
    static constexpr int ROWS = CW / WPR;               // lattice rows of a tile
    static_assert(CW % WPR == 0, "whole tile rows");
    static constexpr int TW = 32 * V;
    // Edge lanes as halo lanes (30 cells a row) and a per-tile barrier of the consumer warps,
    // chosen per set and storage by the sweep at 4096^2 / 2048^2 (GLUPS, no halo / halo /
    // halo + barrier): D2Q16 FP32 29.5 / 35.5 / 30.4; D2Q36 FP32 12.5 / 9.6 / 14.5; D2Q36
    // 16-bit 12.1 / 15.9 / 14.4; D2Q64 FP32 5.38 / 4.95 / 4.97; D2Q64 16-bit 4.37 / 6.40 / 6.28.
    static constexpr bool FP32_Q64 = sizeof(S) == 4 && VS::Q > 40;
    static constexpr bool HALO = WIDE || (!UPW && LW && V == 1 && (LB_TMA_HALO > 0 || (LB_TMA_HALO < 0 && !FP32_Q64)));
    // (store-staged: no per-tile barrier; without per-velocity stores the warps stay together,
    // and the barrier cost 5 %: 16.3 against 17.2 GLUPS for D2Q36-GH FP32 at 4096^2)
    static constexpr bool TILE_SYNC =
        LB_TMA_TILE_SYNC > 0 || (LB_TMA_TILE_SYNC < 0 && !WIDE && (HALO || UPW) && sizeof(S) == 4 && VS::Q == 36);
    // cells a warp produces (store-staged 16-bit: 28, so that a tile row is 7 granules)
    static constexpr int WCELLS = UPW ? 28 : (WIDE && sizeof(S) == 2 ? 28 : (HALO ? 30 : TW));
    static constexpr int TWO = WPR * WCELLS;            // cells a tile row produces
    static constexpr int GX = UPW ? 2 : 1;              // stencil reach (columns and rows) of the box
    static constexpr int BAND = LB_TMA_BAND >= 0 ? LB_TMA_BAND : (LW ? 0 : LB_TMA_BAND_SHIFT);  // tile order
    static constexpr int AL = 16 / (int)sizeof(S);      // TMA x coordinates are multiples of 16 bytes
    static_assert(!WIDE || TWO % AL == 0, "store-staged tile rows are whole 16-byte granules");
    static constexpr int BW = WIDE ? TWO + 2 * AL : ((HALO || UPW) ? 32 + AL : (LW ? TW + 2 * AL : TW + AL));
    static constexpr int BH = LW ? ROWS + 2 * GX : ROWS;
    static constexpr int BOX = BW * BH;                 // elements of one velocity's box
    // stride of the velocity slots in a stage: dense for one 3-D box (Lax-Wendroff),
    // 128-byte aligned for separate boxes (exact shift)
    static constexpr int SLOT = LW ? BOX : ((BOX * (int)sizeof(S) + 127) / 128 * 128) / (int)sizeof(S);
    static constexpr int K = LB_TMA_K > 0 ? LB_TMA_K : (LW ? (VS::Q > 40 ? 12 : 6) : 18);  // velocities per stage
    static constexpr int NG = (VS::Q + K - 1) / K;      // stages per tile
    static constexpr int STAGE_BYTES = (K * SLOT * (int)sizeof(S) + 127) / 128 * 128;
    // output tile of the store-staged kernel: [velocity][row][TWO cells]
    static constexpr int OUT_BYTES = WIDE ? (VS::Q * ROWS * TWO * (int)sizeof(S) + 127) / 128 * 128 : 0;
    static constexpr int NS_FIT = ((WIDE ? LB_TMA_WIDE_SMEM - OUT_BYTES : LB_TMA_SMEM) - 512) / STAGE_BYTES;
    static constexpr int NS = NS_FIT < LB_TMA_NS_TILES * NG ? NS_FIT : LB_TMA_NS_TILES * NG;
    static constexpr int THREADS = 32 * (CW + 1);       // + one producer warp
    // registers a thread may hold: each SM sub-partition's 16384 registers are shared by
    // ceil(warps / 4) warps of the block (255 for 8 warps, 168 for 9..12, 128 for 13..16)
    static constexpr int WARPS_PER_SMSP = (CW + 1 + 3) / 4;
    static constexpr int MAXREG_FIT = 16384 / (32 * WARPS_PER_SMSP) / 8 * 8;
    static constexpr int MAXREG = MAXREG_FIT > 255 ? 255 : MAXREG_FIT;
    // ring, output tile, full/empty barriers of the ring, tile-done and output-free barriers
    static constexpr int SMEM = NS * STAGE_BYTES + OUT_BYTES + 2 * NS * 8 + 16 + 128;  // + alignment slack
    static constexpr int BOX_D = LW ? K : 1;            // velocities per TMA box
};

// ------------------------------------------------------------ equilibrium
// Deviation of the truncated Hermite equilibrium from w rho0, for one cell:
// deq_a = w_a (drho + rho * sum'_{kx+ky<=N} c_kx(ux) c_ky(uy) hn[ix][kx] hn[iy][ky]),
// sum' without the (0,0) term (which is rho itself).  The velocities are visited
// grouped by their x axis node, so only one row of x partial sums is live.
// emit(integral_constant<a>, deq_a) is called once per velocity.
template <class VS, int N, class R, class Emit>
__device__ __forceinline__ void equilibrium_dev(const Tab<R>& t, R drho, R rho, R ux, R uy, R th,
                                                Emit&& emit) {
    constexpr int NA = VS::NA;
    R cx[N + 1], cy[N + 1];
    cx[0] = R(1);
    cy[0] = R(1);
    cx[1] = ux;
    cy[1] = uy;
#pragma unroll
    for (int k = 1; k < N; ++k) {
        cx[k + 1] = ux * cx[k] + R(k) * th * cx[k - 1];
        cy[k + 1] = uy * cy[k] + R(k) * th * cy[k - 1];
    }
    R qy[NA][N + 1];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        qy[j][0] = R(0);
#pragma unroll
        for (int ky = 1; ky <= N; ++ky) qy[j][ky] = cy[ky] * t.hn[j][ky];
    }
    static_for<0, NA>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        // px[0] excludes kx = 0; px[ky>=1] = sum_{kx <= N-ky} cx[kx] hn[I][kx]
        R px[N + 1];
#pragma unroll
        for (int ky = 0; ky <= N; ++ky) {
            R s = (ky == 0) ? R(0) : R(1);
#pragma unroll
            for (int kx = 1; kx <= N - ky; ++kx) s = fma(cx[kx], t.hn[I][kx], s);
            px[ky] = s;
        }
        static_for<0, VS::Q>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (VS::ix(a) == I) {
                constexpr int iy = VS::iy(a);
                R s = px[0];
#pragma unroll
                for (int ky = 1; ky <= N; ++ky) s = fma(px[ky], qy[iy][ky], s);
                emit(ac, t.w[a] * fma(rho, s, drho));
            }
        });
    });
}

// ------------------------------------------------------------ tile geometry
struct Lane {
    int x;          // first cell of the lane
    int xl;         // column read for the lane (x, or nx for lanes past the grid)
    bool own;       // x < nx and not a recomputed overlap cell
};

// TMA-staged Lax-Wendroff with one cell per lane: the warp's edge lanes are halo lanes
// (columns x0 - 1 and x0 + 30), whose y-pass only feeds their neighbours' x-pass, so no
// lane reads an extra column; lanes 1..30 own cells x0 .. x0 + 29.
// (own: the number of cells the warp owns, lanes 1..own; 30, or 28 for the store-staged
// 16-bit kernel, whose lanes 30 and 31 are idle)
__device__ __forceinline__ Lane halo_lane_geometry(int lane, int x0, int tile_start, int nx, int own = 30) {
    Lane g;
    g.x = x0 - 1 + lane;
    g.own = lane >= 1 && lane <= own && g.x < nx && g.x >= tile_start;
    g.xl = g.x;
    return g;
}

// The same for second-order upwind: lanes 0, 1 and 30, 31 are halo lanes (columns
// x0 - 2, x0 - 1, x0 + 28, x0 + 29); lanes 2..29 own cells x0 .. x0 + 27.
__device__ __forceinline__ Lane upwind_lane_geometry(int lane, int x0, int tile_start, int nx) {
    Lane g;
    g.x = x0 - 2 + lane;
    g.own = lane >= 2 && lane <= 29 && g.x < nx && g.x >= tile_start;
    g.xl = g.x;
    return g;
}

// Tile (ty, tx) of the TMA kernel's tile index.  Row-major (B = 0), or column-major within
// bands of B tile rows, so that the tiles in flight at one time (consecutive indices) are
// neighbours in x and in y: the exact-shift sets' boxes, displaced by up to max|e| rows
// and columns, then find the rows of the tiles above and beside them in L2.
template <int B>
__device__ __forceinline__ void tma_tile_coords(int tile, int ntiles_x, int ntiles, int& ty, int& tx) {
    if constexpr (B <= 0) {
        ty = tile / ntiles_x;
        tx = tile - ty * ntiles_x;
    } else {
        const int per_band = B * ntiles_x;
        const int band = tile / per_band;
        const int r = tile - band * per_band;
        const int ntiles_y = ntiles / ntiles_x;
        const int rows = min(B, ntiles_y - band * B);
        tx = r / rows;
        ty = band * B + (r - tx * rows);
    }
}

template <int V>
__device__ __forceinline__ Lane lane_geometry(int lane, int x0, int tile_start, int nx) {
    Lane g;
    g.x = x0 + lane * V;
    g.own = g.x < nx && g.x >= tile_start;
    g.xl = g.x < nx ? g.x : nx;  // the first column past the grid is a valid image
    return g;
}

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Write the lane's V storage values of plane `pl` (pointer to cell (0,0)) at
// every periodic image of (x, y) inside the ghost rim (not at (x, y) itself).
template <class S, class R, int V>
__device__ __forceinline__ void store_images(const Args<R>& A, S* pl, int x, int y, const S (&v)[V]) {
    int ylo = y;
    while (ylo - A.ny >= -A.gy) ylo -= A.ny;
    int xlo = x;
    while (xlo - A.nx >= -kGhostX) xlo -= A.nx;
    for (int yi = ylo; yi < A.ny + A.gy; yi += A.ny) {
        for (int xi = xlo; xi + V <= A.nx + kGhostX; xi += A.nx) {
            if (xi == x && yi == y) continue;
            S* q = pl + (long long)yi * A.pitch + xi;
            if constexpr (V == 2) {
                store_raw2<S>(q, v[0], v[1]);
            } else {
                store_raw<S>(q, v[0]);
            }
        }
    }
}

// Out-of-line image writer (boundary lanes only), so the unrolled callers stay small.
// Copy the q values this thread just stored at (x.., y) to their periodic images.
template <class S, class R, int V>
__device__ __noinline__ void rim_images(const Args<R>& A, S* dst, int q, int x, int y) {
    for (int a = 0; a < q; ++a) {
        S* pl = dst + (long long)a * A.plane + A.origin;
        const S* p = pl + (long long)y * A.pitch + x;
        S v[V];
        v[0] = p[0];
        if constexpr (V == 2) v[V - 1] = p[1];
        store_images<S, R, V>(A, pl, x, y, v);
    }
}

// The same for the store-staged kernel: the values are taken from the output tile in shared
// memory (out[a * ostride]), which the TMA store writes to (x, y) itself.
template <class S, class R>
__device__ __noinline__ void rim_images_tile(const Args<R>& A, S* dst, const S* out, int ostride, int q, int x, int y) {
    for (int a = 0; a < q; ++a) {
        S* pl = dst + (long long)a * A.plane + A.origin;
        const S v[1] = {out[a * ostride]};
        store_images<S, R, 1>(A, pl, x, y, v);
    }
}

// Write the lane's values at (x, y) and at every periodic image.
// (round to nearest: used for the initial state)
template <class S, class R, int V>
__device__ __forceinline__ void store_cells(const Args<R>& A, S* pl, int x, int y, const R (&v)[V], R si) {
    S* p = pl + (long long)y * A.pitch + x;
    S sv[V];
    if constexpr (V == 2) {
        st2<S, R>(p, v[0], v[1], si);
        sv[0] = p[0];
        sv[V - 1] = p[1];
    } else {
        st1<S, R>(p, v[0], si);
        sv[0] = p[0];
    }
    if (x < kGhostX || x + V > A.nx - kGhostX || y < A.gy || y >= A.ny - A.gy) store_images<S, R, V>(A, pl, x, y, sv);
}

// ------------------------------------------------------------ collision (shared)
// Result of colliding one cell (or a packed pair of cells).
template <class T>
struct CellOut {
    T drho, jx, jy;   // deviation moments: rho - rho0, rho u
    T ux, uy, th;     // velocity, T - 1
    T sig;            // sigma_xy = (1 - omega/2) sum xi_x xi_y (f~ - f^eq)   (diag)
    T h;              // sum (f~ - w rho0)^2 / w                               (diag)
};

// The one definition of the per-cell arithmetic; every kernel calls it.  The
// streamed deviations are f(integral_constant<a>) (references, relaxed in place
// when COLLIDE).  T is a scalar or a packed pair of cells.
//  * moments from per-axis-node sums: C[i] = sum_{ix = i} d, Ry[j] = sum_{iy = j} d;
//    rho - rho0 = sum C, rho u_x = sum a_i C[i], rho u_y = sum a_j Ry[j],
//    sum |xi|^2 d = sum a_i^2 (C[i] + Ry[i])  (Sec. 2.2; kinetic T with D = 2)
//  * diagnostics (diag): Pi_xy = sum xi_x xi_y d and H = sum d^2 / w of the
//    streamed state; sigma_xy = (1 - omega/2) (Pi_xy - rho u_x u_y), since the
//    truncated equilibrium carries exactly the xy moment rho u_x u_y of the
//    Maxwellian when the quadrature degree is >= N + 2
//  * equilibrium (Sec. 2.1), per axis: f^eq_a - w rho0 = w_a (drho + rho S'_a),
//    S'_a = sum'_{kx+ky<=N} c_kx(u_x) c_ky(u_y) hn[ix][kx] hn[iy][ky]; for product
//    weights w_a = W_ix W_iy the weights fold into the per-axis factors, so
//    omega (f^eq_a - w_a rho0) = sum_{ky<=N} PX[ix][ky] QY[iy][ky]
//  * relaxation (Eq. 2order): f* = (1 - omega) f~ + omega f^eq, one FMA a velocity
//  * N = 1 (Sec. 3.3, Eq. lbm1): f^eq = w rho (1 + xi.u) has no xy moment, so
//    sigma_xy = (1 - omega/2) Pi_xy, and neither has its force term w rho g xi_y
//  * body force g = (0, g) (Secs. 2.1, 2.2; forced): rho u_y = sum xi_y f~ + rho g hdt,
//    2 rho T gains 2 hdt rho g u_y, sigma_xy gains hdt rho g u_x (the xy moment of
//    the force term), hdt = dt/2 (Eq. 2order; 0 for the first-order scheme of
//    Eq. slb, whose stored variable is f itself), and the force term relaxed with
//    weight omega tau (= dt for Eq. slb, where omega = dt / tau),
//    omega tau g_a = omega w_a rho g sum_{ky>=1} c_kx c_{ky-1} He_kx He_ky / (kx! (ky-1)!),
//    folds into the y factors: c_ky -> c_ky + ky tau g c_{ky-1} (ky >= 1)
template <class VS, int N, class R, class T, bool COLLIDE, class F>
__device__ __forceinline__ CellOut<T> collide_cell(const Tab<R>& t, R rho0, R omega, R sigma_fac, int isothermal,
                                                   bool diag, bool forced, T gf, R tau, R hdt, F&& f) {
    constexpr int NA = VS::NA;
    const T zero = vsplat<T>(R(0));
    T C[NA], Ry[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) C[i] = Ry[i] = zero;
    static_for<0, VS::Q>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        const T v = f(ac);
        C[VS::ix(a)] = vadd(C[VS::ix(a)], v);
        Ry[VS::iy(a)] = vadd(Ry[VS::iy(a)], v);
    });
    T drho = C[0], jx = vmul(vsplat<T>(t.a[0]), C[0]), jy = vmul(vsplat<T>(t.a[0]), Ry[0]);
    T en = vmul(vsplat<T>(t.a2[0]), vadd(C[0], Ry[0]));
#pragma unroll
    for (int i = 1; i < NA; ++i) {
        drho = vadd(drho, C[i]);
        jx = vfma(vsplat<T>(t.a[i]), C[i], jx);
        jy = vfma(vsplat<T>(t.a[i]), Ry[i], jy);
        en = vfma(vsplat<T>(t.a2[i]), vadd(C[i], Ry[i]), en);
    }
    CellOut<T> o;
    T pxy = zero, h = zero;
    if (diag) {
        T P[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) P[i] = zero;
        static_for<0, VS::Q>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            const T v = f(ac);
            P[VS::ix(a)] = vfma(vsplat<T>(t.a[VS::iy(a)]), v, P[VS::ix(a)]);
            h = vfma(vmul(v, vsplat<T>(t.winv[a])), v, h);
        });
#pragma unroll
        for (int i = 0; i < NA; ++i) pxy = vfma(vsplat<T>(t.a[i]), P[i], pxy);
    }
    const T rho = vadd(vsplat<T>(rho0), drho);
    const T rg = forced ? vmul(rho, gf) : zero;  // rho g
    if (forced) jy = vfma(vsplat<T>(hdt), rg, jy);
    const T inv = vrcp(rho);
    const T ux = vmul(jx, inv), uy = vmul(jy, inv);
    const T u2 = vfma(ux, ux, vmul(uy, uy));
    T th = zero;
    if (!isothermal) {
        T e2 = vsub(vsub(en, vadd(drho, drho)), vmul(rho, u2));
        if (forced) e2 = vfma(vmul(vsplat<T>(hdt + hdt), rg), uy, e2);
        th = vmul(vmul(e2, vsplat<T>(R(0.5))), inv);
    }
    o.drho = drho;
    o.jx = jx;
    o.jy = jy;
    o.ux = ux;
    o.uy = uy;
    o.th = th;
    T pneq = pxy;
    if constexpr (N >= 2) {
        pneq = vsub(pxy, vmul(rho, vmul(ux, uy)));
        if (forced) pneq = vfma(vmul(vsplat<T>(hdt), rg), ux, pneq);
    }
    o.sig = vmul(vsplat<T>(sigma_fac), pneq);
    o.h = h;
    if constexpr (COLLIDE) {
        // Hermite coefficients of the Maxwellian, c_{k+1} = u c_k + k (T - 1) c_{k-1}
        T cx[N + 1], cy[N + 1];
        cx[0] = cy[0] = vsplat<T>(R(1));
        cx[1] = ux;
        cy[1] = uy;
#pragma unroll
        for (int k = 1; k < N; ++k) {
            const T kth = vmul(vsplat<T>(R(k)), th);
            cx[k + 1] = vfma(ux, cx[k], vmul(kth, cx[k - 1]));
            cy[k + 1] = vfma(uy, cy[k], vmul(kth, cy[k - 1]));
        }
        if (forced) {
            const T tg = vmul(vsplat<T>(tau), gf);
#pragma unroll
            for (int k = N; k >= 1; --k) cy[k] = vfma(vmul(vsplat<T>(R(k)), tg), cy[k - 1], cy[k]);
        }
        T QY[NA][N + 1];
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            QY[j][0] = vsplat<T>(t.wm[j]);
#pragma unroll
            for (int ky = 1; ky <= N; ++ky)
                QY[j][ky] = vmul(vsplat<T>(VS::kProductWeights ? t.whn[j][ky] : t.hn[j][ky]), cy[ky]);
            // FP32: the first-order factor's small second term (exact momentum identity)
            if constexpr (std::is_same<R, float>::value)
                QY[j][1] = vfma(vsplat<T>(VS::kProductWeights ? t.whn1lo[j] : t.hn1lo[j]), cy[1], QY[j][1]);
        }
        const T om1 = vsplat<T>(R(1) - omega);
        static_for<0, NA>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            // px[0] = sum_{kx>=1} cx hn (the kx = ky = 0 term is rho itself); px[ky>=1] = sum_{kx<=N-ky} cx hn
            T px[N + 1];
#pragma unroll
            for (int ky = 0; ky <= N; ++ky) {
                T sacc = ky == 0 ? zero : vsplat<T>(R(1));
#pragma unroll
                for (int kx = 1; kx <= N - ky; ++kx) sacc = vfma(cx[kx], vsplat<T>(t.hn[I][kx]), sacc);
                if constexpr (std::is_same<R, float>::value) {
                    if (ky == 0) sacc = vfma(cx[1], vsplat<T>(t.hn1lo[I]), sacc);
                }
                px[ky] = sacc;
            }
            if constexpr (VS::kProductWeights) {
                const T ow = vsplat<T>(t.ow[I]);
                T PX[N + 1];
                const T s0 = vfma(rho, px[0], drho);
                PX[0] = vmul(ow, s0);
                if constexpr (std::is_same<R, float>::value) PX[0] = vfma(vsplat<T>(t.owlo[I]), s0, PX[0]);
                const T owr = vmul(ow, rho);
#pragma unroll
                for (int ky = 1; ky <= N; ++ky) PX[ky] = vmul(owr, px[ky]);
                static_for<0, VS::Q>([&](auto ac) {
                    constexpr int a = decltype(ac)::value;
                    if constexpr (VS::ix(a) == I) {
                        constexpr int iy = VS::iy(a);
                        T od = vmul(PX[0], QY[iy][0]);
#pragma unroll
                        for (int ky = 1; ky <= N; ++ky) od = vfma(PX[ky], QY[iy][ky], od);
                        T& fa = f(ac);
                        fa = vfma(fa, om1, od);
                    }
                });
            } else {
                static_for<0, VS::Q>([&](auto ac) {
                    constexpr int a = decltype(ac)::value;
                    if constexpr (VS::ix(a) == I) {
                        constexpr int iy = VS::iy(a);
                        T sacc = px[0];
#pragma unroll
                        for (int ky = 1; ky <= N; ++ky) sacc = vfma(px[ky], QY[iy][ky], sacc);
                        T od = vmul(vsplat<T>(t.oww[a]), vfma(rho, sacc, drho));
                        if constexpr (std::is_same<R, float>::value && VS::kOnLattice) {
                            if constexpr (VS::ex(a) == 0 && VS::ey(a) == 0) od = vfma(vsplat<T>(t.mass_lo), drho, od);
                        }
                        T& fa = f(ac);
                        fa = vfma(fa, om1, od);
                    }
                });
            }
        });
    }
    return o;
}

// Amplitude A_f cos(phi n dt) of the body force at time level n (0 when unforced).
template <class R>
__device__ __forceinline__ R force_at_level(const Args<R>& A, long long lvl) {
    return A.force_amp != 0.0 ? (R)(A.force_amp * cos(A.force_freq * (double)lvl * A.dt)) : R(0);
}

// The same collision with one cell per lane and the velocities taken in pairs (a, a + 1)
// of equal x node (a = ix NA + iy, iy even), each pair one packed f32x2 value: the
// per-velocity work (moment sums, diagnostics, equilibrium, relaxation) runs at half the
// instruction count.  Product-weight Gauss-Hermite sets (NA even), FP32 arithmetic.
// Moments as in collide_cell, with the y-node sums kept as pairs and the x-node sums
// reduced when the x node changes; H = sum_ix (1/W_ix) sum_iy d^2 / W_iy.
template <class VS>
struct PairCollision {
    static constexpr bool value = VS::kProductWeights && !VS::kOnLattice && VS::NA % 2 == 0;
};

// ow, owlo, hn1lo, whn1lo: the relaxation tables of omega (Tab), the handle's own or, in a
// batch, the instance's.
template <class VS, int N, bool COLLIDE, class F>
__device__ __forceinline__ CellOut<float> collide_cell_pairs(const Tab<float>& t, const float* ow_t, const float* owlo_t,
                                                             const float* hn1lo_t, const float* whn1lo_t,
                                                             float rho0, float omega, float sigma_fac, int isothermal,
                                                             bool diag, bool forced, float gf, float tau, float hdt,
                                                             F&& fpair) {
    using R = float;
    constexpr int NA = VS::NA, NP = VS::Q / 2, NJ = NA / 2;
    const f2 z2 = f2{0.f, 0.f};
    f2 Ryp[NJ];
    R C[NA];
#pragma unroll
    for (int j = 0; j < NJ; ++j) Ryp[j] = z2;
    // x-node sums, one pair accumulator live at a time (the pairs come in x-node order)
    static_for<0, NA>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        f2 cp = z2;
        static_for<0, NJ>([&](auto jc) {
            constexpr int J = decltype(jc)::value;
            const f2 v = fpair(std::integral_constant<int, I * NJ + J>{});
            cp = vadd(cp, v);
            Ryp[J] = vadd(Ryp[J], v);
        });
        C[I] = cp.x + cp.y;
    });
    R drho = C[0], jx = t.a[0] * C[0];
    R en = t.a2[0] * C[0];
#pragma unroll
    for (int i = 1; i < NA; ++i) {
        drho += C[i];
        jx = fmaf(t.a[i], C[i], jx);
        en = fmaf(t.a2[i], C[i], en);
    }
    f2 jyp = z2, eyp = z2;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        jyp = vfma(f2{t.a[2 * j], t.a[2 * j + 1]}, Ryp[j], jyp);
        eyp = vfma(f2{t.a2[2 * j], t.a2[2 * j + 1]}, Ryp[j], eyp);
    }
    R jy = jyp.x + jyp.y;
    en += eyp.x + eyp.y;
    CellOut<R> o;
    R pxy = 0.f, h = 0.f;
    if (diag) {
        static_for<0, NA>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            f2 pp = z2, hp = z2;
            static_for<0, NJ>([&](auto jc) {
                constexpr int J = decltype(jc)::value;
                const f2 v = fpair(std::integral_constant<int, I * NJ + J>{});
                pp = vfma(f2{t.a[2 * J], t.a[2 * J + 1]}, v, pp);
                hp = vfma(vmul(v, f2{t.wminv[2 * J], t.wminv[2 * J + 1]}), v, hp);
            });
            pxy = fmaf(t.a[I], pp.x + pp.y, pxy);
            h = fmaf(t.wminv[I], hp.x + hp.y, h);
        });
    }
    const R rho = rho0 + drho;
    const R rg = forced ? __fmul_rn(rho, gf) : 0.f;
    if (forced) jy = fmaf(hdt, rg, jy);
    const R inv = 1.0f / rho;
    const R ux = __fmul_rn(jx, inv), uy = __fmul_rn(jy, inv);
    const R u2 = fmaf(ux, ux, __fmul_rn(uy, uy));
    R th = 0.f;
    if (!isothermal) {
        R e2 = __fsub_rn(__fsub_rn(en, __fadd_rn(drho, drho)), __fmul_rn(rho, u2));
        if (forced) e2 = fmaf(__fmul_rn(hdt + hdt, rg), uy, e2);
        th = __fmul_rn(__fmul_rn(e2, 0.5f), inv);
    }
    o.drho = drho;
    o.jx = jx;
    o.jy = jy;
    o.ux = ux;
    o.uy = uy;
    o.th = th;
    R pneq = pxy;
    if constexpr (N >= 2) {
        pneq = __fsub_rn(pxy, __fmul_rn(rho, __fmul_rn(ux, uy)));
        if (forced) pneq = fmaf(__fmul_rn(hdt, rg), ux, pneq);
    }
    o.sig = __fmul_rn(sigma_fac, pneq);
    o.h = h;
    if constexpr (COLLIDE) {
        R cx[N + 1], cy[N + 1];
        cx[0] = cy[0] = 1.f;
        cx[1] = ux;
        cy[1] = uy;
#pragma unroll
        for (int k = 1; k < N; ++k) {
            const R kth = __fmul_rn((R)k, th);
            cx[k + 1] = fmaf(ux, cx[k], __fmul_rn(kth, cx[k - 1]));
            cy[k + 1] = fmaf(uy, cy[k], __fmul_rn(kth, cy[k - 1]));
        }
        if (forced) {
            const R tg = __fmul_rn(tau, gf);
#pragma unroll
            for (int k = N; k >= 1; --k) cy[k] = fmaf(__fmul_rn((R)k, tg), cy[k - 1], cy[k]);
        }
        // y factors of the y-node pairs: QY[j][ky] = W_j He_ky(a_j)/ky! c_ky(u_y)
        f2 QYp[NJ][N + 1];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            QYp[j][0] = f2{t.wm[2 * j], t.wm[2 * j + 1]};
#pragma unroll
            for (int ky = 1; ky <= N; ++ky)
                QYp[j][ky] = vmul(f2{t.whn[2 * j][ky], t.whn[2 * j + 1][ky]}, vsplat<f2>(cy[ky]));
            // the first-order factor's small second term (exact momentum identity)
            QYp[j][1] = vfma(f2{whn1lo_t[2 * j], whn1lo_t[2 * j + 1]}, vsplat<f2>(cy[1]), QYp[j][1]);
        }
        const f2 om1 = vsplat<f2>(1.f - omega);
        static_for<0, NA>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            R PX[N + 1];
            {
                R px[N + 1];
#pragma unroll
                for (int ky = 0; ky <= N; ++ky) {
                    R sacc = ky == 0 ? 0.f : 1.f;
#pragma unroll
                    for (int kx = 1; kx <= N - ky; ++kx) sacc = fmaf(cx[kx], t.hn[I][kx], sacc);
                    if (ky == 0) sacc = fmaf(cx[1], hn1lo_t[I], sacc);
                    px[ky] = sacc;
                }
                const R ow = ow_t[I];
                const R s0 = fmaf(rho, px[0], drho);
                PX[0] = fmaf(owlo_t[I], s0, __fmul_rn(ow, s0));
                const R owr = __fmul_rn(ow, rho);
#pragma unroll
                for (int ky = 1; ky <= N; ++ky) PX[ky] = __fmul_rn(owr, px[ky]);
            }
            static_for<0, NJ>([&](auto jc) {
                constexpr int J = decltype(jc)::value;
                f2 od = vmul(vsplat<f2>(PX[0]), QYp[J][0]);
#pragma unroll
                for (int ky = 1; ky <= N; ++ky) od = vfma(vsplat<f2>(PX[ky]), QYp[J][ky], od);
                f2& fa = fpair(std::integral_constant<int, I * NJ + J>{});
                fa = vfma(fa, om1, od);
            });
        });
    }
    return o;
}

// Collision and store (or the moment outputs) of the V cells (g.x .., y) whose
// streamed populations are in ft.  Diagnostics are reduced over the warp in
// FP32 and added to acc (lane 0) in FP64.
// OSTRIDE > 0 (store-staged kernel, FP32): the relaxed populations go to the output tile in
// shared memory, out[a * OSTRIDE] for velocity a, instead of to HBM (the periodic images in
// the ghost rim are still written here, from that tile).
template <class VS, int N, class S, class R, int V, int KIND, class T, int OSTRIDE = 0>
__device__ __forceinline__ void collide_store(const Args<R>& A, T (&ft)[VS::Q], S* __restrict__ dst, int y,
                                              const Lane& g, bool diag, R (&acc)[6], int lane, long long lvl,
                                              R gt, S* out = nullptr) {
    constexpr int Q = VS::Q;
    static_assert(OSTRIDE == 0 || V == 1, "output tile: one cell per lane");
    // body force g_y(x_i, t_n) = gt sin(x_i), gt = A_f cos(phi t_n) (driven standing wave, Sec. 4);
    // compiled out of the unforced step kernels
    constexpr bool STEP = (KIND == kStep || KIND == kStepForced);
    const bool forced = (KIND != kStep) && A.force_amp != 0.0;
    // sin(x_i), cos(x_i) of the diagnostics, loaded before the collision so that their
    // latency hides behind it (index clamped: lanes that own no cell add nothing)
    constexpr bool PF =
        LB_DIAG_PREFETCH > 0 || (LB_DIAG_PREFETCH < 0 && ((!VS::kOnLattice && VS::Q == 16) || OSTRIDE > 0));
    R dsin[V], dcos[V];
    if constexpr (STEP && PF) {
        if (diag) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int xi = min(max(g.x + k, 0), A.nx - 1);
                dsin[k] = __ldg(A.sinx + xi);
                dcos[k] = __ldg(A.cosx + xi);
            }
        }
    }
    T gf = vsplat<T>(R(0));
    if (forced) {
        R gl[V];
#pragma unroll
        for (int k = 0; k < V; ++k) gl[k] = gt * A.sinx[min(max(g.x + k, 0), A.nx - 1)];
        if constexpr (V == 2) {
            gf = pack_lanes<T, R>(gl[0], gl[1]);
        } else {
            gf = gl[0];
        }
    }
    CellOut<T> co;
    if constexpr (V == 1 && std::is_same<R, float>::value && PairCollision<VS>::value &&
                  LB_PAIR_COLLISION) {
        // one cell per lane: velocity pairs as packed f32x2 values
        constexpr int NP = Q / 2;
        f2 fp[NP];
        static_for<0, NP>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            fp[m] = f2{ft[2 * m], ft[2 * m + 1]};
        });
        co = collide_cell_pairs<VS, N, STEP>(
            A.tab, A.tab.ow, A.tab.owlo, A.tab.hn1lo, A.tab.whn1lo, A.rho0, A.omega, A.sigma_fac, A.isothermal, diag || KIND == kMoments, forced, gf, A.tau,
            A.hdt, [&](auto mc) -> f2& { return fp[decltype(mc)::value]; });
        static_for<0, NP>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            ft[2 * m] = fp[m].x;
            ft[2 * m + 1] = fp[m].y;
        });
    } else {
        co = collide_cell<VS, N, R, T, STEP>(
            A.tab, A.rho0, A.omega, A.sigma_fac, A.isothermal, diag || KIND == kMoments, forced, gf, A.tau,
            A.hdt, [&](auto ac) -> T& { return ft[decltype(ac)::value]; });
    }
    if constexpr (KIND == kMoments) {
        if (g.own) {
            static_for<0, V>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                const long long c = (long long)y * A.nx + g.x + k;
                if (A.o_rho) A.o_rho[c] = (double)A.rho0 + (double)lane_get<k>(co.drho);
                if (A.o_ux) A.o_ux[c] = (double)lane_get<k>(co.ux);
                if (A.o_uy) A.o_uy[c] = (double)lane_get<k>(co.uy);
                if (A.o_T) A.o_T[c] = 1.0 + (double)lane_get<k>(co.th);
                if (A.o_sxy) A.o_sxy[c] = (double)lane_get<k>(co.sig);
                if (A.o_pop) {
                    const long long pl = (long long)A.ny * A.nx;
#pragma unroll
                    for (int a = 0; a < Q; ++a)
                        A.o_pop[a * pl + c] = (double)A.tab.w[a] * (double)A.rho0 + (double)lane_get<k>(ft[a]);
                }
            });
        }
    }
    if constexpr (STEP && OSTRIDE > 0) {
        if (g.own) {
            // the same stochastic rounding stream as the global stores below (same bits)
            uint32_t r0 = 0;
            if constexpr (Is16<S>::value) r0 = sr_seed(lvl, (long long)y * A.nx + g.x);
            static_for<0, Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                if constexpr (Is16<S>::value) {
                    r0 = sr_next(r0);
                    out[a * OSTRIDE] = to_storage<S, R>(lane_get<0>(ft[a]), store_scale<S, R>(A.tab, a), r0);
                } else {
                    out[a * OSTRIDE] = lane_get<0>(ft[a]);
                }
            });
            if (g.x < kGhostX || g.x + V > A.nx - kGhostX || y < A.gy || y >= A.ny - A.gy)
                rim_images_tile<S, R>(A, dst, out, OSTRIDE, Q, g.x, y);
        }
    }
    if constexpr (STEP && OSTRIDE == 0) {
        if (g.own) {
            S* base = dst + A.origin + (long long)y * A.pitch + g.x;
            uint32_t r0 = 0, r1 = 0;
            if constexpr (Is16<S>::value) {
                r0 = sr_seed(lvl, (long long)y * A.nx + g.x);
                r1 = sr_seed(lvl, (long long)y * A.nx + g.x + 1);
            }
            S* p = base;
            static_for<0, Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                const R si = store_scale<S, R>(A.tab, a);
                if constexpr (Is16<S>::value) {
                    r0 = sr_next(r0);
                    r1 = sr_next(r1);
                }
                if constexpr (Is16<S>::value && V == 2) {
                    const T hs = vmul(ft[a], vsplat<T>(si));
                    __stcs(reinterpret_cast<unsigned int*>(p),
                           to_storage16x2<S>(lane_get<0>(hs), lane_get<1>(hs), r0, r1));
                } else {
                    const S s0 = to_storage<S, R>(lane_get<0>(ft[a]), si, r0);
                    const S s1 = to_storage<S, R>(lane_get<V - 1>(ft[a]), si, r1);
                    if constexpr (V == 2) {
                        store_raw2<S>(p, s0, s1);
                    } else {
                        store_raw<S>(p, s0);
                    }
                }
                p += A.plane;
            });
            // periodic images in the ghost rim (boundary cells only): one out-of-line call
            // that copies the values just stored, so the velocity loop above stays branch-free
            if (g.x < kGhostX || g.x + V > A.nx - kGhostX || y < A.gy || y >= A.ny - A.gy)
                rim_images<S, R, V>(A, dst, Q, g.x, y);
        }
    }
    if constexpr (STEP) {
        // per-thread partial sums over the thread's cells of every tile; reduced once per
        // launch (warp, then FP64 across warps and blocks) in finish_step
        if (diag && g.own) {
            static_for<0, V>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                acc[0] += lane_get<k>(co.drho);
                acc[1] += lane_get<k>(co.jx);
                acc[2] += lane_get<k>(co.jy);
                if constexpr (!PF) {
                    dsin[k] = A.sinx[g.x + k];
                    dcos[k] = A.cosx[g.x + k];
                }
                acc[3] = fma(lane_get<k>(co.uy), dsin[k], acc[3]);
                acc[4] = fma(lane_get<k>(co.sig), dcos[k], acc[4]);
                acc[5] += lane_get<k>(co.h);
            });
        }
    }
}

// Diagnostics of a step launch: each thread sums its own cells in R for at most kDiagFold
// tiles, then the warp folds those partials (a shuffle sum of 32 values) into its FP64 sums
// in shared memory (wsum[warp], lane 0), so the grid sums are FP64 sums of short partials at
// any grid size (a thread's cells per launch grow with the grid: ~200 at 4096^2, ~3300 at
// 16384^2).  Cost of the folds, D2Q36-GH FP32 at 4096^2 (GLUPS): every 16 tiles 17.74,
// every 64 17.87, only at the end 17.94.
#ifndef LB_DIAG_FOLD
#define LB_DIAG_FOLD 64
#endif
constexpr int kDiagFold = LB_DIAG_FOLD;

template <class R>
__device__ __forceinline__ void fold_diag(R (&acc)[6], double* wsum, int lane) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const R sm = warp_sum(acc[i]);
        if (lane == 0) wsum[i] += (double)sm;
        acc[i] = R(0);
    }
}

// End of a step launch: the last fold, per-block FP64 partials, last-block fixed-order sum
// into the diagnostics ring, level advance.  All threads of the block call it; wsum holds
// the per-warp FP64 sums (zeroed by each warp's lane 0 before its first fold).
template <class R, int NWARPS_DIAG>
__device__ __forceinline__ void finish_step(const Args<R>& A, R (&acc)[6], double (*wsum)[6], long long lvl,
                                            bool diag, int warp, int lane) {
    __shared__ bool is_last;
    __shared__ double tot[6];
    if (diag && warp < NWARPS_DIAG) fold_diag(acc, wsum[warp], lane);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (diag) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                double s = 0.0;
                for (int w = 0; w < NWARPS_DIAG; ++w) s += wsum[w][i];
                A.partials[(long long)blockIdx.x * kDiagSlots + i] = s;
            }
        }
        __threadfence();
        const unsigned int t = atomicAdd(A.ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (diag) {
        if (warp < 6) {
            double s = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(A.partials + (long long)b * kDiagSlots + warp);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) tot[warp] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double ncell = (double)A.nx * (double)A.ny;
            const double norm = 2.0 / ncell;
            lb_diag r;
            r.t = (double)lvl * A.dt;
            r.mass = ncell * (double)A.rho0 + tot[0];
            r.mom_x = tot[1];
            r.mom_y = tot[2];
            r.amp = tot[3] * norm;
            r.shear = tot[4] * norm;
            r.hnorm = tot[5];
            const bool bad = !(isfinite(r.mass) && isfinite(r.amp) && isfinite(r.hnorm));
            r.flags = bad ? 1.0 : 0.0;
            if (bad) atomicOr(A.status, 1);
            const long long rec = lvl / A.diag_every;
            A.ring[rec % A.ring_cap] = r;
        }
    }
    if (threadIdx.x == 0) {
        *A.level = lvl + 1;
        *A.ticket = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------ register kernel
// KIND = kStep:    f* (next level) into dst, diagnostics when due.
// KIND = kStepForced: the same with the body force (lb_params.force_amp != 0).
// KIND = kMoments: per-cell rho, u, T, sigma_xy (and optionally f~) of the level; no store.
// UPW: off-lattice streaming by second-order upwind instead of Lax-Wendroff.
template <class VS, int N, class S, class R, int KIND, bool UPW = false>
__global__ void __launch_bounds__(Cfg<VS, S>::THREADS, Cfg<VS, S>::MINB)
    lb_fused_kernel(const __grid_constant__ Args<R> A) {
    constexpr int Q = VS::Q;
    constexpr int V = Cfg<VS, S>::V;
    constexpr int ROWS = Cfg<VS, S>::ROWS;
    constexpr int TW = 32 * V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S* __restrict__ src = static_cast<const S*>(A.src);
    S* __restrict__ dst = static_cast<S*>(A.dst);

    constexpr bool STEP = (KIND == kStep || KIND == kStepForced);
    long long lvl = 0;
    bool diag = false;
    if constexpr (STEP) {
        lvl = __ldcg(A.level);
        diag = (A.diag_every > 0) && (lvl % A.diag_every == 0);
    } else {
        // force phase of the state's level n: the device counter already points past it
        // (the launch that produced f*(n) advanced it to n + 1)
        if (A.force_amp != 0.0) lvl = __ldcg(A.level) - 1;
    }
    R gt = R(0);
    if constexpr (KIND != kStep) gt = force_at_level(A, lvl);
    R acc[6] = {0, 0, 0, 0, 0, 0};
    __shared__ double wsum[ROWS][6];
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) wsum[warp][i] = 0.0;
    }
    int nfold = 0;

    for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const int ty = tile / A.ntiles_x;
        const int tx = tile - ty * A.ntiles_x;
        const int y = ty * ROWS + warp;
        if (y >= A.ny) continue;  // warp-uniform
        const int tile_start = tx * TW;
        const int x0 = (tx == A.ntiles_x - 1) ? A.x0_last : tile_start;
        const Lane g = lane_geometry<V>(lane, x0, tile_start, A.nx);

        using T = typename Pack<R, V>::T;
        T ft[Q];
        static_for<0, Q>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            const R sc = load_scale<S, R>(A.tab, a);
            const S* pl = src + (long long)a * A.plane + A.origin;
            if (A.raw) {
                const S* p = pl + (long long)y * A.pitch + g.xl;
                if constexpr (V == 2) {
                    R v0, v1;
                    ld2<S, R>(p, sc, v0, v1);
                    ft[a] = pack_lanes<T, R>(v0, v1);
                } else {
                    ft[a] = ld1<S, R>(p, sc);
                }
            } else if constexpr (VS::kOnLattice) {
                // exact shift: f~_a(x, y) = f*_a(x - ex, y - ey)
                constexpr int ex = VS::ex(a), ey = VS::ey(a);
                const S* p = pl + (long long)(y - ey) * A.pitch + g.xl - ex;
                if constexpr (V == 2 && (ex % 2 == 0)) {
                    R v0, v1;
                    ld2<S, R>(p, sc, v0, v1);
                    ft[a] = pack_lanes<T, R>(v0, v1);
                } else if constexpr (V == 2) {
                    ft[a] = pack_lanes<T, R>(ld1<S, R>(p, sc), ld1<S, R>(p + 1, sc));
                } else {
                    ft[a] = ld1<S, R>(p, sc);
                }
            } else if constexpr (UPW) {
                // tensor-product second-order upwind (Beam-Warming), one cell per lane: y pass
                // over the cell's row and the two upstream rows, x pass by shuffles from the two
                // upstream lanes; the two lanes at the warp's downstream edge compute the two
                // upstream columns outside the warp
                static_assert(V == 1 && !Is16<S>::value, "upwind streaming: one cell per lane, 32/64-bit");
                constexpr int ix = VS::ix(a), iy = VS::iy(a);
                constexpr int sx = VS::axis_sign(ix), sy = VS::axis_sign(iy);
                const R yf = A.tab.uw[iy][0], yn = A.tab.uw[iy][1], ys = A.tab.uw[iy][2];
                const R xf = A.tab.uw[ix][0], xn = A.tab.uw[ix][1], xs = A.tab.uw[ix][2];
                const S* r0 = pl + (long long)y * A.pitch;
                const S* rn = r0 - (long long)sy * A.pitch;
                const S* rf = r0 - 2LL * sy * A.pitch;
                const R one = R(1);
                // lanes past the grid read the images of columns 0 and 1 (nx, nx + 1)
                const int xu = min(g.x, A.nx + 1);
                const R gv = fma(yf, ld1<S, R>(rf + xu, one), fma(yn, ld1<S, R>(rn + xu, one),
                                                                 ys * ld1<S, R>(r0 + xu, one)));
                // extra column: x0 - 2 + (lane & 1) (lanes 30, 31) for sx > 0,
                // x0 + 32 + (lane & 1) (lanes 0, 1) for sx < 0, clamped into the rim
                const int xe = sx > 0 ? x0 - 2 + (lane & 1) : min(x0 + 32 + (lane & 1), A.nx + 1);
                const R ge = fma(yf, ld1<S, R>(rf + xe, one), fma(yn, ld1<S, R>(rn + xe, one),
                                                                 ys * ld1<S, R>(r0 + xe, one)));
                R g1, g2;
                if constexpr (sx > 0) {
                    g1 = __shfl_up_sync(0xffffffffu, gv, 1);
                    g2 = __shfl_up_sync(0xffffffffu, gv, 2);
                    const R e2 = __shfl_sync(0xffffffffu, ge, 30);  // column x0 - 2
                    const R e1 = __shfl_sync(0xffffffffu, ge, 31);  // column x0 - 1
                    if (lane == 0) { g1 = e1; g2 = e2; }
                    if (lane == 1) g2 = e1;
                } else {
                    g1 = __shfl_down_sync(0xffffffffu, gv, 1);
                    g2 = __shfl_down_sync(0xffffffffu, gv, 2);
                    const R e1 = __shfl_sync(0xffffffffu, ge, 0);   // column x0 + 32
                    const R e2 = __shfl_sync(0xffffffffu, ge, 1);   // column x0 + 33
                    if (lane == 31) { g1 = e1; g2 = e2; }
                    if (lane == 30) g2 = e1;
                }
                ft[a] = fma(xf, g2, fma(xn, g1, xs * gv));
            } else {
                // tensor-product Lax-Wendroff: y pass in registers, x pass by shuffles;
                // the warp's two edge lanes take their outer neighbour from one extra column
                constexpr int ix = VS::ix(a), iy = VS::iy(a);
                const R ly0 = A.tab.lw[iy][0], ly1 = A.tab.lw[iy][1], ly2 = A.tab.lw[iy][2];
                const R lx0 = A.tab.lw[ix][0], lx1 = A.tab.lw[ix][1], lx2 = A.tab.lw[ix][2];
                const S* r0 = pl + (long long)y * A.pitch;
                const S* rm = r0 - A.pitch;
                const S* rp = r0 + A.pitch;
                // the stencil is linear: 16-bit values are scaled once, after it (as in the
                // TMA-staged kernel, so the two give the same bits)
                const R one = R(1);
                const int xe = (lane == 31) ? min(x0 + TW, A.nx) : x0 - 1;
                const R ge = fma(ly0, ld1<S, R>(rm + xe, one), fma(ly1, ld1<S, R>(r0 + xe, one), ly2 * ld1<S, R>(rp + xe, one)));
                if constexpr (V == 2) {
                    R a0v, a1v, b0v, b1v, c0v, c1v;
                    ld2<S, R>(r0 + g.xl, one, a0v, a1v);
                    ld2<S, R>(rm + g.xl, one, b0v, b1v);
                    ld2<S, R>(rp + g.xl, one, c0v, c1v);
                    const T gv = vfma(vsplat<T>(ly0), pack_lanes<T, R>(b0v, b1v),
                                      vfma(vsplat<T>(ly1), pack_lanes<T, R>(a0v, a1v),
                                           vmul(vsplat<T>(ly2), pack_lanes<T, R>(c0v, c1v))));
                    const R gv0 = lane_get<0>(gv), gv1 = lane_get<1>(gv);
                    R gl = __shfl_up_sync(0xffffffffu, gv1, 1);
                    R gr = __shfl_down_sync(0xffffffffu, gv0, 1);
                    gl = (lane == 0) ? ge : gl;
                    gr = (lane == 31) ? ge : gr;
                    ft[a] = pack_lanes<T, R>(fma(lx0, gl, fma(lx1, gv0, lx2 * gv1)),
                                             fma(lx0, gv0, fma(lx1, gv1, lx2 * gr)));
                } else {
                    const R f0 = ld1<S, R>(r0 + g.xl, one);
                    const R fm = ld1<S, R>(rm + g.xl, one);
                    const R fp = ld1<S, R>(rp + g.xl, one);
                    const R gv = fma(ly0, fm, fma(ly1, f0, ly2 * fp));
                    R gl = __shfl_up_sync(0xffffffffu, gv, 1);
                    R gr = __shfl_down_sync(0xffffffffu, gv, 1);
                    gl = (lane == 0) ? ge : gl;
                    gr = (lane == 31) ? ge : gr;
                    ft[a] = fma(lx0, gl, fma(lx1, gv, lx2 * gr));
                }
                if constexpr (Is16<S>::value) ft[a] = vmul(ft[a], vsplat<T>(sc));
            }
        });
        collide_store<VS, N, S, R, V, KIND>(A, ft, dst, y, g, diag, acc, lane, lvl, gt);
        if (STEP && diag && ++nfold == kDiagFold) {  // warp-uniform
            fold_diag(acc, wsum[warp], lane);
            nfold = 0;
        }
    }
    if constexpr (STEP) finish_step<R, ROWS>(A, acc, wsum, lvl, diag, warp, lane);
}

// ------------------------------------------------------------ TMA-staged step kernel
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// try_wait with a suspend-time hint (ns): the waiting thread is suspended in hardware
// until the phase completes or the hint runs out, instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// try_wait with the default (system-dependent) suspend window: the consumers' fast path
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity: gives up after ~2^31 cycles
// (about a second), flags LB_ERR_TIMEOUT in the status word and returns false.
static __device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, int* status) {
    const long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait_sleep(bar, parity)) return true;
        if ((i & 255u) == 255u && clock64() - t0 > (1LL << 31)) {
            atomicOr(status, 2);
            return false;
        }
    }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, status);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    if constexpr (LB_TMA_EVICT_LAST) {
        // the halo rows and columns of a box are read again by the neighbouring tiles:
        // ask L2 to keep the lines (evict-last) so those re-reads do not go to DRAM
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
            "[%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
            "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "l"(pol)
            : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
            "[%2];" ::"r"(smem_u32(dst)),
            "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
            : "memory");
    }
}

// Store-staged kernel, producer side: wait (bounded) until every consumer warp has written
// tile `ti` into the output tile, write it to the cells (x0.., y0..) of dst with one TMA
// tensor store (velocities, rows and columns of the tile; the tensor map clips it at nx and
// ny), wait until the store has read the output tile, and release it.  False on a timeout.
__device__ __forceinline__ bool store_tile(const Args<float>& A, const void* otile, uint64_t* tdone, uint64_t* ofree,
                                           int ti, int x0, int y0) {
    if (!mbar_wait(tdone, (uint32_t)ti & 1u, A.status)) return false;
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(&A.tmap_st)),
        "r"(smem_u32(otile)), "r"(x0), "r"(y0), "r"(0)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    mbar_arrive(ofree);
    return true;
}

// KIND = kStep: one level (store f*, diagnostics, level advance); kMoments: the per-cell
// moments (and optionally f~) of the current level, nothing stored, no level advance.
// WIDE (KIND = kStep only): the store-staged variant (see TmaCfg): consumer warp w owns half
// w % 2 of tile row w / 2; at the end of a tile each consumer warp writes its relaxed cells
// into the output tile, then arrives on the tile-done barrier; the producer, once it has
// issued the next tile's loads, waits for that barrier, writes the tile to HBM with one TMA
// tensor store, waits until the store has read the output tile and releases it (the
// output-free barrier) for the consumers' next tile.
template <class VS, int N, class S, bool UPW = false, int KIND = kStep, bool WIDE = false>
__global__ void __maxnreg__((TmaCfg<VS, S, UPW, WIDE>::MAXREG))
    lb_tma_step_kernel(const __grid_constant__ Args<float> A) {
    static_assert(KIND == kStep || KIND == kMoments, "TMA-staged kinds: step, moments");
    static_assert(!WIDE || KIND == kStep, "the store-staged kernel is a step kernel");
    using R = float;
    using C = TmaCfg<VS, S, UPW, WIDE>;
    constexpr int Q = VS::Q, V = C::V, ROWS = C::ROWS, CW = C::CW, TW = C::TW, AL = C::AL;
    constexpr int NS = C::NS, NG = C::NG, K = C::K, BW = C::BW, BOX = C::BOX, SLOT = C::SLOT;
    constexpr int STAGE_ELEMS = C::STAGE_BYTES / (int)sizeof(S);
    constexpr int OSTRIDE = WIDE ? ROWS * C::TWO : 0;  // output tile: elements per velocity
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations must be 128-byte aligned: align the base explicitly
    unsigned char* const smem_raw =
        smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    S* const stages = reinterpret_cast<S*>(smem_raw);
    S* const otile = reinterpret_cast<S*>(smem_raw + NS * C::STAGE_BYTES);
    uint64_t* const full = reinterpret_cast<uint64_t*>(smem_raw + NS * C::STAGE_BYTES + C::OUT_BYTES);
    uint64_t* const empty = full + NS;
    uint64_t* const tdone = empty + NS;  // store-staged: the consumers have filled the output tile
    uint64_t* const ofree = tdone + 1;   // store-staged: the output tile may be overwritten
    __shared__ int s_abort;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        if constexpr (WIDE) {
            mbar_init(tdone, CW);
            mbar_init(ofree, 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if constexpr (WIDE) mbar_arrive(ofree);  // phase 0: the output tile starts free
    }
    __syncthreads();

    const long long lvl = __ldcg(A.level);
    const bool diag = KIND == kStep && (A.diag_every > 0) && (lvl % A.diag_every == 0);
    R acc[6] = {0, 0, 0, 0, 0, 0};
    __shared__ double wsum[CW][6];
    if (lane == 0 && warp < CW) {
#pragma unroll
        for (int i = 0; i < 6; ++i) wsum[warp][i] = 0.0;
    }
    volatile int* abort_flag = &s_abort;

    if (warp == CW) {
        // ---------------- producer: one thread streams the boxes of every tile
        if (lane == 0) {
            uint32_t it = 0;
            int ti = 0, px0 = 0, py0 = 0;  // store-staged: tiles issued, coordinates of the last
            for (int tile = blockIdx.x; tile < A.ntiles && !*abort_flag; tile += gridDim.x) {
                int ty, tx;
                tma_tile_coords<C::BAND>(tile, A.ntiles_x, A.ntiles, ty, tx);
                // store-staged tiles are not shifted: the store clips the last one at nx
                const int x0 = (!WIDE && tx == A.ntiles_x - 1) ? A.x0_last : tx * C::TWO;
                const int y0 = ty * ROWS;
                for (int grp = 0; grp < NG; ++grp, ++it) {
                    const int s = (int)(it % NS);
                    if (it >= (uint32_t)NS && !mbar_wait(&empty[s], ((it / NS) + 1) & 1u, A.status)) {
                        *abort_flag = 1;
                        break;
                    }
                    // failure-detection test: block 0 withholds the first stage of its first tile,
                    // so its consumers' bounded waits run out (status bit 2, LB_ERR_TIMEOUT)
                    if (A.withhold_stage && blockIdx.x == 0 && tile == (int)blockIdx.x && grp == 0) continue;
                    const int a0 = grp * K;
                    const int na = (Q - a0) < K ? (Q - a0) : K;
                    S* dstage = stages + (long long)s * STAGE_ELEMS;
                    if constexpr (C::LW) {
                        mbar_arrive_expect_tx(&full[s], (uint32_t)(K * BOX * sizeof(S)));
                        const int xs = WIDE ? x0 - AL + kGhostX : ((x0 - C::GX + kGhostX) / AL) * AL;
                        tma_load_3d(dstage, &A.tmap, &full[s], xs, y0 - C::GX + A.gy, a0);
                    } else {
                        mbar_arrive_expect_tx(&full[s], (uint32_t)(na * BOX * sizeof(S)));
                        for (int j = 0; j < na; ++j) {
                            const int a = a0 + j;
                            const int xs = ((x0 - VS::ex(a) + kGhostX) / AL) * AL;
                            tma_load_3d(dstage + j * SLOT, &A.tmap, &full[s], xs, y0 - VS::ey(a) + A.gy, a);
                        }
                    }
                }
                if constexpr (WIDE) {
                    // the previous tile's output, once this tile's loads are on their way
                    if (ti > 0 && !*abort_flag && !store_tile(A, otile, tdone, ofree, ti - 1, px0, py0)) *abort_flag = 1;
                    px0 = x0;
                    py0 = y0;
                    ++ti;
                }
            }
            if constexpr (WIDE) {
                if (ti > 0 && !*abort_flag && !store_tile(A, otile, tdone, ofree, ti - 1, px0, py0)) *abort_flag = 1;
                // every store has written HBM before the block exits
                asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
            }
            // drain: no box may still be in flight when the block exits
            if (*abort_flag) {
                const uint32_t first = it > (uint32_t)NS ? it - NS : 0u;
                for (uint32_t k = first; k < it; ++k) mbar_wait(&full[k % NS], (k / NS) & 1u, A.status);
            }
        }
    } else {
        // ---------------- consumers: warp w owns row y0 + w of every tile
        // stage index and parity advance with the stream of groups (NG per tile)
        int st_i = 0;
        uint32_t st_ph = 0;
        // store-staged: the warp's row of the tile and its half of the row
        const int trow = WIDE ? warp / C::WPR : warp;
        const int half = WIDE ? warp % C::WPR : 0;
        uint32_t ti = 0;  // tiles processed (store-staged: phase of the output-free barrier)
        for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++ti) {
            int ty, tx;
            tma_tile_coords<C::BAND>(tile, A.ntiles_x, A.ntiles, ty, tx);
            const int tile_start = tx * C::TWO + half * C::WCELLS;
            const int x0 = (!WIDE && tx == A.ntiles_x - 1) ? A.x0_last : tile_start;
            const int y = ty * ROWS + trow;
            const Lane g = UPW      ? upwind_lane_geometry(lane, x0, tile_start, A.nx)
                           : C::HALO ? halo_lane_geometry(lane, x0, tile_start, A.nx, C::WCELLS)
                                     : lane_geometry<V>(lane, x0, tile_start, A.nx);
            using T = typename Pack<R, V>::T;
            T ft[Q];
            bool ok = !*abort_flag;
            // Lax-Wendroff: column of this lane's first cell in the box row, and the column
            // whose y-pass the two warp-edge lanes need (x0 - 1 for lane 0, x0 + TW for lane 31)
            // (store-staged: the box starts AL columns left of the tile row)
            const int r_lw = WIDE ? AL - 1 + half * C::WCELLS : (x0 - 1 + kGhostX) & (AL - 1);
            const int c_lw = C::HALO ? r_lw + lane : r_lw + 1 + lane * V;
            const int ce_lw = (lane == 31) ? r_lw + 1 + TW : r_lw;
            static_for<0, NG>([&](auto gc) {
                constexpr int grp = decltype(gc)::value;
                if (ok) {
                    ok = mbar_wait(&full[st_i], st_ph, A.status);
                    if (!ok) *abort_flag = 1;
                }
                if (ok) {
                    const S* st = stages + (long long)st_i * STAGE_ELEMS;
                    static_for<0, K>([&](auto jc) {
                        constexpr int j = decltype(jc)::value;
                        constexpr int a = grp * K + j;
                        if constexpr (a < Q) {
                            const R sc = load_scale<S, R>(A.tab, a);
                            const S* box = st + j * SLOT;
                            if constexpr (UPW) {
                                // second-order upwind: y pass over the lane's column in the cell's
                                // row and its two upstream rows (box row of row y: warp + 2), x pass
                                // from the two upstream lanes (the same operation order as the
                                // plain-load kernel, so the two give the same bits)
                                const R one = R(1);
                                constexpr int ix = VS::ix(a), iy = VS::iy(a);
                                constexpr int sx = VS::axis_sign(ix), sy = VS::axis_sign(iy);
                                const R yf = A.tab.uw[iy][0], yn = A.tab.uw[iy][1], ys = A.tab.uw[iy][2];
                                const R xf = A.tab.uw[ix][0], xn = A.tab.uw[ix][1], xs = A.tab.uw[ix][2];
                                const int c = ((x0 - 2 + kGhostX) & (AL - 1)) + lane;
                                const S* r0 = box + (trow + 2) * BW;
                                const S* rn = r0 - sy * BW;
                                const S* rf = r0 - 2 * sy * BW;
                                const R gv = fma(yf, sld1<S, R>(rf + c, one),
                                                 fma(yn, sld1<S, R>(rn + c, one), ys * sld1<S, R>(r0 + c, one)));
                                R g1, g2;
                                if constexpr (sx > 0) {
                                    g1 = __shfl_up_sync(0xffffffffu, gv, 1);
                                    g2 = __shfl_up_sync(0xffffffffu, gv, 2);
                                } else {
                                    g1 = __shfl_down_sync(0xffffffffu, gv, 1);
                                    g2 = __shfl_down_sync(0xffffffffu, gv, 2);
                                }
                                ft[a] = fma(xf, g2, fma(xn, g1, xs * gv));
                            } else if constexpr (C::LW) {
                                // the stencil is linear: 16-bit values are scaled once, after it
                                const R one = R(1);
                                constexpr int ix = VS::ix(a), iy = VS::iy(a);
                                const R ly0 = A.tab.lw[iy][0], ly1 = A.tab.lw[iy][1], ly2 = A.tab.lw[iy][2];
                                const R lx0 = A.tab.lw[ix][0], lx1 = A.tab.lw[ix][1], lx2 = A.tab.lw[ix][2];
                                const S* rm = box + trow * BW;
                                const S* r0 = rm + BW;
                                const S* rp = r0 + BW;
                                if constexpr (C::HALO) {
                                    // y pass of the lane's column; x pass from the neighbours
                                    const R f0 = sld1<S, R>(r0 + c_lw, one);
                                    const R fm = sld1<S, R>(rm + c_lw, one);
                                    const R fp = sld1<S, R>(rp + c_lw, one);
                                    const R gv = fma(ly0, fm, fma(ly1, f0, ly2 * fp));
                                    const R gl = __shfl_up_sync(0xffffffffu, gv, 1);
                                    const R gr = __shfl_down_sync(0xffffffffu, gv, 1);
                                    ft[a] = fma(lx0, gl, fma(lx1, gv, lx2 * gr));
                                } else if constexpr (V == 2) {
                                    const R ge = fma(ly0, sld1<S, R>(rm + ce_lw, one),
                                                     fma(ly1, sld1<S, R>(r0 + ce_lw, one),
                                                         ly2 * sld1<S, R>(rp + ce_lw, one)));
                                    // y pass on the lane's two cells as one packed pair
                                    R a0v, a1v, b0v, b1v, c0v, c1v;
                                    sld2<S, R>(r0 + c_lw, one, a0v, a1v);
                                    sld2<S, R>(rm + c_lw, one, b0v, b1v);
                                    sld2<S, R>(rp + c_lw, one, c0v, c1v);
                                    const T gv = vfma(vsplat<T>(ly0), pack_lanes<T, R>(b0v, b1v),
                                                      vfma(vsplat<T>(ly1), pack_lanes<T, R>(a0v, a1v),
                                                           vmul(vsplat<T>(ly2), pack_lanes<T, R>(c0v, c1v))));
                                    const R gv0 = lane_get<0>(gv), gv1 = lane_get<1>(gv);
                                    R gl = __shfl_up_sync(0xffffffffu, gv1, 1);
                                    R gr = __shfl_down_sync(0xffffffffu, gv0, 1);
                                    gl = (lane == 0) ? ge : gl;
                                    gr = (lane == 31) ? ge : gr;
                                    ft[a] = pack_lanes<T, R>(fma(lx0, gl, fma(lx1, gv0, lx2 * gv1)),
                                                             fma(lx0, gv0, fma(lx1, gv1, lx2 * gr)));
                                } else {
                                    // one cell per lane, all 32 lanes own cells: the edge lanes
                                    // take their outer column's y pass from an extra read
                                    const R ge = fma(ly0, sld1<S, R>(rm + ce_lw, one),
                                                     fma(ly1, sld1<S, R>(r0 + ce_lw, one),
                                                         ly2 * sld1<S, R>(rp + ce_lw, one)));
                                    const R f0 = sld1<S, R>(r0 + c_lw, one);
                                    const R fm = sld1<S, R>(rm + c_lw, one);
                                    const R fp = sld1<S, R>(rp + c_lw, one);
                                    const R gv = fma(ly0, fm, fma(ly1, f0, ly2 * fp));
                                    R gl = __shfl_up_sync(0xffffffffu, gv, 1);
                                    R gr = __shfl_down_sync(0xffffffffu, gv, 1);
                                    gl = (lane == 0) ? ge : gl;
                                    gr = (lane == 31) ? ge : gr;
                                    ft[a] = fma(lx0, gl, fma(lx1, gv, lx2 * gr));
                                }
                                if constexpr (Is16<S>::value) ft[a] = vmul(ft[a], vsplat<T>(sc));
                            } else {
                                constexpr int ex = VS::ex(a);
                                const int r = (x0 - ex + kGhostX) & (AL - 1);
                                const S* p = box + trow * BW + r + lane * V;
                                if constexpr (V == 2 && (ex % 2 == 0)) {
                                    R v0, v1;
                                    sld2<S, R>(p, sc, v0, v1);
                                    ft[a] = pack_lanes<T, R>(v0, v1);
                                } else if constexpr (V == 2) {
                                    ft[a] = pack_lanes<T, R>(sld1<S, R>(p, sc), sld1<S, R>(p + 1, sc));
                                } else {
                                    ft[a] = sld1<S, R>(p, sc);
                                }
                            }
                        }
                    });
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[st_i]);
                }
                if (++st_i == NS) {
                    st_i = 0;
                    st_ph ^= 1u;
                }
            });
            if constexpr (WIDE) {
                // the output tile is free once the producer's store of the previous tile has read it
                if (ok) {
                    ok = mbar_wait(ofree, ti & 1u, A.status);
                    if (!ok) *abort_flag = 1;
                }
                if (ok && y < A.ny)
                    collide_store<VS, N, S, R, V, KIND, typename Pack<R, V>::T, OSTRIDE>(
                        A, ft, static_cast<S*>(A.dst), y, g, diag, acc, lane, lvl, R(0),
                        otile + trow * C::TWO + (g.x - tx * C::TWO));
                // the generic-proxy writes of the tile become visible to the TMA store; a warp
                // whose wait ran out does not arrive, so the producer's bounded wait runs out
                // too and no store of the tile is issued
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (ok && lane == 0) mbar_arrive(tdone);
            } else {
                if (ok && y < A.ny)
                    collide_store<VS, N, S, R, V, KIND>(A, ft, static_cast<S*>(A.dst), y, g, diag, acc, lane, lvl,
                                                        R(0));
            }
            if (diag && (ti % kDiagFold) == kDiagFold - 1) fold_diag(acc, wsum[warp], lane);  // warp-uniform
            if constexpr (C::TILE_SYNC) {
                // keep the consumer warps within one tile of each other, so a stage is
                // released (and refilled) as soon as the last of them has read it; every
                // consumer warp reaches this barrier once per tile (its waits are bounded)
                asm volatile("bar.sync 1, %0;" ::"r"(CW * 32) : "memory");
                if (*abort_flag) ok = false;
            }
            if (!ok) break;
        }
    }
    __syncthreads();
    if constexpr (KIND == kStep) finish_step<R, CW>(A, acc, wsum, lvl, diag, warp, lane);
}

// ------------------------------------------------------------ init kernel
// f~(0) = f^eq(rho, u, T) per cell (raw layout, no streaming), written to dst with its images.
template <class VS, int N, class S, class R>
__global__ void __launch_bounds__(256) lb_init_kernel(const __grid_constant__ Args<R> A) {
    S* __restrict__ dst = static_cast<S*>(A.dst);
    const long long ncell = (long long)A.nx * A.ny;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / A.nx), x = (int)(c - (long long)y * A.nx);
        double rho = 1.0, ux = 0.0, uy, T = 1.0;
        if (A.i_uy) {
            rho = A.i_rho ? A.i_rho[c] : 1.0;
            ux = A.i_ux ? A.i_ux[c] : 0.0;
            uy = A.i_uy[c];
            T = A.i_T ? A.i_T[c] : 1.0;
        } else {
            const double sx = sinpi(2.0 * (double)x / (double)A.nx);
            const double sy = sinpi(2.0 * (double)y / (double)A.ny);
            uy = A.u0 * sx + A.u1 * sy * sx;
        }
        const R drho = (R)(rho - (double)A.rho0);
        const R th = A.isothermal ? R(0) : (R)(T - 1.0);
        equilibrium_dev<VS, N, R>(A.tab, drho, (R)rho, (R)ux, (R)uy, th, [&](auto ac, R deq) {
            constexpr int a = decltype(ac)::value;
            const R v[1] = {deq};
            store_cells<S, R, 1>(A, dst + (long long)a * A.plane + A.origin, x, y, v, store_scale<S, R>(A.tab, a));
        });
    }
}

// ------------------------------------------------------------ dispatch
template <class VS, int N, class S, class R>
cudaError_t launch_typed(const Launch& L) {
    using C = Cfg<VS, S>;
    using T = TmaCfg<VS, S>;
    constexpr bool kTma = std::is_same<R, float>::value && T::NS >= 2;
    // second-order upwind streaming: Lax-Wendroff sets with 32/64-bit storage; TMA-staged
    // for FP32 storage
    constexpr bool kUpw = !VS::kOnLattice && !Is16<S>::value;
    constexpr bool kUpwTma = kUpw && kTma && std::is_same<S, float>::value;
    // store-staged TMA kernel: Lax-Wendroff sets, FP32 up to 36 velocities (the FP32 output
    // tile of a 64-velocity set leaves too little shared memory for the ring), 16-bit all
    constexpr bool kStore = kTma && !VS::kOnLattice && ((std::is_same<S, float>::value && VS::Q <= 40) || Is16<S>::value);
    if (L.kind == kQueryShape) {
        Shape* sh = static_cast<Shape*>(const_cast<void*>(L.args));
        sh->V = C::V;
        sh->rows = C::ROWS;
        sh->threads = C::THREADS;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &sh->occupancy, lb_fused_kernel<VS, N, S, R, kStep>, C::THREADS, 0);
        if (e != cudaSuccess) return e;
        sh->tma = 0;
        // the TMA-staged kernel of the requested streaming, and its box
        auto tma_shape = [&](auto kernel, auto cfg) -> cudaError_t {
            using TC = decltype(cfg);
            cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 TC::SMEM);  // fixed per kernel: every handle asks the same
            if (r != cudaSuccess) return r;
            r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh->tma_occupancy, kernel, TC::THREADS, TC::SMEM);
            if (r != cudaSuccess) return r;
            sh->tma = sh->tma_occupancy > 0 ? 1 : 0;
            sh->tma_V = TC::V;
            sh->tma_tw = TC::TWO;
            sh->tma_rows = TC::ROWS;
            sh->tma_threads = TC::THREADS;
            sh->tma_smem = TC::SMEM;
            sh->box_w = TC::BW;
            sh->box_h = TC::BH;
            sh->box_d = TC::BOX_D;
            return cudaSuccess;
        };
        if (L.upwind) {
            if constexpr (kUpwTma) {
                e = tma_shape(lb_tma_step_kernel<VS, N, S, true>, TmaCfg<VS, S, true>{});
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(lb_tma_step_kernel<VS, N, S, true, kMoments>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, TmaCfg<VS, S, true>::SMEM);
            }
        } else {
            if constexpr (kTma) {
                e = tma_shape(lb_tma_step_kernel<VS, N, S>, T{});
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(lb_tma_step_kernel<VS, N, S, false, kMoments>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
            }
            sh->st = 0;
            if constexpr (kStore) {
                using TS = TmaCfg<VS, S, false, true>;
                auto kernel = lb_tma_step_kernel<VS, N, S, false, kStep, true>;
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TS::SMEM);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh->st_occupancy, kernel, TS::THREADS, TS::SMEM);
                if (e == cudaSuccess) {
                    sh->st = sh->st_occupancy > 0 ? 1 : 0;
                    sh->st_tw = TS::TWO;
                    sh->st_rows = TS::ROWS;
                    sh->st_threads = TS::THREADS;
                    sh->st_smem = TS::SMEM;
                    sh->st_box_w = TS::BW;
                    sh->st_box_h = TS::BH;
                    // measured at 4096^2 (GLUPS, TMA-staged / store-staged): D2Q36-GH N = 3 13.8 /
                    // 16.2, N = 2 11.4 / 16.9, N = 1 9.8 / 18.1; D2Q16-GH N = 2 38.2 / 31.5
                    sh->st_auto = (sizeof(S) == 4 && VS::Q > 16) ? 1 : 0;
                }
            }
        }
        return e;
    }
    const Args<R>& A = *static_cast<const Args<R>*>(L.args);
    if (L.upwind && (L.kind == kStepTma || L.kind == kMomentsTma)) {
        if constexpr (kUpwTma) {
            using TU = TmaCfg<VS, S, true>;
            if (L.kind == kStepTma)
                lb_tma_step_kernel<VS, N, S, true><<<L.grid, TU::THREADS, TU::SMEM, L.stream>>>(A);
            else
                lb_tma_step_kernel<VS, N, S, true, kMoments><<<L.grid, TU::THREADS, TU::SMEM, L.stream>>>(A);
            return cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    if (L.upwind) {
        if constexpr (kUpw) {
            switch (L.kind) {
                case kStep:
                    lb_fused_kernel<VS, N, S, R, kStep, true><<<L.grid, C::THREADS, 0, L.stream>>>(A);
                    return cudaGetLastError();
                case kStepForced:
                    lb_fused_kernel<VS, N, S, R, kStepForced, true><<<L.grid, C::THREADS, 0, L.stream>>>(A);
                    return cudaGetLastError();
                case kMoments:
                    lb_fused_kernel<VS, N, S, R, kMoments, true><<<L.grid, C::THREADS, 0, L.stream>>>(A);
                    return cudaGetLastError();
                case kInit:
                    break;  // no streaming
                default:
                    return cudaErrorNotSupported;
            }
        } else {
            return cudaErrorNotSupported;
        }
    }
    switch (L.kind) {
        case kStep:
            lb_fused_kernel<VS, N, S, R, kStep><<<L.grid, C::THREADS, 0, L.stream>>>(A);
            break;
        case kStepForced:
            lb_fused_kernel<VS, N, S, R, kStepForced><<<L.grid, C::THREADS, 0, L.stream>>>(A);
            break;
        case kMoments:
            lb_fused_kernel<VS, N, S, R, kMoments><<<L.grid, C::THREADS, 0, L.stream>>>(A);
            break;
        case kInit:
            lb_init_kernel<VS, N, S, R><<<L.grid, 256, 0, L.stream>>>(A);
            break;
        case kStepTma:
            if constexpr (kTma) {
                lb_tma_step_kernel<VS, N, S><<<L.grid, T::THREADS, T::SMEM, L.stream>>>(A);
                break;
            }
            return cudaErrorNotSupported;
        case kMomentsTma:
            if constexpr (kTma) {
                lb_tma_step_kernel<VS, N, S, false, kMoments><<<L.grid, T::THREADS, T::SMEM, L.stream>>>(A);
                break;
            }
            return cudaErrorNotSupported;
        case kStepTmaStore:
            if constexpr (kStore) {
                using TS = TmaCfg<VS, S, false, true>;
                lb_tma_step_kernel<VS, N, S, false, kStep, true><<<L.grid, TS::THREADS, TS::SMEM, L.stream>>>(A);
                break;
            }
            return cudaErrorNotSupported;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Entry point of one (velocity set, storage) translation unit.
template <class VS, class S, class R>
cudaError_t launch_order(const Launch& L) {
    switch (L.n_eq) {
        case 1: return launch_typed<VS, 1, S, R>(L);
        case 2: return launch_typed<VS, 2, S, R>(L);
        case 3: return launch_typed<VS, 3, S, R>(L);
        case 4: return launch_typed<VS, 4, S, R>(L);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbk
