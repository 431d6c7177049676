// Fused collide-stream kernels for sm_103a (templates; instantiated per
// velocity set in k_<set>.cu).
//
// One launch advances every cell by one time level of Eq. 2order:
//   pull-stream   f~_a(x) = S_a[f*_a](x)        exact shift by e_a (on-lattice) or
//                                               tensor-product Lax-Wendroff (off-lattice)
//   moments       rho, rho u, 2 rho T (Sec. 2.2, D = 2)
//   equilibrium   f^eq_a = w_a rho sum_{kx+ky<=N} c_kx(u_x) c_ky(u_y) He_kx He_ky / (kx! ky!)
//                 (Sec. 2.1: the Hermite coefficients of the Maxwellian factorise per
//                 axis, c_k(u, T) = E[He_k(X)], X ~ Normal(u, T), from the recurrence
//                 c_{k+1} = u c_k + k (T - 1) c_{k-1})
//   relax         f*_a = f~_a + omega (f^eq_a - f~_a), omega = dt / (tau + dt/2)
//   store         f*_a (the next launch streams it)
//   diagnostics   FP64 grid sums of the observables of f~ (mass, momentum, the
//                 sin/cos Fourier amplitudes of u_y and sigma_xy, H norm)
// The stored variable is the deviation d = f - w rho0 (16-bit: d / (w S)), so
// moments and equilibrium are formed without the O(1) background and keep
// FP32 precision relative to the O(U0) signal.
//
// Work decomposition: a tile is kRows lattice rows x 32 V columns; warp w of a
// block owns row y0 + w and each lane V consecutive cells, so every
// population-plane access of a warp is one contiguous row segment (coalesced,
// vectorised when V = 2).  The grid is persistent (a multiple of the SM count)
// and walks tiles row-major, so the halo rows a tile re-reads were fetched
// moments earlier by its neighbours and sit in L2.
#pragma once

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
        *reinterpret_cast<float2*>(p) = make_float2(v0, v1);
    } else if constexpr (std::is_same<S, double>::value) {
        *reinterpret_cast<double2*>(p) = make_double2(v0, v1);
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v0 * scinv, v1 * scinv);
    } else {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v0 * scinv, v1 * scinv);
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

__device__ __forceinline__ int wrap_mod(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// compile-time loop: f(integral_constant<int, a>) for a in [A_, Q)
template <int A_, int Q, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (A_ < Q) {
        f(std::integral_constant<int, A_>{});
        static_for<A_ + 1, Q>(f);
    }
}

// ------------------------------------------------------------ equilibrium
// Deviation of the truncated Hermite equilibrium from w rho0, for one cell:
// deq_a = w_a (drho + rho * sum'_{kx+ky<=N} c_kx(ux) c_ky(uy) hn[ix][kx] hn[iy][ky]),
// sum' without the (0,0) term (which is rho itself).  emit(a, deq_a) is called for
// every velocity with a compile-time a after unrolling.
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
    // px[i][0] excludes kx = 0; px[i][ky>=1] = sum_{kx <= N-ky} cx[kx] hn[i][kx]
    R px[NA][N + 1];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
#pragma unroll
        for (int ky = 0; ky <= N; ++ky) {
            R s = (ky == 0) ? R(0) : R(1);
#pragma unroll
            for (int kx = 1; kx <= N - ky; ++kx) s = fma(cx[kx], t.hn[i][kx], s);
            px[i][ky] = s;
        }
    }
    R qy[NA][N + 1];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        qy[j][0] = R(0);
#pragma unroll
        for (int ky = 1; ky <= N; ++ky) qy[j][ky] = cy[ky] * t.hn[j][ky];
    }
    static_for<0, VS::Q>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        constexpr int ix = VS::ix(a), iy = VS::iy(a);
        R s = px[ix][0];
#pragma unroll
        for (int ky = 1; ky <= N; ++ky) s = fma(px[ix][ky], qy[iy][ky], s);
        emit(ac, t.w[a] * fma(rho, s, drho));
    });
}

// ------------------------------------------------------------ streaming
// Pull-stream population a into v[0..V) for the cells (xl .. xl+V-1, y) of this lane.
template <class VS, class S, class R, int V>
struct Streamer {
    static constexpr int TW = 32 * V;

    // exact shift: f~_a(x, y) = f*_a(x - ex, y - ey)
    template <int A_>
    __device__ __forceinline__ static void shift(const Args<R>& A, const S* __restrict__ src, int y,
                                                 bool interior, int xl, R (&v)[V]) {
        constexpr int ex = VS::ex(A_), ey = VS::ey(A_);
        const R sc = load_scale<S, R>(A.tab, A_);
        int ys = y - ey;
        if (A.ny >= VS::kHalo) {
            ys = ys < 0 ? ys + A.ny : (ys >= A.ny ? ys - A.ny : ys);
        } else {
            ys = wrap_mod(ys, A.ny);
        }
        const S* row = src + (long long)A_ * A.plane + (long long)ys * A.pitch;
        if (interior) {
            const int xs = xl - ex;
            if constexpr (V == 2 && (ex % 2 == 0)) {
                ld2<S, R>(row + xs, sc, v[0], v[V - 1]);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) v[k] = ld1<S, R>(row + xs + k, sc);
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = ld1<S, R>(row + wrap_mod(xl + k - ex, A.nx), sc);
        }
    }

    // tensor-product Lax-Wendroff: y pass in registers, x pass through warp shuffles
    template <int A_>
    __device__ __forceinline__ static void laxw(const Args<R>& A, const S* __restrict__ src, int y,
                                                int ym, int yp, int lane, int xl, R (&v)[V]) {
        constexpr int ix = VS::ix(A_), iy = VS::iy(A_);
        const R sc = load_scale<S, R>(A.tab, A_);
        const R ly0 = A.tab.lw[iy][0], ly1 = A.tab.lw[iy][1], ly2 = A.tab.lw[iy][2];
        const R lx0 = A.tab.lw[ix][0], lx1 = A.tab.lw[ix][1], lx2 = A.tab.lw[ix][2];
        const S* base = src + (long long)A_ * A.plane;
        const S* r0 = base + (long long)y * A.pitch;
        const S* rm = base + (long long)ym * A.pitch;
        const S* rp = base + (long long)yp * A.pitch;
        const bool yflat = (A.ny == 1);
        R g[V];
        {
            R f0[V], fm[V], fp[V];
            if constexpr (V == 2) {
                ld2<S, R>(r0 + xl, sc, f0[0], f0[1]);
            } else {
                f0[0] = ld1<S, R>(r0 + xl, sc);
            }
            if (yflat) {
#pragma unroll
                for (int k = 0; k < V; ++k) g[k] = f0[k];
            } else {
                if constexpr (V == 2) {
                    ld2<S, R>(rm + xl, sc, fm[0], fm[1]);
                    ld2<S, R>(rp + xl, sc, fp[0], fp[1]);
                } else {
                    fm[0] = ld1<S, R>(rm + xl, sc);
                    fp[0] = ld1<S, R>(rp + xl, sc);
                }
#pragma unroll
                for (int k = 0; k < V; ++k) g[k] = fma(ly0, fm[k], fma(ly1, f0[k], ly2 * fp[k]));
            }
        }
        // neighbours of the lane's cells along x
        R gl = __shfl_up_sync(0xffffffffu, g[V - 1], 1);
        R gr = __shfl_down_sync(0xffffffffu, g[0], 1);
        const bool needL = (lane == 0);
        const bool needR = (lane == 31) || (xl + V >= A.nx);
        if (needL || needR) {
            auto column = [&](int xc) -> R {
                const R c0 = ld1<S, R>(r0 + xc, sc);
                if (yflat) return c0;
                return fma(ly0, ld1<S, R>(rm + xc, sc), fma(ly1, c0, ly2 * ld1<S, R>(rp + xc, sc)));
            };
            if (needL) gl = column(wrap_mod(xl - 1, A.nx));
            if (needR) gr = column(wrap_mod(xl + V, A.nx));
        }
        if constexpr (V == 2) {
            v[0] = fma(lx0, gl, fma(lx1, g[0], lx2 * g[1]));
            v[1] = fma(lx0, g[0], fma(lx1, g[1], lx2 * gr));
        } else {
            v[0] = fma(lx0, gl, fma(lx1, g[0], lx2 * gr));
        }
    }
};

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ fused kernel
// KIND = kStep:    f* (next level) into dst, diagnostics when due.
// KIND = kMoments: per-cell rho, u, T, sigma_xy (and optionally f~) of the level; no store.
template <class VS, int N, class S, class R, int V, int KIND>
__global__ void __launch_bounds__(kThreads) lb_fused_kernel(const __grid_constant__ Args<R> A) {
    constexpr int Q = VS::Q;
    constexpr int TW = 32 * V;
    using St = Streamer<VS, S, R, V>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S* __restrict__ src = static_cast<const S*>(A.src);
    S* __restrict__ dst = static_cast<S*>(A.dst);

    long long lvl = 0;
    bool diag = false;
    if constexpr (KIND == kStep) {
        lvl = __ldcg(A.level);
        diag = (A.diag_every > 0) && (lvl % A.diag_every == 0);
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const R omega = A.omega;

    for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const int ty = tile / A.ntiles_x;
        const int tx = tile - ty * A.ntiles_x;
        const int y = ty * kRows + warp;
        if (y >= A.ny) continue;  // warp-uniform
        const int x0 = tx * TW;
        const int x = x0 + lane * V;
        const bool active = x < A.nx;
        const int xl = active ? x : 0;

        R ft[Q][V];
        if (A.raw) {
            static_for<0, Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                const R sc = load_scale<S, R>(A.tab, a);
                const S* p = src + (long long)a * A.plane + (long long)y * A.pitch + xl;
                if constexpr (V == 2) {
                    ld2<S, R>(p, sc, ft[a][0], ft[a][1]);
                } else {
                    ft[a][0] = ld1<S, R>(p, sc);
                }
            });
        } else if constexpr (VS::kOnLattice) {
            const bool interior = (x0 - VS::kHalo >= 0) && (x0 + TW + VS::kHalo <= A.nx);
            static_for<0, Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                St::template shift<a>(A, src, y, interior, xl, ft[a]);
            });
        } else {
            const int ym = (y == 0) ? A.ny - 1 : y - 1;
            const int yp = (y + 1 == A.ny) ? 0 : y + 1;
            static_for<0, Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                St::template laxw<a>(A, src, y, ym, yp, lane, xl, ft[a]);
            });
        }

        // moments of f~ (deviation form)
        R drho[V], jx[V], jy[V], en[V];
#pragma unroll
        for (int k = 0; k < V; ++k) drho[k] = jx[k] = jy[k] = en[k] = R(0);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const R ax = A.tab.a[VS::ix(a)], ay = A.tab.a[VS::iy(a)], a2 = A.tab.xi2[a];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                drho[k] += ft[a][k];
                jx[k] = fma(ax, ft[a][k], jx[k]);
                jy[k] = fma(ay, ft[a][k], jy[k]);
                en[k] = fma(a2, ft[a][k], en[k]);
            }
        }

        R sig[V], hh[V], uyv[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const R rho = A.rho0 + drho[k];
            const R inv = R(1) / rho;
            const R ux = jx[k] * inv, uy = jy[k] * inv;
            const R th = A.isothermal ? R(0) : (en[k] - R(2) * drho[k] - rho * (ux * ux + uy * uy)) * R(0.5) * inv;
            uyv[k] = uy;
            R s = R(0), h = R(0);
            equilibrium_dev<VS, N, R>(A.tab, drho[k], rho, ux, uy, th, [&](auto ac, R deq) {
                constexpr int a = decltype(ac)::value;
                const R f = ft[a][k];
                s = fma(A.tab.xixy[a], f - deq, s);
                if constexpr (KIND == kStep) {
                    h = fma(f * f, A.tab.winv[a], h);
                    ft[a][k] = fma(omega, deq - f, f);
                } else {
                    (void)h;
                }
            });
            sig[k] = s * A.sigma_fac;
            hh[k] = h;
            if constexpr (KIND == kMoments) {
                if (active && (x + k) < A.nx) {
                    const long long c = (long long)y * A.nx + x + k;
                    if (A.o_rho) A.o_rho[c] = (double)A.rho0 + (double)drho[k];
                    if (A.o_ux) A.o_ux[c] = (double)ux;
                    if (A.o_uy) A.o_uy[c] = (double)uy;
                    if (A.o_T) A.o_T[c] = 1.0 + (double)th;
                    if (A.o_sxy) A.o_sxy[c] = (double)sig[k];
                    if (A.o_pop) {
                        const long long pl = (long long)A.ny * A.nx;
#pragma unroll
                        for (int a = 0; a < Q; ++a)
                            A.o_pop[a * pl + c] = (double)A.tab.w[a] * (double)A.rho0 + (double)ft[a][k];
                    }
                }
            }
        }

        if constexpr (KIND == kStep) {
            if (active) {
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    S* p = dst + (long long)a * A.plane + (long long)y * A.pitch + x;
                    const R si = store_scale<S, R>(A.tab, a);
                    if constexpr (V == 2) {
                        st2<S, R>(p, ft[a][0], ft[a][1], si);
                    } else {
                        st1<S, R>(p, ft[a][0], si);
                    }
                }
            }
            if (diag) {
                R v6[6] = {0, 0, 0, 0, 0, 0};
                if (active) {
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        v6[0] += drho[k];
                        v6[1] += jx[k];
                        v6[2] += jy[k];
                        v6[3] = fma(uyv[k], A.sinx[x + k], v6[3]);
                        v6[4] = fma(sig[k], A.cosx[x + k], v6[4]);
                        v6[5] += hh[k];
                    }
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const R s = warp_sum(v6[i]);
                    if (lane == 0) acc[i] += (double)s;
                }
            }
        }
    }

    if constexpr (KIND == kStep) {
        __shared__ double red[kRows][6];
        __shared__ bool is_last;
        if (diag) {
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 6; ++i) red[warp][i] = acc[i];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (diag) {
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    double s = 0.0;
                    for (int w = 0; w < kRows; ++w) s += red[w][i];
                    A.partials[(long long)blockIdx.x * kDiagSlots + i] = s;
                }
            }
            __threadfence();
            const unsigned int t = atomicAdd(A.ticket, 1u);
            is_last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            if (diag) {
                __shared__ double tot[6];
                if (warp < 6) {
                    double s = 0.0;
                    for (int b = lane; b < (int)gridDim.x; b += 32)
                        s += __ldcg(A.partials + (long long)b * kDiagSlots + warp);
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
    }
}

// ------------------------------------------------------------ init kernel
// f~(0) = f^eq(rho, u, T) per cell (raw layout, no streaming), written to dst.
template <class VS, int N, class S, class R>
__global__ void __launch_bounds__(kThreads) lb_init_kernel(const __grid_constant__ Args<R> A) {
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
            st1<S, R>(dst + (long long)a * A.plane + (long long)y * A.pitch + x, deq, store_scale<S, R>(A.tab, a));
        });
    }
}

// ------------------------------------------------------------ dispatch
// kind = -1 queries the resident blocks per SM of the step kernel into *(int*)args.
template <class VS, int N, class S, class R>
cudaError_t launch_typed(const Launch& L) {
    constexpr int V = cells_per_thread(VS::Q);
    if (L.kind == -1) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            static_cast<int*>(const_cast<void*>(L.args)), lb_fused_kernel<VS, N, S, R, V, kStep>, kThreads, 0);
    }
    const Args<R>& A = *static_cast<const Args<R>*>(L.args);
    switch (L.kind) {
        case kStep:
            lb_fused_kernel<VS, N, S, R, V, kStep><<<L.grid, kThreads, 0, L.stream>>>(A);
            break;
        case kMoments:
            lb_fused_kernel<VS, N, S, R, V, kMoments><<<L.grid, kThreads, 0, L.stream>>>(A);
            break;
        case kInit:
            lb_init_kernel<VS, N, S, R><<<L.grid, kThreads, 0, L.stream>>>(A);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Entry point of one (velocity set, storage) translation unit.
template <class VS, class S, class R>
cudaError_t launch_order(const Launch& L) {
    switch (L.n_eq) {
        case 2: return launch_typed<VS, 2, S, R>(L);
        case 3: return launch_typed<VS, 3, S, R>(L);
        case 4: return launch_typed<VS, 4, S, R>(L);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbk
