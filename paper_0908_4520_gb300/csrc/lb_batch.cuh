// Persistent multi-instance kernel: many small, uneven lattices in one launch.
//
// Each CTA takes instances from a work queue (an atomic counter over a list
// ordered by decreasing remaining cost, i.e. longest-processing-time first) and
// advances one instance at a time by up to `chunk` time levels, with a block
// barrier between levels: an instance never spans CTAs, so no CTA ever waits
// on another.  An instance whose two population buffers fit the CTA's shared
// memory is copied in once per chunk and stepped entirely on chip; larger ones
// step through global memory (L2-resident at these sizes).  A warp advances
// strips of up to 30 cells of one row: each lane streams one column in y (three
// loads per velocity) and takes its neighbours' columns by shuffles for the x
// pass, the two edge lanes streaming the columns beside the strip, as the
// single-lattice kernels do.  The per-cell arithmetic is collide_cell_pairs(),
// the collision those kernels call, and a cell's operations do not depend on
// the path (on chip or through global memory, a CTA or a warp), so an
// instance's populations are bitwise the same whichever path runs it and
// whatever else shares the launch.  Lax-Wendroff streaming only: the batch
// serves the Gauss-Hermite product sets.
#pragma once

#include "lb_batch.h"
#include "lb_kernels.cuh"

namespace lbk {

constexpr int kBatchMaxWarps = 8;  // warps per CTA (the kernel's launch bound: 256 threads)
constexpr int kStrip = 30;  // cells of a row per warp and pass (two lanes stream the columns beside them)

// the kernel's static shared memory (one copy, whichever instance template runs)
struct BatchShared {
    float red[kBatchMaxWarps][3];           // per-warp partial sums of a level's diagnostics
    int done[kBatchMaxWarps];               // stop flag of each group (the CTA, or each warp)
    float relax[kBatchMaxWarps][4][kMaxNA]; // relaxation tables of each group's instance
};

template <class S>
__device__ __forceinline__ float batch_load(const S* p, float sc) {
    if constexpr (Is16<S>::value) {
        return (std::is_same<S, __half>::value ? __half2float(*reinterpret_cast<const __half*>(p))
                                               : __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p))) *
               sc;
    } else {
        (void)sc;
        return *p;
    }
}

// Advance instance `id` by up to B.chunk levels with the CTA's threads (WARP = false) or with
// one warp of it (WARP = true: small instances, so that a CTA advances several at once; smem is
// then the warp's slice of the shared memory, smem_cap bytes).
template <class VS, int N, class S, bool WARP = false>
__device__ __noinline__ void batch_run(const BatchArgs& B, int id, S* smem, int smem_cap, BatchShared& sh) {
    constexpr int Q = VS::Q;
    BatchInst& in = B.inst[id];
    const Tab<float>& t = B.tab[in.set];
    const int nx = in.nx, ny = in.ny;
    const int ncell = nx * ny;
    const long long pop = (long long)Q * ncell;
    const float omega = in.omega, sigma_fac = in.sigma_fac;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tid = WARP ? lane : (int)threadIdx.x, nthr = WARP ? 32 : (int)blockDim.x;
    const int nwarp = (nthr + 31) >> 5;
    // the instance's relaxation tables (omega W_i and the second terms of the exact FP32
    // identities) in shared memory, one copy per group (the CTA, or each warp)
    float(*rt)[kMaxNA] = sh.relax[WARP ? warp : 0];
    if (tid < VS::NA) {
        rt[0][tid] = in.ow[tid];
        rt[1][tid] = in.owlo[tid];
        rt[2][tid] = in.hn1lo[tid];
        rt[3][tid] = in.whn1lo[tid];
    }
    const float* sinx = B.trig + in.trig_off;
    const float* cosx = sinx + nx;
    float2* hist = B.hist + in.hist_off;
    const int spr = (nx + kStrip - 1) / kStrip;  // strips per row
    const int nstrip = spr * ny;
    int& s_done = sh.done[WARP ? warp : 0];  // the group's stop flag
    auto group_sync = [&]() {
        if constexpr (WARP) {
            __syncwarp();
        } else {
            __syncthreads();
        }
    };

    int level = in.level;
    int cur = in.cur;
    const int stop = min(in.max_level, level + B.chunk - 1);
    // both buffers of an instance that fits the group's shared memory are stepped on chip
    const bool onchip = 2 * pop * (long long)sizeof(S) <= (long long)smem_cap;
    S* const arena = static_cast<S*>(B.arena);
    S* gbuf[2] = {arena + in.off[0], arena + in.off[1]};
    S* buf[2] = {gbuf[0], gbuf[1]};
    if (onchip) {
        buf[0] = smem;
        buf[1] = smem + pop;
        if (level > 0)
            for (long long k = tid; k < pop; k += nthr) buf[cur][k] = gbuf[cur][k];
    }
    if (tid == 0) s_done = in.done;
    group_sync();

    // 16-bit storage: deviation = stored * sc[a] * scale; sc (tables built with S = 1) and
    // scale are powers of two, so the load and store scales are exact inverses
    const float scale = in.scale;
    const float inv_scale = 1.0f / scale;
    for (; level <= stop && !s_done; ++level) {
        const S* src = buf[cur];
        S* dst = buf[level == 0 ? 0 : 1 - cur];
        float pa = 0.f, ps = 0.f, ph = 0.f;
        bool bad = false;
        // strips of up to 30 cells of one row, one per warp at a time: lanes 1..w own cells
        // x0 .. x0 + w - 1; lanes 0 and w + 1 stream the columns beside the strip, so that each
        // lane streams one column in y and takes its neighbours' columns by shuffles for the x
        // pass; lanes past w + 1 repeat lane w + 1's column and own nothing
        for (int s = WARP ? 0 : warp; s < nstrip; s += WARP ? 1 : nwarp) {
            const int y = s / spr, x0 = (s - y * spr) * kStrip;
            const int w = min(kStrip, nx - x0);
            int x = x0 + min(lane, w + 1) - 1;
            x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            const bool own = lane >= 1 && lane <= w;
            const int c = y * nx + x;
            float ft[Q];
            if (level == 0) {
                // f~(0) = f^eq(rho = 1, u_y = u0 sin x, T = 1), rounded through the storage type
                const double sx = sinpi(2.0 * (double)x / (double)nx);
                const float uy = (float)(in.u0 * sx);
                equilibrium_dev<VS, N, float>(t, 0.f, 1.f, 0.f, uy, 0.f, [&](auto ac, float deq) {
                    constexpr int a = decltype(ac)::value;
                    if constexpr (Is16<S>::value) {
                        S tmp;
                        st1<S, float>(&tmp, deq, t.scinv[a] * inv_scale);
                        ft[a] = batch_load<S>(&tmp, t.sc[a] * scale);
                    } else {
                        ft[a] = deq;
                    }
                });
            } else {
                const int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
                const int om = ym * nx + x, op = yp * nx + x;
                const bool rows = ny > 1;  // one row: the three y taps read the same value
                static_for<0, Q>([&](auto ac) {
                    constexpr int a = decltype(ac)::value;
                    constexpr int ix = VS::ix(a), iy = VS::iy(a);
                    const float sc = Is16<S>::value ? t.sc[a] * scale : 1.f;
                    const S* pl = src + (long long)a * ncell;
                    const float v0 = batch_load<S>(pl + c, sc);
                    const float vm = rows ? batch_load<S>(pl + om, sc) : v0;
                    const float vp = rows ? batch_load<S>(pl + op, sc) : v0;
                    const float g = fma(t.lw[iy][0], vm, fma(t.lw[iy][1], v0, t.lw[iy][2] * vp));
                    const float gl = __shfl_up_sync(0xffffffffu, g, 1);
                    const float gr = __shfl_down_sync(0xffffffffu, g, 1);
                    ft[a] = fma(t.lw[ix][0], gl, fma(t.lw[ix][1], g, t.lw[ix][2] * gr));
                });
            }
            // velocity pairs of equal x node as packed f32x2 values (the one-cell-per-lane
            // collision of the single-lattice kernels)
            f2 fp[Q / 2];
            static_for<0, Q / 2>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                fp[m] = f2{ft[2 * m], ft[2 * m + 1]};
            });
            const CellOut<float> co = collide_cell_pairs<VS, N, true>(
                t, rt[0], rt[1], rt[2], rt[3], 1.f, omega, sigma_fac, in.isothermal, true, false, 0.f, 0.f, 0.f,
                [&](auto mc) -> f2& { return fp[decltype(mc)::value]; });
            if (own) {
                static_for<0, Q / 2>([&](auto mc) {
                    constexpr int m = decltype(mc)::value;
                    ft[2 * m] = fp[m].x;
                    ft[2 * m + 1] = fp[m].y;
                });
                uint32_t r = Is16<S>::value ? sr_seed(level, c) : 0u;
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    if constexpr (Is16<S>::value) r = sr_next(r);
                    dst[(long long)a * ncell + c] =
                        to_storage<S, float>(ft[a], Is16<S>::value ? t.scinv[a] * inv_scale : 1.f, r);
                }
                pa = fma(co.uy, sinx[x], pa);
                ps = fma(co.sig, cosx[x], ps);
                ph += co.h;
                bad |= !isfinite(co.h);
            }
        }
        pa = warp_sum(pa);
        ps = warp_sum(ps);
        ph = warp_sum(ph);
        bad = __any_sync(0xffffffffu, bad);
        if (!WARP && lane == 0) {
            sh.red[warp][0] = pa;
            sh.red[warp][1] = ps;
            sh.red[warp][2] = bad ? __int_as_float(0x7fc00000) : ph;
        }
        group_sync();
        if (tid == 0) {
            double A = 0, Sx = 0, H = 0;
            if constexpr (WARP) {
                A = pa;
                Sx = ps;
                H = bad ? (double)__int_as_float(0x7fc00000) : (double)ph;
            } else {
                for (int w = 0; w < nwarp; ++w) {
                    A += sh.red[w][0];
                    Sx += sh.red[w][1];
                    H += sh.red[w][2];
                }
            }
            const double norm = 2.0 / (double)ncell;
            hist[level] = make_float2((float)(A * norm), (float)(Sx * norm));
            if (level == 0) in.h0 = (float)H;
            int d = 0;
            if (!isfinite(H)) {
                in.status |= 1;
                d = 1;
            }
            // stop rule sqrt(H / H0) <= stop_ratio (none for stop_ratio = 0, also where H is 0)
            if (level > 0 && in.stop_ratio2 > 0.f && (double)H <= (double)in.stop_ratio2 * (double)in.h0) d = 1;
            if (level == in.max_level) d = 1;
            s_done = d;
        }
        cur = (level == 0) ? 0 : 1 - cur;
        group_sync();
    }
    if (onchip && level > in.level)
        for (long long k = tid; k < pop; k += nthr) gbuf[cur][k] = buf[cur][k];
    if (tid == 0) {
        in.level = level;
        in.cur = cur;
        in.done = s_done;
    }
    group_sync();
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class S, bool WARP>
__device__ __forceinline__ void batch_dispatch(const BatchArgs& B, int id, S* smem, int smem_cap, BatchShared& sh) {
    const BatchInst& in = B.inst[id];
    switch (in.set * 3 + (in.n_eq - 2)) {
        case 0: batch_run<lbvs::GH4, 2, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 1: batch_run<lbvs::GH4, 3, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 2: batch_run<lbvs::GH4, 4, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 3: batch_run<lbvs::GH6, 2, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 4: batch_run<lbvs::GH6, 3, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 5: batch_run<lbvs::GH6, 4, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 6: batch_run<lbvs::GH8, 2, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 7: batch_run<lbvs::GH8, 3, S, WARP>(B, id, smem, smem_cap, sh); break;
        case 8: batch_run<lbvs::GH8, 4, S, WARP>(B, id, smem, smem_cap, sh); break;
        default: break;
    }
}

// Instances come from two work queues ordered longest-first: the CTA queue (each instance
// advanced by the whole CTA) and, once it is empty, the warp queue (instances of at most
// warp_cells cells, each advanced by one warp with its slice of the shared memory).
template <class S>
__global__ void __launch_bounds__(kBatchMaxWarps * 32) lb_batch_kernel(const __grid_constant__ BatchArgs B) {
    extern __shared__ __align__(16) unsigned char bsm[];
    S* smem = reinterpret_cast<S*>(bsm);
    __shared__ int s_i;
    __shared__ BatchShared sh;
    // start and end of every CTA (the launch's tail: how long the last CTA runs alone)
    if (B.cta_clock && threadIdx.x == 0) B.cta_clock[2 * blockIdx.x] = global_ns();
    for (;;) {
        if (threadIdx.x == 0) s_i = atomicAdd(B.next, 1);
        __syncthreads();
        const int i = s_i;
        __syncthreads();
        if (i >= *B.n_order) break;
        const int id = B.order[i];
        if (B.inst[id].done) continue;
        batch_dispatch<S, false>(B, id, smem, B.smem_cap, sh);
    }
    if (B.n_small) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        // each warp's slice of the shared memory, 16-byte aligned
        const int slice = (B.smem_cap / nwarp) & ~15;
        S* wsm = reinterpret_cast<S*>(bsm + (size_t)warp * slice);
        for (;;) {
            int i = 0;
            if (lane == 0) i = atomicAdd(B.next_small, 1);
            i = __shfl_sync(0xffffffffu, i, 0);
            if (i >= *B.n_small) break;
            const int id = B.order_small[i];
            if (B.inst[id].done) continue;
            batch_dispatch<S, true>(B, id, wsm, slice, sh);
        }
    }
    __syncthreads();
    if (B.cta_clock && threadIdx.x == 0) B.cta_clock[2 * blockIdx.x + 1] = global_ns();
}

}  // namespace lbk
