// Discrete velocity method (DVM) for the linearised BGK equation of the standing
// shear wave, in the reduced form of Sec. 3.3 (Eqs. LBGK, ga, gb): the unknown
// G(x, xi_k, t) at the nodes xi_k of an n-point Gauss-Hermite rule obeys
// dG/dt + xi_k dG/dx = (u - G) / tau + g with u = sum_k w_k G_k and the body force
// g(x, t) = A_f sin(x_i) cos(phi t) (0 for the free wave).  The other reduced function
// (Eq. ga) is homogeneous, starts at zero and stays zero, so the force term of Eq. gb,
// g (G_a + 1), is g itself.
//
// Space-time discretisation (independent of the lattice; the paper solves the DVM with
// Lax-Wendroff): Strang splitting of the relaxation and force, integrated exactly (u gains
// int g dt since sum w_k = 1; G - u decays by exp(-h / tau)), around one Lax-Wendroff
// advection step; dt = cfl dx / max|xi_k|.
// Observables per level: A = 2/nx sum u sin(x_i), S = 2/nx sum sigma cos(x_i),
// sigma = sum_k w_k xi_k G.
//
// One CTA advances one instance (one collision time) through all its levels with G in
// shared memory (FP64); instances run in parallel.  Problems are small (nx x n nodes),
// so the kernel is latency-bound by design; it exists for the DVM cross-check of the
// lattice Boltzmann runs, not as a bandwidth kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_host.h"

namespace {

constexpr int kDvmMaxNodes = 64;
constexpr int kDvmThreads = 256;

struct DvmArgs {
    int nx, nv, nsteps, n_inst;
    double dx, dt, u0;
    double force_amp, force_freq;
    const double* tau;   // n_inst collision times
    double* amp;         // n_inst x (nsteps + 1)
    double* shear;
    double xi[kDvmMaxNodes], w[kDvmMaxNodes];
};

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];  // fixed order
    return s;  // valid in thread 0
}

// A_f int_{t0}^{t0 + h} cos(phi t) dt
__device__ double force_integral(const DvmArgs& A, double t0, double h) {
    if (A.force_amp == 0.0) return 0.0;
    if (A.force_freq == 0.0) return A.force_amp * h;
    return A.force_amp * (sin(A.force_freq * (t0 + h)) - sin(A.force_freq * t0)) / A.force_freq;
}

__global__ void __launch_bounds__(kDvmThreads) lb_dvm_kernel(const __grid_constant__ DvmArgs A) {
    extern __shared__ double sm[];
    const int nx = A.nx, nv = A.nv;
    double* G = sm;                  // nv x nx
    double* u = G + (size_t)nv * nx;  // nx
    double* row = u + nx;            // nx (advection scratch)
    __shared__ double red[kDvmThreads / 32];
    const int inst = blockIdx.x;
    const double tau = A.tau[inst];
    const double decay_half = exp(-0.5 * A.dt / tau);
    // equilibrium start: psi = xi_y u_y, so G = u_y(x) at every node
    for (int idx = threadIdx.x; idx < nv * nx; idx += blockDim.x) {
        const int i = idx % nx;
        G[idx] = A.u0 * sin(i * A.dx);
    }
    __syncthreads();
    for (int s = 0;; ++s) {
        // moments and observables of level s
        double pa = 0.0, ps = 0.0;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double ui = 0.0, si = 0.0;
            for (int k = 0; k < nv; ++k) {
                const double g = G[(size_t)k * nx + i];
                ui += A.w[k] * g;
                si += A.w[k] * A.xi[k] * g;
            }
            u[i] = ui;
            pa += ui * sin(i * A.dx);
            ps += si * cos(i * A.dx);
        }
        const double ta = block_sum(pa, red);
        const double ts = block_sum(ps, red);
        if (threadIdx.x == 0) {
            A.amp[(size_t)inst * (A.nsteps + 1) + s] = 2.0 * ta / nx;
            A.shear[(size_t)inst * (A.nsteps + 1) + s] = 2.0 * ts / nx;
        }
        if (s == A.nsteps) break;
        __syncthreads();
        // half relaxation with the force over [t_s, t_s + dt/2]
        const double c1 = force_integral(A, s * A.dt, 0.5 * A.dt);
        for (int idx = threadIdx.x; idx < nv * nx; idx += blockDim.x) {
            const int i = idx % nx;
            const double ui = u[i];
            G[idx] = (ui + c1 * sin(i * A.dx)) + (G[idx] - ui) * decay_half;
        }
        __syncthreads();
        // Lax-Wendroff advection, node by node, periodic
        for (int k = 0; k < nv; ++k) {
            const double C = A.xi[k] * A.dt / A.dx;
            const double* g = G + (size_t)k * nx;
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const double fm = g[(i - 1 + nx) % nx], f0 = g[i], fp = g[(i + 1) % nx];
                row[i] = f0 - 0.5 * C * (fp - fm) + 0.5 * C * C * (fp - 2.0 * f0 + fm);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nx; i += blockDim.x) G[(size_t)k * nx + i] = row[i];
            __syncthreads();
        }
        // second half relaxation about the advected u, with the force over [t_s + dt/2, t_s + dt]
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double ui = 0.0;
            for (int k = 0; k < nv; ++k) ui += A.w[k] * G[(size_t)k * nx + i];
            u[i] = ui;
        }
        __syncthreads();
        const double c2 = force_integral(A, (s + 0.5) * A.dt, 0.5 * A.dt);
        for (int idx = threadIdx.x; idx < nv * nx; idx += blockDim.x) {
            const int i = idx % nx;
            const double ui = u[i];
            G[idx] = (ui + c2 * sin(i * A.dx)) + (G[idx] - ui) * decay_half;
        }
        __syncthreads();
    }
}

lb_status dvm_fail(lb_status s, const std::string& m) {
    lbh::set_last_error(m);
    return s;
}

}  // namespace

extern "C" {

lb_status lb_dvm_run(int n_inst, const double* tau, int n_nodes, int nx, double cfl, double u0, int nsteps,
                     double* amp, double* shear, void* stream) {
    return lb_dvm_run_forced(n_inst, tau, n_nodes, nx, cfl, u0, 0.0, 0.0, nsteps, amp, shear, stream);
}

lb_status lb_dvm_run_forced(int n_inst, const double* tau, int n_nodes, int nx, double cfl, double u0,
                            double force_amp, double force_freq, int nsteps, double* amp, double* shear,
                            void* stream) {
    if (n_inst < 1 || !tau || !amp || !shear) return dvm_fail(LB_ERR_ARG, "n_inst >= 1 and tau, amp, shear are required");
    if (n_nodes < 1 || n_nodes > kDvmMaxNodes) return dvm_fail(LB_ERR_ARG, "n_nodes must be in [1, 64]");
    if (nx < 3 || nsteps < 0 || !(cfl > 0.0 && cfl <= 1.0) || !std::isfinite(u0))
        return dvm_fail(LB_ERR_ARG, "nx >= 3, nsteps >= 0, 0 < cfl <= 1 and a finite u0 are required");
    if (!std::isfinite(force_amp) || !std::isfinite(force_freq))
        return dvm_fail(LB_ERR_ARG, "force_amp and force_freq must be finite");
    for (int i = 0; i < n_inst; ++i)
        if (!(tau[i] > 0.0) || !std::isfinite(tau[i])) return dvm_fail(LB_ERR_ARG, "collision times must be positive");
    const size_t smem = sizeof(double) * ((size_t)n_nodes * nx + 2 * (size_t)nx);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return dvm_fail(LB_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    if (smem > (size_t)optin)
        return dvm_fail(LB_ERR_UNSUPPORTED, "n_nodes x nx too large for one CTA's shared memory (" +
                                                std::to_string(smem) + " > " + std::to_string(optin) + " bytes)");
    std::vector<double> x, w;
    lbh::gauss_hermite(n_nodes, x, w);
    DvmArgs A{};
    A.nx = nx;
    A.nv = n_nodes;
    A.nsteps = nsteps;
    A.n_inst = n_inst;
    A.dx = 2.0 * M_PI / nx;
    double vmax = 0.0;
    for (int k = 0; k < n_nodes; ++k) {
        A.xi[k] = x[k];
        A.w[k] = w[k];
        vmax = std::max(vmax, std::fabs(x[k]));
    }
    A.dt = cfl * A.dx / (vmax > 0 ? vmax : 1.0);
    A.u0 = u0;
    A.force_amp = force_amp;
    A.force_freq = force_freq;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t rec = (size_t)n_inst * ((size_t)nsteps + 1);
    double *d_tau = nullptr, *d_out = nullptr;
    e = cudaMalloc(&d_tau, sizeof(double) * n_inst);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double) * 2 * rec);
    if (e != cudaSuccess) {
        cudaFree(d_tau);
        return dvm_fail(LB_ERR_NOMEM, "DVM device buffers");
    }
    A.tau = d_tau;
    A.amp = d_out;
    A.shear = d_out + rec;
    e = cudaMemcpyAsync(d_tau, tau, sizeof(double) * n_inst, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lb_dvm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        lb_dvm_kernel<<<n_inst, kDvmThreads, smem, s>>>(A);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(amp, A.amp, sizeof(double) * rec, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(shear, A.shear, sizeof(double) * rec, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_tau);
    cudaFree(d_out);
    if (e != cudaSuccess) return dvm_fail(LB_ERR_CUDA, std::string("DVM run: ") + cudaGetErrorString(e));
    return LB_OK;
}

}  // extern "C"
