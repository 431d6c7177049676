// Host/device descriptors of the persistent multi-instance kernel.
#pragma once

#include "lb_device.h"

namespace lbk {

// Device descriptor of one instance (slot).
struct BatchInst {
    long long off[2];     // element offsets of the two population buffers in the arena
    long long hist_off;   // offset of the (A, S) history (float2 per level)
    long long trig_off;   // offset of the sin/cos(x_i) table (2 nx floats)
    int set;              // 0: D2Q16-GH, 1: D2Q36-GH, 2: D2Q64-GH
    int n_eq;             // 2..4
    int nx, ny;
    int max_level;        // last time level to process
    int level;            // next time level to process (0: not started)
    int cur;              // buffer holding the pending (post-collision) populations
    int done;             // 1: finished (stop rule or max_level)
    int status;           // bit 0: non-finite
    int isothermal;
    float omega, sigma_fac;
    float scale;          // 16-bit storage: deviation = stored * sc[a] * scale (powers of two)
    float stop_ratio2;    // stop once H <= stop_ratio2 * H0 (0: never)
    float h0;             // H at level 0
    float pad;
    double u0;            // shear-wave amplitude
    double dt;
    // relaxation tables of this omega: omega W_i and the second terms of the exact FP32
    // conservation identities (see Tab)
    float ow[kMaxNA], owlo[kMaxNA], hn1lo[kMaxNA], whn1lo[kMaxNA];
};

struct BatchArgs {
    BatchInst* inst;
    const int* order;     // slots in processing order
    const int* n_order;   // number of slots in `order` (device, so a captured graph stays valid)
    int* next;            // work-queue counter (reset before each launch)
    int chunk;            // levels per instance per launch
    int smem_cap;         // bytes of dynamic shared memory available for on-chip instances
    void* arena;          // population storage (the batch's storage type)
    float2* hist;
    const float* trig;
    Tab<float> tab[3];    // per set (weights, nodes, Hermite and Lax-Wendroff tables)
    unsigned long long* cta_clock;  // per CTA: %globaltimer at start and at end (2 grid entries; may be null)
    // warp queue (may be null): instances of at most warp_cells cells, one warp each
    const int* order_small;
    const int* n_small;
    int* next_small;
};

cudaError_t batch_launch_f32(const void* args, int grid, int threads, int smem, cudaStream_t st);
cudaError_t batch_launch_f16(const void* args, int grid, int threads, int smem, cudaStream_t st);
cudaError_t batch_launch_bf16(const void* args, int grid, int threads, int smem, cudaStream_t st);
cudaError_t batch_setup_f32(int threads, int smem, int* occupancy);
cudaError_t batch_setup_f16(int threads, int smem, int* occupancy);
cudaError_t batch_setup_bf16(int threads, int smem, int* occupancy);

}  // namespace lbk
