// Instantiation and launch of the persistent multi-instance kernel for one
// storage type (compiled once per type with LB_BATCH_STORAGE / LB_BATCH_ENTRY).
#include "lb_batch.cuh"

namespace lbk {

namespace {
template <class S>
cudaError_t launch_s(const void* args, int grid, int threads, int smem, cudaStream_t st) {
    const BatchArgs& B = *static_cast<const BatchArgs*>(args);
    lb_batch_kernel<S><<<grid, threads, smem, st>>>(B);
    return cudaGetLastError();
}

template <class S>
cudaError_t setup_s(int threads, int smem, int* occupancy) {
    // the attribute belongs to the kernel, not to a batch: raise it to the device limit once,
    // so batches with different on-chip budgets can coexist
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // (the dynamic limit leaves room for the kernel's own static shared memory)
    cudaFuncAttributes attr{};
    cudaError_t e = cudaFuncGetAttributes(&attr, lb_batch_kernel<S>);
    if (e != cudaSuccess) return e;
    const int room = optin - (int)attr.sharedSizeBytes;
    if (smem > room) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(lb_batch_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, lb_batch_kernel<S>, threads, smem);
}
}  // namespace

#ifndef LB_BATCH_STORAGE
#error "LB_BATCH_STORAGE must name the storage type of this unit"
#endif

cudaError_t LB_BATCH_ENTRY(launch)(const void* args, int grid, int threads, int smem, cudaStream_t st) {
    return launch_s<LB_BATCH_STORAGE>(args, grid, threads, smem, st);
}

cudaError_t LB_BATCH_ENTRY(setup)(int threads, int smem, int* occupancy) {
    return setup_s<LB_BATCH_STORAGE>(threads, smem, occupancy);
}

}  // namespace lbk
