// Instantiations of the alignment kernel for windows of up to 128 bases.
#include "align_kernel.cuh"

namespace scrooge {

cudaError_t launch_align_w128(const AlignParams &p, int lanes, bool sene, int warps_per_block, int blocks,
                                 size_t smem_bytes, cudaStream_t stream) {
    const dim3 grid(blocks), block(32 * warps_per_block);
    switch (lanes * 2 + (sene ? 1 : 0)) {
        case 17:
            kern::align_kernel<4, 8, true><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 16:
            kern::align_kernel<4, 8, false><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 33:
            kern::align_kernel<4, 16, true><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 32:
            kern::align_kernel<4, 16, false><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_w128(int lanes, bool sene, int warps_per_block, size_t smem_bytes, int *blocks) {
    const int threads = 32 * warps_per_block;
    switch (lanes * 2 + (sene ? 1 : 0)) {
        case 17:
            cudaFuncSetAttribute(kern::align_kernel<4, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<4, 8, true>, threads, smem_bytes);
        case 16:
            cudaFuncSetAttribute(kern::align_kernel<4, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<4, 8, false>, threads, smem_bytes);
        case 33:
            cudaFuncSetAttribute(kern::align_kernel<4, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<4, 16, true>, threads, smem_bytes);
        case 32:
            cudaFuncSetAttribute(kern::align_kernel<4, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<4, 16, false>, threads, smem_bytes);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace scrooge
