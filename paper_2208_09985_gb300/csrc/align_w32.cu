// Instantiations of the alignment kernel for windows of up to 32 bases.
#include "align_kernel.cuh"

namespace scrooge {

cudaError_t launch_align_w32(const AlignParams &p, int lanes, bool sene, int warps_per_block, int blocks,
                                 size_t smem_bytes, cudaStream_t stream) {
    const dim3 grid(blocks), block(32 * warps_per_block);
    switch (lanes * 2 + (sene ? 1 : 0)) {
        case 3:
            kern::align_kernel<1, 1, true><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 2:
            kern::align_kernel<1, 1, false><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 5:
            kern::align_kernel<1, 2, true><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 4:
            kern::align_kernel<1, 2, false><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 9:
            kern::align_kernel<1, 4, true><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case 8:
            kern::align_kernel<1, 4, false><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_w32(int lanes, bool sene, int warps_per_block, size_t smem_bytes, int *blocks) {
    const int threads = 32 * warps_per_block;
    switch (lanes * 2 + (sene ? 1 : 0)) {
        case 3:
            cudaFuncSetAttribute(kern::align_kernel<1, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<1, 1, true>, threads, smem_bytes);
        case 2:
            cudaFuncSetAttribute(kern::align_kernel<1, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<1, 1, false>, threads, smem_bytes);
        case 5:
            cudaFuncSetAttribute(kern::align_kernel<1, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<1, 2, true>, threads, smem_bytes);
        case 4:
            cudaFuncSetAttribute(kern::align_kernel<1, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<1, 2, false>, threads, smem_bytes);
        case 9:
            cudaFuncSetAttribute(kern::align_kernel<1, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<1, 4, true>, threads, smem_bytes);
        case 8:
            cudaFuncSetAttribute(kern::align_kernel<1, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern::align_kernel<1, 4, false>, threads, smem_bytes);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace scrooge
