// Instantiations of the alignment kernel for windows of up to 128 bases.
#include "align_kernel.cuh"

namespace scrooge {

namespace {
constexpr int key(int lanes, bool sene, int swp) { return (lanes * 2 + (sene ? 1 : 0)) * 8 + swp; }
}  // namespace

cudaError_t launch_align_w128(const AlignParams &p, int lanes, bool sene, int swp, int warps_per_block,
                             int blocks, size_t smem_bytes, cudaStream_t stream) {
    const dim3 grid(blocks), block(32 * warps_per_block);
    switch (key(lanes, sene, swp)) {
        case key(8, true, 1):
            kern::align_kernel<4, 8, true, 1><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(8, true, 2):
            kern::align_kernel<4, 8, true, 2><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(8, true, 4):
            kern::align_kernel<4, 8, true, 4><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(16, true, 1):
            kern::align_kernel<4, 16, true, 1><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(16, true, 2):
            kern::align_kernel<4, 16, true, 2><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(16, true, 4):
            kern::align_kernel<4, 16, true, 4><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(8, false, 1):
            kern::align_kernel<4, 8, false, 1><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(8, false, 2):
            kern::align_kernel<4, 8, false, 2><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        case key(8, false, 4):
            kern::align_kernel<4, 8, false, 4><<<grid, block, smem_bytes, stream>>>(p);
            return cudaGetLastError();
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_w128(int lanes, bool sene, int swp, int warps_per_block, size_t smem_bytes, int *blocks) {
    const int threads = 32 * warps_per_block;
    switch (key(lanes, sene, swp)) {
        case key(8, true, 1):
            return occupancy_raising_smem(kern::align_kernel<4, 8, true, 1>, threads, smem_bytes, blocks);
        case key(8, true, 2):
            return occupancy_raising_smem(kern::align_kernel<4, 8, true, 2>, threads, smem_bytes, blocks);
        case key(8, true, 4):
            return occupancy_raising_smem(kern::align_kernel<4, 8, true, 4>, threads, smem_bytes, blocks);
        case key(16, true, 1):
            return occupancy_raising_smem(kern::align_kernel<4, 16, true, 1>, threads, smem_bytes, blocks);
        case key(16, true, 2):
            return occupancy_raising_smem(kern::align_kernel<4, 16, true, 2>, threads, smem_bytes, blocks);
        case key(16, true, 4):
            return occupancy_raising_smem(kern::align_kernel<4, 16, true, 4>, threads, smem_bytes, blocks);
        case key(8, false, 1):
            return occupancy_raising_smem(kern::align_kernel<4, 8, false, 1>, threads, smem_bytes, blocks);
        case key(8, false, 2):
            return occupancy_raising_smem(kern::align_kernel<4, 8, false, 2>, threads, smem_bytes, blocks);
        case key(8, false, 4):
            return occupancy_raising_smem(kern::align_kernel<4, 8, false, 4>, threads, smem_bytes, blocks);
        default:
            return cudaErrorInvalidValue;
    }
}

bool supported_w128(int lanes, bool sene, int swp) {
    switch (key(lanes, sene, swp)) {
        case key(8, true, 1):
        case key(8, true, 2):
        case key(8, true, 4):
        case key(16, true, 1):
        case key(16, true, 2):
        case key(16, true, 4):
        case key(8, false, 1):
        case key(8, false, 2):
        case key(8, false, 4):
            return true;
        default:
            return false;
    }
}

}  // namespace scrooge
