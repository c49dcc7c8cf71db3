// inst_large.cu -- launchers of the large-grid (n_f = 256) pipeline.
#include "internal.h"
#include "large.cuh"

namespace enufft {

cudaError_t large_prepare(int P) {
    return cudaFuncSetAttribute(large_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)large_fft_smem_bytes(P));
}

template <int W>
static void launch_spread(const LargeArgs& la, int nblocks, cudaStream_t s) {
    large_spread_kernel<W><<<nblocks, kLSpreadThreads, 0, s>>>(la);
}

cudaError_t large_run_batch(const LargeArgs& la, int nbin_blocks, int nwork, const LargeFftArgs& fa, int W,
                            int fft_grid, cudaStream_t s) {
    if (la.ncells <= 0) return cudaSuccess;
    if (nbin_blocks > 0) large_sort_kernel<<<nbin_blocks, kLSortThreads, 0, s>>>(la);
    constexpr int cells_per_block = kLScaleThreads / 32;
    large_scale_kernel<<<(la.ncells + cells_per_block - 1) / cells_per_block, kLScaleThreads, 0, s>>>(la);
    const int nt = nwork * kLTiles;
    switch (W) {
        case 4: launch_spread<4>(la, nt, s); break;
        case 5: launch_spread<5>(la, nt, s); break;
        case 6: launch_spread<6>(la, nt, s); break;
        case 7: launch_spread<7>(la, nt, s); break;
        case 8: launch_spread<8>(la, nt, s); break;
        default: return cudaErrorInvalidValue;
    }
    large_fft_kernel<<<fft_grid, kLFftThreads, large_fft_smem_bytes(fa.P), s>>>(fa);
    return cudaGetLastError();
}

}  // namespace enufft
