// inst_large.cu -- launchers of the large-grid (n_f = 256) pipeline.
#include "internal.h"
#include "large.cuh"
#include "large_adj.cuh"

namespace enufft {

template <int W>
static cudaError_t interp_attr() {
    return cudaFuncSetAttribute(large_interp_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLInterpSmem);
}

cudaError_t large_prepare(int P) {
    cudaError_t e = cudaFuncSetAttribute(large_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)large_fft_smem_bytes(P));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(large_adj_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)large_adj_fft_smem_bytes(P));
    if (e == cudaSuccess) e = interp_attr<4>();
    if (e == cudaSuccess) e = interp_attr<5>();
    if (e == cudaSuccess) e = interp_attr<6>();
    if (e == cudaSuccess) e = interp_attr<7>();
    if (e == cudaSuccess) e = interp_attr<8>();
    return e;
}

cudaError_t large_run_adjoint_batch(const LargeAdjFftArgs& fa, const LargeInterpArgs& ia, int nwork, int W,
                                    int fft_grid, double* stats, const CellConst* cells, cudaStream_t s) {
    if (fa.ncells <= 0) return cudaSuccess;
    large_adj_fft_kernel<<<fft_grid, kLAdjThreads, large_adj_fft_smem_bytes(fa.P), s>>>(fa);
    if (nwork > 0) {
        switch (W) {
            case 4: large_interp_kernel<4><<<nwork, kLAdjThreads, kLInterpSmem, s>>>(ia); break;
            case 5: large_interp_kernel<5><<<nwork, kLAdjThreads, kLInterpSmem, s>>>(ia); break;
            case 6: large_interp_kernel<6><<<nwork, kLAdjThreads, kLInterpSmem, s>>>(ia); break;
            case 7: large_interp_kernel<7><<<nwork, kLAdjThreads, kLInterpSmem, s>>>(ia); break;
            case 8: large_interp_kernel<8><<<nwork, kLAdjThreads, kLInterpSmem, s>>>(ia); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (fa.mode == 1)
        large_recon_stats_kernel<<<(fa.ncells + 127) / 128, 128, 0, s>>>(fa.cell0, fa.ncells, ia.work, nwork, ia.partial,
                                                                        fa.spec, cells, stats);
    return cudaGetLastError();
}

template <int W, int LT>
static void launch_spread(const LargeArgs& la, int nblocks, cudaStream_t s) {
    large_spread_kernel<W, LT><<<nblocks, kLSpreadThreads, 0, s>>>(la);
}

template <int LT>
static cudaError_t run_batch_tiles(const LargeArgs& la, int nbin_blocks, int nwork, int W, cudaStream_t s) {
    if (nbin_blocks > 0) large_sort_kernel<LT><<<nbin_blocks, kLSortThreads, 0, s>>>(la);
    constexpr int cells_per_block = kLScaleThreads / 32;
    large_scale_kernel<LT><<<(la.ncells + cells_per_block - 1) / cells_per_block, kLScaleThreads, 0, s>>>(la);
    const int nt = nwork * large_tiles(LT);
    switch (W) {
        case 4: launch_spread<4, LT>(la, nt, s); break;
        case 5: launch_spread<5, LT>(la, nt, s); break;
        case 6: launch_spread<6, LT>(la, nt, s); break;
        case 7: launch_spread<7, LT>(la, nt, s); break;
        case 8: launch_spread<8, LT>(la, nt, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t large_run_batch(const LargeArgs& la, int nbin_blocks, int nwork, const LargeFftArgs& fa, int W, int lt,
                            int fft_grid, cudaStream_t s) {
    if (la.ncells <= 0) return cudaSuccess;
    cudaError_t e;
    switch (lt) {
        case 16: e = run_batch_tiles<16>(la, nbin_blocks, nwork, W, s); break;
        case 32: e = run_batch_tiles<32>(la, nbin_blocks, nwork, W, s); break;
        case 64: e = run_batch_tiles<64>(la, nbin_blocks, nwork, W, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    large_fft_kernel<<<fft_grid, kLFftThreads, large_fft_smem_bytes(fa.P), s>>>(fa);
    return cudaGetLastError();
}

}  // namespace enufft
