// large_args.cuh -- constants and kernel arguments of the large-grid (n_f = 256) pipeline.
#pragma once

#include "common.cuh"
#include "ems.cuh"

namespace enufft {

constexpr int kMaxHalfL = 64;                 // P/2 <= 64
constexpr int kLNF = 256;                     // fine grid
constexpr int kLT = 32;                       // default tile side (nodes); 16 and 64 are built too
__host__ __device__ constexpr int large_tiles(int lt) { return (kLNF / lt) * (kLNF / lt); }
constexpr int kLTilesMax = large_tiles(16);   // tiles per cell at the smallest side (256)
constexpr int kLBinBlock = 4096;              // samples per sort block (one cell's consecutive samples)
constexpr int kLSortThreads = 512;
constexpr int kLSpreadThreads = 256;
constexpr int64_t kLSplitPoints = (int64_t)1 << 18;   // samples per spread work item (cells split above)

struct LargeArgs {
    const float* __restrict__ x;
    const float* __restrict__ y;
    const float* __restrict__ h;
    const float* __restrict__ w;
    const CellConst* __restrict__ cells;
    // batch
    int cell0, ncells;                        // cells [cell0, cell0 + ncells)
    int64_t p0;                               // offsets[cell0]
    const int4* __restrict__ blocks;          // sort blocks: {cell - cell0, q_begin - p0, q_end - p0, 0}
    const int2* __restrict__ cell_blocks;     // per batch cell: {first sort block (batch relative), count}
    const int4* __restrict__ work;            // spread work items, largest cells first: {cell - cell0, part, parts, 0}
    int* blk_off;                             // [sort block][tiles + 1]: tile offsets inside the block's range
    float* blk_abs;                           // [sort block][tiles]: sum |w h| / |D| of the block's samples per tile
    float4* rec;                              // [batch points] records {x, y, h, w}, tile-ordered per sort block
    unsigned long long* grid;                 // [ncells][256][256] fine grids, 64-bit two's complement
                                              // fixed point at the cell's scale 2^k (cell_exp)
    int* cell_exp;                            // [ncells] k of each batch cell
    unsigned* status;
    KernelPoly poly;
    int W;                                    // kernel width (the sort orders records by shared-memory bank)
};

constexpr int kLFftThreads = 512;
constexpr int kLRowStride = 272;              // >= 16 * 17 (team workspace), floats
constexpr int kLRowPairs = 32;                // row pairs per round

struct LargeFftArgs {
    const long long* __restrict__ grid;       // batch fine grids (fixed point, see LargeArgs)
    const int* __restrict__ cell_exp;         // [ncells] their scales 2^k
    int cell0, ncells, P;
    float* __restrict__ coeffs;               // all cells
    const cplx<float>* __restrict__ twiddle;  // W_256^j
    float inv_phi[kMaxHalfL + 1];
    int do_ems;
    EmsArgs ems;
    EmsScratch ems_out;
};

__host__ __device__ constexpr size_t large_fft_smem_bytes(int P) {
    return sizeof(cplx<float>) * (size_t)kLNF * (P / 2 + 1) + sizeof(float) * (size_t)2 * kLRowPairs * kLRowStride +
           sizeof(cplx<float>) * kLNF + sizeof(float) * (kMaxHalfL + 1) + 64;
}

}  // namespace enufft
