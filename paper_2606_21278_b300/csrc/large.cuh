// large.cuh -- the type-1 transform for fine grids too large for one block's shared memory
// (n_f = 256, P up to 128): a sorted-by-subgrid pipeline over batches of cells.
//
//   1. bin      every sample: the 32 x 32 tile of the fine grid holding its centre node; per
//               block, shared histograms of tile counts and of sum |w h| / |D|, then one global
//               add per (block, tile);
//   2. scan     per cell: tile offsets in the batch's record buffer;
//   3. scatter  every sample into its tile's range (ranges reserved per block, slots inside a
//               block from a shared counter) as a 16-byte record {x, y, h, w};
//   4. spread   one block per (cell, tile): the tile's samples into a shared (32 + 2 halo)^2 tile in
//               32-bit fixed point at the tile's own scale 2^30 (1 - 2^-8) / S_tile (S_tile bounds
//               every node of the tile), then the tile is added to the cell's binary32 fine grid
//               in global memory (periodic wrap) by red.global.add.f32, row by row;
//   5. fft      one block per cell: row pairs through shared memory in rounds (team FFTs of
//               length 256), the P/2 + 1 needed columns in place, deconvolution/crop written as
//               coalesced rows of the output, and the EMS ranking read straight from the
//               half spectrum.
// The window test, the coordinates and the kernel of step 4 are those of the fused kernel
// (forward.cuh), so both routes compute the same sum.
#pragma once

#include "forward.cuh"
#include "large_args.cuh"

namespace enufft {

// tile of a sample from a plain binary32 evaluation of its grid coordinate (only used to sort:
// the exact coordinates are recomputed in step 4, and the tile halo absorbs a one-node difference)
__device__ __forceinline__ int large_tile_of(const CellConst& cc, float px, float py) {
    const float sx = (px - cc.cxh) * cc.sch + 0.5f * kLNF, sy = (py - cc.cyh) * cc.sch + 0.5f * kLNF;
    int tx = (int)floorf(sx) / kLT, ty = (int)floorf(sy) / kLT;
    tx = tx < 0 ? 0 : (tx > kLNF / kLT - 1 ? kLNF / kLT - 1 : tx);
    ty = ty < 0 ? 0 : (ty > kLNF / kLT - 1 ? kLNF / kLT - 1 : ty);
    if (!(sx == sx) || !(sy == sy)) { tx = 0; ty = 0; }
    return ty * (kLNF / kLT) + tx;
}

// 1. bin: counts and |c| sums per (cell, tile)
static __global__ void __launch_bounds__(256) large_bin_kernel(const __grid_constant__ LargeArgs a) {
    __shared__ int scnt[kLTiles];
    __shared__ float sabs[kLTiles];
    const int4 blk = a.blocks[blockIdx.x];
    const int cl = blk.x, cell = a.cell0 + cl;
    const CellConst& cc = a.cells[cell];
    for (int i = threadIdx.x; i < kLTiles; i += blockDim.x) { scnt[i] = 0; sabs[i] = 0.f; }
    __syncthreads();
    for (int64_t i = blk.y + threadIdx.x; i < blk.z; i += blockDim.x) {
        const int64_t q = a.p0 + i;
        const int t = large_tile_of(cc, a.x[q], a.y[q]);
        atomicAdd(&scnt[t], 1);
        const float v = fabsf(a.w[q] * a.h[q]) * cc.inv_area;
        atomicAdd(&sabs[t], (v <= 3.0e38f) ? v : 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLTiles; i += blockDim.x) {
        if (scnt[i]) {
            atomicAdd(&a.tile_cnt[cl * kLTiles + i], scnt[i]);
            atomicAdd(&a.tile_abs[cl * kLTiles + i], sabs[i]);
        }
    }
}

// 2. scan: per cell, tile offsets into the record buffer; cursors start at the offsets
static __global__ void large_scan_kernel(const __grid_constant__ LargeArgs a) {
    const int cl = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (cl >= a.ncells) return;
    const int base = (int)(a.offsets[a.cell0 + cl] - a.p0);
    const int c0 = a.tile_cnt[cl * kLTiles + lane], c1 = a.tile_cnt[cl * kLTiles + 32 + lane];
    int i0 = c0, i1 = c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v0 = __shfl_up_sync(0xffffffffu, i0, o), v1 = __shfl_up_sync(0xffffffffu, i1, o);
        if (lane >= o) { i0 += v0; i1 += v1; }
    }
    const int tot0 = __shfl_sync(0xffffffffu, i0, 31);
    const int e0 = base + i0 - c0, e1 = base + tot0 + i1 - c1;
    a.tile_off[cl * (kLTiles + 1) + lane] = e0;
    a.tile_off[cl * (kLTiles + 1) + 32 + lane] = e1;
    a.tile_cur[cl * kLTiles + lane] = e0;
    a.tile_cur[cl * kLTiles + 32 + lane] = e1;
    if (lane == 31) a.tile_off[cl * (kLTiles + 1) + kLTiles] = e1 + c1;
}

// 3. scatter into tile-sorted records: each block reserves one range per tile, then fills it
static __global__ void __launch_bounds__(256) large_scatter_kernel(const __grid_constant__ LargeArgs a) {
    __shared__ int scnt[kLTiles];
    __shared__ int sbase[kLTiles];
    const int4 blk = a.blocks[blockIdx.x];
    const int cl = blk.x, cell = a.cell0 + cl;
    const CellConst& cc = a.cells[cell];
    for (int i = threadIdx.x; i < kLTiles; i += blockDim.x) scnt[i] = 0;
    __syncthreads();
    for (int64_t i = blk.y + threadIdx.x; i < blk.z; i += blockDim.x) {
        const int64_t q = a.p0 + i;
        atomicAdd(&scnt[large_tile_of(cc, a.x[q], a.y[q])], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLTiles; i += blockDim.x) {
        sbase[i] = scnt[i] ? atomicAdd(&a.tile_cur[cl * kLTiles + i], scnt[i]) : 0;
        scnt[i] = 0;
    }
    __syncthreads();
    for (int64_t i = blk.y + threadIdx.x; i < blk.z; i += blockDim.x) {
        const int64_t q = a.p0 + i;
        const float px = a.x[q], py = a.y[q];
        const int t = large_tile_of(cc, px, py);
        const int slot = sbase[t] + atomicAdd(&scnt[t], 1);
        a.rec[slot] = make_float4(px, py, a.h[q], a.w[q]);
    }
}

// 4. spread one (cell, tile): fixed point in shared memory, then added to the global fine grid
template <int W>
struct LargeTileCfg {
    static constexpr int HS = W / 2 + 2;                   // halo per side
    static constexpr int TS = kLT + 2 * HS;                // tile rows / columns used
    static constexpr int TSTR = TS | 1;                    // odd row stride
};

template <int W, int J = 0, int I = 0>
__device__ __forceinline__ void tile_taps(unsigned addr, const float (&kx)[W], const float (&ky)[W], float c) {
    constexpr int S = LargeTileCfg<W>::TSTR;
    if constexpr (J < W) {
        if constexpr (I < W) {
            red_smem<J * S + I>(addr, __float2int_rn((c * ky[J]) * kx[I]));
            tile_taps<W, J, I + 1>(addr, kx, ky, c);
        } else {
            tile_taps<W, J + 1, 0>(addr, kx, ky, c);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256) large_spread_kernel(const __grid_constant__ LargeArgs a) {
    using TC = LargeTileCfg<W>;
    __shared__ int tile[TC::TS * TC::TSTR];
    __shared__ CellConst scc;
    const int cl = blockIdx.x / kLTiles, t = blockIdx.x % kLTiles, cell = a.cell0 + cl;
    const int tx0 = (t % (kLNF / kLT)) * kLT - TC::HS, ty0 = (t / (kLNF / kLT)) * kLT - TC::HS;
    {
        const int4* src = reinterpret_cast<const int4*>(a.cells + cell);
        int4* dst = reinterpret_cast<int4*>(&scc);
        for (int i = threadIdx.x; i < (int)(sizeof(CellConst) / 16); i += blockDim.x) dst[i] = src[i];
    }
    for (int i = threadIdx.x; i < TC::TS * TC::TSTR; i += blockDim.x) tile[i] = 0;
    __syncthreads();
    const int r0 = a.tile_off[cl * (kLTiles + 1) + t], r1 = a.tile_off[cl * (kLTiles + 1) + t + 1];
    if (r1 == r0 || !scc.valid) return;
    const float S = a.tile_abs[cl * kLTiles + t];
    const float scale = S > 0x1p-96f ? 0x1p30f * (1.0f - 0x1p-8f) / S : 0x1p126f;
    const FastFrame ff = fast_frame(scc);
    const unsigned taddr = (unsigned)__cvta_generic_to_shared(tile);
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const float4 s = a.rec[i];
        int nx, ny;
        float kx[W], ky[W];
        if (!prep_f32<kLNF, W>(ff, scc.edge, scc, a.poly, s.x, s.y, nx, ny, kx, ky, a.status)) continue;
        const float c = s.w * s.z * ff.inv_area * scale;
        if (!isfinite(c)) {
            atomicOr(a.status, ST_NONFINITE);
            continue;
        }
        const int lx = nx - tx0, ly = ny - ty0;   // inside [0, TS - W] by the halo
        if (lx < 0 || ly < 0 || lx > TC::TS - W || ly > TC::TS - W) {
            atomicOr(a.status, ST_BADCELL);   // cannot happen for samples binned by this cell's frame
            continue;
        }
        tile_taps<W>(taddr + 4u * (unsigned)(ly * TC::TSTR + lx), kx, ky, c);
    }
    __syncthreads();
    const float inv = 1.0f / scale;
    float* g = a.grid + (size_t)cl * kLNF * kLNF;
    for (int i = threadIdx.x; i < TC::TS * TC::TS; i += blockDim.x) {
        const int ly = i / TC::TS, lx = i % TC::TS;
        const int v = tile[ly * TC::TSTR + lx];
        if (v) atomicAdd(g + ((ty0 + ly) & (kLNF - 1)) * kLNF + ((tx0 + lx) & (kLNF - 1)), (float)v * inv);
    }
}

// 5. per-cell 256 x 256 FFT, deconvolution/crop, EMS ranking
// spectrum accessor on the half spectrum C1[k][m] (m = 0..P/2) with the deconvolution applied
struct LargeHalfSpec {
    const cplx<float>* c1;
    const float* inv;
    int c1s, half;
    __device__ __forceinline__ cplx<float> get(int m, int n) const {
        const float f = inv[m < 0 ? -m : m] * inv[n < 0 ? -n : n];
        if (m >= 0) {
            const cplx<float> z = c1[((n + kLNF) & (kLNF - 1)) * c1s + m];
            return {z.re * f, z.im * f};
        }
        const cplx<float> z = c1[((-n + kLNF) & (kLNF - 1)) * c1s - m];
        return {z.re * f, -z.im * f};
    }
};


static __global__ void __launch_bounds__(kLFftThreads) large_fft_kernel(const __grid_constant__ LargeFftArgs a) {
    constexpr int N1 = FftSplit<kLNF>::N1, N2 = FftSplit<kLNF>::N2;   // 16 x 16
    extern __shared__ __align__(16) unsigned char smem[];
    const int P = a.P, half = P / 2, C1S = half + 1;
    cplx<float>* c1 = reinterpret_cast<cplx<float>*>(smem);
    float* rows = reinterpret_cast<float*>(c1 + (size_t)kLNF * C1S);
    cplx<float>* stw = reinterpret_cast<cplx<float>*>(rows + 2 * kLRowPairs * kLRowStride);
    float* sinv = reinterpret_cast<float*>(stw + kLNF);
    const int tid = threadIdx.x, lane = tid & 31, team = tid / N2, tl = tid % N2;
    const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
    for (int i = tid; i < kLNF; i += kLFftThreads) stw[i] = a.twiddle[i];
    for (int i = tid; i <= half; i += kLFftThreads) sinv[i] = a.inv_phi[i];
    for (int cl = blockIdx.x; cl < a.ncells; cl += gridDim.x) {
        const int cell = a.cell0 + cl;
        const float* g = a.grid + (size_t)cl * kLNF * kLNF;
        // ---- rows, in rounds of kLRowPairs pairs
        for (int rp0 = 0; rp0 < kLNF / 2; rp0 += kLRowPairs) {
            __syncthreads();
            for (int i = tid; i < 2 * kLRowPairs * (kLNF / 4); i += kLFftThreads) {
                const int r = i / (kLNF / 4), c4 = i % (kLNF / 4);
                const float4 v = reinterpret_cast<const float4*>(g + (size_t)(2 * rp0 + r) * kLNF)[c4];
                reinterpret_cast<float4*>(rows + r * kLRowStride)[c4] = v;
            }
            __syncthreads();
            if (team < kLRowPairs) {
                float* r0 = rows + (2 * team) * kLRowStride;
                float* r1 = r0 + kLRowStride;
                team_fft<N1, N2, float>(RowPairAcc<float>{r0, r1}, RowPairAcc<float>{r0, r1}, RowPairAcc<float>{r0, r1}, tl,
                                        stw, tmask);
                const int y0 = 2 * (rp0 + team);
                for (int m = tl; m <= half; m += N2) {
                    const int mn = (kLNF - m) & (kLNF - 1);
                    const float zr = r0[m], zi = r1[m], wr = r0[mn], wi = r1[mn];
                    c1[y0 * C1S + m] = cplx<float>{0.5f * (zr + wr), 0.5f * (zi - wi)};
                    c1[(y0 + 1) * C1S + m] = cplx<float>{0.5f * (zi + wi), 0.5f * (wr - zr)};
                }
            }
        }
        __syncthreads();
        // ---- columns m = 0..P/2 in place (workspace in the row buffer)
        for (int m0 = 0; m0 <= half; m0 += kLFftThreads / N2) {
            const int m = m0 + team;
            if (m <= half) {
                cplx<float>* wk = reinterpret_cast<cplx<float>*>(rows) + (size_t)team * team_ws<N1, N2>();
                team_fft<N1, N2, float>(StridedAcc<float, false>{c1 + m, C1S}, PlainAcc<float>{wk},
                                        StridedAcc<float, false>{c1 + m, C1S}, tl, stw, tmask);
            }
            __syncthreads();
        }
        // ---- deconvolve, crop, coalesced rows of the output
        const LargeHalfSpec spec{c1, sinv, C1S, half};
        float2* out = reinterpret_cast<float2*>(a.coeffs + (size_t)cell * P * P * 2);
        for (int i = tid; i < P * P; i += kLFftThreads) {
            const int n = i / P - half, m = i % P - half;
            const cplx<float> v = spec.get(m, n);
            out[i] = make_float2(v.re, v.im);
        }
        if (a.do_ems) ems_rank_block<float, 16>(spec, P, cell, a.ems, a.ems_out, reinterpret_cast<unsigned char*>(rows));
    }
}

}  // namespace enufft
