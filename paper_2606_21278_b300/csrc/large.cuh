// large.cuh -- the type-1 transform for fine grids too large for one block's shared memory
// (n_f = 256, P up to 128): a sorted-by-subgrid pipeline over batches of cells.
//
//   1. sort     per block of up to 4096 consecutive samples of one cell: the LT x LT tile of the
//               fine grid holding each sample's centre node (LT = 16, 32 or 64, chosen per plan), a counting sort by tile inside the
//               block's own range of the record buffer (16-byte records {x, y, h, w}), the tile
//               offsets of the block and its per-tile sums of |w h| / |D|;
//   2. scale    one warp per cell: the bound B of its fine grid's nodes and the grid's scale 2^k;
//   3. spread   one block per (work item, tile), a work item being a cell or, for cells of more than
//               2^18 samples, an interleaved part of its sort blocks (work items largest cell first):
//               S = the sum of the item's sort blocks' per-tile sums bounds every node of its tile; each
//               warp takes the tile's segment of one sort block at a time and spreads its records into a shared (LT + 2 halo)^2 tile in 32-bit fixed
//               point at the item's own scale 2^30 (1 - 2^-8) / S; the tile is then added to the
//               cell's fine grid in global memory (periodic wrap) in 64-bit fixed point at one scale
//               per cell, 2^k with 2^61 / 2^k >= sum of the cell's per-tile sums (a bound of every
//               node, taken in a fixed order by the scale kernel), by red.global.add.u64: integer adds
//               do not depend on the order in which the tiles arrive, so reruns are bit-identical;
//   4. fft      one block per cell: row pairs through shared memory in rounds (team FFTs of
//               length 256), the P/2 + 1 needed columns in place, deconvolution/crop written as
//               coalesced rows of the output, and the EMS ranking read straight from the
//               half spectrum.
// The window test, the coordinates and the kernel of step 3 are those of the fused kernel
// (forward.cuh), so both routes compute the same sum.
#pragma once

#include "forward.cuh"
#include "large_args.cuh"

#ifndef ENUFFT_LSPREAD_MINB
#define ENUFFT_LSPREAD_MINB 5   // co-resident tile-spread blocks per SM the register budget is sized for
#endif

namespace enufft {

// tile of a sample from a plain binary32 evaluation of its grid coordinate (only used to sort:
// the exact coordinates are recomputed in step 4, and the tile halo absorbs a one-node difference)
template <int LT>
__device__ __forceinline__ int large_tile_of(const CellConst& cc, float px, float py) {
    const float sx = (px - cc.cxh) * cc.sch + 0.5f * kLNF, sy = (py - cc.cyh) * cc.sch + 0.5f * kLNF;
    int tx = (int)floorf(sx) / LT, ty = (int)floorf(sy) / LT;
    tx = tx < 0 ? 0 : (tx > kLNF / LT - 1 ? kLNF / LT - 1 : tx);
    ty = ty < 0 ? 0 : (ty > kLNF / LT - 1 ? kLNF / LT - 1 : ty);
    if (!(sx == sx) || !(sy == sy)) { tx = 0; ty = 0; }
    return ty * (kLNF / LT) + tx;
}

// 1. counting sort of one block's samples by tile (per-warp histograms, then a tile-major,
// warp-minor prefix), records written inside the block's own range
// Bank class of a sample in the spread's shared tile: the word of its first node modulo 32, from the
// same plain binary32 coordinate as large_tile_of (only an ordering hint: a node off by one moves
// the sample to another class, never to another result).
template <int LT>
__device__ __forceinline__ int large_class_of(const CellConst& cc, int tile, int W, float px, float py) {
    const int hs = W / 2 + 2, tstr = (LT + 2 * hs) | 1;
    const float sx = (px - cc.cxh) * cc.sch + 0.5f * kLNF, sy = (py - cc.cyh) * cc.sch + 0.5f * kLNF;
    const int r0x = (int)ceilf(sx - 0.5f * W), r0y = (int)ceilf(sy - 0.5f * W);
    const int lx = r0x - ((tile % (kLNF / LT)) * LT - hs), ly = r0y - ((tile / (kLNF / LT)) * LT - hs);
    return (ly * tstr + lx) & 31;
}

template <int LT>
__global__ void __launch_bounds__(kLSortThreads, LT >= 32 ? 2 : 1) large_sort_kernel(const __grid_constant__ LargeArgs a) {
    constexpr int NT = kLSortThreads, PER = kLBinBlock / NT, NW = NT / 32, TT = large_tiles(LT);
    // Inside each tile segment the records are written in rounds: round k holds the k-th record of
    // every bank class present, classes ascending, so the 32 consecutive records one warp
    // instruction of the spread takes mostly lie in different banks (IL; the first KM rounds, the
    // rest after them).  The per-tile |c| sums keep the tile-major, warp-minor order.  Only the
    // 64-node tiles take it: their segments (about 256 records of a sort block) fill the rounds,
    // while the 64-record segments of 32-node tiles leave most rounds short (measured: 27.2 ms per
    // step with 64-node tiles against 28.5 before; 32-node tiles 28.5 against 27.8 without it).
    constexpr bool IL = LT >= 64;
    constexpr int KM = 16;
    __shared__ int hist[NW][TT];
    __shared__ int toff[TT + 1];
    __shared__ float cabs[kLBinBlock];   // |w h| / |D| in tile-major, warp-minor order
    __shared__ int hc[IL ? TT * 32 : 1];                 // records per (tile, class)
    __shared__ unsigned rmask[IL ? TT * KM : 1];         // classes present in round k of tile t
    __shared__ int rstart[IL ? TT * (KM + 1) : 1];       // first position of round k in tile t
    __shared__ int ovf[IL ? TT : 1];                     // records of tile t beyond round KM so far
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int4 blk = a.blocks[blockIdx.x];
    const CellConst& cc = a.cells[a.cell0 + blk.x];
    for (int i = tid; i < NW * TT; i += NT) (&hist[0][0])[i] = 0;
    if constexpr (IL) {
        for (int i = tid; i < TT * 32; i += NT) hc[i] = 0;
        for (int i = tid; i < TT; i += NT) ovf[i] = 0;
    }
    __syncthreads();
    float4 s[PER];
    int tl[PER], rk[PER], kc[PER];   // tile; rank inside (warp, tile); rank inside (tile, class) << 5 | class
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int v = blk.y + tid + NT * i;
        tl[i] = -1;
        if (v < blk.z) {
            const int64_t q = a.p0 + v;
            s[i] = make_float4(a.x[q], a.y[q], a.h[q], a.w[q]);
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        if (blk.y + tid + NT * i < blk.z) {
            tl[i] = large_tile_of<LT>(cc, s[i].x, s[i].y);
            rk[i] = atomicAdd(&hist[warp][tl[i]], 1);
            if constexpr (IL) {
                const int c = large_class_of<LT>(cc, tl[i], a.W, s[i].x, s[i].y);
                kc[i] = (atomicAdd(&hc[tl[i] * 32 + c], 1) << 5) | c;
            }
        }
    }
    __syncthreads();
    if constexpr (IL) {   // round tables: one warp per tile, lane = class
        for (int t = warp; t < TT; t += NW) {
            const int c = hc[t * 32 + lane];
            int run = 0;
#pragma unroll 1
            for (int k = 0; k < KM; ++k) {
                const unsigned m = __ballot_sync(0xffffffffu, c > k);
                if (lane == 0) {
                    rmask[t * KM + k] = m;
                    rstart[t * (KM + 1) + k] = run;
                }
                run += __popc(m);
            }
            if (lane == 0) rstart[t * (KM + 1) + KM] = run;
        }
    }
    if (tid < TT) {   // per tile: warp bases, then the tile's count
        int run = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int c = hist[w][tid];
            hist[w][tid] = run;
            run += c;
        }
        toff[tid] = run;
    }
    __syncthreads();
    if (warp == 0) {       // exclusive scan of the tile counts, PL per lane
        constexpr int PL = TT >= 32 ? TT / 32 : 1;
        int c[PL], sum = 0;
#pragma unroll
        for (int i = 0; i < PL; ++i) {
            const int tt = PL * lane + i;
            c[i] = tt < TT ? toff[tt] : 0;
            sum += c[i];
        }
        int v = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        int run = v - sum;
        __syncwarp();
        int* bo = a.blk_off + (size_t)blockIdx.x * (TT + 1);
#pragma unroll
        for (int i = 0; i < PL; ++i) {
            const int tt = PL * lane + i;
            if (tt < TT) {
                toff[tt] = run;
                bo[tt] = run;
            }
            run += c[i];
        }
        if (lane == 31) {
            toff[TT] = v;
            bo[TT] = v;
        }
    }
    __syncthreads();
    const float inv_area = cc.inv_area;
#pragma unroll
    for (int i = 0; i < PER; ++i)
        if (tl[i] >= 0) {
            const int t = tl[i], slot = toff[t] + hist[warp][t] + rk[i];
            int pos = slot;
            if constexpr (IL) {
                const int k = kc[i] >> 5, c = kc[i] & 31;
                pos = toff[t] + (k < KM ? rstart[t * (KM + 1) + k] + __popc(rmask[t * KM + k] & ((1u << c) - 1u))
                                        : rstart[t * (KM + 1) + KM] + atomicAdd(&ovf[t], 1));
            }
            a.rec[blk.y + pos] = s[i];
            const float v = fabsf(s[i].w * s[i].z) * inv_area;
            cabs[slot] = (v <= 3.0e38f) ? v : 0.0f;
        }
    __syncthreads();
    // per-tile sums over the tile's contiguous slots, eight threads per tile
    for (int t0 = 0; t0 < TT; t0 += NT / 8) {
        const int t = t0 + (tid >> 3), sub = tid & 7;
        float sum = 0.0f;
        if (t < TT)
            for (int i = toff[t] + sub; i < toff[t + 1]; i += 8) sum += cabs[i];
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        sum += __shfl_xor_sync(0xffffffffu, sum, 4);
        if (sub == 0 && t < TT) a.blk_abs[(size_t)blockIdx.x * TT + t] = sum;
    }
}

// 3. spread one (cell, tile): fixed point in shared memory, then added to the global fine grid
template <int W, int LT>
struct LargeTileCfg {
    static constexpr int HS = W / 2 + 2;                   // halo per side
    static constexpr int TS = LT + 2 * HS;                // tile rows / columns used
    static constexpr int TSTR = TS | 1;                    // odd row stride
};

template <int W, int LT, int J = 0, int I = 0>
__device__ __forceinline__ void tile_taps(unsigned addr, const float (&kx)[W], const float (&ky)[W], float c) {
    constexpr int S = LargeTileCfg<W, LT>::TSTR;
    if constexpr (J < W) {
        if constexpr (I < W) {
            red_smem<J * S + I>(addr, __float2int_rn((c * ky[J]) * kx[I]));
            tile_taps<W, LT, J, I + 1>(addr, kx, ky, c);
        } else {
            tile_taps<W, LT, J + 1, 0>(addr, kx, ky, c);
        }
    }
}

template <int W, int LT>
__global__ void __launch_bounds__(kLSpreadThreads, ENUFFT_LSPREAD_MINB) large_spread_kernel(const __grid_constant__ LargeArgs a) {
    using TC = LargeTileCfg<W, LT>;
    constexpr int NT = kLSpreadThreads, NW = NT / 32, TT = large_tiles(LT);
    __shared__ int tile[TC::TS * TC::TSTR];
    __shared__ CellConst scc;
    __shared__ float fsum[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int4 wk = a.work[blockIdx.x / TT];
    const int cl = wk.x, t = blockIdx.x % TT, cell = a.cell0 + cl;
    const int tx0 = (t % (kLNF / LT)) * LT - TC::HS, ty0 = (t / (kLNF / LT)) * LT - TC::HS;
    {
        const int4* src = reinterpret_cast<const int4*>(a.cells + cell);
        int4* dst = reinterpret_cast<int4*>(&scc);
        for (int i = tid; i < (int)(sizeof(CellConst) / 16); i += NT) dst[i] = src[i];
    }
    for (int i = tid; i < TC::TS * TC::TSTR; i += NT) tile[i] = 0;
    const int2 cb = a.cell_blocks[cl];
    // S: the sum of this part's sort blocks' sums for this tile (fixed order per thread, then the
    // warps) bounds every node of the part's tile
    float s = 0.0f;
    for (int j = wk.y + wk.z * tid; j < cb.y; j += wk.z * NT) s += a.blk_abs[(size_t)(cb.x + j) * TT + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) fsum[warp] = s;
    __syncthreads();
    float S = 0.0f;
#pragma unroll
    for (int i = 0; i < NW; ++i) S += fsum[i];
    if (!scc.valid || !(S > 0.0f)) return;   // uniform across the block: nothing to spread
    const float scale = S > 0x1p-96f ? 0x1p30f * (1.0f - 0x1p-8f) / S : 0x1p126f;
    const FastFrame ff = fast_frame(scc);
    const unsigned taddr = (unsigned)__cvta_generic_to_shared(tile);
    // one sort block's segment of this tile per warp at a time (this part's sort blocks: j = part
    // mod parts); the next record is loaded before the current one is spread
    for (int j = wk.y + wk.z * warp; j < cb.y; j += wk.z * NW) {
        const int b = cb.x + j;
        const int* bo = a.blk_off + (size_t)b * (TT + 1);
        const int base = a.blocks[b].y;
        const int r1 = base + bo[t + 1];
        int r = base + bo[t] + lane;
        float4 cur = r < r1 ? a.rec[r] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (; r < r1; r += 32) {
            const float4 nxt = r + 32 < r1 ? a.rec[r + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
            int nx, ny;
            float kx[W], ky[W];
            if (prep_f32<kLNF, W>(ff, scc.edge, scc, a.poly, cur.x, cur.y, nx, ny, kx, ky, a.status)) {
                const float c = cur.w * cur.z * ff.inv_area * scale;
                if (!isfinite(c)) {
                    atomicOr(a.status, ST_NONFINITE);
                } else {
                    const int lx = nx - tx0, ly = ny - ty0;   // inside [0, TS - W] by the halo
                    if (lx < 0 || ly < 0 || lx > TC::TS - W || ly > TC::TS - W)
                        atomicOr(a.status, ST_BADCELL);   // cannot happen for samples sorted by this cell's frame
                    else
                        tile_taps<W, LT>(taddr + 4u * (unsigned)(ly * TC::TSTR + lx), kx, ky, c);
                }
            }
            cur = nxt;
        }
    }
    __syncthreads();
    // tile integers at this item's scale -> the cell's 64-bit fixed point: a binary32 product (the
    // precision binary32 accumulation had), rounded to an integer; every value below 2^61
    const float conv = (float)(ldexp(1.0, a.cell_exp[cl]) / (double)scale);
    unsigned long long* g = a.grid + (size_t)cl * kLNF * kLNF;
    for (int i = tid; i < TC::TS * TC::TS; i += NT) {
        const int ly = i / TC::TS, lx = i % TC::TS;
        const int v = tile[ly * TC::TSTR + lx];
        if (v)
            atomicAdd(g + ((ty0 + ly) & (kLNF - 1)) * kLNF + ((tx0 + lx) & (kLNF - 1)),
                      (unsigned long long)__float2ll_rn(__fmul_rn((float)v, conv)));
    }
}

// 2. the scale of each batch cell's fixed-point grid: B = sum over its sort blocks and tiles of
// the per-tile |c| sums, in a fixed order (lane-strided partial sums, then a fixed shuffle tree),
// and k = 61 - e for B < 2^e, so the grid's integers stay below 2^61 (B is accurate to far better
// than the factor 2 left to 2^62); one warp per cell
constexpr int kLScaleThreads = 256;
template <int LT>
__global__ void __launch_bounds__(kLScaleThreads) large_scale_kernel(const __grid_constant__ LargeArgs a) {
    constexpr int TT = large_tiles(LT);
    const int lane = threadIdx.x & 31;
    const int cl = blockIdx.x * (kLScaleThreads / 32) + (threadIdx.x >> 5);
    if (cl >= a.ncells) return;
    const int2 cb = a.cell_blocks[cl];
    float s = 0.0f;
    for (int i = lane; i < cb.y * TT; i += 32) s += a.blk_abs[(size_t)cb.x * TT + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        int e = 0;
        if (s > 0.0f && isfinite(s)) frexpf(s, &e);
        a.cell_exp[cl] = 61 - e;
    }
}

// fixed-point grid value -> binary32: the integer rounded to binary32, times 2^-k (fs, exact while
// 2^-k is a normal binary32; outside that range the product is taken in binary64)
__device__ __forceinline__ float large_grid_value(long long v, int k, float fs) {
    if (k >= -126 && k <= 126) return __fmul_rn(__ll2float_rn(v), fs);
    return (float)__dmul_rn(__ll2double_rn(v), ldexp(1.0, -k));
}

// 4. per-cell 256 x 256 FFT, deconvolution/crop, EMS ranking
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
        const long long* g = a.grid + (size_t)cl * kLNF * kLNF;
        const int kexp = a.cell_exp[cl];
        const float fs = (kexp >= -126 && kexp <= 126) ? __int_as_float((127 - kexp) << 23) : 0.0f;
        // ---- rows, in rounds of kLRowPairs pairs
        for (int rp0 = 0; rp0 < kLNF / 2; rp0 += kLRowPairs) {
            __syncthreads();
            for (int i = tid; i < 2 * kLRowPairs * (kLNF / 4); i += kLFftThreads) {
                const int r = i / (kLNF / 4), c4 = i % (kLNF / 4);
                const longlong2* src = reinterpret_cast<const longlong2*>(g + (size_t)(2 * rp0 + r) * kLNF) + 2 * c4;
                const longlong2 u0 = src[0], u1 = src[1];
                reinterpret_cast<float4*>(rows + r * kLRowStride)[c4] =
                    make_float4(large_grid_value(u0.x, kexp, fs), large_grid_value(u0.y, kexp, fs),
                                large_grid_value(u1.x, kexp, fs), large_grid_value(u1.y, kexp, fs));
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
