// large_adj.cuh -- adjoint (type-2) of the n_f = 256 route, and its reconstruction mode.
//
// The mirror of large.cuh in two kernels per batch of cells (the fine grid does not fit one block's
// shared memory), with the same Hermitian half spectrum as the fused adjoint (adjoint.cuh):
//   1. fft     one block per cell: F_k = (G_k + conj(G_-k)) / 2 pre-corrected by 1 / (Phi(k_x)
//              Phi(k_y)) on the half spectrum m = 0..P/2 in shared memory, the inverse transforms of
//              those columns, then of the rows in pairs in rounds, each real row pair written to the
//              cell's binary32 fine grid in global memory.  Reconstruction mode builds G from the
//              cell's coefficients restricted to its EMS selection (each selected pair and its
//              partner) and also sums the spectral variances over that set and over the box.
//   2. interp  one block per work item (a cell, or a contiguous part of a large cell): the grid
//              is staged in two overlapping windows of 134 rows (with a column halo), and every
//              sample is interpolated in the pass whose window holds its kernel footprint
//              (v_q = sum_r g_r phi(s_q - r), no atomics); then dL/dh_q = win_q w_q v_q / |D| and
//              dL/dw_q = win_q h_q v_q / |D|, or h_rec(x_q) = v_q with per-item partial sums of the
//              reconstruction diagnostics, added per cell in a fixed order by a third kernel.
#pragma once

#include "adjoint.cuh"
#include "large.cuh"

namespace enufft {

constexpr int kLAdjThreads = 512;
constexpr int kLWinRows = kLNF / 2 + 8;        // rows of one interpolation window (w <= 8)
constexpr int kLWinCols = kLNF + 8;            // columns with a periodic halo
constexpr int kLWinShift = 4;                  // the window's first column is -kLWinShift

struct LargeAdjFftArgs {
    const float* __restrict__ gcoef;     // [n_cells][P][P] complex: G, or the coefficients (mode 1)
    int mode;                            // 0 gradient, 1 reconstruction
    const int32_t* __restrict__ kstar;   // mode 1
    const int32_t* __restrict__ sel;     // mode 1: [n_cells][k_max]
    int k_max;
    int cell0, ncells, P;
    float* __restrict__ grid;            // [ncells][256][256] binary32 fine grids of the batch
    double* __restrict__ spec;           // mode 1: [n_cells][2] spectral variance over the set and the box
    const cplx<float>* __restrict__ twiddle;
    float inv_phi[kMaxHalfL + 1];
};

struct LargeInterpArgs {
    const float* __restrict__ x;
    const float* __restrict__ y;
    const float* __restrict__ h;
    const float* __restrict__ w;
    const int64_t* __restrict__ offsets;
    const CellConst* __restrict__ cells;
    const int4* __restrict__ work;       // {cell - cell0, part, parts, 0}
    int cell0;
    const float* __restrict__ grid;      // batch fine grids
    int mode;
    float* __restrict__ grad_h;          // mode 0 (may be null)
    float* __restrict__ grad_w;          // mode 0 (may be null)
    float* __restrict__ hrec;            // mode 1 (may be null)
    double* __restrict__ partial;        // mode 1: [work item][3] sum (h - h_rec)^2, sum h^2, sum w h^2
    unsigned* status;
    KernelPoly poly;
};

__host__ __device__ constexpr size_t large_adj_fft_smem_bytes(int P) { return large_fft_smem_bytes(P); }
constexpr size_t kLInterpSmem = sizeof(float) * (size_t)kLWinRows * kLWinCols + 64;

// 1. G -> Hermitian half spectrum -> inverse column and row transforms -> global fine grid
static __global__ void __launch_bounds__(kLAdjThreads) large_adj_fft_kernel(const __grid_constant__ LargeAdjFftArgs a) {
    constexpr int N1 = FftSplit<kLNF>::N1, N2 = FftSplit<kLNF>::N2;   // 16 x 16
    extern __shared__ __align__(16) unsigned char smem[];
    const int P = a.P, half = P / 2, C1S = half + 1;
    cplx<float>* c1 = reinterpret_cast<cplx<float>*>(smem);
    float* rows = reinterpret_cast<float*>(c1 + (size_t)kLNF * C1S);
    cplx<float>* stw = reinterpret_cast<cplx<float>*>(rows + 2 * kLRowPairs * kLRowStride);
    float* sinv = reinterpret_cast<float*>(stw + kLNF);
    double* sred = reinterpret_cast<double*>(rows);   // mode 1 reductions (before the rows are used)
    const int tid = threadIdx.x, lane = tid & 31, team = tid / N2, tl = tid % N2;
    const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
    for (int i = tid; i < kLNF; i += kLAdjThreads) stw[i] = a.twiddle[i];
    for (int i = tid; i <= half; i += kLAdjThreads) sinv[i] = a.inv_phi[i];
    for (int cl = blockIdx.x; cl < a.ncells; cl += gridDim.x) {
        const int cell = a.cell0 + cl;
        const cplx<float>* G = reinterpret_cast<const cplx<float>*>(a.gcoef) + (size_t)cell * P * P;
        __syncthreads();   // the previous cell's rows and reductions are done
        if (a.mode == 0) {
            for (int i = tid; i < kLNF * C1S; i += kLAdjThreads) {
                const int m = i % C1S, nr = i / C1S;
                const int n = nr < kLNF / 2 ? nr : nr - kLNF;
                cplx<float> f{0.0f, 0.0f};
                if (n >= -half && n <= half) {
                    if (m <= half - 1 && n <= half - 1) f = G[(n + half) * P + (m + half)];
                    if (m >= 1 - half && n >= 1 - half) {   // -k inside the box
                        const cplx<float> g2 = G[(half - n) * P + (half - m)];
                        f.re += g2.re;
                        f.im -= g2.im;
                    }
                    const float s = 0.5f * sinv[m] * sinv[n < 0 ? -n : n];
                    f.re *= s;
                    f.im *= s;
                }
                c1[i] = f;
            }
        } else {
            // the selected pairs and their partners only; spectral variances (DC excluded)
            for (int i = tid; i < kLNF * C1S; i += kLAdjThreads) c1[i] = cplx<float>{0.0f, 0.0f};
            const int dcp = half * P + half;
            double sa = 0.0, ss = 0.0;
            for (int i = tid; i < P * P; i += kLAdjThreads)
                if (i != dcp) sa += (double)G[i].re * G[i].re + (double)G[i].im * G[i].im;
            int K = a.kstar[cell];
            K = K < 0 ? 0 : (K > a.k_max ? a.k_max : K);
            __syncthreads();   // zeroed half spectrum
            if (tid < 32) {    // one warp adds the (at most 2 K_max) modes, in order, to F
                for (int k = 0; k < K; ++k) {
                    const int p = a.sel[(size_t)cell * a.k_max + k];
                    if (p < 0 || p >= P * P) continue;
                    const int n0 = p / P - half, m0 = p % P - half;
                    for (int s = 0; s < 2; ++s) {
                        const int m = s ? -m0 : m0, n = s ? -n0 : n0;
                        if (s && m == m0 && n == n0) break;   // DC: its own partner
                        if (m < -half || m > half - 1 || n < -half || n > half - 1) continue;
                        const cplx<float> c = G[(n + half) * P + (m + half)];
                        if (lane == 0 && !(m == 0 && n == 0)) ss += (double)c.re * c.re + (double)c.im * c.im;
                        // G_mu adds to F[n][m] (m >= 0) and conj(G_mu) to F[-n][-m] (m <= 0), with the
                        // same pre-correction as above
                        if (lane == 0 && m >= 0) {
                            const float f = 0.5f * sinv[m] * sinv[n < 0 ? -n : n];
                            cplx<float>& d = c1[((n + kLNF) & (kLNF - 1)) * C1S + m];
                            d.re += c.re * f;
                            d.im += c.im * f;
                        }
                        if (lane == 0 && m <= 0) {
                            const float f = 0.5f * sinv[-m] * sinv[n < 0 ? -n : n];
                            cplx<float>& d = c1[((-n + kLNF) & (kLNF - 1)) * C1S - m];
                            d.re += c.re * f;
                            d.im -= c.im * f;
                        }
                    }
                }
            }
            block_sum2(ss, sa, sred);
            if (tid == 0) {
                a.spec[2 * (size_t)cell] = ss;
                a.spec[2 * (size_t)cell + 1] = sa;
            }
        }
        __syncthreads();
        // ---- inverse transforms of the columns m = 0..P/2 along y (workspace in the row buffer)
        for (int m0 = 0; m0 <= half; m0 += kLAdjThreads / N2) {
            const int m = m0 + team;
            if (m <= half) {
                cplx<float>* wk = reinterpret_cast<cplx<float>*>(rows) + (size_t)team * team_ws<N1, N2>();
                team_fft<N1, N2, float>(StridedAcc<float, true>{c1 + m, C1S}, PlainAcc<float>{wk},
                                        StridedAcc<float, true>{c1 + m, C1S}, tl, stw, tmask);
            }
            __syncthreads();
        }
        // ---- rows in pairs: Z[m] = Y_m[y0] + i Y_m[y1] over m in [-P/2, P/2], inverse transform,
        // the two real rows to the fine grid
        float* gout = a.grid + (size_t)cl * kLNF * kLNF;
        for (int rp0 = 0; rp0 < kLNF / 2; rp0 += kLRowPairs) {
            if (team < kLRowPairs) {
                float* r0 = rows + (2 * team) * kLRowStride;
                float* r1 = r0 + kLRowStride;
                const int y0 = 2 * (rp0 + team), y1 = y0 + 1;
                for (int k = tl; k < kLNF; k += N2) {
                    const int m = k < kLNF / 2 ? k : k - kLNF;
                    float zr = 0.0f, zi = 0.0f;
                    if (m >= 0 && m <= half) {
                        const cplx<float> A = c1[y0 * C1S + m], B = c1[y1 * C1S + m];
                        zr = A.re - B.im;
                        zi = A.im + B.re;
                    } else if (m < 0 && m >= -half) {
                        const cplx<float> A = c1[y0 * C1S - m], B = c1[y1 * C1S - m];   // conj(A) + i conj(B)
                        zr = A.re + B.im;
                        zi = -A.im + B.re;
                    }
                    r0[k] = zr;
                    r1[k] = zi;
                }
                __syncwarp(tmask);
                team_fft<N1, N2, float>(RowPairConjAcc<float>{r0, r1}, RowPairAcc<float>{r0, r1},
                                        RowPairConjAcc<float>{r0, r1}, tl, stw, tmask);
            }
            __syncthreads();
            for (int i = tid; i < 2 * kLRowPairs * (kLNF / 4); i += kLAdjThreads) {
                const int r = i / (kLNF / 4), c4 = i % (kLNF / 4);
                reinterpret_cast<float4*>(gout + (size_t)(2 * rp0 + r) * kLNF)[c4] =
                    reinterpret_cast<const float4*>(rows + r * kLRowStride)[c4];
            }
            __syncthreads();
        }
    }
}

// 2. interpolation at the samples of one work item from two staged windows of the cell's grid
template <int W>
static __global__ void __launch_bounds__(kLAdjThreads, 1) large_interp_kernel(const __grid_constant__ LargeInterpArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* win = reinterpret_cast<float*>(smem);   // [kLWinRows][kLWinCols]
    double* sred = reinterpret_cast<double*>(smem);   // reductions, once the window is no longer read
    // first nodes r0 lie in [-W/2, 256 - W/2], so every footprint starts at or after column and row
    // -kLWinShift and its last row is at most 255 + ceil(W/2), inside the pass-1 window
    static_assert(W <= 2 * kLWinShift && kLNF / 2 - kLWinShift + kLWinRows >= kLNF + (W + 1) / 2,
                  "window covers every footprint");
    const int tid = threadIdx.x;
    const int4 wk = a.work[blockIdx.x];
    const int cl = wk.x, cell = a.cell0 + cl;
    const CellConst& cc = a.cells[cell];
    const int64_t c0 = a.offsets[cell], c1 = a.offsets[cell + 1];
    const int64_t len = (c1 - c0 + wk.z - 1) / wk.z;
    const int64_t q0 = c0 + (int64_t)wk.y * len, q1 = min(c1, q0 + len);
    const float* g = a.grid + (size_t)cl * kLNF * kLNF;
    const FastFrame ff = fast_frame(cc);
    float s_err = 0.0f, s_h2 = 0.0f, s_wh2 = 0.0f;
    for (int pass = 0; pass < 2; ++pass) {
        // rows rb .. rb + kLWinRows - 1 and columns -kLWinShift .. kLNF + kLWinShift - 1 (periodic)
        const int rb = pass * (kLNF / 2) - kLWinShift;
        __syncthreads();
        for (int i = tid; i < kLWinRows * kLWinCols; i += kLAdjThreads) {
            const int r = i / kLWinCols, c = i % kLWinCols;
            win[i] = g[(size_t)((rb + r) & (kLNF - 1)) * kLNF + ((c - kLWinShift) & (kLNF - 1))];
        }
        __syncthreads();
        if (!cc.valid) continue;
        for (int64_t q = q0 + tid; q < q1; q += kLAdjThreads) {
            int r0x, r0y;
            float ax, ay;
            const bool in = prep_coords_f32<kLNF, W>(ff, cc.edge, cc, a.x[q], a.y[q], r0x, r0y, ax, ay, a.status);
            // the pass whose window holds rows r0y .. r0y + W - 1
            const int mine = (r0y >= kLNF / 2 - kLWinShift) ? 1 : 0;
            if (in && mine != pass) continue;
            if (!in) {
                if (pass == 0) {
                    if (a.mode == 0) {
                        if (a.grad_h) a.grad_h[q] = 0.0f;
                        if (a.grad_w) a.grad_w[q] = 0.0f;
                    } else if (a.hrec) {
                        a.hrec[q] = 0.0f;
                    }
                }
                continue;
            }
            float kx[W], ky[W];
            kernel_pieces_sym<W>(a.poly, ax, kx);
            kernel_pieces_sym<W>(a.poly, ay, ky);
            const float* gp = win + (r0y - rb) * kLWinCols + (r0x + kLWinShift);
            const float v = gather_taps<W, kLWinCols>(gp, kx, ky, 0.0f, 0.0f);
            const float ph = a.h[q], pw = a.w[q];
            if (a.mode == 0) {
                if (a.grad_h) a.grad_h[q] = pw * v * ff.inv_area;
                if (a.grad_w) a.grad_w[q] = ph * v * ff.inv_area;
            } else {
                const float d = ph - v;
                s_err += d * d;
                s_h2 += ph * ph;
                s_wh2 += pw * ph * ph;
                if (a.hrec) a.hrec[q] = v;
            }
        }
    }
    if (!cc.valid) {   // the routes skip the cell (reported by the forward's frame check)
        for (int64_t q = q0 + tid; q < q1; q += kLAdjThreads) {
            if (a.grad_h) a.grad_h[q] = 0.0f;
            if (a.grad_w) a.grad_w[q] = 0.0f;
            if (a.hrec) a.hrec[q] = 0.0f;
        }
    }
    if (a.mode == 1) {
        double e2 = s_err, h2 = s_h2, wh2 = s_wh2, dummy = 0.0;
        __syncthreads();   // the window is no longer read
        block_sum2(e2, h2, sred);
        block_sum2(wh2, dummy, sred);
        if (tid == 0) {
            a.partial[3 * (size_t)blockIdx.x + 0] = e2;
            a.partial[3 * (size_t)blockIdx.x + 1] = h2;
            a.partial[3 * (size_t)blockIdx.x + 2] = wh2;
        }
    }
}

// 3. reconstruction diagnostics per cell from its items' partial sums, in item order
static __global__ void large_recon_stats_kernel(int cell0, int ncells, const int4* __restrict__ work, int nwork,
                                                const double* __restrict__ partial, const double* __restrict__ spec,
                                                const CellConst* __restrict__ cells, double* __restrict__ stats) {
    const int cl = blockIdx.x * blockDim.x + threadIdx.x;
    if (cl >= ncells) return;
    const int cell = cell0 + cl;
    double e2 = 0.0, h2 = 0.0, wh2 = 0.0;
    for (int i = 0; i < nwork; ++i) {
        if (work[i].x != cl) continue;
        e2 += partial[3 * (size_t)i];
        h2 += partial[3 * (size_t)i + 1];
        wh2 += partial[3 * (size_t)i + 2];
    }
    double* st = stats + 4 * (size_t)cell;
    st[0] = h2 > 0.0 ? sqrt(e2 / h2) : 0.0;
    st[1] = cells[cell].valid ? wh2 / cells[cell].area : 0.0;
    st[2] = spec[2 * (size_t)cell];
    st[3] = spec[2 * (size_t)cell + 1];
}

}  // namespace enufft
