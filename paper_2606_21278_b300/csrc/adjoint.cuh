// adjoint.cuh -- adjoint of the per-cell type-1 transform (a type-2 NUFFT), fused per cell.
//
// For G = dL/dRe(h_mn) + i dL/dIm(h_mn) the gradient of a real loss with respect to the scaled
// samples c_q = w_q h_q / |D| is  v_q = Re sum_mn G_mn e^{+i (k_m x'_q + k_n y'_q)}  (the
// transpose of App. B's quadrature sum).  Writing Re(.) as half the sum with its conjugate gives
// a Hermitian spectrum F_k = (G_k + conj(G_-k)) / 2 on k in [-P/2, P/2]^2, so that
//   1. F is pre-corrected by 1 / (Phi(k_x) Phi(k_y)) (the mirror of the deconvolution),
//   2. a real n_f x n_f grid g = IFFT2(F) is formed (columns m = 0..P/2, then rows in pairs),
//   3. v_q = sum_r g_r phi(s_q - r) is interpolated with the spreading kernel (no atomics),
//   4. dL/dh_q = win_q w_q v_q / |D| and dL/dw_q = win_q h_q v_q / |D| are written.
//
// Reconstruction mode (Sec. 3.2 diagnostics): G is the cell's coefficients restricted to the
// selected mode pairs and their partners, so v_q is the truncated series h_rec (Eq. tri_series) at
// the samples; per cell the kernel also reduces the relative reconstructed RMSE
// (Eq. alps_relative_rmse) and the physical and spectral variances of Eq. spectral_variance.
#pragma once

#include "forward.cuh"

namespace enufft {

template <typename T>
struct AdjArgs {
    const T* __restrict__ x;
    const T* __restrict__ y;
    const T* __restrict__ h;
    const T* __restrict__ w;
    const T* __restrict__ gcoef;   // [n_cells][P][P] complex
    T* __restrict__ grad_h;        // may be null
    T* __restrict__ grad_w;        // may be null
    int mode;                      // 0: gradient from G; 1: reconstruction diagnostics from coefficients
    const int32_t* __restrict__ kstar;   // mode 1: selected pairs per cell
    const int32_t* __restrict__ sel;     // mode 1: [n_cells][k_max] pair indices
    int k_max;
    T* __restrict__ hrec;          // mode 1: h_rec at the samples (may be null)
    double* __restrict__ stats;    // mode 1: [n_cells][4] eps_rel, sigma2_phys, sigma2_spec(set), sigma2_spec(box)
    const int64_t* __restrict__ offsets;
    const CellConst* __restrict__ cells;
    const int* __restrict__ order;
    int n_work;
    int P;
    unsigned* ticket;
    unsigned* status;
    const cplx<T>* __restrict__ twiddle;
    T inv_phi[kMaxHalf + 1];
    KernelPoly poly;
    double beta;
};

template <int W, int GS, int J = 0, int I = 0>
__device__ __forceinline__ float gather_taps(const float* __restrict__ g, const float (&kx)[W], const float (&ky)[W],
                                             float acc_row, float acc) {
    if constexpr (J < W) {
        if constexpr (I < W) {
            return gather_taps<W, GS, J, I + 1>(g, kx, ky, __fmaf_rn(kx[I], g[J * GS + I], acc_row), acc);
        } else {
            return gather_taps<W, GS, J + 1, 0>(g, kx, ky, 0.0f, __fmaf_rn(ky[J], acc_row, acc));
        }
    } else {
        return acc;
    }
}

// block-wide sums of two doubles (every thread calls; thread 0 receives the totals); scratch holds
// 2 doubles per warp
__device__ __forceinline__ void block_sum2(double& u, double& v, double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    if (lane == 0) {
        scratch[2 * warp] = u;
        scratch[2 * warp + 1] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u = 0.0;
        v = 0.0;
        for (int i = 0; i < nw; ++i) {
            u += scratch[2 * i];
            v += scratch[2 * i + 1];
        }
    }
    __syncthreads();
}

template <typename T, int NF, int W>
__global__ void __launch_bounds__(FwdCfg<T, NF, W>::NT, FwdCfg<T, NF, W>::MINB)
type1_adjoint_kernel(const __grid_constant__ AdjArgs<T> a) {
    using CF = FwdCfg<T, NF, W>;
    constexpr int GS = CF::GS, GR = CF::GR, HO = CF::HO, N1 = CF::N1, N2 = CF::N2;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sgrid = reinterpret_cast<T*>(smem);
    cplx<T>* sC1 = reinterpret_cast<cplx<T>*>(smem + CF::grid_bytes);
    cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem + CF::grid_bytes + CF::c1_bytes);
    CellConst* scc = reinterpret_cast<CellConst*>(smem + CF::grid_bytes + CF::c1_bytes + CF::tw_bytes);
    int* sticket = reinterpret_cast<int*>(scc + 1);
    T* sinv = reinterpret_cast<T*>(sticket + 4);

    const int tid = threadIdx.x, lane = tid & 31;
    const int P = a.P, half = P / 2, C1S = half + 1;
    for (int i = tid; i < NF; i += CF::NT) stw[i] = a.twiddle[i];
    for (int i = tid; i <= half; i += CF::NT) sinv[i] = a.inv_phi[i];

    for (;;) {
        if (tid == 0) *sticket = (int)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int tk = *sticket;
        if (tk >= a.n_work) break;
        const int cell = a.order[tk];
        cplx<T>* stage = reinterpret_cast<cplx<T>*>(sgrid);
        {   // per-cell constants; G of this cell into the staging area (coalesced 16-byte loads)
            const int4* src = reinterpret_cast<const int4*>(a.cells + cell);
            int4* dst = reinterpret_cast<int4*>(scc);
            for (int i = tid; i < (int)(sizeof(CellConst) / 16); i += CF::NT) dst[i] = src[i];
            const float4* s4 = reinterpret_cast<const float4*>(a.gcoef + (size_t)cell * P * P * 2);
            float4* d4 = reinterpret_cast<float4*>(stage);
            const int n4 = P * P * (int)sizeof(cplx<T>) / 16;
            if (a.mode == 0)
                for (int i = tid; i < n4; i += CF::NT) d4[i] = s4[i];
            else
                for (int i = tid; i < n4; i += CF::NT) d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        double spec_set = 0.0, spec_all = 0.0;   // mode 1, block totals in thread 0
        if (a.mode == 1) {
            // the selected pairs and their partners; sigma2_spec over them and over the box (no DC)
            const cplx<T>* cf = reinterpret_cast<const cplx<T>*>(a.gcoef) + (size_t)cell * P * P;
            const int dcp = half * P + half;
            for (int i = tid; i < P * P; i += CF::NT)
                if (i != dcp) spec_all += (double)cf[i].re * cf[i].re + (double)cf[i].im * cf[i].im;
            int K = a.kstar[cell];
            K = K < 0 ? 0 : (K > a.k_max ? a.k_max : K);
            for (int k = tid; k < K; k += CF::NT) {
                const int p = a.sel[(size_t)cell * a.k_max + k];
                if (p < 0 || p >= P * P) continue;
                const int n = p / P - half, m = p % P - half;
                const int nn = half - n, mm = half - m;   // partner (-m, -n) in box coordinates
                stage[p] = cf[p];
                if (p != dcp) spec_set += (double)cf[p].re * cf[p].re + (double)cf[p].im * cf[p].im;
                if (nn >= 0 && nn < P && mm >= 0 && mm < P && nn * P + mm != p) {
                    const int pp = nn * P + mm;
                    stage[pp] = cf[pp];
                    spec_set += (double)cf[pp].re * cf[pp].re + (double)cf[pp].im * cf[pp].im;
                }
            }
            block_sum2(spec_set, spec_all, reinterpret_cast<double*>(sC1));
        }
        // ---- 1. Hermitian, pre-corrected half spectrum F[n][m], m = 0..P/2, all n rows (zero padded)
        for (int i = tid; i < NF * C1S; i += CF::NT) {
            const int m = i % C1S, nr = i / C1S;            // nr = n mod n_f
            const int n = nr < NF / 2 ? nr : nr - NF;
            cplx<T> f{T(0), T(0)};
            if (n >= -half && n <= half) {
                if (m <= half - 1 && n <= half - 1) f = stage[(n + half) * P + (m + half)];
                if (m >= 1 - half && n >= 1 - half) {       // -k inside the box
                    const cplx<T> g2 = stage[(half - n) * P + (half - m)];
                    f.re += g2.re;
                    f.im -= g2.im;
                }
                const T s = T(0.5) * sinv[m] * sinv[n < 0 ? -n : n];
                f.re *= s;
                f.im *= s;
            }
            sC1[nr * C1S + m] = f;
        }
        __syncthreads();
        // ---- 2a. inverse FFT of the columns m = 0..P/2 along y
        {
            const int team = tid / N2, t = tid % N2;
            const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
            if (team <= half) {   // workspace in the grid memory (the staged G is no longer needed)
                cplx<T>* wk = reinterpret_cast<cplx<T>*>(sgrid) + (size_t)team * CF::WS_TEAM;
                team_fft<N1, N2, T>(StridedAcc<T, true>{sC1 + team, C1S}, PlainAcc<T>{wk},
                                    StridedAcc<T, true>{sC1 + team, C1S}, t, stw, tmask);
            }
        }
        __syncthreads();
        // ---- 2b. rows in pairs: Z[m] = Y_m[y0] + i Y_m[y1] over m in [-P/2, P/2], inverse FFT
        {
            const int team = tid / N2, t = tid % N2;
            const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
            if (team < NF / 2) {
                T* r0 = sgrid + (HO + 2 * team) * GS + HO;   // core columns of the row pair
                T* r1 = r0 + GS;
                const int y0 = 2 * team, y1 = y0 + 1;
                for (int k = t; k < NF; k += N2) {
                    const int m = k < NF / 2 ? k : k - NF;
                    T zr = T(0), zi = T(0);
                    if (m >= 0 && m <= half) {
                        const cplx<T> A = sC1[y0 * C1S + m], B = sC1[y1 * C1S + m];
                        zr = A.re - B.im;
                        zi = A.im + B.re;
                    } else if (m < 0 && m >= -half) {
                        const cplx<T> A = sC1[y0 * C1S - m], B = sC1[y1 * C1S - m];   // conj(A) + i conj(B)
                        zr = A.re + B.im;
                        zi = -A.im + B.re;
                    }
                    r0[k] = zr;
                    r1[k] = zi;
                }
                __syncwarp(tmask);
                team_fft<N1, N2, T>(RowPairConjAcc<T>{r0, r1}, RowPairAcc<T>{r0 - HO, r1 - HO}, RowPairConjAcc<T>{r0, r1},
                                    t, stw, tmask);
            }
        }
        __syncthreads();
        // ---- periodic halo copy (the mirror of the fold): rows first, then columns of all rows
        for (int i = tid; i < (GR - NF) * NF; i += CF::NT) {
            const int k = i / NF, c = HO + i % NF;
            const int r = k < HO ? k : k + NF;
            const int rw = k < HO ? k + NF : k;
            sgrid[r * GS + c] = sgrid[rw * GS + c];
        }
        __syncthreads();
        for (int i = tid; i < GR * (GR - NF); i += CF::NT) {
            const int r = i / (GR - NF), k = i % (GR - NF);
            const int c = k < HO ? k : k + NF;
            const int cw = k < HO ? k + NF : k;
            sgrid[r * GS + c] = sgrid[r * GS + cw];
        }
        __syncthreads();
        // ---- 3+4. interpolate at the samples and scale (mode 1: reconstruction and its sums)
        T s_err = T(0), s_h2 = T(0), s_wh2 = T(0);
        if (scc->valid) {
            const CellConst& cc = *scc;
            const FastFrame ff = fast_frame(cc);
            const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
            for (int64_t q = q0 + tid; q < q1; q += CF::NT) {
                const T px = a.x[q], py = a.y[q], ph = a.h[q], pw = a.w[q];
                int r0x, r0y;
                T v = T(0);
                bool in;
                if constexpr (sizeof(T) == 4) {
                    float kx[W], ky[W];
                    in = prep_f32<NF, W>(ff, cc.edge, cc, a.poly, px, py, r0x, r0y, kx, ky, a.status);
                    if (in) v = gather_taps<W, GS>(sgrid + (r0y + HO) * GS + (r0x + HO), kx, ky, 0.0f, 0.0f);
                } else {
                    double kx[W], ky[W];
                    in = prep_f64<NF, W>(cc, a.poly, a.beta, px, py, r0x, r0y, kx, ky, a.status);
                    if (in) {
                        const double* gp = reinterpret_cast<const double*>(sgrid) + (r0y + HO) * GS + (r0x + HO);
                        for (int j = 0; j < W; ++j) {
                            double acc = 0.0;
                            for (int i = 0; i < W; ++i) acc += kx[i] * gp[j * GS + i];
                            v += ky[j] * acc;
                        }
                    }
                }
                if (a.mode == 1) {
                    if (in) {
                        const T d = ph - v;
                        s_err += d * d;
                        s_h2 += ph * ph;
                        s_wh2 += pw * ph * ph;
                    }
                    if (a.hrec) a.hrec[q] = in ? v : T(0);
                    continue;
                }
                T gh = T(0), gw = T(0);
                if (in) {
                        if constexpr (sizeof(T) == 4) {
                        gh = pw * v * ff.inv_area;
                        gw = ph * v * ff.inv_area;
                    } else {
                        gh = pw * v / cc.area;
                        gw = ph * v / cc.area;
                    }
                }
                if (a.grad_h) a.grad_h[q] = gh;
                if (a.grad_w) a.grad_w[q] = gw;
            }
        } else {
            const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
            for (int64_t q = q0 + tid; q < q1; q += CF::NT) {
                if (a.grad_h) a.grad_h[q] = T(0);
                if (a.grad_w) a.grad_w[q] = T(0);
                if (a.hrec) a.hrec[q] = T(0);
            }
        }
        if (a.mode == 1) {
            double e2 = (double)s_err, h2 = (double)s_h2, wh2 = (double)s_wh2, dummy = 0.0;
            double* scratch = reinterpret_cast<double*>(sC1);   // the column workspace is free here
            block_sum2(e2, h2, scratch);
            block_sum2(wh2, dummy, scratch);
            if (tid == 0) {
                double* st = a.stats + 4 * (size_t)cell;
                st[0] = h2 > 0.0 ? sqrt(e2 / h2) : 0.0;
                st[1] = scc->valid ? wh2 / scc->area : 0.0;
                st[2] = spec_set;
                st[3] = spec_all;
            }
        }
    }
}

}  // namespace enufft
