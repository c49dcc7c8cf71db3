// forward.cuh -- fused per-cell type-1 transform (+ optional EMS) for fine grids that fit in
// shared memory (n_f = 64 or 128).
//
// One persistent thread block takes cells from an atomic ticket queue (cells ordered largest
// first) and, for each cell, runs every step of Sec. 2.1.2 on chip:
//   1. window + scale (App. A/B): centred coordinates from binary64 per-cell constants through
//      exact binary32 transforms, the mask test (binary32 with a certified margin, binary64 when
//      a sample is closer than the margin to the boundary), c_q = w_q h_q / |D|;
//   2. spread c_q with the exponential-of-semicircle kernel onto a real n_f x n_f grid held in
//      shared memory with a halo (so no per-tap wrap arithmetic), then fold the halo (periodic);
//   3. 2-D FFT: real rows in pairs (one complex FFT per pair, split by conjugate symmetry),
//      then the P/2 + 1 needed columns, each by a team of lanes (fft.cuh);
//   4. deconvolve by 1/(Phi(m) Phi(n)), crop to m, n in [-P/2, P/2) (Hermitian fill of m < 0),
//      stage the P x P spectrum in shared memory;
//   5. optionally EMS on the staged spectrum (ems.cuh), then one coalesced 16-byte-vector store.
// The grid origin is the paper's x' = u + H (App. A), so no phase correction is needed.
#pragma once

#include "common.cuh"
#include "ems.cuh"
#include "fft.cuh"

namespace enufft {

constexpr int kMaxHalf = 64;   // P/2 <= 64

template <typename T>
struct FwdArgs {
    const T* __restrict__ x;
    const T* __restrict__ y;
    const T* __restrict__ h;
    const T* __restrict__ w;
    T* __restrict__ coeffs;
    const int64_t* __restrict__ offsets;
    const CellConst* __restrict__ cells;
    const int* __restrict__ order;
    int n_work;
    int P;
    unsigned* ticket;
    unsigned* status;
    const cplx<T>* __restrict__ twiddle;   // W_nf^j, j in [0, nf)
    T inv_phi[kMaxHalf + 1];               // 1 / Phi(k), k = 0 .. P/2 (grid units)
    KernelPoly poly;                       // binary32 kernel pieces
    double beta;                           // ES shape (binary64 direct evaluation)
    int do_ems;
    EmsArgs ems;
};

template <typename T, int NF, int W>
struct FwdCfg {
    static constexpr int HO = W / 2 + 1;                      // halo offset of node 0
    static constexpr int GR = NF + W + 2;                     // padded grid rows (and used columns)
    static constexpr int GS = ((NF + W + 2 + 3) / 8) * 8 + 4; // row stride, = 4 mod 8 (bank spread)
    static constexpr int C1S_MAX = NF / 4 + 1;                // half-spectrum columns kept (m = 0..P/2)
    static constexpr int NT = NF >= 128 ? 512 : 256;          // threads per block
    // co-resident blocks the register budget is sized for (two 512-thread blocks per SM when the
    // shared-memory footprint allows it, so one block's FFT overlaps the other's spreading)
    static constexpr int MINB = (sizeof(T) == 4 && NF <= 128) ? 2 : 1;
    static constexpr int NWARPS = NT / 32;
    static constexpr int N1 = FftSplit<NF>::N1, N2 = FftSplit<NF>::N2;
    static constexpr int R_EMS = ((NF / 4) * (NF / 4) * 2 / NWARPS + 31) / 32;   // >= J*/nwarps/32
    static constexpr size_t grid_bytes = sizeof(T) * (size_t)GR * GS;
    static constexpr size_t c1_bytes_min = sizeof(cplx<T>) * (size_t)NF * C1S_MAX;
    static constexpr size_t ems_bytes = ems_smem_bytes(NWARPS, kEmsMaxK);
    static constexpr size_t c1_bytes = c1_bytes_min > ems_bytes ? c1_bytes_min : ems_bytes;
    static constexpr size_t tw_bytes = sizeof(cplx<T>) * NF;
    static constexpr size_t smem_bytes = grid_bytes + c1_bytes + tw_bytes + sizeof(CellConst) + 64;
};

__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
    // s + e = a - b exactly (Knuth TwoSum on a + (-b))
    s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
}

// App. A window test in binary64, in the same operation order as its definition (closed sets);
// used for every sample of binary64 plans and for samples inside the binary32 margin.
__device__ __forceinline__ bool window_f64(const CellConst& cc, double x, double y) {
    const double ux = __dsub_rn(x, cc.cx), uy = __dsub_rn(y, cc.cy);
    if (ux < -cc.H || ux > cc.H || uy < -cc.H || uy > cc.H) return false;
    if (cc.mask == 1) return true;
    if (cc.mask == 2) return __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)) <= __dmul_rn(cc.H, cc.H);
    for (int i = 0; i < cc.nv; ++i) {
        const int j = (i + 1 == cc.nv) ? 0 : i + 1;
        const double cr = __dsub_rn(__dmul_rn(__dsub_rn(cc.ux[j], cc.ux[i]), __dsub_rn(uy, cc.uy[i])),
                                    __dmul_rn(__dsub_rn(cc.uy[j], cc.uy[i]), __dsub_rn(ux, cc.ux[i])));
        if (__dmul_rn(cc.orient, cr) < 0.0) return false;
    }
    return true;
}

// binary32 window test with a certified margin: returns 1 inside, 0 outside, -1 undecided
__device__ __forceinline__ int window_f32(const CellConst& cc, float ux, float uy) {
    const float tau = cc.tau;
    int unsure = 0;
    const float bx = fabsf(ux) - cc.Hf, by = fabsf(uy) - cc.Hf;
    if (bx > tau || by > tau) return 0;
    unsure |= (bx > -tau) | (by > -tau);
    if (cc.mask == 0) {
        for (int i = 0; i < cc.nv; ++i) {
            const float f = __fmaf_rn(cc.enx[i], ux, __fmaf_rn(cc.eny[i], uy, -cc.ed[i]));
            if (f > tau) return 0;
            unsure |= f > -tau;
        }
    } else if (cc.mask == 2) {
        const float f = __fmaf_rn(ux, ux, __fmaf_rn(uy, uy, -cc.Hf * cc.Hf));
        const float t2 = 4.0f * tau * cc.Hf;
        if (f > t2) return 0;
        unsure |= f > -t2;
    }
    return unsure ? -1 : 1;
}

// Horner evaluation of the W kernel pieces at u in [-1, 1]
template <int W>
__device__ __forceinline__ void kernel_pieces(const KernelPoly& kp, float u, float (&v)[W]) {
#pragma unroll
    for (int i = 0; i < W; ++i) v[i] = kp.c[i][kMaxDeg - 1];
#pragma unroll
    for (int d = kMaxDeg - 2; d >= 0; --d) {
        if (d < kp.deg) {   // deg is uniform across the grid; unused leading pieces are zero
#pragma unroll
            for (int i = 0; i < W; ++i) v[i] = __fmaf_rn(v[i], u, kp.c[i][d]);
        }
    }
}

// Per-sample setup shared by spreading and interpolation (binary32 path): window test, first
// node r0 of each dimension and the W kernel values there.  Returns false for samples outside
// the window (or non-finite ones, which also latch ST_NONFINITE).
template <int NF, int W>
__device__ __forceinline__ bool prep_f32(const CellConst& cc, const KernelPoly& kp, float px, float py,
                                         int& r0x, int& r0y, float (&kx)[W], float (&ky)[W], unsigned* status) {
    if (!(isfinite(px) && isfinite(py))) {
        atomicOr(status, ST_NONFINITE);
        return false;
    }
    float uxh, uxl, uyh, uyl;
    two_diff(px, cc.cxh, uxh, uxl);
    uxl = __fsub_rn(uxl, cc.cxl);
    two_diff(py, cc.cyh, uyh, uyl);
    uyl = __fsub_rn(uyl, cc.cyl);
    int win = window_f32(cc, uxh + uxl, uyh + uyl);
    if (win < 0) win = window_f64(cc, (double)px, (double)py);
    if (!win) return false;
    // grid coordinate s = u * (n_f / L) + n_f / 2; first node r0 = ceil(s - W/2);
    // t = r0 - s + W/2 in [0, 1) from the hi/lo pieces (one rounding at magnitude < 1)
    const float sx = __fmaf_rn(uxh, cc.sch, 0.5f * NF), sy = __fmaf_rn(uyh, cc.sch, 0.5f * NF);
    r0x = (int)ceilf(sx - 0.5f * W);
    r0y = (int)ceilf(sy - 0.5f * W);
    const float corrx = __fmaf_rn(uxh, cc.scl, uxl * cc.sch), corry = __fmaf_rn(uyh, cc.scl, uyl * cc.sch);
    const float tx = __fmaf_rn(-uxh, cc.sch, (float)(r0x - NF / 2) + 0.5f * W) - corrx;
    const float ty = __fmaf_rn(-uyh, cc.sch, (float)(r0y - NF / 2) + 0.5f * W) - corry;
    kernel_pieces<W>(kp, __fmaf_rn(2.0f, tx, -1.0f), kx);
    kernel_pieces<W>(kp, __fmaf_rn(2.0f, ty, -1.0f), ky);
    return true;
}

// binary64 path: window in binary64, direct kernel evaluation exp(beta (sqrt(1 - z^2) - 1))
template <int NF, int W>
__device__ __forceinline__ bool prep_f64(const CellConst& cc, double beta, double px, double py, int& r0x,
                                         int& r0y, double (&kx)[W], double (&ky)[W], unsigned* status) {
    if (!(isfinite(px) && isfinite(py))) {
        atomicOr(status, ST_NONFINITE);
        return false;
    }
    if (!window_f64(cc, px, py)) return false;
    const double sc = (double)NF / cc.L;
    const double sx = (px - cc.cx) * sc + 0.5 * NF, sy = (py - cc.cy) * sc + 0.5 * NF;
    r0x = (int)ceil(sx - 0.5 * W);
    r0y = (int)ceil(sy - 0.5 * W);
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const double zx = ((double)(r0x + i) - sx) * (2.0 / W), zy = ((double)(r0y + i) - sy) * (2.0 / W);
        kx[i] = exp(beta * (sqrt(fmax(0.0, 1.0 - zx * zx)) - 1.0));
        ky[i] = exp(beta * (sqrt(fmax(0.0, 1.0 - zy * zy)) - 1.0));
    }
    return true;
}

// shared-memory float reduction with a compile-time immediate offset
template <int OFF>
__device__ __forceinline__ void red_smem(unsigned addr, float v) {
    asm volatile("red.shared.add.f32 [%0+%2], %1;" ::"r"(addr), "f"(v), "n"(OFF * 4));
}

template <int W, int GS, int J = 0, int I = 0>
__device__ __forceinline__ void spread_taps(unsigned addr, const float (&kx)[W], const float (&ky)[W], float c) {
    if constexpr (J < W) {
        if constexpr (I < W) {
            red_smem<J * GS + I>(addr, (c * ky[J]) * kx[I]);
            spread_taps<W, GS, J, I + 1>(addr, kx, ky, c);
        } else {
            spread_taps<W, GS, J + 1, 0>(addr, kx, ky, c);
        }
    }
}

// spread one sample (binary32 path); g points at the padded grid
template <int NF, int W, int GS, int HO>
__device__ __forceinline__ void spread_f32(float* __restrict__ g, const CellConst& cc, const KernelPoly& kp,
                                           float px, float py, float ph, float pw, unsigned* status) {
    int r0x, r0y;
    float kx[W], ky[W];
    if (!prep_f32<NF, W>(cc, kp, px, py, r0x, r0y, kx, ky, status)) return;
    const float c = pw * ph * cc.inv_area;
    if (!isfinite(c)) {
        atomicOr(status, ST_NONFINITE);
        return;
    }
    const unsigned addr = (unsigned)__cvta_generic_to_shared(g + (r0y + HO) * GS + (r0x + HO));
    spread_taps<W, GS>(addr, kx, ky, c);
}

// spread one sample (binary64 path)
template <int NF, int W, int GS, int HO>
__device__ __forceinline__ void spread_f64(double* __restrict__ g, const CellConst& cc, double beta,
                                           double px, double py, double ph, double pw, unsigned* status) {
    int r0x, r0y;
    double kx[W], ky[W];
    if (!prep_f64<NF, W>(cc, beta, px, py, r0x, r0y, kx, ky, status)) return;
    const double c = pw * ph / cc.area;
    if (!isfinite(c)) {
        atomicOr(status, ST_NONFINITE);
        return;
    }
    double* gp = g + (r0y + HO) * GS + (r0x + HO);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const double cy = c * ky[j];
#pragma unroll
        for (int i = 0; i < W; ++i) atomicAdd(gp + j * GS + i, cy * kx[i]);
    }
}

template <typename T>
struct StagedSpec {
    const cplx<T>* s;
    int P, half;
    __device__ __forceinline__ cplx<T> get(int m, int n) const { return s[(n + half) * P + (m + half)]; }
};

template <typename T, int NF, int W>
__global__ void __launch_bounds__(FwdCfg<T, NF, W>::NT, FwdCfg<T, NF, W>::MINB)
type1_fused_kernel(const __grid_constant__ FwdArgs<T> a) {
    using CF = FwdCfg<T, NF, W>;
    constexpr int GS = CF::GS, GR = CF::GR, HO = CF::HO, N1 = CF::N1, N2 = CF::N2;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sgrid = reinterpret_cast<T*>(smem);
    cplx<T>* sC1 = reinterpret_cast<cplx<T>*>(smem + CF::grid_bytes);
    cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem + CF::grid_bytes + CF::c1_bytes);
    CellConst* scc = reinterpret_cast<CellConst*>(smem + CF::grid_bytes + CF::c1_bytes + CF::tw_bytes);
    int* sticket = reinterpret_cast<int*>(scc + 1);

    const int tid = threadIdx.x, lane = tid & 31;
    const int P = a.P, half = P / 2, C1S = half + 1;
    for (int i = tid; i < NF; i += CF::NT) stw[i] = a.twiddle[i];

    for (;;) {
        if (tid == 0) *sticket = (int)atomicAdd(a.ticket, 1u);
        __syncthreads();   // also orders the previous cell's last shared-memory reads
        const int tk = *sticket;
        if (tk >= a.n_work) break;
        const int cell = a.order[tk];
        {   // per-cell constants into shared memory; zero the padded grid
            const int* src = reinterpret_cast<const int*>(a.cells + cell);
            int* dst = reinterpret_cast<int*>(scc);
            for (int i = tid; i < (int)(sizeof(CellConst) / 4); i += CF::NT) dst[i] = src[i];
            float4* g4 = reinterpret_cast<float4*>(sgrid);
            const int n4 = (int)(CF::grid_bytes / 16);
            for (int i = tid; i < n4; i += CF::NT) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const CellConst& cc = *scc;
        // ---- step 1+2: window, scale, spread
        if (cc.valid) {
            const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
            int64_t q = q0 + tid;
            for (; q + CF::NT < q1; q += 2 * CF::NT) {   // two samples per thread in flight
                const T x0 = a.x[q], y0 = a.y[q], h0 = a.h[q], w0 = a.w[q];
                const T x1 = a.x[q + CF::NT], y1 = a.y[q + CF::NT], h1 = a.h[q + CF::NT], w1 = a.w[q + CF::NT];
                if constexpr (sizeof(T) == 4) {
                    spread_f32<NF, W, GS, HO>(sgrid, cc, a.poly, x0, y0, h0, w0, a.status);
                    spread_f32<NF, W, GS, HO>(sgrid, cc, a.poly, x1, y1, h1, w1, a.status);
                } else {
                    spread_f64<NF, W, GS, HO>(sgrid, cc, a.beta, x0, y0, h0, w0, a.status);
                    spread_f64<NF, W, GS, HO>(sgrid, cc, a.beta, x1, y1, h1, w1, a.status);
                }
            }
            if (q < q1) {
                if constexpr (sizeof(T) == 4)
                    spread_f32<NF, W, GS, HO>(sgrid, cc, a.poly, a.x[q], a.y[q], a.h[q], a.w[q], a.status);
                else
                    spread_f64<NF, W, GS, HO>(sgrid, cc, a.beta, a.x[q], a.y[q], a.h[q], a.w[q], a.status);
            }
        } else if (tid == 0) {
            atomicOr(a.status, ST_BADCELL);
        }
        __syncthreads();
        // ---- periodic fold of the halo: columns first (all padded rows), then rows
        for (int i = tid; i < GR * (GR - NF); i += CF::NT) {
            const int r = i / (GR - NF), k = i % (GR - NF);
            const int c = k < HO ? k : k + NF;              // halo column
            const int cw = k < HO ? k + NF : k;             // its periodic image inside the core
            sgrid[r * GS + cw] += sgrid[r * GS + c];
        }
        __syncthreads();
        for (int i = tid; i < (GR - NF) * NF; i += CF::NT) {
            const int k = i / NF, c = HO + i % NF;
            const int r = k < HO ? k : k + NF;
            const int rw = k < HO ? k + NF : k;
            sgrid[rw * GS + c] += sgrid[r * GS + c];
        }
        __syncthreads();
        // ---- step 3a: FFT of the rows, two real rows per complex transform; keep m = 0..P/2
        {
            const int team = tid / N2, t = tid % N2;
            const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
            if (team < NF / 2) {
                T* r0 = sgrid + (HO + 2 * team) * GS + HO;
                T* r1 = r0 + GS;
                team_fft<N1, N2, T>(RowPairAcc<T>{r0, r1}, t, stw, tmask);
                for (int m = t; m <= half; m += N2) {
                    const int mn = (NF - m) & (NF - 1);
                    const T zr = r0[m], zi = r1[m], wr = r0[mn], wi = r1[mn];
                    sC1[(2 * team) * C1S + m] = cplx<T>{T(0.5) * (zr + wr), T(0.5) * (zi - wi)};
                    sC1[(2 * team + 1) * C1S + m] = cplx<T>{T(0.5) * (zi + wi), T(0.5) * (wr - zr)};
                }
            }
        }
        __syncthreads();
        // ---- step 3b: FFT of the columns m = 0..P/2
        {
            const int team = tid / N2, t = tid % N2;
            const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
            if (team <= half) team_fft<N1, N2, T>(StridedAcc<T, false>{sC1 + team, C1S}, t, stw, tmask);
        }
        __syncthreads();
        // ---- step 4: deconvolve, crop, Hermitian fill, stage P x P in the (now free) grid memory
        cplx<T>* stage = reinterpret_cast<cplx<T>*>(sgrid);
        for (int i = tid; i < (half + 1) * (P + 1); i += CF::NT) {
            const int m = i % (half + 1), n = i / (half + 1) - half;
            const T f = a.inv_phi[m] * a.inv_phi[n < 0 ? -n : n];
            const cplx<T> z = sC1[((n + NF) & (NF - 1)) * C1S + m];
            const cplx<T> v{z.re * f, z.im * f};
            if (m < half && n < half) stage[(n + half) * P + (m + half)] = v;
            if (m >= 1 && n > -half) stage[(half - n) * P + (half - m)] = cconj(v);
        }
        __syncthreads();
        // ---- step 5: EMS on the staged spectrum (shared scratch in the free half-spectrum area)
        if (a.do_ems)
            ems_block<T, CF::R_EMS>(StagedSpec<T>{stage, P, half}, P, cell, a.ems,
                                    reinterpret_cast<unsigned char*>(sC1));
        {   // coalesced 16-byte stores of the P x P spectrum
            const float4* s4 = reinterpret_cast<const float4*>(stage);
            float4* d4 = reinterpret_cast<float4*>(a.coeffs + (size_t)cell * P * P * 2);
            const int n4 = P * P * (int)sizeof(cplx<T>) / 16;
            for (int i = tid; i < n4; i += CF::NT) d4[i] = s4[i];
        }
    }
}

}  // namespace enufft
