// common.cuh -- device-side types shared by the ENUFFT kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace enufft {

// --------------------------------------------------------------------------------------------
// complex arithmetic (interleaved re, im; matches the C ABI coefficient layout)
// --------------------------------------------------------------------------------------------
template <typename T>
struct cplx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.re * s, a.im * s}; }
// multiply by -i
template <typename T>
__device__ __forceinline__ cplx<T> cmul_mi(cplx<T> a) { return {a.im, -a.re}; }

// --------------------------------------------------------------------------------------------
// device status word (latched conditions, read by enufft_sync_status)
// --------------------------------------------------------------------------------------------
enum : unsigned {
    ST_NONFINITE = 1u,   // a sample had a non-finite coordinate, elevation or weight (skipped)
    ST_TIMEOUT = 2u,     // a bounded wait gave up
    ST_BADCELL = 4u,     // a cell polygon was degenerate (zero area or bad vertex count)
    ST_MOVED = 8u,       // edge frame: a windowed sample had no binary32 local point inside the window
                         // near its own and was placed at the cell centroid
};

// --------------------------------------------------------------------------------------------
// per-cell constants, computed on the device by the frame kernel (App. A), binary64 first
// --------------------------------------------------------------------------------------------
struct CellConst {
    // binary64 frame (App. A): centroid, half-width H, period L = 2H, |D|
    double cx, cy, H, L, area;
    double ux[6], uy[6];   // polygon vertices in the centred frame u = x - xbar (R = I)
    double orient;         // +1 counter-clockwise, -1 clockwise
    int nv, mask, valid, pad_;
    // binary32 fast-path constants
    float cxh, cxl, cyh, cyl;    // centroid as unevaluated binary32 sums hi + lo
    float sch, scl;              // n_f / L as hi + lo
    float inv_area;              // 1 / |D|
    float Hf;                    // H rounded to binary32
    float tau;                   // decision margin (length units) below which the binary64 test decides
    float pad2_[3];
    float4 edge[6];              // outward unit edge normal (x, y) and offset z: inside <=> n.u <= z
};

// binary32 frame constants of the current cell, held in registers by every thread
struct FastFrame {
    float cxh, cxl, cyh, cyl, sch, scl, inv_area, Hf, tau;
    int mask, nv;
};

__device__ __forceinline__ FastFrame fast_frame(const CellConst& cc) {
    return FastFrame{cc.cxh, cc.cxl, cc.cyh, cc.cyl, cc.sch, cc.scl, cc.inv_area, cc.Hf, cc.tau, cc.mask, cc.nv};
}

// Spreading-kernel tables shared by the kernels of one plan (passed by value as a parameter).
constexpr int kMaxW = 16;
constexpr int kMaxDeg = 16;
// monomial coefficients per kernel piece used for width W (binary32 Horner evaluation)
__host__ __device__ constexpr int poly_deg(int W) { return W + 2 < kMaxDeg ? W + 2 : kMaxDeg; }
constexpr int KERNEL_ES = 0;   // exponential of semicircle
constexpr int KERNEL_KB = 1;   // Kaiser-Bessel (Eq. kb_compact), normalised to 1 at the centre
struct KernelPoly {
    int w;            // kernel width (grid points)
    int deg;          // number of monomial coefficients per piece
    float beta;       // shape parameter (ES beta, KB gamma)
    int kind;         // KERNEL_ES or KERNEL_KB
    double inv_norm;  // KB: 1 / I0(gamma), the normalisation to phi(0) = 1
    float c[kMaxW][kMaxDeg];   // piece i: phi_i(u) = sum_d c[i][d] u^d, u = 2 t - 1, t in [0, 1)
};

// kernel value at z in [-1, 1] (binary64): the ES exp(beta (sqrt(1 - z^2) - 1)) or the KB
// I0(gamma sqrt(1 - z^2)) / I0(gamma); shape is beta or gamma
__device__ __forceinline__ double kernel_value_f64(const KernelPoly& kp, double shape, double z) {
    const double r = sqrt(fmax(0.0, 1.0 - z * z));
    return kp.kind == KERNEL_KB ? cyl_bessel_i0(shape * r) * kp.inv_norm : exp(shape * (r - 1.0));
}

}  // namespace enufft
