// edge_frame.cu -- per-call pre-pass of plans with the edge-aligned local frame (App. A,
// Eq. rotation_matrix).
//
// Every route reads sample coordinates relative to the cell constants' origin.  For edge-frame
// plans those constants describe the local frame itself (origin 0, rotated vertices), and this
// kernel writes each sample's local coordinates v = R (x - x-bar) into plan scratch.
//   - Binary64 plans: v in binary64 in the definition's operation order, stored as is (every later
//     window test sees the same v and decides as the definition does).
//   - Binary32 plans (B300's binary64 pipe is narrow, so binary64 work is kept to the rare samples
//     that need it): x - x-bar exactly as a binary32 pair (TwoSum against the centroid's hi + lo),
//     R applied with error-free products to a hi + lo result (~2^-44 relative), then the certified
//     binary32 window test with its margin of 2^-16 H, far above the gap between this v and the
//     definition's binary64 v.  A sample certified inside is stored as the binary32 v (later tests
//     see the same point and certify it again); one certified outside goes to (3H, 3H), which every
//     window test rejects.  A sample within the margin is decided by the definition's binary64
//     computation; if inside, v rounded to binary32 is stored, moved toward the centroid by the
//     smallest of a few growing factors (1 - 2^-23, 1 - 2^-21, ...) that keeps the binary64 test
//     true, the centroid itself as the last resort (it is inside every convex cell, B and the disk;
//     that case latches ST_MOVED, reported by enufft_sync_status).  Later window tests therefore
//     agree with the exact decision.
//   - Non-finite coordinates are copied through, so the routes report them as before.
#include "internal.h"

namespace enufft {

namespace {
constexpr int kEdgeThreads = 256;
constexpr int kEdgeUnroll = 4;   // samples per thread and pass
}

// a * b = p + e exactly (FMA)
__device__ __forceinline__ void ef_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// a + b = s + e exactly (Knuth TwoSum)
__device__ __forceinline__ void ef_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah + al)(bh + bl) + (ch + cl)(dh + dl) as a renormalised binary32 pair
__device__ __forceinline__ void ef_dot2(float ah, float al, float bh, float bl, float ch, float cl, float dh, float dl,
                                        float& rh, float& rl) {
    float p1, e1, p2, e2, sh, se;
    ef_prod(ah, bh, p1, e1);
    ef_prod(ch, dh, p2, e2);
    ef_sum(p1, p2, sh, se);
    float lo = __fadd_rn(se, __fadd_rn(e1, e2));
    lo = __fmaf_rn(ah, bl, lo);
    lo = __fmaf_rn(al, bh, lo);
    lo = __fmaf_rn(ch, dl, lo);
    lo = __fmaf_rn(cl, dh, lo);
    rh = __fadd_rn(sh, lo);
    rl = __fsub_rn(lo, __fsub_rn(rh, sh));
}

// the definition's binary64 decision for a sample within the binary32 margin, and its stored point
__device__ __noinline__ float2 edge_exact_f32(const CellConst& cc, const FrameRot& fr, double px, double py, float far,
                                              unsigned* status) {
    const double dx = __dsub_rn(px, fr.cx), dy = __dsub_rn(py, fr.cy);
    const double ux = __dadd_rn(__dmul_rn(fr.c, dx), __dmul_rn(fr.s, dy));
    const double uy = __dadd_rn(__dmul_rn(-fr.s, dx), __dmul_rn(fr.c, dy));
    if (!window_f64(cc, ux, uy)) return make_float2(far, far);
    float fx = __double2float_rn(ux), fy = __double2float_rn(uy);
    bool in = window_f64(cc, (double)fx, (double)fy);
    for (int k = 0; k < 8 && !in; ++k) {
        const double sh = 1.0 - ldexp(1.0, -23 + 2 * k);
        fx = __double2float_rn(__dmul_rn(ux, sh));
        fy = __double2float_rn(__dmul_rn(uy, sh));
        in = window_f64(cc, (double)fx, (double)fy);
    }
    if (in) return make_float2(fx, fy);
    atomicOr(status, ST_MOVED);   // reported: the stored point is no longer the sample's own
    return make_float2(0.0f, 0.0f);
}

// the local coordinates of one sample (see the file comment)
template <typename T>
__device__ __forceinline__ void edge_local(const CellConst& cc, const FastFrame& ff, const FrameRot& fr, float cxh,
                                           float cxl, float cyh, float cyl, float ch, float cl, float sh, float sl,
                                           float far, T px, T py, T& ox, T& oy, unsigned* status) {
    if (!(isfinite(px) && isfinite(py))) {   // copied through: the routes report them
        ox = px;
        oy = py;
        return;
    }
    if (!cc.valid) {   // the routes skip the cell and report it
        ox = T(0);
        oy = T(0);
        return;
    }
    if constexpr (sizeof(T) == 8) {
        const double dx = __dsub_rn(px, fr.cx), dy = __dsub_rn(py, fr.cy);
        ox = __dadd_rn(__dmul_rn(fr.c, dx), __dmul_rn(fr.s, dy));
        oy = __dadd_rn(__dmul_rn(-fr.s, dx), __dmul_rn(fr.c, dy));
    } else {
        float dxh, dxl, dyh, dyl;
        two_diff(px, cxh, dxh, dxl);
        dxl = __fsub_rn(dxl, cxl);
        two_diff(py, cyh, dyh, dyl);
        dyl = __fsub_rn(dyl, cyl);
        float uxh, uxl, uyh, uyl;
        ef_dot2(ch, cl, dxh, dxl, sh, sl, dyh, dyl, uxh, uxl);     // cos t dx + sin t dy
        ef_dot2(-sh, -sl, dxh, dxl, ch, cl, dyh, dyl, uyh, uyl);   // -sin t dx + cos t dy
        const int win = window_f32(ff, cc.edge, uxh, uyh);
        float2 v;
        if (win > 0)
            v = make_float2(uxh, uyh);
        else if (win == 0)
            v = make_float2(far, far);
        else
            v = edge_exact_f32(cc, fr, (double)px, (double)py, far, status);
        ox = v.x;
        oy = v.y;
    }
}

// one block per cell (persistent over cells, three blocks per SM: launched as one wave of 3 x SMs
// blocks); each thread loads kEdgeUnroll samples before working on them, so that enough loads are
// in flight to stream the coordinates at HBM rate
template <typename T>
static __global__ void __launch_bounds__(kEdgeThreads, 3)
edge_frame_kernel(const T* __restrict__ x, const T* __restrict__ y, const int64_t* __restrict__ offsets,
                  const CellConst* __restrict__ cells, const FrameRot* __restrict__ rot, int64_t n_cells,
                  T* __restrict__ vx, T* __restrict__ vy, unsigned* status) {
    __shared__ __align__(16) CellConst scc;
    __shared__ FrameRot sfr;
    static_assert(sizeof(CellConst) % 16 == 0, "cell constants copied in 16-byte words");
    for (int64_t j = blockIdx.x; j < n_cells; j += gridDim.x) {
        __syncthreads();   // the previous cell's constants are no longer read
        {
            const int4* src = reinterpret_cast<const int4*>(cells + j);
            int4* dst = reinterpret_cast<int4*>(&scc);
            for (int i = threadIdx.x; i < (int)(sizeof(CellConst) / 16); i += blockDim.x) dst[i] = src[i];
            if (threadIdx.x == 0) sfr = rot[j];
        }
        __syncthreads();
        const CellConst& cc = scc;
        const FrameRot fr = sfr;
        const int64_t q0 = offsets[j], q1 = offsets[j + 1];
        const float far = (float)(3.0 * cc.H);
        // binary32 pairs of the centroid and the rotation (binary32 plans)
        const float cxh = (float)fr.cx, cxl = (float)(fr.cx - (double)cxh);
        const float cyh = (float)fr.cy, cyl = (float)(fr.cy - (double)cyh);
        const float ch = (float)fr.c, cl = (float)(fr.c - (double)ch);
        const float sh = (float)fr.s, sl = (float)(fr.s - (double)sh);
        const FastFrame ff = fast_frame(cc);
        constexpr int U = kEdgeUnroll;
        for (int64_t qb = q0 + threadIdx.x; qb < q1; qb += (int64_t)U * blockDim.x) {
            T px[U], py[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int64_t q = qb + (int64_t)k * blockDim.x;
                px[k] = q < q1 ? x[q] : T(0);
                py[k] = q < q1 ? y[q] : T(0);
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int64_t q = qb + (int64_t)k * blockDim.x;
                if (q < q1) {
                    T ox, oy;
                    edge_local<T>(cc, ff, fr, cxh, cxl, cyh, cyl, ch, cl, sh, sl, far, px[k], py[k], ox, oy, status);
                    vx[q] = ox;
                    vy[q] = oy;
                }
            }
        }
    }
}

cudaError_t launch_edge_frame(bool dbl, const void* x, const void* y, const int64_t* offsets, const CellConst* cells,
                              const FrameRot* rot, int64_t n_cells, void* vx, void* vy, unsigned* status, int grid,
                              cudaStream_t s) {
    if (n_cells <= 0) return cudaSuccess;
    if (dbl)
        edge_frame_kernel<double><<<grid, kEdgeThreads, 0, s>>>((const double*)x, (const double*)y, offsets, cells, rot,
                                                                n_cells, (double*)vx, (double*)vy, status);
    else
        edge_frame_kernel<float><<<grid, kEdgeThreads, 0, s>>>((const float*)x, (const float*)y, offsets, cells, rot,
                                                               n_cells, (float*)vx, (float*)vy, status);
    return cudaGetLastError();
}

}  // namespace enufft
