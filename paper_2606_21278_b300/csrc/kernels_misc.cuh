// kernels_misc.cuh -- per-cell frame (App. A), standalone EMS (Sec. 2.2) and the EMS gradient.
#pragma once

#include "common.cuh"
#include "ems.cuh"
#include "internal.h"

namespace enufft {

// ---------------------------------------------------------------------------------------------
// App. A frame of every cell, binary64: centroid, centroid-aligned (R = I) or edge-aligned frame
// (Eq. rotation_matrix: the longest edge made parallel to +x; its centroid and rotation go to rot[j]
// and the cell's own constants describe the local frame, origin 0),
// H = (eta / 2) max extent, L = 2H, |D| of the mask, plus the binary32 fast-path constants.
// Centroid, extents, H, the centred vertices and the orientation follow the definition's
// operation order exactly, because the binary64 window test decides boundary samples with them.
// ---------------------------------------------------------------------------------------------
__device__ inline int clip_side(int n, const double* x, const double* y, int axis, double s, double H, double* ox,
                                double* oy) {
    // keep the part of the polygon with s * coord(axis) <= H (one Sutherland-Hodgman edge)
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1) % n;
        const double ci = s * (axis == 0 ? x[i] : y[i]) - H;
        const double cj = s * (axis == 0 ? x[j] : y[j]) - H;
        const bool in_i = ci <= 0.0, in_j = cj <= 0.0;
        if (in_i) { ox[m] = x[i]; oy[m] = y[i]; ++m; }
        if (in_i != in_j) {
            const double t = ci / (ci - cj);
            ox[m] = x[i] + t * (x[j] - x[i]);
            oy[m] = y[i] + t * (y[j] - y[i]);
            ++m;
        }
    }
    return m;
}

static __global__ void frame_kernel(int64_t n_cells, const int32_t* __restrict__ nverts, const double* __restrict__ verts,
                             double eta, int mask, int nf, int frame, CellConst* __restrict__ out,
                             FrameRot* __restrict__ rot) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n_cells) return;
    CellConst cc;
    memset(&cc, 0, sizeof(cc));
    const int nv = nverts[j];
    cc.nv = nv;
    cc.mask = mask;
    if (nv < 3 || nv > 6) {
        out[j] = cc;
        return;
    }
    const double* v = verts + 12 * j;
    double cx = 0.0, cy = 0.0;
    for (int i = 0; i < nv; ++i) {
        cx = __dadd_rn(cx, v[2 * i]);
        cy = __dadd_rn(cy, v[2 * i + 1]);
    }
    cx = __ddiv_rn(cx, (double)nv);
    cy = __ddiv_rn(cy, (double)nv);
    double rc = 1.0, rs = 0.0;
    if (frame == 1) {
        // longest edge e_i = v_(i+1) - v_i, the first on a tie; (cos t, sin t) = e / |e|
        double best = -1.0, ex = 1.0, ey = 0.0;
        for (int i = 0; i < nv; ++i) {
            const int k = (i + 1) % nv;
            const double dx = __dsub_rn(v[2 * k], v[2 * i]), dy = __dsub_rn(v[2 * k + 1], v[2 * i + 1]);
            const double len = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
            if (len > best) { best = len; ex = dx; ey = dy; }
        }
        if (best > 0.0) {
            rc = __ddiv_rn(ex, best);
            rs = __ddiv_rn(ey, best);
        }
        rot[j] = FrameRot{cx, cy, rc, rs};
    }
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = 0; i < nv; ++i) {
        const double dx = __dsub_rn(v[2 * i], cx), dy = __dsub_rn(v[2 * i + 1], cy);
        if (frame == 1) {   // u = R (x - x-bar)
            cc.ux[i] = __dadd_rn(__dmul_rn(rc, dx), __dmul_rn(rs, dy));
            cc.uy[i] = __dadd_rn(__dmul_rn(-rs, dx), __dmul_rn(rc, dy));
        } else {
            cc.ux[i] = dx;
            cc.uy[i] = dy;
        }
        xmin = fmin(xmin, cc.ux[i]); xmax = fmax(xmax, cc.ux[i]);
        ymin = fmin(ymin, cc.uy[i]); ymax = fmax(ymax, cc.uy[i]);
    }
    const double ex = __dsub_rn(xmax, xmin), ey = __dsub_rn(ymax, ymin);
    const double ext = ex > ey ? ex : ey;
    const double H = __dmul_rn(__dmul_rn(0.5, eta), ext);
    double sa = 0.0;
    for (int i = 0; i < nv; ++i) {
        const int k = (i + 1) % nv;
        sa = __dadd_rn(sa, __dsub_rn(__dmul_rn(cc.ux[i], cc.uy[k]), __dmul_rn(cc.ux[k], cc.uy[i])));
    }
    cc.orient = sa >= 0.0 ? 1.0 : -1.0;
    if (frame == 1) {   // the pre-pass hands every route local coordinates: origin 0
        cx = 0.0;
        cy = 0.0;
    }
    cc.cx = cx;
    cc.cy = cy;
    cc.H = H;
    cc.L = 2.0 * H;
    double area;
    if (mask == 1) {
        area = cc.L * cc.L;
    } else if (mask == 2) {
        area = 3.14159265358979323846 * H * H;
    } else {
        double ax[32], ay[32], bx[32], by[32];
        int n = nv;
        for (int i = 0; i < nv; ++i) { ax[i] = cc.ux[i]; ay[i] = cc.uy[i]; }
        n = clip_side(n, ax, ay, 0, +1.0, H, bx, by);
        n = clip_side(n, bx, by, 0, -1.0, H, ax, ay);
        n = clip_side(n, ax, ay, 1, +1.0, H, bx, by);
        n = clip_side(n, bx, by, 1, -1.0, H, ax, ay);
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const int k = (i + 1) % n;
            s += ax[i] * ay[k] - ax[k] * ay[i];
        }
        area = n >= 3 ? 0.5 * fabs(s) : 0.0;
    }
    cc.area = area;
    cc.valid = (area > 0.0 && H > 0.0) ? 1 : 0;
    // binary32 fast path
    cc.cxh = (float)cx;
    cc.cxl = (float)(cx - (double)cc.cxh);
    cc.cyh = (float)cy;
    cc.cyl = (float)(cy - (double)cc.cyh);
    const double sc = cc.valid ? (double)nf / cc.L : 0.0;
    cc.sch = (float)sc;
    cc.scl = (float)(sc - (double)cc.sch);
    cc.inv_area = cc.valid ? (float)(1.0 / area) : 0.0f;
    cc.Hf = (float)H;
    // margin: >= 10x the worst binary32 rounding of the edge functions (a few ulp of |u| <= 2H)
    cc.tau = (float)(H * 1.52587890625e-05);   // 2^-16 H
    for (int i = 0; i < nv; ++i) {
        const int k = (i + 1) % nv;
        const double dx = cc.ux[k] - cc.ux[i], dy = cc.uy[k] - cc.uy[i];
        const double len = sqrt(dx * dx + dy * dy);
        double nx = 0.0, ny = 0.0;
        if (len > 0.0) {
            nx = cc.orient * dy / len;   // outward normal of a counter-clockwise edge is (dy, -dx)
            ny = -cc.orient * dx / len;
        }
        cc.edge[i] = make_float4((float)nx, (float)ny, (float)(nx * cc.ux[i] + ny * cc.uy[i]), 0.0f);
    }
    out[j] = cc;
}

// ---------------------------------------------------------------------------------------------
// standalone EMS stage 1: one block per cell, energies read from the stored spectrum
// ---------------------------------------------------------------------------------------------
template <typename T>
struct GlobalSpec {
    const cplx<T>* s;
    int P, half;
    __device__ __forceinline__ cplx<T> get(int m, int n) const { return s[(n + half) * P + (m + half)]; }
};

template <typename T, int R>
__global__ void __launch_bounds__(512) ems_rank_kernel(const cplx<T>* __restrict__ coeffs, int P, int64_t n_cells,
                                                       const __grid_constant__ EmsArgs a, EmsScratch out) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int64_t cell = blockIdx.x; cell < n_cells; cell += gridDim.x)
        ems_rank_block<T, R>(GlobalSpec<T>{coeffs + (size_t)cell * P * P, P, P / 2}, P, (int)cell, a, out, smem);
}

// ---------------------------------------------------------------------------------------------
// gradient of the retained power with the selection fixed: G = 2 gp W h on selected pairs
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void ems_backward_kernel(const cplx<T>* __restrict__ coeffs, int P, int64_t n_cells,
                                    const double* __restrict__ W, int w_per_cell, int k_max,
                                    const int32_t* __restrict__ kstar, const int32_t* __restrict__ sel,
                                    const double* __restrict__ gp, cplx<T>* __restrict__ G) {
    const int half = P / 2;
    for (int64_t cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        cplx<T>* g = G + (size_t)cell * P * P;
        const cplx<T>* c = coeffs + (size_t)cell * P * P;
        float4* g4 = reinterpret_cast<float4*>(g);
        const int n4 = P * P * (int)sizeof(cplx<T>) / 16;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int ks = kstar[cell];
        for (int k = threadIdx.x; k < ks; k += blockDim.x) {
            const int p = sel[cell * (int64_t)k_max + k];
            if (p < 0 || p >= P * P) continue;
            const int m = p % P - half, n = p / P - half;
            const int in = (half - n) * P + (half - m);
            const double wt = W ? W[(w_per_cell ? (size_t)cell * P * P : 0) + p] : 1.0;
            const T s = (T)(2.0 * gp[cell] * wt);
            g[p] = cplx<T>{s * c[p].re, s * c[p].im};
            if (in != p) g[in] = cplx<T>{s * c[in].re, s * c[in].im};
        }
        __syncthreads();
    }
}

}  // namespace enufft
