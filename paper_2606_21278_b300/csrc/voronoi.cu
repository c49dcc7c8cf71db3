// voronoi.cu -- Voronoi quadrature weights by raster sampling (App. A, Eqs. voronoi_cell,
// raster_grid, nn_assignment, raster_area, area_partition, voronoi_weights), one block per cell
// (persistent over cells):
//   1. the window decision of every sample (the same certified binary32 test with binary64
//      fallback as the transform, so the windowed set is the transform's);
//   2. the raster points g_ab = (cx - H + (L/Ng)(a + 1/2), cy - H + (L/Ng)(b + 1/2)) in binary64,
//      kept when inside the window; each kept point is assigned to its nearest windowed sample by
//      brute force over shared-memory tiles of the cell's samples, the squared distance taken in
//      binary32 with every operation rounded as written, ties to the lowest sample index; the
//      counts n_q are accumulated by integer atomics (in the output array, reinterpreted);
//   3. w_q = max(n_q, 1/2) |D| / sum_q' max(n_q', 1/2) in binary64, rounded to binary32 (the floor
//      of 1/2 for a sample no raster point reached, then the renormalisation of Eq. area_partition);
//      samples outside the window get 0.
#include "forward.cuh"
#include "internal.h"

namespace enufft {

namespace {
constexpr int kVorThreads = 256;
constexpr int kVorR = 8;          // raster points per thread and pass
constexpr int kVorTile = 2048;    // samples per shared-memory tile
}  // namespace

static __global__ void __launch_bounds__(kVorThreads) voronoi_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                                      const int64_t* __restrict__ offsets,
                                                                      const CellConst* __restrict__ cells, int n_cells,
                                                                      int Ng, float* w, unsigned* status) {
    __shared__ float sx[kVorTile], sy[kVorTile];
    __shared__ CellConst scc;
    __shared__ long long ssum[kVorThreads / 32];
    int* cnt = reinterpret_cast<int*>(w);   // counts first, weights at the end (same slots)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        __syncthreads();   // the previous cell's shared state is no longer read
        {
            const int4* src = reinterpret_cast<const int4*>(cells + cell);
            int4* dst = reinterpret_cast<int4*>(&scc);
            for (int i = tid; i < (int)(sizeof(CellConst) / 16); i += kVorThreads) dst[i] = src[i];
        }
        __syncthreads();
        const CellConst& cc = scc;
        const int64_t q0 = offsets[cell], q1 = offsets[cell + 1];
        if (!cc.valid) {
            for (int64_t q = q0 + tid; q < q1; q += kVorThreads) w[q] = 0.0f;
            if (tid == 0 && q1 > q0) atomicOr(status, ST_BADCELL);
            continue;
        }
        // ---- 1. window decisions: count 0 inside, -1 outside
        const FastFrame ff = fast_frame(cc);
        for (int64_t q = q0 + tid; q < q1; q += kVorThreads) {
            const float px = x[q], py = y[q];
            int in = 0;
            if (isfinite(px) && isfinite(py)) {
                float uxh, uxl, uyh, uyl;
                two_diff(px, ff.cxh, uxh, uxl);
                uxl = __fsub_rn(uxl, ff.cxl);
                two_diff(py, ff.cyh, uyh, uyl);
                uyl = __fsub_rn(uyl, ff.cyl);
                in = window_f32(ff, cc.edge, uxh + uxl, uyh + uyl);
                if (in < 0) in = window_f64(cc, (double)px, (double)py);
            } else {
                atomicOr(status, ST_NONFINITE);
            }
            cnt[q] = in ? 0 : -1;
        }
        __syncthreads();
        // ---- 2. raster points -> nearest windowed sample
        const double x0 = __dsub_rn(cc.cx, cc.H), y0 = __dsub_rn(cc.cy, cc.H), step = __ddiv_rn(cc.L, (double)Ng);
        const int npts = Ng * Ng;
        for (int base = 0; base < npts; base += kVorThreads * kVorR) {
            float X[kVorR], Y[kVorR], best[kVorR];
            int arg[kVorR];
#pragma unroll
            for (int r = 0; r < kVorR; ++r) {
                const int idx = base + tid + kVorThreads * r;
                arg[r] = -1;
                best[r] = INFINITY;
                X[r] = INFINITY;   // points outside the window never take a sample
                Y[r] = INFINITY;
                if (idx < npts) {
                    const int a = idx % Ng, b = idx / Ng;
                    const double Xd = __dadd_rn(x0, __dmul_rn(step, (double)a + 0.5));
                    const double Yd = __dadd_rn(y0, __dmul_rn(step, (double)b + 0.5));
                    int in = window_f32(ff, cc.edge, __double2float_rn(__dsub_rn(Xd, cc.cx)),
                                        __double2float_rn(__dsub_rn(Yd, cc.cy)));
                    if (in < 0) in = window_f64(cc, Xd, Yd);
                    if (in) {
                        X[r] = __double2float_rn(Xd);
                        Y[r] = __double2float_rn(Yd);
                    }
                }
            }
            for (int64_t t0 = q0; t0 < q1; t0 += kVorTile) {
                const int nt = (q1 - t0) < (int64_t)kVorTile ? (int)(q1 - t0) : kVorTile;
                __syncthreads();
                for (int i = tid; i < nt; i += kVorThreads) {
                    const bool in = cnt[t0 + i] >= 0;   // sign set in step 1; later increments keep it
                    sx[i] = in ? x[t0 + i] : INFINITY;
                    sy[i] = in ? y[t0 + i] : INFINITY;
                }
                __syncthreads();
                for (int i = 0; i < nt; ++i) {
                    const float qx = sx[i], qy = sy[i];
#pragma unroll
                    for (int r = 0; r < kVorR; ++r) {
                        const float dx = __fsub_rn(X[r], qx), dy = __fsub_rn(Y[r], qy);
                        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                        if (d2 < best[r]) {
                            best[r] = d2;
                            arg[r] = (int)(t0 - q0) + i;
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kVorR; ++r)
                if (arg[r] >= 0) atomicAdd(&cnt[q0 + arg[r]], 1);
        }
        __syncthreads();
        // ---- 3. floor, renormalisation, weights
        long long s2 = 0;   // sum of 2 max(n_q, 1/2)
        for (int64_t q = q0 + tid; q < q1; q += kVorThreads) {
            const int c = cnt[q];
            if (c >= 0) s2 += c > 0 ? 2LL * c : 1LL;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) ssum[warp] = s2;
        __syncthreads();
        long long S2 = 0;
        for (int i = 0; i < kVorThreads / 32; ++i) S2 += ssum[i];
        const double unit = S2 > 0 ? __ddiv_rn(cc.area, 0.5 * (double)S2) : 0.0;
        for (int64_t q = q0 + tid; q < q1; q += kVorThreads) {
            const int c = cnt[q];
            w[q] = c < 0 ? 0.0f : __double2float_rn(__dmul_rn(c > 0 ? (double)c : 0.5, unit));
        }
    }
}

cudaError_t launch_voronoi(const float* x, const float* y, const int64_t* offsets, const CellConst* cells, int n_cells,
                           int Ng, float* w, unsigned* status, int num_sms, cudaStream_t s) {
    if (n_cells <= 0) return cudaSuccess;
    const int grid = n_cells < 8 * num_sms ? n_cells : 8 * num_sms;
    voronoi_kernel<<<grid, kVorThreads, 0, s>>>(x, y, offsets, cells, n_cells, Ng, w, status);
    return cudaGetLastError();
}

}  // namespace enufft
