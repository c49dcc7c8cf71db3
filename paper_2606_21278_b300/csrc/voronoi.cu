// voronoi.cu -- Voronoi quadrature weights by raster sampling (App. A, Eqs. voronoi_cell,
// raster_grid, nn_assignment, raster_area, area_partition, voronoi_weights), one block per cell
// (persistent over cells):
//   1. the window decision of every sample (the same certified binary32 test with binary64
//      fallback as the transform, so the windowed set is the transform's);
//   2. the raster points g_ab = (cx - H + (L/Ng)(a + 1/2), cy - H + (L/Ng)(b + 1/2)) in binary64,
//      kept when inside the window; each kept point is assigned to its nearest windowed sample
//      (Eq. nn_assignment), ties to the lowest sample index; the counts n_q are accumulated by
//      integer atomics (in the output array, reinterpreted).  The nearest sample is the one of
//      the squared distances d2 = (X - x_q)^2 + (Y - y_q)^2 taken in binary64.  The search runs in
//      binary32 first and keeps the best and the second-best distance; when the gap between them
//      exceeds a certified bound of the binary32 rounding error (plus the binary64 one), the
//      binary32 winner is the binary64 winner.  Otherwise the point is searched again with binary64
//      distances in the definition's operation order.  The search: the cell's windowed samples are
//      sorted by a counting sort into a G x G grid of buckets over B in shared memory (about two per
//      bucket), and each point examines rings of buckets around its own until every sample not yet
//      examined is certainly farther than its best one; cells with more windowed samples than the
//      shared-memory capacity are searched by brute force over tiles of the samples;
//   3. w_q = max(n_q, 1/2) |D| / sum_q' max(n_q', 1/2) in binary64, rounded to binary32 (the floor
//      of 1/2 for a sample no raster point reached, then the renormalisation of Eq. area_partition);
//      samples outside the window get 0.
#include "forward.cuh"
#include "internal.h"

namespace enufft {

namespace {
constexpr int kVorThreads = 512;
constexpr int kVorR = 8;          // raster points per thread and pass (brute force)
constexpr int kVorTile = 2048;    // samples per shared-memory tile (brute force)
constexpr int kVorCap = 16384;    // windowed samples of one cell held in shared memory
constexpr int kVorMaxG = 64;      // buckets per side at most
constexpr size_t kVorSmem = (size_t)kVorCap * 12 + sizeof(int) * (kVorMaxG * kVorMaxG + 1);
static_assert(kVorCap * 8 >= 2 * kVorTile * 4, "brute-force tiles fit in the sample area");
}  // namespace

// raster point idx of a cell in binary64 (Eq. raster_grid)
__device__ __forceinline__ void vor_point_f64(double x0, double y0, double step, int Ng, int idx, double& Xd,
                                              double& Yd) {
    const int a = idx % Ng, b = idx / Ng;
    Xd = __dadd_rn(x0, __dmul_rn(step, (double)a + 0.5));
    Yd = __dadd_rn(y0, __dmul_rn(step, (double)b + 0.5));
}

// raster point idx of a cell: binary32 coordinates (INFINITY when outside the window)
__device__ __forceinline__ void vor_point(const CellConst& cc, const FastFrame& ff, double x0, double y0, double step,
                                          int Ng, int idx, float& X, float& Y) {
    double Xd, Yd;
    vor_point_f64(x0, y0, step, Ng, idx, Xd, Yd);
    int in = window_f32(ff, cc.edge, __double2float_rn(__dsub_rn(Xd, cc.cx)), __double2float_rn(__dsub_rn(Yd, cc.cy)));
    if (in < 0) in = window_f64(cc, Xd, Yd);
    X = in ? __double2float_rn(Xd) : INFINITY;
    Y = in ? __double2float_rn(Yd) : INFINITY;
}

__device__ __forceinline__ float vor_d2(float X, float Y, float qx, float qy) {
    const float dx = __fsub_rn(X, qx), dy = __fsub_rn(Y, qy);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// the definition's squared distance: binary64, every operation rounded as written
__device__ __forceinline__ double vor_d2_f64(double X, double Y, float qx, float qy) {
    const double dx = __dsub_rn(X, (double)qx), dy = __dsub_rn(Y, (double)qy);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Bound of |d2f - d2| for a binary32 distance d2f from the rounded raster point (A: the larger of
// its coordinate magnitudes) to a binary32 sample, against the exact d2 from the binary64 point:
// rounding the point moves it by at most u A, each of the four operations adds a relative u
// (u = 2^-24), and the true distance s is at most sqrt(d2f) + 3 u A; taken with 50 % slack.
__device__ __forceinline__ float vor_err32(float d2f, float A) {
    constexpr float u = 0x1p-24f;
    const float s = sqrtf(d2f) * 1.0001f + 3.0f * u * A;
    return u * (5.0f * A * s + 8.0f * s * s) + 4.0f * u * u * A * A;
}
// Is the binary32 winner (best) certainly the binary64 winner?  Every other candidate has a binary32
// distance >= second, and every sample not examined has an exact squared distance >= lb2.  The
// exact distances then differ by more than the binary32 bounds; a gap of at least one binary32 ulp
// (2^-24 relative) also exceeds the binary64 rounding (five roundings of 2^-53 on each side), so
// the binary64 computation ranks the two the same way.
__device__ __forceinline__ bool vor_certified(float best, float second, float lb2, float A) {
    const float hi_best = best + vor_err32(best, A);
    const float lo_second = second < INFINITY ? second - vor_err32(second, A) : INFINITY;
    return fminf(lo_second, lb2) > hi_best;
}

// brute force over shared-memory tiles of the cell's samples (any cell size): binary32 distances
// with the best and second-best per point, then one more pass in binary64 for the points whose
// binary32 winner is not certified (taken by the whole block when any point needs it)
__device__ void vor_brute(const float* __restrict__ x, const float* __restrict__ y, int64_t q0, int64_t q1,
                          const CellConst& cc, const FastFrame& ff, double x0, double y0, double step, int Ng, int* cnt,
                          float* sx, float* sy) {
    const int tid = threadIdx.x, nt_ = blockDim.x;
    const int npts = Ng * Ng;
    for (int base = 0; base < npts; base += nt_ * kVorR) {
        float X[kVorR], Y[kVorR], best[kVorR], second[kVorR];
        int arg[kVorR];
#pragma unroll
        for (int r = 0; r < kVorR; ++r) {
            const int idx = base + tid + nt_ * r;
            arg[r] = -1;
            best[r] = INFINITY;
            second[r] = INFINITY;
            X[r] = INFINITY;   // points outside the window never take a sample
            Y[r] = INFINITY;
            if (idx < npts) vor_point(cc, ff, x0, y0, step, Ng, idx, X[r], Y[r]);
        }
        for (int64_t t0 = q0; t0 < q1; t0 += kVorTile) {
            const int nt = (q1 - t0) < (int64_t)kVorTile ? (int)(q1 - t0) : kVorTile;
            __syncthreads();
            for (int i = tid; i < nt; i += nt_) {
                const bool in = cnt[t0 + i] >= 0;   // sign set by the window pass; later increments keep it
                sx[i] = in ? x[t0 + i] : INFINITY;
                sy[i] = in ? y[t0 + i] : INFINITY;
            }
            __syncthreads();
            for (int i = 0; i < nt; ++i) {
                const float qx = sx[i], qy = sy[i];
#pragma unroll
                for (int r = 0; r < kVorR; ++r) {
                    const float d2 = vor_d2(X[r], Y[r], qx, qy);
                    if (d2 < best[r]) {   // samples in index order: a tie keeps the lower index
                        second[r] = best[r];
                        best[r] = d2;
                        arg[r] = (int)(t0 - q0) + i;
                    } else if (d2 < second[r]) {
                        second[r] = d2;
                    }
                }
            }
        }
        bool need = false, f64[kVorR];
#pragma unroll
        for (int r = 0; r < kVorR; ++r) {
            f64[r] = arg[r] >= 0 && !vor_certified(best[r], second[r], INFINITY, fmaxf(fabsf(X[r]), fabsf(Y[r])));
            need |= f64[r];
        }
        if (__syncthreads_or(need)) {
            double Xd[kVorR], Yd[kVorR], b64[kVorR];
#pragma unroll
            for (int r = 0; r < kVorR; ++r) {
                vor_point_f64(x0, y0, step, Ng, base + tid + nt_ * r, Xd[r], Yd[r]);
                b64[r] = INFINITY;
            }
            for (int64_t t0 = q0; t0 < q1; t0 += kVorTile) {
                const int nt = (q1 - t0) < (int64_t)kVorTile ? (int)(q1 - t0) : kVorTile;
                __syncthreads();
                for (int i = tid; i < nt; i += nt_) {
                    const bool in = cnt[t0 + i] >= 0;
                    sx[i] = in ? x[t0 + i] : INFINITY;
                    sy[i] = in ? y[t0 + i] : INFINITY;
                }
                __syncthreads();
                if (need) {
                    for (int i = 0; i < nt; ++i) {
                        const float qx = sx[i], qy = sy[i];
#pragma unroll
                        for (int r = 0; r < kVorR; ++r) {
                            if (!f64[r]) continue;
                            const double d2 = vor_d2_f64(Xd[r], Yd[r], qx, qy);
                            if (d2 < b64[r]) {   // index order: a tie keeps the lower index
                                b64[r] = d2;
                                arg[r] = (int)(t0 - q0) + i;
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kVorR; ++r)
            if (arg[r] >= 0) atomicAdd(&cnt[q0 + arg[r]], 1);
    }
}

// exclusive prefix of n <= 8 * blockDim.x integers in shared memory, in place; total at v[n]
__device__ void vor_scan(int* v, int n, int* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    int loc[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = 8 * tid + k;
        loc[k] = i < n ? v[i] : 0;
        s += loc[k];
    }
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    int run = (warp ? wsum[warp - 1] : 0) + incl - s;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = 8 * tid + k;
        if (i < n) v[i] = run;
        run += loc[k];
    }
    if (tid == blockDim.x - 1) v[n] = run;
    __syncthreads();
}

static __global__ void __launch_bounds__(kVorThreads) voronoi_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                                      const int64_t* __restrict__ offsets,
                                                                      const CellConst* __restrict__ cells, int n_cells,
                                                                      int Ng, float* w, unsigned* status) {
    extern __shared__ __align__(16) unsigned char vsm[];
    float2* bxy = reinterpret_cast<float2*>(vsm);                       // [kVorCap] samples by bucket
    int* bidx = reinterpret_cast<int*>(bxy + kVorCap);                  // [kVorCap] their local indices
    int* boff = bidx + kVorCap;                                         // [kVorMaxG^2 + 1] bucket offsets
    float* sx = reinterpret_cast<float*>(vsm);                          // brute force tiles (aliases bxy)
    float* sy = sx + kVorTile;
    __shared__ CellConst scc;
    __shared__ long long ssum[kVorThreads / 32];
    __shared__ int wsum[kVorThreads / 32];
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
        // ---- 1. window decisions: count 0 inside, -1 outside; the number of windowed samples
        const FastFrame ff = fast_frame(cc);
        int nin = 0;
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
            nin += in ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nin += __shfl_xor_sync(0xffffffffu, nin, o);
        if (lane == 0) wsum[warp] = nin;
        __syncthreads();
        int Qw = 0;
        for (int i = 0; i < kVorThreads / 32; ++i) Qw += wsum[i];
        __syncthreads();
        const double x0 = __dsub_rn(cc.cx, cc.H), y0 = __dsub_rn(cc.cy, cc.H), step = __ddiv_rn(cc.L, (double)Ng);
        // ---- 2. raster points -> nearest windowed sample
        if (Qw > kVorCap) {
            vor_brute(x, y, q0, q1, cc, ff, x0, y0, step, Ng, cnt, sx, sy);
        } else if (Qw > 0) {
            int G = (int)sqrtf(0.5f * (float)Qw);
            G = G < 1 ? 1 : (G > kVorMaxG ? kVorMaxG : G);
            const float bx0 = __double2float_rn(x0), by0 = __double2float_rn(y0);
            const float bw = __double2float_rn(__ddiv_rn(cc.L, (double)G)), ibw = 1.0f / bw;
            for (int i = tid; i <= G * G; i += kVorThreads) boff[i] = 0;
            __syncthreads();
            for (int64_t q = q0 + tid; q < q1; q += kVorThreads) {
                if (cnt[q] < 0) continue;
                int bx = (int)((x[q] - bx0) * ibw), by = (int)((y[q] - by0) * ibw);
                bx = bx < 0 ? 0 : (bx >= G ? G - 1 : bx);
                by = by < 0 ? 0 : (by >= G ? G - 1 : by);
                atomicAdd(&boff[by * G + bx], 1);
            }
            __syncthreads();
            vor_scan(boff, G * G, wsum);
            // place every windowed sample: slot = its bucket's offset, advanced atomically
            for (int64_t q = q0 + tid; q < q1; q += kVorThreads) {
                if (cnt[q] < 0) continue;
                const float px = x[q], py = y[q];
                int bx = (int)((px - bx0) * ibw), by = (int)((py - by0) * ibw);
                bx = bx < 0 ? 0 : (bx >= G ? G - 1 : bx);
                by = by < 0 ? 0 : (by >= G ? G - 1 : by);
                const int slot = atomicAdd(&boff[by * G + bx], 1);   // offsets advance to the bucket ends
                bxy[slot] = make_float2(px, py);
                bidx[slot] = (int)(q - q0);
            }
            __syncthreads();
            // boff[b] now holds the end of bucket b = the start of bucket b + 1: shift by one
            int keep[(kVorMaxG * kVorMaxG + kVorThreads) / kVorThreads];
            int nk = 0;
            for (int i = tid; i < G * G; i += kVorThreads) keep[nk++] = boff[i];
            __syncthreads();
            nk = 0;
            for (int i = tid; i < G * G; i += kVorThreads) boff[i + 1] = keep[nk++];
            if (tid == 0) boff[0] = 0;
            __syncthreads();
            const int npts = Ng * Ng;
            for (int idx = tid; idx < npts; idx += kVorThreads) {
                float X, Y;
                vor_point(cc, ff, x0, y0, step, Ng, idx, X, Y);
                if (!(X < INFINITY)) continue;
                int px = (int)((X - bx0) * ibw), py = (int)((Y - by0) * ibw);
                px = px < 0 ? 0 : (px >= G ? G - 1 : px);
                py = py < 0 ? 0 : (py >= G ? G - 1 : py);
                const float A = fmaxf(fabsf(X), fabsf(Y));
                float best = INFINITY, second = INFINITY, lb2 = INFINITY;
                int arg = 0x7fffffff;
                for (int r = 0; r <= G; ++r) {
                    // every sample not yet examined lies in a bucket at least r away by index, so at
                    // least (r - 1) bucket widths from the point: stop once that is certainly farther
                    // than the best distance
                    if (r > 1 && best < INFINITY) {
                        const float lb = 0.999f * (float)(r - 1) * bw;
                        if (lb * lb > best + vor_err32(best, A)) {
                            lb2 = lb * lb;
                            break;
                        }
                    }
                    for (int dy = -r; dy <= r; ++dy) {
                        const int by = py + dy;
                        if (by < 0 || by >= G) continue;
                        const int stepx = (dy == -r || dy == r) ? 1 : 2 * r;
                        for (int dx = -r; dx <= r; dx += (stepx > 0 ? stepx : 1)) {
                            const int bx = px + dx;
                            if (bx < 0 || bx >= G) continue;
                            const int b = by * G + bx;
                            for (int s = boff[b]; s < boff[b + 1]; ++s) {
                                const float2 qv = bxy[s];
                                const float d2 = vor_d2(X, Y, qv.x, qv.y);
                                const int qi = bidx[s];
                                if (d2 < best || (d2 == best && qi < arg)) {
                                    second = best;
                                    best = d2;
                                    arg = qi;
                                } else if (d2 < second) {
                                    second = d2;
                                }
                            }
                            if (r == 0) break;
                        }
                    }
                }
                if (arg != 0x7fffffff && !vor_certified(best, second, lb2, A)) {
                    // the same search with the definition's binary64 distances; it stops once every
                    // sample not examined is farther than the best by more than binary64 rounding
                    double Xd, Yd;
                    vor_point_f64(x0, y0, step, Ng, idx, Xd, Yd);
                    double b64 = INFINITY;
                    arg = 0x7fffffff;
                    for (int r = 0; r <= G; ++r) {
                        if (r > 1 && b64 < INFINITY) {
                            const double lb = 0.999 * (double)(r - 1) * (double)bw;
                            if (lb * lb * (1.0 - 0x1p-40) > b64) break;
                        }
                        for (int dy = -r; dy <= r; ++dy) {
                            const int by = py + dy;
                            if (by < 0 || by >= G) continue;
                            const int stepx = (dy == -r || dy == r) ? 1 : 2 * r;
                            for (int dx = -r; dx <= r; dx += (stepx > 0 ? stepx : 1)) {
                                const int bx = px + dx;
                                if (bx < 0 || bx >= G) continue;
                                const int b = by * G + bx;
                                for (int s = boff[b]; s < boff[b + 1]; ++s) {
                                    const float2 qv = bxy[s];
                                    const double d2 = vor_d2_f64(Xd, Yd, qv.x, qv.y);
                                    const int qi = bidx[s];
                                    if (d2 < b64 || (d2 == b64 && qi < arg)) {
                                        b64 = d2;
                                        arg = qi;
                                    }
                                }
                                if (r == 0) break;
                            }
                        }
                    }
                }
                if (arg != 0x7fffffff) atomicAdd(&cnt[q0 + arg], 1);
            }
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
    cudaError_t e = cudaFuncSetAttribute(voronoi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVorSmem);
    if (e != cudaSuccess) return e;
    const int grid = n_cells < num_sms ? n_cells : num_sms;
    voronoi_kernel<<<grid, kVorThreads, kVorSmem, s>>>(x, y, offsets, cells, n_cells, Ng, w, status);
    return cudaGetLastError();
}

}  // namespace enufft
