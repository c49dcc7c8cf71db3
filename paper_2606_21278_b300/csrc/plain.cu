// plain.cu -- the plain binary32 per-cell path: for every cell its own launch sequence
//   memset of an n_f x n_f binary32 grid in global memory,
//   spread: one thread per sample, window test, kernel taps exp(beta (sqrt(1 - z^2) - 1)) by expf,
//           global atomicAdd of every tap (Sec. 2.1, Eq. discrete_quadrature scaled by 1/|D|),
//   row FFTs: one block per row, radix-2 in shared memory,
//   column FFTs: one block per retained column,
//   deconvolve and crop to the P x P modes.
// This is the straightforward GPU rendering of the type-1 transform, kept as the comparison
// point for the fused kernels; it shares with them only the frame constants and the window test.
#include "forward.cuh"
#include "internal.h"

namespace enufft {

// kernel value at z in [-1, 1] in binary32 library calls: ES exp(beta (sqrt(1 - z^2) - 1)) or KB
// I0(gamma sqrt(1 - z^2)) / I0(gamma)
__device__ __forceinline__ float plain_kernel(int kind, float shape, float inv_norm, float z) {
    const float r = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    return kind == KERNEL_KB ? cyl_bessel_i0f(shape * r) * inv_norm : expf(shape * (r - 1.0f));
}

static __global__ void __launch_bounds__(256) plain_spread_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                                  const float* __restrict__ h, const float* __restrict__ w,
                                                                  int64_t q0, int64_t q1, const CellConst* __restrict__ cells,
                                                                  int cell, int NF, int W, float beta, int kind,
                                                                  float inv_norm, float* grid, unsigned* status) {
    const CellConst& cc = cells[cell];
    const int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1 || !cc.valid) return;
    const float px = x[q], py = y[q];
    if (!(isfinite(px) && isfinite(py))) {
        atomicOr(status, ST_NONFINITE);
        return;
    }
    const FastFrame ff = fast_frame(cc);
    const float ux = (px - cc.cxh) - cc.cxl, uy = (py - cc.cyh) - cc.cyl;
    int win = window_f32(ff, cc.edge, ux, uy);
    if (win < 0) win = window_f64(cc, (double)px, (double)py);
    if (!win) return;
    const float c = w[q] * h[q] * cc.inv_area;
    if (!isfinite(c)) {
        atomicOr(status, ST_NONFINITE);
        return;
    }
    const float sx = ux * cc.sch + 0.5f * NF, sy = uy * cc.sch + 0.5f * NF;
    const int r0x = (int)ceilf(sx - 0.5f * W), r0y = (int)ceilf(sy - 0.5f * W);
    const float zs = 2.0f / W;
    float kx[kMaxW];
    for (int i = 0; i < W; ++i) {
        const float z = ((float)(r0x + i) - sx) * zs;
        kx[i] = plain_kernel(kind, beta, inv_norm, z);
    }
    for (int j = 0; j < W; ++j) {
        const float z = ((float)(r0y + j) - sy) * zs;
        const float cy = c * plain_kernel(kind, beta, inv_norm, z);
        float* row = grid + (size_t)((r0y + j) & (NF - 1)) * NF;
        for (int i = 0; i < W; ++i) atomicAdd(row + ((r0x + i) & (NF - 1)), cy * kx[i]);
    }
}

// in-place radix-2 decimation-in-time FFT (forward, e^{-2 pi i jk/N}) of s[0..N) after bit reversal
__device__ __forceinline__ void plain_fft_smem(cplx<float>* s, const cplx<float>* __restrict__ tw, int N) {
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1, step = N / len;
        for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
            const int i0 = (k / half) * len + (k % half), i1 = i0 + half;
            const cplx<float> t = cmul(s[i1], tw[(k % half) * step]);
            const cplx<float> u = s[i0];
            s[i0] = cadd(u, t);
            s[i1] = csub(u, t);
        }
        __syncthreads();
    }
}

static __global__ void plain_fft_rows_kernel(const float* __restrict__ grid, cplx<float>* __restrict__ buf,
                                             const cplx<float>* __restrict__ tw, int NF, int lg) {
    extern __shared__ cplx<float> s[];
    const int row = blockIdx.x;
    for (int i = threadIdx.x; i < NF; i += blockDim.x)
        s[__brev((unsigned)i) >> (32 - lg)] = cplx<float>{grid[(size_t)row * NF + i], 0.0f};
    __syncthreads();
    plain_fft_smem(s, tw, NF);
    for (int i = threadIdx.x; i < NF; i += blockDim.x) buf[(size_t)row * NF + i] = s[i];
}

static __global__ void plain_fft_cols_kernel(cplx<float>* __restrict__ buf, const cplx<float>* __restrict__ tw, int NF,
                                             int lg, int P) {
    extern __shared__ cplx<float> s[];
    const int col = (blockIdx.x - P / 2) & (NF - 1);
    for (int i = threadIdx.x; i < NF; i += blockDim.x) s[__brev((unsigned)i) >> (32 - lg)] = buf[(size_t)i * NF + col];
    __syncthreads();
    plain_fft_smem(s, tw, NF);
    for (int i = threadIdx.x; i < NF; i += blockDim.x) buf[(size_t)i * NF + col] = s[i];
}

struct PlainInv {
    float v[kMaxHalf + 1];
};

static __global__ void plain_deconv_kernel(const cplx<float>* __restrict__ buf, int NF, int P, const PlainInv inv,
                                           cplx<float>* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * P) return;
    const int n = i / P - P / 2, m = i % P - P / 2;
    const float f = inv.v[m < 0 ? -m : m] * inv.v[n < 0 ? -n : n];
    const cplx<float> z = buf[(size_t)(n & (NF - 1)) * NF + (m & (NF - 1))];
    out[i] = cplx<float>{z.re * f, z.im * f};
}

cudaError_t plain_run(const PlainRun& r, cudaStream_t s) {
    int lg = 0;
    while ((1 << lg) < r.NF) ++lg;
    PlainInv inv;
    for (int k = 0; k <= r.P / 2; ++k) inv.v[k] = (float)r.inv_phi[k];
    const size_t smem = sizeof(cplx<float>) * r.NF;
    const int fthreads = r.NF / 2 < 32 ? 32 : r.NF / 2;
    for (int64_t j = 0; j < r.n_cells; ++j) {
        cudaError_t e = cudaMemsetAsync(r.grid, 0, sizeof(float) * r.NF * r.NF, s);
        if (e != cudaSuccess) return e;
        const int64_t q0 = r.h_off[j], q1 = r.h_off[j + 1];
        if (q1 > q0)
            plain_spread_kernel<<<(unsigned)((q1 - q0 + 255) / 256), 256, 0, s>>>(r.x, r.y, r.h, r.w, q0, q1, r.cells, (int)j,
                                                                                  r.NF, r.W, r.beta, r.kind, r.inv_norm, r.grid,
                                                                                  r.status);
        plain_fft_rows_kernel<<<r.NF, fthreads, smem, s>>>(r.grid, r.buf, r.twiddle, r.NF, lg);
        plain_fft_cols_kernel<<<r.P, fthreads, smem, s>>>(r.buf, r.twiddle, r.NF, lg, r.P);
        plain_deconv_kernel<<<(r.P * r.P + 255) / 256, 256, 0, s>>>(r.buf, r.NF, r.P, inv,
                                                                    r.coeffs + (size_t)j * r.P * r.P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace enufft
