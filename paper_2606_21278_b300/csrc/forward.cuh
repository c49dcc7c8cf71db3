// forward.cuh -- fused per-cell type-1 transform (+ optional EMS) for fine grids that fit in
// shared memory (n_f = 64 or 128).
//
// One persistent thread block takes cells from an atomic ticket queue (cells ordered largest
// first) and, for each cell, runs every step of Sec. 2.1.2 on chip:
//   1. window + scale (App. A/B): centred coordinates from binary64 per-cell constants through
//      exact binary32 transforms, the mask test (binary32 with a certified margin, binary64 when
//      a sample is closer than the margin to the boundary), c_q = w_q h_q / |D|;
//   2. spread c_q with the exponential-of-semicircle kernel onto a real n_f x n_f grid held in
//      shared memory with a halo (so no per-tap wrap arithmetic), then fold the halo (periodic).
//      The binary32 path accumulates in 32-bit fixed point with native integer shared-memory
//      reductions: a per-cell pre-pass bounds every node by S = sum |c_q| (the kernel is <= 1),
//      so each tap is rounded to an integer at scale 2^30 / S and no partial sum can overflow;
//      integer sums are also independent of the order in which samples arrive (bit-reproducible);
//   3. 2-D FFT: real rows in pairs (one complex FFT per pair, split by conjugate symmetry),
//      then the P/2 + 1 needed columns, each by a team of lanes (fft.cuh);
//   4. deconvolve by 1/(Phi(m) Phi(n)) and crop to m, n in [-P/2, P/2) (Hermitian fill of m < 0)
//      straight out of the column transforms into a staged P x P spectrum;
//   5. optionally rank the staged spectrum's mode pairs for EMS (ems.cuh, stage 1), then one
//      coalesced 16-byte-vector store of the spectrum.
// The grid origin is the paper's x' = u + H (App. A), so no phase correction is needed.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "ems.cuh"
#include "fft.cuh"

namespace enufft {

constexpr int kMaxHalf = 64;   // P/2 <= 64
constexpr int kSpreadPerThread = 4;   // samples per thread and chunk of the binary32 spreading

#ifndef ENUFFT_FWD_MINB
#define ENUFFT_FWD_MINB 2   // co-resident 512-thread blocks per SM of the binary32 fused kernels
#endif

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
    EmsScratch ems_out;   // stage-1 EMS results (top keys, counts) per cell
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
    static constexpr int MINB = (sizeof(T) == 4 && NF <= 128) ? ENUFFT_FWD_MINB : 1;
    static constexpr int NWARPS = NT / 32;
    static constexpr int N1 = FftSplit<NF>::N1, N2 = FftSplit<NF>::N2;
    static constexpr int WS_TEAM = team_ws<N1, N2>();          // workspace per team (complex)
    static constexpr int R_EMS = ((NF / 4) * (NF / 4) * 2 + NT - 1) / NT;   // >= J* / threads
    static constexpr size_t grid_bytes = sizeof(T) * (size_t)GR * GS;
    static constexpr size_t c1_bytes_min = sizeof(cplx<T>) * (size_t)NF * C1S_MAX;
    static constexpr size_t ems_bytes = ems_smem_bytes(NWARPS, kEmsMaxK);
    // binary32 spreading takes the samples in chunks of CHUNK, each staged as 16-byte records in the
    // half-spectrum area (free until the row transforms)
    static constexpr int CHUNK = NT * kSpreadPerThread;
    static constexpr size_t rec_bytes = sizeof(T) == 4 ? (size_t)CHUNK * 16 : 0;
    static constexpr size_t c1a_bytes = c1_bytes_min > ems_bytes ? c1_bytes_min : ems_bytes;
    static constexpr size_t c1_bytes = c1a_bytes > rec_bytes ? c1a_bytes : rec_bytes;
    static constexpr size_t tw_bytes = sizeof(cplx<T>) * NF;
    static constexpr size_t tail_bytes =
        sizeof(CellConst) + 16 + sizeof(T) * (kMaxHalf + 1) + 8 * NWARPS + 16 + 2 * 32 * sizeof(int);
    static constexpr size_t smem_bytes = grid_bytes + c1_bytes + tw_bytes + tail_bytes;
    // after the row pass the grid memory holds the staged P x P spectrum followed by the column
    // teams' workspaces
    static constexpr size_t stage_ws_bytes =
        sizeof(cplx<T>) * ((size_t)(NF / 2) * (NF / 2) + (size_t)C1S_MAX * WS_TEAM);
    static_assert(stage_ws_bytes <= grid_bytes, "staging + column workspace must fit in the grid memory");
    static_assert(GS >= WS_TEAM && GS >= NF + W + 2, "row workspace must fit in a padded row");
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

// binary32 window test with a certified margin: returns 1 inside, 0 outside, -1 undecided.  The
// window is the intersection of half-planes (the square B, and the cell's edges or the disk), so the
// test takes the largest excess over the constraints: outside where it exceeds the margin, inside
// where it is below minus the margin, undecided in between.  One multiply-add pair and one maximum
// per edge, over the cell's own edge count (coordinates are finite: callers test that first).
__device__ __forceinline__ int window_f32(const FastFrame& ff, const float4* __restrict__ edge, float ux, float uy) {
    const float tau = ff.tau;
    float f = fmaxf(fabsf(ux) - ff.Hf, fabsf(uy) - ff.Hf);
    if (ff.mask == 0) {
#pragma unroll 1
        for (int i = 0; i < ff.nv; ++i) {
            const float4 e = edge[i];
            f = fmaxf(f, __fmaf_rn(e.x, ux, __fmaf_rn(e.y, uy, -e.z)));
        }
    } else if (ff.mask == 2) {   // the disk's margin is 4 tau H on the squared radius
        const float fc = __fmaf_rn(ux, ux, __fmaf_rn(uy, uy, -ff.Hf * ff.Hf));
        const float t2 = 4.0f * tau * ff.Hf;
        if (fc > t2) return 0;
        if (fc > -t2) f = fmaxf(f, 0.0f);   // undecided unless the square already excludes it
    }
    if (f > tau) return 0;
    return f > -tau ? -1 : 1;
}

// The W kernel pieces at u from the first (W + 1) / 2 fits: the kernel is even, so piece W - 1 - i at
// u equals piece i at -u.  With p_i(u) = E_i(u^2) + u O_i(u^2) both come from one evaluation of the
// even and odd parts (Horner in u^2).
template <int W>
__device__ __forceinline__ void kernel_pieces_sym(const KernelPoly& kp, float u, float (&v)[W]) {
    constexpr int DEG = poly_deg(W), NE = (DEG + 1) / 2, NO = DEG / 2;
    const float u2 = u * u;
#pragma unroll
    for (int i = 0; i < (W + 1) / 2; ++i) {
        float e = kp.c[i][2 * (NE - 1)];
#pragma unroll
        for (int k = NE - 2; k >= 0; --k) e = __fmaf_rn(e, u2, kp.c[i][2 * k]);
        float o = kp.c[i][2 * (NO - 1) + 1];
#pragma unroll
        for (int k = NO - 2; k >= 0; --k) o = __fmaf_rn(o, u2, kp.c[i][2 * k + 1]);
        v[i] = __fmaf_rn(u, o, e);
        if (W - 1 - i != i) v[W - 1 - i] = __fmaf_rn(-u, o, e);
    }
}

// The three-edge case of window_f32 (triangular cells), the edges held in registers.
__device__ __forceinline__ int window_tri_f32(const FastFrame& ff, const float4& e0, const float4& e1, const float4& e2,
                                              float ux, float uy) {
    float f = fmaxf(fabsf(ux) - ff.Hf, fabsf(uy) - ff.Hf);
    f = fmaxf(f, __fmaf_rn(e0.x, ux, __fmaf_rn(e0.y, uy, -e0.z)));
    f = fmaxf(f, __fmaf_rn(e1.x, ux, __fmaf_rn(e1.y, uy, -e1.z)));
    f = fmaxf(f, __fmaf_rn(e2.x, ux, __fmaf_rn(e2.y, uy, -e2.z)));
    if (f > ff.tau) return 0;
    return f > -ff.tau ? -1 : 1;
}

// Per-sample setup shared by spreading and interpolation (binary32 path): window test, first
// node r0 of each dimension and the kernel argument there (prep_f32 adds the W kernel values).
// Returns false for samples outside the window (or non-finite ones, which also latch
// ST_NONFINITE).  This form takes the binary32 window test from the caller (win(ux, uy) as
// window_f32); prep_coords_f32 below uses window_f32 itself.
template <int NF, int W, typename Win>
__device__ __forceinline__ bool prep_coords_win_f32(const FastFrame& ff, const Win& win_f32, const CellConst& cc,
                                                    float px, float py, int& r0x, int& r0y, float& argx, float& argy,
                                                    unsigned* status) {
    if (!(isfinite(px) && isfinite(py))) {
        atomicOr(status, ST_NONFINITE);
        return false;
    }
    float uxh, uxl, uyh, uyl;
    two_diff(px, ff.cxh, uxh, uxl);
    uxl = __fsub_rn(uxl, ff.cxl);
    two_diff(py, ff.cyh, uyh, uyl);
    uyl = __fsub_rn(uyl, ff.cyl);
    int win = win_f32(uxh + uxl, uyh + uyl);
    if (win < 0) win = window_f64(cc, (double)px, (double)py);
    if (!win) return false;
    // grid coordinate s = u * (n_f / L) + n_f / 2; first node r0 = ceil(s - W/2);
    // t = r0 - s + W/2 in [0, 1) from the hi/lo pieces (one rounding at magnitude < 1)
    const float sx = __fmaf_rn(uxh, ff.sch, 0.5f * NF), sy = __fmaf_rn(uyh, ff.sch, 0.5f * NF);
    r0x = (int)ceilf(sx - 0.5f * W);
    r0y = (int)ceilf(sy - 0.5f * W);
    const float corrx = __fmaf_rn(uxh, ff.scl, uxl * ff.sch), corry = __fmaf_rn(uyh, ff.scl, uyl * ff.sch);
    const float tx = __fmaf_rn(-uxh, ff.sch, (float)(r0x - NF / 2) + 0.5f * W) - corrx;
    const float ty = __fmaf_rn(-uyh, ff.sch, (float)(r0y - NF / 2) + 0.5f * W) - corry;
    argx = __fmaf_rn(2.0f, tx, -1.0f);
    argy = __fmaf_rn(2.0f, ty, -1.0f);
    return true;
}

template <int NF, int W>
__device__ __forceinline__ bool prep_coords_f32(const FastFrame& ff, const float4* __restrict__ edge,
                                                const CellConst& cc, float px, float py, int& r0x, int& r0y,
                                                float& argx, float& argy, unsigned* status) {
    return prep_coords_win_f32<NF, W>(ff, [&](float ux, float uy) { return window_f32(ff, edge, ux, uy); }, cc, px, py,
                                      r0x, r0y, argx, argy, status);
}

template <int NF, int W>
__device__ __forceinline__ bool prep_f32(const FastFrame& ff, const float4* __restrict__ edge, const CellConst& cc,
                                         const KernelPoly& kp, float px, float py, int& r0x, int& r0y,
                                         float (&kx)[W], float (&ky)[W], unsigned* status) {
    float ax, ay;
    if (!prep_coords_f32<NF, W>(ff, edge, cc, px, py, r0x, r0y, ax, ay, status)) return false;
    kernel_pieces_sym<W>(kp, ax, kx);
    kernel_pieces_sym<W>(kp, ay, ky);
    return true;
}

// binary64 path: window in binary64, direct kernel evaluation (ES or KB, binary64)
template <int NF, int W>
__device__ __forceinline__ bool prep_f64(const CellConst& cc, const KernelPoly& kp, double beta, double px, double py,
                                         int& r0x, int& r0y, double (&kx)[W], double (&ky)[W], unsigned* status) {
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
        kx[i] = kernel_value_f64(kp, beta, zx);
        ky[i] = kernel_value_f64(kp, beta, zy);
    }
    return true;
}

// shared-memory 32-bit integer reduction (two's complement) with a compile-time immediate offset
template <int OFF>
__device__ __forceinline__ void red_smem(unsigned addr, int v) {
    asm volatile("red.shared.add.u32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF * 4));
}

// Rounding to the nearest integer by one multiply-add: for |v| < 2^22, v + 1.5 * 2^23 lies in
// [2^23, 2^24), where binary32 numbers are the integers, so the sum rounds v to the nearest integer
// and its bit pattern is that integer plus the pattern of 1.5 * 2^23.
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;

// the W x W taps of one sample: cs (c times the cell's fixed-point scale, |cs| <= 2^21) times the
// separable kernel, rounded to integers (products below 2^22 in magnitude)
template <int W, int GS, int J = 0, int I = 0>
__device__ __forceinline__ void spread_taps_rn(unsigned addr, const float (&kx)[W], const float (&ky)[W], float cj,
                                               float cs) {
    if constexpr (J < W) {
        if constexpr (I == 0) cj = cs * ky[J];
        if constexpr (I < W) {
            red_smem<J * GS + I>(addr, __float_as_int(__fmaf_rn(cj, kx[I], kRoundMagic)) - kRoundMagicBits);
            spread_taps_rn<W, GS, J, I + 1>(addr, kx, ky, cj, cs);
        } else {
            spread_taps_rn<W, GS, J + 1, 0>(addr, kx, ky, cj, cs);
        }
    }
}

// Ask L2 for the 128-byte lines of p[q0, q1): one prefetch per line (at an element inside the range),
// spread over the block's threads.
__device__ __forceinline__ void prefetch_l2(const float* __restrict__ p, int64_t q0, int64_t q1, int tid, int nt) {
    for (int64_t q = q0 + (int64_t)tid * 32; q < q1; q += (int64_t)nt * 32)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p + q));
}

// Binary32 spreading of one cell's samples [q0, q1) into the fixed-point grid at word offset 0 of
// `gaddr` (shared-memory address), conflict-free in the shared-memory banks.
//
// The 32 banks of a tap's address (base + j GS + i) differ between two samples exactly when their
// base words differ modulo 32, so samples are scheduled by their class = base mod 32: per chunk of
// CHUNK samples every thread prepares its samples (window, first node, kernel arguments, scaled
// weight) and takes a slot in its class with a shared counter; the records are placed class by
// class; then lane l of every warp spreads only class-l records (warp w takes rounds w, w + warps,
// ...), so the 32 reductions of one instruction always hit 32 different banks.  Integer
// reductions make the result independent of the order of the records.
template <int NF, int W, int GS, int HO, int NT>
__device__ __forceinline__ void spread_cell_f32(unsigned gaddr, int4* __restrict__ srec, int* __restrict__ shist,
                                                const FastFrame& ff, const float4* __restrict__ edge,
                                                const CellConst& cc, const KernelPoly& kp,
                                                const float* __restrict__ x, const float* __restrict__ y,
                                                const float* __restrict__ h, const float* __restrict__ w, int64_t q0,
                                                int64_t q1, float scale, unsigned* status) {
    constexpr int K = kSpreadPerThread, CH = NT * K, NWARPS = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool tri = ff.mask == 0 && ff.nv == 3;
    const float cscale = ff.inv_area * scale;
    int par = 0;
    for (int64_t c0 = q0; c0 < q1; c0 += CH, par ^= 1) {
        int* hist = shist + 32 * par;
        // samples c0 + tid + k NT of this chunk exist for k NT < nrem
        const int nrem = (int)(q1 - c0 < (int64_t)CH ? q1 - c0 : (int64_t)CH) - tid;
        const float *xc = x + c0 + tid, *yc = y + c0 + tid, *hc = h + c0 + tid, *wc = w + c0 + tid;
        float px[K], py[K], ph[K], pw[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool in = k * NT < nrem;
            px[k] = in ? xc[k * NT] : 0.0f;
            py[k] = in ? yc[k * NT] : 0.0f;
            ph[k] = in ? hc[k * NT] : 0.0f;
            pw[k] = in ? wc[k * NT] : 0.0f;
        }
        int4 rec[K];
        int cls[K], slot[K];
        auto prep = [&](const auto& win) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                cls[k] = -1;
                slot[k] = 0;
                rec[k] = make_int4(0, 0, 0, 0);
                int r0x, r0y;
                float ax, ay;
                if (k * NT < nrem && prep_coords_win_f32<NF, W>(ff, win, cc, px[k], py[k], r0x, r0y, ax, ay, status)) {
                    const float cs = pw[k] * ph[k] * cscale;
                    if (!isfinite(cs)) {
                        atomicOr(status, ST_NONFINITE);
                    } else {
                        const int word = (r0y + HO) * GS + (r0x + HO);
                        cls[k] = word & 31;
                        slot[k] = atomicAdd(&hist[cls[k]], 1);
                        rec[k] = make_int4(word, __float_as_int(ax), __float_as_int(ay), __float_as_int(cs));
                    }
                }
            }
        };
        if (tri) {   // triangles: the three edges in registers for the chunk
            const float4 e0 = edge[0], e1 = edge[1], e2 = edge[2];
            prep([&](float ux, float uy) { return window_tri_f32(ff, e0, e1, e2, ux, uy); });
        } else {
            prep([&](float ux, float uy) { return window_f32(ff, edge, ux, uy); });
        }
        __syncthreads();   // every slot taken; the previous chunk's records are spread
        if (warp == 0) shist[32 * (par ^ 1) + lane] = 0;   // the next chunk's counters
        const int cnt = hist[lane];                         // lane l: class l
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int start = incl - cnt;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int st = __shfl_sync(0xffffffffu, start, cls[k] & 31);
            if (cls[k] >= 0) srec[st + slot[k]] = rec[k];
        }
        int maxc = cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
        __syncthreads();   // records in place
        if (c0 + CH < q1) {   // the next chunk's samples toward L2 while this one is spread
            const int64_t n0 = c0 + CH, n1 = min(q1, c0 + 2 * CH);
            prefetch_l2(x, n0, n1, tid, NT);
            prefetch_l2(y, n0, n1, tid, NT);
            prefetch_l2(h, n0, n1, tid, NT);
            prefetch_l2(w, n0, n1, tid, NT);
        }
        for (int r = warp; r < maxc; r += NWARPS) {
            if (r < cnt) {
                const int4 rc = srec[start + r];
                float kx[W], ky[W];
                kernel_pieces_sym<W>(kp, __int_as_float(rc.y), kx);
                kernel_pieces_sym<W>(kp, __int_as_float(rc.z), ky);
                spread_taps_rn<W, GS>(gaddr + 4u * (unsigned)rc.x, kx, ky, 0.0f, __int_as_float(rc.w));
            }
        }
    }
}

// spread one sample (binary64 path)
template <int NF, int W, int GS, int HO>
__device__ __forceinline__ void spread_f64(double* __restrict__ g, const CellConst& cc, const KernelPoly& kp,
                                           double beta, double px, double py, double ph, double pw, unsigned* status) {
    int r0x, r0y;
    double kx[W], ky[W];
    if (!prep_f64<NF, W>(cc, kp, beta, px, py, r0x, r0y, kx, ky, status)) return;
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

// two fixed-point grid rows read as one complex row z = (row0 + i row1) / scale
struct FixedRowPairAcc {
    const int* r0;
    const int* r1;
    float inv_scale;
    __device__ __forceinline__ cplx<float> load(int i) const {
        return {(float)r0[i] * inv_scale, (float)r1[i] * inv_scale};
    }
};

// per-thread sum and maximum of |w_q h_q| / |D| over a cell's samples, reduced over the block (finite
// terms only); red holds 2 * NT / 32 floats
template <int NT>
__device__ __forceinline__ float2 cell_abs_sum_max(const float* __restrict__ h, const float* __restrict__ w, int64_t q0,
                                                   int64_t q1, float inv_area, float* red) {
    float s = 0.0f, m = 0.0f;
    int64_t q = q0 + threadIdx.x;
    for (; q + 3 * NT < q1; q += 4 * NT) {   // four independent sample pairs in flight
        float hv[4], wv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { hv[k] = h[q + k * NT]; wv[k] = w[q + k * NT]; }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v = fabsf(wv[k] * hv[k]);
            v = (v <= 3.0e38f) ? v : 0.0f;
            s += v;
            m = fmaxf(m, v);
        }
    }
    for (; q < q1; q += NT) {
        float v = fabsf(w[q] * h[q]);
        v = (v <= 3.0e38f) ? v : 0.0f;
        s += v;
        m = fmaxf(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        red[NT / 32 + (threadIdx.x >> 5)] = m;
    }
    __syncthreads();
    float t = 0.0f, mx = 0.0f;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        t += red[i];
        mx = fmaxf(mx, red[NT / 32 + i]);
    }
    return make_float2(t * inv_area, mx * inv_area);
}

// contiguous complex workspace accessor
template <typename T>
struct PlainAcc {
    cplx<T>* p;
    __device__ __forceinline__ cplx<T> load(int i) const { return p[i]; }
    __device__ __forceinline__ void store(int i, cplx<T> v) const { p[i] = v; }
};

// output of a column transform (column m, element k = n mod n_f): deconvolve and place it in the
// staged P x P spectrum, directly at (m, n) and by Hermitian symmetry at (-m, -n)
template <typename T, int NF>
struct DeconvStageOut {
    cplx<T>* stage;
    const T* inv_phi;
    int m, P, half;
    __device__ __forceinline__ void store(int k, cplx<T> z) const {
        const int n = k < NF / 2 ? k : k - NF;
        if (n < -half || n > half) return;
        const T f = inv_phi[m] * inv_phi[n < 0 ? -n : n];
        const cplx<T> v{z.re * f, z.im * f};
        if (m < half && n < half) stage[(n + half) * P + (m + half)] = v;
        if (m >= 1 && n > -half) stage[(half - n) * P + (half - m)] = cconj(v);
    }
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
    T* sinv = reinterpret_cast<T*>(sticket + 4);
    float* sred = reinterpret_cast<float*>(sinv + kMaxHalf + 1);   // 2 * NWARPS floats
    int* shist = reinterpret_cast<int*>(sred + 2 * CF::NWARPS);      // 2 x 32 class counters

    const int tid = threadIdx.x, lane = tid & 31;
    const int P = a.P, half = P / 2, C1S = half + 1;
    for (int i = tid; i < NF; i += CF::NT) stw[i] = a.twiddle[i];
    for (int i = tid; i <= half; i += CF::NT) sinv[i] = a.inv_phi[i];
    float inv_scale = 1.0f;   // fixed-point scale of the current cell (binary32 path)

    // tickets: the current cell and, one ahead, the next one (whose samples are requested toward L2
    // while the current cell is transformed)
    if (tid == 0) {
        sticket[0] = (int)atomicAdd(a.ticket, 1u);
        sticket[1] = (int)atomicAdd(a.ticket, 1u);
    }
    for (;;) {
        __syncthreads();   // also orders the previous cell's last shared-memory reads
        const int tk = sticket[0], tkn = sticket[1];
        if (tk >= a.n_work) break;
        const int cell = a.order[tk];
        const int ncell = tkn < a.n_work ? a.order[tkn] : -1;
        {   // per-cell constants into shared memory; zero the padded grid
            const int4* src = reinterpret_cast<const int4*>(a.cells + cell);
            int4* dst = reinterpret_cast<int4*>(scc);
            for (int i = tid; i < (int)(sizeof(CellConst) / 16); i += CF::NT) dst[i] = src[i];
            float4* g4 = reinterpret_cast<float4*>(sgrid);
            const int n4 = (int)(CF::grid_bytes / 16);
            for (int i = tid; i < n4; i += CF::NT) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tid < 64) shist[tid] = 0;
        }
        __syncthreads();
        const CellConst& cc = *scc;
        // ---- step 1+2: window, scale, spread
        if (cc.valid) {
            const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
            int64_t q = q0 + tid;
            if constexpr (sizeof(T) == 4) {
                const FastFrame ff = fast_frame(cc);
                // fixed-point scale: every node of the grid is bounded by S = sum |c_q| (the kernel is
                // <= 1), and every tap by max |c_q|; 2^30 / S keeps the nodes in 32 bits, 2^21 / max
                // keeps each tap below 2^22, where one multiply-add rounds it to an integer
                const float2 sm = cell_abs_sum_max<CF::NT>(a.h, a.w, q0, q1, ff.inv_area, sred);
                const float scale = sm.x > 0x1p-96f ? fminf(0x1p30f / sm.x, 0x1p21f / sm.y) : 0x1p126f;
                inv_scale = 1.0f / scale;
                spread_cell_f32<NF, W, GS, HO, CF::NT>((unsigned)__cvta_generic_to_shared(sgrid),
                                                       reinterpret_cast<int4*>(sC1), shist, ff, cc.edge, cc,
                                                       a.poly, a.x, a.y, a.h, a.w, q0, q1, scale, a.status);
            } else {
                for (; q < q1; q += CF::NT)
                    spread_f64<NF, W, GS, HO>(sgrid, cc, a.poly, a.beta, a.x[q], a.y[q], a.h[q], a.w[q],
                                              a.status);
            }
        } else if (tid == 0) {
            atomicOr(a.status, ST_BADCELL);
        }
        __syncthreads();
        // ---- periodic fold of the halo: columns first (all padded rows), then rows (exact integer
        // adds on the binary32 path's fixed-point grid)
        using Acc = typename std::conditional<sizeof(T) == 4, int, double>::type;
        Acc* sacc = reinterpret_cast<Acc*>(sgrid);
        for (int i = tid; i < GR * (GR - NF); i += CF::NT) {
            const int r = i / (GR - NF), k = i % (GR - NF);
            const int c = k < HO ? k : k + NF;              // halo column
            const int cw = k < HO ? k + NF : k;             // its periodic image inside the core
            sacc[r * GS + cw] += sacc[r * GS + c];
        }
        __syncthreads();
        for (int i = tid; i < (GR - NF) * NF; i += CF::NT) {
            const int k = i / NF, c = HO + i % NF;
            const int r = k < HO ? k : k + NF;
            const int rw = k < HO ? k + NF : k;
            sacc[rw * GS + c] += sacc[r * GS + c];
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            if (ncell >= 0) {   // the next cell's weights and elevations (its sum pass) and first samples
                const int64_t n0 = a.offsets[ncell], n1 = a.offsets[ncell + 1];
                prefetch_l2(a.h, n0, min(n1, n0 + 16384), tid, CF::NT);
                prefetch_l2(a.w, n0, min(n1, n0 + 16384), tid, CF::NT);
                prefetch_l2(a.x, n0, min(n1, n0 + CF::CHUNK), tid, CF::NT);
                prefetch_l2(a.y, n0, min(n1, n0 + CF::CHUNK), tid, CF::NT);
            }
        }
        // ---- step 3a: FFT of the rows, two real rows per complex transform; keep m = 0..P/2
        {
            const int team = tid / N2, t = tid % N2;
            const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
            if (team < NF / 2) {
                T* r0 = sgrid + (HO + 2 * team) * GS;
                T* r1 = r0 + GS;
                // input in the core columns, transposed workspace and output from column 0
                if constexpr (sizeof(T) == 4) {
                    const int* i0 = reinterpret_cast<const int*>(r0) + HO;
                    team_fft<N1, N2, T>(FixedRowPairAcc{i0, i0 + GS, inv_scale}, RowPairAcc<T>{r0, r1},
                                        RowPairAcc<T>{r0, r1}, t, stw, tmask);
                } else {
                    team_fft<N1, N2, T>(RowPairAcc<T>{r0 + HO, r1 + HO}, RowPairAcc<T>{r0, r1}, RowPairAcc<T>{r0, r1},
                                        t, stw, tmask);
                }
                for (int m = t; m <= half; m += N2) {
                    const int mn = (NF - m) & (NF - 1);
                    const T zr = r0[m], zi = r1[m], wr = r0[mn], wi = r1[mn];
                    sC1[(2 * team) * C1S + m] = cplx<T>{T(0.5) * (zr + wr), T(0.5) * (zi - wi)};
                    sC1[(2 * team + 1) * C1S + m] = cplx<T>{T(0.5) * (zi + wi), T(0.5) * (wr - zr)};
                }
            }
        }
        __syncthreads();
        // ---- step 3b + 4: FFT of the columns m = 0..P/2, deconvolved and cropped into the stage
        cplx<T>* stage = reinterpret_cast<cplx<T>*>(sgrid);
        {
            const int team = tid / N2, t = tid % N2;
            const unsigned tmask = ((1u << N2) - 1u) << (lane & ~(N2 - 1));
            if (team <= half) {
                cplx<T>* wk = stage + (size_t)(NF / 2) * (NF / 2) + (size_t)team * CF::WS_TEAM;
                team_fft<N1, N2, T>(StridedAcc<T, false>{sC1 + team, C1S}, PlainAcc<T>{wk},
                                    DeconvStageOut<T, NF>{stage, sinv, team, P, half}, t, stw, tmask);
            }
        }
        __syncthreads();
        // ---- step 5: EMS on the staged spectrum (shared scratch in the free half-spectrum area)
        if (a.do_ems)
            ems_rank_block<T, CF::R_EMS>(StagedSpec<T>{stage, P, half}, P, cell, a.ems, a.ems_out,
                                         reinterpret_cast<unsigned char*>(sC1));
        {   // coalesced 16-byte stores of the P x P spectrum
            const float4* s4 = reinterpret_cast<const float4*>(stage);
            float4* d4 = reinterpret_cast<float4*>(a.coeffs + (size_t)cell * P * P * 2);
            const int n4 = P * P * (int)sizeof(cplx<T>) / 16;
            for (int i = tid; i < n4; i += CF::NT) d4[i] = s4[i];
        }
        if (tid == 0) {
            sticket[0] = sticket[1];
            sticket[1] = (int)atomicAdd(a.ticket, 1u);
        }
    }
}

}  // namespace enufft
