// tc_nudft.cu -- direct NUDFT of small cells on the tensor cores (Eq. discrete_quadrature as a
// dense contraction):
//
//   h^[n][m] = (1/|D|) sum_q win_q w_q h_q e^{-i k_n y'_q} e^{-i k_m x'_q},   k = 2 pi / L,
//
// i.e. D = A^T B with A[q][.] = c_q (e^{-i k_n y'_q})_n and B[q][.] = (e^{-i k_m x'_q})_m over the
// samples q of the cell.  Complex values are stacked as real features (rows 0..63 the real parts
// of modes -P/2 .. P/2-1, rows 64..127 the imaginary parts), so one 128 x 128 real product per
// 16 samples carries the whole P x P complex result (P <= 64):
//   Re h^ = D[re n][re m] - D[im n][im m],   Im h^ = D[re n][im m] + D[im n][re m].
// Each value is split into binary16 hi + lo and the product is accumulated in binary32 as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo * lo term is below 2^-22 of the scale).  The samples'
// weights are scaled by 1 / max |c| of the cell so that every operand lies in [-1, 1].
//
// The tensor core adds the products of every MMA to the binary32 accumulator without rounding to
// nearest, so the accumulator error grows with the number of MMAs it absorbs; each accumulator run
// is therefore limited to 256 samples (two banks of 128 TMEM columns alternate), and finished runs
// are added into the staged spectrum in shared memory with round-to-nearest binary32 additions.
//
// One CTA per cell at a time (two per SM): chunks of 32 samples are turned into operands in shared
// memory (double buffered) by all threads while one thread issues the tcgen05 MMAs of the previous
// chunk; the accumulator lives in tensor memory and is read back once per cell, combined through
// shared memory, written out and ranked for EMS (Sec. 2.2).
#include <cuda_fp16.h>

#include "ems.cuh"
#include "forward.cuh"
#include "internal.h"
#include "tc.cuh"

namespace enufft {

namespace {

constexpr int kTcThreads = 256;
constexpr int kCh = 32;                                   // samples per chunk (K of one stage)
constexpr unsigned kOpBytes = kCh * tc::kTcFeat * 2;      // one operand (8 KB)
constexpr unsigned kStageBytes = 4 * kOpBytes;            // A_hi, A_lo, B_hi, B_lo
constexpr int kHS = 65;                                   // row stride (complex) of the staged spectrum
constexpr unsigned kSpecOff = 2 * kStageBytes;
constexpr unsigned kSpecBytes = 64 * kHS * 8;
constexpr unsigned kPrepOff = kSpecOff + kSpecBytes;
constexpr unsigned kPrepBytes = 2 * 5 * kCh * 4;          // per stage: c, tx hi/lo, ty hi/lo
constexpr unsigned kEmsOff = kPrepOff + kPrepBytes;
constexpr unsigned kEmsBytes = (unsigned)((ems_smem_bytes(kTcThreads / 32, kEmsMaxK) + 15) / 16 * 16);
constexpr unsigned kMiscOff = kEmsOff + kEmsBytes;
constexpr unsigned kSmemBytes = kMiscOff + 128;
constexpr unsigned kWaitLimit = 1u << 22;
constexpr int kBlockChunks = 8;                           // chunks accumulated per TMEM run (256 samples)
constexpr unsigned kTmemCols = 256;                       // two 128-column accumulator banks
static_assert(kCh % 16 == 0 && tc::tc_off(127, kCh - 1) < kOpBytes, "operand layout");
static_assert(kTcThreads == 8 * kCh, "one (sample, feature octet) task per thread and axis");

struct TcSpec {
    const cplx<float>* hs;
    int half;
    __device__ __forceinline__ cplx<float> get(int m, int n) const { return hs[(n + half) * kHS + (m + half)]; }
};

}  // namespace

struct TcArgs {
    const float* __restrict__ x;
    const float* __restrict__ y;
    const float* __restrict__ h;
    const float* __restrict__ w;
    const int64_t* __restrict__ offsets;
    const CellConst* __restrict__ cells;
    const int* __restrict__ list;     // cells of this route
    int n_list, P, NF;
    cplx<float>* __restrict__ coeffs;
    unsigned* status;
    int do_ems;
    EmsArgs ems;
    EmsScratch ems_out;
};

// e^{-2 pi i m (t + 1/2)} for m = m0 .. m0 + 7 (t = th + tl, |t| <= 1/2), zero beyond slot P
__device__ __forceinline__ void tc_phasors(float th, float tl, int m0, int slot0, int P, float (&re)[8], float (&im)[8]) {
    const float fm0 = (float)m0;
    const float p = fm0 * th;
    const float r = (p - rintf(p)) + __fmaf_rn(fm0, tl, __fmaf_rn(fm0, th, -p));
    float s0, c0, s1, c1;
    sincospif(2.0f * r, &s0, &c0);
    sincospif(2.0f * (th + tl), &s1, &c1);
    const float sg = (m0 & 1) ? -1.0f : 1.0f;
    float zr = sg * c0, zi = -sg * s0;     // (-1)^{m0} e^{-2 pi i m0 t}
    const float wr = -c1, wi = s1;         // step: -e^{-2 pi i t}
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool on = slot0 + j < P;
        re[j] = on ? zr : 0.0f;
        im[j] = on ? zi : 0.0f;
        const float nr = zr * wr - zi * wi, ni = zr * wi + zi * wr;
        zr = nr;
        zi = ni;
    }
}

// Setup of one sample (Sec. 2.1, App. A): window test, scaled weight c / max |c|, and the centred
// coordinates u / L of both axes as binary32 hi + lo; writes slot k of a prep buffer (zeros for
// absent, outside or non-finite samples; the latter also latch ST_NONFINITE).
__device__ __forceinline__ void tc_prep_sample(const FastFrame& ff, const CellConst& cc, bool present, float px,
                                               float py, float hv, float wv, float inv_cm, float inv_nf, float* pr,
                                               int k, unsigned* status) {
    float c = 0.0f, txh = 0.0f, txl = 0.0f, tyh = 0.0f, tyl = 0.0f;
    if (present) {
        if (!(isfinite(px) && isfinite(py))) {
            atomicOr(status, ST_NONFINITE);
        } else {
            float uxh, uxl, uyh, uyl;
            two_diff(px, ff.cxh, uxh, uxl);
            uxl = __fsub_rn(uxl, ff.cxl);
            two_diff(py, ff.cyh, uyh, uyl);
            uyl = __fsub_rn(uyl, ff.cyl);
            int win = window_f32(ff, cc.edge, uxh + uxl, uyh + uyl);
            if (win < 0) win = window_f64(cc, (double)px, (double)py);
            if (win) {
                const float cv = wv * hv * ff.inv_area;
                if (!isfinite(cv)) {
                    atomicOr(status, ST_NONFINITE);
                } else {
                    c = cv * inv_cm;
                    const float qx = uxh * ff.sch, qy = uyh * ff.sch;
                    txh = qx * inv_nf;
                    txl = (__fmaf_rn(uxh, ff.sch, -qx) + __fmaf_rn(uxh, ff.scl, uxl * ff.sch)) * inv_nf;
                    tyh = qy * inv_nf;
                    tyl = (__fmaf_rn(uyh, ff.sch, -qy) + __fmaf_rn(uyh, ff.scl, uyl * ff.sch)) * inv_nf;
                }
            }
        }
    }
    pr[k] = c;
    pr[kCh + k] = txh;
    pr[2 * kCh + k] = txl;
    pr[3 * kCh + k] = tyh;
    pr[4 * kCh + k] = tyl;
}

// eight binary32 values -> binary16 hi and lo octets (16 bytes each)
__device__ __forceinline__ void tc_split8(const float (&v)[8], uint4& hi, uint4& lo) {
    unsigned hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __half2 hh = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
        hw[j] = *reinterpret_cast<const unsigned*>(&hh);
        lw[j] = *reinterpret_cast<const unsigned*>(&ll);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// hs[n][m] += (D[re n][re m] - D[im n][im m], D[re n][im m] + D[im n][re m]) for one accumulator
// bank; every thread of the block takes part (TMEM lane quarter warp & 3, column half warp >> 2)
__device__ __forceinline__ void tc_flush(unsigned bank, cplx<float>* hs, int warp, int lane) {
    const int lg = warp & 3, chh = warp >> 2;
    const int row = 32 * lg + lane;
    const unsigned ta = bank + ((unsigned)(32 * lg) << 16) + 32 * chh;
    float vr[32], vi[32];
    {
        float t0[16], t1[16], t2[16], t3[16];
        tc::tmem_ld16(ta, t0);
        tc::tmem_ld16(ta + 16, t1);
        tc::tmem_ld16(ta + 64, t2);
        tc::tmem_ld16(ta + 80, t3);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            vr[j] = t0[j];
            vr[16 + j] = t1[j];
            vi[j] = t2[j];
            vi[16 + j] = t3[j];
        }
    }
    cplx<float>* dst = hs + (row & 63) * kHS + 32 * chh;
    if (row < 64) {
#pragma unroll
        for (int j = 0; j < 32; ++j) dst[j] = cplx<float>{dst[j].re + vr[j], dst[j].im + vi[j]};
    }
    __syncthreads();
    if (row >= 64) {
#pragma unroll
        for (int j = 0; j < 32; ++j) dst[j] = cplx<float>{dst[j].re - vi[j], dst[j].im + vr[j]};
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

static __global__ void __launch_bounds__(kTcThreads, 2) tc_nudft_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tsmem[];
    unsigned char* smem = tsmem;
    cplx<float>* hs = reinterpret_cast<cplx<float>*>(smem + kSpecOff);
    float* prep = reinterpret_cast<float*>(smem + kPrepOff);
    unsigned char* ems_sm = smem + kEmsOff;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + kMiscOff);
    unsigned* tbase = reinterpret_cast<unsigned*>(smem + kMiscOff + 16);
    float* red = reinterpret_cast<float*>(smem + kMiscOff + 32);   // 8 warps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = a.P, half = P / 2;

    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tbase), kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&mbar[0]), 1);
        tc::mbar_init(tc::smem_addr(&mbar[1]), 1);
        tc::mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const unsigned tmem = *tbase;
    const unsigned sbase = tc::smem_addr(smem);
    const unsigned idesc = tc::idesc_f16_f32_mn(128, 128);
    unsigned g = 0;   // chunks issued by this CTA (stage = g & 1, use = g >> 1)

    for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
        const int cell = a.list[li];
        const CellConst& cc = a.cells[cell];
        const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
        const bool valid = cc.valid != 0;
        // ---- scale: max |w h| / |D| over the cell (binary32)
        float cm = 0.0f;
        if (valid)
            for (int64_t q = q0 + tid; q < q1; q += kTcThreads) {
                const float v = fabsf(a.w[q] * a.h[q] * cc.inv_area);
                if (v <= 3.0e38f) cm = fmaxf(cm, v);
            }
        for (int o = 16; o; o >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        if (lane == 0) red[warp] = cm;
        __syncthreads();
        cm = 0.0f;
        for (int i = 0; i < kTcThreads / 32; ++i) cm = fmaxf(cm, red[i]);
        const float inv_cm = cm > 0.0f ? 1.0f / cm : 0.0f;
        const int nch = (valid && cm > 0.0f) ? (int)((q1 - q0 + kCh - 1) / kCh) : 0;
        const FastFrame ff = fast_frame(cc);
        const float inv_nf = 1.0f / (float)a.NF;
        for (int i = tid; i < 64 * kHS; i += kTcThreads) hs[i] = cplx<float>{0.0f, 0.0f};

        if (nch > 0) {
            if (tid < kCh) {
                const int64_t q = q0 + tid;
                const bool ok = q < q1;
                tc_prep_sample(ff, cc, ok, ok ? a.x[q] : 0.0f, ok ? a.y[q] : 0.0f, ok ? a.h[q] : 0.0f,
                               ok ? a.w[q] : 0.0f, inv_cm, inv_nf, prep + (g & 1u) * 5 * kCh, tid, a.status);
            }
            __syncthreads();
        }
        for (int ch = 0; ch < nch; ++ch, ++g) {
            const unsigned st = g & 1u, use = g >> 1;
            if (use > 0 && !tc::mbar_wait(tc::smem_addr(&mbar[st]), (use - 1) & 1u, kWaitLimit))
                atomicOr(a.status, ST_TIMEOUT);
            if (ch >= 2 * kBlockChunks && ch % kBlockChunks == 0) {
                // the run two blocks back is complete (the stage wait covers every earlier MMA):
                // add it to the staged spectrum before its bank is reused
                tc::fence_after_sync();
                tc_flush(tmem + 128u * ((ch / kBlockChunks) & 1), hs, warp, lane);
            }
            const float* pr = prep + st * 5 * kCh;
            // the raw samples of the next chunk are loaded now and set up after this chunk's operands
            const int64_t qn = q0 + (int64_t)(ch + 1) * kCh + tid;
            const bool load_next = tid < kCh && ch + 1 < nch && qn < q1;
            float nx = 0.0f, ny = 0.0f, nh = 0.0f, nw = 0.0f;
            if (load_next) {
                nx = a.x[qn];
                ny = a.y[qn];
                nh = a.h[qn];
                nw = a.w[qn];
            }
            // ---- operands: task (axis, sample k, feature octet o); axis 0 -> A (y, times c), 1 -> B (x)
            unsigned char* stg = smem + st * kStageBytes;
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) {
                const int k = (lane & 7) + 8 * (warp & 3), o = (lane >> 3) + 4 * (warp >> 2);
                const float th = pr[(ax ? 1 : 3) * kCh + k], tl = pr[(ax ? 2 : 4) * kCh + k];
                float re[8], im[8];
                tc_phasors(th, tl, 8 * o - half, 8 * o, P, re, im);
                if (ax == 0) {
                    const float c = pr[k];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        re[j] *= c;
                        im[j] *= c;
                    }
                }
                uint4 rh, rl, ih, il;
                tc_split8(re, rh, rl);
                tc_split8(im, ih, il);
                unsigned char* hi = stg + (ax ? 2 : 0) * kOpBytes;
                unsigned char* lo = hi + kOpBytes;
                *reinterpret_cast<uint4*>(hi + tc::tc_off(8 * o, k)) = rh;
                *reinterpret_cast<uint4*>(lo + tc::tc_off(8 * o, k)) = rl;
                *reinterpret_cast<uint4*>(hi + tc::tc_off(64 + 8 * o, k)) = ih;
                *reinterpret_cast<uint4*>(lo + tc::tc_off(64 + 8 * o, k)) = il;
            }
            if (tid < kCh && ch + 1 < nch)
                tc_prep_sample(ff, cc, load_next, nx, ny, nh, nw, inv_cm, inv_nf, prep + (st ^ 1u) * 5 * kCh, tid, a.status);
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const unsigned s0 = sbase + st * kStageBytes;
                const unsigned acc = tmem + 128u * ((ch / kBlockChunks) & 1);
                const bool first = ch % kBlockChunks == 0;
#pragma unroll
                for (int s = 0; s < kCh / 16; ++s) {
                    const uint64_t ah = tc::smem_desc(s0 + s * 4096, tc::kTcLbo, tc::kTcSbo);
                    const uint64_t al = tc::smem_desc(s0 + kOpBytes + s * 4096, tc::kTcLbo, tc::kTcSbo);
                    const uint64_t bh = tc::smem_desc(s0 + 2 * kOpBytes + s * 4096, tc::kTcLbo, tc::kTcSbo);
                    const uint64_t bl = tc::smem_desc(s0 + 3 * kOpBytes + s * 4096, tc::kTcLbo, tc::kTcSbo);
                    tc::mma_f16(acc, ah, bh, idesc, (!first || s > 0) ? 1u : 0u);
                    tc::mma_f16(acc, ah, bl, idesc, 1u);
                    tc::mma_f16(acc, al, bh, idesc, 1u);
                }
                tc::mma_commit(tc::smem_addr(&mbar[st]));
            }
        }
        // ---- epilogue: the last one or two runs -> staged spectrum, scaled back by max |c|
        if (nch > 0) {
            const unsigned gl = g - 1;
            if (!tc::mbar_wait(tc::smem_addr(&mbar[gl & 1u]), (gl >> 1) & 1u, kWaitLimit)) atomicOr(a.status, ST_TIMEOUT);
            tc::fence_after_sync();
            const int nb = (nch + kBlockChunks - 1) / kBlockChunks;
            for (int b = nb >= 2 ? nb - 2 : 0; b < nb; ++b) tc_flush(tmem + 128u * (b & 1), hs, warp, lane);
            for (int i = tid; i < 64 * kHS; i += kTcThreads) hs[i] = cplx<float>{hs[i].re * cm, hs[i].im * cm};
        }
        __syncthreads();
        {
            float2* out = reinterpret_cast<float2*>(a.coeffs + (size_t)cell * P * P);
            for (int i = tid; i < P * P; i += kTcThreads) {
                const cplx<float> z = hs[(i / P) * kHS + (i % P)];
                out[i] = make_float2(z.re, z.im);
            }
        }
        if (a.do_ems) ems_rank_block<float, 8>(TcSpec{hs, half}, P, cell, a.ems, a.ems_out, ems_sm);
        __syncthreads();
    }
    // ---- every issued MMA has completed (each cell's epilogue waited for its last commit)
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

cudaError_t tc_prepare() {
    return cudaFuncSetAttribute(tc_nudft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

cudaError_t launch_tc_nudft(const TcLaunch& l, cudaStream_t s) {
    if (l.n_list <= 0) return cudaSuccess;
    TcArgs a;
    a.x = l.x;
    a.y = l.y;
    a.h = l.h;
    a.w = l.w;
    a.offsets = l.offsets;
    a.cells = l.cells;
    a.list = l.list;
    a.n_list = l.n_list;
    a.P = l.P;
    a.NF = l.NF;
    a.coeffs = l.coeffs;
    a.status = l.status;
    a.do_ems = l.ems ? 1 : 0;
    if (l.ems) a.ems = *l.ems;
    else memset(&a.ems, 0, sizeof(a.ems));
    a.ems_out = l.ems_out;
    const int grid = l.n_list < 2 * l.num_sms ? l.n_list : 2 * l.num_sms;
    tc_nudft_kernel<<<grid, kTcThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enufft
