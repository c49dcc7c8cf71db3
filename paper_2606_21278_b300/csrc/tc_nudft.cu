// tc_nudft.cu -- direct NUDFT of small cells on the tensor cores (Eq. discrete_quadrature as a
// dense contraction):
//
//   h^[n][m] = (1/|D|) sum_q win_q w_q h_q e^{-i k_n y'_q} e^{-i k_m x'_q},   k = 2 pi / L,
//
// i.e. D = A^T B with A[q][.] = c_q (e^{-i k_n y'_q})_n and B[q][.] = (e^{-i k_m' x'_q})_m'.  The
// samples are real, so the spectrum is Hermitian, h^(-m, -n) = conj h^(m, n), and the phasor of -m'
// is the conjugate of that of m': A carries only n = 0 .. P/2 and B only m' = 0 .. P/2.  With
// P1 = D[re n][re m'], P2 = D[im n][im m'], P3 = D[im n][re m'], P4 = D[re n][im m']
//   h^[n][ m'] = (P1 - P2) + i (P3 + P4),   h^[n][-m'] = (P1 + P2) + i (P3 - P4),
// and the rows n < 0 are the conjugates of these.  Complex values are stacked as real features:
// A has 128 (the real and imaginary parts of n = 1 .. 32 alternate in blocks of 16, so both sit in
// one 32-lane quarter of the accumulator; the real weight of n = 0 at feature 64; features 65 ..
// 127 carry whatever the buffer holds and their accumulator rows are never read), B has 80
// (likewise for m' = 0 .. 31, then the real and imaginary parts of m' = 32), so one 128 x 80 real
// product per 16 samples carries the whole P x P complex result (P <= 64).
// Each value is split into binary16 hi + lo and the product is accumulated in binary32 as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo * lo term is below 2^-22 of the scale).  The samples'
// weights are scaled by 1 / max |c| of the cell so that every operand lies in [-1, 1].
//
// The tensor core adds the products of every MMA to the binary32 accumulator without rounding to
// nearest, so the accumulator error grows with the number of MMAs it absorbs; each accumulator run
// is therefore limited to 256 samples (two banks of TMEM columns alternate), and every thread adds
// its lane's part of a finished run into a running total, also in TMEM, with round-to-nearest
// binary32 additions (no shared memory, no block barrier).  At the end of a cell each spectrum
// entry is formed by one operand thread, which combines the four products of its accumulator lane
// with those of the lane 16 apart by shuffles.
//
// One CTA per cell at a time (two per SM), warp-specialised: two set-up warps each prepare every
// other chunk of samples (window, scaled weight, coordinates, unit phasor steps) into a ring of four
// set-up buffers, with the samples of their next chunk already loaded; one warp issues the tcgen05
// MMAs; eight operand warps turn each chunk of 32 samples into binary16 operands in shared memory
// (four stages), warps 0-3 the B octets and warps 4-7 the A octets, one task per thread.  The
// hand-offs are mbarriers with bounded waits (set-up ready, set-up read, operands written, MMAs
// done), so the operand warps never wait on a block-wide barrier inside a cell.  The spectrum is
// written out and ranked for EMS (Sec. 2.2).
#include <cuda_fp16.h>

#include "ems.cuh"
#include "forward.cuh"
#include "internal.h"
#include "tc.cuh"

namespace enufft {

namespace {

constexpr int kFeatThreads = 256;                         // warps 0..7: operands, TMEM read-back
constexpr int kMmaWarp = kFeatThreads / 32;               // warp 8: MMA issue
constexpr int kPrepWarp0 = kMmaWarp + 1;                  // warps 9, 10: sample set-up of stage 0, 1
constexpr int kTcThreads = kFeatThreads + 3 * 32;
constexpr int kCh = 32;                                   // samples per chunk (K of one stage)
constexpr int kFeatA = 128, kFeatB = 80;                  // stacked features of A (n >= 0) and B (m' >= 0)
using LayA = tc::OpLayout<kFeatA>;
using LayB = tc::OpLayout<kFeatB>;
constexpr unsigned kOpA = kCh * kFeatA * 2;               // one A operand (8 KB)
constexpr unsigned kOpB = kCh * kFeatB * 2;               // one B operand (5 KB)
constexpr unsigned kStageBytes = 2 * kOpA + 2 * kOpB;     // A_hi, A_lo, B_hi, B_lo
constexpr int kStages = 4;                                // operand stages (chunk g uses g % 4)
constexpr int kHS = 65;                                   // row stride (complex) of the staged spectrum
// at the end of a cell the staged spectrum and the EMS scratch take the free stage memory
constexpr unsigned kSpecOff = 0;
constexpr unsigned kSpecBytes = 64 * kHS * 8;
constexpr unsigned kEmsOff = kSpecOff + kSpecBytes;
constexpr unsigned kEmsBytes = (unsigned)((ems_smem_bytes(kTcThreads / 32, kEmsMaxK) + 15) / 16 * 16);
constexpr int kPrepF = 9;                                 // per sample: c, tx hi/lo, ty hi/lo, x and y steps
constexpr int kPrepBufs = 4;                             // ring of set-up buffers (chunk g uses g % 4)
constexpr unsigned kPrepOff = kStages * kStageBytes;
constexpr unsigned kPrepBytes = kPrepBufs * kPrepF * kCh * 4;
constexpr unsigned kMiscOff = kPrepOff + kPrepBytes;
constexpr unsigned kSmemBytes = kMiscOff + 192;
constexpr unsigned kWaitLimit = 1u << 17;                // polls of a bounded wait (about 2.6 s)
constexpr int kBlockChunks = 8;                           // chunks accumulated per TMEM run (256 samples)
constexpr unsigned kTmemCols = 256;                       // run banks at columns 0 and 128, the total beside
static_assert(kEmsOff + kEmsBytes <= kStages * kStageBytes, "spectrum and EMS scratch fit the stage memory");
static_assert(kCh % 16 == 0 && LayA::off(kFeatA - 1, kCh - 1) < kOpA && LayB::off(kFeatB - 1, kCh - 1) < kOpB,
              "operand layout");
static_assert(kStageBytes % 16 == 0 && kOpA % 16 == 0 && kOpB % 16 == 0, "descriptor alignment");
static_assert(kFeatThreads == 8 * kCh, "one (sample, feature octet) task per operand thread and axis");
static_assert(144 + 4 * (kTcThreads / 32) <= 192, "barriers, TMEM base and warp maxima fit the misc area");

constexpr int kFeatN0 = 64;   // A feature of the mode n = 0 (features 65 .. 127 of A are never read)

// feature of the real part of the first mode of octet o (modes 8 o + 1 .. 8 o + 8 of A, 8 o .. 8 o + 7
// of B, o < 4): blocks of 16 real parts followed by their 16 imaginary parts; the imaginary part of a
// mode is 16 features later, except in B's last octet (m' = 32 .. 39: real 64.., imaginary 72..)
__host__ __device__ constexpr int feat_re(int o) { return 32 * (o >> 1) + 8 * (o & 1); }
__host__ __device__ constexpr int feat_im_b(int o) { return o == 4 ? 72 : feat_re(o) + 16; }

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

// c e^{-2 pi i m (t + 1/2)} for m = m0 .. m0 + 7 (t = th + tl, |t| <= 1/2; (wr, wi) = -e^{-2 pi i t}),
// zero from slot `lim` on unless FULL.  The anchor m0 takes one fast sine/cosine of an argument
// reduced to [-pi, pi] (absolute error below 1e-6); the 7 rotations use the accurate step.
template <bool FULL>
__device__ __forceinline__ void tc_phasors(float th, float tl, float wr, float wi, float c, int m0, int slot0, int lim,
                                           float (&re)[8], float (&im)[8], float& nr8, float& ni8) {
    const float fm0 = (float)m0;
    const float p = fm0 * th;
    const float r = (p - rintf(p)) + __fmaf_rn(fm0, tl, __fmaf_rn(fm0, th, -p));
    float s0, c0;
    __sincosf(6.283185307179586f * r, &s0, &c0);
    const float sg = (m0 & 1) ? -c : c;
    float zr = sg * c0, zi = -sg * s0;     // c (-1)^{m0} e^{-2 pi i m0 t}
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool on = FULL || slot0 + j < lim;
        re[j] = on ? zr : 0.0f;
        im[j] = on ? zi : 0.0f;
        const float nr = zr * wr - zi * wi, ni = zr * wi + zi * wr;
        zr = nr;
        zi = ni;
    }
    nr8 = zr;   // the mode m0 + 8
    ni8 = zi;
}

// Setup of one sample (Sec. 2.1, App. A): window test, scaled weight c / max |c|, and the centred
// coordinates u / L of both axes as binary32 hi + lo and the unit steps -e^{-2 pi i u/L}; writes
// slot k of a prep buffer (zeros for absent, outside or non-finite samples; the latter also latch
// ST_NONFINITE).
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
    float sx, cx, sy, cy;
    sincospif(2.0f * (txh + txl), &sx, &cx);
    sincospif(2.0f * (tyh + tyl), &sy, &cy);
    pr[k] = c;
    pr[kCh + k] = txh;
    pr[2 * kCh + k] = txl;
    pr[3 * kCh + k] = tyh;
    pr[4 * kCh + k] = tyl;
    pr[5 * kCh + k] = -cx;
    pr[6 * kCh + k] = sx;
    pr[7 * kCh + k] = -cy;
    pr[8 * kCh + k] = sy;
}

// two binary32 values -> binary16 hi = rn(v) and lo = rn(v - hi), packed in pairs (v0 in the low
// halves).  v - hi is exact in binary32 and formed by one mixed-precision multiply-add per value
// (hi * -1 + v, hi read as binary16), so there is no conversion of hi back to binary32.
__device__ __forceinline__ void tc_split2(float v0, float v1, unsigned& hi, unsigned& lo) {
    asm("{\n\t.reg .f16 h0, h1, m1;\n\t.reg .f32 r0, r1;\n\t"
        "cvt.rn.f16x2.f32 %0, %3, %2;\n\t"
        "mov.b32 {h0, h1}, %0;\n\t"
        "mov.b16 m1, 0xBC00;\n\t"
        "fma.rn.f32.f16 r0, h0, m1, %2;\n\t"
        "fma.rn.f32.f16 r1, h1, m1, %3;\n\t"
        "cvt.rn.f16x2.f32 %1, r1, r0;\n\t}"
        : "=r"(hi), "=r"(lo)
        : "f"(v0), "f"(v1));
}

// eight binary32 values -> binary16 hi and lo octets (16 bytes each)
__device__ __forceinline__ void tc_split8(const float (&v)[8], uint4& hi, uint4& lo) {
    unsigned hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tc_split2(v[2 * j], v[2 * j + 1], hw[j], lw[j]);
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// TMEM column of column c (0 .. 79) of the running total: columns 80 .. 127 and 208 .. 255, beside
// the two 80-column run banks at 0 and 128
__device__ __forceinline__ unsigned total_col(int c) { return c < 48 ? 80u + (unsigned)c : 160u + (unsigned)c; }

// The thread's lane of the finished run in `bank` into the running total (the first run of a cell
// is copied).  Warp w takes lane quarter w & 3 and the accumulator columns of its B modes:
// 0 .. 31 (w < 4) or 32 .. 79 (w >= 4).
__device__ __forceinline__ void tc_accumulate(unsigned tmem, unsigned bank, int warp, bool first) {
    const unsigned lanes = (unsigned)(32 * (warp & 3)) << 16;
    const int nseg = warp < 4 ? 4 : 6, c0 = warp < 4 ? 0 : 32;
#pragma unroll 1
    for (int sg = 0; sg < nseg; ++sg) {   // 8 columns at a time
        const int c = c0 + 8 * sg;
        float v[8], t[8];
        tc::tmem_ld8(tmem + lanes + bank + (unsigned)c, v);
        if (!first) tc::tmem_ld8(tmem + lanes + total_col(c), t);
        tc::tmem_ld_wait();
        if (!first) {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __fadd_rn(v[j], t[j]);
        }
        tc::tmem_st8(tmem + lanes + total_col(c), v);
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
}

// The cell's spectrum from the running total, scaled by `scale`, into hs (every entry written by
// one operand thread).  Warp w reads lane quarter w & 3 and the B modes m' = 16 (w >> 2) .. + 15
// (plus m' = 32 for w >> 2 == 1).  Quarters 0 and 1 hold the A features 32 q + l: the real (l < 16)
// or imaginary (l >= 16) part of the mode n = 16 q + (l & 15) + 1; lanes l and l ^ 16 exchange
// their products, lane l < 16 forms h^(m', n) and lane l >= 16 h^(-m', n), and each also writes
// the conjugate at (-m, -n) (the samples are real).  Quarter 2's lane 0 holds n = 0 (real weight
// only): its lanes 0 and 16 form h^(m', 0) and h^(-m', 0).  A cell without chunks (`empty`) gets
// zeros.
__device__ __forceinline__ void tc_combine(unsigned tmem, cplx<float>* hs, int warp, int lane, int P, float scale,
                                           bool empty) {
    const int lq = warp & 3, hh = warp >> 2, half = P / 2;
    const unsigned lanes = (unsigned)(32 * lq) << 16;
    float vr[16], vi[16];
    float xr = 0.0f, xi = 0.0f;
    if (!empty) {
        tc::tmem_ld16(tmem + lanes + total_col(32 * hh), vr);        // D[f][re m'],  m' = 16 hh + j
        tc::tmem_ld16(tmem + lanes + total_col(32 * hh + 16), vi);   // D[f][im m']
        if (hh == 1) {                                               // m' = 32
            xr = tc::tmem_ld1(tmem + lanes + total_col(64));
            xi = tc::tmem_ld1(tmem + lanes + total_col(72));
        }
        tc::tmem_ld_wait();
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) vr[j] = vi[j] = 0.0f;
    }
    const bool up = lane < 16;
    const bool zrow = lq == 2;                            // n = 0 (lanes 0 and 16 only)
    const int n = zrow ? 0 : 16 * lq + (lane & 15) + 1;
    const bool live = lq < 2 ? n <= half : (zrow && (lane & 15) == 0);
    cplx<float>* row = hs + (n + half) * kHS;             // row n (direct entries, n <= half - 1)
    cplx<float>* crow = hs + (half - n) * kHS;            // row -n (conjugates)
    const bool direct = live && n <= half - 1;
    const bool conj = live && !zrow;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float pr = __shfl_xor_sync(0xffffffffu, vr[j], 16), pi = __shfl_xor_sync(0xffffffffu, vi[j], 16);
        const int mp = 16 * hh + j;
        // lane < 16: vr = P1, vi = P4, pr = P3, pi = P2;  lane >= 16: vr = P3, vi = P2, pr = P1, pi = P4
        // (row n = 0: P2 = P3 = 0, the lane-16 values unused)
        float re, im;
        if (zrow) {
            re = up ? vr[j] : pr;
            im = up ? vi[j] : -pi;
        } else {
            re = up ? vr[j] - pi : pr + vi[j];
            im = up ? pr + vi[j] : vr[j] - pi;
        }
        re *= scale;
        im *= scale;
        if (up) {   // (m', n), m' <= half - 1; conjugate at (-m', -n), m' <= half
            if (direct && mp <= half - 1) row[half + mp] = cplx<float>{re, im};
            if (conj && mp <= half) crow[half - mp] = cplx<float>{re, -im};
        } else {    // (-m', n), 1 <= m' <= half; conjugate at (m', -n) for m' <= half - 1
            if (mp >= 1 && mp <= half) {
                if (direct) row[half - mp] = cplx<float>{re, im};
                if (conj && mp <= half - 1) crow[half + mp] = cplx<float>{re, -im};
            }
        }
    }
    if (hh == 1 && half == 32) {   // m' = 32: (-32, n) from the lane >= 16 side, (32, n) only as the
                                   // conjugate (-32, -n) from the lane < 16 side
        const float pr = __shfl_xor_sync(0xffffffffu, xr, 16), pi = __shfl_xor_sync(0xffffffffu, xi, 16);
        float re, im;
        if (zrow) {
            re = up ? xr : pr;
            im = up ? xi : -pi;
        } else {
            re = up ? xr - pi : pr + xi;
            im = up ? pr + xi : xr - pi;
        }
        re *= scale;
        im *= scale;
        if (up) {
            if (conj) crow[0] = cplx<float>{re, -im};
        } else {
            if (direct) row[0] = cplx<float>{re, im};
        }
    }
}

template <bool FULL>
__global__ void __launch_bounds__(kTcThreads, 2) tc_nudft_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tsmem[];
    unsigned char* smem = tsmem;
    cplx<float>* hs = reinterpret_cast<cplx<float>*>(smem + kSpecOff);
    float* prep = reinterpret_cast<float*>(smem + kPrepOff);
    unsigned char* ems_sm = smem + kEmsOff;
    unsigned long long* bar_mma = reinterpret_cast<unsigned long long*>(smem + kMiscOff);   // [4] MMAs done
    unsigned long long* bar_full = bar_mma + kStages;                                        // [4] operands written
    unsigned long long* bar_prep = bar_full + kStages;                                       // [4] set-up ready
    unsigned long long* bar_pfree = bar_prep + kPrepBufs;                                    // [4] set-up read
    unsigned* tbase = reinterpret_cast<unsigned*>(smem + kMiscOff + 128);
    float* red = reinterpret_cast<float*>(smem + kMiscOff + 144);   // one per warp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = a.P, half = P / 2;

    if (warp == 0) {
        tc::tmem_alloc(tc::smem_addr(tbase), kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(tc::smem_addr(&bar_mma[s]), 1);
            tc::mbar_init(tc::smem_addr(&bar_full[s]), kFeatThreads);
        }
        for (int b = 0; b < kPrepBufs; ++b) {
            tc::mbar_init(tc::smem_addr(&bar_prep[b]), 1);
            tc::mbar_init(tc::smem_addr(&bar_pfree[b]), kFeatThreads / 32);
        }
        tc::mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const unsigned tmem = *tbase;
    const unsigned sbase = tc::smem_addr(smem);
    const unsigned idesc = tc::idesc_f16_f32_mn(kFeatA, kFeatB);
    unsigned g = 0;   // chunks of this CTA so far (stage g % 4, use g / 4 of the stage)

    for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
        const int cell = a.list[li];
        const CellConst& cc = a.cells[cell];
        const int64_t q0 = a.offsets[cell], q1 = a.offsets[cell + 1];
        const bool valid = cc.valid != 0;
        // ---- the samples toward L2 ahead of use: this cell's coordinates when it is the CTA's first,
        // the next cell's four arrays always (the control warp's one-chunk lookahead then waits on
        // L2, not on DRAM)
        if (li == (int)blockIdx.x) {
            prefetch_l2(a.x, q0, q1, tid, kTcThreads);
            prefetch_l2(a.y, q0, q1, tid, kTcThreads);
        }
        if (li + (int)gridDim.x < a.n_list) {
            const int nc = a.list[li + gridDim.x];
            const int64_t n0 = a.offsets[nc], n1 = a.offsets[nc + 1];
            prefetch_l2(a.x, n0, n1, tid, kTcThreads);
            prefetch_l2(a.y, n0, n1, tid, kTcThreads);
            prefetch_l2(a.h, n0, n1, tid, kTcThreads);
            prefetch_l2(a.w, n0, n1, tid, kTcThreads);
        }
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

        if (warp == kMmaWarp) {
            // ---- MMA warp: the three split products of each chunk once its operands are written
            for (int ch = 0; ch < nch; ++ch) {
                const unsigned gc = g + ch, st = gc % kStages;
                if (!tc::mbar_wait(tc::smem_addr(&bar_full[st]), (gc / kStages) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                tc::fence_after_sync();
                if (lane == 0) {
                    const unsigned s0 = sbase + st * kStageBytes;
                    const unsigned acc = tmem + 128u * ((ch / kBlockChunks) & 1);
                    const bool first = ch % kBlockChunks == 0;
#pragma unroll
                    for (int s = 0; s < kCh / 16; ++s) {
                        const uint64_t ah = tc::smem_desc(s0 + s * LayA::kKStep, LayA::kLbo, LayA::kSbo);
                        const uint64_t al = tc::smem_desc(s0 + kOpA + s * LayA::kKStep, LayA::kLbo, LayA::kSbo);
                        const uint64_t bh = tc::smem_desc(s0 + 2 * kOpA + s * LayB::kKStep, LayB::kLbo, LayB::kSbo);
                        const uint64_t bl = tc::smem_desc(s0 + 2 * kOpA + kOpB + s * LayB::kKStep, LayB::kLbo, LayB::kSbo);
                        tc::mma_f16(acc, ah, bh, idesc, (!first || s > 0) ? 1u : 0u);
                        tc::mma_f16(acc, ah, bl, idesc, 1u);
                        tc::mma_f16(acc, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(tc::smem_addr(&bar_mma[st]));
                }
                __syncwarp();
            }
        } else if (warp >= kPrepWarp0) {
            // ---- set-up warp sp: chunks ch with (g + ch) & 1 == sp, each into set-up buffer
            // (g + ch) % 4 once the operand warps have read the chunk four before from it
            const unsigned sp = (unsigned)(warp - kPrepWarp0);
            const FastFrame ff = fast_frame(cc);
            const float inv_nf = 1.0f / (float)a.NF;
            float rx = 0.f, ry = 0.f, rh = 0.f, rw = 0.f;
            bool rv = false;
            auto load = [&](int ch) {
                const int64_t q = q0 + (int64_t)ch * kCh + lane;
                rv = ch < nch && q < q1;
                if (rv) {
                    rx = a.x[q];
                    ry = a.y[q];
                    rh = a.h[q];
                    rw = a.w[q];
                }
            };
            const int c0 = (int)((sp - g) & 1u);
            if (c0 < nch) load(c0);
            for (int ch = c0; ch < nch; ch += 2) {
                const unsigned gc = g + ch, b = gc % kPrepBufs;
                if (gc >= kPrepBufs &&
                    !tc::mbar_wait(tc::smem_addr(&bar_pfree[b]), (gc / kPrepBufs - 1) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                tc_prep_sample(ff, cc, rv, rx, ry, rh, rw, inv_cm, inv_nf, prep + b * kPrepF * kCh, lane, a.status);
                if (ch + 2 < nch) load(ch + 2);
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar_prep[b]));
            }
        } else {
            // ---- operand warps
            const int k = (lane & 7) + 8 * (warp & 3), o = (lane >> 3) + 4 * (warp >> 2);
            for (int ch = 0; ch < nch; ++ch) {
                const unsigned gc = g + ch, st = gc % kStages, use = gc / kStages, b = gc % kPrepBufs;
                if (use > 0 && !tc::mbar_wait(tc::smem_addr(&bar_mma[st]), (use - 1) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                if (ch >= 2 * kBlockChunks && ch % kBlockChunks == 0) {
                    // the run two blocks back is complete (the stage wait covers every earlier MMA):
                    // add it to the running total before its bank is reused
                    tc::fence_after_sync();
                    tc_accumulate(tmem, 128u * ((ch / kBlockChunks) & 1), warp, ch == 2 * kBlockChunks);
                }
                // this chunk's set-up values into registers; the buffer is then free for the set-up warps
                if (!tc::mbar_wait(tc::smem_addr(&bar_prep[b]), (gc / kPrepBufs) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                const float* pr = prep + b * kPrepF * kCh;
                // warps 0-3 take the B octets (x), warps 4-7 the A octets (y): one task per thread
                float ta, tl, wa, wi, ca = 0.f;
                if (warp < 4) {
                    ta = pr[1 * kCh + k];
                    tl = pr[2 * kCh + k];
                    wa = pr[5 * kCh + k];
                    wi = pr[6 * kCh + k];
                } else {
                    ca = pr[k];
                    ta = pr[3 * kCh + k];
                    tl = pr[4 * kCh + k];
                    wa = pr[7 * kCh + k];
                    wi = pr[8 * kCh + k];
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar_pfree[b]));
                unsigned char* stg = smem + st * kStageBytes;
                if (warp >= 4) {   // A: modes n = 8 o' + 1 .. 8 o' + 8 (y) times the scaled weight, o' = o - 4
                    const int oa = o - 4;
                    float re[8], im[8], r8, i8;
                    tc_phasors<FULL>(ta, tl, wa, wi, ca, 8 * oa + 1, 8 * oa, half, re, im, r8, i8);
                    uint4 rh, rl, ih, il;
                    tc_split8(re, rh, rl);
                    tc_split8(im, ih, il);
                    const unsigned fr = LayA::off(feat_re(oa), k), fi = LayA::off(feat_re(oa) + 16, k);
                    *reinterpret_cast<uint4*>(stg + fr) = rh;
                    *reinterpret_cast<uint4*>(stg + kOpA + fr) = rl;
                    *reinterpret_cast<uint4*>(stg + fi) = ih;
                    *reinterpret_cast<uint4*>(stg + kOpA + fi) = il;
                    if (oa == 0) {   // n = 0: the real weight alone, at feature kFeatN0
                        const __half chh = __float2half_rn(ca);
                        const __half chl = __float2half_rn(ca - __half2float(chh));
                        const unsigned f0 = LayA::off(kFeatN0, k);
                        *reinterpret_cast<uint4*>(stg + f0) = make_uint4(__half_as_ushort(chh), 0u, 0u, 0u);
                        *reinterpret_cast<uint4*>(stg + kOpA + f0) = make_uint4(__half_as_ushort(chl), 0u, 0u, 0u);
                    }
                }
                if (warp < 4) {   // B: modes m' = 8 o .. 8 o + 7 (x), o < 4; octet 3 also writes m' = 32 .. 39
                    float re[8], im[8], r8, i8;
                    tc_phasors<FULL>(ta, tl, wa, wi, 1.0f, 8 * o, 8 * o, half + 1, re, im, r8, i8);
                    uint4 rh, rl, ih, il;
                    tc_split8(re, rh, rl);
                    tc_split8(im, ih, il);
                    unsigned char* bhi = stg + 2 * kOpA;
                    const unsigned fr = LayB::off(feat_re(o), k), fi = LayB::off(feat_im_b(o), k);
                    *reinterpret_cast<uint4*>(bhi + fr) = rh;
                    *reinterpret_cast<uint4*>(bhi + kOpB + fr) = rl;
                    *reinterpret_cast<uint4*>(bhi + fi) = ih;
                    *reinterpret_cast<uint4*>(bhi + kOpB + fi) = il;
                    if (o == 3) {   // m' = 32 (P = 64 only) followed by seven zero features
                        const float e = FULL ? r8 : 0.0f, f = FULL ? i8 : 0.0f;
                        const __half eh = __float2half_rn(e), fh = __float2half_rn(f);
                        const __half el = __float2half_rn(e - __half2float(eh)), fl = __float2half_rn(f - __half2float(fh));
                        rh = make_uint4(__half_as_ushort(eh), 0u, 0u, 0u);
                        rl = make_uint4(__half_as_ushort(el), 0u, 0u, 0u);
                        ih = make_uint4(__half_as_ushort(fh), 0u, 0u, 0u);
                        il = make_uint4(__half_as_ushort(fl), 0u, 0u, 0u);
                        const unsigned gr = LayB::off(feat_re(4), k), gi = LayB::off(feat_im_b(4), k);
                        *reinterpret_cast<uint4*>(bhi + gr) = rh;
                        *reinterpret_cast<uint4*>(bhi + kOpB + gr) = rl;
                        *reinterpret_cast<uint4*>(bhi + gi) = ih;
                        *reinterpret_cast<uint4*>(bhi + kOpB + gi) = il;
                    }
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                tc::mbar_arrive(tc::smem_addr(&bar_full[st]));
            }
            // ---- the last one or two runs into the total; once every MMA is done the stage memory is
            // free and takes the spectrum, scaled back by max |c|
            if (nch > 0) {
                const unsigned gl = g + nch - 1;
                if (!tc::mbar_wait(tc::smem_addr(&bar_mma[gl % kStages]), (gl / kStages) & 1u, kWaitLimit))
                    atomicOr(a.status, ST_TIMEOUT);
                tc::fence_after_sync();
                const int nb = (nch + kBlockChunks - 1) / kBlockChunks;
                for (int b = nb >= 2 ? nb - 2 : 0; b < nb; ++b)
                    tc_accumulate(tmem, 128u * (b & 1), warp, b == 0);
            }
            tc_combine(tmem, hs, warp, lane, P, cm, nch == 0);
        }
        g += (unsigned)nch;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
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
    // ---- every issued MMA has completed (each cell's operand warps waited for its last commit)
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// one block waiting on an mbarrier that never completes (no arrivals): the bounded wait gives up
static __global__ void tc_wait_timeout_kernel(unsigned polls, unsigned* status) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_addr(&bar), 1);
        tc::mbar_init_fence();
    }
    __syncthreads();
    if (!tc::mbar_wait(tc::smem_addr(&bar), 0u, polls) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

cudaError_t launch_wait_timeout(unsigned polls, unsigned* status, cudaStream_t s) {
    tc_wait_timeout_kernel<<<1, 32, 0, s>>>(polls, status);
    return cudaGetLastError();
}

cudaError_t tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(tc_nudft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_nudft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    return e;
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
    if (l.P == 64) tc_nudft_kernel<true><<<grid, kTcThreads, kSmemBytes, s>>>(a);
    else tc_nudft_kernel<false><<<grid, kTcThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace enufft
