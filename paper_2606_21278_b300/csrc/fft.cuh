// fft.cuh -- small power-of-two FFTs for the per-cell fine grids (Sec. 2.1.2, step 3).
//
// A length-N transform (N = N1 * N2, N = 64, 128 or 256) is done by a "team" of N2 consecutive
// lanes of one warp with the four-step split
//     Z[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} W_N^{n2 k1} sum_n1 z[N2 n1 + n2] W_N1^{n1 k1},
// each lane holding N1 (step 1) or N2 (step 2) values in registers and exchanging them once
// through shared memory.  The data live wherever the accessor says (a grid row pair, a column
// of the half spectrum, ...), so the same code serves the row and the column passes.
#pragma once

#include "common.cuh"

namespace enufft {

// bit reversal of i over log2(N) bits (folded at compile time inside unrolled loops)
template <int N>
__host__ __device__ constexpr int brev_c(int i) {
    int r = 0;
    for (int b = 1, m = N >> 1; b < N; b <<= 1, m >>= 1)
        if (i & b) r |= m;
    return r;
}

// a * e^{-2 pi i k / 16}; k is a compile-time constant after unrolling, so the branches fold
template <typename T>
__device__ __forceinline__ cplx<T> mul_tw16(cplx<T> a, int k) {
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), r = T(0.70710678118654752440);
    switch (k & 15) {
        case 0: return a;
        case 1: return cmul(a, cplx<T>{c1, -s1});
        case 2: return {(a.re + a.im) * r, (a.im - a.re) * r};
        case 3: return cmul(a, cplx<T>{s1, -c1});
        case 4: return {a.im, -a.re};
        case 5: return cmul(a, cplx<T>{-s1, -c1});
        case 6: return {(a.im - a.re) * r, -(a.re + a.im) * r};
        case 7: return cmul(a, cplx<T>{-c1, -s1});
        case 8: return {-a.re, -a.im};
        default: return cmul(a, cplx<T>{T(0), T(0)});   // not reached for N <= 16
    }
}

// one radix-2 DIT stage of span LEN, then the next (compile-time recursion keeps every index static)
template <int N, int LEN, typename T>
__device__ __forceinline__ void fft_stages(cplx<T> (&a)[N]) {
    if constexpr (LEN <= N) {
#pragma unroll
        for (int i = 0; i < N; i += LEN) {
#pragma unroll
            for (int k = 0; k < LEN / 2; ++k) {
                cplx<T> u = a[i + k];
                cplx<T> v = mul_tw16(a[i + k + LEN / 2], k * (16 / LEN));
                a[i + k] = cadd(u, v);
                a[i + k + LEN / 2] = csub(u, v);
            }
        }
        fft_stages<N, 2 * LEN, T>(a);
    }
}

template <int N, int I, typename T>
__device__ __forceinline__ void bit_reverse(cplx<T> (&a)[N]) {
    if constexpr (I < N) {
        constexpr int J = brev_c<N>(I);
        if constexpr (I < J) {
            cplx<T> t = a[I];
            a[I] = a[J];
            a[J] = t;
        }
        bit_reverse<N, I + 1, T>(a);
    }
}

// In-register forward DFT of length N in {2, 4, 8, 16}, natural order in and out (radix-2 DIT).
template <int N, typename T>
__device__ __forceinline__ void fft_reg(cplx<T> (&a)[N]) {
    bit_reverse<N, 0, T>(a);
    fft_stages<N, 2, T>(a);
}

// Team FFT.  The team is lanes [base, base + N2) of a warp with team-relative lane t; tw is the
// table W_N^j = e^{-2 pi i j / N}, j in [0, N).  Input element n comes from in.load(n); the
// transposed intermediate goes through the workspace `wk` (N2 rows of N1 + 1 entries, the padding
// keeping the transpose free of bank conflicts); output element k goes to out.store(k, .), natural
// order.  The three may alias: every load of a phase completes before the next phase stores.
// Requires N1 >= N2.
template <int N1, int N2, typename T, typename In, typename Wk, typename Out>
__device__ __forceinline__ void team_fft(const In& in, const Wk& wk, const Out& out, int t,
                                         const cplx<T>* __restrict__ tw, unsigned team_mask) {
    static_assert(N1 >= N2 && N1 % N2 == 0, "team FFT split");
    constexpr int WS = N1 + 1;
    cplx<T> a[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) a[n1] = in.load(N2 * n1 + t);
    fft_reg<N1, T>(a);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) a[k1] = cmul(a[k1], tw[t * k1]);
    __syncwarp(team_mask);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) wk.store(t * WS + k1, a[k1]);
    __syncwarp(team_mask);
    constexpr int KK = N1 / N2;
    cplx<T> b[KK][N2];
#pragma unroll
    for (int kk = 0; kk < KK; ++kk) {
        const int k1 = t + kk * N2;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) b[kk][n2] = wk.load(n2 * WS + k1);
        fft_reg<N2, T>(b[kk]);
    }
    __syncwarp(team_mask);
#pragma unroll
    for (int kk = 0; kk < KK; ++kk)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) out.store(t + kk * N2 + N1 * k2, b[kk][k2]);
    __syncwarp(team_mask);
}

// workspace entries a team needs for length N
template <int N1, int N2>
constexpr int team_ws() { return N2 * (N1 + 1); }

// split of a power-of-two length over a team: N = N1 * N2 with N1 >= N2
template <int N>
struct FftSplit;
template <>
struct FftSplit<64> { static constexpr int N1 = 8, N2 = 8; };
template <>
struct FftSplit<128> { static constexpr int N1 = 16, N2 = 8; };
template <>
struct FftSplit<256> { static constexpr int N1 = 16, N2 = 16; };

// accessor: two real rows seen as one complex row z = row0 + i row1 (shared memory)
template <typename T>
struct RowPairAcc {
    T* r0;
    T* r1;
    __device__ __forceinline__ cplx<T> load(int i) const { return {r0[i], r1[i]}; }
    __device__ __forceinline__ void store(int i, cplx<T> v) const { r0[i] = v.re; r1[i] = v.im; }
};

// accessor: two real rows, read and written conjugated (for the inverse transform through
// conj(FFT(conj(z))) on a row pair)
template <typename T>
struct RowPairConjAcc {
    T* r0;
    T* r1;
    __device__ __forceinline__ cplx<T> load(int i) const { return {r0[i], -r1[i]}; }
    __device__ __forceinline__ void store(int i, cplx<T> v) const { r0[i] = v.re; r1[i] = -v.im; }
};

// accessor: strided complex vector (shared memory); Conj = true reads and writes conjugated
template <typename T, bool Conj>
struct StridedAcc {
    cplx<T>* p;
    int stride;
    __device__ __forceinline__ cplx<T> load(int i) const {
        cplx<T> v = p[i * stride];
        if (Conj) v.im = -v.im;
        return v;
    }
    __device__ __forceinline__ void store(int i, cplx<T> v) const {
        if (Conj) v.im = -v.im;
        p[i * stride] = v;
    }
};

}  // namespace enufft
