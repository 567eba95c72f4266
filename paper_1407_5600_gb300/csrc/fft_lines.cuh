// Line FFTs held in registers, shared by the three-pass and five-pass fluid solvers.
//
// A line of N = N1 N2 points is done by N2 threads of one warp.  Thread t holds the N1 points
// x[N2 n1 + t] in registers, does an N1-point DFT, multiplies by W_N^{t k1}, and the line is
// exchanged once through shared memory; then each thread does N1/N2 DFTs of N2 points
// (X[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} W_N^{n2 k1} sum_n1 x[N2 n1 + n2] W_N1^{n1 k1}).
#pragma once
#include "mb_internal.cuh"
#include "dfloat.cuh"

namespace mbk {
namespace {

template <typename T> __device__ __forceinline__ T cm(T a, T b)
{
    return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return T{a.x + b.x, a.y + b.y}; }
// Correctly rounded reciprocals (the float one is a single intrinsic instead of a division).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return T{a.x - b.x, a.y - b.y}; }

__host__ __device__ constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// cos and sin of 2 pi j / 16, j < 8 (the twiddles of the in-register DFTs of up to 16 points;
// after unrolling every index is a constant and the values fold into the arithmetic).
template <typename R> __device__ __forceinline__ R cos16(int j)
{
    switch (j) {
    case 0: return R(1.0);
    case 1: return R(0.92387953251128675613);
    case 2: return R(0.70710678118654752440);
    case 3: return R(0.38268343236508977173);
    case 4: return R(0.0);
    case 5: return R(-0.38268343236508977173);
    case 6: return R(-0.70710678118654752440);
    default: return R(-0.92387953251128675613);
    }
}
// sin(2 pi j / 16) = cos(2 pi (j - 4) / 16), j < 8
template <typename R> __device__ __forceinline__ R sin16(int j) { return cos16<R>(j < 4 ? 4 - j : j - 4); }

// b W_16^j (forward) or b W_16^-j (inverse), with W_16 = exp(-2 pi i / 16); j < 8.
template <bool INV, typename T> __device__ __forceinline__ T twiddle16(T b, int j)
{
    using R = decltype(b.x);
    if (j == 0) return b;
    if (j == 4) return INV ? T{-b.y, b.x} : T{b.y, -b.x};
    const R c = cos16<R>(j), sn = INV ? sin16<R>(j) : -sin16<R>(j);
    return T{b.x * c - b.y * sn, b.x * sn + b.y * c};
}

// One radix-2 stage (butterfly span LEN) of an in-register DIT DFT, then the next stage.  The
// span is a template argument so that every loop has a constant trip count and unrolls fully,
// which turns each twiddle index into a constant.
template <int P, int LEN, bool INV, typename T>
__device__ __forceinline__ void dft_stage(T (&x)[P])
{
    constexpr int HALF = LEN / 2;
#pragma unroll
    for (int s0 = 0; s0 < P; s0 += LEN) {
#pragma unroll
        for (int m = 0; m < HALF; ++m) {
            const T b = twiddle16<INV>(x[s0 + m + HALF], m * (16 / LEN));
            const T a = x[s0 + m];
            x[s0 + m] = cadd(a, b);
            x[s0 + m + HALF] = csub(a, b);
        }
    }
    if constexpr (LEN < P) dft_stage<P, 2 * LEN, INV>(x);
}

// In-register radix-2 DIT DFT of P <= 16 points with constant twiddles W_P^m = W_16^(16 m / P).
template <int P, bool INV, typename T>
__device__ __forceinline__ void reg_dft(T (&x)[P])
{
    static_assert(P <= 16, "in-register DFTs of at most 16 points");
    constexpr int bits = ilog2c(P);
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int r = bitrev(i, bits);
        if (r > i) {
            const T tmp = x[i];
            x[i] = x[r];
            x[r] = tmp;
        }
    }
    if constexpr (P > 1) dft_stage<P, 2, INV>(x);
}

template <int N> struct Split;                  // N = N1 * N2 with N1 >= N2, N1 % N2 == 0
template <> struct Split<4> { static constexpr int N1 = 2, N2 = 2; };
template <> struct Split<8> { static constexpr int N1 = 4, N2 = 2; };
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Split<256> { static constexpr int N1 = 16, N2 = 16; };

// FFTs of `lines` lines of N points held in shared memory; element j of line l is at
// buf[idx(l, j)].  All threads of the block call this; lines are spread over warps with the
// N2 threads of a line inside one warp, so only warp-level synchronisation is needed.
template <int N, bool INV, typename T, typename Idx>
__device__ __forceinline__ void lines_fft(T* buf, int lines, Idx idx, const T* __restrict__ tw)
{
    constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, M = N1 / N2;
    constexpr int LPW = 32 / N2;                 // lines per warp per round
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // consecutive lanes take consecutive lines: with the callers' padded layouts the lanes of
    // a half-warp then fall on distinct shared-memory banks
    const int sub = lane % LPW, t = lane / LPW;
    for (int l0 = warp * LPW; l0 < lines; l0 += nw * LPW) {
        const int l = l0 + sub;
        const bool on = l < lines;
        T a[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) a[n1] = on ? buf[idx(l, N2 * n1 + t)] : T{};
        reg_dft<N1, INV>(a);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            T w = tw[(t * k1) & (N - 1)];
            if (INV) w.y = -w.y;
            a[k1] = cm(a[k1], w);
        }
        __syncwarp();
        if (on) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) buf[idx(l, k1 * N2 + t)] = a[k1];
        }
        __syncwarp();
        T b[M][N2];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2)
                b[m][n2] = on ? buf[idx(l, (t + N2 * m) * N2 + n2)] : T{};
#pragma unroll
        for (int m = 0; m < M; ++m) reg_dft<N2, INV>(b[m]);
        __syncwarp();
        if (on) {
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) buf[idx(l, (t + N2 * m) + N1 * k2)] = b[m][k2];
        }
        __syncwarp();
    }
}

template <bool INV, typename T, typename Idx>
__device__ __forceinline__ void lines_fft_n(int n, T* buf, int lines, Idx idx, const T* tw)
{
    switch (n) {
    case 4: lines_fft<4, INV>(buf, lines, idx, tw); break;
    case 8: lines_fft<8, INV>(buf, lines, idx, tw); break;
    case 16: lines_fft<16, INV>(buf, lines, idx, tw); break;
    case 32: lines_fft<32, INV>(buf, lines, idx, tw); break;
    case 64: lines_fft<64, INV>(buf, lines, idx, tw); break;
    case 128: lines_fft<128, INV>(buf, lines, idx, tw); break;
    default: lines_fft<256, INV>(buf, lines, idx, tw); break;
    }
}

// Padded position of element j of a line of n points: one spare slot every N2 elements (N2 of
// the line FFT), which spreads the strided accesses of the second stage over the banks.
__host__ __device__ __forceinline__ int pad_shift(int n)
{
    return n >= 64 ? 3 : (n >= 16 ? 2 : 1);
}
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> pad_shift(n)); }

// Asynchronous global-to-shared copy of one complex value (no register staging, so every copy
// of a thread is in flight at once), and the wait for all of a thread's copies.
template <typename T> __device__ __forceinline__ void async_copy(T* dst, const T* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Four consecutive grid values (x0 .. x0+3, x0 a multiple of 4) as one vector load.
__device__ __forceinline__ void load4(const float* p, float v[4])
{
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4])
{
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void store4(float* p, const float v[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double v[4])
{
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
// FP64 grids read into, and written from, double-float values.
__device__ __forceinline__ void load4(const double* p, dfloat v[4])
{
    double d[4];
    load4(p, d);
    for (int i = 0; i < 4; ++i) v[i] = dfloat(d[i]);
}
__device__ __forceinline__ void store4(double* p, const dfloat v[4])
{
    const double d[4] = {(double)v[0], (double)v[1], (double)v[2], (double)v[3]};
    store4(p, d);
}

}  // namespace
}  // namespace mbk
