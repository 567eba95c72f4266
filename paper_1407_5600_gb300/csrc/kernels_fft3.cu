// Fluid update in three passes over HBM (Eq. vf with the viscous stress, Crank-Nicolson in
// time, exact discrete projection), each component transformed on its own index grid:
//
//   pass A  per (box, component, z) plane: rhs = (rho/dt) v + (eta/2) L v + f + f_body, then
//           the 2-D real-to-complex FFT of the plane in shared memory     -> spec [z][kx][ky]
//   pass B  per (box, kx, block of ky): FFT along z of all three components, divide by
//           rho/dt + (eta/2) lambda(k), project with the MAC divergence and gradient symbols,
//           set the k = 0 mode, inverse FFT along z                      (in place)
//   pass C  per (box, component, z) plane: 2-D complex-to-real inverse FFT, scale 1/N -> v
//
// Line FFTs: the register-resident line transforms of fft_lines.cuh (lines of up to 128
// points here; the planes of longer sides do not fit in shared memory).
// Real rows are packed two per complex row and separated after the row transform.
#include <cstdlib>
#include <string>

#include "mb_internal.cuh"
#include "fft_lines.cuh"

namespace mbk {

namespace {

template <typename T> __device__ __forceinline__ void load_table(T* dst, const T* src, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace

// Row stride (in complex) of the plane buffer: just room for the padded nx + 2 separated values
// (a 128 x 128 FP32 plane then takes 73 KiB, three blocks per SM).
__host__ __device__ inline int plane_ld(int nx)
{
    return nx + 2 + ((nx + 1) >> pad_shift(nx));
}

// Plane layouts.  Element (packed row p, slot j) of the plane buffer is P[L.at(p, j)]; rows()
// and cols() transform the ny/2 packed rows (slot j = x) and the nx/2 columns (element y of
// column k is slot 2k + (y & 1) of packed row y >> 1).
//
// PadPlane: any power-of-two plane; one pad slot every 2^pad_shift(nx) slots.
struct PadPlane {
    int nx, ny, S, sx;
    __device__ PadPlane(int nx_, int ny_) : nx(nx_), ny(ny_), S(plane_ld(nx_)), sx(pad_shift(nx_)) {}
    __device__ __forceinline__ int row(int p) const { return p * S; }
    __device__ __forceinline__ int off(int j) const { return j + (j >> sx); }
    __device__ __forceinline__ int at(int p, int j) const { return p * S + j + (j >> sx); }
    template <bool INV, typename T> __device__ __forceinline__ void rows(T* P, const T* tw) const
    {
        const int S_ = S, sx_ = sx;
        lines_fft_n<INV>(nx, P, ny / 2, [S_, sx_](int l, int j) { return l * S_ + j + (j >> sx_); }, tw);
    }
    template <bool INV, typename T> __device__ __forceinline__ void cols(T* P, const T* tw) const
    {
        const int S_ = S, sx_ = sx;
        lines_fft_n<INV>(ny, P, nx / 2, [S_, sx_](int k, int y) {
            const int j = 2 * k + (y & 1);
            return (y >> 1) * S_ + j + (j >> sx_);
        }, tw);
    }
};

// Skew128: 128 x 128 planes of float2.  Rows of 148 slots, one pad slot every 16 and a skew of
// SK[(p >> 2) & 7] slots per group of four packed rows, SK = {0, 6, 3, 9, 7, 5, 4, 0}; the row
// lines take lane = 4 t + (line - l0), the column lines lane = 8 (line - l0) + t.  A model of the
// shared-memory banks (8-byte accesses served per half-warp) over every access of the two plane
// passes (loads, both stages of the row and column line FFTs, the separation, the spectrum
// copies) gives this layout 0.63x the wavefronts of the padded one (1.2x the fewest possible);
// 64 rows x 148 slots x 8 B = 74 KiB keeps three planes per SM.  With 128-point lines split
// 16 x 8 (thread t of a line holds elements 8 n1 + t, then 8 (t + 8 m) + n2) every address is
// a per-thread base plus a compile-time offset, so the line FFTs spend no instructions on
// indexing.
struct Skew128 {
    static constexpr int S = 148;
    static constexpr unsigned SKW = 0x04579360u;              // SK[i] = (SKW >> 4 i) & 15
    __host__ __device__ static constexpr int sk(int i) { return (int)((SKW >> (4 * (i & 7))) & 15u); }
    __device__ Skew128(int, int) {}
    __device__ __forceinline__ int row(int p) const { return p * S + sk(p >> 2); }
    __device__ __forceinline__ int off(int j) const { return j + (j >> 4); }
    __device__ __forceinline__ int at(int p, int j) const { return p * S + sk(p >> 2) + j + (j >> 4); }
    // One round: 8 warps x 4 lines; lane = 4 t + (line - l0).  b1 addresses element 8 n1 + t
    // at offset c1(n1); b2 element 8 (t + 8 m) + n2 at c2(m, n2); b1 element (t + 8 m) + 16 k2
    // at c3(m, k2).
    template <bool INV, bool COL>
    __device__ __forceinline__ static void line_round(float2* P, int l, int t, const float2* tw)
    {
        int b1, b2;
        if (COL) {
            b1 = 148 * (t >> 1) + 2 * l + (t & 1) + (l >> 3);
            b2 = 592 * t + 2 * l + (l >> 3) + sk(t);
        } else {
            const int base = l * S + sk(l >> 2);
            b1 = base + t;
            b2 = base + 8 * t + (t >> 1);
        }
        auto c1 = [](int n1) { return COL ? 592 * n1 + sk(n1) : 8 * n1 + (n1 >> 1); };
        auto c2 = [](int m, int n2) { return COL ? 4736 * m + 148 * (n2 >> 1) + (n2 & 1) : 68 * m + n2; };
        auto c3 = [](int m, int k2) { return COL ? 1184 * k2 + 592 * m + sk(2 * k2 + m) : 8 * m + 17 * k2; };
        float2 a[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) a[n1] = P[b1 + c1(n1)];
        reg_dft<16, INV>(a);
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) {
            float2 w = tw[(t * k1) & 127];
            if (INV) w.y = -w.y;
            a[k1] = cm(a[k1], w);
        }
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) P[b1 + c1(k1)] = a[k1];
        __syncwarp();
        float2 b[2][8];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n2 = 0; n2 < 8; ++n2) b[m][n2] = P[b2 + c2(m, n2)];
#pragma unroll
        for (int m = 0; m < 2; ++m) reg_dft<8, INV>(b[m]);
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) P[b1 + c3(m, k2)] = b[m][k2];
        __syncwarp();
    }
    template <bool INV, bool COL> __device__ __forceinline__ static void lines(float2* P, const float2* tw)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int sub = COL ? lane >> 3 : lane & 3, t = COL ? lane & 7 : lane >> 2;
        for (int l0 = warp * 4; l0 < 64; l0 += nw * 4) line_round<INV, COL>(P, l0 + sub, t, tw);
    }
    template <bool INV, typename T> __device__ __forceinline__ void rows(T* P, const T* tw) const
    {
        lines<INV, false>(P, tw);
    }
    template <bool INV, typename T> __device__ __forceinline__ void cols(T* P, const T* tw) const
    {
        lines<INV, true>(P, tw);
    }
};

template <typename L> struct PlaneSlots;
template <> struct PlaneSlots<PadPlane> { static size_t count(int nx, int ny) { return (size_t)(ny / 2) * plane_ld(nx); } };
template <> struct PlaneSlots<Skew128> { static size_t count(int, int) { return 64 * (size_t)Skew128::S; } };

// ------------------------------------------------------------------------------------------
// Pass A.  Plane buffer P[p][pad(j)], p < ny/2: first rows 2p, 2p+1 packed as re + i im; after
// the row FFT and the in-place separation, logical slot 2k + e of row p holds X_{2p+e}[k],
// k <= nx/2.  pad(j) = j + (j >> pad_shift(nx)).
template <typename R, typename K, typename L>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 256 : 512, sizeof(R) == 4 ? 3 : 1)
k_plane_fwd(FluidArgs<R> a, GridGeo g)
{
    dep_wait();
    dep_release();
    using T = typename C2<K>::T;     // K: arithmetic type (FP32, or double-float for FP64)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const L lay(nx, ny);
    T* P = reinterpret_cast<T*>(smem_raw);
    const T* twx = reinterpret_cast<const T*>(a.twk[0]);      // twiddles through L1
    const T* twy = reinterpret_cast<const T*>(a.twk[1]);
    const int z = blockIdx.x, bc = blockIdx.y, comp = bc % 3;
    const R* vc = a.v + (size_t)bc * g.N;
    const R* fc = a.f ? a.f + (size_t)bc * g.N : nullptr;
    const K ih2 = kparam<K>(a.inv_h2, a.inv_h2_32), rho_dt = kparam<K>(a.rho_dt, a.rho_dt32),
            half_eta = kparam<K>(a.half_eta, a.half_eta32);
    const bool body = a.body_prof && comp == a.body_axis;
    const R* pz = vc + (size_t)z * ny * nx;
    const R* pzp = vc + (size_t)((z + 1) & (nz - 1)) * ny * nx;
    const R* pzm = vc + (size_t)((z - 1) & (nz - 1)) * ny * nx;
    const R* pf = fc ? fc + (size_t)z * ny * nx : nullptr;
    R* pclr = a.f_clear && fc ? a.f_clear + (size_t)bc * g.N + (size_t)z * ny * nx : nullptr;
    // each work unit: 4 consecutive x of the two rows 2p, 2p+1
    const int qx = nx / 4, lq = 31 - __clz(qx);   // nx is a power of two
    for (int u = threadIdx.x; u < qx * (ny / 2) && a.no_v; u += blockDim.x) {
        // Stokes limit: the right-hand side is the force density (and body force) alone
        const int x0 = 4 * (u & (qx - 1)), p = u >> lq;
        const int y0 = 2 * p, y1 = y0 + 1;
        const K z0 = kconst<K>(0.0f);
        K r0[4] = {z0, z0, z0, z0}, r1[4] = {z0, z0, z0, z0};
        if (pf) {
            load4(pf + (size_t)y0 * nx + x0, r0);
            load4(pf + (size_t)y1 * nx + x0, r1);
            if (pclr) {
                const K zero[4] = {kconst<K>(0.0f), kconst<K>(0.0f), kconst<K>(0.0f),
                                   kconst<K>(0.0f)};
                store4(pclr + (size_t)y0 * nx + x0, zero);
                store4(pclr + (size_t)y1 * nx + x0, zero);
            }
        }
        if (body) {
            for (int i = 0; i < 4; ++i) {
                const int x = x0 + i;
                r0[i] += K(a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y0 : z)]);
                r1[i] += K(a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y1 : z)]);
            }
        }
        T* rowp = P + lay.row(p);
        for (int i = 0; i < 4; ++i) rowp[lay.off(x0 + i)] = T{r0[i], r1[i]};
    }
    for (int u = threadIdx.x; u < qx * (ny / 2) && !a.no_v; u += blockDim.x) {
        const int x0 = 4 * (u & (qx - 1)), p = u >> lq;
        const int y0 = 2 * p, y1 = y0 + 1;
        const int ym = (y0 - 1) & (ny - 1), yp = (y1 + 1) & (ny - 1);
        K c0[4], c1[4], am[4], ap[4], t[4];
        load4(pz + (size_t)y0 * nx + x0, c0);
        load4(pz + (size_t)y1 * nx + x0, c1);
        load4(pz + (size_t)ym * nx + x0, am);
        load4(pz + (size_t)yp * nx + x0, ap);
        K l0[4], l1[4];
        for (int i = 0; i < 4; ++i) {
            l0[i] = am[i] + c1[i] - kconst<K>(6.0f) * c0[i];
            l1[i] = c0[i] + ap[i] - kconst<K>(6.0f) * c1[i];
        }
        load4(pzp + (size_t)y0 * nx + x0, t);
        for (int i = 0; i < 4; ++i) l0[i] += t[i];
        load4(pzm + (size_t)y0 * nx + x0, t);
        for (int i = 0; i < 4; ++i) l0[i] += t[i];
        load4(pzp + (size_t)y1 * nx + x0, t);
        for (int i = 0; i < 4; ++i) l1[i] += t[i];
        load4(pzm + (size_t)y1 * nx + x0, t);
        for (int i = 0; i < 4; ++i) l1[i] += t[i];
        const int xm = (x0 - 1) & (nx - 1), xp = (x0 + 4) & (nx - 1);
        const K e0m = K(pz[(size_t)y0 * nx + xm]), e0p = K(pz[(size_t)y0 * nx + xp]);
        const K e1m = K(pz[(size_t)y1 * nx + xm]), e1p = K(pz[(size_t)y1 * nx + xp]);
        for (int i = 0; i < 4; ++i) {
            l0[i] += (i == 0 ? e0m : c0[i - 1]) + (i == 3 ? e0p : c0[i + 1]);
            l1[i] += (i == 0 ? e1m : c1[i - 1]) + (i == 3 ? e1p : c1[i + 1]);
        }
        K r0[4], r1[4];
        for (int i = 0; i < 4; ++i) {
            r0[i] = rho_dt * c0[i] + half_eta * (l0[i] * ih2);
            r1[i] = rho_dt * c1[i] + half_eta * (l1[i] * ih2);
        }
        if (pf) {
            load4(pf + (size_t)y0 * nx + x0, t);
            for (int i = 0; i < 4; ++i) r0[i] += t[i];
            load4(pf + (size_t)y1 * nx + x0, t);
            for (int i = 0; i < 4; ++i) r1[i] += t[i];
            if (pclr) {                  // leave f zeroed for the next accumulation
                const K zero[4] = {kconst<K>(0.0f), kconst<K>(0.0f), kconst<K>(0.0f),
                                   kconst<K>(0.0f)};
                store4(pclr + (size_t)y0 * nx + x0, zero);
                store4(pclr + (size_t)y1 * nx + x0, zero);
            }
        }
        if (body) {
            for (int i = 0; i < 4; ++i) {
                const int x = x0 + i;
                r0[i] += K(a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y0 : z)]);
                r1[i] += K(a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y1 : z)]);
            }
        }
        T* rowp = P + lay.row(p);
        for (int i = 0; i < 4; ++i) rowp[lay.off(x0 + i)] = T{r0[i], r1[i]};
    }
    __syncthreads();
    lay.template rows<false>(P, twx);
    __syncthreads();
    // separate the two real rows of each packed row (one warp per packed row, in place)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int p = warp; p < ny / 2; p += nw) {
            T* rowp = P + lay.row(p);
            T ev[3], od[3];        // nx/2 + 1 <= 65 values: at most 3 per lane
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int k = lane + 32 * r;
                if (k < nxh) {
                    const int kr = (nx - k) & (nx - 1);
                    const T Z = rowp[lay.off(k)], Zr = rowp[lay.off(kr)];
                    ev[r] = T{(Z.x + Zr.x) * kconst<K>(0.5f), (Z.y - Zr.y) * kconst<K>(0.5f)};
                    od[r] = T{(Z.y + Zr.y) * kconst<K>(0.5f), (Zr.x - Z.x) * kconst<K>(0.5f)};
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int k = lane + 32 * r;
                if (k < nxh) {
                    rowp[lay.off(2 * k)] = ev[r];
                    rowp[lay.off(2 * k + 1)] = od[r];
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    auto col = [lay](int k, int y) { return lay.at(y >> 1, 2 * k + (y & 1)); };
    // columns k = 0 and k = nx/2 are real: transform them as one complex column
    // Z_y = X_y[0] + i X_y[nx/2], so that nx/2 column lines remain
    for (int y = threadIdx.x; y < ny; y += blockDim.x)
        P[col(0, y)] = T{P[col(0, y)].x, P[col(nx / 2, y)].x};
    __syncthreads();
    lay.template cols<false>(P, twy);
    __syncthreads();
    // A = FFT X[0] = (Z_k + conj Z_-k) / 2,  B = FFT X[nx/2] = (Z_k - conj Z_-k) / (2i)
    if (threadIdx.x < 32) {
        T av[4], bv[4];            // ny <= 128: at most 4 per lane
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = threadIdx.x + 32 * r;
            if (k < ny) {
                const T Zk = P[col(0, k)], Zr = P[col(0, (ny - k) & (ny - 1))];
                av[r] = T{(Zk.x + Zr.x) * kconst<K>(0.5f), (Zk.y - Zr.y) * kconst<K>(0.5f)};
                bv[r] = T{(Zk.y + Zr.y) * kconst<K>(0.5f), (Zr.x - Zk.x) * kconst<K>(0.5f)};
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = threadIdx.x + 32 * r;
            if (k < ny) {
                P[col(0, k)] = av[r];
                P[col(nx / 2, k)] = bv[r];
            }
        }
    }
    __syncthreads();
    T* out = reinterpret_cast<T*>(a.spec) + ((size_t)bc * nz + z) * (size_t)nxh * ny;
    const int ly = 31 - __clz(ny);
    if (blockDim.x % ny == 0) {
        // a thread keeps its y (so its packed row and parity) and steps through k
        const int y = threadIdx.x & (ny - 1), e = y & 1, dk = blockDim.x >> ly;
        const T* rowp = P + lay.row(y >> 1);
        for (int k = threadIdx.x >> ly; k < nxh; k += dk) out[k * ny + y] = rowp[lay.off(2 * k + e)];
    } else {
        for (int i = threadIdx.x; i < nxh * ny; i += blockDim.x) out[i] = P[col(i >> ly, i & (ny - 1))];
    }
}

// 128-point z-lines of the pass-B buffer (FP32, C = 8 columns): element z of line l (component
// l / 8, column l % 8) is at ((l / 8) 144 + z + (z >> 3)) 12 + l % 8.  Same 16 x 8 split as
// lines_fft; thread t of a line addresses a per-thread base plus compile-time offsets (z =
// 8 n1 + t pads to 9 n1 + t, 8 (t + 8 m) + n2 to 9 t + 72 m + n2, t + 8 m + 16 k2 to
// t + 9 m + 18 k2), so the transforms spend no instructions on indexing.
template <bool INV>
__device__ __forceinline__ void zlines128(float2* Bf, const float2* tw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sub = lane & 3, t = lane >> 2;
    for (int l0 = warp * 4; l0 < 24; l0 += nw * 4) {
        const int l = l0 + sub, c = l >> 3, k = l & 7;
        float2* b1 = Bf + (c * 144 + t) * 12 + k;
        float2* b2 = Bf + (c * 144 + 9 * t) * 12 + k;
        float2 a[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) a[n1] = b1[108 * n1];
        reg_dft<16, INV>(a);
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) {
            float2 w = tw[(t * k1) & 127];
            if (INV) w.y = -w.y;
            a[k1] = cm(a[k1], w);
        }
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) b1[108 * k1] = a[k1];
        __syncwarp();
        float2 b[2][8];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n2 = 0; n2 < 8; ++n2) b[m][n2] = b2[(72 * m + n2) * 12];
#pragma unroll
        for (int m = 0; m < 2; ++m) reg_dft<8, INV>(b[m]);
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) b1[(9 * m + 18 * k2) * 12] = b[m][k2];
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Pass B.  CTA = (ky block of width C, kx, box); shared buffer [3][pad(nz)][C + 4].  C is a
// compile-time width (16 FP32, 8 FP64) and the block has 3 C N2 threads, one round of lines.
template <typename R, typename K, int C>
__global__ void __launch_bounds__(3 * C * 8, sizeof(R) == 4 ? 768 / (3 * C * 8) : 1)
k_zsolve(FluidArgs<R> a, GridGeo g)
{
    using T = typename C2<K>::T;
    constexpr int Cp = C + 4;                    // 4 z-rows x 4 lines per half-warp: distinct banks
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int lz = 31 - __clz(nz);
    const int sz = pad_shift(nz), nzp = padded_len(nz);
    T* Bf = reinterpret_cast<T*>(smem_raw);
    T* twz = Bf + 3 * nzp * Cp;
    load_table(twz, reinterpret_cast<const T*>(a.twk[2]), nz);   // set up once: no wait
    dep_wait();
    dep_release();
    const int ky0 = blockIdx.x * C, kx = blockIdx.y, box = blockIdx.z;
    const size_t zstride = (size_t)nxh * ny;
    const size_t cstride = (size_t)nz * zstride;
    T* base = reinterpret_cast<T*>(a.spec) + (size_t)(box * 3) * cstride + (size_t)kx * ny + ky0;
    auto at = [=](int c, int z, int k) { return (c * nzp + z + (z >> sz)) * Cp + k; };
    const int total = 3 * nz * C;
    constexpr bool z128 = sizeof(T) == 8 && C == 8;     // FP32 complex, eight columns
    // 128-point z-lines with 192 threads: thread (zr = tid / 8, k = tid % 8) moves the elements
    // (c = zr / 8, z = zr % 8 + 8 j, k), j < 16, at a fixed stride on both sides
    const bool fast = z128 && nz == 128 && blockDim.x == 3 * 8 * C;
    if (fast) {
        const int k = threadIdx.x & 7, zr = threadIdx.x >> 3, c = zr >> 3, z0 = zr & 7;
        T* sb = Bf + (c * 144 + z0) * 12 + k;
        const T* gb = base + c * cstride + (size_t)z0 * zstride + k;
#pragma unroll
        for (int j = 0; j < 16; ++j) async_copy(sb + 108 * j, gb + (size_t)(8 * j) * zstride);
    } else {
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int k = i % C, zc = i / C, z = zc & (nz - 1), c = zc >> lz;
            async_copy(&Bf[at(c, z, k)], &base[c * cstride + (size_t)z * zstride + k]);
        }
    }
    async_wait_all();
    __syncthreads();
    auto idx = [=](int l, int z) { return at(l / C, z, l % C); };
    if constexpr (z128) {
        if (nz == 128) zlines128<false>(reinterpret_cast<float2*>(Bf), reinterpret_cast<const float2*>(twz));
        else lines_fft_n<false>(nz, Bf, 3 * C, idx, twz);
    } else {
        lines_fft_n<false>(nz, Bf, 3 * C, idx, twz);
    }
    __syncthreads();
    const K* sym = reinterpret_cast<const K*>(a.symk);     // [9][256] cos, sin, lambda
    const K ih = kparam<K>(a.inv_h, a.inv_h32);
    const K csx = sym[0 * 256 + kx], snx = sym[1 * 256 + kx], lx = sym[2 * 256 + kx];
    const K rho_dt = kparam<K>(a.rho_dt, a.rho_dt32);
    const K half_eta = kparam<K>(a.half_eta, a.half_eta32);
    // with blockDim a multiple of C a thread keeps its column k (and ky's symbols) throughout
    const int kfix = threadIdx.x % C;
    const K csy = sym[3 * 256 + ky0 + kfix], sny = sym[4 * 256 + ky0 + kfix];
    const K lxy = lx + sym[5 * 256 + ky0 + kfix];
    const bool colfix = blockDim.x % C == 0;
    for (int i = threadIdx.x; i < nz * C; i += blockDim.x) {
        const int k = colfix ? kfix : i % C, kz = i / C, ky = ky0 + k;
        const K cs[3] = {csx, colfix ? csy : sym[3 * 256 + ky], sym[6 * 256 + kz]};
        const K sn[3] = {snx, colfix ? sny : sym[4 * 256 + ky], sym[7 * 256 + kz]};
        const K lam = (colfix ? lxy : lx + sym[5 * 256 + ky]) + sym[8 * 256 + kz];
        const K cinv = recip(rho_dt + half_eta * lam);
        T W[3];
        for (int c = 0; c < 3; ++c) {
            const T v = Bf[at(c, kz, k)];
            W[c] = T{v.x * cinv, v.y * cinv};
        }
        if (kx == 0 && ky == 0 && kz == 0) {
            for (int c = 0; c < 3; ++c) {
                if (a.mean_state) {              // the only thread of this box at k = 0
                    double m = a.mean_state[3 * box + c];
                    if (a.mean_force) m += a.mean_scale * a.mean_force[3 * box + c];
                    a.mean_state[3 * box + c] = m;
                    W[c] = T{K((double)g.N * m), kconst<K>(0.0f)};
                } else if (a.mean_override) {
                    W[c] = T{K((double)g.N * a.mean_override[3 * box + c]), kconst<K>(0.0f)};
                } else if (a.mean_mode == 1) {
                    W[c] = T{kconst<K>(0.0f), kconst<K>(0.0f)};
                }
            }
        } else {
            // D_a = (e^{i th} - 1)/h, G_a = (1 - e^{-i th})/h, D.G = -lambda:
            // P W = W + G (D.W) / lambda
            K dr = kconst<K>(0.0f), di = kconst<K>(0.0f);
            for (int c = 0; c < 3; ++c) {
                const K Dr = (cs[c] - kconst<K>(1.0f)) * ih, Di = sn[c] * ih;
                dr += Dr * W[c].x - Di * W[c].y;
                di += Dr * W[c].y + Di * W[c].x;
            }
            const K il = recip(lam);
            dr *= il;
            di *= il;
            for (int c = 0; c < 3; ++c) {
                const K Gr = (kconst<K>(1.0f) - cs[c]) * ih, Gi = sn[c] * ih;
                W[c].x += Gr * dr - Gi * di;
                W[c].y += Gr * di + Gi * dr;
            }
        }
        for (int c = 0; c < 3; ++c) Bf[at(c, kz, k)] = W[c];
    }
    __syncthreads();
    if constexpr (z128) {
        if (nz == 128) zlines128<true>(reinterpret_cast<float2*>(Bf), reinterpret_cast<const float2*>(twz));
        else lines_fft_n<true>(nz, Bf, 3 * C, idx, twz);
    } else {
        lines_fft_n<true>(nz, Bf, 3 * C, idx, twz);
    }
    __syncthreads();
    if (fast) {
        const int k = threadIdx.x & 7, zr = threadIdx.x >> 3, c = zr >> 3, z0 = zr & 7;
        const T* sb = Bf + (c * 144 + z0) * 12 + k;
        T* gb = base + c * cstride + (size_t)z0 * zstride + k;
#pragma unroll
        for (int j = 0; j < 16; ++j) gb[(size_t)(8 * j) * zstride] = sb[108 * j];
    } else {
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int k = i % C, zc = i / C, z = zc & (nz - 1), c = zc >> lz;
            base[c * cstride + (size_t)z * zstride + k] = Bf[at(c, z, k)];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Pass C.  Inverse of pass A: columns, then the packed rows Z = X_{2p} + i X_{2p+1} (with the
// Hermitian extension X[nx - k] = conj X[k]), then the real rows, scaled by 1/N.
template <typename R, typename K, typename L>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 256 : 512, sizeof(R) == 4 ? 3 : 1)
k_plane_inv(FluidArgs<R> a, GridGeo g)
{
    // no early release: the next kernel (the interpolation's persistent grid, which splits the
    // blobs evenly over its warps) then starts all its blocks together, not first on the SMs
    // this pass leaves early
    dep_wait();
    using T = typename C2<K>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const L lay(nx, ny);
    T* P = reinterpret_cast<T*>(smem_raw);
    const T* twx = reinterpret_cast<const T*>(a.twk[0]);      // twiddles through L1
    const T* twy = reinterpret_cast<const T*>(a.twk[1]);
    const int z = blockIdx.x, bc = blockIdx.y;
    const T* in = reinterpret_cast<const T*>(a.spec) + ((size_t)bc * nz + z) * (size_t)nxh * ny;
    auto col = [lay](int k, int y) { return lay.at(y >> 1, 2 * k + (y & 1)); };
    const int ly = 31 - __clz(ny);
    if (blockDim.x % ny == 0) {
        const int y = threadIdx.x & (ny - 1), e = y & 1, dk = blockDim.x >> ly;
        T* rowp = P + lay.row(y >> 1);
        for (int k = threadIdx.x >> ly; k < nxh; k += dk) async_copy(&rowp[lay.off(2 * k + e)], &in[k * ny + y]);
    } else {
        for (int i = threadIdx.x; i < nxh * ny; i += blockDim.x) async_copy(&P[col(i >> ly, i & (ny - 1))], &in[i]);
    }
    async_wait_all();
    __syncthreads();
    // columns k = 0 and k = nx/2 invert to real sequences: transform their Hermitian parts as
    // one complex column Z = herm(A) + i herm(B), whose inverse is Re(IFFT A) + i Re(IFFT B)
    if (threadIdx.x < 32) {
        T zv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = threadIdx.x + 32 * r;
            if (k < ny) {
                const int kr = (ny - k) & (ny - 1);
                const T A = P[col(0, k)], Ar = P[col(0, kr)];
                const T Bv = P[col(nx / 2, k)], Br = P[col(nx / 2, kr)];
                // herm(A) = (A_k + conj A_-k) / 2, herm(B) likewise; Z = herm(A) + i herm(B)
                const T ha = T{(A.x + Ar.x) * kconst<K>(0.5f), (A.y - Ar.y) * kconst<K>(0.5f)};
                const T hb = T{(Bv.x + Br.x) * kconst<K>(0.5f), (Bv.y - Br.y) * kconst<K>(0.5f)};
                zv[r] = T{ha.x - hb.y, ha.y + hb.x};
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = threadIdx.x + 32 * r;
            if (k < ny) P[col(0, k)] = zv[r];
        }
    }
    __syncthreads();
    lay.template cols<true>(P, twy);
    __syncthreads();
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        const T zc = P[col(0, y)];
        P[col(0, y)] = T{zc.x, kconst<K>(0.0f)};
        P[col(nx / 2, y)] = T{zc.y, kconst<K>(0.0f)};
    }
    __syncthreads();
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int p = warp; p < ny / 2; p += nw) {
            T* rowp = P + lay.row(p);
            T zv[4];              // nx <= 128 values: at most 4 per lane
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = lane + 32 * r;
                if (k < nx) {
                    const int kk = k <= nx / 2 ? k : nx - k;
                    T e = rowp[lay.off(2 * kk)], o = rowp[lay.off(2 * kk + 1)];
                    if (k == 0 || k == nx / 2) { e.y = kconst<K>(0.0f); o.y = kconst<K>(0.0f); }
                    if (k > nx / 2) { e.y = -e.y; o.y = -o.y; }
                    zv[r] = T{e.x - o.y, e.y + o.x};
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = lane + 32 * r;
                if (k < nx) rowp[lay.off(k)] = zv[r];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    lay.template rows<true>(P, twx);
    __syncthreads();
    const K scale = kparam<K>(a.inv_n, a.inv_n32);
    R* out = a.v_out + (size_t)bc * g.N + (size_t)z * ny * nx;
    const int qx = nx / 4, lq = 31 - __clz(qx);   // nx is a power of two
    for (int u = threadIdx.x; u < qx * (ny / 2); u += blockDim.x) {
        const int x0 = 4 * (u & (qx - 1)), p = u >> lq;
        K r0[4], r1[4];
        const T* rowp = P + lay.row(p);
        for (int i = 0; i < 4; ++i) {
            const T zv = rowp[lay.off(x0 + i)];
            r0[i] = zv.x * scale;
            r1[i] = zv.y * scale;
        }
        store4(out + (size_t)(2 * p) * nx + x0, r0);
        store4(out + (size_t)(2 * p + 1) * nx + x0, r1);
        if (a.v_sum_out) {               // v^n + v^{n+1} for the corrector's single gather
            const size_t o0 = (size_t)bc * g.N + (size_t)z * ny * nx + (size_t)(2 * p) * nx + x0;
            K b0[4], b1[4];
            load4(a.v_sum_base + o0, b0);
            load4(a.v_sum_base + o0 + nx, b1);
            for (int i = 0; i < 4; ++i) {
                b0[i] += r0[i];
                b1[i] += r1[i];
            }
            store4(a.v_sum_out + o0, b0);
            store4(a.v_sum_out + o0 + nx, b1);
        }
    }
}

template <typename R>
cudaError_t launch_fluid3(cudaStream_t st, int B, const GridGeo& g, const FluidArgs<R>& a_in,
                          cudaEvent_t* marks)
{
    const FluidArgs<R> a = with_derived(a_in, g);
    using K = typename FftCompute<R>::type;
    using T = typename C2<K>::T;
    // plane blocks: FP64 planes (one block per SM) take 512 threads to hide latency
    constexpr int PT = sizeof(R) == 4 ? 256 : 512;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    constexpr int CZ = 8;                             // ky columns per z-pass block
    static std::atomic<unsigned> attr{0};     // per instantiation
    if (first_on_device(attr)) {
        const int lim = 200 * 1024;
        cudaFuncSetAttribute(k_plane_fwd<R, K, PadPlane>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_zsolve<R, K, CZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_zsolve<R, K, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_plane_inv<R, K, PadPlane>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if constexpr (sizeof(R) == 4) {
            cudaFuncSetAttribute(k_plane_fwd<R, K, Skew128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            cudaFuncSetAttribute(k_plane_inv<R, K, Skew128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        }
    }
    // FP32 planes of 128 x 128 take the conflict-free layout (MB_PLANE_LAYOUT=pad keeps the
    // padded one, for comparison)
    static const bool skew_off = [] {
        const char* e = std::getenv("MB_PLANE_LAYOUT");
        return e && std::string(e) == "pad";
    }();
    const bool skew = sizeof(R) == 4 && nx == 128 && ny == 128 && !skew_off;
    const size_t smem_plane = (skew ? PlaneSlots<Skew128>::count(nx, ny)
                                    : PlaneSlots<PadPlane>::count(nx, ny)) * sizeof(T);
    const int C = ny >= CZ ? CZ : 4;
    const size_t smem_z = ((size_t)3 * padded_len(nz) * (C + 4) + nz) * sizeof(T);
    auto mark = [&](int i) { if (marks) cudaEventRecord(marks[i], st); };
    mark(0);
    cudaError_t e;
    const dim3 gp(nz, 3 * B), gz(ny / C, nxh, B);
    if constexpr (sizeof(R) == 4) {
        if (skew) e = launch_dep(k_plane_fwd<R, K, Skew128>, gp, dim3(PT), smem_plane, st, a, g);
        else e = launch_dep(k_plane_fwd<R, K, PadPlane>, gp, dim3(PT), smem_plane, st, a, g);
    } else {
        e = launch_dep(k_plane_fwd<R, K, PadPlane>, gp, dim3(PT), smem_plane, st, a, g);
    }
    if (e != cudaSuccess) return e;
    mark(1);
    mark(2);
    if (C == CZ) e = launch_dep(k_zsolve<R, K, CZ>, gz, dim3(3 * CZ * 8), smem_z, st, a, g);
    else e = launch_dep(k_zsolve<R, K, 4>, gz, dim3(3 * 4 * 8), smem_z, st, a, g);
    if (e != cudaSuccess) return e;
    mark(3);
    mark(4);
    if constexpr (sizeof(R) == 4) {
        if (skew) e = launch_dep(k_plane_inv<R, K, Skew128>, gp, dim3(PT), smem_plane, st, a, g);
        else e = launch_dep(k_plane_inv<R, K, PadPlane>, gp, dim3(PT), smem_plane, st, a, g);
    } else {
        e = launch_dep(k_plane_inv<R, K, PadPlane>, gp, dim3(PT), smem_plane, st, a, g);
    }
    if (e != cudaSuccess) return e;
    mark(5);
    return cudaGetLastError();
}
template cudaError_t launch_fluid3<float>(cudaStream_t, int, const GridGeo&,
                                          const FluidArgs<float>&, cudaEvent_t*);
template cudaError_t launch_fluid3<double>(cudaStream_t, int, const GridGeo&,
                                           const FluidArgs<double>&, cudaEvent_t*);

}  // namespace mbk
