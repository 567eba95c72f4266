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
// Line FFTs: a line of N = N1 N2 points is done by N2 threads of one warp.  Thread t holds the
// N1 points x[N2 n1 + t] in registers, does an N1-point DFT, multiplies by W_N^{t k1}, and the
// line is exchanged once through shared memory; then each thread does N1/N2 DFTs of N2 points
// (X[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} W_N^{n2 k1} sum_n1 x[N2 n1 + n2] W_N1^{n1 k1}).
// Real rows are packed two per complex row and separated after the row transform.
#include "mb_internal.cuh"

namespace mbk {

namespace {

template <typename T> __device__ __forceinline__ T cm(T a, T b)
{
    return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return T{a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return T{a.x - b.x, a.y - b.y}; }

__host__ __device__ constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// In-register radix-2 DIT DFT of P points.  tw[j] = W_N^j, j < N; W_P^m = tw[m * stride].
template <int P, typename T>
__device__ __forceinline__ void reg_dft(T (&x)[P], const T* __restrict__ tw, int stride, bool inv)
{
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
#pragma unroll
    for (int len = 2; len <= P; len <<= 1) {
        const int half = len >> 1;
#pragma unroll
        for (int s0 = 0; s0 < P; s0 += len) {
#pragma unroll
            for (int m = 0; m < half; ++m) {
                T b = x[s0 + m + half];
                if (m != 0) {
                    T w = tw[m * (P / len) * stride];
                    if (inv) w.y = -w.y;
                    b = cm(b, w);
                }
                const T a = x[s0 + m];
                x[s0 + m] = cadd(a, b);
                x[s0 + m + half] = csub(a, b);
            }
        }
    }
}

template <int N> struct Split;                  // N = N1 * N2 with N1 >= N2, N1 % N2 == 0
template <> struct Split<4> { static constexpr int N1 = 2, N2 = 2; };
template <> struct Split<8> { static constexpr int N1 = 4, N2 = 2; };
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 16, N2 = 8; };

// FFTs of `lines` lines of N points held in shared memory; element j of line l is at
// buf[idx(l, j)].  All threads of the block call this; lines are spread over warps with the
// N2 threads of a line inside one warp, so only warp-level synchronisation is needed.
template <int N, typename T, typename Idx>
__device__ __forceinline__ void lines_fft(T* buf, int lines, Idx idx, const T* __restrict__ tw,
                                          bool inv)
{
    constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, M = N1 / N2;
    constexpr int LPW = 32 / N2;                 // lines per warp per round
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int t = lane % N2, sub = lane / N2;
    for (int l0 = warp * LPW; l0 < lines; l0 += nw * LPW) {
        const int l = l0 + sub;
        const bool on = l < lines;
        T a[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) a[n1] = on ? buf[idx(l, N2 * n1 + t)] : T{0, 0};
        reg_dft<N1>(a, tw, N2, inv);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            T w = tw[(t * k1) & (N - 1)];
            if (inv) w.y = -w.y;
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
                b[m][n2] = on ? buf[idx(l, (t + N2 * m) * N2 + n2)] : T{0, 0};
#pragma unroll
        for (int m = 0; m < M; ++m) reg_dft<N2>(b[m], tw, N1, inv);
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

template <typename T, typename Idx>
__device__ void lines_fft_n(int n, T* buf, int lines, Idx idx, const T* tw, bool inv)
{
    switch (n) {
    case 4: lines_fft<4>(buf, lines, idx, tw, inv); break;
    case 8: lines_fft<8>(buf, lines, idx, tw, inv); break;
    case 16: lines_fft<16>(buf, lines, idx, tw, inv); break;
    case 32: lines_fft<32>(buf, lines, idx, tw, inv); break;
    case 64: lines_fft<64>(buf, lines, idx, tw, inv); break;
    default: lines_fft<128>(buf, lines, idx, tw, inv); break;
    }
}

template <typename T> __device__ __forceinline__ void load_table(T* dst, const T* src, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace

// Row stride (in complex) of the plane buffer: room for the nx + 2 unpacked values.
__host__ __device__ inline int plane_ld(int nx) { return nx + 2; }

// ------------------------------------------------------------------------------------------
// Pass A.  Plane buffer P[p][j], p < ny/2: first rows 2p, 2p+1 packed as re + i im; after the
// row FFT and the in-place separation, P[p][2k + e] = X_{2p+e}[k] for k <= nx/2.
template <typename R>
__global__ void __launch_bounds__(256)
k_plane_fwd(FluidArgs<R> a, GridGeo g)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int S = plane_ld(nx);
    T* P = reinterpret_cast<T*>(smem_raw);
    T* twx = P + (ny / 2) * S;
    T* twy = twx + nx;
    load_table(twx, reinterpret_cast<const T*>(a.twf[0]), nx);
    load_table(twy, reinterpret_cast<const T*>(a.twf[1]), ny);
    const int z = blockIdx.x, bc = blockIdx.y, comp = bc % 3;
    const R* vc = a.v + (size_t)bc * g.N;
    const R* fc = a.f ? a.f + (size_t)bc * g.N : nullptr;
    const R ih2 = R(g.inv_h * g.inv_h), rho_dt = R(a.rho_dt), half_eta = R(a.half_eta);
    const bool body = a.body_prof && comp == a.body_axis;
    const size_t z0 = (size_t)z * ny, zp = (size_t)((z + 1) & (nz - 1)) * ny,
                 zm = (size_t)((z - 1) & (nz - 1)) * ny;
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int x = i & (nx - 1), y = i / nx;
        const int yp = (y + 1) & (ny - 1), ym = (y - 1) & (ny - 1);
        const size_t row = (z0 + y) * nx;
        const R c = vc[row + x];
        const R lap = ((vc[row + ((x + 1) & (nx - 1))] + vc[row + ((x - 1) & (nx - 1))]) +
                       (vc[(z0 + yp) * nx + x] + vc[(z0 + ym) * nx + x]) +
                       (vc[(zp + y) * nx + x] + vc[(zm + y) * nx + x]) - R(6) * c) * ih2;
        R val = rho_dt * c + half_eta * lap;
        if (fc) val += fc[row + x];
        if (body) val += a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y : z)];
        T* s = P + (y >> 1) * S + x;
        if (y & 1) s->y = val; else s->x = val;
    }
    __syncthreads();
    lines_fft_n(nx, P, ny / 2, [S](int l, int j) { return l * S + j; }, twx, false);
    __syncthreads();
    // separate the two real rows of each packed row (one warp per packed row, in place)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int p = warp; p < ny / 2; p += nw) {
            T* rowp = P + p * S;
            T ev[3], od[3];        // nx/2 + 1 <= 65 values: at most 3 per lane
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int k = lane + 32 * r;
                if (k < nxh) {
                    const T Z = rowp[k], Zr = rowp[(nx - k) & (nx - 1)];
                    ev[r] = T{(Z.x + Zr.x) * R(0.5), (Z.y - Zr.y) * R(0.5)};
                    od[r] = T{(Z.y + Zr.y) * R(0.5), (Zr.x - Z.x) * R(0.5)};
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int k = lane + 32 * r;
                if (k < nxh) {
                    rowp[2 * k] = ev[r];
                    rowp[2 * k + 1] = od[r];
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    lines_fft_n(ny, P, nxh, [S](int k, int y) { return (y >> 1) * S + 2 * k + (y & 1); }, twy,
                false);
    __syncthreads();
    T* out = a.spec + ((size_t)bc * nz + z) * (size_t)nxh * ny;
    for (int i = threadIdx.x; i < nxh * ny; i += blockDim.x) {
        const int y = i % ny, k = i / ny;
        out[i] = P[(y >> 1) * S + 2 * k + (y & 1)];
    }
}

// ------------------------------------------------------------------------------------------
// Pass B.  CTA = (ky block of width C, kx, box); shared buffer [3][nz][C].
template <typename R>
__global__ void __launch_bounds__(256)
k_zsolve(FluidArgs<R> a, GridGeo g, int C)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int Cp = C + 2;                        // padded row: 8 z-rows hit distinct banks
    T* Bf = reinterpret_cast<T*>(smem_raw);
    T* twz = Bf + 3 * nz * Cp;
    load_table(twz, reinterpret_cast<const T*>(a.twf[2]), nz);
    const int ky0 = blockIdx.x * C, kx = blockIdx.y, box = blockIdx.z;
    const size_t zstride = (size_t)nxh * ny;
    const T* base[3];
    for (int c = 0; c < 3; ++c)
        base[c] = a.spec + (size_t)(box * 3 + c) * nz * zstride + (size_t)kx * ny + ky0;
    for (int i = threadIdx.x; i < 3 * nz * C; i += blockDim.x) {
        const int k = i % C, z = (i / C) % nz, c = i / (C * nz);
        Bf[(c * nz + z) * Cp + k] = base[c][(size_t)z * zstride + k];
    }
    __syncthreads();
    auto idx = [C, Cp, nz](int l, int z) { return ((l / C) * nz + z) * Cp + (l % C); };
    lines_fft_n(nz, Bf, 3 * C, idx, twz, false);
    __syncthreads();
    const double* sym = a.sym;
    const R ih = R(g.inv_h);
    const R csx = R(sym[0 * 256 + kx]), snx = R(sym[1 * 256 + kx]), lx = R(sym[2 * 256 + kx]);
    for (int i = threadIdx.x; i < nz * C; i += blockDim.x) {
        const int k = i % C, kz = i / C, ky = ky0 + k;
        const R cs[3] = {csx, R(sym[3 * 256 + ky]), R(sym[6 * 256 + kz])};
        const R sn[3] = {snx, R(sym[4 * 256 + ky]), R(sym[7 * 256 + kz])};
        const R lam = lx + R(sym[5 * 256 + ky]) + R(sym[8 * 256 + kz]);
        const R cinv = R(1) / (R(a.rho_dt) + R(a.half_eta) * lam);
        T W[3];
        for (int c = 0; c < 3; ++c) {
            const T v = Bf[(c * nz + kz) * Cp + k];
            W[c] = T{v.x * cinv, v.y * cinv};
        }
        if (kx == 0 && ky == 0 && kz == 0) {
            for (int c = 0; c < 3; ++c) {
                if (a.mean_override) W[c] = T{R((double)g.N * a.mean_override[3 * box + c]), R(0)};
                else if (a.mean_mode == 1) W[c] = T{R(0), R(0)};
            }
        } else {
            // D_a = (e^{i th} - 1)/h, G_a = (1 - e^{-i th})/h, D.G = -lambda:
            // P W = W + G (D.W) / lambda
            R dr = R(0), di = R(0);
            for (int c = 0; c < 3; ++c) {
                const R Dr = (cs[c] - R(1)) * ih, Di = sn[c] * ih;
                dr += Dr * W[c].x - Di * W[c].y;
                di += Dr * W[c].y + Di * W[c].x;
            }
            const R il = R(1) / lam;
            dr *= il;
            di *= il;
            for (int c = 0; c < 3; ++c) {
                const R Gr = (R(1) - cs[c]) * ih, Gi = sn[c] * ih;
                W[c].x += Gr * dr - Gi * di;
                W[c].y += Gr * di + Gi * dr;
            }
        }
        for (int c = 0; c < 3; ++c) Bf[(c * nz + kz) * Cp + k] = W[c];
    }
    __syncthreads();
    lines_fft_n(nz, Bf, 3 * C, idx, twz, true);
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nz * C; i += blockDim.x) {
        const int k = i % C, z = (i / C) % nz, c = i / (C * nz);
        const_cast<T*>(base[c])[(size_t)z * zstride + k] = Bf[(c * nz + z) * Cp + k];
    }
}

// ------------------------------------------------------------------------------------------
// Pass C.  Inverse of pass A: columns, then the packed rows Z = X_{2p} + i X_{2p+1} (with the
// Hermitian extension X[nx - k] = conj X[k]), then the real rows, scaled by 1/N.
template <typename R>
__global__ void __launch_bounds__(256)
k_plane_inv(FluidArgs<R> a, GridGeo g)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int S = plane_ld(nx);
    T* P = reinterpret_cast<T*>(smem_raw);
    T* twx = P + (ny / 2) * S;
    T* twy = twx + nx;
    load_table(twx, reinterpret_cast<const T*>(a.twf[0]), nx);
    load_table(twy, reinterpret_cast<const T*>(a.twf[1]), ny);
    const int z = blockIdx.x, bc = blockIdx.y;
    const T* in = a.spec + ((size_t)bc * nz + z) * (size_t)nxh * ny;
    for (int i = threadIdx.x; i < nxh * ny; i += blockDim.x) {
        const int y = i % ny, k = i / ny;
        P[(y >> 1) * S + 2 * k + (y & 1)] = in[i];
    }
    __syncthreads();
    lines_fft_n(ny, P, nxh, [S](int k, int y) { return (y >> 1) * S + 2 * k + (y & 1); }, twy,
                true);
    __syncthreads();
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int p = warp; p < ny / 2; p += nw) {
            T* rowp = P + p * S;
            T zv[4];              // nx <= 128 values: at most 4 per lane
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = lane + 32 * r;
                if (k < nx) {
                    const int kk = k <= nx / 2 ? k : nx - k;
                    T e = rowp[2 * kk], o = rowp[2 * kk + 1];
                    if (k == 0 || k == nx / 2) { e.y = R(0); o.y = R(0); }
                    if (k > nx / 2) { e.y = -e.y; o.y = -o.y; }
                    zv[r] = T{e.x - o.y, e.y + o.x};
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = lane + 32 * r;
                if (k < nx) rowp[k] = zv[r];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    lines_fft_n(nx, P, ny / 2, [S](int l, int j) { return l * S + j; }, twx, true);
    __syncthreads();
    const R scale = R(1.0 / (double)g.N);
    R* out = a.v_out + (size_t)bc * g.N + (size_t)z * ny * nx;
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int x = i & (nx - 1), y = i / nx;
        const T zv = P[(y >> 1) * S + x];
        out[i] = ((y & 1) ? zv.y : zv.x) * scale;
    }
}

template <typename R>
cudaError_t launch_fluid3(cudaStream_t st, int B, const GridGeo& g, const FluidArgs<R>& a,
                          cudaEvent_t* marks)
{
    using T = typename C2<R>::T;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    static bool attr[2] = {false, false};
    const int w = sizeof(R) == 8;
    if (!attr[w]) {
        const int lim = 200 * 1024;
        cudaFuncSetAttribute(k_plane_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_zsolve<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_plane_inv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        attr[w] = true;
    }
    const size_t smem_plane = ((size_t)(ny / 2) * plane_ld(nx) + nx + ny) * sizeof(T);
    int C = sizeof(R) == 4 ? 16 : 8;
    if (C > ny) C = ny;
    const size_t smem_z = ((size_t)3 * nz * (C + 2) + nz) * sizeof(T);
    auto mark = [&](int i) { if (marks) cudaEventRecord(marks[i], st); };
    mark(0);
    k_plane_fwd<R><<<dim3(nz, 3 * B), 256, smem_plane, st>>>(a, g);
    mark(1);
    mark(2);
    k_zsolve<R><<<dim3(ny / C, nxh, B), 256, smem_z, st>>>(a, g, C);
    mark(3);
    mark(4);
    k_plane_inv<R><<<dim3(nz, 3 * B), 256, smem_plane, st>>>(a, g);
    mark(5);
    return cudaGetLastError();
}
template cudaError_t launch_fluid3<float>(cudaStream_t, int, const GridGeo&,
                                          const FluidArgs<float>&, cudaEvent_t*);
template cudaError_t launch_fluid3<double>(cudaStream_t, int, const GridGeo&,
                                           const FluidArgs<double>&, cudaEvent_t*);

}  // namespace mbk
