// Fluid update on the periodic MAC grid: Crank-Nicolson viscous step and exact discrete
// projection (Eq. vf with the viscous stress), solved in Fourier space.
//
// Pipeline per box and component (each component transformed on its own index grid):
//   pass 1  rhs = (rho/dt) v + (eta/2) L v + f + f_body, then real-to-complex FFT along x
//           (two real rows packed into one complex row)           -> spec [z][y][kx]
//   pass 2  complex FFT along y                                     (in place)
//   pass 3  complex FFT along z, divide by rho/dt + (eta/2) lambda(k), project with the MAC
//           divergence/gradient symbols, set the k = 0 mode, inverse FFT along z
//   pass 4  inverse FFT along y
//   pass 5  complex-to-real inverse FFT along x, scale 1/N         -> v_out
// Every pass stages its lines in shared memory and runs radix-2 butterflies there; global
// traffic is one coalesced read and one write of the half spectrum per pass.
#include "mb_internal.cuh"

namespace mbk {

template <typename T> __device__ __forceinline__ T cmul(T a, T b)
{
    return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

__device__ __forceinline__ int ilog2(int n) { return 31 - __clz(n); }

// In-place radix-2 decimation-in-time FFT of ngroups*cw lines held in shared memory.
// Line (g, c) stores element j at buf[g*gstride + c + j*estride].  tw[m] = e^{-2 pi i m/n}.
// Forward: X_k = sum_j x_j e^{-2 pi i jk/n}; inverse uses e^{+...} with no scaling.
template <typename T>
__device__ void smem_fft(T* buf, int n, int ngroups, int gstride, int cw, int estride,
                         const T* __restrict__ tw, bool inverse)
{
    const int logn = ilog2(n);
    const int nl = ngroups * cw;
    for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
        const int l = t % nl, j = t / nl;
        const int r = (int)(__brev((unsigned)j) >> (32 - logn));
        if (r > j) {
            T* base = buf + (l / cw) * gstride + (l % cw);
            const T tmp = base[j * estride];
            base[j * estride] = base[r * estride];
            base[r * estride] = tmp;
        }
    }
    __syncthreads();
    for (int s = 1; s <= logn; ++s) {
        const int half = 1 << (s - 1);
        for (int t = threadIdx.x; t < nl * (n >> 1); t += blockDim.x) {
            const int l = t % nl, bf = t / nl;
            const int m = bf & (half - 1);
            const int i0 = ((bf >> (s - 1)) << s) + m;
            T w = tw[m << (logn - s)];
            if (inverse) w.y = -w.y;
            T* base = buf + (l / cw) * gstride + (l % cw);
            const T a = base[i0 * estride];
            const T b = cmul(base[(i0 + half) * estride], w);
            base[i0 * estride] = T{a.x + b.x, a.y + b.y};
            base[(i0 + half) * estride] = T{a.x - b.x, a.y - b.y};
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Pass 1: rhs stencil + R2C along x.  CTA = RP row pairs of one (box, component, z) plane.
template <typename R>
__global__ void __launch_bounds__(256)
k_rhs_fft_x(FluidArgs<R> a, GridGeo g, int RP)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int ld = nx + 1;
    const int yp0 = blockIdx.x * RP;
    const int z = blockIdx.y;
    const int bc = blockIdx.z;
    const int comp = bc % 3;
    const R* vc = a.v + (size_t)bc * g.N;
    const R* fc = a.f ? a.f + (size_t)bc * g.N : nullptr;
    const R ih2 = R(g.inv_h * g.inv_h);
    const R rho_dt = R(a.rho_dt), half_eta = R(a.half_eta);
    const bool body = a.body_prof && comp == a.body_axis;
    const size_t zp = (size_t)((z + 1) & (nz - 1)) * ny, zm = (size_t)((z - 1) & (nz - 1)) * ny;
    const size_t z0 = (size_t)z * ny;
    for (int t = threadIdx.x; t < 2 * RP * nx; t += blockDim.x) {
        const int x = t % nx, r = t / nx;
        const int y = 2 * yp0 + r;
        const int yp = (y + 1) & (ny - 1), ym = (y - 1) & (ny - 1);
        const int xp = (x + 1) & (nx - 1), xm = (x - 1) & (nx - 1);
        R val = R(0);               // Stokes limit (no_v): the right-hand side is f + f_body
        if (!a.no_v) {
            const R vcen = vc[(z0 + y) * nx + x];
            const R lap = ((vc[(z0 + y) * nx + xp] + vc[(z0 + y) * nx + xm]) +
                           (vc[(z0 + yp) * nx + x] + vc[(z0 + ym) * nx + x]) +
                           (vc[(zp + y) * nx + x] + vc[(zm + y) * nx + x]) - R(6) * vcen) * ih2;
            val = rho_dt * vcen + half_eta * lap;
        }
        if (fc) val += fc[(z0 + y) * nx + x];
        if (body) val += a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y : z)];
        T* slot = sb + (r >> 1) * ld + x;
        if (r & 1) slot->y = val; else slot->x = val;
    }
    __syncthreads();
    smem_fft<T>(sb, nx, RP, ld, 1, 1, reinterpret_cast<const T*>(a.tw[0]), false);
    T* out = a.spec + ((size_t)bc * nz + z) * (size_t)ny * nxh;
    for (int t = threadIdx.x; t < RP * nxh; t += blockDim.x) {
        const int k = t % nxh, p = t / nxh;
        const T Z = sb[p * ld + k];
        const T Zr = sb[p * ld + ((nx - k) & (nx - 1))];
        // even row: (Z + conj Zr)/2 ; odd row: -i (Z - conj Zr)/2
        const T Xa{(Z.x + Zr.x) * R(0.5), (Z.y - Zr.y) * R(0.5)};
        const T Xb{(Z.y + Zr.y) * R(0.5), (Zr.x - Z.x) * R(0.5)};
        const int y = 2 * (yp0 + p);
        out[(size_t)y * nxh + k] = Xa;
        out[(size_t)(y + 1) * nxh + k] = Xb;
    }
}

// Pass 2 / 4: complex FFT along y.  CTA = C consecutive kx columns of one (box, comp, z).
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_y(typename C2<R>::T* spec, const R* twy, GridGeo g, int C, bool inverse)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int kx0 = blockIdx.x * C;
    const int cw = min(C, nxh - kx0);
    T* plane = spec + ((size_t)blockIdx.z * nz + blockIdx.y) * (size_t)ny * nxh + kx0;
    for (int t = threadIdx.x; t < ny * cw; t += blockDim.x) {
        const int y = t / cw, c = t % cw;
        sb[y * C + c] = plane[(size_t)y * nxh + c];
    }
    __syncthreads();
    smem_fft<T>(sb, ny, 1, 0, cw, C, reinterpret_cast<const T*>(twy), inverse);
    for (int t = threadIdx.x; t < ny * cw; t += blockDim.x) {
        const int y = t / cw, c = t % cw;
        plane[(size_t)y * nxh + c] = sb[y * C + c];
    }
}

// Pass 3: FFT along z, Crank-Nicolson divide, projection, k = 0 mode, inverse FFT along z.
// CTA = C consecutive kx columns at one ky of one box, all three components.
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_z_solve(FluidArgs<R> a, GridGeo g, int C)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);    // [3][nz][C]
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int kx0 = blockIdx.x * C;
    const int cw = min(C, nxh - kx0);
    const int ky = blockIdx.y;
    const int box = blockIdx.z;
    const size_t zstride = (size_t)ny * nxh;
    T* col[3];
    for (int c = 0; c < 3; ++c)
        col[c] = a.spec + ((size_t)(box * 3 + c) * nz) * zstride + (size_t)ky * nxh + kx0;
    for (int t = threadIdx.x; t < 3 * nz * cw; t += blockDim.x) {
        const int c = t / (nz * cw), rem = t % (nz * cw);
        const int z = rem / cw, k = rem % cw;
        sb[(c * nz + z) * C + k] = col[c][(size_t)z * zstride + k];
    }
    __syncthreads();
    const T* twz = reinterpret_cast<const T*>(a.tw[2]);
    smem_fft<T>(sb, nz, 3, nz * C, cw, C, twz, false);

    const double* cosx = a.sym + 0 * 256;
    const double* sinx = a.sym + 1 * 256;
    const double* lamx = a.sym + 2 * 256;
    const double* cosy = a.sym + 3 * 256;
    const double* siny = a.sym + 4 * 256;
    const double* lamy = a.sym + 5 * 256;
    const double* cosz = a.sym + 6 * 256;
    const double* sinz = a.sym + 7 * 256;
    const double* lamz = a.sym + 8 * 256;
    const R ih = R(g.inv_h);
    for (int t = threadIdx.x; t < nz * cw; t += blockDim.x) {
        const int kz = t / cw, k = t % cw;
        const int kx = kx0 + k;
        T W[3];
        const R lam = R(lamx[kx]) + R(lamy[ky]) + R(lamz[kz]);
        const R cinv = R(1) / (R(a.rho_dt) + R(a.half_eta) * lam);
        for (int c = 0; c < 3; ++c) {
            const T v = sb[(c * nz + kz) * C + k];
            W[c] = T{v.x * cinv, v.y * cinv};
        }
        if (kx == 0 && ky == 0 && kz == 0) {
            for (int c = 0; c < 3; ++c) {
                if (a.mean_override) W[c] = T{R((double)g.N * a.mean_override[3 * box + c]), R(0)};
                else if (a.mean_mode == 1) W[c] = T{R(0), R(0)};
            }
        } else {
            // D_a = (e^{i th} - 1)/h (faces -> centres), G_a = (1 - e^{-i th})/h (centres ->
            // faces); D.G = -lambda, so P W = W + G (D.W) / lambda.
            const R cs[3] = {R(cosx[kx]), R(cosy[ky]), R(cosz[kz])};
            const R sn[3] = {R(sinx[kx]), R(siny[ky]), R(sinz[kz])};
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
        for (int c = 0; c < 3; ++c) sb[(c * nz + kz) * C + k] = W[c];
    }
    __syncthreads();
    smem_fft<T>(sb, nz, 3, nz * C, cw, C, twz, true);
    for (int t = threadIdx.x; t < 3 * nz * cw; t += blockDim.x) {
        const int c = t / (nz * cw), rem = t % (nz * cw);
        const int z = rem / cw, k = rem % cw;
        col[c][(size_t)z * zstride + k] = sb[(c * nz + z) * C + k];
    }
}

// Pass 5: C2R along x.  Two half-spectrum rows form Z = Xa + i Xb (Hermitian extension),
// one inverse complex FFT gives both real rows.
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_x_c2r(FluidArgs<R> a, GridGeo g, int RP)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int ld = nx + 1;
    const int yp0 = blockIdx.x * RP;
    const int z = blockIdx.y;
    const int bc = blockIdx.z;
    const T* in = a.spec + ((size_t)bc * nz + z) * (size_t)ny * nxh;
    for (int t = threadIdx.x; t < RP * nx; t += blockDim.x) {
        const int k = t % nx, p = t / nx;
        const int y = 2 * (yp0 + p);
        T Xa, Xb;
        if (k <= nx / 2) {
            Xa = in[(size_t)y * nxh + k];
            Xb = in[(size_t)(y + 1) * nxh + k];
            if (k == 0 || k == nx / 2) { Xa.y = R(0); Xb.y = R(0); }
        } else {
            Xa = in[(size_t)y * nxh + (nx - k)];
            Xb = in[(size_t)(y + 1) * nxh + (nx - k)];
            Xa.y = -Xa.y;
            Xb.y = -Xb.y;
        }
        sb[p * ld + k] = T{Xa.x - Xb.y, Xa.y + Xb.x};
    }
    __syncthreads();
    smem_fft<T>(sb, nx, RP, ld, 1, 1, reinterpret_cast<const T*>(a.tw[0]), true);
    const R scale = R(1.0 / (double)g.N);
    R* out = a.v_out + (size_t)bc * g.N + (size_t)z * ny * nx;
    for (int t = threadIdx.x; t < 2 * RP * nx; t += blockDim.x) {
        const int x = t % nx, r = t / nx;
        const T zv = sb[(r >> 1) * ld + x];
        out[(size_t)(2 * yp0 + r) * nx + x] = ((r & 1) ? zv.y : zv.x) * scale;
    }
}

template <typename R>
cudaError_t launch_fluid(cudaStream_t st, int B, const GridGeo& g, const FluidArgs<R>& a,
                         cudaEvent_t* marks)
{
    using T = typename C2<R>::T;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int RP = ny / 2 < 4 ? ny / 2 : 4;
    const int C = sizeof(R) == 4 ? 16 : 8;
    static std::atomic<unsigned> attr{0};     // per instantiation
    if (first_on_device(attr)) {
        const int lim = 200 * 1024;
        cudaFuncSetAttribute(k_rhs_fft_x<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_y<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_z_solve<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_x_c2r<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    }
    const size_t smem_x = (size_t)RP * (nx + 1) * sizeof(T);
    const size_t smem_y = (size_t)ny * C * sizeof(T);
    const size_t smem_z = (size_t)3 * nz * C * sizeof(T);
    const unsigned nchunk = (unsigned)((nxh + C - 1) / C);
    auto mark = [&](int i) { if (marks) cudaEventRecord(marks[i], st); };
    mark(0);
    k_rhs_fft_x<R><<<dim3(ny / 2 / RP, nz, 3 * B), 256, smem_x, st>>>(a, g, RP);
    mark(1);
    k_fft_y<R><<<dim3(nchunk, nz, 3 * B), 256, smem_y, st>>>(a.spec, a.tw[1], g, C, false);
    mark(2);
    k_fft_z_solve<R><<<dim3(nchunk, ny, B), 256, smem_z, st>>>(a, g, C);
    mark(3);
    k_fft_y<R><<<dim3(nchunk, nz, 3 * B), 256, smem_y, st>>>(a.spec, a.tw[1], g, C, true);
    mark(4);
    k_fft_x_c2r<R><<<dim3(ny / 2 / RP, nz, 3 * B), 256, smem_x, st>>>(a, g, RP);
    mark(5);
    return cudaGetLastError();
}
template cudaError_t launch_fluid<float>(cudaStream_t, int, const GridGeo&,
                                         const FluidArgs<float>&, cudaEvent_t*);
template cudaError_t launch_fluid<double>(cudaStream_t, int, const GridGeo&,
                                          const FluidArgs<double>&, cudaEvent_t*);

}  // namespace mbk
