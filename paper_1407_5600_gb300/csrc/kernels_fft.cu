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
// Every pass stages its lines in shared memory (padded against bank conflicts) and transforms
// them with the register line FFTs of fft_lines.cuh; global traffic is one coalesced read and
// one write of the half spectrum per pass.  This pipeline takes sides of up to 256 points.
#include "mb_internal.cuh"
#include "fft_lines.cuh"

namespace mbk {

// Padded position of element j of a line of n points (one spare slot every 2^pad_shift).
__device__ __forceinline__ int pj(int j, int sh) { return j + (j >> sh); }

// ------------------------------------------------------------------------------------------
// Pass 1: rhs stencil + R2C along x.  CTA = RP row pairs of one (box, component, z) plane.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1)
k_rhs_fft_x(FluidArgs<R> a, GridGeo g, int RP)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int sx = pad_shift(nx), ld = padded_len(nx) + 1;
    const int yp0 = blockIdx.x * RP;
    const int z = blockIdx.y;
    const int bc = blockIdx.z;
    const int comp = bc % 3;
    const R* vc = a.v + (size_t)bc * g.N;
    const R* fc = a.f ? a.f + (size_t)bc * g.N : nullptr;
    const R ih2 = kparam<R>(a.inv_h2, a.inv_h2_32);
    const R rho_dt = kparam<R>(a.rho_dt, a.rho_dt32);
    const R half_eta = kparam<R>(a.half_eta, a.half_eta32);
    const bool body = a.body_prof && comp == a.body_axis;
    const size_t zp = (size_t)((z + 1) & (nz - 1)) * ny, zm = (size_t)((z - 1) & (nz - 1)) * ny;
    const size_t z0 = (size_t)z * ny;
    // each work unit: 4 consecutive x (one vector load) of the row pair 2p, 2p+1
    const int qx = nx / 4, lq = 31 - __clz(qx);
    const R* pz = vc + z0 * nx;
    const R* pzp = vc + zp * nx;
    const R* pzm = vc + zm * nx;
    const R* pf = fc ? fc + z0 * nx : nullptr;
    for (int u = threadIdx.x; u < qx * RP; u += blockDim.x) {
        const int x0 = 4 * (u & (qx - 1)), p = u >> lq;
        const int y0 = 2 * (yp0 + p), y1 = y0 + 1;
        R r0[4] = {R(0), R(0), R(0), R(0)}, r1[4] = {R(0), R(0), R(0), R(0)}, t[4];
        if (!a.no_v) {              // Stokes limit (no_v): the right-hand side is f + f_body
            const int ym = (y0 - 1) & (ny - 1), yp = (y1 + 1) & (ny - 1);
            R c0[4], c1[4], am[4], ap[4], l0[4], l1[4];
            load4(pz + (size_t)y0 * nx + x0, c0);
            load4(pz + (size_t)y1 * nx + x0, c1);
            load4(pz + (size_t)ym * nx + x0, am);
            load4(pz + (size_t)yp * nx + x0, ap);
            for (int i = 0; i < 4; ++i) {
                l0[i] = am[i] + c1[i] - R(6) * c0[i];
                l1[i] = c0[i] + ap[i] - R(6) * c1[i];
            }
            load4(pzp + (size_t)y0 * nx + x0, t);
            for (int i = 0; i < 4; ++i) l0[i] += t[i];
            load4(pzm + (size_t)y0 * nx + x0, t);
            for (int i = 0; i < 4; ++i) l0[i] += t[i];
            load4(pzp + (size_t)y1 * nx + x0, t);
            for (int i = 0; i < 4; ++i) l1[i] += t[i];
            load4(pzm + (size_t)y1 * nx + x0, t);
            for (int i = 0; i < 4; ++i) l1[i] += t[i];
            const int xm = (x0 - 1) & (nx - 1), xq = (x0 + 4) & (nx - 1);
            const R e0m = pz[(size_t)y0 * nx + xm], e0p = pz[(size_t)y0 * nx + xq];
            const R e1m = pz[(size_t)y1 * nx + xm], e1p = pz[(size_t)y1 * nx + xq];
            for (int i = 0; i < 4; ++i) {
                l0[i] += (i == 0 ? e0m : c0[i - 1]) + (i == 3 ? e0p : c0[i + 1]);
                l1[i] += (i == 0 ? e1m : c1[i - 1]) + (i == 3 ? e1p : c1[i + 1]);
                r0[i] = rho_dt * c0[i] + half_eta * (l0[i] * ih2);
                r1[i] = rho_dt * c1[i] + half_eta * (l1[i] * ih2);
            }
        }
        if (pf) {
            load4(pf + (size_t)y0 * nx + x0, t);
            for (int i = 0; i < 4; ++i) r0[i] += t[i];
            load4(pf + (size_t)y1 * nx + x0, t);
            for (int i = 0; i < 4; ++i) r1[i] += t[i];
        }
        if (body) {
            for (int i = 0; i < 4; ++i) {
                const int x = x0 + i;
                r0[i] += a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y0 : z)];
                r1[i] += a.body_prof[a.body_dir == 0 ? x : (a.body_dir == 1 ? y1 : z)];
            }
        }
        for (int i = 0; i < 4; ++i) sb[p * ld + pj(x0 + i, sx)] = T{r0[i], r1[i]};
    }
    __syncthreads();
    lines_fft_n<false>(nx, sb, RP, [ld, sx](int l, int j) { return l * ld + pj(j, sx); },
                       reinterpret_cast<const T*>(a.twf[0]));
    __syncthreads();
    T* out = a.spec + ((size_t)bc * nz + z) * (size_t)ny * nxh;
    // row p, frequency k <= nx/2: even row (Z + conj Zr)/2, odd row -i (Z - conj Zr)/2
    auto emit = [&](int p, int k) {
        const T Z = sb[p * ld + pj(k, sx)];
        const T Zr = sb[p * ld + pj((nx - k) & (nx - 1), sx)];
        const T Xa{(Z.x + Zr.x) * R(0.5), (Z.y - Zr.y) * R(0.5)};
        const T Xb{(Z.y + Zr.y) * R(0.5), (Zr.x - Z.x) * R(0.5)};
        const int y = 2 * (yp0 + p);
        out[(size_t)y * nxh + k] = Xa;
        out[(size_t)(y + 1) * nxh + k] = Xb;
    };
    const int hx = nx / 2, lh = 31 - __clz(hx);
    for (int t = threadIdx.x; t < RP * hx; t += blockDim.x) emit(t >> lh, t & (hx - 1));
    for (int p = threadIdx.x; p < RP; p += blockDim.x) emit(p, hx);
}

// Pass 2 / 4: complex FFT along y.  CTA = C consecutive kx columns of one (box, comp, z).
template <typename R, bool INV, int C>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1)
k_fft_y(typename C2<R>::T* spec, const R* twy, GridGeo g)
{
    constexpr int LC = C == 16 ? 4 : 3;
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int kx0 = blockIdx.x * C;
    const int cw = min(C, nxh - kx0);
    const int sy = pad_shift(ny), CL = C + 1;
    T* plane = spec + ((size_t)blockIdx.z * nz + blockIdx.y) * (size_t)ny * nxh + kx0;
    // every copy of a thread in flight at once (index arithmetic in shifts: C and ny are
    // powers of two; columns past the last kx are transformed as garbage and not stored)
    for (int t = threadIdx.x; t < ny * C; t += blockDim.x) {
        const int y = t >> LC, c = t & (C - 1);
        if (c < cw) async_copy(&sb[pj(y, sy) * CL + c], &plane[(size_t)y * nxh + c]);
    }
    async_wait_all();
    __syncthreads();
    auto idx = [CL, sy](int l, int j) { return pj(j, sy) * CL + l; };
    const T* tw = reinterpret_cast<const T*>(twy);
    lines_fft_n<INV>(ny, sb, C, idx, tw);
    __syncthreads();
    for (int t = threadIdx.x; t < ny * C; t += blockDim.x) {
        const int y = t >> LC, c = t & (C - 1);
        if (c < cw) plane[(size_t)y * nxh + c] = sb[pj(y, sy) * CL + c];
    }
}

// Pass 3: FFT along z, Crank-Nicolson divide, projection, k = 0 mode, inverse FFT along z.
// CTA = C consecutive kx columns at one ky of one box, all three components.
template <typename R, int C>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1)
k_fft_z_solve(FluidArgs<R> a, GridGeo g)
{
    constexpr int LC = C == 16 ? 4 : 3;
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
    const int sz = pad_shift(nz), PZ = padded_len(nz), CL = C + 1;
    auto at = [=](int c, int z, int k) { return (c * PZ + pj(z, sz)) * CL + k; };
    // z twiddles in shared memory, after the three component columns (ready at the barrier
    // that follows the column copies)
    T* twz = sb + 3 * PZ * CL;
    for (int i = threadIdx.x; i < nz; i += blockDim.x) twz[i] = reinterpret_cast<const T*>(a.twf[2])[i];
    const int lz = 31 - __clz(nz);
    // index arithmetic in shifts (C and nz are powers of two); columns past the last kx are
    // transformed as garbage and not stored
    for (int t = threadIdx.x; t < 3 * nz * C; t += blockDim.x) {
        const int k = t & (C - 1), z = (t >> LC) & (nz - 1), c = t >> (LC + lz);
        if (k < cw) async_copy(&sb[at(c, z, k)], &col[c][(size_t)z * zstride + k]);
    }
    async_wait_all();
    __syncthreads();
    auto idx = [=](int l, int j) { return at(l >> LC, j, l & (C - 1)); };
    lines_fft_n<false>(nz, sb, 3 * C, idx, twz);
    __syncthreads();

    const R* sym = reinterpret_cast<const R*>(a.symr);      // [9][256] cos, sin, lambda
    const R* cosx = sym + 0 * 256;
    const R* sinx = sym + 1 * 256;
    const R* lamx = sym + 2 * 256;
    const R* cosy = sym + 3 * 256;
    const R* siny = sym + 4 * 256;
    const R* lamy = sym + 5 * 256;
    const R* cosz = sym + 6 * 256;
    const R* sinz = sym + 7 * 256;
    const R* lamz = sym + 8 * 256;
    const R ih = kparam<R>(a.inv_h, a.inv_h32);
    const R rho_dt = kparam<R>(a.rho_dt, a.rho_dt32);
    const R half_eta = kparam<R>(a.half_eta, a.half_eta32);
    for (int t = threadIdx.x; t < nz * C; t += blockDim.x) {
        const int kz = t >> LC, k = t & (C - 1);
        const int kx = kx0 + k;
        T W[3];
        const R lam = R(lamx[kx]) + R(lamy[ky]) + R(lamz[kz]);
        const R cinv = recip(rho_dt + half_eta * lam);
        for (int c = 0; c < 3; ++c) {
            const T v = sb[at(c, kz, k)];
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
            const R il = recip(lam);
            dr *= il;
            di *= il;
            for (int c = 0; c < 3; ++c) {
                const R Gr = (R(1) - cs[c]) * ih, Gi = sn[c] * ih;
                W[c].x += Gr * dr - Gi * di;
                W[c].y += Gr * di + Gi * dr;
            }
        }
        for (int c = 0; c < 3; ++c) sb[at(c, kz, k)] = W[c];
    }
    __syncthreads();
    lines_fft_n<true>(nz, sb, 3 * C, idx, twz);
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nz * C; t += blockDim.x) {
        const int k = t & (C - 1), z = (t >> LC) & (nz - 1), c = t >> (LC + lz);
        if (k < cw) col[c][(size_t)z * zstride + k] = sb[at(c, z, k)];
    }
}

// Pass 5: C2R along x.  Two half-spectrum rows form Z = Xa + i Xb (Hermitian extension),
// one inverse complex FFT gives both real rows.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1)
k_fft_x_c2r(FluidArgs<R> a, GridGeo g, int RP)
{
    using T = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int sx = pad_shift(nx), ld = padded_len(nx) + 1;
    const int yp0 = blockIdx.x * RP;
    const int z = blockIdx.y;
    const int bc = blockIdx.z;
    const T* in = a.spec + ((size_t)bc * nz + z) * (size_t)ny * nxh;
    const int lx = 31 - __clz(nx);
    #pragma unroll 4
    for (int t = threadIdx.x; t < RP * nx; t += blockDim.x) {
        const int k = t & (nx - 1), p = t >> lx;
        const int y = 2 * (yp0 + p);
        T Xa, Xb;
        if (k <= nx / 2) {
            Xa = __ldg(in + (size_t)y * nxh + k);
            Xb = __ldg(in + (size_t)(y + 1) * nxh + k);
            if (k == 0 || k == nx / 2) { Xa.y = R(0); Xb.y = R(0); }
        } else {
            Xa = __ldg(in + (size_t)y * nxh + (nx - k));
            Xb = __ldg(in + (size_t)(y + 1) * nxh + (nx - k));
            Xa.y = -Xa.y;
            Xb.y = -Xb.y;
        }
        sb[p * ld + pj(k, sx)] = T{Xa.x - Xb.y, Xa.y + Xb.x};
    }
    __syncthreads();
    lines_fft_n<true>(nx, sb, RP, [ld, sx](int l, int j) { return l * ld + pj(j, sx); },
                      reinterpret_cast<const T*>(a.twf[0]));
    __syncthreads();
    const R scale = kparam<R>(a.inv_n, a.inv_n32);
    R* out = a.v_out + (size_t)bc * g.N + (size_t)z * ny * nx;
    const int qx = nx / 4, lq = 31 - __clz(qx);
    for (int u = threadIdx.x; u < qx * RP; u += blockDim.x) {
        const int x0 = 4 * (u & (qx - 1)), p = u >> lq;
        R r0[4], r1[4];
        for (int i = 0; i < 4; ++i) {
            const T zv = sb[p * ld + pj(x0 + i, sx)];
            r0[i] = zv.x * scale;
            r1[i] = zv.y * scale;
        }
        store4(out + (size_t)(2 * (yp0 + p)) * nx + x0, r0);
        store4(out + (size_t)(2 * (yp0 + p) + 1) * nx + x0, r1);
    }
}

template <typename R>
cudaError_t launch_fluid(cudaStream_t st, int B, const GridGeo& g, const FluidArgs<R>& a_in,
                         cudaEvent_t* marks)
{
    const FluidArgs<R> a = with_derived(a_in, g);
    using T = typename C2<R>::T;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx / 2 + 1;
    const int RP = ny / 2 < 16 ? ny / 2 : 16;
    constexpr int CY = sizeof(R) == 4 ? 16 : 8, CZ5 = 8;
    const int C = CY;
    static std::atomic<unsigned> attr{0};     // per instantiation
    if (first_on_device(attr)) {
        const int lim = 200 * 1024;
        cudaFuncSetAttribute(k_rhs_fft_x<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_y<R, false, CY>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_y<R, true, CY>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_z_solve<R, CZ5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(k_fft_x_c2r<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    }
    const size_t smem_x = (size_t)RP * (padded_len(nx) + 1) * sizeof(T);
    const size_t smem_y = (size_t)padded_len(ny) * (C + 1) * sizeof(T);
    // the z pass holds three components of its columns: 8 columns keep three blocks per SM
    const int Cz = CZ5;
    const size_t smem_z = ((size_t)3 * padded_len(nz) * (Cz + 1) + nz) * sizeof(T);
    const unsigned nchunk = (unsigned)((nxh + C - 1) / C);
    const unsigned nchunk_z = (unsigned)((nxh + Cz - 1) / Cz);
    auto mark = [&](int i) { if (marks) cudaEventRecord(marks[i], st); };
    mark(0);
    k_rhs_fft_x<R><<<dim3(ny / 2 / RP, nz, 3 * B), 256, smem_x, st>>>(a, g, RP);
    mark(1);
    k_fft_y<R, false, CY><<<dim3(nchunk, nz, 3 * B), 256, smem_y, st>>>(a.spec, a.twf[1], g);
    mark(2);
    k_fft_z_solve<R, CZ5><<<dim3(nchunk_z, ny, B), 256, smem_z, st>>>(a, g);
    mark(3);
    k_fft_y<R, true, CY><<<dim3(nchunk, nz, 3 * B), 256, smem_y, st>>>(a.spec, a.twf[1], g);
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
