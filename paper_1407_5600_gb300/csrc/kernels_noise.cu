// Thermal stress of the fluctuating inertial coupling method (Sec. 3: the Gaussian stress
// sigma~ of Eq. vf, on the staggered grid of fluctuating hydrodynamics that the paper cites).
//
// Per box b and step index n, the cells are drawn in groups of four along x (m = 4 G + r;
// the rows hold a multiple of four cells): five Philox4x64-10 blocks (Salmon, Moraes, Dror
// and Shaw, SC'11) with key (seed, 0) and counters (G, n, b, j), j = 0..4, give the 64-bit
// words x0..x19.  Word x_p gives the Box-Muller pair p: u1 = (low 32 bits + 1/2) / 2^32 and
// u2 = (high 32 bits + 1/2) / 2^32, the normals z_2p = sqrt(-2 ln u1) cos(2 pi u2) and
// z_2p+1 = sqrt(-2 ln u1) sin(2 pi u2).  Cell r takes z_9r .. z_9r+8 as the components xx,
// xy, xz, yx, yy, yz, zx, zy, zz of a non-symmetric stress W (words 18 and 19 are unused);
// sigma~ = sqrt(2 eta kT / (h^3 dt)) W.  W_aa sits at the cell centre, W_ab (b != a)
// on the edge at integer a and b coordinates, so the divergence on the faces of component a
// is a backward difference of W_aa plus forward differences of W_ab, and its covariance is
// -L per component: the fluctuation-dissipation partner of the viscous term.  The fluid
// receives -D.sigma~.
//
// The convective stress rho v v of Eq. (vf) (advection = 1) sits on the same nodes: rho v_a v_a
// at the cell centre from the mean of the two v_a faces, rho v_a v_b on the (a, b) edge from
// v_a averaged along b times v_b averaged along a (the conservative centred form), explicit
// at v^n, so one divergence serves both stresses.
//
// Two launches per step: k_stress forms sigma~ + rho v v into a [B][9][N] buffer (one thread
// per group of four cells, each Philox block computed once, vector stores), k_stress_div adds -D.(sigma~ + rho v v) to the force-density grid
// and advances the step index held in device memory (when drawing noise), so captured CUDA
// graphs draw fresh noise on every replay.
#include "mb_internal.cuh"
#include "fft_lines.cuh"

namespace mbk {

namespace {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// One Box-Muller pair from a 64-bit word (FP64: the uniforms are exact doubles).
__device__ __forceinline__ void box_muller(uint64_t x, double& z0, double& z1)
{
    const double u1 = ((double)(uint32_t)x + 0.5) * 0x1p-32;
    const double u2 = ((double)(uint32_t)(x >> 32) + 0.5) * 0x1p-32;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// FP32: the hardware logarithm and sine/cosine (absolute errors of a few 1e-7 on these
// ranges, far inside the FP32 grid's tolerance).  The angle is taken as 2 pi (u2 - 1/2) in
// [-pi, pi], where the fast sine and cosine keep that accuracy, and the pair is negated back:
// cos(2 pi u2) = -cos(2 pi (u2 - 1/2)), likewise for the sine.
__device__ __forceinline__ void box_muller(uint64_t x, float& z0, float& z1)
{
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    const float u1 = ((float)lo + 0.5f) * 0x1p-32f;
    const float r = sqrtf(-2.0f * __logf(u1));
    const float th = 6.283185307179586f * ((float)((int32_t)(hi - 0x80000000u)) + 0.5f) * 0x1p-32f;
    float s, c;
    __sincosf(th, &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// Periodic neighbours of cell m = i + nx (j + ny k) (the sizes are powers of two).
struct Nbr {
    int64_t xm, xp, ym, yp, zm, zp;
    __device__ Nbr(const GridGeo& g, int64_t m)
    {
        const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
        const int i = (int)(m % nx), j = (int)((m / nx) % ny), k = (int)(m / ((int64_t)nx * ny));
        const int64_t row = m - i, plane = m - (int64_t)j * nx - i;
        xm = row + ((i - 1) & (nx - 1));
        xp = row + ((i + 1) & (nx - 1));
        ym = plane + (int64_t)((j - 1) & (ny - 1)) * nx + i;
        yp = plane + (int64_t)((j + 1) & (ny - 1)) * nx + i;
        zm = m + ((int64_t)((k - 1) & (nz - 1)) - k) * nx * ny;
        zp = m + ((int64_t)((k + 1) & (nz - 1)) - k) * nx * ny;
    }
};

// rho v v at the stress nodes of cell m (xx, xy, xz, yx, yy, yz, zx, zy, zz).
template <typename R>
__device__ __forceinline__ void convective(const GridGeo& g, const R* __restrict__ vx, int64_t m,
                                           R rho, R T[9])
{
    const Nbr nb(g, m);
    const R* vy = vx + g.N;
    const R* vz = vy + g.N;
    const R x0 = __ldg(vx + m), y0 = __ldg(vy + m), z0 = __ldg(vz + m);
    const R h = R(0.5);
    const R cx = h * (x0 + __ldg(vx + nb.xp)), cy = h * (y0 + __ldg(vy + nb.yp)),
            cz = h * (z0 + __ldg(vz + nb.zp));
    const R xy = (h * (x0 + __ldg(vx + nb.ym))) * (h * (y0 + __ldg(vy + nb.xm)));
    const R xz = (h * (x0 + __ldg(vx + nb.zm))) * (h * (z0 + __ldg(vz + nb.xm)));
    const R yz = (h * (y0 + __ldg(vy + nb.zm))) * (h * (z0 + __ldg(vz + nb.ym)));
    T[0] += rho * (cx * cx);
    T[1] += rho * xy;
    T[2] += rho * xz;
    T[3] += rho * xy;
    T[4] += rho * (cy * cy);
    T[5] += rho * yz;
    T[6] += rho * xz;
    T[7] += rho * yz;
    T[8] += rho * (cz * cz);
}

template <typename R>
__global__ void __launch_bounds__(256, 2)
k_stress(int B, GridGeo g, uint64_t seed, const uint64_t* __restrict__ step_index, R amp,
         const R* __restrict__ v, R rho, R* __restrict__ W)
{
    const uint64_t n = amp != R(0) ? *step_index : 0;
    const int64_t groups = g.N / 4, total = (int64_t)B * groups;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / groups, G = t - b * groups, m0 = 4 * G;
        R T[4][9];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 9; ++c) T[r][c] = R(0);
        if (amp != R(0)) {
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                uint64_t x[4] = {(uint64_t)G, n, (uint64_t)b, (uint64_t)j};
                philox4x64_10(x, seed, 0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int p = 4 * j + i;             // pair p: normals 2p and 2p + 1
                    if (p < 18) {
                        R z0, z1;
                        box_muller(x[i], z0, z1);
                        T[(2 * p) / 9][(2 * p) % 9] = amp * z0;
                        T[(2 * p + 1) / 9][(2 * p + 1) % 9] = amp * z1;
                    }
                }
            }
        }
        if (v) {
            const R* vx = v + (size_t)b * 3 * g.N;
#pragma unroll
            for (int r = 0; r < 4; ++r) convective(g, vx, m0 + r, rho, T[r]);
        }
        R* Wb = W + (size_t)b * 9 * g.N + m0;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const R q[4] = {T[0][c], T[1][c], T[2][c], T[3][c]};
            store4(Wb + (size_t)c * g.N, q);
        }
    }
}

// f (+)= -D.sigma~ / h on the faces of all three components of cell (i, j, k).
template <typename R>
__global__ void __launch_bounds__(256)
k_stress_div(int B, GridGeo g, const R* __restrict__ W, R* __restrict__ f, int accumulate,
             uint64_t* __restrict__ step_index)
{
    // four consecutive cells along x per thread: vector loads of the stress rows, scalar
    // loads of the two x neighbours outside the four
    const R mih = R(-g.inv_h);
    const int nx = g.n[0];
    const int64_t groups = g.N / 4, total = (int64_t)B * groups;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / groups, m = 4 * (t - b * groups);
        const Nbr nb(g, m);
        const int i0 = (int)(m % nx);
        const int64_t row = m - i0;
        const int64_t xl = row + ((i0 - 1) & (nx - 1)), xr = row + ((i0 + 4) & (nx - 1));
        const int64_t dy = nb.yp - m, dz = nb.zp - m, ey = m - nb.ym, ez = m - nb.zm;
        const R* Wb = W + (size_t)b * 9 * g.N;
        auto row4 = [&](int comp, int64_t cell, R v[4]) { load4(Wb + (size_t)comp * g.N + cell, v); };
        auto one = [&](int comp, int64_t cell) { return __ldg(Wb + (size_t)comp * g.N + cell); };
        R c[4], e[4], d[3][4];
        // x component: W_xx backward in x, W_xy forward in y, W_xz forward in z
        row4(0, m, c);
        const R xxl = one(0, xl);
        for (int i = 0; i < 4; ++i) d[0][i] = c[i] - (i == 0 ? xxl : c[i - 1]);
        row4(1, m, c);
        row4(1, m + dy, e);
        for (int i = 0; i < 4; ++i) d[0][i] += e[i] - c[i];
        row4(2, m, c);
        row4(2, m + dz, e);
        for (int i = 0; i < 4; ++i) d[0][i] += e[i] - c[i];
        // y component: W_yx forward in x, W_yy backward in y, W_yz forward in z
        row4(3, m, c);
        const R yxr = one(3, xr);
        for (int i = 0; i < 4; ++i) d[1][i] = (i == 3 ? yxr : c[i + 1]) - c[i];
        row4(4, m, c);
        row4(4, m - ey, e);
        for (int i = 0; i < 4; ++i) d[1][i] += c[i] - e[i];
        row4(5, m, c);
        row4(5, m + dz, e);
        for (int i = 0; i < 4; ++i) d[1][i] += e[i] - c[i];
        // z component: W_zx forward in x, W_zy forward in y, W_zz backward in z
        row4(6, m, c);
        const R zxr = one(6, xr);
        for (int i = 0; i < 4; ++i) d[2][i] = (i == 3 ? zxr : c[i + 1]) - c[i];
        row4(7, m, c);
        row4(7, m + dy, e);
        for (int i = 0; i < 4; ++i) d[2][i] += e[i] - c[i];
        row4(8, m, c);
        row4(8, m - ez, e);
        for (int i = 0; i < 4; ++i) d[2][i] += c[i] - e[i];
        R* fb = f + (size_t)b * 3 * g.N + m;
        for (int a = 0; a < 3; ++a) {
            R out[4];
            if (accumulate) load4(fb + (size_t)a * g.N, out);
            for (int i = 0; i < 4; ++i) out[i] = accumulate ? out[i] + mih * d[a][i] : mih * d[a][i];
            store4(fb + (size_t)a * g.N, out);
        }
    }
    if (step_index && blockIdx.x == 0 && threadIdx.x == 0) *step_index += 1;
}

unsigned noise_blocks(int64_t total)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const int64_t want = (total + 255) / 256, cap = (int64_t)sms * 8;
    return (unsigned)(want < cap ? want : cap);
}

}  // namespace

template <typename R>
cudaError_t launch_fluid_stress(cudaStream_t st, int B, const GridGeo& g, uint64_t seed,
                                uint64_t* step_index, double amp, const R* v, double rho, R* W,
                                R* f, bool accumulate, int parts)
{
    const int64_t total = (int64_t)B * g.N;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = noise_blocks(total);
    if (parts & 1) k_stress<R><<<blocks, 256, 0, st>>>(B, g, seed, step_index, R(amp), v, R(rho), W);
    if (parts & 2)
        k_stress_div<R><<<blocks, 256, 0, st>>>(B, g, W, f, accumulate ? 1 : 0,
                                                amp != 0.0 ? step_index : nullptr);
    return cudaGetLastError();
}
template cudaError_t launch_fluid_stress<float>(cudaStream_t, int, const GridGeo&, uint64_t,
                                                uint64_t*, double, const float*, double, float*,
                                                float*, bool, int);
template cudaError_t launch_fluid_stress<double>(cudaStream_t, int, const GridGeo&, uint64_t,
                                                 uint64_t*, double, const double*, double,
                                                 double*, double*, bool, int);

}  // namespace mbk
