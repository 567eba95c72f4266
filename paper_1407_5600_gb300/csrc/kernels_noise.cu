// Thermal stress of the fluctuating inertial coupling method (Sec. 3: the Gaussian stress
// sigma~ of Eq. vf, on the staggered grid of fluctuating hydrodynamics that the paper cites).
//
// Per box b, step index n and cell m (x fastest), nine standard normals come from two
// Philox4x64-10 blocks (Salmon, Moraes, Dror and Shaw, SC'11) with key (seed, 0) and counters
// (m, n, b, 0), (m, n, b, 1).  The 64-bit words x0..x4 give five Box-Muller pairs: from x_p,
// u1 = (low 32 bits + 1/2) / 2^32 and u2 = (high 32 bits + 1/2) / 2^32, the normals
// sqrt(-2 ln u1) cos(2 pi u2) and sqrt(-2 ln u1) sin(2 pi u2).  The first nine are the
// components xx, xy, xz, yx, yy, yz, zx, zy, zz of a non-symmetric stress W (the tenth is
// dropped); sigma~ = sqrt(2 eta kT / (h^3 dt)) W.  W_aa sits at the cell centre, W_ab (b != a)
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
// Two launches per step: k_stress forms sigma~ + rho v v into a [B][9][N] buffer (each Philox
// block is computed once), k_stress_div adds -D.(sigma~ + rho v v) to the force-density grid
// and advances the step index held in device memory (when drawing noise), so captured CUDA
// graphs draw fresh noise on every replay.
#include "mb_internal.cuh"

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

// FP32: ln u1 from u1 itself below 1/2 and from 1 - u1 = (~lo + 1/2) / 2^32 above, so that
// the logarithm keeps its relative accuracy as u1 -> 1.
__device__ __forceinline__ void box_muller(uint64_t x, float& z0, float& z1)
{
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    const float ln_u1 = lo < 0x80000000u ? logf(((float)lo + 0.5f) * 0x1p-32f)
                                         : log1pf(-(((float)(~lo) + 0.5f) * 0x1p-32f));
    const float r = sqrtf(-2.0f * ln_u1);
    const float u2 = ((float)hi + 0.5f) * 0x1p-32f;
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
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

template <typename R>
__global__ void __launch_bounds__(256)
k_stress(int B, GridGeo g, uint64_t seed, const uint64_t* __restrict__ step_index, R amp,
         const R* __restrict__ v, R rho, R* __restrict__ W)
{
    const uint64_t n = amp != R(0) ? *step_index : 0;
    const int64_t total = (int64_t)B * g.N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / g.N, m = t - b * g.N;
        R T[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) T[c] = R(0);
        if (amp != R(0)) {
            uint64_t x[8];
            for (int j = 0; j < 2; ++j) {
                uint64_t c[4] = {(uint64_t)m, n, (uint64_t)b, (uint64_t)j};
                philox4x64_10(c, seed, 0);
                for (int i = 0; i < 4; ++i) x[4 * j + i] = c[i];
            }
            R z[10];
#pragma unroll
            for (int p = 0; p < 5; ++p) box_muller(x[p], z[2 * p], z[2 * p + 1]);
#pragma unroll
            for (int c = 0; c < 9; ++c) T[c] = amp * z[c];
        }
        if (v) {
            const Nbr nb(g, m);
            const R* vx = v + (size_t)b * 3 * g.N;
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
        R* Wb = W + (size_t)b * 9 * g.N + m;
#pragma unroll
        for (int c = 0; c < 9; ++c) Wb[(size_t)c * g.N] = T[c];
    }
}

// f (+)= -D.sigma~ / h on the faces of all three components of cell (i, j, k).
template <typename R>
__global__ void __launch_bounds__(256)
k_stress_div(int B, GridGeo g, const R* __restrict__ W, R* __restrict__ f, int accumulate,
             uint64_t* __restrict__ step_index)
{
    const R mih = R(-g.inv_h);
    const int64_t total = (int64_t)B * g.N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / g.N, m = t - b * g.N;
        const Nbr nb(g, m);
        const int64_t xm = nb.xm, xp = nb.xp, ym = nb.ym, yp = nb.yp, zm = nb.zm, zp = nb.zp;
        const R* Wb = W + (size_t)b * 9 * g.N;
        auto w = [&](int comp, int64_t cell) { return __ldg(Wb + (size_t)comp * g.N + cell); };
        R d[3];
        d[0] = (w(0, m) - w(0, xm)) + (w(1, yp) - w(1, m)) + (w(2, zp) - w(2, m));
        d[1] = (w(3, xp) - w(3, m)) + (w(4, m) - w(4, ym)) + (w(5, zp) - w(5, m));
        d[2] = (w(6, xp) - w(6, m)) + (w(7, yp) - w(7, m)) + (w(8, m) - w(8, zm));
        R* fb = f + (size_t)b * 3 * g.N + m;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R add = mih * d[a];
            fb[(size_t)a * g.N] = accumulate ? fb[(size_t)a * g.N] + add : add;
        }
    }
    if (step_index && blockIdx.x == 0 && threadIdx.x == 0) *step_index += 1;
}

unsigned noise_blocks(int64_t total)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int64_t want = (total + 255) / 256, cap = (int64_t)sms * 8;
    return (unsigned)(want < cap ? want : cap);
}

}  // namespace

template <typename R>
cudaError_t launch_fluid_stress(cudaStream_t st, int B, const GridGeo& g, uint64_t seed,
                                uint64_t* step_index, double amp, const R* v, double rho, R* W,
                                R* f, bool accumulate)
{
    const int64_t total = (int64_t)B * g.N;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = noise_blocks(total);
    k_stress<R><<<blocks, 256, 0, st>>>(B, g, seed, step_index, R(amp), v, R(rho), W);
    k_stress_div<R><<<blocks, 256, 0, st>>>(B, g, W, f, accumulate ? 1 : 0,
                                            amp != 0.0 ? step_index : nullptr);
    return cudaGetLastError();
}
template cudaError_t launch_fluid_stress<float>(cudaStream_t, int, const GridGeo&, uint64_t,
                                                uint64_t*, double, const float*, double, float*,
                                                float*, bool);
template cudaError_t launch_fluid_stress<double>(cudaStream_t, int, const GridGeo&, uint64_t,
                                                 uint64_t*, double, const double*, double,
                                                 double*, double*, bool);

}  // namespace mbk
