// Kernels of the adjoint (reverse-mode derivative) of the ICM step, FP64.
//
// The step's position dependence enters through the kernel weights of J and S and through the
// blob forces.  Their transposes are
//   d/dq_i [ sum_a c_ia J_i(q) w_a ]          = sum_a c_ia sum_nodes grad_q(prod Phi) w_a(node)
//   d/dq_i [ <g, S(q) F> ]                    = h^-3 sum_a F_ia sum_nodes grad_q(prod Phi) g_a(node)
// (gradient interpolation with the kernel derivative Phi', continuous because Phi is C^1), and
// the force Jacobian-vector product (dF/dq)^T g = (dF/dq) g (forces derive from a potential),
// bond by bond: J_f (g_i - g_j) with J_f = df/dr.
#include "mb_internal.cuh"
#include "peskin.cuh"

namespace mbk {

namespace {

// Window weights and their derivatives with respect to x = q/h - shift (see peskin_window):
// with t = x - i0 and s = sqrt(1 - 3t^2): dPhi/dt at i0-1, i0, i0+1 = (t/s - 1)/2, -t/s,
// (1 + t/s)/2.
__device__ __forceinline__ int peskin_window_d(double x, double w[3], double dw[3])
{
    const double fl = floor(x + 0.5);
    const double t = x - fl;
    const double s = sqrt(1.0 - 3.0 * t * t);
    w[0] = (2.0 - 3.0 * t - s) / 6.0;
    w[1] = (1.0 + s) / 3.0;
    w[2] = (2.0 + 3.0 * t - s) / 6.0;
    const double ts = t / s;
    dw[0] = 0.5 * (ts - 1.0);
    dw[1] = -ts;
    dw[2] = 0.5 * (1.0 + ts);
    return (int)fl - 1;
}

// out_i += scale * sum_a c_ia grad_{q_i} sum_nodes prod_b Phi_a(node - q_i) w_a(node)
__global__ void __launch_bounds__(256)
k_grad_interp(int64_t nb, const double* __restrict__ q, const double* __restrict__ w,
              const double* __restrict__ c, GridGeo g, double scale, double* __restrict__ out)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    double gr[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        const double ca = c[3 * b + a];
        if (ca == 0.0) continue;
        double wx[3], wy[3], wz[3], dx[3], dy[3], dz[3];
        const int ix = peskin_window_d(q[3 * b] * g.inv_h - mac_shift(a, 0), wx, dx);
        const int iy = peskin_window_d(q[3 * b + 1] * g.inv_h - mac_shift(a, 1), wy, dy);
        const int iz = peskin_window_d(q[3 * b + 2] * g.inv_h - mac_shift(a, 2), wz, dz);
        const double* wa = w + (size_t)a * g.N;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int kz = 0; kz < 3; ++kz) {
            const int zz = (iz + kz) & (nz - 1);
            for (int ky = 0; ky < 3; ++ky) {
                const int yy = (iy + ky) & (ny - 1);
                const size_t row = ((size_t)zz * ny + yy) * nx;
                for (int kx = 0; kx < 3; ++kx) {
                    const double val = wa[row + ((ix + kx) & (nx - 1))];
                    sx += dx[kx] * wy[ky] * wz[kz] * val;
                    sy += wx[kx] * dy[ky] * wz[kz] * val;
                    sz += wx[kx] * wy[ky] * dz[kz] * val;
                }
            }
        }
        gr[0] += ca * sx;
        gr[1] += ca * sy;
        gr[2] += ca * sz;
    }
    // dt/dq = 1/h
    for (int d = 0; d < 3; ++d) out[3 * b + d] += scale * g.inv_h * gr[d];
}

// Hessian-vector product of the blob forces and the spring-stiffness derivative.
//   out_b += sum_bonds J_s(r_bj) (g_b - g_j) + sum_pairs J_r(r_bj) (g_b - g_j)
//   J_s = -k [(1 - r0/|r|) I + (r0/|r|) rhat rhat^T]
//   J_r = k_rep [(r_cut/|r| - 1) I - (r_cut/|r|) rhat rhat^T]         (|r| < r_cut)
//   dL/dk += (1/2) sum_b sum_bonds (f_bond(r_bj)/k) . (g_b - g_j)    (each bond seen twice)
__global__ void __launch_bounds__(256)
k_force_jvp(int64_t nb, const double* __restrict__ q, const double* __restrict__ gF,
            const int32_t* __restrict__ pid, const int32_t* __restrict__ adj_start,
            const int32_t* __restrict__ adj_j, const double* __restrict__ adj_rest,
            double k_spring, double k_rep, double r_cut, const int32_t* __restrict__ cell_start,
            const int32_t* __restrict__ sorted, const int32_t* __restrict__ blob_cell,
            GridGeo g, BinGeo bg, double* __restrict__ out, double* __restrict__ gk)
{
    __shared__ double sh[32];
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double dk = 0.0;
    if (b < nb) {
        const double qb[3] = {q[3 * b], q[3 * b + 1], q[3 * b + 2]};
        const double gb[3] = {gF[3 * b], gF[3 * b + 1], gF[3 * b + 2]};
        double acc[3] = {0.0, 0.0, 0.0};
        for (int e = adj_start[b]; e < adj_start[b + 1]; ++e) {
            const int j = adj_j[e];
            double r[3], dg[3];
            for (int d = 0; d < 3; ++d) {
                r[d] = min_image(qb[d] - q[3 * j + d], g.L[d]);
                dg[d] = gb[d] - gF[3 * j + d];
            }
            const double len = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const double rdg = (r[0] * dg[0] + r[1] * dg[1] + r[2] * dg[2]) / len;
            const double a0 = -k_spring * (1.0 - adj_rest[e] / len);
            const double a1 = -k_spring * (adj_rest[e] / len);
            for (int d = 0; d < 3; ++d) acc[d] += a0 * dg[d] + a1 * rdg * r[d] / len;
            // f_bond / k = -(|r| - r0) r/|r|
            const double fk = -(len - adj_rest[e]) / len;
            dk += 0.5 * fk * (r[0] * dg[0] + r[1] * dg[1] + r[2] * dg[2]);
        }
        if (k_rep != 0.0 && r_cut > 0.0) {
            const int cell = blob_cell[b];
            const int c[3] = {cell % bg.nc[0], (cell / bg.nc[0]) % bg.nc[1],
                              cell / (bg.nc[0] * bg.nc[1])};
            int lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                if (bg.nc[d] >= 3) { lo[d] = -1; hi[d] = 1; }
                else { lo[d] = 0; hi[d] = bg.nc[d] - 1; }
            }
            for (int dz = lo[2]; dz <= hi[2]; ++dz)
                for (int dy = lo[1]; dy <= hi[1]; ++dy)
                    for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                        const int cx = bg.nc[0] >= 3 ? (c[0] + dx + bg.nc[0]) % bg.nc[0] : dx;
                        const int cy = bg.nc[1] >= 3 ? (c[1] + dy + bg.nc[1]) % bg.nc[1] : dy;
                        const int cz = bg.nc[2] >= 3 ? (c[2] + dz + bg.nc[2]) % bg.nc[2] : dz;
                        const int64_t cc = ((int64_t)cz * bg.nc[1] + cy) * bg.nc[0] + cx;
                        for (int t = cell_start[cc]; t < cell_start[cc + 1]; ++t) {
                            const int j = sorted[t];
                            if (j == b || pid[j] == pid[b]) continue;
                            double r[3];
                            for (int d = 0; d < 3; ++d) r[d] = min_image(qb[d] - q[3 * j + d], g.L[d]);
                            const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                            if (r2 >= r_cut * r_cut || r2 == 0.0) continue;
                            const double len = sqrt(r2);
                            double dg[3];
                            for (int d = 0; d < 3; ++d) dg[d] = gb[d] - gF[3 * j + d];
                            const double rdg = (r[0] * dg[0] + r[1] * dg[1] + r[2] * dg[2]) / len;
                            const double a0 = k_rep * (r_cut / len - 1.0);
                            const double a1 = -k_rep * (r_cut / len);
                            for (int d = 0; d < 3; ++d) acc[d] += a0 * dg[d] + a1 * rdg * r[d] / len;
                        }
                    }
        }
        for (int d = 0; d < 3; ++d) out[3 * b + d] += acc[d];
    }
    // block sum of dk, one double atomic per block
    for (int o = 16; o > 0; o >>= 1) dk += __shfl_down_sync(0xffffffffu, dk, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dk;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0 && gk) atomicAdd(gk, x);
    }
}

// out = a x + b y (elementwise), y may be null (then out = a x).
__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_grad_interp(cudaStream_t st, int64_t nb, const double* q, const double* w,
                               const double* c, const GridGeo& g, double scale, double* out)
{
    if (nb <= 0) return cudaSuccess;
    k_grad_interp<<<nblk(nb), 256, 0, st>>>(nb, q, w, c, g, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_force_jvp(cudaStream_t st, int64_t nb, const double* q, const double* gF,
                             const int32_t* pid, const int32_t* adj_start, const int32_t* adj_j,
                             const double* adj_rest, double k_spring, double k_rep, double r_cut,
                             const int32_t* cell_start, const int32_t* sorted,
                             const int32_t* blob_cell, const GridGeo& g, const BinGeo& bg,
                             double* out, double* gk)
{
    if (nb <= 0) return cudaSuccess;
    k_force_jvp<<<nblk(nb), 256, 0, st>>>(nb, q, gF, pid, adj_start, adj_j, adj_rest, k_spring,
                                          k_rep, r_cut, cell_start, sorted, blob_cell, g, bg, out,
                                          gk);
    return cudaGetLastError();
}

cudaError_t launch_axpby(cudaStream_t st, int64_t n, double a, const double* x, double b,
                         const double* y, double* out)
{
    if (n <= 0) return cudaSuccess;
    k_axpby<<<nblk(n), 256, 0, st>>>(n, a, x, b, y, out);
    return cudaGetLastError();
}

}  // namespace mbk
