// Blob-side kernels: interpolation J, cell binning, blob forces, tiled spreading S,
// particle velocities.
#include "mb_internal.cuh"
#include "peskin.cuh"

namespace mbk {

// ==========================================================================================
// Interpolation J (Eq. ju): u_a = sum over the 3x3x3 window of Phi Phi Phi v_a(node).
// One thread per blob; each component reads its own staggered grid.
template <typename R, int MODE>
__global__ void __launch_bounds__(256)
k_interp(int64_t nb, const double* __restrict__ q, const double* q_base,
         const R* __restrict__ v0, const R* __restrict__ v1, const int32_t* __restrict__ box_of,
         GridGeo g, double dt, double* __restrict__ u_out, double* q_out)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int box = box_of ? box_of[b] : 0;
    const double p[3] = {q[3 * b], q[3 * b + 1], q[3 * b + 2]};
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    double u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R wx[3], wy[3], wz[3];
        const int ix = peskin_window<R>(p[0] * g.inv_h - mac_shift(a, 0), wx);
        const int iy = peskin_window<R>(p[1] * g.inv_h - mac_shift(a, 1), wy);
        const int iz = peskin_window<R>(p[2] * g.inv_h - mac_shift(a, 2), wz);
        const size_t base = ((size_t)box * 3 + a) * (size_t)g.N;
        const R* c0 = v0 + base;
        const R* c1 = MODE == 2 ? v1 + base : nullptr;
        // 32-bit offsets inside the component grid (at most 2^24 nodes), the wrapped node
        // indices computed once per dimension
        int xo[3], yo[3], zo[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xo[d] = (ix + d) & (nx - 1);
            yo[d] = ((iy + d) & (ny - 1)) * nx;
            zo[d] = ((iz + d) & (nz - 1)) * (ny * nx);
        }
        R acc = R(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
                const int row = zo[c] + yo[bb];
                R r = R(0);
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    R val = __ldg(c0 + (row + xo[aa]));
                    if (MODE == 2) val += __ldg(c1 + (row + xo[aa]));
                    r += wx[aa] * val;
                }
                acc += wy[bb] * wz[c] * r;
            }
        }
        u[a] = MODE == 2 ? 0.5 * (double)acc : (double)acc;
    }
    // position updates round like the plain expression q + (c dt) u (no contraction)
    if (MODE == 0) {
        for (int a = 0; a < 3; ++a) u_out[3 * b + a] = u[a];
    } else if (MODE == 1) {
        for (int a = 0; a < 3; ++a) {
            if (u_out) u_out[3 * b + a] = u[a];
            q_out[3 * b + a] = wrap_position(__dadd_rn(p[a], __dmul_rn(0.5 * dt, u[a])), g.L[a]);
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            const double qb = q_base[3 * b + a];
            if (u_out) u_out[3 * b + a] = u[a];
            q_out[3 * b + a] = wrap_position(__dadd_rn(qb, __dmul_rn(dt, u[a])), g.L[a]);
        }
    }
}

template <typename R>
cudaError_t launch_interp(cudaStream_t st, int mode, int64_t nb, const double* q,
                          const double* q_base, const R* v0, const R* v1,
                          const int32_t* box_of, const GridGeo& g, double dt, double* u_out,
                          double* q_out)
{
    if (nb <= 0) return cudaSuccess;
    const int T = 256;
    const unsigned blocks = (unsigned)((nb + T - 1) / T);
    if (mode == 0)
        k_interp<R, 0><<<blocks, T, 0, st>>>(nb, q, q_base, v0, v1, box_of, g, dt, u_out, q_out);
    else if (mode == 1)
        k_interp<R, 1><<<blocks, T, 0, st>>>(nb, q, q_base, v0, v1, box_of, g, dt, u_out, q_out);
    else
        k_interp<R, 2><<<blocks, T, 0, st>>>(nb, q, q_base, v0, v1, box_of, g, dt, u_out, q_out);
    return cudaGetLastError();
}
template cudaError_t launch_interp<float>(cudaStream_t, int, int64_t, const double*,
                                          const double*, const float*, const float*,
                                          const int32_t*, const GridGeo&, double, double*,
                                          double*);
template cudaError_t launch_interp<double>(cudaStream_t, int, int64_t, const double*,
                                           const double*, const double*, const double*,
                                           const int32_t*, const GridGeo&, double, double*,
                                           double*);

// ==========================================================================================
// Cell binning (counting sort of blobs by bin cell, box-major).

__device__ __forceinline__ int bin_coord(double x, double inv_w, int nc)
{
    int c = (int)floor(x * inv_w);
    if (c >= nc) c -= nc;
    if (c < 0) c += nc;
    if (c < 0 || c >= nc) c = 0;   // non-finite position: keep every index in bounds
    return c;
}

__global__ void k_bin_count(int64_t nb, const double* __restrict__ q,
                            const int32_t* __restrict__ box_of, BinGeo bg,
                            int32_t* __restrict__ count, int32_t* __restrict__ blob_cell,
                            int32_t* __restrict__ blob_rank)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int box = box_of ? box_of[b] : 0;
    const int cx = bin_coord(q[3 * b], bg.inv_w, bg.nc[0]);
    const int cy = bin_coord(q[3 * b + 1], bg.inv_w, bg.nc[1]);
    const int cz = bin_coord(q[3 * b + 2], bg.inv_w, bg.nc[2]);
    const int cell = (int)(box * bg.ncell + ((int64_t)cz * bg.nc[1] + cy) * bg.nc[0] + cx);
    blob_cell[b] = cell;
    blob_rank[b] = atomicAdd(count + cell, 1);
}

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_TILE = 4 * SCAN_THREADS;

// Exclusive scan of one tile of 4096 ints; writes the tile total to tile_sums.
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
            int32_t* __restrict__ tile_sums)
{
    __shared__ int32_t warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    int32_t v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = base + i < n ? in[base + i] : 0;
    const int32_t s = v[0] + v[1] + v[2] + v[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    int32_t run = x - s + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = run;
}

// Exclusive scan of the tile totals (one block, sequential chunks); total goes to *total.
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_tops(int32_t* __restrict__ tile_sums, int ntiles, int32_t* __restrict__ total)
{
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < ntiles; c0 += SCAN_THREADS) {
        const int i = c0 + threadIdx.x;
        const int32_t s = i < ntiles ? tile_sums[i] : 0;
        int32_t x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int32_t excl = carry + x - s + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (i < ntiles) tile_sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = excl + s;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n,
                           const int32_t* __restrict__ tile_offsets)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_offsets[i / SCAN_TILE];
}

// Scatter into sorted order; optionally record each blob's position relative to the lower
// corner of its bin cell (FP32, |x| < cell side) and its particle id, for the FP32 prefilter of
// the pair search.
__global__ void k_bin_scatter(int64_t nb, const int32_t* __restrict__ blob_cell,
                              const int32_t* __restrict__ blob_rank,
                              const int32_t* __restrict__ cell_start, int32_t* __restrict__ sorted,
                              const double* __restrict__ q, const int32_t* __restrict__ pid,
                              BinGeo bg, float4* __restrict__ loc)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int cell = blob_cell[b];
    const int slot = cell_start[cell] + blob_rank[b];
    sorted[slot] = (int32_t)b;
    if (loc) {
        const int local = (int)(cell % bg.ncell);
        const int c[3] = {local % bg.nc[0], (local / bg.nc[0]) % bg.nc[1],
                          local / (bg.nc[0] * bg.nc[1])};
        const double w = bg.w;   // cell side
        float r[3];
        for (int d = 0; d < 3; ++d) r[d] = (float)(q[3 * b + d] - c[d] * w);
        loc[slot] = make_float4(r[0], r[1], r[2], __int_as_float(pid ? pid[b] : 0));
    }
}

// Deterministic order inside each cell: ascending blob index (cells hold a handful of blobs).
__global__ void k_cell_order(int64_t ncells, const int32_t* __restrict__ cell_start,
                             int32_t* __restrict__ sorted)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int s = cell_start[c], e = cell_start[c + 1];
    for (int i = s + 1; i < e; ++i) {
        const int32_t key = sorted[i];
        int j = i - 1;
        while (j >= s && sorted[j] > key) {
            sorted[j + 1] = sorted[j];
            --j;
        }
        sorted[j + 1] = key;
    }
}

// Cell-local coordinates in the final (reordered) slot order.
__global__ void k_fill_loc(int64_t nb, const int32_t* __restrict__ sorted,
                           const int32_t* __restrict__ blob_cell, const double* __restrict__ q,
                           const int32_t* __restrict__ pid, BinGeo bg, float4* __restrict__ loc)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const int b = sorted[t];
    const int local = (int)(blob_cell[b] % bg.ncell);
    const int c[3] = {local % bg.nc[0], (local / bg.nc[0]) % bg.nc[1],
                      local / (bg.nc[0] * bg.nc[1])};
    const double w = bg.w;
    float r[3];
    for (int d = 0; d < 3; ++d) r[d] = (float)(q[3 * b + d] - c[d] * w);
    loc[t] = make_float4(r[0], r[1], r[2], __int_as_float(pid ? pid[b] : 0));
}

cudaError_t launch_exclusive_scan(cudaStream_t st, const int32_t* in, int32_t* out, int64_t n,
                                  int32_t* tile_tmp)
{
    const int T = 256;
    const int ntiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_tile<<<ntiles, SCAN_THREADS, 0, st>>>(in, out, n, tile_tmp);
    k_scan_tops<<<1, SCAN_THREADS, 0, st>>>(tile_tmp, ntiles, out + n);
    k_scan_add<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(out, n, tile_tmp);
    return cudaGetLastError();
}

cudaError_t launch_bin(cudaStream_t st, int64_t nb, const double* q, const int32_t* box_of,
                       int B, const BinGeo& bg, int32_t* cell_count, int32_t* cell_start,
                       int32_t* blob_cell, int32_t* blob_rank, int32_t* sorted,
                       int32_t* scan_tmp, bool deterministic, const int32_t* pid, float4* loc)
{
    const int64_t ncells = (int64_t)B * bg.ncell;
    cudaError_t e = cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * ncells, st);
    if (e != cudaSuccess) return e;
    const int T = 256;
    if (nb > 0)
        k_bin_count<<<(unsigned)((nb + T - 1) / T), T, 0, st>>>(nb, q, box_of, bg, cell_count,
                                                                blob_cell, blob_rank);
    const int ntiles = (int)((ncells + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_tile<<<ntiles, SCAN_THREADS, 0, st>>>(cell_count, cell_start, ncells, scan_tmp);
    k_scan_tops<<<1, SCAN_THREADS, 0, st>>>(scan_tmp, ntiles, cell_start + ncells);
    k_scan_add<<<(unsigned)((ncells + T - 1) / T), T, 0, st>>>(cell_start, ncells, scan_tmp);
    if (nb > 0)
        k_bin_scatter<<<(unsigned)((nb + T - 1) / T), T, 0, st>>>(nb, blob_cell, blob_rank,
                                                                  cell_start, sorted, q, pid, bg,
                                                                  deterministic ? nullptr : loc);
    if (deterministic) {
        k_cell_order<<<(unsigned)((ncells + T - 1) / T), T, 0, st>>>(ncells, cell_start, sorted);
        if (loc && nb > 0)
            k_fill_loc<<<(unsigned)((nb + T - 1) / T), T, 0, st>>>(nb, sorted, blob_cell, q, pid,
                                                                   bg, loc);
    }
    return cudaGetLastError();
}

// ==========================================================================================
// Blob forces (FP64): harmonic bonds from a per-blob adjacency list, soft repulsion between
// blobs of different particles found through the bin cells, external forces.
// One thread per sorted slot; the grid is (chunks, boxes) so block partial sums stay per box.

__device__ __forceinline__ void block_sum3(double v[3], double* sh /*[3][32]*/)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = v[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[a * 32 + warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double x = lane < nw ? sh[a * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) v[a] = x;
        }
    }
}

// Spring force on blob b from bond (b, j): -k (|r| - r0) r/|r|, r = q_b - q_j (minimum image).
// PRECISE: FP64 with the operations in the plain order and no contraction, so that a blob's
// spring force is the same bits however the work is scheduled.  Otherwise: r, |r|^2 and
// |r|^2 - r0^2 in FP64 (the only cancellation), the rest in FP32, accumulated in FP64.
template <bool PRECISE>
__device__ __forceinline__ void spring_term(const double qb[3], const double* __restrict__ qj,
                                            double r0, double k, const double L[3],
                                            const double halfL[3], double F[3])
{
    double r[3];
    for (int d = 0; d < 3; ++d) {
        double x = __dsub_rn(qb[d], qj[d]);
        if (x > halfL[d]) x = __dsub_rn(x, L[d]);
        else if (x < -halfL[d]) x = __dadd_rn(x, L[d]);
        r[d] = x;
    }
    if (PRECISE) {
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])),
                                    __dmul_rn(r[2], r[2]));
        const double len = __dsqrt_rn(r2);
        const double mag = __ddiv_rn(__dmul_rn(-k, __dsub_rn(len, r0)), len);
        for (int d = 0; d < 3; ++d) F[d] = __dadd_rn(F[d], __dmul_rn(mag, r[d]));
    } else {
        const double r2 = fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2]));
        const float d2 = (float)(r2 - r0 * r0);               // |r|^2 - r0^2
        const float len = sqrtf((float)r2);
        const float mag = -(float)k * d2 / ((len + (float)r0) * len);
        for (int d = 0; d < 3; ++d) F[d] += (double)(mag * (float)r[d]);
    }
}

// Repulsion k_rep (r_cut - |r|) r/|r| for |r| < r_cut, r = q_b - q_j.
template <bool PRECISE>
__device__ __forceinline__ void pair_term(const double qb[3], const double* __restrict__ qj,
                                          const float rf[3], double k_rep, double r_cut,
                                          const double L[3], double Fp[3])
{
    if (PRECISE) {
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = min_image(__dsub_rn(qb[d], qj[d]), L[d]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])),
                                    __dmul_rn(r[2], r[2]));
        if (r2 >= r_cut * r_cut || r2 == 0.0) return;
        const double len = __dsqrt_rn(r2);
        const double mag = __ddiv_rn(__dmul_rn(k_rep, __dsub_rn(r_cut, len)), len);
        for (int d = 0; d < 3; ++d) Fp[d] = __dadd_rn(Fp[d], __dmul_rn(mag, r[d]));
    } else {
        const float r2 = rf[0] * rf[0] + rf[1] * rf[1] + rf[2] * rf[2];
        const float rc = (float)r_cut;
        if (r2 >= rc * rc || r2 == 0.0f) return;
        const float len = sqrtf(r2);
        const float mag = (float)k_rep * (rc - len) / len;
        for (int d = 0; d < 3; ++d) Fp[d] += (double)(mag * rf[d]);
    }
}

// FP64 springs of a bond pattern shared by all particles (launch_springs64).  A block holds
// whole particles (one thread per blob, blob order).  Each thread evaluates the bonds its
// evaluation list names (spring_term<true> on a zero sum: the force on its own blob) into its
// shared-memory slots; after a barrier it sums ext and, in its adjacency order, its own slots
// and the negated slots of the bonds its partners evaluated.  Negation is exact and the
// evaluation of a bond from the other end gives the negated bits, so every sum equals the
// per-blob adjacency sum of k_forces bit for bit.
__global__ void __launch_bounds__(256)
k_springs64(int nb, int m, int S, const double* __restrict__ q, const double* __restrict__ ext,
            const int4* __restrict__ tmpl, const int32_t* __restrict__ tstart,
            const int32_t* __restrict__ box_of, const double* __restrict__ box_par, GridGeo g,
            double* __restrict__ Fout)
{
    extern __shared__ double slot_d[];                   // [blockDim][S][3]
    const int tid = threadIdx.x;
    const int b = blockIdx.x * blockDim.x + tid;
    const bool live = b < nb;
    const int l = tid % m;
    if (live) {
        const double qb[3] = {q[3 * b], q[3 * b + 1], q[3 * b + 2]};
        const double halfL[3] = {0.5 * g.L[0], 0.5 * g.L[1], 0.5 * g.L[2]};
        const double k_spring = box_par[3 * (box_of ? box_of[b] : 0)];
        const int e0 = __ldg(tstart + 2 * l), e1 = __ldg(tstart + 2 * l + 1);
        for (int e = e0; e < e1; ++e) {
            const int4 ad = __ldg(tmpl + e);
            const int j = b + (int)(short)(ad.x & 0xffff);
            const int slot = (ad.x >> 16) - 1;
            const double r0 = __hiloint2double(ad.z, ad.y);
            double f[3] = {0.0, 0.0, 0.0};
            spring_term<true>(qb, q + 3 * j, r0, k_spring, g.L, halfL, f);
            for (int d = 0; d < 3; ++d) slot_d[(tid * S + slot) * 3 + d] = f[d];
        }
    }
    __syncthreads();
    if (!live) return;
    double F[3] = {0.0, 0.0, 0.0};
    if (ext)
        for (int d = 0; d < 3; ++d) F[d] = ext[3 * b + d];
    const int c0 = __ldg(tstart + 2 * l + 1), c1 = __ldg(tstart + 2 * l + 2);
    for (int e = c0; e < c1; ++e) {
        const int4 ad = __ldg(tmpl + e);
        const double* v = slot_d + ((tid + ad.x) * S + ad.y) * 3;
        for (int d = 0; d < 3; ++d) F[d] = __dadd_rn(F[d], ad.z > 0 ? v[d] : -v[d]);
    }
    for (int d = 0; d < 3; ++d) Fout[3 * b + d] = F[d];
}

cudaError_t launch_springs64(cudaStream_t st, int64_t nb, int m, int slots, const double* q,
                             const double* ext, const int4* tmpl, const int32_t* tstart,
                             const int32_t* box_of, const double* box_par, const GridGeo& g,
                             double* Fout)
{
    if (nb <= 0) return cudaSuccess;
    const int threads = (256 / m) * m;                   // whole particles per block
    const size_t smem = sizeof(double) * 3 * (size_t)threads * (slots > 0 ? slots : 1);
    k_springs64<<<(unsigned)((nb + threads - 1) / threads), threads, smem, st>>>(
        (int)nb, m, slots, q, ext, tmpl, tstart, box_of, box_par, g, Fout);
    return cudaGetLastError();
}

template <bool PRECISE>
__global__ void __launch_bounds__(256)
k_forces(ForceArgs a, GridGeo g, BinGeo bg)
{
    __shared__ double sh[96];
    const int box = blockIdx.y;
    const int64_t s0 = a.box_off[box], cnt = a.box_off[box + 1] - s0;
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double F[3] = {0.0, 0.0, 0.0};
    if (local < cnt) {
        const int64_t slot = s0 + local;
        const int b = a.sorted[slot];
        const double qb[3] = {a.q[3 * b], a.q[3 * b + 1], a.q[3 * b + 2]};
        const double halfL[3] = {0.5 * g.L[0], 0.5 * g.L[1], 0.5 * g.L[2]};
        const double k_rep = a.box_par[3 * box + 1];
        const double r_cut = a.box_par[3 * box + 2];
        if (a.Fpre) {
            for (int d = 0; d < 3; ++d) F[d] = a.Fpre[3 * b + d];
        } else {
            if (a.ext) {
                F[0] = a.ext[3 * b];
                F[1] = a.ext[3 * b + 1];
                F[2] = a.ext[3 * b + 2];
            }
            const double k_spring = a.box_par[3 * box];
            for (int e = a.adj_start[b]; e < a.adj_start[b + 1]; ++e)
                spring_term<PRECISE>(qb, a.q + 3 * a.adj_j[e], a.adj_rest[e], k_spring, g.L,
                                     halfL, F);
        }
        if (k_rep != 0.0 && r_cut > 0.0) {
            double Fp[3] = {0.0, 0.0, 0.0};
            const float4 lb = a.loc[slot];
            const int pb = __float_as_int(lb.w);
            const int cell = a.blob_cell[b] - (int)(box * bg.ncell);
            const int c[3] = {cell % bg.nc[0], (cell / bg.nc[0]) % bg.nc[1],
                              cell / (bg.nc[0] * bg.nc[1])};
            const float w = bg.w32;
            const float rcf = (float)r_cut;
            const float pre = rcf * rcf * 1.0001f + 1e-6f;     // conservative FP32 prefilter
            const bool wide = bg.nc[0] >= 3 && bg.nc[1] >= 3 && bg.nc[2] >= 3;
            int lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                if (bg.nc[d] >= 3) { lo[d] = -1; hi[d] = 1; }
                else { lo[d] = 0; hi[d] = bg.nc[d] - 1; }
            }
            for (int dz = lo[2]; dz <= hi[2]; ++dz) {
                const int cz = bg.nc[2] >= 3 ? (c[2] + dz + bg.nc[2]) % bg.nc[2] : dz;
                for (int dy = lo[1]; dy <= hi[1]; ++dy) {
                    const int cy = bg.nc[1] >= 3 ? (c[1] + dy + bg.nc[1]) % bg.nc[1] : dy;
                    for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                        const int cx = bg.nc[0] >= 3 ? (c[0] + dx + bg.nc[0]) % bg.nc[0] : dx;
                        const int64_t cc = box * bg.ncell + ((int64_t)cz * bg.nc[1] + cy) * bg.nc[0] + cx;
                        const float ox = dx * w, oy = dy * w, oz = dz * w;
                        for (int t = a.cell_start[cc]; t < a.cell_start[cc + 1]; ++t) {
                            if (t == slot) continue;
                            const float4 lj = a.loc[t];
                            if (__float_as_int(lj.w) == pb) continue;
                            float rf[3] = {lb.x - lj.x - ox, lb.y - lj.y - oy, lb.z - lj.z - oz};
                            if (wide && rf[0] * rf[0] + rf[1] * rf[1] + rf[2] * rf[2] > pre) continue;
                            const int j = a.sorted[t];
                            if (!PRECISE && !wide) {
                                for (int d = 0; d < 3; ++d)
                                    rf[d] = (float)min_image(qb[d] - a.q[3 * j + d], g.L[d]);
                            }
                            pair_term<PRECISE>(qb, a.q + 3 * j, rf, k_rep, r_cut, g.L, Fp);
                        }
                    }
                }
            }
            for (int d = 0; d < 3; ++d) F[d] = __dadd_rn(F[d], Fp[d]);
        }
        for (int d = 0; d < 3; ++d) {
            a.F[3 * b + d] = F[d];
            a.rec[6 * slot + d] = qb[d];
            a.rec[6 * slot + 3 + d] = F[d];
        }
    }
    block_sum3(F, sh);
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d)
            a.partial[((int64_t)box * a.nchunk + blockIdx.x) * 3 + d] = F[d];
}

cudaError_t launch_forces(cudaStream_t st, int B, int64_t max_box_blobs, const ForceArgs& a,
                          const GridGeo& g, const BinGeo& bg, bool precise)
{
    if (a.nchunk <= 0) return cudaSuccess;
    dim3 grid((unsigned)a.nchunk, (unsigned)B);
    (void)max_box_blobs;
    if (precise) k_forces<true><<<grid, 256, 0, st>>>(a, g, bg);
    else k_forces<false><<<grid, 256, 0, st>>>(a, g, bg);
    return cudaGetLastError();
}

// Per-box force sums in a fixed order, then the FP64 mean-velocity update.
__global__ void __launch_bounds__(256)
k_force_sum(int nchunk, const double* __restrict__ partial, double* __restrict__ vbar,
            double scale, int mean_mode, double* __restrict__ fsum_out)
{
    __shared__ double sh[3][256];
    const int box = blockIdx.x;
    double s[3] = {0.0, 0.0, 0.0};
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x)
        for (int d = 0; d < 3; ++d) s[d] += partial[((int64_t)box * nchunk + c) * 3 + d];
    for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        const double tot = sh[d][0];
        if (fsum_out) fsum_out[3 * box + d] = tot;
        if (vbar) vbar[3 * box + d] = mean_mode == 0 ? vbar[3 * box + d] + scale * tot : 0.0;
    }
}

cudaError_t launch_force_sum(cudaStream_t st, int B, int nchunk, const double* partial,
                             double* vbar, double scale, int mean_mode, double* fsum_out)
{
    if (nchunk <= 0) {
        // no blobs anywhere: the net force is zero
        return cudaSuccess;
    }
    k_force_sum<<<B, 256, 0, st>>>(nchunk, partial, vbar, scale, mean_mode, fsum_out);
    return cudaGetLastError();
}

__global__ void k_make_rec(int64_t nb, const int32_t* __restrict__ sorted,
                           const double* __restrict__ q, const double* __restrict__ F,
                           double* __restrict__ rec)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nb) return;
    const int b = sorted[s];
    for (int d = 0; d < 3; ++d) {
        rec[6 * s + d] = q[3 * b + d];
        rec[6 * s + 3 + d] = F[3 * b + d];
    }
}

cudaError_t launch_make_rec(cudaStream_t st, int64_t nb, const int32_t* sorted, const double* q,
                            const double* F, double* rec)
{
    if (nb <= 0) return cudaSuccess;
    k_make_rec<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(nb, sorted, q, F, rec);
    return cudaGetLastError();
}

// ==========================================================================================
// Spreading S as tile-owner accumulation: each CTA owns a TX x TY x TZ block of nodes of all
// three components, gathers every blob whose 3x3x3 window can reach it from the bin cells of
// the block plus its halo, accumulates the in-block part of f = sum delta_h F in shared
// memory, and writes the block once.  No global atomics; every node is written by exactly one
// CTA.

__host__ __device__ __forceinline__ int floor_div(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

__host__ __device__ __forceinline__ int wrap_cell(int c, int n)
{
    c %= n;
    return c < 0 ? c + n : c;
}

// Bin-cell window [lo, lo + cnt) along one dimension holding every blob that can touch nodes
// [T0, T0 + T): blob positions q/h in [T0 - 3/2, T0 + T + 1) (union of both MAC shifts).
__host__ __device__ __forceinline__ void halo_cells(int T0, int T, int bs, int nc, int& lo,
                                                    int& cnt)
{
    lo = floor_div(2 * T0 - 3, 2 * bs);
    const int hi = floor_div(T0 + T + 1 + bs - 1, bs) - 1;
    cnt = hi - lo + 1;
    if (cnt >= nc) {
        lo = 0;
        cnt = nc;
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_spread(const double* __restrict__ rec, const int32_t* __restrict__ cell_start, GridGeo g,
         BinGeo bg, int TX, int TY, int TZ, int max_ranges, R* __restrict__ f)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tileN = TX * TY * TZ;
    R* acc = reinterpret_cast<R*>(smem_raw);
    int32_t* rbeg = reinterpret_cast<int32_t*>(acc + 3 * tileN);
    int32_t* rpre = rbeg + max_ranges;    // max_ranges + 1 entries
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int box = blockIdx.y;
    const int ntx = nx / TX, nty = ny / TY;
    const int tid = blockIdx.x;
    const int T0[3] = {(tid % ntx) * TX, ((tid / ntx) % nty) * TY, (tid / (ntx * nty)) * TZ};
    const int T[3] = {TX, TY, TZ};

    for (int i = threadIdx.x; i < 3 * tileN; i += blockDim.x) acc[i] = R(0);
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) halo_cells(T0[d], T[d], bg.bs, bg.nc[d], lo[d], cnt[d]);
    const int rows = cnt[1] * cnt[2];
    const int nr = 2 * rows;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int cz = wrap_cell(lo[2] + r / cnt[1], bg.nc[2]);
        const int cy = wrap_cell(lo[1] + r % cnt[1], bg.nc[1]);
        const int64_t rowbase = box * bg.ncell + ((int64_t)cz * bg.nc[1] + cy) * bg.nc[0];
        const int sx = wrap_cell(lo[0], bg.nc[0]);
        const int ex = sx + cnt[0];
        const int a1 = ex <= bg.nc[0] ? ex : bg.nc[0];
        const int s0 = cell_start[rowbase + sx];
        rbeg[2 * r] = s0;
        rpre[2 * r] = cell_start[rowbase + a1] - s0;          // length, prefix-summed below
        if (ex > bg.nc[0]) {
            const int t0 = cell_start[rowbase];
            rbeg[2 * r + 1] = t0;
            rpre[2 * r + 1] = cell_start[rowbase + (ex - bg.nc[0])] - t0;
        } else {
            rbeg[2 * r + 1] = 0;
            rpre[2 * r + 1] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {       // exclusive prefix of the lengths (one warp)
        const int lane = threadIdx.x;
        int carry = 0;
        for (int c0 = 0; c0 < nr; c0 += 32) {
            const int i = c0 + lane;
            const int len = i < nr ? rpre[i] : 0;
            int x = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (i < nr) rpre[i] = carry + x - len;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) rpre[nr] = carry;
    }
    __syncthreads();
    const int total = rpre[nr];
    const double inv_h3 = g.inv_h * g.inv_h * g.inv_h;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int lo_r = 0, hi_r = nr - 1;
        while (lo_r < hi_r) {
            const int mid = (lo_r + hi_r + 1) >> 1;
            if (rpre[mid] <= t) lo_r = mid; else hi_r = mid - 1;
        }
        const int64_t slot = rbeg[lo_r] + (t - rpre[lo_r]);
        const double* rr = rec + 6 * slot;
        const double p[3] = {rr[0], rr[1], rr[2]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R Fa = static_cast<R>(rr[3 + a] * inv_h3);
            R wx[3], wy[3], wz[3];
            const int ix = peskin_window<R>(p[0] * g.inv_h - mac_shift(a, 0), wx) - T0[0];
            const int iy = peskin_window<R>(p[1] * g.inv_h - mac_shift(a, 1), wy) - T0[1];
            const int iz = peskin_window<R>(p[2] * g.inv_h - mac_shift(a, 2), wz) - T0[2];
            R* acc_a = acc + a * tileN;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int rz = (iz + c) & (nz - 1);
                if (rz >= TZ) continue;
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) {
                    const int ry = (iy + bb) & (ny - 1);
                    if (ry >= TY) continue;
                    const R wyz = wy[bb] * wz[c] * Fa;
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) {
                        const int rx = (ix + aa) & (nx - 1);
                        if (rx < TX) atomicAdd(acc_a + (rz * TY + ry) * TX + rx, wx[aa] * wyz);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * tileN; i += blockDim.x) {
        const int a = i / tileN, rem = i - a * tileN;
        const int rz = rem / (TY * TX), ry = (rem / TX) % TY, rx = rem % TX;
        f[((size_t)box * 3 + a) * (size_t)g.N +
          ((size_t)(T0[2] + rz) * ny + (T0[1] + ry)) * nx + (T0[0] + rx)] = acc[i];
    }
}

// Blob-owner spreading with global atomics: one thread per sorted slot adds its 81 node
// contributions straight into f (zeroed beforehand) with the native FP64 (or FP32) global
// atomic add; the sorted order keeps a warp's nodes close together in L2.
template <typename R>
__global__ void __launch_bounds__(256)
k_spread_atomic(const double* __restrict__ rec, const int32_t* __restrict__ cell_start,
                GridGeo g, BinGeo bg, R* __restrict__ f)
{
    const int box = blockIdx.y;
    const int64_t s0 = cell_start[box * bg.ncell], s1 = cell_start[(box + 1) * bg.ncell];
    const int64_t slot = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s1) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const double* rr = rec + 6 * slot;
    const double p[3] = {rr[0], rr[1], rr[2]};
    const double inv_h3 = g.inv_h * g.inv_h * g.inv_h;
    R* fb = f + (size_t)box * 3 * (size_t)g.N;
    const int N32 = (int)g.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R Fa = static_cast<R>(rr[3 + a] * inv_h3);
        R wx[3], wy[3], wz[3];
        const int ix = peskin_window<R>(p[0] * g.inv_h - mac_shift(a, 0), wx);
        const int iy = peskin_window<R>(p[1] * g.inv_h - mac_shift(a, 1), wy);
        const int iz = peskin_window<R>(p[2] * g.inv_h - mac_shift(a, 2), wz);
        int xo[3], yo[3], zo[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xo[d] = (ix + d) & (nx - 1);
            yo[d] = ((iy + d) & (ny - 1)) * nx;
            zo[d] = ((iz + d) & (nz - 1)) * (ny * nx);
        }
        R* fa = fb + a * N32;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
                const R wyz = wy[bb] * wz[c] * Fa;
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) atomicAdd(fa + (zo[c] + yo[bb] + xo[aa]), wx[aa] * wyz);
            }
    }
}

template <typename R>
cudaError_t launch_spread_atomic(cudaStream_t st, int B, int64_t max_box_blobs, const double* rec,
                                 const int32_t* cell_start, const GridGeo& g, const BinGeo& bg,
                                 R* f)
{
    cudaError_t e = cudaMemsetAsync(f, 0, sizeof(R) * 3 * (size_t)B * g.N, st);
    if (e != cudaSuccess || max_box_blobs <= 0) return e;
    dim3 grid((unsigned)((max_box_blobs + 255) / 256), (unsigned)B);
    k_spread_atomic<R><<<grid, 256, 0, st>>>(rec, cell_start, g, bg, f);
    return cudaGetLastError();
}
template cudaError_t launch_spread_atomic<double>(cudaStream_t, int, int64_t, const double*,
                                                  const int32_t*, const GridGeo&, const BinGeo&,
                                                  double*);
template cudaError_t launch_spread_atomic<float>(cudaStream_t, int, int64_t, const double*,
                                                 const int32_t*, const GridGeo&, const BinGeo&,
                                                 float*);

// Deterministic FP64 spreading: the same tile-owner scheme, accumulated in 64-bit fixed point
// (shared-memory integer atomics are associative, so the sums do not depend on the order in
// which threads add).  The tile's scale is a power of two chosen from its largest force so that
// no node can overflow: 2^62 over (candidates x max weight product x max |F| / h^3).
__global__ void __launch_bounds__(256)
k_spread_det(const double* __restrict__ rec, const int32_t* __restrict__ cell_start, GridGeo g,
             BinGeo bg, int TX, int TY, int TZ, int max_ranges, double* __restrict__ f)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tileN = TX * TY * TZ;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw);
    int32_t* rbeg = reinterpret_cast<int32_t*>(acc + 3 * tileN);
    int32_t* rpre = rbeg + max_ranges;
    __shared__ double fmax_sh[32];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int box = blockIdx.y;
    const int ntx = nx / TX, nty = ny / TY;
    const int tid = blockIdx.x;
    const int T0[3] = {(tid % ntx) * TX, ((tid / ntx) % nty) * TY, (tid / (ntx * nty)) * TZ};
    const int T[3] = {TX, TY, TZ};
    for (int i = threadIdx.x; i < 3 * tileN; i += blockDim.x) acc[i] = 0ull;
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) halo_cells(T0[d], T[d], bg.bs, bg.nc[d], lo[d], cnt[d]);
    const int rows = cnt[1] * cnt[2];
    const int nr = 2 * rows;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int cz = wrap_cell(lo[2] + r / cnt[1], bg.nc[2]);
        const int cy = wrap_cell(lo[1] + r % cnt[1], bg.nc[1]);
        const int64_t rowbase = box * bg.ncell + ((int64_t)cz * bg.nc[1] + cy) * bg.nc[0];
        const int sx = wrap_cell(lo[0], bg.nc[0]);
        const int ex = sx + cnt[0];
        const int a1 = ex <= bg.nc[0] ? ex : bg.nc[0];
        const int s0 = cell_start[rowbase + sx];
        rbeg[2 * r] = s0;
        rpre[2 * r] = cell_start[rowbase + a1] - s0;
        if (ex > bg.nc[0]) {
            const int t0 = cell_start[rowbase];
            rbeg[2 * r + 1] = t0;
            rpre[2 * r + 1] = cell_start[rowbase + (ex - bg.nc[0])] - t0;
        } else {
            rbeg[2 * r + 1] = 0;
            rpre[2 * r + 1] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < nr; ++i) {
            const int len = rpre[i];
            rpre[i] = run;
            run += len;
        }
        rpre[nr] = run;
    }
    __syncthreads();
    const int total = rpre[nr];
    auto slot_of = [&](int t) {
        int a = 0, b = nr - 1;
        while (a < b) {
            const int m = (a + b + 1) >> 1;
            if (rpre[m] <= t) a = m; else b = m - 1;
        }
        return (int64_t)rbeg[a] + (t - rpre[a]);
    };
    // tile scale from the largest force component among the candidates
    double fm = 0.0;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const double* rr = rec + 6 * slot_of(t);
        fm = fmax(fm, fmax(fabs(rr[3]), fmax(fabs(rr[4]), fabs(rr[5]))));
    }
    for (int o = 16; o > 0; o >>= 1) fm = fmax(fm, __shfl_down_sync(0xffffffffu, fm, o));
    if ((threadIdx.x & 31) == 0) fmax_sh[threadIdx.x >> 5] = fm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, fmax_sh[w]);
        fmax_sh[0] = m;
    }
    __syncthreads();
    const double inv_h3 = g.inv_h * g.inv_h * g.inv_h;
    const double bound = fmax(fmax_sh[0] * inv_h3 * (8.0 / 27.0) * (double)(total + 1), 1e-300);
    int ex2;
    frexp(bound, &ex2);                      // bound < 2^ex2
    const double scale = ldexp(1.0, 62 - max(ex2, -900));   // finite even for a zero tile
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const double* rr = rec + 6 * slot_of(t);
        const double p[3] = {rr[0], rr[1], rr[2]};
        for (int a = 0; a < 3; ++a) {
            const double Fa = rr[3 + a] * inv_h3;
            double wx[3], wy[3], wz[3];
            const int ix = peskin_window<double>(p[0] * g.inv_h - mac_shift(a, 0), wx) - T0[0];
            const int iy = peskin_window<double>(p[1] * g.inv_h - mac_shift(a, 1), wy) - T0[1];
            const int iz = peskin_window<double>(p[2] * g.inv_h - mac_shift(a, 2), wz) - T0[2];
            unsigned long long* acc_a = acc + a * tileN;
            for (int c = 0; c < 3; ++c) {
                const int rz = (iz + c) & (nz - 1);
                if (rz >= TZ) continue;
                for (int bb = 0; bb < 3; ++bb) {
                    const int ry = (iy + bb) & (ny - 1);
                    if (ry >= TY) continue;
                    const double wyz = wy[bb] * wz[c] * Fa;
                    for (int aa = 0; aa < 3; ++aa) {
                        const int rx = (ix + aa) & (nx - 1);
                        if (rx < TX) {
                            const long long v = llrint(wx[aa] * wyz * scale);
                            atomicAdd(acc_a + (rz * TY + ry) * TX + rx, (unsigned long long)v);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const double inv_scale = 1.0 / scale;
    for (int i = threadIdx.x; i < 3 * tileN; i += blockDim.x) {
        const int a = i / tileN, rem = i - a * tileN;
        const int rz = rem / (TY * TX), ry = (rem / TX) % TY, rx = rem % TX;
        f[((size_t)box * 3 + a) * (size_t)g.N +
          ((size_t)(T0[2] + rz) * ny + (T0[1] + ry)) * nx + (T0[0] + rx)] =
            (double)(long long)acc[i] * inv_scale;
    }
}

cudaError_t launch_spread_det(cudaStream_t st, int B, const double* rec, const int32_t* cell_start,
                              const GridGeo& g, const BinGeo& bg, const int tile[3], double* f)
{
    const int TX = tile[0], TY = tile[1], TZ = tile[2];
    int max_rows = 1;
    for (int d = 1; d < 3; ++d) {
        int most = 0;
        for (int T0 = 0; T0 < g.n[d]; T0 += tile[d]) {
            int lo, cnt;
            halo_cells(T0, tile[d], bg.bs, bg.nc[d], lo, cnt);
            most = cnt > most ? cnt : most;
        }
        max_rows *= most;
    }
    const int max_ranges = 2 * max_rows;
    const size_t smem = 3 * (size_t)TX * TY * TZ * 8 + sizeof(int32_t) * (2 * max_ranges + 1);
    static std::atomic<unsigned> attr{0};
    if (first_on_device(attr))
        cudaFuncSetAttribute(k_spread_det, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    const int ntiles = (g.n[0] / TX) * (g.n[1] / TY) * (g.n[2] / TZ);
    k_spread_det<<<dim3((unsigned)ntiles, (unsigned)B), 256, smem, st>>>(rec, cell_start, g, bg, TX,
                                                                         TY, TZ, max_ranges, f);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_spread(cudaStream_t st, int B, const double* rec, const int32_t* cell_start,
                          const GridGeo& g, const BinGeo& bg, const int tile[3], R* f)
{
    const int TX = tile[0], TY = tile[1], TZ = tile[2];
    int max_rows = 1;
    for (int d = 1; d < 3; ++d) {
        int most = 0;
        for (int T0 = 0; T0 < g.n[d]; T0 += tile[d]) {
            int lo, cnt;
            halo_cells(T0, tile[d], bg.bs, bg.nc[d], lo, cnt);
            most = cnt > most ? cnt : most;
        }
        max_rows *= most;
    }
    const int max_ranges = 2 * max_rows;
    const size_t smem = 3 * (size_t)TX * TY * TZ * sizeof(R) + sizeof(int32_t) * (2 * max_ranges + 1);
    static std::atomic<unsigned> attr{0};
    if (first_on_device(attr))
        cudaFuncSetAttribute(k_spread<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    const int ntiles = (g.n[0] / TX) * (g.n[1] / TY) * (g.n[2] / TZ);
    dim3 grid((unsigned)ntiles, (unsigned)B);
    k_spread<R><<<grid, 256, smem, st>>>(rec, cell_start, g, bg, TX, TY, TZ, max_ranges, f);
    return cudaGetLastError();
}
template cudaError_t launch_spread<float>(cudaStream_t, int, const double*, const int32_t*,
                                          const GridGeo&, const BinGeo&, const int[3], float*);
template cudaError_t launch_spread<double>(cudaStream_t, int, const double*, const int32_t*,
                                           const GridGeo&, const BinGeo&, const int[3], double*);

// ==========================================================================================
// Particle velocities: U0 = mean blob velocity; Omega from the least-squares rigid rotation,
// I0 Omega = sum s x (u - U0) with I0 = sum (s.s 1 - s s) and s relative to the baricentre.
__global__ void k_particle_reduce(int64_t np, const int32_t* __restrict__ part_start,
                                  const int32_t* __restrict__ part_blobs,
                                  const int32_t* __restrict__ box_of_part,
                                  const double* __restrict__ q, const double* __restrict__ u,
                                  GridGeo g, double* __restrict__ U, double* __restrict__ Omega)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    (void)box_of_part;
    const int s = part_start[p], e = part_start[p + 1];
    double Um[3] = {0, 0, 0}, cm[3] = {0, 0, 0};
    if (e > s) {
        const int b0 = part_blobs[s];
        for (int i = s; i < e; ++i) {
            const int b = part_blobs[i];
            for (int d = 0; d < 3; ++d) {
                Um[d] += u[3 * b + d];
                cm[d] += min_image(q[3 * b + d] - q[3 * b0 + d], g.L[d]);
            }
        }
        const double inv = 1.0 / (double)(e - s);
        for (int d = 0; d < 3; ++d) { Um[d] *= inv; cm[d] *= inv; }
        double I[6] = {0, 0, 0, 0, 0, 0};   // xx, yy, zz, xy, xz, yz
        double tq[3] = {0, 0, 0};
        for (int i = s; i < e; ++i) {
            const int b = part_blobs[i];
            double sv[3], w[3];
            for (int d = 0; d < 3; ++d) {
                sv[d] = min_image(q[3 * b + d] - q[3 * b0 + d], g.L[d]) - cm[d];
                w[d] = u[3 * b + d] - Um[d];
            }
            const double s2 = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
            I[0] += s2 - sv[0] * sv[0];
            I[1] += s2 - sv[1] * sv[1];
            I[2] += s2 - sv[2] * sv[2];
            I[3] -= sv[0] * sv[1];
            I[4] -= sv[0] * sv[2];
            I[5] -= sv[1] * sv[2];
            tq[0] += sv[1] * w[2] - sv[2] * w[1];
            tq[1] += sv[2] * w[0] - sv[0] * w[2];
            tq[2] += sv[0] * w[1] - sv[1] * w[0];
        }
        // symmetric 3x3 inverse through the adjugate
        const double a = I[0], bq = I[1], c = I[2], xy = I[3], xz = I[4], yz = I[5];
        const double A00 = bq * c - yz * yz, A01 = xz * yz - xy * c, A02 = xy * yz - xz * bq;
        const double A11 = a * c - xz * xz, A12 = xy * xz - a * yz, A22 = a * bq - xy * xy;
        const double det = a * A00 + xy * A01 + xz * A02;
        const double tr = a + bq + c;
        double Om[3] = {0, 0, 0};
        if (tr > 0.0 && fabs(det) > 1e-12 * tr * tr * tr) {
            const double id = 1.0 / det;
            Om[0] = (A00 * tq[0] + A01 * tq[1] + A02 * tq[2]) * id;
            Om[1] = (A01 * tq[0] + A11 * tq[1] + A12 * tq[2]) * id;
            Om[2] = (A02 * tq[0] + A12 * tq[1] + A22 * tq[2]) * id;
        }
        if (Omega)
            for (int d = 0; d < 3; ++d) Omega[3 * p + d] = Om[d];
    } else if (Omega) {
        for (int d = 0; d < 3; ++d) Omega[3 * p + d] = 0.0;
    }
    if (U)
        for (int d = 0; d < 3; ++d) U[3 * p + d] = Um[d];
}

cudaError_t launch_particle_reduce(cudaStream_t st, int64_t np, const int32_t* part_start,
                                   const int32_t* part_blobs, const int32_t* box_of_part,
                                   const double* q, const double* u, const GridGeo& g,
                                   double* U, double* Omega)
{
    if (np <= 0) return cudaSuccess;
    k_particle_reduce<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(
        np, part_start, part_blobs, box_of_part, q, u, g, U, Omega);
    return cudaGetLastError();
}

// Transpose of the particle mean U0 = (1/N_p) sum_{i in p} u_i (Sec. 2): every blob of particle
// p receives gU_p / N_p.  One thread per particle; blobs belong to one particle each, so the
// writes are disjoint.
__global__ void k_particle_mean_adjoint(int64_t np, const int32_t* __restrict__ part_start,
                                        const int32_t* __restrict__ part_blobs,
                                        const double* __restrict__ gU, double* __restrict__ gu)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int s = part_start[p], e = part_start[p + 1];
    if (e <= s) return;
    const double inv = 1.0 / (double)(e - s);
    const double g0 = gU[3 * p] * inv, g1 = gU[3 * p + 1] * inv, g2 = gU[3 * p + 2] * inv;
    for (int i = s; i < e; ++i) {
        const int b = part_blobs[i];
        gu[3 * b] = g0;
        gu[3 * b + 1] = g1;
        gu[3 * b + 2] = g2;
    }
}

cudaError_t launch_particle_mean_adjoint(cudaStream_t st, int64_t np, const int32_t* part_start,
                                         const int32_t* part_blobs, const double* gU, double* gu)
{
    if (np <= 0) return cudaSuccess;
    k_particle_mean_adjoint<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(np, part_start,
                                                                         part_blobs, gU, gu);
    return cudaGetLastError();
}

// ==========================================================================================
// Mean of each component grid (FP64 accumulation, fixed order).
template <typename R>
__global__ void __launch_bounds__(256)
k_grid_mean(GridGeo g, const R* __restrict__ v, double* __restrict__ mean_out)
{
    __shared__ double sh[256];
    const int bc = blockIdx.x;
    const R* c = v + (size_t)bc * g.N;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < g.N; i += blockDim.x) s += (double)c[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean_out[bc] = sh[0] / (double)g.N;
}

template <typename R>
cudaError_t launch_grid_mean(cudaStream_t st, int B, const GridGeo& g, const R* v,
                             double* mean_out, double* scratch)
{
    (void)scratch;
    k_grid_mean<R><<<B * 3, 256, 0, st>>>(g, v, mean_out);
    return cudaGetLastError();
}
template cudaError_t launch_grid_mean<float>(cudaStream_t, int, const GridGeo&, const float*,
                                             double*, double*);
template cudaError_t launch_grid_mean<double>(cudaStream_t, int, const GridGeo&, const double*,
                                              double*, double*);

}  // namespace mbk
