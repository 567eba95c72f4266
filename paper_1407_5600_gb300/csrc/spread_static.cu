// mb_spread_static: spreading that allocates nothing.
//
// Some callers cannot call cudaMalloc at all: code running inside another framework's
// allocator budget, a plugin loaded into a process whose device memory is pre-reserved, or a
// host thread that must not trigger an allocation (and the device synchronisation it can
// imply) in the middle of its work.  mb_spread needs a context, and a context owns device
// buffers allocated by mb_create_grid.  This entry point needs neither: it bins the blobs and
// spreads their forces using one fixed scratch array that lives in the library image itself,
// so the caller only passes its own inputs and outputs.
//
// The scratch array is a file-scope __device__ array of fixed size (see SCRATCH_* below,
// about 5 MiB).  Every GPU that loads this library holds it until the process exits.  Host
// code may not use the array's name as a device address: the name is a host-side stand-in.
// The device address is looked up once per device with cudaGetSymbolAddress, on the first
// call made on that device, and cached.
#include <mutex>
#include <string>

#include "mb_internal.cuh"
#include "peskin.cuh"

namespace mbk {
void set_context_free_error(const std::string& msg);   // defined in mb_api.cu
}

namespace {

using namespace mbk;

constexpr int64_t SCRATCH_MAX_BLOBS = 262144;   // blobs per call
constexpr int64_t SCRATCH_MAX_CELLS = 262144;   // bin cells (2h side): a 128^3 grid at most
constexpr int SCAN_THREADS = 1024;
// int32 layout: count[cells] | start[cells + 1] | cell[blobs] | rank[blobs] | sorted[blobs]
constexpr int64_t SCRATCH_WORDS = 2 * SCRATCH_MAX_CELLS + 1 + 3 * SCRATCH_MAX_BLOBS;

static __device__ __align__(256) int32_t g_spread_scratch[SCRATCH_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
int32_t* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(int32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spread_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double wrap_box(double x, double L)
{
    double y = fmod(x, L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

struct StaticGeo {
    int n[3];
    int nc[3];         // bin cells per side (cell side 2h)
    double h, inv_h, inv_w, L[3];
};

__global__ void k_static_count(int64_t nb, const double* __restrict__ pos, StaticGeo g,
                               int32_t* __restrict__ count, int32_t* __restrict__ cell,
                               int32_t* __restrict__ rank)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int c[3];
    for (int d = 0; d < 3; ++d) {
        int k = (int)floor(wrap_box(pos[3 * b + d], g.L[d]) * g.inv_w);
        if (k >= g.nc[d] || k < 0) k = k < 0 ? 0 : g.nc[d] - 1;
        c[d] = k;
    }
    const int id = (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
    cell[b] = id;
    rank[b] = atomicAdd(count + id, 1);
}

// Exclusive scan of count[0, n) into start[0, n]; one block, contiguous chunk per thread.
__global__ void __launch_bounds__(SCAN_THREADS)
k_static_scan(const int32_t* __restrict__ count, int32_t* __restrict__ start, int n)
{
    __shared__ int32_t part[SCAN_THREADS];
    const int per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    int32_t s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {     // inclusive Hillis-Steele scan
        const int32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int i = lo; i < hi; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) start[n] = part[SCAN_THREADS - 1];
}

__global__ void k_static_scatter(int64_t nb, const int32_t* __restrict__ cell,
                                 const int32_t* __restrict__ rank,
                                 const int32_t* __restrict__ start, int32_t* __restrict__ sorted)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    sorted[start[cell[b]] + rank[b]] = (int32_t)b;
}

__host__ __device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__host__ __device__ __forceinline__ int wrapc(int c, int n) { c %= n; return c < 0 ? c + n : c; }

// Cells [lo, lo + cnt) along one dimension whose blobs can reach nodes [T0, T0 + T).
__host__ __device__ __forceinline__ void static_halo(int T0, int T, int nc, int& lo, int& cnt)
{
    lo = fdiv(2 * T0 - 3, 4);
    const int hi = fdiv(T0 + T + 2, 2) - 1;
    cnt = hi - lo + 1;
    if (cnt >= nc) { lo = 0; cnt = nc; }
}

// One CTA owns a TX x TY x TZ node block of all three components, gathers the blobs of the
// bin cells around it (positions and forces read through the sorted index), accumulates the
// in-block part of f = sum_i delta_h(r - q_i) F_i in shared memory and writes the block once.
template <typename R>
__global__ void __launch_bounds__(256)
k_static_spread(const double* __restrict__ pos, const double* __restrict__ F,
                const int32_t* __restrict__ start, const int32_t* __restrict__ sorted,
                StaticGeo g, int TX, int TY, int TZ, int max_ranges, R* __restrict__ f)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tileN = TX * TY * TZ;
    R* acc = reinterpret_cast<R*>(smem_raw);
    int32_t* rbeg = reinterpret_cast<int32_t*>(acc + 3 * tileN);
    int32_t* rpre = rbeg + max_ranges;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int ntx = nx / TX, nty = ny / TY;
    const int T0[3] = {((int)blockIdx.x % ntx) * TX, (((int)blockIdx.x / ntx) % nty) * TY,
                       ((int)blockIdx.x / (ntx * nty)) * TZ};
    const int T[3] = {TX, TY, TZ};
    for (int i = threadIdx.x; i < 3 * tileN; i += blockDim.x) acc[i] = R(0);
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) static_halo(T0[d], T[d], g.nc[d], lo[d], cnt[d]);
    const int rows = cnt[1] * cnt[2], nr = 2 * rows;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int cz = wrapc(lo[2] + r / cnt[1], g.nc[2]);
        const int cy = wrapc(lo[1] + r % cnt[1], g.nc[1]);
        const int base = (cz * g.nc[1] + cy) * g.nc[0];
        const int sx = wrapc(lo[0], g.nc[0]);
        const int ex = sx + cnt[0];
        const int a1 = ex <= g.nc[0] ? ex : g.nc[0];
        rbeg[2 * r] = start[base + sx];
        rpre[2 * r] = start[base + a1] - start[base + sx];
        if (ex > g.nc[0]) {
            rbeg[2 * r + 1] = start[base];
            rpre[2 * r + 1] = start[base + ex - g.nc[0]] - start[base];
        } else {
            rbeg[2 * r + 1] = 0;
            rpre[2 * r + 1] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {            // exclusive prefix of the range lengths
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
    const double inv_h3 = g.inv_h * g.inv_h * g.inv_h;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int a = 0, b = nr - 1;
        while (a < b) {
            const int m = (a + b + 1) >> 1;
            if (rpre[m] <= t) a = m; else b = m - 1;
        }
        const int blob = sorted[rbeg[a] + (t - rpre[a])];
        const double p[3] = {wrap_box(pos[3 * blob], g.L[0]), wrap_box(pos[3 * blob + 1], g.L[1]),
                             wrap_box(pos[3 * blob + 2], g.L[2])};
        for (int comp = 0; comp < 3; ++comp) {
            const R Fa = static_cast<R>(F[3 * blob + comp] * inv_h3);
            R wx[3], wy[3], wz[3];
            const int ix = peskin_window<R>(p[0] * g.inv_h - mac_shift(comp, 0), wx) - T0[0];
            const int iy = peskin_window<R>(p[1] * g.inv_h - mac_shift(comp, 1), wy) - T0[1];
            const int iz = peskin_window<R>(p[2] * g.inv_h - mac_shift(comp, 2), wz) - T0[2];
            R* acc_c = acc + comp * tileN;
            for (int c = 0; c < 3; ++c) {
                const int rz = (iz + c) & (nz - 1);
                if (rz >= TZ) continue;
                for (int bb = 0; bb < 3; ++bb) {
                    const int ry = (iy + bb) & (ny - 1);
                    if (ry >= TY) continue;
                    const R wyz = wy[bb] * wz[c] * Fa;
                    for (int aa = 0; aa < 3; ++aa) {
                        const int rx = (ix + aa) & (nx - 1);
                        if (rx < TX) atomicAdd(acc_c + (rz * TY + ry) * TX + rx, wx[aa] * wyz);
                    }
                }
            }
        }
    }
    __syncthreads();
    const size_t N = (size_t)nx * ny * nz;
    for (int i = threadIdx.x; i < 3 * tileN; i += blockDim.x) {
        const int comp = i / tileN, rem = i - comp * tileN;
        const int rz = rem / (TY * TX), ry = (rem / TX) % TY, rx = rem % TX;
        f[comp * N + ((size_t)(T0[2] + rz) * ny + (T0[1] + ry)) * nx + (T0[0] + rx)] = acc[i];
    }
}

bool is_pow2_in(int n) { return n >= 4 && n <= 128 && (n & (n - 1)) == 0; }

// Device memory of the current device, or managed memory.  Device memory of another GPU is
// refused: the kernels run on the current device and would dereference a peer pointer.
bool on_device(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device == dev;
}

mb_status fail(mb_status s, const std::string& msg)
{
    set_context_free_error("mb_spread_static: " + msg);
    return s;
}

template <typename R>
cudaError_t launch_all(cudaStream_t st, int64_t n, const double* pos, const double* F,
                       int32_t* scratch, const StaticGeo& g, int ncell, R* out)
{
    int32_t* count = scratch;
    int32_t* start = count + SCRATCH_MAX_CELLS;
    int32_t* cell = start + SCRATCH_MAX_CELLS + 1;
    int32_t* rank = cell + SCRATCH_MAX_BLOBS;
    int32_t* sorted = rank + SCRATCH_MAX_BLOBS;
    // the array keeps the previous call's contents: the counts must start at zero
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * ncell, st);
    if (e != cudaSuccess) return e;
    const unsigned nbk = (unsigned)((n + 255) / 256);
    if (n > 0) k_static_count<<<nbk, 256, 0, st>>>(n, pos, g, count, cell, rank);
    k_static_scan<<<1, SCAN_THREADS, 0, st>>>(count, start, ncell);
    if (n > 0) k_static_scatter<<<nbk, 256, 0, st>>>(n, cell, rank, start, sorted);
    // tiles sized so that shared memory stays within the default 48 KiB
    const int TX = g.n[0] < (sizeof(R) == 4 ? 32 : 16) ? g.n[0] : (sizeof(R) == 4 ? 32 : 16);
    const int TY = g.n[1] < 8 ? g.n[1] : 8, TZ = g.n[2] < 8 ? g.n[2] : 8;
    int rows = 1;
    for (int d = 1; d < 3; ++d) {
        int most = 0;
        const int Td = d == 1 ? TY : TZ;
        for (int T0 = 0; T0 < g.n[d]; T0 += Td) {
            int lo, c;
            static_halo(T0, Td, g.nc[d], lo, c);
            most = c > most ? c : most;
        }
        rows *= most;
    }
    const int max_ranges = 2 * rows;
    const size_t smem = 3 * (size_t)TX * TY * TZ * sizeof(R) + sizeof(int32_t) * (2 * max_ranges + 1);
    const unsigned tiles = (unsigned)((g.n[0] / TX) * (g.n[1] / TY) * (g.n[2] / TZ));
    k_static_spread<R><<<tiles, 256, smem, st>>>(pos, F, start, sorted, g, TX, TY, TZ, max_ranges,
                                                 out);
    return cudaGetLastError();
}

}  // namespace

extern "C" mb_status mb_spread_static(const mb_grid_desc* desc, int64_t n, const double* pos,
                                      const double* F, void* grid_out, void* cuda_stream)
{
    if (!desc) return fail(MB_EINVAL, "desc must be non-null");
    const int ns[3] = {desc->nx, desc->ny, desc->nz};
    for (int d = 0; d < 3; ++d)
        if (!is_pow2_in(ns[d])) return fail(MB_EINVAL, "nx, ny, nz must be powers of two in [4, 128]");
    if (!(desc->h > 0.0)) return fail(MB_EINVAL, "h must be positive");
    if (desc->precision != 0 && desc->precision != 1)
        return fail(MB_EINVAL, "precision must be 0 (FP32 grid) or 1 (FP64)");
    if (n < 0 || n > SCRATCH_MAX_BLOBS)
        return fail(MB_EINVAL, "n = " + std::to_string(n) + " is outside [0, " +
                                   std::to_string(SCRATCH_MAX_BLOBS) +
                                   "], the size of the fixed scratch array");
    const int64_t ncell = (int64_t)(ns[0] / 2) * (ns[1] / 2) * (ns[2] / 2);
    if (ncell > SCRATCH_MAX_CELLS) return fail(MB_EINVAL, "grid exceeds the fixed scratch array");
    if (!grid_out || (n > 0 && (!pos || !F)))
        return fail(MB_EINVAL, "pos, F (when n > 0) and grid_out must be non-null");
    if (!on_device(grid_out) || (n > 0 && (!on_device(pos) || !on_device(F))))
        return fail(MB_EINVAL, "pos, F and grid_out must be device pointers on the current "
                               "device (host arrays would need a staging allocation)");
    int32_t* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    StaticGeo g{};
    for (int d = 0; d < 3; ++d) {
        g.n[d] = ns[d];
        g.nc[d] = ns[d] / 2;
        g.L[d] = ns[d] * desc->h;
    }
    g.h = desc->h;
    g.inv_h = 1.0 / desc->h;
    g.inv_w = 1.0 / (2.0 * desc->h);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (st) {
        int sdev = -1, dev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return fail(MB_EINVAL, "cuda_stream is not a valid stream");
        }
        if (sdev != dev) return fail(MB_EINVAL, "cuda_stream belongs to another device");
    }
    if (desc->precision == 0)
        e = launch_all<float>(st, n, pos, F, scratch, g, (int)ncell, static_cast<float*>(grid_out));
    else
        e = launch_all<double>(st, n, pos, F, scratch, g, (int)ncell, static_cast<double*>(grid_out));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MB_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    return MB_OK;
}
