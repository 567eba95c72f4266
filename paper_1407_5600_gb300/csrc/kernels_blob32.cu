// Blob-side kernels of the FP32-grid mode, written for GB300's FP32 pipes.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so in this mode a blob position
// is kept as an integer bin cell c (side w = bs h) plus an offset inside the cell held as an
// unevaluated float sum hi + lo (a "float-float" value): q = c w + hi + lo.  The offset spans
// at most w, so hi + lo resolves positions to about 2^-47 w (7e-15 h for w = 2h), finer than
// an FP64 coordinate of a 128h box.  Every update and every difference of positions is done
// with error-free float transformations (TwoSum, the FMA product error), so nothing here runs
// on the FP64 pipe; FP64 positions are produced only when a caller asks for them.
//
// Layout per blob: float4 A = {hi.x, hi.y, hi.z, cell bits}, float4 B = {lo.x, lo.y, lo.z, 0},
// with the cell packed as cx | cy << 10 | cz << 20.
#include <mutex>

#include "mb_internal.cuh"
#include "peskin.cuh"

namespace mbk {

namespace {

__device__ __forceinline__ int cell_unpack(int packed, int d) { return (packed >> (10 * d)) & 1023; }
__device__ __forceinline__ int cell_pack(int cx, int cy, int cz) { return cx | (cy << 10) | (cz << 20); }

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// Moves one coordinate (cell c, offset hi + lo) by a displacement and renormalises the offset
// into [0, w), carrying whole cells into c (periodic over nc cells).
__device__ __forceinline__ void ff_move(int& c, float& hi, float& lo, float delta, float w, int nc)
{
    float s, e;
    two_sum(hi, delta, s, e);
    two_sum(s, lo + e, hi, lo);
    // at most 8 cells per move (a bound, so that a non-finite offset cannot loop)
    for (int it = 0; it < 8 && hi >= w; ++it) {
        float t, te;
        two_sum(hi, -w, t, te);
        two_sum(t, lo + te, hi, lo);
        c = c + 1 == nc ? 0 : c + 1;
    }
    for (int it = 0; it < 8 && hi < 0.0f; ++it) {
        float t, te;
        two_sum(hi, w, t, te);
        two_sum(t, lo + te, hi, lo);
        c = c == 0 ? nc - 1 : c - 1;
    }
}

// A small integer (|i| < 2^22) as a float, exactly, through the float adder: GB300 issues
// integer-float conversions on its narrow FP64 pipe.
__device__ __forceinline__ float small_i2f(int i)
{
    return __int_as_float(0x4B400000 + i) - 12582912.0f;
}

// Peskin window from the split coordinate: x = q/h - shift = c bs + hi/h - shift.  The nearest
// node floor(x + 1/2) by the same adder trick (|x| < 2^22): x + 1/2 rounded to an integer by
// adding and removing 1.5 * 2^23, less one where that rounded up; equal to floorf.
__device__ __forceinline__ int window32(int c, int bs, float hi, float inv_h, float shift, float w[3])
{
    const float x = hi * inv_h - shift;
    const float y = x + 0.5f;
    const float big = y + 12582912.0f;
    float fl = big - 12582912.0f;
    int il = __float_as_int(big) - 0x4B400000;
    if (fl > y) {
        fl -= 1.0f;
        il -= 1;
    }
    const float t = x - fl;
    const float s = sqrtf(1.0f - 3.0f * t * t);
    w[0] = (2.0f - 3.0f * t - s) * (1.0f / 6.0f);
    w[1] = (1.0f + s) * (1.0f / 3.0f);
    w[2] = (2.0f + 3.0f * t - s) * (1.0f / 6.0f);
    return c * bs + il - 1;
}

struct Geo32 {
    int n[3], nc[3];
    int bs;
    float w, inv_h;
    float L[3];
    int64_t N;
    int64_t ncell;
};

__device__ __forceinline__ Geo32 geo32(const GridGeo& g, const BinGeo& bg)
{
    Geo32 r;
    for (int d = 0; d < 3; ++d) {
        r.n[d] = g.n[d];
        r.nc[d] = bg.nc[d];
        r.L[d] = g.L32[d];
    }
    r.bs = bg.bs;
    r.w = bg.w32;
    r.inv_h = g.inv_h32;
    r.N = g.N;
    r.ncell = bg.ncell;
    return r;
}

// Items split evenly over the warps of a grid that the GPU holds at once (persistent_grid), in
// rounds: R = ceil(n / (32 W)) rounds for W warps, c = ceil(n / (R W)) <= 32 items per warp and
// round, round k giving warp w the items [(k W + w) c, (k W + w + 1) c) (lanes c..31 idle).
// Every warp then has the same work to the end, where a grid of one item per thread ends in a
// partial last wave that leaves SMs idle; and each round covers one contiguous window of W c
// items, so that, with the items in cell order, the GPU works through the grid region by region
// (its L2 holds the nodes of a window when the grids do not fit) and neighbouring items share
// an SM's L1.
template <typename Fn>
__device__ __forceinline__ void for_warp_rounds(int64_t n, Fn&& fn)
{
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t R = (n + 32 * W - 1) / (32 * W);
    if (R == 0) return;
    const int64_t c = (n + R * W - 1) / (R * W);
    for (int64_t k = 0; k < R; ++k) {
        const int64_t t = (k * W + w) * c + lane;
        if (lane < c && t < n) fn(t);
    }
}

// ------------------------------------------------------------------------------------------
// Conversions between FP64 positions and the split form.

__global__ void k_split(int64_t nb, const double* __restrict__ q, GridGeo g, BinGeo bg,
                        float4* __restrict__ A, float4* __restrict__ B)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double w = bg.w;
    int c[3];
    float hi[3], lo[3];
    for (int d = 0; d < 3; ++d) {
        double x = wrap_position(q[3 * b + d], g.L[d]);
        int k = (int)floor(x * bg.inv_w);
        if (k >= bg.nc[d]) k = bg.nc[d] - 1;
        if (k < 0) k = 0;
        const double xl = x - k * w;
        c[d] = k;
        hi[d] = (float)xl;
        lo[d] = (float)(xl - (double)hi[d]);
        // rounding of x / w or of the float offset can leave hi just outside [0, w): carry
        ff_move(c[d], hi[d], lo[d], 0.0f, (float)w, bg.nc[d]);
    }
    A[b] = make_float4(hi[0], hi[1], hi[2], __int_as_float(cell_pack(c[0], c[1], c[2])));
    B[b] = make_float4(lo[0], lo[1], lo[2], 0.0f);
}

__global__ void k_unsplit(int64_t nb, const float4* __restrict__ A, const float4* __restrict__ B,
                          BinGeo bg, GridGeo g, double* __restrict__ q)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double w = bg.w;
    const float4 a = A[b], l = B[b];
    const int pk = __float_as_int(a.w);
    const float hi[3] = {a.x, a.y, a.z}, lo[3] = {l.x, l.y, l.z};
    for (int d = 0; d < 3; ++d)
        q[3 * b + d] = wrap_position(cell_unpack(pk, d) * w + (double)hi[d] + (double)lo[d], g.L[d]);
}

// ------------------------------------------------------------------------------------------
// Interpolation J from the split positions (mode 0: u only; 1: predictor; 2: corrector).
// The x nodes ix, ix + 1, ix + 2 (periodic) of a window lie in the two aligned node pairs that
// start at a = ix & ~1 and at (a + 2) mod nx: each row of a window is read with two 8-byte loads
// instead of three 4-byte ones (a third fewer L1 sector lookups per gather), and the three
// weights are laid over the four loaded nodes, the spare node weighted by zero.  The row sum
// keeps the order of the three-term sum, so adding zero times the spare (finite) node changes
// no bit.  Component grids start 8-byte aligned: device allocations, and N and nx are even.
struct XPair {
    int a0, a1;
    float w[4];
};
__device__ __forceinline__ XPair xpair(int ix, int nx, const float wx[3])
{
    XPair p;
    const int i = ix & (nx - 1);
    const bool odd = (i & 1) != 0;
    p.a0 = i & ~1;
    p.a1 = (p.a0 + 2) & (nx - 1);
    p.w[0] = odd ? 0.0f : wx[0];
    p.w[1] = odd ? wx[0] : wx[1];
    p.w[2] = odd ? wx[1] : wx[2];
    p.w[3] = odd ? wx[2] : 0.0f;
    return p;
}
// One row of a window: sum of the x weights times the grid g0 (+ g1 when not null).
__device__ __forceinline__ float xrow(const float* g0, const float* g1, int row, const XPair& p)
{
    float2 lo = __ldg(reinterpret_cast<const float2*>(g0 + row + p.a0));
    float2 hi = __ldg(reinterpret_cast<const float2*>(g0 + row + p.a1));
    if (g1) {
        const float2 lo1 = __ldg(reinterpret_cast<const float2*>(g1 + row + p.a0));
        const float2 hi1 = __ldg(reinterpret_cast<const float2*>(g1 + row + p.a1));
        lo.x += lo1.x;
        lo.y += lo1.y;
        hi.x += hi1.x;
        hi.y += hi1.y;
    }
    float r = p.w[0] * lo.x;
    r += p.w[1] * lo.y;
    r += p.w[2] * hi.x;
    r += p.w[3] * hi.y;
    return r;
}

// Per-dimension windows for both MAC shifts (0 along the component's own axis, 1/2 across).
struct Win2 {
    float w[2][3];
    int i0[2];
};
__device__ __forceinline__ Win2 windows2(int c, int bs, float hi, float inv_h)
{
    Win2 r;
    r.i0[0] = window32(c, bs, hi, inv_h, 0.0f, r.w[0]);
    r.i0[1] = window32(c, bs, hi, inv_h, 0.5f, r.w[1]);
    return r;
}

template <int MODE>
__global__ void __launch_bounds__(256)
k_interp32(int64_t nb, const float4* __restrict__ A, const float4* __restrict__ Bl,
           const float* __restrict__ v0, const float* __restrict__ v1,
           const int32_t* __restrict__ box_of, GridGeo g, BinGeo bg, float dt,
           const float4* A_base, const float4* B_base, float4* A_out, float4* B_out,
           double* __restrict__ u_out, const int32_t* __restrict__ order,
           int32_t* __restrict__ count, int32_t* __restrict__ blob_cell,
           int32_t* __restrict__ blob_rank)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nb) return;
    // blobs in cell order (when known) so that neighbouring threads gather neighbouring nodes
    const int64_t b = order ? order[t] : t;
    const Geo32 G = geo32(g, bg);
    const int box = box_of ? box_of[b] : 0;
    const float4 a = A[b];
    const int pk = __float_as_int(a.w);
    const int c[3] = {cell_unpack(pk, 0), cell_unpack(pk, 1), cell_unpack(pk, 2)};
    const float hi[3] = {a.x, a.y, a.z};
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    float u[3];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        float wx[3], wy[3], wz[3];
        const int ix = window32(c[0], G.bs, hi[0], G.inv_h, comp == 0 ? 0.f : 0.5f, wx);
        const int iy = window32(c[1], G.bs, hi[1], G.inv_h, comp == 1 ? 0.f : 0.5f, wy);
        const int iz = window32(c[2], G.bs, hi[2], G.inv_h, comp == 2 ? 0.f : 0.5f, wz);
        const size_t base = ((size_t)box * 3 + comp) * (size_t)G.N;
        const float* c0 = v0 + base;
        const float* c1 = MODE == 2 ? v1 + base : nullptr;
        // 32-bit offsets inside the component grid, wrapped indices once per dimension
        const XPair xp = xpair(ix, nx, wx);
        int yo[3], zo[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            yo[d] = ((iy + d) & (ny - 1)) * nx;
            zo[d] = ((iz + d) & (nz - 1)) * (ny * nx);
        }
        float acc = 0.0f;
#pragma unroll
        for (int cz = 0; cz < 3; ++cz) {
#pragma unroll
            for (int cy = 0; cy < 3; ++cy) {
                const float r = xrow(c0, MODE == 2 ? c1 : nullptr, zo[cz] + yo[cy], xp);
                acc += wy[cy] * wz[cz] * r;
            }
        }
        u[comp] = MODE == 2 ? 0.5f * acc : acc;
    }
    if (MODE == 0) {
        for (int d = 0; d < 3; ++d) u_out[3 * b + d] = (double)u[d];
        return;
    }
    // move the base position (q^n for both the predictor and the corrector)
    const float4 ab = MODE == 1 ? a : A_base[b];
    const float4 lb = MODE == 1 ? Bl[b] : B_base[b];
    int cc[3] = {cell_unpack(__float_as_int(ab.w), 0), cell_unpack(__float_as_int(ab.w), 1),
                 cell_unpack(__float_as_int(ab.w), 2)};
    float h2[3] = {ab.x, ab.y, ab.z}, l2[3] = {lb.x, lb.y, lb.z};
    const float scale = MODE == 1 ? 0.5f * dt : dt;
    for (int d = 0; d < 3; ++d) ff_move(cc[d], h2[d], l2[d], scale * u[d], G.w, G.nc[d]);
    A_out[b] = make_float4(h2[0], h2[1], h2[2], __int_as_float(cell_pack(cc[0], cc[1], cc[2])));
    B_out[b] = make_float4(l2[0], l2[1], l2[2], 0.0f);
    if (MODE == 1 && count) {        // bin the midpoint position (first step of the cell sort)
        const int cell = (int)(box * G.ncell) + (cc[2] * G.nc[1] + cc[1]) * G.nc[0] + cc[0];
        blob_cell[b] = cell;
        blob_rank[b] = atomicAdd(count + cell, 1);
    }
}

// J v at a split position for all three components: sum over the 27-node windows of one grid
// (v1 == nullptr) or of the sum v0 + v1.
__device__ __forceinline__ void gather32(const int c[3], const float hi[3], const float* v0,
                                         const float* v1, size_t box_base, const Geo32& G,
                                         float u[3])
{
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        float wx[3], wy[3], wz[3];
        const int ix = window32(c[0], G.bs, hi[0], G.inv_h, comp == 0 ? 0.f : 0.5f, wx);
        const int iy = window32(c[1], G.bs, hi[1], G.inv_h, comp == 1 ? 0.f : 0.5f, wy);
        const int iz = window32(c[2], G.bs, hi[2], G.inv_h, comp == 2 ? 0.f : 0.5f, wz);
        // one 64-bit base per component grid, 32-bit offsets inside it (a box grid has at most
        // 2^24 nodes), the wrapped node indices computed once per dimension
        const size_t base = box_base + (size_t)comp * (size_t)G.N;
        const float* g0 = v0 + base;
        const float* g1 = v1 ? v1 + base : nullptr;
        const XPair xp = xpair(ix, nx, wx);
        int yo[3], zo[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            yo[d] = ((iy + d) & (ny - 1)) * nx;
            zo[d] = ((iz + d) & (nz - 1)) * (ny * nx);
        }
        float acc = 0.0f;
#pragma unroll
        for (int cz = 0; cz < 3; ++cz) {
#pragma unroll
            for (int cy = 0; cy < 3; ++cy) {
                const float r = xrow(g0, g1, zo[cz] + yo[cy], xp);
                acc += wy[cy] * wz[cz] * r;
            }
        }
        u[comp] = acc;
    }
}

// The corrector of step n followed by the predictor of step n + 1 for the blob at sorted
// position t:
//   q^{n+1}   = q^n + dt J(q^{n+1/2}) (v^n + v^{n+1}) / 2       (A_base, B_base -> A_out, B_out)
//   q^{n+3/2} = q^{n+1} + (dt/2) J(q^{n+1}) v^{n+1}             (-> Ah_out, Bh_out, binned)
// The second gather reads the nodes the first has just brought into L1.  A (q^{n+1/2}) and
// Ah_out may alias, as may A_base/B_base and A_out/B_out: each thread reads its blob's entries
// before writing them.
struct FusedArgs {
    const float4* A;
    const float* v0;          // corrector: J of v0 (+ v1 when not null), halved
    const float* v1;
    const float* vp;          // predictor of the next step: J of vp (= v^{n+1})
    const int32_t* box_of;
    float dt;
    const float4* A_base;
    const float4* B_base;
    float4* A_out;
    float4* B_out;
    float4* Ah_out;
    float4* Bh_out;
    const int32_t* order;
    int32_t* count;
    int32_t* blob_cell;
    int32_t* blob_rank;
    float4* u_out;            // J(q^{n+1}) v^{n+1}: the blob velocities of the new state
};

__device__ __forceinline__ void fused_blob(int64_t t, const FusedArgs& f, const Geo32& G)
{
    const int64_t b = f.order ? f.order[t] : t;
    const int box = f.box_of ? f.box_of[b] : 0;
    const size_t box_base = (size_t)box * 3 * (size_t)G.N;
    float u[3];
    {
        const float4 a = f.A[b];
        const int pk = __float_as_int(a.w);
        const int c[3] = {cell_unpack(pk, 0), cell_unpack(pk, 1), cell_unpack(pk, 2)};
        const float hi[3] = {a.x, a.y, a.z};
        gather32(c, hi, f.v0, f.v1, box_base, G, u);
    }
    const float4 ab = f.A_base[b], lb = f.B_base[b];
    int cc[3] = {cell_unpack(__float_as_int(ab.w), 0), cell_unpack(__float_as_int(ab.w), 1),
                 cell_unpack(__float_as_int(ab.w), 2)};
    float h2[3] = {ab.x, ab.y, ab.z}, l2[3] = {lb.x, lb.y, lb.z};
    for (int d = 0; d < 3; ++d) ff_move(cc[d], h2[d], l2[d], f.dt * (0.5f * u[d]), G.w, G.nc[d]);
    f.A_out[b] = make_float4(h2[0], h2[1], h2[2], __int_as_float(cell_pack(cc[0], cc[1], cc[2])));
    f.B_out[b] = make_float4(l2[0], l2[1], l2[2], 0.0f);
    gather32(cc, h2, f.vp, nullptr, box_base, G, u);
    f.u_out[b] = make_float4(u[0], u[1], u[2], 0.0f);
    for (int d = 0; d < 3; ++d) ff_move(cc[d], h2[d], l2[d], 0.5f * f.dt * u[d], G.w, G.nc[d]);
    f.Ah_out[b] = make_float4(h2[0], h2[1], h2[2], __int_as_float(cell_pack(cc[0], cc[1], cc[2])));
    f.Bh_out[b] = make_float4(l2[0], l2[1], l2[2], 0.0f);
    const int cell = (int)(box * G.ncell) + (cc[2] * G.nc[1] + cc[1]) * G.nc[0] + cc[0];
    f.blob_cell[b] = cell;
    f.blob_rank[b] = atomicAdd(f.count + cell, 1);
}

__global__ void __launch_bounds__(256, 4)
k_interp32_fused(int64_t nb, FusedArgs f, GridGeo g, BinGeo bg)
{
    dep_wait();
    dep_release();
    const Geo32 G = geo32(g, bg);
    for_warp_rounds(nb, [&](int64_t t) { fused_blob(t, f, G); });
}

// ------------------------------------------------------------------------------------------
// Binning from the packed cells; loc[slot] = {hi, particle id} for the pair prefilter.
__global__ void k_bin_count32(int64_t nb, const float4* __restrict__ A,
                              const int32_t* __restrict__ box_of, BinGeo bg,
                              int32_t* __restrict__ count, int32_t* __restrict__ blob_cell,
                              int32_t* __restrict__ blob_rank)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int pk = __float_as_int(A[b].w);
    const int box = box_of ? box_of[b] : 0;
    const int cell = (int)(box * bg.ncell) +
                     (cell_unpack(pk, 2) * bg.nc[1] + cell_unpack(pk, 1)) * bg.nc[0] +
                     cell_unpack(pk, 0);
    blob_cell[b] = cell;
    blob_rank[b] = atomicAdd(count + cell, 1);
}


// Counting sort in two launches.  k_bin_scan32: each block scans 4096 cell counts in place
// (exclusive, block-local) and publishes its total; the last block to finish (atomic ticket
// after a fence; no block waits for another) scans the block totals into tile offsets, writes
// the grand total and resets the ticket for the next launch.  k_bin_place32: cell_start =
// local scan + tile offset for every cell, and every blob's slot from the same two numbers.
constexpr int BIN_SCAN_THREADS = 1024, BIN_SCAN_LOG = 12;          // 4096 cells per block

__global__ void __launch_bounds__(BIN_SCAN_THREADS)
k_bin_scan32(int32_t* __restrict__ c, int64_t n, int32_t* __restrict__ tile_off,
             int32_t* __restrict__ total, unsigned* __restrict__ ticket)
{
    dep_wait();
    dep_release();
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t block_total;
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x << BIN_SCAN_LOG) + 4 * threadIdx.x;
    int32_t v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = base + i < n ? c[base + i] : 0;
    const int32_t s4 = v[0] + v[1] + v[2] + v[3];
    int32_t x = s4;
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
    int32_t run = x - s4 + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) c[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == BIN_SCAN_THREADS - 1) block_total = run;
    __syncthreads();
    if (threadIdx.x == 0) {
        tile_off[blockIdx.x] = block_total;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int32_t carry = 0;
    for (int c0 = 0; c0 < (int)gridDim.x; c0 += BIN_SCAN_THREADS) {
        const int i = c0 + threadIdx.x;
        const int32_t t = i < (int)gridDim.x ? __ldcg(tile_off + i) : 0;
        int32_t y0 = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, y0, o);
            if (lane >= o) y0 += y;
        }
        __syncthreads();
        if (lane == 31) warp_tot[warp] = y0;
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
        const int32_t excl = carry + y0 - t + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (i < (int)gridDim.x) tile_off[i] = excl;
        carry += warp_tot[31];
    }
    if (threadIdx.x == 0) {
        *total = carry;
        *ticket = 0u;
    }
}

__global__ void __launch_bounds__(256)
k_bin_place32(int64_t nb, int64_t ncells, const int32_t* __restrict__ local,
              const int32_t* __restrict__ tile_off, int32_t* __restrict__ cell_start,
              const int32_t* __restrict__ blob_cell, const int32_t* __restrict__ blob_rank,
              int32_t* __restrict__ sorted, const float4* __restrict__ A,
              const int32_t* __restrict__ pid, float4* __restrict__ loc)
{
    dep_wait();
    dep_release();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ncells) cell_start[i] = local[i] + tile_off[i >> BIN_SCAN_LOG];
    if (i < nb) {
        const int cell = blob_cell[i];
        const int slot = local[cell] + tile_off[cell >> BIN_SCAN_LOG] + blob_rank[i];
        sorted[slot] = (int32_t)i;
        const float4 a = A[i];
        loc[slot] = make_float4(a.x, a.y, a.z, __int_as_float(pid[i]));
    }
}

// ------------------------------------------------------------------------------------------
// Forces.  Springs: the bond vector r = (c_b - c_j) w + (hi_b - hi_j) + (lo_b - lo_j) and the
// extension |r|^2 - r0^2 in float-float (the stiff springs cancel about six digits there),
// the force magnitude in float.  Repulsion: float, from the cell-local coordinates.
__device__ __forceinline__ void spring32(const int cb[3], const float hb[3], const float lb[3],
                                         float4 aj, float4 bj, float r0, float r0h, float r0l,
                                         float k, const Geo32& G, float F[3])
{
    const int pj = __float_as_int(aj.w);
    const float hj[3] = {aj.x, aj.y, aj.z}, lj[3] = {bj.x, bj.y, bj.z};
    float rh[3], rl[3];
    for (int d = 0; d < 3; ++d) {
        int dc = cb[d] - cell_unpack(pj, d);
        const int nc = G.nc[d];
        if (2 * dc > nc) dc -= nc;
        else if (2 * dc < -nc) dc += nc;
        float s, e1, s2, e2;
        two_sum(hb[d], -hj[d], s, e1);
        two_sum(small_i2f(dc) * G.w, s, s2, e2);
        float h, l;
        two_sum(s2, e1 + e2 + (lb[d] - lj[d]), h, l);
        const float half = 0.5f * G.L[d];
        if (h >= half) { float t, te; two_sum(h, -G.L[d], t, te); two_sum(t, l + te, h, l); }
        else if (h < -half) { float t, te; two_sum(h, G.L[d], t, te); two_sum(t, l + te, h, l); }
        rh[d] = h;
        rl[d] = l;
    }
    // |r|^2 as float-float: sum of hi^2 (with exact product errors) and 2 hi lo
    float p[3], pe[3];
    for (int d = 0; d < 3; ++d) {
        p[d] = rh[d] * rh[d];
        pe[d] = fmaf(rh[d], rh[d], -p[d]) + 2.0f * rh[d] * rl[d];
    }
    float s01, e01, P, e2;
    two_sum(p[0], p[1], s01, e01);
    two_sum(s01, p[2], P, e2);
    const float Pl = e01 + e2 + pe[0] + pe[1] + pe[2];
    const float d2 = (P - r0h) + (Pl - r0l);      // P - r0h is exact near the rest length
    // |r| - r0 = d2 / (|r| + r0); the reciprocal square root and the fast divide carry a few
    // ulps of float, far below the float grid's own rounding
    const float len = P * rsqrtf(P);
    const float mag = -k * __fdividef(d2, (len + r0) * len);
    for (int d = 0; d < 3; ++d) F[d] += mag * rh[d];
}

// Spring forces, one thread per blob: the bonds of its adjacency list (entries with the sign
// bit of j set are owned: the opposite force also goes to blob j).  Fs must be zero on entry;
// every contribution is added atomically, a blob's own sum once.
__global__ void __launch_bounds__(256)
k_springs32(int64_t nb, const float4* __restrict__ A, const float4* __restrict__ Bv,
            const int4* __restrict__ adj, const int32_t* __restrict__ adj_start,
            const int32_t* __restrict__ box_of, const float* __restrict__ box_par, GridGeo g,
            BinGeo bg, float* __restrict__ Fs)
{
    dep_wait();
    dep_release();
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int e0 = adj_start[b], e1 = adj_start[b + 1];
    if (e0 == e1) return;
    const Geo32 G = geo32(g, bg);
    const float4 ab = A[b], lbv = Bv[b];
    const int pk = __float_as_int(ab.w);
    const int cb[3] = {cell_unpack(pk, 0), cell_unpack(pk, 1), cell_unpack(pk, 2)};
    const float hb[3] = {ab.x, ab.y, ab.z}, lb[3] = {lbv.x, lbv.y, lbv.z};
    const float k_spring = box_par[3 * (box_of ? box_of[b] : 0)];
    float F[3] = {0.f, 0.f, 0.f};
#pragma unroll 2
    for (int e = e0; e < e1; ++e) {
        const int4 ad = adj[e];
        const int j = ad.x & 0x7fffffff;
        float f[3] = {0.f, 0.f, 0.f};
        spring32(cb, hb, lb, A[j], Bv[j], __int_as_float(ad.y), __int_as_float(ad.z),
                 __int_as_float(ad.w), k_spring, G, f);
        for (int d = 0; d < 3; ++d) F[d] += f[d];
        if (ad.x < 0)
            for (int d = 0; d < 3; ++d) atomicAdd(Fs + 4 * (int64_t)j + d, -f[d]);
    }
    for (int d = 0; d < 3; ++d) atomicAdd(Fs + 4 * b + d, F[d]);
}

// Spring forces when every particle shares one bond pattern (Springs32::tmpl).  A block holds
// whole particles (blockDim = ppb m threads, one per blob, in blob order).  Every bond is
// evaluated once, by the end its evaluation list names, which adds the force to its own sum
// and leaves the opposite force in one of its shared-memory slots; after a barrier each thread
// adds the slots of its collection list.  The pattern spreads the evaluations evenly (an
// icosahedron's 42 bonds: none by the centre, at most 4 by a vertex), no per-blob list is read,
// and each blob's sum has a fixed order and is stored once: no atomics and no zeroing pass.
//   tmpl entries: evaluation {offset | (slot + 1) << 16, r0, r0^2 hi, lo}, collection
//   {offset, slot, 0, 0}; tstart[2l], tstart[2l + 1], tstart[2l + 2] bound blob l's two lists.
__global__ void __launch_bounds__(256)
k_springs32_shared(int nb, int m, int S, const float4* __restrict__ A,
                   const float4* __restrict__ Bv, const int4* __restrict__ tmpl,
                   const int32_t* __restrict__ tstart, const int32_t* __restrict__ box_of,
                   const float* __restrict__ box_par, GridGeo g, BinGeo bg,
                   float4* __restrict__ Fs)
{
    extern __shared__ float slot_f[];                    // [blockDim][S][3]
    dep_wait();
    dep_release();
    const int tid = threadIdx.x;
    const int b = blockIdx.x * blockDim.x + tid;
    const bool live = b < nb;
    const int l = tid % m;
    float F[3] = {0.f, 0.f, 0.f};
    if (live) {
        const Geo32 G = geo32(g, bg);
        const float4 ab = A[b], lbv = Bv[b];
        const int pk = __float_as_int(ab.w);
        const int cb[3] = {cell_unpack(pk, 0), cell_unpack(pk, 1), cell_unpack(pk, 2)};
        const float hb[3] = {ab.x, ab.y, ab.z}, lb[3] = {lbv.x, lbv.y, lbv.z};
        const float k_spring = box_par[3 * (box_of ? box_of[b] : 0)];
        const int e0 = __ldg(tstart + 2 * l), e1 = __ldg(tstart + 2 * l + 1);
        for (int e = e0; e < e1; ++e) {
            const int4 ad = __ldg(tmpl + e);
            const int j = b + (int)(short)(ad.x & 0xffff);
            const int slot = (ad.x >> 16) - 1;
            float f[3] = {0.f, 0.f, 0.f};
            spring32(cb, hb, lb, A[j], Bv[j], __int_as_float(ad.y), __int_as_float(ad.z),
                     __int_as_float(ad.w), k_spring, G, f);
            for (int d = 0; d < 3; ++d) {
                F[d] += f[d];
                slot_f[(tid * S + slot) * 3 + d] = -f[d];
            }
        }
    }
    __syncthreads();
    if (!live) return;
    const int c0 = __ldg(tstart + 2 * l + 1), c1 = __ldg(tstart + 2 * l + 2);
    for (int e = c0; e < c1; ++e) {
        const int4 ad = __ldg(tmpl + e);
        const int p = tid + ad.x;
        for (int d = 0; d < 3; ++d) F[d] += slot_f[(p * S + ad.y) * 3 + d];
    }
    Fs[b] = make_float4(F[0], F[1], F[2], 0.0f);
}

struct Force32Args {
    const int64_t* box_off;
    const int32_t* sorted;
    const float4* A;          // split midpoint positions (blob order)
    const float4* B;
    const float4* loc;        // [slot] hi + particle id
    const float4* Fs;         // [nb] spring forces (k_springs32)
    const float* box_par;     // [B][3] k_spring, k_rep, r_cut
    const int32_t* cell_start;
    const int32_t* blob_cell;
    const float4* ext;        // [nb] or null
    float4* F;                // [nb] blob forces
    float4* rec;              // [2 * slot]: split hi + cell, force
};

__global__ void __launch_bounds__(256)
k_forces32(Force32Args a, GridGeo g, BinGeo bg)
{
    dep_wait();
    dep_release();
    const Geo32 G = geo32(g, bg);
    const int box = blockIdx.y;
    const int64_t s0 = a.box_off[box], cnt = a.box_off[box + 1] - s0;
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= cnt) return;
    const int64_t slot = s0 + local;
    const int b = a.sorted[slot];
    const float4 ab = a.A[b];
    const int pk = __float_as_int(ab.w);
    const int cb[3] = {cell_unpack(pk, 0), cell_unpack(pk, 1), cell_unpack(pk, 2)};
    float F[3] = {0.f, 0.f, 0.f};
    if (a.ext) {
        const float4 e = a.ext[b];
        F[0] = e.x;
        F[1] = e.y;
        F[2] = e.z;
    }
    const float k_rep = a.box_par[3 * box + 1];
    const float r_cut = a.box_par[3 * box + 2];
    {
        const float4 fs = a.Fs[b];
        F[0] += fs.x;
        F[1] += fs.y;
        F[2] += fs.z;
    }
    if (k_rep != 0.0f && r_cut > 0.0f) {
        const float4 me = a.loc[slot];
        const int pb = __float_as_int(me.w);
        const bool wide = G.nc[0] >= 3 && G.nc[1] >= 3 && G.nc[2] >= 3;
        const float rc2 = r_cut * r_cut;
        // Only neighbour cells on the blob's side can hold a partner closer than r_cut <= w:
        // along each axis the lower neighbour if the offset is below r_cut, the upper one if it
        // is above w - r_cut (8 of the 27 cells for r_cut = w/2).
        const float mine[3] = {me.x, me.y, me.z};
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            if (G.nc[d] >= 3 && r_cut <= G.w) {
                lo[d] = mine[d] < r_cut ? -1 : 0;
                hi[d] = mine[d] >= G.w - r_cut ? 1 : 0;
            } else if (G.nc[d] >= 3) {
                lo[d] = -1;
                hi[d] = 1;
            } else {
                lo[d] = 0;
                hi[d] = G.nc[d] - 1;
            }
        }
        float Fp[3] = {0.f, 0.f, 0.f};
        // neighbour cell coordinate with a conditional periodic wrap (no integer division)
        auto nbr = [](int c, int d, int nc) {
            if (nc < 3) return d;
            int x = c + d;
            x += x < 0 ? nc : 0;
            x -= x >= nc ? nc : 0;
            return x;
        };
        const int boxbase = (int)(box * G.ncell);
        auto pair = [&](const float4 lj, float ox, float oy, float oz) {
            float r[3] = {me.x - lj.x - ox, me.y - lj.y - oy, me.z - lj.z - oz};
            if (!wide)
                for (int d = 0; d < 3; ++d) {
                    if (r[d] >= 0.5f * G.L[d]) r[d] -= G.L[d];
                    else if (r[d] < -0.5f * G.L[d]) r[d] += G.L[d];
                }
            const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (r2 >= rc2 || r2 == 0.0f) return;
            // k_rep (r_cut - |r|) / |r| = k_rep (r_cut / |r| - 1)
            const float mag = k_rep * (r_cut * rsqrtf(r2) - 1.0f);
            for (int d = 0; d < 3; ++d) Fp[d] += mag * r[d];
        };
        if (wide && 2.0f * r_cut <= G.w) {
            // at most two cells per axis: read all (up to 8) cell ranges first, so that their
            // loads are in flight together, then visit the candidates
            // cell k = (kx, ky, kz) of a 2 x 2 x 2 block starting at (lo[0], lo[1], lo[2]);
            // absent when the axis has one cell only (hi == lo)
            int cs0[8], cs1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
                cs0[k] = cs1[k] = 0;
                if (lo[0] + kx <= hi[0] && lo[1] + ky <= hi[1] && lo[2] + kz <= hi[2]) {
                    const int cc = boxbase + (nbr(cb[2], lo[2] + kz, G.nc[2]) * G.nc[1] +
                                              nbr(cb[1], lo[1] + ky, G.nc[1])) * G.nc[0] +
                                   nbr(cb[0], lo[0] + kx, G.nc[0]);
                    cs0[k] = a.cell_start[cc];
                    cs1[k] = a.cell_start[cc + 1];
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
                const float ox = small_i2f(lo[0] + kx) * G.w, oy = small_i2f(lo[1] + ky) * G.w,
                            oz = small_i2f(lo[2] + kz) * G.w;
                for (int t = cs0[k]; t < cs1[k]; ++t) {
                    const float4 lj = a.loc[t];
                    if (t == slot || __float_as_int(lj.w) == pb) continue;
                    pair(lj, ox, oy, oz);
                }
            }
        } else {
            for (int dz = lo[2]; dz <= hi[2]; ++dz) {
                const int cz = nbr(cb[2], dz, G.nc[2]);
                for (int dy = lo[1]; dy <= hi[1]; ++dy) {
                    const int cy = nbr(cb[1], dy, G.nc[1]);
                    const int rowc = boxbase + (cz * G.nc[1] + cy) * G.nc[0];
                    for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                        const int cx = nbr(cb[0], dx, G.nc[0]);
                        const int cc = rowc + cx;
                        // cell offset of the neighbour (unwrapped) in the wide case; otherwise
                        // the minimum image of the difference
                        const float ox = small_i2f(wide ? dx : cx - cb[0]) * G.w;
                        const float oy = small_i2f(wide ? dy : cy - cb[1]) * G.w;
                        const float oz = small_i2f(wide ? dz : cz - cb[2]) * G.w;
                        for (int t = a.cell_start[cc]; t < a.cell_start[cc + 1]; ++t) {
                            if (t == slot) continue;
                            const float4 lj = a.loc[t];
                            if (__float_as_int(lj.w) == pb) continue;
                            pair(lj, ox, oy, oz);
                        }
                    }
                }
            }
        }
        for (int d = 0; d < 3; ++d) F[d] += Fp[d];
    }
    a.F[b] = make_float4(F[0], F[1], F[2], 0.f);
    a.rec[2 * slot] = ab;
    a.rec[2 * slot + 1] = make_float4(F[0], F[1], F[2], 0.f);
}

// ------------------------------------------------------------------------------------------
// Spreading from the FP32 records.
// Spreading, one block per tile of TX x TY x TZ nodes (whole bin cells).  The block spreads the
// blobs binned in its cells, each exactly once, into a shared-memory copy of the nodes their
// windows can reach: x over [T0 - 4, T0 + TX + 4) in 16-byte chunks, y and z over
// [T0 - 1, T0 + T + 1] (a blob in the tile has its window start in [T0 - 1, T0 + T - 1]).  The
// copy holds 32-bit fixed-point sums (integer shared-memory atomics), scaled per tile by a power
// of two from a bound on its largest node value: a node receives only blobs within 1.5 h of it
// along each axis, which lie in at most three consecutive bin cells per axis (cells are at
// least 2 h wide), so the bound is a bound on the sum of the blobs' largest force components
// over any 3 x 3 x 3 block of the tile's cells, times the kernel's largest weight (2/3)^3.  The
// block then adds the copy to f (zeroed beforehand) with vector atomics, skipping all-zero
// chunks; nodes shared with neighbouring tiles receive every tile's part.  TXc = 0 takes the
// tile from the arguments (small grids).
template <int TXc, int TYc, int TZc>
__global__ void __launch_bounds__(256)
k_spread32(const float4* __restrict__ rec, const int32_t* __restrict__ cell_start, GridGeo g,
           BinGeo bg, int TXr, int TYr, int TZr, float* __restrict__ f)
{
    dep_wait();
    dep_release();
    const int TX = TXc ? TXc : TXr, TY = TYc ? TYc : TYr, TZ = TZc ? TZc : TZr;
    const int SXC = TX / 4 + 2, SX = 4 * SXC, SY = TY + 3, SZ = TZ + 3;
    const int SN = SX * SY * SZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* acc = reinterpret_cast<int*>(smem_raw);                 // [3][SZ][SY][SX]
    __shared__ int rb[64], rp[65];
    __shared__ float wmax[8];
    const Geo32 G = geo32(g, bg);
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const int box = blockIdx.y;
    const int ntx = nx / TX, nty = ny / TY;
    const int T0[3] = {((int)blockIdx.x % ntx) * TX, (((int)blockIdx.x / ntx) % nty) * TY,
                       ((int)blockIdx.x / (ntx * nty)) * TZ};
    const int ncx = TX / G.bs, ncy = TY / G.bs, ncz = TZ / G.bs;
    const int rows = ncy * ncz;
    // the tile's rows of cells (at most 64): start slot and length, and the exclusive prefix of
    // the lengths, scanned by the first two warps (32 rows each, then the first warp's carry)
    __shared__ int carry0;
    if (threadIdx.x < 64) {
        const int r = threadIdx.x;
        int len = 0;
        if (r < rows) {
            const int cz = T0[2] / G.bs + r / ncy, cy = T0[1] / G.bs + r % ncy;
            const int64_t base = box * G.ncell + ((int64_t)cz * G.nc[1] + cy) * G.nc[0] + T0[0] / G.bs;
            rb[r] = cell_start[base];
            len = cell_start[base + ncx] - rb[r];
        }
        int x = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((r & 31) >= o) x += y;
        }
        rp[r] = x - len;                       // exclusive within the warp
        if (r == 31) carry0 = x;
        if (r == 63) rp[64] = x;               // the second warp's total (carry added below)
    }
    const int ncell = ncx * rows;
    float* cf = reinterpret_cast<float*>(acc + 3 * SN);          // [ncz][ncy][ncx] force sums
    {
        int4* a4 = reinterpret_cast<int4*>(acc);
        for (int i = threadIdx.x; i < 3 * SN / 4; i += blockDim.x) a4[i] = make_int4(0, 0, 0, 0);
        for (int i = threadIdx.x; i < ncell; i += blockDim.x) cf[i] = 0.0f;
    }
    __syncthreads();
    if (threadIdx.x >= 32 && threadIdx.x < 65) rp[threadIdx.x] += carry0;
    __syncthreads();
    const int total = rp[rows];
    // the row holding position t of the tile's blobs: the last r with rp[r] <= t (rows with no
    // blobs share their start with the next row, so take the last of equal starts)
    auto slot_of = [&](int t) {
        int r = 0;
#pragma unroll
        for (int step = 32; step > 0; step >>= 1)
            if (r + step < rows && rp[r + step] <= t) r += step;
        return (int64_t)rb[r] + (t - rp[r]);
    };
    // the tile's fixed-point scale: 2^(30 - e) with 2^e above the node bound: per cell the sum
    // of its blobs' largest force components; a 3 x 3 x 3 block of cells sums at most nine times
    // the largest sum over three cells along x; times (2/3)^3 / h^3 (and 2^-16 for the float
    // sums' rounding)
    const float inv_h3 = G.inv_h * G.inv_h * G.inv_h;
    const int cx0 = T0[0] / G.bs, cy0 = T0[1] / G.bs, cz0 = T0[2] / G.bs;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int64_t slot = slot_of(t);
        const int pk = __float_as_int(rec[2 * slot].w);
        const float4 fv = rec[2 * slot + 1];
        const int c = ((cell_unpack(pk, 2) - cz0) * ncy + (cell_unpack(pk, 1) - cy0)) * ncx +
                      (cell_unpack(pk, 0) - cx0);
        atomicAdd(cf + c, fmaxf(fabsf(fv.x), fmaxf(fabsf(fv.y), fabsf(fv.z))));
    }
    __syncthreads();
    // sums over three neighbouring cells along x by shuffles (one warp per row of cells, lane =
    // cell, ncx <= 32); a 3 x 3 x 3 block sums nine of them
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float fm = 0.f;
    for (int r = warp; r < rows; r += nwarps) {
        const float v = lane < ncx ? cf[r * ncx + lane] : 0.0f;
        float left = __shfl_up_sync(0xffffffffu, v, 1);
        float right = __shfl_down_sync(0xffffffffu, v, 1);
        if (lane == 0) left = 0.0f;
        if (lane == 31) right = 0.0f;
        fm = fmaxf(fm, left + v + right);
    }
    fm *= 9.0f;
    for (int o = 16; o > 0; o >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = fm;
    __syncthreads();
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fm = fmaxf(fm, wmax[w]);
    const float bound = fm * (1.0f + 1.0f / 65536.0f) * (8.0f / 27.0f) * inv_h3;
    int e = 0;
    frexpf(bound, &e);                                           // bound < 2^e
    const float scale = bound > 0.f ? ldexpf(1.0f, 30 - e) : 1.0f;
    // origin of the shared copy in node coordinates
    const int ox = T0[0] - 4, oy = T0[1] - 1, oz = T0[2] - 1;
    // the lanes of a warp take blobs total/32 apart in the cell order (different cell rows):
    // their windows then rarely share shared-memory words or banks
    const int stride = total >> 5, body32 = stride << 5;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int tp = t < body32 ? (t & 31) * stride + (t >> 5) : t;
        const int64_t slot = slot_of(tp);
        const float4 pa = rec[2 * slot], fv = rec[2 * slot + 1];
        const int pk = __float_as_int(pa.w);
        const Win2 wx = windows2(cell_unpack(pk, 0), G.bs, pa.x, G.inv_h);
        const Win2 wy = windows2(cell_unpack(pk, 1), G.bs, pa.y, G.inv_h);
        const Win2 wz = windows2(cell_unpack(pk, 2), G.bs, pa.z, G.inv_h);
        const float Fv[3] = {fv.x * inv_h3 * scale, fv.y * inv_h3 * scale, fv.z * inv_h3 * scale};
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const int sxs = comp == 0 ? 0 : 1, sys = comp == 1 ? 0 : 1, szs = comp == 2 ? 0 : 1;
            // window starts in the copy: [3, TX + 3] and [0, T] for blobs of the tile (offsets
            // in [0, w)); clamped so that no offset can address outside the copy
            const int lx = min(max(wx.i0[sxs] - ox, 0), SX - 3);
            const int ly = min(max(wy.i0[sys] - oy, 0), SY - 3);
            const int lz = min(max(wz.i0[szs] - oz, 0), SZ - 3);
            int* a0 = acc + comp * SN + (lz * SY + ly) * SX + lx;
#pragma unroll
            for (int cz = 0; cz < 3; ++cz) {
                const float wzc = wz.w[szs][cz] * Fv[comp];
#pragma unroll
                for (int cy = 0; cy < 3; ++cy) {
                    const float wyz = wy.w[sys][cy] * wzc;
                    int* row = a0 + (cz * SY + cy) * SX;
#pragma unroll
                    for (int cx = 0; cx < 3; ++cx) atomicAdd(row + cx, __float2int_rn(wx.w[sxs][cx] * wyz));
                }
            }
        }
    }
    __syncthreads();
    const int4* a4 = reinterpret_cast<const int4*>(acc);
    // one 64-bit base for the box, 32-bit offsets inside its three grids (3 N < 2^26)
    float* fb = f + (size_t)box * 3 * (size_t)G.N;
    const int N32 = (int)G.N;
    const float unscale = 1.0f / scale;
    for (int i = threadIdx.x; i < 3 * SY * SZ * SXC; i += blockDim.x) {
        const int4 q = a4[i];
        if ((q.x | q.y | q.z | q.w) == 0) continue;
        const int row = i / SXC, cx = i - row * SXC;
        const int comp = row / (SY * SZ), rr = row - comp * (SY * SZ);
        const int sz = rr / SY, sy = rr - sz * SY;
        const int gx = (ox + 4 * cx) & (nx - 1), gy = (oy + sy) & (ny - 1), gz = (oz + sz) & (nz - 1);
        float* dst = fb + (comp * N32 + (gz * ny + gy) * nx + gx);
        atomicAdd(reinterpret_cast<float4*>(dst),
                  make_float4(q.x * unscale, q.y * unscale, q.z * unscale, q.w * unscale));
    }
}

// External forces to FP32 and their per-box FP64 sums (the exact net force: springs and
// repulsion cancel pairwise).  Grid (chunk of 256 blobs, box); one partial sum per block,
// reduced in a fixed order afterwards.
__global__ void __launch_bounds__(256)
k_ext_prepare(const int64_t* __restrict__ box_off, const double* __restrict__ ext,
              float4* __restrict__ e32, int nchunk, double* __restrict__ partial,
              double* __restrict__ ext_sum, unsigned* __restrict__ ticket)
{
    dep_wait();
    dep_release();
    __shared__ double sh[3][256];
    __shared__ bool last;
    const int box = blockIdx.y;
    const int64_t s0 = box_off[box], cnt = box_off[box + 1] - s0;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x;       // first blob of the chunk
    const int64_t local = first + threadIdx.x;
    // the chunk's 3 x 256 doubles read contiguously (the source may be host memory read over
    // the interconnect), then regrouped per blob through shared memory
    const int64_t nval = 3 * (cnt - first < (int64_t)blockDim.x ? cnt - first : (int64_t)blockDim.x);
    for (int k = 0; k < 3; ++k) {
        const int e = k * (int)blockDim.x + (int)threadIdx.x;
        (&sh[0][0])[e] = e < nval ? ext[3 * (s0 + first) + e] : 0.0;
    }
    __syncthreads();
    double v[3] = {0.0, 0.0, 0.0};
    if (local < cnt) {
        for (int d = 0; d < 3; ++d) v[d] = (&sh[0][0])[3 * threadIdx.x + d];
        e32[s0 + local] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 0; d < 3; ++d) {
        double x = v[d];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[d][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        partial[((int64_t)box * nchunk + blockIdx.x) * 3 + threadIdx.x] = t;
    }
    // the last block to finish (atomic ticket after a fence; no block waits) sums the partials
    // of every box in a fixed order and resets the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int bx = 0; bx < (int)gridDim.y; ++bx) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int c = threadIdx.x; c < nchunk; c += blockDim.x)
            for (int d = 0; d < 3; ++d) t[d] += __ldcg(partial + ((int64_t)bx * nchunk + c) * 3 + d);
        for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] = t[d];
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w)
                for (int d = 0; d < 3; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x < 3) ext_sum[3 * bx + threadIdx.x] = sh[threadIdx.x][0];
        __syncthreads();
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// vbar += scale * sum (mean_mode 0) or 0 (mean_mode 1), per box and component.
__global__ void k_vbar_step(int n, const double* __restrict__ sum, double scale, int mean_mode,
                            double* __restrict__ vbar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vbar[i] = mean_mode == 0 ? vbar[i] + (sum ? scale * sum[i] : 0.0) : 0.0;
}

__global__ void k_forces_to_fp64(int64_t nb, const float4* __restrict__ F, double* __restrict__ out)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const float4 f = F[b];
    out[3 * b] = f.x;
    out[3 * b + 1] = f.y;
    out[3 * b + 2] = f.z;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Blocks of `threads` for a for_warp_rounds kernel over n items: as many as the GPU holds at
// once (SMs x resident blocks of this kernel, found once per kernel and device), fewer when n
// is small.
template <typename K>
unsigned persistent_grid(K kernel, int threads, int64_t n)
{
    struct Entry {
        const void* k;
        int dev, threads, slots;
    };
    static Entry cache[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    int slots = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        int i = 0;
        for (; i < 64 && cache[i].k; ++i)
            if (cache[i].k == (const void*)kernel && cache[i].dev == dev &&
                cache[i].threads == threads) {
                slots = cache[i].slots;
                break;
            }
        if (slots == 0) {
            int sms = 0, per = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
            slots = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
            if (i < 64) cache[i] = Entry{(const void*)kernel, dev, threads, slots};
        }
    }
    const int64_t full = slots;
    const int64_t need = blocks_for(n, threads);
    return (unsigned)(need < full ? (need > 0 ? need : 1) : full);
}

}  // namespace

// ==========================================================================================
// Launchers.

cudaError_t launch_split(cudaStream_t st, int64_t nb, const double* q, const GridGeo& g,
                         const BinGeo& bg, float4* A, float4* B)
{
    if (nb <= 0) return cudaSuccess;
    k_split<<<blocks_for(nb, 256), 256, 0, st>>>(nb, q, g, bg, A, B);
    return cudaGetLastError();
}

cudaError_t launch_unsplit(cudaStream_t st, int64_t nb, const float4* A, const float4* B,
                           const GridGeo& g, const BinGeo& bg, double* q)
{
    if (nb <= 0) return cudaSuccess;
    k_unsplit<<<blocks_for(nb, 256), 256, 0, st>>>(nb, A, B, bg, g, q);
    return cudaGetLastError();
}

cudaError_t launch_interp32(cudaStream_t st, int mode, int64_t nb, const float4* A,
                            const float4* B, const float* v0, const float* v1,
                            const int32_t* box_of, const GridGeo& g, const BinGeo& bg, float dt,
                            const float4* A_base, const float4* B_base, float4* A_out,
                            float4* B_out, double* u_out, const int32_t* order,
                            int32_t* count, int32_t* blob_cell, int32_t* blob_rank)
{
    if (nb <= 0) return cudaSuccess;
    const unsigned nbk = blocks_for(nb, 256);
    if (mode == 0)
        k_interp32<0><<<nbk, 256, 0, st>>>(nb, A, B, v0, v1, box_of, g, bg, dt, A_base, B_base,
                                           A_out, B_out, u_out, order, nullptr, nullptr, nullptr);
    else if (mode == 1)
        k_interp32<1><<<nbk, 256, 0, st>>>(nb, A, B, v0, v1, box_of, g, bg, dt, A_base, B_base,
                                           A_out, B_out, u_out, order, count, blob_cell,
                                           blob_rank);
    else
        k_interp32<2><<<nbk, 256, 0, st>>>(nb, A, B, v0, v1, box_of, g, bg, dt, A_base, B_base,
                                           A_out, B_out, u_out, order, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_interp32_fused(cudaStream_t st, int64_t nb, const float4* A, const float* v0,
                                  const float* v1, const float* vp, const int32_t* box_of,
                                  const GridGeo& g,
                                  const BinGeo& bg, float dt, const float4* A_base,
                                  const float4* B_base, float4* A_out, float4* B_out,
                                  float4* Ah_out, float4* Bh_out, const int32_t* order,
                                  int32_t* count, int32_t* blob_cell, int32_t* blob_rank,
                                  float4* u_out)
{
    if (nb <= 0) return cudaSuccess;
    const FusedArgs f{A, v0, v1, vp, box_of, dt, A_base, B_base, A_out, B_out, Ah_out, Bh_out,
                      order, count, blob_cell, blob_rank, u_out};
    static std::atomic<unsigned> attr{0};
    if (first_on_device(attr))       // no shared memory: all of the SM's L1 for the gathers
        cudaFuncSetAttribute(k_interp32_fused, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    return launch_dep(k_interp32_fused, dim3(persistent_grid(k_interp32_fused, 256, nb)),
                      dim3(256), 0, st, nb, f, g, bg);
}

cudaError_t launch_bin32(cudaStream_t st, int64_t nb, const float4* A, const int32_t* box_of,
                         int Bx, const BinGeo& bg, int32_t* cell_count, int32_t* cell_start,
                         int32_t* blob_cell, int32_t* blob_rank, int32_t* sorted,
                         int32_t* scan_tmp, const int32_t* pid, float4* loc, bool counted)
{
    const int64_t ncells = (int64_t)Bx * bg.ncell;
    cudaError_t e = cudaSuccess;
    if (!counted) {
        e = cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * ncells, st);
        if (e != cudaSuccess) return e;
        if (nb > 0)
            k_bin_count32<<<blocks_for(nb, 256), 256, 0, st>>>(nb, A, box_of, bg, cell_count,
                                                               blob_cell, blob_rank);
    }
    // scan_tmp: [ntiles] tile offsets, then the ticket of the last-block scan (zero between
    // launches)
    const int ntiles = (int)((ncells + (1 << BIN_SCAN_LOG) - 1) >> BIN_SCAN_LOG);
    e = launch_dep(k_bin_scan32, dim3(ntiles), dim3(BIN_SCAN_THREADS), 0, st, cell_count,
                   ncells, scan_tmp, cell_start + ncells,
                   reinterpret_cast<unsigned*>(scan_tmp + ntiles));
    if (e != cudaSuccess) return e;
    const int64_t nthr = nb > ncells ? nb : ncells;
    return launch_dep(k_bin_place32, dim3(blocks_for(nthr, 256)), dim3(256), 0, st, nb, ncells,
                      (const int32_t*)cell_count, (const int32_t*)scan_tmp, cell_start,
                      (const int32_t*)blob_cell, (const int32_t*)blob_rank, sorted, A, pid, loc);
}

cudaError_t launch_forces32(cudaStream_t st, int Bx, int64_t nb, int64_t max_box_blobs,
                            const int64_t* box_off, const int32_t* sorted, const float4* A,
                            const float4* B, const float4* loc, const Springs32& sp,
                            const int32_t* box_of,
                            const float* box_par, const int32_t* cell_start,
                            const int32_t* blob_cell, const float4* ext, float4* Fs, float4* F,
                            float4* rec, const GridGeo& g, const BinGeo& bg)
{
    if (max_box_blobs <= 0) return cudaSuccess;
    cudaError_t e = launch_springs32(st, nb, A, B, sp, box_of, box_par, g, bg, Fs);
    if (e != cudaSuccess) return e;
    Force32Args a{box_off, sorted, A, B, loc, Fs, box_par, cell_start, blob_cell, ext, F, rec};
    dim3 grid(blocks_for(max_box_blobs, 256), (unsigned)Bx);
    return launch_dep(k_forces32, grid, dim3(256), 0, st, a, g, bg);
}

cudaError_t launch_springs32(cudaStream_t st, int64_t nb, const float4* A, const float4* B,
                             const Springs32& sp, const int32_t* box_of,
                             const float* box_par, const GridGeo& g, const BinGeo& bg, float4* Fs)
{
    if (nb <= 0) return cudaSuccess;
    if (sp.tmpl) {
        const int threads = (256 / sp.m) * sp.m;          // whole particles per block
        return launch_dep(k_springs32_shared, dim3(blocks_for(nb, threads)), dim3(threads),
                          sizeof(float) * 3 * threads * sp.slots, st, (int)nb, sp.m, sp.slots,
                          A, B, sp.tmpl, sp.tstart, box_of, box_par, g, bg, Fs);
    }
    cudaError_t e = cudaMemsetAsync(Fs, 0, sizeof(float4) * nb, st);
    if (e != cudaSuccess) return e;
    return launch_dep(k_springs32, dim3(blocks_for(nb, 256)), dim3(256), 0, st, nb, A, B, sp.adj,
                      sp.adj_start, box_of, box_par, g, bg, reinterpret_cast<float*>(Fs));
}

cudaError_t launch_pairs32(cudaStream_t st, int Bx, int64_t max_box_blobs,
                           const int64_t* box_off, const int32_t* sorted, const float4* A,
                           const float4* B, const float4* loc, const int32_t* box_of,
                           const float* box_par, const int32_t* cell_start,
                           const int32_t* blob_cell, const float4* ext, const float4* Fs,
                           float4* F, float4* rec, const GridGeo& g, const BinGeo& bg)
{
    (void)box_of;
    if (max_box_blobs <= 0) return cudaSuccess;
    Force32Args a{box_off, sorted, A, B, loc, Fs, box_par, cell_start, blob_cell, ext, F, rec};
    dim3 grid(blocks_for(max_box_blobs, 256), (unsigned)Bx);
    return launch_dep(k_forces32, grid, dim3(256), 0, st, a, g, bg);
}

// The shared copy (3 components, 16-byte chunks along x) and one force sum per bin cell.
size_t spread32_smem(const int tile[3], int bs)
{
    return (size_t)3 * (tile[0] + 8) * (tile[1] + 3) * (tile[2] + 3) * sizeof(float) +
           (size_t)(tile[0] / bs) * (tile[1] / bs) * (tile[2] / bs) * sizeof(float);
}

bool spread32_tile_ok(const int tile[3], const GridGeo& g, const BinGeo& bg)
{
    bool ok = spread32_smem(tile, bg.bs) <= 200 * 1024;
    for (int d = 0; d < 3; ++d)
        ok = ok && tile[d] >= 4 && tile[d] <= g.n[d] && g.n[d] % tile[d] == 0 && tile[d] % bg.bs == 0;
    return ok && (tile[1] / bg.bs) * (tile[2] / bg.bs) <= 64 && tile[0] / bg.bs <= 32;
}

template <int TX, int TY, int TZ>
cudaError_t launch_spread32_t(cudaStream_t st, int Bx, const float4* rec, const int32_t* cell_start,
                              const GridGeo& g, const BinGeo& bg, const int tile[3], float* f)
{
    const size_t smem = spread32_smem(tile, bg.bs);
    static std::atomic<unsigned> attr{0};
    if (first_on_device(attr))
        cudaFuncSetAttribute(k_spread32<TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    const int ntiles = (g.n[0] / tile[0]) * (g.n[1] / tile[1]) * (g.n[2] / tile[2]);
    return launch_dep(k_spread32<TX, TY, TZ>, dim3((unsigned)ntiles, (unsigned)Bx), dim3(256),
                      smem, st, rec, cell_start, g, bg, tile[0], tile[1], tile[2], f);
}

cudaError_t launch_spread32(cudaStream_t st, int Bx, const float4* rec, const int32_t* cell_start,
                            const GridGeo& g, const BinGeo& bg, const int tile[3], float* f,
                            bool f_is_zero)
{
    if (!spread32_tile_ok(tile, g, bg)) return cudaErrorInvalidValue;
    if (!f_is_zero) {
        const cudaError_t e = cudaMemsetAsync(f, 0, sizeof(float) * 3 * (size_t)Bx * g.N, st);
        if (e != cudaSuccess) return e;
    }
    const int a = tile[0], b = tile[1], c = tile[2];
    if (a == 32 && b == 8 && c == 8) return launch_spread32_t<32, 8, 8>(st, Bx, rec, cell_start, g, bg, tile, f);
    if (a == 16 && b == 8 && c == 8) return launch_spread32_t<16, 8, 8>(st, Bx, rec, cell_start, g, bg, tile, f);
    if (a == 32 && b == 16 && c == 8) return launch_spread32_t<32, 16, 8>(st, Bx, rec, cell_start, g, bg, tile, f);
    if (a == 16 && b == 16 && c == 8) return launch_spread32_t<16, 16, 8>(st, Bx, rec, cell_start, g, bg, tile, f);
    if (a == 64 && b == 8 && c == 8) return launch_spread32_t<64, 8, 8>(st, Bx, rec, cell_start, g, bg, tile, f);
    return launch_spread32_t<0, 0, 0>(st, Bx, rec, cell_start, g, bg, tile, f);
}

cudaError_t launch_ext_prepare(cudaStream_t st, int Bx, int64_t max_box_blobs,
                               const int64_t* box_off, const double* ext, float4* ext32,
                               double* partial, double* ext_sum, unsigned* ticket)
{
    const int nchunk = (int)((max_box_blobs + 255) / 256);
    if (nchunk <= 0) return cudaMemsetAsync(ext_sum, 0, sizeof(double) * 3 * Bx, st);
    return launch_dep(k_ext_prepare, dim3((unsigned)nchunk, (unsigned)Bx), dim3(256), 0, st,
                      box_off, ext, ext32, nchunk, partial, ext_sum, ticket);
}

cudaError_t launch_vbar_step(cudaStream_t st, int Bx, const double* sum, double scale,
                             int mean_mode, double* vbar)
{
    k_vbar_step<<<blocks_for(3 * Bx, 128), 128, 0, st>>>(3 * Bx, sum, scale, mean_mode, vbar);
    return cudaGetLastError();
}

cudaError_t launch_forces_to_fp64(cudaStream_t st, int64_t nb, const float4* F, double* out)
{
    if (nb <= 0) return cudaSuccess;
    k_forces_to_fp64<<<blocks_for(nb, 256), 256, 0, st>>>(nb, F, out);
    return cudaGetLastError();
}

}  // namespace mbk
