// C ABI of libmb.so: context management, argument validation, host/device staging and the
// orchestration of one inertial-coupling step (see include/mb.h for the contract).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "mb_internal.cuh"
#include "peskin.cuh"

using namespace mbk;

bool mbk::pdl_enabled()
{
    static const bool on = [] {
        const char* e = std::getenv("MB_PDL");
        return !(e && std::atoi(e) == 0);
    }();
    return on;
}

namespace {

constexpr int SYM_LEN = 256;   // per-dimension symbol table length (n <= 128 today)

// Stages of one step, in launch order (names returned by mb_stage_name).
enum Stage {
    ST_INTERP_PREDICT, ST_BIN, ST_FORCES, ST_FORCE_SUM, ST_SPREAD, ST_STRESS, ST_FLUID_X_FWD,
    ST_FLUID_Y_FWD, ST_FLUID_Z_SOLVE, ST_FLUID_Y_INV, ST_FLUID_X_INV, ST_INTERP_CORRECT,
    NUM_STAGES
};
const char* const STAGE_NAMES[NUM_STAGES] = {
    "interp_predict", "bin", "forces", "force_sum", "spread", "fluid_stress", "fluid_x_fwd",
    "fluid_y_fwd",
    "fluid_z_solve", "fluid_y_inv", "fluid_x_inv", "interp_correct"};

thread_local std::string g_create_error;

// Host-side fault injection: MB_FAULT_ALLOC=k makes the k-th device allocation of the
// process fail as if the device were out of memory (tests of the MB_ENOMEM path).
long g_alloc_counter = 0;
bool injected_alloc_failure()
{
    static long k = [] {
        const char* s = std::getenv("MB_FAULT_ALLOC");
        return s ? std::atol(s) : 0L;
    }();
    ++g_alloc_counter;
    return k > 0 && g_alloc_counter == k;
}

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

cudaError_t dfree(DBuf& b)
{
    cudaError_t e = cudaSuccess;
    if (b.p) e = cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    return e;
}

// Ensures b holds at least `bytes`; contents are not preserved.  Returns MB_ENOMEM/MB_ECUDA.
mb_status ensure(DBuf& b, size_t bytes, std::string& err, const char* what)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return MB_OK;
    dfree(b);
    if (injected_alloc_failure()) {
        err = std::string("injected allocation failure for ") + what;
        return MB_ENOMEM;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        err = std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) +
              " bytes): " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? MB_ENOMEM : MB_ECUDA;
    }
    b.bytes = bytes;
    return MB_OK;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (readable and writable by kernels over the
// interconnect), or null for any other pointer.
void* mapped_host_ptr(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

struct BoxData {
    bool set = false;
    std::vector<double> pos;
    std::vector<int32_t> pid;
    std::vector<int32_t> bonds;
    std::vector<double> rest;
    int64_t np = 0;
    double k_spring = 0.0, k_rep = 0.0, r_cut = 0.0;
};

}  // namespace

struct mb_ctx {
    mb_grid_desc d{};
    cudaStream_t st = nullptr;
    int device = 0;
    GridGeo g{};
    BinGeo bg{};
    int B = 1;
    size_t rsz = 4;           // bytes per grid real
    int nxh = 0;
    int tile[3] = {8, 8, 8};

    DBuf v[2], vsum, f, spec, vbar, fsum, tw[3], twf[3], sym, symr, body_prof, prof_scratch;
    DBuf twk[3], symk;          // FP64 grids: twiddles and symbols in double-float
    // thermal stress (kT > 0): sigma~ of the current step [B][9][N] and the step index that
    // keys its random numbers (device memory, advanced by the step itself)
    bool thermal = false;
    double thermal_amp = 0.0;
    DBuf W, step_index;
    bool advect = false;        // the convective stress rho v v (explicit at v^n)
    int fft_passes = 3;     // 3: plane/z/plane pipeline; 5: one pass per axis (reference layout)
    int cur = 0;
    int64_t steps_taken = 0;
    double body_cached[4] = {0, 0, 0, 0};
    bool body_valid = false;

    std::vector<BoxData> boxes;
    bool dirty = true;
    int64_t nb = 0, np = 0, max_box_blobs = 0;
    int nchunk = 0;
    std::vector<int64_t> box_off_h, part_off_h;
    std::vector<float> box_par32_h;                // float copy of the box parameters
    DBuf q, qh, u, F, rec, ext, pid, box_of, adj_start, adj_j, adj_rest, part_start,
        part_blobs, box_off, box_par, cell_count, cell_start, blob_cell, blob_rank, sorted,
        loc, scan_tmp, partial, staging_in, staging_out, mean_scratch;
    // FP32-grid mode blob state: positions as bin cell + float-float offset (q^n and midpoint)
    DBuf sA, sB, hA[2], hB[2], F32, rec32, ext32, ext_sum, ext_ticket, adj32, adj32_start, Fs32, u32;
    // the bond pattern common to all particles (tmpl_m blobs each), when there is one
    DBuf tmpl32, tstart32;
    int tmpl_m = 0, tmpl_slots = 0;
    DBuf Fpre64;        // FP64 grids: external + spring forces of the pattern kernel [nb][3]
    // split midpoints: hA/hB[hcur] hold the predictor of the next step when pred_ready (the
    // previous step's fused corrector wrote them); hlast is the buffer of the last step's
    // midpoints (where its forces were evaluated)
    int hcur = 0, hlast = 0;
    bool pred_ready = false;
    bool fuse_interp = true;
    bool f_zero = false;        // ctx->f holds zeros (cleared by the last plane pass)

    bool ext_present = false;
    bool sorted_valid = false;     // `sorted` holds a permutation of the current blobs
    // spreading tile picked by timing candidate shapes on the first FP32-grid step
    bool autotune = true, tuned = false;
    float tile_ms = 0.f;
    // CUDA graphs of one FP32-grid step, one per velocity-buffer parity
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;
    // second stream for the spring forces, which overlap the binning (fork/join events)
    cudaStream_t side = nullptr;
    // fork[0] step start, [1] springs done, [2] stress drawn, [3] external forces converted,
    // [4] blobs binned, [5] bin counts cleared for the next step's predictor
    cudaEvent_t fork[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // a second side stream: the conversion of a single-step call's external forces
    cudaStream_t side2 = nullptr;
    // device-readable external forces of the current single-step call, converted inside the
    // step beside the binning (null: ext32 already holds them or there are none)
    const double* ext_src = nullptr;
    const double* graph_ext_src[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    bool graph_ext[2] = {false, false}, graph_body[2] = {false, false};
    int graph_hcur[2] = {0, 0};
    bool graph_fz[2] = {false, false};
    int64_t graph_launches = 0;        // kernels per graph launch
    // adjoint scratch: blob vectors and grids (FP64 contexts)
    DBuf a_qn, a_u, a_qh, a_gq, a_guc, a_gqh, a_gF, a_gu, a_gk, a_gU;
    DBuf a_vn, a_vp, a_w, a_gw, a_gvp, a_gvn, a_gf, a_tmp, a_zero;
    // standalone-operator scratch
    DBuf s_q, s_F, s_rec, s_cell_count, s_cell_start, s_blob_cell, s_blob_rank, s_sorted,
        s_scan, s_u, s_g0, s_g1, s_g2, s_out;

    // stage timing (CUDA events on the context stream) and kernel launch count
    bool timing = false;
    static constexpr int EV_RING = 64;             // steps recorded before a forced readback
    std::vector<cudaEvent_t> ev_ring;              // EV_RING sets of NUM_STAGES + 1 events
    int ev_pending = 0;
    cudaEvent_t* ev = nullptr;                     // the set used by the current step
    double stage_ms[NUM_STAGES] = {};
    int64_t stage_calls[NUM_STAGES] = {};
    int64_t launches = 0;

    std::string err;
};

namespace {

#define MB_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            cudaGetLastError();                                                           \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return MB_ECUDA;                                                              \
        }                                                                                 \
    } while (0)

#define MB_TRY(expr)                                                                      \
    do {                                                                                  \
        mb_status s_ = (expr);                                                            \
        if (s_ != MB_OK) return s_;                                                       \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); ok = false; }
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

mb_status invalid(mb_ctx* ctx, const std::string& msg)
{
    ctx->err = msg;
    return MB_EINVAL;
}

size_t grid_bytes(const mb_ctx* ctx, int boxes) { return (size_t)boxes * 3 * ctx->g.N * ctx->rsz; }

// Copies an input array to the device if it lives in host memory.
mb_status stage_in(mb_ctx* ctx, const void* p, size_t bytes, DBuf& buf, const void** out,
                   const char* what)
{
    if (is_device_ptr(p)) {
        *out = p;
        return MB_OK;
    }
    MB_TRY(ensure(buf, bytes, ctx->err, what));
    MB_CUDA(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, ctx->st));
    *out = buf.p;
    return MB_OK;
}

// Device destination for an output: the caller's pointer, or a staging buffer.
mb_status out_target(mb_ctx* ctx, void* p, size_t bytes, DBuf& buf, void** dev, bool* host,
                     const char* what)
{
    if (is_device_ptr(p)) {
        *dev = p;
        *host = false;
        return MB_OK;
    }
    MB_TRY(ensure(buf, bytes, ctx->err, what));
    *dev = buf.p;
    *host = true;
    return MB_OK;
}

mb_status finish_out(mb_ctx* ctx, void* p, const void* dev, size_t bytes, bool host)
{
    if (!host) return MB_OK;
    MB_CUDA(cudaMemcpyAsync(p, dev, bytes, cudaMemcpyDeviceToHost, ctx->st));
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    return MB_OK;
}

mb_status copy_to_host(mb_ctx* ctx, const void* p, size_t bytes, void* hostbuf)
{
    if (bytes == 0) return MB_OK;
    if (is_device_ptr(p)) {
        MB_CUDA(cudaMemcpyAsync(hostbuf, p, bytes, cudaMemcpyDeviceToHost, ctx->st));
        MB_CUDA(cudaStreamSynchronize(ctx->st));
    } else {
        std::memcpy(hostbuf, p, bytes);
    }
    return MB_OK;
}

double wrap_host(double x, double L)
{
    double y = std::fmod(x, L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

__global__ void k_wrap(int64_t n, double* q, double L0, double L1, double L2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int d = (int)(i % 3);
    const double L = d == 0 ? L0 : (d == 1 ? L1 : L2);
    double y = fmod(q[i], L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    q[i] = y;
}

// MB_SPRINGS=list keeps the per-blob bond lists even where all particles share one pattern.
bool springs_per_blob()
{
    static const bool on = [] {
        const char* e = std::getenv("MB_SPRINGS");
        return e && std::string(e) == "list";
    }();
    return on;
}

// The box parameters [B][3] rounded to float, stored after the doubles.
const float* box_par32(const mb_ctx* ctx)
{
    return reinterpret_cast<const float*>(static_cast<const double*>(ctx->box_par.p) + 3 * ctx->B);
}

// The bonds of the FP32 spring kernels: the per-blob lists, and the common pattern if any.
Springs32 springs32(const mb_ctx* ctx)
{
    const bool t = ctx->tmpl_m > 0 && !springs_per_blob();
    return Springs32{static_cast<const int4*>(ctx->adj32.p),
                     static_cast<const int32_t*>(ctx->adj32_start.p),
                     t ? static_cast<const int4*>(ctx->tmpl32.p) : nullptr,
                     t ? static_cast<const int32_t*>(ctx->tstart32.p) : nullptr, ctx->tmpl_m,
                     ctx->tmpl_slots};
}

// Choose the bin cell side: a power of two of mesh cells, at least 2 and at least r_cut.
void choose_bins(mb_ctx* ctx, double r_cut)
{
    int bs = 2;
    while (bs * ctx->d.h < r_cut) bs *= 2;
    const int nmin = std::min(ctx->g.n[0], std::min(ctx->g.n[1], ctx->g.n[2]));
    if (bs > nmin) bs = nmin;
    ctx->bg.bs = bs;
    for (int a = 0; a < 3; ++a) ctx->bg.nc[a] = ctx->g.n[a] / bs;
    ctx->bg.ncell = (int64_t)ctx->bg.nc[0] * ctx->bg.nc[1] * ctx->bg.nc[2];
    ctx->bg.inv_w = 1.0 / (bs * ctx->d.h);
    set_float_geo(ctx->bg);
}

// Default spreading tile: {32, 8, 8} nodes, clamped to the grid and raised to whole bin cells.
void pick_tile(mb_ctx* ctx)
{
    const int want[3] = {32, 8, 8};
    for (int d = 0; d < 3; ++d)
        ctx->tile[d] = std::min(std::max(std::min(want[d], ctx->g.n[d]), ctx->bg.bs), ctx->g.n[d]);
}

void drop_graph(mb_ctx* ctx)
{
    for (cudaGraphExec_t& g : ctx->graph_exec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Concatenates the boxes' blobs into the device arrays used by the step.
mb_status rebuild(mb_ctx* ctx)
{
    drop_graph(ctx);
    const int B = ctx->B;
    ctx->box_off_h.assign(B + 1, 0);
    ctx->part_off_h.assign(B + 1, 0);
    double rmax = 0.0;
    for (int b = 0; b < B; ++b) {
        const BoxData& bx = ctx->boxes[b];
        ctx->box_off_h[b + 1] = ctx->box_off_h[b] + (int64_t)bx.pid.size();
        ctx->part_off_h[b + 1] = ctx->part_off_h[b] + bx.np;
        if (bx.k_rep != 0.0) rmax = std::max(rmax, bx.r_cut);
    }
    const int64_t nb = ctx->box_off_h[B], np = ctx->part_off_h[B];
    ctx->nb = nb;
    ctx->np = np;
    ctx->max_box_blobs = 0;
    for (int b = 0; b < B; ++b)
        ctx->max_box_blobs = std::max(ctx->max_box_blobs, ctx->box_off_h[b + 1] - ctx->box_off_h[b]);
    ctx->nchunk = (int)((ctx->max_box_blobs + 255) / 256);
    choose_bins(ctx, rmax);
    pick_tile(ctx);

    std::vector<double> q(3 * nb), par(3 * B);
    std::vector<int32_t> pid(nb), box_of(nb), adj_start(nb + 1, 0), part_start(np + 1, 0),
        part_blobs(nb);
    std::vector<int64_t> off(ctx->box_off_h);
    int64_t nadj = 0;
    for (int b = 0; b < B; ++b) nadj += 2 * (int64_t)(ctx->boxes[b].rest.size());
    std::vector<int32_t> adj_j(nadj);
    std::vector<double> adj_rest(nadj);
    for (int b = 0; b < B; ++b) {
        const BoxData& bx = ctx->boxes[b];
        const int64_t o = ctx->box_off_h[b];
        const int64_t n = (int64_t)bx.pid.size();
        for (int64_t i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a) q[3 * (o + i) + a] = wrap_host(bx.pos[3 * i + a], ctx->g.L[a]);
            pid[o + i] = (int32_t)(ctx->part_off_h[b] + bx.pid[i]);
            box_of[o + i] = b;
        }
        for (size_t e = 0; e < bx.rest.size(); ++e) {
            adj_start[o + bx.bonds[2 * e] + 1]++;
            adj_start[o + bx.bonds[2 * e + 1] + 1]++;
        }
        par[3 * b] = bx.k_spring;
        par[3 * b + 1] = bx.k_rep;
        par[3 * b + 2] = bx.r_cut;
    }
    for (int64_t i = 0; i < nb; ++i) adj_start[i + 1] += adj_start[i];
    {
        std::vector<int32_t> fill(adj_start.begin(), adj_start.end() - 1);
        for (int b = 0; b < B; ++b) {
            const BoxData& bx = ctx->boxes[b];
            const int64_t o = ctx->box_off_h[b];
            for (size_t e = 0; e < bx.rest.size(); ++e) {
                const int64_t i = o + bx.bonds[2 * e], j = o + bx.bonds[2 * e + 1];
                adj_j[fill[i]] = (int32_t)j;
                adj_rest[fill[i]++] = bx.rest[e];
                adj_j[fill[j]] = (int32_t)i;
                adj_rest[fill[j]++] = bx.rest[e];
            }
        }
    }
    for (int64_t i = 0; i < nb; ++i) part_start[pid[i] + 1]++;
    for (int64_t p = 0; p < np; ++p) part_start[p + 1] += part_start[p];
    {
        std::vector<int32_t> fill(part_start.begin(), part_start.end() - 1);
        for (int64_t i = 0; i < nb; ++i) part_blobs[fill[pid[i]]++] = (int32_t)i;
    }

    const int64_t ncells = (int64_t)B * ctx->bg.ncell;
    std::string& E = ctx->err;
    MB_TRY(ensure(ctx->q, sizeof(double) * 3 * nb, E, "q"));
    MB_TRY(ensure(ctx->qh, sizeof(double) * 3 * nb, E, "q_half"));
    MB_TRY(ensure(ctx->u, sizeof(double) * 3 * nb, E, "u"));
    MB_TRY(ensure(ctx->F, sizeof(double) * 3 * nb, E, "F"));
    MB_TRY(ensure(ctx->rec, sizeof(double) * 6 * nb, E, "rec"));
    MB_TRY(ensure(ctx->ext, sizeof(double) * 3 * nb, E, "ext"));
    MB_TRY(ensure(ctx->pid, sizeof(int32_t) * nb, E, "pid"));
    MB_TRY(ensure(ctx->box_of, sizeof(int32_t) * nb, E, "box_of"));
    MB_TRY(ensure(ctx->adj_start, sizeof(int32_t) * (nb + 1), E, "adj_start"));
    MB_TRY(ensure(ctx->adj_j, sizeof(int32_t) * nadj, E, "adj_j"));
    MB_TRY(ensure(ctx->adj_rest, sizeof(double) * nadj, E, "adj_rest"));
    MB_TRY(ensure(ctx->part_start, sizeof(int32_t) * (np + 1), E, "part_start"));
    MB_TRY(ensure(ctx->part_blobs, sizeof(int32_t) * nb, E, "part_blobs"));
    MB_TRY(ensure(ctx->box_off, sizeof(int64_t) * (B + 1), E, "box_off"));
    // [B][3] doubles, then the same rounded to float for the FP32 blob kernels
    MB_TRY(ensure(ctx->box_par, (sizeof(double) + sizeof(float)) * 3 * B, E, "box_par"));
    MB_TRY(ensure(ctx->cell_count, sizeof(int32_t) * ncells, E, "cell_count"));
    MB_TRY(ensure(ctx->cell_start, sizeof(int32_t) * (ncells + 1), E, "cell_start"));
    MB_TRY(ensure(ctx->blob_cell, sizeof(int32_t) * nb, E, "blob_cell"));
    MB_TRY(ensure(ctx->blob_rank, sizeof(int32_t) * nb, E, "blob_rank"));
    MB_TRY(ensure(ctx->sorted, sizeof(int32_t) * nb, E, "sorted"));
    MB_TRY(ensure(ctx->loc, sizeof(float4) * nb, E, "loc"));
    MB_TRY(ensure(ctx->scan_tmp, sizeof(int32_t) * (ncells / 4096 + 2), E, "scan_tmp"));
    // the FP32 binning keeps a zero ticket after its tile offsets
    MB_CUDA(cudaMemsetAsync(ctx->scan_tmp.p, 0, sizeof(int32_t) * (ncells / 4096 + 2), ctx->st));
    MB_TRY(ensure(ctx->partial, sizeof(double) * 3 * B * std::max(ctx->nchunk, 1), E, "partial"));

    cudaStream_t st = ctx->st;
    auto up = [&](DBuf& d, const void* h, size_t bytes) -> mb_status {
        if (bytes) MB_CUDA(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, st));
        return MB_OK;
    };
    MB_TRY(up(ctx->q, q.data(), sizeof(double) * 3 * nb));
    MB_TRY(up(ctx->pid, pid.data(), sizeof(int32_t) * nb));
    MB_TRY(up(ctx->box_of, box_of.data(), sizeof(int32_t) * nb));
    MB_TRY(up(ctx->adj_start, adj_start.data(), sizeof(int32_t) * (nb + 1)));
    MB_TRY(up(ctx->adj_j, adj_j.data(), sizeof(int32_t) * nadj));
    MB_TRY(up(ctx->adj_rest, adj_rest.data(), sizeof(double) * nadj));
    MB_TRY(up(ctx->part_start, part_start.data(), sizeof(int32_t) * (np + 1)));
    MB_TRY(up(ctx->part_blobs, part_blobs.data(), sizeof(int32_t) * nb));
    MB_TRY(up(ctx->box_off, off.data(), sizeof(int64_t) * (B + 1)));
    MB_TRY(up(ctx->box_par, par.data(), sizeof(double) * 3 * B));
    ctx->box_par32_h.assign(par.begin(), par.end());
    MB_CUDA(cudaMemcpyAsync(static_cast<double*>(ctx->box_par.p) + 3 * B, ctx->box_par32_h.data(),
                            sizeof(float) * 3 * B, cudaMemcpyHostToDevice, st));
    // One bond pattern shared by every particle: m blobs each, blob l of particle p numbered
    // p m + l, the same partners (as offsets inside the particle) and the same rest lengths,
    // compared exactly.  The pattern is then stored once and every bond evaluated once, by the
    // end that owner[] names, into slot[] of that end: the light end of a bond to a blob of
    // more than SPRING_LOCAL_MAX bonds, otherwise the end with fewer evaluations so far (the
    // lower index on a tie), so that no blob evaluates many more than the mean.  owner[] and
    // slot[] are per adjacency entry of particle 0 (both entries of a bond alike).
    ctx->tmpl_m = 0;
    ctx->tmpl_slots = 0;
    std::vector<int32_t> owner, slot;
    int64_t pm = 0;
    if (np > 0 && nb % np == 0 && nb / np <= 64) {
        const int64_t m = nb / np;
        auto heavy = [&](int64_t i) { return adj_start[i + 1] - adj_start[i] > SPRING_LOCAL_MAX; };
        bool same = true;
        for (int64_t i = 0; i < nb && same; ++i) same = pid[i] == (int32_t)(i / m);
        for (int64_t i = 0; i < nb && same; ++i) {
            const int64_t l = i % m, base = i - l;
            const int32_t cnt = adj_start[i + 1] - adj_start[i];
            same = cnt == adj_start[l + 1] - adj_start[l];
            for (int32_t k = 0; k < cnt && same; ++k) {
                const int64_t e = adj_start[i] + k, e0 = adj_start[l] + k;
                const int64_t off = adj_j[e] - base;
                same = off >= 0 && off < m && off == adj_j[e0] &&
                       std::memcmp(&adj_rest[e], &adj_rest[e0], sizeof(double)) == 0;
            }
        }
        if (same) {
            owner.assign(adj_start[m], -1);
            slot.assign(adj_start[m], -1);
            std::vector<int> nslot(m, 0);
            for (int64_t l = 0; l < m; ++l) {
                for (int32_t e = adj_start[l]; e < adj_start[l + 1]; ++e) {
                    const int64_t j = adj_j[e];
                    if (j < l) continue;                  // met from its lower end
                    // the matching entry at j: the same occurrence of l among j's partners
                    int occ = 0;
                    for (int32_t f = adj_start[l]; f < e; ++f) occ += adj_j[f] == j;
                    int32_t er = -1;
                    for (int32_t f = adj_start[j]; f < adj_start[j + 1] && er < 0; ++f)
                        if (adj_j[f] == l && occ-- == 0) er = f;
                    const bool hl = heavy(l), hj = heavy(j);
                    const int64_t x = hl && !hj ? j
                                      : (hj && !hl ? l : (nslot[l] <= nslot[j] ? l : j));
                    const int sl = nslot[x]++;
                    owner[e] = (int32_t)x;
                    slot[e] = sl;
                    if (er >= 0) {
                        owner[er] = (int32_t)x;
                        slot[er] = sl;
                    }
                }
            }
            pm = m;
            ctx->tmpl_m = (int)m;
            ctx->tmpl_slots = *std::max_element(nslot.begin(), nslot.end());
        }
    }
    // the pattern's tables: FP32 grids (k_springs32_shared) per local blob its evaluations
    // {offset | (slot + 1) << 16, r0, r0^2 hi, lo} and the slots it collects {offset, slot};
    // FP64 grids (k_springs64) its evaluations {offset | (slot + 1) << 16, r0 low, r0 high} and
    // its whole adjacency in order {offset of the evaluating blob, slot, sign}
    if (pm > 0) {
        std::vector<int32_t> t_start(2 * pm + 1, 0), t;
        for (int64_t l = 0; l < pm; ++l) {
            for (int32_t e = adj_start[l]; e < adj_start[l + 1]; ++e) {
                if (owner[e] != l) continue;
                const int64_t j = adj_j[e];
                const double r0 = adj_rest[e];
                int32_t w[4];
                w[0] = (int32_t)(((uint32_t)(j - l) & 0xffffu) | ((uint32_t)(slot[e] + 1) << 16));
                if (ctx->rsz == 4) {
                    const double r0sq = r0 * r0;
                    const float h = (float)r0sq, lo = (float)(r0sq - (double)h), rf = (float)r0;
                    std::memcpy(&w[1], &rf, 4);
                    std::memcpy(&w[2], &h, 4);
                    std::memcpy(&w[3], &lo, 4);
                } else {
                    std::memcpy(&w[1], &r0, 8);            // low word, then high word
                    w[3] = 0;
                }
                t.insert(t.end(), w, w + 4);
            }
            t_start[2 * l + 1] = (int32_t)(t.size() / 4);
            for (int32_t e = adj_start[l]; e < adj_start[l + 1]; ++e) {
                if (ctx->rsz == 4 && owner[e] == l) continue;
                const int32_t w[4] = {(int32_t)(owner[e] - l), slot[e], owner[e] == l ? 1 : -1, 0};
                t.insert(t.end(), w, w + 4);
            }
            t_start[2 * l + 2] = (int32_t)(t.size() / 4);
        }
        MB_TRY(ensure(ctx->tmpl32, sizeof(int32_t) * std::max<size_t>(t.size(), 4), E,
                      "bond pattern"));
        MB_TRY(ensure(ctx->tstart32, sizeof(int32_t) * (2 * pm + 1), E, "bond pattern"));
        MB_TRY(up(ctx->tmpl32, t.data(), sizeof(int32_t) * t.size()));
        MB_TRY(up(ctx->tstart32, t_start.data(), sizeof(int32_t) * (2 * pm + 1)));
        if (ctx->rsz == 8) MB_TRY(ensure(ctx->Fpre64, sizeof(double) * 3 * nb, E, "spring forces"));
    }
    if (ctx->rsz == 4) {
        MB_TRY(ensure(ctx->sA, sizeof(float4) * nb, E, "split q"));
        MB_TRY(ensure(ctx->sB, sizeof(float4) * nb, E, "split q"));
        for (int i = 0; i < 2; ++i) {
            MB_TRY(ensure(ctx->hA[i], sizeof(float4) * nb, E, "split q_half"));
            MB_TRY(ensure(ctx->hB[i], sizeof(float4) * nb, E, "split q_half"));
        }
        MB_TRY(ensure(ctx->F32, sizeof(float4) * nb, E, "F32"));
        MB_TRY(ensure(ctx->rec32, 2 * sizeof(float4) * nb, E, "rec32"));
        MB_TRY(ensure(ctx->ext32, sizeof(float4) * nb, E, "ext32"));
        MB_TRY(ensure(ctx->ext_sum, sizeof(double) * 3 * B, E, "ext_sum"));
        MB_TRY(ensure(ctx->ext_ticket, sizeof(unsigned), E, "ext ticket"));
        MB_CUDA(cudaMemsetAsync(ctx->ext_ticket.p, 0, sizeof(unsigned), ctx->st));
        // FP32 springs: a bond with one end of more than SPRING_LOCAL_MAX bonds (an
        // icosahedron's centre) is evaluated once, by its other end, which also adds the
        // opposite force to the heavy end; every other bond is evaluated at both ends.  So no
        // thread of a warp iterates over more than SPRING_LOCAL_MAX + its owned bonds.
        auto heavy = [&](int64_t i) { return adj_start[i + 1] - adj_start[i] > SPRING_LOCAL_MAX; };
        std::vector<int32_t> s32(nb + 1, 0);
        std::vector<int32_t> a32;
        a32.reserve(4 * nadj);
        for (int64_t i = 0; i < nb; ++i) {
            for (int32_t e = adj_start[i]; e < adj_start[i + 1]; ++e) {
                const int64_t j = adj_j[e];
                const bool hi = heavy(i), hj = heavy(j);
                if (hi && !hj) continue;                   // j evaluates this bond
                const bool owned = hj && !hi;              // i adds the force to j as well
                const double r0 = adj_rest[e], r0sq = r0 * r0;
                const float h = (float)r0sq, l = (float)(r0sq - (double)h), rf = (float)r0;
                int32_t w[4];
                w[0] = (int32_t)((uint32_t)j | (owned ? 0x80000000u : 0u));
                std::memcpy(&w[1], &rf, 4);
                std::memcpy(&w[2], &h, 4);
                std::memcpy(&w[3], &l, 4);
                a32.insert(a32.end(), w, w + 4);
            }
            s32[i + 1] = (int32_t)(a32.size() / 4);
        }
        MB_TRY(ensure(ctx->adj32, sizeof(int32_t) * std::max<size_t>(a32.size(), 4), E, "adj32"));
        MB_TRY(ensure(ctx->adj32_start, sizeof(int32_t) * (nb + 1), E, "adj32_start"));
        MB_TRY(ensure(ctx->Fs32, sizeof(float4) * nb, E, "spring forces"));
        MB_TRY(ensure(ctx->u32, sizeof(float4) * nb, E, "blob velocities"));
        MB_TRY(up(ctx->adj32, a32.data(), sizeof(int32_t) * a32.size()));
        MB_TRY(up(ctx->adj32_start, s32.data(), sizeof(int32_t) * (nb + 1)));
        MB_CUDA(launch_split(st, nb, static_cast<const double*>(ctx->q.p), ctx->g, ctx->bg,
                             static_cast<float4*>(ctx->sA.p), static_cast<float4*>(ctx->sB.p)));
        ctx->ext_present = false;
        ctx->sorted_valid = false;
        ctx->pred_ready = false;
        ctx->tuned = false;
    }
    // the host vectors die at return: make the copies complete first
    MB_CUDA(cudaStreamSynchronize(st));
    ctx->dirty = false;
    return MB_OK;
}

mb_status ensure_ready(mb_ctx* ctx)
{
    for (int b = 0; b < ctx->B; ++b)
        if (!ctx->boxes[b].set) {
            ctx->err = "box " + std::to_string(b) + " has no particles set (call mb_set_particles)";
            return MB_ESTATE;
        }
    if (ctx->dirty) return rebuild(ctx);
    return MB_OK;
}

// Body-force profile along wave_dir on the component `axis`'s nodes (host sin, FP64).
mb_status set_body(mb_ctx* ctx, const double* body, DBuf& target, bool use_cache)
{
    const double f0 = body[0], axis = body[1], dir = body[2], j = body[3];
    if (!std::isfinite(f0) || !std::isfinite(j) || (axis != 0 && axis != 1 && axis != 2) ||
        (dir != 0 && dir != 1 && dir != 2))
        return invalid(ctx, "body_force must be {f0, axis in 0..2, wave_dir in 0..2, j} with finite f0, j");
    if (use_cache && ctx->body_valid && std::memcmp(ctx->body_cached, body, sizeof(double) * 4) == 0)
        return MB_OK;
    const int ax = (int)axis, wd = (int)dir;
    const int n = ctx->g.n[wd];
    const double L = ctx->g.L[wd];
    const double shift = ax == wd ? 0.0 : 0.5;
    std::vector<double> pd(n);
    std::vector<float> pf(n);
    for (int i = 0; i < n; ++i) {
        pd[i] = f0 * std::sin(2.0 * M_PI * j * ((double)i + shift) * ctx->d.h / L);
        pf[i] = (float)pd[i];
    }
    MB_TRY(ensure(target, sizeof(double) * n, ctx->err, "body profile"));
    const void* src = ctx->rsz == 8 ? (const void*)pd.data() : (const void*)pf.data();
    MB_CUDA(cudaMemcpyAsync(target.p, src, ctx->rsz * n, cudaMemcpyHostToDevice, ctx->st));
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    if (use_cache) {
        std::memcpy(ctx->body_cached, body, sizeof(double) * 4);
        ctx->body_valid = true;
    }
    return MB_OK;
}

template <typename R>
FluidArgs<R> fluid_args(mb_ctx* ctx, const void* v, const void* f, void* v_out,
                        const void* prof, const double* body, const double* mean_override)
{
    FluidArgs<R> a{};
    a.v = static_cast<const R*>(v);
    a.f = static_cast<const R*>(f);
    a.spec = static_cast<typename C2<R>::T*>(ctx->spec.p);
    a.v_out = static_cast<R*>(v_out);
    for (int d = 0; d < 3; ++d) {
        a.tw[d] = static_cast<const R*>(ctx->tw[d].p);
        a.twf[d] = static_cast<const R*>(ctx->twf[d].p);
    }
    a.sym = static_cast<const double*>(ctx->sym.p);
    a.symr = ctx->symr.p;
    for (int d = 0; d < 3; ++d) a.twk[d] = ctx->rsz == 8 ? ctx->twk[d].p : ctx->twf[d].p;
    a.symk = ctx->rsz == 8 ? ctx->symk.p : ctx->symr.p;
    a.body_prof = body ? static_cast<const R*>(prof) : nullptr;
    a.body_axis = body ? (int)body[1] : -1;
    a.body_dir = body ? (int)body[2] : 0;
    a.mean_override = mean_override;
    a.mean_mode = ctx->d.mean_mode;
    a.rho_dt = ctx->d.rho / ctx->d.dt;
    a.half_eta = 0.5 * ctx->d.eta;
    return a;
}

// Accumulates the stage times of every recorded step (waits for the last one).
mb_status drain_stage_events(mb_ctx* ctx)
{
    if (ctx->ev_pending == 0) return MB_OK;
    cudaEvent_t* last = ctx->ev_ring.data() + (size_t)(ctx->ev_pending - 1) * (NUM_STAGES + 1);
    MB_CUDA(cudaEventSynchronize(last[NUM_STAGES]));
    for (int s = 0; s < ctx->ev_pending; ++s) {
        cudaEvent_t* e = ctx->ev_ring.data() + (size_t)s * (NUM_STAGES + 1);
        for (int i = 0; i < NUM_STAGES; ++i) {
            float ms = 0.f;
            MB_CUDA(cudaEventElapsedTime(&ms, e[i], e[i + 1]));
            ctx->stage_ms[i] += ms;
            ctx->stage_calls[i] += 1;
        }
    }
    ctx->ev_pending = 0;
    return MB_OK;
}

// One time step of every box (see mb_step in include/mb.h).
// FP64-mode spreading by blob-owner global atomics (MB_SPREAD64=tile keeps the tile-owner
// shared-memory kernel).
bool spread_atomic64()
{
    static const bool on = [] {
        const char* e = std::getenv("MB_SPREAD64");
        return !(e && std::string(e) == "tile");
    }();
    return on;
}

template <typename R>
mb_status do_step(mb_ctx* ctx, const double* ext, const double* body)
{
    cudaStream_t st = ctx->st;
    const GridGeo& g = ctx->g;
    const int B = ctx->B;
    R* vcur = static_cast<R*>(ctx->v[ctx->cur].p);
    R* vnext = static_cast<R*>(ctx->v[ctx->cur ^ 1].p);
    double* q = static_cast<double*>(ctx->q.p);
    double* qh = static_cast<double*>(ctx->qh.p);
    const int32_t* box_of = static_cast<const int32_t*>(ctx->box_of.p);
    const bool blobs = ctx->nb > 0;
    if (ctx->timing) {
        if (ctx->ev_pending == mb_ctx::EV_RING) MB_TRY(drain_stage_events(ctx));
        ctx->ev = ctx->ev_ring.data() + (size_t)ctx->ev_pending * (NUM_STAGES + 1);
    }
    auto mark = [&](int i) { if (ctx->timing) cudaEventRecord(ctx->ev[i], st); };
    mark(ST_INTERP_PREDICT);
    if (blobs) {
        // u^n = J(q^n) v^n ; q^{n+1/2} = q^n + dt/2 u^n
        MB_CUDA(launch_interp<R>(st, 1, ctx->nb, q, nullptr, vcur, nullptr, box_of, g,
                                 ctx->d.dt, nullptr, qh));
        ctx->launches += 1;
    }
    // FP64 grid, one bond pattern for all particles: the springs once per bond, summed with
    // the external forces in the per-blob order (the same bits); without stage timing on the
    // side stream, beside the binning
    const bool pattern = blobs && ctx->rsz == 8 && ctx->tmpl_m > 0 && !springs_per_blob();
    auto springs64 = [&](cudaStream_t s2) {
        return launch_springs64(s2, ctx->nb, ctx->tmpl_m, ctx->tmpl_slots, qh, ext,
                                static_cast<const int4*>(ctx->tmpl32.p),
                                static_cast<const int32_t*>(ctx->tstart32.p), box_of,
                                static_cast<const double*>(ctx->box_par.p), g,
                                static_cast<double*>(ctx->Fpre64.p));
    };
    const bool side64 = pattern && !ctx->timing;
    if (side64) {
        MB_CUDA(cudaEventRecord(ctx->fork[0], st));
        MB_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork[0], 0));
        MB_CUDA(springs64(ctx->side));
        MB_CUDA(cudaEventRecord(ctx->fork[1], ctx->side));
        ctx->launches += 1;
    }
    mark(ST_BIN);
    if (blobs) {
        MB_CUDA(launch_bin(st, ctx->nb, qh, box_of, B, ctx->bg,
                           static_cast<int32_t*>(ctx->cell_count.p),
                           static_cast<int32_t*>(ctx->cell_start.p),
                           static_cast<int32_t*>(ctx->blob_cell.p),
                           static_cast<int32_t*>(ctx->blob_rank.p),
                           static_cast<int32_t*>(ctx->sorted.p),
                           static_cast<int32_t*>(ctx->scan_tmp.p), ctx->d.deterministic != 0,
                           static_cast<const int32_t*>(ctx->pid.p),
                           static_cast<float4*>(ctx->loc.p)));
        ctx->launches += 5 + 2 * (ctx->d.deterministic != 0);
    }
    mark(ST_FORCES);
    if (blobs) {
        if (side64) {
            MB_CUDA(cudaStreamWaitEvent(st, ctx->fork[1], 0));
        } else if (pattern) {
            MB_CUDA(springs64(st));
            ctx->launches += 1;
        }
        ForceArgs fa{};
        fa.Fpre = pattern ? static_cast<const double*>(ctx->Fpre64.p) : nullptr;
        fa.box_off = static_cast<const int64_t*>(ctx->box_off.p);
        fa.sorted = static_cast<const int32_t*>(ctx->sorted.p);
        fa.q = qh;
        fa.pid = static_cast<const int32_t*>(ctx->pid.p);
        fa.adj_start = static_cast<const int32_t*>(ctx->adj_start.p);
        fa.adj_j = static_cast<const int32_t*>(ctx->adj_j.p);
        fa.adj_rest = static_cast<const double*>(ctx->adj_rest.p);
        fa.box_par = static_cast<const double*>(ctx->box_par.p);
        fa.cell_start = static_cast<const int32_t*>(ctx->cell_start.p);
        fa.blob_cell = static_cast<const int32_t*>(ctx->blob_cell.p);
        fa.ext = ext;
        fa.loc = static_cast<const float4*>(ctx->loc.p);
        fa.F = static_cast<double*>(ctx->F.p);
        fa.rec = static_cast<double*>(ctx->rec.p);
        fa.partial = static_cast<double*>(ctx->partial.p);
        fa.nchunk = ctx->nchunk;
        MB_CUDA(launch_forces(st, B, ctx->max_box_blobs, fa, g, ctx->bg, ctx->rsz == 8));
        ctx->launches += 1;
    }
    mark(ST_FORCE_SUM);
    if (blobs) {
        const double L3 = g.L[0] * g.L[1] * g.L[2];
        MB_CUDA(launch_force_sum(st, B, ctx->nchunk, static_cast<const double*>(ctx->partial.p),
                                 static_cast<double*>(ctx->vbar.p),
                                 ctx->d.dt / (ctx->d.rho * L3), ctx->d.mean_mode,
                                 static_cast<double*>(ctx->fsum.p)));
        ctx->launches += 1;
    }
    mark(ST_SPREAD);
    if (blobs) {
        if (ctx->d.deterministic && sizeof(R) == 8)
            MB_CUDA(launch_spread_det(st, B, static_cast<const double*>(ctx->rec.p),
                                      static_cast<const int32_t*>(ctx->cell_start.p), g, ctx->bg,
                                      ctx->tile, reinterpret_cast<double*>(ctx->f.p)));
        else if (spread_atomic64())
            MB_CUDA(launch_spread_atomic<R>(st, B, ctx->max_box_blobs,
                                            static_cast<const double*>(ctx->rec.p),
                                            static_cast<const int32_t*>(ctx->cell_start.p), g,
                                            ctx->bg, static_cast<R*>(ctx->f.p)));
        else
            MB_CUDA(launch_spread<R>(st, B, static_cast<const double*>(ctx->rec.p),
                                     static_cast<const int32_t*>(ctx->cell_start.p), g, ctx->bg,
                                     ctx->tile, static_cast<R*>(ctx->f.p)));
        ctx->launches += 1;
    }
    mark(ST_STRESS);
    const bool stress = ctx->thermal || ctx->advect;
    if (stress) {
        MB_CUDA(launch_fluid_stress<R>(st, B, g, ctx->d.seed,
                                       static_cast<uint64_t*>(ctx->step_index.p),
                                       ctx->thermal_amp, ctx->advect ? vcur : nullptr,
                                       ctx->d.rho, static_cast<R*>(ctx->W.p),
                                       static_cast<R*>(ctx->f.p), blobs));
        ctx->launches += STRESS_KERNELS;
    }
    const double* mean = ctx->d.mean_mode == 0 ? static_cast<const double*>(ctx->vbar.p) : nullptr;
    FluidArgs<R> fa = fluid_args<R>(ctx, vcur, blobs || stress ? ctx->f.p : nullptr, vnext,
                                    ctx->body_prof.p, body, mean);
    cudaEvent_t* fm = ctx->timing ? ctx->ev + ST_FLUID_X_FWD : nullptr;
    if (ctx->fft_passes == 5) {
        MB_CUDA(launch_fluid<R>(st, B, g, fa, fm));
        ctx->launches += FLUID_KERNELS;
    } else {
        MB_CUDA(launch_fluid3<R>(st, B, g, fa, fm));
        ctx->launches += FLUID3_KERNELS;
    }
    if (blobs) {
        // q^{n+1} = q^n + dt J(q^{n+1/2}) (v^n + v^{n+1})/2
        MB_CUDA(launch_interp<R>(st, 2, ctx->nb, qh, q, vcur, vnext, box_of, g, ctx->d.dt,
                                 nullptr, q));
        ctx->launches += 1;
    }
    mark(NUM_STAGES);
    if (ctx->timing) ctx->ev_pending++;
    ctx->cur ^= 1;
    ctx->steps_taken++;
    return MB_OK;
}

// One Stokes-limit step of every box (integrator 1), FP64 blob positions in either grid
// precision: two half steps, each binning the blobs, computing their forces, spreading them and
// solving the steady zero-mean Stokes flow v = P (-eta L)^{-1} (S F + f_body) (the three-pass
// FFT with the right-hand side f alone and the divide by eta lambda); then
// q^{n+1/2} = q^n + dt/2 J(q^n) v(q^n) and q^{n+1} = q^n + dt J(q^{n+1/2}) v(q^{n+1/2}).
template <typename R>
mb_status do_step_stokes(mb_ctx* ctx, const double* ext, const double* body)
{
    cudaStream_t st = ctx->st;
    const GridGeo& g = ctx->g;
    const int B = ctx->B;
    R* v_half = static_cast<R*>(ctx->v[ctx->cur ^ 1].p);
    R* v_full = static_cast<R*>(ctx->v[ctx->cur].p);
    double* q = static_cast<double*>(ctx->q.p);
    double* qh = static_cast<double*>(ctx->qh.p);
    const int32_t* box_of = static_cast<const int32_t*>(ctx->box_of.p);
    const bool blobs = ctx->nb > 0;
    if (ctx->timing) {
        if (ctx->ev_pending == mb_ctx::EV_RING) MB_TRY(drain_stage_events(ctx));
        ctx->ev = ctx->ev_ring.data() + (size_t)ctx->ev_pending * (NUM_STAGES + 1);
    }
    auto mark = [&](int i) { if (ctx->timing) cudaEventRecord(ctx->ev[i], st); };
    // forces at x into ctx->f, then the Stokes flow into v_out (stage marks on the second half)
    auto half = [&](const double* x, R* v_out, bool marks) -> mb_status {
        if (marks) mark(ST_BIN);
        if (blobs) {
            MB_CUDA(launch_bin(st, ctx->nb, x, box_of, B, ctx->bg,
                               static_cast<int32_t*>(ctx->cell_count.p),
                               static_cast<int32_t*>(ctx->cell_start.p),
                               static_cast<int32_t*>(ctx->blob_cell.p),
                               static_cast<int32_t*>(ctx->blob_rank.p),
                               static_cast<int32_t*>(ctx->sorted.p),
                               static_cast<int32_t*>(ctx->scan_tmp.p), ctx->d.deterministic != 0,
                               static_cast<const int32_t*>(ctx->pid.p),
                               static_cast<float4*>(ctx->loc.p)));
            ctx->launches += 5 + 2 * (ctx->d.deterministic != 0);
        }
        if (marks) mark(ST_FORCES);
        if (blobs) {
            ForceArgs fa{};
            fa.box_off = static_cast<const int64_t*>(ctx->box_off.p);
            fa.sorted = static_cast<const int32_t*>(ctx->sorted.p);
            fa.q = x;
            fa.pid = static_cast<const int32_t*>(ctx->pid.p);
            fa.adj_start = static_cast<const int32_t*>(ctx->adj_start.p);
            fa.adj_j = static_cast<const int32_t*>(ctx->adj_j.p);
            fa.adj_rest = static_cast<const double*>(ctx->adj_rest.p);
            fa.box_par = static_cast<const double*>(ctx->box_par.p);
            fa.cell_start = static_cast<const int32_t*>(ctx->cell_start.p);
            fa.blob_cell = static_cast<const int32_t*>(ctx->blob_cell.p);
            fa.ext = ext;
            fa.loc = static_cast<const float4*>(ctx->loc.p);
            fa.F = static_cast<double*>(ctx->F.p);
            fa.rec = static_cast<double*>(ctx->rec.p);
            fa.partial = static_cast<double*>(ctx->partial.p);
            fa.nchunk = ctx->nchunk;
            MB_CUDA(launch_forces(st, B, ctx->max_box_blobs, fa, g, ctx->bg, ctx->rsz == 8));
            ctx->launches += 1;
        }
        if (marks) mark(ST_FORCE_SUM);
        if (marks) mark(ST_SPREAD);
        if (blobs) {
            if (ctx->d.deterministic && sizeof(R) == 8)
                MB_CUDA(launch_spread_det(st, B, static_cast<const double*>(ctx->rec.p),
                                          static_cast<const int32_t*>(ctx->cell_start.p), g,
                                          ctx->bg, ctx->tile, reinterpret_cast<double*>(ctx->f.p)));
            else
                MB_CUDA(launch_spread<R>(st, B, static_cast<const double*>(ctx->rec.p),
                                         static_cast<const int32_t*>(ctx->cell_start.p), g,
                                         ctx->bg, ctx->tile, static_cast<R*>(ctx->f.p)));
            ctx->launches += 1;
        }
        if (marks) mark(ST_STRESS);        // no thermal or convective stress in this integrator
        FluidArgs<R> fa = fluid_args<R>(ctx, v_out, blobs ? ctx->f.p : nullptr, v_out,
                                        ctx->body_prof.p, body, nullptr);
        fa.no_v = 1;                        // right-hand side S F + f_body
        fa.rho_dt = 0.0;                    // divide by eta lambda: steady Stokes
        fa.half_eta = ctx->d.eta;
        fa.mean_mode = 1;
        cudaEvent_t* fm = marks && ctx->timing ? ctx->ev + ST_FLUID_X_FWD : nullptr;
        if (ctx->fft_passes == 5) {
            MB_CUDA(launch_fluid<R>(st, B, g, fa, fm));
            ctx->launches += FLUID_KERNELS;
        } else {
            MB_CUDA(launch_fluid3<R>(st, B, g, fa, fm));
            ctx->launches += FLUID3_KERNELS;
        }
        return MB_OK;
    };
    mark(ST_INTERP_PREDICT);
    MB_TRY(half(q, v_half, false));
    if (blobs) {
        // q^{n+1/2} = q^n + dt/2 J(q^n) v(q^n)
        MB_CUDA(launch_interp<R>(st, 1, ctx->nb, q, nullptr, v_half, nullptr, box_of, g,
                                 ctx->d.dt, nullptr, qh));
        ctx->launches += 1;
    }
    MB_TRY(half(qh, v_full, true));
    if (blobs) {
        // q^{n+1} = q^n + dt J(q^{n+1/2}) v(q^{n+1/2})  (the mean of a field with itself)
        MB_CUDA(launch_interp<R>(st, 2, ctx->nb, qh, q, v_full, v_full, box_of, g, ctx->d.dt,
                                 nullptr, q));
        ctx->launches += 1;
    }
    mark(NUM_STAGES);
    if (ctx->timing) ctx->ev_pending++;
    ctx->steps_taken++;
    return MB_OK;
}

// One time step of every box in FP32-grid mode: blob positions as bin cell + float-float
// offset, forces and weights on the FP32 pipes, the k = 0 mode from the FP64 external force sum.
// Host-side state after an FP32-grid step has been enqueued (directly or as a graph replay).
void finish_fast_step(mb_ctx* ctx)
{
    ctx->cur ^= 1;
    ctx->steps_taken++;
    ctx->hlast = ctx->hcur;
    if (ctx->nb > 0) ctx->f_zero = ctx->fft_passes == 3;     // the plane pass cleared f
    if (ctx->nb > 0 && ctx->fuse_interp) {
        ctx->hcur ^= 1;
        ctx->pred_ready = true;
    } else {
        ctx->pred_ready = false;
    }
}

mb_status do_step_fast(mb_ctx* ctx, bool ext, const double* body)
{
    cudaStream_t st = ctx->st;
    const GridGeo& g = ctx->g;
    const int B = ctx->B;
    float* vcur = static_cast<float*>(ctx->v[ctx->cur].p);
    float* vnext = static_cast<float*>(ctx->v[ctx->cur ^ 1].p);
    float4* sA = static_cast<float4*>(ctx->sA.p);
    float4* sB = static_cast<float4*>(ctx->sB.p);
    float4* hA = static_cast<float4*>(ctx->hA[ctx->hcur].p);
    float4* hB = static_cast<float4*>(ctx->hB[ctx->hcur].p);
    const int32_t* box_of = static_cast<const int32_t*>(ctx->box_of.p);
    const bool blobs = ctx->nb > 0;
    if (ctx->timing) {
        if (ctx->ev_pending == mb_ctx::EV_RING) MB_TRY(drain_stage_events(ctx));
        ctx->ev = ctx->ev_ring.data() + (size_t)ctx->ev_pending * (NUM_STAGES + 1);
    }
    auto mark = [&](int i) { if (ctx->timing) cudaEventRecord(ctx->ev[i], st); };
    const float dt = (float)ctx->d.dt;
    mark(ST_INTERP_PREDICT);
    if (blobs && !ctx->pred_ready) {
        // the predictor also bins the midpoint positions (counts per cell); the previous
        // step's cell order still groups neighbouring blobs
        MB_CUDA(cudaMemsetAsync(ctx->cell_count.p, 0, sizeof(int32_t) * B * ctx->bg.ncell, st));
        MB_CUDA(launch_interp32(st, 1, ctx->nb, sA, sB, vcur, nullptr, box_of, g, ctx->bg, dt,
                                nullptr, nullptr, hA, hB, nullptr,
                                ctx->sorted_valid ? static_cast<const int32_t*>(ctx->sorted.p)
                                                  : nullptr,
                                static_cast<int32_t*>(ctx->cell_count.p),
                                static_cast<int32_t*>(ctx->blob_cell.p),
                                static_cast<int32_t*>(ctx->blob_rank.p)));
        ctx->launches += 1;
    }
    // the spring forces need only the midpoint positions: without stage timing they run on a
    // second stream while the blobs are binned (fork/join events, also inside captured graphs)
    const bool overlap = blobs && !ctx->timing;
    // a single-step call's external forces (read from the caller's array, possibly page-locked
    // host memory over the interconnect) are converted on a third stream beside the binning and
    // the springs; they are first needed by the repulsion pass
    auto ext_prepare = [&](cudaStream_t s2) {
        return launch_ext_prepare(s2, B, ctx->max_box_blobs,
                                  static_cast<const int64_t*>(ctx->box_off.p), ctx->ext_src,
                                  static_cast<float4*>(ctx->ext32.p),
                                  static_cast<double*>(ctx->partial.p),
                                  static_cast<double*>(ctx->ext_sum.p),
                                  static_cast<unsigned*>(ctx->ext_ticket.p));
    };
    const bool ext_in_step = blobs && ctx->ext_src != nullptr;
    if (ext_in_step && !overlap) {
        MB_CUDA(ext_prepare(st));
        ctx->launches += 1;
    }
    if (overlap) {
        MB_CUDA(cudaEventRecord(ctx->fork[0], st));
        if (ext_in_step) {
            MB_CUDA(cudaStreamWaitEvent(ctx->side2, ctx->fork[0], 0));
            MB_CUDA(ext_prepare(ctx->side2));
            MB_CUDA(cudaEventRecord(ctx->fork[3], ctx->side2));
            ctx->launches += 1;
        }
        MB_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork[0], 0));
        MB_CUDA(launch_springs32(ctx->side, ctx->nb, hA, hB, springs32(ctx), box_of,
                                 box_par32(ctx), g, ctx->bg,
                                 static_cast<float4*>(ctx->Fs32.p)));
        MB_CUDA(cudaEventRecord(ctx->fork[1], ctx->side));
        // the thermal / convective stress needs only the step index and v^n: it is drawn on the
        // side stream too, behind the springs, while the blobs are binned, forced and spread
        if (ctx->thermal || ctx->advect) {
            MB_CUDA(launch_fluid_stress<float>(ctx->side, B, g, ctx->d.seed,
                                               static_cast<uint64_t*>(ctx->step_index.p),
                                               ctx->thermal_amp, ctx->advect ? vcur : nullptr,
                                               ctx->d.rho, static_cast<float*>(ctx->W.p),
                                               static_cast<float*>(ctx->f.p), blobs, 1));
            MB_CUDA(cudaEventRecord(ctx->fork[2], ctx->side));
        }
    }
    mark(ST_BIN);
    if (blobs) {
        MB_CUDA(launch_bin32(st, ctx->nb, hA, box_of, B, ctx->bg,
                             static_cast<int32_t*>(ctx->cell_count.p),
                             static_cast<int32_t*>(ctx->cell_start.p),
                             static_cast<int32_t*>(ctx->blob_cell.p),
                             static_cast<int32_t*>(ctx->blob_rank.p),
                             static_cast<int32_t*>(ctx->sorted.p),
                             static_cast<int32_t*>(ctx->scan_tmp.p),
                             static_cast<const int32_t*>(ctx->pid.p),
                             static_cast<float4*>(ctx->loc.p), true));
        ctx->launches += 2;
        ctx->sorted_valid = true;
    }
    // the fused corrector pass counts the next step's midpoints into cell_count, which the
    // placement has now read: with the side stream it is cleared there, off the step's chain of
    // kernels (whose launches may then overlap one another's first and last blocks)
    const bool clear_side = overlap && ctx->fuse_interp;
    if (clear_side) {
        MB_CUDA(cudaEventRecord(ctx->fork[4], st));
        MB_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork[4], 0));
        MB_CUDA(cudaMemsetAsync(ctx->cell_count.p, 0, sizeof(int32_t) * B * ctx->bg.ncell,
                                ctx->side));
        MB_CUDA(cudaEventRecord(ctx->fork[5], ctx->side));
    }
    mark(ST_FORCES);
    if (blobs) {
        const int64_t* box_off = static_cast<const int64_t*>(ctx->box_off.p);
        const float4* ext4 = ext ? static_cast<const float4*>(ctx->ext32.p) : nullptr;
        if (overlap) {
            MB_CUDA(cudaStreamWaitEvent(st, ctx->fork[1], 0));
            if (ext_in_step) MB_CUDA(cudaStreamWaitEvent(st, ctx->fork[3], 0));
            MB_CUDA(launch_pairs32(st, B, ctx->max_box_blobs, box_off,
                                   static_cast<const int32_t*>(ctx->sorted.p), hA, hB,
                                   static_cast<const float4*>(ctx->loc.p), box_of,
                                   box_par32(ctx),
                                   static_cast<const int32_t*>(ctx->cell_start.p),
                                   static_cast<const int32_t*>(ctx->blob_cell.p), ext4,
                                   static_cast<float4*>(ctx->Fs32.p),
                                   static_cast<float4*>(ctx->F32.p),
                                   static_cast<float4*>(ctx->rec32.p), g, ctx->bg));
        } else {
            MB_CUDA(launch_forces32(st, B, ctx->nb, ctx->max_box_blobs, box_off,
                                    static_cast<const int32_t*>(ctx->sorted.p), hA, hB,
                                    static_cast<const float4*>(ctx->loc.p), springs32(ctx),
                                    box_of,
                                    box_par32(ctx),
                                    static_cast<const int32_t*>(ctx->cell_start.p),
                                    static_cast<const int32_t*>(ctx->blob_cell.p), ext4,
                                    static_cast<float4*>(ctx->Fs32.p),
                                    static_cast<float4*>(ctx->F32.p),
                                    static_cast<float4*>(ctx->rec32.p), g, ctx->bg));
        }
        ctx->launches += 2;
    }
    mark(ST_FORCE_SUM);                 // the mean momentum advances inside the z pass
    mark(ST_SPREAD);
    if (blobs) {
        MB_CUDA(launch_spread32(st, B, static_cast<const float4*>(ctx->rec32.p),
                                static_cast<const int32_t*>(ctx->cell_start.p), g, ctx->bg,
                                ctx->tile, static_cast<float*>(ctx->f.p), ctx->f_zero));
        ctx->launches += 1;
    }
    mark(ST_STRESS);
    const bool stress = ctx->thermal || ctx->advect;
    if (stress) {
        if (overlap) MB_CUDA(cudaStreamWaitEvent(st, ctx->fork[2], 0));
        MB_CUDA(launch_fluid_stress<float>(st, B, g, ctx->d.seed,
                                           static_cast<uint64_t*>(ctx->step_index.p),
                                           ctx->thermal_amp, ctx->advect ? vcur : nullptr,
                                           ctx->d.rho, static_cast<float*>(ctx->W.p),
                                           static_cast<float*>(ctx->f.p), blobs,
                                           overlap ? 2 : 3));
        ctx->launches += STRESS_KERNELS;
    }
    FluidArgs<float> fa = fluid_args<float>(ctx, vcur, blobs || stress ? ctx->f.p : nullptr,
                                            vnext, ctx->body_prof.p, body, nullptr);
    if (ctx->d.mean_mode == 0) {
        const double L3 = g.L[0] * g.L[1] * g.L[2];
        if (ctx->fft_passes == 3) {
            fa.mean_state = static_cast<double*>(ctx->vbar.p);
            fa.mean_force = ext ? static_cast<const double*>(ctx->ext_sum.p) : nullptr;
            fa.mean_scale = ctx->d.dt / (ctx->d.rho * L3);
        } else {
            MB_CUDA(launch_vbar_step(st, B, ext ? static_cast<const double*>(ctx->ext_sum.p) : nullptr,
                                     ctx->d.dt / (ctx->d.rho * L3), 0,
                                     static_cast<double*>(ctx->vbar.p)));
            ctx->launches += 1;
            fa.mean_override = static_cast<const double*>(ctx->vbar.p);
        }
    }
    if (blobs && ctx->fft_passes == 3) fa.f_clear = static_cast<float*>(ctx->f.p);
    const bool vsum = blobs && ctx->fuse_interp && ctx->fft_passes == 3;
    if (vsum) {
        fa.v_sum_base = vcur;
        fa.v_sum_out = static_cast<float*>(ctx->vsum.p);
    }
    cudaEvent_t* fm = ctx->timing ? ctx->ev + ST_FLUID_X_FWD : nullptr;
    if (ctx->fft_passes == 5) {
        MB_CUDA(launch_fluid<float>(st, B, g, fa, fm));
        ctx->launches += FLUID_KERNELS;
    } else {
        MB_CUDA(launch_fluid3<float>(st, B, g, fa, fm));
        ctx->launches += FLUID3_KERNELS;
    }
    if (blobs) {
        if (ctx->fuse_interp) {
            // corrector of this step and predictor of the next (into the other midpoint buffer,
            // with the bin counts the next step sorts by)
            if (clear_side) MB_CUDA(cudaStreamWaitEvent(st, ctx->fork[5], 0));
            else MB_CUDA(cudaMemsetAsync(ctx->cell_count.p, 0, sizeof(int32_t) * B * ctx->bg.ncell, st));
            MB_CUDA(launch_interp32_fused(st, ctx->nb, hA, vsum ? static_cast<const float*>(ctx->vsum.p) : vcur,
                                          vsum ? nullptr : vnext, vnext, box_of, g, ctx->bg, dt, sA,
                                          sB, sA, sB,
                                          static_cast<float4*>(ctx->hA[ctx->hcur ^ 1].p),
                                          static_cast<float4*>(ctx->hB[ctx->hcur ^ 1].p),
                                          static_cast<const int32_t*>(ctx->sorted.p),
                                          static_cast<int32_t*>(ctx->cell_count.p),
                                          static_cast<int32_t*>(ctx->blob_cell.p),
                                          static_cast<int32_t*>(ctx->blob_rank.p),
                                          static_cast<float4*>(ctx->u32.p)));
        } else {
            MB_CUDA(launch_interp32(st, 2, ctx->nb, hA, hB, vcur, vnext, box_of, g, ctx->bg, dt,
                                    sA, sB, sA, sB, nullptr,
                                    static_cast<const int32_t*>(ctx->sorted.p)));
        }
        ctx->launches += 1;
    }
    mark(NUM_STAGES);
    if (ctx->timing) ctx->ev_pending++;
    return MB_OK;
}

// One Stokes-limit step in FP32-grid mode (integrator 1, precision 0): the steps of
// do_step_stokes on the split blob positions of the FP32 path (float-float offsets from bin
// cells, FP32 forces, fixed-point shared-memory spreading).  Forces, spreading and the steady
// solve at q^n give the flow v(q^n); the predictor pass moves the blobs to
// q^{n+1/2} = q^n + dt/2 J v(q^n) and counts them into bins; forces, spreading and the solve at
// q^{n+1/2} give v(q^{n+1/2}), and the corrector pass sets q^{n+1} = q^n + dt J v(q^{n+1/2}).
mb_status do_step_stokes_fast(mb_ctx* ctx, bool ext, const double* body)
{
    cudaStream_t st = ctx->st;
    const GridGeo& g = ctx->g;
    const int B = ctx->B;
    float* v_half = static_cast<float*>(ctx->v[ctx->cur ^ 1].p);
    float* v_full = static_cast<float*>(ctx->v[ctx->cur].p);
    float4* sA = static_cast<float4*>(ctx->sA.p);
    float4* sB = static_cast<float4*>(ctx->sB.p);
    float4* hA = static_cast<float4*>(ctx->hA[0].p);
    float4* hB = static_cast<float4*>(ctx->hB[0].p);
    const int32_t* box_of = static_cast<const int32_t*>(ctx->box_of.p);
    const bool blobs = ctx->nb > 0;
    if (ctx->timing) {
        if (ctx->ev_pending == mb_ctx::EV_RING) MB_TRY(drain_stage_events(ctx));
        ctx->ev = ctx->ev_ring.data() + (size_t)ctx->ev_pending * (NUM_STAGES + 1);
    }
    auto mark = [&](int i) { if (ctx->timing) cudaEventRecord(ctx->ev[i], st); };
    const float dt = (float)ctx->d.dt;
    // forces at (A, B) (binned already when `counted`), spreading, steady flow into v_out
    auto half = [&](const float4* A, const float4* Bp, bool counted, float* v_out,
                    bool marks) -> mb_status {
        if (marks) mark(ST_BIN);
        if (blobs) {
            MB_CUDA(launch_bin32(st, ctx->nb, A, box_of, B, ctx->bg,
                                 static_cast<int32_t*>(ctx->cell_count.p),
                                 static_cast<int32_t*>(ctx->cell_start.p),
                                 static_cast<int32_t*>(ctx->blob_cell.p),
                                 static_cast<int32_t*>(ctx->blob_rank.p),
                                 static_cast<int32_t*>(ctx->sorted.p),
                                 static_cast<int32_t*>(ctx->scan_tmp.p),
                                 static_cast<const int32_t*>(ctx->pid.p),
                                 static_cast<float4*>(ctx->loc.p), counted));
            ctx->launches += counted ? 2 : 3;
            ctx->sorted_valid = true;
        }
        if (marks) mark(ST_FORCES);
        if (blobs) {
            MB_CUDA(launch_forces32(st, B, ctx->nb, ctx->max_box_blobs,
                                    static_cast<const int64_t*>(ctx->box_off.p),
                                    static_cast<const int32_t*>(ctx->sorted.p), A, Bp,
                                    static_cast<const float4*>(ctx->loc.p), springs32(ctx),
                                    box_of,
                                    box_par32(ctx),
                                    static_cast<const int32_t*>(ctx->cell_start.p),
                                    static_cast<const int32_t*>(ctx->blob_cell.p),
                                    ext ? static_cast<const float4*>(ctx->ext32.p) : nullptr,
                                    static_cast<float4*>(ctx->Fs32.p),
                                    static_cast<float4*>(ctx->F32.p),
                                    static_cast<float4*>(ctx->rec32.p), g, ctx->bg));
            ctx->launches += 2;
        }
        if (marks) mark(ST_FORCE_SUM);
        if (marks) mark(ST_SPREAD);
        if (blobs) {
            MB_CUDA(launch_spread32(st, B, static_cast<const float4*>(ctx->rec32.p),
                                    static_cast<const int32_t*>(ctx->cell_start.p), g, ctx->bg,
                                    ctx->tile, static_cast<float*>(ctx->f.p), false));
            ctx->launches += 1;
        }
        if (marks) mark(ST_STRESS);
        FluidArgs<float> fa = fluid_args<float>(ctx, v_out, blobs ? ctx->f.p : nullptr, v_out,
                                                ctx->body_prof.p, body, nullptr);
        fa.no_v = 1;
        fa.rho_dt = 0.0;
        fa.half_eta = ctx->d.eta;
        fa.mean_mode = 1;
        cudaEvent_t* fm = marks && ctx->timing ? ctx->ev + ST_FLUID_X_FWD : nullptr;
        if (ctx->fft_passes == 5) {
            MB_CUDA(launch_fluid<float>(st, B, g, fa, fm));
            ctx->launches += FLUID_KERNELS;
        } else {
            MB_CUDA(launch_fluid3<float>(st, B, g, fa, fm));
            ctx->launches += FLUID3_KERNELS;
        }
        return MB_OK;
    };
    mark(ST_INTERP_PREDICT);
    MB_TRY(half(sA, sB, false, v_half, false));
    if (blobs) {
        // q^{n+1/2} = q^n + dt/2 J(q^n) v(q^n), binned on the way
        MB_CUDA(cudaMemsetAsync(ctx->cell_count.p, 0, sizeof(int32_t) * B * ctx->bg.ncell, st));
        MB_CUDA(launch_interp32(st, 1, ctx->nb, sA, sB, v_half, nullptr, box_of, g, ctx->bg, dt,
                                nullptr, nullptr, hA, hB, nullptr,
                                static_cast<const int32_t*>(ctx->sorted.p),
                                static_cast<int32_t*>(ctx->cell_count.p),
                                static_cast<int32_t*>(ctx->blob_cell.p),
                                static_cast<int32_t*>(ctx->blob_rank.p)));
        ctx->launches += 1;
    }
    MB_TRY(half(hA, hB, true, v_full, true));
    if (blobs) {
        // q^{n+1} = q^n + dt J(q^{n+1/2}) v(q^{n+1/2})  (the mean of a field with itself)
        MB_CUDA(launch_interp32(st, 2, ctx->nb, hA, hB, v_full, v_full, box_of, g, ctx->bg, dt,
                                sA, sB, sA, sB, nullptr,
                                static_cast<const int32_t*>(ctx->sorted.p)));
        ctx->launches += 1;
    }
    mark(NUM_STAGES);
    if (ctx->timing) ctx->ev_pending++;
    ctx->hcur = 0;
    ctx->hlast = 0;
    ctx->pred_ready = false;
    ctx->f_zero = false;
    ctx->steps_taken++;
    return MB_OK;
}

// Times each candidate spreading tile on the current binned records (the first step after
// the blobs were set) and keeps the fastest; choices are cached per geometry and blob count.
struct TuneKey {
    int n[3], B, bs;
    int64_t nb;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(n[0], n[1], n[2], B, bs, nb) < std::tie(o.n[0], o.n[1], o.n[2], o.B, o.bs, o.nb);
    }
};
std::map<TuneKey, std::array<int, 3>> g_tile_cache;
std::mutex g_tile_mu;

mb_status autotune_spread(mb_ctx* ctx)
{
    ctx->tuned = true;
    if (!ctx->autotune || ctx->nb == 0) return MB_OK;
    const TuneKey key{{ctx->g.n[0], ctx->g.n[1], ctx->g.n[2]}, ctx->B, ctx->bg.bs, ctx->nb};
    {
        std::lock_guard<std::mutex> lock(g_tile_mu);
        auto it = g_tile_cache.find(key);
        if (it != g_tile_cache.end()) {
            for (int d = 0; d < 3; ++d) ctx->tile[d] = it->second[d];
            return MB_OK;
        }
    }
    static const int cand[][3] = {{32, 8, 8}, {16, 8, 8}, {32, 16, 8}, {16, 16, 8}, {64, 8, 8}};
    cudaEvent_t e0, e1;
    MB_CUDA(cudaEventCreate(&e0));
    MB_CUDA(cudaEventCreate(&e1));
    // rounds over the candidates (the first warms up), each candidate's fastest launch kept:
    // the candidates differ by a few percent, about the spread of single launches
    constexpr int NCAND = sizeof(cand) / sizeof(cand[0]), ROUNDS = 7;
    float fastest[NCAND];
    for (int i = 0; i < NCAND; ++i) fastest[i] = 1e30f;
    for (int round = 0; round < ROUNDS; ++round) {
        for (int i = 0; i < NCAND; ++i) {
            const int t[3] = {cand[i][0], cand[i][1], cand[i][2]};
            if (!spread32_tile_ok(t, ctx->g, ctx->bg)) continue;
            MB_CUDA(cudaEventRecord(e0, ctx->st));
            MB_CUDA(launch_spread32(ctx->st, ctx->B, static_cast<const float4*>(ctx->rec32.p),
                                    static_cast<const int32_t*>(ctx->cell_start.p), ctx->g,
                                    ctx->bg, t, static_cast<float*>(ctx->f.p)));
            MB_CUDA(cudaEventRecord(e1, ctx->st));
            MB_CUDA(cudaEventSynchronize(e1));
            float one = 0.f;
            MB_CUDA(cudaEventElapsedTime(&one, e0, e1));
            if (round > 0) fastest[i] = std::min(fastest[i], one);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    float best = 1e30f;
    int best_t[3] = {ctx->tile[0], ctx->tile[1], ctx->tile[2]};
    for (int i = 0; i < NCAND; ++i)
        if (fastest[i] < best) {
            best = fastest[i];
            for (int d = 0; d < 3; ++d) best_t[d] = cand[i][d];
        }
    for (int d = 0; d < 3; ++d) ctx->tile[d] = best_t[d];
    ctx->tile_ms = best;
    // the timing runs left a spread grid in f: clear it for the next step
    MB_CUDA(cudaMemsetAsync(ctx->f.p, 0, sizeof(float) * 3 * (size_t)ctx->B * ctx->g.N, ctx->st));
    ctx->f_zero = true;
    std::lock_guard<std::mutex> lock(g_tile_mu);
    g_tile_cache[key] = {best_t[0], best_t[1], best_t[2]};
    return MB_OK;
}

// Captures one FP32-grid step from the current velocity buffer into a CUDA graph (on a private
// stream; nothing executes during the capture).
mb_status capture_graph(mb_ctx* ctx, bool ext, const double* body)
{
    const int cur0 = ctx->cur;
    if (ctx->graph_exec[cur0]) cudaGraphExecDestroy(ctx->graph_exec[cur0]);
    ctx->graph_exec[cur0] = nullptr;
    if (!ctx->cap_stream)
        MB_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = ctx->st;
    const int64_t steps0 = ctx->steps_taken, l0 = ctx->launches;
    const int hcur0 = ctx->hcur, hlast0 = ctx->hlast;
    const bool ready0 = ctx->pred_ready, fz0 = ctx->f_zero;
    ctx->st = ctx->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal);
    mb_status s = MB_OK;
    if (e == cudaSuccess) {
        s = ctx->d.integrator == 1 ? do_step_stokes_fast(ctx, ext, body)
                                   : do_step_fast(ctx, ext, body);
        e = cudaStreamEndCapture(ctx->st, &graph);
    }
    ctx->st = user;
    ctx->cur = cur0;
    ctx->steps_taken = steps0;
    ctx->hcur = hcur0;
    ctx->hlast = hlast0;
    ctx->pred_ready = ready0;
    ctx->f_zero = fz0;
    ctx->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    if (s != MB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("graph capture: ") + cudaGetErrorString(e);
        return MB_ECUDA;
    }
    e = cudaGraphInstantiate(&ctx->graph_exec[cur0], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->graph_exec[cur0] = nullptr;
        ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
        return MB_ECUDA;
    }
    ctx->graph_ext[cur0] = ext;
    ctx->graph_ext_src[cur0] = ctx->ext_src;
    ctx->graph_body[cur0] = body != nullptr;
    ctx->graph_hcur[cur0] = hcur0;
    ctx->graph_fz[cur0] = ctx->f_zero;
    return MB_OK;
}

// n_steps FP32-grid steps, each replaying the captured graph of its parity (stage timing off).
mb_status run_fast_steps(mb_ctx* ctx, int n_steps, bool ext, const double* body)
{
    const bool graphs = ctx->use_graph && !ctx->timing && ctx->nb > 0;
    for (int s = 0; s < n_steps; ++s) {
        // first step after a rebuild, or after the state was set from outside: direct
        if (!graphs || !ctx->sorted_valid || (ctx->fuse_interp && !ctx->pred_ready)) {
            MB_TRY(do_step_fast(ctx, ext, body));
            finish_fast_step(ctx);
            if (!ctx->tuned) MB_TRY(autotune_spread(ctx));
            continue;
        }
        const int c = ctx->cur;
        if (!ctx->graph_exec[c] || ctx->graph_ext[c] != ext ||
            ctx->graph_ext_src[c] != ctx->ext_src ||
            ctx->graph_body[c] != (body != nullptr) || ctx->graph_hcur[c] != ctx->hcur ||
            ctx->graph_fz[c] != ctx->f_zero)
            MB_TRY(capture_graph(ctx, ext, body));
        MB_CUDA(cudaGraphLaunch(ctx->graph_exec[c], ctx->st));
        finish_fast_step(ctx);
        ctx->launches += ctx->graph_launches;
    }
    return MB_OK;
}

// Stokes-limit steps in FP32-grid mode: direct launches until the spreading tile is tuned,
// then replays of a captured graph of one step (keyed by external forces and body force).
mb_status run_stokes_fast_steps(mb_ctx* ctx, int n_steps, bool ext, const double* body)
{
    const bool graphs = ctx->use_graph && !ctx->timing && ctx->nb > 0;
    for (int s = 0; s < n_steps; ++s) {
        if (!graphs || !ctx->tuned) {
            MB_TRY(do_step_stokes_fast(ctx, ext, body));
            if (!ctx->tuned) MB_TRY(autotune_spread(ctx));
            continue;
        }
        const int c = ctx->cur;
        if (!ctx->graph_exec[c] || ctx->graph_ext[c] != ext ||
            ctx->graph_body[c] != (body != nullptr))
            MB_TRY(capture_graph(ctx, ext, body));
        MB_CUDA(cudaGraphLaunch(ctx->graph_exec[c], ctx->st));
        // the state changes of do_step_stokes_fast
        ctx->hcur = ctx->hlast = 0;
        ctx->pred_ready = false;
        ctx->f_zero = false;
        ctx->sorted_valid = true;
        ctx->steps_taken++;
        ctx->launches += ctx->graph_launches;
    }
    return MB_OK;
}

// FP64 blob positions of the current state (from the split form in FP32-grid mode).
mb_status current_positions(mb_ctx* ctx)
{
    if (ctx->rsz == 4 && ctx->nb > 0)
        MB_CUDA(launch_unsplit(ctx->st, ctx->nb, static_cast<const float4*>(ctx->sA.p),
                               static_cast<const float4*>(ctx->sB.p), ctx->g, ctx->bg,
                               static_cast<double*>(ctx->q.p)));
    return MB_OK;
}


mb_status upload_tables(mb_ctx* ctx)
{
    std::vector<double> sym(9 * SYM_LEN, 0.0);
    for (int d = 0; d < 3; ++d) {
        const int n = ctx->g.n[d];
        std::vector<double> twd(n);         // n/2 complex
        std::vector<float> twf(n);
        for (int m = 0; m < n / 2; ++m) {
            const double ang = -2.0 * M_PI * (double)m / (double)n;
            twd[2 * m] = std::cos(ang);
            twd[2 * m + 1] = std::sin(ang);
            twf[2 * m] = (float)twd[2 * m];
            twf[2 * m + 1] = (float)twd[2 * m + 1];
        }
        MB_TRY(ensure(ctx->tw[d], sizeof(double) * n, ctx->err, "twiddles"));
        const void* src = ctx->rsz == 8 ? (const void*)twd.data() : (const void*)twf.data();
        MB_CUDA(cudaMemcpyAsync(ctx->tw[d].p, src, ctx->rsz * n, cudaMemcpyHostToDevice, ctx->st));
        std::vector<double> fd(2 * n);
        std::vector<float> ff(2 * n);
        for (int m = 0; m < n; ++m) {
            const double ang = -2.0 * M_PI * (double)m / (double)n;
            fd[2 * m] = std::cos(ang);
            fd[2 * m + 1] = std::sin(ang);
            ff[2 * m] = (float)fd[2 * m];
            ff[2 * m + 1] = (float)fd[2 * m + 1];
        }
        MB_TRY(ensure(ctx->twf[d], sizeof(double) * 2 * n, ctx->err, "twiddles"));
        const void* srcf = ctx->rsz == 8 ? (const void*)fd.data() : (const void*)ff.data();
        MB_CUDA(cudaMemcpyAsync(ctx->twf[d].p, srcf, ctx->rsz * 2 * n, cudaMemcpyHostToDevice, ctx->st));
        // FP64 grids: the same table in double-float (hi, lo per part) for the three-pass FFT
        std::vector<float> fk(ctx->rsz == 8 ? 4 * n : 0);
        for (size_t i = 0; i < fk.size() / 2; ++i) {
            fk[2 * i] = (float)fd[i];
            fk[2 * i + 1] = (float)(fd[i] - (double)fk[2 * i]);
        }
        if (ctx->rsz == 8) {
            MB_TRY(ensure(ctx->twk[d], sizeof(float) * 4 * n, ctx->err, "twiddles"));
            MB_CUDA(cudaMemcpyAsync(ctx->twk[d].p, fk.data(), sizeof(float) * 4 * n,
                                    cudaMemcpyHostToDevice, ctx->st));
        }
        for (int k = 0; k < n; ++k) {
            const double th = 2.0 * M_PI * (double)k / (double)n;
            const double s = std::sin(0.5 * th);
            sym[(3 * d + 0) * SYM_LEN + k] = std::cos(th);
            sym[(3 * d + 1) * SYM_LEN + k] = std::sin(th);
            sym[(3 * d + 2) * SYM_LEN + k] = 4.0 / (ctx->d.h * ctx->d.h) * s * s;
        }
        MB_CUDA(cudaStreamSynchronize(ctx->st));
    }
    MB_TRY(ensure(ctx->sym, sizeof(double) * sym.size(), ctx->err, "symbols"));
    MB_CUDA(cudaMemcpyAsync(ctx->sym.p, sym.data(), sizeof(double) * sym.size(),
                            cudaMemcpyHostToDevice, ctx->st));
    std::vector<float> symf(sym.begin(), sym.end());
    MB_TRY(ensure(ctx->symr, sizeof(double) * sym.size(), ctx->err, "symbols"));
    if (ctx->rsz == 8)
        MB_CUDA(cudaMemcpyAsync(ctx->symr.p, sym.data(), sizeof(double) * sym.size(),
                                cudaMemcpyHostToDevice, ctx->st));
    if (ctx->rsz == 8) {
        std::vector<float> symd(2 * sym.size());
        for (size_t i = 0; i < sym.size(); ++i) {
            symd[2 * i] = (float)sym[i];
            symd[2 * i + 1] = (float)(sym[i] - (double)symd[2 * i]);
        }
        MB_TRY(ensure(ctx->symk, sizeof(float) * symd.size(), ctx->err, "symbols"));
        MB_CUDA(cudaMemcpyAsync(ctx->symk.p, symd.data(), sizeof(float) * symd.size(),
                                cudaMemcpyHostToDevice, ctx->st));
        MB_CUDA(cudaStreamSynchronize(ctx->st));
    }
    else
        MB_CUDA(cudaMemcpyAsync(ctx->symr.p, symf.data(), sizeof(float) * symf.size(),
                                cudaMemcpyHostToDevice, ctx->st));
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    return MB_OK;
}

void release(mb_ctx* ctx)
{
    drop_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx->cap_stream = nullptr;
    if (ctx->side) cudaStreamDestroy(ctx->side);
    ctx->side = nullptr;
    if (ctx->side2) cudaStreamDestroy(ctx->side2);
    ctx->side2 = nullptr;
    for (cudaEvent_t& e : ctx->fork) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    DBuf* all[] = {&ctx->v[0], &ctx->v[1], &ctx->vsum, &ctx->f, &ctx->spec, &ctx->vbar, &ctx->fsum,
                   &ctx->tw[0], &ctx->tw[1], &ctx->tw[2], &ctx->twf[0], &ctx->twf[1],
                   &ctx->twf[2], &ctx->sym, &ctx->symr, &ctx->body_prof,
                   &ctx->prof_scratch, &ctx->q, &ctx->qh, &ctx->u, &ctx->F, &ctx->rec,
                   &ctx->ext, &ctx->pid, &ctx->box_of, &ctx->adj_start, &ctx->adj_j,
                   &ctx->adj_rest, &ctx->part_start, &ctx->part_blobs, &ctx->box_off,
                   &ctx->box_par, &ctx->cell_count, &ctx->cell_start, &ctx->blob_cell,
                   &ctx->blob_rank, &ctx->sorted, &ctx->loc, &ctx->scan_tmp, &ctx->partial,
                   &ctx->staging_in, &ctx->staging_out, &ctx->mean_scratch, &ctx->s_q,
                   &ctx->s_F, &ctx->s_rec, &ctx->s_cell_count, &ctx->s_cell_start,
                   &ctx->s_blob_cell, &ctx->s_blob_rank, &ctx->s_sorted, &ctx->s_scan,
                   &ctx->s_u, &ctx->s_g0, &ctx->s_g1, &ctx->s_g2, &ctx->s_out, &ctx->sA,
                   &ctx->sB, &ctx->hA[0], &ctx->hA[1], &ctx->hB[0], &ctx->hB[1], &ctx->F32, &ctx->rec32, &ctx->ext32,
                   &ctx->ext_sum, &ctx->ext_ticket, &ctx->adj32, &ctx->adj32_start, &ctx->tmpl32, &ctx->tstart32, &ctx->Fpre64, &ctx->Fs32, &ctx->u32, &ctx->a_qn, &ctx->a_u, &ctx->a_qh,
                   &ctx->a_gq, &ctx->a_guc, &ctx->a_gqh, &ctx->a_gF, &ctx->a_gu, &ctx->a_gk, &ctx->a_gU,
                   &ctx->a_vn, &ctx->a_vp, &ctx->a_w, &ctx->a_gw, &ctx->a_gvp, &ctx->a_gvn,
                   &ctx->a_gf, &ctx->a_tmp, &ctx->a_zero, &ctx->W, &ctx->step_index,
                   &ctx->twk[0], &ctx->twk[1], &ctx->twk[2], &ctx->symk};
    for (DBuf* b : all) dfree(*b);
    for (cudaEvent_t& e : ctx->ev_ring)
        if (e) cudaEventDestroy(e);
    ctx->ev_ring.clear();
}

// Standalone spreading of n blobs into one box grid `out_dev` (device pointer).
template <typename R>
mb_status standalone_spread(mb_ctx* ctx, int64_t n, const double* qd, const double* Fd,
                            R* out_dev)
{
    cudaStream_t st = ctx->st;
    std::string& E = ctx->err;
    BinGeo bg = ctx->bg;
    // standalone operators bin with the default cell size
    {
        int bs = 2;
        const int nmin = std::min(ctx->g.n[0], std::min(ctx->g.n[1], ctx->g.n[2]));
        if (bs > nmin) bs = nmin;
        bg.bs = bs;
        for (int a = 0; a < 3; ++a) bg.nc[a] = ctx->g.n[a] / bs;
        bg.ncell = (int64_t)bg.nc[0] * bg.nc[1] * bg.nc[2];
        bg.inv_w = 1.0 / (bs * ctx->d.h);
        set_float_geo(bg);
    }
    MB_TRY(ensure(ctx->s_q, sizeof(double) * 3 * n, E, "spread q"));
    MB_TRY(ensure(ctx->s_rec, sizeof(double) * 6 * n, E, "spread rec"));
    MB_TRY(ensure(ctx->s_cell_count, sizeof(int32_t) * bg.ncell, E, "spread cells"));
    MB_TRY(ensure(ctx->s_cell_start, sizeof(int32_t) * (bg.ncell + 1), E, "spread cells"));
    MB_TRY(ensure(ctx->s_blob_cell, sizeof(int32_t) * n, E, "spread cells"));
    MB_TRY(ensure(ctx->s_blob_rank, sizeof(int32_t) * n, E, "spread cells"));
    MB_TRY(ensure(ctx->s_sorted, sizeof(int32_t) * n, E, "spread cells"));
    MB_TRY(ensure(ctx->s_scan, sizeof(int32_t) * (bg.ncell / 4096 + 2), E, "spread scan"));
    double* q = static_cast<double*>(ctx->s_q.p);
    if (n > 0) {
        MB_CUDA(cudaMemcpyAsync(q, qd, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
        k_wrap<<<(unsigned)((3 * n + 255) / 256), 256, 0, st>>>(n, q, ctx->g.L[0], ctx->g.L[1],
                                                                ctx->g.L[2]);
        MB_CUDA(cudaGetLastError());
    }
    MB_CUDA(launch_bin(st, n, q, nullptr, 1, bg, static_cast<int32_t*>(ctx->s_cell_count.p),
                       static_cast<int32_t*>(ctx->s_cell_start.p),
                       static_cast<int32_t*>(ctx->s_blob_cell.p),
                       static_cast<int32_t*>(ctx->s_blob_rank.p),
                       static_cast<int32_t*>(ctx->s_sorted.p),
                       static_cast<int32_t*>(ctx->s_scan.p), ctx->d.deterministic != 0));
    MB_CUDA(launch_make_rec(st, n, static_cast<const int32_t*>(ctx->s_sorted.p), q, Fd,
                            static_cast<double*>(ctx->s_rec.p)));
    MB_CUDA(launch_spread<R>(st, 1, static_cast<const double*>(ctx->s_rec.p),
                             static_cast<const int32_t*>(ctx->s_cell_start.p), ctx->g, bg,
                             ctx->tile, out_dev));
    return MB_OK;
}

}  // namespace

namespace mbk {
// Error of the last failed context-free call, reported by mb_last_error(NULL).
void set_context_free_error(const std::string& msg) { g_create_error = msg; }
}  // namespace mbk

// ==========================================================================================
extern "C" {

mb_status mb_create_grid(const mb_grid_desc* desc, void* cuda_stream, mb_ctx** out)
{
    if (out) *out = nullptr;
    if (!desc || !out) {
        g_create_error = "mb_create_grid: desc and out must be non-null";
        return MB_EINVAL;
    }
    const mb_grid_desc& d = *desc;
    const int ns[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a)
        if (!is_pow2(ns[a]) || ns[a] < 4 || ns[a] > 256) {
            g_create_error = "nx, ny, nz must be powers of two in [4, 256]";
            return MB_EINVAL;
        }
    if (d.batch < 1 || d.batch > 65535) {
        g_create_error = "batch must be in [1, 65535]";
        return MB_EINVAL;
    }
    if (!(d.h > 0 && std::isfinite(d.h)) || !(d.rho > 0 && std::isfinite(d.rho)) ||
        !(d.eta > 0 && std::isfinite(d.eta)) || !(d.dt > 0 && std::isfinite(d.dt))) {
        g_create_error = "h, rho, eta and dt must be finite and positive";
        return MB_EINVAL;
    }
    if (d.precision != 0 && d.precision != 1) {
        g_create_error = "precision must be 0 (FP32 grid) or 1 (FP64)";
        return MB_EINVAL;
    }
    if (d.deterministic != 0 && d.deterministic != 1) {
        g_create_error = "deterministic must be 0 or 1";
        return MB_EINVAL;
    }
    if (d.advection != 0 && d.advection != 1) {
        g_create_error = "advection must be 0 or 1 (the rho v v stress)";
        return MB_EINVAL;
    }
    if (d.mean_mode != 0 && d.mean_mode != 1) {
        g_create_error = "mean_mode must be 0 (conserve) or 1 (zero)";
        return MB_EINVAL;
    }
    if (!(d.kT >= 0.0 && std::isfinite(d.kT))) {
        g_create_error = "kT must be finite and >= 0";
        return MB_EINVAL;
    }
    if (d.integrator != 0 && d.integrator != 1) {
        g_create_error = "integrator must be 0 (inertial coupling) or 1 (Stokes limit)";
        return MB_EINVAL;
    }
    if (d.integrator == 1 && d.mean_mode != 1) {
        g_create_error = "the Stokes limit has no steady mean flow under a net force: set mean_mode = 1";
        return MB_EINVAL;
    }
    if (d.integrator == 1 && d.kT != 0.0) {
        g_create_error = "the Stokes-limit integrator is deterministic: set kT = 0";
        return MB_EINVAL;
    }
    if (d.integrator == 1 && d.advection != 0) {
        g_create_error = "the Stokes limit has no convective term: set advection = 0";
        return MB_EINVAL;
    }
    mb_ctx* ctx = new (std::nothrow) mb_ctx();
    if (!ctx) {
        g_create_error = "out of host memory";
        return MB_ENOMEM;
    }
    ctx->d = d;
    ctx->st = static_cast<cudaStream_t>(cuda_stream);
    ctx->B = d.batch;
    ctx->rsz = d.precision == 1 ? 8 : 4;
    for (int a = 0; a < 3; ++a) {
        ctx->g.n[a] = ns[a];
        ctx->g.L[a] = ns[a] * d.h;
    }
    ctx->g.N = (int64_t)ns[0] * ns[1] * ns[2];
    ctx->g.h = d.h;
    ctx->g.inv_h = 1.0 / d.h;
    set_float_geo(ctx->g);
    ctx->nxh = ns[0] / 2 + 1;
    ctx->boxes.resize(ctx->B);
    if (const char* e = std::getenv("MB_FFT_PASSES")) ctx->fft_passes = std::atoi(e) == 5 ? 5 : 3;
    // the three-pass pipeline holds whole planes and lines of up to 128 points on chip; longer
    // sides take the five-pass pipeline (one radix-2 pass per axis, lines of up to 256 points)
    if (ns[0] > 128 || ns[1] > 128 || ns[2] > 128) ctx->fft_passes = 5;
    if (const char* e = std::getenv("MB_NO_GRAPH")) ctx->use_graph = std::atoi(e) == 0;
    if (const char* e = std::getenv("MB_NO_AUTOTUNE")) ctx->autotune = std::atoi(e) == 0;
    if (const char* e = std::getenv("MB_NO_FUSE_INTERP")) ctx->fuse_interp = std::atoi(e) == 0;
    choose_bins(ctx, 0.0);
    pick_tile(ctx);

    auto fail = [&](mb_status s) {
        g_create_error = ctx->err;
        release(ctx);
        delete ctx;
        return s;
    };
    const size_t gb = grid_bytes(ctx, ctx->B);
    const size_t sb = (size_t)ctx->B * 3 * ns[2] * ns[1] * ctx->nxh * 2 * ctx->rsz;
    mb_status s;
    if ((s = ensure(ctx->v[0], gb, ctx->err, "v")) != MB_OK) return fail(s);
    if ((s = ensure(ctx->v[1], gb, ctx->err, "v")) != MB_OK) return fail(s);
    if (ctx->rsz == 4 && (s = ensure(ctx->vsum, gb, ctx->err, "v sum")) != MB_OK) return fail(s);
    if ((s = ensure(ctx->f, gb, ctx->err, "f")) != MB_OK) return fail(s);
    if ((s = ensure(ctx->spec, sb, ctx->err, "spectrum")) != MB_OK) return fail(s);
    if ((s = ensure(ctx->vbar, sizeof(double) * 3 * ctx->B, ctx->err, "vbar")) != MB_OK) return fail(s);
    if ((s = ensure(ctx->fsum, sizeof(double) * 3 * ctx->B, ctx->err, "fsum")) != MB_OK) return fail(s);
    if ((s = ensure(ctx->step_index, sizeof(uint64_t), ctx->err, "step index")) != MB_OK) return fail(s);
    ctx->thermal = d.kT > 0.0;
    ctx->advect = d.advection == 1;
    if (ctx->thermal)
        ctx->thermal_amp = std::sqrt(2.0 * d.eta * d.kT / (d.h * d.h * d.h * d.dt));
    if ((ctx->thermal || ctx->advect) &&
        (s = ensure(ctx->W, 3 * gb, ctx->err, "fluid stress")) != MB_OK)
        return fail(s);
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "no CUDA device";
        return fail(MB_ECUDA);
    }
    if (cudaMemsetAsync(ctx->v[0].p, 0, gb, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->v[1].p, 0, gb, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->vbar.p, 0, sizeof(double) * 3 * ctx->B, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->step_index.p, 0, sizeof(uint64_t), ctx->st) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cudaMemsetAsync failed";
        return fail(MB_ECUDA);
    }
    if ((s = upload_tables(ctx)) != MB_OK) return fail(s);
    // the side stream and fork/join events of the step (created here, never inside a capture)
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking) != cudaSuccess ||
        [&] {
            for (cudaEvent_t& e : ctx->fork)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                    return true;
            return false;
        }()) {
        cudaGetLastError();
        ctx->err = "stream or event creation failed";
        return fail(MB_ECUDA);
    }
    *out = ctx;
    return MB_OK;
}

mb_status mb_destroy(mb_ctx* ctx)
{
    if (!ctx) return MB_OK;
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->st);
    cudaGetLastError();
    release(ctx);
    delete ctx;
    return MB_OK;
}

const char* mb_last_error(const mb_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

mb_status mb_set_particles(mb_ctx* ctx, int box, int64_t n_blobs, const double* pos,
                           const int32_t* particle_id, int64_t n_bonds, const int32_t* bonds,
                           const double* rest_len, double k_spring, double k_rep, double r_cut)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (box < 0 || box >= ctx->B) return invalid(ctx, "box out of range");
    if (n_blobs < 0 || n_bonds < 0) return invalid(ctx, "negative count");
    if (n_blobs > 0 && (!pos || !particle_id)) return invalid(ctx, "pos and particle_id required");
    if (n_bonds > 0 && (!bonds || !rest_len)) return invalid(ctx, "bonds and rest_len required");
    if (!std::isfinite(k_spring) || !std::isfinite(k_rep) || !std::isfinite(r_cut) ||
        k_rep < 0 || r_cut < 0)
        return invalid(ctx, "k_spring must be finite, k_rep and r_cut finite and >= 0");
    const double half_min = 0.5 * ctx->d.h * std::min(ctx->g.n[0], std::min(ctx->g.n[1], ctx->g.n[2]));
    if (k_rep > 0 && r_cut > half_min) return invalid(ctx, "r_cut exceeds half the box");
    if (n_blobs > (int64_t)1 << 30) return invalid(ctx, "too many blobs");
    BoxData bx;
    bx.pos.resize(3 * n_blobs);
    bx.pid.resize(n_blobs);
    bx.bonds.resize(2 * n_bonds);
    bx.rest.resize(n_bonds);
    MB_TRY(copy_to_host(ctx, pos, sizeof(double) * 3 * n_blobs, bx.pos.data()));
    MB_TRY(copy_to_host(ctx, particle_id, sizeof(int32_t) * n_blobs, bx.pid.data()));
    MB_TRY(copy_to_host(ctx, bonds, sizeof(int32_t) * 2 * n_bonds, bx.bonds.data()));
    MB_TRY(copy_to_host(ctx, rest_len, sizeof(double) * n_bonds, bx.rest.data()));
    int64_t maxp = -1;
    for (int64_t i = 0; i < n_blobs; ++i) {
        if (bx.pid[i] < 0) return invalid(ctx, "particle_id must be >= 0");
        maxp = std::max<int64_t>(maxp, bx.pid[i]);
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(bx.pos[3 * i + a])) return invalid(ctx, "non-finite position");
    }
    for (int64_t e = 0; e < n_bonds; ++e) {
        const int32_t i = bx.bonds[2 * e], j = bx.bonds[2 * e + 1];
        if (i < 0 || j < 0 || i >= n_blobs || j >= n_blobs || i == j)
            return invalid(ctx, "bond " + std::to_string(e) + " has an invalid blob index");
        if (!(bx.rest[e] >= 0) || !std::isfinite(bx.rest[e]))
            return invalid(ctx, "rest lengths must be finite and >= 0");
    }
    bx.np = maxp + 1;
    bx.k_spring = k_spring;
    bx.k_rep = k_rep;
    bx.r_cut = r_cut;
    bx.set = true;
    ctx->boxes[box] = std::move(bx);
    ctx->dirty = true;
    ctx->steps_taken = 0;
    return MB_OK;
}

mb_status mb_step(mb_ctx* ctx, int n_steps, const double* ext_blob_force,
                  const double* body_force)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (n_steps < 0) return invalid(ctx, "n_steps must be >= 0");
    MB_TRY(ensure_ready(ctx));
    if (body_force) {
        const void* before = ctx->body_prof.p;
        MB_TRY(set_body(ctx, body_force, ctx->body_prof, true));
        if (ctx->body_prof.p != before) drop_graph(ctx);   // captured steps hold the old buffer
    }
    const double* ext = nullptr;
    if (ctx->d.integrator == 1 && ctx->rsz == 4) {
        // Stokes limit, FP32 grid: the FP32 blob path with the external forces in FP32
        bool has_ext = false;
        if (ext_blob_force && ctx->nb > 0) {
            const void* src = nullptr;
            MB_TRY(stage_in(ctx, ext_blob_force, sizeof(double) * 3 * ctx->nb, ctx->ext, &src, "ext"));
            MB_CUDA(launch_ext_prepare(ctx->st, ctx->B, ctx->max_box_blobs,
                                       static_cast<const int64_t*>(ctx->box_off.p),
                                       static_cast<const double*>(src),
                                       static_cast<float4*>(ctx->ext32.p),
                                       static_cast<double*>(ctx->partial.p),
                                       static_cast<double*>(ctx->ext_sum.p),
                                       static_cast<unsigned*>(ctx->ext_ticket.p)));
            has_ext = true;
        }
        return run_stokes_fast_steps(ctx, n_steps, has_ext, body_force);
    }
    if (ctx->d.integrator == 1) {
        // Stokes limit, FP64 grid: FP64 positions and forces, from the library's copy
        if (ext_blob_force && ctx->nb > 0) {
            const void* src = nullptr;
            MB_TRY(stage_in(ctx, ext_blob_force, sizeof(double) * 3 * ctx->nb, ctx->ext, &src, "ext"));
            if (src != ctx->ext.p)
                MB_CUDA(cudaMemcpyAsync(ctx->ext.p, src, sizeof(double) * 3 * ctx->nb,
                                        cudaMemcpyDeviceToDevice, ctx->st));
            ext = static_cast<const double*>(ctx->ext.p);
        }
        for (int s = 0; s < n_steps; ++s) MB_TRY(do_step_stokes<double>(ctx, ext, body_force));
        return MB_OK;
    }
    if (ext_blob_force && ctx->nb > 0) {
        const void* src = nullptr;
        void* mapped = ctx->rsz == 4 ? mapped_host_ptr(ext_blob_force) : nullptr;
        if (mapped)
            src = mapped;         // page-locked host forces: the kernel reads them directly
        else
            MB_TRY(stage_in(ctx, ext_blob_force, sizeof(double) * 3 * ctx->nb, ctx->ext, &src, "ext"));
        if (ctx->rsz == 4 && n_steps == 1) {
            // one step: converted inside it, beside the binning (the pointer is not kept past
            // this call)
            ctx->ext_src = static_cast<const double*>(src);
            ext = static_cast<const double*>(ctx->ext.p);   // marks forces present
        } else if (ctx->rsz == 4) {
            // converted once into the library's FP32 copy (the steps never read `src`)
            MB_CUDA(launch_ext_prepare(ctx->st, ctx->B, ctx->max_box_blobs,
                                       static_cast<const int64_t*>(ctx->box_off.p),
                                       static_cast<const double*>(src),
                                       static_cast<float4*>(ctx->ext32.p),
                                       static_cast<double*>(ctx->partial.p),
                                       static_cast<double*>(ctx->ext_sum.p),
                                       static_cast<unsigned*>(ctx->ext_ticket.p)));
            ext = static_cast<const double*>(ctx->ext.p);   // marks forces present
        } else {
            if (src != ctx->ext.p)
                MB_CUDA(cudaMemcpyAsync(ctx->ext.p, src, sizeof(double) * 3 * ctx->nb,
                                        cudaMemcpyDeviceToDevice, ctx->st));
            ext = static_cast<const double*>(ctx->ext.p);
        }
    }
    if (ctx->rsz == 4) {
        const mb_status st = run_fast_steps(ctx, n_steps, ext != nullptr, body_force);
        ctx->ext_src = nullptr;
        return st;
    }
    for (int s = 0; s < n_steps; ++s) MB_TRY(do_step<double>(ctx, ext, body_force));
    return MB_OK;
}

mb_status mb_get_forces(mb_ctx* ctx, double* blob_force, double* midpoint_pos)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (ctx->dirty || ctx->steps_taken == 0) {
        ctx->err = "no step has been taken with the current particles";
        return MB_ESTATE;
    }
    const size_t by = sizeof(double) * 3 * ctx->nb;
    if (ctx->nb == 0) return MB_OK;
    if (ctx->rsz == 4) {
        MB_CUDA(launch_forces_to_fp64(ctx->st, ctx->nb, static_cast<const float4*>(ctx->F32.p),
                                      static_cast<double*>(ctx->F.p)));
        MB_CUDA(launch_unsplit(ctx->st, ctx->nb, static_cast<const float4*>(ctx->hA[ctx->hlast].p),
                               static_cast<const float4*>(ctx->hB[ctx->hlast].p), ctx->g, ctx->bg,
                               static_cast<double*>(ctx->qh.p)));
    }
    double* outs[2] = {blob_force, midpoint_pos};
    DBuf* srcs[2] = {&ctx->F, &ctx->qh};
    for (int i = 0; i < 2; ++i) {
        if (!outs[i]) continue;
        void* dst;
        bool host;
        MB_TRY(out_target(ctx, outs[i], by, ctx->staging_out, &dst, &host, "forces"));
        MB_CUDA(cudaMemcpyAsync(dst, srcs[i]->p, by, cudaMemcpyDeviceToDevice, ctx->st));
        MB_TRY(finish_out(ctx, outs[i], dst, by, host));
    }
    return MB_OK;
}

mb_status mb_set_stage_timing(mb_ctx* ctx, int enable)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (enable && ctx->ev_ring.empty()) {
        ctx->ev_ring.assign((size_t)mb_ctx::EV_RING * (NUM_STAGES + 1), nullptr);
        for (cudaEvent_t& e : ctx->ev_ring) MB_CUDA(cudaEventCreate(&e));
    }
    MB_TRY(drain_stage_events(ctx));
    ctx->timing = enable != 0;
    for (int i = 0; i < NUM_STAGES; ++i) {
        ctx->stage_ms[i] = 0.0;
        ctx->stage_calls[i] = 0;
    }
    return MB_OK;
}

mb_status mb_get_stage_times(mb_ctx* ctx, int max_stages, double* ms_total,
                             int64_t* calls, int* n_stages)
{
    if (!ctx || max_stages < 0) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    MB_TRY(drain_stage_events(ctx));
    if (n_stages) *n_stages = NUM_STAGES;
    for (int i = 0; i < NUM_STAGES && i < max_stages; ++i) {
        if (ms_total) ms_total[i] = ctx->stage_ms[i];
        if (calls) calls[i] = ctx->stage_calls[i];
    }
    return MB_OK;
}

const char* mb_stage_name(int stage)
{
    return stage >= 0 && stage < NUM_STAGES ? STAGE_NAMES[stage] : "";
}

mb_status mb_set_step_index(mb_ctx* ctx, uint64_t step)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    MB_CUDA(cudaMemcpyAsync(ctx->step_index.p, &step, sizeof(uint64_t), cudaMemcpyHostToDevice,
                            ctx->st));
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    return MB_OK;
}

mb_status mb_get_step_index(mb_ctx* ctx, uint64_t* step)
{
    if (!ctx) return MB_EINVAL;
    if (!step) return invalid(ctx, "step must be non-null");
    DeviceGuard dg(ctx->device);
    uint64_t v = 0;
    MB_CUDA(cudaMemcpyAsync(&v, ctx->step_index.p, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            ctx->st));
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    *step = v;
    return MB_OK;
}

mb_status mb_get_launch_count(const mb_ctx* ctx, int64_t* launches)
{
    if (!ctx || !launches) return MB_EINVAL;
    *launches = ctx->launches;
    return MB_OK;
}

mb_status mb_set_positions(mb_ctx* ctx, const double* pos)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (!pos) return invalid(ctx, "pos must be non-null");
    MB_TRY(ensure_ready(ctx));
    if (ctx->nb == 0) return MB_OK;
    const size_t by = sizeof(double) * 3 * ctx->nb;
    MB_CUDA(cudaMemcpyAsync(ctx->q.p, pos, by, cudaMemcpyDefault, ctx->st));
    double* q = static_cast<double*>(ctx->q.p);
    k_wrap<<<(unsigned)((3 * ctx->nb + 255) / 256), 256, 0, ctx->st>>>(ctx->nb, q, ctx->g.L[0],
                                                                      ctx->g.L[1], ctx->g.L[2]);
    MB_CUDA(cudaGetLastError());
    if (ctx->rsz == 4)
        MB_CUDA(launch_split(ctx->st, ctx->nb, q, ctx->g, ctx->bg, static_cast<float4*>(ctx->sA.p),
                             static_cast<float4*>(ctx->sB.p)));
    ctx->sorted_valid = false;
    ctx->pred_ready = false;
    ctx->steps_taken = 0;
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    return MB_OK;
}

namespace {

// Copies a caller array (host or device) into a device scratch buffer.
mb_status pull(mb_ctx* ctx, DBuf& dst, const void* src, size_t bytes, const char* what)
{
    MB_TRY(ensure(dst, bytes, ctx->err, what));
    MB_CUDA(cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyDefault, ctx->st));
    return MB_OK;
}

// Copies a device scratch buffer back to a caller array (host or device).
mb_status push(mb_ctx* ctx, void* dst, const DBuf& src, size_t bytes)
{
    MB_CUDA(cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDefault, ctx->st));
    if (!is_device_ptr(dst)) MB_CUDA(cudaStreamSynchronize(ctx->st));
    return MB_OK;
}

mb_status adjoint_preconditions(mb_ctx* ctx)
{
    if (ctx->rsz != 8) return invalid(ctx, "the adjoint is provided for FP64 contexts (precision 1)");
    if (ctx->B != 1) return invalid(ctx, "the adjoint is provided for batch 1");
    return ensure_ready(ctx);
}

// gq += G(q; v, gu) and gv += h^3 S(q) gu (the transpose of u = J(q) v), all on device buffers.
mb_status velocity_adjoint_dev(mb_ctx* ctx, const double* q, const double* v, const double* gu,
                               double* gq, double* gv)
{
    const int64_t n3N = 3 * ctx->g.N;
    const double h3 = ctx->d.h * ctx->d.h * ctx->d.h;
    MB_CUDA(launch_grad_interp(ctx->st, ctx->nb, q, v, gu, ctx->g, 1.0, gq));
    MB_TRY(ensure(ctx->a_tmp, sizeof(double) * n3N, ctx->err, "adjoint grid"));
    double* tmp = static_cast<double*>(ctx->a_tmp.p);
    MB_TRY(standalone_spread<double>(ctx, ctx->nb, q, gu, tmp));
    MB_CUDA(launch_axpby(ctx->st, n3N, 1.0, gv, h3, tmp, gv));
    return MB_OK;
}

}  // namespace

mb_status mb_velocity_adjoint(mb_ctx* ctx, const double* pos, const void* grid_v,
                              const double* grad_u, double* grad_pos, void* grad_v)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (!pos || !grid_v || !grad_u || !grad_pos || !grad_v) return invalid(ctx, "null argument");
    MB_TRY(adjoint_preconditions(ctx));
    const int64_t nb = ctx->nb;
    const size_t bv = sizeof(double) * 3 * nb, bg = sizeof(double) * 3 * ctx->g.N;
    MB_TRY(pull(ctx, ctx->a_qn, pos, bv, "adjoint q"));
    MB_TRY(pull(ctx, ctx->a_vn, grid_v, bg, "adjoint v"));
    MB_TRY(pull(ctx, ctx->a_gu, grad_u, bv, "adjoint gu"));
    MB_TRY(pull(ctx, ctx->a_gq, grad_pos, bv, "adjoint gq"));
    MB_TRY(pull(ctx, ctx->a_gvn, grad_v, bg, "adjoint gv"));
    double* q = static_cast<double*>(ctx->a_qn.p);
    k_wrap<<<(unsigned)((3 * nb + 255) / 256), 256, 0, ctx->st>>>(nb, q, ctx->g.L[0], ctx->g.L[1],
                                                                 ctx->g.L[2]);
    MB_CUDA(cudaGetLastError());
    MB_TRY(velocity_adjoint_dev(ctx, q, static_cast<const double*>(ctx->a_vn.p),
                                static_cast<const double*>(ctx->a_gu.p),
                                static_cast<double*>(ctx->a_gq.p),
                                static_cast<double*>(ctx->a_gvn.p)));
    MB_TRY(push(ctx, grad_pos, ctx->a_gq, bv));
    return push(ctx, grad_v, ctx->a_gvn, bg);
}

mb_status mb_particle_velocity_adjoint(mb_ctx* ctx, const double* pos, const void* grid_v,
                                       const double* grad_U, double* grad_pos, void* grad_v)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (!pos || !grid_v || !grad_U || !grad_pos || !grad_v) return invalid(ctx, "null argument");
    MB_TRY(adjoint_preconditions(ctx));
    const int64_t nb = ctx->nb, np = ctx->np;
    const size_t bv = sizeof(double) * 3 * nb, bg = sizeof(double) * 3 * ctx->g.N;
    MB_TRY(pull(ctx, ctx->a_qn, pos, bv, "adjoint q"));
    MB_TRY(pull(ctx, ctx->a_vn, grid_v, bg, "adjoint v"));
    MB_TRY(pull(ctx, ctx->a_gU, grad_U, sizeof(double) * 3 * (np > 0 ? np : 1), "adjoint gU"));
    MB_TRY(pull(ctx, ctx->a_gq, grad_pos, bv, "adjoint gq"));
    MB_TRY(pull(ctx, ctx->a_gvn, grad_v, bg, "adjoint gv"));
    MB_TRY(ensure(ctx->a_gu, bv, ctx->err, "adjoint gu"));
    MB_CUDA(cudaMemsetAsync(ctx->a_gu.p, 0, bv, ctx->st));
    MB_CUDA(launch_particle_mean_adjoint(ctx->st, np,
                                         static_cast<const int32_t*>(ctx->part_start.p),
                                         static_cast<const int32_t*>(ctx->part_blobs.p),
                                         static_cast<const double*>(ctx->a_gU.p),
                                         static_cast<double*>(ctx->a_gu.p)));
    double* q = static_cast<double*>(ctx->a_qn.p);
    k_wrap<<<(unsigned)((3 * nb + 255) / 256), 256, 0, ctx->st>>>(nb, q, ctx->g.L[0], ctx->g.L[1],
                                                                 ctx->g.L[2]);
    MB_CUDA(cudaGetLastError());
    MB_TRY(velocity_adjoint_dev(ctx, q, static_cast<const double*>(ctx->a_vn.p),
                                static_cast<const double*>(ctx->a_gu.p),
                                static_cast<double*>(ctx->a_gq.p),
                                static_cast<double*>(ctx->a_gvn.p)));
    MB_TRY(push(ctx, grad_pos, ctx->a_gq, bv));
    return push(ctx, grad_v, ctx->a_gvn, bg);
}

mb_status mb_adjoint_step(mb_ctx* ctx, const double* pos_n, const void* grid_v_n,
                          const double* ext_blob_force, const double* body_force,
                          double* grad_pos, void* grad_v, double* grad_k_spring)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (!pos_n || !grid_v_n || !grad_pos || !grad_v) return invalid(ctx, "null argument");
    MB_TRY(adjoint_preconditions(ctx));
    if (ctx->d.integrator != 0)
        return invalid(ctx, "the step adjoint is provided for the inertial coupling integrator");
    if (ctx->thermal || ctx->advect)
        return invalid(ctx, "the step adjoint is provided without the thermal and convective stresses");
    if (body_force) MB_TRY(set_body(ctx, body_force, ctx->prof_scratch, false));
    cudaStream_t st = ctx->st;
    const GridGeo& g = ctx->g;
    const int64_t nb = ctx->nb, n3N = 3 * g.N;
    const size_t bv = sizeof(double) * 3 * nb, bg = sizeof(double) * n3N;
    const double h = ctx->d.h, h3 = h * h * h, dt = ctx->d.dt;
    std::string& E = ctx->err;
    // ---- inputs
    MB_TRY(pull(ctx, ctx->a_qn, pos_n, bv, "adjoint q"));
    MB_TRY(pull(ctx, ctx->a_vn, grid_v_n, bg, "adjoint v"));
    MB_TRY(pull(ctx, ctx->a_gq, grad_pos, bv, "adjoint gq"));
    MB_TRY(pull(ctx, ctx->a_gvp, grad_v, bg, "adjoint gv"));   // becomes dL/dv^{n+1} + gw/2
    const double* ext = nullptr;
    if (ext_blob_force && nb > 0) {
        MB_TRY(pull(ctx, ctx->ext, ext_blob_force, bv, "adjoint ext"));
        ext = static_cast<const double*>(ctx->ext.p);
    }
    for (DBuf* b : {&ctx->a_u, &ctx->a_qh, &ctx->a_guc, &ctx->a_gqh, &ctx->a_gF, &ctx->a_gu})
        MB_TRY(ensure(*b, bv, E, "adjoint blobs"));
    for (DBuf* b : {&ctx->a_vp, &ctx->a_w, &ctx->a_gw, &ctx->a_gvn, &ctx->a_gf, &ctx->a_tmp,
                    &ctx->a_zero})
        MB_TRY(ensure(*b, bg, E, "adjoint grids"));
    MB_TRY(ensure(ctx->a_gk, sizeof(double), E, "adjoint gk"));
    MB_CUDA(cudaMemsetAsync(ctx->a_zero.p, 0, bg, st));
    MB_CUDA(cudaMemsetAsync(ctx->a_gk.p, 0, sizeof(double), st));
    MB_CUDA(cudaMemsetAsync(ctx->a_gqh.p, 0, bv, st));
    double* qn = static_cast<double*>(ctx->a_qn.p);
    double* qh = static_cast<double*>(ctx->a_qh.p);
    double* vn = static_cast<double*>(ctx->a_vn.p);
    double* vp = static_cast<double*>(ctx->a_vp.p);
    double* w = static_cast<double*>(ctx->a_w.p);
    double* f = static_cast<double*>(ctx->f.p);
    double* gq = static_cast<double*>(ctx->a_gq.p);
    double* gqh = static_cast<double*>(ctx->a_gqh.p);
    double* guc = static_cast<double*>(ctx->a_guc.p);
    double* gF = static_cast<double*>(ctx->a_gF.p);
    double* gu = static_cast<double*>(ctx->a_gu.p);
    double* gw = static_cast<double*>(ctx->a_gw.p);
    double* gvp = static_cast<double*>(ctx->a_gvp.p);
    double* gvn = static_cast<double*>(ctx->a_gvn.p);
    double* gf = static_cast<double*>(ctx->a_gf.p);
    double* tmp = static_cast<double*>(ctx->a_tmp.p);
    double* F = static_cast<double*>(ctx->F.p);
    k_wrap<<<(unsigned)((3 * nb + 255) / 256), 256, 0, st>>>(nb, qn, g.L[0], g.L[1], g.L[2]);
    MB_CUDA(cudaGetLastError());
    const BoxData& bx = ctx->boxes[0];
    // ---- recompute the step: u^n, q^{n+1/2}, F, f, v^{n+1}, w = (v^n + v^{n+1})/2
    MB_CUDA(launch_interp<double>(st, 1, nb, qn, nullptr, vn, nullptr, nullptr, g, dt,
                                  static_cast<double*>(ctx->a_u.p), qh));
    MB_CUDA(launch_bin(st, nb, qh, nullptr, 1, ctx->bg, static_cast<int32_t*>(ctx->cell_count.p),
                       static_cast<int32_t*>(ctx->cell_start.p),
                       static_cast<int32_t*>(ctx->blob_cell.p),
                       static_cast<int32_t*>(ctx->blob_rank.p), static_cast<int32_t*>(ctx->sorted.p),
                       static_cast<int32_t*>(ctx->scan_tmp.p), false,
                       static_cast<const int32_t*>(ctx->pid.p), static_cast<float4*>(ctx->loc.p)));
    ForceArgs fa{};
    fa.box_off = static_cast<const int64_t*>(ctx->box_off.p);
    fa.sorted = static_cast<const int32_t*>(ctx->sorted.p);
    fa.q = qh;
    fa.pid = static_cast<const int32_t*>(ctx->pid.p);
    fa.adj_start = static_cast<const int32_t*>(ctx->adj_start.p);
    fa.adj_j = static_cast<const int32_t*>(ctx->adj_j.p);
    fa.adj_rest = static_cast<const double*>(ctx->adj_rest.p);
    fa.box_par = static_cast<const double*>(ctx->box_par.p);
    fa.cell_start = static_cast<const int32_t*>(ctx->cell_start.p);
    fa.blob_cell = static_cast<const int32_t*>(ctx->blob_cell.p);
    fa.ext = ext;
    fa.loc = static_cast<const float4*>(ctx->loc.p);
    fa.F = F;
    fa.rec = static_cast<double*>(ctx->rec.p);
    fa.partial = static_cast<double*>(ctx->partial.p);
    fa.nchunk = ctx->nchunk;
    MB_CUDA(launch_forces(st, 1, ctx->max_box_blobs, fa, g, ctx->bg, true));
    MB_CUDA(launch_spread<double>(st, 1, static_cast<const double*>(ctx->rec.p),
                                  static_cast<const int32_t*>(ctx->cell_start.p), g, ctx->bg,
                                  ctx->tile, f));
    FluidArgs<double> fl = fluid_args<double>(ctx, vn, f, vp, ctx->prof_scratch.p, body_force, nullptr);
    MB_CUDA(launch_fluid3<double>(st, 1, g, fl));
    MB_CUDA(launch_axpby(st, n3N, 0.5, vn, 0.5, vp, w));
    // ---- backward
    // corrector q^{n+1} = q^n + dt J(q^{n+1/2}) w
    MB_CUDA(launch_axpby(st, 3 * nb, dt, gq, 0.0, nullptr, guc));
    MB_CUDA(launch_make_rec(st, nb, static_cast<const int32_t*>(ctx->sorted.p), qh, guc,
                            static_cast<double*>(ctx->rec.p)));
    MB_CUDA(launch_spread<double>(st, 1, static_cast<const double*>(ctx->rec.p),
                                  static_cast<const int32_t*>(ctx->cell_start.p), g, ctx->bg,
                                  ctx->tile, gw));
    MB_CUDA(launch_axpby(st, n3N, h3, gw, 0.0, nullptr, gw));                 // gw = J^T guc
    MB_CUDA(launch_grad_interp(st, nb, qh, w, guc, g, 1.0, gqh));
    MB_CUDA(launch_axpby(st, n3N, 1.0, gvp, 0.5, gw, gvp));                  // dL/dv^{n+1}
    // fluid update v^{n+1} = A v^n + T f (A, T symmetric)
    FluidArgs<double> fa1 = fluid_args<double>(ctx, gvp, nullptr, tmp, nullptr, nullptr, nullptr);
    MB_CUDA(launch_fluid3<double>(st, 1, g, fa1));                           // A gvp
    MB_CUDA(launch_axpby(st, n3N, 1.0, tmp, 0.5, gw, gvn));                  // + gw/2
    FluidArgs<double> fa2 = fluid_args<double>(ctx, ctx->a_zero.p, gvp, gf, nullptr, nullptr, nullptr);
    MB_CUDA(launch_fluid3<double>(st, 1, g, fa2));                           // T gvp
    // spreading f = S(q^{n+1/2}) F
    MB_CUDA(launch_interp<double>(st, 0, nb, qh, nullptr, gf, nullptr, nullptr, g, dt, gF, nullptr));
    MB_CUDA(launch_axpby(st, 3 * nb, 1.0 / h3, gF, 0.0, nullptr, gF));       // gF = S^T gf
    MB_CUDA(launch_grad_interp(st, nb, qh, gf, F, g, 1.0 / h3, gqh));
    // forces F(q^{n+1/2}; k)
    double* gk_dev = static_cast<double*>(ctx->a_gk.p);
    MB_CUDA(launch_force_jvp(st, nb, qh, gF, static_cast<const int32_t*>(ctx->pid.p),
                             static_cast<const int32_t*>(ctx->adj_start.p),
                             static_cast<const int32_t*>(ctx->adj_j.p),
                             static_cast<const double*>(ctx->adj_rest.p), bx.k_spring, bx.k_rep,
                             bx.r_cut, static_cast<const int32_t*>(ctx->cell_start.p),
                             static_cast<const int32_t*>(ctx->sorted.p),
                             static_cast<const int32_t*>(ctx->blob_cell.p), g, ctx->bg, gqh, gk_dev));
    // predictor q^{n+1/2} = q^n + dt/2 J(q^n) v^n
    MB_CUDA(launch_axpby(st, 3 * nb, 1.0, gq, 1.0, gqh, gq));
    MB_CUDA(launch_axpby(st, 3 * nb, 0.5 * dt, gqh, 0.0, nullptr, gu));
    MB_TRY(velocity_adjoint_dev(ctx, qn, vn, gu, gq, gvn));
    // ---- outputs
    MB_TRY(push(ctx, grad_pos, ctx->a_gq, bv));
    MB_TRY(push(ctx, grad_v, ctx->a_gvn, bg));
    if (grad_k_spring) {
        double gk = 0.0;
        MB_CUDA(cudaMemcpyAsync(&gk, gk_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
        MB_CUDA(cudaStreamSynchronize(st));
        double prev = 0.0;
        MB_CUDA(cudaMemcpy(&prev, grad_k_spring, sizeof(double), cudaMemcpyDefault));
        prev += gk;
        MB_CUDA(cudaMemcpy(grad_k_spring, &prev, sizeof(double), cudaMemcpyDefault));
    }
    ctx->steps_taken = 0;     // the recomputation overwrote the last step's forces
    return MB_OK;
}

mb_status mb_get_tuning(const mb_ctx* ctx, int* spread_tile, float* spread_ms)
{
    if (!ctx) return MB_EINVAL;
    if (spread_tile)
        for (int d = 0; d < 3; ++d) spread_tile[d] = ctx->tile[d];
    if (spread_ms) *spread_ms = ctx->tile_ms;
    return MB_OK;
}

mb_status mb_get_counts(const mb_ctx* ctx, int64_t* total_blobs, int64_t* total_particles)
{
    if (!ctx) return MB_EINVAL;
    int64_t nb = 0, np = 0;
    for (const BoxData& b : ctx->boxes) {
        nb += (int64_t)b.pid.size();
        np += b.np;
    }
    if (total_blobs) *total_blobs = nb;
    if (total_particles) *total_particles = np;
    return MB_OK;
}

static mb_status blob_velocities(mb_ctx* ctx)
{
    if (ctx->nb == 0) return MB_OK;
    if (ctx->rsz == 4 && ctx->pred_ready)      // the last step's fused pass gathered them
        MB_CUDA(launch_forces_to_fp64(ctx->st, ctx->nb, static_cast<const float4*>(ctx->u32.p),
                                      static_cast<double*>(ctx->u.p)));
    else if (ctx->rsz == 4)
        MB_CUDA(launch_interp32(ctx->st, 0, ctx->nb, static_cast<const float4*>(ctx->sA.p),
                                static_cast<const float4*>(ctx->sB.p),
                                static_cast<const float*>(ctx->v[ctx->cur].p), nullptr,
                                static_cast<const int32_t*>(ctx->box_of.p), ctx->g, ctx->bg,
                                (float)ctx->d.dt, nullptr, nullptr, nullptr, nullptr,
                                static_cast<double*>(ctx->u.p)));
    else
        MB_CUDA(launch_interp<double>(ctx->st, 0, ctx->nb, static_cast<const double*>(ctx->q.p),
                                      nullptr, static_cast<const double*>(ctx->v[ctx->cur].p),
                                      nullptr, static_cast<const int32_t*>(ctx->box_of.p),
                                      ctx->g, ctx->d.dt, static_cast<double*>(ctx->u.p), nullptr));
    return MB_OK;
}

mb_status mb_get_velocities(mb_ctx* ctx, double* blob_vel, double* blob_pos, double* particle_U,
                            void* grid_v)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    MB_TRY(ensure_ready(ctx));
    if (blob_pos || particle_U) MB_TRY(current_positions(ctx));
    // FP32 grid after a fused step: the velocities were gathered by that step's last pass
    const bool gathered = ctx->rsz == 4 && ctx->pred_ready;
    if (particle_U || (blob_vel && !gathered)) MB_TRY(blob_velocities(ctx));
    if (blob_vel && ctx->nb > 0) {
        void* dst;
        bool host;
        const size_t by = sizeof(double) * 3 * ctx->nb;
        MB_TRY(out_target(ctx, blob_vel, by, ctx->staging_out, &dst, &host, "blob_vel"));
        if (gathered)
            MB_CUDA(launch_forces_to_fp64(ctx->st, ctx->nb, static_cast<const float4*>(ctx->u32.p),
                                          static_cast<double*>(dst)));
        else
            MB_CUDA(cudaMemcpyAsync(dst, ctx->u.p, by, cudaMemcpyDeviceToDevice, ctx->st));
        MB_TRY(finish_out(ctx, blob_vel, dst, by, host));
    }
    if (blob_pos && ctx->nb > 0) {
        void* dst;
        bool host;
        const size_t by = sizeof(double) * 3 * ctx->nb;
        MB_TRY(out_target(ctx, blob_pos, by, ctx->staging_out, &dst, &host, "blob_pos"));
        MB_CUDA(cudaMemcpyAsync(dst, ctx->q.p, by, cudaMemcpyDeviceToDevice, ctx->st));
        MB_TRY(finish_out(ctx, blob_pos, dst, by, host));
    }
    if (particle_U && ctx->np > 0) {
        void* dst;
        bool host;
        const size_t by = sizeof(double) * 3 * ctx->np;
        MB_TRY(out_target(ctx, particle_U, by, ctx->staging_out, &dst, &host, "particle_U"));
        MB_CUDA(launch_particle_reduce(ctx->st, ctx->np,
                                       static_cast<const int32_t*>(ctx->part_start.p),
                                       static_cast<const int32_t*>(ctx->part_blobs.p), nullptr,
                                       static_cast<const double*>(ctx->q.p),
                                       static_cast<const double*>(ctx->u.p), ctx->g,
                                       static_cast<double*>(dst), nullptr));
        MB_TRY(finish_out(ctx, particle_U, dst, by, host));
    }
    if (grid_v) {
        void* dst;
        bool host;
        const size_t by = grid_bytes(ctx, ctx->B);
        MB_TRY(out_target(ctx, grid_v, by, ctx->staging_out, &dst, &host, "grid_v"));
        MB_CUDA(cudaMemcpyAsync(dst, ctx->v[ctx->cur].p, by, cudaMemcpyDeviceToDevice, ctx->st));
        MB_TRY(finish_out(ctx, grid_v, dst, by, host));
    }
    return MB_OK;
}

mb_status mb_get_particle_velocities(mb_ctx* ctx, double* particle_U, double* particle_Omega)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    MB_TRY(ensure_ready(ctx));
    if (ctx->np == 0 || (!particle_U && !particle_Omega)) return MB_OK;
    MB_TRY(current_positions(ctx));
    MB_TRY(blob_velocities(ctx));
    const size_t by = sizeof(double) * 3 * ctx->np;
    void *dU = nullptr, *dW = nullptr;
    bool hU = false, hW = false;
    if (particle_U) MB_TRY(out_target(ctx, particle_U, by, ctx->staging_out, &dU, &hU, "U"));
    if (particle_Omega) MB_TRY(out_target(ctx, particle_Omega, by, ctx->s_out, &dW, &hW, "Omega"));
    MB_CUDA(launch_particle_reduce(ctx->st, ctx->np, static_cast<const int32_t*>(ctx->part_start.p),
                                   static_cast<const int32_t*>(ctx->part_blobs.p), nullptr,
                                   static_cast<const double*>(ctx->q.p),
                                   static_cast<const double*>(ctx->u.p), ctx->g,
                                   static_cast<double*>(dU), static_cast<double*>(dW)));
    if (particle_U) MB_TRY(finish_out(ctx, particle_U, dU, by, hU));
    if (particle_Omega) MB_TRY(finish_out(ctx, particle_Omega, dW, by, hW));
    return MB_OK;
}

mb_status mb_set_velocity_field(mb_ctx* ctx, const void* grid_v)
{
    if (!ctx) return MB_EINVAL;
    if (!grid_v) return invalid(ctx, "grid_v must be non-null");
    DeviceGuard dg(ctx->device);
    const size_t by = grid_bytes(ctx, ctx->B);
    const void* src;
    MB_TRY(stage_in(ctx, grid_v, by, ctx->staging_in, &src, "grid_v"));
    MB_CUDA(cudaMemcpyAsync(ctx->v[ctx->cur].p, src, by, cudaMemcpyDeviceToDevice, ctx->st));
    ctx->pred_ready = false;              // the next predictor must see the new field
    if (ctx->rsz == 4)
        MB_CUDA(launch_grid_mean<float>(ctx->st, ctx->B, ctx->g, static_cast<const float*>(ctx->v[ctx->cur].p),
                                        static_cast<double*>(ctx->vbar.p), nullptr));
    else
        MB_CUDA(launch_grid_mean<double>(ctx->st, ctx->B, ctx->g, static_cast<const double*>(ctx->v[ctx->cur].p),
                                         static_cast<double*>(ctx->vbar.p), nullptr));
    if (ctx->d.mean_mode == 1)
        MB_CUDA(cudaMemsetAsync(ctx->vbar.p, 0, sizeof(double) * 3 * ctx->B, ctx->st));
    MB_CUDA(cudaStreamSynchronize(ctx->st));
    return MB_OK;
}

mb_status mb_spread(mb_ctx* ctx, int64_t n, const double* pos, const double* F, void* grid_out)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (n < 0 || (n > 0 && (!pos || !F)) || !grid_out) return invalid(ctx, "bad spread arguments");
    const void *qd = nullptr, *Fd = nullptr;
    if (n > 0) {
        MB_TRY(stage_in(ctx, pos, sizeof(double) * 3 * n, ctx->s_g0, &qd, "pos"));
        MB_TRY(stage_in(ctx, F, sizeof(double) * 3 * n, ctx->s_F, &Fd, "F"));
    }
    const size_t by = grid_bytes(ctx, 1);
    void* dst;
    bool host;
    MB_TRY(out_target(ctx, grid_out, by, ctx->s_out, &dst, &host, "grid_out"));
    if (ctx->rsz == 4)
        MB_TRY(standalone_spread<float>(ctx, n, static_cast<const double*>(qd),
                                        static_cast<const double*>(Fd), static_cast<float*>(dst)));
    else
        MB_TRY(standalone_spread<double>(ctx, n, static_cast<const double*>(qd),
                                         static_cast<const double*>(Fd), static_cast<double*>(dst)));
    return finish_out(ctx, grid_out, dst, by, host);
}

mb_status mb_interp(mb_ctx* ctx, int64_t n, const double* pos, const void* grid_v, double* u_out)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    if (n < 0 || (n > 0 && (!pos || !u_out)) || !grid_v) return invalid(ctx, "bad interp arguments");
    if (n == 0) return MB_OK;
    const void *qd = nullptr, *vd = nullptr;
    MB_TRY(stage_in(ctx, pos, sizeof(double) * 3 * n, ctx->s_g0, &qd, "pos"));
    MB_TRY(ensure(ctx->s_q, sizeof(double) * 3 * n, ctx->err, "interp q"));
    double* q = static_cast<double*>(ctx->s_q.p);
    MB_CUDA(cudaMemcpyAsync(q, qd, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, ctx->st));
    k_wrap<<<(unsigned)((3 * n + 255) / 256), 256, 0, ctx->st>>>(n, q, ctx->g.L[0], ctx->g.L[1],
                                                                  ctx->g.L[2]);
    MB_CUDA(cudaGetLastError());
    MB_TRY(stage_in(ctx, grid_v, grid_bytes(ctx, 1), ctx->s_g1, &vd, "grid_v"));
    const size_t by = sizeof(double) * 3 * n;
    void* dst;
    bool host;
    MB_TRY(out_target(ctx, u_out, by, ctx->s_out, &dst, &host, "u_out"));
    if (ctx->rsz == 4)
        MB_CUDA(launch_interp<float>(ctx->st, 0, n, q, nullptr, static_cast<const float*>(vd),
                                     nullptr, nullptr, ctx->g, ctx->d.dt,
                                     static_cast<double*>(dst), nullptr));
    else
        MB_CUDA(launch_interp<double>(ctx->st, 0, n, q, nullptr, static_cast<const double*>(vd),
                                      nullptr, nullptr, ctx->g, ctx->d.dt,
                                      static_cast<double*>(dst), nullptr));
    return finish_out(ctx, u_out, dst, by, host);
}

mb_status mb_fluid_update(mb_ctx* ctx, const void* v_in, const void* f, const double* body_force,
                          void* v_out)
{
    if (!ctx) return MB_EINVAL;
    DeviceGuard dg(ctx->device);
    const bool stokes = ctx->d.integrator == 1;
    if ((!v_in && !stokes) || !v_out) return invalid(ctx, "v_in and v_out must be non-null");
    const size_t by = grid_bytes(ctx, 1);
    const void *vd = nullptr, *fd = nullptr;
    if (!stokes) MB_TRY(stage_in(ctx, v_in, by, ctx->s_g1, &vd, "v_in"));
    if (f) MB_TRY(stage_in(ctx, f, by, ctx->s_g2, &fd, "f"));
    if (ctx->advect) {
        // f - rho D.(v_in v_in) in the library's own copy (the caller's f is not written)
        MB_TRY(ensure(ctx->s_g2, by, ctx->err, "f"));
        if (fd && fd != ctx->s_g2.p)
            MB_CUDA(cudaMemcpyAsync(ctx->s_g2.p, fd, by, cudaMemcpyDeviceToDevice, ctx->st));
        MB_TRY(ensure(ctx->W, 3 * by, ctx->err, "fluid stress"));
        if (ctx->rsz == 4)
            MB_CUDA(launch_fluid_stress<float>(ctx->st, 1, ctx->g, 0, nullptr, 0.0,
                                               static_cast<const float*>(vd), ctx->d.rho,
                                               static_cast<float*>(ctx->W.p),
                                               static_cast<float*>(ctx->s_g2.p), fd != nullptr));
        else
            MB_CUDA(launch_fluid_stress<double>(ctx->st, 1, ctx->g, 0, nullptr, 0.0,
                                                static_cast<const double*>(vd), ctx->d.rho,
                                                static_cast<double*>(ctx->W.p),
                                                static_cast<double*>(ctx->s_g2.p), fd != nullptr));
        fd = ctx->s_g2.p;
    }
    if (body_force) MB_TRY(set_body(ctx, body_force, ctx->prof_scratch, false));
    void* dst;
    bool host;
    MB_TRY(out_target(ctx, v_out, by, ctx->s_out, &dst, &host, "v_out"));
    auto stokes_args = [&](auto& a) {
        a.v = a.v_out;                      // unread: the right-hand side is f + f_body
        a.no_v = 1;
        a.rho_dt = 0.0;
        a.half_eta = ctx->d.eta;
    };
    if (ctx->rsz == 4) {
        FluidArgs<float> a = fluid_args<float>(ctx, vd, fd, dst, ctx->prof_scratch.p, body_force, nullptr);
        if (stokes) stokes_args(a);
        if (ctx->fft_passes == 5) MB_CUDA(launch_fluid<float>(ctx->st, 1, ctx->g, a));
        else MB_CUDA(launch_fluid3<float>(ctx->st, 1, ctx->g, a));
    } else {
        FluidArgs<double> a = fluid_args<double>(ctx, vd, fd, dst, ctx->prof_scratch.p, body_force, nullptr);
        if (stokes) stokes_args(a);
        if (ctx->fft_passes == 5) MB_CUDA(launch_fluid<double>(ctx->st, 1, ctx->g, a));
        else MB_CUDA(launch_fluid3<double>(ctx->st, 1, ctx->g, a));
    }
    return finish_out(ctx, v_out, dst, by, host);
}

}  // extern "C"
