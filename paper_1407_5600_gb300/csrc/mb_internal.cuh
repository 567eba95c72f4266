// Internal declarations shared by the translation units of libmb.so.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mb.h"

namespace mbk {

// ------------------------------------------------------------------------------------------
// Geometry passed by value to kernels.
struct GridGeo {
    int n[3];          // cells per side (powers of two)
    int64_t N;         // cells per box
    double h, inv_h;
    double L[3];
    float inv_h32, L32[3];   // the same rounded to float on the host (FP32 blob kernels: no
                             // per-thread conversions on GB300's narrow FP64 pipe)
};

struct BinGeo {
    int nc[3];         // bin cells per side
    int64_t ncell;     // bin cells per box
    int bs;            // bin cell side in mesh cells
    double inv_w;      // 1 / (bs h)
    double w;          // 1 / inv_w (the cell side), and its float rounding; set with inv_w
    float w32;
};

// The float copies of the geometry, from the double fields.
inline void set_float_geo(GridGeo& g)
{
    g.inv_h32 = (float)g.inv_h;
    for (int d = 0; d < 3; ++d) g.L32[d] = (float)g.L[d];
}
inline void set_float_geo(BinGeo& bg)
{
    bg.w = 1.0 / bg.inv_w;
    bg.w32 = (float)bg.w;
}

// True the first time it is called for the current device with this flag set (function
// attributes such as the dynamic shared-memory limit are set once per device).
inline bool first_on_device(std::atomic<unsigned>& done)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned bit = 1u << (dev & 31);
    return (done.fetch_or(bit) & bit) == 0;
}

// Complex helpers on float2 / double2.
template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

// ------------------------------------------------------------------------------------------
// Launchers (each returns cudaGetLastError() after enqueuing).

// Interpolation J of one or two grids at blob positions q.
//   mode 0: u_out = J(q) v0
//   mode 1: u_out = J(q) v0, q_out = wrap(q + 0.5 dt u)            (predictor)
//   mode 2: u = J(q) (v0 + v1)/2, q_out = wrap(q_base + dt u), u_out = u if non-null (corrector)
template <typename R>
cudaError_t launch_interp(cudaStream_t st, int mode, int64_t nb, const double* q,
                          const double* q_base, const R* v0, const R* v1,
                          const int32_t* box_of, const GridGeo& g, double dt, double* u_out,
                          double* q_out);

// Cell binning: count, scan, scatter (and per-cell ordering when deterministic).
cudaError_t launch_bin(cudaStream_t st, int64_t nb, const double* q, const int32_t* box_of,
                       int B, const BinGeo& bg, int32_t* cell_count, int32_t* cell_start,
                       int32_t* blob_cell, int32_t* blob_rank, int32_t* sorted,
                       int32_t* scan_tmp, bool deterministic, const int32_t* pid = nullptr,
                       float4* loc = nullptr);

// Blob forces at q (springs, repulsion, external) in sorted-slot order; writes F (blob order),
// rec (sorted order: q, F) and per-(box, block) partial force sums.
struct ForceArgs {
    const int64_t* box_off;    // [B+1]
    const int32_t* sorted;
    const double* q;
    const int32_t* pid;        // global particle ids
    const int32_t* adj_start;  // [nb+1]
    const int32_t* adj_j;
    const double* adj_rest;
    const double* box_par;     // [B][3]: k_spring, k_rep, r_cut
    const int32_t* cell_start;
    const int32_t* blob_cell;
    const double* ext;         // may be null
    const float4* loc;         // [nb] sorted-order cell-local coordinates and particle id
    double* F;
    double* rec;
    double* partial;           // [B][nchunk][3]
    int nchunk;
    // [nb][3] external plus spring forces already summed (launch_springs64); null: the kernel
    // sums them from ext and the adjacency lists
    const double* Fpre;
};
// precise: FP64 in the plain operation order without contraction (FP64 grid mode).
cudaError_t launch_forces(cudaStream_t st, int B, int64_t max_box_blobs, const ForceArgs& a,
                          const GridGeo& g, const BinGeo& bg, bool precise);

// FP64 spring forces when every particle shares one bond pattern (m blobs, blob l of particle
// p is blob p m + l): each bond evaluated once, in the precise FP64 order, by the end the
// pattern names, and each blob's sum Fout = ext + the bonds in its adjacency order, so the
// result has the bits of the per-blob evaluation of launch_forces (the two ends' evaluations
// are exact negatives).  tmpl: per local blob an evaluation list {offset | (slot + 1) << 16,
// r0 low word, r0 high word, 0} and a sum list in adjacency order {offset of the evaluating
// blob, slot, sign, 0}; tstart[2l], tstart[2l + 1], tstart[2l + 2] bound them.
cudaError_t launch_springs64(cudaStream_t st, int64_t nb, int m, int slots, const double* q,
                             const double* ext, const int4* tmpl, const int32_t* tstart,
                             const int32_t* box_of, const double* box_par, const GridGeo& g,
                             double* Fout);

// Sum partial forces per box (fixed order) and update the FP64 mean velocity:
// vbar += dt * sumF / (rho L^3) when mean_mode == 0, vbar = 0 otherwise; optionally copies
// the force sum to fsum_out [B][3].
cudaError_t launch_force_sum(cudaStream_t st, int B, int nchunk, const double* partial,
                             double* vbar, double scale, int mean_mode, double* fsum_out);

// Sorted records from arbitrary q, F (standalone spreading).
cudaError_t launch_make_rec(cudaStream_t st, int64_t nb, const int32_t* sorted, const double* q,
                            const double* F, double* rec);

// Tile-owner spreading from sorted records.
template <typename R>
cudaError_t launch_spread(cudaStream_t st, int B, const double* rec, const int32_t* cell_start,
                          const GridGeo& g, const BinGeo& bg, const int tile[3], R* f);

// Blob-owner spreading with global atomic adds into f (zeroed by the launcher).
template <typename R>
cudaError_t launch_spread_atomic(cudaStream_t st, int B, int64_t max_box_blobs, const double* rec,
                                 const int32_t* cell_start, const GridGeo& g, const BinGeo& bg,
                                 R* f);

// Deterministic FP64 spreading (64-bit fixed-point shared-memory accumulation).
cudaError_t launch_spread_det(cudaStream_t st, int B, const double* rec, const int32_t* cell_start,
                              const GridGeo& g, const BinGeo& bg, const int tile[3], double* f);

// Particle velocities U0, Omega from blob velocities (particle CSR).
cudaError_t launch_particle_reduce(cudaStream_t st, int64_t np, const int32_t* part_start,
                                   const int32_t* part_blobs, const int32_t* box_of_part,
                                   const double* q, const double* u, const GridGeo& g,
                                   double* U, double* Omega);

// Adjoint of U0 = (1/N_p) sum_i u_i: gu[i] = gU[p(i)] / N_p for every blob of every particle.
cudaError_t launch_particle_mean_adjoint(cudaStream_t st, int64_t np, const int32_t* part_start,
                                         const int32_t* part_blobs, const double* gU,
                                         double* gu);

// Fluid update pipeline on B boxes.
template <typename R>
struct FluidArgs {
    const R* v;            // [B][3][N]
    const R* f;            // [B][3][N] or null
    typename C2<R>::T* spec;   // [B][3][nz][ny][nx/2+1]
    R* v_out;
    const R* tw[3];        // twiddles per dimension, n/2 complex each (interleaved re, im)
    const R* twf[3];       // full tables W_n^j, j < n, per dimension (interleaved re, im)
    const double* sym;     // [3 dims][3][256]: cos, sin, lambda of 2 pi k / n (FP64)
    const void* symr;      // the same tables in the grid precision R
    // the full twiddle tables and the symbols in the three-pass FFT's arithmetic type (the
    // grid precision, or double-float for FP64 grids)
    const void* twk[3];
    const void* symk;
    const R* body_prof;    // body-force profile along wave_dir (null = none)
    int body_axis, body_dir;
    const double* mean_override;   // [B][3] mean velocity to impose at k = 0, or null
    int mean_mode;
    double rho_dt, half_eta;
    double inv_h, inv_h2, inv_n;          // 1/h, 1/h^2, 1/N (set by the launch functions)
    // the five rounded to float on the host: FP32 kernels read these instead of converting
    // per thread on GB300's narrow FP64 pipe
    float rho_dt32, half_eta32, inv_h32, inv_h2_32, inv_n32;
    R* f_clear;            // three-pass FFT: f, zeroed as it is read (null = leave f alone)
    const R* v_sum_base;   // three-pass FFT: v^n; with v_sum_out, also write v^n + v^{n+1}
    R* v_sum_out;
    // three-pass FFT, mean_mode 0: the FP64 mean velocity [B][3], advanced in place by the
    // k = 0 thread (mean_state += mean_scale * mean_force, force optional) and imposed at k = 0
    double* mean_state;
    const double* mean_force;
    double mean_scale;
    int no_v;              // three-pass FFT: right-hand side f (+ body) only (Stokes limit)
};
// marks: null, or 6 events recorded before pass 1 and after each of the 5 passes.
// The derived launch constants of a FluidArgs (1/h, 1/h^2, 1/N and the float roundings), set
// by the launch functions from the final rho_dt and half_eta.
template <typename R> inline FluidArgs<R> with_derived(const FluidArgs<R>& in, const GridGeo& g)
{
    FluidArgs<R> a = in;
    a.inv_h = g.inv_h;
    a.inv_h2 = g.inv_h * g.inv_h;
    a.inv_n = 1.0 / (double)g.N;
    a.rho_dt32 = (float)a.rho_dt;
    a.half_eta32 = (float)a.half_eta;
    a.inv_h32 = (float)a.inv_h;
    a.inv_h2_32 = (float)a.inv_h2;
    a.inv_n32 = (float)a.inv_n;
    return a;
}

// A per-launch constant in the arithmetic type K: the host's float rounding for FP32
// arithmetic, otherwise converted from the double.
template <typename K> __device__ __forceinline__ K kparam(double d, float) { return K(d); }
template <> __device__ __forceinline__ float kparam<float>(double, float f) { return f; }

// ------------------------------------------------------------------------------------------
// Programmatic dependent launch for the chain of kernels of one step.  A kernel launched with
// launch_dep may be scheduled while the kernel before it on the stream is still draining its
// last blocks; it must call dep_wait() before its first access to global memory (and before
// any early return), which returns once every prerequisite grid has completed and its writes
// are visible.  dep_release() lets the next kernel of the chain be scheduled once every block
// of this one has started: its blocks then occupy only the slots this kernel's finished blocks
// free, and wait there.  Both are no-ops for a kernel launched the ordinary way, so the same
// kernels serve direct launches.  MB_PDL=0 launches the chain the ordinary way.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

bool pdl_enabled();

template <typename... P, typename... A>
inline cudaError_t launch_dep(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, A&&... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <typename R>
cudaError_t launch_fluid(cudaStream_t st, int B, const GridGeo& g, const FluidArgs<R>& a,
                         cudaEvent_t* marks = nullptr);
constexpr int FLUID_KERNELS = 5;
// Three-pass variant (plane R2C, z solve, plane C2R); marks as for launch_fluid, with the
// y-pass marks recorded back to back.
template <typename R>
cudaError_t launch_fluid3(cudaStream_t st, int B, const GridGeo& g, const FluidArgs<R>& a,
                          cudaEvent_t* marks = nullptr);
constexpr int FLUID3_KERNELS = 3;

// Thermal and convective stress (kernels_noise.cu): W = amp * normals of step *step_index
// (amp != 0) + rho v v (v != NULL) [parts & 1], then f (+)= -D.W and *step_index += 1
// (amp != 0) [parts & 2].  W is [B][9][N], v and f [B][3][N].
template <typename R>
cudaError_t launch_fluid_stress(cudaStream_t st, int B, const GridGeo& g, uint64_t seed,
                                uint64_t* step_index, double amp, const R* v, double rho, R* W,
                                R* f, bool accumulate, int parts = 3);
constexpr int STRESS_KERNELS = 2;

// Exclusive scan of n ints into out[0..n] (out[n] = total); tile_tmp holds n/4096 + 2 ints.
cudaError_t launch_exclusive_scan(cudaStream_t st, const int32_t* in, int32_t* out, int64_t n,
                                  int32_t* tile_tmp);

// FP32-grid blob pipeline (kernels_blob32.cu): positions as bin cell + float-float offset,
// A = {hi.xyz, packed cell}, B = {lo.xyz, 0} per blob.
cudaError_t launch_split(cudaStream_t st, int64_t nb, const double* q, const GridGeo& g,
                         const BinGeo& bg, float4* A, float4* B);
cudaError_t launch_unsplit(cudaStream_t st, int64_t nb, const float4* A, const float4* B,
                           const GridGeo& g, const BinGeo& bg, double* q);
cudaError_t launch_interp32(cudaStream_t st, int mode, int64_t nb, const float4* A,
                            const float4* B, const float* v0, const float* v1,
                            const int32_t* box_of, const GridGeo& g, const BinGeo& bg, float dt,
                            const float4* A_base, const float4* B_base, float4* A_out,
                            float4* B_out, double* u_out, const int32_t* order = nullptr,
                            int32_t* count = nullptr, int32_t* blob_cell = nullptr,
                            int32_t* blob_rank = nullptr);
// Corrector of step n and predictor of step n + 1 in one pass (blob counts into `count`,
// which must be zero).  Mode-2 + mode-1 semantics of launch_interp32: the corrector gathers
// (v0 + v1) / 2 (v1 may be null when v0 already holds v^n + v^{n+1}), the predictor vp; the
// predictor's velocities (those of the new state) go to u_out.
cudaError_t launch_interp32_fused(cudaStream_t st, int64_t nb, const float4* A, const float* v0,
                                  const float* v1, const float* vp, const int32_t* box_of,
                                  const GridGeo& g,
                                  const BinGeo& bg, float dt, const float4* A_base,
                                  const float4* B_base, float4* A_out, float4* B_out,
                                  float4* Ah_out, float4* Bh_out, const int32_t* order,
                                  int32_t* count, int32_t* blob_cell, int32_t* blob_rank,
                                  float4* u_out);
cudaError_t launch_bin32(cudaStream_t st, int64_t nb, const float4* A, const int32_t* box_of,
                         int Bx, const BinGeo& bg, int32_t* cell_count, int32_t* cell_start,
                         int32_t* blob_cell, int32_t* blob_rank, int32_t* sorted,
                         int32_t* scan_tmp, const int32_t* pid, float4* loc,
                         bool counted = false);
// The bonds of the FP32 spring kernels.  A bond between a blob of at most SPRING_LOCAL_MAX
// bonds and a heavier one (an icosahedron's vertex and centre) is evaluated by the light end
// only, which also supplies the heavy end's opposite force.
//   adj / adj_start: per-blob lists {j (sign bit: also add the opposite force to j), r0,
//   r0^2 as float hi + lo}; bonds between two light or two heavy blobs are evaluated at both
//   ends.
//   tmpl / tstart: when every particle has the same m blobs under one bond pattern (blob l of
//   particle p is blob p m + l; the same partners, as offsets inside the particle, and the same
//   rest lengths in every particle), the pattern once, each bond evaluated once: per local
//   blob l an evaluation list and a collection list (k_springs32_shared), and `slots`
//   evaluations per blob at most.
constexpr int SPRING_LOCAL_MAX = 6;
struct Springs32 {
    const int4* adj;
    const int32_t* adj_start;
    const int4* tmpl;          // null: no common pattern
    const int32_t* tstart;     // [2 m + 1]
    int m;
    int slots;
};
cudaError_t launch_forces32(cudaStream_t st, int Bx, int64_t nb, int64_t max_box_blobs,
                            const int64_t* box_off, const int32_t* sorted, const float4* A,
                            const float4* B, const float4* loc, const Springs32& sp,
                            const int32_t* box_of,
                            const float* box_par, const int32_t* cell_start,
                            const int32_t* blob_cell, const float4* ext, float4* Fs, float4* F,
                            float4* rec, const GridGeo& g, const BinGeo& bg);
// The two halves of launch_forces32, for running the springs on another stream: the spring
// forces (Fs), then the pair forces, sums and sorted records.
cudaError_t launch_springs32(cudaStream_t st, int64_t nb, const float4* A, const float4* B,
                             const Springs32& sp, const int32_t* box_of,
                             const float* box_par, const GridGeo& g, const BinGeo& bg, float4* Fs);
cudaError_t launch_pairs32(cudaStream_t st, int Bx, int64_t max_box_blobs,
                           const int64_t* box_off, const int32_t* sorted, const float4* A,
                           const float4* B, const float4* loc, const int32_t* box_of,
                           const float* box_par, const int32_t* cell_start,
                           const int32_t* blob_cell, const float4* ext, const float4* Fs,
                           float4* F, float4* rec, const GridGeo& g, const BinGeo& bg);
// f = S F from the binned records (zeroes f first unless the caller knows it is zero).  The tile (nodes per block) must satisfy
// spread32_tile_ok: at least 4 and whole bin cells per side, dividing the grid, at most 64 rows
// of cells and 32 cells along x, shared copy within 200 KiB; other tiles return
// cudaErrorInvalidValue.
bool spread32_tile_ok(const int tile[3], const GridGeo& g, const BinGeo& bg);
cudaError_t launch_spread32(cudaStream_t st, int Bx, const float4* rec, const int32_t* cell_start,
                            const GridGeo& g, const BinGeo& bg, const int tile[3], float* f,
                            bool f_is_zero = false);
// External forces to FP32 plus their per-box FP64 sums (partial: [B][chunks][3] scratch;
// ticket: one zeroed unsigned, left zero), in one launch.
cudaError_t launch_ext_prepare(cudaStream_t st, int Bx, int64_t max_box_blobs,
                               const int64_t* box_off, const double* ext, float4* ext32,
                               double* partial, double* ext_sum, unsigned* ticket);
cudaError_t launch_vbar_step(cudaStream_t st, int Bx, const double* sum, double scale,
                             int mean_mode, double* vbar);
cudaError_t launch_forces_to_fp64(cudaStream_t st, int64_t nb, const float4* F, double* out);

// Adjoint kernels (adjoint.cu), FP64.
cudaError_t launch_grad_interp(cudaStream_t st, int64_t nb, const double* q, const double* w,
                               const double* c, const GridGeo& g, double scale, double* out);
cudaError_t launch_force_jvp(cudaStream_t st, int64_t nb, const double* q, const double* gF,
                             const int32_t* pid, const int32_t* adj_start, const int32_t* adj_j,
                             const double* adj_rest, double k_spring, double k_rep, double r_cut,
                             const int32_t* cell_start, const int32_t* sorted,
                             const int32_t* blob_cell, const GridGeo& g, const BinGeo& bg,
                             double* out, double* gk);
cudaError_t launch_axpby(cudaStream_t st, int64_t n, double a, const double* x, double b,
                         const double* y, double* out);

// Reductions / utilities.
template <typename R>
cudaError_t launch_grid_mean(cudaStream_t st, int B, const GridGeo& g, const R* v,
                             double* mean_out /*[B][3]*/, double* scratch);

}  // namespace mbk
