/*
 * mbref — plain FP64 CPU oracle of the multiblob inertial-coupling (ICM) time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls
 * this code; only the tests, the package smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no source with the CUDA path.
 *
 * Every routine is written for clarity, not speed: fixed loop order, IEEE double,
 * no fast-math, no contraction (built with -ffp-contract=off).  Independent loops may run on
 * several host threads (OpenMP) without changing any result (mbref_set_threads).
 *
 * Paper: Vazquez-Quesada, Balboa Usabiaga, Delgado-Buscalioni, "A multiblob approach to
 * colloidal hydrodynamics with inherent lubrication" (arXiv:1407.5600).
 *
 * Conventions (shared with the C ABI only by specification, not by code):
 *   - Periodic box of nx*ny*nz cubic cells of side h; L_b = n_b*h.
 *   - Staggered (MAC) velocity: component a lives on the faces normal to a.
 *     v_x[k][j][i] sits at (i*h, (j+1/2)h, (k+1/2)h); v_y at ((i+1/2)h, j*h, (k+1/2)h);
 *     v_z at ((i+1/2)h, (j+1/2)h, k*h).
 *   - Grids are 3 component arrays stored one after another, each [nz][ny][nx], x fastest.
 *   - Blob arrays are [n][3] (x, y, z), row-major.
 */
#ifndef MBREF_H
#define MBREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double h;        /* mesh size */
    double rho;      /* fluid density rho_f */
    double eta;      /* shear viscosity */
    double dt;       /* time step */
    int mean_mode;   /* 0: the k=0 (mean) mode evolves with the net force; 1: it is held at 0 */
    int advection;   /* 1: the convective stress rho v v of Eq. (vf), explicit at v^n */
} mbref_grid;

/* Number of host threads the oracle's parallel loops use (n <= 0 leaves it unchanged);
 * returns the number in effect (1 when built without OpenMP).  Results do not depend on it. */
int mbref_set_threads(int n);

/* Three-point kernel Phi of Eq. (delta): the Roma-Peskin-Berger function. */
double mbref_phi(double r);

/* f = S F : spreading of blob forces onto the MAC grid (f_i = delta_h(r - q_i) F_i, Sec. 2). */
int mbref_spread(const mbref_grid* g, int64_t n, const double* q, const double* F, double* f);

/* u = J v : interpolation of the MAC velocity at the blobs (Eq. ju). */
int mbref_interp(const mbref_grid* g, int64_t n, const double* q, const double* v, double* u);

/* Unnormalised 3-D DFT  X(k) = sum_j x_j exp(-/+ 2 pi i k.j/n), in place on (re, im),
 * arrays [nz][ny][nx]; inverse != 0 selects the + sign (no 1/N factor). */
int mbref_dft3(int nx, int ny, int nz, double* re, double* im, int inverse);

/* One Crank-Nicolson + projection update of the fluid (Eq. vf with sigma = -eta E, m_e = 0):
 *   (rho/dt - eta/2 L) v_out = P [ (rho/dt + eta/2 L) v + f + f_body - rho D.(v v) ],
 * the last term only with g->advection (see mbref_advection).
 * body = {f0, axis, wave_dir, j} (force density f0 sin(2 pi j x_wave / L_wave) along axis)
 * or NULL. */
int mbref_fluid_update(const mbref_grid* g, const double* v, const double* f,
                       const double* body, double* v_out);

/* Steady Stokes solution v = P (-eta L)^-1 f with the mean mode set to zero. */
int mbref_stokes_solve(const mbref_grid* g, const double* f, double* v);

/* F += harmonic bond forces, F_i = -k (|r_ij| - r0) r_ij/|r_ij| (minimum image). */
int mbref_bond_forces(const mbref_grid* g, int64_t n, const double* q, int64_t nbonds,
                      const int32_t* bonds, const double* rest, double k, double* F);

/* F += soft blob-blob repulsion k_rep (r_cut - r) r_hat for r < r_cut, between blobs of
 * different particles.  Each blob sums over the blobs of the bins around it in ascending index
 * order, which gives the sum over all pairs (mbref_pair_forces_brute) to the bit. */
int mbref_pair_forces(const mbref_grid* g, int64_t n, const double* q, const int32_t* pid,
                      double k_rep, double r_cut, double* F);

/* The same repulsion by its definition: every blob sums over all other blobs in index order. */
int mbref_pair_forces_brute(const mbref_grid* g, int64_t n, const double* q, const int32_t* pid,
                            double k_rep, double r_cut, double* F);

/* Same repulsion, evaluated only for the m blobs listed in idx (F is [m][3], overwritten). */
int mbref_pair_forces_subset(const mbref_grid* g, int64_t n, const double* q,
                             const int32_t* pid, double k_rep, double r_cut, int64_t m,
                             const int64_t* idx, double* F);

/* Thermal stress of the fluctuating ICM (Sec. 3, the stress sigma~ of Eq. vf):
 * kT > 0 adds -D.sigma~, sigma~ = sqrt(2 eta kT/(h^3 dt)) W, to the force density of every
 * step; W is drawn per (seed, step index, box, cell) by mbref_stress_normals, the step index
 * of the s-th step of a call being step0 + s. */
typedef struct {
    double kT;
    uint64_t seed;
    uint64_t step0;
    int64_t box;
} mbref_noise;

/* Philox4x64-10 counter-based generator: out = Philox(ctr, key). */
void mbref_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* W [9][nz][ny][nx]: the standard normals of every cell (components xx, xy, xz, yx, yy, yz,
 * zx, zy, zz), from Philox keyed by (seed, step, box, group of four cells along x) with
 * Box-Muller.  nx must be a multiple of four. */
int mbref_stress_normals(const mbref_grid* g, uint64_t seed, uint64_t step, int64_t box,
                         double* W);

/* f [3][nz][ny][nx] = D.W, the MAC divergence of a stress field W [9][nz][ny][nx] placed
 * with W_aa at cell centres and W_ab on edges (overwrites f). */
int mbref_stress_div(const mbref_grid* g, const double* W, double* f);

/* out = D.(v v): the divergence of the convective tensor v_a v_b on the MAC grid, placed like
 * the thermal stress (v_a v_a at cell centres from the two face values of v_a averaged;
 * v_a v_b on the (a, b) edges from v_a averaged along b and v_b averaged along a), the
 * conservative centred form of the convective term of Eq. (vf). */
int mbref_advection(const mbref_grid* g, const double* v, double* out);

/* nsteps of the neutrally buoyant ICM step (midpoint blob update, CN fluid update),
 * updating q (wrapped into [0, L)) and v in place.  ext ([n][3]), body and noise may be
 * NULL. */
int mbref_step(const mbref_grid* g, int nsteps, int64_t n, double* q, double* v,
               const int32_t* pid, int64_t nbonds, const int32_t* bonds, const double* rest,
               double k_spring, double k_rep, double r_cut, const double* ext,
               const double* body, const mbref_noise* noise);

/* Stokes-limit steps (fluid inertia removed): explicit midpoint rule with the steady,
 * zero-mean Stokes flow of the current forces; v receives the last flow.  Same arguments as
 * mbref_step without the noise (rho and mean_mode of the grid are not used). */
int mbref_stokes_step(const mbref_grid* g, int nsteps, int64_t n, double* q, double* v,
                      const int32_t* pid, int64_t nbonds, const int32_t* bonds,
                      const double* rest, double k_spring, double k_rep, double r_cut,
                      const double* ext, const double* body);

/* Particle translational velocity U0 = mean of u_i (Sec. 2) and angular velocity
 * Omega = I0^-1 sum_i s_i x (u_i - U0) (Eqs. torque, miner0), for np particles whose
 * blobs carry particle ids 0..np-1. */
int mbref_particle_velocities(const mbref_grid* g, int64_t n, const double* q, const double* u,
                              const int32_t* pid, int64_t np, double* U, double* Omega);

#ifdef __cplusplus
}
#endif
#endif
