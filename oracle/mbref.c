/*
 * mbref.c — plain FP64 CPU oracle of the multiblob ICM time step.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, by the package smoke check and by the
 * benchmark's CPU-baseline leg; never by the product path.  It shares no source with the
 * CUDA library.  Written for a reader checking it against the paper, not for speed.
 *
 * Paper: arXiv:1407.5600.  Section, equation and table labels below are the paper's.
 */
#include "mbref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads.  Loops whose iterations write disjoint outputs and read only inputs (blobs of J,
 * pair forces of each blob, lines of the DFT, grid points of the stencils, cells of the noise,
 * components of S) may run on several threads; every output is computed by the same
 * operations in the same order as on one thread, so results do not depend on the thread
 * count.  Sums whose order would change with the split (bond forces, the particle sums) stay
 * serial. */
int mbref_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static const double MBREF_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------------------ */
/* Kernel (Eq. delta).  The paper builds delta_h = h^-3 prod_a Phi(r_a/h) from the
 * 3-point Peskin function of Roma, Peskin and Berger, whose defining properties it lists
 * (Sec. 2): sum_j Phi = 1, sum_j (j - x) Phi = 0 and sum_j Phi^2 = 1/2 at every offset.  */
double mbref_phi(double r)
{
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) {
        double b = 1.0 - a;
        return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * b * b)) / 6.0;
    }
    return 0.0;
}

/* Position of node index i of component comp along dimension dim, in units of h:
 * the MAC face of component comp is at integer index along comp, cell centre otherwise. */
static double node_shift(int comp, int dim) { return comp == dim ? 0.0 : 0.5; }

static int64_t wrap_index(int64_t i, int n)
{
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* The three nodes whose kernel weight can be non-zero (Phi vanishes for |r| >= 3/2):
 * nearest node i0 = floor(x + 1/2) and its two neighbours, x = q/h - shift. */
static void kernel_window(double q, double h, double shift, int n, int64_t idx[3], double w[3])
{
    double x = q / h - shift;
    double i0 = floor(x + 0.5);
    for (int d = 0; d < 3; ++d) {
        double node = i0 + (double)(d - 1);
        w[d] = mbref_phi(node - x);
        idx[d] = wrap_index((int64_t)node, n);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Spreading S (Sec. 2): f(r) = sum_i delta_h(r - q_i) F_i, evaluated at every MAC node. */
int mbref_spread(const mbref_grid* g, int64_t n, const double* q, const double* F, double* f)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const int64_t N = (int64_t)nx * ny * nz;
    const double inv_h3 = 1.0 / (g->h * g->h * g->h);
    memset(f, 0, sizeof(double) * 3 * N);
#pragma omp parallel for schedule(static)
    for (int comp = 0; comp < 3; ++comp) {
        for (int64_t b = 0; b < n; ++b) {
            int64_t ix[3], iy[3], iz[3];
            double wx[3], wy[3], wz[3];
            kernel_window(q[3 * b + 0], g->h, node_shift(comp, 0), nx, ix, wx);
            kernel_window(q[3 * b + 1], g->h, node_shift(comp, 1), ny, iy, wy);
            kernel_window(q[3 * b + 2], g->h, node_shift(comp, 2), nz, iz, wz);
            double* fc = f + comp * N;
            for (int c = 0; c < 3; ++c)
                for (int bb = 0; bb < 3; ++bb)
                    for (int a = 0; a < 3; ++a) {
                        double w = wx[a] * wy[bb] * wz[c] * inv_h3;
                        fc[(iz[c] * ny + iy[bb]) * nx + ix[a]] += w * F[3 * b + comp];
                    }
        }
    }
    return 0;
}

/* Interpolation J (Eq. ju): u_i = integral of delta_h(r - q_i) v(r) dr, the integral being
 * the sum over nodes times h^3, so u_i = sum_nodes prod Phi * v. */
int mbref_interp(const mbref_grid* g, int64_t n, const double* q, const double* v, double* u)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const int64_t N = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < n; ++b) {
        for (int comp = 0; comp < 3; ++comp) {
            int64_t ix[3], iy[3], iz[3];
            double wx[3], wy[3], wz[3];
            kernel_window(q[3 * b + 0], g->h, node_shift(comp, 0), nx, ix, wx);
            kernel_window(q[3 * b + 1], g->h, node_shift(comp, 1), ny, iy, wy);
            kernel_window(q[3 * b + 2], g->h, node_shift(comp, 2), nz, iz, wz);
            const double* vc = v + comp * N;
            double s = 0.0;
            for (int c = 0; c < 3; ++c)
                for (int bb = 0; bb < 3; ++bb)
                    for (int a = 0; a < 3; ++a)
                        s += wx[a] * wy[bb] * wz[c] * vc[(iz[c] * ny + iy[bb]) * nx + ix[a]];
            u[3 * b + comp] = s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Discrete Fourier transform.  One line of length n, stride s: X_k = sum_j x_j e^{-+2 pi i jk/n}.
 * Powers of two use the textbook iterative radix-2 Cooley-Tukey algorithm (bit-reversal
 * permutation, then log2 n butterfly stages, each twiddle evaluated directly by cos/sin);
 * any other length uses the O(n^2) definition. */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static void dft_line(double* re, double* im, int n, int64_t s, int inverse,
                     double* tr, double* ti)
{
    const double sgn = inverse ? 1.0 : -1.0;
    if (!is_pow2(n)) {
        for (int k = 0; k < n; ++k) {
            double ar = 0.0, ai = 0.0;
            for (int j = 0; j < n; ++j) {
                int64_t m = ((int64_t)j * k) % n;
                double ang = sgn * 2.0 * MBREF_PI * (double)m / (double)n;
                double c = cos(ang), sn = sin(ang);
                ar += re[j * s] * c - im[j * s] * sn;
                ai += re[j * s] * sn + im[j * s] * c;
            }
            tr[k] = ar;
            ti[k] = ai;
        }
        for (int k = 0; k < n; ++k) { re[k * s] = tr[k]; im[k * s] = ti[k]; }
        return;
    }
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    for (int j = 0; j < n; ++j) {           /* bit-reversed copy */
        int r = 0;
        for (int b = 0; b < logn; ++b) r |= ((j >> b) & 1) << (logn - 1 - b);
        tr[r] = re[j * s];
        ti[r] = im[j * s];
    }
    /* twiddles e^{-+2 pi i m/n}, m < n/2; a stage of size len uses every (n/len)-th one */
    double* twr = tr + n;
    double* twi = ti + n;
    for (int m = 0; m < n / 2; ++m) {
        double ang = sgn * 2.0 * MBREF_PI * (double)m / (double)n;
        twr[m] = cos(ang);
        twi[m] = sin(ang);
    }
    for (int len = 2; len <= n; len <<= 1) { /* butterflies of size len */
        int half = len / 2;
        for (int start = 0; start < n; start += len) {
            for (int m = 0; m < half; ++m) {
                double wr = twr[m * (n / len)], wi = twi[m * (n / len)];
                int a = start + m, b = start + m + half;
                double br = tr[b] * wr - ti[b] * wi;
                double bi = tr[b] * wi + ti[b] * wr;
                tr[b] = tr[a] - br; ti[b] = ti[a] - bi;
                tr[a] = tr[a] + br; ti[a] = ti[a] + bi;
            }
        }
    }
    for (int k = 0; k < n; ++k) { re[k * s] = tr[k]; im[k * s] = ti[k]; }
}

int mbref_dft3(int nx, int ny, int nz, double* re, double* im, int inverse)
{
    int nmax = nx > ny ? nx : ny;
    if (nz > nmax) nmax = nz;
    int rc = 0;
    /* every line is transformed on its own; each thread has its own line + twiddle scratch */
#pragma omp parallel
    {
        double* tr = (double*)malloc(sizeof(double) * 2 * nmax);
        double* ti = (double*)malloc(sizeof(double) * 2 * nmax);
        if (!tr || !ti) {
#pragma omp atomic write
            rc = 2;
        }
#pragma omp barrier
        if (rc == 0) {
#pragma omp for schedule(static)
            for (int k = 0; k < nz; ++k)             /* along x */
                for (int j = 0; j < ny; ++j) {
                    int64_t o = ((int64_t)k * ny + j) * nx;
                    dft_line(re + o, im + o, nx, 1, inverse, tr, ti);
                }
#pragma omp for schedule(static)
            for (int k = 0; k < nz; ++k)             /* along y */
                for (int i = 0; i < nx; ++i) {
                    int64_t o = (int64_t)k * ny * nx + i;
                    dft_line(re + o, im + o, ny, nx, inverse, tr, ti);
                }
#pragma omp for schedule(static)
            for (int j = 0; j < ny; ++j)             /* along z */
                for (int i = 0; i < nx; ++i) {
                    int64_t o = (int64_t)j * nx + i;
                    dft_line(re + o, im + o, nz, (int64_t)nx * ny, inverse, tr, ti);
                }
        }
        free(tr);
        free(ti);
    }
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Fluid operators on the MAC grid. */

/* 7-point Laplacian of one component grid (each component on its own index grid). */
static void laplacian(const mbref_grid* g, const double* v, double* out)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double ih2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t c = ((int64_t)k * ny + j) * nx + i;
                double xm = v[((int64_t)k * ny + j) * nx + wrap_index(i - 1, nx)];
                double xp = v[((int64_t)k * ny + j) * nx + wrap_index(i + 1, nx)];
                double ym = v[((int64_t)k * ny + wrap_index(j - 1, ny)) * nx + i];
                double yp = v[((int64_t)k * ny + wrap_index(j + 1, ny)) * nx + i];
                double zm = v[(wrap_index(k - 1, nz) * ny + j) * nx + i];
                double zp = v[(wrap_index(k + 1, nz) * ny + j) * nx + i];
                out[c] = ((xm - 2.0 * v[c] + xp) + (ym - 2.0 * v[c] + yp) + (zm - 2.0 * v[c] + zp)) * ih2;
            }
}

/* Body force density f0 sin(2 pi j x_w / L_w) along `axis`, evaluated on that component's
 * nodes, x_w being the node coordinate along wave_dir (viscosity protocol, Sec. 10). */
static void add_body_force(const mbref_grid* g, const double* body, double* f)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    int axis = (int)body[1], wdir = (int)body[2];
    double f0 = body[0], jw = body[3];
    double L = n[wdir] * g->h;
    double* fc = f + axis * N;
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                int idx[3] = {i, j, k};
                double x = ((double)idx[wdir] + node_shift(axis, wdir)) * g->h;
                fc[((int64_t)k * n[1] + j) * n[0] + i] += f0 * sin(2.0 * MBREF_PI * jw * x / L);
            }
}

/* Solve  c(k) W = R  and project:  W <- W - G (D.W) / (D.G)  for every wavevector.
 * D_a = (e^{i th_a} - 1)/h is the face-to-centre divergence symbol, G_a = (1 - e^{-i th_a})/h
 * the centre-to-face gradient symbol, th_a = 2 pi k_a / n_a; c(k) = a0 + a1 * lambda(k) with
 * lambda = sum 4/h^2 sin^2(th/2) the symbol of -L.  mean_zero sets the k = 0 mode to zero. */
static void solve_and_project(const mbref_grid* g, double a0, double a1, int mean_zero,
                              double* re[3], double* im[3])
{
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < nz; ++kz)
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx < nx; ++kx) {
                int64_t c = ((int64_t)kz * ny + ky) * nx + kx;
                double th[3] = {2.0 * MBREF_PI * kx / nx, 2.0 * MBREF_PI * ky / ny,
                                2.0 * MBREF_PI * kz / nz};
                double lam = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double s = sin(0.5 * th[a]);
                    lam += 4.0 / (h * h) * s * s;
                }
                double cc = a0 + a1 * lam;
                double wr[3], wi[3];
                for (int a = 0; a < 3; ++a) { wr[a] = re[a][c] / cc; wi[a] = im[a][c] / cc; }
                if (kx == 0 && ky == 0 && kz == 0) {
                    if (mean_zero)
                        for (int a = 0; a < 3; ++a) { wr[a] = 0.0; wi[a] = 0.0; }
                } else {
                    double Dr[3], Di[3], Gr[3], Gi[3];
                    for (int a = 0; a < 3; ++a) {
                        Dr[a] = (cos(th[a]) - 1.0) / h;  Di[a] = sin(th[a]) / h;
                        Gr[a] = (1.0 - cos(th[a])) / h;  Gi[a] = sin(th[a]) / h;
                    }
                    double divr = 0.0, divi = 0.0, dgr = 0.0, dgi = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        divr += Dr[a] * wr[a] - Di[a] * wi[a];
                        divi += Dr[a] * wi[a] + Di[a] * wr[a];
                        dgr += Dr[a] * Gr[a] - Di[a] * Gi[a];
                        dgi += Dr[a] * Gi[a] + Di[a] * Gr[a];
                    }
                    /* q = div / (D.G) */
                    double den = dgr * dgr + dgi * dgi;
                    double qr = (divr * dgr + divi * dgi) / den;
                    double qi = (divi * dgr - divr * dgi) / den;
                    for (int a = 0; a < 3; ++a) {
                        wr[a] -= Gr[a] * qr - Gi[a] * qi;
                        wi[a] -= Gr[a] * qi + Gi[a] * qr;
                    }
                }
                for (int a = 0; a < 3; ++a) { re[a][c] = wr[a]; im[a][c] = wi[a]; }
            }
}

/* Transform three real component grids, solve, project and transform back. */
static int spectral_solve(const mbref_grid* g, const double* rhs, double a0, double a1,
                          int mean_zero, double* v_out)
{
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    double* re[3];
    double* im[3];
    for (int a = 0; a < 3; ++a) {
        re[a] = (double*)malloc(sizeof(double) * N);
        im[a] = (double*)calloc(N, sizeof(double));
        if (!re[a] || !im[a]) return 2;
        memcpy(re[a], rhs + a * N, sizeof(double) * N);
        mbref_dft3(g->nx, g->ny, g->nz, re[a], im[a], 0);
    }
    solve_and_project(g, a0, a1, mean_zero, re, im);
    for (int a = 0; a < 3; ++a) {
        mbref_dft3(g->nx, g->ny, g->nz, re[a], im[a], 1);
        for (int64_t c = 0; c < N; ++c) v_out[a * N + c] = re[a][c] / (double)N;
        free(re[a]);
        free(im[a]);
    }
    return 0;
}

int mbref_fluid_update(const mbref_grid* g, const double* v, const double* f,
                       const double* body, double* v_out)
{
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    double* rhs = (double*)malloc(sizeof(double) * 3 * N);
    double* lap = (double*)malloc(sizeof(double) * N);
    if (!rhs || !lap) { free(rhs); free(lap); return 2; }
    /* Crank-Nicolson right-hand side of Eq. (vf): (rho/dt) v + (eta/2) L v + f. */
    for (int a = 0; a < 3; ++a) {
        laplacian(g, v + a * N, lap);
        for (int64_t c = 0; c < N; ++c)
            rhs[a * N + c] = g->rho / g->dt * v[a * N + c] + 0.5 * g->eta * lap[c] + f[a * N + c];
    }
    if (g->advection) {
        /* convective stress rho v v of Eq. (vf), explicit at v^n */
        double* adv = (double*)malloc(sizeof(double) * 3 * N);
        if (!adv) { free(rhs); free(lap); return 2; }
        mbref_advection(g, v, adv);
        for (int64_t c = 0; c < 3 * N; ++c) rhs[c] -= g->rho * adv[c];
        free(adv);
    }
    if (body) add_body_force(g, body, rhs);
    int rc = spectral_solve(g, rhs, g->rho / g->dt, 0.5 * g->eta, g->mean_mode == 1, v_out);
    free(rhs);
    free(lap);
    return rc;
}

int mbref_stokes_solve(const mbref_grid* g, const double* f, double* v)
{
    return spectral_solve(g, f, 0.0, g->eta, 1, v);
}

/* ------------------------------------------------------------------------------------ */
/* Forces. */

static double min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

int mbref_bond_forces(const mbref_grid* g, int64_t n, const double* q, int64_t nbonds,
                      const int32_t* bonds, const double* rest, double k, double* F)
{
    const double L[3] = {g->nx * g->h, g->ny * g->h, g->nz * g->h};
    (void)n;
    for (int64_t e = 0; e < nbonds; ++e) {
        int i = bonds[2 * e], j = bonds[2 * e + 1];
        double r[3], r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            r[a] = min_image(q[3 * i + a] - q[3 * j + a], L[a]);
            r2 += r[a] * r[a];
        }
        double len = sqrt(r2);
        double mag = -k * (len - rest[e]) / len;   /* force on i along r_ij = q_i - q_j */
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += mag * r[a];
            F[3 * j + a] -= mag * r[a];
        }
    }
    return 0;
}

/* Contribution of blob j to the repulsion on blob i: k_rep (r_cut - r) r_hat, r = q_i - q_j
 * (minimum image), for r < r_cut and blobs of different particles. */
static void add_pair(const double L[3], const double* q, const int32_t* pid, double k_rep,
                     double r_cut, int64_t i, int64_t j, double out[3])
{
    if (j == i || pid[j] == pid[i]) return;
    double r[3], r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        r[a] = min_image(q[3 * i + a] - q[3 * j + a], L[a]);
        r2 += r[a] * r[a];
    }
    if (r2 >= r_cut * r_cut || r2 == 0.0) return;
    double len = sqrt(r2);
    double mag = k_rep * (r_cut - len) / len;
    for (int a = 0; a < 3; ++a) out[a] += mag * r[a];
}

/* The definition: every other blob j = 0 .. n-1 in turn. */
static void pair_force_brute(const double L[3], int64_t n, const double* q, const int32_t* pid,
                             double k_rep, double r_cut, int64_t i, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    for (int64_t j = 0; j < n; ++j) add_pair(L, q, pid, k_rep, r_cut, i, j, out);
}

/* Bins of side w_a = L_a / nb_a >= r_cut (1 + 1e-6) along each axis.  Two blobs closer than
 * r_cut (minimum image) differ by less than w_a along every axis, so their bins are equal or
 * adjacent (periodically); the margin keeps that true when a coordinate on a bin boundary is
 * rounded into the next bin.  With at least three bins per axis the 27 bins around a blob are
 * distinct, and visiting the blobs listed there in ascending index order adds the same
 * non-zero terms, in the same order, as the definition: the result is the same to the bit
 * (tested).  Fewer bins fall back to the definition. */
typedef struct {
    int nb[3];
    int64_t* start;   /* [nbins + 1] */
    int64_t* list;    /* [n] blob indices, ascending within each bin */
} pair_bins;

static int bin_coord(double x, double L, int nb)
{
    double y = fmod(x, L);
    if (y < 0.0) y += L;
    int c = (int)floor(y / L * nb);
    return c < 0 ? 0 : (c >= nb ? nb - 1 : c);
}

static int64_t blob_bin(const pair_bins* B, const double L[3], const double* q, int64_t i)
{
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = bin_coord(q[3 * i + a], L[a], B->nb[a]);
    return ((int64_t)c[2] * B->nb[1] + c[1]) * B->nb[0] + c[0];
}

/* 0: bins built; 1: too few bins (use the definition); 2: out of memory */
static int build_bins(pair_bins* B, const double L[3], int64_t n, const double* q, double r_cut)
{
    B->start = NULL;
    B->list = NULL;
    for (int a = 0; a < 3; ++a) {
        double m = floor(L[a] / (r_cut * (1.0 + 1e-6)));
        if (m < 3.0) return 1;
        B->nb[a] = m > 1024.0 ? 1024 : (int)m;
    }
    const int64_t nbins = (int64_t)B->nb[0] * B->nb[1] * B->nb[2];
    B->start = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
    B->list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbins);
    if (!B->start || !B->list || !fill) {
        free(B->start); free(B->list); free(fill);
        return 2;
    }
    for (int64_t i = 0; i < n; ++i) B->start[blob_bin(B, L, q, i) + 1] += 1;
    for (int64_t b = 0; b < nbins; ++b) B->start[b + 1] += B->start[b];
    memcpy(fill, B->start, sizeof(int64_t) * (size_t)nbins);
    for (int64_t i = 0; i < n; ++i) B->list[fill[blob_bin(B, L, q, i)]++] = i;
    free(fill);
    return 0;
}

static int cmp_i64(const void* x, const void* y)
{
    int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
    return (a > b) - (a < b);
}

/* Repulsion on blob i from the blobs of the 27 bins around it, in ascending index order.
 * *cand / *cap is a per-thread buffer, grown as needed; returns 2 if that fails. */
static int pair_force_binned(const pair_bins* B, const double L[3], const double* q,
                             const int32_t* pid, double k_rep, double r_cut, int64_t i,
                             int64_t** cand, int64_t* cap, double out[3])
{
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = bin_coord(q[3 * i + a], L[a], B->nb[a]);
    int64_t m = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int bx = (c[0] + dx + B->nb[0]) % B->nb[0];
                const int by = (c[1] + dy + B->nb[1]) % B->nb[1];
                const int bz = (c[2] + dz + B->nb[2]) % B->nb[2];
                const int64_t b = ((int64_t)bz * B->nb[1] + by) * B->nb[0] + bx;
                const int64_t k = B->start[b + 1] - B->start[b];
                if (m + k > *cap) {
                    int64_t nc = 2 * (m + k) + 64;
                    int64_t* p = (int64_t*)realloc(*cand, sizeof(int64_t) * (size_t)nc);
                    if (!p) return 2;
                    *cand = p;
                    *cap = nc;
                }
                memcpy(*cand + m, B->list + B->start[b], sizeof(int64_t) * (size_t)k);
                m += k;
            }
    qsort(*cand, (size_t)m, sizeof(int64_t), cmp_i64);
    out[0] = out[1] = out[2] = 0.0;
    for (int64_t t = 0; t < m; ++t) add_pair(L, q, pid, k_rep, r_cut, i, (*cand)[t], out);
    return 0;
}

/* Repulsion on the m blobs idx[0..m) (all n blobs when idx is NULL), written to out [m][3]
 * (added to it when accumulate is set). */
static int pair_forces_on(const mbref_grid* g, int64_t n, const double* q, const int32_t* pid,
                          double k_rep, double r_cut, int64_t m, const int64_t* idx,
                          int accumulate, int brute, double* out)
{
    const double L[3] = {g->nx * g->h, g->ny * g->h, g->nz * g->h};
    pair_bins B;
    int binned = 0;
    if (!brute) {
        int rc = build_bins(&B, L, n, q, r_cut);
        if (rc == 2) return 2;
        binned = rc == 0;
    }
    int err = 0;
#pragma omp parallel
    {
        int64_t* cand = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t s = 0; s < m; ++s) {
            const int64_t i = idx ? idx[s] : s;
            double fi[3];
            if (binned) {
                if (pair_force_binned(&B, L, q, pid, k_rep, r_cut, i, &cand, &cap, fi)) {
#pragma omp atomic write
                    err = 2;
                    fi[0] = fi[1] = fi[2] = 0.0;
                }
            } else {
                pair_force_brute(L, n, q, pid, k_rep, r_cut, i, fi);
            }
            for (int a = 0; a < 3; ++a)
                out[3 * s + a] = accumulate ? out[3 * s + a] + fi[a] : fi[a];
        }
        free(cand);
    }
    if (binned) {
        free(B.start);
        free(B.list);
    }
    return err;
}

int mbref_pair_forces(const mbref_grid* g, int64_t n, const double* q, const int32_t* pid,
                      double k_rep, double r_cut, double* F)
{
    if (k_rep == 0.0 || r_cut <= 0.0) return 0;
    return pair_forces_on(g, n, q, pid, k_rep, r_cut, n, NULL, 1, 0, F);
}

int mbref_pair_forces_brute(const mbref_grid* g, int64_t n, const double* q, const int32_t* pid,
                            double k_rep, double r_cut, double* F)
{
    if (k_rep == 0.0 || r_cut <= 0.0) return 0;
    return pair_forces_on(g, n, q, pid, k_rep, r_cut, n, NULL, 1, 1, F);
}

int mbref_pair_forces_subset(const mbref_grid* g, int64_t n, const double* q,
                             const int32_t* pid, double k_rep, double r_cut, int64_t m,
                             const int64_t* idx, double* F)
{
    if (k_rep == 0.0 || r_cut <= 0.0) {
        memset(F, 0, sizeof(double) * 3 * (size_t)m);
        return 0;
    }
    return pair_forces_on(g, n, q, pid, k_rep, r_cut, m, idx, 0, 0, F);
}

/* ------------------------------------------------------------------------------------ */
/* Fluctuating stress (Sec. 3: the stress sigma~ of Eq. vf, Gaussian, following the
 * staggered fluctuating hydrodynamics the paper cites).  It is a random 3x3 tensor field
 * W_ab, non-symmetric, each component an independent standard normal per cell, scaled to
 * sigma~ = sqrt(2 eta kT / (h^3 dt)) W; the fluid receives the force density -D.sigma~.
 * Placement on the MAC grid: W_aa at cell centres, W_ab (b != a) on the edge whose a and b
 * coordinates are the integer multiples i_a h, i_b h.  Its divergence on the faces of
 * component a is a backward difference of W_aa and forward differences of W_ab, so that
 * D D^T = -L for each component: the covariance of the noise force is (2 eta kT/(h^3 dt))
 * (-L), which makes the Crank-Nicolson update sample Eq. (ef) exactly at any dt. */

/* Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of two 64x64->128-bit
 * multiplications on a 256-bit counter with a 128-bit key bumped by Weyl constants. */
void mbref_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Nine standard normals of cell m of box `box` at step `step`.  Cells are drawn in groups of
 * four along x (m = 4 G + r, r < 4; rows hold a multiple of four cells): five Philox blocks
 * with key (seed, 0) and counters (G, step, box, j), j = 0..4, give the 64-bit words
 * x_0..x_19; word x_p gives the Box-Muller pair p: u1 = (lo32 + 1/2)/2^32,
 * u2 = (hi32 + 1/2)/2^32, rho = sqrt(-2 ln u1), normals z_2p = rho cos(2 pi u2) and
 * z_2p+1 = rho sin(2 pi u2).  Cell r takes z_9r .. z_9r+8 as W_xx, W_xy, W_xz, W_yx, W_yy,
 * W_yz, W_zx, W_zy, W_zz (pairs 0..17; words 18 and 19 are unused). */
static void cell_normals(uint64_t seed, uint64_t step, int64_t box, int64_t m, double z[9])
{
    const uint64_t key[2] = {seed, 0};
    const int64_t G = m / 4, r = m % 4;
    uint64_t x[20];
    for (int j = 0; j < 5; ++j) {
        const uint64_t ctr[4] = {(uint64_t)G, step, (uint64_t)box, (uint64_t)j};
        mbref_philox4x64(ctr, key, x + 4 * j);
    }
    for (int c = 0; c < 9; ++c) {
        const int q = 9 * (int)r + c, p = q / 2;
        double u1 = ((double)(x[p] & 0xffffffffull) + 0.5) / 4294967296.0;
        double u2 = ((double)(x[p] >> 32) + 0.5) / 4294967296.0;
        double rho = sqrt(-2.0 * log(u1));
        z[c] = q % 2 == 0 ? rho * cos(2.0 * MBREF_PI * u2) : rho * sin(2.0 * MBREF_PI * u2);
    }
}

int mbref_stress_normals(const mbref_grid* g, uint64_t seed, uint64_t step, int64_t box,
                         double* W)
{
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    if (g->nx % 4 != 0) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < N; ++m) {
        double z[9];
        cell_normals(seed, step, box, m, z);
        for (int c = 0; c < 9; ++c) W[c * N + m] = z[c];
    }
    return 0;
}

int mbref_stress_div(const mbref_grid* g, const double* W, double* f)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    const int idx[3] = {i, j, k};
                    double d = 0.0;
                    for (int b = 0; b < 3; ++b) {
                        /* the two stress nodes of component (a, b) around this face */
                        int lo[3] = {idx[0], idx[1], idx[2]}, hi[3] = {idx[0], idx[1], idx[2]};
                        if (b == a) lo[b] = (int)wrap_index(idx[b] - 1, n[b]);   /* centres */
                        else hi[b] = (int)wrap_index(idx[b] + 1, n[b]);          /* edges */
                        const double* Wab = W + (3 * a + b) * N;
                        d += Wab[((int64_t)hi[2] * n[1] + hi[1]) * n[0] + hi[0]]
                           - Wab[((int64_t)lo[2] * n[1] + lo[1]) * n[0] + lo[0]];
                    }
                    f[a * N + ((int64_t)k * n[1] + j) * n[0] + i] = d / g->h;
                }
    return 0;
}

/* The convective tensor M_ab = v_a v_b at the stress nodes: for a = b the square of the mean
 * of the two v_a faces around the cell centre; for b != a, on the edge at integer a and b
 * coordinates, the mean of the two v_a faces on either side along b times the mean of the two
 * v_b faces on either side along a.  Its MAC divergence is the convective term. */
int mbref_advection(const mbref_grid* g, const double* v, double* out)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    double* M = (double*)malloc(sizeof(double) * 9 * N);
    if (!M) return 2;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const int idx[3] = {i, j, k};
                const int64_t c = ((int64_t)k * n[1] + j) * n[0] + i;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        /* neighbour of this cell one step along dimension e, by s = +-1 */
                        int64_t nb_a, nb_b;
                        int t[3] = {idx[0], idx[1], idx[2]};
                        if (a == b) {
                            t[a] = (int)wrap_index(idx[a] + 1, n[a]);
                            nb_a = ((int64_t)t[2] * n[1] + t[1]) * n[0] + t[0];
                            const double m = 0.5 * (v[a * N + c] + v[a * N + nb_a]);
                            M[(3 * a + b) * N + c] = m * m;
                        } else {
                            t[b] = (int)wrap_index(idx[b] - 1, n[b]);
                            nb_b = ((int64_t)t[2] * n[1] + t[1]) * n[0] + t[0];
                            int r[3] = {idx[0], idx[1], idx[2]};
                            r[a] = (int)wrap_index(idx[a] - 1, n[a]);
                            nb_a = ((int64_t)r[2] * n[1] + r[1]) * n[0] + r[0];
                            const double va = 0.5 * (v[a * N + c] + v[a * N + nb_b]);
                            const double vb = 0.5 * (v[b * N + c] + v[b * N + nb_a]);
                            M[(3 * a + b) * N + c] = va * vb;
                        }
                    }
            }
    mbref_stress_div(g, M, out);
    free(M);
    return 0;
}

/* f += -D.sigma~ for the step `step` (nothing when noise is NULL or kT = 0). */
static int add_stress_noise(const mbref_grid* g, const mbref_noise* noise, uint64_t step,
                            double* f)
{
    if (!noise || noise->kT == 0.0) return 0;
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    double* W = (double*)malloc(sizeof(double) * 9 * N);
    double* d = (double*)malloc(sizeof(double) * 3 * N);
    if (!W || !d) { free(W); free(d); return 2; }
    mbref_stress_normals(g, noise->seed, step, noise->box, W);
    const double amp = sqrt(2.0 * g->eta * noise->kT / (g->h * g->h * g->h * g->dt));
    for (int64_t c = 0; c < 9 * N; ++c) W[c] *= amp;
    mbref_stress_div(g, W, d);
    for (int64_t c = 0; c < 3 * N; ++c) f[c] -= d[c];
    free(W);
    free(d);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Time step. */

/* Periodic wrap into [0, L) for a displacement smaller than L. */
static double wrap_pos(double x, double L)
{
    if (x < 0.0) {
        x += L;
        if (x >= L) x -= L;
    } else if (x >= L) {
        x -= L;
    }
    return x;
}

int mbref_step(const mbref_grid* g, int nsteps, int64_t n, double* q, double* v,
               const int32_t* pid, int64_t nbonds, const int32_t* bonds, const double* rest,
               double k_spring, double k_rep, double r_cut, const double* ext,
               const double* body, const mbref_noise* noise)
{
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    const double L[3] = {g->nx * g->h, g->ny * g->h, g->nz * g->h};
    const double dt = g->dt;
    double* u = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* qh = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* f = (double*)malloc(sizeof(double) * 3 * N);
    double* vn = (double*)malloc(sizeof(double) * 3 * N);
    double* vm = (double*)malloc(sizeof(double) * 3 * N);
    if (!u || !qh || !F || !f || !vn || !vm) {
        free(u); free(qh); free(F); free(f); free(vn); free(vm);
        return 2;
    }
    for (int s = 0; s < nsteps; ++s) {
        /* predictor: u^n = J(q^n) v^n (no-slip, Eq. ju); q^{n+1/2} = q^n + dt/2 u^n */
        mbref_interp(g, n, q, v, u);
        for (int64_t b = 0; b < n; ++b)
            for (int a = 0; a < 3; ++a)
                qh[3 * b + a] = wrap_pos(q[3 * b + a] + 0.5 * dt * u[3 * b + a], L[a]);
        /* blob forces at q^{n+1/2}: springs, blob-blob repulsion, external */
        for (int64_t c = 0; c < 3 * n; ++c) F[c] = ext ? ext[c] : 0.0;
        mbref_bond_forces(g, n, qh, nbonds, bonds, rest, k_spring, F);
        mbref_pair_forces(g, n, qh, pid, k_rep, r_cut, F);
        /* neutrally buoyant blobs (m_e = 0): lambda_i = -F_i, so the fluid receives S F */
        mbref_spread(g, n, qh, F, f);
        /* thermal stress of this step (Sec. 3), when kT > 0 */
        if (add_stress_noise(g, noise, (noise ? noise->step0 : 0) + (uint64_t)s, f)) {
            free(u); free(qh); free(F); free(f); free(vn); free(vm);
            return 2;
        }
        mbref_fluid_update(g, v, f, body, vn);
        /* corrector: q^{n+1} = q^n + dt J(q^{n+1/2}) (v^n + v^{n+1})/2 */
        for (int64_t c = 0; c < 3 * N; ++c) vm[c] = 0.5 * (v[c] + vn[c]);
        mbref_interp(g, n, qh, vm, u);
        for (int64_t b = 0; b < n; ++b)
            for (int a = 0; a < 3; ++a)
                q[3 * b + a] = wrap_pos(q[3 * b + a] + dt * u[3 * b + a], L[a]);
        memcpy(v, vn, sizeof(double) * 3 * N);
    }
    free(u); free(qh); free(F); free(f); free(vn); free(vm);
    return 0;
}

/* Stokes limit (Sc -> infinity) of the blob-fluid coupling: the fluid momentum relaxes
 * instantly, so the fluid velocity is the steady Stokes solution for the current forces,
 * v = P (-eta L)^{-1} (S F + f_body) with zero mean (Sec. 3 with the inertia of fluid and
 * particles removed, the regime of the paper's viscosity runs), and the blobs follow it,
 * u = J v.  In time, the explicit midpoint rule (the deterministic part of the Stokes-limit
 * integrator the paper cites): forces and solve at q^n give q^{n+1/2} = q^n + dt/2 u^n, forces
 * and solve at q^{n+1/2} give q^{n+1} = q^n + dt u^{n+1/2}.  v returns the second solve. */
static void all_forces(const mbref_grid* g, int64_t n, const double* x, const int32_t* pid,
                       int64_t nbonds, const int32_t* bonds, const double* rest, double k_spring,
                       double k_rep, double r_cut, const double* ext, double* F)
{
    for (int64_t c = 0; c < 3 * n; ++c) F[c] = ext ? ext[c] : 0.0;
    mbref_bond_forces(g, n, x, nbonds, bonds, rest, k_spring, F);
    mbref_pair_forces(g, n, x, pid, k_rep, r_cut, F);
}

int mbref_stokes_step(const mbref_grid* g, int nsteps, int64_t n, double* q, double* v,
                      const int32_t* pid, int64_t nbonds, const int32_t* bonds,
                      const double* rest, double k_spring, double k_rep, double r_cut,
                      const double* ext, const double* body)
{
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    const double L[3] = {g->nx * g->h, g->ny * g->h, g->nz * g->h};
    const double dt = g->dt;
    double* u = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* qh = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* f = (double*)malloc(sizeof(double) * 3 * N);
    if (!u || !qh || !F || !f) {
        free(u); free(qh); free(F); free(f);
        return 2;
    }
    for (int s = 0; s < nsteps; ++s) {
        /* half step with the forces and the flow of q^n */
        all_forces(g, n, q, pid, nbonds, bonds, rest, k_spring, k_rep, r_cut, ext, F);
        mbref_spread(g, n, q, F, f);
        if (body) add_body_force(g, body, f);
        mbref_stokes_solve(g, f, v);
        mbref_interp(g, n, q, v, u);
        for (int64_t b = 0; b < n; ++b)
            for (int a = 0; a < 3; ++a)
                qh[3 * b + a] = wrap_pos(q[3 * b + a] + 0.5 * dt * u[3 * b + a], L[a]);
        /* full step with the forces and the flow of q^{n+1/2} */
        all_forces(g, n, qh, pid, nbonds, bonds, rest, k_spring, k_rep, r_cut, ext, F);
        mbref_spread(g, n, qh, F, f);
        if (body) add_body_force(g, body, f);
        mbref_stokes_solve(g, f, v);
        mbref_interp(g, n, qh, v, u);
        for (int64_t b = 0; b < n; ++b)
            for (int a = 0; a < 3; ++a)
                q[3 * b + a] = wrap_pos(q[3 * b + a] + dt * u[3 * b + a], L[a]);
    }
    free(u); free(qh); free(F); free(f);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Particle observables (Sec. 2 and Sec. 3.2): U0 = (1/N) sum u_i;
 * Omega solves I0 Omega = sum_i s_i x (u_i - U0), I0 = sum_i (s_i^2 1 - s_i s_i). */
int mbref_particle_velocities(const mbref_grid* g, int64_t n, const double* q, const double* u,
                              const int32_t* pid, int64_t np, double* U, double* Omega)
{
    const double L[3] = {g->nx * g->h, g->ny * g->h, g->nz * g->h};
    int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (np > 0 ? np : 1));
    double* acc = (double*)calloc((size_t)(np > 0 ? np : 1) * 20, sizeof(double));
    if (!first || !acc) { free(first); free(acc); return 2; }
    for (int64_t p = 0; p < np; ++p) first[p] = -1;
    /* pass 1: blob count, sum of u_i, sum of positions relative to the particle's first blob */
    for (int64_t b = 0; b < n; ++b) {
        int64_t p = pid[b];
        if (p < 0 || p >= np) continue;
        if (first[p] < 0) first[p] = b;
        double* A = acc + 20 * p;
        A[0] += 1.0;
        for (int a = 0; a < 3; ++a) {
            A[1 + a] += u[3 * b + a];
            A[4 + a] += min_image(q[3 * b + a] - q[3 * first[p] + a], L[a]);
        }
    }
    for (int64_t p = 0; p < np; ++p) {
        double* A = acc + 20 * p;
        if (A[0] > 0.0)
            for (int a = 0; a < 3; ++a) { A[1 + a] /= A[0]; A[4 + a] /= A[0]; }
    }
    /* pass 2: I0 = sum (s^2 1 - s s) (A[7..15]) and sum s x (u - U0) (A[16..18]),
     * with s_i = q_i - q_0 the blob position relative to the baricentre q_0 */
    for (int64_t b = 0; b < n; ++b) {
        int64_t p = pid[b];
        if (p < 0 || p >= np) continue;
        double* A = acc + 20 * p;
        double s[3], w[3];
        for (int a = 0; a < 3; ++a) {
            s[a] = min_image(q[3 * b + a] - q[3 * first[p] + a], L[a]) - A[4 + a];
            w[a] = u[3 * b + a] - A[1 + a];
        }
        double s2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) A[7 + 3 * a + c] += (a == c ? s2 : 0.0) - s[a] * s[c];
        A[16] += s[1] * w[2] - s[2] * w[1];
        A[17] += s[2] * w[0] - s[0] * w[2];
        A[18] += s[0] * w[1] - s[1] * w[0];
    }
    for (int64_t p = 0; p < np; ++p) {
        double* A = acc + 20 * p;
        double Om[3] = {0.0, 0.0, 0.0};
        double I[3][3];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) I[a][c] = A[7 + 3 * a + c];
        /* 3x3 solve I0 Omega = torque-like sum, by Cramer's rule; a degenerate I0
         * (a single blob, or collinear blobs) leaves Omega = 0 */
        double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1])
                   - I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0])
                   + I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
        double scale = I[0][0] + I[1][1] + I[2][2];
        if (scale > 0.0 && fabs(det) > 1e-12 * scale * scale * scale) {
            for (int col = 0; col < 3; ++col) {
                double M[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) M[a][c] = (c == col) ? A[16 + a] : I[a][c];
                double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                          - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                          + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                Om[col] = dc / det;
            }
        }
        for (int a = 0; a < 3; ++a) { U[3 * p + a] = A[1 + a]; Omega[3 * p + a] = Om[a]; }
    }
    free(first);
    free(acc);
    return 0;
}
