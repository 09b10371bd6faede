/*
 * minimod_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the Minimod acoustic isotropic
 * constant-density time step (the "acoustic isotropic kernel" of the
 * Minimod application, paper section 4.5).  It exists to check the CUDA
 * library and is used only by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark.  The product path never calls it, and
 * it shares no code, header, table or constant with the CUDA library.
 *
 * The paper prints no stencil, coefficient, boundary or source definition,
 * only the application (section 4.5), its workload (1200^3, 1000 steps)
 * and the halo exchange of Listing 1.  The scheme written out here is the
 * standard one that the name "acoustic isotropic, 8th order in space,
 * 2nd order in time" fixes:
 *
 *   lap(u)   = sum over the three axes of  c0*u + sum_{m=1..4} c_m*(u[-m] + u[+m])
 *   u_{n+1}  = G * ( 2 u_n - G u_{n-1} + coef * ( lap(u_n) + [src] r_n ) )
 *   coef     = (v dt / h)^2,   G = g_x g_y g_z (Cerjan sponge)
 *
 * Everything is FP64, computed in the obvious order, one grid point at a
 * time.  Arrays handed in and out are interior-only, x fastest, then y,
 * then z.  Internally the wavefields carry a halo of R = 4 cells on every
 * side, zero (Dirichlet) or wrapped (periodic).
 *
 * Parity pins for each function live in the CPU test suite; the sponge
 * constants, the wavelet delay and the source form are readings, not
 * paper content ("parity unpinned" beyond the properties tested there).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define R 4

/* Coefficients of the 8th-order central second difference on a unit grid:
 * f''(0) ~ c0 f(0) + sum_m c_m (f(m) + f(-m)).  Standard Taylor-table
 * values (exact fractions), not printed in the paper. */
void oracle_stencil_coefficients(double c[5])
{
    c[0] = -205.0 / 72.0;
    c[1] = 8.0 / 5.0;
    c[2] = -1.0 / 5.0;
    c[3] = 8.0 / 315.0;
    c[4] = -1.0 / 560.0;
}

/* Symbol of the 1-D difference operator at wavenumber theta = k h:
 * L(theta) = c0 + 2 sum_m c_m cos(m theta).  Its most negative value is at
 * theta = pi (checked by the tests, which scan theta). */
double oracle_symbol(double theta)
{
    double c[5];
    oracle_stencil_coefficients(c);
    double s = c[0];
    for (int m = 1; m <= 4; ++m) s += 2.0 * c[m] * cos(m * theta);
    return s;
}

/* Stability limit of the leapfrog with this 3-D stencil: the scheme is
 * stable while nu^2 * 3 |L(pi)| <= 4, nu = v dt / h. */
double oracle_nu_max(void)
{
    return sqrt(4.0 / (3.0 * fabs(oracle_symbol(M_PI))));
}

/* Time step from the Courant number nu: dt = nu h / vmax.  courant <= 0
 * selects the default reading of "dt set by CFL 0.5": half the stability
 * limit. */
double oracle_time_step(double h, double vmax, double courant)
{
    double nu = courant > 0.0 ? courant : 0.5 * oracle_nu_max();
    return nu * h / vmax;
}

/* Ricker wavelet of peak frequency f, delayed by t0 = 1/f, sampled at
 * t_n = n dt:  r(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),
 * tau = t - t0. */
void oracle_ricker(double f, double dt, int n, double *out)
{
    double t0 = 1.0 / f;
    for (int i = 0; i < n; ++i) {
        double tau = i * dt - t0;
        double a = M_PI * M_PI * f * f * tau * tau;
        out[i] = (1.0 - 2.0 * a) * exp(-a);
    }
}

/* Cerjan sponge factor along one axis of n cells with a layer of `width`
 * cells at both ends: a cell at distance d from its nearest outer face
 * (d = 0 for the outermost cell) gets exp(-(a (width - d))^2) when
 * d < width, and 1 otherwise. */
void oracle_cerjan_profile(int n, int width, double a, double *g)
{
    for (int i = 0; i < n; ++i) {
        int d = i < n - 1 - i ? i : n - 1 - i;
        if (d < width) {
            double e = a * (double)(width - d);
            g[i] = exp(-e * e);
        } else {
            g[i] = 1.0;
        }
    }
}

/* ---------------------------------------------------------------- */
/* padded-array helpers                                              */

typedef struct {
    int nx, ny, nz;
    long px, py, pz;   /* padded extents */
} grid_t;

static grid_t make_grid(int nx, int ny, int nz)
{
    grid_t g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.px = nx + 2 * R; g.py = ny + 2 * R; g.pz = nz + 2 * R;
    return g;
}

/* index of interior point (i, j, k), halo offsets allowed in [-R, n+R) */
static inline long at(const grid_t *g, long i, long j, long k)
{
    return ((k + R) * g->py + (j + R)) * g->px + (i + R);
}

static void load_interior(const grid_t *g, double *pad, const double *in)
{
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i)
                pad[at(g, i, j, k)] =
                    in ? in[(k * g->ny + j) * g->nx + i] : 0.0;
}

static void store_interior(const grid_t *g, const double *pad, double *out)
{
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i)
                out[(k * g->ny + j) * g->nx + i] = pad[at(g, i, j, k)];
}

static long wrap(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Periodic boundary: every halo cell (face, edge or corner) takes the value
 * of the interior cell it wraps onto. */
static void fill_periodic_halo(const grid_t *g, double *pad)
{
    for (long k = -R; k < g->nz + R; ++k)
        for (long j = -R; j < g->ny + R; ++j)
            for (long i = -R; i < g->nx + R; ++i) {
                int inside = i >= 0 && i < g->nx && j >= 0 && j < g->ny &&
                             k >= 0 && k < g->nz;
                if (!inside)
                    pad[at(g, i, j, k)] = pad[at(g, wrap(i, g->nx),
                                                 wrap(j, g->ny),
                                                 wrap(k, g->nz))];
            }
}

static double lap_at(const grid_t *g, const double *u, const double c[5],
                     long i, long j, long k)
{
    double s = 3.0 * c[0] * u[at(g, i, j, k)];
    for (int m = 1; m <= 4; ++m) {
        s += c[m] * (u[at(g, i - m, j, k)] + u[at(g, i + m, j, k)]);
        s += c[m] * (u[at(g, i, j - m, k)] + u[at(g, i, j + m, k)]);
        s += c[m] * (u[at(g, i, j, k - m)] + u[at(g, i, j, k + m)]);
    }
    return s;
}

/* Discrete Laplacian (dimensionless, unit spacing) of a padded field whose
 * halo the caller has filled: in is (nz+8)(ny+8)(nx+8), out is interior. */
void oracle_laplacian(int nx, int ny, int nz, const double *u_pad,
                      double *out)
{
    grid_t g = make_grid(nx, ny, nz);
    double c[5];
    oracle_stencil_coefficients(c);
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i)
                out[(k * ny + j) * nx + i] = lap_at(&g, u_pad, c, i, j, k);
}

/* Discrete energy at the half step n+1/2 of the source-free, sponge-free
 * scheme:  E = sum (u_{n+1} - u_n)^2 / coef  -  sum u_{n+1} * lap(u_n).
 * It is exactly conserved by the recurrence because lap is symmetric.
 * u_next and u_cur are interior arrays; periodic selects the halo. */
double oracle_energy(int nx, int ny, int nz, const double *coef,
                     const double *u_next, const double *u_cur, int periodic)
{
    grid_t g = make_grid(nx, ny, nz);
    long npad = g.px * g.py * g.pz;
    double *pad = (double *)calloc((size_t)npad, sizeof(double));
    double c[5];
    oracle_stencil_coefficients(c);
    load_interior(&g, pad, u_cur);
    if (periodic) fill_periodic_halo(&g, pad);
    double kin = 0.0, pot = 0.0;
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long q = (k * ny + j) * nx + i;
                double d = u_next[q] - u_cur[q];
                kin += d * d / coef[q];
                pot += u_next[q] * lap_at(&g, pad, c, i, j, k);
            }
    free(pad);
    return kin - pot;
}

/*
 * Run the recurrence for nsteps steps.
 *
 *  vel      nz*ny*nx velocities (m/s)
 *  h, dt    grid spacing (m) and time step (s); coef = (v dt / h)^2
 *  sponge   Cerjan layer width in cells (0: none), a = sponge_a
 *  periodic 0: zero halo (Dirichlet); 1: wrapped halo
 *  src      (sx, sy, sz) and wavelet[0..nsteps): at step n the source adds
 *           wavelet[n] to lap(u_n) at that cell; wavelet NULL = no source
 *  rec      nrec (x, y, z) triples; traces[r*nsteps + n] = u_{n+1}(rec r)
 *  u_cur    in: u_0 (NULL-able via init_cur = 0); out: u_nsteps
 *  u_prev   in: u_{-1}; out: u_{nsteps-1}
 *  norms    if not NULL, norms[n] = sum of u_{n+1}^2 over the interior
 *  nthreads OpenMP threads over z planes (1 = serial)
 *
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_run(int nx, int ny, int nz, const double *vel, double h,
               double dt, int nsteps, int sponge, double sponge_a,
               int periodic, int sx, int sy, int sz, const double *wavelet,
               int nrec, const int *rec_xyz, double *traces, int init_cur,
               double *u_cur, int init_prev, double *u_prev, double *norms,
               int nthreads)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || nsteps < 0 || !vel || !u_cur ||
        !u_prev)
        return -1;
    grid_t g = make_grid(nx, ny, nz);
    long npad = g.px * g.py * g.pz;
    long nint = (long)nx * ny * nz;
    double *a = (double *)calloc((size_t)npad, sizeof(double)); /* u_n     */
    double *b = (double *)calloc((size_t)npad, sizeof(double)); /* u_{n-1} */
    double *coef = (double *)malloc((size_t)nint * sizeof(double));
    double *gx = (double *)malloc((size_t)nx * sizeof(double));
    double *gy = (double *)malloc((size_t)ny * sizeof(double));
    double *gz = (double *)malloc((size_t)nz * sizeof(double));
    if (!a || !b || !coef || !gx || !gy || !gz) {
        free(a); free(b); free(coef); free(gx); free(gy); free(gz);
        return -1;
    }
    for (long q = 0; q < nint; ++q) {
        double nu = vel[q] * dt / h;
        coef[q] = nu * nu;
    }
    oracle_cerjan_profile(nx, sponge, sponge_a, gx);
    oracle_cerjan_profile(ny, sponge, sponge_a, gy);
    oracle_cerjan_profile(nz, sponge, sponge_a, gz);
    load_interior(&g, a, init_cur ? u_cur : NULL);
    load_interior(&g, b, init_prev ? u_prev : NULL);

    double c[5];
    oracle_stencil_coefficients(c);
    if (nthreads < 1) nthreads = 1;

    for (int n = 0; n < nsteps; ++n) {
        if (periodic) fill_periodic_halo(&g, a);
        /* b <- u_{n+1}, computed point by point from a = u_n, b = u_{n-1} */
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < nx; ++i) {
                    long p = at(&g, i, j, k);
                    long q = (k * ny + j) * nx + i;
                    double G = gx[i] * gy[j] * gz[k];
                    double lap = lap_at(&g, a, c, i, j, k);
                    if (wavelet && i == sx && j == sy && k == sz)
                        lap += wavelet[n];
                    b[p] = G * (2.0 * a[p] - G * b[p] + coef[q] * lap);
                }
        double *t = a; a = b; b = t;   /* a = u_{n+1}, b = u_n */
        for (int r = 0; r < nrec; ++r)
            traces[(long)r * nsteps + n] =
                a[at(&g, rec_xyz[3 * r], rec_xyz[3 * r + 1],
                     rec_xyz[3 * r + 2])];
        if (norms) {
            double s = 0.0;
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        double v = a[at(&g, i, j, k)];
                        s += v * v;
                    }
            norms[n] = s;
        }
    }
    store_interior(&g, a, u_cur);
    store_interior(&g, b, u_prev);
    free(a); free(b); free(coef); free(gx); free(gy); free(gz);
    return 0;
}
