/*
 * oracle/stencil.c -- TEST INFRASTRUCTURE ONLY.  Plain FP64 CPU stencils
 * (triple loops, OpenMP over z) that define what the GPU stencil path must
 * compute.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg and reference arm may load this.
 *
 * Grids are [z][y][x] (x fastest).  Values outside [0,n) on any axis are
 * zero ghosts (Dirichlet zero), as deep as the stencil reaches.
 *
 * heat7 (Section III: each point's new value is the average of its
 * neighbours, here in 3D and written in delta form):
 *     u' = u + r * (u[x-1] + u[x+1] + u[y-1] + u[y+1] + u[z-1] + u[z+1] - 6 u)
 * r = 1/6 gives the pure neighbour average.
 *
 * wave25 (Section VI: the 25-point acoustic propagator with HALO = 4,
 * Table I), second-order leapfrog in time with the 8th-order central
 * second difference on each axis:
 *     L(p) = sum_axes [ c0 p + sum_{m=1..4} c_m (p[+m] + p[-m]) ]
 *     c = (-205/72, 8/5, -1/5, 8/315, -1/560)
 *     p_next = 2 p - p_prev + kappa * L(p),   kappa = (v dt / dx)^2
 *     p_next[src] += w
 * kappa is the read-only dataset; the source amplitude w is an input.
 */
#include <stdint.h>
#include <stddef.h>

static const double C8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

static inline double at(const double *f, int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y, int64_t z)
{
    if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz)
        return 0.0;
    return f[(z * ny + y) * nx + x];
}

void oracle_heat7_step(const double *u, double *out, int64_t nx, int64_t ny, int64_t nz, double r)
{
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                double c = at(u, nx, ny, nz, x, y, z);
                double s = at(u, nx, ny, nz, x - 1, y, z) + at(u, nx, ny, nz, x + 1, y, z) +
                           at(u, nx, ny, nz, x, y - 1, z) + at(u, nx, ny, nz, x, y + 1, z) +
                           at(u, nx, ny, nz, x, y, z - 1) + at(u, nx, ny, nz, x, y, z + 1);
                out[(z * ny + y) * nx + x] = c + r * (s - 6.0 * c);
            }
}

/* Dimensionless 8th-order Laplacian L(p) (no kappa). */
void oracle_laplacian8(const double *p, double *out, int64_t nx, int64_t ny, int64_t nz)
{
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                double c = at(p, nx, ny, nz, x, y, z);
                double acc = 3.0 * C8[0] * c;
                for (int m = 1; m <= 4; m++)
                    acc += C8[m] * (at(p, nx, ny, nz, x + m, y, z) + at(p, nx, ny, nz, x - m, y, z) +
                                    at(p, nx, ny, nz, x, y + m, z) + at(p, nx, ny, nz, x, y - m, z) +
                                    at(p, nx, ny, nz, x, y, z + m) + at(p, nx, ny, nz, x, y, z - m));
                out[(z * ny + y) * nx + x] = acc;
            }
}

/* One leapfrog step; src < 0 means no source. */
void oracle_wave25_step(const double *p, const double *p_prev, const double *kappa, double *out,
                        int64_t nx, int64_t ny, int64_t nz, int64_t src, double w)
{
    oracle_laplacian8(p, out, nx, ny, nz);
    int64_t n = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        out[i] = 2.0 * p[i] - p_prev[i] + kappa[i] * out[i];
    if (src >= 0 && src < n)
        out[src] += w;
}

/* nsteps heat steps in place on u, using tmp (same size) as scratch. */
void oracle_heat7_run(double *u, double *tmp, int64_t nx, int64_t ny, int64_t nz, double r, int64_t nsteps)
{
    int64_t n = nx * ny * nz;
    for (int64_t s = 0; s < nsteps; s++) {
        oracle_heat7_step(u, tmp, nx, ny, nz, r);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            u[i] = tmp[i];
    }
}

/* The same heat steps in FP32 (float inputs, float arithmetic in the
 * delta form above, zero ghosts): the CPU doing the GPU's FP32 work, for
 * timing beside the FP64 oracle.  Not a reference: FP32 rounding differs
 * from the FP64 definition by about 1e-7 per step. */
static inline float atf(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y, int64_t z)
{
    if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz)
        return 0.0f;
    return f[(z * ny + y) * nx + x];
}

void oracle_heat7_run_f32(float *u, float *tmp, int64_t nx, int64_t ny, int64_t nz, float r, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; s++) {
        float *in = (s & 1) ? tmp : u, *out = (s & 1) ? u : tmp;
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; z++)
            for (int64_t y = 0; y < ny; y++)
                for (int64_t x = 0; x < nx; x++) {
                    float c = atf(in, nx, ny, nz, x, y, z);
                    float sum = atf(in, nx, ny, nz, x - 1, y, z) + atf(in, nx, ny, nz, x + 1, y, z) +
                                atf(in, nx, ny, nz, x, y - 1, z) + atf(in, nx, ny, nz, x, y + 1, z) +
                                atf(in, nx, ny, nz, x, y, z - 1) + atf(in, nx, ny, nz, x, y, z + 1);
                    out[(z * ny + y) * nx + x] = c + r * (sum - 6.0f * c);
                }
    }
    if (nsteps & 1) {
        int64_t n = nx * ny * nz;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            u[i] = tmp[i];
    }
}

/* nsteps leapfrog steps.  On entry (p, p_prev) = (p^t, p^{t-1}); on return
 * (p^{t+nsteps}, p^{t+nsteps-1}).  Step j (0-based) adds w[t0 + j] at src,
 * where w has at least t0 + nsteps entries (or is NULL). */
void oracle_wave25_run(double *p, double *p_prev, const double *kappa, double *tmp,
                       int64_t nx, int64_t ny, int64_t nz, int64_t src, const double *w,
                       int64_t t0, int64_t nsteps)
{
    int64_t n = nx * ny * nz;
    for (int64_t s = 0; s < nsteps; s++) {
        oracle_wave25_step(p, p_prev, kappa, tmp, nx, ny, nz, src, w ? w[t0 + s] : 0.0);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            p_prev[i] = p[i];
            p[i] = tmp[i];
        }
    }
}
