/*
 * oracle/adjoint.c -- TEST INFRASTRUCTURE ONLY.  FP64 CPU reference of the
 * discrete adjoint of the wave25 leapfrog propagator (oracle/stencil.c), used
 * to check the GPU adjoint and gradient.  Not part of the paper: the
 * differentiation workload asks for the gradient of an L2 receiver misfit
 * with respect to the velocity model.
 *
 * Forward, n = 0 .. N-1, with p^0 = p^{-1} = 0:
 *     p^{n+1} = 2 p^n - p^{n-1} + kappa * L(p^n) + w[n] delta_src
 * Traces: tr[n-1][r] = p^n(rec[r]), n = 1 .. N.
 * Misfit: J = 1/2 sum_{n,r} (tr[n-1][r] - d[n-1][r])^2.
 *
 * Adjoint (transpose of the forward map, L symmetric with zero ghosts):
 *     mu^{N+1} = mu^{N+2} = 0,
 *     mu^m = 2 mu^{m+1} - mu^{m+2} + L(kappa * mu^{m+1}) + S^T res_m,  m = N..1
 *     dJ/dkappa = sum_{n=0}^{N-1} mu^{n+1} * L(p^n)
 * with res_m = tr[m-1] - d[m-1] scattered to the receivers (S^T).
 *
 * Born (linearised forward in kappa), for the dot-product test:
 *     dp^{n+1} = 2 dp^n - dp^{n-1} + kappa * L(dp^n) + dkappa * L(p^n)
 *     dtr[n-1][r] = dp^n(rec[r])
 *
 * Everything runs from scratch with the full wavefield history in memory:
 * plain and slow by design.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_laplacian8(const double *p, double *out, int64_t nx, int64_t ny, int64_t nz);

/* Forward run storing p^0 .. p^N in hist ((N+1) * n doubles) and the traces. */
static void forward_history(const double *kappa, int64_t nx, int64_t ny, int64_t nz, int64_t src, const double *w,
                            int64_t N, const int64_t *rec, int64_t nrec, double *hist, double *traces)
{
    const int64_t n = nx * ny * nz;
    double *lap = (double *)malloc(sizeof(double) * n);
    double *prev = (double *)calloc(n, sizeof(double)); /* p^{-1} = 0 */
    memset(hist, 0, sizeof(double) * n);               /* p^0 = 0 */
    for (int64_t s = 0; s < N; s++) {
        const double *p = hist + s * n;
        const double *pm = s == 0 ? prev : hist + (s - 1) * n;
        double *out = hist + (s + 1) * n;
        oracle_laplacian8(p, lap, nx, ny, nz);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            out[i] = 2.0 * p[i] - pm[i] + kappa[i] * lap[i];
        if (src >= 0 && src < n && w)
            out[src] += w[s];
        for (int64_t r = 0; r < nrec; r++)
            traces[s * nrec + r] = out[rec[r]];
    }
    free(lap);
    free(prev);
}

/* Traces only (returns 0, or -1 on allocation failure). */
int oracle_wave25_traces(const double *kappa, int64_t nx, int64_t ny, int64_t nz, int64_t src, const double *w,
                         int64_t N, const int64_t *rec, int64_t nrec, double *traces)
{
    const int64_t n = nx * ny * nz;
    double *hist = (double *)malloc(sizeof(double) * n * (N + 1));
    if (!hist)
        return -1;
    forward_history(kappa, nx, ny, nz, src, w, N, rec, nrec, hist, traces);
    free(hist);
    return 0;
}

/* Gradient dJ/dkappa for the residual res[N][nrec] (= dJ/dtraces). */
int oracle_wave25_adjoint_grad(const double *kappa, int64_t nx, int64_t ny, int64_t nz, int64_t src, const double *w,
                               int64_t N, const int64_t *rec, int64_t nrec, const double *res, double *grad)
{
    const int64_t n = nx * ny * nz;
    double *hist = (double *)malloc(sizeof(double) * n * (N + 1));
    double *traces = (double *)malloc(sizeof(double) * (N > 0 ? N : 1) * (nrec > 0 ? nrec : 1));
    double *mu1 = (double *)calloc(n, sizeof(double)); /* mu^{m+1} */
    double *mu2 = (double *)calloc(n, sizeof(double)); /* mu^{m+2} */
    double *mu0 = (double *)malloc(sizeof(double) * n);
    double *tmp = (double *)malloc(sizeof(double) * n);
    double *lap = (double *)malloc(sizeof(double) * n);
    if (!hist || !traces || !mu1 || !mu2 || !mu0 || !tmp || !lap)
        return -1;
    forward_history(kappa, nx, ny, nz, src, w, N, rec, nrec, hist, traces);
    memset(grad, 0, sizeof(double) * n);
    for (int64_t m = N; m >= 1; m--) {
        /* mu^m = 2 mu^{m+1} - mu^{m+2} + L(kappa mu^{m+1}) + S^T res_m */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            tmp[i] = kappa[i] * mu1[i];
        oracle_laplacian8(tmp, lap, nx, ny, nz);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            mu0[i] = 2.0 * mu1[i] - mu2[i] + lap[i];
        for (int64_t r = 0; r < nrec; r++)
            mu0[rec[r]] += res[(m - 1) * nrec + r];
        /* gradient term n = m - 1: mu^{m} * L(p^{m-1}) */
        oracle_laplacian8(hist + (m - 1) * n, lap, nx, ny, nz);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            grad[i] += mu0[i] * lap[i];
        double *t = mu2;
        mu2 = mu1;
        mu1 = mu0;
        mu0 = t;
    }
    free(hist);
    free(traces);
    free(mu0);
    free(mu1);
    free(mu2);
    free(tmp);
    free(lap);
    return 0;
}

/* Born traces dtr for a kappa perturbation dkappa. */
int oracle_wave25_born(const double *kappa, const double *dkappa, int64_t nx, int64_t ny, int64_t nz, int64_t src,
                       const double *w, int64_t N, const int64_t *rec, int64_t nrec, double *dtraces)
{
    const int64_t n = nx * ny * nz;
    double *hist = (double *)malloc(sizeof(double) * n * (N + 1));
    double *traces = (double *)malloc(sizeof(double) * (N > 0 ? N : 1) * (nrec > 0 ? nrec : 1));
    double *dp = (double *)calloc(n, sizeof(double));
    double *dpm = (double *)calloc(n, sizeof(double));
    double *dnext = (double *)malloc(sizeof(double) * n);
    double *lap = (double *)malloc(sizeof(double) * n);
    double *lap2 = (double *)malloc(sizeof(double) * n);
    if (!hist || !traces || !dp || !dpm || !dnext || !lap || !lap2)
        return -1;
    forward_history(kappa, nx, ny, nz, src, w, N, rec, nrec, hist, traces);
    for (int64_t s = 0; s < N; s++) {
        oracle_laplacian8(dp, lap, nx, ny, nz);
        oracle_laplacian8(hist + s * n, lap2, nx, ny, nz);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            dnext[i] = 2.0 * dp[i] - dpm[i] + kappa[i] * lap[i] + dkappa[i] * lap2[i];
        for (int64_t r = 0; r < nrec; r++)
            dtraces[s * nrec + r] = dnext[rec[r]];
        double *t = dpm;
        dpm = dp;
        dp = dnext;
        dnext = t;
    }
    free(hist);
    free(traces);
    free(dp);
    free(dpm);
    free(dnext);
    free(lap);
    free(lap2);
    return 0;
}
