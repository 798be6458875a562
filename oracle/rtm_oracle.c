/*
 * FP64 CPU oracle for the RTM hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library. The product (the CUDA library) never calls it, and the
 * two share no code.
 *
 * What it computes (the method is stated in the paper only as "a PDE solver
 * that applies a high order stencil to a 3D block of data in each time step"
 * simulating pressure waves, Sec. I and Sec. II; the discrete recursion below
 * is the reading that the accompanying Python wrapper documents):
 *
 *   L u      = sum over the three axes of
 *              [ a0 u + sum_{k=1..r} a_k (u_{+k} + u_{-k}) ] / dx^2,
 *              zero (Dirichlet) ghost cells outside the padded grid;
 *   u^{n+1}  = g (2 u^n + c L u^n) - g^2 u^{n-1},  g = gx*gy*gz, c = v^2 dt^2;
 *   u^{n+1}[s] += c[s] w^n / dx^3                (source injection);
 *   d[n][j]  = u^{n+1}[rec_j]                     (receiver gather);
 *
 * and the receiver (adjoint) propagation run backward in time,
 *
 *   mu^m     = g (2 mu^{m+1} + c L mu^{m+1}) - g^2 mu^{m+2}, m = nt..1,
 *   mu^m[rec_j] += c g r^{m-1}_j / dx^3,          mu^{nt+1} = mu^{nt+2} = 0,
 *   I(x)    += u^m(x) mu^m(x)                     (zero-lag imaging),
 *   G_i     += mu^m_i (L u^{m-1})_i  (+ mu^m_s w^{m-1} / (dx^3 g_s) at i = s).
 *
 * Loops run z, y, x with x innermost, the order the paper settles on in
 * Sec. III; the z loop is split over OpenMP threads with a dynamic schedule
 * (also Sec. III). Nothing else is blocked, fused or reordered.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int NX, NY, NZ;      /* padded (computational) grid */
    int nb;              /* sponge width; the model region is [nb, N - nb) per axis */
    int r;               /* stencil radius: order 2r in space */
    double dx;           /* grid spacing (m) */
    const double *a;     /* a[0..r] second-derivative weights */
    const double *c;     /* v^2 dt^2 on the padded grid, [NZ][NY][NX] */
    const double *gx;    /* sponge profile along x, NX entries */
    const double *gy;    /* along y, NY entries */
    const double *gz;    /* along z, NZ entries */
} orc_grid;

static size_t lin(const orc_grid *G, int x, int y, int z)
{
    return ((size_t)z * (size_t)G->NY + (size_t)y) * (size_t)G->NX + (size_t)x;
}

/* u at (x, y, z); zero outside the padded grid (Dirichlet ghost cells) */
static double at(const orc_grid *G, const double *u, int x, int y, int z)
{
    if (x < 0 || x >= G->NX || y < 0 || y >= G->NY || z < 0 || z >= G->NZ)
        return 0.0;
    return u[lin(G, x, y, z)];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* lu = L u over the whole padded grid */
void orc_laplacian(const orc_grid *G, const double *u, double *lu)
{
    const double inv_dx2 = 1.0 / (G->dx * G->dx);
#pragma omp parallel for schedule(dynamic)
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                double s = 3.0 * G->a[0] * u[lin(G, x, y, z)];
                for (int k = 1; k <= G->r; k++) {
                    double pair_x = at(G, u, x + k, y, z) + at(G, u, x - k, y, z);
                    double pair_y = at(G, u, x, y + k, z) + at(G, u, x, y - k, z);
                    double pair_z = at(G, u, x, y, z + k) + at(G, u, x, y, z - k);
                    s += G->a[k] * (pair_x + pair_y + pair_z);
                }
                lu[lin(G, x, y, z)] = s * inv_dx2;
            }
}

/* u_next = g (2 u_cur + c lu) - g^2 u_prev, with lu = L u_cur given */
static void leapfrog(const orc_grid *G, const double *u_cur, const double *u_prev,
                     const double *lu, double *u_next)
{
#pragma omp parallel for schedule(dynamic)
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                size_t i = lin(G, x, y, z);
                double g = G->gx[x] * G->gy[y] * G->gz[z];
                u_next[i] = g * (2.0 * u_cur[i] + G->c[i] * lu[i]) - g * g * u_prev[i];
            }
}

/* one time step without sources: u_next = g (2 u_cur + c L u_cur) - g^2 u_prev */
void orc_step(const orc_grid *G, const double *u_cur, const double *u_prev, double *u_next)
{
    size_t n = (size_t)G->NX * G->NY * G->NZ;
    double *lu = (double *)malloc(n * sizeof(double));
    orc_laplacian(G, u_cur, lu);
    leapfrog(G, u_cur, u_prev, lu, u_next);
    free(lu);
}

static double sponge(const orc_grid *G, size_t i)
{
    size_t plane = (size_t)G->NX * G->NY;
    int z = (int)(i / plane);
    int y = (int)((i % plane) / G->NX);
    int x = (int)(i % G->NX);
    return G->gx[x] * G->gy[y] * G->gz[z];
}

/* copy the model region of a padded field into a dense model-grid array */
static void extract_model(const orc_grid *G, const double *u, double *out)
{
    int nx = G->NX - 2 * G->nb, ny = G->NY - 2 * G->nb, nz = G->NZ - 2 * G->nb;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                out[((size_t)z * ny + y) * nx + x] = u[lin(G, x + G->nb, y + G->nb, z + G->nb)];
}

/*
 * Forward modelling from zero initial fields u^{-1} = u^0 = 0.
 *   w        [nt]          source wavelet samples w^n = w(n dt)
 *   src      linear padded index of the source point
 *   rec      [nrec]        linear padded indices of the receivers
 *   data     [nt][nrec]    d[n][j] = u^{n+1}[rec_j]           (may be NULL)
 *   snap_u   [nt][model]   u^{n+1} on the model region         (may be NULL)
 *   snap_lu  [nt][padded]  L u^n on the padded grid            (may be NULL)
 *   u_last   [2][padded]   u^{nt-1}, u^{nt}                    (may be NULL)
 * Returns 0, or -1 if memory could not be allocated.
 */
int orc_forward(const orc_grid *G, int nt, const double *w, int64_t src, int nrec,
                const int64_t *rec, double *data, double *snap_u, double *snap_lu,
                double *u_last)
{
    size_t n = (size_t)G->NX * G->NY * G->NZ;
    size_t nmodel = (size_t)(G->NX - 2 * G->nb) * (G->NY - 2 * G->nb) * (G->NZ - 2 * G->nb);
    double *u_prev = (double *)calloc(n, sizeof(double));
    double *u_cur = (double *)calloc(n, sizeof(double));
    double *u_next = (double *)calloc(n, sizeof(double));
    double *lu = (double *)calloc(n, sizeof(double));
    if (!u_prev || !u_cur || !u_next || !lu) {
        free(u_prev); free(u_cur); free(u_next); free(lu);
        return -1;
    }
    const double dx3 = G->dx * G->dx * G->dx;
    for (int step = 0; step < nt; step++) {
        orc_laplacian(G, u_cur, lu);
        if (snap_lu)
            memcpy(snap_lu + (size_t)step * n, lu, n * sizeof(double));
        leapfrog(G, u_cur, u_prev, lu, u_next);
        u_next[src] += G->c[src] * w[step] / dx3;
        if (data)
            for (int j = 0; j < nrec; j++)
                data[(size_t)step * nrec + j] = u_next[rec[j]];
        if (snap_u)
            extract_model(G, u_next, snap_u + (size_t)step * nmodel);
        double *t = u_prev; u_prev = u_cur; u_cur = u_next; u_next = t;
    }
    if (u_last) {
        memcpy(u_last, u_prev, n * sizeof(double));
        memcpy(u_last + n, u_cur, n * sizeof(double));
    }
    free(u_prev); free(u_cur); free(u_next); free(lu);
    return 0;
}

/*
 * Receiver propagation backward in time with imaging and gradient terms.
 *   resid    [nt][nrec]    r^n, the data injected at the receivers
 *   snap_u   [nt][model]   u^{m} (entry m-1), needed when image != NULL
 *   image    [model]       += sum over m with m % image_every == 0 of u^m mu^m
 *   snap_lu  [nt][padded]  L u^{n} (entry n), needed when grad_acc != NULL
 *   grad_acc [padded]      += sum_m mu^m (L u^{m-1}) (+ source term at src)
 *   src_adj  [nt]          src_adj[n] = mu^{n+1}[src] / g_src      (may be NULL)
 *   mu_last  [2][padded]   mu^2, mu^1                               (may be NULL)
 * Returns 0, or -1 if memory could not be allocated.
 */
int orc_adjoint(const orc_grid *G, int nt, const double *w, int64_t src, int nrec,
                const int64_t *rec, const double *resid, const double *snap_u,
                int image_every, double *image, const double *snap_lu, double *grad_acc,
                double *src_adj, double *mu_last)
{
    size_t n = (size_t)G->NX * G->NY * G->NZ;
    int nx = G->NX - 2 * G->nb, ny = G->NY - 2 * G->nb, nz = G->NZ - 2 * G->nb;
    size_t nmodel = (size_t)nx * ny * nz;
    double *mu_2 = (double *)calloc(n, sizeof(double)); /* mu^{m+2} */
    double *mu_1 = (double *)calloc(n, sizeof(double)); /* mu^{m+1} */
    double *mu_0 = (double *)calloc(n, sizeof(double)); /* mu^{m}   */
    double *lu = (double *)calloc(n, sizeof(double));
    if (!mu_2 || !mu_1 || !mu_0 || !lu) {
        free(mu_2); free(mu_1); free(mu_0); free(lu);
        return -1;
    }
    const double dx3 = G->dx * G->dx * G->dx;
    const double g_src = sponge(G, (size_t)src);
    for (int m = nt; m >= 1; m--) {
        orc_laplacian(G, mu_1, lu);
        leapfrog(G, mu_1, mu_2, lu, mu_0);
        for (int j = 0; j < nrec; j++) {
            size_t i = (size_t)rec[j];
            mu_0[i] += G->c[i] * sponge(G, i) * resid[(size_t)(m - 1) * nrec + j] / dx3;
        }
        if (image && (m % image_every) == 0) {
            const double *u = snap_u + (size_t)(m - 1) * nmodel;
            for (int z = 0; z < nz; z++)
                for (int y = 0; y < ny; y++)
                    for (int x = 0; x < nx; x++) {
                        size_t im = ((size_t)z * ny + y) * nx + x;
                        image[im] += u[im] * mu_0[lin(G, x + G->nb, y + G->nb, z + G->nb)];
                    }
        }
        if (grad_acc) {
            const double *lu_u = snap_lu + (size_t)(m - 1) * n;
            for (size_t i = 0; i < n; i++)
                grad_acc[i] += mu_0[i] * lu_u[i];
            grad_acc[src] += mu_0[src] * w[m - 1] / (dx3 * g_src);
        }
        if (src_adj)
            src_adj[m - 1] = mu_0[src] / g_src;
        double *t = mu_2; mu_2 = mu_1; mu_1 = mu_0; mu_0 = t;
    }
    if (mu_last) {
        memcpy(mu_last, mu_2, n * sizeof(double));
        memcpy(mu_last + n, mu_1, n * sizeof(double));
    }
    free(mu_2); free(mu_1); free(mu_0); free(lu);
    return 0;
}
