/*
 * FP64 CPU ORACLE -- test infrastructure only.
 *
 * Only tests/, the package smoke check and the benchmark's CPU-baseline leg
 * may load this file's library; the product path never does.
 *
 * Plain time stepping of the constant-density acoustic wave equation
 * (Section "Theory", eq. wave_eq):  m u_tt - lap(u) = delta(x - x_s) f(t),
 * with m = 1/v^2.  The paper does not give its discretisation; the readings
 * taken here are:
 *   - second-order leapfrog in time, eighth-order central differences in
 *     space (coefficients -205/72, 8/5, -1/5, 8/315, -1/560), u = 0 outside
 *     the padded grid;
 *   - an absorbing sponge written as a damping term eta u_t, discretised
 *     symmetrically so that the time-stepping matrix stays symmetric in
 *     space and source-receiver reciprocity holds exactly:
 *       (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} + dt^2 v^2 (L u^n + f^n),
 *     a = eta dt / 2, u^0 = u^{-1} = 0;
 *   - a point source of amplitude s at grid point p enters as
 *     f^n = s^n / (dx dz) at p (discrete delta in space).
 * Recorded fields are u^0 .. u^{nt-1}.  Optionally the whole field is
 * transformed on the fly at arbitrary frequencies f_k:
 *       ghat_k(x) = sum_{n=0}^{nt-1} u^n(x) exp(-i 2 pi f_k n dt),
 * with the phase reduced as 2 pi frac(f_k n dt) in double precision.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double C8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

/* Runs nt recorded time levels.  Returns 0 on success, 1 on bad arguments, 2 on
 * allocation failure.
 *   vel, eta  [NZ*NX]   padded velocity (m/s) and damping (1/s), row-major, x fastest
 *   src_p     [nsrc]    injection point indices into the padded grid
 *   src_f     [nsrc*nt] source amplitude per point and time step (may be NULL if nsrc == 0)
 *   rec_p     [nrec]    recording point indices; traces [nrec*nt] (NULL to skip)
 *   freqs     [nf]      Hz; ghat [nf*NZ*NX*2] interleaved re/im accumulators (NULL to skip)
 *   snaps     [nt*NZ*NX] every recorded level (NULL to skip)
 */
int oracle_fd_run(int NZ, int NX, double dz, double dx, double dt, int nt,
                  const double *vel, const double *eta,
                  int nsrc, const int *src_p, const double *src_f,
                  int nrec, const int *rec_p, double *traces,
                  int nf, const double *freqs, double *ghat,
                  double *snaps, int nthreads)
{
    if (NZ <= 0 || NX <= 0 || nt <= 0 || dz <= 0.0 || dx <= 0.0 || dt <= 0.0)
        return 1;
    const long np = (long)NZ * NX;
    double *u_prev = calloc((size_t)np, sizeof(double));
    double *u_cur = calloc((size_t)np, sizeof(double));
    double *u_next = calloc((size_t)np, sizeof(double));
    double *fsrc = calloc((size_t)np, sizeof(double));
    double *cw = nf > 0 ? malloc((size_t)nf * 2 * sizeof(double)) : NULL;
    if (!u_prev || !u_cur || !u_next || !fsrc || (nf > 0 && !cw)) {
        free(u_prev); free(u_cur); free(u_next); free(fsrc); free(cw);
        return 2;
    }
    if (ghat)
        memset(ghat, 0, sizeof(double) * 2 * (size_t)nf * (size_t)np);
    const double idx2 = 1.0 / (dx * dx), idz2 = 1.0 / (dz * dz);
    const double area = dx * dz;
    (void)nthreads;

    for (int n = 0; n < nt; ++n) {
        /* record level n */
        if (traces)
            for (int r = 0; r < nrec; ++r)
                traces[(long)r * nt + n] = u_cur[rec_p[r]];
        if (snaps)
            memcpy(snaps + (long)n * np, u_cur, sizeof(double) * (size_t)np);
        if (ghat) {
            for (int k = 0; k < nf; ++k) {
                double ph = freqs[k] * (double)n * dt;
                ph -= floor(ph);
                cw[2 * k] = cos(2.0 * M_PI * ph);
                cw[2 * k + 1] = -sin(2.0 * M_PI * ph);
            }
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (long p = 0; p < np; ++p) {
                const double u = u_cur[p];
                for (int k = 0; k < nf; ++k) {
                    double *g = ghat + 2 * ((long)k * np + p);
                    g[0] += u * cw[2 * k];
                    g[1] += u * cw[2 * k + 1];
                }
            }
        }
        if (n == nt - 1)
            break;
        /* source term f^n */
        for (int s = 0; s < nsrc; ++s)
            fsrc[src_p[s]] += src_f[(long)s * nt + n] / area;
        /* u^{n+1} */
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (int z = 0; z < NZ; ++z) {
            for (int x = 0; x < NX; ++x) {
                const long p = (long)z * NX + x;
                double lap = 0.0;
                for (int k = -4; k <= 4; ++k) {
                    const double c = C8[k < 0 ? -k : k];
                    if (x + k >= 0 && x + k < NX)
                        lap += c * idx2 * u_cur[p + k];
                    if (z + k >= 0 && z + k < NZ)
                        lap += c * idz2 * u_cur[p + (long)k * NX];
                }
                const double a = 0.5 * eta[p] * dt;
                const double v = vel[p];
                u_next[p] = (2.0 * u_cur[p] - (1.0 - a) * u_prev[p]
                             + dt * dt * v * v * (lap + fsrc[p])) / (1.0 + a);
            }
        }
        for (int s = 0; s < nsrc; ++s)
            fsrc[src_p[s]] = 0.0;
        double *t = u_prev;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = t;
    }
    free(u_prev); free(u_cur); free(u_next); free(fsrc); free(cw);
    return 0;
}
