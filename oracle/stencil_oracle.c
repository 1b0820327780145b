/*
 * Stencil oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU implementation of what the GPU library
 * computes.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this file's library; the GPU library never links it
 * and shares no code with it.
 *
 * What it computes (gather mode, Eq. (stencil-2d9p) and its coefficient
 * matrix, Eq. (stencil-2d9p-cm), generalised to d = 2, 3 dimensions and
 * order r):
 *
 *     B[x] = sum over o in [0, 2r]^d, in lexicographic order, of C^g[o] * A[x + o - r]
 *
 * One call advances the field `steps` times using two array copies used
 * alternately as input and output (Sec. 2.2).  The scatter-mode outer-product
 * formulation of Sec. 3 (Eq. (final)) is an exact re-association of this sum,
 * so the oracle is the definition itself, not the algorithm.
 *
 * Boundary (the paper only computes interior points with a halo of width r,
 * Eq. (final) output indices start at r): `shape` is the interior; with
 * DIRICHLET_ZERO every point outside it reads 0 at every step; with PERIODIC an
 * index is taken modulo the extent in each dimension.
 *
 * Arithmetic: plain multiply then add (compile with -ffp-contract=off), terms
 * summed in the lexicographic order of o, accumulator starts at +0.0.  The
 * result does not depend on the thread count (threads split the outermost
 * dimension only).
 *
 * Parity is pinned by the CPU test suite against: the scatter form
 * (Eq. (stencil-2d9p-scatter) with C^s = J C^g J), Eq. (final) with the
 * corrected column pairing, Algorithm 1, constant fields, linearity,
 * polynomial fields and closed-form Fourier/sine eigenmodes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_DIRICHLET_ZERO 0
#define ORACLE_PERIODIC 1

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

static int64_t wrap_index(int64_t i, int64_t n)
{
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* Value of A at (possibly out-of-range) interior coordinates x[0..ndim-1]. */
static double fetch(int ndim, const int64_t *n, int bc, const double *A, const int64_t *x)
{
    int64_t lin = 0;
    for (int d = 0; d < ndim; ++d) {
        int64_t xi = x[d];
        if (xi < 0 || xi >= n[d]) {
            if (bc == ORACLE_DIRICHLET_ZERO)
                return 0.0;
            xi = wrap_index(xi, n[d]);
        }
        lin = lin * n[d] + xi;
    }
    return A[lin];
}

/* One gather sweep over the whole interior. */
static void sweep(int ndim, const int64_t *n, int r, const double *cg, int bc,
                  const double *A, double *B)
{
    const int w = 2 * r + 1;
    const int64_t inner = (ndim == 3) ? n[1] * n[2] : n[1];
#pragma omp parallel for schedule(static)
    for (int64_t i0 = 0; i0 < n[0]; ++i0) {
        int64_t x[3], y[3];
        for (int64_t rest = 0; rest < inner; ++rest) {
            x[0] = i0;
            if (ndim == 3) {
                x[1] = rest / n[2];
                x[2] = rest % n[2];
            } else {
                x[1] = rest;
            }
            double acc = 0.0;
            int64_t nterm = 1;
            for (int d = 0; d < ndim; ++d)
                nterm *= w;
            for (int64_t t = 0; t < nterm; ++t) {
                /* o = lexicographic multi-index of t, last index fastest */
                int64_t rem = t;
                for (int d = ndim - 1; d >= 0; --d) {
                    int64_t o = rem % w;
                    rem /= w;
                    y[d] = x[d] + o - r;
                }
                double prod = cg[t] * fetch(ndim, n, bc, A, y);
                acc = acc + prod;
            }
            B[i0 * inner + rest] = acc;
        }
    }
}

static int check_args(int ndim, const int64_t *shape, int r, int bc)
{
    if (ndim != 2 && ndim != 3)
        return ORACLE_EINVAL;
    if (r < 1 || r > 8)
        return ORACLE_EINVAL;
    if (bc != ORACLE_DIRICHLET_ZERO && bc != ORACLE_PERIODIC)
        return ORACLE_EINVAL;
    for (int d = 0; d < ndim; ++d)
        if (shape[d] < 1)
            return ORACLE_EINVAL;
    return ORACLE_OK;
}

/*
 * Advance `in` by `steps` gather sweeps; result in `out` (may alias `in`).
 * steps == 0 copies.
 */
int oracle_gather(int ndim, const int64_t *shape, int r, const double *cg, int bc,
                  int64_t steps, const double *in, double *out)
{
    int rc = check_args(ndim, shape, r, bc);
    if (rc)
        return rc;
    if (steps < 0)
        return ORACLE_EINVAL;
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d)
        total *= shape[d];
    if (steps == 0) {
        if (out != in)
            memmove(out, in, (size_t)total * sizeof(double));
        return ORACLE_OK;
    }
    double *a = (double *)malloc((size_t)total * sizeof(double));
    double *b = (double *)malloc((size_t)total * sizeof(double));
    if (!a || !b) {
        free(a);
        free(b);
        return ORACLE_ENOMEM;
    }
    memcpy(a, in, (size_t)total * sizeof(double));
    for (int64_t s = 0; s < steps; ++s) {
        sweep(ndim, shape, r, cg, bc, a, b);
        double *t = a;
        a = b;
        b = t;
    }
    memcpy(out, a, (size_t)total * sizeof(double));
    free(a);
    free(b);
    return ORACLE_OK;
}

/*
 * Values of single output points after `steps` sweeps, each computed on its
 * own dependency cone: a local window of half-width R = r*steps around the
 * point, filled from `in` with the boundary rule, then swept `steps` times.
 * After sweep s only the points within R - r*s of the centre are needed (and
 * correct), so the window shrinks accordingly.  With DIRICHLET_ZERO, window
 * points outside the interior are held at 0 at every step.  Each value equals
 * the corresponding element of oracle_gather bit for bit (same terms, same
 * order).  `max_window` bounds the window's point count (ORACLE_ENOMEM past it).
 */
int oracle_sample(int ndim, const int64_t *shape, int r, const double *cg, int bc,
                  int64_t steps, const double *in, int64_t npts, const int64_t *pts,
                  double *vals, int64_t max_window)
{
    int rc = check_args(ndim, shape, r, bc);
    if (rc)
        return rc;
    if (steps < 0)
        return ORACLE_EINVAL;
    const int64_t R = (int64_t)r * steps;
    const int64_t L = 2 * R + 1;
    int64_t wpts = 1;
    for (int d = 0; d < ndim; ++d) {
        if (L > 0 && wpts > max_window / L)
            return ORACLE_ENOMEM;
        wpts *= L;
    }
    const int w = 2 * r + 1;
    int64_t nterm = 1;
    for (int d = 0; d < ndim; ++d)
        nterm *= w;
    int status = ORACLE_OK;
#pragma omp parallel
    {
        double *u = (double *)malloc((size_t)wpts * sizeof(double));
        double *v = (double *)malloc((size_t)wpts * sizeof(double));
        unsigned char *outside = (unsigned char *)malloc((size_t)wpts);
        const int have_mem = (u && v && outside);
        {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < npts; ++p) {
                if (!have_mem) {
#pragma omp atomic write
                    status = ORACLE_ENOMEM;
                    continue;
                }
                const int64_t *c = pts + p * ndim;
                int64_t x[3], y[3], l[3];
                /* fill the window */
                for (int64_t q = 0; q < wpts; ++q) {
                    int64_t rem = q;
                    int out = 0;
                    for (int d = ndim - 1; d >= 0; --d) {
                        l[d] = rem % L;
                        rem /= L;
                        y[d] = c[d] + l[d] - R;
                        if (y[d] < 0 || y[d] >= shape[d])
                            out = 1;
                    }
                    outside[q] = (unsigned char)(out && bc == ORACLE_DIRICHLET_ZERO);
                    u[q] = fetch(ndim, shape, bc, in, y);
                }
                /* sweeps on the shrinking cone */
                for (int64_t s = 1; s <= steps; ++s) {
                    const int64_t h = R - (int64_t)r * s; /* half-width still needed */
                    int64_t side = 2 * h + 1, cnt = 1;
                    for (int d = 0; d < ndim; ++d)
                        cnt *= side;
                    for (int64_t q = 0; q < cnt; ++q) {
                        int64_t rem = q, lin = 0;
                        for (int d = ndim - 1; d >= 0; --d) {
                            x[d] = R - h + rem % side; /* window coordinate */
                            rem /= side;
                        }
                        for (int d = 0; d < ndim; ++d)
                            lin = lin * L + x[d];
                        if (outside[lin]) {
                            v[lin] = 0.0;
                            continue;
                        }
                        double acc = 0.0;
                        for (int64_t t = 0; t < nterm; ++t) {
                            int64_t rt = t, li = 0;
                            for (int d = ndim - 1; d >= 0; --d) {
                                y[d] = x[d] + rt % w - r;
                                rt /= w;
                            }
                            for (int d = 0; d < ndim; ++d)
                                li = li * L + y[d];
                            double prod = cg[t] * u[li];
                            acc = acc + prod;
                        }
                        v[lin] = acc;
                    }
                    /* copy the freshly computed cone back into u */
                    for (int64_t q = 0; q < cnt; ++q) {
                        int64_t rem = q, lin = 0;
                        for (int d = ndim - 1; d >= 0; --d) {
                            x[d] = R - h + rem % side;
                            rem /= side;
                        }
                        for (int d = 0; d < ndim; ++d)
                            lin = lin * L + x[d];
                        u[lin] = v[lin];
                    }
                }
                int64_t centre = 0;
                for (int d = 0; d < ndim; ++d)
                    centre = centre * L + R;
                vals[p] = u[centre];
            }
        }
        free(u);
        free(v);
        free(outside);
    }
    return status;
}

/* Threads the oracle will use (1 when built without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
