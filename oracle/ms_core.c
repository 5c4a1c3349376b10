/*
 * FP64 reference loops for Gaussian mean-shift clustering.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle the CUDA library is checked
 * against; it shares no code with the library and the library never calls it.
 * Every loop is the plain definition, in float64, one seed at a time
 * (OpenMP only distributes independent seeds over host cores).
 *
 * Paper: "GPU-accelerated Faster Mean Shift with euclidean distance metrics"
 * (arXiv 2112.13891).  Notation follows Sec. II-A:
 *   X = {x_1..x_n} in R^d, bandwidth h, profile k applied to ||x - x_i||^2/h^2.
 * The profile is the Gaussian exp(-u/2) (the paper's Eq. 3 is garbled; the
 * Gaussian is the reading used throughout), whose shadow kernel g is again
 * Gaussian, so the mean of Eq. 6 is the Gaussian-weighted mean
 *   m(y) = sum_i w_i x_i / sum_i w_i,  w_i = exp(-||y - x_i||^2 / (2 h^2)),
 * taken over ALL points (Sec. II-B, Alg. 2: no window search).
 *
 * The flat (uniform) kernel of Eq. 12-15 is the alternative profile
 * (kernel = 1): g = 1 where ||x - x_i||^2 <= h^2, else 0, so the update is the
 * plain mean of the window S_h(y) = {x_i : ||x_i - y|| <= h} (Eq. 13, 15) and
 * the density is the window's count.  An empty window leaves y undefined
 * (NaN), which the callers treat as a failed seed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Squared Euclidean distance, Eq. 2 squared, with exact differences. */
static double sqdist(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = a[k] - b[k];
        s += t * t;
    }
    return s;
}

/*
 * Kernel density estimate of Eq. 1 without its constant 1/(n h^d):
 *   out[i] = sum_j exp(-||Y_i - x_j||^2 / (2 h^2)).
 */
void orc_kde(const double* X, int64_t n, int d, const double* Y, int64_t m, double h,
             double* out) {
    const double inv2h2 = 1.0 / (2.0 * h * h);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += exp(-sqdist(Y + i * d, X + j * d, d) * inv2h2);
        out[i] = s;
    }
}

/* Flat-kernel density: out[i] = |S_h(Y_i)| = #{j : ||Y_i - x_j||^2 <= h^2} (Eq. 12-13). */
void orc_kde_flat(const double* X, int64_t n, int d, const double* Y, int64_t m, double h,
                  double* out) {
    const double h2 = h * h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) c += sqdist(Y + i * d, X + j * d, d) <= h2;
        out[i] = (double)c;
    }
}

/*
 * One Gaussian mean-shift update y <- m(y) for one point y (Eq. 6 / Eq. 9-10
 * with the Gaussian weight, over all n points).  The weights are taken
 * relative to the nearest point, exp(-(D_j - D_min)/(2h^2)); the factor
 * exp(-D_min/(2h^2)) cancels in the ratio, so this is the same mean in real
 * arithmetic and cannot underflow to 0/0.  D is scratch of length n.
 */
static void ms_update_one(const double* X, int64_t n, int d, double inv2h2, const double* y,
                          double* ynew, double* D) {
    double dmin = INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        D[j] = sqdist(y, X + j * d, d);
        if (D[j] < dmin) dmin = D[j];
    }
    double W = 0.0;
    for (int k = 0; k < d; ++k) ynew[k] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double w = exp(-(D[j] - dmin) * inv2h2);
        W += w;
        for (int k = 0; k < d; ++k) ynew[k] += w * X[j * d + k];
    }
    for (int k = 0; k < d; ++k) ynew[k] /= W;
}

/*
 * One flat-kernel update (Eq. 14-15): the mean of the points within distance
 * h of y (inclusive); NaN when the window is empty.
 */
static void ms_update_one_flat(const double* X, int64_t n, int d, double h2, const double* y,
                               double* ynew) {
    int64_t m = 0;
    for (int k = 0; k < d; ++k) ynew[k] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (sqdist(y, X + j * d, d) <= h2) {
            ++m;
            for (int k = 0; k < d; ++k) ynew[k] += X[j * d + k];
        }
    }
    for (int k = 0; k < d; ++k) ynew[k] = m > 0 ? ynew[k] / (double)m : NAN;
}

/* One update for each of m points: Ynew_i = m(Y_i); kernel 0 Gaussian, 1 flat. */
void orc_step_k(const double* X, int64_t n, int d, double h, const double* Y, int64_t m,
                double* Ynew, int kernel) {
    const double inv2h2 = 1.0 / (2.0 * h * h);
#pragma omp parallel
    {
        double* D = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; ++i) {
            if (kernel == 1) ms_update_one_flat(X, n, d, h * h, Y + i * d, Ynew + i * d);
            else ms_update_one(X, n, d, inv2h2, Y + i * d, Ynew + i * d, D);
        }
        free(D);
    }
}

void orc_step(const double* X, int64_t n, int d, double h, const double* Y, int64_t m,
              double* Ynew) {
    orc_step_k(X, n, d, h, Y, m, Ynew, 0);
}

/*
 * Independent trajectories (the iteration loop of Alg. 1 and Alg. 2): for each
 * start point Y_i, repeat y <- m(y) until ||m(y) - y|| <= tol or max_iter
 * updates were made.  On return Y_i holds the last iterate, iters[i] the
 * number of updates made and conv_iter[i] the update index t (1-based) at
 * which the test first held, -1 if it never held, -2 if an update was
 * undefined (flat kernel, empty window; Y_i keeps the last defined iterate).
 */
/*
 * Same, with sphere != 0 for the cosine metric: X and the start points lie on
 * the unit sphere and every update is projected back onto it,
 * y <- m(y) / ||m(y)||, so the step tested against tol is the projected one.
 */
void orc_trajectories_m(const double* X, int64_t n, int d, double h, double tol, int max_iter,
                        double* Y, int64_t m, int32_t* conv_iter, int32_t* iters, int kernel,
                        int sphere);

void orc_trajectories_k(const double* X, int64_t n, int d, double h, double tol, int max_iter,
                        double* Y, int64_t m, int32_t* conv_iter, int32_t* iters, int kernel) {
    orc_trajectories_m(X, n, d, h, tol, max_iter, Y, m, conv_iter, iters, kernel, 0);
}

void orc_trajectories_m(const double* X, int64_t n, int d, double h, double tol, int max_iter,
                        double* Y, int64_t m, int32_t* conv_iter, int32_t* iters, int kernel,
                        int sphere) {
    const double inv2h2 = 1.0 / (2.0 * h * h);
#pragma omp parallel
    {
        double* D = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double ynew[64];
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; ++i) {
            double* y = Y + i * d;
            conv_iter[i] = -1;
            iters[i] = 0;
            for (int t = 1; t <= max_iter; ++t) {
                if (kernel == 1) ms_update_one_flat(X, n, d, h * h, y, ynew);
                else ms_update_one(X, n, d, inv2h2, y, ynew, D);
                if (ynew[0] != ynew[0]) {   /* empty window: the seed fails (-2) */
                    iters[i] = t;
                    conv_iter[i] = -2;
                    break;
                }
                if (sphere) {
                    double nn = 0.0;
                    for (int k = 0; k < d; ++k) nn += ynew[k] * ynew[k];
                    nn = sqrt(nn);
                    if (!(nn > 0.0)) {     /* the mean is the origin: undefined direction */
                        iters[i] = t;
                        conv_iter[i] = -2;
                        break;
                    }
                    for (int k = 0; k < d; ++k) ynew[k] /= nn;
                }
                double step2 = 0.0;
                for (int k = 0; k < d; ++k) {
                    double e = ynew[k] - y[k];
                    step2 += e * e;
                    y[k] = ynew[k];
                }
                iters[i] = t;
                if (sqrt(step2) <= tol) {
                    conv_iter[i] = t;
                    break;
                }
            }
        }
        free(D);
    }
}

void orc_trajectories(const double* X, int64_t n, int d, double h, double tol, int max_iter,
                      double* Y, int64_t m, int32_t* conv_iter, int32_t* iters) {
    orc_trajectories_k(X, n, d, h, tol, max_iter, Y, m, conv_iter, iters, 0);
}

/*
 * Nearest-mode labels (the labelling of Alg. 2): label_j = argmin_k ||x_j - mode_k||,
 * ties to the lowest k; margin_j = (second-nearest distance) - (nearest
 * distance), +inf when there is a single mode.
 */
void orc_label(const double* X, int64_t n, int d, const double* modes, int64_t M,
               int32_t* labels, double* margins) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        double best = INFINITY, second = INFINITY;
        int32_t arg = -1;
        for (int64_t k = 0; k < M; ++k) {
            double dist = sqrt(sqdist(X + j * d, modes + k * d, d));
            if (dist < best) {
                second = best;
                best = dist;
                arg = (int32_t)k;
            } else if (dist < second) {
                second = dist;
            }
        }
        labels[j] = arg;
        margins[j] = second - best;
    }
}
