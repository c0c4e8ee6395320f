/*
 * kb_oracle.c -- plain, slow FP64 CPU oracle for the shift-and-stack likelihood
 * search of Whidden et al., "Fast algorithms for slow moving asteroids"
 * (arXiv:1901.02492).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; it is written directly from
 * the definitions in the paper so that a reader can check it by eye:
 *
 *   weights            Sec. 2.1.5: inverse variance 1/sigma^2, zero for masked pixels
 *   psi / phi images   Sec. 2.1.5: Psi(y) = sum_i n(x_i) T(x_i - y) / sigma_i^2,
 *                                  Phi(y) = sum_i T(x_i - y)^2 / sigma_i^2
 *                      (inverse-variance weighted cross-correlation with the PSF)
 *   trajectory pixels  Sec. 2.1.5 / 2.2: y_i = y_0 + v t_i on the pixel grid
 *   coadd              Sec. 2.1.5: Psi = sum_i Psi_i(y_i), Phi = sum_i Phi_i(y_i)
 *   scores             Sec. 2.1.5: alpha_ML = Psi / Phi, nu = Psi / sqrt(Phi)
 *   search             Sec. 2.2: evaluate nu for every start pixel and velocity
 *   light-curve filter Sec. 3.3: reject observations far from the best-fit flux
 *                      of the others, recompute the likelihood (reading below)
 *   postage stamps     Sec. 3.3: mean / median coadd of science-image stamps along
 *                      a trajectory, and the stamp's central moments
 *   de-duplication     Sec. 3.3: DBSCAN over (x0, y0, vx, vy), the highest-likelihood
 *                      trajectory of each group kept (reading below)
 *   likelihood bound   Sec. 5.3 (searching low-likelihood trajectories less): an upper
 *                      bound on nu over a span of start pixels (derivation below)
 *
 * Readings of points the paper leaves open:
 *   - a pixel is masked when its mask byte is non-zero, when n or sigma^2 is not
 *     finite, when sigma^2 <= 0, or when n exceeds the optional bright-pixel
 *     limit (Sec. 5.2); masked pixels get weight 0 and contribute exactly 0;
 *   - PSF taps that fall outside the image contribute 0 (no renormalisation);
 *   - trajectory pixel = start pixel + floor(v t + 1/2), evaluated in fixed
 *     point: v_q = llround(v * 2^16), t_q = llround((t - t_min) * 2^20),
 *     offset = floor((v_q * t_q + 2^35) / 2^36) in 64-bit integers;
 *   - epochs whose trajectory pixel lies outside the image add nothing and are
 *     not counted in nobs; a trajectory with Phi == 0 is not a valid result;
 *   - per start pixel the k best valid trajectories are kept, ordered by
 *     (nu descending, velocity index ascending), optionally only nu >= nu_min.
 * The oracle sums epochs in time order (ties by epoch index).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int kbo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void kbo_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Sec. 2.1.5: masked pixels carry zero inverse variance, so they add nothing. */
static int pixel_masked(float n, float var, const uint8_t *mask, size_t i, double bright_max) {
    if (mask && mask[i]) return 1;
    if (!isfinite(n) || !isfinite(var)) return 1;
    if (var <= 0.0f) return 1;
    if ((double)n > bright_max) return 1;
    return 0;
}

/* Weights of one epoch: w = 1/sigma^2 and nw = n/sigma^2, both 0 where masked. */
void kbo_weights(const float *sci, const float *var, const uint8_t *mask, size_t npix,
                 double bright_max, double *w, double *nw) {
    for (size_t i = 0; i < npix; ++i) {
        if (pixel_masked(sci[i], var[i], mask, i, bright_max)) {
            w[i] = 0.0;
            nw[i] = 0.0;
        } else {
            w[i] = 1.0 / (double)var[i];
            nw[i] = (double)sci[i] * w[i];
        }
    }
}

/*
 * Sec. 2.1.5, psi and phi images of one epoch by direct 2-D cross-correlation
 * over the full K x K PSF (r = K/2):
 *   psi(y, x) = sum_{dy,dx in [-r,r]} nw(y+dy, x+dx) * T(dy, dx)
 *   phi(y, x) = sum_{dy,dx in [-r,r]}  w(y+dy, x+dx) * T(dy, dx)^2
 * T is stored row-major, T(dy, dx) = psf[(dy + r) * K + (dx + r)].
 */
static void psi_phi_epoch(const double *w, const double *nw, const float *psf, int H, int W, int K,
                          double *psi, double *phi) {
    const int r = K / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double sp = 0.0, sf = 0.0;
            for (int dy = -r; dy <= r; ++dy) {
                int yy = y + dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -r; dx <= r; ++dx) {
                    int xx = x + dx;
                    if (xx < 0 || xx >= W) continue;
                    double t = (double)psf[(dy + r) * K + (dx + r)];
                    size_t i = (size_t)yy * W + xx;
                    sp += nw[i] * t;
                    sf += w[i] * (t * t);
                }
            }
            psi[(size_t)y * W + x] = sp;
            phi[(size_t)y * W + x] = sf;
        }
    }
}

/* All epochs: inputs [N][H][W] (mask may be NULL), psf [N][K][K], outputs [N][H][W]. */
void kbo_psi_phi(const float *sci, const float *var, const uint8_t *mask, const float *psf, int N, int H,
                 int W, int K, double bright_max, double *psi, double *phi) {
    size_t npix = (size_t)H * W;
    double *w = (double *)malloc(npix * sizeof(double));
    double *nw = (double *)malloc(npix * sizeof(double));
    for (int e = 0; e < N; ++e) {
        kbo_weights(sci + e * npix, var + e * npix, mask ? mask + e * npix : NULL, npix, bright_max, w, nw);
        psi_phi_epoch(w, nw, psf + (size_t)e * K * K, H, W, K, psi + e * npix, phi + e * npix);
    }
    free(w);
    free(nw);
}

/* The same definition evaluated at one pixel (x, y) of one epoch. */
void kbo_psi_phi_at(const float *sci, const float *var, const uint8_t *mask, const float *psf, int H, int W,
                    int K, double bright_max, int x, int y, double *psi, double *phi) {
    const int r = K / 2;
    double sp = 0.0, sf = 0.0;
    for (int dy = -r; dy <= r; ++dy) {
        int yy = y + dy;
        if (yy < 0 || yy >= H) continue;
        for (int dx = -r; dx <= r; ++dx) {
            int xx = x + dx;
            if (xx < 0 || xx >= W) continue;
            size_t i = (size_t)yy * W + xx;
            if (pixel_masked(sci[i], var[i], mask, i, bright_max)) continue;
            double t = (double)psf[(dy + r) * K + (dx + r)];
            double w = 1.0 / (double)var[i];
            sp += ((double)sci[i] * w) * t;
            sf += w * (t * t);
        }
    }
    *psi = sp;
    *phi = sf;
}

/* ---- trajectory pixels (fixed point) ------------------------------------ */

int64_t kbo_quant_velocity(double v) { return llround(v * 65536.0); }        /* 2^16 per px/day */
int64_t kbo_quant_time(double dt) { return llround(dt * 1048576.0); }        /* 2^20 per day */

/* floor(a / 2^36) for any signed 64-bit a, written without relying on >> of negatives */
static int64_t floor_div_2p36(int64_t a) {
    const int64_t d = (int64_t)1 << 36;
    if (a >= 0) return a / d;
    return -((-a + d - 1) / d);
}

/* Pixel offset of one velocity component at one time: floor(v t + 1/2) in fixed point. */
int64_t kbo_offset(int64_t vq, int64_t tq) {
    return floor_div_2p36(vq * tq + ((int64_t)1 << 35));
}

/*
 * Offsets for every velocity and epoch, dx/dy laid out [V][N] in the caller's
 * epoch order; times are relative to the earliest epoch (the search starts at
 * every pixel of the earliest image, Sec. 3.2).
 */
void kbo_offsets(const double *times, int N, const double *vx, const double *vy, int V, int32_t *dx,
                 int32_t *dy) {
    double tmin = times[0];
    for (int e = 1; e < N; ++e)
        if (times[e] < tmin) tmin = times[e];
    for (int v = 0; v < V; ++v) {
        int64_t qx = kbo_quant_velocity(vx[v]), qy = kbo_quant_velocity(vy[v]);
        for (int e = 0; e < N; ++e) {
            int64_t tq = kbo_quant_time(times[e] - tmin);
            dx[(size_t)v * N + e] = (int32_t)kbo_offset(qx, tq);
            dy[(size_t)v * N + e] = (int32_t)kbo_offset(qy, tq);
        }
    }
}

/* Epoch indices sorted by (time, index): the order in which the oracle sums. */
static void time_order(const double *times, int N, int *order) {
    for (int e = 0; e < N; ++e) order[e] = e;
    for (int i = 1; i < N; ++i) { /* insertion sort, stable */
        int c = order[i], j = i - 1;
        while (j >= 0 && times[order[j]] > times[c]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = c;
    }
}

/* ---- coadd sums and scores ---------------------------------------------- */

typedef struct {
    int32_t x0, y0, vidx, nobs;
    double psi, phi, nu, alpha;
} kbo_rec;

/*
 * Sec. 2.1.5 coadd of one trajectory: Psi = sum_t psi_t(y_t), Phi = sum_t phi_t(y_t)
 * over the epochs whose pixel is inside the image, in time order.
 */
static void trajectory_sums(const double *psi, const double *phi, int N, int H, int W, const int32_t *dx,
                            const int32_t *dy, const int *order, int x0, int y0, double *P, double *F,
                            int *nobs) {
    size_t npix = (size_t)H * W;
    double sp = 0.0, sf = 0.0;
    int n = 0;
    for (int j = 0; j < N; ++j) {
        int e = order[j];
        int x = x0 + dx[e], y = y0 + dy[e];
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        size_t i = (size_t)e * npix + (size_t)y * W + x;
        sp += psi[i];
        sf += phi[i];
        ++n;
    }
    *P = sp;
    *F = sf;
    *nobs = n;
}

/* Sums for every start pixel at one velocity: Psi, Phi, nobs maps [H][W]. */
void kbo_sums_one_velocity(const double *psi, const double *phi, const double *times, int N, int H, int W,
                           const int32_t *dx_v, const int32_t *dy_v, double *Pmap, double *Fmap,
                           int32_t *nobs) {
    int order[4096];
    time_order(times, N, order);
#pragma omp parallel for schedule(static)
    for (int y0 = 0; y0 < H; ++y0)
        for (int x0 = 0; x0 < W; ++x0) {
            int n;
            size_t i = (size_t)y0 * W + x0;
            trajectory_sums(psi, phi, N, H, W, dx_v, dy_v, order, x0, y0, &Pmap[i], &Fmap[i], &n);
            nobs[i] = n;
        }
}

/* (nu desc, vidx asc): does a rank before b?  Empty slots (vidx < 0) rank last. */
static int ranks_before(double a_nu, int a_v, const kbo_rec *b) {
    if (b->vidx < 0) return 1;
    if (a_nu != b->nu) return a_nu > b->nu;
    return a_v < b->vidx;
}

static void empty_list(int x0, int y0, int k, kbo_rec *out) {
    for (int i = 0; i < k; ++i) {
        out[i].x0 = x0;
        out[i].y0 = y0;
        out[i].vidx = -1;
        out[i].nobs = 0;
        out[i].psi = 0.0;
        out[i].phi = 0.0;
        out[i].nu = -INFINITY;
        out[i].alpha = 0.0;
    }
}

/* Scores of Sec. 2.1.5 for one trajectory and insertion into the sorted list when
 * it is valid (Phi > 0, nu >= nu_min) and ranks among the k best. */
static void offer(double P, double F, int nobs, int v, int k, double nu_min, kbo_rec *out) {
    if (!(F > 0.0)) return;
    double nu = P / sqrt(F);
    double alpha = P / F;
    if (!(nu >= nu_min)) return;
    int pos = k;
    for (int i = 0; i < k; ++i)
        if (ranks_before(nu, v, &out[i])) {
            pos = i;
            break;
        }
    if (pos == k) return;
    for (int i = k - 1; i > pos; --i) out[i] = out[i - 1];
    out[pos].vidx = v;
    out[pos].nobs = nobs;
    out[pos].psi = P;
    out[pos].phi = F;
    out[pos].nu = nu;
    out[pos].alpha = alpha;
}

/*
 * Sec. 2.2 exhaustive search at one start pixel: every velocity, scores of Sec.
 * 2.1.5, keep the k best valid trajectories (Phi > 0 and nu >= nu_min).
 */
static void search_pixel(const double *psi, const double *phi, int N, int H, int W, const int32_t *dx,
                         const int32_t *dy, int V, const int *order, int k, double nu_min, int x0, int y0,
                         kbo_rec *out) {
    empty_list(x0, y0, k, out);
    for (int v = 0; v < V; ++v) {
        double P, F;
        int nobs;
        trajectory_sums(psi, phi, N, H, W, dx + (size_t)v * N, dy + (size_t)v * N, order, x0, y0, &P, &F,
                        &nobs);
        offer(P, F, nobs, v, k, nu_min, out);
    }
}

/* Search over a list of start pixels (px[i], py[i]); out is [npix][k]. */
void kbo_search_pixels(const double *psi, const double *phi, const double *times, int N, int H, int W,
                       const int32_t *dx, const int32_t *dy, int V, int k, double nu_min, const int32_t *px,
                       const int32_t *py, int64_t npix, kbo_rec *out) {
    int order[4096];
    time_order(times, N, order);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < npix; ++i)
        search_pixel(psi, phi, N, H, W, dx, dy, V, order, k, nu_min, px[i], py[i], out + (size_t)i * k);
}

/* Search over the rectangle [x_lo, x_hi) x [y_lo, y_hi); out is [rows][cols][k]. */
void kbo_search_region(const double *psi, const double *phi, const double *times, int N, int H, int W,
                       const int32_t *dx, const int32_t *dy, int V, int k, double nu_min, int x_lo, int x_hi,
                       int y_lo, int y_hi, kbo_rec *out) {
    int order[4096];
    time_order(times, N, order);
    int cols = x_hi - x_lo;
    int64_t n = (int64_t)(y_hi - y_lo) * cols;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int x0 = x_lo + (int)(i % cols), y0 = y_lo + (int)(i / cols);
        search_pixel(psi, phi, N, H, W, dx, dy, V, order, k, nu_min, x0, y0, out + (size_t)i * k);
    }
}

/*
 * One trajectory from the raw inputs, without precomputed planes: psi/phi at each
 * trajectory pixel by the point definition, coadded in time order.  Used to check
 * sampled outputs of full-size searches.
 */
void kbo_trajectory_from_images(const float *sci, const float *var, const uint8_t *mask, const float *psf,
                                const double *times, int N, int H, int W, int K, double bright_max,
                                const int32_t *dx_v, const int32_t *dy_v, int x0, int y0, double *P,
                                double *F, int32_t *nobs) {
    int order[4096];
    time_order(times, N, order);
    size_t npix = (size_t)H * W;
    double sp = 0.0, sf = 0.0;
    int n = 0;
    for (int j = 0; j < N; ++j) {
        int e = order[j];
        int x = x0 + dx_v[e], y = y0 + dy_v[e];
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        double a, b;
        kbo_psi_phi_at(sci + e * npix, var + e * npix, mask ? mask + e * npix : NULL,
                       psf + (size_t)e * K * K, H, W, K, bright_max, x, y, &a, &b);
        sp += a;
        sf += b;
        ++n;
    }
    *P = sp;
    *F = sf;
    *nobs = n;
}

/*
 * The Sec. 2.2 search at listed start pixels straight from the raw images: every
 * trajectory's psi/phi values come from the point definition, so no planes are
 * held.  Used to check sampled pixels of full-size searches.
 */
void kbo_search_pixels_from_images(const float *sci, const float *var, const uint8_t *mask, const float *psf,
                                   const double *times, int N, int H, int W, int K, double bright_max,
                                   const int32_t *dx, const int32_t *dy, int V, int k, double nu_min,
                                   const int32_t *px, const int32_t *py, int64_t npix, kbo_rec *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < npix; ++i) {
        kbo_rec *o = out + (size_t)i * k;
        empty_list(px[i], py[i], k, o);
        for (int v = 0; v < V; ++v) {
            double P, F;
            int32_t nobs;
            kbo_trajectory_from_images(sci, var, mask, psf, times, N, H, W, K, bright_max, dx + (size_t)v * N,
                                       dy + (size_t)v * N, px[i], py[i], &P, &F, &nobs);
            offer(P, F, nobs, v, k, nu_min, o);
        }
    }
}

/* ---- light-curve outlier filter (Sec. 3.3) ------------------------------ */

/*
 * Sec. 3.3: reject the observations of a kept trajectory that lie more than
 * nsigma standard deviations from the best-fit (Kalman) flux at that
 * observation, then recompute the likelihood from the remaining ones.
 *
 * Reading of the unspecified filter: the object's flux is constant (the model
 * of Sec. 2.1), so the Kalman estimate from a set of observations is their
 * inverse-variance weighted mean.  Epoch e's own flux estimate is
 * alpha_e = psi_e / phi_e with variance 1 / phi_e (Sec. 2.1.5 for one image);
 * the estimate from all the other epochs is alpha_rest = (Psi - psi_e) /
 * (Phi - phi_e) with variance 1 / (Phi - phi_e).  Epoch e is rejected when
 *     |alpha_e - alpha_rest| > nsigma * sqrt(1 / phi_e + 1 / (Phi - phi_e)).
 * All decisions use the unfiltered sums (one pass); epochs with phi_e == 0 or
 * with no information in the others (Phi - phi_e == 0) are never rejected.
 * Only epochs whose trajectory pixel is inside the image take part.
 *
 * Outputs: the sums over the kept epochs (time order), the number of kept and
 * of rejected epochs, and rejected[e] = 1 for each rejected epoch e.
 */
void kbo_filter_lightcurve(const double *psi, const double *phi, const double *times, int N, int H, int W,
                           const int32_t *dx, const int32_t *dy, int x0, int y0, double nsigma, double *P_out,
                           double *F_out, int32_t *nkept, int32_t *nrej, uint8_t *rejected) {
    size_t npix = (size_t)H * W;
    int order[4096];
    time_order(times, N, order);
    double P = 0.0, F = 0.0;
    for (int e = 0; e < N; ++e) rejected[e] = 0;
    for (int j = 0; j < N; ++j) { /* the unfiltered coadd */
        int e = order[j], x = x0 + dx[e], y = y0 + dy[e];
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        size_t i = (size_t)e * npix + (size_t)y * W + x;
        P += psi[i];
        F += phi[i];
    }
    double Pk = 0.0, Fk = 0.0;
    int kept = 0, rej = 0;
    for (int j = 0; j < N; ++j) {
        int e = order[j], x = x0 + dx[e], y = y0 + dy[e];
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        size_t i = (size_t)e * npix + (size_t)y * W + x;
        double pe = psi[i], fe = phi[i], rest = F - fe;
        int out = 0;
        if (fe > 0.0 && rest > 0.0) {
            double a_e = pe / fe, a_rest = (P - pe) / rest;
            double sigma = sqrt(1.0 / fe + 1.0 / rest);
            out = fabs(a_e - a_rest) > nsigma * sigma;
        }
        if (out) {
            rejected[e] = 1;
            ++rej;
        } else {
            Pk += pe;
            Fk += fe;
            ++kept;
        }
    }
    *P_out = Pk;
    *F_out = Fk;
    *nkept = kept;
    *nrej = rej;
}

/* ---- coadded postage stamps and central moments (Sec. 3.3) -------------- */

static int cmp_float(const void *a, const void *b) {
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/*
 * Sec. 3.3 postage stamp of one trajectory: for each stamp pixel (sx, sy) in
 * [-r, r]^2, the science values n_e(x0 + dx_e + sx, y0 + dy_e + sy) of the epochs
 * whose pixel is inside the image, finite and not masked, combined as their mean
 * (mode 0) or median (mode 1: the middle value, the mean of the two middle ones
 * for an even count); 0 where no epoch contributes.  Stamp layout [2r+1][2r+1],
 * row sy + r, column sx + r.
 */
void kbo_stamp(const float *sci, const uint8_t *mask, int N, int H, int W, const int32_t *dx, const int32_t *dy,
               int x0, int y0, int r, int mode, float *stamp) {
    int S = 2 * r + 1;
    float vals[4096];
    size_t npix = (size_t)H * W;
    for (int sy = -r; sy <= r; ++sy)
        for (int sx = -r; sx <= r; ++sx) {
            int n = 0;
            double sum = 0.0;
            for (int e = 0; e < N; ++e) {
                int x = x0 + dx[e] + sx, y = y0 + dy[e] + sy;
                if (x < 0 || x >= W || y < 0 || y >= H) continue;
                size_t i = (size_t)e * npix + (size_t)y * W + x;
                float v = sci[i];
                if (!isfinite(v) || (mask && mask[i])) continue;
                vals[n++] = v;
                sum += v;
            }
            float out = 0.0f;
            if (n > 0) {
                if (mode == 0) {
                    out = (float)(sum / n);
                } else {
                    qsort(vals, (size_t)n, sizeof(float), cmp_float);
                    out = (n & 1) ? vals[n / 2] : (float)(0.5 * ((double)vals[n / 2 - 1] + (double)vals[n / 2]));
                }
            }
            stamp[(size_t)(sy + r) * S + (sx + r)] = out;
        }
}

/*
 * Central moments of a stamp over a central aperture, pixel values as weights,
 * coordinates relative to the stamp centre.  The pixels taken are those with
 * x^2 + y^2 <= aperture^2 (every pixel of the stamp when aperture <= 0):
 * m00 = sum I, centroid (mx, my) = sum (x, y) I / m00, and mu20, mu02, mu11 =
 * sum (x - mx)^2 I, (y - my)^2 I, (x - mx)(y - my) I over m00.  All zero when
 * m00 == 0.
 *
 * Reading of Sec. 3.3 (the paper takes "the central moments of the images" of
 * the coadded stamps and compares them with those of a Gaussian centred in the
 * stamp).  Over the whole stamp, the moments of a faint source are dominated by
 * the sky noise of the surrounding pixels: the noise's contribution to the
 * second moments grows with the fourth power of the stamp radius.  An aperture
 * of about two PSF widths keeps the source's light and little noise, so a
 * source's moments come out near those of its PSF and a stamp of pure noise
 * (whose m00 is as likely negative as positive) rarely does.
 */
void kbo_moments(const float *stamp, int r, double aperture, double *m00, double *mx, double *my, double *mu20,
                 double *mu02, double *mu11) {
    int S = 2 * r + 1;
    double a2 = aperture * aperture;
    double s = 0.0, sx = 0.0, sy = 0.0;
    for (int j = 0; j < S; ++j)
        for (int i = 0; i < S; ++i) {
            double x = i - r, y = j - r;
            if (aperture > 0.0 && x * x + y * y > a2) continue;
            double v = stamp[(size_t)j * S + i];
            s += v;
            sx += x * v;
            sy += y * v;
        }
    *m00 = s;
    *mx = *my = *mu20 = *mu02 = *mu11 = 0.0;
    if (s == 0.0) return;
    double cx = sx / s, cy = sy / s, a = 0.0, b = 0.0, c = 0.0;
    for (int j = 0; j < S; ++j)
        for (int i = 0; i < S; ++i) {
            double x0 = i - r, y0 = j - r;
            if (aperture > 0.0 && x0 * x0 + y0 * y0 > a2) continue;
            double v = stamp[(size_t)j * S + i], x = x0 - cx, y = y0 - cy;
            a += x * x * v;
            b += y * y * v;
            c += x * y * v;
        }
    *mx = cx;
    *my = cy;
    *mu20 = a / s;
    *mu02 = b / s;
    *mu11 = c / s;
}

/* ---- Sec. 3.3: DBSCAN de-duplication of candidate trajectories -------------
 *
 * Reading.  The paper groups similar trajectories with DBSCAN over the start
 * pixel and the velocity and keeps the highest-likelihood one of each group.
 * It gives no metric or parameters.  Here the distance between candidates i, j
 * is the Euclidean distance of (x0 w_pos, y0 w_pos, vx w_vel, vy w_vel),
 * evaluated in FP64 as
 *     d2 = ((ax*ax + ay*ay) + au*au) + av*av,
 *     ax = (double)(x0_i - x0_j) * w_pos, ay likewise,
 *     au = ((double)vx_i - (double)vx_j) * w_vel, av likewise,
 * and j is a neighbour of i when d2 <= eps*eps (i is its own neighbour).
 * DBSCAN's definitions then fix:
 *   - core point: at least min_samples neighbours;
 *   - clusters: the connected components of core points under the neighbour
 *     relation, each labelled by the lowest index among its core points;
 *   - border point (not core, with a core neighbour): DBSCAN lets it join any
 *     neighbouring cluster; here it joins the cluster of its nearest core
 *     neighbour (smallest d2, then lowest index), which makes the result unique;
 *   - noise point (neither): a group of its own, labelled by its own index.
 * Candidates with vidx < 0 (empty result slots) take no part: label -1.
 * Of each group the member with the largest nu (then lowest index) is kept.
 */
static double kbo_cluster_d2(const int32_t *x0, const int32_t *y0, const float *vx, const float *vy, double w_pos,
                             double w_vel, long i, long j) {
    double ax = (double)((int64_t)x0[i] - (int64_t)x0[j]) * w_pos;
    double ay = (double)((int64_t)y0[i] - (int64_t)y0[j]) * w_pos;
    double au = ((double)vx[i] - (double)vx[j]) * w_vel;
    double av = ((double)vy[i] - (double)vy[j]) * w_vel;
    return ((ax * ax + ay * ay) + au * au) + av * av;
}

void kbo_cluster(const int32_t *x0, const int32_t *y0, const float *vx, const float *vy, const double *nu,
                 const int32_t *vidx, long n, double w_pos, double w_vel, double eps, int min_samples,
                 int32_t *label, uint8_t *keep, uint8_t *core) {
    const double eps2 = eps * eps;
    /* core points: neighbour counts by brute force */
    for (long i = 0; i < n; ++i) {
        long cnt = 0;
        if (vidx[i] >= 0)
            for (long j = 0; j < n; ++j)
                if (vidx[j] >= 0 && kbo_cluster_d2(x0, y0, vx, vy, w_pos, w_vel, i, j) <= eps2) ++cnt;
        core[i] = vidx[i] >= 0 && cnt >= min_samples;
        label[i] = -1;
        keep[i] = 0;
    }
    /* clusters: breadth-first search over core points, started in index order,
       so each component is labelled by its lowest core index */
    long *queue = (long *)malloc((size_t)(n > 0 ? n : 1) * sizeof(long));
    for (long s = 0; s < n; ++s) {
        if (!core[s] || label[s] >= 0) continue;
        long head = 0, tail = 0;
        queue[tail++] = s;
        label[s] = (int32_t)s;
        while (head < tail) {
            long i = queue[head++];
            for (long j = 0; j < n; ++j)
                if (core[j] && label[j] < 0 && kbo_cluster_d2(x0, y0, vx, vy, w_pos, w_vel, i, j) <= eps2) {
                    label[j] = (int32_t)s;
                    queue[tail++] = j;
                }
        }
    }
    free(queue);
    /* border and noise points */
    for (long i = 0; i < n; ++i) {
        if (vidx[i] < 0 || core[i]) continue;
        long best = -1;
        double bd = 0.0;
        for (long j = 0; j < n; ++j) {
            if (!core[j]) continue;
            double d2 = kbo_cluster_d2(x0, y0, vx, vy, w_pos, w_vel, i, j);
            if (d2 <= eps2 && (best < 0 || d2 < bd)) {
                best = j;
                bd = d2;
            }
        }
        label[i] = best >= 0 ? label[best] : (int32_t)i;
    }
    /* the best member of each group */
    for (long i = 0; i < n; ++i) {
        if (label[i] < 0) continue;
        int best = 1;
        for (long j = 0; j < n && best; ++j)
            if (j != i && label[j] == label[i] && (nu[j] > nu[i] || (nu[j] == nu[i] && j < i))) best = 0;
        keep[i] = (uint8_t)best;
    }
}

/* ---- Sec. 5.3: an upper bound on nu over a span of start pixels ------------
 *
 * For one trajectory, over the epochs whose pixel is in the image, the
 * Cauchy-Schwarz inequality gives
 *     Psi^2 = (sum_t psi_t)^2 <= (sum_t psi_t^2 / phi_t) (sum_t phi_t)
 * (an epoch with phi_t = 0 has psi_t = 0: every weight of its PSF window is 0).
 * With Psi > 0 only the positive psi_t can raise it, so
 *     nu^2 = Psi^2 / Phi <= sum_t max(psi_t, 0)^2 / phi_t,
 * a sum of single-epoch SNRs squared, with equality when psi_t / phi_t is the
 * same for every epoch (a noiseless source).  kbo_snr2_span_max stores, per
 * epoch and row, the largest such term over the columns [x, x + span) that lie
 * in the image (0 if none), for x = -(span - 1) .. W - 1 at index
 * x + span - 1: r is [N][H][W + span - 1].  kbo_span_bound adds one r value
 * per epoch at the span's position shifted by the trajectory's offsets (epochs
 * whose row is outside add 0); it bounds nu^2 of every trajectory that starts
 * in the span [x0, x0 + span) of row y0 with those offsets and has Psi > 0.
 */
void kbo_snr2_span_max(const double *psi, const double *phi, int N, int H, int W, int span, double *r) {
    const int RW = W + span - 1;
    for (int t = 0; t < N; ++t)
        for (int y = 0; y < H; ++y)
            for (int xi = 0; xi < RW; ++xi) {
                const int x = xi - (span - 1);
                const int lo = x < 0 ? 0 : x, hi = x + span < W ? x + span : W;
                double m = 0.0;
                for (int xx = lo; xx < hi; ++xx) {
                    const size_t i = ((size_t)t * H + y) * W + xx;
                    if (phi[i] > 0.0 && psi[i] > 0.0) {
                        const double q = psi[i] * psi[i] / phi[i];
                        if (q > m) m = q;
                    }
                }
                r[((size_t)t * H + y) * RW + xi] = m;
            }
}

double kbo_span_bound(const double *r, int N, int H, int W, int span, const int32_t *dx, const int32_t *dy, int x0,
                      int y0) {
    const int RW = W + span - 1;
    double s = 0.0;
    for (int t = 0; t < N; ++t) {
        const int x = x0 + dx[t], y = y0 + dy[t];
        if (y < 0 || y >= H || x <= -span || x >= W) continue;
        s += r[((size_t)t * H + y) * RW + (x + span - 1)];
    }
    return s;
}
