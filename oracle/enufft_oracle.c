/*
 * enufft_oracle.c -- TEST INFRASTRUCTURE, not product code.
 *
 * A plain, slow, FP64 CPU statement of what the ENUFFT hot path computes, written from the
 * paper (arxiv 2606.21278) and used only by the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark.  It shares no code, header, table or helper with the CUDA
 * library: every quantity is evaluated here directly from its definition.
 *
 *   frame       App. A  (centroid, centroid-aligned frame R = I or edge-aligned frame R of
 *                        Eq. "rotation_matrix", centred coordinates u = R (x - x-bar), half-width H,
 *                        square B, shifted coordinates x' = u + H, masks D = B n {square, cell, circle})
 *   |D|         App. A/B (area of the active quadrature domain)
 *   type-1      App. B, Eq. "discrete_quadrature":  h_mn = 1/|D| sum_q w_q h_q e^{-i(k_m x'_q + k_n y'_q)},
 *               k_m = 2 pi m / L, L = 2H, evaluated by direct summation (the NUFFT of Sec. 2.1.2 is a
 *               fast evaluation of exactly this sum)
 *   EMS         Sec. 2.2, Eqs. "energy", "weighted_e", "sorted_energy", "n_eff", "s_delta", "c_score",
 *               "alpha_c", "f_cum", "k_elastic" (+ the footnote bounding all sums by J_max)
 *   gradient    derivative of the EMS-retained power with the selected set held fixed; it is the
 *               adjoint (type-2 sum) of the quadrature above
 *   weights     App. A Voronoi weights by raster sampling (Eqs. "voronoi_cell", "raster_grid",
 *               "nn_assignment", "raster_area", "area_partition", "voronoi_weights")
 *   diagnostics Sec. 3.2: the truncated series h_rec (Eq. "tri_series") over a set of modes at the
 *               samples, the relative reconstructed RMSE (Eq. "alps_relative_rmse") and the physical
 *               and spectral variances of Parseval's check (Eq. "spectral_variance")
 *
 * Readings where the paper is silent (documented with the build):
 *   - mode box m, n in [-P/2, P/2); EMS candidates are mode pairs +-(m,n) with |m|,|n| <= P/2-1,
 *     represented by the half-plane member (n > 0, or n == 0 and m > 0); DC excluded by default;
 *   - sort ties are broken by ascending pair index p = (n + P/2) P + (m + P/2);
 *   - J_max < 2 gives S_delta = 0; a gap with E_(j+1) = 0 contributes 0; total power 0 gives K* = 0;
 *     K* never exceeds the number of pairs with positive energy;
 *   - HEAD reading (default): N_eff and the denominator of theta use the top J_max = min(J*, K_max)
 *     energies; ALL reading: they use all J* energies;
 *   - hexagon (and any convex polygon) centroid = mean of its vertices, as for triangles.
 *
 * Parity status: every function here is pinned by closed-form or library checks in the tests
 * (regular-grid DFT, plane wave statistics, Gibbs step, polygon Fourier transform, DC term,
 * App. D limits of N_eff / S_delta, finite differences); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ----------------------------------------------------------------------------------------- */
/* App. A: local window                                                                        */
/* ----------------------------------------------------------------------------------------- */

typedef struct {
    double cx, cy;   /* centroid x-bar                                  */
    int edge;        /* 0: centroid-aligned frame (R = I); 1: edge-aligned frame           */
    double rc, rs;   /* edge frame: R = [[rc, rs], [-rs, rc]], (rc, rs) = e_max / |e_max| */
    double H;        /* half-width of the square spectral domain B      */
    double L;        /* period L = 2H                                   */
    double area;     /* |D|, area of the active quadrature domain       */
    int nv;          /* polygon vertex count                            */
    double ux[8], uy[8]; /* polygon vertices in the local frame u = R (x - x-bar)          */
    double orient;   /* +1 counter-clockwise, -1 clockwise              */
    int mask;        /* 0 cell (B n polygon), 1 square (B), 2 circle (B n disk of radius H) */
} oframe;

/* Area of a polygon by the shoelace formula (absolute value). */
static double shoelace(int n, const double *x, const double *y) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        s += x[i] * y[j] - x[j] * y[i];
    }
    return 0.5 * fabs(s);
}

/* Clip a polygon by the half-plane  s * coord(axis) <= H  (Sutherland-Hodgman, one edge). */
static int clip_halfplane(int n, const double *x, const double *y, int axis, double s, double H,
                          double *ox, double *oy) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        double ci = s * (axis == 0 ? x[i] : y[i]) - H;
        double cj = s * (axis == 0 ? x[j] : y[j]) - H;
        int in_i = ci <= 0.0, in_j = cj <= 0.0;
        if (in_i) { ox[m] = x[i]; oy[m] = y[i]; ++m; }
        if (in_i != in_j) {
            double t = ci / (ci - cj);
            ox[m] = x[i] + t * (x[j] - x[i]);
            oy[m] = y[i] + t * (y[j] - y[i]);
            ++m;
        }
    }
    return m;
}

/* Local coordinates u = R (x - x-bar) of a point (App. A): R = I in the centroid-aligned frame;
 * in the edge-aligned frame R = [[cos t, sin t], [-sin t, cos t]] (Eq. rotation_matrix). */
static void local_of(const oframe *f, double x, double y, double *ux, double *uy) {
    double dx = x - f->cx, dy = y - f->cy;
    if (!f->edge) {
        *ux = dx;
        *uy = dy;
    } else {
        *ux = f->rc * dx + f->rs * dy;
        *uy = -f->rs * dx + f->rc * dy;
    }
}

/* Frame of one cell (App. A): centroid, orientation (frame 0: centroid-aligned, R = I; frame 1:
 * edge-aligned, the longest edge e_i = v_(i+1) - v_i -- the first one on a tie -- made parallel to
 * +x), H = (eta/2) max extent in that frame, B = [-H, H]^2, and |D| for the chosen mask.
 * Returns 0, or -1 for a bad polygon or frame. */
static int frame_of(int nv, const double *v, double eta, int mask, int frame, oframe *f) {
    if (nv < 3 || nv > 6 || frame < 0 || frame > 1) return -1;
    memset(f, 0, sizeof(*f));
    f->nv = nv;
    f->mask = mask;
    for (int i = 0; i < nv; ++i) { f->cx += v[2 * i]; f->cy += v[2 * i + 1]; }
    f->cx /= nv;
    f->cy /= nv;
    f->rc = 1.0;
    if (frame == 1) {
        double best = -1.0, ex = 1.0, ey = 0.0;
        for (int i = 0; i < nv; ++i) {
            int k = (i + 1) % nv;
            double dx = v[2 * k] - v[2 * i], dy = v[2 * k + 1] - v[2 * i + 1];
            double len = sqrt(dx * dx + dy * dy);
            if (len > best) { best = len; ex = dx; ey = dy; }
        }
        if (!(best > 0.0)) return -1;
        f->edge = 1;
        f->rc = ex / best;   /* cos theta = e_x / |e_max| */
        f->rs = ey / best;   /* sin theta = e_y / |e_max| */
    }
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = 0; i < nv; ++i) {
        local_of(f, v[2 * i], v[2 * i + 1], &f->ux[i], &f->uy[i]);
        if (f->ux[i] < xmin) xmin = f->ux[i];
        if (f->ux[i] > xmax) xmax = f->ux[i];
        if (f->uy[i] < ymin) ymin = f->uy[i];
        if (f->uy[i] > ymax) ymax = f->uy[i];
    }
    double ext = (xmax - xmin) > (ymax - ymin) ? (xmax - xmin) : (ymax - ymin);
    f->H = 0.5 * eta * ext;
    f->L = 2.0 * f->H;
    double sa = 0.0;
    for (int i = 0; i < nv; ++i) {
        int j = (i + 1) % nv;
        sa += f->ux[i] * f->uy[j] - f->ux[j] * f->uy[i];
    }
    f->orient = sa >= 0.0 ? 1.0 : -1.0;
    if (mask == 1) {
        f->area = f->L * f->L;
    } else if (mask == 2) {
        f->area = ORACLE_PI * f->H * f->H;
    } else {
        /* D = B n cell: clip the polygon by the four sides of B, then shoelace */
        double ax[32], ay[32], bx[32], by[32];
        int n = nv;
        for (int i = 0; i < nv; ++i) { ax[i] = f->ux[i]; ay[i] = f->uy[i]; }
        n = clip_halfplane(n, ax, ay, 0, +1.0, f->H, bx, by);
        n = clip_halfplane(n, bx, by, 0, -1.0, f->H, ax, ay);
        n = clip_halfplane(n, ax, ay, 1, +1.0, f->H, bx, by);
        n = clip_halfplane(n, bx, by, 1, -1.0, f->H, ax, ay);
        f->area = n >= 3 ? shoelace(n, ax, ay) : 0.0;
    }
    return 0;
}

/* Window indicator of a sample (App. A masks, closed sets). */
static int in_window(const oframe *f, double x, double y) {
    double ux, uy;
    local_of(f, x, y, &ux, &uy);
    if (ux < -f->H || ux > f->H || uy < -f->H || uy > f->H) return 0; /* outside B */
    if (f->mask == 1) return 1;
    if (f->mask == 2) return ux * ux + uy * uy <= f->H * f->H;
    for (int i = 0; i < f->nv; ++i) {
        int j = (i + 1) % f->nv;
        double cr = (f->ux[j] - f->ux[i]) * (uy - f->uy[i]) - (f->uy[j] - f->uy[i]) * (ux - f->ux[i]);
        if (f->orient * cr < 0.0) return 0;
    }
    return 1;
}

/* Exported: frame constants of one cell: out = {cx, cy, H, L, |D|, cos t, sin t, u_x[0..5], u_y[0..5]}
 * (19 doubles; the local vertices beyond nv are 0). */
int oracle_frame(int nv, const double *verts, double eta, int mask, int frame, double *out) {
    oframe f;
    if (frame_of(nv, verts, eta, mask, frame, &f)) return -1;
    out[0] = f.cx; out[1] = f.cy; out[2] = f.H; out[3] = f.L; out[4] = f.area;
    out[5] = f.rc; out[6] = f.rs;
    for (int i = 0; i < 6; ++i) { out[7 + i] = f.ux[i]; out[13 + i] = f.uy[i]; }
    return 0;
}

/* Exported: window indicator for Q samples of one cell. */
int oracle_window(int nv, const double *verts, double eta, int mask, int frame, int64_t Q, const double *x,
                  const double *y, int32_t *win) {
    oframe f;
    if (frame_of(nv, verts, eta, mask, frame, &f)) return -1;
    for (int64_t q = 0; q < Q; ++q) win[q] = in_window(&f, x[q], y[q]);
    return 0;
}

/* ----------------------------------------------------------------------------------------- */
/* App. B, Eq. discrete_quadrature: direct FP64 type-1 sum                                     */
/* ----------------------------------------------------------------------------------------- */

/* One cell. coeffs[(n + P/2) * P + (m + P/2)] = (re, im), m, n in [-P/2, P/2). */
static int type1_cell(const oframe *f, int P, int64_t Q, const double *x, const double *y,
                      const double *h, const double *w, double *coeffs) {
    int half = P / 2;
    double *ex = (double *)malloc(sizeof(double) * 2 * P);
    double *ey = (double *)malloc(sizeof(double) * 2 * P);
    if (!ex || !ey) { free(ex); free(ey); return -2; }
    memset(coeffs, 0, sizeof(double) * 2 * (size_t)P * P);
    for (int64_t q = 0; q < Q; ++q) {
        if (!in_window(f, x[q], y[q])) continue;
        double c = w[q] * h[q] / f->area;             /* w_q h_q / |D| */
        double ux, uy;
        local_of(f, x[q], y[q], &ux, &uy);
        double xp = ux + f->H;                        /* x' = u_x + H  */
        double yp = uy + f->H;
        for (int i = 0; i < P; ++i) {
            double k = 2.0 * ORACLE_PI * (double)(i - half) / f->L;   /* k_m = 2 pi m / L */
            ex[2 * i] = cos(k * xp);
            ex[2 * i + 1] = -sin(k * xp);
            ey[2 * i] = cos(k * yp);
            ey[2 * i + 1] = -sin(k * yp);
        }
        for (int in = 0; in < P; ++in) {
            double byr = c * ey[2 * in], byi = c * ey[2 * in + 1];
            double *row = coeffs + 2 * (size_t)in * P;
            for (int im = 0; im < P; ++im) {
                double axr = ex[2 * im], axi = ex[2 * im + 1];
                row[2 * im] += axr * byr - axi * byi;       /* e^{-i k_m x'} e^{-i k_n y'} */
                row[2 * im + 1] += axr * byi + axi * byr;
            }
        }
    }
    free(ex);
    free(ey);
    return 0;
}

static int nthreads_used = 1;

/* Exported: batched type-1 over cells (CSR offsets), OpenMP over cells. */
int oracle_type1_batch(int64_t n_cells, const int64_t *offsets, const int32_t *nverts,
                       const double *verts /* n_cells * 12 */, const double *x, const double *y,
                       const double *h, const double *w, int P, double eta, int mask, int frame,
                       double *coeffs /* n_cells * P * P * 2 */, int nthreads) {
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    nthreads_used = nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
    for (int64_t j = 0; j < n_cells; ++j) {
        oframe f;
        if (frame_of(nverts[j], verts + 12 * j, eta, mask, frame, &f)) { err |= 1; continue; }
        int64_t o = offsets[j], Q = offsets[j + 1] - offsets[j];
        if (type1_cell(&f, P, Q, x + o, y + o, h + o, w + o, coeffs + 2 * (size_t)P * P * j)) err |= 2;
    }
    return err ? -1 : 0;
}

int oracle_threads_used(void) { return nthreads_used; }

/* ----------------------------------------------------------------------------------------- */
/* Adjoint of the quadrature (type-2 sum): v_q = Re sum_mu G_mu e^{+i k_mu . x'_q}             */
/* ----------------------------------------------------------------------------------------- */

static double type2_point(const oframe *f, int P, const double *G, double xq, double yq) {
    int half = P / 2;
    double ux, uy;
    local_of(f, xq, yq, &ux, &uy);
    double xp = ux + f->H, yp = uy + f->H;
    double acc = 0.0;
    for (int in = 0; in < P; ++in) {
        double kn = 2.0 * ORACLE_PI * (double)(in - half) / f->L;
        for (int im = 0; im < P; ++im) {
            double km = 2.0 * ORACLE_PI * (double)(im - half) / f->L;
            double ph = km * xp + kn * yp;
            const double *g = G + 2 * ((size_t)in * P + im);
            acc += g[0] * cos(ph) - g[1] * sin(ph);   /* Re(G e^{i ph}) */
        }
    }
    return acc;
}

/* Exported: gradient of a real loss L(h, w) that depends on the coefficients only, given
 * G = dL/dRe(h_mu) + i dL/dIm(h_mu) for every mode of every cell:
 *   dL/dh_q = win_q w_q v_q / |D|,  dL/dw_q = win_q h_q v_q / |D|,  v_q = Re sum_mu G_mu e^{+i k.x'_q}. */
int oracle_type1_backward_batch(int64_t n_cells, const int64_t *offsets, const int32_t *nverts,
                                const double *verts, const double *x, const double *y, const double *h,
                                const double *w, int P, double eta, int mask, int frame, const double *G,
                                double *grad_h, double *grad_w, int nthreads) {
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
    for (int64_t j = 0; j < n_cells; ++j) {
        oframe f;
        if (frame_of(nverts[j], verts + 12 * j, eta, mask, frame, &f)) { err |= 1; continue; }
        const double *Gj = G + 2 * (size_t)P * P * j;
        for (int64_t q = offsets[j]; q < offsets[j + 1]; ++q) {
            if (!in_window(&f, x[q], y[q])) {
                grad_h[q] = 0.0;
                grad_w[q] = 0.0;
                continue;
            }
            double v = type2_point(&f, P, Gj, x[q], y[q]);
            grad_h[q] = w[q] * v / f.area;
            grad_w[q] = h[q] * v / f.area;
        }
    }
    return err ? -1 : 0;
}

/* ----------------------------------------------------------------------------------------- */
/* App. A: Voronoi quadrature weights by raster sampling                                       */
/* ----------------------------------------------------------------------------------------- */

/* Exported, for binary32 samples.  Per cell: raster points g_ab at the centres of an Ng x Ng grid
 * over B (Eq. raster_grid), X = (cx - H) + (L/Ng)(a + 1/2), Y = (cy - H) + (L/Ng)(b + 1/2) in binary64;
 * kept when in the window (Eq. raster_grid's subset G).  Each kept point goes to the nearest windowed
 * sample (Eq. nn_assignment), the squared distance d2 = (X - x_q)^2 + (Y - y_q)^2 taken in binary64
 * (the samples' binary32 coordinates are exact in binary64), every operation rounded as written; a tie
 * goes to the lowest sample index.  n_q counts the points of sample q; A_q = n_q |D| / |G| (Eq. raster_area).  A windowed sample
 * with n_q = 0 takes the floor n_q = 1/2 and all are renormalised to sum to |D| (Eq. area_partition),
 * so w_q = max(n_q, 1/2) (|D| / sum_q' max(n_q', 1/2)) in binary64, rounded once to binary32 (with
 * no empty cell this is A_q).  Samples outside the window, and samples with a non-finite
 * coordinate, get w = 0 and count -1. */
int oracle_voronoi_weights_f32(int64_t n_cells, const int64_t *offsets, const int32_t *nverts,
                               const double *verts, const float *x, const float *y, double eta, int mask,
                               int Ng, float *w, int32_t *counts, int nthreads) {
    const int frame = 0;   /* the raster of Eq. raster_grid is laid out in the centroid-aligned frame */
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
    for (int64_t j = 0; j < n_cells; ++j) {
        oframe f;
        const int64_t q0 = offsets[j], q1 = offsets[j + 1];
        if (frame_of(nverts[j], verts + 12 * j, eta, mask, frame, &f)) {
            for (int64_t q = q0; q < q1; ++q) { w[q] = 0.0f; counts[q] = -1; }
            err |= 1;
            continue;
        }
        /* a sample with a non-finite coordinate is not a point of D: no Voronoi cell, no weight */
        for (int64_t q = q0; q < q1; ++q)
            counts[q] = (isfinite(x[q]) && isfinite(y[q]) && in_window(&f, (double)x[q], (double)y[q])) ? 0 : -1;
        const double x0 = f.cx - f.H, y0 = f.cy - f.H, step = f.L / Ng;
        for (int b = 0; b < Ng; ++b) {
            for (int a2 = 0; a2 < Ng; ++a2) {
                const double X = x0 + step * (a2 + 0.5), Y = y0 + step * (b + 0.5);
                if (!in_window(&f, X, Y)) continue;
                double best = 0.0;
                int64_t arg = -1;
                for (int64_t q = q0; q < q1; ++q) {
                    if (counts[q] < 0) continue;
                    const double dx = X - (double)x[q], dy = Y - (double)y[q];
                    const double d2 = dx * dx + dy * dy;
                    if (arg < 0 || d2 < best) { best = d2; arg = q; }
                }
                if (arg >= 0) counts[arg] += 1;
            }
        }
        double s = 0.0;   /* sum of max(n_q, 1/2): a multiple of 1/2, exact */
        for (int64_t q = q0; q < q1; ++q)
            if (counts[q] >= 0) s += counts[q] > 0 ? (double)counts[q] : 0.5;
        const double unit = s > 0.0 ? f.area / s : 0.0;
        for (int64_t q = q0; q < q1; ++q)
            w[q] = counts[q] < 0 ? 0.0f : (float)((counts[q] > 0 ? (double)counts[q] : 0.5) * unit);
    }
    return err ? -1 : 0;
}

/* ----------------------------------------------------------------------------------------- */
/* Sec. 3.2 diagnostics: reconstruction at the samples, relative RMSE, Parseval variances       */
/* ----------------------------------------------------------------------------------------- */

/* Exported: for every cell, with the mode set given as a mask over the P x P box:
 *   hrec_q  = Re sum_{mu in set} h_mu e^{+i k_mu . x'_q}   (Eq. tri_series; 0 outside the window)
 *   stats[4 j + 0] = eps_rel = sqrt(sum_q (h_q - hrec_q)^2 / sum_q h_q^2) over the windowed samples
 *                    (Eq. alps_relative_rmse; the 1/Q factors cancel; 0 when every h_q is 0)
 *   stats[4 j + 1] = sigma2_phys = (1/|D|) sum_q w_q h_q^2 over the windowed samples
 *   stats[4 j + 2] = sigma2_spec over the set, (m, n) != (0, 0)
 *   stats[4 j + 3] = sigma2_spec over the whole box, (m, n) != (0, 0)       (Eq. spectral_variance) */
int oracle_reconstruct_batch(int64_t n_cells, const int64_t *offsets, const int32_t *nverts,
                             const double *verts, const double *x, const double *y, const double *h,
                             const double *w, int P, double eta, int mask, int frame, const double *coeffs,
                             const uint8_t *modes, double *hrec, double *stats, int nthreads) {
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
    for (int64_t j = 0; j < n_cells; ++j) {
        oframe f;
        if (frame_of(nverts[j], verts + 12 * j, eta, mask, frame, &f)) { err |= 1; continue; }
        const double *cj = coeffs + 2 * (size_t)P * P * j;
        const uint8_t *sj = modes + (size_t)P * P * j;
        double *G = (double *)calloc(2 * (size_t)P * P, sizeof(double));
        if (!G) { err |= 2; continue; }
        double spec_set = 0.0, spec_all = 0.0;
        for (int i = 0; i < P * P; ++i) {
            const int dc = (i == (P / 2) * P + P / 2);
            const double e = cj[2 * i] * cj[2 * i] + cj[2 * i + 1] * cj[2 * i + 1];
            if (!dc) spec_all += e;
            if (sj[i]) {
                G[2 * i] = cj[2 * i];
                G[2 * i + 1] = cj[2 * i + 1];
                if (!dc) spec_set += e;
            }
        }
        double err2 = 0.0, h2 = 0.0, wh2 = 0.0;
        for (int64_t q = offsets[j]; q < offsets[j + 1]; ++q) {
            if (!in_window(&f, x[q], y[q])) {
                hrec[q] = 0.0;
                continue;
            }
            const double v = type2_point(&f, P, G, x[q], y[q]);
            hrec[q] = v;
            err2 += (h[q] - v) * (h[q] - v);
            h2 += h[q] * h[q];
            wh2 += w[q] * h[q] * h[q];
        }
        free(G);
        stats[4 * j + 0] = h2 > 0.0 ? sqrt(err2 / h2) : 0.0;
        stats[4 * j + 1] = wh2 / f.area;
        stats[4 * j + 2] = spec_set;
        stats[4 * j + 3] = spec_all;
    }
    return err ? -1 : 0;
}

/* ----------------------------------------------------------------------------------------- */
/* Sec. 2.2: Elastic Mode Selection                                                            */
/* ----------------------------------------------------------------------------------------- */

typedef struct { double E; int32_t p; } epair;

static int cmp_desc(const void *a, const void *b) {
    const epair *x = (const epair *)a, *y = (const epair *)b;
    if (x->E > y->E) return -1;
    if (x->E < y->E) return 1;
    return (x->p > y->p) - (x->p < y->p);   /* ties: ascending pair index */
}

/* Energy of the mode pair +-(m, n), Eq. "energy" generalised to pairs.  With fp32 != 0 the
 * energy is formed in binary32 from binary32 coefficients with the fixed evaluation
 * E = fma(re+, re+, im+ * im+) + fma(re-, re-, im- * im-), then times binary32(W); this is
 * the precision the GPU takes this integer-deciding step in. */
static double pair_energy(const double *c, int P, int m, int n, const double *W, int fp32, int dc) {
    int half = P / 2;
    size_t ip = (size_t)(n + half) * P + (m + half);
    size_t in = (size_t)(-n + half) * P + (-m + half);
    if (fp32) {
        float rp = (float)c[2 * ip], ipp = (float)c[2 * ip + 1];
        float rn = (float)c[2 * in], inn = (float)c[2 * in + 1];
        float ep = fmaf(rp, rp, ipp * ipp);   /* compiled with -ffp-contract=off */
        float en = fmaf(rn, rn, inn * inn);
        float e = dc ? ep : ep + en;
        if (W) e = e * (float)W[ip];
        return (double)e;
    }
    double e = c[2 * ip] * c[2 * ip] + c[2 * ip + 1] * c[2 * ip + 1];
    if (!dc) e += c[2 * in] * c[2 * in] + c[2 * in + 1] * c[2 * in + 1];
    if (W) e *= W[ip];
    return e;
}

typedef struct {
    int k_min, k_max;
    double alpha_min, alpha_max, delta, w1, w2;
    int sum_all;      /* 0: HEAD reading (J_max), 1: ALL reading (J*) */
    int include_dc;
    int energy_fp32;
    double sens_eps;  /* relative energy perturbation of the alpha_C sensitivity (diag[11]) */
} oems_params;

/* N_eff, S_delta, C and alpha_C (Eqs. n_eff, s_delta, c_score, alpha_c) of n energies sorted in
 * descending order; M1 (the sum that is the denominator of Eq. f_cum) through *m1. */
static double alpha_of(const epair *e, int J, const oems_params *pp, double *neff_o, double *S_o,
                       double *C_o, double *m1) {
    int Jmax = J < pp->k_max ? J : pp->k_max;                    /* footnote: J_max = min(J*, K_max) */
    int nsum = pp->sum_all ? J : Jmax;
    double M1 = 0.0, M2 = 0.0;
    for (int j = 0; j < nsum; ++j) { M1 += e[j].E; M2 += e[j].E * e[j].E; }
    double neff = M2 > 0.0 ? M1 * M1 / M2 : 0.0;                 /* Eq. n_eff */
    double S = 0.0;                                              /* Eq. s_delta */
    if (Jmax >= 2) {
        for (int j = 0; j < Jmax - 1; ++j)
            if (e[j + 1].E > 0.0) S += exp(-(e[j].E / e[j + 1].E - 1.0) / pp->delta);
        S /= (double)(Jmax - 1);
    }
    double nclip = neff < pp->k_max ? neff : (double)pp->k_max;
    double C = pp->w1 * nclip / pp->k_max + pp->w2 * S;          /* Eq. c_score */
    if (neff_o) *neff_o = neff;
    if (S_o) *S_o = S;
    if (C_o) *C_o = C;
    if (m1) *m1 = M1;
    return pp->alpha_min + (pp->alpha_max - pp->alpha_min) * C;  /* Eq. alpha_c */
}

/* How far alpha_C moves when every energy carries a relative error of eps: the energies in
 * sorted order are scaled by (1 + s (-1)^j eps) for s = +1 and s = -1 (alternating signs move
 * every successive ratio of Eq. s_delta by the most, a factor (1 +- eps) / (1 -+ eps); a common
 * factor would leave alpha_C unchanged), re-sorted, and alpha_C recomputed; the larger of the two
 * absolute changes. */
static double alpha_sensitivity(const epair *e, int J, const oems_params *pp, double alpha) {
    if (J < 1 || !(pp->sens_eps > 0.0)) return 0.0;
    epair *t = (epair *)malloc(sizeof(epair) * J);
    if (!t) return NAN;
    double worst = 0.0;
    for (int s = -1; s <= 1; s += 2) {
        for (int j = 0; j < J; ++j) {
            t[j] = e[j];
            t[j].E = e[j].E * (1.0 + (double)s * ((j & 1) ? -1.0 : 1.0) * pp->sens_eps);
        }
        qsort(t, J, sizeof(epair), cmp_desc);
        double d = fabs(alpha_of(t, J, pp, NULL, NULL, NULL, NULL) - alpha);
        if (d > worst) worst = d;
    }
    free(t);
    return worst;
}

/* Selection core on an unsorted list of J pair energies (Eqs. sorted_energy .. k_elastic).
 * diag (optional, 12 doubles):
 *   N_eff, S_delta, C, alpha_C, total, theta(K*), margin_rank, margin_theta, J*, n_positive,
 *   gap at K_max, alpha_C sensitivity.  margin_rank = (E_(K*) - E_(K*+1)) / E_(K*) and
 *   margin_theta = min(theta(K*) - alpha_C, alpha_C - theta(K*-1)) say how close the selection is
 *   to a tie in the ranking or at the threshold of Eq. k_elastic. */
static void ems_select(epair *e, int J, const oems_params *pp, int32_t *kstar, int32_t *sel,
                       double *retained, double *diag) {
    qsort(e, J, sizeof(epair), cmp_desc);                       /* Eq. sorted_energy */
    int Jmax = J < pp->k_max ? J : pp->k_max;                    /* footnote: J_max = min(J*, K_max) */
    int npos = 0;
    for (int j = 0; j < J; ++j) npos += e[j].E > 0.0;
    double neff, S, C, M1;
    double alpha = alpha_of(e, J, pp, &neff, &S, &C, &M1);
    double total = M1;                                           /* denominator of Eq. f_cum */
    int K = 0;
    double cum = 0.0, theta_k = 0.0;
    if (total > 0.0) {
        int kthr = -1;
        double cs = 0.0;
        for (int j = 0; j < Jmax; ++j) {                         /* Eq. f_cum, Eq. k_elastic */
            cs += e[j].E;
            if (cs >= alpha * total) { kthr = j + 1; break; }
        }
        if (kthr < 0) kthr = pp->k_max;
        K = kthr > pp->k_min ? kthr : pp->k_min;
        if (K > pp->k_max) K = pp->k_max;
        if (K > npos) K = npos;
        if (K > J) K = J;
        for (int j = 0; j < K; ++j) cum += e[j].E;
        theta_k = cum / total;
    }
    *kstar = K;
    for (int j = 0; j < pp->k_max; ++j) sel[j] = j < K ? e[j].p : -1;
    *retained = cum;
    if (diag) {
        double mr = NAN, mt = NAN;
        if (K > 0 && K < J && e[K - 1].E > 0.0) mr = (e[K - 1].E - e[K].E) / e[K - 1].E;
        if (K > 0 && total > 0.0) {
            double prev = (cum - e[K - 1].E) / total;
            double a = theta_k - alpha, b = alpha - prev;
            mt = a < b ? a : b;
        }
        double gk = NAN;   /* gap at the K_max boundary: which pairs form the head */
        if (J > pp->k_max && e[pp->k_max - 1].E > 0.0)
            gk = (e[pp->k_max - 1].E - e[pp->k_max].E) / e[pp->k_max - 1].E;
        diag[0] = neff; diag[1] = S; diag[2] = C; diag[3] = alpha; diag[4] = total;
        diag[5] = theta_k; diag[6] = mr; diag[7] = mt; diag[8] = J; diag[9] = npos;
        diag[10] = gk; diag[11] = alpha_sensitivity(e, J, pp, alpha);
    }
}

/* EMS on one P x P spectrum: pair energies of the symmetric box, then the selection core. */
static int ems_cell(int P, const double *c, const double *W, const oems_params *pp, int32_t *kstar,
                    int32_t *sel, double *retained, double *diag) {
    int half = P / 2, lim = half - 1;
    int cap = (2 * lim + 1) * (2 * lim + 1);
    epair *e = (epair *)malloc(sizeof(epair) * (cap > 0 ? cap : 1));
    if (!e) return -2;
    int J = 0;
    for (int n = -lim; n <= lim; ++n)
        for (int m = -lim; m <= lim; ++m) {
            int canon = (n > 0) || (n == 0 && m > 0);
            int dc = (n == 0 && m == 0);
            if (!(canon || (dc && pp->include_dc))) continue;
            e[J].E = pair_energy(c, P, m, n, W, pp->energy_fp32, dc);
            e[J].p = (n + half) * P + (m + half);
            ++J;
        }
    ems_select(e, J, pp, kstar, sel, retained, diag);
    free(e);
    return 0;
}

/* Exported: EMS over a batch of spectra.  W: NULL, one P*P table shared by all cells
 * (w_per_cell = 0), or one table per cell (w_per_cell = 1). */
int oracle_ems_batch(int64_t n_cells, int P, const double *coeffs, const double *W, int w_per_cell,
                     int k_min, int k_max, double alpha_min, double alpha_max, double delta, double w1,
                     double w2, int sum_all, int include_dc, int energy_fp32, double sens_eps,
                     int32_t *kstar, int32_t *sel, double *retained, double *diag, int nthreads) {
    oems_params pp = {k_min, k_max, alpha_min, alpha_max, delta, w1, w2, sum_all, include_dc, energy_fp32,
                      sens_eps};
    if (k_max < 1 || k_min < 0) return -1;
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(| : err)
#endif
    for (int64_t j = 0; j < n_cells; ++j) {
        const double *Wj = W ? W + (w_per_cell ? (size_t)P * P * j : 0) : NULL;
        if (ems_cell(P, coeffs + 2 * (size_t)P * P * j, Wj, &pp, kstar + j, sel + (size_t)k_max * j,
                     retained + j, diag ? diag + 12 * j : NULL))
            err |= 1;
    }
    return err ? -1 : 0;
}

/* Exported: EMS on an explicit list of J energies (any order), used to check the selection
 * rules on the paper's spectral families; sel receives positions in the input list. */
int oracle_ems_energies(int J, const double *E, int k_min, int k_max, double alpha_min, double alpha_max,
                        double delta, double w1, double w2, int sum_all, double sens_eps, int32_t *kstar,
                        int32_t *sel, double *retained, double *diag) {
    oems_params pp = {k_min, k_max, alpha_min, alpha_max, delta, w1, w2, sum_all, 0, 0, sens_eps};
    if (k_max < 1 || k_min < 0) return -1;
    epair *e = (epair *)malloc(sizeof(epair) * (J > 0 ? J : 1));
    if (!e) return -2;
    for (int j = 0; j < J; ++j) { e[j].E = E[j]; e[j].p = j; }
    ems_select(e, J, &pp, kstar, sel, retained, diag);
    free(e);
    return 0;
}

/* Exported: G = grad_power_j * dP_j / d(coeffs) for the EMS-retained power
 * P_j = sum_{p in S_j} W_p (|h_p|^2 + |h_-p|^2)  (S_j held fixed):  G_mu = 2 gp W_p h_mu on both
 * members of every selected pair, 0 elsewhere. */
int oracle_ems_grad_coeffs(int64_t n_cells, int P, const double *coeffs, const double *W, int w_per_cell,
                           int k_max, const int32_t *kstar, const int32_t *sel, const double *grad_power,
                           double *G) {
    int half = P / 2;
    memset(G, 0, sizeof(double) * 2 * (size_t)P * P * n_cells);
    for (int64_t j = 0; j < n_cells; ++j) {
        const double *c = coeffs + 2 * (size_t)P * P * j;
        const double *Wj = W ? W + (w_per_cell ? (size_t)P * P * j : 0) : NULL;
        double *g = G + 2 * (size_t)P * P * j;
        for (int k = 0; k < kstar[j]; ++k) {
            int p = sel[(size_t)k_max * j + k];
            int m = p % P - half, n = p / P - half;
            size_t ip = (size_t)p, in = (size_t)(-n + half) * P + (-m + half);
            double wt = Wj ? Wj[ip] : 1.0;
            double s = 2.0 * grad_power[j] * wt;
            g[2 * ip] = s * c[2 * ip];
            g[2 * ip + 1] = s * c[2 * ip + 1];
            if (in != ip) {
                g[2 * in] = s * c[2 * in];
                g[2 * in + 1] = s * c[2 * in + 1];
            }
        }
    }
    return 0;
}
