/*
 * tll_oracle.c -- plain FP64 CPU oracle for the batched lens log-likelihood.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file.  It is used by tests/, by __graft_entry__.smoke()
 * and by bench.py's cpu_baseline / reference leg, and nowhere else.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * It computes, slowly and literally, what the paper "CSST Strong Lensing
 * Preparation: Fast Modelling of Galaxy-Galaxy Strong Lenses in the Big Data
 * Era" (arXiv:2503.08586, TinyLensGpu) defines for one parameter vector:
 *
 *   lens equation                 Sec. 2.1, Eq. (1)
 *   image formation               Sec. 2.1, Eq. (2)
 *   4x4 supersampling + binning   Sec. 2.1 (text after Eq. 2)
 *   PSF convolution               Sec. 2.1, Eq. (3)
 *   Gaussian likelihood           Sec. 2.2, Eq. (5)
 *   linear amplitudes (delta fn)  Sec. 2.2, Eq. (6)
 *   d = B L s + n, NNLS           Sec. 2.3, Eq. (7) and the penalty after it
 *   Sersic profile, b_n           Sec. 2.4, Eqs. (8), (9)
 *   elliptical coordinates        Sec. 2.4, Eq. (10)
 *   ellipticity components        Sec. 2.4, Eq. (11)
 *   power-law convergence         Sec. 2.4, Eq. (12): SIE (gamma = 2) and the
 *                                 elliptical power law (EPL, any gamma)
 *   external shear                Sec. 2.4, Eqs. (13), (14)
 *
 * Readings taken where the paper is silent or ambiguous (each one is also
 * listed in the design notes):
 *   R1 grid: pixel (i row, j col) centre at (x0 + j*dpix, y0 + i*dpix);
 *      subpixel (a, c) of an s x s pixel at offset ((c+1/2)/s - 1/2)*dpix in x
 *      and ((a+1/2)/s - 1/2)*dpix in y.  Units: arcsec.
 *   R2 binning: a pixel takes the MEAN of its s*s subpixel values.
 *   R3 convolution: true convolution with the PSF normalised to unit sum,
 *      output the same size as the image, zero outside the image.
 *   R4 SIE: Eq. (12) with gamma = 2 and R replaced by the elliptical radius of
 *      Eq. (10), kappa = theta_E / (2 sqrt(q x'^2 + y'^2/q)); its deflection is
 *      the Kormann et al. (1994) closed form, written out in sie_alpha().
 *      The singular centre is regularised by psi >= 1e-12 arcsec.
 *   R5 shear: (gamma_1, gamma_2) are the Cartesian shear components
 *      gamma_1 = (psi_11 - psi_22)/2, gamma_2 = psi_12, so
 *      psi_ext = gamma_1 (x^2 - y^2)/2 + gamma_2 x y about the origin; this is
 *      Eq. (13) with gamma_1 = -gamma cos 2phi, gamma_2 = -gamma sin 2phi,
 *      which satisfies Eq. (14).
 *   R6 b_n: the exact root of Eq. (9), P(2n, b_n) = 1/2, no approximation.
 *   R7 amplitudes: non-negative least squares over the two unit-amplitude
 *      columns (lens light, lensed source); in "fixed" mode the amplitudes are
 *      the I_e slots of the parameter vector instead.
 *   R8 likelihood: log L = -chi^2/2 - sum_{w>0} log(2 pi sigma^2)/2; a pixel
 *      whose sigma is not finite and > 0, or whose datum is not finite, is
 *      masked (weight 0, no normalisation term).
 *   R9 invalid parameter vectors (|eps| >= 1, r_e <= 0, n outside [0.2, 10],
 *      theta_E < 0, non-finite entries; for the EPL a slope outside
 *      (1, 3)) give log L = -infinity.
 *   R12 EPL: Eq. (12) with R replaced by the elliptical radius of Eq. (10),
 *      kappa = (3 - gamma)/2 (theta_E / R_p)^(gamma - 1); with t = gamma - 1,
 *      b = theta_E sqrt(q) and R = sqrt(q^2 x'^2 + y'^2) = sqrt(q) R_p this is
 *      kappa = (2 - t)/2 (b/R)^t, whose deflection is the closed form of
 *      Tessore & Metcalf (2015), written out in epl_alpha().  gamma = 2 is the
 *      SIE of R4.
 *
 * Parameter vector layout (21 doubles / floats; 22 for the EPL):
 *   [0] theta_E  [1] eps1_m [2] eps2_m [3] x_m [4] y_m [5] gamma_1 [6] gamma_2
 *   [7] I_e^L [8] r_e^L [9] n^L [10] eps1_L [11] eps2_L [12] x_L [13] y_L
 *   [14] I_e^S [15] r_e^S [16] n^S [17] eps1_S [18] eps2_S [19] x_S [20] y_S
 *   [21] gamma (the mass slope; EPL lenses only)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_NPAR 21
#define ORA_MASS_SIE 0
#define ORA_MASS_EPL 1

/* ---------------------------------------------------------------- Eq. (11) */
/* Ellipticity components -> (q, position angle).  Eq. (11):
 * (eps1, eps2) = (1-q)/(1+q) (cos 2 theta_p, sin 2 theta_p), inverted.
 * Returns -1 when |eps| >= 1 (no ellipse). */
int ora_ellipse(double e1, double e2, double *q, double *phi)
{
    double e = sqrt(e1 * e1 + e2 * e2);
    if (!(e < 1.0)) return -1;
    *q = (1.0 - e) / (1.0 + e);
    *phi = 0.5 * atan2(e2, e1);
    return 0;
}

/* ----------------------------------------------------------------- Eq. (9) */
/* Regularised lower incomplete gamma P(a, x) = gamma(a, x) / Gamma(a), from
 * its power series gamma(a,x) = x^a e^{-x} sum_k x^k / (a (a+1) ... (a+k)).
 * All terms are positive, so the sum has no cancellation. */
double ora_gammainc_P(double a, double x)
{
    if (x <= 0.0) return 0.0;
    double term = 1.0 / a, sum = term;
    for (int k = 1; k < 100000; ++k) {
        term *= x / (a + k);
        sum += term;
        if (term < sum * 1e-17) break;
    }
    return exp(a * log(x) - x - lgamma(a)) * sum;
}

/* b_n of Eq. (9): Gamma(2n) = 2 gamma(2n, b_n), i.e. P(2n, b_n) = 1/2.
 * P(2n, .) increases monotonically from 0 to 1, and its median is below 2n,
 * so [0, 2n + 1] brackets the root; plain bisection to the last bit. */
double ora_sersic_bn(double n)
{
    double a = 2.0 * n, lo = 0.0, hi = a + 1.0;
    while (ora_gammainc_P(a, hi) < 0.5) hi *= 2.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (ora_gammainc_P(a, mid) < 0.5) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* --------------------------------------------------- Eqs. (8), (10), (11) */
/* Unit-amplitude elliptical Sersic at (x, y): Eq. (8) with I_e = 1 and R
 * replaced by R_p of Eq. (10), rotated by theta_p about (cx, cy). */
double ora_sersic(double x, double y, double cx, double cy, double q,
                  double phi, double re, double n, double bn)
{
    double c = cos(phi), s = sin(phi);
    double x1 = (x - cx) * c + (y - cy) * s;          /* Eq. (10), first row */
    double x2 = -(x - cx) * s + (y - cy) * c;         /* Eq. (10), second row */
    double Rp = sqrt(x1 * x1 * q + x2 * x2 / q);      /* Eq. (10), third row */
    return exp(-bn * (pow(Rp / re, 1.0 / n) - 1.0)); /* Eq. (8) */
}

/* ------------------------------------------------------------ Eq. (12) */
/* SIE deflection (reading R4).  In the frame rotated by phi about (xc, yc)
 * (the rotation of Eq. 10), with f = sqrt(1 - q^2), psi = sqrt(q^2 x'^2 + y'^2):
 *   alpha_x' = theta_E sqrt(q)/f * atan (f x'/psi)
 *   alpha_y' = theta_E sqrt(q)/f * atanh(f y'/psi)
 * and rotated back by +phi.  For q = 1 (f = 0) it is the singular isothermal
 * sphere, alpha = theta_E (x', y')/r. */
void ora_sie_alpha(double x, double y, double thE, double q, double phi,
                   double xc, double yc, double *ax, double *ay)
{
    double c = cos(phi), s = sin(phi);
    double xp = (x - xc) * c + (y - yc) * s;
    double yp = -(x - xc) * s + (y - yc) * c;
    double psi = sqrt(q * q * xp * xp + yp * yp);
    if (psi < 1e-12) psi = 1e-12;
    double f = sqrt(1.0 - q * q);
    double axp, ayp;
    if (f > 0.0) {
        double pre = thE * sqrt(q) / f;
        axp = pre * atan(f * xp / psi);
        ayp = pre * atanh(f * yp / psi);
    } else {
        axp = thE * xp / psi;
        ayp = thE * yp / psi;
    }
    *ax = axp * c - ayp * s;
    *ay = axp * s + ayp * c;
}

/* EPL deflection (reading R12).  In the frame rotated by phi about
 * (xc, yc), with t = gamma - 1, b = theta_E sqrt(q), R = sqrt(q^2 x'^2 + y'^2)
 * and the elliptical angle R e^{i varphi} = q x' + i y', Tessore & Metcalf
 * (2015) give, as a complex number alpha' = alpha_x' + i alpha_y',
 *   alpha' = 2 b / (1 + q) (b/R)^(t - 1) e^{i varphi}
 *            2F1(1, t/2; 2 - t/2; -(1 - q)/(1 + q) e^{2 i varphi}),
 * the hypergeometric function summed as its power series (the ratio of term
 * n to term n - 1 is z (2n - 2 + t)/(2n + 2 - t), |z| = (1-q)/(1+q) < 1),
 * until a term is below 1e-17 of the sum.  Rotated back by +phi. */
void ora_epl_alpha(double x, double y, double thE, double q, double phi,
                   double xc, double yc, double gamma, double *ax, double *ay)
{
    double c = cos(phi), s = sin(phi);
    double xp = (x - xc) * c + (y - yc) * s;
    double yp = -(x - xc) * s + (y - yc) * c;
    double R = sqrt(q * q * xp * xp + yp * yp);
    if (R < 1e-12) R = 1e-12;
    double t = gamma - 1.0, b = thE * sqrt(q);
    double cv = q * xp / R, sv = yp / R;             /* e^{i varphi} */
    double c2 = cv * cv - sv * sv, s2 = 2.0 * cv * sv;  /* e^{2 i varphi} */
    double zf = -(1.0 - q) / (1.0 + q);
    double tr = 1.0, ti = 0.0, sr = 1.0, si = 0.0;   /* term, sum */
    for (int n = 1; n < 100000; ++n) {
        double ratio = zf * (2.0 * n - 2.0 + t) / (2.0 * n + 2.0 - t);
        double nr = (tr * c2 - ti * s2) * ratio;
        double ni = (tr * s2 + ti * c2) * ratio;
        tr = nr; ti = ni;
        sr += tr; si += ti;
        if (sqrt(tr * tr + ti * ti) < 1e-17 * sqrt(sr * sr + si * si)) break;
    }
    double pre = 2.0 * b / (1.0 + q) * pow(b / R, t - 1.0);
    double axp = pre * (cv * sr - sv * si);
    double ayp = pre * (cv * si + sv * sr);
    *ax = axp * c - ayp * s;
    *ay = axp * s + ayp * c;
}

/* ------------------------------------------------------ Eqs. (13), (14) */
/* External shear potential (reading R5): psi = g1 (x^2 - y^2)/2 + g2 x y. */
double ora_shear_potential(double x, double y, double g1, double g2)
{
    return 0.5 * g1 * (x * x - y * y) + g2 * x * y;
}

/* Its gradient, the shear deflection. */
void ora_shear_alpha(double x, double y, double g1, double g2,
                     double *ax, double *ay)
{
    *ax = g1 * x + g2 * y;
    *ay = g2 * x - g1 * y;
}

/* ------------------------------------------------------------ parameters */
typedef struct {
    int mass;                       /* ORA_MASS_SIE or ORA_MASS_EPL */
    double thE, qm, phim, xm, ym, g1, g2, gamma;
    double IeL, reL, nL, qL, phiL, xL, yL, bL;
    double IeS, reS, nS, qS, phiS, xS, yS, bS;
} ora_model;

/* Decode one parameter vector (21 entries, 22 for the EPL); returns -1 for
 * an invalid vector (R9). */
int ora_decode(const double *p, int mass, ora_model *m)
{
    const int np = mass == ORA_MASS_EPL ? ORA_NPAR + 1 : ORA_NPAR;
    for (int k = 0; k < np; ++k)
        if (!isfinite(p[k])) return -1;
    m->mass = mass;
    m->gamma = 2.0;
    if (mass == ORA_MASS_EPL) {
        if (!(p[21] > 1.0 && p[21] < 3.0)) return -1;
        m->gamma = p[21];
    }
    if (p[0] < 0.0) return -1;
    if (ora_ellipse(p[1], p[2], &m->qm, &m->phim)) return -1;
    if (ora_ellipse(p[10], p[11], &m->qL, &m->phiL)) return -1;
    if (ora_ellipse(p[17], p[18], &m->qS, &m->phiS)) return -1;
    if (!(p[8] > 0.0) || !(p[15] > 0.0)) return -1;
    if (!(p[9] >= 0.2 && p[9] <= 10.0)) return -1;
    if (!(p[16] >= 0.2 && p[16] <= 10.0)) return -1;
    m->thE = p[0]; m->xm = p[3]; m->ym = p[4]; m->g1 = p[5]; m->g2 = p[6];
    m->IeL = p[7]; m->reL = p[8]; m->nL = p[9]; m->xL = p[12]; m->yL = p[13];
    m->IeS = p[14]; m->reS = p[15]; m->nS = p[16]; m->xS = p[19]; m->yS = p[20];
    m->bL = ora_sersic_bn(m->nL);
    m->bS = ora_sersic_bn(m->nS);
    return 0;
}

/* Lens equation, Eq. (1): beta = theta - alpha_SIE(theta) - alpha_shear(theta). */
void ora_trace(const ora_model *m, double x, double y, double *bx, double *by)
{
    double ax, ay, sx, sy;
    if (m->mass == ORA_MASS_EPL)
        ora_epl_alpha(x, y, m->thE, m->qm, m->phim, m->xm, m->ym, m->gamma, &ax, &ay);
    else
        ora_sie_alpha(x, y, m->thE, m->qm, m->phim, m->xm, m->ym, &ax, &ay);
    ora_shear_alpha(x, y, m->g1, m->g2, &sx, &sy);
    *bx = x - ax - sx;
    *by = y - ay - sy;
}

/* Public wrapper of the lens equation for one point (used by the pins). */
int ora_trace_point(const double *p, double x, double y, double *bx, double *by)
{
    ora_model m;
    if (ora_decode(p, ORA_MASS_SIE, &m)) return -1;
    ora_trace(&m, x, y, bx, by);
    return 0;
}

/* ------------------------------------------------------------ the image */
/* Unit-amplitude lens-light and lensed-source columns (the two columns of L in
 * Eq. 7), before the PSF: each subpixel of an s x s grid per pixel (R1) is
 * evaluated with Eq. (2) split into its two terms, then binned by the mean
 * (R2).  Lens light at theta, source at beta(theta) of Eq. (1). */
void ora_columns(const ora_model *m, int ny, int nx, double dpix, int sub,
                 double x0, double y0, double *lens, double *src)
{
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double sl = 0.0, ss = 0.0;
            for (int a = 0; a < sub; ++a)
                for (int c = 0; c < sub; ++c) {
                    double x = x0 + j * dpix + ((c + 0.5) / sub - 0.5) * dpix;
                    double y = y0 + i * dpix + ((a + 0.5) / sub - 0.5) * dpix;
                    double bx, by;
                    sl += ora_sersic(x, y, m->xL, m->yL, m->qL, m->phiL,
                                     m->reL, m->nL, m->bL);
                    ora_trace(m, x, y, &bx, &by);
                    ss += ora_sersic(bx, by, m->xS, m->yS, m->qS, m->phiS,
                                     m->reS, m->nS, m->bS);
                }
            lens[i * nx + j] = sl / (double)(sub * sub);
            src[i * nx + j] = ss / (double)(sub * sub);
        }
}

/* Eq. (3) on the pixel grid (R3): out(i,j) = sum_{r,c} K[r][c] img(i-(r-h), j-(c-h)),
 * h = (k-1)/2, zero outside the image.  The caller passes the PSF already
 * normalised to unit sum. */
void ora_convolve(const double *img, int ny, int nx, const double *psf, int k,
                  double *out)
{
    int h = (k - 1) / 2;
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double acc = 0.0;
            for (int r = 0; r < k; ++r)
                for (int c = 0; c < k; ++c) {
                    int ii = i - (r - h), jj = j - (c - h);
                    if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
                    acc += psf[r * k + c] * img[ii * nx + jj];
                }
            out[i * nx + j] = acc;
        }
}

/* Normalise a PSF to unit sum (R3).  Returns -1 if its sum is not > 0. */
int ora_psf_normalise(const double *psf_in, int k, double *psf_out)
{
    double s = 0.0;
    for (int t = 0; t < k * k; ++t) s += psf_in[t];
    if (!(s > 0.0) || !isfinite(s)) return -1;
    for (int t = 0; t < k * k; ++t) psf_out[t] = psf_in[t] / s;
    return 0;
}

/* Pixel weights w = 1/sigma^2 with the masking rule of R8. */
void ora_weights(const double *data, const double *sigma, int npix, double *w)
{
    for (int t = 0; t < npix; ++t) {
        double s = sigma[t];
        w[t] = (isfinite(s) && s > 0.0 && isfinite(data[t])) ? 1.0 / (s * s) : 0.0;
    }
}

/* chi^2 of Eq. (5) for amplitudes (sl, ss): sum_i w_i (d_i - sl ml_i - ss ms_i)^2,
 * by a direct pass over the pixels. */
double ora_chi2(const double *ml, const double *ms, const double *d,
                const double *w, int npix, double sl, double ss)
{
    double chi2 = 0.0;
    for (int t = 0; t < npix; ++t) {
        if (w[t] == 0.0) continue;
        double r = d[t] - sl * ml[t] - ss * ms[t];
        chi2 += w[t] * r * r;
    }
    return chi2;
}

/* Non-negative least squares over two columns (Sec. 2.3: minimise
 * ||(M s - d)/n|| subject to s >= 0).  The minimiser of a convex quadratic
 * over the quadrant is the unconstrained minimiser of one of its faces
 * {both free, lens only, source only, none} that is feasible; all four are
 * formed from A = M^T W M, b = M^T W d and the best feasible one (by a direct
 * chi^2 pass) is returned.  Ties go to fewer free columns, then the lens
 * column. */
void ora_nnls2(const double *ml, const double *ms, const double *d,
               const double *w, int npix, double *s_out)
{
    double All = 0, Als = 0, Ass = 0, bl = 0, bs = 0;
    for (int t = 0; t < npix; ++t) {
        if (w[t] == 0.0) continue;      /* masked pixel (R8) */
        All += w[t] * ml[t] * ml[t];
        Als += w[t] * ml[t] * ms[t];
        Ass += w[t] * ms[t] * ms[t];
        bl += w[t] * ml[t] * d[t];
        bs += w[t] * ms[t] * d[t];
    }
    double cand[4][2];
    int ok[4] = {1, 0, 0, 0};
    cand[0][0] = 0.0; cand[0][1] = 0.0;
    if (All > 0.0 && bl > 0.0) { ok[1] = 1; cand[1][0] = bl / All; cand[1][1] = 0.0; }
    if (Ass > 0.0 && bs > 0.0) { ok[2] = 1; cand[2][0] = 0.0; cand[2][1] = bs / Ass; }
    double det = All * Ass - Als * Als;
    if (det > 0.0) {
        double sl = (Ass * bl - Als * bs) / det;
        double ss = (All * bs - Als * bl) / det;
        if (sl > 0.0 && ss > 0.0) { ok[3] = 1; cand[3][0] = sl; cand[3][1] = ss; }
    }
    int best = 0;
    double bestc = ora_chi2(ml, ms, d, w, npix, 0.0, 0.0);
    for (int k = 1; k < 4; ++k) {
        if (!ok[k]) continue;
        double c = ora_chi2(ml, ms, d, w, npix, cand[k][0], cand[k][1]);
        if (c < bestc) { bestc = c; best = k; }
    }
    s_out[0] = cand[best][0];
    s_out[1] = cand[best][1];
}

/* A lens: observed image, noise map, PSF and grid, as the oracle holds it. */
typedef struct {
    int ny, nx, sub, k;
    double dpix, x0, y0;
    const double *data, *sigma, *psf; /* psf: raw, normalised here */
    int mass;                         /* ORA_MASS_SIE or ORA_MASS_EPL */
} ora_lens;

/* Everything for one parameter vector.  mode 0: NNLS amplitudes (R7);
 * mode 1: fixed amplitudes from the I_e slots.  Optional outputs (may be
 * NULL): the two blurred unit columns, the blurred model, the amplitudes.
 * Returns log L (R8), -INFINITY for an invalid vector (R9). */
double ora_loglike_full(const ora_lens *L, const double *p, int mode,
                        double *ml_out, double *ms_out, double *model_out,
                        double *amps_out)
{
    ora_model m;
    int npix = L->ny * L->nx;
    if (ora_decode(p, L->mass, &m)) return -INFINITY;
    double *il = malloc(sizeof(double) * npix), *is = malloc(sizeof(double) * npix);
    double *ml = malloc(sizeof(double) * npix), *ms = malloc(sizeof(double) * npix);
    double *w = malloc(sizeof(double) * npix);
    double *psf = malloc(sizeof(double) * L->k * L->k);
    double res = -INFINITY;
    if (!il || !is || !ml || !ms || !w || !psf) goto done;
    if (ora_psf_normalise(L->psf, L->k, psf)) goto done;
    ora_columns(&m, L->ny, L->nx, L->dpix, L->sub, L->x0, L->y0, il, is);
    ora_convolve(il, L->ny, L->nx, psf, L->k, ml);   /* B L_l, Eq. (7) */
    ora_convolve(is, L->ny, L->nx, psf, L->k, ms);   /* B L_s, Eq. (7) */
    ora_weights(L->data, L->sigma, npix, w);
    double s[2];
    if (mode == 0) ora_nnls2(ml, ms, L->data, w, npix, s);
    else { s[0] = m.IeL; s[1] = m.IeS; }
    double chi2 = ora_chi2(ml, ms, L->data, w, npix, s[0], s[1]);
    double norm = 0.0;
    for (int t = 0; t < npix; ++t)
        if (w[t] > 0.0) norm += log(2.0 * M_PI / w[t]);
    res = -0.5 * chi2 - 0.5 * norm;                  /* log of Eq. (5) */
    if (ml_out) memcpy(ml_out, ml, sizeof(double) * npix);
    if (ms_out) memcpy(ms_out, ms, sizeof(double) * npix);
    if (model_out)
        for (int t = 0; t < npix; ++t) model_out[t] = s[0] * ml[t] + s[1] * ms[t];
    if (amps_out) { amps_out[0] = s[0]; amps_out[1] = s[1]; }
done:
    free(il); free(is); free(ml); free(ms); free(w); free(psf);
    return res;
}

/* Unblurred unit columns for one vector (for per-stage parity checks).
 * Returns -1 for an invalid vector. */
int ora_unblurred_columns(const ora_lens *L, const double *p, double *il, double *is)
{
    ora_model m;
    if (ora_decode(p, L->mass, &m)) return -1;
    ora_columns(&m, L->ny, L->nx, L->dpix, L->sub, L->x0, L->y0, il, is);
    return 0;
}

/* Batch of B vectors (params row-major [B][21], [B][22] for the EPL);
 * parallel over vectors only (each vector's arithmetic is unchanged).
 * nthreads <= 0: library default. */
void ora_loglike_batch(const ora_lens *L, const double *params, int B, int mode,
                       double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b)
        out[b] = ora_loglike_full(L, params + (size_t)b * (L->mass == ORA_MASS_EPL
                                                               ? ORA_NPAR + 1 : ORA_NPAR),
                                  mode, NULL, NULL, NULL, NULL);
    (void)nthreads;
}

/* Number of threads an OpenMP region of this library would use. */
int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ================================================================
 * Multi-component light and N-column non-negative least squares.
 *
 * Sec. 2.3, Eq. (7): the lens light and the source light are superpositions
 * of N_l and N_s unit-amplitude profiles; each profile is one column of
 * L = [L_l | L_s], M = B L, and the amplitudes s >= 0 minimise
 * ||(M s - d)/n|| (the penalty after Eq. 7), solved by FNNLS (Bro & de Jong
 * 1997).  Sec. 3.2 models SLACS lenses with two Sersic components per
 * galaxy sharing one centre and one ellipticity, with the indices fixed at 1
 * and 4; Sec. 4.3 names the multiple Gaussian expansion (MGE).  This part of
 * the oracle therefore takes a list of components, each a Sersic (Eq. 8) or
 * a Gaussian, in the lens plane (at theta) or the source plane (at beta of
 * Eq. 1), all components of one plane sharing that plane's centre and
 * ellipticity (Eq. 10, 11).
 *
 * Readings (listed with the others in the design notes):
 *   R13 Gaussian component: unit central intensity, exp(-R_p^2 / (2 sigma^2))
 *       with the R_p of Eq. (10) (the same elliptical radius as the Sersic);
 *       the paper prints no formula for it.  Its scale is sigma (arcsec).
 *   R14 parameter vector of a multi-component model:
 *       [0] theta_E [1] eps1_m [2] eps2_m [3] x_m [4] y_m [5] gamma_1
 *       [6] gamma_2 [7] eps1_L [8] eps2_L [9] x_L [10] y_L [11] eps1_S
 *       [12] eps2_S [13] x_S [14] y_S, then, component by component, the
 *       free values: its scale (r_e or sigma) if free, then its Sersic index
 *       if free; an EPL mass appends its slope last.  Fixed values come from
 *       the component list.  Invalid as R9 (scale <= 0, index outside
 *       [0.2, 10], |eps| >= 1, theta_E < 0, non-finite).
 *   R15 FNNLS tolerance: a column enters the passive set while its gradient
 *       b_j - (A x)_j exceeds 10 eps ||A||_1 n (eps = 2^-52), and a
 *       passive amplitude that reaches a non-positive value leaves it; the
 *       step that would re-enter a column whose least-squares value is not
 *       positive is skipped for that pass (the Lawson-Hanson safeguard).
 * ================================================================ */
#define ORA_COMP_SERSIC 0
#define ORA_COMP_GAUSS 1
#define ORA_PLANE_LENS 0
#define ORA_PLANE_SOURCE 1
#define ORA_FREE_SCALE 1
#define ORA_FREE_INDEX 2
#define ORA_MAXC 64
#define ORA_MHEAD 15

typedef struct {
    int type, plane, flags;
    double scale, index;
} ora_comp_spec;

typedef struct {
    ora_model mass;                 /* mass and shear fields only */
    double qL, phiL, xL, yL, qS, phiS, xS, yS;
    int nc;
    int type[ORA_MAXC], plane[ORA_MAXC];
    double scale[ORA_MAXC], n[ORA_MAXC], bn[ORA_MAXC];
} ora_mmodel;

/* Entries of a multi-component parameter vector (R14), -1 for a bad list. */
int ora_multi_nparam(const ora_comp_spec *c, int nc, int mass)
{
    if (nc < 1 || nc > ORA_MAXC) return -1;
    int np = ORA_MHEAD;
    for (int k = 0; k < nc; ++k) {
        if (c[k].type != ORA_COMP_SERSIC && c[k].type != ORA_COMP_GAUSS) return -1;
        if (c[k].plane != ORA_PLANE_LENS && c[k].plane != ORA_PLANE_SOURCE) return -1;
        if (c[k].flags & ORA_FREE_SCALE) ++np;
        if (c[k].type == ORA_COMP_SERSIC && (c[k].flags & ORA_FREE_INDEX)) ++np;
    }
    return np + (mass == ORA_MASS_EPL ? 1 : 0);
}

/* Decode a multi-component vector (R14); -1 if invalid (R9). */
int ora_decode_multi(const double *p, const ora_comp_spec *c, int nc, int mass,
                     ora_mmodel *m)
{
    int np = ora_multi_nparam(c, nc, mass);
    if (np < 0) return -1;
    for (int k = 0; k < np; ++k)
        if (!isfinite(p[k])) return -1;
    ora_model *mm = &m->mass;
    memset(mm, 0, sizeof *mm);
    mm->mass = mass;
    mm->gamma = 2.0;
    if (mass == ORA_MASS_EPL) {
        if (!(p[np - 1] > 1.0 && p[np - 1] < 3.0)) return -1;
        mm->gamma = p[np - 1];
    }
    if (p[0] < 0.0) return -1;
    if (ora_ellipse(p[1], p[2], &mm->qm, &mm->phim)) return -1;
    if (ora_ellipse(p[7], p[8], &m->qL, &m->phiL)) return -1;
    if (ora_ellipse(p[11], p[12], &m->qS, &m->phiS)) return -1;
    mm->thE = p[0]; mm->xm = p[3]; mm->ym = p[4]; mm->g1 = p[5]; mm->g2 = p[6];
    m->xL = p[9]; m->yL = p[10]; m->xS = p[13]; m->yS = p[14];
    m->nc = nc;
    int slot = ORA_MHEAD;
    for (int k = 0; k < nc; ++k) {
        m->type[k] = c[k].type;
        m->plane[k] = c[k].plane;
        m->scale[k] = (c[k].flags & ORA_FREE_SCALE) ? p[slot++] : c[k].scale;
        m->n[k] = 0.0;
        m->bn[k] = 0.0;
        if (!(m->scale[k] > 0.0) || !isfinite(m->scale[k])) return -1;
        if (c[k].type == ORA_COMP_SERSIC) {
            m->n[k] = (c[k].flags & ORA_FREE_INDEX) ? p[slot++] : c[k].index;
            if (!(m->n[k] >= 0.2 && m->n[k] <= 10.0)) return -1;
            m->bn[k] = ora_sersic_bn(m->n[k]);
        }
    }
    return 0;
}

/* Unit-central-intensity elliptical Gaussian (R13) at (x, y): the R_p of
 * Eq. (10) in the frame rotated by phi about (cx, cy). */
double ora_gauss(double x, double y, double cx, double cy, double q,
                 double phi, double sigma)
{
    double c = cos(phi), s = sin(phi);
    double x1 = (x - cx) * c + (y - cy) * s;
    double x2 = -(x - cx) * s + (y - cy) * c;
    double R2 = x1 * x1 * q + x2 * x2 / q;
    return exp(-R2 / (2.0 * sigma * sigma));
}

/* The nc unit columns of L (Eq. 7) before the PSF, cols[k][npix]: each
 * subpixel of the s x s grid (R1) evaluates every component at theta (lens
 * plane) or at beta(theta) of Eq. (1) (source plane); binned by the mean (R2). */
void ora_multi_columns(const ora_mmodel *m, int ny, int nx, double dpix, int sub,
                       double x0, double y0, double *cols)
{
    int npix = ny * nx;
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double acc[ORA_MAXC] = {0};
            for (int a = 0; a < sub; ++a)
                for (int c = 0; c < sub; ++c) {
                    double x = x0 + j * dpix + ((c + 0.5) / sub - 0.5) * dpix;
                    double y = y0 + i * dpix + ((a + 0.5) / sub - 0.5) * dpix;
                    double bx, by;
                    ora_trace(&m->mass, x, y, &bx, &by);
                    for (int k = 0; k < m->nc; ++k) {
                        int src = m->plane[k] == ORA_PLANE_SOURCE;
                        double px = src ? bx : x, py = src ? by : y;
                        double cx = src ? m->xS : m->xL, cy = src ? m->yS : m->yL;
                        double q = src ? m->qS : m->qL, phi = src ? m->phiS : m->phiL;
                        acc[k] += m->type[k] == ORA_COMP_SERSIC
                                      ? ora_sersic(px, py, cx, cy, q, phi, m->scale[k],
                                                   m->n[k], m->bn[k])
                                      : ora_gauss(px, py, cx, cy, q, phi, m->scale[k]);
                    }
                }
            for (int k = 0; k < m->nc; ++k)
                cols[(size_t)k * npix + i * nx + j] = acc[k] / (double)(sub * sub);
        }
}

/* Solve G z = r for the symmetric positive definite k x k matrix G
 * (row-major) by the Cholesky factorisation G = R^T R; -1 if a pivot is
 * not positive. */
int ora_chol_solve(const double *G, const double *r, int k, double *z)
{
    double R[ORA_MAXC * ORA_MAXC], y[ORA_MAXC];
    for (int i = 0; i < k; ++i)
        for (int j = i; j < k; ++j) {
            double v = G[i * k + j];
            for (int t = 0; t < i; ++t) v -= R[t * k + i] * R[t * k + j];
            if (i == j) {
                if (!(v > 0.0)) return -1;
                R[i * k + i] = sqrt(v);
            } else {
                R[i * k + j] = v / R[i * k + i];
            }
        }
    for (int i = 0; i < k; ++i) {            /* R^T y = r */
        double v = r[i];
        for (int t = 0; t < i; ++t) v -= R[t * k + i] * y[t];
        y[i] = v / R[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {       /* R z = y */
        double v = y[i];
        for (int t = i + 1; t < k; ++t) v -= R[i * k + t] * z[t];
        z[i] = v / R[i * k + i];
    }
    return 0;
}

/* Least squares restricted to the passive set: s_P = A_PP^{-1} b_P, s = 0
 * elsewhere.  -1 if A_PP is not positive definite. */
static int ora_passive_solve(const double *A, const double *b, const int *P, int n,
                             double *s)
{
    int idx[ORA_MAXC], k = 0;
    double G[ORA_MAXC * ORA_MAXC], r[ORA_MAXC], z[ORA_MAXC];
    for (int i = 0; i < n; ++i)
        if (P[i]) idx[k++] = i;
    for (int a = 0; a < k; ++a) {
        r[a] = b[idx[a]];
        for (int c = 0; c < k; ++c) G[a * k + c] = A[idx[a] * n + idx[c]];
    }
    for (int i = 0; i < n; ++i) s[i] = 0.0;
    if (k == 0) return 0;
    if (ora_chol_solve(G, r, k, z)) return -1;
    for (int a = 0; a < k; ++a) s[idx[a]] = z[a];
    return 0;
}

/* FNNLS (Bro & de Jong 1997): min ||Z x - y||^2 subject to x >= 0, given
 * only A = Z^T Z (n x n, row-major, n <= ORA_MAXC) and b = Z^T y -- the
 * Lawson-Hanson active-set method run on the normal equations (Sec. 2.3:
 * the paper's linear solve).  Steps, with R15's tolerance:
 *   start with every column active (held at zero): x = 0, gradient w = b;
 *   while some active column has w_j > tol: make the one with the largest
 *   w_j passive; solve the passive least-squares problem for s; while some
 *   passive s_i <= 0, move x towards s as far as feasibility allows
 *   (alpha = min x_i/(x_i - s_i) over those i), make the columns that reach
 *   zero active, and solve again; then x = s and w = b - A x.
 * Returns the number of outer steps, -1 if the step cap (30 n) ran out. */
int ora_fnnls(const double *A, const double *b, int n, double *x)
{
    int P[ORA_MAXC] = {0}, blocked[ORA_MAXC] = {0};
    double w[ORA_MAXC], s[ORA_MAXC];
    double norm1 = 0.0;
    for (int j = 0; j < n; ++j) {
        double cs = 0.0;
        for (int i = 0; i < n; ++i) cs += fabs(A[i * n + j]);
        if (cs > norm1) norm1 = cs;
    }
    const double tol = 10.0 * 2.220446049250313e-16 * norm1 * n;
    for (int i = 0; i < n; ++i) { x[i] = 0.0; w[i] = b[i]; }
    for (int step = 0; step < 30 * n; ++step) {
        int j = -1;
        double wmax = tol;
        for (int i = 0; i < n; ++i)
            if (!P[i] && !blocked[i] && w[i] > wmax) { wmax = w[i]; j = i; }
        if (j < 0) return step;
        P[j] = 1;
        if (ora_passive_solve(A, b, P, n, s) || !(s[j] > 0.0)) {
            P[j] = 0;             /* Lawson-Hanson safeguard (R15) */
            blocked[j] = 1;
            continue;
        }
        for (int inner = 0; inner <= n; ++inner) {
            double alpha = 2.0;
            int kmin = -1;
            for (int i = 0; i < n; ++i)
                if (P[i] && s[i] <= 0.0) {
                    double a = x[i] / (x[i] - s[i]);
                    if (a < alpha) { alpha = a; kmin = i; }
                }
            if (kmin < 0) break;
            for (int i = 0; i < n; ++i) x[i] += alpha * (s[i] - x[i]);
            x[kmin] = 0.0;
            for (int i = 0; i < n; ++i)
                if (P[i] && x[i] <= 0.0) { P[i] = 0; x[i] = 0.0; }
            if (ora_passive_solve(A, b, P, n, s)) return -1;
        }
        for (int i = 0; i < n; ++i) { x[i] = s[i]; blocked[i] = 0; }
        for (int i = 0; i < n; ++i) {
            double v = b[i];
            for (int k = 0; k < n; ++k) v -= A[i * n + k] * x[k];
            w[i] = v;
        }
    }
    return -1;
}

/* One multi-component vector: columns, PSF (Eq. 3), weights (R8), the
 * normal equations A = M^T W M, b = M^T W d, FNNLS amplitudes, then chi^2
 * by a direct pass over the pixels and log L (Eq. 5).  Optional outputs:
 * the blurred columns [nc][npix], the amplitudes [nc], the blurred model.
 * Returns -INFINITY for an invalid vector. */
double ora_loglike_multi(const ora_lens *L, const ora_comp_spec *c, int nc,
                         const double *p, double *cols_out, double *amps_out,
                         double *model_out)
{
    ora_mmodel m;
    int npix = L->ny * L->nx;
    if (ora_decode_multi(p, c, nc, L->mass, &m)) return -INFINITY;
    double *u = malloc(sizeof(double) * npix * nc), *mc = malloc(sizeof(double) * npix * nc);
    double *w = malloc(sizeof(double) * npix), *psf = malloc(sizeof(double) * L->k * L->k);
    double *mod = malloc(sizeof(double) * npix);
    double res = -INFINITY;
    if (!u || !mc || !w || !psf || !mod) goto done;
    if (ora_psf_normalise(L->psf, L->k, psf)) goto done;
    ora_multi_columns(&m, L->ny, L->nx, L->dpix, L->sub, L->x0, L->y0, u);
    for (int k = 0; k < nc; ++k)
        ora_convolve(u + (size_t)k * npix, L->ny, L->nx, psf, L->k, mc + (size_t)k * npix);
    ora_weights(L->data, L->sigma, npix, w);
    double A[ORA_MAXC * ORA_MAXC] = {0}, b[ORA_MAXC] = {0}, x[ORA_MAXC];
    for (int a = 0; a < nc; ++a) {
        const double *ma = mc + (size_t)a * npix;
        /* masked pixels (R8) carry no term: skipped, not weighted by 0, since
         * their datum may be non-finite and 0 * NaN is NaN */
        for (int t = 0; t < npix; ++t)
            if (w[t] != 0.0) b[a] += w[t] * ma[t] * L->data[t];
        for (int e = 0; e < nc; ++e) {
            const double *me = mc + (size_t)e * npix;
            double v = 0.0;
            for (int t = 0; t < npix; ++t) v += w[t] * ma[t] * me[t];
            A[a * nc + e] = v;
        }
    }
    ora_fnnls(A, b, nc, x);
    double chi2 = 0.0, norm = 0.0;
    for (int t = 0; t < npix; ++t) {
        double mv = 0.0;
        for (int k = 0; k < nc; ++k) mv += x[k] * mc[(size_t)k * npix + t];
        mod[t] = mv;
        if (w[t] == 0.0) continue;
        double r = L->data[t] - mv;
        chi2 += w[t] * r * r;
        norm += log(2.0 * M_PI / w[t]);
    }
    res = -0.5 * chi2 - 0.5 * norm;
    if (cols_out) memcpy(cols_out, mc, sizeof(double) * npix * nc);
    if (amps_out) memcpy(amps_out, x, sizeof(double) * nc);
    if (model_out) memcpy(model_out, mod, sizeof(double) * npix);
done:
    free(u); free(mc); free(w); free(psf); free(mod);
    return res;
}

/* Unblurred multi-component columns [nc][npix]; -1 for an invalid vector. */
int ora_multi_unblurred(const ora_lens *L, const ora_comp_spec *c, int nc,
                        const double *p, double *cols)
{
    ora_mmodel m;
    if (ora_decode_multi(p, c, nc, L->mass, &m)) return -1;
    ora_multi_columns(&m, L->ny, L->nx, L->dpix, L->sub, L->x0, L->y0, cols);
    return 0;
}

/* Batch of B multi-component vectors (row-major [B][nparam]); parallel over
 * vectors only. */
void ora_loglike_multi_batch(const ora_lens *L, const ora_comp_spec *c, int nc,
                             const double *params, int B, double *out, int nthreads)
{
    const int np = ora_multi_nparam(c, nc, L->mass);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b)
        out[b] = np < 0 ? -INFINITY
                        : ora_loglike_multi(L, c, nc, params + (size_t)b * np, NULL, NULL, NULL);
    (void)nthreads;
}

/* ================================================================
 * A sampler loop: the affine-invariant ensemble "stretch move".
 *
 * The paper's sampler (nautilus) runs on the CPU and calls the GPU
 * likelihood for batches of proposals; it names that host round trip as the
 * bottleneck and proposes moving the sampler onto the GPU (Sec. 4.2).  The
 * library's device-side loop runs the stretch move of Goodman & Weare
 * (2010); this is that move written out plainly, for the tests.  Random
 * numbers come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011), a
 * counter-based generator, so both sides draw the same numbers from the
 * same (key, counter).
 *
 * One step updates the two halves of the ensemble of W walkers in turn
 * (half 0 = walkers [0, W/2), half 1 = [W/2, W)).  For walker k of half h,
 * with Philox outputs r0..r3 at key (seed low, seed high) and counter
 * (k, h, step low, step high):
 *   partner  j = (other half's first walker) + floor(r0 (W/2) / 2^32)
 *   stretch  u = (r1 + 1/2) 2^-32, z = ((a - 1) u + 1)^2 / a, which has the
 *            density g(z) ~ 1/sqrt(z) on [1/a, a]
 *   proposal Y = x_j + z (x_k - x_j), in FP64 from the float32 walkers,
 *            rounded once to float32
 *   accept   when log((r2 + 1/2) 2^-32) < (ndim - 1) log z + lp(Y) - lp(x_k)
 *            and every free coordinate of Y lies in [lo, hi] (a uniform
 *            box prior; coordinates with lo == hi are fixed).
 * Every FP64 operation here is a single rounded operation (this file is
 * compiled without contraction), so the proposals are reproducible bit for
 * bit by another implementation that rounds the same way.
 * ================================================================ */
#include <stdint.h>

/* Philox4x32-10: ten rounds of the Philox S-box on a 128-bit counter with a
 * 64-bit key (Salmon et al. 2011, Sec. 5): each round multiplies counter
 * words 0 and 2 by the two round multipliers, takes the high and low
 * halves of the 64-bit products, and mixes them with the other two words
 * and the key; the key advances by the two Weyl constants between rounds. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The four Philox outputs of walker k, half h, at `step`. */
static void ora_walker_rng(uint64_t seed, long long step, int h, int k, uint32_t r[4])
{
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)h, (uint32_t)((uint64_t)step & 0xffffffffu),
                       (uint32_t)((uint64_t)step >> 32)};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    ora_philox4x32_10(ctr, key, r);
}

/* Proposals of half h: Y[k - h W/2][P] (float32), the stretch factors z and
 * the partners j of walkers k of that half. */
void ora_stretch_propose(const float *x, int W, int P, int h, long long step, uint64_t seed,
                         double a, float *Y, double *z_out, int *j_out)
{
    const int half = W / 2, first = h * half, other = (1 - h) * half;
    for (int t = 0; t < half; ++t) {
        const int k = first + t;
        uint32_t r[4];
        ora_walker_rng(seed, step, h, k, r);
        const int j = other + (int)(((uint64_t)r[0] * (uint64_t)half) >> 32);
        const double u = ((double)r[1] + 0.5) * 2.3283064365386963e-10;
        const double w = (a - 1.0) * u + 1.0;
        const double z = w * w / a;
        for (int i = 0; i < P; ++i) {
            const double xj = x[(size_t)j * P + i], xk = x[(size_t)k * P + i];
            const double d = xk - xj;
            const double t2 = z * d;
            Y[(size_t)t * P + i] = (float)(xj + t2);
        }
        z_out[t] = z;
        j_out[t] = j;
    }
}

/* Accept / reject half h given the proposals' log posterior lpY (the caller
 * evaluates them); updates x and lp in place and writes acc[t] = 1 for an
 * accepted move.  Returns the number accepted. */
int ora_stretch_accept(float *x, double *lp, int W, int P, int h, long long step,
                       uint64_t seed, int ndim, const float *Y, const double *z,
                       const double *lpY, const float *lo, const float *hi, int *acc)
{
    const int half = W / 2, first = h * half;
    int n = 0;
    for (int t = 0; t < half; ++t) {
        const int k = first + t;
        uint32_t r[4];
        ora_walker_rng(seed, step, h, k, r);
        int inside = 1;
        for (int i = 0; i < P; ++i) {
            const float v = Y[(size_t)t * P + i];
            if (lo[i] < hi[i] && !(v >= lo[i] && v <= hi[i])) inside = 0;
        }
        const double lpy = inside ? lpY[t] : -INFINITY;
        const double lu = log(((double)r[2] + 0.5) * 2.3283064365386963e-10);
        const double rhs = (ndim - 1) * log(z[t]) + lpy - lp[k];
        acc[t] = lu < rhs;
        if (acc[t]) {
            for (int i = 0; i < P; ++i) x[(size_t)k * P + i] = Y[(size_t)t * P + i];
            lp[k] = lpy;
            ++n;
        }
    }
    return n;
}
