/*
 * cwthf_oracle.c -- plain, slow, fp64 CPU statement of the single-scale
 * CWTHF halo-finding path (arXiv:2501.10622).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the CUDA
 * library under paper_2501_10622_gb300/.  Only the tests, the smoke check and
 * the CPU-baseline leg of bench.py may load it.  It shares no source, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Each function states the definition it follows.  No blocking, fusion or
 * reordering beyond what the definition needs: loops run over cells and
 * particles in index order.
 *
 *   Sec. 2 (step list): the order of the stages (deposit, CWT, maxima,
 *       segmentation, particle assignment, density / particle thresholds).
 *   Sec. 2.1, Eq. 1: cloud-in-cell (CIC) deposit onto grid nodes.
 *   Sec. 2.1, Eq. 2-3: grid CWT = sum over nodes of m_g Psi(w, x - x_g).
 *   Sec. 2.1, Eq. 4: the isotropic 3D Mexican-hat wavelet.
 *   Sec. 2.3: the self-boundness check (orc_unbind: spherical shell
 *       potential, escape speed, iterative exclusion, the 40 % rule).
 *   Sec. 2.3: halo = region around a positive CWT peak, extended down to
 *       the CWT valley; halo centre = centre of mass.
 *   Sec. 2.4 and Table 1: density threshold dens_th (4 x mean density,
 *       grid volume of the segment) and particle threshold particle_th (15).
 *
 * Readings where the paper is silent (every one is also listed in the
 * design notes of the repository):
 *   - grid nodes sit at x_g = g * (L/N), periodic box;
 *   - positions are quantised to F = 10 fractional bits of a cell before the
 *     CIC weights are formed, so every weight product is an exact integer;
 *   - the wavelet is sampled at per-axis minimum-image offsets over the whole
 *     box, so the CWT is the circular convolution of the CIC mass with it;
 *   - maxima are over the 26 periodic neighbours under the strict total order
 *     (C[a] > C[b]) or (C[a] == C[b] and a < b), a, b linear cell indices;
 *   - "segmentation" follows steepest ascent: every cell points at the best
 *     cell of itself + its 26 neighbours under that order; a chain ends at a
 *     maximum; maxima with C > cwt_min seed halos, the rest label -1;
 *   - a particle belongs to the segment of its nearest grid node;
 *   - centres are mass-weighted minimum-image offsets of the quantised
 *     positions about the seed node.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "cwthf_oracle.h"

#define FRAC_BITS 10
#define FRAC_ONE (1LL << FRAC_BITS)
#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Quantisation (reading of Sec. 2.1: positions to F fractional cell bits).  */
/* ------------------------------------------------------------------------ */

/* Fixed-point coordinate of one float coordinate: floor(x * s) wrapped into
 * [0, N * 2^F), with s the quantisation scale below.  Because s has at most
 * 29 significant bits and a float has 24, the fp64 product x*s is exact, so
 * this is the floor of the exact product.  Returns 0 on success, ORC_E_ARG if
 * x is not finite or |x*s| >= 2^40. */
static int quantise_coord(float x, double scale, int64_t modulus, int64_t *q) {
    double t = (double)x * scale;
    if (!isfinite(t) || fabs(t) >= 1099511627776.0) return ORC_E_ARG;
    int64_t v = (int64_t)floor(t);
    v %= modulus;
    if (v < 0) v += modulus;
    *q = v;
    return ORC_OK;
}

/* The scale N * 2^F / L: the fp64 quotient N/L times 2^F (exact), rounded to
 * 29 significant bits (round half to even). */
static double quant_scale(int ng, double L) {
    double s = ((double)ng / L) * (double)FRAC_ONE;
    int e;
    double f = frexp(s, &e); /* s = f 2^e, 0.5 <= f < 1 */
    return ldexp(nearbyint(ldexp(f, 29)), e - 29);
}

int orc_quantise(const float *pos, int64_t np, double L, int ng, int64_t *q) {
    if (ng < 1 || !(L > 0)) return ORC_E_ARG;
    double s = quant_scale(ng, L);
    int64_t mod = (int64_t)ng * FRAC_ONE;
    for (int64_t i = 0; i < np; i++)
        for (int a = 0; a < 3; a++) {
            int rc = quantise_coord(pos[3 * i + a], s, mod, &q[3 * i + a]);
            if (rc) return rc;
        }
    return ORC_OK;
}

/* Integer mass of one particle: 1 when masses are all equal (mass == NULL),
 * else rint(m / mass_unit), round half to even.  Valid range [0, 2^31). */
static int mass_quantum(const float *mass, double mass_unit, int64_t i, int64_t *mq) {
    if (!mass) { *mq = 1; return ORC_OK; }
    double r = rint((double)mass[i] / mass_unit);
    if (!(r >= 0.0) || r >= 2147483648.0) return ORC_E_ARG;
    *mq = (int64_t)r;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1, Eq. 1: cloud-in-cell deposit.                                   */
/* ------------------------------------------------------------------------ */

/* Each particle with fixed-point coordinate q = i*2^F + f (0 <= f < 2^F) per
 * axis gives node i the weight (2^F - f) and node i+1 (mod N) the weight f;
 * the 3D weight is the product over axes.  The mass m_q * wx*wy*wz is
 * accumulated in fp64: every term and every partial sum is an integer, exact
 * while below 2^53, which is checked.  The result is the grid in units of
 * mass_unit * 2^-3F.  *mtot_q receives sum_i m_q (< 2^33 required so that no
 * cell can reach 2^63). */
int orc_cic(const float *pos, const float *mass, double mass_unit, int64_t np, double L, int ng,
            int64_t *grid, int64_t *mtot_q) {
    if (ng < 1 || !(L > 0) || np < 0 || !(mass_unit > 0)) return ORC_E_ARG;
    int64_t ncell = (int64_t)ng * ng * ng;
    double *acc = calloc((size_t)ncell, sizeof(double));
    if (!acc) return ORC_E_NOMEM;
    double s = quant_scale(ng, L);
    int64_t mod = (int64_t)ng * FRAC_ONE;
    int64_t total = 0;
    int rc = ORC_OK;
    for (int64_t p = 0; p < np && rc == ORC_OK; p++) {
        int64_t q[3], mq;
        for (int a = 0; a < 3 && rc == ORC_OK; a++) rc = quantise_coord(pos[3 * p + a], s, mod, &q[a]);
        if (rc == ORC_OK) rc = mass_quantum(mass, mass_unit, p, &mq);
        if (rc) break;
        total += mq;
        if (total >= (1LL << 33)) { rc = ORC_E_OVERFLOW; break; }
        int64_t node[3][2];
        double wgt[3][2];
        for (int a = 0; a < 3; a++) {
            int64_t i = q[a] >> FRAC_BITS, f = q[a] & (FRAC_ONE - 1);
            node[a][0] = i;
            node[a][1] = (i + 1) % ng;
            wgt[a][0] = (double)(FRAC_ONE - f);
            wgt[a][1] = (double)f;
        }
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < 2; dy++)
                for (int dx = 0; dx < 2; dx++) {
                    double contrib = (double)mq * wgt[0][dx] * wgt[1][dy] * wgt[2][dz];
                    int64_t c = (node[2][dz] * ng + node[1][dy]) * ng + node[0][dx];
                    acc[c] += contrib;
                }
    }
    if (rc == ORC_OK) {
        for (int64_t c = 0; c < ncell; c++) {
            if (acc[c] >= 9007199254740992.0) { rc = ORC_E_INEXACT; break; }
            grid[c] = (int64_t)acc[c];
        }
        if (mtot_q) *mtot_q = total;
    }
    free(acc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1, Eq. 4: the isotropic Mexican-hat wavelet in 3D.                 */
/* ------------------------------------------------------------------------ */

double orc_wavelet(double w, double r2) {
    double a = w * w * r2;
    return pow(w, 1.5) * (6.0 - a) * exp(-0.25 * a);
}

/* Minimum-image offset of index n on a periodic axis of length N:
 * n for n <= N/2, n - N above. */
static int64_t min_image(int64_t n, int ng) { return (2 * n <= ng) ? n : n - ng; }

/* The wavelet sampled on the grid spacing at minimum-image offsets:
 * K[n] = Psi(w, dx * |d(n)|), d(n) per axis.  Sec. 2.1 samples the wavelet
 * with the same spacing as the CIC grid before accumulating it. */
void orc_kernel(int ng, double L, double w, double *K) {
    double dx = L / ng;
    for (int64_t z = 0; z < ng; z++)
        for (int64_t y = 0; y < ng; y++)
            for (int64_t x = 0; x < ng; x++) {
                double ox = dx * (double)min_image(x, ng), oy = dx * (double)min_image(y, ng),
                       oz = dx * (double)min_image(z, ng);
                K[(z * ng + y) * ng + x] = orc_wavelet(w, ox * ox + oy * oy + oz * oz);
            }
}

/* ------------------------------------------------------------------------ */
/* Textbook mixed-radix Cooley-Tukey DFT (decimation in time), fp64.         */
/* X[k] = sum_n x[n] exp(sign * 2 pi i n k / n_len), unnormalised.           */
/* ------------------------------------------------------------------------ */

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

/* Roots of unity exp(-2 pi i e / n) for one top-level length n, fp64. */
typedef struct {
    int n;
    double complex *w;
} roots_t;

static int roots_init(roots_t *r, int n) {
    r->n = n;
    r->w = malloc(sizeof(double complex) * (size_t)n);
    if (!r->w) return ORC_E_NOMEM;
    for (int e = 0; e < n; e++) {
        double ang = TWO_PI * (double)e / (double)n;
        r->w[e] = cos(ang) - sin(ang) * I;
    }
    return ORC_OK;
}

/* exp(sign * 2 pi i e / m) for a length m that divides the table's length. */
static double complex unit_root(const roots_t *r, int sign, int64_t e, int m) {
    double complex v = r->w[(e % m) * (r->n / m)];
    return sign < 0 ? v : conj(v);
}

/* x: input with element stride `stride`; X: n outputs; scratch: n entries. */
static void dft_rec(const double complex *x, int64_t stride, int n, double complex *X, int sign,
                    double complex *scratch, const roots_t *roots) {
    if (n == 1) { X[0] = x[0]; return; }
    int p = smallest_factor(n), m = n / p;
    /* Y_r = DFT_m of x[r + p j], j = 0..m-1, stored in X[r m .. r m + m). */
    for (int r = 0; r < p; r++) dft_rec(x + r * stride, stride * p, m, X + (int64_t)r * m, sign, scratch, roots);
    /* X[k] = sum_r w_n^{r k} Y_r[k mod m]. */
    for (int k = 0; k < n; k++) {
        double complex acc = 0;
        for (int r = 0; r < p; r++) acc += unit_root(roots, sign, (int64_t)r * k, n) * X[(int64_t)r * m + k % m];
        scratch[k] = acc;
    }
    memcpy(X, scratch, sizeof(double complex) * (size_t)n);
}

/* In-place 1D DFT of n complex values (re, im separate arrays, unit stride). */
int orc_dft1d(double *re, double *im, int n, int sign) {
    if (n < 1 || (sign != 1 && sign != -1)) return ORC_E_ARG;
    double complex *in = malloc(sizeof(double complex) * (size_t)n * 3);
    if (!in) return ORC_E_NOMEM;
    double complex *out = in + n, *scr = in + 2 * n;
    roots_t roots;
    if (roots_init(&roots, n)) { free(in); return ORC_E_NOMEM; }
    for (int i = 0; i < n; i++) in[i] = re[i] + im[i] * I;
    dft_rec(in, 1, n, out, sign, scr, &roots);
    for (int i = 0; i < n; i++) { re[i] = creal(out[i]); im[i] = cimag(out[i]); }
    free(roots.w);
    free(in);
    return ORC_OK;
}

/* In-place 3D DFT of an n^3 complex array [z][y][x], applied axis by axis. */
static int dft3d(double complex *a, int n, int sign) {
    double complex *line = malloc(sizeof(double complex) * (size_t)n * 3);
    if (!line) return ORC_E_NOMEM;
    double complex *out = line + n, *scr = line + 2 * n;
    roots_t roots;
    if (roots_init(&roots, n)) { free(line); return ORC_E_NOMEM; }
    int64_t n2 = (int64_t)n * n;
    for (int axis = 0; axis < 3; axis++) {
        int64_t step = axis == 0 ? 1 : axis == 1 ? n : n2;
        for (int64_t u = 0; u < n; u++)
            for (int64_t v = 0; v < n; v++) {
                int64_t base = axis == 0 ? (u * n + v) * n : axis == 1 ? u * n2 + v : u * n + v;
                for (int i = 0; i < n; i++) line[i] = a[base + i * step];
                dft_rec(line, 1, n, out, sign, scr, &roots);
                for (int i = 0; i < n; i++) a[base + i * step] = out[i];
            }
    }
    free(roots.w);
    free(line);
    return ORC_OK;
}

int orc_dft3d(double *re, double *im, int n, int sign) {
    if (n < 1 || (sign != 1 && sign != -1)) return ORC_E_ARG;
    int64_t cells = (int64_t)n * n * n;
    double complex *a = malloc(sizeof(double complex) * (size_t)cells);
    if (!a) return ORC_E_NOMEM;
    for (int64_t c = 0; c < cells; c++) a[c] = re[c] + im[c] * I;
    int rc = dft3d(a, n, sign);
    for (int64_t c = 0; c < cells; c++) { re[c] = creal(a[c]); im[c] = cimag(a[c]); }
    free(a);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1, Eq. 2-3: grid CWT of the CIC mass.                              */
/* ------------------------------------------------------------------------ */

/* CIC mass of each node in physical units: grid * mass_unit * 2^-3F. */
static double node_mass(const int64_t *grid, int64_t c, double mass_unit) {
    return (double)grid[c] * (mass_unit / (double)(1LL << (3 * FRAC_BITS)));
}

/* C(x_g) = sum_g' m_g' Psi(w, x_g - x_g'), evaluated as the circular
 * convolution of the node masses with the sampled kernel K through the DFT:
 * C = IDFT(DFT(m) * DFT(K)) / N^3. */
int orc_cwt(const int64_t *grid, int ng, double L, double mass_unit, double w, double *C) {
    if (ng < 1 || !(L > 0) || !(w > 0) || !(mass_unit > 0)) return ORC_E_ARG;
    int64_t cells = (int64_t)ng * ng * ng;
    double complex *m = malloc(sizeof(double complex) * (size_t)cells);
    double complex *k = malloc(sizeof(double complex) * (size_t)cells);
    double *K = malloc(sizeof(double) * (size_t)cells);
    int rc = (m && k && K) ? ORC_OK : ORC_E_NOMEM;
    if (rc == ORC_OK) {
        orc_kernel(ng, L, w, K);
        for (int64_t c = 0; c < cells; c++) { m[c] = node_mass(grid, c, mass_unit); k[c] = K[c]; }
        rc = dft3d(m, ng, -1);
        if (rc == ORC_OK) rc = dft3d(k, ng, -1);
        if (rc == ORC_OK) {
            for (int64_t c = 0; c < cells; c++) m[c] *= k[c];
            rc = dft3d(m, ng, +1);
        }
        if (rc == ORC_OK)
            for (int64_t c = 0; c < cells; c++) C[c] = creal(m[c]) / (double)cells;
    }
    free(m); free(k); free(K);
    return rc;
}

/* Eq. 2 evaluated literally: for every node x, the sum over every node g of
 * m_g Psi(w, x - g) with the minimum-image separation.  O(N^6): tiny grids. */
int orc_cwt_direct(const int64_t *grid, int ng, double L, double mass_unit, double w, double *C) {
    if (ng < 1 || !(L > 0) || !(w > 0) || !(mass_unit > 0)) return ORC_E_ARG;
    double dx = L / ng;
    for (int64_t z = 0; z < ng; z++)
        for (int64_t y = 0; y < ng; y++)
            for (int64_t x = 0; x < ng; x++) {
                double s = 0.0;
                for (int64_t gz = 0; gz < ng; gz++)
                    for (int64_t gy = 0; gy < ng; gy++)
                        for (int64_t gx = 0; gx < ng; gx++) {
                            int64_t g = (gz * ng + gy) * ng + gx;
                            if (grid[g] == 0) continue;
                            double ox = dx * (double)min_image(((x - gx) % ng + ng) % ng, ng);
                            double oy = dx * (double)min_image(((y - gy) % ng + ng) % ng, ng);
                            double oz = dx * (double)min_image(((z - gz) % ng + ng) % ng, ng);
                            s += node_mass(grid, g, mass_unit) * orc_wavelet(w, ox * ox + oy * oy + oz * oz);
                        }
                C[(z * ng + y) * ng + x] = s;
            }
    return ORC_OK;
}

/* Eq. 2 evaluated literally at chosen nodes only: for each requested node x,
 * the sum over every node g of m_g Psi(w, x - g) (minimum-image separation).
 * Terms whose separation has w^2 r^2 > 3000 are exactly zero in fp64 (the
 * factor exp(-w^2 r^2 / 4) underflows to 0), so the loops visit only the
 * offsets within that support (every offset once, also on small grids);
 * the result is the full sum up to the order of the additions.  Cost per
 * node: the support, not N^3. */
/* Sec. 2.1 as the paper evaluates it: the CIC grid's pseudo-particles each add
 * their mass times the wavelet sampled on the grid around them, over a
 * truncated stencil.  Here the stencil is the cube of offsets d with
 * |d_x|, |d_y|, |d_z| <= R (R = gdw_resolution of Table 1 read as a radius),
 * periodic:  C(g) = sum_{d in cube} m(g - d) Psi(w, Delta |d|).  Literal sum,
 * fp64; 2R + 1 <= ng, so that no node is counted twice. */
int orc_cwt_stencil(const int64_t *grid, int ng, double L, double mass_unit, double w, int R, double *C) {
    if (ng < 1 || !(L > 0) || !(w > 0) || !(mass_unit > 0) || R < 0 || 2 * (int64_t)R + 1 > ng) return ORC_E_ARG;
    const double dx = L / ng;
    const int64_t side = 2 * (int64_t)R + 1;
    double *psi = malloc(sizeof(double) * (size_t)(side * side * side));
    if (!psi) return ORC_E_NOMEM;
    for (int64_t dz = -R; dz <= R; dz++)
        for (int64_t dy = -R; dy <= R; dy++)
            for (int64_t dxo = -R; dxo <= R; dxo++) {
                double ox = dx * (double)dxo, oy = dx * (double)dy, oz = dx * (double)dz;
                psi[((dz + R) * side + (dy + R)) * side + (dxo + R)] = orc_wavelet(w, ox * ox + oy * oy + oz * oz);
            }
    for (int64_t z = 0; z < ng; z++)
        for (int64_t y = 0; y < ng; y++)
            for (int64_t x = 0; x < ng; x++) {
                double s = 0.0;
                for (int64_t dz = -R; dz <= R; dz++)
                    for (int64_t dy = -R; dy <= R; dy++)
                        for (int64_t dxo = -R; dxo <= R; dxo++) {
                            int64_t gx = ((x - dxo) % ng + ng) % ng, gy = ((y - dy) % ng + ng) % ng,
                                    gz = ((z - dz) % ng + ng) % ng;
                            int64_t g = (gz * ng + gy) * ng + gx;
                            if (grid[g] == 0) continue;
                            s += node_mass(grid, g, mass_unit) * psi[((dz + R) * side + (dy + R)) * side + (dxo + R)];
                        }
                C[(z * ng + y) * ng + x] = s;
            }
    free(psi);
    return ORC_OK;
}

/* The stencil sum of orc_cwt_stencil at the given linear node indices only
 * (full-size spot checks). */
int orc_cwt_stencil_at(const int64_t *grid, int ng, double L, double mass_unit, double w, int R, const int64_t *nodes,
                       int64_t n_nodes, double *out) {
    if (ng < 1 || !(L > 0) || !(w > 0) || !(mass_unit > 0) || R < 0 || 2 * (int64_t)R + 1 > ng || n_nodes < 0)
        return ORC_E_ARG;
    const double dx = L / ng;
    const int64_t cells = (int64_t)ng * ng * ng;
    for (int64_t i = 0; i < n_nodes; i++) {
        int64_t c = nodes[i];
        if (c < 0 || c >= cells) return ORC_E_ARG;
        int64_t x = c % ng, y = (c / ng) % ng, z = c / ((int64_t)ng * ng);
        double s = 0.0;
        for (int64_t dz = -R; dz <= R; dz++)
            for (int64_t dy = -R; dy <= R; dy++)
                for (int64_t dxo = -R; dxo <= R; dxo++) {
                    int64_t gx = ((x - dxo) % ng + ng) % ng, gy = ((y - dy) % ng + ng) % ng,
                            gz = ((z - dz) % ng + ng) % ng;
                    int64_t g = (gz * ng + gy) * ng + gx;
                    if (grid[g] == 0) continue;
                    double ox = dx * (double)dxo, oy = dx * (double)dy, oz = dx * (double)dz;
                    s += node_mass(grid, g, mass_unit) * orc_wavelet(w, ox * ox + oy * oy + oz * oz);
                }
        out[i] = s;
    }
    return ORC_OK;
}

int orc_cwt_at(const int64_t *grid, int ng, double L, double mass_unit, double w, const int64_t *nodes,
               int64_t n_nodes, double *out) {
    if (ng < 1 || !(L > 0) || !(w > 0) || !(mass_unit > 0) || n_nodes < 0) return ORC_E_ARG;
    const double dx = L / ng;
    const int64_t cells = (int64_t)ng * ng * ng;
    /* offsets d in [-R, R] per axis, capped so that no node is visited twice */
    int64_t R = (int64_t)ceil(sqrt(3000.0) / (w * dx));
    int64_t lo = -(int64_t)(ng / 2) + (ng % 2 == 0 ? 1 : 0), hi = ng / 2; /* ng consecutive offsets */
    int64_t dlo = -R < lo ? lo : -R, dhi = R > hi ? hi : R;
    for (int64_t i = 0; i < n_nodes; i++) {
        int64_t c = nodes[i];
        if (c < 0 || c >= cells) return ORC_E_ARG;
        int64_t x = c % ng, y = (c / ng) % ng, z = c / ((int64_t)ng * ng);
        double s = 0.0;
        for (int64_t dz = dlo; dz <= dhi; dz++)
            for (int64_t dy = dlo; dy <= dhi; dy++)
                for (int64_t dxo = dlo; dxo <= dhi; dxo++) {
                    /* node g = x - d; its minimum-image separation from x is d itself
                       (d lies in the minimum-image range) */
                    int64_t gx = ((x - dxo) % ng + ng) % ng, gy = ((y - dy) % ng + ng) % ng,
                            gz = ((z - dz) % ng + ng) % ng;
                    int64_t g = (gz * ng + gy) * ng + gx;
                    if (grid[g] == 0) continue;
                    double ox = dx * (double)min_image((dxo % ng + ng) % ng, ng);
                    double oy = dx * (double)min_image((dy % ng + ng) % ng, ng);
                    double oz = dx * (double)min_image((dz % ng + ng) % ng, ng);
                    s += node_mass(grid, g, mass_unit) * orc_wavelet(w, ox * ox + oy * oy + oz * oz);
                }
        out[i] = s;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 step 4 and Sec. 2.3: local maxima and steepest-ascent segments.    */
/* ------------------------------------------------------------------------ */

/* Strict total order on cells: a beats b iff C[a] > C[b], or equal values
 * and a has the smaller linear index. */
static int beats(const float *C, int64_t a, int64_t b) {
    return C[a] > C[b] || (C[a] == C[b] && a < b);
}

/* parent[c] = the best cell of {c} and its 26 periodic neighbours.
 * A cell is a local maximum iff parent[c] == c. */
int orc_parent(const float *C, int ng, int32_t *parent) {
    if (ng < 3) return ORC_E_ARG;
    int64_t cells = (int64_t)ng * ng * ng;
    for (int64_t c = 0; c < cells; c++)
        if (isnan(C[c])) return ORC_E_ARG;
    for (int64_t z = 0; z < ng; z++)
        for (int64_t y = 0; y < ng; y++)
            for (int64_t x = 0; x < ng; x++) {
                int64_t c = (z * ng + y) * ng + x, best = c;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            int64_t n = (((z + dz + ng) % ng) * ng + (y + dy + ng) % ng) * ng + (x + dx + ng) % ng;
                            if (beats(C, n, best)) best = n;
                        }
                parent[c] = (int32_t)best;
            }
    return ORC_OK;
}

/* label[c] = the maximum reached by walking parent pointers from c, if that
 * maximum's value exceeds cwt_min (a seed: Sec. 2.3 takes halos around
 * positive CWT peaks), else -1.
 * The walk is sequential, one cell at a time. */
int orc_segment(const float *C, int ng, float cwt_min, int32_t *label) {
    int64_t cells = (int64_t)ng * ng * ng;
    int32_t *parent = malloc(sizeof(int32_t) * (size_t)cells);
    if (!parent) return ORC_E_NOMEM;
    int rc = orc_parent(C, ng, parent);
    if (rc == ORC_OK) {
        for (int64_t c = 0; c < cells; c++) {
            int64_t r = c, steps = 0;
            while (parent[r] != r) {
                r = parent[r];
                if (++steps > cells) { rc = ORC_E_ARG; break; }
            }
            label[c] = (C[r] > cwt_min) ? (int32_t)r : -1;
        }
    }
    free(parent);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 steps 6-7, Sec. 2.3-2.4, Table 1: particle assignment, per-halo    */
/* sums, density and particle thresholds, catalogue.                         */
/* ------------------------------------------------------------------------ */

/* Minimum-image fixed-point offset in [-M/2, M/2) on an axis of M units. */
static int64_t min_image_q(int64_t d, int64_t M) {
    d %= M;
    if (d < 0) d += M;
    if (2 * d >= M) d -= M;
    return d;
}

/* For every particle: nearest node (q + 2^(F-1)) >> F per axis, wrapped, and
 * the label of that node.  Per seed: number of particles, integer mass
 * sum_i m_q, integer first moment sum_i m_q * (q_i - seed*2^F) (minimum image)
 * and the number of cells carrying its label.  A seed is kept as a halo iff
 *   n_part >= particle_th   and
 *   mass / (n_cells * cell volume) >= dens_th * total mass / box volume,
 * evaluated as (double)mq * (double)N^3 >= (dens_th * (double)Mtot) * (double)n_cells.
 * Kept halos are written in increasing seed order; halo_id[i] is the seed of
 * the particle's halo or -1.  Outputs per halo: seed, n_part, n_cells, mass
 * (sum m_q * mass_unit), centre[3] (wrapped into [0, L)), peak = C[seed].
 * *n_halo receives the number of kept halos (cap: at most that many are
 * written; ORC_E_CAPACITY if more exist). */
int orc_assign(const float *pos, const float *mass, double mass_unit, int64_t np, double L, int ng,
               const int32_t *label, const float *C, double dens_th, int64_t particle_th,
               int32_t *halo_id, int64_t cap, int64_t *seed_out, int64_t *npart_out, int64_t *ncell_out,
               double *mass_out, double *centre_out, float *peak_out, int64_t *n_halo) {
    if (ng < 1 || !(L > 0) || np < 0 || !(mass_unit > 0)) return ORC_E_ARG;
    int64_t cells = (int64_t)ng * ng * ng;
    int64_t M = (int64_t)ng * FRAC_ONE;
    double s = quant_scale(ng, L);
    /* per-cell accumulators, indexed by seed cell */
    int64_t *np_c = calloc((size_t)cells, sizeof(int64_t));
    int64_t *mq_c = calloc((size_t)cells, sizeof(int64_t));
    int64_t *mom = calloc((size_t)cells * 3, sizeof(int64_t));
    int64_t *nc_c = calloc((size_t)cells, sizeof(int64_t));
    int32_t *tmp = malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    unsigned char *keepflag = calloc((size_t)cells, 1);
    int rc = (np_c && mq_c && mom && nc_c && tmp && keepflag) ? ORC_OK : ORC_E_NOMEM;
    int64_t mtot = 0;
    for (int64_t c = 0; c < cells && rc == ORC_OK; c++) {
        if (label[c] < -1 || label[c] >= cells) { rc = ORC_E_ARG; break; }
        if (label[c] >= 0) nc_c[label[c]] += 1;
    }
    for (int64_t p = 0; p < np && rc == ORC_OK; p++) {
        int64_t q[3], mq, node[3];
        for (int a = 0; a < 3 && rc == ORC_OK; a++) rc = quantise_coord(pos[3 * p + a], s, M, &q[a]);
        if (rc == ORC_OK) rc = mass_quantum(mass, mass_unit, p, &mq);
        if (rc) break;
        mtot += mq;
        for (int a = 0; a < 3; a++) node[a] = ((q[a] + FRAC_ONE / 2) >> FRAC_BITS) % ng;
        int64_t cell = (node[2] * ng + node[1]) * ng + node[0];
        int32_t lab = label[cell];
        tmp[p] = lab;
        if (lab < 0) continue;
        int64_t sc[3] = {lab % ng, (lab / ng) % ng, lab / ((int64_t)ng * ng)};
        np_c[lab] += 1;
        mq_c[lab] += mq;
        for (int a = 0; a < 3; a++) mom[3 * lab + a] += mq * min_image_q(q[a] - sc[a] * FRAC_ONE, M);
    }
    int64_t kept = 0;
    if (rc == ORC_OK) {
        double ncube = (double)cells;
        double cell_q = (L / (double)ng) / (double)FRAC_ONE;
        for (int64_t c = 0; c < cells; c++) {
            if (label[c] != c) continue; /* seeds are exactly the cells labelled with themselves */
            int keep = np_c[c] >= particle_th &&
                       (double)mq_c[c] * ncube >= (dens_th * (double)mtot) * (double)nc_c[c];
            if (!keep) continue;
            keepflag[c] = 1;
            if (kept < cap) {
                int64_t sc[3] = {c % ng, (c / ng) % ng, c / ((int64_t)ng * ng)};
                seed_out[kept] = c;
                npart_out[kept] = np_c[c];
                ncell_out[kept] = nc_c[c];
                mass_out[kept] = (double)mq_c[c] * mass_unit;
                for (int a = 0; a < 3; a++) {
                    double u = (double)(sc[a] * FRAC_ONE);
                    if (mq_c[c] > 0) u += (double)mom[3 * c + a] / (double)mq_c[c];
                    double x = u * cell_q;
                    if (x >= L) x -= L;
                    else if (x < 0.0) x += L;
                    centre_out[3 * kept + a] = x;
                }
                peak_out[kept] = C ? C[c] : 0.0f;
            }
            kept++;
        }
        for (int64_t p = 0; p < np; p++)
            halo_id[p] = (tmp[p] >= 0 && keepflag[tmp[p]]) ? tmp[p] : -1;
        *n_halo = kept;
        if (kept > cap) rc = ORC_E_CAPACITY;
    }
    free(np_c); free(mq_c); free(mom); free(nc_c); free(tmp); free(keepflag);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 (steps 1-8 and 10 of the step list; the self-boundness check of    */
/* step 9 is not part of this loop), Fig. 1, Sec. 2.2 and App. B, Sec. 2.4:  */
/* the multi-scale identification loop.                                      */
/* ------------------------------------------------------------------------ */

/* App. B, Eq. B1 along one axis.  B is the maximum node with value vb, its
 * two neighbours have values vm and vp; A is the higher and C the lower of
 * the two, and with values measured from C, l1 = v_A - v_C and
 * l2 = v_B - v_C, the quadratic through A, B, C peaks
 * l1^2 / (16 l2 - 8 l1) above B.  Single precision, in this order. */
static float peak_term(float vm, float vb, float vp, float *l1_out, float *l2_out) {
    float va = vm > vp ? vm : vp, vc = vm > vp ? vp : vm;
    float l1 = va - vc, l2 = vb - vc;
    float den = 16.0f * l2 - 8.0f * l1;
    *l1_out = l1;
    *l2_out = l2;
    return den > 0.0f ? (l1 * l1) / den : 0.0f;
}

/* The corrected peak of the maximum at node s of the ng^3 field C (App. B):
 * the node value plus the three axes' quadratic terms (x, y, z in this
 * order), plus, when the next (smaller) scale's grid is finer by the factor
 * ratio = ng / ng_next < 1, the grid-size term
 * (5/16) (2 mean(l2) - mean(l1)) (1 - ratio^2): App. B's cube-average
 * difference with the factor 3/5 removed, as the paper prescribes. */
float orc_corrected_peak(const float *C, int ng, int64_t s, int ng_next) {
    int64_t x = s % ng, y = (s / ng) % ng, z = s / ((int64_t)ng * ng);
    int64_t n = ng;
    float vb = C[s];
    float l1[3], l2[3], t[3];
    int64_t xm = (x + n - 1) % n, xp = (x + 1) % n, ym = (y + n - 1) % n, yp = (y + 1) % n;
    int64_t zm = (z + n - 1) % n, zp = (z + 1) % n;
    t[0] = peak_term(C[(z * n + y) * n + xm], vb, C[(z * n + y) * n + xp], &l1[0], &l2[0]);
    t[1] = peak_term(C[(z * n + ym) * n + x], vb, C[(z * n + yp) * n + x], &l1[1], &l2[1]);
    t[2] = peak_term(C[(zm * n + y) * n + x], vb, C[(zp * n + y) * n + x], &l1[2], &l2[2]);
    float p = ((vb + t[0]) + t[1]) + t[2];
    if (ng_next > 0) {
        float r = (float)ng / (float)ng_next;
        float m1 = ((l1[0] + l1[1]) + l1[2]) / 3.0f, m2 = ((l2[0] + l2[1]) + l2[2]) / 3.0f;
        p = p + (5.0f / 16.0f) * (2.0f * m2 - m1) * (1.0f - r * r);
    }
    return p;
}

/* Sec. 2 (Fig. 1): a maximum of the current scale is a maximum in 4D iff its
 * corrected peak exceeds every node of the next (smaller) scale's field near
 * the same physical position: the 2 x 2 x 2 nodes of that grid enclosing the
 * node's position s * L / ng.  With no next scale (the last one) the
 * comparison is with a zero field. */
int orc_cross_scale(const float *C, int ng, int64_t s, const float *Cn, int ng_next) {
    float p = orc_corrected_peak(C, ng, s, ng_next);
    if (!Cn || ng_next <= 0) return p > 0.0f;
    int64_t c[3] = {s % ng, (s / ng) % ng, s / ((int64_t)ng * ng)};
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = (c[a] * ng_next) / ng; /* floor of the position in next-grid cells */
        hi[a] = (lo[a] + 1) % ng_next;
    }
    int64_t m = ng_next;
    for (int k = 0; k < 8; k++) {
        int64_t gx = (k & 1) ? hi[0] : lo[0], gy = (k & 2) ? hi[1] : lo[1], gz = (k & 4) ? hi[2] : lo[2];
        if (!(p > Cn[(gz * m + gy) * m + gx])) return 0;
    }
    return 1;
}

/* The loop of Fig. 1 on given fields: fields[j] is the fp32 CWT of scale j
 * on an ngs[j]^3 grid, scales ordered from the largest physical scale
 * (smallest k_w) to the smallest.  Scale j is processed with scale j + 1 as
 * its "current_grid" (a zero field after the last scale):
 *   segments of fields[j] (orc_segment, seeds above cwt_min);
 *   groups: the particles that hold no halo id yet, by the label of their
 *     nearest node; per group n_part, integer mass, first moment about the
 *     seed; n_cells = cells of the segment;
 *   keep a group iff n_part >= particle_th, mass / (n_cells cell volume) >=
 *     dens_th * (total mass / box volume) (same operands as orc_assign), and
 *     its seed is a cross-scale maximum (orc_cross_scale);
 *   kept groups, in seed order, take the next halo ids; their particles keep
 *     them for good.
 * Outputs: halo_id[np] (-1: none), and per halo (at most cap): scale index,
 * seed, n_part, n_cells, mass, centre[3], corrected peak. */
int orc_multiscale(const float *pos, const float *mass, double mass_unit, int64_t np, double L, int n_scales,
                   const int *ngs, const float *const *fields, float cwt_min, double dens_th, int64_t particle_th,
                   const float *vel, double G, int max_iter, int32_t *halo_id, int64_t cap, int32_t *scale_out,
                   int64_t *seed_out, int64_t *npart_out, int64_t *ncell_out, double *mass_out, double *centre_out,
                   float *peak_out, int64_t *n_halo, double *margin_out) {
    if (np < 0 || !(L > 0) || !(mass_unit > 0) || n_scales < 1) return ORC_E_ARG;
    int max_ng = 0;
    for (int j = 0; j < n_scales; j++) {
        if (ngs[j] < 3 || !fields[j]) return ORC_E_ARG;
        if (ngs[j] > max_ng) max_ng = ngs[j];
    }
    int64_t max_cells = (int64_t)max_ng * max_ng * max_ng;
    int32_t *lab = malloc(sizeof(int32_t) * (size_t)max_cells);
    int64_t *np_c = malloc(sizeof(int64_t) * (size_t)max_cells), *mq_c = malloc(sizeof(int64_t) * (size_t)max_cells);
    int64_t *nc_c = malloc(sizeof(int64_t) * (size_t)max_cells), *mom = malloc(sizeof(int64_t) * 3 * (size_t)max_cells);
    int32_t *tmp = malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    int32_t *hid_c = malloc(sizeof(int32_t) * (size_t)max_cells);
    /* self-boundness check (vel given): each particle's kept group, its group
     * after the check, the groups' kept members and rounds */
    int32_t *grp = malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    int32_t *bound = malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    int64_t *nk_g = malloc(sizeof(int64_t) * (size_t)max_cells);
    int32_t *it_g = malloc(sizeof(int32_t) * (size_t)max_cells);
    int64_t *rank_c = malloc(sizeof(int64_t) * (size_t)max_cells);
    double margin = INFINITY;
    int rc = (lab && np_c && mq_c && nc_c && mom && tmp && hid_c && grp && bound && nk_g && it_g && rank_c) ? ORC_OK
                                                                                                              : ORC_E_NOMEM;
    if (vel && (!(G >= 0.0) || max_iter < 1)) rc = ORC_E_ARG;
    int64_t mtot = 0, kept = 0;
    for (int64_t p = 0; p < np && rc == ORC_OK; p++) {
        int64_t mq;
        rc = mass_quantum(mass, mass_unit, p, &mq);
        mtot += mq;
        halo_id[p] = -1;
    }
    for (int j = 0; j < n_scales && rc == ORC_OK; j++) {
        const int ng = ngs[j];
        const int64_t cells = (int64_t)ng * ng * ng, M = (int64_t)ng * FRAC_ONE;
        const float *C = fields[j];
        const float *Cn = j + 1 < n_scales ? fields[j + 1] : NULL;
        const int ngn = j + 1 < n_scales ? ngs[j + 1] : 0;
        rc = orc_segment(C, ng, cwt_min, lab);
        if (rc) break;
        for (int64_t c = 0; c < cells; c++) { np_c[c] = mq_c[c] = nc_c[c] = 0; mom[3 * c] = mom[3 * c + 1] = mom[3 * c + 2] = 0; hid_c[c] = -1; }
        for (int64_t c = 0; c < cells; c++)
            if (lab[c] >= 0) nc_c[lab[c]] += 1;
        double s = quant_scale(ng, L);
        for (int64_t p = 0; p < np && rc == ORC_OK; p++) {
            tmp[p] = -1;
            if (halo_id[p] >= 0) continue; /* the particle already belongs to a halo */
            int64_t q[3], mq, node[3];
            for (int a = 0; a < 3 && rc == ORC_OK; a++) rc = quantise_coord(pos[3 * p + a], s, M, &q[a]);
            if (rc == ORC_OK) rc = mass_quantum(mass, mass_unit, p, &mq);
            if (rc) break;
            for (int a = 0; a < 3; a++) node[a] = ((q[a] + FRAC_ONE / 2) >> FRAC_BITS) % ng;
            int32_t l = lab[(node[2] * ng + node[1]) * ng + node[0]];
            tmp[p] = l;
            if (l < 0) continue;
            int64_t sc[3] = {l % ng, (l / ng) % ng, l / ((int64_t)ng * ng)};
            np_c[l] += 1;
            mq_c[l] += mq;
            for (int a = 0; a < 3; a++) mom[3 * l + a] += mq * min_image_q(q[a] - sc[a] * FRAC_ONE, M);
        }
        if (rc) break;
        const double ncube = (double)cells, cell_q = (L / (double)ng) / (double)FRAC_ONE;
        /* steps 7-8: density, particle count and cross-scale checks; kept
         * groups ranked in seed (cell) order */
        int64_t nkept_j = 0;
        for (int64_t c = 0; c < cells; c++) {
            rank_c[c] = -1;
            if (lab[c] != c) continue;
            int keep = np_c[c] >= particle_th && (double)mq_c[c] * ncube >= (dens_th * (double)mtot) * (double)nc_c[c] &&
                       orc_cross_scale(C, ng, c, Cn, ngn);
            if (keep) rank_c[c] = nkept_j++;
        }
        /* step 9: the self-boundness check of every kept group (Sec. 2.3);
         * a discarded group is dropped, and the sums of a kept one are taken
         * again over the members that stay (the ones that get its id) */
        if (vel) {
            for (int64_t p = 0; p < np; p++) grp[p] = (tmp[p] >= 0 && rank_c[tmp[p]] >= 0) ? (int32_t)rank_c[tmp[p]] : -1;
            double mg;
            rc = orc_unbind(pos, vel, mass, mass_unit, np, L, G, grp, nkept_j, max_iter, bound, nk_g, it_g, &mg);
            if (rc) break;
            if (mg < margin) margin = mg;
            for (int64_t c = 0; c < cells; c++)
                if (rank_c[c] >= 0) {
                    if (nk_g[rank_c[c]] == 0) rank_c[c] = -1; /* discarded */
                    np_c[c] = mq_c[c] = 0;
                    mom[3 * c] = mom[3 * c + 1] = mom[3 * c + 2] = 0;
                }
            for (int64_t p = 0; p < np && rc == ORC_OK; p++) {
                if (bound[p] < 0) continue;
                const int32_t l = tmp[p];
                int64_t q[3], mq;
                for (int a = 0; a < 3 && rc == ORC_OK; a++) rc = quantise_coord(pos[3 * p + a], s, M, &q[a]);
                if (rc == ORC_OK) rc = mass_quantum(mass, mass_unit, p, &mq);
                if (rc) break;
                int64_t sc[3] = {l % ng, (l / ng) % ng, l / ((int64_t)ng * ng)};
                np_c[l] += 1;
                mq_c[l] += mq;
                for (int a = 0; a < 3; a++) mom[3 * l + a] += mq * min_image_q(q[a] - sc[a] * FRAC_ONE, M);
            }
            if (rc) break;
        }
        /* step 10: halo ids in seed order, the catalogue */
        for (int64_t c = 0; c < cells; c++) {
            if (rank_c[c] < 0) continue;
            hid_c[c] = (int32_t)kept;
            if (kept < cap) {
                int64_t sc[3] = {c % ng, (c / ng) % ng, c / ((int64_t)ng * ng)};
                scale_out[kept] = j;
                seed_out[kept] = c;
                npart_out[kept] = np_c[c];
                ncell_out[kept] = nc_c[c];
                mass_out[kept] = (double)mq_c[c] * mass_unit;
                for (int a = 0; a < 3; a++) {
                    double u = (double)(sc[a] * FRAC_ONE);
                    if (mq_c[c] > 0) u += (double)mom[3 * c + a] / (double)mq_c[c];
                    double x = u * cell_q;
                    if (x >= L) x -= L;
                    else if (x < 0.0) x += L;
                    centre_out[3 * kept + a] = x;
                }
                peak_out[kept] = orc_corrected_peak(C, ng, c, ngn);
            }
            kept++;
        }
        for (int64_t p = 0; p < np; p++)
            if (halo_id[p] < 0 && tmp[p] >= 0 && hid_c[tmp[p]] >= 0 && (!vel || bound[p] >= 0))
                halo_id[p] = hid_c[tmp[p]];
    }
    free(lab); free(np_c); free(mq_c); free(nc_c); free(mom); free(tmp); free(hid_c);
    free(grp); free(bound); free(nk_g); free(it_g); free(rank_c);
    if (margin_out) *margin_out = margin;
    if (rc == ORC_OK) {
        *n_halo = kept;
        if (kept > cap) rc = ORC_E_CAPACITY;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: the self-boundness check (step 9 of the Sec. 2 step list).      */
/* ------------------------------------------------------------------------ */

/* Every group g (particles with group[i] == g, 0 <= g < n_groups) is checked
 * on its own, following Sec. 2.3 in order:
 *   1. the halo centre is the centre of mass of the group's current members
 *      (mass-weighted mean of the minimum-image offsets from the group's
 *      first member in particle order);
 *   2. assuming spherical symmetry, the potential at member i is that of the
 *      spherical shells of the other members about the centre (shell
 *      theorem): Phi_i = -G sum_{j != i} m_j / max(r_i, r_j), so the local
 *      escape speed is v_esc^2 = -2 Phi_i;
 *   3. members whose speed relative to the group's mass-weighted mean velocity
 *      exceeds v_esc are excluded (all at once), and the centre is recomputed
 *      from the remaining members;
 *   4. steps 1-3 repeat until no member is excluded (at most max_iter rounds);
 *   5. if more than 40 % of the group's particles were excluded (5 excluded >
 *      2 initial), the whole group is discarded.
 * Masses are m_i = m_q * mass_unit with the integer mass quanta of the
 * deposit (1 when mass is NULL).  A zero-mass member adds nothing to any
 * potential; two members both at the centre (max(r_i, r_j) = 0, m_j > 0) make
 * Phi_i infinite, so they stay.  With no mass left the centre is the first
 * member and the mean velocity zero.
 * Outputs: out_group[i] = g for members that stay in a group that is kept,
 * else -1; out_n[g] = members kept (0 if discarded); out_iter[g] = rounds run;
 * *out_margin = the smallest |v_rel^2 - v_esc^2| / v_esc^2 over every
 * decision taken (how close any decision came to the other side). */
int orc_unbind(const float *pos, const float *vel, const float *mass, double mass_unit, int64_t np, double L,
               double G, const int32_t *group, int64_t n_groups, int max_iter, int32_t *out_group, int64_t *out_n,
               int32_t *out_iter, double *out_margin) {
    if (np < 0 || n_groups < 0 || !(L > 0.0) || !(G >= 0.0) || max_iter < 1 || !(mass_unit > 0.0))
        return ORC_E_ARG;
    double margin = INFINITY;
    int64_t *mem = malloc(((size_t)np + 1) * sizeof(int64_t));
    double *m = malloc(((size_t)np + 1) * sizeof(double));
    double *r = malloc(((size_t)np + 1) * sizeof(double));
    char *keep = malloc((size_t)np + 1);
    if (!mem || !m || !r || !keep) {
        free(mem); free(m); free(r); free(keep);
        return ORC_E_NOMEM;
    }
    int rc = ORC_OK;
    for (int64_t i = 0; i < np && rc == ORC_OK; i++) {
        out_group[i] = -1;
        int64_t mq;
        if ((rc = mass_quantum(mass, mass_unit, i, &mq)) != ORC_OK) break;
        m[i] = (double)mq * mass_unit;
    }
    for (int64_t g = 0; g < n_groups && rc == ORC_OK; g++) {
        /* the group's members in particle order */
        int64_t n = 0;
        for (int64_t i = 0; i < np; i++)
            if (group[i] == g) mem[n++] = i;
        const int64_t n0 = n;
        out_n[g] = 0;
        out_iter[g] = 0;
        if (n0 == 0) continue;
        const float *a = pos + 3 * mem[0];
        int it = 0;
        while (it < max_iter) {
            it++;
            /* 1. centre of mass and mean velocity of the current members */
            double M = 0.0, sd[3] = {0.0, 0.0, 0.0}, sv[3] = {0.0, 0.0, 0.0};
            for (int64_t k = 0; k < n; k++) {
                const int64_t i = mem[k];
                M += m[i];
                for (int c = 0; c < 3; c++) {
                    double d = (double)pos[3 * i + c] - (double)a[c];
                    d -= L * floor(d / L + 0.5);
                    sd[c] += m[i] * d;
                    sv[c] += m[i] * (double)vel[3 * i + c];
                }
            }
            double cen[3] = {0.0, 0.0, 0.0}, vb[3] = {0.0, 0.0, 0.0};
            if (M > 0.0)
                for (int c = 0; c < 3; c++) {
                    cen[c] = sd[c] / M;
                    vb[c] = sv[c] / M;
                }
            for (int64_t k = 0; k < n; k++) {
                const int64_t i = mem[k];
                double s2 = 0.0;
                for (int c = 0; c < 3; c++) {
                    double d = (double)pos[3 * i + c] - (double)a[c];
                    d -= L * floor(d / L + 0.5);
                    s2 += (d - cen[c]) * (d - cen[c]);
                }
                r[i] = sqrt(s2);
            }
            /* 2-3. escape speeds from the shell potential; exclusions */
            int64_t kept = 0;
            for (int64_t k = 0; k < n; k++) {
                const int64_t i = mem[k];
                double S = 0.0;
                for (int64_t l = 0; l < n; l++) {
                    const int64_t j = mem[l];
                    if (j == i || !(m[j] > 0.0)) continue;
                    S += m[j] / fmax(r[i], r[j]);
                }
                const double vesc2 = 2.0 * G * S;
                double v2 = 0.0;
                for (int c = 0; c < 3; c++) {
                    const double dv = (double)vel[3 * i + c] - vb[c];
                    v2 += dv * dv;
                }
                keep[i] = !(v2 > vesc2);
                if (vesc2 > 0.0 && isfinite(vesc2)) {
                    const double q = fabs(v2 - vesc2) / vesc2;
                    if (q < margin) margin = q;
                }
                kept += keep[i];
            }
            if (kept == n) break;
            int64_t w = 0;
            for (int64_t k = 0; k < n; k++)
                if (keep[mem[k]]) mem[w++] = mem[k];
            n = w;
        }
        out_iter[g] = it;
        /* 5. more than 40 % excluded: the group is discarded */
        if (5 * (n0 - n) > 2 * n0) continue;
        out_n[g] = n;
        for (int64_t k = 0; k < n; k++) out_group[mem[k]] = (int32_t)g;
    }
    *out_margin = margin;
    free(mem); free(m); free(r); free(keep);
    return rc;
}
