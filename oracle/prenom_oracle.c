/* FP64 CPU oracle of the PRENOM object-NeRF training step (arXiv 2503.01582).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the package smoke check and
 * the benchmark's CPU-baseline leg, never by the product path.
 *
 * Plain, slow and sequential on purpose.  Each function restates one step of
 * the paper in its own order and notation; see prenom_oracle.h for the list.
 * Compile without fast-math and without FP contraction.
 */
#include "prenom_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ================================================================ hash grid
 * §III-B "Object-level NeRFs": the NeRF uses the multiresolution hash encoding
 * of instant-NGP (Müller et al. 2022), which the paper cites for this step.
 * Readings taken here (the paper prints none of these details):
 *   - level resolution N_l = floor(N_min * b^l) with
 *     b = exp((ln N_max - ln N_min) / (L - 1)); a 1e-6 guard keeps products
 *     that are mathematically integral (b^(L-1) * N_min = N_max) from rounding
 *     down;
 *   - a level whose (N_l + 1)^3 grid vertices fit in T entries is stored
 *     densely (x fastest), otherwise through the spatial hash
 *     (x * 1) xor (y * 2654435761) xor (z * 805459861) mod T in uint32 arithmetic;
 *   - a point p in [0,1]^3 sits in cell c0 = min(floor(p N_l), N_l - 1) with
 *     local coordinates w = p N_l - c0 in [0,1].
 */
int orc_level_res(const orc_arch *a, int l)
{
    double b = 1.0;
    if (a->L > 1)
        b = exp((log((double)a->n_max) - log((double)a->n_min)) / (double)(a->L - 1));
    return (int)floor((double)a->n_min * pow(b, (double)l) + 1e-6);
}

static int64_t level_vertices(const orc_arch *a, int l)
{
    int64_t n1 = (int64_t)orc_level_res(a, l) + 1;
    return n1 * n1 * n1;
}

int orc_level_dense(const orc_arch *a, int l)
{
    return level_vertices(a, l) <= ((int64_t)1 << a->log2T);
}

int64_t orc_level_entries(const orc_arch *a, int l)
{
    return orc_level_dense(a, l) ? level_vertices(a, l) : ((int64_t)1 << a->log2T);
}

/* Storage layout (not part of the method): each level's table occupies its
 * entry count rounded up to a multiple of 8 entries, so every level starts
 * on a 64-byte boundary; the padding entries are never addressed. */
int64_t orc_level_offset(const orc_arch *a, int l)
{
    int64_t off = 0;
    for (int i = 0; i < l; ++i)
        off += (orc_level_entries(a, i) + 7) / 8 * 8 * a->F;
    return off;
}

int64_t orc_n_hash_params(const orc_arch *a)
{
    return orc_level_offset(a, a->L);
}

static int mlp_in(const orc_arch *a, int layer)
{
    return layer == 0 ? a->L * a->F : a->width;
}

static int mlp_out(const orc_arch *a, int layer)
{
    return layer == a->hidden ? 4 : a->width;
}

int64_t orc_mlp_offset(const orc_arch *a, int layer)
{
    int64_t off = orc_n_hash_params(a);
    for (int i = 0; i < layer; ++i)
        off += (int64_t)mlp_in(a, i) * mlp_out(a, i);
    return off;
}

int64_t orc_n_mlp_params(const orc_arch *a)
{
    return orc_mlp_offset(a, a->hidden + 1) - orc_n_hash_params(a);
}

int64_t orc_param_count(const orc_arch *a)
{
    return orc_mlp_offset(a, a->hidden + 1);
}

uint32_t orc_grid_index(const orc_arch *a, int l, uint32_t cx, uint32_t cy, uint32_t cz)
{
    if (orc_level_dense(a, l)) {
        uint32_t n1 = (uint32_t)orc_level_res(a, l) + 1u;
        return cx + cy * n1 + cz * n1 * n1;
    }
    uint32_t h = (cx * 1u) ^ (cy * 2654435761u) ^ (cz * 805459861u);
    return h & (((uint32_t)1 << a->log2T) - 1u);
}

static double clamp01(double x)
{
    return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
}

/* Trilinear blend of the 8 corner features, levels concatenated coarse first. */
void orc_encode(const orc_arch *a, const double *theta, const double *p_in, double *enc)
{
    double p[3] = {clamp01(p_in[0]), clamp01(p_in[1]), clamp01(p_in[2])};
    for (int l = 0; l < a->L; ++l) {
        int N = orc_level_res(a, l);
        int64_t off = orc_level_offset(a, l);
        int c0[3];
        double w[3];
        for (int i = 0; i < 3; ++i) {
            double s = p[i] * (double)N;
            double f = floor(s);
            if (f > (double)(N - 1))
                f = (double)(N - 1);
            c0[i] = (int)f;
            w[i] = s - f;
        }
        for (int f = 0; f < a->F; ++f)
            enc[l * a->F + f] = 0.0;
        for (int corner = 0; corner < 8; ++corner) {
            int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
            double wt = (bx ? w[0] : 1.0 - w[0]) * (by ? w[1] : 1.0 - w[1]) * (bz ? w[2] : 1.0 - w[2]);
            uint32_t idx = orc_grid_index(a, l, (uint32_t)(c0[0] + bx), (uint32_t)(c0[1] + by),
                                          (uint32_t)(c0[2] + bz));
            for (int f = 0; f < a->F; ++f)
                enc[l * a->F + f] += wt * theta[off + (int64_t)idx * a->F + f];
        }
    }
}

/* d enc / d theta: each corner entry receives its trilinear weight times denc. */
void orc_encode_backward(const orc_arch *a, const double *p_in, const double *denc, double *grad)
{
    double p[3] = {clamp01(p_in[0]), clamp01(p_in[1]), clamp01(p_in[2])};
    for (int l = 0; l < a->L; ++l) {
        int N = orc_level_res(a, l);
        int64_t off = orc_level_offset(a, l);
        int c0[3];
        double w[3];
        for (int i = 0; i < 3; ++i) {
            double s = p[i] * (double)N;
            double f = floor(s);
            if (f > (double)(N - 1))
                f = (double)(N - 1);
            c0[i] = (int)f;
            w[i] = s - f;
        }
        for (int corner = 0; corner < 8; ++corner) {
            int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
            double wt = (bx ? w[0] : 1.0 - w[0]) * (by ? w[1] : 1.0 - w[1]) * (bz ? w[2] : 1.0 - w[2]);
            uint32_t idx = orc_grid_index(a, l, (uint32_t)(c0[0] + bx), (uint32_t)(c0[1] + by),
                                          (uint32_t)(c0[2] + bz));
            for (int f = 0; f < a->F; ++f)
                grad[off + (int64_t)idx * a->F + f] += wt * denc[l * a->F + f];
        }
    }
}

/* ==================================================================== MLP
 * §III-B "Object-level NeRFs": a shallow MLP maps the encoding to density and
 * colour.  Readings: no biases, ReLU hidden layers, linear 4-wide output o;
 * sigma = exp(min(o_0, 15)) (derivative 0 where the clamp is active),
 * c = sigmoid(o_1..3); no view direction (object-level, Lambertian targets).
 * acts holds the post-ReLU activations, layer-major [H][W].
 */
void orc_mlp_forward(const orc_arch *a, const double *theta, const double *enc,
                     double *acts, double *out4)
{
    const double *x = enc;
    for (int layer = 0; layer <= a->hidden; ++layer) {
        int nin = mlp_in(a, layer), nout = mlp_out(a, layer);
        const double *Wm = theta + orc_mlp_offset(a, layer);
        double *y = layer == a->hidden ? out4 : acts + (int64_t)layer * a->width;
        for (int j = 0; j < nout; ++j) {
            double s = 0.0;
            for (int i = 0; i < nin; ++i)
                s += Wm[(int64_t)j * nin + i] * x[i];
            y[j] = (layer == a->hidden) ? s : (s > 0.0 ? s : 0.0);
        }
        x = y;
    }
}

void orc_mlp_backward(const orc_arch *a, const double *theta, const double *enc,
                      const double *acts, const double *dout4, double *grad, double *denc)
{
    int W = a->width;
    double *dy = (double *)malloc(sizeof(double) * (size_t)(W > 4 ? W : 4));
    double *dx = (double *)malloc(sizeof(double) * (size_t)(W > a->L * a->F ? W : a->L * a->F));
    for (int j = 0; j < 4; ++j)
        dy[j] = dout4[j];
    for (int layer = a->hidden; layer >= 0; --layer) {
        int nin = mlp_in(a, layer), nout = mlp_out(a, layer);
        int64_t woff = orc_mlp_offset(a, layer);
        const double *x = layer == 0 ? enc : acts + (int64_t)(layer - 1) * W;
        for (int j = 0; j < nout; ++j)
            for (int i = 0; i < nin; ++i)
                grad[woff + (int64_t)j * nin + i] += dy[j] * x[i];
        for (int i = 0; i < nin; ++i) {
            double s = 0.0;
            for (int j = 0; j < nout; ++j)
                s += theta[woff + (int64_t)j * nin + i] * dy[j];
            /* ReLU of the layer below: derivative 1 where its output is > 0 */
            dx[i] = (layer == 0) ? s : (x[i] > 0.0 ? s : 0.0);
        }
        if (layer == 0)
            for (int i = 0; i < nin; ++i)
                denc[i] = dx[i];
        else
            for (int i = 0; i < nin; ++i)
                dy[i] = dx[i];
    }
    free(dy);
    free(dx);
}

/* =============================================================== sampling
 * §III-B "Probabilistic Ray Sampling".
 * Ray setup: rays arrive in the object frame; the object's bounding box is the
 * unit cube, so [tn, tf] is the slab intersection of the ray (t >= 0) with
 * [0,1]^3.  A ray that misses it (tf <= tn) gets tn = tf = 0.
 */
int orc_ray_box(const double *o, const double *d, double *tn, double *tf)
{
    double t0 = 0.0, t1 = INFINITY;
    for (int i = 0; i < 3; ++i) {
        if (d[i] != 0.0) {
            double ta = (0.0 - o[i]) / d[i];
            double tb = (1.0 - o[i]) / d[i];
            double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
            if (lo > t0)
                t0 = lo;
            if (hi < t1)
                t1 = hi;
        } else if (o[i] < 0.0 || o[i] > 1.0) {
            t1 = -INFINITY;
        }
    }
    if (!(t1 > t0)) {
        *tn = 0.0;
        *tf = 0.0;
        return 0;
    }
    *tn = t0;
    *tf = t1;
    return 1;
}

/* Prior density F(x): the paper states trilinear interpolation over the fixed
 * grid (§III-B, object state canonicalization, Eq. 3) and reuses F for
 * sampling.  Reading: values sit at voxel centres (i + 1/2)/R, x fastest;
 * g = x R - 1/2 is clamped to [0, R-1]. */
double orc_prior_lookup(const double *grid, int R, const double *x)
{
    int c0[3];
    double w[3];
    for (int i = 0; i < 3; ++i) {
        double g = x[i] * (double)R - 0.5;
        if (g < 0.0)
            g = 0.0;
        if (g > (double)(R - 1))
            g = (double)(R - 1);
        double f = floor(g);
        if (f > (double)(R - 2))
            f = (double)(R - 2);
        c0[i] = (int)f;
        w[i] = g - f;
    }
    double s = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
        int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        double wt = (bx ? w[0] : 1.0 - w[0]) * (by ? w[1] : 1.0 - w[1]) * (bz ? w[2] : 1.0 - w[2]);
        if (wt == 0.0)
            continue; /* a zero weight takes no part, even next to a huge value */
        int64_t idx = ((int64_t)(c0[2] + bz) * R + (c0[1] + by)) * R + (c0[0] + bx);
        s += wt * grid[idx];
    }
    return s;
}

/* Inverse transform sampling on the discrete CDF (cdf[0] = 0 ... cdf[Nc] = 1).
 * Reading: sample k falls in bin b = the first b with cdf[b+1] > u_k (a strict
 * comparison: u on an edge goes to the next bin and an empty bin is never
 * chosen), and moves linearly inside the bin:
 *   t_k = tn + (b + (u_k - cdf[b]) / (cdf[b+1] - cdf[b])) * Delta. */
void orc_cdf_invert(const double *cdf, int Nc, const double *u, int Nr,
                    double tn, double tf, int *bins, double *t)
{
    double delta = (tf - tn) / (double)Nc;
    for (int k = 0; k < Nr; ++k) {
        int b = 0;
        while (b < Nc - 1 && !(cdf[b + 1] > u[k]))
            ++b;
        double frac = (u[k] - cdf[b]) / (cdf[b + 1] - cdf[b]);
        bins[k] = b;
        t[k] = tn + ((double)b + frac) * delta;
    }
}

/* One ray of the sampler: probes, Eq. 4, Eq. 5 (literal product), Eq. 6, the
 * escape rule and the inverse transform.  Readings: Nc equal-width bins of
 * [tn, tf], probe i at the bin centre with delta_i = Delta for every bin;
 * escape when sum rho_term < eps, then the CDF is the uniform one i / Nc.
 * Returns 1 when the ray escaped. */
int orc_sample_ray(const double *grid, int R, const double *o, const double *d,
                   int Nc, int Nr, double eps, const double *u,
                   double *probe_sigma, double *rho_term, double *cdf,
                   int *bins, double *t, double *tn_out, double *tf_out)
{
    double tn, tf;
    int hit = orc_ray_box(o, d, &tn, &tf);
    double delta = (tf - tn) / (double)Nc;
    double trans = 1.0; /* prod_{j<i} (1 - rho_occ_j) */
    double total = 0.0;
    for (int i = 0; i < Nc; ++i) {
        double ti = tn + ((double)i + 0.5) * delta;
        double x[3] = {o[0] + ti * d[0], o[1] + ti * d[1], o[2] + ti * d[2]};
        probe_sigma[i] = hit ? orc_prior_lookup(grid, R, x) : 0.0;
        double rho_occ = 1.0 - exp(-probe_sigma[i] * delta); /* Eq. 4 */
        rho_term[i] = rho_occ * trans;                         /* Eq. 5 */
        trans *= (1.0 - rho_occ);
        total += rho_term[i];
    }
    int escape = !(total >= eps);
    cdf[0] = 0.0;
    if (escape) {
        for (int i = 1; i < Nc; ++i)
            cdf[i] = (double)i / (double)Nc;
    } else {
        double run = 0.0;
        for (int i = 1; i < Nc; ++i) {
            run += rho_term[i - 1];
            cdf[i] = run / total; /* Eq. 6 */
        }
    }
    cdf[Nc] = 1.0;
    orc_cdf_invert(cdf, Nc, u, Nr, tn, tf, bins, t);
    *tn_out = tn;
    *tf_out = tf;
    return escape;
}

/* ============================================================== rendering
 * §III-B "Volume Rendering", Eq. 7 with the weights of Eq. 5 evaluated at the
 * network's densities: w_k = (1 - exp(-sigma_k delta_k)) prod_{j<k} exp(-sigma_j delta_j).
 * Readings: delta_k = t_{k+1} - t_k and, for the last sample, tf - t_{Nr-1}
 * (the ray ends at the bounding box); depth is the unnormalised sum of w t.
 * c is [Nr][3]. */
void orc_composite(int Nr, const double *sigma, const double *c, const double *t, double tf,
                   double *w, double *C, double *D, double *A)
{
    double trans = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    *D = 0.0;
    *A = 0.0;
    for (int k = 0; k < Nr; ++k) {
        double delta = (k + 1 < Nr ? t[k + 1] : tf) - t[k];
        double alpha = 1.0 - exp(-sigma[k] * delta);
        w[k] = alpha * trans;
        trans *= (1.0 - alpha);
        for (int ch = 0; ch < 3; ++ch)
            C[ch] += w[k] * c[k * 3 + ch];
        *D += w[k] * t[k];
        *A += w[k];
    }
}

/* Adjoint of orc_composite for upstream gradients (gC, gD, gA):
 * with v_k = gC . c_k + gD t_k + gA and T_{k+1} = prod_{j<=k} (1 - alpha_j),
 *   dL/dsigma_k = delta_k (T_{k+1} v_k - sum_{j>k} w_j v_j),   dL/dc_k = w_k gC. */
void orc_composite_backward(int Nr, const double *sigma, const double *c, const double *t,
                            double tf, const double *gC, double gD, double gA,
                            double *dsigma, double *dc)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)(Nr > 0 ? Nr : 1));
    double *v = (double *)malloc(sizeof(double) * (size_t)(Nr > 0 ? Nr : 1));
    double *tnext = (double *)malloc(sizeof(double) * (size_t)(Nr > 0 ? Nr : 1));
    double *dl = (double *)malloc(sizeof(double) * (size_t)(Nr > 0 ? Nr : 1));
    double trans = 1.0;
    for (int k = 0; k < Nr; ++k) {
        dl[k] = (k + 1 < Nr ? t[k + 1] : tf) - t[k];
        double alpha = 1.0 - exp(-sigma[k] * dl[k]);
        w[k] = alpha * trans;
        trans *= (1.0 - alpha);
        tnext[k] = trans;
        v[k] = gC[0] * c[k * 3 + 0] + gC[1] * c[k * 3 + 1] + gC[2] * c[k * 3 + 2] + gD * t[k] + gA;
    }
    double suffix = 0.0; /* sum_{j>k} w_j v_j */
    for (int k = Nr - 1; k >= 0; --k) {
        dsigma[k] = dl[k] * (tnext[k] * v[k] - suffix);
        for (int ch = 0; ch < 3; ++ch)
            dc[k * 3 + ch] = w[k] * gC[ch];
        suffix += w[k] * v[k];
    }
    free(w);
    free(v);
    free(tnext);
    free(dl);
}

static double sgn(double x)
{
    return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
}

/* Per-ray terms of Eq. 8 (without the 1/R mean and without L_sigma, which is a
 * per-sample term).  Readings: the photometric norm is squared; a background
 * ray composites C_rand behind the object, so its colour term is
 * || C + (1 - A) C_rand - C_rand ||^2; |x| has subgradient 0 at 0.
 * Returns the ray's loss; writes dL/dC, dL/dD, dL/dA. */
double orc_ray_loss(int is_obj, const double *C, double D, double A, const double *Cgt,
                    double Dgt, const double *crand, double lambda_d,
                    double *gC, double *gD, double *gA)
{
    double L = 0.0;
    if (is_obj) {
        for (int ch = 0; ch < 3; ++ch) {
            double e = C[ch] - Cgt[ch];
            L += e * e;
            gC[ch] = 2.0 * e;
        }
        L += lambda_d * fabs(D - Dgt);
        *gD = lambda_d * sgn(D - Dgt);
        *gA = 0.0;
    } else {
        double dot = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            double r = C[ch] + (1.0 - A) * crand[ch] - crand[ch];
            L += r * r;
            gC[ch] = 2.0 * r;
            dot += 2.0 * r * crand[ch];
        }
        *gD = 0.0;
        *gA = -dot;
    }
    return L;
}

/* ================================================================== batch
 * One training batch of one object: for each ray, sample (or take t_in),
 * encode, run the MLP, composite, add the ray's loss (Eq. 8, Eq. 9, mean over
 * the batch's rays) and, when grad != NULL, accumulate dL/dtheta.  The sample
 * positions do not depend on theta (the prior grid is fixed within a step), so
 * no gradient flows through the sampler.
 * upstream != NULL ([n][5] = dC[3], dD, dA per ray) replaces the loss: the
 * returned value is then sum_r upstream_r . (C_r, D_r, A_r) and the gradient
 * is that of this linear functional (no 1/R, no L_sigma).
 * Colours c_rand may be NULL: background rays then use C_rand = 0. */
double orc_batch(const orc_arch *a, const double *theta, const double *grid, int R,
                 int n, const double *o, const double *d, const double *rgb,
                 const double *depth, const uint8_t *is_obj, const double *crand,
                 const double *u, const double *t_in, int Nc, int Nr, double eps,
                 const double *upstream,
                 double *out_rgb, double *out_depth, double *out_acc,
                 int *out_bins, double *out_t, double *out_sigma, double *grad)
{
    if (n <= 0)
        return 0.0;
    int IN = a->L * a->F, W = a->width, H = a->hidden;
    double *probe = (double *)malloc(sizeof(double) * (size_t)Nc);
    double *rho = (double *)malloc(sizeof(double) * (size_t)Nc);
    double *cdf = (double *)malloc(sizeof(double) * (size_t)(Nc + 1));
    int *bins = (int *)malloc(sizeof(int) * (size_t)Nr);
    double *t = (double *)malloc(sizeof(double) * (size_t)Nr);
    double *pos = (double *)malloc(sizeof(double) * (size_t)Nr * 3);
    double *enc = (double *)malloc(sizeof(double) * (size_t)Nr * IN);
    double *acts = (double *)malloc(sizeof(double) * (size_t)Nr * H * W);
    double *outv = (double *)malloc(sizeof(double) * (size_t)Nr * 4);
    double *sigma = (double *)malloc(sizeof(double) * (size_t)Nr);
    double *col = (double *)malloc(sizeof(double) * (size_t)Nr * 3);
    double *w = (double *)malloc(sizeof(double) * (size_t)Nr);
    double *dsig = (double *)malloc(sizeof(double) * (size_t)Nr);
    double *dcol = (double *)malloc(sizeof(double) * (size_t)Nr * 3);
    double *denc = (double *)malloc(sizeof(double) * (size_t)IN);
    double total = 0.0;
    double inv_r = 1.0 / (double)n;

    for (int r = 0; r < n; ++r) {
        const double *orr = o + 3 * r, *drr = d + 3 * r;
        double tn, tf;
        if (t_in) {
            orc_ray_box(orr, drr, &tn, &tf);
            for (int k = 0; k < Nr; ++k) {
                t[k] = t_in[(int64_t)r * Nr + k];
                bins[k] = -1;
            }
        } else {
            orc_sample_ray(grid, R, orr, drr, Nc, Nr, eps, u + (int64_t)r * Nr, probe, rho, cdf, bins,
                           t, &tn, &tf);
        }
        for (int k = 0; k < Nr; ++k) {
            double *p = pos + 3 * k;
            for (int i = 0; i < 3; ++i)
                p[i] = orr[i] + t[k] * drr[i];
            orc_encode(a, theta, p, enc + (int64_t)k * IN);
            orc_mlp_forward(a, theta, enc + (int64_t)k * IN, acts + (int64_t)k * H * W, outv + 4 * k);
            double o0 = outv[4 * k];
            sigma[k] = exp(o0 < 15.0 ? o0 : 15.0);
            for (int ch = 0; ch < 3; ++ch)
                col[3 * k + ch] = 1.0 / (1.0 + exp(-outv[4 * k + 1 + ch]));
        }
        double C[3], D, A;
        orc_composite(Nr, sigma, col, t, tf, w, C, &D, &A);
        if (out_rgb)
            for (int ch = 0; ch < 3; ++ch)
                out_rgb[3 * r + ch] = C[ch];
        if (out_depth)
            out_depth[r] = D;
        if (out_acc)
            out_acc[r] = A;
        if (out_bins)
            for (int k = 0; k < Nr; ++k)
                out_bins[(int64_t)r * Nr + k] = bins[k];
        if (out_t)
            for (int k = 0; k < Nr; ++k)
                out_t[(int64_t)r * Nr + k] = t[k];
        if (out_sigma)
            for (int k = 0; k < Nr; ++k)
                out_sigma[(int64_t)r * Nr + k] = sigma[k];

        double gC[3], gD, gA;
        int background = 0;
        if (upstream) {
            const double *g = upstream + 5 * r;
            gC[0] = g[0];
            gC[1] = g[1];
            gC[2] = g[2];
            gD = g[3];
            gA = g[4];
            total += gC[0] * C[0] + gC[1] * C[1] + gC[2] * C[2] + gD * D + gA * A;
        } else {
            background = !is_obj[r];
            static const double no_colour[3] = {0.0, 0.0, 0.0}; /* when the caller gives none */
            double Lr = orc_ray_loss(is_obj[r], C, D, A, rgb + 3 * r, depth[r],
                                     crand ? crand + 3 * r : no_colour, a->lambda_d, gC, &gD, &gA);
            if (background) /* L_sigma: sum_j |sigma_j| over background rays (Eq. 8) */
                for (int k = 0; k < Nr; ++k)
                    Lr += a->lambda_sigma * fabs(sigma[k]);
            total += Lr * inv_r;
            for (int ch = 0; ch < 3; ++ch)
                gC[ch] *= inv_r;
            gD *= inv_r;
            gA *= inv_r;
        }
        if (!grad)
            continue;
        orc_composite_backward(Nr, sigma, col, t, tf, gC, gD, gA, dsig, dcol);
        for (int k = 0; k < Nr; ++k) {
            double ds = dsig[k];
            if (background)
                ds += a->lambda_sigma * sgn(sigma[k]) * inv_r;
            double dout[4];
            double o0 = outv[4 * k];
            dout[0] = o0 < 15.0 ? ds * sigma[k] : 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                double cc = col[3 * k + ch];
                dout[1 + ch] = dcol[3 * k + ch] * cc * (1.0 - cc);
            }
            orc_mlp_backward(a, theta, enc + (int64_t)k * IN, acts + (int64_t)k * H * W, dout, grad, denc);
            orc_encode_backward(a, pos + 3 * k, denc, grad);
        }
    }
    free(probe);
    free(rho);
    free(cdf);
    free(bins);
    free(t);
    free(pos);
    free(enc);
    free(acts);
    free(outv);
    free(sigma);
    free(col);
    free(w);
    free(dsig);
    free(dcol);
    free(denc);
    return total;
}

/* =================================================================== Adam
 * §III-B: the loss is back-propagated and the NeRF parameters are optimised
 * with Adam (Kingma & Ba 2015).  Readings: every parameter is updated every
 * step (dense), with bias correction; step is the 1-based step count. */
void orc_adam(int64_t n, double *theta, double *m, double *v, const double *g, int step,
              double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, (double)step);
    double c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1;
        double vh = v[i] / c2;
        theta[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ======================================================== training rays
 * §III-B "Training Data": RGB-D images, instance masks and camera poses of
 * the keyframes supervise the object's NeRF; "Probabilistic Ray Sampling":
 * camera rays are transformed into the object frame with the estimated object
 * pose and bounded by the object's box.  Readings: the object frame is the
 * normalised one of Eq. 3, p_n = R_wo^T (p_w - c) / S + 1/2, so the box is
 * the unit cube and the world ray parameter t (distance along the unit world
 * direction) is kept: o_n = R_wo^T (o_w - c) / S + 1/2, d_n = R_wo^T d_w / S;
 * a pixel (x, y) shoots through its centre (x + 1/2, y + 1/2) of a pinhole
 * camera; its ray is a candidate when it meets the box, and, for a pixel of
 * the object's instance, when its depth is valid (> 0, finite); the depth
 * target of an object ray is the z-depth times the length of the
 * unnormalised camera direction (x', y', 1), i.e. the distance t along the
 * ray; a background ray (inside the box, not the instance) has no depth
 * target.  Rays are drawn uniformly from all candidates of all keyframes
 * (keyframe-major, row-major order): index = floor(r 2^-32 n_candidates) for a
 * 32-bit random word r.
 * Precision: these are geometric decisions that pick integers (candidate or
 * not, which pixel), so they are taken in FP32 with the kernel's operation
 * order (each operation rounded, no contraction); every output is then
 * identical on both sides. */
static int orc_ray_box_f(const float *o, const float *d)
{
    float t0 = 0.0f, t1 = INFINITY;
    for (int i = 0; i < 3; ++i) {
        if (d[i] != 0.0f) {
            const float ta = (0.0f - o[i]) / d[i];
            const float tb = (1.0f - o[i]) / d[i];
            const float lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
            if (lo > t0)
                t0 = lo;
            if (hi < t1)
                t1 = hi;
        } else if (o[i] < 0.0f || o[i] > 1.0f) {
            t1 = -INFINITY;
        }
    }
    return t1 > t0;
}

int orc_pixel_ray(const orc_keyframe *kf, const orc_object_state *st, int x, int y, float *o, float *d, float *rgb,
                  float *depth, uint8_t *is_obj)
{
    const float u = (float)x + 0.5f, v = (float)y + 0.5f;
    const float dc[3] = {(u - kf->cx) / kf->fx, (v - kf->cy) / kf->fy, 1.0f};
    const float *R = kf->R_wc;
    float dw[3];
    for (int a = 0; a < 3; ++a)
        dw[a] = (R[3 * a] * dc[0] + R[3 * a + 1] * dc[1]) + R[3 * a + 2];
    const float nrm = sqrtf((dw[0] * dw[0] + dw[1] * dw[1]) + dw[2] * dw[2]);
    float dh[3], rel[3];
    for (int a = 0; a < 3; ++a) {
        dh[a] = dw[a] / nrm;
        rel[a] = kf->t_wc[a] - st->centre[a];
    }
    const float *Q = st->R_wo;  /* object-to-world; its transpose maps world to object */
    for (int a = 0; a < 3; ++a) {
        o[a] = ((Q[a] * rel[0] + Q[3 + a] * rel[1]) + Q[6 + a] * rel[2]) / st->size[a] + 0.5f;
        d[a] = ((Q[a] * dh[0] + Q[3 + a] * dh[1]) + Q[6 + a] * dh[2]) / st->size[a];
    }
    const int64_t pix = (int64_t)y * kf->width + x;
    const int obj = kf->mask[pix] == st->instance;
    const float D = kf->depth[pix];
    const int valid = D > 0.0f && isfinite(D);
    for (int c = 0; c < 3; ++c)
        rgb[c] = (float)kf->rgb[3 * pix + c] / 255.0f;
    *depth = obj ? D * nrm : 0.0f;
    *is_obj = (uint8_t)obj;
    return orc_ray_box_f(o, d) && (!obj || valid);
}

int64_t orc_make_rays(const orc_keyframe *kfs, int n_kf, const orc_object_state *st, int n, const uint32_t *draws,
                      float *o, float *d, float *rgb, float *depth, uint8_t *is_obj)
{
    int64_t total = 0;
    for (int k = 0; k < n_kf; ++k)
        total += (int64_t)kfs[k].width * kfs[k].height;
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    int64_t count = 0, base = 0;
    float to[3], td[3], tc[3], tdep;
    uint8_t tob;
    for (int k = 0; k < n_kf; ++k) {
        for (int y = 0; y < kfs[k].height; ++y)
            for (int x = 0; x < kfs[k].width; ++x)
                if (orc_pixel_ray(&kfs[k], st, x, y, to, td, tc, &tdep, &tob))
                    cand[count++] = base + (int64_t)y * kfs[k].width + x;
        base += (int64_t)kfs[k].width * kfs[k].height;
    }
    for (int j = 0; j < n; ++j) {
        if (count == 0) {  /* nothing to draw: a ray that misses the box and renders to zero */
            for (int a = 0; a < 3; ++a) {
                o[3 * j + a] = -1.0f;
                d[3 * j + a] = 0.0f;
                rgb[3 * j + a] = 0.0f;
            }
            depth[j] = 0.0f;
            is_obj[j] = 0;
            continue;
        }
        const int64_t pick = cand[(int64_t)(((uint64_t)draws[j] * (uint64_t)count) >> 32)];
        int k = 0;
        int64_t off = pick;
        while (off >= (int64_t)kfs[k].width * kfs[k].height) {
            off -= (int64_t)kfs[k].width * kfs[k].height;
            ++k;
        }
        orc_pixel_ray(&kfs[k], st, (int)(off % kfs[k].width), (int)(off / kfs[k].width), o + 3 * j, d + 3 * j,
                      rgb + 3 * j, depth + j, is_obj + j);
    }
    free(cand);
    return count;
}

/* ========================================================= prior grid
 * §III-A "Normalized mesh generation": the prior density grid is the density
 * output of the NeRF over a cubic grid of resolution R; §III-B refreshes it the
 * same way every m iterations.  Reading: the value of voxel (i, j, k) is the
 * field's density sigma = exp(min(o_0, 15)) at the voxel centre
 * ((i+1/2)/R, (j+1/2)/R, (k+1/2)/R), x fastest -- the convention of the
 * trilinear lookup of Eq. 3. */
void orc_density_grid(const orc_arch *a, const double *theta, int R, double *grid)
{
    const int IN = a->L * a->F, W = a->width, H = a->hidden;
    double *enc = (double *)malloc(sizeof(double) * (size_t)IN);
    double *acts = (double *)malloc(sizeof(double) * (size_t)H * W);
    double out[4];
    for (int k = 0; k < R; ++k)
        for (int j = 0; j < R; ++j)
            for (int i = 0; i < R; ++i) {
                const double p[3] = {(i + 0.5) / R, (j + 0.5) / R, (k + 0.5) / R};
                orc_encode(a, theta, p, enc);
                orc_mlp_forward(a, theta, enc, acts, out);
                grid[((int64_t)k * R + j) * R + i] = exp(out[0] < 15.0 ? out[0] : 15.0);
            }
    free(enc);
    free(acts);
}

/* §III-B "Object State Canonicalization", Eq. 3: for each sampled yaw
 * gamma_g = 2 pi g / n_gamma the object cloud P (n points, object-centred frame,
 * z up) is rotated about z by gamma_g, its extents S_gamma measured, and the
 * normalised cloud P_gamma / S_gamma + 1/2 scored by the summed prior density
 * (trilinear, orc_prior_lookup); the chosen yaw maximises the score.  Reading:
 * "P_gamma / S_gamma + 1/2" centres P_gamma at the midpoint of its extents
 * before the division, so the cloud fills [0, 1]^3; an axis of zero extent
 * maps to 1/2.  Returns the first index of the largest score. */
int orc_canonical_yaw(const double *grid, int R, const double *P, int n, int n_gamma, double *score)
{
    const double two_pi = 6.283185307179586476925286766559;
    double *q = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int best = 0;
    for (int g = 0; g < n_gamma; ++g) {
        const double gamma = two_pi * (double)g / (double)n_gamma;
        const double c = cos(gamma), s = sin(gamma);
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int j = 0; j < n; ++j) {
            const double *x = P + 3 * (int64_t)j;
            double *y = q + 3 * (int64_t)j;
            y[0] = c * x[0] - s * x[1];
            y[1] = s * x[0] + c * x[1];
            y[2] = x[2];
            for (int a = 0; a < 3; ++a) {
                if (y[a] < lo[a]) lo[a] = y[a];
                if (y[a] > hi[a]) hi[a] = y[a];
            }
        }
        double sum = 0.0;
        for (int j = 0; j < n; ++j) {
            double pn[3];
            for (int a = 0; a < 3; ++a) {
                const double S = hi[a] - lo[a];
                pn[a] = S > 0.0 ? (q[3 * (int64_t)j + a] - 0.5 * (lo[a] + hi[a])) / S + 0.5 : 0.5;
            }
            sum += orc_prior_lookup(grid, R, pn);
        }
        score[g] = sum;
        if (sum > score[best])
            best = g;
    }
    free(q);
    return best;
}

/* ============================================================== Reptile
 * §III-A, Eq. 2: after q inner steps on task i, the meta-parameters move toward
 * the task's parameters, theta <- theta + beta (theta_i^(q) - theta).  Reading
 * for a meta-batch of n tasks adapted from the same theta: the batched form of
 * Reptile, theta <- theta + beta (mean_t theta_t^(q) - theta), which is Eq. 2
 * itself for n = 1.  Sum in task order, then the mean, then the step. */
void orc_reptile(int64_t n, double *theta, const double *const *tasks, int n_tasks, double beta)
{
    for (int64_t i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int t = 0; t < n_tasks; ++t)
            sum += tasks[t][i];
        const double mean = sum / (double)n_tasks;
        theta[i] = theta[i] + beta * (mean - theta[i]);
    }
}

/* ============================================================== Philox
 * Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011): each round multiplies counter words
 * 0 and 2 by 0xD2511F53 and 0xCD9E8D57, mixes the 64-bit products' halves with
 * words 1, 3 and the key, and the key is bumped by the Weyl constants
 * 0x9E3779B9 and 0xBB67AE85 between rounds. */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* The library's internal draws, defined here from the generator (a reading;
 * the paper does not say how it draws its uniforms):
 *   key = (seed low 32 bits, seed high 32 bits);
 *   xi_{r,k} = word (k mod 4) of Philox(ctr = (r, k div 4, step, 2 obj)) >> 15, times 2^-17;
 *   u_{r,k}  = ((float)k + xi) / (float)Nr in IEEE single precision (stratified; with 17
 *              random bits k + xi is exact for k < 128, so u stays below 1);
 *   C_rand_r = words 0..2 of Philox(ctr = (r, 0, step, 2 obj + 1)) >> 8, times 2^-24. */
void orc_philox_uniforms(uint64_t seed, uint32_t step, uint32_t obj, int n, int Nr, float *u)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int r = 0; r < n; ++r) {
        for (int k = 0; k < Nr; ++k) {
            uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(k >> 2), step, 2u * obj};
            uint32_t out[4];
            orc_philox4x32_10(ctr, key, out);
            /* 17 random bits: k + xi is exact in FP32 for k < 128, so u < 1 */
            float xi = (float)(out[k & 3] >> 15) * 7.62939453125e-06f;
            volatile float num = (float)k + xi;
            u[(int64_t)r * Nr + k] = num / (float)Nr;
        }
    }
}

void orc_philox_colours(uint64_t seed, uint32_t step, uint32_t obj, int n, float *crand)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int r = 0; r < n; ++r) {
        uint32_t ctr[4] = {(uint32_t)r, 0u, step, 2u * obj + 1u};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        for (int ch = 0; ch < 3; ++ch)
            crand[3 * r + ch] = (float)(out[ch] >> 8) * 5.9604644775390625e-8f;
    }
}
