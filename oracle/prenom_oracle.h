/* FP64 CPU oracle of the PRENOM object-NeRF training step (arXiv 2503.01582).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  Nothing on the product
 * path may include, link or call this code; it shares no code, header, table
 * or constant generator with the CUDA library.
 *
 * Every routine restates one step of the paper (or of the method it cites for
 * that step) literally, in double precision, sequentially, with no blocking,
 * fusion or reordering:
 *   - §III-B "Probabilistic Ray Sampling": equal-interval probes, occupancy
 *     (Eq. 4), termination probability as a literal product (Eq. 5), discrete
 *     CDF (Eq. 6), inverse transform sampling, uniform fallback for escaping
 *     rays;
 *   - §III-B "Object-level NeRFs": multiresolution hash encoding (the cited
 *     instant-NGP method) and a shallow bias-free MLP;
 *   - §III-B "Volume Rendering": colour, depth and opacity compositing (Eq. 7),
 *     the losses L_c, L_d, L_sigma (Eq. 8) and their weighted sum (Eq. 9);
 *   - reverse-mode gradients of that loss and the Adam update that the
 *     paper's last sentence of §III-B names;
 *   - §III-A "Meta-learning": the Reptile outer update (Eq. 2) after inner
 *     training steps (Eq. 1);
 *   - §III-A "Normalized mesh generation" / §III-B: the prior density grid
 *     from the field, and the yaw canonicalisation of Eq. 3;
 *   - §III-B "Training Data": object-frame training rays from RGB-D
 *     keyframes, masks and poses.
 * Readings of points the paper leaves open are listed beside each routine.
 *
 * Parameter vector layout (shared by contract with the library's interface,
 * not by code): hash tables level by level, entry-major with F features per
 * entry, each level padded to a multiple of 8 entries, then one row-major
 * (out x in) matrix per MLP layer: W_1 [W][L*F], W_2..W_H [W][W], W_out [4][W].
 */
#ifndef PRENOM_ORACLE_H
#define PRENOM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int L;       /* levels */
    int F;       /* features per level */
    int log2T;   /* log2 of the hash table size T */
    int n_min;   /* coarsest resolution */
    int n_max;   /* finest resolution */
    int width;   /* hidden width W */
    int hidden;  /* hidden layers H (>= 1) */
    double lambda_d;
    double lambda_sigma;
} orc_arch;

/* ---- hash-grid geometry (instant-NGP multiresolution grid) ---- */
int     orc_level_res(const orc_arch *a, int l);
int     orc_level_dense(const orc_arch *a, int l);
int64_t orc_level_entries(const orc_arch *a, int l);
int64_t orc_level_offset(const orc_arch *a, int l);  /* in floats */
int64_t orc_n_hash_params(const orc_arch *a);
int64_t orc_n_mlp_params(const orc_arch *a);
int64_t orc_param_count(const orc_arch *a);
int64_t orc_mlp_offset(const orc_arch *a, int layer); /* in floats, 0..H */
uint32_t orc_grid_index(const orc_arch *a, int l, uint32_t cx, uint32_t cy, uint32_t cz);

/* ---- sampling (§III-B) ---- */
int    orc_ray_box(const double *o, const double *d, double *tn, double *tf);
double orc_prior_lookup(const double *grid, int R, const double *x);
void   orc_cdf_invert(const double *cdf, int Nc, const double *u, int Nr,
                      double tn, double tf, int *bins, double *t);
int    orc_sample_ray(const double *grid, int R, const double *o, const double *d,
                      int Nc, int Nr, double eps, const double *u,
                      double *probe_sigma, double *rho_term, double *cdf,
                      int *bins, double *t, double *tn, double *tf);

/* ---- field ---- */
void orc_encode(const orc_arch *a, const double *theta, const double *p, double *enc);
void orc_encode_backward(const orc_arch *a, const double *p, const double *denc, double *grad);
void orc_mlp_forward(const orc_arch *a, const double *theta, const double *enc,
                     double *acts, double *out4);
void orc_mlp_backward(const orc_arch *a, const double *theta, const double *enc,
                      const double *acts, const double *dout4, double *grad, double *denc);

/* ---- rendering and loss (§III-B) ---- */
void   orc_composite(int Nr, const double *sigma, const double *c, const double *t, double tf,
                     double *w, double *C, double *D, double *A);
void   orc_composite_backward(int Nr, const double *sigma, const double *c, const double *t,
                              double tf, const double *gC, double gD, double gA,
                              double *dsigma, double *dc);
double orc_ray_loss(int is_obj, const double *C, double D, double A, const double *Cgt,
                    double Dgt, const double *crand, double lambda_d,
                    double *gC, double *gD, double *gA);

/* ---- whole batch: sampling -> encoding -> MLP -> compositing -> loss -> gradients ---- */
double orc_batch(const orc_arch *a, const double *theta, const double *grid, int R,
                 int n, const double *o, const double *d, const double *rgb,
                 const double *depth, const uint8_t *is_obj, const double *crand,
                 const double *u, const double *t_in, int Nc, int Nr, double eps,
                 const double *upstream,
                 double *out_rgb, double *out_depth, double *out_acc,
                 int *out_bins, double *out_t, double *out_sigma, double *grad);

/* ---- Adam (§III-B, last sentence) ---- */
void orc_adam(int64_t n, double *theta, double *m, double *v, const double *g, int step,
              double lr, double beta1, double beta2, double eps);

/* ---- training rays from RGB-D keyframes (§III-B "Training Data") ---- */
typedef struct {
    int width, height;
    const uint8_t *rgb;   /* [H][W][3] */
    const float *depth;   /* [H][W] z-depth */
    const int32_t *mask;  /* [H][W] instance ids */
    float fx, fy, cx, cy;
    float R_wc[9];        /* camera-to-world rotation, row-major */
    float t_wc[3];        /* camera centre */
} orc_keyframe;
typedef struct {
    int instance;
    float R_wo[9];        /* object-to-world rotation, row-major */
    float centre[3];
    float size[3];
} orc_object_state;
int     orc_pixel_ray(const orc_keyframe *kf, const orc_object_state *st, int x, int y, float *o, float *d,
                      float *rgb, float *depth, uint8_t *is_obj);
int64_t orc_make_rays(const orc_keyframe *kfs, int n_kf, const orc_object_state *st, int n, const uint32_t *draws,
                      float *o, float *d, float *rgb, float *depth, uint8_t *is_obj);

/* ---- prior density grid (§III-A mesh generation, §III-B refresh) and Eq. 3 ---- */
void orc_density_grid(const orc_arch *a, const double *theta, int R, double *grid);
int  orc_canonical_yaw(const double *grid, int R, const double *P, int n, int n_gamma, double *score);

/* ---- Reptile outer update (§III-A, Eq. 2; batched over n_tasks) ---- */
void orc_reptile(int64_t n, double *theta, const double *const *tasks, int n_tasks, double beta);

/* ---- Philox4x32-10 counter-based generator (Salmon et al., SC 2011) ---- */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out);
void orc_philox_uniforms(uint64_t seed, uint32_t step, uint32_t obj, int n, int Nr, float *u);
void orc_philox_colours(uint64_t seed, uint32_t step, uint32_t obj, int n, float *crand);

#ifdef __cplusplus
}
#endif
#endif
