/*
 * cwthf_oracle.h -- entry points of the fp64 CPU oracle (test infrastructure).
 * Only the tests, the smoke check and bench.py's CPU-baseline leg load it.
 * Arrays are host memory, row-major [z][y][x] with x fastest; positions are
 * float [np][3] (x, y, z).  Every function returns one of the ORC_* codes.
 */
#ifndef CWTHF_ORACLE_H
#define CWTHF_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_E_ARG 1
#define ORC_E_OVERFLOW 2
#define ORC_E_INEXACT 3
#define ORC_E_NOMEM 4
#define ORC_E_CAPACITY 5

int orc_quantise(const float *pos, int64_t np, double L, int ng, int64_t *q);
int orc_cic(const float *pos, const float *mass, double mass_unit, int64_t np, double L, int ng,
            int64_t *grid, int64_t *mtot_q);
double orc_wavelet(double w, double r2);
void orc_kernel(int ng, double L, double w, double *K);
int orc_dft1d(double *re, double *im, int n, int sign);
int orc_dft3d(double *re, double *im, int n, int sign);
int orc_cwt(const int64_t *grid, int ng, double L, double mass_unit, double w, double *C);
int orc_cwt_direct(const int64_t *grid, int ng, double L, double mass_unit, double w, double *C);
int orc_cwt_stencil(const int64_t *grid, int ng, double L, double mass_unit, double w, int R, double *C);
int orc_cwt_stencil_at(const int64_t *grid, int ng, double L, double mass_unit, double w, int R, const int64_t *nodes,
                       int64_t n_nodes, double *out);
int orc_cwt_at(const int64_t *grid, int ng, double L, double mass_unit, double w, const int64_t *nodes,
               int64_t n_nodes, double *out);
int orc_parent(const float *C, int ng, int32_t *parent);
int orc_segment(const float *C, int ng, float cwt_min, int32_t *label);
int orc_assign(const float *pos, const float *mass, double mass_unit, int64_t np, double L, int ng,
               const int32_t *label, const float *C, double dens_th, int64_t particle_th,
               int32_t *halo_id, int64_t cap, int64_t *seed_out, int64_t *npart_out, int64_t *ncell_out,
               double *mass_out, double *centre_out, float *peak_out, int64_t *n_halo);
float orc_corrected_peak(const float *C, int ng, int64_t s, int ng_next);
int orc_cross_scale(const float *C, int ng, int64_t s, const float *Cn, int ng_next);
int orc_multiscale(const float *pos, const float *mass, double mass_unit, int64_t np, double L, int n_scales,
                   const int *ngs, const float *const *fields, float cwt_min, double dens_th, int64_t particle_th,
                   const float *vel, double G, int max_iter, int32_t *halo_id, int64_t cap, int32_t *scale_out,
                   int64_t *seed_out, int64_t *npart_out, int64_t *ncell_out, double *mass_out, double *centre_out,
                   float *peak_out, int64_t *n_halo, double *margin_out);

int orc_unbind(const float *pos, const float *vel, const float *mass, double mass_unit, int64_t np, double L,
               double G, const int32_t *group, int64_t n_groups, int max_iter, int32_t *out_group, int64_t *out_n,
               int32_t *out_iter, double *out_margin);
#endif
