/*
 * abc_oracle.h -- C interface of the CPU oracle (test infrastructure only;
 * see abc_oracle.c for the definitions and the paper passages they follow).
 */
#ifndef ABC_ORACLE_H
#define ABC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float oracle_uniform(uint32_t w);
float oracle_log2x(float x);
float oracle_exp2x(float y);
void oracle_sincospix(float v, float* sin_out, float* cos_out);
void oracle_box_muller(uint32_t w_radius, uint32_t w_angle, float z[2]);
void oracle_day_pair_normals(uint64_t seed, uint32_t stream, uint64_t i, uint32_t k, float z[10]);
void oracle_prior_draw(const float lo[8], const float hi[8], uint64_t seed, uint32_t stream,
                       uint64_t i, float theta[8]);
int32_t oracle_clamp_count(float x, int32_t c);
float oracle_infection_rate(const float theta[8], int32_t U);
void oracle_hazard(const int32_t X[6], const float theta[8], int64_t P, float h[5]);
void oracle_step(const int32_t X[6], const float theta[8], int64_t P, const float z[5],
                 int variance_literal, int32_t n_out[5], int32_t Y[6]);
int oracle_init_state(const float theta[8], const int32_t ard0[3], int64_t P, int32_t X[6]);
int oracle_simulate(const float theta[8], const int32_t ard0[3], int32_t T, int64_t P,
                    uint64_t seed, uint32_t stream, uint64_t i, int variance_literal,
                    int32_t* traj);
uint64_t oracle_sq_distance(const int32_t* traj, const int32_t* observed, int32_t T);
double oracle_distance_from_sq(uint64_t acc);
int oracle_abc(const float lo[8], const float hi[8], const int32_t* observed, int32_t T, int64_t P,
               double eps, uint64_t n_samples, uint64_t seed, uint32_t stream, uint64_t first_index,
               int variance_literal, int n_threads,
               uint64_t* idx_out, float* theta_out, double* dist_out, uint64_t capacity,
               uint64_t* n_accepted, double* dist_all);
void oracle_log2x_batch(const float* x, float* y, uint64_t n);
void oracle_exp2x_batch(const float* x, float* y, uint64_t n);
void oracle_sincospix_batch(const float* v, float* s, float* c, uint64_t n);
void oracle_uniform_batch(const uint32_t* w, float* u, uint64_t n);
void oracle_normals_batch(uint64_t seed, uint32_t stream, uint64_t first, uint64_t n, uint32_t k,
                          float* z);
void oracle_prior_batch(const float lo[8], const float hi[8], uint64_t seed, uint32_t stream,
                        uint64_t first, uint64_t n, float* theta);
void oracle_step_batch(const int32_t* X, const float* theta, int64_t P, const float* z,
                       int variance_literal, uint64_t m, int32_t* n_out, int32_t* Y);

#ifdef __cplusplus
}
#endif
#endif
