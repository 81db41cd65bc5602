/*
 * sclbm_oracle.h -- plain FP64 CPU oracle for the stochastic-collocation
 * lattice Boltzmann (SC-LBM) hot path of arXiv:2508.18202.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py use it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Conventions (all arrays caller-owned host memory):
 *   cell index     c = x + nx*(y + ny*z)
 *   populations    f[i*ncell + c], i = 0..18, unshifted FP64, "natural"
 *                  layout: f_i(x, t) after streaming into time level t.
 *   flags          uint8 per cell, 0 = fluid, 1 = solid, 2 = beyond the
 *                  mantle of a circular domain (velocity boundary).
 *   faces          0:-x 1:+x 2:-y 3:+y 4:-z 5:+z
 *   face kinds     0 VELOCITY, 1 OUTFLOW, 2 BOUNCE_BACK, 3 FREE_SLIP, 4 PERIODIC
 * Every function returns 0 on success and a negative value on bad input.
 */
#ifndef SCLBM_ORACLE_H
#define SCLBM_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;
  int bc[6];
  double tau0;      /* molecular relaxation time, tau0 = 3 nu + 1/2      */
  double csmag;     /* Smagorinsky constant C_S, 0 = plain BGK           */
  int ramp_steps;   /* T_r of the start-up ramp, 0 = impulsive           */
  double force[3];  /* body force (Guo); zero for the method, used only by
                       the Poiseuille pin                                 */
  int collision;    /* 0: BGK, second-order equilibrium; 1: recursive
                       regularized, third-order D3Q19 equilibrium         */
} oc_params;

int oc_lattice(int* cx, int* cy, int* cz, double* w, int* opp);
int oc_equilibrium(double rho, const double* u, double* feq);
int oc_collide_cell(const oc_params* p, const double* f, double* fpost, double* tau_eff);
/* Third-order D3Q19 Hermite equilibrium of the recursive regularized model. */
int oc_equilibrium3(double rho, const double* u, double* feq);
double oc_ramp(int ramp_steps, long long m);

int oc_init_equilibrium(const oc_params* p, const uint8_t* flags,
                        const double* rho, const double* u, double* f);
int oc_run(const oc_params* p, const uint8_t* flags, const double* uin,
           double* f, long long n0, int n_steps);
int oc_macros(const oc_params* p, const uint8_t* flags, const double* f,
              double* rho, double* u);

int oc_splitmix64(uint64_t seed, int n, uint64_t* out);
int oc_geometry(int nx, int ny, int nz, uint64_t seed, int n_buildings,
                int fp_min, int fp_max, int h_min, int h_max,
                const int32_t* boxes, int n_boxes, uint8_t* flags);
/* Circular domain: flag 2 for every cell whose centre lies more than radius
 * from the axis (nx/2, ny/2); links into such cells take the velocity rule. */
int oc_mark_mantle(int nx, int ny, int nz, double radius, uint8_t* flags);
int oc_probe_columns(int nx, int ny, int nz, uint64_t seed, const uint8_t* flags,
                     int n, int32_t* xy);
int oc_probe_points(int nx, int ny, int nz, uint64_t seed, const uint8_t* flags,
                    int n, int32_t* xyz);
int oc_inflow(int nz, double u_ref, double xi, double alpha, double H,
              double theta_deg, double* uin);

int oc_quadrature(int rule, int d, int level, const double* lo, const double* hi,
                  int* n_out, double* Z, double* w, int cap);

int oc_moments_two_pass(int nq, long long ncell, const double* a, const double* Q,
                        double* mean, double* stdev, long long* n_clamped);
int oc_profiles(int nq, int nx, int ny, int nz, const double* a, const double* Q,
                int n_p, const int32_t* xy, double* prof, double* prof_nodes);
int oc_gpc_basis_size(int d, int degree);
int oc_gpc_basis(int d, int degree, int nq, const double* s, double* phi);
int oc_gpc_basis_family(int d, int degree, int family, int nq, const double* s, double* phi);
int oc_inflow_log(int nz, double u_ref, double xi, double z0, double H, double theta_deg, double* uin);
int oc_gpc_project(int nq, int P, long long ncell, const double* a,
                   const double* Q, const double* phi, double* coef);

int oc_tangent_run(const oc_params* p, const uint8_t* flags, const double* uin,
                   const double* duin, double* f, int n_steps, int n_probe,
                   const int32_t* probes, const double* u_target,
                   double* loss, double* dloss, double* u_probe);

#ifdef __cplusplus
}
#endif
#endif
