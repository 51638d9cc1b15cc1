/*
 * mls6_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 CPU implementation of multilevel summation (MLS) for the
 * r^-6 dispersion kernel (Tameling, Springer, Bientinesi, Ismail, "Multilevel
 * Summation for Dispersion", arXiv 1308.4005).  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the GPU
 * library never calls, links or includes anything from this directory.
 *
 * Conventions (shared by the whole oracle):
 *   - The periodic cell is a 3x3 matrix H (row-major); its COLUMNS are the
 *     lattice vectors, x = H s with fractional s in [0,1)^3.  An orthorhombic
 *     box is H = diag(Lx, Ly, Lz).  Grids deform with the cell: grid node mu
 *     on a level with n points per axis sits at X_mu = H (mu / n).
 *   - Physical energy  E = -1/2 sum_i sum_{j,n}' c_i c_j |x_i - x_j + H n|^-6,
 *     i.e. the quadratic form of Eq. (pot-vec-mat-vec) with xi = c (Sec. II.D,
 *     geometric mixing, c_i = sqrt(C6_i)), halved for the double sum and with
 *     the attractive sign of Eq. (disp-pair-pot).  Forces F = -dE/dx.
 *   - Virial W_ab = -dE/d(eps_ab) under the affine strain H -> (I+eps) H with
 *     fractional coordinates (atoms and grid nodes) held fixed.
 *     Order of the six components: xx, yy, zz, xy, xz, yz.
 *   - Grid arrays are x-fastest: index = i + n0*(j + n1*k).
 */
#ifndef MLS6_ORACLE_H
#define MLS6_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Continuity n (1..4) of the smoothing function gamma used by every entry
 * point below (default 2, Eq. gamma): gamma_n is the order-n Taylor
 * polynomial of u^(-1/2) about u = 1, u = rho^12.  Process-wide setting. */
void orc_set_smoothing(int n);
int  orc_get_smoothing(void);

/* Interpolation order p of the nodal basis Phi used by every entry point
 * below: 3 (default, Eq. Phi-Hermite, cubic, support |t| < 2) or 5 (C^1
 * quintic, support |t| < 3).  Process-wide setting. */
void orc_set_order(int p);
int  orc_get_order(void);

/* Closed forms (Sec. II.A.3-5). */
double orc_gamma(double rho);                 /* Eq. (gamma), C^n variant */
double orc_dgamma(double rho);                /* d gamma / d rho */
double orc_gk(int k, int l, double a, double r);   /* Eqs. (g_0), (g_k), (g_l) */
double orc_dgk(int k, int l, double a, double r);  /* d g_k / dr */
double orc_Phi(double t);                     /* Eq. (Phi-Hermite), order p */
double orc_dPhi(double t);                    /* d Phi / dt */

/* Finest-grid size: per axis the multiple of 2^(levels-1) nearest to L/h
 * (ties to the finer grid), at least 2^(levels-1).  Returns 0 on success. */
int orc_grid_dims(const double L[3], double h, int levels, int n_out[3]);

/* Number of doubles orc_eval writes to level_energy: levels + 3
 * ([0] local part, [1] self term, [2..levels+1] per-level grid energies
 *  -1/2 q^k . e^k, [levels+2] total). */

/* Full MLS evaluation.  x: N*3 Cartesian positions, c: N coefficients.
 * Any output pointer may be NULL.  F: N*3, W: 6, eatom: N (per-atom energy
 * -1/2 c_i (e0_i + e_i) + 1/2 c_self c_i^2, which sums to E),
 * level_energy: levels+3 values as described above.
 * r_img: outer radius (absolute length) of the windowed direct image sum of
 * the coarsest-level table (window from 2^(l-1) a to r_img, complement
 * integrated over space); <= 0 selects 2^(l-1) a + 21 V^(1/3), capped so
 * that (coarsest points) x (images) stays near 3e7.
 * Returns 0 on success, <0 on bad arguments. */
int orc_eval(const double H[9], double a, const int n[3], int levels, double r_img,
             int64_t N, const double* x, const double* c,
             double* E, double* F, double* W, double* eatom, double* level_energy);

/* Same evaluation restricted to the atoms listed in idx (n_idx of them):
 * F (n_idx*3) and eatom (n_idx) for those atoms only; grid_energy receives
 * the grid part -1/2 sum_k q^k.e^k (all atoms).  The local part is computed
 * only for the listed atoms, so this is usable at large N. */
int orc_eval_sample(const double H[9], double a, const int n[3], int levels, double r_img,
                    int64_t N, const double* x, const double* c,
                    int64_t n_idx, const int64_t* idx,
                    double* F, double* eatom, double* grid_energy);

/* Local part only (Eq. g_0) for the atoms listed in idx: e0 (n_idx) is
 * sum_{j,n: r<a} c_j g_0(r) and F (n_idx*3) the local force.  Either output
 * may be NULL. */
int orc_local(const double H[9], double a, int64_t N, const double* x, const double* c,
              int64_t n_idx, const int64_t* idx, double* e0, double* F);

/* Local part for the listed atoms by the two loop forms, for checking one
 * against the other: linked cells (the form every other entry point uses)
 * and all atoms x all images.  e0 (n_idx), F (n_idx*3) and the per-atom
 * virial records W (n_idx*6, 1/2 c_i c_j g_0'/r d (x) d summed over j) may
 * be NULL. */
int orc_local_cells(const double H[9], double a, int64_t N, const double* x, const double* c,
                    int64_t n_idx, const int64_t* idx, double* e0, double* F, double* W);
int orc_local_allpairs(const double H[9], double a, int64_t N, const double* x,
                       const double* c, int64_t n_idx, const int64_t* idx, double* e0,
                       double* F, double* W);

/* Stage export: writes, level after level, q^k, e^k and e^{k,tot} (each of
 * n_k points) for k = 1..levels into out (3 * sum_k n_k doubles). */
int orc_grids(const double H[9], double a, const int n[3], int levels, double r_img,
              int64_t N, const double* x, const double* c, double* out);

/* Coarsest-level periodic tables: T (n_l points) and the six virial tables
 * V_ab (6 * n_l, component-major), for a coarsest grid of nl points. */
int orc_top_table(const double H[9], double a, const int nl[3], int levels, double r_img,
                  double* T, double* V);

/* Exact periodic sum sum_{j,n}' |x_j - x_i + H n|^-6 by windowed direct
 * image summation (window from r_img/4 to r_img) plus the integral of the
 * complement.  r_img >= 30 x (longest cell vector) keeps the aliasing error
 * of the windowed split below ~1e-15 relative.  Any output may be NULL.
 * F: N*3, W: 6. */
int orc_brute(const double H[9], double r_img, int64_t N, const double* x, const double* c,
              double* E, double* F, double* W);

/* OpenMP threads used by the loops above (<=0: library default). */
void orc_set_threads(int n);
int  orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
