// Host side of the multilevel summation library: parameter validation, grid
// hierarchy, stencil and coarsest-level tables (all FP64), device workspace.
//
// Paper: arXiv 1308.4005.  Kernel split Eqs. (gamma), (g_0), (g_k), (g_l);
// level tables Sec. II.A.4 (same arguments on every grid, scaled by
// 2^(-6(k-1))); periodic coarsest level Sec. II.C.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "mls6_internal.h"

namespace mls6 {

// Smoothing function of continuity C^n (Sec. II.A.3): with u = rho^12 the
// kernel rho^-6 is u^(-1/2), and gamma_n is its Taylor polynomial about
// u = 1 to order n, written out in powers of u, gamma_n = sum_k c_k u^k for
// rho < 1 and rho^-6 above.  n = 2 is Eq. (gamma): 15/8 - 5/4 rho^12 +
// 3/8 rho^24; n = 1, 3, 4 are the other continuities of Sec. III.B built
// the same way.
Smooth smooth_coefficients(int n) {
  Smooth s;
  s.n = n;
  for (int k = 0; k < 5; ++k) s.c[k] = 0.0;
  // sum_{j<=n} binom(-1/2, j) (u - 1)^j, expanded: c_k += binom(-1/2, j) binom(j, k) (-1)^(j-k)
  double bj = 1.0;
  for (int j = 0; j <= n; ++j) {
    if (j > 0) bj *= (-0.5 - (j - 1)) / j;
    double bjk = 1.0;  // binom(j, k)
    for (int k = 0; k <= j; ++k) {
      if (k > 0) bjk = bjk * (j - k + 1) / k;
      s.c[k] += bj * bjk * (((j - k) & 1) ? -1.0 : 1.0);
    }
  }
  return s;
}

double gamma_fn(const Smooth& s, double rho) {
  if (rho < 1.0) {
    double r2 = rho * rho, r4 = r2 * r2, u = r4 * r4 * r4;
    double v = s.c[s.n];
    for (int k = s.n - 1; k >= 0; --k) v = v * u + s.c[k];
    return v;
  }
  double r2 = rho * rho;
  return 1.0 / (r2 * r2 * r2);
}

// gamma'(rho)/rho = 12 rho^10 sum_k k c_k u^(k-1) (rho < 1), -6 rho^-8 (rho >= 1).
double dgamma_over_rho(const Smooth& s, double rho) {
  double r2 = rho * rho;
  if (rho < 1.0) {
    double r4 = r2 * r2, u = r4 * r4 * r4, r10 = r4 * r4 * r2;
    double v = s.n * s.c[s.n];
    for (int k = s.n - 1; k >= 1; --k) v = v * u + k * s.c[k];
    return 12.0 * r10 * v;
  }
  double r8 = r2 * r2 * r2 * r2;
  return -6.0 / r8;
}

static double sgamma(const Smooth& sm, double s, double r) {  // s^-6 gamma(r/s)
  double s2 = s * s;
  return gamma_fn(sm, r / s) / (s2 * s2 * s2);
}

static double sdgamma_over_r(const Smooth& sm, double s, double r) {  // (d/dr s^-6 gamma(r/s)) / r
  double s2 = s * s;
  return dgamma_over_rho(sm, r / s) / (s2 * s2 * s2 * s2);
}

// Eqs. (g_0), (g_k), (g_l); exactly 0 beyond the cutoff of levels k < l.
double g_level(const Smooth& sm, int k, int l, double a, double r) {
  if (k == 0) {
    if (r >= a) return 0.0;
    double r2 = r * r;
    return 1.0 / (r2 * r2 * r2) - sgamma(sm, a, r);
  }
  double si = std::ldexp(a, k - 1);
  if (k == l) return sgamma(sm, si, r);
  double so = std::ldexp(a, k);
  if (r >= so) return 0.0;
  return sgamma(sm, si, r) - sgamma(sm, so, r);
}

double dg_level_over_r(const Smooth& sm, int k, int l, double a, double r) {
  if (k == 0) {
    if (r >= a) return 0.0;
    double r2 = r * r;
    return -6.0 / (r2 * r2 * r2 * r2) - sdgamma_over_r(sm, a, r);
  }
  double si = std::ldexp(a, k - 1);
  if (k == l) return sdgamma_over_r(sm, si, r);
  double so = std::ldexp(a, k);
  if (r >= so) return 0.0;
  return sdgamma_over_r(sm, si, r) - sdgamma_over_r(sm, so, r);
}

// ------------------------------------------------------------------------
// Ewald summation of the coarsest-level lattice sums.
//
// g_l is split as (g_l - S) + S with S(r) = r^-6 P(3, beta^2 r^2), the smooth
// (Gaussian-damped) part of r^-6; P(3,x) = 1 - e^-x (1 + x + x^2/2) is the
// regularised lower incomplete gamma function.  Beyond 2^(l-1) a,
// g_l - S = r^-6 e^-x (1 + x + x^2/2) decays like a Gaussian and is summed
// in real space; S is summed in reciprocal space by Poisson summation with
// its Fourier transform
//   S^(k) = (pi^1.5 beta^3 / 3) [(1 - 2 b^2) e^-b^2 + 2 sqrt(pi) b^3 erfc(b)],
//   b = k / (2 beta),
// obtained from r^-6 = (1/2) int_0^inf t^2 e^-t r^2 dt restricted to
// t < beta^2.  The strain derivative of the reciprocal sum follows from
// k -> (1+eps)^-T k and V -> V det(1+eps) at fixed fractional coordinates.
// ------------------------------------------------------------------------

// S(r) and S'(r)/r.
static void smooth_part(double r, double beta, double* S, double* dS_over_r) {
  double x = beta * beta * r * r;
  if (x < 2.0) {
    // S = beta^6 e^-x sum_k x^k/(k+3)!,  S'/r = -6 beta^8 e^-x sum_k x^k/(k+4)!
    double t3 = 1.0 / 6.0, t4 = 1.0 / 24.0, s3 = 0.0, s4 = 0.0, xk = 1.0;
    for (int k = 0; k < 40; ++k) {
      s3 += xk * t3;
      s4 += xk * t4;
      xk *= x;
      t3 /= (k + 4);
      t4 /= (k + 5);
    }
    double ex = std::exp(-x), b2 = beta * beta, b6 = b2 * b2 * b2;
    *S = b6 * ex * s3;
    *dS_over_r = -6.0 * b6 * b2 * ex * s4;
    return;
  }
  double r2 = r * r, r6 = r2 * r2 * r2, ex = std::exp(-x);
  double P = 1.0 - ex * (1.0 + x + 0.5 * x * x);
  *S = P / r6;
  *dS_over_r = -6.0 * P / (r6 * r2) + beta * beta * x * x * ex / r6;
}

static double Shat(double k, double beta) {
  double b = k / (2.0 * beta);
  double c = std::pow(M_PI, 1.5) * beta * beta * beta / 3.0;
  return c * ((1.0 - 2.0 * b * b) * std::exp(-b * b) + 2.0 * std::sqrt(M_PI) * b * b * b * std::erfc(b));
}

static double dShat_dk(double k, double beta) {
  double b = k / (2.0 * beta);
  double dSdb = 2.0 * std::pow(M_PI, 1.5) * beta * beta * beta * b *
                (std::sqrt(M_PI) * b * std::erfc(b) - std::exp(-b * b));
  return dSdb / (2.0 * beta);
}

static void coarse_tables_impl(const Smooth& sm, const double L[3], const int nl[3], int l,
                               double a, double* T, double* V) {
  const double Rl = std::ldexp(a, l - 1);
  const double vol = L[0] * L[1] * L[2];
  const double Rc = std::max(3.8 * std::cbrt(vol), Rl);
  const double beta = 7.5 / Rc;
  const double kc = 13.0 * beta;
  const long np = (long)nl[0] * nl[1] * nl[2];
  double hl[3];
  for (int d = 0; d < 3; ++d) hl[d] = L[d] / nl[d];

  // reciprocal vectors inside kc
  struct KV {
    int j[3];
    double s, ds;  // S^(|k|), S^'(|k|)/|k| (0 at k = 0)
    double k[3];
  };
  std::vector<KV> ks;
  int J[3];
  for (int d = 0; d < 3; ++d) J[d] = (int)std::ceil(kc * L[d] / (2.0 * M_PI));
  for (int j2 = -J[2]; j2 <= J[2]; ++j2)
    for (int j1 = -J[1]; j1 <= J[1]; ++j1)
      for (int j0 = -J[0]; j0 <= J[0]; ++j0) {
        double k3[3] = {2.0 * M_PI * j0 / L[0], 2.0 * M_PI * j1 / L[1], 2.0 * M_PI * j2 / L[2]};
        double kk = std::sqrt(k3[0] * k3[0] + k3[1] * k3[1] + k3[2] * k3[2]);
        if (kk > kc) continue;
        KV v;
        v.j[0] = j0;
        v.j[1] = j1;
        v.j[2] = j2;
        v.s = Shat(kk, beta);
        v.ds = kk > 0.0 ? dShat_dk(kk, beta) / kk : 0.0;
        for (int d = 0; d < 3; ++d) v.k[d] = k3[d];
        ks.push_back(v);
      }

  int M[3];
  for (int d = 0; d < 3; ++d) M[d] = (int)std::ceil(Rc / L[d]) + 1;
  for (long m = 0; m < np; ++m) {
    long m0 = m % nl[0], m1 = (m / nl[0]) % nl[1], m2 = m / ((long)nl[0] * nl[1]);
    double X[3] = {m0 * hl[0], m1 * hl[1], m2 * hl[2]};
    double t = 0.0, w[6] = {0, 0, 0, 0, 0, 0};
    // real space
    for (int i2 = -M[2]; i2 <= M[2]; ++i2)
      for (int i1 = -M[1]; i1 <= M[1]; ++i1)
        for (int i0 = -M[0]; i0 <= M[0]; ++i0) {
          double r3[3] = {X[0] + i0 * L[0], X[1] + i1 * L[1], X[2] + i2 * L[2]};
          double r = std::sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
          if (r >= Rc) continue;
          double f, fp;
          if (r >= Rl) {
            double x = beta * beta * r * r, ex = std::exp(-x), r2 = r * r, r6 = r2 * r2 * r2;
            double Q = ex * (1.0 + x + 0.5 * x * x);
            f = Q / r6;
            fp = -6.0 * Q / (r6 * r2) - beta * beta * x * x * ex / r6;
          } else {
            double S, dS;
            smooth_part(r, beta, &S, &dS);
            f = sgamma(sm, Rl, r) - S;
            fp = sdgamma_over_r(sm, Rl, r) - dS;
          }
          t += f;
          w[0] += fp * r3[0] * r3[0];
          w[1] += fp * r3[1] * r3[1];
          w[2] += fp * r3[2] * r3[2];
          w[3] += fp * r3[0] * r3[1];
          w[4] += fp * r3[0] * r3[2];
          w[5] += fp * r3[1] * r3[2];
        }
    // reciprocal space
    double tr = 0.0, wr[6] = {0, 0, 0, 0, 0, 0};
    for (const KV& v : ks) {
      double ph = 2.0 * M_PI * ((double)v.j[0] * m0 / nl[0] + (double)v.j[1] * m1 / nl[1] +
                                (double)v.j[2] * m2 / nl[2]);
      double cs = std::cos(ph);
      tr += v.s * cs;
      wr[0] += (-v.s - v.ds * v.k[0] * v.k[0]) * cs;
      wr[1] += (-v.s - v.ds * v.k[1] * v.k[1]) * cs;
      wr[2] += (-v.s - v.ds * v.k[2] * v.k[2]) * cs;
      wr[3] += (-v.ds * v.k[0] * v.k[1]) * cs;
      wr[4] += (-v.ds * v.k[0] * v.k[2]) * cs;
      wr[5] += (-v.ds * v.k[1] * v.k[2]) * cs;
    }
    T[m] = t + tr / vol;
    if (V)
      for (int c = 0; c < 6; ++c) V[c * np + m] = w[c] + wr[c] / vol;
  }
}

static int grid_dims_impl(const double box[3], double h, int levels, int n_out[3]) {
  if (!box || !n_out) return MLS6_ERR_ARG;
  if (!(h > 0.0) || !std::isfinite(h)) return MLS6_ERR_ARG;
  if (levels < 1 || levels > kMaxLevels) return MLS6_ERR_GRID;
  long m = 1L << (levels - 1);
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) return MLS6_ERR_BOX;
    double u = box[d] / h / (double)m;
    if (u > 1e6) return MLS6_ERR_SIZE;
    long lo = (long)std::floor(u), hi = lo + 1;
    long pick = (u - (double)lo < (double)hi - u) ? lo : hi;  // tie -> finer
    if (pick < 1) pick = 1;
    n_out[d] = (int)(pick * m);
  }
  // the grid kernels index nodes with 32-bit integers
  if ((double)n_out[0] * n_out[1] * n_out[2] > 2147483647.0) return MLS6_ERR_SIZE;
  return MLS6_OK;
}

static void free_plan(Plan* p) {
  if (!p) return;
  void* ptrs[] = {p->d_pos_w, p->d_cell_of, p->d_cell_count, p->d_cell_start, p->d_sorted,
                  p->d_sorted_idx, p->d_e0, p->d_floc, p->d_rows, p->d_wv, p->d_top_T,
                  p->d_top_V, p->d_epart, p->d_wpart, p->d_out, p->d_flag, p->d_scan,
                  p->d_q1fx, p->d_tcw, p->d_lbw, p->d_lbpot, p->d_mma_rows, p->d_mma_bv,
                  p->d_mma_be};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int k = 1; k <= kMaxLevels; ++k) {
    if (p->d_q[k]) cudaFree(p->d_q[k]);
    if (p->d_e[k]) cudaFree(p->d_e[k]);
    if (p->d_et[k] && p->d_et[k] != p->d_e[k]) cudaFree(p->d_et[k]);
  }
  if (p->h_out) cudaFreeHost(p->h_out);
  for (int i = 0; i < Plan::kStages; ++i) {
    if (p->ev_s[i]) cudaEventDestroy(p->ev_s[i]);
    if (p->ev_e[i]) cudaEventDestroy(p->ev_e[i]);
  }
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  cudaEvent_t evs[] = {p->ev_in, p->ev_out, p->ev_fork, p->ev_join};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (p->cs) cudaStreamDestroy(p->cs);
  if (p->cs2) cudaStreamDestroy(p->cs2);
  delete p;
}

}  // namespace mls6

using namespace mls6;

extern "C" {

int mls6_grid_dims(const double box[3], double h, int levels, int n_out[3]) {
  return grid_dims_impl(box, h, levels, n_out);
}

int mls6_coarse_tables(const double box[3], const int nl[3], int levels, double a, double* T,
                       double* V) {
  if (!box || !nl || !T || levels < 1 || levels > kMaxLevels || !(a > 0.0)) return MLS6_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) return MLS6_ERR_BOX;
    if (nl[d] < 1) return MLS6_ERR_GRID;
  }
  coarse_tables_impl(smooth_coefficients(2), box, nl, levels, a, T, V);
  return MLS6_OK;
}

int mls6_auto_levels(const double box[3], double h) {
  if (!box) return MLS6_ERR_ARG;
  int n1[3];
  int rc = grid_dims_impl(box, h, 1, n1);
  if (rc) return rc;
  int best = 1;
  for (int l = 2; l <= kMaxLevels; ++l) {
    if (grid_dims_impl(box, h, l, n1)) break;
    const int c = std::min(n1[0], std::min(n1[1], n1[2])) >> (l - 1);
    if (c < 4) break;
    best = l;
  }
  return best;
}

int mls6_plan(mls6_plan_t** out, const double box[3], int64_t N, double a, double h, int levels,
              int order, int precision) {
  return mls6_plan_ex(out, box, N, a, h, levels, order, precision, nullptr);
}

int mls6_plan_ex(mls6_plan_t** out, const double box[3], int64_t N, double a, double h,
                 int levels, int order, int precision, const mls6_plan_options* opts) {
  if (!out) return MLS6_ERR_ARG;
  *out = nullptr;
  const int continuity = (opts && opts->continuity) ? opts->continuity : 2;
  const int stencil = opts ? opts->stencil : 0;
  if (continuity < 1 || continuity > 4 || stencil < 0 || stencil > 2) return MLS6_ERR_ARG;
  if (!box || N < 0 || N > (int64_t)1 << 30 || !(a > 0.0) || !std::isfinite(a)) return MLS6_ERR_ARG;
  if (precision != MLS6_FP64 && precision != MLS6_FP32 && precision != MLS6_MIXED)
    return MLS6_ERR_ARG;
  if (order != 3 && order != 5) return MLS6_ERR_ORDER;
  if (levels == 0) {
    levels = mls6_auto_levels(box, h);
    if (levels < 0) return levels;
  }
  int n1[3];
  int rc = grid_dims_impl(box, h, levels, n1);
  if (rc) return rc;

  Plan* p = new (std::nothrow) Plan();
  if (!p) return MLS6_ERR_NOMEM;
  for (int d = 0; d < 3; ++d) p->L[d] = box[d];
  p->a = a;
  p->levels = levels;
  p->prec = precision;
  p->N = N;
  p->stream = 0;
  p->sm = smooth_coefficients(continuity);
  p->stencil_req = stencil;
  p->order = order;
  p->c_self = gamma_fn(p->sm, 0.0) / std::pow(a, 6.0);
  for (int k = 1; k <= levels; ++k) {
    Level& lv = p->lv[k];
    lv.np = 1;
    for (int d = 0; d < 3; ++d) {
      lv.n[d] = n1[d] >> (k - 1);
      lv.h[d] = box[d] / lv.n[d];
      lv.np *= lv.n[d];
    }
  }
  // cell list: width >= a/kCellDiv, neighbour range R = ceil(a/w)
  p->cg.ncell = 1;
  for (int d = 0; d < 3; ++d) {
    int nc = (int)std::floor(kCellDiv * box[d] / a);
    if (nc < 1) nc = 1;
    if (nc > 1024) nc = 1024;
    p->cg.nc[d] = nc;
    p->cg.w[d] = box[d] / nc;
    p->cg.inv_w[d] = nc / box[d];
    p->cg.R[d] = (int)std::ceil(a / p->cg.w[d] * (1.0 - 1e-12));
    p->cg.ncell *= nc;
  }
  // Level-1 stencil taps |m h_1| < 2a (used on levels 1..l-1), in rows of
  // constant (dy, dz) with contiguous dx = -R..R (the cross-section of the
  // cutoff sphere).  Per tap: g_1(r), G = g_1'(r)/r, G dx, G dx^2.
  p->ntaps = p->nrows = p->P = 0;
  if (levels >= 2) {
    const double* h = p->lv[1].h;
    const double c2 = 4.0 * a * a;
    int My = (int)std::ceil(2.0 * a / h[1]) + 1, Mz = (int)std::ceil(2.0 * a / h[2]) + 1;
    for (int dz = -Mz; dz <= Mz; ++dz)
      for (int dy = -My; dy <= My; ++dy) {
        double ryz = (dy * h[1]) * (dy * h[1]) + (dz * h[2]) * (dz * h[2]);
        if (!(ryz < c2)) continue;
        int R = 0;
        while (((R + 1) * h[0]) * ((R + 1) * h[0]) + ryz < c2) ++R;
        p->h_rows.push_back(dy);
        p->h_rows.push_back(dz);
        p->h_rows.push_back(R);
        p->h_rows.push_back(p->ntaps);
        for (int dx = -R; dx <= R; ++dx) {
          double r3[3] = {dx * h[0], dy * h[1], dz * h[2]};
          double r = std::sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
          double G = r > 0.0 ? dg_level_over_r(p->sm, 1, levels, a, r) : 0.0;
          p->h_wv.push_back(g_level(p->sm, 1, levels, a, r));
          p->h_wv.push_back(G);
          p->h_wv.push_back(G * dx);
          p->h_wv.push_back(G * dx * dx);
          p->ntaps++;
        }
        p->nrows++;
        p->P = std::max(p->P, std::max(R, std::max(std::abs(dy), std::abs(dz))));
      }
  }
  // coarsest-level periodic tables
  const Level& top = p->lv[levels];
  p->h_top_T.assign((size_t)top.np, 0.0);
  p->h_top_V.assign((size_t)top.np * 6, 0.0);
  coarse_tables_impl(p->sm, box, top.n, levels, a, p->h_top_T.data(), p->h_top_V.data());

  rc = upload_tables(p);
  if (rc) {
    free_plan(p);
    return rc;
  }
  *out = reinterpret_cast<mls6_plan_t*>(p);
  return MLS6_OK;
}

int mls6_set_stream(mls6_plan_t* plan, void* stream) {
  if (!plan) return MLS6_ERR_ARG;
  reinterpret_cast<Plan*>(plan)->stream = (cudaStream_t)stream;
  return MLS6_OK;
}

int mls6_eval(mls6_plan_t* plan, const void* pos, const void* c, void* forces, double* energy,
              double* virial) {
  if (!plan) return MLS6_ERR_ARG;
  return eval_launch(reinterpret_cast<Plan*>(plan), pos, c, forces, energy, virial, nullptr);
}

int mls6_eval_atoms(mls6_plan_t* plan, const void* pos, const void* c, void* forces,
                    double* energy, double* virial, double* atom_energy) {
  if (!plan) return MLS6_ERR_ARG;
  if (!atom_energy && reinterpret_cast<Plan*>(plan)->N > 0) return MLS6_ERR_ARG;
  return eval_launch(reinterpret_cast<Plan*>(plan), pos, c, forces, energy, virial, atom_energy);
}

int mls6_last_error(mls6_plan_t* plan) {
  if (!plan) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MLS6_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpy(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MLS6_ERR_CUDA;
  return flag_status(flag);
}

int mls6_plan_info(const mls6_plan_t* plan, int* n_grid, double* h_actual, int* levels,
                   int* ntaps) {
  if (!plan) return MLS6_ERR_ARG;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (n_grid)
    for (int k = 1; k <= p->levels; ++k)
      for (int d = 0; d < 3; ++d) n_grid[3 * (k - 1) + d] = p->lv[k].n[d];
  if (h_actual)
    for (int d = 0; d < 3; ++d) h_actual[d] = p->lv[1].h[d];
  if (levels) *levels = p->levels;
  if (ntaps) *ntaps = p->ntaps;
  return MLS6_OK;
}

int mls6_set_tuning(mls6_plan_t* plan, int split, int groups) {
  if (!plan) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (split != 0 && split != 1 && split != 2 && split != 4 && split != 8 && split != 16 &&
      split != 32 && split != 128 && split != 256 && split != 512 && split != kPairCluster)
    return MLS6_ERR_ARG;
  if (split == kPairCluster ? !pair_cl_ok(p) : (split > 8 && !pair_cluster_ok(p)))
    return MLS6_ERR_ARG;
  if (groups != 0 && groups != 1 && groups != 2 && groups != 4) return MLS6_ERR_ARG;
  const int s2 = split ? split : p->pair_split;
  const int g2 = (groups && !p->stencil_global) ? groups : p->stencil_groups;
  if (s2 == p->pair_split && g2 == p->stencil_groups) return MLS6_OK;
  if (p->cs && cudaStreamSynchronize(p->cs) != cudaSuccess) return MLS6_ERR_CUDA;
  if (p->cs2 && cudaStreamSynchronize(p->cs2) != cudaSuccess) return MLS6_ERR_CUDA;
  p->pair_split = s2;
  p->stencil_groups = g2;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return MLS6_OK;
}

int mls6_eval_lb(mls6_plan_t* plan, const void* pos, const void* sigma, const void* epsilon,
                 void* forces, double* energy) {
  if (!plan) return MLS6_ERR_ARG;
  return eval_lb(reinterpret_cast<Plan*>(plan), pos, sigma, epsilon, forces, energy);
}

int mls6_stencil_kind(const mls6_plan_t* plan) {
  if (!plan) return MLS6_ERR_ARG;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (p->levels < 2) return -1;
  return p->stencil_mma ? 3 : p->stencil_tc ? 2 : (p->stencil_global ? 1 : 0);
}

int mls6_get_tuning(const mls6_plan_t* plan, int* split, int* groups) {
  if (!plan) return MLS6_ERR_ARG;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (split) *split = p->pair_split;
  if (groups) *groups = p->stencil_groups;
  return MLS6_OK;
}

void mls6_destroy(mls6_plan_t* plan) { free_plan(reinterpret_cast<Plan*>(plan)); }

const char* mls6_status_string(int s) {
  switch (s) {
    case MLS6_OK: return "ok";
    case MLS6_ERR_ARG: return "invalid argument";
    case MLS6_ERR_GRID: return "invalid grid hierarchy";
    case MLS6_ERR_BOX: return "invalid box";
    case MLS6_ERR_ORDER: return "unsupported interpolation order (3 or 5)";
    case MLS6_ERR_CUDA: return "CUDA runtime error";
    case MLS6_ERR_NOMEM: return "device allocation failed";
    case MLS6_ERR_TIMEOUT: return "a bounded device-side wait ran out (the kernel gave up)";
    case MLS6_ERR_NONFINITE: return "non-finite position or coefficient";
    case MLS6_ERR_SIZE: return "size exceeds a fixed capacity";
    default: return "unknown status";
  }
}

}  // extern "C"
