// Orientation averaging (arXiv:0704.0037, Sec. 2, paragraph on orientation
// averaging): Euler angles (alpha, beta, gamma), z-y-z, R = Rz(alpha) Ry(beta)
// Rz(gamma) takes the particle frame to the laboratory; the incident wave runs
// along laboratory z.  Each (beta, gamma) node needs its own pair of solutions
// (incidence R^T z, polarisations R^T x and R^T y: two right-hand sides of one
// dda_solve); alpha only turns the scattering plane about the incidence axis,
// so it is averaged with the same solutions by evaluating the far field in
// n_alpha planes and combining the two polarisations (which needs a
// polarizability independent of the incident polarisation: CM, RR, CLDR).
// Fixed quadrature, no Romberg adaptivity: Gauss-Legendre in cos(beta),
// uniform nodes in gamma and alpha.
#include <cmath>
#include <vector>

#include "internal.h"

using namespace dda;

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Mat3 { double a[3][3]; };

Mat3 mul(const Mat3& p, const Mat3& q) {
  Mat3 r{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) r.a[i][j] += p.a[i][k] * q.a[k][j];
  return r;
}

Mat3 rz(double t) {
  const double c = std::cos(t), s = std::sin(t);
  return Mat3{{{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}}};
}

Mat3 ry(double t) {
  const double c = std::cos(t), s = std::sin(t);
  return Mat3{{{c, 0.0, s}, {0.0, 1.0, 0.0}, {-s, 0.0, c}}};
}

}  // namespace

extern "C" int dda_orientation_average(dda_t h, const dda_solve_opts* o, int n_alpha, int n_beta,
                                       int n_gamma, int n_theta, const double* theta_deg,
                                       double* q_avg, double* M_avg, dda_solve_info* info) {
  DDA_ON_DEVICE(h);
  if (!o || n_alpha < 1 || n_beta < 1 || n_gamma < 1 || n_theta < 1 || !theta_deg || !q_avg ||
      !M_avg)
    return dda_fail(h, DDA_ERR_ARG, "bad dda_orientation_average arguments");
  if (o->pol == DDA_LDR)
    return dda_fail(h, DDA_ERR_ARG, "orientation averaging needs a polarisation-independent "
                                    "polarizability (CM, RR or CLDR); LDR depends on it");
  if (o->pol < DDA_CM || o->pol > DDA_CLDR) return dda_fail(h, DDA_ERR_ARG, "unknown prescription");
  if (o->checkpoint_every != 0 || o->resume)
    return dda_fail(h, DDA_ERR_ARG, "orientation averaging takes no checkpoints");
  if (o->solver < DDA_QMR_CS || o->solver > DDA_CGNR || !(o->tol > 0.0) || o->maxiter < 1 ||
      (o->prec != DDA_FP64 && o->prec != DDA_FP32_REFINED) ||
      (o->prec == DDA_FP32_REFINED && !(o->inner_tol > 0.0 && o->inner_tol < 1.0)))
    return dda_fail(h, DDA_ERR_ARG, "bad solver options");
  if (!h->w64.have_D || (o->prec == DDA_FP32_REFINED && !h->w32.have_D))
    return dda_fail(h, DDA_ERR_STATE, "D-matrix not built");
  const long long n = 3 * h->g.n_occ;
  void* P = nullptr;
  if (dev_malloc(&P, 2 * (size_t)n * sizeof(c128)) != cudaSuccess) {
    cudaGetLastError();
    return dda_fail(h, DDA_ERR_OOM, "orientation-averaging polarisations");
  }
  std::vector<double> mu, wmu;
  gauss_legendre(n_beta, mu, wmu);
  const int n_dir = n_theta * n_alpha;
  std::vector<double> dirs((size_t)3 * n_dir), F((size_t)2 * n_dir * 6);
  std::vector<double> Msum((size_t)16 * n_theta, 0.0);
  double qe = 0.0, qa = 0.0;
  int rc = DDA_OK, worst = DDA_OK;
  for (int ib = 0; ib < n_beta && rc >= 0; ++ib) {
    for (int ig = 0; ig < n_gamma && rc >= 0; ++ig) {
      const double wk = wmu[ib] / 2.0 / n_gamma;
      const Mat3 R = mul(ry(std::acos(mu[ib])), rz(2.0 * M_PI * ig / n_gamma));
      // incidence R^T z, polarisations R^T x, R^T y (columns of R as rows)
      double prop[6], pol[12] = {0};
      for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 3; ++q) {
          prop[3 * r + q] = R.a[2][q];
          pol[6 * r + 2 * q] = R.a[r][q];
        }
      dda_solve_info inf[2];
      rc = dda_solve_internal(h, o, 2, prop, pol, P, nullptr, 0, inf);
      if (rc < 0) break;
      for (int r = 0; r < 2; ++r) {
        if (info) info[2 * (ib * n_gamma + ig) + r] = inf[r];
        if (inf[r].status != DDA_OK && worst == DDA_OK) worst = inf[r].status;
      }
      // scattering directions n(theta, phi) in the particle frame: R^T n
      for (int ia = 0; ia < n_alpha; ++ia) {
        const double ph = 2.0 * M_PI * ia / n_alpha;
        for (int it = 0; it < n_theta; ++it) {
          const double t = theta_deg[it] * (M_PI / 180.0);
          const double nl[3] = {std::sin(t) * std::cos(ph), std::sin(t) * std::sin(ph), std::cos(t)};
          double* d = dirs.data() + 3 * ((size_t)ia * n_theta + it);
          for (int q = 0; q < 3; ++q) d[q] = R.a[0][q] * nl[0] + R.a[1][q] * nl[1] + R.a[2][q] * nl[2];
        }
      }
      double q[6];
      rc = dda_scatter_internal(h, o->pol, P, 2, prop, pol, n_dir, dirs.data(), nullptr, F.data(), q);
      if (rc < 0) break;
      qe += wk * 0.5 * (q[0] + q[3]);
      qa += wk * 0.5 * (q[1] + q[4]);
      for (int ia = 0; ia < n_alpha; ++ia) {
        const double ph = 2.0 * M_PI * ia / n_alpha;
        const double cp = std::cos(ph), sp = std::sin(ph);
        for (int it = 0; it < n_theta; ++it) {
          const size_t k = (size_t)ia * n_theta + it;
          // laboratory amplitudes R F of the two solutions
          c128 FX[3], FY[3];
          for (int i = 0; i < 3; ++i) {
            FX[i] = mk<double>(0.0, 0.0);
            FY[i] = mk<double>(0.0, 0.0);
            for (int j = 0; j < 3; ++j) {
              FX[i] = FX[i] + scale<double>(mk<double>(F[6 * k + 2 * j], F[6 * k + 2 * j + 1]), R.a[i][j]);
              const size_t k2 = (size_t)n_dir + k;
              FY[i] = FY[i] + scale<double>(mk<double>(F[6 * k2 + 2 * j], F[6 * k2 + 2 * j + 1]), R.a[i][j]);
            }
          }
          const double t = theta_deg[it] * (M_PI / 180.0);
          const double th[3] = {std::cos(t) * cp, std::cos(t) * sp, -std::sin(t)};
          const double phh[3] = {-sp, cp, 0.0};
          c128 tp = mk<double>(0, 0), pp = mk<double>(0, 0), tq = mk<double>(0, 0), pq = mk<double>(0, 0);
          for (int i = 0; i < 3; ++i) {
            const c128 par = scale<double>(FX[i], cp) + scale<double>(FY[i], sp);
            const c128 per = scale<double>(FY[i], cp) - scale<double>(FX[i], sp);
            tp = tp + scale<double>(par, th[i]);
            pp = pp + scale<double>(par, phh[i]);
            tq = tq + scale<double>(per, th[i]);
            pq = pq + scale<double>(per, phh[i]);
          }
          // S1 = phi.F_perp, S2 = theta.F_par, S3 = -theta.F_perp, S4 = -phi.F_par
          const c128 S[4] = {pq, tp, scale<double>(tq, -1.0), scale<double>(pp, -1.0)};
          double m[16];
          mueller_from_S(S, m);
          for (int e = 0; e < 16; ++e) Msum[(size_t)16 * it + e] += wk * m[e] / n_alpha;
        }
      }
    }
  }
  dev_free(P, h->stream);
  if (rc < 0) return rc;
  q_avg[0] = qe;
  q_avg[1] = qa;
  for (size_t i = 0; i < Msum.size(); ++i) M_avg[i] = Msum[i];
  return worst;
}
