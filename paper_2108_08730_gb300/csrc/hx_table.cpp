// Weight-table fit of the adaptive stencil (Section 2.2), host FP64.
//
// Unknowns, node-major as in the paper: w = [w^(0); w^(1); ...], each
// w^(i) = [ws1, ws2, wm1, wm2, wm3] at 1/G_i = i * d_inv_g.  Rows:
//   data rows   H^(i) w^(i) = g^(i)              (one per plane-wave direction)
//   smooth rows sqrt(lambda) (w_l^(i+1) - w_l^(i)) = 0   for l = 0..4
// Ordered node by node, every row touches only the 10 columns of nodes i and
// i+1, so the triangular factor R of a Givens QR stays inside a band of width
// 10.  Rows are rotated into R one at a time (numerically orthogonal, no
// normal equations), then R w = Q^T b is back-substituted.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hx_internal.h"

namespace hx {

namespace {

constexpr int kW = 10;  // band width of R: columns j .. j+9

struct BandQR {
  int n;
  std::vector<double> R;     // n x kW, R[j*kW + k] = R(j, j+k)
  std::vector<double> qtb;   // n
  std::vector<char> filled;  // R row j has been set

  explicit BandQR(int n_) : n(n_), R((size_t)n_ * kW, 0.0), qtb(n_, 0.0), filled(n_, 0) {}

  // Rotate the row (values on columns c0 .. c0+kW-1, rhs b) into R.
  void add_row(int c0, const double* vals, double b) {
    double row[2 * kW];
    std::memset(row, 0, sizeof(row));
    for (int k = 0; k < kW; ++k) row[k] = vals[k];
    for (int j = c0; j < c0 + kW && j < n; ++j) {
      const int o = j - c0;  // position of column j in `row`
      double x = row[o];
      if (x == 0.0) continue;
      double* Rj = &R[(size_t)j * kW];
      if (!filled[j]) {
        for (int k = 0; k < kW && o + k < 2 * kW; ++k) Rj[k] = row[o + k];
        qtb[j] = b;
        filled[j] = 1;
        return;
      }
      const double r = Rj[0];
      const double rho = std::hypot(r, x);
      const double c = r / rho, s = x / rho;
      for (int k = 0; k < kW && o + k < 2 * kW; ++k) {
        const double rk = Rj[k], xk = row[o + k];
        Rj[k] = c * rk + s * xk;
        row[o + k] = -s * rk + c * xk;
      }
      const double t = qtb[j];
      qtb[j] = c * t + s * b;
      b = -s * t + c * b;
    }
  }

  bool solve(std::vector<double>& w) const {
    w.assign(n, 0.0);
    for (int j = n - 1; j >= 0; --j) {
      const double* Rj = &R[(size_t)j * kW];
      if (!filled[j] || Rj[0] == 0.0 || !std::isfinite(Rj[0])) return false;
      double acc = qtb[j];
      for (int k = 1; k < kW && j + k < n; ++k) acc -= Rj[k] * w[j + k];
      w[j] = acc / Rj[0];
    }
    return true;
  }
};

// One data row of Eq. linear_basic at 1/G = inv_g for the unit direction
// (cos(phi)cos(theta), cos(phi)sin(theta), sin(phi)).
void linear_row(double inv_g, double theta, double phi, double H[5], double* g) {
  const double two_pi = 2.0 * M_PI;
  const double ca = std::cos(two_pi * std::cos(phi) * std::cos(theta) * inv_g);
  const double cb = std::cos(two_pi * std::cos(phi) * std::sin(theta) * inv_g);
  const double cc = std::cos(two_pi * std::sin(phi) * inv_g);
  const double A = ca * cb * cc;
  const double B = ca * cb + ca * cc + cb * cc;
  const double C = ca + cb + cc;
  const double K = 2.0 * M_PI * M_PI * inv_g * inv_g;
  H[0] = 0.5 * (3.0 + 3.0 * A - B - C);
  H[1] = 0.5 * (1.0 + 3.0 * A - (5.0 / 3.0) * B + (1.0 / 3.0) * C);
  H[2] = K * (A - 1.0);
  H[3] = K * (6.0 * A - 2.0 * C);
  H[4] = K * (12.0 * A - 4.0 * B);
  *g = 0.5 * ((2.0 * K + 3.0) * A - B + C - 3.0);
}

}  // namespace

int build_weight_table(const double* theta_deg, int n_theta, const double* phi_deg, int n_phi,
                       double inv_g_max, double d_inv_g, double lambda, double* out, int capacity,
                       int* n_g_out, std::string* err) {
  if (!theta_deg || !phi_deg || n_theta < 1 || n_phi < 1) {
    *err = "angle lists must be non-empty";
    return HX_ERR_ARG;
  }
  if (!(d_inv_g > 0.0) || !(inv_g_max > d_inv_g) || !(lambda > 0.0) || !std::isfinite(lambda)) {
    *err = "need 0 < d_inv_g < inv_g_max and lambda > 0";
    return HX_ERR_ARG;
  }
  const int n_g = (int)std::lround(inv_g_max / d_inv_g) + 1;
  if (n_g_out) *n_g_out = n_g;
  if (n_g > 1000000) {
    *err = "table too large";
    return HX_ERR_ARG;
  }
  if (!out || capacity < 7 * n_g) {
    *err = "table_out capacity must be >= 7 * n_g";
    return HX_ERR_ARG;
  }
  const int n = 5 * n_g;
  BandQR qr(n);
  const double sl = std::sqrt(lambda);
  double vals[kW];
  for (int i = 0; i < n_g; ++i) {
    const double inv_g = i * d_inv_g;
    for (int p = 0; p < n_phi; ++p) {
      for (int t = 0; t < n_theta; ++t) {
        double H[5], g;
        linear_row(inv_g, theta_deg[t] * M_PI / 180.0, phi_deg[p] * M_PI / 180.0, H, &g);
        for (int k = 0; k < kW; ++k) vals[k] = k < 5 ? H[k] : 0.0;
        qr.add_row(5 * i, vals, g);
      }
    }
    if (i + 1 < n_g) {
      for (int l = 0; l < 5; ++l) {
        for (int k = 0; k < kW; ++k) vals[k] = 0.0;
        vals[l] = -sl;
        vals[5 + l] = sl;
        qr.add_row(5 * i, vals, 0.0);
      }
    }
  }
  std::vector<double> w;
  if (!qr.solve(w)) {
    *err = "weight fit is rank deficient";
    return HX_ERR_NUMERIC;
  }
  for (int i = 0; i < n_g; ++i) {
    const double ws1 = w[5 * i], ws2 = w[5 * i + 1];
    const double wm1 = w[5 * i + 2], wm2 = w[5 * i + 3], wm3 = w[5 * i + 4];
    double* o = out + 7 * (size_t)i;
    o[0] = ws1;
    o[1] = ws2;
    o[2] = 1.0 - ws1 - ws2;                                  // Eq. eqsws
    o[3] = wm1;
    o[4] = wm2;
    o[5] = wm3;
    o[6] = (1.0 - wm1 - 6.0 * wm2 - 12.0 * wm3) / 8.0;       // Eq. eqswm, per point
  }
  return HX_OK;
}

// Non-adaptive weights (Eq. eq_cost): one weight vector for the plane waves
// of every listed 1/G at once -- the G4 stencil for {1/4}, Gm for
// {1/4, 1/6, 1/8, 1/10}.  Minimum-norm least squares through the normal
// matrix N = H^T H (5 x 5): cyclic Jacobi eigen-decomposition, then
// w = V diag(1/d_k, d_k > 1e-12 max d) V^T H^T g.  A single G gives a rank-3
// H (all five H_l vanish on a plane through (A, B, C) = (1, 3, 3)), so the
// minimum-norm choice matters there.
int fit_joint_weights(const double* inv_g, int n, const double* theta_deg, int n_theta, const double* phi_deg,
                      int n_phi, double* w7, std::string* err) {
  if (!inv_g || n < 1 || !theta_deg || !phi_deg || n_theta < 1 || n_phi < 1 || !w7) {
    *err = "need 1/G values, angle lists and an output";
    return HX_ERR_ARG;
  }
  double N[5][5] = {}, hg[5] = {};
  for (int q = 0; q < n; ++q) {
    if (!(inv_g[q] > 0.0) || !(inv_g[q] <= 0.5)) {
      *err = "1/G values must lie in (0, 0.5]";
      return HX_ERR_ARG;
    }
    for (int p = 0; p < n_phi; ++p)
      for (int t = 0; t < n_theta; ++t) {
        double H[5], g;
        linear_row(inv_g[q], theta_deg[t] * M_PI / 180.0, phi_deg[p] * M_PI / 180.0, H, &g);
        for (int a = 0; a < 5; ++a) {
          hg[a] += H[a] * g;
          for (int b = 0; b < 5; ++b) N[a][b] += H[a] * H[b];
        }
      }
  }
  // cyclic Jacobi: N = V diag(d) V^T
  double V[5][5] = {};
  for (int a = 0; a < 5; ++a) V[a][a] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) {
        tot += N[a][b] * N[a][b];
        if (a != b) off += N[a][b] * N[a][b];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 5; ++q) {
        if (N[p][q] == 0.0) continue;
        const double theta = (N[q][q] - N[p][p]) / (2.0 * N[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 5; ++k) {      // N <- N J
          const double nkp = N[k][p], nkq = N[k][q];
          N[k][p] = c * nkp - s * nkq;
          N[k][q] = s * nkp + c * nkq;
        }
        for (int k = 0; k < 5; ++k) {      // N <- J^T N
          const double npk = N[p][k], nqk = N[q][k];
          N[p][k] = c * npk - s * nqk;
          N[q][k] = s * npk + c * nqk;
        }
        for (int k = 0; k < 5; ++k) {      // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  double dmax = 0.0;
  for (int a = 0; a < 5; ++a) dmax = std::max(dmax, N[a][a]);
  if (!(dmax > 0.0) || !std::isfinite(dmax)) {
    *err = "degenerate joint fit";
    return HX_ERR_NUMERIC;
  }
  double w[5] = {};
  for (int k = 0; k < 5; ++k) {
    if (!(N[k][k] > 1e-12 * dmax)) continue;
    double proj = 0.0;
    for (int a = 0; a < 5; ++a) proj += V[a][k] * hg[a];
    for (int a = 0; a < 5; ++a) w[a] += V[a][k] * proj / N[k][k];
  }
  w7[0] = w[0];
  w7[1] = w[1];
  w7[2] = 1.0 - w[0] - w[1];
  w7[3] = w[2];
  w7[4] = w[3];
  w7[5] = w[4];
  w7[6] = (1.0 - w[2] - 6.0 * w[3] - 12.0 * w[4]) / 8.0;
  return HX_OK;
}

}  // namespace hx
